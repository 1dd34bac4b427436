"""GPU parity of block GCRO-DR (krylov = HZ_KRYLOV_BLOCK with recycle = k) against the
oracle's block_gcrodr, through the C ABI.

The context solves its right-hand sides in batches of block_size; each batch is one block
Krylov space whose cycles are orthogonal to the recycled space C, and the space left by a
batch is used by the next one.  The oracle runs the same batches in the same order.  The
recycled space is chosen from block harmonic Ritz vectors (the library's host eigen-solver,
LAPACK through scipy in the oracle); the two bases of the space differ by rounding, but
the spans agree, so the block step counts are compared to +-1 and, in FP64, the solutions
to 1e-9 (the FP64 path's tolerance); every solution is checked against the tolerance with
the oracle's FP64 operator."""
import numpy as np
import pytest

import synth
from oracle import krylov
from oracle.solver import OracleSolver

pytestmark = pytest.mark.gpu

TOL = 1e-8
PTS = np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.5, 0.5, 0.2], [0.3, 0.8, 0.6], [0.8, 0.7, 0.4],
                [0.45, 0.55, 0.75], [0.15, 0.65, 0.35], [0.6, 0.35, 0.65], [0.35, 0.4, 0.5]])


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def _problem(name, restart):
    p = synth.tiny_problem() if name == "tiny" else synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6,
                                                                            nsub=16)
    p.restart = restart
    return p


_ORACLES = {}


def _oracle(name):
    """The oracle's factorisation and the nine point sources of one configuration."""
    if name not in _ORACLES:
        p = _problem(name, 5)
        S = OracleSolver(p)
        S.factor()
        _ORACLES[name] = (S, S.rhs(PTS * p.mesh.xyz.max(axis=0)))
    return _ORACLES[name]


# (configuration, restart, k): on the tiny mesh GCRO-DR(8, 4) takes seven block steps per
# cycle and 15-18 steps per batch (the lone source: four per cycle), so the space is renewed
# by the later-cycle (G-based) update several times; on the two-level Overthrust-shaped case
# the first batch takes eight steps in one cycle (the first-cycle update) and the next ones
# run against the recycled space.
CASES = [("tiny", 8, 4), ("ovt", 8, 4)]


@pytest.mark.parametrize("name,restart,k", CASES)
def test_block_gcrodr_batches_match_oracle(hzmod, name, restart, k):
    """Two batches of four sources, then one source alone (a batch of one), sharing the
    recycled space: block steps +-1 and solutions to 1e-9 against the oracle."""
    S, B = _oracle(name)
    G = hzmod.Solver(_problem(name, restart), block_size=4, krylov=hzmod.HZ_KRYLOV_BLOCK, recycle=k)
    try:
        G.factor()
        assert G.stats()["recycle_dim"] == 0
        rec = None
        for cols in ([0, 1, 2, 3], [4, 5, 6, 7], [8]):
            Xo, ito, relo, ok, rec = krylov.block_gcrodr(S.apply_A, S.apply_M, B[:, cols], tol=TOL, m=restart,
                                                         k=k, recycle=rec)
            assert ok
            if name == "tiny":
                assert ito > restart - (k + len(cols) - 1) // len(cols)        # more than one cycle
            X, info = G.solve(B[:, cols], tol=TOL)
            for q, j in enumerate(cols):
                itg, st, rel = info[q]
                assert st == 0 and rel <= TOL, info[q]
                assert abs(itg - ito) <= 1, (j, itg, ito)
                err = np.linalg.norm(X[:, q] - Xo[:, q]) / np.linalg.norm(Xo[:, q])
                assert err <= 1e-9, (j, err)
                assert np.linalg.norm(B[:, j] - S.A @ X[:, q]) / np.linalg.norm(B[:, j]) <= TOL
            assert G.stats()["recycle_dim"] == rec[0].shape[1] == k
            print(f"block GCRO-DR({restart}, {k}) {name} sources {cols}: steps gpu {[i[0] for i in info]} "
                  f"oracle {ito}")
    finally:
        G.close()


def test_block_gcrodr_mixed_precision(hzmod):
    """Tiny mesh, GCRO-DR(16, 8), four columns per block, complex64 local solves: two batches
    within one block step of the oracle's FP64 run, every column meeting the tolerance with
    the FP64 operator.  Recycling saves little here (the oracle: 13 block steps for the second
    batch against 14 for block FGMRES(16)); the counts are printed beside block FGMRES."""
    S, B = _oracle("tiny")
    p = _problem("tiny", 16)
    G = hzmod.Solver(p, precision=hzmod.HZ_MIXED, block_size=4, krylov=hzmod.HZ_KRYLOV_BLOCK, recycle=8)
    F = hzmod.Solver(p, precision=hzmod.HZ_MIXED, block_size=4, krylov=hzmod.HZ_KRYLOV_BLOCK)
    try:
        G.factor()
        F.factor()
        rec = None
        for cols in ([0, 1, 2, 3], [4, 5, 6, 7]):
            _, ito, _, ok, rec = krylov.block_gcrodr(S.apply_A, S.apply_M, B[:, cols], tol=TOL, m=16, k=8,
                                                     recycle=rec)
            X, info = G.solve(B[:, cols], tol=TOL)
            _, info_f = F.solve(B[:, cols], tol=TOL)
            assert ok
            for q, j in enumerate(cols):
                assert info[q][1] == 0 and abs(info[q][0] - ito) <= 1, (j, info[q], ito)
                assert np.linalg.norm(B[:, j] - S.A @ X[:, q]) / np.linalg.norm(B[:, j]) <= TOL
            print(f"mixed sources {cols}: block GCRO-DR {info[0][0]} steps (oracle {ito}), "
                  f"block FGMRES {info_f[0][0]}")
    finally:
        G.close()
        F.close()


def test_block_gcrodr_space_carried_to_a_new_frequency(hzmod):
    """recycle_keep with the block form: the space from a batch at f is re-based at 1.03 f
    (C = A_new Ux orthonormalised) before the next batch, as the oracle's rebase_recycle
    does, and that batch follows the oracle (steps +-1, solutions to 1e-9)."""
    S, B = _oracle("tiny")
    p = _problem("tiny", 16)
    G = hzmod.Solver(p, block_size=4, krylov=hzmod.HZ_KRYLOV_BLOCK, recycle=8, recycle_keep=1)
    try:
        G.factor()
        _, _, _, ok, rec = krylov.block_gcrodr(S.apply_A, S.apply_M, B[:, :4], tol=TOL, m=16, k=8)
        G.solve(B[:, :4], tol=TOL)
        f2 = p.freq * 1.03
        G.factor(f2)
        assert G.stats()["recycle_dim"] == 8
        S2 = OracleSolver(p)
        S2.factor(f2)
        B2 = S2.rhs(PTS * p.mesh.xyz.max(axis=0))[:, 4:8]
        Xo, ito, _, ok2, _ = krylov.block_gcrodr(S2.apply_A, S2.apply_M, B2, tol=TOL, m=16, k=8,
                                                 recycle=krylov.rebase_recycle(S2.apply_A, rec))
        X, info = G.solve(B2, tol=TOL)
    finally:
        G.close()
    assert ok and ok2
    for q in range(4):
        assert info[q][1] == 0 and abs(info[q][0] - ito) <= 1, (info[q], ito)
        assert np.linalg.norm(X[:, q] - Xo[:, q]) <= 1e-9 * np.linalg.norm(Xo[:, q])


def test_block_recycling_needs_the_block_solver(hzmod):
    p = _problem("tiny", 8)
    with pytest.raises(hzmod.HzError):
        hzmod.Solver(p, recycle=2, block_size=4)               # pseudo-block: one space per source
    G = hzmod.Solver(p, recycle=2, block_size=4, krylov=hzmod.HZ_KRYLOV_BLOCK)
    G.close()
