"""GPU parity of block FGMRES (krylov = HZ_KRYLOV_BLOCK) against the oracle's
block_fgmres, through the C ABI.

The context solves its right-hand sides in batches of block_size (rounded up to 4, 8
or 16), each batch in one block Krylov space; the oracle runs the same batches.  Both
follow the same steps (block CGS2, column-wise orthonormalisation of each new block,
the same Givens order), so in FP64 the block step counts agree within one and the
solutions to 1e-9, as for the single-vector solve.  In the mixed path the step counts
agree within one and every column meets the tolerance with the oracle's FP64 operator."""
import numpy as np
import pytest

import synth
from oracle import krylov
from oracle.solver import OracleSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


@pytest.fixture(scope="module")
def case():
    p = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    S = OracleSolver(p)
    S.factor()
    ext = p.mesh.xyz.max(axis=0)
    pts = np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.5, 0.5, 0.2], [0.3, 0.8, 0.6],
                    [0.8, 0.7, 0.4], [0.45, 0.55, 0.75]]) * ext
    return p, S, S.rhs(pts)


def _oracle_batches(S, B, width, tol, m):
    X = np.zeros_like(B)
    its = np.zeros(B.shape[1], int)
    for k0 in range(0, B.shape[1], width):
        Xb, it, rel, ok = krylov.block_fgmres(S.apply_A, S.apply_M, B[:, k0:k0 + width], tol=tol, m=m)
        assert ok
        X[:, k0:k0 + width] = Xb
        its[k0:k0 + width] = it
    return X, its


@pytest.mark.parametrize("precision,block,width", [(0, 4, 4), (0, 8, 8), (1, 4, 4), (1, 16, 16)])
def test_block_fgmres_matches_oracle(hzmod, case, precision, block, width):
    p, S, B = case
    Xo, ito = _oracle_batches(S, B, width, p.tol, p.restart)
    G = hzmod.Solver(p, precision=precision, block_size=block, krylov=hzmod.HZ_KRYLOV_BLOCK)
    try:
        G.factor()
        X, info = G.solve(B)
    finally:
        G.close()
    for j in range(B.shape[1]):
        itg, st, rel = info[j]
        assert st == 0 and rel <= p.tol, info[j]
        assert abs(itg - ito[j]) <= 1, (j, itg, ito[j])
        assert np.linalg.norm(B[:, j] - S.A @ X[:, j]) / np.linalg.norm(B[:, j]) <= p.tol
        if precision == 0:
            assert np.linalg.norm(X[:, j] - Xo[:, j]) <= 1e-9 * np.linalg.norm(Xo[:, j])
    print(f"block FGMRES precision={precision} block={block}: steps gpu {[i[0] for i in info]} oracle {list(ito)}")


def test_block_fgmres_small_restart_and_zero_column(hzmod, case):
    """Restarted every 3 block steps, with a zero right-hand side inside the batch: the zero
    column gets x = 0 and no iteration, the others restart until they meet the tolerance."""
    p, S, B = case
    B = B[:, :4].copy()
    B[:, 2] = 0.0
    q = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16, restart=3)
    G = hzmod.Solver(q, block_size=4, krylov=hzmod.HZ_KRYLOV_BLOCK)
    try:
        G.factor()
        X, info = G.solve(B)
    finally:
        G.close()
    assert np.all(X[:, 2] == 0) and info[2][0] == 0 and info[2][1] == 0
    Xo, ito, relo, ok = krylov.block_fgmres(S.apply_A, S.apply_M, B[:, [0, 1, 3]], tol=p.tol, m=3)
    assert ok and ito > 3
    for k, j in enumerate((0, 1, 3)):
        assert info[j][1] == 0 and abs(info[j][0] - ito) <= 1
        assert np.linalg.norm(X[:, j] - Xo[:, k]) <= 1e-9 * np.linalg.norm(Xo[:, k])


def test_block_option_needs_a_block(hzmod, case):
    p, S, B = case
    with pytest.raises(hzmod.HzError):
        hzmod.Solver(p, block_size=1, krylov=hzmod.HZ_KRYLOV_BLOCK)
