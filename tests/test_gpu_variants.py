"""Element-wise parity of the preconditioner on every kernel variant the full-size solve
runs, in both precisions, through the C ABI.

Case: the Overthrust-shaped generator at 1.25 Hz -- coarse (16, 16, 3) cells, 54,925 P2
dofs, 7 subdomains of 11-14k dofs, overlap 2, two levels.  Its subdomains are large
enough that the triangular sweeps and the complex64 factorisation take the same kernel
variants as the 2.37M-dof workload: 128-wide supernodes (112 in FP64), supernodes taller
than one backward row chunk (partial sums added up by the CTA that finishes last),
fronts whose Schur update spans several 128 x 128 tensor-core tiles and several K
stages.  ``sweep_tasks`` forces the wide task shapes (256-row forward tasks, 512-row
backward chunks in complex64) or the narrow ones on every tree level, so each variant
is compared with the oracle element by element; ``hz_get_stats`` reports which ran.

Tolerances.
- FP64: M^{-1} v to 1e-10 relative L2 (two direct solvers, different rounding).
- Mixed: the local solves A_i^{-1} t_i run in complex64 (unit roundoff u = 2^-24) and
  the rest in FP64, so M^{-1} v carries the forward error of backward-stable complex64
  solves, at most about kappa_1(A_i) * u per subdomain.  The bound used is
  max_i kappa_1(A_i) * u with kappa_1 estimated from the oracle's own factors
  (scipy's one-norm estimator on the SuperLU solves); about 2.9e-4 here.
- Full solves: FP64 as in test_gpu_parity; mixed at tol 1e-6 within one iteration
  of the oracle, and, solved to tol 1e-9, within 1e-6 relative L2 of the oracle's
  solution (the mixed path's stated tolerance)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.solver import OracleSolver

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


@pytest.fixture(scope="module")
def case():
    p = synth.overthrust_problem(seed=0, freq=1.25, nsub=7, overlap=2, restart=50, levels=2)
    S = OracleSolver(p)
    S.factor()
    kappa = 0.0
    for sub, lu in zip(S.subs, S.lu):
        A = sub.A.tocsc()
        n = A.shape[0]
        inv = spla.LinearOperator(
            (n, n), dtype=np.complex128,
            matvec=lambda v, lu=lu: lu.solve(np.asarray(v, np.complex128)),
            rmatvec=lambda v, lu=lu: lu.solve(np.asarray(v, np.complex128), trans="H"))
        kappa = max(kappa, spla.norm(A, 1) * spla.onenormest(inv))
    rng = np.random.default_rng(21)
    v = rng.standard_normal(S.n) + 1j * rng.standard_normal(S.n)
    return p, S, kappa, v, S.apply_M(v)


# (precision, sweep_tasks, bwd_chunk): default schedule, wide tasks on every level,
# wide with a shorter chunk (more split column blocks), narrow tasks on every level
SCHEDULES = [("fp64", 0, 0), ("fp64", 1, 0), ("fp64", 2, 0), ("fp64", 1, 96),
             ("mixed", 0, 0), ("mixed", 1, 0), ("mixed", 2, 0), ("mixed", 1, 192)]


VARIANT_KEYS = ["fwd_levels_wide", "fwd_levels_narrow", "bwd_levels_wide", "bwd_levels_narrow", "bwd_split_blocks",
                "tc_tiles", "tc_multi_fronts", "tc_max_kstages", "max_snode_width"]


def _solver(hz, p, prec, sweep, chunk):
    return hz.Solver(p, precision=hz.HZ_MIXED if prec == "mixed" else hz.HZ_FP64, sweep_tasks=sweep,
                     bwd_chunk=chunk)


@pytest.mark.parametrize("prec,sweep,chunk", SCHEDULES)
def test_apply_M_every_variant(hzmod, case, prec, sweep, chunk):
    import torch
    p, S, kappa, v, ref = case
    G = _solver(hzmod, p, prec, sweep, chunk)
    try:
        G.factor()
        st = G.stats()
        z = G.apply_M(torch.from_numpy(v).cuda()).cpu().numpy()
    finally:
        G.close()
    # which variants ran
    assert st["max_snode_width"] == (128 if prec == "mixed" else 112), st
    if sweep == 1:
        assert st["fwd_levels_narrow"] == 0 and st["bwd_levels_narrow"] == 0
        assert st["fwd_levels_wide"] == st["solve_levels"] and st["bwd_levels_wide"] == st["solve_levels"]
        assert st["bwd_split_blocks"] > 0          # supernodes taller than one chunk
    elif sweep == 2:
        assert st["fwd_levels_wide"] == 0 and st["bwd_levels_wide"] == 0
        assert st["bwd_split_blocks"] > 0
    else:                                          # per level: as the host-only analysis plans it
        plan = hzmod.plan(p, precision=hzmod.HZ_MIXED if prec == "mixed" else hzmod.HZ_FP64)
        for key in VARIANT_KEYS:
            assert st[key] == plan[key], (key, st[key], plan[key])
    if prec == "mixed":
        assert st["tc_multi_fronts"] > 0 and st["tc_max_kstages"] > 1, st
        assert st["tc_tiles"] > st["tc_multi_fronts"]
    # the sweeps ran on merged solve trees: separator chains merged on the subdomains'
    # sparse top levels and in the direct coarse factor
    assert st["merged_chains"] > 0 and st["solve_levels"] < st["nlevels"], st
    assert st["coarse_merged_chains"] > 0 and st["coarse_solve_levels"] < st["nlevels_coarse"], st
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    tol = 1e-10 if prec == "fp64" else kappa * U32
    print(f"apply_M {prec} sweep={sweep} chunk={chunk}: rel L2 {err:.3e} (bound {tol:.3e}, "
          f"kappa_1 {kappa:.0f}); stats fwd {st['fwd_levels_wide']}/{st['fwd_levels_narrow']} "
          f"bwd {st['bwd_levels_wide']}/{st['bwd_levels_narrow']} split {st['bwd_split_blocks']} "
          f"tc {st['tc_tiles']} multi {st['tc_multi_fronts']} kstages {st['tc_max_kstages']}")
    assert err <= tol, (err, tol)


def test_fp64_solve_wide_tasks(hzmod, case):
    p, S, kappa, v, ref = case
    b = S.rhs()[:, 0]
    xo, ito, _, ok = S.solve(b)
    assert ok
    G = _solver(hzmod, p, "fp64", 1, 0)
    try:
        G.factor()
        xg, info = G.solve(b)
    finally:
        G.close()
    itg, status, rel = info[0]
    assert status == 0 and rel <= p.tol
    assert abs(itg - ito) <= 1, (itg, ito)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-9


@pytest.mark.parametrize("sweep", [0, 1])
def test_mixed_solve_against_oracle(hzmod, case, sweep):
    """The mixed path against the FP64 oracle: iterations within one at tol 1e-6, and the
    solutions within 1e-6 relative L2 once both are solved to 1e-9."""
    p, S, kappa, v, ref = case
    b = S.rhs()[:, 0]
    G = _solver(hzmod, p, "mixed", sweep, 0)
    try:
        G.factor()
        out = {}
        for tol in (1e-6, 1e-9):
            xo, ito, _, ok = S.solve(b, tol=tol)
            assert ok
            xg, info = G.solve(b, tol=tol)
            itg, status, rel = info[0]
            assert status == 0 and rel <= tol
            assert np.linalg.norm(b - S.A @ xg) / np.linalg.norm(b) <= tol * (1 + 1e-6)
            out[tol] = (itg, ito, np.linalg.norm(xg - xo) / np.linalg.norm(xo))
    finally:
        G.close()
    for tol, (itg, ito, err) in out.items():
        print(f"mixed sweep={sweep} tol {tol:g}: iterations gpu {itg} oracle {ito}; rel L2 vs oracle {err:.3e}")
    itg, ito, _ = out[1e-6]
    assert abs(itg - ito) <= 1, out
    assert out[1e-9][2] <= 1e-6, out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grouped_factorisation_is_bitwise_identical(hzmod, case, prec):
    """factor_group = 2 factorises the 7 subdomains in four groups that reuse one frontal
    workspace; every front sees the same kernels in the same order, so M^{-1} v is bitwise
    that of the all-at-once factorisation (and so matches the oracle as above)."""
    import torch
    p, S, kappa, v, ref = case
    out = []
    for grp in (0, 2):
        G = hzmod.Solver(p, precision=hzmod.HZ_MIXED if prec == "mixed" else hzmod.HZ_FP64, factor_group=grp)
        try:
            G.factor()
            st = G.stats()
            out.append((st["front_bytes"], G.apply_M(torch.from_numpy(v).cuda()).cpu().numpy()))
        finally:
            G.close()
    assert out[1][0] < out[0][0]                       # a smaller workspace
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sweep_autotuner_keeps_parity(hzmod, case, prec):
    """tune_sweeps times six task-shape schedules of the local sweeps at the first hz_factor
    and keeps the fastest; whichever it keeps, M^{-1} v still matches the oracle, and solves
    (whose iterations are then captured as graphs on the tuned task lists) converge."""
    import torch
    p, S, kappa, v, ref = case
    G = hzmod.Solver(p, precision=hzmod.HZ_MIXED if prec == "mixed" else hzmod.HZ_FP64, tune_sweeps=1)
    try:
        G.factor()
        st = G.stats()
        z = G.apply_M(torch.from_numpy(v).cuda()).cpu().numpy()
        b = S.rhs()[:, 0]
        x, info = G.solve(b)
    finally:
        G.close()
    assert st["sweep_chunk"] in ((256, 512) if prec == "mixed" else (128, 256))
    assert st["sweep_scale"] in (0.25, 0.5, 1.0, 2.0)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= (1e-10 if prec == "fp64" else kappa * U32), err
    assert info[0][1] == 0 and np.linalg.norm(b - S.A @ x) / np.linalg.norm(b) <= p.tol
