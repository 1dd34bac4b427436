"""GPU parity of the iterative coarse solve (GMRES on E right-preconditioned by
one-level ORAS on the coarse mesh, coarse_solver = HZ_COARSE_ORAS) against the
oracle's CoarseORAS, through the C ABI.

Both sides run the same inner iteration (one cycle, stop on the Givens estimate);
their inner counts agree unless an estimate lands within rounding of coarse_tol,
so each comparison first checks that the counts are equal.  Tolerances as for the
direct coarse solve: M^{-1} v to 1e-10, FP64 solves to 1e-9 with iterations +-1,
mixed solves to tol with the oracle's FP64 operator."""
import numpy as np
import pytest

import synth
from oracle.solver import OracleSolver

pytestmark = pytest.mark.gpu

TOLH, MH = 1e-3, 40


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def _cases():
    return {
        "ovt": lambda: synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16),
        "cube_p2": lambda: synth.unit_cube_problem(n=8, freq=1.0, order=2, nsub=4, overlap=1, levels=2),
    }


@pytest.fixture(scope="module", params=list(_cases().keys()))
def pair(request, hzmod):
    p = _cases()[request.param]()
    S = OracleSolver(p, coarse_solver="oras", coarse_tol=TOLH, coarse_m=MH)
    S.factor()
    G = hzmod.Solver(p, coarse_solver=hzmod.HZ_COARSE_ORAS, coarse_tol=TOLH, coarse_maxit=MH)
    G.factor()
    yield p, S, G
    G.close()


def test_preconditioner_matches_oracle(pair):
    import torch
    p, S, G = pair
    rng = np.random.default_rng(3)
    v = rng.standard_normal(S.n) + 1j * rng.standard_normal(S.n)
    k0 = G.stats()["coarse_iterations"]
    z = G.apply_M(torch.from_numpy(v).cuda()).cpu().numpy()
    kg = G.stats()["coarse_iterations"] - k0
    ref = S.apply_M(v)
    assert kg == S.coarse_its[-1] and kg >= 1
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    assert err <= 1e-10, err


def test_solve_matches_oracle(pair):
    p, S, G = pair
    b = S.rhs()[:, 0]
    xo, ito, relo, ok = S.solve(b)
    assert ok
    xg, info = G.solve(b)
    itg, st, relg = info[0]
    assert st == 0 and relg <= p.tol
    assert abs(itg - ito) <= 1, (itg, ito)
    assert np.linalg.norm(xg - xo) <= 1e-9 * np.linalg.norm(xo)
    assert np.linalg.norm(b - S.A @ xg) / np.linalg.norm(b) <= p.tol


def test_mixed_precision_and_pseudo_block(hzmod):
    p = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    S = OracleSolver(p)
    ext = p.mesh.xyz.max(axis=0)
    B = S.rhs(np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.5, 0.5, 0.2], [0.3, 0.8, 0.6],
                        [0.8, 0.7, 0.4]]) * ext)
    G1 = hzmod.Solver(p, precision=hzmod.HZ_MIXED, coarse_solver=hzmod.HZ_COARSE_ORAS, coarse_tol=TOLH,
                      coarse_maxit=MH)
    G1.factor()
    X1, i1 = G1.solve(B)
    G1.close()
    GB = hzmod.Solver(p, precision=hzmod.HZ_MIXED, coarse_solver=hzmod.HZ_COARSE_ORAS, coarse_tol=TOLH,
                      coarse_maxit=MH, block_size=4)
    GB.factor()
    XB, iB = GB.solve(B)
    GB.close()
    for j in range(B.shape[1]):
        assert i1[j][1] == 0 and iB[j][1] == 0
        assert abs(iB[j][0] - i1[j][0]) <= 1, (j, iB[j], i1[j])
        for X in (X1, XB):
            assert np.linalg.norm(B[:, j] - S.A @ X[:, j]) / np.linalg.norm(B[:, j]) <= p.tol


def test_tight_inner_tolerance_equals_the_direct_coarse_solve(hzmod):
    """With coarse_tol near rounding level the inner GMRES solves E to that accuracy, so
    M^{-1} v agrees with the direct coarse solve of the same context options."""
    import torch
    p = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    G = hzmod.Solver(p, coarse_solver=hzmod.HZ_COARSE_ORAS, coarse_tol=1e-13, coarse_maxit=63)
    G.factor()
    D = hzmod.Solver(p)
    D.factor()
    v = torch.from_numpy(np.random.default_rng(1).standard_normal(G.n) + 0j).cuda()
    z = G.apply_M(v).cpu().numpy()
    st = G.stats()
    zd = D.apply_M(v).cpu().numpy()
    assert st["coarse_solves"] == 1 and 1 <= st["coarse_iterations"] < 63
    assert np.linalg.norm(z - zd) <= 1e-9 * np.linalg.norm(zd)
    G.close()
    D.close()
