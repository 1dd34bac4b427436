"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (FP64 path): the operator A is the same sum of element terms on both
sides, so A x agrees to 1e-13 relative; M^{-1} differs only by the rounding of
two different direct solvers (supernodal LDL^T without pivoting on the GPU,
SuperLU on the CPU), 1e-10 relative; full solves at tol 1e-6 follow the same
Krylov path, so the solutions agree to <= 1e-9 relative L2 and the iteration
counts within +-1.  Mixed path: the true residual ||b - A x|| / ||b|| computed
with the oracle's FP64 operator is <= tol, the iteration count is within one of the
oracle's, and, solved to 1e-9, the solution is within 1e-6 relative L2 of the
oracle's (element-wise M^{-1} parity of the mixed path is in test_gpu_variants).
"""
import numpy as np
import pytest

import synth
from oracle.solver import OracleSolver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hzmod():
    from paper_2004_06309_gb300 import build, hz
    build.build()
    return hz


def _rand(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def _cases():
    return {
        "tiny": synth.tiny_problem,
        "cube_p2_ragged": lambda: synth.unit_cube_problem(n=10, order=2, nsub=6, overlap=2, freq=1.5),
        "ovt_2lvl": lambda: synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16),
    }


@pytest.fixture(scope="module", params=list(_cases().keys()))
def pair(request, hzmod):
    p = _cases()[request.param]()
    S = OracleSolver(p)
    S.factor()
    G = hzmod.Solver(p)
    G.factor()
    yield p, S, G
    G.close()


def test_apply_A_matches_oracle(pair):
    import torch
    p, S, G = pair
    x = _rand(S.n, 1)
    y = G.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = S.apply_A(x)
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_apply_M_matches_oracle(pair):
    import torch
    p, S, G = pair
    v = _rand(S.n, 2)
    z = G.apply_M(torch.from_numpy(v).cuda()).cpu().numpy()
    ref = S.apply_M(v)
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
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, err
    # true residual with the oracle's operator
    assert np.linalg.norm(b - S.A @ xg) / np.linalg.norm(b) <= p.tol


def test_device_path_and_multiple_rhs(pair):
    import torch
    p, S, G = pair
    B = S.rhs(np.array([[0.3, 0.4, 0.5], [0.6, 0.35, 0.25]]) * (p.mesh.xyz.max(axis=0)))
    X, info = G.solve(torch.from_numpy(B).cuda())
    X = X.cpu().numpy()
    for j in range(2):
        assert info[j][1] == 0
        assert np.linalg.norm(B[:, j] - S.A @ X[:, j]) / np.linalg.norm(B[:, j]) <= p.tol


def test_cgs2_matches_two_gram_schmidt_passes(pair):
    """hz_cgs2 against the oracle's CGS2 formulas (krylov.fgmres: two classical passes)."""
    import torch
    p, S, G = pair
    rng = np.random.default_rng(5)
    for ncols in (1, 7, 33):
        V = rng.standard_normal((S.n, ncols)) + 1j * rng.standard_normal((S.n, ncols))
        V, _ = np.linalg.qr(V)
        w = rng.standard_normal(S.n) + 1j * rng.standard_normal(S.n)
        h1 = V.conj().T @ w
        w1 = w - V @ h1
        h2 = V.conj().T @ w1
        w2 = w1 - V @ h2
        wd = torch.from_numpy(w).cuda()
        h, nrm = G.cgs2(torch.from_numpy(V).cuda(), wd)
        assert np.allclose(h.cpu().numpy(), h1 + h2, rtol=0, atol=1e-12 * np.abs(h1).max())
        assert np.allclose(wd.cpu().numpy(), w2, rtol=0, atol=1e-12 * np.abs(w).max())
        assert abs(nrm - np.linalg.norm(w2)) <= 1e-12 * np.linalg.norm(w2)


def test_point_sources_match_oracle(pair):
    p, S, G = pair
    pts = np.array([[0.31, 0.47, 0.52]]) * p.mesh.xyz.max(axis=0)
    bg = G.point_sources(pts)
    bo = S.rhs(pts)
    assert np.abs(bg - bo).max() <= 1e-13


def test_rerun_is_bitwise_identical(pair):
    p, S, G = pair
    b = S.rhs()[:, 0]
    x1, i1 = G.solve(b)
    x2, i2 = G.solve(b)
    assert np.array_equal(x1, x2) and i1 == i2


def test_mixed_precision_reaches_tolerance(hzmod):
    p = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    S = OracleSolver(p)
    S.factor()
    b = S.rhs()[:, 0]
    xo, ito, _, _ = S.solve(b)
    G = hzmod.Solver(p, precision=hzmod.HZ_MIXED)
    G.factor()
    xg, info = G.solve(b)
    assert info[0][1] == 0
    assert np.linalg.norm(b - S.A @ xg) / np.linalg.norm(b) <= p.tol
    assert abs(info[0][0] - ito) <= 1, (info[0][0], ito)
    xo9, _, _, _ = S.solve(b, tol=1e-9)
    xg9, info9 = G.solve(b, tol=1e-9)
    assert info9[0][1] == 0
    assert np.linalg.norm(xg9 - xo9) <= 1e-6 * np.linalg.norm(xo9)
    G.close()


def test_edge_cases(hzmod):
    p = synth.tiny_problem()
    G = hzmod.Solver(p)
    b = np.zeros(G.n, np.complex128)
    with pytest.raises(hzmod.HzError) as e:
        G.solve(b)
    assert e.value.status == hzmod.HZ_ERR_STATE
    G.factor()
    x, info = G.solve(b)                       # zero right-hand side
    assert np.all(x == 0) and info[0][0] == 0
    bad = np.full(G.n, np.nan + 0j)
    x, info = G.solve(bad, check=False)
    assert info[0][1] == hzmod.HZ_ERR_BREAKDOWN
    G.close()


def test_one_subdomain_is_one_iteration(hzmod):
    p = synth.unit_cube_problem(n=6, nsub=1, overlap=0)
    G = hzmod.Solver(p)
    G.factor()
    S = OracleSolver(p)
    x, info = G.solve(S.rhs()[:, 0])
    assert info[0][0] == 1 and info[0][2] < 1e-10
    G.close()


@pytest.mark.parametrize("precision,block", [(0, 4), (0, 8), (1, 16)])
def test_pseudo_block_matches_one_at_a_time(hzmod, precision, block):
    """Pseudo-block FGMRES: each right-hand side keeps its own Krylov space and stopping
    decisions, so iterations match the one-at-a-time solve (+-1 for rounding in the
    batched operators) and, in FP64, the solutions agree to 1e-9; every column meets
    the tolerance with the oracle's operator.  Six sources with block 4 exercise a
    padded second batch."""
    p = synth.small_overthrust(levels=2, cells=(5, 5, 3), freq=0.6, nsub=16)
    S = OracleSolver(p)
    ext = p.mesh.xyz.max(axis=0)
    pts = np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.5, 0.5, 0.2], [0.3, 0.8, 0.6],
                    [0.8, 0.7, 0.4], [0.45, 0.55, 0.75]]) * ext
    B = S.rhs(pts)
    G1 = hzmod.Solver(p, precision=precision)
    G1.factor()
    X1, i1 = G1.solve(B)
    G1.close()
    GB = hzmod.Solver(p, precision=precision, block_size=block)
    GB.factor()
    XB, iB = GB.solve(B)
    GB.close()
    for j in range(B.shape[1]):
        assert iB[j][1] == 0
        assert abs(iB[j][0] - i1[j][0]) <= 1, (j, iB[j], i1[j])
        assert np.linalg.norm(B[:, j] - S.A @ XB[:, j]) / np.linalg.norm(B[:, j]) <= p.tol
        if precision == 0:
            assert np.linalg.norm(XB[:, j] - X1[:, j]) <= 1e-9 * np.linalg.norm(X1[:, j])


def test_graph_path_matches_eager_path(hzmod):
    """On a non-default stream every inner iteration runs as a captured CUDA graph; the
    result must be bitwise identical to the eager launches on the default stream."""
    import torch
    p = synth.small_overthrust(levels=2, cells=(4, 4, 2), freq=0.5, nsub=8)
    S = OracleSolver(p)
    b = S.rhs()[:, 0]
    G0 = hzmod.Solver(p, spmv_lanes=4)          # same SpMV summation order in both contexts
    G0.factor()
    x0, i0 = G0.solve(b)
    G0.close()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        G1 = hzmod.Solver(p, stream=s, spmv_lanes=4)
        G1.factor()
        x1, i1 = G1.solve(b)
        x2, i2 = G1.solve(b)           # second solve replays the captured graphs
        G1.close()
    assert i0 == i1 == i2
    assert np.array_equal(x0, x1) and np.array_equal(x1, x2)
