"""End-to-end pins for the oracle solve: brute-force dense solve, reciprocity,
attenuation lowering the iteration count."""
import numpy as np

import synth
from oracle.solver import OracleSolver


def test_tiny_config_against_dense_solve():
    p = synth.tiny_problem()
    S = OracleSolver(p)
    S.factor()
    b = S.rhs()[:, 0]
    Ad = S.A.toarray()
    xd = np.linalg.solve(Ad, b)
    assert np.linalg.norm(Ad @ xd - b) <= 1e-12 * np.linalg.norm(b)
    x, it, rel, ok = S.solve(b)
    assert ok and rel <= 1e-6
    assert np.linalg.norm(b - Ad @ x) <= 1e-6 * np.linalg.norm(b)
    assert np.linalg.norm(x - xd) <= 1e-4 * np.linalg.norm(xd)
    assert 5 <= it <= 30


def test_reciprocity():
    """A is complex symmetric, so the field of a source at s read at r equals the
    field of a source at r read at s."""
    p = synth.unit_cube_problem(n=8, nsub=8, overlap=1)
    S = OracleSolver(p)
    S.factor()
    pts = np.array([[0.25, 0.25, 0.5], [0.75, 0.625, 0.375]])
    ids = [int(round(x * 8)) + 9 * (int(round(y * 8)) + 9 * int(round(z * 8))) for x, y, z in pts]
    B = S.rhs(pts)
    X, its, rels, ok = S.solve(B, tol=1e-11)
    assert all(ok)
    assert abs(X[ids[1], 0] - X[ids[0], 1]) <= 1e-8 * abs(X[ids[1], 0])


def test_attenuation_lowers_iteration_count():
    its = []
    for Q in (1e6, 20.0):
        p = synth.small_overthrust(levels=1, cells=(4, 4, 2), freq=0.6, nsub=8, Q=Q)
        S = OracleSolver(p)
        S.factor()
        _, it, rel, ok = S.solve(S.rhs()[:, 0])
        assert ok
        its.append(it)
    assert its[1] < its[0], its
