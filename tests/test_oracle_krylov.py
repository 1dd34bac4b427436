"""Pins for the oracle's FGMRES/CGS2/Givens: the minimal-residual property against an
explicit Krylov least-squares problem, unitarity of the rotations, restarts, breakdown."""
import numpy as np
import pytest

from oracle import krylov


def test_givens_rotation_zeroes_and_is_unitary():
    rng = np.random.default_rng(0)
    for _ in range(50):
        a = complex(*rng.standard_normal(2))
        b = abs(rng.standard_normal()) + 0.0j
        c, s = krylov.givens(a, b)
        G = np.array([[c, s], [-np.conj(s), c]])
        assert np.allclose(G.conj().T @ G, np.eye(2), atol=1e-14)
        r = G @ np.array([a, b])
        assert abs(r[1]) < 1e-14 and abs(abs(r[0]) - np.hypot(abs(a), abs(b))) < 1e-13
    c, s = krylov.givens(0.0, 2.0)
    assert c == 0.0 and s == 1.0


def test_residual_history_is_the_krylov_minimum():
    """GMRES without restart and with M = I minimises ||b - A x|| over K_k(A, b);
    compare the Givens estimate with lstsq over an explicit Krylov basis."""
    rng = np.random.default_rng(1)
    n = 60
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    hist = []
    x, it, rel, ok = krylov.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-10, m=n, history=hist)
    assert ok and rel <= 1e-10
    Kb = [b / np.linalg.norm(b)]
    for k in range(1, 12):
        Q, _ = np.linalg.qr(np.stack(Kb, axis=1))
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        rmin = np.linalg.norm(b - A @ Q @ y) / np.linalg.norm(b)
        assert abs(hist[k - 1] - rmin) <= 1e-9 * max(rmin, 1e-3), (k, hist[k - 1], rmin)
        Kb.append(A @ Kb[-1]); Kb[-1] /= np.linalg.norm(Kb[-1])


def test_restarted_and_preconditioned_solution():
    rng = np.random.default_rng(2)
    n = 80
    A = np.diag(np.linspace(1, 20, n)).astype(complex) + 0.3j * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n) + 0j
    Minv = np.diag(1.0 / np.diag(A))
    x, it, rel, ok = krylov.fgmres(lambda v: A @ v, lambda v: Minv @ v, b, tol=1e-8, m=5)
    assert ok
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-8
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-6)
    assert it > 5   # needed at least one restart


def test_exact_preconditioner_is_one_iteration():
    rng = np.random.default_rng(3)
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 5 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    Ainv = np.linalg.inv(A)
    x, it, rel, ok = krylov.fgmres(lambda v: A @ v, lambda v: Ainv @ v, b, tol=1e-8, m=10)
    assert ok and it == 1
