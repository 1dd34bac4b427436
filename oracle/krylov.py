"""Oracle: restarted right-preconditioned FGMRES(m) with CGS2 and Givens rotations.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

GMRES is the Krylov solver of the method; its stopping rule is the relative
residual ||A x - b|| / ||b|| <= tol (experiments section, tol = 1e-6).
Readings: right preconditioning in the flexible form (the preconditioned
vectors z_j are stored, x = x0 + Z_m y); orthogonalisation by two passes of
classical Gram-Schmidt (CGS2) with the Hermitian inner product; complex
Givens rotations

    rho = sqrt(|a|^2 + |b|^2),  c = |a| / rho,  s = (a/|a|) conj(b) / rho
    (a = 0:  c = 0, s = 1),

applied as [c, s; -conj(s), c]; happy breakdown when h_{j+1,j} <= 1e-14 ||w_0||
(w_0 = A z_j before orthogonalisation).  The iteration count is the total
number of inner iterations over all cycles.  Convergence is declared only
after the true residual has been checked: at the end of a cycle, or as soon
as the Givens estimate |g_{j+1}| / ||b|| crosses tol (the cycle then ends, the
true residual is formed, and a failed check restarts from the current x).
x0 = 0.
"""
from __future__ import annotations

import numpy as np


def givens(a, b):
    """(c, s) with [c, s; -conj(s), c] [a; b] = [r; 0]."""
    aa = abs(a)
    if aa == 0.0:
        return 0.0, 1.0 + 0.0j
    rho = np.sqrt(aa * aa + abs(b) ** 2)
    return aa / rho, (a / aa) * np.conj(b) / rho


def fgmres(apply_A, apply_M, b, tol=1e-6, m=30, maxit=1000, history=None, verify=True):
    """Solve A x = b.  Returns (x, iterations, true relative residual, converged).

    ``verify=False`` (an inner solve) ends at the first cycle end -- the Givens
    estimate crossing tol, a happy breakdown or ``maxit`` -- without forming the
    true residual, and returns the estimate in its place."""
    b = np.asarray(b, np.complex128)
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, np.complex128)
    if bnorm == 0.0:
        return x, 0, 0.0, True
    r = b.copy()
    beta = bnorm
    its = 0
    while True:
        V = np.zeros((n, m + 1), np.complex128)
        Zs = np.zeros((n, m), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            Zs[:, j] = apply_M(V[:, j])
            w = apply_A(Zs[:, j])
            w0 = np.linalg.norm(w)
            Vj = V[:, : j + 1]
            h1 = Vj.conj().T @ w
            w = w - Vj @ h1
            h2 = Vj.conj().T @ w
            w = w - Vj @ h2
            h = h1 + h2
            hn = np.linalg.norm(w)
            H[: j + 1, j] = h
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            est = abs(g[j + 1]) / bnorm
            if history is not None:
                history.append(est)
            breakdown = hn <= 1e-14 * w0
            if breakdown or est <= tol or its >= maxit:
                break
            V[:, j + 1] = w / hn
        y = np.zeros(k, np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: k] @ y[i + 1: k]) / H[i, i]
        x = x + Zs[:, :k] @ y
        if not verify:
            return x, its, est, est <= tol
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol:
            return x, its, rel, True
        if its >= maxit:
            return x, its, rel, False
        beta = np.linalg.norm(r)
