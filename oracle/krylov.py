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


# ---------------------------------------------------------------------------
# Block FGMRES: one block Krylov space for s right-hand sides (the block form the
# experiments section sets beside pseudo-block GMRES for many sources).  Right
# preconditioning in the flexible form, x0 = 0.  Per cycle:
#   * the block residual is factored R = V_0 beta (column-wise CGS2 among its columns,
#     beta upper triangular);
#   * block step j: Z_j = M^{-1} V_j, W = A Z_j; two classical Gram-Schmidt passes of
#     all s columns against V_0..V_j (H_{i,j} = h1 + h2); then the columns of W are
#     orthonormalised among themselves, column by column (CGS2 against the new block's
#     earlier columns), giving V_{j+1} and the upper-triangular H_{j+1,j};
#   * the band Hessenberg matrix is reduced column by column by the Givens rotations of
#     fgmres, each between the diagonal row and one of the s rows below it (bottom
#     row first), and the same rotations are applied to G = [beta; 0]; the residual of
#     right-hand side i is estimated by the norm of column i of G's rows below the
#     triangle;
#   * the cycle ends when every estimate / ||b_i|| <= tol, on a happy breakdown (a
#     column of the new block at or below 1e-14 of ||A z|| of its column) or at maxit;
#     then x += Z R^{-1} G_top and the true residuals are checked, restarting from them
#     if any misses tol.
# The iteration count is the number of block steps (each applies M^{-1} and A once per
# right-hand side).  Columns that are zero keep x = 0 and take no part.
# ---------------------------------------------------------------------------
def _block_orthonormalise(W, w0):
    """Column-wise CGS2 among the columns of W: W = Q R (R upper triangular).  Returns
    (Q, R, breakdown) with breakdown when a column's remaining norm is <= 1e-14 of w0."""
    n, s = W.shape
    Q = np.zeros((n, s), np.complex128)
    R = np.zeros((s, s), np.complex128)
    brk = False
    for c in range(s):
        w = W[:, c].copy()
        if c > 0:
            Qc = Q[:, :c]
            q1 = Qc.conj().T @ w
            w = w - Qc @ q1
            q2 = Qc.conj().T @ w
            w = w - Qc @ q2
            R[:c, c] = q1 + q2
        nrm = np.linalg.norm(w)
        R[c, c] = nrm
        brk = brk or nrm <= 1e-14 * w0[c]
        Q[:, c] = w / nrm if nrm > 0.0 else 0.0
    return Q, R, brk


def block_fgmres(apply_A, apply_M, B, tol=1e-6, m=30, maxit=1000, diagnostics=None):
    """Solve A X = B for the columns of B together.  Returns (X, iterations, true
    relative residuals, converged) with one residual per column.  A dict passed as
    ``diagnostics`` receives the last cycle's basis V, the stored Z and the unrotated
    block Hessenberg matrix (keys "V", "Z", "H")."""
    B = np.asarray(B, np.complex128)
    n, s_all = B.shape
    X = np.zeros_like(B)
    bn_all = np.linalg.norm(B, axis=0)
    act = np.nonzero(bn_all > 0.0)[0]
    rel_all = np.zeros(s_all)
    if len(act) == 0:
        return X, 0, rel_all, True
    Bc = B[:, act]
    bn = bn_all[act]
    s = len(act)
    Xc = np.zeros((n, s), np.complex128)
    R0 = Bc.copy()
    its = 0
    while True:
        V0, beta, _ = _block_orthonormalise(R0, np.linalg.norm(R0, axis=0))
        V = [V0]
        Zs = []
        ncol = (m + 1) * s
        H = np.zeros((ncol, m * s), np.complex128)
        G = np.zeros((ncol, s), np.complex128)
        G[:s, :] = beta
        rots = []                                     # (row i, row r, c, sn) in order
        Hraw = np.zeros_like(H) if diagnostics is not None else None
        k = 0
        for j in range(m):
            Zj = np.column_stack([apply_M(V[j][:, c]) for c in range(s)])
            Zs.append(Zj)
            W = np.column_stack([apply_A(Zj[:, c]) for c in range(s)])
            w0 = np.linalg.norm(W, axis=0)
            Vb = np.hstack(V)
            h1 = Vb.conj().T @ W
            W = W - Vb @ h1
            h2 = Vb.conj().T @ W
            W = W - Vb @ h2
            Qn, Rn, brk = _block_orthonormalise(W, w0)
            V.append(Qn)
            c0 = j * s
            H[: (j + 1) * s, c0: c0 + s] = h1 + h2
            H[(j + 1) * s: (j + 2) * s, c0: c0 + s] = Rn
            if diagnostics is not None:
                Hraw[:, c0: c0 + s] = H[:, c0: c0 + s]
                diagnostics["V"] = np.hstack(V)
                diagnostics["Z"] = np.hstack(Zs)
                diagnostics["H"] = Hraw[: (j + 2) * s, : (j + 1) * s].copy()
            for c in range(s):
                col = c0 + c
                for (i, r, cs, sn) in rots:
                    t = cs * H[i, col] + sn * H[r, col]
                    H[r, col] = -np.conj(sn) * H[i, col] + cs * H[r, col]
                    H[i, col] = t
                for r in range(col + s, col, -1):        # bottom row first
                    cs, sn = givens(H[col, col], H[r, col])
                    t = cs * H[col, col] + sn * H[r, col]
                    H[r, col] = 0.0
                    H[col, col] = t
                    gi = cs * G[col, :] + sn * G[r, :]
                    G[r, :] = -np.conj(sn) * G[col, :] + cs * G[r, :]
                    G[col, :] = gi
                    rots.append((col, r, cs, sn))
            its += 1
            k = j + 1
            est = np.linalg.norm(G[k * s: (k + 1) * s, :], axis=0) / bn
            if brk or np.all(est <= tol) or its >= maxit:
                break
        p = k * s
        Rt = H[:p, :p]
        Y = np.zeros((p, s), np.complex128)
        for i in range(p - 1, -1, -1):
            Y[i, :] = (G[i, :] - Rt[i, i + 1: p] @ Y[i + 1: p, :]) / Rt[i, i]
        Xc = Xc + np.hstack(Zs) @ Y
        R0 = Bc - np.column_stack([apply_A(Xc[:, c]) for c in range(s)])
        rel = np.linalg.norm(R0, axis=0) / bn
        if np.all(rel <= tol) or its >= maxit:
            X[:, act] = Xc
            rel_all[act] = rel
            return X, its, rel_all, bool(np.all(rel <= tol))


# ---------------------------------------------------------------------------
# GCRO-DR: GMRES with deflated restarting and subspace recycling (Parks, de Sturler,
# Mackey, Johnson, Maiti 2006), the Krylov-recycling method the paper names as its
# next step for many right-hand sides.  Right preconditioning with a fixed M: the
# iteration runs on A M^{-1} in the preconditioned space, and a recycled space is
# kept in both spaces, Uh (preconditioned) and Ux = M^{-1} Uh, with C = A Ux,
# C^H C = I.  Per cycle:
#   * r is made orthogonal to C (x += Ux C^H r, r -= C C^H r);
#   * Arnoldi on (I - C C^H) A M^{-1}: each new vector is orthogonalised against
#     [C, V] by CGS2; the C coefficients form B, the V ones the Hessenberg H;
#   * the least-squares problem min || [0; beta e1] - [[D, B], [0, H]] [y1; y2] ||
#     splits: y2 by Givens on H (as in fgmres), y1 = -D^{-1} B y2, so that
#     x += Z y2 - Ux (B y2) (D scales Uh to unit columns);
#   * at the cycle end, if the true residual misses tol, k harmonic Ritz vectors
#     (smallest |theta|) of the cycle's space become the new recycled space:
#       first cycle:  (H_m + |h_{m+1,m}|^2 H_m^{-H} e_m e_m^H) z = theta z,
#       later:        G^H G z = theta G^H (Vh^H Wh) z,  G = [[D, B], [0, H]],
#                     Vh = [C, V_{p+1}],  Wh = [Uh D, V_p];
#     with P their eigenvectors: [Q, R] = qr(G P), C = Vh Q, Uh = Wh P R^{-1},
#     Ux = Wx P R^{-1} (Wx = [Ux D, Z_p]).
# A recycled space passed in (from the previous right-hand side at the same A and
# M) is used from the first cycle on; cycles hold m vectors in all (k recycled,
# m - k new).  Convergence and iteration counting follow fgmres.
# ---------------------------------------------------------------------------
def _arnoldi_cycle(apply_A, apply_M, r, beta, C, p, bnorm, tol, its, maxit, history):
    n = r.shape[0]
    kk = 0 if C is None else C.shape[1]
    V = np.zeros((n, p + 1), np.complex128)
    Zs = np.zeros((n, p), np.complex128)
    H = np.zeros((p + 1, p), np.complex128)
    B = np.zeros((kk, p), np.complex128)
    R = np.zeros((p + 1, p), np.complex128)          # Givens-rotated copy of H
    cs = np.zeros(p)
    sn = np.zeros(p, np.complex128)
    g = np.zeros(p + 1, np.complex128)
    g[0] = beta
    V[:, 0] = r / beta
    k = 0
    for j in range(p):
        Zs[:, j] = apply_M(V[:, j])
        w = apply_A(Zs[:, j])
        w0 = np.linalg.norm(w)
        Q = V[:, : j + 1] if kk == 0 else np.hstack([C, V[:, : j + 1]])
        h1 = Q.conj().T @ w
        w = w - Q @ h1
        h2 = Q.conj().T @ w
        w = w - Q @ h2
        h = h1 + h2
        hn = np.linalg.norm(w)
        B[:, j] = h[:kk]
        H[: j + 1, j] = h[kk:]
        H[j + 1, j] = hn
        col = H[: j + 2, j].copy()
        for i in range(j):
            t = cs[i] * col[i] + sn[i] * col[i + 1]
            col[i + 1] = -np.conj(sn[i]) * col[i] + cs[i] * col[i + 1]
            col[i] = t
        cs[j], sn[j] = givens(col[j], col[j + 1])
        col[j] = cs[j] * col[j] + sn[j] * col[j + 1]
        col[j + 1] = 0.0
        R[: j + 2, j] = col
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        its += 1
        k = j + 1
        est = abs(g[j + 1]) / bnorm
        if history is not None:
            history.append(est)
        if hn > 0.0:
            V[:, j + 1] = w / hn          # kept even at the last step: it spans A Z with V
        if hn <= 1e-14 * w0 or est <= tol or its >= maxit:
            break
    y = np.zeros(k, np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1: k] @ y[i + 1: k]) / R[i, i]
    return V[:, : k + 1], Zs[:, :k], H[: k + 1, :k], B[:, :k], y, its


def _smallest_harmonic(Mat_a, Mat_b, k):
    """Eigenvectors of Mat_a z = theta Mat_b z for the k smallest |theta|."""
    import scipy.linalg as sla
    th, Z = sla.eig(Mat_a, Mat_b)
    th = np.where(np.isfinite(th), th, np.inf)
    order = np.argsort(np.abs(th), kind="stable")
    return Z[:, order[:k]]


def gcrodr(apply_A, apply_M, b, tol=1e-6, m=50, k=10, recycle=None, maxit=1000, history=None):
    """Solve A x = b.  Returns (x, iterations, true relative residual, converged, recycle)
    where recycle = (Ux, Uh, C) for the next right-hand side at the same A and M."""
    b = np.asarray(b, np.complex128)
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    x = np.zeros(n, np.complex128)
    if bnorm == 0.0:
        return x, 0, 0.0, True, recycle
    Ux = Uh = C = None
    if recycle is not None:
        Ux, Uh, C = recycle
    r = b.copy()
    its = 0
    while True:
        if C is not None:                                   # r orthogonal to C
            c = C.conj().T @ r
            x = x + Ux @ c
            r = r - C @ c
        beta = np.linalg.norm(r)
        p = m if C is None else m - C.shape[1]
        V, Zs, H, B, y, its = _arnoldi_cycle(apply_A, apply_M, r, beta, C, p, bnorm, tol, its, maxit,
                                             history)
        kc = y.shape[0]
        x = x + Zs @ y
        if C is not None:
            x = x - Ux @ (B @ y)
        r = b - apply_A(x)
        rel = np.linalg.norm(r) / bnorm
        # new recycled space from this cycle (kept for the next right-hand side as well)
        if C is None:
            Ux, Uh, C = _first_recycle(V, Zs, H, kc, k)
        else:
            kk = C.shape[1]
            dn = 1.0 / np.linalg.norm(Uh, axis=0)
            D = np.diag(dn)
            G = np.zeros((kk + kc + 1, kk + kc), np.complex128)
            G[:kk, :kk] = D
            G[:kk, kk:] = B
            G[kk:, kk:] = H
            Vh = np.hstack([C, V])
            Wh = np.hstack([Uh * dn, V[:, :kc]])
            Wx = np.hstack([Ux * dn, Zs])
            P = _smallest_harmonic(G.conj().T @ G, G.conj().T @ (Vh.conj().T @ Wh), min(k, kk + kc))
            Q, Rq = np.linalg.qr(G @ P)
            Rinv = np.linalg.inv(Rq)
            C = Vh @ Q
            Uh = Wh @ P @ Rinv
            Ux = Wx @ P @ Rinv
        if rel <= tol or its >= maxit:
            return x, its, rel, rel <= tol, (Ux, Uh, C)


def block_gcrodr(apply_A, apply_M, B, tol=1e-6, m=30, k=8, recycle=None, maxit=1000):
    """Block GCRO-DR: block FGMRES (block_fgmres's steps) with a recycled space (gcrodr's),
    for the s columns of B together.  Returns (X, iterations, true relative residuals,
    converged, recycle) with recycle = (Ux, Uh, C) for the next block at the same A and M.

    Per cycle: R is made orthogonal to C (X += Ux C^H R, R -= C C^H R) and factored R = V_0 beta;
    each block step orthogonalises A M^{-1} V_j against [C, V_0..V_j] by CGS2 (the C
    coefficients form B, the V ones the block Hessenberg H), then the new block column by
    column; p = m - ceil(k_now / s) block steps at most.  The least-squares problem splits as
    in gcrodr: Y2 from the band Hessenberg by the Givens rotations of block_fgmres, Y1 = -D^{-1} B
    Y2, so X += Z Y2 - Ux (B Y2).  At the cycle end the k harmonic Ritz vectors of smallest
    |theta| form the new space:
      first cycle:  (H_m + H_m^{-H} E (H_{+}^H H_{+}) E^H) z = theta z, H_{+} the s x s block below
                    H_m and E its last s columns of the identity;
      later:        G^H G z = theta G^H (Vh^H Wh) z as in gcrodr, with block matrices.
    The iteration count is the number of block steps."""
    B = np.asarray(B, np.complex128)
    n, s = B.shape
    bn = np.linalg.norm(B, axis=0)
    assert np.all(bn > 0.0)
    X = np.zeros_like(B)
    Ux = Uh = C = None
    if recycle is not None:
        Ux, Uh, C = recycle
    R0 = B.copy()
    its = 0
    while True:
        kk = 0 if C is None else C.shape[1]
        if kk:
            c = C.conj().T @ R0
            X = X + Ux @ c
            R0 = R0 - C @ c
        V0, beta, _ = _block_orthonormalise(R0, np.linalg.norm(R0, axis=0))
        p = max(1, m - (kk + s - 1) // s)
        V, Zs = [V0], []
        H = np.zeros(((p + 1) * s, p * s), np.complex128)
        Bc = np.zeros((kk, p * s), np.complex128)
        Hr = np.zeros_like(H)                               # Givens-rotated copy
        G = np.zeros(((p + 1) * s, s), np.complex128)
        G[:s, :] = beta
        rots = []
        ks = 0
        for j in range(p):
            Zj = np.column_stack([apply_M(V[j][:, c]) for c in range(s)])
            Zs.append(Zj)
            W = np.column_stack([apply_A(Zj[:, c]) for c in range(s)])
            w0 = np.linalg.norm(W, axis=0)
            Q = np.hstack(([C] if kk else []) + V)
            h1 = Q.conj().T @ W
            W = W - Q @ h1
            h2 = Q.conj().T @ W
            W = W - Q @ h2
            h = h1 + h2
            Qn, Rn, brk = _block_orthonormalise(W, w0)
            V.append(Qn)
            c0 = j * s
            Bc[:, c0: c0 + s] = h[:kk]
            H[: (j + 1) * s, c0: c0 + s] = h[kk:]
            H[(j + 1) * s: (j + 2) * s, c0: c0 + s] = Rn
            Hr[:, c0: c0 + s] = H[:, c0: c0 + s]
            for q in range(s):
                col = c0 + q
                for (i, r, cs, sn) in rots:
                    t = cs * Hr[i, col] + sn * Hr[r, col]
                    Hr[r, col] = -np.conj(sn) * Hr[i, col] + cs * Hr[r, col]
                    Hr[i, col] = t
                for r in range(col + s, col, -1):
                    cs, sn = givens(Hr[col, col], Hr[r, col])
                    t = cs * Hr[col, col] + sn * Hr[r, col]
                    Hr[r, col] = 0.0
                    Hr[col, col] = t
                    gi = cs * G[col, :] + sn * G[r, :]
                    G[r, :] = -np.conj(sn) * G[col, :] + cs * G[r, :]
                    G[col, :] = gi
                    rots.append((col, r, cs, sn))
            its += 1
            ks = j + 1
            est = np.linalg.norm(G[ks * s: (ks + 1) * s, :], axis=0) / bn
            if brk or np.all(est <= tol) or its >= maxit:
                break
        kc = ks * s
        Y = np.zeros((kc, s), np.complex128)
        for i in range(kc - 1, -1, -1):
            Y[i, :] = (G[i, :] - Hr[i, i + 1: kc] @ Y[i + 1: kc, :]) / Hr[i, i]
        Zb = np.hstack(Zs)
        Vb = np.hstack(V)                                   # kc + s columns
        X = X + Zb @ Y
        if kk:
            X = X - Ux @ (Bc[:, :kc] @ Y)
        R0 = B - np.column_stack([apply_A(X[:, c]) for c in range(s)])
        rel = np.linalg.norm(R0, axis=0) / bn
        Hm = H[: kc + s, :kc]
        if k > 0:
            if not kk:
                Hsq = Hm[:kc, :kc]
                Hp = Hm[kc: kc + s, kc - s: kc]
                E = np.zeros((kc, s), np.complex128)
                E[kc - s:, :] = np.eye(s)
                F = np.linalg.solve(Hsq.conj().T, E)
                Mh = Hsq + F @ (Hp.conj().T @ Hp) @ E.conj().T
                P = _smallest_harmonic(Mh, np.eye(kc), min(k, kc))
                Qg, Rq = np.linalg.qr(Hm @ P)
                Rinv = np.linalg.inv(Rq)
                C = Vb @ Qg
                Uh = Vb[:, :kc] @ P @ Rinv
                Ux = Zb @ P @ Rinv
            else:
                dn = 1.0 / np.linalg.norm(Uh, axis=0)
                Gm = np.zeros((kk + kc + s, kk + kc), np.complex128)
                Gm[:kk, :kk] = np.diag(dn)
                Gm[:kk, kk:] = Bc[:, :kc]
                Gm[kk:, kk:] = Hm
                Vh = np.hstack([C, Vb])
                Wh = np.hstack([Uh * dn, Vb[:, :kc]])
                Wx = np.hstack([Ux * dn, Zb])
                P = _smallest_harmonic(Gm.conj().T @ Gm, Gm.conj().T @ (Vh.conj().T @ Wh), min(k, kk + kc))
                Qg, Rq = np.linalg.qr(Gm @ P)
                Rinv = np.linalg.inv(Rq)
                C = Vh @ Qg
                Uh = Wh @ P @ Rinv
                Ux = Wx @ P @ Rinv
        if np.all(rel <= tol) or its >= maxit:
            rec = None if C is None else (Ux, Uh, C)
            return X, its, rel, bool(np.all(rel <= tol)), rec


def rebase_recycle(apply_A, recycle):
    """Carry a recycled space (Ux, Uh, C) over to a new operator (Parks et al. 2006, for a
    sequence of matrices): C' = A_new Ux is orthonormalised column by column (CGS2),
    C' = Q R, and the space becomes (Ux R^{-1}, Uh R^{-1}, Q), so that C = A_new Ux and
    C^H C = I hold again.  Uh keeps the old preconditioned side; it only steers the choice
    of the next recycled space."""
    Ux, Uh, C = recycle
    AU = np.column_stack([apply_A(Ux[:, i]) for i in range(Ux.shape[1])])
    Q, R, _ = _block_orthonormalise(AU, np.linalg.norm(AU, axis=0))
    Rinv = np.linalg.inv(R)
    return Ux @ Rinv, Uh @ Rinv, Q


def _first_recycle(V, Zs, H, kc, k):
    """Recycled space from a plain GMRES cycle: harmonic Ritz vectors of H_m."""
    Hm = H[:kc, :kc]
    hl = H[kc, kc - 1]
    em = np.zeros(kc, np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(Hm.conj().T, em)
    Mh = Hm + (abs(hl) ** 2) * np.outer(f, em)
    P = _smallest_harmonic(Mh, np.eye(kc), min(k, kc))
    Q, Rq = np.linalg.qr(H @ P)
    Rinv = np.linalg.inv(Rq)
    C = V @ Q
    Uh = V[:, :kc] @ P @ Rinv
    Ux = Zs @ P @ Rinv
    return Ux, Uh, C
