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


# --- GCRO-DR (Krylov recycling) ---------------------------------------------

def _dense(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3 + spread * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    return A


def test_gcrodr_without_recycling_is_fgmres():
    rng = np.random.default_rng(2)
    n = 80
    A = _dense(n, 3)
    M = np.diag(1.0 / np.diag(A))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x1, i1, r1, ok1 = krylov.fgmres(lambda v: A @ v, lambda v: M @ v, b, tol=1e-10, m=12)
    x2, i2, r2, ok2, rec = krylov.gcrodr(lambda v: A @ v, lambda v: M @ v, b, tol=1e-10, m=12, k=0)
    assert ok1 and ok2 and i1 == i2
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)


def test_recycled_space_invariants():
    """C = A Ux with orthonormal C, and Ux = M^{-1} Uh, after a solve and after a second
    one that reuses and updates the space (a wrong G, B or index breaks these)."""
    rng = np.random.default_rng(4)
    n = 90
    A = _dense(n, 5, spread=2.0)
    Minv = np.linalg.inv(np.diag(np.diag(A)) + 0.3 * np.eye(n))
    rec = None
    for _ in range(2):
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x, it, rel, ok, rec = krylov.gcrodr(lambda v: A @ v, lambda v: Minv @ v, b, tol=1e-9, m=14, k=5,
                                            recycle=rec)
        assert ok and np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)
        Ux, Uh, C = rec
        assert np.abs(C.conj().T @ C - np.eye(C.shape[1])).max() <= 1e-12
        assert np.abs(A @ Ux - C).max() <= 1e-12 * np.abs(C).max()
        assert np.abs(Minv @ Uh - Ux).max() <= 1e-12 * np.abs(Ux).max()


def test_harmonic_ritz_space_is_invariant_when_the_cycle_spans_everything():
    """With m >= n the first cycle's Krylov space is the whole space, the harmonic Ritz
    pairs are exact eigenpairs, and the recycled space is the span of the k eigenvectors
    of A M^{-1} with the smallest |eigenvalue| (checked against numpy's eigensolver)."""
    rng = np.random.default_rng(6)
    n = 10
    lam = np.array([0.05, 0.1, 0.2, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0]) * (1 + 0.1j)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, it, rel, ok, rec = krylov.gcrodr(lambda v: A @ v, lambda v: v, b, tol=1e-12, m=n, k=3)
    Ux, Uh, C = rec
    ev, EV = np.linalg.eig(A)
    small = EV[:, np.argsort(np.abs(ev))[:3]]
    Qs, _ = np.linalg.qr(small)
    Qu, _ = np.linalg.qr(Uh)
    # the two 3-dimensional subspaces coincide: singular values of Qs^H Qu are all 1
    sv = np.linalg.svd(Qs.conj().T @ Qu, compute_uv=False)
    assert np.all(np.abs(sv - 1.0) <= 1e-8), sv


def test_deflated_restarting_beats_plain_restarting_on_small_outliers():
    """A few eigenvalues near zero stall restarted GMRES; GCRO-DR(m, k) deflates them
    across restarts and needs fewer iterations (the method's reason to exist)."""
    rng = np.random.default_rng(7)
    n = 200
    lam = np.concatenate([[1e-3, 2e-3, 4e-3, 8e-3], rng.uniform(1.0, 2.0, n - 4)]).astype(np.complex128)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    A = Q @ np.diag(lam) @ Q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xf, itf, rf, okf = krylov.fgmres(lambda v: A @ v, lambda v: v, b, tol=1e-8, m=10, maxit=3000)
    xg, itg, rg, okg, _ = krylov.gcrodr(lambda v: A @ v, lambda v: v, b, tol=1e-8, m=10, k=4, maxit=3000)
    assert okg and rg <= 1e-8
    assert itg < itf, (itg, itf)


def test_recycling_helps_the_next_right_hand_side():
    import synth
    from oracle.solver import OracleSolver
    p = synth.tiny_problem()
    S = OracleSolver(p)
    S.factor()
    ext = p.mesh.xyz.max(axis=0)
    B = S.rhs(np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.3, 0.8, 0.6]]) * ext)
    rec = None
    its_rec, its_plain = [], []
    for j in range(B.shape[1]):
        x, it, rel, ok, rec = krylov.gcrodr(S.apply_A, S.apply_M, B[:, j], tol=1e-6, m=20, k=8, recycle=rec)
        assert ok and np.linalg.norm(B[:, j] - S.A @ x) <= 1e-6 * np.linalg.norm(B[:, j])
        its_rec.append(it)
        its_plain.append(krylov.fgmres(S.apply_A, S.apply_M, B[:, j], tol=1e-6, m=20)[1])
    assert its_rec[0] == its_plain[0]                 # nothing recycled yet
    assert sum(its_rec[1:]) < sum(its_plain[1:]), (its_rec, its_plain)


# --- block FGMRES ------------------------------------------------------------------

def _block_problem(n=60, s=3, seed=7):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 3 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    d = 1.0 + rng.uniform(0, 1, n)                       # a diagonal right preconditioner
    B = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    return A, (lambda v: A @ v), (lambda v: v / d), d, B


def test_block_fgmres_with_one_column_is_fgmres():
    A, fa, fm, d, B = _block_problem()
    x1, i1, r1, o1 = krylov.fgmres(fa, fm, B[:, 0], tol=1e-10, m=8)
    X, ib, rb, ob = krylov.block_fgmres(fa, fm, B[:, :1], tol=1e-10, m=8)
    assert o1 and ob and i1 == ib
    assert np.linalg.norm(X[:, 0] - x1) <= 1e-12 * np.linalg.norm(x1)


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_block_fgmres_minimises_over_the_block_krylov_space(k):
    """After k block steps of one cycle, each column's residual is the least-squares minimum
    of ||b_i - A M^{-1} K y|| over the whole block Krylov space K = [B, A M^{-1} B, ...]
    (every column searches the space spanned by all the columns' Krylov vectors)."""
    A, fa, fm, d, B = _block_problem()
    s = B.shape[1]
    X, its, rel, ok = krylov.block_fgmres(fa, fm, B, tol=1e-300, m=20, maxit=k)
    assert its == k
    blocks = [B]
    for _ in range(1, k):
        Q = blocks[-1]
        blocks.append(np.column_stack([fa(fm(Q[:, c])) for c in range(s)]))
    Q, _ = np.linalg.qr(np.hstack(blocks))
    AMQ = np.column_stack([fa(fm(Q[:, c])) for c in range(Q.shape[1])])
    for i in range(s):
        y, *_ = np.linalg.lstsq(AMQ, B[:, i], rcond=None)
        rmin = np.linalg.norm(B[:, i] - AMQ @ y) / np.linalg.norm(B[:, i])
        r_block = np.linalg.norm(B[:, i] - A @ X[:, i]) / np.linalg.norm(B[:, i])
        assert abs(r_block - rmin) <= 1e-9 * max(rmin, 1e-6), (k, i, r_block, rmin)
        assert abs(rel[i] - r_block) <= 1e-12


def test_block_fgmres_needs_no_more_steps_than_its_slowest_column():
    """The block space contains each column's own Krylov space of the same step count, so
    without restarts the block solve converges in at most as many steps as the slowest
    single-column solve, and it solves every column."""
    A, fa, fm, d, B = _block_problem(n=80, s=4, seed=3)
    single = [krylov.fgmres(fa, fm, B[:, i], tol=1e-8, m=80)[1] for i in range(4)]
    X, its, rel, ok = krylov.block_fgmres(fa, fm, B, tol=1e-8, m=80)
    assert ok and its <= max(single), (its, single)
    assert np.all(rel <= 1e-8)
    assert np.linalg.norm(X - np.linalg.solve(A, B)) <= 1e-6 * np.linalg.norm(np.linalg.solve(A, B))


def test_block_fgmres_restarts_and_zero_columns():
    A, fa, fm, d, B = _block_problem(n=60, s=3, seed=11)
    B[:, 1] = 0.0
    X, its, rel, ok = krylov.block_fgmres(fa, fm, B, tol=1e-9, m=3)
    assert ok and its > 3                                # several cycles
    assert np.all(X[:, 1] == 0) and rel[1] == 0.0
    for i in (0, 2):
        assert np.linalg.norm(B[:, i] - A @ X[:, i]) <= 1e-9 * np.linalg.norm(B[:, i])


def test_block_arnoldi_relation_and_orthonormal_basis():
    """A Z = V H holds to rounding and V^H V = I on a problem whose Krylov vectors align
    quickly (a few dominant eigenvalues), where one classical Gram-Schmidt pass would lose
    orthogonality: the second pass and its coefficients are needed for both."""
    rng = np.random.default_rng(5)
    n, s = 120, 3
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    ev = np.concatenate([[1e4, 5e3, 2e3, 1e3], 1.0 + rng.uniform(0, 1, n - 4)])
    A = (Q * ev) @ Q.conj().T
    B = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    dg = {}
    krylov.block_fgmres(lambda v: A @ v, lambda v: v, B, tol=1e-300, m=12, maxit=12, diagnostics=dg)
    V, Z, H = dg["V"], dg["Z"], dg["H"]
    assert np.linalg.norm(V.conj().T @ V - np.eye(V.shape[1])) <= 1e-12
    rel = np.linalg.norm(A @ Z - V @ H) / np.linalg.norm(A @ Z)
    assert rel <= 1e-13, rel


# --- recycling across operators (a new frequency) -------------------------------------

def _recycled_space(n=80, k=5, seed=9):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 2 + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    _, _, _, ok, rec = krylov.gcrodr(lambda v: A @ v, lambda v: v, b, tol=1e-8, m=20, k=k)
    assert ok
    return A, rec, rng


def test_rebase_restores_the_recycling_invariants_for_a_new_operator():
    """C = A_new Ux and C^H C = I after the rebase; Ux keeps its span; rebasing on the same
    operator returns the same space."""
    A, (Ux, Uh, C), rng = _recycled_space()
    n = A.shape[0]
    A2 = A + 0.3 * np.diag(rng.uniform(0, 1, n)) + 0.05j * np.eye(n)
    Ux2, Uh2, C2 = krylov.rebase_recycle(lambda v: A2 @ v, (Ux, Uh, C))
    assert np.linalg.norm(A2 @ Ux2 - C2) <= 1e-13 * np.linalg.norm(A2)
    assert np.linalg.norm(C2.conj().T @ C2 - np.eye(C2.shape[1])) <= 1e-13
    P = Ux @ np.linalg.pinv(Ux)                          # projector on span(Ux)
    assert np.linalg.norm(P @ Ux2 - Ux2) <= 1e-10 * np.linalg.norm(Ux2)
    Ux3, Uh3, C3 = krylov.rebase_recycle(lambda v: A @ v, (Ux, Uh, C))
    assert np.linalg.norm(Ux3 - Ux) <= 1e-12 * np.linalg.norm(Ux)
    assert np.linalg.norm(C3 - C) <= 1e-12 and np.linalg.norm(Uh3 - Uh) <= 1e-12 * np.linalg.norm(Uh)


def test_rebased_space_helps_at_a_nearby_frequency():
    """Tiny configuration, GCRO-DR(20, 8): a space recycled over three sources at f carried
    to 1.03 f cuts the next source's iterations against a fresh start (11 against 14)."""
    import synth
    from oracle.solver import OracleSolver
    p = synth.tiny_problem()
    S = OracleSolver(p)
    S.factor()
    pts = np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.5, 0.5, 0.2], [0.3, 0.8, 0.6]])
    B = S.rhs(pts)
    rec = None
    for j in range(3):
        _, _, _, ok, rec = krylov.gcrodr(S.apply_A, S.apply_M, B[:, j], tol=1e-6, m=20, k=8, recycle=rec)
    S2 = OracleSolver(p)
    S2.factor(p.freq * 1.03)
    b = S2.rhs(pts)[:, 3]
    rb = krylov.rebase_recycle(S2.apply_A, rec)
    _, it_rec, rel, ok, _ = krylov.gcrodr(S2.apply_A, S2.apply_M, b, tol=1e-6, m=20, k=8, recycle=rb)
    _, it_new, _, _, _ = krylov.gcrodr(S2.apply_A, S2.apply_M, b, tol=1e-6, m=20, k=8)
    assert ok and it_rec < it_new, (it_rec, it_new)


# --- block GCRO-DR ---------------------------------------------------------------------

def _orth_block_krylov(op, R, p):
    """An orthonormal basis of the block Krylov space span[R, op R, ..., op^{p-1} R], built
    by repeated application and a full QR (independent of the Arnoldi recurrences)."""
    blocks = [np.linalg.qr(R)[0]]
    for _ in range(p - 1):
        blocks.append(np.linalg.qr(op(blocks[-1]))[0])
    return np.linalg.qr(np.hstack(blocks))[0]


def _harmonic_ritz_span(A, W, k):
    """Span of the k harmonic Ritz vectors of A over span(W) with the smallest |theta|, from
    the definition: u = W z with (A u - theta u) orthogonal to A W, i.e.
    (AW)^H (AW) z = theta (AW)^H W z."""
    import scipy.linalg as sla
    AW = A @ W
    th, Z = sla.eig(AW.conj().T @ AW, AW.conj().T @ W)
    return np.linalg.qr(W @ Z[:, np.argsort(np.abs(th))[:k]])[0]


def _same_span(Q1, U):
    Q2 = np.linalg.qr(U)[0]
    sv = np.linalg.svd(Q1.conj().T @ Q2, compute_uv=False)
    return np.abs(sv - 1.0).max()


def test_block_gcrodr_with_one_column_is_gcrodr():
    rng = np.random.default_rng(11)
    n = 100
    A = _dense(n, 12, spread=2.0)
    d = 1.0 + rng.uniform(0, 1, n)
    fa, fm = (lambda v: A @ v), (lambda v: v / d)
    r1 = r2 = None
    for _ in range(3):                                   # fresh, then two solves that recycle
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        x1, i1, _, ok1, r1 = krylov.gcrodr(fa, fm, b, tol=1e-9, m=12, k=4, recycle=r1)
        X2, i2, _, ok2, r2 = krylov.block_gcrodr(fa, fm, b[:, None], tol=1e-9, m=12, k=4, recycle=r2)
        assert ok1 and ok2 and i1 == i2
        assert np.linalg.norm(x1 - X2[:, 0]) <= 1e-12 * np.linalg.norm(x1)
        # the same recycled space (its basis is the eigenvectors' up to rounding in the
        # harmonic Ritz problem, which the two forms of the first-cycle matrix round differently)
        assert _same_span(np.linalg.qr(r1[0])[0], r2[0]) <= 1e-9
        assert _same_span(r1[2], r2[2]) <= 1e-9


def test_block_gcrodr_without_recycling_is_block_fgmres():
    A, fa, fm, d, B = _block_problem()
    X1, i1, _, ok1 = krylov.block_fgmres(fa, fm, B, tol=1e-10, m=5)
    X2, i2, _, ok2, rec = krylov.block_gcrodr(fa, fm, B, tol=1e-10, m=5, k=0)
    assert ok1 and ok2 and i1 == i2 and rec is None
    assert np.linalg.norm(X1 - X2) <= 1e-13 * np.linalg.norm(X1)


def test_block_gcrodr_first_cycle_recycles_the_block_harmonic_ritz_space():
    """One cycle of p = 4 block steps (M = I, s = 3): every column's residual is the
    minimum over the block Krylov space, and span(Ux) is that of the k harmonic Ritz
    vectors of A over the space with the smallest |theta| (the block first-cycle formula
    with H_{+} in place of h_{m+1,m}); C = A Ux, C^H C = I."""
    rng = np.random.default_rng(13)
    n, s, p, k = 70, 3, 4, 5
    A = _dense(n, 14, spread=1.5)
    B = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    X, it, rel, ok, (Ux, Uh, C) = krylov.block_gcrodr(lambda v: A @ v, lambda v: v, B, tol=1e-15, m=p, k=k,
                                                      maxit=p)
    assert it == p and Ux.shape == (n, k)
    K = _orth_block_krylov(lambda V: A @ V, B, p)
    for j in range(s):
        y = np.linalg.lstsq(A @ K, B[:, j], rcond=None)[0]
        rmin = np.linalg.norm(B[:, j] - A @ K @ y) / np.linalg.norm(B[:, j])
        assert abs(rel[j] - rmin) <= 1e-10 * rmin, (j, rel[j], rmin)
    assert _same_span(_harmonic_ritz_span(A, K, k), Ux) <= 1e-8
    assert np.linalg.norm(A @ Ux - C) <= 1e-12 * np.linalg.norm(C)
    assert np.linalg.norm(C.conj().T @ C - np.eye(k)) <= 1e-13


def test_block_gcrodr_recycled_cycle_minimises_and_updates_the_space():
    """A second block (M = I) with the first block's space: one cycle of p = m - ceil(k/s)
    block steps.  Each column's residual is the minimum over span(Ux_old) + the block
    Krylov space of (I - C C^H) A started at (I - C C^H) B; the new space is the k harmonic
    Ritz vectors of A over span[Ux_old, that Krylov space]."""
    rng = np.random.default_rng(15)
    n, s, m, k = 70, 3, 6, 5
    A = _dense(n, 16, spread=1.5)
    fa = lambda v: A @ v
    B1 = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    _, _, _, ok, rec = krylov.block_gcrodr(fa, lambda v: v, B1, tol=1e-8, m=m, k=k)
    assert ok
    Ux0, Uh0, C0 = rec
    p = m - (k + s - 1) // s
    B2 = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    X, it, rel, ok, (Ux, Uh, C) = krylov.block_gcrodr(fa, lambda v: v, B2, tol=1e-15, m=m, k=k, recycle=rec,
                                                      maxit=p)
    assert it == p
    Pc = lambda V: V - C0 @ (C0.conj().T @ V)
    K = _orth_block_krylov(lambda V: Pc(A @ V), Pc(B2), p)
    W = np.linalg.qr(np.hstack([Ux0, K]))[0]
    for j in range(s):
        y = np.linalg.lstsq(A @ W, B2[:, j], rcond=None)[0]
        rmin = np.linalg.norm(B2[:, j] - A @ W @ y) / np.linalg.norm(B2[:, j])
        assert abs(rel[j] - rmin) <= 1e-9 * rmin, (j, rel[j], rmin)
    assert _same_span(_harmonic_ritz_span(A, W, k), Ux) <= 1e-8
    assert np.linalg.norm(A @ Ux - C) <= 1e-12 * np.linalg.norm(C)
    assert np.linalg.norm(C.conj().T @ C - np.eye(k)) <= 1e-13


def test_block_gcrodr_recycling_cuts_the_next_blocks_steps():
    """Tiny configuration, three sources per block: a block that reuses the previous
    block's space needs fewer block steps than block FGMRES on it."""
    import synth
    from oracle.solver import OracleSolver
    p = synth.tiny_problem()
    S = OracleSolver(p)
    S.factor()
    ext = p.mesh.xyz.max(axis=0)
    pts = np.array([[0.2, 0.3, 0.3], [0.7, 0.2, 0.5], [0.5, 0.5, 0.2],
                    [0.3, 0.8, 0.6], [0.8, 0.7, 0.4], [0.45, 0.55, 0.75]]) * ext
    B = S.rhs(pts)
    _, it1, _, ok, rec = krylov.block_gcrodr(S.apply_A, S.apply_M, B[:, :3], tol=1e-6, m=10, k=8)
    assert ok
    X, it2, rel, ok, _ = krylov.block_gcrodr(S.apply_A, S.apply_M, B[:, 3:], tol=1e-6, m=10, k=8, recycle=rec)
    _, it_plain, _, _ = krylov.block_fgmres(S.apply_A, S.apply_M, B[:, 3:], tol=1e-6, m=10)
    assert ok and np.all(np.linalg.norm(B[:, 3:] - S.A @ X, axis=0) <= 1e-6 * np.linalg.norm(B[:, 3:], axis=0))
    assert it2 < it_plain, (it2, it_plain)
