"""Pins for the oracle's coarse space (Eq. 3): exact reproduction of coarse
quadratics by Z, E complex symmetric, coarse = fine gives one iteration."""
import numpy as np
import scipy.sparse as sp

import synth
from oracle import coarse, fem
from oracle.solver import OracleSolver


def test_interpolation_reproduces_coarse_quadratics():
    p = synth.small_overthrust(levels=2, cells=(3, 3, 2), freq=0.8, nsub=2)
    A, dm, dd = fem.global_system(p)
    Z, cdm, keep = coarse.interpolation(p, dm)
    # q vanishes on the top face z = 0, so it lies in the constrained coarse space
    def q(X):
        return X[:, 2] * (1.0 + 0.3 * X[:, 0] - 0.2 * X[:, 1] + 0.5 * X[:, 2])
    qH = q(cdm.coords())[keep]
    qh = q(dm.coords())
    assert np.abs(Z @ qH - qh).max() <= 1e-12 * np.abs(qh).max()
    assert Z.shape == (dm.n, len(keep))
    assert np.all(np.isreal(Z.data))


def test_coarse_operator_complex_symmetric():
    p = synth.small_overthrust(levels=2, cells=(3, 3, 2), freq=0.8, nsub=2)
    A, dm, dd = fem.global_system(p)
    Z, _, _ = coarse.interpolation(p, dm)
    E = coarse.coarse_operator(Z, A)
    assert abs(E - E.T).max() <= 1e-13 * abs(E).max()


def test_coarse_equal_fine_gives_one_iteration():
    """With Gamma_H = Gamma, Z is the identity on free dofs and M^{-1} = A^{-1}."""
    p = synth.unit_cube_problem(n=6, nsub=8, overlap=1)
    p.levels = 2
    p.coarse = p.mesh
    p.fine_parent = np.arange(p.mesh.tets.shape[0], dtype=np.int32)
    S = OracleSolver(p)
    free = np.setdiff1d(np.arange(S.n), S.ddofs)
    assert (S.Z - sp.eye(S.n, format="csr")[:, free]).count_nonzero() == 0
    S.factor()
    x, it, rel, ok = S.solve(S.rhs()[:, 0])
    assert ok and it == 1


def test_two_level_beats_one_level_when_coarse_mesh_resolves_the_wave():
    its = {}
    for levels in (1, 2):
        p = synth.small_overthrust(levels=levels, cells=(4, 4, 2), freq=0.5, nsub=16)
        S = OracleSolver(p)
        S.factor()
        _, it, rel, ok = S.solve(S.rhs()[:, 0])
        assert ok
        its[levels] = it
    assert its[2] < its[1], its


# --- the paper's coarse solve: inner GMRES with one-level ORAS on the coarse mesh ---

def _coarse_setup(nsub=4, cells=(4, 4, 2), freq=0.5, part=None):
    p = synth.small_overthrust(levels=2, cells=cells, freq=freq, nsub=nsub)
    if part is not None:
        p.elem_part = part(p)
    S = OracleSolver(p, coarse_solver="oras", coarse_tol=1e-12, coarse_m=60)
    return p, S


def test_coarse_partition_recovers_an_induced_partition():
    rng = np.random.default_rng(4)
    p = synth.small_overthrust(levels=2, cells=(4, 4, 2), freq=0.5, nsub=5)
    truth = rng.integers(0, 5, p.coarse.tets.shape[0])
    p.elem_part = truth[p.fine_parent].astype(np.int32)
    assert np.array_equal(coarse.coarse_partition(p), truth)


def test_coarse_partition_of_unity_sums_to_one():
    p, S = _coarse_setup()
    tot = np.zeros(S.cor.nH)
    for dofs, D in zip(S.cor.dofs, S.cor.D):
        np.add.at(tot, dofs, D)
    assert np.abs(tot - 1.0).max() <= 1e-14


def test_one_coarse_subdomain_local_operator_is_E():
    p, S = _coarse_setup(nsub=1)
    S.factor()
    E1 = S.cor.E_loc[0]
    assert np.array_equal(S.cor.dofs[0], np.arange(S.cor.nH))
    assert abs(E1 - S.E).max() <= 1e-13 * abs(S.E).max()


def test_local_coarse_rows_inside_a_subdomain_equal_rows_of_E():
    """A coarse dof whose every coarse element lies in Gamma_H,i has a basis function
    supported inside the subdomain and off its artificial interface: its row of E_i is
    its row of E (a wrong region, a misplaced absorbing term or a transposed operand
    breaks this)."""
    p, S = _coarse_setup(nsub=4)
    S.factor()
    cdm = S.cdm
    newid = np.full(cdm.n, -1, np.int64)
    newid[S.ckeep] = np.arange(len(S.ckeep))
    part = coarse.coarse_partition(p)
    checked = 0
    for i, (dofs, Ei) in enumerate(zip(S.cor.dofs, S.cor.E_loc)):
        reg = S.cor.regions[i]
        elems = np.unique(p.fine_parent[reg])                  # Gamma_H,i
        inside = np.zeros(p.coarse.tets.shape[0], bool)
        inside[elems] = True
        bad = np.zeros(cdm.n, bool)                           # dofs of elements outside
        bad[np.unique(cdm.elem_dofs[~inside].ravel())] = True
        interior = np.nonzero(~bad[S.ckeep])[0]               # free ids, support inside
        loc = np.full(S.cor.nH, -1, np.int64)
        loc[dofs] = np.arange(len(dofs))
        rows = interior[loc[interior] >= 0]
        Er = S.E[rows][:, dofs].toarray()
        El = Ei.tocsr()[loc[rows]].toarray()
        assert np.abs(El - Er).max() <= 1e-12 * abs(S.E).max()
        checked += len(rows)
        assert abs(Ei - Ei.T).max() <= 1e-13 * abs(Ei).max()
    assert checked > 0


def test_single_coarse_subdomain_inner_solve_is_exact_in_one_iteration():
    p, S = _coarse_setup(nsub=1)
    S.factor()
    D = OracleSolver(p)
    D.factor()
    v = np.random.default_rng(2).standard_normal(S.n) + 0j
    y = S.coarse_correction(v)
    assert S.coarse_its[-1] == 1
    yd = D.coarse_correction(v)
    assert np.linalg.norm(y - yd) <= 1e-12 * np.linalg.norm(yd)


def test_tight_inner_tolerance_reproduces_the_direct_coarse_solve():
    p, S = _coarse_setup(nsub=8)
    S.factor()
    D = OracleSolver(p)
    D.factor()
    b = D.rhs()[:, 0]
    xd, itd, _, okd = D.solve(b)
    xs, its, _, oks = S.solve(b)
    assert okd and oks and abs(its - itd) <= 1
    assert np.linalg.norm(xs - xd) <= 1e-9 * np.linalg.norm(xd)
    # looser inner tolerances: fewer inner iterations, still a convergent outer solve
    prev = None
    for tolH in (1e-8, 1e-4, 1e-1):
        T = OracleSolver(p, coarse_solver="oras", coarse_tol=tolH, coarse_m=60)
        T.factor()
        x, it, rel, ok = T.solve(b)
        assert ok and rel <= p.tol
        m = max(T.coarse_its)
        assert prev is None or m <= prev
        prev = m


def test_local_coarse_operators_equal_direct_coarse_assembly_in_a_homogeneous_medium():
    """In a homogeneous medium the Galerkin projection Z_i^T A_i^h Z_i of the fine
    Robin problem equals the same Robin problem assembled directly on the coarse
    mesh (nested P2 spaces, exact integrals): a second route to every E_i, through
    the coarse elements and coarse interface faces instead of the fine ones."""
    from oracle import dd
    p = synth.unit_cube_problem(n=8, freq=1.0, order=2, nsub=4, overlap=1, levels=2)
    S = OracleSolver(p, coarse_solver="oras")
    S.factor()
    cm = p.coarse
    cc = np.full(cm.tets.shape[0], p.c[0])
    subs = dd.grow_subdomains(cm, S.cor.part, p.nsub, p.overlap, S.cdm)
    w = 2 * np.pi * p.freq
    newid = np.full(S.cdm.n, -1, np.int64)
    newid[S.ckeep] = np.arange(len(S.ckeep))
    for i, s in enumerate(subs):
        K, Mp, Bp = dd.local_parts(cm, cc, p.order, S.cdm, s)
        Ad = (K.astype(np.complex128) - w * w * Mp - 1j * w * Bp).tocsr()
        full = s.dofs[newid[s.dofs] >= 0]
        Ed = Ad[full][:, full]
        assert np.array_equal(newid[full], S.cor.dofs[i])
        assert abs(Ed - S.cor.E_loc[i]).max() <= 1e-12 * abs(Ed).max()
