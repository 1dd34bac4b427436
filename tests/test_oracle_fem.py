"""Pins for the oracle's discretisation (Eq. 1-2): closed forms, patch tests,
an independent quadrature and a manufactured plane wave converging at order p+1."""
import math

import numpy as np
import pytest

import synth
from oracle import fem
from tests.quad import tet_rule, tri_rule


def _jittered_cube(n, amp=0.15, seed=3):
    a = np.linspace(0.0, 1.0, n + 1)
    m = synth.kuhn_box_mesh(a, a, a)
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    interior = np.all((m.xyz > 1e-12) & (m.xyz < 1 - 1e-12), axis=1)
    m.xyz = m.xyz.copy()
    m.xyz[interior] += rng.uniform(-amp * h, amp * h, size=(interior.sum(), 3))
    return m


def test_monomial_formula_against_duffy_quadrature():
    lam, w = tet_rule(10)
    rng = np.random.default_rng(0)
    for _ in range(20):
        a = rng.integers(0, 4, size=4)
        exact = math.prod(math.factorial(int(x)) for x in a) * 6 / math.factorial(int(a.sum()) + 3)
        quad = np.sum(w * np.prod(lam ** a, axis=1))
        assert abs(exact - quad) < 1e-13
        assert abs(fem._pint({tuple(int(x) for x in a): 1.0}, 3) - exact) < 1e-15
    lam2, w2 = tri_rule(10)
    for _ in range(10):
        a = rng.integers(0, 4, size=3)
        exact = math.prod(math.factorial(int(x)) for x in a) * 2 / math.factorial(int(a.sum()) + 2)
        assert abs(np.sum(w2 * np.prod(lam2 ** a, axis=1)) - exact) < 1e-13
        assert abs(fem._pint({tuple(int(x) for x in a): 1.0}, 2) - exact) < 1e-15


def test_p2_tet_mass_matches_textbook_420_matrix():
    # Classical P2 tetrahedron mass matrix, |T|/420 times: vertex diagonal 6,
    # vertex-vertex 1, vertex / edge through it -4, vertex / edge not through it -6,
    # edge diagonal 32, edges sharing a vertex 16, opposite edges 8.
    Mref, _ = fem.reference_tensors(2)
    edges = fem.TET_EDGES
    T = np.zeros((10, 10))
    for a in range(10):
        for b in range(10):
            if a < 4 and b < 4:
                T[a, b] = 6 if a == b else 1
            elif a < 4 or b < 4:
                v, e = (a, b - 4) if a < 4 else (b, a - 4)
                T[a, b] = -4 if v in edges[e] else -6
            else:
                ea, eb = edges[a - 4], edges[b - 4]
                T[a, b] = 32 if a == b else (16 if set(ea) & set(eb) else 8)
    assert np.allclose(Mref, T / 420.0, atol=1e-15, rtol=0)


def test_p1_matrices_closed_form():
    Mref, _ = fem.reference_tensors(1)
    assert np.allclose(Mref, (np.ones((4, 4)) + np.eye(4)) / 20.0)
    rng = np.random.default_rng(1)
    xyz = rng.standard_normal((4, 3))
    tets = np.array([[0, 1, 2, 3]])
    Ke, Me = fem.element_matrices(xyz, tets, 1)
    vol, g = fem.tet_geometry(xyz, tets)
    assert abs(vol[0] - abs(np.linalg.det(np.stack([xyz[1] - xyz[0], xyz[2] - xyz[0], xyz[3] - xyz[0]]))) / 6) < 1e-14
    # grad lambda from the inverse of the affine map, independent of the oracle
    P = np.hstack([np.ones((4, 1)), xyz])
    grads = np.linalg.inv(P)[1:].T                  # row a = grad lambda_a
    assert np.allclose(Ke[0], vol[0] * grads @ grads.T, atol=1e-13)


def test_p2_triangle_face_mass_textbook():
    # P2 triangle mass, |F|/180: vertex diag 6, vertex-vertex -1, vertex/opposite edge -4,
    # vertex/adjacent edge 0, edge diag 32, edge-edge 16.
    M = fem.face_reference_mass(2)
    edges = fem.TRI_EDGES
    T = np.zeros((6, 6))
    for a in range(6):
        for b in range(6):
            if a < 3 and b < 3:
                T[a, b] = 6 if a == b else -1
            elif a < 3 or b < 3:
                v, e = (a, b - 3) if a < 3 else (b, a - 3)
                T[a, b] = 0 if v in edges[e] else -4
            else:
                T[a, b] = 32 if a == b else 16
    assert np.allclose(M, T / 180.0, atol=1e-15)


@pytest.mark.parametrize("order", [1, 2])
def test_element_matrices_against_quadrature(order):
    """Element K and M on a random tet against Duffy quadrature of the Lagrange basis
    evaluated from its nodal definition (Vandermonde inverse), not from the oracle."""
    rng = np.random.default_rng(2)
    xyz = rng.standard_normal((4, 3))
    tets = np.array([[0, 1, 2, 3]])
    Ke, Me = fem.element_matrices(xyz, tets, order)
    # nodes of the element and a monomial basis in x,y,z
    nodes = xyz.copy() if order == 1 else np.vstack(
        [xyz] + [0.5 * (xyz[i] + xyz[j]) for (i, j) in fem.TET_EDGES])
    exps = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if order == 2:
        exps += [(2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]
    V = np.array([[np.prod(p ** np.array(e)) for e in exps] for p in nodes])
    C = np.linalg.inv(V)                            # column a: coefficients of phi_a
    lam, w = tet_rule(6)
    pts = lam @ xyz
    vol = abs(np.linalg.det(np.stack([xyz[1] - xyz[0], xyz[2] - xyz[0], xyz[3] - xyz[0]]))) / 6
    Phi = np.array([[np.prod(p ** np.array(e)) for e in exps] for p in pts]) @ C
    dPhi = []
    for ax in range(3):
        cols = []
        for e in exps:
            e = np.array(e)
            if e[ax] == 0:
                cols.append(np.zeros(len(pts)))
            else:
                e2 = e.copy(); e2[ax] -= 1
                cols.append(e[ax] * np.prod(pts ** e2, axis=1))
        dPhi.append(np.stack(cols, axis=1) @ C)
    Mq = vol * np.einsum("q,qa,qb->ab", w, Phi, Phi)
    Kq = vol * sum(np.einsum("q,qa,qb->ab", w, d, d) for d in dPhi)
    assert np.allclose(Me[0], Mq, atol=1e-12)
    assert np.allclose(Ke[0], Kq, atol=1e-11)


@pytest.mark.parametrize("order", [1, 2])
def test_patch_tests_on_jittered_mesh(order):
    """K annihilates constants; for P2, (K q)_a = -Lap(q) int phi_a at interior dofs
    for any quadratic q (integration by parts), and sum(M) = volume."""
    m = _jittered_cube(4)
    ne = m.tets.shape[0]
    dm, K, Mp, Bp = fem.assemble_parts(m, np.ones(ne, np.complex128), order)
    one = np.ones(dm.n)
    assert np.abs(K @ one).max() < 1e-12
    assert abs((Mp @ one).sum().real - 1.0) < 1e-12
    X = dm.coords()
    lin = 1.0 + 2 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2]
    interior = np.ones(dm.n, bool)
    bnd = np.unique(dm.face_dofs(m.faces).ravel())
    interior[bnd] = False
    assert np.abs((K @ lin)[interior]).max() < 1e-12
    if order == 2:
        q = X[:, 0] ** 2 + 3 * X[:, 1] * X[:, 2] - 0.5 * X[:, 2] ** 2 + X[:, 0] * X[:, 1]
        lap = 2.0 - 1.0
        mass_rows = (Mp @ one).real
        assert np.abs((K @ q)[interior] + lap * mass_rows[interior]).max() < 1e-12


def _l2_error(mesh, dm, order, uh, k, d):
    lam, w = tet_rule(6)
    vol, _ = fem.tet_geometry(mesh.xyz, mesh.tets)
    phi = fem.eval_basis(order, lam)                 # (q, nb)
    pts = np.einsum("qa,eai->eqi", lam, mesh.xyz[mesh.tets])
    uex = np.exp(1j * k * (pts @ d))
    uq = np.einsum("qa,ea->eq", phi, uh[dm.elem_dofs])
    err = np.sum(vol[:, None] * w[None] * np.abs(uq - uex) ** 2)
    return math.sqrt(err)


@pytest.mark.parametrize("order,slope", [(1, 1.8), (2, 2.8)])
def test_plane_wave_manufactured_solution_converges(order, slope):
    k = 4.0 + 0.1j
    d = np.array([0.3, 0.5, 0.8]); d /= np.linalg.norm(d)
    errs, hs = [], []
    for n in ([4, 8, 16] if order == 1 else [2, 4, 8]):
        a = np.linspace(0.0, 1.0, n + 1)
        m = synth.kuhn_box_mesh(a, a, a)
        uh, dm = fem.plane_wave_solve(m, order, k, d)
        errs.append(_l2_error(m, dm, order, uh, k, d))
        hs.append(1.0 / n)
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert rates[-1] >= slope, (errs, rates)


def test_assembled_matrix_is_complex_symmetric_and_dirichlet_identity():
    p = synth.small_overthrust(levels=1, cells=(3, 3, 2), freq=0.8, nsub=2)
    A, dm, dd = fem.global_system(p)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()   # up to summation order
    assert np.iscomplexobj(A.data)
    sub = A[dd][:, dd].toarray()
    assert np.array_equal(sub, np.eye(len(dd)))
    rest = np.setdiff1d(np.arange(dm.n), dd)
    assert abs(A[dd][:, rest]).max() == 0.0


def test_point_source_at_vertex_is_unit_vector():
    p = synth.tiny_problem()
    A, dm, dd = fem.global_system(p)
    b = fem.point_sources(p, dm, dd, p.sources)[:, 0]
    v = 6 + 13 * (6 + 13 * 6)
    e = np.zeros(dm.n); e[v] = -1.0
    assert np.allclose(b, e, atol=1e-14)


@pytest.mark.parametrize("make", [
    lambda: synth.unit_cube_problem(n=5, order=2, nsub=4, overlap=1, freq=1.5),
    lambda: synth.small_overthrust(levels=2, cells=(4, 4, 2), freq=0.5, nsub=8),
    lambda: synth.unit_cube_problem(n=6, order=1, nsub=4, overlap=1, freq=1.2),
], ids=["cube_p2", "overthrust_p2", "cube_p1"])
def test_sampled_rows_equal_rows_of_the_global_system(make):
    """Rows assembled from only the elements and absorbing faces holding their dof are the
    rows of the whole assembly: Dirichlet rows, absorbing-boundary rows, vertex and edge
    dofs, interior rows, and an unsorted sample with a repeated row."""
    p = make()
    A, dm, dd = fem.global_system(p)
    B = fem.global_system(p, freq=0.8 * p.freq)[0]
    abc = p.mesh.faces[p.mesh.face_tag == fem.TAG_ABC]
    on_abc = np.setdiff1d(np.unique(dm.face_dofs(abc).ravel()), dd)
    rng = np.random.default_rng(4)
    rows = np.concatenate([dd[:5], on_abc[:7], rng.choice(dm.n, 40, replace=False), [dm.n - 1, 0, 0]])
    assert len(dd) and len(on_abc) and (p.order == 1 or dm.n - 1 >= dm.nv)   # every kind of row
    R, dm2, dd2 = fem.sampled_rows(p, rows)
    assert np.array_equal(dd2, dd)
    ref = A[rows].toarray()
    got = R.toarray()
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    assert np.array_equal(got != 0, ref != 0)                        # same sparsity, no dropped term
    Rf = fem.sampled_rows(p, rows, freq=0.8 * p.freq, dm=dm)[0].toarray()
    assert np.abs(Rf - B[rows].toarray()).max() <= 1e-14 * np.abs(ref).max()
