"""Oracle: finite-element discretisation of the Helmholtz problem, Eq. (1)-(2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Problem (Eq. 1): (Delta + k^2(x)) u = b in Omega, k = omega / c(x), c complex
in attenuating media; first-order absorbing conditions on the four vertical
faces and the bottom, homogeneous Dirichlet on the top face (Section
"Iterative solver ...", and the experiments section).

Reading used for the signs (time dependence e^{-i omega t}): the outgoing
absorbing condition is d_n u - i k u = 0, so the weak form of Eq. (1) gives

    A = K - M_{k^2} - i B_k,     rhs = -F,   F_a = int b phi_a,

with K_ab = int grad phi_a . grad phi_b, (M_{k^2})_ab = int k^2 phi_a phi_b and
(B_k)_ab = int_{absorbing faces} k phi_a phi_b (k of the element owning the
face).  Because c is constant per element, A = K - omega^2 M' - i omega B' with
M' = int c^{-2} phi phi and B' = int_{ABC} c^{-1} phi phi.

Integrals are exact: every integrand is a polynomial in barycentric
coordinates, integrated with  int_T lambda^alpha = alpha! d! |T| / (|alpha|+d)!
(d = 3 on tets, 2 on faces).  No quadrature tables.

Dof numbering (shared convention with the CUDA library, an interface, not
code): vertex dofs are the mesh vertices in input order; P2 edge dofs follow,
one per mesh edge, edges sorted by (smaller vertex id, larger vertex id).
Local node order on a tet is v0..v3, e01, e02, e03, e12, e13, e23; on a face
v0..v2, e01, e02, e12.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

TAG_DIRICHLET = 0
TAG_ABC = 1

TET_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
TRI_EDGES = [(0, 1), (0, 2), (1, 2)]


# ---------------------------------------------------------------------------
# Polynomials in barycentric coordinates: {exponent tuple: coefficient}
# ---------------------------------------------------------------------------

def _pmul(p, q):
    out = {}
    for a, ca in p.items():
        for b, cb in q.items():
            e = tuple(x + y for x, y in zip(a, b))
            out[e] = out.get(e, 0.0) + ca * cb
    return out


def _pderiv(p, var):
    out = {}
    for a, ca in p.items():
        if a[var] > 0:
            e = list(a)
            e[var] -= 1
            e = tuple(e)
            out[e] = out.get(e, 0.0) + ca * a[var]
    return out


def _pint(p, d):
    """Integral over the simplex of dimension d divided by its measure."""
    s = 0.0
    for a, ca in p.items():
        num = math.prod(math.factorial(x) for x in a) * math.factorial(d)
        s += ca * num / math.factorial(sum(a) + d)
    return s


def _basis(order, nvert):
    """Lagrange basis on a simplex with ``nvert`` vertices as polynomials in lambda."""
    def mono(*idx):
        e = [0] * nvert
        for i in idx:
            e[i] += 1
        return tuple(e)

    if order == 1:
        return [{mono(i): 1.0} for i in range(nvert)]
    edges = TET_EDGES if nvert == 4 else TRI_EDGES
    out = [{mono(i, i): 2.0, mono(i): -1.0} for i in range(nvert)]
    out += [{mono(i, j): 4.0} for (i, j) in edges]
    return out


@lru_cache(maxsize=None)
def reference_tensors(order):
    """(Mref, Sref): Mref[a,b] = int phi_a phi_b / |T|,
    Sref[a,b,p,q] = int (d phi_a / d lambda_p)(d phi_b / d lambda_q) / |T|."""
    B = _basis(order, 4)
    nb = len(B)
    Mref = np.zeros((nb, nb))
    Sref = np.zeros((nb, nb, 4, 4))
    dB = [[_pderiv(b, p) for p in range(4)] for b in B]
    for a in range(nb):
        for b in range(nb):
            Mref[a, b] = _pint(_pmul(B[a], B[b]), 3)
            for p in range(4):
                for q in range(4):
                    Sref[a, b, p, q] = _pint(_pmul(dB[a][p], dB[b][q]), 3)
    return Mref, Sref


@lru_cache(maxsize=None)
def face_reference_mass(order):
    B = _basis(order, 3)
    nb = len(B)
    M = np.zeros((nb, nb))
    for a in range(nb):
        for b in range(nb):
            M[a, b] = _pint(_pmul(B[a], B[b]), 2)
    return M


def eval_basis(order, lam):
    """Values of the tet basis at barycentric points lam (..., 4)."""
    lam = np.asarray(lam, np.float64)
    if order == 1:
        return lam.copy()
    vals = [lam[..., i] * (2 * lam[..., i] - 1) for i in range(4)]
    vals += [4 * lam[..., i] * lam[..., j] for (i, j) in TET_EDGES]
    return np.stack(vals, axis=-1)


# ---------------------------------------------------------------------------
# Geometry
# ---------------------------------------------------------------------------

def tet_geometry(xyz, tets):
    """Volumes |T| (ne,) and barycentric gradients grad lambda (ne, 4, 3)."""
    v = xyz[tets]
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)  # columns
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)                       # rows are grad lambda_1..3
    g = np.empty((len(tets), 4, 3))
    g[:, 1:] = Jinv
    g[:, 0] = -Jinv.sum(axis=1)
    return np.abs(det) / 6.0, g


def tri_area(xyz, tri):
    v = xyz[tri]
    return 0.5 * np.linalg.norm(np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), axis=1)


def barycentric(xyz, tet, pts):
    """Barycentric coordinates of pts (k,3) in each tet of ``tet`` (k,4)."""
    v = xyz[tet]
    J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
    l = np.linalg.solve(J, (pts - v[:, 0])[..., None])[..., 0]
    return np.concatenate([1.0 - l.sum(axis=1, keepdims=True), l], axis=1)


# ---------------------------------------------------------------------------
# Dofs
# ---------------------------------------------------------------------------

class DofMap:
    """Global dof numbering for P1 or P2 on a tet mesh (see module docstring)."""

    def __init__(self, xyz, tets, order):
        self.order = order
        self.nv = nv = xyz.shape[0]
        self.xyz = xyz
        self.tets = tets
        if order == 1:
            self.edges = np.zeros((0, 2), np.int64)
            self.elem_dofs = tets.astype(np.int64)
        else:
            e = np.stack([tets[:, [i, j]] for (i, j) in TET_EDGES], axis=1).reshape(-1, 2)
            e = np.sort(e, axis=1).astype(np.int64)
            key = e[:, 0] * nv + e[:, 1]
            ukey, inv = np.unique(key, return_inverse=True)
            self.edge_keys = ukey
            self.edges = np.stack([ukey // nv, ukey % nv], axis=1)
            self.elem_dofs = np.concatenate(
                [tets.astype(np.int64), nv + inv.reshape(-1, 6)], axis=1)
        self.n = nv + len(self.edges)

    def edge_id(self, a, b):
        a = np.asarray(a, np.int64)
        b = np.asarray(b, np.int64)
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        k = lo * self.nv + hi
        idx = np.searchsorted(self.edge_keys, k)
        assert np.all(self.edge_keys[idx] == k)
        return idx

    def face_dofs(self, faces):
        faces = faces.astype(np.int64)
        if self.order == 1:
            return faces
        ed = [self.nv + self.edge_id(faces[:, i], faces[:, j]) for (i, j) in TRI_EDGES]
        return np.concatenate([faces, np.stack(ed, axis=1)], axis=1)

    def coords(self):
        """Node coordinate of every dof (vertex or edge midpoint)."""
        if self.order == 1:
            return self.xyz.copy()
        mid = 0.5 * (self.xyz[self.edges[:, 0]] + self.xyz[self.edges[:, 1]])
        return np.concatenate([self.xyz, mid], axis=0)

    def dirichlet_dofs(self, faces, face_tag):
        top = faces[face_tag == TAG_DIRICHLET]
        if len(top) == 0:
            return np.zeros(0, np.int64)
        return np.unique(self.face_dofs(top).ravel())


def face_owner(tets, faces):
    """Index of the (unique) tet having each boundary face."""
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    tf = np.sort(tets[:, loc].reshape(-1, 3).astype(np.int64), axis=1)
    nv = int(tets.max()) + 1
    key = (tf[:, 0] * nv + tf[:, 1]) * nv + tf[:, 2]
    order = np.argsort(key, kind="stable")
    fs = np.sort(faces.astype(np.int64), axis=1)
    fk = (fs[:, 0] * nv + fs[:, 1]) * nv + fs[:, 2]
    pos = np.searchsorted(key[order], fk)
    assert np.all(key[order][pos] == fk)
    return order[pos] // 4


# ---------------------------------------------------------------------------
# Assembly
# ---------------------------------------------------------------------------

def element_matrices(xyz, tets, order):
    """Per-element stiffness K_e and unit-coefficient mass M_e, exact."""
    vol, g = tet_geometry(xyz, tets)
    Mref, Sref = reference_tensors(order)
    G = np.einsum("epi,eqi->epq", g, g)
    Ke = vol[:, None, None] * np.einsum("epq,abpq->eab", G, Sref)
    Me = vol[:, None, None] * Mref[None]
    return Ke, Me


def face_matrices(xyz, faces, order):
    area = tri_area(xyz, faces)
    return area[:, None, None] * face_reference_mass(order)[None]


def _coo(n, dofs, mats):
    nb = dofs.shape[1]
    r = np.repeat(dofs, nb, axis=1).ravel()
    c = np.tile(dofs, (1, nb)).ravel()
    return sp.coo_matrix((mats.ravel(), (r, c)), shape=(n, n)).tocsr()


def assemble_parts(mesh, c, order, elems=None, faces=None, face_coef_elem=None, dm=None):
    """Frequency-independent pieces (K, M', B') over a subset of elements.

    ``faces``/``face_coef_elem``: the boundary faces carrying the absorbing
    term and the element whose c weights each one.  Defaults: the global mesh
    with its ABC faces.
    """
    if dm is None:
        dm = DofMap(mesh.xyz, mesh.tets, order)
    if elems is None:
        elems = np.arange(mesh.tets.shape[0])
    Ke, Me = element_matrices(mesh.xyz, mesh.tets[elems], order)
    ed = dm.elem_dofs[elems]
    K = _coo(dm.n, ed, Ke)
    Mp = _coo(dm.n, ed, Me * (1.0 / c[elems] ** 2)[:, None, None])
    if faces is None:
        sel = mesh.face_tag == TAG_ABC
        faces = mesh.faces[sel]
        face_coef_elem = face_owner(mesh.tets, faces)
    if len(faces):
        Fe = face_matrices(mesh.xyz, faces, order)
        Bp = _coo(dm.n, dm.face_dofs(faces), Fe * (1.0 / c[face_coef_elem])[:, None, None])
    else:
        Bp = sp.csr_matrix((dm.n, dm.n), dtype=np.complex128)
    return dm, K, Mp, Bp


def helmholtz_matrix(K, Mp, Bp, freq):
    """A(omega) = K - omega^2 M' - i omega B', omega = 2 pi f (before Dirichlet)."""
    w = 2.0 * np.pi * freq
    return (K.astype(np.complex128) - (w * w) * Mp - (1j * w) * Bp).tocsr()


def apply_dirichlet(A, ddofs):
    """Symmetric elimination: rows and columns of ``ddofs`` become identity."""
    n = A.shape[0]
    keep = np.ones(n)
    keep[ddofs] = 0.0
    P = sp.diags(keep)
    I = sp.diags(1.0 - keep)
    out = (P @ A @ P + I).tocsr()
    out.eliminate_zeros()
    out.sort_indices()
    return out


def global_system(problem, freq=None):
    """Assembled global A (complex symmetric, Dirichlet rows identity) and DofMap."""
    freq = problem.freq if freq is None else freq
    dm, K, Mp, Bp = assemble_parts(problem.mesh, problem.c, problem.order)
    A = helmholtz_matrix(K, Mp, Bp, freq)
    dd = dm.dirichlet_dofs(problem.mesh.faces, problem.mesh.face_tag)
    return apply_dirichlet(A, dd), dm, dd


def sampled_rows(problem, rows, freq=None, dm=None):
    """Rows ``rows`` of the assembled global A of ``global_system`` (Eq. 1-2, after the
    symmetric Dirichlet elimination), for problems too large to assemble whole.

    Row i of the assembled matrix is the sum of the element terms of the elements whose
    dof lists hold i and of the absorbing-face terms of the faces whose dof lists hold
    i; no other term touches it.  So the assembly is restricted to exactly those
    elements and faces, and the requested rows are read off.  The owner of such a face
    holds the face, hence dof i, so it is among the kept elements.  The elimination then
    zeroes the Dirichlet columns of every row and turns Dirichlet rows into identity
    rows, as ``apply_dirichlet`` does for the whole matrix.

    Returns (rows of A as CSR, shape (len(rows), n), the DofMap, the Dirichlet dofs).
    """
    freq = problem.freq if freq is None else freq
    mesh = problem.mesh
    if dm is None:
        dm = DofMap(mesh.xyz, mesh.tets, problem.order)
    rows = np.asarray(rows, np.int64)
    want = np.zeros(dm.n, bool)
    want[rows] = True
    elems = np.nonzero(want[dm.elem_dofs].any(axis=1))[0]
    abc = mesh.faces[mesh.face_tag == TAG_ABC]
    if len(abc):
        abc = abc[want[dm.face_dofs(abc)].any(axis=1)]
    owner = elems[face_owner(mesh.tets[elems], abc)] if len(abc) else np.zeros(0, np.int64)
    _, K, Mp, Bp = assemble_parts(mesh, problem.c, problem.order, elems=elems, faces=abc,
                                  face_coef_elem=owner, dm=dm)
    A = helmholtz_matrix(K, Mp, Bp, freq)[rows]
    dd = dm.dirichlet_dofs(mesh.faces, mesh.face_tag)
    keep = np.ones(dm.n)
    keep[dd] = 0.0
    ident = sp.coo_matrix((1.0 - keep[rows], (np.arange(len(rows)), rows)), shape=A.shape)
    out = (sp.diags(keep[rows]) @ A @ sp.diags(keep) + ident).tocsr()
    out.eliminate_zeros()
    out.sort_indices()
    return out, dm, dd


def locate(xyz, tets, pts):
    """For each point, the lowest-index tet that contains it and its barycentrics."""
    out_e = np.empty(len(pts), np.int64)
    out_l = np.empty((len(pts), 4))
    vmin = xyz[tets].min(axis=1)
    vmax = xyz[tets].max(axis=1)
    for k, p in enumerate(np.asarray(pts, np.float64)):
        cand = np.nonzero(np.all((vmin <= p + 1e-12) & (vmax >= p - 1e-12), axis=1))[0]
        lam = barycentric(xyz, tets[cand], np.repeat(p[None], len(cand), 0))
        ok = np.nonzero(lam.min(axis=1) >= -1e-12)[0]
        assert len(ok), f"point {p} outside the mesh"
        out_e[k] = cand[ok[0]]
        out_l[k] = lam[ok[0]]
    return out_e, out_l


def point_sources(problem, dm, ddofs, pts):
    """rhs columns b_j = -F_j with F_j,a = phi_a(x_s) (Eq. 1 sign), zero on Dirichlet dofs."""
    e, lam = locate(problem.mesh.xyz, problem.mesh.tets, pts)
    vals = eval_basis(problem.order, lam)
    B = np.zeros((dm.n, len(pts)), np.complex128)
    for j in range(len(pts)):
        np.add.at(B[:, j], dm.elem_dofs[e[j]], -vals[j])
    B[ddofs, :] = 0.0
    return B


# ---------------------------------------------------------------------------
# Oracle-only inhomogeneous path: plane-wave manufactured solution
# ---------------------------------------------------------------------------

def outward_normals(xyz, tets, faces):
    owner = face_owner(tets, faces)
    v = xyz[faces]
    nrm = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    opp = xyz[tets[owner]].sum(axis=1) - v.sum(axis=1)     # the owner's fourth vertex
    sgn = np.sign(np.einsum("fi,fi->f", opp - v[:, 0], nrm))
    return -sgn[:, None] * nrm


def plane_wave_solve(mesh, order, k, d):
    """FE solution of (Delta + k^2) u = 0 with u = exp(i k d.x) on the Dirichlet top
    and d_n u - i k u = g := i k (d.n - 1) u on the absorbing faces.

    Homogeneous medium: c = 1/k at omega = 1.  The Robin datum enters as
    int_F g phi_a with g replaced by its Lagrange interpolant on the face.
    Returns (u_h, DofMap).
    """
    d = np.asarray(d, np.float64) / np.linalg.norm(d)
    ne = mesh.tets.shape[0]
    c = np.full(ne, 1.0 / k, np.complex128)
    dm, K, Mp, Bp = assemble_parts(mesh, c, order)
    A = helmholtz_matrix(K, Mp, Bp, 1.0 / (2.0 * np.pi))
    X = dm.coords()
    uex = np.exp(1j * k * (X @ d))
    abc = mesh.faces[mesh.face_tag == TAG_ABC]
    nrm = outward_normals(mesh.xyz, mesh.tets, abc)
    fd = dm.face_dofs(abc)
    g = 1j * k * ((nrm @ d)[:, None] - 1.0) * uex[fd]          # nodal values per face
    Fm = face_matrices(mesh.xyz, abc, order)
    rhs = np.zeros(dm.n, np.complex128)
    np.add.at(rhs, fd.ravel(), np.einsum("fab,fb->fa", Fm, g).ravel())
    dd = dm.dirichlet_dofs(mesh.faces, mesh.face_tag)
    ud = np.zeros(dm.n, np.complex128)
    ud[dd] = uex[dd]
    rhs = rhs - A @ ud
    rhs[dd] = ud[dd]
    Ad = apply_dirichlet(A, dd)
    import scipy.sparse.linalg as spla
    return spla.spsolve(Ad.tocsc(), rhs), dm
