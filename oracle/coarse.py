"""Oracle: coarse space of the two-level preconditioner, Eq. (3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (3): M^{-1} = M_1^{-1} (I - A Q) + Q, Q = Z E^{-1} Z^T, E = Z^T A Z, where
Z^T is the interpolation between the finite-element space on the fine mesh
Gamma and the one on a coarse mesh Gamma_H.

Readings: Gamma is one uniform refinement of Gamma_H (so the coarse space is
nested in the fine one and Z is *exact* Lagrange interpolation of the coarse
basis at the fine nodes, an n x n_H real matrix); the coarse space carries the
same element order and the same homogeneous Dirichlet condition on the top
face (coarse top dofs are removed, so Z maps into the constrained fine space);
Z^T is the plain transpose and E uses the transpose, not the conjugate
transpose, so E stays complex symmetric.  Exact interpolation weights are
dyadic rationals; entries below 1e-12 are rounding noise and are dropped.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dd, fem, krylov


def interpolation(problem, dm):
    """Z (csr, real, n x n_H) and the coarse DofMap / kept coarse dof ids."""
    cm = problem.coarse
    cdm = fem.DofMap(cm.xyz, cm.tets, problem.order)
    cdir = cdm.dirichlet_dofs(cm.faces, cm.face_tag)
    keep = np.ones(cdm.n, bool)
    keep[cdir] = False
    newid = np.full(cdm.n, -1, np.int64)
    newid[keep] = np.arange(keep.sum())

    # one fine element per fine dof (lowest element index listing it)
    ne = dm.elem_dofs.shape[0]
    nb = dm.elem_dofs.shape[1]
    flat = dm.elem_dofs.ravel()
    el = np.repeat(np.arange(ne), nb)
    first = np.full(dm.n, ne, np.int64)
    np.minimum.at(first, flat, el)
    pts = dm.coords()
    ce = problem.fine_parent[first]
    lam = fem.barycentric(cm.xyz, cm.tets[ce], pts)
    vals = fem.eval_basis(problem.order, lam)                 # (n, nbH)
    cols = cdm.elem_dofs[ce]
    rows = np.repeat(np.arange(dm.n)[:, None], vals.shape[1], axis=1)
    ddofs = dm.dirichlet_dofs(problem.mesh.faces, problem.mesh.face_tag)
    isdir = np.zeros(dm.n, bool)
    isdir[ddofs] = True
    m = (np.abs(vals) > 1e-12) & keep[cols] & ~isdir[rows]
    Z = sp.coo_matrix((vals[m], (rows[m], newid[cols[m]])), shape=(dm.n, int(keep.sum()))).tocsr()
    Z.sum_duplicates()
    Z.sort_indices()
    return Z, cdm, np.nonzero(keep)[0]


def coarse_operator(Z, A):
    """E = Z^T A Z (plain transpose)."""
    E = (Z.T @ A @ Z).tocsr()
    E.sort_indices()
    return E


# ---------------------------------------------------------------------------
# The paper's coarse solve: E y = r_H by GMRES preconditioned with one-level
# ORAS on Gamma_H, with the same spatial partition as the fine level.
#
# Readings (the paper gives the method in one sentence):
# * coarse partition: a coarse element belongs to the part that holds most of
#   its fine children (ties: the lowest part id);
# * coarse overlap and partition of unity: the fine recipe applied to Gamma_H
#   (delta layers of coarse elements, chi = 1 - l/delta), restricted to the free
#   coarse dofs;
# * local coarse operators: E_i = Z_i^T A_i^h Z_i, the Galerkin projection of the
#   fine Robin problem on the fine elements inside Gamma_H,i (absorbing faces on
#   its artificial interfaces, global conditions elsewhere), so that E_i uses the
#   same fine coefficients as E = Z^T A Z;
# * inner GMRES: x0 = 0, right preconditioning, CGS2 and the Givens rotations of
#   the outer solve, one cycle of at most m_H iterations ending when the estimate
#   |g_{j+1}| / ||r_H|| <= tol_H (no restart, no true-residual check).  The coarse
#   correction is then not a fixed linear map, hence the flexible outer GMRES.
# ---------------------------------------------------------------------------
def coarse_partition(problem):
    """Part of every coarse element: the majority part of its fine children."""
    neH = problem.coarse.tets.shape[0]
    counts = np.zeros((neH, problem.nsub), np.int64)
    np.add.at(counts, (problem.fine_parent, problem.elem_part), 1)
    return np.argmax(counts, axis=1)


class _Region:
    def __init__(self, elems):
        self.elems = elems


class CoarseORAS:
    """One-level ORAS on the coarse mesh (Eq. 4 with Gamma_H, E_i, D_H,i) and the
    GMRES solve of E it preconditions."""

    def __init__(self, problem, dm, Z, cdm, keep):
        self.p = problem
        self.dm = dm
        self.Z = Z.tocsc()
        cm = problem.coarse
        self.part = coarse_partition(problem)
        subs = dd.grow_subdomains(cm, self.part, problem.nsub, problem.overlap, cdm)
        newid = np.full(cdm.n, -1, np.int64)
        newid[keep] = np.arange(len(keep))
        self.dofs, self.D, self.regions = [], [], []
        for s in subs:
            k = newid[s.dofs]
            m = k >= 0
            self.dofs.append(k[m])
            self.D.append(s.D[m])
            self.regions.append(np.nonzero(np.isin(problem.fine_parent, s.elems))[0])
        self.nH = len(keep)

    def factor(self, freq):
        w = 2.0 * np.pi * freq
        self.E_loc, self.lu = [], []
        for dofs, reg in zip(self.dofs, self.regions):
            K, Mp, Bp = dd.local_parts(self.p.mesh, self.p.c, self.p.order, self.dm, _Region(reg))
            Ah = (K.astype(np.complex128) - (w * w) * Mp - (1j * w) * Bp).tocsr()
            Zi = self.Z[:, dofs]
            Ei = (Zi.T @ Ah @ Zi).tocsc()
            Ei.sort_indices()
            self.E_loc.append(Ei)
            self.lu.append(spla.splu(Ei))

    def apply(self, r):
        """M_{1,H}^{-1} r = sum_i R_H,i^T D_H,i E_i^{-1} R_H,i r."""
        z = np.zeros(self.nH, np.complex128)
        for dofs, D, lu in zip(self.dofs, self.D, self.lu):
            z[dofs] += D * lu.solve(r[dofs])
        return z

    def solve(self, E, r, tol, m):
        """y ~ E^{-1} r by the inner GMRES; returns (y, inner iterations)."""
        y, its, est, ok = krylov.fgmres(lambda v: E @ v, self.apply, r, tol=tol, m=m, maxit=m,
                                        verify=False)
        return y, its
