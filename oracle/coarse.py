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

from . import fem


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
