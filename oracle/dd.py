"""Oracle: overlapping decomposition, partition of unity, local absorbing matrices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (4): M_1^{-1} = sum_i R_i^T D_i A_i^{-1} R_i, where R_i is the Boolean
restriction to the dofs of the overlapping subdomain Gamma_i, D_i the local
diagonal partition of unity and A_i the local Helmholtz operator with
absorbing (Robin) conditions on the artificial interfaces -- the ORAS
ingredient that distinguishes it from RAS with local Dirichlet problems.

Readings (where the paper is silent):
* overlap: ``delta`` layers of elements, each layer adds every element that
  shares a vertex with the current subdomain;
* partition of unity: vertex weight chi_i(v) = 1 - l_i(v)/delta, where l_i(v)
  is the layer at which v entered Gamma_i (0 for the non-overlapping part),
  edge weight = mean of its two end vertices, then D_i = chi_i / sum_j chi_j;
  with delta = 0 every chi is 1;
* interface condition: the same first-order impedance as the outer absorbing
  boundary, -i omega int c^{-1} phi phi, with c of the subdomain element that
  owns the face; faces on the global boundary keep their global condition;
  Dirichlet dofs are identity rows in A_i as in A.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem

_FACE_LOC = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


class Subdomain:
    def __init__(self, elems, layer_v, dofs, weights):
        self.elems = elems          # element ids of Gamma_i (sorted)
        self.layer_v = layer_v      # dict-like: vertex -> layer (array over all vertices, -1 outside)
        self.dofs = dofs            # R_i as sorted global dof ids
        self.chi = weights          # chi_i on self.dofs
        self.D = None               # partition of unity on self.dofs
        self.A = None               # local matrix (csr), per frequency


def vertex_element_adjacency(tets, nv):
    ne = tets.shape[0]
    rows = np.repeat(np.arange(ne), 4)
    return sp.csr_matrix((np.ones(ne * 4, np.int8), (tets.ravel(), rows)), shape=(nv, ne))


def grow_subdomains(mesh, elem_part, nsub, delta, dm):
    """Gamma_i for every part: delta element layers grown through shared vertices."""
    nv = mesh.xyz.shape[0]
    VE = vertex_element_adjacency(mesh.tets, nv)
    subs = []
    for i in range(nsub):
        inside = elem_part == i
        layer = np.full(nv, -1, np.int64)
        layer[np.unique(mesh.tets[inside])] = 0
        for l in range(1, delta + 1):
            vin = layer >= 0
            touched = (VE.T @ vin.astype(np.int8)) > 0
            newe = touched & ~inside
            inside = inside | touched
            nvts = np.unique(mesh.tets[newe])
            fresh = nvts[layer[nvts] < 0]
            layer[fresh] = l
        elems = np.nonzero(inside)[0]
        dofs = np.unique(dm.elem_dofs[elems].ravel())
        if delta == 0:
            chi = np.ones(len(dofs))
        else:
            chiv = 1.0 - layer / float(delta)
            chi = np.empty(len(dofs))
            isv = dofs < dm.nv
            chi[isv] = chiv[dofs[isv]]
            ed = dm.edges[dofs[~isv] - dm.nv]
            chi[~isv] = 0.5 * (chiv[ed[:, 0]] + chiv[ed[:, 1]])
        subs.append(Subdomain(elems, layer, dofs, chi))
    total = np.zeros(dm.n)
    for s in subs:
        np.add.at(total, s.dofs, s.chi)
    assert np.all(total > 0), "a dof is not covered by any non-overlapping part"
    for s in subs:
        s.D = s.chi / total[s.dofs]
    return subs


def subdomain_faces(mesh, elems):
    """Faces of Gamma_i that belong to one of its elements only, with that element."""
    t = mesh.tets[elems]
    f = t[:, _FACE_LOC].reshape(-1, 3)
    owner = np.repeat(elems, 4)
    fs = np.sort(f, axis=1).astype(np.int64)
    nv = mesh.xyz.shape[0]
    key = (fs[:, 0] * nv + fs[:, 1]) * nv + fs[:, 2]
    u, idx, cnt = np.unique(key, return_index=True, return_counts=True)
    sel = idx[cnt == 1]
    return f[sel], owner[sel], key[sel]


def local_parts(mesh, c, order, dm, sub):
    """(K_i, M'_i, B'_i) of Gamma_i in global numbering, B' holding the ABC on
    global absorbing faces and the Robin term on artificial interfaces."""
    nv = mesh.xyz.shape[0]
    f, owner, key = subdomain_faces(mesh, sub.elems)
    gf = np.sort(mesh.faces.astype(np.int64), axis=1)
    gkey = (gf[:, 0] * nv + gf[:, 1]) * nv + gf[:, 2]
    gorder = np.argsort(gkey)
    pos = np.searchsorted(gkey[gorder], key)
    pos = np.minimum(pos, len(gkey) - 1)
    on_boundary = gkey[gorder][pos] == key
    tag = np.full(len(key), -1)
    tag[on_boundary] = mesh.face_tag[gorder][pos[on_boundary]]
    absorbing = (~on_boundary) | (tag == fem.TAG_ABC)
    _, K, Mp, Bp = fem.assemble_parts(mesh, c, order, elems=sub.elems,
                                      faces=f[absorbing], face_coef_elem=owner[absorbing],
                                      dm=dm)
    return K, Mp, Bp


def build_local_matrices(problem, dm, subs, ddofs, freq, robin=True):
    """A_i(omega) restricted to R_i (local numbering = sorted global dofs).

    ``robin=False`` gives the RAS variant (artificial interfaces without the
    absorbing term) used as an ablation.
    """
    is_dir = np.zeros(dm.n, bool)
    is_dir[ddofs] = True
    w = 2.0 * np.pi * freq
    for s in subs:
        K, Mp, Bp = local_parts(problem.mesh, problem.c, problem.order, dm, s)
        if not robin:
            gf, go = _global_abc_faces_of(problem.mesh, s.elems)
            _, _, _, Bp = fem.assemble_parts(problem.mesh, problem.c, problem.order,
                                             elems=s.elems, dm=dm, faces=gf,
                                             face_coef_elem=go)
        Ag = (K.astype(np.complex128) - (w * w) * Mp - (1j * w) * Bp).tocsr()
        Al = Ag[s.dofs][:, s.dofs].tocsr()
        ld = np.nonzero(is_dir[s.dofs])[0]
        s.A = fem.apply_dirichlet(Al, ld)
    return subs


def _global_abc_faces_of(mesh, elems):
    f, owner, key = subdomain_faces(mesh, elems)
    nv = mesh.xyz.shape[0]
    sel = mesh.face_tag == fem.TAG_ABC
    gf = np.sort(mesh.faces[sel].astype(np.int64), axis=1)
    gkey = (gf[:, 0] * nv + gf[:, 1]) * nv + gf[:, 2]
    m = np.isin(key, gkey)
    return f[m], owner[m]
