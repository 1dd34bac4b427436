"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module produces *inputs only*: tetrahedral meshes (vertices, tets,
tagged boundary faces), per-element complex wave speeds, the nested coarse
mesh with its fine-to-coarse element map, element partitions and source
positions.  It contains none of the solver's arithmetic: no basis
functions, no assembly, no decomposition, no Krylov method.

Conventions
-----------
* Units are km, km/s and Hz.  ``z`` points down; the free surface is
  ``z = 0`` (top face, homogeneous Dirichlet in the method), the other five
  faces are absorbing.
* Boundary face tags: ``TAG_DIRICHLET = 0`` (top), ``TAG_ABC = 1``.
* Attenuation: ``c = v * (1 - 1j/(2Q))`` (a constant-Q complex velocity).

Meshes are tensor-product grids (optionally graded per axis) where every
hexahedral cell is cut into the six Kuhn tetrahedra that share the cell's
main diagonal.  Halving every interval of such a grid yields a mesh whose
tetrahedra are nested in those of the original one, which is how the
two-level hierarchy is built.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

TAG_DIRICHLET = 0
TAG_ABC = 1

# The six axis orders of the Kuhn split: vertex path (0,0,0) -> +e_a -> +e_b -> (1,1,1).
_KUHN_PERMS = list(itertools.permutations((0, 1, 2)))


@dataclass
class Mesh:
    xyz: np.ndarray          # (nv, 3) float64
    tets: np.ndarray         # (ne, 4) int32
    faces: np.ndarray        # (nf, 3) int32, boundary faces
    face_tag: np.ndarray     # (nf,) int8
    shape: tuple = ()        # cell counts (nx, ny, nz) of the tensor grid
    axes: tuple = ()         # (xs, ys, zs) node coordinates


@dataclass
class Problem:
    """A complete synthetic solve description (mesh, medium, hierarchy, sources)."""
    name: str
    mesh: Mesh
    c: np.ndarray                    # (ne,) complex128 wave speed per element
    freq: float                      # Hz
    order: int                       # 1 or 2
    nsub: int
    overlap: int
    levels: int                      # 1 or 2
    restart: int
    tol: float
    elem_part: np.ndarray            # (ne,) int32
    sources: np.ndarray              # (nsrc, 3) float64
    coarse: Mesh | None = None       # nested coarse mesh for levels == 2
    fine_parent: np.ndarray | None = None   # (ne,) int32 coarse element of each fine element
    meta: dict = field(default_factory=dict)


def kuhn_box_mesh(xs, ys, zs) -> Mesh:
    """Tensor grid with nodes xs x ys x zs, each cell split into 6 Kuhn tets.

    Vertex (i, j, k) has index ``i + nx1*(j + ny1*k)``; cells are visited with
    ``i`` fastest, and each cell contributes its six tets in the order of
    ``itertools.permutations((0, 1, 2))``.
    """
    xs = np.asarray(xs, np.float64)
    ys = np.asarray(ys, np.float64)
    zs = np.asarray(zs, np.float64)
    nx1, ny1, nz1 = len(xs), len(ys), len(zs)
    nx, ny, nz = nx1 - 1, ny1 - 1, nz1 - 1
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    xyz = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()

    def vid(di, dj, dk):
        return (ci + di) + nx1 * ((cj + dj) + ny1 * (ck + dk))

    tets = np.empty((nx * ny * nz, 6, 4), np.int64)
    for t, perm in enumerate(_KUHN_PERMS):
        off = [0, 0, 0]
        tets[:, t, 0] = vid(0, 0, 0)
        for s, ax in enumerate(perm):
            off[ax] = 1
            tets[:, t, s + 1] = vid(*off)
    tets = tets.reshape(-1, 4).astype(np.int32)
    faces, tags = boundary_faces(xyz, tets, z_top=zs[0])
    return Mesh(xyz=xyz, tets=tets, faces=faces, face_tag=tags,
                shape=(nx, ny, nz), axes=(xs, ys, zs))


def boundary_faces(xyz, tets, z_top=0.0):
    """Faces that belong to exactly one tet, tagged top (z == z_top) or ABC."""
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    f = tets[:, loc].reshape(-1, 3)
    fs = np.sort(f, axis=1)
    _, idx, cnt = np.unique(fs, axis=0, return_index=True, return_counts=True)
    bf = f[np.sort(idx[cnt == 1])]
    ztop = np.all(np.abs(xyz[bf, 2] - z_top) < 1e-12, axis=1)
    tags = np.where(ztop, TAG_DIRICHLET, TAG_ABC).astype(np.int8)
    return bf.astype(np.int32), tags


def refine_axis(a):
    """Insert the midpoint of every interval."""
    a = np.asarray(a, np.float64)
    out = np.empty(2 * len(a) - 1)
    out[0::2] = a
    out[1::2] = 0.5 * (a[:-1] + a[1:])
    return out


def nested_parent(fine: Mesh, coarse: Mesh) -> np.ndarray:
    """Coarse tet that contains each fine tet (fine grid = coarse grid halved)."""
    nxH, nyH, nzH = coarse.shape
    nx, ny, nz = fine.shape
    assert (nx, ny, nz) == (2 * nxH, 2 * nyH, 2 * nzH)
    ne = fine.tets.shape[0]
    cell = np.arange(ne) // 6
    i = cell % nx
    j = (cell // nx) % ny
    k = cell // (nx * ny)
    ccell = (i // 2) + nxH * ((j // 2) + nyH * (k // 2))
    cen = fine.xyz[fine.tets].sum(axis=1) / 4.0
    parent = np.full(ne, -1, np.int64)
    best = np.full(ne, -np.inf)
    for t in range(6):
        ce = ccell * 6 + t
        v = coarse.xyz[coarse.tets[ce]]                # (ne, 4, 3)
        J = np.stack([v[:, 1] - v[:, 0], v[:, 2] - v[:, 0], v[:, 3] - v[:, 0]], axis=2)
        lam = np.linalg.solve(J, (cen - v[:, 0])[..., None])[..., 0]
        lam = np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)
        score = lam.min(axis=1)
        upd = score > best
        parent[upd] = ce[upd]
        best[upd] = score[upd]
    assert np.all(best > 1e-9), "fine tets are not nested in the coarse mesh"
    return parent.astype(np.int32)


def rcb_partition(xyz, tets, nparts, weights=None):
    """Recursive coordinate bisection of element centroids into ``nparts`` parts.

    Each split sorts the elements along the axis of largest centroid extent
    (ties broken by element index) and cuts at the count given by the part
    weights.  ``weights`` (length nparts) lets parts be uneven.
    """
    ne = tets.shape[0]
    v = xyz[tets]
    cen = ((v[:, 0] + v[:, 1]) + v[:, 2]) + v[:, 3]
    cen = cen * 0.25
    w = np.ones(nparts) if weights is None else np.asarray(weights, np.float64)
    part = np.empty(ne, np.int32)

    def rec(ids, p0, p1):
        if p1 - p0 == 1:
            part[ids] = p0
            return
        pm = (p0 + p1) // 2
        c = cen[ids]
        ext = c.max(axis=0) - c.min(axis=0)
        ax = int(np.argmax(ext))
        order = np.lexsort((ids, c[:, ax]))
        frac = w[p0:pm].sum() / w[p0:p1].sum()
        cut = int(round(len(ids) * frac))
        rec(ids[order[:cut]], p0, pm)
        rec(ids[order[cut:]], pm, p1)

    rec(np.arange(ne), 0, nparts)
    return part


# ----------------------------------------------------------------------------
# Configurations
# ----------------------------------------------------------------------------

def unit_cube_problem(n=12, freq=1.2, order=1, nsub=8, overlap=1, levels=1,
                      c=1.0 * (1 - 0.01j), restart=30, tol=1e-6, source=(0.5, 0.5, 0.5),
                      coarse_n=None):
    """Homogeneous unit cube, n^3 cells x 6 Kuhn tets.

    With the defaults this is the tiny configuration: 12^3 cells, P1,
    c = 1 - 0.01i, f = 1.2 Hz (10 points per wavelength at h = 1/12), a point
    source at the centre vertex, 2x2x2 subdomains with overlap 1, one-level
    ORAS and GMRES(30) to 1e-6.  ``levels=2`` builds a nested coarse mesh with
    ``coarse_n = n // 2`` cells per side.
    """
    coarse = None
    parent = None
    if levels == 2:
        nH = coarse_n if coarse_n is not None else n // 2
        assert 2 * nH == n
        a = np.linspace(0.0, 1.0, nH + 1)
        coarse = kuhn_box_mesh(a, a, a)
        af = refine_axis(a)
        mesh = kuhn_box_mesh(af, af, af)
        parent = nested_parent(mesh, coarse)
    else:
        a = np.linspace(0.0, 1.0, n + 1)
        mesh = kuhn_box_mesh(a, a, a)
    ne = mesh.tets.shape[0]
    cc = np.full(ne, complex(c), np.complex128)
    part = rcb_partition(mesh.xyz, mesh.tets, nsub)
    return Problem(name=f"cube{n}_P{order}", mesh=mesh, c=cc, freq=freq, order=order,
                   nsub=nsub, overlap=overlap, levels=levels, restart=restart, tol=tol,
                   elem_part=part, sources=np.array([source], np.float64),
                   coarse=coarse, fine_parent=parent)


def tiny_problem():
    """The tiny configuration (about 2.2k P1 dofs, 8 subdomains, one level)."""
    return unit_cube_problem()


# --- Overthrust-shaped synthetic medium ---------------------------------------

OVT_X, OVT_Y, OVT_Z = 20.0, 20.0, 4.65


class OverthrustModel:
    """Seeded layered medium with two thrust-fold surfaces and 5% random texture.

    Eight layers whose velocities rise from 2.0 to 6.0 km/s with depth.  The
    layer interfaces are displaced by (1) a tanh ramp across a dipping fault
    trace of random strike and (2) a Gaussian anticline at a random position,
    each a few hundred metres high.  A multiplicative Gaussian random field
    (standard deviation 5%, about 0.5 km correlation length) is laid on top
    and the result clipped to [2.0, 6.0] km/s.
    """

    def __init__(self, seed=0, Q=100.0, nlayers=8):
        rng = np.random.default_rng(seed)
        self.Q = Q
        self.v = np.linspace(2.0, 6.0, nlayers)
        base = np.linspace(0.0, OVT_Z, nlayers + 1)[1:-1]
        self.z0 = base + rng.uniform(-0.12, 0.12, size=base.shape)
        th = rng.uniform(0, np.pi)
        self.fault = dict(nx=np.cos(th), ny=np.sin(th), d=rng.uniform(7.0, 13.0),
                          amp=rng.uniform(0.25, 0.45), width=rng.uniform(0.8, 1.6))
        self.anti = dict(x=rng.uniform(6.0, 14.0), y=rng.uniform(6.0, 14.0),
                         amp=rng.uniform(0.2, 0.4), s=rng.uniform(2.0, 4.0))
        # random texture on a 0.25 km lattice, smoothed to ~0.5 km correlation
        from scipy.ndimage import gaussian_filter
        from scipy.interpolate import RegularGridInterpolator
        dx = 0.25
        gx = np.arange(0.0, OVT_X + dx / 2, dx)
        gy = np.arange(0.0, OVT_Y + dx / 2, dx)
        gz = np.arange(0.0, OVT_Z + dx, dx)
        noise = rng.standard_normal((len(gx), len(gy), len(gz)))
        noise = gaussian_filter(noise, sigma=0.5 / dx, mode="wrap")
        noise *= 0.05 / noise.std()
        self._tex = RegularGridInterpolator((gx, gy, gz), noise, bounds_error=False,
                                            fill_value=None)

    def surfaces(self, x, y):
        f = self.fault
        a = self.anti
        F1 = f["amp"] * np.tanh((x * f["nx"] + y * f["ny"] - f["d"]) / f["width"])
        F2 = -a["amp"] * np.exp(-((x - a["x"]) ** 2 + (y - a["y"]) ** 2) / (2 * a["s"] ** 2))
        return F1 + F2

    def velocity(self, pts):
        pts = np.asarray(pts, np.float64)
        x, y, z = pts[:, 0], pts[:, 1], pts[:, 2]
        shift = self.surfaces(x, y)
        layer = np.zeros(len(x), np.int64)
        for zl in self.z0:
            layer += (z > zl + shift).astype(np.int64)
        v = self.v[layer] * (1.0 + self._tex(pts))
        return np.clip(v, 2.0, 6.0)

    def mean_velocity_profile(self, z):
        layer = np.searchsorted(self.z0, z, side="left")
        return self.v[np.minimum(layer, len(self.v) - 1)]


def _graded_z(model, nzH):
    """nzH coarse z intervals, equally spaced in travel time through the mean profile."""
    zz = np.linspace(0.0, OVT_Z, 2001)
    slow = 1.0 / model.mean_velocity_profile(zz)
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (slow[1:] + slow[:-1]) * np.diff(zz))])
    return np.interp(np.linspace(0.0, tau[-1], nzH + 1), tau, zz)


def overthrust_cells(freq, coarse_elems_per_wavelength=1.25):
    """Coarse cell counts (nx, ny, nz) for frequency ``freq``, with
    ``coarse_elems_per_wavelength`` coarse element edges per local wavelength (the
    fine mesh, its uniform refinement, has twice as many).

    The experiments section meshes with element edges of 1/5 of the local wavelength
    on the fine mesh and 1/2.5 on the coarse one (``coarse_elems_per_wavelength =
    2.5``; its 22M-dof Cartesian grid at 5 Hz fits that reading).  The default 1.25
    is half that resolution: the one at which the 5 Hz workload has about 2M dofs.
    A tensor grid cannot follow the local wavelength laterally, so x and y resolve
    the slowest velocity (2 km/s); in depth the spacing is graded at equal travel
    time through the mean profile, so nz follows the vertical travel time.  The
    default gives (63, 63, 9) at 5 Hz (2.37M fine P2 dofs), the paper's resolution
    the same cells at 2.5 Hz."""
    lam = 2.0 / freq
    nxy = int(np.ceil(OVT_X * coarse_elems_per_wavelength / lam - 1e-9))
    tau = (OVT_Z / 8.0) * float(np.sum(1.0 / np.linspace(2.0, 6.0, 8)))
    nz = max(2, int(np.ceil(coarse_elems_per_wavelength * tau * freq - 1e-9)))
    return (nxy, nxy, nz)


def overthrust_problem(seed=0, freq=5.0, cells=None, order=2, nsub=64, overlap=2,
                       levels=2, restart=50, tol=1e-6, Q=100.0, sources=None,
                       part_jitter=0.0):
    """Overthrust-shaped 20 x 20 x 4.65 km model meshed for frequency ``freq``.

    ``cells`` are the COARSE cell counts (nx, ny, nz), by default
    ``overthrust_cells(freq)``; the fine mesh halves every interval, so at 5 Hz the
    fine P2 space holds 253 x 253 x 37 = 2.37M dofs.  ``part_jitter`` > 0 draws
    uneven part weights in [1 - j, 1 + j].
    """
    if cells is None:
        cells = overthrust_cells(freq)
    model = OverthrustModel(seed=seed, Q=Q)
    nxH, nyH, nzH = cells
    xH = np.linspace(0.0, OVT_X, nxH + 1)
    yH = np.linspace(0.0, OVT_Y, nyH + 1)
    zH = _graded_z(model, nzH)
    coarse = kuhn_box_mesh(xH, yH, zH)
    mesh = kuhn_box_mesh(refine_axis(xH), refine_axis(yH), refine_axis(zH))
    parent = nested_parent(mesh, coarse) if levels == 2 else None
    cen = (((mesh.xyz[mesh.tets[:, 0]] + mesh.xyz[mesh.tets[:, 1]]) + mesh.xyz[mesh.tets[:, 2]])
           + mesh.xyz[mesh.tets[:, 3]]) * 0.25
    v = model.velocity(cen)
    c = v * (1.0 - 1j / (2.0 * Q))
    weights = None
    if part_jitter > 0:
        rng = np.random.default_rng(seed + 1000)
        weights = rng.uniform(1.0 - part_jitter, 1.0 + part_jitter, size=nsub)
    part = rcb_partition(mesh.xyz, mesh.tets, nsub, weights)
    if sources is None:
        sources = np.array([[2.5, 2.5, 0.58]])
    return Problem(name=f"overthrust_s{seed}_{freq:g}Hz", mesh=mesh, c=c.astype(np.complex128),
                   freq=freq, order=order, nsub=nsub, overlap=overlap, levels=levels,
                   restart=restart, tol=tol, elem_part=part,
                   sources=np.asarray(sources, np.float64), coarse=coarse,
                   fine_parent=parent, meta=dict(seed=seed, Q=Q, cells=cells))


def surface_source_grid(nx=16, ny=8, depth=0.05):
    """Sources on an nx x ny grid evenly spread over the 20 x 20 km top, at ``depth`` km."""
    xs = (np.arange(nx) + 0.5) * OVT_X / nx
    ys = (np.arange(ny) + 0.5) * OVT_Y / ny
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, depth)], axis=1)


def small_overthrust(seed=0, freq=1.0, cells=(6, 6, 3), nsub=8, overlap=2, levels=2,
                     order=2, restart=50, **kw):
    """A scaled-down Overthrust-shaped case the oracle solves in seconds."""
    return overthrust_problem(seed=seed, freq=freq, cells=cells, order=order, nsub=nsub,
                              overlap=overlap, levels=levels, restart=restart, **kw)
