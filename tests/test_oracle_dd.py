"""Pins for the oracle's decomposition (Eq. 4): partition of unity, coverage,
single-subdomain reduction to the global operator, ORAS vs RAS, N_d = 1."""
import numpy as np
import pytest

import synth
from oracle import dd, fem
from oracle.solver import OracleSolver


@pytest.mark.parametrize("overlap", [0, 1, 2])
def test_partition_of_unity_sums_to_one(overlap):
    p = synth.small_overthrust(levels=1, cells=(3, 3, 2), freq=0.8, nsub=4, overlap=overlap)
    A, dm, ddofs = fem.global_system(p)
    subs = dd.grow_subdomains(p.mesh, p.elem_part, p.nsub, p.overlap, dm)
    total = np.zeros(dm.n)
    for s in subs:
        np.add.at(total, s.dofs, s.D)
    assert np.abs(total - 1.0).max() <= 1e-15
    for i, s in enumerate(subs):
        own = np.nonzero(p.elem_part == i)[0]
        assert np.all(np.isin(own, s.elems))
        assert np.all(s.D >= 0)


def test_overlap_grows_by_vertex_layers():
    p = synth.unit_cube_problem(n=8, nsub=8, overlap=1)
    A, dm, ddofs = fem.global_system(p)
    subs = dd.grow_subdomains(p.mesh, p.elem_part, p.nsub, 1, dm)
    s = subs[0]
    own = p.elem_part == 0
    own_v = np.unique(p.mesh.tets[own])
    touching = np.nonzero(np.any(np.isin(p.mesh.tets, own_v), axis=1))[0]
    assert np.array_equal(np.sort(touching), s.elems)
    # chi is 1 on the core vertices and 0 on the outermost layer
    assert np.all(s.layer_v[own_v] == 0)


def test_single_subdomain_local_matrix_equals_global():
    p = synth.small_overthrust(levels=1, cells=(3, 3, 2), freq=0.8, nsub=1, overlap=0)
    S = OracleSolver(p)
    S.factor()
    d = (S.subs[0].A - S.A)
    assert abs(d).max() <= 1e-14 * abs(S.A).max()
    assert np.array_equal(S.subs[0].dofs, np.arange(S.n))


def test_one_subdomain_converges_in_one_iteration():
    p = synth.unit_cube_problem(n=6, nsub=1, overlap=0)
    S = OracleSolver(p)
    S.factor()
    x, it, rel, ok = S.solve(S.rhs()[:, 0])
    assert ok and it == 1 and rel < 1e-10


def test_robin_interfaces_beat_dirichlet_interfaces():
    """The absorbing interface condition is what makes ORAS better than RAS."""
    p = synth.unit_cube_problem(n=12, nsub=8, overlap=1)
    its = {}
    for robin in (True, False):
        S = OracleSolver(p, robin=robin)
        S.factor()
        _, it, rel, ok = S.solve(S.rhs()[:, 0])
        assert ok
        its[robin] = it
    assert its[True] < its[False], its


def test_robin_term_lives_on_artificial_interfaces_only():
    """A_i differs from the restricted global operator only in rows of dofs on the
    artificial boundary of Gamma_i, which are exactly the dofs with zero PU weight;
    the difference carries the -i omega int c^{-1} phi phi impedance (negative
    imaginary diagonal)."""
    p = synth.unit_cube_problem(n=6, nsub=8, overlap=1)
    S = OracleSolver(p)
    S.factor()
    for s in S.subs:
        diff = (s.A - S.A[s.dofs][:, s.dofs]).tocoo()
        big = np.abs(diff.data) > 1e-12
        rows = np.unique(diff.row[big])
        assert len(rows) > 0
        assert np.all(s.D[rows] == 0.0)
    R = OracleSolver(p, robin=False)
    R.factor()
    for s, r in zip(S.subs, R.subs):
        imp = (s.A - r.A).tocsr()
        rows = np.unique(imp.tocoo().row[np.abs(imp.tocoo().data) > 1e-14])
        assert len(rows) > 0 and np.all(s.D[rows] == 0.0)
        assert np.all(imp.diagonal()[rows].imag < 0)
        assert np.abs(imp.diagonal()[rows].real).max() < 0.05 * np.abs(imp.diagonal()[rows].imag).max()
