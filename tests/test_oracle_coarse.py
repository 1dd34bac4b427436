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
