"""Pins of the oracle's linear-simplex (multi-quadrature-point) cell problem
(CPU only): the Fourier symbols against the real-space gradient of the
linear interpolant on every simplex, the projector's defining properties,
and elastic solves against the assembled periodic FE problem on simplices
and against the laminate closed form."""
import numpy as np
import pytest

import oracle
from oracle.simplex import SimplexRVE, simplex_symbols, _b_matrix
from oracle.solver import TRParams, load_path
from synth import circular_inclusion, laminate
from tests import fe_simplex as fs

TIGHT = dict(eta_eq=1e-12, eta_cg=1e-12, R0=1e9, Rmax=1e9, max_cg=5000)
STIFF = oracle.Phase(10.0, 0.2)


@pytest.mark.parametrize("dims", [(6, 4), (4, 3, 5)])
def test_symbols_match_real_space_simplex_gradients(dims):
    """B(k) u_hat of the symbols equals the FFT of the strains that the
    general simplex gradient formula gives for random nodal displacements."""
    d = len(dims)
    shape = tuple(reversed(dims))
    rng = np.random.default_rng(0)
    u = rng.standard_normal((d,) + shape)
    B = fs.strain_matrix(dims)
    eps = (B @ u.reshape(-1)).reshape((-1, len(oracle.simplex.kuhn_permutations(d))) + shape)
    uh = np.fft.fftn(u, axes=tuple(range(1, d + 1)))
    Bk = _b_matrix(simplex_symbols(shape))
    epsh = np.einsum("cqa...,a...->cq...", Bk, uh)
    ref = np.fft.fftn(eps, axes=tuple(range(2, d + 2)))
    np.testing.assert_allclose(epsh, ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("dims", [(6, 4), (4, 3, 5)])
def test_projector_properties(dims):
    d = len(dims)
    shape = tuple(reversed(dims))
    pm = np.zeros(shape, np.uint8)
    nc = 3 if d == 2 else 6
    free = np.zeros(nc, bool)
    free[0] = True
    rve = SimplexRVE(pm, [oracle.Phase(1.0, 0.3)], free_mask=free)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((nc,) + rve.shape)
    y = rng.standard_normal((nc,) + rve.shape)
    gx = rve.G(x)
    np.testing.assert_allclose(rve.G(gx), gx, atol=1e-12)
    assert abs(rve.dot(x, rve.G(y)) - rve.dot(gx, y)) < 1e-10 * rve.norm(x) * rve.norm(y)
    # a compatible field (strains of nodal displacements, plus a mean on the
    # free component) is left unchanged
    u = rng.standard_normal((d,) + shape)
    comp = (fs.strain_matrix(dims) @ u.reshape(-1)).reshape((nc,) + rve.shape)
    comp[0] += 0.37
    np.testing.assert_allclose(rve.G(comp), comp, atol=1e-12)
    # a strain-controlled mean is removed
    unif = np.zeros((nc,) + rve.shape)
    unif[1] = 1.0
    np.testing.assert_allclose(rve.G(unif), 0.0, atol=1e-12)


@pytest.mark.parametrize("dims,free", [
    ((6, 6), None),
    ((6, 6), np.array([False, True, True])),
    ((4, 4, 4), None),
    ((4, 4, 4), np.array([True, True, False, True, True, True])),
])
def test_elastic_solve_matches_assembled_simplex_fe(dims, free):
    d = len(dims)
    if d == 2:
        pm = circular_inclusion(dims, 0.3)
        E = np.array([1e-3, 0.0, 0.0]) if free is not None else np.array([1e-3, -2e-4, 3e-4])
    else:
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        pm[1:3, 1:3, 0:2] = 1
        pm[3, 0, 3] = 1
        E = np.array([0, 0, 1e-3, 0, 0, 0.0]) if free is not None else np.array([1e-3, -2e-4, 3e-4, 1e-4, 0, 2e-4])
    rve = SimplexRVE(pm, [oracle.Phase(1.0, 0.3), STIFF], free_mask=free)
    res = load_path(rve, [E], TRParams(**TIGHT))
    assert res["reports"][0].converged
    ref, _ = fs.solve_elastic(dims, rve.params.lam, rve.params.mu, E, free)
    assert np.max(np.abs(res["eps"] - ref)) / np.max(np.abs(ref)) < 1e-9


def test_laminate_closed_form_on_simplices():
    """A bilayer normal to z: the per-layer strains of the closed form are
    piecewise linear displacements, which the simplices represent exactly."""
    from tests.test_oracle_solver import _laminate_exact
    pa, pb = oracle.Phase(1.0, 0.3), oracle.Phase(10.0, 0.2)
    dims = (4, 4, 8)
    pm = laminate(dims, axis=2)
    E = np.array([2e-4, -1e-4, 1e-3, 3e-4, -2e-4, 1e-4])
    rve = SimplexRVE(pm, [pa, pb])
    res = load_path(rve, [E], TRParams(**TIGHT))
    ea, eb = _laminate_exact(pa, pb, E)
    eps = res["eps"]  # (6, 6 simplices, z, y, x)
    np.testing.assert_allclose(eps[:, :, :4].reshape(6, -1), np.repeat(ea[:, None], 6 * 64, 1), atol=1e-15)
    np.testing.assert_allclose(eps[:, :, 4:].reshape(6, -1), np.repeat(eb[:, None], 6 * 64, 1), atol=1e-15)


def test_homogeneous_damaging_cell_matches_the_voxel_cell():
    """A homogeneous damaging cell under uniaxial load (the rest free) stays
    uniform on simplices and on voxels alike: the same mean stress through
    the onset of damage, one kappa per simplex."""
    dims = (4, 4, 4)
    pm = np.zeros((4, 4, 4), np.uint8)
    ph = [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3)]
    free = np.array([True, True, False, True, True, True])
    incs = [np.array([0, 0, 8e-5, 0, 0, 0])] * 3
    prm = TRParams(eta_eq=1e-10, eta_cg=1e-10, R0=1.0, Rmax=1.0, max_nr=200)
    a = load_path(SimplexRVE(pm, ph, free_mask=free), incs, prm)
    b = load_path(oracle.RVE(pm, ph, free_mask=free), incs, prm)
    assert all(r.converged for r in a["reports"])
    np.testing.assert_allclose(a["mean_stress"], b["mean_stress"], rtol=1e-9, atol=1e-15)
    assert a["kappa"].shape == (6,) + pm.shape and a["kappa"].max() > 1e-4
