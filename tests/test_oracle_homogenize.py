"""Pins of the oracle's effective secant stiffness (CPU only): the closed
form of a homogeneous, uniformly damaged medium, the assembled periodic FE
homogenisation (brute force, no Fourier symbol), symmetry, and the Voigt /
Reuss bounds."""
import numpy as np
import pytest

import oracle
from oracle.homogenize import effective_stiffness
from synth import circular_inclusion, random_spheres
from tests import fe_bruteforce as fe


def _mandel_C(lam, mu, nc):
    nd = 2 if nc == 3 else 3
    C = 2.0 * mu * np.eye(nc)
    C[:nd, :nd] += lam
    return C


@pytest.mark.parametrize("dims", [(6, 4), (4, 6, 4)])
def test_homogeneous_uniform_damage_closed_form(dims):
    nc = 3 if len(dims) == 2 else 6
    pm = np.zeros(tuple(reversed(dims)), np.uint8)
    rve = oracle.RVE(pm, [oracle.Phase(2.0, 0.25)])
    d = 0.3
    C = effective_stiffness(rve, np.full(pm.shape, d))
    lam, mu = 2.0 * 0.25 / (1.25 * 0.5), 2.0 / 2.5
    np.testing.assert_allclose(C, (1 - d) * _mandel_C(lam, mu, nc), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dims", [(8, 8), (4, 4, 4)])
def test_matches_assembled_fe_homogenisation(dims):
    """Columns of C_bar equal the mean stresses of the assembled periodic FE
    solutions for unit mean strains, with the damaged moduli per voxel."""
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    if nd == 2:
        pm = circular_inclusion(dims, 0.3)
    else:
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        pm[1:3, 1:3, 0:2] = 1
        pm[3, 0, 3] = 1
    rve = oracle.RVE(pm, [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), oracle.Phase(10.0, 0.2)])
    D = np.where(pm == 0, np.random.default_rng(0).uniform(0, 0.8, pm.shape), 0.0)
    C = effective_stiffness(rve, D)
    lam = rve.params.lam * (1 - D)
    mu = rve.params.mu * (1 - D)
    ref = np.zeros((nc, nc))
    for j in range(nc):
        E = np.zeros(nc)
        E[j] = 1.0
        eps, _ = fe.solve_elastic(dims, lam, mu, E)
        tr = sum(eps[i] for i in range(nd))
        sig = 2 * mu * eps
        for i in range(nd):
            sig[i] = sig[i] + lam * tr
        ref[:, j] = sig.reshape(nc, -1).mean(axis=1)
    np.testing.assert_allclose(C, ref, rtol=1e-9, atol=1e-12)


def test_symmetric_and_between_reuss_and_voigt():
    dims = (8, 6, 10)
    pm = random_spheres(dims, count=3, rmin=1.5, rmax=2.5, seed=3)
    rve = oracle.RVE(pm, [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), oracle.Phase(10.0, 0.2)])
    D = np.where(pm == 0, np.random.default_rng(1).uniform(0, 0.9, pm.shape), 0.0)
    C = effective_stiffness(rve, D)
    np.testing.assert_allclose(C, C.T, rtol=0, atol=1e-9 * np.abs(C).max())
    Cv = np.zeros((6, 6))
    Sr = np.zeros((6, 6))
    lam = rve.params.lam * (1 - D)
    mu = rve.params.mu * (1 - D)
    for l, m in zip(lam.ravel(), mu.ravel()):
        Cl = _mandel_C(l, m, 6)
        Cv += Cl
        Sr += np.linalg.inv(Cl)
    Cv /= pm.size
    Cr = np.linalg.inv(Sr / pm.size)
    assert np.linalg.eigvalsh(Cv - C).min() > -1e-9
    assert np.linalg.eigvalsh(C - Cr).min() > -1e-9
