"""Pins of the oracle's eigenstrain loading (Algorithm 2: the material is
evaluated at eps + eps_eig; Sec. 3.3 imposes it on the ASR product sites
under free expansion).  CPU only.

Each case has an answer fixed without the oracle: closed forms of
homogeneous media and laminates (written out below from elasticity, not
from the oracle's material code), and the equivalence of a uniform
eigenstrain on every phase with a shifted macroscopic strain."""
import math

import numpy as np
import pytest

import oracle
from oracle.solver import TRParams, load_path
from synth import gel_sites, laminate, random_circles, random_spheres

TIGHT = dict(eta_eq=1e-12, eta_cg=1e-12, R0=1e9, Rmax=1e9, max_cg=5000, max_nr=50)


def _lame(E, nu):
    # written out independently of oracle.lame
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def _solve(pm, phases, table, dE, free, prm=None):
    rve = oracle.RVE(pm, phases, free_mask=np.asarray(free, bool), eigenstrain=table)
    return load_path(rve, [np.asarray(dE, float)], prm or TRParams(**TIGHT)), rve


@pytest.mark.parametrize("dims", [(6, 4), (4, 6, 5)])
def test_homogeneous_free_expansion(dims):
    """One phase, every mean component stress-free, no macroscopic load:
    the cell takes the stress-free strain eps = -eps_eig exactly."""
    nc = 3 if len(dims) == 2 else 6
    pm = np.zeros(tuple(reversed(dims)), np.uint8)
    eig = np.array([3e-4, -1e-4, 2e-4, 1e-4, -2e-4, 5e-5][:nc])
    res, _ = _solve(pm, [oracle.Phase(1.0, 0.3)], eig[None, :], np.zeros(nc), [True] * nc)
    np.testing.assert_allclose(res["mean_strain"][-1], -eig, atol=1e-16)
    np.testing.assert_allclose(res["eps"].reshape(nc, -1), np.repeat(-eig[:, None], pm.size, 1), atol=1e-16)
    np.testing.assert_allclose(res["sigma"], 0.0, atol=1e-16)


def test_homogeneous_constrained_expansion():
    """3D, isotropic eigenstrain a I, eps_zz held at zero, the rest free:
    eps_xx = eps_yy = -a (3 lam + 2 mu) / (2 (lam + mu)) and
    sigma_zz = lam (2 eps_xx + 3 a) + 2 mu a."""
    lam, mu = _lame(2.0, 0.25)
    a = 4e-4
    pm = np.zeros((4, 4, 4), np.uint8)
    eig = np.array([[a, a, a, 0, 0, 0]])
    res, _ = _solve(pm, [oracle.Phase(2.0, 0.25)], eig, np.zeros(6), [True, True, False, True, True, True])
    s = -a * (3 * lam + 2 * mu) / (2 * (lam + mu))
    np.testing.assert_allclose(res["mean_strain"][-1], [s, s, 0, 0, 0, 0], atol=1e-16)
    np.testing.assert_allclose(res["mean_stress"][-1], [0, 0, lam * (2 * s + 3 * a) + 2 * mu * a, 0, 0, 0],
                               rtol=1e-12, atol=1e-16)


def test_homogeneous_damage_from_eigenstrain():
    """Fully strain-controlled damaging medium at zero mean strain with an
    isotropic eigenstrain a I: eps stays 0, kappa = sqrt(3) a is taken from
    the evaluated strain, D from the bilinear law (Eq. (A.3)),
    sigma = (1 - D)(3 lam + 2 mu) a on the normal components."""
    k0, kf = 1e-4, 1e-3
    a = 2e-4
    lam, mu = _lame(1.0, 0.3)
    pm = np.zeros((4, 4, 4), np.uint8)
    res, rve = _solve(pm, [oracle.Phase(1.0, 0.3, True, k0, kf)], np.array([[a, a, a, 0, 0, 0]]),
                      np.zeros(6), [False] * 6)
    kap = math.sqrt(3) * a
    D = kf * (kap - k0) / (kap * (kf - k0))
    np.testing.assert_allclose(res["eps"], 0.0, atol=0)
    np.testing.assert_allclose(res["kappa"], kap, rtol=1e-14)
    np.testing.assert_allclose(res["mean_stress"][-1], [(1 - D) * (3 * lam + 2 * mu) * a] * 3 + [0] * 3,
                               rtol=1e-13)


def _laminate_expansion(pa, pb, a, frac, plane_strain):
    """Bilayer normal to the last axis, layer A (fraction ``frac``) with the
    isotropic eigenstrain a I, free expansion.  The in-plane strain s is
    shared; the out-of-plane stress vanishes in both layers; the in-plane
    mean stress vanishes: f k_A (s + a) + (1 - f) k_B s = 0 with k the
    in-plane modulus under zero out-of-plane stress (biaxial in 3D,
    plane strain uniaxial in 2D)."""
    (la, ma), (lb, mb) = _lame(pa.E, pa.nu), _lame(pb.E, pb.nu)
    if plane_strain:
        k = lambda l, m: 4 * m * (l + m) / (l + 2 * m)  # noqa: E731
        ninp = 1
    else:
        k = lambda l, m: 2 * m * (3 * l + 2 * m) / (l + 2 * m)  # noqa: E731
        ninp = 2
    ka, kb = k(la, ma), k(lb, mb)
    s = -frac * ka * a / (frac * ka + (1 - frac) * kb)
    # out-of-plane evaluated strain u from (l + 2m) u + l * ninp * v = 0
    ua = -ninp * la * (s + a) / (la + 2 * ma)
    ub = -ninp * lb * s / (lb + 2 * mb)
    return s, ua - a, ub


@pytest.mark.parametrize("dims", [(4, 8), (4, 4, 8)])
def test_laminate_free_expansion_closed_form(dims):
    pa, pb = oracle.Phase(1.0, 0.3), oracle.Phase(10.0, 0.2)
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = laminate(dims, axis=nd - 1)
    a = 3e-4
    table = np.zeros((2, nc))
    table[0, :nd] = a
    res, _ = _solve(pm, [pa, pb], table, np.zeros(nc), [True] * nc)
    s, za, zb = _laminate_expansion(pa, pb, a, 0.5, nd == 2)
    half = dims[-1] // 2
    eps = res["eps"]
    ea = np.zeros(nc)
    eb = np.zeros(nc)
    ea[:nd - 1] = s
    eb[:nd - 1] = s
    ea[nd - 1], eb[nd - 1] = za, zb
    na = eps[:, :half].reshape(nc, -1).shape[1]
    np.testing.assert_allclose(eps[:, :half].reshape(nc, -1), np.repeat(ea[:, None], na, 1), atol=1e-15)
    np.testing.assert_allclose(eps[:, half:].reshape(nc, -1), np.repeat(eb[:, None], na, 1), atol=1e-15)
    np.testing.assert_allclose(res["mean_stress"][-1], 0.0, atol=1e-15)


@pytest.mark.parametrize("dims", [(16, 12), (8, 6, 10)])
def test_uniform_eigenstrain_equals_shifted_load(dims):
    """An eigenstrain e on every phase under mean-strain control E gives the
    same evaluated strain field as the load E + e without eigenstrain
    (heterogeneous, damaging): eps_A + e = eps_B, equal stress and damage."""
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = random_circles(dims, 0.3, rmin=2.0, rmax=3.0, seed=4) if nd == 2 else \
        random_spheres(dims, count=3, rmin=1.5, rmax=2.5, seed=5)
    phases = [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), oracle.Phase(10.0, 0.2)]
    e = np.array([1.5e-4, -0.5e-4, 1e-4, 0.3e-4, 0.2e-4, -0.1e-4][:nc])
    E = np.array([0.5e-4, 0.2e-4, 0.4e-4, 0.0, 0.1e-4, 0.0][:nc])
    prm = TRParams(eta_eq=1e-11, eta_cg=1e-3, R0=1e-2, Rmax=1e-2, max_nr=200, max_cg=2000)
    ra, _ = _solve(pm, phases, np.repeat(e[None, :], 2, 0), E, [False] * nc, prm)
    rb, _ = _solve(pm, phases, None, E + e, [False] * nc, prm)
    assert ra["reports"][0].converged and rb["reports"][0].converged
    assert ra["kappa"].max() > 1e-4  # damage reached
    shape = (nc,) + (1,) * nd
    np.testing.assert_allclose(ra["eps"] + e.reshape(shape), rb["eps"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(ra["sigma"], rb["sigma"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(ra["kappa"], rb["kappa"], rtol=0, atol=1e-12)


def test_gel_sites_expansion_cracks_the_host():
    """ASR-like 2D cell (aggregate discs, gel pixels inside them with a
    growing expansion, free expansion): the mean stress stays zero, the
    mean strain grows with the gel expansion, and damage starts next to the
    gel sites (Sec. 3.3)."""
    dims = (24, 24)
    pm = gel_sites(random_circles(dims, 0.4, rmin=3.0, rmax=5.0, seed=6), 4, seed=7)
    phases = [oracle.Phase(12.0, 0.3, True, 2.5e-4, 2.5e-3), oracle.Phase(59.0, 0.3, True, 1.7e-4, 1.7e-3),
              oracle.Phase(11.0, 0.18)]
    rve = oracle.RVE(pm, phases, free_mask=np.ones(3, bool))
    tables = []
    for n in range(1, 5):
        t = np.zeros((3, 3))
        t[2, :2] = -n * 5e-4  # stress-free expansion n * 5e-4 of the gel
        tables.append(t)
    prm = TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=1e-2, Rmax=1e-2, max_nr=300)
    res = load_path(rve, [np.zeros(3)] * 4, prm, eigenstrains=tables)
    assert all(r.converged for r in res["reports"])
    np.testing.assert_allclose(res["mean_stress"], 0.0, atol=1e-9)
    ms = res["mean_strain"][:, :2].mean(axis=1)
    assert np.all(np.diff(ms) > 0) and ms[0] > 0
    damaged = res["kappa"] > np.where(pm == 0, 2.5e-4, 1.7e-4)
    assert damaged.any()
    # every damaged voxel lies within a few voxels of a gel site (periodic)
    sites = np.argwhere(pm == 2)
    for v in np.argwhere(damaged & (pm != 2)):
        d = np.abs(sites - v)
        d = np.minimum(d, np.array(pm.shape) - d)
        assert np.sqrt((d ** 2).sum(axis=1)).min() <= 6.0
