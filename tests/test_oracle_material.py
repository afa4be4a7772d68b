"""Pins of the oracle's constitutive law against closed forms (CPU only)."""
import numpy as np
import pytest

import oracle


def test_lame_closed_form():
    lam, mu = oracle.lame(1.0, 0.3)
    assert np.isclose(lam, 0.3 / (1.3 * 0.4))
    assert np.isclose(mu, 1.0 / 2.6)
    # bulk modulus identity K = lam + 2/3 mu = E / (3 (1 - 2 nu))
    assert np.isclose(lam + 2.0 * mu / 3.0, 1.0 / (3.0 * 0.4))


@pytest.mark.parametrize("E,nu", [(1.0, 0.3), (10.0, 0.2)])
def test_uniaxial_stress_3d(E, nu):
    """eps = diag(1, -nu, -nu) is the strain of uniaxial stress E."""
    lam, mu = oracle.lame(E, nu)
    eps = np.array([1.0, -nu, -nu, 0.0, 0.0, 0.0]).reshape(6, 1)
    sig = oracle.elastic_stress(eps, lam, mu)
    np.testing.assert_allclose(sig.ravel(), [E, 0, 0, 0, 0, 0], atol=1e-12)


def test_plane_strain_uniaxial():
    """Plane strain with sigma_22 = 0: eps_22 = -nu/(1-nu) eps_11 and
    sigma_11 = E/(1-nu^2) eps_11."""
    E, nu = 1.0, 0.3
    lam, mu = oracle.lame(E, nu)
    eps = np.array([1.0, -nu / (1 - nu), 0.0]).reshape(3, 1)
    sig = oracle.elastic_stress(eps, lam, mu)
    np.testing.assert_allclose(sig.ravel(), [E / (1 - nu ** 2), 0, 0], atol=1e-12)


def test_shear_mandel_scaling():
    """Engineering shear gamma -> tau = mu gamma; Mandel slot holds sqrt2 eps_12."""
    lam, mu = oracle.lame(1.0, 0.3)
    gamma = 1e-3
    eps = np.array([0, 0, 0, 0, 0, np.sqrt(2) * gamma / 2]).reshape(6, 1)
    sig = oracle.elastic_stress(eps, lam, mu)
    assert np.isclose(sig[5, 0] / np.sqrt(2), mu * gamma)


def test_principal_strains_and_kappa():
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    lam = np.array([2e-3, -1e-3, 5e-4])
    t = Q @ np.diag(lam) @ Q.T
    m = oracle.tensor_to_mandel(t[None])[:, 0].reshape(6, 1)
    w = np.sort(oracle.principal_strains(m)[0])
    np.testing.assert_allclose(w, np.sort(lam), atol=1e-15)
    k = oracle.kappa_of_strain(m)[0]
    assert np.isclose(k, np.sqrt(2e-3 ** 2 + 5e-4 ** 2))
    # compression only -> no tension measure
    assert oracle.kappa_of_strain(-np.abs(m) * 0 + np.array([-1, -2, -3, 0, 0, 0.]).reshape(6, 1))[0] == 0.0
    # plane strain: the out-of-plane zero is not tensile
    assert np.isclose(oracle.kappa_of_strain(np.array([1e-3, -1e-3, 0.0]).reshape(3, 1))[0], 1e-3)


def test_bilinear_damage_scalar_curve():
    """Uniaxial scalar curve sigma = (1 - D) E kappa: elastic to kappa0, peak
    E kappa0, linear softening of slope -E kappa0/(kappaf - kappa0)
    (= -E/9 for kappa0 = 1e-4, kappaf = 1e-3), zero from kappaf on."""
    E, k0, kf = 1.0, 1e-4, 1e-3
    kap = np.linspace(0, 1.5e-3, 3001)
    D = oracle.damage_of_kappa(kap, k0, kf)
    s = (1 - D) * E * kap
    assert np.isclose(s.max(), E * k0)
    assert np.isclose(kap[np.argmax(s)], k0)
    soft = (kap > k0 * 1.01) & (kap < kf * 0.99)
    slope = np.diff(s[soft]) / np.diff(kap[soft])
    np.testing.assert_allclose(slope, -E / 9.0, rtol=1e-9)
    assert np.all(s[kap >= kf] == 0.0)
    assert np.all(D[kap <= k0] == 0.0)
    # the paper's form D = (kappa - kappa0)(1 + alpha)/kappa with alpha = k0/(kf-k0)
    alpha = k0 / (kf - k0)
    mid = (kap > k0) & (kap < kf)
    np.testing.assert_allclose(D[mid], (kap[mid] - k0) * (1 + alpha) / kap[mid], rtol=1e-12)


def test_history_max_and_unloading():
    ph = [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3)]
    params = oracle.PhaseParams(np.zeros((1, 1), np.uint8), ph)
    eps_hi = np.array([5e-4, 0, 0]).reshape(3, 1, 1)
    _, D_hi, k_hi = oracle.evaluate(eps_hi, params)
    # unloading to a smaller strain keeps the damage of the history
    _, D_lo, k_lo = oracle.evaluate(eps_hi * 0.1, params, kappa_hist=k_hi)
    assert np.isclose(D_lo, D_hi) and np.isclose(k_lo, k_hi)
    _, D_fresh, _ = oracle.evaluate(eps_hi * 0.1, params)
    assert D_fresh[0, 0] == 0.0
