"""Symmetric consistent damage tangent on the GPU (needs a GB300): the
Hessian-vector product against the oracle at loading states, the
trust-region load path with it against the oracle (the same equilibrium as
the secant Hessian in far fewer Newton iterations), and what it leaves
unchanged (the secant effective stiffness, the option check)."""
import numpy as np
import pytest

import oracle
from oracle.consistent import ConsistentRVE, consistent_tangent_apply, positive_part
from synth import circular_inclusion, random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)


def _solver(dims, pm, phases, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, phases, precision=precision, **kw)


def _phases(ph):
    return [oracle.Phase(*p) if p[2] else oracle.Phase(p[0], p[1]) for p in ph]


def _to_dev(a, precision):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if precision == 32 else np.float64)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dims", [(32, 24), (24, 20, 18), (32, 32, 32)])
def test_consistent_hessp_matches_oracle(dims, precision):
    """A loading state with every matrix voxel softening (kappa well inside
    (kappa0, kappaf), history 0.7 kappa_trial): G : B_sym : v against the
    oracle."""
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = circular_inclusion(dims, 0.3) if nd == 2 else random_spheres(dims, count=3, rmin=1.5, rmax=3.0, seed=5)
    rng = np.random.default_rng(3)
    eps = rng.standard_normal((nc,) + pm.shape) * 4e-5
    eps[:nd] += 2.5e-4
    if precision == 32:
        eps = eps.astype(np.float32).astype(np.float64)
    kt = np.sqrt(np.sum(positive_part(eps) ** 2, axis=0))
    kh = 0.7 * kt
    if precision == 32:
        kh = kh.astype(np.float32).astype(np.float64)
    orv = oracle.RVE(pm, _phases([MATRIX, STIFF]))
    assert ((kt > 1.2e-4) & (kt < 8e-4))[pm == 0].all()
    v = orv.G(rng.standard_normal((nc,) + pm.shape))
    ref = orv.G(consistent_tangent_apply(v, eps, kh, orv.params, sym=True))
    s = _solver(dims, pm, [MATRIX, STIFF], precision, hessian=1)
    s.set_state(_to_dev(eps, precision), _to_dev(kh, precision))
    out = s.hessp(_to_dev(v, precision)).cpu().numpy()
    sec = orv.G(orv.tangent(orv.stress(eps, kh)[1], v))
    assert _rel(ref, sec) > 1e-2  # the rank-one part matters here
    assert _rel(out, ref) < (4e-5 if precision == 32 else 1e-10), _rel(out, ref)
    s.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_consistent_load_path_matches_oracle(precision):
    """16x12x10 spheres, uniaxial eps_zz through the damage onset: the same
    equilibrium as the oracle with the consistent Hessian (and as the secant
    solver), with a Newton iteration count close to the oracle's."""
    from oracle.solver import TRParams, load_path
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    free = [1, 1, 0, 1, 1, 1]
    incs = [np.array([0, 0, 5e-5, 0, 0, 0]), np.array([0, 0, 2e-5, 0, 0, 0])]
    R0 = 10 * np.sqrt(pm.size) * 5e-5
    ref = load_path(ConsistentRVE(pm, _phases([MATRIX, STIFF]), free_mask=np.array(free, bool)), incs,
                    TRParams(eta_eq=1e-9, eta_cg=1e-3, R0=R0, Rmax=R0, max_nr=500))
    eta = 1e-9 if precision == 64 else 1e-6
    s = _solver(dims, pm, [MATRIX, STIFF], precision, hessian=1, eta_eq=eta, eta_cg=1e-3, R0=R0, Rmax=R0,
                max_nr=500)
    reps = [s.solve_step(dE, free_mask=free) for dE in incs]
    assert all(r["converged"] for r in reps)
    ms = np.array([r["mean_stress"][:6] for r in reps])
    tol = 1e-6 if precision == 64 else 1e-4
    assert np.max(np.abs(ms[:, 2] - ref["mean_stress"][:, 2]) / np.abs(ref["mean_stress"][:, 2])) < tol
    eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
    assert _rel(eps, ref["eps"]) < (1e-6 if precision == 64 else 1e-4)
    n_gpu = sum(r["nr_iters"] for r in reps)
    n_ref = sum(r.nr_iters for r in ref["reports"])
    assert n_gpu <= n_ref + 6 and n_gpu < 60, (n_gpu, n_ref)
    s.close()


def test_effective_stiffness_stays_secant_and_option_is_checked():
    from paper_2207_10657_gb300.binding import RveError
    dims = (12, 16, 10)
    pm = random_spheres(dims, count=3, rmin=1.5, rmax=3.0, seed=5)
    rng = np.random.default_rng(4)
    eps = rng.standard_normal((6,) + pm.shape) * 4e-5
    eps[:3] += 2.5e-4
    kh = 0.7 * np.sqrt(np.sum(positive_part(eps) ** 2, axis=0))
    cs = []
    for h in (0, 1):
        s = _solver(dims, pm, [MATRIX, STIFF], 64, hessian=h)
        s.set_state(_to_dev(eps, 64), _to_dev(kh, 64))
        cs.append(np.array(s.effective_stiffness(tol=1e-11)[0]))
        s.close()
    np.testing.assert_allclose(cs[1], cs[0], rtol=1e-9, atol=1e-14)
    with pytest.raises(RveError):
        _solver(dims, pm, [MATRIX, STIFF], 64, hessian=2)
