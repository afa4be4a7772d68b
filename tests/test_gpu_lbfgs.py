"""L-BFGS load steps on the GPU (needs a GB300): the quasi-Newton solver with
the first-order incremental energy in its line search, against the FP64
oracle's L-BFGS (same algorithm, same decisions up to rounding), against the
trust-region solver's equilibrium at full size, and its argument checks."""
import numpy as np
import pytest

import oracle
from oracle.lbfgs import LBFGSParams, load_path_lbfgs
from synth import circular_inclusion, gel_sites, random_circles, random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)


def _solver(dims, pm, phases, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, phases, precision=precision, **kw)


def _oracle_rve(pm, phases, free=None):
    return oracle.RVE(pm, [oracle.Phase(*p) if p[2] else oracle.Phase(p[0], p[1]) for p in phases], free_mask=free)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("dims", [(32, 24), (12, 16, 10)])
def test_elastic_lbfgs_matches_oracle(dims, precision):
    """Elastic cell, general strain-controlled load: the converged strain
    field of the oracle's L-BFGS; in FP64 the iteration counts agree too.
    A second increment with another memory length reuses the context."""
    nd = len(dims)
    nc = 3 if nd == 2 else 6
    pm = circular_inclusion(dims, 0.3) if nd == 2 else random_spheres(dims, count=3, rmin=1.5, rmax=3.0, seed=5)
    phases = [(1.0, 0.3, False, 0.0, 0.0), STIFF]
    E = np.array([1e-3, -2e-4, 3e-4, 1e-4, 0.0, 2e-4][:nc])
    eta = 1e-10 if precision == 64 else 1e-6
    ref = load_path_lbfgs(_oracle_rve(pm, phases), [E, 0.5 * E], LBFGSParams(eta_eq=eta, m=5, max_iter=2000))
    s = _solver(dims, pm, phases, precision, eta_eq=eta)
    r1 = s.solve_step_lbfgs(E, memory=5, max_iter=2000)
    r2 = s.solve_step_lbfgs(0.5 * E, memory=5, max_iter=2000)
    assert r1["converged"] and r2["converged"]
    eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
    assert _rel(eps, ref["eps"]) < (1e-8 if precision == 64 else 1e-4)
    if precision == 64:
        assert abs(r1["nr_iters"] - ref["reports"][0].iters) <= 2, (r1["nr_iters"], ref["reports"][0].iters)
    # another memory length on the same context
    r3 = s.solve_step_lbfgs(0.25 * E, memory=9, max_iter=2000)
    assert r3["converged"]
    s.close()


def test_lbfgs_damage_onset_fp32_matches_oracle():
    """16x12x10 spheres in a damaging matrix, uniaxial eps_zz (the rest
    free), two increments that damage the matrix: FP32 fields within 1e-4 of
    the oracle's L-BFGS, the same damaged voxels."""
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    phases = [MATRIX, STIFF]
    free = [1, 1, 0, 1, 1, 1]
    incs = [np.array([0, 0, 5e-5, 0, 0, 0]), np.array([0, 0, 2e-5, 0, 0, 0])]
    ref = load_path_lbfgs(_oracle_rve(pm, phases, np.array(free, bool)), incs,
                          LBFGSParams(eta_eq=1e-9, m=8, max_iter=3000))
    s = _solver(dims, pm, phases, 32, eta_eq=1e-6)
    reps = [s.solve_step_lbfgs(dE, free_mask=free, memory=8, max_iter=3000) for dE in incs]
    assert all(r["converged"] for r in reps)
    ms = np.array([r["mean_stress"][:6] for r in reps])
    assert np.max(np.abs(ms[:, 2] - ref["mean_stress"][:, 2]) / np.abs(ref["mean_stress"][:, 2])) < 1e-4
    st = s.get_state()
    assert _rel(st["eps"].cpu().numpy().astype(np.float64), ref["eps"]) < 1e-4
    kap = st["kappa"].cpu().numpy().astype(np.float64)
    near = np.abs(ref["kappa"] - 1e-4) <= 1e-3 * 1e-4
    assert (ref["kappa"] > 1e-4).any()
    assert np.array_equal((kap > 1e-4)[~near], (ref["kappa"] > 1e-4)[~near])
    s.close()


def test_lbfgs_with_gel_eigenstrain_2d_fp64():
    """The ASR-like 2D cell (gel voxels expanding, free expansion) through
    two increments by L-BFGS, against the oracle's L-BFGS."""
    dims = (32, 32)
    pm = gel_sites(random_circles(dims, 0.4, rmin=3.0, rmax=6.0, seed=6), 6, seed=7)
    phases = [(12.0, 0.3, True, 2.5e-4, 2.5e-3), (59.0, 0.3, True, 10.0 / 59000.0, 100.0 / 59000.0),
              (11.0, 0.18, False, 0.0, 0.0)]
    tables = []
    for n in (1, 2):
        t = np.zeros((3, 3))
        t[2, :2] = -n * 5e-4
        tables.append(t)
    orv = _oracle_rve(pm, phases, np.ones(3, bool))
    ref = load_path_lbfgs(orv, [np.zeros(3)] * 2, LBFGSParams(eta_eq=1e-9, m=8, max_iter=5000), eigenstrains=tables)
    s = _solver(dims, pm, phases, 64, eta_eq=1e-9)
    reps = []
    for t in tables:
        s.set_eigenstrain(t)
        reps.append(s.solve_step_lbfgs(np.zeros(3), free_mask=[1, 1, 1], memory=8, max_iter=5000))
    assert all(r["converged"] for r in reps)
    st = s.get_state()
    assert _rel(st["eps"].cpu().numpy(), ref["eps"]) < 1e-6
    np.testing.assert_allclose(np.array([r["mean_strain"][:3] for r in reps]), ref["mean_strain"], rtol=1e-6,
                               atol=1e-12)
    s.close()


def test_lbfgs_reaches_trust_region_equilibrium_128cube_fp32():
    """The elastic first increment of the sphere-cell load path at 128^3:
    L-BFGS and trust-region Newton-CG end at the same equilibrium."""
    dims = (128, 128, 128)
    pm = random_spheres(dims, count=48, rmin=4.0, rmax=10.0, seed=0)
    phases = [MATRIX, STIFF]
    free = [1, 1, 0, 1, 1, 1]
    dE = [0.0, 0.0, 5e-5, 0.0, 0.0, 0.0]
    sa = _solver(dims, pm, phases, 32, eta_eq=1e-6)
    ra = sa.solve_step_lbfgs(dE, free_mask=free, memory=5, max_iter=1000)
    sb = _solver(dims, pm, phases, 32, eta_eq=1e-6, eta_cg=1e-2)
    rb = sb.solve_step(dE, free_mask=free)
    assert ra["converged"] and rb["converged"]
    assert abs(ra["mean_stress"][2] - rb["mean_stress"][2]) <= 1e-5 * abs(rb["mean_stress"][2])
    ea, eb = sa.get_state()["eps"], sb.get_state()["eps"]
    assert float(torch.linalg.vector_norm((ea - eb).double()) / torch.linalg.vector_norm(eb.double())) < 1e-4
    assert ra["hv_products"] == 0 and ra["cg_iters"] >= ra["nr_iters"]
    sa.close()
    sb.close()


def test_lbfgs_rejects_bad_arguments():
    from paper_2207_10657_gb300.binding import RveError
    pm = np.zeros((8, 8), np.uint8)
    s = _solver((8, 8), pm, [(1.0, 0.3, False, 0.0, 0.0)], 32)
    for mem, it in ((0, 10), (17, 10), (5, 0)):
        with pytest.raises(RveError):
            s.solve_step_lbfgs([1e-4, 0, 0], memory=mem, max_iter=it)
    s.close()
