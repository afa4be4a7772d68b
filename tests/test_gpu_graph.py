"""The Steihaug-CG iterations run on the device (a CUDA graph whose WHILE
node repeats Algorithm 1's iteration until an exit or a restart) and give
the same load steps as the host-stepped loop (needs a GB300).

The host-stepped loop is selected with rve_set_device_loop(h, 0): both run
the same kernels in the same order, so the
reports (Newton and CG iteration counts, restarts, rejections) must be
identical and the stresses equal to the last bit in FP64 and to FP32
rounding in FP32; the device loop must wait on the host far less (about
twice per Steihaug solve plus once per restart, instead of once per
iteration)."""
import numpy as np
import pytest

from synth import circular_inclusion, random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)


def _path(dims, pm, phases, incs, free, precision, host_stepped, **opts):
    from paper_2207_10657_gb300 import RVESolver, binding, build
    build.build()
    s = RVESolver(dims, pm, phases, precision=precision, **opts)
    if host_stepped:
        binding.rve_set_device_loop(s.h, False)
    reps, s0 = [], s.sync_count
    for dE in incs:
        reps.append(s.solve_step(dE, free_mask=free, raise_on_error=False))
    syncs = s.sync_count - s0
    eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
    s.close()
    return reps, syncs, eps


CASES = [
    # 2D config-1 cell through the damage onset (compiled passes, fused CG)
    ((32, 32), "disc", [[1e-4, 0, 0]] * 3, [0, 1, 1], 32, dict(max_nr=400, max_cg=500)),
    ((32, 32), "disc", [[1e-4, 0, 0]] * 3, [0, 1, 1], 64, dict(max_nr=400, max_cg=500, eta_eq=1e-8, eta_cg=1e-10)),
    # 3D spheres, compiled 32^3 and a generic 16x12x10 grid, secant and consistent Hessians
    ((32, 32, 32), "spheres", [[0, 0, 4e-5, 0, 0, 0]] * 2, [1, 1, 0, 1, 1, 1], 32, dict(max_nr=300)),
    ((32, 32, 32), "spheres", [[0, 0, 4e-5, 0, 0, 0]] * 2, [1, 1, 0, 1, 1, 1], 32, dict(max_nr=300, hessian=1)),
    ((16, 12, 10), "spheres", [[0, 0, 4e-5, 0, 0, 0]] * 2, [1, 1, 0, 1, 1, 1], 64, dict(max_nr=300)),
]


@pytest.mark.parametrize("dims,kind,incs,free,precision,opts", CASES)
def test_device_loop_matches_host_loop(dims, kind, incs, free, precision, opts):
    if kind == "disc":
        pm = circular_inclusion(dims, 0.3)
        phases = [MATRIX, (10.0, 0.3, False, 0.0, 0.0)]
    else:
        pm = random_spheres(dims, count=6, rmin=2.0, rmax=4.0, seed=7)
        phases = [MATRIX, (10.0, 0.2, False, 0.0, 0.0)]
    R0 = 10 * np.sqrt(np.prod(dims)) * float(np.linalg.norm(incs[0]))
    opts = dict(opts, R0=R0, Rmax=R0)
    dev, sync_dev, eps_dev = _path(dims, pm, phases, incs, free, precision, False, **opts)
    host, sync_host, eps_host = _path(dims, pm, phases, incs, free, precision, True, **opts)
    keys = ("nr_iters", "cg_iters", "hv_products", "restarts", "rejected", "boundary_hits", "converged", "status")
    for a, b in zip(dev, host):
        assert {k: a[k] for k in keys} == {k: b[k] for k in keys}
        tol = 0.0 if precision == 64 else 1e-6
        np.testing.assert_allclose(a["mean_stress"], b["mean_stress"], rtol=tol, atol=0)
    assert np.array_equal(eps_dev, eps_host) or precision == 32
    assert float(np.linalg.norm(eps_dev - eps_host) / np.linalg.norm(eps_host)) < (1e-14 if precision == 64 else 1e-6)
    cg = sum(r["cg_iters"] for r in host)
    print(f"\n{dims} P{precision}: CG iterations {cg}, host waits {sync_host} (host-stepped) -> {sync_dev} (device loop)")
    assert sync_dev < sync_host
    assert sync_host - sync_dev >= cg - 2 * sum(r["nr_iters"] for r in host) - sum(r["restarts"] for r in host)
