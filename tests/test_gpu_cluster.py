"""The cluster passes: the x and y transforms of each direction of the 3D
FP32 product in one pass (clusters of four CTAs holding one component of a
z-plane, the y transform split 4 x N/4 across their shared memories;
Nx = Ny in {64, 96, 128, 192, 256}; rve_solver_opts.passes = 3), needs a
GB300.

Checked through the C ABI, element by element: the projection (with and
without stress-controlled components) and the Hessian-vector product on a
damage snapshot against the FP64 oracle at the FP32 parity tolerance of the
other passes (2e-6 / 1e-5 relative L2), and against the five separate
compiled passes (the default passes = 0) on the same input, and one
load step (gradient with its norm, device-side Steihaug loop) against the
same step on the five passes.  Grids cover every cluster length, thin z
(4 planes) and the odd half-spectrum width N/2 + 1.  The fused Steihaug-CG
update of the inverse cluster pass, and its dot product with a second field
are compared with the oracle's steihaug_cg in tests/test_gpu_steihaug.py
(passes = 3 on the 64 x 64 x 16 cell)."""
import numpy as np
import pytest

import oracle
from synth import random_spheres, damage_snapshot, random_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
GRIDS = [(64, 64, 16), (96, 96, 8), (128, 128, 6), (192, 192, 4), (256, 256, 4), (64, 64, 64)]


def _solver(dims, pm, passes=3):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, [MATRIX, STIFF], precision=32, passes=passes)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("dims", GRIDS)
def test_cluster_projection_matches_oracle_and_five_pass(dims):
    pm = random_spheres(dims, count=4, rmin=1.5, rmax=3.0, seed=2)
    s, s5 = _solver(dims, pm), _solver(dims, pm, passes=0)
    for free in (None, [1, 0, 0, 0, 1, 1]):
        if free is not None:
            s.set_free_mask(free)
            s5.set_free_mask(free)
        v = random_field(6, dims, seed=7)
        out = s.project(_dev(v)).cpu().numpy()
        out5 = s5.project(_dev(v)).cpu().numpy()
        ref = oracle.project(v, None if free is None else np.array(free, bool))
        assert _rel(out, ref) < 2e-6, (dims, free)
        assert _rel(out, out5) < 2e-6, (dims, free)
    s.close()
    s5.close()


@pytest.mark.parametrize("dims", GRIDS)
def test_cluster_hessp_matches_oracle_and_five_pass(dims):
    pm = random_spheres(dims, count=4, rmin=1.5, rmax=3.0, seed=4)
    D = damage_snapshot(pm, dmax=0.9, seed=1)
    s, s5 = _solver(dims, pm), _solver(dims, pm, passes=0)
    s.set_damage(_dev(D))
    s5.set_damage(_dev(D))
    v = random_field(6, dims, seed=2)
    out = s.hessp(_dev(v)).cpu().numpy()
    out5 = s5.hessp(_dev(v)).cpu().numpy()
    ref = oracle.RVE(pm, [oracle.Phase(*MATRIX), oracle.Phase(STIFF[0], STIFF[1])]).hessp(D.astype(np.float64), v)
    assert _rel(out, ref) < 1e-5
    assert _rel(out, out5) < 2e-6
    # in-place (aliased) call
    x = _dev(v)
    s.hessp(x, out=x)
    assert _rel(x.cpu().numpy(), ref) < 1e-5
    s.close()
    s5.close()


def test_cluster_load_step_matches_five_pass():
    """One elastic load step at 128 x 128 x 32 (device-side Steihaug loop on
    the cluster passes) against the same step on the five passes: the same
    Newton and CG iteration counts, mean stress to 1e-6, strain field to
    1e-5 relative L2."""
    dims = (128, 128, 32)
    pm = random_spheres(dims, count=12, rmin=3.0, rmax=6.0, seed=5)
    out = []
    for passes in (3, 0):
        s = _solver(dims, pm, passes=passes)
        rep = s.solve_step([0, 0, 5e-5, 0, 0, 0], free_mask=[1, 1, 0, 1, 1, 1])
        out.append((rep, s.get_state()["eps"].cpu().numpy().astype(np.float64)))
        s.close()
    (r0, e0), (r3, e3) = out
    assert r0["converged"] and r3["converged"]
    assert r0["nr_iters"] == r3["nr_iters"] and r0["cg_iters"] == r3["cg_iters"]
    assert _rel(np.array(r0["mean_stress"]), np.array(r3["mean_stress"])) < 1e-6
    assert _rel(e0, e3) < 1e-5
