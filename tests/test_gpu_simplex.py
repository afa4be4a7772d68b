"""The linear-triangle (multi-quadrature-point) discretisation on the GPU
(rve_solver_opts.element = 1, 2D) against the FP64 oracle's SimplexRVE
(needs a GB300).

Every pixel is split along its main diagonal into the triangles of axis
order (x, y) and (y, x), one strain each (oracle/simplex.py).  Checked
through the C ABI, element by element: the projection (compiled passes at
32 / 64 / 128, generic passes at other lengths and in FP64), the
Hessian-vector product on a damage snapshot with one damage value per
triangle, an elastic load step under mixed control, and a load path through
the damage onset.  Tolerances as the voxel-element parity tests: 2e-6
relative L2 for single FP32 products, 1e-11 in FP64; solves at their
residual."""
import numpy as np
import pytest

import oracle
from oracle.simplex import SimplexRVE
from oracle.solver import TRParams, load_path
from synth import circular_inclusion, random_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.3, False, 0.0, 0.0)
TOL = {32: 2e-6, 64: 1e-11}
GRIDS = [(32, 32), (64, 32), (32, 128), (12, 10), (30, 40), (2, 2), (96, 48)]


def _solver(dims, pm, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, [MATRIX, STIFF], precision=precision, element=1, **kw)


def _orv(pm, free=None):
    return SimplexRVE(pm, [oracle.Phase(*MATRIX), oracle.Phase(STIFF[0], STIFF[1])], free_mask=free)


def _dev(a, precision):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32 if precision == 32 else np.float64)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", GRIDS)
def test_simplex_projection_matches_oracle(dims, precision):
    pm = circular_inclusion(dims, 0.3) if min(dims) >= 8 else np.zeros(tuple(reversed(dims)), np.uint8)
    s = _solver(dims, pm, precision)
    rng = np.random.default_rng(3)
    for free in (None, [1, 0, 1]):
        if free is not None:
            s.set_free_mask(free)
        v = rng.standard_normal((3, 2) + tuple(reversed(dims)))
        out = s.project(_dev(v, precision)).cpu().numpy()
        ref = _orv(pm, None if free is None else np.array(free, bool)).G(v)
        assert _rel(out, ref) < TOL[precision], (dims, free)
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(32, 32), (64, 32), (30, 40)])
def test_simplex_hessp_matches_oracle(dims, precision):
    pm = circular_inclusion(dims, 0.3)
    s = _solver(dims, pm, precision)
    rng = np.random.default_rng(5)
    D = np.where(pm[None] == 0, rng.uniform(0.0, 0.9, (2,) + pm.shape), 0.0)  # one damage per triangle
    D = D.astype(np.float32).astype(np.float64)
    s.set_damage(_dev(D, precision))
    orv = _orv(pm)
    v = orv.G(rng.standard_normal((3, 2) + pm.shape))
    v = v.astype(np.float32).astype(np.float64)
    out = s.hessp(_dev(v, precision)).cpu().numpy()
    ref = orv.hessp(D, v)
    assert _rel(out, ref) < TOL[precision]
    # symmetric on compatible fields
    w = orv.G(rng.standard_normal((3, 2) + pm.shape))
    hw = s.hessp(_dev(w, precision)).cpu().numpy()
    assert abs(np.sum(w * out) - np.sum(v * hw)) < 10 * TOL[precision] * np.linalg.norm(out) * np.linalg.norm(w)
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(32, 32), (30, 40)])
def test_simplex_elastic_step_matches_oracle(dims, precision):
    """An elastic load step (below the damage threshold) under mixed control
    on the triangles: mean stress and strain field against the oracle."""
    pm = circular_inclusion(dims, 0.3)
    free = [0, 1, 1]
    dE = [3e-5, 0.0, 0.0]
    npt = 2 * dims[0] * dims[1]
    R0 = 10 * np.sqrt(npt) * 3e-5
    tol = dict(eta_eq=1e-6 if precision == 32 else 1e-10, eta_cg=1e-2 if precision == 32 else 1e-10)
    s = _solver(dims, pm, precision, R0=R0, Rmax=R0, max_cg=2000, **tol)
    rep = s.solve_step(dE, free_mask=free)
    eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
    s.close()
    ref = load_path(_orv(pm, np.array(free, bool)), [np.array(dE)],
                    TRParams(eta_eq=1e-12, eta_cg=1e-12, R0=R0, Rmax=R0, max_cg=5000))
    assert rep["converged"] and ref["reports"][0].converged
    assert eps.shape == (3, 2) + pm.shape
    ms = np.array(rep["mean_stress"][:3])
    assert _rel(ms, ref["mean_stress"][0]) < (1e-5 if precision == 32 else 1e-10)
    assert _rel(eps, ref["eps"]) < (1e-4 if precision == 32 else 1e-9)


@pytest.mark.parametrize("precision", [32, 64])
def test_simplex_load_path_through_onset_matches_oracle(precision):
    """eps_xx += 4e-5 then += 2e-6 on a 32 x 32 centred inclusion (other
    components free): elastic, then damage starts on the triangles next to
    the inclusion (the next increment of 2e-6 already snaps back and needs
    more than 400 Newton iterations in the oracle, so the path stops here);
    mean stress per increment and the damaged set (kappa > kappa0 per
    triangle, excluding triangles within 1e-3 of it)."""
    dims = (32, 32)
    pm = circular_inclusion(dims, 0.3)
    free = [0, 1, 1]
    incs = [np.array([4e-5, 0.0, 0.0]), np.array([2e-6, 0.0, 0.0])]
    R0 = 10 * np.sqrt(2 * 32 * 32) * 4e-5
    eta = 1e-6 if precision == 32 else 1e-8
    s = _solver(dims, pm, precision, R0=R0, Rmax=R0, eta_eq=eta, eta_cg=1e-2, max_nr=400, max_cg=2000)
    sig = []
    for dE in incs:
        rep = s.solve_step(list(dE), free_mask=free)
        assert rep["converged"]
        sig.append(rep["mean_stress"][:3])
    kap = s.get_state()["kappa"].cpu().numpy().astype(np.float64)
    s.close()
    ref = load_path(_orv(pm, np.array(free, bool)), incs,
                    TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=400, max_cg=2000))
    assert all(r.converged for r in ref["reports"])
    scale = np.max(np.abs(ref["mean_stress"][:, 0]))
    for n in range(len(incs)):
        assert abs(sig[n][0] - ref["mean_stress"][n][0]) / scale < (1e-4 if precision == 32 else 1e-6), n
    k0 = 1e-4
    dmg, dref = kap > k0, ref["kappa"] > k0
    near = np.abs(ref["kappa"] - k0) <= 1e-3 * k0
    assert dref.sum() > 0
    assert np.array_equal(dmg & ~near, dref & ~near)
