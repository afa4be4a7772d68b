"""The linear-tetrahedron (multi-quadrature-point) discretisation on the GPU
(rve_solver_opts.element = 1, 3D) against the FP64 oracle's SimplexRVE
(needs a GB300).

Every voxel is split along its main diagonal into the six Kuhn tetrahedra
of the permutations of (x, y, z), one strain each (oracle/simplex.py); the
spectral passes transform 36 lines per voxel and solve a 3 x 3 Hermitian
system per frequency.  Checked through the C ABI, element by element: the
projection (with and without stress-controlled components, on grids with
odd-sized half spectra, 2-point axes and a ragged tile), the
Hessian-vector product on a damage snapshot with one damage value per
tetrahedron, an elastic load step under mixed control, and a load path
through the damage onset.  Tolerances as the voxel-element parity tests:
2e-6 relative L2 for single FP32 products, 1e-11 in FP64; solves at their
residual."""
import numpy as np
import pytest

import oracle
from oracle.simplex import SimplexRVE
from oracle.solver import TRParams, load_path

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
TOL = {32: 2e-6, 64: 1e-11}
GRIDS = [(8, 6, 4), (12, 10, 8), (16, 16, 16), (6, 4, 10), (2, 2, 2), (32, 8, 6), (10, 30, 12)]


def _sphere(dims, r):
    """One centred sphere of radius r (voxel centres inside get phase 1)."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    return (((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2) <= r * r).astype(np.uint8)


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
def test_tet_projection_matches_oracle(dims, precision):
    pm = _sphere(dims, min(dims) / 3) if min(dims) >= 4 else np.zeros(tuple(reversed(dims)), np.uint8)
    s = _solver(dims, pm, precision)
    assert s.nq == 6
    rng = np.random.default_rng(3)
    for free in (None, [1, 0, 0, 0, 1, 1]):
        if free is not None:
            s.set_free_mask(free)
        v = rng.standard_normal((6, 6) + tuple(reversed(dims)))
        out = s.project(_dev(v, precision)).cpu().numpy()
        ref = _orv(pm, None if free is None else np.array(free, bool)).G(v)
        assert _rel(out, ref) < TOL[precision], (dims, free)
        # a projector: G(G v) = G v
        out2 = s.project(_dev(out, precision)).cpu().numpy()
        assert _rel(out2, out) < TOL[precision], (dims, free)
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("dims", [(12, 10, 8), (16, 16, 16)])
def test_tet_hessp_matches_oracle(dims, precision):
    pm = _sphere(dims, min(dims) / 3)
    s = _solver(dims, pm, precision)
    rng = np.random.default_rng(5)
    D = np.where(pm[None] == 0, rng.uniform(0.0, 0.9, (6,) + pm.shape), 0.0)  # one damage per tetrahedron
    D = D.astype(np.float32).astype(np.float64)
    s.set_damage(_dev(D, precision))
    orv = _orv(pm)
    v = orv.G(rng.standard_normal((6, 6) + pm.shape))
    v = v.astype(np.float32).astype(np.float64)
    out = s.hessp(_dev(v, precision)).cpu().numpy()
    ref = orv.hessp(D, v)
    assert _rel(out, ref) < TOL[precision]
    # symmetric on compatible fields
    w = orv.G(rng.standard_normal((6, 6) + pm.shape))
    hw = s.hessp(_dev(w, precision)).cpu().numpy()
    assert abs(np.sum(w * out) - np.sum(v * hw)) < 10 * TOL[precision] * np.linalg.norm(out) * np.linalg.norm(w)
    s.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_tet_elastic_step_matches_oracle(precision):
    """An elastic load step (below the damage threshold) under mixed control
    on the tetrahedra of a 10 x 8 x 6 cell with a centred sphere: mean stress
    and strain field against the oracle."""
    dims = (10, 8, 6)
    pm = _sphere(dims, 2.2)
    free = [0, 1, 1, 1, 1, 1]
    dE = [3e-5, 0.0, 0.0, 0.0, 0.0, 0.0]
    npt = 6 * 10 * 8 * 6
    R0 = 10 * np.sqrt(npt) * 3e-5
    tol = dict(eta_eq=1e-6 if precision == 32 else 1e-10, eta_cg=1e-2 if precision == 32 else 1e-10)
    s = _solver(dims, pm, precision, R0=R0, Rmax=R0, max_cg=2000, **tol)
    rep = s.solve_step(dE, free_mask=free)
    eps = s.get_state()["eps"].cpu().numpy().astype(np.float64)
    s.close()
    ref = load_path(_orv(pm, np.array(free, bool)), [np.array(dE)],
                    TRParams(eta_eq=1e-12, eta_cg=1e-12, R0=R0, Rmax=R0, max_cg=5000))
    assert rep["converged"] and ref["reports"][0].converged
    assert eps.shape == (6, 6) + pm.shape
    ms = np.array(rep["mean_stress"][:6])
    assert _rel(ms, ref["mean_stress"][0]) < (1e-5 if precision == 32 else 1e-10)
    assert _rel(eps, ref["eps"]) < (1e-4 if precision == 32 else 1e-9)


@pytest.mark.parametrize("precision", [32, 64])
def test_tet_load_path_through_onset_matches_oracle(precision):
    """Uniaxial eps_zz += 5e-5 then += 1e-5 (other components free) on an
    8^3 cell with a centred stiff sphere: elastic, then damage starts on
    tetrahedra next to the sphere; mean stress per increment and the damaged
    set (kappa > kappa0 per tetrahedron, excluding tetrahedra within 1e-3 of
    it)."""
    dims = (8, 8, 8)
    pm = _sphere(dims, 2.0)
    free = [1, 1, 0, 1, 1, 1]
    incs = [np.array([0, 0, 5e-5, 0, 0, 0.0]), np.array([0, 0, 1e-5, 0, 0, 0.0])]
    R0 = 10 * np.sqrt(6 * 512) * 5e-5
    eta = 1e-6 if precision == 32 else 1e-8
    s = _solver(dims, pm, precision, R0=R0, Rmax=R0, eta_eq=eta, eta_cg=1e-2, max_nr=400, max_cg=2000)
    sig = []
    for dE in incs:
        rep = s.solve_step(list(dE), free_mask=free)
        assert rep["converged"]
        sig.append(rep["mean_stress"][:6])
    kap = s.get_state()["kappa"].cpu().numpy().astype(np.float64)
    s.close()
    ref = load_path(_orv(pm, np.array(free, bool)), incs,
                    TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R0, Rmax=R0, max_nr=400, max_cg=2000))
    assert all(r.converged for r in ref["reports"])
    scale = np.max(np.abs(ref["mean_stress"][:, 2]))
    for n in range(len(incs)):
        assert abs(sig[n][2] - ref["mean_stress"][n][2]) / scale < (1e-4 if precision == 32 else 1e-6), n
    k0 = 1e-4
    dmg, dref = kap > k0, ref["kappa"] > k0
    near = np.abs(ref["kappa"] - k0) <= 1e-3 * k0
    assert dref.sum() > 0
    assert np.array_equal(dmg & ~near, dref & ~near)


def test_tet_grid_limits():
    """The generic passes hold the 36 lines of one x row / one z column per
    block: rve_create refuses larger rows and columns with RVE_ERR_ARG."""
    from paper_2207_10657_gb300 import RVESolver, build
    from paper_2207_10657_gb300.binding import RveError
    build.build()
    for dims, prec in (((256, 8, 8), 32), ((8, 8, 384), 32), ((8, 8, 192), 64)):
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        with pytest.raises(RveError, match="element 1 in 3D"):
            RVESolver(dims, pm, [MATRIX], precision=prec, element=1)
    # the largest admitted sizes are created
    for dims, prec in (((216, 4, 4), 32), ((4, 4, 320), 32), ((4, 4, 160), 64)):
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        RVESolver(dims, pm, [MATRIX], precision=prec, element=1).close()
