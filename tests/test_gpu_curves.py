"""Stress-strain curves on the GPU against closed forms and stored oracle
paths (needs a GB300).

* The bilayer laminate of the third configuration (normal to z, 50/50, the
  damaging matrix and the stiff elastic phase) loaded along its layers
  (eps_xx, the other mean components stress-free) through the whole
  softening branch of the damaging layer (damage up to 0.99): every
  increment's mean stress and transverse strain against the closed form of
  tests/test_oracle_solver.py (which pins the oracle on the same path), at
  32^3 (compiled passes) in FP32 and FP64 and at 64^3 in FP32.
* The second configuration's sphere model on a 32^3 cell in its increments
  of 4e-5 against the oracle's path stored by tests/golden/make_config2_32.py
  (FP64, relative residual 1e-8), with the plain (secant) Hessian in FP32 and
  the consistent one in FP64: mean stress per increment (1e-5 relative in
  the elastic range, 1e-4 along damage), the strain field at 2048 stored
  points (1e-4 relative L2) and the damaged-voxel set (identical except
  voxels within 1e-3 of kappa0), up to the first increment the oracle does
  not converge within 400 Newton iterations (a snap-back); that increment
  is run on the GPU too and its outcome printed (pytest -s).
* The third configuration's mixed path (eps_zz and eps_yz ramped together,
  the other four components stress-free) on its sphere model (three times
  the spheres) at 32^3 against tests/golden/make_config3_32.py's stored
  oracle path in the same way, with both stressed components (zz, yz)
  compared per increment.
"""
import json
import os

import numpy as np
import pytest

import oracle
from synth import laminate
from tests.test_oracle_solver import _laminate_parallel_softening

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config2_32.json")
GOLDEN3 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config3_32.json")


def _solver(dims, pm, precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, [MATRIX, STIFF], precision=precision, **kw)


@pytest.mark.parametrize("n,precision", [(32, 32), (32, 64), (64, 32)])
def test_laminate_parallel_softening_curve(n, precision):
    dims = (n, n, n)
    pm = laminate(dims, axis=2)
    inc = 4.5e-5
    R0 = 10 * np.sqrt(n ** 3) * inc
    eta = 1e-6 if precision == 32 else 1e-10
    s = _solver(dims, pm, precision, R0=R0, Rmax=R0, eta_eq=eta, eta_cg=1e-2, max_nr=200)
    pa, pb = oracle.Phase(*MATRIX), oracle.Phase(STIFF[0], STIFF[1])
    tol = 1e-5 if precision == 32 else 1e-9
    peak = 0.0
    rows = []
    for k in range(20):
        rep = s.solve_step([inc, 0, 0, 0, 0, 0], free_mask=[0, 1, 1, 1, 1, 1])
        assert rep["converged"], k
        sxx, e = _laminate_parallel_softening(pa, pb, (k + 1) * inc)
        peak = max(peak, abs(sxx))
        rows.append((k + 1, sxx, rep["mean_stress"][0], rep["mean_strain"][1], e))
        assert abs(rep["mean_stress"][0] - sxx) <= tol * peak, (k, rep["mean_stress"][0], sxx)
        assert abs(rep["mean_strain"][1] - e) <= tol * abs(e) * 10, (k, rep["mean_strain"][1], e)
    st = s.get_state()
    kap = st["kappa"].cpu().numpy()
    s.close()
    print(f"\n{n}^3 FP{precision}: increment, sigma_xx closed form, GPU")
    for r in rows:
        print(f"  {r[0]:2d}  {r[1]: .9e}  {r[2]: .9e}")
    # the damaging layer holds one uniform kappa = eps_xx, the elastic one none
    np.testing.assert_allclose(kap[: n // 2], 20 * inc, rtol=1e-5 if precision == 32 else 1e-12)
    assert np.all(kap[n // 2:] == 0)


@pytest.mark.parametrize("precision,hessian", [(32, 0), (64, 1)])
def test_config2_path_32cube_matches_stored_oracle(precision, hessian):
    import sys
    sys.path.insert(0, os.path.dirname(GOLDEN))
    from make_config2_32 import cell, INC, K0
    with open(GOLDEN) as f:
        ref = json.load(f)
    pm = cell()
    R0 = ref["R0"]
    eta = 1e-6 if precision == 32 else 1e-8
    s = _solver((32, 32, 32), pm, precision, R0=R0, Rmax=R0, eta_eq=eta, eta_cg=1e-2, max_nr=400,
                max_cg=1000, hessian=hessian)
    sample = np.array(ref["sample_points"])
    print(f"\nFP{precision} hessian={hessian}: increment, oracle sigma_zz, GPU sigma_zz, Newton (oracle, GPU)")
    scale = 0.0
    for rec in ref["increments"]:
        rep = s.solve_step([0, 0, INC, 0, 0, 0], free_mask=ref["free_mask"], raise_on_error=False)
        so, sg = rec["mean_stress"], rep["mean_stress"]
        print(f"  {rec['n']}  {so[2]: .9e}  {sg[2]: .9e}  ({rec['nr_iters']}, {rep['nr_iters']}) "
              f"converged ({rec['converged']}, {rep['converged']})")
        if not rec["converged"]:
            break  # the oracle's snap-back: no reference for this increment
        assert rep["converged"]
        scale = max(scale, abs(so[2]))
        damaged = len(rec["damaged"]) > 0
        rel = abs(sg[2] - so[2]) / scale
        assert rel < (1e-4 if damaged else 1e-5), (rec["n"], rel)
        st = s.get_state()
        eps = st["eps"].cpu().numpy().astype(np.float64).reshape(6, -1)[:, sample]
        eref = np.array(rec["strain_sample"])
        assert np.linalg.norm(eps - eref) / np.linalg.norm(eref) < 1e-4
        kap = st["kappa"].cpu().numpy().astype(np.float64).ravel()
        near = np.zeros(kap.size, bool)
        near[rec["near_threshold"]] = True
        got = np.flatnonzero((kap > K0) & ~near)
        assert np.array_equal(got, np.array(rec["damaged"], dtype=got.dtype)), (rec["n"], got.size, len(rec["damaged"]))
    s.close()


@pytest.mark.parametrize("precision,hessian", [(32, 0), (64, 1)])
def test_config3_mixed_path_32cube_matches_stored_oracle(precision, hessian):
    import sys
    sys.path.insert(0, os.path.dirname(GOLDEN3))
    from make_config3_32 import cell, INC, K0
    with open(GOLDEN3) as f:
        ref = json.load(f)
    pm = cell()
    R0 = ref["R0"]
    eta = 1e-6 if precision == 32 else 1e-8
    s = _solver((32, 32, 32), pm, precision, R0=R0, Rmax=R0, eta_eq=eta, eta_cg=1e-2, max_nr=400,
                max_cg=1000, hessian=hessian)
    sample = np.array(ref["sample_points"])
    print(f"\nFP{precision} hessian={hessian}: increment, oracle (sigma_zz, sigma_yz), GPU, Newton (oracle, GPU)")
    scale = np.zeros(2)
    for rec in ref["increments"]:
        rep = s.solve_step(list(INC), free_mask=ref["free_mask"], raise_on_error=False)
        so, sg = np.array(rec["mean_stress"])[[2, 3]], np.array(rep["mean_stress"])[[2, 3]]
        print(f"  {rec['n']}  {so}  {sg}  ({rec['nr_iters']}, {rep['nr_iters']}) "
              f"converged ({rec['converged']}, {rep['converged']})")
        if not rec["converged"]:
            break  # the oracle's snap-back: no reference for this increment
        assert rep["converged"]
        scale = np.maximum(scale, np.abs(so))
        damaged = len(rec["damaged"]) > 0
        rel = np.abs(sg - so) / scale
        assert np.all(rel < (1e-4 if damaged else 1e-5)), (rec["n"], rel)
        st = s.get_state()
        eps = st["eps"].cpu().numpy().astype(np.float64).reshape(6, -1)[:, sample]
        eref = np.array(rec["strain_sample"])
        assert np.linalg.norm(eps - eref) / np.linalg.norm(eref) < 1e-4
        kap = st["kappa"].cpu().numpy().astype(np.float64).ravel()
        near = np.zeros(kap.size, bool)
        near[rec["near_threshold"]] = True
        got = np.flatnonzero((kap > K0) & ~near)
        assert np.array_equal(got, np.array(rec["damaged"], dtype=got.dtype)), (rec["n"], got.size, len(rec["damaged"]))
    s.close()
