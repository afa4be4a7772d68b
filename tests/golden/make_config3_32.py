"""Writes config3_32.json: the FP64 oracle's mixed load path of the third
configuration (shear and uniaxial strain ramped together) on its sphere
model scaled to a 32^3 cell, the stored reference of tests/test_gpu_curves.py.
Calls only oracle/ and synth/.

Cell: 32^3, 18 non-overlapping spheres of radius U[2, 5] (seed 0; three
times the second configuration's count), stiff elastic spheres E = 10,
nu = 0.2 in a damaging matrix E = 1, nu = 0.3, kappa0 = 1e-4, kappaf = 1e-3.
Each of the configuration's 40 increments adds eps_zz = 5e-5 and
eps_yz = 2.5e-5 (Mandel component sqrt2 * eps_yz), so that eps_zz and the
engineering shear reach 2e-3 together; the other four mean components are
stress-free.  Algorithm 2 with the symmetric consistent tangent as the
Hessian, relative residual 1e-8, at most 400 Newton iterations per
increment; the path is stored up to and including the first increment that
does not converge.

    python tests/golden/make_config3_32.py   (about ten minutes)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle.consistent import ConsistentRVE  # noqa: E402
from oracle.solver import TRParams, trust_region_step  # noqa: E402
from synth import random_spheres  # noqa: E402

N = 32
K0 = 1e-4
INC = [0.0, 0.0, 5e-5, np.sqrt(2.0) * 2.5e-5, 0.0, 0.0]
FREE = [1, 1, 0, 0, 1, 1]


def cell():
    return random_spheres((N, N, N), count=18, rmin=2.0, rmax=5.0, seed=0)


def main(max_incs=40):
    pm = cell()
    free = np.array(FREE, bool)
    rve = ConsistentRVE(pm, [oracle.Phase(1.0, 0.3, True, K0, 1e-3), oracle.Phase(10.0, 0.2)], free_mask=free)
    inc = np.array(INC)
    R = 10.0 * np.sqrt(N ** 3) * float(np.linalg.norm(inc))
    prm = TRParams(eta_eq=1e-8, eta_cg=1e-2, R0=R, Rmax=R, max_nr=400, max_cg=1000)
    eps = np.zeros((6,) + pm.shape)
    hist = np.zeros(pm.shape)
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(N ** 3, size=2048, replace=False))
    out = {"cell": "32^3, 18 spheres r~U[2,5] seed 0 (synth.random_spheres)", "increment": INC,
           "free_mask": FREE, "R0": R, "eta_eq": 1e-8, "max_nr": 400,
           "sample_points": sample.tolist(), "increments": []}
    for n in range(max_incs):
        eps = eps + inc.reshape(6, 1, 1, 1)
        eps, sig, kap, R, rep = trust_region_step(rve, eps, hist, R, prm)
        rec = {"n": n + 1, "converged": bool(rep.converged), "nr_iters": rep.nr_iters,
               "mean_stress": rve.mean(sig).tolist()}
        if rep.converged:
            hist = np.maximum(hist, kap)
            flat = hist.ravel()
            near = np.abs(flat - K0) <= 1e-3 * K0
            rec["damaged"] = np.flatnonzero((flat > K0) & ~near).tolist()
            rec["near_threshold"] = np.flatnonzero(near).tolist()
            rec["strain_sample"] = eps.reshape(6, -1)[:, sample].tolist()
        out["increments"].append(rec)
        print(n + 1, rep.converged, rep.nr_iters, rec["mean_stress"][2], rec["mean_stress"][3], flush=True)
        if not rep.converged:
            break
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_32.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
