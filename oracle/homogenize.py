"""Effective (homogenised) secant stiffness of the cell at a frozen damage
field (oracle).  TEST INFRASTRUCTURE ONLY, like the rest of this package.

Sec. 3.3 reports the deterioration of the cell as the ratio of the norms of
the effective stiffness tensor during ASR expansion and of the intact cell,
||C_bar|| / ||C_bar_0||.  The paper does not print how C_bar is formed;
reading (first-order homogenisation of the linearised cell problem, with the
secant stiffness B = (1 - D) C the solver's Hessian uses):

* for every Mandel unit mean strain e_j, find the compatible zero-mean
  fluctuation x_j with G : B : (e_j + x_j) = 0 (every mean component
  strain-controlled, Ghat(0) = 0), by CG on the Hessian-vector product of
  Eq. (8) (Steihaug CG of Algorithm 1 without a radius);
* column j of C_bar is the volume average <B : (e_j + x_j)>;
* ||C_bar|| is the Frobenius norm of the Mandel matrix.
"""
import math

import numpy as np

from .solver import steihaug_cg


def effective_stiffness(rve, D, tol=1e-12, max_iter=20000):
    """C_bar (ncomp x ncomp Mandel matrix) at frozen damage D; ``tol`` is
    the relative CG residual."""
    nc = rve.ncomp
    C = np.zeros((nc, nc))
    saved = rve.free_mask
    rve.free_mask = np.zeros(nc, dtype=bool)
    try:
        for j in range(nc):
            e = np.zeros((nc,) + rve.shape)
            e[j] = 1.0
            g = rve.hessp(D, e)
            gn = rve.norm(g)
            z = np.zeros_like(e)
            if gn > 0.0:
                z, info = steihaug_cg(lambda v: rve.hessp(D, v), g, math.inf, tol * gn, max_iter, rve.dot)
                if info["reason"] not in ("converged", "zero_rhs"):
                    raise RuntimeError(f"effective stiffness: CG ended with {info['reason']}")
            C[:, j] = rve.mean(rve.tangent(D, e + z))
    finally:
        rve.free_mask = saved
    return C
