"""Periodic 1D three-spring system of Sec. 3.1 (oracle).

Three nodes on a periodic line, springs k (node 0-1), k (node 1-2) and the
damage spring k0 closing the period (node 2 - node 0).  After its threshold
gamma0 the damage spring softens with tangent alpha*k, so the post-peak
nodal stiffness is Eq. (21) with eigenvalues 0, 3k and (2 alpha + 1) k.

Reading (the figure with the geometry is missing): the problem is posed in
"strain" space like the RVE -- the unknowns are the three spring
elongations gamma with the mean stretch imposed, sum(gamma) = 3 xbar; the
compatible fluctuations are the zero-sum vectors, so G = I - 1 1^T / 3.
The damage spring is treated as non-linear elastic (no unloading history),
which makes its energy explicit and the standard trust region applicable:
f(gamma) = k gamma up to gamma0, k gamma0 + alpha k (gamma - gamma0) after,
and (for alpha < 0) zero once that reaches zero.
"""
import numpy as np


class Spring1D:
    def __init__(self, k=1.0, gamma0=0.1, alpha=-1.0):
        self.k, self.gamma0, self.alpha = float(k), float(gamma0), float(alpha)
        self.ncomp = 1
        self.shape = (3,)
        self.ndim = 1

    # incidence of elongations on nodal displacements: gamma = B u (+ mean)
    B = np.array([[-1.0, 1.0, 0.0], [0.0, -1.0, 1.0], [1.0, 0.0, -1.0]])

    def _damage_force(self, g):
        k, g0, a = self.k, self.gamma0, self.alpha
        if g <= g0:
            return k * g, k
        f = k * g0 + a * k * (g - g0)
        if a < 0.0 and f <= 0.0:
            return 0.0, 0.0
        return f, a * k

    def _damage_energy(self, g):
        k, g0, a = self.k, self.gamma0, self.alpha
        if g <= g0:
            return 0.5 * k * g * g
        e0 = 0.5 * k * g0 * g0
        if a < 0.0:
            g_end = g0 - g0 / a  # force reaches zero
            gg = min(g, g_end)
        else:
            gg = g
        t = gg - g0
        return e0 + k * g0 * t + 0.5 * a * k * t * t

    def stiffnesses(self, gamma):
        return np.array([self.k, self.k, self._damage_force(gamma[2])[1]])

    def nodal_stiffness(self, gamma):
        """K = B^T diag(k_s) B (Eq. (21) in the post-peak range)."""
        return self.B.T @ np.diag(self.stiffnesses(gamma)) @ self.B

    # -- problem interface used by the generic solver ---------------------
    def stress(self, gamma, hist=None):
        f = np.array([self.k * gamma[0], self.k * gamma[1], self._damage_force(gamma[2])[0]])
        return f, self.stiffnesses(gamma), None

    @staticmethod
    def gradient(f):
        return f - f.mean()

    def G(self, x):
        return x - x.mean()

    def tangent(self, kt, v):
        return kt * v

    def hessp(self, kt, v):
        return self.G(kt * v)

    def energy(self, gamma, hist=None):
        return 0.5 * self.k * (gamma[0] ** 2 + gamma[1] ** 2) + self._damage_energy(gamma[2])

    @staticmethod
    def dot(a, b):
        return float(np.dot(a, b))

    def norm(self, a):
        return float(np.sqrt(np.dot(a, a)))

    def mean(self, f):
        return np.array([f.mean()])
