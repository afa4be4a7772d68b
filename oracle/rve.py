"""The discretised RVE problem seen by the solvers (oracle).

Sec. 2: the unknown is the total strain field eps = E + eps~ on the voxel
quadrature points (Eq. (1)); equilibrium is Ghat : sigmahat = 0 (Eq. (6));
the Newton system is G : B : d_eps = -G : sigma (Eq. (8)); the total energy
is a sum over quadrature points (Eq. (11)) with gradient sigma and Hessian B
(Eqs. (12)-(13)).  In the strain-space formulation the gradient restricted
to compatible directions is G : sigma and the Hessian-vector product on a
compatible v is G : (B : v).

Norms and dot products are unnormalised Euclidean sums over every voxel and
Mandel entry (so the trust radius scales with sqrt(#points), Sec. 3.2).

Eigenstrain (Algorithm 2, and Sec. 3.3 for the ASR product sites): the
material is evaluated at eps_eval = eps + eps_eig, where eps_eig is a
per-phase Mandel vector gathered onto the voxels of that phase.  The
unknown stays eps: the gradient, the Hessian and the convergence measures
are those of eps; only the constitutive evaluation sees the shifted strain.
The sign is the paper's (added to the strain), so a stress-free expansion e
of a phase is eps_eig = -e.
"""
import numpy as np

from .fourier import project
from .material import PhaseParams, evaluate, tangent_apply, elastic_stress
from .tensors import ncomp_of


class RVE:
    def __init__(self, phase_map, phases, free_mask=None, naive_dft=False, eigenstrain=None):
        self.phase_map = np.asarray(phase_map)
        self.nphase = len(phases)
        self.shape = self.phase_map.shape
        self.ndim = self.phase_map.ndim
        self.ncomp = ncomp_of(self.ndim)
        self.nvox = int(np.prod(self.shape))
        self.params = PhaseParams(self.phase_map, phases)
        self.free_mask = (np.zeros(self.ncomp, dtype=bool) if free_mask is None
                          else np.asarray(free_mask, dtype=bool))
        self.naive = naive_dft
        self.eig = None
        self.set_eigenstrain(eigenstrain)

    def set_eigenstrain(self, table):
        """Per-phase eigenstrain table of shape (nphase, ncomp) (None: none),
        gathered to a field (ncomp, *grid) on the voxels of each phase."""
        if table is None:
            self.eig = None
            return
        t = np.asarray(table, dtype=np.float64)
        if t.shape != (self.nphase, self.ncomp):
            raise ValueError(f"eigenstrain table must have shape {(self.nphase, self.ncomp)}")
        self.eig = np.stack([t[self.phase_map, c] for c in range(self.ncomp)])

    def eval_strain(self, eps):
        """eps_eval = eps + eps_eig (Algorithm 2)."""
        return eps if self.eig is None else eps + self.eig

    # -- linear algebra on fields -------------------------------------------
    @staticmethod
    def dot(a, b):
        return float(np.sum(a * b))

    def norm(self, a):
        return float(np.sqrt(self.dot(a, a)))

    def G(self, x):
        """Compatibility projection (Eqs. (4)-(5))."""
        return project(x, self.free_mask, naive=self.naive)

    # -- material ----------------------------------------------------------
    def stress(self, eps, kappa_hist):
        """(sigma, D, kappa) at strain ``eps`` and committed history, the
        material evaluated at eps + eps_eig."""
        return evaluate(self.eval_strain(eps), self.params, kappa_hist)

    def tangent(self, D, v):
        return tangent_apply(v, D, self.params.lam, self.params.mu)

    def hessp(self, D, v):
        """H v = G : ((1 - D) C : v), the matrix-free Hessian-vector product
        of Eq. (8) with the secant tangent frozen at damage D."""
        return self.G(self.tangent(D, v))

    def gradient(self, sigma):
        """Energy gradient in compatible directions, G : sigma."""
        return self.G(sigma)

    def energy_frozen(self, eps, D):
        """W = sum_Q 1/2 (1 - D) e : C : e with D frozen and e = eps + eps_eig
        (Eq. (11))."""
        e = self.eval_strain(eps)
        return 0.5 * float(np.sum((1.0 - D) * e * elastic_stress(e, self.params.lam, self.params.mu)))

    def mean(self, field):
        """Volume average of a Mandel field, shape (ncomp,)."""
        return field.reshape(self.ncomp, -1).mean(axis=1)
