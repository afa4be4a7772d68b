"""Plain, slow FP64 CPU oracle for the ringing-free FFT homogenisation solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The
product path (the CUDA library and its Python binding) never imports, calls
or links anything here, and this package imports nothing from the product.

It restates the paper's method in the most direct form that can be checked by
eye: full complex DFTs (numpy's FFT, or a naive O(N^2)-per-axis DFT on tiny
grids), the projection written per frequency, the constitutive law per voxel,
and the two algorithms (Steihaug CG, trust-region Newton with the first-order
incremental energy) step by step in the paper's order; ``lbfgs`` holds the
quasi-Newton alternative the paper mentions (L-BFGS with the first-order
energy in its line search).  Every function cites
the section / equation / algorithm it follows.

Equation numbers follow the paper's sequential numbering: (1) strain split,
(2a/b) equilibrium / compatibility, (4)-(6) projection, (7)-(8) Newton
linearisation, (9) projection from a discrete derivative, (10) spectral
derivative, (11) total energy, (12)-(13) gradient and Hessian, (14)
quadratic model, (15) exact ratio, (18) first-order incremental energy, (19)
approximate ratio, (20) restart measure, (21) 1D spring stiffness, (22)
damaged Young's modulus; appendix (A.1) tension strain measure, (A.3)
bilinear damage variable.

Pins: see ``tests/test_oracle_*.py``.  Parity unpinned beyond the oracle
itself: the softening stress-strain curves of the 3D sphere models (the paper
prints no numbers for them); every other function has an independent pin.
"""

from .tensors import mandel_to_tensor, tensor_to_mandel, ncomp_of, normal_comps
from .fourier import (
    fft,
    ifft,
    dft_naive,
    gradient_symbol,
    gradient_symbol_at,
    project_one,
    project_hat,
    project,
)
from .material import (
    Phase,
    lame,
    PhaseParams,
    elastic_stress,
    principal_strains,
    kappa_of_strain,
    damage_of_kappa,
    evaluate,
    tangent_apply,
)
from .rve import RVE
from .solver import steihaug_cg, TRParams, trust_region_step, load_path
from .lbfgs import LBFGSParams, lbfgs_step, load_path_lbfgs, two_loop

__all__ = [
    "mandel_to_tensor", "tensor_to_mandel", "ncomp_of", "normal_comps",
    "fft", "ifft", "dft_naive", "gradient_symbol", "gradient_symbol_at", "project_one", "project_hat", "project",
    "Phase", "lame", "PhaseParams", "elastic_stress", "principal_strains",
    "kappa_of_strain", "damage_of_kappa", "evaluate", "tangent_apply",
    "RVE", "steihaug_cg", "TRParams", "trust_region_step", "load_path",
    "LBFGSParams", "lbfgs_step", "load_path_lbfgs", "two_loop",
]
