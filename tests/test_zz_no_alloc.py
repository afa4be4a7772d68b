"""rve_project_noalloc: the projection for callers that must not allocate
device memory (fixed-budget real-time or embedded loops, frameworks whose
caching allocator owns all device memory, code that must not trigger the
implicit synchronisation of cudaMalloc/cudaFree).  Its scratch is a fixed
16 MiB device array inside the library instead of a context workspace.

The tests call it through the C ABI several times in a row (different
grids, so every call overwrites the previous call's scratch) and check each
output against the context-based rve_project and against the FP64 oracle's
projection, within the FP32 tolerance of the other parity tests (2e-6
relative L2).  The grids include the largest ones the documented limit
admits in 2D (1024 x 1024) and 3D (80^3).  The file is collected last.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-6


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def _check_cases(cases):
    from paper_2207_10657_gb300 import RVESolver, binding, build
    from synth import random_field
    build.build()
    stream = torch.cuda.current_stream()
    for dims, free in cases:
        nc = 6 if len(dims) == 3 else 3
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        v32 = random_field(nc, dims, seed=21, dtype=np.float32)
        v = torch.from_numpy(v32).cuda()
        ref_solver = RVESolver(dims, pm, [(1.0, 0.3, False, 0.0, 0.0)], precision=32)
        if free is not None:
            ref_solver.set_free_mask(free)
        ref = ref_solver.project(v)
        out = torch.full_like(v, float("nan"))
        st = binding.rve_project_noalloc(dims, v.data_ptr(), out.data_ptr(), free, stream.cuda_stream)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < TOL, dims
        fm = None if free is None else np.array(free[:nc], bool)
        exact = torch.from_numpy(oracle.project(v32.astype(np.float64), fm))
        assert _rel(out.cpu(), exact) < TOL, dims
        ref_solver.close()


def test_noalloc_projection_matches_context_projection_and_oracle():
    _check_cases([((64, 48, 40), [1, 1, 0, 1, 1, 1]), ((96, 128), None)])


def test_noalloc_projection_at_the_size_limit():
    """1024^2 in 2D (3 * 1024 * 513 = 1,575,936 complex values) and 80^3 in
    3D (6 * 80 * 80 * 41 = 1,574,400), both within the 2,087,936 limit."""
    _check_cases([((1024, 1024), [1, 0, 1]), ((80, 80, 80), None)])


def test_noalloc_rejects_grids_over_the_limit():
    from paper_2207_10657_gb300 import binding, build
    build.build()
    v = torch.zeros(6 * 8, dtype=torch.float32, device="cuda")
    # 96^3 needs 6*96*96*49 = 2709504 complex values > 2087936
    assert binding.rve_project_noalloc((96, 96, 96), v.data_ptr(), v.data_ptr()) == -1
    assert binding.rve_project_noalloc((7, 8, 8), v.data_ptr(), v.data_ptr()) == -1
