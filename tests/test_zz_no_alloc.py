"""rve_project_noalloc: the projection for callers that must not allocate
device memory (fixed-budget real-time or embedded loops, frameworks whose
caching allocator owns all device memory, code that must not trigger the
implicit synchronisation of cudaMalloc/cudaFree).  Its scratch is a fixed
16 MiB device array inside the library instead of a context workspace.

The test calls it through the C ABI twice in a row (two grids, so the second
call overwrites the first call's scratch) and checks each output against the
context-based rve_project, within the FP32 tolerance of the other parity
tests (2e-6 relative L2).  It lives in its own file, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 2e-6


def _rel(a, b):
    return float(torch.linalg.vector_norm((a - b).double()) / torch.linalg.vector_norm(b.double()))


def test_noalloc_projection_matches_context_projection_twice():
    from paper_2207_10657_gb300 import RVESolver, binding, build
    from synth import random_field
    build.build()
    cases = [((64, 48, 40), [1, 1, 0, 1, 1, 1]), ((96, 128), None)]
    stream = torch.cuda.current_stream()
    for dims, free in cases:
        nc = 6 if len(dims) == 3 else 3
        pm = np.zeros(tuple(reversed(dims)), np.uint8)
        v = torch.from_numpy(random_field(nc, dims, seed=21, dtype=np.float32)).cuda()
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
        ref_solver.close()


def test_noalloc_rejects_grids_over_the_limit():
    from paper_2207_10657_gb300 import binding, build
    build.build()
    v = torch.zeros(6 * 8, dtype=torch.float32, device="cuda")
    # 96^3 needs 6*96*96*49 = 2709504 complex values > 2087936
    assert binding.rve_project_noalloc((96, 96, 96), v.data_ptr(), v.data_ptr()) == -1
    assert binding.rve_project_noalloc((7, 8, 8), v.data_ptr(), v.data_ptr()) == -1
