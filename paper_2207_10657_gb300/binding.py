"""ctypes binding of librve.so (include/rve.h), same names as the C ABI.

Argument marshalling only: every computation runs in the library's CUDA
kernels.  PyTorch supplies device memory and the stream.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librve.so")

RVE_OK = 0
STATUS = {0: "RVE_OK", -1: "RVE_ERR_ARG", -2: "RVE_ERR_CUDA", -3: "RVE_ERR_OOM",
          -4: "RVE_ERR_NOT_CONVERGED", -5: "RVE_ERR_NONFINITE", -6: "RVE_ERR_TIMEOUT"}


class rve_phase(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("damaging", ctypes.c_int),
                ("kappa0", ctypes.c_double), ("kappaf", ctypes.c_double)]


class rve_solver_opts(ctypes.Structure):
    _fields_ = [("eta_eq", ctypes.c_double), ("eta_nr", ctypes.c_double), ("eta_cg", ctypes.c_double),
                ("eta_up", ctypes.c_double), ("R0", ctypes.c_double), ("Rmax", ctypes.c_double),
                ("max_nr", ctypes.c_int), ("max_cg", ctypes.c_int), ("restart_thr", ctypes.c_double),
                ("precision", ctypes.c_int), ("hessian", ctypes.c_int), ("passes", ctypes.c_int),
                ("element", ctypes.c_int)]


class rve_step_report(ctypes.Structure):
    _fields_ = [("nr_iters", ctypes.c_int), ("cg_iters", ctypes.c_int), ("hv_products", ctypes.c_int),
                ("restarts", ctypes.c_int), ("rejected", ctypes.c_int), ("boundary_hits", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double), ("R", ctypes.c_double),
                ("mean_stress", ctypes.c_double * 6), ("mean_strain", ctypes.c_double * 6)]


class rve_cg_report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("hv_products", ctypes.c_int),
                ("restarts", ctypes.c_int)]


CG_EXIT = {1: "converged", 2: "boundary", 3: "negative_curvature", 4: "max_iter", 5: "zero_rhs"}


class RveError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes)
_SIGS = [
    ("rve_default_opts", None, [ctypes.POINTER(rve_solver_opts)]),
    ("rve_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                                  ctypes.POINTER(rve_phase), ctypes.c_int, ctypes.POINTER(rve_solver_opts),
                                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("rve_set_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    ("rve_set_damage", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_set_free_mask", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8)]),
    ("rve_set_eigenstrain", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("rve_hessp", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_project", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_energy_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("rve_solve_step", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_uint8), ctypes.c_void_p,
                                      ctypes.POINTER(rve_step_report)]),
    ("rve_steihaug", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                    ctypes.POINTER(rve_cg_report)]),
    ("rve_solve_step_lbfgs", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_uint8), ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(rve_step_report)]),
    ("rve_effective_stiffness", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    ("rve_pass_timing", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("rve_pass_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("rve_project_noalloc", ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_void_p]),
    ("rve_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(rve_phase), ctypes.c_int,
                                        ctypes.POINTER(rve_solver_opts), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("rve_batch_solve_step", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(rve_step_report)]),
    ("rve_batch_hessp", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                                       ctypes.POINTER(ctypes.c_void_p)]),
    ("rve_batch_set_damage", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("rve_batch_get_state", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_batch_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("rve_batch_set_schedule", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("rve_batch_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    ("rve_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("rve_batch_hv_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_batch_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_batch_destroy", None, [ctypes.c_void_p]),
    ("rve_fno_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_ulonglong, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    ("rve_fno_param_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_fno_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_fno_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_fno_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                       ctypes.c_void_p]),
    ("rve_fno_loss_grad", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("rve_fno_adam_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("rve_fno_pack_features", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p]),
    ("rve_fno_unpack_output", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                             ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    ("rve_fno_pack_target", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_float, ctypes.c_void_p]),
    ("rve_fno_increment", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    ("rve_fno_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("rve_fno_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_fno_destroy", None, [ctypes.c_void_p]),
    ("rve_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("rve_hv_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_sync_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("rve_set_device_loop", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("rve_destroy", None, [ctypes.c_void_p]),
]

EXPORTED = [n for n, _, _ in _SIGS]


def lib(path=None):
    """Load librve.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: build it with paper_2207_10657_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(p)
    for name, res, args in _SIGS:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def check(status, handle=None):
    if status != RVE_OK:
        msg = lib().rve_last_error(handle).decode()
        raise RveError(status, msg)


# ----------------------------------------------------------------- wrappers
def rve_default_opts():
    o = rve_solver_opts()
    lib().rve_default_opts(ctypes.byref(o))
    return o


def rve_create(dims, ndim, phase_ids_ptr, phases, opts=None, stream=0):
    d = (ctypes.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))
    arr = (rve_phase * len(phases))(*[rve_phase(*p) for p in phases])
    h = ctypes.c_void_p()
    st = lib().rve_create(d, ndim, ctypes.c_void_p(phase_ids_ptr), arr, len(phases),
                          ctypes.byref(opts) if opts is not None else None,
                          ctypes.c_void_p(stream), ctypes.byref(h))
    check(st, None)
    return h


def rve_set_state(h, strain_ptr, kappa_ptr=0):
    check(lib().rve_set_state(h, ctypes.c_void_p(strain_ptr), ctypes.c_void_p(kappa_ptr or None)), h)


def rve_get_state(h, strain_ptr=0, kappa_ptr=0, stress_ptr=0, damage_ptr=0):
    check(lib().rve_get_state(h, ctypes.c_void_p(strain_ptr or None), ctypes.c_void_p(kappa_ptr or None),
                              ctypes.c_void_p(stress_ptr or None), ctypes.c_void_p(damage_ptr or None)), h)


def rve_set_damage(h, damage_ptr):
    check(lib().rve_set_damage(h, ctypes.c_void_p(damage_ptr)), h)


def rve_set_free_mask(h, mask):
    m = (ctypes.c_uint8 * 6)(*[1 if x else 0 for x in (list(mask) + [0] * (6 - len(mask)))])
    check(lib().rve_set_free_mask(h, m), h)


def rve_set_eigenstrain(h, table):
    """table: nphase rows of ncomp Mandel values (host), or None to remove."""
    if table is None:
        check(lib().rve_set_eigenstrain(h, None, 0), h)
        return
    rows = [list(map(float, r)) for r in table]
    flat = [x for r in rows for x in r]
    arr = (ctypes.c_double * len(flat))(*flat)
    check(lib().rve_set_eigenstrain(h, arr, len(rows)), h)


def rve_hessp(h, v_ptr, out_ptr):
    check(lib().rve_hessp(h, ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr)), h)


def rve_project(h, v_ptr, out_ptr):
    check(lib().rve_project(h, ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr)), h)


def rve_energy_grad(h, p_ptr=0, grad_ptr=0):
    dW, dm = ctypes.c_double(), ctypes.c_double()
    check(lib().rve_energy_grad(h, ctypes.c_void_p(p_ptr or None), ctypes.byref(dW), ctypes.byref(dm),
                                ctypes.c_void_p(grad_ptr or None)), h)
    return dW.value, dm.value


def rve_solve_step(h, dE, free_mask=None, init_ptr=0, raise_on_error=True):
    de = (ctypes.c_double * 6)(*(list(dE) + [0.0] * (6 - len(dE))))
    fm = None
    if free_mask is not None:
        fm = (ctypes.c_uint8 * 6)(*[1 if x else 0 for x in (list(free_mask) + [0] * (6 - len(free_mask)))])
    rep = rve_step_report()
    st = lib().rve_solve_step(h, de, fm, ctypes.c_void_p(init_ptr or None), ctypes.byref(rep))
    if raise_on_error:
        check(st, h)
    return st, rep


def rve_steihaug(h, R, eta_cg, z_ptr):
    rep = rve_cg_report()
    check(lib().rve_steihaug(h, float(R), float(eta_cg), ctypes.c_void_p(z_ptr), ctypes.byref(rep)), h)
    return rep


def rve_solve_step_lbfgs(h, dE, free_mask=None, memory=5, max_iter=500, raise_on_error=True):
    de = (ctypes.c_double * 6)(*(list(dE) + [0.0] * (6 - len(dE))))
    fm = None
    if free_mask is not None:
        fm = (ctypes.c_uint8 * 6)(*[1 if x else 0 for x in (list(free_mask) + [0] * (6 - len(free_mask)))])
    rep = rve_step_report()
    st = lib().rve_solve_step_lbfgs(h, de, fm, int(memory), int(max_iter), ctypes.byref(rep))
    if raise_on_error:
        check(st, h)
    return st, rep


def rve_effective_stiffness(h, ncomp, tol=1e-6, max_cg=2000):
    """(C_bar as ncomp rows of ncomp floats, total CG iterations)."""
    out = (ctypes.c_double * (ncomp * ncomp))()
    it = ctypes.c_int(0)
    check(lib().rve_effective_stiffness(h, float(tol), int(max_cg), out, ctypes.byref(it)), h)
    return [list(out[i * ncomp:(i + 1) * ncomp]) for i in range(ncomp)], it.value


PASS_NAMES = ["xfwd_tangent", "y_fwd", "z_proj", "y_inv", "x_inv", "y_proj_2d", "trial", "cg_vec"]


def rve_pass_timing(h, enable=True):
    check(lib().rve_pass_timing(h, 1 if enable else 0), h)


def rve_pass_stats(h):
    n = len(PASS_NAMES)
    counts = (ctypes.c_longlong * n)()
    ms = (ctypes.c_double * n)()
    check(lib().rve_pass_stats(h, counts, ms, n), h)
    return {PASS_NAMES[i]: (counts[i], ms[i]) for i in range(n)}


def rve_project_noalloc(dims, v_ptr, out_ptr, free_mask=None, stream=0):
    """Projection with no device allocation (scratch in a fixed 16 MiB
    device array inside the library); returns the status code."""
    d = (ctypes.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))
    fm = None
    if free_mask is not None:
        fm = (ctypes.c_uint8 * 6)(*[1 if x else 0 for x in (list(free_mask) + [0] * (6 - len(free_mask)))])
    return lib().rve_project_noalloc(d, len(dims), ctypes.c_void_p(v_ptr), ctypes.c_void_p(out_ptr), fm,
                                     ctypes.c_void_p(stream))


def _bcheck(status, handle):
    if status != RVE_OK:
        raise RveError(status, lib().rve_batch_last_error(handle).decode())


def rve_batch_create(dims_list, phase_ptrs, phases, opts=None, stream=0):
    n = len(dims_list)
    dims = (ctypes.c_int * (3 * n))(*[x for d in dims_list for x in (list(d) + [1] * (3 - len(d)))])
    nd = (ctypes.c_int * n)(*[len(d) for d in dims_list])
    ptrs = (ctypes.c_void_p * n)(*phase_ptrs)
    arr = (rve_phase * len(phases))(*[rve_phase(*p) for p in phases])
    h = ctypes.c_void_p()
    st = lib().rve_batch_create(n, dims, nd, ptrs, arr, len(phases),
                                ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(stream),
                                ctypes.byref(h))
    _bcheck(st, None)
    return h


def rve_batch_solve_step(h, dE_list, free_masks=None, raise_on_error=True):
    n = len(dE_list)
    de = (ctypes.c_double * (6 * n))(*[x for d in dE_list for x in (list(d) + [0.0] * (6 - len(d)))])
    fm = None
    if free_masks is not None:
        fm = (ctypes.c_uint8 * (6 * n))(*[1 if x else 0 for m in free_masks for x in (list(m) + [0] * (6 - len(m)))])
    reps = (rve_step_report * n)()
    st = lib().rve_batch_solve_step(h, de, fm, reps)
    if raise_on_error:
        _bcheck(st, h)
    return st, list(reps)


def rve_batch_hessp(h, v_ptrs, out_ptrs):
    n = len(v_ptrs)
    vs = (ctypes.c_void_p * n)(*v_ptrs)
    os_ = (ctypes.c_void_p * n)(*out_ptrs)
    _bcheck(lib().rve_batch_hessp(h, vs, os_), h)


def rve_batch_set_damage(h, i, damage_ptr):
    _bcheck(lib().rve_batch_set_damage(h, i, ctypes.c_void_p(damage_ptr)), h)


def rve_batch_get_state(h, i, strain_ptr=0, kappa_ptr=0, stress_ptr=0, damage_ptr=0):
    _bcheck(lib().rve_batch_get_state(h, i, ctypes.c_void_p(strain_ptr or None), ctypes.c_void_p(kappa_ptr or None),
                                      ctypes.c_void_p(stress_ptr or None), ctypes.c_void_p(damage_ptr or None)), h)


def rve_batch_reset(h):
    _bcheck(lib().rve_batch_reset(h), h)


def rve_batch_set_schedule(h, schedule):
    _bcheck(lib().rve_batch_set_schedule(h, (ctypes.c_int * 4)(*schedule)), h)


def rve_batch_autotune(h, reps=3):
    """Pick the fastest batched-pass schedule; returns (default ms, chosen ms, schedule) per product."""
    base, ms = ctypes.c_double(), ctypes.c_double()
    sched = (ctypes.c_int * 4)()
    _bcheck(lib().rve_batch_autotune(h, reps, ctypes.byref(base), ctypes.byref(ms), sched), h)
    return base.value, ms.value, list(sched)


def rve_batch_hv_count(h):
    return lib().rve_batch_hv_count(h)


def rve_batch_launch_count(h):
    return lib().rve_batch_launch_count(h)


def rve_batch_destroy(h):
    lib().rve_batch_destroy(h)


def _fcheck(status, handle):
    if status != RVE_OK:
        raise RveError(status, lib().rve_fno_last_error(handle).decode())


def _dims3(dims):
    return (ctypes.c_int * 3)(*(list(dims) + [1] * (3 - len(dims))))


def rve_fno_create(cin, width, cout, layers, modes, seed=0, stream=0):
    h = ctypes.c_void_p()
    _fcheck(lib().rve_fno_create(cin, width, cout, layers, modes, seed, ctypes.c_void_p(stream), ctypes.byref(h)),
            None)
    return h


def rve_fno_param_count(h):
    return lib().rve_fno_param_count(h)


def rve_fno_set_params(h, params_ptr):
    _fcheck(lib().rve_fno_set_params(h, ctypes.c_void_p(params_ptr)), h)


def rve_fno_get_params(h, params_ptr=0, grad_ptr=0):
    _fcheck(lib().rve_fno_get_params(h, ctypes.c_void_p(params_ptr or None), ctypes.c_void_p(grad_ptr or None)), h)


def rve_fno_forward(h, batch, dims, x_ptr, y_ptr):
    _fcheck(lib().rve_fno_forward(h, batch, _dims3(dims), ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr)), h)


def rve_fno_loss_grad(h, batch, dims, x_ptr, t_ptr):
    loss = ctypes.c_double()
    _fcheck(lib().rve_fno_loss_grad(h, batch, _dims3(dims), ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr),
                                    ctypes.byref(loss)), h)
    return loss.value


def rve_fno_adam_step(h, lr):
    _fcheck(lib().rve_fno_adam_step(h, lr), h)


def rve_fno_pack_features(h, dims, phase_ptr, damage_ptr, d1_ptr, d2_ptr, scale, x_ptr, kappa_ptr=0, kappa_scale=1.0):
    _fcheck(lib().rve_fno_pack_features(h, _dims3(dims), ctypes.c_void_p(phase_ptr), ctypes.c_void_p(damage_ptr or None),
                                        ctypes.c_void_p(kappa_ptr or None), kappa_scale,
                                        ctypes.c_void_p(d1_ptr or None), ctypes.c_void_p(d2_ptr or None),
                                        scale, ctypes.c_void_p(x_ptr)), h)


def rve_fno_unpack_output(h, dims, y_ptr, scale, out_ptr, base_ptr=0):
    _fcheck(lib().rve_fno_unpack_output(h, _dims3(dims), ctypes.c_void_p(y_ptr), scale,
                                        ctypes.c_void_p(base_ptr or None), ctypes.c_void_p(out_ptr)), h)


def rve_fno_pack_target(h, dims, field_ptr, scale, t_ptr, base_ptr=0):
    _fcheck(lib().rve_fno_pack_target(h, _dims3(dims), ctypes.c_void_p(field_ptr), ctypes.c_void_p(base_ptr or None),
                                      scale, ctypes.c_void_p(t_ptr)), h)


def rve_fno_increment(h, dims, new_ptr, old_ptr, dE, out_ptr):
    d = (ctypes.c_double * 6)(*(list(dE) + [0.0] * (6 - len(dE))))
    _fcheck(lib().rve_fno_increment(h, _dims3(dims), ctypes.c_void_p(new_ptr), ctypes.c_void_p(old_ptr), d,
                                    ctypes.c_void_p(out_ptr)), h)


def rve_fno_launch_count(h):
    return lib().rve_fno_launch_count(h)


def rve_fno_destroy(h):
    lib().rve_fno_destroy(h)


def rve_last_error(h):
    return lib().rve_last_error(h).decode()


def rve_hv_count(h):
    return lib().rve_hv_count(h)


def rve_sync_count(h):
    return lib().rve_sync_count(h)


def rve_set_device_loop(h, enable=True):
    check(lib().rve_set_device_loop(h, 1 if enable else 0), h)


def rve_launch_count(h):
    return lib().rve_launch_count(h)


def rve_destroy(h):
    lib().rve_destroy(h)
