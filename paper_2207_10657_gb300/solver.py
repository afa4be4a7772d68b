"""PyTorch-facing wrapper over the C ABI: tensors in, tensors out.

Torch provides device memory and the CUDA stream; all arithmetic runs in
librve.so.  Shapes follow the library layout: a field is (ncomp, Nz, Ny, Nx)
in 3D or (ncomp, Ny, Nx) in 2D, Mandel components, C-contiguous.
"""
from dataclasses import dataclass

import torch

from . import binding as B


@dataclass
class Phase:
    """One material phase (Appendix A): isotropic E, nu; optional damage with
    the bilinear law between kappa0 and kappaf."""
    E: float
    nu: float
    damaging: bool = False
    kappa0: float = 0.0
    kappaf: float = 0.0

    def as_tuple(self):
        return (float(self.E), float(self.nu), 1 if self.damaging else 0, float(self.kappa0), float(self.kappaf))


def make_opts(precision=32, **kw):
    o = B.rve_default_opts()
    o.precision = int(precision)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _report_dict(rep):
    return {
        "nr_iters": rep.nr_iters, "cg_iters": rep.cg_iters, "hv_products": rep.hv_products,
        "restarts": rep.restarts, "rejected": rep.rejected, "boundary_hits": rep.boundary_hits,
        "converged": bool(rep.converged), "rel_residual": rep.rel_residual, "R": rep.R,
        "mean_stress": list(rep.mean_stress), "mean_strain": list(rep.mean_strain),
    }


class RVESolver:
    def __init__(self, dims, phase_ids, phases, precision=32, stream=None, **opts):
        if not torch.cuda.is_available():
            raise RuntimeError("RVESolver needs a CUDA device (there is no CPU path)")
        self.dims = tuple(int(d) for d in dims)
        self.ndim = len(self.dims)
        self.ncomp = 3 if self.ndim == 2 else 6
        self.shape = tuple(reversed(self.dims))
        self.dtype = torch.float32 if precision == 32 else torch.float64
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ids = torch.as_tensor(phase_ids, dtype=torch.uint8).to(self.device).contiguous()
        if tuple(ids.shape) != self.shape:
            raise ValueError(f"phase_ids shape {tuple(ids.shape)} != grid {self.shape}")
        self._ids = ids
        self.phases = [p if isinstance(p, Phase) else Phase(*p) for p in phases]
        self.opts = make_opts(precision, **opts)
        # strain points per voxel with the Kuhn-simplex element: 2 triangles
        # (2D), 6 tetrahedra (3D)
        self.nq = (6 if self.ndim == 3 else 2) if self.opts.element == 1 else 1
        self.fshape = ((self.ncomp, self.nq) if self.nq > 1 else (self.ncomp,)) + self.shape
        self.sshape = ((self.nq,) if self.nq > 1 else ()) + self.shape
        self._in()
        self.h = B.rve_create(self.dims, self.ndim, ids.data_ptr(), [p.as_tuple() for p in self.phases],
                              self.opts, self.stream.cuda_stream)

    # ------------------------------------------------------------ helpers
    def field(self, fill=None):
        """A strain-sized field: (ncomp, [nq,] *grid) of the context's type."""
        t = torch.empty(self.fshape, dtype=self.dtype, device=self.device)
        if fill is not None:
            t.fill_(fill)
        return t

    def scalar_field(self):
        """One value per strain point: ([nq,] *grid)."""
        return torch.empty(self.sshape, dtype=self.dtype, device=self.device)

    def _chk(self, t, kind="field"):
        want = self.fshape if kind == "field" else self.sshape
        dt = self.dtype
        if t.device != self.device or t.dtype != dt or tuple(t.shape) != want or not t.is_contiguous():
            raise ValueError(f"expected contiguous {dt} {kind} of shape {want} on {self.device}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")
        return t.data_ptr()

    def _in(self):
        """The library's stream waits for the work the caller's current
        stream has queued (inputs written there)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _out(self):
        """The caller's current stream waits for the library's stream
        (outputs written there)."""
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    # ------------------------------------------------------------ API
    def hessp(self, v, out=None):
        out = self.field() if out is None else out
        self._in()
        B.rve_hessp(self.h, self._chk(v), self._chk(out))
        self._out()
        return out

    def project(self, v, out=None):
        out = self.field() if out is None else out
        self._in()
        B.rve_project(self.h, self._chk(v), self._chk(out))
        self._out()
        return out

    def set_state(self, eps, kappa=None):
        self._in()
        B.rve_set_state(self.h, self._chk(eps), self._chk(kappa, "scalar") if kappa is not None else 0)

    def get_state(self):
        eps, sig = self.field(), self.field()
        kap, dmg = self.scalar_field(), self.scalar_field()
        self._in()
        B.rve_get_state(self.h, eps.data_ptr(), kap.data_ptr(), sig.data_ptr(), dmg.data_ptr())
        self._out()
        return {"eps": eps, "sigma": sig, "kappa": kap, "damage": dmg}

    def set_damage(self, D):
        self._in()
        B.rve_set_damage(self.h, self._chk(D, "scalar"))

    def set_free_mask(self, mask):
        B.rve_set_free_mask(self.h, mask)

    def set_eigenstrain(self, table):
        """Per-phase eigenstrain (nphase rows of ncomp Mandel values) added to
        the strain before every constitutive evaluation (Algorithm 2); None
        removes it.  A stress-free expansion e of a phase is a row of -e."""
        if table is not None:
            rows = [list(r) for r in table]
            if len(rows) != len(self.phases) or any(len(r) != self.ncomp for r in rows):
                raise ValueError(f"eigenstrain table must be {len(self.phases)} x {self.ncomp}")
            table = rows
        B.rve_set_eigenstrain(self.h, table)

    def energy_grad(self, p=None, want_grad=True):
        grad = self.field() if want_grad else None
        self._in()
        dW, dm = B.rve_energy_grad(self.h, self._chk(p) if p is not None else 0,
                                   grad.data_ptr() if grad is not None else 0)
        self._out()
        return dW, dm, grad

    def solve_step(self, dE, free_mask=None, init=None, raise_on_error=True):
        self._in()
        st, rep = B.rve_solve_step(self.h, dE, free_mask, self._chk(init) if init is not None else 0,
                                   raise_on_error)
        d = _report_dict(rep)
        d["status"] = st
        return d

    def steihaug(self, R, eta_cg, out=None):
        """One Steihaug-CG solve (Algorithm 1) at the state with radius R:
        returns (z, report dict with the exit reason)."""
        out = self.field() if out is None else out
        self._in()
        rep = B.rve_steihaug(self.h, R, eta_cg, self._chk(out))
        self._out()
        return out, {"reason": B.CG_EXIT.get(rep.status, str(rep.status)), "iters": rep.iters,
                     "hv_products": rep.hv_products, "restarts": rep.restarts}

    def solve_step_lbfgs(self, dE, free_mask=None, memory=5, max_iter=500, raise_on_error=True):
        """One load step by L-BFGS with the first-order incremental energy in
        its line search (report: nr_iters = iterations, cg_iters = line-search
        trials, rejected = step halvings, restarts = skipped pairs)."""
        self._in()
        st, rep = B.rve_solve_step_lbfgs(self.h, dE, free_mask, memory, max_iter, raise_on_error)
        d = _report_dict(rep)
        d["status"] = st
        return d

    def effective_stiffness(self, tol=1e-6, max_cg=2000):
        """Effective secant stiffness (ncomp x ncomp Mandel, nested lists) at
        the current damage field, and the CG iterations it took."""
        return B.rve_effective_stiffness(self.h, self.ncomp, tol, max_cg)

    @property
    def hv_count(self):
        return B.rve_hv_count(self.h)

    @property
    def launch_count(self):
        return B.rve_launch_count(self.h)

    @property
    def sync_count(self):
        """Host waits that read the device scalars (counter)."""
        return B.rve_sync_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            B.rve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RVEBatch:
    """Many RVEs of uneven sizes (2D / 3D mixed), FP32, solved in lockstep by
    the batched launches of the library (one persistent launch per pass)."""

    def __init__(self, dims_list, phase_ids_list, phases, stream=None, **opts):
        if not torch.cuda.is_available():
            raise RuntimeError("RVEBatch needs a CUDA device (there is no CPU path)")
        self.dims = [tuple(int(x) for x in d) for d in dims_list]
        self.n = len(self.dims)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.shapes = [tuple(reversed(d)) for d in self.dims]
        self.ncomp = [3 if len(d) == 2 else 6 for d in self.dims]
        self._ids = []
        for ids, shp in zip(phase_ids_list, self.shapes):
            t = torch.as_tensor(ids, dtype=torch.uint8).to(self.device).contiguous()
            if tuple(t.shape) != shp:
                raise ValueError(f"phase_ids shape {tuple(t.shape)} != grid {shp}")
            self._ids.append(t)
        self.phases = [p if isinstance(p, Phase) else Phase(*p) for p in phases]
        self.opts = make_opts(32, **opts)
        self._in()
        self.h = B.rve_batch_create(self.dims, [t.data_ptr() for t in self._ids],
                                    [p.as_tuple() for p in self.phases], self.opts, self.stream.cuda_stream)

    def _in(self):
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _out(self):
        cur = torch.cuda.current_stream(self.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def field(self, i):
        return torch.empty((self.ncomp[i],) + self.shapes[i], dtype=torch.float32, device=self.device)

    def hessp(self, vs):
        outs = [self.field(i) for i in range(self.n)]
        for i, v in enumerate(vs):
            if v.dtype != torch.float32 or tuple(v.shape) != (self.ncomp[i],) + self.shapes[i] or not v.is_contiguous():
                raise ValueError(f"member {i}: bad field")
        self._in()
        B.rve_batch_hessp(self.h, [v.data_ptr() for v in vs], [o.data_ptr() for o in outs])
        self._out()
        return outs

    def set_damage(self, i, D):
        D = D.contiguous()
        self._in()
        B.rve_batch_set_damage(self.h, i, D.data_ptr())

    def get_state(self, i):
        eps, sig = self.field(i), self.field(i)
        kap = torch.empty(self.shapes[i], dtype=torch.float32, device=self.device)
        dmg = torch.empty_like(kap)
        self._in()
        B.rve_batch_get_state(self.h, i, eps.data_ptr(), kap.data_ptr(), sig.data_ptr(), dmg.data_ptr())
        self._out()
        return {"eps": eps, "sigma": sig, "kappa": kap, "damage": dmg}

    def reset(self):
        B.rve_batch_reset(self.h)

    def autotune(self, reps=3):
        """Choose the fastest tile / radix-order schedule of the batched
        passes by timing; returns {"ms_per_product", "ms_per_product_default",
        "schedule"}."""
        base, ms, sched = B.rve_batch_autotune(self.h, reps)
        return {"ms_per_product": ms, "ms_per_product_default": base,
                "schedule": {"x_div": sched[0], "y_div": sched[1], "z_div": sched[2],
                             "radix_reversed": bool(sched[3])}}

    def solve_step(self, dE_list, free_masks=None, raise_on_error=True):
        st, reps = B.rve_batch_solve_step(self.h, dE_list, free_masks, raise_on_error)
        out = [_report_dict(r) for r in reps]
        for o in out:
            o["status"] = st
        return out

    @property
    def hv_count(self):
        return B.rve_batch_hv_count(self.h)

    @property
    def launch_count(self):
        return B.rve_batch_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            B.rve_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
