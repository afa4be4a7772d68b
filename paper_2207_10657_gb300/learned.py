"""Learned warm start: a spectral neural operator (library kernels) that
proposes the next load step's strain-fluctuation increment.

The proposal only seeds the trust-region solve (``rve_solve_step``'s
``init_incr``, projected onto compatible fields by the library); the plain
solver still decides convergence, so accuracy is unchanged and only the
iteration count can drop.  Torch supplies device memory only.
"""
import time

import numpy as np
import torch

from . import binding as B

CIN, WIDTH, COUT = 16, 32, 6


def pack_params(p, layers):
    """Oracle-layout parameter dict -> the library's packed FP32 vector
    (weights stored [in][out])."""
    parts = [p["Wl"].T.ravel(), p["bl"].ravel()]
    for l in range(layers):
        parts += [p[f"W{l}"].T.ravel(), p[f"b{l}"].ravel(), p[f"R{l}"].ravel()]
    parts += [p["Wq"].T.ravel(), p["bq"].ravel()]
    return np.concatenate(parts).astype(np.float32)


def unpack_grads(vec, cin, width, cout, layers, modes):
    """Packed vector -> dict in the oracle's layout."""
    out, off = {}, 0

    def take(n):
        nonlocal off
        v = vec[off:off + n]
        off += n
        return v
    out["Wl"] = take(cin * width).reshape(cin, width).T
    out["bl"] = take(width)
    for l in range(layers):
        out[f"W{l}"] = take(width * width).reshape(width, width).T
        out[f"b{l}"] = take(width)
        out[f"R{l}"] = take(modes ** 3 * 4 * width * width).reshape(modes, modes, modes, 2 * width, 2 * width)
    out["Wq"] = take(width * cout).reshape(width, cout).T
    out["bq"] = take(cout)
    return out


class SpectralOperator:
    """Handle on the library's network (forward, loss/gradient, Adam)."""

    def __init__(self, layers=4, modes=16, seed=0, cin=CIN, cout=COUT, stream=None, residual=True):
        self.layers, self.modes, self.cin, self.cout = layers, modes, cin, cout
        # residual: the network predicts the change of the fluctuation
        # increment from the last step (exact zero in the elastic range)
        self.residual = residual
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = B.rve_fno_create(cin, WIDTH, cout, layers, modes, seed, self.stream.cuda_stream)
        self.nparam = B.rve_fno_param_count(self.h)

    def set_params(self, vec):
        v = np.ascontiguousarray(vec, dtype=np.float32)
        assert v.size == self.nparam
        B.rve_fno_set_params(self.h, v.ctypes.data)

    def get_params(self, want_grad=False):
        p = np.empty(self.nparam, np.float32)
        g = np.empty(self.nparam, np.float32) if want_grad else None
        B.rve_fno_get_params(self.h, p.ctypes.data, g.ctypes.data if g is not None else 0)
        return (p, g) if want_grad else p

    def forward(self, X, dims):
        Y = torch.empty(X.shape[:-1] + (self.cout,), dtype=torch.float32, device=X.device)
        B.rve_fno_forward(self.h, X.shape[0], dims, X.data_ptr(), Y.data_ptr())
        return Y

    def loss_grad(self, X, T, dims):
        return B.rve_fno_loss_grad(self.h, X.shape[0], dims, X.data_ptr(), T.data_ptr())

    def adam_step(self, lr):
        B.rve_fno_adam_step(self.h, lr)

    def features(self, dims, phase, damage, d1, d2, scale, kappa=None, kappa_scale=1.0):
        nz, ny, nx = dims[2], dims[1], dims[0]
        X = torch.empty((1, nz, ny, nx, self.cin), dtype=torch.float32, device=phase.device)
        ptr = (lambda t: t.data_ptr() if t is not None else 0)
        B.rve_fno_pack_features(self.h, dims, phase.data_ptr(), ptr(damage), ptr(d1), ptr(d2), scale, X.data_ptr(),
                                ptr(kappa), kappa_scale)
        return X

    def to_field(self, Y, dims, scale, base=None):
        out = torch.empty((self.cout, dims[2], dims[1], dims[0]), dtype=torch.float32, device=Y.device)
        B.rve_fno_unpack_output(self.h, dims, Y.data_ptr(), scale, out.data_ptr(),
                                base.data_ptr() if base is not None else 0)
        return out

    @property
    def launch_count(self):
        return B.rve_fno_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            B.rve_fno_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- pipeline
def _sync(stream):
    stream.synchronize()


class IncrementTracker:
    """Follows one solver along its load path and keeps what the network
    reads: the last two converged fluctuation increments (SoA FP32 fields,
    eps_n - eps_{n-1} - dE_n) and the strain of the last converged state."""

    def __init__(self, solver, net):
        # history variable in units of the smallest damage threshold
        k0 = [p.kappa0 for p in solver.phases if p.damaging and p.kappa0 > 0]
        self.kappa_scale = 1.0 / min(k0) if k0 else 1.0
        if solver.dtype != torch.float32:
            raise ValueError("the warm start works on FP32 solver fields")
        self.s, self.net = solver, net
        self.dims = tuple(solver.dims)
        self.d1 = torch.zeros((solver.ncomp,) + solver.shape, dtype=torch.float32, device=solver.device)
        self.d2 = torch.zeros_like(self.d1)
        st = solver.get_state()
        self.eps = st["eps"]
        self.kappa = st["kappa"]
        self.damage = st["damage"]
        self.steps = 0

    def features(self, dE):
        scale = 1.0 / max(float(np.linalg.norm(dE)), 1e-30)
        return self.net.features(self.dims, self.s._ids, self.damage, self.d1, self.d2, scale,
                                 self.kappa, self.kappa_scale)

    def predict(self, dE):
        """Predicted fluctuation increment of the next step (SoA field)."""
        nrm = float(np.linalg.norm(dE))
        Y = self.net.forward(self.features(dE), self.dims)
        return self.net.to_field(Y, self.dims, nrm, self.d1 if self.net.residual else None)

    def advance(self, dE, eps_new=None, kappa_new=None):
        """Record a converged step: shift the increments and the state."""
        st = self.s.get_state() if eps_new is None else None
        eps_new = st["eps"] if eps_new is None else eps_new
        kappa_new = st["kappa"] if kappa_new is None else kappa_new
        incr = torch.empty_like(self.d1)
        B.rve_fno_increment(self.net.h, self.dims, eps_new.data_ptr(), self.eps.data_ptr(), dE, incr.data_ptr())
        self.d2, self.d1 = self.d1, incr
        self.eps, self.kappa = eps_new, kappa_new
        if st is not None:
            self.damage = st["damage"]
        else:
            self.s.set_state(eps_new, kappa_new)
            self.damage = self.s.get_state()["damage"]
        self.steps += 1
        return incr


def generate_samples(net, cells, phases, dE, free_mask, steps, max_samples=None, time_budget_s=None, **opts):
    """Training pairs from the plain solver: for every cell, load steps of
    constant increment dE until one does not converge or `steps` are done.
    Returns channels-last inputs X and targets T (lists of (1, Nz, Ny, Nx, .)
    device tensors; with a residual network the target is the change of the
    fluctuation increment) and a per-step log."""
    from .solver import RVESolver
    Xs, Ts, log = [], [], []
    t0 = time.perf_counter()
    nrm = float(np.linalg.norm(dE))
    for ci, pm in enumerate(cells):
        dims = tuple(reversed(pm.shape))
        s = RVESolver(dims, pm, phases, precision=32, stream=net.stream, **opts)
        tr = IncrementTracker(s, net)
        for k in range(steps):
            X = tr.features(dE)
            rep = s.solve_step(dE, free_mask=free_mask, raise_on_error=False)
            log.append({"cell": ci, "step": k + 1, "nr": rep["nr_iters"], "hv": rep["hv_products"],
                        "converged": rep["converged"]})
            if not rep["converged"]:
                break
            base = tr.d1
            incr = tr.advance(dE)
            T = torch.empty(X.shape[:-1] + (net.cout,), dtype=torch.float32, device=X.device)
            B.rve_fno_pack_target(net.h, dims, incr.data_ptr(), 1.0 / nrm, T.data_ptr(),
                                  base.data_ptr() if net.residual else 0)
            Xs.append(X)
            Ts.append(T)
            if max_samples and len(Xs) >= max_samples:
                break
        s.close()
        if (max_samples and len(Xs) >= max_samples) or (time_budget_s and time.perf_counter() - t0 > time_budget_s):
            break
    _sync(net.stream)
    return Xs, Ts, log


def train(net, Xs, Ts, dims, iters, batch=4, lr=1e-3, lr_final=None, seed=0, log_every=0):
    """Adam on minibatches drawn from (Xs, Ts); cosine-decayed learning rate.
    Returns the loss history."""
    rng = np.random.default_rng(seed)
    n = len(Xs)
    batch = min(batch, n, 8)
    hist = []
    lr_final = lr * 0.05 if lr_final is None else lr_final
    for it in range(iters):
        idx = rng.choice(n, size=batch, replace=False)
        X = torch.cat([Xs[i] for i in idx]).contiguous()
        T = torch.cat([Ts[i] for i in idx]).contiguous()
        L = net.loss_grad(X, T, dims)
        a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * it / max(iters - 1, 1)))
        net.adam_step(a)
        hist.append(L)
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {L:.4e} lr {a:.2e}", flush=True)
    return hist


def _rel_err(a, ref):
    """Relative L2 distance, computed on the host (reporting only)."""
    r = ref.detach().cpu().numpy().astype(np.float64)
    d = (a.detach().cpu().numpy().astype(np.float64) - r) if a is not None else -r
    return float(np.linalg.norm(d) / max(np.linalg.norm(r), 1e-300))


def compare_warm_start(net, pm, phases, dE, free_mask, steps, arms=("plain", "learned", "previous"), **opts):
    """Load steps along the plain path of one cell; each step is solved from
    the same converged state by every arm, in its own solver context:
      plain    -- the uniform predictor eps += dE (the method as published),
      learned  -- eps += dE + G(network prediction),
      previous -- eps += dE + G(last fluctuation increment) (non-learned
                  extrapolation, for reference).
    Times include the network inference.  Each record also holds the
    relative distance of every arm's starting increment from the converged
    one (plain: 1).  Returns one record per step."""
    from .solver import RVESolver
    dims = tuple(reversed(pm.shape))
    ctx = {a: RVESolver(dims, pm, phases, precision=32, stream=net.stream, **opts) for a in arms}
    tr = IncrementTracker(ctx["plain"], net)
    st = net.stream
    out = []
    for k in range(steps):
        rec = {"step": k + 1}
        res, inits = {}, {}
        for a in arms:
            s = ctx[a]
            s.set_state(tr.eps, tr.kappa)
            _sync(st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h0 = s.hv_count
            e0.record(st)
            init = None
            if a == "learned":
                init = tr.predict(dE)
            elif a == "previous" and tr.steps > 0:
                init = tr.d1
            rep = s.solve_step(dE, free_mask=free_mask, init=init, raise_on_error=False)
            e1.record(st)
            _sync(st)
            inits[a] = init
            rec[a] = {"ms": e0.elapsed_time(e1), "hv": s.hv_count - h0, "nr": rep["nr_iters"],
                      "converged": rep["converged"], "mean_stress": rep["mean_stress"]}
            if a == "plain":
                stp = s.get_state()
                res = {"eps": stp["eps"], "kappa": stp["kappa"]}
        out.append(rec)
        if not rec["plain"]["converged"]:
            break
        actual = tr.advance(dE, res["eps"], res["kappa"])
        for a in arms:
            rec[a]["start_err"] = _rel_err(inits[a], actual)
    for s in ctx.values():
        s.close()
    return out
