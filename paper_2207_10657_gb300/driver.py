"""Load-path driver: Algorithm 2's outer loop over macroscopic increments
around a solver context, with what a long production run needs on top of
the library's load step:

* failure handling -- a load step that does not converge (RVE_ERR_NOT_CONVERGED
  from the trust-region or L-BFGS step) leaves the committed history
  untouched; the driver restores the strain of the last converged state and
  splits the increment in two halves (the eigenstrain table interpolated
  linearly), recursively up to ``max_halvings`` times, before giving up;
* checkpoint / resume -- the converged state (strain, committed history),
  the next increment index, the eigenstrain table in force and the last
  trust radius go to an ``.npz`` file every ``checkpoint_every`` increments;
  ``resume`` puts them back into a context;
* a JSON-lines log, one record per solved (sub-)increment.

The driver holds no arithmetic of the method: it only calls the context's
solve_step / solve_step_lbfgs, get_state / set_state and set_eigenstrain.
Any object with those methods works (the tests drive a host-side fake to
inject failures without a GPU).
"""
import json
import os
import time

import numpy as np


def _copy(x):
    return x.clone() if hasattr(x, "clone") else np.array(x, copy=True)


def _host(x):
    return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)


class LoadPathDriver:
    def __init__(self, solver, solver_kind="trust_region", lbfgs_memory=5, lbfgs_max_iter=500,
                 max_halvings=4, log_path=None, checkpoint_path=None, checkpoint_every=1):
        if solver_kind not in ("trust_region", "lbfgs"):
            raise ValueError("solver_kind must be 'trust_region' or 'lbfgs'")
        self.s = solver
        self.kind = solver_kind
        self.lbfgs_memory = lbfgs_memory
        self.lbfgs_max_iter = lbfgs_max_iter
        self.max_halvings = max_halvings
        self.log_path = log_path
        self.ckpt_path = checkpoint_path
        self.ckpt_every = max(1, int(checkpoint_every))
        self.eig = None          # eigenstrain table in force
        self.last_R = None
        self.records = []

    # ----------------------------------------------------------- one step
    def _solve(self, dE, free_mask):
        if self.kind == "lbfgs":
            return self.s.solve_step_lbfgs(dE, free_mask=free_mask, memory=self.lbfgs_memory,
                                           max_iter=self.lbfgs_max_iter, raise_on_error=False)
        return self.s.solve_step(dE, free_mask=free_mask, raise_on_error=False)

    def _set_eig(self, table):
        self.s.set_eigenstrain(table)  # None removes it
        self.eig = None if table is None else np.array(table, dtype=np.float64, copy=True)

    def _log(self, rec):
        self.records.append(rec)
        if self.log_path:
            with open(self.log_path, "a") as f:
                f.write(json.dumps(rec) + "\n")

    def _step(self, step, dE, free_mask, eig_from, eig_to, depth):
        """Solve one (sub-)increment; on failure restore and halve."""
        st = self.s.get_state()
        eps0, kap0 = _copy(st["eps"]), _copy(st["kappa"])
        if eig_to is not None:
            self._set_eig(eig_to)
        t0 = time.perf_counter()
        rep = self._solve(dE, free_mask)
        rec = {"step": step, "depth": depth, "dE": [float(x) for x in dE], "converged": bool(rep["converged"]),
               "nr_iters": rep["nr_iters"], "cg_iters": rep["cg_iters"], "hv_products": rep["hv_products"],
               "rel_residual": rep["rel_residual"], "R": rep["R"],
               "mean_stress": [float(x) for x in rep["mean_stress"]],
               "mean_strain": [float(x) for x in rep["mean_strain"]],
               "seconds": time.perf_counter() - t0}
        self._log(rec)
        if rep["converged"]:
            self.last_R = rep["R"]
            return [rec]
        # back to the converged state (the history was not committed)
        self.s.set_state(eps0, kap0)
        if eig_to is not None:
            self._set_eig(eig_from)
        if depth >= self.max_halvings:
            raise RuntimeError(f"load step {step} did not converge after {depth} halvings of the increment "
                               "(state left at the last converged one)")
        half = [0.5 * float(x) for x in dE]
        mid = None
        if eig_to is not None:
            a = np.zeros_like(np.asarray(eig_to, dtype=np.float64)) if eig_from is None else np.asarray(eig_from)
            mid = 0.5 * (a + np.asarray(eig_to, dtype=np.float64))
        out = self._step(step, half, free_mask, eig_from, mid, depth + 1)
        out += self._step(step, half, free_mask, mid, eig_to, depth + 1)
        return out

    # ----------------------------------------------------------- path
    def run(self, increments, free_mask=None, eigenstrains=None, start=0):
        """Solve increments[start:] (eigenstrains, if given, has one table or
        None per increment).  Returns the records of the converged
        (sub-)increments, one list per increment."""
        out = []
        for n in range(start, len(increments)):
            eig_to = None if eigenstrains is None else eigenstrains[n]
            recs = self._step(n, list(increments[n]), free_mask, self.eig, eig_to, 0)
            out.append([r for r in recs if r["converged"]])
            if self.ckpt_path and ((n + 1 - start) % self.ckpt_every == 0 or n + 1 == len(increments)):
                self.save_checkpoint(self.ckpt_path, n + 1)
        return out

    # ----------------------------------------------------------- checkpoints
    def save_checkpoint(self, path, next_step):
        st = self.s.get_state()
        tmp = path + ".tmp.npz"
        np.savez(tmp, eps=_host(st["eps"]), kappa=_host(st["kappa"]), next_step=np.int64(next_step),
                 eig=np.zeros(0) if self.eig is None else self.eig,
                 last_R=np.float64(np.nan if self.last_R is None else self.last_R))
        os.replace(tmp, path)

    @staticmethod
    def load_checkpoint(path):
        with np.load(path) as z:
            return {"eps": z["eps"], "kappa": z["kappa"], "next_step": int(z["next_step"]),
                    "eig": None if z["eig"].size == 0 else z["eig"], "last_R": float(z["last_R"])}

    def resume(self, path, to_device=None):
        """Load a checkpoint into the context; returns the index of the next
        increment.  ``to_device`` converts host arrays to the context's
        field type (e.g. a torch tensor on its device)."""
        ck = self.load_checkpoint(path)
        conv = to_device if to_device is not None else (lambda a: a)
        self.s.set_state(conv(ck["eps"]), conv(ck["kappa"]))
        if ck["eig"] is not None:
            self._set_eig(ck["eig"])
        self.last_R = None if np.isnan(ck["last_R"]) else ck["last_R"]
        return ck["next_step"]
