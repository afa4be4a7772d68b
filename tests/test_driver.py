"""Load-path driver on the host (no GPU): non-convergence handled by
restoring the converged state and halving the increment (failures injected
by a fake solver context), eigenstrain interpolation of the halves,
checkpoint / resume equal to an uninterrupted run, and the JSON-lines log."""
import json

import numpy as np
import pytest

from paper_2207_10657_gb300.driver import LoadPathDriver


class FakeSolver:
    """Host stand-in for a solver context: a step converges only when its
    load change (increment plus eigenstrain change) is at most ``limit``;
    a failed step scrambles the strain and commits nothing, like a real
    context that stopped at max_nr."""

    def __init__(self, limit=0.4):
        self.limit = limit
        self.eps = np.zeros((6, 2, 2))
        self.kappa = np.zeros((2, 2))
        self.eig = None
        self.eig_conv = np.zeros((2, 6))
        self.calls = []

    def get_state(self):
        return {"eps": self.eps.copy(), "kappa": self.kappa.copy()}

    def set_state(self, eps, kappa):
        self.eps = np.array(eps, copy=True)
        self.kappa = np.array(kappa, copy=True)

    def set_eigenstrain(self, table):
        self.eig = None if table is None else np.array(table, dtype=np.float64)

    def _step(self, dE, kind):
        self.calls.append(kind)
        eig = np.zeros((2, 6)) if self.eig is None else self.eig
        load = np.linalg.norm(dE) + np.linalg.norm(eig - self.eig_conv)
        rep = {"nr_iters": 3, "cg_iters": 10, "hv_products": 10, "rel_residual": 1e-7, "R": 1.0,
               "mean_stress": [0.0] * 6, "mean_strain": [0.0] * 6}
        if load > self.limit + 1e-12:
            self.eps += 123.0  # garbage left behind by a failed step
            rep.update(converged=False)
            return rep
        self.eps += np.asarray(dE, dtype=np.float64).reshape(6, 1, 1)
        self.kappa = np.maximum(self.kappa, np.abs(self.eps).max(axis=0))
        self.eig_conv = eig.copy()
        rep.update(converged=True, mean_strain=list(self.eps.mean(axis=(1, 2))))
        return rep

    def solve_step(self, dE, free_mask=None, raise_on_error=True):
        return self._step(dE, "tr")

    def solve_step_lbfgs(self, dE, free_mask=None, memory=5, max_iter=500, raise_on_error=True):
        return self._step(dE, "lbfgs")


def _inc(x):
    return [0.0, 0.0, x, 0.0, 0.0, 0.0]


def test_failed_step_is_restored_and_halved(tmp_path):
    s = FakeSolver(limit=0.4)
    log = tmp_path / "log.jsonl"
    d = LoadPathDriver(s, log_path=str(log))
    out = d.run([_inc(0.3), _inc(1.0), _inc(0.3)])
    # 1.0 -> two halves of 0.5 (fail) -> four quarters of 0.25
    assert [len(o) for o in out] == [1, 4, 1]
    assert all(r["depth"] == 2 for r in out[1])
    np.testing.assert_allclose(s.eps[2], 1.6)
    np.testing.assert_allclose(s.eps[[0, 1, 3, 4, 5]], 0.0)
    lines = [json.loads(x) for x in log.read_text().splitlines()]
    assert sum(not r["converged"] for r in lines) == 3  # 1.0, and both 0.5 halves
    assert sum(r["converged"] for r in lines) == 6


def test_gives_up_after_max_halvings():
    s = FakeSolver(limit=0.1)
    d = LoadPathDriver(s, max_halvings=2)
    with pytest.raises(RuntimeError, match="did not converge"):
        d.run([_inc(1.0)])
    # the state is the last converged one, not the garbage of the failures
    assert np.all(np.abs(s.eps) < 1.0)


def test_eigenstrain_change_is_interpolated_over_the_halves():
    s = FakeSolver(limit=0.4)
    d = LoadPathDriver(s)
    t1 = np.zeros((2, 6))
    t1[1, :3] = -0.2           # |change| = 0.35: one step
    t2 = np.zeros((2, 6))
    t2[1, :3] = -0.6           # |change| = 0.69: two halves
    out = d.run([_inc(0.0), _inc(0.0)], eigenstrains=[t1, t2])
    assert [len(o) for o in out] == [1, 2]
    np.testing.assert_allclose(s.eig, t2)
    np.testing.assert_allclose(d.eig, t2)


def test_checkpoint_resume_equals_uninterrupted_run(tmp_path):
    incs = [_inc(0.3), _inc(1.0), _inc(0.2), _inc(0.35)]
    ref = FakeSolver()
    LoadPathDriver(ref).run(incs)
    ck = tmp_path / "state.npz"
    a = FakeSolver()
    LoadPathDriver(a, checkpoint_path=str(ck), checkpoint_every=1).run(incs[:2])
    b = FakeSolver()
    db = LoadPathDriver(b, checkpoint_path=str(ck))
    start = db.resume(str(ck))
    assert start == 2
    db.run(incs, start=start)
    np.testing.assert_allclose(b.eps, ref.eps)
    np.testing.assert_allclose(b.kappa, ref.kappa)
    assert LoadPathDriver.load_checkpoint(str(ck))["next_step"] == 4


def test_lbfgs_kind_calls_the_lbfgs_step():
    s = FakeSolver()
    LoadPathDriver(s, solver_kind="lbfgs").run([_inc(0.1)])
    assert s.calls == ["lbfgs"]
    with pytest.raises(ValueError):
        LoadPathDriver(s, solver_kind="newton")
