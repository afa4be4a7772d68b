"""Non-finite input is reported by status, not by a fault (needs a GB300).

The failure is injected on the host: a NaN written into the strain field or
the history handed to rve_set_state.  Every solver entry point must return
RVE_ERR_NONFINITE (-5), and the context must stay usable: a finite state set
afterwards solves normally."""
import numpy as np
import pytest

from synth import random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
NONFINITE = -5


def _ctx(precision, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=5)
    return RVESolver(dims, pm, [MATRIX, STIFF], precision=precision, **kw), dims


def _fields(s, where):
    eps = s.field(0.0)
    eps[2] += 2e-5  # elastic (kappa stays below kappa0 near the inclusions too)
    kap = s.scalar_field()
    kap.zero_()
    if where == "strain":
        eps[1, 3, 4, 5] = float("nan")
    elif where == "history":
        kap[2, 1, 7] = float("nan")
    else:
        eps[0, 0, 0, 0] = float("inf")
    return eps, kap


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("where", ["strain", "history", "inf"])
def test_nonfinite_state_is_reported(precision, where):
    from paper_2207_10657_gb300 import binding as B
    s, dims = _ctx(precision)
    fm = [1, 1, 0, 1, 1, 1]
    dE = [0, 0, 1e-5, 0, 0, 0]
    for call in ("solve_step", "lbfgs", "steihaug"):
        eps, kap = _fields(s, where)
        s.set_state(eps, kap)
        if call == "solve_step":
            rep = s.solve_step(dE, free_mask=fm, raise_on_error=False)
            assert rep["status"] == NONFINITE, (call, rep)
        elif call == "lbfgs":
            rep = s.solve_step_lbfgs(dE, free_mask=fm, raise_on_error=False)
            assert rep["status"] == NONFINITE, (call, rep)
        else:
            with pytest.raises(B.RveError) as ei:
                s.steihaug(1.0, 1e-2)
            assert ei.value.status == NONFINITE
    # still usable: a finite state solves
    eps = s.field(0.0)
    s.set_state(eps, None)
    rep = s.solve_step(dE, free_mask=fm)
    assert rep["converged"] and np.isfinite(rep["mean_stress"]).all()
    torch.cuda.synchronize()
    s.close()
