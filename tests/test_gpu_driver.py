"""Load-path driver around a real context (needs a GB300): checkpoint /
resume in a fresh context equals the uninterrupted path, and a load step
that cannot converge leaves the context at the last converged state."""
import numpy as np
import pytest

from synth import random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
FREE = [1, 1, 0, 1, 1, 1]


def _solver(dims, pm, **kw):
    from paper_2207_10657_gb300 import RVESolver, build
    build.build()
    return RVESolver(dims, pm, [MATRIX, STIFF], precision=64, **kw)


def test_checkpoint_resume_on_device(tmp_path):
    from paper_2207_10657_gb300.driver import LoadPathDriver
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    incs = [[0, 0, 2e-5, 0, 0, 0]] * 3
    opts = dict(eta_eq=1e-10, R0=1.0, Rmax=1.0, max_nr=200)
    ref = _solver(dims, pm, **opts)
    LoadPathDriver(ref).run(incs, free_mask=FREE)
    ck = str(tmp_path / "ck.npz")
    a = _solver(dims, pm, **opts)
    LoadPathDriver(a, checkpoint_path=ck, log_path=str(tmp_path / "log.jsonl")).run(incs[:2], free_mask=FREE)
    a.close()
    b = _solver(dims, pm, **opts)
    db = LoadPathDriver(b)
    start = db.resume(ck, to_device=lambda x: torch.from_numpy(x).cuda())
    assert start == 2
    b.set_free_mask(FREE)
    db.run(incs, free_mask=FREE, start=start)
    eb, er = b.get_state()["eps"], ref.get_state()["eps"]
    assert float(torch.linalg.vector_norm(eb - er) / torch.linalg.vector_norm(er)) < 1e-9
    assert len((tmp_path / "log.jsonl").read_text().splitlines()) == 2
    ref.close()
    b.close()


def test_unconverged_step_restores_the_state():
    from paper_2207_10657_gb300.driver import LoadPathDriver
    dims = (16, 12, 10)
    pm = random_spheres(dims, count=3, rmin=2.0, rmax=3.0, seed=7)
    s = _solver(dims, pm, eta_eq=1e-12, eta_cg=1e-1, max_nr=1)
    st0 = s.get_state()
    eps0, kap0 = st0["eps"].clone(), st0["kappa"].clone()
    with pytest.raises(RuntimeError, match="did not converge"):
        LoadPathDriver(s, max_halvings=1).run([[0, 0, 2e-5, 0, 0, 0]], free_mask=FREE)
    st = s.get_state()
    assert torch.equal(st["eps"], eps0) and torch.equal(st["kappa"], kap0)
    s.close()
