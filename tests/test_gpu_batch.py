"""Batched solver (many RVEs of uneven sizes in one launch per pass) against
independent single-RVE contexts and the oracle (needs a GB300)."""
import numpy as np
import pytest

import oracle
from synth import circular_inclusion, random_circles, random_spheres, damage_snapshot, random_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)

# mixed 2D / 3D members, fast and generic axis lengths, ragged tiles
DIMS = [(64, 64), (96, 60), (32, 32, 32), (48, 40, 30), (16, 24, 20), (128, 72)]


def _micro(dims, seed):
    if len(dims) == 2:
        return random_circles(dims, target_frac=0.25, seed=seed)
    return random_spheres(dims, count=4, rmin=2.0, rmax=4.0, seed=seed)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batched_hessp_matches_single_and_oracle():
    from paper_2207_10657_gb300 import RVEBatch, RVESolver, build
    build.build()
    pms = [_micro(d, 10 + i) for i, d in enumerate(DIMS)]
    Ds = [damage_snapshot(pm, dmax=0.9, seed=20 + i) for i, pm in enumerate(pms)]
    vs = [random_field(3 if len(d) == 2 else 6, d, seed=30 + i, dtype=np.float32) for i, d in enumerate(DIMS)]
    b = RVEBatch(DIMS, pms, [MATRIX, STIFF])
    for i, D in enumerate(Ds):
        b.set_damage(i, torch.from_numpy(D).cuda())
    outs = b.hessp([torch.from_numpy(v).cuda() for v in vs])
    for i, d in enumerate(DIMS):
        s = RVESolver(d, pms[i], [MATRIX, STIFF], precision=32)
        s.set_damage(torch.from_numpy(Ds[i]).cuda())
        ref = s.hessp(torch.from_numpy(vs[i]).cuda()).cpu().numpy()
        s.close()
        got = outs[i].cpu().numpy()
        assert _rel(got, ref) < 2e-6, (d, _rel(got, ref))
        if i in (1, 3):
            orv = oracle.RVE(pms[i], [oracle.Phase(1.0, 0.3, True, 1e-4, 1e-3), oracle.Phase(10.0, 0.2)])
            o = orv.hessp(Ds[i].astype(np.float64), vs[i].astype(np.float64))
            assert _rel(got, o) < 1e-5, d
    b.close()


def test_every_schedule_gives_the_same_products():
    """Every schedule the autotuner may pick (tile divisors 1, 2, 4 per pass,
    natural or reversed radix order) gives the same batched Hv as the single
    contexts; the tuned schedule is kept for later calls."""
    from paper_2207_10657_gb300 import RVEBatch, RVESolver, binding as B, build
    build.build()
    dims = [(64, 64), (96, 60), (32, 32, 32), (48, 40, 30), (16, 24, 20)]
    pms = [_micro(d, 60 + i) for i, d in enumerate(dims)]
    vs = [random_field(3 if len(d) == 2 else 6, d, seed=70 + i, dtype=np.float32) for i, d in enumerate(dims)]
    refs = []
    for i, d in enumerate(dims):
        s = RVESolver(d, pms[i], [MATRIX, STIFF], precision=32)
        refs.append(s.hessp(torch.from_numpy(vs[i]).cuda()).cpu().numpy())
        s.close()
    b = RVEBatch(dims, pms, [MATRIX, STIFF])
    for sx in (1, 2, 4):
        for sy in (1, 2, 4):
            for sz in (1, 2, 4):
                for rev in (0, 1):
                    B.rve_batch_set_schedule(b.h, [sx, sy, sz, rev])
                    outs = b.hessp([torch.from_numpy(v).cuda() for v in vs])
                    for i in range(len(dims)):
                        assert _rel(outs[i].cpu().numpy(), refs[i]) < 2e-6, (dims[i], sx, sy, sz, rev)
    with pytest.raises(B.RveError):
        B.rve_batch_set_schedule(b.h, [3, 1, 1, 0])
    tuned = b.autotune(reps=2)
    assert tuned["ms_per_product"] > 0 and tuned["ms_per_product"] <= tuned["ms_per_product_default"]
    outs = b.hessp([torch.from_numpy(v).cuda() for v in vs])
    for i in range(len(dims)):
        assert _rel(outs[i].cpu().numpy(), refs[i]) < 2e-6, (dims[i], tuned)
    b.close()


def test_batched_load_steps_match_single_contexts():
    """Two load increments (elastic, then the onset of damage) per member,
    each member with its own load direction: the batched lockstep solve
    takes the same Newton / CG iterations as independent single-RVE solves
    and reaches the same homogenised stress.  The elastic increment must
    converge; at the onset of damage a member may localise and exhaust the
    Newton cap, identically on both sides."""
    from paper_2207_10657_gb300 import RVEBatch, RVESolver, build
    build.build()
    rng = np.random.default_rng(4)
    pms = [_micro(d, 40 + i) for i, d in enumerate(DIMS)]
    dEs, frees = [], []
    for d in DIMS:
        nc = 3 if len(d) == 2 else 6
        a = rng.standard_normal(nc)
        a *= 4e-5 / np.linalg.norm(a)
        dEs.append(list(a))
        frees.append([0] * nc)
    opts = dict(eta_eq=1e-6, eta_cg=1e-2, max_nr=200)
    b = RVEBatch(DIMS, pms, [MATRIX, STIFF], **opts)
    singles = [RVESolver(d, pms[i], [MATRIX, STIFF], precision=32, **opts) for i, d in enumerate(DIMS)]
    for step in range(2):
        reps = b.solve_step(dEs, frees, raise_on_error=False)
        for i, s in enumerate(singles):
            rs = s.solve_step(dEs[i], free_mask=frees[i], raise_on_error=False)
            if step == 0:
                assert reps[i]["converged"] and rs["converged"], (i, step, reps[i], rs)
            assert reps[i]["converged"] == rs["converged"]
            assert abs(reps[i]["nr_iters"] - rs["nr_iters"]) <= 2, (i, step, reps[i], rs)
            sb = np.array(reps[i]["mean_stress"])
            ss = np.array(rs["mean_stress"])
            assert np.linalg.norm(sb - ss) <= 1e-4 * np.linalg.norm(ss), (i, step, sb, ss)
    for s in singles:
        s.close()
    b.close()


def test_batched_consistent_load_steps_match_single_contexts():
    """The same two increments with the symmetric consistent tangent as the
    Hessian (rve_solver_opts.hessian = 1) on both sides: the batched solve
    prepares the tangent's per-voxel data member by member and carries it
    through the captured CG iteration; Newton iteration counts (within 1),
    convergence and homogenised stress (1e-4 relative) as the single
    contexts; a member that localises at the onset exhausts the Newton cap
    on both sides."""
    from paper_2207_10657_gb300 import RVEBatch, RVESolver, build
    build.build()
    rng = np.random.default_rng(4)
    pms = [_micro(d, 40 + i) for i, d in enumerate(DIMS)]
    dEs, frees = [], []
    for d in DIMS:
        nc = 3 if len(d) == 2 else 6
        a = rng.standard_normal(nc)
        a *= 4e-5 / np.linalg.norm(a)
        dEs.append(list(a))
        frees.append([0] * nc)
    opts = dict(eta_eq=1e-6, eta_cg=1e-2, max_nr=200, hessian=1)
    b = RVEBatch(DIMS, pms, [MATRIX, STIFF], **opts)
    singles = [RVESolver(d, pms[i], [MATRIX, STIFF], precision=32, **opts) for i, d in enumerate(DIMS)]
    for step in range(2):
        reps = b.solve_step(dEs, frees, raise_on_error=False)
        for i, s in enumerate(singles):
            rs = s.solve_step(dEs[i], free_mask=frees[i], raise_on_error=False)
            if step == 0:
                assert reps[i]["converged"] and rs["converged"], (i, step, reps[i], rs)
            assert reps[i]["converged"] == rs["converged"], (i, step, reps[i], rs)
            if not rs["converged"]:  # localised: both sides exhaust the Newton cap
                assert reps[i]["nr_iters"] == rs["nr_iters"] == 200
                continue
            assert abs(reps[i]["nr_iters"] - rs["nr_iters"]) <= 1, (i, step, reps[i], rs)
            sb = np.array(reps[i]["mean_stress"])
            ss = np.array(rs["mean_stress"])
            assert np.linalg.norm(sb - ss) <= 1e-4 * np.linalg.norm(ss), (i, step, sb, ss)
    for s in singles:
        s.close()
    b.close()


def test_batched_2d_elastic_step_matches_oracle():
    """A single elastic increment on a batch of 2D cells agrees with the
    oracle's trust-region solve to the solver tolerance."""
    from paper_2207_10657_gb300 import RVEBatch, build
    from oracle.solver import TRParams, load_path
    build.build()
    dims = [(32, 32), (40, 24)]
    pms = [circular_inclusion(dims[0], 0.3), _micro(dims[1], 7)]
    phases = [(1.0, 0.3, False, 0.0, 0.0), (10.0, 0.3, False, 0.0, 0.0)]
    dE = [[1e-3, 0.0, 0.0], [0.0, 5e-4, 2e-4]]
    b = RVEBatch(dims, pms, phases, eta_eq=1e-7, eta_cg=1e-6, R0=1.0, Rmax=1.0)
    reps = b.solve_step(dE, [[0, 1, 1], [0, 0, 0]])
    for i, d in enumerate(dims):
        orv = oracle.RVE(pms[i], [oracle.Phase(1.0, 0.3), oracle.Phase(10.0, 0.3)],
                         free_mask=np.array([[0, 1, 1], [0, 0, 0]][i], bool))
        ref = load_path(orv, [np.array(dE[i])], TRParams(eta_eq=1e-10, eta_cg=1e-10, R0=1.0, Rmax=1.0))
        sref = ref["mean_stress"][-1]
        assert np.linalg.norm(np.array(reps[i]["mean_stress"][:3]) - sref) <= 1e-5 * np.linalg.norm(sref)
    b.close()
