"""Learned warm start end to end on the GPU: training pairs from the plain
solver, training by the library's own forward / backward / Adam kernels, and
the A/B against the plain method on a held-out, larger cell (needs a GB300).

What the trained network gains: a starting increment closer to the
converged one than the uniform predictor's; what it may not change: the
converged result (the plain solver still decides convergence)."""
import numpy as np
import pytest

from synth import random_spheres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MATRIX = (1.0, 0.3, True, 1e-4, 1e-3)
STIFF = (10.0, 0.2, False, 0.0, 0.0)
FREE = [1, 1, 0, 1, 1, 1]
DE = [0.0, 0.0, 1e-5, 0.0, 0.0, 0.0]
OPTS = dict(eta_eq=1e-6, eta_cg=1e-2, max_nr=150)


def _cell(n, seed):
    # 48 spheres, radius U[4, 10] voxels at 128^3, scaled with the grid
    return random_spheres((n, n, n), count=48, rmin=4.0 * n / 128, rmax=10.0 * n / 128, seed=seed)


def test_trained_warm_start_starts_closer_and_leaves_result_unchanged():
    from paper_2207_10657_gb300 import build
    from paper_2207_10657_gb300.learned import SpectralOperator, compare_warm_start, generate_samples, train
    build.build()
    net = SpectralOperator(layers=4, modes=8, seed=0)
    cells = [_cell(32, 100 + i) for i in range(10)]
    Xs, Ts, log = generate_samples(net, cells, [MATRIX, STIFF], DE, FREE, 6, **OPTS)
    assert len(Xs) >= 30
    zero = np.mean([float((T ** 2).mean()) for T in Ts])
    hist = train(net, Xs, Ts, (32, 32, 32), 300, batch=4, lr=2e-3, seed=1)
    assert np.mean(hist[-30:]) < 0.2 * zero, (zero, hist[:3], hist[-3:])
    recs = compare_warm_start(net, _cell(48, 999), [MATRIX, STIFF], DE, FREE, 5, **OPTS)
    assert len(recs) == 5
    for r in recs:
        p, l, v = r["plain"], r["learned"], r["previous"]
        assert p["converged"] and l["converged"] and v["converged"], r
        # the same equilibrium to the solver tolerance
        sp, sl = np.array(p["mean_stress"]), np.array(l["mean_stress"])
        assert np.linalg.norm(sl - sp) <= 1e-5 * np.linalg.norm(sp), r
        # a better start than the uniform predictor (whose distance is 1)
        assert p["start_err"] == pytest.approx(1.0)
        assert l["start_err"] < 0.5, r
    net.close()
