"""Seeded microstructure and field generators (inputs only, no solver arithmetic).

The paper's own workloads (2D concrete meso-structures with Fuller-graded
aggregates, Sec. 3.3) are not available; these stand in for them:

* ``circular_inclusion`` -- one centred disc of a given area fraction (2D).
* ``random_spheres`` -- non-overlapping spheres placed by random sequential
  addition with periodic wrap (3D), radius uniform in [rmin, rmax].
* ``random_circles`` -- the 2D analogue, stopped at a target area fraction.
* ``laminate`` -- a two-layer laminate normal to one axis, interfaces on voxel
  faces.
* ``gel_sites`` -- single voxels drawn at random inside one phase and given
  another phase id (the ASR product sites inside aggregates, Sec. 3.3).
* ``damage_snapshot`` -- a damage field drawn U[0, dmax] on damaging voxels.
* ``random_field`` -- an N(0, 1) field with ``ncomp`` components.
"""
from __future__ import annotations

import math

import numpy as np


def grid_shape(dims):
    """numpy array shape (x fastest) for grid ``dims`` = (Nx, Ny[, Nz])."""
    return tuple(int(n) for n in reversed(tuple(dims)))


def circular_inclusion(dims, vol_frac=0.3):
    """Centred disc: pixels whose centres lie within r = sqrt(f*Nx*Ny/pi) of
    the grid centre get phase 1, the rest phase 0."""
    nx, ny = dims
    r = math.sqrt(vol_frac * nx * ny / math.pi)
    y, x = np.meshgrid(np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    inside = (x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2 <= r * r
    return inside.astype(np.uint8)


def _periodic_dist2(c, pts, box):
    d = np.abs(pts - c)
    d = np.minimum(d, box - d)
    return np.sum(d * d, axis=-1)


def _place(ndim, dims, count, rmin, rmax, seed, target_frac, max_tries):
    rng = np.random.default_rng(seed)
    box = np.asarray(dims, dtype=np.float64)
    centres = []
    radii = []
    nvox = float(np.prod(box))
    frac = 0.0
    tries = 0
    while tries < max_tries:
        if count is not None and len(centres) >= count:
            break
        if target_frac is not None and frac >= target_frac:
            break
        tries += 1
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(0.0, 1.0, size=ndim) * box
        if centres:
            d2 = _periodic_dist2(c, np.asarray(centres), box)
            if np.any(d2 < (np.asarray(radii) + r) ** 2):
                continue
        centres.append(c)
        radii.append(r)
        ball = (4.0 / 3.0) * math.pi * r ** 3 if ndim == 3 else math.pi * r * r
        frac += ball / nvox
    return np.asarray(centres).reshape(-1, ndim), np.asarray(radii)


def _rasterise(dims, centres, radii):
    shape = grid_shape(dims)
    ndim = len(dims)
    phase = np.zeros(shape, dtype=np.uint8)
    box = np.asarray(dims, dtype=np.float64)
    for c, r in zip(centres, radii):
        lo = np.floor(c - r).astype(int)
        hi = np.ceil(c + r).astype(int)
        axes = [np.arange(lo[a], hi[a] + 1) for a in range(ndim)]
        mesh = np.meshgrid(*axes, indexing="ij")  # index order x, y[, z]
        d2 = np.zeros(mesh[0].shape)
        for a in range(ndim):
            d2 += (mesh[a] + 0.5 - c[a]) ** 2
        inside = d2 <= r * r
        idx = [np.mod(mesh[a][inside], dims[a]) for a in range(ndim)]
        phase[tuple(reversed(idx))] = 1
    return phase


def random_spheres(dims, count=48, rmin=4.0, rmax=10.0, seed=0,
                   target_frac=None, max_tries=200000):
    """Non-overlapping spheres (3D) by random sequential addition with
    periodic wrap.  With ``target_frac`` set, spheres are added until that
    volume fraction is reached (``count`` then acts as an upper bound unless
    None).  Returns a uint8 phase map (1 = sphere)."""
    centres, radii = _place(3, dims, count, rmin, rmax, seed, target_frac, max_tries)
    return _rasterise(dims, centres, radii)


def random_circles(dims, target_frac=0.3, rmin=None, rmax=None, seed=0,
                   max_tries=200000):
    """Non-overlapping discs (2D) up to an area fraction."""
    n = min(dims)
    rmin = rmin if rmin is not None else max(2.0, n / 32.0)
    rmax = rmax if rmax is not None else max(rmin + 1.0, n / 8.0)
    centres, radii = _place(2, dims, None, rmin, rmax, seed, target_frac, max_tries)
    return _rasterise(dims, centres, radii)


def laminate(dims, axis=2, frac=0.5):
    """Two-layer laminate normal to ``axis`` (0=x, 1=y, 2=z): voxels with
    index < frac*N along that axis are phase 0, the rest phase 1."""
    shape = grid_shape(dims)
    n = dims[axis]
    cut = int(round(frac * n))
    idx = np.arange(n) >= cut
    ndim = len(dims)
    view = [1] * ndim
    view[ndim - 1 - axis] = n
    return np.broadcast_to(idx.reshape(view), shape).astype(np.uint8).copy()


def gel_sites(phase, count, host=1, site=2, seed=3):
    """Copy of ``phase`` with ``count`` distinct voxels of phase ``host``,
    drawn uniformly without replacement, set to phase ``site``."""
    rng = np.random.default_rng(seed)
    out = np.array(phase, dtype=np.uint8, copy=True)
    cand = np.flatnonzero(out == host)
    if count > cand.size:
        raise ValueError("more sites than host voxels")
    pick = rng.choice(cand, size=count, replace=False)
    out.reshape(-1)[pick] = site
    return out


def damage_snapshot(phase, damaging_phases=(0,), dmax=0.9, seed=1, dtype=np.float32):
    """Damage field drawn U[0, dmax] on voxels of the damaging phases, 0
    elsewhere (a mid-softening snapshot for Hessian-vector benchmarks)."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.0, dmax, size=phase.shape)
    mask = np.isin(phase, np.asarray(damaging_phases, dtype=phase.dtype))
    return np.where(mask, d, 0.0).astype(dtype)


def random_field(ncomp, dims, seed=2, dtype=np.float64):
    """N(0, 1) field of shape (ncomp, *grid)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((ncomp,) + grid_shape(dims)).astype(dtype)


def five_smooth_sizes(lo, hi):
    """All integers in [lo, hi] whose prime factors are 2, 3 and 5."""
    out = []
    for n in range(lo, hi + 1):
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out
