"""Seeded synthetic point sets for the Voronoi path.

This module holds only input generation: it has none of the tessellation's
arithmetic and is shared by the GPU tests, the oracle tests and ``bench.py``.
All randomness comes from numpy's counter-based Philox generator.

The paper's own data (LCDM N-body snapshots of ~3.5 M and ~27.5 M particles,
a Gadget2 halo catalogue and an SDSS mock slice; Performance and
Implementation sections) are not available, so these generators stand in
with the shapes the benchmark workloads name:

* ``uniform``: Poisson points in a periodic box.
* ``sc_lattice`` / ``bcc_lattice``: lattices, optionally perturbed by a few
  1e-9 per coordinate so that they are in general position.
* ``clustered``: 60 % of the points in NFW halos (halo masses from a power
  law of slope -1.9 over three decades, particle count proportional to mass
  and at least 20, concentration U(5, 15), virial radius from a mean
  overdensity of 200), 25 % along random straight filaments (length U(5, 20)
  box units, Gaussian cross-section of width 0.5), 15 % uniform; wrapped
  into the periodic box, exact duplicates redrawn.
* ``halo_uniform_mix``: uniform points plus a fraction in NFW halos.
* ``halo_sets``: many independent NFW halos of log-uniform sizes, each in
  its own bounding box [-1, 1]^3.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def _wrap(x, L, dtype):
    """Wrap into [0, L) in the target precision (a value that rounds to L becomes 0)."""
    x = np.asarray(x, dtype=np.float64)
    x = x - L * np.floor(x / L)
    y = x.astype(dtype)
    y[y >= dtype(L)] = dtype(0)
    y[y < 0] = dtype(0)
    return y


def _redraw_duplicates(x, L, g, dtype):
    """Replace exact duplicate rows by fresh uniform points until none are left."""
    for _ in range(100):
        v = np.ascontiguousarray(x).view(np.dtype((np.void, x.dtype.itemsize * 3))).ravel()
        _, first, counts = np.unique(v, return_index=True, return_counts=True)
        if (counts == 1).all():
            return x
        keep = np.zeros(len(x), bool)
        keep[first] = True
        dup = ~keep
        x[dup] = _wrap(g.random((int(dup.sum()), 3)) * L, L, dtype)
    raise RuntimeError("could not remove duplicates")


def uniform(N, seed=0, L=1.0, dtype=np.float64):
    g = rng(seed)
    x = _wrap(g.random((N, 3)) * L, L, dtype)
    return _redraw_duplicates(x, L, g, dtype)


def sc_lattice(n, L=1.0, perturb=0.0, seed=0, dtype=np.float64):
    """Simple-cubic lattice with n^3 sites at ((a+1/2) L/n, ...)."""
    g1 = (np.arange(n) + 0.5) * (L / n)
    x = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    if perturb:
        x = x + rng(seed).uniform(-perturb, perturb, x.shape)
    return _wrap(x, L, dtype)


def bcc_lattice(m, L=1.0, perturb=0.0, seed=0, dtype=np.float64):
    """Body-centred cubic lattice: 2 m^3 sites, cube corners (a L/m) plus centres."""
    g1 = np.arange(m) * (L / m) + 0.25 * (L / m)
    a = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    x = np.concatenate([a, a + 0.5 * (L / m)])
    if perturb:
        x = x + rng(seed).uniform(-perturb, perturb, x.shape)
    return _wrap(x, L, dtype)


def _nfw_m(x):
    return np.log1p(x) - x / (1.0 + x)


def _nfw_radii(g, n, c, rvir):
    """Radii with NFW enclosed-mass CDF truncated at rvir (bisection on x = r/rs)."""
    u = g.random(n) * _nfw_m(c)
    lo = np.zeros(n)
    hi = np.full(n, float(c))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        less = _nfw_m(mid) < u
        lo = np.where(less, mid, lo)
        hi = np.where(less, hi, mid)
    return 0.5 * (lo + hi) * (rvir / c)


def _isotropic(g, n):
    v = g.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _halo_counts(g, n_total, n_halo, slope=-1.9, span=1e3, nmin=20):
    """Particle counts per halo, proportional to power-law masses, >= nmin, summing to n_total."""
    if n_halo * nmin > n_total:
        raise ValueError("%d halos of at least %d particles do not fit in %d" % (n_halo, nmin, n_total))
    a = slope + 1.0
    u = g.random(n_halo)
    M = (1.0 + u * (span ** a - 1.0)) ** (1.0 / a)
    cnt = np.maximum(nmin, np.floor(M / M.sum() * n_total)).astype(np.int64)
    # fix the total: remove the excess from the largest halos (never below nmin), or add the remainder to them
    order = np.argsort(-M)
    diff = int(n_total - cnt.sum())
    while diff != 0:
        if diff > 0:
            k = min(diff, n_halo)
            cnt[order[:k]] += 1
            diff -= k
        else:
            room = np.nonzero(cnt[order] > nmin)[0]
            k = min(-diff, len(room))
            cnt[order[room[:k]]] -= 1
            diff += k
    return cnt


def _halos(g, n_total, n_halo, L, nbar):
    cnt = _halo_counts(g, n_total, n_halo)
    centres = g.random((n_halo, 3)) * L
    conc = g.uniform(5.0, 15.0, n_halo)
    rvir = (3.0 * cnt / (4.0 * np.pi * 200.0 * nbar)) ** (1.0 / 3.0)
    out = np.empty((n_total, 3))
    o = 0
    for h in range(n_halo):
        n = int(cnt[h])
        r = _nfw_radii(g, n, conc[h], rvir[h])
        out[o:o + n] = centres[h] + r[:, None] * _isotropic(g, n)
        o += n
    return out


def _filaments(g, n_total, L, n_fil=1000, lmin=5.0, lmax=20.0, width=0.5):
    length = g.uniform(lmin, lmax, n_fil)
    cnt = np.floor(length / length.sum() * n_total).astype(np.int64)
    cnt[np.argsort(-length)[: n_total - cnt.sum()]] += 1
    start = g.random((n_fil, 3)) * L
    direc = _isotropic(g, n_fil)
    fid = np.repeat(np.arange(n_fil), cnt)
    t = g.random(n_total) * length[fid]
    off = g.normal(scale=width, size=(n_total, 3))
    dv = direc[fid]
    off -= (off * dv).sum(1, keepdims=True) * dv  # perpendicular offset only
    return start[fid] + t[:, None] * dv + off


def clustered(N, L=100.0, seed=1, n_halo=None, f_halo=0.60, f_fil=0.25, dtype=np.float32):
    """Halo + filament + uniform mixture in a periodic box of side L.  2000 halos and 1000
    filaments at 2,097,152 points; fewer (in proportion) for smaller sets, at least one."""
    g = rng(seed)
    scale = min(1.0, N / 2097152.0)
    if n_halo is None:
        n_halo = max(1, int(round(2000 * scale)))
    n_fil = max(1, int(round(1000 * scale)))
    nbar = N / L ** 3
    nh = int(round(f_halo * N))
    nf = int(round(f_fil * N))
    nu = N - nh - nf
    x = np.concatenate([_halos(g, nh, n_halo, L, nbar), _filaments(g, nf, L, n_fil=n_fil), g.random((nu, 3)) * L])
    x = _wrap(x, L, dtype)
    x = x[g.permutation(N)]
    return _redraw_duplicates(x, L, g, dtype)


def halo_uniform_mix(N, L=1.0, seed=3, f_halo=0.30, n_halo=None, dtype=np.float32):
    g = rng(seed)
    if n_halo is None:
        n_halo = max(1, int(round(2000 * min(1.0, N / 1048576.0))))
    nbar = N / L ** 3
    nh = int(round(f_halo * N))
    x = np.concatenate([_halos(g, nh, n_halo, L, nbar), g.random((N - nh, 3)) * L])
    x = _wrap(x, L, dtype)
    x = x[g.permutation(N)]
    return _redraw_duplicates(x, L, g, dtype)


def halo_sets(n_sets=4096, nmin=64, nmax=65536, seed=6, dtype=np.float32):
    """Independent NFW halos (r_vir = 1, c ~ U(5,15)) of log-uniform size, each in the box [-1,1]^3.
    Returns (points [sum n, 3], offsets [n_sets+1])."""
    g = rng(seed)
    sizes = np.floor(np.exp(g.uniform(np.log(nmin), np.log(nmax), n_sets))).astype(np.int64)
    off = np.zeros(n_sets + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    pts = np.empty((off[-1], 3), dtype)
    for s in range(n_sets):
        n = int(sizes[s])
        c = g.uniform(5.0, 15.0)
        p = _nfw_radii(g, n, c, 1.0)[:, None] * _isotropic(g, n)
        p = np.clip(p, -1.0, 1.0).astype(dtype)
        # exact duplicates inside a set: redraw them uniformly in the ball
        for _ in range(100):
            v = np.ascontiguousarray(p).view(np.dtype((np.void, p.dtype.itemsize * 3))).ravel()
            _, first, counts = np.unique(v, return_index=True, return_counts=True)
            if (counts == 1).all():
                break
            keep = np.zeros(n, bool)
            keep[first] = True
            d = ~keep
            p[d] = (g.random((int(d.sum()), 3)) * 2.0 - 1.0).astype(dtype)
        pts[off[s]:off[s + 1]] = p
    return pts, off


def unit_masses(N, dtype=np.float32):
    return np.ones(N, dtype)
