"""The seeded input generators (no GPU): determinism, ranges, no duplicates, and the distributions of the
stated recipe (NFW radii, power-law halo counts, filament cross-sections, log-uniform set sizes)."""
import numpy as np
import pytest

from paper_1601_06429_gb300 import inputs


def _no_duplicates(x):
    v = np.ascontiguousarray(x).view(np.dtype((np.void, x.dtype.itemsize * 3))).ravel()
    return len(np.unique(v)) == len(x)


def test_same_seed_same_points_other_seed_other_points():
    a = inputs.clustered(20000, L=10.0, seed=1)
    b = inputs.clustered(20000, L=10.0, seed=1)
    c = inputs.clustered(20000, L=10.0, seed=2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_periodic_sets_are_half_open_and_duplicate_free(dtype):
    for x, L in ((inputs.uniform(5000, seed=0, dtype=dtype), 1.0),
                 (inputs.clustered(50000, L=10.0, seed=1, dtype=dtype), 10.0),
                 (inputs.halo_uniform_mix(50000, L=1.0, seed=3, dtype=dtype), 1.0)):
        assert x.dtype == dtype and x.shape[1] == 3
        assert (x >= 0).all() and (x < dtype(L)).all()
        assert _no_duplicates(x)


def test_wrap_maps_values_that_round_to_the_box_length_to_zero():
    x = inputs._wrap(np.array([[1.0 - 1e-12, -1e-12, 0.5]]), 1.0, np.float32)
    assert x.tolist() == [[0.0, 0.0, 0.5]]


def test_halo_counts_sum_minimum_and_power_law():
    g = inputs.rng(0)
    cnt = inputs._halo_counts(g, 1_000_000, 2000)
    assert cnt.sum() == 1_000_000 and cnt.min() >= 20
    # masses of slope -1.9 over three decades: the largest halo holds far more than the median one
    assert cnt.max() / np.median(cnt) > 50
    with pytest.raises(ValueError):
        inputs._halo_counts(g, 100, 10)


def test_nfw_radii_follow_the_truncated_enclosed_mass_profile():
    g = inputs.rng(1)
    c, rvir, n = 10.0, 2.0, 200000
    r = inputs._nfw_radii(g, n, c, rvir)
    assert (r >= 0).all() and (r <= rvir).all()
    # empirical CDF against M(r c / rvir) / M(c) at a few radii (Kolmogorov bound ~ 1.6 / sqrt(n))
    m = lambda t: np.log1p(t) - t / (1 + t)  # noqa: E731
    for q in (0.05, 0.1, 0.25, 0.5, 0.9):
        cdf = m(q * c) / m(c)
        assert abs((r <= q * rvir).mean() - cdf) < 1.6 / np.sqrt(n) + 1e-3


def test_isotropic_directions_are_unit_and_centred():
    v = inputs._isotropic(inputs.rng(2), 100000)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    assert np.abs(v.mean(0)).max() < 0.01
    assert np.allclose((v ** 2).mean(0), 1.0 / 3.0, atol=0.01)


def test_filament_offsets_are_perpendicular_gaussians():
    g = inputs.rng(3)
    n_fil, n = 4, 40000
    x = inputs._filaments(g, n, 100.0, n_fil=n_fil, width=0.5)
    assert x.shape == (n, 3)
    # replay the generator's draws to recover each point's filament axis
    g = inputs.rng(3)
    length = g.uniform(5.0, 20.0, n_fil)
    cnt = np.floor(length / length.sum() * n).astype(np.int64)
    cnt[np.argsort(-length)[: n - cnt.sum()]] += 1
    start = g.random((n_fil, 3)) * 100.0
    d = inputs._isotropic(g, n_fil)
    fid = np.repeat(np.arange(n_fil), cnt)
    rel = x - start[fid]
    along = (rel * d[fid]).sum(1)
    perp = rel - along[:, None] * d[fid]
    assert (along >= 0).all() and (along <= length[fid]).all()
    # a 2D isotropic Gaussian of sigma 0.5 per axis: E|perp|^2 = 2 sigma^2
    assert abs((perp ** 2).sum(1).mean() - 0.5) < 0.02


def test_clustered_mixture_fractions():
    # 60 % of the points in halos and 25 % in thin filaments: the typical nearest-neighbour distance of the
    # clustered set is far below that of a uniform set of the same mean density
    from scipy.spatial import cKDTree

    N, L = 65536, 25.0
    x = inputs.clustered(N, L=L, seed=1).astype(np.float64)
    u = inputs.uniform(N, seed=1, L=L)
    dx = cKDTree(x, boxsize=L).query(x, k=2)[0][:, 1]
    du = cKDTree(u, boxsize=L).query(u, k=2)[0][:, 1]
    assert np.median(dx) < 0.5 * np.median(du)
    # the uniform 15 % keeps the largest gaps close to the uniform set's
    assert np.quantile(dx, 0.999) > 0.5 * np.quantile(du, 0.999)


def test_halo_sets_sizes_boxes_and_duplicates():
    pts, off = inputs.halo_sets(n_sets=512, nmin=64, nmax=4096, seed=6)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == len(pts)
    assert sizes.min() >= 64 and sizes.max() < 4096
    # log-uniform: the mean of log(size) is the midpoint of [log 64, log 4096] (up to the floor)
    assert abs(np.log(sizes).mean() - 0.5 * (np.log(64) + np.log(4096))) < 0.15
    assert (np.abs(pts) <= 1.0).all()
    for s in range(0, 512, 37):
        assert _no_duplicates(pts[off[s]:off[s + 1]])


def test_lattices():
    x = inputs.sc_lattice(4)
    assert x.shape == (64, 3) and np.allclose(np.unique(x[:, 0]), (np.arange(4) + 0.5) / 4)
    b = inputs.bcc_lattice(3)
    assert b.shape == (54, 3) and _no_duplicates(b)
    p = inputs.bcc_lattice(3, perturb=1e-9, seed=0)
    assert 0 < np.abs(p - b).max() <= 1e-9 + 1e-16
