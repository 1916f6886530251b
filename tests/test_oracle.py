"""Pins of the FP64 oracle against what the mathematics fixes.

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign, a transposed operand, a missed periodic image) fails one of
them: lattice closed forms, invariants of a tessellation, the exact
predicate against rational arithmetic, brute force against the certified
k-d tree mode, the Poisson-Voronoi means of Meijering (1953), and finite
differences for the derivatives.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1601_06429_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# lattices
# --------------------------------------------------------------------------
def test_sc_lattice_cubes(oracle_mod):
    n = 16
    a = 1.0 / n
    x = inputs.sc_lattice(n)
    r = oracle_mod.cells(x, 0.0, 1.0, True, which=np.arange(0, n ** 3, 97), mode="brute")
    assert np.allclose(r["vol"], a ** 3, rtol=1e-13, atol=0)
    assert (r["nface"] == 6).all() and (r["nvert"] == 8).all() and (r["nedge"] == 12).all()
    assert np.allclose(r["f_area"], a * a, rtol=1e-12)
    assert np.allclose(r["f_dist"], a / 2, rtol=1e-12)
    # the exactly degenerate vertices (8 cells meet) are decided by the exact predicate
    assert r["counters"][1] > 0 and r["counters"][2] > 0


def test_sc_lattice_perturbed(oracle_mod):
    n = 16
    a = 1.0 / n
    x = inputs.sc_lattice(n, perturb=1e-9, seed=0)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    assert abs(r["vol"].sum() - 1.0) < 1e-12
    assert np.allclose(r["vol"], a ** 3, rtol=1e-6)
    off = r["face_off"]
    # the perturbation splits every 4-cell edge into a sliver facet of area
    # ~ a * 1e-9 and every 8-cell vertex into facets of area ~ 1e-18: exactly
    # six facets keep an area of order a^2
    big = r["f_area"] > 1e-6 * a * a
    nbig = np.add.reduceat(big.astype(np.int64), off[:-1])
    assert (nbig == 6).all()
    # perturbation splits the 8-cell vertices: some cells have more than 6 facets
    assert r["nface"].max() > 6
    assert r["counters"][2] == 0  # no exact zero: general position


@pytest.mark.parametrize("perturb", [0.0, 1e-9])
def test_bcc_truncated_octahedra(oracle_mod, perturb):
    m = 8
    a = 1.0 / m
    x = inputs.bcc_lattice(m, perturb=perturb, seed=0)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    assert abs(r["vol"].sum() - 1.0) < 1e-12
    assert np.allclose(r["vol"], a ** 3 / 2, rtol=1e-6)
    assert (r["nface"] == 14).all()
    assert (r["nvert"] == 24).all() and (r["nedge"] == 36).all()
    A = r["f_area"].reshape(-1, 14)
    D = r["f_dist"].reshape(-1, 14)
    o = np.argsort(A, axis=1)
    A = np.take_along_axis(A, o, 1)
    D = np.take_along_axis(D, o, 1)
    assert np.allclose(A[:, :6], a * a / 8, rtol=1e-6)
    assert np.allclose(A[:, 6:], 3 * math.sqrt(3) * a * a / 16, rtol=1e-6)
    assert np.allclose(D[:, :6], a / 2, rtol=1e-6)
    assert np.allclose(D[:, 6:], a * math.sqrt(3) / 4, rtol=1e-6)
    # divergence theorem: V = 1/3 sum A h
    assert np.allclose((A * D).sum(1) / 3, a ** 3 / 2, rtol=1e-6)


# --------------------------------------------------------------------------
# invariants on Poisson points
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def poisson(oracle_mod):
    x = inputs.uniform(4096, seed=0)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")
    return x, r


def test_total_volume_and_euler(poisson):
    x, r = poisson
    assert abs(r["vol"].sum() - 1.0) < 1e-12
    assert (r["nvert"] - r["nedge"] + r["nface"] == 2).all()
    # simple polytope: every vertex has degree 3, so 2E = 3V
    assert (2 * r["nedge"] == 3 * r["nvert"]).all()
    assert r["counters"][3] == 0


def test_divergence_theorem_and_closed_surface(poisson):
    x, r = poisson
    off = r["face_off"]
    vol_div = np.add.reduceat(r["f_area"] * r["f_dist"], off[:-1]) / 3.0
    assert np.allclose(vol_div, r["vol"], rtol=1e-10)
    # sum_f A_f n_f = 0 with n_f the unit normal towards the neighbour image
    L = 1.0
    i = np.repeat(np.arange(len(x)), np.diff(off))
    d = x[r["f_nbr"]] + r["f_shift"] * L - x[i]
    n = d / np.linalg.norm(d, axis=1, keepdims=True)
    s = np.zeros((len(x), 3))
    np.add.at(s, i, r["f_area"][:, None] * n)
    scale = r["vol"] ** (2.0 / 3.0)
    assert (np.abs(s).max(1) / scale).max() < 1e-10


def test_neighbour_symmetry_shared_facets(poisson):
    x, r = poisson
    off = r["face_off"]
    i = np.repeat(np.arange(len(x)), np.diff(off))
    j = r["f_nbr"]
    key = {}
    for f in range(len(j)):
        key[(int(i[f]), int(j[f]), tuple(r["f_shift"][f]))] = f
    for (a, b, s), f in key.items():
        g = key.get((b, a, tuple(-np.array(s))))
        assert g is not None, "facet (%d,%d) has no partner" % (a, b)
        assert abs(r["f_area"][f] - r["f_area"][g]) <= 1e-9 * r["f_area"][f] + 1e-15
        # same facet seen from both sides: centroids agree up to the image shift
        cf = r["f_cen"][f]
        cg = r["f_cen"][g] + np.array(s)
        assert np.abs(cf - cg).max() < 1e-12


def test_meijering_face_statistics(poisson):
    x, r = poisson
    gold = json.load(open(os.path.join(GOLD, "paper_values.json")))
    faces = 2 + 48 * math.pi ** 2 / 35
    m = r["nface"].mean()
    se = r["nface"].std() / math.sqrt(len(x))
    assert abs(m - faces) < 4 * se
    assert abs(r["nvert"].mean() - 96 * math.pi ** 2 / 35) < 8 * se
    lo, hi = gold["poisson_faces_per_cell"]["range"]
    assert lo <= m <= hi


def test_brute_equals_certified(poisson, oracle_mod):
    x, r = poisson
    c = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    assert np.array_equal(c["nface"], r["nface"])
    assert np.abs(c["vol"] - r["vol"]).max() < 1e-15
    o1, n1 = oracle_mod.neighbours(r)
    o2, n2 = oracle_mod.neighbours(c)
    assert np.array_equal(o1, o2) and np.array_equal(n1, n2)


def test_kept_tree_equals_certified(poisson, oracle_mod):
    """The k-d tree built once and kept (oracle.Tree) gives the brute-force cells on any subset, in any order,
    over several calls; its build time is reported."""
    x, r = poisson
    t = oracle_mod.Tree(x, 0.0, 1.0, True)
    assert t.build_seconds >= 0.0
    for which in (np.arange(len(x)), np.random.default_rng(3).permutation(len(x))[:300]):
        c = t.cells(which)
        assert np.array_equal(c["nface"], r["nface"][which])
        assert np.abs(c["vol"] - r["vol"][which]).max() < 1e-15
        o1, n1 = oracle_mod.neighbours(oracle_mod.cells(x, 0.0, 1.0, True, which=which, mode="brute"))
        o2, n2 = oracle_mod.neighbours(c)
        assert np.array_equal(o1, o2) and np.array_equal(n1, n2)
    t.close()


def test_invariance_scale_translate_permute(oracle_mod):
    x = inputs.uniform(512, seed=3)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")
    # scale by 2 (exact in binary): volumes scale by 8
    r2 = oracle_mod.cells(2.0 * x, 0.0, 2.0, True, mode="brute")
    assert np.allclose(r2["vol"], 8.0 * r["vol"], rtol=1e-13)
    # periodic translation by an exactly representable shift
    xs = np.mod(x + 0.375, 1.0)
    r3 = oracle_mod.cells(xs, 0.0, 1.0, True, mode="brute")
    assert np.allclose(r3["vol"], r["vol"], rtol=1e-9)
    # permutation
    p = np.random.default_rng(0).permutation(len(x))
    r4 = oracle_mod.cells(x[p], 0.0, 1.0, True, mode="brute")
    assert np.abs(r4["vol"] - r["vol"][p]).max() < 1e-15
    o, ids = oracle_mod.neighbours(r)
    o4, ids4 = oracle_mod.neighbours(r4)
    inv = np.argsort(p)
    for k in range(0, len(x), 37):
        a = np.sort(inv[ids[o[p[k]]:o[p[k] + 1]]])
        assert np.array_equal(a, ids4[o4[k]:o4[k + 1]])


def test_rectangular_lattice_in_an_anisotropic_periodic_box(oracle_mod):
    """A rectangular lattice (spacings 1/4, 2/4, 3/4 in a 1 x 2 x 3 periodic box): every cell is the
    rectangular box of the spacings, with its six facets at half spacings, and the cells tile the box."""
    lo, hi = np.zeros(3), np.array([1.0, 2.0, 3.0])
    n = 4
    a = hi / n
    g = [(np.arange(n) + 0.5) * a[c] for c in range(3)]
    x = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    x = x + inputs.rng(3).uniform(-1e-9, 1e-9, x.shape)  # general position
    r = oracle_mod.cells(x, lo, hi, True, mode="brute")
    assert abs(r["vol"].sum() - 6.0) < 1e-12
    assert np.allclose(r["vol"], np.prod(a), rtol=1e-7)
    off = r["face_off"]
    big = r["f_area"] > 1e-6 * a.min() ** 2
    # the six large facets of each cell: areas a_y a_z, a_x a_z, a_x a_y (two each) at half spacings
    for k in range(0, len(x), 7):
        sel = np.nonzero(big[off[k]:off[k + 1]])[0] + off[k]
        assert len(sel) == 6
        areas = np.sort(r["f_area"][sel])
        want = np.sort(np.repeat([a[1] * a[2], a[0] * a[2], a[0] * a[1]], 2))
        assert np.allclose(areas, want, rtol=1e-6)
        assert np.allclose(np.sort(r["f_dist"][sel]), np.sort(np.repeat(a / 2, 2)), rtol=1e-6)
    rc = oracle_mod.cells(x, lo, hi, True, mode="certified")
    assert np.abs(rc["vol"] - r["vol"]).max() < 1e-15


def test_cell_moments_closed_forms(oracle_mod):
    """Cell centroid and second moment (integral of |y - x_i|^2) against closed forms: the cubes of the SC
    lattice (centroid at the site, a^5 / 4), a one-point bounded box (the whole box) and two points split
    by their bisector (two half boxes)."""
    n = 8
    a = 1.0 / n
    x = inputs.sc_lattice(n)
    which = np.arange(0, n ** 3, 37)
    r = oracle_mod.cells(x, 0.0, 1.0, True, which=which, mode="brute")
    assert np.allclose(r["cen"], x[which], rtol=0, atol=1e-15)
    assert np.allclose(r["mom2"], a ** 5 / 4, rtol=1e-12, atol=0)

    def box_moments(lo, hi, p):
        lo, hi, p = map(np.asarray, (lo, hi, p))
        V = np.prod(hi - lo)
        c = 0.5 * (lo + hi)
        return V, c, V * np.sum((hi - lo) ** 2 / 12.0 + (c - p) ** 2)

    lo, hi, p = [1.0, 2.0, 4.0], [3.5, 3.25, 5.0], [2.0, 3.0, 4.5]
    r = oracle_mod.cells(np.array([p]), lo, hi, False, mode="brute")
    V, c, m2 = box_moments(lo, hi, p)
    assert abs(r["vol"][0] - V) < 1e-14 and np.allclose(r["cen"][0], c, atol=1e-14)
    assert abs(r["mom2"][0] - m2) < 1e-13 * m2
    pts = np.array([[0.2, 0.3, 0.6], [0.8, 0.3, 0.6]])  # bisector x = 0.5
    r = oracle_mod.cells(pts, 0.0, 1.0, False, mode="brute")
    for k, (l0, h0) in enumerate(((0.0, 0.5), (0.5, 1.0))):
        V, c, m2 = box_moments([l0, 0.0, 0.0], [h0, 1.0, 1.0], pts[k])
        assert abs(r["vol"][k] - V) < 1e-15 and np.allclose(r["cen"][k], c, atol=1e-15)
        assert abs(r["mom2"][k] - m2) < 1e-14


def test_bounded_box_total_volume(oracle_mod):
    pts, off = inputs.halo_sets(n_sets=3, nmin=64, nmax=400, seed=6, dtype=np.float32)
    for s in range(3):
        p = pts[off[s]:off[s + 1]].astype(np.float64)
        r = oracle_mod.cells(p, -1.0, 1.0, False, mode="certified")
        assert abs(r["vol"].sum() - 8.0) < 1e-11
        rb = oracle_mod.cells(p, -1.0, 1.0, False, mode="brute")
        assert np.abs(rb["vol"] - r["vol"]).max() < 1e-14
        assert (r["nvert"] - r["nedge"] + r["nface"] == 2).all()


def test_tiny_periodic_sets_multiple_images(oracle_mod):
    # N = 2: each cell touches the other particle through several images and
    # its own images; volumes still add up to the box
    x = np.array([[0.1, 0.2, 0.3], [0.6, 0.55, 0.9]])
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")
    assert abs(r["vol"].sum() - 1.0) < 1e-14
    o, ids = oracle_mod.neighbours(r)
    assert list(ids[o[0]:o[1]]) == [1] and list(ids[o[1]:o[2]]) == [0]
    # one point: the cell is the whole periodic cube with six self-image facets
    r1 = oracle_mod.cells(x[:1], 0.0, 1.0, True, mode="brute")
    assert abs(r1["vol"][0] - 1.0) < 1e-15 and r1["nface"][0] == 6
    o1, ids1 = oracle_mod.neighbours(r1)
    assert len(ids1) == 0


def test_duplicate_points_raise(oracle_mod):
    x = inputs.uniform(64, seed=1)
    x[5] = x[9]
    with pytest.raises(RuntimeError):
        oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")


# --------------------------------------------------------------------------
# exact predicate against rational arithmetic
# --------------------------------------------------------------------------
def _rational_side(xi, pa, pb, pc, pj):
    """Vertex of the three bisectors by Cramer's rule in exact rationals,
    then the sign of d_j.v - |d_j|^2/2."""
    F = [[Fraction(float(c)) for c in p] for p in (xi, pa, pb, pc, pj)]
    d = [[F[k][c] - F[0][c] for c in range(3)] for k in range(1, 5)]
    h = [sum(c * c for c in dk) / 2 for dk in d]
    N = d[:3]

    def det3(m):
        return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
                + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))

    D = det3(N)
    v = []
    for c in range(3):
        M = [list(row) for row in N]
        for r in range(3):
            M[r][c] = h[r]
        v.append(det3(M) / D)
    s = sum(d[3][c] * v[c] for c in range(3)) - h[3]
    return (s > 0) - (s < 0)


def test_exact_predicate_random(oracle_mod):
    g = np.random.default_rng(11)
    for _ in range(300):
        p = g.random((5, 3))
        want = _rational_side(*p)
        assert oracle_mod.insphere_side(*p) == want
        assert oracle_mod.insphere_side(*p, exact_only=True) == want


def test_exact_predicate_degenerate_and_near(oracle_mod):
    base = np.array([0.5, 0.25, 0.125])
    s = 2.0 ** -10
    xi = base
    pa = base + s * np.array([2.0, 0, 0])
    pb = base + s * np.array([0, 2.0, 0])
    pc = base + s * np.array([0, 0, 2.0])
    on = base + s * np.array([2.0, 2.0, 0])  # on the circumsphere centred at base + s(1,1,1)
    assert _rational_side(xi, pa, pb, pc, on) == 0
    assert oracle_mod.insphere_side(xi, pa, pb, pc, on) == 0
    # one ulp inwards / outwards along x
    inside = on.copy()
    inside[0] = np.nextafter(on[0], 0.0)
    outside = on.copy()
    outside[0] = np.nextafter(on[0], 1.0)
    for q in (inside, outside):
        want = _rational_side(xi, pa, pb, pc, q)
        assert want != 0
        assert oracle_mod.insphere_side(xi, pa, pb, pc, q) == want
        assert oracle_mod.insphere_side(xi, pa, pb, pc, q, exact_only=True) == want
    # generic points with FP64 full-mantissa coordinates near degeneracy
    g = np.random.default_rng(5)
    for _ in range(100):
        c = g.random(3)
        R = 0.1 + 0.1 * g.random()
        dirs = g.normal(size=(5, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        p = c + R * dirs  # nearly cospherical up to rounding
        want = _rational_side(*p)
        assert oracle_mod.insphere_side(*p) == want
        assert oracle_mod.insphere_side(*p, exact_only=True) == want


# --------------------------------------------------------------------------
# gradient, grid, adjoint
# --------------------------------------------------------------------------
def test_gradient_linear_field_exact(oracle_mod):
    x = inputs.uniform(1024, seed=2)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    off, ids, disp = oracle_mod.neighbour_displacements(r, x)
    g_true = np.array([0.3, -1.7, 2.5])
    # field values seen from each cell through the facet displacement
    fself = np.zeros(len(x))
    fall = np.zeros(len(x))
    grads = []
    for k in range(0, len(x), 17):
        a, b = off[k], off[k + 1]
        vals = 4.0 + disp[a:b] @ g_true  # rho_j - rho_i = g . d_ij exactly linear
        fall[:] = 0.0
        fall[ids[a:b]] = vals
        g = oracle_mod.gradient(np.array([4.0]), np.array([0, b - a]), np.arange(b - a), disp[a:b], vals)
        grads.append(g[0])
    assert np.allclose(np.array(grads), g_true[None, :], rtol=1e-10, atol=1e-10)


def test_gradient_lattice_zero(oracle_mod):
    x = inputs.bcc_lattice(6)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    dens = oracle_mod.density(np.ones(len(x)), r["vol"])
    off, ids, disp = oracle_mod.neighbour_displacements(r, x)
    g = oracle_mod.gradient(dens, off, ids, disp, dens)
    assert np.abs(g).max() < 1e-6 * dens.max()


def test_green_gauss_gradient_linear_field_exact(oracle_mod):
    """Closed form: on every cell that no box wall bounds, the Green-Gauss gradient of a linear field is the
    field's gradient; a constant field gives zero on every cell, walls included."""
    x = inputs.uniform(1500, seed=12)
    r = oracle_mod.cells(x, 0.0, 1.0, False, mode="certified")
    g_true = np.array([0.3, -1.7, 2.5])
    phi = 4.0 + x @ g_true
    g = oracle_mod.gradient_green_gauss(r, x, phi, phi, 0.0, 1.0)
    off = r["face_off"]
    interior = np.array([(r["f_nbr"][off[k]:off[k + 1]] >= 0).all() for k in range(len(x))])
    assert interior.sum() > 500
    assert np.abs(g[interior] - g_true[None, :]).max() < 1e-9
    # wall cells see rho_i on the wall: not exact, but the estimate stays of the field's size
    assert np.abs(g[~interior]).max() < 10 * np.abs(g_true).max()
    c = np.full(len(x), 3.0)
    assert np.abs(oracle_mod.gradient_green_gauss(r, x, c, c, 0.0, 1.0)).max() < 1e-12


def test_green_gauss_gradient_periodic_lattice_zero(oracle_mod):
    x = inputs.bcc_lattice(6)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    dens = oracle_mod.density(np.ones(len(x)), r["vol"])
    g = oracle_mod.gradient_green_gauss(r, x, dens, dens, 0.0, 1.0)
    assert np.abs(g).max() < 1e-6 * dens.max()


@pytest.mark.parametrize("periodic", [True, False])
def test_grid_volume_partition_of_unity(oracle_mod, periodic):
    """The cells tile every voxel: with unit densities every voxel average is 1."""
    x = inputs.uniform(500, seed=3)
    g = oracle_mod.grid_volume_density(x, np.ones(len(x)), 0.0, 1.0, 5, periodic=periodic)
    assert np.abs(g - 1.0).max() < 1e-12


def test_grid_volume_mass_and_single_voxel(oracle_mod):
    x = inputs.uniform(500, seed=3)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    d = np.random.default_rng(1).random(len(x))
    mass = (d * r["vol"]).sum()
    g = oracle_mod.grid_volume_density(x, d, 0.0, 1.0, 4)
    assert abs(g.sum() / 64 - mass) < 1e-12 * mass  # sum of averages x voxel volume = total mass
    g1 = oracle_mod.grid_volume_density(x, d, 0.0, 1.0, 1)
    assert abs(g1.ravel()[0] - mass) < 1e-12 * mass  # one voxel: the box


def test_grid_volume_lattice_cells_are_voxels(oracle_mod):
    """SC lattice with one site per voxel: each voxel is exactly one cell (its walls lie on the cell faces,
    a degenerate case for the exact predicates), so each voxel takes its site's density."""
    x = inputs.sc_lattice(4)
    d = np.arange(len(x), dtype=np.float64)
    g = oracle_mod.grid_volume_density(x, d, 0.0, 1.0, 4)
    a = np.floor(x * 4).astype(int)
    assert np.abs(g[a[:, 2], a[:, 1], a[:, 0]] - d).max() < 1e-12


def test_face_cubic_moment_of_a_cube(oracle_mod):
    """Closed form: a face of the cube of side a (SC lattice) at distance a/2 has
    integral |y|^2 y dA = (a/2)(a^4/4 + a^4/6) = 5 a^5 / 24 along its normal, zero across."""
    x = inputs.sc_lattice(4)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")
    a = 0.25
    n = (r["f_cen"][:6] - x[0]) / (a / 2)
    assert np.abs(r["f_m3"][:6] - 5 * a ** 5 / 24 * n).max() < 1e-12


def test_weighted_cvt_gradient_finite_differences(oracle_mod):
    """dE_w/dx against central differences of E_w = sum_i w_i E_i (the oracle's cell second moments)."""
    x = inputs.uniform(300, seed=5)
    w = np.random.default_rng(2).random(300) + 0.5
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    g = oracle_mod.cvt_weighted_gradient(r, x, w)

    def E(xx):
        return float((w * oracle_mod.cells(xx % 1.0, 0.0, 1.0, True, mode="certified")["mom2"]).sum())

    for k in (3, 77, 150):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[k, c] += 1e-5
            xm[k, c] -= 1e-5
            fd = (E(xp) - E(xm)) / 2e-5
            assert abs(fd - g[k, c]) <= 1e-6 * np.abs(g[k]).max(), (k, c, fd, g[k, c])
    # equal weights: the facet terms cancel and the gradient is the centroidal one, 2 w V (x - z)
    g1 = oracle_mod.cvt_weighted_gradient(r, x, np.full(300, 2.0))
    assert np.allclose(g1, 4.0 * r["vol"][:, None] * (x - r["cen"]), rtol=0, atol=1e-15)


def test_grid_nearest_matches_kdtree(oracle_mod):
    scipy_spatial = pytest.importorskip("scipy.spatial")
    x = inputs.uniform(300, seed=4)
    G, S = 8, 2
    idx = oracle_mod.grid_nearest(x, 0.0, 1.0, G, S, True)
    pts = np.array([oracle_mod.grid_point(0.0, 1.0, G, S, q // S ** 3, q % S ** 3) for q in range(G ** 3 * S ** 3)])
    t = scipy_spatial.cKDTree(x, boxsize=1.0)
    d, j = t.query(pts)
    assert np.array_equal(idx.reshape(-1), j)


def test_nearest_points_matches_grid_nearest_and_kdtree(oracle_mod):
    """The nearest-particle query for arbitrary points: on the grid's own sub-points it equals grid_nearest, and on
    random points (periodic and bounded) it equals a scipy k-d tree query."""
    scipy_spatial = pytest.importorskip("scipy.spatial")
    x = inputs.uniform(300, seed=4)
    G, S = 6, 1
    pts = np.array([oracle_mod.grid_point(0.0, 1.0, G, S, q, 0) for q in range(G ** 3)])
    assert np.array_equal(oracle_mod.nearest_points(x, pts, 0.0, 1.0, True),
                          oracle_mod.grid_nearest(x, 0.0, 1.0, G, S, True).reshape(-1))
    q = np.random.default_rng(2).random((500, 3))
    assert np.array_equal(oracle_mod.nearest_points(x, q, 0.0, 1.0, True),
                          scipy_spatial.cKDTree(x, boxsize=1.0).query(q)[1])
    assert np.array_equal(oracle_mod.nearest_points(x, q, 0.0, 1.0, False), scipy_spatial.cKDTree(x).query(q)[1])


def test_grid_density_lattice_constant(oracle_mod):
    x = inputs.sc_lattice(8, perturb=1e-9)
    r = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    dens = oracle_mod.density(np.ones(len(x)), r["vol"])
    grid = oracle_mod.grid_density(x, dens, 0.0, 1.0, 16, 2)
    assert np.allclose(grid, len(x), rtol=1e-6)


def _vols(oracle_mod, x):
    return oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")


def test_volume_adjoint_invariants_and_fd(oracle_mod):
    x = inputs.uniform(64, seed=7)
    r = _vols(oracle_mod, x)
    N = len(x)
    # sum_i dV_i/dx_k = 0 (total volume fixed)
    tot = oracle_mod.volume_adjoint(r, x, g_vol=np.ones(N))
    assert np.abs(tot).max() < 1e-12
    # central finite differences of V_i with respect to x_k
    h = 1e-6
    g = np.random.default_rng(0).random(N)
    ana = oracle_mod.volume_adjoint(r, x, g_vol=g)
    for k in (0, 5, 17):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (g @ _vols(oracle_mod, xp)["vol"] - g @ _vols(oracle_mod, xm)["vol"]) / (2 * h)
            assert abs(fd - ana[k, c]) < 1e-7 * max(1.0, abs(ana[k, c]))
    # translation invariance of each V_i: sum_k dV_i/dx_k = 0
    for i in (0, 3):
        e = np.zeros(N)
        e[i] = 1.0
        assert np.abs(oracle_mod.volume_adjoint(r, x, g_vol=e).sum(0)).max() < 1e-12


def test_cvt_energy_gradient_fd(oracle_mod):
    x = inputs.uniform(64, seed=8)
    r = _vols(oracle_mod, x)
    ana = oracle_mod.volume_adjoint(r, x, g_energy=1.0)
    h = 1e-6
    for k in (1, 9):
        for c in range(3):
            xp = x.copy()
            xm = x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (_vols(oracle_mod, xp)["mom2"].sum() - _vols(oracle_mod, xm)["mom2"].sum()) / (2 * h)
            assert abs(fd - ana[k, c]) < 1e-7
    # lattice: centroid = site, so the CVT gradient vanishes
    xl = inputs.bcc_lattice(3)
    rl = oracle_mod.cells(xl, 0.0, 1.0, True, mode="brute")
    assert np.abs(oracle_mod.volume_adjoint(rl, xl, g_energy=1.0)).max() < 1e-12
