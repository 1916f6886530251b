"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (per particle, max over the compared particles):
  * neighbour lists: identical sets (both sides decide every facet with
    error-bounded predicates and an exact fallback, so the comparison is exact);
  * volume and density: |d|/|ref| <= 1e-6 on the FP64 path, <= 2e-5 on the
    FP32-filtered path;
  * gradient: ||dg|| / max(||g_ref||, 1e-3 rho_i / l_i) <= 1e-4 on both paths
    (l_i = V_i^(1/3));
  * grid: the nearest particle is decided in FP64 with the same evaluation
    order on both sides, so grid values are compared exactly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1601_06429_gb300 import binding as vt
from paper_1601_06429_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_06429_gb300.build import build

    build()
    vt.load_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def gpu_run(x, lo, hi, periodic=True, precision="plain64", mass=None, grid=None, **kw):
    pos = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    m = None if mass is None else torch.from_numpy(np.ascontiguousarray(mass)).cuda()
    h = vt.vt_build(pos, m, (lo,) * 3, (hi,) * 3, periodic, precision, **kw)
    vol, off, ids = vt.cells(h)
    dens = vt.density(h)
    grad = vt.gradient(h)
    out = dict(h=h, vol=vol.cpu().numpy().astype(np.float64), off=off.cpu().numpy(), ids=ids.cpu().numpy(),
               dens=dens.cpu().numpy().astype(np.float64), grad=grad.cpu().numpy().astype(np.float64))
    if grid is not None:
        out["grid"] = vt.grid_density(h, grid[0], grid[1]).cpu().numpy().astype(np.float64)
    out["stats"] = vt.vt_status(h)
    return out


def check_cells(g, o, oracle_mod, which, vol_tol):
    """Volumes and densities (unit masses) of the cells `which` per particle, and their neighbour lists exactly."""
    ooff, oids = oracle_mod.neighbours(o)
    vr = np.abs(g["vol"][which] - o["vol"]) / o["vol"]
    assert vr.max() <= vol_tol, "volume rel err %g" % vr.max()
    dr = np.abs(g["dens"][which] - 1.0 / o["vol"]) * o["vol"]
    assert dr.max() <= vol_tol, "density rel err %g" % dr.max()
    bad = 0
    for k, i in enumerate(which):
        a = g["ids"][g["off"][i]:g["off"][i + 1]]
        b = oids[ooff[k]:ooff[k + 1]]
        if not np.array_equal(a, b):
            bad += 1
    assert bad == 0, "%d cells with neighbour lists different from the oracle" % bad


def check_gradient(g, x, o, oracle_mod, which, lo, hi, floor, tol):
    dens_o = oracle_mod.density(np.ones(len(which)), o["vol"])
    noff, nids, disp = oracle_mod.neighbour_displacements(o, x.astype(np.float64), lo, hi)
    # the oracle gradient needs rho_j of every neighbour: take the GPU-independent oracle volumes
    assert len(which) == len(x)
    g_ref = oracle_mod.gradient(dens_o, noff, nids, disp, dens_o)
    ell = o["vol"] ** (1.0 / 3.0)
    den = np.maximum(np.linalg.norm(g_ref, axis=1), floor * dens_o / ell)
    err = np.linalg.norm(g["grad"] - g_ref, axis=1) / den
    assert err.max() <= tol, "gradient err %g" % err.max()


# ---------------------------------------------------------------- small uniform (4096, FP64)
@pytest.fixture(scope="module")
def uniform4096(oracle_mod):
    x = inputs.uniform(4096, seed=0)
    return x, oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")


def test_uniform4096_plain64_all_outputs(uniform4096, oracle_mod):
    x, o = uniform4096
    g = gpu_run(x, 0.0, 1.0, True, "plain64", grid=(32, 1))
    which = np.arange(len(x))
    check_cells(g, o, oracle_mod, which, 1e-6)
    assert np.abs(g["dens"] - 1.0 / o["vol"]).max() <= 1e-6 * (1.0 / o["vol"]).max()
    check_gradient(g, x, o, oracle_mod, which, 0.0, 1.0, 1e-3, 1e-4)
    ref_grid = oracle_mod.grid_density(x, 1.0 / o["vol"], 0.0, 1.0, 32, 1)
    assert np.abs(g["grid"] - ref_grid).max() <= 1e-6 * ref_grid.max()
    assert g["stats"]["rc"] == 0 and g["stats"]["n_faces"] == len(g["ids"])


def test_uniform4096_filter32(uniform4096, oracle_mod):
    x, o = uniform4096
    g = gpu_run(x, 0.0, 1.0, True, "filter32")
    check_cells(g, o, oracle_mod, np.arange(len(x)), 2e-5)
    assert abs(g["vol"].sum() - 1.0) < 1e-6


@pytest.mark.parametrize("tpc", [1, 4, 8])
def test_uniform4096_thread_per_cell(uniform4096, oracle_mod, tpc):
    """The thread-per-cell and lane-group clipping kernels (cells they cannot finish go to the warp kernel) against
    the oracle."""
    x, o = uniform4096
    g = gpu_run(x, 0.0, 1.0, True, "filter32", threads_per_cell=tpc)
    check_cells(g, o, oracle_mod, np.arange(len(x)), 2e-5)
    assert abs(g["vol"].sum() - 1.0) < 1e-6
    check_gradient(g, x, o, oracle_mod, np.arange(len(x)), 0.0, 1.0, 1e-3, 1e-4)
    # it finishes nearly every cell of a uniform set itself
    assert g["stats"]["n_handed_over"] <= 0.05 * len(x), g["stats"]["n_handed_over"]


def test_uniform_fp32_inputs_both_precisions(oracle_mod):
    x = inputs.uniform(4096 + 7, seed=5, dtype=np.float32)  # ragged last bucket
    o = oracle_mod.cells(x.astype(np.float64), 0.0, 1.0, True, mode="certified")
    for prec, tol in (("plain64", 1e-6), ("filter32", 2e-5)):
        g = gpu_run(x, 0.0, 1.0, True, prec)
        check_cells(g, o, oracle_mod, np.arange(len(x)), tol)


@pytest.mark.parametrize("prec,tol", [("plain64", 1e-6), ("filter32", 2e-5)])
def test_anisotropic_periodic_box(oracle_mod, prec, tol):
    """A periodic box of sides 1 x 2 x 3 (every length handled per axis): 6000 uniform points against the oracle,
    all outputs but the grid."""
    lo, hi = np.zeros(3), np.array([1.0, 2.0, 3.0])
    x = inputs.uniform(6000, seed=17) * hi
    o = oracle_mod.cells(x, lo, hi, True, mode="certified")
    pos = torch.from_numpy(x).cuda()
    h = vt.vt_build(pos, None, tuple(lo), tuple(hi), True, prec)
    vol, off, ids = vt.cells(h)
    g = dict(vol=vol.cpu().numpy(), off=off.cpu().numpy(), ids=ids.cpu().numpy(),
             dens=vt.density(h).cpu().numpy(), grad=vt.gradient(h).cpu().numpy())
    check_cells(g, o, oracle_mod, np.arange(len(x)), tol)
    assert abs(g["vol"].sum() / 6.0 - 1.0) < (1e-9 if prec == "plain64" else 1e-6)
    check_gradient(g, x, o, oracle_mod, np.arange(len(x)), lo, hi, 1e-3, 1e-4)


# ---------------------------------------------------------------- lattices
@pytest.mark.parametrize("kind", ["sc", "bcc"])
def test_perturbed_lattices(kind, oracle_mod):
    x = inputs.sc_lattice(16, perturb=1e-9, seed=0) if kind == "sc" else inputs.bcc_lattice(8, perturb=1e-9, seed=0)
    o = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    g = gpu_run(x, 0.0, 1.0, True, "plain64", grid=(32, 1))
    which = np.arange(len(x))
    check_cells(g, o, oracle_mod, which, 1e-6)
    check_gradient(g, x, o, oracle_mod, which, 0.0, 1.0, 1e-3, 1e-4)
    ref_grid = oracle_mod.grid_density(x, 1.0 / o["vol"], 0.0, 1.0, 32, 1)
    assert np.abs(g["grid"] - ref_grid).max() <= 1e-6 * ref_grid.max()


def test_unperturbed_sc_lattice_exact_path(oracle_mod):
    x = inputs.sc_lattice(16)
    o = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    g = gpu_run(x, 0.0, 1.0, True, "plain64")
    check_cells(g, o, oracle_mod, np.arange(len(x)), 1e-9)
    assert g["stats"]["n_exact_cells"] > 0 and g["stats"]["n_exact_zero"] > 0
    assert (np.diff(g["off"]) == 6).all()


# ---------------------------------------------------------------- clustered, FP32
@pytest.fixture(scope="module")
def clustered64k(oracle_mod):
    N = 65536
    L = float(np.float32(100.0 * (N / 2097152) ** (1.0 / 3.0)))
    x = inputs.clustered(N, L=L, seed=1)
    return x, L, oracle_mod.cells(x.astype(np.float64), 0.0, L, True, mode="certified")


@pytest.mark.parametrize("prec,tol,tpc", [("filter32", 2e-5, 32), ("filter32", 2e-5, 1), ("filter32", 2e-5, 4),
                                          ("filter32", 2e-5, 8), ("plain64", 1e-6, 32)])
def test_clustered64k_all_cells(clustered64k, oracle_mod, prec, tol, tpc):
    x, L, o = clustered64k
    g = gpu_run(x, 0.0, L, True, prec, threads_per_cell=tpc)
    check_cells(g, o, oracle_mod, np.arange(len(x)), tol)
    assert abs(g["vol"].sum() / L ** 3 - 1.0) < 1e-6
    check_gradient(g, x, o, oracle_mod, np.arange(len(x)), 0.0, L, 1e-3, 1e-4)


# ---------------------------------------------------------------- Green-Gauss gradient
@pytest.mark.parametrize("prec,floor", [("plain64", 1e-3), ("filter32", 1e-3)])
def test_green_gauss_gradient_matches_oracle(uniform4096, oracle_mod, prec, floor):
    x, o = uniform4096
    h = vt.vt_build(torch.from_numpy(x).cuda(), None, (0.0,) * 3, (1.0,) * 3, True, prec)
    got = vt.gradient_gg(h).double().cpu().numpy()
    dens_o = 1.0 / o["vol"]
    ref = oracle_mod.gradient_green_gauss(o, x, dens_o, dens_o, 0.0, 1.0)
    ell = o["vol"] ** (1.0 / 3.0)
    den = np.maximum(np.linalg.norm(ref, axis=1), floor * dens_o / ell)
    assert (np.linalg.norm(got - ref, axis=1) / den).max() <= 1e-4


def test_green_gauss_gradient_of_a_linear_density(oracle_mod):
    """Masses chosen so that the density is a linear field (m_i = phi(x_i) V_i with the oracle's volumes): the
    GPU Green-Gauss gradient recovers the field's gradient on every cell no wall bounds."""
    x = inputs.uniform(3000, seed=13)
    o = oracle_mod.cells(x, 0.0, 1.0, False, mode="certified")
    g_true = np.array([0.3, -1.7, 2.5])
    m = (4.0 + x @ g_true) * o["vol"]
    h = vt.vt_build(torch.from_numpy(x).cuda(), torch.from_numpy(m).cuda(), (0.0,) * 3, (1.0,) * 3, False, "plain64")
    got = vt.gradient_gg(h).double().cpu().numpy()
    off = o["face_off"]
    interior = np.array([(o["f_nbr"][off[k]:off[k + 1]] >= 0).all() for k in range(len(x))])
    assert np.abs(got[interior] - g_true[None, :]).max() < 1e-3


# ---------------------------------------------------------------- volume-averaged grid
@pytest.mark.parametrize("prec", ["plain64", "filter32"])
def test_grid_volume_matches_oracle(uniform4096, oracle_mod, prec):
    x, o = uniform4096
    h = vt.vt_build(torch.from_numpy(x).cuda(), None, (0.0,) * 3, (1.0,) * 3, True, prec)
    got = vt.grid_density_volume(h, 16).double().cpu().numpy()
    assert vt.vt_status(h)["n_grid_failed"] == 0
    ref = oracle_mod.grid_volume_density(x, 1.0 / o["vol"], 0.0, 1.0, 16)
    assert np.abs(got - ref).max() <= 2e-5 * ref.max()


def test_grid_volume_partition_of_unity_and_bounded(oracle_mod):
    """Masses equal to the cell volumes make every density 1: every voxel average is then 1 (each voxel is
    tiled by the cell parts, none counted twice); and a bounded halo set against the oracle."""
    L = float(np.float32(31.5))
    x = inputs.clustered(65536, L=L, seed=1)
    pos = torch.from_numpy(x).cuda()
    h = vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, "filter32")
    vol, _, _ = vt.cells(h)
    h2 = vt.vt_build(pos, vol.clone(), (0.0,) * 3, (L,) * 3, True, "filter32")
    g = vt.grid_density_volume(h2, 32).double().cpu().numpy()
    assert vt.vt_status(h2)["n_grid_failed"] == 0
    assert np.abs(g - 1.0).max() < 2e-4
    pts, off = inputs.halo_sets(n_sets=1, nmin=3000, nmax=3001, seed=6)
    xb = pts[off[0]:off[1]].astype(np.float64)
    o = oracle_mod.cells(xb, -1.0, 1.0, False, mode="certified")
    hb = vt.vt_build(torch.from_numpy(xb).cuda(), None, (-1.0,) * 3, (1.0,) * 3, False, "plain64")
    got = vt.grid_density_volume(hb, 12).double().cpu().numpy()
    ref = oracle_mod.grid_volume_density(xb, 1.0 / o["vol"], -1.0, 1.0, 12, periodic=False)
    assert np.abs(got - ref).max() <= 1e-5 * ref.max()


# ---------------------------------------------------------------- bounded box
def test_bounded_halo_sets(oracle_mod):
    pts, off = inputs.halo_sets(n_sets=3, nmin=300, nmax=5000, seed=6, dtype=np.float32)
    for s in range(3):
        x = pts[off[s]:off[s + 1]]
        o = oracle_mod.cells(x.astype(np.float64), -1.0, 1.0, False, mode="certified")
        for prec, tol, tpc in (("filter32", 2e-5, 32), ("filter32", 2e-5, 1), ("filter32", 2e-5, 4),
                               ("filter32", 2e-5, 8), ("plain64", 1e-6, 32)):
            g = gpu_run(x, -1.0, 1.0, False, prec, threads_per_cell=tpc)
            check_cells(g, o, oracle_mod, np.arange(len(x)), tol)
            assert abs(g["vol"].sum() - 8.0) < 8e-6


# ---------------------------------------------------------------- backward
def test_backward_matches_oracle_adjoint(oracle_mod):
    x = inputs.uniform(512, seed=9)
    o = oracle_mod.cells(x, 0.0, 1.0, True, mode="brute")
    gV = np.random.default_rng(1).random(len(x))
    ref = oracle_mod.volume_adjoint(o, x, g_vol=gV, g_energy=0.7)
    pos = torch.from_numpy(x).cuda()
    h = vt.vt_build(pos, None, (0.0,) * 3, (1.0,) * 3, True, "plain64")
    got = vt.backward(h, torch.from_numpy(gV), 0.7).cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * scale


# ---------------------------------------------------------------- errors
def test_error_paths():
    x = inputs.uniform(1000, seed=2)
    xd = x.copy()
    xd[10] = xd[20]
    with pytest.raises(vt.VTError) as e:
        gpu_run(xd, 0.0, 1.0, True, "plain64")
    assert e.value.code == vt.VT_ERR_DUPLICATE
    xn = x.copy()
    xn[3, 1] = np.nan
    with pytest.raises(vt.VTError) as e:
        gpu_run(xn, 0.0, 1.0)
    assert e.value.code == vt.VT_ERR_INVALID
    xo = x.copy()
    xo[4, 2] = 1.0  # periodic boxes are half open
    with pytest.raises(vt.VTError) as e:
        gpu_run(xo, 0.0, 1.0)
    assert e.value.code == vt.VT_ERR_INVALID
    with pytest.raises(vt.VTError) as e:
        gpu_run(x[:2], 0.0, 1.0)
    assert e.value.code == vt.VT_ERR_UNSUPPORTED
    # a handle still works after failed builds
    g = gpu_run(x, 0.0, 1.0)
    assert abs(g["vol"].sum() - 1.0) < 1e-9


# ---------------------------------------------------------------- full-size configurations, sampled
@pytest.fixture(scope="module")
def clustered16M(oracle_mod):
    """The benchmark workload (16,777,216 clustered FP32 points, box 200, seed 2) and the oracle's k-d tree over all
    of it (certified mode), built once for the tests below."""
    x = inputs.clustered(16777216, L=200.0, seed=2)
    tree = oracle_mod.Tree(x.astype(np.float64), 0.0, 200.0, True)
    yield x, tree
    tree.close()


def check_sampled(g, x, L, tree, oracle_mod, which, grad_which, tol):
    """Volumes, densities and neighbour lists of the cells `which`, and the least-squares gradient of the cells
    `grad_which` (the oracle cells of all their neighbours give the rho_j), against the oracle on the kept tree."""
    o = tree.cells(which)
    check_cells(g, o, oracle_mod, which, tol)
    nb = np.unique(np.concatenate([g["ids"][g["off"][i]:g["off"][i + 1]] for i in grad_which] + [grad_which]))
    on = tree.cells(nb)
    dens_all = np.zeros(len(x))
    dens_all[nb] = 1.0 / on["vol"]
    og = tree.cells(grad_which)
    noff, nids, disp = oracle_mod.neighbour_displacements(og, x.astype(np.float64), 0.0, L)
    g_ref = oracle_mod.gradient(dens_all[grad_which], noff, nids, disp, dens_all)
    ell = og["vol"] ** (1.0 / 3.0)
    den = np.maximum(np.linalg.norm(g_ref, axis=1), 1e-3 * dens_all[grad_which] / ell)
    err = np.linalg.norm(g["grad"][grad_which] - g_ref, axis=1) / den
    assert err.max() <= 1e-4, "gradient err %g" % err.max()


def test_clustered_2M_subsample_and_grid(oracle_mod):
    """The 2,097,152-point clustered set (box 100, seed 1) with its 256^3 grid, FP32 filter: 16,384 sampled cells
    (seed 2), the exact kernel's cells and 512 FP64-decided ones against the oracle, gradients of 2048 of them;
    1024 random grid nodes (seed 3) take the density of the particle the oracle finds nearest to the node centre
    (brute force over all points), equal to the GPU's own density of that particle, and within 2e-5 of the
    oracle's density."""
    x = inputs.clustered(2097152, L=100.0, seed=1)
    L, G = 100.0, 256
    tree = oracle_mod.Tree(x.astype(np.float64), 0.0, L, True)
    g = gpu_run(x, 0.0, L, True, "filter32", grid=(G, 1))
    assert g["stats"]["device_error"] == 0
    N = len(x)
    assert abs(g["vol"].sum() / L ** 3 - 1.0) < 1e-6
    i = np.repeat(np.arange(N), np.diff(g["off"]))
    assert np.array_equal(np.sort(i.astype(np.int64) * N + g["ids"]), np.sort(g["ids"].astype(np.int64) * N + i))
    flags = vt.cell_flags(g["h"]).cpu().numpy()
    rng = np.random.default_rng(2)
    sub = np.sort(rng.choice(N, 16384, replace=False))
    fp64 = np.nonzero(flags & vt.VT_CELL_FP64)[0]
    which = np.unique(np.concatenate([sub, np.nonzero(flags & vt.VT_CELL_EXACT)[0],
                                      rng.choice(fp64, min(512, len(fp64)), replace=False)]))
    check_sampled(g, x, L, tree, oracle_mod, which, sub[::8], 2e-5)
    nodes = np.sort(np.random.default_rng(3).choice(G ** 3, 1024, replace=False))
    centres = np.array([oracle_mod.grid_point(0.0, L, G, 1, q, 0) for q in nodes])
    near = oracle_mod.nearest_points(x.astype(np.float64), centres, 0.0, L, True)
    grid = g["grid"].reshape(-1)[nodes]
    assert np.array_equal(grid, g["dens"][near])
    od = 1.0 / tree.cells(np.unique(near))["vol"]
    dref = od[np.searchsorted(np.unique(near), near)]
    assert (np.abs(grid - dref) / dref).max() <= 2e-5
    tree.close()


def test_clustered_16M_subsample_filter32(clustered16M, oracle_mod):
    """FP32 filter at full size: the 65,536-particle subsample (seed 2), every cell the exact kernel finished and
    1024 of the cells that needed FP64 decisions, against the oracle (volumes and densities to 2e-5, neighbour lists
    exactly); the least-squares gradient of all 65,536 (oracle cells of their ~1 M neighbours); total volume and
    neighbour symmetry over every particle."""
    x, tree = clustered16M
    g = gpu_run(x, 0.0, 200.0, True, "filter32")
    assert g["stats"]["device_error"] == 0
    N = len(x)
    assert abs(g["vol"].sum() / 200.0 ** 3 - 1.0) < 1e-6
    i = np.repeat(np.arange(N), np.diff(g["off"]))
    assert np.array_equal(np.sort(i.astype(np.int64) * N + g["ids"]), np.sort(g["ids"].astype(np.int64) * N + i))
    flags = vt.cell_flags(g["h"]).cpu().numpy()
    rng = np.random.default_rng(2)
    sub = np.sort(rng.choice(N, 65536, replace=False))
    exact = np.nonzero(flags & vt.VT_CELL_EXACT)[0]
    fp64 = np.nonzero(flags & vt.VT_CELL_FP64)[0]
    assert g["stats"]["n_exact_cells"] == len(exact) and len(fp64) > 0
    which = np.unique(np.concatenate([sub, exact, rng.choice(fp64, min(1024, len(fp64)), replace=False)]))
    check_sampled(g, x, 200.0, tree, oracle_mod, which, sub, 2e-5)


def test_clustered_16M_subsample_plain64(clustered16M, oracle_mod):
    """The plain FP64 path on the same workload: 8192 sampled cells (seed 8) plus the exact kernel's, volumes and
    densities to 1e-6 (the outputs are FP32 numbers, rounded once), neighbours exactly, gradients of 1024."""
    x, tree = clustered16M
    g = gpu_run(x, 0.0, 200.0, True, "plain64")
    assert g["stats"]["device_error"] == 0
    flags = vt.cell_flags(g["h"]).cpu().numpy()
    rng = np.random.default_rng(8)
    sub = np.sort(rng.choice(len(x), 8192, replace=False))
    which = np.unique(np.concatenate([sub, np.nonzero(flags & vt.VT_CELL_EXACT)[0]]))
    check_sampled(g, x, 200.0, tree, oracle_mod, which, sub[:1024], 1e-6)
