"""Differentiation through the Voronoi cells (torch.autograd.Function over vt_backward) and Lloyd steps.

Workload: the 1,048,576-point halo (30 %) + uniform mixture in the unit periodic box, FP32 (the adjoint and
finite-difference checks on 256 random particles at full size, and the Lloyd steps), and a 32,768-point version
of the same recipe for the checks over every particle.
Checks:
  * dL/dx of L = sum_i w_i log(rho_i), w ~ U(0,1), against the oracle's analytic adjoint (all particles)
    and against central finite differences of the oracle's FP64 volumes (h = 1e-4 scaled by the local
    spacing, Richardson extrapolation over h and h/2) on random particles;
  * the energy gradient 2 V (x - z) through autograd against the oracle;
  * 50 Lloyd steps on the full set: the centroidal energy never increases; a BCC lattice is a fixed point.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1601_06429_gb300 import autograd as vta
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


@pytest.fixture(scope="module")
def mix32k(oracle_mod):
    x = inputs.halo_uniform_mix(32768, L=1.0, seed=3)
    o = oracle_mod.cells(x.astype(np.float64), 0.0, 1.0, True, mode="certified")
    w = inputs.rng(4).random(len(x))
    return x, o, w


def _gpu_grad(x, w, precision):
    pos = torch.from_numpy(x).cuda().requires_grad_(True)
    vol, energy = vta.cells(pos, (0.0,) * 3, (1.0,) * 3, True, precision)
    wt = torch.from_numpy(w).to(device=pos.device, dtype=pos.dtype)
    loss = (wt * torch.log(1.0 / vol)).sum()  # unit masses: rho = 1 / V
    loss.backward()
    return pos.grad.double().cpu().numpy(), vol.double().detach().cpu().numpy()


def test_log_density_loss_matches_oracle_adjoint(mix32k, oracle_mod):
    x, o, w = mix32k
    g, vol = _gpu_grad(x, w, "filter32")
    ref = oracle_mod.volume_adjoint(o, x.astype(np.float64), g_vol=-w / o["vol"])
    scale = np.linalg.norm(ref, axis=1)
    err = np.linalg.norm(g - ref, axis=1)
    # FP32 facet data: relative 1e-4 of each particle's gradient, with a floor at 1e-5 of the largest
    assert (err <= 1e-4 * scale + 1e-5 * scale.max()).all(), (err / np.maximum(scale, 1e-30)).max()


def test_finite_differences_on_random_particles(mix32k, oracle_mod):
    x, o, w = mix32k
    x64 = x.astype(np.float64)
    g, _ = _gpu_grad(x, w, "filter32")
    noff, nids = oracle_mod.neighbours(o)
    ell = o["vol"] ** (1.0 / 3.0)
    rng = np.random.default_rng(5)
    pick = rng.choice(len(x), 16, replace=False)

    def loss_local(xp, cells):
        r = oracle_mod.cells(xp, 0.0, 1.0, True, which=cells, mode="certified")
        return float(np.sum(w[cells] * -np.log(r["vol"])))

    for k in pick:
        cells = np.unique(np.concatenate([[k], nids[noff[k]:noff[k + 1]]])).astype(np.int64)
        h0 = 1e-4 * min(1.0, ell[k] / ell.mean())
        for c in range(3):
            def fd(h):
                xp = x64.copy()
                xm = x64.copy()
                xp[k, c] += h
                xm[k, c] -= h
                return (loss_local(xp % 1.0, cells) - loss_local(xm % 1.0, cells)) / (2 * h)
            d1, d2 = fd(h0), fd(h0 / 2)
            rich = (4 * d2 - d1) / 3
            assert abs(rich - g[k, c]) <= 1e-3 * max(abs(rich), 1e-3 * np.abs(g[k]).max() + 1e-12), (k, c, rich, g[k, c])


def test_energy_gradient_matches_oracle(mix32k, oracle_mod):
    x, o, _ = mix32k
    pos = torch.from_numpy(x).cuda().requires_grad_(True)
    vol, energy = vta.cells(pos, (0.0,) * 3, (1.0,) * 3, True, "filter32")
    energy.sum().backward()
    g = pos.grad.double().cpu().numpy()
    ref = oracle_mod.volume_adjoint(o, x.astype(np.float64), g_energy=1.0)
    scale = np.linalg.norm(ref, axis=1)
    assert (np.linalg.norm(g - ref, axis=1) <= 1e-3 * scale + 1e-5 * scale.max()).all()
    e = energy.double().detach().cpu().numpy()
    assert np.allclose(e, o["mom2"], rtol=1e-4, atol=1e-6 * np.abs(o["mom2"]).max())


def test_lloyd_50_steps_energy_decreases():
    x = torch.from_numpy(inputs.halo_uniform_mix(1048576, L=1.0, seed=3)).cuda()
    energies = []
    for _ in range(50):
        x, E = vta.lloyd_step(x, (0.0,) * 3, (1.0,) * 3)
        energies.append(E)
    e = np.array(energies)
    assert (np.diff(e) <= 1e-5 * e[:-1]).all(), np.diff(e).max()
    assert e[-1] < 0.9 * e[0]


def test_lattice_is_a_lloyd_fixed_point():
    x = torch.from_numpy(inputs.bcc_lattice(16, dtype=np.float32)).cuda().requires_grad_(True)
    vol, energy = vta.cells(x, (0.0,) * 3, (1.0,) * 3, True, "filter32")
    energy.sum().backward()
    step = x.grad / (2.0 * vol[:, None].detach())
    assert float(step.abs().max()) < 1e-5 * (1.0 / 16)


def test_weighted_cvt_gradient_matches_oracle(oracle_mod):
    """dE_w/dx for E_w = sum_i w_i E_i (per-cell weights) against the oracle, on 4096 uniform points (FP64 path),
    and with equal weights against vt_backward's centroidal-energy term."""
    x = inputs.uniform(4096, seed=0)
    o = oracle_mod.cells(x, 0.0, 1.0, True, mode="certified")
    w = np.random.default_rng(9).random(len(x)) + 0.5
    ref = oracle_mod.cvt_weighted_gradient(o, x, w)
    h = vt.vt_build(torch.from_numpy(x).cuda(), None, (0.0,) * 3, (1.0,) * 3, True, "plain64")
    got = vt.backward_weighted(h, torch.from_numpy(w)).cpu().numpy()
    assert vt.vt_status(h)["n_grid_failed"] == 0
    scale = np.linalg.norm(ref, axis=1)
    assert (np.linalg.norm(got - ref, axis=1) <= 1e-4 * scale + 1e-5 * scale.max()).all()
    eq = vt.backward_weighted(h, torch.full((len(x),), 0.7, dtype=torch.float64)).cpu().numpy()
    ref_eq = vt.backward(h, torch.zeros(len(x), dtype=torch.float64), 0.7).cpu().numpy()
    assert np.abs(eq - ref_eq).max() <= 1e-6 * np.abs(ref_eq).max()


def test_lloyd_runner_matches_autograd_steps_and_graph_replay():
    """LloydRunner (vt_rebuild in one handle; optionally one CUDA graph per step) against lloyd_step through
    autograd, and the graph replay against the eager runner bit for bit."""
    x0 = torch.from_numpy(inputs.halo_uniform_mix(262144, L=1.0, seed=3)).cuda()
    ref, E0 = vta.lloyd_step(x0, (0.0,) * 3, (1.0,) * 3)
    r = vta.LloydRunner(x0)
    # the constructor already took one step (outside any capture)
    d = torch.remainder(r.x - ref + 0.5, 1.0) - 0.5
    assert float(d.abs().max()) < 1e-5
    eager = vta.LloydRunner(x0)
    graph = vta.LloydRunner(x0, graph=True)  # capturing records the step without running it
    energies = []
    for _ in range(10):
        e1 = float(eager.step())
        e2 = float(graph.step())
        energies.append(e1)
        assert e1 == e2
        assert torch.equal(eager.x, graph.x)
    assert graph.status()["rc"] == 0
    e = np.array(energies)
    assert (np.diff(e) <= 1e-5 * e[:-1]).all()


def _local_extract(x64, k, rad):
    """The points within `rad` (minimum periodic image) of particle k in the unit box, in a frame centred on x_k
    (no wrap), with their indices; particle k is row 0."""
    d = x64 - x64[k]
    d -= np.round(d)
    sel = np.nonzero((d * d).sum(1) < rad * rad)[0]
    sel = np.concatenate([[k], sel[sel != k]])
    return d[sel], sel


def test_log_density_adjoint_full_size_config(oracle_mod):
    """The 1,048,576-point halo (30 %) + uniform set at full size: dL/dx of L = sum_i w_i log(rho_i) (w ~ U(0,1),
    seed 4) through autograd against the oracle's analytic adjoint on 256 random particles (seed 5), and against
    central finite differences of the oracle's FP64 volumes with Richardson extrapolation (h_k = 1e-4
    min(1, l_k / mean l), then h_k / 2; divided by 4 while a facet appears or vanishes within the step, where the
    loss is not smooth).  A cell depends only on the points within twice its largest vertex
    distance of its site, so each difference is taken on the points near x_k, in a bounded box around them that
    no cell of interest reaches; the unperturbed extract reproduces the global oracle's volumes first."""
    N = 1048576
    x = inputs.halo_uniform_mix(N, L=1.0, seed=3)
    w = inputs.rng(4).random(N)
    g, vol = _gpu_grad(x, w, "filter32")
    h = vt.vt_build(torch.from_numpy(x).cuda(), None, (0.0,) * 3, (1.0,) * 3, True, "filter32")
    _, noff_g, ids_g = vt.cells(h)
    noff_g, ids_g = noff_g.cpu().numpy(), ids_g.cpu().numpy()
    pick = np.sort(np.random.default_rng(5).choice(N, 256, replace=False))
    x64 = x.astype(np.float64)
    tree = oracle_mod.Tree(x64, 0.0, 1.0, True)
    S = np.unique(np.concatenate([pick] + [ids_g[noff_g[k]:noff_g[k + 1]] for k in pick]))
    o = tree.cells(S)
    pos_in_S = {int(i): n for n, i in enumerate(S)}
    ooff, oids = oracle_mod.neighbours(o)
    for k in pick:
        n = pos_in_S[int(k)]
        assert np.array_equal(ids_g[noff_g[k]:noff_g[k + 1]], oids[ooff[n]:ooff[n + 1]]), k
    # analytic adjoint: every term of dL/dx_k comes from the cells of k and its neighbours, all in S
    gV = np.zeros(N)
    gV[S] = -w[S] / o["vol"]
    ref = oracle_mod.volume_adjoint(o, x64, g_vol=gV)[pick]
    scale = np.linalg.norm(ref, axis=1)
    err = np.linalg.norm(g[pick] - ref, axis=1)
    assert (err <= 1e-4 * scale + 1e-5 * scale.max()).all(), (err / scale).max()
    # finite differences on local extracts
    ell = vol ** (1.0 / 3.0)
    rmax = dict(zip(S.tolist(), o["rmax"]))
    vS = dict(zip(S.tolist(), o["vol"]))
    for k in pick:
        cells_k = np.unique(np.concatenate([[k], ids_g[noff_g[k]:noff_g[k + 1]]]))
        dist = np.linalg.norm((x64[cells_k] - x64[k]) - np.round(x64[cells_k] - x64[k]), axis=1)
        reach = max(dist[q] + rmax[int(j)] for q, j in enumerate(cells_k))
        rad = max(dist[q] + 2.0 * rmax[int(j)] for q, j in enumerate(cells_k)) * 1.05 + 1e-3 * ell[k]
        loc, sel = _local_extract(x64, k, rad)
        B = 1.5 * max(rad, reach)
        order = np.argsort(sel[1:])
        idx = np.array([0 if j == k else 1 + order[np.searchsorted(sel[1:][order], j)] for j in cells_k])
        assert (sel[idx] == cells_k).all()
        r0 = oracle_mod.cells(loc, -B, B, False, which=idx, mode="certified")
        assert np.allclose(r0["vol"], [vS[int(j)] for j in cells_k], rtol=1e-12, atol=0), k
        wk = w[cells_k]

        def loss_local(dk):
            lp = loc.copy()
            lp[0] += dk
            r = oracle_mod.cells(lp, -B, B, False, which=idx, mode="certified")
            return float(np.sum(wk * -np.log(r["vol"]))), tuple(r["nface"])

        same = loss_local(np.zeros(3))[1]
        h0 = 1e-4 * min(1.0, ell[k] / ell.mean())
        for c in range(3):
            e = np.zeros(3)
            e[c] = 1.0

            def fd(hh):
                (lp, sp), (lm, sm) = loss_local(hh * e), loss_local(-hh * e)
                return (lp - lm) / (2 * hh), sp == same and sm == same

            # the loss is smooth only while no facet of these cells appears or vanishes: where one does within
            # the step, the step is divided by 4 until the facet counts at +-h equal the unperturbed ones
            hh = h0
            for _ in range(8):
                (d1, s1), (d2, s2) = fd(hh), fd(hh / 2)
                if s1 and s2:
                    break
                hh /= 4
            assert s1 and s2, (k, c)
            rich = (4 * d2 - d1) / 3
            assert abs(rich - g[k, c]) <= 1e-3 * max(abs(rich), 1e-3 * np.abs(g[k]).max() + 1e-12), (k, c, rich,
                                                                                                        g[k, c])
    tree.close()
