"""Owned-cell builds (vt_build_owned), cell radii (vt_cell_radius) and the decomposed form with the library as the
engine of every rank.

* vt_build_owned over all the particles, with the first half owned: the owned rows equal a vt_build of the same
  points bit for bit (same sort, same kernel, same candidates), the other rows have volume 0 and no neighbours;
* the radius of every cell bounds the oracle's largest vertex distance from above, tightly;
* the decomposed form (ranks as threads of this process on the one GPU, each with its own buffer zone and owned
  build): the union of the ranks' cells against the FP64 oracle of the whole set, at the single-GPU tolerances.
  The ranks' kernels never wait on one another: every exchange happens on the host between launches.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1601_06429_gb300 import binding as vt
from paper_1601_06429_gb300 import inputs
from paper_1601_06429_gb300 import sharded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1601_06429_gb300.build import build

    build()
    vt.load_library()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _clustered(N=65536, seed=1):
    L = float(np.float32(100.0 * (N / 2097152) ** (1.0 / 3.0)))
    return inputs.clustered(N, L=L, seed=seed), L


@pytest.mark.parametrize("prec", ["filter32", "plain64"])
def test_owned_build_equals_full_build_on_owned_rows(prec):
    x, L = _clustered()
    pos = torch.from_numpy(x).cuda()
    N, n_own = len(x), len(x) // 2
    full = vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, prec)
    own = vt.vt_build_owned(pos, n_own, None, (0.0,) * 3, (L,) * 3, True, prec)
    fv, fo, fi = (t.cpu().numpy() for t in vt.cells(full))
    ov, oo, oi = (t.cpu().numpy() for t in vt.cells(own))
    assert np.array_equal(ov[:n_own], fv[:n_own]) and (ov[n_own:] == 0).all()
    assert (np.diff(oo)[n_own:] == 0).all()
    for i in range(0, n_own, 7):
        assert np.array_equal(oi[oo[i]:oo[i + 1]], fi[fo[i]:fo[i + 1]])
    assert np.array_equal(vt.cell_radius(own).cpu().numpy()[:n_own], vt.cell_radius(full).cpu().numpy()[:n_own])
    assert (vt.density(own).cpu().numpy()[n_own:] == 0).all()
    st = vt.vt_status(own)
    assert st["rc"] == 0 and st["n_faces"] == oo[-1]


def test_cell_radius_bounds_the_oracle(oracle_mod):
    x, L = _clustered(16384, seed=4)
    o = oracle_mod.cells(x.astype(np.float64), 0.0, L, True, mode="certified")
    for prec in ("filter32", "plain64"):
        h = vt.vt_build(torch.from_numpy(x).cuda(), None, (0.0,) * 3, (L,) * 3, True, prec)
        r = vt.cell_radius(h).double().cpu().numpy()
        assert (r >= o["rmax"]).all()
        assert (r <= o["rmax"] * (1 + 1e-3)).all(), (r / o["rmax"]).max()


def _run_threads(x, L, W, **kw):
    comms = sharded.ThreadComm.group(W)
    parts = [None] * W
    errs = []
    split = np.array_split(np.arange(len(x)), W)

    def work(r):
        try:
            torch.cuda.set_device(0)
            parts[r] = sharded.cells_sharded(comms[r], x[split[r]], split[r], 0.0, L, **kw)
        except Exception as e:  # noqa: BLE001 - reported below
            errs.append(e)
            comms[r].s.barrier.abort()

    th = [threading.Thread(target=work, args=(r,)) for r in range(W)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return parts


@pytest.mark.parametrize("W", [2, 4, 8])
def test_decomposed_cells_match_the_oracle(W, oracle_mod):
    x, L = _clustered()
    parts = _run_threads(x, L, W)
    x64 = x.astype(np.float64)
    o = oracle_mod.cells(x64, 0.0, L, True, mode="certified")
    ooff, oids = oracle_mod.neighbours(o)
    dens = 1.0 / o["vol"]
    noff, nids, disp = oracle_mod.neighbour_displacements(o, x64, 0.0, L)
    g_ref = oracle_mod.gradient(dens, noff, nids, disp, dens)
    seen = np.zeros(len(x), bool)
    for p in parts:
        g = p["gid"]
        assert not seen[g].any()
        seen[g] = True
        assert (np.abs(p["vol"] - o["vol"][g]) / o["vol"][g]).max() <= 2e-5
        assert (np.abs(p["dens"] - dens[g]) / dens[g]).max() <= 2e-5
        den = np.maximum(np.linalg.norm(g_ref[g], axis=1), 1e-3 * dens[g] / o["vol"][g] ** (1 / 3))
        assert (np.linalg.norm(p["grad"] - g_ref[g], axis=1) / den).max() <= 1e-4
        for k, i in enumerate(g):
            assert np.array_equal(p["ids"][p["off"][k]:p["off"][k + 1]], oids[ooff[i]:ooff[i + 1]])
    assert seen.all()
