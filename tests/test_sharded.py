"""The decomposed (multi-rank) form of the cells on CPU: bricks, buffer zones, certificate, re-indexing.

The ranks run as threads of this process (ThreadComm) and as two gloo processes (DistComm over
torch.distributed).  The cell engine of each rank is the FP64 oracle (certified mode on the rank's particles and
buffer; test infrastructure only), so the union of the ranks' owned cells must equal the oracle's cells of the
whole periodic set: volumes, densities and least-squares gradients to FP64 rounding, neighbour lists (global ids)
exactly.  The library's own engine is exercised the same way on a GPU (test_gpu_sharded.py).
"""
import os
import socket
import threading

import numpy as np
import pytest

from paper_1601_06429_gb300 import inputs
from paper_1601_06429_gb300 import sharded


def oracle_engine(pos, n_cells, lo, hi):
    """Cells of rows [0, n_cells) of a rank's particles with the oracle, in the engine's output form."""
    import oracle

    x = np.asarray(pos, np.float64)
    t = oracle.Tree(x, lo, hi, True)
    o = t.cells(np.arange(n_cells))
    t.close()
    off, ids = oracle.neighbours(o)
    dens = 1.0 / o["vol"]
    dens_all = np.zeros(len(x))
    dens_all[:n_cells] = dens
    noff, nids, disp = oracle.neighbour_displacements(o, x, lo, hi)
    grad = np.zeros((n_cells, 3))
    # the gradient of a cell whose neighbours all have cells (the owned ones, by the certificate)
    done = np.array([(nids[noff[k]:noff[k + 1]] < n_cells).all() for k in range(n_cells)])
    if done.any():
        sel = np.nonzero(done)[0]
        sub_off = np.concatenate([[0], np.cumsum(np.diff(noff)[sel])])
        sub_ids = np.concatenate([nids[noff[k]:noff[k + 1]] for k in sel])
        sub_disp = np.concatenate([disp[noff[k]:noff[k + 1]] for k in sel])
        grad[sel] = oracle.gradient(dens[sel], sub_off, sub_ids, sub_disp, dens_all)
    return dict(vol=o["vol"], dens=dens, grad=grad, rad=o["rmax"], off=off, ids=ids)


def reference(x, L):
    import oracle

    o = oracle.cells(x.astype(np.float64), 0.0, L, True, mode="certified")
    off, ids = oracle.neighbours(o)
    dens = 1.0 / o["vol"]
    noff, nids, disp = oracle.neighbour_displacements(o, x.astype(np.float64), 0.0, L)
    return dict(vol=o["vol"], dens=dens, grad=oracle.gradient(dens, noff, nids, disp, dens), off=off, ids=ids)


def check_union(parts, ref, N):
    seen = np.zeros(N, bool)
    for p in parts:
        g = p["gid"]
        assert not seen[g].any(), "a particle owned twice"
        seen[g] = True
        assert np.allclose(p["vol"], ref["vol"][g], rtol=1e-12, atol=0)
        assert np.allclose(p["dens"], ref["dens"][g], rtol=1e-12, atol=0)
        scale = np.maximum(np.linalg.norm(ref["grad"][g], axis=1), 1e-3 * ref["dens"][g] / ref["vol"][g] ** (1 / 3))
        assert (np.linalg.norm(p["grad"] - ref["grad"][g], axis=1) / scale).max() < 1e-9
        for k, i in enumerate(g):
            assert np.array_equal(p["ids"][p["off"][k]:p["off"][k + 1]], ref["ids"][ref["off"][i]:ref["off"][i + 1]])
    assert seen.all(), "a particle owned by no rank"


def run_threads(x, L, W, **kw):
    comms = sharded.ThreadComm.group(W)
    parts = [None] * W
    errs = []
    split = np.array_split(np.random.default_rng(0).permutation(len(x)), W)  # any input split

    def work(r):
        try:
            parts[r] = sharded.cells_sharded(comms[r], x[split[r]], split[r], 0.0, L, engine=oracle_engine, **kw)
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


def test_brick_grid_and_gaps():
    assert sharded.brick_grid(1) == (1, 1, 1) and sharded.brick_grid(2) == (2, 1, 1)
    assert sharded.brick_grid(8) == (2, 2, 2) and sharded.brick_grid(32) == (4, 4, 2)  # the paper's example
    assert sharded.brick_grid(6) == (6, 1, 1)  # not a power of two: slabs
    lo, L = np.zeros(3), np.ones(3)
    blo, bhi = sharded.brick_bounds(1, (2, 1, 1), lo, L)
    assert np.allclose(blo, [0.5, 0, 0]) and np.allclose(bhi, [1, 1, 1])
    pts = np.array([[0.7, 0.2, 0.2], [0.45, 0.5, 0.5], [0.02, 0.5, 0.5]])
    g = sharded.gap_to_brick(pts, blo, bhi, L)
    assert np.allclose(g, [0.0, 0.05, 0.02])  # the last one across the periodic boundary
    assert np.array_equal(sharded.brick_of(pts, (2, 1, 1), lo, L), [1, 0, 0])


@pytest.mark.parametrize("W", [2, 8])
def test_threads_union_equals_whole_set(W):
    x = inputs.uniform(1200, seed=21)
    parts = run_threads(x, 1.0, W)
    check_union(parts, reference(x, 1.0), len(x))


def test_clustered_set_and_buffer_doubling():
    """Clustered points, and a first buffer far too thin (a tenth of the spacing): the certificate fails and the
    buffer doubles until every computed cell is certified; the result is still the exact tessellation."""
    L = float(np.float32(16.0))
    x = inputs.clustered(1500, L=L, seed=3)
    parts = run_threads(x, L, 4, border_factor=0.1)
    assert parts[0]["rounds"] > 1 and all(p["t1"] == parts[0]["t1"] for p in parts)
    check_union(parts, reference(x, L), len(x))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, out_dir):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x = inputs.uniform(1000, seed=22)
        mine = np.arange(rank, len(x), world)
        p = sharded.cells_sharded(sharded.DistComm(), x[mine], mine, 0.0, 1.0, engine=oracle_engine)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), **{k: v for k, v in p.items()})
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    parts = []
    for r in range(2):
        d = np.load(tmp_path / ("rank%d.npz" % r))
        parts.append({k: d[k] for k in d.files})
    x = inputs.uniform(1000, seed=22)
    check_union(parts, reference(x, 1.0), len(x))
