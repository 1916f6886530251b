"""Multi-GPU form of the per-particle cells: the paper's domain decomposition with buffer zones.

PARAVT (Implementation section) splits the box into sub-volumes, one per MPI task (equal-volume cuts by powers
of two, nx * ny * nz = number of tasks), gives each task the particles of its sub-volume plus the boundary
particles of a buffer zone (BORDERFACTOR times the mean inter-particle distance), lets every task tessellate on
its own, and gathers the outputs re-indexed to the real particle ids; AUTOBORDER thickens a buffer that is too
thin.  Here there is one rank per GPU and the tessellation of each rank runs in the library's kernels
(``vt_build_owned``):

1. route: every particle goes to the rank whose brick holds it (one all-to-all exchange);
2. buffer: every rank sends each other rank its particles within ``t2`` of that rank's brick (periodic
   distance), marked near (within ``t1``) or far -- one all-to-all exchange per mark;
3. local cells: ``vt_build_owned`` over the rows [owned, near, far] computes the cells of the owned and near
   particles; the near cells give the owned cells' neighbours their densities, so the density gradient needs no
   second exchange;
4. certificate (in place of the paper's warnings about a thin buffer): a computed cell is exact when every
   particle within twice its radius is held, i.e. ``gap(x_i, brick) + 2 R_i <= t2``, and the neighbours of an
   owned cell are all computed when ``2 R_i <= t1``; if a cell of any rank fails, every rank doubles ``t1``
   (``t2 = 2 t1``) and redoes steps 2-4 (AUTOBORDER, applied to the whole decomposition);
5. the outputs of the owned particles, with neighbour lists in global ids (ascending), stay on their rank.

The exchange goes through a small communicator interface: :class:`DistComm` (``torch.distributed``: NCCL between
GPUs, gloo on CPU) or :class:`ThreadComm` (ranks as threads of one process).  The cell engine is a callable, by
default :func:`gpu_engine`.  Only the orchestration (brick membership, buffer selection, certificate,
re-indexing) runs on the host, in numpy; no particle data passes through any other route.
"""
from __future__ import annotations

import threading

import numpy as np


# ---------------------------------------------------------------- decomposition
def brick_grid(world_size: int):
    """(nx, ny, nz) of the equal-volume decomposition: cuts by two on the axes in turn (x first) when the world
    size is a power of two (32 -> 4 x 4 x 2, the paper's example), else slabs along x."""
    W = int(world_size)
    if W < 1:
        raise ValueError("world size")
    if W & (W - 1):
        return (W, 1, 1)
    n = [1, 1, 1]
    a = 0
    while n[0] * n[1] * n[2] < W:
        n[a] *= 2
        a = (a + 1) % 3
    return tuple(n)


def brick_bounds(rank, grid, lo, L):
    """(lo, hi) of brick ``rank`` (x fastest), FP64 [3] each."""
    nx, ny, nz = grid
    idx = np.array([rank % nx, (rank // nx) % ny, rank // (nx * ny)], np.float64)
    n = np.array(grid, np.float64)
    blo = lo + idx * (L / n)
    bhi = lo + (idx + 1.0) * (L / n)
    return blo, bhi


def brick_of(pos, grid, lo, L):
    """Rank of the brick that holds each position ([N,3], inside the box)."""
    n = np.array(grid)
    c = np.floor((np.asarray(pos, np.float64) - lo) / (L / n)).astype(np.int64)
    c = np.clip(c, 0, n - 1)
    return c[:, 0] + n[0] * (c[:, 1] + n[1] * c[:, 2])


def gap_to_brick(pos, blo, bhi, L, periodic=True):
    """Distance from each position to the brick [blo, bhi] (periodic: the nearest image of the brick)."""
    x = np.asarray(pos, np.float64)
    shifts = (-1.0, 0.0, 1.0) if periodic else (0.0,)
    g2 = np.zeros(len(x))
    for a in range(3):
        ga = None
        for s in shifts:
            d = np.maximum(np.maximum(blo[a] + s * L[a] - x[:, a], x[:, a] - (bhi[a] + s * L[a])), 0.0)
            ga = d if ga is None else np.minimum(ga, d)
        g2 += ga * ga
    return np.sqrt(g2)


# ---------------------------------------------------------------- communicators
class DistComm:
    """Exchange through torch.distributed (initialised by the caller): NCCL between GPUs, gloo on CPU."""

    def __init__(self, device=None):
        import torch.distributed as dist

        self.dist = dist
        self.rank = dist.get_rank()
        self.size = dist.get_world_size()
        self.device = device

    def alltoallv(self, parts):
        """parts[d] (a numpy array, same trailing shape and dtype on every rank) goes to rank d; returns the list of
        what each rank sent here."""
        import torch

        dev = self.device if self.device is not None else "cpu"
        tail = parts[0].shape[1:]
        counts = torch.tensor([len(p) for p in parts], dtype=torch.int64, device=dev)
        recv_counts = torch.empty_like(counts)
        self.dist.all_to_all_single(recv_counts, counts)
        rc = [int(v) for v in recv_counts.cpu()]
        flat = torch.from_numpy(np.ascontiguousarray(np.concatenate(parts, axis=0))).to(dev)
        out = torch.empty((sum(rc),) + tuple(tail), dtype=flat.dtype, device=dev)
        self.dist.all_to_all_single(out, flat, rc, [len(p) for p in parts])
        out = out.cpu().numpy()
        res, o = [], 0
        for c in rc:
            res.append(out[o:o + c])
            o += c
        return res

    def _allreduce(self, v, op):
        import torch

        dev = self.device if self.device is not None else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def allreduce_max(self, v: float) -> float:
        return self._allreduce(v, self.dist.ReduceOp.MAX)

    def allreduce_sum(self, v: float) -> float:
        return self._allreduce(v, self.dist.ReduceOp.SUM)


class ThreadComm:
    """Ranks as threads of one process (``ThreadComm.group(W)`` gives one communicator per rank); every call is
    collective over the group."""

    class _Shared:
        def __init__(self, size):
            self.size = size
            self.barrier = threading.Barrier(size)
            self.box = [None] * size

    def __init__(self, shared, rank):
        self.s = shared
        self.rank = rank
        self.size = shared.size

    @classmethod
    def group(cls, size):
        sh = cls._Shared(size)
        return [cls(sh, r) for r in range(size)]

    def _exchange(self, item):
        self.s.barrier.wait()
        self.s.box[self.rank] = item
        self.s.barrier.wait()
        got = list(self.s.box)
        self.s.barrier.wait()
        return got

    def alltoallv(self, parts):
        got = self._exchange(parts)
        return [np.array(got[src][self.rank], copy=True) for src in range(self.size)]

    def allreduce_max(self, v: float) -> float:
        return max(float(x) for x in self._exchange(float(v)))

    def allreduce_sum(self, v: float) -> float:
        return float(sum(float(x) for x in self._exchange(float(v))))


# ---------------------------------------------------------------- engine
class EngineRefused(RuntimeError):
    """An engine could not compute the cells of a rank's rows because its buffer zone does not bound them."""


def gpu_engine(pos, n_cells, box_lo, box_hi, precision="filter32", device=None):
    """The cells of rows [0, n_cells) of ``pos`` (numpy [N,3]; the other rows are buffer particles) through the
    library (vt_build_owned): volume, density, least-squares gradient, radius, neighbour CSR (local rows)."""
    import torch

    from . import binding as vt

    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    try:
        h = vt.vt_build_owned(x, n_cells, None, box_lo, box_hi, True, precision)
    except vt.VTError as e:
        if e.code in (vt.VT_ERR_UNSUPPORTED, vt.VT_ERR_SECURITY, vt.VT_ERR_CAPACITY):
            raise EngineRefused(str(e)) from e
        raise
    vol, off, ids = vt.cells(h)
    out = dict(vol=vol.cpu().numpy()[:n_cells], dens=vt.density(h).cpu().numpy()[:n_cells],
               grad=vt.gradient(h).cpu().numpy()[:n_cells], rad=vt.cell_radius(h).cpu().numpy()[:n_cells],
               off=off.cpu().numpy()[:n_cells + 1], ids=ids.cpu().numpy())
    vt.vt_destroy(h)
    return out


# ---------------------------------------------------------------- one rank
def cells_sharded(comm, pos, gid, box_lo, box_hi, engine=gpu_engine, border_factor=2.0, max_rounds=8):
    """The cells of every particle, decomposed over the ranks of ``comm``.

    ``pos`` [n,3] and ``gid`` [n] (int64, global ids) are this rank's share of the input (any split); the box is
    periodic.  Returns a dict for the particles this rank owns after routing: ``gid`` (ascending), ``vol``,
    ``dens``, ``grad``, neighbour CSR ``off``/``ids`` in global ids, and ``t1`` (the near-buffer thickness that
    certified every cell) and ``rounds``."""
    lo = np.broadcast_to(np.asarray(box_lo, np.float64), (3,)).copy()
    hi = np.broadcast_to(np.asarray(box_hi, np.float64), (3,)).copy()
    L = hi - lo
    W, r = comm.size, comm.rank
    grid = brick_grid(W)
    pos = np.asarray(pos)
    gid = np.asarray(gid, np.int64)
    # 1. route to the owners
    owner = brick_of(pos, grid, lo, L)
    got_p = comm.alltoallv([pos[owner == d] for d in range(W)])
    got_g = comm.alltoallv([gid[owner == d] for d in range(W)])
    own_p = np.concatenate(got_p, axis=0)
    own_g = np.concatenate(got_g)
    order = np.argsort(own_g, kind="stable")
    own_p, own_g = own_p[order], own_g[order]
    n_own = len(own_g)
    blo, bhi = brick_bounds(r, grid, lo, L)
    # the mean inter-particle distance of the whole set sets the first buffer (BORDERFACTOR x spacing)
    n_all = comm.allreduce_sum(float(n_own))
    t1 = border_factor * float(np.cbrt(np.prod(L) / max(n_all, 1.0)))
    gaps = [gap_to_brick(own_p, *brick_bounds(d, grid, lo, L), L) for d in range(W)]
    for rounds in range(1, max_rounds + 1):
        t2 = 2.0 * t1
        # 2. buffer particles for every other rank, near then far
        near = [own_p[(gaps[d] <= t1)] if d != r else own_p[:0] for d in range(W)]
        far = [own_p[(gaps[d] > t1) & (gaps[d] <= t2)] if d != r else own_p[:0] for d in range(W)]
        near_g = [own_g[(gaps[d] <= t1)] if d != r else own_g[:0] for d in range(W)]
        far_g = [own_g[(gaps[d] > t1) & (gaps[d] <= t2)] if d != r else own_g[:0] for d in range(W)]
        rn_p, rn_g = comm.alltoallv(near), comm.alltoallv(near_g)
        rf_p, rf_g = comm.alltoallv(far), comm.alltoallv(far_g)
        rows = np.concatenate([own_p] + rn_p + rf_p, axis=0)
        row_g = np.concatenate([own_g] + rn_g + rf_g)
        n_near = sum(len(a) for a in rn_g)
        n_cells = n_own + n_near
        # 3. local cells of the owned and near particles; a near cell that the buffer does not bound can grow past
        # what the engine accepts (e.g. wider than a quarter box): that too is a failed certificate
        try:
            res = engine(rows, n_cells, lo, hi)
        except EngineRefused:
            res = None
        # 4. certificate
        if res is None:
            bad = 1.0
        else:
            g_rows = gap_to_brick(rows[:n_cells], blo, bhi, L)
            rad = np.asarray(res["rad"], np.float64)
            ok_all = (g_rows + 2.0 * rad <= t2) & (rad > 0)
            ok_own = 2.0 * rad[:n_own] <= t1
            bad = float(np.count_nonzero(~ok_all) + np.count_nonzero(~ok_own))
        if comm.allreduce_max(bad) == 0.0:
            break
        t1 *= 2.0
    else:
        raise RuntimeError("buffer zone not certified after %d doublings" % max_rounds)
    # 5. owned outputs, neighbours in global ids
    off = np.asarray(res["off"], np.int64)
    ids_local = np.asarray(res["ids"], np.int64)[:off[n_own]]
    ids_g = row_g[ids_local]
    cnt = np.diff(off[:n_own + 1])
    owner_row = np.repeat(np.arange(n_own), cnt)
    o = np.lexsort((ids_g, owner_row))
    return dict(gid=own_g, vol=np.asarray(res["vol"])[:n_own], dens=np.asarray(res["dens"])[:n_own],
                grad=np.asarray(res["grad"])[:n_own], off=np.concatenate([[0], np.cumsum(cnt)]),
                ids=ids_g[o], t1=t1, rounds=rounds, n_buffer=len(row_g) - n_own)

