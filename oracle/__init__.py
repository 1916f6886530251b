"""FP64 CPU oracle for the per-particle Voronoi path (PARAVT, arXiv:1601.06429).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use this package.
The GPU library never imports it, and it shares no code with the GPU path.
It imports nothing from the harness either (``tests/work_per_cell.py`` calls it to print the per-cell
work counters that ``bench.py`` keeps as its table of algorithmic flops per cell).

What each function follows in the paper:

* :func:`cells` -- the Voronoi cell of every particle (Introduction), its
  volume from the facets and the neighbours that share a facet
  (Implementation section); periodic boxes (Abstract, Discussion).  Exact
  definition: intersection of the bisector half-spaces, computed in
  ``vt_oracle.c`` with exact side predicates.
* :func:`density` -- density = particle mass / cell volume (Implementation).
* :func:`gradient` -- the density gradient "from density and neighbour
  information" (Implementation).  The paper gives no formula; the reading
  used here is the unweighted least-squares fit of a linear field over the
  Voronoi neighbours, ``(sum d d^T) g = sum d (rho_j - rho_i)``.
* :func:`grid_density` -- densities on a regular grid (Implementation).  The
  paper gives no formula; the reading used here is: each node takes the
  density of the cell that contains the node centre (the nearest particle),
  optionally averaged over S^3 stratified sub-points of the node's voxel.
* :func:`volume_adjoint` -- dV_i/dx_k from facet area, centroid and
  separation.  The paper has no backward pass; this is the derivative of the
  exact volume (moving bisector planes), see the function docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vt_oracle.c")
# VT_ORACLE_SANITIZE=1 builds and loads a separate copy under AddressSanitizer and UndefinedBehaviorSanitizer
# (the process needs the sanitizer runtimes preloaded: LD_PRELOAD="$(gcc -print-file-name=libasan.so)
# $(gcc -print-file-name=libubsan.so)" ASAN_OPTIONS=detect_leaks=0).
_SANITIZE = os.environ.get("VT_ORACLE_SANITIZE") == "1"
_LIB = os.path.join(_HERE, "liboracle_san.so" if _SANITIZE else "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``vt_oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        opt = (["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                "-fno-sanitize-recover=undefined"] if _SANITIZE else ["-O2"])
        cmd = ["gcc"] + opt + ["-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        lib.oracle_cells.argtypes = [i64, P, P, P, i32, P, i64, i32, i32] + [P] * 16 + [i32]
        lib.oracle_cells.restype = i32
        lib.oracle_tree_new.argtypes = [i64, P, P, P, i32]
        lib.oracle_tree_new.restype = P
        lib.oracle_tree_build_seconds.argtypes = [P]
        lib.oracle_tree_build_seconds.restype = ctypes.c_double
        lib.oracle_tree_cells.argtypes = [P, P, i64, i32] + [P] * 16 + [i32]
        lib.oracle_tree_cells.restype = i32
        lib.oracle_tree_free.argtypes = [P]
        lib.oracle_tree_free.restype = None
        lib.oracle_insphere_side.argtypes = [P, P, P, P, P, i32]
        lib.oracle_insphere_side.restype = i32
        lib.oracle_grid_nearest.argtypes = [i64, P, P, P, i32, i32, i32, P, i32]
        lib.oracle_grid_nearest.restype = i32
        lib.oracle_nearest_points.argtypes = [i64, P, P, P, i32, i64, P, P, i32]
        lib.oracle_nearest_points.restype = i32
        lib.oracle_grid_point.argtypes = [P, P, i32, i32, i64, i64, P]
        lib.oracle_grid_volume.argtypes = [i64, P, P, P, i32, i32, P, P, P, i32]
        lib.oracle_grid_volume.restype = i32
        lib.oracle_grid_point.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _box(box_lo, box_hi):
    lo = np.ascontiguousarray(np.broadcast_to(np.asarray(box_lo, dtype=np.float64), (3,)))
    hi = np.ascontiguousarray(np.broadcast_to(np.asarray(box_hi, dtype=np.float64), (3,)))
    return lo, hi


def cells(pos, box_lo=0.0, box_hi=1.0, periodic=True, which=None, mode="brute", face_cap=160, nthreads=0):
    """Voronoi cells of the particles ``which`` (default: all).

    ``pos``: [N,3] positions (any float dtype, converted exactly to FP64;
    periodic boxes need them in [lo, hi)).  ``mode``: ``"brute"`` examines
    all 27N-1 periodic images of every particle, ``"certified"`` enumerates
    them from a k-d tree in radius passes (same result).

    Returns a dict with per-cell ``vol``, ``cen`` (cell centroid),
    ``mom2`` (integral of |y - x_i|^2 over the cell), ``rmax`` (largest vertex distance), ``nface``, ``nvert``,
    ``nedge``, ``ntest`` (planes examined) and ``ncut`` (planes that cut),
    the faces in CSR form (``face_off``, ``f_nbr`` (neighbour id, -1-w for
    box wall w), ``f_shift`` (periodic image), ``f_area``, ``f_cen``,
    ``f_dist``, ``f_m3`` = integral of |y - x_i|^2 (y - x_i) over the facet), and ``counters`` = (predicates,
    exact fallbacks, exact
    zeros, failed cells).
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lo, hi = _box(box_lo, box_hi)
    return _run_cells(pos.shape[0], which, face_cap,
                      lambda wh, n, out: lib.oracle_cells(pos.shape[0], _ptr(pos), _ptr(lo), _ptr(hi),
                                                          int(bool(periodic)), _ptr(wh), n,
                                                          {"brute": 0, "certified": 1}[mode], face_cap, *out,
                                                          int(nthreads)))


def _run_cells(N, which, face_cap, call):
    """Allocate the per-cell and per-facet outputs, run ``call(which, n, pointers)`` and package the result."""
    if which is None:
        wh = None
        n = N
    else:
        wh = np.ascontiguousarray(which, dtype=np.int64)
        n = wh.shape[0]
    vol = np.zeros(n)
    cen = np.zeros((n, 3))
    mom2 = np.zeros(n)
    rmax = np.zeros(n)
    nface = np.zeros(n, np.int32)
    nvert = np.zeros(n, np.int32)
    nedge = np.zeros(n, np.int32)
    ntest = np.zeros(n, np.int64)
    ncut = np.zeros(n, np.int64)
    f_nbr = np.zeros(n * face_cap, np.int64)
    f_shift = np.zeros((n * face_cap, 3), np.int32)
    f_area = np.zeros(n * face_cap)
    f_cen = np.zeros((n * face_cap, 3))
    f_dist = np.zeros(n * face_cap)
    f_m3 = np.zeros((n * face_cap, 3))
    counters = np.zeros(4, np.int64)
    rc = call(wh, n, [_ptr(a) for a in (vol, cen, mom2, rmax, nface, nvert, nedge, ntest, ncut, f_nbr, f_shift,
                                        f_area, f_cen, f_dist, f_m3, counters)])
    if rc != 0:
        raise RuntimeError("oracle_cells failed with code %d on %d cell(s)" % (rc, int(counters[3])))
    nf = nface.astype(np.int64)
    face_off = np.zeros(n + 1, np.int64)
    face_off[1:] = np.cumsum(nf)
    sel = (np.arange(face_cap)[None, :] < nf[:, None]).reshape(-1)
    return dict(which=wh if wh is not None else np.arange(N, dtype=np.int64), vol=vol, cen=cen, mom2=mom2, rmax=rmax,
                nface=nface, nvert=nvert, nedge=nedge, ntest=ntest, ncut=ncut, face_off=face_off,
                f_nbr=f_nbr[sel], f_shift=f_shift[sel], f_area=f_area[sel], f_cen=f_cen[sel],
                f_dist=f_dist[sel], f_m3=f_m3[sel], counters=counters)


class Tree:
    """Certified mode with the k-d tree built once (by the constructor) for many :meth:`cells` calls on the same
    point set; ``build_seconds`` is the wall time the tree took.  The results equal ``cells(..., mode="certified")``.
    """

    def __init__(self, pos, box_lo=0.0, box_hi=1.0, periodic=True):
        self._lib = _load()
        self.pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        self.lo, self.hi = _box(box_lo, box_hi)
        self._t = self._lib.oracle_tree_new(self.pos.shape[0], _ptr(self.pos), _ptr(self.lo), _ptr(self.hi),
                                            int(bool(periodic)))
        if not self._t:
            raise MemoryError("oracle_tree_new")
        self.build_seconds = float(self._lib.oracle_tree_build_seconds(self._t))

    def cells(self, which=None, face_cap=160, nthreads=0):
        t = self._t
        return _run_cells(self.pos.shape[0], which, face_cap,
                          lambda wh, n, out: self._lib.oracle_tree_cells(t, _ptr(wh), n, face_cap, *out,
                                                                         int(nthreads)))

    def close(self):
        if self._t:
            self._lib.oracle_tree_free(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def neighbours(res, self_ids=None):
    """Neighbour lists read off the facets (Implementation section): distinct
    particle ids j != i that share a facet with i, ascending; facets with
    i's own images and box walls are not neighbours.  CSR (off, ids)."""
    wh = res["which"] if self_ids is None else np.asarray(self_ids)
    off = res["face_off"]
    out_off = np.zeros(len(off), np.int64)
    ids = []
    for k in range(len(off) - 1):
        nb = res["f_nbr"][off[k]:off[k + 1]]
        nb = np.unique(nb[(nb >= 0) & (nb != wh[k])])
        ids.append(nb)
        out_off[k + 1] = out_off[k] + len(nb)
    return out_off, (np.concatenate(ids) if ids else np.zeros(0, np.int64))


def neighbour_displacements(res, pos, box_lo=0.0, box_hi=1.0):
    """For each listed cell and each distinct neighbour j (order of
    :func:`neighbours`), the displacement x_j + sL - x_i of the image that
    shares a facet with i; if several images do, the one nearest to x_i."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    lo, hi = _box(box_lo, box_hi)
    L = hi - lo
    wh = res["which"]
    off = res["face_off"]
    noff, nids = neighbours(res)
    disp = np.zeros((len(nids), 3))
    for k in range(len(off) - 1):
        i = wh[k]
        nb = res["f_nbr"][off[k]:off[k + 1]]
        sh = res["f_shift"][off[k]:off[k + 1]]
        for q in range(noff[k], noff[k + 1]):
            j = nids[q]
            m = np.nonzero(nb == j)[0]
            d = pos[j][None, :] + sh[m] * L[None, :] - pos[i][None, :]
            disp[q] = d[np.argmin((d * d).sum(1))]
    return noff, nids, disp


def density(mass, vol):
    """Voronoi density m_i / V_i (Implementation section)."""
    return np.asarray(mass, dtype=np.float64) / np.asarray(vol, dtype=np.float64)


def gradient(dens_self, nbr_off, nbr_ids, disp, dens_all):
    """Least-squares density gradient over the Voronoi neighbours.

    For cell i with neighbours j and displacements d_ij, solves
    ``(sum_j d d^T) g = sum_j d (rho_j - rho_i)`` in FP64 (numpy.linalg.solve
    on the 3x3 normal equations).  ``dens_self[k]`` is rho_i of the k-th
    listed cell, ``dens_all`` indexes rho_j by particle id."""
    dens_all = np.asarray(dens_all, dtype=np.float64)
    n = len(nbr_off) - 1
    g = np.zeros((n, 3))
    for k in range(n):
        a, b = nbr_off[k], nbr_off[k + 1]
        D = disp[a:b]
        f = dens_all[nbr_ids[a:b]] - dens_self[k]
        M = D.T @ D
        g[k] = np.linalg.solve(M, D.T @ f)
    return g


def gradient_green_gauss(res, pos, dens_self, dens_all, box_lo=0.0, box_hi=1.0):
    """Green-Gauss density gradient (the Voronoi form of moving-mesh codes, cited in the Introduction):
    the divergence theorem over the cell, grad rho_i = (1/V_i) * surface integral of rho n, with rho at each
    facet centroid interpolated linearly between the two sites and rho_i on box walls.  Using
    sum_f A_f n_f = 0 and sum_f A_f (c_f - m_f) x n_f = 0 on a closed cell this becomes
    ``(1/V_i) sum_f A_f (rho_j - rho_i) c_f / |d_f|`` over the facets between particles, c_f the facet
    centroid relative to x_i, d_f the image displacement; facets with the cell's own images add nothing.
    ``dens_self[k]`` is rho_i of the k-th listed cell, ``dens_all`` indexes rho_j by particle id."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    lo, hi = _box(box_lo, box_hi)
    L = hi - lo
    dens_all = np.asarray(dens_all, dtype=np.float64)
    off = res["face_off"]
    n = len(off) - 1
    owner = np.repeat(np.arange(n), np.diff(off))
    i = res["which"][owner]
    j = res["f_nbr"]
    inner = j >= 0
    d = pos[np.where(inner, j, 0)] + res["f_shift"] * L[None, :] - pos[i]
    r = np.sqrt((d * d).sum(1))
    c = res["f_cen"] - pos[i]
    w = np.where(inner, res["f_area"] * (dens_all[np.where(inner, j, 0)] - np.asarray(dens_self)[owner]) /
                 np.where(inner, r, 1.0), 0.0)
    g = np.zeros((n, 3))
    np.add.at(g, owner, w[:, None] * c)
    return g / res["vol"][:, None]


def cvt_weighted_gradient(res, pos, w, box_lo=0.0, box_hi=1.0):
    """Gradient of the weighted centroidal energy E_w = sum_i w_i integral over V_i of |y - x_i|^2 with respect to
    every listed site (all particles must be listed).  Moving x_k changes cell k's integrand, 2 w_k V_k (x_k - z_k),
    and moves each facet f between k and j along its normal by (y - x_k).delta / |d_f| at facet point y; since
    |y - x_k| = |y - x_j| on the facet, the energy densities on its two sides differ by (w_k - w_j) |y - x_k|^2, so
    dE_w/dx_k = 2 w_k V_k (x_k - z_k) + sum_f (w_k - w_j) / |d_f| integral_f |y - x_k|^2 (y - x_k) dA.
    Box walls do not move.  ``w`` indexes by particle id."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64)
    wh = res["which"]
    assert len(wh) == len(pos)
    own = 2.0 * (w[wh] * res["vol"])[:, None] * (pos[wh] - res["cen"])
    off = res["face_off"]
    owner = np.repeat(np.arange(len(off) - 1), np.diff(off))
    j = res["f_nbr"]
    inner = j >= 0
    wj = np.where(inner, w[np.where(inner, j, 0)], 0.0)
    coef = np.where(inner, (w[wh[owner]] - wj) / np.where(inner, 2.0 * res["f_dist"], 1.0), 0.0)
    g = own.copy()
    np.add.at(g, owner, coef[:, None] * res["f_m3"])
    return g


def grid_nearest(pos, box_lo, box_hi, G, S=1, periodic=True, nthreads=0):
    """Index of the nearest particle for every node sub-point of a G^3 grid
    (brute force; ties to the lower index).  Returns [G^3, S^3] int64, node
    (a,b,c) at row (c*G + b)*G + a."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    lo, hi = _box(box_lo, box_hi)
    out = np.zeros((G ** 3, S ** 3), np.int64)
    lib.oracle_grid_nearest(pos.shape[0], _ptr(pos), _ptr(lo), _ptr(hi), int(bool(periodic)), G, S, _ptr(out),
                            int(nthreads))
    return out


def nearest_points(pos, queries, box_lo, box_hi, periodic=True, nthreads=0):
    """Index of the nearest particle of each query point (brute force, ties to the lower index, the distance
    evaluated as in :func:`grid_nearest`).  Returns [M] int64."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(queries, dtype=np.float64).reshape(-1, 3)
    lo, hi = _box(box_lo, box_hi)
    out = np.zeros(q.shape[0], np.int64)
    lib.oracle_nearest_points(pos.shape[0], _ptr(pos), _ptr(lo), _ptr(hi), int(bool(periodic)), q.shape[0], _ptr(q),
                              _ptr(out), int(nthreads))
    return out


def grid_density(pos, dens, box_lo, box_hi, G, S=1, periodic=True, nthreads=0):
    """Grid density: node value = mean over its S^3 sub-points of the density
    of the cell containing the sub-point.  Returns [G,G,G] indexed [c,b,a]."""
    idx = grid_nearest(pos, box_lo, box_hi, G, S, periodic, nthreads)
    d = np.asarray(dens, dtype=np.float64)[idx].mean(axis=1)
    return d.reshape(G, G, G)


def grid_volume_density(pos, dens, box_lo, box_hi, G, periodic=True, nthreads=0):
    """Volume-weighted average density of each voxel of a G^3 grid (Implementation section, exact reading):
    ``grid[v] = sum_i dens_i |V_i & voxel v| / |voxel v|``, voxel (a,b,c) = [lo + a h, lo + (a+1) h] per axis
    with h = L/G; every overlap is the cell clipped by the voxel's six walls with the exact predicates.
    Returns [G, G, G] indexed [c][b][a] (x fastest)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    lo, hi = _box(box_lo, box_hi)
    out = np.zeros(G * G * G)
    counters = np.zeros(4, np.int64)
    rc = lib.oracle_grid_volume(pos.shape[0], _ptr(pos), _ptr(lo), _ptr(hi), int(bool(periodic)), int(G),
                                _ptr(dens), _ptr(out), _ptr(counters), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_grid_volume failed with code %d" % rc)
    return out.reshape(G, G, G)


def grid_point(box_lo, box_hi, G, S, node, sub):
    lib = _load()
    lo, hi = _box(box_lo, box_hi)
    g = np.zeros(3)
    lib.oracle_grid_point(_ptr(lo), _ptr(hi), G, S, int(node), int(sub), _ptr(g))
    return g


def insphere_side(xi, pa, pb, pc, pj, exact_only=False):
    """Exact side predicate: +1 when the vertex of the bisectors of x_i with
    p_a, p_b, p_c lies strictly on p_j's side of their bisector (p_j strictly
    inside the circumsphere of x_i, p_a, p_b, p_c), 0 on it, -1 otherwise."""
    lib = _load()
    arrs = [np.ascontiguousarray(v, dtype=np.float64).reshape(3) for v in (xi, pa, pb, pc, pj)]
    return lib.oracle_insphere_side(*[_ptr(a) for a in arrs], 1 if exact_only else 0)


def volume_adjoint(res, pos, box_lo=0.0, box_hi=1.0, g_vol=None, g_energy=None):
    """dL/dx_k for L = sum_i gV_i V_i + gE sum_i E_i, from facet data.

    Derivation (not in the paper): facet (i,j) lies on the plane
    2 y.r = |x_j|^2 - |x_i|^2 (r = x_j - x_i).  Moving x_j by delta moves the
    plane with normal velocity (y - x_j).delta / |r| at facet point y, so
        dV_i/dx_j = A_ij (x_j - c_ij) / |r_ij|,
        dV_i/dx_i = sum_j A_ij (c_ij - x_i) / |r_ij|,
    with A_ij, c_ij the facet area and centroid.  For the CVT energy
    E = sum_i integral_{V_i} |y - x_i|^2 the facet terms cancel and
    dE/dx_i = 2 V_i (x_i - z_i), z_i the cell centroid.
    ``res`` must hold every cell (which = all).  Facets with box walls and
    with i's own images contribute only through their fixed planes (walls:
    nothing; own images: the pair (i, i) moves rigidly).
    """
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    N = pos.shape[0]
    lo, hi = _box(box_lo, box_hi)
    L = hi - lo
    out = np.zeros((N, 3))
    wh = res["which"]
    off = res["face_off"]
    if g_vol is not None:
        gV = np.asarray(g_vol, dtype=np.float64)
        i = np.repeat(wh, np.diff(off))            # cell of each facet
        j = res["f_nbr"]
        keep = (j >= 0) & (j != i)                 # walls and own images do not move
        i, j = i[keep], j[keep]
        xj = pos[j] + res["f_shift"][keep] * L     # the image that shares the facet
        r = np.linalg.norm(xj - pos[i], axis=1)
        A = res["f_area"][keep]
        c = res["f_cen"][keep]
        w = (gV[i] * A / r)[:, None]
        np.add.at(out, i, w * (c - pos[i]))        # dV_i/dx_i term
        np.add.at(out, j, w * (xj - c))            # dV_i/dx_j term
    if g_energy is not None:
        ge = float(g_energy)
        out[wh] += ge * 2.0 * res["vol"][:, None] * (pos[wh] - res["cen"])
    return out
