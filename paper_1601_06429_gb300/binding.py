"""Thin Python binding of the C ABI in ``include/vt_gb300.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls; all the
work happens in the CUDA kernels behind them.  Tensors are torch CUDA tensors
(PyTorch supplies device memory and the stream).  If the compiled library is
missing the functions raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvt_gb300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "vt_gb300.h")

VT_OK = 0
VT_ERR_INVALID = -1
VT_ERR_OOM = -2
VT_ERR_CUDA = -3
VT_ERR_DUPLICATE = -4
VT_ERR_SECURITY = -5
VT_ERR_UNSUPPORTED = -6
VT_ERR_CAPACITY = -7
VT_ERR_NUMERIC = -8
VT_F32 = 0
VT_F64 = 1
VT_PLAIN64 = 0
VT_FILTER32 = 1


class vt_params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("k_target", ctypes.c_int), ("max_passes", ctypes.c_int),
                ("face_pool", ctypes.c_int), ("threads_per_cell", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class vt_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_faces", ctypes.c_int64), ("n_cut", ctypes.c_int64),
                ("n_tested", ctypes.c_int64), ("n_passes", ctypes.c_int64), ("n_fp64_fallbacks", ctypes.c_int64),
                ("n_exact_cells", ctypes.c_int64), ("n_exact_preds", ctypes.c_int64),
                ("n_exact_zero", ctypes.c_int64), ("max_faces", ctypes.c_int64), ("device_error", ctypes.c_int32),
                ("error_particle", ctypes.c_int32), ("n_launches", ctypes.c_int64), ("t_sort_ms", ctypes.c_double),
                ("t_clip_ms", ctypes.c_double), ("reserved", ctypes.c_int64 * 3), ("n_handed_over", ctypes.c_int64),
                ("n_bucket_passes", ctypes.c_int64), ("n_grid_failed", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}
        d["error_detail"] = int(self.reserved[0])
        d["n_collect"] = int(self.reserved[1])
        d["n_collected"] = int(self.reserved[2])
        return d


class VTError(RuntimeError):
    def __init__(self, code, where="", detail=0, particle=-1):
        self.code = int(code)
        self.detail = int(detail)
        self.particle = int(particle)
        msg = error_string(code)
        extra = " [detail %d, particle %d]" % (detail, particle) if detail else ""
        super().__init__("%s: %s (%d)%s" % (where or "vt", msg, code, extra))


_lib = None


def load_library(path: str = LIB_PATH):
    """Load ``libvt_gb300.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libvt_gb300.so not found at %s: build it with paper_1601_06429_gb300.build.build()"
                           % path)
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32 = ctypes.c_int
    i64 = ctypes.c_int64
    lib.vt_default_params.argtypes = [ctypes.POINTER(vt_params)]
    lib.vt_default_params.restype = i32
    lib.vt_build.argtypes = [ctypes.POINTER(P), P, i32, P, i64, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(vt_params), P]
    lib.vt_build.restype = i32
    lib.vt_build_owned.argtypes = [ctypes.POINTER(P), P, i32, P, i64, i64, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), i32, ctypes.POINTER(vt_params), P]
    lib.vt_build_owned.restype = i32
    lib.vt_cell_radius.argtypes = [P, P]
    lib.vt_cell_radius.restype = i32
    lib.vt_build_batched.argtypes = [ctypes.POINTER(P), P, i32, P, ctypes.POINTER(i64), i32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(vt_params), P]
    lib.vt_autotune_batched.argtypes = [P, i32, ctypes.POINTER(i64), i32, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(vt_params), i64, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), P]
    lib.vt_autotune_batched.restype = i32
    lib.vt_build_batched.restype = i32
    lib.vt_rebuild.argtypes = [P, P, P]
    lib.vt_rebuild.restype = i32
    lib.vt_cells.argtypes = [P, P, P, P, ctypes.POINTER(i64)]
    lib.vt_cells.restype = i32
    lib.vt_cell_flags.argtypes = [P, P]
    lib.vt_cell_flags.restype = i32
    lib.vt_density.argtypes = [P, P]
    lib.vt_density.restype = i32
    lib.vt_gradient.argtypes = [P, P]
    lib.vt_gradient.restype = i32
    lib.vt_gradient_gg.argtypes = [P, P]
    lib.vt_gradient_gg.restype = i32
    lib.vt_grid_density.argtypes = [P, i32, i32, P]
    lib.vt_grid_density.restype = i32
    lib.vt_grid_density_volume.argtypes = [P, i32, P]
    lib.vt_grid_density_volume.restype = i32
    lib.vt_backward_weighted.argtypes = [P, P, P]
    lib.vt_backward_weighted.restype = i32
    lib.vt_moments.argtypes = [P, P, P]
    lib.vt_moments.restype = i32
    lib.vt_backward.argtypes = [P, P, ctypes.c_double, P]
    lib.vt_backward.restype = i32
    lib.vt_status.argtypes = [P, ctypes.POINTER(vt_stats)]
    lib.vt_status.restype = i32
    lib.vt_volumes_noalloc.argtypes = [P, i32, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       i32, P, P]
    lib.vt_volumes_noalloc.restype = i32
    lib.vt_probe_fp32_tflops.argtypes = [ctypes.POINTER(ctypes.c_double), P]
    lib.vt_probe_fp32_tflops.restype = i32
    lib.vt_probe_fp64_tflops.argtypes = [ctypes.POINTER(ctypes.c_double), P]
    lib.vt_probe_fp64_tflops.restype = i32
    lib.vt_debug_fail_alloc.argtypes = [i32]
    lib.vt_debug_fail_alloc.restype = i32
    lib.vt_last_error_detail.argtypes = [ctypes.POINTER(ctypes.c_int)]
    lib.vt_last_error_detail.restype = i32
    lib.vt_error_string.argtypes = [i32]
    lib.vt_error_string.restype = ctypes.c_char_p
    lib.vt_destroy.argtypes = [P]
    lib.vt_destroy.restype = None
    lib.vt_release_memory.argtypes = []
    lib.vt_release_memory.restype = i32
    _lib = lib
    return lib


def header_symbols(path: str = HEADER):
    """Names of the entry points declared in the public header."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vt_[a-z_]+)\s*\(", txt)))


def error_string(code: int) -> str:
    try:
        return load_library().vt_error_string(int(code)).decode()
    except Exception:  # library missing: still describe the code
        return "code %d" % code


def _check(rc, where):
    if rc != VT_OK:
        raise VTError(rc, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _arg(t, device, numel, dtype, what):
    """Host-side check of a tensor handed to the library.  The C ABI takes plain pointers, so a tensor on
    another device, of another dtype, strided, or too small would be read or written out of bounds; such a
    tensor raises VT_ERR_INVALID here instead.  None passes (the C call decides whether it is allowed)."""
    if t is None:
        return
    import torch

    if not (isinstance(t, torch.Tensor) and t.device == device and t.dtype == dtype and t.is_contiguous()
            and t.numel() >= numel):
        raise VTError(VT_ERR_INVALID, "%s: needs a contiguous %s tensor on %s with at least %d elements"
                      % (what, dtype, device, numel))


def _stream_ptr(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def vt_probe_fp32_tflops(stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU in TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(load_library().vt_probe_fp32_tflops(ctypes.byref(v), _stream_ptr(stream)), "vt_probe_fp32_tflops")
    return float(v.value)


def vt_probe_fp64_tflops(stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s."""
    v = ctypes.c_double(0.0)
    _check(load_library().vt_probe_fp64_tflops(ctypes.byref(v), _stream_ptr(stream)), "vt_probe_fp64_tflops")
    return float(v.value)


def vt_last_error_detail():
    """(reason, particle) of the last failed vt_build on this thread."""
    part = ctypes.c_int(-1)
    det = load_library().vt_last_error_detail(ctypes.byref(part))
    return int(det), int(part.value)


def vt_debug_fail_alloc(nth: int) -> int:
    """Fault injection for tests: the nth workspace allocation of the next builds fails (VT_ERR_OOM);
    nth <= 0 disarms.  Returns the previous setting."""
    return int(load_library().vt_debug_fail_alloc(int(nth)))


def vt_default_params() -> vt_params:
    p = vt_params()
    _check(load_library().vt_default_params(ctypes.byref(p)), "vt_default_params")
    return p


class Handle:
    """Owns a ``vt_handle``; destroyed with the object (or by :func:`vt_destroy`)."""

    def __init__(self, ptr, N, dtype, device, stream):
        self.ptr = ptr
        self.N = N
        self.dtype = dtype
        self.device = device
        self.stream = stream

    def __del__(self):
        try:
            vt_destroy(self)
        except Exception:
            pass


def vt_build(pos, mass=None, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), periodic=True, precision="filter32",
             k_target=24, max_passes=1000, face_pool=24, stream=None, radius_policy=1, threads_per_cell=0) -> Handle:
    """Voronoi cells of all particles; ``pos`` is a CUDA [N,3] float32/float64 tensor."""
    import torch

    lib = load_library()
    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dim() == 2 and pos.shape[1] == 3):
        raise VTError(VT_ERR_INVALID, "vt_build: pos must be a CUDA [N,3] tensor")
    if pos.dtype not in (torch.float32, torch.float64):
        raise VTError(VT_ERR_INVALID, "vt_build: pos dtype")
    pos = pos.contiguous()
    if mass is not None:
        mass = mass.to(device=pos.device, dtype=pos.dtype).contiguous()
    p = _params(precision, k_target, max_passes, face_pool, radius_policy, threads_per_cell)
    lo = (ctypes.c_double * 3)(*[float(v) for v in (box_lo if hasattr(box_lo, "__len__") else (box_lo,) * 3)])
    hi = (ctypes.c_double * 3)(*[float(v) for v in (box_hi if hasattr(box_hi, "__len__") else (box_hi,) * 3)])
    h = ctypes.c_void_p()
    dt = VT_F32 if pos.dtype == torch.float32 else VT_F64
    with torch.cuda.device(pos.device):
        rc = lib.vt_build(ctypes.byref(h), _ptr(pos), dt, _ptr(mass), pos.shape[0], lo, hi, int(bool(periodic)),
                          ctypes.byref(p), _stream_ptr(stream))
    if rc != VT_OK:
        part = ctypes.c_int(-1)
        det = lib.vt_last_error_detail(ctypes.byref(part))
        raise VTError(rc, "vt_build", det, part.value)
    return Handle(h, pos.shape[0], pos.dtype, pos.device, stream)


def vt_build_owned(pos, n_owned, mass=None, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), periodic=True,
                   precision="filter32", k_target=24, max_passes=1000, face_pool=24, stream=None,
                   radius_policy=1) -> Handle:
    """Cells of the first ``n_owned`` rows of ``pos`` (CUDA [N,3]); the other rows are buffer particles."""
    import torch

    lib = load_library()
    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dim() == 2 and pos.shape[1] == 3):
        raise VTError(VT_ERR_INVALID, "vt_build_owned: pos must be a CUDA [N,3] tensor")
    if pos.dtype not in (torch.float32, torch.float64):
        raise VTError(VT_ERR_INVALID, "vt_build_owned: pos dtype")
    pos = pos.contiguous()
    if mass is not None:
        mass = mass.to(device=pos.device, dtype=pos.dtype).contiguous()
    p = _params(precision, k_target, max_passes, face_pool, radius_policy, 0)
    lo = (ctypes.c_double * 3)(*[float(v) for v in (box_lo if hasattr(box_lo, "__len__") else (box_lo,) * 3)])
    hi = (ctypes.c_double * 3)(*[float(v) for v in (box_hi if hasattr(box_hi, "__len__") else (box_hi,) * 3)])
    h = ctypes.c_void_p()
    dt = VT_F32 if pos.dtype == torch.float32 else VT_F64
    with torch.cuda.device(pos.device):
        rc = lib.vt_build_owned(ctypes.byref(h), _ptr(pos), dt, _ptr(mass), pos.shape[0], int(n_owned), lo, hi,
                                int(bool(periodic)), ctypes.byref(p), _stream_ptr(stream))
    if rc != VT_OK:
        part = ctypes.c_int(-1)
        det = lib.vt_last_error_detail(ctypes.byref(part))
        raise VTError(rc, "vt_build_owned", det, part.value)
    return Handle(h, pos.shape[0], pos.dtype, pos.device, stream)


def _params(precision, k_target, max_passes, face_pool, radius_policy, threads_per_cell=0) -> vt_params:
    p = vt_default_params()
    p.precision = {"filter32": VT_FILTER32, "plain64": VT_PLAIN64}[precision] if isinstance(precision, str) \
        else int(precision)
    p.k_target = int(k_target)
    p.max_passes = int(max_passes)
    p.face_pool = int(face_pool)
    p.reserved[0] = int(radius_policy)
    p.threads_per_cell = int(threads_per_cell)
    return p


def _i32p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def vt_autotune_batched(pos, set_off, boxes, precision="filter32", sample=0, stream=None, **kw):
    """Per-set (k_target, threads_per_cell) chosen by timing trial builds per size class; two int32 arrays."""
    import numpy as np
    import torch

    lib = load_library()
    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dim() == 2 and pos.shape[1] == 3
            and pos.dtype in (torch.float32, torch.float64)):
        raise VTError(VT_ERR_INVALID, "vt_autotune_batched: pos must be a CUDA [N,3] float tensor")
    pos = pos.contiguous()
    off = np.ascontiguousarray(np.asarray(set_off, dtype=np.int64))
    bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 6))
    n_sets = len(off) - 1
    p = _params(precision, kw.get("k_target", 24), kw.get("max_passes", 1000), kw.get("face_pool", 24), 1)
    k_out = np.zeros(n_sets, np.int32)
    t_out = np.zeros(n_sets, np.int32)
    dt = VT_F32 if pos.dtype == torch.float32 else VT_F64
    with torch.cuda.device(pos.device):
        _check(lib.vt_autotune_batched(_ptr(pos), dt, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n_sets,
                                       bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(p),
                                       int(sample), _i32p(k_out), _i32p(t_out), _stream_ptr(stream)),
               "vt_autotune_batched")
    return k_out, t_out


def vt_build_batched(pos, set_off, boxes, mass=None, precision="filter32", k_target=24, max_passes=1000,
                     face_pool=24, stream=None, radius_policy=1, threads_per_cell=0, set_k=None,
                     set_tpc=None) -> Handle:
    """Voronoi cells of independent bounded sets: ``pos`` a CUDA [N,3] tensor, set s the rows
    [set_off[s], set_off[s+1]) inside ``boxes[s] = (lo x, lo y, lo z, hi x, hi y, hi z)``."""
    import numpy as np
    import torch

    lib = load_library()
    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dim() == 2 and pos.shape[1] == 3):
        raise VTError(VT_ERR_INVALID, "vt_build_batched: pos must be a CUDA [N,3] tensor")
    if pos.dtype not in (torch.float32, torch.float64):
        raise VTError(VT_ERR_INVALID, "vt_build_batched: pos dtype")
    pos = pos.contiguous()
    if mass is not None:
        mass = mass.to(device=pos.device, dtype=pos.dtype).contiguous()
    off = np.ascontiguousarray(np.asarray(set_off, dtype=np.int64))
    bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64).reshape(-1, 6))
    n_sets = len(off) - 1
    if n_sets < 1 or bx.shape[0] != n_sets or off[-1] != pos.shape[0]:
        raise VTError(VT_ERR_INVALID, "vt_build_batched: set_off / boxes / pos sizes disagree")
    p = _params(precision, k_target, max_passes, face_pool, radius_policy, threads_per_cell)
    sk = None if set_k is None else np.ascontiguousarray(np.asarray(set_k, dtype=np.int32))
    st = None if set_tpc is None else np.ascontiguousarray(np.asarray(set_tpc, dtype=np.int32))
    if (sk is not None and sk.shape != (n_sets,)) or (st is not None and st.shape != (n_sets,)):
        raise VTError(VT_ERR_INVALID, "vt_build_batched: set_k / set_tpc need one entry per set")
    h = ctypes.c_void_p()
    dt = VT_F32 if pos.dtype == torch.float32 else VT_F64
    with torch.cuda.device(pos.device):
        rc = lib.vt_build_batched(ctypes.byref(h), _ptr(pos), dt, _ptr(mass),
                                  off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n_sets,
                                  bx.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _i32p(sk), _i32p(st),
                                  ctypes.byref(p), _stream_ptr(stream))
    if rc != VT_OK:
        part = ctypes.c_int(-1)
        det = lib.vt_last_error_detail(ctypes.byref(part))
        raise VTError(rc, "vt_build_batched", det, part.value)
    return Handle(h, pos.shape[0], pos.dtype, pos.device, stream)


def vt_rebuild(h: Handle, pos, mass=None) -> None:
    """New positions for the handle's particles (same N, dtype and sets); no allocation, no synchronisation,
    so the call can be captured in a CUDA graph.  Device-side errors come back from vt_status."""
    import torch

    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and tuple(pos.shape) == (h.N, 3) and pos.dtype == h.dtype
            and pos.is_contiguous()):
        raise VTError(VT_ERR_INVALID, "vt_rebuild: pos must be a contiguous CUDA [N,3] tensor of the handle's dtype")
    if mass is not None and not (isinstance(mass, torch.Tensor) and mass.is_cuda and mass.dtype == h.dtype
                                 and mass.is_contiguous() and mass.numel() == h.N):
        raise VTError(VT_ERR_INVALID, "vt_rebuild: mass must be a contiguous CUDA [N] tensor of the handle's dtype")
    _check(load_library().vt_rebuild(h.ptr, _ptr(pos), _ptr(mass)), "vt_rebuild")


def vt_cells(h: Handle, vol=None, nbr_off=None, nbr_id=None, count=True):
    """Fill any of ``vol`` [N], ``nbr_off`` int64 [N+1], ``nbr_id`` int32 [nnz]; returns nnz (None with
    ``count=False``, the form to use inside a CUDA graph capture)."""
    import torch

    _arg(vol, h.device, h.N, h.dtype, "vt_cells vol")
    _arg(nbr_off, h.device, h.N + 1, torch.int64, "vt_cells nbr_off")
    _arg(nbr_id, h.device, 0, torch.int32, "vt_cells nbr_id")
    n = ctypes.c_int64(0)
    if nbr_id is not None and count:
        # room for the facets: the size query first (free unless the handle was rebuilt)
        _check(load_library().vt_cells(h.ptr, None, None, None, ctypes.byref(n)), "vt_cells")
        _arg(nbr_id, h.device, int(n.value), torch.int32, "vt_cells nbr_id")
    _check(load_library().vt_cells(h.ptr, _ptr(vol), _ptr(nbr_off), _ptr(nbr_id),
                                   ctypes.byref(n) if count else None), "vt_cells")
    return int(n.value) if count else None


def vt_cell_radius(h: Handle, rad) -> None:
    """Bound of each cell's largest vertex distance into ``rad`` ([N], input order, the handle's dtype)."""
    _arg(rad, h.device, h.N, h.dtype, "vt_cell_radius rad")
    _check(load_library().vt_cell_radius(h.ptr, _ptr(rad)), "vt_cell_radius")


def cell_radius(h: Handle):
    import torch

    r = torch.empty(h.N, dtype=h.dtype, device=h.device)
    vt_cell_radius(h, r)
    return r


VT_CELL_FP64 = 1
VT_CELL_EXACT = 2


def vt_cell_flags(h: Handle, flags) -> None:
    """Fallback flags of every cell into ``flags`` (uint8 [N], input order): VT_CELL_FP64, VT_CELL_EXACT."""
    import torch

    _arg(flags, h.device, h.N, torch.uint8, "vt_cell_flags flags")
    _check(load_library().vt_cell_flags(h.ptr, _ptr(flags)), "vt_cell_flags")


def cell_flags(h: Handle):
    import torch

    f = torch.empty(h.N, dtype=torch.uint8, device=h.device)
    vt_cell_flags(h, f)
    return f


def vt_density(h: Handle, dens) -> None:
    _arg(dens, h.device, h.N, h.dtype, "vt_density dens")
    _check(load_library().vt_density(h.ptr, _ptr(dens)), "vt_density")


def vt_gradient(h: Handle, grad) -> None:
    _arg(grad, h.device, 3 * h.N, h.dtype, "vt_gradient grad")
    _check(load_library().vt_gradient(h.ptr, _ptr(grad)), "vt_gradient")


def vt_gradient_gg(h: Handle, grad) -> None:
    _arg(grad, h.device, 3 * h.N, h.dtype, "vt_gradient_gg grad")
    _check(load_library().vt_gradient_gg(h.ptr, _ptr(grad)), "vt_gradient_gg")


def vt_grid_density(h: Handle, G: int, S: int, grid) -> None:
    _arg(grid, h.device, max(int(G), 0) ** 3, h.dtype, "vt_grid_density grid")
    _check(load_library().vt_grid_density(h.ptr, int(G), int(S), _ptr(grid)), "vt_grid_density")


def vt_grid_density_volume(h: Handle, G: int, grid) -> None:
    _arg(grid, h.device, max(int(G), 0) ** 3, h.dtype, "vt_grid_density_volume grid")
    _check(load_library().vt_grid_density_volume(h.ptr, int(G), _ptr(grid)), "vt_grid_density_volume")


def grid_density_volume(h: Handle, G: int):
    import torch

    g = torch.empty(G, G, G, dtype=h.dtype, device=h.device)
    vt_grid_density_volume(h, G, g)
    return g


def vt_backward_weighted(h: Handle, w, dE_dpos) -> None:
    _arg(w, h.device, h.N, h.dtype, "vt_backward_weighted w")
    _arg(dE_dpos, h.device, 3 * h.N, h.dtype, "vt_backward_weighted dE_dpos")
    _check(load_library().vt_backward_weighted(h.ptr, _ptr(w), _ptr(dE_dpos)), "vt_backward_weighted")


def backward_weighted(h: Handle, w):
    """Gradient of sum_i w_i integral_{V_i} |y - x_i|^2 with respect to the positions, [N,3]."""
    import torch

    w = w.to(device=h.device, dtype=h.dtype).contiguous()
    out = torch.empty(h.N, 3, dtype=h.dtype, device=h.device)
    vt_backward_weighted(h, w, out)
    return out


def vt_moments(h: Handle, centroid=None, energy=None) -> None:
    _arg(centroid, h.device, 3 * h.N, h.dtype, "vt_moments centroid")
    _arg(energy, h.device, h.N, h.dtype, "vt_moments energy")
    _check(load_library().vt_moments(h.ptr, _ptr(centroid), _ptr(energy)), "vt_moments")


def vt_backward(h: Handle, dL_dV, dL_dE: float, dL_dpos) -> None:
    _arg(dL_dV, h.device, h.N, h.dtype, "vt_backward dL_dV")
    _arg(dL_dpos, h.device, 3 * h.N, h.dtype, "vt_backward dL_dpos")
    _check(load_library().vt_backward(h.ptr, _ptr(dL_dV), float(dL_dE), _ptr(dL_dpos)), "vt_backward")


def vt_status(h: Handle) -> dict:
    st = vt_stats()
    rc = load_library().vt_status(h.ptr, ctypes.byref(st))
    d = st.as_dict()
    d["rc"] = rc
    return d


def vt_destroy(h: Handle) -> None:
    if h is not None and h.ptr is not None and h.ptr.value:
        load_library().vt_destroy(h.ptr)
        h.ptr = None


def vt_release_memory() -> None:
    """Give the unused memory of the library's workspace pool on the current device back (synchronises)."""
    _check(load_library().vt_release_memory(), "vt_release_memory")


VT_NOALLOC_MAX_N = 8192


def vt_volumes_noalloc(pos, box_lo, box_hi, periodic, vol, stream=None) -> None:
    """Cell volumes of at most VT_NOALLOC_MAX_N particles into ``vol`` without any device allocation
    (for callers that cannot allocate); ``pos`` and ``vol`` are CUDA tensors the caller owns."""
    import torch

    if not (isinstance(pos, torch.Tensor) and pos.is_cuda and pos.dim() == 2 and pos.shape[1] == 3
            and pos.dtype in (torch.float32, torch.float64) and pos.is_contiguous()):
        raise VTError(VT_ERR_INVALID, "vt_volumes_noalloc: pos must be a contiguous CUDA [N,3] float tensor")
    _arg(vol, pos.device, pos.shape[0], pos.dtype, "vt_volumes_noalloc vol")
    if stream is not None and stream.device != pos.device:
        # the C side launches on the current device and picks that device's scratch array
        raise VTError(VT_ERR_INVALID, "vt_volumes_noalloc: stream on %s, tensors on %s" % (stream.device, pos.device))
    lo = (ctypes.c_double * 3)(*[float(v) for v in (box_lo if hasattr(box_lo, "__len__") else (box_lo,) * 3)])
    hi = (ctypes.c_double * 3)(*[float(v) for v in (box_hi if hasattr(box_hi, "__len__") else (box_hi,) * 3)])
    dt = VT_F32 if pos.dtype == torch.float32 else VT_F64
    lib = load_library()
    with torch.cuda.device(pos.device):
        _check(lib.vt_volumes_noalloc(_ptr(pos), dt, pos.shape[0], lo, hi, int(bool(periodic)), _ptr(vol),
                                      _stream_ptr(stream)), "vt_volumes_noalloc")


# ---------------------------------------------------------------- convenience wrappers
def cells(h: Handle):
    """(vol [N], nbr_off int64 [N+1], nbr_id int32 [nnz]) as new CUDA tensors."""
    import torch

    nnz = vt_cells(h)
    vol = torch.empty(h.N, dtype=h.dtype, device=h.device)
    off = torch.empty(h.N + 1, dtype=torch.int64, device=h.device)
    ids = torch.empty(max(nnz, 1), dtype=torch.int32, device=h.device)
    vt_cells(h, vol, off, ids)
    return vol, off, ids[:nnz]


def density(h: Handle):
    import torch

    d = torch.empty(h.N, dtype=h.dtype, device=h.device)
    vt_density(h, d)
    return d


def gradient(h: Handle):
    import torch

    g = torch.empty(h.N, 3, dtype=h.dtype, device=h.device)
    vt_gradient(h, g)
    return g


def gradient_gg(h: Handle):
    import torch

    g = torch.empty(h.N, 3, dtype=h.dtype, device=h.device)
    vt_gradient_gg(h, g)
    return g


def grid_density(h: Handle, G: int, S: int = 1):
    import torch

    g = torch.empty(G, G, G, dtype=h.dtype, device=h.device)
    vt_grid_density(h, G, S, g)
    return g


def moments(h: Handle):
    """(centroid [N,3], energy [N]) as new CUDA tensors."""
    import torch

    c = torch.empty(h.N, 3, dtype=h.dtype, device=h.device)
    e = torch.empty(h.N, dtype=h.dtype, device=h.device)
    vt_moments(h, c, e)
    return c, e


def backward(h: Handle, dL_dV=None, dL_dE: float = 0.0):
    import torch

    out = torch.empty(h.N, 3, dtype=h.dtype, device=h.device)
    if dL_dV is not None:
        dL_dV = dL_dV.to(device=h.device, dtype=h.dtype).contiguous()
    vt_backward(h, dL_dV, dL_dE, out)
    return out
