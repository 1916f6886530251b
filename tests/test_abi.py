"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/vt_gb300.h declares; argument checks
that return before any device work behave as documented.  No GPU needed."""
import ctypes
import os

import pytest

from paper_1601_06429_gb300 import binding
from paper_1601_06429_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return binding.load_library()


def test_exports_every_declared_symbol(lib):
    names = binding.header_symbols()
    assert {"vt_build", "vt_cells", "vt_density", "vt_gradient", "vt_grid_density", "vt_backward", "vt_status",
            "vt_destroy", "vt_error_string", "vt_default_params", "vt_last_error_detail"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_default_params_and_error_strings(lib):
    p = binding.vt_default_params()
    assert p.precision == binding.VT_FILTER32 and p.k_target == 24 and p.max_passes == 1000 and p.face_pool == 24
    assert p.threads_per_cell == 0 and list(p.reserved) == [1, 0, 0]
    assert lib.vt_default_params(None) == binding.VT_ERR_INVALID
    for code in range(0, -9, -1):
        assert binding.error_string(code) != "unknown error code"
    assert binding.error_string(-99) == "unknown error code"


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes mirrors of vt_params and vt_stats have the sizes and field offsets the C compiler
    gives the header's structs."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"vt_params": [f for f, _ in binding.vt_params._fields_],
              "vt_stats": [f for f, _ in binding.vt_stats._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vt_gb300.h"', "int main(void) {"]
    for s, fs in fields.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % s)
        for f in fs:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (s, f))
    lines.append("return 0; }")
    src = tmp_path / "sizes.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for s, fs in fields.items():
        t = getattr(binding, s)
        want.append(ctypes.sizeof(t))
        want += [getattr(t, f).offset for f in fs]
    assert got == want


def test_build_rejects_bad_arguments_without_device_work(lib):
    h = ctypes.c_void_p(123)
    lo = (ctypes.c_double * 3)(0, 0, 0)
    hi = (ctypes.c_double * 3)(1, 1, 1)
    bad_hi = (ctypes.c_double * 3)(1, 0, 1)
    fake = ctypes.c_void_p(16)
    assert lib.vt_build(None, fake, 0, None, 10, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    assert lib.vt_build(ctypes.byref(h), None, 0, None, 10, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    assert h.value is None  # *h is cleared on error
    assert lib.vt_build(ctypes.byref(h), fake, 0, None, 0, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    assert lib.vt_build(ctypes.byref(h), fake, 7, None, 10, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    assert lib.vt_build(ctypes.byref(h), fake, 0, None, 10, lo, bad_hi, 1, None, None) == binding.VT_ERR_INVALID
    p = binding.vt_default_params()
    p.k_target = 2
    assert lib.vt_build(ctypes.byref(h), fake, 0, None, 10, lo, hi, 1, ctypes.byref(p), None) == binding.VT_ERR_INVALID
    # owned builds: 1 <= n_owned <= N
    assert lib.vt_build_owned(ctypes.byref(h), fake, 0, None, 10, 0, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    assert lib.vt_build_owned(ctypes.byref(h), fake, 0, None, 10, 11, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    assert lib.vt_build_owned(None, fake, 0, None, 10, 5, lo, hi, 1, None, None) == binding.VT_ERR_INVALID
    # FP32 filter needs a box length representable in FP32
    p = binding.vt_default_params()
    odd = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    assert lib.vt_build(ctypes.byref(h), fake, 0, None, 10, lo, odd, 1, ctypes.byref(p), None) == \
        binding.VT_ERR_UNSUPPORTED


def test_batched_rejects_bad_sets_without_device_work(lib):
    """vt_build_batched and vt_autotune_batched check set_off, n_sets, the boxes and the per-set parameters on the
    host before they touch the device."""
    h = ctypes.c_void_p(123)
    fake = ctypes.c_void_p(16)
    I64 = ctypes.c_int64 * 4
    I32 = ctypes.c_int32 * 3
    box = [0.0, 0.0, 0.0, 1.0, 1.0, 1.0]
    boxes = (ctypes.c_double * 18)(*(box * 3))
    good = I64(0, 5, 5, 9)
    k_out, t_out = I32(), I32()

    def batched(off, n, bx=boxes, dtype=0, set_k=None, set_tpc=None, p=None):
        return lib.vt_build_batched(ctypes.byref(h), fake, dtype, None, off, n, bx, set_k, set_tpc,
                                    ctypes.byref(p) if p is not None else None, None)

    def tune(off, n, bx=boxes, dtype=0):
        return lib.vt_autotune_batched(fake, dtype, off, n, bx, None, 0, k_out, t_out, None)

    assert lib.vt_build_batched(None, fake, 0, None, good, 3, boxes, None, None, None, None) == binding.VT_ERR_INVALID
    bad_cases = [
        (I64(0, 5, 5, 9), 0),           # no sets
        (I64(0, 5, 5, 9), 65537),       # more than VT_MAX_SETS
        (I64(1, 5, 5, 9), 3),           # set_off[0] != 0
        (I64(0, 5, 4, 9), 3),           # decreasing offsets
        (I64(0, 0, 0, 0), 3),           # no points at all
    ]
    for off, n in bad_cases:
        h.value = 123
        assert batched(off, n) == binding.VT_ERR_INVALID, (list(off), n)
        assert h.value is None
        assert tune(off, n) == binding.VT_ERR_INVALID, (list(off), n)
    assert batched(good, 3, dtype=7) == binding.VT_ERR_INVALID
    assert tune(good, 3, dtype=7) == binding.VT_ERR_INVALID
    flat = (ctypes.c_double * 18)(*(box * 2 + [0.0, 0.0, 0.0, 1.0, 0.0, 1.0]))  # set 2's box has no height
    assert batched(good, 3, bx=flat) == binding.VT_ERR_INVALID
    assert batched(good, 3, set_k=I32(24, 7, 24)) == binding.VT_ERR_INVALID        # k_target below 8
    assert batched(good, 3, set_k=I32(24, 121, 24)) == binding.VT_ERR_INVALID      # k_target above 120
    assert batched(good, 3, set_tpc=I32(32, 1, 2)) == binding.VT_ERR_INVALID       # only 1, 4, 8 or 32 threads per cell
    assert batched(good, 3, set_tpc=I32(16, 1, 4)) == binding.VT_ERR_INVALID
    p = binding.vt_default_params()
    p.threads_per_cell = 2
    assert batched(good, 3, p=p) == binding.VT_ERR_INVALID
    assert lib.vt_autotune_batched(fake, 0, good, 3, boxes, None, 0, None, t_out, None) == binding.VT_ERR_INVALID


def test_newer_calls_reject_null_arguments(lib):
    fake = ctypes.c_void_p(16)
    assert lib.vt_rebuild(None, fake, None) == binding.VT_ERR_INVALID
    assert lib.vt_gradient_gg(None, fake) == binding.VT_ERR_INVALID
    assert lib.vt_grid_density_volume(None, 8, fake) == binding.VT_ERR_INVALID
    assert lib.vt_backward_weighted(None, fake, fake) == binding.VT_ERR_INVALID
    assert lib.vt_moments(None, fake, fake) == binding.VT_ERR_INVALID
    assert lib.vt_probe_fp32_tflops(None, None) == binding.VT_ERR_INVALID
    assert lib.vt_probe_fp64_tflops(None, None) == binding.VT_ERR_INVALID


def test_calls_reject_null_handle(lib):
    assert lib.vt_cells(None, None, None, None, None) == binding.VT_ERR_INVALID
    assert lib.vt_density(None, None) == binding.VT_ERR_INVALID
    assert lib.vt_cell_flags(None, None) == binding.VT_ERR_INVALID
    assert lib.vt_cell_radius(None, None) == binding.VT_ERR_INVALID
    assert lib.vt_gradient(None, None) == binding.VT_ERR_INVALID
    assert lib.vt_grid_density(None, 8, 1, None) == binding.VT_ERR_INVALID
    assert lib.vt_backward(None, None, 0.0, None) == binding.VT_ERR_INVALID
    assert lib.vt_status(None, None) == binding.VT_ERR_INVALID
    lib.vt_destroy(None)  # ignored


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError):
        binding.load_library(str(tmp_path / "missing.so"))


def test_binding_checks_tensors_before_the_library_sees_them(lib):
    """The binding refuses output and input tensors of the wrong dtype, device, layout or size before the C
    call (which only sees raw pointers).  A handle on the CPU device with no library handle behind it: every
    call below must be refused by the binding's own check."""
    import torch

    N = 10
    h = binding.Handle(None, N, torch.float32, torch.device("cpu"), None)
    f32 = lambda *s: torch.zeros(*s, dtype=torch.float32)  # noqa: E731
    bad = {
        "wrong dtype": torch.zeros(N, dtype=torch.float64),
        "too small": f32(N - 1),
        "strided": f32(2 * N)[::2],
        "not a tensor": [0.0] * N,
    }
    for why, t in bad.items():
        for call in (lambda: binding.vt_cells(h, t), lambda: binding.vt_density(h, t),
                     lambda: binding.vt_moments(h, None, t), lambda: binding.vt_backward(h, t, 0.0, f32(N, 3)),
                     lambda: binding.vt_backward_weighted(h, t, f32(N, 3))):
            with pytest.raises(binding.VTError, match="needs a contiguous") as e:
                call()
            assert e.value.code == binding.VT_ERR_INVALID, why
    for call in (lambda: binding.vt_gradient(h, f32(N, 2)), lambda: binding.vt_gradient_gg(h, f32(N, 2)),
                 lambda: binding.vt_backward(h, None, 0.0, f32(N, 2)), lambda: binding.vt_moments(h, f32(N, 2)),
                 lambda: binding.vt_grid_density(h, 4, 1, f32(63)),
                 lambda: binding.vt_grid_density_volume(h, 4, f32(4, 4, 3)),
                 lambda: binding.vt_cells(h, None, torch.zeros(N, dtype=torch.int64)),
                 lambda: binding.vt_cells(h, None, None, torch.zeros(5, dtype=torch.int64))):
        with pytest.raises(binding.VTError, match="needs a contiguous"):
            call()
    # a tensor that passes the check goes on to the library, which refuses the missing handle
    with pytest.raises(binding.VTError) as e:
        binding.vt_density(h, f32(N))
    assert e.value.code == binding.VT_ERR_INVALID and "needs a contiguous" not in str(e.value)


class _FakeLib:
    """Stands in for libvt_gb300.so: records each call's arguments, answers the size query with `nnz`."""

    def __init__(self, nnz):
        self.nnz = nnz
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append((name, args))
            if name == "vt_cells" and args[4] is not None:
                args[4]._obj.value = self.nnz
            return 0
        return f


def test_binding_accepts_the_tensors_its_callers_pass(monkeypatch):
    """The call patterns of the benchmark step, the captured rebuild step, the per-set loop and the convenience
    wrappers, against a recording fake of the library on CPU tensors: every valid tensor passes the checks and
    reaches the C call as its own data pointer."""
    import torch

    N, G, nnz = 12, 4, 50
    fake = _FakeLib(nnz)
    monkeypatch.setattr(binding, "_lib", fake)
    h = binding.Handle(ctypes.c_void_p(None), N, torch.float32, torch.device("cpu"), None)
    vol, dens, w = (torch.zeros(N) for _ in range(3))
    grad, dpos = torch.zeros(N, 3), torch.zeros(N, 3)
    off = torch.zeros(N + 1, dtype=torch.int64)
    ids = torch.zeros(24 * N, dtype=torch.int32)
    grid = torch.zeros(G, G, G)
    assert binding.vt_cells(h) == nnz
    assert binding.vt_cells(h, vol, off, ids) == nnz
    binding.vt_density(h, dens)
    binding.vt_gradient(h, grad)
    binding.vt_grid_density(h, G, 1, grid)
    binding.vt_backward(h, w, 0.0, dpos)
    binding.vt_moments(h, grad, vol)
    binding.vt_moments(h, None, vol)
    assert binding.vt_cells(h, vol, off, None, count=False) is None
    # per-set slices of whole-batch buffers
    hs = binding.Handle(ctypes.c_void_p(None), 5, torch.float32, torch.device("cpu"), None)
    binding.vt_cells(hs, vol[3:8], off[:6], ids[:nnz])
    binding.vt_density(hs, dens[3:8])
    binding.vt_gradient(hs, grad[3:8])
    binding.vt_backward(hs, w[3:8], 0.0, dpos[3:8])
    # the convenience wrappers allocate on the handle's device
    v, o, i = binding.cells(h)
    assert v.shape == (N,) and o.shape == (N + 1,) and i.shape == (nnz,)
    for r in (binding.density(h), binding.gradient(h), binding.gradient_gg(h), binding.grid_density(h, G),
              binding.grid_density_volume(h, G), binding.backward(h, torch.ones(N, dtype=torch.float64)),
              binding.backward_weighted(h, torch.ones(N, dtype=torch.float64)), *binding.moments(h)):
        assert r.device == h.device and r.dtype == h.dtype
    names = [c[0] for c in fake.calls]
    assert "vt_backward_weighted" in names and "vt_grid_density_volume" in names
    # the pointers are the tensors' own
    density_calls = [a for n, a in fake.calls if n == "vt_density"]
    assert density_calls[0][1].value == dens.data_ptr()
    assert density_calls[1][1].value == dens[3:8].data_ptr()
    h.ptr = hs.ptr = None


def test_build_lists_every_source_and_header():
    """Every CUDA translation unit is compiled and every header is a rebuild dependency."""
    from paper_1601_06429_gb300 import build as b

    files = os.listdir(b.CSRC)
    assert sorted(f for f in files if f.endswith(".cu")) == sorted(b.SOURCES)
    assert sorted(f for f in files if f.endswith(".cuh")) == sorted(b.HEADERS)


def test_noalloc_binding_runs_on_the_tensors_device(monkeypatch):
    """vt_volumes_noalloc launches on the current device and uses that device's scratch array, so the binding
    makes the tensors' device current around the C call and refuses a stream of another device.  CPU tensors
    that report a CUDA device stand in for device tensors; a recording fake stands in for the library."""
    import contextlib

    import torch

    class OnDevice1(torch.Tensor):
        @property
        def is_cuda(self):
            return True

        @property
        def device(self):
            return torch.device("cuda", 1)

    class FakeStream:
        def __init__(self, index):
            self.device = torch.device("cuda", index)
            self.cuda_stream = 4242

    current = []
    seen = []

    @contextlib.contextmanager
    def fake_device(d):
        current.append(torch.device(d))
        try:
            yield
        finally:
            current.pop()

    class Lib:
        def vt_volumes_noalloc(self, *args):
            seen.append((current[-1] if current else None, args))
            return 0

    monkeypatch.setattr(binding, "_lib", Lib())
    monkeypatch.setattr(torch.cuda, "device", fake_device)
    monkeypatch.setattr(binding, "_stream_ptr", lambda s: ctypes.c_void_p(s.cuda_stream if s is not None else 7))
    pos = torch.zeros(16, 3).as_subclass(OnDevice1)
    vol = torch.zeros(16).as_subclass(OnDevice1)
    binding.vt_volumes_noalloc(pos, 0.0, 1.0, True, vol)
    binding.vt_volumes_noalloc(pos, 0.0, 1.0, True, vol, stream=FakeStream(1))
    assert [d for d, _ in seen] == [torch.device("cuda", 1)] * 2
    assert seen[1][1][-1].value == 4242 and seen[0][1][0].value == pos.data_ptr()
    with pytest.raises(binding.VTError) as e:
        binding.vt_volumes_noalloc(pos, 0.0, 1.0, True, vol, stream=FakeStream(0))
    assert e.value.code == binding.VT_ERR_INVALID and len(seen) == 2


def test_alloc_failure_hook_arms_and_disarms(lib):
    """The fault-injection hook only sets a host counter: arming returns the previous setting, and nth <= 0
    disarms it (the GPU tests use it to make a build run out of memory)."""
    assert lib.vt_debug_fail_alloc(0) == 0
    assert lib.vt_debug_fail_alloc(3) == 0
    assert lib.vt_debug_fail_alloc(5) == 3
    assert lib.vt_debug_fail_alloc(-1) == 5
    assert lib.vt_debug_fail_alloc(0) == 0
