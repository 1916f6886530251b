"""Failure paths that end in an error code, never in a fault or a hang.

* An exhausted candidate-pass budget: with max_passes = 1 most cells of a
  clustered set cannot reach the security radius (the bounded device loop
  gives up), so vt_build returns VT_ERR_SECURITY, promptly, and the next build
  on the same device works.
* An allocation failure, injected on the host into the handle's allocator
  (vt_debug_fail_alloc): at every allocation of vt_build and vt_build_batched
  the call returns VT_ERR_OOM, frees what it had allocated (device memory does
  not creep up over many failed builds) and leaves the library usable.

Nothing here faults, traps or hangs the GPU.
"""
import time

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
    yield
    vt.vt_debug_fail_alloc(0)


def _clustered(N=65536, seed=1):
    L = float(np.float32(100.0 * (N / 2097152) ** (1.0 / 3.0)))
    return inputs.clustered(N, L=L, seed=seed), L


def _volumes(h):
    v, _, _ = vt.cells(h)
    return v.cpu().numpy()


@pytest.mark.parametrize("prec", ["filter32", "plain64"])
def test_exhausted_pass_budget_returns_security_error(prec):
    x, L = _clustered()
    pos = torch.from_numpy(x).cuda()
    t0 = time.perf_counter()
    with pytest.raises(vt.VTError) as e:
        vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, prec, max_passes=1)
    assert e.value.code == vt.VT_ERR_SECURITY
    assert time.perf_counter() - t0 < 30.0
    # the same set with the default budget: every cell is certified
    h = vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, prec)
    assert abs(_volumes(h).astype(np.float64).sum() / L ** 3 - 1.0) < 1e-6
    assert vt.vt_status(h)["rc"] == 0


def test_exhausted_pass_budget_in_a_rebuild_is_sticky():
    """vt_rebuild does not synchronise: the security failure comes back from vt_status.  The handle is built on
    a lattice, whose cells all certify in the first pass, and rebuilt on clustered points, most of whose cells
    need more than one."""
    lat = inputs.sc_lattice(16, perturb=1e-9, seed=0)
    h = vt.vt_build(torch.from_numpy(lat).cuda(), None, (0.0,) * 3, (1.0,) * 3, True, "filter32", max_passes=1)
    assert vt.vt_status(h)["rc"] == 0
    x = inputs.clustered(len(lat), L=1.0, seed=3).astype(np.float64)
    vt.vt_rebuild(h, torch.from_numpy(x).cuda())
    assert vt.vt_status(h)["rc"] == vt.VT_ERR_SECURITY
    vt.vt_destroy(h)


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    vt.vt_release_memory()  # the workspace pool keeps freed memory for reuse: hand it back before measuring
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failure_returns_oom_and_leaks_nothing():
    x, L = _clustered(32768, seed=2)
    pos = torch.from_numpy(x).cuda()
    ref = _volumes(vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, "filter32"))
    free0 = _free_bytes()
    failed = 0
    for nth in range(1, 200):
        vt.vt_debug_fail_alloc(nth)
        try:
            h = vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, "filter32")
        except vt.VTError as e:
            assert e.code == vt.VT_ERR_OOM
            failed += 1
            continue
        # nth is past the last allocation: the hook did not fire and the build is whole
        assert vt.vt_debug_fail_alloc(0) > 0
        assert np.array_equal(_volumes(h), ref)
        vt.vt_destroy(h)
        break
    else:
        pytest.fail("the hook fired at every index")
    assert failed >= 10  # every workspace array of the handle was a failure point
    # repeat the failures: a leak of any of them would add up to far more than the slack
    for _ in range(3):
        for nth in range(1, failed + 1):
            vt.vt_debug_fail_alloc(nth)
            with pytest.raises(vt.VTError) as e:
                vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, "filter32")
            assert e.value.code == vt.VT_ERR_OOM
    assert free0 - _free_bytes() < 64 << 20
    h = vt.vt_build(pos, None, (0.0,) * 3, (L,) * 3, True, "filter32")
    assert np.array_equal(_volumes(h), ref)


def test_injected_allocation_failure_in_batched_build():
    pts, off = inputs.halo_sets(n_sets=8, nmin=64, nmax=4096, seed=6)
    pos = torch.from_numpy(pts).cuda()
    boxes = np.tile([-1.0, -1.0, -1.0, 1.0, 1.0, 1.0], (8, 1))
    ref = _volumes(vt.vt_build_batched(pos, off, boxes))
    for nth in (1, 5, 12):
        vt.vt_debug_fail_alloc(nth)
        with pytest.raises(vt.VTError) as e:
            vt.vt_build_batched(pos, off, boxes)
        assert e.value.code == vt.VT_ERR_OOM
    assert vt.vt_debug_fail_alloc(0) == 0
    assert np.array_equal(_volumes(vt.vt_build_batched(pos, off, boxes)), ref)
