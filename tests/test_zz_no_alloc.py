"""The allocation-free volume entry point (for callers that cannot call cudaMalloc).

It must give the same volumes as vt_build + vt_cells on the same points, on
two calls in a row (the scratch array it shares between calls keeps the last
call's contents, so the second call checks that everything that must start
from zero is cleared).  This file is collected last on purpose.
"""
import ctypes

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


def _reference_volumes(pos, lo, hi, periodic):
    h = vt.vt_build(pos, None, (lo,) * 3, (hi,) * 3, periodic, "filter32")
    vol = torch.empty(pos.shape[0], dtype=pos.dtype, device=pos.device)
    vt.vt_cells(h, vol)
    torch.cuda.synchronize()
    vt.vt_destroy(h)
    return vol.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["uniform", "clustered", "bounded"])
def test_noalloc_volumes_match_vt_cells_twice(case):
    if case == "uniform":
        x, lo, hi, periodic = inputs.uniform(4096 + 11, seed=3, dtype=np.float32), 0.0, 1.0, True
    elif case == "clustered":
        N = vt.VT_NOALLOC_MAX_N
        L = float(np.float32(100.0 * (N / 2097152) ** (1.0 / 3.0)))
        x, lo, hi, periodic = inputs.clustered(N, L=L, seed=5), 0.0, L, True
    else:
        pts, off = inputs.halo_sets(n_sets=2, nmin=2000, nmax=6000, seed=6, dtype=np.float32)
        x, lo, hi, periodic = pts[off[1]:off[2]], -1.0, 1.0, False
    pos = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ref = _reference_volumes(pos, lo, hi, periodic)
    for _ in range(2):
        vol = torch.full((pos.shape[0],), -1.0, dtype=pos.dtype, device=pos.device)
        vt.vt_volumes_noalloc(pos, (lo,) * 3, (hi,) * 3, periodic, vol)
        torch.cuda.synchronize()
        got = vol.cpu().numpy().astype(np.float64)
        assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()


def test_noalloc_rejects_oversized_sets():
    x = inputs.uniform(vt.VT_NOALLOC_MAX_N + 1, seed=1, dtype=np.float32)
    pos = torch.from_numpy(x).cuda()
    vol = torch.empty(pos.shape[0], dtype=pos.dtype, device=pos.device)
    with pytest.raises(vt.VTError) as e:
        vt.vt_volumes_noalloc(pos, (0.0,) * 3, (1.0,) * 3, True, vol)
    assert e.value.code == vt.VT_ERR_CAPACITY
