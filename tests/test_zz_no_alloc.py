"""The allocation-free volume entry point (for callers that cannot call cudaMalloc).

Some callers cannot allocate device memory: code that runs inside another
library's memory pool, hosts that forbid allocation after start-up, or code
that must not let an allocation synchronise the device.  vt_volumes_noalloc
serves them from one fixed device array.  It runs the same kernels as
vt_build + vt_cells with the default parameters, so on the same points it must
give the same volumes bit for bit, and each volume must agree with the FP64
oracle to the FP32 path's tolerance (2e-5 relative, per particle).  Both are
checked on two calls in a row: the array keeps the last call's contents, so
the second call shows that everything that must start from zero is cleared.
This file is collected last on purpose.
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


def _case(case):
    """(points, box lo, box hi, periodic) of each parity case."""
    if case == "uniform":
        return inputs.uniform(4096 + 11, seed=3, dtype=np.float32), 0.0, 1.0, True
    if case == "uniform_f64":
        return inputs.uniform(4096 + 11, seed=4, dtype=np.float64), 0.0, 1.0, True
    if case == "clustered":
        N = vt.VT_NOALLOC_MAX_N
        L = float(np.float32(100.0 * (N / 2097152) ** (1.0 / 3.0)))
        return inputs.clustered(N, L=L, seed=5), 0.0, L, True
    pts, off = inputs.halo_sets(n_sets=2, nmin=2000, nmax=6000, seed=6, dtype=np.float32)
    # a bounded box whose walls are not FP32 numbers
    return pts[off[1]:off[2]], -1.1, 1.3, False


def _vt_cells_volumes(pos, lo, hi, periodic):
    h = vt.vt_build(pos, None, (lo,) * 3, (hi,) * 3, periodic, "filter32")
    vol = torch.empty(pos.shape[0], dtype=pos.dtype, device=pos.device)
    vt.vt_cells(h, vol)
    torch.cuda.synchronize()
    vt.vt_destroy(h)
    return vol.cpu().numpy()


@pytest.mark.parametrize("case", ["uniform", "uniform_f64", "clustered", "bounded"])
def test_noalloc_volumes_match_vt_cells_and_oracle_twice(case, oracle_mod):
    x, lo, hi, periodic = _case(case)
    pos = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    ref = _vt_cells_volumes(pos, lo, hi, periodic)
    o = oracle_mod.cells(x.astype(np.float64), lo, hi, periodic, mode="certified")
    for _ in range(2):
        vol = torch.full((pos.shape[0],), -1.0, dtype=pos.dtype, device=pos.device)
        vt.vt_volumes_noalloc(pos, (lo,) * 3, (hi,) * 3, periodic, vol)
        torch.cuda.synchronize()
        got = vol.cpu().numpy()
        assert np.array_equal(got, ref), "differs from vt_build + vt_cells"
        rel = np.abs(got.astype(np.float64) - o["vol"]) / o["vol"]
        assert rel.max() <= 2e-5, "volume rel err %g vs the oracle" % rel.max()


def test_noalloc_rejects_oversized_sets():
    x = inputs.uniform(vt.VT_NOALLOC_MAX_N + 1, seed=1, dtype=np.float32)
    pos = torch.from_numpy(x).cuda()
    vol = torch.empty(pos.shape[0], dtype=pos.dtype, device=pos.device)
    with pytest.raises(vt.VTError) as e:
        vt.vt_volumes_noalloc(pos, (0.0,) * 3, (1.0,) * 3, True, vol)
    assert e.value.code == vt.VT_ERR_CAPACITY
