"""vt_rebuild (new positions in an existing handle's workspace) and its capture in a CUDA graph.

Workload: the 1,048,576-point halo + uniform mixture in the unit periodic box (FP32) and the 64-set batch of
bounded NFW halos.  A rebuild computes every cell exactly as a fresh vt_build does (each cell is computed by one
warp from the same inputs), so volumes, neighbour lists, densities and gradients are compared bit for bit.
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


BOX = ((0.0,) * 3, (1.0,) * 3)


def outputs(h):
    vol, off, ids = vt.cells(h)
    return dict(vol=vol.cpu(), off=off.cpu(), ids=ids.cpu(), dens=vt.density(h).cpu(), grad=vt.gradient(h).cpu())


def same(a, b):
    for k in a:
        assert torch.equal(a[k], b[k]), k


def test_rebuild_equals_fresh_build():
    x0 = torch.from_numpy(inputs.halo_uniform_mix(1048576, L=1.0, seed=3)).cuda()
    x1 = torch.from_numpy(inputs.halo_uniform_mix(1048576, L=1.0, seed=8)).cuda()
    h = vt.vt_build(x0, None, *BOX, True, "filter32")
    vt.vt_rebuild(h, x1)
    got = outputs(h)
    assert vt.vt_status(h)["rc"] == 0
    same(got, outputs(vt.vt_build(x1, None, *BOX, True, "filter32")))
    vt.vt_rebuild(h, x0)  # and back
    same(outputs(h), outputs(vt.vt_build(x0, None, *BOX, True, "filter32")))


def test_rebuild_batched_sets():
    pts, off = inputs.halo_sets(n_sets=64, nmin=64, nmax=4096, seed=6, dtype=np.float32)
    pts2, _ = inputs.halo_sets(n_sets=64, nmin=64, nmax=4096, seed=6, dtype=np.float32)
    # other points with the same set sizes: each set mirrored through its centre
    pts2 = -pts2
    boxes = np.tile([-1.0, -1.0, -1.0, 1.0, 1.0, 1.0], (64, 1))
    h = vt.vt_build_batched(torch.from_numpy(pts).cuda(), off, boxes)
    vt.vt_rebuild(h, torch.from_numpy(pts2).cuda())
    same(outputs(h), outputs(vt.vt_build_batched(torch.from_numpy(pts2).cuda(), off, boxes)))


def test_graph_capture_and_replay():
    N = 262144
    xs = [torch.from_numpy(inputs.halo_uniform_mix(N, L=1.0, seed=s)).cuda() for s in (3, 8, 9)]
    s = torch.cuda.Stream()
    static_x = xs[0].clone()
    w = torch.rand(N, device="cuda")
    vol = torch.empty(N, device="cuda")
    off = torch.empty(N + 1, dtype=torch.int64, device="cuda")
    dens = torch.empty(N, device="cuda")
    grad = torch.empty(N, 3, device="cuda")
    dpos = torch.empty(N, 3, device="cuda")
    with torch.cuda.stream(s):
        h = vt.vt_build(static_x, None, *BOX, True, "filter32", stream=s)
        vt.vt_rebuild(h, static_x)  # one call outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vt.vt_rebuild(h, static_x)
        vt.vt_cells(h, vol, off, None, count=False)
        vt.vt_density(h, dens)
        vt.vt_gradient(h, grad)
        vt.vt_backward(h, w, 0.5, dpos)
    for x in (xs[1], xs[2], xs[0]):
        static_x.copy_(x)
        g.replay()
        torch.cuda.synchronize()
        assert vt.vt_status(h)["rc"] == 0
        ref = vt.vt_build(x, None, *BOX, True, "filter32")
        rv, ro, _ = vt.cells(ref)
        assert torch.equal(vol, rv) and torch.equal(off, ro)
        assert torch.equal(dens, vt.density(ref)) and torch.equal(grad, vt.gradient(ref))
        assert torch.equal(dpos, vt.backward(ref, w, 0.5))
        # the neighbour list after the replay, outside the capture: ask for the size first
        n = vt.vt_cells(h)
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        vt.vt_cells(h, None, None, ids)
        assert torch.equal(ids, vt.cells(ref)[2])


def test_rebuild_errors_are_sticky_and_cleared():
    x = torch.from_numpy(inputs.uniform(8192, seed=1, dtype=np.float32)).cuda()
    h = vt.vt_build(x, None, *BOX, True, "filter32")
    bad = x.clone()
    bad[100, 1] = float("nan")
    vt.vt_rebuild(h, bad)
    assert vt.vt_status(h)["rc"] == vt.VT_ERR_INVALID
    bad = x.clone()
    bad[7, 0] = 1.5
    vt.vt_rebuild(h, bad)
    assert vt.vt_status(h)["rc"] == vt.VT_ERR_INVALID
    vt.vt_rebuild(h, x)
    assert vt.vt_status(h)["rc"] == 0
    same(outputs(h), outputs(vt.vt_build(x, None, *BOX, True, "filter32")))


def test_rebuild_reports_a_full_facet_pool():
    # a perturbed BCC lattice has 14 facets per cell; uniform points have 15.5 on average
    lat = torch.from_numpy(inputs.bcc_lattice(16, perturb=1e-4, seed=2, dtype=np.float32)).cuda()
    N = lat.shape[0]
    h = vt.vt_build(lat, None, *BOX, True, "filter32", face_pool=14)
    vt.vt_rebuild(h, torch.from_numpy(inputs.uniform(N, seed=4, dtype=np.float32)).cuda())
    assert vt.vt_status(h)["rc"] == vt.VT_ERR_CAPACITY
    vt.vt_rebuild(h, lat)
    assert vt.vt_status(h)["rc"] == 0
