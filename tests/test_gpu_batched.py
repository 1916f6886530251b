"""Batched independent sets (vt_build_batched) against the FP64 oracle and against per-set vt_build calls.

Workload: independent NFW halos (r_vir = 1, c ~ U(5,15)) of log-uniform size, each in its own bounded box,
FP32; small batches here, and sampled sets of the 4096-set batch (sizes 64 .. 65536, about 38.7 M points).
Tolerances are those of the single-set parity tests: identical neighbour sets, volumes to relative 2e-5
(FP32 filter) or 1e-6 (FP64 path).
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


def unit_boxes(n_sets):
    return np.tile(np.array([-1.0, -1.0, -1.0, 1.0, 1.0, 1.0]), (n_sets, 1))


def run_batched(pts, off, boxes, precision="filter32", threads_per_cell=0):
    pos = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    h = vt.vt_build_batched(pos, off, boxes, precision=precision, threads_per_cell=threads_per_cell)
    vol, noff, ids = vt.cells(h)
    return h, vol.double().cpu().numpy(), noff.cpu().numpy(), ids.cpu().numpy()


def check_set(s, off, box, vol, noff, ids, pts, oracle_mod, tol):
    """Set s of a batched result against the oracle run on that set alone."""
    a, b = int(off[s]), int(off[s + 1])
    if b == a:
        return
    x = pts[a:b].astype(np.float64)
    o = oracle_mod.cells(x, box[:3], box[3:], False, mode="certified")
    ooff, oids = oracle_mod.neighbours(o)
    rel = np.abs(vol[a:b] - o["vol"]) / o["vol"]
    assert rel.max() <= tol, (s, rel.max())
    for k in range(b - a):
        got = ids[noff[a + k]:noff[a + k + 1]]
        assert ((got >= a) & (got < b)).all(), (s, k, "neighbour outside the set")
        assert np.array_equal(got - a, oids[ooff[k]:ooff[k + 1]]), (s, k)
    bv = np.prod(box[3:] - box[:3])
    assert abs(vol[a:b].sum() - bv) <= 1e-5 * bv


@pytest.fixture(scope="module")
def sets64():
    return inputs.halo_sets(n_sets=64, nmin=64, nmax=4096, seed=6, dtype=np.float32)


@pytest.mark.parametrize("precision,tol,tpc", [("filter32", 2e-5, 32), ("filter32", 2e-5, 1), ("filter32", 2e-5, 4),
                                               ("filter32", 2e-5, 8), ("plain64", 1e-6, 32)])
def test_batched_matches_oracle_every_set(sets64, oracle_mod, precision, tol, tpc):
    pts, off = sets64
    boxes = unit_boxes(len(off) - 1)
    h, vol, noff, ids = run_batched(pts, off, boxes, precision, tpc)
    for s in range(len(off) - 1):
        check_set(s, off, boxes[s], vol, noff, ids, pts, oracle_mod, tol)
    st = vt.vt_status(h)
    assert st["rc"] == 0 and st["n_faces"] == len(ids)


def test_batched_equals_per_set_builds(sets64):
    pts, off = sets64
    boxes = unit_boxes(len(off) - 1)
    h, vol, noff, ids = run_batched(pts, off, boxes)
    dens = vt.density(h).double().cpu().numpy()
    grad = vt.gradient(h).double().cpu().numpy()
    cen, energy = vt.moments(h)
    cen = cen.double().cpu().numpy()
    energy = energy.double().cpu().numpy()
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        pos = torch.from_numpy(np.ascontiguousarray(pts[a:b])).cuda()
        hs = vt.vt_build(pos, None, (-1.0,) * 3, (1.0,) * 3, False, "filter32")
        v1, o1, i1 = vt.cells(hs)
        v1 = v1.double().cpu().numpy()
        assert np.array_equal(o1.cpu().numpy(), noff[a:b + 1] - noff[a])
        assert np.array_equal(i1.cpu().numpy(), ids[noff[a]:noff[b]] - a)
        assert (np.abs(vol[a:b] - v1) <= 4e-5 * v1).all()
        assert (np.abs(dens[a:b] - 1.0 / v1) <= 4e-5 / v1).all()
        g1 = vt.gradient(hs).double().cpu().numpy()
        sc = np.linalg.norm(g1, axis=1) + 1e-1 * (1.0 / v1) / v1 ** (1.0 / 3.0)
        assert (np.linalg.norm(grad[a:b] - g1, axis=1) <= 1e-3 * sc).all(), s
        c1, e1 = vt.moments(hs)
        assert np.allclose(cen[a:b], c1.double().cpu().numpy(), rtol=0, atol=1e-5)
        assert np.allclose(energy[a:b], e1.double().cpu().numpy(), rtol=1e-4, atol=0)


def test_batched_varied_boxes_and_degenerate_sets(oracle_mod):
    """Sets in boxes of different centres and sizes, with an empty set, a one-point set and a two-point set."""
    base, boff = inputs.halo_sets(n_sets=6, nmin=100, nmax=3000, seed=11, dtype=np.float64)
    g = inputs.rng(12)
    parts, sizes, boxes = [], [], []
    for s in range(6):
        c = g.uniform(-50.0, 50.0, 3)
        hw = g.uniform(0.25, 4.0)
        parts.append(c + hw * base[boff[s]:boff[s + 1]])
        sizes.append(boff[s + 1] - boff[s])
        boxes.append(np.concatenate([c - hw, c + hw]))
        if s == 1:  # empty set
            parts.append(np.zeros((0, 3)))
            sizes.append(0)
            boxes.append(np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0]))
        if s == 3:  # one point: its cell is the whole box
            parts.append(np.array([[2.0, 3.0, 4.5]]))
            sizes.append(1)
            boxes.append(np.array([1.0, 2.0, 4.0, 3.5, 3.25, 5.0]))
        if s == 4:  # two points: the box cut by one bisector
            parts.append(np.array([[0.25, 0.5, 0.5], [0.75, 0.5, 0.5]]))
            sizes.append(2)
            boxes.append(np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0]))
    pts = np.concatenate(parts)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    boxes = np.array(boxes)
    for precision, tol, tpc in (("plain64", 1e-6, 32), ("filter32", 2e-5, 32), ("filter32", 2e-5, 1),
                                ("filter32", 2e-5, 4), ("filter32", 2e-5, 8)):
        h, vol, noff, ids = run_batched(pts, off, boxes, precision, tpc)
        for s in range(len(sizes)):
            check_set(s, off, boxes[s], vol, noff, ids, pts, oracle_mod, tol)
        one = int(off[5])  # sets: 0, 1, empty, 2, 3, one point, 4, two points, 5
        assert sizes[5] == 1 and abs(vol[one] - 2.5 * 1.25 * 1.0) <= tol * 3.125
        two = int(off[7])
        assert sizes[7] == 2 and np.allclose(vol[two:two + 2], 0.5, rtol=tol)


def test_per_set_configuration_matches_oracle(sets64, oracle_mod):
    """Each set with its own k_target and kernel (1, 4, 8 or 32 threads per cell), mixed in one batch."""
    pts, off = sets64
    n_sets = len(off) - 1
    g = np.random.default_rng(21)
    set_k = g.choice([16, 24, 32, 48, 64], n_sets).astype(np.int32)
    set_tpc = g.choice([1, 4, 8, 32], n_sets).astype(np.int32)
    boxes = unit_boxes(n_sets)
    pos = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    h = vt.vt_build_batched(pos, off, boxes, set_k=set_k, set_tpc=set_tpc)
    vol, noff, ids = vt.cells(h)
    vol, noff, ids = vol.double().cpu().numpy(), noff.cpu().numpy(), ids.cpu().numpy()
    for s in range(n_sets):
        check_set(s, off, boxes[s], vol, noff, ids, pts, oracle_mod, 2e-5)


def test_autotune_choices_are_valid_and_change_no_cell(sets64):
    pts, off = sets64
    n_sets = len(off) - 1
    boxes = unit_boxes(n_sets)
    pos = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    set_k, set_tpc = vt.vt_autotune_batched(pos, off, boxes, sample=16384)
    assert set(set_k.tolist()) <= {16, 24, 32, 48, 64} and set(set_tpc.tolist()) <= {1, 4, 8, 32}
    # sets of one size class share their choice
    cls = np.floor(np.log2(np.diff(off))).astype(int)
    for c in np.unique(cls):
        assert len(set(zip(set_k[cls == c].tolist(), set_tpc[cls == c].tolist()))) == 1
    _, v0, o0, i0 = run_batched(pts, off, boxes)
    h = vt.vt_build_batched(pos, off, boxes, set_k=set_k, set_tpc=set_tpc)
    v1, o1, i1 = vt.cells(h)
    assert np.array_equal(o1.cpu().numpy(), o0) and np.array_equal(i1.cpu().numpy(), i0)
    assert (np.abs(v1.double().cpu().numpy() - v0) <= 4e-5 * v0).all()


def test_batched_errors():
    pts, off = inputs.halo_sets(n_sets=4, nmin=64, nmax=256, seed=6, dtype=np.float32)
    boxes = unit_boxes(4)
    pos = torch.from_numpy(pts).cuda()
    h = vt.vt_build_batched(pos, off, boxes)
    with pytest.raises(vt.VTError) as e:
        vt.grid_density(h, 8)
    assert e.value.code == vt.VT_ERR_UNSUPPORTED
    bad = boxes.copy()
    bad[2] = [0.0, 0.0, 0.0, 0.5, 0.5, 0.5]  # set 2's points leave its box
    with pytest.raises(vt.VTError) as e:
        vt.vt_build_batched(pos, off, bad)
    assert e.value.code == vt.VT_ERR_INVALID
    rev = off.copy()
    rev[1], rev[2] = rev[2], rev[1]
    with pytest.raises(vt.VTError) as e:
        vt.vt_build_batched(pos, rev, boxes)
    assert e.value.code == vt.VT_ERR_INVALID
    with pytest.raises(vt.VTError) as e:  # k_target out of range for one set
        vt.vt_build_batched(pos, off, boxes, set_k=np.array([40, 40, 4, 40], np.int32))
    assert e.value.code == vt.VT_ERR_INVALID


@pytest.fixture(scope="module")
def sets4096():
    return inputs.halo_sets()


def test_halo_sets_4096_sampled(sets4096, oracle_mod):
    """The 4096-set batch at full size (about 38.7 M points, FP32 filter): every set's volumes sum to its box,
    neighbour lists stay inside their set and are symmetric, and 12 sampled sets (the largest, the smallest and
    10 random ones) match the oracle exactly in their neighbours."""
    pts, off = sets4096
    n_sets = len(off) - 1
    boxes = unit_boxes(n_sets)
    h, vol, noff, ids = run_batched(pts, off, boxes)
    assert vt.vt_status(h)["rc"] == 0
    sid = np.repeat(np.arange(n_sets), np.diff(off))
    sums = np.bincount(sid, weights=vol, minlength=n_sets)
    assert np.abs(sums - 8.0).max() <= 1e-4
    owner = np.repeat(np.arange(len(pts)), np.diff(noff))
    assert (sid[owner] == sid[ids]).all()
    # symmetry: (i, j) present iff (j, i) present
    fwd = owner.astype(np.int64) * len(pts) + ids
    bwd = ids.astype(np.int64) * len(pts) + owner
    assert np.array_equal(np.sort(fwd), np.sort(bwd))
    sizes = np.diff(off)
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))}
    pick |= set(inputs.rng(13).choice(n_sets, 10, replace=False).tolist())
    for s in sorted(pick):
        check_set(s, off, boxes[s], vol, noff, ids, pts, oracle_mod, 2e-5)


def test_halo_sets_4096_graph_replay(sets4096):
    """The 4096-set batch as one captured CUDA graph: a batched handle (per-set k_target from the autotuner) is
    rebuilt inside the capture together with volumes, CSR offsets, densities and gradients; replays on new
    positions of the same set sizes (each set mirrored through its centre, then the original) equal a fresh
    batched build of those positions bit for bit, neighbour lists included."""
    pts, off = sets4096
    n_sets = len(off) - 1
    boxes = unit_boxes(n_sets)
    N = len(pts)
    set_k, set_tpc = vt.vt_autotune_batched(torch.from_numpy(pts).cuda(), off, boxes, sample=65536)
    s = torch.cuda.Stream()
    static = torch.from_numpy(pts).cuda()
    vol = torch.empty(N, device="cuda")
    noff = torch.empty(N + 1, dtype=torch.int64, device="cuda")
    dens = torch.empty(N, device="cuda")
    grad = torch.empty(N, 3, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        h = vt.vt_build_batched(static, off, boxes, stream=s, set_k=set_k, set_tpc=set_tpc)
        vt.vt_rebuild(h, static)  # one call outside the capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        vt.vt_rebuild(h, static)
        vt.vt_cells(h, vol, noff, None, count=False)
        vt.vt_density(h, dens)
        vt.vt_gradient(h, grad)
    for new in (-pts, pts):
        static.copy_(torch.from_numpy(np.ascontiguousarray(new)))
        g.replay()
        torch.cuda.synchronize()
        assert vt.vt_status(h)["rc"] == 0
        ref = vt.vt_build_batched(torch.from_numpy(np.ascontiguousarray(new)).cuda(), off, boxes, set_k=set_k,
                                  set_tpc=set_tpc)
        rv, ro, ri = vt.cells(ref)
        assert torch.equal(vol, rv) and torch.equal(noff, ro)
        assert torch.equal(dens, vt.density(ref)) and torch.equal(grad, vt.gradient(ref))
        n = vt.vt_cells(h)
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        vt.vt_cells(h, None, None, ids)
        assert torch.equal(ids, ri)
        vt.vt_destroy(ref)
    vt.vt_destroy(h)
