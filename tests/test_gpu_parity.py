"""GPU parity: the CUDA path through the C ABI against the float64 oracle (and,
for the sort and scan primitives, against numpy's stable sort and cumsum) on
seeded inputs."""
import math

import numpy as np
import pytest

import oracle as O
from scenegen import camera_c0, look_camera, make_floor_scene, quantize_attributes, walk_cameras
from tests.gpu_helpers import (clear_tau, compare_cut, compare_image, compare_tile_lists,
                               compare_tile_order_f64)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_15186_gb300 import Renderer
    r = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22, pair_capacity=1 << 24)
    yield r
    r.close()


# ---------------------------------------------------------------------------
# primitives: onesweep radix sort and chained scan
# ---------------------------------------------------------------------------

def _sort_check(R, keys_np, begin=0, end=None):
    kb = keys_np.dtype.itemsize
    end = 8 * kb if end is None else end
    n = len(keys_np)
    vals_np = np.arange(n, dtype=np.uint32)
    tdt = torch.int32 if kb == 4 else torch.int64
    k = torch.from_numpy(keys_np.view(np.int32 if kb == 4 else np.int64).copy()).cuda()
    v = torch.from_numpy(vals_np.view(np.int32).copy()).cuda()
    R.sort_pairs(k, v, begin, end)
    R.synchronize()
    gk = k.cpu().numpy().view(keys_np.dtype)
    gv = v.cpu().numpy().view(np.uint32)
    mask = (1 << (end - begin)) - 1 if end - begin < 64 else (1 << 64) - 1
    dig = (keys_np.astype(np.uint64) >> np.uint64(begin)) & np.uint64(mask)
    o = np.argsort(dig, kind="stable")
    assert np.array_equal(gv, vals_np[o])
    assert np.array_equal(gk, keys_np[o])


@pytest.mark.parametrize("n", [0, 1, 7, 4095, 4096, 4097, 100_003])
def test_sort_u32_random(R, n):
    rng = np.random.default_rng(n)
    _sort_check(R, rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32))


def test_sort_u32_few_distinct_and_partial_bits(R):
    rng = np.random.default_rng(1)
    _sort_check(R, rng.integers(0, 5, 50_000).astype(np.uint32))         # heavy ties: stability
    _sort_check(R, np.full(20_000, 77, np.uint32))                         # all equal
    _sort_check(R, rng.integers(0, 2 ** 32, 30_000, dtype=np.uint64).astype(np.uint32), 4, 20)
    _sort_check(R, np.arange(30_000, 0, -1).astype(np.uint32) << np.uint32(16), 16, 32)


@pytest.mark.parametrize("n", [1, 12_345, 200_001])
def test_sort_u64(R, n):
    rng = np.random.default_rng(7 + n)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64) ^ (rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63))
    _sort_check(R, keys)
    # (tile << 32 | depth bits) keys with all-distinct tiles and shared depths
    tiles = rng.permutation(n).astype(np.uint64)
    _sort_check(R, (tiles << np.uint64(32)) | np.uint64(0x3F800000), 0, 64)


@pytest.mark.parametrize("n", [0, 1, 2047, 2048, 2049, 1_000_003])
def test_scan_u32(R, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 100, n).astype(np.int32)
    t = torch.from_numpy(x).cuda()
    out, total = R.scan_u32(t)
    R.synchronize()
    want = np.concatenate([[0], np.cumsum(x)[:-1]]) if n else np.zeros(0)
    assert np.array_equal(out.cpu().numpy(), want.astype(np.int32))
    assert int(total.item()) == int(x.sum())


# ---------------------------------------------------------------------------
# cut
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("tau", [0.0, 4.0, 16.0, 40.0, 200.0])
def test_cut_matches_oracle(R, box10k, tau):
    R.load_scene(box10k)
    cams = [camera_c0(tau), look_camera((-3.0, 2.0, 1.5), 0.0, 64, 64, fx=60.0, tau=tau)]
    ids, off = R.select_cut(cams)
    ids, off = ids.cpu().numpy(), off.cpu().numpy()
    for c, cam in enumerate(cams):
        compare_cut(ids[off[c]:off[c + 1]], box10k, cam)


def _many_cams(tau):
    cams = [camera_c0(tau)]
    for i in range(10):
        cams.append(look_camera((-3.0 + 0.9 * i, 2.0 - 0.5 * i, 1.2 + 0.1 * i), 0.6 * i,
                                64 + 8 * i, 48, fx=40.0 + 9.0 * i, tau=tau * (0.5 + 0.15 * i)))
    return cams


@pytest.mark.parametrize("tau", [0.0, 4.0, 16.0, 60.0])
def test_cut_many_cameras_matches_oracle(R, box10k, tau):
    """Eleven cameras take the camera-blocked two-pass cut (chunks of 8 and 3):
    each camera's cut equals the oracle's away from tau, and equals the
    single-camera kernel's cut bit for bit."""
    R.load_scene(box10k)
    cams = _many_cams(tau)
    ids, off = R.select_cut(cams)
    ids, off = ids.cpu().numpy(), off.cpu().numpy()
    for c, cam in enumerate(cams):
        compare_cut(ids[off[c]:off[c + 1]], box10k, cam)
        one, o1 = R.select_cut([cam])
        assert np.array_equal(one[: int(o1[1].item())].cpu().numpy(), ids[off[c]:off[c + 1]])


def test_cut_many_cameras_capacity(R, box10k):
    from paper_2603_15186_gb300 import NgsError
    R.load_scene(box10k)
    cams = _many_cams(0.0)
    with pytest.raises(NgsError) as e:
        R.select_cut(cams, cap=1000)
    assert e.value.status == 4
    ids, off = R.select_cut(cams)
    assert int(off[-1].item()) == 11 * 10_000     # tau = 0: every camera's cut is all leaves


# ---------------------------------------------------------------------------
# frustum-culled and shared cuts
# ---------------------------------------------------------------------------

def _compare_groups(ids, off, scene, cams, gb, frustum, guard):
    ids, off = ids.cpu().numpy(), off.cpu().numpy()
    want, woff, near = O.select_cut_shared(scene, cams, gb, frustum=frustum, guard=guard)
    M = scene.n_nodes
    for g in range(len(gb) - 1):
        got = ids[off[g]:off[g + 1]]
        assert np.all(np.diff(got) > 0)
        a, b = np.zeros(M, bool), np.zeros(M, bool)
        a[got] = True
        b[want[woff[g]:woff[g + 1]]] = True
        bad = (a != b) & (near[g] == 0)
        assert not bad.any(), f"group {g}: {int(bad.sum())} decisions differ"
        assert near[g].mean() < 0.01


def _group_walk_cams(scene):
    taus = [5.0, 6.0, 12.0, 4.0, 20.0, 10.0, 30.0, 8.0, 16.0, 40.0]
    cams = walk_cameras(scene, 10, 21, 160, 120, fx=150.0, taus=taus)
    cams[3] = look_camera((-3.0, 3.0, 1.5), math.pi, 33, 17, fx=30.0, tau=2.0)  # outside, away
    cams[7].width, cams[7].height, cams[7].cx, cams[7].cy = 97, 61, 40.0, 35.5   # off-centre
    return cams


@pytest.mark.parametrize("frustum,guard", [(False, 0.0), (True, 0.0), (True, 32.0)])
def test_shared_cut_matches_oracle(R, small_floor, frustum, guard):
    """Groups of 1, 1, 3 and 5 cameras: every group's cut equals the oracle's
    on every node whose decisions (tau threshold, frustum planes, for any
    member, at the node or its parent) are not within float32 reach."""
    R.load_scene(small_floor)
    cams = _group_walk_cams(small_floor)
    gb = [0, 1, 3, 4, 10]
    ids, off = R.select_cut_shared(cams, gb, frustum=frustum, guard=guard)
    _compare_groups(ids, off, small_floor, cams, gb, frustum, guard)
    if frustum:
        assert int(off[3].item()) == int(off[2].item())   # the camera facing away sees nothing


def test_shared_cut_of_single_cameras_is_the_plain_cut(R, small_floor):
    R.load_scene(small_floor)
    cams = _group_walk_cams(small_floor)
    ids, off = R.select_cut(cams)
    ids2, off2 = R.select_cut_shared(cams, list(range(len(cams) + 1)), frustum=False)
    n = int(off[-1].item())
    assert torch.equal(off, off2) and torch.equal(ids[:n], ids2[:n])


@pytest.mark.parametrize("guard", [0.0, 32.0])
def test_frustum_cut_per_camera_blocked_equals_single_pass(R, small_floor, guard):
    """Frustum-culled cuts of groups of one camera: the camera-blocked
    two-pass kernel (four or more cameras) gives each camera the same ids as
    the single-pass kernel on that camera alone, and agrees with the oracle
    away from flagged decisions."""
    R.load_scene(small_floor)
    cams = _group_walk_cams(small_floor)
    n = len(cams)
    ids, off = R.select_cut_shared(cams, list(range(n + 1)), frustum=True, guard=guard)
    ids, off = ids.cpu().numpy(), off.cpu().numpy()
    for c in range(n):
        one, o1 = R.select_cut_shared([cams[c]], [0, 1], frustum=True, guard=guard)
        assert np.array_equal(ids[off[c]:off[c + 1]], one[: int(o1[1].item())].cpu().numpy())
    _compare_groups(torch.from_numpy(ids), torch.from_numpy(off), small_floor, cams,
                    list(range(n + 1)), True, guard)


def test_shared_cut_rejects_bad_groups_and_reports_capacity(R, small_floor):
    from paper_2603_15186_gb300 import NgsError
    R.load_scene(small_floor)
    cams = _group_walk_cams(small_floor)
    for gb in ([0, 5], [1, 10], [0, 4, 4, 10], [0, 6, 3, 10]):
        with pytest.raises(NgsError) as e:
            R.select_cut_shared(cams, gb)
        assert e.value.status == 1
    with pytest.raises(NgsError) as e:
        R.select_cut_shared(cams, [0, 10], guard=-1.0)
    assert e.value.status == 1
    with pytest.raises(NgsError) as e:
        R.select_cut_shared(cams, [0, 4, 10], cap=100)
    assert e.value.status == 4
    # the context survives: the next call succeeds and agrees with the oracle
    ids, off = R.select_cut_shared(cams, [0, 4, 10])
    _compare_groups(ids, off, small_floor, cams, [0, 4, 10], True, 0.0)


# ---------------------------------------------------------------------------
# full render
# ---------------------------------------------------------------------------

def _render_one(R, scene, cam, tile=(16, 16)):
    R.set_tile(*tile)
    img = R.render([cam])[0].cpu().numpy()
    return img


@pytest.mark.parametrize("tau", [0.0, 4.0])
def test_render_small_box_view(R, box10k, tau):
    """The 10k-leaf box scene seen by the 128x128 camera at (2, 2, 1.2)."""
    R.load_scene(box10k)
    cam = camera_c0(tau)
    ref = O.render(box10k, cam, tile=(16, 16))
    assert ref.near.sum() == 0
    R.set_node_ids(True)
    img = _render_one(R, box10k, cam)
    compare_image(img, ref)
    n_tiles = len(ref.ranges)
    rng, nodes = R.tile_lists(0, n_tiles, len(ref.keys) + 4096)
    compare_tile_lists(rng, nodes, ref, (16, 16))
    pairs, _, _ = compare_tile_order_f64(rng, nodes, box10k.pos, cam)
    assert pairs > 1000
    # without node ids the same render gives the same pixels, and the tile
    # lists report their ranges only
    R.set_node_ids(False)
    assert np.array_equal(_render_one(R, box10k, cam), img)
    rng2, _ = R.tile_ranges(0, n_tiles, len(ref.keys) + 4096)
    assert np.array_equal(rng2, rng)
    with pytest.raises(RuntimeError, match="INVALID_ARG"):
        R.tile_lists(0, n_tiles, len(ref.keys) + 4096)


def test_large_footprints_span_many_tiles_and_windows(R, box10k):
    """A close, long-focal camera on the box scene with 8x8 tiles: Gaussians
    cover up to hundreds of tiles, so a record's pairs spread over several
    pair chunks and a chunk can start inside a record; the tile lists and
    the image still match the oracle's."""
    R.load_scene(box10k)
    cam = look_camera((1.0, 2.0, 1.2), 0.0, 512, 384, fx=600.0, tau=0.0)
    ref = O.render(box10k, cam, tile=(8, 8))
    area = (ref.rect[:, 2] - ref.rect[:, 0] + 1) * (ref.rect[:, 3] - ref.rect[:, 1] + 1)
    assert area.max() > 2048          # one record holds more than a whole pair chunk
    R.set_node_ids(True)
    img = _render_one(R, box10k, cam, tile=(8, 8))
    compare_image(img, ref)
    n_tiles = len(ref.ranges)
    rng, nodes = R.tile_lists(0, n_tiles, len(ref.keys) + 4096)
    compare_tile_lists(rng, nodes, ref, (8, 8))
    R.set_node_ids(False)
    R.set_tile(16, 16)


def _floor_cams(scene):
    cams = walk_cameras(scene, 4, 77, 160, 120, fx=150.0, tau=0.0)
    cams[1].width, cams[1].height, cams[1].cx, cams[1].cy = 97, 61, 48.5, 30.5   # ragged tiles
    cams[1].tau = 2.0
    cams[2].width, cams[2].height, cams[2].cx, cams[2].cy = 320, 240, 160.0, 120.0
    cams[2].fx = cams[2].fy = 300.0
    cams[2].tau = 5.0
    cams[3].tau = 9.0
    return [clear_tau(scene, c) for c in cams]


def test_render_batch_matches_oracle_and_plain(R, small_floor):
    R.load_scene(small_floor)
    cams = _floor_cams(small_floor)
    R.set_tile(16, 16)
    R.set_mode("batched")
    imgs = [t.cpu().numpy() for t in R.render(cams)]
    for cam, img in zip(cams, imgs):
        ref = O.render(small_floor, cam)
        assert ref.near.sum() == 0
        compare_image(img, ref)
    # the plain per-view path computes the same bits
    R.set_mode("plain")
    plain = [t.cpu().numpy() for t in R.render(cams)]
    R.set_mode("batched")
    for a, b in zip(imgs, plain):
        assert np.array_equal(a, b)
    # tile lists of the last camera (plain mode leaves each camera's buffers in turn)
    R.set_mode("plain")
    R.set_node_ids(True)
    R.render([cams[2]])
    R.set_node_ids(False)
    ref = O.render(small_floor, cams[2])
    rng, nodes = R.tile_lists(0, len(ref.ranges), len(ref.keys) + 65536)
    compare_tile_lists(rng, nodes, ref, (16, 16))
    pairs, _, _ = compare_tile_order_f64(rng, nodes, small_floor.pos, cams[2])
    assert pairs > 1000
    R.set_mode("batched")


def test_composite_order_changes_no_pixel(R, small_floor):
    """Batched compositing in longest-list-first order and in tile order
    (several sub-batches of small tiles): the same bits, and the launch tail
    is measured in the longest-first form."""
    R.load_scene(small_floor)
    cams = _floor_cams(small_floor) * 3
    R.set_tile(8, 8)
    R.set_mode("batched")
    try:
        R.set_composite_order(True)
        a = [t.cpu().numpy() for t in R.render(cams)]
        st = R.stats()
        assert st["composite_tail_ms"] >= 0.0
        R.set_composite_order(False)
        b = [t.cpu().numpy() for t in R.render(cams)]
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    finally:
        R.set_composite_order(True)
        R.set_tile(16, 16)


def test_lod_blend_matches_oracle(R, small_floor):
    """Level-of-detail blending (each cut node moved toward its parent by its
    granularity position): images against the oracle's blended render, the
    same bits batched and plain and for another tile shape, tile lists
    against the oracle's, and at tau = 0 the plain render bit for bit."""
    R.load_scene(small_floor)
    cams = _floor_cams(small_floor)
    extra = walk_cameras(small_floor, 2, 78, 160, 120, fx=150.0, tau=20.0)[1]
    cams.append(clear_tau(small_floor, extra))
    R.set_tile(16, 16)
    R.set_mode("batched")
    plain_imgs = [t.cpu().numpy() for t in R.render(cams)]
    R.set_lod_blend(True)
    try:
        imgs = [t.cpu().numpy() for t in R.render(cams)]
        changed = 0
        for cam, img, pimg in zip(cams, imgs, plain_imgs):
            ref = O.render(small_floor, cam, blend=True)
            compare_image(img, ref)
            if cam.tau == 0.0:
                assert np.array_equal(img, pimg)
            else:
                changed += int(not np.array_equal(img, pimg))
        assert changed >= 2
        R.set_mode("plain")
        for a, b in zip(imgs, [t.cpu().numpy() for t in R.render(cams)]):
            assert np.array_equal(a, b)
        R.set_node_ids(True)
        R.render([cams[2]])
        R.set_node_ids(False)
        ref = O.render(small_floor, cams[2], blend=True)
        rng, nodes = R.tile_lists(0, len(ref.ranges), len(ref.keys) + 65536)
        compare_tile_lists(rng, nodes, ref, (16, 16))
        R.set_mode("batched")
        R.set_tile(32, 32)
        R.set_cta(16, 16)
        for a, b in zip(imgs, [t.cpu().numpy() for t in R.render(cams)]):
            assert np.array_equal(a, b)
    finally:
        R.set_lod_blend(False)
        R.set_mode("batched")
        R.set_tile(16, 16)
        R.set_cta(0, 0)


def test_pixels_independent_of_tile_shape_batch_and_graph(R, small_floor):
    R.load_scene(small_floor)
    cams = _floor_cams(small_floor)
    R.set_tile(16, 16)
    R.set_batch(128)
    base = [t.cpu().numpy() for t in R.render(cams)]
    again = [t.cpu().numpy() for t in R.render(cams)]   # replays the captured graph
    assert R.stats()["graph_replayed"] == 1
    for tile in [(8, 8), (16, 8), (16, 32), (32, 16), (32, 32)]:
        for batch in [64, 256]:
            R.set_tile(*tile)
            R.set_batch(batch)
            out = [t.cpu().numpy() for t in R.render(cams)]
            for a, b in zip(base, out):
                assert np.array_equal(a, b), (tile, batch)
    for a, b in zip(base, again):
        assert np.array_equal(a, b)
    # large binning tiles composited as smaller blocks, batched and plain
    for tile, cta in [((32, 32), (16, 16)), ((32, 32), (16, 8)), ((32, 16), (16, 16)),
                      ((16, 16), (8, 8)), ((16, 32), (16, 16))]:
        R.set_tile(*tile)
        R.set_cta(*cta)
        R.set_batch(128)
        for mode in ("batched", "plain"):
            R.set_mode(mode)
            out = [t.cpu().numpy() for t in R.render(cams)]
            st = R.stats()
            assert (st["cta_w"], st["cta_h"]) == cta
            for a, b in zip(base, out):
                assert np.array_equal(a, b), (tile, cta, mode)
        R.set_mode("batched")
    R.set_cta(0, 0)
    # alone vs in a batch
    R.set_tile(16, 16)
    R.set_batch(128)
    for i, cam in enumerate(cams):
        alone = R.render([cam])[0].cpu().numpy()
        assert np.array_equal(alone, base[i])


@pytest.mark.parametrize("blend", [False, True])
def test_block_cull_is_conservative(R, small_floor, box10k, blend):
    """Skipping node blocks that provably hold no visible Gaussian changes
    nothing: same visible Gaussians, same pairs, same image bits; with
    level-of-detail blending too (bounds over the nodes and their parents)."""
    extra = walk_cameras(small_floor, 2, 78, 160, 120, fx=150.0, tau=20.0)[1]
    for scene, cams in [(small_floor, _floor_cams(small_floor) + [extra]),
                        (box10k, [camera_c0(0.0), camera_c0(10.0),
                                  look_camera((-3.0, 2.0, 1.5), 0.3, 64, 48, fx=60.0, tau=6.0)])]:
        R.load_scene(scene)
        R.set_lod_blend(blend)
        outs, work = [], []
        for on in (True, False):
            R.set_block_cull(on)
            outs.append([t.cpu().numpy() for t in R.render(cams)])
            st = R.stats()
            work.append((st["visible_total"], st["pair_total"]))
        R.set_block_cull(True)
        R.set_lod_blend(False)
        assert work[0] == work[1]
        for a, b in zip(*outs):
            assert np.array_equal(a, b)


def test_planner_estimate_changes_sub_batches_not_pixels(small_floor):
    """The planner's pairs-per-pixel estimate decides how cameras are grouped
    into sub-batches (with a pair buffer of 2^22 slots, 48 pairs per pixel fit
    about 87k pixels per sub-batch, 4 fit about 1 Mpix); the images do not
    depend on it."""
    from paper_2603_15186_gb300 import Renderer
    r = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22, pair_capacity=1 << 22)
    r.load_scene(small_floor)
    cams = _floor_cams(small_floor)
    out, subs = [], []
    for ppp in (48, 4):
        r.set_pairs_per_pixel(ppp)
        out.append([t.cpu().numpy() for t in r.render(cams)])
        subs.append(r.stats()["sub_batches"])
    assert subs[0] > subs[1] >= 1, subs
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    from paper_2603_15186_gb300 import NgsError
    with pytest.raises(NgsError):
        r.set_pairs_per_pixel(0)
    r.close()


def test_autotune_keeps_pixels(R, small_floor):
    R.load_scene(small_floor)
    cams = _floor_cams(small_floor)
    R.set_tile(16, 16)
    R.set_batch(128)
    base = [t.cpu().numpy() for t in R.render(cams)]
    res = R.autotune(cams, reps=1)
    from paper_2603_15186_gb300 import _lib
    assert (res["tile"], res["cta"]) in _lib.TUNE_SHAPES
    assert res["batch"] in (64, 128, 256)
    assert all(v > 0 for v in res["ms"].values()) and len(res["ms"]) == 3 * len(_lib.TUNE_SHAPES)
    out = [t.cpu().numpy() for t in R.render(cams)]
    st = R.stats()
    assert (st["tile_w"], st["tile_h"], st["batch"]) == (*res["tile"], res["batch"])
    assert (st["cta_w"], st["cta_h"]) == res["cta"]
    for a, b in zip(base, out):
        assert np.array_equal(a, b)
    R.set_tile(16, 16)
    R.set_cta(0, 0)
    R.set_batch(128)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_slice_occupancy_matches_oracle(R, small_floor, dtype):
    """GS-slice occupancy of every leaf against the oracle: per plane and cell
    the largest capped slice value within 1e-3 (cells whose value sits at the
    1/255 cut-off on either side excepted, under 1% of them), and the
    occupancy mask equal away from the threshold."""
    from types import SimpleNamespace
    if dtype == "f32":
        R.load_scene(small_floor)
        ref_scene = small_floor
    else:
        stored, deq = quantize_attributes(small_floor, dtype)
        R.load_scene(small_floor, attr_dtype=dtype, stored=stored)
        ref_scene = O.SceneArrays(small_floor, overrides=deq)
    lo, hi = small_floor.aabb_min[0], small_floor.aabb_max[0]
    grid = SimpleNamespace(x0=float(lo[0]) - 0.013, y0=float(lo[1]) + 0.007, cell=0.04,
                           nx=int((hi[0] - lo[0]) / 0.04) + 2, ny=int((hi[1] - lo[1]) / 0.04) + 1,
                           z0=0.05, dz=0.1, nz=13, threshold=0.5)
    val, occ = R.slice_occupancy(grid)
    torch.cuda.synchronize()
    got, gocc = val.cpu().numpy().astype(np.float64), occ.cpu().numpy()
    want, wocc = O.slice_occupancy(ref_scene, grid)
    cut = 1.0 / 255.0 + 1e-3
    exempt = (np.minimum(got, want) <= cut) & (np.abs(got - want) > 1e-3)
    assert exempt.mean() < 0.01
    assert np.abs(got - want)[~exempt].max() <= 1e-3
    near = np.abs(want - grid.threshold) <= 1e-3
    assert np.array_equal(gocc[~near], wocc[~near])
    assert wocc.any() and (want > 0).mean() > 0.05
    # a grid beside the scene holds nothing; sizes are checked
    far = SimpleNamespace(**{**vars(grid), "x0": float(hi[0]) + 5.0, "nz": 1})
    v2, o2 = R.slice_occupancy(far)
    assert float(v2.max()) == 0.0 and int(o2.max()) == 0
    from paper_2603_15186_gb300 import NgsError
    with pytest.raises(NgsError):
        R.slice_occupancy(SimpleNamespace(**{**vars(grid), "nx": 0}))


def test_nav_fields_and_paths_match_oracle(R, small_floor):
    """Blocked map, breadth-first distance fields and agent paths on the GPU's
    slice occupancy of the small floor, bit for bit against the oracle on the
    same occupancy (integer results: no tolerance)."""
    from types import SimpleNamespace
    R.load_scene(small_floor)
    lo, hi = small_floor.aabb_min[0], small_floor.aabb_max[0]
    grid = SimpleNamespace(x0=float(lo[0]), y0=float(lo[1]), cell=0.05,
                           nx=int((hi[0] - lo[0]) / 0.05) + 1, ny=int((hi[1] - lo[1]) / 0.05) + 1,
                           z0=0.05, dz=0.1, nz=13, threshold=0.5)
    _, occ = R.slice_occupancy(grid)
    occ_h = occ.cpu().numpy()
    rng = np.random.default_rng(31)
    b_ref = O.nav_blocked(occ_h, 1, 9, 2)
    free = np.argwhere(b_ref == 0)
    goals = [tuple(int(v) for v in free[k][::-1]) for k in rng.choice(len(free), 5, replace=False)]
    goals.append((-1, 3))                                  # outside the grid: nothing reachable
    blocked, dist = R.nav_fields(occ, goals, 1, 9, 2)
    torch.cuda.synchronize()
    assert np.array_equal(blocked.cpu().numpy(), b_ref)
    dist_h = dist.cpu().numpy().view(np.uint32)
    refs = [O.nav_field(b_ref, g) for g in goals]
    for g in range(len(goals)):
        assert np.array_equal(dist_h[g], refs[g]), g
    assert np.all(dist_h[-1] == 0xFFFFFFFF) and (dist_h[0] < 0xFFFFFFFF).mean() > 0.3
    starts = [(int(rng.integers(grid.nx)), int(rng.integers(grid.ny)), int(rng.integers(len(goals))))
              for _ in range(200)]
    paths, lens = R.nav_paths(dist, starts, 600)
    paths, lens = paths.cpu().numpy(), lens.cpu().numpy()
    for a, (i, j, g) in enumerate(starts):
        ref = O.nav_path(refs[g], (i, j), 600)
        assert lens[a] == len(ref) and np.array_equal(paths[a, :lens[a]], ref), a
    assert (lens > 1).sum() > 50


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reduced_precision_attributes(R, small_floor, dtype):
    stored, deq = quantize_attributes(small_floor, dtype)
    R.load_scene(small_floor, attr_dtype=dtype, stored=stored)
    cams = _floor_cams(small_floor)[:2]
    imgs = [t.cpu().numpy() for t in R.render(cams)]
    sa = O.SceneArrays(small_floor, overrides=deq)
    for cam, img in zip(cams, imgs):
        ref = O.render(sa, cam)
        compare_image(img, ref)


def test_edge_cases(R, small_floor):
    R.load_scene(small_floor)
    base = walk_cameras(small_floor, 1, 5, 64, 48, fx=60.0, tau=0.0)[0]
    away = look_camera((-3.0, 3.0, 1.5), math.pi, 33, 17, fx=30.0)   # outside, facing away
    tiny = look_camera(base.pos, 1.0, 1, 1, fx=1.0)
    coarse = look_camera((-20.0, -20.0, 10.0), math.radians(40), 40, 30, fx=35.0, tau=1e30)
    cams = [base, away, tiny, coarse]
    imgs = [t.cpu().numpy() for t in R.render(cams)]
    for cam, img in zip(cams, imgs):
        ref = O.render(small_floor, cam)
        compare_image(img, ref)
    ids, off = R.select_cut([coarse])
    assert ids[: int(off[1].item())].cpu().tolist() == [0]


def test_capacity_error_is_reported_and_context_survives(small_floor):
    from paper_2603_15186_gb300 import NgsError, Renderer
    r = Renderer(device=0, cut_capacity=1 << 20, record_capacity=1 << 20, pair_capacity=1000)
    r.load_scene(small_floor)
    cam = walk_cameras(small_floor, 1, 5, 160, 120, fx=150.0, tau=0.0)[0]
    with pytest.raises(NgsError) as e:
        r.render([cam])
    assert e.value.status == 4
    r.close()
    r2 = Renderer(device=0, cut_capacity=1 << 20, record_capacity=1 << 20, pair_capacity=1 << 22)
    r2.load_scene(small_floor)
    img = r2.render([cam])[0].cpu().numpy()
    compare_image(img, O.render(small_floor, cam))
    r2.close()


def test_bounded_wait_times_out_and_context_survives(small_floor):
    """A device-side wait that can never be satisfied gives up by itself and
    reports NGS_ERR_DEVICE_TIMEOUT; no trap, no hang, and the same context then
    renders correctly."""
    import ctypes as C
    import time
    from paper_2603_15186_gb300 import Renderer
    r = Renderer(device=0, cut_capacity=1 << 20, record_capacity=1 << 20, pair_capacity=1 << 22)
    r.load_scene(small_floor)
    t = time.time()
    st = r.L.ngs_selftest_wait_timeout(r.h, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 6  # NGS_ERR_DEVICE_TIMEOUT
    assert time.time() - t < 30
    cam = walk_cameras(small_floor, 1, 5, 96, 72, fx=90.0, tau=0.0)[0]
    compare_image(r.render([cam])[0].cpu().numpy(), O.render(small_floor, cam))
    r.close()


def test_invalid_hierarchy_rejected(R, box10k):
    from paper_2603_15186_gb300 import NgsError
    import copy
    bad = copy.copy(box10k)
    bad.parent = box10k.parent.copy()
    bad.parent[5] = 7   # a child whose parent id is not smaller than its own
    with pytest.raises(NgsError) as e:
        R.load_scene(bad)
    assert e.value.status == 2


def test_unsupported_tile_shape_rejected(R, small_floor):
    from paper_2603_15186_gb300 import NgsError
    R.load_scene(small_floor)
    cam = walk_cameras(small_floor, 1, 5, 64, 48, fx=60.0, tau=0.0)[0]
    R.set_tile(8, 32)            # both dimensions are valid alone, the pair is not built
    with pytest.raises(NgsError) as e:
        R.render([cam])
    assert e.value.status == 1
    R.set_tile(16, 32)
    img = R.render([cam])[0].cpu().numpy()
    R.set_tile(16, 16)
    assert np.array_equal(img, R.render([cam])[0].cpu().numpy())
    # a compositing block that does not divide the tile
    R.set_cta(32, 16)
    with pytest.raises(NgsError) as e:
        R.render([cam])
    assert e.value.status == 1
    R.set_cta(0, 0)
    assert np.array_equal(img, R.render([cam])[0].cpu().numpy())
