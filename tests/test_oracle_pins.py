"""Pins of the float64 oracle against facts fixed outside it: hand-worked
values, closed forms, library routines (scipy rotations and spherical
harmonics, numpy sorting), invariants and brute force. CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from scenegen import Camera, build_hierarchy, camera_c0, look_camera, yaw_rotation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


class _Tree:
    """Minimal scene container for hand-made hierarchies."""

    def __init__(self, n, aabb_min, aabb_max, parent, child_count):
        self.pos = np.zeros((n, 3), np.float32)
        self.quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
        self.log_scale = np.full((n, 3), -3.0, np.float32)
        self.opacity = np.full(n, 0.5, np.float32)
        self.sh = np.zeros((n, 16, 3), np.float32)
        self.parent = np.asarray(parent, np.int32)
        self.child_count = np.asarray(child_count, np.int32)
        self.aabb_min = np.asarray(aabb_min, np.float32)
        self.aabb_max = np.asarray(aabb_max, np.float32)


def _scene_from_leaves(pos, quat=None, log_scale=None, opacity=None, sh=None):
    n = len(pos)
    pos = np.asarray(pos, np.float32)
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quat is None else np.asarray(quat, np.float32)
    log_scale = np.full((n, 3), -4.0, np.float32) if log_scale is None else np.asarray(log_scale, np.float32)
    opacity = np.full(n, 0.5, np.float32) if opacity is None else np.asarray(opacity, np.float32)
    if sh is None:
        sh = np.zeros((n, 16, 3), np.float32)
    return build_hierarchy(pos, quat, log_scale, opacity, np.asarray(sh, np.float32))


# ---------------------------------------------------------------------------
# scene generator (shared input)
# ---------------------------------------------------------------------------

def test_hierarchy_structure(box10k):
    s = box10k
    M = s.n_nodes
    assert s.parent[0] == -1 and np.all(s.parent[1:] >= 0)
    assert int((s.child_count == 0).sum()) == s.n_leaves == 10_000
    # breadth-first: parents precede children, children contiguous
    assert np.all(s.parent[1:] < np.arange(1, M))
    inner = np.flatnonzero(s.child_count > 0)
    for n in inner[:2000]:
        kids = np.arange(s.child_begin[n], s.child_begin[n] + s.child_count[n])
        assert np.all(s.parent[kids] == n)
    assert np.all(np.bincount(s.parent[1:], minlength=M) == s.child_count)
    # no single-child chains; at most 8 children below the deepest grid level
    assert s.child_count[inner].min() >= 2 and s.child_count[inner].max() <= 8
    assert np.all(np.diff(s.depth) >= 0)


def test_aabb_nesting(box10k):
    s = box10k
    c = np.arange(1, s.n_nodes)
    p = s.parent[c]
    assert np.all(s.aabb_min[c] >= s.aabb_min[p]) and np.all(s.aabb_max[c] <= s.aabb_max[p])
    # a parent box is exactly the union of its children's boxes
    inner = np.flatnonzero(s.child_count > 0)
    for n in inner[:500]:
        kids = slice(s.child_begin[n], s.child_begin[n] + s.child_count[n])
        assert np.array_equal(s.aabb_min[kids].min(0), s.aabb_min[n])
        assert np.array_equal(s.aabb_max[kids].max(0), s.aabb_max[n])


def test_moment_matching_matches_weighted_mixture():
    from scenegen import make_uniform_box_scene
    s = make_uniform_box_scene(3000, seed=5, keep_fp64=True)
    inner = np.flatnonzero(s.child_count > 0)
    for n in inner[:300]:
        kids = np.arange(s.child_begin[n], s.child_begin[n] + s.child_count[n])
        w = s.opacity64[kids]
        mu = s.mean64[kids]
        # mixture mean / covariance: weighted Sigma_i plus numpy's weighted
        # covariance of the child means
        mix_mu = np.average(mu, axis=0, weights=w)
        mix_cov = np.average(s.cov64[kids], axis=0, weights=w) + np.cov(mu.T, aweights=w, bias=True)
        np.testing.assert_allclose(s.mean64[n], mix_mu, rtol=0, atol=1e-12)
        np.testing.assert_allclose(s.cov64[n], mix_cov, rtol=1e-10, atol=1e-15)
    # the stored (quaternion, log-scale) of interior nodes reproduce Sigma_p to float32 precision
    sig = O.cov3d(s.quat[inner[:300]], s.log_scale[inner[:300]])
    np.testing.assert_allclose(sig, s.cov64[inner[:300]], rtol=2e-5, atol=1e-9)


# ---------------------------------------------------------------------------
# cut
# ---------------------------------------------------------------------------

def _golden_cut():
    with open(os.path.join(GOLDEN, "cut_two_leaf_tree.json")) as f:
        g = json.load(f)
    t = _Tree(3, g["aabb_min"], g["aabb_max"], g["parent"], g["child_count"])
    return g, t


def test_cut_hand_worked_tree():
    g, t = _golden_cut()
    for tau, want in g["cuts"].items():
        cam = Camera(pos=np.array(g["camera_pos"], np.float32), R_wc=np.eye(3, dtype=np.float32),
                     fx=g["fx"], fy=g["fx"], cx=8, cy=8, width=16, height=16, tau=float(tau))
        ids, near, s = O.select_cut(t, cam, with_s=True)
        assert ids.tolist() == want, tau
        np.testing.assert_array_equal(s, g["s"])
        if tau == "20":
            assert near.tolist() == g["near_at_tau_20"]
    cam = Camera(pos=np.array(g["camera_pos"], np.float32), R_wc=np.eye(3, dtype=np.float32),
                 fx=g["fx"], fy=g["fx"], cx=8, cy=8, width=16, height=16, tau=10.0)
    assert O.select_cut(t, cam)[1].tolist() == g["near_at_tau_10"]
    # camera inside the root box: s(root) = inf, the root is never taken
    cam.pos = np.array([0.5, 0.5, 0.5], np.float32)
    cam.tau = 1e30
    assert O.select_cut(t, cam)[0].tolist() == [1, 2]


def test_blend_weight_hand_worked_tree():
    """Parent weights of the level-of-detail blend on the hand-worked tree."""
    g, t = _golden_cut()
    for tau, want in g["blend_parent_weight"].items():
        cam = Camera(pos=np.array(g["camera_pos"], np.float32), R_wc=np.eye(3, dtype=np.float32),
                     fx=g["fx"], fy=g["fx"], cx=8, cy=8, width=16, height=16, tau=float(tau))
        got = [O.blend_gaussian(t, cam, n)[0] for n in range(3)]
        np.testing.assert_allclose(got, want, atol=1e-6, err_msg=tau)
    # camera inside the root box: s(parent) = inf, leaves are never blended
    cam = Camera(pos=np.array([0.5, 0.5, 0.5], np.float32), R_wc=np.eye(3, dtype=np.float32),
                 fx=g["fx"], fy=g["fx"], cx=8, cy=8, width=16, height=16, tau=15.0)
    assert [O.blend_gaussian(t, cam, n)[0] for n in range(3)] == [0.0, 0.0, 0.0]
    # the weight formula's edge cases
    assert O.blend_parent_weight(10.0, math.inf, 5.0) == 0.0
    assert O.blend_parent_weight(10.0, 10.0, 5.0) == 0.0      # s(p) <= s(n)
    assert O.blend_parent_weight(10.0, 20.0, 25.0) == 1.0     # tau beyond s(p): clamped


def test_blend_interpolates_attributes():
    """At parent weight v the rendered Gaussian is the node's attributes moved
    by v toward the parent's: mean (float32, one fused step), covariance from
    scipy's rotation, opacity and SH, each linear in v."""
    g, t = _golden_cut()
    rng = np.random.default_rng(12)
    t.pos = rng.normal(0.5, 0.3, (3, 3)).astype(np.float32)
    t.quat = rng.normal(size=(3, 4)).astype(np.float32)
    t.log_scale = rng.normal(-3.0, 0.5, (3, 3)).astype(np.float32)
    t.opacity = rng.uniform(0.1, 0.9, 3).astype(np.float32)
    t.sh = rng.normal(0, 0.3, (3, 16, 3)).astype(np.float32)

    def sigma(i):
        q = t.quat[i].astype(np.float64)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        return R @ np.diag(np.exp(2.0 * t.log_scale[i].astype(np.float64))) @ R.T

    for tau, want in g["blend_parent_weight"].items():
        cam = Camera(pos=np.array(g["camera_pos"], np.float32), R_wc=np.eye(3, dtype=np.float32),
                     fx=g["fx"], fy=g["fx"], cx=8, cy=8, width=16, height=16, tau=float(tau))
        for n in (1, 2):
            v, mu, S, op, sh = O.blend_gaussian(t, cam, n)
            assert abs(v - want[n]) <= 1e-6
            # float32 mean: the float32 difference, then one rounding of
            # v * difference + mean (the float64 product of two float32 values is
            # exact)
            diff = (t.pos[0] - t.pos[n]).astype(np.float32)
            mu_want = (np.float64(np.float32(v)) * diff.astype(np.float64) +
                       t.pos[n].astype(np.float64)).astype(np.float32)
            np.testing.assert_allclose(mu, mu_want, rtol=0, atol=1.2e-7)
            np.testing.assert_allclose(S, sigma(n) + v * (sigma(0) - sigma(n)), rtol=1e-12, atol=1e-15)
            assert op == pytest.approx(t.opacity[n] + v * (t.opacity[0] - t.opacity[n]), abs=1e-15)
            np.testing.assert_allclose(sh, t.sh[n] + v * (t.sh[0].astype(np.float64) - t.sh[n]),
                                       rtol=0, atol=1e-15)
        # without blending every node keeps its own attributes
        v, mu, S, op, sh = O.blend_gaussian(t, cam, 1, blend=False)
        assert v == 0.0 and np.array_equal(mu, t.pos[1]) and op == np.float64(t.opacity[1])
        np.testing.assert_allclose(S, sigma(1), rtol=1e-12, atol=1e-15)


def test_granularity_f32_close_to_float64(box10k):
    cam = camera_c0(4.0)
    _, _, s64 = O.select_cut(box10k, cam, with_s=True)
    sa = O.SceneArrays(box10k)
    for n in range(0, box10k.n_nodes, 97):
        s32 = O.granularity_f32(sa, cam, n)
        if math.isinf(s64[n]):
            assert math.isinf(s32)
        else:
            assert abs(s32 - s64[n]) <= 1e-6 * s64[n], n


def test_blend_at_tau_zero_is_the_plain_render(box10k):
    """At tau = 0 every cut node is a leaf finer than tau (parent weight 0),
    so the blended render is the plain one, bit for bit."""
    cam = camera_c0(0.0)
    a = O.render(box10k, cam)
    b = O.render(box10k, cam, blend=True)
    assert np.array_equal(a.image, b.image) and np.array_equal(a.vals, b.vals)
    c = O.render(box10k, camera_c0(10.0), blend=True)
    d = O.render(box10k, camera_c0(10.0))
    assert not np.array_equal(c.image, d.image)   # nodes in transition move toward parents


def _check_antichain_cover(s, ids):
    sel = np.zeros(s.n_nodes, bool)
    sel[ids] = True
    leaves = np.flatnonzero(s.child_count == 0)
    count = sel[leaves].astype(np.int64)
    anc = s.parent[leaves].astype(np.int64)
    while np.any(anc >= 0):
        a = anc >= 0
        count[a] += sel[anc[a]]
        anc[a] = s.parent[anc[a]]
    assert np.all(count == 1), "every leaf must have exactly one selected ancestor-or-self"
    # antichain: no selected node has a selected ancestor
    anc = s.parent[ids].astype(np.int64)
    while np.any(anc >= 0):
        a = anc >= 0
        assert not np.any(sel[anc[a]])
        anc[a] = s.parent[anc[a]]


@pytest.mark.parametrize("tau", [0.0, 4.0, 16.0, 40.0, 120.0])
def test_cut_invariants(box10k, tau):
    cam = camera_c0(tau)
    ids, near = O.select_cut(box10k, cam)
    assert np.all(np.diff(ids) > 0)
    _check_antichain_cover(box10k, ids)
    if tau == 0.0:
        assert np.array_equal(ids, np.flatnonzero(box10k.child_count == 0))


def test_cut_coarsens_with_tau(box10k):
    prev = None
    s = box10k
    for tau in [0.0, 8.0, 16.0, 32.0, 64.0, 1e30]:
        cam = look_camera((-3.0, 2.0, 1.5), 0.0, 64, 64, fx=60.0, tau=tau)
        ids, _ = O.select_cut(s, cam)
        if prev is not None:
            # every node of the finer cut has an ancestor-or-self in the coarser one
            sel = np.zeros(s.n_nodes, bool)
            sel[ids] = True
            cur = prev.astype(np.int64)
            hit = sel[cur].copy()
            while not hit.all():
                live = ~hit
                cur[live] = s.parent[cur[live]]
                assert np.all(cur[live] >= 0)
                hit[live] = sel[cur[live]]
            assert len(ids) <= len(prev)
        prev = ids
    assert prev.tolist() == [0]  # tau = inf, camera outside the root box: just the root


# ---------------------------------------------------------------------------
# frustum-culled and shared cuts
# ---------------------------------------------------------------------------

def _boxes(lo, hi):
    n = len(lo)
    return _Tree(n, lo, hi, [-1] * n, [0] * n)


def _camera_at_origin(R, guard_note=None):
    return Camera(pos=np.zeros(3, np.float32), R_wc=np.asarray(R, np.float32), fx=100.0,
                  fy=100.0, cx=50.0, cy=50.0, width=100, height=100, tau=0.0)


def test_frustum_hand_worked_boxes():
    """R = I, fx = fy = 100, cx = cy = 50, 100x100: the view volume is z >= 0.2,
    -z/2 <= x <= z/2, -z/2 <= y <= z/2 (worked by hand per box below); the same
    boxes rotated into the frame of a camera looking along +x give the same
    answers (camera x = -world y, camera y = -world z, camera z = world x)."""
    boxes = [  # lo, hi, culled at guard 0, culled at guard 400
        ((-1, -1, 4), (1, 1, 6), False, False),       # straight ahead
        ((-1, -1, -6), (1, 1, -4), True, True),       # behind the camera
        ((-10, -1, 4), (-5, 1, 6), True, False),      # left: 100(-5) + 50(6) < 0; corner u = -33.3
        ((-10, -1, 4), (-2, 1, 6), False, False),     # reaches in: corner (-2, ., 6) has u = 16.7
        ((5, -1, 4), (10, 1, 6), True, False),        # right: -100(5) + 50(6) < 0
        ((-1, 5, 4), (1, 10, 6), True, False),        # below the image: -100(5) + 50(6) < 0
        ((-1, -10, 4), (1, -5, 6), True, False),      # above the image
        ((-1, -1, -1), (1, 1, 0.1), True, True),      # in front of the camera but before z = 0.2
        ((-1, -1, -1), (1, 1, 0.3), False, False),    # crosses z = 0.2
    ]
    lo = np.array([b[0] for b in boxes], np.float32)
    hi = np.array([b[1] for b in boxes], np.float32)
    want0 = [b[2] for b in boxes]
    want400 = [b[3] for b in boxes]
    cam = _camera_at_origin(np.eye(3))
    c0, u0 = O.frustum_state(_boxes(lo, hi), cam, 0.0)
    c4, u4 = O.frustum_state(_boxes(lo, hi), cam, 400.0)
    assert c0.tolist() == want0 and c4.tolist() == want400
    assert not u0.any() and not u4.any()
    # camera looking along +x (yaw 0, level): t = (-y, -z, x); box (lo, hi) in
    # the camera frame becomes the world box below
    wlo = np.stack([lo[:, 2], -hi[:, 0], -hi[:, 1]], 1)
    whi = np.stack([hi[:, 2], -lo[:, 0], -lo[:, 1]], 1)
    camx = _camera_at_origin(yaw_rotation(0.0))
    cx, _ = O.frustum_state(_boxes(wlo, whi), camx, 0.0)
    assert cx.tolist() == want0
    # a box whose left-plane maximum is exactly 0 (100(-3) + 50(6)) is kept, and unsure
    c, u = O.frustum_state(_boxes([(-10, -1, 4)], [(-3, 1, 6)]), cam, 0.0)
    assert c.tolist() == [False] and u.tolist() == [True]


@pytest.mark.parametrize("guard", [0.0, 10.0])
def test_frustum_is_exact_for_an_axis_aligned_camera(guard):
    """With R = I the view volume's cross-section at depth z is the rectangle
    [(-g - cx) z / fx, (W + g - cx) z / fx] x [(-g - cy) z / fy, (H + g - cy) z / fy],
    which only grows with z: a box meets the volume iff the point of its far
    face (z = hi.z >= 0.2) closest to that rectangle's centre projects inside.
    The cull must be exactly that (off-centre principal point, W != H, fx != fy)."""
    rng = np.random.default_rng(11)
    cam = Camera(pos=np.zeros(3, np.float32), R_wc=np.eye(3, dtype=np.float32), fx=120.0,
                 fy=90.0, cx=70.0, cy=40.0, width=160, height=100, tau=0.0)
    c = rng.uniform([-8, -8, -2], [8, 8, 10], (4000, 3))
    h = rng.uniform(0.05, 2.0, (4000, 3))
    lo, hi = (c - h).astype(np.float32), (c + h).astype(np.float32)
    culled, unsure = O.frustum_state(_boxes(lo, hi), cam, guard)
    z = hi[:, 2].astype(np.float64)
    zz = np.maximum(z, 0.2)
    xc = ((-guard - cam.cx) + (cam.width + guard - cam.cx)) / 2 * zz / cam.fx
    yc = ((-guard - cam.cy) + (cam.height + guard - cam.cy)) / 2 * zz / cam.fy
    w = np.stack([np.clip(xc, lo[:, 0], hi[:, 0]), np.clip(yc, lo[:, 1], hi[:, 1]), z], 1)
    meets = _inside_view(cam, w, guard + 1e-9)
    assert np.array_equal(culled[~unsure], ~meets[~unsure])
    assert 0.2 < culled.mean() < 0.8 and unsure.sum() <= 2


def _inside_view(cam, pts, guard):
    t = (pts - cam.pos.astype(np.float64)) @ cam.R_wc.astype(np.float64).T
    ok = t[..., 2] >= 0.2
    z = np.where(ok, t[..., 2], 1.0)
    u = cam.fx * t[..., 0] / z + cam.cx
    v = cam.fy * t[..., 1] / z + cam.cy
    return ok & (u >= -guard) & (u <= cam.width + guard) & (v >= -guard) & (v <= cam.height + guard)


@pytest.mark.parametrize("guard", [0.0, 24.0])
def test_frustum_cull_agrees_with_projection(box10k, guard):
    """No sampled point (8 corners + 24 random points) of a culled box projects
    inside the view; a box with such a point is never culled. Culls nest down
    the tree."""
    s = box10k
    rng = np.random.default_rng(3)
    cams = [camera_c0(0.0), look_camera((-3.0, 2.0, 1.5), 0.3, 64, 48, fx=60.0),
            look_camera((2.0, 2.0, 1.5), 2.0, 80, 60, fx=50.0, pitch=-0.4),
            look_camera((6.0, -1.0, 4.0), 2.5, 96, 96, fx=90.0, pitch=-0.6)]
    lo = s.aabb_min.astype(np.float64)
    hi = s.aabb_max.astype(np.float64)
    corners = np.stack([np.stack([(hi if (k >> a) & 1 else lo)[:, a] for a in range(3)], 1)
                        for k in range(8)], 1)
    rand = lo[:, None] + rng.random((len(lo), 24, 3)) * (hi - lo)[:, None]
    pts = np.concatenate([corners, rand], 1)
    n_culled = []
    for cam in cams:
        culled, unsure = O.frustum_state(s, cam, guard)
        inside = _inside_view(cam, pts, guard).any(1)
        assert not np.any(culled & inside & ~unsure)
        assert unsure.sum() < 0.001 * len(culled)
        kids = np.arange(1, s.n_nodes)
        assert np.all(culled[kids] | ~culled[s.parent[kids]])
        n_culled.append(int(culled.sum()))
    assert min(n_culled) < s.n_nodes // 2 and max(n_culled) > s.n_nodes // 2, n_culled


def _leaf_paths(s):
    """[leaves, depth] node ids root first, padded with -1 after the leaf."""
    leaves = np.flatnonzero(s.child_count == 0)
    chains = [leaves.astype(np.int64)]
    while np.any(chains[-1] >= 0):
        prev = chains[-1]
        chains.append(np.where(prev >= 0, s.parent[np.maximum(prev, 0)], -1))
    chains = np.stack(chains[:-1], 1)[:, ::-1]          # root first, -1 padding in front
    out = np.full_like(chains, -1)
    for i, row in enumerate(chains):
        r = row[row >= 0]
        out[i, :len(r)] = r
    return out


def _group_cams():
    return [look_camera((0.5, 0.6, 1.2), 0.2, 64, 48, fx=60.0, tau=6.0),
            look_camera((1.2, 0.9, 1.2), 1.4, 64, 48, fx=60.0, tau=3.0),
            look_camera((2.5, 2.8, 1.4), -2.0, 96, 64, fx=80.0, tau=9.0),
            look_camera((3.2, 1.0, 0.9), 3.0, 48, 48, fx=40.0, tau=4.5)]


def test_shared_cut_of_one_camera_is_its_cut(box10k):
    for tau in [0.0, 5.0, 20.0]:
        cam = look_camera((-1.0, 1.0, 1.5), 0.4, 64, 48, fx=60.0, tau=tau)
        ids, _ = O.select_cut(box10k, cam)
        a, off, _ = O.select_cut_shared(box10k, [cam], [0, 1], frustum=False)
        assert np.array_equal(a, ids) and off.tolist() == [0, len(ids)]
        culled, _ = O.frustum_state(box10k, cam)
        b, _, _ = O.select_cut_shared(box10k, [cam], [0, 1], frustum=True)
        assert np.array_equal(b, ids[~culled[ids]])


@pytest.mark.parametrize("frustum", [False, True])
def test_shared_cut_is_the_deepest_member_choice_per_path(box10k, frustum):
    """Brute force over root-to-leaf paths: with c's own cut at depth n_c on a
    path and its first culled node at depth i_c (none: past the leaf), the
    group's cut holds the path's node at depth max_c min(i_c, n_c) when some
    member keeps that node, and nothing else on the path."""
    s = box10k
    cams = _group_cams()
    paths = _leaf_paths(s)
    depth = (paths >= 0).sum(1)
    gb = [0, 1, len(cams)]       # a single camera, then three together
    ids, off, near = O.select_cut_shared(s, cams, gb, frustum=frustum)
    for g in range(len(gb) - 1):
        members = cams[gb[g]:gb[g + 1]]
        sel = np.zeros(s.n_nodes, bool)
        sel[ids[off[g]:off[g + 1]]] = True
        D = np.zeros(len(paths), np.int64)
        kept_any = np.zeros(s.n_nodes, bool)
        for cam in members:
            own = np.zeros(s.n_nodes, bool)
            own[O.select_cut(s, cam)[0]] = True
            culled = O.frustum_state(s, cam)[0] if frustum else np.zeros(s.n_nodes, bool)
            kept_any |= ~culled
            on = np.where(paths >= 0, own[np.maximum(paths, 0)], False)
            assert np.all(on.sum(1) == 1)
            n_c = on.argmax(1)
            cu = np.where(paths >= 0, culled[np.maximum(paths, 0)], False)
            i_c = np.where(cu.any(1), cu.argmax(1), depth)
            D = np.maximum(D, np.minimum(i_c, n_c))
        rows = np.arange(len(paths))
        at = paths[rows, D]
        want = np.zeros_like(paths, dtype=bool)
        want[rows, D] = kept_any[at]
        got = np.where(paths >= 0, sel[np.maximum(paths, 0)], False)
        clean = ~np.where(paths >= 0, near[g][np.maximum(paths, 0)], False).any(1)
        assert clean.mean() > 0.97
        assert np.array_equal(got[clean], want[clean])
        if frustum:
            assert np.all(kept_any[ids[off[g]:off[g + 1]]])


def test_shared_cut_covers_what_members_see(box10k):
    """Antichain, and every leaf some member keeps has exactly one selected
    ancestor-or-self; a finer member's tau makes the shared cut at least as
    fine as its own."""
    s = box10k
    cams = _group_cams()
    ids, off, _ = O.select_cut_shared(s, cams, [0, len(cams)], frustum=True)
    sel = np.zeros(s.n_nodes, bool)
    sel[ids] = True
    kept = np.zeros(s.n_nodes, bool)
    for cam in cams:
        kept |= ~O.frustum_state(s, cam)[0]
    leaves = np.flatnonzero((s.child_count == 0) & kept)
    count = sel[leaves].astype(np.int64)
    anc = s.parent[leaves].astype(np.int64)
    while np.any(anc >= 0):
        a = anc >= 0
        count[a] += sel[anc[a]]
        anc[a] = s.parent[anc[a]]
    assert len(leaves) > 0 and np.all(count == 1)
    anc = s.parent[ids].astype(np.int64)
    while np.any(anc >= 0):
        a = anc >= 0
        assert not np.any(sel[anc[a]])
        anc[a] = s.parent[anc[a]]
    # unculled, all four cameras' cuts are coarser than or equal to the shared one
    full, _, _ = O.select_cut_shared(s, cams, [0, len(cams)], frustum=False)
    fsel = np.zeros(s.n_nodes, bool)
    fsel[full] = True
    for cam in cams:
        own, _ = O.select_cut(s, cam)
        for n in own[:: max(1, len(own) // 500)]:
            # n or one of its ancestors is selected, or n has selected descendants
            a, hit = int(n), False
            while a >= 0 and not hit:
                hit = fsel[a]
                a = int(s.parent[a])
            assert not hit or fsel[n], "the shared cut must not be coarser than a member's"


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------

def test_cov3d_matches_scipy_rotation():
    rng = np.random.default_rng(3)
    q = rng.normal(size=(50, 4)).astype(np.float32)
    s = rng.normal(-2, 0.5, size=(50, 3)).astype(np.float32)
    got = O.cov3d(q, s)
    qn = q.astype(np.float64) / np.linalg.norm(q.astype(np.float64), axis=1, keepdims=True)
    R = Rotation.from_quat(np.concatenate([qn[:, 1:], qn[:, :1]], 1)).as_matrix()
    want = np.einsum("nij,nj,nkj->nik", R, np.exp(2 * s.astype(np.float64)), R)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(O.cov3d(-q, s), got, rtol=1e-13, atol=1e-16)


def test_sigma2d_closed_form_on_axis():
    cam = camera_c0(0.0)  # at (2, 2, 1.2) looking +x, fx = fy = 120
    z = 1.5
    ls = np.log(np.array([0.02, 0.05, 0.03], np.float32))
    sc = _scene_from_leaves([[2.0 + z, 2.0, 1.2]], log_scale=[ls], opacity=[0.9])
    pre, key, rect = O.preprocess(sc, cam, np.array([0], np.int32))
    sx, sy, sz = np.exp(ls.astype(np.float64))
    # camera x = -world y, camera y = -world z, camera z = world x
    want_a = cam.fx ** 2 * sy ** 2 / z ** 2 + 0.3
    want_c = cam.fy ** 2 * sz ** 2 / z ** 2 + 0.3
    assert pre[0, O.PC.VISIBLE] == 1
    np.testing.assert_allclose(pre[0, O.PC.COV_A], want_a, rtol=1e-12)
    np.testing.assert_allclose(pre[0, O.PC.COV_C], want_c, rtol=1e-12)
    assert abs(pre[0, O.PC.COV_B]) < 1e-12
    np.testing.assert_allclose([pre[0, O.PC.U], pre[0, O.PC.V]], [64.0, 64.0], atol=1e-12)
    np.testing.assert_allclose(pre[0, O.PC.DEPTH], z, rtol=1e-12)


def _pixel_of_world(cam, x):
    R = cam.R_wc.astype(np.float64)
    t = R @ (np.asarray(x, np.float64) - cam.pos.astype(np.float64))
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


def test_sigma2d_equals_linearised_projection():
    """Sigma2D - 0.3 I equals Jw Sigma Jw^T with Jw the finite-difference
    Jacobian of the world -> pixel map (the EWA local affine approximation)."""
    rng = np.random.default_rng(7)
    for trial in range(20):
        cam = look_camera(rng.uniform(-1, 1, 3), rng.uniform(-3, 3), 96, 72, fx=80.0 + 40 * trial,
                          pitch=rng.uniform(-0.4, 0.4))
        fwd = cam.R_wc[2].astype(np.float64)
        mu = cam.pos + fwd * rng.uniform(1, 4) + rng.normal(0, 0.3, 3)
        q = rng.normal(size=4)
        ls = rng.normal(-2.5, 0.4, 3)
        sc = _scene_from_leaves([mu], quat=[q], log_scale=[ls], opacity=[0.7])
        pre, _, _ = O.preprocess(sc, cam, np.array([0], np.int32))
        if pre[0, O.PC.VISIBLE] == 0:
            continue
        mu32 = sc.pos[0].astype(np.float64)
        h = 1e-6
        J = np.stack([(_pixel_of_world(cam, mu32 + h * e) - _pixel_of_world(cam, mu32 - h * e)) / (2 * h)
                      for e in np.eye(3)], axis=1)
        S = O.cov3d(sc.quat[0], sc.log_scale[0])[0]
        want = J @ S @ J.T
        got = np.array([[pre[0, O.PC.COV_A], pre[0, O.PC.COV_B]],
                        [pre[0, O.PC.COV_B], pre[0, O.PC.COV_C]]]) - 0.3 * np.eye(2)
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=1e-6 * np.abs(want).max())
        np.testing.assert_allclose([pre[0, O.PC.U], pre[0, O.PC.V]], _pixel_of_world(cam, mu32),
                                   rtol=0, atol=1e-9)


# ---------------------------------------------------------------------------
# spherical harmonics
# ---------------------------------------------------------------------------

def test_sh_basis_matches_scipy():
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(1)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = O.sh_basis(d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)  # complex, Condon-Shortley phase included
            if m > 0:
                want = math.sqrt(2) * Y.real
            elif m < 0:
                want = math.sqrt(2) * Y.imag
            else:
                want = Y.real
            np.testing.assert_allclose(got[:, l * l + l + m], want, atol=1e-12, err_msg=f"l={l} m={m}")


def test_sh_basis_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates these polynomials exactly
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    Y = O.sh_basis(dirs)
    G = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_dc_only_colour_is_view_independent():
    rng = np.random.default_rng(2)
    cam = camera_c0(0.0)
    pts = np.array([[3.0, 2.0, 1.2], [3.5, 1.6, 1.0], [2.8, 2.3, 1.5]], np.float32)
    sh = np.zeros((3, 16, 3), np.float32)
    sh[:, 0, :] = rng.normal(0, 0.5, (3, 3))
    sc = _scene_from_leaves(pts, sh=sh, opacity=[0.6, 0.6, 0.6])
    ids, _ = O.select_cut(sc, cam)
    pre, _, _ = O.preprocess(sc, cam, ids)
    C0 = 0.5 / math.sqrt(math.pi)
    for row, g in zip(pre, ids):
        want = np.maximum(0.0, C0 * sc.sh[g, 0].astype(np.float64) + 0.5)
        np.testing.assert_allclose(row[[O.PC.R, O.PC.G, O.PC.B]], want, atol=1e-15)


# ---------------------------------------------------------------------------
# compositing
# ---------------------------------------------------------------------------

def _aim_camera():
    """A rotated camera (yaw 30 deg, pitch 10 deg) so that a transposed rotation
    or a swapped axis moves the projected point."""
    return look_camera((0.3, -0.2, 1.1), math.radians(30), 32, 24, fx=100.0, pitch=math.radians(10))


def _world_at_pixel(cam, i, j, depth):
    t = np.array([(i + 0.5 - cam.cx) * depth / cam.fx, (j + 0.5 - cam.cy) * depth / cam.fy, depth])
    return cam.pos.astype(np.float64) + cam.R_wc.astype(np.float64).T @ t


def _dc_for_colour(c):
    C0 = 0.5 / math.sqrt(math.pi)
    sh = np.zeros((16, 3), np.float32)
    sh[0] = (np.asarray(c) - 0.5) / C0
    return sh


def test_lone_gaussian_centre_pixel_is_o_times_c():
    cam = _aim_camera()
    mu = _world_at_pixel(cam, 20, 9, 2.0)
    sc = _scene_from_leaves([mu], log_scale=[np.log([0.01, 0.01, 0.01])], opacity=[0.7],
                            sh=[_dc_for_colour([0.8, 0.3, 0.55])])
    r = O.render(sc, cam, tile=(8, 8))
    C0 = 0.5 / math.sqrt(math.pi)
    c = C0 * sc.sh[0, 0].astype(np.float64) + 0.5
    o = float(sc.opacity[0])
    np.testing.assert_allclose(r.image[:, 9, 20], o * c, rtol=1e-9)
    lum = r.image.sum(0)
    assert np.unravel_index(np.argmax(lum), lum.shape) == (9, 20)
    assert lum[9, 19] < 0.6 * lum[9, 20]


def test_two_gaussians_on_one_ray_front_first():
    cam = _aim_camera()
    near_mu, far_mu = _world_at_pixel(cam, 12, 12, 1.5), _world_at_pixel(cam, 12, 12, 3.0)
    c1, c2 = [0.9, 0.2, 0.1], [0.1, 0.4, 0.95]
    sc = _scene_from_leaves([far_mu, near_mu], log_scale=[np.log([0.01] * 3)] * 2,
                            opacity=[0.6, 0.45], sh=[_dc_for_colour(c2), _dc_for_colour(c1)])
    r = O.render(sc, cam)
    C0 = 0.5 / math.sqrt(math.pi)
    col = C0 * sc.sh[:, 0].astype(np.float64) + 0.5
    o = sc.opacity.astype(np.float64)
    # node order from the octree is unknown; identify front/back by depth
    front = int(np.argmin(r.pre[:, O.PC.DEPTH]))
    back = 1 - front
    gid = r.ids
    want = o[gid[front]] * col[gid[front]] + (1 - o[gid[front]]) * o[gid[back]] * col[gid[back]]
    np.testing.assert_allclose(r.image[:, 12, 12], want, rtol=1e-8)


def test_opacity_clamps_at_099():
    cam = _aim_camera()
    mu = _world_at_pixel(cam, 5, 5, 2.0)
    sc = _scene_from_leaves([mu], log_scale=[np.log([0.01] * 3)], opacity=[0.9990],
                            sh=[_dc_for_colour([0.5, 0.6, 0.7])])
    r = O.render(sc, cam)
    C0 = 0.5 / math.sqrt(math.pi)
    c = C0 * sc.sh[0, 0].astype(np.float64) + 0.5
    np.testing.assert_allclose(r.image[:, 5, 5], 0.99 * c, rtol=1e-9)


def test_alpha_08_stack_stops_after_five_layers():
    """T after k layers of alpha 0.8 is 0.2^k; the 6th would bring T to
    6.4e-5 < 1e-4, so it and every later layer are dropped."""
    cam = _aim_camera()
    n = 8
    mus = [_world_at_pixel(cam, 16, 12, 1.0 + 0.25 * k) for k in range(n)]
    rng = np.random.default_rng(4)
    cols = rng.uniform(0.1, 0.9, (n, 3))
    sc = _scene_from_leaves(mus, log_scale=[np.log([0.005] * 3)] * n, opacity=[0.8] * n,
                            sh=[_dc_for_colour(c) for c in cols])
    r = O.render(sc, cam)
    C0 = 0.5 / math.sqrt(math.pi)
    gid = r.ids[np.argsort(r.pre[:, O.PC.DEPTH])]
    col = C0 * sc.sh[gid, 0].astype(np.float64) + 0.5
    a = float(np.float32(0.8))
    want = sum(a * (1 - a) ** k * col[k] for k in range(5))
    np.testing.assert_allclose(r.image[:, 12, 16], want, rtol=1e-7)


def test_nothing_visible_is_black():
    cam = _aim_camera()
    behind = cam.pos - 2.0 * cam.R_wc[2]
    sc = _scene_from_leaves([behind, behind + 0.1], opacity=[0.9, 0.9])
    r = O.render(sc, cam)
    assert len(r.keys) == 0 and np.all(r.image == 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bruteforce_equals_tiled(seed):
    rng = np.random.default_rng(100 + seed)
    n = 200
    cam = look_camera((0.0, 0.0, 0.0), 0.0, 32, 32, fx=30.0)
    pos = np.stack([rng.uniform(0.5, 3, n), rng.uniform(-1.5, 1.5, n), rng.uniform(-1.5, 1.5, n)], 1)
    q = rng.normal(size=(n, 4))
    ls = rng.normal(-2.2, 0.5, (n, 3))
    op = 1 / (1 + np.exp(-rng.normal(0, 1.5, n)))
    sh = rng.normal(0, 0.05, (n, 16, 3))
    sh[:, 0] = rng.normal(0, 0.5, (n, 3))
    sc = _scene_from_leaves(pos, quat=q, log_scale=ls, opacity=op, sh=sh)
    for tile in [(16, 16), (8, 8), (16, 8)]:
        r = O.render(sc, cam, tile=tile)
        bf, fl = O.render_bruteforce(r.pre, r.key, cam=cam)
        assert np.array_equal(bf.reshape(32, 32, 3).transpose(2, 0, 1), r.image)
        assert np.array_equal(fl.reshape(32, 32), r.flags)


def test_binning_sort_matches_numpy_stable_sort(small_floor):
    from scenegen import walk_cameras
    cam = walk_cameras(small_floor, 1, 7, 160, 120, tau=0.0)[0]
    ids, _ = O.select_cut(small_floor, cam)
    pre, key, rect = O.preprocess(small_floor, cam, ids, (16, 16))
    keys, vals, ranges = O.bin_pairs(rect, key, cam, (16, 16))
    tx, ty = O.tiles_xy(cam, (16, 16))
    # pairs rebuilt from the rectangles; ordered by numpy's stable sort
    rk, rv = [], []
    for i in np.flatnonzero(pre[:, O.PC.VISIBLE] > 0):
        x0, y0, x1, y1 = rect[i]
        for y in range(y0, y1 + 1):
            for x in range(x0, x1 + 1):
                rk.append((np.uint64(y * tx + x) << np.uint64(32)) | np.uint64(key[i]))
                rv.append(i)
    rk, rv = np.array(rk, np.uint64), np.array(rv, np.uint32)
    o = np.argsort(rk, kind="stable")
    assert np.array_equal(keys, rk[o]) and np.array_equal(vals, rv[o])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    cnt = np.bincount(tiles, minlength=tx * ty)
    assert np.array_equal(ranges[:, 1] - ranges[:, 0], cnt)
    assert len(keys) > 1000


# ---------------------------------------------------------------------------
# GS-slice occupancy (Sec. III-C)
# ---------------------------------------------------------------------------

def _sigma_scipy(quat, log_scale):
    q = np.asarray(quat, np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return R @ np.diag(np.exp(2.0 * np.asarray(log_scale, np.float64))) @ R.T


def test_slice_axis_aligned_closed_form():
    """An axis-aligned Gaussian slices without shift (alpha = beta = 0), with
    lambda = 1 / sigma_z^2 and C = diag(1 / sigma_x^2, 1 / sigma_y^2)."""
    ls = np.array([-3.0, -2.5, -2.0], np.float32)
    p = O.slice_params([1, 0, 0, 0], ls)
    s2 = np.exp(2.0 * ls.astype(np.float64))
    np.testing.assert_allclose(p[:2], [0.0, 0.0], atol=1e-9)
    np.testing.assert_allclose(p[2], 1.0 / s2[2], rtol=1e-12)
    np.testing.assert_allclose(p[3:6], [1.0 / s2[0], 0.0, 1.0 / s2[1]], rtol=1e-12, atol=1e-9)


def test_slice_is_the_3d_gaussian_on_the_plane():
    """The slice identity: o G2D((x, y), z) = o G3D((x, y, z)) for any point;
    lambda is the Schur complement 1 / Sigma_zz and mu(z) the conditional mean
    mu_xy + Sigma_xy,z (z - mu_z) / Sigma_zz (Sigma from scipy's rotation)."""
    rng = np.random.default_rng(21)
    n = 40
    t = _Tree(n, np.zeros((n, 3)), np.ones((n, 3)), [-1] + [0] * (n - 1), [n - 1] + [0] * (n - 1))
    t.pos = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    t.quat = rng.normal(size=(n, 4)).astype(np.float32)
    t.log_scale = rng.normal(-3.0, 0.6, (n, 3)).astype(np.float32)
    t.opacity = rng.uniform(0.05, 0.95, n).astype(np.float32)
    for g in range(n):
        S = _sigma_scipy(t.quat[g], t.log_scale[g])
        Si = np.linalg.inv(S)
        p = O.slice_params(t.quat[g], t.log_scale[g])
        assert p[2] == pytest.approx(1.0 / S[2, 2], rel=1e-9)
        np.testing.assert_allclose(p[:2], -S[:2, 2] / S[2, 2], rtol=1e-9, atol=1e-12)
        for _ in range(5):
            x = t.pos[g].astype(np.float64) + rng.normal(0, 0.05, 3)
            d = x - t.pos[g]
            want = float(t.opacity[g]) * math.exp(-0.5 * d @ Si @ d)
            got = O.slice_value(t, g, x[0], x[1], x[2])
            assert got == pytest.approx(want, rel=1e-9, abs=1e-300)


def test_slice_occupancy_against_brute_force():
    """Per plane and cell, the oracle's occupancy value equals the brute-force
    maximum over every leaf of min(0.99, o G3D) (values below 1/255 dropped),
    with G3D from scipy's covariance; the mask is value >= threshold."""
    from types import SimpleNamespace
    rng = np.random.default_rng(5)
    pos = np.column_stack([rng.uniform(0, 1.0, 60), rng.uniform(0, 0.8, 60),
                           rng.uniform(0, 0.6, 60)])
    s = _scene_from_leaves(pos, quat=rng.normal(size=(60, 4)),
                           log_scale=rng.normal(-2.8, 0.4, (60, 3)),
                           opacity=rng.uniform(0.02, 0.99, 60))
    grid = SimpleNamespace(x0=-0.05, y0=0.02, cell=0.04, nx=29, ny=21, z0=0.03, dz=0.1, nz=6,
                           threshold=0.3)
    val, occ = O.slice_occupancy(s, grid)
    leaves = np.flatnonzero(s.child_count == 0)
    xs = grid.x0 + (np.arange(grid.nx) + 0.5) * grid.cell
    ys = grid.y0 + (np.arange(grid.ny) + 0.5) * grid.cell
    X, Y = np.meshgrid(xs, ys)
    for k in range(grid.nz):
        z = grid.z0 + k * grid.dz
        want = np.zeros((grid.ny, grid.nx))
        for g in leaves:
            Si = np.linalg.inv(_sigma_scipy(s.quat[g], s.log_scale[g]))
            mu = s.pos[g].astype(np.float64)
            d = np.stack([X - mu[0], Y - mu[1], np.full_like(X, z - mu[2])], -1)
            a = np.float64(s.opacity[g]) * np.exp(-0.5 * np.einsum("...i,ij,...j->...", d, Si, d))
            a = np.where(a >= 1.0 / 255.0, np.minimum(a, 0.99), 0.0)
            want = np.maximum(want, a)
        np.testing.assert_allclose(val[k], want, rtol=1e-9, atol=1e-12)
        assert np.array_equal(occ[k], (val[k] >= grid.threshold).astype(np.uint8))
    assert (val > 0).mean() > 0.2 and occ.any()


# ---------------------------------------------------------------------------
# navigable map, distance fields, shortest paths
# ---------------------------------------------------------------------------

def test_nav_hand_worked_detour():
    with open(os.path.join(GOLDEN, "nav_detour_grid.json")) as f:
        g = json.load(f)
    b = np.array(g["blocked"], np.uint8)
    d = O.nav_field(b, g["goal"]).astype(np.int64)
    d[d == 0xFFFFFFFF] = -1
    assert d.tolist() == g["dist"]
    assert O.nav_path(O.nav_field(b, g["goal"]), g["path_from"], 64).tolist() == g["path"]


def test_nav_field_free_grid_is_manhattan_and_matches_scipy():
    """Without obstacles the field is the Manhattan distance; with random
    obstacles it equals scipy's unweighted shortest paths on the grid graph."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import shortest_path
    ny, nx = 23, 31
    d = O.nav_field(np.zeros((ny, nx), np.uint8), (7, 11)).astype(np.int64)
    jj, ii = np.mgrid[0:ny, 0:nx]
    assert np.array_equal(d, np.abs(ii - 7) + np.abs(jj - 11))
    rng = np.random.default_rng(8)
    b = (rng.random((ny, nx)) < 0.28).astype(np.uint8)
    b[11, 7] = 0
    idx = np.arange(ny * nx).reshape(ny, nx)
    rows, cols = [], []
    for (dj, di) in ((0, 1), (1, 0)):
        a = idx[: ny - dj, : nx - di]
        c = idx[dj:, di:]
        ok = (b[: ny - dj, : nx - di] == 0) & (b[dj:, di:] == 0)
        rows += list(a[ok]); cols += list(c[ok])
    G = coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(ny * nx, ny * nx))
    ref = shortest_path(G, directed=False, unweighted=True, indices=idx[11, 7])
    got = O.nav_field(b, (7, 11)).astype(np.float64).ravel()
    got[got == 0xFFFFFFFF] = np.inf
    ref[b.ravel() == 1] = np.inf
    assert np.array_equal(got, ref)


def test_nav_paths_descend_the_field():
    rng = np.random.default_rng(9)
    b = (rng.random((40, 50)) < 0.2).astype(np.uint8)
    b[20, 25] = 0
    d = O.nav_field(b, (25, 20))
    for _ in range(30):
        s = (int(rng.integers(50)), int(rng.integers(40)))
        p = O.nav_path(d, s, 500)
        if d[s[1], s[0]] == 0xFFFFFFFF:
            assert len(p) == 0
            continue
        assert len(p) == int(d[s[1], s[0]]) + 1 and tuple(p[0]) == s and tuple(p[-1]) == (25, 20)
        steps = np.abs(np.diff(p, axis=0)).sum(1)
        assert np.all(steps == 1) and not b[p[:, 1], p[:, 0]].any()
        assert np.array_equal(d[p[:, 1], p[:, 0]], np.arange(len(p))[::-1])


def test_nav_blocked_against_numpy_dilation():
    from scipy.ndimage import binary_dilation
    rng = np.random.default_rng(10)
    occ = (rng.random((6, 30, 40)) < 0.02).astype(np.uint8)
    got = O.nav_blocked(occ, 1, 4, 2)
    want = binary_dilation(occ[1:5].any(0), structure=np.ones((5, 5), bool))
    assert np.array_equal(got.astype(bool), want)
