"""Synthetic hierarchical Gaussian scenes.

A scene is a set of leaf Gaussians (position, rotation quaternion, per-axis
log-scale, opacity, degree-3 SH colour coefficients) organised in a tree whose
leaves are the fine Gaussians and whose interior nodes are coarser aggregates
of them (the hierarchical 3DGS representation of Sec. III-B). The tree built
here is an 8-ary octree over the leaf positions: a cell holding more than 8
leaves is split into its non-empty octants, a cell holding 2..8 leaves becomes
a node whose children are those leaves, and single-child chains are collapsed.
Every interior node carries a Gaussian moment-matched to its children with
opacity weights, and an axis-aligned box that is the union of its children's
boxes (a leaf's box is its mean +- 3 standard deviations per axis), so boxes
nest from the root down.

Node ids are breadth-first: the root is 0 and the children of every node are
contiguous. All stored attributes are float32 (the renderer's input precision);
the moment matching itself is done in float64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Optional

import numpy as np
from scipy.spatial.transform import Rotation

MORTON_BITS = 21  # bits per axis of the octree quantisation grid (63-bit codes)


@dataclass
class Camera:
    """Pinhole camera in the OpenCV frame (x right, y down, z forward).

    ``R_wc`` maps world directions to camera directions: t = R_wc (x - pos).
    """
    pos: np.ndarray          # (3,) float32
    R_wc: np.ndarray         # (3,3) float32, rows = camera axes in world coordinates
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    tau: float               # cut granularity in pixels

    @property
    def pixels(self) -> int:
        return int(self.width) * int(self.height)


@dataclass
class Scene:
    pos: np.ndarray          # (M,3) float32 means
    quat: np.ndarray         # (M,4) float32 (w,x,y,z), unit norm
    log_scale: np.ndarray    # (M,3) float32 natural log of per-axis std
    opacity: np.ndarray      # (M,)  float32 in (0,1)
    sh: np.ndarray           # (M,16,3) float32 SH coefficients, coefficient-major
    parent: np.ndarray       # (M,)  int32, -1 for the root
    child_begin: np.ndarray  # (M,)  int32, -1 for leaves
    child_count: np.ndarray  # (M,)  int32, 0 for leaves
    aabb_min: np.ndarray     # (M,3) float32
    aabb_max: np.ndarray     # (M,3) float32
    n_leaves: int
    depth: np.ndarray = field(default=None)          # (M,) int32 tree depth (root 0)
    cov64: Optional[np.ndarray] = field(default=None)  # (M,3,3) float64 matched covariances
    mean64: Optional[np.ndarray] = field(default=None)  # (M,3) float64 matched means
    opacity64: Optional[np.ndarray] = field(default=None)  # (M,) float64 matched opacities
    meta: Dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.parent.shape[0])

    def leaf_mask(self) -> np.ndarray:
        return self.child_count == 0

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.pos, self.quat, self.log_scale, self.opacity,
                                      self.sh, self.parent, self.child_begin,
                                      self.child_count, self.aabb_min, self.aabb_max))


# ---------------------------------------------------------------------------
# leaf attribute distributions
# ---------------------------------------------------------------------------

def _leaf_attributes(rng: np.random.Generator, n: int):
    """log-scales ~ N(-3.5, 0.5) per axis, uniform unit quaternions, opacity =
    sigmoid(N(0, 1.5)), SH DC ~ N(0, 0.5) and bands 1..3 ~ N(0, 0.05)."""
    log_scale = rng.normal(-3.5, 0.5, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, size=n)))
    sh = np.empty((n, 16, 3))
    sh[:, 0, :] = rng.normal(0.0, 0.5, size=(n, 3))
    sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, 15, 3))
    return (q.astype(np.float32), log_scale.astype(np.float32),
            opacity.astype(np.float32), sh.astype(np.float32))


# ---------------------------------------------------------------------------
# octree construction
# ---------------------------------------------------------------------------

def _spread_bits(v: np.ndarray) -> np.ndarray:
    """Interleave-prepare a 21-bit integer: bit i moves to bit 3i."""
    x = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def _morton_codes(pos: np.ndarray) -> np.ndarray:
    lo = pos.min(axis=0).astype(np.float64)
    side = float((pos.max(axis=0) - lo).max())
    side = side * (1.0 + 1e-9) if side > 0 else 1.0
    g = np.floor((pos.astype(np.float64) - lo) / side * (1 << MORTON_BITS))
    g = np.clip(g, 0, (1 << MORTON_BITS) - 1).astype(np.uint64)
    return ((_spread_bits(g[:, 0]) << np.uint64(2)) | (_spread_bits(g[:, 1]) << np.uint64(1))
            | _spread_bits(g[:, 2]))


def _octree_topology(pos: np.ndarray):
    """Return (tmp_parent, tmp_sortkey, tmp_leaf) for the octree over ``pos``.

    Temporary node ids are assigned top-down (a parent's id is smaller than its
    children's). ``tmp_leaf`` is the leaf index of a leaf node, -1 otherwise.
    ``tmp_sortkey`` orders siblings (the position of their first leaf in Morton
    order)."""
    L = pos.shape[0]
    codes = _morton_codes(pos)
    order = np.argsort(codes, kind="stable")
    codes_s = codes[order]

    parents, sortkeys, leaves = [], [], []
    next_id = 0

    def new_nodes(par, key, leaf):
        nonlocal next_id
        n = len(par)
        ids = np.arange(next_id, next_id + n, dtype=np.int64)
        next_id += n
        parents.append(np.asarray(par, dtype=np.int64))
        sortkeys.append(np.asarray(key, dtype=np.int64))
        leaves.append(np.asarray(leaf, dtype=np.int64))
        return ids

    def small_cells(par_ids, seg_lo, seg_cnt):
        """Segments of 2..8 (or, at the deepest level, more) leaves: an interior
        node each, whose children are the segment's leaves."""
        if len(seg_lo) == 0:
            return
        node_ids = new_nodes(par_ids, seg_lo, np.full(len(seg_lo), -1))
        rep_par = np.repeat(node_ids, seg_cnt)
        starts = np.repeat(seg_lo - np.concatenate(([0], np.cumsum(seg_cnt)[:-1])), seg_cnt)
        spos = np.arange(int(seg_cnt.sum()), dtype=np.int64) + starts
        new_nodes(rep_par, spos, order[spos])

    if L == 1:
        new_nodes([-1], [0], [order[0]])
        return (np.concatenate(parents), np.concatenate(sortkeys), np.concatenate(leaves))
    root = new_nodes([-1], [0], [-1])
    if L <= 8:
        spos = np.arange(L)
        new_nodes(np.repeat(root, L), spos, order[spos])
        return (np.concatenate(parents), np.concatenate(sortkeys), np.concatenate(leaves))

    cell_node = root.copy()
    cell_lo = np.array([0], dtype=np.int64)
    cell_cnt = np.array([L], dtype=np.int64)
    for level in range(MORTON_BITS):
        if len(cell_node) == 0:
            break
        shift = np.uint64(3 * (MORTON_BITS - 1 - level))
        total = int(cell_cnt.sum())
        cell_of = np.repeat(np.arange(len(cell_node)), cell_cnt)
        starts_rep = np.repeat(cell_lo - np.concatenate(([0], np.cumsum(cell_cnt)[:-1])), cell_cnt)
        idx = np.arange(total, dtype=np.int64) + starts_rep
        digit = (codes_s[idx] >> shift) & np.uint64(7)
        brk = np.ones(total, dtype=bool)
        brk[1:] = (cell_of[1:] != cell_of[:-1]) | (digit[1:] != digit[:-1])
        sstart = np.flatnonzero(brk)
        seg_lo = idx[sstart]
        seg_cell = cell_of[sstart]
        seg_cnt = np.diff(np.append(sstart, total))
        nchild = np.bincount(seg_cell, minlength=len(cell_node))
        # a cell with one non-empty octant collapses into it (same node, next level)
        collapse = nchild[seg_cell] == 1
        keep = ~collapse
        s_lo, s_cell, s_cnt = seg_lo[keep], seg_cell[keep], seg_cnt[keep]
        s_par = cell_node[s_cell]
        one = s_cnt == 1
        if one.any():
            new_nodes(s_par[one], s_lo[one], order[s_lo[one]])
        small = (s_cnt >= 2) & (s_cnt <= 8)
        small_cells(s_par[small], s_lo[small], s_cnt[small])
        big = s_cnt > 8
        big_ids = new_nodes(s_par[big], s_lo[big], np.full(int(big.sum()), -1))
        nxt_node = np.concatenate([cell_node[seg_cell[collapse]], big_ids])
        nxt_lo = np.concatenate([seg_lo[collapse], s_lo[big]])
        nxt_cnt = np.concatenate([seg_cnt[collapse], s_cnt[big]])
        o = np.argsort(nxt_lo, kind="stable")
        cell_node, cell_lo, cell_cnt = nxt_node[o], nxt_lo[o], nxt_cnt[o]
    if len(cell_node):
        # deepest grid level reached with more than 8 coincident leaves: one node
        # takes them all as children
        rep_par = np.repeat(cell_node, cell_cnt)
        starts = np.repeat(cell_lo - np.concatenate(([0], np.cumsum(cell_cnt)[:-1])), cell_cnt)
        spos = np.arange(int(cell_cnt.sum()), dtype=np.int64) + starts
        new_nodes(rep_par, spos, order[spos])
    return (np.concatenate(parents), np.concatenate(sortkeys), np.concatenate(leaves))


def _bfs_order(tmp_parent: np.ndarray, tmp_key: np.ndarray):
    """Breadth-first ids: depth by depth, children grouped by their parent's id
    and ordered by ``tmp_key``. Returns (new_id_of_tmp, depth_of_tmp)."""
    n = len(tmp_parent)
    depth = np.zeros(n, dtype=np.int64)
    anc = tmp_parent.copy()
    while True:
        act = anc >= 0
        if not act.any():
            break
        depth[act] += 1
        anc[act] = tmp_parent[anc[act]]
    new_id = np.full(n, -1, dtype=np.int64)
    nxt = 0
    for d in range(int(depth.max()) + 1):
        at = np.flatnonzero(depth == d)
        if d == 0:
            o = at
        else:
            o = at[np.lexsort((tmp_key[at], new_id[tmp_parent[at]]))]
        new_id[o] = np.arange(nxt, nxt + len(o))
        nxt += len(o)
    return new_id, depth


def _cov_from_quat_scale(quat_wxyz: np.ndarray, log_scale: np.ndarray) -> np.ndarray:
    """float64 covariances R diag(exp(2 s)) R^T; the rotation matrix comes from
    scipy's quaternion routine (scalar-last order)."""
    q = quat_wxyz.astype(np.float64)
    R = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], axis=1)).as_matrix()
    s2 = np.exp(2.0 * log_scale.astype(np.float64))
    return np.einsum("nij,nj,nkj->nik", R, s2, R)


def _quat_scale_from_cov(cov: np.ndarray):
    w, V = np.linalg.eigh(cov)
    w = np.maximum(w, 1e-30)
    det = np.linalg.det(V)
    V[det < 0, :, 0] *= -1.0
    q = Rotation.from_matrix(V).as_quat()  # x,y,z,w
    q = np.concatenate([q[:, 3:], q[:, :3]], axis=1)
    q[q[:, 0] < 0] *= -1.0
    return q, 0.5 * np.log(w)


def build_hierarchy(leaf_pos, leaf_quat, leaf_log_scale, leaf_opacity, leaf_sh,
                    keep_fp64: bool = False) -> Scene:
    """Octree hierarchy with opacity-weighted moment-matched interior nodes.

    For an interior node p with children i and weights w_i = o_i:
      mu_p    = sum w_i mu_i / W
      Sigma_p = sum w_i (Sigma_i + (mu_i - mu_p)(mu_i - mu_p)^T) / W
      SH_p    = sum w_i SH_i / W,   o_p = sum w_i o_i / W,  W = sum w_i
    Sigma_p is stored as (quaternion, log-scale) from its eigendecomposition.
    """
    L = leaf_pos.shape[0]
    tp, tk, tl = _octree_topology(leaf_pos)
    new_id, tdepth = _bfs_order(tp, tk)
    M = len(tp)
    parent = np.full(M, -1, dtype=np.int64)
    has_par = tp >= 0
    parent[new_id[has_par]] = new_id[tp[has_par]]
    depth = np.zeros(M, dtype=np.int64)
    depth[new_id] = tdepth
    leaf_of = np.full(M, -1, dtype=np.int64)
    leaf_of[new_id] = tl
    child_count = np.bincount(parent[1:], minlength=M).astype(np.int64) if M > 1 else np.zeros(1, np.int64)
    child_begin = np.full(M, -1, dtype=np.int64)
    if M > 1:
        # BFS ids: a node's children are contiguous and appear in parent order
        kids = np.arange(1, M)
        first = np.ones(M - 1, dtype=bool)
        first[1:] = parent[2:] != parent[1:-1]
        child_begin[parent[kids[first]]] = kids[first]

    is_leaf = leaf_of >= 0
    assert int(is_leaf.sum()) == L
    assert np.all((child_count == 0) == is_leaf)

    mean = np.zeros((M, 3))
    cov = np.zeros((M, 3, 3))
    opac = np.zeros(M)
    sh = np.zeros((M, 16, 3))
    quat = np.zeros((M, 4))
    logs = np.zeros((M, 3))
    li = leaf_of[is_leaf]
    mean[is_leaf] = leaf_pos[li].astype(np.float64)
    cov[is_leaf] = _cov_from_quat_scale(leaf_quat[li], leaf_log_scale[li])
    opac[is_leaf] = leaf_opacity[li].astype(np.float64)
    sh[is_leaf] = leaf_sh[li].astype(np.float64)
    quat[is_leaf] = leaf_quat[li].astype(np.float64)
    logs[is_leaf] = leaf_log_scale[li].astype(np.float64)

    # leaf boxes from the float32-stored leaf attributes
    bmin = np.zeros((M, 3), dtype=np.float32)
    bmax = np.zeros((M, 3), dtype=np.float32)
    sig = np.sqrt(np.einsum("nii->ni", cov[is_leaf]))
    bmin[is_leaf] = (mean[is_leaf] - 3.0 * sig).astype(np.float32)
    bmax[is_leaf] = (mean[is_leaf] + 3.0 * sig).astype(np.float32)

    for d in range(int(depth.max()) - 1, -1, -1):
        nodes = np.flatnonzero((depth == d) & ~is_leaf)
        if len(nodes) == 0:
            continue
        cb = child_begin[nodes]
        cc = child_count[nodes]
        lo, hi = int(cb[0]), int(cb[-1] + cc[-1])
        assert hi - lo == int(cc.sum())
        ch = np.arange(lo, hi)
        rel = cb - lo
        w = opac[ch]
        W = np.add.reduceat(w, rel)
        mu = np.add.reduceat(w[:, None] * mean[ch], rel, axis=0) / W[:, None]
        dlt = mean[ch] - np.repeat(mu, cc, axis=0)
        c2 = cov[ch] + dlt[:, :, None] * dlt[:, None, :]
        cv = np.add.reduceat(w[:, None, None] * c2, rel, axis=0) / W[:, None, None]
        cv = 0.5 * (cv + np.transpose(cv, (0, 2, 1)))
        mean[nodes] = mu
        cov[nodes] = cv
        opac[nodes] = np.add.reduceat(w * w, rel) / W
        sh[nodes] = np.add.reduceat(w[:, None, None] * sh[ch], rel, axis=0) / W[:, None, None]
        q, s = _quat_scale_from_cov(cv)
        quat[nodes] = q
        logs[nodes] = s
        bmin[nodes] = np.minimum.reduceat(bmin[ch], rel, axis=0)
        bmax[nodes] = np.maximum.reduceat(bmax[ch], rel, axis=0)

    sc = Scene(pos=mean.astype(np.float32), quat=quat.astype(np.float32),
               log_scale=logs.astype(np.float32), opacity=opac.astype(np.float32),
               sh=sh.astype(np.float32), parent=parent.astype(np.int32),
               child_begin=child_begin.astype(np.int32), child_count=child_count.astype(np.int32),
               aabb_min=bmin, aabb_max=bmax, n_leaves=L, depth=depth.astype(np.int32))
    if keep_fp64:
        sc.cov64 = cov
        sc.mean64 = mean
        sc.opacity64 = opac
    return sc


# ---------------------------------------------------------------------------
# layouts
# ---------------------------------------------------------------------------

def make_uniform_box_scene(n_leaves: int, seed: int, box=(4.0, 4.0, 3.0),
                           keep_fp64: bool = False) -> Scene:
    """Leaves uniform in [0,bx]x[0,by]x[0,bz] (the small 10k-leaf scene)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, 1.0, size=(n_leaves, 3)) * np.asarray(box)
    q, s, o, sh = _leaf_attributes(rng, n_leaves)
    sc = build_hierarchy(pos.astype(np.float32), q, s, o, sh, keep_fp64=keep_fp64)
    sc.meta = {"layout": "uniform_box", "box": list(box), "seed": seed, "leaves": n_leaves}
    return sc


def wall_segments(size_x, size_y, grid=4.0, door=1.0, extra_y_walls=(), extra_door=4.0):
    """Axis-aligned wall segments (axis, coord, lo, hi) on a ``grid``-metre grid,
    every grid cell side carrying a centred doorway gap of ``door`` metres."""
    segs = []
    xs = list(np.arange(0.0, size_x + 1e-9, grid))
    if xs[-1] < size_x - 1e-9:
        xs.append(size_x)
    ys = list(np.arange(0.0, size_y + 1e-9, grid))
    if ys[-1] < size_y - 1e-9:
        ys.append(size_y)
    for axis, coords, other in (("x", xs, ys), ("y", ys, xs)):
        for c in coords:
            for a, b in zip(other[:-1], other[1:]):
                mid = 0.5 * (a + b)
                g = min(door, 0.5 * (b - a))
                segs.append((axis, c, a, mid - 0.5 * g))
                segs.append((axis, c, mid + 0.5 * g, b))
    for y in extra_y_walls:
        mid = 0.5 * size_x
        segs.append(("y", y, 0.0, mid - 0.5 * extra_door))
        segs.append(("y", y, mid + 0.5 * extra_door, size_x))
    return [s for s in segs if s[3] - s[2] > 1e-6]


def make_floor_scene(n_leaves: int, seed: int, size=(20.0, 15.0, 3.0), n_clusters: int = 40,
                     cluster_size: int = 5000, extra_y_walls=(), keep_fp64: bool = False) -> Scene:
    """Multi-room floor: a floor plane (z ~ N(0, 1 cm)), wall slabs (1 cm
    thickness spread) on a 4 m grid with 1 m doorways, and furniture clusters
    (isotropic N(0, 0.3 m) blobs clipped to z >= 0). The leaves not in clusters
    are split between floor and walls in proportion to their areas."""
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    n_furn = min(n_clusters * cluster_size, n_leaves // 2)
    n_clusters_eff = max(1, n_furn // cluster_size) if n_furn else 0
    segs = wall_segments(sx, sy, extra_y_walls=extra_y_walls)
    seg_len = np.array([s[3] - s[2] for s in segs])
    wall_area = float(seg_len.sum() * sz)
    floor_area = sx * sy
    rest = n_leaves - n_furn
    n_wall = int(round(rest * wall_area / (wall_area + floor_area)))
    n_floor = rest - n_wall
    parts = []
    # floor
    fp = np.empty((n_floor, 3))
    fp[:, 0] = rng.uniform(0, sx, n_floor)
    fp[:, 1] = rng.uniform(0, sy, n_floor)
    fp[:, 2] = rng.normal(0.0, 0.01, n_floor)
    parts.append(fp)
    # walls
    which = rng.choice(len(segs), size=n_wall, p=seg_len / seg_len.sum())
    t = rng.uniform(0, 1, n_wall)
    wp = np.empty((n_wall, 3))
    lo = np.array([segs[i][2] for i in range(len(segs))])[which]
    hi = np.array([segs[i][3] for i in range(len(segs))])[which]
    c = np.array([segs[i][1] for i in range(len(segs))])[which]
    along = lo + t * (hi - lo)
    normal = c + rng.normal(0.0, 0.01, n_wall)
    isx = np.array([segs[i][0] == "x" for i in range(len(segs))])[which]
    wp[:, 0] = np.where(isx, normal, along)
    wp[:, 1] = np.where(isx, along, normal)
    wp[:, 2] = rng.uniform(0, sz, n_wall)
    parts.append(wp)
    # furniture
    if n_furn:
        cent = np.empty((n_clusters_eff, 3))
        cent[:, 0] = rng.uniform(0.6, sx - 0.6, n_clusters_eff)
        cent[:, 1] = rng.uniform(0.6, sy - 0.6, n_clusters_eff)
        cent[:, 2] = 0.4
        members = np.repeat(np.arange(n_clusters_eff), cluster_size)[:n_furn]
        members = np.concatenate([members, rng.integers(0, n_clusters_eff, n_furn - len(members))])
        bp = cent[members] + rng.normal(0.0, 0.3, size=(n_furn, 3))
        bp[:, 2] = np.abs(bp[:, 2])
        parts.append(bp)
    pos = np.concatenate(parts).astype(np.float32)
    pos = pos[rng.permutation(len(pos))]
    q, s, o, sh = _leaf_attributes(rng, n_leaves)
    sc = build_hierarchy(pos, q, s, o, sh, keep_fp64=keep_fp64)
    sc.meta = {"layout": "floor", "size": list(size), "seed": seed, "leaves": n_leaves,
               "clusters": n_clusters_eff, "walls": segs, "extra_y_walls": list(extra_y_walls)}
    return sc


# name -> (builder, kwargs); the floor scenes are the multi-room stand-ins for the
# captured office floors the simulator renders
SCENE_PRESETS = {
    "box10k": (make_uniform_box_scene, dict(n_leaves=10_000, seed=0)),
    "floor1m": (make_floor_scene, dict(n_leaves=1_000_000, seed=1, size=(20.0, 15.0, 3.0),
                                       n_clusters=40)),
    "floor4m": (make_floor_scene, dict(n_leaves=4_000_000, seed=2, size=(25.0, 12.0, 3.0),
                                       n_clusters=160)),
    "floor8m": (make_floor_scene, dict(n_leaves=8_000_000, seed=4, size=(30.0, 20.0, 3.0),
                                       n_clusters=160, extra_y_walls=(10.0,))),
}


def make_scene(name: str, **overrides) -> Scene:
    fn, kw = SCENE_PRESETS[name]
    kw = dict(kw)
    kw.update(overrides)
    return fn(**kw)


def _to_bf16_rne(a: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (nearest-even), returned as uint16 bit patterns."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    rnd = ((b >> 16) & 1) + 0x7FFF
    return ((b + rnd) >> 16).astype(np.uint16)


def _bf16_to_f32(u: np.ndarray) -> np.ndarray:
    return (u.astype(np.uint32) << 16).view(np.float32)


def quantize_attributes(scene: Scene, dtype: str):
    """Reduced-precision storage of SH, log-scales and opacities.

    Returns (stored, dequantised): ``stored`` maps attribute name to the array
    handed to the renderer (float16 arrays, or uint16 bfloat16 bit patterns);
    ``dequantised`` maps it to float32 arrays holding exactly the stored values,
    which is what the float64 oracle must see for kernel parity."""
    out, deq = {}, {}
    for name in ("sh", "log_scale", "opacity"):
        a = getattr(scene, name)
        if dtype == "f16":
            h = a.astype(np.float16)
            out[name] = h
            deq[name] = h.astype(np.float32)
        elif dtype == "bf16":
            u = _to_bf16_rne(a)
            out[name] = u
            deq[name] = _bf16_to_f32(u).reshape(a.shape)
        elif dtype == "f32":
            out[name] = a
            deq[name] = a
        else:
            raise ValueError(dtype)
    return out, deq
