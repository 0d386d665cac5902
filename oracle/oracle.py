"""Python face of the float64 oracle (test infrastructure only).

Each function follows one step of the render path as the C++ source states it:
``select_cut`` (level-of-detail cut, Sec. III-B), ``preprocess`` (EWA projection
and SH colour of 3DGS, Sec. III-A), ``bin_pairs`` ((tile, depth) keys and a
stable sort), ``composite_tiled`` (front-to-back blending) and
``render_bruteforce`` (per-pixel blending over every visible Gaussian, no
tiles). ``render`` chains them for one camera. With ``blend``, preprocess
renders each cut node with its level-of-detail blended attributes
(``blend_gaussian``: moved toward its parent's by the parent weight
``blend_parent_weight`` of the granularities, Sec. III-B's interpolated
transitions). ``frustum_state`` and ``select_cut_shared`` give the cut's
variants: nodes culled against the five planes of a camera's view volume, and
one cut for a group of cameras (Sec. III-B's per-view, dynamic selection).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from types import SimpleNamespace

import numpy as np

from . import build as _build

PC = SimpleNamespace(VISIBLE=0, U=1, V=2, CONIC_A=3, CONIC_B=4, CONIC_C=5, COV_A=6, COV_B=7,
                     COV_C=8, DEPTH=9, OPACITY=10, R=11, G=12, B=13, HX=14, HY=15,
                     EU=16, EV=17, EB=18, EC=19, EDET=20, EQL=21, EHX=22, EHY=23, NCOLS=24)


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("quat", C.c_void_p),
                ("log_scale", C.c_void_p), ("opacity", C.c_void_p), ("sh", C.c_void_p),
                ("parent", C.c_void_p), ("child_count", C.c_void_p),
                ("aabb_min", C.c_void_p), ("aabb_max", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("pos", C.c_double * 3), ("R", C.c_double * 9), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("tau", C.c_double)]


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
            L.orc_select_cut.restype = i64
            L.orc_select_cut.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), vp, vp, vp]
            L.orc_preprocess.restype = None
            L.orc_preprocess.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), vp, i64, i32, i32,
                                         i32, vp, vp, vp]
            L.orc_granularity_f32.restype = C.c_float
            L.orc_granularity_f32.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), i64]
            L.orc_blend_parent_weight.restype = C.c_float
            L.orc_blend_parent_weight.argtypes = [C.c_float, C.c_float, C.c_float]
            L.orc_blend_gaussian.restype = C.c_double
            L.orc_blend_gaussian.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), i64, i32, vp,
                                             vp, vp, vp]
            L.orc_count_pairs.restype = i64
            L.orc_count_pairs.argtypes = [vp, i64]
            L.orc_bin_pairs.restype = None
            L.orc_bin_pairs.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp]
            L.orc_composite_tiled.restype = None
            L.orc_composite_tiled.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp, vp]
            L.orc_render_bruteforce.restype = None
            L.orc_render_bruteforce.argtypes = [vp, vp, i64, vp, i64, vp, vp]
            L.orc_sh_basis.restype = None
            L.orc_sh_basis.argtypes = [vp, vp]
            L.orc_cov3d.restype = None
            L.orc_cov3d.argtypes = [vp, vp, vp]
            L.orc_depth_f32.restype = C.c_float
            L.orc_depth_f32.argtypes = [vp, C.POINTER(_Camera)]
            L.orc_exponent_error.restype = C.c_double
            L.orc_exponent_error.argtypes = [vp, C.c_double, C.c_double]
            L.orc_view_depth64.restype = C.c_double
            L.orc_view_depth64.argtypes = [vp, C.POINTER(_Camera)]
            L.orc_alternatives.restype = None
            L.orc_alternatives.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp, i64, i32, vp, vp]
            L.orc_num_threads.restype = i32
            L.orc_set_threads.restype = None
            L.orc_set_threads.argtypes = [i32]
            L.orc_slice_params.restype = None
            L.orc_slice_params.argtypes = [vp, vp, vp]
            L.orc_slice_value.restype = C.c_double
            L.orc_slice_value.argtypes = [C.POINTER(_Scene), i64, C.c_double, C.c_double,
                                          C.c_double]
            L.orc_nav_blocked.restype = None
            L.orc_nav_blocked.argtypes = [vp, i32, i32, i32, i32, i32, vp]
            L.orc_nav_field.restype = None
            L.orc_nav_field.argtypes = [vp, i32, i32, i32, i32, vp]
            L.orc_nav_path.restype = i32
            L.orc_nav_path.argtypes = [vp, i32, i32, i32, i32, i32, vp]
            L.orc_slice_occupancy.restype = None
            L.orc_slice_occupancy.argtypes = [C.POINTER(_Scene), C.c_double, C.c_double,
                                              C.c_double, i32, i32, C.c_double, C.c_double, i32,
                                              C.c_double, vp, vp]
            L.orc_frustum_state.restype = None
            L.orc_frustum_state.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), C.c_double,
                                            vp]
            L.orc_select_cut_shared.restype = i64
            L.orc_select_cut_shared.argtypes = [C.POINTER(_Scene), vp, vp, i32, i32, C.c_double,
                                                vp, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class SceneArrays:
    """Contiguous float32/int32 views of a scene (optionally with dequantised
    attributes substituted), kept alive while the oracle reads them."""

    def __init__(self, scene, overrides=None):
        ov = overrides or {}
        get = lambda k, dt: np.ascontiguousarray(ov.get(k, getattr(scene, k)), dtype=dt)
        self.pos = get("pos", np.float32)
        self.quat = get("quat", np.float32)
        self.log_scale = get("log_scale", np.float32)
        self.opacity = get("opacity", np.float32)
        self.sh = get("sh", np.float32)
        self.parent = get("parent", np.int32)
        self.child_count = get("child_count", np.int32)
        self.aabb_min = get("aabb_min", np.float32)
        self.aabb_max = get("aabb_max", np.float32)
        self.n = int(self.parent.shape[0])
        self.c = _Scene(self.n, _p(self.pos).value, _p(self.quat).value, _p(self.log_scale).value,
                        _p(self.opacity).value, _p(self.sh).value, _p(self.parent).value,
                        _p(self.child_count).value, _p(self.aabb_min).value,
                        _p(self.aabb_max).value)


def _as_scene(scene):
    return scene if isinstance(scene, SceneArrays) else SceneArrays(scene)


def camera_struct(cam) -> _Camera:
    c = _Camera()
    for k in range(3):
        c.pos[k] = float(np.float32(cam.pos[k]))
    R = np.asarray(cam.R_wc, dtype=np.float32).reshape(9)
    for k in range(9):
        c.R[k] = float(R[k])
    c.fx, c.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    c.cx, c.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.tau = float(np.float32(cam.tau))
    return c


def select_cut(scene, cam, with_s: bool = False):
    """Level-of-detail cut at the camera's tau. Returns (ids ascending int32,
    near uint8[M]) and, with ``with_s``, the granularity s(n) as float64."""
    sa = _as_scene(scene)
    ids = np.empty(sa.n, dtype=np.int32)
    near = np.empty(sa.n, dtype=np.uint8)
    s = np.empty(sa.n, dtype=np.float64) if with_s else None
    cc = camera_struct(cam)
    k = lib().orc_select_cut(C.byref(sa.c), C.byref(cc), _p(ids), _p(near),
                             _p(s) if with_s else None)
    out = (ids[:k].copy(), near)
    return out + (s,) if with_s else out


def frustum_state(scene, cam, guard: float = 0.0):
    """Frustum cull of every node's box for a view volume widened by ``guard``
    pixels: (culled bool[M], unsure bool[M]); unsure marks a plane value
    within 1e-5 of its scale that no other plane overrides."""
    sa = _as_scene(scene)
    out = np.empty(sa.n, dtype=np.uint8)
    lib().orc_frustum_state(C.byref(sa.c), C.byref(camera_struct(cam)), float(guard), _p(out))
    return (out & 1).astype(bool), (out & 2).astype(bool)


def select_cut_shared(scene, cams, group_begin, frustum: bool = True, guard: float = 0.0):
    """One cut per group of cameras, group g = cams[group_begin[g]:group_begin[g+1]],
    optionally frustum-culled: (ids int32 concatenated group after group,
    offsets int64[n_groups + 1], near uint8[n_groups, M])."""
    sa = _as_scene(scene)
    gb = np.ascontiguousarray(group_begin, dtype=np.int32)
    ng = len(gb) - 1
    assert ng >= 1 and gb[0] == 0 and gb[-1] == len(cams) and np.all(np.diff(gb) >= 1)
    carr = (_Camera * len(cams))(*[camera_struct(c) for c in cams])
    ids = np.empty(max(ng * sa.n, 1), dtype=np.int32)
    off = np.empty(ng + 1, dtype=np.int64)
    near = np.empty((ng, sa.n), dtype=np.uint8)
    k = lib().orc_select_cut_shared(C.byref(sa.c), C.cast(carr, C.c_void_p), _p(gb), ng,
                                    1 if frustum else 0, float(guard), _p(ids), _p(off),
                                    _p(near))
    return ids[:k].copy(), off, near


def preprocess(scene, cam, ids, tile=(16, 16), blend=False):
    """Per cut slot: float64 table (columns PC.*), float32 depth-key bits and
    the inclusive tile rectangle (x0, y0, x1, y1). ``blend``: level-of-detail
    blended attributes."""
    sa = _as_scene(scene)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    n = len(ids)
    pre = np.empty((n, PC.NCOLS), dtype=np.float64)
    key = np.empty(n, dtype=np.uint32)
    rect = np.empty((n, 4), dtype=np.int32)
    cc = camera_struct(cam)
    lib().orc_preprocess(C.byref(sa.c), C.byref(cc), _p(ids), n, int(tile[0]), int(tile[1]),
                         1 if blend else 0, _p(pre), _p(key), _p(rect))
    return pre, key, rect


def tiles_xy(cam, tile):
    return (-(-int(cam.width) // tile[0]), -(-int(cam.height) // tile[1]))


def bin_pairs(rect, key, cam, tile=(16, 16)):
    """Sorted (tile << 32 | depth) keys, slot values and per-tile [start, end)."""
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    n = len(key)
    L = lib()
    P = L.orc_count_pairs(_p(rect), n)
    tx, ty = tiles_xy(cam, tile)
    keys = np.empty(P, dtype=np.uint64)
    vals = np.empty(P, dtype=np.uint32)
    ranges = np.empty((tx * ty, 2), dtype=np.int64)
    L.orc_bin_pairs(_p(rect), _p(key), n, tx, ty, _p(keys), _p(vals), _p(ranges))
    return keys, vals, ranges


def composite_tiled(pre, vals, ranges, cam, tile=(16, 16)):
    """Image [3, H, W] float64 (every decision in float64) and per-pixel flags
    [H, W]: 1 where some threshold or stop decision was near threshold (a
    float32 renderer may take it the other way; ``alternatives`` lists the
    outcomes)."""
    H, W = int(cam.height), int(cam.width)
    img = np.empty((3, H, W), dtype=np.float64)
    flags = np.empty((H, W), dtype=np.uint8)
    pre = np.ascontiguousarray(pre, dtype=np.float64)
    vals = np.ascontiguousarray(vals, dtype=np.uint32)
    ranges = np.ascontiguousarray(ranges, dtype=np.int64)
    lib().orc_composite_tiled(_p(pre), _p(vals), _p(ranges), W, H, int(tile[0]), int(tile[1]),
                              _p(img), _p(flags))
    return img, flags


def alternatives(pre, vals, ranges, cam, pixels, tile=(16, 16), max_out=64):
    """Every outcome of the near-threshold decisions of the tiled compositing
    at ``pixels`` ((n, 2) integer (x, y)): (rgb [n, max_out, 3] float64,
    count [n] int32; count = max_out + 1 when there were more outcomes, and
    negative when a decision's error bound was too large to enumerate)."""
    pixels = np.ascontiguousarray(pixels, dtype=np.int32).reshape(-1, 2)
    n = len(pixels)
    out = np.zeros((n, max_out, 3), dtype=np.float64)
    cnt = np.zeros(n, dtype=np.int32)
    if n:
        pre = np.ascontiguousarray(pre, dtype=np.float64)
        vals = np.ascontiguousarray(vals, dtype=np.uint32)
        ranges = np.ascontiguousarray(ranges, dtype=np.int64)
        lib().orc_alternatives(_p(pre), _p(vals), _p(ranges), int(cam.width), int(cam.height),
                               int(tile[0]), int(tile[1]), _p(pixels), n, int(max_out), _p(out),
                               _p(cnt))
    return out, cnt


def render_bruteforce(pre, key, pixels=None, cam=None):
    """Per-pixel blending of every visible Gaussian in (depth, slot) order.
    ``pixels`` is an (n, 2) array of integer (x, y); default: every pixel of
    ``cam``. Returns (rgb [n, 3], flags [n])."""
    if pixels is None:
        yy, xx = np.mgrid[0:int(cam.height), 0:int(cam.width)]
        pixels = np.stack([xx.ravel(), yy.ravel()], axis=1)
    pixels = np.ascontiguousarray(pixels, dtype=np.int32)
    pre = np.ascontiguousarray(pre, dtype=np.float64)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty((len(pixels), 3), dtype=np.float64)
    flags = np.empty(len(pixels), dtype=np.uint8)
    lib().orc_render_bruteforce(_p(pre), _p(key), len(key), _p(pixels), len(pixels), _p(out),
                                _p(flags))
    return out, flags


def render(scene, cam, tile=(16, 16), ids=None, blend=False):
    """Full tiled render of one camera (``blend``: level-of-detail blending).
    Returns a namespace with the cut, the preprocess table, sorted pairs,
    ranges, the image and its flags."""
    sa = _as_scene(scene)
    near = None
    if ids is None:
        ids, near = select_cut(sa, cam)
    pre, key, rect = preprocess(sa, cam, ids, tile, blend)
    keys, vals, ranges = bin_pairs(rect, key, cam, tile)
    img, flags = composite_tiled(pre, vals, ranges, cam, tile)
    return SimpleNamespace(ids=ids, near=near, pre=pre, key=key, rect=rect, keys=keys, vals=vals,
                           ranges=ranges, image=img, flags=flags, tile=tuple(tile), cam=cam)


def sh_basis(dirs):
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    out = np.empty((len(dirs), 16), dtype=np.float64)
    L = lib()
    for i in range(len(dirs)):
        L.orc_sh_basis(_p(dirs[i]), out[i].ctypes.data_as(C.c_void_p))
    return out


def cov3d(quat, log_scale):
    quat = np.ascontiguousarray(np.atleast_2d(quat), dtype=np.float32)
    log_scale = np.ascontiguousarray(np.atleast_2d(log_scale), dtype=np.float32)
    out = np.empty((len(quat), 3, 3), dtype=np.float64)
    L = lib()
    for i in range(len(quat)):
        L.orc_cov3d(_p(quat[i]), _p(log_scale[i]), out[i].ctypes.data_as(C.c_void_p))
    return out


def exponent_error(row, dx, dy):
    """Bound on a float32 renderer's error in log2(o G) of the Gaussian of
    preprocess row ``row`` at pixel offset (dx, dy) (the oracle's float32 error
    model)."""
    row = np.ascontiguousarray(row, dtype=np.float64)
    return float(lib().orc_exponent_error(_p(row), float(dx), float(dy)))


def view_depth64(mu, cam):
    """The float64 view depth R_2 . (mu - c) of one mean (no float32 step)."""
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    return float(lib().orc_view_depth64(_p(mu), C.byref(camera_struct(cam))))


def depth_f32(mu, cam):
    """The float32 view depth used for the near-plane cull and the sort key."""
    mu = np.ascontiguousarray(mu, dtype=np.float32)
    cc = camera_struct(cam)
    return lib().orc_depth_f32(_p(mu), C.byref(cc))


def granularity_f32(scene, cam, node):
    """s(node) in the renderer's float32 operation sequence."""
    sa = _as_scene(scene)
    cc = camera_struct(cam)
    return float(lib().orc_granularity_f32(C.byref(sa.c), C.byref(cc), int(node)))


def blend_parent_weight(s_n, s_p, tau):
    """Parent weight v of the level-of-detail blend (float32)."""
    return float(lib().orc_blend_parent_weight(float(s_n), float(s_p), float(tau)))


def blend_gaussian(scene, cam, node, blend=True):
    """(v, mu float32 [3], Sigma [3, 3], opacity, sh [16, 3]) of a node as rendered."""
    sa = _as_scene(scene)
    cc = camera_struct(cam)
    mu = np.empty(3, dtype=np.float32)
    S = np.empty((3, 3), dtype=np.float64)
    op = np.empty(1, dtype=np.float64)
    sh = np.empty((16, 3), dtype=np.float64)
    v = lib().orc_blend_gaussian(C.byref(sa.c), C.byref(cc), int(node), 1 if blend else 0,
                                 _p(mu), _p(S), _p(op), _p(sh))
    return float(v), mu, S, float(op[0]), sh


def slice_params(quat, log_scale):
    """(alpha, beta, lambda, cxx, cxy, cyy, cxz, cyz, czz) of the GS slice of a
    Gaussian (Sec. III-C)."""
    q = np.ascontiguousarray(quat, dtype=np.float32)
    ls = np.ascontiguousarray(log_scale, dtype=np.float32)
    out = np.empty(9, dtype=np.float64)
    lib().orc_slice_params(_p(q), _p(ls), _p(out))
    return out


def slice_value(scene, g, x, y, z):
    """o G2D((x, y), z) of Gaussian g (no cap, no cut-off)."""
    sa = _as_scene(scene)
    return float(lib().orc_slice_value(C.byref(sa.c), int(g), float(x), float(y), float(z)))


def slice_occupancy(scene, grid):
    """Per plane and cell the largest slice value of the leaves (float64
    [nz, ny, nx]) and the occupancy mask at grid.threshold (uint8).
    ``grid``: x0, y0, cell, nx, ny, z0, dz, nz, threshold."""
    sa = _as_scene(scene)
    g = grid
    val = np.empty((g.nz, g.ny, g.nx), dtype=np.float64)
    occ = np.empty((g.nz, g.ny, g.nx), dtype=np.uint8)
    lib().orc_slice_occupancy(C.byref(sa.c), float(g.x0), float(g.y0), float(g.cell), int(g.nx),
                              int(g.ny), float(g.z0), float(g.dz), int(g.nz), float(g.threshold),
                              _p(val), _p(occ))
    return val, occ


def nav_blocked(occ, k_lo, k_hi, inflate):
    """Blocked cells [ny, nx] (uint8): some plane in [k_lo, k_hi] occupied
    within Chebyshev distance ``inflate``."""
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    nz, ny, nx = occ.shape
    out = np.empty((ny, nx), dtype=np.uint8)
    lib().orc_nav_blocked(_p(occ), nx, ny, int(k_lo), int(k_hi), int(inflate), _p(out))
    return out


def nav_field(blocked, goal):
    """4-connected breadth-first distances (uint32, 0xffffffff unreachable)
    from goal = (i, j) over the free cells."""
    blocked = np.ascontiguousarray(blocked, dtype=np.uint8)
    ny, nx = blocked.shape
    out = np.empty((ny, nx), dtype=np.uint32)
    lib().orc_nav_field(_p(blocked), nx, ny, int(goal[0]), int(goal[1]), _p(out))
    return out


def nav_path(dist, start, max_len):
    """Shortest path (cells (i, j), start first) descending the field."""
    dist = np.ascontiguousarray(dist, dtype=np.uint32)
    ny, nx = dist.shape
    path = np.zeros((max_len, 2), dtype=np.int32)
    n = lib().orc_nav_path(_p(dist), nx, ny, int(start[0]), int(start[1]), int(max_len), _p(path))
    return path[:n].copy()


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on."""
    lib().orc_set_threads(int(n))


__all__ = ["PC", "SceneArrays", "camera_struct", "select_cut", "preprocess", "bin_pairs",
           "composite_tiled", "render_bruteforce", "render", "sh_basis", "cov3d", "depth_f32",
           "view_depth64", "alternatives", "exponent_error",
           "tiles_xy", "num_threads", "set_threads", "lib", "granularity_f32", "blend_parent_weight",
           "blend_gaussian", "slice_params", "slice_value", "slice_occupancy", "nav_blocked",
           "nav_field", "nav_path", "frustum_state", "select_cut_shared"]
