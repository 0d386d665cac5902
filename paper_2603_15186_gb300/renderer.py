"""Python binding of the renderer: argument marshalling over the C ABI only.

Every stage of the render path runs in the CUDA kernels of libngs.so; this
module converts cameras and scene arrays to the ABI's structs and hands device
memory (PyTorch tensors) and streams to it."""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import check


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the renderer needs a CUDA device; none is available")
    return torch


def camera_struct(cam) -> _lib.Camera:
    """From any object with pos, R_wc, fx, fy, cx, cy, width, height, tau."""
    c = _lib.Camera()
    pos = np.asarray(cam.pos, dtype=np.float32).reshape(3)
    R = np.asarray(cam.R_wc, dtype=np.float32).reshape(9)
    for k in range(3):
        c.pos[k] = float(pos[k])
    for k in range(9):
        c.R_wc[k] = float(R[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.tau = int(cam.width), int(cam.height), float(cam.tau)
    return c


def camera_array(cams: Sequence) -> C.Array:
    arr = (_lib.Camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = camera_struct(cam)
    return arr


def _stream_ptr(stream):
    if stream is None:
        torch = _torch()
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Renderer:
    """One renderer context on one GPU: a resident scene plus work buffers."""

    def __init__(self, device: int = 0, tile=(16, 16), batch: int = 128,
                 cut_capacity: int = 0, record_capacity: int = 0, pair_capacity: int = 0,
                 max_tiles_per_batch: int = 0):
        self.L = _lib.load()
        cfg = _lib.Config(device, int(tile[0]), int(tile[1]), int(batch), int(cut_capacity),
                          int(record_capacity), int(pair_capacity), int(max_tiles_per_batch), 0)
        h = C.c_void_p()
        check(self.L.ngs_create(C.byref(cfg), C.byref(h)), "ngs_create")
        self.h = h
        self.device = device
        self._keep = []
        self.attr_dtype = "f32"

    def close(self):
        if getattr(self, "h", None):
            self.L.ngs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration -----------------------------------------------------
    def set_mode(self, mode: str):
        m = {"batched": _lib.NGS_MODE_BATCHED, "plain": _lib.NGS_MODE_PLAIN}[mode]
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_MODE, m), "ngs_set_option(mode)")

    def set_tile(self, w: int, h: int):
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_TILE_W, int(w)), "tile_w")
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_TILE_H, int(h)), "tile_h")

    def set_cta(self, w: int, h: int):
        """Pixel block of one compositing CTA (0, 0: the whole tile)."""
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_CTA_W, int(w)), "cta_w")
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_CTA_H, int(h)), "cta_h")

    def set_pairs_per_pixel(self, v: int):
        """The sub-batch planner's estimate of (tile, Gaussian) pairs per pixel."""
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_PAIRS_PER_PIXEL, int(v)),
              "pairs_per_pixel")

    def set_batch(self, b: int):
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_BATCH, int(b)), "batch")

    def set_graph(self, on: bool):
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_GRAPH, 1 if on else 0), "graph")

    def set_block_cull(self, on: bool):
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_BLOCK_CULL, 1 if on else 0), "block cull")

    def set_lod_blend(self, on: bool):
        """Level-of-detail blending of every cut node toward its parent."""
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_LOD_BLEND, 1 if on else 0), "lod blend")

    def set_composite_order(self, longest_first: bool):
        """Batched compositing takes tiles longest list first (default) or in
        tile order; the images are the same."""
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_COMPOSITE_ORDER, 1 if longest_first else 0),
              "composite order")

    def set_node_ids(self, on: bool):
        """Renders also keep each visible Gaussian's node id, which tile_lists
        reports; the images are the same."""
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_NODE_IDS, 1 if on else 0), "node ids")

    def set_stage_timing(self, on: bool):
        check(self.L.ngs_set_option(self.h, _lib.NGS_OPT_STAGE_TIMING, 1 if on else 0),
              "stage timing")

    def stage_times(self) -> dict:
        """Milliseconds per stage of the last render (stage timing must be on)."""
        ms = np.zeros(len(_lib.STAGES), dtype=np.float64)
        check(self.L.ngs_stage_times(self.h, ms.ctypes.data_as(C.c_void_p), len(ms)),
              "ngs_stage_times")
        return dict(zip(_lib.STAGES, ms.tolist()))

    # -- scene ---------------------------------------------------------------
    def load_scene(self, scene, attr_dtype: str = "f32", stored=None):
        """``scene``: arrays pos, quat, log_scale, opacity, sh, parent, child_begin,
        child_count, aabb_min, aabb_max. For f16/bf16, ``stored`` maps sh,
        log_scale and opacity to float16 / bfloat16-bit (uint16) arrays."""
        dt = {"f32": _lib.NGS_F32, "f16": _lib.NGS_F16, "bf16": _lib.NGS_BF16}[attr_dtype]
        f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
        i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
        pos, quat = f32(scene.pos), f32(scene.quat)
        if dt == _lib.NGS_F32:
            ls, op, sh = f32(scene.log_scale), f32(scene.opacity), f32(scene.sh)
        else:
            want = np.float16 if dt == _lib.NGS_F16 else np.uint16
            ls = np.ascontiguousarray(stored["log_scale"], dtype=want)
            op = np.ascontiguousarray(stored["opacity"], dtype=want)
            sh = np.ascontiguousarray(stored["sh"], dtype=want)
        par, cb, cc = i32(scene.parent), i32(scene.child_begin), i32(scene.child_count)
        bmin, bmax = f32(scene.aabb_min), f32(scene.aabb_max)
        n = int(par.shape[0])
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        g = _lib.Gaussians(n, p(pos), p(quat), p(ls), p(op), p(sh), dt)
        hh = _lib.Hierarchy(p(par), p(cb), p(cc), p(bmin), p(bmax))
        check(self.L.ngs_load_scene(self.h, C.byref(g), C.byref(hh)), "ngs_load_scene")
        self.attr_dtype = attr_dtype
        self.n_nodes = n

    # -- rendering -----------------------------------------------------------
    def new_images(self, cams) -> list:
        torch = _torch()
        return [torch.empty((3, int(c.height), int(c.width)), dtype=torch.float32,
                            device=f"cuda:{self.device}") for c in cams]

    def render(self, cams, images: Optional[list] = None, stream=None, sync: bool = True):
        """Renders ``cams`` into ``images`` (new CUDA tensors [3, H, W] if None)."""
        if images is None:
            images = self.new_images(cams)
        arr = camera_array(cams)
        ptrs = (C.c_void_p * len(cams))(*[C.c_void_p(t.data_ptr()) for t in images])
        st = _stream_ptr(stream)
        check(self.L.ngs_render(self.h, arr, len(cams), ptrs, st), "ngs_render")
        if sync:
            check(self.L.ngs_synchronize(self.h, st), "ngs_synchronize")
        return images

    def autotune(self, cams, images: Optional[list] = None, reps: int = 3, stream=None) -> dict:
        """Times every (tile, compositing block) shape x staging batch on ``cams``
        and keeps the fastest."""
        if images is None:
            images = self.new_images(cams)
        arr = camera_array(cams)
        ptrs = (C.c_void_p * len(cams))(*[C.c_void_p(t.data_ptr()) for t in images])
        res = _lib.TuneResult()
        check(self.L.ngs_autotune(self.h, arr, len(cams), ptrs, int(reps), _stream_ptr(stream),
                                  C.byref(res)), "ngs_autotune")
        names = [f"{t[0]}x{t[1]}:{k[0]}x{k[1]}/{b}" for t, k in _lib.TUNE_SHAPES
                 for b in _lib.TUNE_BATCHES]
        return {"tile": (res.tile_w, res.tile_h), "cta": (res.cta_w, res.cta_h),
                "batch": res.batch, "ms": dict(zip(names, [round(x, 3) for x in res.ms]))}

    def render_host(self, cams, out: Optional[List[np.ndarray]] = None, stream=None):
        """Renders and copies every image into host arrays [3, H, W] float32."""
        if out is None:
            out = [np.empty((3, int(c.height), int(c.width)), dtype=np.float32) for c in cams]
        arr = camera_array(cams)
        ptrs = (C.c_void_p * len(cams))(*[C.c_void_p(o.ctypes.data) for o in out])
        check(self.L.ngs_render_host(self.h, arr, len(cams), ptrs, _stream_ptr(stream)),
              "ngs_render_host")
        return out

    def render_host_ptrs(self, cams_arr, n, ptrs, stream=None):
        """Lowest-overhead host-buffer call: pre-built camera array and pointers."""
        check(self.L.ngs_render_host(self.h, cams_arr, n, ptrs, _stream_ptr(stream)),
              "ngs_render_host")

    def synchronize(self, stream=None):
        check(self.L.ngs_synchronize(self.h, _stream_ptr(stream)), "ngs_synchronize")

    def stats(self) -> dict:
        s = _lib.Stats()
        check(self.L.ngs_last_stats(self.h, C.byref(s)), "ngs_last_stats")
        return {k: getattr(s, k) for k, _ in _lib.Stats._fields_}

    def slice_occupancy(self, grid, value=None, occ=None, stream=None):
        """GS-slice occupancy of the loaded scene's leaves. ``grid``: any object
        with x0, y0, cell, nx, ny, z0, dz, nz, threshold. Returns (value float32
        CUDA tensor [nz, ny, nx], occupancy uint8 tensor of the same shape)."""
        torch = _torch()
        shape = (int(grid.nz), int(grid.ny), int(grid.nx))
        dev = f"cuda:{self.device}"
        if value is None:
            value = torch.empty(shape, dtype=torch.float32, device=dev)
        if occ is None:
            occ = torch.empty(shape, dtype=torch.uint8, device=dev)
        g = _lib.SliceGrid(float(grid.x0), float(grid.y0), float(grid.cell), int(grid.nx),
                           int(grid.ny), float(grid.z0), float(grid.dz), int(grid.nz),
                           float(grid.threshold))
        check(self.L.ngs_slice_occupancy(self.h, C.byref(g), C.c_void_p(value.data_ptr()),
                                         C.c_void_p(occ.data_ptr()), _stream_ptr(stream)),
              "ngs_slice_occupancy")
        return value, occ

    def nav_fields(self, occ, goals, k_lo: int, k_hi: int, inflate: int, stream=None):
        """Blocked map (uint8 [ny, nx]) and one breadth-first distance field per
        goal (int64 view of uint32 [n_goals, ny, nx]) from an occupancy tensor
        [nz, ny, nx] on the device; ``goals``: (i, j) cells."""
        torch = _torch()
        nz, ny, nx = (int(v) for v in occ.shape)
        g = np.ascontiguousarray(np.asarray(goals, dtype=np.int32).reshape(-1, 2))
        blocked = torch.empty((ny, nx), dtype=torch.uint8, device=occ.device)
        dist = torch.empty((len(g), ny, nx), dtype=torch.int32, device=occ.device)
        check(self.L.ngs_nav_fields(self.h, C.c_void_p(occ.data_ptr()), nx, ny, nz, int(k_lo),
                                    int(k_hi), int(inflate), g.ctypes.data_as(C.c_void_p), len(g),
                                    C.c_void_p(blocked.data_ptr()), C.c_void_p(dist.data_ptr()),
                                    _stream_ptr(stream)), "ngs_nav_fields")
        return blocked, dist

    def nav_paths(self, dist, starts, max_len: int, stream=None):
        """Paths (int32 [n, max_len, 2]) and lengths (int32 [n]) for starts
        (i, j, goal index) descending the fields ``dist`` [n_goals, ny, nx]."""
        torch = _torch()
        n_goals, ny, nx = (int(v) for v in dist.shape)
        s = torch.as_tensor(np.asarray(starts, dtype=np.int32).reshape(-1, 3), device=dist.device)
        n = int(s.shape[0])
        paths = torch.zeros((n, int(max_len), 2), dtype=torch.int32, device=dist.device)
        lens = torch.zeros(n, dtype=torch.int32, device=dist.device)
        check(self.L.ngs_nav_paths(self.h, C.c_void_p(dist.data_ptr()), nx, ny, n_goals,
                                   C.c_void_p(s.data_ptr()), n, int(max_len),
                                   C.c_void_p(paths.data_ptr()), C.c_void_p(lens.data_ptr()),
                                   _stream_ptr(stream)), "ngs_nav_paths")
        return paths, lens

    def select_cut(self, cams, cap: Optional[int] = None, stream=None):
        """Per-camera LOD cuts: (ids int32 CUDA tensor, offsets int64 CUDA tensor)."""
        torch = _torch()
        cap = int(cap if cap is not None else len(cams) * self.n_nodes)
        ids = torch.empty(max(cap, 1), dtype=torch.int32, device=f"cuda:{self.device}")
        off = torch.empty(len(cams) + 1, dtype=torch.int64, device=f"cuda:{self.device}")
        arr = camera_array(cams)
        check(self.L.ngs_select_cut(self.h, arr, len(cams), C.c_void_p(ids.data_ptr()),
                                    C.c_void_p(off.data_ptr()), cap, _stream_ptr(stream)),
              "ngs_select_cut")
        return ids, off

    def select_cut_shared(self, cams, group_begin, frustum: bool = True, guard: float = 0.0,
                          cap: Optional[int] = None, stream=None):
        """One LOD cut per group of cameras (group g = cams[group_begin[g]:
        group_begin[g+1]]), optionally frustum-culled with a guard band of
        ``guard`` pixels: (ids int32 CUDA tensor, offsets int64 CUDA tensor
        [n_groups + 1])."""
        torch = _torch()
        gb = np.ascontiguousarray(group_begin, dtype=np.int32)
        ng = len(gb) - 1
        cap = int(cap if cap is not None else max(ng, 1) * self.n_nodes)
        ids = torch.empty(max(cap, 1), dtype=torch.int32, device=f"cuda:{self.device}")
        off = torch.empty(max(ng, 0) + 1, dtype=torch.int64, device=f"cuda:{self.device}")
        arr = camera_array(cams)
        check(self.L.ngs_select_cut_shared(self.h, arr, len(cams), gb.ctypes.data_as(C.c_void_p),
                                           ng, _lib.CUT_FRUSTUM if frustum else 0, float(guard),
                                           C.c_void_p(ids.data_ptr()), C.c_void_p(off.data_ptr()),
                                           cap, _stream_ptr(stream)), "ngs_select_cut_shared")
        return ids, off

    def tile_lists(self, cam_index: int, n_tiles: int, cap: int):
        """(ranges [tiles, 2] int64, node ids int32) of one camera of the last
        render, which must have been made with set_node_ids(True)."""
        ranges = np.zeros((n_tiles, 2), dtype=np.int64)
        nodes = np.zeros(max(cap, 1), dtype=np.int32)
        npairs = C.c_int64()
        check(self.L.ngs_debug_tile_lists(self.h, cam_index, ranges.ctypes.data_as(C.c_void_p),
                                          nodes.ctypes.data_as(C.c_void_p), cap,
                                          C.byref(npairs)), "ngs_debug_tile_lists")
        return ranges, nodes[:npairs.value]

    def tile_ranges(self, cam_index: int, n_tiles: int, cap: int):
        """(ranges [tiles, 2] int64, number of pairs) of one camera of the
        last render; needs no node ids."""
        ranges = np.zeros((n_tiles, 2), dtype=np.int64)
        npairs = C.c_int64()
        check(self.L.ngs_debug_tile_lists(self.h, cam_index, ranges.ctypes.data_as(C.c_void_p),
                                          None, cap, C.byref(npairs)), "ngs_debug_tile_lists")
        return ranges, npairs.value

    def sort_pairs(self, keys, vals, begin_bit: int = 0, end_bit: Optional[int] = None,
                   stream=None):
        """Stable radix sort in place of CUDA tensors keys (uint32/int32 or
        uint64/int64 bit patterns) and vals (32-bit)."""
        kb = keys.element_size()
        end_bit = 8 * kb if end_bit is None else end_bit
        check(self.L.ngs_sort_pairs(self.h, C.c_void_p(keys.data_ptr()),
                                    C.c_void_p(vals.data_ptr()), keys.numel(), kb, begin_bit,
                                    end_bit, _stream_ptr(stream)), "ngs_sort_pairs")

    def scan_u32(self, x, out=None, stream=None):
        torch = _torch()
        out = torch.empty_like(x) if out is None else out
        total = torch.zeros(1, dtype=x.dtype, device=x.device)
        check(self.L.ngs_scan_u32(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                  x.numel(), C.c_void_p(total.data_ptr()), _stream_ptr(stream)),
              "ngs_scan_u32")
        return out, total


class Server:
    """Continuous-batching render service over a Renderer's resident scene."""

    def __init__(self, renderer: Renderer, lanes: int = 2, max_cams: int = 64,
                 pair_budget: int = 0, pairs_per_pixel: float = 0.0,
                 lane_record_capacity: int = 0, lane_pair_capacity: int = 0):
        self.L = renderer.L
        self.renderer = renderer
        cfg = _lib.ServerConfig(int(lanes), int(max_cams), int(pair_budget), float(pairs_per_pixel),
                                int(lane_record_capacity), int(lane_pair_capacity))
        h = C.c_void_p()
        _torch().cuda.set_device(renderer.device)
        check(self.L.ngs_server_start(renderer.h, C.byref(cfg), C.byref(h)), "ngs_server_start")
        self.h = h

    def submit(self, cam, image) -> int:
        t = C.c_uint64()
        check(self.L.ngs_server_submit(self.h, C.byref(camera_struct(cam)),
                                       C.c_void_p(image.data_ptr()), C.byref(t)),
              "ngs_server_submit")
        return t.value

    def submit_struct(self, cam_struct, image_ptr: int) -> int:
        t = C.c_uint64()
        check(self.L.ngs_server_submit(self.h, C.byref(cam_struct), C.c_void_p(image_ptr),
                                       C.byref(t)), "ngs_server_submit")
        return t.value

    def poll(self, ticket: int):
        done, lat = C.c_int32(), C.c_double()
        check(self.L.ngs_server_poll(self.h, ticket, C.byref(done), C.byref(lat)), "ngs_server_poll")
        return bool(done.value), lat.value

    def wait_all(self, timeout_ms: int = 600_000):
        check(self.L.ngs_server_wait_all(self.h, int(timeout_ms)), "ngs_server_wait_all")

    def stats(self) -> dict:
        s = _lib.ServerStats()
        check(self.L.ngs_server_stats(self.h, C.byref(s)), "ngs_server_stats")
        return {k: getattr(s, k) for k, _ in _lib.ServerStats._fields_}

    def stop(self):
        if getattr(self, "h", None):
            check(self.L.ngs_server_stop(self.h), "ngs_server_stop")
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
