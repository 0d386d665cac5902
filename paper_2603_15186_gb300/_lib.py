"""ctypes declarations of the C ABI in include/ngs.h (names and layouts match)."""
import ctypes as C
import os

from . import build as _build

NGS_OK = 0
STATUS_NAMES = {0: "NGS_OK", 1: "NGS_ERR_INVALID_ARG", 2: "NGS_ERR_INVALID_HIERARCHY",
                3: "NGS_ERR_OUT_OF_MEMORY", 4: "NGS_ERR_CAPACITY", 5: "NGS_ERR_CUDA",
                6: "NGS_ERR_DEVICE_TIMEOUT", 7: "NGS_ERR_NOT_LOADED"}
NGS_F32, NGS_F16, NGS_BF16 = 0, 1, 2
NGS_MODE_BATCHED, NGS_MODE_PLAIN = 0, 1
NGS_OPT_MODE, NGS_OPT_TILE_W, NGS_OPT_TILE_H, NGS_OPT_BATCH, NGS_OPT_GRAPH = 1, 2, 3, 4, 5
NGS_OPT_STAGE_TIMING = 6
NGS_OPT_BLOCK_CULL = 7
NGS_OPT_CTA_W, NGS_OPT_CTA_H = 8, 9
NGS_OPT_PAIRS_PER_PIXEL = 10
NGS_OPT_LOD_BLEND = 11
NGS_OPT_COMPOSITE_ORDER = 12
NGS_OPT_NODE_IDS = 13
# (binning tile, compositing block) candidates of ngs_autotune, in its order
TUNE_SHAPES = [((8, 8), (8, 8)), ((16, 8), (16, 8)), ((16, 16), (16, 16)), ((16, 32), (16, 32)),
               ((32, 16), (32, 16)), ((32, 32), (32, 32)), ((16, 16), (16, 8)),
               ((16, 32), (16, 16)), ((32, 16), (16, 16)), ((32, 32), (16, 16)),
               ((32, 32), (32, 16)), ((32, 32), (16, 8))]
TUNE_BATCHES = [64, 128, 256]
STAGES = ["cut_preprocess", "gather_keys", "depth_hist", "depth_pass0", "depth_pass1", "depth_pass2",
          "depth_pass3", "pair_offsets", "duplicate", "tile_hist", "tile_pass0", "tile_pass1",
          "tile_pass2", "ranges", "composite"]

# every entry point include/ngs.h declares
EXPORTS = ["ngs_strerror", "ngs_create", "ngs_destroy", "ngs_set_option", "ngs_load_scene",
           "ngs_select_cut", "ngs_render", "ngs_render_host", "ngs_synchronize",
           "ngs_last_stats", "ngs_stage_times", "ngs_debug_tile_lists", "ngs_sort_pairs",
           "ngs_scan_u32", "ngs_sort_pairs_static", "ngs_sort_pairs_static_status",
           "ngs_autotune", "ngs_server_start",
           "ngs_server_submit", "ngs_server_poll", "ngs_server_wait_all", "ngs_server_stats",
           "ngs_server_stop", "ngs_selftest_wait_timeout", "ngs_slice_occupancy",
           "ngs_nav_fields", "ngs_nav_paths", "ngs_select_cut_shared"]
CUT_FRUSTUM = 1


class NgsError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("R_wc", C.c_float * 9), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32), ("tau", C.c_float)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("pos", C.c_void_p), ("quat", C.c_void_p),
                ("log_scale", C.c_void_p), ("opacity", C.c_void_p), ("sh", C.c_void_p),
                ("attr_dtype", C.c_int32)]


class Hierarchy(C.Structure):
    _fields_ = [("parent", C.c_void_p), ("child_begin", C.c_void_p), ("child_count", C.c_void_p),
                ("aabb_min", C.c_void_p), ("aabb_max", C.c_void_p)]


class Config(C.Structure):
    _fields_ = [("device", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("batch", C.c_int32), ("cut_capacity", C.c_int64),
                ("record_capacity", C.c_int64), ("pair_capacity", C.c_int64),
                ("max_tiles_per_batch", C.c_int32), ("reserved", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("cta_w", C.c_int32),
                ("cta_h", C.c_int32), ("batch", C.c_int32), ("reserved", C.c_int32),
                ("ms", C.c_float * (3 * len(TUNE_SHAPES)))]


class SliceGrid(C.Structure):
    _fields_ = [("x0", C.c_float), ("y0", C.c_float), ("cell", C.c_float), ("nx", C.c_int32),
                ("ny", C.c_int32), ("z0", C.c_float), ("dz", C.c_float), ("nz", C.c_int32),
                ("threshold", C.c_float)]


class ServerConfig(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("max_cams", C.c_int32), ("pair_budget", C.c_int64),
                ("pairs_per_pixel", C.c_double), ("lane_record_capacity", C.c_int64),
                ("lane_pair_capacity", C.c_int64)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("launches", C.c_int64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("mean_ms", C.c_double), ("max_ms", C.c_double), ("mpix", C.c_double),
                ("span_s", C.c_double), ("requeued", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("cut_total", C.c_int64), ("visible_total", C.c_int64),
                ("pair_total", C.c_int64), ("records_staged", C.c_int64),
                ("evaluations", C.c_int64), ("sub_batches", C.c_int32),
                ("graph_replayed", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("batch", C.c_int32), ("mode", C.c_int32), ("kernels", C.c_int32),
                ("cta_w", C.c_int32), ("cta_h", C.c_int32), ("reserved", C.c_int32),
                ("composite_tail_ms", C.c_double), ("candidate_total", C.c_int64)]


_lib = None


def load(build_if_missing: bool = True):
    """Loads libngs.so (building it in-tree first if needed). Raises if the
    library cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libngs.so not found at {path}")
    L = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    L.ngs_strerror.restype = C.c_char_p
    L.ngs_strerror.argtypes = [i32]
    L.ngs_create.restype = i32
    L.ngs_create.argtypes = [C.POINTER(Config), C.POINTER(vp)]
    L.ngs_destroy.restype = i32
    L.ngs_destroy.argtypes = [vp]
    L.ngs_set_option.restype = i32
    L.ngs_set_option.argtypes = [vp, i32, i64]
    L.ngs_load_scene.restype = i32
    L.ngs_load_scene.argtypes = [vp, C.POINTER(Gaussians), C.POINTER(Hierarchy)]
    L.ngs_select_cut.restype = i32
    L.ngs_select_cut.argtypes = [vp, C.POINTER(Camera), i32, vp, vp, i64, vp]
    L.ngs_select_cut_shared.restype = i32
    L.ngs_select_cut_shared.argtypes = [vp, C.POINTER(Camera), i32, vp, i32, C.c_uint32,
                                        C.c_float, vp, vp, i64, vp]
    L.ngs_render.restype = i32
    L.ngs_render.argtypes = [vp, C.POINTER(Camera), i32, C.POINTER(vp), vp]
    L.ngs_render_host.restype = i32
    L.ngs_render_host.argtypes = [vp, C.POINTER(Camera), i32, C.POINTER(vp), vp]
    L.ngs_synchronize.restype = i32
    L.ngs_synchronize.argtypes = [vp, vp]
    L.ngs_last_stats.restype = i32
    L.ngs_last_stats.argtypes = [vp, C.POINTER(Stats)]
    L.ngs_stage_times.restype = i32
    L.ngs_stage_times.argtypes = [vp, vp, i32]
    L.ngs_debug_tile_lists.restype = i32
    L.ngs_debug_tile_lists.argtypes = [vp, i32, vp, vp, i64, C.POINTER(i64)]
    L.ngs_sort_pairs.restype = i32
    L.ngs_sort_pairs.argtypes = [vp, vp, vp, i64, i32, i32, i32, vp]
    L.ngs_sort_pairs_static.restype = i32
    L.ngs_sort_pairs_static.argtypes = [vp, vp, i64, i32, i32, i32, vp]
    L.ngs_sort_pairs_static_status.restype = i32
    L.ngs_sort_pairs_static_status.argtypes = [vp]
    L.ngs_nav_fields.restype = i32
    L.ngs_nav_fields.argtypes = [vp, vp, i32, i32, i32, i32, i32, i32, vp, i32, vp, vp, vp]
    L.ngs_nav_paths.restype = i32
    L.ngs_nav_paths.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, vp, vp, vp]
    L.ngs_slice_occupancy.restype = i32
    L.ngs_slice_occupancy.argtypes = [vp, C.POINTER(SliceGrid), vp, vp, vp]
    L.ngs_autotune.restype = i32
    L.ngs_autotune.argtypes = [vp, C.POINTER(Camera), i32, C.POINTER(vp), i32, vp,
                               C.POINTER(TuneResult)]
    L.ngs_server_start.restype = i32
    L.ngs_server_start.argtypes = [vp, C.POINTER(ServerConfig), C.POINTER(vp)]
    L.ngs_server_submit.restype = i32
    L.ngs_server_submit.argtypes = [vp, C.POINTER(Camera), vp, C.POINTER(C.c_uint64)]
    L.ngs_server_poll.restype = i32
    L.ngs_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(i32), C.POINTER(C.c_double)]
    L.ngs_server_wait_all.restype = i32
    L.ngs_server_wait_all.argtypes = [vp, i32]
    L.ngs_server_stats.restype = i32
    L.ngs_server_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.ngs_server_stop.restype = i32
    L.ngs_server_stop.argtypes = [vp]
    L.ngs_selftest_wait_timeout.restype = i32
    L.ngs_selftest_wait_timeout.argtypes = [vp, vp]
    L.ngs_scan_u32.restype = i32
    L.ngs_scan_u32.argtypes = [vp, vp, vp, i64, vp, vp]
    _lib = L
    return L


def check(status, where=""):
    if status != NGS_OK:
        raise NgsError(status, where)
