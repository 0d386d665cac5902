// Host runtime behind the C ABI of include/ngs.h: context and device
// residency of the scene, validation, the sub-batch planner, the plain
// (per-view, host-synchronised) and batched (device-sized, graph-replayed)
// render paths, and the standalone sort/scan entry points.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "ngs_internal.cuh"
#include "cut.h"
#include "nav.h"

using namespace ngs;

namespace {

constexpr uint32_t kEpochStride = 32;   // epoch values reserved per sub-batch
constexpr int kMaxCamsPerBatch = 1024;
// ngs_select_cut takes the camera-blocked two-pass cut from this many cameras on
constexpr int kCutBlockedMinCams = 4;
constexpr int kMaxCamsPerCall = 1 << 16;
constexpr int kTuneShapes = NGS_TUNE_SHAPES;
// renders of one ngs_render_host call after a pair-buffer overflow
constexpr int kCapacityRetries = 4;

struct SubBatch {
    int c0, c1;          // cameras [c0, c1)
    uint32_t n_tiles;
    int tile_passes;     // radix passes over the tile id
};

float half_to_float(uint16_t h) {
    const uint32_t s = (uint32_t)(h >> 15) << 31;
    uint32_t e = (h >> 10) & 0x1f, m = h & 0x3ff;
    uint32_t bits;
    if (e == 0) {
        if (m == 0) {
            bits = s;
        } else {  // subnormal: renormalise
            int sh = 0;
            while (!(m & 0x400)) { m <<= 1; ++sh; }
            m &= 0x3ff;
            bits = s | ((uint32_t)(127 - 15 - sh + 1) << 23) | (m << 13);
        }
    } else if (e == 31) {
        bits = s | 0x7f800000u | (m << 13);
    } else {
        bits = s | ((e - 15 + 127) << 23) | (m << 13);
    }
    float f;
    std::memcpy(&f, &bits, 4);
    return f;
}

float bf16_to_float(uint16_t h) {
    const uint32_t bits = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &bits, 4);
    return f;
}

}  // namespace

struct ngs_ctx {
    int device = 0;
    int num_sms = 0;
    ngs_config cfg{};
    int mode = NGS_MODE_BATCHED;
    int tile_w = 16, tile_h = 16, batch = 128;
    int cta_w = 0, cta_h = 0;          // block one compositing CTA covers (0: the tile)
    bool use_graph = true;
    bool block_cull = true;
    bool lod_blend = false;            // level-of-detail blending toward parents
    bool composite_order = true;       // batched compositing takes tiles longest list first
    bool node_ids = false;             // keep each record's node id (ngs_debug_tile_lists)
    bool last_node_ids = false;        // the last render kept them
    SceneDev scene;
    bool loaded = false;
    bool owns_scene = true;           // false for serving lanes sharing a scene
    uint64_t scene_version = 0;

    Work w;
    bool work_ready = false;
    uint32_t *stats_dev = nullptr;     // per sub-batch: cut, visible, pairs, pad
    int stats_cap = 0;
    uint32_t *cut_off32 = nullptr;     // scratch for ngs_select_cut offsets
    CutCam *cut_cams = nullptr;        // ngs_select_cut_shared: cameras and groups
    int32_t *cut_groups = nullptr;
    uint32_t *cut_counts = nullptr;    // many-camera ngs_select_cut: (camera, block) counts
    uint32_t *cut_poff = nullptr;      // and their scanned offsets

    // occupancy-derived persistent grids
    int grid_cut = 0, grid_pre = 0, grid_sort32 = 0, grid_sort64 = 0, grid_scan = 0,
        grid_dup = 0, grid_ranges = 0;

    // graph cache
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<int64_t> gkey;
    uint64_t epoch_used = 0;

    // last render
    std::vector<SubBatch> last_plan;
    std::vector<DevCamera> host_cams;
    ngs_stats stats{};
    ngs_status latched = NGS_OK;
    bool stats_pending = false;
    double pairs_per_pixel = 48.0;     // planner estimate, raised from observations

    // optional per-kernel timing: kMarks events per sub-batch (or per camera
    // in the plain path), recorded on the render stream / into the graph
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    int ev_groups = 0;
    int kernels_per_render = 0;

    // batched renders record ev_sb[k] once sub-batch k's images are complete
    // (into the graph as external event nodes), so that ngs_render_host can
    // copy a sub-batch's images to the host while the next ones render, on
    // copy_stream; ev_copied joins the copies back into the caller's stream
    std::vector<cudaEvent_t> ev_sb;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied = nullptr;

    // navigation scratch (occupied-any map, goals, frontier queues), grown on demand
    unsigned char *nav_tmp = nullptr;
    size_t nav_tmp_bytes = 0;

    // standalone sort/scan scratch
    void *sort_tmp_keys = nullptr;
    uint32_t *sort_tmp_vals = nullptr;
    int64_t sort_tmp_cap = 0;
};

namespace {

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e__ = (call);                                                           \
        if (e__ != cudaSuccess) {                                                           \
            std::fprintf(stderr, "ngs: %s failed: %s (%s:%d)\n", #call,                    \
                         cudaGetErrorString(e__), __FILE__, __LINE__);                      \
            return e__ == cudaErrorMemoryAllocation ? NGS_ERR_OUT_OF_MEMORY : NGS_ERR_CUDA; \
        }                                                                                   \
    } while (0)

template <typename T>
ngs_status dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return NGS_ERR_OUT_OF_MEMORY;
    }
    return NGS_OK;
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

__global__ void k_bump_epoch(uint32_t *epoch, uint32_t inc) { *epoch += inc; }

__global__ void k_offsets_to_i64(const uint32_t *in, int64_t *out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = in[i];
}

// One look-back whose predecessor never publishes in this epoch: the bounded
// wait gives up and latches kErrTimeout (failure-detection self-test).
__global__ void k_wait_probe(const uint64_t *status, const uint32_t *epoch_ptr, int *err) {
    uint32_t prev = 0;
    look_back(status, 1, 1, *epoch_ptr + kEpochStride - 1, &prev, err);
}

// per sub-batch: cut, visible and pair totals, and the cut + preprocess
// candidates (slots allocated, the low word of the 64-bit counter)
__global__ void k_copy_stats(const uint32_t *counters, uint32_t *stats) {
    if (threadIdx.x < 3) stats[threadIdx.x] = counters[threadIdx.x];
    if (threadIdx.x == 3) stats[3] = counters[CNT_ALLOC];
}

void free_work(ngs_ctx *c) {
    Work &w = c->w;
    dfree(w.counters); dfree(w.epoch); dfree(w.status); dfree(w.err); dfree(w.cut_ids);
    dfree(w.cut_off); dfree(w.vis_count); dfree(w.part_list); dfree(w.group_list); dfree(w.part_info); dfree(w.part_pos); dfree(w.rec); dfree(w.rect); dfree(w.rect_sorted); dfree(w.node_id); dfree(w.poff); dfree(w.chunk_first); dfree(w.ranges);
    dfree(w.hist); dfree(w.cams); dfree(w.work64); dfree(w.order);
    for (int i = 0; i < 2; ++i) {
        dfree(w.dkey[i]); dfree(w.didx[i]); dfree(w.pkey[i]); dfree(w.pval[i]);
    }
    dfree(c->stats_dev);
    dfree(c->cut_off32);
    dfree(c->cut_cams);
    dfree(c->cut_groups);
    dfree(c->cut_counts);
    dfree(c->cut_poff);
    c->w = Work();
    c->stats_dev = nullptr;
    c->cut_off32 = nullptr;
    c->cut_cams = nullptr;
    c->cut_groups = nullptr;
    c->cut_counts = nullptr;
    c->cut_poff = nullptr;
    c->work_ready = false;
}

void free_scene(ngs_ctx *c) {
    SceneDev &s = c->scene;
    if (c->owns_scene) {
        dfree(s.box_lo); dfree(s.box_hi); dfree(s.pos4); dfree(s.quat); dfree(s.sop); dfree(s.sh);
        dfree(s.blk_lo); dfree(s.blk_hi); dfree(s.blk_lo_b); dfree(s.blk_hi_b);
    }
    c->scene = SceneDev();
    c->loaded = false;
}

void drop_graph(ngs_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gkey.clear();
}

// Event marks inside one sub-batch; stage k runs between mark k and k + 1.
enum : int {
    MK_START = 0, MK_CUT = 1, MK_PRE = 2, MK_DHIST = 3, MK_DPASS0 = 4, MK_POFF = 8, MK_DUP = 9,
    MK_THIST = 10, MK_TPASS0 = 11, MK_RANGES = 14, MK_COMPOSITE = 15, kMarks = 16
};

ngs_status ensure_events(ngs_ctx *c, int groups) {
    if (!c->timing) return NGS_OK;
    const int need = groups * kMarks;
    while ((int)c->ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->ev.push_back(e);
    }
    c->ev_groups = groups;
    return NGS_OK;
}

// Records e on st; under stream capture as an external event node (which the
// host and other streams can wait on after each graph launch). The external
// flag is only accepted while the stream is capturing.
void record_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

ngs_status ensure_sb_events(ngs_ctx *c, int n) {
    while ((int)c->ev_sb.size() < n) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        c->ev_sb.push_back(e);
    }
    return NGS_OK;
}

void mark(ngs_ctx *c, int group, int k, cudaStream_t st) {
    // under stream capture an event-record node that the host can wait on and
    // time after each graph launch
    if (c->timing) record_event(c->ev[(size_t)group * kMarks + k], st);
}

struct SortHook {
    ngs_ctx *c;
    int group, first_mark;
    cudaStream_t st;
};

void sort_hook(void *user, int step) {
    SortHook *h = (SortHook *)user;
    mark(h->c, h->group, h->first_mark + step, h->st);
}

ngs_status ensure_work(ngs_ctx *c) {
    if (c->work_ready) return NGS_OK;
    Work &w = c->w;
    w.cut_cap = c->cfg.cut_capacity;
    w.rec_cap = c->cfg.record_capacity;
    w.pair_cap = c->cfg.pair_capacity;
    w.ranges_cap = 1 << 24;
    w.cams_cap = kMaxCamsPerCall;
    const int64_t nblk = (c->scene.n + cut_partition_nodes() - 1) / cut_partition_nodes();
    int64_t sw = std::max<int64_t>(nblk * kMaxCamsPerBatch, 1);
    sw = std::max<int64_t>(sw, (std::max(w.rec_cap, w.pair_cap) + sort_partition() - 1) /
                                   sort_partition() * 256);
    sw = std::max<int64_t>(sw, (w.rec_cap + scan_partition() - 1) / scan_partition());
    w.status_words = sw;
    ngs_status st = NGS_OK;
    auto A = [&](ngs_status s) { if (st == NGS_OK) st = s; };
    A(dalloc(&w.counters, N_COUNTERS));
    A(dalloc(&w.epoch, 1));
    A(dalloc(&w.status, (size_t)sw));
    A(dalloc(&w.err, 1));
    A(dalloc(&w.cut_ids, (size_t)w.cut_cap));
    A(dalloc(&w.cut_off, kMaxCamsPerBatch + 1));
    A(dalloc(&w.vis_count, kMaxCamsPerBatch));
    w.part_cap = std::max<int64_t>(1, (c->scene.n + cutpre_partition_nodes() - 1) /
                                          cutpre_partition_nodes() * kMaxCamsPerBatch);
    A(dalloc(&w.part_list, (size_t)w.part_cap));
    A(dalloc(&w.group_list, (size_t)w.part_cap));
    A(dalloc(&w.part_info, (size_t)w.part_cap));
    A(dalloc(&w.part_pos, (size_t)w.part_cap));
    A(dalloc((unsigned char **)&w.rec, (size_t)w.rec_cap * sizeof(Rec32)));
    A(dalloc(&w.rect, (size_t)w.rec_cap));
    A(dalloc(&w.rect_sorted, (size_t)w.rec_cap));
    A(dalloc(&w.poff, (size_t)w.rec_cap));
    A(dalloc(&w.chunk_first, (size_t)dup_chunks(w.pair_cap)));
    for (int i = 0; i < 2; ++i) {
        A(dalloc(&w.dkey[i], (size_t)w.rec_cap));
        A(dalloc(&w.didx[i], (size_t)w.rec_cap));
        A(dalloc(&w.pkey[i], (size_t)w.pair_cap));
        A(dalloc(&w.pval[i], (size_t)w.pair_cap));
    }
    A(dalloc(&w.ranges, (size_t)w.ranges_cap));
    A(dalloc(&w.hist, 8 * 256));
    A(dalloc(&w.cams, (size_t)w.cams_cap));
    c->stats_cap = 4096;
    A(dalloc(&c->stats_dev, (size_t)c->stats_cap * 4));
    A(dalloc(&c->cut_off32, kMaxCamsPerBatch + 1));
    A(dalloc(&c->cut_cams, kMaxCamsPerBatch));
    A(dalloc(&c->cut_groups, kMaxCamsPerBatch + 1));
    A(dalloc(&c->cut_counts, (size_t)(nblk * kMaxCamsPerBatch)));
    A(dalloc(&c->cut_poff, (size_t)(nblk * kMaxCamsPerBatch)));
    A(dalloc(&w.work64, kWork64Words));
    A(dalloc(&w.order, (size_t)w.ranges_cap));
    if (st != NGS_OK) {
        free_work(c);
        return st;
    }
    CK(cudaMemset(w.status, 0, (size_t)sw * sizeof(uint64_t)));
    CK(cudaMemset(w.epoch, 0, sizeof(uint32_t)));
    CK(cudaMemset(w.err, 0, sizeof(int)));
    CK(cudaMemset(w.counters, 0, N_COUNTERS * sizeof(uint32_t)));
    CK(cudaDeviceSynchronize());
    c->epoch_used = 0;
    c->work_ready = true;
    return NGS_OK;
}

// Keeps the 30-bit epoch space from wrapping: once most of it is used, the
// status words are cleared (outside any graph) and the epoch restarts.
ngs_status epoch_guard(ngs_ctx *c, cudaStream_t st, uint64_t need) {
    if (c->epoch_used + need < (1ull << 29)) {
        c->epoch_used += need;
        return NGS_OK;
    }
    CK(cudaStreamSynchronize(st));
    CK(cudaMemset(c->w.status, 0, (size_t)c->w.status_words * sizeof(uint64_t)));
    CK(cudaMemset(c->w.epoch, 0, sizeof(uint32_t)));
    CK(cudaDeviceSynchronize());
    c->epoch_used = need;
    return NGS_OK;
}

// tile shapes the compositing kernel is built for
bool tile_supported(int w, int h) {
    return (w == 8 && h == 8) || (w == 16 && h == 8) || (w == 16 && h == 16) ||
           (w == 16 && h == 32) || (w == 32 && h == 16) || (w == 32 && h == 32);
}

// block one compositing CTA covers: the tile itself, or a compiled shape that
// splits the tile into equal blocks
int cta_w_of(const ngs_ctx *c) { return c->cta_w > 0 ? c->cta_w : c->tile_w; }
int cta_h_of(const ngs_ctx *c) { return c->cta_h > 0 ? c->cta_h : c->tile_h; }
bool split_supported(const ngs_ctx *c) {
    const int w = cta_w_of(c), h = cta_h_of(c);
    return tile_supported(w, h) && c->tile_w % w == 0 && c->tile_h % h == 0;
}

constexpr int kMaxImageSide = 32768;
// the binning stages pack tile coordinates (tiles of at least 8 pixels) and a
// launch's camera index into 8 bytes (pack_rect)
static_assert(kMaxImageSide / 8 <= (int)kRectCoordMax && kMaxCamsPerBatch <= 65536,
              "packed tile rectangle");

bool camera_ok(const ngs_camera &k) {
    if (k.width <= 0 || k.height <= 0 || k.width > kMaxImageSide || k.height > kMaxImageSide)
        return false;
    const float v[] = {k.pos[0], k.pos[1], k.pos[2], k.fx, k.fy, k.cx, k.cy, k.tau};
    for (float f : v)
        if (!std::isfinite(f)) return false;
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(k.R_wc[i])) return false;
    return k.fx > 0 && k.fy > 0 && k.tau >= 0;
}

void fill_cam(DevCamera &d, const ngs_camera &k, int tw, int th, float *image) {
    std::memset(&d, 0, sizeof(d));
    for (int i = 0; i < 9; ++i) d.R[i] = k.R_wc[i];
    for (int i = 0; i < 3; ++i) {
        d.pos[i] = k.pos[i];
        d.posd[i] = (double)k.pos[i];
        d.Rz[i] = (double)k.R_wc[6 + i];
    }
    d.fx = k.fx; d.fy = k.fy; d.cx = k.cx; d.cy = k.cy; d.tau = k.tau;
    d.width = k.width; d.height = k.height;
    d.tiles_x = (k.width + tw - 1) / tw;
    d.tiles_y = (k.height + th - 1) / th;
    d.image = image;
    // cross products of the rows of R_wc (float64, then rounded)
    auto cross = [&](int a, int b, float *out) {
        const double ax = k.R_wc[3 * a], ay = k.R_wc[3 * a + 1], az = k.R_wc[3 * a + 2];
        const double bx = k.R_wc[3 * b], by = k.R_wc[3 * b + 1], bz = k.R_wc[3 * b + 2];
        out[0] = (float)(ay * bz - az * by);
        out[1] = (float)(az * bx - ax * bz);
        out[2] = (float)(ax * by - ay * bx);
    };
    cross(0, 1, d.X01);
    cross(0, 2, d.X02);
    cross(2, 1, d.X21);
}

// The five planes of the camera's view volume widened by `guard` pixels, in
// world terms: a_k = R^T m_k for the camera-frame normals m_k of the near,
// left, right, top and bottom half-spaces m_k . t + b_k >= 0.
void fill_cut_cam(CutCam &d, const ngs_camera &k, float guard) {
    std::memset(&d, 0, sizeof(d));
    const double g = guard, W = k.width, H = k.height;
    const double m[5][3] = {{0.0, 0.0, 1.0},
                            {k.fx, 0.0, k.cx + g},
                            {-k.fx, 0.0, W + g - k.cx},
                            {0.0, k.fy, k.cy + g},
                            {0.0, -k.fy, H + g - k.cy}};
    for (int j = 0; j < 5; ++j)
        for (int i = 0; i < 3; ++i)
            d.a[j][i] = (float)(m[j][0] * k.R_wc[i] + m[j][1] * k.R_wc[3 + i] +
                                m[j][2] * k.R_wc[6 + i]);
    d.b0 = -kNearZ;
    for (int i = 0; i < 3; ++i) d.pos[i] = k.pos[i];
    d.fx = k.fx;
    d.tau = k.tau;
}

int bits_for(uint32_t n) {
    int b = 0;
    while (b < 32 && ((uint64_t)1 << b) < n) ++b;
    return b;
}

// Splits cameras into sub-batches: at most kMaxCamsPerBatch cameras, at most
// max_tiles tiles (one camera alone may exceed it), cut and record bounds
// (a camera's cut is an antichain of the tree, so it holds at most as many
// nodes as the tree has leaves) and an estimate of the pairs.
std::vector<SubBatch> plan(ngs_ctx *c, std::vector<DevCamera> &cams, int max_cams_per_batch) {
    std::vector<SubBatch> out;
    const int64_t per_cam = c->scene.n_leaves > 0 ? c->scene.n_leaves : c->scene.n;
    const int64_t max_tiles = c->cfg.max_tiles_per_batch;
    // the visible Gaussians of a sub-batch (at most per_cam per camera) share
    // the record slots
    const int64_t cams_by_cut =
        std::max<int64_t>(1, c->w.rec_cap / std::max<int64_t>(per_cam, 1));
    int i = 0;
    const int N = (int)cams.size();
    while (i < N) {
        SubBatch sb{i, i, 0, 0};
        int64_t tiles = 0;
        double pairs = 0;
        while (sb.c1 < N) {
            const DevCamera &d = cams[sb.c1];
            const int64_t t = (int64_t)d.tiles_x * d.tiles_y;
            const double p = c->pairs_per_pixel * (double)d.width * d.height;
            const int cnt = sb.c1 - sb.c0;
            if (cnt > 0 && (tiles + t > max_tiles || cnt + 1 > max_cams_per_batch ||
                            cnt + 1 > cams_by_cut || pairs + p > (double)c->w.pair_cap))
                break;
            cams[sb.c1].tile_base = (uint32_t)tiles;
            tiles += t;
            pairs += p;
            ++sb.c1;
        }
        sb.n_tiles = (uint32_t)tiles;
        sb.tile_passes = (bits_for(sb.n_tiles) + 7) / 8;
        out.push_back(sb);
        i = sb.c1;
    }
    return out;
}

// Enqueues the whole pipeline of one sub-batch with device-resident counts
// (no host synchronisation): suitable for graph capture.
void enqueue_batched(ngs_ctx *c, const SubBatch &sb, int sb_index, cudaStream_t st) {
    Work &w = c->w;
    const int nc = sb.c1 - sb.c0;
    const DevCamera *cams = w.cams + sb.c0;
    mark(c, sb_index, MK_START, st);
    cudaMemsetAsync(w.counters, 0, N_COUNTERS * sizeof(uint32_t), st);
    cudaMemsetAsync(w.ranges, 0, (size_t)sb.n_tiles * sizeof(uint2), st);
    k_bump_epoch<<<1, 1, 0, st>>>(w.epoch, kEpochStride);
    uint32_t eo = 0;
    launch_cutpre(c->scene, cams, nc, w.rec, w.rec_cap, w.dkey[1], w.rect,
                  c->node_ids ? w.node_id : nullptr, w.vis_count,
                  w.counters, w.part_list, w.group_list, w.part_info, w.err, c->tile_w, c->tile_h,
                  c->block_cull ? 1 : 0, c->lod_blend ? 1 : 0, c->grid_pre, st);
    mark(c, sb_index, MK_CUT, st);
    launch_gather_keys(w.vis_count, nc, c->scene, w.part_info, w.part_pos, w.part_list,
                       w.dkey[1], w.dkey[0], w.didx[0], w.counters, w.rec_cap, w.hist, w.err,
                       c->num_sms * 8, st);
    mark(c, sb_index, MK_PRE, st);
    SortHook dh{c, sb_index, MK_DHIST, st};
    SortArgs da{};
    da.keys[0] = w.dkey[0]; da.keys[1] = w.dkey[1];
    da.vals[0] = w.didx[0]; da.vals[1] = w.didx[1];
    da.n_dev = w.counters + CNT_VIS; da.n_host = -1; da.n_max = w.rec_cap;
    da.key_bytes = 4; da.begin_bit = 0; da.end_bit = 32; da.vals_identity = false;
    da.hist = w.hist; da.tickets = w.counters + TK_SORT0; da.status = w.status;
    da.epoch = w.epoch; da.epoch_off = eo; da.err = w.err;
    da.hook = c->timing ? sort_hook : nullptr; da.hook_user = &dh;
    da.skip_last_keys = true;   // later stages read the record order only
    da.hist_ready = true;       // counted by the key gather
    launch_sort(da, c->grid_sort32, st);
    eo += 4;
    const int dsel = 4 & 1;  // four passes: the result is back in buffer 0
    // the tile sort's digit histograms are counted by the offset scan
    cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * 256 * 3, st);
    launch_pair_offsets(w.rect, w.didx[dsel], w.counters + CNT_VIS, w.poff, w.counters,
                        w.pair_cap, w.counters + TK_SCAN, w.status, w.epoch, eo++, w.err,
                        w.chunk_first, w.rect_sorted, cams, w.hist, sb.tile_passes,
                        c->grid_scan, st);
    mark(c, sb_index, MK_POFF, st);
    launch_duplicate(w.rect_sorted, w.didx[dsel], w.poff, w.chunk_first, w.counters + CNT_VIS,
                     w.counters + CNT_PAIRS, w.pair_cap, cams, w.pkey[0], w.pval[0], w.err,
                     c->grid_dup, st);
    mark(c, sb_index, MK_DUP, st);
    int psel = 0;
    SortHook th{c, sb_index, MK_THIST, st};
    if (sb.tile_passes > 0) {
        SortArgs pa{};
        pa.keys[0] = w.pkey[0]; pa.keys[1] = w.pkey[1];
        pa.vals[0] = w.pval[0]; pa.vals[1] = w.pval[1];
        pa.n_dev = w.counters + CNT_PAIRS; pa.n_host = -1; pa.n_max = w.pair_cap;
        pa.key_bytes = 4; pa.begin_bit = 0; pa.end_bit = 8 * sb.tile_passes;
        pa.vals_identity = false;
        pa.hist_ready = true;   // counted by the offset scan
        pa.hist = w.hist; pa.tickets = w.counters + TK_SORT0 + 4; pa.status = w.status;
        pa.epoch = w.epoch; pa.epoch_off = eo; pa.err = w.err;
        pa.hook = c->timing ? sort_hook : nullptr; pa.hook_user = &th;
        pa.ranges = w.ranges;   // the last pass records the tile ranges
        launch_sort(pa, c->grid_sort32, st);
        eo += sb.tile_passes;
        psel = sb.tile_passes & 1;
    }
    for (int k = MK_THIST + 1 + sb.tile_passes; k < MK_RANGES; ++k) mark(c, sb_index, k, st);
    if (sb.tile_passes == 0) mark(c, sb_index, MK_THIST, st);
    if (sb.tile_passes == 0)
        launch_ranges(w.pkey[psel], w.counters + CNT_PAIRS, w.ranges, c->grid_ranges, st, w.err);
    mark(c, sb_index, MK_RANGES, st);
    const int cw = cta_w_of(c), ch = cta_h_of(c);
    const int64_t items = (int64_t)sb.n_tiles * (c->tile_w / cw) * (c->tile_h / ch);
    const int cgrid = (int)std::min<int64_t>(
        items, (int64_t)c->num_sms *
                   std::max(1, composite_blocks_per_sm(c->scene.attr_dtype, cw, ch, c->batch)));
    if (c->composite_order) launch_tile_order(w.ranges, sb.n_tiles, w.order, w.err, st);
    launch_composite(c->scene.attr_dtype, c->tile_w, c->tile_h, cw, ch, c->batch, true, cams, nc,
                     sb.n_tiles, w.ranges, w.pval[psel], w.rec, w.counters + TK_COMPOSITE,
                     std::max(cgrid, 1), w.err, w.work64,
                     c->composite_order ? w.order : nullptr,
                     sb_index < kTailSlots ? w.work64 + 2 + 2 * sb_index : nullptr, st);
    mark(c, sb_index, MK_COMPOSITE, st);
    record_event(c->ev_sb[sb_index], st);
    if (sb_index < c->stats_cap / 4)
        k_copy_stats<<<1, 32, 0, st>>>(w.counters, c->stats_dev + 4 * sb_index);
}

int kernels_of(const SubBatch &sb, bool batched, bool order) {
    // epoch bump, live partitions, fused cut + preprocess, partition scan and
    // key gather (which also counts the depth histograms); depth sort (digit
    // scan, 4 passes); pair offsets, duplication; tile sort (digit scan and
    // passes, the last one writing the tile ranges) or, with a single tile,
    // the ranges kernel; compositing; and in the batched path the stats copy
    return 5 + 5 + 2 + (sb.tile_passes > 0 ? 1 + sb.tile_passes : 1) + 1 + (batched ? 1 : 0) +
           (batched && order ? 1 : 0);
}

ngs_status read_u32(const uint32_t *d, uint32_t *h, cudaStream_t st) {
    CK(cudaMemcpyAsync(h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return NGS_OK;
}

ngs_status check_err(ngs_ctx *c) {
    int e = 0;
    CK(cudaMemcpy(&e, c->w.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        CK(cudaMemset(c->w.err, 0, sizeof(int)));
        return (ngs_status)e;
    }
    return NGS_OK;
}

// Raises the planner's pairs-per-pixel estimate to 1.25x the densest
// sub-batch of the last batched render (pairs counted by the device, also when
// they overflowed the buffer), so that the next plan of the same cameras fits.
// Synchronous (reads the per-sub-batch counts).
ngs_status learn_pair_density(ngs_ctx *c) {
    if (c->mode != NGS_MODE_BATCHED || c->last_plan.empty() || !c->work_ready) return NGS_OK;
    const int n = std::min<int>((int)c->last_plan.size(), c->stats_cap / 4);
    std::vector<uint32_t> h((size_t)4 * std::max(n, 1));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(h.data(), c->stats_dev, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost));
    double dens = 0.0;
    for (int i = 0; i < n; ++i) {
        const SubBatch &sb = c->last_plan[i];
        int64_t pix = 0;
        for (int k = sb.c0; k < sb.c1 && k < (int)c->host_cams.size(); ++k)
            pix += (int64_t)c->host_cams[k].width * c->host_cams[k].height;
        if (pix > 0) dens = std::max(dens, (double)h[4 * i + 2] / (double)pix);
    }
    c->pairs_per_pixel = std::min(4096.0, std::max(c->pairs_per_pixel, 1.25 * dens));
    return NGS_OK;
}

// Plain per-view path: one camera at a time, every stage sized from counts
// read back to the host, one CTA per partition, no graph.
ngs_status render_plain(ngs_ctx *c, int n_cams, cudaStream_t st) {
    Work &w = c->w;
    c->last_plan.clear();
    int64_t cut_tot = 0, vis_tot = 0, pair_tot = 0;
    ngs_status es0 = ensure_events(c, n_cams);
    if (es0 != NGS_OK) return es0;
    CK(cudaMemsetAsync(w.work64, 0, kWork64Words * sizeof(unsigned long long), st));
    c->kernels_per_render = 0;
    for (int ci = 0; ci < n_cams; ++ci) {
        SubBatch sb{ci, ci + 1, 0, 0};
        DevCamera &d = c->host_cams[ci];
        d.tile_base = 0;
        sb.n_tiles = (uint32_t)d.tiles_x * d.tiles_y;
        sb.tile_passes = (bits_for(sb.n_tiles) + 7) / 8;
        CK(cudaMemcpyAsync(w.cams + ci, &d, sizeof(DevCamera), cudaMemcpyHostToDevice, st));
        const DevCamera *cams = w.cams + ci;
        ngs_status es = epoch_guard(c, st, kEpochStride);
        if (es != NGS_OK) return es;
        mark(c, ci, MK_START, st);
        CK(cudaMemsetAsync(w.counters, 0, N_COUNTERS * sizeof(uint32_t), st));
        CK(cudaMemsetAsync(w.ranges, 0, (size_t)sb.n_tiles * sizeof(uint2), st));
        k_bump_epoch<<<1, 1, 0, st>>>(w.epoch, kEpochStride);
        uint32_t eo = 0;
        const int64_t nblk = (c->scene.n + cutpre_partition_nodes() - 1) / cutpre_partition_nodes();
        launch_cutpre(c->scene, cams, 1, w.rec, w.rec_cap, w.dkey[1], w.rect,
                      c->node_ids ? w.node_id : nullptr, w.vis_count,
                      w.counters, w.part_list, w.group_list, w.part_info, w.err, c->tile_w, c->tile_h,
                      c->block_cull ? 1 : 0, c->lod_blend ? 1 : 0,
                      (int)std::min<int64_t>(nblk, c->grid_pre), st);
        eo++;
        mark(c, ci, MK_CUT, st);
        uint32_t n_cut = 0, n_vis = 0, n_pairs = 0;
        ngs_status s = read_u32(w.vis_count, &n_vis, st);
        if (s != NGS_OK) return s;
        if ((s = read_u32(w.counters + CNT_CUT, &n_cut, st)) != NGS_OK) return s;
        if ((s = check_err(c)) != NGS_OK) return s;
        launch_gather_keys(w.vis_count, 1, c->scene, w.part_info, w.part_pos, w.part_list,
                           w.dkey[1], w.dkey[0], w.didx[0], w.counters, w.rec_cap, w.hist, w.err,
                           (int)std::max<int64_t>(1, std::min<int64_t>(nblk / 8 + 1,
                                                                       8 * c->num_sms)), st);
        mark(c, ci, MK_PRE, st);
        eo++;
        if ((s = check_err(c)) != NGS_OK) return s;
        const int gsort_v = std::max<int64_t>(1, ((int64_t)n_vis + sort_partition() - 1) /
                                                     sort_partition());
        SortArgs da{};
        da.keys[0] = w.dkey[0]; da.keys[1] = w.dkey[1];
        da.vals[0] = w.didx[0]; da.vals[1] = w.didx[1];
        da.n_dev = nullptr; da.n_host = n_vis; da.n_max = w.rec_cap;
        da.key_bytes = 4; da.begin_bit = 0; da.end_bit = 32; da.vals_identity = false;
        da.hist = w.hist; da.tickets = w.counters + TK_SORT0; da.status = w.status;
        da.epoch = w.epoch; da.epoch_off = eo; da.err = w.err;
        SortHook dh{c, ci, MK_DHIST, st};
        da.hook = c->timing ? sort_hook : nullptr; da.hook_user = &dh;
        da.skip_last_keys = true;   // later stages read the record order only
        da.hist_ready = true;       // counted by the key gather
        launch_sort(da, std::min(gsort_v, c->grid_sort32), st);
        eo += 4;
        const int gscan = std::max<int64_t>(1, ((int64_t)n_vis + scan_partition() - 1) /
                                                   scan_partition());
        CK(cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * 256 * 3, st));
        launch_pair_offsets(w.rect, w.didx[0], w.counters + CNT_VIS, w.poff, w.counters,
                            w.pair_cap, w.counters + TK_SCAN, w.status, w.epoch, eo++, w.err,
                            w.chunk_first, w.rect_sorted, cams, w.hist, sb.tile_passes, gscan,
                            st);
        mark(c, ci, MK_POFF, st);
        if ((s = read_u32(w.counters + CNT_PAIRS, &n_pairs, st)) != NGS_OK) return s;
        if ((s = check_err(c)) != NGS_OK) return s;
        if ((int64_t)n_pairs > w.pair_cap) return NGS_ERR_CAPACITY;
        const int gdup = (int)std::max<int64_t>(
            1, std::min<int64_t>(((int64_t)n_pairs + 2047) / 2048, 8 * (int64_t)c->num_sms));
        launch_duplicate(w.rect_sorted, w.didx[0], w.poff, w.chunk_first, w.counters + CNT_VIS,
                         w.counters + CNT_PAIRS, w.pair_cap, cams, w.pkey[0], w.pval[0], w.err,
                         gdup, st);
        mark(c, ci, MK_DUP, st);
        int psel = 0;
        SortHook th{c, ci, MK_THIST, st};
        if (sb.tile_passes > 0) {
            const int gsort_p = std::max<int64_t>(1, ((int64_t)n_pairs + sort_partition() - 1) /
                                                         sort_partition());
            SortArgs pa{};
            pa.keys[0] = w.pkey[0]; pa.keys[1] = w.pkey[1];
            pa.vals[0] = w.pval[0]; pa.vals[1] = w.pval[1];
            pa.n_dev = nullptr; pa.n_host = n_pairs; pa.n_max = w.pair_cap;
            pa.key_bytes = 4; pa.begin_bit = 0; pa.end_bit = 8 * sb.tile_passes;
            pa.vals_identity = false;
            pa.hist_ready = true;   // counted by the offset scan
            pa.hist = w.hist; pa.tickets = w.counters + TK_SORT0 + 4; pa.status = w.status;
            pa.epoch = w.epoch; pa.epoch_off = eo; pa.err = w.err;
            pa.hook = c->timing ? sort_hook : nullptr; pa.hook_user = &th;
            pa.ranges = w.ranges;   // the last pass records the tile ranges
            launch_sort(pa, std::min(gsort_p, c->grid_sort32), st);
            eo += sb.tile_passes;
            psel = sb.tile_passes & 1;
        }
        const int grng = std::max<int64_t>(1, std::min<int64_t>(((int64_t)n_pairs + 255) / 256,
                                                                 (int64_t)c->num_sms * 16));
        for (int k = MK_THIST + 1 + sb.tile_passes; k < MK_RANGES; ++k) mark(c, ci, k, st);
        if (sb.tile_passes == 0) mark(c, ci, MK_THIST, st);
        if (sb.tile_passes == 0)
            launch_ranges(w.pkey[psel], w.counters + CNT_PAIRS, w.ranges, grng, st, w.err);
        mark(c, ci, MK_RANGES, st);
        const int cw = cta_w_of(c), ch = cta_h_of(c);
        const uint32_t items = sb.n_tiles * (uint32_t)((c->tile_w / cw) * (c->tile_h / ch));
        launch_composite(c->scene.attr_dtype, c->tile_w, c->tile_h, cw, ch, c->batch, false,
                         cams, 1, sb.n_tiles, w.ranges, w.pval[psel], w.rec,
                         w.counters + TK_COMPOSITE, (int)std::max<uint32_t>(items, 1), w.err,
                         w.work64, nullptr, nullptr, st);
        mark(c, ci, MK_COMPOSITE, st);
        CK(cudaGetLastError());
        c->kernels_per_render += kernels_of(sb, false, false);
        cut_tot += n_cut; vis_tot += n_vis; pair_tot += n_pairs;
        c->last_plan.push_back(sb);
        c->last_plan.back().c0 = ci;
    }
    c->stats.cut_total = cut_tot;
    c->stats_pending = false;
    c->stats.visible_total = vis_tot;
    c->stats.pair_total = pair_tot;
    c->stats.sub_batches = n_cams;
    c->stats.graph_replayed = 0;
    c->stats.candidate_total = -1;
    return NGS_OK;
}

ngs_status render_batched(ngs_ctx *c, int n_cams, cudaStream_t st) {
    Work &w = c->w;
    std::vector<SubBatch> sbs = plan(c, c->host_cams, kMaxCamsPerBatch);
    // graph key: layout of the cameras and every setting the launches bake in
    std::vector<int64_t> key;
    key.reserve(8 + 3 * n_cams);
    key.push_back(n_cams); key.push_back(c->tile_w); key.push_back(c->tile_h);
    key.push_back(c->batch); key.push_back((int64_t)c->scene_version);
    key.push_back(cta_w_of(c)); key.push_back(cta_h_of(c));
    key.push_back(c->lod_blend ? 1 : 0);
    key.push_back(c->composite_order ? 1 : 0);
    for (int i = 0; i < n_cams; ++i) {
        key.push_back(c->host_cams[i].width);
        key.push_back(c->host_cams[i].height);
        key.push_back(c->host_cams[i].tile_base);
    }
    ngs_status es = epoch_guard(c, st, kEpochStride * sbs.size());
    if (es != NGS_OK) return es;
    if ((es = ensure_events(c, (int)sbs.size())) != NGS_OK) return es;
    if ((es = ensure_sb_events(c, (int)sbs.size())) != NGS_OK) return es;
    key.push_back(c->timing ? 1 : 0);
    c->kernels_per_render = 0;
    for (const SubBatch &sb : sbs) c->kernels_per_render += kernels_of(sb, true, c->composite_order);
    CK(cudaMemcpyAsync(w.cams, c->host_cams.data(), sizeof(DevCamera) * n_cams,
                       cudaMemcpyHostToDevice, st));
    if (c->use_graph) {
        if (!(c->gexec && key == c->gkey)) {
            drop_graph(c);
            if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            cudaMemsetAsync(w.work64, 0, kWork64Words * sizeof(unsigned long long), c->cap_stream);
            for (size_t i = 0; i < sbs.size(); ++i) enqueue_batched(c, sbs[i], (int)i, c->cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
            if (e != cudaSuccess) {
                std::fprintf(stderr, "ngs: graph capture failed: %s\n", cudaGetErrorString(e));
                return NGS_ERR_CUDA;
            }
            e = cudaGraphInstantiate(&c->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                c->gexec = nullptr;
                return NGS_ERR_CUDA;
            }
            c->gkey = key;
            c->stats.graph_replayed = 0;
        } else {
            c->stats.graph_replayed = 1;
        }
        CK(cudaGraphLaunch(c->gexec, st));
    } else {
        CK(cudaMemsetAsync(w.work64, 0, kWork64Words * sizeof(unsigned long long), st));
        for (size_t i = 0; i < sbs.size(); ++i) enqueue_batched(c, sbs[i], (int)i, st);
        c->stats.graph_replayed = 0;
    }
    CK(cudaGetLastError());
    c->last_plan = sbs;
    c->stats.sub_batches = (int32_t)sbs.size();
    c->stats.cut_total = c->stats.visible_total = c->stats.pair_total = -1;  // filled on demand
    c->stats.candidate_total = -1;
    c->stats_pending = true;
    return NGS_OK;
}

ngs_status render_common(ngs_ctx *c, const ngs_camera *cams, int32_t n_cams,
                         float *const *images, cudaStream_t st) {
    if (!c) return NGS_ERR_INVALID_ARG;
    if (!c->loaded) return NGS_ERR_NOT_LOADED;
    if (!cams || !images || n_cams <= 0 || n_cams > kMaxCamsPerCall) return NGS_ERR_INVALID_ARG;
    if (!tile_supported(c->tile_w, c->tile_h) || !split_supported(c)) return NGS_ERR_INVALID_ARG;
    for (int i = 0; i < n_cams; ++i)
        if (!camera_ok(cams[i]) || !images[i]) return NGS_ERR_INVALID_ARG;
    ngs_status s = ensure_work(c);
    if (s != NGS_OK) return s;
    if (c->node_ids && !c->w.node_id) {
        s = dalloc(&c->w.node_id, (size_t)c->w.rec_cap);
        if (s != NGS_OK) return s;
    }
    if (c->latched != NGS_OK) {
        s = c->latched;
        c->latched = NGS_OK;
        return s;
    }
    c->host_cams.resize(n_cams);
    for (int i = 0; i < n_cams; ++i) {
        fill_cam(c->host_cams[i], cams[i], c->tile_w, c->tile_h, images[i]);
        if ((int64_t)c->host_cams[i].tiles_x * c->host_cams[i].tiles_y > (1 << 24))
            return NGS_ERR_INVALID_ARG;
    }
    c->stats.tile_w = c->tile_w; c->stats.tile_h = c->tile_h;
    c->stats.batch = c->batch; c->stats.mode = c->mode;
    c->last_node_ids = c->node_ids;
    c->stats.cta_w = cta_w_of(c); c->stats.cta_h = cta_h_of(c);
    return c->mode == NGS_MODE_PLAIN ? render_plain(c, n_cams, st) : render_batched(c, n_cams, st);
}

bool valid_box(const float *lo, const float *hi) {
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(lo[k]) || !std::isfinite(hi[k]) || lo[k] > hi[k]) return false;
    return true;
}

ngs_status validate(const ngs_gaussians *g, const ngs_hierarchy *h) {
    const int64_t n = g->n;
    if (n < 1 || n >= (int64_t)1 << 31) return NGS_ERR_INVALID_ARG;
    if (!g->pos || !g->quat || !g->log_scale || !g->opacity || !g->sh) return NGS_ERR_INVALID_ARG;
    if (g->attr_dtype != NGS_F32 && g->attr_dtype != NGS_F16 && g->attr_dtype != NGS_BF16)
        return NGS_ERR_INVALID_ARG;
    if (!h->parent || !h->child_begin || !h->child_count || !h->aabb_min || !h->aabb_max)
        return NGS_ERR_INVALID_ARG;
    if (h->parent[0] != -1) return NGS_ERR_INVALID_HIERARCHY;
    int64_t kids = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!valid_box(h->aabb_min + 3 * i, h->aabb_max + 3 * i)) return NGS_ERR_INVALID_HIERARCHY;
        const int32_t p = h->parent[i];
        if (i > 0 && (p < 0 || p >= i)) return NGS_ERR_INVALID_HIERARCHY;
        const int32_t cc = h->child_count[i], cb = h->child_begin[i];
        if (cc < 0) return NGS_ERR_INVALID_HIERARCHY;
        if (cc > 0) {
            if (cb <= i || (int64_t)cb + cc > n) return NGS_ERR_INVALID_HIERARCHY;
            for (int32_t k = cb; k < cb + cc; ++k) {
                if (h->parent[k] != i) return NGS_ERR_INVALID_HIERARCHY;
                for (int a = 0; a < 3; ++a)
                    if (h->aabb_min[3 * k + a] < h->aabb_min[3 * i + a] ||
                        h->aabb_max[3 * k + a] > h->aabb_max[3 * i + a])
                        return NGS_ERR_INVALID_HIERARCHY;
            }
        }
        kids += cc;
    }
    if (kids != n - 1) return NGS_ERR_INVALID_HIERARCHY;
    return NGS_OK;
}

}  // namespace

// A context that renders the parent's resident scene (no copy) with its own
// work buffers, streams and graph cache: one lane of the serving loop.
ngs_status ngs::lane_create(ngs_ctx *parent, int64_t record_capacity, int64_t pair_capacity,
                            ngs_ctx **out) {
    if (!parent || !out || !parent->loaded) return NGS_ERR_NOT_LOADED;
    ngs_config cfg = parent->cfg;
    if (record_capacity > 0) cfg.record_capacity = record_capacity;
    if (pair_capacity > 0) cfg.pair_capacity = pair_capacity;
    ngs_status s = ngs_create(&cfg, out);
    if (s != NGS_OK) return s;
    ngs_ctx *l = *out;
    l->scene = parent->scene;
    l->owns_scene = false;
    l->loaded = true;
    l->scene_version = parent->scene_version;
    l->tile_w = parent->tile_w; l->tile_h = parent->tile_h; l->batch = parent->batch;
    l->cta_w = parent->cta_w; l->cta_h = parent->cta_h;
    l->use_graph = false;   // every launch has a different camera mix
    l->block_cull = parent->block_cull;
    l->lod_blend = parent->lod_blend;
    l->composite_order = parent->composite_order;
    l->pairs_per_pixel = parent->pairs_per_pixel;
    return NGS_OK;
}

double ngs::ctx_pairs_per_pixel(const ngs_ctx *c) { return c->pairs_per_pixel; }

extern "C" {

NGS_API const char *ngs_strerror(ngs_status s) {
    switch (s) {
    case NGS_OK: return "ok";
    case NGS_ERR_INVALID_ARG: return "invalid argument";
    case NGS_ERR_INVALID_HIERARCHY: return "invalid hierarchy";
    case NGS_ERR_OUT_OF_MEMORY: return "out of device memory";
    case NGS_ERR_CAPACITY: return "work buffer capacity exceeded";
    case NGS_ERR_CUDA: return "CUDA error";
    case NGS_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case NGS_ERR_NOT_LOADED: return "no scene loaded";
    }
    return "unknown status";
}

NGS_API ngs_status ngs_create(const ngs_config *cfg, ngs_ctx **out) {
    if (!out) return NGS_ERR_INVALID_ARG;
    *out = nullptr;
    ngs_config c{};
    if (cfg) c = *cfg;
    if (c.tile_w == 0) c.tile_w = 16;
    if (c.tile_h == 0) c.tile_h = 16;
    if (c.batch == 0) c.batch = 128;
    if (c.cut_capacity <= 0) c.cut_capacity = (int64_t)1 << 27;
    if (c.record_capacity <= 0) c.record_capacity = (int64_t)1 << 26;
    if (c.pair_capacity <= 0) c.pair_capacity = (int64_t)1 << 29;
    if (c.max_tiles_per_batch <= 0) c.max_tiles_per_batch = 1 << 16;
    const bool tile_ok = tile_supported(c.tile_w, c.tile_h);
    if (!tile_ok || (c.batch != 64 && c.batch != 128 && c.batch != 256)) return NGS_ERR_INVALID_ARG;
    if (c.cut_capacity >= ((int64_t)1 << 31) || c.record_capacity >= ((int64_t)1 << 31) ||
        c.pair_capacity >= ((int64_t)1 << 31) || c.max_tiles_per_batch > (1 << 24))
        return NGS_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev) {
        cudaGetLastError();
        return NGS_ERR_CUDA;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return NGS_ERR_CUDA;
    ngs_ctx *x = new (std::nothrow) ngs_ctx();
    if (!x) return NGS_ERR_OUT_OF_MEMORY;
    x->device = c.device;
    x->cfg = c;
    x->tile_w = c.tile_w; x->tile_h = c.tile_h; x->batch = c.batch;
    cudaDeviceGetAttribute(&x->num_sms, cudaDevAttrMultiProcessorCount, c.device);
    sort_init_attributes();
    cutpre_init_attributes();
    composite_init_attributes();
    x->grid_cut = 4 * x->num_sms;
    x->grid_pre = 4 * x->num_sms;
    x->grid_sort32 = 2 * x->num_sms;
    x->grid_sort64 = 2 * x->num_sms;
    x->grid_scan = 5 * x->num_sms;
    x->grid_dup = 8 * x->num_sms;
    x->grid_ranges = 16 * x->num_sms;
    *out = x;
    return NGS_OK;
}

NGS_API ngs_status ngs_destroy(ngs_ctx *c) {
    if (!c) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->nav_tmp) dfree(c->nav_tmp);
    drop_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->ev_copied) cudaEventDestroy(c->ev_copied);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_sb) cudaEventDestroy(e);
    free_work(c);
    free_scene(c);
    dfree(c->sort_tmp_keys);
    dfree(c->sort_tmp_vals);
    delete c;
    return NGS_OK;
}

NGS_API ngs_status ngs_set_option(ngs_ctx *c, int32_t opt, int64_t v) {
    if (!c) return NGS_ERR_INVALID_ARG;
    switch (opt) {
    case NGS_OPT_MODE:
        if (v != NGS_MODE_BATCHED && v != NGS_MODE_PLAIN) return NGS_ERR_INVALID_ARG;
        c->mode = (int)v;
        return NGS_OK;
    case NGS_OPT_TILE_W:
    case NGS_OPT_TILE_H: {
        int tw = opt == NGS_OPT_TILE_W ? (int)v : c->tile_w;
        int th = opt == NGS_OPT_TILE_H ? (int)v : c->tile_h;
        // either dimension may be set first: an unsupported pair is held until
        // the other dimension completes it, and a render rejects it
        if (!(tw == 8 || tw == 16 || tw == 32) || !(th == 8 || th == 16 || th == 32))
            return NGS_ERR_INVALID_ARG;
        c->tile_w = tw; c->tile_h = th;
        drop_graph(c);
        return NGS_OK;
    }
    case NGS_OPT_CTA_W:
    case NGS_OPT_CTA_H: {
        // 0 restores "the whole tile"; other shapes are checked at render
        // against the tile shape in force then
        if (!(v == 0 || v == 8 || v == 16 || v == 32)) return NGS_ERR_INVALID_ARG;
        (opt == NGS_OPT_CTA_W ? c->cta_w : c->cta_h) = (int)v;
        drop_graph(c);
        return NGS_OK;
    }
    case NGS_OPT_PAIRS_PER_PIXEL:
        if (v < 1 || v > 4096) return NGS_ERR_INVALID_ARG;
        c->pairs_per_pixel = (double)v;
        return NGS_OK;
    case NGS_OPT_BATCH:
        if (v != 64 && v != 128 && v != 256) return NGS_ERR_INVALID_ARG;
        c->batch = (int)v;
        drop_graph(c);
        return NGS_OK;
    case NGS_OPT_GRAPH:
        c->use_graph = v != 0;
        if (!c->use_graph) drop_graph(c);
        return NGS_OK;
    case NGS_OPT_STAGE_TIMING:
        c->timing = v != 0;
        drop_graph(c);
        return NGS_OK;
    case NGS_OPT_BLOCK_CULL:
        c->block_cull = v != 0;
        drop_graph(c);
        return NGS_OK;
    case NGS_OPT_LOD_BLEND:
        c->lod_blend = v != 0;
        drop_graph(c);
        return NGS_OK;
    case NGS_OPT_COMPOSITE_ORDER:
        c->composite_order = v != 0;
        drop_graph(c);
        return NGS_OK;
    case NGS_OPT_NODE_IDS:
        c->node_ids = v != 0;
        drop_graph(c);
        return NGS_OK;
    }
    return NGS_ERR_INVALID_ARG;
}

NGS_API ngs_status ngs_load_scene(ngs_ctx *c, const ngs_gaussians *g, const ngs_hierarchy *h) {
    if (!c || !g || !h) return NGS_ERR_INVALID_ARG;
    ngs_status s = validate(g, h);
    if (s != NGS_OK) return s;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    drop_graph(c);
    free_scene(c);
    free_work(c);   // status words and cut bounds depend on the node count
    const int64_t n = g->n;
    std::vector<float4> lo(n), hi(n), p4(n), q(n);
    const size_t esz = g->attr_dtype == NGS_F32 ? 4 : 2;
    std::vector<unsigned char> sop((size_t)n * 4 * esz);
    for (int64_t i = 0; i < n; ++i) {
        int32_t par = h->parent[i], cc = h->child_count[i];
        float pf, cf;
        std::memcpy(&pf, &par, 4);
        std::memcpy(&cf, &cc, 4);
        lo[i] = make_float4(h->aabb_min[3 * i], h->aabb_min[3 * i + 1], h->aabb_min[3 * i + 2], pf);
        hi[i] = make_float4(h->aabb_max[3 * i], h->aabb_max[3 * i + 1], h->aabb_max[3 * i + 2], cf);
        double o;
        if (g->attr_dtype == NGS_F32) {
            o = ((const float *)g->opacity)[i];
            float *d = (float *)sop.data() + 4 * i;
            const float *ls = (const float *)g->log_scale + 3 * i;
            d[0] = ls[0]; d[1] = ls[1]; d[2] = ls[2]; d[3] = (float)o;
        } else {
            const uint16_t ov = ((const uint16_t *)g->opacity)[i];
            o = g->attr_dtype == NGS_F16 ? half_to_float(ov) : bf16_to_float(ov);
            uint16_t *d = (uint16_t *)sop.data() + 4 * i;
            const uint16_t *ls = (const uint16_t *)g->log_scale + 3 * i;
            d[0] = ls[0]; d[1] = ls[1]; d[2] = ls[2]; d[3] = ov;
        }
        // alpha <= o everywhere, so a node with 255 o < 1 never reaches 1/255;
        // 255 o is exact in float64
        const uint32_t flags = (255.0 * o < 1.0) ? kNodeCullOpacity : 0u;
        float ff;
        std::memcpy(&ff, &flags, 4);
        p4[i] = make_float4(g->pos[3 * i], g->pos[3 * i + 1], g->pos[3 * i + 2], ff);
        q[i] = make_float4(g->quat[4 * i], g->quat[4 * i + 1], g->quat[4 * i + 2], g->quat[4 * i + 3]);
    }
    // per-block bounds for the block-level cull of the fused cut + preprocess
    const int64_t bs = cutpre_partition_nodes();
    const int64_t nb = (n + bs - 1) / bs;
    std::vector<float4> blo(nb), bhi(nb), blo_b(nb), bhi_b(nb);
    auto log_scale_of = [&](int64_t i, int k) -> double {
        if (g->attr_dtype == NGS_F32) return ((const float *)g->log_scale)[3 * i + k];
        const uint16_t hv = ((const uint16_t *)g->log_scale)[3 * i + k];
        return g->attr_dtype == NGS_F16 ? half_to_float(hv) : bf16_to_float(hv);
    };
    auto opacity_of = [&](int64_t i) -> double {
        if (g->attr_dtype == NGS_F32) return ((const float *)g->opacity)[i];
        const uint16_t hv = ((const uint16_t *)g->opacity)[i];
        return g->attr_dtype == NGS_F16 ? half_to_float(hv) : bf16_to_float(hv);
    };
    for (int64_t b = 0; b < nb; ++b) {
        // own: the block's nodes; both: the block's nodes and their parents
        float mn[2][3], mx[2][3];
        double smax[2] = {0.0, 0.0}, kmax[2] = {0.0, 0.0};
        for (int w = 0; w < 2; ++w)
            for (int k = 0; k < 3; ++k) { mn[w][k] = INFINITY; mx[w][k] = -INFINITY; }
        for (int64_t i = b * bs; i < std::min(n, (b + 1) * bs); ++i) {
            const int64_t par = h->parent[i];
            for (int src = 0; src < 2; ++src) {
                const int64_t j = src == 0 ? i : par;
                if (j < 0) continue;
                for (int w = src; w < 2; ++w) {
                    for (int k = 0; k < 3; ++k) {
                        mn[w][k] = std::min(mn[w][k], g->pos[3 * j + k]);
                        mx[w][k] = std::max(mx[w][k], g->pos[3 * j + k]);
                    }
                    const double ls = std::max(log_scale_of(j, 0),
                                               std::max(log_scale_of(j, 1), log_scale_of(j, 2)));
                    smax[w] = std::max(smax[w], std::exp(ls));
                    const double o = opacity_of(j);
                    if (255.0 * o >= 1.0) kmax[w] = std::max(kmax[w], 2.0 * std::log(255.0 * o));
                }
            }
        }
        blo[b] = make_float4(mn[0][0], mn[0][1], mn[0][2], (float)(smax[0] * (1.0 + 1e-5)));
        bhi[b] = make_float4(mx[0][0], mx[0][1], mx[0][2], (float)(kmax[0] * (1.0 + 1e-5) + 1e-6));
        blo_b[b] = make_float4(mn[1][0], mn[1][1], mn[1][2], (float)(smax[1] * (1.0 + 1e-5)));
        bhi_b[b] = make_float4(mx[1][0], mx[1][1], mx[1][2], (float)(kmax[1] * (1.0 + 1e-5) + 1e-6));
    }
    SceneDev &d = c->scene;
    ngs_status st = NGS_OK;
    auto A = [&](ngs_status x) { if (st == NGS_OK) st = x; };
    A(dalloc(&d.box_lo, n)); A(dalloc(&d.box_hi, n)); A(dalloc(&d.pos4, n)); A(dalloc(&d.quat, n));
    A(dalloc(&d.blk_lo, nb)); A(dalloc(&d.blk_hi, nb));
    A(dalloc(&d.blk_lo_b, nb)); A(dalloc(&d.blk_hi_b, nb));
    A(dalloc((unsigned char **)&d.sop, (size_t)n * 4 * esz));
    A(dalloc((unsigned char **)&d.sh, (size_t)n * 48 * esz));
    if (st != NGS_OK) {
        free_scene(c);
        return st;
    }
    CK(cudaMemcpy(d.box_lo, lo.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.box_hi, hi.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.pos4, p4.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.quat, q.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.sop, sop.data(), sop.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.sh, g->sh, (size_t)n * 48 * esz, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.blk_lo, blo.data(), nb * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.blk_hi, bhi.data(), nb * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.blk_lo_b, blo_b.data(), nb * sizeof(float4), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d.blk_hi_b, bhi_b.data(), nb * sizeof(float4), cudaMemcpyHostToDevice));
    d.nblk = nb;
    d.n = n;
    d.n_leaves = 0;
    for (int64_t i = 0; i < n; ++i) d.n_leaves += h->child_count[i] == 0 ? 1 : 0;
    d.attr_dtype = g->attr_dtype;
    c->loaded = true;
    ++c->scene_version;
    return NGS_OK;
}

NGS_API ngs_status ngs_select_cut(ngs_ctx *c, const ngs_camera *cams, int32_t n_cams,
                                  int32_t *d_ids, int64_t *d_offsets, int64_t cap, void *stream) {
    if (!c) return NGS_ERR_INVALID_ARG;
    if (!c->loaded) return NGS_ERR_NOT_LOADED;
    if (!cams || !d_ids || !d_offsets || n_cams <= 0 || n_cams > kMaxCamsPerBatch || cap < 0)
        return NGS_ERR_INVALID_ARG;
    for (int i = 0; i < n_cams; ++i)
        if (!camera_ok(cams[i])) return NGS_ERR_INVALID_ARG;
    // a cut is an antichain of the tree (at most one id per leaf): below this
    // bound the 32-bit offsets cannot wrap
    if ((int64_t)n_cams * std::max<int64_t>(c->scene.n_leaves, 1) >= ((int64_t)1 << 32))
        return NGS_ERR_CAPACITY;
    cudaSetDevice(c->device);
    ngs_status s = ensure_work(c);
    if (s != NGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<DevCamera> hc(n_cams);
    for (int i = 0; i < n_cams; ++i) fill_cam(hc[i], cams[i], c->tile_w, c->tile_h, nullptr);
    Work &w = c->w;
    if ((s = epoch_guard(c, st, kEpochStride)) != NGS_OK) return s;
    CK(cudaMemcpyAsync(w.cams, hc.data(), sizeof(DevCamera) * n_cams, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w.counters, 0, N_COUNTERS * sizeof(uint32_t), st));
    k_bump_epoch<<<1, 1, 0, st>>>(w.epoch, kEpochStride);
    const int64_t cap32 = std::min<int64_t>(cap, (1ll << 32) - 1);
    if (n_cams >= kCutBlockedMinCams) {
        // count per (camera, block), scan in camera-major order, write
        const SceneDev &sc = c->scene;
        const int64_t nblk = (sc.n + cut_partition_nodes() - 1) / cut_partition_nodes();
        const int64_t np = nblk * n_cams;
        launch_cut_blocked(false, sc.box_lo, sc.box_hi, sc.n, w.cams, nullptr, n_cams,
                           c->cut_counts, nullptr, cap32, w.counters + TK_CUT, w.err, c->grid_cut,
                           st);
        const int64_t sparts = (np + scan_partition() - 1) / scan_partition();
        launch_scan_u32(c->cut_counts, c->cut_poff, nullptr, np, c->cut_off32,
                        w.counters + TK_SCAN, w.status, w.epoch, 0, w.err,
                        (int)std::min<int64_t>(sparts, c->grid_scan), st);
        launch_cut_cam_offsets(c->cut_poff, c->cut_off32, nblk, n_cams, cap32, d_offsets,
                               w.counters, w.err, st);
        launch_cut_blocked(true, sc.box_lo, sc.box_hi, sc.n, w.cams, nullptr, n_cams,
                           c->cut_poff, (uint32_t *)d_ids, cap32, w.counters + TK_PRE, w.err,
                           c->grid_cut, st);
    } else {
        launch_cut(c->scene, w.cams, n_cams, (uint32_t *)d_ids, cap32, c->cut_off32, w.counters,
                   w.counters + TK_CUT, w.status, w.epoch, 0, w.err, c->grid_cut, st);
        k_offsets_to_i64<<<(n_cams + 256) / 256, 256, 0, st>>>(c->cut_off32, d_offsets, n_cams);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return check_err(c);
}

NGS_API ngs_status ngs_select_cut_shared(ngs_ctx *c, const ngs_camera *cams, int32_t n_cams,
                                         const int32_t *group_begin, int32_t n_groups,
                                         uint32_t flags, float guard_px, int32_t *d_ids,
                                         int64_t *d_offsets, int64_t cap, void *stream) {
    if (!c) return NGS_ERR_INVALID_ARG;
    if (!c->loaded) return NGS_ERR_NOT_LOADED;
    if (!cams || !group_begin || !d_ids || !d_offsets || n_cams <= 0 ||
        n_cams > kMaxCamsPerBatch || n_groups <= 0 || n_groups > n_cams || cap < 0)
        return NGS_ERR_INVALID_ARG;
    if ((flags & ~(uint32_t)NGS_CUT_FRUSTUM) != 0 || !std::isfinite(guard_px) || guard_px < 0.0f)
        return NGS_ERR_INVALID_ARG;
    if (group_begin[0] != 0 || group_begin[n_groups] != n_cams) return NGS_ERR_INVALID_ARG;
    for (int32_t g = 0; g < n_groups; ++g)
        if (group_begin[g + 1] <= group_begin[g]) return NGS_ERR_INVALID_ARG;
    for (int i = 0; i < n_cams; ++i)
        if (!camera_ok(cams[i])) return NGS_ERR_INVALID_ARG;
    if ((int64_t)n_groups * std::max<int64_t>(c->scene.n_leaves, 1) >= ((int64_t)1 << 32))
        return NGS_ERR_CAPACITY;
    cudaSetDevice(c->device);
    ngs_status s = ensure_work(c);
    if (s != NGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<CutCam> hc(n_cams);
    for (int i = 0; i < n_cams; ++i) fill_cut_cam(hc[i], cams[i], guard_px);
    Work &w = c->w;
    if ((s = epoch_guard(c, st, kEpochStride)) != NGS_OK) return s;
    CK(cudaMemcpyAsync(c->cut_cams, hc.data(), sizeof(CutCam) * n_cams, cudaMemcpyHostToDevice,
                       st));
    CK(cudaMemcpyAsync(c->cut_groups, group_begin, sizeof(int32_t) * (n_groups + 1),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(w.counters, 0, N_COUNTERS * sizeof(uint32_t), st));
    k_bump_epoch<<<1, 1, 0, st>>>(w.epoch, kEpochStride);
    const int64_t cap32 = std::min<int64_t>(cap, (1ll << 32) - 1);
    if (n_groups == n_cams && n_cams >= kCutBlockedMinCams && (flags & NGS_CUT_FRUSTUM)) {
        // one frustum-culled cut per camera: the camera-blocked two-pass form
        const SceneDev &sc = c->scene;
        const int64_t nblk = (sc.n + cut_partition_nodes() - 1) / cut_partition_nodes();
        const int64_t np = nblk * n_cams;
        launch_cut_blocked(false, sc.box_lo, sc.box_hi, sc.n, nullptr, c->cut_cams, n_cams,
                           c->cut_counts, nullptr, cap32, w.counters + TK_CUT, w.err, c->grid_cut,
                           st);
        const int64_t sparts = (np + scan_partition() - 1) / scan_partition();
        launch_scan_u32(c->cut_counts, c->cut_poff, nullptr, np, c->cut_off32,
                        w.counters + TK_SCAN, w.status, w.epoch, 0, w.err,
                        (int)std::min<int64_t>(sparts, c->grid_scan), st);
        launch_cut_cam_offsets(c->cut_poff, c->cut_off32, nblk, n_cams, cap32, d_offsets,
                               w.counters, w.err, st);
        launch_cut_blocked(true, sc.box_lo, sc.box_hi, sc.n, nullptr, c->cut_cams, n_cams,
                           c->cut_poff, (uint32_t *)d_ids, cap32, w.counters + TK_PRE, w.err,
                           c->grid_cut, st);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        return check_err(c);
    }
    launch_cut_shared((flags & NGS_CUT_FRUSTUM) != 0, c->scene.box_lo, c->scene.box_hi,
                      c->scene.n, c->cut_cams, c->cut_groups, n_groups, (uint32_t *)d_ids,
                      cap32, c->cut_off32, w.counters,
                      w.counters + TK_CUT, w.status, w.epoch, 0, w.err, c->grid_cut, st);
    k_offsets_to_i64<<<(n_groups + 256) / 256, 256, 0, st>>>(c->cut_off32, d_offsets, n_groups);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return check_err(c);
}

NGS_API ngs_status ngs_render(ngs_ctx *c, const ngs_camera *cams, int32_t n_cams,
                              float *const *d_images, void *stream) {
    if (c) cudaSetDevice(c->device);
    return render_common(c, cams, n_cams, d_images, (cudaStream_t)stream);
}

NGS_API ngs_status ngs_selftest_wait_timeout(ngs_ctx *c, void *stream) {
    if (!c) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (!c->loaded && !c->work_ready) c->scene.n = 1;
    ngs_status s = ensure_work(c);
    if (s != NGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // a fresh epoch value: no status word carries it
    if ((s = epoch_guard(c, st, kEpochStride)) != NGS_OK) return s;
    k_bump_epoch<<<1, 1, 0, st>>>(c->w.epoch, kEpochStride);
    k_wait_probe<<<1, 1, 0, st>>>(c->w.status, c->w.epoch, c->w.err);
    CK(cudaGetLastError());
    return ngs_synchronize(c, stream);
}

NGS_API ngs_status ngs_synchronize(ngs_ctx *c, void *stream) {
    if (!c) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (c->latched != NGS_OK) {
        ngs_status s = c->latched;
        c->latched = NGS_OK;
        return s;
    }
    if (!c->work_ready) return NGS_OK;
    const ngs_status s = check_err(c);
    // a batched render that overflowed the pair buffer: the next plan of the
    // same cameras uses the densities the device counted
    if (s == NGS_ERR_CAPACITY) learn_pair_density(c);
    return s;
}

NGS_API ngs_status ngs_render_host(ngs_ctx *c, const ngs_camera *cams, int32_t n_cams,
                                   float *const *h_images, void *stream) {
    if (!c) return NGS_ERR_INVALID_ARG;
    if (!cams || !h_images || n_cams <= 0) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    size_t total = 0;
    for (int i = 0; i < n_cams; ++i) {
        if (!camera_ok(cams[i]) || !h_images[i]) return NGS_ERR_INVALID_ARG;
        total += (size_t)3 * cams[i].width * cams[i].height;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // Page-locked host memory that the device can address (cudaHostAlloc'd or
    // registered, mapped): the compositing kernels write the pixels straight
    // into it, so the images cross to the host while the render runs
    {
        std::vector<float *> hdev(n_cams);
        bool mapped = true;
        for (int i = 0; i < n_cams && mapped; ++i) {
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, h_images[i]) != cudaSuccess ||
                a.type != cudaMemoryTypeHost || !a.devicePointer) {
                cudaGetLastError();   // an unregistered pointer is not an error here
                mapped = false;
            } else {
                hdev[i] = static_cast<float *>(a.devicePointer);
            }
        }
        if (mapped) {
            ngs_status s = NGS_OK;
            for (int attempt = 0; attempt < kCapacityRetries; ++attempt) {
                if ((s = render_common(c, cams, n_cams, hdev.data(), st)) != NGS_OK) return s;
                s = ngs_synchronize(c, stream);
                if (s != NGS_ERR_CAPACITY || c->mode != NGS_MODE_BATCHED) break;
            }
            return s;
        }
    }
    // otherwise device images carved from one buffer owned by the call
    static thread_local float *dbuf = nullptr;
    static thread_local size_t dcap = 0;
    if (total > dcap) {
        dfree(dbuf);
        dbuf = nullptr;
        dcap = 0;
        if (dalloc(&dbuf, total) != NGS_OK) return NGS_ERR_OUT_OF_MEMORY;
        dcap = total;
    }
    std::vector<float *> dimg(n_cams);
    size_t off = 0;
    for (int i = 0; i < n_cams; ++i) {
        dimg[i] = dbuf + off;
        off += (size_t)3 * cams[i].width * cams[i].height;
    }
    // cameras [i0, i1) to the host, consecutive images whose host buffers
    // also follow each other in one copy
    auto copy_out = [&](int i0, int i1, cudaStream_t cs) -> ngs_status {
        for (int i = i0; i < i1;) {
            size_t bytes = sizeof(float) * 3 * cams[i].width * cams[i].height;
            int j = i + 1;
            while (j < i1 && h_images[j] == h_images[j - 1] + 3 * (size_t)cams[j - 1].width *
                                                                 cams[j - 1].height) {
                bytes += sizeof(float) * 3 * cams[j].width * cams[j].height;
                ++j;
            }
            CK(cudaMemcpyAsync(h_images[i], dimg[i], bytes, cudaMemcpyDeviceToHost, cs));
            i = j;
        }
        return NGS_OK;
    };
    // a batched render whose pairs overflow the buffer is planned again from
    // the densities the device counted (smaller sub-batches) and redone;
    // each sub-batch's images are copied out as soon as they are complete
    ngs_status s = NGS_OK;
    for (int attempt = 0; attempt < kCapacityRetries; ++attempt) {
        s = render_common(c, cams, n_cams, dimg.data(), st);
        if (s != NGS_OK) return s;
        if (c->mode != NGS_MODE_BATCHED) {
            if ((s = copy_out(0, n_cams, st)) != NGS_OK) return s;
            return ngs_synchronize(c, stream);
        }
        if (!c->copy_stream) CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->ev_copied) CK(cudaEventCreateWithFlags(&c->ev_copied, cudaEventDisableTiming));
        for (size_t k = 0; k < c->last_plan.size(); ++k) {
            CK(cudaStreamWaitEvent(c->copy_stream, c->ev_sb[k], 0));
            if ((s = copy_out(c->last_plan[k].c0, c->last_plan[k].c1, c->copy_stream)) != NGS_OK)
                return s;
        }
        CK(cudaEventRecord(c->ev_copied, c->copy_stream));
        CK(cudaStreamWaitEvent(st, c->ev_copied, 0));
        s = ngs_synchronize(c, stream);
        if (s != NGS_ERR_CAPACITY) break;
    }
    return s;
}

NGS_API ngs_status ngs_last_stats(ngs_ctx *c, ngs_stats *out) {
    if (!c || !out) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    if (c->work_ready) {
        unsigned long long w64[kWork64Words] = {};
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(w64, c->w.work64, sizeof(w64), cudaMemcpyDeviceToHost));
        c->stats.records_staged = (int64_t)w64[0];
        c->stats.evaluations = (int64_t)w64[1];
        // per sub-batch: ~(first CTA to find the queue empty), last CTA's end
        double tail = 0.0;
        if (c->mode == NGS_MODE_BATCHED)
            for (int k = 0; k < kTailSlots && k < (int)c->last_plan.size(); ++k) {
                const unsigned long long t0 = ~w64[2 + 2 * k], t1 = w64[3 + 2 * k];
                if (w64[2 + 2 * k] && t1 >= t0) tail += (double)(t1 - t0) * 1e-6;
            }
        c->stats.composite_tail_ms = tail;
    }
    c->stats.kernels = c->kernels_per_render;
    if (c->stats_pending && c->work_ready) {
        c->stats_pending = false;
        CK(cudaDeviceSynchronize());
        const int n = std::min<int>((int)c->last_plan.size(), c->stats_cap / 4);
        std::vector<uint32_t> h((size_t)4 * std::max(n, 1));
        CK(cudaMemcpy(h.data(), c->stats_dev, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost));
        int64_t a = 0, b = 0, p = 0, q = 0;
        for (int i = 0; i < n; ++i) {
            a += h[4 * i]; b += h[4 * i + 1]; p += h[4 * i + 2]; q += h[4 * i + 3];
        }
        c->stats.cut_total = a; c->stats.visible_total = b; c->stats.pair_total = p;
        c->stats.candidate_total = q;
        // keep the planner's pair estimate above what was observed
        ngs_status ls = learn_pair_density(c);
        if (ls != NGS_OK) return ls;
    }
    *out = c->stats;
    return NGS_OK;
}

NGS_API ngs_status ngs_autotune(ngs_ctx *c, const ngs_camera *cams, int32_t n_cams,
                                float *const *d_images, int32_t reps, void *stream,
                                ngs_tune_result *out) {
    if (!c || !out || reps <= 0) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    // (binning tile, compositing block) candidates, as listed in ngs.h
    static const int kShapes[kTuneShapes][4] = {
        {8, 8, 8, 8},     {16, 8, 16, 8},   {16, 16, 16, 16}, {16, 32, 16, 32},
        {32, 16, 32, 16}, {32, 32, 32, 32}, {16, 16, 16, 8},  {16, 32, 16, 16},
        {32, 16, 16, 16}, {32, 32, 16, 16}, {32, 32, 32, 16}, {32, 32, 16, 8}};
    static const int kBatches[3] = {64, 128, 256};
    cudaStream_t st = (cudaStream_t)stream;
    const int mode = c->mode;
    const bool graph = c->use_graph, timing = c->timing;
    c->mode = NGS_MODE_BATCHED;
    c->use_graph = true;
    c->timing = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 3.4e38f;
    int bt = 2, bb = 1;
    ngs_status s = NGS_OK;
    for (int t = 0; t < kTuneShapes && s == NGS_OK; ++t)
        for (int b = 0; b < 3 && s == NGS_OK; ++b) {
            c->tile_w = kShapes[t][0];
            c->tile_h = kShapes[t][1];
            c->cta_w = kShapes[t][2];
            c->cta_h = kShapes[t][3];
            c->batch = kBatches[b];
            drop_graph(c);
            // capture + one warm-up replay, then the timed replays
            for (int k = 0; k < 2 && s == NGS_OK; ++k) s = render_common(c, cams, n_cams, d_images, st);
            if (s == NGS_OK) s = ngs_synchronize(c, stream);
            if (s != NGS_OK) break;
            cudaEventRecord(e0, st);
            for (int k = 0; k < reps && s == NGS_OK; ++k) s = render_common(c, cams, n_cams, d_images, st);
            cudaEventRecord(e1, st);
            if (s == NGS_OK) s = ngs_synchronize(c, stream);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            out->ms[t * 3 + b] = ms / reps;
            if (s == NGS_OK && ms / reps < best) { best = ms / reps; bt = t; bb = b; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tile_w = kShapes[bt][0];
    c->tile_h = kShapes[bt][1];
    c->cta_w = kShapes[bt][2];
    c->cta_h = kShapes[bt][3];
    c->batch = kBatches[bb];
    c->mode = mode;
    c->use_graph = graph;
    c->timing = timing;
    drop_graph(c);
    out->tile_w = c->tile_w;
    out->tile_h = c->tile_h;
    out->cta_w = c->cta_w;
    out->cta_h = c->cta_h;
    out->batch = c->batch;
    out->reserved = 0;
    return s;
}

NGS_API ngs_status ngs_stage_times(ngs_ctx *c, double *ms, int32_t n) {
    if (!c || !ms || n <= 0) return NGS_ERR_INVALID_ARG;
    if (!c->timing || c->ev_groups == 0) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const int groups = c->mode == NGS_MODE_PLAIN ? (int)c->host_cams.size()
                                                 : (int)c->last_plan.size();
    for (int k = 0; k < n; ++k) ms[k] = 0.0;
    for (int g = 0; g < groups && g < c->ev_groups; ++g) {
        CK(cudaEventSynchronize(c->ev[(size_t)g * kMarks + kMarks - 1]));
        for (int k = 0; k + 1 < kMarks && k < n; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, c->ev[(size_t)g * kMarks + k],
                                    c->ev[(size_t)g * kMarks + k + 1]));
            ms[k] += t;
        }
    }
    return NGS_OK;
}

NGS_API ngs_status ngs_debug_tile_lists(ngs_ctx *c, int32_t cam, int64_t *h_ranges,
                                        int32_t *h_nodes, int64_t cap, int64_t *n_pairs) {
    if (!c || !h_ranges || !n_pairs) return NGS_ERR_INVALID_ARG;
    if (c->last_plan.empty() || cam < 0 || cam >= (int32_t)c->host_cams.size())
        return NGS_ERR_INVALID_ARG;
    // node ids exist only for a render made with NGS_OPT_NODE_IDS on
    if (h_nodes && (!c->last_node_ids || !c->w.node_id)) return NGS_ERR_INVALID_ARG;
    // the work buffers hold the last sub-batch only
    const SubBatch &sb = c->last_plan.back();
    if (cam < sb.c0 || cam >= sb.c1) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    CK(cudaDeviceSynchronize());
    Work &w = c->w;
    const DevCamera &d = c->host_cams[cam];
    const int64_t nt = (int64_t)d.tiles_x * d.tiles_y;
    std::vector<uint2> rg(nt);
    CK(cudaMemcpy(rg.data(), w.ranges + d.tile_base, nt * sizeof(uint2), cudaMemcpyDeviceToHost));
    uint32_t npairs = 0;
    CK(cudaMemcpy(&npairs, w.counters + CNT_PAIRS, 4, cudaMemcpyDeviceToHost));
    const int psel = sb.tile_passes & 1;
    int64_t lo = INT64_MAX, hi = 0;
    for (int64_t t = 0; t < nt; ++t) rg[t].x = ~rg[t].x;   // stored as ~first
    for (int64_t t = 0; t < nt; ++t)
        if (rg[t].y > rg[t].x) { lo = std::min<int64_t>(lo, rg[t].x); hi = std::max<int64_t>(hi, rg[t].y); }
    if (lo == INT64_MAX) lo = hi = 0;
    *n_pairs = hi - lo;
    for (int64_t t = 0; t < nt; ++t) {
        h_ranges[2 * t] = rg[t].y > rg[t].x ? (int64_t)rg[t].x - lo : 0;
        h_ranges[2 * t + 1] = rg[t].y > rg[t].x ? (int64_t)rg[t].y - lo : 0;
    }
    if (hi - lo > cap) return NGS_ERR_CAPACITY;
    if (hi > lo && h_nodes) {
        std::vector<uint32_t> vals(hi - lo);
        CK(cudaMemcpy(vals.data(), w.pval[psel] + lo, (hi - lo) * 4, cudaMemcpyDeviceToHost));
        // copy the node ids of the span of records the pairs refer to once,
        // then look them up
        uint32_t r0 = UINT32_MAX, r1 = 0;
        for (int64_t k = 0; k < hi - lo; ++k) {
            r0 = std::min(r0, vals[k]);
            r1 = std::max(r1, vals[k]);
        }
        std::vector<uint32_t> ids((size_t)r1 - r0 + 1);
        CK(cudaMemcpy(ids.data(), w.node_id + r0, ids.size() * sizeof(uint32_t),
                      cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < hi - lo; ++k) h_nodes[k] = (int32_t)ids[vals[k] - r0];
    }
    (void)npairs;
    return NGS_OK;
}

NGS_API ngs_status ngs_slice_occupancy(ngs_ctx *c, const ngs_slice_grid *grid, float *d_value,
                                       uint8_t *d_occ, void *stream) {
    if (!c || !grid || !d_value) return NGS_ERR_INVALID_ARG;
    if (!c->loaded) return NGS_ERR_NOT_LOADED;
    const ngs_slice_grid &g = *grid;
    const float f[] = {g.x0, g.y0, g.cell, g.z0, g.dz, g.threshold};
    for (float v : f)
        if (!std::isfinite(v)) return NGS_ERR_INVALID_ARG;
    if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0 || !(g.cell > 0.0f) || !(g.dz > 0.0f))
        return NGS_ERR_INVALID_ARG;
    if ((int64_t)g.nx * g.ny * g.nz >= ((int64_t)1 << 31)) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    SliceGrid sg{g.x0, g.y0, g.cell, g.nx, g.ny, g.z0, g.dz, g.nz, g.threshold};
    ngs_status es = ensure_work(c);
    if (es != NGS_OK) return es;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemsetAsync(c->w.work64, 0, 2 * sizeof(unsigned long long), st));
    launch_slice(c->scene, sg, d_value, d_occ, c->w.work64 + 1, c->num_sms, st);
    CK(cudaGetLastError());
    return NGS_OK;
}

NGS_API ngs_status ngs_nav_fields(ngs_ctx *c, const uint8_t *d_occ, int32_t nx, int32_t ny,
                                  int32_t nz, int32_t k_lo, int32_t k_hi, int32_t inflate,
                                  const int32_t *goals, int32_t n_goals, uint8_t *d_blocked,
                                  uint32_t *d_dist, void *stream) {
    if (!c || !d_occ || !goals || !d_blocked || !d_dist) return NGS_ERR_INVALID_ARG;
    if (nx <= 0 || ny <= 0 || nz <= 0 || n_goals <= 0 || n_goals > 4096) return NGS_ERR_INVALID_ARG;
    if (k_lo < 0 || k_hi >= nz || k_lo > k_hi || inflate < 0 || inflate > 64)
        return NGS_ERR_INVALID_ARG;
    const int64_t plane = (int64_t)nx * ny;
    if (plane >= ((int64_t)1 << 30) || plane * n_goals >= ((int64_t)1 << 31))
        return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const size_t a_bytes = ((size_t)plane + 255) & ~(size_t)255;
    const size_t g_bytes = ((size_t)n_goals * sizeof(int2) + 255) & ~(size_t)255;
    const size_t need = a_bytes + g_bytes + (size_t)n_goals * 2 * plane * sizeof(uint32_t);
    cudaStream_t st = (cudaStream_t)stream;
    if (need > c->nav_tmp_bytes) {
        CK(cudaStreamSynchronize(st));
        if (c->nav_tmp) dfree(c->nav_tmp);
        c->nav_tmp = nullptr;
        c->nav_tmp_bytes = 0;
        ngs_status s = dalloc(&c->nav_tmp, need);
        if (s != NGS_OK) return s;
        c->nav_tmp_bytes = need;
    }
    std::vector<int2> hg((size_t)n_goals);
    for (int32_t g = 0; g < n_goals; ++g) hg[g] = make_int2(goals[2 * g], goals[2 * g + 1]);
    int2 *dg = reinterpret_cast<int2 *>(c->nav_tmp + a_bytes);
    CK(cudaMemcpyAsync(dg, hg.data(), (size_t)n_goals * sizeof(int2), cudaMemcpyHostToDevice, st));
    const int e = launch_nav_fields(d_occ, nx, ny, k_lo, k_hi, inflate, dg, n_goals, c->nav_tmp,
                                    reinterpret_cast<uint32_t *>(c->nav_tmp + a_bytes + g_bytes),
                                    d_blocked, d_dist, c->num_sms, st);
    if (e != 0) {
        std::fprintf(stderr, "ngs: nav fields: %s\n", cudaGetErrorString((cudaError_t)e));
        return NGS_ERR_CUDA;
    }
    return NGS_OK;
}

NGS_API ngs_status ngs_nav_paths(ngs_ctx *c, const uint32_t *d_dist, int32_t nx, int32_t ny,
                                 int32_t n_goals, const int32_t *d_starts, int32_t n,
                                 int32_t max_len, int32_t *d_paths, int32_t *d_len, void *stream) {
    if (!c || !d_dist || (n > 0 && (!d_starts || !d_paths || !d_len))) return NGS_ERR_INVALID_ARG;
    if (nx <= 0 || ny <= 0 || n_goals <= 0 || n < 0 || max_len <= 0) return NGS_ERR_INVALID_ARG;
    if ((int64_t)n * max_len >= ((int64_t)1 << 31)) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    launch_nav_paths(d_dist, nx, ny, n_goals, reinterpret_cast<const int3 *>(d_starts), n, max_len,
                     reinterpret_cast<int2 *>(d_paths), d_len, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return NGS_OK;
}

NGS_API ngs_status ngs_sort_pairs(ngs_ctx *c, void *d_keys, uint32_t *d_vals, int64_t n,
                                  int32_t key_bytes, int32_t begin_bit, int32_t end_bit,
                                  void *stream) {
    if (!c || (key_bytes != 4 && key_bytes != 8) || n < 0 || n >= ((int64_t)1 << 31))
        return NGS_ERR_INVALID_ARG;
    if (begin_bit < 0 || end_bit > 8 * key_bytes || begin_bit > end_bit) return NGS_ERR_INVALID_ARG;
    if (n > 0 && (!d_keys || !d_vals)) return NGS_ERR_INVALID_ARG;
    if (n == 0 || begin_bit == end_bit) return NGS_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->loaded && !c->work_ready) {
        // no scene: size the shared work state for sorting alone
        c->scene.n = 1;
    }
    ngs_status s = ensure_work(c);
    if (s != NGS_OK) return s;
    const int64_t parts = (n + sort_partition() - 1) / sort_partition();
    if (parts * 256 > c->w.status_words) return NGS_ERR_CAPACITY;
    if (n > c->sort_tmp_cap) {
        dfree(c->sort_tmp_keys);
        dfree(c->sort_tmp_vals);
        c->sort_tmp_keys = nullptr;
        c->sort_tmp_vals = nullptr;
        c->sort_tmp_cap = 0;
        if (dalloc((unsigned char **)&c->sort_tmp_keys, (size_t)n * key_bytes) != NGS_OK ||
            dalloc(&c->sort_tmp_vals, (size_t)n) != NGS_OK)
            return NGS_ERR_OUT_OF_MEMORY;
        c->sort_tmp_cap = n;
    }
    const int passes = sort_passes(begin_bit, end_bit);
    if ((s = epoch_guard(c, st, kEpochStride)) != NGS_OK) return s;
    CK(cudaMemsetAsync(c->w.counters, 0, N_COUNTERS * sizeof(uint32_t), st));
    k_bump_epoch<<<1, 1, 0, st>>>(c->w.epoch, kEpochStride);
    SortArgs a{};
    a.keys[0] = d_keys; a.keys[1] = c->sort_tmp_keys;
    a.vals[0] = d_vals; a.vals[1] = c->sort_tmp_vals;
    a.n_dev = nullptr; a.n_host = n; a.n_max = n;
    a.key_bytes = key_bytes; a.begin_bit = begin_bit; a.end_bit = end_bit;
    a.vals_identity = false;
    a.hist = c->w.hist; a.tickets = c->w.counters + TK_SORT0; a.status = c->w.status;
    a.epoch = c->w.epoch; a.epoch_off = 0; a.err = c->w.err;
    const int grid = (int)std::min<int64_t>(parts, key_bytes == 8 ? c->grid_sort64 : c->grid_sort32);
    launch_sort(a, std::max(grid, 1), st);
    if (passes & 1) {
        CK(cudaMemcpyAsync(d_keys, c->sort_tmp_keys, (size_t)n * key_bytes,
                           cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(d_vals, c->sort_tmp_vals, (size_t)n * 4, cudaMemcpyDeviceToDevice, st));
    }
    CK(cudaGetLastError());
    return NGS_OK;
}

NGS_API ngs_status ngs_scan_u32(ngs_ctx *c, const uint32_t *d_in, uint32_t *d_out, int64_t n,
                                uint32_t *d_total, void *stream) {
    if (!c || n < 0 || n >= ((int64_t)1 << 31)) return NGS_ERR_INVALID_ARG;
    if (n > 0 && (!d_in || !d_out)) return NGS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->loaded && !c->work_ready) c->scene.n = 1;
    ngs_status s = ensure_work(c);
    if (s != NGS_OK) return s;
    const int64_t parts = (n + scan_partition() - 1) / scan_partition();
    if (parts > c->w.status_words) return NGS_ERR_CAPACITY;
    if ((s = epoch_guard(c, st, kEpochStride)) != NGS_OK) return s;
    CK(cudaMemsetAsync(c->w.counters, 0, N_COUNTERS * sizeof(uint32_t), st));
    k_bump_epoch<<<1, 1, 0, st>>>(c->w.epoch, kEpochStride);
    if (n == 0) {
        if (d_total) CK(cudaMemsetAsync(d_total, 0, 4, st));
        return NGS_OK;
    }
    launch_scan_u32(d_in, d_out, nullptr, n, d_total, c->w.counters + TK_SCAN, c->w.status,
                    c->w.epoch, 0, c->w.err, (int)std::min<int64_t>(parts, c->grid_scan), st);
    CK(cudaGetLastError());
    return NGS_OK;
}

}  // extern "C"
