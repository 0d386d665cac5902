// Internal declarations shared by the renderer's translation units.
//
// Device data layout (structure of arrays, one entry per hierarchy node):
//   box_lo[n]  float4 (min.x, min.y, min.z, parent id as int bits)
//   box_hi[n]  float4 (max.x, max.y, max.z, child count as int bits)
//   pos4[n]    float4 (mean.x, mean.y, mean.z, flags as int bits)
//   quat[n]    float4 (w, x, y, z)
//   sop[n]     4 x A  (log_scale.x, .y, .z, opacity), A = float | half | bf16
//   sh[n]      48 x A (16 coefficients x RGB)
// Per render sub-batch (work buffers):
//   cut ids (uint32), compositing records (Rec32 / Rec16), depth keys and
//   record indices (double-buffered for the sort), tile rectangles, pair keys
//   and values (double-buffered), tile ranges.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ngs.h"

namespace ngs {

// ---------------------------------------------------------------------------
// constants of the render definition
// ---------------------------------------------------------------------------
constexpr float kNearZ = 0.2f;               // near plane on view z
constexpr double kNearZd = 0.2;
constexpr float kBlur = 0.3f;                // dilation added to the 2D covariance
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kRectMargin = 1.0f / 64.0f;  // pixels added to the support box
constexpr float kLog2e = 1.4426950408889634f;
// log2(1/255): alpha >= 1/255  <=>  log2(alpha) >= -log2(255)
constexpr float kLog2AlphaMin = -7.9943534368588578f;
// compositing drops a tile-list record whose largest log2 falloff over the
// tile's pixel-centre rectangle stays below log2(1/255) - kTileMarginLog2 (a
// margin far above float32 error, so no pixel that could reach 1/255 is lost)
constexpr float kTileMarginLog2 = 0.014426950408889634f;

constexpr uint32_t kNodeCullOpacity = 1u;    // pos4.w flag: 255 * opacity < 1

// error codes latched in the device status word (same values as ngs_status)
constexpr int kErrCapacity = NGS_ERR_CAPACITY;
constexpr int kErrTimeout = NGS_ERR_DEVICE_TIMEOUT;

// spin limit of every bounded device-side wait (look-back); a wait that runs
// out latches kErrTimeout and the kernel leaves the partition unfinished
constexpr uint32_t kSpinLimit = 1u << 20;

// ---------------------------------------------------------------------------
// per-camera table in device memory
// ---------------------------------------------------------------------------
struct DevCamera {
    float R[9];
    float pos[3];
    float fx, fy, cx, cy, tau;
    int32_t width, height, tiles_x, tiles_y;
    uint32_t tile_base;      // first tile id of this camera within its sub-batch
    uint32_t pad0;
    double posd[3];          // camera centre and depth row of R_wc in float64
    double Rz[3];
    float *image;            // [3][height][width]
    int64_t pad1;
    // cross products of the rows of R_wc: R0 x R1, R0 x R2, R2 x R1 (world
    // terms), for the normal of the projected Gaussian's two screen rows
    float X01[3], X02[3], X21[3];
    float pad2[3];
};
static_assert(sizeof(DevCamera) % 16 == 0, "DevCamera alignment");

// compositing records: centre (x, y); the log2 falloff of the Gaussian as
// L - (F1 dx + F2 dy)^2 - (F3 dy)^2 with L = log2(opacity) and F1, F2, F3 the
// Cholesky factors of the conic scaled by sqrt(log2(e) / 2) (this factored
// form keeps the thin direction of an elongated footprint, which rounding the
// three conic coefficients would lose); the colour, plus the half-widths of
// the support box (float32 record; float16 rounded up in the compact one)
struct __align__(16) Rec32 {
    float4 a;   // x, y, F1, F2
    float4 b;   // F3, L, r, g
    float4 c;   // bl, hx, hy, 0
};
struct __align__(16) Rec16 {
    float4 a;   // x, y, F1, F2
    float4 b;   // F3, L, half2(r, g) bits, half2(bl, max(hx, hy)) bits
};

// A visible Gaussian's tile rectangle [x0, x1] x [y0, y1] (tile coordinates of
// its camera, below 4096: images are at most 32768 pixels wide and high, tiles
// at least 8) and its camera within the launch (below 65536) in 8 bytes:
// x0 | y0 << 12 | camera bits 0-7 << 24, x1 | y1 << 12 | camera bits 8-15 << 24.
constexpr uint32_t kRectCoordMax = 4096;
struct RectU {
    uint32_t x0, y0, x1, y1, cam;
};
__host__ __device__ __forceinline__ uint2 pack_rect(uint32_t x0, uint32_t y0, uint32_t x1,
                                                    uint32_t y1, uint32_t cam) {
    return make_uint2(x0 | (y0 << 12) | ((cam & 0xffu) << 24),
                      x1 | (y1 << 12) | ((cam >> 8) << 24));
}
__host__ __device__ __forceinline__ RectU unpack_rect(const uint2 r) {
    RectU u;
    u.x0 = r.x & 0xfffu; u.y0 = (r.x >> 12) & 0xfffu;
    u.x1 = r.y & 0xfffu; u.y1 = (r.y >> 12) & 0xfffu;
    u.cam = (r.x >> 24) | ((r.y >> 24) << 8);
    return u;
}

struct SceneDev {
    int64_t n = 0;
    // nodes without children: a cut is an antichain of the tree, so no camera
    // selects more Gaussians than this
    int64_t n_leaves = 0;
    int32_t attr_dtype = NGS_F32;
    float4 *box_lo = nullptr, *box_hi = nullptr, *pos4 = nullptr, *quat = nullptr;
    void *sop = nullptr;     // [n][4] of attr type
    void *sh = nullptr;      // [n][48] of attr type
    // per block of cutpre_partition_nodes() consecutive nodes: box of the means
    // (xyz) with the largest scale (lo.w) and the largest 2 ln(255 o) (hi.w)
    float4 *blk_lo = nullptr, *blk_hi = nullptr;
    // the same bounds over the block's nodes and their parents: every
    // level-of-detail blend of a node with its parent lies within them
    float4 *blk_lo_b = nullptr, *blk_hi_b = nullptr;
    int64_t nblk = 0;
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void latch_error(int *status, int code) {
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Chained-scan status word: [63:62] flag (1 aggregate, 2 inclusive prefix),
// [61:32] epoch (30 bits), [31:0] value. A word whose epoch differs from the
// reader's belongs to an earlier scan and counts as "not yet published".
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint32_t kEpochMask = (1u << 30) - 1u;

__device__ __forceinline__ uint64_t pack_status(uint64_t flag, uint32_t epoch, uint32_t v) {
    return flag | ((uint64_t)(epoch & kEpochMask) << 32) | (uint64_t)v;
}

__device__ __forceinline__ void publish(uint64_t *slot, uint64_t word) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(slot), "l"(word) : "memory");
}

__device__ __forceinline__ uint64_t peek(const uint64_t *slot) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(slot) : "memory");
    return v;
}

// Granularity of a node box seen from camera centre (px, py, pz):
// s = fx * (longest box side) / (distance from the centre to the box), +inf
// when the centre is inside the box (level-of-detail cut, Sec. III-B). Its
// value feeds the level-of-detail blend weight; cut decisions use
// fine_enough below.
__device__ __forceinline__ float granularity(const float4 lo, const float4 hi, const float px,
                                             const float py, const float pz, const float fx) {
    const float gx = fmaxf(fmaxf(__fsub_rn(lo.x, px), 0.0f), __fsub_rn(px, hi.x));
    const float gy = fmaxf(fmaxf(__fsub_rn(lo.y, py), 0.0f), __fsub_rn(py, hi.y));
    const float gz = fmaxf(fmaxf(__fsub_rn(lo.z, pz), 0.0f), __fsub_rn(pz, hi.z));
    const float d2 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmul_rn(gz, gz)));
    const float ext = fmaxf(fmaxf(__fsub_rn(hi.x, lo.x), __fsub_rn(hi.y, lo.y)),
                            __fsub_rn(hi.z, lo.z));
    if (d2 == 0.0f) return __int_as_float(0x7f800000);
    return __fdiv_rn(__fmul_rn(fx, ext), __fsqrt_rn(d2));
}

// s(n) <= tau for the node box lo..hi, decided without the square root and
// the division of the granularity: fx ext <= tau sqrt(d2) <=> (fx ext)^2 <=
// tau^2 d2 (both sides >= 0), false when the camera is inside the box (s =
// +inf). Every kernel that takes a cut decision uses this one sequence of
// rounded operations, so all cut forms agree bit for bit; it differs from a
// comparison of the rounded granularity only within a few units in the last
// place of the threshold, far inside the 1e-5 tolerance around tau.
__device__ __forceinline__ float box_extent(const float4 lo, const float4 hi) {
    return fmaxf(fmaxf(__fsub_rn(hi.x, lo.x), __fsub_rn(hi.y, lo.y)), __fsub_rn(hi.z, lo.z));
}
// The same with the camera-independent box extent and the camera's tau^2
// (__fmul_rn(tau, tau)) taken beforehand: the same rounded operations.
__device__ __forceinline__ bool fine_enough_pre(const float4 lo, const float4 hi, const float ext,
                                                const float px, const float py, const float pz,
                                                const float fx, const float tau2) {
    const float gx = fmaxf(fmaxf(__fsub_rn(lo.x, px), 0.0f), __fsub_rn(px, hi.x));
    const float gy = fmaxf(fmaxf(__fsub_rn(lo.y, py), 0.0f), __fsub_rn(py, hi.y));
    const float gz = fmaxf(fmaxf(__fsub_rn(lo.z, pz), 0.0f), __fsub_rn(pz, hi.z));
    const float d2 = __fmaf_rn(gx, gx, __fmaf_rn(gy, gy, __fmul_rn(gz, gz)));
    if (d2 == 0.0f) return false;
    const float a = __fmul_rn(fx, ext);
    return __fmul_rn(a, a) <= __fmul_rn(tau2, d2);
}
__device__ __forceinline__ bool fine_enough(const float4 lo, const float4 hi, const float px,
                                            const float py, const float pz, const float fx,
                                            const float tau) {
    return fine_enough_pre(lo, hi, box_extent(lo, hi), px, py, pz, fx, __fmul_rn(tau, tau));
}

// The cut rule for node `node`: (leaf or s(n) <= tau) and (root or s(parent) > tau).
__device__ __forceinline__ bool cut_selects(const float4 *__restrict__ box_lo,
                                            const float4 *__restrict__ box_hi, int64_t node,
                                            float px, float py, float pz, float fx, float tau) {
    const float4 lo = box_lo[node], hi = box_hi[node];
    const int parent = __float_as_int(lo.w);
    const int nchild = __float_as_int(hi.w);
    const bool own = (nchild == 0) || fine_enough(lo, hi, px, py, pz, fx, tau);
    if (!own) return false;
    if (parent < 0) return true;
    return !fine_enough(box_lo[parent], box_hi[parent], px, py, pz, fx, tau);
}

// Decoupled look-back for one running sum: returns the exclusive prefix of
// partition `part` over the chain whose words sit at status[j * stride]. The
// caller has already published its own aggregate. The words of the next
// kLookBackWindow predecessors are requested together (one memory round trip
// per window) and consumed in order until an inclusive prefix is found; a
// window that reaches an unpublished word is requested again from there.
// Returns false (and latches kErrTimeout) if a predecessor never publishes
// within the spin limit.
constexpr int kLookBackWindow = 8;

__device__ __forceinline__ bool look_back(const uint64_t *status, int64_t part, int64_t stride,
                                          uint32_t epoch, uint32_t *excl, int *err) {
    uint32_t acc = 0;
    int64_t j = part - 1;
    uint32_t spins = 0;
    const uint32_t ep = epoch & kEpochMask;
    while (j >= 0) {
        uint64_t w[kLookBackWindow];
#pragma unroll
        for (int k = 0; k < kLookBackWindow; ++k)
            w[k] = j - k >= 0 ? peek(status + (j - k) * stride) : 0ull;
        bool stalled = false;
#pragma unroll
        for (int k = 0; k < kLookBackWindow; ++k) {
            if (stalled || j < 0) continue;
            const uint32_t e = (uint32_t)(w[k] >> 32) & kEpochMask;
            const uint64_t flag = w[k] & (3ull << 62);
            if (e != ep || flag == 0) {
                stalled = true;
                continue;
            }
            acc += (uint32_t)w[k];
            if (flag == kFlagPrefix) {
                *excl = acc;
                return true;
            }
            --j;
        }
        if (stalled && ++spins > kSpinLimit) {
            latch_error(err, kErrTimeout);
            *excl = acc;
            return false;
        }
    }
    *excl = acc;
    return true;
}

// ---------------------------------------------------------------------------
// work-buffer bundle for one render sub-batch
// ---------------------------------------------------------------------------
struct Work {
    // counters (device): [0] cut total, [1] visible total, [2] pair total,
    // [3..] tickets; zeroed at the start of each sub-batch
    uint32_t *counters = nullptr;
    uint32_t *epoch = nullptr;        // device epoch base, bumped per sub-batch
    uint64_t *status = nullptr;       // chained-scan words
    int64_t status_words = 0;
    int *err = nullptr;               // latched device error
    uint32_t *cut_ids = nullptr;      int64_t cut_cap = 0;
    uint32_t *cut_off = nullptr;      // [cams + 1]
    uint32_t *vis_count = nullptr;    // [cams] visible Gaussians per camera
    // cut+preprocess partition tables, [cams][node blocks]: live partition ids,
    // (record offset, count), dense position of the first record
    uint32_t *part_list = nullptr;
    uint2 *group_list = nullptr;
    uint2 *part_info = nullptr;
    uint32_t *part_pos = nullptr;
    int64_t part_cap = 0;
    void *rec = nullptr;              int64_t rec_cap = 0;
    uint32_t *dkey[2] = {nullptr, nullptr};
    uint32_t *didx[2] = {nullptr, nullptr};
    uint2 *rect = nullptr;            // tile rectangle and camera (pack_rect)
    uint2 *rect_sorted = nullptr;     // the visible rects in depth order
    uint32_t *node_id = nullptr;      // node of each record, kept on request only
    uint32_t *poff = nullptr;         // pair offsets per sorted record
    uint32_t *chunk_first = nullptr;  // first sorted record of each pair chunk
    uint32_t *pkey[2] = {nullptr, nullptr};
    uint32_t *pval[2] = {nullptr, nullptr};
    int64_t pair_cap = 0;
    uint2 *ranges = nullptr;          int64_t ranges_cap = 0;
    uint32_t *hist = nullptr;         // [passes][256] radix histograms
    DevCamera *cams = nullptr;        int64_t cams_cap = 0;
    // compositing work counters: [0] records staged, [1] pixel-Gaussian
    // evaluations, then per sub-batch (up to kTailSlots) the tail words of its
    // compositing launch
    unsigned long long *work64 = nullptr;
    uint32_t *order = nullptr;        // compositing work order of a sub-batch's tiles
};

constexpr int kTailSlots = 64;
constexpr int kWork64Words = 2 + 2 * kTailSlots;

// ticket slots in Work::counters
enum : int {
    CNT_CUT = 0, CNT_VIS = 1, CNT_PAIRS = 2, TK_CUT = 3, TK_PRE = 4, TK_SCAN = 5, TK_DUP = 6,
    TK_SORT0 = 8,             // 8 .. 8 + 16: one ticket per sort pass
    CNT_ALLOC = 24,           // 24, 25: 64-bit record allocation counter
    CNT_LIVE = 26,            // live cut+preprocess partitions
    CNT_GROUPS = 27,          // groups of live partitions (same node block)
    TK_COMPOSITE = 28, N_COUNTERS = 32
};

// ---------------------------------------------------------------------------
// kernel launchers (one translation unit each)
// ---------------------------------------------------------------------------
// cut: cameras [0, n_cams) of the table; writes ids (ascending per camera),
// offsets [n_cams + 1] and counters[CNT_CUT]
void launch_cut(const SceneDev &sc, const DevCamera *cams, int n_cams, uint32_t *ids,
                int64_t cap, uint32_t *offsets, uint32_t *counters, uint32_t *ticket,
                uint64_t *status, const uint32_t *epoch, uint32_t epoch_off, int *err,
                int grid, cudaStream_t st);
int cut_partition_nodes();

// fused cut + preprocess of cameras [0, n_cams): the candidates of each
// partition (block of cutpre_partition_nodes() nodes, camera) in node order at
// an atomically allocated offset of rec / dkey_sparse / rect, invisible ones
// as holes (key 0xffffffff); (offset, visible | candidates << 16) per
// partition in part_info[camera * nblk + block]; visible Gaussians per
// camera in vis_count; counters[CNT_CUT], [CNT_LIVE], [CNT_GROUPS],
// [CNT_ALLOC], [TK_PRE]. part_list and group_list hold part_cap entries.
// blend: level-of-detail blending of every node toward its parent.
// node_id (may be null): each visible record's node id.
void launch_cutpre(const SceneDev &sc, const DevCamera *cams, int n_cams, void *rec,
                   int64_t rec_cap, uint32_t *dkey_sparse, uint2 *rect, uint32_t *node_id,
                   uint32_t *vis_count,
                   uint32_t *counters, uint32_t *part_list, uint2 *group_list, uint2 *part_info,
                   int *err, int tile_w, int tile_h, int use_block_cull, int blend, int grid,
                   cudaStream_t st);
int cutpre_partition_nodes();
void cutpre_init_attributes();
// dense depth keys (camera-major, node order) and their record indices for the
// sort, and the depth sort's digit histograms in hist[4][256]; counters[CNT_VIS]
void launch_gather_keys(const uint32_t *vis_count, int n_cams, const SceneDev &sc,
                        const uint2 *part_info, uint32_t *part_pos, const uint32_t *part_list,
                        const uint32_t *dkey_sparse, uint32_t *dkey, uint32_t *didx,
                        uint32_t *counters, int64_t cap, uint32_t *hist, int *err, int grid,
                        cudaStream_t st);

// radix sort (onesweep) of (uint32 | uint64 key, uint32 value) pairs; n from
// device memory (*n_dev) or host (n_host >= 0). Result lands in buffer
// `out_sel` (0 or 1) of the double buffers; the number of passes decides it.
struct SortArgs {
    void *keys[2];
    uint32_t *vals[2];
    const uint32_t *n_dev;
    int64_t n_host;
    int64_t n_max;            // bound on n (status array and grid sizing)
    int key_bytes;
    int begin_bit, end_bit;
    bool vals_identity;       // first pass takes value = input index
    bool hist_ready;          // hist already holds the digit counts (no upsweep)
    uint32_t *hist;           // [passes][256]
    // last pass: skip_last_keys writes the values only (the sorted keys are
    // not needed afterwards); a non-null ranges (32-bit tile keys only) also
    // records every key's [first, end) there, encoded as in k_ranges (x holds
    // ~first, so zeroed entries mean "no pairs"), and implies skip_last_keys
    bool skip_last_keys;
    uint2 *ranges;
    uint32_t *tickets;        // one per pass
    uint64_t *status;
    const uint32_t *epoch;
    uint32_t epoch_off;
    int *err;
    // optional hook run on the host after the histogram (step 0) and after
    // every digit pass (step p + 1): used to record timing events
    void (*hook)(void *user, int step);
    void *hook_user;
};
int sort_passes(int begin_bit, int end_bit);
int sort_partition();
size_t sort_smem_bytes(int key_bytes);
void sort_init_attributes();
void launch_sort(const SortArgs &a, int grid, cudaStream_t st);

// exclusive scan of uint32 (device-count or host-count)
void launch_scan_u32(const uint32_t *in, uint32_t *out, const uint32_t *n_dev, int64_t n_host,
                     uint32_t *total, uint32_t *ticket, uint64_t *status, const uint32_t *epoch,
                     uint32_t epoch_off, int *err, int grid, cudaStream_t st);
int scan_partition();

// binning: tiles-touched scan over depth order (also the first record of every
// pair chunk, chunk_first[dup_chunks(pair_cap)], and the rects in depth order
// in rect_sorted); with hist, it also adds the digit counts
// of the pairs' tile keys (camera tile base + row * tiles_x + column) for
// `passes` 8-bit radix passes to hist[passes][256] (zeroed by the caller)
void launch_pair_offsets(const uint2 *rect, const uint32_t *sorted_idx, const uint32_t *n_vis,
                         uint32_t *poff, uint32_t *counters, int64_t pair_cap, uint32_t *ticket,
                         uint64_t *status, const uint32_t *epoch, uint32_t epoch_off, int *err,
                         uint32_t *chunk_first, uint2 *rect_sorted, const DevCamera *cams,
                         uint32_t *hist, int passes, int grid, cudaStream_t st);
int64_t dup_chunks(int64_t pair_cap);
// emits the pairs from the depth-ordered rects and their record indices
// (sorted_idx, as given to launch_pair_offsets)
void launch_duplicate(const uint2 *rect_sorted, const uint32_t *sorted_idx, const uint32_t *poff,
                      const uint32_t *chunk_first, const uint32_t *n_vis, const uint32_t *n_pairs,
                      int64_t pair_cap, const DevCamera *cams, uint32_t *pkey, uint32_t *pval,
                      int *err, int grid, cudaStream_t st);
void launch_ranges(const uint32_t *pkey, const uint32_t *n_pairs, uint2 *ranges, int grid,
                   cudaStream_t st, const int *err);

// compositing of tiles [0, n_tiles) of a sub-batch
// GS-slice occupancy grid (see include/ngs.h, ngs_slice_grid)
struct SliceGrid {
    float x0, y0, cell;
    int32_t nx, ny;
    float z0, dz;
    int32_t nz;
    float threshold;
};
// value: [nz][ny][nx] float32, zeroed here; occ (optional): the mask
void launch_slice(const SceneDev &sc, const SliceGrid &g, float *value, uint8_t *occ,
                  unsigned long long *work, int num_sms, cudaStream_t st);

// tile_w x tile_h: binning tile; cta_w x cta_h: the block one CTA composites
// (equal to the tile, or a compiled shape dividing it). order (optional, a
// permutation of the tiles): the order in which persistent CTAs take them.
// tail (optional, 2 words zeroed by the caller): ~(time the first CTA found
// the work queue empty) and the time the last CTA finished, as atomicMax.
void launch_composite(int attr_dtype, int tile_w, int tile_h, int cta_w, int cta_h, int batch,
                      bool persistent, const DevCamera *cams, int n_cams, uint32_t n_tiles,
                      const uint2 *ranges, const uint32_t *pval, const void *rec,
                      uint32_t *ticket, int grid, const int *err, unsigned long long *work64,
                      const uint32_t *order, unsigned long long *tail, cudaStream_t st);
// the tiles [0, n_tiles) of a sub-batch, longest list first (classes of half
// an octave), into order[n_tiles]
void launch_tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, const int *err,
                       cudaStream_t st);
int composite_blocks_per_sm(int attr_dtype, int tile_w, int tile_h, int batch);
void composite_init_attributes();

// serving lanes: contexts sharing a parent's resident scene
ngs_status lane_create(ngs_ctx *parent, int64_t record_capacity, int64_t pair_capacity,
                       ngs_ctx **out);
// the planner's current pairs-per-pixel estimate of a context
double ctx_pairs_per_pixel(const ngs_ctx *c);

inline size_t rec_bytes(int attr_dtype) {
    return attr_dtype == NGS_F32 ? sizeof(Rec32) : sizeof(Rec16);
}

}  // namespace ngs
