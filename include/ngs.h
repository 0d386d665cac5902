/*
 * ngs.h - C ABI of the GB300 hierarchical Gaussian-splatting renderer.
 *
 * The renderer draws camera views of a hierarchical 3D Gaussian Splatting
 * scene: a tree whose leaves are fine anisotropic Gaussians and whose interior
 * nodes are coarser aggregates (NavGSim, Sec. III-B). Per view it selects a
 * level-of-detail cut of the tree at a pixel granularity tau (Sec. III-B:
 * Gaussians are picked from different levels per view), projects the cut's
 * Gaussians to screen with the EWA approximation and degree-3 spherical
 * harmonic colour, bins them into screen tiles by duplicated (tile, depth)
 * keys and a radix sort, and blends each pixel front to back (Sec. III-A: views
 * rendered in real time from camera intrinsics and extrinsics alone).
 *
 * Conventions shared by every call
 *  - All functions return an ngs_status; nothing throws or exits across the ABI.
 *  - Device pointers ("d_" prefix) are CUDA device addresses on the context's
 *    device; host pointers are ordinary host memory. Streams are passed as
 *    `void *` holding a cudaStream_t (NULL = legacy default stream).
 *  - Work enqueued on a stream is asynchronous. Errors detected on the device
 *    (capacity overflow, a bounded wait that gave up) are latched in the
 *    context and returned by ngs_synchronize() and by the next call; the
 *    context stays usable after NGS_ERR_CAPACITY and NGS_ERR_INVALID_ARG.
 *  - Scene arrays passed to ngs_load_scene are copied; the caller keeps
 *    ownership. Images and cut buffers are caller-owned device memory.
 *  - One context is used from one host thread at a time.
 */
#ifndef NGS_H
#define NGS_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NGS_API __attribute__((visibility("default")))

typedef enum {
    NGS_OK = 0,
    NGS_ERR_INVALID_ARG = 1,        /* bad pointer, size, camera or option */
    NGS_ERR_INVALID_HIERARCHY = 2,  /* scene tree fails validation at load */
    NGS_ERR_OUT_OF_MEMORY = 3,      /* device allocation failed */
    NGS_ERR_CAPACITY = 4,           /* a work buffer (cut, records, pairs) was too small */
    NGS_ERR_CUDA = 5,               /* a CUDA runtime call failed */
    NGS_ERR_DEVICE_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    NGS_ERR_NOT_LOADED = 7          /* render or cut requested before ngs_load_scene */
} ngs_status;

typedef enum { NGS_F32 = 0, NGS_F16 = 1, NGS_BF16 = 2 } ngs_dtype;

/* Pinhole camera, OpenCV frame (x right, y down, z forward). A world point x
 * maps to t = R_wc (x - pos) and to pixel (fx t.x / t.z + cx, fy t.y / t.z + cy);
 * pixel (i, j) is sampled at (i + 0.5, j + 0.5). R_wc is row-major. tau is the
 * level-of-detail granularity in pixels (0 selects every leaf). */
typedef struct {
    float pos[3];
    float R_wc[9];
    float fx, fy, cx, cy;
    int32_t width, height;
    float tau;
} ngs_camera;

/* One entry per hierarchy node (leaves and interior nodes alike), node ids as
 * in ngs_hierarchy. pos [n][3] and quat [n][4] (w, x, y, z; normalised by the
 * renderer) are float32. log_scale [n][3] (natural log of the per-axis standard
 * deviation), opacity [n] (in (0, 1)) and sh [n][16][3] (degree-3 SH
 * coefficients, coefficient-major, RGB minor) are of type attr_dtype: float32,
 * float16, or bfloat16 (as uint16 bit patterns). Reduced-precision attributes
 * are stored as given and widened to float32 in the kernels. */
typedef struct {
    int64_t n;
    const float *pos;
    const float *quat;
    const void *log_scale;
    const void *opacity;
    const void *sh;
    int32_t attr_dtype;
} ngs_gaussians;

/* Tree over the same n nodes. Node 0 is the root (parent -1); ids are
 * breadth-first so the children of a node are child_begin .. child_begin +
 * child_count - 1, all with larger ids than their parent; leaves have
 * child_count 0. aabb_min/aabb_max [n][3] float32: every child's box lies in
 * its parent's box. Validated at load (NGS_ERR_INVALID_HIERARCHY otherwise). */
typedef struct {
    const int32_t *parent;
    const int32_t *child_begin;
    const int32_t *child_count;
    const float *aabb_min;
    const float *aabb_max;
} ngs_hierarchy;

typedef struct ngs_ctx ngs_ctx;

/* Context configuration. Zero fields take defaults. Capacities bound the work
 * buffers of one sub-batch of cameras: cut_capacity (selected node ids),
 * record_capacity (visible Gaussians after culling), pair_capacity ((tile,
 * Gaussian) pairs). A render whose sub-batch exceeds a capacity latches
 * NGS_ERR_CAPACITY and leaves the affected images undefined. */
typedef struct {
    int32_t device;
    int32_t tile_w, tile_h;          /* tile shape: 8x8, 16x8, 16x16, 16x32, 32x16 or 32x32
                                        (default 16x16) */
    int32_t batch;                   /* records staged per compositing round: 64, 128, 256 (default 128) */
    int64_t cut_capacity;            /* default 2^27 */
    int64_t record_capacity;         /* default 2^26 */
    int64_t pair_capacity;           /* default 2^29 */
    int32_t max_tiles_per_batch;     /* tiles per sub-batch, <= 65536 (default 65536) */
    int32_t reserved;
} ngs_config;

/* Render paths (ngs_set_option NGS_OPT_MODE). BATCHED: all cameras of a call
 * in sub-batches, persistent device-sized kernels, replayed from a CUDA graph
 * when the camera layout repeats. PLAIN: one camera at a time, sizes read back
 * to the host between stages, no graph. Both compute identical pixels. */
enum { NGS_MODE_BATCHED = 0, NGS_MODE_PLAIN = 1 };
enum { NGS_OPT_MODE = 1, NGS_OPT_TILE_W = 2, NGS_OPT_TILE_H = 3, NGS_OPT_BATCH = 4,
       NGS_OPT_GRAPH = 5, NGS_OPT_STAGE_TIMING = 6, NGS_OPT_BLOCK_CULL = 7,
       NGS_OPT_CTA_W = 8, NGS_OPT_CTA_H = 9, NGS_OPT_PAIRS_PER_PIXEL = 10,
       NGS_OPT_LOD_BLEND = 11, NGS_OPT_COMPOSITE_ORDER = 12, NGS_OPT_NODE_IDS = 13 };
/* NGS_OPT_TILE_W / NGS_OPT_TILE_H: tile width 8, 16 or 32, height 8, 16 or 32;
 * a render accepts the shapes 8x8, 16x8, 16x16, 16x32, 32x16 and 32x32
 * (INVALID_ARG else).
 * Every shape gives the same pixels.
 * NGS_OPT_CTA_W / NGS_OPT_CTA_H (default 0 = the tile): the pixel block one
 * compositing CTA covers. A tile may be composited as equal blocks of a
 * supported shape that divides it (e.g. a 32x32 tile as four 16x16 blocks):
 * binning and sorting work on the large tiles (fewer pairs), each block walks
 * its tile's list and skips the Gaussians that cannot reach it. A shape that
 * does not divide the tile is rejected at render (INVALID_ARG). Same pixels.
 * NGS_OPT_LOD_BLEND (default 0): level-of-detail blending (Sec. III-B: the
 * transitions between levels are interpolated). A selected node n other than
 * the root is rendered with its attributes moved toward its parent p's by the
 * parent weight v = 1 - clamp((s(p) - tau) / (s(p) - s(n)), 0, 1) (0 where s(p)
 * is infinite or s(p) <= s(n)): mean mu_n + v (mu_p - mu_n), and likewise the
 * 3D covariance, the opacity and the SH coefficients. v and the mean are
 * evaluated in float32 by a fixed IEEE operation sequence. v = 0 for every
 * node at tau = 0, where the images equal the plain ones bit for bit. While it
 * is on, the pre-culls bound the segment from a node's mean to its parent's
 * with the larger scale and opacity of the two (a blended Gaussian lies
 * within those bounds).
 * NGS_OPT_PAIRS_PER_PIXEL (1..4096, default 48): the planner's estimate of
 * (tile, Gaussian) pairs per pixel, used to fit sub-batches into
 * pair_capacity; it is raised automatically to 1.25x the densest sub-batch a
 * render observed (read by ngs_last_stats, and by ngs_synchronize when it
 * returns NGS_ERR_CAPACITY, so that rendering the same cameras again fits). A
 * render whose pairs still exceed the capacity latches NGS_ERR_CAPACITY.
 * NGS_OPT_BLOCK_CULL (default 1): skip, per camera, node blocks that provably
 * hold no visible Gaussian; 0 tests every node (same images, slower).
 * NGS_OPT_COMPOSITE_ORDER (default 1): the batched path's persistent
 * compositing CTAs take the tiles of a sub-batch in order of decreasing list
 * length (classes of half an octave), so that long lists do not start last;
 * 0 takes them in tile order. Same images.
 * NGS_OPT_NODE_IDS (default 0): renders also keep each visible Gaussian's node
 * id (4 bytes per record_capacity entry, allocated at the first such render),
 * which ngs_debug_tile_lists reports. Same images. */

typedef struct {
    int64_t cut_total;       /* selected nodes over all cameras of the last render */
    int64_t visible_total;   /* Gaussians kept after culling */
    int64_t pair_total;      /* (tile, Gaussian) pairs */
    int64_t records_staged;  /* records gathered into shared memory by compositing */
    int64_t evaluations;     /* pixel-Gaussian evaluations done by compositing */
    int32_t sub_batches;     /* sub-batches of the last render */
    int32_t graph_replayed;  /* 1 if the last render replayed a captured graph */
    int32_t tile_w, tile_h, batch, mode;
    int32_t kernels;         /* kernel launches of the last render */
    int32_t cta_w, cta_h;    /* compositing block of the last render */
    int32_t reserved;
    /* batched path: milliseconds, summed over the sub-batches, from the moment
     * the first compositing CTA of a launch found its work queue empty to the
     * end of the launch's last CTA (the launch's tail); 0 in the plain path */
    double composite_tail_ms;
    /* batched path: (node, camera) candidates the fused cut + preprocess
     * passed to its full preprocess (the visible ones and the holes left by
     * those that turned out invisible); -1 in the plain path */
    int64_t candidate_total;
} ngs_stats;

NGS_API const char *ngs_strerror(ngs_status s);

/* Creates a context on cfg->device (cfg may be NULL for defaults). */
NGS_API ngs_status ngs_create(const ngs_config *cfg, ngs_ctx **out);
NGS_API ngs_status ngs_destroy(ngs_ctx *ctx);
NGS_API ngs_status ngs_set_option(ngs_ctx *ctx, int32_t option, int64_t value);

/* Copies a scene (host arrays) to the device, replacing any previous one.
 * Synchronous. Validates the hierarchy (root 0, contiguous children, parent
 * ids, nested boxes, leaf child counts). */
NGS_API ngs_status ngs_load_scene(ngs_ctx *ctx, const ngs_gaussians *g, const ngs_hierarchy *h);

/* Level-of-detail cut (Sec. III-B): for camera c, node n is selected iff
 * (n is a leaf or s(n) <= tau_c) and (n is the root or s(parent(n)) > tau_c),
 * with s(n) = fx * (longest side of box(n)) / (distance from pos to box(n)),
 * s = +inf when the camera is inside the box. Writes the selected ids of
 * camera c, ascending, to d_ids[d_offsets[c] .. d_offsets[c+1]) (device
 * int32, capacity cap entries; d_offsets: device int64 [n_cams + 1]);
 * 1 <= n_cams <= 1024. A cut holds at most one id per leaf, and the offsets
 * are counted in 32 bits: a call with n_cams x (leaves of the scene) >= 2^32
 * returns NGS_ERR_CAPACITY before any work (split the cameras over calls).
 * Synchronises the stream. Returns NGS_ERR_CAPACITY if the cuts exceed cap
 * (the offsets still hold their sizes). */
NGS_API ngs_status ngs_select_cut(ngs_ctx *ctx, const ngs_camera *cams, int32_t n_cams,
                                  int32_t *d_ids, int64_t *d_offsets, int64_t cap, void *stream);

/* Frustum-culled and shared cuts (Sec. III-B: the levels are selected per
 * view, dynamically).
 *  - Frustum cull (flags & NGS_CUT_FRUSTUM): the view volume of a camera with
 *    a guard band of g = guard_px pixels, {x : t_z >= 0.2, -g <= u <= W + g,
 *    -g <= v <= H + g} (t = R_wc (x - pos), u = fx t_x / t_z + cx,
 *    v = fy t_y / t_z + cy), is the intersection of five half-spaces (near,
 *    left, right, top, bottom); a node whose box lies wholly outside one of
 *    them is culled, and with it its subtree.
 *  - Shared cuts: the cameras form n_groups consecutive groups, group g being
 *    cams[group_begin[g] .. group_begin[g + 1]) (host int32 [n_groups + 1],
 *    group_begin[0] = 0, strictly ascending, group_begin[n_groups] = n_cams).
 *    Node n is fine enough for a group when every member culls it (cull on)
 *    or has s(n) <= tau; n is selected iff (leaf or fine(n)) and (root or not
 *    fine(parent)) and, with the cull on, some member keeps it. On every
 *    root-to-leaf path this is the deepest of the members' own choices, so
 *    each member gets at least the detail it asks for wherever it sees.
 * A group of one camera without the cull gives ngs_select_cut's cut.
 * 1 <= n_groups <= n_cams <= 1024. Output as ngs_select_cut, per group: ascending ids in d_ids[d_offsets[g] ..
 * d_offsets[g + 1]) (device int32 [cap], device int64 [n_groups + 1]).
 * NGS_ERR_INVALID_ARG for a bad group table, unknown flags, a negative or
 * non-finite guard, or a bad camera; NGS_ERR_CAPACITY if the cuts exceed cap
 * (the offsets still hold their sizes), or before any work when n_groups x
 * (leaves of the scene) >= 2^32. Synchronises the stream. */
#define NGS_CUT_FRUSTUM 1
NGS_API ngs_status ngs_select_cut_shared(ngs_ctx *ctx, const ngs_camera *cams, int32_t n_cams,
                                         const int32_t *group_begin, int32_t n_groups,
                                         uint32_t flags, float guard_px, int32_t *d_ids,
                                         int64_t *d_offsets, int64_t cap, void *stream);

/* Renders n_cams views (host camera array) into d_images[c] (host array of
 * device pointers), each float32 planar [3][height][width], background 0.
 * Per pixel p and the Gaussians g of its tile in (depth, node id) order:
 * alpha = min(0.99, o_g exp(-1/2 d^T conic_g d)), skipped if alpha < 1/255;
 * blending stops before the Gaussian that would bring T below 1e-4;
 * C += alpha T c_g; T *= 1 - alpha. Asynchronous on `stream`. */
NGS_API ngs_status ngs_render(ngs_ctx *ctx, const ngs_camera *cams, int32_t n_cams,
                              float *const *d_images, void *stream);

/* As ngs_render into host memory, then synchronises the stream. h_images[c]
 * holds 3 x H x W floats. Page-locked memory the device can address
 * (cudaHostAlloc'd or registered and mapped) is written directly by the
 * render kernels; other host memory (pageable) receives a copy of each
 * sub-batch's images as soon as they are complete, while the next sub-batches
 * render. A buffer smaller than its image is undefined behaviour either way
 * (written past its end). A batched render whose pairs
 * overflowed pair_capacity is planned again from the pair counts the device
 * reported (smaller sub-batches) and redone, up to 4 renders in all; it
 * returns NGS_ERR_CAPACITY only if that does not suffice (for example one
 * camera alone exceeds the capacity). */
NGS_API ngs_status ngs_render_host(ngs_ctx *ctx, const ngs_camera *cams, int32_t n_cams,
                                   float *const *h_images, void *stream);

/* Failure-detection self-test: launches one device-side wait on a status
 * word that nothing will ever publish. The wait is bounded (about 2^20 polls,
 * well under a second): it gives up, latches NGS_ERR_DEVICE_TIMEOUT, and the
 * kernel returns. Synchronises and returns that status; the context stays
 * usable. */
NGS_API ngs_status ngs_selftest_wait_timeout(ngs_ctx *ctx, void *stream);

/* Waits for the stream and returns (then clears) any latched device error. */
NGS_API ngs_status ngs_synchronize(ngs_ctx *ctx, void *stream);

/* Candidates of ngs_autotune, as (binning tile / compositing block):
 *   0 8x8/8x8      1 16x8/16x8     2 16x16/16x16   3 16x32/16x32
 *   4 32x16/32x16  5 32x32/32x32   6 16x16/16x8    7 16x32/16x16
 *   8 32x16/16x16  9 32x32/16x16  10 32x32/32x16  11 32x32/16x8
 * each with the compositing batches {64, 128, 256}. */
#define NGS_TUNE_SHAPES 12

/* Result of ngs_autotune: the chosen tile shape, compositing block and staging
 * batch, and the measured milliseconds of one render of the given cameras for
 * every candidate (index = shape index * 3 + batch index). */
typedef struct {
    int32_t tile_w, tile_h, cta_w, cta_h, batch;
    int32_t reserved;
    float ms[NGS_TUNE_SHAPES * 3];
} ngs_tune_result;

/* Autotuner of the batched path: renders `cams` (into d_images) with every
 * candidate shape and compositing batch, each captured in its CUDA graph,
 * warmed up and timed over `reps` replays with CUDA events on `stream`, then
 * keeps the fastest setting in the context. All candidates give bit-identical
 * images. Synchronous. */
NGS_API ngs_status ngs_autotune(ngs_ctx *ctx, const ngs_camera *cams, int32_t n_cams,
                                float *const *d_images, int32_t reps, void *stream,
                                ngs_tune_result *out);

/* Synchronises the device and fills *out for the last render. */
NGS_API ngs_status ngs_last_stats(ngs_ctx *ctx, ngs_stats *out);

/* With NGS_OPT_STAGE_TIMING on, every kernel of a render is bracketed by CUDA
 * events on the render stream (captured into the graph when one is used).
 * After synchronising, ms[k] (k < n, n <= 15) receives the milliseconds of
 * stage k summed over the last render's sub-batches (batched) or cameras
 * (plain): 0 fused cut + preprocess, 1 dense depth keys, 2 depth histogram,
 * 3..6 depth digit passes,
 * 7 pair offsets, 8 pair duplication, 9 tile histogram, 10..12 tile digit
 * passes, 13 tile ranges, 14 compositing. Unused passes read 0. */
NGS_API ngs_status ngs_stage_times(ngs_ctx *ctx, double *ms, int32_t n);

/* Tile lists of the last render, for camera `cam` of a single-sub-batch
 * render, copied to host memory after synchronising: h_ranges [tiles][2]
 * (int64 start, end into h_nodes) and h_nodes [cap] (int32 node ids in
 * per-tile depth order). *n_pairs receives the number of pairs; returns
 * NGS_ERR_CAPACITY if it exceeds cap. tiles = ceil(W/tile_w)*ceil(H/tile_h).
 * h_nodes may be NULL (ranges only); non-NULL needs a last render made with
 * NGS_OPT_NODE_IDS on (NGS_ERR_INVALID_ARG else). */
NGS_API ngs_status ngs_debug_tile_lists(ngs_ctx *ctx, int32_t cam, int64_t *h_ranges,
                                        int32_t *h_nodes, int64_t cap, int64_t *n_pairs);

/* GS-slice occupancy (Sec. III-C: the scene's Gaussians cut by horizontal
 * planes give the floor-level occupancy used for collision checks). Plane k
 * lies at height z0 + k dz; cell (i, j) of a plane spans [x0 + i cell, x0 +
 * (i + 1) cell) x [y0 + j cell, y0 + (j + 1) cell). */
typedef struct {
    float x0, y0, cell;
    int32_t nx, ny;
    float z0, dz;
    int32_t nz;
    float threshold;      /* a cell is occupied where its value >= threshold */
} ngs_slice_grid;

/* Cuts every leaf Gaussian of the loaded scene by the grid's planes. A plane at
 * height z cuts G3D(x) = exp(-1/2 (x - mu)^T Sigma^-1 (x - mu)) in the 2D
 * Gaussian exp(-1/2 lambda (z - mu_z)^2) exp(-1/2 [x - mu(z)]^T C [x - mu(z)]),
 * C the xy block of Sigma^-1, (alpha, beta) = C^-1 (c_xz, c_yz), mu(z) = mu_xy -
 * (z - mu_z) (alpha, beta), lambda = c_zz - alpha^2 c_xx - beta^2 c_yy -
 * 2 alpha beta c_xy. d_value [nz][ny][nx] (device float32, caller-owned)
 * receives per cell the largest min(0.99, o G2D(cell centre, z)) over the
 * leaves for which that value is >= 1/255 (0 if none); d_occ (device uint8,
 * same shape, may be NULL) receives value >= threshold. Asynchronous on
 * `stream`. NGS_ERR_INVALID_ARG for a non-positive size, cell or dz, a
 * non-finite field, or nx * ny * nz >= 2^31; NGS_ERR_NOT_LOADED without a
 * scene. */
NGS_API ngs_status ngs_slice_occupancy(ngs_ctx *ctx, const ngs_slice_grid *grid, float *d_value,
                                       uint8_t *d_occ, void *stream);

/* Navigation on the slice occupancy (Sec. III-C: navigable areas for
 * collision checks and path planning; Sec. IV-A: expert trajectories from a
 * shortest-path planner). d_occ: device uint8 [nz][ny][nx] (e.g. the d_occ of
 * ngs_slice_occupancy). d_blocked (device uint8 [ny][nx]) receives 1 where some
 * plane k_lo..k_hi (the robot's height range) is occupied within Chebyshev
 * distance `inflate` cells (the robot's footprint; 0..64). For each goal g
 * (host int32 [n_goals][2] = cell (i, j)), d_dist + g * ny * nx (device uint32)
 * receives the 4-connected breadth-first step count from the goal over the
 * free cells, 0xffffffff where unreachable (also everywhere when the goal is
 * blocked or outside the grid). Synchronous: returns once the fields are
 * complete. The context keeps a scratch buffer for it (two frontier queues of
 * ny * nx entries per goal), grown on demand. */
NGS_API ngs_status ngs_nav_fields(ngs_ctx *ctx, const uint8_t *d_occ, int32_t nx, int32_t ny,
                                  int32_t nz, int32_t k_lo, int32_t k_hi, int32_t inflate,
                                  const int32_t *goals, int32_t n_goals, uint8_t *d_blocked,
                                  uint32_t *d_dist, void *stream);

/* Shortest paths for n agents: d_starts (device int32 [n][3]) = start cell
 * (i, j) and goal index. Each path descends its goal's field from the start,
 * taking the first neighbour in the order (+x, -x, +y, -y) whose distance is
 * one less; d_paths (device int32 [n][max_len][2]) receives its cells from the
 * start to the goal and d_len [n] their number (0 when the start is unreachable;
 * at most max_len). Asynchronous on `stream`. */
NGS_API ngs_status ngs_nav_paths(ngs_ctx *ctx, const uint32_t *d_dist, int32_t nx, int32_t ny,
                                 int32_t n_goals, const int32_t *d_starts, int32_t n,
                                 int32_t max_len, int32_t *d_paths, int32_t *d_len, void *stream);

/* Stable LSD radix sort (onesweep: one histogram pass, then one chained-scan
 * scatter pass per 8-bit digit) of n (key, value) pairs by key bits
 * [begin_bit, end_bit). d_keys/d_vals: device arrays sorted in place; keys are
 * uint32 (key_bytes 4) or uint64 (key_bytes 8), values uint32. Scratch comes
 * from the context (grown on demand). n < 2^31. */
NGS_API ngs_status ngs_sort_pairs(ngs_ctx *ctx, void *d_keys, uint32_t *d_vals, int64_t n,
                                  int32_t key_bytes, int32_t begin_bit, int32_t end_bit,
                                  void *stream);

/* Exclusive prefix sum of n uint32 values (decoupled look-back, one pass):
 * d_out[i] = sum of d_in[0..i); d_total (device uint32, may be NULL) gets the
 * sum of all n. d_in and d_out may alias. n < 2^31. */
NGS_API ngs_status ngs_scan_u32(ngs_ctx *ctx, const uint32_t *d_in, uint32_t *d_out, int64_t n,
                                uint32_t *d_total, void *stream);

/* ------------------------------------------------------------------------
 * Serving loop: continuous batching of render requests from many agents
 * against the scene resident in `ctx` (the simulator's agents render views as
 * they walk, Sec. IV-B). A worker thread owns `lanes` render lanes (a stream
 * and work buffers each; the scene is shared, not copied). A free lane admits
 * the oldest waiting requests while they fit its camera limit and its
 * sort-buffer budget (estimated pairs = pixels x pairs_per_pixel, at least one
 * request per launch) and renders them as one batch; requests arriving
 * meanwhile join the next launch, and launches of different lanes overlap on
 * the device. Each request's image is the same bits as when rendered alone.
 * A launch whose (tile, Gaussian) pairs overflow its lane's buffer does not
 * fail its requests: the lane re-plans from the pairs the device counted,
 * admission raises its estimate to the lane's, and the requests return to the
 * front of the queue (a request is failed after 3 such launches).
 * The scene must not be reloaded while a server runs.
 * ------------------------------------------------------------------------ */
typedef struct ngs_server ngs_server;

typedef struct {
    int32_t lanes;                  /* concurrent render lanes (default 2, max 8) */
    int32_t max_cams;               /* cameras per launch (default 64, max 1024) */
    int64_t pair_budget;            /* admission budget per launch, pairs (default 2^29) */
    double pairs_per_pixel;         /* admission estimate (default 48) */
    int64_t lane_record_capacity;   /* per-lane work buffers (0: the context's) */
    int64_t lane_pair_capacity;
} ngs_server_config;

typedef struct {
    int64_t submitted, completed, failed, launches;
    double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> completion latency */
    double mpix;                              /* megapixels of completed requests */
    double span_s;                            /* first submit -> last completion */
    int64_t requeued;                         /* requests put back after a launch overflowed */
} ngs_serving_stats;

/* Starts the worker thread on the calling thread's current device. */
NGS_API ngs_status ngs_server_start(ngs_ctx *ctx, const ngs_server_config *cfg,
                                    ngs_server **out);
/* Queues one request (thread-safe, non-blocking): camera *cam rendered into
 * d_image (device float32 [3][H][W], caller-owned, untouched until the
 * request completes). *ticket identifies it for ngs_server_poll. */
NGS_API ngs_status ngs_server_submit(ngs_server *s, const ngs_camera *cam, float *d_image,
                                     uint64_t *ticket);
/* *done = 1 once the request's image is complete; *latency_ms its latency. */
NGS_API ngs_status ngs_server_poll(ngs_server *s, uint64_t ticket, int32_t *done,
                                   double *latency_ms);
/* Waits until every submitted request completed (NGS_ERR_DEVICE_TIMEOUT after
 * timeout_ms). */
NGS_API ngs_status ngs_server_wait_all(ngs_server *s, int32_t timeout_ms);
NGS_API ngs_status ngs_server_stats(ngs_server *s, ngs_serving_stats *out);
/* Drains the queue, joins the worker and frees the lanes. */
NGS_API ngs_status ngs_server_stop(ngs_server *s);

/* Allocation-free form of ngs_sort_pairs, for callers that cannot allocate
 * device memory where they sort (a host application whose own pool owns all
 * device memory, loops where cudaMalloc/cudaFree would synchronise the device,
 * or code without a renderer context). The paper has no counterpart; it is a
 * service of this library. Same sort, same arguments and results as
 * ngs_sort_pairs, but its scratch is one fixed device array inside the
 * library (about 6.3 MB, held by every GPU that loads the library until the
 * process exits), so it needs no context and calls no allocator.
 *  - n <= 524288 (2^19) pairs; larger n returns NGS_ERR_CAPACITY.
 *  - The first call on each device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - Every call shares the array: calls whose work overlaps on the GPU
 *    (different streams, unordered threads) race and give undefined results.
 *  - Asynchronous on `stream`. A device-side wait that gives up (its kernels
 *    still finish, the result is then undefined) is latched in the array and
 *    reported by ngs_sort_pairs_static_status(); it does not stop later calls. */
NGS_API ngs_status ngs_sort_pairs_static(void *d_keys, uint32_t *d_vals, int64_t n,
                                         int32_t key_bytes, int32_t begin_bit, int32_t end_bit,
                                         void *stream);

/* Status of the allocation-free sort on the calling thread's current device:
 * synchronises `stream`, then returns (and clears) the first device-side
 * error latched by an ngs_sort_pairs_static call on this device since the
 * previous query (NGS_OK if none, or if no call has run on the device).
 * Allocates nothing. Query on the stream the sorts ran on, or after they
 * completed. */
NGS_API ngs_status ngs_sort_pairs_static_status(void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NGS_H */
