// K1: level-of-detail cut of the Gaussian hierarchy (NavGSim Sec. III-B:
// per view, Gaussians are taken from the level of the tree whose granularity
// matches the requested one).
//
// Node n is selected for camera c iff
//     (n is a leaf or s_c(n) <= tau_c) and (n is the root or s_c(parent(n)) > tau_c)
// with s_c(n) = fx * (longest side of box(n)) / (distance from the camera
// centre to box(n)), s = +inf when the centre lies inside the box. Boxes nest,
// so s never decreases towards the root and every root-to-leaf path holds
// exactly one selected node.
//
// Variants (Sec. III-B's per-view, dynamic selection of levels): a frustum
// cull drops the nodes whose box lies wholly outside one of the five planes of
// a camera's view volume (near plane 0.2, image rectangle widened by a guard
// band), and a group of cameras can share one cut, in which a node is fine
// enough when it is for every member that does not cull it. Boxes nest and the
// float32 tests below are monotone in the box bounds (each step rounds
// monotonically), so both the cull and "fine enough" spread from a node to its
// whole subtree and the result stays an antichain of the tree.
//
// One pass, order preserving: partitions are (camera or group, block of 2048
// nodes) in camera-major order, taken from an atomic ticket so every
// predecessor of a partition is already running; each partition counts its
// selected nodes, finds its output offset by decoupled look-back and writes
// the ids in ascending order. HBM traffic per node and camera: the node's two box words
// (32 B) plus its parent's (mostly L1/L2 hits: siblings share a parent), and
// 4 B per selected node.
#include "ngs_internal.cuh"
#include "cut.h"

namespace ngs {

constexpr int kCutThreads = 256;
constexpr int kCutItems = 8;
constexpr int kCutPart = kCutThreads * kCutItems;

int cut_partition_nodes() { return kCutPart; }

// Selection of the plain cut: one camera per unit.
struct PlainSelect {
    const float4 *box_lo, *box_hi;
    const DevCamera *cams;
    float px, py, pz, fx, tau;
    __device__ __forceinline__ void begin(int c) {
        px = cams[c].pos[0]; py = cams[c].pos[1]; pz = cams[c].pos[2];
        fx = cams[c].fx; tau = cams[c].tau;
    }
    __device__ __forceinline__ bool operator()(int64_t node) const {
        return cut_selects(box_lo, box_hi, node, px, py, pz, fx, tau);
    }
};

// True when the box lies wholly outside one of the camera's five half-spaces:
// the largest value of a_k . (x - pos) + b_k over the box (per axis the larger
// of the two faces' terms) is negative.
__device__ __forceinline__ bool frustum_culled(const CutCam &k, const float4 lo, const float4 hi) {
    const float dl0 = __fsub_rn(lo.x, k.pos[0]), dh0 = __fsub_rn(hi.x, k.pos[0]);
    const float dl1 = __fsub_rn(lo.y, k.pos[1]), dh1 = __fsub_rn(hi.y, k.pos[1]);
    const float dl2 = __fsub_rn(lo.z, k.pos[2]), dh2 = __fsub_rn(hi.z, k.pos[2]);
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const float t0 = fmaxf(__fmul_rn(k.a[j][0], dl0), __fmul_rn(k.a[j][0], dh0));
        const float t1 = fmaxf(__fmul_rn(k.a[j][1], dl1), __fmul_rn(k.a[j][1], dh1));
        const float t2 = fmaxf(__fmul_rn(k.a[j][2], dl2), __fmul_rn(k.a[j][2], dh2));
        const float m = __fadd_rn(__fadd_rn(__fadd_rn(t0, t1), t2), j == 0 ? k.b0 : 0.0f);
        if (m < 0.0f) return true;
    }
    return false;
}

// Selection of a shared cut: one group of cameras per unit. n is fine enough
// for the group when every member culls it (kFrustum) or has s(n) <= tau; n is
// selected iff (leaf or fine(n)) and (root or not fine(parent)) and, with
// kFrustum, some member keeps it.
template <bool kFrustum>
struct SharedSelect {
    const float4 *box_lo, *box_hi;
    const CutCam *cams;
    const int32_t *group_begin;
    int c0, c1;
    __device__ __forceinline__ void begin(int g) {
        c0 = group_begin[g];
        c1 = group_begin[g + 1];
    }
    __device__ __forceinline__ bool operator()(int64_t node) const {
        const float4 lo = box_lo[node], hi = box_hi[node];
        const int parent = __float_as_int(lo.w);
        const bool leaf = __float_as_int(hi.w) == 0;
        float4 plo = lo, phi = hi;
        if (parent >= 0) {
            plo = box_lo[parent];
            phi = box_hi[parent];
        }
        bool fine_p = true, seen = !kFrustum;
        for (int c = c0; c < c1; ++c) {
            const CutCam &k = cams[c];
            bool vis_n = true, vis_p = true;
            if (kFrustum) {
                vis_n = !frustum_culled(k, lo, hi);
                // a culled parent culls the node, so a kept node's parent is kept
                vis_p = vis_n || (parent >= 0 && !frustum_culled(k, plo, phi));
                seen = seen || vis_n;
            }
            // neither a leaf nor fine enough for this member: not selected
            if (!leaf && vis_n &&
                !fine_enough(lo, hi, k.pos[0], k.pos[1], k.pos[2], k.fx, k.tau))
                return false;
            if (parent >= 0 && fine_p && vis_p &&
                !fine_enough(plo, phi, k.pos[0], k.pos[1], k.pos[2], k.fx, k.tau))
                fine_p = false;
        }
        return (parent < 0 || !fine_p) && seen;
    }
};

// Persistent loop over (unit, node block) partitions: count the selected
// nodes of the block, find the output offset by decoupled look-back, write
// the ids in ascending order.
template <class Select>
__device__ __forceinline__ void cut_partitions(Select sel, int64_t n_nodes, int n_units,
                                               uint32_t *__restrict__ ids, int64_t cap,
                                               uint32_t *__restrict__ offsets,
                                               uint32_t *__restrict__ counters, uint32_t *ticket,
                                               uint64_t *status, const uint32_t *epoch_ptr,
                                               uint32_t epoch_off, int *err) {
    __shared__ uint32_t s_part;
    __shared__ uint32_t s_cnt[kCutItems * 8];   // per (item row, warp), then exclusive
    __shared__ uint32_t s_excl;
    if (*err) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nblk = (n_nodes + kCutPart - 1) / kCutPart;
    const int64_t nparts = nblk * n_units;
    const uint32_t epoch = *epoch_ptr + epoch_off;
    for (;;) {
        if (tid == 0) s_part = atomicAdd(ticket, 1u);
        __syncthreads();
        const int64_t part = s_part;
        if (part >= nparts) break;
        const int c = (int)(part / nblk);
        const int64_t b = part - (int64_t)c * nblk;
        sel.begin(c);
        uint32_t bal[kCutItems];
#pragma unroll
        for (int k = 0; k < kCutItems; ++k) {
            const int64_t node = b * kCutPart + k * kCutThreads + tid;
            const bool on = node < n_nodes && sel(node);
            bal[k] = __ballot_sync(0xffffffffu, on);
            if (lane == 0) s_cnt[k * 8 + warp] = __popc(bal[k]);
        }
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the 64 (row, warp) counts in node order
            const uint32_t v0 = s_cnt[2 * lane], v1 = s_cnt[2 * lane + 1];
            uint32_t incl = v0 + v1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t excl = incl - (v0 + v1);
            s_cnt[2 * lane] = excl;
            s_cnt[2 * lane + 1] = excl + v0;
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (lane == 0) {
                uint64_t *slot = status + part;
                uint32_t prev = 0;
                if (part == 0) {
                    publish(slot, pack_status(kFlagPrefix, epoch, total));
                } else {
                    publish(slot, pack_status(kFlagAgg, epoch, total));
                    look_back(status, part, 1, epoch, &prev, err);
                    publish(slot, pack_status(kFlagPrefix, epoch, prev + total));
                }
                s_excl = prev;
                if (b == 0) offsets[c] = prev;
                if (part == nparts - 1) {
                    offsets[n_units] = prev + total;
                    counters[CNT_CUT] = prev + total;
                    if ((int64_t)prev + total > cap) latch_error(err, kErrCapacity);
                }
            }
        }
        __syncthreads();
        const uint32_t base = s_excl;
#pragma unroll
        for (int k = 0; k < kCutItems; ++k) {
            if ((bal[k] >> lane) & 1u) {
                const uint32_t pos = base + s_cnt[k * 8 + warp] + __popc(bal[k] & lanemask_lt());
                if (pos < cap) ids[pos] = (uint32_t)(b * kCutPart + k * kCutThreads + tid);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kCutThreads)
k_cut(const float4 *__restrict__ box_lo, const float4 *__restrict__ box_hi, int64_t n_nodes,
      const DevCamera *__restrict__ cams, int n_cams, uint32_t *__restrict__ ids, int64_t cap,
      uint32_t *__restrict__ offsets, uint32_t *__restrict__ counters, uint32_t *ticket,
      uint64_t *status, const uint32_t *epoch_ptr, uint32_t epoch_off, int *err) {
    PlainSelect sel{box_lo, box_hi, cams, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    cut_partitions(sel, n_nodes, n_cams, ids, cap, offsets, counters, ticket, status, epoch_ptr,
                   epoch_off, err);
}

template <bool kFrustum>
__global__ void __launch_bounds__(kCutThreads)
k_cut_shared(const float4 *__restrict__ box_lo, const float4 *__restrict__ box_hi,
             int64_t n_nodes, const CutCam *__restrict__ cams,
             const int32_t *__restrict__ group_begin, int n_groups, uint32_t *__restrict__ ids,
             int64_t cap, uint32_t *__restrict__ offsets, uint32_t *__restrict__ counters,
             uint32_t *ticket, uint64_t *status, const uint32_t *epoch_ptr, uint32_t epoch_off,
             int *err) {
    SharedSelect<kFrustum> sel{box_lo, box_hi, cams, group_begin, 0, 0};
    cut_partitions(sel, n_nodes, n_groups, ids, cap, offsets, counters, ticket, status,
                   epoch_ptr, epoch_off, err);
}

// Many-camera plain cut. A partition is (node block b, chunk of kCutCams
// cameras), taken in block-major order so that a block's boxes come from HBM
// once and from L2 for its other chunks; every camera of the chunk is tested
// on the node and parent boxes loaded once. Pass 1 stores each camera's count
// for the block; pass 2 (after a scan of the counts in camera-major order)
// recomputes the selection and writes the ids at the scanned offset plus the
// prefix within the block. No partition waits on another.
// With kFrustum (a frustum-culled cut per camera, i.e. shared cuts in groups of
// one) a node is also dropped when its box lies outside one of the camera's
// five planes: for a single camera that is its plain cut minus the culled
// nodes (a culled parent culls the node).
constexpr int kCutCams = 8;
static_assert(kCutThreads / 32 == kCutCams, "one warp scans one camera's row counts");

template <bool kWrite, bool kFrustum>
__global__ void __launch_bounds__(kCutThreads)
k_cut_blocked(const float4 *__restrict__ box_lo, const float4 *__restrict__ box_hi,
              int64_t n_nodes, const DevCamera *__restrict__ cams,
              const CutCam *__restrict__ ccams, int n_cams,
              uint32_t *__restrict__ part_vals, uint32_t *__restrict__ ids, int64_t cap,
              uint32_t *ticket, const int *err) {
    __shared__ float s_cam[kCutCams][5];                   // pos xyz, fx, tau^2 (rounded)
    __shared__ CutCam s_ccam[kFrustum ? kCutCams : 1];     // the cameras' planes
    __shared__ uint32_t s_bal[kCutCams][kCutItems * 8];    // ballot per (camera, row, warp)
    __shared__ uint32_t s_off[kCutCams][kCutItems * 8];    // its exclusive offset in the block
    __shared__ uint32_t s_part;
    if (*err) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nblk = (n_nodes + kCutPart - 1) / kCutPart;
    const int nchunk = (n_cams + kCutCams - 1) / kCutCams;
    const int64_t nparts = nblk * nchunk;
    for (;;) {
        if (tid == 0) s_part = atomicAdd(ticket, 1u);
        __syncthreads();
        const int64_t part = s_part;
        if (part >= nparts) break;
        const int64_t b = part / nchunk;
        const int c0 = (int)(part - b * nchunk) * kCutCams;
        const int nc = min(kCutCams, n_cams - c0);
        if (tid < kCutCams * 5) {
            const int j = tid / 5, f = tid - 5 * j;
            float v = 0.0f;
            if (j < nc) {
                if (kFrustum) {
                    const CutCam &k = ccams[c0 + j];
                    v = f < 3 ? k.pos[f] : (f == 3 ? k.fx : __fmul_rn(k.tau, k.tau));
                } else {
                    const DevCamera &k = cams[c0 + j];
                    v = f < 3 ? k.pos[f] : (f == 3 ? k.fx : __fmul_rn(k.tau, k.tau));
                }
            }
            s_cam[j][f] = v;
        }
        if (kFrustum && tid < kCutCams * (int)(sizeof(CutCam) / 4)) {
            const int j = tid / (int)(sizeof(CutCam) / 4), f = tid - j * (int)(sizeof(CutCam) / 4);
            if (j < nc)
                reinterpret_cast<float *>(&s_ccam[j])[f] =
                    reinterpret_cast<const float *>(&ccams[c0 + j])[f];
        }
        __syncthreads();
#pragma unroll 1
        for (int k = 0; k < kCutItems; ++k) {
            const int64_t node = b * kCutPart + k * kCutThreads + tid;
            const bool valid = node < n_nodes;
            float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo, plo = lo, phi = lo;
            int parent = -1;
            bool leaf = true;
            if (valid) {
                lo = box_lo[node];
                hi = box_hi[node];
                parent = __float_as_int(lo.w);
                leaf = __float_as_int(hi.w) == 0;
                if (parent >= 0) {
                    plo = box_lo[parent];
                    phi = box_hi[parent];
                }
            }
            // kFrustum: the cameras whose view volume the union of the warp's
            // node boxes can meet (a box outside a half-space has every box it
            // contains outside too, also in float32: the tests are monotone in
            // the bounds); the others cull all 32 nodes without a test per node
            uint32_t live = (1u << nc) - 1u;
            if (kFrustum) {
                const float inf = __int_as_float(0x7f800000);
                float4 ulo = valid ? lo : make_float4(inf, inf, inf, 0.f);
                float4 uhi = valid ? hi : make_float4(-inf, -inf, -inf, 0.f);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ulo.x = fminf(ulo.x, __shfl_xor_sync(0xffffffffu, ulo.x, o));
                    ulo.y = fminf(ulo.y, __shfl_xor_sync(0xffffffffu, ulo.y, o));
                    ulo.z = fminf(ulo.z, __shfl_xor_sync(0xffffffffu, ulo.z, o));
                    uhi.x = fmaxf(uhi.x, __shfl_xor_sync(0xffffffffu, uhi.x, o));
                    uhi.y = fmaxf(uhi.y, __shfl_xor_sync(0xffffffffu, uhi.y, o));
                    uhi.z = fmaxf(uhi.z, __shfl_xor_sync(0xffffffffu, uhi.z, o));
                }
                uint32_t keep = 0;
                if (ulo.x <= uhi.x) {   // some valid node
#pragma unroll 1
                    for (int j = 0; j < nc; ++j)
                        if (!frustum_culled(s_ccam[j], ulo, uhi)) keep |= 1u << j;
                }
                live = keep;
            }
            const float ext_n = box_extent(lo, hi), ext_p = box_extent(plo, phi);
            uint32_t m = 0;   // bit j: camera j selects the node
#pragma unroll
            for (int j = 0; j < kCutCams; ++j) {
                if (valid && j < nc && ((live >> j) & 1u)) {
                    const float px = s_cam[j][0], py = s_cam[j][1], pz = s_cam[j][2];
                    const float fx = s_cam[j][3], tau2 = s_cam[j][4];
                    // the rule of cut_selects, parent first (most nodes lie below the cut)
                    if ((parent < 0 ||
                         !fine_enough_pre(plo, phi, ext_p, px, py, pz, fx, tau2)) &&
                        (leaf || fine_enough_pre(lo, hi, ext_n, px, py, pz, fx, tau2)))
                        m |= 1u << j;
                }
            }
            if (kFrustum) {
                // not unrolled: the planes stay in shared memory instead of
                // occupying registers for all cameras of the chunk at once
                uint32_t rest = m;
#pragma unroll 1
                while (rest) {
                    const int j = __ffs(rest) - 1;
                    rest &= rest - 1;
                    if (frustum_culled(s_ccam[j], lo, hi)) m &= ~(1u << j);
                }
            }
#pragma unroll
            for (int j = 0; j < kCutCams; ++j) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (m >> j) & 1u);
                if (lane == 0) s_bal[j][k * 8 + warp] = bal;
            }
        }
        __syncthreads();
        if (warp < nc) {
            // warp j: exclusive scan of camera j's 64 (row, warp) counts in node order
            const int j = warp;
            const uint32_t v0 = __popc(s_bal[j][2 * lane]), v1 = __popc(s_bal[j][2 * lane + 1]);
            uint32_t incl = v0 + v1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const uint32_t excl = incl - (v0 + v1);
            s_off[j][2 * lane] = excl;
            s_off[j][2 * lane + 1] = excl + v0;
            if (!kWrite && lane == 31) part_vals[(int64_t)(c0 + j) * nblk + b] = incl;
        }
        if (kWrite) {
            __syncthreads();
            for (int j = 0; j < nc; ++j) {
                const uint64_t base = part_vals[(int64_t)(c0 + j) * nblk + b];
#pragma unroll
                for (int k = 0; k < kCutItems; ++k) {
                    const uint32_t bal = s_bal[j][k * 8 + warp];
                    if ((bal >> lane) & 1u) {
                        const uint64_t pos =
                            base + s_off[j][k * 8 + warp] + __popc(bal & lanemask_lt());
                        if (pos < (uint64_t)cap)
                            ids[pos] = (uint32_t)(b * kCutPart + k * kCutThreads + tid);
                    }
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_cut_cam_offsets(const uint32_t *__restrict__ part_off,
                                  const uint32_t *__restrict__ total, int64_t nblk, int n_cams,
                                  int64_t cap, int64_t *__restrict__ offsets,
                                  uint32_t *__restrict__ counters, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n_cams) return;
    const uint32_t t = *total;
    offsets[i] = i < n_cams ? (int64_t)part_off[(int64_t)i * nblk] : (int64_t)t;
    if (i == n_cams) {
        counters[CNT_CUT] = t;
        if ((int64_t)t > cap) latch_error(err, kErrCapacity);
    }
}

void launch_cut_blocked(bool write, const float4 *box_lo, const float4 *box_hi, int64_t n_nodes,
                        const DevCamera *cams, const CutCam *ccams, int n_cams,
                        uint32_t *part_vals, uint32_t *ids, int64_t cap, uint32_t *ticket,
                        const int *err, int grid, cudaStream_t st) {
    if (ccams) {
        if (write)
            k_cut_blocked<true, true><<<grid, kCutThreads, 0, st>>>(
                box_lo, box_hi, n_nodes, cams, ccams, n_cams, part_vals, ids, cap, ticket, err);
        else
            k_cut_blocked<false, true><<<grid, kCutThreads, 0, st>>>(
                box_lo, box_hi, n_nodes, cams, ccams, n_cams, part_vals, ids, cap, ticket, err);
    } else if (write) {
        k_cut_blocked<true, false><<<grid, kCutThreads, 0, st>>>(
            box_lo, box_hi, n_nodes, cams, ccams, n_cams, part_vals, ids, cap, ticket, err);
    } else {
        k_cut_blocked<false, false><<<grid, kCutThreads, 0, st>>>(
            box_lo, box_hi, n_nodes, cams, ccams, n_cams, part_vals, ids, cap, ticket, err);
    }
}

void launch_cut_cam_offsets(const uint32_t *part_off, const uint32_t *total, int64_t nblk,
                            int n_cams, int64_t cap, int64_t *offsets, uint32_t *counters,
                            int *err, cudaStream_t st) {
    k_cut_cam_offsets<<<(n_cams + 256) / 256, 256, 0, st>>>(part_off, total, nblk, n_cams, cap,
                                                            offsets, counters, err);
}

void launch_cut(const SceneDev &sc, const DevCamera *cams, int n_cams, uint32_t *ids, int64_t cap,
                uint32_t *offsets, uint32_t *counters, uint32_t *ticket, uint64_t *status,
                const uint32_t *epoch, uint32_t epoch_off, int *err, int grid, cudaStream_t st) {
    k_cut<<<grid, kCutThreads, 0, st>>>(sc.box_lo, sc.box_hi, sc.n, cams, n_cams, ids, cap,
                                        offsets, counters, ticket, status, epoch, epoch_off, err);
}

void launch_cut_shared(bool frustum, const float4 *box_lo, const float4 *box_hi, int64_t n_nodes,
                       const CutCam *cams, const int32_t *group_begin, int n_groups,
                       uint32_t *ids, int64_t cap, uint32_t *offsets, uint32_t *counters,
                       uint32_t *ticket, uint64_t *status, const uint32_t *epoch,
                       uint32_t epoch_off, int *err, int grid, cudaStream_t st) {
    if (frustum)
        k_cut_shared<true><<<grid, kCutThreads, 0, st>>>(box_lo, box_hi, n_nodes, cams,
                                                         group_begin, n_groups, ids, cap, offsets,
                                                         counters, ticket, status, epoch,
                                                         epoch_off, err);
    else
        k_cut_shared<false><<<grid, kCutThreads, 0, st>>>(box_lo, box_hi, n_nodes, cams,
                                                          group_begin, n_groups, ids, cap,
                                                          offsets, counters, ticket, status,
                                                          epoch, epoch_off, err);
}

}  // namespace ngs
