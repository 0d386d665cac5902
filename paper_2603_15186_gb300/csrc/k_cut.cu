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
// One pass, order preserving: partitions are (camera, block of 2048 nodes) in
// camera-major order, taken from an atomic ticket so every predecessor of a
// partition is already running; each partition counts its selected nodes,
// finds its output offset by decoupled look-back and writes the ids in
// ascending order. HBM traffic per node and camera: the node's two box words
// (32 B) plus its parent's (mostly L1/L2 hits: siblings share a parent), and
// 4 B per selected node.
#include "ngs_internal.cuh"

namespace ngs {

constexpr int kCutThreads = 256;
constexpr int kCutItems = 8;
constexpr int kCutPart = kCutThreads * kCutItems;

int cut_partition_nodes() { return kCutPart; }

__global__ void __launch_bounds__(kCutThreads)
k_cut(const float4 *__restrict__ box_lo, const float4 *__restrict__ box_hi, int64_t n_nodes,
      const DevCamera *__restrict__ cams, int n_cams, uint32_t *__restrict__ ids, int64_t cap,
      uint32_t *__restrict__ offsets, uint32_t *__restrict__ counters, uint32_t *ticket,
      uint64_t *status, const uint32_t *epoch_ptr, uint32_t epoch_off, int *err) {
    __shared__ uint32_t s_part;
    __shared__ uint32_t s_cnt[kCutItems * 8];   // per (item row, warp), then exclusive
    __shared__ uint32_t s_excl;
    if (*err) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nblk = (n_nodes + kCutPart - 1) / kCutPart;
    const int64_t nparts = nblk * n_cams;
    const uint32_t epoch = *epoch_ptr + epoch_off;
    for (;;) {
        if (tid == 0) s_part = atomicAdd(ticket, 1u);
        __syncthreads();
        const int64_t part = s_part;
        if (part >= nparts) break;
        const int c = (int)(part / nblk);
        const int64_t b = part - (int64_t)c * nblk;
        const float px = cams[c].pos[0], py = cams[c].pos[1], pz = cams[c].pos[2];
        const float fx = cams[c].fx, tau = cams[c].tau;
        uint32_t bal[kCutItems];
#pragma unroll
        for (int k = 0; k < kCutItems; ++k) {
            const int64_t node = b * kCutPart + k * kCutThreads + tid;
            const bool sel =
                node < n_nodes && cut_selects(box_lo, box_hi, node, px, py, pz, fx, tau);
            bal[k] = __ballot_sync(0xffffffffu, sel);
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
                    offsets[n_cams] = prev + total;
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

void launch_cut(const SceneDev &sc, const DevCamera *cams, int n_cams, uint32_t *ids, int64_t cap,
                uint32_t *offsets, uint32_t *counters, uint32_t *ticket, uint64_t *status,
                const uint32_t *epoch, uint32_t epoch_off, int *err, int grid, cudaStream_t st) {
    k_cut<<<grid, kCutThreads, 0, st>>>(sc.box_lo, sc.box_hi, sc.n, cams, n_cams, ids, cap,
                                        offsets, counters, ticket, status, epoch, epoch_off, err);
}

}  // namespace ngs
