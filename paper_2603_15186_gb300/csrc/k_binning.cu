// K3/K4/K6: tile binning by duplicated keys.
//
// The (tile, depth) ordering of the pairs is produced in two stable stages
// that together equal one stable sort on the 64-bit key (tile << 32 | depth):
//   1. the visible Gaussians (records, in camera-major, node-id order) are
//      radix-sorted by their 32-bit depth key;
//   2. K3 scans, in that depth order, the number of tiles each one touches
//      (decoupled look-back, one pass) and K4 writes one (tile, record) pair per
//      touched tile at those offsets, so the pair array is ordered by
//      (depth, node id, tile);
//   3. the pairs are radix-sorted stably by tile id (16 bits for a sub-batch of
//      at most 65536 tiles), which leaves each tile's list in (depth, node id)
//      order;
//   4. K6 finds each tile's [first, end) in the sorted pair array.
// The radix passes on the depth digits thus run over Gaussians, not over
// pairs, which is where the bytes are saved.
#include "ngs_internal.cuh"

namespace ngs {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanPart = kScanThreads * kScanItems;

int scan_partition() { return kScanPart; }

// K4 works on chunks of kDupChunk consecutive pairs
constexpr int kDupThreads = 256;
constexpr int kDupChunk = 2048;
constexpr int kDupWindow = 512;       // records staged at a time
int64_t dup_chunks(int64_t pair_cap) { return pair_cap / kDupChunk + 1; }

__device__ __forceinline__ uint32_t rect_area(const uint2 r) {
    const RectU u = unpack_rect(r);
    return (u.x1 - u.x0 + 1u) * (u.y1 - u.y0 + 1u);
}

// Block-wide exclusive scan of kScanItems values per thread (blocked layout:
// thread t holds items t*kScanItems .. +kScanItems-1); returns the block total.
__device__ __forceinline__ uint32_t block_scan(uint32_t v[kScanItems], uint32_t *s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint32_t t = v[i];
        v[i] = sum;
        sum += t;
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        if (w < warp) wbase += s_warp[w];
        total += s_warp[w];
    }
    const uint32_t off = wbase + incl - sum;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) v[i] += off;
    return total;
}

// Exclusive scan with one-pass decoupled look-back. Input element i is
// in[i] (kGather = false) or area(rect[idx[i]]) (kGather = true).
// With kGather, also chunk_first[c] = the input position whose output range
// [out[i], out[i] + in_i) holds element c * kDupChunk (c < chunk_cap), and
// rect_out[i] = rect[idx[i]]: the one gather of the rects in depth order, so
// that the pair emission reads them sequentially.
// Global memory is read and written warp-striped (consecutive lanes,
// consecutive elements: whole sectors per instruction); the scan itself runs
// on kScanItems consecutive elements per thread, exchanged through a shared
// array padded by one word per 32 (conflict-free both ways).
__device__ __forceinline__ int scan_slot(int k) { return k + (k >> 5); }

// Digit counts of the radix passes over the consecutive tile keys
// [k0, k0 + w) (one row of a Gaussian's tile rectangle). Pass 0 (the low 8
// bits): w >> 8 to every digit (full) and one to each digit of the cyclic run
// of w & 255 digits from k0 & 255, added as +1/-1 at its ends (d0, a
// difference array read back by a prefix sum); passes 1, 2: a count per
// digit value the run crosses (hh).
struct TileDigits {
    uint32_t d0[257];
    uint32_t full;
    uint32_t hh[2][256];
};
__device__ __forceinline__ void tile_digits_add(TileDigits &H, uint32_t k0, uint32_t w,
                                                int passes) {
    const uint32_t full = w >> 8, r = w & 255u, d = k0 & 255u;
    if (full) atomicAdd(&H.full, full);
    if (r) {
        atomicAdd(&H.d0[d], 1u);
        if (d + r <= 256u) {
            atomicAdd(&H.d0[d + r], 0xffffffffu);
        } else {
            atomicAdd(&H.d0[0], 1u);
            atomicAdd(&H.d0[d + r - 256u], 0xffffffffu);
        }
    }
    // tile keys stay below 2^24 (a sub-batch's tiles), so k0 + w fits 32 bits
    for (int q = 1; q < passes; ++q) {
        const int sh = 8 * q;
        const uint32_t e = k0 + w;
        for (uint32_t v = k0 >> sh; (v << sh) < e; ++v) {
            const uint32_t lo = max(v << sh, k0), hi = min((v + 1) << sh, e);
            atomicAdd(&H.hh[q - 1][v & 255u], hi - lo);
        }
    }
}

template <bool kGather>
__global__ void __launch_bounds__(kScanThreads, 4)
k_scan(const uint32_t *__restrict__ in, const uint2 *__restrict__ rect,
       const uint32_t *__restrict__ idx, uint32_t *out, const uint32_t *n_dev, int64_t n_host,
       uint32_t *total_out, int64_t total_cap, uint32_t *ticket, uint64_t *status,
       const uint32_t *epoch_ptr, uint32_t epoch_off, int *err, uint32_t *chunk_first,
       int64_t chunk_cap, uint2 *__restrict__ rect_out, const DevCamera *__restrict__ cams,
       uint32_t *hist, int passes) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    __shared__ uint32_t s_val[kScanPart + kScanPart / 32];
    __shared__ uint32_t s_part, s_prev;
    __shared__ TileDigits s_td;
    if (*err) return;
    const int tid = threadIdx.x;
    if (kGather && hist) {
        for (int i = tid; i < (int)(sizeof(TileDigits) / 4); i += kScanThreads)
            reinterpret_cast<uint32_t *>(&s_td)[i] = 0;
        __syncthreads();
    }
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int64_t nparts = (n + kScanPart - 1) / kScanPart;
    const uint32_t epoch = *epoch_ptr + epoch_off;
    if (nparts == 0 && blockIdx.x == 0 && tid == 0 && total_out) *total_out = 0;
    for (;;) {
        if (tid == 0) s_part = atomicAdd(ticket, 1u);
        __syncthreads();
        const int64_t part = s_part;
        if (part >= nparts) break;
        const int64_t pbase = part * kScanPart;
        // striped: element pbase + i * threads + tid
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int k = i * kScanThreads + tid;
            const int64_t j = pbase + k;
            uint32_t v = 0;
            if (j < n) {
                if (kGather) {
                    const uint2 rr = rect[idx[j]];
                    v = rect_area(rr);
                    rect_out[j] = rr;
                } else {
                    v = in[j];
                }
            }
            s_val[scan_slot(k)] = v;
        }
        __syncthreads();
        // blocked: elements pbase + tid * kScanItems + i
        uint32_t v[kScanItems], a[kScanItems];
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            v[i] = s_val[scan_slot(tid * kScanItems + i)];
            a[i] = v[i];
        }
        const uint32_t total = block_scan(v, s_warp);
        if (tid == 0) {
            uint64_t *slot = status + part;
            uint32_t prev = 0;
            if (part == 0) {
                publish(slot, pack_status(kFlagPrefix, epoch, total));
            } else {
                publish(slot, pack_status(kFlagAgg, epoch, total));
                look_back(status, part, 1, epoch, &prev, err);
                publish(slot, pack_status(kFlagPrefix, epoch, prev + total));
            }
            s_prev = prev;
            // a running total that crosses 2^32 wraps in the partition where it happens
            if (total_cap >= 0 && prev + total < prev) latch_error(err, kErrCapacity);
            if (part == nparts - 1) {
                const uint64_t all = (uint64_t)prev + total;
                if (total_out) *total_out = (uint32_t)all;
                if (total_cap >= 0 && (int64_t)all > total_cap) latch_error(err, kErrCapacity);
            }
        }
        if (kGather && hist && tid >= 32) {
            // while warp 0 looks back, the other warps count the tile digits
            // of the partition's Gaussians (each its tile keys, rectangle row
            // by row), reading back the depth-ordered rects just written
#pragma unroll 1
            for (int k = tid - 32; k < kScanPart && pbase + k < n; k += kScanThreads - 32) {
                const RectU u = unpack_rect(rect_out[pbase + k]);
                const uint32_t tb = cams[u.cam].tile_base;
                const uint32_t tsx = (uint32_t)cams[u.cam].tiles_x;
                for (uint32_t ty = u.y0; ty <= u.y1; ++ty)
                    tile_digits_add(s_td, tb + ty * tsx + u.x0, u.x1 - u.x0 + 1u, passes);
            }
        }
        __syncthreads();
        const uint32_t prev = s_prev;
        const int64_t base = pbase + (int64_t)tid * kScanItems;
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const uint32_t lo = prev + v[i];
            s_val[scan_slot(tid * kScanItems + i)] = lo;
            const int64_t j = base + i;
            if (kGather && a[i] && j < n) {
                const uint64_t hi = (uint64_t)lo + a[i];
                for (uint64_t c = ((uint64_t)lo + kDupChunk - 1) / kDupChunk;
                     c * kDupChunk < hi && (int64_t)c < chunk_cap; ++c)
                    chunk_first[c] = (uint32_t)j;
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kScanItems; ++i) {
            const int k = i * kScanThreads + tid;
            if (pbase + k < n) out[pbase + k] = s_val[scan_slot(k)];
        }
        __syncthreads();
    }
    if (kGather && hist) {
        // the CTA's digit counts into hist: pass 0 from the prefix sum of its
        // difference array (one digit per thread), passes 1, 2 directly
        static_assert(kScanThreads == 256, "one thread per digit");
        const int lane = tid & 31, warp = tid >> 5;
        __syncthreads();
        uint32_t x = s_td.d0[tid];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += t;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        for (int w = 0; w < warp; ++w) x += s_warp[w];
        const uint32_t c0 = x + s_td.full;
        if (c0) atomicAdd(&hist[tid], c0);
        for (int q = 1; q < passes; ++q) {
            const uint32_t v = s_td.hh[q - 1][tid];
            if (v) atomicAdd(&hist[q * 256 + tid], v);
        }
    }
}

void launch_scan_u32(const uint32_t *in, uint32_t *out, const uint32_t *n_dev, int64_t n_host,
                     uint32_t *total, uint32_t *ticket, uint64_t *status, const uint32_t *epoch,
                     uint32_t epoch_off, int *err, int grid, cudaStream_t st) {
    k_scan<false><<<grid, kScanThreads, 0, st>>>(in, nullptr, nullptr, out, n_dev, n_host, total,
                                                 -1, ticket, status, epoch, epoch_off, err,
                                                 nullptr, 0, nullptr, nullptr, nullptr, 0);
}

void launch_pair_offsets(const uint2 *rect, const uint32_t *sorted_idx, const uint32_t *n_vis,
                         uint32_t *poff, uint32_t *counters, int64_t pair_cap, uint32_t *ticket,
                         uint64_t *status, const uint32_t *epoch, uint32_t epoch_off, int *err,
                         uint32_t *chunk_first, uint2 *rect_sorted, const DevCamera *cams,
                         uint32_t *hist, int passes, int grid, cudaStream_t st) {
    k_scan<true><<<grid, kScanThreads, 0, st>>>(nullptr, rect, sorted_idx, poff, n_vis, -1,
                                                counters + CNT_PAIRS, pair_cap, ticket, status,
                                                epoch, epoch_off, err, chunk_first,
                                                dup_chunks(pair_cap), rect_sorted, cams,
                                                passes > 0 ? hist : nullptr, passes);
}

// K4: the pair array is cut into chunks of kDupChunk pairs, so every CTA
// iteration writes the same number of pairs however many tiles a Gaussian
// covers. A chunk starts at the record chunk_first[c] (from K3); its records
// are staged kDupWindow at a time (first pair, first tile key, tile-row
// stride and rectangle width with its reciprocal; record index from the
// depth order K3 scanned). Each pair finds
// its record through a map of the window's pairs: every record marks its first
// pair with its window index and a block-wide running maximum fills the rest
// (record starts increase with the index). The tile-digit histograms of the
// radix passes that follow are counted by K3, per rectangle row.
__global__ void __launch_bounds__(kDupThreads)
k_duplicate(const uint2 *__restrict__ rect_sorted, const uint32_t *__restrict__ sorted_idx,
            const uint32_t *__restrict__ poff, const uint32_t *__restrict__ chunk_first,
            const uint32_t *n_vis_p, const uint32_t *n_pairs_p, int64_t pair_cap,
            const DevCamera *__restrict__ cams, uint32_t *__restrict__ pkey,
            uint32_t *__restrict__ pval, int *err) {
    constexpr int kPer = kDupChunk / kDupThreads;   // map entries per thread
    __shared__ uint32_t s_off[kDupWindow + 1];
    __shared__ uint4 s_rec[kDupWindow];    // (first tile key, tiles_x, width, 1 / width)
    __shared__ uint32_t s_idx[kDupWindow];
    __shared__ uint16_t s_map[kDupChunk];  // window index of each pair's record
    __shared__ uint32_t s_warp[kDupThreads / 32];
    static_assert(kDupWindow <= 65536 && kDupChunk % kDupThreads == 0, "map layout");
    if (*err) return;
    const uint32_t n_vis = *n_vis_p, n_pairs = *n_pairs_p;
    if ((int64_t)n_pairs > pair_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) latch_error(err, kErrCapacity);
        return;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n_chunks = ((int64_t)n_pairs + kDupChunk - 1) / kDupChunk;
    for (int64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint32_t p0 = (uint32_t)(ch * kDupChunk);
        const uint32_t p1 = (uint32_t)min((int64_t)n_pairs, ch * kDupChunk + kDupChunk);
        int64_t r0 = chunk_first[ch];
        uint32_t q = p0;   // first pair of the chunk not yet written
        while (q < p1) {
            const int64_t rem = (int64_t)n_vis - r0;
            const int cnt = rem < kDupWindow ? (int)rem : kDupWindow;
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kPer; ++i) s_map[tid * kPer + i] = 0;
            for (int j = tid; j < cnt; j += kDupThreads) {
                const RectU u = unpack_rect(rect_sorted[r0 + j]);
                const uint32_t w = u.x1 - u.x0 + 1u;
                const uint32_t tb = cams[u.cam].tile_base, tsx = (uint32_t)cams[u.cam].tiles_x;
                s_rec[j] = make_uint4(tb + u.y0 * tsx + u.x0, tsx, w,
                                      __float_as_uint(1.0f / (float)w));
                s_idx[j] = sorted_idx[r0 + j];
                s_off[j] = poff[r0 + j];
            }
            if (tid == 0) s_off[cnt] = (r0 + cnt < (int64_t)n_vis) ? poff[r0 + cnt] : n_pairs;
            __syncthreads();
            const uint32_t q1 = min(p1, s_off[cnt]);
            // mark each record's first pair in [q, q1) (record 0 may start before q)
            for (int j = tid + 1; j < cnt; j += kDupThreads) {
                const uint32_t st = s_off[j];
                if (st < q1) s_map[st - q] = (uint16_t)j;
            }
            __syncthreads();
            {
                // running maximum over the map, kPer consecutive entries per thread
                uint32_t m[kPer], run = 0;
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    run = max(run, (uint32_t)s_map[tid * kPer + i]);
                    m[i] = run;
                }
                uint32_t incl = run;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl = max(incl, t);
                }
                if (lane == 31) s_warp[warp] = incl;
                uint32_t before = __shfl_up_sync(0xffffffffu, incl, 1);
                if (lane == 0) before = 0;
                __syncthreads();
#pragma unroll
                for (int w = 0; w < kDupThreads / 32; ++w)
                    if (w < warp) before = max(before, s_warp[w]);
#pragma unroll
                for (int i = 0; i < kPer; ++i) s_map[tid * kPer + i] = (uint16_t)max(before, m[i]);
            }
            __syncthreads();
            for (uint32_t p = q + tid; p < q1; p += kDupThreads) {
                const int j = s_map[p - q];
                const uint4 r = s_rec[j];
                // tile (tx, ty) = k mod / div width: a float quotient, then one
                // integer correction (its error is below 1 for k < 2^24)
                const uint32_t k = p - s_off[j];
                int ty = (int)((float)k * __uint_as_float(r.w));
                int tx = (int)k - ty * (int)r.z;
                if (tx < 0) { --ty; tx += (int)r.z; }
                else if (tx >= (int)r.z) { ++ty; tx -= (int)r.z; }
                pkey[p] = r.x + (uint32_t)ty * r.y + (uint32_t)tx;
                pval[p] = s_idx[j];
            }
            q = q1;
            r0 += cnt;
            if (cnt == 0) break;
        }
    }
}

void launch_duplicate(const uint2 *rect_sorted, const uint32_t *sorted_idx, const uint32_t *poff,
                      const uint32_t *chunk_first, const uint32_t *n_vis, const uint32_t *n_pairs,
                      int64_t pair_cap, const DevCamera *cams, uint32_t *pkey, uint32_t *pval,
                      int *err, int grid, cudaStream_t st) {
    k_duplicate<<<grid, kDupThreads, 0, st>>>(rect_sorted, sorted_idx, poff, chunk_first, n_vis,
                                              n_pairs, pair_cap, cams, pkey, pval, err);
}

// K6: ranges[t] = [first, end) of tile t in the sorted pair keys, stored as
// (~first, end) so that a zeroed entry reads as an empty range (first =
// 0xffffffff > end = 0) for tiles without pairs. The last pass of the tile
// sort writes the same encoding while it scatters (k_onesweep, kOut = 2); this
// kernel covers sub-batches of a single tile, which need no tile sort.
__global__ void k_ranges(const uint32_t *__restrict__ pkey, const uint32_t *n_pairs_p,
                         uint2 *__restrict__ ranges, const int *err) {
    if (*err) return;
    const int64_t n = *n_pairs_p;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = pkey[i];
        if (i == 0 || pkey[i - 1] != k) ranges[k].x = ~(uint32_t)i;
        if (i == n - 1 || pkey[i + 1] != k) ranges[k].y = (uint32_t)(i + 1);
    }
}

void launch_ranges(const uint32_t *pkey, const uint32_t *n_pairs, uint2 *ranges, int grid,
                   cudaStream_t st, const int *err) {
    k_ranges<<<grid, 256, 0, st>>>(pkey, n_pairs, ranges, err);
}

}  // namespace ngs
