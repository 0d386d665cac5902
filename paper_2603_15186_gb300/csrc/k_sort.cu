// K5: stable least-significant-digit radix sort of (key, value) pairs in the
// "onesweep" arrangement: one upsweep kernel builds the digit histograms of
// every pass from a single read of the keys, then each 8-bit digit pass is one
// kernel that ranks a 4096-key partition in shared memory and finds, for each
// of the 256 digits, the partition's global offset by decoupled look-back over
// the preceding partitions (no separate scan kernel per pass).
//
// Stability: keys are loaded warp-striped (item i of lane l is key
// base + 32 ITEMS w + 32 i + l), each warp ranks its items in that order (peers
// = lanes holding the same digit, from one shared-memory OR of lane bits per
// item), warps are offset in order, and partitions in ticket order; equal
// digits therefore keep their input order, which is what the two-stage binning
// needs.
//
// Forward progress: partition ids come from an atomic ticket, so every
// partition a look-back waits on is held by a CTA that is already running.
// Every wait is bounded (kSpinLimit) and latches kErrTimeout if it runs out.
//
// HBM per pass: read key + value, write key + value (16 B/pair for 32-bit
// keys, 24 B for 64-bit), plus the upsweep's one read of the keys.
// Partitions are 8192 keys (32-bit) or 4096 (64-bit) over 512 threads: long
// runs per digit keep the scattered writes close to whole sectors, and values
// are read only once the keys are ranked, which keeps two CTAs resident.
#include "ngs_internal.cuh"

namespace ngs {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;
constexpr int kSortPart = kSortThreads * kSortItems;   // 4096 keys
constexpr int kRadix = 256;
constexpr int kMaxPasses = 8;

int sort_partition() { return kSortPart; }   // smallest partition of any key width
int sort_passes(int begin_bit, int end_bit) { return (end_bit - begin_bit + 7) / 8; }

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift, uint32_t mask) {
    return (uint32_t)(key >> shift) & mask;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
k_upsweep(const K *__restrict__ keys, const uint32_t *n_dev, int64_t n_host, int begin_bit,
          int end_bit, uint32_t *__restrict__ hist, const int *err) {
    __shared__ uint32_t s_h[kMaxPasses][kRadix];
    if (*err) return;
    const int passes = (end_bit - begin_bit + 7) / 8;
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kSortThreads) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) {
            const int sh = begin_bit + 8 * p;
            const int bits = min(8, end_bit - sh);
            atomicAdd(&s_h[p][digit_of(k, sh, (1u << bits) - 1u)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) {
        const uint32_t v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

// hist[p][d] -> exclusive prefix over d (one block per pass)
__global__ void k_digit_scan(uint32_t *hist, const int *err) {
    __shared__ uint32_t s_w[kSortWarps];
    if (*err) return;
    uint32_t *h = hist + blockIdx.x * kRadix;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t v = h[tid];
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += s_w[w];
    h[tid] = wbase + incl - v;
}

// Partition shape per key width: 512 threads; 16 (32-bit keys) or 8 (64-bit
// keys) items per thread, i.e. 8192 or 4096 keys per partition.
template <typename K> struct SortShape;
template <> struct SortShape<uint32_t> { static constexpr int kItems = 16; };
template <> struct SortShape<uint64_t> { static constexpr int kItems = 8; };
constexpr int kOsThreads = 512;
constexpr int kOsWarps = kOsThreads / 32;

template <typename K>
struct SortSmem {
    static constexpr int kPart = kOsThreads * SortShape<K>::kItems;
    uint32_t whist[kOsWarps][kRadix];     // per-warp digit counts, then warp offsets
    uint32_t match[kOsWarps][kRadix];     // per-warp lane masks of one item's digits (kept 0)
    uint32_t gstart[kRadix];              // global output position of staged slot 0 of each digit's run
    uint32_t wtot[kRadix / 32];
    K keys[kPart];
    uint32_t vals[kPart];
    uint32_t part;
};

// kOut: 0 writes keys and values; 1 values only (last pass of a sort whose
// keys are not needed afterwards); 2 values only, plus the [first, end) range
// of every key in the sorted output (last pass of the tile sort, 32-bit keys):
// within a partition equal keys are adjacent in the staged order and land on
// consecutive output positions, so each run of equal keys contributes its
// first and end position with one atomicMax each (first stored as ~first), and
// the runs a key has in several partitions combine to its global range.
template <typename K, bool kIdentity, int kOut>
__global__ void __launch_bounds__(kOsThreads, 2)
k_onesweep(const K *__restrict__ kin, const uint32_t *__restrict__ vin, K *__restrict__ kout,
           uint32_t *__restrict__ vout, const uint32_t *n_dev, int64_t n_host, int shift,
           uint32_t mask, const uint32_t *__restrict__ digit_base, uint64_t *status,
           uint32_t *ticket, const uint32_t *epoch_ptr, uint32_t epoch_off, int *err,
           uint2 *__restrict__ ranges) {
    constexpr int ITEMS = SortShape<K>::kItems;
    constexpr int PART = SortSmem<K>::kPart;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem<K> &S = *reinterpret_cast<SortSmem<K> *>(smem_raw);
    if (*err) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int64_t nparts = (n + PART - 1) / PART;
    const uint32_t epoch = *epoch_ptr + epoch_off;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < kOsWarps * kRadix; i += kOsThreads) (&S.match[0][0])[i] = 0;
    for (;;) {
        if (tid == 0) S.part = atomicAdd(ticket, 1u);
        for (int i = tid; i < kOsWarps * kRadix; i += kOsThreads) (&S.whist[0][0])[i] = 0;
        __syncthreads();
        const int64_t part = S.part;
        if (part >= nparts) break;
        const int64_t base = part * PART + (int64_t)warp * (ITEMS * 32);
        // keys first; values are loaded only after ranking, to keep few live registers
        K key[ITEMS];
        uint32_t rank[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int64_t idx = base + i * 32 + lane;
            key[i] = idx < n ? kin[idx] : (K)0;
        }
        // rank of each item among the warp's earlier items with its digit:
        // the lanes sharing a digit (peers) are found by one shared-memory OR
        // of the lane bits into the warp's mask of that digit (the lowest
        // peer clears it again). (A shortcut for warps whose lanes all share
        // one digit cost more in its test than it saved, even on depth keys.)
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const bool valid = base + i * 32 + lane < n;
            const uint32_t d = digit_of(key[i], shift, mask);
            if (valid) atomicOr(&S.match[warp][d], 1u << lane);
            __syncwarp();
            const uint32_t peers = valid ? S.match[warp][d] : 0u;
            uint32_t before = 0;
            if (valid) before = S.whist[warp][d];
            __syncwarp();
            if (valid && (peers & lt) == 0) {
                S.whist[warp][d] = before + __popc(peers);
                S.match[warp][d] = 0u;
            }
            __syncwarp();
            rank[i] = before + __popc(peers & lt);
        }
        __syncthreads();
        // threads 0..255 own one digit each: warp offsets and the partition's
        // total (published at once for the successors' look-back), then the
        // block-local scan of the totals
        uint32_t run = 0, incl = 0, ds = 0;
        uint64_t *slot = status + part * kRadix + tid;
        if (tid < kRadix) {
            const int d = tid;
#pragma unroll
            for (int w = 0; w < kOsWarps; ++w) {
                const uint32_t t = S.whist[w][d];
                S.whist[w][d] = run;
                run += t;
            }
            publish(slot, pack_status(part == 0 ? kFlagPrefix : kFlagAgg, epoch, run));
            incl = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) S.wtot[warp] = incl;
        }
        __syncthreads();
        if (tid < kRadix) {
            // block-local start of digit d, folded into every warp's offset of
            // d (one lookup per item when staging)
            uint32_t wbase = 0;
            for (int w = 0; w < warp; ++w) wbase += S.wtot[w];
            ds = wbase + incl - run;
#pragma unroll
            for (int w = 0; w < kOsWarps; ++w) S.whist[w][tid] += ds;
        }
        __syncthreads();
        // stage the keys in digit order, then request the values (they arrive
        // while the digit owners look back)
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            if (base + i * 32 + lane < n) {
                const uint32_t d = digit_of(key[i], shift, mask);
                rank[i] += S.whist[warp][d];
                S.keys[rank[i]] = key[i];
            }
        }
        uint32_t val[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const int64_t idx = base + i * 32 + lane;
            val[i] = kIdentity ? (uint32_t)idx : (idx < n ? vin[idx] : 0u);
        }
        if (tid < kRadix) {
            // the partition's exclusive prefix of digit d by decoupled look-back;
            // output position = gstart[d] + staged position (modulo 2^32)
            uint32_t prev = 0;
            if (part > 0) {
                look_back(status + tid, part, kRadix, epoch, &prev, err);
                publish(slot, pack_status(kFlagPrefix, epoch, prev + run));
            }
            S.gstart[tid] = digit_base[tid] + prev - ds;
        }
#pragma unroll
        for (int i = 0; i < ITEMS; ++i)
            if (base + i * 32 + lane < n) S.vals[rank[i]] = val[i];
        __syncthreads();
        const int64_t rem = n - part * PART;
        const int cnt = rem < PART ? (int)rem : PART;
        for (int j = tid; j < cnt; j += kOsThreads) {
            const K k = S.keys[j];
            const uint32_t d = digit_of(k, shift, mask);
            const int64_t g = (int64_t)(S.gstart[d] + (uint32_t)j);
            // digit counts that disagree with the keys (a caller's histogram)
            // would place a key outside [0, n): never written there
            if (g >= n) continue;
            if (kOut == 0) kout[g] = k;
            vout[g] = S.vals[j];
            if (kOut == 2) {
                const uint32_t t = (uint32_t)k;
                if (j == 0 || S.keys[j - 1] != k) atomicMax(&ranges[t].x, ~(uint32_t)g);
                if (j + 1 == cnt || S.keys[j + 1] != k) atomicMax(&ranges[t].y, (uint32_t)g + 1u);
            }
        }
        __syncthreads();
    }
}

size_t sort_smem_bytes(int key_bytes) {
    return key_bytes == 8 ? sizeof(SortSmem<uint64_t>) : sizeof(SortSmem<uint32_t>);
}

template <typename K>
static void set_sort_attr() {
    const int b = (int)sizeof(SortSmem<K>);
    cudaFuncSetAttribute(k_onesweep<K, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_onesweep<K, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_onesweep<K, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    cudaFuncSetAttribute(k_onesweep<K, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

void sort_init_attributes() {
    set_sort_attr<uint32_t>();
    set_sort_attr<uint64_t>();
    cudaFuncSetAttribute(k_onesweep<uint32_t, false, 2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SortSmem<uint32_t>));
}

template <typename K, bool kIdentity>
static void launch_pass(int out, int grid, size_t smem, cudaStream_t st, const K *kin,
                        const uint32_t *vin, K *kout, uint32_t *vout, const SortArgs &a, int sh,
                        uint32_t mask, int p) {
    const uint32_t *base = a.hist + p * kRadix;
    if (out == 1)
        k_onesweep<K, kIdentity, 1><<<grid, kOsThreads, smem, st>>>(
            kin, vin, kout, vout, a.n_dev, a.n_host, sh, mask, base, a.status, a.tickets + p,
            a.epoch, a.epoch_off + p, a.err, nullptr);
    else
        k_onesweep<K, kIdentity, 0><<<grid, kOsThreads, smem, st>>>(
            kin, vin, kout, vout, a.n_dev, a.n_host, sh, mask, base, a.status, a.tickets + p,
            a.epoch, a.epoch_off + p, a.err, nullptr);
}

template <typename K>
static void launch_sort_t(const SortArgs &a, int grid, cudaStream_t st) {
    const int passes = sort_passes(a.begin_bit, a.end_bit);
    const size_t smem = sizeof(SortSmem<K>);
    if (!a.hist_ready) {
        cudaMemsetAsync(a.hist, 0, sizeof(uint32_t) * kRadix * passes, st);
        k_upsweep<K><<<grid, kSortThreads, 0, st>>>((const K *)a.keys[0], a.n_dev, a.n_host,
                                                    a.begin_bit, a.end_bit, a.hist, a.err);
    }
    k_digit_scan<<<passes, kRadix, 0, st>>>(a.hist, a.err);
    if (a.hook) a.hook(a.hook_user, 0);
    for (int p = 0; p < passes; ++p) {
        const int src = p & 1, dst = src ^ 1;
        const int sh = a.begin_bit + 8 * p;
        const int bits = std::min(8, a.end_bit - sh);
        const uint32_t mask = (1u << bits) - 1u;
        const bool last = p == passes - 1;
        const K *kin = (const K *)a.keys[src];
        K *kout = (K *)a.keys[dst];
        if (last && a.ranges && sizeof(K) == 4 && !(p == 0 && a.vals_identity))
            k_onesweep<uint32_t, false, 2><<<grid, kOsThreads, smem, st>>>(
                (const uint32_t *)kin, a.vals[src], (uint32_t *)kout, a.vals[dst], a.n_dev,
                a.n_host, sh, mask, a.hist + p * kRadix, a.status, a.tickets + p, a.epoch,
                a.epoch_off + p, a.err, a.ranges);
        else if (p == 0 && a.vals_identity)
            launch_pass<K, true>(last && a.skip_last_keys ? 1 : 0, grid, smem, st, kin, nullptr,
                                 kout, a.vals[dst], a, sh, mask, p);
        else
            launch_pass<K, false>(last && a.skip_last_keys ? 1 : 0, grid, smem, st, kin,
                                  a.vals[src], kout, a.vals[dst], a, sh, mask, p);
        if (a.hook) a.hook(a.hook_user, p + 1);
    }
}

void launch_sort(const SortArgs &a, int grid, cudaStream_t st) {
    if (a.key_bytes == 8) launch_sort_t<uint64_t>(a, grid, st);
    else launch_sort_t<uint32_t>(a, grid, st);
}

}  // namespace ngs
