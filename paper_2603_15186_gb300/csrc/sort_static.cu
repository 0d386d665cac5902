// Allocation-free variant of the standalone radix sort (ngs_sort_pairs_static).
//
// Some callers cannot allocate device memory at the point where they sort:
// code that runs while another component owns every device allocation (a
// host application with its own memory pool), latency-critical loops where a
// cudaMalloc / cudaFree would synchronise the device, and contexts where no
// renderer context exists at all. For them this entry point takes its scratch
// (alternate key and value buffers, digit histograms, tickets, look-back
// status words, an epoch counter and an error word) from one file-scope device
// array of fixed size, g_sort_scratch, which every GPU that loads the library
// holds until the process exits. It calls no cudaMalloc, cudaFree or other
// allocating routine.
//
// The array is shared by every call on a device and keeps the last call's
// contents: tickets and histograms are cleared at the start of each call, and
// the look-back status words are told apart from earlier calls' by an epoch
// that each call advances. A device-side error of a call (a bounded look-back
// wait that gave up) is moved, by the next call's first kernel, from the
// working error word into a latched word, so that it stops no later call;
// ngs_sort_pairs_static_status() returns and clears it. Calls whose work
// overlaps on the GPU (different streams, or different host threads without
// ordering) race on the array and give undefined results.
//
// Host code must not hand the array's name to a kernel: in host code it is a
// stand-in symbol, not a device address. Its device address is looked up once
// per device with cudaGetSymbolAddress (with that device current) on the first
// call made on that device, which is why the first call on each device should
// happen before any stream capture.
#include <algorithm>
#include <mutex>

#include "ngs_internal.cuh"

namespace ngs {

namespace {

constexpr int64_t kStaticMaxPairs = (int64_t)1 << 19;     // 524,288 pairs
constexpr int kStaticMaxDevices = 64;
constexpr int64_t kStaticParts = (kStaticMaxPairs + 4095) / 4096;

// byte layout of the scratch array (every region 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffKeys = 0;                                         // alternate keys (u64 max)
constexpr size_t kOffVals = align256(kOffKeys + 8 * kStaticMaxPairs);   // alternate values
constexpr size_t kOffStatus = align256(kOffVals + 4 * kStaticMaxPairs); // look-back words
constexpr size_t kOffHist = align256(kOffStatus + 8 * 256 * kStaticParts);
constexpr size_t kOffTickets = align256(kOffHist + 4 * 8 * 256);
constexpr size_t kOffEpoch = align256(kOffTickets + 4 * 8);
constexpr size_t kOffErr = align256(kOffEpoch + 4);       // error of the running call
constexpr size_t kOffLatched = kOffErr + 4;                 // first error since the last query
constexpr size_t kScratchBytes = align256(kOffLatched + 4);

}  // namespace

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
unsigned char *g_addr[kStaticMaxDevices] = {};
uint64_t g_calls[kStaticMaxDevices] = {};
int g_sms[kStaticMaxDevices] = {};

// Start of a call: keeps the previous call's error (if any) in the latched
// word, clears the working error word and advances the epoch.
__global__ void k_static_begin(uint32_t *epoch, uint32_t inc, int *err, int *latched) {
    if (*err != 0 && *latched == 0) *latched = *err;
    *err = 0;
    *epoch += inc;
}

}  // namespace

int64_t sort_static_max_pairs() { return kStaticMaxPairs; }
size_t sort_static_scratch_bytes() { return kScratchBytes; }

// Returns NGS_OK and the scratch device address for the current device,
// looking it up (and preparing the kernels' shared-memory limits) on first use.
static ngs_status static_scratch(int dev, unsigned char **out, int *sms) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (dev < 0 || dev >= kStaticMaxDevices) return NGS_ERR_INVALID_ARG;
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NGS_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return NGS_ERR_CUDA;
        sort_init_attributes();
        g_addr[dev] = (unsigned char *)p;
        g_sms[dev] = n;
    }
    *out = g_addr[dev];
    *sms = g_sms[dev];
    return NGS_OK;
}

}  // namespace ngs

using namespace ngs;

extern "C" NGS_API ngs_status ngs_sort_pairs_static(void *d_keys, uint32_t *d_vals, int64_t n,
                                                    int32_t key_bytes, int32_t begin_bit,
                                                    int32_t end_bit, void *stream) {
    if ((key_bytes != 4 && key_bytes != 8) || n < 0) return NGS_ERR_INVALID_ARG;
    if (begin_bit < 0 || end_bit > 8 * key_bytes || begin_bit > end_bit) return NGS_ERR_INVALID_ARG;
    if (n > kStaticMaxPairs) return NGS_ERR_CAPACITY;
    if (n > 0 && (!d_keys || !d_vals)) return NGS_ERR_INVALID_ARG;
    if (n == 0 || begin_bit == end_bit) return NGS_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NGS_ERR_CUDA;
    unsigned char *base = nullptr;
    int sms = 0;
    ngs_status s = static_scratch(dev, &base, &sms);
    if (s != NGS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *tickets = (uint32_t *)(base + kOffTickets);
    uint32_t *epoch = (uint32_t *)(base + kOffEpoch);
    uint64_t *status = (uint64_t *)(base + kOffStatus);
    int *err = (int *)(base + kOffErr);
    const int passes = sort_passes(begin_bit, end_bit);
    {
        // the 30-bit epoch advances 32 per call; long before it wraps, the
        // status words are cleared and the epoch restarts
        std::lock_guard<std::mutex> lock(g_mu);
        if (++g_calls[dev] >= ((uint64_t)1 << 24)) {
            g_calls[dev] = 1;
            if (cudaMemsetAsync(status, 0, 8 * 256 * kStaticParts, st) != cudaSuccess ||
                cudaMemsetAsync(epoch, 0, 4, st) != cudaSuccess)
                return NGS_ERR_CUDA;
        }
    }
    if (cudaMemsetAsync(tickets, 0, 4 * 8, st) != cudaSuccess) return NGS_ERR_CUDA;
    k_static_begin<<<1, 1, 0, st>>>(epoch, 32u, err, (int *)(base + kOffLatched));
    SortArgs a{};
    a.keys[0] = d_keys; a.keys[1] = base + kOffKeys;
    a.vals[0] = d_vals; a.vals[1] = (uint32_t *)(base + kOffVals);
    a.n_dev = nullptr; a.n_host = n; a.n_max = n;
    a.key_bytes = key_bytes; a.begin_bit = begin_bit; a.end_bit = end_bit;
    a.vals_identity = false;
    a.hist = (uint32_t *)(base + kOffHist);   // cleared by the launcher
    a.tickets = tickets; a.status = status;
    a.epoch = epoch; a.epoch_off = 0; a.err = err;
    a.hook = nullptr; a.hook_user = nullptr;
    const int64_t parts = (n + sort_partition() - 1) / sort_partition();
    const int grid = (int)std::min<int64_t>(parts, 2 * (int64_t)sms);
    launch_sort(a, grid < 1 ? 1 : grid, st);
    if (passes & 1) {
        if (cudaMemcpyAsync(d_keys, base + kOffKeys, (size_t)n * key_bytes,
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(d_vals, base + kOffVals, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                            st) != cudaSuccess)
            return NGS_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? NGS_OK : NGS_ERR_CUDA;
}

extern "C" NGS_API ngs_status ngs_sort_pairs_static_status(void *stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NGS_ERR_CUDA;
    if (dev < 0 || dev >= kStaticMaxDevices) return NGS_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        base = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) return NGS_ERR_CUDA;
    if (!base) return NGS_OK;   // no call has run on this device yet
    int words[2] = {0, 0};      // working and latched error words
    if (cudaMemcpyAsync(words, base + kOffErr, sizeof(words), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemsetAsync(base + kOffErr, 0, sizeof(words), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NGS_ERR_CUDA;
    return (ngs_status)(words[1] != 0 ? words[1] : words[0]);
}
