// Navigable map and shortest paths on the GS-slice occupancy (NavGSim
// Sec. III-C: the slices give the navigable area for collision checks and path
// planning; Sec. IV-A: expert trajectories come from a shortest-path planner).
//
//  - blocked(i, j): some plane k in [k_lo, k_hi] (the robot's height range) is
//    occupied at a cell within Chebyshev distance `inflate` of (i, j).
//  - One distance field per goal: 4-connected breadth-first steps over free
//    cells, UINT32_MAX where unreachable. One CTA per goal runs the whole
//    search on a frontier queue in global memory: level by level, its threads
//    expand the frontier's cells and admit each unreached free neighbour once
//    (atomicCAS from UINT32_MAX to L + 1), appending it to the next frontier.
//    The distances are the breadth-first ones whatever the order inside a
//    level; every cell enters a frontier at most once, so the loop ends after
//    at most one level per cell. No CTA waits on another.
//  - A path descends a field from its start, taking the first neighbour in the
//    order (+x, -x, +y, -y) whose distance is one less, one thread per agent.
#include "ngs_internal.cuh"
#include "nav.h"

namespace ngs {

constexpr uint32_t kNavUnreached = 0xFFFFFFFFu;

__global__ void k_nav_any(const uint8_t *__restrict__ occ, int64_t plane, int k_lo, int k_hi,
                          uint8_t *__restrict__ any) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < plane;
         c += (int64_t)gridDim.x * blockDim.x) {
        uint8_t a = 0;
        for (int k = k_lo; k <= k_hi; ++k) a |= occ[(int64_t)k * plane + c];
        any[c] = a ? 1 : 0;
    }
}

__global__ void k_nav_dilate(const uint8_t *__restrict__ any, int nx, int ny, int r,
                             uint8_t *__restrict__ blocked) {
    const int64_t plane = (int64_t)nx * ny;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < plane;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % nx), j = (int)(c / nx);
        uint8_t b = 0;
        for (int dj = -r; dj <= r && !b; ++dj) {
            const int y = j + dj;
            if (y < 0 || y >= ny) continue;
            for (int di = -r; di <= r; ++di) {
                const int x = i + di;
                if (x >= 0 && x < nx && any[(int64_t)y * nx + x]) { b = 1; break; }
            }
        }
        blocked[c] = b;
    }
}

__global__ void k_nav_init(const uint8_t *__restrict__ blocked, int nx, int ny,
                           const int2 *__restrict__ goals, int n_goals,
                           uint32_t *__restrict__ dist) {
    const int64_t plane = (int64_t)nx * ny, total = plane * n_goals;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int g = (int)(t / plane);
        const int64_t c = t - (int64_t)g * plane;
        const int2 q = goals[g];
        const bool goal = q.x >= 0 && q.x < nx && q.y >= 0 && q.y < ny &&
                          c == (int64_t)q.y * nx + q.x && !blocked[c];
        dist[t] = goal ? 0u : kNavUnreached;
    }
}

__global__ void __launch_bounds__(1024)
k_nav_bfs(const uint8_t *__restrict__ blocked, int nx, int ny, const int2 *__restrict__ goals,
          uint32_t *dist, uint32_t *queues) {
    __shared__ uint32_t s_next, s_cur;
    const int g = blockIdx.x, tid = threadIdx.x;
    const int64_t plane = (int64_t)nx * ny;
    uint32_t *dg = dist + (int64_t)g * plane;
    uint32_t *cur = queues + (int64_t)g * 2 * plane, *nxt = cur + plane;
    const int2 q = goals[g];
    if (tid == 0) {
        const bool ok = q.x >= 0 && q.x < nx && q.y >= 0 && q.y < ny &&
                        !blocked[(int64_t)q.y * nx + q.x];
        if (ok) cur[0] = (uint32_t)((int64_t)q.y * nx + q.x);
        s_cur = ok ? 1u : 0u;
        s_next = 0;
    }
    __syncthreads();
    for (uint32_t level = 0; s_cur > 0; ++level) {
        const uint32_t ncur = s_cur;
        for (uint32_t k = tid; k < ncur; k += blockDim.x) {
            const uint32_t c = cur[k];
            const int i = (int)(c % (uint32_t)nx), j = (int)(c / (uint32_t)nx);
            const int ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (ni[e] < 0 || ni[e] >= nx || nj[e] < 0 || nj[e] >= ny) continue;
                const uint32_t n = (uint32_t)nj[e] * (uint32_t)nx + (uint32_t)ni[e];
                if (blocked[n] || dg[n] != kNavUnreached) continue;
                if (atomicCAS(&dg[n], kNavUnreached, level + 1u) == kNavUnreached)
                    nxt[atomicAdd(&s_next, 1u)] = n;
            }
        }
        __syncthreads();
        if (tid == 0) {
            s_cur = s_next;
            s_next = 0;
        }
        uint32_t *t = cur;
        cur = nxt;
        nxt = t;
        __syncthreads();
    }
}

__global__ void k_nav_paths(const uint32_t *__restrict__ dist, int nx, int ny, int n_goals,
                            const int3 *__restrict__ starts, int n, int max_len,
                            int2 *__restrict__ paths, int32_t *__restrict__ lens) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const int3 s = starts[a];
    int len = 0;
    if (s.z >= 0 && s.z < n_goals && s.x >= 0 && s.x < nx && s.y >= 0 && s.y < ny && max_len > 0) {
        const uint32_t *dg = dist + (int64_t)s.z * nx * ny;
        uint32_t d = dg[(int64_t)s.y * nx + s.x];
        int i = s.x, j = s.y;
        if (d != kNavUnreached) {
            for (;;) {
                paths[(int64_t)a * max_len + len] = make_int2(i, j);
                ++len;
                if (d == 0 || len >= max_len) break;
                const int ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
                for (int e = 0; e < 4; ++e) {
                    if (ni[e] < 0 || ni[e] >= nx || nj[e] < 0 || nj[e] >= ny) continue;
                    if (dg[(int64_t)nj[e] * nx + ni[e]] == d - 1u) { i = ni[e]; j = nj[e]; break; }
                }
                --d;
            }
        }
    }
    lens[a] = len;
}

static int nav_grid(int64_t work, int num_sms) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)num_sms * 16));
}

// scratch: any [ny * nx] bytes, goals [n_goals] int2, queues [n_goals][2][ny * nx]
// u32; returns 0 or a cudaError_t (synchronises the stream)
int launch_nav_fields(const uint8_t *occ, int nx, int ny, int k_lo, int k_hi, int inflate,
                      const int2 *d_goals, int n_goals, uint8_t *any, uint32_t *queues,
                      uint8_t *blocked, uint32_t *dist, int num_sms, cudaStream_t st) {
    const int64_t plane = (int64_t)nx * ny;
    k_nav_any<<<nav_grid(plane, num_sms), 256, 0, st>>>(occ, plane, k_lo, k_hi, any);
    k_nav_dilate<<<nav_grid(plane, num_sms), 256, 0, st>>>(any, nx, ny, inflate, blocked);
    k_nav_init<<<nav_grid(plane * n_goals, num_sms), 256, 0, st>>>(blocked, nx, ny, d_goals,
                                                                   n_goals, dist);
    k_nav_bfs<<<n_goals, 1024, 0, st>>>(blocked, nx, ny, d_goals, dist, queues);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return (int)e;
}

void launch_nav_paths(const uint32_t *dist, int nx, int ny, int n_goals, const int3 *starts,
                      int n, int max_len, int2 *paths, int32_t *lens, cudaStream_t st) {
    if (n > 0)
        k_nav_paths<<<(n + 127) / 128, 128, 0, st>>>(dist, nx, ny, n_goals, starts, n, max_len,
                                                     paths, lens);
}

}  // namespace ngs
