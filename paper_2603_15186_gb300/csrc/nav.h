// Launchers of the navigation kernels (k_nav.cu), used by the C ABI.
#ifndef NGS_NAV_H
#define NGS_NAV_H

#include <cuda_runtime.h>
#include <stdint.h>

namespace ngs {

// navigable map and breadth-first distance fields (synchronises `st`; returns
// 0 or a cudaError_t), and shortest paths by descent
int launch_nav_fields(const uint8_t *occ, int nx, int ny, int k_lo, int k_hi, int inflate,
                      const int2 *d_goals, int n_goals, uint8_t *any, uint32_t *queues,
                      uint8_t *blocked, uint32_t *dist, int num_sms, cudaStream_t st);
void launch_nav_paths(const uint32_t *dist, int nx, int ny, int n_goals, const int3 *starts,
                      int n, int max_len, int2 *paths, int32_t *lens, cudaStream_t st);

}  // namespace ngs

#endif
