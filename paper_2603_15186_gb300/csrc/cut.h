// Frustum-culled and shared level-of-detail cuts (k_cut.cu), used by the C ABI.
#ifndef NGS_CUT_H
#define NGS_CUT_H

#include <cuda_runtime.h>
#include <stdint.h>

namespace ngs {

struct DevCamera;

// One camera of a shared cut: the five planes of its view volume in world
// terms, P_k(x) = a[k] . (x - pos) + (k == 0 ? b0 : 0), in the order near,
// left, right, top, bottom (a node whose box has P_k < 0 everywhere for some k
// is culled), and the inputs of its granularity test.
struct CutCam {
    float a[5][3];
    float b0;
    float pos[3];
    float fx, tau;
    float pad[3];
};
static_assert(sizeof(CutCam) == 96, "CutCam layout");

// Group g of the cameras is cams[group_begin[g] .. group_begin[g + 1]); its
// cut goes to ids[offsets[g] .. offsets[g + 1]) (ascending node ids), the
// total to counters[CNT_CUT]. The status words, ticket and epoch follow the
// plain cut's conventions.
void launch_cut_shared(bool frustum, const float4 *box_lo, const float4 *box_hi, int64_t n_nodes,
                       const CutCam *cams, const int32_t *group_begin, int n_groups,
                       uint32_t *ids, int64_t cap, uint32_t *offsets, uint32_t *counters,
                       uint32_t *ticket, uint64_t *status, const uint32_t *epoch,
                       uint32_t epoch_off, int *err, int grid, cudaStream_t st);

// Plain cut for many cameras (ngs_select_cut), in two passes over (block of
// cut_partition_nodes() nodes, chunk of up to 8 cameras) partitions taken in
// block-major order. The counting pass writes part_vals[c * nblk + b] = the
// selected nodes of camera c in block b; a chained scan of those counts in
// camera-major order gives each (camera, block) its output offset; the
// writing pass reads those offsets from part_vals and writes the ids. Both
// passes return at once if *err is set. With ccams (instead of cams, which is
// then unused) each camera's cut is frustum-culled against its planes: the
// shared cut of a group of one camera.
void launch_cut_blocked(bool write, const float4 *box_lo, const float4 *box_hi, int64_t n_nodes,
                        const DevCamera *cams, const CutCam *ccams, int n_cams,
                        uint32_t *part_vals, uint32_t *ids, int64_t cap, uint32_t *ticket,
                        const int *err, int grid, cudaStream_t st);

// offsets[c] = part_off[c * nblk] for c < n_cams, offsets[n_cams] = *total
// (int64); latches the capacity error when *total exceeds cap.
void launch_cut_cam_offsets(const uint32_t *part_off, const uint32_t *total, int64_t nblk,
                            int n_cams, int64_t cap, int64_t *offsets, uint32_t *counters,
                            int *err, cudaStream_t st);

}  // namespace ngs

#endif
