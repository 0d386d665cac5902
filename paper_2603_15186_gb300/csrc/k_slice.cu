// GS-slice occupancy (NavGSim Sec. III-C): every leaf Gaussian is cut by a set
// of horizontal planes z_k = z0 + k dz; on each plane the cut is the 2D
// Gaussian
//   G2D(x, z) = exp(-1/2 lambda (z - mu_z)^2) exp(-1/2 [x - mu(z)]^T C [x - mu(z)])
// with C the xy block of Sigma^-1, mu(z) = mu_xy - (z - mu_z) (alpha, beta) and
// lambda the Schur complement. Per plane and grid cell the kernel keeps the
// largest slice value a = min(0.99, o G2D(cell centre, z_k)) over the leaves
// whose a reaches 1/255; a cell is occupied where that value reaches the
// threshold.
//
// In float32 the slice parameters are taken in their well-conditioned forms
// (equal to the paper's by the block-inverse identities): lambda = 1 /
// Sigma_zz, (alpha, beta) = -(Sigma_xz, Sigma_yz) / Sigma_zz, C = (R S^-2 R^T)
// restricted to xy, so no difference of large terms appears.
//
// One thread per node (interior nodes return at once): planes within the
// slice's vertical support, cells of each slice's support box (the ellipse
// where a >= 1/255, widened by a relative 1e-4 and 1e-6 m), each value folded
// into the cell with atomicMax on its bits (non-negative floats order like
// their bit patterns, so the result does not depend on the order).
#include "ngs_internal.cuh"

namespace ngs {

template <typename A>
__device__ __forceinline__ void load_sop(const void *p, int64_t i, float v[4]);
template <>
__device__ __forceinline__ void load_sop<float>(const void *p, int64_t i, float v[4]) {
    const float4 t = reinterpret_cast<const float4 *>(p)[i];
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void load_sop<__half>(const void *p, int64_t i, float v[4]) {
    const uint2 t = reinterpret_cast<const uint2 *>(p)[i];
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
template <>
__device__ __forceinline__ void load_sop<__nv_bfloat16>(const void *p, int64_t i, float v[4]) {
    const uint2 t = reinterpret_cast<const uint2 *>(p)[i];
    v[0] = __uint_as_float(t.x << 16); v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16); v[3] = __uint_as_float(t.y & 0xffff0000u);
}

template <typename A>
__global__ void __launch_bounds__(256)
k_slice(SceneDev sc, SliceGrid g, uint32_t *__restrict__ value_bits,
        unsigned long long *work) {
    const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= sc.n) return;
    if (__float_as_int(sc.box_hi[node].w) != 0) return;            // leaves only
    const float4 p = sc.pos4[node];
    if (__float_as_uint(p.w) & kNodeCullOpacity) return;           // 255 o < 1
    float so[4];
    load_sop<A>(sc.sop, node, so);
    const float o = so[3];
    const float K = 2.0f * logf(255.0f * o);                       // a >= 1/255 <=> q <= K
    const float4 q4 = sc.quat[node];
    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float s2[3], is2[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        s2[k] = expf(2.0f * so[k]);
        is2[k] = expf(-2.0f * so[k]);
    }
    // Sigma's z row and Sigma^-1's xy block
    float sxz = 0.f, syz = 0.f, szz = 0.f, cxx = 0.f, cxy = 0.f, cyy = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        sxz += R[k] * s2[k] * R[6 + k];
        syz += R[3 + k] * s2[k] * R[6 + k];
        szz += R[6 + k] * s2[k] * R[6 + k];
        cxx += R[k] * is2[k] * R[k];
        cxy += R[k] * is2[k] * R[3 + k];
        cyy += R[3 + k] * is2[k] * R[3 + k];
    }
    const float lambda = 1.0f / szz;
    const float alpha = -sxz / szz, beta = -syz / szz;
    const float det = cxx * cyy - cxy * cxy;
    if (!(det > 0.0f) || !(K >= 0.0f)) return;
    // planes within the vertical support lambda z'^2 <= K
    const float rz = sqrtf(K / lambda) * 1.0001f + 1e-6f;
    int k0 = (int)ceilf((p.z - rz - g.z0) / g.dz), k1 = (int)floorf((p.z + rz - g.z0) / g.dz);
    k0 = max(k0, 0);
    k1 = min(k1, g.nz - 1);
    const float ixx = cyy / det, iyy = cxx / det;                  // C^-1 diagonal
    const int64_t plane = (int64_t)g.nx * g.ny;
    unsigned long long evals = 0;
    for (int k = k0; k <= k1; ++k) {
        const float zp = (g.z0 + (float)k * g.dz) - p.z;
        const float ez = lambda * zp * zp;
        const float rem = K - ez;
        if (rem < 0.0f) continue;
        const float hx = sqrtf(rem * ixx) * 1.0001f + 1e-6f, hy = sqrtf(rem * iyy) * 1.0001f + 1e-6f;
        const float mx = p.x - zp * alpha, my = p.y - zp * beta;
        const int i0 = max(0, (int)ceilf((mx - hx - g.x0) / g.cell - 0.5f));
        const int i1 = min(g.nx - 1, (int)floorf((mx + hx - g.x0) / g.cell - 0.5f));
        const int j0 = max(0, (int)ceilf((my - hy - g.y0) / g.cell - 0.5f));
        const int j1 = min(g.ny - 1, (int)floorf((my + hy - g.y0) / g.cell - 0.5f));
        uint32_t *vk = value_bits + (int64_t)k * plane;
        for (int j = j0; j <= j1; ++j) {
            const float dy = g.y0 + ((float)j + 0.5f) * g.cell - my;
            for (int i = i0; i <= i1; ++i) {
                const float dx = g.x0 + ((float)i + 0.5f) * g.cell - mx;
                const float q = ez + cxx * dx * dx + 2.0f * cxy * dx * dy + cyy * dy * dy;
                const float a = o * expf(-0.5f * q);
                ++evals;
                if (a >= (1.0f / 255.0f))
                    atomicMax(&vk[(int64_t)j * g.nx + i], __float_as_uint(fminf(0.99f, a)));
            }
        }
    }
    if (work && evals) atomicAdd(work, evals);
}

__global__ void k_slice_mask(const uint32_t *__restrict__ value_bits, int64_t n, float threshold,
                             uint8_t *__restrict__ occ) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        occ[i] = __uint_as_float(value_bits[i]) >= threshold ? 1 : 0;
}

void launch_slice(const SceneDev &sc, const SliceGrid &g, float *value, uint8_t *occ,
                  unsigned long long *work, int num_sms, cudaStream_t st) {
    const int64_t cells = (int64_t)g.nx * g.ny * g.nz;
    cudaMemsetAsync(value, 0, (size_t)cells * sizeof(float), st);
    const int64_t blocks = (sc.n + 255) / 256;
    uint32_t *bits = reinterpret_cast<uint32_t *>(value);
    if (blocks > 0) {
        switch (sc.attr_dtype) {
        case NGS_F16: k_slice<__half><<<(unsigned)blocks, 256, 0, st>>>(sc, g, bits, work); break;
        case NGS_BF16:
            k_slice<__nv_bfloat16><<<(unsigned)blocks, 256, 0, st>>>(sc, g, bits, work);
            break;
        default: k_slice<float><<<(unsigned)blocks, 256, 0, st>>>(sc, g, bits, work); break;
        }
    }
    if (occ)
        k_slice_mask<<<std::max(1, (int)std::min<int64_t>((cells + 255) / 256, 16 * num_sms)), 256, 0,
                       st>>>(bits, cells, g.threshold, occ);
}

}  // namespace ngs
