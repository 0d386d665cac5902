// K2: per cut Gaussian, the 3DGS screen-space preprocess that NavGSim's
// renderer inherits (Sec. III-A/III-B): view transform, near-plane cull, EWA
// projection of the 3D covariance, Sigma2D = J W Sigma W^T J^T + 0.3 I, its
// inverse (the conic), the pixel centre, degree-3 SH colour seen from the
// camera, the tile rectangle of the support, and the depth sort key.
//
// Support: alpha = min(0.99, o exp(-1/2 d^T conic d)) reaches 1/255 only inside
// the ellipse d^T conic d <= K = 2 ln(255 o), whose axis-aligned bounding box
// has half-widths sqrt(K Sigma2D_xx), sqrt(K Sigma2D_yy); the rectangle covers
// the tiles touched by that box widened by 1/64 pixel, so it is conservative
// under float32 rounding and the pixels do not depend on the tile shape.
//
// Depth key: the view depth z = fma(R20, d0, fma(R21, d1, R22 d2)) with
// d_k = mu_k - c_k, every operation a single IEEE float32 rounding; its bits
// are the sort key and it decides the near-plane cull. The oracle evaluates
// the same sequence, so keys and culls agree bit for bit. No float64 anywhere.
//
// Output: each partition (block of nodes, camera) takes one slot per candidate
// (a Gaussian that passed the cut and the conservative cull) with one atomic
// allocation; visible ones are written to their slots in node order, the
// others leave a hole; (first slot, visible and candidate counts) go to a
// partition table. The dense depth-sort input is then gathered in
// camera-major, node-id order through a scan of that table, so depth ties are
// broken by node id whatever the allocation order was.
// HBM per cut Gaussian: 4 B id + 16 B position (always); quaternion
// 16 B and scale/opacity 16 B (f32) or 8 B (f16/bf16) for those in front of
// the near plane; SH 192 B (f32) or 96 B for those with a non-empty rectangle;
// written per visible one: record 48 B (f32) or 32 B, key 4 B, rect 8 B
// (tile rectangle, camera index; pack_rect), and the node id (4 B) when the
// caller asks for it.
#include <algorithm>

#include "ngs_internal.cuh"

namespace ngs {

constexpr int kPreThreads = 256;
constexpr int kPreItems = 4;                          // phase-A nodes per thread
constexpr int kPrePart = kPreThreads * kPreItems;     // nodes per partition


template <typename A> struct Attr;
template <> struct Attr<float> {
    static __device__ __forceinline__ void load4(const void *p, int64_t i, float v[4]) {
        const float4 t = reinterpret_cast<const float4 *>(p)[i];
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    // rows i and j side by side: f(h, row i value, row j value)
    template <typename F>
    static __device__ __forceinline__ void stream_sh2(const void *p, int64_t i, int64_t j, F f) {
        const float4 *a = reinterpret_cast<const float4 *>(p) + i * 12;
        const float4 *b = reinterpret_cast<const float4 *>(p) + j * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float4 t = a[k], u = b[k];
            f(4 * k, t.x, u.x); f(4 * k + 1, t.y, u.y); f(4 * k + 2, t.z, u.z);
            f(4 * k + 3, t.w, u.w);
        }
    }
    template <int kUnused, typename F>
    static __device__ __forceinline__ void stream_sh(const void *p, int64_t i, F f) {
        const float4 *s = reinterpret_cast<const float4 *>(p) + i * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float4 t = s[k];
            f(4 * k, t.x); f(4 * k + 1, t.y); f(4 * k + 2, t.z); f(4 * k + 3, t.w);
        }
    }
};
template <> struct Attr<__half> {
    static __device__ __forceinline__ void load4(const void *p, int64_t i, float v[4]) {
        const uint2 t = reinterpret_cast<const uint2 *>(p)[i];
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&t.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&t.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    template <typename F>
    static __device__ __forceinline__ void stream_sh2(const void *p, int64_t i, int64_t j, F f) {
        const uint4 *a = reinterpret_cast<const uint4 *>(p) + i * 6;
        const uint4 *b = reinterpret_cast<const uint4 *>(p) + j * 6;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const uint4 t = a[k], u = b[k];
            const uint32_t w[4] = {t.x, t.y, t.z, t.w}, x[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 va = __half22float2(*reinterpret_cast<const __half2 *>(&w[q]));
                const float2 vb = __half22float2(*reinterpret_cast<const __half2 *>(&x[q]));
                f(8 * k + 2 * q, va.x, vb.x); f(8 * k + 2 * q + 1, va.y, vb.y);
            }
        }
    }
    template <int kUnused, typename F>
    static __device__ __forceinline__ void stream_sh(const void *p, int64_t i, F f) {
        const uint4 *s = reinterpret_cast<const uint4 *>(p) + i * 6;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const uint4 t = s[k];
            const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(&w[j]));
                f(8 * k + 2 * j, v.x); f(8 * k + 2 * j + 1, v.y);
            }
        }
    }
};
template <> struct Attr<__nv_bfloat16> {
    static __device__ __forceinline__ float2 bf2(uint32_t w) {
        // bfloat16 -> float32 is exact: the 16 bits are the high half of the float
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
    static __device__ __forceinline__ void load4(const void *p, int64_t i, float v[4]) {
        const uint2 t = reinterpret_cast<const uint2 *>(p)[i];
        const float2 a = bf2(t.x), b = bf2(t.y);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    template <typename F>
    static __device__ __forceinline__ void stream_sh2(const void *p, int64_t i, int64_t j, F f) {
        const uint4 *a = reinterpret_cast<const uint4 *>(p) + i * 6;
        const uint4 *b = reinterpret_cast<const uint4 *>(p) + j * 6;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const uint4 t = a[k], u = b[k];
            const uint32_t w[4] = {t.x, t.y, t.z, t.w}, x[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 va = bf2(w[q]), vb = bf2(x[q]);
                f(8 * k + 2 * q, va.x, vb.x); f(8 * k + 2 * q + 1, va.y, vb.y);
            }
        }
    }
    template <int kUnused, typename F>
    static __device__ __forceinline__ void stream_sh(const void *p, int64_t i, F f) {
        const uint4 *s = reinterpret_cast<const uint4 *>(p) + i * 6;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const uint4 t = s[k];
            const uint32_t w[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 v = bf2(w[j]);
                f(8 * k + 2 * j, v.x); f(8 * k + 2 * j + 1, v.y);
            }
        }
    }
};

// Real SH basis to degree 3 in the 3DGS sign convention (standard real SH
// times (-1)^|m|), index l*l + l + m; constants are the normalisations
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0) folded with
// the polynomial coefficients. The 48 coefficients are streamed from memory
// in storage order (coefficient-major), each channel accumulating k = 0..15.
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = 0.28209479177387814f;
    Y[1] = -0.48860251190291992f * y;
    Y[2] = 0.48860251190291992f * z;
    Y[3] = -0.48860251190291992f * x;
    Y[4] = 1.0925484305920792f * x * y;
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.54627421529603959f * (xx - yy);
    Y[9] = -0.59004358992664352f * y * (3.0f * xx - yy);
    Y[10] = 2.8906114426405538f * x * y * z;
    Y[11] = -0.45704579946446572f * y * (4.0f * zz - xx - yy);
    Y[12] = 0.37317633259011540f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -0.45704579946446572f * x * (4.0f * zz - xx - yy);
    Y[14] = 1.4453057213202769f * z * (xx - yy);
    Y[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
}

template <typename A>
__device__ __forceinline__ void sh_colour(const void *sh, int64_t node, float x, float y,
                                          float z, float rgb[3]) {
    float Y[16];
    sh_basis(x, y, z, Y);
    float acc[3] = {0.5f, 0.5f, 0.5f};
    Attr<A>::template stream_sh<3>(sh, node, [&](int h, float v) {
        acc[h % 3] = __fmaf_rn(Y[h / 3], v, acc[h % 3]);
    });
    rgb[0] = fmaxf(acc[0], 0.0f);
    rgb[1] = fmaxf(acc[1], 0.0f);
    rgb[2] = fmaxf(acc[2], 0.0f);
}

// The same with the coefficients of `node` moved toward those of `par` by v.
template <typename A>
__device__ __forceinline__ void sh_colour_blend(const void *sh, int64_t node, int64_t par,
                                                float v, float x, float y, float z,
                                                float rgb[3]) {
    float Y[16];
    sh_basis(x, y, z, Y);
    float acc[3] = {0.5f, 0.5f, 0.5f};
    Attr<A>::stream_sh2(sh, node, par, [&](int h, float cn, float cp) {
        acc[h % 3] = __fmaf_rn(Y[h / 3], __fmaf_rn(v, __fsub_rn(cp, cn), cn), acc[h % 3]);
    });
    rgb[0] = fmaxf(acc[0], 0.0f);
    rgb[1] = fmaxf(acc[1], 0.0f);
    rgb[2] = fmaxf(acc[2], 0.0f);
}

// Parent weight of the level-of-detail blend (Sec. III-B: transitions between
// levels are interpolated): v = 1 - clamp((s(p) - tau) / (s(p) - s(n)), 0, 1),
// 0 when s(p) is infinite or s(p) <= s(n). Every step one IEEE float32
// operation, the same sequence as the oracle's, so the blended mean and the
// depth key derived from it agree bit for bit.
__device__ __forceinline__ float blend_parent_weight(float s_n, float s_p, float tau) {
    if (!(s_p < __int_as_float(0x7f800000))) return 0.0f;
    const float den = __fsub_rn(s_p, s_n);
    if (!(den > 0.0f)) return 0.0f;
    const float w = fminf(fmaxf(__fdiv_rn(__fsub_rn(s_p, tau), den), 0.0f), 1.0f);
    return __fsub_rn(1.0f, w);
}

// Sigma = R(q) S^2 R(q)^T from a quaternion (w, x, y, z, normalised here) and
// log-scales; upper triangle S00, S01, S02, S11, S12, S22.
__device__ __forceinline__ void cov3d(const float4 q4, const float ls[3], float S[6]) {
    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z),
                R02 = 2.f * (x * z + w * y);
    const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z),
                R12 = 2.f * (y * z - w * x);
    const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x),
                R22 = 1.f - 2.f * (x * x + y * y);
    const float s0 = expf(ls[0]), s1 = expf(ls[1]), s2 = expf(ls[2]);
    const float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
    const float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
    const float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
    S[0] = M00 * M00 + M01 * M01 + M02 * M02;
    S[1] = M00 * M10 + M01 * M11 + M02 * M12;
    S[2] = M00 * M20 + M01 * M21 + M02 * M22;
    S[3] = M10 * M10 + M11 * M11 + M12 * M12;
    S[4] = M10 * M20 + M11 * M21 + M12 * M22;
    S[5] = M20 * M20 + M21 * M21 + M22 * M22;
}

struct PreOut {
    float x, y, F1, F2, F3, L, r, g, bl, hx, hy;
    uint32_t key;
    uint32_t rx0, ry0, rx1, ry1;   // tile rectangle
};

// Camera fields the phase-A tests read, staged in shared memory per group.
struct CamLite {
    float R[9];
    float pos[3];
    float fx, fy, cx, cy, tau;
    int32_t tiles_x, tiles_y;
    float tau2;   // __fmul_rn(tau, tau), as the cut test takes it
};

// Camera-independent inputs of the conservative cull of one node: its
// position word (mean + load-time flags), K = 2 ln(255 o) and the largest
// scale.
struct NodeCull {
    float4 p;
    float K, smax;
};

// Cheap conservative test (phase A of the fused kernel): false only for a
// Gaussian that cannot touch any tile of the camera.
__device__ __forceinline__ bool precull(const CamLite &cam, const NodeCull &nd, int tile_w,
                                        int tile_h) {
    const float4 p = nd.p;
    if (__float_as_uint(p.w) & kNodeCullOpacity) return false;
    const float dx = __fsub_rn(p.x, cam.pos[0]);
    const float dy = __fsub_rn(p.y, cam.pos[1]);
    const float dz = __fsub_rn(p.z, cam.pos[2]);
    // float32 view depth: its distance from the float64 depth is below
    // 1e-6 (|dx| + |dy| + |dz|), so a Gaussian this far behind the near plane is
    // culled without evaluating the float64 depth
    const float tz32 = __fmaf_rn(cam.R[6], dx, __fmaf_rn(cam.R[7], dy, __fmul_rn(cam.R[8], dz)));
    const float margin = 1e-6f * (fabsf(dx) + fabsf(dy) + fabsf(dz)) + 1e-6f;
    if (tz32 < kNearZ - margin) return false;
    if (tz32 <= 2.0f * kNearZ) return true;
    // Lateral test: with T0, T1 the rows of J W, Sigma2D_xx = T0 Sigma T0^T + 0.3
    // <= |T0|^2 smax^2 + 0.3 (smax the largest scale), so the support box of the
    // tile rectangle is no wider than hb; a box that misses the tile grid by more
    // than the float32 slack can have no tile.
    const float tx = __fmaf_rn(cam.R[0], dx, __fmaf_rn(cam.R[1], dy, __fmul_rn(cam.R[2], dz)));
    const float ty = __fmaf_rn(cam.R[3], dx, __fmaf_rn(cam.R[4], dy, __fmul_rn(cam.R[5], dz)));
    const float K = nd.K, smax = nd.smax;
    // approximate reciprocal and square roots (relative error ~1e-7, far
    // inside the slack of the test below)
    const float iz = __fdividef(1.0f, tz32);
    const float u = cam.fx * tx * iz + cam.cx, v = cam.fy * ty * iz + cam.cy;
    // a centre inside the tile grid: its support box meets a tile whatever
    // its size (the test below would keep it too)
    if (u >= 0.0f && u < (float)(cam.tiles_x * tile_w) && v >= 0.0f &&
        v < (float)(cam.tiles_y * tile_h))
        return true;
    const float ax = cam.fx * iz, bx = -cam.fx * tx * iz * iz;
    const float ay = cam.fy * iz, by = -cam.fy * ty * iz * iz;
    const float t00 = ax * cam.R[0] + bx * cam.R[6], t01 = ax * cam.R[1] + bx * cam.R[7],
                t02 = ax * cam.R[2] + bx * cam.R[8];
    const float t10 = ay * cam.R[3] + by * cam.R[6], t11 = ay * cam.R[4] + by * cam.R[7],
                t12 = ay * cam.R[5] + by * cam.R[8];
    const float s2 = smax * smax;
    const float qx = K * ((t00 * t00 + t01 * t01 + t02 * t02) * s2 + kBlur);
    const float qy = K * ((t10 * t10 + t11 * t11 + t12 * t12) * s2 + kBlur);
    const float hxb = (qx > 0.0f ? qx * rsqrtf(qx) : 0.0f) * 1.0002f + kRectMargin;
    const float hyb = (qy > 0.0f ? qy * rsqrtf(qy) : 0.0f) * 1.0002f + kRectMargin;
    const float sx = 1e-4f * (fabsf(u) + hxb) + 0.02f, sy = 1e-4f * (fabsf(v) + hyb) + 0.02f;
    if (u + hxb + sx < 0.0f || u - hxb - sx >= (float)(cam.tiles_x * tile_w)) return false;
    if (v + hyb + sy < 0.0f || v - hyb - sy >= (float)(cam.tiles_y * tile_h)) return false;
    return true;
}

// Block-level form of precull: true only if no Gaussian whose mean lies in the
// box lo.xyz..hi.xyz, with scales <= lo.w and 2 ln(255 o) <= hi.w, can pass
// precull for this camera. Depth and the normalised image coordinate
// r = t.x / t.z (linear-fractional, so extreme at box corners when t.z > 0)
// are bounded over the 8 corners; the support half-width is bounded with the
// smallest depth and the largest |T0|^2 = (fx / z)^2 |W0 - r W2|^2 over the r
// range (convex in r); every bound carries slack well above float32 error.
template <typename Cam>
__device__ __forceinline__ bool block_culled(const float4 lo, const float4 hi, const Cam &cam,
                                             int tile_w, int tile_h) {
    float tzmin = INFINITY, tzmax = -INFINITY, dmax = 0.0f;
    float t[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float dx = ((k & 1) ? hi.x : lo.x) - cam.pos[0];
        const float dy = ((k & 2) ? hi.y : lo.y) - cam.pos[1];
        const float dz = ((k & 4) ? hi.z : lo.z) - cam.pos[2];
        t[k][0] = cam.R[0] * dx + cam.R[1] * dy + cam.R[2] * dz;
        t[k][1] = cam.R[3] * dx + cam.R[4] * dy + cam.R[5] * dz;
        t[k][2] = cam.R[6] * dx + cam.R[7] * dy + cam.R[8] * dz;
        tzmin = fminf(tzmin, t[k][2]);
        tzmax = fmaxf(tzmax, t[k][2]);
        dmax = fmaxf(dmax, fabsf(dx) + fabsf(dy) + fabsf(dz));
    }
    const float eps = 4e-6f * dmax + 4e-6f;
    if (tzmax + eps < kNearZ) return true;           // all behind the near plane
    if (tzmin - eps <= 2.0f * kNearZ) return false;  // precull keeps these unconditionally
    float rx0 = INFINITY, rx1 = -INFINITY, ry0 = INFINITY, ry1 = -INFINITY;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float iz = 1.0f / t[k][2];
        rx0 = fminf(rx0, t[k][0] * iz); rx1 = fmaxf(rx1, t[k][0] * iz);
        ry0 = fminf(ry0, t[k][1] * iz); ry1 = fmaxf(ry1, t[k][1] * iz);
    }
    rx0 -= 1e-5f * (fabsf(rx0) + 1.0f); rx1 += 1e-5f * (fabsf(rx1) + 1.0f);
    ry0 -= 1e-5f * (fabsf(ry0) + 1.0f); ry1 += 1e-5f * (fabsf(ry1) + 1.0f);
    const float sK = sqrtf(fmaxf(hi.w, 0.0f)), sig = lo.w;
    const float izmax = 1.0f / (tzmin - eps);
    const float n2 = cam.R[6] * cam.R[6] + cam.R[7] * cam.R[7] + cam.R[8] * cam.R[8];
    {
        const float n0 = cam.R[0] * cam.R[0] + cam.R[1] * cam.R[1] + cam.R[2] * cam.R[2];
        const float d02 = cam.R[0] * cam.R[6] + cam.R[1] * cam.R[7] + cam.R[2] * cam.R[8];
        const float q = fmaxf(n0 - 2.0f * rx0 * d02 + rx0 * rx0 * n2,
                              n0 - 2.0f * rx1 * d02 + rx1 * rx1 * n2);
        const float H = (sK * sig * cam.fx * izmax * sqrtf(fmaxf(q, 0.0f)) + sqrtf(kBlur) * sK) *
                            1.001f + kRectMargin + 0.05f;
        const float umin = cam.fx * rx0 + cam.cx, umax = cam.fx * rx1 + cam.cx;
        const float sl = 1e-4f * (fmaxf(fabsf(umin), fabsf(umax)) + H) + 0.05f;
        if (umax + H + sl < 0.0f) return true;
        if (umin - H - sl >= (float)(cam.tiles_x * tile_w)) return true;
    }
    {
        const float n1 = cam.R[3] * cam.R[3] + cam.R[4] * cam.R[4] + cam.R[5] * cam.R[5];
        const float d12 = cam.R[3] * cam.R[6] + cam.R[4] * cam.R[7] + cam.R[5] * cam.R[8];
        const float q = fmaxf(n1 - 2.0f * ry0 * d12 + ry0 * ry0 * n2,
                              n1 - 2.0f * ry1 * d12 + ry1 * ry1 * n2);
        const float H = (sK * sig * cam.fy * izmax * sqrtf(fmaxf(q, 0.0f)) + sqrtf(kBlur) * sK) *
                            1.001f + kRectMargin + 0.05f;
        const float vmin = cam.fy * ry0 + cam.cy, vmax = cam.fy * ry1 + cam.cy;
        const float sl = 1e-4f * (fmaxf(fabsf(vmin), fabsf(vmax)) + H) + 0.05f;
        if (vmax + H + sl < 0.0f) return true;
        if (vmin - H - sl >= (float)(cam.tiles_y * tile_h)) return true;
    }
    return false;
}

// Error-free transformations (Knuth's TwoSum; the product's error by a fused
// multiply-add): s + e = a + b and p + e = a b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// R . (hi + lo) as a compensated dot product (the sum of the rounded terms
// with the running rounding errors added back): close to a faithful rounding
// of the exact value, however much the three terms cancel.
__device__ __forceinline__ float dot3_compensated(const float *R, const float hi[3],
                                                  const float lo[3]) {
    float s, c, p, e, q;
    two_prod(R[0], hi[0], s, c);
    two_prod(R[1], hi[1], p, e);
    two_sum(s, p, s, q);
    c = __fadd_rn(c, __fadd_rn(q, e));
    two_prod(R[2], hi[2], p, e);
    two_sum(s, p, s, q);
    c = __fadd_rn(c, __fadd_rn(q, e));
    c = __fmaf_rn(R[0], lo[0], __fmaf_rn(R[1], lo[1], __fmaf_rn(R[2], lo[2], c)));
    return __fadd_rn(s, c);
}

constexpr float kHalfLog2e = 0.72134752044448170f;   // log2(e) / 2

// Full preprocess of a Gaussian that passed precull (phase B); returns whether// Full preprocess of a Gaussian that passed precull (phase B); returns whether
// it is visible (in front of the near plane and touching at least one tile).
// kBlend: the node is rendered with its level-of-detail blended attributes
// (moved toward its parent's by blend_parent_weight): mean and opacity in one
// fused step each, covariance and SH coefficients element by element.
template <typename A, bool kBlend = false>
__device__ __forceinline__ bool preprocess_one(const SceneDev &sc, const DevCamera &cam,
                                               uint32_t node, int tile_w, int tile_h,
                                               PreOut &o) {
    float4 p = sc.pos4[node];
    float vb = 0.0f;   // parent weight of the blend
    int par = -1;
    if (kBlend) {
        const float4 lo = sc.box_lo[node], hi = sc.box_hi[node];
        par = __float_as_int(lo.w);
        if (par >= 0)
            vb = blend_parent_weight(
                granularity(lo, hi, cam.pos[0], cam.pos[1], cam.pos[2], cam.fx),
                granularity(sc.box_lo[par], sc.box_hi[par], cam.pos[0], cam.pos[1], cam.pos[2],
                            cam.fx),
                cam.tau);
    }
    const bool mix = kBlend && vb > 0.0f;
    float sp[4];
    if (mix) {
        const float4 pp = sc.pos4[par];
        p.x = __fmaf_rn(vb, __fsub_rn(pp.x, p.x), p.x);
        p.y = __fmaf_rn(vb, __fsub_rn(pp.y, p.y), p.y);
        p.z = __fmaf_rn(vb, __fsub_rn(pp.z, p.z), p.z);
        Attr<A>::load4(sc.sop, par, sp);
    }
    const float dx = __fsub_rn(p.x, cam.pos[0]);
    const float dy = __fsub_rn(p.y, cam.pos[1]);
    const float dz = __fsub_rn(p.z, cam.pos[2]);
    const float tx = __fmaf_rn(cam.R[0], dx, __fmaf_rn(cam.R[1], dy, __fmul_rn(cam.R[2], dz)));
    const float ty = __fmaf_rn(cam.R[3], dx, __fmaf_rn(cam.R[4], dy, __fmul_rn(cam.R[5], dz)));
    float so[4];
    Attr<A>::load4(sc.sop, node, so);
    float opac = so[3];
    if (mix) opac = __fmaf_rn(vb, __fsub_rn(sp[3], opac), opac);
    // without blending, nodes with 255 o < 1 never get here (load-time flag)
    if (kBlend && !(255.0f * opac >= 1.0f)) return false;
    const float K = 2.0f * logf(255.0f * opac);
    // view depth in the fixed float32 operation sequence that the near-plane
    // cull and the sort key use
    const float tz = __fmaf_rn(cam.R[6], dx, __fmaf_rn(cam.R[7], dy, __fmul_rn(cam.R[8], dz)));
    if (!(tz > kNearZ)) return false;
    // The view vector of the projection. Close to the camera plane and far off
    // the axis (sum_k |R_2k d_k| > 8 t_z) the depth is a sum that cancels, and
    // its rounding would turn the footprint of the (then very elongated)
    // Gaussian; there it is recomputed from the exact differences with
    // compensated products.
    float txp = tx, typ = ty, tzp = tz;
    if (fabsf(cam.R[6] * dx) + fabsf(cam.R[7] * dy) + fabsf(cam.R[8] * dz) > 8.0f * tz) {
        float hi[3], lo[3];
        two_sum(p.x, -cam.pos[0], hi[0], lo[0]);
        two_sum(p.y, -cam.pos[1], hi[1], lo[1]);
        two_sum(p.z, -cam.pos[2], hi[2], lo[2]);
        txp = dot3_compensated(cam.R, hi, lo);
        typ = dot3_compensated(cam.R + 3, hi, lo);
        tzp = dot3_compensated(cam.R + 6, hi, lo);
    }

    // 3D covariance from the normalised quaternion and the scales
    const float4 q4 = sc.quat[node];
    const float qn = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
    const float w = q4.x * qn, x = q4.y * qn, y = q4.z * qn, z = q4.w * qn;
    const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z),
                R02 = 2.f * (x * z + w * y);
    const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z),
                R12 = 2.f * (y * z - w * x);
    const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x),
                R22 = 1.f - 2.f * (x * x + y * y);
    const float s0 = expf(so[0]), s1 = expf(so[1]), s2 = expf(so[2]);
    const float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
    const float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
    const float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
    float S00 = M00 * M00 + M01 * M01 + M02 * M02;
    float S01 = M00 * M10 + M01 * M11 + M02 * M12;
    float S02 = M00 * M20 + M01 * M21 + M02 * M22;
    float S11 = M10 * M10 + M11 * M11 + M12 * M12;
    float S12 = M10 * M20 + M11 * M21 + M12 * M22;
    float S22 = M20 * M20 + M21 * M21 + M22 * M22;
    if (mix) {
        float Sp[6];
        cov3d(sc.quat[par], sp, Sp);
        S00 = __fmaf_rn(vb, __fsub_rn(Sp[0], S00), S00);
        S01 = __fmaf_rn(vb, __fsub_rn(Sp[1], S01), S01);
        S02 = __fmaf_rn(vb, __fsub_rn(Sp[2], S02), S02);
        S11 = __fmaf_rn(vb, __fsub_rn(Sp[3], S11), S11);
        S12 = __fmaf_rn(vb, __fsub_rn(Sp[4], S12), S12);
        S22 = __fmaf_rn(vb, __fsub_rn(Sp[5], S22), S22);
    }

    // T = J W (2x3): rows (fx/z) W0 - (fx x/z^2) W2 and (fy/z) W1 - (fy y/z^2) W2
    const float iz = 1.0f / tzp;
    const float ax = cam.fx * iz, bx = -cam.fx * txp * iz * iz;
    const float ay = cam.fy * iz, by = -cam.fy * typ * iz * iz;
    const float T00 = ax * cam.R[0] + bx * cam.R[6], T01 = ax * cam.R[1] + bx * cam.R[7],
                T02 = ax * cam.R[2] + bx * cam.R[8];
    const float T10 = ay * cam.R[3] + by * cam.R[6], T11 = ay * cam.R[4] + by * cam.R[7],
                T12 = ay * cam.R[5] + by * cam.R[8];
    float ca, cb, cc, det;
    if (!mix) {
        // Sigma2D - 0.3 I = M diag(s^2) M^T with M = T Rq: the projections of the
        // Gaussian's axes, summed as positive squares; det by Cauchy-Binet,
        // sum over axis pairs of (s_i s_j)^2 (minor of M)^2, each minor being
        // n . (axis k) for the normal n = T0 x T1 taken from the camera's row
        // cross products (the rows of T are nearly parallel for a Gaussian
        // far off the axis, so neither a c - b^2 nor T0 x T1 is formed)
        const float m00 = T00 * R00 + T01 * R10 + T02 * R20;
        const float m01 = T00 * R01 + T01 * R11 + T02 * R21;
        const float m02 = T00 * R02 + T01 * R12 + T02 * R22;
        const float m10 = T10 * R00 + T11 * R10 + T12 * R20;
        const float m11 = T10 * R01 + T11 * R11 + T12 * R21;
        const float m12 = T10 * R02 + T11 * R12 + T12 * R22;
        const float q00 = s0 * m00, q01 = s1 * m01, q02 = s2 * m02;
        const float q10 = s0 * m10, q11 = s1 * m11, q12 = s2 * m12;
        const float ap = q00 * q00 + q01 * q01 + q02 * q02;
        const float cp = q10 * q10 + q11 * q11 + q12 * q12;
        cb = q00 * q10 + q01 * q11 + q02 * q12;
        const float aa = ax * ay, ab = ax * by, ba = bx * ay;
        const float n0 = aa * cam.X01[0] + ab * cam.X02[0] + ba * cam.X21[0];
        const float n1 = aa * cam.X01[1] + ab * cam.X02[1] + ba * cam.X21[1];
        const float n2 = aa * cam.X01[2] + ab * cam.X02[2] + ba * cam.X21[2];
        const float g0 = s1 * s2 * (n0 * R00 + n1 * R10 + n2 * R20);
        const float g1 = s0 * s2 * (n0 * R01 + n1 * R11 + n2 * R21);
        const float g2 = s0 * s1 * (n0 * R02 + n1 * R12 + n2 * R22);
        ca = ap + kBlur;
        cc = cp + kBlur;
        det = g0 * g0 + g1 * g1 + g2 * g2 + kBlur * (ap + cp) + kBlur * kBlur;
    } else {
        // U = T Sigma for the blended covariance
        const float U00 = T00 * S00 + T01 * S01 + T02 * S02;
        const float U01 = T00 * S01 + T01 * S11 + T02 * S12;
        const float U02 = T00 * S02 + T01 * S12 + T02 * S22;
        const float U10 = T10 * S00 + T11 * S01 + T12 * S02;
        const float U11 = T10 * S01 + T11 * S11 + T12 * S12;
        const float U12 = T10 * S02 + T11 * S12 + T12 * S22;
        ca = U00 * T00 + U01 * T01 + U02 * T02 + kBlur;
        cb = U00 * T10 + U01 * T11 + U02 * T12;
        cc = U10 * T10 + U11 * T11 + U12 * T12 + kBlur;
        det = ca * cc - cb * cb;
    }
    if (!(det > 0.0f)) return false;
    const float u = __fmaf_rn(cam.fx * iz, txp, cam.cx);
    const float v = __fmaf_rn(cam.fy * iz, typ, cam.cy);

    // support box and tile rectangle
    const float hx = sqrtf(K * ca) + kRectMargin;
    const float hy = sqrtf(K * cc) + kRectMargin;
    const float itw = 1.0f / (float)tile_w, ith = 1.0f / (float)tile_h;
    int x0 = (int)floorf((u - hx) * itw), x1 = (int)floorf((u + hx) * itw);
    int y0 = (int)floorf((v - hy) * ith), y1 = (int)floorf((v + hy) * ith);
    x0 = max(x0, 0); y0 = max(y0, 0);
    x1 = min(x1, cam.tiles_x - 1); y1 = min(y1, cam.tiles_y - 1);
    if (x0 > x1 || y0 > y1) return false;

    // colour seen along camera -> mean
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    float rgb[3];
    if (mix) sh_colour_blend<A>(sc.sh, node, par, vb, dx * inv, dy * inv, dz * inv, rgb);
    else sh_colour<A>(sc.sh, node, dx * inv, dy * inv, dz * inv, rgb);

    // Cholesky factors of the conic (c, -b; -b, a) / det, scaled by
    // sqrt(log2(e) / 2): F1 = sqrt(k c / det), F2 = -b sqrt(k / (c det)),
    // F3 = sqrt(k / c)
    const float sdet = sqrtf(det);
    const float F3 = sqrtf(kHalfLog2e / cc);
    o.x = u;
    o.y = v;
    o.F1 = F3 * cc / sdet;
    o.F2 = -cb * F3 / sdet;
    o.F3 = F3;
    o.L = log2f(opac);
    o.r = rgb[0]; o.g = rgb[1]; o.bl = rgb[2];
    o.hx = hx; o.hy = hy;
    o.key = __float_as_uint(tz);
    o.rx0 = (uint32_t)x0; o.ry0 = (uint32_t)y0;
    o.rx1 = (uint32_t)x1; o.ry1 = (uint32_t)y1;
    return true;
}

__device__ __forceinline__ void store_rec(Rec32 *rec, int64_t i, const PreOut &o) {
    rec[i].a = make_float4(o.x, o.y, o.F1, o.F2);
    rec[i].b = make_float4(o.F3, o.L, o.r, o.g);
    rec[i].c = make_float4(o.bl, o.hx, o.hy, 0.f);
}
__device__ __forceinline__ void store_rec(Rec16 *rec, int64_t i, const PreOut &o) {
    const __half2 rg = __floats2half2_rn(o.r, o.g);
    const __half2 b0 = __halves2half2(__float2half_rn(o.bl), __float2half_ru(fmaxf(o.hx, o.hy)));
    rec[i].a = make_float4(o.x, o.y, o.F1, o.F2);
    rec[i].b = make_float4(o.F3, o.L, __uint_as_float(*reinterpret_cast<const uint32_t *>(&rg)),
                           __uint_as_float(*reinterpret_cast<const uint32_t *>(&b0)));
}

// Live partitions: the (node block, camera) pairs that survive the block-level
// cull, appended to part_list, and grouped: a group is a run of up to
// kGroupCams live partitions of the same node block (one half-warp's chunk of
// cameras), recorded as (first entry, count) in group_list. Groups come out
// block-major, so groups running at the same time mostly read the same node
// block through L2. Culled partitions get an empty entry in the partition
// table.
constexpr int kGroupCams = 16;

__global__ void k_live_parts(SceneDev sc, const DevCamera *__restrict__ cams, int n_cams,
                             int64_t nblk, uint32_t *__restrict__ part_list,
                             uint2 *__restrict__ group_list, uint2 *__restrict__ part_info,
                             uint32_t *counters, int tile_w, int tile_h, int use_block_cull,
                             int blend, const int *err) {
    // with level-of-detail blending a node's Gaussian may move toward its
    // parent: the bounds then cover the block's nodes and their parents
    const float4 *__restrict__ blo = blend ? sc.blk_lo_b : sc.blk_lo;
    const float4 *__restrict__ bhi = blend ? sc.blk_hi_b : sc.blk_hi;
    if (*err) return;
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int64_t nch = (n_cams + kGroupCams - 1) / kGroupCams;
    const int64_t nq = nblk * nch;   // (block, chunk of kGroupCams cameras)
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q0 = 2 * (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5); q0 < nq;
         q0 += 2 * warps) {
        const int64_t q = q0 + half;
        bool live = false;
        uint32_t t = 0;
        if (q < nq) {
            const int64_t b = q / nch;
            const int c = (int)(q - b * nch) * kGroupCams + hl;
            if (c < n_cams) {
                t = (uint32_t)(b * n_cams + c);
                live = !(use_block_cull && block_culled(blo[b], bhi[b], cams[c], tile_w, tile_h));
                if (!live) part_info[(int64_t)c * nblk + b] = make_uint2(0u, 0u);
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, live);
        const uint32_t n_lo = __popc(bal & 0xffffu), n_hi = __popc(bal >> 16);
        uint32_t base = 0, gbase = 0;
        if (lane == 0 && bal) {
            base = atomicAdd(&counters[CNT_LIVE], (uint32_t)__popc(bal));
            gbase = atomicAdd(&counters[CNT_GROUPS], (n_lo ? 1u : 0u) + (n_hi ? 1u : 0u));
            if (n_lo) group_list[gbase++] = make_uint2(base, n_lo);
            if (n_hi) group_list[gbase] = make_uint2(base + n_lo, n_hi);
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if (live) part_list[base + __popc(bal & lanemask_lt())] = t;
    }
}

// Fused cut + preprocess over groups of live partitions (one node block and up
// to kGroupCams cameras), taken from an atomic ticket.
//  - Phase A loads each node's box, parent box, position and scale/opacity
//    once for the whole group and applies the cut rule and the conservative
//    cull for every camera of it (one ballot per camera, item and warp).
//  - The (node, camera) candidates of the group are listed node-major, and
//    each partition takes output space for its candidates with one atomic; a
//    candidate's slot is its rank among its camera's candidates in node order.
//  - Phase B preprocesses the list densely (neighbouring entries mostly share a
//    node, so its attributes are read once into L1) and writes each result
//    straight to its slot; a candidate that turns out invisible leaves its
//    slot with the key kKeyHole, which the key gather skips.
//  - Per partition: (first slot, visible | candidates << 16) in part_info.
constexpr uint32_t kKeyHole = 0xffffffffu;   // a NaN pattern: never a depth key

template <typename R>
struct CutPreSmem {
    uint16_t ent[kGroupCams * kPrePart];        // node-major candidates: node << 4 | camera
    uint32_t balw[kGroupCams][kPreItems * 8];   // candidate ballot per (camera, item, warp)
    uint32_t cex[kGroupCams][kPreItems * 8];    // candidates of the camera before (item, warp)
    unsigned long long off[kGroupCams];         // first slot of each camera's partition
    uint32_t ncand[kGroupCams], nvis[kGroupCams], sel[kGroupCams];
    CamLite cam[kGroupCams];
    uint32_t gcam[kGroupCams];
    uint32_t wsum[kPreThreads / 32];
    uint32_t goff, gcnt;
};
static_assert(kGroupCams <= 16 && kPrePart <= 4096, "entries pack node and camera in 16 bits");

template <typename A, typename R, bool kBlend>
__global__ void __launch_bounds__(kPreThreads, kBlend ? 3 : 0)
k_cutpre(SceneDev sc, const DevCamera *__restrict__ cams, int n_cams, R *__restrict__ rec,
         int64_t rec_cap, uint32_t *__restrict__ dkey, uint2 *__restrict__ rect,
         uint32_t *__restrict__ node_out,
         uint32_t *__restrict__ vis_count, uint32_t *counters,
         const uint32_t *__restrict__ part_list, const uint2 *__restrict__ group_list,
         uint2 *__restrict__ part_info, int *err, int tile_w, int tile_h) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CutPreSmem<R> &S = *reinterpret_cast<CutPreSmem<R> *>(smem_raw);
    if (*err) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nblk = (sc.n + kPrePart - 1) / kPrePart;
    const uint32_t n_groups = counters[CNT_GROUPS];
    unsigned long long *alloc = reinterpret_cast<unsigned long long *>(counters + CNT_ALLOC);
    for (;;) {
        if (tid == 0) {
            const uint32_t i = atomicAdd(&counters[TK_PRE], 1u);
            const uint2 g = i < n_groups ? group_list[i] : make_uint2(0u, 0u);
            S.goff = g.x;
            S.gcnt = g.y;
        }
        __syncthreads();
        const int gcnt = (int)S.gcnt;
        if (gcnt == 0) break;
        const uint32_t goff = S.goff;
        const int64_t b = part_list[goff] / (uint32_t)n_cams;
        if (tid < gcnt) {
            const int c = (int)(part_list[goff + tid] - b * n_cams);
            const DevCamera &d = cams[c];
            CamLite &l = S.cam[tid];
            for (int k = 0; k < 9; ++k) l.R[k] = d.R[k];
            l.pos[0] = d.pos[0]; l.pos[1] = d.pos[1]; l.pos[2] = d.pos[2];
            l.fx = d.fx; l.fy = d.fy; l.cx = d.cx; l.cy = d.cy; l.tau = d.tau;
            l.tau2 = __fmul_rn(d.tau, d.tau);
            l.tiles_x = d.tiles_x; l.tiles_y = d.tiles_y;
            S.gcam[tid] = (uint32_t)c;
            S.sel[tid] = 0;
            S.nvis[tid] = 0;
        }
        __syncthreads();
        // phase A: per node, one set of loads for every camera of the group;
        // mask[k]: the cameras for which node k of this thread is a candidate
        uint32_t mask[kPreItems];
#pragma unroll 1
        for (int k = 0; k < kPreItems; ++k) {
            const int64_t node = b * kPrePart + k * kPreThreads + tid;
            const bool valid = node < sc.n;
            float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo, plo = lo, phi = lo;
            NodeCull nd;
            nd.p = lo;
            float so[4] = {1.f, 1.f, 1.f, 1.f};
            if (valid) {
                lo = sc.box_lo[node];
                hi = sc.box_hi[node];
                nd.p = sc.pos4[node];
                Attr<A>::load4(sc.sop, node, so);
            }
            const int par = __float_as_int(lo.w);
            const bool leaf = __float_as_int(hi.w) == 0;
            if (valid && par >= 0) {
                plo = sc.box_lo[par];
                phi = sc.box_hi[par];
            }
            nd.K = 2.0f * logf(255.0f * so[3]);
            nd.smax = expf(fmaxf(fmaxf(so[0], so[1]), so[2]));
            // blending: the Gaussian's mean lies on the segment from the node's
            // mean to its parent's, its scale and opacity below the larger of
            // the two; the box of that segment with those bounds is tested
            // like a block of means (conservative)
            float4 seg_lo = nd.p, seg_hi = nd.p;
            bool seg_dead = false;
            if (kBlend) {
                float K = 255.0f * so[3] >= 1.0f ? nd.K : -INFINITY;
                float smax = nd.smax;
                if (valid && par >= 0) {
                    const float4 pp = sc.pos4[par];
                    float sq[4];
                    Attr<A>::load4(sc.sop, par, sq);
                    seg_lo = make_float4(fminf(nd.p.x, pp.x), fminf(nd.p.y, pp.y),
                                         fminf(nd.p.z, pp.z), 0.f);
                    seg_hi = make_float4(fmaxf(nd.p.x, pp.x), fmaxf(nd.p.y, pp.y),
                                         fmaxf(nd.p.z, pp.z), 0.f);
                    if (255.0f * sq[3] >= 1.0f) K = fmaxf(K, 2.0f * logf(255.0f * sq[3]));
                    smax = fmaxf(smax, expf(fmaxf(fmaxf(sq[0], sq[1]), sq[2])));
                }
                seg_dead = !(K >= 0.0f);   // opacity below 1/255 at both ends
                seg_lo.w = smax * (1.0f + 1e-5f);
                seg_hi.w = K * (1.0f + 1e-5f) + 1e-6f;
            }
            // the boxes' extents do not depend on the camera
            const float ext_n = box_extent(lo, hi), ext_p = box_extent(plo, phi);
            uint32_t m = 0;
            for (int i = 0; i < gcnt; ++i) {
                const CamLite &cam = S.cam[i];
                const bool sel =
                    valid &&
                    (leaf || fine_enough_pre(lo, hi, ext_n, cam.pos[0], cam.pos[1], cam.pos[2],
                                             cam.fx, cam.tau2)) &&
                    (par < 0 || !fine_enough_pre(plo, phi, ext_p, cam.pos[0], cam.pos[1],
                                                 cam.pos[2], cam.fx, cam.tau2));
                const bool cand =
                    sel && (kBlend ? !seg_dead && !block_culled(seg_lo, seg_hi, cam, tile_w, tile_h)
                                   : precull(cam, nd, tile_w, tile_h));
                m |= cand ? 1u << i : 0u;
                const uint32_t nsel = __popc(__ballot_sync(0xffffffffu, sel));
                const uint32_t bal = __ballot_sync(0xffffffffu, cand);
                if (lane == 0) {
                    S.balw[i][k * 8 + warp] = bal;
                    if (nsel) atomicAdd(&S.sel[i], nsel);
                }
            }
            mask[k] = m;
        }
        __syncthreads();
        // per camera: candidates before each (item, warp) in node order, and
        // the partition's output space
        for (int i = warp; i < gcnt; i += kPreThreads / 32) {
            const uint32_t v = lane < kPreItems * 8 ? __popc(S.balw[i][lane]) : 0u;
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane < kPreItems * 8) S.cex[i][lane] = incl - v;
            if (lane == 31) {
                S.ncand[i] = incl;
                unsigned long long off = 0;
                if (incl) {
                    off = atomicAdd(alloc, (unsigned long long)incl);
                    if (off + incl > (unsigned long long)rec_cap) latch_error(err, kErrCapacity);
                }
                S.off[i] = off;
            }
        }
        // node-major entry list: node v = k * kPreThreads + tid has popc(mask[k])
        // entries, one per candidate camera in camera order
        uint32_t base = 0;
#pragma unroll
        for (int k = 0; k < kPreItems; ++k) {
            const uint32_t v = __popc(mask[k]);
            uint32_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) S.wsum[warp] = incl;
            __syncthreads();
            uint32_t wb = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < kPreThreads / 32; ++w) {
                if (w < warp) wb += S.wsum[w];
                tot += S.wsum[w];
            }
            uint32_t e = base + wb + incl - v;
            const uint32_t nodev = (uint32_t)(k * kPreThreads + tid);
            for (uint32_t mm = mask[k]; mm; mm &= mm - 1)
                S.ent[e++] = (uint16_t)((nodev << 4) | (uint32_t)(__ffs(mm) - 1));
            base += tot;
            __syncthreads();   // S.wsum is reused by the next item
        }
        const int nent = (int)base;
        // phase B: preprocess every (node, camera) candidate straight into its slot
        for (int e = tid; e < nent; e += kPreThreads) {
            const uint32_t en = S.ent[e];
            const int i = (int)(en & 15u);
            const uint32_t v = en >> 4;
            const int k = (int)(v / kPreThreads), w = (int)((v % kPreThreads) >> 5),
                      l = (int)(v & 31u);
            const uint32_t rank = S.cex[i][k * 8 + w] + __popc(S.balw[i][k * 8 + w] & ((1u << l) - 1u));
            const unsigned long long pos = S.off[i] + rank;
            if (pos >= (unsigned long long)rec_cap) continue;   // capacity already latched
            const int c = (int)S.gcam[i];
            PreOut o;
            const uint32_t node = (uint32_t)(b * kPrePart + v);
            if (preprocess_one<A, kBlend>(sc, cams[c], node, tile_w, tile_h, o)) {
                store_rec(rec, (int64_t)pos, o);
                dkey[pos] = o.key;
                rect[pos] = pack_rect(o.rx0, o.ry0, o.rx1, o.ry1, (uint32_t)c);
                if (node_out) node_out[pos] = node;
                atomicAdd(&S.nvis[i], 1u);
            } else {
                dkey[pos] = kKeyHole;
            }
        }
        __syncthreads();
        if (tid < gcnt) {
            const int c = (int)S.gcam[tid];
            const uint32_t nv = S.nvis[tid];
            part_info[(int64_t)c * nblk + b] =
                make_uint2((uint32_t)min(S.off[tid], (unsigned long long)rec_cap),
                           nv | (S.ncand[tid] << 16));
            if (nv) atomicAdd(&vis_count[c], nv);
            if (S.sel[tid]) atomicAdd(&counters[CNT_CUT], S.sel[tid]);
        }
        __syncthreads();
    }
}

// Dense depth-sort input, part 1: per camera (one CTA each), the position of
// every partition's first record in the camera-major, node-order sequence;
// block 0 also stores the visible total.
__global__ void __launch_bounds__(1024)
k_part_scan(const uint32_t *__restrict__ vis_count, int n_cams, int64_t nblk,
            const uint2 *__restrict__ part_info, uint32_t *__restrict__ part_pos,
            uint32_t *counters, int64_t cap, int *err) {
    __shared__ uint32_t s_w[32];
    __shared__ uint32_t s_base, s_total;
    if (*err) return;
    const int c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // exclusive scan of the (at most 1024) per-camera counts
    auto block_scan = [&](uint32_t v, uint32_t &total) -> uint32_t {
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncthreads();
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        uint32_t wb = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < warp) wb += s_w[w];
            tot += s_w[w];
        }
        total = tot;
        return wb + incl - v;
    };
    uint32_t tot;
    const uint32_t ex = block_scan(tid < n_cams ? vis_count[tid] : 0u, tot);
    if (tid == c) s_base = ex;
    if (tid == 0) s_total = tot;
    __syncthreads();
    if (c == 0 && tid == 0) {
        counters[CNT_VIS] = s_total;
        if ((int64_t)s_total > cap) latch_error(err, kErrCapacity);
    }
    uint32_t carry = s_base;
    for (int64_t b0 = 0; b0 < nblk; b0 += 1024) {
        const int64_t b = b0 + tid;
        const uint32_t n = b < nblk ? part_info[(int64_t)c * nblk + b].y & 0xffffu : 0u;
        uint32_t chunk;
        const uint32_t e = block_scan(n, chunk);
        if (b < nblk) part_pos[(int64_t)c * nblk + b] = carry + e;
        carry += chunk;
    }
}

// Dense depth-sort input, part 2: one warp per live partition copies the keys
// of its visible Gaussians (skipping holes) and writes their record indices at
// the partition's dense position. On the
// way it counts the digit histograms of the four 8-bit passes of the depth
// sort into hist[4][256] (zeroed beforehand): positive float depths share
// their high digits, so a warp whose keys agree on a digit adds its count once
// instead of contending on one shared-memory counter.
__global__ void __launch_bounds__(256)
k_part_gather(const uint32_t *__restrict__ part_list, int n_cams, int64_t nblk,
              const uint2 *__restrict__ part_info, const uint32_t *__restrict__ part_pos,
              const uint32_t *__restrict__ dkey_sparse, uint32_t *__restrict__ dkey,
              uint32_t *__restrict__ didx, const uint32_t *counters, int64_t cap,
              uint32_t *hist, const int *err) {
    __shared__ uint32_t s_h[4][256];
    if (*err) return;
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * 256; i += blockDim.x) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const uint32_t n_live = counters[CNT_LIVE];
    const int lane = tid & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + tid) >> 5; i < n_live; i += nw) {
        const uint32_t t = part_list[i];
        const uint32_t b = t / (uint32_t)n_cams, c = t - b * (uint32_t)n_cams;
        const int64_t idx = (int64_t)c * nblk + b;
        const uint2 info = part_info[idx];
        const uint32_t ncand = info.y >> 16;
        int64_t pos = part_pos[idx];
        // the partition's slots hold its candidates in node order; the visible
        // ones are packed to their dense positions, holes are skipped. Four
        // rows of 32 slots are requested at once (one memory round trip), then
        // packed row by row. Uniform trip count: every lane reaches the warp
        // collectives
        constexpr int kRows = 4;
        for (uint32_t k0 = 0; k0 < ncand; k0 += 32 * kRows) {
            uint32_t keys[kRows];
#pragma unroll
            for (int u = 0; u < kRows; ++u) {
                const uint32_t k = k0 + 32 * u + lane;
                keys[u] = kKeyHole;
                if (k < ncand && (int64_t)info.x + k < cap) keys[u] = dkey_sparse[info.x + k];
            }
#pragma unroll
            for (int u = 0; u < kRows; ++u) {
                const uint32_t k = k0 + 32 * u + lane;
                const uint32_t key = keys[u];
                const bool vis = key != kKeyHole;
                const uint32_t vb = __ballot_sync(0xffffffffu, vis);
                const int64_t dst = pos + __popc(vb & lanemask_lt());
                const bool valid = vis && dst < cap;
                if (valid) {
                    dkey[dst] = key;
                    didx[dst] = info.x + k;
                }
                pos += __popc(vb);
                const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
                if (vmask) {
                    const int leader = __ffs(vmask) - 1;
#pragma unroll
                    for (int qd = 0; qd < 4; ++qd) {
                        const uint32_t d = (key >> (8 * qd)) & 255u;
                        const uint32_t dl = __shfl_sync(0xffffffffu, d, leader);
                        if (__all_sync(0xffffffffu, !valid || d == dl)) {
                            if (lane == leader) atomicAdd(&s_h[qd][d], (uint32_t)__popc(vmask));
                        } else if (valid) {
                            atomicAdd(&s_h[qd][d], 1u);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < 4 * 256; i += blockDim.x) {
        const uint32_t v = (&s_h[0][0])[i];
        if (v) atomicAdd(&hist[i], v);
    }
}

template <bool kBlend>
static void launch_cutpre_t(const SceneDev &sc, const DevCamera *cams, int n_cams, void *rec,
                            int64_t rec_cap, uint32_t *dkey_sparse, uint2 *rect,
                            uint32_t *node_id, uint32_t *vis_count, uint32_t *counters,
                            uint32_t *part_list,
                            uint2 *group_list, uint2 *part_info, int *err, int tile_w, int tile_h,
                            int grid, cudaStream_t st) {
    switch (sc.attr_dtype) {
    case NGS_F16:
        k_cutpre<__half, Rec16, kBlend><<<grid, kPreThreads, sizeof(CutPreSmem<Rec16>), st>>>(
            sc, cams, n_cams, (Rec16 *)rec, rec_cap, dkey_sparse, rect, node_id, vis_count,
            counters, part_list, group_list, part_info, err, tile_w, tile_h);
        break;
    case NGS_BF16:
        k_cutpre<__nv_bfloat16, Rec16, kBlend>
            <<<grid, kPreThreads, sizeof(CutPreSmem<Rec16>), st>>>(
                sc, cams, n_cams, (Rec16 *)rec, rec_cap, dkey_sparse, rect, node_id, vis_count,
                counters, part_list, group_list, part_info, err, tile_w, tile_h);
        break;
    default:
        k_cutpre<float, Rec32, kBlend><<<grid, kPreThreads, sizeof(CutPreSmem<Rec32>), st>>>(
            sc, cams, n_cams, (Rec32 *)rec, rec_cap, dkey_sparse, rect, node_id, vis_count,
            counters, part_list, group_list, part_info, err, tile_w, tile_h);
        break;
    }
}

void launch_cutpre(const SceneDev &sc, const DevCamera *cams, int n_cams, void *rec,
                   int64_t rec_cap, uint32_t *dkey_sparse, uint2 *rect, uint32_t *node_id,
                   uint32_t *vis_count, uint32_t *counters, uint32_t *part_list,
                   uint2 *group_list, uint2 *part_info,
                   int *err, int tile_w, int tile_h, int use_block_cull, int blend, int grid,
                   cudaStream_t st) {
    const int64_t nblk = (sc.n + kPrePart - 1) / kPrePart;
    cudaMemsetAsync(vis_count, 0, (size_t)n_cams * sizeof(uint32_t), st);
    const int64_t nq = nblk * ((n_cams + kGroupCams - 1) / kGroupCams);
    // 8 warps per CTA, two (block, camera chunk) items per warp and iteration
    const int lgrid = (int)std::min<int64_t>((nq + 15) / 16, 8 * 1024);
    k_live_parts<<<std::max(lgrid, 1), 256, 0, st>>>(sc, cams, n_cams, nblk, part_list,
                                                     group_list, part_info, counters, tile_w,
                                                     tile_h, use_block_cull, blend, err);
    if (blend)
        launch_cutpre_t<true>(sc, cams, n_cams, rec, rec_cap, dkey_sparse, rect, node_id,
                              vis_count, counters, part_list, group_list, part_info, err,
                              tile_w, tile_h, grid, st);
    else
        launch_cutpre_t<false>(sc, cams, n_cams, rec, rec_cap, dkey_sparse, rect, node_id,
                               vis_count, counters, part_list, group_list, part_info, err,
                               tile_w, tile_h, grid, st);
}

void launch_gather_keys(const uint32_t *vis_count, int n_cams, const SceneDev &sc,
                        const uint2 *part_info, uint32_t *part_pos, const uint32_t *part_list,
                        const uint32_t *dkey_sparse, uint32_t *dkey, uint32_t *didx,
                        uint32_t *counters, int64_t cap, uint32_t *hist, int *err, int grid,
                        cudaStream_t st) {
    const int64_t nblk = (sc.n + kPrePart - 1) / kPrePart;
    k_part_scan<<<n_cams, 1024, 0, st>>>(vis_count, n_cams, nblk, part_info, part_pos, counters,
                                         cap, err);
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 4 * 256, st);
    k_part_gather<<<grid, 256, 0, st>>>(part_list, n_cams, nblk, part_info, part_pos, dkey_sparse,
                                        dkey, didx, counters, cap, hist, err);
}

int cutpre_partition_nodes() { return kPrePart; }

template <bool kBlend>
static void cutpre_attr() {
    cudaFuncSetAttribute(k_cutpre<float, Rec32, kBlend>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(CutPreSmem<Rec32>));
    cudaFuncSetAttribute(k_cutpre<__half, Rec16, kBlend>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(CutPreSmem<Rec16>));
    cudaFuncSetAttribute(k_cutpre<__nv_bfloat16, Rec16, kBlend>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(CutPreSmem<Rec16>));
}

void cutpre_init_attributes() {
    cutpre_attr<false>();
    cutpre_attr<true>();
}

}  // namespace ngs
