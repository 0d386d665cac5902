// K7: per-tile front-to-back alpha compositing (3DGS rasterisation as used by
// the H3DGS engine, Sec. III-A/III-B).
//
// One CTA renders one tile (TW x TH threads, one pixel each). The tile's
// Gaussians, in (depth, node id) order, are staged in shared memory BATCH
// records at a time (one cooperative gather of 48 B (float32) or 32 B
// (float16 colour) records), and for every record and tile row the falloff
// exponent is rewritten as a quadratic in the pixel's column offset lx within
// its 16-pixel column block, so that per pixel it costs two fused
// multiply-adds; every thread then walks the batch:
//   q = (A lx + a1) lx + a0 = A dx^2 + B dx dy + C dy^2 + L
//                                          (log2 of o * Gaussian falloff)
//   skip if q < log2(1/255)                (alpha < 1/255)
//   alpha = min(0.99, 2^q)
//   stop if T (1 - alpha) < 1e-4           (this Gaussian is not blended)
//   C += alpha T c;  T *= 1 - alpha
// and the CTA leaves its list as soon as a block-wide ballot
// (__syncthreads_count) finds every pixel finished. Every floating-point step
// is an explicitly rounded operation whose inputs depend only on the pixel and
// the Gaussian (the column block is fixed by the pixel, not by the tile), so a
// pixel's value depends only on its own Gaussian sequence: the same bits for any
// tile shape, batch size, camera batch or launch form.
//
// Launch forms: one CTA per tile (grid = tiles), or persistent CTAs that take
// tiles from an atomic ticket (batched renders, where one launch covers the
// tiles of many cameras).
#include "ngs_internal.cuh"

namespace ngs {

__device__ __forceinline__ void rec_colour(const Rec32 &r, float &cr, float &cg, float &cb) {
    cr = r.b.z; cg = r.b.w; cb = r.c.x;
}
__device__ __forceinline__ void rec_colour(const Rec16 &r, float &cr, float &cg, float &cb) {
    const uint32_t u = __float_as_uint(r.b.z), w = __float_as_uint(r.b.w);
    const float2 rg = __half22float2(*reinterpret_cast<const __half2 *>(&u));
    cr = rg.x; cg = rg.y;
    cb = __low2float(*reinterpret_cast<const __half2 *>(&w));   // high half: support size
}

__device__ __forceinline__ void set_sentinel(Rec32 &r) {
    r.a = make_float4(0.f, 0.f, 0.f, 0.f);
    r.b = make_float4(0.f, __int_as_float(0xff800000), 0.f, 0.f);
    r.c = make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ void set_sentinel(Rec16 &r) {
    r.a = make_float4(0.f, 0.f, 0.f, 0.f);
    r.b = make_float4(0.f, __int_as_float(0xff800000), 0.f, 0.f);
}

// log2 of o times the Gaussian falloff at pixel centre (fpx, fpy)
template <typename R>
__device__ __forceinline__ float exponent(const R &r, float fpx, float fpy) {
    const float dx = __fsub_rn(fpx, r.a.x), dy = __fsub_rn(fpy, r.a.y);
    return __fmaf_rn(r.a.z, __fmul_rn(dx, dx),
                     __fmaf_rn(r.a.w, __fmul_rn(dx, dy), __fmaf_rn(r.b.x, __fmul_rn(dy, dy), r.b.y)));
}

// Largest q = A dx^2 + B dx dy + C dy^2 + L (A, C < 0) over the rectangle
// [ex0, ex1] x [ey0, ey1] of offsets from the Gaussian centre: L when the
// centre is inside, else the best of the four edges, each a 1D concave
// quadratic maximised in closed form and clamped to the edge.
__device__ __forceinline__ float rect_qmax(float A, float B, float C, float L, float ex0,
                                           float ex1, float ey0, float ey1) {
    if (ex0 <= 0.0f && 0.0f <= ex1 && ey0 <= 0.0f && 0.0f <= ey1) return L;
    const float sy = -B / (2.0f * C), sx = -B / (2.0f * A);
    float y = fminf(fmaxf(sy * ex0, ey0), ey1);
    float best = A * ex0 * ex0 + B * ex0 * y + C * y * y;
    y = fminf(fmaxf(sy * ex1, ey0), ey1);
    best = fmaxf(best, A * ex1 * ex1 + B * ex1 * y + C * y * y);
    float x = fminf(fmaxf(sx * ey0, ex0), ex1);
    best = fmaxf(best, A * x * x + B * x * ey0 + C * ey0 * ey0);
    x = fminf(fmaxf(sx * ey1, ex0), ex1);
    best = fmaxf(best, A * x * x + B * x * ey1 + C * ey1 * ey1);
    return best + L;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename R, int TW, int TH, int BATCH>
__global__ void __launch_bounds__(TW *TH)
k_composite(const DevCamera *__restrict__ cams, int n_cams, uint32_t n_tiles,
            const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval,
            const R *__restrict__ rec, uint32_t *ticket, int persistent, const int *err,
            unsigned long long *work64) {
    constexpr int NT = TW * TH;
    constexpr int kPer = (BATCH + NT - 1) / NT;   // records gathered per thread per round
    __shared__ uint32_t s_wsum[(NT + 31) / 32];
    // dynamic shared memory: BATCH records, then per (record, tile row) the
    // exponent as a quadratic in the pixel's column offset lx within its
    // 16-pixel column block: q = (A lx + a1) lx + a0, stored (a1, a0, A, 0)
    extern __shared__ float4 smem_dyn[];
    R *s_rec = reinterpret_cast<R *>(smem_dyn);
    float4 *s_coef = smem_dyn + BATCH * (sizeof(R) / sizeof(float4));
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_evals;
    __shared__ uint32_t s_staged;
    if (*err) return;
    const int tid = threadIdx.x;
    const int lx = tid % TW, ly = tid / TW;
    uint32_t tile = blockIdx.x;
    for (;;) {
        if (persistent) {
            if (tid == 0) s_tile = atomicAdd(ticket, 1u);
            __syncthreads();
            tile = s_tile;
        }
        if (tile >= n_tiles) break;
        int lo = 0, hi = n_cams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cams[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
        }
        const DevCamera &cam = cams[lo];
        const uint32_t local = tile - cam.tile_base;
        const int tx = (int)(local % (uint32_t)cam.tiles_x), ty = (int)(local / (uint32_t)cam.tiles_x);
        const int x0 = tx * TW, y0 = ty * TH;
        const int px = x0 + lx, py = y0 + ly;
        const bool inside = px < cam.width && py < cam.height;
        // column reference: the centre of the first pixel of px's 16-pixel block
        // (the same for every tile shape, so a pixel's arithmetic never depends
        // on how the image is tiled)
        const float xref = (float)(x0 & ~15) + 0.5f;
        // the tile's pixel-centre rectangle (whole tile, also where it overhangs)
        const float tile_x0c = (float)x0 + 0.5f, tile_x1c = (float)(x0 + TW) - 0.5f;
        const float tile_y0c = (float)y0 + 0.5f, tile_y1c = (float)(y0 + TH) - 0.5f;
        const float lxf = (float)(px & 15);
        const uint2 rg = ranges[tile];
        float T = 1.0f, cr = 0.0f, cg = 0.0f, cb = 0.0f;
        bool done = !inside;
        uint32_t evals = 0;
        if (work64 && tid == 0) { s_evals = 0; s_staged = 0; }
        // round r's records are requested during round r - 1 (software pipeline)
        R mine[kPer];
        if (rg.x < rg.y) {
            const int n0 = (int)min((uint32_t)BATCH, rg.y - rg.x);
#pragma unroll
            for (int f = 0; f < kPer; ++f)
                if (tid * kPer + f < n0) mine[f] = rec[pval[rg.x + tid * kPer + f]];
        }
        for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
            if (__syncthreads_count(!done) == 0) break;
            const int n = (int)min((uint32_t)BATCH, rg.y - start);
            // keep, in list order, the records whose support reaches the tile's
            // pixel-centre rectangle
            uint32_t keepmask = 0, nkeep = 0;
#pragma unroll
            for (int f = 0; f < kPer; ++f) {
                const int j = tid * kPer + f;
                if (j < n) {
                    const float q = rect_qmax(mine[f].a.z, mine[f].a.w, mine[f].b.x, mine[f].b.y,
                                              tile_x0c - mine[f].a.x, tile_x1c - mine[f].a.x,
                                              tile_y0c - mine[f].a.y, tile_y1c - mine[f].a.y);
                    if (q >= kLog2AlphaMin - kTileMarginLog2) {
                        keepmask |= 1u << f;
                        ++nkeep;
                    }
                }
            }
            uint32_t incl = nkeep;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if ((tid & 31) >= o) incl += t;
            }
            if ((tid & 31) == 31) s_wsum[tid >> 5] = incl;
            __syncthreads();
            uint32_t wb = 0, nk = 0;
#pragma unroll
            for (int w = 0; w < (NT + 31) / 32; ++w) {
                if (w < (tid >> 5)) wb += s_wsum[w];
                nk += s_wsum[w];
            }
            uint32_t pos = wb + incl - nkeep;
#pragma unroll
            for (int f = 0; f < kPer; ++f)
                if ((keepmask >> f) & 1u) s_rec[pos++] = mine[f];
            {
                const uint32_t nxt = start + BATCH;
                if (nxt < rg.y) {
                    const int nn = (int)min((uint32_t)BATCH, rg.y - nxt);
#pragma unroll
                    for (int f = 0; f < kPer; ++f)
                        if (tid * kPer + f < nn) mine[f] = rec[pval[nxt + tid * kPer + f]];
                }
            }
            const int n4 = ((int)nk + 3) & ~3;
            for (int j = (int)nk + tid; j < n4; j += NT) set_sentinel(s_rec[j]);   // q = -inf
            if (work64 && tid == 0) s_staged += n;
            __syncthreads();
            for (int e = tid; e < n4 * TH; e += NT) {
                const int j = e / TH, r = e - j * TH;
                const R &rr = s_rec[j];
                const float A = rr.a.z, B = rr.a.w, C = rr.b.x, L = rr.b.y;
                const float dxt = __fsub_rn(xref, rr.a.x);
                const float dy = __fsub_rn((float)(y0 + r) + 0.5f, rr.a.y);
                const float bdy = __fmul_rn(B, dy);
                const float a1 = __fmaf_rn(__fadd_rn(A, A), dxt, bdy);
                const float a0 = __fmaf_rn(__fmaf_rn(A, dxt, bdy), dxt,
                                           __fmaf_rn(C, __fmul_rn(dy, dy), L));
                s_coef[j * TH + r] = make_float4(a1, a0, A, 0.0f);
            }
            __syncthreads();
            if (!done) {
                int j = 0;
                for (; j < n4; j += 4) {
                    // the four exponents do not depend on T: evaluate them together,
                    // then blend in list order
                    float q[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 c = s_coef[(j + u) * TH + ly];
                        q[u] = __fmaf_rn(__fmaf_rn(c.z, lxf, c.x), lxf, c.y);
                    }
                    int u = 0;
#pragma unroll
                    for (; u < 4; ++u) {
                        if (q[u] < kLog2AlphaMin) continue;
                        const float alpha = fminf(kAlphaMax, ex2_approx(q[u]));
                        const float test_T = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                        if (test_T < kTMin) { done = true; break; }
                        float gr, gg, gb;
                        rec_colour(s_rec[j + u], gr, gg, gb);
                        const float w = __fmul_rn(alpha, T);
                        cr = __fmaf_rn(w, gr, cr);
                        cg = __fmaf_rn(w, gg, cg);
                        cb = __fmaf_rn(w, gb, cb);
                        T = test_T;
                    }
                    if (done) { j += u + 1; break; }
                }
                evals += (uint32_t)min(j, (int)nk);
            }
        }
        if (work64) {
            __syncthreads();
            atomicAdd(&s_evals, (unsigned long long)evals);
            __syncthreads();
            if (tid == 0) {
                atomicAdd(&work64[0], (unsigned long long)s_staged);
                atomicAdd(&work64[1], s_evals);
            }
        }
        if (inside) {
            const int64_t plane = (int64_t)cam.width * cam.height;
            const int64_t p = (int64_t)py * cam.width + px;
            cam.image[p] = cr;
            cam.image[plane + p] = cg;
            cam.image[2 * plane + p] = cb;
        }
        if (!persistent) break;
        __syncthreads();
    }
}

template <typename R, int TW, int TH, int BATCH>
constexpr size_t comp_smem() {
    return (size_t)BATCH * sizeof(R) + (size_t)BATCH * TH * sizeof(float4);
}

template <typename R, int TW, int TH, int BATCH>
static void set_attr() {
    cudaFuncSetAttribute(k_composite<R, TW, TH, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)comp_smem<R, TW, TH, BATCH>());
}

template <typename R>
static void set_attr_r() {
    set_attr<R, 8, 8, 64>(); set_attr<R, 8, 8, 128>(); set_attr<R, 8, 8, 256>();
    set_attr<R, 16, 8, 64>(); set_attr<R, 16, 8, 128>(); set_attr<R, 16, 8, 256>();
    set_attr<R, 16, 16, 64>(); set_attr<R, 16, 16, 128>(); set_attr<R, 16, 16, 256>();
}

void composite_init_attributes() {
    set_attr_r<Rec32>();
    set_attr_r<Rec16>();
}

template <typename R, int TW, int TH>
static void launch_b(int batch, const DevCamera *cams, int n_cams, uint32_t n_tiles,
                     const uint2 *ranges, const uint32_t *pval, const void *rec, uint32_t *ticket,
                     int persistent, int grid, const int *err, unsigned long long *work64,
                     cudaStream_t st) {
    const R *r = (const R *)rec;
    switch (batch) {
    case 64:
        k_composite<R, TW, TH, 64><<<grid, TW * TH, comp_smem<R, TW, TH, 64>(), st>>>(cams, n_cams, n_tiles, ranges, pval,
                                                             r, ticket, persistent, err, work64);
        break;
    case 256:
        k_composite<R, TW, TH, 256><<<grid, TW * TH, comp_smem<R, TW, TH, 256>(), st>>>(cams, n_cams, n_tiles, ranges, pval,
                                                              r, ticket, persistent, err, work64);
        break;
    default:
        k_composite<R, TW, TH, 128><<<grid, TW * TH, comp_smem<R, TW, TH, 128>(), st>>>(cams, n_cams, n_tiles, ranges, pval,
                                                              r, ticket, persistent, err, work64);
        break;
    }
}

template <typename R>
static void launch_r(int tile_w, int tile_h, int batch, const DevCamera *cams, int n_cams,
                     uint32_t n_tiles, const uint2 *ranges, const uint32_t *pval, const void *rec,
                     uint32_t *ticket, int persistent, int grid, const int *err,
                     unsigned long long *work64, cudaStream_t st) {
    if (tile_w == 8 && tile_h == 8)
        launch_b<R, 8, 8>(batch, cams, n_cams, n_tiles, ranges, pval, rec, ticket, persistent, grid,
                          err, work64, st);
    else if (tile_w == 16 && tile_h == 8)
        launch_b<R, 16, 8>(batch, cams, n_cams, n_tiles, ranges, pval, rec, ticket, persistent,
                           grid, err, work64, st);
    else
        launch_b<R, 16, 16>(batch, cams, n_cams, n_tiles, ranges, pval, rec, ticket, persistent,
                            grid, err, work64, st);
}

void launch_composite(int attr_dtype, int tile_w, int tile_h, int batch, bool persistent,
                      const DevCamera *cams, int n_cams, uint32_t n_tiles, const uint2 *ranges,
                      const uint32_t *pval, const void *rec, uint32_t *ticket, int grid,
                      const int *err, unsigned long long *work64, cudaStream_t st) {
    if (attr_dtype == NGS_F32)
        launch_r<Rec32>(tile_w, tile_h, batch, cams, n_cams, n_tiles, ranges, pval, rec, ticket,
                        persistent ? 1 : 0, grid, err, work64, st);
    else
        launch_r<Rec16>(tile_w, tile_h, batch, cams, n_cams, n_tiles, ranges, pval, rec, ticket,
                        persistent ? 1 : 0, grid, err, work64, st);
}

template <typename R, int TW, int TH, int BATCH>
static int occ() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_composite<R, TW, TH, BATCH>, TW * TH,
                                                  comp_smem<R, TW, TH, BATCH>());
    return n;
}

template <typename R, int TW, int TH>
static int occ_b(int batch) {
    return batch == 64 ? occ<R, TW, TH, 64>() : batch == 256 ? occ<R, TW, TH, 256>()
                                                              : occ<R, TW, TH, 128>();
}

template <typename R>
static int occ_r(int tile_w, int tile_h, int batch) {
    if (tile_w == 8 && tile_h == 8) return occ_b<R, 8, 8>(batch);
    if (tile_w == 16 && tile_h == 8) return occ_b<R, 16, 8>(batch);
    return occ_b<R, 16, 16>(batch);
}

int composite_blocks_per_sm(int attr_dtype, int tile_w, int tile_h, int batch) {
    return attr_dtype == NGS_F32 ? occ_r<Rec32>(tile_w, tile_h, batch)
                                 : occ_r<Rec16>(tile_w, tile_h, batch);
}

}  // namespace ngs
