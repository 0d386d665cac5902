// K7: per-tile front-to-back alpha compositing (3DGS rasterisation as used by
// the H3DGS engine, Sec. III-A/III-B).
//
// One CTA renders one tile (TW x TH threads, one pixel each). The tile's
// Gaussians, in (depth, node id) order, are staged in shared memory BATCH
// records at a time (one cooperative gather of 48 B (float32) or 32 B
// (float16 colour) records), and for every record and tile row the falloff
// exponent, kept in the factored form L - (F1 dx + F2 dy)^2 - (F3 dy)^2, is
// rewritten as a quadratic in the pixel's column offset lx within its 16-pixel
// column block, so that per pixel it costs two fused multiply-adds; every
// thread then walks the batch:
//   q = (A lx + a1) lx + a0 = L - (F1 dx + F2 dy)^2 - (F3 dy)^2, A = -F1^2
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
// A CTA covers a TW x TH block of pixels: a whole binning tile, or one of the
// sub_x x sub_y equal blocks a binning tile is split into (work item = tile *
// sub_x * sub_y + block, row-major within the tile). Each block walks its
// tile's whole list and keeps only the records that can reach it, so large
// binning tiles (few pairs to sort) can be composited by small CTAs (few warps
// waiting on one another at the staging barriers, early exit per block). The
// pixels do not depend on the split either.
//
// Launch forms: one CTA per work item (grid = items), or persistent CTAs that
// take items from an atomic ticket (batched renders, where one launch covers
// the tiles of many cameras).
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

// Largest q = L - (F1 x + F2 y)^2 - (F3 y)^2 over the rectangle [ex0, ex1] x
// [ey0, ey1] of offsets (x, y) from the Gaussian centre: L when the centre is
// inside, else the best of the four edges, each a 1D concave quadratic
// maximised in closed form (on x = const at y = -F1 F2 x / (F2^2 + F3^2), on
// y = const at x = -F2 y / F1) and clamped to the edge; every value is taken
// in the factored form, which does not cancel.
__device__ __forceinline__ float rect_qmax(float F1, float F2, float F3, float L, float ex0,
                                           float ex1, float ey0, float ey1) {
    if (ex0 <= 0.0f && 0.0f <= ex1 && ey0 <= 0.0f && 0.0f <= ey1) return L;
    auto qf = [&](float x, float y) {
        const float p = fmaf(F1, x, F2 * y), e = F3 * y;
        return -fmaf(p, p, e * e);
    };
    // the slopes only place the point evaluated on each edge: an approximate
    // quotient moves it by a relative 1e-6, which lowers the value found by far
    // less than the threshold margin (the maximum is flat there)
    const float sy = __fdividef(-F1 * F2, fmaf(F2, F2, F3 * F3)), sx = __fdividef(-F2, F1);
    float best = qf(ex0, fminf(fmaxf(sy * ex0, ey0), ey1));
    best = fmaxf(best, qf(ex1, fminf(fmaxf(sy * ex1, ey0), ey1)));
    best = fmaxf(best, qf(fminf(fmaxf(sx * ey0, ex0), ex1), ey0));
    best = fmaxf(best, qf(fminf(fmaxf(sx * ey1, ex0), ex1), ey1));
    return best + L;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Conservative bounding box of the pixel-centre offsets where a record can
// still pass the alpha threshold: the ellipse (F1 dx + F2 dy)^2 + (F3 dy)^2 <=
// kappa, kappa = L - log2(1/255) + kTileMarginLog2, has half-widths
// sqrt(kappa (F2^2 + F3^2)) / (F1 F3) and sqrt(kappa) / F3 (no cancellation in
// the factored form); the box is widened by a relative 2^-10 and by 1/64 px,
// far more than the relative 1e-6 of the approximate square roots and
// quotients taken here. Returned as (xmin, xmax, ymin, ymax) in pixel
// coordinates.
__device__ __forceinline__ float4 record_box(float x, float y, float F1, float F2, float F3,
                                            float L) {
    const float kappa = L - (kLog2AlphaMin - kTileMarginLog2);
    const float inf = __int_as_float(0x7f800000);
    if (!(kappa >= 0.0f)) return make_float4(inf, -inf, inf, -inf);   // empty
    if (!(F1 > 0.0f) || !(F3 > 0.0f)) return make_float4(-inf, inf, -inf, inf);
    const float grow = 1.0f + 0.0009765625f;
    const float sk = kappa > 0.0f ? kappa * rsqrtf(kappa) : 0.0f;
    const float m = fmaf(F2, F2, F3 * F3);   // >= F3^2 > 0
    const float hx = fmaf(__fdividef(sk * (m * rsqrtf(m)), F1 * F3), grow, 0.015625f);
    const float hy = fmaf(__fdividef(sk, F3), grow, 0.015625f);
    return make_float4(x - hx, x + hx, y - hy, y + hy);
}

// colour and the lx^2 coefficient -F1^2 of a staged record, each value twice,
// as register pairs for packed two-pixel arithmetic: (r, r, g, g), (b, b, A, A)
struct PairRec {
    float4 rg;
    float4 bA;
};

// A warp renders a WBW x BH block (64 pixels, two per thread) of the tile:
// 8x8 in 8-wide tiles, 16x4 otherwise; 32-wide tiles hold two blocks side by
// side. A warp block lies in one 16-pixel column block and holds NRPW row
// pairs, for which the warp computes its records' coefficient sets.
template <typename R, int TW, int TH, int BATCH>
struct CompLayout {
    static constexpr int WBW = TW < 16 ? TW : 16;      // width of a warp's block
    static constexpr int BH = 64 / WBW;                // rows of a warp's block
    static constexpr int NWX = TW / WBW;               // warp blocks across the tile
    static constexpr int NW = NWX * (TH / BH);         // warps per tile
    static constexpr int NT = 32 * NW;                 // threads: two pixels each
    static constexpr int NRPW = BH / 2;                // row pairs per warp block
    static constexpr int kListStride = BATCH + 4;      // u32 entries per warp list
    static constexpr size_t rec_off = 0;
    static constexpr size_t coef_off = rec_off + (size_t)BATCH * sizeof(R);
    static constexpr size_t pair_off =
        coef_off + (size_t)NW * kListStride * NRPW * sizeof(float4);
    static constexpr size_t box_off = pair_off + (size_t)(BATCH + 1) * sizeof(PairRec);
    static constexpr size_t list_off = box_off + (size_t)BATCH * sizeof(float4);
    static constexpr size_t bytes = list_off + (size_t)NW * kListStride * sizeof(uint32_t);
    static_assert(TW == 8 || TW == 16 || TW == 32, "tile width 8, 16 or 32");
    static_assert(TH % BH == 0, "tile of whole warp blocks");
    static_assert(NT <= 1024, "at most 1024 threads");
    static_assert(BATCH % 4 == 0, "lists padded to groups of four");
};

__device__ __forceinline__ float finite_or_max(float v) { return fminf(v, 3.402823466e38f); }

// at least five 128-thread CTAs per SM (at most 102 registers): measured
// faster than both more registers (4 CTAs) and fewer (6 or 7, with spills)
template <typename R, int TW, int TH, int BATCH>
__global__ void __launch_bounds__(CompLayout<R, TW, TH, BATCH>::NT,
                                  (5 * 128) / CompLayout<R, TW, TH, BATCH>::NT)
k_composite(const DevCamera *__restrict__ cams, int n_cams, uint32_t n_tiles,
            const uint2 *__restrict__ ranges, const uint32_t *__restrict__ pval,
            const R *__restrict__ rec, uint32_t *ticket, int persistent, const int *err,
            unsigned long long *work64, int sub_x, int sub_y, const uint32_t *__restrict__ order,
            unsigned long long *tail) {
    using Lay = CompLayout<R, TW, TH, BATCH>;
    constexpr int NT = Lay::NT, BH = Lay::BH, WBW = Lay::WBW, NWX = Lay::NWX;
    constexpr int NRPW = Lay::NRPW;
    constexpr int kPer = (BATCH + NT - 1) / NT;   // records gathered per thread per round
    __shared__ uint32_t s_wsum[Lay::NW];
    // dynamic shared memory, per round: the tile's kept records; per warp, for
    // each entry of its record list and each pair of rows r, r + 1 of its pixel
    // block, the exponent as a quadratic in the pixel's column offset lx within
    // its 16-pixel column block, q = (A lx + a1) lx + a0, stored (a1_r,
    // a1_r+1, a0_r, a0_r+1) at (warp * list stride + entry) * NRPW + row pair;
    // the records' PairRec; their reach boxes; one record list per warp. Record
    // index BATCH is a sentinel (zero colour; its coefficient sets hold
    // q = -inf).
    extern __shared__ float4 smem_dyn[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(smem_dyn);
    R *s_rec = reinterpret_cast<R *>(sm + Lay::rec_off);
    float4 *s_coef = reinterpret_cast<float4 *>(sm + Lay::coef_off);
    PairRec *s_pair = reinterpret_cast<PairRec *>(sm + Lay::pair_off);
    float4 *s_box = reinterpret_cast<float4 *>(sm + Lay::box_off);
    uint32_t *s_list = reinterpret_cast<uint32_t *>(sm + Lay::list_off);
    __shared__ uint32_t s_tile;
    if (*err) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // warp -> WBW x BH pixel block of the tile; thread -> the pixels (lx, ly)
    // and (lx, ly + 1)
    const int bx = (warp % NWX) * WBW, by = (warp / NWX) * BH;
    const int lx = bx + lane % WBW, ly = by + 2 * (lane / WBW);
    const int rp = lane / WBW;                        // the lane's row pair in its block
    const int wcb = TW < 16 ? 0 : bx >> 4;            // the warp's 16-pixel column block
    uint32_t *my_list = s_list + warp * Lay::kListStride;
    float4 *my_coef = s_coef + (size_t)warp * Lay::kListStride * NRPW;
    const float inf = __int_as_float(0x7f800000);
    if (tid == 0) {
        s_pair[BATCH].rg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        s_pair[BATCH].bA = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    const float2 kMinusOne2 = make_float2(-1.0f, -1.0f);
    unsigned long long evals = 0, staged = 0;
    const uint32_t nsub = (uint32_t)(sub_x * sub_y);
    const uint32_t n_items = n_tiles * nsub;
    uint32_t item = blockIdx.x;
    for (;;) {
        if (persistent) {
            if (tid == 0) s_tile = atomicAdd(ticket, 1u);
            __syncthreads();
            item = s_tile;
        }
        if (item >= n_items) {
            // the first CTA to find the queue empty marks the start of the tail
            if (tail && tid == 0) atomicMax(&tail[0], ~globaltimer_ns());
            break;
        }
        uint32_t tile = nsub == 1 ? item : item / nsub;
        const int sub = (int)(item - tile * nsub);
        if (order) tile = order[tile];   // tiles taken longest list first
        int lo = 0, hi = n_cams - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cams[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
        }
        const DevCamera &cam = cams[lo];
        const uint32_t local = tile - cam.tile_base;
        const int tx = (int)(local % (uint32_t)cam.tiles_x), ty = (int)(local / (uint32_t)cam.tiles_x);
        const int x0 = (tx * sub_x + sub % sub_x) * TW, y0 = (ty * sub_y + sub / sub_x) * TH;
        const int px = x0 + lx, py = y0 + ly;
        const bool in0 = px < cam.width && py < cam.height;
        const bool in1 = px < cam.width && py + 1 < cam.height;
        // column reference: the centre of the first pixel of px's 16-pixel block
        // (the same for every tile shape, so a pixel's arithmetic never depends
        // on how the image is tiled)
        const float xref = (float)(x0 & ~15) + 0.5f;
        // the tile's and the warp block's pixel-centre rectangles (whole tile,
        // also where it overhangs the image)
        const float tile_x0c = (float)x0 + 0.5f, tile_x1c = (float)(x0 + TW) - 0.5f;
        const float tile_y0c = (float)y0 + 0.5f, tile_y1c = (float)(y0 + TH) - 0.5f;
        const float blk_x0c = (float)(x0 + bx) + 0.5f, blk_x1c = blk_x0c + (float)(WBW - 1);
        const float blk_y0c = (float)(y0 + by) + 0.5f, blk_y1c = blk_y0c + (float)(BH - 1);
        const float lxf = (float)(px & 15);
        const float2 lx2 = make_float2(lxf, lxf);
        const uint2 rgs = ranges[tile];
        const uint2 rg = make_uint2(~rgs.x, rgs.y);   // stored as (~first, end)
        // T = 0 marks a finished pixel (also one outside the image)
        float2 T2 = make_float2(in0 ? 1.0f : 0.0f, in1 ? 1.0f : 0.0f);
        float2 cr2 = make_float2(0.0f, 0.0f), cg2 = cr2, cb2 = cr2;
        // round r's records are requested during round r - 1 (software pipeline)
        R mine[kPer];
        if (rg.x < rg.y) {
            const int n0 = (int)min((uint32_t)BATCH, rg.y - rg.x);
#pragma unroll
            for (int f = 0; f < kPer; ++f)
                if (tid * kPer + f < n0) mine[f] = rec[pval[rg.x + tid * kPer + f]];
        }
        for (uint32_t start = rg.x; start < rg.y; start += BATCH) {
            if (__syncthreads_count(T2.x > 0.0f || T2.y > 0.0f) == 0) break;
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
                if (lane >= o) incl += t;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            uint32_t wb = 0, nk = 0;
#pragma unroll
            for (int w = 0; w < Lay::NW; ++w) {
                if (w < warp) wb += s_wsum[w];
                nk += s_wsum[w];
            }
            uint32_t pos = wb + incl - nkeep;
#pragma unroll
            for (int f = 0; f < kPer; ++f)
                if ((keepmask >> f) & 1u) {
                    const R &m = mine[f];
                    s_rec[pos] = m;
                    float gr, gg, gb;
                    rec_colour(m, gr, gg, gb);
                    // finite colours: a record blended with weight 0 then leaves
                    // the sums unchanged
                    gr = finite_or_max(gr); gg = finite_or_max(gg); gb = finite_or_max(gb);
                    s_pair[pos].rg = make_float4(gr, gr, gg, gg);
                    const float A = -__fmul_rn(m.a.z, m.a.z);
                    s_pair[pos].bA = make_float4(gb, gb, A, A);
                    s_box[pos] = record_box(m.a.x, m.a.y, m.a.z, m.a.w, m.b.x, m.b.y);
                    ++pos;
                }
            {
                const uint32_t nxt = start + BATCH;
                if (nxt < rg.y) {
                    const int nn = (int)min((uint32_t)BATCH, rg.y - nxt);
#pragma unroll
                    for (int f = 0; f < kPer; ++f)
                        if (tid * kPer + f < nn) mine[f] = rec[pval[nxt + tid * kPer + f]];
                }
            }
            if (tid == 0) staged += (unsigned long long)n;
            __syncthreads();
            // each warp lists, in order, the kept records whose reach box meets
            // its block (skipped records have q < log2(1/255) at all its pixels)
            const bool warp_live = __any_sync(0xffffffffu, T2.x > 0.0f || T2.y > 0.0f);
            int len = 0;
            if (warp_live) {
                for (int c = 0; c < (int)nk; c += 32) {
                    const int j = c + lane;
                    bool hit = false;
                    if (j < (int)nk) {
                        const float4 b = s_box[j];
                        hit = b.y >= blk_x0c && b.x <= blk_x1c && b.w >= blk_y0c && b.z <= blk_y1c;
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                    if (hit) my_list[len + __popc(bal & lanemask_lt())] = (uint32_t)j;
                    len += __popc(bal);
                }
                if (lane < ((4 - (len & 3)) & 3)) my_list[len + lane] = (uint32_t)BATCH;
            }
            // the warp's coefficient sets for its own list entries and row
            // pairs (padding entries get the sentinel's q = -inf)
            if (warp_live) {
                const int len4w = (len + 3) & ~3;
                for (int e = lane; e < len4w * NRPW; e += 32) {
                    const int i = e / NRPW, r = e - i * NRPW;
                    float4 cfv = make_float4(0.0f, 0.0f, -inf, -inf);
                    if (i < len) {
                        const R &rr = s_rec[my_list[i]];
                        const float F1 = rr.a.z, F2 = rr.a.w, F3 = rr.b.x, L = rr.b.y;
                        const float dxt = __fsub_rn(xref + (float)(16 * wcb), rr.a.x);
                        const float m2f1 = __fmul_rn(-2.0f, F1);
                        const int p = (by >> 1) + r;
                        float a1[2], a0[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            // q(lx) = L - (p0 + F1 lx)^2 - (F3 dy)^2, p0 = F1 dxt + F2 dy
                            const float dy = __fsub_rn((float)(y0 + 2 * p + h) + 0.5f, rr.a.y);
                            const float p0 = __fmaf_rn(F1, dxt, __fmul_rn(F2, dy));
                            const float e = __fmul_rn(F3, dy);
                            a1[h] = __fmul_rn(m2f1, p0);
                            a0[h] = __fmaf_rn(-p0, p0, __fmaf_rn(-e, e, L));
                        }
                        cfv = make_float4(a1[0], a1[1], a0[0], a0[1]);
                    }
                    my_coef[e] = cfv;
                }
                __syncwarp();
            }
            if (T2.x > 0.0f || T2.y > 0.0f) {
                // both pixels in packed (f32x2) arithmetic, every step the same
                // rounded operation per pixel as a scalar evaluation:
                //   q = (A lx + a1) lx + a0; alpha = min(0.99, 2^q), 0 if
                //   q < log2(1/255); T' = T (1 - alpha); a pixel ends (unblended)
                //   at the record with T' < 1e-4; else C += (alpha T) c, T = T'.
                // The threshold decision is an exact 0/1 factor mq (a record
                // below it gets alpha = 0 and T' = T: no per-record branch). A
                // group of four records is first blended as if no pixel ended in
                // it; only if a live pixel's T' fell below 1e-4 somewhere in the
                // group (T only decreases, so its last T' tells) is the group
                // redone from its start with the stop decision per record (factor
                // m: the ending record gets weight alpha (T m) = 0 and leaves
                // T = T' m = 0). With m = 1 both forms round identically, so the
                // bits do not depend on where the groups fall. An ended pixel
                // keeps T = 0 exactly (a live T stays >= 1e-4 * (1 - 0.99)), and a
                // lane leaves after the group in which both its pixels ended.
                const bool alive_x = T2.x > 0.0f, alive_y = T2.y > 0.0f;
                int end_x = -1, end_y = -1, groups = 0;
                const int len4 = (len + 3) & ~3;
                // alpha of list entry e (its record index j) at both pixels
                auto alpha2 = [&](int e, uint32_t j) {
                    const float4 cf = my_coef[e * NRPW + rp];
                    const float4 bA = s_pair[j].bA;
                    const float2 t = __ffma2_rn(make_float2(bA.z, bA.w), lx2, make_float2(cf.x, cf.y));
                    const float2 q = __ffma2_rn(t, lx2, make_float2(cf.z, cf.w));
                    const float2 mq = make_float2(q.x >= kLog2AlphaMin ? 1.0f : 0.0f,
                                                  q.y >= kLog2AlphaMin ? 1.0f : 0.0f);
                    return __fmul2_rn(make_float2(fminf(kAlphaMax, ex2_approx(q.x)),
                                                  fminf(kAlphaMax, ex2_approx(q.y))),
                                      mq);
                };
#pragma unroll 1
                for (int i = 0; i < len4; i += 4) {
                    const uint4 jv = *reinterpret_cast<const uint4 *>(my_list + i);
                    const uint32_t jj[4] = {jv.x, jv.y, jv.z, jv.w};
                    float2 Tn = T2, rn = cr2, gn = cg2, bn = cb2;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 al = alpha2(i + u, jj[u]);
                        const float2 w2 = __fmul2_rn(al, Tn);
                        const PairRec &pr = s_pair[jj[u]];
                        const float4 c_rg = pr.rg;
                        const float4 c_b = pr.bA;
                        rn = __ffma2_rn(w2, make_float2(c_rg.x, c_rg.y), rn);
                        gn = __ffma2_rn(w2, make_float2(c_rg.z, c_rg.w), gn);
                        bn = __ffma2_rn(w2, make_float2(c_b.x, c_b.y), bn);
                        Tn = __ffma2_rn(w2, kMinusOne2, Tn);   // T (1 - alpha) as T - alpha T
                    }
                    ++groups;
                    if ((Tn.x < kTMin && Tn.x != 0.0f) || (Tn.y < kTMin && Tn.y != 0.0f)) {
                        // a live pixel ends in this group: redo it with the stop test
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const float2 al = alpha2(i + u, jj[u]);
                            const float2 w = __fmul2_rn(al, T2);
                            const float2 t2 = __ffma2_rn(w, kMinusOne2, T2);
                            const float2 m = make_float2(t2.x >= kTMin ? 1.0f : 0.0f,
                                                         t2.y >= kTMin ? 1.0f : 0.0f);
                            const float2 w2 = __fmul2_rn(w, m);
                            const PairRec &pr = s_pair[jj[u]];
                            const float4 c_rg = pr.rg;
                            const float4 c_b = pr.bA;
                            cr2 = __ffma2_rn(w2, make_float2(c_rg.x, c_rg.y), cr2);
                            cg2 = __ffma2_rn(w2, make_float2(c_rg.z, c_rg.w), cg2);
                            cb2 = __ffma2_rn(w2, make_float2(c_b.x, c_b.y), cb2);
                            T2 = __fmul2_rn(t2, m);
                        }
                        if (end_x < 0 && T2.x == 0.0f) end_x = groups;
                        if (end_y < 0 && T2.y == 0.0f) end_y = groups;
                        if (!(T2.x > 0.0f || T2.y > 0.0f)) break;
                    } else {
                        T2 = Tn; cr2 = rn; cg2 = gn; cb2 = bn;
                    }
                }
                // groups of four counted per pixel alive at their start
                evals += 4ull * (uint32_t)((alive_x ? (end_x >= 0 ? end_x : groups) : 0) +
                                           (alive_y ? (end_y >= 0 ? end_y : groups) : 0));
            }
        }
        const int64_t plane = (int64_t)cam.width * cam.height;
        const int64_t p0 = (int64_t)py * cam.width + px;
        if (in0) {
            cam.image[p0] = cr2.x;
            cam.image[plane + p0] = cg2.x;
            cam.image[2 * plane + p0] = cb2.x;
        }
        if (in1) {
            const int64_t p1 = p0 + cam.width;
            cam.image[p1] = cr2.y;
            cam.image[plane + p1] = cg2.y;
            cam.image[2 * plane + p1] = cb2.y;
        }
        if (!persistent) break;
        __syncthreads();
    }
    if (work64) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) evals += __shfl_down_sync(0xffffffffu, evals, o);
        if (lane == 0 && evals) atomicAdd(&work64[1], evals);
        if (tid == 0 && staged) atomicAdd(&work64[0], staged);
    }
    if (tail && tid == 0) atomicMax(&tail[1], globaltimer_ns());
}

// Work order of a persistent compositing launch: the tiles of a sub-batch
// sorted by the length of their lists, longest first, in 63 classes (half
// octaves of the length; empty lists last), so that the longest lists start
// first and the launch does not end waiting on a late long one. One CTA; the
// order within a class is whatever the shared-memory atomics give (the pixels
// do not depend on the order in which tiles are composited).
__device__ __forceinline__ uint32_t length_class(uint2 rg) {
    const uint32_t first = ~rg.x;
    if (!(first < rg.y)) return 63u;
    const uint32_t len = rg.y - first;
    const int lg = 31 - __clz(len);
    const uint32_t half = lg > 0 ? (len >> (lg - 1)) & 1u : 0u;
    return 62u - min(62u, 2u * (uint32_t)lg + half);
}

__global__ void __launch_bounds__(1024)
k_tile_order(const uint2 *__restrict__ ranges, uint32_t n_tiles, uint32_t *__restrict__ order,
             const int *err) {
    __shared__ uint32_t s_hist[64], s_cur[64];
    if (*err) return;
    if (threadIdx.x < 64) s_hist[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x)
        atomicAdd(&s_hist[length_class(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int k = 0; k < 64; ++k) {
            s_cur[k] = acc;
            acc += s_hist[k];
        }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x)
        order[atomicAdd(&s_cur[length_class(ranges[t])], 1u)] = t;
}

void launch_tile_order(const uint2 *ranges, uint32_t n_tiles, uint32_t *order, const int *err,
                       cudaStream_t st) {
    k_tile_order<<<1, 1024, 0, st>>>(ranges, n_tiles, order, err);
}

template <typename R, int TW, int TH, int BATCH>
constexpr size_t comp_smem() {
    return CompLayout<R, TW, TH, BATCH>::bytes;
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
    set_attr<R, 16, 32, 64>(); set_attr<R, 16, 32, 128>(); set_attr<R, 16, 32, 256>();
    set_attr<R, 32, 16, 64>(); set_attr<R, 32, 16, 128>(); set_attr<R, 32, 16, 256>();
    set_attr<R, 32, 32, 64>(); set_attr<R, 32, 32, 128>(); set_attr<R, 32, 32, 256>();
}

void composite_init_attributes() {
    set_attr_r<Rec32>();
    set_attr_r<Rec16>();
}

struct CompLaunch {
    const DevCamera *cams;
    int n_cams;
    uint32_t n_tiles;
    const uint2 *ranges;
    const uint32_t *pval;
    const void *rec;
    uint32_t *ticket;
    int persistent, grid;
    const int *err;
    unsigned long long *work64;
    int sub_x, sub_y;
    const uint32_t *order;
    unsigned long long *tail;
    cudaStream_t st;
};

template <typename R, int TW, int TH, int BATCH>
static void launch_one(const CompLaunch &a) {
    k_composite<R, TW, TH, BATCH>
        <<<a.grid, CompLayout<R, TW, TH, BATCH>::NT, comp_smem<R, TW, TH, BATCH>(), a.st>>>(
            a.cams, a.n_cams, a.n_tiles, a.ranges, a.pval, (const R *)a.rec, a.ticket,
            a.persistent, a.err, a.work64, a.sub_x, a.sub_y, a.order, a.tail);
}

template <typename R, int TW, int TH>
static void launch_b(int batch, const CompLaunch &a) {
    if (batch == 64) launch_one<R, TW, TH, 64>(a);
    else if (batch == 256) launch_one<R, TW, TH, 256>(a);
    else launch_one<R, TW, TH, 128>(a);
}

template <typename R>
static void launch_r(int w, int h, int batch, const CompLaunch &a) {
    if (w == 8 && h == 8) launch_b<R, 8, 8>(batch, a);
    else if (w == 16 && h == 8) launch_b<R, 16, 8>(batch, a);
    else if (w == 16 && h == 32) launch_b<R, 16, 32>(batch, a);
    else if (w == 32 && h == 16) launch_b<R, 32, 16>(batch, a);
    else if (w == 32 && h == 32) launch_b<R, 32, 32>(batch, a);
    else launch_b<R, 16, 16>(batch, a);
}

void launch_composite(int attr_dtype, int tile_w, int tile_h, int cta_w, int cta_h, int batch,
                      bool persistent, const DevCamera *cams, int n_cams, uint32_t n_tiles,
                      const uint2 *ranges, const uint32_t *pval, const void *rec,
                      uint32_t *ticket, int grid, const int *err, unsigned long long *work64,
                      const uint32_t *order, unsigned long long *tail, cudaStream_t st) {
    const CompLaunch a{cams, n_cams, n_tiles, ranges, pval, rec, ticket, persistent ? 1 : 0,
                       grid, err, work64, tile_w / cta_w, tile_h / cta_h, order, tail, st};
    if (attr_dtype == NGS_F32) launch_r<Rec32>(cta_w, cta_h, batch, a);
    else launch_r<Rec16>(cta_w, cta_h, batch, a);
}

template <typename R, int TW, int TH, int BATCH>
static int occ() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_composite<R, TW, TH, BATCH>, CompLayout<R, TW, TH, BATCH>::NT,
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
    if (tile_w == 16 && tile_h == 32) return occ_b<R, 16, 32>(batch);
    if (tile_w == 32 && tile_h == 16) return occ_b<R, 32, 16>(batch);
    if (tile_w == 32 && tile_h == 32) return occ_b<R, 32, 32>(batch);
    return occ_b<R, 16, 16>(batch);
}

int composite_blocks_per_sm(int attr_dtype, int tile_w, int tile_h, int batch) {
    return attr_dtype == NGS_F32 ? occ_r<Rec32>(tile_w, tile_h, batch)
                                 : occ_r<Rec16>(tile_w, tile_h, batch);
}

}  // namespace ngs
