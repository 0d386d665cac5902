// Reference (oracle) implementation of the hierarchical 3DGS render path, in
// float64, for tests and for the CPU baseline only. TEST INFRASTRUCTURE: only
// the test-suite, the smoke entry point and the benchmark's CPU-baseline leg
// load this library; the renderer never calls it and shares no code with it.
//
// What is computed (hierarchical 3D Gaussian Splatting, Sec. III-B: a tree of
// Gaussians, a level-of-detail cut chosen per view, then 3DGS rasterisation of
// the cut from camera intrinsics and extrinsics, Sec. III-A):
//   1. cut       : per node n, granularity s(n) = fx * ext(n) / dist(cam, box(n))
//                  (ext = longest box side, dist = distance from the camera
//                  centre to the box, s = +inf inside it). n is selected iff
//                  (n is a leaf or s(n) <= tau) and (n is the root or
//                  s(parent(n)) > tau).
//   2. preprocess: EWA projection of each cut Gaussian (Sigma2D = J W Sigma
//                  W^T J^T + 0.3 I), its conic, pixel centre, view depth,
//                  degree-3 SH colour, and the tile rectangle covering the
//                  bounding box of its support (the ellipse where alpha >= 1/255)
//                  widened by 1/64 pixel.
//   3. binning   : one (tile, depth) key per Gaussian and overlapped tile,
//                  ordered by a stable sort (std::stable_sort), tile ranges.
//   4. composite : per pixel, front-to-back alpha blending over its tile's list.
//   5. brute force: per pixel over every visible Gaussian in depth order, no
//                  tiles, as an independent check of 3-4.
//   Optional level-of-detail blending (Sec. III-B: transitions between levels
//   are interpolated): a selected node n with parent p is rendered with its
//   attributes moved toward p's, parent weight
//       v = 1 - clamp((s(p) - tau) / (s(p) - s(n)), 0, 1)
//   (v = 0 for the root, when s(p) is infinite or s(p) <= s(n)): mean
//   mu_n + v (mu_p - mu_n), covariance, opacity and SH likewise. v is 0 where
//   tau has just reached s(n) from below (n itself) and 1 where tau is about
//   to reach s(p) (n has become its parent); a leaf finer than tau keeps v = 0.
//   Frustum-culled and shared cuts (Sec. III-B: the selection of levels is
//   made per view, dynamically): the cut can drop the nodes whose box lies
//   outside one of the five planes of a camera's view volume, and one cut can
//   serve a group of cameras (the deepest of the members' choices per path).
// Every floating-point step is float64 except where a step's result decides an
// integer that the renderer must reproduce exactly: the near-plane cull and the
// depth sort key use the float32 view depth computed by one fixed sequence of
// IEEE float operations, the renderer's own precision (the file is compiled
// with -ffp-contract=off so that no other fused multiply-add appears).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

typedef struct {
    int64_t n;                 // nodes
    const float *pos;          // [n][3]
    const float *quat;         // [n][4] w,x,y,z
    const float *log_scale;    // [n][3]
    const float *opacity;      // [n]
    const float *sh;           // [n][16][3]
    const int32_t *parent;     // [n], -1 root
    const int32_t *child_count;// [n]
    const float *aabb_min;     // [n][3]
    const float *aabb_max;     // [n][3]
} orc_scene;

typedef struct {
    double pos[3];
    double R[9];               // world->camera rows (OpenCV: x right, y down, z forward)
    double fx, fy, cx, cy;
    int32_t width, height;
    double tau;
} orc_camera;

// per cut slot, columns of the float64 preprocess table; PC_E* are bounds on
// how far a float32 renderer's values may lie from these (see "float32 error
// model" below): centre (px), the entries b and c of Sigma2D (px^2), the
// relative error of its determinant, log2 of the opacity, and the support
// half-widths (px)
enum {
    PC_VISIBLE = 0, PC_U, PC_V, PC_CONIC_A, PC_CONIC_B, PC_CONIC_C, PC_COV_A, PC_COV_B,
    PC_COV_C, PC_DEPTH, PC_OPACITY, PC_R, PC_G, PC_B, PC_HX, PC_HY,
    PC_EU, PC_EV, PC_EB, PC_EC, PC_EDET, PC_EQL, PC_EHX, PC_EHY, PC_NCOLS
};

static const double kNear = 0.2;           // near plane (view z)
static const double kBlur = 0.3;           // screen-space dilation added to Sigma2D
static const double kAlphaMin = 1.0 / 255.0;
static const double kAlphaMax = 0.99;
static const double kTMin = 1e-4;
static const double kRectMargin = 1.0 / 64.0;   // pixels added to the support radius

void orc_cov3d(const float *quat, const float *log_scale, double *out);

// ---------------------------------------------------------------------------
// 1. cut
// ---------------------------------------------------------------------------

static double granularity(const orc_scene *sc, const orc_camera *cam, int64_t n) {
    double d2 = 0.0, ext = 0.0;
    for (int k = 0; k < 3; ++k) {
        double lo = sc->aabb_min[3 * n + k], hi = sc->aabb_max[3 * n + k];
        double p = cam->pos[k];
        double g = 0.0;
        if (p < lo) g = lo - p;
        else if (p > hi) g = p - hi;
        d2 += g * g;
        ext = std::max(ext, hi - lo);
    }
    if (d2 == 0.0) return INFINITY;
    return cam->fx * ext / std::sqrt(d2);
}

// The granularity in the renderer's precision (float32, one IEEE operation per
// step, no contraction), used only for the blend weight, so that the blended
// mean, and with it the float32 depth key, is the same bit pattern on both
// sides.
float orc_granularity_f32(const orc_scene *sc, const orc_camera *cam, int64_t n) {
    const float px = (float)cam->pos[0], py = (float)cam->pos[1], pz = (float)cam->pos[2];
    const float *lo = sc->aabb_min + 3 * n, *hi = sc->aabb_max + 3 * n;
    const float gx = std::fmax(std::fmax(lo[0] - px, 0.0f), px - hi[0]);
    const float gy = std::fmax(std::fmax(lo[1] - py, 0.0f), py - hi[1]);
    const float gz = std::fmax(std::fmax(lo[2] - pz, 0.0f), pz - hi[2]);
    const float d2 = std::fma(gx, gx, std::fma(gy, gy, gz * gz));
    const float ext = std::fmax(std::fmax(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    if (d2 == 0.0f) return INFINITY;
    return ((float)cam->fx * ext) / std::sqrt(d2);
}

// Parent weight of the level-of-detail blend (float32, as the renderer).
float orc_blend_parent_weight(float s_n, float s_p, float tau) {
    if (!(s_p < INFINITY)) return 0.0f;
    const float den = s_p - s_n;
    if (!(den > 0.0f)) return 0.0f;
    const float w = std::fmin(std::fmax((s_p - tau) / den, 0.0f), 1.0f);
    return 1.0f - w;
}

// Attributes of node g as rendered: its own, or, with blend, moved toward its
// parent's by the parent weight v. mu: float32 (it decides the depth key);
// Sigma: 3x3 row-major; sh: [16][3]. Returns v.
double orc_blend_gaussian(const orc_scene *sc, const orc_camera *cam, int64_t g, int32_t blend,
                          float *mu, double *Sigma, double *opac, double *sh) {
    float v = 0.0f;
    const int32_t par = sc->parent[g];
    if (blend && par >= 0)
        v = orc_blend_parent_weight(orc_granularity_f32(sc, cam, g),
                                    orc_granularity_f32(sc, cam, par), (float)cam->tau);
    orc_cov3d(sc->quat + 4 * g, sc->log_scale + 3 * g, Sigma);
    *opac = sc->opacity[g];
    for (int k = 0; k < 3; ++k) mu[k] = sc->pos[3 * g + k];
    for (int k = 0; k < 48; ++k) sh[k] = sc->sh[48 * g + k];
    if (v > 0.0f) {
        double Sp[9];
        orc_cov3d(sc->quat + 4 * par, sc->log_scale + 3 * par, Sp);
        const double vd = v;
        for (int k = 0; k < 3; ++k)
            mu[k] = std::fma(v, sc->pos[3 * par + k] - mu[k], mu[k]);
        for (int k = 0; k < 9; ++k) Sigma[k] += vd * (Sp[k] - Sigma[k]);
        *opac += vd * ((double)sc->opacity[par] - *opac);
        for (int k = 0; k < 48; ++k) sh[k] += vd * ((double)sc->sh[48 * par + k] - sh[k]);
    }
    return v;
}

// Writes the selected node ids (ascending) and returns their count. If
// near_out is given, near_out[n] = 1 when s(n) or s(parent(n)) lies within
// 1e-5 relative of tau (a decision the float32 renderer may take either way).
// If s_out is given it receives s(n).
int64_t orc_select_cut(const orc_scene *sc, const orc_camera *cam, int32_t *ids_out,
                       uint8_t *near_out, double *s_out) {
    const int64_t n = sc->n;
    std::vector<double> s(n);
    for (int64_t i = 0; i < n; ++i) s[i] = granularity(sc, cam, i);
    const double tau = cam->tau;
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        bool leaf = sc->child_count[i] == 0;
        int32_t par = sc->parent[i];
        bool own = leaf || s[i] <= tau;
        bool up = (par < 0) || s[par] > tau;
        if (own && up) ids_out[cnt++] = (int32_t)i;
        if (near_out) {
            bool nr = std::fabs(s[i] - tau) <= 1e-5 * tau;
            if (par >= 0) nr = nr || std::fabs(s[par] - tau) <= 1e-5 * tau;
            near_out[i] = nr ? 1 : 0;
        }
        if (s_out) s_out[i] = s[i];
    }
    return cnt;
}

// ---------------------------------------------------------------------------
// float32 error model of a renderer (test infrastructure: which decisions a
// float32 evaluation of steps 2 and 4 may take differently from float64)
// ---------------------------------------------------------------------------
//
// A renderer that evaluates the same definitions in float32 (unit roundoff
// u = 2^-24) differs from the float64 values of this oracle by rounding. The
// bounds below are first-order forward error bounds: every elementary float32
// operation (add, multiply, fused multiply-add, division, square root) is
// charged u times the magnitude of its result, a k-term dot product k u times
// the sum of its terms' magnitudes, and the library functions (exp, log,
// reciprocal square root) 4 u relative; they are evaluated at the float64
// values. They describe a renderer that takes the steps in this numerically
// stable form (the float32 renderer of this project does):
//   view vector  t_r = R_r . (mu - c): 6 u sum_k |R_rk d_k| (d_k = mu_k - c_k
//                rounded, three products, two sums); where the depth cancels
//                (sum_k |R_2k d_k| > 8 t_z) from the exact differences with
//                compensated products: 2 u |t_r| + 12 u^2 sum_k |R_rk d_k|
//   centre       u = fx t_x / t_z + cx: fx/t_z (e_tx + |t_x| (3u + e_tz/t_z)) + u|u|
//   J W rows     T_r: every entry within tau_r (from the errors of t and 1/t_z)
//   Sigma2D      from the projections m_rk = T_r . (axis k of the Gaussian)
//                scaled by s_k: a - 0.3 = sum_k (s_k m_0k)^2, c - 0.3 likewise,
//                b = sum_k s_k^2 m_0k m_1k; the errors of the projections
//                (from tau_r, the axes' 8 u and the dot products) bound those
//                of b and c by Cauchy-Schwarz, with no amplification by the
//                footprint's elongation
//   determinant  by Cauchy-Binet, sum_k (s_i s_j)^2 (n . axis_k)^2 + 0.3 (a' + c')
//                + 0.09 (a', c' without the 0.3) with n = T_0 x T_1 from the
//                camera's row cross products (positive terms: a relative error
//                of a few u plus the propagated errors of n); a blended
//                Gaussian (no axes) takes a c - b^2 with the usual cancellation
//   conic        factored: q = log2 o - k [(l11 dx + l21 dy)^2 + (l22 dy)^2],
//                k = log2(e)/2, l11 = sqrt(c/det), l21 = -b/sqrt(c det),
//                l22 = 1/sqrt(c): relative errors of c and det scale the
//                factors, the error of b moves l21
//   exponent     the factors' errors times the factored terms at the pixel,
//                the centre error times |grad q|, the log2 o error, 8 u times
//                the factored terms' magnitudes for evaluating them relative to
//                a reference column up to 16 px from the pixel, plus 2e-6 for
//                the hardware exp2 (relative error below 2^-20)
//   support      h = sqrt(K a) + 1/64, K = 2 ln(255 o): (h - 1/64) (e_K/K + e_a/a)/2
//                + 3 u h
// Against an independent numpy float32 evaluation of these steps the bounds
// hold with room; no further safety factor is applied (kErrSafety = 1).
// A decision of step 4 is "near threshold" when the float64 value lies within
// this bound of the threshold: alpha >= 1/255 (|log2(o G) - log2(1/255)| <=
// E_q) and T (1 - alpha) >= 1e-4 (relative error of T accumulated from the
// (1 - alpha) factors). Such a decision may go either way in float32. Where
// the bound itself exceeds kEqMax the pixel is not enumerated but marked
// unchecked.
static const double kU32 = 5.9604644775390625e-08;   // 2^-24
static const double kErrSafety = 1.0;
static const double kLog2e = 1.4426950408889634;

// ---------------------------------------------------------------------------
// 2. preprocess
// ---------------------------------------------------------------------------

// Real spherical harmonics up to degree 3, orthonormal on the unit sphere, in
// the sign convention of 3DGS (the standard real basis times (-1)^|m|), index
// l*l + l + m. Direction (x, y, z) must be unit length.
void orc_sh_basis(const double *dir, double *out) {
    const double x = dir[0], y = dir[1], z = dir[2];
    const double pi = M_PI;
    const double xx = x * x, yy = y * y, zz = z * z;
    out[0] = 0.5 * std::sqrt(1.0 / pi);
    const double c1 = std::sqrt(3.0 / (4.0 * pi));
    out[1] = -c1 * y;
    out[2] = c1 * z;
    out[3] = -c1 * x;
    const double c2a = 0.5 * std::sqrt(15.0 / pi);
    const double c2b = 0.25 * std::sqrt(5.0 / pi);
    const double c2c = 0.25 * std::sqrt(15.0 / pi);
    out[4] = c2a * x * y;
    out[5] = -c2a * y * z;
    out[6] = c2b * (2.0 * zz - xx - yy);
    out[7] = -c2a * x * z;
    out[8] = c2c * (xx - yy);
    const double c3a = 0.25 * std::sqrt(35.0 / (2.0 * pi));
    const double c3b = 0.5 * std::sqrt(105.0 / pi);
    const double c3c = 0.25 * std::sqrt(21.0 / (2.0 * pi));
    const double c3d = 0.25 * std::sqrt(7.0 / pi);
    const double c3e = 0.25 * std::sqrt(105.0 / pi);
    out[9] = -c3a * y * (3.0 * xx - yy);
    out[10] = c3b * x * y * z;
    out[11] = -c3c * y * (4.0 * zz - xx - yy);
    out[12] = c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    out[13] = -c3c * x * (4.0 * zz - xx - yy);
    out[14] = c3e * z * (xx - yy);
    out[15] = -c3a * x * (xx - 3.0 * yy);
}

// Sigma = R(q) S S^T R(q)^T, q = (w, x, y, z) normalised, S = diag(exp(log_scale)).
// Output: the symmetric 3x3 matrix, row-major.
void orc_cov3d(const float *quat, const float *log_scale, double *out) {
    double w = quat[0], x = quat[1], y = quat[2], z = quat[3];
    const double nq = std::sqrt(w * w + x * x + y * y + z * z);
    w /= nq; x /= nq; y /= nq; z /= nq;
    const double R[9] = {
        1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
        2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
        2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
    double s2[3];
    for (int k = 0; k < 3; ++k) s2[k] = std::exp(2.0 * (double)log_scale[k]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * s2[k] * R[3 * j + k];
            out[3 * i + j] = acc;
        }
}

// The view depth that decides integers: the near-plane cull and the depth
// sort key. Both are taken in the renderer's precision, float32, with one
// fixed sequence of IEEE operations so that both sides agree bit for bit:
// d_k = mu_k - c_k (float subtraction), z = fma(R20, d0, fma(R21, d1, R22 * d2)).
float orc_depth_f32(const float *mu, const orc_camera *cam) {
    const float d0 = mu[0] - (float)cam->pos[0];
    const float d1 = mu[1] - (float)cam->pos[1];
    const float d2 = mu[2] - (float)cam->pos[2];
    const float p2 = (float)cam->R[8] * d2;
    return std::fma((float)cam->R[6], d0, std::fma((float)cam->R[7], d1, p2));
}

// For each cut slot i (node ids[i]) fills out[i*PC_NCOLS + col], depth_key[i]
// (float32 bits of the rounded depth) and rect[i*4..] = (x0, y0, x1, y1), the
// inclusive tile range. Invisible slots get PC_VISIBLE = 0 and rect (0,0,-1,-1).
// With blend, each node is rendered with its level-of-detail blended
// attributes (orc_blend_gaussian).
void orc_preprocess(const orc_scene *sc, const orc_camera *cam, const int32_t *ids, int64_t n,
                    int32_t tile_w, int32_t tile_h, int32_t blend, double *out,
                    uint32_t *depth_key, int32_t *rect) {
    const int32_t tiles_x = (cam->width + tile_w - 1) / tile_w;
    const int32_t tiles_y = (cam->height + tile_h - 1) / tile_h;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *o = out + i * PC_NCOLS;
        for (int c = 0; c < PC_NCOLS; ++c) o[c] = 0.0;
        int32_t *rc = rect + 4 * i;
        rc[0] = 0; rc[1] = 0; rc[2] = -1; rc[3] = -1;
        depth_key[i] = 0xFFFFFFFFu;
        const int64_t g = ids[i];
        float mu[3];
        double S[9], opac, shg[48];
        orc_blend_gaussian(sc, cam, g, blend, mu, S, &opac, shg);
        const float z32 = orc_depth_f32(mu, cam);
        if (!(z32 > (float)kNear)) continue;
        if (255.0 * opac < 1.0) continue;
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = (double)mu[k] - cam->pos[k];
        const double tz = cam->R[6] * d[0] + cam->R[7] * d[1] + cam->R[8] * d[2];
        const double tx = cam->R[0] * d[0] + cam->R[1] * d[1] + cam->R[2] * d[2];
        const double ty = cam->R[3] * d[0] + cam->R[4] * d[1] + cam->R[5] * d[2];
        // Jacobian of (fx x/z, fy y/z) at t
        const double J[6] = {cam->fx / tz, 0.0, -cam->fx * tx / (tz * tz),
                             0.0, cam->fy / tz, -cam->fy * ty / (tz * tz)};
        double T[6];   // J * W
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[3 * r + k] * cam->R[3 * k + c];
                T[3 * r + c] = acc;
            }
        double TS[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += T[3 * r + k] * S[3 * k + c];
                TS[3 * r + c] = acc;
            }
        double C2[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += TS[3 * r + k] * T[3 * c + k];
                C2[2 * r + c] = acc;
            }
        const double a = C2[0] + kBlur, b = C2[1], cc = C2[3] + kBlur;
        const double det = a * cc - b * b;
        if (!(det > 0.0)) continue;
        const double u = cam->fx * tx / tz + cam->cx;
        const double v = cam->fy * ty / tz + cam->cy;
        // support: alpha >= 1/255 <=> d^T conic d <= K = 2 ln(255 o); the
        // ellipse's axis-aligned bounding box has half-widths sqrt(K a), sqrt(K c)
        const double K = 2.0 * std::log(255.0 * opac);
        const double hx = std::sqrt(K * a) + kRectMargin;
        const double hy = std::sqrt(K * cc) + kRectMargin;
        // float32 error model (see above)
        {
            const double uu = kU32;
            double m[3] = {0.0, 0.0, 0.0};
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 3; ++k) m[r] += std::fabs(cam->R[3 * r + k] * d[k]);
            const double t3[3] = {tx, ty, tz};
            // plain and compensated view vector; near the renderer's switch
            // (sum |R_2k d_k| = 8 t_z) the larger of the two
            double et[3];
            const bool comp = m[2] > 8.0 * tz * (1.0 + 1e-5);
            const bool plain = m[2] < 8.0 * tz * (1.0 - 1e-5);
            for (int r = 0; r < 3; ++r) {
                const double ep = 6.0 * uu * m[r];
                const double ec_ = 2.0 * uu * std::fabs(t3[r]) + 12.0 * uu * uu * m[r];
                et[r] = comp ? ec_ : plain ? ep : std::max(ep, ec_);
            }
            const double etx = et[0], ety = et[1], etz = et[2];
            const double rz = etz / tz;
            const double eu = cam->fx / tz * (etx + std::fabs(tx) * (3.0 * uu + rz)) + uu * std::fabs(u);
            const double ev = cam->fy / tz * (ety + std::fabs(ty) * (3.0 * uu + rz)) + uu * std::fabs(v);
            // rows of T = J W: relative errors of their coefficients and the
            // bounds of the entry errors
            const double ax = cam->fx / tz, bx = cam->fx * std::fabs(tx) / (tz * tz);
            const double ay = cam->fy / tz, by = cam->fy * std::fabs(ty) / (tz * tz);
            const double r_ax = 2.0 * uu + rz, r_ay = r_ax;
            const double r_bx = 5.0 * uu + 2.0 * rz + (std::fabs(tx) > 0.0 ? etx / std::fabs(tx) : 0.0);
            const double r_by = 5.0 * uu + 2.0 * rz + (std::fabs(ty) > 0.0 ? ety / std::fabs(ty) : 0.0);
            const double tau0 = ax * r_ax + bx * r_bx + 2.0 * uu * (ax + bx);
            const double tau1 = ay * r_ay + by * r_by + 2.0 * uu * (ay + by);
            const int32_t par = sc->parent[g];
            const bool blended = blend && par >= 0 &&
                                 orc_blend_parent_weight(orc_granularity_f32(sc, cam, g),
                                                         orc_granularity_f32(sc, cam, par),
                                                         (float)cam->tau) > 0.0f;
            double eb, ec, ea, edet;
            if (!blended) {
                // the Gaussian's axes (columns of R(q)) and scales
                double w = sc->quat[4 * g], x = sc->quat[4 * g + 1], y = sc->quat[4 * g + 2],
                       z = sc->quat[4 * g + 3];
                const double nq = std::sqrt(w * w + x * x + y * y + z * z);
                w /= nq; x /= nq; y /= nq; z /= nq;
                const double Rq[9] = {
                    1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
                    2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
                    2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
                double sk[3];
                for (int k = 0; k < 3; ++k) sk[k] = std::exp((double)sc->log_scale[3 * g + k]);
                double q[2][3], dq[2][3];
                const double tau[2] = {tau0, tau1};
                for (int r = 0; r < 2; ++r)
                    for (int k = 0; k < 3; ++k) {
                        double mrk = 0.0, colsum = 0.0, tsum = 0.0, absprod = 0.0;
                        for (int j = 0; j < 3; ++j) {
                            mrk += T[3 * r + j] * Rq[3 * j + k];
                            colsum += std::fabs(Rq[3 * j + k]);
                            tsum += std::fabs(T[3 * r + j]);
                            absprod += std::fabs(T[3 * r + j] * Rq[3 * j + k]);
                        }
                        const double dm = tau[r] * colsum + 8.0 * uu * tsum + 3.0 * uu * absprod;
                        q[r][k] = sk[k] * mrk;
                        dq[r][k] = sk[k] * dm + 5.0 * uu * std::fabs(q[r][k]);
                    }
                double a2 = 0.0, c2 = 0.0, b1 = 0.0, bab = 0.0, dq0 = 0.0, dq1 = 0.0;
                for (int k = 0; k < 3; ++k) {
                    a2 += q[0][k] * q[0][k];
                    c2 += q[1][k] * q[1][k];
                    b1 += q[0][k] * q[1][k];
                    bab += std::fabs(q[0][k] * q[1][k]);
                    dq0 += dq[0][k] * dq[0][k];
                    dq1 += dq[1][k] * dq[1][k];
                }
                ea = 2.0 * std::sqrt(a2 * dq0) + 3.0 * uu * a2 + uu * a;
                ec = 2.0 * std::sqrt(c2 * dq1) + 3.0 * uu * c2 + uu * cc;
                eb = std::sqrt(dq0 * c2) + std::sqrt(a2 * dq1) + 3.0 * uu * bab;
                // determinant: n = T0 x T1 from the row cross products
                const double aa = ax * ay, ab = ax * by, ba = bx * ay;
                const double dn = aa * (r_ax + r_ay + uu) + ab * (r_ax + r_by + uu) +
                                  ba * (r_bx + r_ay + uu) + 4.0 * uu * (aa + ab + ba);
                double n[3];
                for (int j = 0; j < 3; ++j)
                    n[j] = T[(j + 1) % 3] * T[3 + (j + 2) % 3] - T[(j + 2) % 3] * T[3 + (j + 1) % 3];
                const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                double ddet = 0.0, detp = 0.0;
                for (int k = 0; k < 3; ++k) {
                    const double si = sk[(k + 1) % 3] * sk[(k + 2) % 3];
                    double nk = 0.0, nabs = 0.0;
                    for (int j = 0; j < 3; ++j) {
                        nk += n[j] * Rq[3 * j + k];
                        nabs += std::fabs(n[j] * Rq[3 * j + k]);
                    }
                    const double gk = si * nk;
                    const double dg = si * (std::sqrt(3.0) * dn + 8.0 * std::sqrt(3.0) * uu * nn +
                                            3.0 * uu * nabs) + 10.0 * uu * std::fabs(gk);
                    detp += gk * gk;
                    ddet += 2.0 * std::fabs(gk) * dg;
                }
                ddet += 3.0 * uu * detp + kBlur * (ea + ec) + 2.0 * uu * det;
                edet = ddet / det;
            } else {
                // blended covariance (no axes): entries of T Sigma T^T and a c - b^2
                double tr = S[0] + S[4] + S[8];
                double Sp[9];
                orc_cov3d(sc->quat + 4 * par, sc->log_scale + 3 * par, Sp);
                tr += Sp[0] + Sp[4] + Sp[8];
                const double eS = 25.0 * uu * tr;
                double t0 = 0.0, t1 = 0.0, M00 = 0.0, M01 = 0.0, M11 = 0.0, N0 = 0.0, N1 = 0.0;
                for (int k = 0; k < 3; ++k) { t0 += std::fabs(T[k]); t1 += std::fabs(T[3 + k]); }
                for (int j = 0; j < 3; ++j)
                    for (int k = 0; k < 3; ++k) {
                        const double sjk = std::fabs(S[3 * j + k]);
                        M00 += std::fabs(T[j]) * sjk * std::fabs(T[k]);
                        M01 += std::fabs(T[j]) * sjk * std::fabs(T[3 + k]);
                        M11 += std::fabs(T[3 + j]) * sjk * std::fabs(T[3 + k]);
                        N0 += sjk * std::fabs(T[k]);
                        N1 += sjk * std::fabs(T[3 + k]);
                    }
                ea = 2.0 * tau0 * N0 + t0 * t0 * eS + 7.0 * uu * M00 + uu * a;
                ec = 2.0 * tau1 * N1 + t1 * t1 * eS + 7.0 * uu * M11 + uu * cc;
                eb = tau0 * N1 + tau1 * N0 + t0 * t1 * eS + 7.0 * uu * M01 + uu * std::fabs(b);
                edet = (cc * ea + a * ec + 2.0 * std::fabs(b) * eb + 3.0 * uu * (a * cc + b * b)) / det;
            }
            const double eql = 8.0 * uu * std::max(1.0, std::fabs(std::log2(opac)));
            // support half-widths
            const double eK = 2.0 * 6.0 * uu * std::max(1.0, std::fabs(std::log(255.0 * opac)));
            const double ehx = 0.5 * (hx - kRectMargin) * (eK / K + ea / a) + 3.0 * uu * hx;
            const double ehy = 0.5 * (hy - kRectMargin) * (eK / K + ec / cc) + 3.0 * uu * hy;
            o[PC_EU] = kErrSafety * eu; o[PC_EV] = kErrSafety * ev;
            o[PC_EB] = kErrSafety * eb; o[PC_EC] = kErrSafety * ec;
            o[PC_EDET] = kErrSafety * edet; o[PC_EQL] = kErrSafety * eql;
            o[PC_EHX] = kErrSafety * ehx; o[PC_EHY] = kErrSafety * ehy;
        }
        int32_t x0 = (int32_t)std::floor((u - hx) / tile_w);
        int32_t x1 = (int32_t)std::floor((u + hx) / tile_w);
        int32_t y0 = (int32_t)std::floor((v - hy) / tile_h);
        int32_t y1 = (int32_t)std::floor((v + hy) / tile_h);
        x0 = std::max(x0, 0); y0 = std::max(y0, 0);
        x1 = std::min(x1, tiles_x - 1); y1 = std::min(y1, tiles_y - 1);
        // centre and support box are kept even when no tile is touched, so a
        // comparison can tell which rectangles sit on a tile boundary
        o[PC_U] = u; o[PC_V] = v; o[PC_HX] = hx; o[PC_HY] = hy; o[PC_DEPTH] = tz;
        if (x0 > x1 || y0 > y1) continue;
        // colour: SH evaluated at the world-space direction camera -> mean
        double dir[3], nd = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) dir[k] = d[k] / nd;
        double Y[16];
        orc_sh_basis(dir, Y);
        double rgb[3];
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < 16; ++k) acc += Y[k] * shg[3 * k + ch];
            rgb[ch] = std::max(0.0, acc + 0.5);
        }
        o[PC_VISIBLE] = 1.0;
        o[PC_U] = u; o[PC_V] = v;
        o[PC_CONIC_A] = cc / det; o[PC_CONIC_B] = -b / det; o[PC_CONIC_C] = a / det;
        o[PC_COV_A] = a; o[PC_COV_B] = b; o[PC_COV_C] = cc;
        o[PC_DEPTH] = tz; o[PC_OPACITY] = opac;
        o[PC_R] = rgb[0]; o[PC_G] = rgb[1]; o[PC_B] = rgb[2];
        o[PC_HX] = hx; o[PC_HY] = hy;
        std::memcpy(&depth_key[i], &z32, 4);
        rc[0] = x0; rc[1] = y0; rc[2] = x1; rc[3] = y1;
    }
}

// ---------------------------------------------------------------------------
// 3. binning
// ---------------------------------------------------------------------------

int64_t orc_count_pairs(const int32_t *rect, int64_t n) {
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *r = rect + 4 * i;
        if (r[2] >= r[0] && r[3] >= r[1]) p += (int64_t)(r[2] - r[0] + 1) * (r[3] - r[1] + 1);
    }
    return p;
}

// Emits one pair per (slot, overlapped tile) in slot order and, within a slot,
// row-major tile order; key = tile << 32 | depth_key, value = slot. The pairs
// are then stably sorted by key and ranges[t] = [first, end) of tile t.
void orc_bin_pairs(const int32_t *rect, const uint32_t *depth_key, int64_t n, int32_t tiles_x,
                   int32_t tiles_y, uint64_t *keys, uint32_t *vals, int64_t *ranges) {
    std::vector<std::pair<uint64_t, uint32_t>> pr;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t *r = rect + 4 * i;
        for (int32_t ty = r[1]; ty <= r[3]; ++ty)
            for (int32_t tx = r[0]; tx <= r[2]; ++tx) {
                const uint64_t tile = (uint64_t)ty * tiles_x + tx;
                pr.push_back({(tile << 32) | depth_key[i], (uint32_t)i});
            }
    }
    std::stable_sort(pr.begin(), pr.end(),
                     [](const std::pair<uint64_t, uint32_t> &a,
                        const std::pair<uint64_t, uint32_t> &b) { return a.first < b.first; });
    const int64_t ntiles = (int64_t)tiles_x * tiles_y;
    for (int64_t t = 0; t < ntiles; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    for (size_t k = 0; k < pr.size(); ++k) {
        keys[k] = pr[k].first;
        vals[k] = pr[k].second;
        const int64_t t = (int64_t)(pr[k].first >> 32);
        if (k == 0 || (pr[k - 1].first >> 32) != (uint64_t)t) ranges[2 * t] = (int64_t)k;
        ranges[2 * t + 1] = (int64_t)k + 1;
    }
}

// ---------------------------------------------------------------------------
// 4./5. compositing
// ---------------------------------------------------------------------------

// Bound E_q on how far a float32 renderer's exponent q = log2(o G) of
// Gaussian g at the pixel offset (dx, dy) may lie from the float64 value (the
// error model above; g's error columns are filled by the preprocess).
static double exponent_error(const double *g, double dx, double dy) {
    const double k = 0.5 * kLog2e;
    const double a = g[PC_COV_A], b = g[PC_COV_B], c = g[PC_COV_C];
    const double det = a * c - b * b;
    const double l11 = std::sqrt(c / det), l21 = -b / std::sqrt(c * det), l22 = 1.0 / std::sqrt(c);
    const double p = l11 * dx + l21 * dy, e = l22 * dy;
    const double uu = kU32;
    const double ec = g[PC_EC] / c, ed = g[PC_EDET];
    // errors of the factors (relative errors of c and det scale them, b's
    // moves l21), then of the two squared terms at the pixel
    const double dl11 = l11 * (0.5 * ec + 0.5 * ed + 3.0 * uu);
    const double dl21 = std::fabs(l21) * (0.5 * ec + 0.5 * ed + 3.0 * uu) + g[PC_EB] / std::sqrt(c * det);
    const double dl22 = l22 * (0.5 * ec + 2.0 * uu);
    const double big = std::fabs(l11 * dx) + std::fabs(l21 * dy);
    const double e_fac = k * (2.0 * std::fabs(p) * (dl11 * std::fabs(dx) + dl21 * std::fabs(dy)) +
                              2.0 * e * e * dl22 / l22);
    // centre: q moves by its gradient times the centre error
    const double e_ctr = 2.0 * k * (std::fabs(p) * l11 * g[PC_EU] +
                                    std::fabs(p * l21 + e * l22) * g[PC_EV]);
    // evaluation relative to a reference column up to 16 px away
    const double pw = std::fabs(l11) * (std::fabs(dx) + 16.0) + std::fabs(l21 * dy);
    const double L = std::log2(g[PC_OPACITY]);
    const double e_eval = 8.0 * uu * (k * (pw * pw + e * e + 2.0 * std::fabs(p) * big) + std::fabs(L));
    return e_fac + e_ctr + e_eval + g[PC_EQL] + 2e-6;
}

static const double kLog2AlphaMin = -7.9943534368588578;   // log2(1/255)
static const double kEqMax = 2.0;                           // log2 units: a factor 4 in alpha

// exponent_error for one preprocess row (exported for the tests that pin it)
double orc_exponent_error(const double *g, double dx, double dy) {
    return exponent_error(g, dx, dy);
}

// One front-to-back walk of a pixel's list (step 4), in float64, from list
// position k with transmittance T (relative float32 error bound relT) and
// colour C. At position k the threshold and stop decisions may be forced
// (force_pass / force_stop: -1 = take the float64 decision, 0/1 = the given
// outcome). When `alts` is given, every near-threshold decision met on the way
// also spawns the walk that takes it the other way, and every walk appends its
// final colour to *alts (at most max_alts; *overflow is set beyond that).
// Returns the number of near-threshold decisions met on this walk.
static int walk_pixel(const double *pre, const uint32_t *list, int64_t len, int64_t k, double px,
                      double py, double T, double relT, const double *C0, int force_pass,
                      int force_stop, std::vector<double> *alts, int max_alts, bool *overflow,
                      double *rgb_out, bool *unchecked) {
    double C[3] = {C0[0], C0[1], C0[2]};
    int near = 0;
    for (; k < len; ++k) {
        const double *g = pre + (int64_t)list[k] * PC_NCOLS;
        const double dx = px - g[PC_U], dy = py - g[PC_V];
        const double power = -0.5 * (g[PC_CONIC_A] * dx * dx + g[PC_CONIC_C] * dy * dy) -
                             g[PC_CONIC_B] * dx * dy;
        const double a = g[PC_OPACITY] * std::exp(power);
        const double q = a > 0.0 ? std::log2(a) : -INFINITY;
        const double eq = exponent_error(g, dx, dy);
        bool pass = a >= kAlphaMin;
        if (force_pass >= 0) {
            pass = force_pass != 0;
        } else if (std::fabs(q - kLog2AlphaMin) <= eq) {
            if (eq > kEqMax) {
                if (unchecked) *unchecked = true;
            } else {
                ++near;
                if (alts) walk_pixel(pre, list, len, k, px, py, T, relT, C, pass ? 0 : 1, -1,
                                     alts, max_alts, overflow, nullptr, unchecked);
            }
        }
        force_pass = -1;
        if (!pass) {
            force_stop = -1;
            continue;
        }
        // a Gaussian taken against its float64 decision has alpha at the threshold
        const double alpha = std::max(std::min(kAlphaMax, a), a < kAlphaMin ? kAlphaMin : 0.0);
        const double test_T = T * (1.0 - alpha);
        // relative float32 error of T (1 - alpha): T's, alpha's through 1 - alpha, rounding
        const double rel = relT + alpha * M_LN2 * eq / (1.0 - alpha) + 2.0 * kU32;
        bool stop = test_T < kTMin;
        if (force_stop >= 0) {
            stop = force_stop != 0;
        } else if (std::fabs(test_T - kTMin) <= kTMin * rel) {
            ++near;
            if (alts) walk_pixel(pre, list, len, k, px, py, T, relT, C, 1, stop ? 0 : 1, alts,
                                 max_alts, overflow, nullptr, unchecked);
        }
        force_stop = -1;
        if (stop) break;
        C[0] += alpha * T * g[PC_R];
        C[1] += alpha * T * g[PC_G];
        C[2] += alpha * T * g[PC_B];
        T = test_T;
        relT = rel;
    }
    if (alts) {
        if ((int)(alts->size() / 3) < max_alts) {
            alts->push_back(C[0]); alts->push_back(C[1]); alts->push_back(C[2]);
        } else {
            *overflow = true;
        }
    }
    if (rgb_out) { rgb_out[0] = C[0]; rgb_out[1] = C[1]; rgb_out[2] = C[2]; }
    return near;
}

// Blends the Gaussians list[0..len) (slots into the preprocess table, front to
// back) at pixel centre (px, py), every decision in float64. Returns the flag:
// 1 when some threshold or stop decision on the way was near threshold (a
// float32 renderer may take it the other way; orc_alternatives lists the
// outcomes), 2 when a near-threshold decision's bound exceeded kEqMax (the
// outcomes are not enumerated), else 0.
static int blend_pixel(const double *pre, const uint32_t *list, int64_t len, double px, double py,
                       double *rgb_out, int64_t *n_used) {
    const double zero[3] = {0.0, 0.0, 0.0};
    bool unchecked = false;
    const int near = walk_pixel(pre, list, len, 0, px, py, 1.0, 0.0, zero, -1, -1, nullptr, 0,
                                nullptr, rgb_out, &unchecked);
    if (n_used) *n_used = 0;
    return unchecked ? 2 : near > 0 ? 1 : 0;
}

// Tiled compositing. image: [3][H][W] float64, flags: [H][W].
void orc_composite_tiled(const double *pre, const uint32_t *vals, const int64_t *ranges,
                         int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                         double *image, uint8_t *flags) {
    const int32_t tiles_x = (width + tile_w - 1) / tile_w;
    const int32_t tiles_y = (height + tile_h - 1) / tile_h;
    const int64_t hw = (int64_t)width * height;
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < (int64_t)tiles_x * tiles_y; ++t) {
        const int32_t tx = (int32_t)(t % tiles_x), ty = (int32_t)(t / tiles_x);
        const int64_t r0 = ranges[2 * t], r1 = ranges[2 * t + 1];
        for (int32_t ly = 0; ly < tile_h; ++ly)
            for (int32_t lx = 0; lx < tile_w; ++lx) {
                const int32_t x = tx * tile_w + lx, y = ty * tile_h + ly;
                if (x >= width || y >= height) continue;
                double rgb[3];
                const int f = blend_pixel(pre, vals + r0, r1 - r0, x + 0.5, y + 0.5, rgb, nullptr);
                const int64_t p = (int64_t)y * width + x;
                image[p] = rgb[0]; image[hw + p] = rgb[1]; image[2 * hw + p] = rgb[2];
                if (flags) flags[p] = (uint8_t)f;
            }
    }
}

// Brute force: every visible slot, ordered by (depth_key, slot), at every
// requested pixel; no tiles, no rectangles. pix: [npix][2] (x, y) integer pixel
// coordinates; out: [npix][3]; flags: [npix].
void orc_render_bruteforce(const double *pre, const uint32_t *depth_key, int64_t n,
                           const int32_t *pix, int64_t npix, double *out, uint8_t *flags) {
    std::vector<uint32_t> order;
    for (int64_t i = 0; i < n; ++i)
        if (pre[i * PC_NCOLS + PC_VISIBLE] != 0.0) order.push_back((uint32_t)i);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return depth_key[a] < depth_key[b]; });
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        double rgb[3];
        const int f = blend_pixel(pre, order.data(), (int64_t)order.size(), pix[2 * p] + 0.5,
                                  pix[2 * p + 1] + 0.5, rgb, nullptr);
        out[3 * p] = rgb[0]; out[3 * p + 1] = rgb[1]; out[3 * p + 2] = rgb[2];
        if (flags) flags[p] = (uint8_t)f;
    }
}

// Every outcome of the near-threshold decisions of the tiled compositing at
// the pixels pix[0..npix) ((x, y) integer pairs): for pixel p, n_out[p]
// outcomes (the float64 walk and each combination of near-threshold decisions
// taken the other way, as its walks meet them) in out[p][0..n_out[p])[3]; at
// most max_out, n_out[p] = max_out + 1 when there were more (out holds the
// first max_out). n_out[p] is negated when some decision's bound exceeded
// kEqMax (that decision was taken the float64 way only: unchecked).
void orc_alternatives(const double *pre, const uint32_t *vals, const int64_t *ranges,
                      int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                      const int32_t *pix, int64_t npix, int32_t max_out, double *out,
                      int32_t *n_out) {
    const int32_t tiles_x = (width + tile_w - 1) / tile_w;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        const int32_t x = pix[2 * p], y = pix[2 * p + 1];
        const int64_t t = (int64_t)(y / tile_h) * tiles_x + x / tile_w;
        const int64_t r0 = ranges[2 * t], r1 = ranges[2 * t + 1];
        std::vector<double> alts;
        bool overflow = false, unchecked = false;
        const double zero[3] = {0.0, 0.0, 0.0};
        walk_pixel(pre, vals + r0, r1 - r0, 0, x + 0.5, y + 0.5, 1.0, 0.0, zero, -1, -1, &alts,
                   max_out, &overflow, nullptr, &unchecked);
        const int n = (int)(alts.size() / 3);
        for (int k = 0; k < 3 * n; ++k) out[(int64_t)p * max_out * 3 + k] = alts[k];
        n_out[p] = overflow ? max_out + 1 : n;
        if (unchecked) n_out[p] = -n_out[p];
    }
}

// The float64 view depth of a mean: R_2 . (mu - c) (the depth that orders
// Gaussians front to back; no rounding beyond float64).
double orc_view_depth64(const float *mu, const orc_camera *cam) {
    double z = 0.0;
    for (int k = 0; k < 3; ++k) z += cam->R[6 + k] * ((double)mu[k] - cam->pos[k]);
    return z;
}

// ---------------------------------------------------------------------------
// 6. GS-slice occupancy (Sec. III-C, Eqs. for G3D, Sigma3D^-1, G2D, alpha/beta,
//    lambda and mu(z); derivation in the supplementary section)
// ---------------------------------------------------------------------------
//
// A horizontal plane at height z cuts the 3D Gaussian
// G3D(x) = exp(-1/2 (x - mu)^T Sigma^-1 (x - mu)), Sigma^-1 = [[cxx cxy cxz],
// [cxy cyy cyz], [cxz cyz czz]], in the 2D Gaussian
//   G2D(x, z) = exp(-1/2 lambda (z - mu_z)^2) exp(-1/2 [x - mu(z)]^T C [x - mu(z)])
// with C = [[cxx cxy], [cxy cyy]], (alpha, beta) solving C (alpha, beta)^T =
// (cxz, cyz)^T, lambda = czz - alpha^2 cxx - beta^2 cyy - 2 alpha beta cxy and
// mu(z) = (mu_x, mu_y) - (z - mu_z) (alpha, beta). (Readings: the second
// exponent carries the factor -1/2, as the derivation implies; the printed
// "(y' + beta y')" is (y' + beta z').)

// The slice of one Gaussian: out[0..9] = alpha, beta, lambda, C (cxx, cxy, cyy),
// and Sigma^-1 (cxz, cyz, czz), from Sigma^-1 = R S^-2 R^T.
void orc_slice_params(const float *quat, const float *log_scale, double *out) {
    double w = quat[0], x = quat[1], y = quat[2], z = quat[3];
    const double nq = std::sqrt(w * w + x * x + y * y + z * z);
    w /= nq; x /= nq; y /= nq; z /= nq;
    const double R[9] = {
        1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
        2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
        2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
    double is2[3];
    for (int k = 0; k < 3; ++k) is2[k] = std::exp(-2.0 * (double)log_scale[k]);
    double c[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * is2[k] * R[3 * j + k];
            c[3 * i + j] = acc;
        }
    const double cxx = c[0], cxy = c[1], cxz = c[2], cyy = c[4], cyz = c[5], czz = c[8];
    const double det = cxx * cyy - cxy * cxy;
    const double alpha = (cxz * cyy - cyz * cxy) / det;
    const double beta = (cyz * cxx - cxz * cxy) / det;
    const double lambda = czz - alpha * alpha * cxx - beta * beta * cyy - 2.0 * alpha * beta * cxy;
    const double o[9] = {alpha, beta, lambda, cxx, cxy, cyy, cxz, cyz, czz};
    for (int k = 0; k < 9; ++k) out[k] = o[k];
}

// Slice value of Gaussian g at (x, y) on the plane at height z:
// o G2D(x, z) (before the 0.99 cap and the 1/255 cut-off).
double orc_slice_value(const orc_scene *sc, int64_t g, double x, double y, double z) {
    double p[9];
    orc_slice_params(sc->quat + 4 * g, sc->log_scale + 3 * g, p);
    const double zp = z - sc->pos[3 * g + 2];
    const double mx = sc->pos[3 * g] - zp * p[0], my = sc->pos[3 * g + 1] - zp * p[1];
    const double dx = x - mx, dy = y - my;
    const double q2 = p[3] * dx * dx + 2.0 * p[4] * dx * dy + p[5] * dy * dy;
    return sc->opacity[g] * std::exp(-0.5 * p[2] * zp * zp) * std::exp(-0.5 * q2);
}

// Occupancy grid of the leaves (child_count 0): value[k][j][i] = the largest
// a = min(0.99, o G2D(c_ij, z_k)) over the leaves with a >= 1/255 (0 if none),
// c_ij = (x0 + (i + 1/2) cell, y0 + (j + 1/2) cell), z_k = z0 + k dz;
// occ = value >= threshold. Each slice is visited over the cells of the bounding
// box of its support ellipse (exactly where a >= 1/255), widened by 1e-9 m.
void orc_slice_occupancy(const orc_scene *sc, double x0, double y0, double cell, int32_t nx,
                         int32_t ny, double z0, double dz, int32_t nz, double threshold,
                         double *value, uint8_t *occ) {
    const int64_t plane = (int64_t)nx * ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t k = 0; k < nz; ++k) {
        double *vk = value + k * plane;
        for (int64_t c = 0; c < plane; ++c) vk[c] = 0.0;
        const double z = z0 + k * dz;
        for (int64_t g = 0; g < sc->n; ++g) {
            if (sc->child_count[g] != 0) continue;
            const double o = sc->opacity[g];
            if (255.0 * o < 1.0) continue;
            const double K = 2.0 * std::log(255.0 * o);   // a >= 1/255 <=> exponent sum <= K
            double p[9];
            orc_slice_params(sc->quat + 4 * g, sc->log_scale + 3 * g, p);
            const double zp = z - sc->pos[3 * g + 2];
            const double rem = K - p[2] * zp * zp;
            if (rem < 0.0) continue;
            const double det = p[3] * p[5] - p[4] * p[4];
            const double hx = std::sqrt(rem * p[5] / det) + 1e-9;
            const double hy = std::sqrt(rem * p[3] / det) + 1e-9;
            const double mx = sc->pos[3 * g] - zp * p[0], my = sc->pos[3 * g + 1] - zp * p[1];
            // cells whose centre lies in [m - h, m + h]
            const int64_t i0 = std::max<int64_t>(0, (int64_t)std::ceil((mx - hx - x0) / cell - 0.5));
            const int64_t i1 = std::min<int64_t>(nx - 1, (int64_t)std::floor((mx + hx - x0) / cell - 0.5));
            const int64_t j0 = std::max<int64_t>(0, (int64_t)std::ceil((my - hy - y0) / cell - 0.5));
            const int64_t j1 = std::min<int64_t>(ny - 1, (int64_t)std::floor((my + hy - y0) / cell - 0.5));
            for (int64_t j = j0; j <= j1; ++j)
                for (int64_t i = i0; i <= i1; ++i) {
                    const double dx = x0 + (i + 0.5) * cell - mx, dy = y0 + (j + 0.5) * cell - my;
                    const double q2 = p[3] * dx * dx + 2.0 * p[4] * dx * dy + p[5] * dy * dy;
                    const double a = o * std::exp(-0.5 * (p[2] * zp * zp + q2));
                    if (a < kAlphaMin) continue;
                    const double v = std::min(kAlphaMax, a);
                    if (v > vk[j * nx + i]) vk[j * nx + i] = v;
                }
        }
        if (occ)
            for (int64_t c = 0; c < plane; ++c) occ[k * plane + c] = vk[c] >= threshold ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// 7. Navigable map, shortest-path distance fields and paths (Sec. III-C: the
//    slices give the navigable area for collision checks and path planning;
//    Sec. IV-A: trajectories from a shortest-path planner)
// ---------------------------------------------------------------------------
//
// blocked(i, j): some plane k in [k_lo, k_hi] (the robot's height range) is
// occupied at a cell within Chebyshev distance `inflate` of (i, j) (the robot's
// footprint). Distance field of a goal: breadth-first 4-connected steps over
// free cells (UINT32_MAX where unreachable, blocked, or when the goal itself is
// blocked). A path from a start cell descends the field one step at a time,
// taking the first neighbour in the order (+x, -x, +y, -y) whose distance is
// one less, until the goal.

static const uint32_t kUnreached = 0xFFFFFFFFu;

void orc_nav_blocked(const uint8_t *occ, int32_t nx, int32_t ny, int32_t k_lo, int32_t k_hi,
                     int32_t inflate, uint8_t *blocked) {
    const int64_t plane = (int64_t)nx * ny;
    std::vector<uint8_t> any(plane, 0);
    for (int32_t k = k_lo; k <= k_hi; ++k)
        for (int64_t c = 0; c < plane; ++c) any[c] |= occ[k * plane + c];
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            uint8_t b = 0;
            for (int32_t dj = -inflate; dj <= inflate && !b; ++dj)
                for (int32_t di = -inflate; di <= inflate && !b; ++di) {
                    const int32_t a = i + di, c = j + dj;
                    if (a >= 0 && a < nx && c >= 0 && c < ny && any[(int64_t)c * nx + a]) b = 1;
                }
            blocked[(int64_t)j * nx + i] = b;
        }
}

void orc_nav_field(const uint8_t *blocked, int32_t nx, int32_t ny, int32_t gi, int32_t gj,
                   uint32_t *dist) {
    const int64_t plane = (int64_t)nx * ny;
    for (int64_t c = 0; c < plane; ++c) dist[c] = kUnreached;
    if (gi < 0 || gi >= nx || gj < 0 || gj >= ny || blocked[(int64_t)gj * nx + gi]) return;
    std::vector<int64_t> q;
    q.reserve(plane);
    dist[(int64_t)gj * nx + gi] = 0;
    q.push_back((int64_t)gj * nx + gi);
    for (size_t h = 0; h < q.size(); ++h) {
        const int64_t c = q[h];
        const int32_t i = (int32_t)(c % nx), j = (int32_t)(c / nx);
        const int32_t ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
        for (int e = 0; e < 4; ++e) {
            if (ni[e] < 0 || ni[e] >= nx || nj[e] < 0 || nj[e] >= ny) continue;
            const int64_t n = (int64_t)nj[e] * nx + ni[e];
            if (blocked[n] || dist[n] != kUnreached) continue;
            dist[n] = dist[c] + 1;
            q.push_back(n);
        }
    }
}

// Writes the path's cells (i, j) from the start to the goal into path
// [max_len][2]; returns its length (0 if the start is unreachable; at most
// max_len cells are written).
int32_t orc_nav_path(const uint32_t *dist, int32_t nx, int32_t ny, int32_t si, int32_t sj,
                     int32_t max_len, int32_t *path) {
    if (si < 0 || si >= nx || sj < 0 || sj >= ny) return 0;
    uint32_t d = dist[(int64_t)sj * nx + si];
    if (d == kUnreached) return 0;
    int32_t i = si, j = sj, len = 0;
    for (;;) {
        if (len < max_len) { path[2 * len] = i; path[2 * len + 1] = j; }
        ++len;
        if (d == 0 || len >= max_len) break;
        const int32_t ni[4] = {i + 1, i - 1, i, i}, nj[4] = {j, j, j + 1, j - 1};
        for (int e = 0; e < 4; ++e) {
            if (ni[e] < 0 || ni[e] >= nx || nj[e] < 0 || nj[e] >= ny) continue;
            if (dist[(int64_t)nj[e] * nx + ni[e]] == d - 1) { i = ni[e]; j = nj[e]; break; }
        }
        --d;
    }
    return std::min(len, max_len);
}

// ---------------------------------------------------------------------------
// 8. Frustum-culled and shared cuts (Sec. III-B: Gaussians are taken from the
//    tree's levels per view, dynamically)
// ---------------------------------------------------------------------------
//
// View volume of a camera with a guard band of g pixels:
//     {x : t_z >= 0.2, -g <= u <= W + g, -g <= v <= H + g},
// t = R (x - pos), u = fx t_x / t_z + cx, v = fy t_y / t_z + cy. Where t_z > 0
// it is the intersection of five half-spaces m_k . t + b_k >= 0:
//     near   m = (0, 0, 1), b = -0.2
//     left   m = (fx, 0, cx + g)          right  m = (-fx, 0, W + g - cx)
//     top    m = (0, fy, cy + g)          bottom m = (0, -fy, H + g - cy)
// (u >= -g  <=>  fx t_x + (cx + g) t_z >= 0, and so on). In world terms
// P_k(x) = a_k . (x - pos) + b_k with a_k = R^T m_k. A node is culled when its
// box lies wholly outside one half-space: max over the box of P_k < 0, the
// maximum of a linear function over a box being the sum over the axes of the
// larger of its values at the two faces. Boxes nest, so a culled node's
// subtree is culled.
//
// Shared cut of a group G of cameras (cull on or off): n is fine enough for G
// when every member c culls n (cull on) or has s_c(n) <= tau_c; n is selected
// iff (leaf or fine(n)) and (root or not fine(parent)) and, with the cull on,
// some member keeps n. "fine" only grows towards the leaves (boxes nest, so
// s_c shrinks and culls spread downwards), so the selection is an antichain;
// on each root-to-leaf path it is the deepest of the members' own choices.

static void frustum_planes(const orc_camera *cam, double guard, double a[5][3], double b[5]) {
    const double W = cam->width, H = cam->height;
    const double m[5][3] = {{0.0, 0.0, 1.0},
                            {cam->fx, 0.0, cam->cx + guard},
                            {-cam->fx, 0.0, W + guard - cam->cx},
                            {0.0, cam->fy, cam->cy + guard},
                            {0.0, -cam->fy, H + guard - cam->cy}};
    for (int k = 0; k < 5; ++k) {
        for (int i = 0; i < 3; ++i)
            a[k][i] = m[k][0] * cam->R[i] + m[k][1] * cam->R[3 + i] + m[k][2] * cam->R[6 + i];
        b[k] = k == 0 ? -kNear : 0.0;
    }
}

// Bit 0: culled; bit 1: a plane's value lies within 1e-5 of its scale
// (sum_i |a_ki| max(|lo_i - p_i|, |hi_i - p_i|) + |b_k|) and no plane culls the
// box by more than that, so the float32 renderer may decide either way.
static int frustum_state(const orc_scene *sc, const orc_camera *cam, const double a[5][3],
                         const double b[5], int64_t n) {
    bool culled = false, sure_cull = false, unsure = false;
    for (int k = 0; k < 5; ++k) {
        double mx = b[k], scale = std::fabs(b[k]);
        for (int i = 0; i < 3; ++i) {
            const double dl = (double)sc->aabb_min[3 * n + i] - cam->pos[i];
            const double dh = (double)sc->aabb_max[3 * n + i] - cam->pos[i];
            mx += std::max(a[k][i] * dl, a[k][i] * dh);
            scale += std::fabs(a[k][i]) * std::max(std::fabs(dl), std::fabs(dh));
        }
        if (mx < 0.0) culled = true;
        if (mx < -1e-5 * scale) sure_cull = true;
        if (std::fabs(mx) <= 1e-5 * scale) unsure = true;
    }
    return (culled ? 1 : 0) | (unsure && !sure_cull ? 2 : 0);
}

void orc_frustum_state(const orc_scene *sc, const orc_camera *cam, double guard, uint8_t *out) {
    double a[5][3], b[5];
    frustum_planes(cam, guard, a, b);
    for (int64_t n = 0; n < sc->n; ++n) out[n] = (uint8_t)frustum_state(sc, cam, a, b, n);
}

// Group g is cams[group_begin[g] .. group_begin[g + 1]). Writes the groups'
// cuts (ascending ids, group after group) to ids_out and their offsets to
// offsets_out[0 .. n_groups]; returns the total. near_out (optional,
// [n_groups][n]): 1 where, for some member, s(n) or s(parent) lies within
// 1e-5 relative of tau, or the cull of n or of its parent is unsure.
int64_t orc_select_cut_shared(const orc_scene *sc, const orc_camera *cams,
                              const int32_t *group_begin, int32_t n_groups, int32_t frustum,
                              double guard, int32_t *ids_out, int64_t *offsets_out,
                              uint8_t *near_out) {
    const int64_t n = sc->n;
    std::vector<uint8_t> fine(n), seen(n), unsure(n);
    int64_t cnt = 0;
    for (int32_t g = 0; g < n_groups; ++g) {
        offsets_out[g] = cnt;
        std::fill(fine.begin(), fine.end(), 1);
        std::fill(seen.begin(), seen.end(), frustum ? 0 : 1);
        std::fill(unsure.begin(), unsure.end(), 0);
        for (int32_t c = group_begin[g]; c < group_begin[g + 1]; ++c) {
            const orc_camera *cam = &cams[c];
            double a[5][3], b[5];
            frustum_planes(cam, guard, a, b);
            for (int64_t i = 0; i < n; ++i) {
                const double s = granularity(sc, cam, i);
                bool culled = false;
                if (frustum) {
                    const int st = frustum_state(sc, cam, a, b, i);
                    culled = st & 1;
                    if (st & 2) unsure[i] = 1;
                }
                if (!culled) seen[i] = 1;
                if (!culled && !(s <= cam->tau)) fine[i] = 0;
                if (std::fabs(s - cam->tau) <= 1e-5 * cam->tau) unsure[i] = 1;
            }
        }
        for (int64_t i = 0; i < n; ++i) {
            const bool leaf = sc->child_count[i] == 0;
            const int32_t par = sc->parent[i];
            if ((leaf || fine[i]) && (par < 0 || !fine[par]) && seen[i]) ids_out[cnt++] = (int32_t)i;
            if (near_out) near_out[(int64_t)g * n + i] = (unsure[i] || (par >= 0 && unsure[par])) ? 1 : 0;
        }
    }
    offsets_out[n_groups] = cnt;
    return cnt;
}

int32_t orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

// Threads of the parallel loops from now on (n >= 1; used to time the oracle
// single-threaded and on every core).
void orc_set_threads(int32_t n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

}  // extern "C"
