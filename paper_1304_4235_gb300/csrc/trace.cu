// Column tracing (Sec. 3.2 and Eq. colden): for each (origin particle,
// HEALPix direction) the segment r_i + t n_k, t in [0, l_ray], is walked
// through the LBVH and every smoothing sphere it crosses adds
//   A_j x_j * int W(q) du      (A_j = sigma_th m_j/m_p (8/pi) / h_j^2)
// with the line integral in closed form: the M4 spline of Eq. spline via
// antiderivatives of q, q^2, q^3 along the chord, or the truncated Gaussian
// of Eq. Gt via the erf form I(h,b,z1,z2).
//
// Work distribution: a persistent grid; each warp takes tasks of 32
// Morton-consecutive origins in one direction from an atomic queue, so the
// 32 rays of a warp are parallel and start close together.  The warp walks
// the tree as one packet: a child is entered when any lane's segment crosses
// its box (warp vote), so every lane follows the same path and stack and the
// node fetches are broadcasts; at a leaf each lane tests its own segment
// against the leaf's spheres.  The packet visits the union of the lanes'
// nodes (a beam about as wide as the 32 origins' spread, comparable to h),
// in exchange for uniform control flow.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace urchin {

namespace {

struct TraceParams {
    const float2* ktab;           // [kKTab + 1] full-chord M4 table (value, slope x dt)
    const float4* nodes;
    int n_nodes;
    int n;
    const float4* xyzh;
    const float* w32;
    const double* w64;
    const double* dirs;
    int R;
    double l_ray;
    const int32_t* items;
    int64_t n_items;
    int64_t row_stride, k_stride;
    const int32_t* out_row;
    void* out;
    unsigned* counter;
    unsigned* status;
    unsigned long long* hits;
    int periodic;
    double Lbox;
    int nimg;
    float root_lo[3], root_hi[3];
    double gt_t2, gt_t, gt_pref;
    int64_t n_chunks;
    // stored-segment modes
    uint32_t* counts;             // MODE_COUNT: hits per ray, index k * n_items + item
    const uint64_t* row_ptr;      // MODE_FILL: first segment of each ray (same index), size + 1
    int32_t* seg_col;             // MODE_FILL: Morton index of the particle, or NULL:
    uint16_t* seg_lo;             //   its low 16 bits
    uint8_t* seg_hi;              //   and high 8 bits (indices below 2^24)
    void* seg_val;                // MODE_FILL: A_j * chord integral (float or double)
    const float* A32;
    const double* A64;
    // transpose mode
    const void* coef;             // MODE_SCATTER: coefficient of each ray, indexed like out
    double* xbar;                 // MODE_SCATTER: xbar[j] += coef * A_j * chord integral (Morton)
    const int32_t* order;         // [R * n_items] per-direction item order, or NULL
    // near/far split
    void* out_near;               // [slot + k * near_k_stride] near column (x = 1)
    int64_t near_k_stride;
};

constexpr int MODE_TAU = 0, MODE_COUNT = 1, MODE_FILL = 2, MODE_SCATTER = 3;

// Where a ray's hits go: the running column sum, and in MODE_FILL the
// cursor into the ray's stored segment list.
template <typename Real>
struct Sink {
    Real sum, comp;
    unsigned nhit, ntest;
    int64_t pos, end;
    Real coef;                    // MODE_SCATTER
    Real near, near_c;            // near/far: near column and its compensation
    double ox, oy, oz;            // near/far: shifted origin in double (the near test)
    uint32_t lo_pend, hi_pend;    // MODE_FILL, split indices: halves / bytes of the current word
};

// Near/far split (Sec. 3.3.3): particle j is near the ray's origin when the
// origin lies inside j's smoothing sphere.  For a crossed sphere that is the
// case exactly when its chord starts before the origin, tc - ch < 0 (the
// origin at distance^2 = tc^2 + b^2 < h^2); that test decides unless the
// origin sits within rounding of the sphere's surface, where the distance is
// compared in double from the float positions (the differences are exact),
// like the reference definition, so both sides classify every pair alike.
template <typename Real>
__device__ __forceinline__ bool is_near(const Sink<Real>& k, float4 q, Real tc, Real ch)
{
    const Real gap = tc - ch;
    if (fabs((double)gap) > 1e-4 * (double)q.w) return gap < Real(0);
    const double ex = (double)q.x - k.ox, ey = (double)q.y - k.oy, ez = (double)q.z - k.oz;
    const double hh = (double)q.w;
    return ex * ex + ey * ey + ez * ez < hh * hh;
}

template <typename Real> struct RealOps;
template <> struct RealOps<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float erf_(float x) { return erff(x); }
    static __device__ __forceinline__ float weight(const TraceParams& P, int j) { return __ldg(P.w32 + j); }
};
template <> struct RealOps<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double erf_(double x) { return erf(x); }
    static __device__ __forceinline__ double weight(const TraceParams& P, int j) { return __ldg(P.w64 + j); }
};

// ---- M4 chord integrals in units of h -------------------------------------
// With q = sqrt(beta^2 + a^2) and L(a) = asinh(a/beta) = ln(a + q) - ln(beta):
//   inner piece (q <= 1/2), integrand 1 - 6q^2 + 6q^3:
//     Fi(a) = a(1 - 6b2 - 2a^2) + 3/2 a q^3 + 9/4 b2 a q + 9/4 b2^2 L
//   outer piece (1/2 < q <= 1), integrand 2(1-q)^3:
//     Fo(a) = a(2 + 6b2 + 2a^2) - 3 a q - 1/2 a q^3 - 3/4 b2 a q - (3 b2 + 3/4 b2^2) L
// and the odd antiderivative from 0 is H(a) = Fi(a) for a <= s, else
// Fo(a) + Fi(s) - Fo(s) with s = sqrt(1/4 - b2) (b2 < 1/4), where
//   Fi(s) - Fo(s) = -s(1/4 + 13/2 b2) + (3 b2 + 3 b2^2) L(s).
// At the chord end a = c = sqrt(1 - b2) (q = 1):
//   Fo(c) = c(1/2 + 13/4 b2) - (3 b2 + 3/4 b2^2) L(c).
template <typename Real>
__device__ __forceinline__ Real m4_join(Real b2, Real lb, Real& s_out)
{
    using O = RealOps<Real>;
    Real s = O::sqrt_(Real(0.25) - b2);
    s_out = s;
    Real Ls = b2 > Real(0) ? O::log_(s + Real(0.5)) - lb : Real(0);
    return -s * (Real(0.25) + Real(6.5) * b2) + (Real(3) * b2 + Real(3) * b2 * b2) * Ls;
}

template <typename Real>
__device__ __forceinline__ Real m4_full(Real b2, Real c)
{
    using O = RealOps<Real>;
    Real lb = b2 > Real(0) ? Real(0.5) * O::log_(b2) : Real(0);
    Real Lc = b2 > Real(0) ? O::log_(c + Real(1)) - lb : Real(0);
    Real H = c * (Real(0.5) + Real(3.25) * b2) - (Real(3) * b2 + Real(0.75) * b2 * b2) * Lc;
    if (b2 < Real(0.25)) {
        Real s;
        H += m4_join(b2, lb, s);
    }
    return Real(2) * H;
}

template <typename Real>
__device__ __forceinline__ Real m4_H(Real b2, Real lb, Real a)
{
    using O = RealOps<Real>;
    Real q = O::sqrt_(b2 + a * a);
    Real La = b2 > Real(0) ? O::log_(a + q) - lb : Real(0);
    Real q3 = q * q * q;
    if (b2 < Real(0.25)) {
        Real s;
        Real join = m4_join(b2, lb, s);
        if (a <= s)
            return a * (Real(1) - Real(6) * b2 - Real(2) * a * a) + Real(1.5) * a * q3 +
                   Real(2.25) * b2 * a * q + Real(2.25) * b2 * b2 * La;
        return a * (Real(2) + Real(6) * b2 + Real(2) * a * a) - Real(3) * a * q - Real(0.5) * a * q3 -
               Real(0.75) * b2 * a * q - (Real(3) * b2 + Real(0.75) * b2 * b2) * La + join;
    }
    return a * (Real(2) + Real(6) * b2 + Real(2) * a * a) - Real(3) * a * q - Real(0.5) * a * q3 -
           Real(0.75) * b2 * a * q - (Real(3) * b2 + Real(0.75) * b2 * b2) * La;
}

template <typename Real>
__device__ __forceinline__ Real m4_part(Real b2, Real u1, Real u2)
{
    using O = RealOps<Real>;
    Real lb = b2 > Real(0) ? Real(0.5) * O::log_(b2) : Real(0);
    Real g2 = u2 >= Real(0) ? m4_H(b2, lb, u2) : -m4_H(b2, lb, -u2);
    Real g1 = u1 >= Real(0) ? m4_H(b2, lb, u1) : -m4_H(b2, lb, -u1);
    return g2 - g1;
}

// ---- truncated Gaussian (Eq. Gt, I(h,b,z1,z2)) ----------------------------
template <typename Real>
__device__ __forceinline__ Real gt_chord(const TraceParams& P, Real b2, Real u1, Real u2)
{
    using O = RealOps<Real>;
    Real t = Real(P.gt_t);
    return Real(P.gt_pref) * O::exp_(-Real(P.gt_t2) * b2) * (O::erf_(t * u2) - O::erf_(t * u1));
}

// ---- FP32 chord evaluation ------------------------------------------------
// The antiderivatives above lose about two digits in FP32 over the outer
// spline piece (terms of order 4 cancel to the small value of 2(1-q)^3), so
// the FP32 path evaluates
//   * full chords from a table of K(t) = int W du over the whole chord,
//     t = b^2/h^2, with cubic Hermite interpolation (values and slopes at
//     kKTab + 1 nodes, built on the host in double and staged in shared
//     memory), and
//   * partial chords piece by piece: the inner piece (q <= 1/2) by the
//     antiderivative Fi (well conditioned), the outer piece by 8-point
//     Gauss-Legendre quadrature of 2(1-q)^3, a smooth non-negative
//     integrand on [s, c].
__device__ __forceinline__ float m4_full_tab(const float2* tab, float t)
{
    float x = fminf(t, 1.0f) * (float)kKTab;
    int i = min((int)x, kKTab - 1);
    float f = x - (float)i;
    float2 a = tab[i], b = tab[i + 1];
    float f2 = f * f, f3 = f2 * f;
    return (2.f * f3 - 3.f * f2 + 1.f) * a.x + (f3 - 2.f * f2 + f) * a.y + (3.f * f2 - 2.f * f3) * b.x +
           (f3 - f2) * b.y;
}

__device__ __forceinline__ float m4_inner_prim_f(float b2, float a)
{
    float q = sqrtf(b2 + a * a);
    float L = b2 > 0.f ? logf(a + q) - 0.5f * logf(b2) : 0.f;
    return a * (1.f - 6.f * b2 - 2.f * a * a) + 1.5f * a * q * q * q + 2.25f * b2 * a * q + 2.25f * b2 * b2 * L;
}

// Gauss-Legendre nodes and weights on [-1, 1], n = 8
__constant__ float kGLx[8] = {-0.9602898564975363f, -0.7966664774136267f, -0.5255324099163290f,
                              -0.1834346424956498f, 0.1834346424956498f,  0.5255324099163290f,
                              0.7966664774136267f,  0.9602898564975363f};
__constant__ float kGLw[8] = {0.1012285362903763f, 0.2223810344533745f, 0.3137066458778873f,
                              0.3626837833783620f, 0.3626837833783620f, 0.3137066458778873f,
                              0.2223810344533745f, 0.1012285362903763f};

__device__ __forceinline__ float m4_outer_gl(float b2, float a1, float a2)
{
    const float m = 0.5f * (a1 + a2), r = 0.5f * (a2 - a1);
    float acc = 0.f;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        float u = fmaf(r, kGLx[g], m);
        float v = 1.f - sqrtf(fmaf(u, u, b2));
        acc = fmaf(kGLw[g], v * v * v, acc);
    }
    return 2.f * r * acc;
}

// int_{a1}^{a2} M4shape du for 0 <= a1 < a2 <= c
__device__ __forceinline__ float m4_piece_f(float b2, float a1, float a2)
{
    const float s = b2 < 0.25f ? sqrtf(0.25f - b2) : 0.f;
    float r = 0.f;
    if (a1 < s) r += m4_inner_prim_f(b2, fminf(a2, s)) - m4_inner_prim_f(b2, a1);
    const float lo = fmaxf(a1, s);
    if (a2 > lo) r += m4_outer_gl(b2, lo, a2);
    return r;
}

__device__ __forceinline__ float m4_part_f(float b2, float u1, float u2)
{
    float t = 0.f;
    if (u1 < 0.f) t += m4_piece_f(b2, fmaxf(0.f, -u2), -u1);
    if (u2 > 0.f) t += m4_piece_f(b2, fmaxf(0.f, u1), u2);
    return t;
}

// a*b - c*d with one rounding (Kahan's difference of products via FMA)
__device__ __forceinline__ float dop(float a, float b, float c, float d)
{
    float w = c * d;
    float e = fmaf(-c, d, w);
    float f = fmaf(a, b, -w);
    return f + e;
}

struct Kahan {
    __device__ __forceinline__ static void add(float& s, float& c, float v)
    {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ static void add(double& s, double& c, double v)
    {
        double y = v - c;
        double t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Segment [0, L] of o + t d against an axis-aligned box (float slab test).
__device__ __forceinline__ bool seg_box(float ox, float oy, float oz, float ix, float iy, float iz,
                                        float L, float4 lo, float4 hi)
{
    float tx0 = (lo.x - ox) * ix, tx1 = (hi.x - ox) * ix;
    float ty0 = (lo.y - oy) * iy, ty1 = (hi.y - oy) * iy;
    float tz0 = (lo.z - oz) * iz, tz1 = (hi.z - oz) * iz;
    float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), L));
    return tn <= tf;
}

__device__ __forceinline__ float safe_inv(double d)
{
    return fabs(d) > 1e-20 ? (float)(1.0 / d) : copysignf(1e30f, (float)d);
}

// Particle index of stored segment pos: an int32, or split into 16 + 8 bits.
// A lane writes its ray's segments at consecutive positions from a multiple
// of 8 to a multiple of 8 (the padding), so the split halves and bytes are
// gathered in the sink and written as whole 32-bit words.
template <typename Real>
__device__ __forceinline__ void store_index(const TraceParams& P, Sink<Real>& k, int64_t pos, int j)
{
    if (P.seg_col) {
        P.seg_col[pos] = j;
        return;
    }
    const uint32_t lo = (uint32_t)j & 0xffffu, hi = ((uint32_t)j >> 16) & 0xffu;
    if (pos & 1) reinterpret_cast<uint32_t*>(P.seg_lo)[pos >> 1] = k.lo_pend | (lo << 16);
    else k.lo_pend = lo;
    const int sh = (int)(pos & 3) * 8;
    k.hi_pend = (sh == 0 ? 0u : k.hi_pend) | (hi << sh);
    if ((pos & 3) == 3) reinterpret_cast<uint32_t*>(P.seg_hi)[pos >> 2] = k.hi_pend;
}

// FP32 hit evaluation: cheap rejection, then the impact parameter from an
// error-free cross product, then the tabulated / piecewise chord integral.
template <int KERNEL, int MODE, bool NF>
__device__ __forceinline__ void leaf_hits_f32(const TraceParams& P, const float2* tab, int ref, int cnt,
                                              float sx, float sy, float sz, float dx, float dy, float dz,
                                              float L, Sink<float>& k, unsigned& err)
{
    if (ref < 0 || cnt > kLeafMax || ref + cnt > P.n) return;   // never true for a well-formed tree
    k.ntest += (unsigned)cnt;
    for (int j = ref; j < ref + cnt; ++j) {
        float4 q = __ldg(P.xyzh + j);
        float ex = q.x - sx, ey = q.y - sy, ez = q.z - sz;
        float cx = ey * dz - ez * dy, cy = ez * dx - ex * dz, cz = ex * dy - ey * dx;
        float h2 = q.w * q.w;
        if (cx * cx + cy * cy + cz * cz >= 1.0001f * h2) continue;
        cx = dop(ey, dz, ez, dy);
        cy = dop(ez, dx, ex, dz);
        cz = dop(ex, dy, ey, dx);
        float b2 = cx * cx + cy * cy + cz * cz;
        if (b2 >= h2) continue;
        float tc = ex * dx + ey * dy + ez * dz;
        float ch = sqrtf(h2 - b2);
        if (tc + ch <= 0.f || tc - ch >= L) continue;
        const bool near = NF && is_near(k, q, tc, ch);
        if (!near) ++k.nhit;
        if (MODE == MODE_COUNT) continue;
        float ih = 1.f / q.w;
        float beta2 = b2 * ih * ih;
        float F;
        if (tc - ch >= 0.f && tc + ch <= L) {
            if (KERNEL == URCHIN_KERNEL_M4) F = m4_full_tab(tab, beta2);
            else F = gt_chord<float>(P, beta2, -ch * ih, ch * ih);
        } else {
            float u1 = (fmaxf(0.f, tc - ch) - tc) * ih;
            float u2 = (fminf(L, tc + ch) - tc) * ih;
            if (KERNEL == URCHIN_KERNEL_M4) F = m4_part_f(beta2, u1, u2);
            else F = gt_chord<float>(P, beta2, u1, u2);
        }
        if (MODE == MODE_SCATTER) {
            atomicAdd(P.xbar + j, (double)(k.coef * (__ldg(P.A32 + j) * F)));
            continue;
        }
        if (near) {
            Kahan::add(k.near, k.near_c, __ldg(P.A32 + j) * F);
            continue;
        }
        Kahan::add(k.sum, k.comp, __ldg(P.w32 + j) * F);
        if (MODE == MODE_FILL) {
            if (k.pos < k.end) {
                store_index(P, k, k.pos, j);
                static_cast<float*>(P.seg_val)[k.pos] = __ldg(P.A32 + j) * F;
                ++k.pos;
            } else {
                err |= kStSegment;
            }
        }
    }
}

template <typename Real, int KERNEL, int MODE, bool NF>
__device__ __forceinline__ void leaf_hits(const TraceParams& P, int ref, int cnt, Real sx, Real sy, Real sz,
                                          Real dx, Real dy, Real dz, Real L, Sink<Real>& k, unsigned& err)
{
    using O = RealOps<Real>;
    if (ref < 0 || cnt > kLeafMax || ref + cnt > P.n) return;   // never true for a well-formed tree
    k.ntest += (unsigned)cnt;
    for (int j = ref; j < ref + cnt; ++j) {
        float4 q = __ldg(P.xyzh + j);
        Real ex = Real(q.x) - sx, ey = Real(q.y) - sy, ez = Real(q.z) - sz;
        Real tc = ex * dx + ey * dy + ez * dz;
        Real cx = ey * dz - ez * dy, cy = ez * dx - ex * dz, cz = ex * dy - ey * dx;
        Real b2 = cx * cx + cy * cy + cz * cz;
        Real h = Real(q.w);
        Real h2 = h * h;
        if (b2 >= h2) continue;
        Real ch = O::sqrt_(h2 - b2);
        if (tc + ch <= Real(0) || tc - ch >= L) continue;
        const bool near = NF && is_near(k, q, tc, ch);
        if (!near) ++k.nhit;
        if (MODE == MODE_COUNT) continue;
        Real ih = Real(1) / h;
        Real beta2 = b2 * ih * ih;
        Real F;
        if (tc - ch >= Real(0) && tc + ch <= L) {
            Real c = ch * ih;
            if (KERNEL == URCHIN_KERNEL_M4) F = m4_full(beta2, c);
            else F = gt_chord(P, beta2, -c, c);
        } else {
            Real u1 = (fmax(Real(0), tc - ch) - tc) * ih;
            Real u2 = (fmin(L, tc + ch) - tc) * ih;
            if (KERNEL == URCHIN_KERNEL_M4) F = m4_part(beta2, u1, u2);
            else F = gt_chord(P, beta2, u1, u2);
        }
        if (MODE == MODE_SCATTER) {
            const Real A = sizeof(Real) == 4 ? Real(__ldg(P.A32 + j)) : Real(__ldg(P.A64 + j));
            atomicAdd(P.xbar + j, (double)(k.coef * (A * F)));
            continue;
        }
        if (near) {
            const Real A = sizeof(Real) == 4 ? Real(__ldg(P.A32 + j)) : Real(__ldg(P.A64 + j));
            Kahan::add(k.near, k.near_c, A * F);
            continue;
        }
        Kahan::add(k.sum, k.comp, O::weight(P, j) * F);
        if (MODE == MODE_FILL) {
            if (k.pos < k.end) {
                store_index(P, k, k.pos, j);
                const Real A = sizeof(Real) == 4 ? Real(__ldg(P.A32 + j)) : Real(__ldg(P.A64 + j));
                static_cast<Real*>(P.seg_val)[k.pos] = A * F;
                ++k.pos;
            } else {
                err |= kStSegment;
            }
        }
    }
}

template <typename Real, int KERNEL, int MODE, bool NF>
__device__ void ray_column(const TraceParams& P, const float2* tab, float4 o, Real dx, Real dy, Real dz,
                           bool live, Sink<Real>& sk, unsigned& err, unsigned& nvisit)
{
    const Real L = Real(P.l_ray);
    const float Lf = (float)P.l_ray * 1.000001f + 1e-30f;
    const float ix = safe_inv((double)dx), iy = safe_inv((double)dy), iz = safe_inv((double)dz);
    const int nimg = P.periodic ? P.nimg : 0;
    const float4 rlo = make_float4(P.root_lo[0], P.root_lo[1], P.root_lo[2], 0.f);
    const float4 rhi = make_float4(P.root_hi[0], P.root_hi[1], P.root_hi[2], 0.f);
    int stack[kStackMax];
    for (int ax = -nimg; ax <= nimg; ++ax)
    for (int ay = -nimg; ay <= nimg; ++ay)
    for (int az = -nimg; az <= nimg; ++az) {
        // images of the particles at r_j + a L are reached by shifting the
        // origin to r_i - a L
        Real sx = Real(o.x) - Real(ax) * Real(P.Lbox);
        Real sy = Real(o.y) - Real(ay) * Real(P.Lbox);
        Real sz = Real(o.z) - Real(az) * Real(P.Lbox);
        float fx = (float)sx, fy = (float)sy, fz = (float)sz;
        if (!__any_sync(0xffffffffu, live && seg_box(fx, fy, fz, ix, iy, iz, Lf, rlo, rhi))) continue;
        if (NF) {
            sk.ox = (double)o.x - (double)ax * P.Lbox;
            sk.oy = (double)o.y - (double)ay * P.Lbox;
            sk.oz = (double)o.z - (double)az * P.Lbox;
        }
        int sp = 0;
        int node = 0;
        // a traversal visits every internal node at most once; the cap only
        // guards against a malformed tree
        int budget = P.n_nodes + 1;
        for (;;) {
            if (--budget < 0) {
                err |= kStVisit;
                break;
            }
            if ((unsigned)node >= (unsigned)P.n_nodes) {   // never true for a well-formed tree
                err |= kStVisit;
                break;
            }
            ++nvisit;
            const float4* nd = P.nodes + 4 * (int64_t)node;
            float4 a = __ldg(nd), b = __ldg(nd + 1), c = __ldg(nd + 2), d = __ldg(nd + 3);
            int lref = __float_as_int(a.w), lcnt = __float_as_int(b.w);
            int rref = __float_as_int(c.w), rcnt = __float_as_int(d.w);
            bool hl = __any_sync(0xffffffffu, live && seg_box(fx, fy, fz, ix, iy, iz, Lf, a, b));
            bool hr = __any_sync(0xffffffffu, live && rcnt >= 0 && seg_box(fx, fy, fz, ix, iy, iz, Lf, c, d));
            if (hl && lcnt > 0) {
                if (live) {
                    if constexpr (sizeof(Real) == 4)
                        leaf_hits_f32<KERNEL, MODE, NF>(P, tab, lref, lcnt, sx, sy, sz, dx, dy, dz, L, sk, err);
                    else
                        leaf_hits<Real, KERNEL, MODE, NF>(P, lref, lcnt, sx, sy, sz, dx, dy, dz, L, sk, err);
                }
                hl = false;
            }
            if (hr && rcnt > 0) {
                if (live) {
                    if constexpr (sizeof(Real) == 4)
                        leaf_hits_f32<KERNEL, MODE, NF>(P, tab, rref, rcnt, sx, sy, sz, dx, dy, dz, L, sk, err);
                    else
                        leaf_hits<Real, KERNEL, MODE, NF>(P, rref, rcnt, sx, sy, sz, dx, dy, dz, L, sk, err);
                }
                hr = false;
            }
            if (hl && hr) {
                if (sp < kStackMax) stack[sp++] = rref;
                else err |= kStStack;
                node = lref;
            } else if (hl) {
                node = lref;
            } else if (hr) {
                node = rref;
            } else {
                if (sp == 0) break;
                node = stack[--sp];
            }
        }
    }
}

template <typename Real, int KERNEL, int MODE, bool NF>
__global__ void __launch_bounds__(256) k_trace(TraceParams P)
{
    extern __shared__ double s_dirs[];
    float2* s_tab = reinterpret_cast<float2*>(s_dirs + 3 * P.R);
    for (int t = threadIdx.x; t < 3 * P.R; t += blockDim.x) s_dirs[t] = P.dirs[t];
    if (sizeof(Real) == 4 && KERNEL == URCHIN_KERNEL_M4)
        for (int t = threadIdx.x; t <= kKTab; t += blockDim.x) s_tab[t] = P.ktab[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long total = (unsigned long long)P.n_chunks * (unsigned long long)P.R;
    unsigned err = 0;
    unsigned long long hits = 0, tests = 0, visits = 0;
    for (;;) {
        unsigned task = 0;
        if (lane == 0) task = atomicAdd(P.counter, 1u);
        task = __shfl_sync(0xffffffffu, task, 0);
        if ((unsigned long long)task >= total) break;
        const int k = (int)(task / P.n_chunks);
        const int64_t chunk = (int64_t)(task % P.n_chunks);
        const int64_t slot = chunk * 32 + lane;
        // every lane takes part in the packet's votes; lanes past the end of
        // the origin list (and, in the transpose, rays with a zero
        // coefficient) are carried along without a segment
        bool live = slot < P.n_items;
        const int64_t item = !live ? 0 : (P.order ? (int64_t)P.order[(int64_t)k * P.n_items + slot] : slot);
        const int32_t org = live ? (P.items ? P.items[item] : (int32_t)item) : 0;
        float4 o = __ldg(P.xyzh + org);
        Real dx = Real(s_dirs[3 * k]), dy = Real(s_dirs[3 * k + 1]), dz = Real(s_dirs[3 * k + 2]);
        unsigned nvisit = 0;
        Sink<Real> sk{Real(0), Real(0), 0u, 0u, 0, 0, Real(0), Real(0), Real(0), 0.0, 0.0, 0.0};
        const int64_t ray = (int64_t)k * P.n_items + item;
        const int64_t orow = live ? (P.out_row ? (int64_t)P.out_row[item] : item) : 0;
        if (live && MODE == MODE_FILL) {
            sk.pos = (int64_t)P.row_ptr[ray];
            sk.end = (int64_t)P.row_ptr[ray + 1];
        }
        if (live && MODE == MODE_SCATTER) {
            sk.coef = static_cast<const Real*>(P.coef)[orow * P.row_stride + (int64_t)k * P.k_stride];
            live = sk.coef != Real(0);
        }
        ray_column<Real, KERNEL, MODE, NF>(P, s_tab, o, dx, dy, dz, live, sk, err, nvisit);
        if (slot < P.n_items) {
            hits += sk.nhit;
            tests += sk.ntest;
            visits += nvisit;
            if (MODE == MODE_COUNT) {
                P.counts[ray] = (sk.nhit + (unsigned)kSegPad - 1u) / (unsigned)kSegPad * (unsigned)kSegPad;
            } else if (MODE != MODE_SCATTER) {
                if (MODE == MODE_FILL) {
                    // the padding (fewer than kSegPad entries) holds zero values
                    if (sk.end - sk.pos >= kSegPad || sk.pos > sk.end) err |= kStSegment;
                    else
                        for (int64_t q = sk.pos; q < sk.end; ++q) {
                            store_index(P, sk, q, 0);
                            static_cast<Real*>(P.seg_val)[q] = Real(0);
                        }
                }
                static_cast<Real*>(P.out)[orow * P.row_stride + (int64_t)k * P.k_stride] = sk.sum;
                if (NF) {
                    const int64_t at = P.near_k_stride > 0 ? (int64_t)org + (int64_t)k * P.near_k_stride
                                                           : orow * P.row_stride + (int64_t)k * P.k_stride;
                    static_cast<Real*>(P.out_near)[at] = sk.near;
                }
            }
        }
    }
    if (err && P.status) atomicOr(P.status, err);
    if (P.hits) {
        for (int o = 16; o > 0; o >>= 1) {
            hits += __shfl_xor_sync(0xffffffffu, hits, o);
            tests += __shfl_xor_sync(0xffffffffu, tests, o);
            visits += __shfl_xor_sync(0xffffffffu, visits, o);
        }
        if (lane == 0) {
            atomicAdd(P.hits, hits);
            atomicAdd(P.hits + 1, tests);
            atomicAdd(P.hits + 2, visits);
        }
    }
}

template <typename Real, int KERNEL, int MODE, bool NF>
int launch_one(const TraceParams& P, cudaStream_t s)
{
    const void* fn = (const void*)k_trace<Real, KERNEL, MODE, NF>;
    const size_t smem = sizeof(double) * 3 * (size_t)P.R +
                        ((sizeof(Real) == 4 && KERNEL == URCHIN_KERNEL_M4) ? sizeof(float2) * (kKTab + 1) : 0);
    int grid = 0;
    URCHIN_TRY(grid_for(fn, 256, smem, &grid));
    int64_t tasks = P.n_chunks * P.R;
    int64_t need = (tasks + 7) / 8;       // 8 warps per block
    if (need < grid) grid = (int)std::max<int64_t>(need, 1);
    k_trace<Real, KERNEL, MODE, NF><<<grid, 256, smem, s>>>(P);
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

template <typename Real, int KERNEL>
int dispatch_k(const TraceParams& P, int mode, bool nf, cudaStream_t s)
{
    if (nf) {
        if (mode == MODE_COUNT) return launch_one<Real, KERNEL, MODE_COUNT, true>(P, s);
        if (mode == MODE_FILL) return launch_one<Real, KERNEL, MODE_FILL, true>(P, s);
        if (mode == MODE_SCATTER) return set_error(URCHIN_ERR_ARG, "trace: no transpose with the near/far split");
        return launch_one<Real, KERNEL, MODE_TAU, true>(P, s);
    }
    if (mode == MODE_COUNT) return launch_one<Real, KERNEL, MODE_COUNT, false>(P, s);
    if (mode == MODE_FILL) return launch_one<Real, KERNEL, MODE_FILL, false>(P, s);
    if (mode == MODE_SCATTER) return launch_one<Real, KERNEL, MODE_SCATTER, false>(P, s);
    return launch_one<Real, KERNEL, MODE_TAU, false>(P, s);
}

int dispatch_mode(const TraceParams& P, int precision, int kernel, int mode, bool nf, cudaStream_t s)
{
    if (precision == URCHIN_F64) {
        if (kernel == URCHIN_KERNEL_GT) return dispatch_k<double, URCHIN_KERNEL_GT>(P, mode, nf, s);
        return dispatch_k<double, URCHIN_KERNEL_M4>(P, mode, nf, s);
    }
    if (kernel == URCHIN_KERNEL_GT) return dispatch_k<float, URCHIN_KERNEL_GT>(P, mode, nf, s);
    return dispatch_k<float, URCHIN_KERNEL_M4>(P, mode, nf, s);
}

}  // namespace

// Full-chord M4 integral in double from the antiderivatives above:
// K(t) = 2 H(c), H(c) = Fo(c) [+ Fi(s) - Fo(s) when t < 1/4].
static double m4_full_host(double t)
{
    if (t >= 1.0) return 0.0;
    const double c = std::sqrt(1.0 - t);
    const double lb = t > 0.0 ? 0.5 * std::log(t) : 0.0;
    const double Lc = t > 0.0 ? std::log(c + 1.0) - lb : 0.0;
    double H = c * (0.5 + 3.25 * t) - (3.0 * t + 0.75 * t * t) * Lc;
    if (t < 0.25) {
        const double sv = std::sqrt(0.25 - t);
        const double Ls = t > 0.0 ? std::log(sv + 0.5) - lb : 0.0;
        H += -sv * (0.25 + 6.5 * t) + (3.0 * t + 3.0 * t * t) * Ls;
    }
    return 2.0 * H;
}

void m4_full_table(float2* out)
{
    const double h = 1e-5;
    for (int i = 0; i <= kKTab; ++i) {
        const double t = (double)i / kKTab;
        double d;
        if (t < 2 * h) d = (-3.0 * m4_full_host(t) + 4.0 * m4_full_host(t + h) - m4_full_host(t + 2 * h)) / (2 * h);
        else if (t > 1.0 - 2 * h) d = (3.0 * m4_full_host(t) - 4.0 * m4_full_host(t - h) + m4_full_host(t - 2 * h)) / (2 * h);
        else d = (m4_full_host(t + h) - m4_full_host(t - h)) / (2 * h);
        out[i] = make_float2((float)m4_full_host(t), (float)(d / kKTab));
    }
}

int launch_trace(const TraceJob& job, cudaStream_t s)
{
    if (job.n_items <= 0) return URCHIN_OK;
    const urchin_bvh* b = job.bvh;
    TraceParams P;
    P.ktab = b->ktab;
    P.nodes = b->nodes;
    P.n_nodes = b->n_nodes;
    P.n = (int)b->n;
    P.xyzh = b->xyzh;
    P.w32 = job.w32;
    P.w64 = job.w64;
    P.dirs = job.dirs_dev;
    P.R = job.R;
    P.l_ray = job.l_ray;
    P.items = job.items;
    P.n_items = job.n_items;
    P.row_stride = job.row_stride;
    P.k_stride = job.k_stride;
    P.out_row = job.out_row;
    P.out = job.out;
    P.counter = job.counter;
    P.status = job.status;
    P.hits = job.hits;
    P.periodic = b->periodic;
    P.Lbox = b->L;
    // every image within l_ray + h_max of the box can reach the segment
    P.nimg = b->periodic ? (int)std::ceil((job.l_ray + (double)b->hmax) / b->L) : 0;
    for (int a = 0; a < 3; ++a) {
        P.root_lo[a] = b->root_lo[a];
        P.root_hi[a] = b->root_hi[a];
    }
    GtConst g = gt_constants();
    P.gt_t2 = g.t2;
    P.gt_t = g.t;
    P.gt_pref = g.pref;
    P.n_chunks = (job.n_items + 31) / 32;
    if ((unsigned long long)P.n_chunks * (unsigned long long)job.R >= 0xffffffffull)
        return set_error(URCHIN_ERR_ARG, "trace: too many rays for one launch");
    URCHIN_TRY_CUDA(cudaMemsetAsync(job.counter, 0, sizeof(unsigned), s));
    P.counts = job.counts;
    P.row_ptr = job.row_ptr;
    P.seg_col = job.seg_col;
    P.seg_lo = job.seg_lo;
    P.seg_hi = job.seg_hi;
    P.seg_val = job.seg_val;
    P.A32 = b->A32;
    P.A64 = b->A64;
    P.coef = job.coef;
    P.xbar = job.xbar;
    P.order = job.order;
    P.out_near = job.out_near;
    P.near_k_stride = job.near_k_stride;
    if (job.near_far && !job.out_near && job.mode != MODE_COUNT)
        return set_error(URCHIN_ERR_ARG, "trace: near/far split without a near-column output");
    if (job.mode == MODE_FILL && !job.seg_col && !(job.seg_lo && job.seg_hi && b->n <= (int64_t(1) << 24)))
        return set_error(URCHIN_ERR_ARG, "trace: segment fill without a particle-index array");
    return dispatch_mode(P, job.precision, job.kernel, job.mode, job.near_far != 0, s);
}

namespace {

__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t quant10(float f)
{
    return (uint32_t)fminf(fmaxf(f * 1024.f, 0.f), 1023.f);
}

// keys of the items for one direction: Morton code of (u, v, t / E) in the
// frame (e1, e2, d), coordinates relative to c scaled by inv into [0, 1)
__global__ void k_ray_keys(const float4* __restrict__ xyzh, const int32_t* __restrict__ items, int64_t n_items,
                           float3 e1, float3 e2, float3 d, float3 c, float inv, float inv_E, uint32_t* keys,
                           int32_t* vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(xyzh + (items ? items[i] : (int32_t)i));
        const float rx = p.x - c.x, ry = p.y - c.y, rz = p.z - c.z;
        const float u = (rx * e1.x + ry * e1.y + rz * e1.z) * inv + 0.5f;
        const float v = (rx * e2.x + ry * e2.y + rz * e2.z) * inv + 0.5f;
        const float t = (rx * d.x + ry * d.y + rz * d.z) * inv * inv_E + 0.5f;
        keys[i] = (spread10(quant10(u)) << 2) | (spread10(quant10(v)) << 1) | spread10(quant10(t));
        vals[i] = (int32_t)i;
    }
}

}  // namespace

size_t ray_order_tmp_bytes(int64_t n_items)
{
    Layout lay;
    lay.take(sizeof(uint32_t) * (size_t)n_items);
    lay.take(radix_tmp_bytes(n_items));
    return lay.bytes;
}

int ray_order(const urchin_bvh* b, const int32_t* items, int64_t n_items, const double* dirs, int R,
              int32_t* order, void* tmp, cudaStream_t s)
{
    if (n_items <= 0) return URCHIN_OK;
    Layout lay;
    const size_t o_k = lay.take(sizeof(uint32_t) * (size_t)n_items);
    const size_t o_t = lay.take(radix_tmp_bytes(n_items));
    uint32_t* keys = reinterpret_cast<uint32_t*>(static_cast<char*>(tmp) + o_k);
    void* rt = static_cast<char*>(tmp) + o_t;
    const double E = kRayOrderElongation;
    const float3 c = make_float3(0.5f * (b->root_lo[0] + b->root_hi[0]), 0.5f * (b->root_lo[1] + b->root_hi[1]),
                                 0.5f * (b->root_lo[2] + b->root_hi[2]));
    const double ex = b->root_hi[0] - b->root_lo[0], ey = b->root_hi[1] - b->root_lo[1],
                 ez = b->root_hi[2] - b->root_lo[2];
    const double diam = std::sqrt(ex * ex + ey * ey + ez * ez);
    const float inv = (float)(1.0 / std::max(diam, 1e-30));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_items + 255) / 256, 4096));
    for (int k = 0; k < R; ++k) {
        const double dx = dirs[3 * k], dy = dirs[3 * k + 1], dz = dirs[3 * k + 2];
        // e1 perpendicular to d, from the coordinate axis least aligned with it
        double ax = 0, ay = 0, az = 0;
        if (std::fabs(dx) <= std::fabs(dy) && std::fabs(dx) <= std::fabs(dz)) ax = 1;
        else if (std::fabs(dy) <= std::fabs(dz)) ay = 1;
        else az = 1;
        double e1x = dy * az - dz * ay, e1y = dz * ax - dx * az, e1z = dx * ay - dy * ax;
        const double nn = std::sqrt(e1x * e1x + e1y * e1y + e1z * e1z);
        e1x /= nn;
        e1y /= nn;
        e1z /= nn;
        const double e2x = dy * e1z - dz * e1y, e2y = dz * e1x - dx * e1z, e2z = dx * e1y - dy * e1x;
        int32_t* vals = order + (size_t)k * n_items;
        k_ray_keys<<<grid, 256, 0, s>>>(b->xyzh, items, n_items, make_float3((float)e1x, (float)e1y, (float)e1z),
                                        make_float3((float)e2x, (float)e2y, (float)e2z),
                                        make_float3((float)dx, (float)dy, (float)dz), c, inv, (float)(1.0 / E),
                                        keys, vals);
        URCHIN_TRY(launched());
        URCHIN_TRY(radix_sort_pairs(keys, vals, n_items, 30, rt, s));
    }
    return URCHIN_OK;
}

// w[s] = A[s] x[perm[s]]
__global__ void k_weights(const float* __restrict__ A32, const double* __restrict__ A64,
                          const int32_t* __restrict__ perm, const double* __restrict__ x, int64_t n,
                          float* w32, double* w64)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        double xv = x[perm[s]];
        if (w64) w64[s] = A64[s] * xv;
        if (w32) w32[s] = (float)(A64[s] * xv);
    }
}

int launch_weights(const urchin_bvh* b, const double* x_orig, float* w32, double* w64, cudaStream_t s)
{
    unsigned grid = (unsigned)std::min<int64_t>((b->n + 255) / 256, 4096);
    k_weights<<<grid, 256, 0, s>>>(b->A32, b->A64, b->perm, x_orig, b->n, w32, w64);
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

// origins (original indices) -> Morton slots; an index out of range flags
// the status word and maps to slot 0
__global__ void k_map_origins(const int32_t* __restrict__ origins, const int32_t* __restrict__ inv,
                              int64_t n_orig, int64_t n, int32_t* items, unsigned* status)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_orig;
         o += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = origins[o];
        if (i < 0 || i >= n) {
            atomicOr(status, kStOrigin);
            items[o] = 0;
        } else {
            items[o] = inv[i];
        }
    }
}

int launch_map_origins(const urchin_bvh* bvh, const int32_t* origins, int64_t n_orig, int32_t* items,
                       unsigned* status, cudaStream_t s)
{
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_orig + 255) / 256, 4096));
    k_map_origins<<<grid, 256, 0, s>>>(origins, bvh->inv, n_orig, bvh->n, items, status);
    return launched();
}

}  // namespace urchin

namespace urchin {
namespace {

// Argument checks shared by the column entry points (status 1 = valid no-op)
int check_trace_args(const char* fn, const urchin_bvh* bvh, const void* x, const double* dirs, int R, double l_ray,
                     const int32_t* origins, int64_t n_orig, int kernel, int precision, const void* buf)
{
    if (!bvh || !x || !dirs) return set_error(URCHIN_ERR_ARG, "%s: NULL bvh, input or dirs", fn);
    if (R < 1 || R > URCHIN_MAX_RAYS)
        return set_error(URCHIN_ERR_ARG, "%s: R = %d out of range [1, %d]", fn, R, URCHIN_MAX_RAYS);
    if (!(l_ray >= 0.0) || !std::isfinite(l_ray))
        return set_error(URCHIN_ERR_ARG, "%s: l_ray must be finite and >= 0", fn);
    if (kernel != URCHIN_KERNEL_M4 && kernel != URCHIN_KERNEL_GT)
        return set_error(URCHIN_ERR_ARG, "%s: unknown kernel %d", fn, kernel);
    if (precision != URCHIN_F32 && precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "%s: unknown precision %d", fn, precision);
    if (n_orig < 0) return set_error(URCHIN_ERR_ARG, "%s: n_orig < 0", fn);
    if (n_orig == 0) return 1;
    if (!origins && n_orig != bvh->n) return set_error(URCHIN_ERR_ARG, "%s: origins NULL requires n_orig == n", fn);
    if (!buf) return set_error(URCHIN_ERR_ARG, "%s: output or cotangent array is NULL", fn);
    for (int i = 0; i < 3 * R; ++i)
        if (!std::isfinite(dirs[i])) return set_error(URCHIN_ERR_ARG, "%s: non-finite direction", fn);
    for (int k = 0; k < R; ++k) {
        double nn = dirs[3 * k] * dirs[3 * k] + dirs[3 * k + 1] * dirs[3 * k + 1] + dirs[3 * k + 2] * dirs[3 * k + 2];
        if (std::fabs(nn - 1.0) > 1e-6)
            return set_error(URCHIN_ERR_ARG, "%s: direction %d is not a unit vector", fn, k);
    }
    return URCHIN_OK;
}

// x_bar[perm[s]] += xm[s]
__global__ void k_unpermute_add(const int32_t* __restrict__ perm, const double* __restrict__ xm, int64_t n,
                                double* x_bar)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        x_bar[perm[s]] += xm[s];
}

}  // namespace
}  // namespace urchin

namespace urchin {
namespace {

int trace_columns_impl(const char* fn, const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                       double l_ray, const int32_t* origins, int64_t n_orig, int kernel, int precision,
                       void* tau_out, void* near_out, cudaStream_t s)
{
    {
        const int c = check_trace_args(fn, bvh, x, dirs, R, l_ray, origins, n_orig, kernel, precision, tau_out);
        if (c != URCHIN_OK) return c > 0 ? URCHIN_OK : c;
    }
    const int64_t n = bvh->n;
    const bool f64 = precision == URCHIN_F64;
    Layout lay;
    size_t o_ctr = lay.take(2 * sizeof(unsigned));
    size_t o_dirs = lay.take(sizeof(double) * 3 * (size_t)R);
    size_t o_w = lay.take((f64 ? sizeof(double) : sizeof(float)) * (size_t)n);
    size_t o_items = lay.take(origins ? sizeof(int32_t) * (size_t)n_orig : 0);
    const bool ordered = n_orig >= kRayOrderMinItems;
    size_t o_ord = lay.take(ordered ? sizeof(int32_t) * (size_t)R * (size_t)n_orig : 0);
    size_t o_otmp = lay.take(ordered ? ray_order_tmp_bytes(n_orig) : 0);
    Scratch scr;
    URCHIN_TRY(scr.alloc(lay.bytes, s));
    unsigned* ctr = scr.at<unsigned>(o_ctr);
    URCHIN_TRY_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(scr.at<double>(o_dirs), dirs, sizeof(double) * 3 * (size_t)R,
                                    cudaMemcpyHostToDevice, s));
    URCHIN_TRY(launch_weights(bvh, x, f64 ? nullptr : scr.at<float>(o_w), f64 ? scr.at<double>(o_w) : nullptr, s));
    TraceJob job{};
    job.bvh = bvh;
    job.w32 = f64 ? nullptr : scr.at<float>(o_w);
    job.w64 = f64 ? scr.at<double>(o_w) : nullptr;
    job.dirs_dev = scr.at<double>(o_dirs);
    job.R = R;
    job.l_ray = l_ray;
    job.n_items = n_orig;
    job.row_stride = R;
    job.k_stride = 1;
    job.out = tau_out;
    job.kernel = kernel;
    job.precision = precision;
    job.counter = ctr;
    job.status = ctr + 1;
    if (origins) {
        int32_t* items = scr.at<int32_t>(o_items);
        URCHIN_TRY(launch_map_origins(bvh, origins, n_orig, items, ctr + 1, s));
        job.items = items;
        job.out_row = nullptr;
    } else {
        // all particles, in Morton order for coherence; row = original index
        job.items = nullptr;
        job.out_row = bvh->perm;
    }
    if (n_orig >= kRayOrderMinItems) {
        URCHIN_TRY(ray_order(bvh, job.items, n_orig, dirs, R, scr.at<int32_t>(o_ord), scr.at<void>(o_otmp), s));
        job.order = scr.at<int32_t>(o_ord);
    }
    job.near_far = near_out ? 1 : 0;
    job.out_near = near_out;
    job.near_k_stride = 0;                      // same layout as tau_out
    URCHIN_TRY(launch_trace(job, s));
    unsigned st = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&st, ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    scr.release();
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    if (st & kStOrigin) return set_error(URCHIN_ERR_ARG, "%s: origin index out of range", fn);
    if (st & kStStack) return set_error(URCHIN_ERR_CUDA, "%s: traversal stack overflow", fn);
    if (st & kStVisit) return set_error(URCHIN_ERR_CUDA, "%s: malformed tree (visit limit)", fn);
    return URCHIN_OK;
}

}  // namespace
}  // namespace urchin

extern "C" int urchin_trace_columns(const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                                    double l_ray, const int32_t* origins, int64_t n_orig, int kernel,
                                    int precision, void* tau_out, urchin_stream_t stream)
{
    urchin::clear_error();
    return urchin::trace_columns_impl("urchin_trace_columns", bvh, x, dirs, R, l_ray, origins, n_orig, kernel,
                                      precision, tau_out, nullptr, (cudaStream_t)stream);
}

extern "C" int urchin_trace_columns_nearfar(const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                                            double l_ray, const int32_t* origins, int64_t n_orig, int kernel,
                                            int precision, void* tau_far_out, void* tau_near_out,
                                            urchin_stream_t stream)
{
    urchin::clear_error();
    if (n_orig > 0 && !tau_near_out)
        return urchin::set_error(URCHIN_ERR_ARG, "urchin_trace_columns_nearfar: tau_near_out is NULL");
    return urchin::trace_columns_impl("urchin_trace_columns_nearfar", bvh, x, dirs, R, l_ray, origins, n_orig,
                                      kernel, precision, tau_far_out, tau_near_out, (cudaStream_t)stream);
}

extern "C" int urchin_trace_columns_vjp(const urchin_bvh* bvh, const double* dirs, int R, double l_ray,
                                        const int32_t* origins, int64_t n_orig, int kernel, int precision,
                                        const void* tau_bar, double* x_bar, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    {
        const int c = check_trace_args("urchin_trace_columns_vjp", bvh, tau_bar ? tau_bar : (const void*)dirs,
                                       dirs, R, l_ray, origins, n_orig, kernel, precision, x_bar);
        if (c != URCHIN_OK) return c > 0 ? URCHIN_OK : c;
        if (!tau_bar) return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_vjp: tau_bar is NULL");
    }
    const int64_t n = bvh->n;
    Layout lay;
    size_t o_ctr = lay.take(2 * sizeof(unsigned));
    size_t o_dirs = lay.take(sizeof(double) * 3 * (size_t)R);
    size_t o_xm = lay.take(sizeof(double) * (size_t)n);
    size_t o_items = lay.take(origins ? sizeof(int32_t) * (size_t)n_orig : 0);
    Scratch scr;
    URCHIN_TRY(scr.alloc(lay.bytes, s));
    unsigned* ctr = scr.at<unsigned>(o_ctr);
    double* xm = scr.at<double>(o_xm);
    URCHIN_TRY_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), s));
    URCHIN_TRY_CUDA(cudaMemsetAsync(xm, 0, sizeof(double) * (size_t)n, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(scr.at<double>(o_dirs), dirs, sizeof(double) * 3 * (size_t)R,
                                    cudaMemcpyHostToDevice, s));
    TraceJob job{};
    job.bvh = bvh;
    job.dirs_dev = scr.at<double>(o_dirs);
    job.R = R;
    job.l_ray = l_ray;
    job.n_items = n_orig;
    job.row_stride = R;
    job.k_stride = 1;
    job.kernel = kernel;
    job.precision = precision;
    job.counter = ctr;
    job.status = ctr + 1;
    job.mode = 3;
    job.coef = tau_bar;
    job.xbar = xm;
    if (origins) {
        int32_t* items = scr.at<int32_t>(o_items);
        URCHIN_TRY(launch_map_origins(bvh, origins, n_orig, items, ctr + 1, s));
        job.items = items;
        job.out_row = nullptr;
    } else {
        job.items = nullptr;
        job.out_row = bvh->perm;
    }
    URCHIN_TRY(launch_trace(job, s));
    unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
    k_unpermute_add<<<grid, 256, 0, s>>>(bvh->perm, xm, n, x_bar);
    URCHIN_TRY(launched());
    unsigned st = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&st, ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    scr.release();
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    if (st & kStOrigin) return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_vjp: origin index out of range");
    if (st & kStStack) return set_error(URCHIN_ERR_CUDA, "urchin_trace_columns_vjp: traversal stack overflow");
    if (st & kStVisit) return set_error(URCHIN_ERR_CUDA, "urchin_trace_columns_vjp: malformed tree (visit limit)");
    return URCHIN_OK;
}
