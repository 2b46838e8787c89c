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
    // MODE_CHUNK: segment lists in chunks of kChunk entries taken while tracing
    uint32_t* chunk_head;         // [R * n] first chunk of each ray (rays with hits)
    uint32_t* chunk_next;         // [cap] the chunk after each chunk of a ray
    unsigned long long* chunk_counter;   // chunks handed out (may exceed cap: then the lists are incomplete)
    unsigned long long chunk_cap;
    int2* chunk_seg;              // [cap * kChunk] (particle, value bits): one 8-byte store per full chord
};

constexpr int MODE_TAU = 0, MODE_COUNT = 1, MODE_FILL = 2, MODE_SCATTER = 3, MODE_CHUNK = 4;
// MODE_CHUNK: the columns as in MODE_TAU, the hit counts as in MODE_COUNT, and
// every ray's segments stored while tracing, in chunks of kChunk entries that
// the warp takes from a global counter kStash at a time (the counts are not
// known before the traversal); the chunks of a ray are linked through
// chunk_next.  Used by the solver's first sweep, so that a solve of two sweeps
// traces once.
constexpr int kChunk = kChunkEntries;   // entries per chunk (a multiple of kSegPad)
constexpr int kStash = 64;        // chunks a warp takes from the counter at a time

// Where a ray's hits go: the running column sum, and in MODE_FILL the
// cursor into the ray's stored segment list.
template <typename Real>
struct Sink {
    Real sum, comp;               // full chords, in traversal order
    Real psum, pcomp;             // partial chords (FP32 queue), in the ray's queue order
    unsigned nhit, ntest;
    int64_t pos, end;
    Real coef;                    // MODE_SCATTER
    Real near, near_c;            // near/far: near column and its compensation
    double ox, oy, oz;            // near/far: shifted origin in double (the near test)
    uint32_t lo_pend, hi_pend;    // MODE_FILL, split indices: halves / bytes of the current word
    int64_t ray;                  // MODE_CHUNK: row k n + origin slot
    int2* cw;                     // MODE_CHUNK: the ray's current chunk
    int coff;                     // MODE_CHUNK: entries used in it (kChunk: none or full; kChunk + 1: pool exhausted)
    uint32_t cur;                 // MODE_CHUNK: its index (kNoChunk before the first)
};
constexpr uint32_t kNoChunk = 0xffffffffu;

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
    return fma(ez, ez, fma(ey, ey, __dmul_rn(ex, ex))) < __dmul_rn(hh, hh);
}

// Rounded arithmetic the compiler may not contract into multiply-adds.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

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

// int_{a1}^{a2} M4shape(sqrt(b2 + u^2)) du for 0 <= a1 <= a2 <= sqrt(1 - b2):
// the inner piece (q <= 1/2) by its antiderivative Fi (Fi(0) = 0), the
// outer piece by 6-point Gauss-Legendre quadrature of 2(1 - q)^3 (within
// 6e-8 of the integral for every b2 and interval; K(0) = 0.75).  Integrating
// over the interval itself keeps a short piece's relative accuracy (as a
// difference of antiderivatives from 0 it would lose it).
__constant__ float kGL6x[6] = {-0.9324695142031521f, -0.6612093864662645f, -0.2386191860831969f,
                               0.2386191860831969f,  0.6612093864662645f,  0.9324695142031521f};
__constant__ float kGL6w[6] = {0.1713244923791704f, 0.3607615730481386f, 0.4679139345726910f,
                               0.4679139345726910f, 0.3607615730481386f, 0.1713244923791704f};

__device__ __forceinline__ float m4_inner_fi(float b2, float rb, float a)
{
    const float q = sqrtf(fmaf(a, a, b2));
    const float L = b2 > 0.f ? logf((a + q) * rb) : 0.f;
    return a * (1.f - 6.f * b2 - 2.f * a * a) + 1.5f * a * q * q * q + 2.25f * b2 * a * q + 2.25f * b2 * b2 * L;
}

__device__ __forceinline__ float m4_seg_f(float b2, float a1, float a2)
{
    const float s = b2 < 0.25f ? sqrtf(0.25f - b2) : 0.f;
    const float rb = b2 > 0.f ? rsqrtf(b2) : 0.f;
    float r = 0.f;
    if (a1 < s) {
        r = m4_inner_fi(b2, rb, fminf(a2, s));
        if (a1 > 0.f) r -= m4_inner_fi(b2, rb, a1);
    }
    const float lo = fmaxf(a1, s);
    if (a2 > lo) {
        const float m = 0.5f * (lo + a2), h = 0.5f * (a2 - lo);
        float acc = 0.f;
#pragma unroll
        for (int g = 0; g < 6; ++g) {
            const float u = fmaf(h, kGL6x[g], m);
            const float v = 1.f - sqrtf(fmaf(u, u, b2));
            acc = fmaf(kGL6w[g], v * v * v, acc);
        }
        r += 2.f * h * acc;
    }
    return r;
}

// Partial M4 chord over [u1, u2] (units of h, -c <= u1 < u2 <= c).  A chord
// that straddles the closest approach (u1 < 0 < u2) is the sum of its two
// halves, and a half that the segment does not clip is K(b2)/2 from the
// full-chord table, so a chord clipped at one end costs one piece; a chord
// on one side (the segment starts past the closest approach, or ends
// before it) is integrated over its own interval.
__device__ __forceinline__ float m4_part_q(const float2* tab, float b2, float u1, float u2, bool clip_lo,
                                           bool clip_hi)
{
    const bool straddle = u1 < 0.f && u2 > 0.f;
    // the first piece: the clipped half of a straddling chord, or the chord
    float a1 = straddle ? 0.f : fminf(fabsf(u1), fabsf(u2));
    float a2 = straddle ? (clip_hi ? u2 : -u1) : fmaxf(fabsf(u1), fabsf(u2));
    float F = m4_seg_f(b2, a1, a2);
    if (straddle) {
        if (clip_hi && clip_lo) F += m4_seg_f(b2, 0.f, -u1);
        else F += 0.5f * m4_full_tab(tab, b2);
    }
    return F;
}

// a*b - c*d with one rounding (Kahan's difference of products via FMA)
__device__ __forceinline__ float dop(float a, float b, float c, float d)
{
    float w = __fmul_rn(c, d);
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

// ---- the packet's beam ------------------------------------------------------
// The 32 rays of a packet are parallel (one direction d).  In a frame
// (e1, e2, d) anchored at one live lane's origin B, a lane's segment is the
// point (u_i, v_i) across the direction and the depth interval
// [t_i, t_i + l_ray] along it; the beam is the box [u_lo, u_hi] x [v_lo, v_hi]
// of the live lanes' points and the depth range [t_lo, t_hi + l_ray].  A
// particle can only be crossed by some lane if its sphere reaches that box:
// lateral distance from (u_j, v_j) to the box below h_j and depth range
// [t_j - h_j, t_j + h_j] overlapping.  At a leaf, lanes 0..cnt-1 test one
// particle each against the beam (one warp instruction stream for the whole
// leaf) and only the particles that pass are tested per lane.  The test is
// made conservative by a margin of a few float roundings of the coordinates,
// so it never drops a crossing: every lane's hits, and the order in which it
// sums them, are those of the unfiltered loop.
struct Beam {
    float bx, by, bz;             // anchor B
    float e1x, e1y, e1z, e2x, e2y, e2z, dx, dy, dz;
    float ulo, uhi, vlo, vhi, tlo, thi;
    float eps;                    // absolute margin of the projections
};

__device__ __forceinline__ float wmin(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float wmax(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Called by all 32 lanes with the same direction; (fx, fy, fz) is the
// lane's (shifted) origin.  Writes the warp's beam to shared memory (out,
// one per warp) and returns false when no lane is live.
__device__ __forceinline__ bool make_beam(Beam* out, bool live, float fx, float fy, float fz, float dx, float dy,
                                          float dz, float L)
{
    const unsigned lv = __ballot_sync(0xffffffffu, live);
    if (!lv) return false;
    Beam B;
    const int a = __ffs(lv) - 1;
    B.bx = __shfl_sync(0xffffffffu, fx, a);
    B.by = __shfl_sync(0xffffffffu, fy, a);
    B.bz = __shfl_sync(0xffffffffu, fz, a);
    B.dx = dx;
    B.dy = dy;
    B.dz = dz;
    // e1 perpendicular to d, from the coordinate axis least aligned with it
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (fabsf(dx) <= fabsf(dy) && fabsf(dx) <= fabsf(dz)) ax = 1.f;
    else if (fabsf(dy) <= fabsf(dz)) ay = 1.f;
    else az = 1.f;
    float e1x = dy * az - dz * ay, e1y = dz * ax - dx * az, e1z = dx * ay - dy * ax;
    const float inv = rsqrtf(e1x * e1x + e1y * e1y + e1z * e1z);
    e1x *= inv;
    e1y *= inv;
    e1z *= inv;
    B.e1x = e1x;
    B.e1y = e1y;
    B.e1z = e1z;
    B.e2x = dy * e1z - dz * e1y;
    B.e2y = dz * e1x - dx * e1z;
    B.e2z = dx * e1y - dy * e1x;
    const float rx = fx - B.bx, ry = fy - B.by, rz = fz - B.bz;
    const float u = rx * B.e1x + ry * B.e1y + rz * B.e1z;
    const float v = rx * B.e2x + ry * B.e2y + rz * B.e2z;
    const float t = rx * dx + ry * dy + rz * dz;
    B.ulo = wmin(live ? u : INFINITY);
    B.uhi = wmax(live ? u : -INFINITY);
    B.vlo = wmin(live ? v : INFINITY);
    B.vhi = wmax(live ? v : -INFINITY);
    B.tlo = wmin(live ? t : INFINITY);
    B.thi = wmax(live ? t : -INFINITY) + L;
    // roundings of the projections: a few ulp of the coordinates' magnitude
    const float span = fmaxf(fmaxf(B.uhi - B.ulo, B.vhi - B.vlo), B.thi - B.tlo);
    B.eps = 1e-5f * (span + fabsf(B.bx) + fabsf(B.by) + fabsf(B.bz));
    __syncwarp();                    // the previous beam's readers are done
    if ((threadIdx.x & 31) == 0) *out = B;
    __syncwarp();
    return true;
}

// Mask of the leaf's particles (bit l for particle ref + l) that the beam can
// reach.  Every lane calls it; lanes 0..cnt-1 test one particle each.
__device__ __forceinline__ unsigned beam_mask(const TraceParams& P, const Beam& B, int ref, int cnt)
{
    const int lane = threadIdx.x & 31;
    bool pass = false;
    if (lane < cnt && ref >= 0 && cnt <= kLeafMax && ref + cnt <= P.n) {
        const float4 q = __ldg(P.xyzh + ref + lane);
        const float rx = q.x - B.bx, ry = q.y - B.by, rz = q.z - B.bz;
        const float u = rx * B.e1x + ry * B.e1y + rz * B.e1z;
        const float v = rx * B.e2x + ry * B.e2y + rz * B.e2z;
        const float t = rx * B.dx + ry * B.dy + rz * B.dz;
        const float hh = q.w * 1.00001f + B.eps + 1e-5f * (fabsf(rx) + fabsf(ry) + fabsf(rz));
        const float du = fmaxf(fmaxf(B.ulo - u, u - B.uhi), 0.f);
        const float dv = fmaxf(fmaxf(B.vlo - v, v - B.vhi), 0.f);
        pass = du * du + dv * dv < hh * hh && t + hh > B.tlo && t - hh < B.thi;
    }
    return __ballot_sync(0xffffffffu, pass);
}
static_assert(kLeafMax <= 32, "a leaf's particles are filtered one per lane");

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

// ---- deferred partial chords ------------------------------------------------
// A partial chord (a sphere cut by the segment's start or end) takes the
// piecewise evaluation of m4_part_f, an order of magnitude more arithmetic
// than a full chord's table lookup, and with rays of a few smoothing lengths
// most hits are partial (every sphere holding the origin or the end point).
// Evaluated where it is met, a warp would run that code for the few lanes
// whose ray met one.  Instead the warp appends its partial chords to a queue
// in shared memory and evaluates them 32 at a time, one per lane; every ray
// then adds its own results in queue order (the lanes of one ray's items
// found with a match), so the sums stay deterministic.
constexpr int kPQ = 64;           // queue capacity per warp; a round takes 32
constexpr int kPQNear = 32;       // owner flag: a near particle (near/far split)
constexpr int kPQClipLo = 64;     // owner flag: the segment's start cuts the chord
constexpr int kPQClipHi = 128;    // owner flag: the segment's end cuts the chord
struct PartItem {
    float beta2, u1, u2;          // chord in units of h: b^2/h^2 and [u1, u2]
    int j;                        // particle (Morton slot)
    int owner;                    // lane of the ray | kPQNear | kPQClipLo | kPQClipHi
    float coef;                   // MODE_SCATTER: the ray's coefficient
    int64_t pos;                  // MODE_FILL: the segment's position
};
struct PartQueue {
    PartItem item[kPQ];
    float val[32];                // results of the round being flushed
    unsigned own[64];             // per owner (lane, lane + kPQNear): items of the round
};

// Byte offset of the queues in k_trace's dynamic shared memory: after the
// directions (double[3R]) and the FP32 M4 table, 16-byte aligned.
__host__ __device__ __forceinline__ size_t trace_queue_offset(int R, int kernel)
{
    const size_t b = sizeof(double) * 3 * (size_t)R + (kernel == URCHIN_KERNEL_M4 ? sizeof(float2) * (kKTab + 1) : 0);
    return (b + 15) & ~size_t(15);
}

// Evaluate the first n (<= 32) queued chords, one per lane, and move the
// rest to the front.  Every lane of the warp calls it.  Inlined: as a called
// function its reference arguments kept the ray's running state (sums,
// cursor, queue length) in local memory for the whole traversal, which cost
// 7 % of the traversal's time.
template <int KERNEL, int MODE, bool NF>
__device__ __forceinline__ void flush_partials(const TraceParams& P, const float2* tab, PartQueue* pq, int& count,
                                               int n, Sink<float>& k)
{
    const int lane = threadIdx.x & 31;
    int owner = -1;
    float v = 0.f;
    if (lane < n) {
        const PartItem it = pq->item[lane];
        const float F = KERNEL == URCHIN_KERNEL_M4
                            ? m4_part_q(tab, it.beta2, it.u1, it.u2, (it.owner & kPQClipLo) != 0,
                                        (it.owner & kPQClipHi) != 0)
                            : gt_chord<float>(P, it.beta2, it.u1, it.u2);
        const float A = __ldg(P.A32 + it.j);
        if (MODE == MODE_SCATTER) {
            atomicAdd(P.xbar + it.j, (double)(it.coef * (A * F)));
        } else {
            const bool near = NF && (it.owner & kPQNear);
            v = near ? A * F : __ldg(P.w32 + it.j) * F;
            if (MODE == MODE_FILL && !near) static_cast<float*>(P.seg_val)[it.pos] = A * F;
            if (MODE == MODE_CHUNK && it.pos >= 0) P.chunk_seg[it.pos] = make_int2(it.j, __float_as_int(A * F));
            owner = it.owner & (31 | kPQNear);
        }
    }
    if (MODE != MODE_SCATTER) {
        pq->val[lane] = v;
        const unsigned same = __match_any_sync(0xffffffffu, owner);
        if (owner >= 0 && (same & ((1u << lane) - 1u)) == 0u) pq->own[owner] = same;
        __syncwarp();
        for (unsigned m = pq->own[lane]; m; m &= m - 1) Kahan::add(k.psum, k.pcomp, pq->val[__ffs(m) - 1]);
        if (NF)
            for (unsigned m = pq->own[lane + kPQNear]; m; m &= m - 1)
                Kahan::add(k.near, k.near_c, pq->val[__ffs(m) - 1]);
        __syncwarp();
        pq->own[lane] = 0u;
        pq->own[lane + kPQNear] = 0u;
    }
    const int rest = count - n;
    PartItem tail;
    if (lane < rest) tail = pq->item[n + lane];
    __syncwarp();
    if (lane < rest) pq->item[lane] = tail;
    __syncwarp();
    count = rest;
}

// MODE_CHUNK: `want` consecutive chunks from the warp's block of chunks in
// shared memory, a new block of kStash (or more) from the global counter when
// it runs out.  Called by lane 0 with the warp converged.
__device__ __forceinline__ unsigned long long chunk_block(const TraceParams& P, unsigned long long* stash, int want)
{
    unsigned long long b = stash[0];
    if (b + (unsigned long long)want > stash[1]) {
        const unsigned long long take = want > kStash ? (unsigned long long)want : (unsigned long long)kStash;
        b = atomicAdd(P.chunk_counter, take);
        stash[1] = b + take;
    }
    stash[0] = b + (unsigned long long)want;
    return b;
}

// FP32 hit evaluation: cheap rejection, then the impact parameter from an
// error-free cross product; full chords from the table at once, partial
// chords queued for flush_partials.  Every lane of the warp calls it (the
// queue is shared); lanes that are not live only take part in the queue.
template <int KERNEL, int MODE, bool NF>
__device__ __forceinline__ void leaf_hits_f32(const TraceParams& P, const float2* tab, PartQueue* pq, int& pq_count,
                                              unsigned long long* stash, int ref, int cnt, unsigned mask, bool live,
                                              float sx, float sy, float sz, float dx, float dy, float dz, float L,
                                              Sink<float>& k, unsigned& err)
{
    if (ref < 0 || cnt > kLeafMax || ref + cnt > P.n) return;   // never true for a well-formed tree
    if (live) k.ntest += (unsigned)__popc(mask);
    const int lane = threadIdx.x & 31;
    for (unsigned m = mask; m; m &= m - 1) {
        const int j = ref + __ffs(m) - 1;
        bool part = false, near = false, store = false;
        int clip = 0;
        float beta2 = 0.f, u1 = 0.f, u2 = 0.f, segv = 0.f;
        int64_t spos = 0;
        if (live) {
            // The hit decision is written with explicit roundings (no
            // multiply-add contraction left to the compiler), so that the
            // counting and the filling traversal, separate instantiations,
            // find exactly the same hits.
            const float4 q = __ldg(P.xyzh + j);
            const float ex = q.x - sx, ey = q.y - sy, ez = q.z - sz;
            float cx = __fsub_rn(__fmul_rn(ey, dz), __fmul_rn(ez, dy));
            float cy = __fsub_rn(__fmul_rn(ez, dx), __fmul_rn(ex, dz));
            float cz = __fsub_rn(__fmul_rn(ex, dy), __fmul_rn(ey, dx));
            const float h2 = __fmul_rn(q.w, q.w);
            bool hit = fmaf(cz, cz, fmaf(cy, cy, __fmul_rn(cx, cx))) < __fmul_rn(1.0001f, h2);
            float b2 = 0.f, tc = 0.f, ch = 0.f;
            if (hit) {
                cx = dop(ey, dz, ez, dy);
                cy = dop(ez, dx, ex, dz);
                cz = dop(ex, dy, ey, dx);
                b2 = fmaf(cz, cz, fmaf(cy, cy, __fmul_rn(cx, cx)));
                hit = b2 < h2;
            }
            if (hit) {
                tc = fmaf(ez, dz, fmaf(ey, dy, __fmul_rn(ex, dx)));
                ch = sqrtf(__fsub_rn(h2, b2));
                hit = __fadd_rn(tc, ch) > 0.f && __fsub_rn(tc, ch) < L;
            }
            if (hit) {
                near = NF && is_near(k, q, tc, ch);
                if (!near) ++k.nhit;
                if (MODE == MODE_CHUNK && !near) store = true;
                if (MODE != MODE_COUNT) {
                    const float ih = 1.f / q.w;
                    beta2 = b2 * ih * ih;
                    if (MODE == MODE_FILL && !near) {
                        // the index is written now, in order; a partial chord's value at the flush
                        if (k.pos < k.end) {
                            store_index(P, k, k.pos, j);
                            spos = k.pos++;
                        } else {
                            err |= kStSegment;
                            hit = false;
                        }
                    }
                    if (hit && __fsub_rn(tc, ch) >= 0.f && __fadd_rn(tc, ch) <= L) {
                        const float F = KERNEL == URCHIN_KERNEL_M4 ? m4_full_tab(tab, beta2)
                                                                   : gt_chord<float>(P, beta2, -ch * ih, ch * ih);
                        const float A = __ldg(P.A32 + j);
                        if (MODE == MODE_SCATTER) {
                            atomicAdd(P.xbar + j, (double)(k.coef * (A * F)));
                        } else if (near) {
                            Kahan::add(k.near, k.near_c, A * F);
                        } else {
                            Kahan::add(k.sum, k.comp, __ldg(P.w32 + j) * F);
                            if (MODE == MODE_FILL) static_cast<float*>(P.seg_val)[spos] = A * F;
                            if (MODE == MODE_CHUNK) segv = A * F;
                        }
                    } else if (hit) {
                        part = true;
                        clip = (__fsub_rn(tc, ch) < 0.f ? kPQClipLo : 0) | (__fadd_rn(tc, ch) > L ? kPQClipHi : 0);
                        u1 = (fmaxf(0.f, tc - ch) - tc) * ih;
                        u2 = (fminf(L, tc + ch) - tc) * ih;
                    }
                }
            }
        }
        if (MODE == MODE_COUNT) continue;
        if constexpr (MODE == MODE_CHUNK) {
            // with the warp converged: a new chunk for every ray whose chunk
            // is full (or that has none yet), then the segment's index (and a
            // full chord's value; a partial chord's at the flush)
            const bool need = store && k.coff == kChunk;
            const unsigned nm = __ballot_sync(0xffffffffu, need);
            if (nm) {
                unsigned long long base = 0;
                if (lane == 0) base = chunk_block(P, stash, __popc(nm));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (need) {
                    const unsigned long long c = base + (unsigned long long)__popc(nm & ((1u << lane) - 1u));
                    if (c < P.chunk_cap) {
                        if (k.cur == kNoChunk) P.chunk_head[k.ray] = (uint32_t)c;
                        else P.chunk_next[k.cur] = (uint32_t)c;
                        k.cur = (uint32_t)c;
                        k.cw = P.chunk_seg + c * (unsigned long long)kChunk;
                        k.coff = 0;
                    } else {
                        k.coff = kChunk + 1;        // the pool is exhausted: this ray stores no more
                    }
                }
            }
            spos = -1;
            if (store && k.coff < kChunk) {
                // a partial chord's entry is written whole at the flush
                if (!part) k.cw[k.coff] = make_int2(j, __float_as_int(segv));
                else spos = (int64_t)k.cur * kChunk + k.coff;
                ++k.coff;
            }
        }
        const unsigned pb = __ballot_sync(0xffffffffu, part);
        if (!pb) continue;
        if (part) {
            PartItem& it = pq->item[pq_count + __popc(pb & ((1u << lane) - 1u))];
            it.beta2 = beta2;
            it.u1 = u1;
            it.u2 = u2;
            it.j = j;
            it.owner = lane | (near ? kPQNear : 0) | clip;
            it.coef = MODE == MODE_SCATTER ? k.coef : 0.f;
            it.pos = spos;
        }
        pq_count += __popc(pb);
        __syncwarp();
        if (pq_count >= 32) flush_partials<KERNEL, MODE, NF>(P, tab, pq, pq_count, 32, k);
    }
}

template <typename Real, int KERNEL, int MODE, bool NF>
__device__ __forceinline__ void leaf_hits(const TraceParams& P, int ref, int cnt, unsigned mask, Real sx, Real sy,
                                          Real sz, Real dx, Real dy, Real dz, Real L, Sink<Real>& k, unsigned& err)
{
    using O = RealOps<Real>;
    if (ref < 0 || cnt > kLeafMax || ref + cnt > P.n) return;   // never true for a well-formed tree
    k.ntest += (unsigned)__popc(mask);
    for (unsigned m = mask; m; m &= m - 1) {
        const int j = ref + __ffs(m) - 1;
        // explicit roundings in the hit decision, as in leaf_hits_f32
        float4 q = __ldg(P.xyzh + j);
        Real ex = Real(q.x) - sx, ey = Real(q.y) - sy, ez = Real(q.z) - sz;
        Real tc = fma(ez, dz, fma(ey, dy, mul_rn(ex, dx)));
        Real cx = sub_rn(mul_rn(ey, dz), mul_rn(ez, dy));
        Real cy = sub_rn(mul_rn(ez, dx), mul_rn(ex, dz));
        Real cz = sub_rn(mul_rn(ex, dy), mul_rn(ey, dx));
        Real b2 = fma(cz, cz, fma(cy, cy, mul_rn(cx, cx)));
        Real h = Real(q.w);
        Real h2 = mul_rn(h, h);
        if (b2 >= h2) continue;
        Real ch = O::sqrt_(sub_rn(h2, b2));
        if (add_rn(tc, ch) <= Real(0) || sub_rn(tc, ch) >= L) continue;
        const bool near = NF && is_near(k, q, tc, ch);
        if (!near) ++k.nhit;
        if (MODE == MODE_COUNT) continue;
        Real ih = Real(1) / h;
        Real beta2 = b2 * ih * ih;
        Real F;
        if (sub_rn(tc, ch) >= Real(0) && add_rn(tc, ch) <= L) {
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
__device__ void ray_column(const TraceParams& P, const float2* tab, Beam* beam, PartQueue* pq, int& pq_count,
                           unsigned long long* stash, float4 o, Real dx, Real dy, Real dz, bool live, Sink<Real>& sk,
                           unsigned& err, unsigned& nvisit)
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
        if (!make_beam(beam, live, fx, fy, fz, (float)dx, (float)dy, (float)dz, Lf)) continue;
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
            // leaf children: left then right, through one call site
            const bool leaf_l = hl && lcnt > 0, leaf_r = hr && rcnt > 0;
#pragma unroll 1
            for (int q = leaf_l ? 0 : 1; q < (leaf_r ? 2 : 1); ++q) {
                const int ref = q == 0 ? lref : rref, cnt = q == 0 ? lcnt : rcnt;
                const unsigned mask = beam_mask(P, *beam, ref, cnt);
                if (mask) {
                    if constexpr (sizeof(Real) == 4)
                        leaf_hits_f32<KERNEL, MODE, NF>(P, tab, pq, pq_count, stash, ref, cnt, mask, live, sx, sy,
                                                        sz, dx, dy, dz, L, sk, err);
                    else if (live)
                        leaf_hits<Real, KERNEL, MODE, NF>(P, ref, cnt, mask, sx, sy, sz, dx, dy, dz, L, sk, err);
                }
            }
            hl = hl && !leaf_l;
            hr = hr && !leaf_r;
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

// Three blocks of 256 per SM (80 registers a thread): with four (64
// registers) the spills cost more than the fourth block's warps hide; with
// two (no spills) too few warps are left to hide the loads.  The transpose
// keeps four: its FP64 atomic adds want the warps more than the registers.
template <typename Real, int KERNEL, int MODE, bool NF>
__global__ void __launch_bounds__(256, MODE == MODE_SCATTER ? 4 : 3) k_trace(TraceParams P)
{
    extern __shared__ double s_dirs[];
    float2* s_tab = reinterpret_cast<float2*>(s_dirs + 3 * P.R);
    __shared__ Beam s_beam[256 / 32];
    __shared__ unsigned long long s_stash[256 / 32][2];   // MODE_CHUNK: the warp's block of chunks
    // the warps' partial-chord queues (FP32 modes that evaluate chords), after the table
    constexpr bool kQueue = sizeof(Real) == 4 && MODE != MODE_COUNT;
    PartQueue* pq = nullptr;
    if (kQueue) {
        const size_t off = trace_queue_offset(P.R, KERNEL);
        pq = reinterpret_cast<PartQueue*>(reinterpret_cast<unsigned char*>(s_dirs) + off) + (threadIdx.x >> 5);
        pq->own[threadIdx.x & 31] = 0u;
        pq->own[(threadIdx.x & 31) + kPQNear] = 0u;
    }
    int pq_count = 0;
    if ((threadIdx.x & 31) == 0) {
        s_stash[threadIdx.x >> 5][0] = 0ull;
        s_stash[threadIdx.x >> 5][1] = 0ull;
    }
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
        Sink<Real> sk{Real(0), Real(0), Real(0), Real(0), 0u, 0u, 0, 0, Real(0), Real(0), Real(0), 0.0, 0.0, 0.0};
        // stored-segment rows are indexed by direction and Morton slot (rows
        // of particles not in the item list stay empty)
        const int64_t ray = (int64_t)k * P.n + org;
        sk.ray = ray;
        sk.cw = nullptr;
        sk.coff = kChunk;
        sk.cur = kNoChunk;
        const int64_t orow = live ? (P.out_row ? (int64_t)P.out_row[item] : item) : 0;
        if (live && MODE == MODE_FILL) {
            sk.pos = (int64_t)P.row_ptr[ray];
            sk.end = (int64_t)P.row_ptr[ray + 1];
        }
        if (live && MODE == MODE_SCATTER) {
            sk.coef = static_cast<const Real*>(P.coef)[orow * P.row_stride + (int64_t)k * P.k_stride];
            live = sk.coef != Real(0);
        }
        ray_column<Real, KERNEL, MODE, NF>(P, s_tab, s_beam + (threadIdx.x >> 5), pq, pq_count,
                                           s_stash[threadIdx.x >> 5], o, dx, dy, dz, live, sk, err, nvisit);
        if constexpr (kQueue) {
            if (pq_count > 0) flush_partials<KERNEL, MODE, NF>(P, s_tab, pq, pq_count, pq_count, sk);
        }
        if (slot < P.n_items) {
            hits += sk.nhit;
            tests += sk.ntest;
            visits += nvisit;
            if (MODE == MODE_COUNT || MODE == MODE_CHUNK || (MODE == MODE_TAU && P.counts))
                P.counts[ray] = (sk.nhit + (unsigned)kSegPad - 1u) / (unsigned)kSegPad * (unsigned)kSegPad;
            if (MODE != MODE_COUNT && MODE != MODE_SCATTER) {
                if (MODE == MODE_CHUNK && sk.coff < kChunk) {
                    // zero entries up to a multiple of kSegPad (inside the chunk)
                    for (; (sk.coff & (kSegPad - 1)) != 0; ++sk.coff) sk.cw[sk.coff] = make_int2(0, 0);
                }
                if (MODE == MODE_FILL) {
                    // the padding (fewer than kSegPad entries) holds zero values
                    if (sk.end - sk.pos >= kSegPad || sk.pos > sk.end) err |= kStSegment;
                    else
                        for (int64_t q = sk.pos; q < sk.end; ++q) {
                            store_index(P, sk, q, 0);
                            static_cast<Real*>(P.seg_val)[q] = Real(0);
                        }
                }
                // full and partial chords are summed apart, each in an order that
                // depends on the ray alone (not on the rays sharing its warp)
                static_cast<Real*>(P.out)[orow * P.row_stride + (int64_t)k * P.k_stride] =
                    (sk.sum + sk.psum) - (sk.comp + sk.pcomp);
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
    const size_t smem = (sizeof(Real) == 4 && MODE != MODE_COUNT)
                            ? trace_queue_offset(P.R, KERNEL) + sizeof(PartQueue) * (256 / 32)
                            : sizeof(double) * 3 * (size_t)P.R +
                                  ((sizeof(Real) == 4 && KERNEL == URCHIN_KERNEL_M4) ? sizeof(float2) * (kKTab + 1) : 0);
    if (smem > 48 * 1024) URCHIN_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
        if (mode == MODE_CHUNK) return set_error(URCHIN_ERR_ARG, "trace: no chunked segment lists with the near/far split");
        return launch_one<Real, KERNEL, MODE_TAU, true>(P, s);
    }
    if (mode == MODE_COUNT) return launch_one<Real, KERNEL, MODE_COUNT, false>(P, s);
    if (mode == MODE_FILL) return launch_one<Real, KERNEL, MODE_FILL, false>(P, s);
    if (mode == MODE_SCATTER) return launch_one<Real, KERNEL, MODE_SCATTER, false>(P, s);
    if (mode == MODE_CHUNK) {
        if constexpr (sizeof(Real) == 4) return launch_one<Real, KERNEL, MODE_CHUNK, false>(P, s);
        return set_error(URCHIN_ERR_ARG, "trace: chunked segment lists are FP32 only");
    }
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
    P.chunk_head = job.chunk_head;
    P.chunk_next = job.chunk_next;
    P.chunk_counter = job.chunk_counter;
    P.chunk_cap = job.chunk_cap;
    P.chunk_seg = job.chunk_seg;
    if (job.near_far && !job.out_near && job.mode != MODE_COUNT)
        return set_error(URCHIN_ERR_ARG, "trace: near/far split without a near-column output");
    if (job.mode == MODE_FILL && !job.seg_col && !(job.seg_lo && job.seg_hi && b->n <= (int64_t(1) << 24)))
        return set_error(URCHIN_ERR_ARG, "trace: segment fill without a particle-index array");
    if (job.mode == MODE_CHUNK && (!job.chunk_head || !job.chunk_next || !job.chunk_counter || !job.counts ||
                                   !job.chunk_seg || job.chunk_cap == 0 || job.chunk_cap > 0xffffffffull))
        return set_error(URCHIN_ERR_ARG, "trace: chunked segment lists need heads, links, a counter and counts");
    return dispatch_mode(P, job.precision, job.kernel, job.mode, job.near_far != 0, s);
}

namespace {

// Every third bit of a 64-bit word from the low 21 bits of v (the standard
// Morton interleave).
__device__ __forceinline__ uint64_t spread21(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x001f00000000ffffull;
    x = (x | x << 16) & 0x001f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t quant21(float f)
{
    return (uint32_t)fminf(fmaxf(f * 2097152.f, 0.f), 2097151.f);
}

// keys of the items for one direction: the 63-bit Morton code of
// (u, v, t / E) in the frame (e1, e2, d), coordinates relative to c scaled by
// inv into [0, 1), as its low 32 bits (lo) and high 31 bits (hi)
__global__ void k_ray_keys(const float4* __restrict__ xyzh, const int32_t* __restrict__ items, int64_t n_items,
                           float3 e1, float3 e2, float3 d, float3 c, float inv, float inv_E, uint32_t* lo,
                           uint32_t* hi, int32_t* vals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_items;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(xyzh + (items ? items[i] : (int32_t)i));
        const float rx = p.x - c.x, ry = p.y - c.y, rz = p.z - c.z;
        const float u = (rx * e1.x + ry * e1.y + rz * e1.z) * inv + 0.5f;
        const float v = (rx * e2.x + ry * e2.y + rz * e2.z) * inv + 0.5f;
        const float t = (rx * d.x + ry * d.y + rz * d.z) * inv * inv_E + 0.5f;
        const uint64_t key = (spread21(quant21(u)) << 2) | (spread21(quant21(v)) << 1) | spread21(quant21(t));
        lo[i] = (uint32_t)key;
        hi[i] = (uint32_t)(key >> 32);
        vals[i] = (int32_t)i;
    }
}

// key[p] = hi[vals[p]]: the high words in the order of the first sort
__global__ void k_gather_hi(const uint32_t* __restrict__ hi, const int32_t* __restrict__ vals, int64_t n,
                            uint32_t* key)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        key[p] = hi[vals[p]];
}

}  // namespace

size_t ray_order_tmp_bytes(int64_t n_items)
{
    Layout lay;
    lay.take(sizeof(uint32_t) * (size_t)n_items);
    lay.take(sizeof(uint32_t) * (size_t)n_items);
    lay.take(radix_tmp_bytes(n_items));
    return lay.bytes;
}

double ray_order_elongation(const urchin_bvh* b, double l_ray)
{
    const double hg = b->hgeo > 0.f ? (double)b->hgeo : 1.0;
    return std::min(64.0, std::max(1.0, l_ray / (2.0 * hg)));
}

int ray_order(const urchin_bvh* b, const int32_t* items, int64_t n_items, const double* dirs, int R, double l_ray,
              int32_t* order, void* tmp, cudaStream_t s)
{
    if (n_items <= 0) return URCHIN_OK;
    Layout lay;
    const size_t o_lo = lay.take(sizeof(uint32_t) * (size_t)n_items);
    const size_t o_hi = lay.take(sizeof(uint32_t) * (size_t)n_items);
    const size_t o_t = lay.take(radix_tmp_bytes(n_items));
    uint32_t* lo = reinterpret_cast<uint32_t*>(static_cast<char*>(tmp) + o_lo);
    uint32_t* hi = reinterpret_cast<uint32_t*>(static_cast<char*>(tmp) + o_hi);
    void* rt = static_cast<char*>(tmp) + o_t;
    const double E = ray_order_elongation(b, l_ray);
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
                                        lo, hi, vals);
        URCHIN_TRY(launched());
        // least significant word first; the radix sort is stable, so the
        // second pass leaves equal high words in low-word order
        URCHIN_TRY(radix_sort_pairs(lo, vals, n_items, 32, rt, s));
        k_gather_hi<<<grid, 256, 0, s>>>(hi, vals, n_items, lo);
        URCHIN_TRY(launched());
        URCHIN_TRY(radix_sort_pairs(lo, vals, n_items, 31, rt, s));
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
        URCHIN_TRY(ray_order(bvh, job.items, n_orig, dirs, R, l_ray, scr.at<int32_t>(o_ord), scr.at<void>(o_otmp), s));
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
