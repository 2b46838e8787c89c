// Device helpers for the ionisation equilibrium of App. C3, shared by the
// standalone equilibrium kernel and the solver's fused sweep kernels.
#pragma once

#include "common.cuh"

namespace urchin {

// Precision-matched math for the spectral fold: single-precision intrinsics
// in the FP32 path, double in the FP64 path.
__device__ __forceinline__ float exp2_p(float x) { return exp2f(x); }
__device__ __forceinline__ double exp2_p(double x) { return exp2(x); }
__device__ __forceinline__ float exp_p(float x) { return expf(x); }
__device__ __forceinline__ double exp_p(double x) { return exp(x); }
__device__ __forceinline__ float log_p(float x) { return logf(x); }
__device__ __forceinline__ double log_p(double x) { return log(x); }

// ---- the binned fold of Eq. gamma_shld ------------------------------------
// Per ray, Gamma_k / Gamma_thin = exp(-s_min tau) S with
//   S = sum_j wn_j exp(-(s_j - s_min) tau),  wn_j = w_j / Gamma_thin,
// evaluated as sum_j wn_j 2^(-e2_j tau) with e2_j = (s_j - s_min) log2(e).
// In FP32 the coefficient is held as a float head e2_j plus a float tail
// e2t_j (their sum equals the double value to ~2^-48), and the exponent is
// formed without rounding: p = e2_j tau rounded, err = fma(e2_j, tau, -p)
// exactly, plus e2t_j tau, so 2^-(p + err) = 2^-p (1 - ln2 err) to second
// order in err (|err| <= 2^-23 |p|).  Rounding the exponent to float would
// leave a relative error growing like 6e-8 s tau (6e-6 at s tau = 100); with
// the split what remains is exp2f's and the weights' rounding, ~2e-7 per
// term, for any tau.

// Block-wide preparation in shared memory (every thread of the block calls
// it; at most 1024 threads): sh[0] = Gamma_thin = sum_j w_j, sh[1] = s_min,
// e2 and wn as above, e2t the FP32 tail (NULL in FP64), sj = s_j (or NULL).
// With q4 (FP32), the same e2, e2t and wn are written packed, q4[j] =
// {e2, e2t, wn, 0}, for fold_ray_q4, and e2, e2t and wn are not written.
template <typename Real>
__device__ void fold_prepare(const double* s, const double* w, int F, Real* e2, Real* e2t, Real* wn, Real* sj,
                             double* sh, float4* q4 = nullptr)
{
    __shared__ double red[32][2];
    double tot = 0.0, smin = 1e300;
    for (int j = threadIdx.x; j < F; j += blockDim.x) {
        tot += w[j];
        smin = fmin(smin, s[j]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        smin = fmin(smin, __shfl_xor_sync(0xffffffffu, smin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = tot;
        red[threadIdx.x >> 5][1] = smin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, m = 1e300;
        for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) {
            t += red[i][0];
            m = fmin(m, red[i][1]);
        }
        sh[0] = t;
        sh[1] = m;
    }
    __syncthreads();
    const double g = sh[0], m = sh[1];
    for (int j = threadIdx.x; j < F; j += blockDim.x) {
        const double c = (s[j] - m) * 1.4426950408889634;
        if (q4) {
            const float h = (float)c;
            q4[j] = make_float4(h, (float)(c - (double)h), (float)(w[j] / g), 0.f);
        } else {
            e2[j] = (Real)c;
            if (e2t) e2t[j] = (Real)(c - (double)(Real)c);
            wn[j] = (Real)(w[j] / g);
        }
        if (sj) sj[j] = (Real)s[j];
    }
    __syncthreads();
}

// S (and, with kTan, S2 = sum_j wn_j s_j exp(-(s_j - s_min) tau), the
// tangent's sum) of one ray, compensated sums.
template <bool kTan>
__device__ __forceinline__ void fold_ray(float tau, const float* e2, const float* e2t, const float* wn,
                                         const float* sj, int F, float& S_out, float& S2_out)
{
    // a NaN column stays NaN; columns beyond 1e30 (every term but the s_min
    // bin underflows) are clamped so that the exponent's error stays finite
    tau = tau < 1e30f ? tau : (tau == tau ? 1e30f : tau);
    float S = 0.f, c = 0.f, S2 = 0.f, c2 = 0.f;
    for (int j = 0; j < F; ++j) {
        const float p = e2[j] * tau;
        const float err = fmaf(e2t[j], tau, fmaf(e2[j], tau, -p));
        const float v0 = wn[j] * exp2f(-p);
        const float v = fmaf(-v0, err * 0.6931471805599453f, v0);
        const float yy = v - c;
        const float t = S + yy;
        c = (t - S) - yy;
        S = t;
        if (kTan) {
            const float v2 = v * sj[j];
            const float y2 = v2 - c2;
            const float t2 = S2 + y2;
            c2 = (t2 - S2) - y2;
            S2 = t2;
        }
    }
    S_out = S;
    S2_out = S2;
}

// fold_ray<false> in FP32 with each bin's three coefficients read as one
// 16-byte word, q = {e2, e2t, wn, 0} (the same arithmetic in the same order,
// so the same S bit for bit; one shared-memory load per bin instead of three).
__device__ __forceinline__ float fold_ray_q4(float tau, const float4* q4, int F)
{
    tau = tau < 1e30f ? tau : (tau == tau ? 1e30f : tau);
    float S = 0.f, c = 0.f;
    for (int j = 0; j < F; ++j) {
        const float4 q = q4[j];
        const float p = q.x * tau;
        const float err = fmaf(q.y, tau, fmaf(q.x, tau, -p));
        const float v0 = q.z * exp2f(-p);
        const float v = fmaf(-v0, err * 0.6931471805599453f, v0);
        const float yy = v - c;
        const float t = S + yy;
        c = (t - S) - yy;
        S = t;
    }
    return S;
}

template <bool kTan>
__device__ __forceinline__ void fold_ray(double tau, const double* e2, const double*, const double* wn,
                                         const double* sj, int F, double& S_out, double& S2_out)
{
    double S = 0.0, c = 0.0, S2 = 0.0, c2 = 0.0;
    for (int j = 0; j < F; ++j) {
        const double v = wn[j] * exp2(-e2[j] * tau);
        const double yy = v - c;
        const double t = S + yy;
        c = (t - S) - yy;
        S = t;
        if (kTan) {
            const double v2 = v * sj[j];
            const double y2 = v2 - c2;
            const double t2 = S2 + y2;
            c2 = (t2 - S2) - y2;
            S2 = t2;
        }
    }
    S_out = S;
    S2_out = S2;
}

// ln x for x > 0 as e ln2 + ln m with x = m 2^e, m in [1/2, 1): the float
// logarithm of the mantissa is accurate to 6e-8 absolute, where logf(x) of
// a small x (|ln x| ~ 10) is only accurate to an ulp of 10, 1e-6.
__device__ __forceinline__ double log_split(float x)
{
    int e;
    const float m = frexpf(x, &e);
    return fma((double)e, 0.6931471805599453, (double)logf(m));
}
__device__ __forceinline__ double log_split(double x) { return log(x); }

// ln(Gamma_k / Gamma_thin) = -s_min tau + ln S, the product in double (in
// float its rounding, ~6e-8 s_min tau, would reach 1e-5 at s_min tau ~ 170).
template <typename Real>
__device__ __forceinline__ double ray_lnrate(double smin, Real tau, Real S)
{
    return fma(-smin, (double)tau, log_split(S));
}

// Fold of one ray behind H I, He I and He II columns (t0, t1, t2):
// ln(Gamma_k / Gamma_thin) = ln sum_j wn_j exp(-E_j), E_j = s_j t0 + s1_j t1 +
// s2_j t2, in FP32 with each E_j formed as a float pair (head + tail): the
// cross sections split into float heads and tails (the tail arrays), every
// product split exactly by a fused multiply-add, the three products added
// with error-free sums.  The sum runs against the smallest E_j so far (the
// partial sum rescaled when a smaller one appears), so that no term
// overflows; the head difference of two close exponents is exact, and the
// result is accurate to ~1e-7 in ln Gamma for any column.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ double fold_ray_he(float t0, float t1, float t2, const float* s0, const float* s0t,
                                              const float* s1, const float* s1t, const float* s2, const float* s2t,
                                              const float* wn, int F)
{
    float mh = INFINITY, ml = 0.f, S = 0.f, c = 0.f;
    for (int j = 0; j < F; ++j) {
        const float p0 = s0[j] * t0, p1 = s1[j] * t1, p2 = s2[j] * t2;
        const float e0 = fmaf(s0t[j], t0, fmaf(s0[j], t0, -p0));
        const float e1 = fmaf(s1t[j], t1, fmaf(s1[j], t1, -p1));
        const float e2 = fmaf(s2t[j], t2, fmaf(s2[j], t2, -p2));
        float q, r1, hi, r2;
        two_sum(p0, p1, q, r1);
        two_sum(q, p2, hi, r2);
        const float lo = ((r1 + r2) + (e0 + e1)) + e2;
        if (hi < mh) {
            if (S != 0.f) {
                const float f = expf(-((mh - hi) + (ml - lo)));
                S *= f;
                c *= f;
            }
            mh = hi;
            ml = lo;
        }
        const float v = wn[j] * expf(-((hi - mh) + (lo - ml)));
        const float yy = v - c;
        const float u = S + yy;
        c = (u - S) - yy;
        S = u;
    }
    return -((double)mh + (double)ml) + log_split(S);
}

// Running log-sum-exp over a particle's rays, ln((1/R) sum_k exp(l_k)): the
// maximum in double, the sum of exp(l_k - max) >= 1 in the columns'
// precision.
template <typename Real>
struct RayMean {
    double m = -INFINITY;
    Real acc = Real(0);
    __device__ __forceinline__ void add(double l)
    {
        if (l == -INFINITY) return;      // a ray with no transmitted flux adds nothing
        if (l > m) {
            acc = acc * exp_p((Real)(m - l)) + Real(1);
            m = l;
        } else {
            acc += exp_p((Real)(l - m));
        }
    }
    __device__ __forceinline__ double mean(int R) const { return m + log_split(acc / (Real)R); }
};

struct Rates {
    double alphaA, alphaB, gamma_c;   // cm^3 s^-1
};

// Hui & Gnedin (1997) fits, lambda = 2 T_HI / T with T_HI = 157807 K:
//   alpha_A = 1.269e-13 lambda^1.503 / [1 + (lambda/0.522)^0.470]^1.923
//   alpha_B = 2.753e-14 lambda^1.500 / [1 + (lambda/2.740)^0.407]^2.242
//   gamma   = 21.11 T^-3/2 e^(-lambda/2) lambda^-1.089 / [1 + (lambda/0.354)^0.874]^1.101
// (App. C3 names fits of this kind for the temperature dependence.)
// Evaluated with one logarithm, six exponentials and three log1p (FP64 is the
// slow path of this GPU; no pow, no logarithm of a constant): each bracket as
// exp(-p log1p((lambda/c)^q)), the powers of lambda from ll = ln lambda, and
// ln T = ln 315614 - ll.
__device__ __forceinline__ Rates hg97_rates(double T)
{
    constexpr double kLn0522 = -0.6500876910994983;     // ln 0.522
    constexpr double kLn2740 = 1.007957920399979;       // ln 2.740
    constexpr double kLn0354 = -1.0384583658483626;     // ln 0.354
    constexpr double kLn2THI = 12.662275226919286;      // ln 315614
    const double lam = 315614.0 / T;
    const double ll = log(lam);
    const double uA = exp(0.470 * (ll - kLn0522));
    const double uB = exp(0.407 * (ll - kLn2740));
    const double uC = exp(0.874 * (ll - kLn0354));
    Rates r;
    r.alphaA = 1.269e-13 * exp(1.503 * ll - 1.923 * log1p(uA));
    r.alphaB = 2.753e-14 * exp(1.500 * ll - 2.242 * log1p(uB));
    // T^-3/2 lambda^-1.089 = exp(-1.5 (ln 315614 - ll) - 1.089 ll)
    r.gamma_c = 21.11 * exp(-1.5 * kLn2THI + 0.411 * ll - 0.5 * lam - 1.101 * log1p(uC));
    return r;
}

// Physical root of R x^2 + Q x + P = 0 (Eq. xroots, x_-), with
// R = (gamma_c + alpha) n_H, Q = -[Gamma + alpha n_H + R (1+y)],
// P = alpha n_H (1+y), evaluated as 2P / (-Q + sqrt(Q^2 - 4PR)); the
// discriminant is formed as (Gamma + e)^2 + 4 Gamma alpha n_H with
// e = R(1+y) - alpha n_H = alpha n_H y + gamma_c n_H (1+y) >= 0, an exact
// rewrite whose terms never cancel.
__device__ __forceinline__ double x_equilibrium(double Gamma, double nH, double alpha, double gamma_c, double y)
{
    const double an = alpha * nH;
    const double Rc = (gamma_c + alpha) * nH;
    const double Q = -(Gamma + an + Rc * (1.0 + y));
    const double P = an * (1.0 + y);
    const double e = an * y + gamma_c * nH * (1.0 + y);
    const double disc = (Gamma + e) * (Gamma + e) + 4.0 * Gamma * an;
    return 2.0 * P / (-Q + sqrt(disc));
}

// d x / d Gamma of the root above (for tangents): differentiating
// R x^2 + Q x + P = 0 with dQ/dGamma = -1 gives dx/dGamma = x / (2 R x + Q).
__device__ __forceinline__ double dx_dgamma(double x, double nH, double alpha, double gamma_c, double Gamma,
                                            double y)
{
    const double Rc = (gamma_c + alpha) * nH;
    const double Q = -(Gamma + alpha * nH + Rc * (1.0 + y));
    return x / (2.0 * Rc * x + Q);
}

// Near/far split (Sec. 3.3.3): the near particles of a ray's origin are
// modelled as a uniform hydrogen slab of thickness tau_near = N_H sigma_th
// (all hydrogen, x = 1), with the origin's density and temperature, lit by
// the far-attenuated radiation of that ray's direction, i.e. its share
// (1/N_ray) of the rate, Gamma_far at the slab's surface; the particle's
// rate is the sum over rays of the slabs' bottom rates (Eq. gammashld).  For
// radiation at the threshold (the slab appendix, y = 0) the depth at which
// the equilibrium neutral fraction is x obeys
//   z nH sigma = (1/x0 - 1/x) + ln[x (1-x0) / (x0 (1-x))]
//                + (1/x_ce) ln[x (x_ce - x0) / (x0 (x_ce - x))],
// x0 the equilibrium at Gamma_far, x_ce = alpha / (alpha + gamma_c), and the
// rate at depth x is nH (1-x)(alpha+gamma_c)(x_ce - x) / x.  Returns
// ln(Gamma_bottom / Gamma_thin) from ln(Gamma_far / Gamma_thin): Newton's
// method on y = ln[x / (x_ce - x)] (which resolves both a strongly ionised
// bottom, x << x_ce, and a neutral one, x_ce - x below double resolution),
// kept inside a bracket (bisection when a step leaves it).  Every 1 - x is
// formed as c + (x_ce - x), c = 1 - x_ce = gamma_c / (alpha + gamma_c), and
// x_ce - x0 from the surface equilibrium D (c + D) = Gamma_far x0 /
// (nH (alpha + gamma_c)): no cancellation in cold, nearly neutral gas where
// x_ce rounds to 1.
__device__ __forceinline__ double log1pexp(double y) { return y > 0.0 ? y + log1p(exp(-y)) : log1p(exp(y)); }

__device__ __forceinline__ double slab_lnratio(double lnr_far, double gthin, double tau_near, double nH,
                                               double alpha, double gamma_c)
{
    if (!(tau_near > 0.0)) return lnr_far;
    const double ag = alpha + gamma_c;
    const double xce = alpha / ag;
    const double G0 = gthin * exp(lnr_far);
    if (!(G0 > 0.0)) return lnr_far - xce * tau_near;   // no ionised layer: neutral attenuation
    const double c = gamma_c / ag;                      // 1 - x_ce
    const double x0 = x_equilibrium(G0, nH, alpha, gamma_c, 0.0);
    const double K = G0 * x0 / (nH * ag);
    const double d0 = 2.0 * K / (c + sqrt(c * c + 4.0 * K));   // x_ce - x0
    const double lxce = log(xce), lx0 = log(x0), ld0 = log(d0);
    // depth(y) - tau_near = c0 - 1/x + lx - log(c + e) + (lx - le) / x_ce - tau_near
    const double c0 = 1.0 / x0 - lx0 + log(c + d0) + (ld0 - lx0) / xce;
    double ylo = lx0 - ld0, yhi = lxce - ld0 + xce * tau_near + 50.0;
    // first guess from the dominant terms: an ionised bottom where
    // 1/x ~ 1/x0 - tau_near, else a neutral layer attenuating like x_ce
    const double q = 1.0 / x0 - tau_near;
    double y;
    if (q * xce > 1.5) {
        const double xg = 1.0 / q;
        y = log(xg) - log(xce - xg);
    } else {
        y = lxce - ld0 + xce * (tau_near - (1.0 / x0 - 1.0 / xce));
    }
    y = fmin(yhi, fmax(ylo, y));
    for (int it = 0; it < 100; ++it) {
        const double lx = lxce - log1pexp(-y), le = lxce - log1pexp(y);
        const double x = exp(lx), e = exp(le);
        const double f = c0 - 1.0 / x + lx - log(c + e) + (lx - le) / xce - tau_near;
        if (f > 0.0) yhi = y;                            // too deep
        else ylo = y;
        // d depth / dy with dx/dy = x e / x_ce (and x + e = x_ce)
        const double fp = (e / x + e + x * e / (c + e) + 1.0) / xce;
        double yn = y - f / fp;
        if (fabs(yn - y) <= 1e-15 * (1.0 + fabs(y))) {   // converged (rounding may put it a hair
            y = yn;                                        // outside the bracket)
            break;
        }
        if (!(yn > ylo && yn < yhi)) yn = 0.5 * (ylo + yhi);
        const bool done = yhi - ylo <= 1e-15 * (1.0 + fabs(y));
        y = yn;
        if (done) break;
    }
    const double lx = lxce - log1pexp(-y), le = lxce - log1pexp(y);
    return log(nH) + log(c + exp(le)) + log(ag) + le - lx - log(gthin);
}

// ---- polychromatic slab ---------------------------------------------------
// ln Gamma_spec(tau) = ln sum_b w_b exp(-s_b tau) tabulated on u = ln(1 + tau)
// in [0, umax] (nt intervals): tab[i] = (value, d value / du), evaluated by
// cubic Hermite interpolation; past umax the tail is linear in tau with
// slope -s_min (the hardest bin dominates).
struct SpecTable {
    const double2* tab;
    int nt;
    double umax;
    double smin;
    const float2* tab32;          // the same table as (ln(Gamma_spec / Gamma_thin), d/du) in float
    double lnthin;                // ln Gamma_thin
};

__device__ __forceinline__ double spec_lnrate(const SpecTable& S, double tau)
{
    const double u = log1p(tau);
    if (u >= S.umax) {
        const double tm = expm1(S.umax);
        return S.tab[S.nt].x - S.smin * (tau - tm);
    }
    const double pos = u / S.umax * (double)S.nt;
    int i = (int)pos;
    i = i < 0 ? 0 : (i >= S.nt ? S.nt - 1 : i);
    const double h = S.umax / (double)S.nt;
    const double f = pos - (double)i;
    const double2 a = S.tab[i], b = S.tab[i + 1];
    const double f2 = f * f, f3 = f2 * f;
    return (2.0 * f3 - 3.0 * f2 + 1.0) * a.x + (f3 - 2.0 * f2 + f) * h * a.y + (3.0 * f2 - 2.0 * f3) * b.x +
           (f3 - f2) * h * b.y;
}

// d ln Gamma_spec / d tau = -(mean s weighted by the attenuated spectrum)
__device__ __forceinline__ double spec_slope(const SpecTable& S, double tau)
{
    const double u = log1p(tau);
    if (u >= S.umax) return -S.smin;
    const double pos = u / S.umax * (double)S.nt;
    int i = (int)pos;
    i = i < 0 ? 0 : (i >= S.nt ? S.nt - 1 : i);
    const double f = pos - (double)i;
    return ((1.0 - f) * S.tab[i].y + f * S.tab[i + 1].y) / (1.0 + tau);
}

// The slab of near particles lit by the polychromatic spectrum after the far
// column tau_far (the numerical slab solution for Eq. gammashldk, y = 0):
// with t = sigma_th nH z, dtau_HI/dt = x_eq(Gamma_spec(tau_far + tau_HI)),
// equivalently t(tau_HI) = int_0^tau_HI dv / x(v).  The integral is summed
// over panels in v whose width keeps the change of ln Gamma at the panel's
// start slope at 2 (|d ln x / d ln Gamma| <= 1, so 1/x is close to an
// exponential across a panel), each by 8-point Gauss-Legendre; the panel
// where t reaches tau_near is solved by Newton's method on its own
// quadrature.  Against adaptive Dormand-Prince integration of the same slab
// (60 seeded cases) this scheme is within 1.4e-10 in ln Gamma with at most
// 144 evaluations of x per ray, 4-point panels of width 1/2 within 2.3e-9
// with up to 276.  Once x is within 1e-10
// of x_ce the rest of the slab is uniform (1/x = 1/x_ce).  Returns
// ln(Gamma_bottom / Gamma_thin).
__device__ __forceinline__ double slab_x(const SpecTable& S, double tau, double lnscale, double nH, double alpha,
                                         double gc)
{
    return x_equilibrium(exp(spec_lnrate(S, tau) + lnscale), nH, alpha, gc, 0.0);
}

__device__ __forceinline__ double slab_panel(const SpecTable& S, double tf, double ls, double a, double b,
                                             double nH, double alpha, double gc)
{
    // 8-point Gauss-Legendre of 1/x over [a, b]
    const double g[4] = {0.18343464249564978, 0.525532409916329, 0.7966664774136267, 0.9602898564975362};
    const double wq[4] = {0.36268378337836166, 0.3137066458778869, 0.22238103445337443, 0.10122853629037706};
    const double m = 0.5 * (a + b), r = 0.5 * (b - a);
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        acc += wq[q] * (1.0 / slab_x(S, tf + m - r * g[q], ls, nH, alpha, gc) +
                        1.0 / slab_x(S, tf + m + r * g[q], ls, nH, alpha, gc));
    return r * acc;
}

__device__ __forceinline__ double slab_poly_lnratio(const SpecTable& S, double gthin, double tau_far,
                                                    double tau_near, double nH, double alpha, double gc,
                                                    double lnscale)
{
    // the slab is lit by the tabulated spectrum scaled by e^lnscale (a ray's share)
    if (!(tau_near > 0.0)) return spec_lnrate(S, tau_far) + lnscale - log(gthin);
    const double xce = alpha / (alpha + gc);
    double v = 0.0, t = 0.0;
    for (int panel = 0; panel < 100000; ++panel) {
        const double xv = slab_x(S, tau_far + v, lnscale, nH, alpha, gc);
        if (xv >= xce * (1.0 - 1e-10)) {            // neutral plateau: the rest is uniform
            v += (tau_near - t) * xce;
            break;
        }
        const double sl = -spec_slope(S, tau_far + v);
        const double dv = 2.0 / fmax(sl, 1e-300);
        const double dt = slab_panel(S, tau_far, lnscale, v, v + dv, nH, alpha, gc);
        if (t + dt < tau_near) {
            t += dt;
            v += dv;
            continue;
        }
        // t(v + e) = t + int_v^{v+e} 1/x = tau_near: Newton from the linear guess
        double e = dv * (tau_near - t) / dt;
        for (int it = 0; it < 30; ++it) {
            const double g = t + slab_panel(S, tau_far, lnscale, v, v + e, nH, alpha, gc) - tau_near;
            const double step = g * slab_x(S, tau_far + v + e, lnscale, nH, alpha, gc);
            double en = e - step;
            en = fmin(fmax(en, 0.0), dv);
            const bool done = fabs(en - e) <= 1e-14 * (v + dv);
            e = en;
            if (done) break;
        }
        v += e;
        break;
    }
    return spec_lnrate(S, tau_far + v) + lnscale - log(gthin);
}

// The polychromatic slab with FP32 evaluations of the spectrum table and of
// x_eq (the FP32 sweep; FP64 is limited on this part): x_eq from the root
// scaled by alpha n_H, x = 2 / ((g + 2 + c) + sqrt((g + c)^2 + 4 g)) with
// g = Gamma / (alpha n_H) and c = gamma_c / alpha (no cancellation, no
// under- or overflow), the table as ln(Gamma_spec / Gamma_thin) so that its
// rounding is relative to the thin rate; panel sums, the depth t and the
// returned rate in double.  Against adaptive FP64 integration of the same
// slab (80 seeded cases, emulated) within 1.8e-6 in ln Gamma.
__device__ __forceinline__ float spec_lnrel32(const SpecTable& S, float tau)
{
    const float u = log1pf(tau);
    const float umax = (float)S.umax;
    if (u >= umax) return S.tab32[S.nt].x - (float)S.smin * (tau - (float)expm1(S.umax));
    const float pos = u / umax * (float)S.nt;
    int i = (int)pos;
    i = i < 0 ? 0 : (i >= S.nt ? S.nt - 1 : i);
    const float h = umax / (float)S.nt;
    const float f = pos - (float)i;
    const float2 a = S.tab32[i], b = S.tab32[i + 1];
    const float f2 = f * f, f3 = f2 * f;
    return (2.f * f3 - 3.f * f2 + 1.f) * a.x + (f3 - 2.f * f2 + f) * h * a.y + (3.f * f2 - 2.f * f3) * b.x +
           (f3 - f2) * h * b.y;
}

__device__ __forceinline__ float spec_slope32(const SpecTable& S, float tau)
{
    const float u = log1pf(tau);
    if (u >= (float)S.umax) return -(float)S.smin;
    const float pos = u / (float)S.umax * (float)S.nt;
    int i = (int)pos;
    i = i < 0 ? 0 : (i >= S.nt ? S.nt - 1 : i);
    const float f = pos - (float)i;
    return ((1.f - f) * S.tab32[i].y + f * S.tab32[i + 1].y) / (1.f + tau);
}

// x_eq at depth tau: off = ln(Gamma_thin) + lnscale - ln(alpha n_H), c = gamma_c / alpha
__device__ __forceinline__ float slab_x32(const SpecTable& S, float tau, float off, float c)
{
    const float g = expf(spec_lnrel32(S, tau) + off);
    const float gc = g + c;
    return 2.f / ((g + 2.f + c) + sqrtf(gc * gc + 4.f * g));
}

__device__ __forceinline__ double slab_panel32(const SpecTable& S, double tf, float off, float c, double a, double b)
{
    const float g[4] = {0.18343464249564978f, 0.525532409916329f, 0.7966664774136267f, 0.9602898564975362f};
    const float wq[4] = {0.36268378337836166f, 0.3137066458778869f, 0.22238103445337443f, 0.10122853629037706f};
    const double m = 0.5 * (a + b), r = 0.5 * (b - a);
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        acc += wq[q] * (1.f / slab_x32(S, (float)(tf + m - r * g[q]), off, c) +
                        1.f / slab_x32(S, (float)(tf + m + r * g[q]), off, c));
    return r * (double)acc;
}

__device__ __forceinline__ double slab_poly_lnratio32(const SpecTable& S, double gthin, double tau_far,
                                                      double tau_near, double nH, double alpha, double gc,
                                                      double lnscale)
{
    if (!(tau_near > 0.0)) return spec_lnrate(S, tau_far) + lnscale - log(gthin);
    const float off = (float)(S.lnthin + lnscale - log(alpha * nH));
    const float c = (float)(gc / alpha);
    const float xce = 1.f / (1.f + c);
    double v = 0.0, t = 0.0;
    for (int panel = 0; panel < 100000; ++panel) {
        const float xv = slab_x32(S, (float)(tau_far + v), off, c);
        if (xv >= xce * (1.f - 1e-6f)) {            // neutral plateau: the rest is uniform
            v += (tau_near - t) * (double)xce;
            break;
        }
        const double sl = -(double)spec_slope32(S, (float)(tau_far + v));
        const double dv = 2.0 / fmax(sl, 1e-300);
        const double dt = slab_panel32(S, tau_far, off, c, v, v + dv);
        if (t + dt < tau_near) {
            t += dt;
            v += dv;
            continue;
        }
        double e = dv * (tau_near - t) / dt;
        for (int it = 0; it < 30; ++it) {
            const double gg = t + slab_panel32(S, tau_far, off, c, v, v + e) - tau_near;
            const double step = gg * (double)slab_x32(S, (float)(tau_far + v + e), off, c);
            double en = e - step;
            en = fmin(fmax(en, 0.0), dv);
            const bool done = fabs(en - e) <= 1e-6 * (v + dv);
            e = en;
            if (done) break;
        }
        v += e;
        break;
    }
    return spec_lnrate(S, tau_far + v) + lnscale - log(gthin);
}

}  // namespace urchin
