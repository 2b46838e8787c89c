// Shielded photoionisation rate (Eq. gamma_shld) and ionisation equilibrium
// (App. C3, Eqs. dxdt / xroots / xphys).
//
// Gamma: for one origin with columns tau_k (threshold optical depth) and a
// binned spectrum (s_j = sigma_j / sigma_th, w_j with sum w_j = Gamma_thin),
//   Gamma / Gamma_thin = (1/R) sum_k sum_j w^_j exp(-s_j tau_k),  w^ = w / Gamma_thin.
// Each ray's inner sum is factored as exp(-s_min tau_k) S_k with
//   S_k = sum_j w^_j exp(-(s_j - s_min) tau_k)  in [w^_jmin, 1],
// so ln(Gamma_k / Gamma_thin) = -s_min tau_k + ln S_k never underflows; the
// rays are then combined with a log-sum-exp in double, which keeps tau_eff
// finite where Gamma itself underflows.
#include <algorithm>
#include <cmath>

#include "spectral_device.cuh"

namespace urchin {

namespace {

constexpr int kGammaThreads = 256;

// Threads (local, k) fold ray k of row `local` (fold_ray: the exponent of
// every bin formed without rounding error); the per-row log-sum-exp runs with
// one thread per row packed into the first lanes.
template <typename Real>
__global__ void __launch_bounds__(kGammaThreads) k_gamma(GammaJob J)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kF32 = sizeof(Real) == 4;
    double* lk = reinterpret_cast<double*>(smem_raw);
    Real* e2 = reinterpret_cast<Real*>(lk + kGammaThreads);
    Real* wn = e2 + J.F;
    Real* e2t = kF32 ? wn + J.F : nullptr;
    __shared__ double sh[2];
    fold_prepare<Real>(J.s, J.w, J.F, e2, e2t, wn, nullptr, sh);
    const int rows_per_block = kGammaThreads / J.R;
    const int local = threadIdx.x / J.R;
    const int k = threadIdx.x % J.R;
    const double gthin = sh[0];
    const double smin = sh[1];
    for (int64_t row0 = (int64_t)blockIdx.x * rows_per_block; row0 < J.n_rows;
         row0 += (int64_t)gridDim.x * rows_per_block) {
        const int64_t row = row0 + local;
        if (local < rows_per_block && row < J.n_rows) {
            const Real tau = static_cast<const Real*>(J.tau)[row * J.row_stride + (int64_t)k * J.k_stride];
            Real S, S2;
            fold_ray<false>(tau, e2, e2t, wn, nullptr, J.F, S, S2);
            lk[local * J.R + k] = ray_lnrate(smin, tau, S);
        }
        __syncthreads();
        const int p = threadIdx.x;
        const int64_t prow = row0 + p;
        if (p < rows_per_block && prow < J.n_rows) {
            RayMean<Real> lse;
            for (int r = 0; r < J.R; ++r) lse.add(lk[p * J.R + r]);
            const double lmean = lse.mean(J.R);     // ln(Gamma / Gamma_thin)
            J.gamma_out[prow] = gthin * exp(lmean);
            if (J.tau_eff_out) J.tau_eff_out[prow] = (float)(-lmean);
        }
        __syncthreads();
    }
}

template <typename Real>
int launch_gamma_t(const GammaJob& J, cudaStream_t s)
{
    // per-ray log rates (double), then e2, wn and (FP32) the tail e2t
    const size_t smem = sizeof(double) * kGammaThreads + (sizeof(Real) == 4 ? 3 : 2) * (size_t)J.F * sizeof(Real);
    auto fn = k_gamma<Real>;
    if (smem > 48 * 1024)
        URCHIN_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int rows_per_block = kGammaThreads / J.R;
    int64_t need = (J.n_rows + rows_per_block - 1) / rows_per_block;
    int grid = 0;
    URCHIN_TRY(grid_for((const void*)fn, kGammaThreads, smem, &grid));
    if (need < grid) grid = (int)std::max<int64_t>(need, 1);
    fn<<<grid, kGammaThreads, smem, s>>>(J);
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

__global__ void k_equilibrium(const double* __restrict__ gamma, const float* __restrict__ tau_eff,
                              const double* __restrict__ nH, const double* __restrict__ T, int64_t n,
                              int case_rule, double y, double* x_out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Rates r = hg97_rates(T[i]);
        bool caseB = case_rule == URCHIN_CASE_B ||
                     (case_rule == URCHIN_CASE_AUTO && tau_eff[i] >= 1.0f);
        x_out[i] = x_equilibrium(gamma[i], nH[i], caseB ? r.alphaB : r.alphaA, r.gamma_c, y);
    }
}

// Reverse mode of Eq. gamma_shld, in double.  With c_o = gamma_bar_o / R:
//   tau_bar_ok = -c_o sum_b w_b s_b exp(-s_b tau_ok)
//              = -sign(c_o) exp(ln|c_o| - s_min tau_ok + ln sum_b w_b s_b exp(-(s_b - s_min) tau_ok)),
// written so that a large |c_o| (deeply shielded origins) does not overflow
// where exp(-s_min tau) underflows.
template <typename Real>
__global__ void k_gamma_vjp_tau(const Real* __restrict__ tau, int64_t n_rays, int R, const double* __restrict__ sv,
                                const double* __restrict__ wv, int F, const double* __restrict__ gbar, Real* tau_bar)
{
    extern __shared__ double sm[];
    double* ss = sm;
    double* ws = sm + F;
    __shared__ double smin_s;
    for (int b = threadIdx.x; b < F; b += blockDim.x) {
        ss[b] = sv[b];
        ws[b] = wv[b] * sv[b];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = ss[0];
        for (int b = 1; b < F; ++b) m = fmin(m, ss[b]);
        smin_s = m;
    }
    __syncthreads();
    const double smin = smin_s;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const double c = gbar[r / R] / (double)R;
        const double t = (double)tau[r];
        double S = 0.0;
        for (int b = 0; b < F; ++b) S += ws[b] * exp(-(ss[b] - smin) * t);
        double v = 0.0;
        if (c != 0.0 && S > 0.0) v = -copysign(exp(log(fabs(c)) - smin * t + log(S)), c);
        tau_bar[r] = (Real)v;
    }
}

// w_bar_b partial sums over rays r with a coefficient c_r = sg_r exp(lc_r):
// partial[block * F + b] = sum over the block's rays of sg_r exp(lc_r - s_b tau_r).
// Rays are staged in tiles; each thread owns a set of bins, so no two
// threads add to the same sum.
constexpr int kWTile = 128;
template <typename Real>
__global__ void k_wbar_tiles(const Real* __restrict__ tau, int64_t n_rays, const double* __restrict__ lc_in,
                             const double* __restrict__ sg_in, const double* __restrict__ sv, int F, double* partial)
{
    extern __shared__ double sm[];
    double* ss = sm;
    double* acc = sm + F;
    double* tt = acc + F;
    double* lc = tt + kWTile;
    double* sg = lc + kWTile;
    for (int b = threadIdx.x; b < F; b += blockDim.x) {
        ss[b] = sv[b];
        acc[b] = 0.0;
    }
    const int64_t tiles = (n_rays + kWTile - 1) / kWTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < kWTile; i += blockDim.x) {
            const int64_t r = tile * kWTile + i;
            const bool in = r < n_rays;
            tt[i] = in ? (double)tau[r] : 0.0;
            lc[i] = in ? lc_in[r] : -INFINITY;
            sg[i] = in ? sg_in[r] : 0.0;
        }
        __syncthreads();
        for (int b = threadIdx.x; b < F; b += blockDim.x) {
            const double sb = ss[b];
            double a = acc[b];
            for (int i = 0; i < kWTile; ++i) a += sg[i] * exp(lc[i] - sb * tt[i]);
            acc[b] = a;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < F; b += blockDim.x) partial[(int64_t)blockIdx.x * F + b] = acc[b];
}

// The FP32 form of k_wbar_tiles: with l_r = lc_r - s_min tau_r and m the
// largest l_r of the tile, every term is sg_r exp(l_r - m) (a float in
// [-1, 1], from one double exp per ray) times exp(-(s_b - s_min) tau_r)
// (the fold's float exponent with its rounding error carried, see
// fold_ray), summed over the tile in float with compensation and added to
// the bin's double sum times exp(m): one double operation per tile and bin
// instead of a double exp per ray and bin.
__global__ void k_wbar_tiles_f32(const float* __restrict__ tau, int64_t n_rays, const double* __restrict__ lc_in,
                                 const double* __restrict__ sg_in, const double* __restrict__ sv, int F,
                                 double* partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* acc = reinterpret_cast<double*>(smem_raw);           // [F]
    double* ld = acc + F;                                         // [kWTile]
    float* e2 = reinterpret_cast<float*>(ld + kWTile);            // [F]
    float* e2t = e2 + F;                                          // [F]
    float* tt = e2t + F;                                          // [kWTile]
    float* fr = tt + kWTile;                                      // [kWTile]
    __shared__ double sh_smin, sh_m;
    if (threadIdx.x == 0) {
        double m = sv[0];
        for (int b = 1; b < F; ++b) m = fmin(m, sv[b]);
        sh_smin = m;
    }
    __syncthreads();
    const double smin = sh_smin;
    for (int b = threadIdx.x; b < F; b += blockDim.x) {
        const double c = (sv[b] - smin) * 1.4426950408889634;
        e2[b] = (float)c;
        e2t[b] = (float)(c - (double)(float)c);
        acc[b] = 0.0;
    }
    const int64_t tiles = (n_rays + kWTile - 1) / kWTile;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < kWTile; i += blockDim.x) {
            const int64_t r = tile * kWTile + i;
            const bool in = r < n_rays;
            const float t = in ? tau[r] : 0.f;
            tt[i] = t < 1e30f ? t : (t == t ? 1e30f : t);
            ld[i] = in ? fma(-smin, (double)t, lc_in[r]) : -INFINITY;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            double m = -INFINITY;
            for (int i = threadIdx.x; i < kWTile; i += 32) m = fmax(m, ld[i]);
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (threadIdx.x == 0) sh_m = m;
        }
        __syncthreads();
        const double m = sh_m;
        if (!(m > -INFINITY)) continue;                            // no coefficient in this tile
        for (int i = threadIdx.x; i < kWTile; i += blockDim.x) {
            const int64_t r = tile * kWTile + i;
            fr[i] = (r < n_rays && ld[i] > -INFINITY) ? (float)(sg_in[r] * exp(ld[i] - m)) : 0.f;
        }
        __syncthreads();
        const double em = exp(m);
        for (int b = threadIdx.x; b < F; b += blockDim.x) {
            const float eb = e2[b], ebt = e2t[b];
            float S = 0.f, c = 0.f;
            for (int i = 0; i < kWTile; ++i) {
                const float t = tt[i];
                const float p = eb * t;
                const float err = fmaf(ebt, t, fmaf(eb, t, -p));
                const float v0 = fr[i] * exp2f(-p);
                const float v = fmaf(-v0, err * 0.6931471805599453f, v0);
                const float yy = v - c;
                const float u = S + yy;
                c = (u - S) - yy;
                S = u;
            }
            acc[b] = fma((double)S, em, acc[b]);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < F; b += blockDim.x) partial[(int64_t)blockIdx.x * F + b] = acc[b];
}

// per-ray coefficient of Eq. gamma_shld's reverse mode: c_r = gamma_bar_o / R
__global__ void k_gamma_coef(int64_t n_rays, int R, const double* __restrict__ gbar, double* lc, double* sg)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
        const double c = gbar[r / R] / (double)R;
        lc[r] = c != 0.0 ? log(fabs(c)) : -INFINITY;
        sg[r] = c < 0.0 ? -1.0 : 1.0;
    }
}

// out[b] += sum over blocks of partial[block * F + b] (fixed order)
__global__ void k_sum_partials(const double* __restrict__ partial, int nb, int F, double* out)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < F; b += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nb; ++q) t += partial[(int64_t)q * F + b];
        out[b] += t;
    }
}

// gamma_bar_i = x_bar_i dx_i/dGamma_i (App. C3 root, case as in k_equilibrium)
__global__ void k_equilibrium_vjp(const double* __restrict__ gamma, const float* __restrict__ tau_eff,
                                  const double* __restrict__ nH, const double* __restrict__ T, int64_t n,
                                  int case_rule, double y, const double* __restrict__ x_bar, double* gamma_bar)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        Rates r = hg97_rates(T[i]);
        bool caseB = case_rule == URCHIN_CASE_B ||
                     (case_rule == URCHIN_CASE_AUTO && tau_eff[i] >= 1.0f);
        const double alpha = caseB ? r.alphaB : r.alphaA;
        const double x = x_equilibrium(gamma[i], nH[i], alpha, r.gamma_c, y);
        gamma_bar[i] = x_bar[i] * dx_dgamma(x, nH[i], alpha, r.gamma_c, gamma[i], y);
    }
}

// Near/far rate per origin (Eqs. gammafar, gammashldk, gammashld), one
// thread per origin, in double: ln(Gamma_far,k / Gamma_thin) by the factored
// fold, the slab solution per ray, then a log-sum-exp over the rays.
template <typename Real>
__global__ void k_gamma_nearfar(const Real* __restrict__ tf, const Real* __restrict__ tn, int64_t n_orig, int R,
                                const double* __restrict__ sv, const double* __restrict__ wv, int F,
                                const double* __restrict__ nH, const double* __restrict__ T,
                                const uint8_t* __restrict__ caseB, SpecTable poly, double* gamma_out,
                                float* tau_eff_out)
{
    extern __shared__ double sm[];
    double* ss = sm;
    double* ws = sm + F;
    __shared__ double sh[2];
    if (threadIdx.x == 0) {
        double g = 0.0, m = sv[0];
        for (int b = 0; b < F; ++b) {
            g += wv[b];
            m = fmin(m, sv[b]);
        }
        sh[0] = g;
        sh[1] = m;
    }
    __syncthreads();
    const double gthin = sh[0], smin = sh[1];
    for (int b = threadIdx.x; b < F; b += blockDim.x) {
        ss[b] = sv[b] - smin;
        ws[b] = wv[b] / gthin;
    }
    __syncthreads();
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_orig; o += (int64_t)gridDim.x * blockDim.x) {
        const Rates r = hg97_rates(T[o]);
        const double alpha = (caseB && caseB[o]) ? r.alphaB : r.alphaA;
        double m = -INFINITY, acc = 0.0;
        for (int k = 0; k < R; ++k) {
            const double t = (double)tf[o * R + k];
            double l;
            // the ray's share (1/R) of the radiation lights its slab; rates add over rays
            const double lnR = log((double)R);
            if (poly.tab) {
                // FP32 columns: the slab's table and x_eq in FP32 (see slab_poly_lnratio32)
                l = (sizeof(Real) == 4 ? slab_poly_lnratio32(poly, gthin, t, (double)tn[o * R + k], nH[o], alpha,
                                                             r.gamma_c, -lnR)
                                       : slab_poly_lnratio(poly, gthin, t, (double)tn[o * R + k], nH[o], alpha,
                                                           r.gamma_c, -lnR)) +
                    lnR;
            } else {
                double S = 0.0;
                for (int b = 0; b < F; ++b) S += ws[b] * exp(-ss[b] * t);
                l = slab_lnratio(-smin * t + log(S) - lnR, gthin, (double)tn[o * R + k], nH[o], alpha, r.gamma_c) +
                    lnR;
            }
            if (!(l > -INFINITY)) continue;
            if (l > m) {
                acc = acc * exp(m - l) + 1.0;
                m = l;
            } else {
                acc += exp(l - m);
            }
        }
        const double lr = m + log(acc / (double)R);
        gamma_out[o] = gthin * exp(lr);
        if (tau_eff_out) tau_eff_out[o] = (float)(-lr);
    }
}

// tab[i] = (ln sum_b w_b e^{-s_b tau_i}, d/du), tau_i = e^{u_i} - 1, u_i = i umax / nt,
// in double with the factored sum; smin_out[0] = min_b s_b
__global__ void k_spec_table(const double* __restrict__ sv, const double* __restrict__ wv, int F, int nt,
                             double umax, double2* tab, float2* tab32, double* smin_out)
{
    double smin = sv[0], gthin = 0.0;
    for (int b = 1; b < F; ++b) smin = fmin(smin, sv[b]);
    for (int b = 0; b < F; ++b) gthin += wv[b];
    const double lnthin = log(gthin);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        smin_out[0] = smin;
        smin_out[1] = lnthin;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nt; i += gridDim.x * blockDim.x) {
        const double u = umax * (double)i / (double)nt;
        const double tau = expm1(u);
        double S = 0.0, S1 = 0.0;
        for (int b = 0; b < F; ++b) {
            const double e = wv[b] * exp(-(sv[b] - smin) * tau);
            S += e;
            S1 += sv[b] * e;
        }
        // d/du = (d/dtau)(1 + tau), d ln Gamma / d tau = -S1 / S
        tab[i] = make_double2(-smin * tau + log(S), -(S1 / S) * (1.0 + tau));
        tab32[i] = make_float2((float)(-smin * tau + log(S) - lnthin), (float)(-(S1 / S) * (1.0 + tau)));
    }
}

// Rate behind H I, He I and He II columns, one thread per origin in double:
// per ray E_j = s_j tau + s1_j tau1 + s2_j tau2, ln sum_j w^_j exp(-E_j) with
// the smallest E_j factored out, then a log-sum-exp over the rays.
template <typename Real>
__global__ void k_gamma_he(const Real* __restrict__ t0, const Real* __restrict__ t1, const Real* __restrict__ t2,
                           int64_t n_orig, int R, const double* __restrict__ sv, const double* __restrict__ s1v,
                           const double* __restrict__ s2v, const double* __restrict__ wv, int F, double* gamma_out,
                           float* tau_eff_out)
{
    extern __shared__ double sm[];
    double* ss = sm;
    double* s1 = sm + F;
    double* s2 = sm + 2 * F;
    double* ws = sm + 3 * F;
    __shared__ double gsh;
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int b = 0; b < F; ++b) g += wv[b];
        gsh = g;
    }
    __syncthreads();
    const double gthin = gsh;
    for (int b = threadIdx.x; b < F; b += blockDim.x) {
        ss[b] = sv[b];
        s1[b] = s1v[b];
        s2[b] = s2v[b];
        ws[b] = wv[b] / gthin;
    }
    __syncthreads();
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_orig; o += (int64_t)gridDim.x * blockDim.x) {
        double m = -INFINITY, acc = 0.0;
        for (int k = 0; k < R; ++k) {
            const double a = (double)t0[o * R + k], b1 = (double)t1[o * R + k], b2 = (double)t2[o * R + k];
            double emin = INFINITY;
            for (int b = 0; b < F; ++b) emin = fmin(emin, ss[b] * a + s1[b] * b1 + s2[b] * b2);
            double S = 0.0;
            for (int b = 0; b < F; ++b) S += ws[b] * exp(-(ss[b] * a + s1[b] * b1 + s2[b] * b2 - emin));
            const double l = -emin + log(S);
            if (!(l > -INFINITY)) continue;
            if (l > m) {
                acc = acc * exp(m - l) + 1.0;
                m = l;
            } else {
                acc += exp(l - m);
            }
        }
        const double lr = m + log(acc / (double)R);
        gamma_out[o] = gthin * exp(lr);
        if (tau_eff_out) tau_eff_out[o] = (float)(-lr);
    }
}


template <typename Real>
int gamma_vjp_t(const Real* tau, int64_t n_orig, int R, const urchin_spectrum* sp, const double* gbar,
                Real* tau_bar, double* w_bar, cudaStream_t s)
{
    const int64_t n_rays = n_orig * (int64_t)R;
    const int F = sp->F;
    if (tau_bar) {
        const size_t smem = sizeof(double) * 2 * (size_t)F;
        auto fn = k_gamma_vjp_tau<Real>;
        if (smem > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int grid = 0;
        URCHIN_TRY(grid_for((const void*)fn, 256, smem, &grid));
        grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (n_rays + 255) / 256));
        fn<<<grid, 256, smem, s>>>(tau, n_rays, R, sp->s, sp->w, F, gbar, tau_bar);
        URCHIN_TRY(launched());
    }
    if (w_bar) {
        Scratch cf;
        URCHIN_TRY(cf.alloc(2 * sizeof(double) * (size_t)n_rays + 256, s));
        double* lc = cf.at<double>(0);
        double* sg = lc + n_rays;
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_rays + 255) / 256, 4096));
        k_gamma_coef<<<g, 256, 0, s>>>(n_rays, R, gbar, lc, sg);
        URCHIN_TRY(launched());
        URCHIN_TRY(launch_wbar(tau, sizeof(Real) == 8 ? URCHIN_F64 : URCHIN_F32, n_rays, lc, sg, sp->s, F, w_bar, s));
        cf.release();
    }
    return URCHIN_OK;
}

}  // namespace

size_t spec_table_bytes() { return sizeof(double2) * (kSpecTab + 1) + 64 + sizeof(float2) * (kSpecTab + 1); }

int build_spec_table(const double* s, const double* w, int F, void* buf, SpecTable* out, cudaStream_t st)
{
    double2* tab = static_cast<double2*>(buf);
    double* sc = reinterpret_cast<double*>(tab + kSpecTab + 1);          // smin, ln Gamma_thin
    float2* tab32 = reinterpret_cast<float2*>(reinterpret_cast<char*>(sc) + 64);
    k_spec_table<<<(kSpecTab + 256) / 256, 256, 0, st>>>(s, w, F, kSpecTab, log1p(kSpecTauMax), tab, tab32, sc);
    URCHIN_TRY(launched());
    double h[2] = {0.0, 0.0};
    URCHIN_TRY_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(st));
    *out = SpecTable{tab, kSpecTab, log1p(kSpecTauMax), h[0], tab32, h[1]};
    return URCHIN_OK;
}

int launch_wbar(const void* tau, int precision, int64_t n_rays, const double* lc, const double* sg, const double* sv,
                int F, double* w_bar, cudaStream_t s)
{
    if (n_rays <= 0) return URCHIN_OK;
    const bool f64 = precision == URCHIN_F64;
    const size_t smem = f64 ? sizeof(double) * (2 * (size_t)F + 3 * kWTile)
                            : sizeof(double) * ((size_t)F + kWTile) + sizeof(float) * (2 * (size_t)F + 2 * kWTile);
    const void* fn = f64 ? (const void*)k_wbar_tiles<double> : (const void*)k_wbar_tiles_f32;
    if (smem > 48 * 1024)
        URCHIN_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t tiles = (n_rays + kWTile - 1) / kWTile;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, 608));
    Scratch part;
    URCHIN_TRY(part.alloc(sizeof(double) * (size_t)nb * F, s));
    if (precision == URCHIN_F64)
        k_wbar_tiles<double><<<nb, 256, smem, s>>>(static_cast<const double*>(tau), n_rays, lc, sg, sv, F,
                                                   part.at<double>(0));
    else
        k_wbar_tiles_f32<<<nb, 256, smem, s>>>(static_cast<const float*>(tau), n_rays, lc, sg, sv, F,
                                               part.at<double>(0));
    URCHIN_TRY(launched());
    k_sum_partials<<<(F + 255) / 256, 256, 0, s>>>(part.at<double>(0), nb, F, w_bar);
    URCHIN_TRY(launched());
    part.release();
    return URCHIN_OK;
}

int launch_gamma(const GammaJob& J, cudaStream_t s)
{
    if (J.n_rows <= 0) return URCHIN_OK;
    if (J.precision == URCHIN_F64) return launch_gamma_t<double>(J, s);
    return launch_gamma_t<float>(J, s);
}

int launch_equilibrium(const double* gamma, const float* tau_eff, const double* nH, const double* T,
                       int64_t n, int case_rule, double y, double* x_out, cudaStream_t s)
{
    if (n <= 0) return URCHIN_OK;
    unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_equilibrium<<<grid, 256, 0, s>>>(gamma, tau_eff, nH, T, n, case_rule, y, x_out);
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

}  // namespace urchin

extern "C" int urchin_gamma(const void* tau, int precision, int64_t n_orig, int R, const urchin_spectrum* sp,
                            double* gamma_out, float* tau_eff_out, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (precision != URCHIN_F32 && precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma: unknown precision %d", precision);
    if (R < 1 || R > URCHIN_MAX_RAYS) return set_error(URCHIN_ERR_ARG, "urchin_gamma: R = %d out of range", R);
    if (n_orig < 0) return set_error(URCHIN_ERR_ARG, "urchin_gamma: n_orig < 0");
    if (!sp || !sp->s || !sp->w) return set_error(URCHIN_ERR_ARG, "urchin_gamma: NULL spectrum");
    if (sp->F < 1 || sp->F > URCHIN_MAX_BINS)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma: F = %d out of range [1, %d]", sp->F, URCHIN_MAX_BINS);
    if (spectrum_has_he(sp)) return set_error(URCHIN_ERR_ARG, "urchin_gamma: helium spectrum (use urchin_gamma_he)");
    if (n_orig == 0) return URCHIN_OK;
    if (!tau || !gamma_out) return set_error(URCHIN_ERR_ARG, "urchin_gamma: NULL tau or gamma_out");
    GammaJob J{};
    J.tau = tau;
    J.precision = precision;
    J.n_rows = n_orig;
    J.R = R;
    J.row_stride = R;
    J.k_stride = 1;
    J.s = sp->s;
    J.w = sp->w;
    J.F = sp->F;
    J.gamma_out = gamma_out;
    J.tau_eff_out = tau_eff_out;
    return launch_gamma(J, (cudaStream_t)stream);
}

extern "C" int urchin_equilibrium(const double* gamma, const float* tau_eff, const double* nH, const double* T,
                                  int64_t n, int case_rule, double y, double* x_out, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (n < 0) return set_error(URCHIN_ERR_ARG, "urchin_equilibrium: n < 0");
    if (case_rule != URCHIN_CASE_A && case_rule != URCHIN_CASE_B && case_rule != URCHIN_CASE_AUTO)
        return set_error(URCHIN_ERR_ARG, "urchin_equilibrium: unknown case_rule %d", case_rule);
    if (!(y >= 0.0) || !std::isfinite(y)) return set_error(URCHIN_ERR_ARG, "urchin_equilibrium: y must be >= 0");
    if (n == 0) return URCHIN_OK;
    if (!gamma || !nH || !T || !x_out) return set_error(URCHIN_ERR_ARG, "urchin_equilibrium: NULL array");
    if (case_rule == URCHIN_CASE_AUTO && !tau_eff)
        return set_error(URCHIN_ERR_ARG, "urchin_equilibrium: CASE_AUTO needs tau_eff");
    return launch_equilibrium(gamma, tau_eff, nH, T, n, case_rule, y, x_out, (cudaStream_t)stream);
}

extern "C" int urchin_gamma_vjp(const void* tau, int precision, int64_t n_orig, int R, const urchin_spectrum* sp,
                                const double* gamma_bar, void* tau_bar_out, double* w_bar, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (precision != URCHIN_F32 && precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: unknown precision %d", precision);
    if (R < 1 || R > URCHIN_MAX_RAYS) return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: R = %d out of range", R);
    if (n_orig < 0) return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: n_orig < 0");
    if (!sp || !sp->s || !sp->w) return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: NULL spectrum");
    if (sp->F < 1 || sp->F > URCHIN_MAX_BINS)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: F = %d out of range [1, %d]", sp->F, URCHIN_MAX_BINS);
    if (spectrum_has_he(sp)) return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: no helium columns in reverse mode");
    if (n_orig == 0) return URCHIN_OK;
    if (!tau || !gamma_bar) return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: NULL tau or gamma_bar");
    if (!tau_bar_out && !w_bar) return set_error(URCHIN_ERR_ARG, "urchin_gamma_vjp: no output requested");
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == URCHIN_F64)
        return gamma_vjp_t<double>(static_cast<const double*>(tau), n_orig, R, sp, gamma_bar,
                                   static_cast<double*>(tau_bar_out), w_bar, s);
    return gamma_vjp_t<float>(static_cast<const float*>(tau), n_orig, R, sp, gamma_bar,
                              static_cast<float*>(tau_bar_out), w_bar, s);
}

extern "C" int urchin_equilibrium_vjp(const double* gamma, const float* tau_eff, const double* nH, const double* T,
                                      int64_t n, int case_rule, double y, const double* x_bar, double* gamma_bar_out,
                                      urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (n < 0) return set_error(URCHIN_ERR_ARG, "urchin_equilibrium_vjp: n < 0");
    if (case_rule != URCHIN_CASE_A && case_rule != URCHIN_CASE_B && case_rule != URCHIN_CASE_AUTO)
        return set_error(URCHIN_ERR_ARG, "urchin_equilibrium_vjp: unknown case_rule %d", case_rule);
    if (!(y >= 0.0) || !std::isfinite(y)) return set_error(URCHIN_ERR_ARG, "urchin_equilibrium_vjp: y must be >= 0");
    if (n == 0) return URCHIN_OK;
    if (!gamma || !nH || !T || !x_bar || !gamma_bar_out)
        return set_error(URCHIN_ERR_ARG, "urchin_equilibrium_vjp: NULL array");
    if (case_rule == URCHIN_CASE_AUTO && !tau_eff)
        return set_error(URCHIN_ERR_ARG, "urchin_equilibrium_vjp: CASE_AUTO needs tau_eff");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_equilibrium_vjp<<<grid, 256, 0, s>>>(gamma, tau_eff, nH, T, n, case_rule, y, x_bar, gamma_bar_out);
    return launched();
}

extern "C" int urchin_gamma_nearfar(const void* tau_far, const void* tau_near, int precision, int64_t n_orig, int R,
                                    const urchin_spectrum* sp, const double* nH, const double* T,
                                    const unsigned char* caseB, int slab, double* gamma_out, float* tau_eff_out,
                                    urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (precision != URCHIN_F32 && precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: unknown precision %d", precision);
    if (R < 1 || R > URCHIN_MAX_RAYS) return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: R = %d out of range", R);
    if (n_orig < 0) return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: n_orig < 0");
    if (!sp || !sp->s || !sp->w) return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: NULL spectrum");
    if (sp->F < 1 || sp->F > URCHIN_MAX_BINS)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: F = %d out of range [1, %d]", sp->F, URCHIN_MAX_BINS);
    if (n_orig == 0) return URCHIN_OK;
    if (slab != URCHIN_SLAB_THRESHOLD && slab != URCHIN_SLAB_SPECTRUM)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: unknown slab model %d", slab);
    if (spectrum_has_he(sp)) return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: the slab is hydrogen only");
    if (!tau_far || !tau_near || !nH || !T || !gamma_out)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_nearfar: NULL tau_far, tau_near, nH, T or gamma_out");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch tb;
    SpecTable poly{nullptr, kSpecTab, log1p(kSpecTauMax), 0.0, nullptr, 0.0};
    if (slab == URCHIN_SLAB_SPECTRUM) {
        URCHIN_TRY(tb.alloc(spec_table_bytes(), s));
        URCHIN_TRY(build_spec_table(sp->s, sp->w, sp->F, tb.at<void>(0), &poly, s));
    }
    const size_t smem = sizeof(double) * 2 * (size_t)sp->F;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_orig + 127) / 128, 4096));
    if (precision == URCHIN_F64) {
        if (smem > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(k_gamma_nearfar<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        k_gamma_nearfar<double><<<grid, 128, smem, s>>>(static_cast<const double*>(tau_far),
                                                        static_cast<const double*>(tau_near), n_orig, R, sp->s,
                                                        sp->w, sp->F, nH, T, caseB, poly, gamma_out, tau_eff_out);
    } else {
        if (smem > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(k_gamma_nearfar<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        k_gamma_nearfar<float><<<grid, 128, smem, s>>>(static_cast<const float*>(tau_far),
                                                       static_cast<const float*>(tau_near), n_orig, R, sp->s,
                                                       sp->w, sp->F, nH, T, caseB, poly, gamma_out, tau_eff_out);
    }
    URCHIN_TRY(launched());
    tb.release();
    return URCHIN_OK;
}

extern "C" int urchin_gamma_he(const void* tau, const void* tau_he1, const void* tau_he2, int precision,
                               int64_t n_orig, int R, const urchin_spectrum* sp, double* gamma_out,
                               float* tau_eff_out, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (precision != URCHIN_F32 && precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_he: unknown precision %d", precision);
    if (R < 1 || R > URCHIN_MAX_RAYS) return set_error(URCHIN_ERR_ARG, "urchin_gamma_he: R = %d out of range", R);
    if (n_orig < 0) return set_error(URCHIN_ERR_ARG, "urchin_gamma_he: n_orig < 0");
    if (!sp || !sp->s || !sp->w || !sp->s_he1 || !sp->s_he2)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_he: the spectrum needs s, w, s_he1 and s_he2");
    if (sp->F < 1 || sp->F > URCHIN_MAX_BINS)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_he: F = %d out of range [1, %d]", sp->F, URCHIN_MAX_BINS);
    if (n_orig == 0) return URCHIN_OK;
    if (!tau || !tau_he1 || !tau_he2 || !gamma_out)
        return set_error(URCHIN_ERR_ARG, "urchin_gamma_he: NULL column or gamma_out");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t smem = sizeof(double) * 4 * (size_t)sp->F;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_orig + 127) / 128, 4096));
    if (precision == URCHIN_F64) {
        if (smem > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(k_gamma_he<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        k_gamma_he<double><<<grid, 128, smem, s>>>(static_cast<const double*>(tau), static_cast<const double*>(tau_he1),
                                                   static_cast<const double*>(tau_he2), n_orig, R, sp->s, sp->s_he1,
                                                   sp->s_he2, sp->w, sp->F, gamma_out, tau_eff_out);
    } else {
        if (smem > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(k_gamma_he<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem));
        k_gamma_he<float><<<grid, 128, smem, s>>>(static_cast<const float*>(tau), static_cast<const float*>(tau_he1),
                                                  static_cast<const float*>(tau_he2), n_orig, R, sp->s, sp->s_he1,
                                                  sp->s_he2, sp->w, sp->F, gamma_out, tau_eff_out);
    }
    return launched();
}

