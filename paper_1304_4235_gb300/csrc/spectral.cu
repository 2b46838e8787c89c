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

// Shared spectrum prepared by every block: coefficients of exp2 and the
// normalised weights, plus Gamma_thin and s_min.
template <typename Real>
__device__ void load_spectrum(const double* s, const double* w, int F, Real* e2, Real* wn, double* sh)
{
    // sh[0] = Gamma_thin, sh[1] = s_min
    __shared__ double red[kGammaThreads / 32][2];
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
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            t += red[i][0];
            m = fmin(m, red[i][1]);
        }
        sh[0] = t;
        sh[1] = m;
    }
    __syncthreads();
    const double g = sh[0], m = sh[1];
    for (int j = threadIdx.x; j < F; j += blockDim.x) {
        // exp(-(s_j - s_min) tau) = exp2(-e2_j tau) with e2_j = (s_j - s_min) log2(e)
        e2[j] = (Real)((s[j] - m) * 1.4426950408889634);
        wn[j] = (Real)(w[j] / g);
    }
    __syncthreads();
}

template <typename Real>
__device__ __forceinline__ Real ray_log_rate(Real tau, const Real* e2, const Real* wn, int F, Real smin)
{
    Real S = Real(0), c = Real(0);
    for (int j = 0; j < F; ++j) {
        Real v = wn[j] * exp2_p(-e2[j] * tau);
        Real y = v - c;
        Real t = S + y;
        c = (t - S) - y;
        S = t;
    }
    return -smin * tau + log_p(S);
}

// Threads (local, k) fold ray k of row `local`; the per-row log-sum-exp runs
// with one thread per row packed into the first lanes.
template <typename Real>
__global__ void __launch_bounds__(kGammaThreads) k_gamma(GammaJob J)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Real* e2 = reinterpret_cast<Real*>(smem_raw);
    Real* wn = e2 + J.F;
    Real* lk = reinterpret_cast<Real*>(smem_raw + ((2 * (size_t)J.F * sizeof(Real) + 15) & ~size_t(15)));
    __shared__ double sh[2];
    load_spectrum<Real>(J.s, J.w, J.F, e2, wn, sh);
    const int rows_per_block = kGammaThreads / J.R;
    const int local = threadIdx.x / J.R;
    const int k = threadIdx.x % J.R;
    const double gthin = sh[0];
    const Real smin = (Real)sh[1];
    for (int64_t row0 = (int64_t)blockIdx.x * rows_per_block; row0 < J.n_rows;
         row0 += (int64_t)gridDim.x * rows_per_block) {
        const int64_t row = row0 + local;
        if (local < rows_per_block && row < J.n_rows) {
            const Real tau = static_cast<const Real*>(J.tau)[row * J.row_stride + (int64_t)k * J.k_stride];
            lk[local * J.R + k] = ray_log_rate<Real>(tau, e2, wn, J.F, smin);
        }
        __syncthreads();
        const int p = threadIdx.x;
        const int64_t prow = row0 + p;
        if (p < rows_per_block && prow < J.n_rows) {
            const Real* l = lk + p * J.R;
            Real m = l[0];
            for (int r = 1; r < J.R; ++r) m = m > l[r] ? m : l[r];
            Real acc = Real(0);
            for (int r = 0; r < J.R; ++r) acc += exp_p(l[r] - m);
            const double lmean = (double)(m + log_p(acc / (Real)J.R));    // ln(Gamma / Gamma_thin)
            J.gamma_out[prow] = gthin * exp(lmean);
            if (J.tau_eff_out) J.tau_eff_out[prow] = (float)(-lmean);
        }
        __syncthreads();
    }
}

template <typename Real>
int launch_gamma_t(const GammaJob& J, cudaStream_t s)
{
    size_t smem = ((2 * (size_t)J.F * sizeof(Real) + 15) & ~size_t(15)) + sizeof(Real) * kGammaThreads;
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

}  // namespace

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
