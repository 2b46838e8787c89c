// Iteration driver of Sec. 4: x starts at x_thin, sweep 0 traces every
// particle and freezes those with tau_eff < tau_skip, later sweeps trace the
// non-frozen particles and update them all from the previous sweep's x
// (Jacobi), until max |dx|/x < dx_tol.
//
// State lives in Morton order on the device.  A sweep is two kernels: the
// persistent traversal (columns of all active rays) and a fused kernel that
// folds each particle's R columns through the spectrum, solves the
// equilibrium in FP64, writes x and the tracer weight A_j x_j, and reduces
// max |dx|/x.  The host reads that scalar once per sweep.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "linalg.cuh"
#include "solver.cuh"
#include "spectral_device.cuh"

namespace urchin {

namespace {

constexpr int kSweepThreads = 256;

__global__ void k_setup(const urchin_bvh b, const double* __restrict__ nH, const double* __restrict__ T,
                        const double* __restrict__ x_in, int warm, double gthin, int case_rule, double y,
                        double* nHm, double* aA, double* aB, double* gc, double* x, float* w32, double* w64,
                        float* xs32, double* xs64, unsigned* status)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < b.n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = b.perm[s];
        double n_ = nH[i], t_ = T[i];
        if (!(n_ > 0.0) || !(t_ > 0.0) || !isfinite(n_) || !isfinite(t_)) atomicOr(status, kStInput);
        Rates r = hg97_rates(t_);
        nHm[s] = n_;
        aA[s] = r.alphaA;
        aB[s] = r.alphaB;
        gc[s] = r.gamma_c;
        double xv;
        if (warm) {
            xv = x_in[i];
            if (!(xv > 0.0) || !(xv <= 1.0)) atomicOr(status, kStWarm);
        } else {
            // x_thin: Gamma = Gamma_thin, tau_eff = 0 (case A unless forced to B)
            xv = x_equilibrium(gthin, n_, case_rule == URCHIN_CASE_B ? r.alphaB : r.alphaA, r.gamma_c, y);
        }
        x[s] = xv;
        double wv = b.A64[s] * xv;
        if (w32) w32[s] = (float)wv;
        if (w64) w64[s] = wv;
        if (xs32) xs32[s] = (float)xv;
        if (xs64) xs64[s] = xv;
    }
}

// The active list's ray order from the order of all particles (Solver::
// derive_list_order): list positions of the particles, each direction's
// full order flagged where its particle is active, and the compacted slots
// mapped to list positions.
__global__ void k_list_pos(const int32_t* __restrict__ list, int64_t na, int64_t n, int32_t* __restrict__ pos)
{
    for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = list[a];
        if ((uint64_t)i < (uint64_t)n) pos[i] = (int32_t)a;
    }
}

__global__ void k_order_flags(const int32_t* __restrict__ order, const uint8_t* __restrict__ active, int64_t n,
                              uint8_t* __restrict__ flags)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = order[t];
        flags[t] = (uint64_t)i < (uint64_t)n && active[i] ? 1 : 0;
    }
}

__global__ void k_order_map(const int32_t* __restrict__ order, const int32_t* __restrict__ pos, int64_t na,
                            int32_t* __restrict__ out)
{
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < na; m += (int64_t)gridDim.x * blockDim.x)
        out[m] = pos[order[out[m]]];
}

__global__ void k_finish(const int32_t* __restrict__ perm, const double* __restrict__ x, int64_t n, double* x_out)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        x_out[perm[s]] = x[s];
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* addr, double v)
{
    // non-negative doubles order like their bit patterns
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// The per-particle end of a sweep, from ln(Gamma/Gamma_thin) of item prow:
// the freeze decision (sweep 0), the recombination case (latched at
// tau_eff >= 1), the FP64 equilibrium root and the convergence counters, then
// x (and its copies) or xeq_out.  Returns the particle's Morton slot, or -1
// when it is not updated (frozen in sweep 0).
__device__ __forceinline__ int32_t particle_update(const SweepArgs& A, int64_t prow, double lmean, double gthin,
                                                   double* xn_out, double* G_out, double* alpha_out,
                                                   double& my_max, unsigned long long& my_above,
                                                   unsigned long long& my_switch, unsigned& err)
{
    const double G = gthin * exp(lmean);
    const double te = -lmean;
    const int32_t i = A.items ? A.items[prow] : (int32_t)prow;
    bool update = true;
    if (A.sweep0) {
        update = !(te < A.tau_skip);
        A.active[i] = update ? 1 : 0;
    }
    if (A.gamma_out) A.gamma_out[prow] = G;
    if (A.tau_eff_out) A.tau_eff_out[prow] = (float)te;
    if (!update) return -1;
    // case B iff tau_eff >= 1, latched once reached (see urchin_solve)
    bool caseB = A.case_rule == URCHIN_CASE_B;
    if (A.case_rule == URCHIN_CASE_AUTO) {
        const bool latched = A.latch[i] != 0;
        if (A.latch_frozen) {
            caseB = latched;
            if (te >= 1.0 && !latched) ++my_switch;
        } else {
            caseB = latched || te >= 1.0;
            A.latch[i] = caseB ? 1 : 0;
        }
    }
    const double alpha = caseB ? A.aB[i] : A.aA[i];
    const double xo = A.x[i];
    const double xn = x_equilibrium(G, A.nH[i], alpha, A.gc[i], A.y);
    if (!isfinite(xn) || !(xn > 0.0)) err |= kStNonfinite;
    const double rel = fabs(xn - xo) / xo;
    my_max = fmax(my_max, rel);
    if (rel >= A.tol) ++my_above;
    if (A.xeq_out) {
        A.xeq_out[prow] = xn;
    } else {
        A.x[i] = xn;
        const double wv = A.A64[i] * xn;
        if (A.w32) A.w32[i] = (float)wv;
        if (A.w64) A.w64[i] = wv;
        if (A.xs32) A.xs32[i] = (float)xn;
        if (A.xs64) A.xs64[i] = xn;
    }
    *xn_out = xn;
    *G_out = G;
    *alpha_out = alpha;
    return i;
}

// Warp-wide reduction of the convergence counters into the call's scalars.
__device__ __forceinline__ void sweep_counters(const SweepArgs& A, double my_max, unsigned long long my_above,
                                               unsigned long long my_switch, unsigned err)
{
    for (int o = 16; o > 0; o >>= 1) {
        my_max = fmax(my_max, __shfl_xor_sync(0xffffffffu, my_max, o));
        my_above += __shfl_xor_sync(0xffffffffu, my_above, o);
        my_switch += __shfl_xor_sync(0xffffffffu, my_switch, o);
        err |= __shfl_xor_sync(0xffffffffu, err, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (my_max > 0.0) atomic_max_pos(A.maxrel, my_max);
        if (my_above && A.n_above) atomicAdd(A.n_above, my_above);
        if (my_switch && A.n_switch) atomicAdd(A.n_switch, my_switch);
        if (err) atomicOr(A.status, err);
    }
}

// The plain sweep without tangent, one thread per particle: its R rays are
// folded in turn (Eq. gamma_shld, fold_ray) with a running log-sum-exp over
// the rays, then every lane takes its particle's FP64 update at once (the
// ray-parallel layout of k_sweep leaves all but one warp of the block idle
// during the FP64 part).
template <typename Real>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_pp(SweepArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kF32 = sizeof(Real) == 4;
    // FP32: the packed coefficients {e2, e2t, wn, 0} of fold_ray_q4; FP64:
    // e2 and wn
    float4* q4 = kF32 ? reinterpret_cast<float4*>(smem_raw) : nullptr;
    Real* e2 = kF32 ? nullptr : reinterpret_cast<Real*>(smem_raw);
    Real* wn = kF32 ? nullptr : e2 + A.F;
    __shared__ double sh[2];
    fold_prepare<Real>(A.s, A.w, A.F, e2, nullptr, wn, nullptr, sh, q4);
    const double gthin = sh[0];
    const double smin = sh[1];
    const Real* tau = static_cast<const Real*>(A.tau);
    double my_max = 0.0;
    unsigned long long my_above = 0, my_switch = 0;
    unsigned err = 0;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < A.n_items;
         row += (int64_t)gridDim.x * blockDim.x) {
        RayMean<Real> lse;
        for (int k = 0; k < A.R; ++k) {
            const Real t = tau[row + (int64_t)k * A.k_stride];
            Real S, S2;
            if constexpr (kF32) S = fold_ray_q4(t, q4, A.F);
            else fold_ray<false>(t, e2, nullptr, wn, nullptr, A.F, S, S2);
            lse.add(ray_lnrate(smin, t, S));
        }
        double xn, G, alpha;
        particle_update(A, row, lse.mean(A.R), gthin, &xn, &G, &alpha, my_max, my_above, my_switch, err);
    }
    sweep_counters(A, my_max, my_above, my_switch, err);
}

// Instantiations of the sweep: the plain fold, the near/far split (slab of the
// near particles), the helium columns.  Separate so that the plain sweep keeps
// the register footprint (and occupancy) of the fold alone.
constexpr int kSweepPlain = 0, kSweepNearFar = 1, kSweepHelium = 2;

// One sweep's spectral fold + equilibrium update (see file comment).  With
// want_tangent, also stores per ray c_tk = (1/E) dE/dGamma dGamma/dtau_k for
// the Newton tangent (in log-safe form).
//
// Threads (local, k) fold ray k of particle `local` through the spectrum in
// the columns' precision; the per-particle tail (the log-sum-exp over rays,
// then the FP64 equilibrium) runs with one thread per particle packed into
// the first lanes, so the FP64 work is not spread over mostly idle warps.
template <typename Real, int VAR>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(SweepArgs A)
{
    constexpr bool kHe = VAR == kSweepHelium;
    constexpr bool kNF = VAR == kSweepNearFar;
    constexpr bool kF32 = sizeof(Real) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // per-ray log rates in double, then the spectrum arrays (sweep_smem_bytes)
    double* lk = reinterpret_cast<double*>(smem_raw);
    double* lk2 = lk + kSweepThreads;
    Real* e2 = reinterpret_cast<Real*>(lk2 + kSweepThreads);
    Real* wn = e2 + A.F;
    Real* sj = wn + A.F;
    Real* e2t = kF32 ? sj + A.F : nullptr;
    Real* sh1 = sj + (kF32 ? 2 : 1) * A.F;      // helium cross sections (kHe) and, in FP32,
    Real* sh2 = sh1 + A.F;                      // the float tails of all three (fold_ray_he)
    Real* sjt = sh2 + A.F;
    Real* sh1t = sjt + A.F;
    Real* sh2t = sh1t + A.F;
    __shared__ double sh[2];
    fold_prepare<Real>(A.s, A.w, A.F, e2, e2t, wn, (A.want_tangent || kHe) ? sj : nullptr, sh);
    if (kHe) {
        for (int j = threadIdx.x; j < A.F; j += blockDim.x) {
            sh1[j] = (Real)A.s_he1[j];
            sh2[j] = (Real)A.s_he2[j];
            if (kF32) {
                sjt[j] = (Real)(A.s[j] - (double)(Real)A.s[j]);
                sh1t[j] = (Real)(A.s_he1[j] - (double)(Real)A.s_he1[j]);
                sh2t[j] = (Real)(A.s_he2[j] - (double)(Real)A.s_he2[j]);
            }
        }
        __syncthreads();
    }
    const int rows_per_block = kSweepThreads / A.R;
    const int local = threadIdx.x / A.R;
    const int k = threadIdx.x % A.R;
    const double gthin = sh[0];
    const double smin = sh[1];
    double my_max = 0.0;
    unsigned long long my_above = 0, my_switch = 0;
    unsigned err = 0;
    for (int64_t row0 = (int64_t)blockIdx.x * rows_per_block; row0 < A.n_items;
         row0 += (int64_t)gridDim.x * rows_per_block) {
        const int64_t row = row0 + local;
        if (local < rows_per_block && row < A.n_items) {
            const Real tau = static_cast<const Real*>(A.tau)[row + (int64_t)k * A.k_stride];
            // (near/far: tau is the far column; the slab of near particles is applied below)
            const bool fold = !((kNF && A.near_far == URCHIN_SLAB_SPECTRUM) || kHe);
            Real S = Real(0), S2 = Real(0);
            if (fold) {
                if (A.want_tangent) fold_ray<true>(tau, e2, e2t, wn, sj, A.F, S, S2);
                else fold_ray<false>(tau, e2, e2t, wn, nullptr, A.F, S, S2);
            }
            // ln(Gamma_k / Gamma_thin) = -s_min tau_k + ln S_k
            double lkv = fold ? ray_lnrate(smin, tau, S) : 0.0;
            if (kHe && kF32) {
                // H I, He I and He II columns: E_j = s_j tau + s1_j tau1 + s2_j tau2 (fold_ray_he)
                const int32_t ir = A.items ? A.items[row] : (int32_t)row;
                const float t1 = static_cast<const float*>(A.tau_he1)[ir + (int64_t)k * A.near_k_stride];
                const float t2 = static_cast<const float*>(A.tau_he2)[ir + (int64_t)k * A.near_k_stride];
                lkv = fold_ray_he((float)tau, t1, t2, (const float*)sj, (const float*)sjt, (const float*)sh1,
                                  (const float*)sh1t, (const float*)sh2, (const float*)sh2t, (const float*)wn, A.F);
            } else if (kHe) {
                // H I, He I and He II columns: E_j = s_j tau + s1_j tau1 + s2_j tau2, the
                // smallest E_j factored out of the sum
                const int32_t ir = A.items ? A.items[row] : (int32_t)row;
                const Real t1 = static_cast<const Real*>(A.tau_he1)[ir + (int64_t)k * A.near_k_stride];
                const Real t2 = static_cast<const Real*>(A.tau_he2)[ir + (int64_t)k * A.near_k_stride];
                Real emin = sj[0] * tau + sh1[0] * t1 + sh2[0] * t2;
                for (int j = 1; j < A.F; ++j) {
                    const Real e = sj[j] * tau + sh1[j] * t1 + sh2[j] * t2;
                    emin = e < emin ? e : emin;
                }
                Real Sh = Real(0), ch = Real(0);
                for (int j = 0; j < A.F; ++j) {
                    const Real v = wn[j] * exp_p(emin - (sj[j] * tau + sh1[j] * t1 + sh2[j] * t2));
                    const Real yy = v - ch;
                    const Real t = Sh + yy;
                    ch = (t - Sh) - yy;
                    Sh = t;
                }
                lkv = -(double)emin + (double)log_p(Sh);
            }
            if (kNF) {
                // Eq. gammashldk: the far radiation enters the slab of near particles, in
                // the particle's recombination case before this sweep
                const int32_t ir = A.items ? A.items[row] : (int32_t)row;
                const bool cB = A.case_rule == URCHIN_CASE_B || (A.case_rule == URCHIN_CASE_AUTO && A.latch[ir]);
                const double tn = (double)static_cast<const Real*>(A.tau_near)[ir + (int64_t)k * A.near_k_stride];
                const double al = cB ? A.aB[ir] : A.aA[ir];
                // each slab is lit by its ray's share (1/R) of the radiation and the
                // particle's rate is the sum of the slabs' bottom rates: scale by 1/R
                // into the slab and by R out of it (the ray combination below is a mean)
                const double lnR = log((double)A.R);
                if (A.near_far == URCHIN_SLAB_SPECTRUM)
                    // FP32 sweep: the slab's table and x_eq in FP32 (slab_poly_lnratio32)
                    lkv = (kF32 ? slab_poly_lnratio32(A.poly, gthin, (double)tau, tn, A.nH[ir], al, A.gc[ir], -lnR)
                                : slab_poly_lnratio(A.poly, gthin, (double)tau, tn, A.nH[ir], al, A.gc[ir], -lnR)) +
                          lnR;
                else
                    lkv = slab_lnratio(lkv - lnR, gthin, tn, A.nH[ir], al, A.gc[ir]) + lnR;
            }
            lk[local * A.R + k] = lkv;
            if (A.want_tangent) lk2[local * A.R + k] = ray_lnrate(smin, tau, S2 > Real(1e-37) ? S2 : Real(1e-37));
        }
        __syncthreads();
        const int p = threadIdx.x;
        const int64_t prow = row0 + p;
        if (p < rows_per_block && prow < A.n_items) {
            const double* l = lk + p * A.R;
            RayMean<Real> lse;
            for (int r = 0; r < A.R; ++r) lse.add(l[r]);
            const double lmean_r = lse.mean(A.R);     // ln(Gamma/Gamma_thin)
            double xn, G, alpha;
            const int32_t i = particle_update(A, prow, lmean_r, gthin, &xn, &G, &alpha, my_max, my_above,
                                              my_switch, err);
            if (i >= 0 && A.xeq_out && A.want_tangent) {
                // elasticity Gamma dE/dGamma / E and per-ray dGamma/dtau_k / Gamma
                const double dEdG = dx_dgamma(xn, A.nH[i], alpha, A.gc[i], G, A.y);
                const double elas = (G > 0.0) ? G * dEdG / xn : 0.0;
                const double* l2 = lk2 + p * A.R;
                for (int r = 0; r < A.R; ++r) {
                    const double dlog = (double)exp_p((Real)(l2[r] - lmean_r)) / (double)A.R;
                    A.ctan[prow + (int64_t)r * A.k_stride] = -elas * dlog;
                }
            }
        }
        __syncthreads();
    }
    sweep_counters(A, my_max, my_above, my_switch, err);
}

// z_i = x_i v_a on the active particles (zero elsewhere, pre-cleared), and the
// tracer weights A_i z_i when the tangent columns are traced
__global__ void k_tangent_vector(const int32_t* __restrict__ items, int64_t n_act, const double* __restrict__ v,
                                 const double* __restrict__ x, const double* __restrict__ A64, float* z32,
                                 double* z64, float* wz32, double* wz64)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_act; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = items[a];
        const double z = x[i] * v[a];
        if (z32) z32[i] = (float)z;
        if (z64) z64[i] = z;
        if (wz32) wz32[i] = (float)(A64[i] * z);
        if (wz64) wz64[i] = A64[i] * z;
    }
}

// (J v)_a = v_a - sum_k c_ak dtau_ak
template <typename Real>
__global__ void k_jv(const double* __restrict__ v, const double* __restrict__ ctan, const Real* __restrict__ dtau,
                     int64_t n_act, int R, double* out)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_act; a += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < R; ++k) acc += ctan[a + (int64_t)k * n_act] * (double)dtau[a + (int64_t)k * n_act];
        out[a] = v[a] - acc;
    }
}

__global__ void k_gather_x(const int32_t* __restrict__ items, int64_t n_act, const double* __restrict__ x,
                           double* out)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_act; a += (int64_t)gridDim.x * blockDim.x)
        out[a] = x[items[a]];
}

// Newton residual -G_a = ln E_a - ln x_a
__global__ void k_residual(const int32_t* __restrict__ items, int64_t n_act, const double* __restrict__ x,
                           const double* __restrict__ E, double* r)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_act; a += (int64_t)gridDim.x * blockDim.x)
        r[a] = log(E[a]) - log(x[items[a]]);
}

// x_a <- x_a exp(lam d_a) (step limited to a factor e, x <= 1), or x_a <- E_a
// when E is given; refresh the tracer weights and the column-precision copy
__global__ void k_set_x(const int32_t* __restrict__ items, int64_t n_act, const double* __restrict__ d,
                        double lam, const double* __restrict__ xbase, const double* __restrict__ E, double* x,
                        const double* __restrict__ A64, float* w32, double* w64, float* xs32, double* xs64)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n_act; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = items[a];
        double xn;
        if (E) {
            xn = E[a];
        } else {
            const double step = fmin(fmax(lam * d[a], -1.0), 1.0);
            xn = fmin(1.0, xbase[a] * exp(step));
        }
        x[i] = xn;
        const double wv = A64[i] * xn;
        if (w32) w32[i] = (float)wv;
        if (w64) w64[i] = wv;
        if (xs32) xs32[i] = (float)xn;
        if (xs64) xs64[i] = xn;
    }
}

// density order: value = original index of each active item
__global__ void k_orig_keys(const int32_t* __restrict__ list, const int32_t* __restrict__ perm, int64_t na,
                            uint32_t* keys, int32_t* vals)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = perm[list[a]];
        keys[a] = (uint32_t)o;
        vals[a] = o;
    }
}

// key = bits of float(n_H) inverted, so an ascending sort is high to low density
__global__ void k_density_keys(const int32_t* __restrict__ vals, const double* __restrict__ nH_orig, int64_t na,
                               uint32_t* keys)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x)
        keys[a] = ~__float_as_uint((float)nH_orig[vals[a]]);
}

// block of each density rank a: block b holds ranks [b na / B, (b+1) na / B)
__global__ void k_block_of(const int32_t* __restrict__ vals, const int32_t* __restrict__ inv, int64_t na, int B,
                           uint32_t* block_of_slot)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        int64_t b = (a * B) / na;
        while (b + 1 < B && ((b + 1) * na) / B <= a) ++b;
        while (b > 0 && (b * na) / B > a) --b;
        block_of_slot[inv[vals[a]]] = (uint32_t)b;
    }
}

__global__ void k_block_keys(const int32_t* __restrict__ list, const uint32_t* __restrict__ block_of_slot, int64_t na,
                             uint32_t* keys, int32_t* vals)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        keys[a] = block_of_slot[list[a]];
        vals[a] = list[a];
    }
}

__global__ void k_iota(int32_t* out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

// v_m[s] = v[perm[s]] (original -> Morton order)
__global__ void k_to_morton(const int32_t* __restrict__ perm, const double* __restrict__ v, int64_t n, double* vm)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        vm[s] = v[perm[s]];
}

// out[perm[s]] = (v_m[s] - jv[s]) and E_out[perm[s]] = E[s]
__global__ void k_tangent_out(const int32_t* __restrict__ perm, const double* __restrict__ vm,
                              const double* __restrict__ jv, const double* __restrict__ E, int64_t n,
                              double* dlnE_out, double* E_out)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        dlnE_out[perm[s]] = vm[s] - jv[s];
        if (E_out) E_out[perm[s]] = E[s];
    }
}

// out[b] += *v
__global__ void k_add_scalar(double* out, int F, const double* __restrict__ v)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < F) out[b] += *v;
}

// per-particle state (original order): bit 0 case B latched, bit 1 frozen
__global__ void k_state_out(const int32_t* __restrict__ perm, const uint8_t* __restrict__ active,
                            const uint8_t* __restrict__ latch, int64_t n, int case_rule, uint8_t* state)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const bool caseB = case_rule == URCHIN_CASE_B || (case_rule == URCHIN_CASE_AUTO && latch[s]);
        state[perm[s]] = (uint8_t)((caseB ? 1 : 0) | (active[s] ? 0 : 2));
    }
}

__global__ void k_state_in(const int32_t* __restrict__ perm, const uint8_t* __restrict__ state, int64_t n,
                           uint8_t* active, uint8_t* latch, unsigned* status)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t st = state[perm[s]];
        if (st & ~3u) atomicOr(status, kStInput);
        active[s] = (st & 2) ? 0 : 1;
        latch[s] = st & 1;
    }
}

// b_a = x_bar_i x_i (the cotangent in u = ln x), i = items[a]
__global__ void k_adj_rhs(const int32_t* __restrict__ items, int64_t na, const int32_t* __restrict__ perm,
                          const double* __restrict__ xbar_orig, const double* __restrict__ x, double* b)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = items[a];
        b[a] = xbar_orig[perm[i]] * x[i];
    }
}

// ray coefficients of J_u^T nu: coef[k na + a] = nu_a (E_a / x_a) c_ak, where
// c_ak = d ln E_a / d tau_ak from the sweep kernel
template <typename Real>
__global__ void k_adj_coef(const int32_t* __restrict__ items, int64_t na, int R, const double* __restrict__ nu,
                           const double* __restrict__ E, const double* __restrict__ x, const double* __restrict__ ctan,
                           Real* coef)
{
    const int64_t total = na * (int64_t)R;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < total; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = r % na;
        coef[r] = (Real)(nu[a] * (E[a] / x[items[a]]) * ctan[r]);
    }
}

// out_a = nu_a - x_i z_i: (I - J_u^T) nu from the scattered z = J^T (nu / x)
__global__ void k_adj_apply(const int32_t* __restrict__ items, int64_t na, const double* __restrict__ nu,
                            const double* __restrict__ x, const double* __restrict__ z, double* out)
{
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = items[a];
        out[a] = nu[a] - x[i] * z[i];
    }
}

// frozen particles f: t_f = (x_bar_f + z_f) dx_f/dGamma at Gamma_thin (their
// x = x_thin depends on Gamma_thin = sum_b w_b); 0 for the others; one_s = 1
__global__ void k_adj_frozen(const uint8_t* __restrict__ active, const int32_t* __restrict__ perm,
                             const double* __restrict__ xbar_orig, const double* __restrict__ z,
                             const double* __restrict__ x, const double* __restrict__ nH,
                             const double* __restrict__ aA, const double* __restrict__ aB,
                             const double* __restrict__ gc, int64_t n, double gthin, double y, int case_rule,
                             double* t, double* one)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        one[s] = 1.0;
        if (active[s]) {
            t[s] = 0.0;
            continue;
        }
        const double alpha = case_rule == URCHIN_CASE_B ? aB[s] : aA[s];
        t[s] = (xbar_orig[perm[s]] + z[s]) * dx_dgamma(x[s], nH[s], alpha, gc[s], gthin, y);
    }
}

// Per-ray coefficients of the active particles' w_bar term:
//   w_bar_b += sum_a phi_a (1/R) sum_k exp(-s_b tau_ak) / Gamma_a,
//   phi_a = nu_a (E_a / x_a) elas_a,  elas_a = Gamma_a (dE_a/dGamma_a) / E_a,
// as lc = ln|phi_a / (R Gamma_thin)| - ln(Gamma_a / Gamma_thin), sg = sign
// (Gamma_a recomputed from tau with the sweep's fold: fold_ray, the
// per-ray log rates and their log-sum-exp in double).
template <typename Real>
__global__ void k_adj_wcoef(const int32_t* __restrict__ items, int64_t na, int R, const Real* __restrict__ tau,
                            const double* __restrict__ sv, const double* __restrict__ wv, int F,
                            const double* __restrict__ nu, const double* __restrict__ E, const double* __restrict__ x,
                            const double* __restrict__ nH, const double* __restrict__ aA,
                            const double* __restrict__ aB, const double* __restrict__ gc,
                            const uint8_t* __restrict__ latch, int case_rule, double y, double* lc, double* sg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool kF32 = sizeof(Real) == 4;
    Real* e2 = reinterpret_cast<Real*>(smem_raw);
    Real* wn = e2 + F;
    Real* e2t = kF32 ? wn + F : nullptr;
    __shared__ double sh[2];
    fold_prepare<Real>(sv, wv, F, e2, e2t, wn, nullptr, sh);
    const double gthin = sh[0], smin = sh[1];
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < na; a += (int64_t)gridDim.x * blockDim.x) {
        RayMean<Real> lse;
        for (int k = 0; k < R; ++k) {
            const Real t = tau[a + (int64_t)k * na];
            Real S, S2;
            fold_ray<false>(t, e2, e2t, wn, nullptr, F, S, S2);
            lse.add(ray_lnrate(smin, t, S));
        }
        const double lnr = lse.mean(R);                    // ln(Gamma_a / Gamma_thin)
        const int32_t i = items[a];
        const double G = gthin * exp(lnr);
        const bool caseB = case_rule == URCHIN_CASE_B || (case_rule == URCHIN_CASE_AUTO && latch[i]);
        const double alpha = caseB ? aB[i] : aA[i];
        const double elas = G > 0.0 ? G * dx_dgamma(E[a], nH[i], alpha, gc[i], G, y) / E[a] : 0.0;
        const double phi = nu[a] * (E[a] / x[i]) * elas;
        const double l0 = phi != 0.0 ? log(fabs(phi) / ((double)R * gthin)) - lnr : -INFINITY;
        const double sgn = phi < 0.0 ? -1.0 : 1.0;
        for (int k = 0; k < R; ++k) {
            lc[a + (int64_t)k * na] = l0;
            sg[a + (int64_t)k * na] = sgn;
        }
    }
}

}  // namespace

int launch_sweep(const SweepArgs& A, cudaStream_t s)
{
    if (A.n_items <= 0) return URCHIN_OK;
    const size_t rsz = A.precision == URCHIN_F64 ? sizeof(double) : sizeof(float);
    // plain sweeps without tangent: one thread per particle (0.152 ms against
    // 0.184 ms per sweep of the 262144-particle halo for the ray-parallel layout)
    if (!A.he && !A.near_far && !A.want_tangent) {
        // e2 and wn (FP64), or the packed {e2, e2t, wn, 0} (FP32)
        const size_t sm = (A.precision == URCHIN_F64 ? 2 : 4) * (size_t)A.F * rsz;
        const void* fp = A.precision == URCHIN_F64 ? (const void*)k_sweep_pp<double> : (const void*)k_sweep_pp<float>;
        if (sm > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(fp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int g = 0;
        URCHIN_TRY(grid_for(fp, kSweepThreads, sm, &g));
        const int64_t need = (A.n_items + kSweepThreads - 1) / kSweepThreads;
        if (need < g) g = (int)std::max<int64_t>(need, 1);
        void* args[] = {const_cast<SweepArgs*>(&A)};
        URCHIN_TRY_CUDA(cudaLaunchKernel(fp, dim3(g), dim3(kSweepThreads), args, sm, s));
        return launched();
    }
    const bool f64 = A.precision == URCHIN_F64;
    // two per-ray log-rate arrays in double, then e2, wn, s, (FP32) e2t, (helium) s1, s2 and
    // their three FP32 tails
    const size_t smem =
        2 * sizeof(double) * kSweepThreads + ((f64 ? 3 : 4) + (A.he ? (f64 ? 2 : 5) : 0)) * (size_t)A.F * rsz;
    const int var = A.he ? kSweepHelium : (A.near_far ? kSweepNearFar : kSweepPlain);
    const void* fns[2][3] = {
        {(const void*)k_sweep<float, kSweepPlain>, (const void*)k_sweep<float, kSweepNearFar>,
         (const void*)k_sweep<float, kSweepHelium>},
        {(const void*)k_sweep<double, kSweepPlain>, (const void*)k_sweep<double, kSweepNearFar>,
         (const void*)k_sweep<double, kSweepHelium>}};
    const void* fn = fns[f64 ? 1 : 0][var];
    if (smem > 48 * 1024)
        URCHIN_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int rows_per_block = kSweepThreads / A.R;
    int64_t need = (A.n_items + rows_per_block - 1) / rows_per_block;
    int grid = 0;
    URCHIN_TRY(grid_for(fn, kSweepThreads, smem, &grid));
    if (need < grid) grid = (int)std::max<int64_t>(need, 1);
    void* args[] = {const_cast<SweepArgs*>(&A)};
    URCHIN_TRY_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kSweepThreads), args, smem, s));
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

int Solver::init(const urchin_bvh* bvh_, const urchin_solve_params* P_, double* x_inout, cudaStream_t s_)
{
    bvh = bvh_;
    P = *P_;
    s = s_;
    n = bvh->n;
    f64 = P.precision == URCHIN_F64;
    const size_t rsz = f64 ? sizeof(double) : sizeof(float);
    const bool may_store = P.segments != URCHIN_SEG_RECOMPUTE;
    const int64_t rays = (int64_t)P.R * n;
    Layout lay;
    size_t o_misc = lay.take(128);
    size_t o_dirs = lay.take(sizeof(double) * 3 * (size_t)P.R);
    size_t o_x = lay.take(sizeof(double) * (size_t)n);
    size_t o_nH = lay.take(sizeof(double) * (size_t)n);
    size_t o_aA = lay.take(sizeof(double) * (size_t)n);
    size_t o_aB = lay.take(sizeof(double) * (size_t)n);
    size_t o_gc = lay.take(sizeof(double) * (size_t)n);
    size_t o_w = lay.take(rsz * (size_t)n);
    size_t o_xs = lay.take(may_store ? rsz * (size_t)n : 0);
    size_t o_act = lay.take((size_t)n);
    size_t o_latch = lay.take((size_t)n);
    size_t o_list = lay.take(sizeof(int32_t) * (size_t)n);
    size_t o_tau = lay.take(rsz * (size_t)rays);
    size_t o_tn = lay.take(P.near_far ? rsz * (size_t)rays : 0);
    size_t o_pt = lay.take(P.near_far == URCHIN_SLAB_SPECTRUM ? spec_table_bytes() : 0);
    const bool he = spectrum_has_he(&P.spectrum);
    size_t o_h1 = lay.take(he ? rsz * (size_t)rays : 0);
    size_t o_h2 = lay.take(he ? rsz * (size_t)rays : 0);
    size_t o_comp = lay.take(compact_tmp_bytes(n));
    size_t o_cnt = lay.take(may_store ? sizeof(uint32_t) * (size_t)rays : 0);
    size_t o_rp = lay.take(may_store ? sizeof(uint64_t) * (size_t)(rays + 1) : 0);
    size_t o_st = lay.take(may_store ? scan64_tmp_bytes(rays) : 0);
    URCHIN_TRY(scr.alloc(lay.bytes, s));
    misc = scr.at<unsigned long long>(o_misc);   // [0] maxrel, [1] counter+status, [2] count, [3..5] profile
    dirs = scr.at<double>(o_dirs);
    x = scr.at<double>(o_x);
    nH = scr.at<double>(o_nH);
    aA = scr.at<double>(o_aA);
    aB = scr.at<double>(o_aB);
    gc = scr.at<double>(o_gc);
    w32 = f64 ? nullptr : scr.at<float>(o_w);
    w64 = f64 ? scr.at<double>(o_w) : nullptr;
    if (may_store) {
        xs32 = f64 ? nullptr : scr.at<float>(o_xs);
        xs64 = f64 ? scr.at<double>(o_xs) : nullptr;
        counts = scr.at<uint32_t>(o_cnt);
        row_ptr = scr.at<uint64_t>(o_rp);
        scan_tmp = scr.at<void>(o_st);
    }
    active = scr.at<uint8_t>(o_act);
    latch = scr.at<uint8_t>(o_latch);
    list = scr.at<int32_t>(o_list);
    tau = scr.at<void>(o_tau);
    tau_near = P.near_far ? scr.at<void>(o_tn) : nullptr;
    tau_he1 = he ? scr.at<void>(o_h1) : nullptr;
    tau_he2 = he ? scr.at<void>(o_h2) : nullptr;
    if (P.near_far == URCHIN_SLAB_SPECTRUM)
        URCHIN_TRY(build_spec_table(P.spectrum.s, P.spectrum.w, P.spectrum.F, scr.at<void>(o_pt), &poly, s));
    comp_tmp = scr.at<void>(o_comp);
    counter = reinterpret_cast<unsigned*>(misc + 1);
    status = counter + 1;
    hits = P.profile ? misc + 3 : nullptr;
    URCHIN_TRY_CUDA(cudaMemsetAsync(misc, 0, 128, s));
    URCHIN_TRY_CUDA(cudaMemsetAsync(latch, 0, (size_t)n, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(dirs, P.dirs, sizeof(double) * 3 * (size_t)P.R, cudaMemcpyHostToDevice, s));
    std::vector<double> wh((size_t)P.spectrum.F);
    URCHIN_TRY_CUDA(cudaMemcpyAsync(wh.data(), P.spectrum.w, sizeof(double) * wh.size(), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    gthin = 0.0;
    for (double v : wh) gthin += v;
    if (!(gthin > 0.0) || !std::isfinite(gthin))
        return set_error(URCHIN_ERR_ARG, "urchin_solve: spectrum weights must sum to a finite Gamma_thin > 0");
    unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_setup<<<grid, 256, 0, s>>>(*bvh, P.nH, P.T, x_inout, P.warm_start, gthin, P.case_rule, P.y, nH, aA, aB, gc,
                                 x, w32, w64, xs32, xs64, status);
    URCHIN_TRY(launched());
    unsigned st = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    if (st & kStInput) return set_error(URCHIN_ERR_ARG, "urchin_solve: n_H and T must be finite and > 0");
    if (st & kStWarm) return set_error(URCHIN_ERR_ARG, "urchin_solve: warm-start x must lie in (0, 1]");
    return URCHIN_OK;
}

// Profile mode: a start/stop event pair recorded on the launching stream
// around each timed launch, resolved in finish().
int Solver::begin_timed(int kind, cudaEvent_t* stop)
{
    *stop = nullptr;
    if (!P.profile) return URCHIN_OK;
    cudaEvent_t a, b;
    URCHIN_TRY_CUDA(cudaEventCreate(&a));
    URCHIN_TRY_CUDA(cudaEventCreate(&b));
    events.push_back(a);
    events.push_back(b);
    event_kind.push_back(kind);
    URCHIN_TRY_CUDA(cudaEventRecord(a, s));
    *stop = b;
    return URCHIN_OK;
}

int Solver::end_timed(cudaEvent_t stop)
{
    if (stop) URCHIN_TRY_CUDA(cudaEventRecord(stop, s));
    return URCHIN_OK;
}

int Solver::timed_sweep(const SweepArgs& A, cudaStream_t st)
{
    cudaEvent_t stop;
    URCHIN_TRY(begin_timed(2, &stop));
    URCHIN_TRY(launch_sweep(A, st));
    URCHIN_TRY(end_timed(stop));
    stats.sweep_launches += 1;
    return URCHIN_OK;
}

// Algorithmic bytes of one stored-segment launch over `items` (profile mode):
// every segment of the evaluated rays read once (index and value), each
// column written once, the x vector gathered once.
int Solver::count_spmv(const int32_t* items, int64_t n_items)
{
    stats.spmv_launches += 1;
    if (!P.profile) return URCHIN_OK;
    const size_t vsz = f64 ? sizeof(double) : sizeof(float);
    int64_t seg = 0;
    if (items == list && n_items == n_act && active_nnz >= 0) {
        seg = active_nnz;
    } else {
        unsigned long long* acc = misc + 9;
        URCHIN_TRY_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s));
        URCHIN_TRY(launch_row_nnz(row_ptr, items, n_items, n, P.R, acc, s));
        unsigned long long h = 0;
        URCHIN_TRY_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
        URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
        seg = (int64_t)h;
        if (items == list && n_items == n_act) active_nnz = seg;
    }
    const int64_t isz = (seg_col || chunked) ? (int64_t)sizeof(int32_t) : (int64_t)(sizeof(uint16_t) + sizeof(uint8_t));
    stats.spmv_bytes += seg * (isz + (int64_t)vsz) + n_items * P.R * (int64_t)vsz + n * (int64_t)vsz;
    return URCHIN_OK;
}

int Solver::timed_trace(TraceJob& job)
{
    job.counter = counter;
    job.status = status;
    job.hits = hits;
    cudaEvent_t stop;
    URCHIN_TRY(begin_timed(0, &stop));
    URCHIN_TRY(launch_trace(job, s));
    URCHIN_TRY(end_timed(stop));
    stats.trace_launches += 1;
    return URCHIN_OK;
}

int Solver::order_for(const int32_t* items, int64_t n_items, const int32_t** out)
{
    *out = nullptr;
    if (n_items <= 0) return URCHIN_OK;
    for (const OrderEntry& e : orders)
        if (e.items == items && e.n == n_items) {
            *out = e.order;
            return URCHIN_OK;
        }
    if (!ord_base) {
        ord_cap = 2 * (int64_t)P.R * n;
        Layout lay;
        const size_t o_o = lay.take(sizeof(int32_t) * (size_t)ord_cap);
        const size_t o_t = lay.take(ray_order_tmp_bytes(n));
        URCHIN_TRY(ord.alloc(lay.bytes, s));
        ord_base = ord.at<int32_t>(o_o);
        ord_tmp = ord.at<void>(o_t);
    }
    const int64_t need = (int64_t)P.R * n_items;
    if (n_items > n || n_items < kRayOrderMinItems) return URCHIN_OK;   // item order
    if (ord_used + need > ord_cap) items_changed();
    int32_t* o = ord_base + ord_used;
    URCHIN_TRY(ray_order(bvh, items, n_items, P.dirs, P.R, P.l_ray, o, ord_tmp, s));
    ord_used += need;
    orders.push_back(OrderEntry{items, n_items, o});
    *out = o;
    return URCHIN_OK;
}

// The ray order of the active list, derived from sweep 0's order of all
// particles instead of sorted afresh: ray_order sorts stably by a key of the
// origin alone, and the list holds the active particles in ascending Morton
// slot, so the full order restricted to the list is exactly the order a sort
// of the list would give (2 R radix passes over the list saved per solve).
int Solver::derive_list_order(const int32_t* full)
{
    const int64_t na = n_act;
    const int64_t rn = (int64_t)P.R * n;
    if (full != ord_base || na < kRayOrderMinItems || na > n || rn + (int64_t)P.R * na > ord_cap) return URCHIN_OK;
    int32_t* pos = static_cast<int32_t*>(ord_tmp);
    uint8_t* flags = reinterpret_cast<uint8_t*>(static_cast<char*>(ord_tmp) + (((size_t)n * 4 + 255) & ~size_t(255)));
    int32_t* out = ord_base + rn;
    uint32_t* cnt = reinterpret_cast<uint32_t*>(misc + 2);
    const unsigned ga = (unsigned)std::max<int64_t>(1, std::min<int64_t>((na + 255) / 256, 4096));
    const unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
    k_list_pos<<<ga, 256, 0, s>>>(list, na, n, pos);
    URCHIN_TRY(launched());
    for (int k = 0; k < P.R; ++k) {
        k_order_flags<<<gn, 256, 0, s>>>(full + (int64_t)k * n, active, n, flags);
        URCHIN_TRY(launched());
        URCHIN_TRY(compact_indices(flags, n, out + (int64_t)k * na, cnt, comp_tmp, s));
        k_order_map<<<ga, 256, 0, s>>>(full + (int64_t)k * n, pos, na, out + (int64_t)k * na);
        URCHIN_TRY(launched());
    }
    orders.push_back(OrderEntry{nullptr, n, ord_base});
    orders.push_back(OrderEntry{list, na, out});
    ord_used = rn + (int64_t)P.R * na;
    return URCHIN_OK;
}

int Solver::trace(const int32_t* items, int64_t n_items, const float* tw32, const double* tw64)
{
    TraceJob job{};
    job.bvh = bvh;
    job.w32 = tw32;
    job.w64 = tw64;
    job.dirs_dev = dirs;
    job.R = P.R;
    job.l_ray = P.l_ray;
    job.items = items;
    job.n_items = n_items;
    job.row_stride = 1;
    job.k_stride = n_items;
    job.out_row = nullptr;
    job.out = tau;
    job.kernel = P.kernel;
    job.precision = P.precision;
    job.mode = 0;
    job.near_far = P.near_far;
    job.out_near = tau_near;
    job.near_k_stride = n;
    URCHIN_TRY(order_for(items, n_items, &job.order));
    URCHIN_TRY(timed_trace(job));
    stats.traversals += 1;
    stats.rays += n_items * P.R;
    return URCHIN_OK;
}

// rows of the stored segments (direction-major, Morton slot) of particles
// that are not active are emptied before the lists are built
__global__ void k_clear_inactive_rows(const uint8_t* __restrict__ active, int64_t n, int R, uint32_t* counts)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * R; i += (int64_t)gridDim.x * blockDim.x)
        if (!active[i % n]) counts[i] = 0u;
}

// Columns of the current x for the rays of `items` into tau (k-major), from
// the stored segments once they exist.  The segment lists (SEG_STORE, or
// SEG_AUTO where they fit in memory) come from per-ray hit counts and one
// filling traversal, which also gives that sweep's columns:
//   * SEG_STORE (and SEG_AUTO with density blocks, or `build`): a counting
//     and a filling traversal at once;
//   * SEG_AUTO otherwise: sweep 0 traces recomputed columns and counts every
//     ray's hits on the way, sweep 1 recomputes too, and the lists are built
//     in sweep 2, for the particles still active: a solve that converges in
//     two sweeps (an optically thin box) never writes them, one that goes on
//     pays one traversal more than storing at once (262144-particle halo:
//     292 sweeps, 0.86 s; one traversal 0.04 s).
constexpr int kAutoStoreSweep = 2;

// The stored lists for a product: rows (row_ptr) or linked chunks.
void Solver::spmv_lists(SpmvArgs& A) const
{
    A.row_ptr = row_ptr;
    A.col = seg_col;
    A.lo = seg_lo;
    A.hi = seg_hi;
    A.val = seg_val;
    if (chunked) {
        A.chunk_head = chunk_head;
        A.chunk_next = chunk_next;
        A.row_cnt = counts;
        A.chunk_seg = chunk_seg;
    }
}

// The hit-count sample of trace_chunked: the first 32 Morton slots of every
// block of 32 * stride (a packet of neighbouring origins, traced as coherently
// as in the full traversal), up to n.
__global__ void k_sample_origins(int32_t* out, int64_t m, int64_t stride)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = (int32_t)((t / 32) * 32 * stride + (t % 32));
}

// The first sweep's traversal of every particle, storing each ray's segments
// in chunks as it goes (MODE_CHUNK).  The number of segments is not known in
// advance: it is estimated from the hit counts of a sample of 1/64 of the
// origins (32 neighbouring slots in every 2048), with room for 15 % more, for half a chunk per ray and for the
// warps' unused blocks.  When the lists do not fit, or the estimate proves
// short (some rays' lists are then incomplete), the lists are dropped and the
// solve goes on as without them: the columns and counts of this traversal are
// complete either way.
int Solver::trace_chunked(TraceJob& job)
{
    const int64_t rays = (int64_t)P.R * n;
    const int64_t stride = 64, block = 32 * stride, nb = (n + block - 1) / block;
    const int64_t m = (nb - 1) * 32 + std::min<int64_t>(32, n - (nb - 1) * block);
    const double entry_bytes = 8.0;               // particle index + value
    uint64_t* total = reinterpret_cast<uint64_t*>(misc + 6);
    unsigned long long cap = 0;
    {
        Scratch smp;
        URCHIN_TRY(smp.alloc(sizeof(int32_t) * (size_t)m, s));
        int32_t* org = smp.at<int32_t>(0);
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 4096));
        k_sample_origins<<<g, 256, 0, s>>>(org, m, stride);
        URCHIN_TRY(launched());
        TraceJob cj = job;
        cj.items = org;
        cj.n_items = m;
        cj.k_stride = m;
        cj.mode = 1;
        cj.order = nullptr;
        cj.counter = counter;
        cj.status = status;
        cj.hits = nullptr;
        URCHIN_TRY(launch_trace(cj, s));
        URCHIN_TRY(scan_counts_u64(counts, row_ptr, rays, scan_tmp, total, s));
        uint64_t sample = 0;
        URCHIN_TRY_CUDA(cudaMemcpyAsync(&sample, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
        URCHIN_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)rays, s));
        const double est = (double)sample * (double)n / (double)m;
        int dev = 0, sms = 0;
        URCHIN_TRY_CUDA(cudaGetDevice(&dev));
        URCHIN_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const double chunks = (1.15 * est + 0.5 * kChunkEntries * (double)rays) / kChunkEntries +
                              (double)sms * 64.0 * 64.0 + 4096.0;
        size_t free_b = 0, total_b = 0;
        URCHIN_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
        const double per_chunk = entry_bytes * kChunkEntries + 4.0;
        const double avail = 0.85 * (double)(free_b + pool_idle_bytes()) - 4.0 * (double)rays;
        if (chunks * per_chunk <= avail && chunks < 4.0e9) cap = (unsigned long long)chunks;
    }
    if (cap > 0) {
        const size_t entries = (size_t)cap * kChunkEntries;
        Layout lay;
        const size_t o_ctr = lay.take(sizeof(unsigned long long));
        const size_t o_head = lay.take(sizeof(uint32_t) * (size_t)rays);
        const size_t o_next = lay.take(sizeof(uint32_t) * (size_t)cap);
        const size_t o_seg = lay.take(sizeof(int2) * entries);
        if (chunk_mem.alloc(lay.bytes, s) != URCHIN_OK) {
            clear_error();
            cap = 0;
        } else {
            unsigned long long* ctr = chunk_mem.at<unsigned long long>(o_ctr);
            URCHIN_TRY_CUDA(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s));
            chunk_head = chunk_mem.at<uint32_t>(o_head);
            chunk_next = chunk_mem.at<uint32_t>(o_next);
            job.mode = 4;
            job.chunk_head = chunk_head;
            job.chunk_next = chunk_next;
            job.chunk_counter = ctr;
            job.chunk_cap = cap;
            job.chunk_seg = chunk_mem.at<int2>(o_seg);
            URCHIN_TRY(timed_trace(job));
            unsigned long long used = 0;
            URCHIN_TRY_CUDA(cudaMemcpyAsync(&used, ctr, sizeof(used), cudaMemcpyDeviceToHost, s));
            URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
            if (used <= cap) {
                chunk_seg = job.chunk_seg;
                chunked = true;
                stored = true;
                stats.segments_stored = 1;
                URCHIN_TRY(scan_counts_u64(counts, row_ptr, rays, scan_tmp, total, s));
                URCHIN_TRY_CUDA(cudaMemcpyAsync(row_ptr + rays, total, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
                uint64_t nnz = 0;
                URCHIN_TRY_CUDA(cudaMemcpyAsync(&nnz, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
                URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
                stats.nnz = (int64_t)nnz;
                return URCHIN_OK;
            }
            // the estimate was short: the lists are incomplete, the columns are not
            chunk_mem.release();
            chunk_head = chunk_next = nullptr;
            return URCHIN_OK;
        }
    }
    job.mode = 0;
    return timed_trace(job);
}

// From the fourth sweep on, the chunked lists of the active rows are copied
// into rows (the 7-byte layout of the row product, which streams at the
// bandwidth bound where following chunk links does not) when both fit at
// once; the chunks are then released.  A solve of two or three sweeps keeps
// the chunks.
constexpr int kCompactSweep = 3;

int Solver::compact_chunks()
{
    const int64_t rays = (int64_t)P.R * n;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rays + 255) / 256, 4096));
    k_clear_inactive_rows<<<g, 256, 0, s>>>(active, n, P.R, counts);
    URCHIN_TRY(launched());
    uint64_t* total = reinterpret_cast<uint64_t*>(misc + 6);
    URCHIN_TRY(scan_counts_u64(counts, row_ptr, rays, scan_tmp, total, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(row_ptr + rays, total, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    uint64_t nnz = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&nnz, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    const bool split = n <= (int64_t(1) << 24);
    Layout lay;
    const size_t o_col = split ? 0 : lay.take(sizeof(int32_t) * (size_t)nnz);
    const size_t o_lo = split ? lay.take(sizeof(uint16_t) * (size_t)nnz) : 0;
    const size_t o_hi = split ? lay.take(sizeof(uint8_t) * (size_t)nnz) : 0;
    const size_t o_val = lay.take(sizeof(float) * (size_t)nnz);
    size_t free_b = 0, total_b = 0;
    URCHIN_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if ((double)lay.bytes > 0.85 * (double)(free_b + pool_idle_bytes()) || seg.alloc(lay.bytes, s) != URCHIN_OK) {
        clear_error();
        return URCHIN_OK;                          // keep the chunks
    }
    ChunkCompactArgs C{};
    C.head = chunk_head;
    C.next = chunk_next;
    C.seg = chunk_seg;
    C.cnt = counts;
    C.row_ptr = row_ptr;
    C.rows = rays;
    C.col = split ? nullptr : seg.at<int32_t>(o_col);
    C.lo = split ? seg.at<uint16_t>(o_lo) : nullptr;
    C.hi = split ? seg.at<uint8_t>(o_hi) : nullptr;
    C.val = seg.at<float>(o_val);
    URCHIN_TRY(launch_chunk_compact(C, s));
    seg_col = C.col;
    seg_lo = C.lo;
    seg_hi = C.hi;
    seg_val = C.val;
    chunked = false;
    chunk_mem.release();
    chunk_head = chunk_next = nullptr;
    chunk_seg = nullptr;
    stats.nnz = (int64_t)nnz;
    active_nnz = -1;
    return URCHIN_OK;
}

int Solver::columns(const int32_t* items, int64_t n_items, int sweep0, bool build)
{
    if (!sweep0 && chunked && !compact_tried && stats.iterations >= kCompactSweep) {
        compact_tried = true;
        URCHIN_TRY(compact_chunks());
    }
    if (!sweep0 && stored) {
        SpmvArgs A{};
        spmv_lists(A);
        A.xvec = f64 ? (const void*)xs64 : (const void*)xs32;
        A.items = items;
        A.n_items = n_items;
        A.n_rows_per_k = n;
        A.R = P.R;
        A.precision = P.precision;
        A.out = tau;
        cudaEvent_t stop;
        URCHIN_TRY(begin_timed(1, &stop));
        URCHIN_TRY(launch_spmv(A, s));
        URCHIN_TRY(end_timed(stop));
        URCHIN_TRY(count_spmv(items, n_items));
        stats.traversals += 1;
        stats.rays += n_items * P.R;
        return URCHIN_OK;
    }
    if (P.segments == URCHIN_SEG_RECOMPUTE || store_declined || (stored && sweep0))
        return trace(items, n_items, w32, w64);
    TraceJob job{};
    job.bvh = bvh;
    job.w32 = w32;
    job.w64 = w64;
    job.dirs_dev = dirs;
    job.R = P.R;
    job.l_ray = P.l_ray;
    job.items = items;
    job.n_items = n_items;
    job.row_stride = 1;
    job.k_stride = n_items;
    job.out = tau;
    job.kernel = P.kernel;
    job.precision = P.precision;
    job.counts = counts;
    job.near_far = P.near_far;
    job.out_near = tau_near;
    job.near_k_stride = n;
    URCHIN_TRY(order_for(items, n_items, &job.order));
    const int64_t rays = (int64_t)P.R * n;
    const bool deferred = P.segments == URCHIN_SEG_AUTO && !build && P.blocks <= 1;
    if (deferred && !counts_ready) {
        // recomputed columns, every ray's hits counted on the way; for a
        // first sweep over every particle the segment lists are kept too
        // (in chunks) where they fit, so that the next sweeps need no traversal
        URCHIN_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)rays, s));
        if (!f64 && !P.near_far && items == nullptr && n_items == n) {
            URCHIN_TRY(trace_chunked(job));
        } else {
            job.mode = 0;
            URCHIN_TRY(timed_trace(job));
        }
        counts_ready = true;
        counted_all = items == nullptr && n_items == n;
        stats.traversals += 1;
        stats.rays += n_items * P.R;
        return URCHIN_OK;
    }
    if (deferred && stats.iterations < kAutoStoreSweep) return trace(items, n_items, w32, w64);
    if (!counts_ready || (!counted_all && items == nullptr)) {
        URCHIN_TRY_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (size_t)rays, s));
        job.mode = 1;
        URCHIN_TRY(timed_trace(job));
        stats.traversals += 1;
    } else if (items != nullptr) {
        // counts from a traversal of every particle: keep the active rows only
        const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rays + 255) / 256, 4096));
        k_clear_inactive_rows<<<g, 256, 0, s>>>(active, n, P.R, counts);
        URCHIN_TRY(launched());
    }
    counts_ready = true;
    uint64_t* total = reinterpret_cast<uint64_t*>(misc + 6);
    URCHIN_TRY(scan_counts_u64(counts, row_ptr, rays, scan_tmp, total, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(row_ptr + rays, total, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    uint64_t nnz = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&nnz, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    const size_t vsz = f64 ? sizeof(double) : sizeof(float);
    // FP32 segments keep the particle index as 16 + 8 bits (7 bytes per segment)
    const bool split = !f64 && n <= (int64_t(1) << 24);
    const size_t isz = split ? sizeof(uint16_t) + sizeof(uint8_t) : sizeof(int32_t);
    const size_t need = (size_t)nnz * (isz + vsz) + 1024;
    bool fits = true;
    if (P.segments == URCHIN_SEG_AUTO) {
        size_t free_b = 0, total_b = 0;
        URCHIN_TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
        // memory the library's pool keeps reserved from earlier calls is available too
        fits = need < (size_t)(0.85 * (double)(free_b + pool_idle_bytes()));
    }
    if (fits) {
        Layout lay;
        size_t o_col = split ? 0 : lay.take(sizeof(int32_t) * (size_t)nnz);
        size_t o_lo = split ? lay.take(sizeof(uint16_t) * (size_t)nnz) : 0;
        size_t o_hi = split ? lay.take(sizeof(uint8_t) * (size_t)nnz) : 0;
        size_t o_val = lay.take(vsz * (size_t)nnz);
        int st = seg.alloc(lay.bytes, s);
        if (st != URCHIN_OK) {
            if (P.segments == URCHIN_SEG_STORE) return st;
            fits = false;
            clear_error();
        } else {
            seg_col = split ? nullptr : seg.at<int32_t>(o_col);
            seg_lo = split ? seg.at<uint16_t>(o_lo) : nullptr;
            seg_hi = split ? seg.at<uint8_t>(o_hi) : nullptr;
            seg_val = seg.at<void>(o_val);
        }
    }
    if (!fits) {
        store_declined = true;
        return trace(items, n_items, w32, w64);
    }
    stored = true;
    stats.segments_stored = 1;
    stats.nnz = (int64_t)nnz;
    job.counts = nullptr;
    job.mode = 2;
    job.row_ptr = row_ptr;
    job.seg_col = seg_col;
    job.seg_lo = seg_lo;
    job.seg_hi = seg_hi;
    job.seg_val = seg_val;
    URCHIN_TRY(timed_trace(job));
    stats.traversals += 1;
    stats.rays += n_items * P.R;
    return URCHIN_OK;
}

// Columns of the tangent vector (z = x v on the active particles) into tau.
int Solver::linear_columns(const int32_t* items, int64_t n_items, const float* z32, const double* z64,
                           float* wz32, double* wz64)
{
    stats.rays += n_items * P.R;
    stats.traversals += 1;
    if (stored) {
        SpmvArgs A{};
        spmv_lists(A);
        A.xvec = f64 ? (const void*)z64 : (const void*)z32;
        A.items = items;
        A.n_items = n_items;
        A.n_rows_per_k = n;
        A.R = P.R;
        A.precision = P.precision;
        A.out = tau;
        cudaEvent_t stop;
        URCHIN_TRY(begin_timed(1, &stop));
        URCHIN_TRY(launch_spmv(A, s));
        URCHIN_TRY(end_timed(stop));
        return count_spmv(items, n_items);
    }
    TraceJob job{};
    job.bvh = bvh;
    job.w32 = wz32;
    job.w64 = wz64;
    job.dirs_dev = dirs;
    job.R = P.R;
    job.l_ray = P.l_ray;
    job.items = items;
    job.n_items = n_items;
    job.row_stride = 1;
    job.k_stride = n_items;
    job.out = tau;
    job.kernel = P.kernel;
    job.precision = P.precision;
    job.mode = 0;
    URCHIN_TRY(order_for(items, n_items, &job.order));
    return timed_trace(job);
}

SweepArgs Solver::sweep_args(const int32_t* items, int64_t n_items, int sweep0)
{
    SweepArgs A{};
    A.tau = tau;
    A.precision = P.precision;
    A.k_stride = n_items;
    A.items = items;
    A.n_items = n_items;
    A.R = P.R;
    A.s = P.spectrum.s;
    A.w = P.spectrum.w;
    A.F = P.spectrum.F;
    A.x = x;
    A.A64 = bvh->A64;
    A.w32 = w32;
    A.w64 = w64;
    A.xs32 = xs32;
    A.xs64 = xs64;
    A.nH = nH;
    A.aA = aA;
    A.aB = aB;
    A.gc = gc;
    A.y = P.y;
    A.case_rule = P.case_rule;
    A.tau_skip = P.tau_skip;
    A.sweep0 = sweep0;
    A.active = active;
    A.latch = latch;
    A.maxrel = misc;
    A.n_above = misc + 7;
    A.n_switch = misc + 8;
    A.tol = P.tol;
    A.status = status;
    A.near_far = P.near_far;
    A.tau_near = tau_near;
    A.near_k_stride = n;
    A.poly = poly;
    A.he = tau_he1 ? 1 : 0;
    A.tau_he1 = tau_he1;
    A.tau_he2 = tau_he2;
    A.s_he1 = P.spectrum.s_he1;
    A.s_he2 = P.spectrum.s_he2;
    return A;
}

int Solver::read_scalars(double* maxrel, unsigned* st)
{
    unsigned long long h[8];
    URCHIN_TRY_CUDA(cudaMemcpyAsync(h, misc, sizeof(h), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    double m;
    memcpy(&m, &h[0], sizeof(double));
    *maxrel = m;
    *st = (unsigned)(h[1] >> 32);
    last_above = (int64_t)h[7];
    if (*st & kStNonfinite) return set_error(URCHIN_ERR_NONFINITE, "urchin_solve: non-finite neutral fraction");
    if (*st & (kStStack | kStVisit)) return set_error(URCHIN_ERR_CUDA, "urchin_solve: traversal stack/visit limit hit");
    if (*st & kStSegment) return set_error(URCHIN_ERR_CUDA, "urchin_solve: segment fill disagrees with its count");
    return URCHIN_OK;
}

void Solver::record(double maxrel)
{
    const int i = stats.iterations - 1;
    if (i < 0 || i >= P.max_iter) return;
    if (P.history_maxrel) P.history_maxrel[i] = maxrel;
    if (P.history_unconverged) P.history_unconverged[i] = last_above;
}

int Solver::first_sweep()
{
    // sweep 0: every particle traced; tau_eff < tau_skip freezes it
    URCHIN_TRY_CUDA(cudaMemsetAsync(misc, 0, sizeof(unsigned long long), s));
        URCHIN_TRY_CUDA(cudaMemsetAsync(misc + 7, 0, sizeof(unsigned long long), s));
    URCHIN_TRY(columns(nullptr, n, 1));
    URCHIN_TRY(timed_sweep(sweep_args(nullptr, n, 1), s));
    uint32_t* cnt = reinterpret_cast<uint32_t*>(misc + 2);
    URCHIN_TRY(compact_indices(active, n, list, cnt, comp_tmp, s));
    const int32_t* full = nullptr;                // sweep 0's ray order of all particles
    for (const OrderEntry& e : orders)
        if (e.items == nullptr && e.n == n) full = e.order;
    items_changed();
    uint32_t hc = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    double m;
    unsigned st;
    URCHIN_TRY(read_scalars(&m, &st));
    n_act = hc;
    if (full) URCHIN_TRY(derive_list_order(full));
    stats.n_active = n_act;
    stats.particle_updates += n_act;
    stats.iterations = 1;
    stats.max_rel_dx = m;
    record(m);
    return URCHIN_OK;
}

// Regroup the active list (Morton order) into the blocks of the high-to-low
// density order; inside a block the items stay in Morton order (a block's
// updates are simultaneous, so their order does not matter, and Morton
// order keeps the block's rays coherent).
int Solver::order_by_density()
{
    const int64_t na = n_act;
    const int B = (int)std::min<int64_t>(P.blocks, std::max<int64_t>(na, 1));
    block_lo.assign(1, 0);
    if (B <= 1 || na == 0) {
        block_lo.push_back(na);
        return URCHIN_OK;
    }
    Layout lay;
    size_t o_k = lay.take(sizeof(uint32_t) * (size_t)na);
    size_t o_v = lay.take(sizeof(int32_t) * (size_t)na);
    size_t o_b = lay.take(sizeof(uint32_t) * (size_t)n);
    size_t o_t = lay.take(radix_tmp_bytes(na));
    Scratch tmp;
    URCHIN_TRY(tmp.alloc(lay.bytes, s));
    uint32_t* keys = tmp.at<uint32_t>(o_k);
    int32_t* vals = tmp.at<int32_t>(o_v);
    uint32_t* blk = tmp.at<uint32_t>(o_b);
    void* rt = tmp.at<void>(o_t);
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((na + 255) / 256, 4096));
    k_orig_keys<<<g, 256, 0, s>>>(list, bvh->perm, na, keys, vals);
    URCHIN_TRY(launched());
    URCHIN_TRY(radix_sort_pairs(keys, vals, na, 30, rt, s));          // by particle index
    k_density_keys<<<g, 256, 0, s>>>(vals, P.nH, na, keys);
    URCHIN_TRY(launched());
    URCHIN_TRY(radix_sort_pairs(keys, vals, na, 32, rt, s));          // stable: high to low density
    k_block_of<<<g, 256, 0, s>>>(vals, bvh->inv, na, B, blk);
    URCHIN_TRY(launched());
    k_block_keys<<<g, 256, 0, s>>>(list, blk, na, keys, vals);
    URCHIN_TRY(launched());
    int bits = 1;
    while ((1 << bits) < B) ++bits;
    URCHIN_TRY(radix_sort_pairs(keys, vals, na, bits, rt, s));        // stable: Morton order inside blocks
    URCHIN_TRY_CUDA(cudaMemcpyAsync(list, vals, sizeof(int32_t) * (size_t)na, cudaMemcpyDeviceToDevice, s));
    items_changed();
    tmp.release();
    for (int b = 1; b <= B; ++b) block_lo.push_back(((int64_t)b * na) / B);
    return URCHIN_OK;
}

// The fixed helium columns of every ray (all particles, [i + k n]): one
// traversal per species with tracer weights A_j he_j (the columns are linear
// in the weights; the helium fractions do not change during the solve).
int Solver::he_columns()
{
    if (!tau_he1) return URCHIN_OK;
    const size_t rsz = f64 ? sizeof(double) : sizeof(float);
    Scratch wt;
    URCHIN_TRY(wt.alloc(rsz * (size_t)n, s));
    float* hw32 = f64 ? nullptr : wt.at<float>(0);
    double* hw64 = f64 ? wt.at<double>(0) : nullptr;
    const double* src[2] = {P.he1, P.he2};
    void* dst[2] = {tau_he1, tau_he2};
    for (int q = 0; q < 2; ++q) {
        URCHIN_TRY(launch_weights(bvh, src[q], hw32, hw64, s));
        TraceJob job{};
        job.bvh = bvh;
        job.w32 = hw32;
        job.w64 = hw64;
        job.dirs_dev = dirs;
        job.R = P.R;
        job.l_ray = P.l_ray;
        job.items = nullptr;
        job.n_items = n;
        job.row_stride = 1;
        job.k_stride = n;
        job.out_row = nullptr;
        job.out = dst[q];
        job.kernel = P.kernel;
        job.precision = P.precision;
        job.mode = 0;
        URCHIN_TRY(order_for(nullptr, n, &job.order));
        URCHIN_TRY(timed_trace(job));
        stats.traversals += 1;
    }
    wt.release();
    return URCHIN_OK;
}

int Solver::plain()
{
    URCHIN_TRY(he_columns());
    URCHIN_TRY(first_sweep());
    if (stats.max_rel_dx < P.tol) {
        stats.converged = 1;
        return URCHIN_OK;
    }
    return plain_sweeps(-1.0);
}

// Sweeps after sweep 0 until converged, out of iterations, or (stop_fraction
// >= 0) at most stop_fraction of the non-frozen particles above tol.
int Solver::plain_sweeps(double stop_fraction)
{
    URCHIN_TRY(order_by_density());
    while (stats.iterations < P.max_iter) {
        URCHIN_TRY_CUDA(cudaMemsetAsync(misc, 0, sizeof(unsigned long long), s));
        URCHIN_TRY_CUDA(cudaMemsetAsync(misc + 7, 0, sizeof(unsigned long long), s));
        for (size_t b = 0; b + 1 < block_lo.size(); ++b) {
            const int64_t lo = block_lo[b], m = block_lo[b + 1] - block_lo[b];
            if (m <= 0) continue;
            URCHIN_TRY(columns(list + lo, m, 0));
            URCHIN_TRY(timed_sweep(sweep_args(list + lo, m, 0), s));
        }
        double m;
        unsigned st;
        URCHIN_TRY(read_scalars(&m, &st));
        stats.iterations += 1;
        stats.particle_updates += n_act;
        stats.max_rel_dx = m;
        record(m);
        if (m < P.tol) {
            stats.converged = 1;
            break;
        }
        if (stop_fraction >= 0.0 && (double)last_above <= stop_fraction * (double)n_act) break;
    }
    return URCHIN_OK;
}

// One evaluation of the sweep map at the current x without updating it:
// E = E(Gamma(x)), the tangent factors, max |E - x| / x, and the residual
// r = ln E - ln x (into V0) with its 2-norm.
int Solver::evaluate(int frozen, double* V0, double* E, double* ctan, double* dtmp, double* hdev, double* maxrel,
                     double* norm, int64_t* switches, int tangent)
{
    const int64_t na = n_act;
    const unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((na + 255) / 256, 2048));
    URCHIN_TRY_CUDA(cudaMemsetAsync(misc, 0, sizeof(unsigned long long), s));
    URCHIN_TRY_CUDA(cudaMemsetAsync(misc + 7, 0, 2 * sizeof(unsigned long long), s));
    URCHIN_TRY(columns(list, na, 0));
    SweepArgs A = sweep_args(list, na, 0);
    A.want_tangent = tangent;
    A.ctan = tangent ? ctan : nullptr;
    A.xeq_out = E;
    A.latch_frozen = frozen;
    URCHIN_TRY(timed_sweep(A, s));
    k_residual<<<g1, 256, 0, s>>>(list, na, x, E, V0);
    URCHIN_TRY(launched());
    URCHIN_TRY(launch_dots(V0, na, 1, V0, na, dtmp, hdev, s));
    double r2 = 0.0;
    unsigned long long sw = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&r2, hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&sw, misc + 8, sizeof(sw), cudaMemcpyDeviceToHost, s));
    unsigned st;
    URCHIN_TRY(read_scalars(maxrel, &st));
    *norm = std::sqrt(std::max(r2, 0.0));
    *switches = (int64_t)sw;
    stats.iterations += 1;
    stats.particle_updates += na;
    stats.max_rel_dx = *maxrel;
    record(*maxrel);
    return URCHIN_OK;
}

// Newton-Krylov on the fixed point of the sweep map, in u = ln x over the
// non-frozen particles: G(u) = u - ln E(Gamma(x)), with each particle's
// recombination case held at its value in the evaluation.  J v = v - C dtau(x v)
// where dtau is the column of the tangent vector (columns are linear in x)
// and C holds c_ak = (1/E) dE/dGamma dGamma/dtau_k from the sweep kernel.
// Each step solves J d = -G by GMRES(m) to relative residual eta
// (Eisenstat-Walker), then backtracks x <- x exp(lam d), lam = 1, 1/2, ...,
// until ||G||_2 decreases.  Within a step the recombination cases are held
// at the latch of the step's base point, so G is smooth along the search;
// when an accepted point has particles newly past tau_eff = 1 the latch is
// updated there by a plain evaluation.  It stops when max |E - x| / x <
// dx_tol with no case left to switch and returns x <- E: the same test and
// the same final update as the plain sweep.  Every evaluation of the sweep
// map counts as one iteration.
int Solver::newton()
{
    URCHIN_TRY(first_sweep());
    if (stats.max_rel_dx < P.tol || n_act == 0) {
        stats.converged = 1;
        return URCHIN_OK;
    }
    // plain sweeps as the predictor until few particles are left above tol
    URCHIN_TRY(plain_sweeps(P.newton_switch > 0.0 ? P.newton_switch : 0.01));
    stats.newton_start = stats.iterations;
    if (stats.converged || stats.iterations >= P.max_iter) return URCHIN_OK;
    const int m = P.gmres_m;
    const int64_t na = n_act;
    const size_t rsz = f64 ? sizeof(double) : sizeof(float);
    Layout lay;
    size_t o_V = lay.take(sizeof(double) * (size_t)(m + 1) * na);
    size_t o_E = lay.take(sizeof(double) * (size_t)na);
    size_t o_c = lay.take(sizeof(double) * (size_t)na * P.R);
    size_t o_d = lay.take(sizeof(double) * (size_t)na);
    size_t o_xb = lay.take(sizeof(double) * (size_t)na);
    size_t o_Eb = lay.take(sizeof(double) * (size_t)na);
    size_t o_z = lay.take(rsz * (size_t)n);
    size_t o_wz = lay.take(stored ? 0 : rsz * (size_t)n);
    size_t o_dt = lay.take(dots_tmp_bytes(m + 1));
    size_t o_h = lay.take(sizeof(double) * (size_t)(m + 2));
    URCHIN_TRY(nk.alloc(lay.bytes, s));
    double* V = nk.at<double>(o_V);
    double* E = nk.at<double>(o_E);
    double* ctan = nk.at<double>(o_c);
    double* d = nk.at<double>(o_d);
    double* xb = nk.at<double>(o_xb);
    double* Eb = nk.at<double>(o_Eb);
    float* z32 = f64 ? nullptr : nk.at<float>(o_z);
    double* z64 = f64 ? nk.at<double>(o_z) : nullptr;
    float* wz32 = (stored || f64) ? nullptr : nk.at<float>(o_wz);
    double* wz64 = (stored || !f64) ? nullptr : nk.at<double>(o_wz);
    double* dtmp = nk.at<double>(o_dt);
    double* hdev = nk.at<double>(o_h);
    const unsigned g1 = (unsigned)std::max<int64_t>(1, std::min<int64_t>((na + 255) / 256, 2048));
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hcol(m + 2), y(m);
    double eta = P.newton_eta > 0.0 ? P.newton_eta : 0.1, prev_norm = -1.0;
    double mrel = 0.0, norm = 0.0;
    int64_t sw = 0;
    URCHIN_TRY(evaluate(0, V, E, ctan, dtmp, hdev, &mrel, &norm, &sw));
    for (;;) {
        if (mrel < P.tol || stats.iterations >= P.max_iter || norm == 0.0) {
            // converged (or out of evaluations): finish with the plain update
            k_set_x<<<g1, 256, 0, s>>>(list, na, nullptr, 0.0, nullptr, E, x, bvh->A64, w32, w64, xs32, xs64);
            URCHIN_TRY(launched());
            if (mrel < P.tol) stats.converged = 1;
            break;
        }
        // GMRES(m) for J d = r, r = -G already in V0, d0 = 0
        const double beta = norm;
        if (P.newton_eta > 0.0) eta = P.newton_eta;
        else if (prev_norm > 0.0) eta = std::min(0.1, std::max(1e-3, 0.9 * (beta / prev_norm) * (beta / prev_norm)));
        prev_norm = beta;
        URCHIN_TRY(launch_axpby(0.0, V, 1.0 / beta, V, na, s));
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = V + (size_t)j * na;
            double* w = V + (size_t)(j + 1) * na;
            if (z32) URCHIN_TRY_CUDA(cudaMemsetAsync(z32, 0, sizeof(float) * (size_t)n, s));
            if (z64) URCHIN_TRY_CUDA(cudaMemsetAsync(z64, 0, sizeof(double) * (size_t)n, s));
            if (wz32) URCHIN_TRY_CUDA(cudaMemsetAsync(wz32, 0, sizeof(float) * (size_t)n, s));
            if (wz64) URCHIN_TRY_CUDA(cudaMemsetAsync(wz64, 0, sizeof(double) * (size_t)n, s));
            k_tangent_vector<<<g1, 256, 0, s>>>(list, na, vj, x, bvh->A64, z32, z64, wz32, wz64);
            URCHIN_TRY(launched());
            URCHIN_TRY(linear_columns(list, na, z32, z64, wz32, wz64));
            if (f64) k_jv<double><<<g1, 256, 0, s>>>(vj, ctan, static_cast<const double*>(tau), na, P.R, w);
            else k_jv<float><<<g1, 256, 0, s>>>(vj, ctan, static_cast<const float*>(tau), na, P.R, w);
            URCHIN_TRY(launched());
            std::fill(hcol.begin(), hcol.end(), 0.0);
            for (int pass = 0; pass < 2; ++pass) {     // classical Gram-Schmidt, twice
                URCHIN_TRY(launch_dots(V, na, j + 1, w, na, dtmp, hdev, s));
                URCHIN_TRY(launch_subtract(w, V, na, j + 1, hdev, na, s));
                std::vector<double> hh(j + 1);
                URCHIN_TRY_CUDA(cudaMemcpyAsync(hh.data(), hdev, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
                URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i) hcol[i] += hh[i];
            }
            URCHIN_TRY(launch_dots(w, na, 1, w, na, dtmp, hdev, s));
            double hn2 = 0.0;
            URCHIN_TRY_CUDA(cudaMemcpyAsync(&hn2, hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
            URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
            const double hn = std::sqrt(std::max(hn2, 0.0));
            hcol[j + 1] = hn;
            if (hn > 0.0) URCHIN_TRY(launch_axpby(0.0, w, 1.0 / hn, w, na, s));
            for (int i = 0; i < j; ++i) {              // earlier Givens rotations
                const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = a;
            }
            const double r = std::hypot(hcol[j], hcol[j + 1]);
            cs[j] = r > 0.0 ? hcol[j] / r : 1.0;
            sn[j] = r > 0.0 ? hcol[j + 1] / r : 0.0;
            hcol[j] = r;
            hcol[j + 1] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
            kdim = j + 1;
            if (std::fabs(gv[j + 1]) <= eta * beta || hn == 0.0) break;
        }
        for (int i = kdim - 1; i >= 0; --i) {          // y = H^-1 g, d = V y
            double acc = gv[i];
            for (int k = i + 1; k < kdim; ++k) acc -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0.0 ? acc / H[(size_t)i * m + i] : 0.0;
        }
        for (int i = 0; i < kdim; ++i) y[i] = -y[i];
        URCHIN_TRY_CUDA(cudaMemcpyAsync(hdev, y.data(), sizeof(double) * kdim, cudaMemcpyHostToDevice, s));
        URCHIN_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * (size_t)na, s));
        URCHIN_TRY(launch_subtract(d, V, na, kdim, hdev, na, s));
        // backtracking on ||G||_2 from the base point (x, E saved); when no
        // trial decreases it, take the plain step x <- E(Gamma(x)) instead
        k_gather_x<<<g1, 256, 0, s>>>(list, na, x, xb);
        URCHIN_TRY(launched());
        URCHIN_TRY_CUDA(cudaMemcpyAsync(Eb, E, sizeof(double) * (size_t)na, cudaMemcpyDeviceToDevice, s));
        double lam = 1.0;
        bool accepted = false;
        for (int ls = 0; ls < 3 && stats.iterations < P.max_iter; ++ls) {
            k_set_x<<<g1, 256, 0, s>>>(list, na, d, lam, xb, nullptr, x, bvh->A64, w32, w64, xs32, xs64);
            URCHIN_TRY(launched());
            double mrel_t, norm_t;
            int64_t sw_t = 0;
            URCHIN_TRY(evaluate(1, V, E, ctan, dtmp, hdev, &mrel_t, &norm_t, &sw_t));
            if (norm_t <= (1.0 - 1e-4 * lam) * norm) {
                mrel = mrel_t;
                norm = norm_t;
                sw = sw_t;
                accepted = true;
                break;
            }
            lam *= 0.5;
        }
        if (!accepted) {
            stats.newton_fallbacks += 1;
            k_set_x<<<g1, 256, 0, s>>>(list, na, nullptr, 0.0, nullptr, Eb, x, bvh->A64, w32, w64, xs32, xs64);
            URCHIN_TRY(launched());
            if (stats.iterations >= P.max_iter) break;
            URCHIN_TRY(evaluate(0, V, E, ctan, dtmp, hdev, &mrel, &norm, &sw));
            continue;
        }
        if (sw > 0 && stats.iterations < P.max_iter) {
            // cases newly past tau_eff = 1: latch them and re-evaluate here
            URCHIN_TRY(evaluate(0, V, E, ctan, dtmp, hdev, &mrel, &norm, &sw));
        }
    }
    return URCHIN_OK;
}

// z[j] += sum over the active rays (k, a) of coef[k na + a] A_j K_ajk, for
// every particle j (Morton): the transpose of the columns, by a scatter
// traversal or over the stored segments.
int Solver::transpose_columns(const void* coef, double* z)
{
    stats.traversals += 1;
    stats.rays += n_act * P.R;
    if (stored) {
        SpmvTArgs A{};
        A.row_ptr = row_ptr;
        A.col = seg_col;
        A.lo = seg_lo;
        A.hi = seg_hi;
        A.val = seg_val;
        A.coef = coef;
        A.items = list;
        A.n_items = n_act;
        A.n_rows_per_k = n;
        A.R = P.R;
        A.precision = P.precision;
        A.z = z;
        cudaEvent_t stop;
        URCHIN_TRY(begin_timed(1, &stop));
        URCHIN_TRY(launch_spmv_t(A, s));
        return end_timed(stop);
    }
    TraceJob job{};
    job.bvh = bvh;
    job.dirs_dev = dirs;
    job.R = P.R;
    job.l_ray = P.l_ray;
    job.items = list;
    job.n_items = n_act;
    job.row_stride = 1;
    job.k_stride = n_act;
    job.out_row = nullptr;
    job.kernel = P.kernel;
    job.precision = P.precision;
    job.mode = 3;
    job.coef = coef;
    job.xbar = z;
    URCHIN_TRY(order_for(list, n_act, &job.order));
    return timed_trace(job);
}

// Reverse mode at a converged state x* (held in x): with the cases and the
// frozen set of the forward solve (state), solve
//   (I - J_u^T) nu = x_bar (.) x*        (J_u: sweep-map Jacobian in ln x)
// by restarted GMRES, each product one transposed column pass, then
//   w_bar_b += sum_a nu_a (E_a/x_a) elas_a dGamma_a/dw_b / Gamma_a
//            + [cold start] sum_f (x_bar_f + (J^T mu)_f) dx_f/dGamma(Gamma_thin),
// the frozen particles' x_thin depending on Gamma_thin = sum_b w_b.
int Solver::adjoint(const uint8_t* state_orig, const double* xbar_orig, int cold_start, double* w_bar)
{
    const unsigned gn = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
    k_state_in<<<gn, 256, 0, s>>>(bvh->perm, state_orig, n, active, latch, status);
    URCHIN_TRY(launched());
    uint32_t* cnt = reinterpret_cast<uint32_t*>(misc + 2);
    URCHIN_TRY(compact_indices(active, n, list, cnt, comp_tmp, s));
    items_changed();
    uint32_t hc = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    double mrel;
    unsigned st;
    URCHIN_TRY(read_scalars(&mrel, &st));
    if (st & kStInput) return set_error(URCHIN_ERR_ARG, "urchin_solve_vjp: state values must be in 0..3");
    n_act = hc;
    stats.n_active = n_act;
    if (P.segments != URCHIN_SEG_RECOMPUTE) URCHIN_TRY(columns(nullptr, n, 1, true));   // builds the stored segments
    const int64_t na = n_act;
    const int m = P.gmres_m;
    const size_t rsz = f64 ? sizeof(double) : sizeof(float);
    const int64_t nr = std::max<int64_t>(na * P.R, 1);
    Layout lay;
    size_t o_E = lay.take(sizeof(double) * (size_t)std::max<int64_t>(na, 1));
    size_t o_c = lay.take(sizeof(double) * (size_t)nr);
    size_t o_b = lay.take(sizeof(double) * (size_t)std::max<int64_t>(na, 1));
    size_t o_nu = lay.take(sizeof(double) * (size_t)std::max<int64_t>(na, 1));
    size_t o_V0 = lay.take(sizeof(double) * (size_t)std::max<int64_t>(na, 1));
    size_t o_cf = lay.take(rsz * (size_t)nr);
    size_t o_z = lay.take(sizeof(double) * (size_t)n);
    size_t o_t = lay.take(sizeof(double) * (size_t)n);
    size_t o_one = lay.take(sizeof(double) * (size_t)n);
    size_t o_lc = lay.take(sizeof(double) * (size_t)nr);
    size_t o_sg = lay.take(sizeof(double) * (size_t)nr);
    size_t o_dt = lay.take(dots_tmp_bytes(2));
    size_t o_h = lay.take(sizeof(double) * 4);
    size_t o_g = lay.take(gmres_work_bytes(std::max<int64_t>(na, 1), m));
    URCHIN_TRY(nk.alloc(lay.bytes, s));
    double* E = nk.at<double>(o_E);
    double* ctan = nk.at<double>(o_c);
    double* b = nk.at<double>(o_b);
    double* nu = nk.at<double>(o_nu);
    double* V0 = nk.at<double>(o_V0);
    void* coef = nk.at<void>(o_cf);
    double* z = nk.at<double>(o_z);
    double* t = nk.at<double>(o_t);
    double* one = nk.at<double>(o_one);
    double* lc = nk.at<double>(o_lc);
    double* sg = nk.at<double>(o_sg);
    double* dtmp = nk.at<double>(o_dt);
    double* hdev = nk.at<double>(o_h);
    void* gw = nk.at<void>(o_g);
    const unsigned ga = (unsigned)std::max<int64_t>(1, std::min<int64_t>((na + 255) / 256, 2048));
    const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nr + 255) / 256, 4096));
    GmresResult gres;
    if (na > 0) {
        // E, c_ak and the columns at x*, cases held at the forward solve's
        double norm;
        int64_t sw;
        URCHIN_TRY(evaluate(1, V0, E, ctan, dtmp, hdev, &mrel, &norm, &sw, 1));
        k_adj_rhs<<<ga, 256, 0, s>>>(list, na, bvh->perm, xbar_orig, x, b);
        URCHIN_TRY(launched());
        auto matvec = [&](const double* v, double* out) -> int {
            if (f64) k_adj_coef<double><<<gr, 256, 0, s>>>(list, na, P.R, v, E, x, ctan, static_cast<double*>(coef));
            else k_adj_coef<float><<<gr, 256, 0, s>>>(list, na, P.R, v, E, x, ctan, static_cast<float*>(coef));
            URCHIN_TRY(launched());
            URCHIN_TRY_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)n, s));
            URCHIN_TRY(transpose_columns(coef, z));
            k_adj_apply<<<ga, 256, 0, s>>>(list, na, v, x, z, out);
            return launched();
        };
        URCHIN_TRY(gmres_solve(matvec, b, nu, na, m, P.tol, P.max_iter, gw, &gres, s));
        stats.iterations = gres.matvecs;
        stats.max_rel_dx = gres.rel_residual;
        stats.converged = gres.rel_residual <= P.tol ? 1 : 0;
        // active particles: w_bar_b += sum_a phi_a rho_ab
        // e2, wn and (FP32) the tail e2t of fold_prepare
        const size_t smem = (f64 ? 2 * sizeof(double) : 3 * sizeof(float)) * (size_t)P.spectrum.F;
        const void* fw = f64 ? (const void*)k_adj_wcoef<double> : (const void*)k_adj_wcoef<float>;
        if (smem > 48 * 1024)
            URCHIN_TRY_CUDA(cudaFuncSetAttribute(fw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (f64)
            k_adj_wcoef<double><<<ga, 256, smem, s>>>(list, na, P.R, static_cast<const double*>(tau), P.spectrum.s,
                                                      P.spectrum.w, P.spectrum.F, nu, E, x, nH, aA, aB, gc, latch,
                                                      P.case_rule, P.y, lc, sg);
        else
            k_adj_wcoef<float><<<ga, 256, smem, s>>>(list, na, P.R, static_cast<const float*>(tau), P.spectrum.s,
                                                     P.spectrum.w, P.spectrum.F, nu, E, x, nH, aA, aB, gc, latch,
                                                     P.case_rule, P.y, lc, sg);
        URCHIN_TRY(launched());
        URCHIN_TRY(launch_wbar(tau, P.precision, na * P.R, lc, sg, P.spectrum.s, P.spectrum.F, w_bar, s));
        // z = J^T mu over every particle, for the frozen term
        if (f64) k_adj_coef<double><<<gr, 256, 0, s>>>(list, na, P.R, nu, E, x, ctan, static_cast<double*>(coef));
        else k_adj_coef<float><<<gr, 256, 0, s>>>(list, na, P.R, nu, E, x, ctan, static_cast<float*>(coef));
        URCHIN_TRY(launched());
        URCHIN_TRY_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)n, s));
        URCHIN_TRY(transpose_columns(coef, z));
    } else {
        URCHIN_TRY_CUDA(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)n, s));
        stats.converged = 1;
    }
    if (cold_start && na < n) {
        k_adj_frozen<<<gn, 256, 0, s>>>(active, bvh->perm, xbar_orig, z, x, nH, aA, aB, gc, n, gthin, P.y,
                                         P.case_rule, t, one);
        URCHIN_TRY(launched());
        URCHIN_TRY(launch_dots(t, n, 1, one, n, dtmp, hdev, s));
        k_add_scalar<<<(P.spectrum.F + 255) / 256, 256, 0, s>>>(w_bar, P.spectrum.F, hdev);
        URCHIN_TRY(launched());
    }
    URCHIN_TRY(read_scalars(&mrel, &st));
    return URCHIN_OK;
}

// Sweep-map tangent at the current x (see urchin_tangent): one traversal for
// E and the factors c_ik, one for the columns of x v.
int Solver::tangent(const double* v_orig, double* E_orig, double* dlnE_orig)
{
    const size_t rsz = f64 ? sizeof(double) : sizeof(float);
    Layout lay;
    size_t o_E = lay.take(sizeof(double) * (size_t)n);
    size_t o_c = lay.take(sizeof(double) * (size_t)n * P.R);
    size_t o_v = lay.take(sizeof(double) * (size_t)n);
    size_t o_jv = lay.take(sizeof(double) * (size_t)n);
    size_t o_z = lay.take(rsz * (size_t)n);
    size_t o_wz = lay.take(rsz * (size_t)n);
    URCHIN_TRY(nk.alloc(lay.bytes, s));
    double* E = nk.at<double>(o_E);
    double* ctan = nk.at<double>(o_c);
    double* vm = nk.at<double>(o_v);
    double* jv = nk.at<double>(o_jv);
    float* z32 = f64 ? nullptr : nk.at<float>(o_z);
    double* z64 = f64 ? nk.at<double>(o_z) : nullptr;
    float* wz32 = f64 ? nullptr : nk.at<float>(o_wz);
    double* wz64 = f64 ? nk.at<double>(o_wz) : nullptr;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
    k_iota<<<g, 256, 0, s>>>(list, n);
    URCHIN_TRY(launched());
    items_changed();
    n_act = n;
    URCHIN_TRY(trace(list, n, w32, w64));
    URCHIN_TRY_CUDA(cudaMemsetAsync(misc, 0, sizeof(unsigned long long), s));
    SweepArgs A = sweep_args(list, n, 0);
    A.want_tangent = 1;
    A.ctan = ctan;
    A.xeq_out = E;
    URCHIN_TRY(timed_sweep(A, s));
    k_to_morton<<<g, 256, 0, s>>>(bvh->perm, v_orig, n, vm);
    URCHIN_TRY(launched());
    k_tangent_vector<<<g, 256, 0, s>>>(list, n, vm, x, bvh->A64, z32, z64, wz32, wz64);
    URCHIN_TRY(launched());
    URCHIN_TRY(linear_columns(list, n, z32, z64, wz32, wz64));
    if (f64) k_jv<double><<<g, 256, 0, s>>>(vm, ctan, static_cast<const double*>(tau), n, P.R, jv);
    else k_jv<float><<<g, 256, 0, s>>>(vm, ctan, static_cast<const float*>(tau), n, P.R, jv);
    URCHIN_TRY(launched());
    k_tangent_out<<<g, 256, 0, s>>>(bvh->perm, vm, jv, E, n, dlnE_orig, E_orig);
    URCHIN_TRY(launched());
    double m;
    unsigned st;
    URCHIN_TRY(read_scalars(&m, &st));
    nk.release();
    scr.release();
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    return URCHIN_OK;
}

int Solver::finish(double* x_inout)
{
    unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    if (x_inout) {
        k_finish<<<grid, 256, 0, s>>>(bvh->perm, x, n, x_inout);
        URCHIN_TRY(launched());
    }
    if (P.profile) {
        unsigned long long h[3] = {0, 0, 0};
        URCHIN_TRY_CUDA(cudaMemcpyAsync(h, hits, sizeof(h), cudaMemcpyDeviceToHost, s));
        URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
        stats.hits = (int64_t)h[0];
        stats.sphere_tests = (int64_t)h[1];
        stats.node_visits = (int64_t)h[2];
        double total[3] = {0.0, 0.0, 0.0};
        for (size_t i = 0; i + 1 < events.size(); i += 2) {
            float ms = 0.f;
            URCHIN_TRY_CUDA(cudaEventElapsedTime(&ms, events[i], events[i + 1]));
            total[event_kind[i / 2]] += ms;
        }
        stats.trace_s = total[0] * 1e-3;
        stats.spmv_s = total[1] * 1e-3;
        stats.sweep_s = total[2] * 1e-3;
    }
    nk.release();
    seg.release();
    chunk_mem.release();
    ord.release();
    scr.release();
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    return URCHIN_OK;
}

Solver::~Solver()
{
    for (cudaEvent_t e : events) cudaEventDestroy(e);
}

}  // namespace urchin

extern "C" int urchin_tangent(const urchin_bvh* bvh, const urchin_solve_params* P, const double* x,
                              const double* v, double* E_out, double* dlnE_out, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (!bvh || !P || !x || !v || !dlnE_out)
        return set_error(URCHIN_ERR_ARG, "urchin_tangent: NULL bvh, params, x, v or dlnE_out");
    if (P->R < 1 || P->R > URCHIN_MAX_RAYS || !P->dirs)
        return set_error(URCHIN_ERR_ARG, "urchin_tangent: bad ray set (R = %d)", P->R);
    for (int k = 0; k < P->R; ++k) {
        const double* d = P->dirs + 3 * k;
        double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!std::isfinite(nn) || std::fabs(nn - 1.0) > 1e-6)
            return set_error(URCHIN_ERR_ARG, "urchin_tangent: direction %d is not a unit vector", k);
    }
    if (!(P->l_ray >= 0.0) || !std::isfinite(P->l_ray)) return set_error(URCHIN_ERR_ARG, "urchin_tangent: bad l_ray");
    if (P->spectrum.F < 1 || P->spectrum.F > URCHIN_MAX_BINS || !P->spectrum.s || !P->spectrum.w)
        return set_error(URCHIN_ERR_ARG, "urchin_tangent: bad spectrum");
    if (!P->nH || !P->T || !(P->y >= 0.0)) return set_error(URCHIN_ERR_ARG, "urchin_tangent: bad nH, T or y");
    if (P->kernel != URCHIN_KERNEL_M4 && P->kernel != URCHIN_KERNEL_GT)
        return set_error(URCHIN_ERR_ARG, "urchin_tangent: unknown kernel");
    if (P->precision != URCHIN_F32 && P->precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "urchin_tangent: unknown precision");
    if (P->case_rule != URCHIN_CASE_A && P->case_rule != URCHIN_CASE_B && P->case_rule != URCHIN_CASE_AUTO)
        return set_error(URCHIN_ERR_ARG, "urchin_tangent: unknown case_rule");
    if (P->near_far) return set_error(URCHIN_ERR_ARG, "urchin_tangent: no tangent of the near/far split");
    if (spectrum_has_he(&P->spectrum)) return set_error(URCHIN_ERR_ARG, "urchin_tangent: no helium in the tangent");
    urchin_solve_params Q = *P;
    Q.warm_start = 1;
    Q.segments = URCHIN_SEG_RECOMPUTE;
    Q.profile = 0;
    Q.tol = Q.tol > 0.0 ? Q.tol : 1e-3;
    Q.max_iter = 1;
    cudaStream_t s = (cudaStream_t)stream;
    Solver S;
    int st = S.init(bvh, &Q, const_cast<double*>(x), s);
    if (st == URCHIN_OK) st = S.tangent(v, E_out, dlnE_out);
    if (st != URCHIN_OK) cudaStreamSynchronize(s);
    return st;
}

namespace urchin {
namespace {

int check_solve_params(const char* fn, const urchin_bvh* bvh, const urchin_solve_params* P, const void* x)
{
    if (!bvh || !P || !x) return set_error(URCHIN_ERR_ARG, "%s: NULL bvh, params or x", fn);
    if (P->R < 1 || P->R > URCHIN_MAX_RAYS || !P->dirs)
        return set_error(URCHIN_ERR_ARG, "%s: bad ray set (R = %d)", fn, P->R);
    for (int k = 0; k < P->R; ++k) {
        const double* d = P->dirs + 3 * k;
        double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!std::isfinite(nn) || std::fabs(nn - 1.0) > 1e-6)
            return set_error(URCHIN_ERR_ARG, "%s: direction %d is not a unit vector", fn, k);
    }
    if (!(P->l_ray >= 0.0) || !std::isfinite(P->l_ray)) return set_error(URCHIN_ERR_ARG, "%s: bad l_ray", fn);
    if (P->spectrum.F < 1 || P->spectrum.F > URCHIN_MAX_BINS || !P->spectrum.s || !P->spectrum.w)
        return set_error(URCHIN_ERR_ARG, "%s: bad spectrum", fn);
    if (!P->nH || !P->T) return set_error(URCHIN_ERR_ARG, "%s: NULL nH or T", fn);
    if (!(P->tol > 0.0) || !(P->tau_skip >= 0.0) || P->max_iter < 1 || !(P->y >= 0.0))
        return set_error(URCHIN_ERR_ARG, "%s: need tol > 0, tau_skip >= 0, max_iter >= 1, y >= 0", fn);
    if (P->kernel != URCHIN_KERNEL_M4 && P->kernel != URCHIN_KERNEL_GT)
        return set_error(URCHIN_ERR_ARG, "%s: unknown kernel", fn);
    if (P->precision != URCHIN_F32 && P->precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "%s: unknown precision", fn);
    if (P->case_rule != URCHIN_CASE_A && P->case_rule != URCHIN_CASE_B && P->case_rule != URCHIN_CASE_AUTO)
        return set_error(URCHIN_ERR_ARG, "%s: unknown case_rule", fn);
    if (P->method != URCHIN_METHOD_PLAIN && P->method != URCHIN_METHOD_NEWTON)
        return set_error(URCHIN_ERR_ARG, "%s: unknown method", fn);
    if (P->segments != URCHIN_SEG_RECOMPUTE && P->segments != URCHIN_SEG_STORE && P->segments != URCHIN_SEG_AUTO)
        return set_error(URCHIN_ERR_ARG, "%s: unknown segments mode", fn);
    if (!std::isfinite(P->newton_eta) || !(P->newton_eta < 1.0))
        return set_error(URCHIN_ERR_ARG, "%s: newton_eta must be finite and < 1", fn);
    if (spectrum_has_he(&P->spectrum) && (!P->spectrum.s_he1 || !P->spectrum.s_he2 || !P->he1 || !P->he2))
        return set_error(URCHIN_ERR_ARG, "%s: helium needs spectrum s_he1 and s_he2 and params he1 and he2", fn);
    return URCHIN_OK;
}

}  // namespace
}  // namespace urchin

extern "C" int urchin_solve(const urchin_bvh* bvh, const urchin_solve_params* P, double* x_inout,
                            urchin_solve_stats* stats, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof(*stats));
    URCHIN_TRY(check_solve_params("urchin_solve", bvh, P, x_inout));
    if (P->method != URCHIN_METHOD_PLAIN && (P->gmres_m < 1 || P->gmres_m > 64))
        return set_error(URCHIN_ERR_ARG, "urchin_solve: gmres_m must be in [1, 64]");
    if (P->near_far != 0 && P->near_far != URCHIN_SLAB_THRESHOLD && P->near_far != URCHIN_SLAB_SPECTRUM)
        return set_error(URCHIN_ERR_ARG, "urchin_solve: near_far must be 0, URCHIN_SLAB_THRESHOLD or URCHIN_SLAB_SPECTRUM");
    if (P->near_far && (P->method != URCHIN_METHOD_PLAIN || P->blocks > 1 || P->y != 0.0))
        return set_error(URCHIN_ERR_ARG, "urchin_solve: the near/far split needs the plain Jacobi method and y = 0");
    if (spectrum_has_he(&P->spectrum) && (P->method != URCHIN_METHOD_PLAIN || P->blocks > 1 || P->near_far))
        return set_error(URCHIN_ERR_ARG, "urchin_solve: helium needs the plain Jacobi method without near/far split");
    cudaStream_t s = (cudaStream_t)stream;
    Solver S;
    int st = S.init(bvh, P, x_inout, s);
    if (st == URCHIN_OK) st = S.run();
    if (st == URCHIN_OK && P->state) {
        unsigned grid = (unsigned)std::min<int64_t>((S.n + 255) / 256, 4096);
        k_state_out<<<grid, 256, 0, s>>>(bvh->perm, S.active, S.latch, S.n, P->case_rule, P->state);
        st = launched();
    }
    if (st == URCHIN_OK) st = S.finish(x_inout);
    else cudaStreamSynchronize(s);
    S.stats.wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S.stats;
    if (st != URCHIN_OK) return st;
    if (!S.stats.converged)
        return set_error(URCHIN_ERR_NOT_CONVERGED, "urchin_solve: max |dx|/x = %.3e after %d iterations",
                         S.stats.max_rel_dx, S.stats.iterations);
    return URCHIN_OK;
}

extern "C" int urchin_solve_vjp(const urchin_bvh* bvh, const urchin_solve_params* P, const double* x_star,
                                const double* x_bar, double* w_bar, urchin_solve_stats* stats,
                                urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    auto t0 = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof(*stats));
    URCHIN_TRY(check_solve_params("urchin_solve_vjp", bvh, P, x_star));
    if (!x_bar || !w_bar || !P->state)
        return set_error(URCHIN_ERR_ARG, "urchin_solve_vjp: NULL x_bar, w_bar or params->state");
    if (P->near_far) return set_error(URCHIN_ERR_ARG, "urchin_solve_vjp: no adjoint of the near/far split");
    if (spectrum_has_he(&P->spectrum)) return set_error(URCHIN_ERR_ARG, "urchin_solve_vjp: no helium in reverse mode");
    if (P->gmres_m < 1 || P->gmres_m > 64)
        return set_error(URCHIN_ERR_ARG, "urchin_solve_vjp: gmres_m must be in [1, 64]");
    urchin_solve_params Q = *P;
    Q.warm_start = 1;                      // x = x*
    Q.history_maxrel = nullptr;
    Q.history_unconverged = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    Solver S;
    int st = S.init(bvh, &Q, const_cast<double*>(x_star), s);
    if (st == URCHIN_OK) st = S.adjoint(P->state, x_bar, P->warm_start ? 0 : 1, w_bar);
    if (st == URCHIN_OK) st = S.finish(nullptr);
    else cudaStreamSynchronize(s);
    S.stats.wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S.stats;
    if (st != URCHIN_OK) return st;
    if (!S.stats.converged)
        return set_error(URCHIN_ERR_NOT_CONVERGED, "urchin_solve_vjp: GMRES relative residual %.3e after %d products",
                         S.stats.max_rel_dx, S.stats.iterations);
    return URCHIN_OK;
}
