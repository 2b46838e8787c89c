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

struct Rates {
    double alphaA, alphaB, gamma_c;   // cm^3 s^-1
};

// Hui & Gnedin (1997) fits, lambda = 2 T_HI / T with T_HI = 157807 K:
//   alpha_A = 1.269e-13 lambda^1.503 / [1 + (lambda/0.522)^0.470]^1.923
//   alpha_B = 2.753e-14 lambda^1.500 / [1 + (lambda/2.740)^0.407]^2.242
//   gamma   = 21.11 T^-3/2 e^(-lambda/2) lambda^-1.089 / [1 + (lambda/0.354)^0.874]^1.101
// (App. C3 names fits of this kind for the temperature dependence.)
__device__ __forceinline__ Rates hg97_rates(double T)
{
    const double lam = 315614.0 / T;
    const double ll = log(lam);
    Rates r;
    r.alphaA = 1.269e-13 * exp(1.503 * ll) / pow(1.0 + exp(0.470 * (ll - log(0.522))), 1.923);
    r.alphaB = 2.753e-14 * exp(1.500 * ll) / pow(1.0 + exp(0.407 * (ll - log(2.740))), 2.242);
    r.gamma_c = 21.11 * pow(T, -1.5) * exp(-0.5 * lam - 1.089 * ll) /
                pow(1.0 + exp(0.874 * (ll - log(0.354))), 1.101);
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

}  // namespace urchin
