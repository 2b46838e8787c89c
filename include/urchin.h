/*
 * urchin.h -- C ABI of the GB300 reverse ray tracer for self-shielding from
 * the UV background (Altay & Theuns, "Urchin: A Reverse Ray Tracer for
 * Astrophysical Applications", arXiv:1304.4235).
 *
 * The library computes, for every SPH gas particle, the hydrogen columns
 * along N_ray HEALPix rays cast outward from the particle (Sec. 3.2,
 * Eq. colden), folds them through a binned UV-background spectrum into the
 * shielded photoionisation rate (Eq. gamma_shld), solves the ionisation
 * equilibrium for the neutral fraction x (App. C3, Eq. xroots) and iterates
 * to convergence (Sec. 4).  All arithmetic runs in CUDA kernels for sm_103a.
 *
 * Conventions shared by every entry point
 *   - Pointers documented as "device" are CUDA device pointers owned by the
 *     caller; "host" pointers are ordinary host memory read during the call.
 *   - Calls are asynchronous on `stream` (NULL = legacy default stream)
 *     unless stated otherwise; outputs are valid once the stream reaches
 *     the call.  urchin_solve synchronises the stream (it reads a
 *     convergence scalar once per sweep).
 *   - Every call returns URCHIN_OK (0) or a negative URCHIN_ERR_* status; no
 *     exception, abort or device trap crosses the ABI.  urchin_last_error()
 *     returns a message for the calling thread's most recent failure.
 *   - Lengths (positions, h, box side, l_ray) share one caller-chosen unit;
 *     `unit_cm` converts it to cm.  Columns are returned as threshold
 *     optical depth tau = sigma_th N_HI with sigma_th = 2^9 pi/(3 e^4)
 *     alpha_fs pi a_0^2 = 6.3043e-18 cm^2 (App. C1, Eq. sigma_ana).
 *   - Work arrays the library needs are taken from a stream-ordered memory
 *     pool the library keeps per device (cudaMallocFromPoolAsync) and
 *     released on the same stream before the call returns.  Released memory
 *     stays reserved in that pool for later calls (mapping and unmapping the
 *     14 GB of stored segments of a 262144-particle solve costs ~30 ms);
 *     urchin_trim_memory returns it to the device.  urchin_build_bvh's
 *     result holds device memory until urchin_free_bvh.
 */
#ifndef URCHIN_H
#define URCHIN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define URCHIN_API __attribute__((visibility("default")))
#else
#define URCHIN_API
#endif

/* A cudaStream_t (the runtime's stream handle type). */
typedef struct CUstream_st* urchin_stream_t;

/* ---- status codes ------------------------------------------------------ */
#define URCHIN_OK                 0
#define URCHIN_ERR_ARG           -1   /* invalid argument (NULL, size, range)   */
#define URCHIN_ERR_CUDA          -2   /* a CUDA runtime call failed             */
#define URCHIN_ERR_NOMEM         -3   /* device allocation failed               */
#define URCHIN_ERR_NOT_CONVERGED -4   /* solve hit max_iter before dx_tol       */
#define URCHIN_ERR_NONFINITE     -5   /* NaN/Inf in an input or a result        */

/* ---- options ----------------------------------------------------------- */
#define URCHIN_KERNEL_M4        0     /* cubic spline, Eq. spline               */
#define URCHIN_KERNEL_GT        1     /* truncated Gaussian, Eq. Gt             */
#define URCHIN_F32              0     /* columns and spectral sum in float      */
#define URCHIN_F64              1     /* everything in double                   */
#define URCHIN_CASE_A           0     /* case A recombination everywhere        */
#define URCHIN_CASE_B           1     /* case B recombination everywhere        */
#define URCHIN_CASE_AUTO        2     /* case B iff tau_eff >= 1 (Sec. 4)       */
#define URCHIN_XSEC_VERNER      0     /* Verner et al. 1996 fit, App. C1        */
#define URCHIN_XSEC_HYDROGENIC  1     /* exact hydrogenic, Eq. sigma_ana        */
#define URCHIN_XSEC_POWERLAW    2     /* sigma_th (nu/nu_th)^-3, Eq. sigma_pwr  */
#define URCHIN_XSEC_HEII        3     /* He II: exact hydrogenic, Z = 2 (54.4 eV) */
#define URCHIN_METHOD_PLAIN     0     /* Jacobi fixed point (Sec. 4)            */
#define URCHIN_METHOD_NEWTON    1     /* Newton-Krylov on the same fixed point  */

/* Slab model for the near particles of the near/far split (Sec. 3.3.3) */
#define URCHIN_SLAB_THRESHOLD   1     /* analytic slab, radiation at threshold   */
#define URCHIN_SLAB_SPECTRUM    2     /* numerical slab, the binned spectrum     */
#define URCHIN_SEG_RECOMPUTE    0     /* trace the BVH every sweep              */
#define URCHIN_SEG_STORE        1     /* store per-ray segment lists once       */
#define URCHIN_SEG_AUTO         2     /* store when the lists fit in memory     */
/* A stored segment is the FP32 value and the particle's Morton index split
 * into 16 + 8 bits (7 bytes; n <= 2^24), or FP64 value and int32 index (12
 * bytes); each ray's list is padded with zero entries to a multiple of 8.
 * URCHIN_SEG_AUTO in FP32 (no near/far split, blocks <= 1) keeps the lists
 * of the first sweep's traversal itself, in linked chunks of 32 (index,
 * value) pairs of 8 bytes sized from a sampled estimate, so that a solve of
 * two sweeps traces once; from the fourth sweep the active rows are copied
 * into the 7-byte row layout when both fit.  When the chunks do not fit or
 * the estimate proves short, the lists are stored from the third sweep (a
 * counting and a filling traversal) where they fit, else every sweep traces. */

#define URCHIN_MAX_RAYS       192     /* HEALPix N_side <= 4                    */
#define URCHIN_MAX_BINS      4096     /* frequency bins                         */
#define URCHIN_NOALLOC_SCRATCH_BYTES (16u << 20)   /* fixed work array of
                                     urchin_trace_columns_noalloc (16 MiB)    */

/* ---- data -------------------------------------------------------------- */

/* SPH particles, structure of arrays (Eq. nhi: r_i, h_i, m_i). */
typedef struct {
    int64_t       n;        /* particle count, >= 1                            */
    const float*  pos_x;    /* device [n] position                             */
    const float*  pos_y;    /* device [n]                                      */
    const float*  pos_z;    /* device [n]                                      */
    const float*  h;        /* device [n] smoothing length = kernel support
                               radius (W vanishes at |r - r_i| = h_i), > 0     */
    const double* mass_H;   /* device [n] hydrogen mass in proton masses
                               (m_i / m_p of Eq. nhi), >= 0                    */
} urchin_particles;

/* Simulation volume.  Periodic boxes are the cube [0, L)^3; rays then sum
 * every periodic image of every particle they reach. */
typedef struct {
    int    periodic;        /* 0 = isolated, 1 = periodic cube                 */
    double L;               /* box side (length unit), > 0 when periodic       */
    double unit_cm;         /* cm per length unit, > 0                         */
} urchin_box;

/* Binned UV-background spectrum (Eq. gamma_shld, Sec. 3.3.3):
 * Gamma/Gamma_thin = (1/N_ray) sum_k sum_j w_j exp(-s_j tau_k) / sum_j w_j.
 * Optional helium (the paper treats hydrogen only): the bins' He I and He II
 * cross sections in the same units; the exponent then becomes
 * s_j tau_k + s_he1_j tau_he1_k + s_he2_j tau_he2_k with the helium columns
 * tau_he (N_He sigma_th).  Only urchin_gamma_he and the plain urchin_solve
 * accept a spectrum with helium cross sections; the other calls return
 * URCHIN_ERR_ARG for it. */
typedef struct {
    int           F;        /* bins, 1..URCHIN_MAX_BINS                        */
    const double* s;        /* device [F] sigma(nu_j) / sigma_th, >= 0         */
    const double* w;        /* device [F] rate weights (s^-1), >= 0, with
                               sum_j w_j = Gamma_thin > 0                      */
    const double* s_he1;    /* device [F] sigma_HeI(nu_j) / sigma_th, or NULL  */
    const double* s_he2;    /* device [F] sigma_HeII(nu_j) / sigma_th, or NULL
                               (both or neither)                               */
} urchin_spectrum;

/* Opaque bounding-volume hierarchy over the particles' smoothing spheres
 * (Morton-ordered copy of the particle data plus a binary radix tree). */
typedef struct urchin_bvh urchin_bvh;

/* ---- entry points ------------------------------------------------------ */

/* Message for this thread's most recent failing call ("" if none). */
URCHIN_API const char* urchin_last_error(void);

/* Library version string. */
URCHIN_API const char* urchin_version(void);

/* Number of CUDA kernels this library has launched in this process
 * (instrumentation for benchmarks; no counterpart in the paper). */
URCHIN_API int64_t urchin_kernel_launches(void);

/* Return the device memory held by the library's work-array pool of
 * `device` (-1: every device the library has used) to the device, except
 * blocks still in use or whose stream-ordered release has not completed
 * (synchronise the streams of earlier calls first).  *reserved_out (may be
 * NULL) receives the bytes the pool(s) still reserve afterwards.  No
 * counterpart in the paper.  Errors: ERR_ARG (device out of range),
 * ERR_CUDA. */
URCHIN_API int urchin_trim_memory(int device, uint64_t* reserved_out);

/* HEALPix ray directions (Sec. 3.2; App. A: N_pix = 12 N_side^2): the unit
 * vectors to the pixel centres of the ring scheme of Gorski et al. (2005),
 * written to host `dirs_out[12 nside^2 * 3]` (x, y, z per ray).  Host only,
 * no GPU work.  Errors: ERR_ARG if nside < 1 or 12 nside^2 > URCHIN_MAX_RAYS
 * or dirs_out is NULL. */
URCHIN_API int urchin_healpix_dirs(int nside, double* dirs_out);

/* Binned spectrum weights for Eq. gamma_shld from a sampled UVB (host only):
 * E_edges[F+1] bin edges in eV (increasing, first >= 13.6057 eV), J[F] the
 * specific intensity at the geometric bin centres (any amplitude).  Writes
 * host s_out[F] = sigma(E_j)/sigma_th and w_out[F] proportional to
 * J_j sigma(E_j) / E_j (E_{j+1/2} - E_{j-1/2}), normalised to
 * sum w = gamma_thin (Eq. gamma with the 4 pi/h factors absorbed).
 * `xsec` selects the cross section (URCHIN_XSEC_*).  Errors: ERR_ARG. */
URCHIN_API int urchin_spectrum_weights(int F, const double* E_edges, const double* J, int xsec,
                            double gamma_thin, double* s_out, double* w_out);

/* Cross-section ratios for the bins (host only): s_out[j] =
 * sigma(E_j) / sigma_th at the geometric bin centres E_j of the F+1 edges
 * (eV, increasing), zero below the species' threshold.  xsec:
 * URCHIN_XSEC_VERNER / _HYDROGENIC / _POWERLAW (H I, App. C1) or
 * URCHIN_XSEC_HEII (He II, the exact hydrogenic form with Z = 2, for the
 * helium columns, which the paper does not treat).  Errors: ERR_ARG. */
URCHIN_API int urchin_cross_section_ratio(int F, const double* E_edges, int xsec, double* s_out);

/* Build the BVH (no counterpart in the paper, which does not describe its
 * search structure): Morton codes of the sphere centres, radix sort, binary
 * radix tree, bottom-up bounds, and a Morton-ordered copy of the particles.
 * The particle arrays are only read during the call.  `*out` receives a
 * library-owned object; release it with urchin_free_bvh.  The call
 * synchronises `stream`.  Errors: ERR_ARG (NULL, n < 1, h <= 0 or
 * non-positive sizes), ERR_NONFINITE (NaN/Inf in positions, h or mass),
 * ERR_NOMEM, ERR_CUDA. */
URCHIN_API int urchin_build_bvh(const urchin_particles* p, const urchin_box* box,
                     urchin_bvh** out, urchin_stream_t stream);

/* Release a BVH (NULL is ignored).  Synchronous. */
URCHIN_API void urchin_free_bvh(urchin_bvh* bvh);

/* Particle count of a BVH, or -1 for NULL. */
URCHIN_API int64_t urchin_bvh_size(const urchin_bvh* bvh);

/* Columns, Eq. colden: for origin o and direction k,
 *   tau[o*R + k] = sigma_th sum_j (m_j x_j / m_p) int_0^{l_ray} W(|r_i + t n_k - r_j| / h_j) dt,
 * summed over every particle (and periodic image) whose smoothing sphere
 * the segment crosses, the origin particle included (its half chord).
 *   x        device [n] neutral fractions (double, original particle order)
 *   dirs     host [R*3] unit directions (e.g. from urchin_healpix_dirs)
 *   R        1..URCHIN_MAX_RAYS
 *   l_ray    segment length >= 0 (length unit)
 *   origins  device [n_orig] particle indices (original order), or NULL for
 *            all n particles (then n_orig must equal n)
 *   kernel   URCHIN_KERNEL_M4 or URCHIN_KERNEL_GT
 *   precision URCHIN_F32: tau_out is float[n_orig*R]; URCHIN_F64: double
 * Errors: ERR_ARG, ERR_NOMEM, ERR_CUDA.  n_orig = 0 is a no-op. */
URCHIN_API int urchin_trace_columns(const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                         double l_ray, const int32_t* origins, int64_t n_orig,
                         int kernel, int precision, void* tau_out, urchin_stream_t stream);

/* Column tracing that allocates nothing (the paper has no counterpart: this
 * is a deployment variant of urchin_trace_columns, with the same arguments,
 * output and errors).  It is meant for callers that cannot call cudaMalloc
 * or cudaMallocAsync: code running inside a framework whose caching
 * allocator owns the device memory pool, services that pin a fixed memory
 * budget, or setups that treat any allocation on the hot path as an error.
 * Its work space (work-queue counter, status word, directions, per-particle
 * weights, mapped origins) lives in one file-scope device array of
 * URCHIN_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps
 * until the process exits; the call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *   - Size limit: 256 + 24 R + (4 or 8) n + 4 n_orig bytes (each part
 *     rounded up to 256) must fit in the array; larger requests return
 *     URCHIN_ERR_ARG and leave everything untouched.
 *   - The columns are bit for bit those of urchin_trace_columns (a ray sums
 *     its hits in the tree's fixed depth-first order, whichever rays share
 *     its warp), but the rays are traced in the order of the origin list:
 *     the per-direction ray ordering that urchin_trace_columns sorts into
 *     extra memory for 16384 or more origins is skipped, so large calls run
 *     slower.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) and caches it per device ordinal; make that
 *     first call before any stream capture.  The cache assumes the device
 *     keeps one CUDA context for the life of the process (after
 *     cudaDeviceReset it is stale).
 *   - Every call shares the one array and clears what must start at zero;
 *     calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on it and must be serialised by the caller.
 *   - It synchronises `stream` before returning, to read its status word. */
URCHIN_API int urchin_trace_columns_noalloc(const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                                            double l_ray, const int32_t* origins, int64_t n_orig,
                                            int kernel, int precision, void* tau_out,
                                            urchin_stream_t stream);

/* Columns with the near/far split of Sec. 3.3.3: for the ray (o, k), a
 * crossed particle j is near when the origin lies inside j's smoothing
 * sphere (|r_j - r_o| < h_j, j contributes to the density at r_o in
 * Eq. nhi; the origin itself is always near) and far otherwise:
 *   tau_far_out[o*R + k]  = sigma_th sum_far  (m_j x_j / m_p) int W dt
 *   tau_near_out[o*R + k] = sigma_th sum_near (m_j / m_p) int W dt   (x = 1)
 * The near test is made in double from the float positions.  Arguments,
 * layouts and errors as urchin_trace_columns. */
URCHIN_API int urchin_trace_columns_nearfar(const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                                            double l_ray, const int32_t* origins, int64_t n_orig, int kernel,
                                            int precision, void* tau_far_out, void* tau_near_out,
                                            urchin_stream_t stream);

/* Shielded rate with the near/far split (Eqs. gammafar, gammashldk,
 * gammashld): per ray the far rate Gamma_far,k = sum_j w_j exp(-s_j tau_far,k)
 * lights a uniform hydrogen slab of thickness tau_near,k with the origin's
 * nH and T (device [n_orig] double) and recombination case (caseB device
 * [n_orig], nonzero = case B; NULL = case A); the slab solution (y = 0)
 * gives the rate at its far side, and gamma_out[o] = (1/R) sum_k of those.
 *   slab = URCHIN_SLAB_THRESHOLD: the appendix's analytic solution for
 *          radiation at the threshold, lit with the far rate;
 *   slab = URCHIN_SLAB_SPECTRUM: the numerical slab solution for the binned
 *          spectrum hardened by tau_far (dtau_HI/dt = x_eq(Gamma(tau_far +
 *          tau_HI)) over the slab, t = N_H sigma_th depth), the paper's
 *          polychromatic G computed per ray instead of tabulated.
 * tau_eff_out as in urchin_gamma (may be NULL).  tau_far / tau_near as
 * written by urchin_trace_columns_nearfar.  Errors: ERR_ARG, ERR_NOMEM,
 * ERR_CUDA. */
URCHIN_API int urchin_gamma_nearfar(const void* tau_far, const void* tau_near, int precision, int64_t n_orig,
                                    int R, const urchin_spectrum* sp, const double* nH, const double* T,
                                    const unsigned char* caseB, int slab, double* gamma_out, float* tau_eff_out,
                                    urchin_stream_t stream);

/* Shielded rate, Eq. gamma_shld: for each of n_orig particles with R columns
 * tau[o*R + k] (float for URCHIN_F32, double for URCHIN_F64),
 *   gamma_out[o]   = (1/R) sum_k sum_j w_j exp(-s_j tau_ok)     (device, double)
 *   tau_eff_out[o] = -ln(gamma_out[o] / sum_j w_j)              (device, float;
 *                    may be NULL)
 * tau_eff stays finite where gamma underflows double.  Errors: ERR_ARG,
 * ERR_CUDA. */
URCHIN_API int urchin_gamma(const void* tau, int precision, int64_t n_orig, int R,
                 const urchin_spectrum* sp, double* gamma_out, float* tau_eff_out,
                 urchin_stream_t stream);

/* The rate behind hydrogen and helium columns (helium is not in the paper,
 * which treats hydrogen only): with the spectrum's s, s_he1, s_he2,
 *   gamma_out[o] = (1/R) sum_k sum_j w_j exp(-(s_j tau + s_he1_j tau_he1
 *                                               + s_he2_j tau_he2)[o*R + k]),
 * tau_eff_out as in urchin_gamma.  tau, tau_he1, tau_he2 device
 * [n_orig*R] of the precision's type (helium columns in units of N_He
 * sigma_th).  Errors: ERR_ARG (also when the spectrum lacks s_he1 / s_he2),
 * ERR_CUDA. */
URCHIN_API int urchin_gamma_he(const void* tau, const void* tau_he1, const void* tau_he2, int precision,
                               int64_t n_orig, int R, const urchin_spectrum* sp, double* gamma_out,
                               float* tau_eff_out, urchin_stream_t stream);

/* Ionisation equilibrium, App. C3 (Eqs. dxdt, xroots): the physical root
 * x_- of R x^2 + Q x + P = 0 with R = (gamma_c + alpha) n_H,
 * Q = -[Gamma + alpha n_H + R (1+y)], P = alpha n_H (1+y), in FP64, where
 * alpha = alpha_A or alpha_B(T) and gamma_c(T) are the Hui & Gnedin (1997)
 * fits.  case_rule URCHIN_CASE_AUTO takes case B where tau_eff >= 1 (then
 * tau_eff must not be NULL).  All arrays device [n], double except tau_eff.
 * Errors: ERR_ARG, ERR_CUDA. */
URCHIN_API int urchin_equilibrium(const double* gamma, const float* tau_eff, const double* nH,
                       const double* T, int64_t n, int case_rule, double y,
                       double* x_out, urchin_stream_t stream);

typedef struct {
    int             R;            /* rays per particle                         */
    const double*   dirs;         /* host [R*3]                                */
    double          l_ray;        /* ray length (length unit)                  */
    urchin_spectrum spectrum;     /* device arrays                             */
    const double*   nH;           /* device [n] hydrogen density (cm^-3)       */
    const double*   T;            /* device [n] temperature (K)                */
    double          y;            /* electrons from heavier elements per H     */
    double          tol;          /* dx_tol: stop when max |dx|/x < tol        */
    double          tau_skip;     /* freeze particles with tau_eff < tau_skip
                                     after the first sweep                     */
    int             max_iter;     /* sweep limit (plain) / Newton step limit   */
    int             method;       /* URCHIN_METHOD_*                           */
    int             segments;     /* URCHIN_SEG_*                              */
    int             gmres_m;      /* Krylov dimension per Newton step          */
    int             kernel;       /* URCHIN_KERNEL_*                           */
    int             precision;    /* URCHIN_F32 / URCHIN_F64 (columns, Gamma)  */
    int             case_rule;    /* URCHIN_CASE_*                             */
    int             warm_start;   /* 0: start from x_thin; 1: from x_inout     */
    int             profile;      /* 1: time every traversal with CUDA events
                                     and count kernel-chord evaluations        */
    double*         history_maxrel;      /* host [max_iter] or NULL: max |dx|/x
                                            after each sweep / Newton step     */
    int64_t*        history_unconverged; /* host [max_iter] or NULL: particles
                                            with |dx|/x >= tol at that point   */
    int             blocks;       /* update order after sweep 0 (plain method):
                                     1 = Jacobi (all x from the previous
                                     sweep); B > 1 = the Sec. 4 order, high to
                                     low density, in B blocks updated in
                                     sequence (float32 n_H descending, ties by
                                     particle index; block b holds ranks
                                     [b m / B, (b+1) m / B) of the m
                                     non-frozen particles)                     */
    double          newton_switch; /* NEWTON: plain sweeps run until at most this
                                      fraction of the non-frozen particles has
                                      |dx|/x >= tol, then Newton-Krylov takes
                                      over (<= 0: 0.01)                        */
    double          newton_eta;   /* NEWTON: GMRES relative residual per step
                                     (<= 0: Eisenstat-Walker, 0.1 ... 1e-3)   */
    unsigned char*  state;        /* device [n] or NULL, original order:
                                     urchin_solve writes, urchin_solve_vjp
                                     reads each particle's final state,
                                     bit 0 = recombination case B,
                                     bit 1 = frozen after sweep 0             */
    const double*   he1;          /* device [n] or NULL: He I atoms per H atom of
                                     each particle (n_He/n_H times the He I
                                     fraction, fixed), original order; needed
                                     when the spectrum has s_he1 / s_he2      */
    const double*   he2;          /* device [n] or NULL: He II atoms per H atom */
    int             near_far;     /* 0: off; URCHIN_SLAB_THRESHOLD or
                                     URCHIN_SLAB_SPECTRUM: the near/far split
                                     of Sec. 3.3.3 (plain method, blocks <= 1,
                                     y = 0): far particles give tau_far, the
                                     origin's near particles (those whose
                                     smoothing sphere holds it) a slab of
                                     thickness tau_near (x = 1); each ray's
                                     rate is that slab's solution (see
                                     urchin_gamma_nearfar) lit by the far-
                                     attenuated radiation, in the particle's
                                     case before the sweep                    */
} urchin_solve_params;

typedef struct {
    int     iterations;           /* sweeps (plain) or Newton steps            */
    int     traversals;           /* BVH traversals + stored-segment sweeps    */
    int64_t rays;                 /* rays evaluated (value and tangent)        */
    int64_t particle_updates;     /* x updates of non-frozen particles         */
    int64_t n_active;             /* particles not frozen after sweep 0        */
    int64_t nnz;                  /* stored segments, each ray padded to a
                                     multiple of 8 (0 in recompute mode)       */
    double  max_rel_dx;           /* last max |dx|/x over non-frozen particles */
    double  wall_s;               /* host wall time of the call                */
    int     converged;            /* 1 if max_rel_dx < tol                     */
    int     segments_stored;      /* 1 if the stored-segment mode ran          */
    int64_t hits;                 /* ray-sphere chord evaluations (profile=1)  */
    double  trace_s;              /* GPU time of the traversals (profile=1)    */
    int     trace_launches;       /* traversal kernel launches                 */
    int64_t sphere_tests;         /* ray-sphere tests at leaves (profile=1)    */
    int64_t node_visits;          /* internal nodes visited (profile=1)        */
    int     newton_fallbacks;     /* Newton steps replaced by a plain sweep    */
    int     newton_start;         /* iterations done before Newton took over   */
    double  spmv_s;               /* GPU time of stored-segment sweeps (profile=1) */
    int     spmv_launches;        /* stored-segment column launches            */
    int64_t spmv_bytes;           /* algorithmic bytes of those launches:
                                     segments read (index + value), columns
                                     written, x gathered once per launch       */
    double  sweep_s;              /* GPU time of the spectral/equilibrium
                                     kernel (profile=1)                        */
    int     sweep_launches;
} urchin_solve_stats;

/* Iterate to the equilibrium neutral fraction (Sec. 4): x starts at x_thin
 * (Gamma = Gamma_thin) unless warm_start; sweep 0 traces every particle and
 * freezes those with tau_eff < tau_skip at their current x; each later sweep
 * recomputes Gamma for all non-frozen particles from the previous sweep's x
 * (Jacobi) and updates them; the run stops when max |dx|/x < tol.
 * URCHIN_METHOD_NEWTON runs those sweeps until at most `newton_switch` of
 * the non-frozen particles remain above tol, then solves the same fixed
 * point x = E(Gamma(x)) with a Newton-Krylov iteration in ln x (GMRES with
 * tangent columns, backtracking, plain-sweep fallback).
 * With helium (spectrum s_he1 / s_he2, params he1 / he2; plain method,
 * no near/far split, blocks <= 1) the fixed He I and He II columns of every
 * ray are traced once, with weights he1 / he2, and attenuate the spectrum in
 * every sweep.
 * x_inout is device [n] double in the original particle order.  `stats` may be NULL.
 * Synchronises `stream`.  Returns URCHIN_ERR_NOT_CONVERGED (x_inout then
 * holds the last iterate) when max_iter is reached first. */
URCHIN_API int urchin_solve(const urchin_bvh* bvh, const urchin_solve_params* params,
                 double* x_inout, urchin_solve_stats* stats, urchin_stream_t stream);

/* Tangent of the sweep map that Newton-Krylov linearises (Sec. 4 iteration,
 * Eq. colden, Eq. gamma_shld, Eq. xroots): for the map x -> E(Gamma(x)) of
 * one sweep over all particles, with each particle's recombination case
 * taken from its tau_eff at x (params->case_rule, no latch), writes
 *   E_out[i]    = E_i(x)                                   (device, may be NULL)
 *   dlnE_out[i] = sum_j (d ln E_i / d ln x_j) v_j          (device)
 *              = sum_k c_ik dtau_ik,  dtau = columns of the vector x v,
 *     c_ik = (1/E_i) dE_i/dGamma_i dGamma_i/dtau_ik,
 * i.e. the directional derivative in ln x.  x and v are device [n] double in
 * the original particle order.  Uses params' R, dirs, l_ray, spectrum, nH, T,
 * y, kernel, precision and case_rule; the columns are traced (no stored
 * segments).  Synchronises `stream`.  Errors: as urchin_solve. */
URCHIN_API int urchin_tangent(const urchin_bvh* bvh, const urchin_solve_params* params, const double* x,
                              const double* v, double* E_out, double* dlnE_out, urchin_stream_t stream);

/* ---- Reverse mode (adjoints) -------------------------------------------
 * Each *_vjp call is the transpose of the forward call of the same name:
 * given the cotangent of the forward output it returns the cotangent of the
 * inputs.  Accumulating outputs (+=) are marked; the caller zeroes them. */

/* Transpose of Eq. colden: the columns are linear in x, tau = M x, so
 *   x_bar[j] += sum_{o,k} tau_bar[o*R + k] sigma_th (m_j/m_p) int W dt
 * over every ray (o, k) that crosses particle j (and its periodic images).
 * Arguments as urchin_trace_columns; tau_bar has tau_out's layout and type
 * (float for URCHIN_F32, double for URCHIN_F64); x_bar is device [n] double
 * in the original order, accumulated with atomics (the order of the
 * additions, hence the last bits, varies between runs).  Rays whose
 * tau_bar is zero are not traced.  Synchronises `stream`.  Errors: as
 * urchin_trace_columns. */
URCHIN_API int urchin_trace_columns_vjp(const urchin_bvh* bvh, const double* dirs, int R, double l_ray,
                                        const int32_t* origins, int64_t n_orig, int kernel, int precision,
                                        const void* tau_bar, double* x_bar, urchin_stream_t stream);

/* Transpose of Eq. gamma_shld, in double: with c_o = gamma_bar[o] / R,
 *   tau_bar_out[o*R + k] = -c_o sum_b w_b s_b exp(-s_b tau_ok)      (overwritten;
 *                          type of tau; may be NULL)
 *   w_bar[b]            += sum_{o,k} c_o exp(-s_b tau_ok)           (device [F]; may be NULL)
 * i.e. dL/dtau and dL/dw for the spectrum weights w (s held fixed).  One of
 * the outputs must be given.  Errors: ERR_ARG, ERR_NOMEM, ERR_CUDA. */
URCHIN_API int urchin_gamma_vjp(const void* tau, int precision, int64_t n_orig, int R,
                                const urchin_spectrum* sp, const double* gamma_bar, void* tau_bar_out,
                                double* w_bar, urchin_stream_t stream);

/* Transpose of urchin_equilibrium: gamma_bar_out[i] = x_bar[i] dx_i/dGamma_i,
 * dx/dGamma = x / (2 R x + Q) (implicit differentiation of the quadratic;
 * the case choice is held).  Arguments as urchin_equilibrium.  Errors: ERR_ARG,
 * ERR_CUDA. */
URCHIN_API int urchin_equilibrium_vjp(const double* gamma, const float* tau_eff, const double* nH,
                                      const double* T, int64_t n, int case_rule, double y,
                                      const double* x_bar, double* gamma_bar_out, urchin_stream_t stream);

/* Gradient of a loss L(x*) with respect to the spectrum weights w_b, where
 * x* is the converged state of urchin_solve (implicit function theorem at
 * the Sec. 4 fixed point; the paper has no derivatives, this is its
 * adjoint).  Inputs: the same params as the forward solve, with
 * params->state holding the state that solve wrote; x_star = its output;
 * x_bar = dL/dx* (device [n] double, original order).  With the cases and
 * the frozen set held, non-frozen particles satisfy x_a = E_a(Gamma_a(x, w))
 * and (unless params->warm_start) frozen ones x_f = E_f(Gamma_thin), with
 * Gamma_thin = sum_b w_b.  The call solves (I - J_u)^T nu = x_bar (.) x* for
 * the sweep-map Jacobian in ln x by restarted GMRES(params->gmres_m), to
 * relative residual params->tol in at most params->max_iter products (each
 * one transposed column pass: scatter traversal, or the stored segments
 * when params->segments allows), then
 *   w_bar[b] += dL/dw_b                                  (device [F], accumulated).
 * stats: iterations = products, max_rel_dx = final relative residual,
 * converged, traversals, rays.  Synchronises `stream`.  Errors: as
 * urchin_solve; ERR_NOT_CONVERGED when the residual target is not met
 * (w_bar then holds the gradient of the last iterate). */
URCHIN_API int urchin_solve_vjp(const urchin_bvh* bvh, const urchin_solve_params* params,
                                const double* x_star, const double* x_bar, double* w_bar,
                                urchin_solve_stats* stats, urchin_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* URCHIN_H */
