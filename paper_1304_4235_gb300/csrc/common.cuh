// Internal declarations shared by the translation units of liburchin.
// Nothing here is part of the public ABI (include/urchin.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>

#include "urchin.h"

namespace urchin {

// ---- error reporting ------------------------------------------------------
int set_error(int status, const char* fmt, ...);
void clear_error();

#define URCHIN_TRY_CUDA(call)                                                          \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            if (e_ == cudaErrorMemoryAllocation) {                                     \
                cudaGetLastError();                                                    \
                return ::urchin::set_error(URCHIN_ERR_NOMEM, "%s: out of device memory", \
                                           #call);                                     \
            }                                                                          \
            return ::urchin::set_error(URCHIN_ERR_CUDA, "%s failed: %s (%s:%d)", #call,    \
                                       cudaGetErrorString(e_), __FILE__, __LINE__);    \
        }                                                                              \
    } while (0)

#define URCHIN_TRY(expr)                 \
    do {                                 \
        int s_ = (expr);                 \
        if (s_ != URCHIN_OK) return s_;  \
    } while (0)

// ---- physical constants (SI-free, cgs) ------------------------------------
constexpr double kPi = 3.14159265358979323846;
// App. C1, Eq. sigma_ana: sigma_th = 2^9 pi/(3 e^4) alpha_fs pi a_0^2
double sigma_th_cm2();
constexpr double kRydbergEV = 13.605693122994;

// Truncated Gaussian constants of Eq. Gt in units of h: t = A h = 2 pi^(1/6),
// D = erf(t) - 2 t exp(-t^2)/sqrt(pi); chord prefactor sqrt(pi)/(2 t D).
struct GtConst {
    double t2;      // t^2
    double t;       // t
    double pref;    // sqrt(pi) / (2 t D)
};
GtConst gt_constants();

// ---- stream-ordered scratch ----------------------------------------------
// One cudaMallocAsync block released with cudaFreeAsync on the same stream.
struct Scratch {
    void* ptr = nullptr;
    cudaStream_t stream = nullptr;
    Scratch() = default;
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;
    ~Scratch() { release(); }
    int alloc(size_t bytes, cudaStream_t s);
    void release();
    template <typename T>
    T* at(size_t offset_bytes) const { return reinterpret_cast<T*>(static_cast<char*>(ptr) + offset_bytes); }
};

// Bump allocator used to carve one Scratch block into aligned arrays.
struct Layout {
    size_t bytes = 0;
    size_t take(size_t n) {
        size_t off = (bytes + 255) & ~size_t(255);
        bytes = off + n;
        return off;
    }
};

int grid_for(const void* kernel, int block, size_t smem, int* grid_out);

// The calling device's work-array pool (created on first use, keeps freed
// memory reserved), and the bytes it holds reserved but unused.
int library_pool(cudaMemPool_t* out);
size_t pool_idle_bytes();

// Check the launch just made and count it (urchin_kernel_launches).
int launched();

// ---- scans ----------------------------------------------------------------
// Exclusive prefix sum of n uint32 values (in may alias out).  `tmp` needs
// scan_tmp_bytes(n) bytes of device memory.
size_t scan_tmp_bytes(int64_t n);
int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, void* tmp,
                       uint32_t* total_dev, cudaStream_t s);

// Exclusive prefix sum of n uint32 counts into uint64 offsets.
size_t scan64_tmp_bytes(int64_t n);
int scan_counts_u64(const uint32_t* in, uint64_t* out, int64_t n, void* tmp, uint64_t* total_dev,
                    cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
size_t radix_tmp_bytes(int64_t n);
int radix_sort_pairs(uint32_t* keys, int32_t* vals, int64_t n, int bits, void* tmp,
                     cudaStream_t s);

// Stream compaction: out[m] = i for every i with flags[i] != 0, in order;
// *count_dev = m.  `tmp` needs compact_tmp_bytes(n).
size_t compact_tmp_bytes(int64_t n);
int compact_indices(const uint8_t* flags, int64_t n, int32_t* out, uint32_t* count_dev, void* tmp,
                    cudaStream_t s);

}  // namespace urchin

// ---- the BVH object --------------------------------------------------------
// Internal node layout (64 bytes, 4 float4), both children in one node:
//   n[0] = (left.lo.xyz, left.ref)    n[1] = (left.hi.xyz, left.count)
//   n[2] = (right.lo.xyz, right.ref)  n[3] = (right.hi.xyz, right.count)
// ref/count are int bit patterns: count == 0 -> ref is an internal node
// index; count > 0 -> leaf holding particles [ref, ref + count) in Morton
// order.  An empty child has lo > hi.  Node 0 is the root.
struct urchin_bvh {
    int64_t n = 0;
    int periodic = 0;
    double L = 0.0;
    double unit_cm = 1.0;
    float hmax = 0.f;
    float hgeo = 0.f;             // geometric mean of h
    float root_lo[3] = {0, 0, 0};
    float root_hi[3] = {0, 0, 0};
    int device = 0;
    int n_nodes = 0;
    float4* nodes = nullptr;      // [4 * n_nodes]
    float4* xyzh = nullptr;       // [n] Morton order
    float* A32 = nullptr;         // [n] sigma_th (m/m_p) (8/pi) / (h unit_cm)^2
    double* A64 = nullptr;        // [n]
    int32_t* perm = nullptr;      // [n] Morton slot -> original index
    int32_t* inv = nullptr;       // [n] original index -> Morton slot
    float2* ktab = nullptr;       // [kKTab + 1] full-chord M4 table
};

namespace urchin {

// Bits of the device status word shared by the kernels of one call.
constexpr unsigned kStStack = 1u;       // traversal stack overflow
constexpr unsigned kStOrigin = 2u;      // origin index out of range
constexpr unsigned kStNonfinite = 4u;   // non-finite or non-positive x
constexpr unsigned kStInput = 8u;       // n_H or T not finite and > 0
constexpr unsigned kStWarm = 16u;       // warm-start x outside (0, 1]
constexpr unsigned kStVisit = 32u;      // traversal visit limit (malformed tree)
constexpr unsigned kStSegment = 64u;    // stored-segment fill disagrees with its count

constexpr int kLeafMax = 32;      // subtrees with <= kLeafMax particles become leaves
constexpr int kSegPad = 8;        // stored rays are padded to a multiple of kSegPad segments (zero
                                  // values, particle 0) so the SpMV reads 8 segments per lane
constexpr int kKTab = 2048;       // intervals of the full-chord M4 table in t = b^2/h^2

// Full-chord M4 integral K(t) = int_{-c}^{c} shape(sqrt(t + u^2)) du, c = sqrt(1-t),
// tabulated at t_i = i / kKTab as (K(t_i), dK/dt(t_i) / kKTab), host side.
void m4_full_table(float2* out /* [kKTab + 1] */);
constexpr int kChunkEntries = 32;   // MODE_CHUNK: segment entries per chunk
constexpr int kStackMax = 64;     // traversal stack (tree depth <= 62 for 30-bit codes)

// Column tracing shared by urchin_trace_columns and urchin_solve.
struct TraceJob {
    const urchin_bvh* bvh;
    const float* w32;             // [n] A_j x_j, Morton order (F32)
    const double* w64;            // [n] (F64)
    const double* dirs_dev;       // [R*3]
    int R;
    double l_ray;
    const int32_t* items;         // [n_items] Morton origin per item, NULL = identity
    int64_t n_items;
    int64_t row_stride;           // out index = row * row_stride + k * k_stride
    int64_t k_stride;
    const int32_t* out_row;       // [n_items] output row per item, NULL = item index
    void* out;                    // float or double
    int kernel;
    int precision;
    unsigned int* counter;        // one device uint (work queue), zeroed here
    unsigned int* status;         // one device uint: error flags (may be NULL)
    unsigned long long* hits;     // chord evaluations (may be NULL)
    int mode;                     // 0: columns, 1: count hits per ray, 2: fill segments (+ columns),
                                  // 3: transpose (scatter coef * A_j * chord into xbar),
                                  // 4: columns + counts + segments in linked chunks (FP32, no near/far)
    uint32_t* counts;             // mode 1 (and mode 0 when not NULL): [R * n], index k * n + the origin's
                                  //    Morton slot: hits rounded up to a multiple of kSegPad
    const uint64_t* row_ptr;      // mode 2: [R * n + 1] offsets of each ray's segments (same index)
    int32_t* seg_col;             // mode 2: Morton index of the particle per segment, or NULL:
    uint16_t* seg_lo;             //    its low 16 bits and
    uint8_t* seg_hi;              //    its high 8 bits (FP32 segments, every index below 2^24)
    void* seg_val;                // mode 2: A_j * chord integral per segment (precision's type)
    const void* coef;             // mode 3: per-ray coefficient (precision's type), indexed like out
    double* xbar;                 // mode 3: [n] Morton order, accumulated with atomics
    const int32_t* order;         // [R * n_items] or NULL: order[k * n_items + i] = the item that the
                                  // i-th lane slot of direction k traces (ray_order)
    int near_far;                 // 1: split near / far particles (Sec. 3.3.3): out (and the stored
                                  //    segments, and the hit counts) take far particles only
    void* out_near;               // near_far: hydrogen column (x = 1) of the near particles, in tau units,
                                  //    at [origin's Morton slot + k * near_k_stride] (modes 0 and 2)
    int64_t near_k_stride;
    uint32_t* chunk_head;         // mode 4: [R * n] first chunk of each ray (index k * n + slot)
    uint32_t* chunk_next;         // mode 4: [chunk_cap] next chunk of the same ray
    unsigned long long* chunk_counter;   // mode 4: chunks handed out, zeroed by the caller; above
                                  //    chunk_cap some rays' lists are incomplete
    unsigned long long chunk_cap; // mode 4: chunks that chunk_seg holds (32 entries each)
    int2* chunk_seg;              // mode 4: [chunk_cap * 32] entries (particle index, value bits), a
                                  //    ray's entries padded with (0, 0) to a multiple of kSegPad
};
int launch_trace(const TraceJob& job, cudaStream_t s);

// Per-direction traversal order of the items: for each direction k the
// origins sorted by a 63-bit Morton code in the frame (e1, e2, d_k) with the
// axis along d_k compressed by a factor E, so that 32 consecutive origins
// form a beam along the ray direction, about E times longer than wide.
// Rays share their sphere crossings when the beam is narrow against h and
// short against l_ray, so E = l_ray / (2 h_geo), h_geo the geometric mean of
// h, clamped to [1, 64].  Measured traversal of all rays: 262144-particle
// halo (l_ray / 2h_geo ~ 20) E = 16: 43 ms, 4: 51, 1: 58; the 256^3
// log-normal box (~2) E = 16: 1.06 s, 4: 0.90, 1: 0.87 (30-bit keys, E = 16:
// 1.34 s).  On the 4096-particle lattice the order costs more than it saves
// (sort launches, and 9.1 instead of 7.4 sphere tests per hit), so short
// lists keep item order.  order needs R * n_items int32; tmp needs
// ray_order_tmp_bytes(n_items).
constexpr int64_t kRayOrderMinItems = 16384;
double ray_order_elongation(const urchin_bvh* bvh, double l_ray);
size_t ray_order_tmp_bytes(int64_t n_items);
int ray_order(const urchin_bvh* bvh, const int32_t* items, int64_t n_items, const double* dirs_host, int R,
              double l_ray, int32_t* order, void* tmp, cudaStream_t s);

// w_bar[b] += sum_r sg[r] exp(lc[r] - s_b tau[r]) over n_rays rays (tau in
// the precision's type; the coefficient of ray r is sg[r] exp(lc[r]))
int launch_wbar(const void* tau, int precision, int64_t n_rays, const double* lc, const double* sg, const double* s,
                int F, double* w_bar, cudaStream_t st);

// A spectrum with helium cross sections (urchin_gamma_he, plain urchin_solve)
inline bool spectrum_has_he(const urchin_spectrum* sp) { return sp && (sp->s_he1 || sp->s_he2); }

// Table of ln sum_b w_b exp(-s_b tau) on u = ln(1 + tau) for the
// polychromatic slab (spectral_device.cuh, SpecTable): kSpecTab intervals
// up to tau = kSpecTauMax, in double and (relative to Gamma_thin) in float.
// buf needs spec_table_bytes() of device memory; synchronises st.
constexpr int kSpecTab = 4096;
constexpr double kSpecTauMax = 1e7;
struct SpecTable;
size_t spec_table_bytes();
int build_spec_table(const double* s, const double* w, int F, void* buf, SpecTable* out, cudaStream_t st);

// Origins (original particle indices) to Morton slots: items[o] =
// inv[origins[o]]; an index outside [0, n) sets kStOrigin in *status.
int launch_map_origins(const urchin_bvh* bvh, const int32_t* origins, int64_t n_orig, int32_t* items,
                       unsigned* status, cudaStream_t s);

// w = A * x gathered into Morton order: w[s] = A[s] * x[perm[s]]
int launch_weights(const urchin_bvh* bvh, const double* x_orig, float* w32, double* w64,
                   cudaStream_t s);

// Spectral rate per origin (Eq. gamma_shld).
struct GammaJob {
    const void* tau;              // tau index = row * row_stride + k * k_stride
    int precision;
    int64_t n_rows;
    int R;
    int64_t row_stride, k_stride;
    const double* s;              // [F] device
    const double* w;              // [F] device
    int F;
    double* gamma_out;            // [n_rows]
    float* tau_eff_out;           // [n_rows] or NULL
};
int launch_gamma(const GammaJob& job, cudaStream_t s);

// Rates of App. C3 (Hui & Gnedin 1997) on the device, per particle.
int launch_equilibrium(const double* gamma, const float* tau_eff, const double* nH,
                       const double* T, int64_t n, int case_rule, double y, double* x_out,
                       cudaStream_t s);

}  // namespace urchin
