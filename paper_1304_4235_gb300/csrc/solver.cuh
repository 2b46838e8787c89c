// Solver state shared by the plain (Jacobi) and Newton-Krylov drivers.
#pragma once

#include <cstring>
#include <vector>

#include "common.cuh"
#include "linalg.cuh"
#include "spectral_device.cuh"

namespace urchin {

struct SweepArgs {
    const void* tau;           // float or double per precision
    int precision;
    int64_t k_stride;          // tau[row + k * k_stride]
    const int32_t* items;      // Morton particle per row (NULL = identity)
    int64_t n_items;
    int R;
    const double* s;
    const double* w;
    int F;
    double* x;                 // Morton order
    const double* A64;
    float* w32;
    double* w64;
    float* xs32;               // optional: x as float (stored-segment sweeps)
    double* xs64;
    const double* nH;
    const double* aA;
    const double* aB;
    const double* gc;
    double y;
    int case_rule;
    double tau_skip;
    int sweep0;
    uint8_t* active;           // written in sweep 0
    uint8_t* latch;            // case B latched (CASE_AUTO), Morton order
    int latch_frozen;          // 1: cases from the latch only, latch not written;
                               //    count particles that would switch (n_switch)
    unsigned long long* n_switch;
    unsigned long long* maxrel;
    unsigned long long* n_above;   // count of updated particles with |dx|/x >= tol
    double tol;
    unsigned* status;
    double* gamma_out;         // [n_items] optional
    float* tau_eff_out;        // [n_items] optional
    int near_far;              // Sec. 3.3.3 split: tau holds the far columns; the near
    const void* tau_near;      //   columns (x = 1) are at tau_near[i + k * near_k_stride]
    int64_t near_k_stride;     //   (i the Morton slot) and enter through the slab solution
    SpecTable poly;            // near_far == URCHIN_SLAB_SPECTRUM: ln Gamma_spec(tau) table
    int he;                    // helium: fixed columns tau_he1/2[i + k * near_k_stride] (Morton
    const void* tau_he1;       //   slot i) attenuate the bins with the cross sections s_he1/2
    const void* tau_he2;
    const double* s_he1;
    const double* s_he2;
    int want_tangent;          // Newton: keep x, emit E and tangent factors
    double* ctan;              // [n_items * R] (k-major, stride k_stride)
    double* xeq_out;           // [n_items]
};

int launch_sweep(const SweepArgs& A, cudaStream_t s);

struct Solver {
    const urchin_bvh* bvh = nullptr;
    urchin_solve_params P{};
    cudaStream_t s = nullptr;
    int64_t n = 0;
    int64_t n_act = 0;
    int64_t last_above = 0;
    bool f64 = false;
    double gthin = 0.0;
    urchin_solve_stats stats{};
    Scratch scr;
    unsigned long long* misc = nullptr;
    unsigned* counter = nullptr;
    unsigned* status = nullptr;
    double* dirs = nullptr;
    double* x = nullptr;
    double* nH = nullptr;
    double* aA = nullptr;
    double* aB = nullptr;
    double* gc = nullptr;
    float* w32 = nullptr;
    double* w64 = nullptr;
    uint8_t* active = nullptr;
    uint8_t* latch = nullptr;
    int32_t* list = nullptr;
    void* tau = nullptr;
    void* tau_near = nullptr;                    // near/far: [R * n] near columns, Morton slot + k n
    SpecTable poly{nullptr, 0, 0.0, 0.0, nullptr, 0.0};   // near/far with the polychromatic slab
    void* tau_he1 = nullptr;                     // helium: [R * n] fixed columns, Morton slot + k n
    void* tau_he2 = nullptr;
    int he_columns();
    void* comp_tmp = nullptr;
    unsigned long long* hits = nullptr;          // misc[3..5], counted when P.profile
    std::vector<cudaEvent_t> events;             // start/stop pairs of each timed launch
    std::vector<int> event_kind;                 // 0 traversal, 1 stored-segment columns, 2 sweep
    int begin_timed(int kind, cudaEvent_t* stop);
    int end_timed(cudaEvent_t stop);
    // stored segments
    bool stored = false;
    float* xs32 = nullptr;                       // x in the precision of the columns (Morton)
    double* xs64 = nullptr;
    uint32_t* counts = nullptr;
    uint64_t* row_ptr = nullptr;
    void* scan_tmp = nullptr;
    int32_t* seg_col = nullptr;                  // particle index per segment, or NULL when
    uint16_t* seg_lo = nullptr;                  // split into 16 + 8 bits (FP32 segments,
    uint8_t* seg_hi = nullptr;                   // n <= 2^24: 7 bytes per segment instead of 8)
    void* seg_val = nullptr;
    Scratch seg;
    // segment lists stored by the first sweep's traversal in linked chunks
    // (SEG_AUTO, FP32): later sweeps read them instead of tracing again
    bool chunked = false;
    bool compact_tried = false;
    Scratch chunk_mem;
    uint32_t* chunk_head = nullptr;
    uint32_t* chunk_next = nullptr;
    int2* chunk_seg = nullptr;
    int trace_chunked(TraceJob& job);
    int compact_chunks();
    void spmv_lists(SpmvArgs& A) const;
    // per-direction traversal orders, cached per item list (any permutation
    // is correct; a stale one only costs coherence)
    Scratch ord;
    int32_t* ord_base = nullptr;
    void* ord_tmp = nullptr;
    int64_t ord_cap = 0, ord_used = 0;
    struct OrderEntry {
        const int32_t* items;
        int64_t n;
        int32_t* order;
    };
    std::vector<OrderEntry> orders;
    int order_for(const int32_t* items, int64_t n_items, const int32_t** out);
    int derive_list_order(const int32_t* full);
    void items_changed()
    {
        orders.clear();
        ord_used = 0;
    }
    // Newton-Krylov
    Scratch nk;

    ~Solver();
    int columns(const int32_t* items, int64_t n_items, int sweep0, bool build = false);
    bool counts_ready = false;                   // counts[] hold every ray's hits (rows by Morton slot)
    bool counted_all = false;                    // ... counted over all n particles
    bool store_declined = false;                 // SEG_AUTO: the lists did not fit
    int linear_columns(const int32_t* items, int64_t n_items, const float* z32, const double* z64,
                       float* wz32, double* wz64);
    int timed_trace(TraceJob& job);
    int timed_sweep(const SweepArgs& A, cudaStream_t st);
    int count_spmv(const int32_t* items, int64_t n_items);
    int64_t active_nnz = -1;
    int evaluate(int frozen, double* V0, double* E, double* ctan, double* dtmp, double* hdev, double* maxrel,
                 double* norm, int64_t* switches, int tangent = 1);

    int init(const urchin_bvh* bvh, const urchin_solve_params* P, double* x_inout, cudaStream_t s);
    int trace(const int32_t* items, int64_t n_items, const float* tw32, const double* tw64);
    SweepArgs sweep_args(const int32_t* items, int64_t n_items, int sweep0);
    int read_scalars(double* maxrel, unsigned* status);
    void record(double maxrel);
    int first_sweep();
    int order_by_density();
    std::vector<int64_t> block_lo;               // block b = list[block_lo[b], block_lo[b+1])
    int plain();
    int plain_sweeps(double stop_fraction);
    int newton();
    int run() { return P.method == URCHIN_METHOD_NEWTON ? newton() : plain(); }
    int finish(double* x_inout);
    int tangent(const double* v_orig, double* E_orig, double* dlnE_orig);
    // reverse mode at a converged state (urchin_solve_vjp)
    int adjoint(const uint8_t* state_orig, const double* xbar_orig, int cold_start, double* w_bar);
    int transpose_columns(const void* coef, double* z);   // z[j] += sum_rays coef A_j K (Morton, all j)
};

}  // namespace urchin
