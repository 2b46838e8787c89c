// Stored-segment columns and dense vector kernels (see linalg.cu).
#pragma once

#include "common.cuh"

namespace urchin {

struct SpmvArgs {
    const uint64_t* row_ptr;     // [R * n_rows_per_k + 1]
    const int32_t* col;          // [nnz] Morton particle index
    const void* val;             // [nnz] A_j * chord integral (float or double)
    const void* xvec;            // [n] vector the columns are linear in (Morton order, same type)
    const int32_t* items;        // [n_items] Morton particle of each evaluated ray origin (NULL = identity)
    int64_t n_items;
    int64_t n_rows_per_k;        // particles in the stored layout
    int R;
    int precision;
    void* out;                   // [R * n_items], index k * n_items + item
};
int launch_spmv(const SpmvArgs& A, cudaStream_t s);

// acc += number of segments of the rays (k, items[a]) (profiling)
int launch_row_nnz(const uint64_t* row_ptr, const int32_t* items, int64_t n_items, int64_t n_rows_per_k, int R,
                   unsigned long long* acc, cudaStream_t s);

size_t dots_tmp_bytes(int count);
// out[i] = V_i . w for i < count (V row-major with leading dimension ld),
// deterministic two-pass reduction; tmp needs dots_tmp_bytes(count).
int launch_dots(const double* V, int64_t ld, int count, const double* w, int64_t n, double* tmp, double* out,
                cudaStream_t s);
int launch_subtract(double* w, const double* V, int64_t ld, int count, const double* coef, int64_t n,
                    cudaStream_t s);
int launch_axpby(double alpha, const double* x, double beta, double* y, int64_t n, cudaStream_t s);

}  // namespace urchin
