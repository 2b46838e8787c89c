// Stored-segment columns and dense vector kernels (see linalg.cu).
#pragma once

#include <cmath>
#include <vector>

#include "common.cuh"

namespace urchin {

struct SpmvArgs {
    const uint64_t* row_ptr;     // [R * n_rows_per_k + 1], multiples of kSegPad
    const int32_t* col;          // [nnz] Morton particle index (padding: 0), or NULL:
    const uint16_t* lo;          //   its low 16 bits
    const uint8_t* hi;           //   and high 8 bits (FP32 only)
    const void* val;             // [nnz] A_j * chord integral (float or double; padding: 0)
    const void* xvec;            // [n] vector the columns are linear in (Morton order, same type)
    const int32_t* items;        // [n_items] Morton particle of each evaluated ray origin (NULL = identity)
    int64_t n_items;
    int64_t n_rows_per_k;        // particles in the stored layout
    int R;
    int precision;
    void* out;                   // [R * n_items], index k * n_items + item
    // FP32 lists in linked chunks of kChunkEntries (the traversal's MODE_CHUNK)
    // instead of rows: row_ptr, col, lo, hi and val are then unused
    const uint32_t* chunk_head;  // [R * n_rows_per_k] first chunk of each row, or NULL: row-major lists
    const uint32_t* chunk_next;  // the next chunk of the same row
    const uint32_t* row_cnt;     // [R * n_rows_per_k] entries of each row (padded with zero values)
    const int2* chunk_seg;       // [chunks * kChunkEntries] entries (particle index, value bits)
};
int launch_spmv(const SpmvArgs& A, cudaStream_t s);

// Chunked lists (MODE_CHUNK) copied into rows: row r's entries to
// [row_ptr[r], row_ptr[r] + cnt[r]) as a particle index (int32 col, or 16 + 8
// bits in lo / hi) and a value.  Rows with cnt 0 are skipped.
struct ChunkCompactArgs {
    const uint32_t* head;
    const uint32_t* next;
    const int2* seg;
    const uint32_t* cnt;         // [rows]
    const uint64_t* row_ptr;     // [rows + 1]
    int64_t rows;
    int32_t* col;                // or NULL:
    uint16_t* lo;
    uint8_t* hi;
    float* val;
};
int launch_chunk_compact(const ChunkCompactArgs& A, cudaStream_t s);

// Transpose of the stored columns: z[col_e] += coef[k * n_items + a] * val_e
// over the segments of every ray (k, items[a]); z is double [n] (Morton),
// accumulated with atomics; coef has the precision's type.
struct SpmvTArgs {
    const uint64_t* row_ptr;
    const int32_t* col;          // as SpmvArgs
    const uint16_t* lo;
    const uint8_t* hi;
    const void* val;
    const void* coef;            // [R * n_items]
    const int32_t* items;        // NULL = identity
    int64_t n_items;
    int64_t n_rows_per_k;
    int R;
    int precision;
    double* z;
};
int launch_spmv_t(const SpmvTArgs& A, cudaStream_t s);

// Restarted GMRES(m) for A v = b on device vectors of length n, from v = 0.
// matvec(in, out) computes out = A in.  Stops when ||b - A v|| <= rtol ||b||
// or after max_matvec products.  work needs gmres_work_bytes(n, m).
struct GmresResult {
    int matvecs = 0;
    double rel_residual = 0.0;
};
size_t gmres_work_bytes(int64_t n, int m);
template <typename MatVec>
int gmres_solve(MatVec&& matvec, const double* b, double* v, int64_t n, int m, double rtol, int max_matvec,
                void* work, GmresResult* res, cudaStream_t s);

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

inline size_t gmres_work_bytes(int64_t n, int m)
{
    Layout lay;
    lay.take(sizeof(double) * (size_t)(m + 1) * (size_t)n);
    lay.take(sizeof(double) * (size_t)n);
    lay.take(dots_tmp_bytes(m + 1));
    lay.take(sizeof(double) * (size_t)(m + 2));
    return lay.bytes;
}

namespace detail {
inline int host_dots(const double* V, int64_t ld, int count, const double* w, int64_t n, double* tmp, double* hdev,
                     double* out, cudaStream_t s)
{
    URCHIN_TRY(launch_dots(V, ld, count, w, n, tmp, hdev, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(out, hdev, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    return URCHIN_OK;
}
}  // namespace detail

template <typename MatVec>
int gmres_solve(MatVec&& matvec, const double* b, double* v, int64_t n, int m, double rtol, int max_matvec,
                void* work, GmresResult* res, cudaStream_t s)
{
    Layout lay;
    const size_t o_V = lay.take(sizeof(double) * (size_t)(m + 1) * (size_t)n);
    const size_t o_r = lay.take(sizeof(double) * (size_t)n);
    const size_t o_t = lay.take(dots_tmp_bytes(m + 1));
    const size_t o_h = lay.take(sizeof(double) * (size_t)(m + 2));
    char* base = static_cast<char*>(work);
    double* V = reinterpret_cast<double*>(base + o_V);
    double* r = reinterpret_cast<double*>(base + o_r);
    double* tmp = reinterpret_cast<double*>(base + o_t);
    double* hdev = reinterpret_cast<double*>(base + o_h);
    *res = GmresResult{};
    URCHIN_TRY_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * (size_t)n, s));
    double bb = 0.0;
    URCHIN_TRY(detail::host_dots(b, n, 1, b, n, tmp, hdev, &bb, s));
    const double bnorm = std::sqrt(std::max(bb, 0.0));
    if (!(bnorm > 0.0)) return URCHIN_OK;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(r, b, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    double beta = bnorm;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hcol(m + 2), y(m), hh(m + 1);
    for (;;) {
        res->rel_residual = beta / bnorm;
        if (beta <= rtol * bnorm || res->matvecs >= max_matvec) break;
        URCHIN_TRY_CUDA(cudaMemcpyAsync(V, r, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        URCHIN_TRY(launch_axpby(0.0, V, 1.0 / beta, V, n, s));
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m && res->matvecs < max_matvec; ++j) {
            double* vj = V + (size_t)j * n;
            double* w = V + (size_t)(j + 1) * n;
            URCHIN_TRY(matvec(vj, w));
            res->matvecs += 1;
            std::fill(hcol.begin(), hcol.end(), 0.0);
            for (int pass = 0; pass < 2; ++pass) {     // classical Gram-Schmidt, twice
                URCHIN_TRY(detail::host_dots(V, n, j + 1, w, n, tmp, hdev, hh.data(), s));
                URCHIN_TRY(launch_subtract(w, V, n, j + 1, hdev, n, s));
                for (int i = 0; i <= j; ++i) hcol[i] += hh[i];
            }
            double hn2 = 0.0;
            URCHIN_TRY(detail::host_dots(w, n, 1, w, n, tmp, hdev, &hn2, s));
            const double hn = std::sqrt(std::max(hn2, 0.0));
            hcol[j + 1] = hn;
            if (hn > 0.0) URCHIN_TRY(launch_axpby(0.0, w, 1.0 / hn, w, n, s));
            for (int i = 0; i < j; ++i) {              // earlier Givens rotations
                const double a = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
                hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
                hcol[i] = a;
            }
            const double rr = std::hypot(hcol[j], hcol[j + 1]);
            cs[j] = rr > 0.0 ? hcol[j] / rr : 1.0;
            sn[j] = rr > 0.0 ? hcol[j + 1] / rr : 0.0;
            hcol[j] = rr;
            hcol[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
            kdim = j + 1;
            if (std::fabs(g[j + 1]) <= rtol * bnorm || hn == 0.0) break;
        }
        if (kdim == 0) break;
        for (int i = kdim - 1; i >= 0; --i) {          // y = H^-1 g, v += V y
            double acc = g[i];
            for (int k = i + 1; k < kdim; ++k) acc -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0.0 ? acc / H[(size_t)i * m + i] : 0.0;
        }
        for (int i = 0; i < kdim; ++i) y[i] = -y[i];
        URCHIN_TRY_CUDA(cudaMemcpyAsync(hdev, y.data(), sizeof(double) * kdim, cudaMemcpyHostToDevice, s));
        URCHIN_TRY(launch_subtract(v, V, n, kdim, hdev, n, s));
        // true residual r = b - A v for the restart and the stop test
        URCHIN_TRY(matvec(v, r));
        res->matvecs += 1;
        URCHIN_TRY(launch_axpby(1.0, b, -1.0, r, n, s));
        double rr2 = 0.0;
        URCHIN_TRY(detail::host_dots(r, n, 1, r, n, tmp, hdev, &rr2, s));
        beta = std::sqrt(std::max(rr2, 0.0));
    }
    return URCHIN_OK;
}

}  // namespace urchin
