// Stored-segment columns (sparse matrix-vector product) and the small dense
// vector kernels of the Newton-Krylov solver.
//
// With the per-ray segment lists stored once (column j, value A_j * chord
// integral), a sweep's columns are tau_r = sum_e val_e x_{col_e}: a stream
// over the segment arrays (7 bytes per segment in FP32: value + 24-bit
// particle index split into 16 + 8 bits) with a gather of x from L2.  Rows
// are indexed k * n + particle (direction-major), as written by the fill
// traversal.
#include <algorithm>

#include "linalg.cuh"

namespace urchin {

namespace {

constexpr int kSpmvThreads = 256;

// One warp per ray; lanes stride the ray's segments four at a time (int32
// indices: FP64, and FP32 beyond 2^24 particles).
template <typename Real>
__global__ void __launch_bounds__(kSpmvThreads) k_spmv(SpmvArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kSpmvThreads / 32);
    const int64_t total = (int64_t)A.R * A.n_items;
    const Real* val = static_cast<const Real*>(A.val);
    const Real* xv = static_cast<const Real*>(A.xvec);
    Real* out = static_cast<Real*>(A.out);
    for (int64_t w = (int64_t)blockIdx.x * (kSpmvThreads / 32) + (threadIdx.x >> 5); w < total; w += warps) {
        const int64_t k = w / A.n_items;
        const int64_t a = w - k * A.n_items;
        const int64_t i = A.items ? (int64_t)A.items[a] : a;
        const int64_t row = k * A.n_rows_per_k + i;
        const int64_t beg = (int64_t)A.row_ptr[row], end = (int64_t)A.row_ptr[row + 1];
        Real s = Real(0), c = Real(0);
        int64_t e = beg + lane;
        for (; e + 96 < end; e += 128) {
            const int32_t j0 = __ldcs(A.col + e), j1 = __ldcs(A.col + e + 32);
            const int32_t j2 = __ldcs(A.col + e + 64), j3 = __ldcs(A.col + e + 96);
            const Real v0 = __ldcs(val + e), v1 = __ldcs(val + e + 32);
            const Real v2 = __ldcs(val + e + 64), v3 = __ldcs(val + e + 96);
            const Real t = (v0 * __ldg(xv + j0) + v1 * __ldg(xv + j1)) + (v2 * __ldg(xv + j2) + v3 * __ldg(xv + j3));
            const Real y = t - c;
            const Real u = s + y;
            c = (u - s) - y;
            s = u;
        }
        for (; e < end; e += 32) {
            const Real t = __ldcs(val + e) * __ldg(xv + __ldcs(A.col + e));
            const Real y = t - c;
            const Real u = s + y;
            c = (u - s) - y;
            s = u;
        }
        s -= c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[a + k * A.n_items] = s;
    }
}

// FP32 with the split index (every particle index below 2^24): rays padded
// to a multiple of 8 segments, each lane takes 8 consecutive segments with two
// 16-byte value loads, one 16-byte load of the eight low halves and one
// 8-byte load of the eight high bytes of the indices.  Measured on the
// 262144-particle halo, ms per sweep: int32 indices with strided 4-byte loads
// 2.72, with 16-byte loads of 4 segments per lane 2.55-2.62; split indices
// with strided loads 3.13, with 4 segments per lane 2.64, with 8 segments per
// lane (this loop: as many load requests as the int32 16-byte loop, 7 bytes
// per segment instead of 8) 2.47.
__global__ void __launch_bounds__(kSpmvThreads) k_spmv8(SpmvArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kSpmvThreads / 32);
    const int64_t total = (int64_t)A.R * A.n_items;
    const float* val = static_cast<const float*>(A.val);
    const float* xv = static_cast<const float*>(A.xvec);
    float* out = static_cast<float*>(A.out);
    for (int64_t w = (int64_t)blockIdx.x * (kSpmvThreads / 32) + (threadIdx.x >> 5); w < total; w += warps) {
        const int64_t k = w / A.n_items;
        const int64_t a = w - k * A.n_items;
        const int64_t i = A.items ? (int64_t)A.items[a] : a;
        const int64_t row = k * A.n_rows_per_k + i;
        const int64_t beg = (int64_t)A.row_ptr[row], end = (int64_t)A.row_ptr[row + 1];
        float s = 0.f, c = 0.f;
        for (int64_t e = beg + 8 * lane; e < end; e += 256) {
            const float4 v0 = __ldcs(reinterpret_cast<const float4*>(val + e));
            const float4 v1 = __ldcs(reinterpret_cast<const float4*>(val + e + 4));
            const uint4 l = __ldcs(reinterpret_cast<const uint4*>(A.lo + e));
            const uint2 h = __ldcs(reinterpret_cast<const uint2*>(A.hi + e));
            const int j0 = (int)((l.x & 0xffffu) | ((h.x & 0xffu) << 16));
            const int j1 = (int)((l.x >> 16) | ((h.x & 0xff00u) << 8));
            const int j2 = (int)((l.y & 0xffffu) | (h.x & 0xff0000u));
            const int j3 = (int)((l.y >> 16) | ((h.x >> 24) << 16));
            const int j4 = (int)((l.z & 0xffffu) | ((h.y & 0xffu) << 16));
            const int j5 = (int)((l.z >> 16) | ((h.y & 0xff00u) << 8));
            const int j6 = (int)((l.w & 0xffffu) | (h.y & 0xff0000u));
            const int j7 = (int)((l.w >> 16) | ((h.y >> 24) << 16));
            const float t = ((v0.x * __ldg(xv + j0) + v0.y * __ldg(xv + j1)) + (v0.z * __ldg(xv + j2) + v0.w * __ldg(xv + j3))) +
                            ((v1.x * __ldg(xv + j4) + v1.y * __ldg(xv + j5)) + (v1.z * __ldg(xv + j6) + v1.w * __ldg(xv + j7)));
            const float y = t - c;
            const float u = s + y;
            c = (u - s) - y;
            s = u;
        }
        s -= c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[a + k * A.n_items] = s;
    }
}

// FP32 columns from chunked lists: four rays per warp, eight lanes per ray
// and four entries per lane in each chunk of kChunkEntries (32), each group
// following its own row's links, so that a warp keeps four chains of
// dependent loads in flight; the next link is read before the chunk's entries.
constexpr int kChunkLanes = 8;
__global__ void __launch_bounds__(kSpmvThreads) k_spmv_chunk(SpmvArgs A)
{
    const int lane = threadIdx.x & 31;
    const int sub = lane & (kChunkLanes - 1);
    const int64_t groups = (int64_t)gridDim.x * (kSpmvThreads / kChunkLanes);
    const int64_t total = (int64_t)A.R * A.n_items;
    const float* xv = static_cast<const float*>(A.xvec);
    float* out = static_cast<float*>(A.out);
    // every lane of the warp loops alike (the group count per warp is fixed)
    const int64_t first = ((int64_t)blockIdx.x * kSpmvThreads + threadIdx.x) / kChunkLanes;
    for (int64_t w0 = first - (lane / kChunkLanes); w0 < total; w0 += groups) {
        const int64_t w = w0 + lane / kChunkLanes;
        uint32_t cnt = 0, ch = 0;
        int64_t a = 0, k = 0;
        if (w < total) {
            k = w / A.n_items;
            a = w - k * A.n_items;
            const int64_t i = A.items ? (int64_t)A.items[a] : a;
            const int64_t row = k * A.n_rows_per_k + i;
            cnt = A.row_cnt[row];
            ch = cnt ? A.chunk_head[row] : 0u;
        }
        float s = 0.f, c = 0.f;
        for (uint32_t done = 0; done < cnt; done += kChunkEntries) {
            const uint32_t nxt = done + kChunkEntries < cnt ? __ldg(A.chunk_next + ch) : 0u;
            const int4* q4 = reinterpret_cast<const int4*>(A.chunk_seg + (int64_t)ch * kChunkEntries + 4 * sub);
            const uint32_t at = done + 4u * (uint32_t)sub;
            if (at < cnt) {            // rows hold whole multiples of kSegPad (8) entries
                const int4 p = __ldcs(q4), r = __ldcs(q4 + 1);
                const float t = (__int_as_float(p.y) * __ldg(xv + p.x) + __int_as_float(p.w) * __ldg(xv + p.z)) +
                                (__int_as_float(r.y) * __ldg(xv + r.x) + __int_as_float(r.w) * __ldg(xv + r.z));
                const float y = t - c;
                const float u = s + y;
                c = (u - s) - y;
                s = u;
            }
            ch = nxt;
        }
        s -= c;
#pragma unroll
        for (int o = kChunkLanes / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sub == 0 && w < total) out[a + k * A.n_items] = s;
    }
}

// One warp per row: the row's chunks in order, one entry per lane.
__global__ void __launch_bounds__(kSpmvThreads) k_chunk_compact(ChunkCompactArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kSpmvThreads / 32);
    for (int64_t r = (int64_t)blockIdx.x * (kSpmvThreads / 32) + (threadIdx.x >> 5); r < A.rows; r += warps) {
        const uint32_t cnt = A.cnt[r];
        if (cnt == 0) continue;
        const uint64_t base = A.row_ptr[r];
        uint32_t ch = A.head[r];
        for (uint32_t done = 0; done < cnt; done += kChunkEntries) {
            const uint32_t nxt = done + kChunkEntries < cnt ? __ldg(A.next + ch) : 0u;
            if (done + (uint32_t)lane < cnt) {
                const int2 q = __ldcs(A.seg + (int64_t)ch * kChunkEntries + lane);
                const uint64_t pos = base + done + (uint32_t)lane;
                if (A.col) {
                    A.col[pos] = q.x;
                } else {
                    A.lo[pos] = (uint16_t)((unsigned)q.x & 0xffffu);
                    A.hi[pos] = (uint8_t)(((unsigned)q.x >> 16) & 0xffu);
                }
                A.val[pos] = __int_as_float(q.y);
            }
            ch = nxt;
        }
    }
}

// One warp per ray: the ray's coefficient times each stored segment value is
// added to z at the segment's particle.
template <typename Real>
__global__ void __launch_bounds__(kSpmvThreads) k_spmv_t(SpmvTArgs A)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (kSpmvThreads / 32);
    const int64_t total = (int64_t)A.R * A.n_items;
    const Real* val = static_cast<const Real*>(A.val);
    const Real* coef = static_cast<const Real*>(A.coef);
    for (int64_t w = (int64_t)blockIdx.x * (kSpmvThreads / 32) + (threadIdx.x >> 5); w < total; w += warps) {
        const Real c = coef[w];
        if (c == Real(0)) continue;
        const int64_t k = w / A.n_items;
        const int64_t a = w - k * A.n_items;
        const int64_t i = A.items ? (int64_t)A.items[a] : a;
        const int64_t row = k * A.n_rows_per_k + i;
        const int64_t beg = (int64_t)A.row_ptr[row], end = (int64_t)A.row_ptr[row + 1];
        for (int64_t e = beg + lane; e < end; e += 32) {
            const Real v = __ldcs(val + e);
            if (v != Real(0)) {   // padding is zero
                const int32_t j = A.col ? __ldcs(A.col + e) : (int32_t)__ldcs(A.lo + e) | ((int32_t)__ldcs(A.hi + e) << 16);
                atomicAdd(A.z + j, (double)(c * v));
            }
        }
    }
}

// partial[i * nb + b] = sum over block b's share of V_i . w
__global__ void k_dots(const double* __restrict__ V, int64_t ld, int count, const double* __restrict__ w,
                       int64_t n, double* partial)
{
    __shared__ double red[8];
    const int i = blockIdx.y;
    const double* v = V + (int64_t)i * ld;
    double acc = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        acc += v[t] * w[t];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        partial[(int64_t)i * gridDim.x + blockIdx.x] = t;
    }
    (void)count;
}

__global__ void k_dots_reduce(const double* partial, int nb, int count, double* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += partial[(int64_t)i * nb + b];
    out[i] = t;
}

// w -= sum_i coef[i] V_i
__global__ void k_subtract(double* __restrict__ w, const double* __restrict__ V, int64_t ld, int count,
                           const double* __restrict__ coef, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[t];
        for (int i = 0; i < count; ++i) acc -= coef[i] * V[(int64_t)i * ld + t];
        w[t] = acc;
    }
}

// y = alpha x + beta y
__global__ void k_axpby(double alpha, const double* __restrict__ x, double beta, double* __restrict__ y, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        y[t] = alpha * x[t] + beta * y[t];
}

__global__ void k_row_nnz(const uint64_t* __restrict__ row_ptr, const int32_t* __restrict__ items, int64_t n_items,
                          int64_t n_rows_per_k, int R, unsigned long long* acc)
{
    unsigned long long t = 0;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < (int64_t)R * n_items;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = w / n_items, a = w - k * n_items;
        const int64_t row = k * n_rows_per_k + (items ? items[a] : a);
        t += row_ptr[row + 1] - row_ptr[row];
    }
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(acc, t);
}

unsigned grid1(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2048)); }

}  // namespace

int launch_chunk_compact(const ChunkCompactArgs& A, cudaStream_t s)
{
    if (A.rows <= 0) return URCHIN_OK;
    int grid = 0;
    URCHIN_TRY(grid_for((const void*)k_chunk_compact, kSpmvThreads, 0, &grid));
    k_chunk_compact<<<grid, kSpmvThreads, 0, s>>>(A);
    return launched();
}

int launch_spmv(const SpmvArgs& A, cudaStream_t s)
{
    if (A.n_items <= 0) return URCHIN_OK;
    int64_t warps = (int64_t)A.R * A.n_items;
    int grid = 0;
    // FP32 takes the split-index loop (the solver splits indices whenever n <=
    // 2^24); the strided loop serves FP64 and FP32 with int32 indices
    const void* fn = A.precision == URCHIN_F64 ? (const void*)k_spmv<double>
                                               : (A.col ? (const void*)k_spmv<float> : (const void*)k_spmv8);
    if (A.precision == URCHIN_F64 && !A.col) return set_error(URCHIN_ERR_ARG, "spmv: FP64 segments need int32 indices");
    if (A.chunk_head) {
        if (A.precision == URCHIN_F64 || !A.chunk_next || !A.row_cnt || !A.chunk_seg)
            return set_error(URCHIN_ERR_ARG, "spmv: chunked lists are FP32, with links and row counts");
        fn = (const void*)k_spmv_chunk;
    }
    URCHIN_TRY(grid_for(fn, kSpmvThreads, 0, &grid));
    int64_t need = (warps + 7) / 8;
    if (need < grid) grid = (int)std::max<int64_t>(need, 1);
    void* args[] = {const_cast<SpmvArgs*>(&A)};
    URCHIN_TRY_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kSpmvThreads), args, 0, s));
    return launched();
}

int launch_spmv_t(const SpmvTArgs& A, cudaStream_t s)
{
    if (A.n_items <= 0) return URCHIN_OK;
    int64_t warps = (int64_t)A.R * A.n_items;
    int grid = 0;
    const void* fn = A.precision == URCHIN_F64 ? (const void*)k_spmv_t<double> : (const void*)k_spmv_t<float>;
    URCHIN_TRY(grid_for(fn, kSpmvThreads, 0, &grid));
    int64_t need = (warps + 7) / 8;
    if (need < grid) grid = (int)std::max<int64_t>(need, 1);
    if (A.precision == URCHIN_F64) k_spmv_t<double><<<grid, kSpmvThreads, 0, s>>>(A);
    else k_spmv_t<float><<<grid, kSpmvThreads, 0, s>>>(A);
    return launched();
}

int launch_row_nnz(const uint64_t* row_ptr, const int32_t* items, int64_t n_items, int64_t n_rows_per_k, int R,
                   unsigned long long* acc, cudaStream_t s)
{
    k_row_nnz<<<grid1((int64_t)R * n_items), 256, 0, s>>>(row_ptr, items, n_items, n_rows_per_k, R, acc);
    return launched();
}

size_t dots_tmp_bytes(int count) { return sizeof(double) * (size_t)count * 256 + 256; }

int launch_dots(const double* V, int64_t ld, int count, const double* w, int64_t n, double* tmp, double* out,
                cudaStream_t s)
{
    const int nb = (int)std::min<int64_t>(256, std::max<int64_t>(1, (n + 255) / 256));
    dim3 g((unsigned)nb, (unsigned)count);
    k_dots<<<g, 256, 0, s>>>(V, ld, count, w, n, tmp);
    URCHIN_TRY(launched());
    k_dots_reduce<<<(count + 63) / 64, 64, 0, s>>>(tmp, nb, count, out);
    return launched();
}

int launch_subtract(double* w, const double* V, int64_t ld, int count, const double* coef, int64_t n,
                    cudaStream_t s)
{
    k_subtract<<<grid1(n), 256, 0, s>>>(w, V, ld, count, coef, n);
    return launched();
}

int launch_axpby(double alpha, const double* x, double beta, double* y, int64_t n, cudaStream_t s)
{
    k_axpby<<<grid1(n), 256, 0, s>>>(alpha, x, beta, y, n);
    return launched();
}

}  // namespace urchin
