// Error reporting, constants, scratch memory, and the device scan / radix
// sort / compaction primitives used by the BVH build and the solver.
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstring>
#include <string>

#include "common.cuh"

namespace urchin {

static thread_local char g_last_error[512] = "";

int set_error(int status, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}

void clear_error() { g_last_error[0] = '\0'; }

double sigma_th_cm2()
{
    const double alpha_fs = 7.2973525693e-3;       // CODATA 2018
    const double bohr_cm = 5.29177210903e-9;       // CODATA 2018
    const double e4 = std::exp(4.0);
    return 512.0 * kPi / (3.0 * e4) * alpha_fs * kPi * bohr_cm * bohr_cm;
}

GtConst gt_constants()
{
    GtConst c;
    c.t = 2.0 * std::pow(kPi, 1.0 / 6.0);
    c.t2 = c.t * c.t;
    double D = std::erf(c.t) - 2.0 * c.t * std::exp(-c.t2) / std::sqrt(kPi);
    c.pref = std::sqrt(kPi) / (2.0 * c.t * D);
    return c;
}

// ---- the library's memory pool ---------------------------------------------
// One stream-ordered pool per device whose release threshold keeps freed
// memory reserved: the default pool returns it to the device at every
// synchronisation, and mapping 14 GB again costs ~12 ms (unmapping ~20 ms).
constexpr int kMaxDevices = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[kMaxDevices];
static bool g_pool_made[kMaxDevices];

int library_pool(cudaMemPool_t* out)
{
    int dev = 0;
    URCHIN_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(URCHIN_ERR_CUDA, "device %d beyond the pool table", dev);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool_made[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        URCHIN_TRY_CUDA(cudaMemPoolCreate(&g_pool[dev], &props));
        uint64_t keep = UINT64_MAX;
        URCHIN_TRY_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        g_pool_made[dev] = true;
    }
    *out = g_pool[dev];
    return URCHIN_OK;
}

size_t pool_idle_bytes()
{
    cudaMemPool_t pool;
    if (library_pool(&pool) != URCHIN_OK) {
        clear_error();
        return 0;
    }
    uint64_t reserved = 0, used = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return reserved > used ? (size_t)(reserved - used) : 0;
}

int Scratch::alloc(size_t bytes, cudaStream_t s)
{
    release();
    stream = s;
    if (bytes == 0) bytes = 256;
    cudaMemPool_t pool;
    URCHIN_TRY(library_pool(&pool));
    cudaError_t e = cudaMallocFromPoolAsync(&ptr, bytes, pool, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? URCHIN_ERR_NOMEM : URCHIN_ERR_CUDA,
                         "cudaMallocFromPoolAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    return URCHIN_OK;
}

void Scratch::release()
{
    if (ptr) cudaFreeAsync(ptr, stream);
    ptr = nullptr;
}

static std::atomic<long long> g_launches{0};

int launched()
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(URCHIN_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return URCHIN_OK;
}

int grid_for(const void* kernel, int block, size_t smem, int* grid_out)
{
    int dev = 0, sms = 0, per_sm = 0;
    URCHIN_TRY_CUDA(cudaGetDevice(&dev));
    URCHIN_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    URCHIN_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
    if (per_sm < 1) per_sm = 1;
    *grid_out = sms * per_sm;
    return URCHIN_OK;
}

// ---------------------------------------------------------------------------
// Exclusive scan: tiles of kScanTile values per block, recursive on tile sums.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total.
template <typename T>
__device__ T block_excl_scan(T v, T* total)
{
    __shared__ T warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T ws = (lane < kScanThreads / 32) ? warp_sums[lane] : T(0);
        T wi = warp_incl_scan(ws);
        if (lane < kScanThreads / 32) warp_sums[lane] = wi - ws;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    T r = incl - v + warp_sums[wid];
    __syncthreads();
    return r;
}

template <typename TIn, typename TOut>
__global__ void k_scan_tiles(const TIn* in, TOut* out, int64_t n, TOut* tile_sums, TOut* total_dev)
{
    __shared__ TOut tot;
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    TOut v[kScanItems];
    TOut sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? (TOut)in[base + i] : TOut(0);
        sum += v[i];
    }
    TOut pre = block_excl_scan<TOut>(sum, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) {
        if (tile_sums) tile_sums[blockIdx.x] = tot;
        if (total_dev && gridDim.x == 1) *total_dev = tot;
    }
}

template <typename T>
__global__ void k_scan_add(T* out, int64_t n, const T* tile_pre)
{
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    T add = tile_pre[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x)
        if (base + i < n) out[base + i] += add;
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

template <typename T>
static size_t scan_tmp_bytes_t(int64_t n)
{
    size_t bytes = 0;
    int64_t m = n;
    while (m > kScanTile) {
        m = ceil_div(m, kScanTile);
        bytes += ((size_t)m * sizeof(T) + 255) & ~size_t(255);
    }
    return bytes + 256;
}

size_t scan_tmp_bytes(int64_t n) { return scan_tmp_bytes_t<uint32_t>(n); }
size_t scan64_tmp_bytes(int64_t n) { return scan_tmp_bytes_t<uint64_t>(n); }

template <typename TIn, typename TOut>
static int scan_t(const TIn* in, TOut* out, int64_t n, void* tmp, TOut* total_dev, cudaStream_t s)
{
    if (n <= 0) {
        if (total_dev) URCHIN_TRY_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(TOut), s));
        return URCHIN_OK;
    }
    int64_t tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        k_scan_tiles<TIn, TOut><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev);
        URCHIN_TRY(launched());
        return URCHIN_OK;
    }
    TOut* sums = static_cast<TOut*>(tmp);
    void* rest = static_cast<char*>(tmp) + (((size_t)tiles * sizeof(TOut) + 255) & ~size_t(255));
    k_scan_tiles<TIn, TOut><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums, nullptr);
    URCHIN_TRY(launched());
    URCHIN_TRY((scan_t<TOut, TOut>(sums, sums, tiles, rest, total_dev, s)));
    k_scan_add<TOut><<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, sums);
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

int scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, void* tmp, uint32_t* total_dev,
                       cudaStream_t s)
{
    return scan_t<uint32_t, uint32_t>(in, out, n, tmp, total_dev, s);
}

int scan_counts_u64(const uint32_t* in, uint64_t* out, int64_t n, void* tmp, uint64_t* total_dev,
                    cudaStream_t s)
{
    return scan_t<uint32_t, uint64_t>(in, out, n, tmp, total_dev, s);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, 4-bit digits, 256 threads x 16 items per tile.
// ---------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;
constexpr int kRadixDigits = 16;

__global__ void k_radix_hist(const uint32_t* keys, int64_t n, int shift, uint32_t* hist, int nblocks)
{
    __shared__ uint32_t cnt[kRadixDigits];
    if (threadIdx.x < kRadixDigits) cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 15u], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kRadixDigits) hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                                int64_t n, int shift, const uint32_t* offsets, int nblocks)
{
    constexpr int W = kRadixThreads / 32;
    __shared__ uint32_t running[kRadixDigits];
    __shared__ uint32_t wcnt[W][kRadixDigits + 1];
    __shared__ uint32_t wpre[W][kRadixDigits + 1];
    __shared__ uint32_t rtot[kRadixDigits];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < kRadixDigits)
        running[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const uint32_t lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = 0; r < kRadixRounds; ++r) {
        for (int t = threadIdx.x; t < W * (kRadixDigits + 1); t += blockDim.x)
            (&wcnt[0][0])[t] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        int32_t val = valid ? vin[i] : 0;
        uint32_t d = valid ? ((key >> shift) & 15u) : (uint32_t)kRadixDigits;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (rank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < kRadixDigits) {
            uint32_t acc = 0;
            for (int w = 0; w < W; ++w) {
                wpre[w][threadIdx.x] = acc;
                acc += wcnt[w][threadIdx.x];
            }
            rtot[threadIdx.x] = acc;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = running[d] + wpre[wid][d] + rank;
            if (pos < n) {          // always true for a consistent histogram
                kout[pos] = key;
                vout[pos] = val;
            }
        }
        __syncthreads();
        if (threadIdx.x < kRadixDigits) running[threadIdx.x] += rtot[threadIdx.x];
        __syncthreads();
    }
}

size_t radix_tmp_bytes(int64_t n)
{
    int64_t nblocks = ceil_div(n, kRadixTile);
    size_t b = 0;
    b += ((size_t)n * 4 + 255) & ~size_t(255);                      // alt keys
    b += ((size_t)n * 4 + 255) & ~size_t(255);                      // alt vals
    b += ((size_t)nblocks * kRadixDigits * 4 + 255) & ~size_t(255); // histogram
    b += scan_tmp_bytes(nblocks * kRadixDigits);
    return b;
}

int radix_sort_pairs(uint32_t* keys, int32_t* vals, int64_t n, int bits, void* tmp, cudaStream_t s)
{
    if (n <= 1) return URCHIN_OK;
    int64_t nblocks = ceil_div(n, kRadixTile);
    char* p = static_cast<char*>(tmp);
    uint32_t* k2 = reinterpret_cast<uint32_t*>(p);
    p += ((size_t)n * 4 + 255) & ~size_t(255);
    int32_t* v2 = reinterpret_cast<int32_t*>(p);
    p += ((size_t)n * 4 + 255) & ~size_t(255);
    uint32_t* hist = reinterpret_cast<uint32_t*>(p);
    p += ((size_t)nblocks * kRadixDigits * 4 + 255) & ~size_t(255);
    void* stmp = p;
    int passes = (bits + 3) / 4;
    uint32_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    for (int pass = 0; pass < passes; ++pass) {
        int shift = 4 * pass;
        k_radix_hist<<<(unsigned)nblocks, kRadixThreads, 0, s>>>(ka, n, shift, hist, (int)nblocks);
        URCHIN_TRY(launched());
        URCHIN_TRY(scan_exclusive_u32(hist, hist, nblocks * kRadixDigits, stmp, nullptr, s));
        k_radix_scatter<<<(unsigned)nblocks, kRadixThreads, 0, s>>>(ka, va, kb, vb, n, shift, hist,
                                                                    (int)nblocks);
        URCHIN_TRY(launched());
        uint32_t* tk = ka; ka = kb; kb = tk;
        int32_t* tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        URCHIN_TRY_CUDA(cudaMemcpyAsync(keys, ka, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
        URCHIN_TRY_CUDA(cudaMemcpyAsync(vals, va, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    }
    return URCHIN_OK;
}

// ---------------------------------------------------------------------------
// Compaction
// ---------------------------------------------------------------------------
__global__ void k_flags_u32(const uint8_t* flags, uint32_t* out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = flags[i] ? 1u : 0u;
}

__global__ void k_compact_scatter(const uint8_t* flags, const uint32_t* pos, int64_t n, int32_t* out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i] && pos[i] < n) out[pos[i]] = (int32_t)i;
}

size_t compact_tmp_bytes(int64_t n)
{
    return (((size_t)n * 4 + 255) & ~size_t(255)) + scan_tmp_bytes(n);
}

int compact_indices(const uint8_t* flags, int64_t n, int32_t* out, uint32_t* count_dev, void* tmp,
                    cudaStream_t s)
{
    uint32_t* pos = static_cast<uint32_t*>(tmp);
    void* stmp = static_cast<char*>(tmp) + (((size_t)n * 4 + 255) & ~size_t(255));
    unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 4096);
    if (grid == 0) grid = 1;
    k_flags_u32<<<grid, 256, 0, s>>>(flags, pos, n);
    URCHIN_TRY(launched());
    URCHIN_TRY(scan_exclusive_u32(pos, pos, n, stmp, count_dev, s));
    k_compact_scatter<<<grid, 256, 0, s>>>(flags, pos, n, out);
    URCHIN_TRY(launched());
    return URCHIN_OK;
}

}  // namespace urchin

extern "C" const char* urchin_last_error(void) { return urchin::g_last_error; }

extern "C" const char* urchin_version(void) { return "urchin-gb300 0.1 (sm_103a)"; }

extern "C" int64_t urchin_kernel_launches(void) { return (int64_t)urchin::g_launches.load(); }

extern "C" int urchin_trim_memory(int device, uint64_t* reserved_out)
{
    using namespace urchin;
    clear_error();
    if (device < -1 || device >= kMaxDevices) return set_error(URCHIN_ERR_ARG, "urchin_trim_memory: bad device %d", device);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    uint64_t total = 0;
    for (int d = 0; d < kMaxDevices; ++d) {
        if ((device >= 0 && d != device) || !g_pool_made[d]) continue;
        URCHIN_TRY_CUDA(cudaMemPoolTrimTo(g_pool[d], 0));
        uint64_t r = 0;
        URCHIN_TRY_CUDA(cudaMemPoolGetAttribute(g_pool[d], cudaMemPoolAttrReservedMemCurrent, &r));
        total += r;
    }
    if (reserved_out) *reserved_out = total;
    return URCHIN_OK;
}
