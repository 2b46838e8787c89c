// urchin_trace_columns_noalloc: column tracing for callers that cannot
// allocate device memory.  It gives the same columns as urchin_trace_columns
// (bit for bit: a ray sums its hits in the tree's fixed depth-first order,
// whichever rays share its warp), but its work arrays (the traversal's
// work-queue counter and status word, the ray directions, the per-particle
// tracer weights and the mapped origin list) live in one fixed array in this
// file instead of coming from the stream-ordered allocator.  It traces the
// rays in the order of the origin list, without the per-direction ray
// ordering that the allocating call sorts into extra memory for large
// origin sets, so calls with many origins run slower.
//
// The array is a file-scope __device__ variable, so every GPU that loads the
// library holds it until the process exits.  Host code cannot use the
// array's name as a device address; the address is looked up once per
// device with cudaGetSymbolAddress (on the first call made on that device)
// and cached, which assumes the device keeps the same CUDA context for the
// life of the process (after cudaDeviceReset the cached address is stale).
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace urchin {
namespace {

__device__ __align__(256) unsigned char g_trace_scratch[URCHIN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_trace_scratch on the current device.
int scratch_address(void** out)
{
    int dev = 0;
    URCHIN_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(URCHIN_ERR_CUDA, "urchin_trace_columns_noalloc: device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_trace_scratch);
        if (e != cudaSuccess || !p)
            return set_error(URCHIN_ERR_CUDA, "urchin_trace_columns_noalloc: cudaGetSymbolAddress failed: %s",
                             cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return URCHIN_OK;
}

}  // namespace
}  // namespace urchin

extern "C" int urchin_trace_columns_noalloc(const urchin_bvh* bvh, const double* x, const double* dirs, int R,
                                            double l_ray, const int32_t* origins, int64_t n_orig, int kernel,
                                            int precision, void* tau_out, urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    cudaStream_t s = (cudaStream_t)stream;
    if (!bvh || !x || !dirs) return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: NULL bvh, x or dirs");
    if (R < 1 || R > URCHIN_MAX_RAYS)
        return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: R = %d out of range [1, %d]", R,
                         URCHIN_MAX_RAYS);
    if (!(l_ray >= 0.0) || !std::isfinite(l_ray))
        return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: l_ray must be finite and >= 0");
    if (kernel != URCHIN_KERNEL_M4 && kernel != URCHIN_KERNEL_GT)
        return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: unknown kernel %d", kernel);
    if (precision != URCHIN_F32 && precision != URCHIN_F64)
        return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: unknown precision %d", precision);
    if (n_orig < 0) return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: n_orig < 0");
    if (n_orig == 0) return URCHIN_OK;
    if (!origins && n_orig != bvh->n)
        return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: origins NULL requires n_orig == n");
    if (!tau_out) return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: tau_out is NULL");
    for (int k = 0; k < R; ++k) {
        const double* d = dirs + 3 * k;
        const double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!std::isfinite(nn) || std::fabs(nn - 1.0) > 1e-6)
            return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: direction %d is not a unit vector", k);
    }
    const int64_t n = bvh->n;
    const bool f64 = precision == URCHIN_F64;
    Layout lay;
    const size_t o_ctr = lay.take(2 * sizeof(unsigned));
    const size_t o_dirs = lay.take(sizeof(double) * 3 * (size_t)R);
    const size_t o_w = lay.take((f64 ? sizeof(double) : sizeof(float)) * (size_t)n);
    const size_t o_items = lay.take(origins ? sizeof(int32_t) * (size_t)n_orig : 0);
    if (lay.bytes > (size_t)URCHIN_NOALLOC_SCRATCH_BYTES)
        return set_error(URCHIN_ERR_ARG,
                         "urchin_trace_columns_noalloc: this call needs %zu bytes of work space, more than the "
                         "fixed %zu-byte array (fewer particles or origins, or use urchin_trace_columns)",
                         lay.bytes, (size_t)URCHIN_NOALLOC_SCRATCH_BYTES);
    void* base = nullptr;
    URCHIN_TRY(scratch_address(&base));
    char* scr = static_cast<char*>(base);
    unsigned* ctr = reinterpret_cast<unsigned*>(scr + o_ctr);
    double* ddirs = reinterpret_cast<double*>(scr + o_dirs);
    float* w32 = f64 ? nullptr : reinterpret_cast<float*>(scr + o_w);
    double* w64 = f64 ? reinterpret_cast<double*>(scr + o_w) : nullptr;
    // the array keeps the previous call's contents: clear what must start at zero
    URCHIN_TRY_CUDA(cudaMemsetAsync(ctr, 0, 2 * sizeof(unsigned), s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(ddirs, dirs, sizeof(double) * 3 * (size_t)R, cudaMemcpyHostToDevice, s));
    URCHIN_TRY(launch_weights(bvh, x, w32, w64, s));
    TraceJob job{};
    job.bvh = bvh;
    job.w32 = w32;
    job.w64 = w64;
    job.dirs_dev = ddirs;
    job.R = R;
    job.l_ray = l_ray;
    job.n_items = n_orig;
    job.row_stride = R;
    job.k_stride = 1;
    job.out = tau_out;
    job.kernel = kernel;
    job.precision = precision;
    job.counter = ctr;
    job.status = ctr + 1;
    if (origins) {
        int32_t* items = reinterpret_cast<int32_t*>(scr + o_items);
        URCHIN_TRY(launch_map_origins(bvh, origins, n_orig, items, ctr + 1, s));
        job.items = items;
        job.out_row = nullptr;
    } else {
        job.items = nullptr;
        job.out_row = bvh->perm;
    }
    URCHIN_TRY(launch_trace(job, s));
    unsigned st = 0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&st, ctr + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    if (st & kStOrigin) return set_error(URCHIN_ERR_ARG, "urchin_trace_columns_noalloc: origin index out of range");
    if (st & kStStack) return set_error(URCHIN_ERR_CUDA, "urchin_trace_columns_noalloc: traversal stack overflow");
    if (st & kStVisit) return set_error(URCHIN_ERR_CUDA, "urchin_trace_columns_noalloc: malformed tree");
    return URCHIN_OK;
}
