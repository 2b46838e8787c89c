// Linear BVH over the particles' smoothing spheres.
//
// The paper does not describe its search structure; this is a Morton-code
// LBVH: 30-bit Morton codes of the sphere centres, stable radix sort, the
// binary radix tree of Karras (2012, "Maximizing parallelism in the
// construction of BVHs, octrees and k-d trees"), bottom-up refit of sphere
// bounds, then a packed two-children-per-node layout in which subtrees of
// at most kLeafMax particles become leaves.  The particle data are copied
// into Morton order so that a leaf is a contiguous range.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "common.cuh"

namespace urchin {

namespace {

__device__ __forceinline__ unsigned f2ord(float f)
{
    unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__host__ __device__ __forceinline__ float ord2f(unsigned u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
#else
    unsigned v = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    float f;
    memcpy(&f, &v, 4);
    return f;
#endif
}

// bounds[0..2] min centre, [3..5] max centre, [6] max h (ordered encoding);
// bounds[7] error bits: 1 = non-finite, 2 = h <= 0 or mass < 0
// logh_sum accumulates sum ln h (the geometric mean of h sets the shape of
// the traversal's ray packets)
__global__ void k_bounds(const float* __restrict__ x, const float* __restrict__ y,
                         const float* __restrict__ z, const float* __restrict__ h,
                         const double* __restrict__ m, int64_t n, unsigned* bounds, double* logh_sum)
{
    unsigned mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu};
    unsigned mx[4] = {0u, 0u, 0u, 0u};
    unsigned err = 0;
    double lsum = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float c[3] = {x[i], y[i], z[i]};
        float hi = h[i];
        double mi = m[i];
        bool fin = isfinite(c[0]) && isfinite(c[1]) && isfinite(c[2]) && isfinite(hi) && isfinite(mi);
        if (!fin) { err |= 1u; continue; }
        if (!(hi > 0.f) || mi < 0.0) err |= 2u;
        else lsum += (double)logf(hi);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            unsigned o = f2ord(c[a]);
            mn[a] = min(mn[a], o);
            mx[a] = max(mx[a], o);
        }
        mx[3] = max(mx[3], f2ord(hi));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], off));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], off));
        }
        mx[3] = max(mx[3], __shfl_xor_sync(0xffffffffu, mx[3], off));
        err |= __shfl_xor_sync(0xffffffffu, err, off);
        lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bounds[a], mn[a]);
            atomicMax(&bounds[3 + a], mx[a]);
        }
        atomicMax(&bounds[6], mx[3]);
        if (err) atomicOr(&bounds[7], err);
        atomicAdd(logh_sum, lsum);
    }
}

__device__ __forceinline__ unsigned spread10(unsigned v)
{
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__global__ void k_morton(const float* __restrict__ x, const float* __restrict__ y,
                         const float* __restrict__ z, int64_t n, const unsigned* bounds,
                         uint32_t* codes, int32_t* idx)
{
    float lo[3], inv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = ord2f(bounds[a]);
        float ext = ord2f(bounds[3 + a]) - lo[a];
        inv[a] = ext > 0.f ? 1.0f / ext : 0.f;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float c[3] = {x[i], y[i], z[i]};
        unsigned q[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float u = (c[a] - lo[a]) * inv[a];
            u = fminf(fmaxf(u * 1024.f, 0.f), 1023.f);
            q[a] = (unsigned)u;
        }
        codes[i] = (spread10(q[0]) << 2) | (spread10(q[1]) << 1) | spread10(q[2]);
        idx[i] = (int32_t)i;
    }
}

__global__ void k_gather(const float* __restrict__ x, const float* __restrict__ y,
                         const float* __restrict__ z, const float* __restrict__ h,
                         const double* __restrict__ m, const int32_t* __restrict__ order, int64_t n,
                         double mass_to_A, double unit_cm, float4* xyzh, float* A32, double* A64,
                         int32_t* perm, int32_t* inv, unsigned* err)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = order[s];
        if (i < 0 || i >= n) {     // a permutation from the sort; never true
            atomicOr(err, 8u);
            continue;
        }
        float hi = h[i];
        xyzh[s] = make_float4(x[i], y[i], z[i], hi);
        double hcm = (double)hi * unit_cm;
        // A_j = sigma_th (m_j/m_p) (8/pi) / h_j^2: threshold optical depth per
        // unit dimensionless chord integral of a fully neutral particle
        double A = mass_to_A * m[i] / (hcm * hcm);
        A64[s] = A;
        A32[s] = (float)A;
        perm[s] = i;
        inv[i] = (int32_t)s;
    }
}

__device__ __forceinline__ int delta(const uint32_t* __restrict__ codes, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    uint32_t a = codes[i], b = codes[j];
    if (a != b) return __clz(a ^ b);
    return 32 + __clz((unsigned)i ^ (unsigned)j);
}

// Karras (2012) binary radix tree: internal node i covers a Morton range and
// splits it at the highest differing bit.  Children are encoded >= 0 for an
// internal node, ~leaf for a leaf (particle).
__global__ void k_karras(const uint32_t* __restrict__ codes, int n, int32_t* child_l, int32_t* child_r,
                         int32_t* first, int32_t* last, int32_t* parent_int, int32_t* parent_leaf)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(codes, n, i, i - d);
    int lmax = 2;
    while (delta(codes, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = delta(codes, n, i, j);
    int s = 0;
    for (int div = 2;; div <<= 1) {
        int t = (l + div - 1) / div;
        if (delta(codes, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    int g = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    first[i] = lo;
    last[i] = hi;
    if (lo == g) { child_l[i] = ~g; parent_leaf[g] = i; }
    else { child_l[i] = g; parent_int[g] = i; }
    if (hi == g + 1) { child_r[i] = ~(g + 1); parent_leaf[g + 1] = i; }
    else { child_r[i] = g + 1; parent_int[g + 1] = i; }
    if (i == 0) parent_int[0] = -1;
}

// Conservative sphere bounds: rounded outward and padded by 1e-6 of the
// coordinate scale so float slab tests never cull a sphere a ray crosses.
__device__ __forceinline__ void sphere_box(float4 p, float lo[3], float hi[3])
{
    float pad = 1e-6f * (fmaxf(fmaxf(fabsf(p.x), fabsf(p.y)), fabsf(p.z)) + p.w);
    lo[0] = __fsub_rd(__fsub_rd(p.x, p.w), pad);
    lo[1] = __fsub_rd(__fsub_rd(p.y, p.w), pad);
    lo[2] = __fsub_rd(__fsub_rd(p.z, p.w), pad);
    hi[0] = __fadd_ru(__fadd_ru(p.x, p.w), pad);
    hi[1] = __fadd_ru(__fadd_ru(p.y, p.w), pad);
    hi[2] = __fadd_ru(__fadd_ru(p.z, p.w), pad);
}

__device__ __forceinline__ void child_box(int32_t c, const float4* __restrict__ xyzh, const float* boxes,
                                          float lo[3], float hi[3])
{
    if (c < 0) {
        sphere_box(xyzh[~c], lo, hi);
    } else {
        const float* b = boxes + 6 * (int64_t)c;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = __ldcg(b + a);
            hi[a] = __ldcg(b + 3 + a);
        }
    }
}

__global__ void k_refit(const float4* __restrict__ xyzh, int n, const int32_t* child_l,
                        const int32_t* child_r, const int32_t* parent_int, const int32_t* parent_leaf,
                        float* boxes, unsigned* visits, unsigned* err)
{
    int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= n) return;
    int p = parent_leaf[leaf];
    // the tree is at most 62 levels deep (30-bit codes, 32-bit index
    // tie-break); the cap only guards against a malformed parent chain
    for (int level = 0; p >= 0; ++level) {
        if (level > 128) {
            atomicOr(err, 4u);
            return;
        }
        __threadfence();
        unsigned old = atomicAdd(&visits[p], 1u);
        if (old == 0) return;          // sibling subtree not finished yet
        __threadfence();
        float llo[3], lhi[3], rlo[3], rhi[3];
        child_box(child_l[p], xyzh, boxes, llo, lhi);
        child_box(child_r[p], xyzh, boxes, rlo, rhi);
        float* b = boxes + 6 * (int64_t)p;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            __stcg(b + a, fminf(llo[a], rlo[a]));
            __stcg(b + 3 + a, fmaxf(lhi[a], rhi[a]));
        }
        p = parent_int[p];
    }
}

__device__ __forceinline__ void pack_child(int32_t c, const float4* __restrict__ xyzh, const float* boxes,
                                           const int32_t* first, const int32_t* last, float4* out0,
                                           float4* out1)
{
    float lo[3], hi[3];
    child_box(c, xyzh, boxes, lo, hi);
    int ref, cnt;
    if (c < 0) {
        ref = ~c;
        cnt = 1;
    } else {
        int size = last[c] - first[c] + 1;
        if (size <= kLeafMax) { ref = first[c]; cnt = size; }
        else { ref = c; cnt = 0; }
    }
    *out0 = make_float4(lo[0], lo[1], lo[2], __int_as_float(ref));
    *out1 = make_float4(hi[0], hi[1], hi[2], __int_as_float(cnt));
}

__global__ void k_pack(const float4* __restrict__ xyzh, int n, const int32_t* child_l,
                       const int32_t* child_r, const int32_t* first, const int32_t* last,
                       const float* boxes, float4* nodes)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    float4 a, b, c, d;
    pack_child(child_l[i], xyzh, boxes, first, last, &a, &b);
    pack_child(child_r[i], xyzh, boxes, first, last, &c, &d);
    nodes[4 * (int64_t)i + 0] = a;
    nodes[4 * (int64_t)i + 1] = b;
    nodes[4 * (int64_t)i + 2] = c;
    nodes[4 * (int64_t)i + 3] = d;
}

// n == 1: one root whose left child is the single particle, right child empty
__global__ void k_pack_single(const float4* __restrict__ xyzh, float4* nodes)
{
    float lo[3], hi[3];
    sphere_box(xyzh[0], lo, hi);
    nodes[0] = make_float4(lo[0], lo[1], lo[2], __int_as_float(0));
    nodes[1] = make_float4(hi[0], hi[1], hi[2], __int_as_float(1));
    nodes[2] = make_float4(1.f, 1.f, 1.f, __int_as_float(0));
    nodes[3] = make_float4(-1.f, -1.f, -1.f, __int_as_float(-1));   // count < 0: no child
}

void free_bvh_arrays(urchin_bvh* b)
{
    if (!b) return;
    cudaFree(b->nodes);
    cudaFree(b->xyzh);
    cudaFree(b->A32);
    cudaFree(b->A64);
    cudaFree(b->perm);
    cudaFree(b->inv);
    cudaFree(b->ktab);
    b->ktab = nullptr;
    b->nodes = nullptr;
    b->xyzh = nullptr;
    b->A32 = nullptr;
    b->A64 = nullptr;
    b->perm = nullptr;
    b->inv = nullptr;
}

int build(const urchin_particles* p, const urchin_box* box, urchin_bvh* b, cudaStream_t s)
{
    const int64_t n = p->n;
    b->n = n;
    b->periodic = box->periodic ? 1 : 0;
    b->L = box->L;
    b->unit_cm = box->unit_cm;
    URCHIN_TRY_CUDA(cudaGetDevice(&b->device));
    b->n_nodes = (int)std::max<int64_t>(1, n - 1);
    URCHIN_TRY_CUDA(cudaMalloc(&b->nodes, sizeof(float4) * 4 * (size_t)b->n_nodes));
    URCHIN_TRY_CUDA(cudaMalloc(&b->xyzh, sizeof(float4) * (size_t)n));
    URCHIN_TRY_CUDA(cudaMalloc(&b->A32, sizeof(float) * (size_t)n));
    URCHIN_TRY_CUDA(cudaMalloc(&b->A64, sizeof(double) * (size_t)n));
    URCHIN_TRY_CUDA(cudaMalloc(&b->perm, sizeof(int32_t) * (size_t)n));
    URCHIN_TRY_CUDA(cudaMalloc(&b->inv, sizeof(int32_t) * (size_t)n));
    URCHIN_TRY_CUDA(cudaMalloc(&b->ktab, sizeof(float2) * (kKTab + 1)));
    {
        static float2 table[kKTab + 1];
        static bool ready = false;
        static std::mutex mu;
        std::lock_guard<std::mutex> lock(mu);
        if (!ready) {
            m4_full_table(table);
            ready = true;
        }
        URCHIN_TRY_CUDA(cudaMemcpyAsync(b->ktab, table, sizeof(table), cudaMemcpyHostToDevice, s));
        URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    }

    const int64_t ni = std::max<int64_t>(1, n - 1);
    Layout lay;
    size_t o_bounds = lay.take(8 * sizeof(unsigned));
    size_t o_logh = lay.take(sizeof(double));
    size_t o_codes = lay.take((size_t)n * 4);
    size_t o_idx = lay.take((size_t)n * 4);
    size_t o_radix = lay.take(radix_tmp_bytes(n));
    size_t o_cl = lay.take((size_t)ni * 4);
    size_t o_cr = lay.take((size_t)ni * 4);
    size_t o_first = lay.take((size_t)ni * 4);
    size_t o_last = lay.take((size_t)ni * 4);
    size_t o_pint = lay.take((size_t)ni * 4);
    size_t o_pleaf = lay.take((size_t)n * 4);
    size_t o_boxes = lay.take((size_t)ni * 6 * 4);
    size_t o_visits = lay.take((size_t)ni * 4);
    Scratch scr;
    URCHIN_TRY(scr.alloc(lay.bytes, s));
    unsigned* bounds = scr.at<unsigned>(o_bounds);
    uint32_t* codes = scr.at<uint32_t>(o_codes);
    int32_t* idx = scr.at<int32_t>(o_idx);

    unsigned init[8] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u, 0u, 0u};
    URCHIN_TRY_CUDA(cudaMemcpyAsync(bounds, init, sizeof(init), cudaMemcpyHostToDevice, s));
    double* logh = scr.at<double>(o_logh);
    URCHIN_TRY_CUDA(cudaMemsetAsync(logh, 0, sizeof(double), s));
    unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 2048);
    k_bounds<<<grid, 256, 0, s>>>(p->pos_x, p->pos_y, p->pos_z, p->h, p->mass_H, n, bounds, logh);
    URCHIN_TRY(launched());
    unsigned hb[8];
    double lh = 0.0;
    URCHIN_TRY_CUDA(cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(&lh, logh, sizeof(double), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    b->hgeo = (float)std::exp(lh / (double)n);
    if (hb[7] & 1u) return set_error(URCHIN_ERR_NONFINITE, "urchin_build_bvh: NaN/Inf in positions, h or mass_H");
    if (hb[7] & 2u) return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: h must be > 0 and mass_H >= 0");
    b->hmax = ord2f(hb[6]);

    k_morton<<<grid, 256, 0, s>>>(p->pos_x, p->pos_y, p->pos_z, n, bounds, codes, idx);
    URCHIN_TRY(launched());
    URCHIN_TRY(radix_sort_pairs(codes, idx, n, 30, scr.at<void>(o_radix), s));
    const double mass_to_A = sigma_th_cm2() * 8.0 / kPi;
    k_gather<<<grid, 256, 0, s>>>(p->pos_x, p->pos_y, p->pos_z, p->h, p->mass_H, idx, n, mass_to_A,
                                  b->unit_cm, b->xyzh, b->A32, b->A64, b->perm, b->inv,
                                  bounds + 7);
    URCHIN_TRY(launched());

    if (n == 1) {
        k_pack_single<<<1, 1, 0, s>>>(b->xyzh, b->nodes);
        URCHIN_TRY(launched());
    } else {
        int32_t* cl = scr.at<int32_t>(o_cl);
        int32_t* cr = scr.at<int32_t>(o_cr);
        int32_t* first = scr.at<int32_t>(o_first);
        int32_t* last = scr.at<int32_t>(o_last);
        int32_t* pint = scr.at<int32_t>(o_pint);
        int32_t* pleaf = scr.at<int32_t>(o_pleaf);
        float* boxes = scr.at<float>(o_boxes);
        unsigned* visits = scr.at<unsigned>(o_visits);
        int ninode = (int)(n - 1);
        unsigned gi = (unsigned)((ninode + 255) / 256);
        unsigned gl = (unsigned)((n + 255) / 256);
        URCHIN_TRY_CUDA(cudaMemsetAsync(visits, 0, (size_t)ninode * 4, s));
        k_karras<<<gi, 256, 0, s>>>(codes, (int)n, cl, cr, first, last, pint, pleaf);
        URCHIN_TRY(launched());
        k_refit<<<gl, 256, 0, s>>>(b->xyzh, (int)n, cl, cr, pint, pleaf, boxes, visits, bounds + 7);
        URCHIN_TRY(launched());
        k_pack<<<gi, 256, 0, s>>>(b->xyzh, (int)n, cl, cr, first, last, boxes, b->nodes);
        URCHIN_TRY(launched());
    }
    float4 root[4];
    URCHIN_TRY_CUDA(cudaMemcpyAsync(root, b->nodes, sizeof(root), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, s));
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    if (hb[7] & 12u) return set_error(URCHIN_ERR_CUDA, "urchin_build_bvh: internal consistency check failed (%u)",
                                      hb[7]);
    b->root_lo[0] = std::min(root[0].x, root[2].x);
    b->root_lo[1] = std::min(root[0].y, root[2].y);
    b->root_lo[2] = std::min(root[0].z, root[2].z);
    b->root_hi[0] = std::max(root[1].x, root[3].x);
    b->root_hi[1] = std::max(root[1].y, root[3].y);
    b->root_hi[2] = std::max(root[1].z, root[3].z);
    scr.release();
    URCHIN_TRY_CUDA(cudaStreamSynchronize(s));
    return URCHIN_OK;
}

}  // namespace

}  // namespace urchin

extern "C" int urchin_build_bvh(const urchin_particles* p, const urchin_box* box, urchin_bvh** out,
                                urchin_stream_t stream)
{
    using namespace urchin;
    clear_error();
    if (!out) return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: out is NULL");
    *out = nullptr;
    if (!p || !box) return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: particles or box is NULL");
    if (p->n < 1 || p->n > (int64_t)0x3fffffff)
        return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: n = %lld out of range [1, 2^30)", (long long)p->n);
    if (!p->pos_x || !p->pos_y || !p->pos_z || !p->h || !p->mass_H)
        return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: a particle array is NULL");
    if (!(box->unit_cm > 0.0) || !std::isfinite(box->unit_cm))
        return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: unit_cm must be finite and > 0");
    if (box->periodic && (!(box->L > 0.0) || !std::isfinite(box->L)))
        return set_error(URCHIN_ERR_ARG, "urchin_build_bvh: periodic box needs finite L > 0");
    urchin_bvh* b = new (std::nothrow) urchin_bvh();
    if (!b) return set_error(URCHIN_ERR_NOMEM, "urchin_build_bvh: host allocation failed");
    int st = build(p, box, b, (cudaStream_t)stream);
    if (st != URCHIN_OK) {
        free_bvh_arrays(b);
        delete b;
        return st;
    }
    *out = b;
    return URCHIN_OK;
}

extern "C" void urchin_free_bvh(urchin_bvh* bvh)
{
    if (!bvh) return;
    cudaDeviceSynchronize();
    urchin::free_bvh_arrays(bvh);
    delete bvh;
}

extern "C" int64_t urchin_bvh_size(const urchin_bvh* bvh) { return bvh ? bvh->n : -1; }
