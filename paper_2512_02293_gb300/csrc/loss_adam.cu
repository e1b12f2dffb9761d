// loss_adam.cu -- the colour/depth L1 terms of Eq. 6 with their image
// gradients, and the Adam step of the mapping iteration.
//
// Loss: grid (pixel blocks, view).  Pass 1 reduces |I_hat - I|, |D_hat - D| over
// D > 0 and the valid-pixel count of each view (block reduction, three atomics
// per block into a per-view accumulator in the workspace); pass 2 writes the
// signed, normalised image gradients and the per-view loss terms.
// Adam: one grid-stride launch over the 4-element chunks of all parameter
// groups, float4 loads/stores where a group is 16-byte aligned; the step
// counter lives on the device so the launch can be replayed from a CUDA graph.
#include <math.h>

#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kLossThreads = 256;
constexpr int kLossItems = 4;

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

__global__ void __launch_bounds__(kLossThreads) k_loss_reduce(gs_image img, const float* __restrict__ tc,
                                                             const float* __restrict__ td, Views views,
                                                             float* __restrict__ acc) {
    pdl_enter();
    const int v = blockIdx.y;
    const ViewParams& vp = views.v[v];
    const int HW = vp.W * vp.H;
    const int base = blockIdx.x * kLossThreads * kLossItems;
    if (base >= HW) return;
    const float* c = img.color + 3 * (size_t)vp.pix_base;
    const float* t = tc + 3 * (size_t)vp.pix_base;
    const float* d = img.depth + vp.pix_base;
    const float* t1 = td + vp.pix_base;
    float sc = 0.f, sd = 0.f, nv = 0.f;
#pragma unroll
    for (int k = 0; k < kLossItems; k++) {
        const int p = base + k * kLossThreads + threadIdx.x;
        if (p < HW) {
            sc += fabsf(c[p] - t[p]) + fabsf(c[HW + p] - t[HW + p]) + fabsf(c[2 * HW + p] - t[2 * HW + p]);
            const float tdv = t1[p];
            if (tdv > 0.f) {
                sd += fabsf(d[p] - tdv);
                nv += 1.f;
            }
        }
    }
    __shared__ float s[3][kLossThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { s[0][warp] = sc; s[1][warp] = sd; s[2][warp] = nv; }
    __syncthreads();
    if (threadIdx.x < 3) {
        float x = 0.f;
#pragma unroll
        for (int w = 0; w < kLossThreads / 32; w++) x += s[threadIdx.x][w];
        atomicAdd(acc + 4 * v + threadIdx.x, x);
    }
}

__global__ void __launch_bounds__(kLossThreads) k_loss_grad(gs_image img, const float* __restrict__ tc,
                                                           const float* __restrict__ td, Views views,
                                                           const float* __restrict__ acc, float lc, float ld,
                                                           float* __restrict__ dc, float* __restrict__ dd,
                                                           float* __restrict__ terms) {
    pdl_enter();
    const int v = blockIdx.y;
    const ViewParams& vp = views.v[v];
    const int HW = vp.W * vp.H;
    const int base = blockIdx.x * kLossThreads * kLossItems;
    if (base >= HW) return;
    const float nvalid = acc[4 * v + 2];
    const float kc = lc / (3.0f * (float)HW);
    const float kd = nvalid > 0.f ? ld / nvalid : 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        terms[2 * v] = acc[4 * v] / (3.0f * (float)HW);
        terms[2 * v + 1] = nvalid > 0.f ? acc[4 * v + 1] / nvalid : 0.f;
    }
    const float* c = img.color + 3 * (size_t)vp.pix_base;
    const float* t = tc + 3 * (size_t)vp.pix_base;
    float* g = dc + 3 * (size_t)vp.pix_base;
#pragma unroll
    for (int k = 0; k < kLossItems; k++) {
        const int p = base + k * kLossThreads + threadIdx.x;
        if (p < HW) {
            g[p] = kc * sgnf(c[p] - t[p]);
            g[HW + p] = kc * sgnf(c[HW + p] - t[HW + p]);
            g[2 * HW + p] = kc * sgnf(c[2 * HW + p] - t[2 * HW + p]);
            const float tdv = td[vp.pix_base + p];
            dd[vp.pix_base + p] = tdv > 0.f ? kd * sgnf(img.depth[vp.pix_base + p] - tdv) : 0.f;
        }
    }
}

struct AdamArgs {
    gs_adam_group g[8];
    int64_t chunk_end[8];      // cumulative float4 chunks per group
    int vec[8];                // the group's four arrays are 16-byte aligned (float4 loads and stores)
    int n_groups;
    float b1, b2, eps;
    int32_t* d_step;
    unsigned total_blocks;
};

constexpr int kAdamThreads = 256;

__device__ __forceinline__ void adam_elem(float& p, float g, float& m, float& v, float b1, float b2, float ib1,
                                          float ib2, float lr, float rbc1, float rbc2, float eps) {
    m = b1 * m + ib1 * g;
    v = b2 * v + ib2 * g * g;
    // fast division (numerator times the approximate reciprocal, within 2 ulp), IEEE square root
    p -= lr * __fdividef(m * rbc1, __fsqrt_rn(v * rbc2) + eps);
}

// One float4 chunk c of the concatenated groups.
__device__ __forceinline__ void adam_chunk(const AdamArgs& args, int64_t c, float b1, float b2, float ib1, float ib2,
                                           float rbc1, float rbc2, float eps) {
    int k = 0;
    while (c >= args.chunk_end[k]) k++;
    const gs_adam_group& G = args.g[k];
    const int64_t i0 = 4 * (c - (k ? args.chunk_end[k - 1] : 0));
    const float lr = G.lr;
    if (args.vec[k] && i0 + 3 < G.n) {
        float4 p = *reinterpret_cast<const float4*>(G.param + i0);
        const float4 g = *reinterpret_cast<const float4*>(G.grad + i0);
        float4 m = *reinterpret_cast<const float4*>(G.m + i0);
        float4 v = *reinterpret_cast<const float4*>(G.v + i0);
        adam_elem(p.x, g.x, m.x, v.x, b1, b2, ib1, ib2, lr, rbc1, rbc2, eps);
        adam_elem(p.y, g.y, m.y, v.y, b1, b2, ib1, ib2, lr, rbc1, rbc2, eps);
        adam_elem(p.z, g.z, m.z, v.z, b1, b2, ib1, ib2, lr, rbc1, rbc2, eps);
        adam_elem(p.w, g.w, m.w, v.w, b1, b2, ib1, ib2, lr, rbc1, rbc2, eps);
        *reinterpret_cast<float4*>(G.param + i0) = p;
        *reinterpret_cast<float4*>(G.m + i0) = m;
        *reinterpret_cast<float4*>(G.v + i0) = v;
    } else {
        for (int64_t i = i0; i < i0 + 4 && i < G.n; i++) {
            float p = G.param[i], m = G.m[i], v = G.v[i];
            adam_elem(p, G.grad[i], m, v, b1, b2, ib1, ib2, lr, rbc1, rbc2, eps);
            G.param[i] = p; G.m[i] = m; G.v[i] = v;
        }
    }
}

// Grid-stride over 4-element chunks of all groups, two chunks per thread and
// round (their loads in flight together); the last block to finish advances the
// device step counter (each block reads it before finishing).
__global__ void __launch_bounds__(kAdamThreads, 4) k_adam(AdamArgs args) {
    __shared__ float s_bc[2];
    __shared__ int s_t;
    pdl_enter();
    if (threadIdx.x == 0) {
        const int t = args.d_step[0] + 1;
        s_t = t;
        s_bc[0] = 1.0f / (1.0f - powf(args.b1, (float)t));
        s_bc[1] = 1.0f / (1.0f - powf(args.b2, (float)t));
    }
    __syncthreads();
    const float rbc1 = s_bc[0], rbc2 = s_bc[1];
    const float b1 = args.b1, b2 = args.b2, eps = args.eps;
    const float ib1 = 1.0f - b1, ib2 = 1.0f - b2;
    const int64_t total = args.chunk_end[args.n_groups - 1];
    const int64_t stride = (int64_t)gridDim.x * kAdamThreads;
    for (int64_t c = (int64_t)blockIdx.x * kAdamThreads + threadIdx.x; c < total; c += 2 * stride) {
        const int64_t c1 = c + stride;
        const bool has1 = c1 < total;
        int k0 = 0, k1 = 0;
        while (c >= args.chunk_end[k0]) k0++;
        if (has1)
            while (c1 >= args.chunk_end[k1]) k1++;
        const gs_adam_group& G0 = args.g[k0];
        const gs_adam_group& G1 = args.g[k1];
        const int64_t i0 = 4 * (c - (k0 ? args.chunk_end[k0 - 1] : 0));
        const int64_t i1 = has1 ? 4 * (c1 - (k1 ? args.chunk_end[k1 - 1] : 0)) : 0;
        const bool vec0 = args.vec[k0] && i0 + 3 < G0.n;
        const bool vec1 = has1 && args.vec[k1] && i1 + 3 < G1.n;
        if (vec0 && vec1) {
            // both chunks' loads issued before any store
            float4 p0 = *reinterpret_cast<const float4*>(G0.param + i0);
            const float4 g0 = *reinterpret_cast<const float4*>(G0.grad + i0);
            float4 m0 = *reinterpret_cast<const float4*>(G0.m + i0);
            float4 v0 = *reinterpret_cast<const float4*>(G0.v + i0);
            float4 p1 = *reinterpret_cast<const float4*>(G1.param + i1);
            const float4 g1 = *reinterpret_cast<const float4*>(G1.grad + i1);
            float4 m1 = *reinterpret_cast<const float4*>(G1.m + i1);
            float4 v1 = *reinterpret_cast<const float4*>(G1.v + i1);
            const float lr0 = G0.lr, lr1 = G1.lr;
            adam_elem(p0.x, g0.x, m0.x, v0.x, b1, b2, ib1, ib2, lr0, rbc1, rbc2, eps);
            adam_elem(p0.y, g0.y, m0.y, v0.y, b1, b2, ib1, ib2, lr0, rbc1, rbc2, eps);
            adam_elem(p0.z, g0.z, m0.z, v0.z, b1, b2, ib1, ib2, lr0, rbc1, rbc2, eps);
            adam_elem(p0.w, g0.w, m0.w, v0.w, b1, b2, ib1, ib2, lr0, rbc1, rbc2, eps);
            adam_elem(p1.x, g1.x, m1.x, v1.x, b1, b2, ib1, ib2, lr1, rbc1, rbc2, eps);
            adam_elem(p1.y, g1.y, m1.y, v1.y, b1, b2, ib1, ib2, lr1, rbc1, rbc2, eps);
            adam_elem(p1.z, g1.z, m1.z, v1.z, b1, b2, ib1, ib2, lr1, rbc1, rbc2, eps);
            adam_elem(p1.w, g1.w, m1.w, v1.w, b1, b2, ib1, ib2, lr1, rbc1, rbc2, eps);
            *reinterpret_cast<float4*>(G0.param + i0) = p0;
            *reinterpret_cast<float4*>(G0.m + i0) = m0;
            *reinterpret_cast<float4*>(G0.v + i0) = v0;
            *reinterpret_cast<float4*>(G1.param + i1) = p1;
            *reinterpret_cast<float4*>(G1.m + i1) = m1;
            *reinterpret_cast<float4*>(G1.v + i1) = v1;
        } else {
            adam_chunk(args, c, b1, b2, ib1, ib2, rbc1, rbc2, eps);
            if (has1) adam_chunk(args, c1, b1, b2, ib1, ib2, rbc1, rbc2, eps);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(reinterpret_cast<unsigned*>(args.d_step + 1), 1u);
        if (prev == args.total_blocks - 1) {
            args.d_step[0] = s_t;
            args.d_step[1] = 0;
            __threadfence();
        }
    }
}

// Zero-fill of up to three float buffers (float4 stores for a 16-byte aligned
// first buffer): the accumulators a following kernel adds into.  A kernel rather
// than memset nodes, so that the launch chain stays programmatic.
__global__ void __launch_bounds__(256) k_zero(float* a, int64_t na, float* b, int64_t nb, float* c, int64_t nc) {
    pdl_enter();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(a) & 15u) == 0) {
        head = na / 4 * 4;
        for (int64_t k = t0; k < na / 4; k += stride) reinterpret_cast<float4*>(a)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int64_t k = head + t0; k < na; k += stride) a[k] = 0.f;
    for (int64_t k = t0; k < nb; k += stride) b[k] = 0.f;
    for (int64_t k = t0; k < nc; k += stride) c[k] = 0.f;
}

}  // namespace

cudaError_t launch_zero(float* a, int64_t na, float* b, int64_t nb, float* c, int64_t nc, cudaStream_t s) {
    if (a == nullptr) na = 0;
    if (b == nullptr) nb = 0;
    if (c == nullptr) nc = 0;
    int64_t work = na / 4 + 4;
    if (nb > work) work = nb;
    if (nc > work) work = nc;
    if (na + nb + nc == 0) return cudaSuccess;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = ceil_div(work, 256), cap = 4 * (int64_t)sms;
    const cudaError_t e = launch_pdl(k_zero, (unsigned)(want < cap ? want : cap), 256, 0, s, a, na, b, nb, c, nc);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

size_t loss_workspace(int32_t n_views) { return align_up(sizeof(float) * 4 * (size_t)n_views, 256); }

cudaError_t launch_loss(const gs_image& img, const float* tc, const float* td, const Views& views, float lc, float ld,
                        float* dc, float* dd, float* terms, void* ws, cudaStream_t s) {
    float* acc = static_cast<float*>(ws);
    cudaError_t err = launch_zero(acc, 4 * (int64_t)views.n, nullptr, 0, nullptr, 0, s);
    if (err != cudaSuccess) return err;
    int max_hw = 0;
    for (int v = 0; v < views.n; v++) max_hw = max(max_hw, views.v[v].W * views.v[v].H);
    dim3 grid((unsigned)ceil_div(max_hw, kLossThreads * kLossItems), (unsigned)views.n);
    err = launch_pdl(k_loss_reduce, grid, kLossThreads, 0, s, img, tc, td, views, acc);
    if (err == cudaSuccess)
        err = launch_pdl(k_loss_grad, grid, kLossThreads, 0, s, img, tc, td, views, acc, lc, ld, dc, dd, terms);
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

// ------------------------------------------------ allocation-free loss variant
//
// gs_loss_noalloc keeps the per-view accumulators that gs_loss places in the
// caller's workspace in this file-scope device array instead.  Every device
// that loads the library holds it (4 floats per view, GS_NOALLOC_LOSS_MAX_VIEWS
// views, 512 bytes) until the process exits.  Host code cannot use the array's
// name as a device address, so its address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
static __device__ __align__(256) float g_noalloc_loss_scratch[4 * GS_NOALLOC_LOSS_MAX_VIEWS];

constexpr int kMaxDevices = 64;
static float* g_noalloc_loss_ptr[kMaxDevices] = {};
static std::mutex g_noalloc_loss_mutex;

cudaError_t noalloc_loss_scratch(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_loss_mutex);
    if (g_noalloc_loss_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_loss_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_loss_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_noalloc_loss_ptr[dev];
    return cudaSuccess;
}

cudaError_t launch_adam(const gs_adam_group* groups, int n_groups, float b1, float b2, float eps, int32_t* d_step,
                        cudaStream_t s) {
    AdamArgs a;
    int64_t run = 0;
    for (int k = 0; k < 8; k++) {
        a.g[k] = k < n_groups ? groups[k] : gs_adam_group{};
        if (k < n_groups) run += ceil_div(groups[k].n, 4);
        a.chunk_end[k] = run;
        const gs_adam_group& G = a.g[k];
        a.vec[k] = ((reinterpret_cast<uintptr_t>(G.param) | reinterpret_cast<uintptr_t>(G.grad) |
                     reinterpret_cast<uintptr_t>(G.m) | reinterpret_cast<uintptr_t>(G.v)) & 15u) == 0;
    }
    a.n_groups = n_groups;
    a.b1 = b1; a.b2 = b2; a.eps = eps;
    a.d_step = d_step;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = ceil_div(run > 0 ? run : 1, kAdamThreads);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adam, kAdamThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int64_t full = (int64_t)per_sm * sms;                                // one resident wave
    const unsigned blocks = (unsigned)(want < full ? want : full);
    a.total_blocks = blocks;
    const cudaError_t e = launch_pdl(k_adam, blocks, kAdamThreads, 0, s, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gs
