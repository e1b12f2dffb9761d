// raster.cu -- front-to-back alpha compositing of colour and depth (Sec. 3.3:
// a pixel's colour is the alpha blend of the Gaussians covering it, and the
// mapper renders both colour and depth per keyframe) and its backward pass.
//
// One CTA per tile, one thread per pixel.  The tile's depth-sorted splats are
// staged through shared memory in batches (one splat per thread, coalesced
// gathers of float2/float4 rows), then every pixel walks the batch with
// broadcast shared-memory reads.  The CTA leaves as soon as all its pixels are
// saturated.
//
// The backward pass walks each tile's list back to front from the per-pixel
// checkpoint (T_final, n_contrib) written by the forward pass: it rebuilds the
// transmittance before each splat by T_before = T_after / (1 - alpha) and keeps
// the colour/depth "behind" a splat as a running normalised sum, so no
// per-splat state is stored by the forward pass.  Per-splat gradients are
// summed over the 32 pixels of a warp by a transposed butterfly (10 values in
// 12 shuffles, each lane ends with one finished sum), accumulated per tile in
// shared memory, and flushed with one vector atomic per (tile, splat).
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ int view_of_tile(const Views& views, int g) {
    int v = 0;
    for (int k = 1; k < views.n; k++)
        if (g >= views.v[k].tile_base) v = k;
    return v;
}

template <int T>
__global__ void __launch_bounds__(T * T) k_render_fwd(const float2* __restrict__ xy, const float4* __restrict__ conic_o,
                                                     const float4* __restrict__ rgbd, const uint32_t* __restrict__ vals,
                                                     const uint2* __restrict__ ranges, Views views, RenderConsts rc,
                                                     gs_image img) {
    constexpr int B = T * T;
    __shared__ float2 s_xy[B];
    __shared__ float4 s_q[B];
    __shared__ float4 s_cd[B];
    const int g = blockIdx.x;
    const int v = view_of_tile(views, g);
    const ViewParams& vp = views.v[v];
    const int lt = g - vp.tile_base;
    const int tx = lt % vp.tiles_x, ty = lt / vp.tiles_x;
    const int px = tx * T + (threadIdx.x % T), py = ty * T + (threadIdx.x / T);
    const bool inside = px < vp.W && py < vp.H;
    const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    const uint2 range = ranges[g];
    const float amin = rc.alpha_min, amax = rc.alpha_max, tcut = rc.T_cut;

    float Tr = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t start = range.x; start < range.y; start += B) {
        if (__syncthreads_count(done) == B) break;
        const uint32_t j = start + threadIdx.x;
        if (j < range.y) {
            const uint32_t e = vals[j];
            const float4 c = conic_o[e];
            float4 q;
            scale_conic(c.x, c.y, c.z, &q.x, &q.y, &q.z);
            q.w = c.w;
            s_xy[threadIdx.x] = xy[e];
            s_q[threadIdx.x] = q;
            s_cd[threadIdx.x] = rgbd[e];
        }
        __syncthreads();
        const int cnt = min((uint32_t)B, range.y - start);
        if (!done) {
            for (int k = 0; k < cnt; k++) {
                const float2 m = s_xy[k];
                const float4 q = s_q[k];
                const float dx = __fsub_rn(sx, m.x), dy = __fsub_rn(sy, m.y);
                const float p2 = splat_power2(q.x, q.y, q.z, dx, dy);
                if (p2 > 0.f) continue;
                const float a = fminf(amax, __fmul_rn(q.w, splat_weight(p2)));
                if (a < amin) continue;
                const float test = __fmaf_rn(-a, Tr, Tr);
                if (test < tcut) { done = true; break; }
                const float4 cd = s_cd[k];
                const float w = __fmul_rn(a, Tr);
                cr = __fmaf_rn(cd.x, w, cr);
                cg = __fmaf_rn(cd.y, w, cg);
                cb = __fmaf_rn(cd.z, w, cb);
                dd = __fmaf_rn(cd.w, w, dd);
                Tr = test;
                last = start - range.x + (uint32_t)k + 1u;
            }
        }
    }
    if (inside) {
        const int HW = vp.W * vp.H;
        const int pix = py * vp.W + px;
        float* col = img.color + 3 * (size_t)vp.pix_base;
        col[pix] = cr + Tr * rc.bg[0];
        col[HW + pix] = cg + Tr * rc.bg[1];
        col[2 * HW + pix] = cb + Tr * rc.bg[2];
        img.depth[vp.pix_base + pix] = dd;
        img.T_final[vp.pix_base + pix] = Tr;
        img.n_contrib[vp.pix_base + pix] = last;
    }
}

// Warp sum of 10 values by a transposed butterfly: after 12 shuffles lane l
// (l even) holds the full sum of value 5*b4 + (3*b3 + 2*b2 + b1) when that slot
// is valid, and adds it into acc[slot].
__device__ __forceinline__ void warp_reduce10_add(const float (&v)[10], float* acc, int lane) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1, b0 = lane & 1;
    float r[6];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const float keep = b4 ? v[j + 5] : v[j];
        const float send = b4 ? v[j] : v[j + 5];
        r[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
    r[5] = 0.f;
    float s[4];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float keep = b3 ? r[j + 3] : r[j];
        const float send = b3 ? r[j] : r[j + 3];
        s[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    s[3] = 0.f;
    float t[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const float keep = b2 ? s[j + 2] : s[j];
        const float send = b2 ? s[j] : s[j + 2];
        t[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float u;
    {
        const float keep = b1 ? t[1] : t[0];
        const float send = b1 ? t[0] : t[1];
        u = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    u += __shfl_xor_sync(0xffffffffu, u, 1);
    const int k = 3 * b3 + 2 * b2 + b1;
    if (b0 == 0 && (2 * b2 + b1) < 3 && k < 5) atomicAdd(acc + 5 * b4 + k, u);
}

template <int T>
__global__ void __launch_bounds__(T * T) k_render_bwd(const float2* __restrict__ xy, const float4* __restrict__ conic_o,
                                                     const float4* __restrict__ rgbd, const uint32_t* __restrict__ vals,
                                                     const uint2* __restrict__ ranges, Views views, RenderConsts rc,
                                                     const float* __restrict__ T_final,
                                                     const uint32_t* __restrict__ n_contrib,
                                                     const float* __restrict__ dL_dcolor,
                                                     const float* __restrict__ dL_ddepth, float* __restrict__ g2d) {
    constexpr int NT = T * T;
    constexpr int B = NT < 256 ? NT : 256;
    __shared__ float2 s_xy[B];
    __shared__ float4 s_q[B];      // scaled conic + opacity
    __shared__ float4 s_c[B];      // raw conic A, B, C
    __shared__ float4 s_cd[B];     // r, g, b, z
    __shared__ uint32_t s_e[B];
    __shared__ float s_acc[B * 10];
    __shared__ uint32_t s_maxn;
    const int g = blockIdx.x;
    const int v = view_of_tile(views, g);
    const ViewParams& vp = views.v[v];
    const int lt = g - vp.tile_base;
    const int tx = lt % vp.tiles_x, ty = lt / vp.tiles_x;
    const int px = tx * T + (threadIdx.x % T), py = ty * T + (threadIdx.x / T);
    const bool inside = px < vp.W && py < vp.H;
    const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    const uint2 range = ranges[g];
    const int lane = threadIdx.x & 31;
    const float amin = rc.alpha_min, amax = rc.alpha_max;

    float Tr = 1.f, gcr = 0.f, gcg = 0.f, gcb = 0.f, gd = 0.f;
    uint32_t np = 0;
    if (inside) {
        const int HW = vp.W * vp.H;
        const int pix = py * vp.W + px;
        Tr = T_final[vp.pix_base + pix];
        np = n_contrib[vp.pix_base + pix];
        const float* dc = dL_dcolor + 3 * (size_t)vp.pix_base;
        gcr = dc[pix];
        gcg = dc[HW + pix];
        gcb = dc[2 * HW + pix];
        gd = dL_ddepth[vp.pix_base + pix];
    }
    if (threadIdx.x == 0) s_maxn = 0u;
    __syncthreads();
    if (np > 0) atomicMax(&s_maxn, np);
    __syncthreads();
    const uint32_t list_end = min(range.x + s_maxn, range.y);   // a checkpoint never points past the list
    // colour / depth behind the current splat, normalised by the transmittance after it
    float Sr = rc.bg[0], Sg = rc.bg[1], Sb = rc.bg[2], Sd = 0.f;

    for (int64_t bend = list_end; bend > (int64_t)range.x; bend -= B) {
        const uint32_t bstart = (uint32_t)(bend - B > (int64_t)range.x ? bend - B : (int64_t)range.x);
        const int cnt = (int)(bend - bstart);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const uint32_t e = vals[bstart + threadIdx.x];
            const float4 c = conic_o[e];
            float4 q;
            scale_conic(c.x, c.y, c.z, &q.x, &q.y, &q.z);
            q.w = c.w;
            s_xy[threadIdx.x] = xy[e];
            s_q[threadIdx.x] = q;
            s_c[threadIdx.x] = c;
            s_cd[threadIdx.x] = rgbd[e];
            s_e[threadIdx.x] = e;
#pragma unroll
            for (int k = 0; k < 10; k++) s_acc[threadIdx.x * 10 + k] = 0.f;
        }
        __syncthreads();
        for (int k = cnt - 1; k >= 0; k--) {
            const uint32_t pos = bstart + (uint32_t)k - range.x;   // position in the tile list
            bool contrib = pos < np;
            float gv[10];
#pragma unroll
            for (int q = 0; q < 10; q++) gv[q] = 0.f;
            if (contrib) {
                const float2 m = s_xy[k];
                const float4 q = s_q[k];
                const float dx = __fsub_rn(sx, m.x), dy = __fsub_rn(sy, m.y);
                const float p2 = splat_power2(q.x, q.y, q.z, dx, dy);
                float G = 0.f, araw = 0.f, a = 0.f;
                if (p2 > 0.f) {
                    contrib = false;
                } else {
                    G = splat_weight(p2);
                    araw = __fmul_rn(q.w, G);
                    a = fminf(amax, araw);
                    if (a < amin) contrib = false;
                }
                if (contrib) {
                    const float4 cd = s_cd[k];
                    const float one_m = 1.0f - a;
                    const float Tb = Tr / one_m;
                    const float w = a * Tb;
                    const float dLda = Tb * ((cd.x - Sr) * gcr + (cd.y - Sg) * gcg + (cd.z - Sb) * gcb + (cd.w - Sd) * gd);
                    Sr = a * cd.x + one_m * Sr;
                    Sg = a * cd.y + one_m * Sg;
                    Sb = a * cd.z + one_m * Sb;
                    Sd = a * cd.w + one_m * Sd;
                    Tr = Tb;
                    gv[7] = gcr * w;
                    gv[8] = gcg * w;
                    gv[9] = gcb * w;
                    gv[6] = gd * w;
                    if (araw < amax) {
                        const float4 c = s_c[k];
                        const float dpow = dLda * a;          // d alpha / d power = alpha
                        gv[5] = dLda * G;                     // d alpha / d o = exp(power)
                        gv[0] = dpow * (c.x * dx + c.y * dy);
                        gv[1] = dpow * (c.y * dx + c.z * dy);
                        gv[2] = -0.5f * dpow * dx * dx;
                        gv[3] = -dpow * dx * dy;
                        gv[4] = -0.5f * dpow * dy * dy;
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) warp_reduce10_add(gv, s_acc + k * 10, lane);
        }
        __syncthreads();
        if (threadIdx.x < cnt) {
            const float* a = s_acc + threadIdx.x * 10;
            bool any = false;
#pragma unroll
            for (int k = 0; k < 10; k++) any |= (a[k] != 0.f);
            if (any) {
                float4* dst = reinterpret_cast<float4*>(g2d) + 3 * (size_t)s_e[threadIdx.x];
                atomicAdd(dst, make_float4(a[0], a[1], a[2], a[3]));
                atomicAdd(dst + 1, make_float4(a[4], a[5], a[6], 0.f));
                atomicAdd(dst + 2, make_float4(a[7], a[8], a[9], 0.f));
            }
        }
    }
}

}  // namespace

cudaError_t launch_render_fwd(const gs_projected& pr, const gs_bins& bins, const Views& views,
                              const RenderConsts& rc, const gs_image& img, cudaStream_t s) {
    const int grid = views.total_tiles;
    if (grid == 0) return cudaSuccess;
    const float2* xy = reinterpret_cast<const float2*>(pr.xy);
    const float4* co = reinterpret_cast<const float4*>(pr.conic_o);
    const float4* cd = reinterpret_cast<const float4*>(pr.rgbd);
    const uint2* rg = reinterpret_cast<const uint2*>(bins.ranges);
    switch (rc.tile) {
        case 8: k_render_fwd<8><<<grid, 64, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img); break;
        case 16: k_render_fwd<16><<<grid, 256, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img); break;
        case 32: k_render_fwd<32><<<grid, 1024, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_projected& pr, const gs_bins& bins, const gs_image& img, const float* dc,
                              const float* dd, const Views& views, const RenderConsts& rc, float* g2d, cudaStream_t s) {
    const int grid = views.total_tiles;
    if (grid == 0) return cudaSuccess;
    const float2* xy = reinterpret_cast<const float2*>(pr.xy);
    const float4* co = reinterpret_cast<const float4*>(pr.conic_o);
    const float4* cd = reinterpret_cast<const float4*>(pr.rgbd);
    const uint2* rg = reinterpret_cast<const uint2*>(bins.ranges);
    switch (rc.tile) {
        case 8:
            k_render_bwd<8><<<grid, 64, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d);
            break;
        case 16:
            k_render_bwd<16><<<grid, 256, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d);
            break;
        case 32:
            k_render_bwd<32><<<grid, 1024, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gs
