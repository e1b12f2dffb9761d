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

// Thread layout: a tile of T x T pixels is split into 8 x 8 blocks, one warp
// per block; lane l covers column l % 8 and rows l / 8 and l / 8 + 4 of its
// block (two pixels per lane), so a warp's pixels are spatially compact and
// tend to saturate together.
template <int T>
struct TileShape {
    static constexpr int kWarps = (T / 8) * (T / 8);
    static constexpr int kThreads = kWarps * 32;
};

__device__ __forceinline__ void lane_pixels(int T, int tid, int* x, int* y0) {
    const int w = tid >> 5, l = tid & 31;
    const int bx = w % (T / 8), by = w / (T / 8);
    *x = bx * 8 + (l & 7);
    *y0 = by * 8 + (l >> 3);
}

// Forward state of one pixel.
struct FwdPix {
    float T, r, g, b, d;
    uint32_t last;
    bool done;
};

__device__ __forceinline__ void fwd_pixel(FwdPix& P, float dx, float sy, float2 m, float4 q, const float4* cd,
                                          float amin, float amax, float tcut, uint32_t pos) {
    if (P.done) return;
    const float dy = __fsub_rn(sy, m.y);
    const float p2 = splat_power2(q.x, q.y, q.z, dx, dy);
    if (p2 > 0.f) return;
    const float a = fminf(amax, __fmul_rn(q.w, splat_weight(p2)));
    if (a < amin) return;
    const float test = __fmaf_rn(-a, P.T, P.T);
    if (test < tcut) { P.done = true; return; }
    const float4 c = *cd;
    const float w = __fmul_rn(a, P.T);
    P.r = __fmaf_rn(c.x, w, P.r);
    P.g = __fmaf_rn(c.y, w, P.g);
    P.b = __fmaf_rn(c.z, w, P.b);
    P.d = __fmaf_rn(c.w, w, P.d);
    P.T = test;
    P.last = pos + 1u;
}

template <int T>
__global__ void __launch_bounds__(TileShape<T>::kThreads) k_render_fwd(
        const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
        const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, Views views, RenderConsts rc,
        gs_image img) {
    constexpr int NT = TileShape<T>::kThreads;
    constexpr int B = 2 * NT < 1024 ? 2 * NT : 1024;   // splats per shared-memory batch
    __shared__ float2 s_xy[B];
    __shared__ float4 s_q[B];
    __shared__ float4 s_cd[B];
    const int g = blockIdx.x;
    const int v = view_of_tile(views, g);
    const ViewParams& vp = views.v[v];
    const int lt = g - vp.tile_base;
    const int tx = lt % vp.tiles_x, ty = lt / vp.tiles_x;
    int ox, oy;
    lane_pixels(T, threadIdx.x, &ox, &oy);
    const int px = tx * T + ox, py0 = ty * T + oy, py1 = py0 + 4;
    const bool in0 = px < vp.W && py0 < vp.H, in1 = px < vp.W && py1 < vp.H;
    const float sx = (float)px + 0.5f, sy0 = (float)py0 + 0.5f, sy1 = (float)py1 + 0.5f;
    const uint2 range = ranges[g];
    const float amin = rc.alpha_min, amax = rc.alpha_max, tcut = rc.T_cut;

    FwdPix P0 = {1.f, 0.f, 0.f, 0.f, 0.f, 0u, !in0};
    FwdPix P1 = {1.f, 0.f, 0.f, 0.f, 0.f, 0u, !in1};
    for (uint32_t start = range.x; start < range.y; start += B) {
        if (__syncthreads_count(P0.done && P1.done) == NT) break;
        for (int k = threadIdx.x; k < B; k += NT) {
            const uint32_t j = start + k;
            if (j < range.y) {
                const uint32_t e = vals[j];
                const float4 c = conic_o[e];
                float4 q;
                scale_conic(c.x, c.y, c.z, &q.x, &q.y, &q.z);
                q.w = c.w;
                s_xy[k] = xy[e];
                s_q[k] = q;
                s_cd[k] = rgbd[e];
            }
        }
        __syncthreads();
        const int cnt = min((uint32_t)B, range.y - start);
        if (__any_sync(0xffffffffu, !(P0.done && P1.done))) {
            for (int k = 0; k < cnt; k++) {
                const float2 m = s_xy[k];
                const float4 q = s_q[k];
                const float dx = __fsub_rn(sx, m.x);
                const uint32_t pos = start - range.x + (uint32_t)k;
                fwd_pixel(P0, dx, sy0, m, q, &s_cd[k], amin, amax, tcut, pos);
                fwd_pixel(P1, dx, sy1, m, q, &s_cd[k], amin, amax, tcut, pos);
                if ((k & 15) == 15 && __all_sync(0xffffffffu, P0.done && P1.done)) break;
            }
        }
    }
    const int HW = vp.W * vp.H;
    float* col = img.color + 3 * (size_t)vp.pix_base;
    if (in0) {
        const int pix = py0 * vp.W + px;
        col[pix] = P0.r + P0.T * rc.bg[0];
        col[HW + pix] = P0.g + P0.T * rc.bg[1];
        col[2 * HW + pix] = P0.b + P0.T * rc.bg[2];
        img.depth[vp.pix_base + pix] = P0.d;
        img.T_final[vp.pix_base + pix] = P0.T;
        img.n_contrib[vp.pix_base + pix] = P0.last;
    }
    if (in1) {
        const int pix = py1 * vp.W + px;
        col[pix] = P1.r + P1.T * rc.bg[0];
        col[HW + pix] = P1.g + P1.T * rc.bg[1];
        col[2 * HW + pix] = P1.b + P1.T * rc.bg[2];
        img.depth[vp.pix_base + pix] = P1.d;
        img.T_final[vp.pix_base + pix] = P1.T;
        img.n_contrib[vp.pix_base + pix] = P1.last;
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

// Gradient slots per splat: 0 d mx, 1 d my, 2 d A, 3 d B, 4 d C, 5 d o, 6 d z,
// 7..9 d rgb.  The flush writes them as the three float4 rows of grad2d.
// Backward state of one pixel: transmittance after the current splat, the
// image gradients and the colour/depth behind the current splat normalised by
// that transmittance.
struct BwdPix {
    float T;
    uint32_t np;
    float gr, gg, gb, gd;
    float Sr, Sg, Sb, Sd;
};

__device__ __forceinline__ bool bwd_pixel(BwdPix& P, float dx, float sy, float2 m, float4 q, float4 c, float4 cd,
                                          float amin, float amax, uint32_t pos, float (&gv)[10]) {
    if (pos >= P.np) return false;
    const float dy = __fsub_rn(sy, m.y);
    const float p2 = splat_power2(q.x, q.y, q.z, dx, dy);
    if (p2 > 0.f) return false;
    const float G = splat_weight(p2);
    const float araw = __fmul_rn(q.w, G);
    const float a = fminf(amax, araw);
    if (a < amin) return false;
    const float one_m = 1.0f - a;
    const float Tb = __fdividef(P.T, one_m);      // transmittance before this splat
    const float w = a * Tb;
    const float dr = cd.x - P.Sr, dg = cd.y - P.Sg, db = cd.z - P.Sb, dz = cd.w - P.Sd;
    const float dLda = Tb * (dr * P.gr + dg * P.gg + db * P.gb + dz * P.gd);
    P.Sr = fmaf(a, dr, P.Sr);
    P.Sg = fmaf(a, dg, P.Sg);
    P.Sb = fmaf(a, db, P.Sb);
    P.Sd = fmaf(a, dz, P.Sd);
    P.T = Tb;
    gv[7] = fmaf(P.gr, w, gv[7]);
    gv[8] = fmaf(P.gg, w, gv[8]);
    gv[9] = fmaf(P.gb, w, gv[9]);
    gv[6] = fmaf(P.gd, w, gv[6]);
    if (araw < amax) {                            // alpha not clamped
        const float dpow = dLda * a;              // d alpha / d power = alpha
        gv[5] = fmaf(dLda, G, gv[5]);             // d alpha / d o = exp(power)
        gv[0] = fmaf(dpow, fmaf(c.x, dx, c.y * dy), gv[0]);
        gv[1] = fmaf(dpow, fmaf(c.y, dx, c.z * dy), gv[1]);
        const float hx = -0.5f * dpow * dx;
        gv[2] = fmaf(hx, dx, gv[2]);
        gv[3] = fmaf(-dpow * dx, dy, gv[3]);
        gv[4] = fmaf(-0.5f * dpow * dy, dy, gv[4]);
    }
    return true;
}

template <int T>
__global__ void __launch_bounds__(TileShape<T>::kThreads) k_render_bwd(
        const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
        const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges, Views views, RenderConsts rc,
        const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
        const float* __restrict__ dL_dcolor, const float* __restrict__ dL_ddepth, float* __restrict__ g2d) {
    constexpr int NT = TileShape<T>::kThreads;
    constexpr int B = 2 * NT < 256 ? 2 * NT : 256;
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
    int ox, oy;
    lane_pixels(T, threadIdx.x, &ox, &oy);
    const int px = tx * T + ox, py0 = ty * T + oy, py1 = py0 + 4;
    const bool in0 = px < vp.W && py0 < vp.H, in1 = px < vp.W && py1 < vp.H;
    const float sx = (float)px + 0.5f, sy0 = (float)py0 + 0.5f, sy1 = (float)py1 + 0.5f;
    const uint2 range = ranges[g];
    const int lane = threadIdx.x & 31;
    const float amin = rc.alpha_min, amax = rc.alpha_max;
    const int HW = vp.W * vp.H;
    const float* dc = dL_dcolor + 3 * (size_t)vp.pix_base;

    BwdPix P0, P1;
    P0.np = 0; P1.np = 0; P0.T = 1.f; P1.T = 1.f;
    P0.gr = P0.gg = P0.gb = P0.gd = 0.f;
    P1.gr = P1.gg = P1.gb = P1.gd = 0.f;
    P0.Sr = P1.Sr = rc.bg[0]; P0.Sg = P1.Sg = rc.bg[1]; P0.Sb = P1.Sb = rc.bg[2]; P0.Sd = P1.Sd = 0.f;
    if (in0) {
        const int pix = py0 * vp.W + px;
        P0.T = T_final[vp.pix_base + pix];
        P0.np = n_contrib[vp.pix_base + pix];
        P0.gr = dc[pix]; P0.gg = dc[HW + pix]; P0.gb = dc[2 * HW + pix];
        P0.gd = dL_ddepth[vp.pix_base + pix];
    }
    if (in1) {
        const int pix = py1 * vp.W + px;
        P1.T = T_final[vp.pix_base + pix];
        P1.np = n_contrib[vp.pix_base + pix];
        P1.gr = dc[pix]; P1.gg = dc[HW + pix]; P1.gb = dc[2 * HW + pix];
        P1.gd = dL_ddepth[vp.pix_base + pix];
    }
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(P0.np, P1.np));   // this warp's deepest pixel
    if (threadIdx.x == 0) s_maxn = 0u;
    __syncthreads();
    if (lane == 0 && wmax > 0) atomicMax(&s_maxn, wmax);
    __syncthreads();
    const uint32_t list_end = min(range.x + s_maxn, range.y);   // a checkpoint never points past the list

    for (int64_t bend = list_end; bend > (int64_t)range.x; bend -= B) {
        const uint32_t bstart = (uint32_t)(bend - B > (int64_t)range.x ? bend - B : (int64_t)range.x);
        const int cnt = (int)(bend - bstart);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += NT) {
            const uint32_t e = vals[bstart + k];
            const float4 c = conic_o[e];
            float4 q;
            scale_conic(c.x, c.y, c.z, &q.x, &q.y, &q.z);
            q.w = c.w;
            s_xy[k] = xy[e];
            s_q[k] = q;
            s_c[k] = c;
            s_cd[k] = rgbd[e];
            s_e[k] = e;
#pragma unroll
            for (int r = 0; r < 10; r++) s_acc[k * 10 + r] = 0.f;
        }
        __syncthreads();
        // this warp only needs positions below its deepest pixel
        const int64_t lim = (int64_t)wmax - (int64_t)(bstart - range.x);
        const int kmax = lim < cnt ? (int)(lim > 0 ? lim : 0) : cnt;
        for (int k = kmax - 1; k >= 0; k--) {
            const uint32_t pos = bstart + (uint32_t)k - range.x;
            const float2 m = s_xy[k];
            const float4 q = s_q[k];
            const float4 c = s_c[k];
            const float4 cd = s_cd[k];
            const float dx = __fsub_rn(sx, m.x);
            float gv[10];
#pragma unroll
            for (int r = 0; r < 10; r++) gv[r] = 0.f;
            bool any = bwd_pixel(P0, dx, sy0, m, q, c, cd, amin, amax, pos, gv);
            any |= bwd_pixel(P1, dx, sy1, m, q, c, cd, amin, amax, pos, gv);
            if (__any_sync(0xffffffffu, any)) warp_reduce10_add(gv, s_acc + k * 10, lane);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += NT) {
            const float* a = s_acc + k * 10;
            bool nz = false;
#pragma unroll
            for (int r = 0; r < 10; r++) nz |= (a[r] != 0.f);
            if (nz) {
                float4* dst = reinterpret_cast<float4*>(g2d) + 3 * (size_t)s_e[k];
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
        case 8: k_render_fwd<8><<<grid, TileShape<8>::kThreads, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img); break;
        case 16: k_render_fwd<16><<<grid, TileShape<16>::kThreads, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img); break;
        case 32: k_render_fwd<32><<<grid, TileShape<32>::kThreads, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img); break;
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
            k_render_bwd<8><<<grid, TileShape<8>::kThreads, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d);
            break;
        case 16:
            k_render_bwd<16><<<grid, TileShape<16>::kThreads, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d);
            break;
        case 32:
            k_render_bwd<32><<<grid, TileShape<32>::kThreads, 0, s>>>(xy, co, cd, bins.vals, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gs
