// gs_internal.cuh -- shared definitions of the libgs CUDA translation units.
// Not part of the public ABI (see include/gs.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

// Per-view constants, passed to kernels by value (kernel parameter space).
struct ViewParams {
    float Rcw[9];      // world-to-camera rotation R_wc^T, row-major
    float tcw[3];      // -R_wc^T t_wc
    float centre[3];   // camera centre t_wc (SH viewing direction)
    float fx, fy, cx, cy;
    int32_t W, H;
    int32_t tiles_x, tiles_y;
    int32_t tile_base;  // first global tile of this view
    int32_t pix_base;   // first pixel of this view
};

struct Views {
    int32_t n;
    int32_t total_tiles;
    int32_t total_pixels;
    int32_t pad;
    ViewParams v[GS_MAX_VIEWS];
};

struct RenderConsts {
    int32_t tile;
    float near_plane, alpha_min, alpha_max, T_cut, dilation, radius_sigma;
    float bg[3];
    int32_t sh_degree;
    int32_t splat_stages;   // 0 (library's choice), 2 or 3: see gs_render_params
    int32_t block_masks;    // 1: the rasterisers read gs_bins.masks; 0: they test
};

// Host helpers (api.cu).
bool make_views(const gs_camera* cams, int32_t n_views, int32_t tile, Views* out);
RenderConsts make_consts(const gs_render_params* p);

// Binning plan (api.cu -> binsort.cu).
struct SortPlan {
    int64_t capacity;
    int32_t total_tiles;
    int32_t tile;          // tile size (the block masks)
    float alpha_min;       // the rasterisers' culling threshold (the block masks)
    int32_t block_masks;   // write gs_bins.masks
    int32_t cull_tiles;    // keep only the (entry, tile) pairs whose splat can reach 0.99 alpha_min in the tile
};
SortPlan make_sort_plan(int64_t key_capacity, int32_t total_tiles, int32_t tile, float alpha_min,
                        int32_t block_masks, int32_t cull_tiles);
size_t bin_sort_workspace(int64_t n_entries, int64_t capacity, int32_t total_tiles);

constexpr int kGradStride = 12;                  // floats per entry of the 2D-gradient scratch

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Programmatic dependent launch.  The mapping kernels are launched with
// programmatic stream serialisation, so a kernel's CTAs may be dispatched while
// the previous kernel on the stream drains.  Every such kernel calls pdl_wait()
// (griddepcontrol.wait: returns once every prerequisite grid has completed and
// its memory is visible) before its first global memory access, then
// pdl_trigger() (griddepcontrol.launch_dependents) so that the next kernel can
// be dispatched in turn.  Without a programmatic prerequisite both are no-ops.
#ifdef __CUDACC__
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}
#endif

// Launchers (one translation unit each).
cudaError_t launch_project(const gs_gaussians& g, const Views& views, const RenderConsts& rc,
                           const gs_projected& out, cudaStream_t s, const float* xi = nullptr);
// L2 read-bandwidth probe (binsort.cu): reps grid-stride passes over buf[n], n % 4 == 0
cudaError_t launch_l2_read(const float* buf, int64_t n, int reps, float* out, cudaStream_t s);
cudaError_t launch_bin_sort(const gs_projected& pr, int64_t n_entries, const Views& views,
                            const SortPlan& plan, const gs_bins& bins, void* ws, cudaStream_t s);
// The Eq. 6 colour and depth L1 terms fused into the rasterisers: the forward
// pass sums |I_hat - I|, |D_hat - D| over D > 0 and the count of D > 0 per view
// (per-CTA partials, finished by the last CTA into acc and the loss terms); the
// backward pass forms each pixel's dL/dI_hat and dL/dD_hat from the images and
// those totals instead of reading gradient images.
struct FusedLoss {
    const float* tc;        // target colour, planar per view like gs_image.color
    const float* td;        // target depth
    const float* color;     // rendered colour (read by the backward pass)
    const float* depth;     // rendered depth (read by the backward pass)
    float* partial;         // [forward CTAs][n_views][3]
    float* acc;             // [n_views][4]: sum |I_hat - I|, sum_{D > 0} |D_hat - D|, count D > 0, 0
    float* terms;           // [n_views][2]: L_c, L_d (unweighted means)
    int* ticket;            // zero between launches (the last CTA resets it)
    uint32_t* item_cost;    // [work items] deepest n_contrib of each 8 x 4 block (forward), or null
    uint32_t* order;        // [work items] item order, deepest blocks first (backward; next forward), or null
    uint32_t* order_tag;    // [2] (n, n ^ kOrderTagMagic) once order holds a permutation of n items
    float lc, ld;
};
constexpr int kFusedMaxCtas = 4096;              // bound on a forward raster grid (partial slots)
constexpr int kOrderMaxItems = 65536;            // work items the cost-ordered rasterisers handle
constexpr uint32_t kOrderTagMagic = 0x9E3779B9u;
size_t fused_loss_workspace(int32_t n_views);
// acc, partial, item_cost and order inside a fused-loss workspace
void fused_loss_layout(void* ws, int32_t n_views, FusedLoss* fl);

cudaError_t launch_render_fwd(const gs_projected& pr, const gs_bins& bins, const Views& views,
                              const RenderConsts& rc, const gs_image& img, cudaStream_t s,
                              const FusedLoss* fl = nullptr);
cudaError_t launch_loss(const gs_image& img, const float* tc, const float* td, const Views& views,
                        float lc, float ld, float* dc, float* dd, float* terms, void* ws, cudaStream_t s);
// g2d_zero floats of g2d are zeroed first (the accumulators the backward adds into).
cudaError_t launch_render_bwd(const gs_projected& pr, const gs_bins& bins, const gs_image& img,
                              const float* dc, const float* dd, const Views& views, const RenderConsts& rc,
                              float* g2d, int64_t g2d_zero, cudaStream_t s, const FusedLoss* fl = nullptr);
cudaError_t launch_project_bwd(const gs_gaussians& g, const Views& views, const RenderConsts& rc,
                               const float* g2d, float lambda_iso, const gs_grads& grads, float* iso_loss,
                               cudaStream_t s, const float* xi = nullptr);
cudaError_t noalloc_loss_scratch(float** out);
// zero na, nb, nc floats at a, b, c (null or 0: skipped) with one kernel launch
cudaError_t launch_zero(float* a, int64_t na, float* b, int64_t nb, float* c, int64_t nc, cudaStream_t s);
cudaError_t launch_extract_patches(const float* color, const float* depth, const gs_camera& cam,
                                   const int32_t* uv, int64_t n, uint16_t* X, int* status, cudaStream_t s);
cudaError_t launch_insert(const float* color, const float* depth, const gs_camera& cam, const int32_t* uv,
                          int64_t n, float stride, const float* Y, const gs_map_slots& dst, int64_t offset,
                          int sh_degree, int* status, cudaStream_t s);
cudaError_t launch_loop_closure(const gs_map_slots& map, const int32_t* anchor, const float* before,
                                const float* after, const float* ds, int K, int* status, cudaStream_t s);
size_t ba_workspace(int K, int E, int P, int n);
cudaError_t launch_ba_step(const gs_ba_problem& pr, float lambda, float eps, float* cost, void* ws, cudaStream_t s);
cudaError_t launch_mlp_pack(const gs_mlp_params& p, const gs_mlp_packed& q, cudaStream_t s);
cudaError_t launch_mlp_fwd(const gs_mlp_packed& w, const uint16_t* X, int64_t n, float* Y, uint16_t* Z1,
                           uint16_t* Z2, const float* T, float* dY, float* loss, float loss_scale, int* status,
                           cudaStream_t s);
cudaError_t launch_mlp_bwd(const gs_mlp_packed& w, const uint16_t* X, const uint16_t* Z1, const uint16_t* Z2,
                           const float* dY, int64_t n, const gs_mlp_grads& g, int* status, cudaStream_t s);
uint32_t set_mlp_wait_polls(uint32_t polls);    // returns the previous limit
cudaError_t launch_adam(const gs_adam_group* groups, int n_groups, float b1, float b2, float eps,
                        int32_t* d_step, cudaStream_t s);

// ---------------------------------------------------------------- device side

#ifdef __CUDACC__
// log2(e): the splat weight is evaluated as exp2(power * log2 e).
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// first statement of every kernel launched by launch_pdl
__device__ __forceinline__ void pdl_enter() {
    pdl_wait();
    pdl_trigger();
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The splat's shared-memory form: conic pre-scaled so that the exponent comes
// out in log2 units, p2 = log2(e) * power.  Forward and backward both call
// splat_power2 / splat_alpha with identical operands, and every rounding step
// is an explicit intrinsic, so the two passes take identical decisions.
struct SplatGeom {
    float mx, my;       // projected mean
    float qa, qb, qc;   // -0.5 log2e A, -log2e B, -0.5 log2e C
    float o;            // opacity
};

__device__ __forceinline__ void scale_conic(float A, float B, float C, float* qa, float* qb, float* qc) {
    *qa = __fmul_rn(-0.5f * kLog2e, A);
    *qb = __fmul_rn(-kLog2e, B);
    *qc = __fmul_rn(-0.5f * kLog2e, C);
}

// p2 = qa dx^2 + qb dx dy + qc dy^2 with dx = px - mx, dy = py - my.
__device__ __forceinline__ float splat_power2(float qa, float qb, float qc, float dx, float dy) {
    float u = __fmaf_rn(qb, dy, __fmul_rn(qa, dx));   // qa dx + qb dy
    float w = __fmul_rn(qc, dy);                      // qc dy
    return __fmaf_rn(dx, u, __fmul_rn(w, dy));        // dx (qa dx + qb dy) + qc dy^2
}

__device__ __forceinline__ float splat_weight(float p2) { return ex2_approx(p2); }

// View of global tile g (tile bases ascend with the view index).
__device__ __forceinline__ int view_of_tile(const Views& views, int g) {
    int v = 0;
    for (int k = 1; k < views.n; k++)
        if (g >= views.v[k].tile_base) v = k;
    return v;
}

// Warp-level culling.  A splat is dropped from a warp's batch only if its
// weight o exp(power) stays below alpha_min (with a 1 % margin for rounding) at
// every pixel sample of the warp's 8 x 4 block, so dropping it changes no
// pixel.  The maximum of the concave power over the block's sample rectangle
// [x0, x1] x [y0, y1] lies at the mean if the mean is inside, else on an edge,
// where it is the clamped optimum of a 1-D quadratic; p2 is power * log2(e).
__device__ __forceinline__ float edge_max_p2(float qa, float qb, float qc, float fixed_d, float lo, float hi,
                                             bool fixed_is_x) {
    // fixed_is_x: dx = fixed_d, maximise over dy in [lo, hi]; else dy fixed, dx free
    const float qf = fixed_is_x ? qa : qc, qv = fixed_is_x ? qc : qa;
    float t = qv < 0.f ? -qb * fixed_d / (2.f * qv) : lo;   // stationary point of qv t^2 + qb f t
    t = fminf(fmaxf(t, lo), hi);
    return qf * fixed_d * fixed_d + qb * fixed_d * t + qv * t * t;
}

__device__ __forceinline__ bool splat_reaches_block(const float2 m, const float4 q, float x0, float x1, float y0,
                                                    float y1, float amin) {
    if (m.x >= x0 && m.x <= x1 && m.y >= y0 && m.y <= y1) return true;
    const float dx0 = x0 - m.x, dx1 = x1 - m.x, dy0 = y0 - m.y, dy1 = y1 - m.y;
    float p = edge_max_p2(q.x, q.y, q.z, dx0, dy0, dy1, true);
    p = fmaxf(p, edge_max_p2(q.x, q.y, q.z, dx1, dy0, dy1, true));
    p = fmaxf(p, edge_max_p2(q.x, q.y, q.z, dy0, dx0, dx1, false));
    p = fmaxf(p, edge_max_p2(q.x, q.y, q.z, dy1, dx0, dx1, false));
    return q.w * splat_weight(p) >= 0.99f * amin;
}

// Bit b is set when the splat (projected mean m, scaled conic and opacity q)
// can reach pixel block b of the T x T tile (tx, ty) of its view: the blocks are
// 8 x 4 pixels, row-major within the tile, as the rasterisers walk them.  Written
// once per key by the binning, read by both rasterisers instead of testing.
//
// For a negative-definite power p2 (every conic the projection writes) p2 is
// concave with its maximum 0 at the mean, so over a block's box of pixel centres
// its maximum lies on the box edges that face the mean (or is 0 when the mean is
// inside): the vertical edge at dx = clamp(0, dx0, dx1) and the horizontal edge at
// dy = clamp(0, dy0, dy1), each maximised at its clamped stationary point (where
// the mean is level with the box, the "edge" is a line through the box, a lower
// bound that the other edge dominates).  The bit is set when that maximum reaches
// log2(0.99 alpha_min / o), lowered by 0.004 against rounding, so the mask is a
// superset of the blocks where any pixel's weight reaches 0.99 alpha_min and
// drops nothing that blends.  Any other conic takes the rasterisers' own test.
template <int T>
__device__ __forceinline__ uint32_t splat_block_mask(const float2 m, const float4 q, int tx, int ty, float amin) {
    constexpr int bw = T / 8, nb = (T / 8) * (T / 4);
    const float thr = 0.99f * amin;
    if (q.w < thr) return 0u;                           // o 2^p2 <= o < 0.99 alpha_min everywhere
    const float qa = q.x, qb = q.y, qc = q.z;
    uint32_t mask = 0;
    if (!(qa < 0.f && qc < 0.f && 4.f * qa * qc - qb * qb > 0.f)) {
#pragma unroll
        for (int b = 0; b < nb; b++) {
            const float bx0 = (float)(tx * T + (b % bw) * 8) + 0.5f;
            const float by0 = (float)(ty * T + (b / bw) * 4) + 0.5f;
            if (splat_reaches_block(m, q, bx0, bx0 + 7.f, by0, by0 + 3.f, amin)) mask |= 1u << b;
        }
        return mask;
    }
    const float L = __log2f(__fdividef(thr, q.w)) - 0.004f;
    const float rx = __fdividef(-qb, 2.f * qc);         // stationary dy / dx on a vertical line
    const float ry = __fdividef(-qb, 2.f * qa);         // stationary dx / dy on a horizontal line
    const float ox = (float)(tx * T) + 0.5f - m.x, oy = (float)(ty * T) + 0.5f - m.y;
#pragma unroll
    for (int b = 0; b < nb; b++) {
        const float dx0 = ox + (float)((b % bw) * 8), dx1 = dx0 + 7.f;
        const float dy0 = oy + (float)((b / bw) * 4), dy1 = dy0 + 3.f;
        const float vx = fminf(fmaxf(0.f, dx0), dx1), vy = fminf(fmaxf(0.f, dy0), dy1);
        const float ty_ = fminf(fmaxf(rx * vx, dy0), dy1), tx_ = fminf(fmaxf(ry * vy, dx0), dx1);
        const float pv = vx * fmaf(qa, vx, qb * ty_) + qc * ty_ * ty_;
        const float ph = vy * fmaf(qc, vy, qb * tx_) + qa * tx_ * tx_;
        if (fmaxf(pv, ph) >= L) mask |= 1u << b;
    }
    return mask;
}
#endif

// Quaternion (w, x, y, z) of a rotation matrix (row-major), by the larger-of-
// four-candidates method (Shepperd, 1978).
__device__ __forceinline__ void rot_to_quat(const float* R, float* q) {
    const float tr = R[0] + R[4] + R[8];
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
        const float s = sqrtf(fmaxf(1.f + tr, 0.f)) * 2.f;
        q[0] = 0.25f * s;
        q[1] = (R[7] - R[5]) / s; q[2] = (R[2] - R[6]) / s; q[3] = (R[3] - R[1]) / s;
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
        const float s = sqrtf(fmaxf(1.f + R[0] - R[4] - R[8], 0.f)) * 2.f;
        q[0] = (R[7] - R[5]) / s; q[1] = 0.25f * s;
        q[2] = (R[1] + R[3]) / s; q[3] = (R[2] + R[6]) / s;
    } else if (R[4] >= R[8]) {
        const float s = sqrtf(fmaxf(1.f + R[4] - R[0] - R[8], 0.f)) * 2.f;
        q[0] = (R[2] - R[6]) / s; q[1] = (R[1] + R[3]) / s;
        q[2] = 0.25f * s; q[3] = (R[5] + R[7]) / s;
    } else {
        const float s = sqrtf(fmaxf(1.f + R[8] - R[0] - R[4], 0.f)) * 2.f;
        q[0] = (R[3] - R[1]) / s; q[1] = (R[2] + R[6]) / s;
        q[2] = (R[5] + R[7]) / s; q[3] = 0.25f * s;
    }
}

// Hamilton product a * b
__device__ __forceinline__ void quat_mul(const float* a, const float* b, float* c) {
    c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

}  // namespace gs
