// api.cu -- the extern "C" entry points of libgs (declared in include/gs.h):
// host-side argument checks, per-view constants, workspace carving, launches.
#include <math.h>
#include <string.h>

#include "gs_internal.cuh"

namespace gs {

size_t loss_workspace(int32_t n_views);

bool make_views(const gs_camera* cams, int32_t n_views, int32_t tile, Views* out) {
    memset(out, 0, sizeof(*out));
    if (cams == nullptr || n_views < 1 || n_views > GS_MAX_VIEWS) return false;
    if (tile != 8 && tile != 16 && tile != 32) return false;
    int64_t tiles = 0, pixels = 0;
    out->n = n_views;
    for (int v = 0; v < n_views; v++) {
        const gs_camera& c = cams[v];
        if (c.width < 1 || c.height < 1 || c.width > (1 << 16) || c.height > (1 << 16)) return false;
        if (!(isfinite(c.fx) && isfinite(c.fy) && isfinite(c.cx) && isfinite(c.cy)) || c.fx == 0.f || c.fy == 0.f)
            return false;
        ViewParams& p = out->v[v];
        for (int k = 0; k < 9; k++)
            if (!isfinite(c.R_wc[k])) return false;
        for (int k = 0; k < 3; k++)
            if (!isfinite(c.t_wc[k])) return false;
        // R_cw = R_wc^T, t_cw = -R_wc^T t_wc (accumulated in double, rounded once)
        for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++) p.Rcw[3 * r + q] = c.R_wc[3 * q + r];
        for (int r = 0; r < 3; r++) {
            double s = 0.0;
            for (int q = 0; q < 3; q++) s -= (double)c.R_wc[3 * q + r] * (double)c.t_wc[q];
            p.tcw[r] = (float)s;
            p.centre[r] = c.t_wc[r];
        }
        p.fx = c.fx; p.fy = c.fy; p.cx = c.cx; p.cy = c.cy;
        p.W = c.width; p.H = c.height;
        p.tiles_x = (c.width + tile - 1) / tile;
        p.tiles_y = (c.height + tile - 1) / tile;
        p.tile_base = (int32_t)tiles;
        p.pix_base = (int32_t)pixels;
        tiles += (int64_t)p.tiles_x * p.tiles_y;
        pixels += (int64_t)c.width * c.height;
        if (tiles >= (1ll << 31) || pixels >= (1ll << 31)) return false;
    }
    out->total_tiles = (int32_t)tiles;
    out->total_pixels = (int32_t)pixels;
    return true;
}

RenderConsts make_consts(const gs_render_params* p) {
    RenderConsts c;
    c.tile = p->tile;
    c.near_plane = p->near_plane;
    c.alpha_min = p->alpha_min;
    c.alpha_max = p->alpha_max;
    c.T_cut = p->T_cut;
    c.dilation = p->dilation;
    c.radius_sigma = p->radius_sigma;
    c.bg[0] = p->bg[0]; c.bg[1] = p->bg[1]; c.bg[2] = p->bg[2];
    c.sh_degree = p->sh_degree;
    c.splat_stages = p->splat_stages;
    c.block_masks = p->block_masks;
    return c;
}

static bool params_ok(const gs_render_params* p) {
    if (p == nullptr) return false;
    if (p->tile != 8 && p->tile != 16 && p->tile != 32) return false;
    if (p->sh_degree != 0 && p->sh_degree != 3) return false;
    if (p->splat_stages != 0 && p->splat_stages != 2 && p->splat_stages != 3) return false;
    if (p->block_masks != 0 && p->block_masks != 1) return false;
    if (p->cull_tiles != 0 && p->cull_tiles != 1) return false;
    if (!(p->near_plane > 0.f) || !isfinite(p->near_plane)) return false;
    if (!(p->alpha_min >= 0.f) || !(p->alpha_max <= 1.f) || !(p->alpha_min <= p->alpha_max)) return false;
    if (!(p->T_cut >= 0.f) || !(p->T_cut < 1.f)) return false;
    if (!(p->dilation >= 0.f) || !isfinite(p->dilation)) return false;
    if (!(p->radius_sigma > 0.f) || !isfinite(p->radius_sigma)) return false;
    for (int k = 0; k < 3; k++)
        if (!isfinite(p->bg[k])) return false;
    return true;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

static bool gaussians_ok(const gs_gaussians* g, int32_t n_views) {
    if (g == nullptr || g->n < 0) return false;
    if (g->n * (int64_t)n_views >= (1ll << 31)) return false;
    if (g->n == 0) return true;
    if (!g->mean || !g->quat || !g->log_scale || !g->opacity_logit || !g->color) return false;
    return aligned(g->quat, 16);
}

// An empty map may pass all-NULL projected arrays.
static bool projected_ok(const gs_projected* p) {
    if (p == nullptr) return false;
    if (!p->xy && !p->conic_o && !p->rgbd && !p->rect && !p->radius && !p->tiles_touched) return true;
    if (!p->xy || !p->conic_o || !p->rgbd || !p->rect || !p->radius || !p->tiles_touched) return false;
    return aligned(p->xy, 8) && aligned(p->conic_o, 16) && aligned(p->rgbd, 16) && aligned(p->rect, 16);
}

static bool image_ok(const gs_image* im) {
    return im != nullptr && im->color && im->depth && im->T_final && im->n_contrib;
}

static bool bins_ok(const gs_bins* b) {
    return b != nullptr && b->keys && b->vals && b->masks && b->ranges && b->num_keys && b->status &&
           b->key_capacity >= 0 &&
           b->key_capacity < (1ll << 32) && aligned(b->ranges, 8);
}

static size_t render_bwd_workspace(int64_t n_entries) {
    return align_up(sizeof(float) * kGradStride * (size_t)n_entries, 256);
}

static int32_t cuda_status(cudaError_t e) { return e == cudaSuccess ? GS_OK : GS_ERR_CUDA; }

}  // namespace gs

using namespace gs;

extern "C" {

int32_t gs_abi_version(void) { return GS_ABI_VERSION; }

const char* gs_status_string(int32_t s) {
    switch (s) {
        case GS_OK: return "GS_OK";
        case GS_ERR_INVALID_ARG: return "GS_ERR_INVALID_ARG";
        case GS_ERR_CAPACITY: return "GS_ERR_CAPACITY";
        case GS_ERR_CUDA: return "GS_ERR_CUDA";
        case GS_ERR_TIMEOUT: return "GS_ERR_TIMEOUT";
        case GS_ERR_NUMERIC: return "GS_ERR_NUMERIC";
        case GS_ERR_UNSUPPORTED: return "GS_ERR_UNSUPPORTED";
        default: return "GS_ERR_UNKNOWN";
    }
}

int64_t gs_total_tiles(const gs_camera* cams, int32_t n_views, int32_t tile) {
    Views v;
    if (!make_views(cams, n_views, tile, &v)) return -1;
    return v.total_tiles;
}

int64_t gs_total_pixels(const gs_camera* cams, int32_t n_views) {
    Views v;
    if (!make_views(cams, n_views, 16, &v)) return -1;
    return v.total_pixels;
}

size_t gs_workspace_size(int64_t n, int32_t n_views, const gs_camera* cams, const gs_render_params* params,
                         int64_t key_capacity) {
    Views v;
    if (n < 0 || key_capacity < 0 || !params_ok(params) || !make_views(cams, n_views, params->tile, &v)) return 0;
    const int64_t E = n * n_views;
    size_t a = bin_sort_workspace(E, key_capacity, v.total_tiles);
    size_t b = loss_workspace(n_views);
    size_t c = render_bwd_workspace(E);
    size_t m = a > b ? a : b;
    return m > c ? m : c;
}

int32_t gs_project(const gs_gaussians* g, const gs_camera* cams, int32_t n_views, const gs_render_params* params,
                   gs_projected* out, void* stream) {
    return gs_project_perturbed(g, cams, n_views, params, nullptr, out, stream);
}

int32_t gs_project_perturbed(const gs_gaussians* g, const gs_camera* cams, int32_t n_views,
                             const gs_render_params* params, const float* xi, gs_projected* out, void* stream) {
    if (!params_ok(params) || !gaussians_ok(g, n_views)) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    if (g->n > 0 && !projected_ok(out)) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_project(*g, views, make_consts(params), *out, static_cast<cudaStream_t>(stream), xi));
}

int32_t gs_bin_sort(const gs_projected* proj, int64_t n, const gs_camera* cams, int32_t n_views,
                    const gs_render_params* params, gs_bins* bins, void* ws, size_t ws_bytes, void* stream) {
    if (!params_ok(params) || n < 0 || !bins_ok(bins)) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    if (n * (int64_t)n_views >= (1ll << 31)) return GS_ERR_INVALID_ARG;
    if (n > 0 && !projected_ok(proj)) return GS_ERR_INVALID_ARG;
    const size_t need = bin_sort_workspace(n * n_views, bins->key_capacity, views.total_tiles);
    if (ws == nullptr || ws_bytes < need || !aligned(ws, 256)) return GS_ERR_INVALID_ARG;
    SortPlan plan =
        make_sort_plan(bins->key_capacity, views.total_tiles, params->tile, params->alpha_min, params->block_masks,
                       params->cull_tiles);
    return cuda_status(launch_bin_sort(*proj, n, views, plan, *bins, ws, static_cast<cudaStream_t>(stream)));
}

int32_t gs_render_fwd(const gs_projected* proj, const gs_bins* bins, const gs_camera* cams, int32_t n_views,
                      const gs_render_params* params, gs_image* img, void* stream) {
    if (!params_ok(params) || !bins_ok(bins) || !projected_ok(proj) || !image_ok(img)) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_render_fwd(*proj, *bins, views, make_consts(params), *img,
                                         static_cast<cudaStream_t>(stream)));
}

size_t gs_fused_loss_workspace_size(int32_t n_views) {
    if (n_views < 1 || n_views > GS_MAX_VIEWS) return 0;
    return fused_loss_workspace(n_views);
}

int32_t gs_render_fwd_loss(const gs_projected* proj, const gs_bins* bins, const gs_camera* cams, int32_t n_views,
                           const gs_render_params* params, gs_image* img, const float* target_color,
                           const float* target_depth, float* loss_terms, void* loss_ws, size_t loss_ws_bytes,
                           void* stream) {
    if (!params_ok(params) || !bins_ok(bins) || !projected_ok(proj) || !image_ok(img)) return GS_ERR_INVALID_ARG;
    if (!target_color || !target_depth || !loss_terms) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    if (loss_ws == nullptr || !aligned(loss_ws, 256) || loss_ws_bytes < fused_loss_workspace(n_views))
        return GS_ERR_INVALID_ARG;
    FusedLoss fl = {};
    fl.tc = target_color; fl.td = target_depth;
    fl.terms = loss_terms;
    fl.ticket = bins->status + 3;
    fused_loss_layout(loss_ws, n_views, &fl);
    return cuda_status(launch_render_fwd(*proj, *bins, views, make_consts(params), *img,
                                         static_cast<cudaStream_t>(stream), &fl));
}

int32_t gs_render_bwd_raster_loss(const gs_projected* proj, const gs_bins* bins, const gs_image* img,
                                  const float* target_color, const float* target_depth, float lambda_c,
                                  float lambda_d, const void* loss_ws, size_t loss_ws_bytes, const gs_camera* cams,
                                  int32_t n_views, const gs_render_params* params, int64_t n, float* grad2d,
                                  void* stream) {
    if (!params_ok(params) || !bins_ok(bins) || !projected_ok(proj) || !image_ok(img)) return GS_ERR_INVALID_ARG;
    if (!target_color || !target_depth || !grad2d || !aligned(grad2d, 16) || n < 0) return GS_ERR_INVALID_ARG;
    if (!isfinite(lambda_c) || !isfinite(lambda_d)) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    if (loss_ws == nullptr || !aligned(loss_ws, 256) || loss_ws_bytes < fused_loss_workspace(n_views))
        return GS_ERR_INVALID_ARG;
    const int64_t E = n * n_views;
    if (E >= (1ll << 31)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (E == 0) return GS_OK;
    FusedLoss fl = {};
    fl.tc = target_color; fl.td = target_depth;
    fl.color = img->color; fl.depth = img->depth;
    fl.lc = lambda_c; fl.ld = lambda_d;
    fused_loss_layout(const_cast<void*>(loss_ws), n_views, &fl);
    return cuda_status(launch_render_bwd(*proj, *bins, *img, nullptr, nullptr, views, make_consts(params), grad2d,
                                         kGradStride * E, s, &fl));
}

int32_t gs_loss(const gs_image* img, const float* target_color, const float* target_depth, const gs_camera* cams,
                int32_t n_views, float lambda_c, float lambda_d, float* dL_dcolor, float* dL_ddepth, float* loss_terms,
                void* ws, size_t ws_bytes, void* stream) {
    if (!image_ok(img) || !target_color || !target_depth || !dL_dcolor || !dL_ddepth || !loss_terms)
        return GS_ERR_INVALID_ARG;
    if (!isfinite(lambda_c) || !isfinite(lambda_d)) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, 16, &views)) return GS_ERR_INVALID_ARG;
    if (ws == nullptr || ws_bytes < loss_workspace(n_views) || !aligned(ws, 256)) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_loss(*img, target_color, target_depth, views, lambda_c, lambda_d, dL_dcolor, dL_ddepth,
                                   loss_terms, ws, static_cast<cudaStream_t>(stream)));
}

// the static scratch array of gs_loss_noalloc must cover every view count the
// view checks (make_views) accept below its own limit
static_assert(GS_NOALLOC_LOSS_MAX_VIEWS <= GS_MAX_VIEWS, "no-alloc loss limit above the view limit");

int32_t gs_loss_noalloc(const gs_image* img, const float* target_color, const float* target_depth,
                        const gs_camera* cams, int32_t n_views, float lambda_c, float lambda_d, float* dL_dcolor,
                        float* dL_ddepth, float* loss_terms, void* stream) {
    if (!image_ok(img) || !target_color || !target_depth || !dL_dcolor || !dL_ddepth || !loss_terms)
        return GS_ERR_INVALID_ARG;
    if (!isfinite(lambda_c) || !isfinite(lambda_d)) return GS_ERR_INVALID_ARG;
    if (n_views < 1 || n_views > GS_NOALLOC_LOSS_MAX_VIEWS) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, 16, &views)) return GS_ERR_INVALID_ARG;
    float* scratch = nullptr;
    if (noalloc_loss_scratch(&scratch) != cudaSuccess) return GS_ERR_CUDA;
    // launch_loss zeroes the accumulators it uses before accumulating
    return cuda_status(launch_loss(*img, target_color, target_depth, views, lambda_c, lambda_d, dL_dcolor, dL_ddepth,
                                   loss_terms, scratch, static_cast<cudaStream_t>(stream)));
}

int32_t gs_render_bwd_raster(const gs_projected* proj, const gs_bins* bins, const gs_image* img,
                             const float* dL_dcolor, const float* dL_ddepth, const gs_camera* cams, int32_t n_views,
                             const gs_render_params* params, int64_t n, float* grad2d, void* stream) {
    if (!params_ok(params) || !bins_ok(bins) || !projected_ok(proj) || !image_ok(img)) return GS_ERR_INVALID_ARG;
    if (!dL_dcolor || !dL_ddepth || !grad2d || !aligned(grad2d, 16) || n < 0) return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    const int64_t E = n * n_views;
    if (E >= (1ll << 31)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (E == 0) return GS_OK;
    return cuda_status(launch_render_bwd(*proj, *bins, *img, dL_dcolor, dL_ddepth, views, make_consts(params),
                                         grad2d, kGradStride * E, s));
}

int32_t gs_project_bwd(const gs_gaussians* g, const gs_camera* cams, int32_t n_views, const gs_render_params* params,
                       const float* grad2d, float lambda_iso, gs_grads* grads, float* iso_loss, void* stream) {
    return gs_project_bwd_perturbed(g, cams, n_views, params, nullptr, grad2d, lambda_iso, grads, iso_loss, stream);
}

int32_t gs_project_bwd_perturbed(const gs_gaussians* g, const gs_camera* cams, int32_t n_views,
                                 const gs_render_params* params, const float* xi, const float* grad2d,
                                 float lambda_iso, gs_grads* grads, float* iso_loss, void* stream) {
    if (!params_ok(params) || !gaussians_ok(g, n_views) || grads == nullptr || !isfinite(lambda_iso))
        return GS_ERR_INVALID_ARG;
    if (g->n > 0 && (!grad2d || !aligned(grad2d, 16) || !grads->mean || !grads->quat || !grads->log_scale ||
                     !grads->opacity_logit || !grads->color || !aligned(grads->quat, 16)))
        return GS_ERR_INVALID_ARG;
    Views views;
    if (!make_views(cams, n_views, params->tile, &views)) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    e = launch_zero(grads->pose, 6 * (int64_t)n_views, iso_loss, 1, nullptr, 0, s);
    if (e == cudaSuccess && g->n > 0)
        e = launch_project_bwd(*g, views, make_consts(params), grad2d, lambda_iso, *grads, iso_loss, s, xi);
    return cuda_status(e);
}

int32_t gs_render_bwd(const gs_gaussians* g, const gs_projected* proj, const gs_bins* bins, const gs_image* img,
                      const float* dL_dcolor, const float* dL_ddepth, const gs_camera* cams, int32_t n_views,
                      const gs_render_params* params, float lambda_iso, gs_grads* grads, float* iso_loss, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!gaussians_ok(g, n_views)) return GS_ERR_INVALID_ARG;
    const int64_t E = g->n * n_views;
    if (ws == nullptr || ws_bytes < render_bwd_workspace(E) || !aligned(ws, 256)) return GS_ERR_INVALID_ARG;
    float* g2d = static_cast<float*>(ws);
    int32_t st = gs_render_bwd_raster(proj, bins, img, dL_dcolor, dL_ddepth, cams, n_views, params, g->n, g2d, stream);
    if (st != GS_OK) return st;
    return gs_project_bwd(g, cams, n_views, params, g2d, lambda_iso, grads, iso_loss, stream);
}

int32_t gs_adam_step(const gs_adam_group* groups, int32_t n_groups, float beta1, float beta2, float eps,
                     int32_t* d_step, void* stream) {
    if (groups == nullptr || n_groups < 1 || n_groups > 8 || d_step == nullptr) return GS_ERR_INVALID_ARG;
    if (!(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f)) return GS_ERR_INVALID_ARG;
    for (int k = 0; k < n_groups; k++) {
        const gs_adam_group& G = groups[k];
        if (G.n < 0 || G.reserved != 0 || !isfinite(G.lr)) return GS_ERR_INVALID_ARG;
        if (G.n > 0 && (!G.param || !G.grad || !G.m || !G.v)) return GS_ERR_INVALID_ARG;
    }
    return cuda_status(launch_adam(groups, n_groups, beta1, beta2, eps, d_step, static_cast<cudaStream_t>(stream)));
}

int32_t gs_mapping_step(const gs_mapping_step_args* a, void* stream) {
    if (a == nullptr || a->gaussians == nullptr || a->bins == nullptr || a->ws == nullptr) return GS_ERR_INVALID_ARG;
    const int64_t n = a->gaussians->n;
    // ws serves the sort and then the 2D-gradient scratch of the backward pass,
    // so it must hold the larger of the two (gs_workspace_size), not just what
    // gs_bin_sort checks for
    const size_t need = gs_workspace_size(n, a->n_views, a->cams, a->params, a->bins->key_capacity);
    if (need == 0 || a->ws_bytes < need || !aligned(a->ws, 256)) return GS_ERR_INVALID_ARG;
    float* grad2d = static_cast<float*>(a->ws);
    int32_t st = gs_project(a->gaussians, a->cams, a->n_views, a->params, a->proj, stream);
    if (st == GS_OK)
        st = gs_bin_sort(a->proj, n, a->cams, a->n_views, a->params, a->bins, a->ws, a->ws_bytes, stream);
    if (st == GS_OK)
        st = gs_render_fwd_loss(a->proj, a->bins, a->cams, a->n_views, a->params, a->img, a->target_color,
                                a->target_depth, a->loss_terms, a->loss_ws, a->loss_ws_bytes, stream);
    if (st == GS_OK)
        st = gs_render_bwd_raster_loss(a->proj, a->bins, a->img, a->target_color, a->target_depth, a->lambda_c,
                                       a->lambda_d, a->loss_ws, a->loss_ws_bytes, a->cams, a->n_views, a->params, n,
                                       grad2d, stream);
    if (st == GS_OK)
        st = gs_project_bwd(a->gaussians, a->cams, a->n_views, a->params, grad2d, a->lambda_iso, a->grads,
                            a->iso_loss, stream);
    if (st == GS_OK)
        st = gs_adam_step(a->adam_groups, a->n_adam_groups, a->beta1, a->beta2, a->adam_eps, a->d_step, stream);
    return st;
}

int32_t gs_read_device_status(const int32_t* d_status, void* stream, int32_t* host_status) {
    if (d_status == nullptr || host_status == nullptr) return GS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(host_status, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GS_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? GS_OK : GS_ERR_CUDA;
}

int32_t gs_l2_read_probe(const float* buf, int64_t n, int32_t reps, float* out, void* stream) {
    if (buf == nullptr || out == nullptr || n <= 0 || n % 4 != 0 || reps < 1 || !aligned(buf, 16))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_l2_read(buf, n, reps, out, static_cast<cudaStream_t>(stream)));
}

int32_t gs_mlp_pack(const gs_mlp_params* p, const gs_mlp_packed* q, void* stream) {
    if (p == nullptr || q == nullptr) return GS_ERR_INVALID_ARG;
    if (!p->W1 || !p->b1 || !p->W2 || !p->b2 || !p->W3 || !p->b3) return GS_ERR_INVALID_ARG;
    if (!q->W1a || !q->W2a || !q->W3a || !q->W2t || !q->gelu_tab || !q->dgelu_tab) return GS_ERR_INVALID_ARG;
    if (!aligned(q->W1a, 16) || !aligned(q->W2a, 16) || !aligned(q->W3a, 16) || !aligned(q->W2t, 16))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_mlp_pack(*p, *q, static_cast<cudaStream_t>(stream)));
}

static bool mlp_packed_ok(const gs_mlp_packed* q) {
    return q != nullptr && q->W1a && q->W2a && q->W3a && q->W2t && q->gelu_tab && q->dgelu_tab &&
           aligned(q->W1a, 16) && aligned(q->W2a, 16) && aligned(q->W3a, 16) && aligned(q->W2t, 16);
}

int32_t gs_mlp_fwd(const gs_mlp_packed* q, const uint16_t* X, int64_t n, float* Y, uint16_t* Z1, uint16_t* Z2,
                   const float* T, float* dY, float* loss, float loss_scale, int32_t* d_status, void* stream) {
    if (!mlp_packed_ok(q) || n < 0 || (n > 0 && (!X || !aligned(X, 16)))) return GS_ERR_INVALID_ARG;
    if ((Y && !aligned(Y, 16)) || (Z1 && !aligned(Z1, 16)) || (Z2 && !aligned(Z2, 16))) return GS_ERR_INVALID_ARG;
    if ((Z1 == nullptr) != (Z2 == nullptr)) return GS_ERR_INVALID_ARG;
    if (T && (!aligned(T, 16) || !dY || !aligned(dY, 16) || !loss || !isfinite(loss_scale))) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_mlp_fwd(*q, X, n, Y, Z1, Z2, T, dY, loss, loss_scale, d_status,
                                      static_cast<cudaStream_t>(stream)));
}

int32_t gs_mlp_bwd(const gs_mlp_packed* q, const uint16_t* X, const uint16_t* Z1, const uint16_t* Z2,
                   const float* dY, int64_t n, const gs_mlp_grads* g, int32_t* d_status, void* stream) {
    if (!mlp_packed_ok(q) || n < 0 || g == nullptr) return GS_ERR_INVALID_ARG;
    if (!g->W1 || !g->b1 || !g->W2 || !g->b2 || !g->W3 || !g->b3) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!X || !Z1 || !Z2 || !dY || !aligned(X, 16) || !aligned(Z1, 16) || !aligned(Z2, 16) ||
                  !aligned(dY, 16)))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_mlp_bwd(*q, X, Z1, Z2, dY, n, *g, d_status, static_cast<cudaStream_t>(stream)));
}

int64_t gs_mlp_set_wait_polls(int64_t polls) {
    if (polls > (int64_t)UINT32_MAX) return -1;
    return (int64_t)set_mlp_wait_polls(polls < 0 ? GS_MLP_WAIT_POLLS_DEFAULT : (uint32_t)polls);
}

static bool keyframe_ok(const float* color, const float* depth, const gs_camera* cam, const int32_t* uv, int64_t n) {
    if (cam == nullptr || n < 0) return false;
    Views views;
    if (!make_views(cam, 1, 16, &views)) return false;
    return n == 0 || (color && depth && uv && aligned(uv, 8));
}

int32_t gs_extract_patches(const float* color, const float* depth, const gs_camera* cam, const int32_t* uv,
                           int64_t n, uint16_t* X, int32_t* d_status, void* stream) {
    if (!keyframe_ok(color, depth, cam, uv, n) || (n > 0 && (!X || !aligned(X, 16)))) return GS_ERR_INVALID_ARG;
    return cuda_status(launch_extract_patches(color, depth, *cam, uv, n, X, d_status,
                                              static_cast<cudaStream_t>(stream)));
}

int32_t gs_insert_gaussians(const float* color, const float* depth, const gs_camera* cam, const int32_t* uv,
                            int64_t n, float stride, const float* Y, const gs_map_slots* dst, int64_t offset,
                            int32_t sh_degree, int32_t* d_status, void* stream) {
    if (!keyframe_ok(color, depth, cam, uv, n) || dst == nullptr || !(stride > 0.f) || !isfinite(stride))
        return GS_ERR_INVALID_ARG;
    if (sh_degree != 0 && sh_degree != 3) return GS_ERR_INVALID_ARG;
    if (offset < 0 || offset + n > dst->capacity) return GS_ERR_INVALID_ARG;
    if (n > 0 && (!dst->mean || !dst->quat || !dst->log_scale || !dst->opacity_logit || !dst->color))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_insert(color, depth, *cam, uv, n, stride, Y, *dst, offset, sh_degree, d_status,
                                     static_cast<cudaStream_t>(stream)));
}

int32_t gs_loop_closure_update(const gs_map_slots* map, const int32_t* anchor, const float* pose_before,
                               const float* pose_after, const float* scale_change, int32_t n_keyframes,
                               int32_t* d_status, void* stream) {
    if (map == nullptr || map->capacity < 0 || n_keyframes < 1) return GS_ERR_INVALID_ARG;
    if (map->capacity > 0 && (!map->mean || !map->quat || !map->log_scale || !aligned(map->quat, 16) || !anchor ||
                              !pose_before || !pose_after || !scale_change))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_loop_closure(*map, anchor, pose_before, pose_after, scale_change, n_keyframes,
                                           d_status, static_cast<cudaStream_t>(stream)));
}

size_t gs_ba_workspace_size(int32_t K, int32_t E, int32_t h, int32_t w, int32_t n_fixed, int32_t inertial) {
    if (K < 1 || E < 0 || h < 1 || w < 1 || n_fixed < 0 || n_fixed > K) return 0;
    return ba_workspace(K, E, h * w, (inertial ? 15 : 6) * (K - n_fixed));
}

int32_t gs_ba_step(const gs_ba_problem* pr, float lambda, float eps, float* cost, void* ws, size_t ws_bytes,
                   void* stream) {
    if (pr == nullptr || cost == nullptr) return GS_ERR_INVALID_ARG;
    const int K = pr->n_keyframes, E = pr->n_edges, h = pr->height, w = pr->width;
    if (K < 1 || E < 0 || h < 1 || w < 1 || pr->n_fixed < 0 || pr->n_fixed > K) return GS_ERR_INVALID_ARG;
    if ((int64_t)h * w >= (1 << 26) || (int64_t)E * h * w * 12 >= (1ll << 40)) return GS_ERR_INVALID_ARG;
    if (!(lambda >= 0.f) || !(eps >= 0.f) || !isfinite(lambda) || !isfinite(eps)) return GS_ERR_INVALID_ARG;
    if (!isfinite(pr->fx) || !isfinite(pr->fy) || !isfinite(pr->cx) || !isfinite(pr->cy) || pr->fx == 0.f ||
        pr->fy == 0.f)
        return GS_ERR_INVALID_ARG;
    if (!pr->poses || !pr->disp || !pr->status || (E > 0 && (!pr->targets || !pr->weights || !pr->ii || !pr->jj)))
        return GS_ERR_INVALID_ARG;
    const bool inertial = pr->imu != nullptr;
    if (inertial && (!pr->vel || !pr->bias || !pr->bias_hat)) return GS_ERR_INVALID_ARG;
    if (inertial && (!isfinite(pr->gravity[0]) || !isfinite(pr->gravity[1]) || !isfinite(pr->gravity[2])))
        return GS_ERR_INVALID_ARG;
    if (K - pr->n_fixed > (inertial ? 15 : 31)) return GS_ERR_UNSUPPORTED;
    const int bs = inertial ? 15 : 6;
    if (ws == nullptr || !aligned(ws, 256) || ws_bytes < ba_workspace(K, E, h * w, bs * (K - pr->n_fixed)))
        return GS_ERR_INVALID_ARG;
    return cuda_status(launch_ba_step(*pr, lambda, eps, cost, ws, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
