/*
 * gs_oracle.c -- plain, slow FP64 CPU oracle of the Gaussian-splatting mapping
 * step of VIGS-SLAM (Sec. 3.3, "Gaussian Splatting Mapping", Eq. 6).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  It shares no code, header,
 * table or constant with the CUDA library and includes nothing from it.
 *
 * What it follows:
 *  - Sec. 3.3 "Preliminary": each Gaussian has a colour c in R^3 (direct RGB
 *    instead of spherical harmonics), an opacity o in [0,1], a mean mu and a
 *    covariance Sigma; a pixel's colour is the alpha blend of the visible
 *    Gaussians.  Sigma = R(q) diag(s)^2 R(q)^T with s = exp(log_scale) and
 *    o = sigmoid(logit) (the parameterisation of the 3D Gaussian splatting
 *    work that Sec. 3.3 builds on).
 *  - Sec. 3.3 "Map Management": colour and depth are rendered from a keyframe
 *    pose; L = lambda_d L_d + lambda_c L_c + lambda_iso L_iso (Eq. 6) with
 *    L_c = |I_hat - I|_1 and L_d = |D_hat - D|_1.
 *  - Sec. 3.3 "Loop Closure Gaussian Update": keyframe poses (R_k, t_k) map
 *    camera coordinates to the world, x_world = R_k x_loc + t_k; the renderer
 *    therefore uses R_cw = R_k^T, t_cw = -R_k^T t_k.
 *
 * Readings where the paper is silent (they are the same parameters the CUDA
 * library takes, not shared code): pixel (u,v) sampled at (u+0.5, v+0.5);
 * near-plane cull z <= near; low-pass dilation of the 2D covariance; splat
 * radius ceil(k_sigma sqrt(lambda_max)); alpha = min(alpha_max, o exp(power)),
 * splats with alpha < alpha_min skipped; a pixel stops before blending a splat
 * that would take its transmittance below T_cut, and n_contrib counts the
 * splats visited up to and including the last one blended; rendered depth is
 * the alpha-blended camera z of the means; background colour bg; pose
 * gradient w.r.t. a left perturbation T_cw <- Exp(xi) T_cw, xi = (rho, phi);
 * quaternions (w, x, y, z), normalised inside the projection.
 *
 * "smooth mode" (prm[10] != 0) sets alpha_min = 0, alpha_max = 1, T_cut = 0
 * and makes every Gaussian cover the whole tile grid, so the rendered image is
 * a differentiable function of every parameter (used for finite differences).
 *
 * Array conventions: all per-Gaussian arrays are row-major [n][k] doubles.
 * cam[18] = {fx, fy, cx, cy, width, height, R_wc (9, row-major), t_wc (3)}.
 * prm[12] = {tile, near, alpha_min, alpha_max, T_cut, dilation, k_sigma,
 *            bg_r, bg_g, bg_b, smooth, sh_degree}.
 * Images are planar: colour [3][H][W], depth / T_final / n_contrib [H][W].
 *
 * Threads (or_set_threads): the loops over Gaussians and tiles may run on
 * several host threads (OpenMP).  Each such loop either writes outputs that no
 * other iteration touches, or records its contributions to shared sums and
 * adds them up afterwards in the serial loop's order, so every result is
 * bit-identical to the one-thread run.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1;

/* Host threads of the parallel loops (>= 1); returns the previous count. */
int or_set_threads(int n) {
    int prev = g_threads;
    g_threads = n < 1 ? 1 : n;
    return prev;
}

/* Processors available to the parallel loops (1 without OpenMP). */
int or_num_procs(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

typedef struct {
    double fx, fy, cx, cy;
    int W, H;
    double Rwc[9], twc[3];
    double Rcw[9], tcw[3];
} Cam;

typedef struct {
    int tile;
    double near_plane, a_min, a_max, T_cut, dil, k_sigma, bg[3];
    int smooth, sh_degree;
} Prm;

static Cam cam_from(const double* c) {
    Cam k;
    k.fx = c[0]; k.fy = c[1]; k.cx = c[2]; k.cy = c[3];
    k.W = (int)c[4]; k.H = (int)c[5];
    for (int i = 0; i < 9; i++) k.Rwc[i] = c[6 + i];
    for (int i = 0; i < 3; i++) k.twc[i] = c[15 + i];
    /* R_cw = R_wc^T ; t_cw = -R_wc^T t_wc */
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) k.Rcw[r * 3 + q] = k.Rwc[q * 3 + r];
    for (int r = 0; r < 3; r++) {
        k.tcw[r] = 0.0;
        for (int q = 0; q < 3; q++) k.tcw[r] -= k.Rcw[r * 3 + q] * k.twc[q];
    }
    return k;
}

static Prm prm_from(const double* p) {
    Prm m;
    m.tile = (int)p[0];
    m.near_plane = p[1];
    m.a_min = p[2]; m.a_max = p[3]; m.T_cut = p[4];
    m.dil = p[5]; m.k_sigma = p[6];
    m.bg[0] = p[7]; m.bg[1] = p[8]; m.bg[2] = p[9];
    m.smooth = p[10] != 0.0;
    m.sh_degree = (int)p[11];
    if (m.smooth) { m.a_min = 0.0; m.a_max = 1.0; m.T_cut = 0.0; }
    return m;
}

static int tiles_x_of(const Cam* c, const Prm* p) { return (c->W + p->tile - 1) / p->tile; }
static int tiles_y_of(const Cam* c, const Prm* p) { return (c->H + p->tile - 1) / p->tile; }

/* 3x3 helpers, row-major */
static void matmul3(const double* A, const double* B, double* C) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += A[i * 3 + k] * B[k * 3 + j];
            T[i * 3 + j] = s;
        }
    memcpy(C, T, sizeof(T));
}
static void transpose3(const double* A, double* B) {
    double T[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[i * 3 + j] = A[j * 3 + i];
    memcpy(B, T, sizeof(T));
}

/* Rotation of the normalised quaternion (w, x, y, z). */
void or_quat_to_rot(const double* q_in, double* R) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Real spherical harmonics up to degree 3 of a unit direction, index l*l+l+m,
 * orthonormal on the sphere (no Condon-Shortley phase).  Written from the
 * closed forms of the real harmonics; the constants are computed, not tabled. */
void or_sh_basis(const double* d, double* Y) {
    const double pi = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = k1 * y; Y[2] = k1 * z; Y[3] = k1 * x;
    double k2a = 0.5 * sqrt(15.0 / pi), k2b = 0.25 * sqrt(5.0 / pi), k2c = 0.25 * sqrt(15.0 / pi);
    Y[4] = k2a * x * y; Y[5] = k2a * y * z; Y[6] = k2b * (3 * z * z - 1);
    Y[7] = k2a * x * z; Y[8] = k2c * (x * x - y * y);
    double k3a = 0.25 * sqrt(35.0 / (2 * pi)), k3b = 0.5 * sqrt(105.0 / pi), k3c = 0.25 * sqrt(21.0 / (2 * pi));
    double k3d = 0.25 * sqrt(7.0 / pi), k3e = 0.25 * sqrt(105.0 / pi);
    Y[9] = k3a * y * (3 * x * x - y * y);
    Y[10] = k3b * x * y * z;
    Y[11] = k3c * y * (5 * z * z - 1);
    Y[12] = k3d * (5 * z * z * z - 3 * z);
    Y[13] = k3c * x * (5 * z * z - 1);
    Y[14] = k3e * z * (x * x - y * y);
    Y[15] = k3a * x * (x * x - 3 * y * y);
}

/* Gradient of sum_k w[k] Y_k(d) with respect to the components of d, taken
 * term by term from the closed forms above (d is treated as a free 3-vector;
 * the caller applies the derivative of the normalisation). */
static void sh_basis_grad(const double* d, const double* w, double* gd) {
    const double pi = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    double k1 = sqrt(3.0 / (4.0 * pi));
    double k2a = 0.5 * sqrt(15.0 / pi), k2b = 0.25 * sqrt(5.0 / pi), k2c = 0.25 * sqrt(15.0 / pi);
    double k3a = 0.25 * sqrt(35.0 / (2 * pi)), k3b = 0.5 * sqrt(105.0 / pi), k3c = 0.25 * sqrt(21.0 / (2 * pi));
    double k3d = 0.25 * sqrt(7.0 / pi), k3e = 0.25 * sqrt(105.0 / pi);
    double gx = 0, gy = 0, gz = 0;
    gy += w[1] * k1; gz += w[2] * k1; gx += w[3] * k1;
    gx += w[4] * k2a * y; gy += w[4] * k2a * x;
    gy += w[5] * k2a * z; gz += w[5] * k2a * y;
    gz += w[6] * k2b * 6 * z;
    gx += w[7] * k2a * z; gz += w[7] * k2a * x;
    gx += w[8] * k2c * 2 * x; gy -= w[8] * k2c * 2 * y;
    gx += w[9] * k3a * 6 * x * y; gy += w[9] * k3a * (3 * x * x - 3 * y * y);
    gx += w[10] * k3b * y * z; gy += w[10] * k3b * x * z; gz += w[10] * k3b * x * y;
    gy += w[11] * k3c * (5 * z * z - 1); gz += w[11] * k3c * 10 * y * z;
    gz += w[12] * k3d * (15 * z * z - 3);
    gx += w[13] * k3c * (5 * z * z - 1); gz += w[13] * k3c * 10 * x * z;
    gx += w[14] * k3e * 2 * x * z; gy -= w[14] * k3e * 2 * y * z; gz += w[14] * k3e * (x * x - y * y);
    gx += w[15] * k3a * (3 * x * x - 3 * y * y); gy -= w[15] * k3a * 6 * x * y;
    gd[0] = gx; gd[1] = gy; gd[2] = gz;
}

/* Tile rectangle [x0, x1) x [y0, y1) of a splat of integer radius r centred at
 * (mx, my) in sample coordinates: the tiles whose span [k t, (k+1) t) meets
 * [m - r, m + r], clamped to the grid.  Returns the number of tiles. */
static int tile_rect(double mx, double my, int r, int tile, int tx, int ty, int* rect) {
    double fx0 = floor((mx - r) / tile), fx1 = floor((mx + r) / tile) + 1;
    double fy0 = floor((my - r) / tile), fy1 = floor((my + r) / tile) + 1;
    if (fx0 < 0) fx0 = 0;
    if (fy0 < 0) fy0 = 0;
    if (fx1 > tx) fx1 = tx;
    if (fy1 > ty) fy1 = ty;
    if (!(fx1 > fx0) || !(fy1 > fy0)) { rect[0] = rect[1] = rect[2] = rect[3] = 0; return 0; }
    rect[0] = (int)fx0; rect[1] = (int)fy0; rect[2] = (int)fx1; rect[3] = (int)fy1;
    return (rect[2] - rect[0]) * (rect[3] - rect[1]);
}

int or_tile_rect(double mx, double my, int r, int tile, int tx, int ty, int* rect) {
    return tile_rect(mx, my, r, tile, tx, ty, rect);
}

/* Everything the projection computes for one Gaussian in one view. */
typedef struct {
    int visible;
    double R[9], s[3], M[9], Sigma[9];
    double pc[3], Sigma_c[9], J[6], cov2[3], det, conic[3], xy[2];
    double opacity, rgb[3], rgb_raw[3], dir[3], dist;
    int radius, rect[4], tiles;
    double margin;
} Proj;

static void project_one(const double* mu, const double* q, const double* ls, double logit,
                        const double* col, const Cam* c, const Prm* p, Proj* o) {
    memset(o, 0, sizeof(*o));
    o->margin = 1e30;
    or_quat_to_rot(q, o->R);
    for (int j = 0; j < 3; j++) o->s[j] = exp(ls[j]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) o->M[i * 3 + j] = o->R[i * 3 + j] * o->s[j];
    double Mt[9];
    transpose3(o->M, Mt);
    matmul3(o->M, Mt, o->Sigma);                        /* Sigma = M M^T */
    for (int r = 0; r < 3; r++) {
        o->pc[r] = c->tcw[r];
        for (int k = 0; k < 3; k++) o->pc[r] += c->Rcw[r * 3 + k] * mu[k];
    }
    o->opacity = 1.0 / (1.0 + exp(-logit));
    /* colour: direct RGB (degree 0) or degree-3 SH along the viewing ray */
    if (p->sh_degree == 0) {
        for (int k = 0; k < 3; k++) o->rgb[k] = o->rgb_raw[k] = col[k];
    } else {
        double dv[3], d2 = 0;
        for (int k = 0; k < 3; k++) { dv[k] = mu[k] - c->twc[k]; d2 += dv[k] * dv[k]; }
        o->dist = sqrt(d2);
        for (int k = 0; k < 3; k++) o->dir[k] = dv[k] / o->dist;
        double Y[16];
        or_sh_basis(o->dir, Y);
        for (int ch = 0; ch < 3; ch++) {
            double v = 0.5;
            for (int k = 0; k < 16; k++) v += col[k * 3 + ch] * Y[k];
            o->rgb_raw[ch] = v;
            o->rgb[ch] = v < 0 ? 0.0 : v;
        }
    }
    double z = o->pc[2];
    if (z <= p->near_plane) return;
    double Rt[9], tmp[9];
    transpose3(c->Rcw, Rt);
    matmul3(c->Rcw, o->Sigma, tmp);
    matmul3(tmp, Rt, o->Sigma_c);                        /* W Sigma W^T */
    double x = o->pc[0], y = o->pc[1];
    o->J[0] = c->fx / z; o->J[1] = 0.0;       o->J[2] = -c->fx * x / (z * z);
    o->J[3] = 0.0;       o->J[4] = c->fy / z; o->J[5] = -c->fy * y / (z * z);
    /* cov2 = J Sigma_c J^T + dil I  (2x2 symmetric: a, b, c) */
    double JS[6];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += o->J[i * 3 + k] * o->Sigma_c[k * 3 + j];
            JS[i * 3 + j] = s;
        }
    double C2[4];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += JS[i * 3 + k] * o->J[j * 3 + k];
            C2[i * 2 + j] = s;
        }
    o->cov2[0] = C2[0] + p->dil;
    o->cov2[1] = C2[1];
    o->cov2[2] = C2[3] + p->dil;
    o->det = o->cov2[0] * o->cov2[2] - o->cov2[1] * o->cov2[1];
    if (!(o->det > 0.0)) return;
    o->conic[0] = o->cov2[2] / o->det;
    o->conic[1] = -o->cov2[1] / o->det;
    o->conic[2] = o->cov2[0] / o->det;
    o->xy[0] = c->fx * x / z + c->cx;
    o->xy[1] = c->fy * y / z + c->cy;
    double mid = 0.5 * (o->cov2[0] + o->cov2[2]);
    double disc = mid * mid - o->det;
    if (disc < 0.1) disc = 0.1;
    double lmax = mid + sqrt(disc);
    double rr = p->k_sigma * sqrt(lmax);
    /* a radius only selects tiles; 2^24 px already covers any image */
    o->radius = rr < 16777216.0 ? (int)ceil(rr) : 16777216;
    double fr = rr - floor(rr);
    o->margin = fr < 1 - fr ? fr : 1 - fr;   /* distance of the radius to an integer */
    if (o->radius <= 0) return;
    int tx = tiles_x_of(c, p), ty = tiles_y_of(c, p);
    if (p->smooth) {
        o->rect[0] = 0; o->rect[1] = 0; o->rect[2] = tx; o->rect[3] = ty;
        o->tiles = tx * ty;
    } else {
        /* keys and rectangles are taken from the fp32-rounded centre */
        double mx = (double)(float)o->xy[0], my = (double)(float)o->xy[1];
        o->tiles = tile_rect(mx, my, o->radius, p->tile, tx, ty, o->rect);
        double e[4] = {mx - o->radius, mx + o->radius, my - o->radius, my + o->radius};
        for (int k = 0; k < 4; k++) {
            double f = e[k] / p->tile - floor(e[k] / p->tile);
            double m = (f < 1 - f ? f : 1 - f) * p->tile;
            if (m < o->margin) o->margin = m;
        }
    }
    o->visible = o->tiles > 0;
}

/* Projection of n Gaussians into one view (Sec. 3.3 "Preliminary" + EWA). */
void or_project(long n, const double* mean, const double* quat, const double* log_scale,
                const double* logit, const double* color, const double* cam, const double* prm,
                double* xy, double* cov2, double* conic, double* depth, double* opacity,
                double* rgb, int* radius, int* rect, int* tiles, double* margin) {
    Cam c = cam_from(cam);
    Prm p = prm_from(prm);
    int nc = p.sh_degree == 0 ? 3 : 48;
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long i = 0; i < n; i++) {
        Proj o;
        project_one(mean + 3 * i, quat + 4 * i, log_scale + 3 * i, logit[i], color + nc * i, &c, &p, &o);
        xy[2 * i] = o.xy[0]; xy[2 * i + 1] = o.xy[1];
        for (int k = 0; k < 3; k++) {
            cov2[3 * i + k] = o.cov2[k];
            conic[3 * i + k] = o.visible ? o.conic[k] : 0.0;
            rgb[3 * i + k] = o.rgb[k];
        }
        depth[i] = o.pc[2];
        opacity[i] = o.opacity;
        radius[i] = o.visible ? o.radius : 0;
        for (int k = 0; k < 4; k++) rect[4 * i + k] = o.visible ? o.rect[k] : 0;
        tiles[i] = o.visible ? o.tiles : 0;
        margin[i] = o.margin;
    }
}

/* ---------------------------------------------------------------- binning */

typedef struct { uint64_t key; uint32_t val; } KV;

static int kv_cmp(const void* a, const void* b) {
    const KV* x = (const KV*)a;
    const KV* y = (const KV*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

static uint32_t f32_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Number of (entry, tile) pairs. */
long or_bin_count(long n_entries, const int* rect) {
    long m = 0;
    for (long e = 0; e < n_entries; e++)
        m += (long)(rect[4 * e + 2] - rect[4 * e]) * (rect[4 * e + 3] - rect[4 * e + 1]);
    return m;
}

/* Keys, values and per-tile ranges by enumeration and a comparison sort.
 * Entry e belongs to view view_of[e]; its tiles are numbered
 * tile_base[v] + ty * tiles_x[v] + tx.  key = (global tile << 32) | bits(depth
 * as fp32); value = e; order = (key, e), which is what a stable sort of the
 * enumeration (made in entry order) by key gives.  ranges[2g] / [2g+1] = the
 * [start, end) of global tile g in the sorted list (0, 0 when empty). */
long or_bin_sort(long n_entries, const float* depth, const int* rect, const int* view_of,
                 const int* tile_base, const int* tiles_x, long total_tiles,
                 uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
    long m = or_bin_count(n_entries, rect);
    KV* kv = (KV*)malloc(sizeof(KV) * (m > 0 ? m : 1));
    long k = 0;
    for (long e = 0; e < n_entries; e++) {
        int v = view_of[e];
        for (int ty = rect[4 * e + 1]; ty < rect[4 * e + 3]; ty++)
            for (int tx = rect[4 * e]; tx < rect[4 * e + 2]; tx++) {
                uint64_t g = (uint64_t)(tile_base[v] + ty * tiles_x[v] + tx);
                kv[k].key = (g << 32) | f32_bits(depth[e]);
                kv[k].val = (uint32_t)e;
                k++;
            }
    }
    qsort(kv, m, sizeof(KV), kv_cmp);
    for (long g = 0; g < 2 * total_tiles; g++) ranges[g] = 0;
    for (long i = 0; i < m; i++) {
        keys[i] = kv[i].key;
        vals[i] = kv[i].val;
        long g = (long)(kv[i].key >> 32);
        if (i == 0 || (long)(kv[i - 1].key >> 32) != g) ranges[2 * g] = (uint32_t)i;
        if (i == m - 1 || (long)(kv[i + 1].key >> 32) != g) ranges[2 * g + 1] = (uint32_t)(i + 1);
    }
    free(kv);
    return m;
}

/* ------------------------------------------------------------- compositing */

typedef struct { double z; long idx; } ZI;

static int zi_cmp(const void* a, const void* b) {
    const ZI* x = (const ZI*)a;
    const ZI* y = (const ZI*)b;
    if (x->z != y->z) return x->z < y->z ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/* The Gaussians whose rectangle covers tile (tx, ty), ordered front to back
 * by (depth, index). */
static long tile_list(long n, const double* depth, const int* rect, int tx, int ty, ZI* out) {
    long m = 0;
    for (long i = 0; i < n; i++) {
        const int* r = rect + 4 * i;
        if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) {
            out[m].z = depth[i];
            out[m].idx = i;
            m++;
        }
    }
    qsort(out, m, sizeof(ZI), zi_cmp);
    return m;
}

/* Per-pixel record of one pass over a tile list. */
typedef struct {
    long list_pos;   /* position in the tile list */
    long idx;        /* Gaussian */
    double alpha, T_before, G, dx, dy;
    int clamped;
} Blend;

/* Composite one pixel front to back.  Returns the number of blended splats
 * written to `bl` and fills the pixel outputs.  *margin receives the smallest
 * relative distance of any threshold decision to its threshold. */
static long composite_pixel(const ZI* list, long m, double sx, double sy,
                            const double* xy, const double* conic, const double* opacity,
                            const double* rgb, const double* depth, const Prm* p,
                            double* C, double* D, double* T_out, int* n_out, double* margin,
                            Blend* bl) {
    double T = 1.0;
    double c3[3] = {0, 0, 0}, d = 0;
    long nb = 0, last = -1;
    double mg = 1e30;
    for (long k = 0; k < m; k++) {
        long i = list[k].idx;
        double dx = sx - xy[2 * i], dy = sy - xy[2 * i + 1];
        double A = conic[3 * i], B = conic[3 * i + 1], Cc = conic[3 * i + 2];
        double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        if (!p->smooth && power > 0.0) continue;
        double G = exp(power);
        double a_raw = opacity[i] * G;
        double alpha = a_raw < p->a_max ? a_raw : p->a_max;
        if (!p->smooth) {
            double r = fabs(a_raw - p->a_min) / p->a_min;
            if (r < mg) mg = r;
        }
        if (alpha < p->a_min) continue;
        double test = T * (1.0 - alpha);
        if (!p->smooth) {
            double r = fabs(test - p->T_cut) / p->T_cut;
            if (r < mg) mg = r;
        }
        if (test < p->T_cut) break;
        double w = alpha * T;
        for (int ch = 0; ch < 3; ch++) c3[ch] += rgb[3 * i + ch] * w;
        d += depth[i] * w;
        if (bl) {
            bl[nb].list_pos = k; bl[nb].idx = i; bl[nb].alpha = alpha; bl[nb].T_before = T;
            bl[nb].G = G; bl[nb].dx = dx; bl[nb].dy = dy; bl[nb].clamped = !(a_raw < p->a_max);
        }
        nb++;
        T = test;
        last = k;
    }
    for (int ch = 0; ch < 3; ch++) C[ch] = c3[ch] + T * p->bg[ch];
    *D = d;
    *T_out = T;
    *n_out = (int)(last + 1);
    *margin = mg;
    return nb;
}

/* Forward render of one view from per-Gaussian projected quantities. */
void or_render_fwd(long n, const double* xy, const double* conic, const double* opacity,
                   const double* rgb, const double* depth, const int* rect,
                   const double* cam, const double* prm,
                   double* out_color, double* out_depth, double* out_T, int* out_n, double* out_margin) {
    Cam c = cam_from(cam);
    Prm p = prm_from(prm);
    int t = p.tile, tx = tiles_x_of(&c, &p), ty = tiles_y_of(&c, &p);
    long HW = (long)c.W * c.H;
    /* tiles in row-major order; each pixel is written by its own tile only */
#pragma omp parallel num_threads(g_threads)
    {
        ZI* list = (ZI*)malloc(sizeof(ZI) * (n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
        for (long b = 0; b < (long)tx * ty; b++) {
            int by = (int)(b / tx), bx = (int)(b % tx);
            long m = tile_list(n, depth, rect, bx, by, list);
            for (int py = by * t; py < (by + 1) * t && py < c.H; py++)
                for (int px = bx * t; px < (bx + 1) * t && px < c.W; px++) {
                    double C3[3], D, T, mg;
                    int np;
                    composite_pixel(list, m, px + 0.5, py + 0.5, xy, conic, opacity, rgb, depth, &p,
                                    C3, &D, &T, &np, &mg, NULL);
                    long pix = (long)py * c.W + px;
                    for (int ch = 0; ch < 3; ch++) out_color[ch * HW + pix] = C3[ch];
                    out_depth[pix] = D;
                    out_T[pix] = T;
                    out_n[pix] = np;
                    out_margin[pix] = mg;
                }
        }
        free(list);
    }
}

/* One blended (pixel, splat) pair's additions to the per-Gaussian gradients
 * of the compositing backward, in the form the serial loop adds them. */
typedef struct {
    long idx;
    int clamped;                  /* alpha = alpha_max: no opacity / conic / xy terms */
    double rgb[3], depth, opacity, conic[3], xy[2];
} Contrib;

typedef struct {
    Contrib* c;
    long n, cap;
} ContribList;

static void contrib_push(ContribList* L, const Contrib* x) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->c = (Contrib*)realloc(L->c, sizeof(Contrib) * L->cap);
    }
    L->c[L->n++] = *x;
}

/* The contributions of every pixel of tile (bx, by), pixels in row-major
 * order, each pixel's blended splats front to back.  d colour / d alpha_j is
 * taken straight from the product form C = sum_i c_i alpha_i T_i + bg T_final
 * with T_i = prod_{k<i} (1 - alpha_k). */
static void tile_backward(long n, int bx, int by, const double* xy, const double* conic, const double* opacity,
                          const double* rgb, const double* depth, const int* rect, const Cam* c, const Prm* p,
                          const double* dL_dcolor, const double* dL_ddepth, ZI* list, Blend* bl, double* sufC,
                          double* sufD, ContribList* out) {
    int t = p->tile;
    long HW = (long)c->W * c->H;
    long m = tile_list(n, depth, rect, bx, by, list);
    for (int py = by * t; py < (by + 1) * t && py < c->H; py++)
        for (int px = bx * t; px < (bx + 1) * t && px < c->W; px++) {
            double C3[3], D, T, mg;
            int np;
            long nb = composite_pixel(list, m, px + 0.5, py + 0.5, xy, conic, opacity, rgb, depth, p, C3, &D,
                                      &T, &np, &mg, bl);
            long pix = (long)py * c->W + px;
            double gC[3] = {dL_dcolor[pix], dL_dcolor[HW + pix], dL_dcolor[2 * HW + pix]};
            double gD = dL_ddepth[pix];
            /* suffix sums of the contributions behind blended splat j, plus background */
            for (int ch = 0; ch < 3; ch++) sufC[3 * nb + ch] = p->bg[ch] * T;
            sufD[nb] = 0.0;
            for (long j = nb - 1; j >= 0; j--) {
                long i = bl[j].idx;
                double w = bl[j].alpha * bl[j].T_before;
                for (int ch = 0; ch < 3; ch++) sufC[3 * j + ch] = sufC[3 * (j + 1) + ch] + rgb[3 * i + ch] * w;
                sufD[j] = sufD[j + 1] + depth[i] * w;
            }
            for (long j = 0; j < nb; j++) {
                long i = bl[j].idx;
                double a = bl[j].alpha, Tb = bl[j].T_before, w = a * Tb;
                double dC_da[3], dD_da;
                Contrib r;
                memset(&r, 0, sizeof(r));
                r.idx = i;
                for (int ch = 0; ch < 3; ch++)
                    dC_da[ch] = rgb[3 * i + ch] * Tb - sufC[3 * (j + 1) + ch] / (1.0 - a);
                dD_da = depth[i] * Tb - sufD[j + 1] / (1.0 - a);
                double dL_da = gD * dD_da;
                for (int ch = 0; ch < 3; ch++) {
                    dL_da += gC[ch] * dC_da[ch];
                    r.rgb[ch] = gC[ch] * w;
                }
                r.depth = gD * w;
                r.clamped = bl[j].clamped;
                if (!r.clamped) {    /* alpha = alpha_max is flat in o and power */
                    double G = bl[j].G;
                    r.opacity = dL_da * G;
                    double dL_dpow = dL_da * opacity[i] * G;
                    double dx = bl[j].dx, dy = bl[j].dy;
                    double A = conic[3 * i], B = conic[3 * i + 1], Cc = conic[3 * i + 2];
                    /* power = -1/2 (A dx^2 + C dy^2) - B dx dy, dx = sample - mean */
                    r.conic[0] = dL_dpow * (-0.5 * dx * dx);
                    r.conic[1] = dL_dpow * (-dx * dy);
                    r.conic[2] = dL_dpow * (-0.5 * dy * dy);
                    r.xy[0] = dL_dpow * (A * dx + B * dy);
                    r.xy[1] = dL_dpow * (B * dx + Cc * dy);
                }
                contrib_push(out, &r);
            }
        }
}

/* Backward of the compositing for one view: accumulates (+=) the gradient of
 * sum_pix <dL_dcolor, colour> + <dL_ddepth, depth> into per-Gaussian
 * gradients of xy (2), conic (3), opacity (1), rgb (3) and depth (1).  The
 * tiles' contributions are formed (in parallel when threads > 1) and added in
 * tile order, pixel order, splat order: the order of one serial pass. */
void or_render_bwd(long n, const double* xy, const double* conic, const double* opacity,
                   const double* rgb, const double* depth, const int* rect,
                   const double* cam, const double* prm,
                   const double* dL_dcolor, const double* dL_ddepth,
                   double* g_xy, double* g_conic, double* g_opacity, double* g_rgb, double* g_depth) {
    Cam c = cam_from(cam);
    Prm p = prm_from(prm);
    int tx = tiles_x_of(&c, &p), ty = tiles_y_of(&c, &p);
    long n_tiles = (long)tx * ty;
    long chunk = g_threads > 1 ? 4L * g_threads : 1L;      /* tiles whose contributions are held at once */
    ContribList* lists = (ContribList*)calloc((size_t)chunk, sizeof(ContribList));
    for (long b0 = 0; b0 < n_tiles; b0 += chunk) {
        long b1 = b0 + chunk < n_tiles ? b0 + chunk : n_tiles;
#pragma omp parallel num_threads(g_threads)
        {
            ZI* list = (ZI*)malloc(sizeof(ZI) * (n > 0 ? n : 1));
            Blend* bl = (Blend*)malloc(sizeof(Blend) * (n > 0 ? n : 1));
            double* sufC = (double*)malloc(sizeof(double) * 3 * (n + 1));
            double* sufD = (double*)malloc(sizeof(double) * (n + 1));
#pragma omp for schedule(dynamic, 1)
            for (long b = b0; b < b1; b++) {
                lists[b - b0].n = 0;
                tile_backward(n, (int)(b % tx), (int)(b / tx), xy, conic, opacity, rgb, depth, rect, &c, &p,
                              dL_dcolor, dL_ddepth, list, bl, sufC, sufD, &lists[b - b0]);
            }
            free(list); free(bl); free(sufC); free(sufD);
        }
        for (long b = b0; b < b1; b++) {
            const ContribList* L = &lists[b - b0];
            for (long k = 0; k < L->n; k++) {
                const Contrib* r = &L->c[k];
                long i = r->idx;
                for (int ch = 0; ch < 3; ch++) g_rgb[3 * i + ch] += r->rgb[ch];
                g_depth[i] += r->depth;
                if (r->clamped) continue;
                g_opacity[i] += r->opacity;
                for (int q = 0; q < 3; q++) g_conic[3 * i + q] += r->conic[q];
                g_xy[2 * i] += r->xy[0];
                g_xy[2 * i + 1] += r->xy[1];
            }
        }
    }
    for (long k = 0; k < chunk; k++) free(lists[k].c);
    free(lists);
}

/* Backward of the projection for one view: accumulates (+=) into parameter
 * gradients and the 6-vector pose gradient (rho, phi) of a left perturbation
 * T_cw <- Exp(xi) T_cw, from per-Gaussian gradients of the projected
 * quantities.  Entries that were not visible contribute nothing. */
void or_project_bwd(long n, const double* mean, const double* quat, const double* log_scale,
                    const double* logit, const double* color, const double* cam, const double* prm,
                    const double* g_xy, const double* g_conic, const double* g_opacity,
                    const double* g_rgb, const double* g_depth,
                    double* g_mean, double* g_quat, double* g_log_scale, double* g_logit,
                    double* g_color, double* g_pose) {
    Cam c = cam_from(cam);
    Prm p = prm_from(prm);
    int nc = p.sh_degree == 0 ? 3 : 48;
    /* each Gaussian's pose-gradient terms, added up in Gaussian order afterwards */
    double* pose_terms = g_pose ? (double*)malloc(sizeof(double) * 6 * (n > 0 ? n : 1)) : NULL;
    char* visible = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long i = 0; i < n; i++) {
        Proj o;
        const double* q = quat + 4 * i;
        project_one(mean + 3 * i, q, log_scale + 3 * i, logit[i], color + nc * i, &c, &p, &o);
        if (!o.visible) continue;
        visible[i] = 1;
        double z = o.pc[2], x = o.pc[0], y = o.pc[1];
        double a = o.cov2[0], b = o.cov2[1], cc = o.cov2[2], det = o.det, det2 = det * det;
        const double* gq = g_conic + 3 * i;
        /* conic = (c, -b, a) / det */
        double Ga = gq[0] * (-cc * cc / det2) + gq[1] * (b * cc / det2) + gq[2] * (-b * b / det2);
        double Gb = gq[0] * (2 * b * cc / det2) + gq[1] * (-(det + 2 * b * b) / det2) + gq[2] * (2 * a * b / det2);
        double Gc = gq[0] * (-b * b / det2) + gq[1] * (a * b / det2) + gq[2] * (-a * a / det2);
        double G2[4] = {Ga, 0.5 * Gb, 0.5 * Gb, Gc};   /* symmetric gradient of the 2x2 covariance */
        /* G_J = 2 G2 J Sigma_c ; G_Sigma_c = J^T G2 J */
        double JS[6], GJ[6], GSc[9];
        for (int r = 0; r < 2; r++)
            for (int j = 0; j < 3; j++) {
                double s = 0;
                for (int k = 0; k < 3; k++) s += o.J[r * 3 + k] * o.Sigma_c[k * 3 + j];
                JS[r * 3 + j] = s;
            }
        for (int r = 0; r < 2; r++)
            for (int j = 0; j < 3; j++) GJ[r * 3 + j] = 2.0 * (G2[r * 2] * JS[j] + G2[r * 2 + 1] * JS[3 + j]);
        for (int r = 0; r < 3; r++)
            for (int j = 0; j < 3; j++) {
                double s = 0;
                for (int u = 0; u < 2; u++)
                    for (int v = 0; v < 2; v++) s += o.J[u * 3 + r] * G2[u * 2 + v] * o.J[v * 3 + j];
                GSc[r * 3 + j] = s;
            }
        double gu = g_xy[2 * i], gv = g_xy[2 * i + 1];
        double Gpc[3];
        Gpc[0] = gu * c.fx / z + GJ[2] * (-c.fx / (z * z));
        Gpc[1] = gv * c.fy / z + GJ[5] * (-c.fy / (z * z));
        Gpc[2] = -gu * c.fx * x / (z * z) - gv * c.fy * y / (z * z) + g_depth[i]
                 + GJ[0] * (-c.fx / (z * z)) + GJ[2] * (2 * c.fx * x / (z * z * z))
                 + GJ[4] * (-c.fy / (z * z)) + GJ[5] * (2 * c.fy * y / (z * z * z));
        /* mean: p_c = W mu + t */
        for (int k = 0; k < 3; k++) {
            double s = 0;
            for (int r = 0; r < 3; r++) s += c.Rcw[r * 3 + k] * Gpc[r];
            g_mean[3 * i + k] += s;
        }
        /* G_Sigma = W^T G_Sigma_c W ; G_M = 2 G_Sigma M */
        double Wt[9], tmp[9], GS[9], GM[9];
        transpose3(c.Rcw, Wt);
        matmul3(Wt, GSc, tmp);
        matmul3(tmp, c.Rcw, GS);
        matmul3(GS, o.M, GM);
        for (int k = 0; k < 9; k++) GM[k] *= 2.0;
        double GR[9];
        for (int r = 0; r < 3; r++)
            for (int j = 0; j < 3; j++) GR[r * 3 + j] = GM[r * 3 + j] * o.s[j];
        for (int j = 0; j < 3; j++) {
            double gs = 0;
            for (int r = 0; r < 3; r++) gs += GM[r * 3 + j] * o.R[r * 3 + j];
            g_log_scale[3 * i + j] += gs * o.s[j];
        }
        /* rotation of the normalised quaternion */
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double w = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
        double dW[9] = {0, -2 * qz, 2 * qy, 2 * qz, 0, -2 * qx, -2 * qy, 2 * qx, 0};
        double dX[9] = {0, 2 * qy, 2 * qz, 2 * qy, -4 * qx, -2 * w, 2 * qz, 2 * w, -4 * qx};
        double dY[9] = {-4 * qy, 2 * qx, 2 * w, 2 * qx, 0, 2 * qz, -2 * w, 2 * qz, -4 * qy};
        double dZ[9] = {-4 * qz, -2 * w, 2 * qx, 2 * w, -4 * qz, 2 * qy, 2 * qx, 2 * qy, 0};
        double gqn[4] = {0, 0, 0, 0};
        for (int k = 0; k < 9; k++) {
            gqn[0] += GR[k] * dW[k]; gqn[1] += GR[k] * dX[k];
            gqn[2] += GR[k] * dY[k]; gqn[3] += GR[k] * dZ[k];
        }
        double qhat[4] = {w, qx, qy, qz};
        double dot = 0;
        for (int k = 0; k < 4; k++) dot += qhat[k] * gqn[k];
        for (int k = 0; k < 4; k++) g_quat[4 * i + k] += (gqn[k] - qhat[k] * dot) / qn;
        /* opacity = sigmoid(logit) */
        g_logit[i] += g_opacity[i] * o.opacity * (1.0 - o.opacity);
        /* colour */
        double Gcenter[3] = {0, 0, 0};
        if (p.sh_degree == 0) {
            for (int k = 0; k < 3; k++) g_color[3 * i + k] += g_rgb[3 * i + k];
        } else {
            double Y[16], gr[3], wsum[16];
            or_sh_basis(o.dir, Y);
            for (int ch = 0; ch < 3; ch++) gr[ch] = o.rgb_raw[ch] < 0 ? 0.0 : g_rgb[3 * i + ch];
            for (int k = 0; k < 16; k++) {
                wsum[k] = 0;
                for (int ch = 0; ch < 3; ch++) {
                    g_color[48 * i + 3 * k + ch] += gr[ch] * Y[k];
                    wsum[k] += gr[ch] * color[48 * i + 3 * k + ch];
                }
            }
            double gdir[3];
            sh_basis_grad(o.dir, wsum, gdir);
            /* dir = v / |v|, v = mu - centre */
            double dd = 0;
            for (int k = 0; k < 3; k++) dd += o.dir[k] * gdir[k];
            for (int k = 0; k < 3; k++) {
                double gv3 = (gdir[k] - o.dir[k] * dd) / o.dist;
                g_mean[3 * i + k] += gv3;
                Gcenter[k] -= gv3;
            }
        }
        if (g_pose) {
            /* rho: p_c += rho ; phi: p_c += phi x p_c, W <- (I + [phi]x) W */
            double GSS[9];
            matmul3(GSc, o.Sigma_c, GSS);
            double gphi[3];
            gphi[0] = o.pc[1] * Gpc[2] - o.pc[2] * Gpc[1] + 2.0 * (GSS[7] - GSS[5]);
            gphi[1] = o.pc[2] * Gpc[0] - o.pc[0] * Gpc[2] + 2.0 * (GSS[2] - GSS[6]);
            gphi[2] = o.pc[0] * Gpc[1] - o.pc[1] * Gpc[0] + 2.0 * (GSS[3] - GSS[1]);
            double grho[3] = {Gpc[0], Gpc[1], Gpc[2]};
            /* camera centre C = -R_cw^T t_cw moves by -R_cw^T rho under rho */
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++) grho[r] -= c.Rcw[r * 3 + k] * Gcenter[k];
            for (int k = 0; k < 3; k++) { pose_terms[6 * i + k] = grho[k]; pose_terms[6 * i + 3 + k] = gphi[k]; }
        }
    }
    if (g_pose)
        for (long i = 0; i < n; i++) {
            if (!visible[i]) continue;
            for (int k = 0; k < 3; k++) {
                g_pose[k] += pose_terms[6 * i + k];
                g_pose[3 + k] += pose_terms[6 * i + 3 + k];
            }
        }
    free(pose_terms);
    free(visible);
}

/* ------------------------------------------------------------------ losses */

/* Eq. 6 colour and depth terms of one view: L_c = mean over 3HW of |I_hat - I|,
 * L_d = mean over pixels with D > 0 of |D_hat - D|; sign(0) = 0.  Writes
 * dL/dI_hat = lambda_c sign / (3HW) and dL/dD_hat = lambda_d sign / n_valid. */
void or_l1_loss(long HW, const double* color, const double* depth, const double* tcolor,
                const double* tdepth, double lambda_c, double lambda_d, double* out_terms,
                double* dcolor, double* ddepth) {
    double sc = 0, sd = 0;
    long nv = 0;
    for (long k = 0; k < 3 * HW; k++) {
        double r = color[k] - tcolor[k];
        sc += fabs(r);
        dcolor[k] = lambda_c * ((r > 0) - (r < 0)) / (3.0 * HW);
    }
    for (long k = 0; k < HW; k++)
        if (tdepth[k] > 0) nv++;
    for (long k = 0; k < HW; k++) {
        if (tdepth[k] > 0) {
            double r = depth[k] - tdepth[k];
            sd += fabs(r);
            ddepth[k] = lambda_d * ((r > 0) - (r < 0)) / (double)nv;
        } else {
            ddepth[k] = 0.0;
        }
    }
    out_terms[0] = sc / (3.0 * HW);
    out_terms[1] = nv > 0 ? sd / nv : 0.0;
}

/* Isotropic regulariser (the MonoGS form cited in Sec. 3.3):
 * L_iso = (1/n) sum_i sum_j |s_ij - mean_j s_ij| with s = exp(log_scale).
 * Returns L_iso and adds lambda dL_iso/dlog_scale into g_log_scale. */
double or_iso_loss(long n, const double* log_scale, double lambda, double* g_log_scale) {
    double L = 0;
    for (long i = 0; i < n; i++) {
        double s[3], m = 0;
        for (int j = 0; j < 3; j++) { s[j] = exp(log_scale[3 * i + j]); m += s[j] / 3.0; }
        double sg[3];
        for (int j = 0; j < 3; j++) {
            double r = s[j] - m;
            L += fabs(r);
            sg[j] = (r > 0) - (r < 0);
        }
        double sum_sg = sg[0] + sg[1] + sg[2];
        for (int k = 0; k < 3; k++) {
            double ds = sg[k] - sum_sg / 3.0;     /* d/ds_k sum_j |s_j - mean| */
            g_log_scale[3 * i + k] += lambda * ds * s[k] / (double)n;
        }
    }
    return n > 0 ? L / (double)n : 0.0;
}

/* Adam with bias correction (the optimiser of the mapping iterations). */
void or_adam(long n, double* param, const double* grad, double* m, double* v,
             double lr, double beta1, double beta2, double eps, int step) {
    double bc1 = 1.0 - pow(beta1, step), bc2 = 1.0 - pow(beta2, step);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long k = 0; k < n; k++) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * grad[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * grad[k] * grad[k];
        double mh = m[k] / bc1, vh = v[k] / bc2;
        param[k] -= lr * mh / (sqrt(vh) + eps);
    }
}
