// project.cu -- EWA projection of the Gaussian map into every view and its
// backward pass (Sec. 3.3 "Preliminary": mean, covariance from rotation and
// scale, opacity, direct RGB colour; degree-3 SH colour as an option).
//
// One thread per Gaussian loops over the views, so the activation of the
// parameters (quaternion normalisation, exp of the log-scales, 3D covariance)
// is done once per Gaussian however many views are rendered.  Inputs are read
// as SoA rows (float4 for the quaternion); outputs are written as float2 /
// float4 / int4 rows per entry.
#include <math.h>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kProjThreads = 256;
constexpr int kMaxRadius = 1 << 24;

struct Activated {
    float mu[3];
    float q[4];          // normalised (w, x, y, z)
    float qnorm;
    float R[9];
    float s[3];
    float M[9];          // R diag(s)
    float S[6];          // Sigma = M M^T: xx, xy, xz, yy, yz, zz
    float o;
};

__device__ __forceinline__ void activate(const gs_gaussians& g, int i, Activated& a) {
    a.mu[0] = g.mean[3 * i]; a.mu[1] = g.mean[3 * i + 1]; a.mu[2] = g.mean[3 * i + 2];
    float4 q = reinterpret_cast<const float4*>(g.quat)[i];
    float nn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    a.qnorm = nn;
    float inv = 1.0f / nn;
    float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    a.q[0] = w; a.q[1] = x; a.q[2] = y; a.q[3] = z;
    a.R[0] = 1.f - 2.f * (y * y + z * z); a.R[1] = 2.f * (x * y - w * z);       a.R[2] = 2.f * (x * z + w * y);
    a.R[3] = 2.f * (x * y + w * z);       a.R[4] = 1.f - 2.f * (x * x + z * z); a.R[5] = 2.f * (y * z - w * x);
    a.R[6] = 2.f * (x * z - w * y);       a.R[7] = 2.f * (y * z + w * x);       a.R[8] = 1.f - 2.f * (x * x + y * y);
#pragma unroll
    for (int j = 0; j < 3; j++) a.s[j] = expf(g.log_scale[3 * i + j]);
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int j = 0; j < 3; j++) a.M[3 * r + j] = a.R[3 * r + j] * a.s[j];
    const float* M = a.M;
    a.S[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    a.S[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    a.S[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    a.S[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    a.S[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    a.S[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    a.o = 1.0f / (1.0f + expf(-g.opacity_logit[i]));
}

// Real spherical harmonics of degree <= 3 of a unit direction, index l*l+l+m,
// orthonormal on the sphere; the constants are the closed-form normalisations
// of the real harmonics (e.g. 1/(2 sqrt(pi)), sqrt(3/(4 pi)), 1/2 sqrt(15/pi)).
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
    const float c0 = (float)(0.5 / 1.7724538509055159);               // 1 / (2 sqrt(pi))
    const float c1 = (float)(0.4886025119029199);                      // sqrt(3 / (4 pi))
    const float c2a = (float)(1.0925484305920792), c2b = (float)(0.31539156525252005), c2c = (float)(0.5462742152960396);
    const float c3a = (float)(0.5900435899266435), c3b = (float)(2.890611442640554), c3c = (float)(0.4570457994644658);
    const float c3d = (float)(0.3731763325901154), c3e = (float)(1.445305721320277);
    Y[0] = c0;
    Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    Y[4] = c2a * x * y; Y[5] = c2a * y * z; Y[6] = c2b * (3.f * z * z - 1.f); Y[7] = c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    Y[9] = c3a * y * (3.f * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = c3c * y * (5.f * z * z - 1.f);
    Y[12] = c3d * (5.f * z * z * z - 3.f * z);
    Y[13] = c3c * x * (5.f * z * z - 1.f);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = c3a * x * (x * x - 3.f * y * y);
}

// d/d(x,y,z) of sum_k w_k Y_k, the components treated as free variables.
__device__ __forceinline__ void sh_grad(float x, float y, float z, const float* w, float* gd) {
    const float c1 = (float)(0.4886025119029199);
    const float c2a = (float)(1.0925484305920792), c2b = (float)(0.31539156525252005), c2c = (float)(0.5462742152960396);
    const float c3a = (float)(0.5900435899266435), c3b = (float)(2.890611442640554), c3c = (float)(0.4570457994644658);
    const float c3d = (float)(0.3731763325901154), c3e = (float)(1.445305721320277);
    float gx = w[3] * c1, gy = w[1] * c1, gz = w[2] * c1;
    gx += c2a * (w[4] * y + w[7] * z) + c2c * w[8] * 2.f * x;
    gy += c2a * (w[4] * x + w[5] * z) - c2c * w[8] * 2.f * y;
    gz += c2a * (w[5] * y + w[7] * x) + c2b * w[6] * 6.f * z;
    gx += w[9] * c3a * 6.f * x * y + w[10] * c3b * y * z + w[13] * c3c * (5.f * z * z - 1.f) +
          w[14] * c3e * 2.f * x * z + w[15] * c3a * (3.f * x * x - 3.f * y * y);
    gy += w[9] * c3a * (3.f * x * x - 3.f * y * y) + w[10] * c3b * x * z + w[11] * c3c * (5.f * z * z - 1.f) -
          w[14] * c3e * 2.f * y * z - w[15] * c3a * 6.f * x * y;
    gz += w[10] * c3b * x * y + w[11] * c3c * 10.f * y * z + w[12] * c3d * (15.f * z * z - 3.f) +
          w[13] * c3c * 10.f * x * z + w[14] * c3e * (x * x - y * y);
    gd[0] = gx; gd[1] = gy; gd[2] = gz;
}

// Camera-dependent part of the projection for one view.
struct ViewProj {
    bool visible;
    float pc[3];
    float inv_z;
    float T[6];          // J W, 2x3 row-major
    float a, b, c, det;
    float conic[3];
    float u, v;
    int radius;
    int rect[4];
    int tiles;
};

__device__ __forceinline__ void project_view(const Activated& A, const ViewParams& vp, const RenderConsts& rc,
                                             ViewProj& P) {
    P.visible = false;
    P.tiles = 0;
    P.radius = 0;
    const float* W = vp.Rcw;
#pragma unroll
    for (int r = 0; r < 3; r++)
        P.pc[r] = W[3 * r] * A.mu[0] + W[3 * r + 1] * A.mu[1] + W[3 * r + 2] * A.mu[2] + vp.tcw[r];
    const float z = P.pc[2];
    if (!(z > rc.near_plane)) return;
    const float iz = 1.0f / z;
    P.inv_z = iz;
    const float j00 = vp.fx * iz, j02 = -vp.fx * P.pc[0] * iz * iz;
    const float j11 = vp.fy * iz, j12 = -vp.fy * P.pc[1] * iz * iz;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        P.T[k] = j00 * W[k] + j02 * W[6 + k];
        P.T[3 + k] = j11 * W[3 + k] + j12 * W[6 + k];
    }
    // Sigma T^T columns
    const float* S = A.S;
    float st0[3], st1[3];
    st0[0] = S[0] * P.T[0] + S[1] * P.T[1] + S[2] * P.T[2];
    st0[1] = S[1] * P.T[0] + S[3] * P.T[1] + S[4] * P.T[2];
    st0[2] = S[2] * P.T[0] + S[4] * P.T[1] + S[5] * P.T[2];
    st1[0] = S[0] * P.T[3] + S[1] * P.T[4] + S[2] * P.T[5];
    st1[1] = S[1] * P.T[3] + S[3] * P.T[4] + S[4] * P.T[5];
    st1[2] = S[2] * P.T[3] + S[4] * P.T[4] + S[5] * P.T[5];
    P.a = P.T[0] * st0[0] + P.T[1] * st0[1] + P.T[2] * st0[2] + rc.dilation;
    P.b = P.T[0] * st1[0] + P.T[1] * st1[1] + P.T[2] * st1[2];
    P.c = P.T[3] * st1[0] + P.T[4] * st1[1] + P.T[5] * st1[2] + rc.dilation;
    P.det = P.a * P.c - P.b * P.b;
    if (!(P.det > 0.0f)) return;
    const float idet = 1.0f / P.det;
    P.conic[0] = P.c * idet;
    P.conic[1] = -P.b * idet;
    P.conic[2] = P.a * idet;
    P.u = vp.fx * P.pc[0] * iz + vp.cx;
    P.v = vp.fy * P.pc[1] * iz + vp.cy;
    const float mid = 0.5f * (P.a + P.c);
    const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - P.det));
    const float rr = ceilf(rc.radius_sigma * sqrtf(lam));
    P.radius = rr < (float)kMaxRadius ? (int)rr : kMaxRadius;
    if (P.radius <= 0) return;
    // Covered tiles from the fp32 centre.  With r an integer and the tile a
    // power of two, floor((m - r) / t) = (floor(m) - r) >> log2(t) exactly, so the
    // rectangle needs only integer arithmetic (centres are clamped to +-2^29,
    // far outside any grid, before the conversion).
    const int sh = rc.tile == 8 ? 3 : (rc.tile == 16 ? 4 : 5);
    const int ix = (int)floorf(fminf(fmaxf(P.u, -536870912.f), 536870912.f));
    const int iy = (int)floorf(fminf(fmaxf(P.v, -536870912.f), 536870912.f));
    const int x0 = max((ix - P.radius) >> sh, 0), x1 = min(((ix + P.radius) >> sh) + 1, vp.tiles_x);
    const int y0 = max((iy - P.radius) >> sh, 0), y1 = min(((iy + P.radius) >> sh) + 1, vp.tiles_y);
    if (x1 <= x0 || y1 <= y0) return;
    P.rect[0] = x0; P.rect[1] = y0; P.rect[2] = x1; P.rect[3] = y1;
    P.tiles = (P.rect[2] - P.rect[0]) * (P.rect[3] - P.rect[1]);
    P.visible = true;
}

__device__ __forceinline__ void view_colour(const gs_gaussians& g, int i, const Activated& A, const ViewParams& vp,
                                            int sh_degree, float* rgb, float* raw, float* dir, float* dist) {
    if (sh_degree == 0) {
        rgb[0] = raw[0] = g.color[3 * i];
        rgb[1] = raw[1] = g.color[3 * i + 1];
        rgb[2] = raw[2] = g.color[3 * i + 2];
        return;
    }
    float d0 = A.mu[0] - vp.centre[0], d1 = A.mu[1] - vp.centre[1], d2 = A.mu[2] - vp.centre[2];
    float dd = sqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    float inv = 1.0f / dd;
    dir[0] = d0 * inv; dir[1] = d1 * inv; dir[2] = d2 * inv;
    *dist = dd;
    float Y[16];
    sh_eval(dir[0], dir[1], dir[2], Y);
    const float* c = g.color + 48 * (size_t)i;
    float r0 = 0.5f, r1 = 0.5f, r2 = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; k++) {
        r0 += c[3 * k] * Y[k];
        r1 += c[3 * k + 1] * Y[k];
        r2 += c[3 * k + 2] * Y[k];
    }
    raw[0] = r0; raw[1] = r1; raw[2] = r2;
    rgb[0] = fmaxf(r0, 0.f); rgb[1] = fmaxf(r1, 0.f); rgb[2] = fmaxf(r2, 0.f);
}

// The views as this CTA uses them, in shared memory: the per-view constants,
// each pose moved to Exp(xi_v) T_cw on the device when a tangent xi ([n_views][6],
// (rho, phi)) is given: R <- Exp(phi) R (Rodrigues), t <- Exp(phi) t + rho (the
// translation to first order), camera centre -R^T t.  The pose gradient of the
// backward then refers to a further left perturbation of the moved pose.
__device__ __forceinline__ void views_to_shared(const Views& views, const float* __restrict__ xi, ViewParams* s_vp) {
    constexpr int kWords = sizeof(ViewParams) / sizeof(uint32_t);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(views.v);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_vp);
    for (int k = threadIdx.x; k < views.n * kWords; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    if (xi != nullptr && (int)threadIdx.x < views.n) {
        ViewParams& vp = s_vp[threadIdx.x];
        const float* x = xi + 6 * threadIdx.x;
        const float p0 = x[3], p1 = x[4], p2 = x[5];
        const float th2 = p0 * p0 + p1 * p1 + p2 * p2, th = sqrtf(th2);
        // Exp(phi) = I + a K + b K^2, K = [phi]x; a = sin th / th, b = (1 - cos th) / th^2
        const float a = th < 1e-4f ? 1.f - th2 / 6.f : sinf(th) / th;
        const float b = th < 1e-4f ? 0.5f - th2 / 24.f : (1.f - cosf(th)) / th2;
        const float K[9] = {0.f, -p2, p1, p2, 0.f, -p0, -p1, p0, 0.f};
        float E[9];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const float kk = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
                E[3 * r + c] = (r == c ? 1.f : 0.f) + a * K[3 * r + c] + b * kk;
            }
        float R[9], t[3];
#pragma unroll
        for (int r = 0; r < 3; r++) {
#pragma unroll
            for (int c = 0; c < 3; c++)
                R[3 * r + c] = E[3 * r] * vp.Rcw[c] + E[3 * r + 1] * vp.Rcw[3 + c] + E[3 * r + 2] * vp.Rcw[6 + c];
            t[r] = E[3 * r] * vp.tcw[0] + E[3 * r + 1] * vp.tcw[1] + E[3 * r + 2] * vp.tcw[2] + x[r];
        }
#pragma unroll
        for (int k = 0; k < 9; k++) vp.Rcw[k] = R[k];
#pragma unroll
        for (int r = 0; r < 3; r++) {
            vp.tcw[r] = t[r];
            vp.centre[r] = -(R[r] * t[0] + R[3 + r] * t[1] + R[6 + r] * t[2]);
        }
    }
    __syncthreads();
}

template <int SH>
__global__ void __launch_bounds__(kProjThreads) k_project(gs_gaussians g, Views views, RenderConsts rc,
                                                          gs_projected out, const float* __restrict__ xi) {
    __shared__ ViewParams s_vp[GS_MAX_VIEWS];
    pdl_enter();
    views_to_shared(views, xi, s_vp);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = (int)g.n;
    if (i >= n) return;
    Activated A;
    activate(g, i, A);
    for (int v = 0; v < views.n; v++) {
        const ViewParams& vp = s_vp[v];
        const size_t e = (size_t)v * n + i;
        ViewProj P;
        project_view(A, vp, rc, P);
        if (!P.visible) {
            reinterpret_cast<float2*>(out.xy)[e] = make_float2(0.f, 0.f);
            reinterpret_cast<float4*>(out.conic_o)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4*>(out.rgbd)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<int4*>(out.rect)[e] = make_int4(0, 0, 0, 0);
            out.radius[e] = 0;
            out.tiles_touched[e] = 0u;
            continue;
        }
        float rgb[3], raw[3], dir[3], dist;
        view_colour(g, i, A, vp, SH, rgb, raw, dir, &dist);
        reinterpret_cast<float2*>(out.xy)[e] = make_float2(P.u, P.v);
        reinterpret_cast<float4*>(out.conic_o)[e] = make_float4(P.conic[0], P.conic[1], P.conic[2], A.o);
        reinterpret_cast<float4*>(out.rgbd)[e] = make_float4(rgb[0], rgb[1], rgb[2], P.pc[2]);
        reinterpret_cast<int4*>(out.rect)[e] = make_int4(P.rect[0], P.rect[1], P.rect[2], P.rect[3]);
        out.radius[e] = P.radius;
        out.tiles_touched[e] = (uint32_t)P.tiles;
    }
}

// ------------------------------------------------------------------ backward

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Chain rule from the per-entry gradients of (xy, conic, opacity, rgb, z),
// summed over views, to mean, quaternion, log-scale, logit and colour; per-view
// pose tangent (rho, phi) of T_cw <- Exp(xi) T_cw; plus the isotropic
// regulariser on the scales.
template <int SH>
__global__ void __launch_bounds__(kProjThreads, SH == 0 ? 3 : 1) k_project_bwd(gs_gaussians g, Views views,
                                                                               RenderConsts rc,
                                                              const float* __restrict__ g2d, float lambda_iso,
                                                              float inv_n, gs_grads grads, float* iso_loss,
                                                              const float* __restrict__ xi) {
    __shared__ ViewParams s_vp[GS_MAX_VIEWS];
    pdl_enter();
    views_to_shared(views, xi, s_vp);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = (int)g.n;
    const bool active = i < n;
    __shared__ float s_red[kProjThreads / 32][7];
    Activated A;
    if (active) activate(g, i, A);
    float G_mu[3] = {0.f, 0.f, 0.f};
    float G_S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // symmetric world-covariance gradient (xx, xy, xz, yy, yz, zz)
    float G_o = 0.f;
    float G_rgb[3] = {0.f, 0.f, 0.f};
    float G_sh[SH == 0 ? 1 : 48];
    if constexpr (SH != 0) {
#pragma unroll
        for (int k = 0; k < 48; k++) G_sh[k] = 0.f;
    }
    for (int v = 0; v < views.n; v++) {
        const ViewParams& vp = s_vp[v];
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        ViewProj P;
        P.visible = false;
        if (active) project_view(A, vp, rc, P);
        if (P.visible) {
            const size_t e = (size_t)v * n + i;
            const float4 ga = reinterpret_cast<const float4*>(g2d)[3 * e];      // gx, gy, gA, gB
            const float4 gb = reinterpret_cast<const float4*>(g2d)[3 * e + 1];  // gC, go, gz, -
            const float4 gc = reinterpret_cast<const float4*>(g2d)[3 * e + 2];  // gr, gg, gb, -
            // conic = (c, -b, a) / det
            const float a = P.a, b = P.b, c = P.c;
            const float id = 1.0f / P.det, id2 = id * id;
            const float gA = ga.z, gB = ga.w, gC = gb.x;
            const float Ga = (-c * c * gA + b * c * gB - b * b * gC) * id2;
            const float Gb = (2.f * b * c * gA - (P.det + 2.f * b * b) * gB + 2.f * a * b * gC) * id2;
            const float Gc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
            const float g00 = Ga, g01 = 0.5f * Gb, g11 = Gc;   // symmetric 2x2
            // Sigma_2 = T Sigma T^T: G_Sigma += T^T G2 T ; G_T = 2 G2 T Sigma
            const float* T = P.T;
            const float* S = A.S;
            float GT2[6];    // G2 T  (2x3)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                GT2[k] = g00 * T[k] + g01 * T[3 + k];
                GT2[3 + k] = g01 * T[k] + g11 * T[3 + k];
            }
            G_S[0] += T[0] * GT2[0] + T[3] * GT2[3];
            G_S[1] += T[0] * GT2[1] + T[3] * GT2[4];
            G_S[2] += T[0] * GT2[2] + T[3] * GT2[5];
            G_S[3] += T[1] * GT2[1] + T[4] * GT2[4];
            G_S[4] += T[1] * GT2[2] + T[4] * GT2[5];
            G_S[5] += T[2] * GT2[2] + T[5] * GT2[5];
            float GT[6];     // 2 G2 T Sigma
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const float x0 = GT2[3 * r], x1 = GT2[3 * r + 1], x2 = GT2[3 * r + 2];
                GT[3 * r] = 2.f * (x0 * S[0] + x1 * S[1] + x2 * S[2]);
                GT[3 * r + 1] = 2.f * (x0 * S[1] + x1 * S[3] + x2 * S[4]);
                GT[3 * r + 2] = 2.f * (x0 * S[2] + x1 * S[4] + x2 * S[5]);
            }
            // T = J W: G_J = G_T W^T, G_W = J^T G_T
            const float* W = vp.Rcw;
            float GJ[6];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    GJ[3 * r + k] = GT[3 * r] * W[3 * k] + GT[3 * r + 1] * W[3 * k + 1] + GT[3 * r + 2] * W[3 * k + 2];
            const float iz = P.inv_z, iz2 = iz * iz, iz3 = iz2 * iz;
            const float x = P.pc[0], y = P.pc[1];
            const float fx = vp.fx, fy = vp.fy;
            const float j00 = fx * iz, j02 = -fx * x * iz2, j11 = fy * iz, j12 = -fy * y * iz2;
            float GW[9];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                GW[k] = j00 * GT[k];
                GW[3 + k] = j11 * GT[3 + k];
                GW[6 + k] = j02 * GT[k] + j12 * GT[3 + k];
            }
            const float gu = ga.x, gv = ga.y;
            float Gp[3];
            Gp[0] = gu * fx * iz - GJ[2] * fx * iz2;
            Gp[1] = gv * fy * iz - GJ[5] * fy * iz2;
            Gp[2] = -gu * fx * x * iz2 - gv * fy * y * iz2 + gb.z - GJ[0] * fx * iz2 + GJ[2] * 2.f * fx * x * iz3 -
                    GJ[4] * fy * iz2 + GJ[5] * 2.f * fy * y * iz3;
            // colour
            float gcen[3] = {0.f, 0.f, 0.f};
            if constexpr (SH == 0) {
                G_rgb[0] += gc.x; G_rgb[1] += gc.y; G_rgb[2] += gc.z;
            } else {
                float rgb[3], raw[3], dir[3], dist;
                view_colour(g, i, A, vp, SH, rgb, raw, dir, &dist);
                const float gr0 = raw[0] < 0.f ? 0.f : gc.x;
                const float gr1 = raw[1] < 0.f ? 0.f : gc.y;
                const float gr2 = raw[2] < 0.f ? 0.f : gc.z;
                float Y[16], wsum[16];
                sh_eval(dir[0], dir[1], dir[2], Y);
                const float* cf = g.color + 48 * (size_t)i;
#pragma unroll
                for (int k = 0; k < 16; k++) {
                    G_sh[3 * k] += gr0 * Y[k];
                    G_sh[3 * k + 1] += gr1 * Y[k];
                    G_sh[3 * k + 2] += gr2 * Y[k];
                    wsum[k] = gr0 * cf[3 * k] + gr1 * cf[3 * k + 1] + gr2 * cf[3 * k + 2];
                }
                float gd[3];
                sh_grad(dir[0], dir[1], dir[2], wsum, gd);
                const float dot = dir[0] * gd[0] + dir[1] * gd[1] + dir[2] * gd[2];
                const float idist = 1.0f / dist;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float gvk = (gd[k] - dir[k] * dot) * idist;
                    G_mu[k] += gvk;
                    gcen[k] = -gvk;
                }
            }
            G_o += gb.y;
            // mean: p_c = W mu + t
#pragma unroll
            for (int k = 0; k < 3; k++) G_mu[k] += W[k] * Gp[0] + W[3 + k] * Gp[1] + W[6 + k] * Gp[2];
            // pose: rho moves p_c (and the camera centre by -W^T rho); phi rotates p_c and W
            const float* pc = P.pc;
            float GWWt[9];   // G_W W^T
#pragma unroll
            for (int r = 0; r < 3; r++)
#pragma unroll
                for (int k = 0; k < 3; k++)
                    GWWt[3 * r + k] = GW[3 * r] * W[3 * k] + GW[3 * r + 1] * W[3 * k + 1] + GW[3 * r + 2] * W[3 * k + 2];
#pragma unroll
            for (int k = 0; k < 3; k++)
                pose[k] = Gp[k] - (W[3 * k] * gcen[0] + W[3 * k + 1] * gcen[1] + W[3 * k + 2] * gcen[2]);
            pose[3] = pc[1] * Gp[2] - pc[2] * Gp[1] + (GWWt[7] - GWWt[5]);
            pose[4] = pc[2] * Gp[0] - pc[0] * Gp[2] + (GWWt[2] - GWWt[6]);
            pose[5] = pc[0] * Gp[1] - pc[1] * Gp[0] + (GWWt[3] - GWWt[1]);
        }
        if (grads.pose != nullptr) {
            // block reduction of the 6 pose components, one atomic per component per block
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const float s = warp_sum(pose[k]);
                if (lane == 0) s_red[warp][k] = s;
            }
            __syncthreads();
            if (threadIdx.x < 6) {
                float s = 0.f;
#pragma unroll
                for (int w = 0; w < kProjThreads / 32; w++) s += s_red[w][threadIdx.x];
                atomicAdd(grads.pose + 6 * v + threadIdx.x, s);
            }
            __syncthreads();
        }
    }
    float iso_part = 0.f;
    if (active) {
        // Sigma = M M^T: G_M = 2 G_Sigma M (G_Sigma symmetric, stored as 6 unique entries)
        const float Gs[9] = {G_S[0], G_S[1], G_S[2], G_S[1], G_S[3], G_S[4], G_S[2], G_S[4], G_S[5]};
        float GM[9];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int j = 0; j < 3; j++)
                GM[3 * r + j] = 2.f * (Gs[3 * r] * A.M[j] + Gs[3 * r + 1] * A.M[3 + j] + Gs[3 * r + 2] * A.M[6 + j]);
        float Gls[3];
#pragma unroll
        for (int j = 0; j < 3; j++)
            Gls[j] = (GM[j] * A.R[j] + GM[3 + j] * A.R[3 + j] + GM[6 + j] * A.R[6 + j]) * A.s[j];
        if (lambda_iso != 0.f || iso_loss != nullptr) {
            const float m = (A.s[0] + A.s[1] + A.s[2]) * (1.0f / 3.0f);
            float sg[3];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const float r = A.s[j] - m;
                iso_part += fabsf(r);
                sg[j] = (r > 0.f) ? 1.f : ((r < 0.f) ? -1.f : 0.f);
            }
            const float ssum = (sg[0] + sg[1] + sg[2]) * (1.0f / 3.0f);
#pragma unroll
            for (int j = 0; j < 3; j++) Gls[j] += lambda_iso * inv_n * (sg[j] - ssum) * A.s[j];
        }
        float GR[9];
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int j = 0; j < 3; j++) GR[3 * r + j] = GM[3 * r + j] * A.s[j];
        const float w = A.q[0], x = A.q[1], y = A.q[2], z = A.q[3];
        float gq[4];
        gq[0] = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
        gq[1] = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] + w * GR[7] -
                       2.f * x * GR[8]);
        gq[2] = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] + z * GR[7] -
                       2.f * y * GR[8]);
        gq[3] = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] + y * GR[5] +
                       x * GR[6] + y * GR[7]);
        const float dot = w * gq[0] + x * gq[1] + y * gq[2] + z * gq[3];
        const float iq = 1.0f / A.qnorm;
        reinterpret_cast<float4*>(grads.quat)[i] =
            make_float4((gq[0] - w * dot) * iq, (gq[1] - x * dot) * iq, (gq[2] - y * dot) * iq, (gq[3] - z * dot) * iq);
        grads.mean[3 * i] = G_mu[0];
        grads.mean[3 * i + 1] = G_mu[1];
        grads.mean[3 * i + 2] = G_mu[2];
        grads.log_scale[3 * i] = Gls[0];
        grads.log_scale[3 * i + 1] = Gls[1];
        grads.log_scale[3 * i + 2] = Gls[2];
        grads.opacity_logit[i] = G_o * A.o * (1.f - A.o);
        if constexpr (SH == 0) {
            grads.color[3 * i] = G_rgb[0];
            grads.color[3 * i + 1] = G_rgb[1];
            grads.color[3 * i + 2] = G_rgb[2];
        } else {
#pragma unroll
            for (int k = 0; k < 48; k++) grads.color[48 * (size_t)i + k] = G_sh[k];
        }
    }
    if (iso_loss != nullptr) {
        const float s = warp_sum(iso_part);
        if ((threadIdx.x & 31) == 0) atomicAdd(iso_loss, s * inv_n);
    }
}

}  // namespace

cudaError_t launch_project(const gs_gaussians& g, const Views& views, const RenderConsts& rc,
                           const gs_projected& out, cudaStream_t s, const float* xi) {
    if (g.n == 0) return cudaSuccess;
    const int blocks = (int)ceil_div(g.n, kProjThreads);
    const cudaError_t e = rc.sh_degree == 0 ? launch_pdl(k_project<0>, blocks, kProjThreads, 0, s, g, views, rc, out, xi)
                                            : launch_pdl(k_project<3>, blocks, kProjThreads, 0, s, g, views, rc, out, xi);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const gs_gaussians& g, const Views& views, const RenderConsts& rc,
                               const float* g2d, float lambda_iso, const gs_grads& grads, float* iso_loss,
                               cudaStream_t s, const float* xi) {
    if (g.n == 0) return cudaSuccess;
    const int blocks = (int)ceil_div(g.n, kProjThreads);
    const float inv_n = 1.0f / (float)g.n;
    const cudaError_t e =
        rc.sh_degree == 0
            ? launch_pdl(k_project_bwd<0>, blocks, kProjThreads, 0, s, g, views, rc, g2d, lambda_iso, inv_n, grads,
                         iso_loss, xi)
            : launch_pdl(k_project_bwd<3>, blocks, kProjThreads, 0, s, g, views, rc, g2d, lambda_iso, inv_n, grads,
                         iso_loss, xi);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gs
