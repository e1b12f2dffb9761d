// insert.cu -- keyframe insertion of new Gaussians (Sec. 3.3 "Map Management":
// a new keyframe's pixels are back-projected with their depth into new
// Gaussians whose opacity starts at 0.5) and the 7 x 7 RGB-D patches that the
// learned initialiser reads.
//
// Heuristic initialisation of a Gaussian at pixel (u, v) with depth d > 0:
//   mean       = R_wc (((u + 0.5 - cx) / fx) d, ((v + 0.5 - cy) / fy) d, d) + t_wc
//   log_scale  = log(d * stride / f),  f = (fx + fy) / 2, on all three axes
//                (the footprint of one sample of a grid with `stride` px spacing)
//   quaternion = (1, 0, 0, 0);  opacity logit = 0 (opacity 0.5);  colour = pixel RGB
// With network outputs y (gs_mlp_fwd): log_scale = heuristic + y[0..2], the
// rotation is the camera-to-world rotation composed with the camera-frame
// quaternion y[3..6] (normalised), and the opacity logit is y[7].
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr float kSH0 = 0.28209479177387814f;     // Y_0^0 = 1 / (2 sqrt(pi))

__device__ __forceinline__ uint16_t f2bf16(float x) {
    // round to nearest even (finite inputs)
    const uint32_t u = __float_as_uint(x);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

struct Cam {
    float fx, fy, cx, cy;
    int W, H;
    float R[9], t[3];
};

__device__ __forceinline__ bool sample_pixel(const int32_t* uv, int64_t k, const Cam& c, int* u, int* v) {
    *u = uv[2 * k];
    *v = uv[2 * k + 1];
    return *u >= 0 && *u < c.W && *v >= 0 && *v < c.H;
}

__global__ void k_extract_patches(const float* __restrict__ color, const float* __restrict__ depth, Cam c,
                                  const int32_t* __restrict__ uv, int64_t n, uint16_t* __restrict__ X,
                                  int* status) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    int u, v;
    uint16_t* row = X + k * GS_MLP_IN_STRIDE;
    if (!sample_pixel(uv, k, c, &u, &v)) {
        if (status) atomicCAS(status, 0, GS_ERR_INVALID_ARG);
        for (int i = 0; i < GS_MLP_IN_STRIDE; i++) row[i] = 0;
        return;
    }
    const int HW = c.W * c.H;
    const float fbar = 0.5f * (c.fx + c.fy);
    const float dc = depth[v * c.W + u];
    const float dscale = dc > 0.f ? fbar / (7.f * dc) : 0.f;
    uint32_t packed[GS_MLP_IN_STRIDE / 2];
    for (int p = 0; p < 49; p++) {
        const int x = min(max(u + p % 7 - 3, 0), c.W - 1), y = min(max(v + p / 7 - 3, 0), c.H - 1);
        const int pix = y * c.W + x;
        const float d = depth[pix];
        float dz;
        if (p == 24) dz = dc > 0.f ? logf(dc) : 0.f;
        else dz = (d > 0.f && dc > 0.f) ? (d - dc) * dscale : 0.f;
        packed[2 * p] = (uint32_t)f2bf16(color[pix]) | ((uint32_t)f2bf16(color[HW + pix]) << 16);
        packed[2 * p + 1] = (uint32_t)f2bf16(color[2 * HW + pix]) | ((uint32_t)f2bf16(dz) << 16);
    }
    packed[98] = 0x3F80u;     // column 196: the bias input 1, 197..207: 0
    for (int i = 99; i < GS_MLP_IN_STRIDE / 2; i++) packed[i] = 0u;
    uint4* out = reinterpret_cast<uint4*>(row);
    for (int i = 0; i < GS_MLP_IN_STRIDE / 8; i++)
        out[i] = make_uint4(packed[4 * i], packed[4 * i + 1], packed[4 * i + 2], packed[4 * i + 3]);
}

__global__ void k_insert(const float* __restrict__ color, const float* __restrict__ depth, Cam c,
                         const int32_t* __restrict__ uv, int64_t n, float stride, const float* __restrict__ Y,
                         gs_map_slots dst, int64_t offset, int sh_degree, int* status) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = offset + k;
    const int ncol = sh_degree == 3 ? 48 : 3;
    int u, v;
    const bool inside = sample_pixel(uv, k, c, &u, &v);
    if (!inside && status) atomicCAS(status, 0, GS_ERR_INVALID_ARG);
    const float d = inside ? depth[v * c.W + u] : 0.f;
    float* col = dst.color + i * ncol;
    for (int j = 0; j < ncol; j++) col[j] = 0.f;
    if (!(d > 0.f)) {
        // no depth: an inert Gaussian (transparent, tiny) at the camera centre
        for (int a = 0; a < 3; a++) { dst.mean[3 * i + a] = c.t[a]; dst.log_scale[3 * i + a] = -10.f; }
        dst.quat[4 * i] = 1.f; dst.quat[4 * i + 1] = dst.quat[4 * i + 2] = dst.quat[4 * i + 3] = 0.f;
        dst.opacity_logit[i] = -30.f;
        return;
    }
    const float xc = ((float)u + 0.5f - c.cx) / c.fx * d, yc = ((float)v + 0.5f - c.cy) / c.fy * d;
    for (int a = 0; a < 3; a++)
        dst.mean[3 * i + a] = c.R[3 * a] * xc + c.R[3 * a + 1] * yc + c.R[3 * a + 2] * d + c.t[a];
    const float s0 = logf(d * stride / (0.5f * (c.fx + c.fy)));
    const int HW = c.W * c.H, pix = v * c.W + u;
    const float rgb[3] = {color[pix], color[HW + pix], color[2 * HW + pix]};
    for (int a = 0; a < 3; a++) col[a] = sh_degree == 3 ? (rgb[a] - 0.5f) / kSH0 : rgb[a];
    float q[4] = {1.f, 0.f, 0.f, 0.f}, ls[3] = {s0, s0, s0}, logit = 0.f;
    if (Y != nullptr) {
        const float* y = Y + k * GS_MLP_OUT;
        for (int a = 0; a < 3; a++) ls[a] = s0 + y[a];
        const float nq = sqrtf(y[3] * y[3] + y[4] * y[4] + y[5] * y[5] + y[6] * y[6]);
        if (nq > 1e-12f) {
            const float qc[4] = {y[3] / nq, y[4] / nq, y[5] / nq, y[6] / nq};
            float qwc[4];
            rot_to_quat(c.R, qwc);
            quat_mul(qwc, qc, q);
        }
        logit = y[7];
    }
    for (int a = 0; a < 3; a++) dst.log_scale[3 * i + a] = ls[a];
    for (int a = 0; a < 4; a++) dst.quat[4 * i + a] = q[a];
    dst.opacity_logit[i] = logit;
}

Cam to_cam(const gs_camera& g) {
    Cam c;
    c.fx = g.fx; c.fy = g.fy; c.cx = g.cx; c.cy = g.cy; c.W = g.width; c.H = g.height;
    for (int i = 0; i < 9; i++) c.R[i] = g.R_wc[i];
    for (int i = 0; i < 3; i++) c.t[i] = g.t_wc[i];
    return c;
}

}  // namespace

cudaError_t launch_extract_patches(const float* color, const float* depth, const gs_camera& cam,
                                   const int32_t* uv, int64_t n, uint16_t* X, int* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_extract_patches<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(color, depth, to_cam(cam), uv, n, X, status);
    return cudaGetLastError();
}

cudaError_t launch_insert(const float* color, const float* depth, const gs_camera& cam, const int32_t* uv,
                          int64_t n, float stride, const float* Y, const gs_map_slots& dst, int64_t offset,
                          int sh_degree, int* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_insert<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(color, depth, to_cam(cam), uv, n, stride, Y, dst, offset,
                                                         sh_degree, status);
    return cudaGetLastError();
}

}  // namespace gs
