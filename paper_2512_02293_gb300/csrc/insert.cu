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

// One warp per sample: lane l forms window pixels l and l + 32 (8 bytes each: the
// BF16 R, G, B and depth slot), so a row is written as contiguous 8-byte pieces;
// pieces 49 .. 51 are the bias input and the padding.
constexpr int kPatchWarps = 8;

__global__ void __launch_bounds__(kPatchWarps * 32) k_extract_patches(
        const float* __restrict__ color, const float* __restrict__ depth, Cam c, const int32_t* __restrict__ uv,
        int64_t n, uint16_t* __restrict__ X, int* status) {
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * (int64_t)kPatchWarps + (threadIdx.x >> 5);
    if (k >= n) return;
    uint2* row = reinterpret_cast<uint2*>(X + k * GS_MLP_IN_STRIDE);
    constexpr int kPieces = GS_MLP_IN_STRIDE / 4;     // 52
    int u, v;
    if (!sample_pixel(uv, k, c, &u, &v)) {
        if (status && lane == 0) atomicCAS(status, 0, GS_ERR_INVALID_ARG);
        for (int q = lane; q < kPieces; q += 32) row[q] = make_uint2(0u, 0u);
        return;
    }
    const int HW = c.W * c.H;
    const float fbar = 0.5f * (c.fx + c.fy);
    const float dc = depth[v * c.W + u];
    const float dscale = dc > 0.f ? fbar / (7.f * dc) : 0.f;
    for (int q = lane; q < kPieces; q += 32) {
        uint2 piece;
        if (q < 49) {
            const int x = min(max(u + q % 7 - 3, 0), c.W - 1), y = min(max(v + q / 7 - 3, 0), c.H - 1);
            const int pix = y * c.W + x;
            const float d = depth[pix];
            float dz;
            if (q == 24) dz = dc > 0.f ? logf(dc) : 0.f;
            else dz = (d > 0.f && dc > 0.f) ? (d - dc) * dscale : 0.f;
            piece.x = (uint32_t)f2bf16(color[pix]) | ((uint32_t)f2bf16(color[HW + pix]) << 16);
            piece.y = (uint32_t)f2bf16(color[2 * HW + pix]) | ((uint32_t)f2bf16(dz) << 16);
        } else {
            piece = make_uint2(q == 49 ? 0x3F80u : 0u, 0u);   // column 196: the bias input 1; 197 .. 207: 0
        }
        row[q] = piece;
    }
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
    if (!(d > 0.f)) {
        for (int j = 0; j < ncol; j++) col[j] = 0.f;
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
    for (int j = 3; j < ncol; j++) col[j] = 0.f;
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
    k_extract_patches<<<(unsigned)((n + kPatchWarps - 1) / kPatchWarps), kPatchWarps * 32, 0, s>>>(
        color, depth, to_cam(cam), uv, n, X, status);
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
