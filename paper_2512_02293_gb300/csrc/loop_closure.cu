// loop_closure.cu -- the loop-closure Gaussian update (Sec. 3.3 "Loop Closure
// Gaussian Update", Eq. 7 and Eq. 8): after pose-graph bundle adjustment moves
// keyframe k from (R_k^-, t_k^-) to (R_k^+, t_k^+) with scale change ds_k, each
// Gaussian anchored to k follows it, so the map stays consistent without
// re-optimising it:
//   mean:        mu+ = R_k^+ (ds_k (R_k^-)^T (mu- - t_k^-)) + t_k^+              (Eq. 7)
//   covariance:  Sigma+ = R_k^+ (ds_k^2 (R_k^-)^T Sigma- R_k^-) (R_k^+)^T        (Eq. 8)
// With Sigma = R(q) S^2 R(q)^T this is q+ = q(R_k^+ (R_k^-)^T) * q and
// log s+ = log s + log ds_k; opacity and colour are unchanged.
// One thread per Gaussian, in place; 84 bytes moved per Gaussian (HBM bound).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kLcThreads = 256;

__global__ void __launch_bounds__(kLcThreads) k_loop_closure(gs_map_slots map, const int32_t* __restrict__ anchor,
                                                              const float* __restrict__ before,
                                                              const float* __restrict__ after,
                                                              const float* __restrict__ ds, int K, int* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= map.capacity) return;
    const int k = anchor[i];
    if (k < 0 || k >= K || !(ds[k] > 0.f)) {          // bad anchor or scale: leave the Gaussian as it is
        if (status) atomicCAS(status, 0, GS_ERR_INVALID_ARG);
        return;
    }
    const float* pm = before + 12 * k;                 // R^- row-major, t^-
    const float* pp = after + 12 * k;                  // R^+ row-major, t^+
    float Rm[9], Rp[9], tm[3], tp[3];
#pragma unroll
    for (int j = 0; j < 9; j++) { Rm[j] = __ldg(pm + j); Rp[j] = __ldg(pp + j); }
#pragma unroll
    for (int j = 0; j < 3; j++) { tm[j] = __ldg(pm + 9 + j); tp[j] = __ldg(pp + 9 + j); }
    const float s = __ldg(ds + k);
    // Eq. 7: into the old keyframe frame, scale, out of the new one
    float d[3], x[3];
#pragma unroll
    for (int a = 0; a < 3; a++) d[a] = map.mean[3 * i + a] - tm[a];
#pragma unroll
    for (int a = 0; a < 3; a++) x[a] = s * (Rm[a] * d[0] + Rm[3 + a] * d[1] + Rm[6 + a] * d[2]);
#pragma unroll
    for (int a = 0; a < 3; a++)
        map.mean[3 * i + a] = Rp[3 * a] * x[0] + Rp[3 * a + 1] * x[1] + Rp[3 * a + 2] * x[2] + tp[a];
    // Eq. 8: rotate by R^+ (R^-)^T, scale the axes by ds
    float A[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
            A[3 * r + c] = Rp[3 * r] * Rm[3 * c] + Rp[3 * r + 1] * Rm[3 * c + 1] + Rp[3 * r + 2] * Rm[3 * c + 2];
    float qa[4], q[4], qn[4];
    rot_to_quat(A, qa);
    const float4 q4 = reinterpret_cast<const float4*>(map.quat)[i];
    q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
    quat_mul(qa, q, qn);
    reinterpret_cast<float4*>(map.quat)[i] = make_float4(qn[0], qn[1], qn[2], qn[3]);
    const float ls = logf(s);
#pragma unroll
    for (int a = 0; a < 3; a++) map.log_scale[3 * i + a] += ls;
}

}  // namespace

cudaError_t launch_loop_closure(const gs_map_slots& map, const int32_t* anchor, const float* before,
                                const float* after, const float* ds, int K, int* status, cudaStream_t s) {
    if (map.capacity == 0) return cudaSuccess;
    k_loop_closure<<<(unsigned)((map.capacity + kLcThreads - 1) / kLcThreads), kLcThreads, 0, s>>>(map, anchor, before, after, ds, K, status);
    return cudaGetLastError();
}

}  // namespace gs
