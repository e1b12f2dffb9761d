// mlp.cu -- the learned initialiser of newly inserted Gaussians: a perceptron
// 196 -> 128 -> 128 -> 8 with GELU over a 7 x 7 RGB-D keyframe patch, predicting
// the log-scale offsets, camera-frame rotation and opacity logit of the Gaussian
// inserted at the patch centre (the keyframe insertion of Sec. 3.3 "Map
// Management" gives only the opacity; the network replaces the heuristic for
// the rest).  BF16 weights, inputs and layer-to-layer activations, FP32
// accumulation in tensor memory, on the fifth-generation tensor cores.
//
// Biases ride in the GEMMs: each layer's input has one extra column of ones
// (input column 196, hidden column 128) and each packed weight matrix carries
// its bias in that column, so W [rows][K] times the augmented input gives
// W x + b, and the weight gradient's extra column is the bias gradient.
//
//   layer 1:  Z1 = X_aug  W1a^T   M 128 (samples)  N 128  K 208 (196 + ones + 11 zero)
//   layer 2:  Z2 = H1_aug W2a^T   M 128            N 128  K 144 (128 + ones + 15 zero)
//   layer 3:  Y  = H2_aug W3a^T   M 128            N 16   K 144 (8 outputs + 8 zero rows)
//   backward: dH1 = dZ2 W2 (B = W2^T), dW2a += dZ2^T H1_aug, dW1a += dZ1^T X_aug,
//             dW3 / db3 and dH2 = dY W3 on the CUDA cores (8 outputs).
//
// One CTA of 512 threads per SM walks tiles of 128 samples; the four threads of
// sample row r (tensor-memory lane r of every accumulator) split its columns.
#include <cuda_bf16.h>

#include <atomic>

#include "gs_internal.cuh"
#include "tc.cuh"

namespace gs {
namespace {

constexpr int kIn = 196, kK1 = 208, kHid = 128, kK2 = 144, kOut = 8, kN3 = 16;
constexpr int kTile = 128;
// Both kernels run 16 warps: warp w reaches tensor-memory lanes 32 (w % 4) ..
// 32 (w % 4) + 31 (sample rows) and takes column group w / 4 of every epilogue.
constexpr int kFwdThreads = 512, kColGroups = kFwdThreads / 128;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kWaitPolls = GS_MLP_WAIT_POLLS_DEFAULT;   // mbarrier polls before GS_ERR_TIMEOUT (default)
constexpr uint32_t kDrainPolls = 1u << 26;    // bound of the wait for in-flight MMAs after a timeout

// Poll limit of the mbarrier waits of the next launches (gs_mlp_set_wait_polls).
std::atomic<uint32_t> g_wait_polls{kWaitPolls};

__device__ __forceinline__ uint16_t f2bf(float x) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&h);
}
__device__ __forceinline__ float bf2f(uint32_t u16) { return __uint_as_float(u16 << 16); }
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// d/dz z Phi(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status != nullptr) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------- weights
// FP32 master parameters -> the BF16 operands of the GEMMs (bias columns folded in).
__global__ void k_mlp_pack(gs_mlp_params p, gs_mlp_packed q) {
    const int n1 = kHid * kK1, n2 = kHid * kK2, n3 = kN3 * kK2, n4 = kHid * kHid;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3 + n4; i += gridDim.x * blockDim.x) {
        if (i < n1) {
            const int r = i / kK1, c = i % kK1;
            q.W1a[i] = f2bf(c < kIn ? p.W1[r * kIn + c] : (c == kIn ? p.b1[r] : 0.f));
        } else if (i < n1 + n2) {
            const int j = i - n1, r = j / kK2, c = j % kK2;
            q.W2a[j] = f2bf(c < kHid ? p.W2[r * kHid + c] : (c == kHid ? p.b2[r] : 0.f));
        } else if (i < n1 + n2 + n3) {
            const int j = i - n1 - n2, r = j / kK2, c = j % kK2;
            q.W3a[j] = f2bf(r < kOut ? (c < kHid ? p.W3[r * kHid + c] : (c == kHid ? p.b3[r] : 0.f)) : 0.f);
        } else {
            const int j = i - n1 - n2 - n3, r = j / kHid, c = j % kHid;     // W2t[r][c] = W2[c][r]
            q.W2t[j] = f2bf(p.W2[c * kHid + r]);
        }
    }
    // the activation and its derivative at every BF16 input
    for (int z = blockIdx.x * blockDim.x + threadIdx.x; z < 65536; z += gridDim.x * blockDim.x) {
        const float x = bf2f((uint32_t)z);
        q.gelu_tab[z] = f2bf(gelu(x));
        q.dgelu_tab[z] = gelu_grad(x);
    }
}

// Copy a row-major BF16 matrix [R][K] from global memory into the K-major
// core-matrix layout of tc.cuh (consecutive threads take consecutive rows, so
// each group of 8 threads writes 128 contiguous bytes).
__device__ __forceinline__ void fill_kmajor(uint8_t* dst, const uint16_t* __restrict__ src, int R, int K) {
    const int KB = K / 8;
    for (int q = threadIdx.x; q < R * KB; q += blockDim.x) {
        const int r = q % R, c = q / R;
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(src + (size_t)r * K) + c);
        *reinterpret_cast<uint4*>(dst + tc::kmajor_offset(r, c * 8, K)) = v;
    }
}

// Chunk c (8 values, columns 8c .. 8c+7) of sample row `row` of the input X,
// with the bias column set: columns >= 196 are 1 at 196 and 0 beyond, and rows
// past n are zero.
__device__ __forceinline__ uint4 x_chunk(const uint16_t* __restrict__ X, int64_t row, int64_t n, int c) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (row >= n) return v;
    if (c < kIn / 8) return __ldg(reinterpret_cast<const uint4*>(X + row * kK1) + c);
    if (c == kIn / 8) {   // columns 192..199: four inputs, the ones column, zeros
        const uint2 lo = __ldg(reinterpret_cast<const uint2*>(X + row * kK1 + 8 * c));
        v.x = lo.x; v.y = lo.y; v.z = 0x3F80u; v.w = 0u;   // bf16(1.0) at column 196
    }
    return v;
}

// ---------------------------------------------------------------- forward
// Shared-memory plan of the forward kernel (bytes): the three weight operands
// stay resident, X and H are the per-tile operands (H holds H1, then H2).
constexpr uint32_t kFwdW1 = 0;                                  // 128 x 208
constexpr uint32_t kFwdW2 = kFwdW1 + kHid * kK1 * 2;            // 128 x 144
constexpr uint32_t kFwdW3 = kFwdW2 + kHid * kK2 * 2;            // 16 x 144
constexpr uint32_t kFwdX = kFwdW3 + kN3 * kK2 * 2;              // 128 x 208
constexpr uint32_t kFwdH = kFwdX + kTile * kK1 * 2;             // 128 x 144
constexpr uint32_t kFwdBar = kFwdH + kTile * kK2 * 2;           // mbarrier (8 B) + tensor-memory base (4 B)
constexpr uint32_t kFwdSmem = kFwdBar + 16;

struct MlpFwdArgs {
    gs_mlp_packed w;
    const uint16_t* X;
    int64_t n;
    float* Y;            // [n][8] or null
    uint16_t* Z1;        // [n][128] pre-activations (training) or null
    uint16_t* Z2;
    const float* T;      // [n][8] targets (training) or null
    float* dY;           // [n][8] d loss / d Y, written when T is given
    float* loss;         // += loss_scale * sum (Y - T)^2, when T is given
    float loss_scale;
    int* status;
    uint32_t wait_polls; // mbarrier polls before a wait gives up
};

// Hidden-layer epilogue for this thread's sample row and columns [c_lo, c_hi):
// accumulator -> Z = bf16, H = bf16(gelu(Z)) into the next layer's K-major
// operand, Z to global memory.
__device__ __forceinline__ void hidden_epilogue(uint32_t tacc, uint8_t* sH, int r, int64_t row, int64_t n,
                                                uint16_t* __restrict__ Zout, int c_lo, int c_hi,
                                                const uint16_t* __restrict__ gtab) {
#pragma unroll 1
    for (int c0 = c_lo; c0 < c_hi; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tacc + (uint32_t)c0, v);
        uint32_t zp[8], hp[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const uint16_t z0 = f2bf(v[2 * i]), z1 = f2bf(v[2 * i + 1]);
            zp[i] = pack2(z0, z1);
            hp[i] = pack2(__ldg(gtab + z0), __ldg(gtab + z1));
        }
        *reinterpret_cast<uint4*>(sH + tc::kmajor_offset(r, c0, kK2)) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
        *reinterpret_cast<uint4*>(sH + tc::kmajor_offset(r, c0 + 8, kK2)) = make_uint4(hp[4], hp[5], hp[6], hp[7]);
        if (Zout != nullptr && row < n) {
            uint4* zrow = reinterpret_cast<uint4*>(Zout + row * kHid + c0);
            zrow[0] = make_uint4(zp[0], zp[1], zp[2], zp[3]);
            zrow[1] = make_uint4(zp[4], zp[5], zp[6], zp[7]);
        }
    }
}

// Issue the K loop of one GEMM (one thread) and commit it to the barrier.
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, uint32_t sa, uint32_t sb, int K, uint32_t idesc,
                                           bool accumulate, uint32_t bar) {
    tc::fence_after_sync();
    for (int s = 0; s < K / 16; s++)
        tc::mma_bf16(d_tmem, tc::kstep_desc(sa, K, s), tc::kstep_desc(sb, K, s), idesc, accumulate || s > 0);
    tc::mma_commit(bar);
}

// Every thread waits (at most `polls` polls) for the barrier phase; the outcome
// is made uniform.  If any thread gave up, the MMAs of that phase may still be
// running: thread 0 then waits for them (bounded again) before the CTA goes on
// to report the timeout and release its tensor memory, so nothing is freed
// under an MMA in flight.
__device__ __forceinline__ bool wait_all(uint32_t bar, uint32_t& phase, uint32_t polls) {
    const bool ok = tc::mbar_wait(bar, phase, polls);
    const bool all = __syncthreads_and(ok) != 0;
    if (!all) {
        if (threadIdx.x == 0) tc::mbar_wait(bar, phase, kDrainPolls);
        __syncthreads();
    }
    phase ^= 1u;
    tc::fence_after_sync();
    return all;
}

// Sync point after this thread wrote shared-memory operands: visible to the
// tensor core, prior tensor-memory reads ordered before the next MMA.
// 16-byte asynchronous copy global -> shared (zero-filled when !valid; src must
// then still be a readable address)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void operands_ready() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
}

__global__ void __launch_bounds__(kFwdThreads, 1) k_mlp_fwd(MlpFwdArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cg = warp >> 2;            // tensor-memory lane quarter, column group
    const int r = quarter * 32 + lane;                       // this thread's sample row in the tile
    uint8_t* sX = sm + kFwdX;
    uint8_t* sH = sm + kFwdH;
    const uint32_t bar = tc::smem_addr(sm + kFwdBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kFwdBar + 8);

    fill_kmajor(sm + kFwdW1, a.w.W1a, kHid, kK1);
    fill_kmajor(sm + kFwdW2, a.w.W2a, kHid, kK2);
    fill_kmajor(sm + kFwdW3, a.w.W3a, kN3, kK2);
    if (cg == 0) {   // constant augmentation of H: column 128 = 1, columns 129..143 = 0
        *reinterpret_cast<uint4*>(sH + tc::kmajor_offset(r, kHid, kK2)) = make_uint4(0x3F80u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sH + tc::kmajor_offset(r, kHid + 8, kK2)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) tc::mbar_init(bar, 1);
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), kTmemCols);
    operands_ready();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t tD1 = tbase, tD2 = tbase + 128, tD3 = tbase + 256;
    const uint32_t sa_x = tc::smem_addr(sX), sa_h = tc::smem_addr(sH);
    const uint32_t sa_w1 = tc::smem_addr(sm + kFwdW1), sa_w2 = tc::smem_addr(sm + kFwdW2);
    const uint32_t sa_w3 = tc::smem_addr(sm + kFwdW3);
    const int c_lo = cg * (kHid / kColGroups), c_hi = c_lo + kHid / kColGroups;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t n_tiles = (a.n + kTile - 1) / kTile;
    // the four threads of a sample row take every fourth 8-value chunk of its X row;
    // the next tile's chunks are loaded into registers while this tile computes
    constexpr int kXc = (kK1 / 8 + kColGroups - 1) / kColGroups;
    uint4 xn[kXc];
    auto load_x = [&](int64_t tile) {
#pragma unroll
        for (int q = 0; q < kXc; q++) {
            const int c = cg + q * kColGroups;
            xn[q] = c < kK1 / 8 ? x_chunk(a.X, tile * kTile + r, a.n, c) : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    if ((int64_t)blockIdx.x < n_tiles) load_x(blockIdx.x);
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t row0 = t * kTile, row = row0 + r;
#pragma unroll
        for (int q = 0; q < kXc; q++) {
            const int c = cg + q * kColGroups;
            if (c < kK1 / 8) *reinterpret_cast<uint4*>(sX + tc::kmajor_offset(r, 8 * c, kK1)) = xn[q];
        }
        operands_ready();
        if (tid == 0) issue_gemm(tD1, sa_x, sa_w1, kK1, tc::idesc_bf16(128, kHid), false, bar);
        if (t + gridDim.x < n_tiles) load_x(t + gridDim.x);     // in flight during the epilogues
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        hidden_epilogue(tD1 + lane_off, sH, r, row, a.n, a.Z1, c_lo, c_hi, a.w.gelu_tab);
        operands_ready();
        if (tid == 0) issue_gemm(tD2, sa_h, sa_w2, kK2, tc::idesc_bf16(128, kHid), false, bar);
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        hidden_epilogue(tD2 + lane_off, sH, r, row, a.n, a.Z2, c_lo, c_hi, a.w.gelu_tab);
        operands_ready();
        if (tid == 0) issue_gemm(tD3, sa_h, sa_w3, kK2, tc::idesc_bf16(128, kN3), false, bar);
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        if (cg == 0) {                       // the 8 outputs: one column group (warp-uniform)
            float y[16];
            tc::tmem_ld16(tD3 + lane_off, y);
            float part = 0.f;
            if (row < a.n) {
                if (a.Y != nullptr) {
                    float4* yr = reinterpret_cast<float4*>(a.Y + row * kOut);
                    yr[0] = make_float4(y[0], y[1], y[2], y[3]);
                    yr[1] = make_float4(y[4], y[5], y[6], y[7]);
                }
                if (a.T != nullptr) {
                    const float4* tr = reinterpret_cast<const float4*>(a.T + row * kOut);
                    const float4 t0 = tr[0], t1 = tr[1];
                    const float d[8] = {y[0] - t0.x, y[1] - t0.y, y[2] - t0.z, y[3] - t0.w,
                                        y[4] - t1.x, y[5] - t1.y, y[6] - t1.z, y[7] - t1.w};
                    float gr[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) { part += d[i] * d[i]; gr[i] = 2.f * a.loss_scale * d[i]; }
                    float4* dr = reinterpret_cast<float4*>(a.dY + row * kOut);
                    dr[0] = make_float4(gr[0], gr[1], gr[2], gr[3]);
                    dr[1] = make_float4(gr[4], gr[5], gr[6], gr[7]);
                }
            }
            if (a.T != nullptr) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                if (lane == 0) atomicAdd(a.loss, a.loss_scale * part);
            }
        }
        tc::fence_before_sync();
        __syncthreads();      // tensor memory and shared operands are reused by the next tile
    }
    if (!ok && tid == 0) set_status(a.status, GS_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

// ---------------------------------------------------------------- backward
// Shared-memory plan (bytes).  "x^T" operands are contracted over the tile's 128
// samples (K = sample) by the weight-gradient GEMMs; they are stored MN-major
// (tc.cuh), so the thread that owns a sample writes 8 consecutive rows of one as
// one 16-byte store.
constexpr uint32_t kBwdW2t = 0;                                 // W2^T [128 i][128 j]         B of dH1
constexpr uint32_t kBwdW3f = kBwdW2t + kHid * kHid * 2;         // W3 as float [8][128]
constexpr uint32_t kBwdA2 = kBwdW3f + kOut * kHid * 4;          // dZ2 [128 b][128 j]           A of dH1
                                                                //   later dZ1^T [128 i][128 b] A of dW1
constexpr uint32_t kBwdA2t = kBwdA2 + kTile * kHid * 2;         // dZ2^T [128 j][128 b]         A of dW2
                                                                //   first H2 [128 b][128 j] row-major
constexpr uint32_t kBwdB2 = kBwdA2t + kHid * kTile * 2;         // H1_aug^T [144 i][128 b]      B of dW2
constexpr uint32_t kBwdB1 = kBwdB2 + kK2 * kTile * 2;           // X_aug^T [208 k][128 b]       B of dW1
constexpr uint32_t kBwdDY = kBwdB1 + kK1 * kTile * 2;           // dY [128 b][8] float
constexpr uint32_t kBwdBar = kBwdDY + kTile * kOut * 4;
constexpr uint32_t kBwdSmem = kBwdBar + 16;
// tensor-memory columns of the three accumulators
constexpr uint32_t kTdH1 = 0, kTdW2 = 128, kTdW1 = 288;

struct MlpBwdArgs {
    gs_mlp_packed w;
    const uint16_t *X, *Z1, *Z2;
    const float* dY;
    int64_t n;
    gs_mlp_grads g;      // zeroed before the launch; accumulated with atomics
    int* status;
    uint32_t wait_polls; // mbarrier polls before a wait gives up
};

__global__ void __launch_bounds__(kFwdThreads, 1) k_mlp_bwd(MlpBwdArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cg = warp >> 2;            // tensor-memory lane quarter, column group
    const int r = quarter * 32 + lane;                       // this thread's sample (or weight) row
    float* sW3f = reinterpret_cast<float*>(sm + kBwdW3f);
    uint8_t* sA2 = sm + kBwdA2;
    uint8_t* sA2t = sm + kBwdA2t;
    uint8_t* sB2 = sm + kBwdB2;
    uint8_t* sB1 = sm + kBwdB1;
    float* sDY = reinterpret_cast<float*>(sm + kBwdDY);
    const uint32_t bar = tc::smem_addr(sm + kBwdBar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kBwdBar + 8);

    fill_kmajor(sm + kBwdW2t, a.w.W2t, kHid, kHid);
    for (int i = tid; i < kOut * kHid; i += kFwdThreads)
        sW3f[i] = bf2f(a.w.W3a[(i / kHid) * kK2 + (i % kHid)]);
    // constant rows of H1_aug^T: row 128 = 1 (the ones column of H1), rows 129..143 = 0
    for (int k = tid; k < 2 * kTile; k += kFwdThreads) {
        const int b = k % kTile, q = k / kTile;
        *reinterpret_cast<uint4*>(sB2 + tc::mnmajor_offset(kHid + 8 * q, b, kTile)) =
            make_uint4(q == 0 ? 0x3F80u : 0u, 0u, 0u, 0u);
    }
    for (int b = tid; b < kTile; b += kFwdThreads)       // X_aug^T rows 200..207: zeros
        *reinterpret_cast<uint4*>(sB1 + tc::mnmajor_offset(kK1 - 8, b, kTile)) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) tc::mbar_init(bar, 1);
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), kTmemCols);
    operands_ready();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t sa_a2 = tc::smem_addr(sA2), sa_a2t = tc::smem_addr(sA2t), sa_b2 = tc::smem_addr(sB2);
    const uint32_t sa_b1 = tc::smem_addr(sB1), sa_w2t = tc::smem_addr(sm + kBwdW2t);
    const int jw = tid & (kHid - 1), part = tid >> 7;        // dW3: hidden unit, quarter of the samples
    float acc3[kOut];
#pragma unroll
    for (int o = 0; o < kOut; o++) acc3[o] = 0.f;
    float accb3 = 0.f;
    uint32_t phase = 0;
    bool ok = true, first = true;
    const int64_t n_tiles = (a.n + kTile - 1) / kTile;
    // this thread's hidden columns: chunks 4 cg .. 4 cg + 3 (32 values) of Z2 and Z1,
    // and its sample's dY, loaded for tile t + gridDim.x while tile t's last GEMM
    // runs, and used by steps (1), (3) and (5) of the next tile
    constexpr int kZc = kHid / 8 / kColGroups;
    uint4 z2c[kZc], z1c[kZc];
    float4 dy0, dy1;
    auto load_rows = [&](int64_t tile) {
        const int64_t rw = tile * kTile + r;
        const bool v = tile < n_tiles && rw < a.n;
#pragma unroll
        for (int q = 0; q < kZc; q++) {
            const int c = kZc * cg + q;
            z2c[q] = v ? __ldg(reinterpret_cast<const uint4*>(a.Z2 + rw * kHid) + c) : make_uint4(0u, 0u, 0u, 0u);
            z1c[q] = v ? __ldg(reinterpret_cast<const uint4*>(a.Z1 + rw * kHid) + c) : make_uint4(0u, 0u, 0u, 0u);
        }
        dy0 = v ? __ldg(reinterpret_cast<const float4*>(a.dY + rw * kOut)) : make_float4(0.f, 0.f, 0.f, 0.f);
        dy1 = v ? __ldg(reinterpret_cast<const float4*>(a.dY + rw * kOut) + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    load_rows(blockIdx.x);
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int64_t row = t * kTile + r;
        const bool valid = row < a.n;
        // (1) X_aug^T, dY and H2 (row-major, for the CUDA-core dW3) of this sample
#pragma unroll 1
        for (int c = cg; c < kIn / 8 + 1; c += kColGroups) {
            // the inputs are needed only by the dW1 GEMM at the end of the tile: copied
            // asynchronously, waited for just before it; the partial chunk 24 (4 inputs,
            // the ones column) by a plain store; chunk 25 holds zeros from the start
            uint8_t* dst = sB1 + tc::mnmajor_offset(8 * c, r, kTile);
            if (c < kIn / 8) cp_async16(tc::smem_addr(dst), a.X + (valid ? row : 0) * kK1 + 8 * c, valid);
            else *reinterpret_cast<uint4*>(dst) = x_chunk(a.X, row, a.n, c);
        }
        const float dy[kOut] = {dy0.x, dy0.y, dy0.z, dy0.w, dy1.x, dy1.y, dy1.z, dy1.w};
        if (cg == 0) {
            reinterpret_cast<float4*>(sDY + r * kOut)[0] = dy0;
            reinterpret_cast<float4*>(sDY + r * kOut)[1] = dy1;
        }
        uint16_t* sH2 = reinterpret_cast<uint16_t*>(sA2t);   // [b][j], aliases dZ2^T until step (3)
#pragma unroll
        for (int q = 0; q < kZc; q++) {
            const int c = kZc * cg + q;
            const uint32_t w[4] = {z2c[q].x, z2c[q].y, z2c[q].z, z2c[q].w};
            uint32_t h[4];
#pragma unroll
            for (int i = 0; i < 4; i++)
                h[i] = pack2(__ldg(a.w.gelu_tab + (w[i] & 0xFFFFu)), __ldg(a.w.gelu_tab + (w[i] >> 16)));
            *reinterpret_cast<uint4*>(sH2 + r * kHid + 8 * c) = make_uint4(h[0], h[1], h[2], h[3]);
        }
        __syncthreads();
        // (2) dW3[o][j] += sum_b dY[b][o] H2[b][j] (thread j, a quarter of the samples); db3
#pragma unroll 4
        for (int b = part * 32; b < part * 32 + 32; b++) {
            const float h = bf2f(sH2[b * kHid + jw]);
            const float4 d0 = reinterpret_cast<const float4*>(sDY + b * kOut)[0];
            const float4 d1 = reinterpret_cast<const float4*>(sDY + b * kOut)[1];
            acc3[0] += d0.x * h; acc3[1] += d0.y * h; acc3[2] += d0.z * h; acc3[3] += d0.w * h;
            acc3[4] += d1.x * h; acc3[5] += d1.y * h; acc3[6] += d1.z * h; acc3[7] += d1.w * h;
        }
        if (tid < kOut)
            for (int b = 0; b < kTile; b++) accb3 += sDY[b * kOut + tid];
        __syncthreads();
        // (3) dZ2 = bf16((dY W3) * gelu'(Z2)) as dZ2 rows and dZ2^T; H1 = bf16(gelu(Z1)) as H1_aug^T
#pragma unroll
        for (int q = 0; q < kZc; q++) {
            const int c = kZc * cg + q;
            const uint32_t w[4] = {z2c[q].x, z2c[q].y, z2c[q].z, z2c[q].w};
            uint16_t g[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const int j = 8 * c + i;
                float dh = 0.f;
#pragma unroll
                for (int o = 0; o < kOut; o++) dh += dy[o] * sW3f[o * kHid + j];
                const uint32_t zb = (i & 1) ? (w[i >> 1] >> 16) : (w[i >> 1] & 0xFFFFu);
                g[i] = f2bf(dh * __ldg(a.w.dgelu_tab + zb));
            }
            const uint4 gp = make_uint4(pack2(g[0], g[1]), pack2(g[2], g[3]), pack2(g[4], g[5]), pack2(g[6], g[7]));
            *reinterpret_cast<uint4*>(sA2t + tc::mnmajor_offset(8 * c, r, kTile)) = gp;
            *reinterpret_cast<uint4*>(sA2 + tc::kmajor_offset(r, 8 * c, kHid)) = gp;
            const uint32_t w1[4] = {z1c[q].x, z1c[q].y, z1c[q].z, z1c[q].w};
            uint32_t hp[4];
#pragma unroll
            for (int i = 0; i < 4; i++)
                hp[i] = pack2(__ldg(a.w.gelu_tab + (w1[i] & 0xFFFFu)), __ldg(a.w.gelu_tab + (w1[i] >> 16)));
            *reinterpret_cast<uint4*>(sB2 + tc::mnmajor_offset(8 * c, r, kTile)) =
                make_uint4(hp[0], hp[1], hp[2], hp[3]);
        }
        operands_ready();
        // (4) dH1 = dZ2 W2 and dW2_aug += dZ2^T H1_aug
        if (tid == 0) {
            tc::fence_after_sync();
            for (int st = 0; st < kHid / 16; st++)
                tc::mma_bf16(tbase + kTdH1, tc::kstep_desc(sa_a2, kHid, st), tc::kstep_desc(sa_w2t, kHid, st),
                             tc::idesc_bf16(128, kHid), st > 0);
            for (int st = 0; st < kTile / 16; st++)
                tc::mma_bf16(tbase + kTdW2, tc::kstep_desc(sa_a2t, kTile, st), tc::kstep_desc(sa_b2, kTile, st),
                             tc::idesc_bf16_mn(128, kK2, true, true), !first || st > 0);
            tc::mma_commit(bar);
        }
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        // (5) dZ1 = bf16(dH1 * gelu'(Z1)) as dZ1^T (over the dZ2 buffer, whose GEMM is done)
        uint8_t* sA1t = sA2;
#pragma unroll
        for (int h2 = 0; h2 < kZc / 2; h2++) {
            const int c0 = 8 * kZc * cg + 16 * h2;
            float v[16];
            tc::tmem_ld16(tbase + kTdH1 + lane_off + (uint32_t)c0, v);
            const uint32_t w[8] = {z1c[2 * h2].x, z1c[2 * h2].y, z1c[2 * h2].z, z1c[2 * h2].w,
                                   z1c[2 * h2 + 1].x, z1c[2 * h2 + 1].y, z1c[2 * h2 + 1].z, z1c[2 * h2 + 1].w};
            uint32_t gp[8];
#pragma unroll
            for (int i = 0; i < 8; i++)
                gp[i] = pack2(f2bf(v[2 * i] * __ldg(a.w.dgelu_tab + (w[i] & 0xFFFFu))),
                              f2bf(v[2 * i + 1] * __ldg(a.w.dgelu_tab + (w[i] >> 16))));
            *reinterpret_cast<uint4*>(sA1t + tc::mnmajor_offset(c0, r, kTile)) = make_uint4(gp[0], gp[1], gp[2], gp[3]);
            *reinterpret_cast<uint4*>(sA1t + tc::mnmajor_offset(c0 + 8, r, kTile)) =
                make_uint4(gp[4], gp[5], gp[6], gp[7]);
        }
        load_rows(t + gridDim.x);          // the next tile's rows, in flight during the dW1 GEMM
        cp_async_wait_all();
        operands_ready();
        // (6) dW1_aug += dZ1^T X_aug
        if (tid == 0) {
            tc::fence_after_sync();
            for (int st = 0; st < kTile / 16; st++)
                tc::mma_bf16(tbase + kTdW1, tc::kstep_desc(sa_a2, kTile, st), tc::kstep_desc(sa_b1, kTile, st),
                             tc::idesc_bf16_mn(128, kK1, true, true), !first || st > 0);
            tc::mma_commit(bar);
        }
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        first = false;
    }
    if (!ok && tid == 0) set_status(a.status, GS_ERR_TIMEOUT);
    cp_async_wait_all();     // after a timeout this thread's input copies may still be in flight
    if (ok && !first) {
        // accumulated weight gradients of this CTA -> global (row r of dW1_aug, dW2_aug; every fourth chunk)
#pragma unroll 1
        for (int c0 = 16 * cg; c0 < kK1; c0 += 16 * kColGroups) {
            float v[16];
            tc::tmem_ld16(tbase + kTdW1 + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int k = c0 + i;
                if (k < kIn) atomicAdd(a.g.W1 + r * kIn + k, v[i]);
                else if (k == kIn) atomicAdd(a.g.b1 + r, v[i]);
            }
        }
#pragma unroll 1
        for (int c0 = 16 * cg; c0 < kK2; c0 += 16 * kColGroups) {
            float v[16];
            tc::tmem_ld16(tbase + kTdW2 + lane_off + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int k = c0 + i;
                if (k < kHid) atomicAdd(a.g.W2 + r * kHid + k, v[i]);
                else if (k == kHid) atomicAdd(a.g.b2 + r, v[i]);
            }
        }
#pragma unroll
        for (int o = 0; o < kOut; o++) atomicAdd(a.g.W3 + o * kHid + jw, acc3[o]);
        if (tid < kOut) atomicAdd(a.g.b3 + tid, accb3);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

}  // namespace

uint32_t set_mlp_wait_polls(uint32_t polls) { return g_wait_polls.exchange(polls); }

static int sm_count() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

cudaError_t launch_mlp_pack(const gs_mlp_params& p, const gs_mlp_packed& q, cudaStream_t s) {
    k_mlp_pack<<<2 * sm_count(), 256, 0, s>>>(p, q);
    return cudaGetLastError();
}

cudaError_t launch_mlp_fwd(const gs_mlp_packed& w, const uint16_t* X, int64_t n, float* Y, uint16_t* Z1,
                           uint16_t* Z2, const float* T, float* dY, float* loss, float loss_scale, int* status,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
    MlpFwdArgs a{w, X, n, Y, Z1, Z2, T, dY, loss, loss_scale, status, g_wait_polls.load()};
    k_mlp_fwd<<<grid, kFwdThreads, kFwdSmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_bwd(const gs_mlp_packed& w, const uint16_t* X, const uint16_t* Z1, const uint16_t* Z2,
                           const float* dY, int64_t n, const gs_mlp_grads& g, int* status, cudaStream_t s) {
    const size_t sizes[6] = {sizeof(float) * kHid * kIn, sizeof(float) * kHid, sizeof(float) * kHid * kHid,
                             sizeof(float) * kHid, sizeof(float) * kOut * kHid, sizeof(float) * kOut};
    float* ptrs[6] = {g.W1, g.b1, g.W2, g.b2, g.W3, g.b3};
    for (int i = 0; i < 6; i++) {
        cudaError_t e = cudaMemsetAsync(ptrs[i], 0, sizes[i], s);
        if (e != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
    MlpBwdArgs a{w, X, Z1, Z2, dY, n, g, status, g_wait_polls.load()};
    k_mlp_bwd<<<grid, kFwdThreads, kBwdSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gs
