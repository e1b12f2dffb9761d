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
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <atomic>
#include <climits>
#include <mutex>

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
__device__ __forceinline__ void operands_ready() {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
}

// ---------------------------------------------------------------- forward
// The activation in shared memory: the packed tables' entries for the BF16
// inputs with 2^-10 <= |z| < 2^4 (bit patterns 0x3A80 .. 0x417F of either sign,
// 14 binades), where nearly every pre-activation falls.  Slot = magnitude
// offset (11 bits, 0 .. 0x6FF) | sign << 11, so the index takes no branch; the
// rare inputs outside are patched from the full tables in global memory.  A
// random lookup in shared memory costs a few bank conflicts, one in a 128 KB
// global table many L1 wavefronts.
constexpr uint32_t kTabLo = 0x3A80u, kTabSpan = 0x0700u;
constexpr int kTabEntries = 4096;

__device__ __forceinline__ uint32_t tab_slot(uint32_t z, bool& miss) {
    const uint32_t i = (z & 0x7FFFu) - kTabLo;       // wraps below the range
    miss = i >= kTabSpan;
    return (i & 0x7FFu) | ((z >> 4) & 0x800u);
}
// BF16 bit pattern of slot i, or 0xFFFFFFFF for the unused slots
__device__ __forceinline__ uint32_t tab_bits(int i) {
    return (uint32_t)(i & 0x7FF) < kTabSpan ? ((uint32_t)(i & 0x800) << 4) | (kTabLo + (uint32_t)(i & 0x7FF))
                                            : 0xFFFFFFFFu;
}
// bf16(gelu) of both BF16 halves of w; `miss` if either lies outside the compact table
__device__ __forceinline__ uint32_t gelu2(uint32_t w, const uint16_t* s_tab, bool& miss) {
    bool m0, m1;
    const uint32_t lo = s_tab[tab_slot(w & 0xFFFFu, m0)], hi = s_tab[tab_slot(w >> 16, m1)];
    miss = m0 | m1;
    return lo | (hi << 16);
}
__device__ __forceinline__ uint32_t gelu2_global(uint32_t w, const uint16_t* __restrict__ g_tab) {
    return (uint32_t)__ldg(g_tab + (w & 0xFFFFu)) | ((uint32_t)__ldg(g_tab + (w >> 16)) << 16);
}
// BF16 pair (lower half = a) rounded to nearest
__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}
// Compact table from the full one (slots without an input get 0).
template <typename T>
__device__ __forceinline__ void fill_tab(T* s_tab, const T* __restrict__ g_tab) {
    for (int i = threadIdx.x; i < kTabEntries; i += blockDim.x) {
        const uint32_t z = tab_bits(i);
        s_tab[i] = z != 0xFFFFFFFFu ? __ldg(g_tab + z) : T(0);
    }
}

// One tile of X in shared memory, as TMA lands it: columns 0 .. 191 in three
// boxes of 64 columns x 128 rows with the 128-byte swizzle (16 KB each, rows of
// 128 bytes, the layout of tc::smem_desc_sw128), then columns 192 .. 207 as two
// unswizzled chunks of 8 columns (element (r, k) at (k / 8 - 24) 2048 + r 16 +
// (k % 8) 2).  Columns 196 .. 199 of the first chunk lie outside the tensor map
// and arrive as zeros, as do rows past n; the second chunk stays zero.  A copy
// of 128-byte rows costs one request per row where 8-column boxes cost 8.
constexpr uint32_t kXChunk = kTile * 16;
constexpr uint32_t kXBox = kTile * 128;                 // one 64-column box
constexpr uint32_t kXTail = 3 * kXBox;                  // the two 8-column chunks
constexpr uint32_t kXBytes = kXTail + 2 * kXChunk;
constexpr uint32_t kXTx = 3 * kXBox + kXChunk;          // bytes per tile of X
static_assert(kXBytes == (uint32_t)kTile * kK1 * 2, "X tile size");

// descriptor of K step s (16 columns) of an X tile at sx (1024-byte aligned)
__device__ __forceinline__ uint64_t x_desc(uint32_t sx, int s) {
    return s < 12 ? tc::smem_desc_sw128(sx + (uint32_t)(s / 4) * kXBox + (uint32_t)(s % 4) * 32u)
                  : tc::smem_desc(sx + kXTail, kXChunk, 128u);
}

// Shared-memory plan of the forward kernel (bytes): the three weight operands
// stay resident; X is a two-stage ring of TMA destinations; then the activation
// table, the layer-1 bias (added in the epilogue, since the tensor map zero-fills
// the ones column) and the barriers.
constexpr uint32_t kFwdX = 0;                                   // 2 x (128 x 208), 1024-byte aligned
constexpr uint32_t kFwdW1 = kFwdX + 2 * kXBytes;                // 128 x 208
constexpr uint32_t kFwdW2 = kFwdW1 + kHid * kK1 * 2;            // 128 x 144
constexpr uint32_t kFwdW3 = kFwdW2 + kHid * kK2 * 2;            // 16 x 144
constexpr uint32_t kFwdTab = kFwdW3 + kN3 * kK2 * 2;            // 4096 BF16
constexpr uint32_t kFwdB1 = kFwdTab + kTabEntries * 2;          // 128 FP32
constexpr uint32_t kFwdBar = kFwdB1 + kHid * 4;
// barriers (8 bytes each): x_full[2], g1[2], g2[2], g3[2], h1[2], h2[2], drain; then
// the tensor-memory base and the abort flag
constexpr int kBarXFull = 0, kBarG1 = 2, kBarG2 = 4, kBarG3 = 6, kBarH1 = 8, kBarH2 = 10, kBarDrain = 12;
constexpr uint32_t kFwdSmem = kFwdBar + 13 * 8 + 8;
static_assert(kFwdX % 1024 == 0 && kXBytes % 1024 == 0, "swizzled TMA destinations are 1024-byte aligned");
static_assert(kFwdSmem <= 227 * 1024, "shared memory of one CTA");

// Tensor memory of the forward: two slots of 256 columns, one per tile in flight.
// D: the 128 x 128 FP32 accumulator of layers 1 and 2; D3: layer 3 (N 16);
// H: the next layer's A operand, 128 x 144 BF16 packed two per column (72
// columns; columns 64 .. 71 hold the ones column and zeros, written once).
constexpr uint32_t kSlotCols = 256, kColD = 0, kColD3 = 128, kColH = 160;

// The epilogue warps are 0 .. 15, warp 16 issues the copies and the MMAs.
constexpr int kEpiThreads = 512, kCtlWarp = kEpiThreads / 32, kFwdThreads2 = kEpiThreads + 32;

struct MlpFwdArgs {
    gs_mlp_packed w;
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

// Poll the barrier phase at most `polls` times; give up early once another
// thread of the CTA has raised the abort flag, and raise it on a timeout.
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, uint32_t polls,
                                              volatile int* abort_flag) {
    for (uint32_t i = 0; i < polls; i++) {
        if (tc::mbar_test(bar, parity)) return true;
        if ((i & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}
// The same for a whole warp, with a warp-uniform outcome (the tensor-memory
// loads and stores that follow are warp-collective).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, uint32_t polls, volatile int* abort_flag) {
    const bool ok = __all_sync(0xffffffffu, wait_or_abort(bar, parity, polls, abort_flag));
    tc::fence_after_sync();
    return ok;
}

// Hidden-layer epilogue of this thread's sample row, columns 32 cg .. 32 cg + 31,
// in two halves of 16: accumulator (+ bias) -> Z = bf16 (to global memory when
// Zrow is set) -> H = bf16(gelu(Z)) into tensor memory as the next layer's A
// operand.
__device__ __forceinline__ void hidden_epilogue(uint32_t tD, uint32_t tH, int cg, const float* bias,
                                                uint16_t* Zrow, const uint16_t* s_tab,
                                                const uint16_t* __restrict__ g_tab) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
        const int c0 = 32 * cg + 16 * half;
        float v[16];
        tc::tmem_ld16(tD + (uint32_t)c0, v);
        if (bias != nullptr) {
#pragma unroll
            for (int i = 0; i < 16; i += 4) {
                const float4 b = *reinterpret_cast<const float4*>(bias + c0 + i);
                v[i] += b.x; v[i + 1] += b.y; v[i + 2] += b.z; v[i + 3] += b.w;
            }
        }
        uint32_t zp[8], hp[8], miss = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            zp[i] = bf16x2(v[2 * i], v[2 * i + 1]);
            bool m;
            hp[i] = gelu2(zp[i], s_tab, m);
            miss |= (uint32_t)m << i;
        }
        if (miss != 0) {          // inputs outside the compact table (rare)
#pragma unroll
            for (int i = 0; i < 8; i++)
                if (miss & (1u << i)) hp[i] = gelu2_global(zp[i], g_tab);
        }
        if (Zrow != nullptr) {
            uint4* zr = reinterpret_cast<uint4*>(Zrow + c0);
            zr[0] = make_uint4(zp[0], zp[1], zp[2], zp[3]);
            zr[1] = make_uint4(zp[4], zp[5], zp[6], zp[7]);
        }
        tc::tmem_st8(tH + (uint32_t)(c0 / 2), hp);
    }
}

// This warp is done with a stage: its tensor-memory accesses are ordered
// before one arrival on the barrier (16 arrivals complete a phase).
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
    tc::fence_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(bar);
}

// Output layer of the tile's 128 samples (warps with cg == 0): Y, and in
// training dY and the loss.
__device__ __forceinline__ void output_epilogue(const MlpFwdArgs& a, uint32_t tD3, int64_t row, int lane) {
    float y[16];
    tc::tmem_ld16(tD3, y);
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

// The CTA walks its tiles t = blockIdx.x + k gridDim.x in pairs (slots 0 and 1),
// so that the tensor core runs one tile's GEMM while the epilogue warps work on
// the other's.  Per pair, the MMA order is
//   G2(a) G2(b) G3(a) G1(a') G3(b) G1(b')       (G1 of the first pair up front)
// and the epilogue order E1(a) E1(b) E2(a) E2(b) Out(a) Out(b); X(a') is copied
// by TMA as soon as G1(a) has consumed X(a).  Each barrier completes once per
// pair, so every wait uses the pair's parity.
__global__ void __launch_bounds__(kFwdThreads2, 1) k_mlp_fwd(const __grid_constant__ CUtensorMap xmap_sw,
                                                              const __grid_constant__ CUtensorMap xmap,
                                                              MlpFwdArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint16_t* s_tab = reinterpret_cast<uint16_t*>(sm + kFwdTab);
    float* s_b1 = reinterpret_cast<float*>(sm + kFwdB1);
    const uint32_t bars = tc::smem_addr(sm + kFwdBar);
    auto bar = [&](int i) { return bars + 8u * (uint32_t)i; };
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kFwdBar + 13 * 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kFwdBar + 13 * 8 + 4);

    fill_kmajor(sm + kFwdW1, a.w.W1a, kHid, kK1);
    fill_kmajor(sm + kFwdW2, a.w.W2a, kHid, kK2);
    fill_kmajor(sm + kFwdW3, a.w.W3a, kN3, kK2);
    for (int i = tid; i < 2 * kTile; i += blockDim.x)      // chunk 25 (columns 200 .. 207) of both stages
        *reinterpret_cast<uint4*>(sm + kFwdX + (i / kTile) * kXBytes + kXTail + kXChunk + (i % kTile) * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    fill_tab(s_tab, a.w.gelu_tab);
    for (int j = tid; j < kHid; j += blockDim.x) s_b1[j] = bf2f(a.w.W1a[j * kK1 + kIn]);
    if (tid == 0) {
        for (int i = 0; i < 13; i++)
            tc::mbar_init(bar(i), (i == kBarH1 || i == kBarH1 + 1 || i == kBarH2 || i == kBarH2 + 1) ? 16u : 1u);
        *abort_flag = 0;
    }
    if (warp == kCtlWarp) tc::tmem_alloc(tc::smem_addr(tslot), kTmemCols);
    operands_ready();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const int64_t n_tiles = (a.n + kTile - 1) / kTile;
    const int cnt = (int)((n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);   // tiles of this CTA (>= 1)
    const uint32_t polls = a.wait_polls;

    if (warp < kCtlWarp) {
        // ------------------------------------------------ epilogue warps
        const int q = warp & 3, cg = warp >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int r = q * 32 + lane;
        if (cg == 0) {   // H columns 64 .. 71 of both slots: the ones column (K index 128) and zeros
            uint32_t ones[16] = {0x3F80u};
            for (int s = 0; s < 2; s++) tc::tmem_st16(tbase + lane_off + s * kSlotCols + kColH + 64, ones);
        }
        bool ok = true;
        for (int k = 0; k < cnt && ok; k += 2) {
            const uint32_t par = (uint32_t)(k >> 1) & 1u;
            const int nslot = k + 1 < cnt ? 2 : 1;
            for (int s = 0; s < nslot && ok; s++) {          // E1
                if (!(ok = warp_wait(bar(kBarG1 + s), par, polls, abort_flag))) break;
                const int64_t row = (blockIdx.x + (int64_t)(k + s) * gridDim.x) * kTile + r;
                const uint32_t ts = tbase + lane_off + s * kSlotCols;
                hidden_epilogue(ts + kColD, ts + kColH, cg, s_b1,
                                a.Z1 != nullptr && row < a.n ? a.Z1 + row * kHid : nullptr, s_tab, a.w.gelu_tab);
                warp_arrive(bar(kBarH1 + s));
            }
            for (int s = 0; s < nslot && ok; s++) {          // E2
                if (!(ok = warp_wait(bar(kBarG2 + s), par, polls, abort_flag))) break;
                const int64_t row = (blockIdx.x + (int64_t)(k + s) * gridDim.x) * kTile + r;
                const uint32_t ts = tbase + lane_off + s * kSlotCols;
                hidden_epilogue(ts + kColD, ts + kColH, cg, nullptr,
                                a.Z2 != nullptr && row < a.n ? a.Z2 + row * kHid : nullptr, s_tab, a.w.gelu_tab);
                warp_arrive(bar(kBarH2 + s));
            }
            if (cg == 0) {
                for (int s = 0; s < nslot && ok; s++) {      // outputs
                    if (!(ok = warp_wait(bar(kBarG3 + s), par, polls, abort_flag))) break;
                    const int64_t row = (blockIdx.x + (int64_t)(k + s) * gridDim.x) * kTile + r;
                    output_epilogue(a, tbase + lane_off + s * kSlotCols + kColD3, row, lane);
                }
            }
        }
    } else if (lane == 0) {
        // ------------------------------------------------ copies and MMAs (one thread)
        const uint32_t sw1 = tc::smem_addr(sm + kFwdW1), sw2 = tc::smem_addr(sm + kFwdW2);
        const uint32_t sw3 = tc::smem_addr(sm + kFwdW3);
        uint32_t xpar = 0u, pending = 0u;      // bit s: parity of slot s's next copy; a copy in flight
        auto load_x = [&](int k) {
            if (k >= cnt) return;
            const int s = k & 1;
            const int y = (int)((blockIdx.x + (int64_t)k * gridDim.x) * kTile);
            const uint32_t sxs = tc::smem_addr(sm + kFwdX) + (uint32_t)s * kXBytes;
            tc::mbar_arrive_expect_tx(bar(kBarXFull + s), kXTx);
#pragma unroll
            for (int c = 0; c < 3; c++) tc::tma_load_2d(sxs + (uint32_t)c * kXBox, &xmap_sw, 64 * c, y, bar(kBarXFull + s));
            tc::tma_load_2d(sxs + kXTail, &xmap, 192, y, bar(kBarXFull + s));
            pending |= 1u << s;
        };
        auto wait_x = [&](int s) {
            if (!wait_or_abort(bar(kBarXFull + s), (xpar >> s) & 1u, polls, abort_flag)) return false;
            xpar ^= 1u << s;
            pending &= ~(1u << s);
            return true;
        };
        // descriptors of K step 0; step st adds st times the step's byte offset >> 4
        // to the start-address field (no carry: shared addresses stay below 2^18)
        const uint32_t sx0 = tc::smem_addr(sm + kFwdX), sx1 = sx0 + kXBytes;
        const uint64_t dx0 = x_desc(sx0, 0), dx1 = x_desc(sx1, 0), dt0 = x_desc(sx0, 12), dt1 = x_desc(sx1, 12);
        const uint64_t dw1 = tc::kstep_desc(sw1, kK1, 0), dw2 = tc::kstep_desc(sw2, kK2, 0);
        const uint64_t dw3 = tc::kstep_desc(sw3, kK2, 0);
        auto gemm1 = [&](int s) {
            const uint32_t d = tbase + s * kSlotCols + kColD;
            const uint64_t dx = s ? dx1 : dx0, dt = s ? dt1 : dt0;
#pragma unroll
            for (int st = 0; st < kK1 / 16; st++)
                tc::mma_bf16(d, st < 12 ? dx + (uint64_t)(((st / 4) * kXBox + (st % 4) * 32) >> 4) : dt,
                             dw1 + (uint64_t)(st * 16), tc::idesc_bf16(128, kHid), st > 0);
            tc::mma_commit(bar(kBarG1 + s));
        };
        auto gemm_h = [&](int s, uint32_t col, uint64_t dw, uint32_t idesc, int g) {
            const uint32_t h = tbase + s * kSlotCols + kColH;
#pragma unroll
            for (int st = 0; st < kK2 / 16; st++)
                tc::mma_bf16_ts(tbase + s * kSlotCols + col, h + 8u * (uint32_t)st, dw + (uint64_t)(st * 16), idesc,
                                st > 0);
            tc::mma_commit(bar(g + s));
        };
        bool ok = true;
        load_x(0);
        load_x(1);
        if ((ok = wait_x(0))) gemm1(0);
        if (ok && cnt > 1 && (ok = wait_x(1))) gemm1(1);
        for (int k = 0; k < cnt && ok; k += 2) {
            const uint32_t par = (uint32_t)(k >> 1) & 1u;
            const bool has_b = k + 1 < cnt;
            if (!(ok = wait_or_abort(bar(kBarG1), par, polls, abort_flag))) break;
            load_x(k + 2);                                           // X(a) consumed
            if (!(ok = wait_or_abort(bar(kBarH1), par, polls, abort_flag))) break;
            tc::fence_after_sync();
            gemm_h(0, kColD, dw2, tc::idesc_bf16(128, kHid), kBarG2);
            if (has_b) {
                if (!(ok = wait_or_abort(bar(kBarG1 + 1), par, polls, abort_flag))) break;
                load_x(k + 3);
                if (!(ok = wait_or_abort(bar(kBarH1 + 1), par, polls, abort_flag))) break;
                tc::fence_after_sync();
                gemm_h(1, kColD, dw2, tc::idesc_bf16(128, kHid), kBarG2);
            }
            if (!(ok = wait_or_abort(bar(kBarH2), par, polls, abort_flag))) break;
            tc::fence_after_sync();
            gemm_h(0, kColD3, dw3, tc::idesc_bf16(128, kN3), kBarG3);
            if (k + 2 < cnt) {                                       // D(a) read by E2(a): next tile's layer 1
                if (!(ok = wait_x(0))) break;
                gemm1(0);
            }
            if (has_b) {
                if (!(ok = wait_or_abort(bar(kBarH2 + 1), par, polls, abort_flag))) break;
                tc::fence_after_sync();
                gemm_h(1, kColD3, dw3, tc::idesc_bf16(128, kN3), kBarG3);
                if (k + 3 < cnt) {
                    if (!(ok = wait_x(1))) break;
                    gemm1(1);
                }
            }
        }
        // drain: every MMA issued and every copy in flight completes before the
        // CTA frees its tensor memory and exits (bounded again)
        tc::mma_commit(bar(kBarDrain));
        tc::mbar_wait(bar(kBarDrain), 0, kDrainPolls);
        for (int s = 0; s < 2; s++)
            if (pending & (1u << s)) tc::mbar_wait(bar(kBarXFull + s), (xpar >> s) & 1u, kDrainPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kCtlWarp) {
        tc::fence_after_sync();
        if (lane == 0 && *abort_flag) set_status(a.status, GS_ERR_TIMEOUT);
        tc::tmem_dealloc(tbase, kTmemCols);
    }
}

// ---------------------------------------------------------------- backward
// Every contraction runs on the tensor cores.  Per tile of 128 samples b:
//   (1) dH2 = dY W3           A = dY split [b][32], B = W3 split [j][32]   (K 32)
//   (2) Z2 pass: H2 = bf16(gelu(Z2)), dZ2 = bf16(dH2 * gelu'(Z2))
//   (3) dH1 = dZ2 W2          A = dZ2 [b][j], B = W2^T [i][j]             (K 128)
//       dW3_split += H2^T dY  A = H2^T [j][b], B = dY split^T [n][b]      (K 128 = b)
//   (4) Z1 pass: H1 = bf16(gelu(Z1)) -> H1_aug^T; then dZ1 = bf16(dH1 * gelu'(Z1))
//   (5) dW2_aug += dZ2^T H1_aug   A = dZ2 (read transposed), B = H1_aug^T [i][b]
//       dW1_aug += dZ1^T X_aug    A = dZ1^T [i][b], B = X_aug^T [k][b]   (TMA)
// dY is FP32; it enters the tensor core as three BF16 parts h + m + l (h =
// bf16(dY), m = bf16(dY - h), l = bf16(dY - h - m)), which hold its 24-bit
// significand, so with BF16 W3 / H2 every product is exact and only the FP32
// accumulation rounds, as on the CUDA cores.  dW3 is the sum of its three part
// columns; db3 is summed on the CUDA cores.
//
// The per-tile operands share one layout: element (sample b, column c) at
// (c / 8) 2048 + b 16 + (c % 8) 2 (chunks of 8 columns x 128 samples, as TMA
// lands X).  Read with leading byte offset 2048 / stride byte offset 128 it is
// the K-major operand [b][c]; with 128 / 2048 the MN-major operand [c][b].  So
// one copy of dZ2 serves as A of dH1 (K-major) and, transposed, as A of dW2.
//
// The activation: one 8-byte entry {gelu'(z) FP32, bf16(gelu(z))} per BF16
// input with 2^-9 <= |z| < 2^4 (13 binades, slot = offset + sign * span),
// others from the full tables in global memory.
constexpr uint32_t kBTabLo = 0x3B00u, kBTabSpan = 0x0680u;
constexpr int kBTabEntries = 2 * kBTabSpan;

__device__ __forceinline__ uint32_t btab_slot(uint32_t z, bool& miss) {
    const uint32_t i = (z & 0x7FFFu) - kBTabLo;
    miss = i >= kBTabSpan;
    return min(i, kBTabSpan - 1u) + (z >> 15) * kBTabSpan;
}

// Shared-memory plan (bytes)
constexpr uint32_t kBwdW2t = 0;                                   // W2^T [128 i][128 j], K-major
constexpr uint32_t kBwdW3s = kBwdW2t + kHid * kHid * 2;           // W3 split [128 j][32], K-major
constexpr uint32_t kBwdDYs = kBwdW3s + kHid * 32 * 2;             // dY split, chunk layout (4 chunks)
constexpr uint32_t kBwdP1 = kBwdDYs + 4 * kXChunk;                // H2^T, then dZ1^T (16 chunks)
constexpr uint32_t kBwdDZ2 = kBwdP1 + 16 * kXChunk;               // dZ2 (16 chunks)
constexpr uint32_t kBwdH1 = kBwdDZ2 + 16 * kXChunk;               // H1_aug^T (18 chunks)
constexpr uint32_t kBwdX = kBwdH1 + 18 * kXChunk;                 // X_aug^T (26 chunks, TMA)
constexpr uint32_t kBwdTab = kBwdX + 26 * kXChunk;                // 3328 x 8 bytes
constexpr uint32_t kBwdBar = kBwdTab + kBTabEntries * 8;          // MMA, X and drain barriers, tmem base
constexpr uint32_t kBwdB3 = kBwdBar + 32;                         // db3 of this CTA (8 FP32)
constexpr uint32_t kBwdSmem = kBwdB3 + 32;
static_assert(kBwdX % 128 == 0, "TMA destination is 128-byte aligned");
// X_aug^T: chunks 0 .. 24 copied per tile (8 columns each, unswizzled), chunk 25 stays zero
constexpr int kBwdXLoads = kIn / 8 + 1;
constexpr uint32_t kBwdXTx = kBwdXLoads * kXChunk;
static_assert(kBwdSmem <= 227 * 1024, "shared memory of one CTA");
// tensor-memory columns: dH (dH2, then dH1), the dW3 parts, dW1_aug, dW2_aug
constexpr uint32_t kTdH = 0, kTdW3 = 128, kTdW1 = 160, kTdW2 = 368;
static_assert(kTdW2 + kK2 <= kTmemCols, "tensor-memory columns");

__device__ __forceinline__ uint64_t chunk_kmajor(uint32_t base, int s) { return tc::smem_desc(base + 4096u * s, 2048u, 128u); }
__device__ __forceinline__ uint64_t chunk_mnmajor(uint32_t base, int s) { return tc::smem_desc(base + 256u * s, 128u, 2048u); }

struct MlpBwdArgs {
    gs_mlp_packed w;
    const uint16_t *Z1, *Z2;
    const float* dY;
    int64_t n;
    gs_mlp_grads g;      // zeroed before the launch; accumulated with atomics
    int* status;
    uint32_t wait_polls; // mbarrier polls before a wait gives up
};

__global__ void __launch_bounds__(kEpiThreads, 1) k_mlp_bwd(const __grid_constant__ CUtensorMap xmap, MlpBwdArgs a) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cg = warp >> 2;            // tensor-memory lane quarter, column group
    const int r = quarter * 32 + lane;                       // this thread's sample (or weight) row
    const uint2* s_tab = reinterpret_cast<const uint2*>(sm + kBwdTab);
    const uint32_t bar = tc::smem_addr(sm + kBwdBar), xbar = bar + 8, dbar = bar + 16;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kBwdBar + 24);
    float* s_b3 = reinterpret_cast<float*>(sm + kBwdB3);

    fill_kmajor(sm + kBwdW2t, a.w.W2t, kHid, kHid);
    for (int i = tid; i < kHid * 4; i += kEpiThreads) {       // W3 split: columns 8p + o = W3[o][j], p < 3
        const int j = i % kHid, c = i / kHid;
        uint32_t v[4] = {0u, 0u, 0u, 0u};
        if (c < 3)
            for (int o = 0; o < kOut; o += 2)
                v[o / 2] = pack2(a.w.W3a[o * kK2 + j], a.w.W3a[(o + 1) * kK2 + j]);
        *reinterpret_cast<uint4*>(sm + kBwdW3s + tc::kmajor_offset(j, 8 * c, 32)) = make_uint4(v[0], v[1], v[2], v[3]);
    }
    for (int i = tid; i < kBTabEntries; i += kEpiThreads) {
        const uint32_t z = (i < (int)kBTabSpan ? 0u : 0x8000u) | (kBTabLo + (uint32_t)i % kBTabSpan);
        reinterpret_cast<uint2*>(sm + kBwdTab)[i] =
            make_uint2(__float_as_uint(__ldg(a.w.dgelu_tab + z)), (uint32_t)__ldg(a.w.gelu_tab + z));
    }
    if (tid < kTile) {
        // H1_aug^T rows 128 .. 143: the ones row and zeros; X_aug^T rows 200 .. 207: zeros
        *reinterpret_cast<uint4*>(sm + kBwdH1 + 16 * kXChunk + tid * 16) = make_uint4(0x3F80u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sm + kBwdH1 + 17 * kXChunk + tid * 16) = make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sm + kBwdX + 25 * kXChunk + tid * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid < kOut) s_b3[tid] = 0.f;
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(xbar, 1);
        tc::mbar_init(dbar, 1);
    }
    if (warp == 0) tc::tmem_alloc(tc::smem_addr(tslot), kTmemCols);
    operands_ready();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t s_w2t = tc::smem_addr(sm + kBwdW2t), s_w3s = tc::smem_addr(sm + kBwdW3s);
    const uint32_t s_dys = tc::smem_addr(sm + kBwdDYs), s_p1 = tc::smem_addr(sm + kBwdP1);
    const uint32_t s_dz2 = tc::smem_addr(sm + kBwdDZ2), s_h1 = tc::smem_addr(sm + kBwdH1);
    const uint32_t s_x = tc::smem_addr(sm + kBwdX);
    const int64_t n_tiles = (a.n + kTile - 1) / kTile;

    auto load_x = [&](int64_t tile) {     // thread 0
        tc::mbar_arrive_expect_tx(xbar, kBwdXTx);
        for (int c = 0; c < kBwdXLoads; c++)
            tc::tma_load_2d(s_x + (uint32_t)c * kXChunk, &xmap, 8 * c, (int)(tile * kTile), xbar);
    };
    // this thread's sample row of Z1 and Z2 (columns 32 cg .. 32 cg + 31) and dY
    // (column group 0), for a tile; each is loaded for the next tile as soon as
    // this tile has used it, so the loads have most of a tile to arrive
    constexpr int kZc = kHid / 8 / kColGroups;
    uint4 z2c[kZc], z1c[kZc];
    float4 dy0 = make_float4(0.f, 0.f, 0.f, 0.f), dy1 = dy0;
    auto load_z2dy = [&](int64_t tile) {
        const int64_t rw = tile * kTile + r;
        const bool v = tile < n_tiles && rw < a.n;
#pragma unroll
        for (int q = 0; q < kZc; q++)
            z2c[q] = v ? __ldg(reinterpret_cast<const uint4*>(a.Z2 + rw * kHid) + kZc * cg + q)
                       : make_uint4(0u, 0u, 0u, 0u);
        if (cg == 0) {
            dy0 = v ? __ldg(reinterpret_cast<const float4*>(a.dY + rw * kOut)) : make_float4(0.f, 0.f, 0.f, 0.f);
            dy1 = v ? __ldg(reinterpret_cast<const float4*>(a.dY + rw * kOut) + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto load_z1 = [&](int64_t tile) {
        const int64_t rw = tile * kTile + r;
        const bool v = tile < n_tiles && rw < a.n;
#pragma unroll
        for (int q = 0; q < kZc; q++)
            z1c[q] = v ? __ldg(reinterpret_cast<const uint4*>(a.Z1 + rw * kHid) + kZc * cg + q)
                       : make_uint4(0u, 0u, 0u, 0u);
    };

    uint32_t phase = 0, xphase = 0;
    bool ok = true, first = true, x_inflight = false;
    if (tid == 0 && (int64_t)blockIdx.x < n_tiles) { load_x(blockIdx.x); x_inflight = true; }
    load_z2dy(blockIdx.x);
    load_z1(blockIdx.x);
    for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        // (1) the dY split of this sample -> chunks 0 .. 3; dH2 = dY W3
        if (cg == 0) {
            const float dy[kOut] = {dy0.x, dy0.y, dy0.z, dy0.w, dy1.x, dy1.y, dy1.z, dy1.w};
            uint32_t hp[4], mp[4], lp[4];
#pragma unroll
            for (int o = 0; o < kOut; o += 2) {
                const uint32_t h = bf16x2(dy[o], dy[o + 1]);
                const float r0 = dy[o] - bf2f(h & 0xFFFFu), r1 = dy[o + 1] - bf2f(h >> 16);
                const uint32_t m = bf16x2(r0, r1);
                const uint32_t l = bf16x2(r0 - bf2f(m & 0xFFFFu), r1 - bf2f(m >> 16));
                hp[o / 2] = h; mp[o / 2] = m; lp[o / 2] = l;
            }
#pragma unroll
            for (int o = 0; o < kOut; o++) {      // db3: this warp's 32 samples
                float sum = dy[o];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
                if (lane == 0) atomicAdd(s_b3 + o, sum);
            }
            uint8_t* d = sm + kBwdDYs + r * 16;
            *reinterpret_cast<uint4*>(d) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
            *reinterpret_cast<uint4*>(d + kXChunk) = make_uint4(mp[0], mp[1], mp[2], mp[3]);
            *reinterpret_cast<uint4*>(d + 2 * kXChunk) = make_uint4(lp[0], lp[1], lp[2], lp[3]);
            *reinterpret_cast<uint4*>(d + 3 * kXChunk) = make_uint4(0u, 0u, 0u, 0u);
        }
        operands_ready();
        if (tid == 0) {
            tc::fence_after_sync();
            for (int s = 0; s < 2; s++)
                tc::mma_bf16(tbase + kTdH, chunk_kmajor(s_dys, s), tc::kstep_desc(s_w3s, 32, s),
                             tc::idesc_bf16(128, kHid), s > 0);
            tc::mma_commit(bar);
        }
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        // (2) Z2 pass -> H2^T (P1) and dZ2, in two halves of 16 columns
#pragma unroll
        for (int half = 0; half < 2; half++) {
            float dh[16];
            tc::tmem_ld16(tbase + kTdH + lane_off + 32u * cg + 16u * half, dh);
#pragma unroll
            for (int c = 2 * half; c < 2 * half + 2; c++) {
                const uint32_t ws[4] = {z2c[c].x, z2c[c].y, z2c[c].z, z2c[c].w};
                uint32_t hp[4], dz[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int l = 8 * (c - 2 * half) + 2 * u;
                    const uint32_t w = ws[u];
                    bool m0, m1;
                    uint2 e0 = s_tab[btab_slot(w & 0xFFFFu, m0)], e1 = s_tab[btab_slot(w >> 16, m1)];
                    if (m0 | m1) {        // inputs outside the compact table (rare)
                        e0 = make_uint2(__float_as_uint(__ldg(a.w.dgelu_tab + (w & 0xFFFFu))), __ldg(a.w.gelu_tab + (w & 0xFFFFu)));
                        e1 = make_uint2(__float_as_uint(__ldg(a.w.dgelu_tab + (w >> 16))), __ldg(a.w.gelu_tab + (w >> 16)));
                    }
                    hp[u] = (e0.y & 0xFFFFu) | (e1.y << 16);
                    dz[u] = bf16x2(dh[l] * __uint_as_float(e0.x), dh[l + 1] * __uint_as_float(e1.x));
                }
                const uint32_t off = (uint32_t)(4 * cg + c) * kXChunk + r * 16;
                *reinterpret_cast<uint4*>(sm + kBwdP1 + off) = make_uint4(hp[0], hp[1], hp[2], hp[3]);
                *reinterpret_cast<uint4*>(sm + kBwdDZ2 + off) = make_uint4(dz[0], dz[1], dz[2], dz[3]);
            }
        }
        operands_ready();
        // (3) dH1 = dZ2 W2; dW3 parts += H2^T dY split
        if (tid == 0) {
            tc::fence_after_sync();
            for (int s = 0; s < kHid / 16; s++)
                tc::mma_bf16(tbase + kTdH, chunk_kmajor(s_dz2, s), tc::kstep_desc(s_w2t, kHid, s),
                             tc::idesc_bf16(128, kHid), s > 0);
            for (int s = 0; s < kTile / 16; s++)
                tc::mma_bf16(tbase + kTdW3, chunk_mnmajor(s_p1, s), chunk_mnmajor(s_dys, s),
                             tc::idesc_bf16_mn(128, 32, true, true), !first || s > 0);
            tc::mma_commit(bar);
        }
        // (4) Z1 pass, first half (under the MMAs): H1 -> H1_aug^T, gelu'(Z1) kept
        float g1[32];
        {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const uint32_t ws[4] = {z1c[c].x, z1c[c].y, z1c[c].z, z1c[c].w};
                uint32_t hp[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int i = 4 * c + u;
                    const uint32_t w = ws[u];
                    bool m0, m1;
                    uint2 e0 = s_tab[btab_slot(w & 0xFFFFu, m0)], e1 = s_tab[btab_slot(w >> 16, m1)];
                    if (m0 | m1) {
                        e0 = make_uint2(__float_as_uint(__ldg(a.w.dgelu_tab + (w & 0xFFFFu))), __ldg(a.w.gelu_tab + (w & 0xFFFFu)));
                        e1 = make_uint2(__float_as_uint(__ldg(a.w.dgelu_tab + (w >> 16))), __ldg(a.w.gelu_tab + (w >> 16)));
                    }
                    hp[u] = (e0.y & 0xFFFFu) | (e1.y << 16);
                    g1[2 * i] = __uint_as_float(e0.x);
                    g1[2 * i + 1] = __uint_as_float(e1.x);
                }
                *reinterpret_cast<uint4*>(sm + kBwdH1 + (uint32_t)(4 * cg + c) * kXChunk + r * 16) =
                    make_uint4(hp[0], hp[1], hp[2], hp[3]);
            }
        }
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        // (4) second half: dZ1 = bf16(dH1 * gelu'(Z1)) -> dZ1^T (over H2^T, whose GEMM is done)
#pragma unroll
        for (int half = 0; half < 2; half++) {
            float dh[16];
            tc::tmem_ld16(tbase + kTdH + lane_off + 32u * cg + 16u * half, dh);
#pragma unroll
            for (int c = 0; c < 2; c++) {
                uint32_t v[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int i = 8 * half + 4 * c + u, l = 8 * c + 2 * u;
                    v[u] = bf16x2(dh[l] * g1[2 * i], dh[l + 1] * g1[2 * i + 1]);
                }
                *reinterpret_cast<uint4*>(sm + kBwdP1 + (uint32_t)(4 * cg + 2 * half + c) * kXChunk + r * 16) =
                    make_uint4(v[0], v[1], v[2], v[3]);
            }
        }
        // X of this tile (TMA): the ones column 196 of X_aug (zero-filled by the copy)
        const bool x_ok = wait_all(xbar, xphase, a.wait_polls);
        if (tid == 0) x_inflight = false;     // on a timeout wait_all has waited for the copy (bounded)
        if (!(ok = x_ok)) break;
        if (cg == 0) *reinterpret_cast<uint16_t*>(sm + kBwdX + (kIn / 8) * kXChunk + r * 16 + (kIn % 8) * 2) = 0x3F80u;
        operands_ready();
        // (5) dW2_aug += dZ2^T H1_aug; dW1_aug += dZ1^T X_aug
        if (tid == 0) {
            tc::fence_after_sync();
            for (int s = 0; s < kTile / 16; s++)
                tc::mma_bf16(tbase + kTdW2, chunk_mnmajor(s_dz2, s), chunk_mnmajor(s_h1, s),
                             tc::idesc_bf16_mn(128, kK2, true, true), !first || s > 0);
            for (int s = 0; s < kTile / 16; s++)
                tc::mma_bf16(tbase + kTdW1, chunk_mnmajor(s_p1, s), chunk_mnmajor(s_x, s),
                             tc::idesc_bf16_mn(128, kK1, true, true), !first || s > 0);
            tc::mma_commit(bar);
        }
        load_z2dy(t + gridDim.x);
        load_z1(t + gridDim.x);
        if (!(ok = wait_all(bar, phase, a.wait_polls))) break;
        first = false;
        if (tid == 0 && t + gridDim.x < n_tiles) { load_x(t + gridDim.x); x_inflight = true; }
    }
    if (tid == 0) {
        if (!ok) set_status(a.status, GS_ERR_TIMEOUT);
        // nothing in flight when the CTA frees its tensor memory (bounded waits)
        tc::mma_commit(dbar);
        tc::mbar_wait(dbar, 0, kDrainPolls);
        if (x_inflight) tc::mbar_wait(xbar, xphase, kDrainPolls);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (ok && !first) {
        // accumulated weight gradients of this CTA -> global (row r of dW1_aug, dW2_aug, dW3 parts)
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
        if (cg == 0) {
            float v[32];
            tc::tmem_ld32(tbase + kTdW3 + lane_off, v);
#pragma unroll
            for (int o = 0; o < kOut; o++) atomicAdd(a.g.W3 + o * kHid + r, (v[o] + v[8 + o]) + v[16 + o]);
            if (tid < kOut) atomicAdd(a.g.b3 + tid, s_b3[tid]);
        }
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

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query
// (no link-time dependency on the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// X as a 2-D tensor of 196 BF16 columns (the inputs; the row stride is 208
// values) and n rows, copied in boxes of 8 columns x 128 rows (unswizzled) or
// 64 columns x 128 rows (128-byte swizzle); columns past 195 and rows past n
// arrive as zeros.
static cudaError_t x_tensor_map(CUtensorMap* m, const uint16_t* X, int64_t n, bool swizzled = false) {
    if (n > (int64_t)INT_MAX - kTile) return cudaErrorInvalidValue;    // TMA row coordinates are 32-bit
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (encode == nullptr) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)kIn, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)kK1 * 2};
    const cuuint32_t box[2] = {swizzled ? 64u : 8u, (cuuint32_t)kTile};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swizzled ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

cudaError_t launch_mlp_fwd(const gs_mlp_packed& w, const uint16_t* X, int64_t n, float* Y, uint16_t* Z1,
                           uint16_t* Z2, const float* T, float* dY, float* loss, float loss_scale, int* status,
                           cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    CUtensorMap xmap_sw, xmap;
    cudaError_t e = x_tensor_map(&xmap_sw, X, n, true);
    if (e == cudaSuccess) e = x_tensor_map(&xmap, X, n);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
    MlpFwdArgs a{w, n, Y, Z1, Z2, T, dY, loss, loss_scale, status, g_wait_polls.load()};
    k_mlp_fwd<<<grid, kFwdThreads2, kFwdSmem, s>>>(xmap_sw, xmap, a);
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
    CUtensorMap xmap;
    cudaError_t e = x_tensor_map(&xmap, X, n);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
    MlpBwdArgs a{w, Z1, Z2, dY, n, g, status, g_wait_polls.load()};
    k_mlp_bwd<<<grid, kEpiThreads, kBwdSmem, s>>>(xmap, a);
    return cudaGetLastError();
}

}  // namespace gs
