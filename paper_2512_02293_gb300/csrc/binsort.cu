// binsort.cu -- tile binning and depth sort of the projected splats.
//
//   1. k_scan_reduce   : per-block sums of tiles_touched (256 entries a block)
//   2. k_scan_blocks   : exclusive scan of the block sums (one CTA), M, overflow flag
//   3. k_duplicate     : block-local scan + emission of one key per (entry, tile):
//                        key = (global tile << 32) | bits(float z), value = entry.
//                        Entries covering many tiles are emitted by their whole
//                        warp, so a large splat near the camera does not leave
//                        one thread writing hundreds of keys alone.
//   4. LSD radix sort  : passes of up to 9-bit digits over the 31 depth bits and
//                        the tile bits; each pass is k_radix_hist (per-block
//                        digit counts) -> k_radix_scan (one CTA per digit) ->
//                        k_radix_scatter (stable: per-warp ranks from match_any,
//                        per-digit warp prefixes in shared memory).  Blocks hold
//                        1024 keys, so even a few hundred thousand keys give
//                        several blocks per SM and short serial chains.
//   5. k_tile_ranges   : [start, end) of every tile in the sorted list
//
// The key's bit 31 (the sign of z > 0) is always 0, so the sort runs over the
// 31 depth bits and the tile bits only.  Kernels never read M on the host: grids
// are sized for the key capacity and blocks past M return at once, which keeps
// the whole sequence free of host synchronisation (capturable in a CUDA graph).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 1;
constexpr int kScanBlock = kScanThreads * kScanItems;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 4;
constexpr int kSortBlock = kSortThreads * kSortItems;
constexpr int kMaxDigitBits = 9;
constexpr int kRadixMax = 1 << kMaxDigitBits;            // buckets of the widest digit
constexpr int kDigitsPerThread = kRadixMax / kSortThreads;
constexpr int kBigEntry = 8;                             // keys an entry emits by itself

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive block scan of one value per thread (blockDim.x == kThreads).
template <int kThreads>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* total, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kThreads / 32 ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kThreads / 32) s_warp[lane] = wi - w;   // exclusive warp offsets
        if (lane == kThreads / 32 - 1) s_warp[kThreads / 32] = wi;
    }
    __syncthreads();
    uint32_t r = s_warp[warp] + inc - x;
    *total = s_warp[kThreads / 32];
    __syncthreads();
    return r;
}

// Also zeroes the tile ranges (k_tile_ranges writes only the tiles that have keys).
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ tt, int64_t E,
                                                             uint32_t* __restrict__ block_sums,
                                                             uint32_t* __restrict__ ranges, int64_t n_range_words) {
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    pdl_enter();
    for (int64_t k = (int64_t)blockIdx.x * kScanThreads + threadIdx.x; k < n_range_words;
         k += (int64_t)gridDim.x * kScanThreads)
        ranges[k] = 0u;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        const int64_t e = (int64_t)blockIdx.x * kScanBlock + (int64_t)k * kScanThreads + threadIdx.x;
        if (e < E) s += tt[e];
    }
    uint32_t total;
    block_exclusive_scan<kScanThreads>(s, &total, s_warp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// One CTA: exclusive scan of nb block sums in place; M = total.
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t* __restrict__ block_sums, int nb,
                                                      uint32_t* __restrict__ num_keys, int64_t capacity,
                                                      int32_t* __restrict__ status) {
    __shared__ uint32_t s_warp[1024 / 32 + 1];
    pdl_enter();
    const int chunk = (nb + 1023) / 1024;
    const int lo = threadIdx.x * chunk;
    uint32_t s = 0;
    for (int k = 0; k < chunk; k++)
        if (lo + k < nb) s += block_sums[lo + k];
    uint32_t total;
    uint32_t run = block_exclusive_scan<1024>(s, &total, s_warp);
    for (int k = 0; k < chunk; k++) {
        if (lo + k < nb) {
            uint32_t v = block_sums[lo + k];
            block_sums[lo + k] = run;
            run += v;
        }
    }
    if (threadIdx.x == 0) {
        *num_keys = total;
        if ((int64_t)total > capacity) *status = GS_ERR_CAPACITY;
    }
}

// Emission of the keys of one entry: key = (tile << 32) | z bits, value =
// entry, written at [off, off + cnt) in row-major order over its rectangle.
__device__ __forceinline__ void emit_keys(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, int64_t capacity,
                                          uint32_t off, int k0, int k1, int kstep, int4 r, int tb, int tx,
                                          uint32_t zbits, uint32_t e) {
    const int w = r.z - r.x;
    for (int k = k0; k < k1; k += kstep) {
        const int64_t pos = (int64_t)off + k;
        if (pos < capacity) {
            const uint64_t g = (uint64_t)(tb + (r.y + k / w) * tx + r.x + k % w);
            keys[pos] = (g << 32) | (uint64_t)zbits;
            vals[pos] = e;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_duplicate(const uint32_t* __restrict__ tt, const int4* __restrict__ rect,
                                                           const float4* __restrict__ rgbd, int64_t E, int64_t n,
                                                           const uint32_t* __restrict__ block_offsets, Views views,
                                                           int64_t capacity, uint64_t* __restrict__ keys,
                                                           uint32_t* __restrict__ vals) {
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    pdl_enter();
    const int lane = threadIdx.x & 31;
    uint32_t carry = block_offsets[blockIdx.x];
    for (int k = 0; k < kScanItems; k++) {
        const int64_t e = (int64_t)blockIdx.x * kScanBlock + (int64_t)k * kScanThreads + threadIdx.x;
        const uint32_t cnt = e < E ? tt[e] : 0u;
        uint32_t total;
        const uint32_t off = carry + block_exclusive_scan<kScanThreads>(cnt, &total, s_warp);
        carry += total;
        int4 r = make_int4(0, 0, 1, 1);
        int tb = 0, tx = 1;
        uint32_t zbits = 0;
        if (cnt > 0) {
            const int v = (int)(e / n);
            r = rect[e];
            zbits = __float_as_uint(rgbd[e].w);
            tb = views.v[v].tile_base;
            tx = views.v[v].tiles_x;
        }
        if (cnt > 0 && cnt <= (uint32_t)kBigEntry)
            emit_keys(keys, vals, capacity, off, 0, (int)cnt, 1, r, tb, tx, zbits, (uint32_t)e);
        uint32_t big = __ballot_sync(0xffffffffu, cnt > (uint32_t)kBigEntry);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            int4 br;
            br.x = __shfl_sync(0xffffffffu, r.x, src);
            br.y = __shfl_sync(0xffffffffu, r.y, src);
            br.z = __shfl_sync(0xffffffffu, r.z, src);
            br.w = __shfl_sync(0xffffffffu, r.w, src);
            const uint32_t boff = __shfl_sync(0xffffffffu, off, src);
            const int bcnt = (int)__shfl_sync(0xffffffffu, cnt, src);
            const int btb = __shfl_sync(0xffffffffu, tb, src), btx = __shfl_sync(0xffffffffu, tx, src);
            const uint32_t bz = __shfl_sync(0xffffffffu, zbits, src);
            const uint32_t be = (uint32_t)__shfl_sync(0xffffffffu, (uint32_t)e, src);
            emit_keys(keys, vals, capacity, boff, lane, bcnt, 32, br, btb, btx, bz, be);
        }
    }
}

// digit of the compacted key ((tile << 31) | z bits) at [shift, shift + bits)
__device__ __forceinline__ uint32_t key_digit(uint64_t key, int shift, uint32_t mask) {
    const uint64_t c = ((key >> 32) << 31) | (key & 0x7fffffffull);
    return (uint32_t)(c >> shift) & mask;
}

__device__ __forceinline__ int64_t sort_count(const uint32_t* num_keys, int64_t capacity) {
    const int64_t m = (int64_t)*num_keys;
    return m < capacity ? m : capacity;
}

// Per-block digit counts, stored digit-major: counts[d * nb + b].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys,
                                                            const uint32_t* __restrict__ num_keys, int64_t capacity,
                                                            int shift, int bits, uint32_t* __restrict__ counts) {
    pdl_enter();
    const int64_t M = sort_count(num_keys, capacity);
    const int nb = (int)ceil_div(M, kSortBlock);
    if ((int)blockIdx.x >= nb) return;
    __shared__ uint32_t h[kSortWarps][kRadixMax];
    const int radix = 1 << bits;
    for (int k = threadIdx.x; k < kSortWarps * kRadixMax; k += kSortThreads) (&h[0][0])[k] = 0u;
    __syncthreads();
    const uint32_t mask = (uint32_t)radix - 1u;
    const int warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
    uint64_t key[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t idx = base + (int64_t)r * kSortThreads + threadIdx.x;
        key[r] = idx < M ? keys[idx] : 0ull;
    }
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t idx = base + (int64_t)r * kSortThreads + threadIdx.x;
        if (idx < M) atomicAdd(&h[warp][key_digit(key[r], shift, mask)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < radix; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) s += h[w][d];
        counts[(int64_t)d * nb + blockIdx.x] = s;
    }
}

// One warp per digit: exclusive scan (in place) of that digit's per-block
// counts counts[d * nb .. d * nb + nb) with shuffle scans over chunks of 32 and
// a running carry; the digit's total goes to digit_total[d].
constexpr int kDigitScanThreads = 256;
constexpr int kDigitScanWarps = kDigitScanThreads / 32;

__global__ void __launch_bounds__(kDigitScanThreads) k_radix_scan(uint32_t* __restrict__ counts,
                                                                 uint32_t* __restrict__ digit_total,
                                                                 const uint32_t* __restrict__ num_keys,
                                                                 int64_t capacity, int radix) {
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * kDigitScanWarps + (threadIdx.x >> 5);
    if (d >= radix) return;
    const int64_t M = sort_count(num_keys, capacity);
    const int nb = (int)ceil_div(M, kSortBlock);
    uint32_t* c = counts + (int64_t)d * nb;
    uint32_t carry = 0;
    for (int i0 = 0; i0 < nb; i0 += 32) {
        const int i = i0 + lane;
        const uint32_t x = i < nb ? c[i] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (i < nb) c[i] = carry + inc - x;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) digit_total[d] = carry;
}

// Stable scatter.  Each round places 256 consecutive keys: ranks inside a warp
// come from match_any, the offsets of earlier warps from a per-digit prefix in
// shared memory, and s_base carries the digit's running position across rounds.
// Counts are double-buffered so that a round needs two barriers.  Thread t owns
// digits t and t + 256 of the bookkeeping.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               const uint32_t* __restrict__ offsets,
                                                               const uint32_t* __restrict__ digit_total,
                                                               const uint32_t* __restrict__ num_keys,
                                                               int64_t capacity, int shift, int bits) {
    pdl_enter();
    const int64_t M = sort_count(num_keys, capacity);
    const int nb = (int)ceil_div(M, kSortBlock);
    if ((int)blockIdx.x >= nb) return;
    __shared__ uint32_t s_base[kRadixMax];
    __shared__ uint32_t s_rbase[kRadixMax];
    __shared__ uint32_t s_cnt[2][kSortWarps][kRadixMax];
    __shared__ uint32_t s_warp[kSortThreads / 32 + 1];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int radix = 1 << bits;
    const uint32_t mask = (uint32_t)radix - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortBlock;
    uint64_t key[kSortItems];
    uint32_t val[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int64_t idx = base + (int64_t)r * kSortThreads + tid;
        key[r] = idx < M ? kin[idx] : 0ull;
        val[r] = idx < M ? vin[idx] : 0u;
    }
    // digit base = keys of smaller digits in the whole list + this digit's keys in earlier blocks
    uint32_t dt[kDigitsPerThread];
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kDigitsPerThread; q++) {
        const int d = tid * kDigitsPerThread + q;
        dt[q] = d < radix ? digit_total[d] : 0u;
        sum += dt[q];
    }
    uint32_t tot;
    uint32_t run0 = block_exclusive_scan<kSortThreads>(sum, &tot, s_warp);
#pragma unroll
    for (int q = 0; q < kDigitsPerThread; q++) {
        const int d = tid * kDigitsPerThread + q;
        if (d < radix) s_base[d] = run0 + offsets[(int64_t)d * nb + blockIdx.x];
        run0 += dt[q];
    }
    for (int k = tid; k < 2 * kSortWarps * kRadixMax; k += kSortThreads) (&s_cnt[0][0][0])[k] = 0u;
    __syncthreads();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < kSortItems; r++) {
        const int buf = r & 1;
        const int64_t idx = base + (int64_t)r * kSortThreads + tid;
        const bool valid = idx < M;
        const uint32_t d = valid ? key_digit(key[r], shift, mask) : (uint32_t)kRadixMax;   // sentinel
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) s_cnt[buf][warp][d] = __popc(peers);
        __syncthreads();
        for (int dd = tid; dd < radix; dd += kSortThreads) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kSortWarps; w++) {
                const uint32_t c = s_cnt[buf][w][dd];
                s_cnt[buf][w][dd] = run;
                run += c;
                s_cnt[buf ^ 1][w][dd] = 0u;
            }
            s_rbase[dd] = s_base[dd];
            s_base[dd] += run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s_rbase[d] + s_cnt[buf][warp][d] + rank;
            kout[pos] = key[r];
            vout[pos] = val[r];
        }
    }
}

__global__ void k_tile_ranges(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ num_keys,
                              int64_t capacity, uint2* __restrict__ ranges) {
    pdl_enter();
    const int64_t M = sort_count(num_keys, capacity);
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= M) return;
    const uint32_t t = (uint32_t)(keys[s] >> 32);
    if (s == 0 || (uint32_t)(keys[s - 1] >> 32) != t) ranges[t].x = (uint32_t)s;
    if (s == M - 1 || (uint32_t)(keys[s + 1] >> 32) != t) ranges[t].y = (uint32_t)(s + 1);
}

}  // namespace

SortPlan make_sort_plan(int64_t key_capacity, int32_t total_tiles) {
    SortPlan p;
    p.capacity = key_capacity;
    p.total_tiles = total_tiles;
    return p;
}

// Workspace layout of launch_bin_sort (offsets in bytes, 256-byte aligned):
//   block sums   : ceil(E / kScanBlock) u32
//   counts       : kRadixMax * ceil(capacity / kSortBlock) u32
//   digit totals : kRadixMax u32
//   keys (alt)   : capacity u64
//   vals (alt)   : capacity u32
static size_t ws_block_sums(int64_t E) { return align_up(sizeof(uint32_t) * (size_t)(ceil_div(E, kScanBlock) + 1), 256); }
static size_t ws_counts(int64_t cap) {
    return align_up(sizeof(uint32_t) * (size_t)kRadixMax * (size_t)(ceil_div(cap, kSortBlock) + 1), 256);
}

size_t bin_sort_workspace(int64_t n_entries, int64_t capacity, int32_t total_tiles) {
    (void)total_tiles;
    return ws_block_sums(n_entries) + ws_counts(capacity) + align_up(sizeof(uint32_t) * kRadixMax, 256) +
           align_up(sizeof(uint64_t) * (size_t)capacity, 256) + align_up(sizeof(uint32_t) * (size_t)capacity, 256);
}

cudaError_t launch_bin_sort(const gs_projected& pr, int64_t n, const Views& views, const SortPlan& plan,
                            const gs_bins& bins, void* ws, cudaStream_t s) {
    const int64_t E = n * views.n;
    const int64_t cap = plan.capacity;
    char* p = static_cast<char*>(ws);
    uint32_t* block_sums = reinterpret_cast<uint32_t*>(p);
    p += ws_block_sums(E);
    uint32_t* counts = reinterpret_cast<uint32_t*>(p);
    p += ws_counts(cap);
    uint32_t* digit_total = reinterpret_cast<uint32_t*>(p);
    p += align_up(sizeof(uint32_t) * kRadixMax, 256);
    uint64_t* keys_alt = reinterpret_cast<uint64_t*>(p);
    p += align_up(sizeof(uint64_t) * (size_t)cap, 256);
    uint32_t* vals_alt = reinterpret_cast<uint32_t*>(p);

    cudaError_t err = cudaSuccess;
    if (E == 0) {
        err = cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)views.total_tiles, s);
        if (err != cudaSuccess) return err;
        return cudaMemsetAsync(bins.num_keys, 0, sizeof(uint32_t), s);
    }
    // passes over the compacted key (tile << 31 | z bits), digits of at most 9 bits
    int tile_bits = 0;
    while ((1ll << tile_bits) < (int64_t)plan.total_tiles) tile_bits++;
    const int bits = 31 + tile_bits;
    const int n_passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    int width[8], shift[8];
    for (int k = 0, sh = 0; k < n_passes; k++) {
        width[k] = bits / n_passes + (k < bits % n_passes ? 1 : 0);
        shift[k] = sh;
        sh += width[k];
    }
    const int nb_scan = (int)ceil_div(E, kScanBlock);
    err = launch_pdl(k_scan_reduce, nb_scan, kScanThreads, 0, s, pr.tiles_touched, E, block_sums, bins.ranges,
                     2 * (int64_t)views.total_tiles);
    if (err == cudaSuccess)
        err = launch_pdl(k_scan_blocks, 1, 1024, 0, s, block_sums, nb_scan, bins.num_keys, cap, bins.status);
    if (err != cudaSuccess) return err;
    // The duplicated list goes into the buffer that makes the last pass land in bins.keys.
    uint64_t* k0 = (n_passes % 2 == 0) ? bins.keys : keys_alt;
    uint32_t* v0 = (n_passes % 2 == 0) ? bins.vals : vals_alt;
    uint64_t* k1 = (n_passes % 2 == 0) ? keys_alt : bins.keys;
    uint32_t* v1 = (n_passes % 2 == 0) ? vals_alt : bins.vals;
    err = launch_pdl(k_duplicate, nb_scan, kScanThreads, 0, s, pr.tiles_touched,
                     reinterpret_cast<const int4*>(pr.rect), reinterpret_cast<const float4*>(pr.rgbd), E, n,
                     block_sums, views, cap, k0, v0);
    if (err != cudaSuccess) return err;
    const int nb_sort = (int)ceil_div(cap, kSortBlock);
    for (int pass = 0; pass < n_passes; pass++) {
        err = launch_pdl(k_radix_hist, nb_sort, kSortThreads, 0, s, k0, bins.num_keys, cap, shift[pass], width[pass],
                         counts);
        const int radix = 1 << width[pass];
        if (err == cudaSuccess)
            err = launch_pdl(k_radix_scan, (unsigned)ceil_div(radix, kDigitScanWarps), kDigitScanThreads, 0, s, counts,
                             digit_total, bins.num_keys, cap, radix);
        if (err == cudaSuccess)
            err = launch_pdl(k_radix_scatter, nb_sort, kSortThreads, 0, s, k0, v0, k1, v1, counts, digit_total,
                             bins.num_keys, cap, shift[pass], width[pass]);
        if (err != cudaSuccess) return err;
        uint64_t* tk = k0; k0 = k1; k1 = tk;
        uint32_t* tv = v0; v0 = v1; v1 = tv;
    }
    const int nb_rng = (int)ceil_div(cap, 256);
    err = launch_pdl(k_tile_ranges, nb_rng, 256, 0, s, bins.keys, bins.num_keys, cap,
                     reinterpret_cast<uint2*>(bins.ranges));
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

}  // namespace gs
