// binsort.cu -- tile binning and depth sort of the projected splats.
//
// The paper does not describe this step (Sec. 3.3 renders with the 3D Gaussian
// splatting rasteriser it builds on, whose compositing walks each tile's splats
// front to back).  The result is the list of keys (global tile << 32) | bits(z),
// one per (entry, covered tile), in ascending key order with equal keys in entry
// order, and each tile's [start, end) in it.  Since (tile, z bits, entry) is
// unique, the order is unique, so it does not matter how it is reached:
//
//   1. k_bin_zero    : zero the per-tile key counts (workspace)
//   2. k_bin_count   : one atomic increment of a tile's count per (entry, covered
//                      tile); entries covering many tiles are counted by their
//                      whole warp.  Each tile has kStripes counters (the lane
//                      picks one), so that the thousands of keys of a deep tile
//                      do not queue on one address
//   3. k_bin_stripes : per tile (one warp), the exclusive scan of its stripe counters (each
//                      becomes its stripe's offset inside the tile) and the total
//   4. k_bin_offsets : one CTA: exclusive scan of the tile totals in coalesced
//                      rounds -> ranges [start, end) of every tile (clamped to
//                      the key capacity), M, the overflow flag; the totals
//                      become the tiles' starts
//   5. k_bin_scatter : every (entry, tile) pair claims a slot of its tile's
//                      segment with an atomic on its stripe's cursor and writes
//                      the composite (z bits << 32) | entry there (in no fixed
//                      order)
//   6. k_tile_sort   : sorts every tile's segment by the composite, i.e. by
//                      (z, entry), and writes key = (tile << 32) | z bits and
//                      value = entry: a CTA of 1024 threads sorts one tile of more
//                      than kSmallCap keys (a bitonic network in shared memory up
//                      to kSegCap keys, a stable LSD radix sort through the
//                      workspace's second key buffer above that) or, split into
//                      four groups of 256 threads with their own barriers, four
//                      smaller tiles at once.
//
// z > near > 0, so the fp32 bits of z are positive and ordered like z.  Kernels
// never read M on the host: grids are sized by entries and tiles, every write
// is bounded by the key capacity, so the sequence is free of host
// synchronisation (capturable in a CUDA graph).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kBinThreads = 256;
constexpr int kBigEntry = 8;                             // keys an entry handles by itself
constexpr int kScanThreads = 1024;
constexpr int kSortThreads = 1024;                       // a tile-sort CTA
constexpr int kGroup = 256;                              // threads of a small-tile group
constexpr int kGroups = kSortThreads / kGroup;
constexpr int kSmallCap = 2 * kGroup;                    // keys a group sorts (one pair per thread)
constexpr int kSegCap = 4 * kSortThreads;                // keys a CTA sorts in shared memory
constexpr int kRadixThreads = 256;                       // threads that work in the radix path
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kStripes = 32;                             // counters per tile (stripe = lane)

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

__global__ void __launch_bounds__(kBinThreads) k_bin_zero(uint32_t* __restrict__ cnt, int64_t words,
                                                         uint32_t* __restrict__ sort_ctrs) {
    pdl_enter();
    if (blockIdx.x == 0 && threadIdx.x < 4) sort_ctrs[threadIdx.x] = 0u;
    for (int64_t t = (int64_t)blockIdx.x * kBinThreads + threadIdx.x; t < words; t += (int64_t)gridDim.x * kBinThreads)
        cnt[t] = 0u;
}

// Global tile of the k-th covered tile (row-major over the rectangle r) of an
// entry of a view with tile base tb and tx tiles per row.
__device__ __forceinline__ uint32_t covered_tile(int4 r, int tb, int tx, int k) {
    const int w = r.z - r.x;
    return (uint32_t)(tb + (r.y + k / w) * tx + r.x + k % w);
}

// The culling test of the rasterisers (0.99 alpha_min) at tile granularity, for
// one entry: whether its splat can reach 0.99 alpha_min anywhere in a tile's box
// of pixel centres.  For a negative-definite power the maximum over the box lies
// on the two edges that face the mean (0 with the mean inside), each maximised at
// its clamped stationary point, as for the block masks; it is compared with
// log2(0.99 alpha_min / o) - 0.004 against rounding.  An opacity below 0.99
// alpha_min reaches no tile; any other conic keeps every tile.  Every rounding
// step is an explicit intrinsic, so that the count and the scatter, which both
// evaluate the test, take the same decisions whatever the compiler contracts.
struct TileCull {
    float mx, my, qa, qb, qc, rx, ry, L;
    int mode;                                  // 0: test, 1: every tile, 2: no tile
};

__device__ __forceinline__ TileCull tile_cull_of(const float2 m, const float4 c, float amin) {
    TileCull t;
    float4 q;
    scale_conic(c.x, c.y, c.z, &q.x, &q.y, &q.z);
    q.w = c.w;
    const float thr = __fmul_rn(0.99f, amin);
    t.mx = m.x; t.my = m.y; t.qa = q.x; t.qb = q.y; t.qc = q.z;
    t.rx = t.ry = t.L = 0.f;
    if (q.w < thr) {
        t.mode = 2;
    } else if (!(q.x < 0.f && q.z < 0.f && __fsub_rn(__fmul_rn(__fmul_rn(4.f, q.x), q.z), __fmul_rn(q.y, q.y)) > 0.f)) {
        t.mode = 1;
    } else {
        t.mode = 0;
        t.L = __fsub_rn(__log2f(__fdividef(thr, q.w)), 0.004f);
        t.rx = __fdividef(-q.y, __fmul_rn(2.f, q.z));
        t.ry = __fdividef(-q.y, __fmul_rn(2.f, q.x));
    }
    return t;
}

// Tile (tx, ty) of T x T pixels of the entry's view.
__device__ __forceinline__ bool tile_reached(const TileCull& t, int tx, int ty, int T) {
    if (t.mode != 0) return t.mode == 1;
    const float dx0 = __fsub_rn(__fadd_rn((float)(tx * T), 0.5f), t.mx), dx1 = __fadd_rn(dx0, (float)(T - 1));
    const float dy0 = __fsub_rn(__fadd_rn((float)(ty * T), 0.5f), t.my), dy1 = __fadd_rn(dy0, (float)(T - 1));
    const float vx = fminf(fmaxf(0.f, dx0), dx1), vy = fminf(fmaxf(0.f, dy0), dy1);
    const float sy = fminf(fmaxf(__fmul_rn(t.rx, vx), dy0), dy1), sx = fminf(fmaxf(__fmul_rn(t.ry, vy), dx0), dx1);
    const float pv = __fmaf_rn(vx, __fmaf_rn(t.qa, vx, __fmul_rn(t.qb, sy)), __fmul_rn(__fmul_rn(t.qc, sy), sy));
    const float ph = __fmaf_rn(vy, __fmaf_rn(t.qc, vy, __fmul_rn(t.qb, sx)), __fmul_rn(__fmul_rn(t.qa, sx), sx));
    return fmaxf(pv, ph) >= t.L;
}

// Operands of the tile culling (kCull): projected means and conics, tile size.
struct CullArgs {
    const float2* xy;
    const float4* conic_o;
    int T;
    float amin;
};

// Calls f(tile, entry, z bits) once for every (entry, covered tile) pair of this
// thread's entry e (with kCull, only for the tiles the entry's splat can reach);
// entries with more than kBigEntry tiles are enumerated by the whole warp (32
// tiles at a time), so one large splat near the camera does not leave a single
// thread looping over hundreds of tiles.  With kClaim, f has claim(tile) -> slot
// and write(slot, entry, z bits), and a small entry's claims are all in flight
// before its writes.  The count and the scatter take the same decisions: the
// same function of the same operands.
template <bool kClaim = false, bool kCull = false, typename F>
__device__ __forceinline__ void for_each_key(const uint32_t* __restrict__ tt, const int4* __restrict__ rect,
                                             const float4* __restrict__ rgbd, int64_t E, int64_t n,
                                             const Views& views, const CullArgs& ca, F f) {
    const int lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    const uint32_t cnt = e < E ? tt[e] : 0u;
    int4 r = make_int4(0, 0, 1, 1);
    int tb = 0, tx = 1;
    uint32_t zbits = 0;
    TileCull tc{};
    if (cnt > 0) {
        const int v = (int)(e / n);
        r = rect[e];
        tb = views.v[v].tile_base;
        tx = views.v[v].tiles_x;
        if (rgbd != nullptr) zbits = __float_as_uint(rgbd[e].w);
        if constexpr (kCull)
            if (cnt <= (uint32_t)kBigEntry) tc = tile_cull_of(ca.xy[e], ca.conic_o[e], ca.amin);
    }
    auto keep = [&](const TileCull& t, const int4& rr, int k) -> bool {
        if constexpr (kCull) {
            const int w = rr.z - rr.x;
            return tile_reached(t, rr.x + k % w, rr.y + k / w, ca.T);
        } else {
            return true;
        }
    };
    const bool small = cnt > 0 && cnt <= (uint32_t)kBigEntry;
    if constexpr (kClaim) {
        // two phases for the scatter: all of this entry's slot claims (atomics) in
        // flight together, then the writes
        uint32_t pos[kBigEntry];
        uint32_t claimed = 0;
#pragma unroll
        for (int k = 0; k < kBigEntry; k++)
            if (small && k < (int)cnt && keep(tc, r, k)) {
                pos[k] = f.claim(covered_tile(r, tb, tx, k));
                claimed |= 1u << k;
            }
#pragma unroll
        for (int k = 0; k < kBigEntry; k++)
            if ((claimed >> k) & 1u) f.write(pos[k], (uint32_t)e, zbits);
    } else if (small) {
        for (int k = 0; k < (int)cnt; k++)
            if (keep(tc, r, k)) f(covered_tile(r, tb, tx, k), (uint32_t)e, zbits);
    }
    uint32_t big = __ballot_sync(0xffffffffu, cnt > (uint32_t)kBigEntry);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        int4 br;
        br.x = __shfl_sync(0xffffffffu, r.x, src);
        br.y = __shfl_sync(0xffffffffu, r.y, src);
        br.z = __shfl_sync(0xffffffffu, r.z, src);
        br.w = __shfl_sync(0xffffffffu, r.w, src);
        const int bcnt = (int)__shfl_sync(0xffffffffu, cnt, src);
        const int btb = __shfl_sync(0xffffffffu, tb, src), btx = __shfl_sync(0xffffffffu, tx, src);
        const uint32_t bz = __shfl_sync(0xffffffffu, zbits, src);
        const uint32_t be = (uint32_t)__shfl_sync(0xffffffffu, (uint32_t)e, src);
        TileCull btc{};
        if constexpr (kCull) btc = tile_cull_of(ca.xy[be], ca.conic_o[be], ca.amin);   // the same on every lane
        for (int k = lane; k < bcnt; k += 32) {
            if (!keep(btc, br, k)) continue;
            if constexpr (kClaim) f.write(f.claim(covered_tile(br, btb, btx, k)), be, bz);
            else f(covered_tile(br, btb, btx, k), be, bz);
        }
    }
}

template <bool kCull>
__global__ void __launch_bounds__(kBinThreads) k_bin_count(const uint32_t* __restrict__ tt, const int4* __restrict__ rect,
                                                          int64_t E, int64_t n, Views views,
                                                          uint32_t* __restrict__ cnt, CullArgs ca) {
    pdl_enter();
    uint32_t* mine = cnt + (size_t)(threadIdx.x & 31) * (size_t)views.total_tiles;     // this lane's stripe
    for_each_key<false, kCull>(tt, rect, nullptr, E, n, views, ca,
                               [&](uint32_t g, uint32_t, uint32_t) { atomicAdd(mine + g, 1u); });
}

// Per tile (one warp, lane = stripe): each stripe counter becomes the exclusive
// prefix of the stripes before it (its offset inside the tile); total[t] = the
// tile's key count.
__global__ void __launch_bounds__(kBinThreads) k_bin_stripes(uint32_t* __restrict__ cnt, int total_tiles,
                                                            uint32_t* __restrict__ total) {
    pdl_enter();
    const int t = (int)(((int64_t)blockIdx.x * kBinThreads + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (t >= total_tiles) return;                    // warp-uniform
    uint32_t* c = cnt + (size_t)lane * total_tiles + t;
    const uint32_t v = *c;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    *c = inc - v;
    if (lane == 31) total[t] = inc;
}

// One CTA: ranges[t] = [start, start + count) of every tile with keys (both
// clamped to the capacity, so that no reader of the ranges leaves the key
// buffers after an overflow) and (0, 0) for an empty tile, cnt[t] = start (the
// tile's first slot for the scatter), M, the overflow flag; and the work lists
// of the per-tile sort: the tiles of more than kSmallCap keys (sorted by a whole
// CTA) and the others with keys (sorted by a group), in no particular order,
// with their lengths in sort_ctrs[0], sort_ctrs[1].
__global__ void __launch_bounds__(kScanThreads) k_bin_offsets(uint32_t* __restrict__ cnt, int total_tiles,
                                                             uint2* __restrict__ ranges,
                                                             uint32_t* __restrict__ num_keys, int64_t capacity,
                                                             int32_t* __restrict__ status,
                                                             uint32_t* __restrict__ big_list,
                                                             uint32_t* __restrict__ small_list,
                                                             uint32_t* __restrict__ sort_ctrs) {
    __shared__ uint32_t s_warp[kScanThreads / 32 + 1];
    __shared__ uint32_t s_nbig, s_nsmall;
    pdl_enter();
    if (threadIdx.x == 0) s_nbig = s_nsmall = 0u;
    const int lane = threadIdx.x & 31;
    const uint32_t cap = (uint32_t)capacity;     // < 2^32 (host check)
    uint32_t carry = 0;
    for (int base = 0; base < total_tiles; base += kScanThreads) {
        const int t = base + (int)threadIdx.x;
        const uint32_t c = t < total_tiles ? cnt[t] : 0u;
        uint32_t total;
        const uint32_t st = carry + block_exclusive_scan<kScanThreads>(c, &total, s_warp);
        uint32_t len = 0;                                   // the tile's length as the sort sees it
        if (t < total_tiles) {
            const uint2 rg = c > 0 ? make_uint2(min(st, cap), min(st + c, cap)) : make_uint2(0u, 0u);   // (0, 0): empty
            ranges[t] = rg;
            cnt[t] = st;
            len = rg.y - rg.x;
        }
        carry += total;
        const bool big = len > (uint32_t)kSmallCap, small = len > 0 && !big;
        const uint32_t bb = __ballot_sync(0xffffffffu, big), sb = __ballot_sync(0xffffffffu, small);
        uint32_t ob = 0, os = 0;
        if (lane == 0) {
            if (bb) ob = atomicAdd(&s_nbig, (uint32_t)__popc(bb));
            if (sb) os = atomicAdd(&s_nsmall, (uint32_t)__popc(sb));
        }
        ob = __shfl_sync(0xffffffffu, ob, 0);
        os = __shfl_sync(0xffffffffu, os, 0);
        const uint32_t below = lanemask_lt();
        if (big) big_list[ob + __popc(bb & below)] = (uint32_t)t;
        if (small) small_list[os + __popc(sb & below)] = (uint32_t)t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sort_ctrs[0] = s_nbig;
        sort_ctrs[1] = s_nsmall;
    }
    if (threadIdx.x == 0) {
        *num_keys = carry;
        if ((int64_t)carry > capacity) *status = GS_ERR_CAPACITY;
    }
}

template <bool kCull>
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter(const uint32_t* __restrict__ tt,
                                                            const int4* __restrict__ rect,
                                                            const float4* __restrict__ rgbd, int64_t E, int64_t n,
                                                            Views views, const uint32_t* __restrict__ start,
                                                            uint32_t* __restrict__ stripes, int64_t capacity,
                                                            uint64_t* __restrict__ comp, CullArgs ca) {
    pdl_enter();
    struct Claim {
        const uint32_t* start;
        uint32_t* mine;          // this lane's stripe
        int64_t capacity;
        uint64_t* comp;
        __device__ uint32_t claim(uint32_t g) const { return start[g] + atomicAdd(mine + g, 1u); }
        __device__ void write(uint32_t pos, uint32_t e, uint32_t zbits) const {
            if ((int64_t)pos < capacity) comp[pos] = ((uint64_t)zbits << 32) | e;
        }
    };
    const Claim c{start, stripes + (size_t)(threadIdx.x & 31) * (size_t)views.total_tiles, capacity, comp};
    for_each_key<true, kCull>(tt, rect, rgbd, E, n, views, ca, c);
}

// Shared memory of k_tile_sort: the groups' keys, one large tile's keys, or the
// radix path's bookkeeping (one at a time).
struct RadixSmem {
    uint32_t hist[kRadix];
    uint32_t base[kRadix];
    uint32_t rbase[kRadix];
    uint32_t cnt[2][kRadixWarps][kRadix];
    uint32_t warp[kRadixThreads / 32 + 1];
};
union SortSmem {
    uint64_t group_keys[kGroups][2][kSmallCap];   // the groups' own sorts (two buffers each)
    uint64_t keys[2][kSegCap];                    // a CTA's sort of one larger tile (two buffers)
    RadixSmem rx;
};

// Exclusive scan of one value per thread over the first kRadixThreads threads;
// every thread of the CTA must call it (it contains CTA barriers).
__device__ __forceinline__ uint32_t radix_exclusive_scan(uint32_t x, uint32_t* s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool act = tid < kRadixThreads;
    uint32_t inc = act ? x : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (act && lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kRadixWarps ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kRadixWarps) s_warp[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t r = act ? s_warp[warp] + inc - x : 0u;
    __syncthreads();
    return r;
}

// Stable LSD radix sort of the n composites at a (scratch b, same length) by
// 8-bit digits over bits [0, ebits) (the entry) and [32, 63) (the z bits).  The
// first kRadixThreads threads do the work, the others take part in the CTA
// barriers only.  Each pass: digit histogram, its exclusive scan, then a stable
// scatter in rounds of kRadixThreads keys (ranks within a warp from match_any,
// earlier warps' counts of the digit from a per-round table).  Returns the
// buffer holding the result.
__device__ uint64_t* seg_radix_sort(uint64_t* a, uint64_t* b, int n, int ebits, RadixSmem& sm) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool act = tid < kRadixThreads;
    const uint32_t lt = lanemask_lt();
    int shifts[12], np = 0;
    for (int s = 0; s < ebits; s += kRadixBits) shifts[np++] = s;
    for (int s = 32; s < 63; s += kRadixBits) shifts[np++] = s;
    uint64_t* src = a;
    uint64_t* dst = b;
    for (int p = 0; p < np; p++) {
        const int sh = shifts[p];
        if (act) sm.hist[tid] = 0u;
        __syncthreads();
        for (int i = tid; i < n; i += kSortThreads) atomicAdd(&sm.hist[(uint32_t)(src[i] >> sh) & (kRadix - 1)], 1u);
        __syncthreads();
        const uint32_t base = radix_exclusive_scan(act ? sm.hist[tid] : 0u, sm.warp);
        if (act) sm.base[tid] = base;
        for (int k = tid; k < 2 * kRadixWarps * kRadix; k += kSortThreads) (&sm.cnt[0][0][0])[k] = 0u;
        __syncthreads();
        for (int r0 = 0, round = 0; r0 < n; r0 += kRadixThreads, round++) {
            const int buf = round & 1;
            const int i = r0 + tid;
            const bool valid = act && i < n;
            const uint64_t key = valid ? src[i] : 0ull;
            const uint32_t d = valid ? (uint32_t)(key >> sh) & (kRadix - 1) : (uint32_t)kRadix;   // sentinel
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0) sm.cnt[buf][warp][d] = __popc(peers);
            __syncthreads();
            if (act) {   // thread tid owns digit tid: earlier warps' counts, then the digit's running base
                uint32_t run = 0;
#pragma unroll
                for (int w = 0; w < kRadixWarps; w++) {
                    const uint32_t c = sm.cnt[buf][w][tid];
                    sm.cnt[buf][w][tid] = run;
                    run += c;
                    sm.cnt[buf ^ 1][w][tid] = 0u;
                }
                sm.rbase[tid] = sm.base[tid];
                sm.base[tid] += run;
            }
            __syncthreads();
            if (valid) dst[sm.rbase[d] + sm.cnt[buf][warp][d] + rank] = key;
        }
        __syncthreads();
        uint64_t* t = src; src = dst; dst = t;
    }
    return src;
}
static_assert(kRadix == kRadixThreads, "one digit per working thread in the radix bookkeeping");

__device__ __forceinline__ void group_sync(int g) {
    asm volatile("bar.sync %0, %1;" :: "r"(g + 1), "r"(kGroup) : "memory");
}

// Sorts the composites s[0, P) in shared memory (P a power of two >= 32; t a
// second buffer of P) by NT threads (tid in [0, NT)) that meet at sync():
// each warp sorts runs of 32 in registers (a bitonic network over its lanes,
// no barrier), then log2(P / 32) merge levels double the runs.  At each level
// thread tid writes outputs [tid k, tid k + k) (k = P / NT, at least 1) of
// its pair of runs: a binary search on the merge path finds how many of the
// first outputs come from the first run, then k sequential merge steps.  The
// composites are unique (z bits, entry), so the order is the sorted one however
// the work is split.  Returns the buffer that holds the result.
template <int NT, typename Sync>
__device__ __forceinline__ uint64_t* merge_sort_smem(uint64_t* s, uint64_t* t, int P, int tid, Sync sync) {
    const int lane = tid & 31, wid = tid >> 5;
    for (int c = wid; c < P / 32; c += NT / 32) {
        uint64_t x = s[c * 32 + lane];
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint64_t y = __shfl_xor_sync(0xffffffffu, x, j);
                const bool up = (lane & k) == 0, lower = (lane & j) == 0;   // k = 32: ascending
                // the lower lane of an ascending pair keeps the smaller key, and so on
                x = ((x < y) == (lower == up)) ? x : y;
            }
        s[c * 32 + lane] = x;
    }
    sync();
    uint64_t* src = s;
    uint64_t* dst = t;
    const int k = P >= NT ? P / NT : 1;
    for (int r = 32; r < P; r <<= 1) {
        const int o = tid * k;
        if (o < P) {
            const int pair = o / (2 * r), d = o - pair * 2 * r;
            const uint64_t* A = src + pair * 2 * r;
            const uint64_t* B = A + r;
            int lo = d > r ? d - r : 0, hi = d < r ? d : r;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A[mid] < B[d - mid - 1]) lo = mid + 1;
                else hi = mid;
            }
            int i = lo, j = d - lo;
            for (int q = 0; q < k; q++) {
                const bool take_a = i < r && (j >= r || A[i] < B[j]);
                dst[o + q] = take_a ? A[i++] : B[j++];
            }
        }
        sync();
        uint64_t* tmp = src;
        src = dst;
        dst = tmp;
    }
    return src;
}

// Merge sort of a tile of n <= kSmallCap composites by one group of kGroup
// threads in its two shared-memory buffers (P = n rounded up to a power of two,
// at least 32, padded with the largest value; the group's own named barrier).
__device__ __forceinline__ void sort_group_tile(uint64_t* __restrict__ seg, uint32_t* __restrict__ vseg, int n,
                                                uint64_t tile_hi, uint64_t* s, uint64_t* t, int g) {
    const int gt = threadIdx.x & (kGroup - 1);
    int P = 32;
    while (P < n) P <<= 1;
    for (int i = gt; i < P; i += kGroup) s[i] = i < n ? seg[i] : ~0ull;
    group_sync(g);
    const uint64_t* res = merge_sort_smem<kGroup>(s, t, P, gt, [&]() { group_sync(g); });
    for (int i = gt; i < n; i += kGroup) {
        const uint64_t c = res[i];
        seg[i] = tile_hi | (c >> 32);
        vseg[i] = (uint32_t)c;
    }
    group_sync(g);
}

// The same by the whole CTA for n <= kSegCap.
__device__ __forceinline__ void sort_cta_tile(uint64_t* __restrict__ seg, uint32_t* __restrict__ vseg, int n,
                                              uint64_t tile_hi, uint64_t* s, uint64_t* t) {
    const int tid = threadIdx.x;
    int P = 32;
    while (P < n) P <<= 1;
    for (int i = tid; i < P; i += kSortThreads) s[i] = i < n ? seg[i] : ~0ull;
    __syncthreads();
    const uint64_t* res = merge_sort_smem<kSortThreads>(s, t, P, tid, []() { __syncthreads(); });
    for (int i = tid; i < n; i += kSortThreads) {
        const uint64_t c = res[i];
        seg[i] = tile_hi | (c >> 32);
        vseg[i] = (uint32_t)c;
    }
}

// Two passes over the work lists of k_bin_offsets, each claimed dynamically
// with an atomic counter (sort_ctrs[2], [3], zeroed by k_bin_zero), so that the
// large tiles, which cluster in the image, spread over all CTAs: first each CTA
// claims tiles of more than kSmallCap keys and sorts them with all its threads
// (shared memory up to kSegCap keys, the radix path above), then each of its
// groups claims tiles of at most kSmallCap keys and sorts them on its own.  Every
// stage of a sort is one compare-exchange per thread (two for the largest
// shared-memory tiles).
__global__ void __launch_bounds__(kSortThreads, 2) k_tile_sort(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                              uint64_t* __restrict__ alt,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ big_list,
                                                              const uint32_t* __restrict__ small_list,
                                                              uint32_t* __restrict__ sort_ctrs, int ebits) {
    extern __shared__ __align__(16) unsigned char s_sort_raw[];   // SortSmem, dynamic (above 48 KB)
    SortSmem& sm = *reinterpret_cast<SortSmem*>(s_sort_raw);
    __shared__ uint32_t s_claim[1 + kGroups];
    pdl_enter();
    const int tid = threadIdx.x, g = tid / kGroup;
    const uint32_t n_big = sort_ctrs[0], n_small = sort_ctrs[1];
    for (;;) {
        if (tid == 0) s_claim[0] = atomicAdd(&sort_ctrs[2], 1u);
        __syncthreads();
        const uint32_t r = s_claim[0];
        __syncthreads();                        // read by every thread before the next claim
        if (r >= n_big) break;
        const uint32_t t = big_list[r];
        const uint2 rg = ranges[t];
        const int n = (int)(rg.y - rg.x);
        uint64_t* seg = keys + rg.x;
        uint32_t* vseg = vals + rg.x;
        const uint64_t tile_hi = (uint64_t)t << 32;
        if (n <= kSegCap) {
            sort_cta_tile(seg, vseg, n, tile_hi, sm.keys[0], sm.keys[1]);
        } else {
            const uint64_t* res = seg_radix_sort(seg, alt + rg.x, n, ebits, sm.rx);
            for (int i = tid; i < n; i += kSortThreads) {
                const uint64_t c = res[i];
                seg[i] = tile_hi | (c >> 32);       // same index, same thread: in place is safe
                vseg[i] = (uint32_t)c;
            }
        }
        __syncthreads();                        // shared memory is reused by the next tile
    }
    for (;;) {
        if ((tid & (kGroup - 1)) == 0) s_claim[1 + g] = atomicAdd(&sort_ctrs[3], 1u);
        group_sync(g);
        const uint32_t r = s_claim[1 + g];
        group_sync(g);
        if (r >= n_small) break;
        const uint32_t t = small_list[r];
        const uint2 rg = ranges[t];
        sort_group_tile(keys + rg.x, vals + rg.x, (int)(rg.y - rg.x), (uint64_t)t << 32, sm.group_keys[g][0],
                        sm.group_keys[g][1], g);
    }
}

// One thread per key of the sorted lists: the key's block mask (gs_bins.masks),
// from the splat of its entry with the rasterisers' operands (mean, scaled
// conic and opacity) and their culling test.  Keys past M (the device count,
// clamped to the capacity) are left alone.
template <int T>
__global__ void __launch_bounds__(kBinThreads) k_bin_masks(const uint64_t* __restrict__ keys,
                                                          const uint32_t* __restrict__ vals,
                                                          const uint32_t* __restrict__ num_keys, int64_t capacity,
                                                          const float2* __restrict__ xy,
                                                          const float4* __restrict__ conic_o, Views views,
                                                          float amin, uint32_t* __restrict__ masks) {
    pdl_enter();
    const int64_t k = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
    const int64_t M = min((int64_t)*num_keys, capacity);
    if (k >= M) return;
    const int t = (int)(keys[k] >> 32);
    const uint32_t e = vals[k];
    const int v = view_of_tile(views, t);
    const int lt = t - views.v[v].tile_base;
    const float4 c = conic_o[e];
    float4 q;
    scale_conic(c.x, c.y, c.z, &q.x, &q.y, &q.z);
    q.w = c.w;
    masks[k] = splat_block_mask<T>(xy[e], q, lt % views.v[v].tiles_x, lt / views.v[v].tiles_x, amin);
}

}  // namespace

SortPlan make_sort_plan(int64_t key_capacity, int32_t total_tiles, int32_t tile, float alpha_min,
                        int32_t block_masks, int32_t cull_tiles) {
    SortPlan p;
    p.capacity = key_capacity;
    p.total_tiles = total_tiles;
    p.tile = tile;
    p.alpha_min = alpha_min;
    p.block_masks = block_masks;
    p.cull_tiles = cull_tiles;
    return p;
}

// Workspace layout of launch_bin_sort (offsets in bytes, 256-byte aligned):
//   stripe counters / cursors : kStripes x total_tiles u32 (stripe-major)
//   tile totals / starts      : total_tiles u32
//   sort work lists           : 2 x total_tiles u32 (large tiles, small tiles) + 4 u32 counters
//   composites (alt)          : capacity u64 (the radix path's second buffer)
static size_t ws_stripes(int32_t total_tiles) {
    return align_up(sizeof(uint32_t) * (size_t)kStripes * (size_t)total_tiles, 256);
}
static size_t ws_totals(int32_t total_tiles) { return align_up(sizeof(uint32_t) * (size_t)(total_tiles + 1), 256); }
static size_t ws_lists(int32_t total_tiles) { return align_up(sizeof(uint32_t) * (2 * (size_t)total_tiles + 4), 256); }

size_t bin_sort_workspace(int64_t n_entries, int64_t capacity, int32_t total_tiles) {
    (void)n_entries;
    return ws_stripes(total_tiles) + ws_totals(total_tiles) + ws_lists(total_tiles) +
           align_up(sizeof(uint64_t) * (size_t)(capacity > 0 ? capacity : 1), 256);
}

cudaError_t launch_bin_sort(const gs_projected& pr, int64_t n, const Views& views, const SortPlan& plan,
                            const gs_bins& bins, void* ws, cudaStream_t s) {
    const int64_t E = n * views.n;
    const int64_t cap = plan.capacity;
    const int T = plan.total_tiles;
    char* p = static_cast<char*>(ws);
    uint32_t* stripes = reinterpret_cast<uint32_t*>(p);
    p += ws_stripes(T);
    uint32_t* totals = reinterpret_cast<uint32_t*>(p);
    p += ws_totals(T);
    uint32_t* big_list = reinterpret_cast<uint32_t*>(p);
    uint32_t* small_list = big_list + T;
    uint32_t* sort_ctrs = small_list + T;
    p += ws_lists(T);
    uint64_t* alt = reinterpret_cast<uint64_t*>(p);

    cudaError_t err = cudaSuccess;
    if (E == 0 || T == 0) {
        err = cudaMemsetAsync(bins.ranges, 0, sizeof(uint32_t) * 2 * (size_t)T, s);
        if (err != cudaSuccess) return err;
        return cudaMemsetAsync(bins.num_keys, 0, sizeof(uint32_t), s);
    }
    int ebits = 0;
    while ((1ll << ebits) < E) ebits++;

    const int nb_entries = (int)ceil_div(E, kBinThreads);
    const int4* rect = reinterpret_cast<const int4*>(pr.rect);
    const float4* rgbd = reinterpret_cast<const float4*>(pr.rgbd);
    const int64_t words = (int64_t)kStripes * T;
    const int nb_zero = (int)(ceil_div(words, kBinThreads) < 4096 ? ceil_div(words, kBinThreads) : 4096);
    err = launch_pdl(k_bin_zero, nb_zero, kBinThreads, 0, s, stripes, words, sort_ctrs);
    const CullArgs ca{reinterpret_cast<const float2*>(pr.xy), reinterpret_cast<const float4*>(pr.conic_o), plan.tile,
                      plan.alpha_min};
    if (err == cudaSuccess)
        err = launch_pdl(plan.cull_tiles ? k_bin_count<true> : k_bin_count<false>, nb_entries, kBinThreads, 0, s,
                         pr.tiles_touched, rect, E, n, views, stripes, ca);
    if (err == cudaSuccess)
        err = launch_pdl(k_bin_stripes, (int)ceil_div((int64_t)T * 32, kBinThreads), kBinThreads, 0, s, stripes, T,
                         totals);
    if (err == cudaSuccess)
        err = launch_pdl(k_bin_offsets, 1, kScanThreads, 0, s, totals, T, reinterpret_cast<uint2*>(bins.ranges),
                         bins.num_keys, cap, bins.status, big_list, small_list, sort_ctrs);
    if (err == cudaSuccess)
        err = launch_pdl(plan.cull_tiles ? k_bin_scatter<true> : k_bin_scatter<false>, nb_entries, kBinThreads, 0,
                         s, pr.tiles_touched, rect, rgbd, E, n, views, totals, stripes, cap, bins.keys, ca);
    if (err == cudaSuccess) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // the sort's shared memory is above the 48 KB static limit: opt in (per
        // device; not a stream operation, so it may run during capture)
        err = cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SortSmem));
        if (err != cudaSuccess) return err;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_sort, kSortThreads, sizeof(SortSmem));
        const int64_t full = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        const int grid = (int)(T < full ? T : full);
        err = launch_pdl(k_tile_sort, grid, kSortThreads, sizeof(SortSmem), s, bins.keys, bins.vals, alt,
                         reinterpret_cast<const uint2*>(bins.ranges), (const uint32_t*)big_list,
                         (const uint32_t*)small_list, sort_ctrs, ebits);
    }
    if (err == cudaSuccess && plan.block_masks) {
        const int grid = (int)ceil_div(cap > 0 ? cap : 1, kBinThreads);
        auto kernel = plan.tile == 8 ? k_bin_masks<8> : plan.tile == 16 ? k_bin_masks<16> : k_bin_masks<32>;
        err = launch_pdl(kernel, grid, kBinThreads, 0, s, (const uint64_t*)bins.keys, (const uint32_t*)bins.vals,
                         (const uint32_t*)bins.num_keys, cap, reinterpret_cast<const float2*>(pr.xy),
                         reinterpret_cast<const float4*>(pr.conic_o), views, plan.alpha_min, bins.masks);
    }
    if (err != cudaSuccess) return err;
    return cudaGetLastError();
}

// L2 read probe (a measurement helper, not part of the method): every CTA
// streams its grid-stride share of buf `reps` times with 16-byte loads cached in
// L2 only; four independent sums keep four loads in flight per thread; one
// atomic per CTA into *out keeps the loads from being dropped.
__global__ void __launch_bounds__(kBinThreads) k_l2_read(const float4* __restrict__ buf, int64_t n4, int reps,
                                                        float* __restrict__ out) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    const int64_t stride = (int64_t)gridDim.x * kBinThreads;
    for (int r = 0; r < reps; r++) {
        int64_t i = (int64_t)blockIdx.x * kBinThreads + threadIdx.x;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++)
                asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                             : "=f"(v[u].x), "=f"(v[u].y), "=f"(v[u].z), "=f"(v[u].w) : "l"(buf + i + u * stride));
            a0 += (v[0].x + v[0].y) + (v[0].z + v[0].w);
            a1 += (v[1].x + v[1].y) + (v[1].z + v[1].w);
            a2 += (v[2].x + v[2].y) + (v[2].z + v[2].w);
            a3 += (v[3].x + v[3].y) + (v[3].z + v[3].w);
        }
        for (; i < n4; i += stride) {
            float4 v;
            asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(buf + i));
            a0 += (v.x + v.y) + (v.z + v.w);
        }
    }
    float sum = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ float s_w[kBinThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kBinThreads / 32; w++) t += s_w[w];
        atomicAdd(out, t);
    }
}

cudaError_t launch_l2_read(const float* buf, int64_t n, int reps, float* out, cudaStream_t s) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_l2_read<<<8 * sms, kBinThreads, 0, s>>>(reinterpret_cast<const float4*>(buf), n / 4, reps, out);
    return cudaGetLastError();
}

}  // namespace gs
