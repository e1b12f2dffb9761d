// raster.cu -- front-to-back alpha compositing of colour and depth (Sec. 3.3:
// a pixel's colour is the alpha blend of the Gaussians covering it, and the
// mapper renders both colour and depth per keyframe) and its backward pass.
//
// Work item = one 8 x 4 block of pixels of one tile (one pixel per lane); a
// persistent grid's warps take items from a device counter (views of uneven
// size balance across SMs) and each works through its tile's depth-sorted
// list on its own:
// lane l gathers splat base + l of the list into the warp's shared-memory ring
// (cp.async), culls it, and the warp parks the kept splats in its compositing
// slots and composites them with broadcast reads while the next two batches
// of 32 (and the list entries of the batch after those) are already in flight.  A lane's per-splat tests are
// predicates, not branches, so a warp never diverges inside a batch.  Before compositing, the warp drops the splats that cannot reach
// alpha_min anywhere in its block.  There is no CTA-wide barrier, so a warp
// stops as soon as its own 32 pixels are saturated and takes the next item; the
// depth of a tile's deepest pixels (up to ~8x the mean) only costs its own warp.
//
// The backward pass walks the same lists back to front from the per-pixel
// checkpoint (T_final, n_contrib) written by the forward pass: it rebuilds the
// transmittance before each splat by T_before = T_after / (1 - alpha) and keeps
// the colour/depth "behind" a splat as a running normalised sum, so no
// per-splat state is stored by the forward pass.  A warp starts at its own
// deepest pixel.  Per-splat gradients are summed over the warp's 32 pixels by a
// transposed butterfly (10 values in 12 shuffles; each lane ends with one
// finished sum); two splats are reduced together so that their shuffle chains
// overlap, and the ten sums go to global memory as ten atomics.
//
// With the loss fused in (gs_render_fwd_loss / gs_render_bwd_raster_loss) the
// forward pass also sums the Eq. 6 L1 terms per view and records each block's
// deepest n_contrib; when a launch has few blocks per SM, one CTA sorts the
// blocks by that depth and both passes take the deepest blocks first, so that
// no long walk starts when the queue is nearly empty.
#include "gs_internal.cuh"

namespace gs {
namespace {

__device__ __forceinline__ float sgnf(float x) { return x > 0.f ? 1.f : (x < 0.f ? -1.f : 0.f); }

// 4-byte asynchronous copy global -> shared (no register held while in flight)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n\tcp.async.commit_group;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Gather of one splat's rows into shared memory without registers: 8 + 16 + 16
// bytes as one commit group (committed even when the lane copies nothing, so
// that every lane's group count advances by one per batch).
__device__ __forceinline__ void cp_async_splat(float2* dxy, float4* dco, float4* dcd, const float2* xy,
                                               const float4* conic_o, const float4* rgbd, uint32_t e, bool valid) {
    if (valid) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" :: "r"((uint32_t)__cvta_generic_to_shared(dxy)),
                     "l"(xy + e) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"((uint32_t)__cvta_generic_to_shared(dco)),
                     "l"(conic_o + e) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" :: "r"((uint32_t)__cvta_generic_to_shared(dcd)),
                     "l"(rgbd + e) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// all but this lane's newest commit group have landed
__device__ __forceinline__ void cp_async_wait_all_but_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// A tile of T x T pixels is covered by (T / 8) x (T / 4) warps; lane l of warp w
// is pixel (8 (w % (T/8)) + l % 8, 4 (w / (T/8)) + l / 8) of the tile.
template <int T>
struct TileShape {
    static constexpr int kWarps = (T / 8) * (T / 4);    // 8 x 4 pixel blocks per tile
};

__device__ __forceinline__ void lane_pixel(int T, int tid, int* x, int* y) {
    const int w = tid >> 5, l = tid & 31;
    *x = (w % (T / 8)) * 8 + (l & 7);
    *y = (w / (T / 8)) * 4 + (l >> 3);
}

// One splat as the rasterisers read it.
struct Splat {
    float2 xy;
    float4 q;     // -0.5 log2e A, -log2e B, -0.5 log2e C, opacity
    float4 cd;    // r, g, b, z
};


__device__ __forceinline__ Splat load_splat(const float2* __restrict__ xy, const float4* __restrict__ conic_o,
                                            const float4* __restrict__ rgbd, uint32_t e) {
    Splat s;
    const float4 c = conic_o[e];
    scale_conic(c.x, c.y, c.z, &s.q.x, &s.q.y, &s.q.z);
    s.q.w = c.w;
    s.xy = xy[e];
    s.cd = rgbd[e];
    return s;
}

// Persistent launch: kRasterThreads-thread CTAs, as many as fit on the GPU;
// every warp repeatedly takes the next work item -- one 8 x 4 pixel block of
// one tile of one view -- from a device counter and processes it alone.
constexpr int kRasterThreads = 256;
constexpr int kRasterWarps = kRasterThreads / 32;

// Fused loss, end of the forward launch: this CTA's per-view sums go to its
// partial slot; the last CTA to finish adds all slots into acc and writes the
// loss terms (the same expressions as the stand-alone loss), then resets the
// ticket.  Called by every thread of the CTA after its item loop.
__device__ void fused_loss_finish(const FusedLoss& fl, const Views& views, const float* s_loss) {
    __shared__ int s_last;
    __shared__ float s_red[kRasterThreads / 32][3];
    __syncthreads();
    float* mine = fl.partial + (size_t)blockIdx.x * views.n * 3;
    for (int k = threadIdx.x; k < views.n * 3; k += kRasterThreads) mine[k] = s_loss[k];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(fl.ticket, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int v = 0; v < views.n; v++) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int c = threadIdx.x; c < (int)gridDim.x; c += kRasterThreads) {
            const float* p = fl.partial + ((size_t)c * views.n + v) * 3;
            a0 += __ldcg(p); a1 += __ldcg(p + 1); a2 += __ldcg(p + 2);
        }
        a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
        if (lane == 0) { s_red[w][0] = a0; s_red[w][1] = a1; s_red[w][2] = a2; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float t0 = 0.f, t1 = 0.f, t2 = 0.f;
            for (int k = 0; k < kRasterThreads / 32; k++) { t0 += s_red[k][0]; t1 += s_red[k][1]; t2 += s_red[k][2]; }
            const int HW = views.v[v].W * views.v[v].H;
            fl.acc[4 * v] = t0; fl.acc[4 * v + 1] = t1; fl.acc[4 * v + 2] = t2; fl.acc[4 * v + 3] = 0.f;
            fl.terms[2 * v] = t0 / (3.0f * (float)HW);
            fl.terms[2 * v + 1] = t2 > 0.f ? t1 / t2 : 0.f;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *fl.ticket = 0;
}


// The persistent launches' work queue over n items.  Plain: every warp draws
// items from a device counter until it draws one >= n, so a launch makes n +
// (its warps) increments.  Spread (a launch that walks a cost-ordered list,
// deepest first): warp w of CTA c takes item w * gridDim.x + c first, without
// the counter, so that the deepest items of the first round go to the first
// warps of different CTAs instead of to the warps that happen to draw first
// (which tend to share an SM); the later draws take items from gridDim.x *
// warps on.  Either way the warp that draws the last value returns the counter
// to zero for the next launch (no reset on the stream).
struct WorkQueue {
    int* counter;
    int n, base, total;
    bool spread;
    __device__ WorkQueue(int* c, int n_items, bool spread_first) : counter(c), n(n_items), spread(spread_first) {
        const int warps = (int)gridDim.x * kRasterWarps;
        base = spread ? warps : 0;                                        // items handed out without the counter
        total = spread ? max(n - warps, 0) + min(warps, n) : n + warps;   // increments of one launch
    }
    __device__ __forceinline__ int first(int lane) {
        if (spread) return (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x;
        return next(lane);
    }
    __device__ __forceinline__ int next(int lane) {
        int item = 0;
        if (lane == 0) {
            const int d = atomicAdd(counter, 1);
            if (d == total - 1) *counter = 0;
            item = base + d;
        }
        return __shfl_sync(0xffffffffu, item, 0);
    }
};

// Prefetch: RING keeps two batches of splats in flight through a shared-memory
// ring (a launch with few blocks per SM, where a lone warp's deep walk would
// otherwise wait a gather latency per batch); without it one batch is in
// flight in registers, and the smaller shared footprint leaves more L1 for the
// splats that the warps of a tile share (a launch with many blocks per SM).
template <int T, bool LOSS, bool RING, bool MASKS>
__global__ void __launch_bounds__(kRasterThreads, 4) k_render_fwd(
        const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
        const uint32_t* __restrict__ vals, const uint32_t* __restrict__ masks, const uint2* __restrict__ ranges,
        Views views, RenderConsts rc, gs_image img, int* __restrict__ queue, int n_items, FusedLoss fl) {
    constexpr int W = TileShape<T>::kWarps;     // pixel blocks per tile
    // the batch's kept splats in pairs (slots 2i, 2i + 1), so that the weights of
    // two splats are formed by packed FP32x2 operations: {-mx, -mx', -my, -my'},
    // {qa, qa', qb, qb'}, {qc, qc', o, o'}
    __shared__ float4 s_pm[kRasterWarps][16];
    __shared__ float4 s_pab[kRasterWarps][16];
    __shared__ float4 s_pco[kRasterWarps][16];
    __shared__ float4 s_cd[kRasterWarps][32];
    __shared__ uint32_t s_pos[kRasterWarps][32];
    __shared__ float s_loss[LOSS ? GS_MAX_VIEWS * 3 : 1];    // per-view sums of this CTA (fused loss)
    __shared__ float s_tgt[LOSS ? kRasterWarps : 1][4][32];   // each lane's targets, fetched at the item's start
    __shared__ float s_lacc[LOSS ? kRasterWarps : 1][3][32];  // each lane's running sums for the warp's view lv
    // the next batches' splats, gathered by cp.async: two slots of 32 per warp (RING)
    __shared__ float2 r_xy[RING ? kRasterWarps : 1][2][32];
    __shared__ float4 r_co[RING ? kRasterWarps : 1][2][32];
    __shared__ float4 r_cd[RING ? kRasterWarps : 1][2][32];
    pdl_enter();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lv = -1;                                               // view of the sums in s_lacc (warp-uniform)
    if constexpr (LOSS) {
        for (int k = threadIdx.x; k < views.n * 3; k += kRasterThreads) s_loss[k] = 0.f;
        for (int k = 0; k < 3; k++) s_lacc[w][k][lane] = 0.f;
        __syncthreads();
    }
    // the warp's lane sums of view lv into the CTA's per-view sums
    auto flush_lanes = [&]() {
        if (lv < 0) return;
        for (int k = 0; k < 3; k++) {
            const float x = warp_sum(s_lacc[w][k][lane]);
            s_lacc[w][k][lane] = 0.f;
            if (lane == 0) atomicAdd(&s_loss[3 * lv + k], x);
        }
    };
    const uint32_t lt_mask = (1u << lane) - 1u;
    const float amin = rc.alpha_min, amax = rc.alpha_max, tcut = rc.T_cut;
    // the order the previous backward pass left, if it is a permutation of these items
    bool ordered = false;
    if constexpr (LOSS)
        ordered = fl.order != nullptr && fl.order_tag[0] == (uint32_t)n_items &&
                  fl.order_tag[1] == ((uint32_t)n_items ^ kOrderTagMagic);
    WorkQueue wq(queue, n_items, ordered);
    for (int raw = wq.first(lane); raw < n_items; raw = wq.next(lane)) {
        int item = raw;
        if (ordered) {                           // (an index out of range can only come from a foreign workspace)
            const uint32_t o = fl.order[raw];
            item = o < (uint32_t)n_items ? (int)o : raw;
        }
        const int g = item / W, blk = item % W;
        const int v = view_of_tile(views, g);
        const ViewParams& vp = views.v[v];
        const int lt = g - vp.tile_base;
        const int tx = lt % vp.tiles_x, ty = lt / vp.tiles_x;
        int ox, oy;
        lane_pixel(T, blk * 32 + lane, &ox, &oy);
        const int px = tx * T + ox, py = ty * T + oy;
        const bool inside = px < vp.W && py < vp.H;
        if (!__any_sync(0xffffffffu, inside)) {               // block entirely outside the image
            if (LOSS && fl.item_cost != nullptr && lane == 0) fl.item_cost[item] = 0u;
            continue;
        }
        if constexpr (LOSS) {
            if (inside) {
                const int HW = vp.W * vp.H, pix = py * vp.W + px;
                const float* t = fl.tc + 3 * (size_t)vp.pix_base;
                cp_async4(&s_tgt[w][0][lane], t + pix);
                cp_async4(&s_tgt[w][1][lane], t + HW + pix);
                cp_async4(&s_tgt[w][2][lane], t + 2 * HW + pix);
                cp_async4(&s_tgt[w][3][lane], fl.td + vp.pix_base + pix);
            }
        }
        const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
        const float2 sx2 = make_float2(sx, sx), sy2 = make_float2(sy, sy);
        // sample rectangle of this 8 x 4 block (the culling test without block masks)
        const float bx0 = (float)(tx * T + (blk % (T / 8)) * 8) + 0.5f;
        const float by0 = (float)(ty * T + (blk / (T / 8)) * 4) + 0.5f;
        const float bx1 = bx0 + 7.f, by1 = by0 + 3.f;
        constexpr bool use_masks = MASKS;
        const uint2 range = ranges[g];

        float Tr = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f;
        uint32_t last = 0;
        bool done = !inside;
        // RING: while batch b is composited, the splats of batches b + 1 and b + 2
        // are in flight into the warp's two ring slots (cp.async, no registers
        // held; batch b has left its slot for the compositing slots) and the list
        // entries of batch b + 3 into a register.  Otherwise the splats of batch
        // b + 1 and the list entries of b + 2 are in flight in registers.  Either
        // way a splat load never waits on its index.
        // With block masks, the mask of each list position (gs_bins.masks) is in flight with its
        // list entry; m0 is the mask of batch b, m1 (and m2 with the ring) those of the batches after.
        Splat nxt;
        uint32_t nidx = 0, m0 = 0, m1 = 0, m2 = 0;
        const uint32_t bbit = 1u << blk;
        int slot_b = 0;                                  // ring slot of batch b
        if constexpr (RING) {
            const bool v0 = range.x + lane < range.y, v1 = range.x + 32 + lane < range.y;
            const uint32_t i0 = v0 ? vals[range.x + lane] : 0u, i1 = v1 ? vals[range.x + 32 + lane] : 0u;
            m0 = v0 && use_masks ? masks[range.x + lane] : 0u;
            m1 = v1 && use_masks ? masks[range.x + 32 + lane] : 0u;
            // with masks, only the splats that reach this block are gathered
            cp_async_splat(&r_xy[w][0][lane], &r_co[w][0][lane], &r_cd[w][0][lane], xy, conic_o, rgbd, i0,
                           v0 && (!use_masks || (m0 & bbit) != 0u));
            cp_async_splat(&r_xy[w][1][lane], &r_co[w][1][lane], &r_cd[w][1][lane], xy, conic_o, rgbd, i1,
                           v1 && (!use_masks || (m1 & bbit) != 0u));
            if (range.x + 64 + lane < range.y) {
                nidx = vals[range.x + 64 + lane];
                if (use_masks) m2 = masks[range.x + 64 + lane];
            }
        } else {
            if (range.x + lane < range.y) {
                if (use_masks) m0 = masks[range.x + lane];
                if (!use_masks || (m0 & bbit) != 0u) nxt = load_splat(xy, conic_o, rgbd, vals[range.x + lane]);
            }
            if (range.x + 32 + lane < range.y) {
                nidx = vals[range.x + 32 + lane];
                if (use_masks) m1 = masks[range.x + 32 + lane];
            }
        }
        for (uint32_t base = range.x; base < range.y; base += 32) {
            if constexpr (RING) {
                cp_async_wait_all_but_one();             // this lane's splat of batch b has landed
                nxt.xy = r_xy[w][slot_b][lane];
                const float4 c = r_co[w][slot_b][lane];
                scale_conic(c.x, c.y, c.z, &nxt.q.x, &nxt.q.y, &nxt.q.z);
                nxt.q.w = c.w;
                nxt.cd = r_cd[w][slot_b][lane];
            }
            const bool keep = base + lane < range.y &&
                              (use_masks ? (m0 & bbit) != 0u
                                         : splat_reaches_block(nxt.xy, nxt.q, bx0, bx1, by0, by1, amin));
            const uint32_t kept = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) {
                const int slot = __popc(kept & lt_mask), pi = slot >> 1, h = slot & 1;
                float* pm = reinterpret_cast<float*>(&s_pm[w][pi]);
                float* pab = reinterpret_cast<float*>(&s_pab[w][pi]);
                float* pco = reinterpret_cast<float*>(&s_pco[w][pi]);
                pm[h] = -nxt.xy.x; pm[2 + h] = -nxt.xy.y;
                pab[h] = nxt.q.x; pab[2 + h] = nxt.q.y;
                pco[h] = nxt.q.z; pco[2 + h] = nxt.q.w;
                s_cd[w][slot] = nxt.cd;
                s_pos[w][slot] = base - range.x + lane;
            }
            __syncwarp();
            if constexpr (RING) {   // batch b + 2 into batch b's slot (this lane has read its entry)
                cp_async_splat(&r_xy[w][slot_b][lane], &r_co[w][slot_b][lane], &r_cd[w][slot_b][lane], xy, conic_o,
                               rgbd, nidx, base + 64 + lane < range.y && (!use_masks || (m2 & bbit) != 0u));
                m0 = m1;
                m1 = m2;
                nidx = 0u;
                m2 = 0u;
                if (base + 96 + lane < range.y) {
                    nidx = vals[base + 96 + lane];
                    if (use_masks) m2 = masks[base + 96 + lane];
                }
                slot_b ^= 1;
            } else {
                if (base + 32 + lane < range.y && (!use_masks || (m1 & bbit) != 0u))
                    nxt = load_splat(xy, conic_o, rgbd, nidx);
                m0 = m1;
                if (base + 64 + lane < range.y) {
                    nidx = vals[base + 64 + lane];
                    if (use_masks) m1 = masks[base + 64 + lane];
                }
            }
            // warp-uniform loop; a lane's tests (power > 0, alpha < alpha_min, the
            // transmittance cutoff) become predicates, so the warp never diverges
            const int cnt = __popc(kept);
            int last_k = -1;                         // batch slot of this lane's last blended splat
            // one compositing step of splat k given its power p2 and alpha a
            auto step = [&](int k, float p2, float a) {
                const float test = __fmaf_rn(-a, Tr, Tr);
                const bool blend = !done && !(p2 > 0.f) && !(a < amin);
                const bool stop = blend && test < tcut;
                const bool b = blend && !stop;
                done = done || stop;
                const float4 c = s_cd[w][k];
                const float wgt = b ? __fmul_rn(a, Tr) : 0.f;
                cr = __fmaf_rn(c.x, wgt, cr);
                cg = __fmaf_rn(c.y, wgt, cg);
                cb = __fmaf_rn(c.z, wgt, cb);
                dd = __fmaf_rn(c.w, wgt, dd);
                Tr = b ? test : Tr;
                last_k = b ? k : last_k;
            };
            // splat k alone (the same operations as splat_power2 / splat_weight)
            auto alpha = [&](int k, float* p2, float* a) {
                const int h = k & 1;
                const float4 m = s_pm[w][k >> 1], ab = s_pab[w][k >> 1], co = s_pco[w][k >> 1];
                const float dx = __fadd_rn(sx, h ? m.y : m.x), dy = __fadd_rn(sy, h ? m.w : m.z);
                *p2 = splat_power2(h ? ab.y : ab.x, h ? ab.w : ab.z, h ? co.y : co.x, dx, dy);
                *a = fminf(amax, __fmul_rn(h ? co.w : co.z, splat_weight(p2[0])));
            };
            // splats 2i and 2i + 1 by packed FP32x2 operations: each element is
            // rounded as the scalar intrinsics round it, so the results are identical
            auto alpha_pair = [&](int i, float* p2, float* a) {
                const float4 m = s_pm[w][i], ab = s_pab[w][i], co = s_pco[w][i];
                const float2 dx = __fadd2_rn(sx2, make_float2(m.x, m.y));
                const float2 dy = __fadd2_rn(sy2, make_float2(m.z, m.w));
                const float2 u = __ffma2_rn(make_float2(ab.z, ab.w), dy, __fmul2_rn(make_float2(ab.x, ab.y), dx));
                const float2 q = __fmul2_rn(make_float2(co.x, co.y), dy);
                const float2 pw = __ffma2_rn(dx, u, __fmul2_rn(q, dy));
                const float2 ao = __fmul2_rn(make_float2(co.z, co.w), make_float2(splat_weight(pw.x), splat_weight(pw.y)));
                p2[0] = pw.x; p2[1] = pw.y;
                a[0] = fminf(amax, ao.x); a[1] = fminf(amax, ao.y);
            };
            // groups of four: the four weights do not depend on the transmittance, so
            // they are formed before the four serial steps; the warp checks for
            // saturation once per group (a saturated lane blends nothing more either way)
            int k = 0;
            bool all_done = false;
            for (; k + 4 <= cnt; k += 4) {
                float p2[4], a[4];
                alpha_pair(k >> 1, &p2[0], &a[0]);
                alpha_pair((k >> 1) + 1, &p2[2], &a[2]);
#pragma unroll
                for (int u = 0; u < 4; u++) step(k + u, p2[u], a[u]);
                if ((all_done = __all_sync(0xffffffffu, done))) break;
            }
            if (!all_done)
                for (; k < cnt; k++) {
                    float p2, a;
                    alpha(k, &p2, &a);
                    step(k, p2, a);
                }
            if (last_k >= 0) last = s_pos[w][last_k] + 1u;
            if (__all_sync(0xffffffffu, done)) break;
        }
        if constexpr (RING) {
            cp_async_wait_all();                 // no gather into the ring outlives the item
            __syncwarp();
        }
        float ec = 0.f, ed = 0.f, nv = 0.f;
        if (inside) {
            const int HW = vp.W * vp.H;
            const int pix = py * vp.W + px;
            float* col = img.color + 3 * (size_t)vp.pix_base;
            const float fr = cr + Tr * rc.bg[0], fg = cg + Tr * rc.bg[1], fb = cb + Tr * rc.bg[2];
            col[pix] = fr;
            col[HW + pix] = fg;
            col[2 * HW + pix] = fb;
            img.depth[vp.pix_base + pix] = dd;
            img.T_final[vp.pix_base + pix] = Tr;
            img.n_contrib[vp.pix_base + pix] = last;
            if constexpr (LOSS) {
                cp_async_wait_all();             // this lane's own copies
                ec = fabsf(fr - s_tgt[w][0][lane]) + fabsf(fg - s_tgt[w][1][lane]) + fabsf(fb - s_tgt[w][2][lane]);
                const float tdv = s_tgt[w][3][lane];
                if (tdv > 0.f) {
                    ed = fabsf(dd - tdv);
                    nv = 1.f;
                }
            }
        }
        if constexpr (LOSS) {
            if (fl.item_cost != nullptr) {       // the block's deepest walk, for the backward's item order
                const uint32_t deepest = __reduce_max_sync(0xffffffffu, inside ? last : 0u);
                if (lane == 0) fl.item_cost[item] = deepest;
            }
            if (v != lv) {                       // rare: items of one view are taken together, except
                                                 // that the depth order may interleave views
                flush_lanes();
                lv = v;
            }
            s_lacc[w][0][lane] += ec;
            s_lacc[w][1][lane] += ed;
            s_lacc[w][2][lane] += nv;
        }
        __syncwarp();
    }
    if constexpr (LOSS) {
        flush_lanes();
        fused_loss_finish(fl, views, s_loss);
    }
}

// Transposed butterfly over the warp for two independent sets of 10 values:
// after 12 shuffle stages per set, lane l holds the full sum of slot
// 5 * b4 + 3 * b3 + 2 * b2 + b1 (bits of l) when that slot exists and l is even.
// The two sets' shuffles are interleaved so their latencies overlap.
__device__ __forceinline__ void warp_reduce10x2(const float (&va)[10], const float (&vb)[10], int lane, float* ua,
                                                float* ub) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    float ra[6], rb[6];
#pragma unroll
    for (int j = 0; j < 5; j++) {
        const float ka = b4 ? va[j + 5] : va[j], sa = b4 ? va[j] : va[j + 5];
        const float kb = b4 ? vb[j + 5] : vb[j], sb = b4 ? vb[j] : vb[j + 5];
        ra[j] = ka + __shfl_xor_sync(0xffffffffu, sa, 16);
        rb[j] = kb + __shfl_xor_sync(0xffffffffu, sb, 16);
    }
    ra[5] = 0.f; rb[5] = 0.f;
    float ta[4], tb[4];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const float ka = b3 ? ra[j + 3] : ra[j], sa = b3 ? ra[j] : ra[j + 3];
        const float kb = b3 ? rb[j + 3] : rb[j], sb = b3 ? rb[j] : rb[j + 3];
        ta[j] = ka + __shfl_xor_sync(0xffffffffu, sa, 8);
        tb[j] = kb + __shfl_xor_sync(0xffffffffu, sb, 8);
    }
    ta[3] = 0.f; tb[3] = 0.f;
    float wa[2], wb[2];
#pragma unroll
    for (int j = 0; j < 2; j++) {
        const float ka = b2 ? ta[j + 2] : ta[j], sa = b2 ? ta[j] : ta[j + 2];
        const float kb = b2 ? tb[j + 2] : tb[j], sb = b2 ? tb[j] : tb[j + 2];
        wa[j] = ka + __shfl_xor_sync(0xffffffffu, sa, 4);
        wb[j] = kb + __shfl_xor_sync(0xffffffffu, sb, 4);
    }
    float xa = (b1 ? wa[1] : wa[0]) + __shfl_xor_sync(0xffffffffu, b1 ? wa[0] : wa[1], 2);
    float xb = (b1 ? wb[1] : wb[0]) + __shfl_xor_sync(0xffffffffu, b1 ? wb[0] : wb[1], 2);
    xa += __shfl_xor_sync(0xffffffffu, xa, 1);
    xb += __shfl_xor_sync(0xffffffffu, xb, 1);
    *ua = xa;
    *ub = xb;
}

// Gradient slots per splat: 0 d mx, 1 d my, 2 d A, 3 d B, 4 d C, 5 d o, 6 d z,
// 7..9 d rgb; in the 12-float grad2d row slot s sits at s (s < 7) or s + 1.
__device__ __forceinline__ int slot_of_lane(int lane) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1;
    const int k = 3 * b3 + 2 * b2 + b1;
    if ((lane & 1) || (2 * b2 + b1) >= 3 || k >= 5) return -1;
    return 5 * b4 + k;
}

// Backward state of one pixel: transmittance after the current splat, the
// image gradients and the colour/depth behind the current splat normalised by
// that transmittance.
struct BwdPix {
    float T;
    uint32_t np;
    float gr, gg, gb, gd;
    float Sr, Sg, Sb, Sd;
};

// Branch-free: every lane evaluates the splat, and the ones that did not blend it
// in the forward pass (past their checkpoint, power > 0, alpha < alpha_min -- the
// forward's tests, written the same way) keep their state and contribute zeros:
// their alpha enters the updates as 0 (ac), so no select per update is needed.
// m = (mean x, mean y, list position, entry) with the last two as bit patterns;
// q = scaled conic + opacity (the decisions); c = the raw conic A, B, C (the
// gradient formulas).
__device__ __forceinline__ bool bwd_pixel(BwdPix& P, float sx, float sy, const float4 m, const float4 q,
                                          const float4 cd, const float4 c, float amin, float amax, float (&gv)[10]) {
    const float dx = __fsub_rn(sx, m.x), dy = __fsub_rn(sy, m.y);
    const float p2 = splat_power2(q.x, q.y, q.z, dx, dy);
    const float G = splat_weight(p2);
    const float araw = __fmul_rn(q.w, G);
    const float a = fminf(amax, araw);
    const bool blend = __float_as_uint(m.z) < P.np && !(p2 > 0.f) && !(a < amin);
    const float ac = blend ? a : 0.f;                     // alpha of a blended splat, else 0
    const float Tb = __fdividef(P.T, 1.0f - a);           // transmittance before this splat
    const float w = ac * Tb;
    const float dr = cd.x - P.Sr, dg = cd.y - P.Sg, db = cd.z - P.Sb, dz = cd.w - P.Sd;
    const float dLda = Tb * (dr * P.gr + dg * P.gg + db * P.gb + dz * P.gd);
    P.Sr = fmaf(ac, dr, P.Sr);
    P.Sg = fmaf(ac, dg, P.Sg);
    P.Sb = fmaf(ac, db, P.Sb);
    P.Sd = fmaf(ac, dz, P.Sd);
    P.T = blend ? Tb : P.T;
    const bool free_alpha = blend && araw < amax;        // alpha not clamped
    const float dpow = free_alpha ? dLda * a : 0.f;       // d alpha / d power = alpha
    const float e = dpow * dx, f = dpow * dy;             // power = -(A dx^2 + 2 B dx dy + C dy^2) / 2
    gv[0] = fmaf(c.x, e, c.y * f);                        // d mean x
    gv[1] = fmaf(c.y, e, c.z * f);                        // d mean y
    gv[2] = -0.5f * e * dx;                               // d A
    gv[3] = -e * dy;                                      // d B
    gv[4] = -0.5f * f * dy;                               // d C
    gv[5] = free_alpha ? dLda * G : 0.f;                  // d opacity: d alpha / d o = exp(power)
    gv[6] = P.gd * w;
    gv[7] = P.gr * w;
    gv[8] = P.gg * w;
    gv[9] = P.gb * w;
    return blend;
}

// A warp's kept splats of one batch in pairs (slots 2i, 2i + 1 as elements 0
// and 1 of pair i), so that the two splats' pixel-independent operands load as
// packed FP32x2 pairs.
struct BwdPairs {
    float4 nm[16];     // -mean x 0, -mean x 1, -mean y 0, -mean y 1
    float4 qab[16];    // scaled conic qa 0, qa 1, qb 0, qb 1
    float4 qco[16];    // qc 0, qc 1, opacity 0, opacity 1
    float4 rg[16];     // r 0, r 1, g 0, g 1
    float4 bz[16];     // b 0, b 1, z 0, z 1
    float4 ab[16];     // raw conic A 0, A 1, B 0, B 1
    float2 c[16];      // raw conic C 0, C 1
    uint4 pe[16];      // list position 0, 1, entry 0, 1
};

// Splat 1 of pair i (the farther) and then splat 0 for one pixel: bwd_pixel
// twice, with every operation that does not depend on the pixel's running state
// (transmittance, colour behind) done for both splats at once by packed FP32x2
// intrinsics, each element rounded as the scalar operation rounds it.  ga / gb
// receive splat 1's / splat 0's gradients; returns whether each blended.
__device__ __forceinline__ void bwd_pair(BwdPix& P, const float2 sx2, const float2 sy2, const BwdPairs& S, int i,
                                         float amin, float amax, float (&ga)[10], float (&gb)[10], bool* b1,
                                         bool* b0) {
    const float4 nm = S.nm[i], qab = S.qab[i], qco = S.qco[i], rg = S.rg[i], bz = S.bz[i], ab = S.ab[i];
    const float2 C = S.c[i];
    const uint4 pe = S.pe[i];
    const float2 dx = __fadd2_rn(sx2, make_float2(nm.x, nm.y)), dy = __fadd2_rn(sy2, make_float2(nm.z, nm.w));
    const float2 u = __ffma2_rn(make_float2(qab.z, qab.w), dy, __fmul2_rn(make_float2(qab.x, qab.y), dx));
    const float2 wq = __fmul2_rn(make_float2(qco.x, qco.y), dy);
    const float2 p2 = __ffma2_rn(dx, u, __fmul2_rn(wq, dy));
    const float2 G = make_float2(splat_weight(p2.x), splat_weight(p2.y));
    const float2 araw = __fmul2_rn(make_float2(qco.z, qco.w), G);
    const float a0 = fminf(amax, araw.x), a1 = fminf(amax, araw.y);
    const bool bl1 = pe.y < P.np && !(p2.y > 0.f) && !(a1 < amin);
    const bool bl0 = pe.x < P.np && !(p2.x > 0.f) && !(a0 < amin);
    const float ac1 = bl1 ? a1 : 0.f, ac0 = bl0 ? a0 : 0.f;
    const float2 om = __ffma2_rn(make_float2(-1.f, -1.f), make_float2(a0, a1), make_float2(1.f, 1.f));   // 1 - a
    // the running state, splat 1 then splat 0
    const float Tb1 = __fdividef(P.T, om.y);
    const float T1 = bl1 ? Tb1 : P.T;
    const float Tb0 = __fdividef(T1, om.x);
    P.T = bl0 ? Tb0 : T1;
    const float dr1 = rg.y - P.Sr, dg1 = rg.w - P.Sg, db1 = bz.y - P.Sb, dz1 = bz.w - P.Sd;
    P.Sr = fmaf(ac1, dr1, P.Sr);
    P.Sg = fmaf(ac1, dg1, P.Sg);
    P.Sb = fmaf(ac1, db1, P.Sb);
    P.Sd = fmaf(ac1, dz1, P.Sd);
    const float dr0 = rg.x - P.Sr, dg0 = rg.z - P.Sg, db0 = bz.x - P.Sb, dz0 = bz.z - P.Sd;
    P.Sr = fmaf(ac0, dr0, P.Sr);
    P.Sg = fmaf(ac0, dg0, P.Sg);
    P.Sb = fmaf(ac0, db0, P.Sb);
    P.Sd = fmaf(ac0, dz0, P.Sd);
    // gradients of both splats
    const float2 Tb = make_float2(Tb0, Tb1);
    const float2 w = __fmul2_rn(make_float2(ac0, ac1), Tb);
    float2 sum = __fmul2_rn(make_float2(dr0, dr1), make_float2(P.gr, P.gr));
    sum = __ffma2_rn(make_float2(dg0, dg1), make_float2(P.gg, P.gg), sum);
    sum = __ffma2_rn(make_float2(db0, db1), make_float2(P.gb, P.gb), sum);
    sum = __ffma2_rn(make_float2(dz0, dz1), make_float2(P.gd, P.gd), sum);
    const float2 dLda = __fmul2_rn(Tb, sum);
    const bool fr1 = bl1 && araw.y < amax, fr0 = bl0 && araw.x < amax;     // alpha not clamped
    const float2 dpa = __fmul2_rn(dLda, make_float2(a0, a1));               // d alpha / d power = alpha
    const float2 dpow = make_float2(fr0 ? dpa.x : 0.f, fr1 ? dpa.y : 0.f);
    const float2 e = __fmul2_rn(dpow, dx), f = __fmul2_rn(dpow, dy);
    const float2 A2 = make_float2(ab.x, ab.y), B2 = make_float2(ab.z, ab.w);
    const float2 g0 = __ffma2_rn(A2, e, __fmul2_rn(B2, f));                                 // d mean x
    const float2 g1 = __ffma2_rn(B2, e, __fmul2_rn(C, f));                                  // d mean y
    const float2 g2 = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), e), dx);             // d A
    const float2 g3 = __fmul2_rn(__fmul2_rn(make_float2(-1.f, -1.f), e), dy);               // d B
    const float2 g4 = __fmul2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), f), dy);             // d C
    const float2 gG = __fmul2_rn(dLda, G);                                                   // d alpha / d o = G
    const float2 g6 = __fmul2_rn(make_float2(P.gd, P.gd), w), g7 = __fmul2_rn(make_float2(P.gr, P.gr), w);
    const float2 g8 = __fmul2_rn(make_float2(P.gg, P.gg), w), g9 = __fmul2_rn(make_float2(P.gb, P.gb), w);
    ga[0] = g0.y; ga[1] = g1.y; ga[2] = g2.y; ga[3] = g3.y; ga[4] = g4.y;
    ga[5] = fr1 ? gG.y : 0.f; ga[6] = g6.y; ga[7] = g7.y; ga[8] = g8.y; ga[9] = g9.y;
    gb[0] = g0.x; gb[1] = g1.x; gb[2] = g2.x; gb[3] = g3.x; gb[4] = g4.x;
    gb[5] = fr0 ? gG.x : 0.f; gb[6] = g6.x; gb[7] = g7.x; gb[8] = g8.x; gb[9] = g9.x;
    *b1 = bl1;
    *b0 = bl0;
}

// Backward of one work item (pixel block blk of tile g) by one warp, using the
// warp's shared-memory slot S (its kept splats, in pairs).
template <int T, bool LOSS, bool MASKS>
__device__ __forceinline__ void bwd_item(
        int g, int blk, BwdPairs& S,
        const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
        const uint32_t* __restrict__ vals, const uint32_t* __restrict__ masks, const uint2* __restrict__ ranges,
        const Views& views, const RenderConsts& rc, const float* __restrict__ T_final,
        const uint32_t* __restrict__ n_contrib,
        const float* __restrict__ dL_dcolor, const float* __restrict__ dL_ddepth, float* __restrict__ g2d,
        const FusedLoss& fl) {
    const int lane = threadIdx.x & 31;
    const int v = view_of_tile(views, g);
    const ViewParams& vp = views.v[v];
    const int lt = g - vp.tile_base;
    const int tx = lt % vp.tiles_x, ty = lt / vp.tiles_x;
    int ox, oy;
    lane_pixel(T, blk * 32 + lane, &ox, &oy);
    const int px = tx * T + ox, py = ty * T + oy;
    const bool inside = px < vp.W && py < vp.H;
    const float sx = (float)px + 0.5f, sy = (float)py + 0.5f;
    const float2 sx2 = make_float2(sx, sx), sy2 = make_float2(sy, sy);
    const float bx0 = (float)(tx * T + (blk % (T / 8)) * 8) + 0.5f, by0 = (float)(ty * T + (blk / (T / 8)) * 4) + 0.5f;
    const float bx1 = bx0 + 7.f, by1 = by0 + 3.f;
    constexpr bool use_masks = MASKS;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint2 range = ranges[g];
    const float amin = rc.alpha_min, amax = rc.alpha_max;

    BwdPix P;
    P.np = 0; P.T = 1.f;
    P.gr = P.gg = P.gb = P.gd = 0.f;
    P.Sr = rc.bg[0]; P.Sg = rc.bg[1]; P.Sb = rc.bg[2]; P.Sd = 0.f;
    if (inside) {
        const int HW = vp.W * vp.H;
        const int pix = py * vp.W + px;
        P.T = T_final[vp.pix_base + pix];
        P.np = n_contrib[vp.pix_base + pix];
        if constexpr (LOSS) {
            // the gradient of Eq. 6's colour and depth L1 terms, as the stand-alone loss forms it
            const float* c = fl.color + 3 * (size_t)vp.pix_base;
            const float* t = fl.tc + 3 * (size_t)vp.pix_base;
            const float kc = fl.lc / (3.0f * (float)HW);
            const float nvalid = fl.acc[4 * v + 2];
            const float kd = nvalid > 0.f ? fl.ld / nvalid : 0.f;
            P.gr = kc * sgnf(c[pix] - t[pix]);
            P.gg = kc * sgnf(c[HW + pix] - t[HW + pix]);
            P.gb = kc * sgnf(c[2 * HW + pix] - t[2 * HW + pix]);
            const float tdv = fl.td[vp.pix_base + pix];
            P.gd = tdv > 0.f ? kd * sgnf(fl.depth[vp.pix_base + pix] - tdv) : 0.f;
        } else {
            const float* dc = dL_dcolor + 3 * (size_t)vp.pix_base;
            P.gr = dc[pix]; P.gg = dc[HW + pix]; P.gb = dc[2 * HW + pix];
            P.gd = dL_ddepth[vp.pix_base + pix];
        }
    }
    // this warp needs the list only up to its deepest pixel (a checkpoint never points past the list)
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, P.np);
    const uint32_t top = min(range.x + wmax, range.y);
    if (top <= range.x) return;
    const int slot = slot_of_lane(lane);
    const int col = slot < 7 ? slot : slot + 1;
    // batches of 32 list positions [lo, hi) walk down from top; the next batch's
    // splats and the list entries of the one below it are in flight in registers
    auto below = [&](uint32_t b) { return b > range.x + 32 ? b - 32 : range.x; };
    uint32_t lo = below(top);
    float2 n_xy = make_float2(0.f, 0.f);
    float4 n_q = make_float4(0.f, 0.f, 0.f, 0.f), n_cd = n_q, n_c = n_q;
    uint32_t n_e = 0, nn_e = 0, n_m = 0, nn_m = 0;    // list entries and their block masks
    const uint32_t bbit = 1u << blk;
    auto fetch = [&](uint32_t e, uint32_t m) {
        n_e = e;
        n_m = m;
        if (use_masks && (m & bbit) == 0u) return;     // culled by its mask: nothing to gather
        n_c = conic_o[e];
        scale_conic(n_c.x, n_c.y, n_c.z, &n_q.x, &n_q.y, &n_q.z);
        n_q.w = n_c.w;
        n_xy = xy[e];
        n_cd = rgbd[e];
    };
    if (lo + lane < top) fetch(vals[lo + lane], use_masks ? masks[lo + lane] : 0u);
    if (lo > range.x && below(lo) + lane < lo) {
        nn_e = vals[below(lo) + lane];
        if (use_masks) nn_m = masks[below(lo) + lane];
    }
    for (uint32_t hi = top; hi > range.x; hi = lo, lo = below(lo)) {
        const bool keep = lo + lane < hi && (use_masks ? (n_m & bbit) != 0u
                                                       : splat_reaches_block(n_xy, n_q, bx0, bx1, by0, by1, amin));
        const uint32_t kept = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {
            const int sl = __popc(kept & lt_mask), pi = sl >> 1, h = sl & 1;
            float* nm = reinterpret_cast<float*>(&S.nm[pi]);
            float* qab = reinterpret_cast<float*>(&S.qab[pi]);
            float* qco = reinterpret_cast<float*>(&S.qco[pi]);
            float* rg = reinterpret_cast<float*>(&S.rg[pi]);
            float* bz = reinterpret_cast<float*>(&S.bz[pi]);
            float* ab = reinterpret_cast<float*>(&S.ab[pi]);
            uint32_t* pe = reinterpret_cast<uint32_t*>(&S.pe[pi]);
            nm[h] = -n_xy.x; nm[2 + h] = -n_xy.y;
            qab[h] = n_q.x; qab[2 + h] = n_q.y;
            qco[h] = n_q.z; qco[2 + h] = n_q.w;
            rg[h] = n_cd.x; rg[2 + h] = n_cd.y;
            bz[h] = n_cd.z; bz[2 + h] = n_cd.w;
            ab[h] = n_c.x; ab[2 + h] = n_c.y;
            reinterpret_cast<float*>(&S.c[pi])[h] = n_c.z;
            pe[h] = lo + lane - range.x; pe[2 + h] = n_e;
        }
        __syncwarp();
        const uint32_t nlo = below(lo);
        if (lo > range.x && nlo + lane < lo) fetch(nn_e, nn_m);
        if (nlo > range.x && below(nlo) + lane < nlo) {
            nn_e = vals[below(nlo) + lane];
            if (use_masks) nn_m = masks[below(nlo) + lane];
        }
        const int cnt = __popc(kept);
        if (cnt & 1) {                       // the farthest kept splat alone: element 0 of the last pair
            const int pi = cnt >> 1;
            const float4 nm = S.nm[pi], qab = S.qab[pi], qco = S.qco[pi], rg = S.rg[pi], bz = S.bz[pi], ab = S.ab[pi];
            const uint4 pe = S.pe[pi];
            const float4 m = make_float4(-nm.x, -nm.z, __uint_as_float(pe.x), __uint_as_float(pe.z));
            float ga[10], gb[10];
            const bool ca = bwd_pixel(P, sx, sy, m, make_float4(qab.x, qab.z, qco.x, qco.z),
                                      make_float4(rg.x, rg.z, bz.x, bz.z), make_float4(ab.x, ab.z, S.c[pi].x, 0.f),
                                      amin, amax, ga);
#pragma unroll
            for (int r = 0; r < 10; r++) gb[r] = 0.f;
            if (__any_sync(0xffffffffu, ca)) {
                float ua, ub;
                warp_reduce10x2(ga, gb, lane, &ua, &ub);
                if (slot >= 0) atomicAdd(g2d + (size_t)kGradStride * pe.z + col, ua);
            }
        }
        for (int pi = (cnt >> 1) - 1; pi >= 0; pi--) {
            float ga[10], gb[10];
            bool ca, cb;
            bwd_pair(P, sx2, sy2, S, pi, amin, amax, ga, gb, &ca, &cb);
            const bool anya = __any_sync(0xffffffffu, ca), anyb = __any_sync(0xffffffffu, cb);
            if (anya || anyb) {
                float ua, ub;
                warp_reduce10x2(ga, gb, lane, &ua, &ub);
                if (slot >= 0) {
                    const uint4 pe = S.pe[pi];
                    if (anya) atomicAdd(g2d + (size_t)kGradStride * pe.w + col, ua);
                    if (anyb) atomicAdd(g2d + (size_t)kGradStride * pe.z + col, ub);
                }
            }
        }
    }
}

// Two occupancies (kCtas CTAs per SM): few work items per SM (a single 640x480
// view: ~60) run best with 2 CTAs and 90 registers, where the deepest blocks'
// chains are shorter; many (a keyframe window: ~900) with 3 CTAs and 80.
template <int T, int kCtas, bool LOSS, bool MASKS>
__global__ void __launch_bounds__(kRasterThreads, kCtas) k_render_bwd(
        const float2* __restrict__ xy, const float4* __restrict__ conic_o, const float4* __restrict__ rgbd,
        const uint32_t* __restrict__ vals, const uint32_t* __restrict__ masks, const uint2* __restrict__ ranges,
        Views views, RenderConsts rc, const float* __restrict__ T_final, const uint32_t* __restrict__ n_contrib,
        const float* __restrict__ dL_dcolor, const float* __restrict__ dL_ddepth, float* __restrict__ g2d,
        int* __restrict__ queue, int n_items, FusedLoss fl) {
    constexpr int W = TileShape<T>::kWarps;
    __shared__ BwdPairs s_pairs[kRasterWarps];
    pdl_enter();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WorkQueue wq(queue, n_items, LOSS && fl.order != nullptr);
    for (int raw = wq.first(lane); raw < n_items; raw = wq.next(lane)) {
        const int item = (LOSS && fl.order != nullptr) ? (int)fl.order[raw] : raw;
        bwd_item<T, LOSS, MASKS>(item / W, item % W, s_pairs[w], xy, conic_o, rgbd, vals, masks,
                          ranges, views, rc, T_final, n_contrib, dL_dcolor, dL_ddepth, g2d, fl);
        __syncwarp();
    }
}

}  // namespace

// The backward's item order: the forward's per-item costs (deepest n_contrib of
// the 8 x 4 block) counting-sorted in descending order (costs above the last
// bucket share it; items of one bucket in any order), so that the longest
// walks start first and the launch does not end on one deep block.  One CTA.
constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 2048;

__global__ void __launch_bounds__(kOrderThreads) k_item_order(const uint32_t* __restrict__ cost,
                                                              uint32_t* __restrict__ order, uint32_t* tag, int n,
                                                              float* __restrict__ zero, int64_t zero_n) {
    __shared__ uint32_t h[kOrderBuckets];
    __shared__ uint32_t s_warp[kOrderThreads / 32];
    pdl_enter();
    if (blockIdx.x > 0) {            // the other CTAs zero the backward's 2D-gradient accumulators meanwhile
        const int64_t stride = (int64_t)(gridDim.x - 1) * kOrderThreads;
        const int64_t t0 = (int64_t)(blockIdx.x - 1) * kOrderThreads + threadIdx.x;
        for (int64_t k = t0; k < zero_n / 4; k += stride)
            reinterpret_cast<float4*>(zero)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t k = zero_n / 4 * 4 + t0; k < zero_n; k += stride) zero[k] = 0.f;
        return;
    }
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    auto bucket = [](uint32_t c) { return (uint32_t)(kOrderBuckets - 1) - min(c, (uint32_t)(kOrderBuckets - 1)); };
    for (int k = t; k < kOrderBuckets; k += kOrderThreads) h[k] = 0u;
    __syncthreads();
    for (int i = t; i < n; i += kOrderThreads) atomicAdd(&h[bucket(cost[i])], 1u);
    __syncthreads();
    // exclusive scan of the 2048 buckets, two per thread
    const uint32_t a = h[2 * t], b = h[2 * t + 1];
    uint32_t inc = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t wv = s_warp[lane];
        uint32_t wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_warp[lane] = wi - wv;
    }
    __syncthreads();
    const uint32_t excl = s_warp[warp] + inc - (a + b);
    h[2 * t] = excl;
    h[2 * t + 1] = excl + a;
    __syncthreads();
    for (int i = t; i < n; i += kOrderThreads) order[atomicAdd(&h[bucket(cost[i])], 1u)] = (uint32_t)i;
    __syncthreads();
    if (t == 0) {                                 // the order now holds a permutation of the n items
        tag[0] = (uint32_t)n;
        tag[1] = (uint32_t)n ^ kOrderTagMagic;
    }
}
static_assert(kOrderBuckets == 2 * kOrderThreads, "two buckets per thread in the scan");

// A launch with at most this many 8 x 4 pixel blocks per SM (a single 640x480
// view: ~60) is "few": its time is bounded by its deepest blocks' walks, so both
// passes take the blocks deepest first, the forward keeps two batches in flight
// per warp and the backward runs 2 CTAs per SM (90 registers); a keyframe window
// (~900 per SM) is bound by throughput instead.
constexpr int kFewItemsPerSm = 256;

// CTAs of a persistent raster launch: every SM filled to the kernel's occupancy
// (host-side occupancy query; no stream operation, so it may run during capture).
template <typename K>
static int persistent_grid(K kernel, int n_items) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRasterThreads, 0);
    if (per_sm < 1) per_sm = 1;
    const int want = (n_items + kRasterWarps - 1) / kRasterWarps;
    const int g = sms * per_sm;
    return want < g ? want : g;
}

size_t fused_loss_workspace(int32_t n_views) {
    return align_up(sizeof(float) * 4 * (size_t)n_views, 256) +
           align_up(sizeof(float) * (size_t)kFusedMaxCtas * n_views * 3, 256) + 256 +
           2 * sizeof(uint32_t) * kOrderMaxItems;
}

void fused_loss_layout(void* ws, int32_t n_views, FusedLoss* fl) {
    char* p = static_cast<char*>(ws);
    fl->acc = reinterpret_cast<float*>(p);
    p += align_up(sizeof(float) * 4 * (size_t)n_views, 256);
    fl->partial = reinterpret_cast<float*>(p);
    p += align_up(sizeof(float) * (size_t)kFusedMaxCtas * n_views * 3, 256);
    fl->order_tag = reinterpret_cast<uint32_t*>(p);
    p += 256;
    fl->item_cost = reinterpret_cast<uint32_t*>(p);
    fl->order = fl->item_cost + kOrderMaxItems;
}

// One tile size and mask mode of the forward launch: the fused-loss or plain
// kernel, with one or two batches of splats in flight per warp.
template <int TT, bool M>
static cudaError_t fwd_tile(const float2* xy, const float4* co, const float4* cd, const gs_bins& bins,
                            const uint2* rg, const Views& views, const RenderConsts& rc, const gs_image& img,
                            int* queue, int sms, cudaStream_t s, const FusedLoss* fl) {
    const int n_items = views.total_tiles * TileShape<TT>::kWarps;
    const bool few = rc.splat_stages == 0 ? n_items <= kFewItemsPerSm * sms : rc.splat_stages == 3;
    if (fl) {
        const int grid = few ? persistent_grid(k_render_fwd<TT, true, true, M>, n_items)
                             : persistent_grid(k_render_fwd<TT, true, false, M>, n_items);
        if (grid > kFusedMaxCtas) return cudaErrorInvalidConfiguration;
        FusedLoss f = *fl;
        if (n_items > kOrderMaxItems) f.item_cost = f.order = nullptr;
        return few ? launch_pdl(k_render_fwd<TT, true, true, M>, grid, kRasterThreads, 0, s, xy, co, cd, bins.vals,
                                bins.masks, rg, views, rc, img, queue, n_items, f)
                   : launch_pdl(k_render_fwd<TT, true, false, M>, grid, kRasterThreads, 0, s, xy, co, cd, bins.vals,
                                bins.masks, rg, views, rc, img, queue, n_items, f);
    }
    const int grid = few ? persistent_grid(k_render_fwd<TT, false, true, M>, n_items)
                         : persistent_grid(k_render_fwd<TT, false, false, M>, n_items);
    return few ? launch_pdl(k_render_fwd<TT, false, true, M>, grid, kRasterThreads, 0, s, xy, co, cd, bins.vals,
                            bins.masks, rg, views, rc, img, queue, n_items, FusedLoss{})
               : launch_pdl(k_render_fwd<TT, false, false, M>, grid, kRasterThreads, 0, s, xy, co, cd, bins.vals,
                            bins.masks, rg, views, rc, img, queue, n_items, FusedLoss{});
}

cudaError_t launch_render_fwd(const gs_projected& pr, const gs_bins& bins, const Views& views,
                              const RenderConsts& rc, const gs_image& img, cudaStream_t s, const FusedLoss* fl) {
    if (views.total_tiles == 0) return cudaSuccess;
    const float2* xy = reinterpret_cast<const float2*>(pr.xy);
    const float4* co = reinterpret_cast<const float4*>(pr.conic_o);
    const float4* cd = reinterpret_cast<const float4*>(pr.rgbd);
    const uint2* rg = reinterpret_cast<const uint2*>(bins.ranges);
    int* queue = bins.status + 1;      // zero between launches (see WorkQueue)
    cudaError_t e = cudaSuccess;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int pick = rc.block_masks ? 1 : 0;
#define ARGS_FWD xy, co, cd, bins, rg, views, rc, img, queue, sms, s, fl
    switch (rc.tile) {
        case 8: e = pick ? fwd_tile<8, true>(ARGS_FWD) : fwd_tile<8, false>(ARGS_FWD); break;
        case 16: e = pick ? fwd_tile<16, true>(ARGS_FWD) : fwd_tile<16, false>(ARGS_FWD); break;
        case 32: e = pick ? fwd_tile<32, true>(ARGS_FWD) : fwd_tile<32, false>(ARGS_FWD); break;
        default: return cudaErrorInvalidValue;
    }
#undef ARGS_FWD
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const gs_projected& pr, const gs_bins& bins, const gs_image& img, const float* dc,
                              const float* dd, const Views& views, const RenderConsts& rc, float* g2d,
                              int64_t g2d_zero, cudaStream_t s, const FusedLoss* fl) {
    if (views.total_tiles == 0) return launch_zero(g2d, g2d_zero, nullptr, 0, nullptr, 0, s);
    const float2* xy = reinterpret_cast<const float2*>(pr.xy);
    const float4* co = reinterpret_cast<const float4*>(pr.conic_o);
    const float4* cd = reinterpret_cast<const float4*>(pr.rgbd);
    const uint2* rg = reinterpret_cast<const uint2*>(bins.ranges);
    int* queue = bins.status + 2;      // zero between launches (see WorkQueue)
    cudaError_t e = cudaSuccess;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

#define GS_BWD_LAUNCH_M(TT, C, L, M, F)                                                                \
    launch_pdl(k_render_bwd<TT, C, L, M>, persistent_grid(k_render_bwd<TT, C, L, M>, n_items), kRasterThreads, 0, \
               s, xy, co, cd, bins.vals, bins.masks, rg, views, rc, img.T_final, img.n_contrib, dc, dd, g2d, queue, \
               n_items, F)
#define GS_BWD_LAUNCH(TT, C, L, F) \
    (rc.block_masks ? GS_BWD_LAUNCH_M(TT, C, L, true, F) : GS_BWD_LAUNCH_M(TT, C, L, false, F))
    switch (rc.tile) {
#define GS_BWD(TT)                                                                                     \
    case TT: {                                                                                         \
        const int n_items = views.total_tiles * TileShape<TT>::kWarps;                                \
        const bool few = n_items <= kFewItemsPerSm * sms;                                             \
        FusedLoss f = fl ? *fl : FusedLoss{};                                                          \
        /* few items per SM: deepest blocks first (costs from the fused forward); the order's launch  \
           zeroes the 2D gradients with its other CTAs, else a zero-fill launch does */                \
        if (fl && few && n_items <= kOrderMaxItems) {                                                  \
            const int64_t zb = ceil_div(g2d_zero / 4 + 1, (int64_t)kOrderThreads);                     \
            e = launch_pdl(k_item_order, (unsigned)(1 + (zb < 2 * sms ? zb : 2 * sms)), kOrderThreads, 0, s, \
                           (const uint32_t*)f.item_cost, f.order, f.order_tag, n_items, g2d, g2d_zero); \
        } else {                                                                                       \
            f.order = nullptr;                                                                         \
            e = launch_zero(g2d, g2d_zero, nullptr, 0, nullptr, 0, s);                                 \
        }                                                                                              \
        if (e != cudaSuccess) return e;                                                                \
        if (few && fl)                                                                                 \
            e = GS_BWD_LAUNCH(TT, 2, true, f);                                                         \
        else if (few)                                                                                  \
            e = GS_BWD_LAUNCH(TT, 2, false, FusedLoss{});                                              \
        else if (fl)                                                                                   \
            e = GS_BWD_LAUNCH(TT, 3, true, f);                                                         \
        else                                                                                           \
            e = GS_BWD_LAUNCH(TT, 3, false, FusedLoss{});                                              \
        break;                                                                                         \
    }
        GS_BWD(8)
        GS_BWD(16)
        GS_BWD(32)
#undef GS_BWD
#undef GS_BWD_LAUNCH
#undef GS_BWD_LAUNCH_M
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace gs
