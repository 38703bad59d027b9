// exw_engine.cuh -- the forward pass (stages (a0), (a), (b), (c) for P_1..P_3, Sec. IV-B) of any number of frames
// or streams as ONE warp-specialised persistent kernel: one CTA per SM, 25 warps.
//
// Work items of all streams (a stream = one source frame with its outputs) sit in one queue, laid out diagonally --
// motion-bounds regions of stream d, tile plans of stream d-1, target tiles of stream d-2, fix-ups of stream d-3
// -- so an item's dependencies (the previous stage of its own stream) come earlier in the queue.
//
//   producer warp:   takes items in queue order, waits (bounded) until the item's stage may start, and hands the
//                    item to the consumers in one of two shared-memory slots.  For a target tile it stages the
//                    tile's source window (depth, motion, colour) into the slot's buffer with TMA loads
//                    (cp.async.bulk.tensor, mbarrier completion) and, while they land, writes the tile's plan, its
//                    splat candidates and the per-fraction constants of uniform tiles, one item ahead of the
//                    consumers.
//   3 x 8 consumer warps: a bounds item gives each half group one 32 x 32 source region, a plan item each warp one
//                    target tile, a fix-up item all of them a slice; for a target tile all of them splat (modes
//                    1-3), then group g computes fraction k0 + g -- each thread a 2 x 2 pixel block -- fills and
//                    stores it.  Every consumer warp releases the slot through a second mbarrier.  Only the slots
//                    whose groups share state start with a consumer-wide vote (engine_consumer).
//
// Tiles whose candidate sources all carry one motion (plan modes 0 and 5) are pure translations: the winner of
// target q is the source q - o_k when that pixel is valid and carries the tile's motion, so no splat is needed.
// Other tiles splat their candidate sources into per-fraction region keys (from the window, or from global memory
// when the landing rectangle is wider than a window) and gather through the keys.  Every result is bit-identical
// to the per-tile passes of exw_tile.cuh (same arithmetic in the same order).
#pragma once

#include "exw_items.cuh"
#include "exw_tma.cuh"

namespace exw {

constexpr int kGroupThreads = 256;                          // one fraction: 16 x 16 blocks of 2 x 2 pixels
constexpr int kConsumerThreads = kMaxFrac * kGroupThreads;  // 768
constexpr int kConsumerWarps = kConsumerThreads / 32;       // 24
constexpr int kEngineThreads = kConsumerThreads + 32;       // + the producer warp
constexpr int kBarConsumers = 1;                            // named barriers: 1 all consumers, 2 + g group g,
constexpr int kBarBounds = 11;  // 5 + h half group h (bounds), 11 + g group g (bounds)
constexpr int kMaxStreams = 48;                             // streams per launch (kernel-parameter space)
constexpr int kRegionsPerHalf = 4;  // a bounds item: four regions per half group (4 warps), one after the other
constexpr int kRegionsPerItem = 2 * kMaxFrac * kRegionsPerHalf;
constexpr int kPlansPerWarp = 2;                            // a plan item: two tiles per consumer warp
constexpr int kPlansPerItem = kConsumerWarps * kPlansPerWarp;
constexpr uint32_t kFixupItems = 8u;                        // fix-up items per stream (with the fill)
// Every wait of the engine is bounded in time.  The producer gives up on a stage or on a buffer's release after
// kProducerWaitNs, and then hands no further slot over (it raises the abort flag); a consumer gives up on a slot
// only after kConsumerWaitNs, four times longer, and waits for a slot only once the producer has handed over the
// previous one.  So a consumer never gives up on a slot the producer still hands over: all consumers take the same
// slots, which lets the slots without a consumer-wide vote use group barriers.
constexpr uint64_t kProducerWaitNs = 1000000000ull;
constexpr uint64_t kConsumerWaitNs = 4000000000ull;
constexpr uint64_t kInjectedWaitNs = 5000000ull;  // the injected fault gives up after 5 ms

// Slot kinds.
constexpr int kSlotEnd = 0, kSlotBounds = 1, kSlotPlans = 2, kSlotTile = 3, kSlotFixup = 4;

// Per stream, in the kernel parameters.
struct EngineStream {
    TileParams p;
    int cdt;     // EXW_F32 / EXW_F16
    int tma;     // stage this stream's tiles with TMA windows (else every tile reads global memory)
    int nregions, ntiles, nfix;
};
struct EngineSeg {
    int start;         // first queue index of the segment
    uint16_t stream;
    uint16_t stage;    // 0 bounds, 1 plans, 2 tiles, 3 fix-up
};
struct EngineParams {
    int n, nseg, total, inject;
    int pair_smooth;  // two smooth tiles of a stream that follow each other share one slot
    uint64_t ahead;  // streams whose bounds and plans were computed before the launch (bit s = stream s)
    uint32_t *queue, *status;
    EngineStream st[kMaxStreams];
    EngineSeg seg[4 * kMaxStreams];
    CUtensorMap maps[kMaxStreams][3];  // colour, depth, motion
};

// Per-fraction constants of a uniform tile (computed by the producer).
struct alignas(16) UniformFrac {  // 16-byte aligned: its fields load as vectors
    int ox, oy;               // whole-pixel offset o_k
    uint32_t flags;           // kTapX, kTapY: a tap column / row exists; kMirX, kMirY: taps at -1
    float W00, W10, W01, W11; // bilinear weights, constant over the tile
    float inv[8];             // 1 / (sum of the weights of tap subset j), j = a10 | a01 << 1 | a11 << 2
};
constexpr uint32_t kTapX = 1u, kTapY = 2u, kMirX = 4u, kMirY = 8u;

// The scalars of a stream the per-pixel code needs, held in registers for a whole tile (the slot's parameters sit
// in shared memory, and every barrier would otherwise reload them).
struct FrameDims {
    int W, H, L, k0, nfrac;
};
__device__ __forceinline__ FrameDims dims_of(const TileParams &p) { return FrameDims{p.W, p.H, p.L, p.k0, p.nfrac}; }

// What the producer hands the consumers with each buffer.
struct alignas(16) TileSlot {
    int kind, stream, index, cdt;  // the stream's parameters are read from the launch's (ep.st[stream].p)
    TilePlan plan;            // tile: its plan (mode 3 for every tile of a stream without TMA windows)
    int X0, Y0;
    UniformFrac u[kMaxFrac];  // modes 0, 5
    // mode 5: a second smooth tile of the same stream, the next in the queue, shares the slot (its colour window
    // follows the first one's in the buffer)
    int pair, index2, X02, Y02, wx02, wy02;
    union {
        SplatTile pdesc[kPlanDesc];  // modes 1-3: the plan's candidates of the tile
        UniformFrac u2[kMaxFrac];    // mode 5, paired: the second tile's constants
    };
};

constexpr int kWindowBytes = 64512;  // both window shapes (56 x 48 FP32, 64 x 56 FP16) hold 64,512 bytes
static_assert(64 * 16 * kConsumerWarps <= kWindowBytes, "the coarse pass's per-warp scratch fits one buffer");
static_assert(sizeof(SplatTile) == sizeof(float4), "the candidate list doubles as one float4 per consumer thread");
static_assert(2 * kRegionsPerHalf * 32 <= kGroupThreads, "a bounds item's partials (32 float4 a region) fit a group's scratch");
static_assert(sizeof(Window<float, WinShape<0>::xf32, WinShape<0>::yf32>) == kWindowBytes &&
                  sizeof(Window<__half, WinShape<0>::xf16, WinShape<0>::yf16>) == kWindowBytes &&
                  sizeof(Window<float, WinShape<1>::xf32, WinShape<1>::yf32>) == kWindowBytes &&
                  sizeof(Window<__half, WinShape<1>::xf16, WinShape<1>::yf16>) == kWindowBytes,
              "one buffer size for every shape and colour type");

struct EngineSmem {
    alignas(128) unsigned char win[2][kWindowBytes];  // TMA destinations, double-buffered
    uint64_t key[2][kMaxFrac][kRegionN];             // region keys per fraction (modes 1-3), a set per splat slot parity
    TileSlot slot[2];                                // the item in each buffer
    // A splat's candidate list; between splats per group 256 float4 of scratch (group g from float4 256 g): the fill's
    // pyramid (32 per warp: level 1 of its blocks, then level 2 in the first 8 and levels 3-4 in the next 20) and a
    // bounds item's partials (the first 64)
    SplatTile cand[kConsumerThreads];
    uint32_t ncand;
    uint32_t snext[2];                               // the next splat chunk of the tile in each buffer
    int abort;                                       // a bounded wait ran out: every warp leaves
    uint64_t full[2], empty[2];
};

// The shared memory stays within the 196 KB carve-out (with the 1 KB the system keeps per CTA): the next larger one
// leaves 28 KB of L1 instead of 60, which measured 6% slower at 1080p.
static_assert(sizeof(EngineSmem) <= 196 * 1024 - 1024, "the engine's shared memory fits the 196 KB carve-out");

template <typename CT, int WX, int WY>
__device__ __forceinline__ Window<CT, WX, WY> &window(EngineSmem &s, int b) {
    return *reinterpret_cast<Window<CT, WX, WY> *>(s.win[b]);
}

// ------------------------------------------------------------------------------------------------------------
// Barriers
// ------------------------------------------------------------------------------------------------------------
__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Barrier over n threads that also returns whether any of them passed v = true.
__device__ __forceinline__ bool bar_red_or(int id, int n, bool v) {
    uint32_t r;
    asm volatile(
        "{\n"
        " .reg .pred p, q;\n"
        " setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, %2, %3, p;\n"
        " selp.u32 %0, 1, 0, q;\n"
        "}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(n)
        : "memory");
    return r != 0u;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}
// Wait on an mbarrier phase for at most limit_ns; gives up early when another warp raised the abort flag.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *mbar, uint32_t parity, const volatile int *abort,
                                                   uint64_t limit_ns) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(mbar, parity)) return true;
        if ((i & 15u) == 0u) {
            if (*abort || globaltimer_ns() - t0 > limit_ns) return false;
            __nanosleep(64);
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Producer
// ------------------------------------------------------------------------------------------------------------

// Constants of fraction kk of a uniform tile, by the lanes 8 kk .. 8 kk + 7 of the producer warp (lane 8 kk + j
// writes inv[j]).
__device__ __forceinline__ void uniform_frac(UniformFrac &u, const TileParams &p, uint32_t umx, uint32_t umy, int kk,
                                             int j) {
    const int k = p.k0 + kk;
    const int ox = axis_off_of(umx, k, p.L), oy = axis_off_of(umy, k, p.L);
    int sx, sy;
    const float rx = residual(__uint_as_float(umx), k, p.L, ox, sx);
    const float ry = residual(__uint_as_float(umy), k, p.L, oy, sy);
    const float wx1 = fabsf(rx), wy1 = fabsf(ry);
    const float wx0 = 1.0f - wx1, wy0 = 1.0f - wy1;
    const float W00 = __fmul_rn(wx0, wy0), W10 = __fmul_rn(wx1, wy0), W01 = __fmul_rn(wx0, wy1),
                W11 = __fmul_rn(wx1, wy1);
    u.inv[j] = __frcp_rn(weight_sum(W00, (j & 1) ? W10 : 0.0f, (j & 2) ? W01 : 0.0f, (j & 4) ? W11 : 0.0f));
    if (j == 0) {
        u.ox = ox;
        u.oy = oy;
        u.flags = (sx != 0 ? kTapX : 0u) | (sy != 0 ? kTapY : 0u) | (sx < 0 ? kMirX : 0u) | (sy < 0 ? kMirY : 0u);
        u.W00 = W00;
        u.W10 = W10;
        u.W01 = W01;
        u.W11 = W11;
    }
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Lane 0 waits until *counter >= target; false when the limit ran out, the workspace status reports an error or
// the CTA aborts.
__device__ __forceinline__ bool stage_wait(const uint32_t *counter, uint32_t target, uint64_t limit_ns,
                                           const uint32_t *status, const volatile int *abort) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 0;; ++i) {
        if (ld_acquire(counter) >= target) return true;
        if (*(const volatile uint32_t *)status != 0u || *abort || globaltimer_ns() - t0 > limit_ns) return false;
        __nanosleep(i < 64 ? 32 : 256);
    }
}

struct QueueItem {
    int item, stream, stage, local;  // item >= total: no more items
};

// A producer's items increase, so its segment index only moves forward: seg is the last segment found.
__device__ __forceinline__ QueueItem decode(const EngineParams &ep, int item, int &seg) {
    QueueItem q{item, 0, 0, 0};
    if (item < ep.total) {
        while (seg + 1 < ep.nseg && ep.seg[seg + 1].start <= item) ++seg;
        q.stream = ep.seg[seg].stream;
        q.stage = ep.seg[seg].stage;
        q.local = item - ep.seg[seg].start;
    }
    return q;
}

template <int SHAPE>
__device__ inline void engine_producer(EngineSmem &s, const EngineParams &ep) {
    using WS = WinShape<SHAPE>;
    constexpr int kWords = (int)(sizeof(TilePlan) / 4);
    const int lane = threadIdx.x & 31;
    // streams whose previous stage is known complete (the injected fault makes stream 0's tiles wait)
    uint64_t planned = ep.ahead & (ep.inject ? ~1ull : ~0ull), bounded = ep.ahead, coarsed = 0ull;
    // Two items of look-ahead: the queue position of item i + 2 and, when its stream's plans are known complete,
    // the plan of item i + 1 are requested while item i is handed over.
    int qa = 0, qb = 0;
    if (lane == 0) {
        qa = (int)atomicAdd(ep.queue, 1u);
        qb = qa < ep.total ? (int)atomicAdd(ep.queue, 1u) : ep.total;
    }
    int seg = 0;
    QueueItem cur = decode(ep, __shfl_sync(0xFFFFFFFFu, qa, 0), seg);
    int word = 0;
    bool have_word = false, have_desc = false;
    uint4 desc0 = make_uint4(0u, 0u, 0u, 0u), desc1 = desc0;  // the current item's candidates (look-ahead)
    for (uint32_t i = 0;; ++i) {
        const int b = (int)(i & 1u);
        const QueueItem nxt = decode(ep, cur.item < ep.total ? __shfl_sync(0xFFFFFFFFu, qb, 0) : ep.total, seg);
        if (lane == 0 && nxt.item < ep.total) qb = (int)atomicAdd(ep.queue, 1u);
        int nword = 0;
        bool nhave = false, nhave_desc = false;
        uint4 ndesc0 = make_uint4(0u, 0u, 0u, 0u), ndesc1 = ndesc0;
        if (nxt.item < ep.total && nxt.stage == 2 && (planned & (1ull << nxt.stream))) {
            const TileParams &np = ep.st[nxt.stream].p;
            nword = lane < kWords ? __ldcg(reinterpret_cast<const int *>(np.plans + nxt.local) + lane) : 0;
            nhave = true;
            // and its splat candidates (what the next slot copies into shared memory)
            const int nm = __shfl_sync(0xFFFFFFFFu, nword, 0), nd = __shfl_sync(0xFFFFFFFFu, nword, 3);
            if (nm >= 1 && nm <= 3 && nd > 0) {
                const uint4 *src = reinterpret_cast<const uint4 *>(np.pdesc + (size_t)nxt.local * kPlanDesc);
                if (lane < nd) ndesc0 = __ldcg(src + lane);
                if (lane + 32 < nd) ndesc1 = __ldcg(src + lane + 32);
                nhave_desc = true;
            }
        }
        const int item = cur.item, stream = cur.stream, stage = cur.stage, local = cur.local;
        const EngineStream &st = ep.st[stream];
        const TileParams &p = st.p;
        bool ok = true;
        // the item's stage may start once the previous stage of its stream is complete
        if (item < ep.total && stage > 0) {
            const uint64_t bit = 1ull << stream;
            const uint64_t known = stage == 1 ? bounded : stage == 2 ? planned : coarsed;
            if (!(known & bit)) {
                const bool injected = ep.inject && stream == 0 && stage == 2;
                // fix-ups: item 0 (the coarse pass) waits for every (tile, fraction) count, the others for it
                const bool first_fix = stage == 3 && local == 0;
                const uint32_t *counter = stage == 1 ? &p.fh->bdone
                                          : stage == 2 ? &p.fh->pdone
                                          : first_fix ? &p.fh->done : &p.fh->cready;
                const uint32_t target = stage == 1   ? (uint32_t)st.nregions
                                        : stage == 2 ? (uint32_t)st.ntiles + (injected ? 1u : 0u)
                                        : first_fix  ? (uint32_t)st.ntiles * (uint32_t)p.nfrac : 1u;
                if (lane == 0)
                    ok = stage_wait(counter, target, injected ? kInjectedWaitNs : kProducerWaitNs, ep.status,
                                    &s.abort);
                ok = __shfl_sync(0xFFFFFFFFu, (int)ok, 0) != 0;
                if (ok && !first_fix) {
                    if (stage == 1) bounded |= bit;
                    else if (stage == 2) planned |= bit;
                    else coarsed |= bit;
                }
            }
        }
        // A fix-up item of a stream where every tile of every fraction has a valid pixel has nothing to do: it takes
        // no slot (the stream's tile count, complete here, covers every count of tiles without one); for the first
        // item the producer releases the stream's other fix-ups itself.
        if (ok && item < ep.total && stage == 3) {
            bool none = true;
            if (lane == 0)
                for (int kk = 0; kk < p.nfrac; ++kk) none = none && __ldcg(&p.fh->ninvalid[kk]) == 0u;
            if (__shfl_sync(0xFFFFFFFFu, (int)none, 0) != 0) {
                if (lane == 0 && local == 0)
                    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&p.fh->cready), "r"(1u) : "memory");
                cur = nxt;
                word = nword;
                have_word = nhave;
                have_desc = nhave_desc;
                desc0 = ndesc0;
                desc1 = ndesc1;
                --i;  // no slot was handed over: the next item takes this one
                continue;
            }
        }
        if (ok && i >= 2) {  // the consumers' release of this buffer's previous use
            if (lane == 0) ok = mbar_wait_or_abort(&s.empty[b], ((i >> 1) - 1u) & 1u, &s.abort, kProducerWaitNs);
            ok = __shfl_sync(0xFFFFFFFFu, (int)ok, 0) != 0;
        }
        if (!ok) {
            if (lane == 0) {
                atomicCAS(ep.status, 0u, (uint32_t)EXW_ERR_TIMEOUT);
                *(volatile int *)&s.abort = 1;
                // the CTA must not end while a window it requested is still landing in its shared memory: wait
                // (bounded) for the last two slots handed over, whose copies the consumers may not have waited for
                for (uint32_t j = i >= 2u ? i - 2u : 0u; j < i; ++j)
                    mbar_wait_bounded(&s.full[j & 1u], (j >> 1) & 1u, kWaitLimit);
            }
            return;
        }
        TileSlot &sl = s.slot[b];
        if (item >= ep.total) {
            if (lane == 0) {
                sl.kind = kSlotEnd;
                mbar_arrive(&s.full[b]);
            }
            return;
        }
        const int kind = stage == 0 ? kSlotBounds : stage == 1 ? kSlotPlans : stage == 2 ? kSlotTile : kSlotFixup;
        int mode = -1, wx0 = 0, wy0 = 0, wx02 = 0, wy02 = 0;
        bool pair = false;
        if (kind == kSlotTile) {
            if (!have_word) word = lane < kWords ? __ldcg(reinterpret_cast<const int *>(p.plans + local) + lane) : 0;
            mode = __shfl_sync(0xFFFFFFFFu, word, 0);
            wx0 = __shfl_sync(0xFFFFFFFFu, word, 1);
            wy0 = __shfl_sync(0xFFFFFFFFu, word, 2);
            const int ndesc = __shfl_sync(0xFFFFFFFFu, word, 3);
            if (!st.tma && mode != 4) mode = 3;  // no window: every tile reads global memory
            // two smooth tiles in a row (the second one's plan already read): one slot, one pass of the pipeline
            pair = ep.pair_smooth && mode == 5 && nhave && nxt.stream == stream && nxt.stage == 2 &&
                   __shfl_sync(0xFFFFFFFFu, nword, 0) == 5;
            if (pair) {
                wx02 = __shfl_sync(0xFFFFFFFFu, nword, 1);
                wy02 = __shfl_sync(0xFFFFFFFFu, nword, 2);
            }
            // the window copies first: they land while the rest of the slot is written (the slot's arrival, last,
            // completes the phase together with their bytes)
            if (lane == 0 && (mode == 0 || mode == 1 || mode == 5)) {
                const CUtensorMap *m = ep.maps[stream];
                unsigned char *wb = s.win[b];
                // a window holds npx pixels: depth (4 B), motion (8 B), colour (3 c B) planes in this order
                const int npx = st.cdt == EXW_F16 ? WS::xf16 * WS::yf16 : WS::xf32 * WS::yf32;
                const uint32_t cbytes = (uint32_t)npx * 3u * (st.cdt == EXW_F16 ? 2u : 4u);
                fence_proxy_async_smem();
                if (mode == 5) {  // smooth: only the colour is read, at the buffer's start
                    mbar_expect_tx(&s.full[b], pair ? 2u * cbytes : cbytes);
                    tma_load_3d(wb, &m[0], wx0, wy0, 0, &s.full[b]);
                    if (pair) tma_load_3d(wb + cbytes, &m[0], wx02, wy02, 0, &s.full[b]);
                } else {
                    mbar_expect_tx(&s.full[b], (uint32_t)kWindowBytes);
                    tma_load_2d(wb, &m[1], wx0, wy0, &s.full[b]);
                    tma_load_3d(wb + 4 * npx, &m[2], wx0, wy0, 0, &s.full[b]);
                    tma_load_3d(wb + 12 * npx, &m[0], wx0, wy0, 0, &s.full[b]);
                }
            }
            if (lane < kWords) reinterpret_cast<int *>(&sl.plan)[lane] = word;
            const int X0 = (local % p.n5x) * kFillTile, Y0 = (local / p.n5x) * kFillTile;
            if (mode >= 1 && mode <= 3 && ndesc > 0) {  // the splat's candidates, as the plan found them
                uint4 *dst = reinterpret_cast<uint4 *>(sl.pdesc);
                if (have_desc) {  // loaded with the look-ahead
                    if (lane < ndesc) dst[lane] = desc0;
                    if (lane + 32 < ndesc) dst[lane + 32] = desc1;
                } else {
                    const uint4 *src = reinterpret_cast<const uint4 *>(p.pdesc + (size_t)local * kPlanDesc);
                    if (lane < ndesc) dst[lane] = __ldcg(src + lane);
                    if (lane + 32 < ndesc) dst[lane + 32] = __ldcg(src + lane + 32);
                }
            }
            if (mode == 0 || mode == 5) {
                const uint32_t umx = (uint32_t)__shfl_sync(0xFFFFFFFFu, word, 16);
                const uint32_t umy = (uint32_t)__shfl_sync(0xFFFFFFFFu, word, 17);
                if (lane < 8 * p.nfrac) uniform_frac(sl.u[lane >> 3], p, umx, umy, lane >> 3, lane & 7);
            }
            if (pair) {
                const int X02 = (nxt.local % p.n5x) * kFillTile, Y02 = (nxt.local / p.n5x) * kFillTile;
                const uint32_t umx = (uint32_t)__shfl_sync(0xFFFFFFFFu, nword, 16);
                const uint32_t umy = (uint32_t)__shfl_sync(0xFFFFFFFFu, nword, 17);
                if (lane < 8 * p.nfrac)
                    uniform_frac(sl.u2[lane >> 3], p, umx, umy, lane >> 3, lane & 7);
                if (lane == 0) {
                    sl.index2 = nxt.local;
                    sl.X02 = X02;
                    sl.Y02 = Y02;
                    sl.wx02 = wx02;
                    sl.wy02 = wy02;
                }
            }
            if (lane == 0) {
                sl.plan.mode = mode;
                sl.X0 = X0;
                sl.Y0 = Y0;
                sl.pair = pair ? 1 : 0;
            }
        }
        __syncwarp();
        if (lane == 0) {
            sl.kind = kind;
            sl.stream = stream;
            sl.index = local;
            sl.cdt = st.cdt;
            s.snext[b] = 0u;  // the splat's chunk claims start over
            if (kind == kSlotTile) atomicAdd(&p.fh->nmode[mode], pair ? 2u : 1u);
            mbar_arrive(&s.full[b]);
        }
        if (pair) {  // the second tile is taken: the item after it comes next
            cur = decode(ep, __shfl_sync(0xFFFFFFFFu, qb, 0), seg);
            if (lane == 0 && cur.item < ep.total) qb = (int)atomicAdd(ep.queue, 1u);
            have_word = false;
            have_desc = false;
        } else {
            cur = nxt;
            word = nword;
            have_word = nhave;
            have_desc = nhave_desc;
            desc0 = ndesc0;
            desc1 = ndesc1;
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Uniform tiles
// ------------------------------------------------------------------------------------------------------------

// The source words of one fraction of a uniform tile (all threads of its group): for the kWordSide x kWordSide source
// pixels from (bx0, by0) -- the fraction's sources of the tile's region R, R - o_k grown by one -- the depth bits of a
// valid pixel with motion (mx, my), the bits with the sign set for a valid pixel with another motion, all ones for a
// pixel without valid depth or outside the frame.  Read from the staged window into the group's words.
constexpr int kWordSide = kRegion + 2;
static_assert((kWordSide * kWordSide + 1) / 2 <= kRegionN, "a fraction's source words fit its part of a key set");
template <typename CT, int WX, int WY>
__device__ __forceinline__ void group_source_words(const Window<CT, WX, WY> &w, int wx0, int wy0, const FrameDims &d,
                                                   uint32_t *words, int bx0, int by0, float mx, float my, int tg) {
    for (int c = tg; c < kWordSide * kWordSide; c += kGroupThreads) {
        const int y = by0 + c / kWordSide, x = bx0 + c % kWordSide;
        uint32_t v = 0xFFFFFFFFu;
        // (every such pixel inside the frame lies in the window, which holds the sources of all fractions)
        if ((unsigned)x < (unsigned)d.W && (unsigned)y < (unsigned)d.H && (unsigned)(x - wx0) < (unsigned)WX &&
            (unsigned)(y - wy0) < (unsigned)WY) {
            const int i = (y - wy0) * WX + (x - wx0);
            const uint32_t db = __float_as_uint(w.depth[i]);
            if (depth_ok(db)) v = (w.mv[0][i] == mx && w.mv[1][i] == my) ? db : (db | 0x80000000u);
        }
        words[c] = v;
    }
}

// One 2 x 2 block of a uniform tile for one fraction.  The block's cells are addressed in a frame mirrored so that
// the taps lie at +1 in x and y: mirrored column j <-> source column SX + c(j), c(j) = MX ? 2 - j : j - 1 (rows
// likewise), pixels at j, i in {1, 2}; the mirror flags are runtime values (one code copy for the four cases).  Frame checks for tiles near the border (one code path for every tile:
// the kernel is sensitive to its instruction footprint); every shared-memory index stays inside the window and the
// fraction's source words (words, kWordSide x kWordSide from (bx0, by0)).  Results c[], m[] are in true pixel order
// (dy * 2 + dx).
template <typename CT, int WX, int WY>
__device__ __forceinline__ void uniform_block(const Window<CT, WX, WY> &w, int wx0, int wy0, const FrameDims &p,
                                              const UniformFrac &u, int TX, int TY, const uint32_t *words, int bx0,
                                              int by0, float4 c[4], uint8_t m[4]) {
    const bool MX = (u.flags & kMirX) != 0, MY = (u.flags & kMirY) != 0;
    const int SX = TX - u.ox, SY = TY - u.oy;
    int cidx[4], ridx[4], wcol[4], wrow[4];
    bool fc[4], fr[4], sc[4], sr[4], tc[4], tr[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int dcol = MX ? 2 - j : j - 1, drow = MY ? 2 - j : j - 1;
        const int sx = SX + dcol, tx = TX + dcol;
        sc[j] = (unsigned)sx < (unsigned)p.W;
        tc[j] = (unsigned)tx < (unsigned)p.W;
        fc[j] = sc[j] && tc[j];
        cidx[j] = min(max(sx, wx0), wx0 + WX - 1) - wx0;  // a no-op inside the frame: keeps any index in the window
        wcol[j] = min(max(sx - bx0, 0), kWordSide - 1);
        const int sy = SY + drow, ty = TY + drow;
        sr[j] = (unsigned)sy < (unsigned)p.H;
        tr[j] = (unsigned)ty < (unsigned)p.H;
        fr[j] = sr[j] && tr[j];
        ridx[j] = (min(max(sy, wy0), wy0 + WY - 1) - wy0) * WX;
        wrow[j] = min(max(sy - by0, 0), kWordSide - 1) * kWordSide;
    }
    auto V = [&](int i, int j) -> uint32_t { return words[wrow[i] + wcol[j]]; };
    // validated word of a target cell: the source word if it is a winner, else all ones
    auto D = [&](uint32_t v, int i, int j) -> uint32_t {
        const uint32_t x = v | (uint32_t)((int32_t)v >> 31);
        return (fc[j] && fr[i]) ? x : 0xFFFFFFFFu;
    };
    const uint32_t v01 = V(0, 1), v02 = V(0, 2);
    const uint32_t v10 = V(1, 0), v11 = V(1, 1), v12 = V(1, 2), v13 = V(1, 3);
    const uint32_t v20 = V(2, 0), v21 = V(2, 1), v22 = V(2, 2), v23 = V(2, 3);
    const uint32_t v31 = V(3, 1), v32 = V(3, 2), v33 = V(3, 3);
    const uint32_t d01 = D(v01, 0, 1), d02 = D(v02, 0, 2);
    const uint32_t d10 = D(v10, 1, 0), d11 = D(v11, 1, 1), d12 = D(v12, 1, 2), d13 = D(v13, 1, 3);
    const uint32_t d20 = D(v20, 2, 0), d21 = D(v21, 2, 1), d22 = D(v22, 2, 2), d23 = D(v23, 2, 3);
    const uint32_t d31 = D(v31, 3, 1), d32 = D(v32, 3, 2);

    // Decisions of the four pixels (mirrored positions (1,1), (1,2), (2,1), (2,2)).
    bool ok[4];
    int sel[4];
    uint8_t mk[4];
    auto decide = [&](int q, uint32_t dq, uint32_t dl, uint32_t dr, uint32_t du, uint32_t dd, uint32_t tx_,
                      uint32_t ty_, uint32_t txy, bool in, bool exj, bool eyi) {
        const bool empty = dq == 0xFFFFFFFFu;
        const bool crack = !empty && is_crack(dq, dl, dr, du, dd);
        ok[q] = in && !empty && !crack;
        mk[q] = !in ? (uint8_t)0 : empty ? (uint8_t)EXW_MASK_EMPTY : crack ? (uint8_t)EXW_MASK_CRACK : (uint8_t)0;
        const float Dp = __uint_as_float(dq);
        const bool a10 = exj && tap_agrees(fabsf(__uint_as_float(tx_)), Dp);
        const bool a01 = eyi && tap_agrees(fabsf(__uint_as_float(ty_)), Dp);
        const bool a11 = exj && eyi && tap_agrees(fabsf(__uint_as_float(txy)), Dp);
        sel[q] = (a10 ? 1 : 0) | (a01 ? 2 : 0) | (a11 ? 4 : 0);
    };
    const bool tx = (u.flags & kTapX) != 0, ty = (u.flags & kTapY) != 0;
    const bool ex2 = tx && sc[2], ex3 = tx && sc[3];
    const bool ey2 = ty && sr[2], ey3 = ty && sr[3];
    decide(0, d11, d10, d12, d01, d21, v12, v21, v22, tc[1] && tr[1], ex2, ey2);
    decide(1, d12, d11, d13, d02, d22, v13, v22, v23, tc[2] && tr[1], ex3, ey2);
    decide(2, d21, d20, d22, d11, d31, v22, v31, v32, tc[1] && tr[2], ex2, ey3);
    decide(3, d22, d21, d23, d12, d32, v23, v32, v33, tc[2] && tr[2], ex3, ey3);
    float inv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) inv[q] = u.inv[sel[q]];

    // Colour, one channel at a time (9 cells: mirrored rows / columns 1..3).
    float out[4][3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const CT *cp = w.col[ch];
        float C[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) C[i][j] = to_f<CT>(cp[ridx[i + 1] + cidx[j + 1]]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = q >> 1, j = q & 1;  // mirrored pixel (i + 1, j + 1)
            float n = __fmul_rn(u.W00, C[i][j]);
            n = (sel[q] & 1) ? fmaf(u.W10, C[i][j + 1], n) : n;
            n = (sel[q] & 2) ? fmaf(u.W01, C[i + 1][j], n) : n;
            n = (sel[q] & 4) ? fmaf(u.W11, C[i + 1][j + 1], n) : n;
            out[q][ch] = ok[q] ? storage_round<CT>(__fmul_rn(n, inv[q])) : 0.0f;
        }
    }
    // true pixel t = (ti, tj) <- mirrored pixel (MY ? 1 - ti : ti, MX ? 1 - tj : tj), by selects
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int ti = t >> 1, tj = t & 1;
        const int qa = ((ti) << 1) | (tj), qx = ((ti) << 1) | (1 - tj), qy = ((1 - ti) << 1) | (tj),
                  qxy = ((1 - ti) << 1) | (1 - tj);
        auto pick = [&](auto v0, auto vx, auto vy, auto vxy) { return MY ? (MX ? vxy : vy) : (MX ? vx : v0); };
        c[t] = make_float4(pick(out[qa][0], out[qx][0], out[qy][0], out[qxy][0]),
                           pick(out[qa][1], out[qx][1], out[qy][1], out[qxy][1]),
                           pick(out[qa][2], out[qx][2], out[qy][2], out[qxy][2]),
                           pick(ok[qa], ok[qx], ok[qy], ok[qxy]) ? 1.0f : 0.0f);
        m[t] = pick(mk[qa], mk[qx], mk[qy], mk[qxy]);
    }
}

template <typename CT, int WX, int WY>
__device__ __forceinline__ void uniform_block_any(const Window<CT, WX, WY> &w, int wx0, int wy0, const FrameDims &p,
                                                  const UniformFrac &u, int TX, int TY, const uint32_t *words, int bx0,
                                                  int by0, float4 c[4], uint8_t m[4]) {
    uniform_block<CT, WX, WY>(w, wx0, wy0, p, u, TX, TY, words, bx0, by0, c, m);
}

// ------------------------------------------------------------------------------------------------------------
// Tiles through splat keys (modes 1-3)
// ------------------------------------------------------------------------------------------------------------
__device__ __forceinline__ void engine_splat_pixel(uint64_t (*key)[kRegionN], const FrameDims &p, int x, int y,
                                                   uint32_t db, uint32_t ux, uint32_t uy, uint32_t fm, int RX0,
                                                   int RY0) {
    if (!depth_ok(db) || !finite_bits(ux) || !finite_bits(uy)) return;
    const AxisDec dx = axis_dec(ux, p.L), dy = axis_dec(uy, p.L);
    if (!dx.land || !dy.land) return;
    const uint64_t kv = pack_key_local(db, x, y);
    for (int kk = 0; kk < p.nfrac; ++kk) {
        if (!(fm & (1u << kk))) continue;
        const int k = p.k0 + kk;
        const int gx = x + axis_off(dx, k), gy = y + axis_off(dy, k);
        if ((unsigned)gx >= (unsigned)p.W || (unsigned)gy >= (unsigned)p.H) continue;
        const int rx = gx - RX0, ry = gy - RY0;
        if ((unsigned)rx < (unsigned)kRegion && (unsigned)ry < (unsigned)kRegion)
            atomicMin((unsigned long long *)&key[kk][ry * kRegion + rx], (unsigned long long)kv);
    }
}

// Union of the landing rectangles of a plan held in shared memory.
__device__ __forceinline__ Rect plan_union(const TilePlan &pl, int nfrac) {
    Rect U{1 << 30, -(1 << 30), 1 << 30, -(1 << 30)};
    for (int kk = 0; kk < nfrac; ++kk) {
        const Rect R{pl.rect[kk][0], pl.rect[kk][1], pl.rect[kk][2], pl.rect[kk][3]};
        if (R.empty()) continue;
        U.x0 = min(U.x0, R.x0);
        U.x1 = max(U.x1, R.x1);
        U.y0 = min(U.y0, R.y0);
        U.y1 = max(U.y1, R.y1);
    }
    return U;
}

constexpr int kMaxSplatTiles = kConsumerThreads;

// Describe the 8 x 8 source tiles overlapping rectangle U (all consumer threads, no barrier).  Returns the count.
__device__ __forceinline__ int describe_tiles(SplatTile *out, const TileParams &p, const FrameDims &d, Rect U,
                                              int RX0, int RY0, int tid) {
    const int tx0 = U.x0 >> 3, ty0 = U.y0 >> 3, ntx = (U.x1 >> 3) - tx0 + 1;
    const int nt = ntx * ((U.y1 >> 3) - ty0 + 1);
    for (int t = tid; t < nt && t < kMaxSplatTiles; t += kConsumerThreads) {
        const int bx = tx0 + t % ntx, by = ty0 + t / ntx;
        SplatTile st{};
        st.bx = (uint16_t)bx;
        st.by = (uint16_t)by;
        const float4 b = __ldcg(p.tile_bounds + (size_t)by * p.nbx + bx);
        const float2 dr = __ldcg(p.tile_depth + (size_t)by * p.nbx + bx);  // issued with the bounds
        if (b.x <= b.y) {
            const bool uni = b.x == b.y && b.z == b.w;
            uint32_t fm = 0;
            const BoundsDec bd = bounds_dec(b, d.L);
            for (int kk = 0; kk < d.nfrac; ++kk) {
                int ox0, ox1, oy0, oy1;
                bounds_offsets(bd, d.k0 + kk, ox0, ox1, oy0, oy1);
                if (8 * bx + 7 + ox1 >= RX0 && 8 * bx + ox0 < RX0 + kRegion && 8 * by + 7 + oy1 >= RY0 &&
                    8 * by + oy0 < RY0 + kRegion)
                    fm |= 1u << kk;
                st.ox[kk] = (int8_t)max(-128, min(127, ox0));
                st.oy[kk] = (int8_t)max(-128, min(127, oy0));
            }
            st.fm = (uint8_t)fm;
            // offsets of a tile that reaches R lie within the window's span, far inside int8
            st.clean = uni && dr.x > 0.0f ? 1 : 0;
        }
        out[t] = st;
    }
    return nt < kMaxSplatTiles ? nt : kMaxSplatTiles;
}

// Splat the pixels of rectangle U from the staged window for all fractions (all consumer threads): candidate
// 8 x 8 tiles only, a warp per tile (two pixels per lane); a clean tile splats with its precomputed offsets.
// Pixel q & 63 of candidate tile st (q >> 6 of the list), from the staged window, for every fraction it reaches.
template <typename CT, int WX, int WY>
__device__ __forceinline__ void splat_window_pixel(uint64_t (*key)[kRegionN], const FrameDims &d,
                                                   const WinAcc<CT, WX, WY> &a, Rect U, const SplatTile &st, int q,
                                                   int RX0, int RY0) {
    if (!st.fm) return;
    const int x = 8 * st.bx + (q & 7), y = 8 * st.by + ((q >> 3) & 7);
    if (x < U.x0 || x > U.x1 || y < U.y0 || y > U.y1) return;
    const int i = a.at(x, y);
    const uint32_t db = __float_as_uint(a.w->depth[i]);
    if (st.clean) {
        const uint64_t kv = pack_key_local(db, x, y);
#pragma unroll
        for (int kk = 0; kk < kMaxFrac; ++kk) {
            if (!(st.fm & (1u << kk))) continue;
            const int gx = x + st.ox[kk], gy = y + st.oy[kk];
            if ((unsigned)gx >= (unsigned)d.W || (unsigned)gy >= (unsigned)d.H) continue;
            const int rx = gx - RX0, ry = gy - RY0;
            if ((unsigned)rx < (unsigned)kRegion && (unsigned)ry < (unsigned)kRegion)
                atomicMin((unsigned long long *)&key[kk][ry * kRegion + rx], (unsigned long long)kv);
        }
    } else {
        engine_splat_pixel(key, d, x, y, db, __float_as_uint(a.w->mv[0][i]), __float_as_uint(a.w->mv[1][i]), st.fm,
                           RX0, RY0);
    }
}

// A warp's next chunk of 32 candidate pixels (lane 0 claims, every lane gets it).
__device__ __forceinline__ int claim_chunk(uint32_t *next) {
    int c = 0;
    if ((threadIdx.x & 31) == 0) c = (int)atomicAdd(next, 1u);
    return __shfl_sync(0xFFFFFFFFu, c, 0);
}

template <typename CT, int WX, int WY>
__device__ __forceinline__ void engine_splat_window(EngineSmem &s, uint64_t (*key)[kRegionN], const TileParams &p,
                                                    const FrameDims &d, const WinAcc<CT, WX, WY> &a, Rect U, int RX0,
                                                    int RY0, int tid, const SplatTile *pre, int npre, uint32_t *next) {
    if (npre == 0) {  // too many candidates for the plan: described here, half a tile per warp and round
        const int nt = describe_tiles(s.cand, p, d, U, RX0, RY0, tid);
        bar_sync(kBarConsumers, kConsumerThreads);
        for (int q = tid; q < 64 * nt; q += kConsumerThreads) splat_window_pixel(key, d, a, U, s.cand[q >> 6], q, RX0, RY0);
        return;
    }
    // the plan's candidates, in chunks of half a tile that the warps claim: the warps that start the slot early
    // take more of them
    const int nchunk = 2 * npre, lane = tid & 31;
    int c = claim_chunk(next);
    while (c < nchunk) {
        int nx = 0;
        if (lane == 0) nx = (int)atomicAdd(next, 1u);  // the next claim, in flight while this chunk splats
        const int q = 32 * c + lane;
        splat_window_pixel(key, d, a, U, pre[q >> 6], q, RX0, RY0);
        c = __shfl_sync(0xFFFFFFFFu, nx, 0);
    }
}

// Splat from global memory: the 8 x 8 source tiles whose bounds reach R, 64 threads per tile (all consumers).  A
// clean candidate (one exact motion, every pixel can land) splats with its precomputed offsets and reads only the
// depth of its pixels.
__device__ __forceinline__ void splat_global_candidate(uint64_t (*key)[kRegionN], const TileParams &p,
                                                       const FrameDims &d, const SplatTile &st, int RX0, int RY0,
                                                       int tid);

__device__ inline void engine_splat_global(EngineSmem &s, uint64_t (*key)[kRegionN], const TileParams &p,
                                           const FrameDims &d, int RX0, int RY0, int tid, const SplatTile *pre,
                                           int npre, uint32_t *next) {
    if (npre > 0) {  // the plan's candidates, in chunks of half a tile that the warps claim
        const int nchunk = 2 * npre, lane = tid & 31;
        int c = claim_chunk(next);
        while (c < nchunk) {
            int nx = 0;
            if (lane == 0) nx = (int)atomicAdd(next, 1u);
            splat_global_candidate(key, p, d, pre[c >> 1], RX0, RY0, 32 * (c & 1) + lane);
            c = __shfl_sync(0xFFFFFFFFu, nx, 0);
        }
        return;
    }
    int bx0, bx1, by0, by1;
    if (!frame_window(p, RX0, RY0, bx0, bx1, by0, by1)) return;
    const int nbxr = bx1 - bx0 + 1;
    const int total = nbxr * (by1 - by0 + 1);
    for (int base = 0; base < total; base += kConsumerThreads) {
        if (tid == 0) s.ncand = 0u;
        bar_sync(kBarConsumers, kConsumerThreads);
        const int idx = base + tid;
        if (idx < total) {
            const int by = by0 + idx / nbxr, bx = bx0 + idx % nbxr;
            const float4 b = __ldcg(p.tile_bounds + (size_t)by * p.nbx + bx);
            const float2 dr = __ldcg(p.tile_depth + (size_t)by * p.nbx + bx);  // issued with the bounds
            if (b.x <= b.y) {
                SplatTile st{};
                uint32_t fm = 0;
                bool small = true;  // every offset fits an int8 (else a clean tile still splats per pixel)
                const BoundsDec bd = bounds_dec(b, p.L);
                for (int kk = 0; kk < p.nfrac; ++kk) {
                    int ox0, ox1, oy0, oy1;
                    bounds_offsets(bd, p.k0 + kk, ox0, ox1, oy0, oy1);
                    const int tx0 = 8 * bx + ox0, tx1 = 8 * bx + 7 + ox1;
                    const int ty0 = 8 * by + oy0, ty1 = 8 * by + 7 + oy1;
                    if (tx1 >= RX0 && tx0 < RX0 + kRegion && ty1 >= RY0 && ty0 < RY0 + kRegion) fm |= 1u << kk;
                    small = small && ox0 >= -128 && ox0 <= 127 && oy0 >= -128 && oy0 <= 127;
                    st.ox[kk] = (int8_t)max(-128, min(127, ox0));
                    st.oy[kk] = (int8_t)max(-128, min(127, oy0));
                }
                if (fm) {
                    st.bx = (uint16_t)bx;
                    st.by = (uint16_t)by;
                    st.fm = (uint8_t)fm;
                    st.clean = b.x == b.y && b.z == b.w && dr.x > 0.0f && small ? 1 : 0;
                    s.cand[atomicAdd(&s.ncand, 1u)] = st;
                }
            }
        }
        bar_sync(kBarConsumers, kConsumerThreads);
        const int nc = (int)s.ncand;
        for (int c0 = 0; c0 < nc; c0 += kConsumerThreads / 64) {
            const int ci = c0 + (tid >> 6);
            if (ci < nc) splat_global_candidate(key, p, d, s.cand[ci], RX0, RY0, tid);
        }
        bar_sync(kBarConsumers, kConsumerThreads);
    }
}

// One pixel (of 64 threads' 8 x 8 tile) of a candidate source tile, from global memory.
__device__ __forceinline__ void splat_global_candidate(uint64_t (*key)[kRegionN], const TileParams &p,
                                                       const FrameDims &d, const SplatTile &st, int RX0, int RY0,
                                                       int tid) {
    const int x = 8 * st.bx + (tid & 7), y = 8 * st.by + ((tid >> 3) & 7);
    if (x >= p.W || y >= p.H) return;
    const size_t i = (size_t)y * p.W + x;
    const uint32_t db = __float_as_uint(__ldg(p.depth + i));
    if (st.clean) {
        const uint64_t kv = pack_key_local(db, x, y);
#pragma unroll
        for (int kk = 0; kk < kMaxFrac; ++kk) {
            if (!(st.fm & (1u << kk))) continue;
            const int gx = x + st.ox[kk], gy = y + st.oy[kk];
            if ((unsigned)gx >= (unsigned)d.W || (unsigned)gy >= (unsigned)d.H) continue;
            const int rx = gx - RX0, ry = gy - RY0;
            if ((unsigned)rx < (unsigned)kRegion && (unsigned)ry < (unsigned)kRegion)
                atomicMin((unsigned long long *)&key[kk][ry * kRegion + rx], (unsigned long long)kv);
        }
    } else {
        const size_t plane = (size_t)p.W * p.H;
        engine_splat_pixel(key, d, x, y, db, __float_as_uint(__ldg(p.mv + i)),
                           __float_as_uint(__ldg(p.mv + plane + i)), st.fm, RX0, RY0);
    }
}

// Stage (b) for one target pixel (gx, gy) at region cell r from the keys kw (as 32-bit words) through accessor a.
template <typename CT, class Acc>
__device__ __forceinline__ void gather_pixel(const uint32_t *kw, const Acc &a, const FrameDims &p, int k, int gx,
                                             int gy, int r, float4 &c, uint8_t &m) {
    const bool in = gx < p.W && gy < p.H;
    const uint32_t dq = kw[2 * r + 1];
    const bool empty = dq == 0xFFFFFFFFu;
    const bool crack = !empty && is_crack(dq, kw[2 * (r - 1) + 1], kw[2 * (r + 1) + 1], kw[2 * (r - kRegion) + 1],
                                          kw[2 * (r + kRegion) + 1]);
    m = !in ? (uint8_t)0 : empty ? (uint8_t)EXW_MASK_EMPTY : crack ? (uint8_t)EXW_MASK_CRACK : (uint8_t)0;
    const bool ok = in && !empty && !crack;
    const uint32_t lo = kw[2 * r];
    int px = (int)(lo & 0x3FFFu), py = (int)(lo >> 14);
    if (!ok) {
        px = a.safe_x();
        py = a.safe_y();
    }
    const auto i00 = a.at(px, py);
    int sx, sy;
    const float rx = residual(a.mx(i00), k, p.L, gx - px, sx);
    const float ry = residual(a.my(i00), k, p.L, gy - py, sy);
    const float wx1 = fabsf(rx), wy1 = fabsf(ry);
    const float wx0 = 1.0f - wx1, wy0 = 1.0f - wy1;
    const bool ex = sx != 0 && (unsigned)(px + sx) < (unsigned)p.W;
    const bool ey = sy != 0 && (unsigned)(py + sy) < (unsigned)p.H;
    const auto i10 = ex ? i00 + sx : i00;
    const auto ir = sy > 0 ? i00 + a.stride() : i00 - a.stride();
    const auto i01 = ey ? ir : i00;
    const auto i11 = (ex && ey) ? ir + sx : i00;
    const float Dp = __uint_as_float(dq);
    const bool a10 = ex && tap_agrees(a.d(i10), Dp);
    const bool a01 = ey && tap_agrees(a.d(i01), Dp);
    const bool a11 = ex && ey && tap_agrees(a.d(i11), Dp);
    const float w00 = __fmul_rn(wx0, wy0);
    const float w10 = a10 ? __fmul_rn(wx1, wy0) : 0.0f;
    const float w01 = a01 ? __fmul_rn(wx0, wy1) : 0.0f;
    const float w11 = a11 ? __fmul_rn(wx1, wy1) : 0.0f;
    const float den = weight_sum(w00, w10, w01, w11);
    float v[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float n = __fmul_rn(w00, a.c(ch, i00));
        const float c10 = a.c(ch, i10), c01 = a.c(ch, i01), c11 = a.c(ch, i11);
        n = a10 ? fmaf(w10, c10, n) : n;
        n = a01 ? fmaf(w01, c01, n) : n;
        n = a11 ? fmaf(w11, c11, n) : n;
        v[ch] = n;
    }
    const float inv = __frcp_rn(den);
    c = make_float4(ok ? storage_round<CT>(__fmul_rn(v[0], inv)) : 0.0f,
                    ok ? storage_round<CT>(__fmul_rn(v[1], inv)) : 0.0f,
                    ok ? storage_round<CT>(__fmul_rn(v[2], inv)) : 0.0f, ok ? 1.0f : 0.0f);
}

template <typename CT, class Acc>
__device__ __forceinline__ void gather_block(const uint64_t *keys, const Acc &a, const FrameDims &p, int k, int TX,
                                             int TY, int bx, int by, float4 c[4], uint8_t m[4]) {
    const uint32_t *kw = reinterpret_cast<const uint32_t *>(keys);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int dy = t >> 1, dx = t & 1;
        const int r = (2 * by + dy + 1) * kRegion + (2 * bx + dx + 1);
        gather_pixel<CT>(kw, a, p, k, TX + dx, TY + dy, r, c[t], m[t]);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Epilogue: fill (pull-push levels 1..5 of the tile, Sec. IV-B stage (c)) and stores
// ------------------------------------------------------------------------------------------------------------

// Levels 3, 4 and 5 of a group's tile from its level-2 nodes (one warp; every lane returns l5, lane L < 16 its
// level-3 node L = (L >> 2, L & 3), lane L < 4 its level-4 node).
__device__ __forceinline__ void upper_levels(const float4 *l2, float4 &l3, float4 &l4, float4 &l5) {
    const int lane = threadIdx.x & 31;
    const int L = lane & 15;
    const int I = L >> 2, J = L & 3;
    const float4 *c = l2 + (2 * I) * 8 + 2 * J;
    l3 = mean4(c[0], c[1], c[8], c[9]);
    const int b4 = 8 * ((lane & 3) >> 1) + 2 * (lane & 1);
    const float4 q0 = shfl4_idx(l3, b4), q1 = shfl4_idx(l3, b4 + 1), q2 = shfl4_idx(l3, b4 + 4),
                 q3 = shfl4_idx(l3, b4 + 5);
    l4 = mean4(q0, q1, q2, q3);
    l5 = mean4(shfl4_idx(l4, 0), shfl4_idx(l4, 1), shfl4_idx(l4, 2), shfl4_idx(l4, 3));
}

// upper_levels through shared memory, for the fill of a tile: level-2 node (i, j) at l2[32 i + j] (row i in warp
// i's scratch), up 20 float4 of the warp's own scratch (level 3, then level 4).  Every lane returns l5, the level-3
// node (w >> 1, bx >> 2) and the level-4 node (w >> 2, bx >> 3) above its block; the same nodes and order as
// upper_levels.
__device__ __forceinline__ void upper_levels_smem(const float4 *l2, float4 *up, int w, int bx, float4 &v3, float4 &v4,
                                                  float4 &l5) {
    const int lane = threadIdx.x & 31;
    if (lane < 16) {
        const float4 *c = l2 + (2 * (lane >> 2)) * 32 + 2 * (lane & 3);
        up[lane] = mean4(c[0], c[1], c[32], c[33]);
    }
    __syncwarp();
    if (lane < 4) {
        const int b4 = 8 * (lane >> 1) + 2 * (lane & 1);
        up[16 + lane] = mean4(up[b4], up[b4 + 1], up[b4 + 4], up[b4 + 5]);
    }
    __syncwarp();
    l5 = mean4(up[16], up[17], up[18], up[19]);
    v3 = up[(w >> 1) * 4 + (bx >> 2)];
    v4 = up[16 + (w >> 2) * 2 + (bx >> 3)];
    __syncwarp();  // every read of the scratch before the warp's next use of it
}

template <typename CT>
__device__ __forceinline__ void store_block(const FrameDims &p, CT *oc, uint8_t *om, int TX, int TY, const float4 c[4],
                                            const uint8_t m[4], const bool write[4], bool vec) {
    const size_t plane = (size_t)p.W * p.H;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
        const int gy = TY + dy;
        if (gy >= p.H || TX >= p.W) continue;
        const size_t q = (size_t)gy * p.W + TX;
        const float4 a = c[2 * dy], b = c[2 * dy + 1];
        if (vec) {  // both pixels in the frame (W even), 2-element aligned rows
            *reinterpret_cast<uint16_t *>(om + q) = (uint16_t)(m[2 * dy] | (m[2 * dy + 1] << 8));
            if (write[2 * dy]) {
                if (sizeof(CT) == 2) {
                    *reinterpret_cast<__half2 *>(oc + q) = __floats2half2_rn(a.x, b.x);
                    *reinterpret_cast<__half2 *>(oc + plane + q) = __floats2half2_rn(a.y, b.y);
                    *reinterpret_cast<__half2 *>(oc + 2 * plane + q) = __floats2half2_rn(a.z, b.z);
                } else {
                    *reinterpret_cast<float2 *>(oc + q) = make_float2(a.x, b.x);
                    *reinterpret_cast<float2 *>(oc + plane + q) = make_float2(a.y, b.y);
                    *reinterpret_cast<float2 *>(oc + 2 * plane + q) = make_float2(a.z, b.z);
                }
            }
        } else {
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                if (TX + dx >= p.W) continue;
                const float4 v = dx ? b : a;
                om[q + dx] = m[2 * dy + dx];
                if (!write[2 * dy + dx]) continue;
                oc[q + dx] = to_storage<CT>(v.x);
                oc[plane + q + dx] = to_storage<CT>(v.y);
                oc[2 * plane + q + dx] = to_storage<CT>(v.z);
            }
        }
    }
}

// Items (tile, fraction) a group has published but not yet counted: thread 0 of the group publishes every node
// of the group's tiles and counts them in batches -- when the group moves to another stream or kind of item,
// when it waits for its next item, and before it leaves -- behind one fence per batch.  The stream's first fix-up
// item starts once the count is complete.
struct PendingCount {
    FrameHeader *fh = nullptr;
    uint32_t n = 0;
    __device__ __forceinline__ void flush() {
        if (n != 0u) {
            __threadfence();
            atomicAdd(&fh->done, n);
            n = 0u;
        }
    }
    __device__ __forceinline__ void add(FrameHeader *f) {
        if (f != fh) {
            flush();
            fh = f;
        }
        ++n;
    }
};

// Lazy level-5 nodes.  A tile-fraction without a hole is left as it is by the fill, and its level-5 node matters
// only to the coarse pass of a fraction with a tile without any valid pixel -- which most frames never run.  Such a
// tile publishes a placeholder instead of building its pyramid; when a coarse pass needs the node (it lies under
// the first valid ancestor of an invalid tile), one warp computes it: a smooth tile from its source colour
// (smooth_node), any other from its stored outputs (output_node).
constexpr float kNodeLazy = 2.0f;       // .w of a smooth tile's node that is not computed
constexpr float kNodeNeeded = 3.0f;     // .w of a lazy smooth node the coarse pass needs
constexpr float kNodeLazyOut = 4.0f;    // .w of the node of another tile-fraction without a hole, not computed
constexpr float kNodeNeededOut = 5.0f;  // .w of such a node the coarse pass needs

// Fill and store one fraction of the tile for the calling group.  The group first votes on whether the tile has a
// hole (a barrier that also orders every read of the splat keys before their next initialisation).  Without one the
// fill leaves the tile as it is: the group stores, and the tile publishes a lazy node computed from its stored outputs
// only if a coarse pass needs it (the group's stores are ordered before thread 0's count by a second barrier).  With
// holes the pyramid is built: a second group barrier, at which a warp without holes only arrives unless it is warp 0,
// which builds the upper levels.  c[] .w = validity.
template <typename CT>
__device__ __forceinline__ void fill_store_block(EngineSmem &s, const TileParams &p, const FrameDims &d, CT *oc,
                                                 uint8_t *om, int g, int kk, int tile, int TX, int TY, float4 c[4],
                                                 const uint8_t m[4], bool vec) {
    const int tg = threadIdx.x & (kGroupThreads - 1);
    const int lane = tg & 31, w = tg >> 5;
    const bool holes = __any_sync(0xFFFFFFFFu, (m[0] | m[1] | m[2] | m[3]) != 0);  // in the warp's rows
    const bool all[4] = {true, true, true, true};
    if (!bar_red_or(2 + g, kGroupThreads, holes)) {
        store_block<CT>(d, oc, om, TX, TY, c, m, all, vec);
        if (w == 0) bar_sync(2 + g, kGroupThreads);  // thread 0 counts the tile after every store of the group
        else asm volatile("bar.arrive %0, %1;" ::"r"(2 + g), "r"(kGroupThreads) : "memory");
        if (tg == 0) publish_node(p, make_float4(0.f, 0.f, 0.f, kNodeLazyOut), kk, tile);
        return;
    }
    // level 1 of the group's 2 x 2 blocks in the group's scratch (thread tg = block (tg & 15, tg >> 4)); a warp's
    // level-2 nodes (its row w of them) from four of its level-1 nodes, then in the first 8 of its slots.  No later
    // slot touches the scratch before every warp of the group is done with it (each slot that does starts behind a
    // barrier of the whole group or of all consumers).
    const float4 n1 = mean4(c[0], c[1], c[2], c[3]);
    float4 *l1 = reinterpret_cast<float4 *>(s.cand) + g * kGroupThreads;
    l1[tg] = n1;
    __syncwarp();
    float4 n2o = n1;
    if ((lane & 17) == 0) n2o = mean4(n1, l1[tg + 1], l1[tg + 16], l1[tg + 17]);
    __syncwarp();  // every read of the warp's level-1 slots before they hold its level-2 nodes
    float4 *l2 = l1;  // level-2 node (i, j) at l2[32 i + j]
    if ((lane & 17) == 0) l2[32 * w + (lane >> 1)] = n2o;
    if (!holes && w != 0) {  // needs no upper level
        asm volatile("bar.arrive %0, %1;" ::"r"(2 + g), "r"(kGroupThreads) : "memory");
        store_block<CT>(d, oc, om, TX, TY, c, m, all, vec);
        return;
    }
    bar_sync(2 + g, kGroupThreads);
    float4 *up = l1 + 32 * w + 8;  // the warp's slots after its level-2 nodes, read by no one else: levels 3 and 4
    const int bx = lane & 15;
    if (!holes) {
        if (w == 0) {
            float4 v3, v4, l5;
            upper_levels_smem(l2, up, w, bx, v3, v4, l5);
            if (lane == 0) publish_node(p, l5, kk, tile);
        }
        store_block<CT>(d, oc, om, TX, TY, c, m, all, vec);
        return;
    }
    const float4 n2 = l2[32 * w + (bx >> 1)];  // level 2 of this thread's block
    bool deep = false;  // a hole whose level-1 and level-2 ancestors are both invalid
#pragma unroll
    for (int t = 0; t < 4; ++t) deep = deep || (m[t] != 0 && n1.w == 0.0f && n2.w == 0.0f);
    // push: first valid ancestor (tile rows 4w..4w+3: level-3 node (w >> 1, bx >> 2), level-4 (w >> 2, bx >> 3));
    // without a deep hole in the warp levels 3-5 are not read
    float4 v3 = n2, v4 = n2, l5 = n2;
    if (w == 0 || __any_sync(0xFFFFFFFFu, deep)) upper_levels_smem(l2, up, w, bx, v3, v4, l5);
    if (w == 0 && lane == 0) publish_node(p, l5, kk, tile);
    const float4 push = n1.w != 0.0f ? n1 : n2.w != 0.0f ? n2 : v3.w != 0.0f ? v3 : v4.w != 0.0f ? v4 : l5;
    bool write[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const bool hole = m[t] != 0;
        if (hole) c[t] = push;
        write[t] = !hole || push.w != 0.0f;
    }
    store_block<CT>(d, oc, om, TX, TY, c, m, write, vec);
}

// Level-2 node of a column pair's 4 x 4 block from this lane's column of four pixels (all valid; the same pyramid
// as mean4 over valid children): level 1 by a shuffle with the neighbouring column, level 2 with the next pair.
// Meaningful on lanes with (lane & 3) == 0: the node (row band, lane >> 2).
template <typename CT>
__device__ __forceinline__ float4 smooth_level2(const CT out[4][3]) {
    const int lane = threadIdx.x & 31;
    float4 px[4], pp[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        px[r] = make_float4(to_f<CT>(out[r][0]), to_f<CT>(out[r][1]), to_f<CT>(out[r][2]), 1.0f);
        pp[r] = make_float4(__shfl_xor_sync(0xFFFFFFFFu, px[r].x, 1), __shfl_xor_sync(0xFFFFFFFFu, px[r].y, 1),
                            __shfl_xor_sync(0xFFFFFFFFu, px[r].z, 1), 1.0f);
    }
    const bool odd = lane & 1;
    // level 1: rows 0-1 (A) and 2-3 (B) of this column pair, children in (row, column) order
    const float4 A = odd ? mean4(pp[0], px[0], pp[1], px[1]) : mean4(px[0], pp[0], px[1], pp[1]);
    const float4 B = odd ? mean4(pp[2], px[2], pp[3], px[3]) : mean4(px[2], pp[2], px[3], pp[3]);
    const float4 Ap = make_float4(__shfl_xor_sync(0xFFFFFFFFu, A.x, 2), __shfl_xor_sync(0xFFFFFFFFu, A.y, 2),
                                  __shfl_xor_sync(0xFFFFFFFFu, A.z, 2), 1.0f);
    const float4 Bp = make_float4(__shfl_xor_sync(0xFFFFFFFFu, B.x, 2), __shfl_xor_sync(0xFFFFFFFFu, B.y, 2),
                                  __shfl_xor_sync(0xFFFFFFFFu, B.z, 2), 1.0f);
    const bool right = lane & 2;
    return right ? mean4(Ap, A, Bp, B) : mean4(A, Ap, B, Bp);
}

// The lazy smooth node, recomputed by one warp: the tile's outputs again from the source colour (the same arithmetic
// as smooth_column_t, so the same bits), then the same pyramid.

template <typename CT> __device__ __forceinline__ float load_out(const CT *q);
template <> __device__ __forceinline__ float load_out<float>(const float *q) { return __ldcg(q); }
template <> __device__ __forceinline__ float load_out<__half>(const __half *q) {
    return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(q))));
}

// The level-5 node of a tile-fraction without a hole from its stored outputs (one warp): the 2 x 2 blocks, the
// order and the levels of fill_store_block, warp row w of the group as loop step w (a pixel outside the frame is
// invalid, as in the gather), so the same bits.
template <typename CT>
__device__ float4 output_node(const TileParams &p, int tile, int kk, float4 *l2) {
    const int lane = threadIdx.x & 31, bx = lane & 15;
    const int X0 = (tile % p.n5x) * kFillTile, Y0 = (tile / p.n5x) * kFillTile;
    const size_t plane = (size_t)p.W * p.H;
    const CT *oc = (const CT *)p.out_color[kk];
#pragma unroll 1
    for (int w = 0; w < kFillTile / 4; ++w) {
        const int TX = X0 + 2 * bx, TY = Y0 + 2 * (2 * w + (lane >> 4));
        float4 c[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int x = TX + (t & 1), y = TY + (t >> 1);
            c[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (x < p.W && y < p.H) {
                const size_t q = (size_t)y * p.W + x;
                c[t] = make_float4(load_out<CT>(oc + q), load_out<CT>(oc + plane + q), load_out<CT>(oc + 2 * plane + q),
                                   1.0f);
            }
        }
        const float4 n1 = mean4(c[0], c[1], c[2], c[3]);
        const float4 a1 = shfl4_xor(n1, 1), a16 = shfl4_xor(n1, 16), a17 = shfl4_xor(n1, 17);
        const float4 n2o = mean4(n1, a1, a16, a17);
        if ((lane & 17) == 0) l2[w * 8 + (lane >> 1)] = n2o;
    }
    __syncwarp();
    float4 l3, l4, l5;
    upper_levels(l2, l3, l4, l5);
    __syncwarp();
    return l5;
}

template <typename CT>
__device__ float4 smooth_node(const TileParams &p, int tile, int kk, float4 *l2) {
    const int lane = threadIdx.x & 31;
    const uint32_t umx = __ldcg(&p.plans[tile].umx), umy = __ldcg(&p.plans[tile].umy);
    const int k = p.k0 + kk;
    // the fraction's constants, as uniform_frac computes them
    const int ox = axis_off_of(umx, k, p.L), oy = axis_off_of(umy, k, p.L);
    int sx, sy;
    const float rx = residual(__uint_as_float(umx), k, p.L, ox, sx);
    const float ry = residual(__uint_as_float(umy), k, p.L, oy, sy);
    const float wx1 = fabsf(rx), wy1 = fabsf(ry);
    const float wx0 = 1.0f - wx1, wy0 = 1.0f - wy1;
    const float W00 = __fmul_rn(wx0, wy0), W10 = __fmul_rn(wx1, wy0), W01 = __fmul_rn(wx0, wy1),
                W11 = __fmul_rn(wx1, wy1);
    const bool EX = sx != 0, EY = sy != 0;
    const int j = (EX ? 1 : 0) | (EY ? 2 : 0) | (EX && EY ? 4 : 0);
    const float inv = __frcp_rn(weight_sum(W00, (j & 1) ? W10 : 0.0f, (j & 2) ? W01 : 0.0f, (j & 4) ? W11 : 0.0f));
    const int X0 = (tile % p.n5x) * kFillTile, Y0 = (tile / p.n5x) * kFillTile;
    const size_t plane = (size_t)p.W * p.H;
    const CT *col = (const CT *)p.color;
    const int cx = X0 + lane - ox, tx = cx + sx;  // source column and tap column (inside the frame: a smooth tile)
#pragma unroll 2
    for (int w = 0; w < kFillTile / 4; ++w) {
        CT out[4][3];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int cy = Y0 + 4 * w + r - oy, ty = cy + sy;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const CT *cp = col + ch * plane;
                float n = __fmul_rn(W00, to_f<CT>(cp[(size_t)cy * p.W + cx]));
                if (EX) n = fmaf(W10, to_f<CT>(cp[(size_t)cy * p.W + tx]), n);
                if (EY) n = fmaf(W01, to_f<CT>(cp[(size_t)ty * p.W + cx]), n);
                if (EX && EY) n = fmaf(W11, to_f<CT>(cp[(size_t)ty * p.W + tx]), n);
                out[r][ch] = to_storage<CT>(__fmul_rn(n, inv));
            }
        }
        const float4 n2 = smooth_level2<CT>(out);
        if ((lane & 3) == 0) l2[w * 8 + (lane >> 2)] = n2;
    }
    __syncwarp();
    float4 l3, l4, l5;
    upper_levels(l2, l3, l4, l5);
    __syncwarp();
    return l5;
}

// Coarse levels of the pyramid of one fraction above level 5 (all consumer threads): level 6 from the level-5
// nodes, each further level from the one below, mean4 over the valid children.
__device__ inline void coarse_levels(const float4 *nodes, float4 *cz, int n5x, int n5y) {
    const int tid = threadIdx.x, nt = kConsumerThreads;
    const float4 *child = nodes;
    int cw = n5x, ch = n5y, off = 0;
    while (cw > 1 || ch > 1) {
        const int pw = (cw + 1) / 2, ph = (ch + 1) / 2;
        float4 *par = cz + off;
        for (int node = tid; node < pw * ph; node += nt) {
            const int i = node / pw, j = node - i * pw;
            float4 c[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ci = 2 * i + (q >> 1), cj = 2 * j + (q & 1);
                c[q] = (ci < ch && cj < cw) ? __ldcg(child + ci * cw + cj) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            par[node] = mean4(c[0], c[1], c[2], c[3]);
        }
        __threadfence_block();
        bar_sync(kBarConsumers, kConsumerThreads);
        child = par;
        off += pw * ph;
        cw = pw;
        ch = ph;
    }
}

// Coarse levels of the pyramid and the value of every tile without a valid pixel (all consumer threads).  Lazy
// level-5 nodes are computed first where a fill value depends on them: in the subtree of the first valid ancestor
// of some tile without a valid pixel.  That ancestor is found without the pyramid: an ancestor d levels above
// level 5 is valid when a level-5 node of its 2^d x 2^d block is (a lazy node is valid).  scratch: 64 float4 per
// consumer warp of shared memory.
// (Not inlined, like the fix-up slice: the engine's throughput depends on how compact the code of its frequent
// items stays in the instruction cache.)
static __device__ __noinline__ void engine_coarse_pass(const TileParams &p, float4 *scratch, int cdt) {
    const int tid = threadIdx.x, nt = kConsumerThreads, lane = tid & 31, wid = tid >> 5;
    const int n5 = p.n5x * p.n5y;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const uint32_t cnt = __ldcg(&p.fh->ninvalid[kk]);
        if (cnt == 0u) continue;
        float4 *nodes = p.nodes + (size_t)kk * n5;
        float4 *cz = p.coarse + (size_t)kk * p.ncoarse;
        const uint32_t *list = p.list + (size_t)kk * n5;
        // 1. per tile without a valid pixel (a warp each): the block of its first valid ancestor; its lazy nodes
        //    are needed
        bool any = false;
        for (uint32_t e = wid; e < cnt; e += kConsumerWarps) {
            const uint32_t tile = __ldcg(list + e);
            const int tx = (int)(tile % (uint32_t)p.n5x), ty = (int)(tile / (uint32_t)p.n5x);
            for (int d = 1; (1 << (d - 1)) < max(p.n5x, p.n5y); ++d) {
                const int bx0 = (tx >> d) << d, by0 = (ty >> d) << d;
                const int bw = min(1 << d, p.n5x - bx0), bh = min(1 << d, p.n5y - by0);
                bool valid = false;
                for (int c = lane; c < bw * bh && !valid; c += 32)
                    valid = __ldcg(&nodes[(by0 + c / bw) * p.n5x + bx0 + c % bw].w) != 0.0f;
                if (!__any_sync(0xFFFFFFFFu, valid)) continue;
                for (int c = lane; c < bw * bh; c += 32) {
                    float *w = &nodes[(by0 + c / bw) * p.n5x + bx0 + c % bw].w;
                    const float lw = __ldcg(w);
                    if (lw == kNodeLazy || lw == kNodeLazyOut) {
                        *w = lw == kNodeLazy ? kNodeNeeded : kNodeNeededOut;
                        any = true;
                    }
                }
                break;
            }
        }
        __threadfence_block();
        // 2. the needed lazy nodes, one warp per tile
        if (bar_red_or(kBarConsumers, kConsumerThreads, any)) {
            float4 *l2 = scratch + 64 * wid;
            for (int base = 32 * wid; base < n5; base += 32 * kConsumerWarps) {
                const int i = base + lane;
                const float nw = i < n5 ? __ldcg(&nodes[i].w) : 0.0f;
                unsigned m = __ballot_sync(0xFFFFFFFFu, nw == kNodeNeeded || nw == kNodeNeededOut);
                const unsigned mo = __ballot_sync(0xFFFFFFFFu, nw == kNodeNeededOut);
                while (m) {
                    const int b = __ffs(m) - 1, t = base + b;
                    m &= m - 1u;
                    float4 v;
                    if (mo & (1u << b))
                        v = cdt == EXW_F16 ? output_node<__half>(p, t, kk, l2) : output_node<float>(p, t, kk, l2);
                    else
                        v = cdt == EXW_F16 ? smooth_node<__half>(p, t, kk, l2) : smooth_node<float>(p, t, kk, l2);
                    if (lane == 0) {
                        nodes[t] = v;
                        atomicAdd(&p.fh->nlazy[(mo >> b) & 1u], 1u);
                    }
                }
            }
            __threadfence_block();
            bar_sync(kBarConsumers, kConsumerThreads);
        }
        // 3. the coarse levels (the ancestors of lazy nodes that were not needed are never read), then each invalid
        //    tile's first valid ancestor
        coarse_levels(nodes, cz, p.n5x, p.n5y);
        for (uint32_t e = tid; e < cnt; e += nt) {
            const uint32_t tile = __ldcg(list + e);
            int ax = (int)(tile % (uint32_t)p.n5x), ay = (int)(tile / (uint32_t)p.n5x);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            int w = p.n5x, h = p.n5y, o = 0;
            while (w > 1 || h > 1) {
                const int pw = (w + 1) / 2, ph = (h + 1) / 2;
                ax >>= 1;
                ay >>= 1;
                const float4 c = __ldcg(cz + o + ay * pw + ax);
                if (c.w != 0.0f) {
                    v = c;
                    break;
                }
                o += pw * ph;
                w = pw;
                h = ph;
            }
            p.fillval[(size_t)kk * n5 + e] = make_float4(v.x, v.y, v.z, 1.0f);
        }
        bar_sync(kBarConsumers, kConsumerThreads);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Smooth uniform tiles (plan mode 5): every target is its source's bilinear resampling with all taps
// ------------------------------------------------------------------------------------------------------------

// One column of four pixels (tile rows 4w..4w+3 of column lane; w = warp in the group): out[r] = colour of row r.
// Lanes are consecutive columns, so every shared-memory access of a warp is conflict-free.
template <typename CT, int WX, int WY, bool MY, bool EX, bool EY>
__device__ __forceinline__ void smooth_column_t(const CT *col, int wx0, int wy0, const UniformFrac &u, int X0, int Y0,
                                                CT out[4][3]) {
    const int tg = threadIdx.x & (kGroupThreads - 1);
    const int lane = tg & 31, w = tg >> 5;
    const int sx = EX ? ((u.flags & kMirX) ? -1 : 1) : 0;
    const int cx = X0 + lane - u.ox - wx0;                          // window column of the source
    const int ry = Y0 + 4 * w - u.oy - wy0 + (MY ? -1 : 0);         // window row of loaded row 0
    const float inv = u.inv[(EX ? 1 : 0) | (EY ? 2 : 0) | (EX && EY ? 4 : 0)];
    const float W00 = u.W00, W10 = u.W10, W01 = u.W01, W11 = u.W11;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const CT *cp = col + ch * (WX * WY) + ry * WX + cx;
        float C[5][2];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            if (!EY && i == (MY ? 0 : 4)) continue;  // the tap row is not read without a y tap
            C[i][0] = to_f<CT>(cp[i * WX]);
            if (EX) C[i][1] = to_f<CT>(cp[i * WX + sx]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int ic = MY ? r + 1 : r, it = MY ? r : r + 1;  // centre row, tap row
            float n = __fmul_rn(W00, C[ic][0]);
            if (EX) n = fmaf(W10, C[ic][1], n);
            if (EY) n = fmaf(W01, C[it][0], n);
            if (EX && EY) n = fmaf(W11, C[it][1], n);
            out[r][ch] = to_storage<CT>(__fmul_rn(n, inv));
        }
    }
}

// col: plane 0 of the tile's colour window (WX x WY per plane, planes consecutive).
template <typename CT, int WX, int WY>
__device__ __forceinline__ void smooth_column(const CT *col, int wx0, int wy0, const UniformFrac &u, int X0, int Y0,
                                              CT out[4][3]) {
    const bool my = (u.flags & kMirY) != 0;
    switch (u.flags & (kTapX | kTapY)) {
        case kTapX | kTapY:
            if (my) smooth_column_t<CT, WX, WY, true, true, true>(col, wx0, wy0, u, X0, Y0, out);
            else smooth_column_t<CT, WX, WY, false, true, true>(col, wx0, wy0, u, X0, Y0, out);
            break;
        case kTapX: smooth_column_t<CT, WX, WY, false, true, false>(col, wx0, wy0, u, X0, Y0, out); break;
        case kTapY:
            if (my) smooth_column_t<CT, WX, WY, true, false, true>(col, wx0, wy0, u, X0, Y0, out);
            else smooth_column_t<CT, WX, WY, false, false, true>(col, wx0, wy0, u, X0, Y0, out);
            break;
        default: smooth_column_t<CT, WX, WY, false, false, false>(col, wx0, wy0, u, X0, Y0, out); break;
    }
}

template <typename CT>
__device__ __forceinline__ void store_column(const FrameDims &p, CT *oc, uint8_t *om, int X0, int Y0,
                                             const CT out[4][3]) {
    const int tg = threadIdx.x & (kGroupThreads - 1);
    const int lane = tg & 31, w = tg >> 5;
    const int x = X0 + lane;
    if (x >= p.W) return;
    const size_t plane = (size_t)p.W * p.H;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int y = Y0 + 4 * w + r;
        if (y >= p.H) continue;
        const size_t q = (size_t)y * p.W + x;
        oc[q] = out[r][0];
        oc[plane + q] = out[r][1];
        oc[2 * plane + q] = out[r][2];
        om[q] = 0;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Consumers
// ------------------------------------------------------------------------------------------------------------
// One target tile for the calling group (fraction k0 + g); the splat (modes 1-3) is done.
template <typename CT, int WX, int WY, bool FILL>
__device__ __forceinline__ void tile_group(EngineSmem &s, const TileSlot &sl, const TileParams &p, int b, int g,
                                           uint64_t (*key)[kRegionN], uint64_t (*idle)[kRegionN]) {
    const FrameDims d = dims_of(p);
    const int tg = threadIdx.x & (kGroupThreads - 1);
    const int bx = tg & 15, by = tg >> 4;
    const int mode = sl.plan.mode, tile = sl.index, X0 = sl.X0, Y0 = sl.Y0;
    const int wx0 = sl.plan.wx0, wy0 = sl.plan.wy0;
    const int kk = g, k = d.k0 + kk;
    const int TX = X0 + 2 * bx, TY = Y0 + 2 * by;
    CT *oc = (CT *)p.out_color[kk];
    uint8_t *om = p.out_mask[kk];
    const bool vec = (d.W % 2) == 0 && ((uintptr_t)oc % (2 * sizeof(CT))) == 0 && ((uintptr_t)om % 2) == 0;
    Window<CT, WX, WY> &win = window<CT, WX, WY>(s, b);
    if (mode == 5) {  // colour windows at the buffer's start: the slot's tile, then the paired one
        const int n = sl.pair ? 2 : 1;
#pragma unroll 1
        for (int q = 0; q < n; ++q) {  // one copy of the code for both tiles
            const CT *col = reinterpret_cast<const CT *>(s.win[b]) + q * 3 * WX * WY;
            const int x0 = q ? sl.X02 : X0, y0 = q ? sl.Y02 : Y0;
            CT out[4][3];
            smooth_column<CT, WX, WY>(col, q ? sl.wx02 : wx0, q ? sl.wy02 : wy0, q ? sl.u2[kk] : sl.u[kk], x0, y0,
                                      out);
            store_column<CT>(d, oc, om, x0, y0, out);
        }
        // no hole: the fill leaves the tile as it is, and its level-5 node is computed only if a coarse pass needs it
        if (FILL && (threadIdx.x & (kGroupThreads - 1)) == 0) {
            publish_node(p, make_float4(0.f, 0.f, 0.f, kNodeLazy), kk, tile);
            if (n == 2) publish_node(p, make_float4(0.f, 0.f, 0.f, kNodeLazy), kk, sl.index2);
        }
        return;
    }
    float4 c[4];
    uint8_t m[4];
    // uniform tile: the fraction's source words in the group's part of the key set no splat uses before the next
    // one (empty again when the group is done)
    uint32_t *words = reinterpret_cast<uint32_t *>(idle[kk]);
    if (mode == 0) {
        const UniformFrac &u = sl.u[kk];
        const int bx0 = X0 - 2 - u.ox, by0 = Y0 - 2 - u.oy;  // (R - o_k grown by one)
        // the slot's first barrier, which every warp of the group reaches only after its earlier slots: their
        // emptying of these cells (by other threads than the ones that write the words) is done
        bar_sync(kBarBounds + g, kGroupThreads);
        group_source_words(win, wx0, wy0, d, words, bx0, by0, __uint_as_float(sl.plan.umx),
                           __uint_as_float(sl.plan.umy), tg);
        bar_sync(kBarBounds + g, kGroupThreads);  // every word before any read of them
        uniform_block_any<CT, WX, WY>(win, wx0, wy0, d, u, TX, TY, words, bx0, by0, c, m);
    } else if (mode == 1) {
        const WinAcc<CT, WX, WY> wa{&win, wx0, wy0};
        gather_block<CT>(key[kk], wa, d, k, TX, TY, bx, by, c, m);
    } else if (mode == 2 || mode == 3) {
        const GlobalAcc<CT> ga{(const CT *)p.color, p.depth, p.mv, d.W, (size_t)d.W * d.H};
        gather_block<CT>(key[kk], ga, d, k, TX, TY, bx, by, c, m);
    } else {  // 4: nothing lands
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            c[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            m[t] = (TX + (t & 1) < d.W && TY + (t >> 1) < d.H) ? (uint8_t)EXW_MASK_EMPTY : (uint8_t)0;
        }
    }
    if (FILL) {
        fill_store_block<CT>(s, p, d, oc, om, g, kk, tile, TX, TY, c, m, vec);
    } else {
        const bool all[4] = {true, true, true, true};
        store_block<CT>(d, oc, om, TX, TY, c, m, all, vec);
        if (mode <= 3)
            bar_sync(2 + g, kGroupThreads);  // every key or word read of the group is done before they are emptied
    }
    // the group's keys empty again for the next splat into this set (its reads ended at the barrier above or at
    // the fill's first barrier); a uniform tile's words likewise
    if (mode >= 1 && mode <= 3)
        for (int r = tg; r < kRegionN; r += kGroupThreads) key[kk][r] = kKeyEmpty;
    if (mode == 0)
        for (int r = tg; r < (kWordSide * kWordSide + 1) / 2; r += kGroupThreads) idle[kk][r] = kKeyEmpty;
}

// The splat of a tile (modes 1-3) into key set `key`, all consumer threads; the set is empty (every group emptied its
// fraction's keys after its last gather from them).  Ends with a consumer-wide barrier, which also orders every
// use of the other key set in earlier slots before the next splat into it.
template <typename CT, int WX, int WY>
__device__ __forceinline__ void tile_splat(EngineSmem &s, const TileSlot &sl, const TileParams &p, int b, int tid,
                                           uint64_t (*key)[kRegionN]) {
    const FrameDims d = dims_of(p);
    const int mode = sl.plan.mode;
    const int RX0 = sl.X0 - 1, RY0 = sl.Y0 - 1;
    const int npre = sl.plan.ndesc;  // the plan's candidates in sl.pdesc (0: none stored)
    if (mode == 1) {
        const WinAcc<CT, WX, WY> wa{&window<CT, WX, WY>(s, b), sl.plan.wx0, sl.plan.wy0};
        engine_splat_window(s, key, p, d, wa, plan_union(sl.plan, d.nfrac), RX0, RY0, tid, sl.pdesc, npre,
                            &s.snext[b]);
    } else {
        engine_splat_global(s, key, p, d, RX0, RY0, tid, sl.pdesc, npre, &s.snext[b]);
    }
    bar_sync(kBarConsumers, kConsumerThreads);
}

struct HalfGroupBarrier {  // the 4 warps of half group h: named barrier 5 + h
    int id;
    __device__ __forceinline__ void operator()() const { bar_sync(id, kGroupThreads / 2); }
};

template <bool FILL, int SHAPE>
__device__ void engine_consumer(EngineSmem &s, const EngineParams &ep) {
    uint32_t *status = ep.status;
    using WS = WinShape<SHAPE>;
    const int tid = threadIdx.x;  // 0 .. 767
    const int g = tid >> 8, tg = tid & (kGroupThreads - 1);
    const int lane = tid & 31, w = tid >> 5;
    PendingCount pend;  // thread 0 of each group
    uint32_t nsplat = 0;  // splat slots taken: slot n's keys are set n & 1
    for (uint32_t i = 0;; ++i) {
        const int b = (int)(i & 1u);
        // the next item is not ready: count what this group published before blocking (the producer may be
        // waiting for exactly that count)
        if (FILL && tg == 0 && pend.n != 0u && !mbar_test_wait(&s.full[b], (i >> 1) & 1u)) pend.flush();
        const bool ok = mbar_wait_or_abort(&s.full[b], (i >> 1) & 1u, &s.abort, kConsumerWaitNs);
        const TileSlot &sl = s.slot[b];
        const int kind = ok ? sl.kind : kSlotEnd;
        const int mode = kind == kSlotTile ? sl.plan.mode : -1;
        // the stream's parameters (the end slot, and a slot that never arrived, name no stream)
        const TileParams &p = ep.st[kind == kSlotEnd ? 0 : sl.stream].p;
        // The consumer-wide vote: every thread agrees that the slot arrived, and every group has finished the slots
        // before it.  Slots that share nothing between the groups and use no barrier that an earlier slot's warps may
        // still be due at (the fill's group barriers) -- smooth tiles (each group its own fraction, no barrier),
        // bounds items (each half group its own region, partials and barriers), plan items (a warp per tile),
        // fix-up slices after the first (plain stores) -- go on without it; a thread whose wait ran out meets the
        // others at the next slot's vote, which every other kind of slot (the end included) takes.
        // A splat tile whose candidates the plan stored takes none either: its keys are the set the slot before
        // did not use, emptied by every group after its last gather from them -- which the consumer-wide barrier
        // closing the previous splat ordered before this one's splat -- and its first barrier is that closing
        // barrier, which every warp reaches only after its earlier slots.
        const bool splat = kind == kSlotTile && mode >= 1 && mode <= 3;
        // So does a uniform tile: each group builds its fraction's source words in its part of the key set no
        // splat uses before the next one, behind a group barrier.
        const bool solo = (kind == kSlotTile && (mode == 5 || mode == 0)) || (splat && sl.plan.ndesc > 0) ||
                          kind == kSlotBounds || kind == kSlotPlans || (kind == kSlotFixup && sl.index != 0);
        if (!solo && bar_red_or(kBarConsumers, kConsumerThreads, !ok)) {
            if (tid == 0) {  // (the slot may never have been written: its parameters are not used here)
                atomicCAS(status, 0u, (uint32_t)EXW_ERR_TIMEOUT);
                *(volatile int *)&s.abort = 1;
            }
            return;
        }
        if (FILL && tg == 0 && (kind != kSlotTile || p.fh != pend.fh)) pend.flush();
        if (kind == kSlotEnd) return;
        if (kind == kSlotBounds) {
            const int h = tid >> 7, th = tid & 127;  // half group: 4 warps, 8 rows each, 24 loads in flight
            const int nrx = (p.W + 31) / 32, nreg = nrx * ((p.H + 31) / 32);
            // the partials live in the group's scratch (a part per region, so a region's partials never overwrite the
            // previous one's while its last warp still reads them): every warp of the group is done with its last fill
            bar_sync(kBarBounds + g, kGroupThreads);
            uint32_t done = 0u;
#pragma unroll 1
            for (int j = 0; j < kRegionsPerHalf; ++j) {
                const int region = sl.index * kRegionsPerItem + h * kRegionsPerHalf + j;
                float4 *part = reinterpret_cast<float4 *>(s.cand) + g * kGroupThreads + 32 * (kRegionsPerHalf * (h & 1) + j);
                if (region >= nreg) break;
                bounds_region<4>(p.depth, p.mv, p.W, p.H, const_cast<float4 *>(p.tile_bounds),
                                 const_cast<float2 *>(p.tile_depth), const_cast<float4 *>(p.region_bounds), p.fh,
                                 region % nrx, region / nrx, part, true, th, HalfGroupBarrier{5 + h});
                ++done;
            }
            if (done != 0u && th < 32) {  // warp 0 of the half group wrote the bounds: one fence, one count
                __threadfence();
                __syncwarp();
                if (th == 0) atomicAdd(&p.fh->bdone, done);
            }
            // the group's bounds partials are free again (its own barrier: a bounds slot takes no vote, and a warp may
            // still be due at barrier 2 + g of an earlier tile, where warps without holes only arrive)
            bar_sync(kBarBounds + g, kGroupThreads);
        } else if (kind == kSlotPlans) {
            uint32_t done = 0u;
#pragma unroll 1
            for (int j = 0; j < kPlansPerWarp; ++j) {
                const int tile = sl.index * kPlansPerItem + j * kConsumerWarps + w;
                if (tile >= p.n5x * p.n5y) break;
                if (sl.cdt == EXW_F16) plan_tile<__half, WS::xf16, WS::yf16>(p, tile);
                else plan_tile<float, WS::xf32, WS::yf32>(p, tile);
                ++done;
            }
            if (done != 0u && lane == 0) {  // one fence and one count for the warp's plans
                __threadfence();
                atomicAdd(&p.fh->pdone, done);
            }
        } else if (kind == kSlotFixup) {
            if (sl.index == 0) {  // every node of the stream is counted: build the coarse levels, then release
                __threadfence();
                float4 *scratch = reinterpret_cast<float4 *>(s.win[b]);  // no window lands in a fix-up slot's buffer
                engine_coarse_pass(p, scratch, sl.cdt);
                fence_proxy_async_smem();  // the scratch writes before a later window lands in this buffer
                __threadfence();
                bar_sync(kBarConsumers, kConsumerThreads);
                if (tid == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&p.fh->cready), "r"(1u) : "memory");
            }
            if (sl.cdt == EXW_F16) fixup_slice<__half>(p, (uint32_t)sl.index, kFixupItems, tid, kConsumerThreads);
            else fixup_slice<float>(p, (uint32_t)sl.index, kFixupItems, tid, kConsumerThreads);
        } else {  // target tile
            uint64_t(*key)[kRegionN] = s.key[nsplat & 1u];
            if (splat) {
                if (sl.cdt == EXW_F16) tile_splat<__half, WS::xf16, WS::yf16>(s, sl, p, b, tid, key);
                else tile_splat<float, WS::xf32, WS::yf32>(s, sl, p, b, tid, key);
                ++nsplat;
            }
            if (g < p.nfrac) {
                uint64_t(*idle)[kRegionN] = s.key[(nsplat + 1u) & 1u];  // after this slot's splat, if any
                if (sl.cdt == EXW_F16) tile_group<__half, WS::xf16, WS::yf16, FILL>(s, sl, p, b, g, key, idle);
                else tile_group<float, WS::xf32, WS::yf32, FILL>(s, sl, p, b, g, key, idle);
                if (FILL && tg == 0) {
                    pend.add(p.fh);
                    if (mode == 5 && sl.pair) pend.add(p.fh);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s.empty[b]);
    }
}

}  // namespace exw
