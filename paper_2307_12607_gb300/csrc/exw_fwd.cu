// exw_fwd.cu -- forward tile kernels: fused splat+gather+fill, staged gather, staged fill, coarse fix-up.
//
// A CTA owns one 32 x 32 target tile Q (grid = ceil(W/32) x ceil(H/32)).  The fused kernel builds the keys of
// Q plus a one-pixel ring in shared memory by splatting every source 8 x 8 block whose motion bounds can reach
// it (64-bit shared atomicMin), then gathers colour per pixel with lane = x (coalesced 128-byte rows), builds
// pyramid levels 1..5 of the tile in shared memory and fills holes from them.  Tiles with no valid pixel are
// filled afterwards from the coarse levels, which the last CTA to finish computes (a done-counter in the
// workspace; no grid-wide barrier and no spin).
#include "exw_device.cuh"
#include "exw_internal.h"

namespace exw {

constexpr int kThreads = 256;
constexpr int kRegionN = kRegion * kRegion;

struct FusedSmem {
    uint64_t key[kMaxFrac][kRegionN];
    FillSmem fill;
    uint32_t cand[kThreads];
    uint32_t ncand;
    int last;
};

// ------------------------------------------------------------------------------------------------------------
// Stage (b) for one pixel of a tile from shared keys of the region (tile + ring).  Returns the mask; c[] is the
// colour rounded to the storage type (0 for holes).
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__device__ __forceinline__ uint8_t warp_pixel(const uint64_t *sk, int x, int y, int k, const TileParams &p, float c[3]) {
    const uint64_t kq = sk[(y + 1) * kRegion + (x + 1)];
    c[0] = c[1] = c[2] = 0.0f;
    if (kq == kKeyEmpty) return (uint8_t)EXW_MASK_EMPTY;
    if (is_crack(kq, sk[(y + 1) * kRegion + x], sk[(y + 1) * kRegion + x + 2], sk[y * kRegion + x + 1],
                 sk[(y + 2) * kRegion + x + 1]))
        return (uint8_t)EXW_MASK_CRACK;
    const uint32_t lo = (uint32_t)kq;
    float v[3];
    gather_pixel<CT>(key_dbits(kq), (int)(lo & 0x3FFFu), (int)(lo >> 14), k, p.L, (const CT *)p.color, p.depth,
                     p.mv, p.W, p.H, (size_t)p.W * p.H, v);
    c[0] = storage_round<CT>(v[0]);
    c[1] = storage_round<CT>(v[1]);
    c[2] = storage_round<CT>(v[2]);
    return 0;
}

// ------------------------------------------------------------------------------------------------------------
// Coarse levels of the pyramid (above level 5) for every fraction with invalid tiles, and the value each invalid
// tile receives (its first valid ancestor; 0 when the frame has no valid pixel).  Run by one CTA.
// ------------------------------------------------------------------------------------------------------------
__device__ void coarse_pass(const TileParams &p) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n5 = p.n5x * p.n5y;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const uint32_t cnt = __ldcg(&p.fh->ninvalid[kk]);
        if (cnt == 0u) continue;
        const float4 *child = p.nodes + (size_t)kk * n5;
        float4 *cz = p.coarse + (size_t)kk * p.ncoarse;
        int cw = p.n5x, ch = p.n5y, off = 0;
        while (cw > 1 || ch > 1) {
            const int pw = (cw + 1) / 2, ph = (ch + 1) / 2;
            float4 *par = cz + off;
            for (int node = tid; node < pw * ph; node += nt) {
                const int i = node / pw, j = node - (node / pw) * pw;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                int c = 0;
                for (int a = 0; a < 2; ++a) {
                    for (int b = 0; b < 2; ++b) {
                        const int ci = 2 * i + a, cj = 2 * j + b;
                        if (ci >= ch || cj >= cw) continue;
                        const float4 v = __ldcg(child + ci * cw + cj);
                        if (v.w != 0.0f) {
                            a0 += v.x;
                            a1 += v.y;
                            a2 += v.z;
                            ++c;
                        }
                    }
                }
                const float fc = (float)c;
                par[node] = c ? make_float4(a0 / fc, a1 / fc, a2 / fc, 1.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            child = par;
            off += pw * ph;
            cw = pw;
            ch = ph;
        }
        for (uint32_t e = tid; e < cnt; e += nt) {
            const uint32_t tile = __ldcg(p.list + (size_t)kk * n5 + e);
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
        __syncthreads();
    }
}

// Write the level-5 node of this tile for fraction kk; list the tile if it has no valid pixel.
__device__ __forceinline__ void publish_node(const TileParams &p, const FillSmem &fs, int kk) {
    const float4 node = fs.lv[340];
    const int n5 = p.n5x * p.n5y;
    const int tile = blockIdx.y * p.n5x + blockIdx.x;
    p.nodes[(size_t)kk * n5 + tile] = node;
    if (node.w == 0.0f) {
        const uint32_t slot = atomicAdd(&p.fh->ninvalid[kk], 1u);
        p.list[(size_t)kk * n5 + slot] = (uint32_t)tile;
    }
}

// The last CTA to finish runs the coarse pass.
__device__ __forceinline__ void finish_grid(const TileParams &p, int *last) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t total = gridDim.x * gridDim.y;
        *last = atomicAdd(&p.fh->done, 1u) == total - 1u;
    }
    __syncthreads();
    if (*last) {
        __threadfence();
        coarse_pass(p);
    }
}

// ------------------------------------------------------------------------------------------------------------
// Shared-memory splat of every candidate source block into the region keys of all fractions.
// ------------------------------------------------------------------------------------------------------------
__device__ __forceinline__ void splat_region(FusedSmem &s, const TileParams &p, int RX0, int RY0) {
    const int tid = threadIdx.x;
    const uint32_t a0 = __ldcg(&p.fh->acc[0]), a1 = __ldcg(&p.fh->acc[1]);
    const uint32_t a2 = __ldcg(&p.fh->acc[2]), a3 = __ldcg(&p.fh->acc[3]);
    if (a1 == 0u) return;  // no source pixel can land anywhere (block-uniform)
    const uint32_t fminx = __float_as_uint(-float_unorder(a0)), fmaxx = __float_as_uint(float_unorder(a1));
    const uint32_t fminy = __float_as_uint(-float_unorder(a2)), fmaxy = __float_as_uint(float_unorder(a3));
    int xlo = 1 << 30, xhi = -(1 << 30), ylo = 1 << 30, yhi = -(1 << 30);
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const int k = p.k0 + kk;
        const int ox0 = axis_step(fminx, k, p.L).off, ox1 = axis_step(fmaxx, k, p.L).off;
        const int oy0 = axis_step(fminy, k, p.L).off, oy1 = axis_step(fmaxy, k, p.L).off;
        xlo = min(xlo, RX0 - ox1);
        xhi = max(xhi, RX0 + kRegion - 1 - ox0);
        ylo = min(ylo, RY0 - oy1);
        yhi = max(yhi, RY0 + kRegion - 1 - oy0);
    }
    const int bx0 = max(0, xlo >> 3), bx1 = min(p.nbx - 1, xhi >> 3);
    const int by0 = max(0, ylo >> 3), by1 = min(p.nby - 1, yhi >> 3);
    if (bx1 < bx0 || by1 < by0) return;
    const int nbxr = bx1 - bx0 + 1;
    const int total = nbxr * (by1 - by0 + 1);
    const size_t plane = (size_t)p.W * p.H;
    for (int base = 0; base < total; base += kThreads) {
        if (tid == 0) s.ncand = 0u;
        __syncthreads();
        const int idx = base + tid;
        if (idx < total) {
            const int bx = bx0 + idx % nbxr, by = by0 + idx / nbxr;
            const float4 b = __ldg(p.tile_bounds + (size_t)by * p.nbx + bx);
            if (b.x <= b.y) {
                uint32_t fm = 0;
                for (int kk = 0; kk < p.nfrac; ++kk) {
                    const int k = p.k0 + kk;
                    const int tx0 = 8 * bx + axis_step(__float_as_uint(b.x), k, p.L).off;
                    const int tx1 = 8 * bx + 7 + axis_step(__float_as_uint(b.y), k, p.L).off;
                    const int ty0 = 8 * by + axis_step(__float_as_uint(b.z), k, p.L).off;
                    const int ty1 = 8 * by + 7 + axis_step(__float_as_uint(b.w), k, p.L).off;
                    if (tx1 >= RX0 && tx0 < RX0 + kRegion && ty1 >= RY0 && ty0 < RY0 + kRegion) fm |= 1u << kk;
                }
                if (fm) {
                    const uint32_t slot = atomicAdd(&s.ncand, 1u);
                    s.cand[slot] = (uint32_t)bx | ((uint32_t)by << 12) | (fm << 24);
                }
            }
        }
        __syncthreads();
        const int nc = (int)s.ncand;
        for (int c0 = 0; c0 < nc; c0 += kThreads / 64) {
            const int ci = c0 + (tid >> 6);
            if (ci < nc) {
                const uint32_t e = s.cand[ci];
                const int bx = (int)(e & 0xFFFu), by = (int)((e >> 12) & 0xFFFu);
                const uint32_t fm = e >> 24;
                const int x = 8 * bx + (tid & 7), y = 8 * by + ((tid >> 3) & 7);
                if (x < p.W && y < p.H) {
                    const size_t i = (size_t)y * p.W + x;
                    const uint32_t db = __float_as_uint(__ldg(p.depth + i));
                    const uint32_t ux = __float_as_uint(__ldg(p.mv + i));
                    const uint32_t uy = __float_as_uint(__ldg(p.mv + plane + i));
                    if (depth_ok(db) && finite_bits(ux) && finite_bits(uy)) {
                        const uint64_t key = pack_key_local(db, x, y);
                        for (int kk = 0; kk < p.nfrac; ++kk) {
                            if (!(fm & (1u << kk))) continue;
                            const int k = p.k0 + kk;
                            const AxisStep sx = axis_step(ux, k, p.L), sy = axis_step(uy, k, p.L);
                            if (!sx.ok || !sy.ok) continue;
                            const int gx = x + sx.off, gy = y + sy.off;
                            if (gx < 0 || gx >= p.W || gy < 0 || gy >= p.H) continue;
                            const int rx = gx - RX0, ry = gy - RY0;
                            if ((unsigned)rx < (unsigned)kRegion && (unsigned)ry < (unsigned)kRegion)
                                atomicMin((unsigned long long *)&s.key[kk][ry * kRegion + rx], (unsigned long long)key);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------------------
// Fused stages (a)+(b)+(c) for all fractions of one target tile.
// ------------------------------------------------------------------------------------------------------------
template <typename CT, bool FILL>
__global__ void __launch_bounds__(kThreads) fused_kernel(TileParams p) {
    __shared__ __align__(16) FusedSmem s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    for (int i = tid; i < p.nfrac * kRegionN; i += kThreads) (&s.key[0][0])[i] = kKeyEmpty;
    __syncthreads();
    splat_region(s, p, X0 - 1, Y0 - 1);
    __syncthreads();
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const int k = p.k0 + kk;
        CT *oc = (CT *)p.out_color[kk];
        uint8_t *om = p.out_mask[kk];
        uint8_t mreg[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int y = wid + 8 * j, gy = Y0 + y;
            const bool in = gx < p.W && gy < p.H;
            float c[3] = {0.f, 0.f, 0.f};
            uint8_t m = 0;
            if (in) m = warp_pixel<CT>(s.key[kk], lane, y, k, p, c);
            mreg[j] = m;
            if (FILL) {
                s.fill.v0[0][y][lane] = c[0];
                s.fill.v0[1][y][lane] = c[1];
                s.fill.v0[2][y][lane] = c[2];
                s.fill.m0[y][lane] = in && m == 0;
            } else if (in) {
                const size_t q = (size_t)gy * p.W + gx;
                oc[q] = to_storage<CT>(c[0]);
                oc[plane + q] = to_storage<CT>(c[1]);
                oc[2 * plane + q] = to_storage<CT>(c[2]);
                om[q] = m;
            }
        }
        if (FILL) {
            __syncthreads();
            pull_tile(s.fill);
            const bool tile_valid = s.fill.lv[340].w != 0.0f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int y = wid + 8 * j, gy = Y0 + y;
                if (gx >= p.W || gy >= p.H) continue;
                const size_t q = (size_t)gy * p.W + gx;
                om[q] = mreg[j];
                if (!tile_valid) continue;  // every pixel is a hole; the coarse fix-up writes them
                float c0 = s.fill.v0[0][y][lane], c1 = s.fill.v0[1][y][lane], c2 = s.fill.v0[2][y][lane];
                if (mreg[j]) {
                    const float4 v = push_value(s.fill, y, lane);
                    c0 = v.x;
                    c1 = v.y;
                    c2 = v.z;
                }
                oc[q] = to_storage<CT>(c0);
                oc[plane + q] = to_storage<CT>(c1);
                oc[2 * plane + q] = to_storage<CT>(c2);
            }
            if (tid == 0) publish_node(p, s.fill, kk);
            __syncthreads();
        }
    }
    if (FILL) finish_grid(p, &s.last);
}

// ------------------------------------------------------------------------------------------------------------
// Staged stage (b): keys from global memory (exw_splat_motion), one fraction, no fill.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void __launch_bounds__(kThreads) warp_tiles_kernel(TileParams p) {
    __shared__ uint64_t key[kRegionN];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    const uint32_t npix = (uint32_t)p.W * (uint32_t)p.H;
    for (int i = tid; i < kRegionN; i += kThreads) {
        const int ry = i / kRegion, rx = i - ry * kRegion;
        const int gx = X0 - 1 + rx, gy = Y0 - 1 + ry;
        uint64_t kv = kKeyEmpty;
        if (gx >= 0 && gx < p.W && gy >= 0 && gy < p.H) {
            const uint64_t g = __ldg((const unsigned long long *)p.keys + (size_t)gy * p.W + gx);
            const uint32_t idx = (uint32_t)g;
            if (g != kKeyEmpty && idx < npix) {  // a malformed key reads as empty instead of faulting
                const uint32_t py = idx / (uint32_t)p.W, px = idx - py * (uint32_t)p.W;
                kv = pack_key_local(key_dbits(g), (int)px, (int)py);
            }
        }
        key[i] = kv;
    }
    __syncthreads();
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    CT *oc = (CT *)p.out_color[0];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = wid + 8 * j, gy = Y0 + y;
        if (gx >= p.W || gy >= p.H) continue;
        float c[3];
        const uint8_t m = warp_pixel<CT>(key, lane, y, p.k0, p, c);
        const size_t q = (size_t)gy * p.W + gx;
        oc[q] = to_storage<CT>(c[0]);
        oc[plane + q] = to_storage<CT>(c[1]);
        oc[2 * plane + q] = to_storage<CT>(c[2]);
        p.out_mask[0][q] = m;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Staged stage (c): pull-push of an existing colour + mask, in place.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void __launch_bounds__(kThreads) fill_tiles_kernel(TileParams p) {
    __shared__ __align__(16) FillSmem fs;
    __shared__ int last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int X0 = blockIdx.x * kFillTile, Y0 = blockIdx.y * kFillTile;
    const size_t plane = (size_t)p.W * p.H;
    const int gx = X0 + lane;
    CT *oc = (CT *)p.out_color[0];
    bool hole[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int y = wid + 8 * j, gy = Y0 + y;
        const bool in = gx < p.W && gy < p.H;
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
        uint8_t m = 1;
        if (in) {
            const size_t q = (size_t)gy * p.W + gx;
            m = __ldg(p.mask_in + q);
            c0 = load_c<CT>(oc + q);
            c1 = load_c<CT>(oc + plane + q);
            c2 = load_c<CT>(oc + 2 * plane + q);
        }
        hole[j] = in && m != 0;
        fs.v0[0][y][lane] = c0;
        fs.v0[1][y][lane] = c1;
        fs.v0[2][y][lane] = c2;
        fs.m0[y][lane] = in && m == 0;
    }
    __syncthreads();
    pull_tile(fs);
    if (fs.lv[340].w != 0.0f) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!hole[j]) continue;
            const int y = wid + 8 * j;
            const size_t q = (size_t)(Y0 + y) * p.W + gx;
            const float4 v = push_value(fs, y, lane);
            oc[q] = to_storage<CT>(v.x);
            oc[plane + q] = to_storage<CT>(v.y);
            oc[2 * plane + q] = to_storage<CT>(v.z);
        }
    }
    if (tid == 0) publish_node(p, fs, 0);
    finish_grid(p, &last);
}

// ------------------------------------------------------------------------------------------------------------
// Fix-up: every tile without a valid pixel takes the coarse value chosen for it.
// ------------------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void __launch_bounds__(kThreads) fixup_kernel(TileParams p) {
    const int n5 = p.n5x * p.n5y;
    const size_t plane = (size_t)p.W * p.H;
    for (int kk = 0; kk < p.nfrac; ++kk) {
        const uint32_t cnt = p.fh->ninvalid[kk];
        CT *oc = (CT *)p.out_color[kk];
        for (uint32_t e = blockIdx.x; e < cnt; e += gridDim.x) {
            const uint32_t tile = p.list[(size_t)kk * n5 + e];
            const float4 v = p.fillval[(size_t)kk * n5 + e];
            const int X0 = (int)(tile % (uint32_t)p.n5x) * kFillTile, Y0 = (int)(tile / (uint32_t)p.n5x) * kFillTile;
            const CT c0 = to_storage<CT>(v.x), c1 = to_storage<CT>(v.y), c2 = to_storage<CT>(v.z);
            for (int i = threadIdx.x; i < kFillTile * kFillTile; i += kThreads) {
                const int gx = X0 + (i & 31), gy = Y0 + (i >> 5);
                if (gx >= p.W || gy >= p.H) continue;
                const size_t q = (size_t)gy * p.W + gx;
                oc[q] = c0;
                oc[plane + q] = c1;
                oc[2 * plane + q] = c2;
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Launchers
// ------------------------------------------------------------------------------------------------------------
static dim3 tile_grid(const TileParams &p) { return dim3((unsigned)p.n5x, (unsigned)p.n5y, 1); }

cudaError_t launch_fused(const TileParams &p, exw_dtype cdt, bool fill, cudaStream_t s) {
    const dim3 g = tile_grid(p);
    timing_begin("exw_fused", s);
    if (cdt == EXW_F32) {
        if (fill) fused_kernel<float, true><<<g, kThreads, 0, s>>>(p);
        else fused_kernel<float, false><<<g, kThreads, 0, s>>>(p);
    } else {
        if (fill) fused_kernel<__half, true><<<g, kThreads, 0, s>>>(p);
        else fused_kernel<__half, false><<<g, kThreads, 0, s>>>(p);
    }
    count_launch();
    timing_end("exw_fused", s);
    return cudaGetLastError();
}

cudaError_t launch_warp_tiles(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const dim3 g = tile_grid(p);
    timing_begin("exw_warp_tiles", s);
    if (cdt == EXW_F32) warp_tiles_kernel<float><<<g, kThreads, 0, s>>>(p);
    else warp_tiles_kernel<__half><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_warp_tiles", s);
    return cudaGetLastError();
}

cudaError_t launch_fill_tiles(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const dim3 g = tile_grid(p);
    timing_begin("exw_fill_tiles", s);
    if (cdt == EXW_F32) fill_tiles_kernel<float><<<g, kThreads, 0, s>>>(p);
    else fill_tiles_kernel<__half><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_fill_tiles", s);
    return cudaGetLastError();
}

cudaError_t launch_fixup(const TileParams &p, exw_dtype cdt, cudaStream_t s) {
    const int n5 = p.n5x * p.n5y;
    const unsigned g = (unsigned)(n5 < 304 ? n5 : 304);
    timing_begin("exw_fixup", s);
    if (cdt == EXW_F32) fixup_kernel<float><<<g, kThreads, 0, s>>>(p);
    else fixup_kernel<__half><<<g, kThreads, 0, s>>>(p);
    count_launch();
    timing_end("exw_fixup", s);
    return cudaGetLastError();
}

}  // namespace exw
