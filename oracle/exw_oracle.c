/*
 * exw_oracle.c -- plain, slow, FP64 CPU oracle for the ExWarp warping fast path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this file; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg do.  It shares no code, header, table or helper with the CUDA
 * library: it is a direct transcription of the definitions below, pixel by pixel, in double precision.
 *
 * What the paper fixes (ExWarp, arXiv 2307.12607):
 *   - Sec. II-B: warping reprojects every location of one image to a location in a second image.
 *   - Sec. I and Sec. III-B: the fast path warps the last rendered frame with its motion vectors; the warped
 *     frame contains invalid pixels ("holes") that are marked and then filled.
 *   - Sec. IV-A/IV-B: three new frames P_1..P_3 are shown at t + i/4 between F_t and F_{t+1}, built from F_t only.
 *   - Sec. V-A2: in forward warping several source pixels can land on one target; depth resolves the conflict.
 * Everything finer than that (rounding, tie break, bilinear taps, the hole rule, the fill) the paper leaves
 * open.  This oracle takes one reading of each, stated at each function; the CUDA path follows the same readings.
 *
 * Layouts: colour planar [3][H][W] (double here), depth [H][W] float, motion [2][H][W] float (plane 0 = x),
 * keys [H][W] uint64, mask [H][W] uint8.  Pixel p = (x, y) has linear index i = y*W + x.
 *
 * Parity status: every function here is pinned by the CPU tests (closed forms, invariants, brute force, finite
 * differences and exact-arithmetic checks); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EMPTY 0xFFFFFFFFFFFFFFFFull
#define MASK_EMPTY 1u
#define MASK_CRACK 2u

static uint32_t float_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

static float bits_float(uint32_t u) {
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

/* A source pixel takes part in the splat when its depth is positive and finite and both motion components are
 * finite.  Reading: the paper does not say what to do with missing data; such pixels simply never land. */
static int splattable(float depth, float mx, float my) {
    return isfinite(depth) && depth > 0.0f && isfinite(mx) && isfinite(my);
}

/* Displacement of fraction k/denom of the motion, rounded half up to a whole pixel:
 *     off = floor(1/2 + k * mv / denom).
 * Sec. IV-B places P_k at t + k/4, so the surface at p has moved by (k/4) * mv (reading: linear motion over the
 * frame interval).  Pixel centres sit at integer coordinates, so the target pixel is the one whose centre is
 * nearest, ties going up.  For float mv and small k, k * mv has at most 26 significant bits and dividing by a
 * power of two is exact, so the double expression below is exact whenever the answer can land in a frame.
 * Returns 0 when |off| is too large to land in any frame. */
int oracle_target_offset(float mv, int k, int denom, long long *off) {
    double d = (double)k * (double)mv / (double)denom;
    double t = floor(0.5 + d);
    if (!(fabs(t) < 1.0e9)) return 0;
    *off = (long long)t;
    return 1;
}

/* Forward splat (Sec. II-B, Sec. V-A2).  Every splattable source pixel p goes to T(p) = p + off; where several
 * land on one target the nearest depth wins, and among equal depths the smallest source index.  Encoded as
 *     key[q] = min over {p : T(p) = q} of (bits(D(p)) << 32) | i_p,     EMPTY = 2^64 - 1.
 * Positive finite float bit patterns order like their values, so the minimum key is the nearest surface. */
void oracle_splat(const float *depth, const float *mv, int W, int H, int k, int denom, uint64_t *keys) {
    const size_t n = (size_t)W * (size_t)H;
    for (size_t q = 0; q < n; ++q) keys[q] = ORACLE_EMPTY;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const size_t i = (size_t)y * W + x;
            const float D = depth[i], mx = mv[i], my = mv[n + i];
            if (!splattable(D, mx, my)) continue;
            long long ox, oy;
            if (!oracle_target_offset(mx, k, denom, &ox)) continue;
            if (!oracle_target_offset(my, k, denom, &oy)) continue;
            const long long qx = x + ox, qy = y + oy;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
            const uint64_t key = ((uint64_t)float_bits(D) << 32) | (uint64_t)i;
            const size_t q = (size_t)qy * W + (size_t)qx;
            if (key < keys[q]) keys[q] = key;
        }
    }
}

/* Hole marking (Sec. III-B, Sec. III-C: invalid pixels of the warped frame).  Reading, two causes:
 *   bit 0 EMPTY: nothing landed on q.
 *   bit 1 CRACK: something landed, but at least 3 of q's in-frame 4-neighbours received a surface nearer by more
 *         than D_q / 32, i.e. q shows background through a crack in a foreground surface:
 *         count{ n : key[n] != EMPTY and D_q - D_n > D_q / 32 } >= 3,
 *         with D taken from the winning keys. */
void oracle_mask(const uint64_t *keys, int W, int H, uint8_t *mask) {
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const size_t q = (size_t)y * W + x;
            uint8_t m = 0;
            if (keys[q] == ORACLE_EMPTY) {
                m = MASK_EMPTY;
            } else {
                const double Dq = (double)bits_float((uint32_t)(keys[q] >> 32));
                const int nx[4] = {x - 1, x + 1, x, x};
                const int ny[4] = {y, y, y - 1, y + 1};
                int count = 0;
                for (int j = 0; j < 4; ++j) {
                    if (nx[j] < 0 || nx[j] >= W || ny[j] < 0 || ny[j] >= H) continue;
                    const uint64_t kn = keys[(size_t)ny[j] * W + nx[j]];
                    if (kn == ORACLE_EMPTY) continue;
                    const double Dn = (double)bits_float((uint32_t)(kn >> 32));
                    if (Dq - Dn > Dq / 32.0) ++count;
                }
                if (count >= 3) m = MASK_CRACK;
            }
            mask[q] = m;
        }
    }
}

/* The bilinear taps of winner p along one axis, given the residual rho = (T(p) - p) - k*mv/denom, which lies in
 * (-1/2, 1/2].  Target q's centre corresponds to source position p + rho (reading: motion locally constant), so
 * the colour is sampled there: one tap at p when rho = 0, else taps p and p + sign(rho) with weights 1 - |rho|
 * and |rho|.  dw[] holds d weight / d rho for the adjoint. */
static int axis_taps(double rho, int *off, double *w, double *dw) {
    if (rho == 0.0) {
        off[0] = 0; w[0] = 1.0; dw[0] = 0.0;
        return 1;
    }
    const int s = rho > 0.0 ? 1 : -1;
    off[0] = 0; w[0] = 1.0 - fabs(rho); dw[0] = -(double)s;
    off[1] = s; w[1] = fabs(rho);        dw[1] = (double)s;
    return 2;
}

/* A tap t takes part when it is inside the frame and its depth agrees with the winner's:
 * |D(t) - D(p)| <= D(p) / 32 (reading: taps across a depth edge belong to another surface). */
static int tap_agrees(double Dt, double Dp) {
    return fabs(Dt - Dp) <= Dp / 32.0;
}

/* Backward bilinear gather of colour through the splatted field (Sec. II-B, Sec. III-B), plus the hole mask.
 *     out(q) = sum_{t in A} w_t C(t) / sum_{t in A} w_t        for q not a hole,
 *     out(q) = 0                                              for a hole (mask != 0),
 * where A are the participating taps of q's winner p.  p itself always takes part with weight >= 1/4. */
void oracle_warp(const double *color, const float *depth, const float *mv, const uint64_t *keys, int W, int H,
                 int k, int denom, double *out, uint8_t *mask) {
    const size_t n = (size_t)W * (size_t)H;
    oracle_mask(keys, W, H, mask);
    for (int qy = 0; qy < H; ++qy) {
        for (int qx = 0; qx < W; ++qx) {
            const size_t q = (size_t)qy * W + qx;
            if (mask[q] != 0) {
                for (int c = 0; c < 3; ++c) out[c * n + q] = 0.0;
                continue;
            }
            const size_t p = (size_t)(keys[q] & 0xFFFFFFFFull);
            const int px = (int)(p % (size_t)W), py = (int)(p / (size_t)W);
            const double rx = (double)(qx - px) - (double)k * (double)mv[p] / (double)denom;
            const double ry = (double)(qy - py) - (double)k * (double)mv[n + p] / (double)denom;
            int ox[2], oy[2];
            double wx[2], wy[2], dwx[2], dwy[2];
            const int nx = axis_taps(rx, ox, wx, dwx);
            const int ny = axis_taps(ry, oy, wy, dwy);
            const double Dp = (double)depth[p];
            double num[3] = {0.0, 0.0, 0.0}, den = 0.0, wsum = 0.0;
            for (int b = 0; b < ny; ++b) {
                for (int a = 0; a < nx; ++a) {
                    const double w = wx[a] * wy[b];
                    wsum += w;
                    const int tx = px + ox[a], ty = py + oy[b];
                    if (tx < 0 || tx >= W || ty < 0 || ty >= H) continue;
                    const size_t t = (size_t)ty * W + tx;
                    if (!tap_agrees((double)depth[t], Dp)) continue;
                    for (int c = 0; c < 3; ++c) num[c] += w * color[c * n + t];
                    den += w;
                }
            }
            (void)wsum; /* the bilinear weights of the full tap set sum to 1; checked by the tests */
            for (int c = 0; c < 3; ++c) out[c * n + q] = num[c] / den;
        }
    }
}

/* Sum of the bilinear weights of q's full tap set (participating or not); 1 up to rounding.  Exposed so the
 * tests can check the partition of unity directly. */
double oracle_weight_sum(const float *mv, const uint64_t *keys, int W, int H, int k, int denom, int q) {
    const size_t n = (size_t)W * (size_t)H;
    if (keys[q] == ORACLE_EMPTY) return 0.0;
    const size_t p = (size_t)(keys[q] & 0xFFFFFFFFull);
    const int px = (int)(p % (size_t)W), py = (int)(p / (size_t)W);
    const int qx = q % W, qy = q / W;
    const double rx = (double)(qx - px) - (double)k * (double)mv[p] / (double)denom;
    const double ry = (double)(qy - py) - (double)k * (double)mv[n + p] / (double)denom;
    int ox[2], oy[2];
    double wx[2], wy[2], dwx[2], dwy[2];
    const int nx = axis_taps(rx, ox, wx, dwx);
    const int ny = axis_taps(ry, oy, wy, dwy);
    double s = 0.0;
    for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a) s += wx[a] * wy[b];
    return s;
}

/* Pull-push hole filling (Sec. III-C: holes must be filled before a warped frame can be shown; the paper leaves
 * the fill to its network, so the warp-only path takes the classic pull-push reading):
 *   level 0: v0 = colour, m0 = (mask == 0); level l+1 has ceil(H_l/2) x ceil(W_l/2) nodes, down to 1 x 1.
 *   pull:  node (i, j) of level l+1 averages its valid in-frame children (2i+a, 2j+b), taken in the order
 *          (a,b) = (0,0), (0,1), (1,0), (1,1); it is valid when any child is.
 *   push:  from coarse to fine, every invalid node takes the value of its parent (i>>1, j>>1); an invalid 1 x 1
 *          top (no valid pixel anywhere) becomes 0.
 *   Valid pixels keep their colour; holes take the pushed level-0 value. */
void oracle_fill_holes(double *color, const uint8_t *mask, int W, int H) {
    const size_t n = (size_t)W * (size_t)H;
    int Ws[40], Hs[40];
    int L = 0;
    Ws[0] = W; Hs[0] = H;
    while (Ws[L] > 1 || Hs[L] > 1) {
        Ws[L + 1] = (Ws[L] + 1) / 2;
        Hs[L + 1] = (Hs[L] + 1) / 2;
        ++L;
    }
    /* storage for all levels: values [3] and validity per node */
    size_t total = 0, offs[40];
    for (int l = 0; l <= L; ++l) { offs[l] = total; total += (size_t)Ws[l] * Hs[l]; }
    double *v = (double *)calloc(total * 3, sizeof(double));
    unsigned char *m = (unsigned char *)calloc(total, 1);
    for (size_t q = 0; q < n; ++q) {
        m[q] = mask[q] == 0;
        for (int c = 0; c < 3; ++c) v[3 * q + c] = color[c * n + q];
    }
    for (int l = 0; l < L; ++l) {
        const int Wc = Ws[l], Hc = Hs[l], Wp = Ws[l + 1], Hp = Hs[l + 1];
        for (int i = 0; i < Hp; ++i) {
            for (int j = 0; j < Wp; ++j) {
                double s[3] = {0.0, 0.0, 0.0};
                int cnt = 0;
                for (int a = 0; a < 2; ++a) {
                    for (int b = 0; b < 2; ++b) {
                        const int ci = 2 * i + a, cj = 2 * j + b;
                        if (ci >= Hc || cj >= Wc) continue;
                        const size_t cidx = offs[l] + (size_t)ci * Wc + cj;
                        if (!m[cidx]) continue;
                        for (int c = 0; c < 3; ++c) s[c] += v[3 * cidx + c];
                        ++cnt;
                    }
                }
                const size_t pidx = offs[l + 1] + (size_t)i * Wp + j;
                m[pidx] = cnt > 0;
                for (int c = 0; c < 3; ++c) v[3 * pidx + c] = cnt > 0 ? s[c] / (double)cnt : 0.0;
            }
        }
    }
    if (!m[offs[L]]) {
        for (int c = 0; c < 3; ++c) v[3 * offs[L] + c] = 0.0;
        m[offs[L]] = 1;
    }
    for (int l = L - 1; l >= 0; --l) {
        const int Wc = Ws[l], Hc = Hs[l], Wp = Ws[l + 1];
        for (int i = 0; i < Hc; ++i) {
            for (int j = 0; j < Wc; ++j) {
                const size_t cidx = offs[l] + (size_t)i * Wc + j;
                if (m[cidx]) continue;
                const size_t pidx = offs[l + 1] + (size_t)(i >> 1) * Wp + (j >> 1);
                for (int c = 0; c < 3; ++c) v[3 * cidx + c] = v[3 * pidx + c];
                m[cidx] = 1;
            }
        }
    }
    for (size_t q = 0; q < n; ++q) {
        if (mask[q] == 0) continue;
        for (int c = 0; c < 3; ++c) color[c * n + q] = v[3 * q + c];
    }
    free(v);
    free(m);
}

/* Adjoint of the gather (reading: the warp is differentiated with every integer decision held fixed -- T(p), the
 * winner, the tap set, tap participation and the mask).  With out_c(q) = N_c / S, N_c = sum_A w_t C_c(t),
 * S = sum_A w_t and rho = (T(p) - p) - k mv(p) / denom:
 *     d out_c / d C_c(t)  = w_t / S                                          (t in A)
 *     d out_c / d rho_a   = sum_A (d w_t / d rho_a) (C_c(t) - out_c) / S      (quotient rule)
 *     d rho_a / d mv_a(p) = -k / denom
 * Given g = dL/d out, accumulates grad_color[c][t] += g_c(q) w_t / S and
 * grad_mv[a][p] += -(k/denom) sum_c g_c(q) d out_c / d rho_a.  Holes contribute nothing (their output is 0). */
void oracle_warp_backward(const double *grad_out, const double *color, const float *depth, const float *mv,
                          const uint64_t *keys, int W, int H, int k, int denom, double *grad_color,
                          double *grad_mv) {
    const size_t n = (size_t)W * (size_t)H;
    uint8_t *mask = (uint8_t *)malloc(n ? n : 1);
    oracle_mask(keys, W, H, mask);
    for (int qy = 0; qy < H; ++qy) {
        for (int qx = 0; qx < W; ++qx) {
            const size_t q = (size_t)qy * W + qx;
            if (mask[q] != 0) continue;
            const size_t p = (size_t)(keys[q] & 0xFFFFFFFFull);
            const int px = (int)(p % (size_t)W), py = (int)(p / (size_t)W);
            const double rx = (double)(qx - px) - (double)k * (double)mv[p] / (double)denom;
            const double ry = (double)(qy - py) - (double)k * (double)mv[n + p] / (double)denom;
            int ox[2], oy[2];
            double wx[2], wy[2], dwx[2], dwy[2];
            const int nx = axis_taps(rx, ox, wx, dwx);
            const int ny = axis_taps(ry, oy, wy, dwy);
            const double Dp = (double)depth[p];
            /* participating taps */
            size_t tidx[4];
            double tw[4], tdx[4], tdy[4];
            int na = 0;
            for (int b = 0; b < ny; ++b) {
                for (int a = 0; a < nx; ++a) {
                    const int tx = px + ox[a], ty = py + oy[b];
                    if (tx < 0 || tx >= W || ty < 0 || ty >= H) continue;
                    const size_t t = (size_t)ty * W + tx;
                    if (!tap_agrees((double)depth[t], Dp)) continue;
                    tidx[na] = t;
                    tw[na] = wx[a] * wy[b];
                    tdx[na] = dwx[a] * wy[b];
                    tdy[na] = wx[a] * dwy[b];
                    ++na;
                }
            }
            double S = 0.0;
            for (int j = 0; j < na; ++j) S += tw[j];
            double outc[3];
            for (int c = 0; c < 3; ++c) {
                double N = 0.0;
                for (int j = 0; j < na; ++j) N += tw[j] * color[c * n + tidx[j]];
                outc[c] = N / S;
            }
            double gx = 0.0, gy = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double g = grad_out[c * n + q];
                double drx = 0.0, dry = 0.0;
                for (int j = 0; j < na; ++j) {
                    const double diff = color[c * n + tidx[j]] - outc[c];
                    drx += tdx[j] * diff;
                    dry += tdy[j] * diff;
                    grad_color[c * n + tidx[j]] += g * tw[j] / S;
                }
                gx += g * drx / S;
                gy += g * dry / S;
            }
            const double scale = -(double)k / (double)denom;
            grad_mv[p] += scale * gx;
            grad_mv[n + p] += scale * gy;
        }
    }
    free(mask);
}

/* Motion bounds over the splattable pixels of each block x block tile (the halo that bounds how far a source
 * pixel can land): per tile [min mv_x, max mv_x, min mv_y, max mv_y], each component first clamped to
 * [-65536, 65536] (beyond that no fraction of the motion can land in a 16384-pixel frame) and -0 read as +0.  A tile without
 * splattable pixels reports [+inf, -inf, +inf, -inf].  frame[4] receives the same over the whole frame. */
void oracle_motion_bounds(const float *depth, const float *mv, int W, int H, int block, float *tiles,
                          float *frame) {
    const size_t n = (size_t)W * (size_t)H;
    const int nbx = (W + block - 1) / block, nby = (H + block - 1) / block;
    for (int t = 0; t < nbx * nby; ++t) {
        tiles[4 * t + 0] = INFINITY; tiles[4 * t + 1] = -INFINITY;
        tiles[4 * t + 2] = INFINITY; tiles[4 * t + 3] = -INFINITY;
    }
    frame[0] = INFINITY; frame[1] = -INFINITY; frame[2] = INFINITY; frame[3] = -INFINITY;
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            const size_t i = (size_t)y * W + x;
            const float D = depth[i];
            float mx = mv[i], my = mv[n + i];
            if (!splattable(D, mx, my)) continue;
            mx = mx < -65536.0f ? -65536.0f : (mx > 65536.0f ? 65536.0f : mx);
            my = my < -65536.0f ? -65536.0f : (my > 65536.0f ? 65536.0f : my);
            if (mx == 0.0f) mx = 0.0f; /* one zero: -0 and +0 are the same motion */
            if (my == 0.0f) my = 0.0f;
            float *b = tiles + 4 * ((size_t)(y / block) * nbx + (x / block));
            if (mx < b[0]) b[0] = mx;
            if (mx > b[1]) b[1] = mx;
            if (my < b[2]) b[2] = my;
            if (my > b[3]) b[3] = my;
            if (mx < frame[0]) frame[0] = mx;
            if (mx > frame[1]) frame[1] = mx;
            if (my < frame[2]) frame[2] = my;
            if (my > frame[3]) frame[3] = my;
        }
    }
}

/* Motion-variance features Var_x(F_mv), Var_y(F_mv) of the environment vector E_t (Sec. IV-C, Eq. 1; the feature
 * is motivated in Sec. III-D): over every pixel whose two motion components are finite, the population variance
 * of the x component and of the y component, by two passes in FP64 -- the mean, then the mean of the squared
 * deviations.  out[0] = the number of pixels counted, out[1] = Var_x, out[2] = Var_y (0 and 0 for an empty set). */
void oracle_mv_variance(const float *mv, int W, int H, double *out) {
    const size_t n = (size_t)W * (size_t)H;
    double cnt = 0.0, sx = 0.0, sy = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!isfinite(mv[i]) || !isfinite(mv[n + i])) continue;
        cnt += 1.0;
        sx += (double)mv[i];
        sy += (double)mv[n + i];
    }
    out[0] = cnt;
    out[1] = out[2] = 0.0;
    if (cnt == 0.0) return;
    const double mx = sx / cnt, my = sy / cnt;
    double vx = 0.0, vy = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (!isfinite(mv[i]) || !isfinite(mv[n + i])) continue;
        const double dx = (double)mv[i] - mx, dy = (double)mv[n + i] - my;
        vx += dx * dx;
        vy += dy * dy;
    }
    out[1] = vx / cnt;
    out[2] = vy / cnt;
}

/* Mean squared difference of two colour images [3][H][W] over all 3 W H values, FP64: the MSE of the reward's
 * PSNR = 10 log10(255^2 / MSE) (Sec. IV-C, Eq. 3) for colours in [0, 1] scaled by 255. */
double oracle_color_mse(const double *a, const double *b, int W, int H) {
    const size_t n = 3 * (size_t)W * (size_t)H;
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const double d = a[i] - b[i];
        s += d * d;
    }
    return s / (double)n;
}

/* Structural similarity of two colour images [3][H][W] (the SSIM of the reward, Sec. IV-C, Eq. 3; the paper names
 * it without a formula, read as the standard index of Wang, Bovik, Sheikh and Simoncelli, 2004): per channel and
 * per position of an 11 x 11 Gaussian window (sigma 1.5, weights normalised to sum 1) lying wholly inside the
 * image, with weighted means mu, variances sigma^2 = E[v^2] - mu^2 and covariance sigma_xy = E[ab] - mu_a mu_b,
 *     SSIM = (2 mu_a mu_b + C1)(2 sigma_ab + C2) / ((mu_a^2 + mu_b^2 + C1)(sigma_a^2 + sigma_b^2 + C2)),
 * C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = 1 (colours in [0, 1]); the result is the mean over channels and positions.
 * Needs W, H >= 11 (else returns NaN).  Straight FP64 sums over the 121 taps. */
double oracle_ssim(const double *a, const double *b, int W, int H) {
    if (W < 11 || H < 11) return NAN;
    double g[11], gs = 0.0;
    for (int i = 0; i < 11; ++i) {
        g[i] = exp(-((double)(i - 5) * (double)(i - 5)) / (2.0 * 1.5 * 1.5));
        gs += g[i];
    }
    for (int i = 0; i < 11; ++i) g[i] /= gs;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    const size_t plane = (size_t)W * (size_t)H;
    double total = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double *pa = a + c * plane, *pb = b + c * plane;
        for (int y = 0; y + 11 <= H; ++y) {
            for (int x = 0; x + 11 <= W; ++x) {
                double ma = 0.0, mb = 0.0, saa = 0.0, sbb = 0.0, sab = 0.0;
                for (int i = 0; i < 11; ++i) {
                    for (int j = 0; j < 11; ++j) {
                        const double w = g[i] * g[j];
                        const double va = pa[(size_t)(y + i) * W + (x + j)], vb = pb[(size_t)(y + i) * W + (x + j)];
                        ma += w * va;
                        mb += w * vb;
                        saa += w * va * va;
                        sbb += w * vb * vb;
                        sab += w * va * vb;
                    }
                }
                const double va2 = saa - ma * ma, vb2 = sbb - mb * mb, cab = sab - ma * mb;
                total += ((2.0 * ma * mb + C1) * (2.0 * cab + C2)) / ((ma * ma + mb * mb + C1) * (va2 + vb2 + C2));
            }
        }
    }
    return total / (3.0 * (double)(W - 10) * (double)(H - 10));
}

/* Depth and motion of a warped frame, so that it can be warped again (the recursive warps W(P_1), W(P_2) of the
 * decision paths S5 and S6, Table V; the paper leaves the motion of a predicted frame open, read as the motion of
 * the surface that landed there): a target that is not a hole (mask 0) takes the depth and motion of its winner,
 * the source in its key; a hole gets depth NaN (it never lands again) and motion 0. */
void oracle_carry_motion(const uint64_t *keys, const uint8_t *mask, const float *depth, const float *mv, int W, int H,
                         float *depth_out, float *mv_out) {
    const size_t n = (size_t)W * (size_t)H;
    for (size_t q = 0; q < n; ++q) {
        if (mask[q] == 0 && keys[q] != ORACLE_EMPTY) {
            const size_t p = (size_t)(keys[q] & 0xFFFFFFFFull);
            depth_out[q] = depth[p];
            mv_out[q] = mv[p];
            mv_out[n + q] = mv[n + p];
        } else {
            depth_out[q] = NAN;
            mv_out[q] = 0.0f;
            mv_out[n + q] = 0.0f;
        }
    }
}
