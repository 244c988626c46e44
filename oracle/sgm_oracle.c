/*
 * CPU oracle for the SGM hot path of Hernandez-Juarez et al., "Embedded
 * real-time stereo estimation via Semi-Global Matching on the GPU"
 * (arXiv 1610.04121).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously-correct
 * statement of what the GPU path must compute.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Every quantity is an int32 and every loop follows the paper's definitions
 * in the paper's order; there is no blocking, fusion or vectorisation.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *  - s(u, v) = 1 if u >= v, else 0 (Section 3.1, Eq. 1).
 *  - Bit k of the CSCT feature is the k-th comparison of Eq. 1 in its printed
 *    order: i = 1..4 (outer), j = -3..3 (inner), then the three i = 0 pairs
 *    j = 1..3; bit 0 is the least significant bit.
 *  - The feature is 0 wherever the 9x7 window leaves the image
 *    (4 <= x <= W-5 and 3 <= y <= H-4 are the valid centres).
 *  - In Eq. 2 a match column x-d < 0 uses the feature 0.
 *  - Eq. 3 at the first pixel of a path (p - r outside the image) is
 *    L_r(p, d) = MC(p, d); disparities d-1 < 0 and d+1 >= D drop out of
 *    the minimum.
 *  - Eq. 4 breaks ties toward the lowest d.
 *  - The 3x3 median (Section 2, stage 4) takes the 5th of the 9 sorted
 *    values in the interior and copies the raw disparity on the one-pixel
 *    border ring (and everywhere when W < 3 or H < 3).
 *  - Path sets: 2 paths = left-to-right and top-to-bottom; 4 paths adds
 *    right-to-left and bottom-to-top; 8 paths adds the four diagonals
 *    (Section 4).
 *  - The full Census transform the paper compares CSCT against (CT,
 *    Section 2, related work): every pixel of the 9x7 window but the centre
 *    against the centre, bit k = s(I(x+i, y+j), I(x, y)) for the k-th
 *    (j, i) of j = -3..3 (outer), i = -4..4 (inner) with (0, 0) skipped:
 *    62 bits, LSB first, 0 wherever the window leaves the image.
 *  - The post-filters the paper announces for later work (Section 5:
 *    left-right consistency check, sub-pixel disparity, adaptive P2) are
 *    named there without a definition; oracle_sgm_ex states the readings
 *    taken here, each from the standard SGM formulation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EXPORT __attribute__((visibility("default")))

/* s(u, v) of Eq. 1. */
static int census_s(int u, int v) { return u >= v ? 1 : 0; }

static int pixel(const uint8_t *I, int W, int x, int y) { return (int)I[(size_t)y * W + x]; }

/*
 * Eq. 1 (Section 3.1): the 9x7 center-symmetric Census transform of pixel
 * (x, y); 0 when the window leaves the image.
 */
ORACLE_EXPORT uint32_t oracle_csct_at(const uint8_t *I, int W, int H, int x, int y) {
    uint32_t f = 0;
    int inside = (x - 4 >= 0) && (x + 4 <= W - 1) && (y - 3 >= 0) && (y + 3 <= H - 1);
    if (!inside) return 0;
    int k = 0;
    for (int i = 1; i <= 4; ++i) {
        for (int j = -3; j <= 3; ++j) {
            int bit = census_s(pixel(I, W, x + i, y + j), pixel(I, W, x - i, y - j));
            f |= (uint32_t)bit << k;
            ++k;
        }
    }
    for (int j = 1; j <= 3; ++j) {
        int bit = census_s(pixel(I, W, x, y + j), pixel(I, W, x, y - j));
        f |= (uint32_t)bit << k;
        ++k;
    }
    return f;
}

/* Eq. 1 over the whole image: F[y*W + x] = CSCT(I, x, y). */
ORACLE_EXPORT void oracle_csct(const uint8_t *I, int W, int H, uint32_t *F) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) F[(size_t)y * W + x] = oracle_csct_at(I, W, H, x, y);
}

/*
 * The full 9x7 Census transform (CT) of pixel (x, y): the 62 comparisons of a
 * window pixel against the centre, s(I(neighbour), I(centre)); 0 when the
 * window leaves the image.
 */
ORACLE_EXPORT uint64_t oracle_ct62_at(const uint8_t *I, int W, int H, int x, int y) {
    uint64_t f = 0;
    int inside = (x - 4 >= 0) && (x + 4 <= W - 1) && (y - 3 >= 0) && (y + 3 <= H - 1);
    if (!inside) return 0;
    int k = 0;
    for (int j = -3; j <= 3; ++j) {
        for (int i = -4; i <= 4; ++i) {
            if (i == 0 && j == 0) continue;
            int bit = census_s(pixel(I, W, x + i, y + j), pixel(I, W, x, y));
            f |= (uint64_t)bit << k;
            ++k;
        }
    }
    return f;
}

/* CT over the whole image: F[y*W + x] = CT(I, x, y). */
ORACLE_EXPORT void oracle_ct62(const uint8_t *I, int W, int H, uint64_t *F) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) F[(size_t)y * W + x] = oracle_ct62_at(I, W, H, x, y);
}

/* bitcount of a 64-bit feature difference, a plain loop over the 64 bits. */
ORACLE_EXPORT int oracle_bitcount64(uint64_t v) {
    int c = 0;
    for (int b = 0; b < 64; ++b) c += (int)((v >> b) & 1u);
    return c;
}

/* Eq. 2 with CT features: MC = bitcount(F_base(x, y) XOR F_match(x-d, y)). */
ORACLE_EXPORT void oracle_cost64(const uint64_t *Fb, const uint64_t *Fm, int W, int H, int D, uint8_t *MC) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d) {
                uint64_t m = (x - d >= 0) ? Fm[(size_t)y * W + (x - d)] : 0;
                MC[((size_t)y * W + x) * D + d] = (uint8_t)oracle_bitcount64(Fb[(size_t)y * W + x] ^ m);
            }
}

/* bitcount of Eq. 2, written as a plain loop over the 32 bit positions. */
ORACLE_EXPORT int oracle_bitcount(uint32_t v) {
    int c = 0;
    for (int b = 0; b < 32; ++b) c += (int)((v >> b) & 1u);
    return c;
}

/* Match feature used by Eq. 2: zero left of the image. */
static uint32_t match_feature(const uint32_t *Fm, int W, int x, int y) {
    if (x < 0) return 0;
    return Fm[(size_t)y * W + x];
}

/*
 * Eq. 2 (Section 3.1): MC(x, y, d) = bitcount(F_base(x, y) XOR F_match(x-d, y)).
 * Output layout MC[y][x][d], d fastest (Section 3.1, layout discussion).
 */
ORACLE_EXPORT void oracle_cost(const uint32_t *Fb, const uint32_t *Fm, int W, int H, int D, uint8_t *MC) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d) {
                uint32_t v = Fb[(size_t)y * W + x] ^ match_feature(Fm, W, x - d, y);
                MC[((size_t)y * W + x) * D + d] = (uint8_t)oracle_bitcount(v);
            }
}

/*
 * Adaptive P2 (announced in Section 5; reading): for the step from q to p
 * the jump penalty is P2(p, q) = max(P1, P2 / (1 + |I_b(p) - I_b(q)|)), integer
 * division, I_b the base image: a large intensity step along the path makes
 * a disparity jump cheaper, never cheaper than P1.
 */
static int adaptive_p2(const uint8_t *Ib, int W, int x, int y, int qx, int qy, int P1, int P2) {
    int g = pixel(Ib, W, x, y) - pixel(Ib, W, qx, qy);
    if (g < 0) g = -g;
    int v = P2 / (1 + g);
    return v > P1 ? v : P1;
}

/*
 * Eq. 3 (Section 3.2) along one direction r = (rx, ry), rx, ry in {-1, 0, 1}.
 * The predecessor of p = (x, y) is q = (x - rx, y - ry).  Pixels are visited
 * so that q is always finished before p.  L[y][x][d] (int32) receives L_r.
 * Ib = NULL: the constant P2 of Eq. 3; otherwise P2 at each step is
 * adaptive_p2 of the base image Ib.
 */
ORACLE_EXPORT void oracle_aggregate_ex(const uint8_t *MC, const uint8_t *Ib, int W, int H, int D, int P1, int P2,
                                       int rx, int ry, int32_t *L) {
    int y0 = (ry >= 0) ? 0 : H - 1, y1 = (ry >= 0) ? H : -1, sy = (ry >= 0) ? 1 : -1;
    int x0 = (rx >= 0) ? 0 : W - 1, x1 = (rx >= 0) ? W : -1, sx = (rx >= 0) ? 1 : -1;
    for (int y = y0; y != y1; y += sy) {
        for (int x = x0; x != x1; x += sx) {
            const uint8_t *mc = MC + ((size_t)y * W + x) * D;
            int32_t *out = L + ((size_t)y * W + x) * D;
            int qx = x - rx, qy = y - ry;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
                for (int d = 0; d < D; ++d) out[d] = mc[d];
                continue;
            }
            const int p2 = Ib ? adaptive_p2(Ib, W, x, y, qx, qy, P1, P2) : P2;
            const int32_t *prev = L + ((size_t)qy * W + qx) * D;
            int32_t mprev = prev[0];
            for (int k = 1; k < D; ++k)
                if (prev[k] < mprev) mprev = prev[k];
            for (int d = 0; d < D; ++d) {
                int32_t best = prev[d];
                if (d - 1 >= 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
                if (d + 1 < D && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
                if (mprev + p2 < best) best = mprev + p2;
                out[d] = (int32_t)mc[d] + best - mprev;
            }
        }
    }
}

/* Eq. 3 with the constant P2. */
ORACLE_EXPORT void oracle_aggregate(const uint8_t *MC, int W, int H, int D, int P1, int P2, int rx, int ry,
                                    int32_t *L) {
    oracle_aggregate_ex(MC, NULL, W, H, D, P1, P2, rx, ry, L);
}

/* The direction set for n_paths in {2, 4, 8}; returns the count, or 0. */
ORACLE_EXPORT int oracle_directions(int n_paths, int *rx, int *ry) {
    static const int dx[8] = {1, 0, -1, 0, 1, -1, 1, -1};
    static const int dy[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    if (n_paths != 2 && n_paths != 4 && n_paths != 8) return 0;
    for (int i = 0; i < n_paths; ++i) {
        rx[i] = dx[i];
        ry[i] = dy[i];
    }
    return n_paths;
}

/* Eq. 4 (Section 3.2): disparity = the lowest d minimising S(p, d). */
ORACLE_EXPORT void oracle_wta(const int32_t *S, int W, int H, int D, uint8_t *disp) {
    for (size_t p = 0; p < (size_t)W * H; ++p) {
        const int32_t *s = S + p * D;
        int best = 0;
        for (int d = 1; d < D; ++d)
            if (s[d] < s[best]) best = d;
        disp[p] = (uint8_t)best;
    }
}

/* 3x3 median of stage 4 (Section 2). */
ORACLE_EXPORT void oracle_median3x3(const uint8_t *in, int W, int H, uint8_t *out) {
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            if (x == 0 || y == 0 || x == W - 1 || y == H - 1) {
                out[p] = in[p];
                continue;
            }
            int v[9], n = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) v[n++] = in[(size_t)(y + j) * W + (x + i)];
            /* insertion sort */
            for (int a = 1; a < 9; ++a) {
                int t = v[a], b = a - 1;
                while (b >= 0 && v[b] > t) {
                    v[b + 1] = v[b];
                    --b;
                }
                v[b + 1] = t;
            }
            out[p] = (uint8_t)v[4];
        }
    }
}

/*
 * Stages 3-4 of Section 2 on a cost cube MC[y][x][d]: the aggregated paths
 * (Eq. 3), S, the winner-take-all disparity (Eq. 4) and the 3x3 median.
 * Optional debug outputs (NULL to skip): S (int32 [H][W][D]), raw disparity
 * (uint8 [H][W]).  Returns 0, or -2 if memory runs out.
 */
static int aggregate_and_select(const uint8_t *MC, int W, int H, int D, int P1, int P2, int npaths, const int *rx,
                                const int *ry, uint8_t *disp_out, uint8_t *raw_out, int32_t *S_out) {
    size_t n = (size_t)W * H;
    int32_t *L = (int32_t *)malloc(n * D * sizeof(int32_t));
    int32_t *S = (int32_t *)calloc(n * D, sizeof(int32_t));
    uint8_t *raw = (uint8_t *)malloc(n);
    int rc = 0;
    if (!L || !S || !raw) {
        rc = -2;
        goto done;
    }
    for (int r = 0; r < npaths; ++r) {
        oracle_aggregate(MC, W, H, D, P1, P2, rx[r], ry[r], L);
        for (size_t i = 0; i < n * D; ++i) S[i] += L[i];
    }
    oracle_wta(S, W, H, D, raw);
    if (W < 3 || H < 3)
        memcpy(disp_out, raw, n);
    else
        oracle_median3x3(raw, W, H, disp_out);
    if (raw_out) memcpy(raw_out, raw, n);
    if (S_out) memcpy(S_out, S, n * D * sizeof(int32_t));
done:
    free(L);
    free(S);
    free(raw);
    return rc;
}

/*
 * The whole path of Section 2, stages 2-4: features, matching cost, the
 * aggregated paths, S, the winner-take-all disparity and the 3x3 median.
 * Optional debug outputs (NULL to skip): Fb/Fm features (uint32 [H][W]),
 * S (int32 [H][W][D]), raw disparity (uint8 [H][W]).
 * Returns 0, or -1 on bad arguments, -2 if memory runs out.
 */
ORACLE_EXPORT int oracle_sgm(const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                             int n_paths, uint8_t *disp_out, uint8_t *raw_out, uint32_t *Fb_out, uint32_t *Fm_out,
                             int32_t *S_out) {
    int rx[8], ry[8];
    if (W < 1 || H < 1 || D < 1 || D > 256 || !left || !right || !disp_out) return -1;
    int npaths = oracle_directions(n_paths, rx, ry);
    if (npaths == 0) return -1;
    size_t n = (size_t)W * H;
    uint32_t *Fb = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *Fm = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint8_t *MC = (uint8_t *)malloc(n * D);
    int rc = -2;
    if (Fb && Fm && MC) {
        oracle_csct(left, W, H, Fb);
        oracle_csct(right, W, H, Fm);
        oracle_cost(Fb, Fm, W, H, D, MC);
        rc = aggregate_and_select(MC, W, H, D, P1, P2, npaths, rx, ry, disp_out, raw_out, S_out);
        if (Fb_out) memcpy(Fb_out, Fb, n * sizeof(uint32_t));
        if (Fm_out) memcpy(Fm_out, Fm, n * sizeof(uint32_t));
    }
    free(Fb);
    free(Fm);
    free(MC);
    return rc;
}

/* oracle_sgm with the full 9x7 Census (62-bit features, uint64 [H][W]). */
ORACLE_EXPORT int oracle_sgm_ct62(const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                                  int n_paths, uint8_t *disp_out, uint8_t *raw_out, uint64_t *Fb_out,
                                  uint64_t *Fm_out, int32_t *S_out) {
    int rx[8], ry[8];
    if (W < 1 || H < 1 || D < 1 || D > 256 || !left || !right || !disp_out) return -1;
    int npaths = oracle_directions(n_paths, rx, ry);
    if (npaths == 0) return -1;
    size_t n = (size_t)W * H;
    uint64_t *Fb = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *Fm = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint8_t *MC = (uint8_t *)malloc(n * D);
    int rc = -2;
    if (Fb && Fm && MC) {
        oracle_ct62(left, W, H, Fb);
        oracle_ct62(right, W, H, Fm);
        oracle_cost64(Fb, Fm, W, H, D, MC);
        rc = aggregate_and_select(MC, W, H, D, P1, P2, npaths, rx, ry, disp_out, raw_out, S_out);
        if (Fb_out) memcpy(Fb_out, Fb, n * sizeof(uint64_t));
        if (Fm_out) memcpy(Fm_out, Fm, n * sizeof(uint64_t));
    }
    free(Fb);
    free(Fm);
    free(MC);
    return rc;
}

/*
 * The same quantities at one pixel only, for checks on images too large for
 * oracle_sgm: S(p, .) at p = (px, py) (int32 [D]) and its raw disparity.
 * For each direction r, Eq. 3 is evaluated along the single path that ends
 * at p, starting from the first pixel of that path inside the image; the
 * costs along the path come from Eq. 1 and Eq. 2 evaluated at each pixel.
 * Returns the raw disparity, or -1 on bad arguments, -2 if memory runs out.
 */
ORACLE_EXPORT int oracle_pixel(const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                               int n_paths, int px, int py, int32_t *S_out) {
    int rx[8], ry[8];
    if (W < 1 || H < 1 || D < 1 || D > 256 || px < 0 || px >= W || py < 0 || py >= H) return -1;
    int npaths = oracle_directions(n_paths, rx, ry);
    if (npaths == 0) return -1;
    int32_t *S = (int32_t *)calloc((size_t)D, sizeof(int32_t));
    int32_t *Lprev = (int32_t *)malloc((size_t)D * sizeof(int32_t));
    int32_t *Lcur = (int32_t *)malloc((size_t)D * sizeof(int32_t));
    int result = -2;
    if (!S || !Lprev || !Lcur) goto done;
    for (int r = 0; r < npaths; ++r) {
        /* walk back from p to the first pixel of the path inside the image */
        int x = px, y = py, len = 1;
        while (x - rx[r] >= 0 && x - rx[r] < W && y - ry[r] >= 0 && y - ry[r] < H) {
            x -= rx[r];
            y -= ry[r];
            ++len;
        }
        for (int step = 0; step < len; ++step) {
            uint32_t fb = oracle_csct_at(left, W, H, x, y);
            int32_t mprev = 0;
            if (step > 0) {
                mprev = Lprev[0];
                for (int k = 1; k < D; ++k)
                    if (Lprev[k] < mprev) mprev = Lprev[k];
            }
            for (int d = 0; d < D; ++d) {
                uint32_t fm = (x - d >= 0) ? oracle_csct_at(right, W, H, x - d, y) : 0u;
                int mc = oracle_bitcount(fb ^ fm);
                if (step == 0) {
                    Lcur[d] = mc;
                } else {
                    int32_t best = Lprev[d];
                    if (d - 1 >= 0 && Lprev[d - 1] + P1 < best) best = Lprev[d - 1] + P1;
                    if (d + 1 < D && Lprev[d + 1] + P1 < best) best = Lprev[d + 1] + P1;
                    if (mprev + P2 < best) best = mprev + P2;
                    Lcur[d] = mc + best - mprev;
                }
            }
            int32_t *t = Lprev;
            Lprev = Lcur;
            Lcur = t;
            x += rx[r];
            y += ry[r];
        }
        for (int d = 0; d < D; ++d) S[d] += Lprev[d];
    }
    result = 0;
    for (int d = 1; d < D; ++d)
        if (S[d] < S[result]) result = d;
    if (S_out) memcpy(S_out, S, (size_t)D * sizeof(int32_t));
done:
    free(S);
    free(Lprev);
    free(Lcur);
    return result;
}

/* floor(n / d) for d > 0. */
static long floor_div(long n, long d) {
    long q = n / d;
    if (n % d != 0 && n < 0) q -= 1;
    return q;
}

/*
 * Sub-pixel disparity (announced in Section 5; reading): the vertex of the
 * parabola through (d-1, S(d-1)), (d, S(d)), (d+1, S(d+1)) at the winner d
 * of Eq. 4, in 1/16 pixel: 16 d + round(16 * (S(d-1) - S(d+1)) /
 * (2 (S(d-1) + S(d+1) - 2 S(d)))), halves rounded up, i.e.
 * 16 d + floor((16 num + den) / (2 den)).  At d = 0 and d = D-1 the value is
 * 16 d.  Because ties of Eq. 4 go to the lowest d, S(d-1) > S(d) and the
 * denominator is positive; the offset lies in [-8, 8].
 */
ORACLE_EXPORT int oracle_subpixel(const int32_t *S, int D, int d) {
    if (d <= 0 || d >= D - 1) return 16 * d;
    const long num = (long)S[d - 1] - S[d + 1];
    const long den = (long)S[d - 1] + S[d + 1] - 2L * S[d];
    return 16 * d + (int)floor_div(16 * num + den, 2 * den);
}

/* The 3x3 median of stage 4 on 16-bit values (same border reading). */
ORACLE_EXPORT void oracle_median3x3_u16(const uint16_t *in, int W, int H, uint16_t *out) {
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            if (x == 0 || y == 0 || x == W - 1 || y == H - 1) {
                out[p] = in[p];
                continue;
            }
            int v[9], n = 0;
            for (int j = -1; j <= 1; ++j)
                for (int i = -1; i <= 1; ++i) v[n++] = in[(size_t)(y + j) * W + (x + i)];
            for (int a = 1; a < 9; ++a) {
                int t = v[a], b = a - 1;
                while (b >= 0 && v[b] > t) {
                    v[b + 1] = v[b];
                    --b;
                }
                v[b + 1] = t;
            }
            out[p] = (uint16_t)v[4];
        }
    }
}

/*
 * One matching pass: features (CSCT of Eq. 1, or the full Census when
 * census_full), costs (Eq. 2), the aggregated paths (Eq. 3, adaptive P2 from
 * the base image when ap2), S and the winner-take-all disparity (Eq. 4).
 * S (int32 [H][W][D]) and raw (uint8 [H][W]) are outputs.  Returns 0 or -2.
 */
static int matching_pass(const uint8_t *base, const uint8_t *match, int W, int H, int D, int P1, int P2, int npaths,
                         const int *rx, const int *ry, int census_full, int ap2, int32_t *S, uint8_t *raw) {
    size_t n = (size_t)W * H;
    uint8_t *MC = (uint8_t *)malloc(n * D);
    int32_t *L = (int32_t *)malloc(n * D * sizeof(int32_t));
    void *Fb = malloc(n * 8), *Fm = malloc(n * 8);
    int rc = -2;
    if (MC && L && Fb && Fm) {
        if (census_full) {
            oracle_ct62(base, W, H, (uint64_t *)Fb);
            oracle_ct62(match, W, H, (uint64_t *)Fm);
            oracle_cost64((const uint64_t *)Fb, (const uint64_t *)Fm, W, H, D, MC);
        } else {
            oracle_csct(base, W, H, (uint32_t *)Fb);
            oracle_csct(match, W, H, (uint32_t *)Fm);
            oracle_cost((const uint32_t *)Fb, (const uint32_t *)Fm, W, H, D, MC);
        }
        memset(S, 0, n * D * sizeof(int32_t));
        for (int r = 0; r < npaths; ++r) {
            oracle_aggregate_ex(MC, ap2 ? base : NULL, W, H, D, P1, P2, rx[r], ry[r], L);
            for (size_t i = 0; i < n * D; ++i) S[i] += L[i];
        }
        oracle_wta(S, W, H, D, raw);
        rc = 0;
    }
    free(MC);
    free(L);
    free(Fb);
    free(Fm);
    return rc;
}

static void mirror_rows(const uint8_t *in, int W, int H, uint8_t *out) {
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) out[(size_t)y * W + x] = in[(size_t)y * W + (W - 1 - x)];
}

#define ORACLE_POST_SUBPIXEL 1u
#define ORACLE_POST_LR_CHECK 2u
#define ORACLE_POST_ADAPTIVE_P2 4u
#define ORACLE_DISP16_INVALID 0xFFFFu

/*
 * The path with the post-filters announced in Section 5, output in 1/16
 * pixel (uint16 [H][W]):
 *  1. the left pass (base = left, match = right) gives S and the
 *     winner-take-all disparity d_L (Eq. 4), with adaptive P2 when asked;
 *  2. v = oracle_subpixel(S, d_L) with SUBPIXEL, else 16 d_L;
 *  3. out = the 3x3 median of v (the border ring copied);
 *  4. with LR_CHECK (reading): the right image's disparity d_R is the same
 *     pass on the mirrored pair (base = mirrored right, match = mirrored
 *     left; adaptive P2 from its own base), mirrored back, so that right
 *     pixel x matches left pixel x + d_R(x); a left pixel x is consistent
 *     when x - d_L(x) >= 0 and |d_L(x) - d_R(x - d_L(x))| <= 1 (integer
 *     winner-take-all disparities of both passes); out = 0xFFFF elsewhere.
 * Without post-filters out = 16 * the output of oracle_sgm.  Optional debug
 * outputs: d_L and d_R (uint8 [H][W], original coordinates).
 * Returns 0, -1 on bad arguments, -2 if memory runs out.
 */
ORACLE_EXPORT int oracle_sgm_ex(const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                                int n_paths, int census_full, unsigned post, uint16_t *out16, uint8_t *dL_out,
                                uint8_t *dR_out) {
    int rx[8], ry[8];
    if (W < 1 || H < 1 || D < 1 || D > 256 || !left || !right || !out16) return -1;
    int npaths = oracle_directions(n_paths, rx, ry);
    if (npaths == 0) return -1;
    const int ap2 = (post & ORACLE_POST_ADAPTIVE_P2) != 0;
    size_t n = (size_t)W * H;
    int32_t *S = (int32_t *)malloc(n * D * sizeof(int32_t));
    uint8_t *dL = (uint8_t *)malloc(n), *dRm = (uint8_t *)malloc(n);
    uint8_t *mb = (uint8_t *)malloc(n), *mm = (uint8_t *)malloc(n);
    uint16_t *v = (uint16_t *)malloc(n * sizeof(uint16_t));
    int rc = -2;
    if (!S || !dL || !dRm || !mb || !mm || !v) goto done;
    if ((rc = matching_pass(left, right, W, H, D, P1, P2, npaths, rx, ry, census_full, ap2, S, dL)) != 0) goto done;
    for (size_t p = 0; p < n; ++p)
        v[p] = (uint16_t)((post & ORACLE_POST_SUBPIXEL) ? oracle_subpixel(S + p * D, D, dL[p]) : 16 * dL[p]);
    if (W < 3 || H < 3)
        memcpy(out16, v, n * sizeof(uint16_t));
    else
        oracle_median3x3_u16(v, W, H, out16);
    if (post & ORACLE_POST_LR_CHECK) {
        mirror_rows(right, W, H, mb);
        mirror_rows(left, W, H, mm);
        if ((rc = matching_pass(mb, mm, W, H, D, P1, P2, npaths, rx, ry, census_full, ap2, S, dRm)) != 0) goto done;
        for (int y = 0; y < H; ++y) {
            for (int x = 0; x < W; ++x) {
                const int d = dL[(size_t)y * W + x], xr = x - d;
                int ok = xr >= 0;
                if (ok) {
                    const int dr = dRm[(size_t)y * W + (W - 1 - xr)];
                    ok = (d - dr <= 1) && (dr - d <= 1);
                }
                if (!ok) out16[(size_t)y * W + x] = (uint16_t)ORACLE_DISP16_INVALID;
            }
        }
        if (dR_out) mirror_rows(dRm, W, H, dR_out);
    } else if (dR_out) {
        memset(dR_out, 0, n);
    }
    if (dL_out) memcpy(dL_out, dL, n);
done:
    free(S);
    free(dL);
    free(dRm);
    free(mb);
    free(mm);
    free(v);
    return rc;
}

/*
 * The same computation as oracle_sgm (CSCT features), with its independent
 * parts spread over `nthreads` POSIX threads.  It exists to time the CPU
 * baseline on every host core; the parity reference stays oracle_sgm, and a
 * test checks that both give identical disparities.  The work splits along
 * what the definitions leave independent: rows of the Census (Eq. 1), of the
 * matching cost (Eq. 2), of the sum and the winner-take-all (Eq. 4) and of the
 * median; and, for Eq. 3, whole directions, each one's rows (horizontal
 * paths, whose predecessors lie in the same row) or columns (vertical paths)
 * in bands.  Diagonal directions run whole on one thread each.
 */
#include <pthread.h>

typedef struct {
    int kind; /* 0 census rows, 1 cost rows, 2 aggregation band, 3 sum and WTA rows, 4 median rows */
    int a0, a1; /* rows (kinds 0, 1, 3, 4) or the band's rows / columns (kind 2) */
    int img, r; /* census: 0 left, 1 right; aggregation: direction index */
} oracle_task;

typedef struct {
    const uint8_t *left, *right;
    int W, H, D, P1, P2, npaths, rx[8], ry[8];
    uint32_t *Fb, *Fm;
    uint8_t *MC, *raw, *disp;
    int32_t *L; /* npaths cubes */
    oracle_task *tasks;
    int ntasks;
    int next; /* next task, taken under the lock */
    pthread_mutex_t lock;
} oracle_job;

/* Eq. 3 for direction r over the pixels x in [x0, x1), y in [y0, y1) of a band
 * that holds every predecessor of its pixels; the loop is oracle_aggregate_ex's. */
static void aggregate_band(const oracle_job *J, int r, int x0b, int x1b, int y0b, int y1b) {
    const int W = J->W, H = J->H, D = J->D, rx = J->rx[r], ry = J->ry[r];
    int32_t *L = J->L + (size_t)r * W * H * D;
    int y0 = (ry >= 0) ? y0b : y1b - 1, y1 = (ry >= 0) ? y1b : y0b - 1, sy = (ry >= 0) ? 1 : -1;
    int x0 = (rx >= 0) ? x0b : x1b - 1, x1 = (rx >= 0) ? x1b : x0b - 1, sx = (rx >= 0) ? 1 : -1;
    for (int y = y0; y != y1; y += sy) {
        for (int x = x0; x != x1; x += sx) {
            const uint8_t *mc = J->MC + ((size_t)y * W + x) * D;
            int32_t *out = L + ((size_t)y * W + x) * D;
            int qx = x - rx, qy = y - ry;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
                for (int d = 0; d < D; ++d) out[d] = mc[d];
                continue;
            }
            const int32_t *prev = L + ((size_t)qy * W + qx) * D;
            int32_t mprev = prev[0];
            for (int k = 1; k < D; ++k)
                if (prev[k] < mprev) mprev = prev[k];
            for (int d = 0; d < D; ++d) {
                int32_t best = prev[d];
                if (d - 1 >= 0 && prev[d - 1] + J->P1 < best) best = prev[d - 1] + J->P1;
                if (d + 1 < D && prev[d + 1] + J->P1 < best) best = prev[d + 1] + J->P1;
                if (mprev + J->P2 < best) best = mprev + J->P2;
                out[d] = (int32_t)mc[d] + best - mprev;
            }
        }
    }
}

static void run_task(oracle_job *J, const oracle_task *t) {
    const int W = J->W, H = J->H, D = J->D;
    if (t->kind == 0) {
        const uint8_t *I = t->img ? J->right : J->left;
        uint32_t *F = t->img ? J->Fm : J->Fb;
        for (int y = t->a0; y < t->a1; ++y)
            for (int x = 0; x < W; ++x) F[(size_t)y * W + x] = oracle_csct_at(I, W, H, x, y);
    } else if (t->kind == 1) {
        for (int y = t->a0; y < t->a1; ++y)
            for (int x = 0; x < W; ++x)
                for (int d = 0; d < D; ++d) {
                    uint32_t v = J->Fb[(size_t)y * W + x] ^ match_feature(J->Fm, W, x - d, y);
                    J->MC[((size_t)y * W + x) * D + d] = (uint8_t)oracle_bitcount(v);
                }
    } else if (t->kind == 2) {
        const int r = t->r;
        if (J->ry[r] == 0)
            aggregate_band(J, r, 0, W, t->a0, t->a1); /* horizontal: rows */
        else if (J->rx[r] == 0)
            aggregate_band(J, r, t->a0, t->a1, 0, H); /* vertical: columns */
        else
            aggregate_band(J, r, 0, W, 0, H); /* diagonal: whole */
    } else if (t->kind == 3) {
        for (size_t p = (size_t)t->a0 * W; p < (size_t)t->a1 * W; ++p) {
            int best = 0;
            int32_t sbest = 0;
            for (int d = 0; d < D; ++d) {
                int32_t s = 0;
                for (int r = 0; r < J->npaths; ++r) s += J->L[((size_t)r * W * H + p) * D + d];
                if (d == 0 || s < sbest) {
                    sbest = s;
                    best = d;
                }
            }
            J->raw[p] = (uint8_t)best;
        }
    } else {
        for (int y = t->a0; y < t->a1; ++y) {
            for (int x = 0; x < W; ++x) {
                size_t p = (size_t)y * W + x;
                if (W < 3 || H < 3 || x == 0 || y == 0 || x == W - 1 || y == H - 1) {
                    J->disp[p] = J->raw[p];
                    continue;
                }
                int v[9], n = 0;
                for (int j = -1; j <= 1; ++j)
                    for (int i = -1; i <= 1; ++i) v[n++] = J->raw[(size_t)(y + j) * W + (x + i)];
                for (int a = 1; a < 9; ++a) {
                    int tv = v[a], b = a - 1;
                    while (b >= 0 && v[b] > tv) {
                        v[b + 1] = v[b];
                        --b;
                    }
                    v[b + 1] = tv;
                }
                J->disp[p] = (uint8_t)v[4];
            }
        }
    }
}

static void *worker(void *arg) {
    oracle_job *J = (oracle_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int i = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (i >= J->ntasks) return NULL;
        run_task(J, &J->tasks[i]);
    }
}

/* Runs J->tasks on nthreads threads (the calling thread included) and waits. */
static void run_phase(oracle_job *J, int nthreads) {
    pthread_t th[256];
    int started = 0;
    J->next = 0;
    for (int i = 1; i < nthreads && i < 256; ++i)
        if (pthread_create(&th[started], NULL, worker, J) == 0) ++started;
    worker(J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
}

/* Tasks of rows [0, n) in bands of about n / (4 nthreads) rows. */
static int add_bands(oracle_task *t, int k, int kind, int n, int nthreads, int img, int r) {
    int bands = 4 * nthreads;
    if (bands > n) bands = n;
    for (int b = 0; b < bands; ++b) {
        t[k].kind = kind;
        t[k].a0 = (int)((long)n * b / bands);
        t[k].a1 = (int)((long)n * (b + 1) / bands);
        t[k].img = img;
        t[k].r = r;
        ++k;
    }
    return k;
}

ORACLE_EXPORT int oracle_sgm_threads(const uint8_t *left, const uint8_t *right, int W, int H, int D, int P1, int P2,
                                     int n_paths, uint8_t *disp_out, int nthreads) {
    oracle_job J;
    memset(&J, 0, sizeof J);
    if (W < 1 || H < 1 || D < 1 || D > 256 || !left || !right || !disp_out) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    J.npaths = oracle_directions(n_paths, J.rx, J.ry);
    if (J.npaths == 0) return -1;
    J.left = left;
    J.right = right;
    J.W = W;
    J.H = H;
    J.D = D;
    J.P1 = P1;
    J.P2 = P2;
    J.disp = disp_out;
    size_t n = (size_t)W * H;
    J.Fb = (uint32_t *)malloc(n * sizeof(uint32_t));
    J.Fm = (uint32_t *)malloc(n * sizeof(uint32_t));
    J.MC = (uint8_t *)malloc(n * D);
    J.raw = (uint8_t *)malloc(n);
    J.L = (int32_t *)malloc((size_t)J.npaths * n * D * sizeof(int32_t));
    int maxt = 8 * nthreads * (J.npaths + 2) + 16;
    J.tasks = (oracle_task *)malloc((size_t)maxt * sizeof(oracle_task));
    int rc = -2;
    if (J.Fb && J.Fm && J.MC && J.raw && J.L && J.tasks) {
        pthread_mutex_init(&J.lock, NULL);
        int k = add_bands(J.tasks, 0, 0, H, nthreads, 0, 0);
        J.ntasks = add_bands(J.tasks, k, 0, H, nthreads, 1, 0);
        run_phase(&J, nthreads);
        J.ntasks = add_bands(J.tasks, 0, 1, H, nthreads, 0, 0);
        run_phase(&J, nthreads);
        k = 0;
        for (int r = 0; r < J.npaths; ++r) {
            if (J.ry[r] == 0)
                k = add_bands(J.tasks, k, 2, H, nthreads, 0, r);
            else if (J.rx[r] == 0)
                k = add_bands(J.tasks, k, 2, W, nthreads, 0, r);
            else
                k = add_bands(J.tasks, k, 2, 1, nthreads, 0, r);
        }
        J.ntasks = k;
        run_phase(&J, nthreads);
        J.ntasks = add_bands(J.tasks, 0, 3, H, nthreads, 0, 0);
        run_phase(&J, nthreads);
        J.ntasks = add_bands(J.tasks, 0, 4, H, nthreads, 0, 0);
        run_phase(&J, nthreads);
        pthread_mutex_destroy(&J.lock);
        rc = 0;
    }
    free(J.Fb);
    free(J.Fm);
    free(J.MC);
    free(J.raw);
    free(J.L);
    free(J.tasks);
    return rc;
}
