/*
 * Plain CPU oracle for Oriented FAST over an image pyramid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant generator
 * with the CUDA library: every definition below is written out again from the
 * paper (arXiv 2506.07164) and from the readings listed in the design notes.
 *
 * Style: single-threaded, plain loops over pixels, no SIMD, no blocking, no
 * fusion.  Integer work is done in int32/int64 exactly; the few floating
 * point steps are float64 and must be compiled with -ffp-contract=off so that
 * no multiply-add is fused.
 *
 * Contents (each function names the passage it follows):
 *   ora_level_sizes   pyramid level sizes            (Sec. 1, Sec. 6.1: "decrease exponentially")
 *   ora_resize        bilinear level-to-level resize (pyramid, Sec. 1)
 *   ora_ring_masks    bright / dark flags            (Eq. 1, Fig. 3)
 *   ora_has_arc9      nine contiguous flags, cyclic  (Sec. 3.1, Alg. 2 with wraparound)
 *   ora_is_corner     FAST segment test at t         (Eq. 1 + Sec. 3.1)
 *   ora_fast_score    largest t at which the test passes
 *   ora_score_map     score map over the detect region
 *   ora_cell_thresh   per-cell threshold (t_hi, fallback t_lo)
 *   ora_nms           strict 3x3 non-maximum suppression (Fig. 1 "NMS")
 *   ora_harris_sums   Sobel gradients + 7x7 window sums (Eqs. 2-4, Alg. 3)
 *   ora_harris_key    exact ranking key det(M) - k trace(M)^2 (Eq. 3)
 *   ora_level_quotas  features per level
 *   ora_orient        intensity-centroid orientation (Fig. 1 "Centroid")
 *   ora_detect        the whole chain for one frame
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Fig. 2(a): the 16 pixels of the radius-3 Bresenham circle around I_p, in
 * cyclic (clockwise from the top) order; (dx, dy) with y pointing down. */
static const int ORA_RING[16][2] = {
    {0, -3}, {1, -3}, {2, -2}, {3, -1}, {3, 0}, {3, 1}, {2, 2}, {1, 3},
    {0, 3}, {-1, 3}, {-2, 2}, {-3, 1}, {-3, 0}, {-3, -1}, {-2, -2}, {-1, -3}};

#define ORA_ARC 9 /* "9 (or more) continuous surrounding pixels", Sec. 3.1 */

/* ------------------------------------------------------------------ pyramid */

/* Level sizes.  Level l has scale s_l = scale^l (s_0 = 1, each a float64
 * product of the previous one and the float scale); w_l = floor(W / s_l + 0.5),
 * h_l likewise.  Writes s_l too when `level_scale` is not NULL. */
void ora_level_sizes(int W, int H, int levels, float scale, int* ws, int* hs,
                     double* level_scale) {
    double s = 1.0;
    for (int l = 0; l < levels; ++l) {
        if (l == 0) {
            ws[l] = W;
            hs[l] = H;
        } else {
            double fw = floor((double)W / s + 0.5);
            double fh = floor((double)H / s + 0.5);
            ws[l] = (int)fw;
            hs[l] = (int)fh;
        }
        if (level_scale) level_scale[l] = s;
        s = s * (double)scale;
    }
}

/* Source coordinate of destination index `d` along one axis, for a bilinear
 * resize from n_src to n_dst samples with pixel centres aligned:
 *   s = (d + 0.5) * (n_src / n_dst) - 0.5, clamped to [0, n_src - 1];
 *   i0 = floor(s), i1 = min(i0 + 1, n_src - 1), a = lrint((s - i0) * 2048). */
static void ora_src_coord(int d, int n_src, int n_dst, int* i0, int* i1, int* a) {
    double ratio = (double)n_src / (double)n_dst;
    double s = ((double)d + 0.5) * ratio - 0.5;
    if (s < 0.0) s = 0.0;
    if (s > (double)(n_src - 1)) s = (double)(n_src - 1);
    double f = floor(s);
    *i0 = (int)f;
    *i1 = (*i0 + 1 < n_src) ? *i0 + 1 : n_src - 1;
    *a = (int)lrint((s - f) * 2048.0);
}

/* Bilinear resize of level l-1 (src) to level l (dst), weights in units of
 * 1/2048 and one rounding at the end:
 *   out = ((2048-ay)((2048-ax) p00 + ax p01) + ay((2048-ax) p10 + ax p11) + 2^21) >> 22 */
void ora_resize(const uint8_t* src, int sw, int sh, int spitch, uint8_t* dst, int dw,
                int dh, int dpitch) {
    for (int y = 0; y < dh; ++y) {
        int y0, y1, ay;
        ora_src_coord(y, sh, dh, &y0, &y1, &ay);
        for (int x = 0; x < dw; ++x) {
            int x0, x1, ax;
            ora_src_coord(x, sw, dw, &x0, &x1, &ax);
            int32_t p00 = src[(int64_t)y0 * spitch + x0];
            int32_t p01 = src[(int64_t)y0 * spitch + x1];
            int32_t p10 = src[(int64_t)y1 * spitch + x0];
            int32_t p11 = src[(int64_t)y1 * spitch + x1];
            int32_t top = (2048 - ax) * p00 + ax * p01;
            int32_t bot = (2048 - ax) * p10 + ax * p11;
            int32_t v = ((2048 - ay) * top + ay * bot + (1 << 21)) >> 22;
            dst[(int64_t)y * dpitch + x] = (uint8_t)v;
        }
    }
}

/* --------------------------------------------------------------------- FAST */

/* Eq. 1: ring pixel i is bright when I_i >= I_p + t and dark when
 * I_i <= I_p - t.  Bit i (i = 0..15, ring order) of *bright / *dark is set
 * accordingly (Fig. 3 keeps the two groups in the two halves of one word). */
void ora_ring_masks(const int ring[16], int center, int t, uint32_t* bright,
                    uint32_t* dark) {
    uint32_t b = 0, d = 0;
    for (int i = 0; i < 16; ++i) {
        if (ring[i] >= center + t) b |= 1u << i;
        if (ring[i] <= center - t) d |= 1u << i;
    }
    *bright = b;
    *dark = d;
}

/* Sec. 3.1 / Alg. 2: is there a run of at least 9 set bits in the 16-bit
 * mask, read cyclically (the run may wrap from bit 15 to bit 0)?  Alg. 2
 * appends 8 bits to make the wrap visible and checks 16 windows of 9 bits;
 * this does the same by indexing modulo 16. */
int ora_has_arc9(uint32_t mask16) {
    for (int start = 0; start < 16; ++start) {
        int all = 1;
        for (int k = 0; k < ORA_ARC; ++k) {
            if (!((mask16 >> ((start + k) % 16)) & 1u)) {
                all = 0;
                break;
            }
        }
        if (all) return 1;
    }
    return 0;
}

/* The FAST segment test at threshold t (Eq. 1 and Sec. 3.1). */
int ora_is_corner(const int ring[16], int center, int t) {
    uint32_t b, d;
    ora_ring_masks(ring, center, t, &b, &d);
    return ora_has_arc9(b) || ora_has_arc9(d);
}

/* Score: the largest threshold at which the segment test still passes,
 *   s = max over start j and sign sg of  min over k=0..8 of  sg * (I_{j+k} - I_p).
 * For every t >= 1, ora_is_corner(t) <=> s >= t.  May be <= 0 (no corner). */
int ora_fast_score(const int ring[16], int center) {
    int best = -1000;
    for (int sg = -1; sg <= 1; sg += 2) {
        for (int j = 0; j < 16; ++j) {
            int m = 1000;
            for (int k = 0; k < ORA_ARC; ++k) {
                int d = sg * (ring[(j + k) % 16] - center);
                if (d < m) m = d;
            }
            if (m > best) best = m;
        }
    }
    return best;
}

static void ora_gather_ring(const uint8_t* img, int pitch, int x, int y, int ring[16]) {
    for (int i = 0; i < 16; ++i)
        ring[i] = img[(int64_t)(y + ORA_RING[i][1]) * pitch + (x + ORA_RING[i][0])];
}

/* Score map of one level: out[y*w + x] = max(s(p), 0) for p in the detect
 * region R = [border, w-border) x [border, h-border), 0 elsewhere.  Requires
 * border >= 3 so the ring stays inside the image. */
void ora_score_map(const uint8_t* img, int w, int h, int pitch, int border, uint8_t* out) {
    memset(out, 0, (size_t)w * (size_t)h);
    for (int y = border; y < h - border; ++y) {
        for (int x = border; x < w - border; ++x) {
            int ring[16];
            ora_gather_ring(img, pitch, x, y, ring);
            int s = ora_fast_score(ring, img[(int64_t)y * pitch + x]);
            out[(int64_t)y * w + x] = (uint8_t)(s > 0 ? s : 0);
        }
    }
}

/* Per-cell threshold.  Cells are cell x cell squares anchored at (border,
 * border) covering R (the last row / column of cells may be partial).  A cell
 * takes t_hi when some pixel in it scores >= t_hi, else t_lo.  Output is
 * ncx * ncy bytes, ncx = ceil((w - 2 border) / cell). */
void ora_cell_thresh(const uint8_t* score, int w, int h, int border, int cell, int t_hi,
                     int t_lo, uint8_t* T) {
    int rw = w - 2 * border, rh = h - 2 * border;
    if (rw <= 0 || rh <= 0) return;
    int ncx = (rw + cell - 1) / cell, ncy = (rh + cell - 1) / cell;
    for (int cy = 0; cy < ncy; ++cy) {
        for (int cx = 0; cx < ncx; ++cx) {
            int strong = 0;
            for (int y = border + cy * cell; y < border + (cy + 1) * cell && y < h - border; ++y)
                for (int x = border + cx * cell; x < border + (cx + 1) * cell && x < w - border; ++x)
                    if (score[(int64_t)y * w + x] >= t_hi) strong = 1;
            T[cy * ncx + cx] = (uint8_t)(strong ? t_hi : t_lo);
        }
    }
}

/* Strict 3x3 non-maximum suppression.  S(p) = s(p) when p is a candidate
 * (s(p) >= T of its cell), else 0; pixels outside R count as 0.  p survives
 * when S(p) > 0 and S(p) > S(q) for each of its 8 neighbours q.  Survivors
 * are written in raster order as x, y pairs; returns how many. */
int ora_nms(const uint8_t* score, int w, int h, int border, int cell, const uint8_t* T,
            int32_t* out_xy, int cap) {
    int rw = w - 2 * border, rh = h - 2 * border;
    if (rw <= 0 || rh <= 0) return 0;
    int ncx = (rw + cell - 1) / cell;
    int n = 0;
    for (int y = border; y < h - border; ++y) {
        for (int x = border; x < w - border; ++x) {
            int S[3][3];
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = x + dx, qy = y + dy, v = 0;
                    if (qx >= border && qx < w - border && qy >= border && qy < h - border) {
                        int s = score[(int64_t)qy * w + qx];
                        int t = T[((qy - border) / cell) * ncx + (qx - border) / cell];
                        v = (s >= t) ? s : 0;
                    }
                    S[dy + 1][dx + 1] = v;
                }
            }
            int c = S[1][1], keep = c > 0;
            for (int dy = 0; dy < 3; ++dy)
                for (int dx = 0; dx < 3; ++dx)
                    if (!(dy == 1 && dx == 1) && !(c > S[dy][dx])) keep = 0;
            if (keep) {
                if (n < cap) {
                    out_xy[2 * n] = x;
                    out_xy[2 * n + 1] = y;
                }
                ++n;
            }
        }
    }
    return n;
}

/* ------------------------------------------------------------------- Harris */

/* Eqs. 2-4: gradients by the 3x3 Sobel operator written out in 2-D,
 *   gx(x,y) = sum_{dy=-1..1} w(dy) * (I(x+1, y+dy) - I(x-1, y+dy)),
 *   gy(x,y) = sum_{dx=-1..1} w(dx) * (I(x+dx, y+1) - I(x+dx, y-1)),
 * w = (1, 2, 1); then the second-moment sums over the block x block window
 * centred on (x, y):  A = sum gx^2, B = sum gy^2, C = sum gx gy  (exact int32). */
void ora_harris_sums(const uint8_t* img, int pitch, int x, int y, int block, int32_t* A,
                     int32_t* B, int32_t* C) {
    static const int wgt[3] = {1, 2, 1};
    int r = block / 2;
    int32_t a = 0, b = 0, c = 0;
    for (int v = -r; v <= r; ++v) {
        for (int u = -r; u <= r; ++u) {
            int px = x + u, py = y + v;
            int gx = 0, gy = 0;
            for (int k = -1; k <= 1; ++k) {
                gx += wgt[k + 1] * ((int)img[(int64_t)(py + k) * pitch + px + 1] -
                                    (int)img[(int64_t)(py + k) * pitch + px - 1]);
                gy += wgt[k + 1] * ((int)img[(int64_t)(py + 1) * pitch + px + k] -
                                    (int)img[(int64_t)(py - 1) * pitch + px + k]);
            }
            a += gx * gx;
            b += gy * gy;
            c += gx * gy;
        }
    }
    *A = a;
    *B = b;
    *C = c;
}

static int64_t ora_gcd(int64_t a, int64_t b) {
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* k as an exact fraction num/den: k is rounded to a multiple of 1e-6 and the
 * fraction reduced (0.04 -> 1/25).  Returns 0 on success, -1 when k is outside
 * [0, 0.25] or den > 3000 (the key would not fit int64). */
int ora_k_fraction(float k, int64_t* num, int64_t* den) {
    double kd = (double)k;
    if (!(kd >= 0.0 && kd <= 0.25)) return -1;
    int64_t kq = (int64_t)llrint(kd * 1e6);
    int64_t g = ora_gcd(kq, 1000000);
    if (g == 0) g = 1000000;
    *num = kq / g;
    *den = 1000000 / g;
    return (*den > 3000) ? -1 : 0;
}

/* Eq. 3 as an exact integer: R = det(M) - k trace(M)^2 with det = AB - C^2,
 * trace = A + B and k = num/den, scaled by den so that it is an integer:
 *   key = den * (A*B - C*C) - num * (A+B)^2. */
int64_t ora_harris_key(int32_t A, int32_t B, int32_t C, int64_t num, int64_t den) {
    int64_t det = (int64_t)A * (int64_t)B - (int64_t)C * (int64_t)C;
    int64_t tr = (int64_t)A + (int64_t)B;
    return den * det - num * tr * tr;
}

/* Reported response: the Harris score key/den times the gradient
 * normalisation factor (1 / (4 * block * 255))^4 (Alg. 3 multiplies its score
 * by a positive constant it calls factor). */
double ora_harris_response(int64_t key, int64_t den, int block) {
    double f = 1.0 / (4.0 * (double)block * 255.0);
    return ((double)key / (double)den) * (f * f * f * f);
}

/* -------------------------------------------------------------- orientation */

/* Intensity centroid over the disc u^2 + v^2 <= radius^2 around (x, y):
 *   m10 = sum u I(x+u, y+v),  m01 = sum v I(x+u, y+v)  (v points down),
 *   theta = atan2(m01, m10) in float64, atan2(0, 0) = 0. */
void ora_orient(const uint8_t* img, int pitch, int x, int y, int radius, int32_t* m10,
                int32_t* m01, double* theta) {
    int32_t a = 0, b = 0;
    for (int v = -radius; v <= radius; ++v) {
        for (int u = -radius; u <= radius; ++u) {
            if (u * u + v * v > radius * radius) continue;
            int I = img[(int64_t)(y + v) * pitch + (x + u)];
            a += u * I;
            b += v * I;
        }
    }
    *m10 = a;
    *m01 = b;
    *theta = (a == 0 && b == 0) ? 0.0 : atan2((double)b, (double)a);
}

/* ------------------------------------------------------------------ quotas */

/* Features per level, proportional to level area (ratio f = 1/scale^2):
 *   n_l = min(round(N (1-f)/(1-f^L) f^l), N - sum_{j<l} n_j) for l < L-1,
 *   n_{L-1} = N - sum_{j<L-1} n_j;   round = floor(x + 0.5);
 * f^l and f^L are repeated float64 products. */
void ora_level_quotas(int N, int L, float scale, int* n) {
    double s = (double)scale;
    double f = 1.0 / (s * s);
    double fL = 1.0;
    for (int l = 0; l < L; ++l) fL = fL * f;
    double c = (1.0 - f) / (1.0 - fL);
    int used = 0;
    double fl = 1.0;
    for (int l = 0; l < L; ++l) {
        if (l == L - 1) {
            n[l] = N - used;
        } else {
            double q = (double)N * c * fl;
            int r = (int)floor(q + 0.5);
            if (r > N - used) r = N - used;
            n[l] = r;
        }
        used += n[l];
        fl = fl * f;
    }
}

/* ----------------------------------------------------------------- top-N */

typedef struct {
    int64_t key;
    int32_t x, y;
} ora_cand;

/* Rank order: key descending, then y ascending, then x ascending. */
static int ora_cand_cmp(const void* pa, const void* pb) {
    const ora_cand* a = (const ora_cand*)pa;
    const ora_cand* b = (const ora_cand*)pb;
    if (a->key != b->key) return (a->key > b->key) ? -1 : 1;
    if (a->y != b->y) return (a->y < b->y) ? -1 : 1;
    if (a->x != b->x) return (a->x < b->x) ? -1 : 1;
    return 0;
}

/* Sort (key, x, y) triples into rank order in place (full sort). */
void ora_rank_sort(int64_t* key, int32_t* x, int32_t* y, int n) {
    ora_cand* c = (ora_cand*)malloc(sizeof(ora_cand) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        c[i].key = key[i];
        c[i].x = x[i];
        c[i].y = y[i];
    }
    qsort(c, (size_t)n, sizeof(ora_cand), ora_cand_cmp);
    for (int i = 0; i < n; ++i) {
        key[i] = c[i].key;
        x[i] = c[i].x;
        y[i] = c[i].y;
    }
    free(c);
}

/* --------------------------------------------------------------- pipeline */

/* One keypoint as the oracle reports it. */
typedef struct {
    double x, y;        /* level-0 coordinates: (x_l, y_l) * s_l */
    int32_t x_l, y_l, level;
    int32_t fast_score; /* s(p) */
    int64_t key;        /* exact Harris key (see ora_harris_key) */
    double response;    /* ora_harris_response(key) */
    double angle;       /* ora_orient theta */
    int32_t A, B, C;
    int32_t m10, m01;
} ora_keypoint;

typedef struct {
    int border, cell, block, radius;
    int t_hi, t_lo; /* t_lo == t_hi: a plain threshold */
} ora_config;

/* Whole chain for one frame (level-major, rank order within each level).
 * Returns the number of keypoints written, or -1 on bad arguments.
 * `level_counts` (optional, `levels` ints) receives the survivors of NMS per level. */
int ora_detect(const uint8_t* img, int W, int H, int pitch, int levels, float scale,
               const ora_config* cfg, float harris_k, int n_features, ora_keypoint* out,
               int cap, int* level_counts) {
    if (!img || W <= 0 || H <= 0 || pitch < W || levels < 1 || !(scale > 1.0f) || !cfg)
        return -1;
    int64_t knum, kden;
    if (ora_k_fraction(harris_k, &knum, &kden) != 0) return -1;

    int* ws = (int*)malloc(sizeof(int) * (size_t)levels);
    int* hs = (int*)malloc(sizeof(int) * (size_t)levels);
    double* sl = (double*)malloc(sizeof(double) * (size_t)levels);
    int* quota = (int*)malloc(sizeof(int) * (size_t)levels);
    ora_level_sizes(W, H, levels, scale, ws, hs, sl);
    ora_level_quotas(n_features, levels, scale, quota);

    /* The pyramid: level 0 is the input, level l is resized from level l-1. */
    uint8_t** lev = (uint8_t**)calloc((size_t)levels, sizeof(uint8_t*));
    int* lp = (int*)malloc(sizeof(int) * (size_t)levels);
    lev[0] = (uint8_t*)img;
    lp[0] = pitch;
    int nlev = levels;
    for (int l = 1; l < levels; ++l) {
        if (ws[l] < 1 || hs[l] < 1) {
            nlev = l;
            break;
        }
        lev[l] = (uint8_t*)malloc((size_t)ws[l] * (size_t)hs[l]);
        lp[l] = ws[l];
        ora_resize(lev[l - 1], ws[l - 1], hs[l - 1], lp[l - 1], lev[l], ws[l], hs[l], lp[l]);
    }

    int total = 0;
    for (int l = 0; l < levels; ++l) {
        if (level_counts) level_counts[l] = 0;
        if (l >= nlev) continue;
        int w = ws[l], h = hs[l];
        if (w - 2 * cfg->border <= 0 || h - 2 * cfg->border <= 0) continue;
        uint8_t* score = (uint8_t*)malloc((size_t)w * (size_t)h);
        ora_score_map(lev[l], w, h, lp[l], cfg->border, score);
        int ncx = (w - 2 * cfg->border + cfg->cell - 1) / cfg->cell;
        int ncy = (h - 2 * cfg->border + cfg->cell - 1) / cfg->cell;
        uint8_t* T = (uint8_t*)malloc((size_t)ncx * (size_t)ncy);
        ora_cell_thresh(score, w, h, cfg->border, cfg->cell, cfg->t_hi, cfg->t_lo, T);
        int cap_c = w * h;
        int32_t* xy = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)cap_c);
        int nc = ora_nms(score, w, h, cfg->border, cfg->cell, T, xy, cap_c);
        if (level_counts) level_counts[l] = nc;

        int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
        int32_t* cx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
        int32_t* cy = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc > 0 ? nc : 1));
        for (int i = 0; i < nc; ++i) {
            int32_t A, B, C;
            cx[i] = xy[2 * i];
            cy[i] = xy[2 * i + 1];
            ora_harris_sums(lev[l], lp[l], cx[i], cy[i], cfg->block, &A, &B, &C);
            key[i] = ora_harris_key(A, B, C, knum, kden);
        }
        ora_rank_sort(key, cx, cy, nc);
        int keep = nc < quota[l] ? nc : quota[l];
        for (int i = 0; i < keep && total < cap; ++i) {
            ora_keypoint* kp = &out[total++];
            kp->x_l = cx[i];
            kp->y_l = cy[i];
            kp->level = l;
            kp->x = (double)cx[i] * sl[l];
            kp->y = (double)cy[i] * sl[l];
            kp->fast_score = score[(int64_t)cy[i] * w + cx[i]];
            ora_harris_sums(lev[l], lp[l], cx[i], cy[i], cfg->block, &kp->A, &kp->B, &kp->C);
            kp->key = key[i];
            kp->response = ora_harris_response(key[i], kden, cfg->block);
            ora_orient(lev[l], lp[l], cx[i], cy[i], cfg->radius, &kp->m10, &kp->m01, &kp->angle);
        }
        free(key);
        free(cx);
        free(cy);
        free(xy);
        free(T);
        free(score);
    }
    for (int l = 1; l < levels; ++l) free(lev[l]);
    free(lev);
    free(lp);
    free(ws);
    free(hs);
    free(sl);
    free(quota);
    return total;
}

/* Per-level intermediate results for parity checks: the pyramid level image
 * (w*h bytes, pitch w) and its score map.  Returns 0, or -1 when the level is empty. */
int ora_pyramid_level(const uint8_t* img, int W, int H, int pitch, int levels, float scale,
                      int level, uint8_t* out, int* out_w, int* out_h) {
    int* ws = (int*)malloc(sizeof(int) * (size_t)levels);
    int* hs = (int*)malloc(sizeof(int) * (size_t)levels);
    ora_level_sizes(W, H, levels, scale, ws, hs, NULL);
    *out_w = ws[level];
    *out_h = hs[level];
    int ok = 0;
    for (int l = 0; l <= level; ++l)
        if (ws[l] < 1 || hs[l] < 1) ok = -1;
    if (ok == 0) {
        uint8_t* cur = (uint8_t*)malloc((size_t)W * (size_t)H);
        for (int y = 0; y < H; ++y) memcpy(cur + (size_t)y * W, img + (size_t)y * pitch, (size_t)W);
        for (int l = 1; l <= level; ++l) {
            uint8_t* nxt = (uint8_t*)malloc((size_t)ws[l] * (size_t)hs[l]);
            ora_resize(cur, ws[l - 1], hs[l - 1], ws[l - 1], nxt, ws[l], hs[l], ws[l]);
            free(cur);
            cur = nxt;
        }
        memcpy(out, cur, (size_t)ws[level] * (size_t)hs[level]);
        free(cur);
    }
    free(ws);
    free(hs);
    return ok;
}
