/*
 * CPU ORACLE of the iterative stereo method (Pillai, Ramalingam, Leonard,
 * "High-Performance and Tunable Stereo Reconstruction", Alg. 1-4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * restatement of the method that the CUDA library is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it.  It shares no code, header or table with the CUDA library.
 *
 * Every loop runs in raster order with the strict comparisons the paper
 * writes.  Where the paper is silent the reading used is stated at the
 * function.  Floating point: plane coefficients are solved in fp64 and rounded
 * to fp32; the interpolated disparity is evaluated in fp32 with two fused
 * multiply-adds, because the rounding of that value decides the integer
 * census column.  Build with -ffp-contract=off.
 *
 * Pins (tests/test_oracle_pins.py): census and Omega_I against brute force
 * on tiny images; FAST and epipolar argmin against brute force; Delaunay
 * against the empty-circumcircle property, the Euler count and a brute-force
 * enumeration; planes against exact dyadic planes; raster against the
 * partition property; refinement/resampling against the integer-shift
 * closed form and brute-force tie-breaks.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_OK 0
#define OR_E_CAP (-2)     /* an output buffer is too small */
#define OR_E_INVAL (-1)
#define OR_E_RASTER (-3)  /* a pixel was claimed twice: not a partition */

typedef struct {
    int t_lo, t_hi;       /* census-bit cost thresholds (Table 1) */
    int t_grad;           /* Omega_I gradient threshold */
    int t_fast;           /* FAST intensity threshold */
    int kp_per_bin;       /* keypoints kept per 12x10 bin */
    int uniq_margin;      /* epipolar uniqueness margin */
} or_params;

static int popc32(uint32_t x) {
    int n = 0;
    while (x) { n += (int)(x & 1u); x >>= 1; }
    return n;
}

/* ---------------------------------------------------------------------- */
/* Census 5x5 (Sec. III-C, "Census window-based matching on a 5x5 patch").  */
/* Bit b enumerates the 24 non-centre offsets row by row, dy = -2..2, dx =  */
/* -2..2, bit 0 at (-2,-2); the bit is set when the neighbour is strictly   */
/* darker than the centre.  Pixels within 2 of the border get 0.            */
/* ---------------------------------------------------------------------- */
void or_census(const uint8_t* I, int W, int H, uint32_t* out) {
    for (int v = 0; v < H; v++) {
        for (int u = 0; u < W; u++) {
            uint32_t code = 0;
            if (u >= 2 && u < W - 2 && v >= 2 && v < H - 2) {
                int bit = 0;
                int p = I[v * W + u];
                for (int dy = -2; dy <= 2; dy++) {
                    for (int dx = -2; dx <= 2; dx++) {
                        if (dx == 0 && dy == 0) continue;
                        if (I[(v + dy) * W + (u + dx)] < p) code |= (1u << bit);
                        bit++;
                    }
                }
            }
            out[v * W + u] = code;
        }
    }
}

/* Omega_I, the high-gradient subset (Sec. III; operator not given).
 * Reading: inside the 2-pixel border and |dI/du| + |dI/dv| >= t_grad with
 * central differences. */
void or_omega(const uint8_t* L, int W, int H, int t_grad, uint8_t* out) {
    for (int v = 0; v < H; v++) {
        for (int u = 0; u < W; u++) {
            int in = 0;
            if (u >= 2 && u < W - 2 && v >= 2 && v < H - 2) {
                int gx = abs((int)L[v * W + u + 1] - (int)L[v * W + u - 1]);
                int gy = abs((int)L[(v + 1) * W + u] - (int)L[(v - 1) * W + u]);
                in = (gx + gy >= t_grad);
            }
            out[v * W + u] = (uint8_t)in;
        }
    }
}

/* ---------------------------------------------------------------------- */
/* FAST keypoints sampled from 12x10 spatial bins (Sec. III-A).             */
/* Reading: FAST-9 on the radius-3 Bresenham circle; score = max over the   */
/* bright and dark sets of the summed excess over the threshold; 3x3        */
/* non-maximum suppression, equal scores resolved towards the smaller       */
/* raster index; per bin the K best by (score desc, raster index asc);      */
/* output in bin raster order, then rank.                                   */
/* ---------------------------------------------------------------------- */
static const int FAST_DX[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
static const int FAST_DY[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

/* FAST score of pixel (u,v): 0 when it is not a corner. */
int or_fast_score(const uint8_t* I, int W, int H, int u, int v, int t) {
    if (u < 3 || u >= W - 3 || v < 3 || v >= H - 3) return 0;
    int p = I[v * W + u];
    int cls[16];
    int sb = 0, sd = 0;
    for (int i = 0; i < 16; i++) {
        int q = I[(v + FAST_DY[i]) * W + (u + FAST_DX[i])];
        if (q > p + t) { cls[i] = 1; sb += q - p - t; }
        else if (q < p - t) { cls[i] = -1; sd += p - q - t; }
        else cls[i] = 0;
    }
    /* a contiguous arc (cyclic) of at least 9 of one class */
    int corner = 0;
    for (int s = 0; s < 16 && !corner; s++) {
        for (int want = -1; want <= 1; want += 2) {
            int run = 0;
            for (int k = 0; k < 16; k++) {
                if (cls[(s + k) % 16] == want) run++;
                else break;
            }
            if (run >= 9) { corner = 1; break; }
        }
    }
    if (!corner) return 0;
    return sb > sd ? sb : sd;
}

typedef struct { int score; int idx; } or_kp;

static int kp_cmp(const void* a, const void* b) {
    const or_kp* x = (const or_kp*)a;
    const or_kp* y = (const or_kp*)b;
    if (x->score != y->score) return x->score > y->score ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Writes up to cap keypoints as (u, v) pairs into out_uv; returns the count
 * or OR_E_CAP. */
int or_fast_keypoints(const uint8_t* I, int W, int H, int t_fast, int K,
                      int32_t* out_uv, int cap) {
    int* S = (int*)calloc((size_t)W * H, sizeof(int));
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++)
            S[v * W + u] = or_fast_score(I, W, H, u, v, t_fast);
    /* collect survivors of non-maximum suppression per bin */
    int nb = 120;
    or_kp** bins = (or_kp**)calloc(nb, sizeof(or_kp*));
    int* cnt = (int*)calloc(nb, sizeof(int));
    int* bcap = (int*)calloc(nb, sizeof(int));
    for (int v = 0; v < H; v++) {
        for (int u = 0; u < W; u++) {
            int s = S[v * W + u];
            if (s <= 0) continue;
            int keep = 1;
            int me = v * W + u;
            for (int dy = -1; dy <= 1 && keep; dy++) {
                for (int dx = -1; dx <= 1; dx++) {
                    if (dx == 0 && dy == 0) continue;
                    int uu = u + dx, vv = v + dy;
                    if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
                    int sn = S[vv * W + uu];
                    int other = vv * W + uu;
                    if (sn > s || (sn == s && other < me)) { keep = 0; break; }
                }
            }
            if (!keep) continue;
            int bx = (12 * u) / W, by = (10 * v) / H;
            int b = by * 12 + bx;
            if (cnt[b] == bcap[b]) {
                bcap[b] = bcap[b] ? 2 * bcap[b] : 16;
                bins[b] = (or_kp*)realloc(bins[b], sizeof(or_kp) * bcap[b]);
            }
            bins[b][cnt[b]].score = s;
            bins[b][cnt[b]].idx = me;
            cnt[b]++;
        }
    }
    int n = 0, err = 0;
    for (int b = 0; b < nb; b++) {
        if (cnt[b] > 1) qsort(bins[b], cnt[b], sizeof(or_kp), kp_cmp);
        int take = cnt[b] < K ? cnt[b] : K;
        for (int r = 0; r < take; r++) {
            if (n >= cap) { err = 1; break; }
            out_uv[2 * n] = bins[b][r].idx % W;
            out_uv[2 * n + 1] = bins[b][r].idx / W;
            n++;
        }
        free(bins[b]);
    }
    free(bins); free(cnt); free(bcap); free(S);
    return err ? OR_E_CAP : n;
}

/* ---------------------------------------------------------------------- */
/* Epipolar matching of query pixels along their row (Sec. III-A and        */
/* Alg. 4 SparseEpipolarStereo).  Reading: search d in [0, min(N_D-1,u-2)], */
/* cost = Hamming distance of the census codes, d* the first minimum;       */
/* accept when cost(d*) < t_lo and every d with |d - d*| >= 2 costs at      */
/* least cost(d*) + margin.  out_d[i] = d* or -1 when rejected.             */
/* ---------------------------------------------------------------------- */
void or_epipolar_match(const uint32_t* cL, const uint32_t* cR, int W, int H,
                       const int32_t* q_uv, int n, int dmax, int t_lo, int margin,
                       int32_t* out_d) {
    for (int i = 0; i < n; i++) {
        int u = q_uv[2 * i], v = q_uv[2 * i + 1];
        out_d[i] = -1;
        if (u < 2 || u >= W - 2 || v < 2 || v >= H - 2) continue;
        int dlim = dmax - 1 < u - 2 ? dmax - 1 : u - 2;
        uint32_t cl = cL[v * W + u];
        int best = 99, dbest = -1;
        for (int d = 0; d <= dlim; d++) {
            int c = popc32(cl ^ cR[v * W + (u - d)]);
            if (c < best) { best = c; dbest = d; }
        }
        if (dbest < 0 || best >= t_lo) continue;
        int ok = 1;
        for (int d = 0; d <= dlim; d++) {
            if (abs(d - dbest) < 2) continue;
            int c = popc32(cl ^ cR[v * W + (u - d)]);
            if (c < best + margin) { ok = 0; break; }
        }
        if (ok) out_d[i] = dbest;
    }
}

/* ---------------------------------------------------------------------- */
/* Delaunay triangulation of the support points (Sec. III-A, Alg. 1).       */
/* Reading: the unique triangulation of the exact integer predicates with   */
/* cocircular ties resolved by symbolic perturbation of the lifted          */
/* coordinate x^2+y^2 (Edelsbrunner-Muecke, "Simulation of Simplicity",    */
/* 1990), a smaller point index carrying a larger perturbation.  Points     */
/* arrive in canonical order (sorted by (v, u)).  Algorithm here: gift      */
/* wrapping from one Delaunay edge; for each directed edge the apex is the  */
/* left point whose circle through the edge holds no other left point.     */
/* O(n) per edge, O(n^2) overall: slow and plain.                           */
/* ---------------------------------------------------------------------- */
static int64_t orient2(const int32_t* P, int a, int b, int c) {
    int64_t ax = P[2 * a], ay = P[2 * a + 1];
    int64_t bx = P[2 * b], by = P[2 * b + 1];
    int64_t cx = P[2 * c], cy = P[2 * c + 1];
    return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

/* 1 when d lies inside the circle through a, b, c (orient2(a,b,c) > 0) in the
 * perturbed configuration.  The lifted determinant with rows (x, y, x^2+y^2, 1)
 * is linear in each lifted value; a perturbation eps_i of point i adds
 * eps_i times the cofactor of that entry, which is +orient(b,c,d),
 * -orient(a,c,d), +orient(a,b,d), -orient(a,b,c) for rows a, b, c, d. */
int or_incircle_sos(const int32_t* P, int a, int b, int c, int d) {
    if (d == a || d == b || d == c) return 0;
    int64_t dx = P[2 * d], dy = P[2 * d + 1];
    int64_t adx = P[2 * a] - dx, ady = P[2 * a + 1] - dy;
    int64_t bdx = P[2 * b] - dx, bdy = P[2 * b + 1] - dy;
    int64_t cdx = P[2 * c] - dx, cdy = P[2 * c + 1] - dy;
    int64_t al = adx * adx + ady * ady;
    int64_t bl = bdx * bdx + bdy * bdy;
    int64_t cl = cdx * cdx + cdy * cdy;
    int64_t det = adx * (bdy * cl - cdy * bl) - ady * (bdx * cl - cdx * bl) + al * (bdx * cdy - cdx * bdy);
    if (det != 0) return det > 0;
    int ids[4] = {a, b, c, d};
    int64_t cof[4];
    cof[0] = orient2(P, b, c, d);
    cof[1] = -orient2(P, a, c, d);
    cof[2] = orient2(P, a, b, d);
    cof[3] = -orient2(P, a, b, c);
    int used[4] = {0, 0, 0, 0};
    for (int r = 0; r < 4; r++) {
        int m = -1;
        for (int k = 0; k < 4; k++)
            if (!used[k] && (m < 0 || ids[k] < ids[m])) m = k;
        used[m] = 1;
        if (cof[m] != 0) return cof[m] > 0;
    }
    return 0;
}

typedef struct { int64_t* keys; size_t mask; } edge_set;

static int es_has_or_add(edge_set* s, int64_t key, int add) {
    size_t h = (size_t)((uint64_t)key * 0x9E3779B97F4A7C15ull >> 17) & s->mask;
    while (s->keys[h] != -1) {
        if (s->keys[h] == key) return 1;
        h = (h + 1) & s->mask;
    }
    if (add) s->keys[h] = key;
    return 0;
}

static int tri_cmp(const void* a, const void* b) {
    const int32_t* x = (const int32_t*)a;
    const int32_t* y = (const int32_t*)b;
    for (int i = 0; i < 3; i++)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

/* P: n points (u, v) in canonical order, no duplicates, coordinates in
 * [0, 16383] (the int64 in-circle determinant then cannot overflow).  Writes triangles as
 * sorted index triples (i < j < k), ascending; returns the count, or
 * OR_E_CAP. */
int or_delaunay(const int32_t* P, int n, int32_t* tri, int cap) {
    if (n < 3) return 0;
    /* starting edge: point 0 and its nearest neighbour (smallest index on ties);
     * the circle on that segment as diameter holds no other point, so the edge
     * belongs to every perturbed Delaunay triangulation */
    int q = -1;
    int64_t bestd = 0;
    for (int m = 1; m < n; m++) {
        int64_t ddx = (int64_t)P[2 * m] - P[0], ddy = (int64_t)P[2 * m + 1] - P[1];
        int64_t dd = ddx * ddx + ddy * ddy;
        if (q < 0 || dd < bestd) { q = m; bestd = dd; }
    }
    size_t sz = 16;
    while (sz < (size_t)n * 16) sz <<= 1;
    edge_set done;
    done.keys = (int64_t*)malloc(sz * sizeof(int64_t));
    for (size_t i = 0; i < sz; i++) done.keys[i] = -1;
    done.mask = sz - 1;
    size_t scap = 64, sp = 0;
    int32_t* stack = (int32_t*)malloc(scap * 2 * sizeof(int32_t));
    stack[0] = 0; stack[1] = q; stack[2] = q; stack[3] = 0; sp = 2;
    int T = 0, err = 0;
    while (sp > 0) {
        sp--;
        int i = stack[2 * sp], j = stack[2 * sp + 1];
        int64_t key = (int64_t)i * n + j;
        if (es_has_or_add(&done, key, 0)) continue;
        /* apex: the left point whose circle through (i, j) contains no other left point */
        int k = -1;
        for (int m = 0; m < n; m++) {
            if (m == i || m == j) continue;
            if (orient2(P, i, j, m) <= 0) continue;
            if (k < 0 || or_incircle_sos(P, i, j, k, m)) k = m;
        }
        es_has_or_add(&done, key, 1);
        if (k < 0) continue; /* hull edge: nothing on its left */
        es_has_or_add(&done, (int64_t)j * n + k, 1);
        es_has_or_add(&done, (int64_t)k * n + i, 1);
        if (T >= cap) { err = 1; break; }
        int32_t t3[3] = {i, j, k};
        /* sort the triple */
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2 - a; b++)
                if (t3[b] > t3[b + 1]) { int32_t tmp = t3[b]; t3[b] = t3[b + 1]; t3[b + 1] = tmp; }
        memcpy(tri + 3 * T, t3, sizeof(t3));
        T++;
        int32_t nxt[6] = {j, i, k, j, i, k};
        for (int e = 0; e < 3; e++) {
            int a = nxt[2 * e], b = nxt[2 * e + 1];
            if (es_has_or_add(&done, (int64_t)a * n + b, 0)) continue;
            if (sp + 1 >= scap) {
                scap *= 2;
                stack = (int32_t*)realloc(stack, scap * 2 * sizeof(int32_t));
            }
            stack[2 * sp] = a; stack[2 * sp + 1] = b; sp++;
        }
    }
    free(stack);
    free(done.keys);
    if (err) return OR_E_CAP;
    qsort(tri, T, 3 * sizeof(int32_t), tri_cmp);
    return T;
}

/* ---------------------------------------------------------------------- */
/* Disparity plane per triangle (Eq. 3, "solving a linear system").         */
/* Reading: Cramer's rule in fp64 over the vertices in index order          */
/* (p0, p1, p2) = (i, j, k); coefficients rounded to fp32.                  */
/* ---------------------------------------------------------------------- */
void or_planes(const int32_t* P, const float* D, const int32_t* tri, int T, float* abc) {
    for (int t = 0; t < T; t++) {
        int i = tri[3 * t], j = tri[3 * t + 1], k = tri[3 * t + 2];
        int64_t u0 = P[2 * i], v0 = P[2 * i + 1];
        int64_t u1 = P[2 * j], v1 = P[2 * j + 1];
        int64_t u2 = P[2 * k], v2 = P[2 * k + 1];
        int64_t det = (u1 - u0) * (v2 - v0) - (u2 - u0) * (v1 - v0);
        double d0 = (double)D[i], d1 = (double)D[j], d2 = (double)D[k];
        double dd1 = d1 - d0, dd2 = d2 - d0;
        double na = dd1 * (double)(v2 - v0) - dd2 * (double)(v1 - v0);
        double nb = (double)(u1 - u0) * dd2 - (double)(u2 - u0) * dd1;
        double A = na / (double)det;
        double B = nb / (double)det;
        double C = d0 - A * (double)u0 - B * (double)v0;
        abc[3 * t] = (float)A;
        abc[3 * t + 1] = (float)B;
        abc[3 * t + 2] = (float)C;
    }
}

/* ---------------------------------------------------------------------- */
/* Pixel -> triangle lookup table (Sec. III-B).  Reading: pixel centres at  */
/* integer (u, v), the lattice of the vertices; a pixel belongs to a        */
/* triangle when every edge function is positive, or zero on a top or left  */
/* edge.  Per triangle, every pixel of its bounding box is tested.          */
/* ---------------------------------------------------------------------- */
static int top_left(int64_t ax, int64_t ay, int64_t bx, int64_t by) {
    int64_t dx = bx - ax, dy = by - ay;
    return (dy == 0 && dx > 0) || dy < 0;
}

int or_raster(const int32_t* P, const int32_t* tri, int T, int W, int H, int32_t* planeidx) {
    for (int i = 0; i < W * H; i++) planeidx[i] = -1;
    for (int t = 0; t < T; t++) {
        int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        if (orient2(P, a, b, c) < 0) { int tmp = b; b = c; c = tmp; }
        int64_t x[3] = {P[2 * a], P[2 * b], P[2 * c]};
        int64_t y[3] = {P[2 * a + 1], P[2 * b + 1], P[2 * c + 1]};
        int64_t x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
        for (int e = 1; e < 3; e++) {
            if (x[e] < x0) x0 = x[e];
            if (x[e] > x1) x1 = x[e];
            if (y[e] < y0) y0 = y[e];
            if (y[e] > y1) y1 = y[e];
        }
        if (x0 < 0) x0 = 0;
        if (y0 < 0) y0 = 0;
        if (x1 > W - 1) x1 = W - 1;
        if (y1 > H - 1) y1 = H - 1;
        for (int64_t v = y0; v <= y1; v++) {
            for (int64_t u = x0; u <= x1; u++) {
                int inside = 1;
                for (int e = 0; e < 3 && inside; e++) {
                    int64_t ax = x[e], ay = y[e], bx = x[(e + 1) % 3], by = y[(e + 1) % 3];
                    int64_t E = (bx - ax) * (v - ay) - (by - ay) * (u - ax);
                    if (!(E > 0 || (E == 0 && top_left(ax, ay, bx, by)))) inside = 0;
                }
                if (!inside) continue;
                if (planeidx[v * W + u] != -1) return OR_E_RASTER;
                planeidx[v * W + u] = t;
            }
        }
    }
    return OR_OK;
}

/* Interpolated disparity of Eq. 3: D_it = fma(a, u, fma(b, v, c)) in fp32. */
float or_interp(const float* abc, int t, int u, int v) {
    return fmaf(abc[3 * t], (float)u, fmaf(abc[3 * t + 1], (float)v, abc[3 * t + 2]));
}

/* DisparityInterpolation (Alg. 1): the dense map D_it over the lookup table,
 * NaN where a pixel has no triangle. */
void or_interp_map(const int32_t* planeidx, const float* abc, int W, int H, float* out) {
    for (int v = 0; v < H; v++)
        for (int u = 0; u < W; u++) {
            int t = planeidx[v * W + u];
            out[v * W + u] = t >= 0 ? or_interp(abc, t, u, v) : NAN;
        }
}

/* ---------------------------------------------------------------------- */
/* One pass of DisparityInterpolation + CostEvaluation (Alg. 2) +           */
/* DisparityRefinement (Alg. 3) in raster order over Omega_I.               */
/* A pixel is evaluated when it is in Omega_I, lies in a triangle, and the  */
/* rounded disparity k = rint(D_it) keeps the right window inside the image */
/* (2 <= u - k <= W - 3).  Cells: (u / sz, v / sz) on a ceil(H/sz) x         */
/* ceil(W/sz) grid.  Cg holds the least cost below t_lo (first in raster    */
/* order on ties), Cb the largest cost above t_hi (first in raster order).  */
/* mask: bit0 in Omega_I, bit1 evaluated, bit2 cost < t_lo, bit3 > t_hi.    */
/* Cg is written as (u, v, d, cost) with gw = 1 when written; Cb as          */
/* (u, v, cost) with bw = 1 when written.                                   */
/* ---------------------------------------------------------------------- */
void or_validate(const uint32_t* cL, const uint32_t* cR, const uint8_t* omega,
                 const int32_t* planeidx, const float* abc, int W, int H, int sz,
                 int t_lo, int t_hi, float* Df, uint8_t* Cf, uint8_t* mask,
                 int32_t* cg_uv, float* cg_d, int32_t* cg_cost, uint8_t* cg_w,
                 int32_t* cb_uv, int32_t* cb_cost, uint8_t* cb_w) {
    int Wc = (W + sz - 1) / sz, Hc = (H + sz - 1) / sz;
    for (int c = 0; c < Wc * Hc; c++) {
        cg_uv[2 * c] = 0; cg_uv[2 * c + 1] = 0; cg_d[c] = 0.0f; cg_cost[c] = t_lo; cg_w[c] = 0;
        cb_uv[2 * c] = 0; cb_uv[2 * c + 1] = 0; cb_cost[c] = t_hi; cb_w[c] = 0;
    }
    for (int v = 0; v < H; v++) {
        for (int u = 0; u < W; u++) {
            int p = v * W + u;
            mask[p] = 0;
            if (!omega[p]) continue;
            mask[p] = 1;
            int t = planeidx[p];
            if (t < 0) continue;
            float d = or_interp(abc, t, u, v);
            float kf = nearbyintf(d);
            float col = (float)u - kf;
            if (!(col >= 2.0f && col <= (float)(W - 3))) continue;
            int k = (int)kf;
            mask[p] |= 2;
            int cost = popc32(cL[p] ^ cR[p - k]);
            if (cost < Cf[p]) {
                Df[p] = d;
                Cf[p] = (uint8_t)cost;
            }
            int cell = (v / sz) * Wc + (u / sz);
            if (cost < t_lo) {
                mask[p] |= 4;
                if (cost < cg_cost[cell]) {
                    cg_uv[2 * cell] = u; cg_uv[2 * cell + 1] = v;
                    cg_d[cell] = d; cg_cost[cell] = cost; cg_w[cell] = 1;
                }
            }
            if (cost > t_hi) {
                mask[p] |= 8;
                if (cost > cb_cost[cell]) {
                    cb_uv[2 * cell] = u; cb_uv[2 * cell + 1] = v;
                    cb_cost[cell] = cost; cb_w[cell] = 1;
                }
            }
        }
    }
}

/* ---------------------------------------------------------------------- */
/* Support set bookkeeping.  A support point is (u, v, d), integer pixel,    */
/* fp32 disparity.  Canonical order: sorted by (v, u).                      */
/* ---------------------------------------------------------------------- */
typedef struct { int32_t u, v; float d; } or_sp;

static int sp_cmp(const void* a, const void* b) {
    const or_sp* x = (const or_sp*)a;
    const or_sp* y = (const or_sp*)b;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return (x->u > y->u) - (x->u < y->u);
}

/* ---------------------------------------------------------------------- */
/* SupportResampling (Alg. 4).  Reading of the garbled loop: cells in       */
/* raster order; a written Cg cell adds (u, v, D_it); a written Cb cell adds */
/* (u, v) to X; X is matched by epipolar search and accepted matches join.  */
/* A pixel already in the support set keeps its point; within one round a   */
/* Cg point is taken before an X match.  Returns the new count or OR_E_CAP. */
/* S (capacity cap) is updated in place and left in canonical order.       */
/* ---------------------------------------------------------------------- */
int or_resample(const uint32_t* cL, const uint32_t* cR, int W, int H, int sz,
                const int32_t* cg_uv, const float* cg_d, const uint8_t* cg_w,
                const int32_t* cb_uv, const uint8_t* cb_w, int dmax, int t_lo, int margin,
                or_sp* S, int n, int cap) {
    int Wc = (W + sz - 1) / sz, Hc = (H + sz - 1) / sz, nc = Wc * Hc;
    uint8_t* occ = (uint8_t*)calloc((size_t)W * H, 1);
    for (int i = 0; i < n; i++) occ[S[i].v * W + S[i].u] = 1;
    int32_t* X = (int32_t*)malloc(sizeof(int32_t) * 2 * (nc + 1));
    int nx = 0, err = 0;
    for (int c = 0; c < nc; c++) {
        if (cg_w[c]) {
            int u = cg_uv[2 * c], v = cg_uv[2 * c + 1];
            if (!occ[v * W + u]) {
                if (n >= cap) { err = 1; break; }
                S[n].u = u; S[n].v = v; S[n].d = cg_d[c]; n++;
                occ[v * W + u] = 1;
            }
        }
        if (cb_w[c]) {
            X[2 * nx] = cb_uv[2 * c]; X[2 * nx + 1] = cb_uv[2 * c + 1]; nx++;
        }
    }
    if (!err && nx > 0) {
        int32_t* dm = (int32_t*)malloc(sizeof(int32_t) * nx);
        or_epipolar_match(cL, cR, W, H, X, nx, dmax, t_lo, margin, dm);
        for (int i = 0; i < nx && !err; i++) {
            if (dm[i] < 0) continue;
            int u = X[2 * i], v = X[2 * i + 1];
            if (occ[v * W + u]) continue;
            if (n >= cap) { err = 1; break; }
            S[n].u = u; S[n].v = v; S[n].d = (float)dm[i]; n++;
            occ[v * W + u] = 1;
        }
        free(dm);
    }
    free(X);
    free(occ);
    if (err) return OR_E_CAP;
    qsort(S, n, sizeof(or_sp), sp_cmp);
    return n;
}

/* ---------------------------------------------------------------------- */
/* Alg. 1: the whole method for one pair.                                   */
/* Outputs D_f, C_f, the last pass's mask and plane-index map, and a trace: */
/* support sets S_1..S_iters concatenated as (u, v, d) float triples with   */
/* their sizes in n_support[it], and triangle counts in n_tri[it].          */
/* Returns OR_OK or an error code.                                          */
/* ---------------------------------------------------------------------- */
int or_run(const uint8_t* L, const uint8_t* R, int W, int H, int dmax, int iters, int cell,
           const or_params* prm, float* Df, uint8_t* Cf, uint8_t* mask, int32_t* planeidx,
           float* trace_sup, int trace_cap, int32_t* n_support, int32_t* n_tri) {
    if (W < 5 || H < 5 || dmax < 1 || dmax > 256 || iters < 1 || cell < 1) return OR_E_INVAL;
    if (!(0 <= prm->t_lo && prm->t_lo <= prm->t_hi && prm->t_hi < 24)) return OR_E_INVAL;
    size_t N = (size_t)W * H;
    uint32_t* cL = (uint32_t*)malloc(N * 4);
    uint32_t* cR = (uint32_t*)malloc(N * 4);
    uint8_t* omega = (uint8_t*)malloc(N);
    or_census(L, W, H, cL);
    or_census(R, W, H, cR);
    or_omega(L, W, H, prm->t_grad, omega);
    /* D_f <- 0, C_f <- t_hi (Alg. 1) */
    for (size_t p = 0; p < N; p++) { Df[p] = 0.0f; Cf[p] = (uint8_t)prm->t_hi; }
    /* S_1 <- SparseStereo(I_l, I_r) */
    int kcap = 120 * (prm->kp_per_bin > 0 ? prm->kp_per_bin : 1);
    int32_t* kp = (int32_t*)malloc(sizeof(int32_t) * 2 * kcap);
    int nk = or_fast_keypoints(L, W, H, prm->t_fast, prm->kp_per_bin, kp, kcap);
    int32_t* kd = (int32_t*)malloc(sizeof(int32_t) * (nk > 0 ? nk : 1));
    or_epipolar_match(cL, cR, W, H, kp, nk, dmax, prm->t_lo, prm->uniq_margin, kd);
    int scap = (int)(N < 1000 ? 1000 : N);
    or_sp* S = (or_sp*)malloc(sizeof(or_sp) * scap);
    int n = 0;
    for (int i = 0; i < nk; i++) {
        if (kd[i] < 0) continue;
        S[n].u = kp[2 * i]; S[n].v = kp[2 * i + 1]; S[n].d = (float)kd[i]; n++;
    }
    qsort(S, n, sizeof(or_sp), sp_cmp);
    free(kp); free(kd);

    int sz = cell;
    int rc = OR_OK, tpos = 0;
    int Wc0 = (W + 0) / 1, Hc0 = H; /* cells never exceed pixels */
    size_t ncmax = (size_t)Wc0 * Hc0;
    int32_t* cg_uv = (int32_t*)malloc(sizeof(int32_t) * 2 * ncmax);
    float* cg_d = (float*)malloc(sizeof(float) * ncmax);
    int32_t* cg_cost = (int32_t*)malloc(sizeof(int32_t) * ncmax);
    uint8_t* cg_w = (uint8_t*)malloc(ncmax);
    int32_t* cb_uv = (int32_t*)malloc(sizeof(int32_t) * 2 * ncmax);
    int32_t* cb_cost = (int32_t*)malloc(sizeof(int32_t) * ncmax);
    uint8_t* cb_w = (uint8_t*)malloc(ncmax);
    int32_t* P = (int32_t*)malloc(sizeof(int32_t) * 2 * scap);
    float* D = (float*)malloc(sizeof(float) * scap);
    int tcap = 2 * scap + 16;
    int32_t* tri = (int32_t*)malloc(sizeof(int32_t) * 3 * tcap);
    float* abc = (float*)malloc(sizeof(float) * 3 * tcap);
    for (int it = 1; it <= iters; it++) {
        /* trace S_it */
        n_support[it - 1] = n;
        for (int i = 0; i < n; i++) {
            if (tpos + 3 > trace_cap) { rc = OR_E_CAP; break; }
            trace_sup[tpos++] = (float)S[i].u;
            trace_sup[tpos++] = (float)S[i].v;
            trace_sup[tpos++] = S[i].d;
        }
        if (rc != OR_OK) break;
        /* G(S_it) <- DelaunayTriangulation(S_it) */
        for (int i = 0; i < n; i++) { P[2 * i] = S[i].u; P[2 * i + 1] = S[i].v; D[i] = S[i].d; }
        int T = or_delaunay(P, n, tri, tcap);
        if (T < 0) { rc = T; break; }
        n_tri[it - 1] = T;
        or_planes(P, D, tri, T, abc);
        /* D_it <- DisparityInterpolation(G(S_it)) via the lookup table */
        int r = or_raster(P, tri, T, W, H, planeidx);
        if (r != OR_OK) { rc = r; break; }
        /* C_it <- CostEvaluation; C_g, C_b <- DisparityRefinement */
        or_validate(cL, cR, omega, planeidx, abc, W, H, sz, prm->t_lo, prm->t_hi, Df, Cf, mask,
                    cg_uv, cg_d, cg_cost, cg_w, cb_uv, cb_cost, cb_w);
        if (it != iters) {
            /* S_{it+1} <- SupportResampling(C_g, C_b, S_it) */
            int m = or_resample(cL, cR, W, H, sz, cg_uv, cg_d, cg_w, cb_uv, cb_w, dmax,
                                prm->t_lo, prm->uniq_margin, S, n, scap);
            if (m < 0) { rc = m; break; }
            n = m;
            sz = sz / 2 > 1 ? sz / 2 : 1;
        }
    }
    free(cL); free(cR); free(omega); free(S);
    free(cg_uv); free(cg_d); free(cg_cost); free(cg_w);
    free(cb_uv); free(cb_cost); free(cb_w);
    free(P); free(D); free(tri); free(abc);
    return rc;
}
