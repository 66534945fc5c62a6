// sm_103a kernels of the stereo hot path.  Every kernel is persistent over a
// work list: one launch may cover many frame pairs (PairBatch), with blocks
// striding over (pair, tile) items.  Nothing here waits on another block.
#include <cstdio>

#include "internal.h"

namespace stereo {

// ---------------------------------------------------------------- plumbing
int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

constexpr int kTileW = 32;   // census / FAST score / validate tile: one warp per row
constexpr int kTileH = 8;

int work_items(WorkKind k, const PairDev& p) {
    switch (k) {
        case WK_CENSUS:
        case WK_FAST_SCORE:
        case WK_VALIDATE: return cdiv(p.W, kTileW) * cdiv(p.H, kTileH);
        case WK_FAST_BINS: return kFastBins;
        case WK_MATCH_KP: return cdiv((long long)kFastBins * p.K, 8);
        case WK_TRI: return cdiv(p.T, 256);
        case WK_SCAN: return 1;
        case WK_RASTER: return p.tiles_x * p.tiles_y;
        case WK_RESAMPLE: return cdiv((long long)p.Wc * p.Hc, 8);
        default: return 0;
    }
}

__device__ __forceinline__ int find_pair(const int* off, int n, int item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Runs body(pair, local_item) for every work item of the batch; items are
// block-uniform, so bodies may use __syncthreads.
#define FOR_EACH_ITEM(b, BODY)                                                  \
    for (int item_ = blockIdx.x; item_ < (b).total; item_ += gridDim.x) {       \
        if ((b).pd) {                                                           \
            int pi_ = find_pair((b).work_off, (b).npairs, item_);               \
            const PairDev& P_ = (b).pd[pi_];                                    \
            int local_ = item_ - __ldg((b).work_off + pi_);                     \
            BODY(P_, local_);                                                   \
        } else {                                                                \
            BODY((b).one, item_);                                               \
        }                                                                       \
    }

static int grid_for(int total, int per_sm) {
    int cap = sm_count() * per_sm;
    return total < cap ? total : cap;
}

// ---------------------------------------------------------------- census + Omega_I
// Census 5x5 (Sec. III-C) of L and R and the Omega_I bit map of L.  One
// 32x8 tile per block; rows are staged with a 2-pixel halo in shared memory.
__device__ __forceinline__ uint32_t census_at(const uint8_t (*s)[kTileW + 4], int r, int c) {
    const int p = s[r][c];
    uint32_t code = 0;
    int bit = 0;
#pragma unroll
    for (int dy = -2; dy <= 2; dy++) {
#pragma unroll
        for (int dx = -2; dx <= 2; dx++) {
            if (dx == 0 && dy == 0) continue;
            code |= (uint32_t)(s[r + dy][c + dx] < p) << bit;
            bit++;
        }
    }
    return code;
}

__device__ __forceinline__ void census_body(const PairDev& P, int local, const Params& prm) {
    __shared__ uint8_t sL[kTileH + 4][kTileW + 4];
    __shared__ uint8_t sR[kTileH + 4][kTileW + 4];
    const int W = P.W, H = P.H;
    const int tx_n = (W + kTileW - 1) / kTileW;
    const int u0 = (local % tx_n) * kTileW, v0 = (local / tx_n) * kTileH;
    for (int i = threadIdx.x; i < (kTileH + 4) * (kTileW + 4); i += blockDim.x) {
        int r = i / (kTileW + 4), c = i % (kTileW + 4);
        int v = min(max(v0 + r - 2, 0), H - 1), u = min(max(u0 + c - 2, 0), W - 1);
        sL[r][c] = P.L[(size_t)v * W + u];
        sR[r][c] = P.R[(size_t)v * W + u];
    }
    __syncthreads();
    const int lx = threadIdx.x % kTileW, ly = threadIdx.x / kTileW;
    const int u = u0 + lx, v = v0 + ly;
    const bool inimg = u < W && v < H;
    const bool interior = u >= 2 && u < W - 2 && v >= 2 && v < H - 2;
    uint32_t cl = 0, cr = 0;
    bool om = false;
    if (interior) {
        cl = census_at(sL, ly + 2, lx + 2);
        cr = census_at(sR, ly + 2, lx + 2);
        int gx = abs((int)sL[ly + 2][lx + 3] - (int)sL[ly + 2][lx + 1]);
        int gy = abs((int)sL[ly + 3][lx + 2] - (int)sL[ly + 1][lx + 2]);
        om = gx + gy >= prm.t_grad;
    }
    if (inimg) {
        size_t p = (size_t)v * W + u;
        if (P.cL) P.cL[p] = cl;
        if (P.cR) P.cR[p] = cr;
    }
    unsigned bits = __ballot_sync(0xffffffffu, om);
    if (lx == 0 && v < H && P.omega) P.omega[(size_t)v * ((W + 31) / 32) + (u0 >> 5)] = bits;
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_census(PairBatch b, Params prm) {
#define BODY(P, l) census_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// ---------------------------------------------------------------- FAST score
// FAST-9 on the radius-3 Bresenham circle (Sec. III-A, [rosten2006machine]).
__constant__ int8_t c_fast_dx[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
__constant__ int8_t c_fast_dy[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};

__device__ __forceinline__ bool has_run9(uint32_t m16) {
    uint32_t x = m16 | (m16 << 16);
    uint32_t r = x;
#pragma unroll
    for (int i = 1; i < 9; i++) r &= x >> i;
    return (r & 0xFFFFu) != 0;
}

__device__ __forceinline__ void fast_score_body(const PairDev& P, int local, const Params& prm) {
    __shared__ uint8_t s[kTileH + 6][kTileW + 6];
    const int W = P.W, H = P.H;
    const int tx_n = (W + kTileW - 1) / kTileW;
    const int u0 = (local % tx_n) * kTileW, v0 = (local / tx_n) * kTileH;
    for (int i = threadIdx.x; i < (kTileH + 6) * (kTileW + 6); i += blockDim.x) {
        int r = i / (kTileW + 6), c = i % (kTileW + 6);
        int v = min(max(v0 + r - 3, 0), H - 1), u = min(max(u0 + c - 3, 0), W - 1);
        s[r][c] = P.L[(size_t)v * W + u];
    }
    __syncthreads();
    const int lx = threadIdx.x % kTileW, ly = threadIdx.x / kTileW;
    const int u = u0 + lx, v = v0 + ly;
    if (u < W && v < H) {
        int score = 0;
        if (u >= 3 && u < W - 3 && v >= 3 && v < H - 3) {
            const int p = s[ly + 3][lx + 3];
            const int t = prm.t_fast;
            uint32_t mb = 0, md = 0;
            int sb = 0, sd = 0;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                int q = s[ly + 3 + c_fast_dy[i]][lx + 3 + c_fast_dx[i]];
                if (q > p + t) { mb |= 1u << i; sb += q - p - t; }
                else if (q < p - t) { md |= 1u << i; sd += p - q - t; }
            }
            if (has_run9(mb) || has_run9(md)) score = sb > sd ? sb : sd;
        }
        P.fast_score[(size_t)v * W + u] = (int16_t)score;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_fast_score(PairBatch b, Params prm) {
#define BODY(P, l) fast_score_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// ---------------------------------------------------------------- FAST bins: NMS + top-K
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long x, unsigned long long* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long y = threadIdx.x < nw ? red[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long z = __shfl_xor_sync(0xffffffffu, y, o);
            y = z > y ? z : y;
        }
        if (threadIdx.x == 0) red[32] = y;
    }
    __syncthreads();
    unsigned long long r = red[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void fast_bins_body(const PairDev& P, int bin, const Params& prm) {
    __shared__ unsigned long long red[33];
    const int W = P.W, H = P.H, K = P.K;
    const int bx = bin % kFastBinsX, by = bin / kFastBinsX;
    // pixels with floor(12u/W) == bx, floor(10v/H) == by
    const int ua = (bx * W + kFastBinsX - 1) / kFastBinsX, ub = ((bx + 1) * W + kFastBinsX - 1) / kFastBinsX;
    const int va = (by * H + kFastBinsY - 1) / kFastBinsY, vb = ((by + 1) * H + kFastBinsY - 1) / kFastBinsY;
    const int bw = ub - ua, n = bw * (vb - va);
    unsigned long long top[kMaxK];
    int cnt = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int u = ua + i % bw, v = va + i / bw;
        const int me = v * W + u;
        const int s = P.fast_score[me];
        if (s <= 0) continue;
        bool keep = true;
#pragma unroll
        for (int dy = -1; dy <= 1; dy++) {
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) {
                if (dx == 0 && dy == 0) continue;
                const int uu = u + dx, vv = v + dy;
                if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
                const int o = vv * W + uu;
                const int sn = P.fast_score[o];
                if (sn > s || (sn == s && o < me)) keep = false;
            }
        }
        if (!keep) continue;
        unsigned long long key = ((unsigned long long)s << 32) | (0xFFFFFFFFu - (unsigned)me);
        // insertion into a descending list of at most K
        int pos = cnt < K ? cnt : K;
        while (pos > 0 && top[pos - 1] < key) {
            if (pos < K) top[pos] = top[pos - 1];
            pos--;
        }
        if (pos < K) {
            top[pos] = key;
            if (cnt < K) cnt++;
        }
    }
    int head = 0;
    int32_t* out = P.kp_uv + (size_t)bin * K * 2;
    for (int r = 0; r < K; r++) {
        unsigned long long mine = head < cnt ? top[head] : 0ull;
        unsigned long long best = block_max_u64(mine, red);
        if (best != 0ull && mine == best) head++;
        if (threadIdx.x == 0) {
            if (best == 0ull) {
                out[2 * r] = -1;
                out[2 * r + 1] = -1;
            } else {
                const unsigned me = 0xFFFFFFFFu - (unsigned)(best & 0xFFFFFFFFu);
                out[2 * r] = (int)(me % (unsigned)W);
                out[2 * r + 1] = (int)(me / (unsigned)W);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_fast_bins(PairBatch b, Params prm) {
#define BODY(P, l) fast_bins_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// ---------------------------------------------------------------- epipolar matching
// One warp per query (Sec. III-A; Alg. 4 SparseEpipolarStereo).  Lanes stride
// the disparity range; the argmin packs (cost << 8) | d, so ties go to the
// smallest d.  The uniqueness test is a second minimum over |d - d*| >= 2.
__device__ __forceinline__ int warp_match(const uint32_t* __restrict__ cL, const uint32_t* __restrict__ cR,
                                          int W, int H, int u, int v, int dmax, int t_lo, int margin) {
    const int lane = threadIdx.x & 31;
    if (u < 2 || u >= W - 2 || v < 2 || v >= H - 2) return -1;
    const int dlim = min(dmax - 1, u - 2);
    const size_t p = (size_t)v * W + u;
    const uint32_t cl = __ldg(cL + p);
    const uint32_t* row = cR + p;
    uint32_t cost[8];
    uint32_t best = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int d = lane + 32 * j;
        cost[j] = 0xFFu;
        if (d <= dlim) {
            cost[j] = __popc(cl ^ __ldg(row - d));
            best = min(best, (cost[j] << 8) | (uint32_t)d);
        }
    }
    best = __reduce_min_sync(0xffffffffu, best);
    const int cstar = (int)(best >> 8), dstar = (int)(best & 255u);
    if (cstar >= t_lo) return -1;
    uint32_t second = 0xFFu;
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int d = lane + 32 * j;
        if (d <= dlim && abs(d - dstar) >= 2) second = min(second, cost[j]);
    }
    second = __reduce_min_sync(0xffffffffu, second);
    if (second != 0xFFu && (int)second < cstar + margin) return -1;
    return dstar;
}

__device__ __forceinline__ void match_kp_body(const PairDev& P, int local, const Params& prm) {
    const int q = local * 8 + (threadIdx.x >> 5);
    if (q >= kFastBins * P.K) return;
    const int u = P.kp_uv[2 * q], v = P.kp_uv[2 * q + 1];
    int d = -1;
    if (u >= 0) d = warp_match(P.cL, P.cR, P.W, P.H, u, v, P.dmax, prm.t_lo, prm.margin);
    if ((threadIdx.x & 31) == 0) P.kp_d[q] = d;
}

__global__ void __launch_bounds__(256) k_match_kp(PairBatch b, Params prm) {
#define BODY(P, l) match_kp_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

__global__ void __launch_bounds__(256) k_match_list(const uint32_t* cL, const uint32_t* cR, int W, int H,
                                                    const int32_t* q, int n, int dmax, Params prm, int32_t* out) {
    for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < n; i += gridDim.x * 8) {
        const int u = q[2 * i], v = q[2 * i + 1];
        int d = -1;
        if (u >= 0) d = warp_match(cL, cR, W, H, u, v, dmax, prm.t_lo, prm.margin);
        if ((threadIdx.x & 31) == 0) out[i] = d;
    }
}

// ---------------------------------------------------------------- raster (Sec. III-B)
// Triangles are binned to 16x16 tiles by bounding box (count, scan, fill);
// then each tile's pixels test the tile's triangles with exact integer edge
// functions and the top-left rule.  The rule partitions the hull, so the
// order of a tile's list does not matter.
__device__ __forceinline__ void tri_tiles(const int32_t* t6, int W, int H, int& tx0, int& tx1, int& ty0, int& ty1) {
    int x0 = min(t6[0], min(t6[2], t6[4])), x1 = max(t6[0], max(t6[2], t6[4]));
    int y0 = min(t6[1], min(t6[3], t6[5])), y1 = max(t6[1], max(t6[3], t6[5]));
    x0 = max(x0, 0); y0 = max(y0, 0); x1 = min(x1, W - 1); y1 = min(y1, H - 1);
    tx0 = x0 / kRasterTile; tx1 = x1 / kRasterTile; ty0 = y0 / kRasterTile; ty1 = y1 / kRasterTile;
}

__device__ __forceinline__ void raster_count_body(const PairDev& P, int local) {
    const int t = local * 256 + threadIdx.x;
    if (t >= P.T) return;
    int tx0, tx1, ty0, ty1;
    tri_tiles(P.tri_uv + 6 * (size_t)t, P.W, P.H, tx0, tx1, ty0, ty1);
    for (int ty = ty0; ty <= ty1; ty++)
        for (int tx = tx0; tx <= tx1; tx++) atomicAdd(P.tile_cnt + ty * P.tiles_x + tx, 1);
}

__global__ void __launch_bounds__(256) k_raster_count(PairBatch b) {
#define BODY(P, l) raster_count_body(P, l)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

__device__ __forceinline__ void raster_scan_body(const PairDev& P, int) {
    __shared__ int warp_sums[32];
    const int n = P.tiles_x * P.tiles_y;
    const int chunk = (n + blockDim.x - 1) / blockDim.x;
    const int a = min(n, (int)threadIdx.x * chunk), e = min(n, a + chunk);
    int s = 0;
    for (int i = a; i < e; i++) s += P.tile_cnt[i];
    // exclusive scan of s across the block
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        warp_sums[lane] = ws;
    }
    __syncthreads();
    int run = x - s + (w > 0 ? warp_sums[w - 1] : 0);
    for (int i = a; i < e; i++) {
        P.tile_off[i] = run;
        run += P.tile_cnt[i];
        P.tile_cnt[i] = 0;
    }
    if (threadIdx.x == blockDim.x - 1) P.tile_off[n] = run;
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_raster_scan(PairBatch b) {
#define BODY(P, l) raster_scan_body(P, l)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

__device__ __forceinline__ void raster_fill_body(const PairDev& P, int local) {
    const int t = local * 256 + threadIdx.x;
    if (t >= P.T) return;
    int tx0, tx1, ty0, ty1;
    tri_tiles(P.tri_uv + 6 * (size_t)t, P.W, P.H, tx0, tx1, ty0, ty1);
    for (int ty = ty0; ty <= ty1; ty++)
        for (int tx = tx0; tx <= tx1; tx++) {
            const int tile = ty * P.tiles_x + tx;
            const int pos = atomicAdd(P.tile_cnt + tile, 1);
            const int at = P.tile_off[tile] + pos;
            if (at < P.tile_cap) P.tile_list[at] = t;
        }
}

__global__ void __launch_bounds__(256) k_raster_fill(PairBatch b) {
#define BODY(P, l) raster_fill_body(P, l)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

struct EdgeSet {  // three edge functions A*u + B*v + C >= bias, and the id
    int A[3], B[3], C[3];
    int bias;     // bit e set: edge e needs E >= 1 (not a top or left edge)
    int id;
};

__device__ __forceinline__ void raster_pixels_body(const PairDev& P, int local) {
    __shared__ EdgeSet s[256];
    const int tile = local;
    const int tx = tile % P.tiles_x, ty = tile / P.tiles_x;
    const int u = tx * kRasterTile + (threadIdx.x % kRasterTile);
    const int v = ty * kRasterTile + (threadIdx.x / kRasterTile);
    const int beg = min(P.tile_off[tile], P.tile_cap), end = min(P.tile_off[tile + 1], P.tile_cap);
    int hit = -1;
    for (int base = beg; base < end; base += 256) {
        const int i = base + threadIdx.x;
        if (i < end) {
            const int t = P.tile_list[i];
            const int32_t* q = P.tri_uv + 6 * (size_t)t;
            int x[3] = {q[0], q[2], q[4]}, y[3] = {q[1], q[3], q[5]};
            const long long o = (long long)(x[1] - x[0]) * (y[2] - y[0]) - (long long)(y[1] - y[0]) * (x[2] - x[0]);
            if (o < 0) {  // make the orientation positive
                int tx_ = x[1]; x[1] = x[2]; x[2] = tx_;
                int ty_ = y[1]; y[1] = y[2]; y[2] = ty_;
            }
            EdgeSet e;
            e.bias = 0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int ax = x[k], ay = y[k], bx = x[(k + 1) % 3], by = y[(k + 1) % 3];
                const int dx = bx - ax, dy = by - ay;
                // E(u, v) = dx * (v - ay) - dy * (u - ax)
                e.A[k] = -dy;
                e.B[k] = dx;
                e.C[k] = dy * ax - dx * ay;
                const bool tl = (dy == 0 && dx > 0) || dy < 0;
                if (!tl) e.bias |= 1 << k;
            }
            e.id = t;
            s[threadIdx.x] = e;
        }
        __syncthreads();
        const int m = min(256, end - base);
        for (int j = 0; j < m; j++) {
            const EdgeSet& e = s[j];
            const int e0 = e.A[0] * u + e.B[0] * v + e.C[0];
            const int e1 = e.A[1] * u + e.B[1] * v + e.C[1];
            const int e2 = e.A[2] * u + e.B[2] * v + e.C[2];
            if (e0 >= (e.bias & 1) && e1 >= ((e.bias >> 1) & 1) && e2 >= ((e.bias >> 2) & 1)) hit = e.id;
        }
        __syncthreads();
    }
    if (u < P.W && v < P.H) P.planeidx[(size_t)v * P.W + u] = hit;
}

__global__ void __launch_bounds__(256) k_raster_pixels(PairBatch b) {
#define BODY(P, l) raster_pixels_body(P, l)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// ---------------------------------------------------------------- fused validate (Alg. 2 + Alg. 3)
// Per pixel: Omega_I bit, plane lookup, fp32 interpolation (Eq. 3), census
// Hamming cost at the rounded disparity, the strict-< update of (D_f, C_f),
// the validation mask, and the per-cell C_g / C_b keys reduced in shared
// memory before one global atomicMin per cell and tile.
constexpr int kMaxLocalCells = 256;

__device__ __forceinline__ void validate_body(const PairDev& P, int local, const Params& prm) {
    __shared__ uint32_t s_g[kMaxLocalCells], s_b[kMaxLocalCells];
    const int W = P.W, H = P.H;
    const int tx_n = (W + kTileW - 1) / kTileW;
    const int u0 = (local % tx_n) * kTileW, v0 = (local / tx_n) * kTileH;
    const int lx = threadIdx.x % kTileW, ly = threadIdx.x / kTileW;
    const int u = u0 + lx, v = v0 + ly;
    const bool cells = P.cg_key != nullptr;
    const int sz = P.sz;
    const int cx0 = u0 / sz, cy0 = v0 / sz;
    const int ncx = min(u0 + kTileW - 1, W - 1) / sz - cx0 + 1;
    const int ncy = min(v0 + kTileH - 1, H - 1) / sz - cy0 + 1;
    if (cells) {
        for (int i = threadIdx.x; i < ncx * ncy; i += blockDim.x) { s_g[i] = kNoKey; s_b[i] = kNoKey; }
        __syncthreads();
    }
    if (u < W && v < H) {
        const size_t p = (size_t)v * W + u;
        const bool om = (__ldg(P.omega + (size_t)v * ((W + 31) >> 5) + (u >> 5)) >> (u & 31)) & 1u;
        uint8_t m = om ? 1 : 0;
        int cost = -1;
        float d = 0.0f;
        if (om) {
            const int t = __ldg(P.planeidx + p);
            if (t >= 0) {
                const float a = __ldg(P.abc + 3 * t), bb = __ldg(P.abc + 3 * t + 1), c = __ldg(P.abc + 3 * t + 2);
                d = __fmaf_rn(a, (float)u, __fmaf_rn(bb, (float)v, c));
                const float kf = rintf(d);
                const float col = (float)u - kf;
                if (col >= 2.0f && col <= (float)(W - 3)) {
                    const int k = (int)kf;
                    cost = __popc(__ldg(P.cL + p) ^ __ldg(P.cR + p - k));
                    m |= 2;
                    if (cost < prm.t_lo) m |= 4;
                    if (cost > prm.t_hi) m |= 8;
                }
            }
        }
        if (P.first_pass) {
            const bool upd = cost >= 0 && cost < prm.t_hi;
            P.Df[p] = upd ? d : 0.0f;
            P.Cf[p] = (uint8_t)(upd ? cost : prm.t_hi);
        } else if (cost >= 0) {
            if (cost < (int)P.Cf[p]) {
                P.Df[p] = d;
                P.Cf[p] = (uint8_t)cost;
            }
        }
        if (P.mask) P.mask[p] = m;
        if (cells && (m & 12)) {
            const int lc = (v / sz - cy0) * ncx + (u / sz - cx0);
            if (m & 4) atomicMin(s_g + lc, ((uint32_t)cost << 27) | (uint32_t)p);
            if (m & 8) atomicMin(s_b + lc, ((uint32_t)(24 - cost) << 27) | (uint32_t)p);
        }
    }
    if (cells) {
        __syncthreads();
        for (int i = threadIdx.x; i < ncx * ncy; i += blockDim.x) {
            const size_t cell = (size_t)(cy0 + i / ncx) * P.Wc + (cx0 + i % ncx);
            if (s_g[i] != kNoKey) atomicMin(P.cg_key + cell, s_g[i]);
            if (s_b[i] != kNoKey) atomicMin(P.cb_key + cell, s_b[i]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_validate(PairBatch b, Params prm) {
#define BODY(P, l) validate_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// ---------------------------------------------------------------- resample + match (Alg. 4)
// One warp per cell: a C_g key becomes the interpolated disparity at its
// pixel; a C_b key is matched along its row by the same warp search.
__device__ __forceinline__ void resample_body(const PairDev& P, int local, const Params& prm) {
    const int cell = local * 8 + (threadIdx.x >> 5);
    if (cell >= P.Wc * P.Hc) return;
    const int lane = threadIdx.x & 31;
    const uint32_t gk = P.cg_key[cell], bk = P.cb_key[cell];
    if (lane == 0) {
        float d = __int_as_float(0x7fc00000);
        if (gk != kNoKey) {
            const uint32_t p = gk & kIdxMask;
            const int u = (int)(p % (uint32_t)P.W), v = (int)(p / (uint32_t)P.W);
            const int t = P.planeidx[p];
            d = __fmaf_rn(P.abc[3 * t], (float)u, __fmaf_rn(P.abc[3 * t + 1], (float)v, P.abc[3 * t + 2]));
        }
        P.cg_d[cell] = d;
    }
    int xd = -1;
    if (bk != kNoKey) {
        const uint32_t p = bk & kIdxMask;
        const int u = (int)(p % (uint32_t)P.W), v = (int)(p / (uint32_t)P.W);
        xd = warp_match(P.cL, P.cR, P.W, P.H, u, v, P.dmax, prm.t_lo, prm.margin);
    }
    if (lane == 0) P.x_d[cell] = xd;
}

__global__ void __launch_bounds__(256) k_resample(PairBatch b, Params prm) {
#define BODY(P, l) resample_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

__global__ void k_fill_u32(uint32_t* p, uint32_t value, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = value;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_census(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_census<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_fast_score(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_fast_score<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_fast_bins(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_fast_bins<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_match_kp(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_match_kp<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_raster_count(const PairBatch& b, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_raster_count<<<grid_for(b.total, 8), 256, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_raster_scan(const PairBatch& b, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_raster_scan<<<grid_for(b.total, 2), 1024, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_raster_fill(const PairBatch& b, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_raster_fill<<<grid_for(b.total, 8), 256, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_raster_pixels(const PairBatch& b, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_raster_pixels<<<grid_for(b.total, 8), 256, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_validate(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_validate<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_resample(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_resample<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_fill_u32(uint32_t* p, uint32_t value, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > sm_count() * 8) grid = sm_count() * 8;
    k_fill_u32<<<grid, 256, 0, s>>>(p, value, n);
    return cudaGetLastError();
}
cudaError_t launch_match_list(const uint32_t* cL, const uint32_t* cR, int W, int H, const int32_t* q, int n,
                              int dmax, const Params& prm, int32_t* out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_match_list<<<grid_for(cdiv(n, 8), 8), 256, 0, s>>>(cL, cR, W, H, q, n, dmax, prm, out);
    return cudaGetLastError();
}

}  // namespace stereo
