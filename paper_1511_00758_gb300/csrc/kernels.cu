// sm_103a kernels of the stereo hot path.  Every kernel is persistent over a
// work list: one launch may cover many frame pairs (PairBatch), with blocks
// striding over (pair, tile) items.  Nothing here waits on another block.
#include <cstdio>
#include <cstdlib>

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

static int validate_items(WorkKind k, const PairDev& p);

constexpr int kScanCols = 128;  // census and FAST score: a warp's strip of columns
constexpr int kScanRows = 14;   // and rows per strip item (a multiple of the 7-row ring; 7 on small launches)
__host__ __device__ __forceinline__ int scan_rows(const PairDev& p) { return p.scan_rows == 7 ? 7 : kScanRows; }

int work_items(WorkKind k, const PairDev& p) {
    switch (k) {
        case WK_CENSUS:
        case WK_FAST_SCORE: return cdiv(p.W, kScanCols) * cdiv(p.H, scan_rows(p));
        case WK_VALIDATE:
        case WK_VALIDATE_UNIT:
        case WK_VALIDATE_C4:
        case WK_VALIDATE_C2:
        case WK_VALIDATE_ANY:
        case WK_VALIDATE_MIXED: return validate_items(k, p);
        case WK_VALIDATE_BULK: return cdiv(p.W, 128) * cdiv(p.H, 8);
        case WK_FAST_BINS: return kFastBins;
        case WK_MATCH_KP: return cdiv((long long)kFastBins * p.K, 8);
        case WK_CLEAR: return cdiv((long long)p.W * p.H, 4096);
        case WK_FILL: return p.cg_key ? cdiv((long long)p.Wc * p.Hc, kFillCells) : 0;
        case WK_RASTER:
            if (p.mesh_raster) return 0;
            return (p.small_batch ? cdiv(p.n_batch, 8) : cdiv(p.n_small, 256)) + cdiv(p.raster_items, 8) +
                   (p.n_hull >= 0 ? cdiv(p.H, 8) : 0) + (p.cg_key ? cdiv((long long)p.Wc * p.Hc, kFillCells) : 0);
        case WK_RESAMPLE: return cdiv((long long)p.Wc * p.Hc, 256);
        default: return 0;
    }
}

void set_cell_size(PairDev& p, int sz) {
    p.sz = sz;
    p.sz_shift = -1;
    for (int s = 0; s < 31; s++)
        if ((1 << s) == sz) p.sz_shift = s;
    p.sz_magic = (uint32_t)(0xFFFFFFFFull / (unsigned)sz + 1ull);
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

// At least one block: a launch with no work still runs (one idle block), so
// a round's graph keeps the same nodes whatever its groups hold.
static int grid_for(int total, int per_sm) {
    int cap = sm_count() * per_sm;
    return total < 1 ? 1 : (total < cap ? total : cap);
}

// ---------------------------------------------------------------- census + Omega_I
// Census 5x5 (Sec. III-C) of L and R and the Omega_I bit map of L.  One warp per
// strip of 128 columns x kScanRows rows: lane l owns the four columns
// u0 + 4l .. u0 + 4l + 3 and slides down the strip keeping the rows it needs in
// registers, each row as three words (the lane's own four bytes and the four on
// either side, taken from the neighbouring lanes by shuffles, the strip's edge
// lanes loading theirs).  A row is read once per strip, as aligned words with a
// funnel shift for the row's misalignment; only the first and last rows of an
// image (where the aligned span would leave the buffer) are read byte by byte.
// Bytes outside the image read as 0: they are seen only by border pixels, whose
// outputs are fixed (code 0, not in Omega_I).


struct Row3 {
    uint32_t l, c, r;  // bytes u-4 .. u-1, u .. u+3, u+4 .. u+7 of the lane's columns u .. u+3
};

__device__ __forceinline__ uint32_t byte_at(const uint8_t* img, size_t n, long long i) {
    return i >= 0 && (size_t)i < n ? (uint32_t)__ldg(img + i) : 0u;
}

// A row's loads in flight: the three aligned words of the lane (fast) or the
// finished bytes (edge rows, read byte by byte).  issue_row() starts them,
// finish_row() (a row later, so the loads overlap a row of work) makes the Row3.
struct RowLoad {
    uint32_t a, b, c;
    int sh;     // the row's misalignment in bits; -1: a, b, c are already l, c, r
};

// Row v of img (W x H) around the lane's columns u0 + 4 lane ..; v and u0 warp-uniform.
__device__ __forceinline__ RowLoad issue_row(const uint8_t* img, int W, int H, int v, int u0, int lane) {
    RowLoad x{0u, 0u, 0u, -1};
    if (v < 0 || v >= H) return x;
    const size_t n = (size_t)W * H;
    const long long base = (long long)v * W + u0;  // byte offset of the strip's first column
    const uintptr_t a = (uintptr_t)(img + base), a0 = a & ~(uintptr_t)3;
    if (a0 >= (uintptr_t)img + 4 && a0 + 4 * 34 <= (uintptr_t)img + n) {  // words -1 .. 33 all inside
        const uint32_t* w = reinterpret_cast<const uint32_t*>(a0);
        x.a = __ldg(w + lane);
        x.b = __ldg(w + lane + 1);
        x.c = __ldg(w + (lane == 0 ? -1 : lane + 2));
        x.sh = (int)(a & 3) * 8;
    } else {
        const long long o = base + 4 * lane;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            x.a |= byte_at(img, n, o - 4 + j) << (8 * j);
            x.b |= byte_at(img, n, o + j) << (8 * j);
            x.c |= byte_at(img, n, o + 4 + j) << (8 * j);
        }
    }
    return x;
}

__device__ __forceinline__ Row3 finish_row(const RowLoad& x, int lane) {
    if (x.sh < 0) return Row3{x.a, x.b, x.c};  // warp-uniform
    Row3 y;
    y.c = __funnelshift_r(x.a, x.b, x.sh);
    const uint32_t edge = lane == 0 ? __funnelshift_r(x.c, x.a, x.sh) : __funnelshift_r(x.b, x.c, x.sh);
    const uint32_t up = __shfl_up_sync(0xffffffffu, y.c, 1), dn = __shfl_down_sync(0xffffffffu, y.c, 1);
    y.l = lane == 0 ? edge : up;
    y.r = lane == 31 ? edge : dn;
    return y;
}

// The four bytes at column offset dx (-3 .. 3) from the lane's columns.
__device__ __forceinline__ uint32_t shifted(const Row3& x, int dx) {
    return dx == -3 ? __funnelshift_r(x.l, x.c, 8) : dx == -2 ? __funnelshift_r(x.l, x.c, 16)
         : dx == -1 ? __funnelshift_r(x.l, x.c, 24) : dx == 0 ? x.c
         : dx == 1  ? __funnelshift_r(x.c, x.r, 8) : dx == 2 ? __funnelshift_r(x.c, x.r, 16)
                    : __funnelshift_r(x.c, x.r, 24);
}

// Census codes of the lane's four pixels from rows v-2 .. v+2 (ring slots s0 ..
// s0+4 mod 7).  A neighbour's four comparisons N < C are done at once on bytes:
// with H = 0x80 in every byte, d = (N | H) - (C & ~H) never borrows across bytes
// and its top bit is set when the low seven bits of N are >= those of C, so the
// top bit of (~N & C) | (~(N ^ C) & ~d) is N < C.  Neighbour k (raster order of
// the 5x5 window without its centre) lands in bit k of each pixel's code.
template <int S0>
__device__ __forceinline__ void census4(const Row3 (&ring)[7], uint32_t out[4]) {
    const uint32_t C = ring[(S0 + 2) % 7].c;
    const uint32_t Cl = C & 0x7F7F7F7Fu;
    uint32_t acc[3] = {0u, 0u, 0u};
    int k = 0;
#pragma unroll
    for (int dy = 0; dy < 5; dy++) {
#pragma unroll
        for (int dx = -2; dx <= 2; dx++) {
            if (dy == 2 && dx == 0) continue;
            const uint32_t N = shifted(ring[(S0 + dy) % 7], dx);
            const uint32_t d = (N | 0x80808080u) - Cl;
            const uint32_t lt = (~N & C) | (~(N ^ C) & ~d);  // top bit of each byte: N < C
            const int i = k & 7;
            acc[k >> 3] |= (lt >> (7 - i)) & (0x01010101u << i);
            k++;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const uint32_t lo = __byte_perm(acc[0], acc[1], (unsigned)(j | ((4 + j) << 4))) & 0xFFFFu;
        out[j] = lo | (__byte_perm(acc[2], 0u, 0x4440u | j) << 16);
    }
}

// One output row v of the strip: ring slot K + 3 holds row v (slots mod 7).
template <int K>
__device__ __forceinline__ void census_row(const PairDev& P, const Params& prm, const Row3 (&rl)[7],
                                           const Row3 (&rr)[7], int v, int u0, int lane) {
    const int W = P.W, H = P.H;
    const int ub = u0 + 4 * lane;
    uint32_t cl[4], cr[4] = {0u, 0u, 0u, 0u};
    census4<(K + 1) % 7>(rl, cl);
    if (P.cR) census4<(K + 1) % 7>(rr, cr);
    // Omega_I: |I(u+1) - I(u-1)| + |I(v+1) - I(v-1)| >= t_grad
    const uint32_t E = shifted(rl[(K + 3) % 7], 1), Wd = shifted(rl[(K + 3) % 7], -1);
    const uint32_t Sd = rl[(K + 4) % 7].c, Nd = rl[(K + 2) % 7].c;
    const bool row_in = v >= 2 && v < H - 2;
    unsigned om = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int u = ub + j;
        if (!row_in || u < 2 || u >= W - 2) {
            cl[j] = 0u;
            cr[j] = 0u;
        } else {
            const int gx = abs((int)((E >> (8 * j)) & 0xFFu) - (int)((Wd >> (8 * j)) & 0xFFu));
            const int gy = abs((int)((Sd >> (8 * j)) & 0xFFu) - (int)((Nd >> (8 * j)) & 0xFFu));
            om |= (unsigned)(gx + gy >= prm.t_grad) << j;
        }
    }
    const size_t p = (size_t)v * W + ub;
    if (ub < W) {
        const uintptr_t al = (P.cL ? (uintptr_t)(P.cL + p) : 0) | (P.cR ? (uintptr_t)(P.cR + p) : 0);
        if (ub + 3 < W && (al & 15) == 0) {
            if (P.cL) *reinterpret_cast<uint4*>(P.cL + p) = make_uint4(cl[0], cl[1], cl[2], cl[3]);
            if (P.cR) *reinterpret_cast<uint4*>(P.cR + p) = make_uint4(cr[0], cr[1], cr[2], cr[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++)
                if (ub + j < W) {
                    if (P.cL) P.cL[p + j] = cl[j];
                    if (P.cR) P.cR[p + j] = cr[j];
                }
        }
    }
    // each omega word: 32 columns from eight adjacent lanes
    unsigned bits = om << (4 * (lane & 7));
    bits |= __shfl_xor_sync(0xffffffffu, bits, 1);
    bits |= __shfl_xor_sync(0xffffffffu, bits, 2);
    bits |= __shfl_xor_sync(0xffffffffu, bits, 4);
    const int words = (W + 31) >> 5, wi = (u0 >> 5) + (lane >> 3);
    if ((lane & 7) == 0 && wi < words && P.omega) P.omega[(size_t)v * words + wi] = bits;
}

// One strip item of ROWS rows (a compile-time count, so the ring's turns unroll).
template <int ROWS>
__device__ __forceinline__ void census_item(const PairDev& P, const Params& prm, int local, int lane) {
    const int nsx = (P.W + kScanCols - 1) / kScanCols;
    const int u0 = (local % nsx) * kScanCols, v0 = (local / nsx) * ROWS;
    Row3 rl[7], rr[7];
    // slot (i + 3 + d) mod 7 holds row v0 + i + d: rows v0 - 3 .. v0 + 1 first, v0 + 2 in flight
#pragma unroll
    for (int k = 0; k < 5; k++) {
        rl[k] = finish_row(issue_row(P.L, P.W, P.H, v0 - 3 + k, u0, lane), lane);
        rr[k] = P.cR ? finish_row(issue_row(P.R, P.W, P.H, v0 - 3 + k, u0, lane), lane) : Row3{0u, 0u, 0u};
    }
    RowLoad nl = issue_row(P.L, P.W, P.H, v0 + 2, u0, lane);
    RowLoad nr = P.cR ? issue_row(P.R, P.W, P.H, v0 + 2, u0, lane) : RowLoad{0u, 0u, 0u, -1};
    for (int g = 0; g < ROWS / 7; g++) {
        const int vg = v0 + 7 * g;
        if (vg >= P.H) break;
        // row v: finish row v + 2 (issued a row ago), issue row v + 3, then row v's outputs
#define ROW(K)                                                                            \
    {                                                                                     \
        const int v = vg + K;                                                             \
        rl[(K + 5) % 7] = finish_row(nl, lane);                                           \
        if (P.cR) rr[(K + 5) % 7] = finish_row(nr, lane);                                 \
        nl = issue_row(P.L, P.W, P.H, v + 3, u0, lane);                                   \
        if (P.cR) nr = issue_row(P.R, P.W, P.H, v + 3, u0, lane);                         \
        if (v < P.H) census_row<K>(P, prm, rl, rr, v, u0, lane);                          \
    }
        ROW(0) ROW(1) ROW(2) ROW(3) ROW(4) ROW(5) ROW(6)
#undef ROW
    }
}

// Every pair of a launch takes the same strip rows (ROWS: 7 or kScanRows).
template <int ROWS>
__global__ void __launch_bounds__(256) k_census(PairBatch b, Params prm) {
    const int lane = threadIdx.x & 31;
    for (int item = blockIdx.x * 8 + (threadIdx.x >> 5); item < b.total; item += gridDim.x * 8) {
        const PairDev* Pp = &b.one;
        int local = item;
        if (b.pd) {
            const int pi = find_pair(b.work_off, b.npairs, item);
            Pp = b.pd + pi;
            local = item - __ldg(b.work_off + pi);
        }
        census_item<ROWS>(*Pp, prm, local, lane);
    }
}

// ---------------------------------------------------------------- FAST score
// FAST-9 on the radius-3 Bresenham circle (Sec. III-A, [rosten2006machine]),
// same tiling as the census with a 3-pixel halo.
// Circle offsets, folded to constants once the loop over i is unrolled.
__device__ constexpr int fast_dx(int i) {
    return i == 0 || i == 8 ? 0 : i == 1 || i == 7 ? 1 : i == 2 || i == 6 ? 2 : i >= 3 && i <= 5 ? 3
         : i == 9 || i == 15 ? -1 : i == 10 || i == 14 ? -2 : -3;
}
__device__ constexpr int fast_dy(int i) { return fast_dx((i + 12) & 15); }  // the same circle a quarter turn on

__device__ __forceinline__ bool has_run9(uint32_t m16) {
    uint32_t x = m16 | (m16 << 16);
    uint32_t r = x;
#pragma unroll
    for (int i = 1; i < 9; i++) r &= x >> i;
    return (r & 0xFFFFu) != 0;
}

// One output row w of a FAST strip (ring slot K + 3 holds row w, slots mod 7 hold
// rows w - 3 .. w + 3).  With t >= 0 a circle pixel q is brighter when
// q > min(p + t, 255) and darker when q < max(p - t, 0) (the clamps only remove
// comparisons that can never hold); both are tested on the lane's four pixels at
// once with the borrow-free byte compare of the census, and the results gathered
// into each pixel's two 16-bit masks.  The sums of the score are taken only for
// the pixels whose masks hold a run of nine.  A negative t keeps the per-pixel
// rule with brighter tested first.
template <int K>
__device__ __forceinline__ void fast_row(const PairDev& P, int t, const Row3 (&rl)[7], int w, int u0, int lane) {
    const int W = P.W, H = P.H;
    const int ub = u0 + 4 * lane;
    const uint32_t P4 = rl[(K + 3) % 7].c;
    bool corner[4];
    int score[4] = {0, 0, 0, 0};
    const bool row_in = w >= 3 && w < H - 3;
    if (t >= 0) {
        uint32_t HI = 0u, LO = 0u;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int p = (int)((P4 >> (8 * j)) & 0xFFu);
            HI |= (uint32_t)min(p + t, 255) << (8 * j);
            LO |= (uint32_t)max(p - t, 0) << (8 * j);
        }
        const uint32_t HIh = HI | 0x80808080u, LOl = LO & 0x7F7F7F7Fu;
        uint32_t bl = 0u, bh = 0u, dl = 0u, dh = 0u;  // bit i of pixel j's masks: byte j, bit i (i < 8) of *l
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const uint32_t Q = shifted(rl[(K + 3 + fast_dy(i) + 7) % 7], fast_dx(i));
            const uint32_t db = HIh - (Q & 0x7F7F7F7Fu);
            const uint32_t br = (~HI & Q) | (~(HI ^ Q) & ~db);  // top bit of each byte: HI < Q
            const uint32_t dd = (Q | 0x80808080u) - LOl;
            const uint32_t dk = (~Q & LO) | (~(Q ^ LO) & ~dd);  // top bit of each byte: Q < LO
            const int b = i & 7;
            if (i < 8) {
                bl |= (br >> (7 - b)) & (0x01010101u << b);
                dl |= (dk >> (7 - b)) & (0x01010101u << b);
            } else {
                bh |= (br >> (7 - b)) & (0x01010101u << b);
                dh |= (dk >> (7 - b)) & (0x01010101u << b);
            }
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int u = ub + j;
            const uint32_t mb = ((bl >> (8 * j)) & 0xFFu) | (((bh >> (8 * j)) & 0xFFu) << 8);
            const uint32_t md = ((dl >> (8 * j)) & 0xFFu) | (((dh >> (8 * j)) & 0xFFu) << 8);
            corner[j] = row_in && u >= 3 && u < W - 3 && (has_run9(mb) || has_run9(md));
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            if (!corner[j]) continue;
            const int p = (int)((P4 >> (8 * j)) & 0xFFu);
            int sb = 0, sd = 0;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int q = (int)((shifted(rl[(K + 3 + fast_dy(i) + 7) % 7], fast_dx(i)) >> (8 * j)) & 0xFFu);
                sb += max(q - p - t, 0);
                sd += max(p - q - t, 0);
            }
            score[j] = sb > sd ? sb : sd;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int u = ub + j;
            if (!row_in || u < 3 || u >= W - 3) continue;
            const int p = (int)((P4 >> (8 * j)) & 0xFFu);
            uint32_t mb = 0u, md = 0u;
            int sb = 0, sd = 0;
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int q = (int)((shifted(rl[(K + 3 + fast_dy(i) + 7) % 7], fast_dx(i)) >> (8 * j)) & 0xFFu);
                if (q > p + t) {
                    mb |= 1u << i;
                    sb += q - p - t;
                } else if (q < p - t) {
                    md |= 1u << i;
                    sd += p - q - t;
                }
            }
            if (has_run9(mb) || has_run9(md)) score[j] = sb > sd ? sb : sd;
        }
    }
    if (ub >= W) return;
    int16_t* out = P.fast_score + (size_t)w * W + ub;
    if (ub + 3 < W && ((uintptr_t)out & 7) == 0) {
        *reinterpret_cast<uint2*>(out) = make_uint2(((uint32_t)score[0] & 0xFFFFu) | ((uint32_t)score[1] << 16),
                                                    ((uint32_t)score[2] & 0xFFFFu) | ((uint32_t)score[3] << 16));
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (ub + j < W) out[j] = (int16_t)score[j];
    }
}

template <int ROWS>
__device__ __forceinline__ void fast_item(const PairDev& P, int t, int local, int lane) {
    const int nsx = (P.W + kScanCols - 1) / kScanCols;
    const int u0 = (local % nsx) * kScanCols, v0 = (local / nsx) * ROWS;
    Row3 rl[7];
    // slot (i + 3 + d) mod 7 holds row v0 + i + d: rows v0 - 3 .. v0 + 2 first, v0 + 3 in flight
#pragma unroll
    for (int k = 0; k < 6; k++) rl[k] = finish_row(issue_row(P.L, P.W, P.H, v0 - 3 + k, u0, lane), lane);
    RowLoad nl = issue_row(P.L, P.W, P.H, v0 + 3, u0, lane);
    for (int g = 0; g < ROWS / 7; g++) {
        const int vg = v0 + 7 * g;
        if (vg >= P.H) break;
#define ROW(K)                                                                            \
    {                                                                                     \
        const int w = vg + K;                                                             \
        rl[(K + 6) % 7] = finish_row(nl, lane);                                           \
        nl = issue_row(P.L, P.W, P.H, w + 4, u0, lane);                                   \
        if (w < P.H) fast_row<K>(P, t, rl, w, u0, lane);                                  \
    }
        ROW(0) ROW(1) ROW(2) ROW(3) ROW(4) ROW(5) ROW(6)
#undef ROW
    }
}

// FAST-9 scores of L in warp strips like the census: lane l owns four columns and
// slides down the strip with rows w - 3 .. w + 3 in its ring (row w + 4 in flight).
template <int ROWS>
__global__ void __launch_bounds__(256) k_fast_score(PairBatch b, Params prm) {
    const int lane = threadIdx.x & 31;
    for (int item = blockIdx.x * 8 + (threadIdx.x >> 5); item < b.total; item += gridDim.x * 8) {
        const PairDev* Pp = &b.one;
        int local = item;
        if (b.pd) {
            const int pi = find_pair(b.work_off, b.npairs, item);
            Pp = b.pd + pi;
            local = item - __ldg(b.work_off + pi);
        }
        fast_item<ROWS>(*Pp, prm.t_fast, local, lane);
    }
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
// The query's left census code cl is passed in.
__device__ __forceinline__ int warp_match_code(const uint32_t* __restrict__ cR, int W, int H, int u, int v,
                                               uint32_t cl, int dmax, int t_lo, int margin) {
    const int lane = threadIdx.x & 31;
    if (u < 2 || u >= W - 2 || v < 2 || v >= H - 2) return -1;
    const int dlim = min(dmax - 1, u - 2);
    const size_t p = (size_t)v * W + u;
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

// The same for a query whose left code is read here.
__device__ __forceinline__ int warp_match(const uint32_t* __restrict__ cL, const uint32_t* __restrict__ cR,
                                          int W, int H, int u, int v, int dmax, int t_lo, int margin) {
    if (u < 2 || u >= W - 2 || v < 2 || v >= H - 2) return -1;
    return warp_match_code(cR, W, H, u, v, __ldg(cL + (size_t)v * W + u), dmax, t_lo, margin);
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

// ---------------------------------------------------------------- raster + interpolation (Sec. III-B)
// Pixel -> triangle lookup table and the interpolated prior D_it (Eq. 3) by
// exact scan conversion.  A pixel (u, v) belongs to the positively oriented
// triangle when every edge function E(u, v) = A u + B v + C is > 0, or == 0
// on a top or left edge.  The rule partitions the hull: every pixel is
// written by exactly one triangle, in any order; pixels outside keep the
// cleared values (-1, NaN).  D_it = fma(a, u, fma(b, v, c)) in fp32.
// Small triangles (bounding box of at most kSmallArea pixels): a warp takes
// 32 of them and covers each box in turn with its 32 lanes.  Larger ones: one
// warp per work item of kRasterRows rows by kRasterCols columns of the box;
// one lane per row bounds the row by exact int32 floor/ceil division, then
// the lanes stride the columns of the item.
struct TriEdges {
    int x[3], y[3];
    int A[3], B[3], C[3], bias[3];
};

// Edge function of the directed edge a -> b (interior on its positive side)
// and the fill-rule bias: a pixel on the edge (E == 0) is kept only on a top
// or left edge.  Triangles and the hull use this one definition, so a hull
// edge decides every pixel exactly as the triangle behind it does.
__device__ __forceinline__ void edge_fn(int ax, int ay, int bx, int by, int& A, int& B, int& C, int& bias) {
    const int dx = bx - ax, dy = by - ay;
    A = -dy;
    B = dx;
    C = dy * ax - dx * ay;
    bias = ((dy == 0 && dx > 0) || dy < 0) ? 0 : 1;
}

__device__ __forceinline__ void tri_setup(const int32_t* __restrict__ tri_uv, int t, TriEdges& e) {
    const int32_t* q = tri_uv + 6 * (size_t)t;
    int x[3] = {__ldg(q), __ldg(q + 2), __ldg(q + 4)};
    int y[3] = {__ldg(q + 1), __ldg(q + 3), __ldg(q + 5)};
    const long long o = (long long)(x[1] - x[0]) * (y[2] - y[0]) - (long long)(y[1] - y[0]) * (x[2] - x[0]);
    if (o < 0) {  // positive orientation
        int s = x[1]; x[1] = x[2]; x[2] = s;
        s = y[1]; y[1] = y[2]; y[2] = s;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        e.x[k] = x[k];
        e.y[k] = y[k];
        edge_fn(x[k], y[k], x[(k + 1) % 3], y[(k + 1) % 3], e.A[k], e.B[k], e.C[k], e.bias[k]);
    }
}

__device__ __forceinline__ bool tri_is_small(const int32_t* __restrict__ q, int W, int H) {
    const int x0 = max(0, min(q[0], min(q[2], q[4]))), x1 = min(W - 1, max(q[0], max(q[2], q[4])));
    const int y0 = max(0, min(q[1], min(q[3], q[5]))), y1 = min(H - 1, max(q[1], max(q[3], q[5])));
    return x1 < x0 || y1 < y0 || (x1 - x0 + 1) * (y1 - y0 + 1) <= kSmallArea;
}

// Work items of a large triangle: 8-row by cols-column blocks of its clipped box.
__device__ __forceinline__ int tri_col_chunks(const int32_t* __restrict__ q, int W, int cols = kRasterCols) {
    const int x0 = max(0, min(q[0], min(q[2], q[4]))), x1 = min(W - 1, max(q[0], max(q[2], q[4])));
    return (x1 - x0) / cols + 1;
}
__device__ __forceinline__ int tri_chunks(const int32_t* __restrict__ q, int W, int H) {
    if (tri_is_small(q, W, H)) return 0;
    const int y0 = max(0, min(q[1], min(q[3], q[5])));
    const int y1 = min(H - 1, max(q[1], max(q[3], q[5])));
    return ((y1 - y0) / kRasterRows + 1) * tri_col_chunks(q, W);
}


// Small triangles, 32 to a warp: lane i sets triangle i up in shared memory;
// then the warp splits into groups of G lanes (G = the widest box of the 32,
// rounded up to a power of two, at most 32) and each group walks one box
// down its columns, G adjacent pixels per row, so the stores of a row are
// contiguous.  The bias is folded into C: a pixel is inside when the three
// edge values are all >= 0.
struct SmallTri {
    int A[3], B[3], C[3];
    int x0, y0, bw, bh;
    float a, b, c;
    int t;
};

__device__ __forceinline__ void raster_small_warp(const int32_t* __restrict__ tri_uv, const float* __restrict__ abc,
                                                  const int32_t* __restrict__ list, int n, int W, int H,
                                                  int32_t* __restrict__ pidx, float* __restrict__ dit,
                                                  SmallTri* __restrict__ s) {
    const int lane = threadIdx.x & 31;
    int bw = 0;
    if (lane < n) {
        const int t = __ldg(list + lane);
        TriEdges e;
        tri_setup(tri_uv, t, e);
        SmallTri q;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            q.A[k] = e.A[k];
            q.B[k] = e.B[k];
            q.C[k] = e.C[k] - e.bias[k];
        }
        const int x0 = max(0, min(e.x[0], min(e.x[1], e.x[2]))), x1 = min(W - 1, max(e.x[0], max(e.x[1], e.x[2])));
        const int y0 = max(0, min(e.y[0], min(e.y[1], e.y[2]))), y1 = min(H - 1, max(e.y[0], max(e.y[1], e.y[2])));
        q.x0 = x0;
        q.y0 = y0;
        q.bw = max(0, x1 - x0 + 1);
        q.bh = max(0, y1 - y0 + 1);
        q.a = q.b = q.c = 0.0f;
        if (dit) {  // planes are only read when D_it is written (abc may be null otherwise)
            q.a = __ldg(abc + 3 * t);
            q.b = __ldg(abc + 3 * t + 1);
            q.c = __ldg(abc + 3 * t + 2);
        }
        q.t = t;
        s[lane] = q;
        bw = q.bw;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) bw = max(bw, __shfl_xor_sync(0xffffffffu, bw, o));
    __syncwarp();
    const int lg = bw > 16 ? 5 : bw > 8 ? 4 : bw > 4 ? 3 : bw > 2 ? 2 : bw > 1 ? 1 : 0;
    const int G = 1 << lg, ng = 32 >> lg, lx = lane & (G - 1);
    for (int i = lane >> lg; i < n; i += ng) {
        const int A0 = s[i].A[0], A1 = s[i].A[1], A2 = s[i].A[2];
        const int B0 = s[i].B[0], B1 = s[i].B[1], B2 = s[i].B[2];
        const int C0 = s[i].C[0], C1 = s[i].C[1], C2 = s[i].C[2];
        const int x0 = s[i].x0, y0 = s[i].y0, tw = s[i].bw, th = s[i].bh, t = s[i].t;
        const float pa = s[i].a, pb = s[i].b, pc = s[i].c;
        for (int cx = lx; cx < tw; cx += G) {
            const int u = x0 + cx;
            int e0 = A0 * u + B0 * y0 + C0;
            int e1 = A1 * u + B1 * y0 + C1;
            int e2 = A2 * u + B2 * y0 + C2;
            const float uf = (float)u;
            float vf = (float)y0;
            size_t p = (size_t)y0 * W + u;
            for (int r = 0; r < th; r++) {
                if ((e0 | e1 | e2) >= 0) {
                    if (pidx) pidx[p] = t;
                    if (dit) dit[p] = __fmaf_rn(pa, uf, __fmaf_rn(pb, vf, pc));  // D_it = fma(a, u, fma(b, v, c))
                }
                e0 += B0;
                e1 += B1;
                e2 += B2;
                vf += 1.0f;
                p += W;
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ int floordiv32(int a, int b) {  // b > 0
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

__device__ __forceinline__ void raster_chunk_tc(const int32_t* __restrict__ tri_uv, const float* __restrict__ abc,
                                                int t, int item, int W, int H, int32_t* __restrict__ pidx,
                                                float* __restrict__ dit, int cols) {
    const int lane = threadIdx.x & 31;
    // item -> (row block, column block) of the triangle's clipped box
    const int ncol = tri_col_chunks(tri_uv + 6 * (size_t)t, W, cols);
    const int c = item / ncol, cc = item - c * ncol;
    TriEdges e;
    tri_setup(tri_uv, t, e);
    float pa = 0.0f, pb = 0.0f, pc = 0.0f;
    if (dit) {  // planes are only read when D_it is written (abc may be null otherwise)
        pa = __ldg(abc + 3 * t);
        pb = __ldg(abc + 3 * t + 1);
        pc = __ldg(abc + 3 * t + 2);
    }
    const int ymin = max(0, min(e.y[0], min(e.y[1], e.y[2])));
    const int ymax = min(H - 1, max(e.y[0], max(e.y[1], e.y[2])));
    const int v0 = ymin + c * kRasterRows;
    const int vr = v0 + (lane & (kRasterRows - 1));
    const int bx0 = max(0, min(e.x[0], min(e.x[1], e.x[2]))) + cc * cols;
    int lo = bx0, hi = min(W - 1, bx0 + cols - 1);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        // A u + B v + C >= bias  <=>  A u >= R
        const int R = e.bias[k] - e.B[k] * vr - e.C[k];
        if (e.A[k] > 0) lo = max(lo, -floordiv32(-R, e.A[k]));       // u >= ceil(R / A)
        else if (e.A[k] < 0) hi = min(hi, floordiv32(-R, -e.A[k]));  // u <= floor(R / A)
        else if (R > 0) hi = -1;
    }
    const int nrows = min(kRasterRows, ymax - v0 + 1);
    for (int r = 0; r < nrows; r++) {
        const int a = __shfl_sync(0xffffffffu, lo, r), b = __shfl_sync(0xffffffffu, hi, r);
        const int v = v0 + r;
        const float rowterm = __fmaf_rn(pb, (float)v, pc);  // D_it = fma(a, u, fma(b, v, c))
        int32_t* prow = pidx ? pidx + (size_t)v * W : nullptr;
        float* drow = dit ? dit + (size_t)v * W : nullptr;
        for (int u = a + lane; u <= b; u += 32) {
            if (prow) prow[u] = t;
            if (drow) drow[u] = __fmaf_rn(pa, (float)u, rowterm);
        }
    }
}

__device__ __forceinline__ void raster_clear_body(const PairDev& P, int local) {
    const size_t n = (size_t)P.W * P.H;
    const size_t base = (size_t)local * 4096;
    int32_t* pidx = P.planeidx;
    float* dit = P.Dit;
    const float qnan = __int_as_float(0x7fc00000);
    for (size_t i = base + 4 * threadIdx.x; i < base + 4096 && i < n; i += 4 * blockDim.x) {
        if (i + 4 <= n) {
            if (pidx) reinterpret_cast<int4*>(pidx)[i / 4] = make_int4(-1, -1, -1, -1);
            if (dit) reinterpret_cast<float4*>(dit)[i / 4] = make_float4(qnan, qnan, qnan, qnan);
        } else {
            for (size_t j = i; j < n; j++) {
                if (pidx) pidx[j] = -1;
                if (dit) dit[j] = qnan;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_raster_clear(PairBatch b) {
#define BODY(P, l) raster_clear_body(P, l)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// Pixels outside the convex hull of the support points, one warp per row.
// The hull is the union of the triangles, and with the fill rule a pixel is
// inside the hull exactly when it passes every hull edge, so on row v the
// covered pixels are the interval [lo, hi] cut by the hull edges; the pixels
// outside it get the cleared values (-1, NaN) and the triangles write the
// rest: every pixel is written once.
__device__ __forceinline__ void hull_row_clear(const int32_t* __restrict__ hull, int nh, int v, int W,
                                               int32_t* __restrict__ pidx, float* __restrict__ dit) {
    const int lane = threadIdx.x & 31;
    int lo = nh > 0 ? 0 : W, hi = W - 1;
    for (int j = lane; j < nh; j += 32) {
        const int4 h = __ldg(reinterpret_cast<const int4*>(hull) + j);
        int A, B, C, bias;
        edge_fn(h.x, h.y, h.z, h.w, A, B, C, bias);
        const int R = bias - B * v - C;  // A u + B v + C >= bias  <=>  A u >= R
        if (A > 0) lo = max(lo, -floordiv32(-R, A));
        else if (A < 0) hi = min(hi, floordiv32(-R, -A));
        else if (R > 0) lo = W;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lo = max(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = min(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    lo = min(lo, W);
    const float qnan = __int_as_float(0x7fc00000);
    int32_t* prow = pidx ? pidx + (size_t)v * W : nullptr;
    float* drow = dit ? dit + (size_t)v * W : nullptr;
    for (int u = lane; u < lo; u += 32) {
        if (prow) prow[u] = -1;
        if (drow) drow[u] = qnan;
    }
    for (int u = max(hi + 1, lo) + lane; u < W; u += 32) {
        if (prow) prow[u] = -1;
        if (drow) drow[u] = qnan;
    }
}

// Work of one pair: blocks of small triangles (8 warp batches each, or 256
// triangles when no batches are given), ceil(items / 8) blocks of
// large-triangle work items (one per warp), then, when the hull is given,
// ceil(H / 8) blocks of hull row clears, and, when the pair has cell records,
// blocks that reset kFillCells of them each for the validate's atomic minima
// (the raster runs just before it, so no launch of its own is needed).
__device__ __forceinline__ void fill_cells_range(const PairDev& P, int chunk) {
    const size_t n = (size_t)P.Wc * P.Hc;
    const size_t end = min(n, (size_t)(chunk + 1) * kFillCells);
    for (size_t i = (size_t)chunk * kFillCells + threadIdx.x; i < end; i += blockDim.x) {
        P.cg_key[i] = kNoKey;
        P.cb_key[i] = kNoKey;
    }
}

__device__ __forceinline__ void raster_body(const PairDev& P, int local, SmallTri* s) {
    const int nsb = P.small_batch ? (P.n_batch + 7) / 8 : (P.n_small + 255) / 256;
    const int ncb = (P.raster_items + 7) / 8;
    const int w = threadIdx.x >> 5;
    if (local < nsb) {
        int i0, n;
        if (P.small_batch) {  // host-cut batches of about equal box area
            const int bi = local * 8 + w;
            if (bi >= P.n_batch) return;
            i0 = __ldg(P.small_batch + bi);
            n = __ldg(P.small_batch + bi + 1) - i0;
        } else {
            i0 = local * 256 + w * 32;
            n = min(32, P.n_small - i0);
        }
        if (n > 0) raster_small_warp(P.tri_uv, P.abc, P.small_tri + i0, n, P.W, P.H, P.planeidx, P.Dit, s + w * 32);
        return;
    }
    if (local < nsb + ncb) {
        const int item = (local - nsb) * 8 + w;
        if (item >= P.raster_items) return;
        const int t = __ldg(P.item_tri + item);
        raster_chunk_tc(P.tri_uv, P.abc, t, item - __ldg(P.tri_rows + t), P.W, P.H, P.planeidx, P.Dit,
                        P.raster_cols > 0 ? P.raster_cols : kRasterCols);
        return;
    }
    const int nhb = P.n_hull >= 0 ? (P.H + 7) / 8 : 0;
    if (local < nsb + ncb + nhb) {
        const int v = (local - nsb - ncb) * 8 + w;
        if (v < P.H) hull_row_clear(P.hull, P.n_hull, v, P.W, P.planeidx, P.Dit);
        return;
    }
    fill_cells_range(P, local - nsb - ncb - nhb);
}

__global__ void __launch_bounds__(256) k_raster(PairBatch b) {
    __shared__ SmallTri s[256];
#define BODY(P, l) raster_body(P, l, s)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// Raster of meshes built on the device (the re-tessellation between passes):
// the lists and their sizes come from each pair's mesh header.  Work of a
// pair, in blocks: small triangles 256 to a block (32 per warp, in box width
// class order), large-triangle work items 8 to a block (one per warp; the
// item's triangle found by binary search of the item prefix), hull row
// clears 8 rows to a block, then the resets of the pass's cell records.
__device__ __forceinline__ int raster_mesh_blocks(const PairDev& P, const MeshDev& M) {
    const MeshHdr& h = *M.hdr;
    return (h.n_small + 255) / 256 + (h.n_items + 7) / 8 + (P.H + 7) / 8 +
           (P.cg_key ? (P.Wc * P.Hc + kFillCells - 1) / kFillCells : 0);
}

__global__ void __launch_bounds__(256) k_raster_mesh(const PairDev* __restrict__ pd, const MeshDev* __restrict__ md,
                                                     int np) {
    __shared__ SmallTri s[256];
    __shared__ int pre[kMeshBatch + 1];
    if (threadIdx.x < 32) {  // prefix of the pairs' block counts (np <= 64)
        const int l = threadIdx.x;
        int s0 = l < np ? raster_mesh_blocks(pd[l], md[l]) : 0;
        int s1 = l + 32 < np ? raster_mesh_blocks(pd[l + 32], md[l + 32]) : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x0 = __shfl_up_sync(0xffffffffu, s0, o), x1 = __shfl_up_sync(0xffffffffu, s1, o);
            if (l >= o) {
                s0 += x0;
                s1 += x1;
            }
        }
        const int tot0 = __shfl_sync(0xffffffffu, s0, 31);
        if (l == 0) pre[0] = 0;
        pre[l + 1] = s0;
        pre[l + 33] = tot0 + s1;
    }
    __syncthreads();
    const int total = pre[np];
    const int w = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int p = 0, hi = np - 1;
        while (p < hi) {
            const int mid = (p + hi + 1) >> 1;
            if (pre[mid] <= item) p = mid;
            else hi = mid - 1;
        }
        int local = item - pre[p];
        const PairDev& P = pd[p];
        const MeshDev& M = md[p];
        const int n_small = M.hdr->n_small, n_items = M.hdr->n_items;
        const int nsb = (n_small + 255) / 256, ncb = (n_items + 7) / 8, nhb = (P.H + 7) / 8;
        if (local < nsb) {
            const int i0 = local * 256 + w * 32;
            const int n = min(32, n_small - i0);
            if (n > 0) raster_small_warp(M.tri_uv, M.abc, M.small + i0, n, P.W, P.H, P.planeidx, P.Dit, s + w * 32);
            continue;
        }
        local -= nsb;
        if (local < ncb) {
            const int it = local * 8 + w;
            if (it < n_items) {
                int lo = 0, up = M.hdr->n_large - 1;  // the last large triangle whose first item is <= it
                while (lo < up) {
                    const int mid = (lo + up + 1) >> 1;
                    if (__ldg(M.lrows + mid) <= it) lo = mid;
                    else up = mid - 1;
                }
                raster_chunk_tc(M.tri_uv, M.abc, __ldg(M.large + lo), it - __ldg(M.lrows + lo), P.W, P.H, P.planeidx,
                                P.Dit, M.cols);
            }
            continue;
        }
        local -= ncb;
        if (local < nhb) {
            const int v = local * 8 + w;
            if (v < P.H) hull_row_clear(M.hull, M.hdr->n_hull, v, P.W, P.planeidx, P.Dit);
            continue;
        }
        fill_cells_range(P, local - nhb);
    }
}

cudaError_t launch_raster_mesh(const PairBatch& b, const MeshDev* md, cudaStream_t s) {
    if (b.npairs <= 0) return cudaSuccess;
    if (b.npairs > kMeshBatch || !b.pd) return cudaErrorInvalidValue;
    k_raster_mesh<<<sm_count() * 8, 256, 0, s>>>(b.pd, md, b.npairs);
    return cudaGetLastError();
}

// Device-built work lists for callers without a host copy of the triangles,
// in three launches over blocks of 1024 triangles: per-block totals, a scan
// of the block totals, then each block's exclusive scan written out.
// rows[T + 1]: work-item prefix of the large triangles; small[0..n): the small
// triangles in index order, small[T] = n; blk[2 * nblk]: block offsets.
constexpr int kListBlock = 1024;

__device__ __forceinline__ void tri_kind(const int32_t* __restrict__ tri_uv, int T, int W, int H, int t, int& chunks,
                                         int& small) {
    chunks = 0;
    small = 0;
    if (t < T) {
        const int32_t* q = tri_uv + 6 * (size_t)t;
        chunks = tri_chunks(q, W, H);
        small = tri_is_small(q, W, H) ? 1 : 0;
    }
}

// Block-wide inclusive scan of two counters (1024 threads).
__device__ __forceinline__ void block_scan2(int& a, int& b, int (*ws)[32]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int xa = __shfl_up_sync(0xffffffffu, a, o), xb = __shfl_up_sync(0xffffffffu, b, o);
        if (lane >= o) { a += xa; b += xb; }
    }
    if (lane == 31) { ws[0][w] = a; ws[1][w] = b; }
    __syncthreads();
    if (w == 0) {
        int sa = ws[0][lane], sb = ws[1][lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int xa = __shfl_up_sync(0xffffffffu, sa, o), xb = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) { sa += xa; sb += xb; }
        }
        ws[0][lane] = sa;
        ws[1][lane] = sb;
    }
    __syncthreads();
    if (w > 0) { a += ws[0][w - 1]; b += ws[1][w - 1]; }
}

__global__ void __launch_bounds__(kListBlock) k_lists_count(const int32_t* __restrict__ tri_uv, int T, int W, int H,
                                                            int32_t* __restrict__ blk) {
    __shared__ int ws[2][32];
    int c, s;
    tri_kind(tri_uv, T, W, H, blockIdx.x * kListBlock + threadIdx.x, c, s);
    block_scan2(c, s, ws);
    if (threadIdx.x == kListBlock - 1) {
        blk[2 * blockIdx.x] = c;
        blk[2 * blockIdx.x + 1] = s;
    }
}

__global__ void __launch_bounds__(kListBlock) k_lists_scan(int32_t* __restrict__ blk, int nblk, int T,
                                                           int32_t* __restrict__ rows, int32_t* __restrict__ small) {
    __shared__ int ws[2][32];
    int carry_c = 0, carry_s = 0;
    for (int base = 0; base < nblk; base += kListBlock) {  // exclusive scan of the block totals
        const int i = base + threadIdx.x;
        int c = i < nblk ? blk[2 * i] : 0, s = i < nblk ? blk[2 * i + 1] : 0;
        const int c0 = c, s0 = s;
        block_scan2(c, s, ws);
        if (i < nblk) {
            blk[2 * i] = carry_c + c - c0;
            blk[2 * i + 1] = carry_s + s - s0;
        }
        __syncthreads();  // every thread is done reading ws inside the scan
        if (threadIdx.x == kListBlock - 1) { ws[0][0] = c; ws[1][0] = s; }
        __syncthreads();
        carry_c += ws[0][0];
        carry_s += ws[1][0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        rows[T] = carry_c;
        small[T] = carry_s;
    }
}

__global__ void __launch_bounds__(kListBlock) k_lists_write(const int32_t* __restrict__ tri_uv, int T, int W, int H,
                                                            const int32_t* __restrict__ blk, int32_t* __restrict__ rows,
                                                            int32_t* __restrict__ small) {
    __shared__ int ws[2][32];
    const int t = blockIdx.x * kListBlock + threadIdx.x;
    int c, s;
    tri_kind(tri_uv, T, W, H, t, c, s);
    const int c0 = c, s0 = s;
    block_scan2(c, s, ws);
    if (t < T) {
        rows[t] = blk[2 * blockIdx.x] + c - c0;
        if (s0) small[blk[2 * blockIdx.x + 1] + s - 1] = t;
    }
}

__global__ void __launch_bounds__(256) k_raster_dev(const int32_t* __restrict__ tri_uv, const float* __restrict__ abc,
                                                    const int32_t* __restrict__ rows,
                                                    const int32_t* __restrict__ small, int T, int W, int H,
                                                    int32_t* __restrict__ pidx, float* __restrict__ dit) {
    __shared__ SmallTri s[256];
    const int nsmall = __ldg(small + T);
    const int w = threadIdx.x >> 5;
    for (int i0 = (blockIdx.x * 8 + w) * 32; i0 < nsmall; i0 += gridDim.x * 8 * 32)
        raster_small_warp(tri_uv, abc, small + i0, min(32, nsmall - i0), W, H, pidx, dit, s + w * 32);
    const int total = __ldg(rows + T);
    const int nw = gridDim.x * 8;
    for (int item = blockIdx.x * 8 + (threadIdx.x >> 5); item < total; item += nw) {
        int lo = 0, hi = T - 1;  // the last t with rows[t] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(rows + mid) <= item) lo = mid; else hi = mid - 1;
        }
        raster_chunk_tc(tri_uv, abc, lo, item - __ldg(rows + lo), W, H, pidx, dit, kRasterCols);
    }
}

// ---------------------------------------------------------------- fused validate (Alg. 2 + Alg. 3)
// Per pixel: Omega_I bit, plane lookup, fp32 interpolation (Eq. 3), census
// Hamming cost at the rounded disparity, the strict-< update of (D_f, C_f),
// the validation mask, and the per-cell C_g / C_b keys.
// Work unit: a strip of 32 columns by sh rows, one warp; lane l owns column
// u0 + l, so every row access of the warp is 128 contiguous bytes (no
// alignment assumption on W).  The warp first issues the loads of all its
// rows (D_it, left census, C_f, Omega_I), then the right-census gathers at
// u - rint(D_it), so each lane keeps up to eight independent chains in
// flight.  sh divides the cell side, so a strip lies in one row of cells: a
// lane keeps its running key minima in registers and the warp reduces them
// across the lanes of each cell once per strip (no shared memory, no block
// barrier), one global atomicMin per cell and strip.  Work item = one strip
// per warp.
constexpr int kVH = 8;  // also the bulk variant's tile height

__device__ __forceinline__ uint32_t cell_div(uint32_t x, int shift, uint32_t magic) {
    return shift >= 0 ? (x >> shift) : __umulhi(x, magic);
}

// Kernel variant (cell-side class) of a pair.  Strips are 8 rows high when
// there are no cells or the cell side is a power of two: 8 or more (one row
// of cells per strip), 4 or 2 (keys kept per row of cells inside the strip),
// 1 (every pixel committed where it is made).  Any other side takes the
// largest divisor of sz up to 8 as strip height.
__host__ __device__ __forceinline__ WorkKind validate_kind_of(const PairDev& p) {
    if (!p.cg_key) return WK_VALIDATE;
    if (p.sz_shift < 0) return WK_VALIDATE_ANY;
    if (p.sz >= 8) return WK_VALIDATE;
    if (p.sz == 4) return WK_VALIDATE_C4;
    if (p.sz == 2) return WK_VALIDATE_C2;
    return WK_VALIDATE_UNIT;
}

__host__ __device__ __forceinline__ int validate_strip_rows(const PairDev& p) {
    const WorkKind k = validate_kind_of(p);
    if (k == WK_VALIDATE_C4) return 4;  // a strip holds one row of cells
    if (k == WK_VALIDATE_C2) return 2;
    if (k != WK_VALIDATE_ANY) return 8;
    for (int h = 8; h > 1; h--)
        if (p.sz % h == 0) return h;
    return 1;
}

WorkKind validate_kind(const PairDev& p) { return validate_kind_of(p); }

static int validate_items(WorkKind k, const PairDev& p) {
    if (k != WK_VALIDATE_MIXED && validate_kind(p) != k) return 0;
    return cdiv(p.W, 32) * cdiv(p.H, validate_strip_rows(p));
}

// Commits the lanes' key minima of one row of cells: the lanes of a cell are
// contiguous; the cell's first lane commits.  Every lane of the warp calls it.
// Power-of-two sides: cells are aligned groups of min(sz, 32) lanes, reduced
// by butterfly shuffles.  Other sides: a segmented suffix minimum keyed on
// the cell column.
template <bool GENERIC>
__device__ __forceinline__ void commit_cells(uint32_t kg, uint32_t kb, int cx, int cy, int lane, bool lane_in,
                                             int sz, int Wc, uint32_t* __restrict__ cg, uint32_t* __restrict__ cb) {
    bool lead;
    if (!GENERIC) {
        const int seg = min(sz, 32);
        for (int o = 1; o < seg; o <<= 1) {
            kg = min(kg, __shfl_xor_sync(0xffffffffu, kg, o));
            kb = min(kb, __shfl_xor_sync(0xffffffffu, kb, o));
        }
        lead = (lane & (seg - 1)) == 0;
    } else {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t g2 = __shfl_down_sync(0xffffffffu, kg, o);
            const uint32_t b2 = __shfl_down_sync(0xffffffffu, kb, o);
            const int c2 = __shfl_down_sync(0xffffffffu, cx, o);
            if (lane + o < 32 && c2 == cx) {
                kg = min(kg, g2);
                kb = min(kb, b2);
            }
        }
        const int cprev = __shfl_up_sync(0xffffffffu, cx, 1);  // every lane takes part
        lead = lane == 0 || cprev != cx;
    }
    if (lead && lane_in) {
        const int cell = cy * Wc + cx;
        if (kg != kNoKey) atomicMin(cg + cell, kg);
        if (kb != kNoKey) atomicMin(cb + cell, kb);
    }
}

// Reduces keys over aligned groups of seg lanes (a power-of-two cell side)
// and commits from each group's first lane.  Every lane of the warp calls it.
__device__ __forceinline__ void commit_p2(uint32_t kg, uint32_t kb, int lane, bool in, int seg, int cell,
                                          uint32_t* __restrict__ cg, uint32_t* __restrict__ cb) {
    for (int o = 1; o < seg; o <<= 1) {
        kg = min(kg, __shfl_xor_sync(0xffffffffu, kg, o));
        kb = min(kb, __shfl_xor_sync(0xffffffffu, kb, o));
    }
    if ((lane & (seg - 1)) == 0 && in) {
        if (kg != kNoKey) atomicMin(cg + cell, kg);
        if (kb != kNoKey) atomicMin(cb + cell, kb);
    }
}

// A pair's fields as the strip kernels read them.  Batches pass up to
// kVBatch of them by value in the kernel parameters (constant bank), so the
// compiler can reload a field where it is used instead of holding it in a
// register for the whole strip: measured about 30% faster than descriptors
// in global memory.
struct VDesc {
    const uint32_t* omega;
    const float* dit;
    const uint32_t* cL;
    const uint32_t* cR;
    float* Df;
    uint8_t* Cf;
    uint8_t* mask;
    uint32_t* cg;
    uint32_t* cb;
    int W, H, first, sz, shift, Wc, sh, kind;
    uint32_t magic;
};

struct VBatch {
    VDesc d[kVBatch];
    int off[kVBatch + 1];  // exclusive prefix of the pairs' strips
    int npairs, total;
};

// Strip s (32 columns x ROWS rows) of a pair whose cell side is a power of
// two (or that has no cells).  NCR: rows of cells inside the strip; the keys
// of row of cells c live in kg_c / kb_c.  4- and 2-pixel cells take strips of
// 4 and 2 rows (one row of cells each): two or four rows of cells in an
// 8-row strip measured 1.4-1.5 times slower (4096x4096: 167 and 172 us
// against 122 and 117).  UNIT: 1-pixel cells, every key committed where it
// is made.  (The one-pass row loop and the branch-form key updates are kept
// as written: equivalent forms measured up to 2 times slower.)
template <int NCR, bool UNIT, int ROWS = 8>
__device__ __forceinline__ void validate_strip_p2(const VDesc& a, int s, int t_lo, int t_hi) {
    constexpr int kRows = ROWS, RB = ROWS, RPC = kRows / NCR;
    const int W = a.W, H = a.H, shift = a.shift, first = a.first, sz = a.sz;
    const int sx_n = (W + 31) / 32;
    const int lane = threadIdx.x & 31;
    const bool cells = a.cg != nullptr;
    const int u0 = (s % sx_n) * 32, v0 = (s / sx_n) * kRows;
    const int u = u0 + lane;
    const bool in = u < W;
    const int uc = min(u, W - 1);
    uint32_t kg0 = kNoKey, kb0 = kNoKey, kg1 = kNoKey, kb1 = kNoKey;
    uint32_t kg2 = kNoKey, kb2 = kNoKey, kg3 = kNoKey, kb3 = kNoKey;
    const int nrows = min(kRows, H - v0);
#pragma unroll
    for (int r0 = 0; r0 < kRows; r0 += RB) {
        float d[RB];
        uint32_t cl[RB];
        uint32_t cfw[(RB + 3) / 4] = {};  // C_f bytes, four to a register
        uint32_t omb = 0;                 // Omega_I bit of each row
#pragma unroll
        for (int r = 0; r < RB; r++) {  // first level: every row's independent loads
            const int v = v0 + r0 + r;
            const bool ok = in && (r0 + r) < nrows;
            const int p = v * W + uc;  // pixel indices fit in 27 bits
            const uint32_t ow = (r0 + r) < nrows ? __ldg(a.omega + v * sx_n + (u0 >> 5)) : 0u;
            d[r] = ok ? __ldg(a.dit + p) : __int_as_float(0x7fc00000);
            cl[r] = ok ? __ldg(a.cL + p) : 0u;
            if (!first && ok) cfw[r >> 2] |= (uint32_t)a.Cf[p] << (8 * (r & 3));
            if (ok) omb |= ((ow >> lane) & 1u) << r;
        }
        int cost[RB];
#pragma unroll
        for (int r = 0; r < RB; r++) {  // second level: the right census at u - rint(D_it)
            const int v = v0 + r0 + r;
            const float col = (float)u - rintf(d[r]);  // NaN outside the mesh: not evaluated
            cost[r] = -1;
            if (((omb >> r) & 1u) && col >= 2.0f && col <= (float)(W - 3))
                cost[r] = __popc(cl[r] ^ __ldg(a.cR + v * W + (int)col));
        }
#pragma unroll
        for (int r = 0; r < RB; r++) {
            const int v = v0 + r0 + r;
            if (!in || (r0 + r) >= nrows) continue;
            const int p = v * W + u;
            const int cj = cost[r];
            uint8_t m = (omb >> r) & 1u;
            if (cj >= 0) m |= 2 | (cj < t_lo ? 4 : 0) | (cj > t_hi ? 8 : 0);
            if (first) {
                const bool upd = cj >= 0 && cj < t_hi;
                a.Df[p] = upd ? d[r] : 0.0f;
                a.Cf[p] = (uint8_t)(upd ? cj : t_hi);
            } else if (cj >= 0 && cj < (int)((cfw[r >> 2] >> (8 * (r & 3))) & 0xFFu)) {
                a.Df[p] = d[r];
                a.Cf[p] = (uint8_t)cj;
            }
            a.mask[p] = m;  // required (a null check here measured about 20% slower)
            if (cells) {
                const uint32_t pk = (uint32_t)p;
                if (UNIT) {
                    const int cell = v * a.Wc + u;
                    if (cj >= 0 && cj < t_lo) atomicMin(a.cg + cell, ((uint32_t)cj << 27) | pk);
                    if (cj > t_hi) atomicMin(a.cb + cell, ((uint32_t)(24 - cj) << 27) | pk);
                } else {
                    const int c = (r0 + r) / RPC;  // a constant once the loop is unrolled
                    if (cj >= 0 && cj < t_lo) {
                        const uint32_t k = ((uint32_t)cj << 27) | pk;
                        if (c == 0) kg0 = min(kg0, k);
                        else if (c == 1) kg1 = min(kg1, k);
                        else if (c == 2) kg2 = min(kg2, k);
                        else kg3 = min(kg3, k);
                    }
                    if (cj > t_hi) {
                        const uint32_t k = ((uint32_t)(24 - cj) << 27) | pk;
                        if (c == 0) kb0 = min(kb0, k);
                        else if (c == 1) kb1 = min(kb1, k);
                        else if (c == 2) kb2 = min(kb2, k);
                        else kb3 = min(kb3, k);
                    }
                }
            }
        }
    }
    if (cells && !UNIT) {  // cells are aligned groups of min(sz, 32) lanes
        const int seg = min(sz, 32);
        const int cell = (v0 >> shift) * a.Wc + (u >> shift);
        commit_p2(kg0, kb0, lane, in, seg, cell, a.cg, a.cb);
        if (NCR > 1 && RPC < nrows) commit_p2(kg1, kb1, lane, in, seg, cell + a.Wc, a.cg, a.cb);
        if (NCR > 2 && 2 * RPC < nrows) commit_p2(kg2, kb2, lane, in, seg, cell + 2 * a.Wc, a.cg, a.cb);
        if (NCR > 3 && 3 * RPC < nrows) commit_p2(kg3, kb3, lane, in, seg, cell + 3 * a.Wc, a.cg, a.cb);
    }
}

// Strip s (32 columns x a.sh rows) of a pair whose cell side is not a power
// of two; a.sh divides sz, so the strip lies in one row of cells.
__device__ __forceinline__ void validate_strip_any(const VDesc& a, int s, int t_lo, int t_hi) {
    const int W = a.W, first = a.first, sh = a.sh;
    const int sx_n = (W + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int u0 = (s % sx_n) * 32, v0 = (s / sx_n) * sh;
    const int u = u0 + lane;
    const bool in = u < W;
    const int uc = min(u, W - 1);
    const int nrows = min(sh, a.H - v0);
    uint32_t kg = kNoKey, kb = kNoKey;
    float d[8];
    uint32_t cl[8];
    uint32_t cfw[2] = {};
    uint32_t omb = 0;
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const int v = v0 + r;
        const bool ok = in && r < nrows;
        const int p = v * W + uc;
        const uint32_t ow = r < nrows ? __ldg(a.omega + v * sx_n + (u0 >> 5)) : 0u;
        d[r] = ok ? __ldg(a.dit + p) : __int_as_float(0x7fc00000);
        cl[r] = ok ? __ldg(a.cL + p) : 0u;
        if (!first && ok) cfw[r >> 2] |= (uint32_t)a.Cf[p] << (8 * (r & 3));
        if (ok) omb |= ((ow >> lane) & 1u) << r;
    }
    int cost[8];
#pragma unroll
    for (int r = 0; r < 8; r++) {
        const float col = (float)u - rintf(d[r]);
        cost[r] = -1;
        if (((omb >> r) & 1u) && col >= 2.0f && col <= (float)(W - 3))
            cost[r] = __popc(cl[r] ^ __ldg(a.cR + (v0 + r) * W + (int)col));
    }
#pragma unroll
    for (int r = 0; r < 8; r++) {
        if (!in || r >= nrows) continue;
        const int p = (v0 + r) * W + u;
        const int cj = cost[r];
        uint8_t m = (omb >> r) & 1u;
        if (cj >= 0) m |= 2 | (cj < t_lo ? 4 : 0) | (cj > t_hi ? 8 : 0);
        if (first) {
            const bool upd = cj >= 0 && cj < t_hi;
            a.Df[p] = upd ? d[r] : 0.0f;
            a.Cf[p] = (uint8_t)(upd ? cj : t_hi);
        } else if (cj >= 0 && cj < (int)((cfw[r >> 2] >> (8 * (r & 3))) & 0xFFu)) {
            a.Df[p] = d[r];
            a.Cf[p] = (uint8_t)cj;
        }
        a.mask[p] = m;
        if (a.cg) {
            if (cj >= 0 && cj < t_lo) kg = min(kg, ((uint32_t)cj << 27) | (uint32_t)p);
            if (cj > t_hi) kb = min(kb, ((uint32_t)(24 - cj) << 27) | (uint32_t)p);
        }
    }
    if (a.cg)
        commit_cells<true>(kg, kb, (int)cell_div(uc, a.shift, a.magic), (int)cell_div(v0, a.shift, a.magic), lane, in,
                           a.sz, a.Wc, a.cg, a.cb);
}

// Strip s of descriptor a under its own variant (MIXED) or the kernel's (KIND).
template <int KIND>
__device__ __forceinline__ void validate_dispatch(const VDesc& a, int s, const Params& prm) {
    switch (KIND == WK_VALIDATE_MIXED ? a.kind : KIND) {
        case WK_VALIDATE: validate_strip_p2<1, false>(a, s, prm.t_lo, prm.t_hi); break;
        case WK_VALIDATE_UNIT: validate_strip_p2<1, true>(a, s, prm.t_lo, prm.t_hi); break;
        case WK_VALIDATE_C4: validate_strip_p2<1, false, 4>(a, s, prm.t_lo, prm.t_hi); break;
        case WK_VALIDATE_C2: validate_strip_p2<1, false, 2>(a, s, prm.t_lo, prm.t_hi); break;
        default: validate_strip_any(a, s, prm.t_lo, prm.t_hi); break;
    }
}

// Warps stride over the batch's strips; each strip finds its pair in the
// batch's prefix table (kernel parameters).
// The 4- and 2-row strips of 4- and 2-pixel cells fit 32 registers: eight blocks an SM.
template <int KIND>
__global__ void __launch_bounds__(256, (KIND == WK_VALIDATE_C4 || KIND == WK_VALIDATE_C2) ? 8 : 4)
    k_validate(const __grid_constant__ VBatch b, Params prm) {
    const int nw = gridDim.x * (blockDim.x >> 5);
    if (b.npairs == 1) {  // one pair: its fields are fixed constant-bank operands
        for (int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < b.total; s += nw)
            validate_dispatch<KIND>(b.d[0], s, prm);
        return;
    }
    for (int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < b.total; s += nw) {
        int lo = 0, hi = b.npairs - 1;  // the last pair whose first strip is <= s
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.off[mid] <= s) lo = mid;
            else hi = mid - 1;
        }
        validate_dispatch<KIND>(b.d[lo], s - b.off[lo], prm);
    }
}

// ---------------------------------------------------------------- fused validate: bulk-copy pipeline
// The same computation as k_validate, organised for Blackwell's asynchronous
// bulk copies.  Persistent blocks of one producer warp and eight consumer
// warps (one per tile row) share a ring of kBS shared-memory stages guarded
// by mbarriers.  Per tile the producer bulk-copies (cp.async.bulk) each row's
// D_it, left census, C_f and Omega_I words into a stage; when they land it
// takes the row's range of right-census columns u - rint(D_it) over the
// evaluable pixels and bulk-copies that window of the right census too.  The
// consumers then read every input from shared memory; a row whose column
// range is wider than the window, and the last bytes of a buffer (copies stop
// at the last 16-byte boundary inside it), fall back to global loads.
// Every mbarrier wait is bounded: on timeout the thread sets *prm.err and
// leaves, and the producer first waits (bounded) for its own copies.
constexpr int kBS = 4;                       // ring stages
constexpr int kVW = 128, kVJ = kVW / 32;      // tile width (pixels), pixels per lane
constexpr int kMaxLocalCells = kVW * kVH;    // cells of one tile at most (1-pixel cells)
constexpr int kBRowD = 136;                  // 4-byte words per staged D_it / cL row
constexpr int kBRowF = 160;                  // bytes per staged C_f row
constexpr int kBRowO = 8;                    // words per staged Omega_I row
constexpr int kBRowR = 264;                  // words per staged right-census window row
constexpr int kBWinMax = kBRowR - 8;         // widest column range staged
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a bounded wait gives up after one second

// Pair descriptor and local work index of a batch item.
__device__ __forceinline__ const PairDev& item_pair(const PairBatch& b, int item, int& local) {
    if (b.pd) {
        const int pi = find_pair(b.work_off, b.npairs, item);
        local = item - __ldg(b.work_off + pi);
        return b.pd[pi];
    }
    local = item;
    return b.one;
}

struct BulkRowMeta {
    int d_off, d_cnt;   // staged D_it / cL: element of pixel u0, elements present
    int f_off, f_cnt;   // staged C_f bytes
    int o_off, o_cnt;   // staged Omega_I words
    int r_base, r_cnt;  // right census: global column of element 0 (-1: no window), elements present
};

struct __align__(16) BulkStage {
    float d[kVH][kBRowD];
    uint32_t cl[kVH][kBRowD];
    uint32_t cr[kVH][kBRowR];
    uint8_t cf[kVH][kBRowF];
    uint32_t om[kVH][kBRowO];
    BulkRowMeta meta[kVH];
};

struct __align__(16) BulkSmem {
    BulkStage st[kBS];
    uint32_t g[2][kMaxLocalCells], b[2][kMaxLocalCells];
    unsigned long long full1[kBS], full2[kBS], empty[kBS];
    unsigned long long cdone[2];  // consumer warps finished their cell minima (per cell buffer)
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the completion of the phase with the given parity: gives
// up (false) after kWaitLimitNs of wall time on the GPU's global timer, so
// the bound does not depend on how long one poll takes.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_test_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned i = 0;; i++) {
        if (mbar_test_wait(bar, parity)) return true;
        if (i > 32) {
            __nanosleep(64);
            if (global_ns() - t0 > kWaitLimitNs) return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

struct BulkCopy {
    const void* src;
    void* dst;
    unsigned bytes;
};

// Plan the copy of elements [e0, e0 + n) of a buffer of ntot elements of es
// bytes (16-byte aligned base) into dst: the 16-byte aligned span around them,
// never past the last 16-byte boundary inside the buffer.
__device__ __forceinline__ void plan_row(const void* base, size_t ntot, int es, size_t e0, int n, void* dst, int& off,
                                         int& cnt, BulkCopy* cps, int& ncp) {
    const uintptr_t b = (uintptr_t)base;
    const uintptr_t s = b + e0 * es, e = b + (e0 + n) * es;
    const uintptr_t as = s & ~(uintptr_t)15;
    uintptr_t ae = (e + 15) & ~(uintptr_t)15;
    const uintptr_t lim = (b + ntot * es) & ~(uintptr_t)15;
    if (ae > lim) ae = lim;
    off = (int)((s - as) / es);
    cnt = 0;
    if (n <= 0 || ae <= as) return;
    cnt = (int)((ae - as) / es);
    cps[ncp].src = (const void*)as;
    cps[ncp].dst = dst;
    cps[ncp].bytes = (unsigned)(ae - as);
    ncp++;
}

__device__ __forceinline__ void bulk_producer(const PairBatch& b, const Params& prm, BulkSmem& sm) {
    const int lane = threadIdx.x & 31;
    if (prm.withhold) return;  // testing: no copy is issued, no stage released, so the consumers' waits run out
    int k = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < b.total; item += gridDim.x, k++) {
        const int s = k % kBS;
        const unsigned use = (unsigned)(k / kBS);
        if (!mbar_wait(&sm.empty[s], (use & 1u) ^ 1u)) { ok = false; break; }
        int local;
        const PairDev& P = item_pair(b, item, local);
        const int W = P.W, H = P.H;
        const size_t N = (size_t)W * H;
        const int words = (W + 31) >> 5;
        const int tx_n = (W + kVW - 1) / kVW;
        const int u0 = (local % tx_n) * kVW, v0 = (local / tx_n) * kVH;
        BulkStage& st = sm.st[s];
        // phase A: lane r < 8 plans row r's first-level copies
        BulkCopy cps[4];
        int ncp = 0;
        unsigned bytes = 0;
        if (lane < kVH) {
            const int r = lane, v = v0 + r;
            BulkRowMeta m{};
            if (v < H) {
                const int n = min(kVW, W - u0);
                const size_t e0 = (size_t)v * W + u0;
                plan_row(P.Dit, N, 4, e0, n, st.d[r], m.d_off, m.d_cnt, cps, ncp);
                int o2, c2;
                plan_row(P.cL, N, 4, e0, n, st.cl[r], o2, c2, cps, ncp);
                m.d_cnt = min(m.d_cnt, c2);  // the two planned spans coincide in position
                if (!P.first_pass) plan_row(P.Cf, N, 1, e0, n, st.cf[r], m.f_off, m.f_cnt, cps, ncp);
                plan_row(P.omega, (size_t)H * words, 4, (size_t)v * words + (u0 >> 5), min(kVJ, words - (u0 >> 5)),
                         st.om[r], m.o_off, m.o_cnt, cps, ncp);
            }
            st.meta[r] = m;
            for (int i = 0; i < ncp; i++) bytes += cps[i].bytes;
        }
        const unsigned total = __reduce_add_sync(0xffffffffu, bytes);
        if (lane == 0) mbar_arrive_expect_tx(&sm.full1[s], total);
        __syncwarp();
        for (int i = 0; i < ncp; i++) bulk_g2s(cps[i].dst, cps[i].src, cps[i].bytes, &sm.full1[s]);
        // phase B: once the first-level rows landed, stage each row's right-census window
        if (!mbar_wait(&sm.full1[s], use & 1u)) { ok = false; break; }
        int my_lo = 0x7fffffff, my_hi = -1;
        for (int r = 0; r < kVH; r++) {
            const int v = v0 + r;
            int lo = 0x7fffffff, hi = -1;
            if (v < H) {
                const BulkRowMeta& m = st.meta[r];
#pragma unroll
                for (int j = 0; j < kVJ; j++) {
                    const int u = u0 + lane + 32 * j;
                    if (u >= W) continue;
                    const int oi = m.o_off + j;
                    const uint32_t ow = oi < m.o_cnt ? st.om[r][oi] : __ldg(P.omega + (size_t)v * words + (u0 >> 5) + j);
                    if (!((ow >> lane) & 1u)) continue;
                    const int di = m.d_off + lane + 32 * j;
                    const float d = di < m.d_cnt ? st.d[r][di] : __ldg(P.Dit + (size_t)v * W + u);
                    const float col = (float)u - rintf(d);
                    if (col >= 2.0f && col <= (float)(W - 3)) {
                        lo = min(lo, (int)col);
                        hi = max(hi, (int)col);
                    }
                }
            }
            lo = __reduce_min_sync(0xffffffffu, lo);
            hi = __reduce_max_sync(0xffffffffu, hi);
            if (lane == r) { my_lo = lo; my_hi = hi; }
        }
        ncp = 0;
        bytes = 0;
        if (lane < kVH) {
            const int r = lane, v = v0 + r;
            BulkRowMeta& m = st.meta[r];
            m.r_base = -1;
            m.r_cnt = 0;
            if (v < H && my_hi >= my_lo && my_hi - my_lo + 1 <= kBWinMax) {
                int off;
                plan_row(P.cR, N, 4, (size_t)v * W + my_lo, my_hi - my_lo + 1, st.cr[r], off, m.r_cnt, cps, ncp);
                m.r_base = my_lo - off;
            }
            for (int i = 0; i < ncp; i++) bytes += cps[i].bytes;
        }
        __syncwarp();  // row metadata written before the release below
        const unsigned total2 = __reduce_add_sync(0xffffffffu, bytes);
        if (lane == 0) mbar_arrive_expect_tx(&sm.full2[s], total2);
        __syncwarp();
        for (int i = 0; i < ncp; i++) bulk_g2s(cps[i].dst, cps[i].src, cps[i].bytes, &sm.full2[s]);
    }
    // drain: the copies this warp issued for the last stages land before it leaves
    for (int j = max(0, k - kBS); j < k; j++) {
        const int s = j % kBS;
        const unsigned use = (unsigned)(j / kBS);
        mbar_wait(&sm.full1[s], use & 1u);
        mbar_wait(&sm.full2[s], use & 1u);
    }
    if (!ok && lane == 0 && prm.err) atomicExch(prm.err, 1);
}

__device__ __forceinline__ void bulk_consumer(const PairBatch& b, const Params& prm, BulkSmem& sm, int r) {
    const int lane = threadIdx.x & 31;
    const int ct = threadIdx.x - 32;  // consumer thread index, 0..255
    const int t_lo = prm.t_lo, t_hi = prm.t_hi;
    int k = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < b.total; item += gridDim.x, k++) {
        const int s = k % kBS;
        const unsigned use = (unsigned)(k / kBS);
        if (!mbar_wait(&sm.full2[s], use & 1u)) { ok = false; break; }
        int local;
        const PairDev& P = item_pair(b, item, local);
        const int W = P.W, H = P.H, Wc = P.Wc, first = P.first_pass, sz = P.sz, shift = P.sz_shift;
        const uint32_t magic = P.sz_magic;
        const int words = (W + 31) >> 5;
        const int tx_n = (W + kVW - 1) / kVW;
        const int u0 = (local % tx_n) * kVW, v0 = (local / tx_n) * kVH;
        const int v = v0 + r;
        const bool cells = P.cg_key != nullptr;
        const int cb = k & 1;
        const int cx0 = cell_div(u0, shift, magic), cy0 = cell_div(v0, shift, magic);
        const int ncx = cell_div(min(u0 + kVW - 1, W - 1), shift, magic) - cx0 + 1;
        const int ncy = cell_div(min(v0 + kVH - 1, H - 1), shift, magic) - cy0 + 1;
        const BulkStage& st = sm.st[s];
        if (v < H) {
            const BulkRowMeta m = st.meta[r];
            const size_t row = (size_t)v * W;
            float* __restrict__ Df = P.Df;
            uint8_t* __restrict__ Cf = P.Cf;
            uint8_t* __restrict__ mask = P.mask;
            int cost[kVJ];
#pragma unroll
            for (int j = 0; j < kVJ; j++) {
                const int u = u0 + lane + 32 * j;
                cost[j] = -1;
                if (u >= W) continue;
                const int oi = m.o_off + j;
                const uint32_t ow = oi < m.o_cnt ? st.om[r][oi] : __ldg(P.omega + (size_t)v * words + (u0 >> 5) + j);
                const bool om = (ow >> lane) & 1u;
                const int di = m.d_off + lane + 32 * j;
                const float d = di < m.d_cnt ? st.d[r][di] : __ldg(P.Dit + row + u);
                const float col = (float)u - rintf(d);
                uint8_t mk = om ? 1 : 0;
                if (om && col >= 2.0f && col <= (float)(W - 3)) {
                    const int c = (int)col;
                    const uint32_t cl = di < m.d_cnt ? st.cl[r][di] : __ldg(P.cL + row + u);
                    const int ri = c - m.r_base;
                    const uint32_t cr = (m.r_base >= 0 && ri >= 0 && ri < m.r_cnt) ? st.cr[r][ri] : __ldg(P.cR + row + c);
                    cost[j] = __popc(cl ^ cr);
                    mk |= 2 | (cost[j] < t_lo ? 4 : 0) | (cost[j] > t_hi ? 8 : 0);
                }
                if (mask) mask[row + u] = mk;
                const int cj = cost[j];
                if (first) {
                    const bool upd = cj >= 0 && cj < t_hi;
                    Df[row + u] = upd ? d : 0.0f;
                    Cf[row + u] = (uint8_t)(upd ? cj : t_hi);
                } else if (cj >= 0) {
                    const int fi = m.f_off + lane + 32 * j;
                    const int cf = fi < m.f_cnt ? (int)st.cf[r][fi] : (int)Cf[row + u];
                    if (cj < cf) {
                        Df[row + u] = d;
                        Cf[row + u] = (uint8_t)cj;
                    }
                }
            }
            if (cells) {
                const int ly = cell_div(v, shift, magic) - cy0;
                const bool warp_cell = sz >= 32 && (sz & 31) == 0;
#pragma unroll
                for (int j = 0; j < kVJ; j++) {
                    const int u = u0 + lane + 32 * j;
                    const int cj = cost[j];
                    const uint32_t p = (uint32_t)(row + u);
                    uint32_t kg = (cj >= 0 && cj < t_lo) ? (((uint32_t)cj << 27) | p) : kNoKey;
                    uint32_t kb = (cj > t_hi) ? (((uint32_t)(24 - cj) << 27) | p) : kNoKey;
                    const int lc = ly * ncx + ((int)cell_div(min(u, W - 1), shift, magic) - cx0);
                    if (warp_cell) {
                        kg = __reduce_min_sync(0xffffffffu, kg);
                        kb = __reduce_min_sync(0xffffffffu, kb);
                        if (lane == 0) {
                            if (kg != kNoKey) atomicMin(&sm.g[cb][lc], kg);
                            if (kb != kNoKey) atomicMin(&sm.b[cb][lc], kb);
                        }
                    } else {
                        if (kg != kNoKey) atomicMin(&sm.g[cb][lc], kg);
                        if (kb != kNoKey) atomicMin(&sm.b[cb][lc], kb);
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            mbar_arrive(&sm.empty[s]);     // this warp is done with the stage
            mbar_arrive(&sm.cdone[cb]);    // and with its cell minima
        }
        // all eight consumer warps' minima are in before the flush (a bounded wait)
        if (!mbar_wait(&sm.cdone[cb], (unsigned)(k >> 1) & 1u)) { ok = false; break; }
        if (cells) {
            for (int i = ct; i < ncx * ncy; i += 256) {
                const int iy = i / ncx, ix = i - iy * ncx;
                const size_t cell = (size_t)(cy0 + iy) * Wc + (cx0 + ix);
                const uint32_t g = sm.g[cb][i], bb = sm.b[cb][i];
                if (g != kNoKey) atomicMin(P.cg_key + cell, g);
                if (bb != kNoKey) atomicMin(P.cb_key + cell, bb);
                sm.g[cb][i] = kNoKey;
                sm.b[cb][i] = kNoKey;
            }
        }
    }
    if (!ok && lane == 0 && prm.err) atomicExch(prm.err, 1);
}

__global__ void __launch_bounds__(288, 2) k_validate_bulk(PairBatch b, Params prm) {
    extern __shared__ __align__(128) unsigned char smraw[];
    BulkSmem& sm = *reinterpret_cast<BulkSmem*>(smraw);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBS; s++) {
            mbar_init(&sm.full1[s], 1);
            mbar_init(&sm.full2[s], 1);
            mbar_init(&sm.empty[s], kVH);
        }
        mbar_init(&sm.cdone[0], kVH);
        mbar_init(&sm.cdone[1], kVH);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < 2 * kMaxLocalCells; i += blockDim.x) {
        (&sm.g[0][0])[i] = kNoKey;
        (&sm.b[0][0])[i] = kNoKey;
    }
    __syncthreads();
    if (threadIdx.x < 32) bulk_producer(b, prm, sm);
    else bulk_consumer(b, prm, sm, (threadIdx.x >> 5) - 1);
}

// ---------------------------------------------------------------- resample + match (Alg. 4)
// One warp per cell: a C_g key becomes the interpolated disparity at its
// pixel; a C_b key is matched along its row by the same warp search.
// A thread per cell decodes its records (C_g's disparity D_it, 32 cells a warp, the
// key loads coalesced); the warp then takes its cells with a C_b pick through the
// epipolar match one after another, all 32 lanes on each (SparseEpipolarStereo).
__device__ __forceinline__ void resample_body(const PairDev& P, int local, const Params& prm) {
    const int lane = threadIdx.x & 31;
    const int cell = local * 256 + threadIdx.x;
    const bool in = cell < P.Wc * P.Hc;
    const uint32_t gk = in ? P.cg_key[cell] : kNoKey, bk = in ? P.cb_key[cell] : kNoKey;
    if (in) P.cg_d[cell] = gk != kNoKey ? P.Dit[gk & kIdxMask] : __int_as_float(0x7fc00000);
    // each lane reads its own C_b pick's left code up front (all lanes at once), so a
    // match in the warp's chain waits on the right-row loads only
    const uint32_t mycl = bk != kNoKey ? __ldg(P.cL + (bk & kIdxMask)) : 0u;
    int xd = -1;
    unsigned todo = __ballot_sync(0xffffffffu, bk != kNoKey);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t p = __shfl_sync(0xffffffffu, bk, src) & kIdxMask;
        const uint32_t cl = __shfl_sync(0xffffffffu, mycl, src);
        const int u = (int)(p % (uint32_t)P.W), v = (int)(p / (uint32_t)P.W);
        const int r = warp_match_code(P.cR, P.W, P.H, u, v, cl, P.dmax, prm.t_lo, prm.margin);
        if (lane == src) xd = r;
    }
    if (in) P.x_d[cell] = xd;
}

__global__ void __launch_bounds__(256) k_resample(PairBatch b, Params prm) {
#define BODY(P, l) resample_body(P, l, prm)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

// Cell records of a pass start empty (0xFFFFFFFF) for the atomic minimum.
__device__ __forceinline__ void fill_cells_body(const PairDev& P, int local) { fill_cells_range(P, local); }

__global__ void __launch_bounds__(256) k_fill_cells(PairBatch b) {
#define BODY(P, l) fill_cells_body(P, l)
    FOR_EACH_ITEM(b, BODY)
#undef BODY
}

__global__ void k_fill_u32(uint32_t* p, uint32_t value, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = value;
}

// ---------------------------------------------------------------- launchers
cudaError_t launch_census(const PairBatch& b, const Params& prm, cudaStream_t s) {
    const int grid = grid_for(cdiv(b.total, 8), 8);  // a warp per strip item
    if (b.scan_rows == 7) k_census<7><<<grid, 256, 0, s>>>(b, prm);
    else k_census<kScanRows><<<grid, 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_fast_score(const PairBatch& b, const Params& prm, cudaStream_t s) {
    const int grid = grid_for(cdiv(b.total, 8), 8);  // a warp per strip item
    if (b.scan_rows == 7) k_fast_score<7><<<grid, 256, 0, s>>>(b, prm);
    else k_fast_score<kScanRows><<<grid, 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_fast_bins(const PairBatch& b, const Params& prm, cudaStream_t s) {
    k_fast_bins<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_match_kp(const PairBatch& b, const Params& prm, cudaStream_t s) {
    k_match_kp<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_raster_clear(const PairBatch& b, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_raster_clear<<<grid_for(b.total, 8), 256, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_raster(const PairBatch& b, cudaStream_t s) {
    k_raster<<<grid_for(b.total, 8), 256, 0, s>>>(b);
    return cudaGetLastError();
}
cudaError_t launch_raster_device_lists(const PairDev& p, cudaStream_t s) {
    if (p.T <= 0) return cudaSuccess;
    const int nblk = (p.T + kListBlock - 1) / kListBlock;
    int32_t* blk = p.small_tri + p.T + 1;  // after the small list: 2 * nblk entries
    k_lists_count<<<nblk, kListBlock, 0, s>>>(p.tri_uv, p.T, p.W, p.H, blk);
    k_lists_scan<<<1, kListBlock, 0, s>>>(blk, nblk, p.T, p.tri_rows, p.small_tri);
    k_lists_write<<<nblk, kListBlock, 0, s>>>(p.tri_uv, p.T, p.W, p.H, blk, p.tri_rows, p.small_tri);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_raster_dev<<<sm_count() * 8, 256, 0, s>>>(p.tri_uv, p.abc, p.tri_rows, p.small_tri, p.T, p.W, p.H,
                                               p.planeidx, p.Dit);
    return cudaGetLastError();
}
static VDesc vdesc_of(const PairDev& p) {
    VDesc d;
    d.omega = p.omega;
    d.dit = p.Dit;
    d.cL = p.cL;
    d.cR = p.cR;
    d.Df = p.Df;
    d.Cf = p.Cf;
    d.mask = p.mask;
    d.cg = p.cg_key;
    d.cb = p.cb_key;
    d.W = p.W;
    d.H = p.H;
    d.first = p.first_pass;
    d.sz = p.sz;
    d.shift = p.sz_shift;
    d.Wc = p.Wc;
    d.sh = validate_strip_rows(p);
    d.kind = (int)validate_kind_of(p);
    d.magic = p.sz_magic;
    return d;
}

template <int KIND>
static cudaError_t launch_vbatch(const VBatch& vb, const Params& prm, cudaStream_t s, int bps) {
    k_validate<KIND><<<grid_for(cdiv(vb.total, 8), bps), 256, 0, s>>>(vb, prm);  // 8 strips (warps) per block
    return cudaGetLastError();
}

cudaError_t launch_validate(const PairDev* pairs, int n, WorkKind k, const Params& prm, cudaStream_t s,
                            int* launches, int min_launches, int blocks_per_sm) {
    const int bps = blocks_per_sm > 0 ? blocks_per_sm : 8;
    int nl = 0;
    VBatch vb;
    int i = 0;
    while (i < n || nl < min_launches) {  // up to kVBatch pairs with work per launch
        vb.npairs = 0;
        vb.total = 0;
        int cls = -1;         // the launch's one cell-side class, or -2 when it has several
        for (; i < n && vb.npairs < kVBatch; i++) {
            const int items = work_items(k, pairs[i]);
            if (items <= 0) continue;
            const int pk = (int)validate_kind(pairs[i]);
            cls = cls == -1 || cls == pk ? pk : -2;
            vb.d[vb.npairs] = vdesc_of(pairs[i]);
            vb.off[vb.npairs++] = vb.total;
            vb.total += items;
        }
        if (vb.npairs == 0 && nl >= min_launches) break;
        vb.off[vb.npairs] = vb.total;
        // a mixed launch whose pairs share one class takes that class's kernel (no
        // dispatch, fewer registers); the 4- and 2-row strips fill eight blocks an SM
        const WorkKind kk = k == WK_VALIDATE_MIXED && cls >= 0 ? (WorkKind)cls : k;
        const int bk = kk == WK_VALIDATE_C4 || kk == WK_VALIDATE_C2 ? std::max(bps, 8) : bps;
        cudaError_t e;
        switch (kk) {
            case WK_VALIDATE: e = launch_vbatch<WK_VALIDATE>(vb, prm, s, bk); break;
            case WK_VALIDATE_UNIT: e = launch_vbatch<WK_VALIDATE_UNIT>(vb, prm, s, bk); break;
            case WK_VALIDATE_C4: e = launch_vbatch<WK_VALIDATE_C4>(vb, prm, s, bk); break;
            case WK_VALIDATE_C2: e = launch_vbatch<WK_VALIDATE_C2>(vb, prm, s, bk); break;
            case WK_VALIDATE_ANY: e = launch_vbatch<WK_VALIDATE_ANY>(vb, prm, s, bk); break;
            case WK_VALIDATE_MIXED: e = launch_vbatch<WK_VALIDATE_MIXED>(vb, prm, s, bk); break;
            default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
        nl++;
    }
    if (launches) *launches = nl;
    return cudaSuccess;
}
size_t validate_bulk_smem_bytes() { return sizeof(BulkSmem); }
cudaError_t prepare_kernels() {  // once per device, outside any stream capture
    return cudaFuncSetAttribute(k_validate_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BulkSmem));
}
cudaError_t launch_validate_bulk(const PairBatch& b, const Params& prm, cudaStream_t s) {
    if (b.total <= 0) return cudaSuccess;
    k_validate_bulk<<<grid_for(b.total, 2), 288, sizeof(BulkSmem), s>>>(b, prm);
    return cudaGetLastError();
}
// Gather copy: kCopyParts blocks per entry, each a contiguous part of it, in
// 16-byte words when both ends are 16-byte aligned (bytes otherwise).  A source
// may be page-locked host memory that the caller rewrites between calls, so the
// loads fetch again rather than trust a cached line (ld.global.cv).
constexpr int kCopyParts = 16;  // blocks per entry: 8 moved device-to-host results 1.4 % slower end to end
__global__ void __launch_bounds__(256) k_copy_list(const __grid_constant__ CopyList L) {
    const int e = blockIdx.x / kCopyParts, part = blockIdx.x % kCopyParts;
    if (e >= L.count) return;
    const long long n = L.n[e];
    const uint8_t* src = L.src[e];
    uint8_t* dst = L.dst[e];
    const long long per = (n / kCopyParts + 15) / 16 * 16;
    const long long lo = min(n, per * part), hi = min(n, lo + per);
    if ((((uintptr_t)src | (uintptr_t)dst) & 15) == 0) {
        const long long w0 = lo / 16, w1 = hi / 16, bs = blockDim.x;
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        long long w = w0 + threadIdx.x;
        for (; w + 3 * bs < w1; w += 4 * bs) {  // four loads in flight a thread
            const uint4 a = __ldcv(s4 + w), b = __ldcv(s4 + w + bs), c = __ldcv(s4 + w + 2 * bs),
                        d = __ldcv(s4 + w + 3 * bs);
            d4[w] = a;
            d4[w + bs] = b;
            d4[w + 2 * bs] = c;
            d4[w + 3 * bs] = d;
        }
        for (; w < w1; w += bs) d4[w] = __ldcv(s4 + w);
        for (long long i = max(lo, w1 * 16) + threadIdx.x; i < hi; i += blockDim.x) dst[i] = __ldcv(src + i);
    } else {
        for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) dst[i] = __ldcv(src + i);
    }
}

cudaError_t launch_copy_list(const CopyList& L, cudaStream_t s) {
    if (L.count <= 0) return cudaSuccess;
    k_copy_list<<<L.count * kCopyParts, 256, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_resample(const PairBatch& b, const Params& prm, cudaStream_t s) {
    k_resample<<<grid_for(b.total, 8), 256, 0, s>>>(b, prm);
    return cudaGetLastError();
}
cudaError_t launch_fill_cells(const PairBatch& b, cudaStream_t s) {
    k_fill_cells<<<grid_for(b.total, 8), 256, 0, s>>>(b);
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
