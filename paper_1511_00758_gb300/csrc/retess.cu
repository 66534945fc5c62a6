// On-device re-tessellation between passes (Alg. 1: DelaunayTriangulation of
// S_{it+1} after SupportResampling), planes (Eq. 3) and the raster inputs of
// the next pass.
//
// S_{it+1} = S_it + the pass's new points, and every new point is a pixel
// that the pass evaluated, so it lies in the closed hull of G(S_it) and the
// pass's own plane-index map names a triangle that contains it.  The mesh of
// the previous pass therefore stays on the device and the new points are
// inserted into it, in rounds: every pending point claims the triangle it
// lies in (and the neighbour, when it lies on an edge); a point that holds
// all its claims splits them (1 -> 3 inside a triangle, 2 -> 4 on an inner
// edge, 1 -> 2 on a hull edge), and the points left in a split triangle move
// to the piece that contains them.  Then Lawson flips restore the Delaunay
// property: an edge whose opposite vertex lies inside the circle of the
// triangle is flipped, each triangle in at most one flip per round, until no
// edge is illegal.  The orientation test is exact in int64 and the in-circle
// test is the same symbolically perturbed one as the host triangulation
// (Edelsbrunner & Muecke's Simulation of Simplicity on the lifted coordinate,
// a point earlier in (v, u) order carrying the larger perturbation); with it
// every flip is valid and the flips end at the unique triangulation of the
// perturbed point set, the one the host routine returns.
//
// Before the last pass the triangles are put in canonical order (rank of
// the sorted canonical vertex triple), the ranks of the vertices coming from
// a W x H bit map of the vertex pixels: the canonical index of (u, v) is the
// number of vertex pixels before it in raster order, which is (v, u) order.
//
// Everything runs in one launch per pass over up to kMeshBatch pairs, one
// thread-block cluster per pair: the cluster's blocks share the pair's items
// and meet at the hardware cluster barrier between phases (pairs are
// independent meshes, so nothing waits across clusters), and every loop
// decision is read after a barrier, so all blocks of a cluster take it alike.
// The phases are latency-bound (short chains of dependent loads with a
// barrier after each), so the rounds, not the bytes, set the time.  Loops are
// bounded: a pair that does not finish sets its error code.
#include <cooperative_groups.h>

#include "internal.h"

namespace cg = cooperative_groups;

namespace stereo {

namespace {

constexpr int kMeshThreads = 1024;  // one block per SM (61 registers a thread)
constexpr int kMaxInsertRounds = 4096;
constexpr int kMaxFlipRounds = 1 << 15;
constexpr int kSoloItems = kMeshThreads;  // rounds this small run in one block
constexpr int kScanChunk = 256;   // elements per warp in the two-level scans (8 a lane)
constexpr unsigned long long kNoClaim = ~0ull;
constexpr int kDropped = -3;  // edge code of a pending point not found in its triangle

size_t al(size_t x) { return (x + 255) / 256 * 256; }

__device__ __forceinline__ uint32_t vkey(int2 p) { return ((uint32_t)p.y << 14) | (uint32_t)p.x; }

__device__ __forceinline__ long long orient(int2 a, int2 b, int2 c) {
    return (long long)(b.x - a.x) * (c.y - a.y) - (long long)(b.y - a.y) * (c.x - a.x);
}

// d strictly inside the circle of the positively oriented (a, b, c), in the
// perturbed configuration: at an exact tie the sign is that of the cofactor
// of the lifted entry of the point earliest in (v, u) order, then the next.
__device__ __forceinline__ bool incircle_sos(int2 a, int2 b, int2 c, int2 d) {
    const long long ax = a.x - d.x, ay = a.y - d.y;
    const long long bx = b.x - d.x, by = b.y - d.y;
    const long long cx = c.x - d.x, cy = c.y - d.y;
    const long long la = ax * ax + ay * ay, lb = bx * bx + by * by, lc = cx * cx + cy * cy;
    const long long det = la * (bx * cy - by * cx) - lb * (ax * cy - ay * cx) + lc * (ax * by - ay * bx);
    if (det != 0) return det > 0;
    uint32_t k[4] = {vkey(a), vkey(b), vkey(c), vkey(d)};
    for (int r = 0; r < 4; r++) {
        int m = 0;
        for (int j = 1; j < 4; j++)
            if (k[j] < k[m]) m = j;
        long long cof;
        switch (m) {
            case 0: cof = orient(b, c, d); break;
            case 1: cof = -orient(a, c, d); break;
            case 2: cof = orient(a, b, d); break;
            default: cof = -orient(a, b, c); break;
        }
        if (cof != 0) return cof > 0;
        k[m] = 0xFFFFFFFFu;
    }
    return false;
}

__device__ __forceinline__ int vtx(const int4& t, int k) { return k == 0 ? t.x : k == 1 ? t.y : t.z; }
__device__ __forceinline__ int& vtx(int4& t, int k) { return k == 0 ? t.x : k == 1 ? t.y : t.z; }
__device__ __forceinline__ int ref_of(const int4& r, int k) { return k == 0 ? r.x : k == 1 ? r.y : r.z; }
__device__ __forceinline__ int& ref_of(int4& r, int k) { return k == 0 ? r.x : k == 1 ? r.y : r.z; }
__device__ __forceinline__ int smap_ref(const int4& s, int k) { return k == 0 ? s.y : k == 1 ? s.z : s.w; }
__device__ __forceinline__ int mk_ref(int t, int e) { return (t << 2) | e; }

// A position packed as (v << 14) | u (u, v < 16384), and back.
__device__ __forceinline__ int pk(int2 p) { return (p.y << 14) | p.x; }
__device__ __forceinline__ int2 unpk(int k) { return make_int2(k & 0x3FFF, k >> 14); }

// Conversions to and from fp64 built from the IEEE-754 bit layouts with integer
// instructions: this GPU has few fp64 units, and the plane solve would otherwise
// spend a quarter of its fp64 issue on conversions.  Each is exact (to fp64) or
// round-to-nearest-even (to fp32); zeros, subnormals, infinities and results out
// of fp32's normal range take the hardware conversion.
__device__ __forceinline__ double i2d(int x) {  // exact for every int
    if (x == 0) return 0.0;
    const unsigned long long a = x < 0 ? (unsigned long long)(-(long long)x) : (unsigned long long)x;
    const int e = 63 - __clzll((long long)a);
    const unsigned long long mant = (a << (52 - e)) & ((1ull << 52) - 1ull);
    const unsigned long long sign = x < 0 ? 1ull << 63 : 0ull;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 1023) << 52) | mant));
}
__device__ __forceinline__ double f2d(float f) {  // exact
    const unsigned u = __float_as_uint(f), e8 = (u >> 23) & 0xFFu;
    if (e8 == 0u || e8 == 255u) return (double)f;
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                            ((unsigned long long)(e8 - 127u + 1023u) << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ float d2f_rn(double x) {  // round to nearest, ties to even
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e8 = (int)((b >> 52) & 0x7FF) - 1023 + 127;
    if (e8 <= 0 || e8 >= 254) return __double2float_rn(x);
    const unsigned long long m = b & ((1ull << 52) - 1ull), rem = m & ((1ull << 29) - 1ull), half = 1ull << 28;
    unsigned m23 = (unsigned)(m >> 29);
    unsigned bits = ((unsigned)(b >> 63) << 31) | ((unsigned)e8 << 23);
    if (rem > half || (rem == half && (m23 & 1u))) m23++;  // a carry out of the fraction raises the exponent
    return __uint_as_float(bits + m23);
}

// q in the closed triangle with packed vertex positions tp (all three edge functions >= 0)
__device__ __forceinline__ bool contains(const int4& tp, int2 q) {
    const int2 a = unpk(tp.x), b = unpk(tp.y), c = unpk(tp.z);
    return orient(b, c, q) >= 0 && orient(c, a, q) >= 0 && orient(a, b, q) >= 0;
}

}  // namespace

// ---------------------------------------------------------------- sizes
int mesh_vertex_cap(int W, int H, int seed_points, int iters, int cell) {
    long long n = seed_points;
    int sz = cell;
    for (int it = 1; it < iters; it++) {
        n += 2ll * ((W + sz - 1) / sz) * ((H + sz - 1) / sz);
        sz = sz / 2 > 1 ? sz / 2 : 1;
    }
    const long long px = (long long)W * H;
    return (int)(n < px ? n : px);
}

namespace {
__host__ __device__ __forceinline__ int scan_chunks(int n) { return (n + kScanChunk - 1) / kScanChunk; }
int scan_cap_of(int W, int H, int n_cap, int t_cap) {
    const int words = (int)(((long long)W * H + 31) / 32);
    int m = words > n_cap + 1 ? words : n_cap + 1;
    if (t_cap + 1 > m) m = t_cap + 1;
    return scan_chunks(m) + 2;
}
}  // namespace

// The arrays in carving order; size_t x[] of element counts and sizes.
#define MESH_ARRAYS(X)                                      \
    X(hdr, MeshHdr, 1)                                      \
    X(pos, int2, n_cap)                                     \
    X(vpass, uint8_t, n_cap)                                \
    X(vcanon, int4, n_cap)                                  \
    X(dmap, float, (size_t)W * H)                           \
    X(occ, uint32_t, words)                                 \
    X(wpre, uint32_t, words + 1)                            \
    X(tr, TriRec, t_cap)                                    \
    X(cl, ClaimRec, t_cap)                                  \
    X(alist, int, (size_t)2 * t_cap)                        \
    X(smap, int4, t_cap)                                    \
    X(gcnt, int, (size_t)n_cap + 1)                         \
    X(tperm, int, t_cap)                                    \
    X(tpass, uint32_t, n_cap)                               \
    X(tpos, uint32_t, n_cap)                                \
    X(plist, int4, (size_t)2 * p_cap)                       \
    X(pkey, unsigned long long, p_cap)                      \
    X(scan, int, scap)                                      \
    X(large, int, (size_t)t_cap + 1)                        \
    X(lrows, int, (size_t)t_cap + 1)                        \
    X(tri_uv, int32_t, (size_t)6 * t_cap)                   \
    X(abc, float, (size_t)3 * t_cap)                        \
    X(small, int32_t, (size_t)t_cap + 1)                    \
    X(hull, int4, n_cap)

size_t mesh_bytes(int W, int H, int n_cap, int t_cap, int p_cap) {
    const size_t words = ((size_t)W * H + 31) / 32;
    const int scap = scan_cap_of(W, H, n_cap, t_cap);
    size_t b = 0;
#define SZ(name, type, count) b += al(sizeof(type) * (size_t)(count));
    MESH_ARRAYS(SZ)
#undef SZ
    return b;
}

void mesh_carve(MeshDev& m, void* block, int W, int H, int n_cap, int t_cap, int p_cap) {
    const size_t words = ((size_t)W * H + 31) / 32;
    const int scap = scan_cap_of(W, H, n_cap, t_cap);
    char* p = (char*)block;
    MeshDev z{};
    m = z;
#define CV(name, type, count)                     \
    m.name = (decltype(m.name))(p);               \
    p += al(sizeof(type) * (size_t)(count));
    MESH_ARRAYS(CV)
#undef CV
    m.n_cap = n_cap;
    m.t_cap = t_cap;
    m.p_cap = p_cap;
    m.scan_cap = scap;
    m.W = W;
    m.H = H;
}

// ---------------------------------------------------------------- phase plumbing
namespace {

__device__ __forceinline__ int words_of(const MeshDev& m) { return (int)(((long long)m.W * m.H + 31) / 32); }

__device__ __forceinline__ int warp_excl_scan(int x, int& total) {
    const int l = threadIdx.x & 31;
    int s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, s, o);
        if (l >= o) s += y;
    }
    total = __shfl_sync(0xffffffffu, s, 31);
    return s - x;
}

// Two-level exclusive scan of f(in[0..n)) into out[0..n) (out may be in),
// over three phases separated by cluster barriers: (A) a warp sums each chunk
// of kScanChunk elements into chunk[c]; (B) one warp per array scans the
// chunk sums and stores the total; (C) a warp writes each chunk's prefixes
// (lane l owns kScanChunk / 32 consecutive elements).
template <class F>
__device__ __forceinline__ void scan_a(const uint32_t* in, int n, int* chunk, int c, F f) {
    const int l = threadIdx.x & 31;
    const int base = c * kScanChunk;
    int s = 0;
    for (int i = base + l; i < base + kScanChunk && i < n; i += 32) s += f(in[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) chunk[c] = s;
}
__device__ __forceinline__ void scan_b(int* chunk, int nch, int* total) {
    const int l = threadIdx.x & 31;
    int carry = 0;
    for (int b = 0; b < nch; b += 32) {
        const int x = b + l < nch ? chunk[b + l] : 0;
        int tot;
        const int e = warp_excl_scan(x, tot);
        if (b + l < nch) chunk[b + l] = carry + e;
        carry += tot;
    }
    if (l == 0 && total) *total = carry;
}
template <class F>
__device__ __forceinline__ void scan_c(const uint32_t* in, uint32_t* out, int n, const int* chunk, int c, F f) {
    const int l = threadIdx.x & 31;
    constexpr int per = kScanChunk / 32;
    const int i0 = c * kScanChunk + per * l;
    int s = 0;
#pragma unroll
    for (int i = i0; i < i0 + per; i++)
        if (i < n) s += f(in[i]);
    int tot;
    int run = chunk[c] + warp_excl_scan(s, tot);
    for (int i = i0; i < i0 + per && i < n; i++) {
        const int x = f(in[i]);
        out[i] = (uint32_t)run;
        run += x;
    }
}
struct Ident {
    __device__ int operator()(uint32_t x) const { return (int)x; }
};
struct Popc {
    __device__ int operator()(uint32_t x) const { return __popc(x); }
};

}  // namespace

// ---------------------------------------------------------------- mesh edits
// Triangle t = (v0, v1, v2) has edge k from v(k+1) to v(k+2), opposite v(k),
// the interior on its positive side; its record holds the vertices' packed
// positions and, per edge k, (s << 2) | e naming the twin edge e of the
// neighbour s.  An edit writes the new pieces whole, their outer edges still
// naming the old neighbours, and records in smap[old slot] (stamped with the
// round) where each old edge went; relink() then moves those names through
// the neighbours' records.
namespace {

__device__ __forceinline__ int4 pks_of(const TriRec& r) { return make_int4(r.a.x, r.a.y, r.a.z, 0); }
__device__ __forceinline__ int4 refs_of(const TriRec& r) { return make_int4(r.a.w, r.b.x, r.b.y, 0); }

// the whole record of t: positions p, neighbour refs r, no point pending
__device__ __forceinline__ void put_tri(const MeshDev& m, int t, int4 p, int4 r) {
    m.tr[t].a = make_int4(p.x, p.y, p.z, r.x);
    m.tr[t].b = make_int4(r.y, r.z, 0, 0);
}
__device__ __forceinline__ int* ref_ptr(const MeshDev& m, int t, int e) {
    return e == 0 ? &m.tr[t].a.w : &m.tr[t].b.x + (e - 1);
}
__device__ __forceinline__ int get_ref(const MeshDev& m, int t, int e) { return *ref_ptr(m, t, e); }
__device__ __forceinline__ void set_ref(const MeshDev& m, int t, int e, int r) { *ref_ptr(m, t, e) = r; }

__device__ __forceinline__ int4 smap_rec(int stamp, int k, int r_k, int k1, int r_k1, int k2, int r_k2) {
    int r[3];
    r[k] = r_k;
    r[k1] = r_k1;
    r[k2] = r_k2;
    return make_int4(stamp, r[0], r[1], r[2]);
}

// p (packed position pkp) strictly inside t: pieces replace vertex k by p
// (piece k keeps old edge k); piece j's edge k is the twin of piece k's edge j.
// t keeps the claim that won it (the round resets it); the points left in t
// are counted in the pieces they move to.
__device__ __forceinline__ bool split3(const MeshDev& m, int t, int pkp, int stamp) {
    const int base = atomicAdd(&m.hdr->T, 2);
    if (base + 2 > m.t_cap) {
        m.hdr->err = 1;
        return false;
    }
    const TriRec o = m.tr[t];
    const int4 op = pks_of(o), r = refs_of(o);
    const int s0 = t, s1 = base, s2 = base + 1;
    put_tri(m, s0, make_int4(pkp, op.y, op.z, 0), make_int4(r.x, mk_ref(s1, 0), mk_ref(s2, 0), 0));
    put_tri(m, s1, make_int4(op.x, pkp, op.z, 0), make_int4(mk_ref(s0, 1), r.y, mk_ref(s2, 1), 0));
    put_tri(m, s2, make_int4(op.x, op.y, pkp, 0), make_int4(mk_ref(s0, 2), mk_ref(s1, 2), r.z, 0));
    m.smap[t] = make_int4(stamp, mk_ref(s0, 0), mk_ref(s1, 1), mk_ref(s2, 2));
    m.smap[s1] = m.smap[s2] = make_int4(stamp, -1, -1, -1);  // new this round: no old edges to map
    m.cl[s0].acc = 0ull;
    m.cl[s1] = m.cl[s2] = ClaimRec{kNoClaim, 0ull};
    return true;
}

// p on edge k of t (from b = v(k+1) to c = v(k+2)), strictly between b and c.
// t splits into A (c replaced by p, slot t) and B (b replaced by p); when the
// edge is inner, its twin edge j of n splits n into A' (b replaced, slot n)
// and B' (c replaced).  A's edge k (b -> p) is the twin of edge j of B',
// B's edge k (p -> c) the twin of edge j of A'.
__device__ __forceinline__ bool split_edge(const MeshDev& m, int t, int k, int n, int j, int pkp, int stamp) {
    const int need = n >= 0 ? 2 : 1;
    const int base = atomicAdd(&m.hdr->T, need);
    if (base + need > m.t_cap) {
        m.hdr->err = 1;
        return false;
    }
    const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
    const TriRec ot = m.tr[t];
    const int4 pt = pks_of(ot), rt = refs_of(ot);
    const int sB = base, sB2 = n >= 0 ? base + 1 : -1;
    int4 pA = pt, pB = pt;
    vtx(pA, k2) = pkp;
    vtx(pB, k1) = pkp;
    int4 rA = rt, rB = rt;
    ref_of(rA, k) = n >= 0 ? mk_ref(sB2, j) : -1;
    ref_of(rA, k1) = mk_ref(sB, k2);
    ref_of(rB, k2) = mk_ref(t, k1);
    ref_of(rB, k) = n >= 0 ? mk_ref(n, j) : -1;
    put_tri(m, t, pA, rA);
    put_tri(m, sB, pB, rB);
    m.smap[t] = smap_rec(stamp, k, -1, k1, mk_ref(sB, k1), k2, mk_ref(t, k2));
    m.smap[sB] = make_int4(stamp, -1, -1, -1);
    m.cl[t].acc = 0ull;
    m.cl[sB] = ClaimRec{kNoClaim, 0ull};
    if (n >= 0) {
        const int j1 = j == 2 ? 0 : j + 1, j2 = j == 0 ? 2 : j - 1;
        const TriRec on = m.tr[n];
        const int4 pn = pks_of(on), rn = refs_of(on);
        int4 pA2 = pn, pB2 = pn;
        vtx(pA2, j2) = pkp;  // w(j+2) = b
        vtx(pB2, j1) = pkp;  // w(j+1) = c
        int4 rA2 = rn, rB2 = rn;
        ref_of(rA2, j) = mk_ref(sB, k);
        ref_of(rA2, j1) = mk_ref(sB2, j2);
        ref_of(rB2, j2) = mk_ref(n, j1);
        ref_of(rB2, j) = mk_ref(t, k);
        put_tri(m, n, pA2, rA2);
        put_tri(m, sB2, pB2, rB2);
        m.smap[n] = smap_rec(stamp, j, -1, j1, mk_ref(sB2, j1), j2, mk_ref(n, j2));
        m.smap[sB2] = make_int4(stamp, -1, -1, -1);
        m.cl[n].acc = 0ull;
        m.cl[sB2] = ClaimRec{kNoClaim, 0ull};
    }
    return true;
}

// Flip edge k of t (twin edge j of n): with x = v(k), b = v(k+1), c = v(k+2)
// of t and y = w(j) of n, the pieces are t' = (x, b, y) and n' = (y, c, x);
// edge 1 of each is the new diagonal, edges 0 and 2 are old outer edges.
__device__ __forceinline__ void flip(const MeshDev& m, int t, int k, int n, int j, int stamp) {
    const int k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
    const int j1 = j == 2 ? 0 : j + 1, j2 = j == 0 ? 2 : j - 1;
    const TriRec Rt = m.tr[t], Rn = m.tr[n];
    const int4 pt = pks_of(Rt), pn = pks_of(Rn), rt = refs_of(Rt), rn = refs_of(Rn);
    const int px = vtx(pt, k), pb = vtx(pt, k1), pc = vtx(pt, k2), py = vtx(pn, j);
    put_tri(m, t, make_int4(px, pb, py, 0), make_int4(ref_of(rn, j1), mk_ref(n, 1), ref_of(rt, k2), 0));
    put_tri(m, n, make_int4(py, pc, px, 0), make_int4(ref_of(rt, k1), mk_ref(t, 1), ref_of(rn, j2), 0));
    m.smap[t] = smap_rec(stamp, k, -1, k1, mk_ref(n, 0), k2, mk_ref(t, 2));
    m.smap[n] = smap_rec(stamp, j, -1, j1, mk_ref(t, 0), j2, mk_ref(n, 2));
}

// Outer edge e of a piece s made this round: its name of the old neighbour
// (m', i) goes through m''s record when m' was edited this round too (that
// edit links its own side); otherwise the neighbour is told about s.
__device__ __forceinline__ void relink(const MeshDev& m, int s, int e, int stamp) {
    const int r = get_ref(m, s, e);
    if (r < 0) return;
    const int mm = r >> 2, i = r & 3;
    const int4 sm = m.smap[mm];
    if (sm.x == stamp) set_ref(m, s, e, smap_ref(sm, i));
    else set_ref(m, mm, i, mk_ref(s, e));
}

}  // namespace

// ---------------------------------------------------------------- the pass kernel
namespace {

// A 32-bit mix of an edge id and a round (the murmur3 finaliser applied to
// their combination): an arbitrary but fixed priority per edge and round.
__device__ __forceinline__ unsigned mix32(unsigned x, unsigned r) {
    unsigned h = x * 0x9E3779B1u ^ (r + 0x7F4A7C15u);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// Claim priority of a pending point: squared distance from the mean of the
// points pending in its triangle (sum s of their (u, v), count c), then the
// vertex slot (unique).  The point nearest the middle of the points, not of
// the triangle, splits them most evenly between the pieces, which keeps the
// rounds few where the points crowd one corner of a large triangle.  The key
// only orders the claims (the triangulation reached does not depend on it);
// the fp32 square of a non-negative distance orders as its bit pattern.
__device__ __forceinline__ unsigned long long claim_key(unsigned long long s, int c, int2 q, int vid) {
    const float mu = (float)(unsigned)(s >> 32) / (float)c, mv = (float)(unsigned)(s & 0xFFFFFFFFu) / (float)c;
    const float dx = (float)q.x - mu, dy = (float)q.y - mv;
    return ((unsigned long long)__float_as_uint(dx * dx + dy * dy) << 27) | (unsigned)vid;
}

__device__ __forceinline__ void count_pending(const MeshDev& m, int t, int2 q) {
    atomicAdd(&m.cl[t].acc, ((unsigned long long)q.x << 32) | (unsigned)q.y);
    atomicAdd(&m.tr[t].b.z, 1);
}

__device__ __forceinline__ int ld_int(const int* p) { return *(const volatile int*)p; }

// The pass's candidate points of each lane of a warp, two a lane (want[k]: the
// lane has candidate k, at pixel px[k] with disparity d[k]; the first wins when
// both name one pixel), join S_{it+1} unless a point already holds the pixel.
// The counters take one atomic per warp, and the two candidates' atomics and
// loads are in flight together (every lane of the warp calls this).
__device__ __forceinline__ void add_points(const MeshDev& m, const bool (&want)[2], const uint32_t (&px)[2],
                                           const float (&d)[2], int T0) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    bool isnew[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const uint32_t bit = 1u << (px[k] & 31);
        isnew[k] = want[k] && !(atomicOr(m.occ + (px[k] >> 5), bit) & bit);  // a point already there keeps it
    }
    const unsigned nm0 = __ballot_sync(0xffffffffu, isnew[0]), nm1 = __ballot_sync(0xffffffffu, isnew[1]);
    if ((nm0 | nm1) == 0u) return;
    const int nn = __popc(nm0) + __popc(nm1);
    int bv = 0, bs = 0;
    if (lane == 0) {
        bv = atomicAdd(&m.hdr->n, nn);
        bs = atomicAdd(&m.hdr->n_new, nn);
    }
    bv = __shfl_sync(0xffffffffu, bv, 0);
    bs = __shfl_sync(0xffffffffu, bs, 0);
    int t[2] = {-1, -1};
    int2 q[2];
    bool ok[2] = {false, false};
    int vid[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int o = k == 0 ? __popc(nm0 & below) : __popc(nm0) + __popc(nm1 & below);
        vid[k] = bv + o;
        q[k] = make_int2((int)(px[k] % (uint32_t)m.W), (int)(px[k] / (uint32_t)m.W));
        if (!isnew[k]) continue;
        if (vid[k] >= m.n_cap || bs + o >= m.p_cap) {
            m.hdr->err = 1;
            isnew[k] = false;
            continue;
        }
        t[k] = m.planeidx[px[k]];
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
        if (!isnew[k]) continue;
        m.pos[vid[k]] = q[k];
        m.vpass[vid[k]] = (uint8_t)m.pass;
        m.dmap[px[k]] = d[k];
        if (t[k] < 0 || t[k] >= T0) m.hdr->err = 2;  // an evaluated pixel always has a triangle
        else ok[k] = true;
    }
    const unsigned om0 = __ballot_sync(0xffffffffu, ok[0]), om1 = __ballot_sync(0xffffffffu, ok[1]);
    if ((om0 | om1) == 0u) return;
    int bp = 0;
    if (lane == 0) {
        bp = atomicAdd(&m.hdr->n_pl[0], __popc(om0) + __popc(om1));
        atomicAdd(&m.hdr->total_new, __popc(om0) + __popc(om1));
    }
    bp = __shfl_sync(0xffffffffu, bp, 0);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        if (!ok[k]) continue;
        const int o = k == 0 ? __popc(om0 & below) : __popc(om0) + __popc(om1 & below);
        m.plist[bp + o] = make_int4(vid[k], t[k], -1, pk(q[k]));
        count_pending(m, t[k], q[k]);
    }
}

// Where q lies in triangle t (packed positions tp, neighbours rt): -1 inside,
// else the edge code of the worklist record; -2 when it is not in t (an error).
__device__ __forceinline__ int classify(int4 tp, int4 rt, int2 q) {
    const int2 a = unpk(tp.x), b = unpk(tp.y), c = unpk(tp.z);
    const long long o[3] = {orient(b, c, q), orient(c, a, q), orient(a, b, q)};
    int k = -1;
    for (int i = 0; i < 3; i++) {
        if (o[i] < 0) return -2;
        if (o[i] == 0) {
            if (k >= 0) return -2;  // on two edges: a vertex (never: pixels of vertices are skipped)
            k = i;
        }
    }
    if (k < 0) return -1;
    const int r = ref_of(rt, k);
    const int n = r >= 0 ? r >> 2 : -1, j = r >= 0 ? r & 3 : 0;
    return ((n + 1) << 4) | (j << 2) | k;
}

// The triangle a pending point at q moves to when its triangle t was split in
// the round with this stamp: the piece that contains it (the pieces are named
// by t's record); t itself when t was not split; -1 when no piece holds it (an
// error).  split tells which.
__device__ __forceinline__ int relocate(const MeshDev& m, int t, int2 q, int stamp, bool& split) {
    const int4 st = m.smap[t];
    split = st.x == stamp;
    if (!split) return t;
    for (int k = 0; k < 3; k++) {
        const int r = smap_ref(st, k);
        if (r >= 0 && contains(m.tr[r >> 2].a, q)) return r >> 2;
    }
    return -1;
}

// One pair per thread-block cluster: the cluster's blocks share the pair's
// items and meet at the cluster barrier between phases, so each pair runs at
// its own pace and no barrier spans the grid.
__global__ void __launch_bounds__(kMeshThreads) k_mesh_pass(const MeshDev* __restrict__ mdg, int np) {
    cg::cluster_group cl = cg::this_cluster();
    const int nblk = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    if ((int)gridDim.x != np * nblk) {  // clusters that do not tile the pairs: no descriptor is read past np
        if (blockIdx.x == 0 && (int)threadIdx.x < np) atomicExch(&mdg[threadIdx.x].hdr->err, 4);
        return;  // every block leaves (the test is uniform over the grid)
    }
    __shared__ MeshDev sm;  // the pair's descriptor
    for (int i = threadIdx.x; i < (int)(sizeof(MeshDev) / 4); i += blockDim.x)
        reinterpret_cast<int*>(&sm)[i] = reinterpret_cast<const int*>(mdg + blockIdx.x / nblk)[i];
    __syncthreads();
    const MeshDev& m = sm;
    MeshHdr* hd = m.hdr;
    const bool lead = rank == 0 && threadIdx.x == 0;
    const int t0 = rank * blockDim.x + threadIdx.x, tstride = nblk * blockDim.x;
    const int w0 = rank * (blockDim.x >> 5) + (threadIdx.x >> 5), wstride = nblk * (blockDim.x >> 5);
    auto items = [&](int n, auto body) {
        for (int i = t0; i < n; i += tstride) body(i);
    };
    auto warp_items = [&](int n, auto body) {
        for (int i = w0; i < n; i += wstride) body(i);
    };
    const int words = words_of(m);

    // ---- 0: take over the seed mesh; reset the pass's counters
    if (lead) {
        if (m.seed_T > 0) {
            hd->n = m.seed_n;
            hd->T = m.seed_T;
            hd->stamp = 0;
            hd->err = 0;
        }
        hd->n_new = hd->n_small = hd->n_large = hd->n_items = hd->n_hull = 0;
        for (int c = 0; c < kMeshClasses; c++) hd->cls[c] = hd->cls_fill[c] = 0;
        hd->rounds = hd->flips = hd->frounds = hd->edge_ins = 0;
        hd->n_pl[0] = hd->n_pl[1] = hd->n_al[0] = hd->n_al[1] = 0;
        hd->total_new = hd->inserted = 0;
        hd->step = hd->fdone = 0;
    }
    if (m.seed_T > 0) {
        items(words, [&](int i) { m.occ[i] = 0u; });
        items(m.seed_n, [&](int i) {
            const int2 q = make_int2(m.seed_pos[2 * i], m.seed_pos[2 * i + 1]);
            m.pos[i] = q;
            m.vpass[i] = 1;
            m.dmap[(size_t)q.y * m.W + q.x] = m.seed_d[i];
        });
        items(m.seed_T, [&](int i) {
            const int4 st = m.seed_tri[i];
            put_tri(m, i,
                    make_int4(pk(make_int2(m.seed_pos[2 * st.x], m.seed_pos[2 * st.x + 1])),
                              pk(make_int2(m.seed_pos[2 * st.y], m.seed_pos[2 * st.y + 1])),
                              pk(make_int2(m.seed_pos[2 * st.z], m.seed_pos[2 * st.z + 1])), 0),
                    m.seed_opp[i]);
            m.cl[i] = ClaimRec{kNoClaim, 0ull};
            m.smap[i] = make_int4(0, -1, -1, -1);
        });
    } else {  // a mesh kept from the last pass: its claims start empty, no point pending
        items(ld_int(&hd->T), [&](int i) {
            m.cl[i] = ClaimRec{kNoClaim, 0ull};
            m.tr[i].b.z = 0;
        });
    }
    cl.sync();
    if (m.seed_T > 0)
        items(m.seed_n, [&](int i) {
            const int2 q = m.pos[i];
            const uint32_t px = (uint32_t)q.y * (uint32_t)m.W + (uint32_t)q.x;
            atomicOr(m.occ + (px >> 5), 1u << (px & 31));
        });
    cl.sync();

    // ---- 1: collect the new points (cell records in raster order of cells, or a list)
    {
        const int T0 = ld_int(&hd->T);
        const int nc = m.cg_key ? m.ncells : m.list_n;
        // whole warps iterate together (the counters are taken a warp at a time)
        for (int c = t0; c < (nc + 31) / 32 * 32; c += tstride) {
            const bool in = c < nc;
            bool want[2] = {false, false};
            uint32_t px[2] = {0u, 0u};
            float d[2] = {0.0f, 0.0f};
            if (m.cg_key) {  // the cell's C_g pick, then its accepted C_b match
                const uint32_t gk = in ? m.cg_key[c] : kNoKey, bk = in ? m.cb_key[c] : kNoKey;
                const int xd = bk != kNoKey ? m.x_d[c] : -1;
                want[0] = gk != kNoKey;
                px[0] = gk & kIdxMask;
                d[0] = want[0] ? m.cg_d[c] : 0.0f;
                want[1] = xd >= 0;
                px[1] = bk & kIdxMask;
                d[1] = (float)xd;
            } else if (in) {
                want[0] = true;
                px[0] = (uint32_t)m.list_uv[2 * c + 1] * (uint32_t)m.W + (uint32_t)m.list_uv[2 * c];
            }
            add_points(m, want, px, d, T0);
        }
    }
    cl.sync();

    // ---- 2: insertion rounds over a worklist of the points still pending; each
    // record carries the point's position, so a phase reads the record and the
    // triangle's vertices, positions and neighbours side by side.
    // A round runs over the cluster's threads with the cluster barrier between its
    // phases.  A round with no more items than a block has threads runs in block 0
    // alone, with the block barrier between its phases (far cheaper, and the
    // round's data stays in one SM), and block 0 goes on while the rounds stay that
    // small; the others wait at the cluster barrier, then read the round and step
    // counts from the header.  Most rounds are small: the worklists shrink fast and
    // the flips end in chains of a few flips a round.
    const int stamp0 = ld_int(&hd->stamp);
    int step = 0, ins_rounds = 0, flip_rounds = 0;
    const int b0 = threadIdx.x, bstride = blockDim.x;
    auto sync = [&](bool solo) {
        if (solo) __syncthreads();
        else cl.sync();
    };
    auto ins_round = [&](bool solo) {
        const int i0 = solo ? b0 : t0, is = solo ? bstride : tstride;
        auto its = [&](int n, auto body) {
            for (int i = i0; i < n; i += is) body(i);
        };
        const int stamp = stamp0 + (++step);
        const int wb = ins_rounds & 1;  // this round's worklist; survivors go to the other
        const int npl = ld_int(&hd->n_pl[wb]);
        int4* wl = m.plist + wb * m.p_cap;
        int4* wn = m.plist + (wb ^ 1) * m.p_cap;
        if (lead) hd->n_pl[wb ^ 1] = 0;
        // claim the triangle (and the neighbour across the edge the point lies on)
        its(npl, [&](int i) {
            const int4 rec = wl[i];
            const int t = rec.y;
            if (t < 0) return;
            const int2 q = unpk(rec.w);
            const TriRec R = m.tr[t];
            const int code = classify(pks_of(R), refs_of(R), q);
            if (code == -2) {  // dropped in the next phase: the loop's counts change only after a barrier
                hd->err = 2;
                wl[i].z = kDropped;
                return;
            }
            const unsigned long long key = claim_key(m.cl[t].acc, R.b.z, q, rec.x);
            m.pkey[i] = key;
            wl[i].z = code;
            atomicMin(&m.cl[t].key, key);
            if (code >= 0 && (code >> 4) > 0) atomicMin(&m.cl[(code >> 4) - 1].key, key);
        });
        sync(solo);
        // a point holding all its claims splits them
        its(npl, [&](int i) {
            const int4 rec = wl[i];
            const int t = rec.y;
            if (t < 0) return;
            const int code = rec.z;
            if (code == kDropped) {
                wl[i].y = -1;
                atomicAdd(&hd->inserted, 1);
                return;
            }
            const unsigned long long key = m.pkey[i];
            const int n = code >= 0 ? (code >> 4) - 1 : -1;
            if (m.cl[t].key != key || (n >= 0 && m.cl[n].key != key)) return;
            const bool ok = code < 0 ? split3(m, t, rec.w, stamp)
                                     : split_edge(m, t, code & 3, n, (code >> 2) & 3, rec.w, stamp);
            if (code >= 0) atomicAdd(&hd->edge_ins, 1);
            wl[i].y = ok ? -2 - t : -1;
            atomicAdd(&hd->inserted, 1);
        });
        sync(solo);
        // link the pieces to their neighbours; the others move to the piece they lie in
        // and stay on the worklist
        its(npl, [&](int i) {
            const int4 rec = wl[i];
            const int lt = rec.y;
            if (lt == -1) return;
            const int code = rec.z;
            const int n = code >= 0 ? (code >> 4) - 1 : -1;
            if (lt <= -2) {
                const int t = -2 - lt;
                const int4 st = m.smap[t];
                for (int k = 0; k < 3; k++) {
                    const int r = smap_ref(st, k);
                    if (r >= 0) relink(m, r >> 2, r & 3, stamp);
                }
                if (n >= 0) {
                    const int4 sn = m.smap[n];
                    for (int k = 0; k < 3; k++) {
                        const int r = smap_ref(sn, k);
                        if (r >= 0) relink(m, r >> 2, r & 3, stamp);
                    }
                    m.cl[n].key = kNoClaim;
                }
                m.cl[t].key = kNoClaim;
                return;
            }
            m.cl[lt].key = kNoClaim;
            if (n >= 0) m.cl[n].key = kNoClaim;
            const int2 q = unpk(rec.w);
            bool split;
            const int nt = relocate(m, lt, q, stamp, split);
            if (nt < 0) {
                hd->err = 2;
                atomicAdd(&hd->inserted, 1);
                return;
            }
            if (split) count_pending(m, nt, q);  // t's count still holds the point when t was not split
            wn[atomicAdd(&hd->n_pl[wb ^ 1], 1)] = make_int4(rec.x, nt, -1, rec.w);
        });
        sync(solo);
        ins_rounds++;
    };
    auto ins_pending = [&] {
        return ins_rounds < kMaxInsertRounds && ld_int(&hd->inserted) < ld_int(&hd->total_new);
    };
    while (ins_pending()) {
        if (ld_int(&hd->n_pl[ins_rounds & 1]) > kSoloItems) {
            ins_round(false);
            continue;
        }
        if (rank == 0) {
            do ins_round(true);
            while (ins_pending() && ld_int(&hd->n_pl[ins_rounds & 1]) <= kSoloItems);
            if (lead) {
                hd->rounds = ins_rounds;
                hd->step = step;
            }
        }
        cl.sync();
        ins_rounds = ld_int(&hd->rounds);
        step = ld_int(&hd->step);
    }
    if (ins_rounds == kMaxInsertRounds && lead) hd->err = 3;

    // ---- 3: flip rounds, once every point is in.  Round 0 checks every triangle
    // touched by the insertions; later rounds a worklist: the triangles flipped in
    // the round before and the proposers whose flip lost.  A proposal claims both
    // triangles of its edge with (round tag << 44) | (priority << 25) | edge: the
    // tag falls with each round so that a newer claim beats any older one (no
    // reset), the priority is a hash of the edge and the round; tkey[t] holds t's
    // own best proposal.  The flip of a winning edge is made by its lower slot
    // when that one proposed it, else by the other.
    if (step > 0) {
        const int T = ld_int(&hd->T);
        int flips_seen = 0;  // the flip count when the round began
        // one flip round; true when it flipped nothing (the mesh is Delaunay)
        auto flip_round = [&](bool solo) {
            const int i0 = solo ? b0 : t0, is = solo ? bstride : tstride;
            auto its = [&](int n, auto body) {
                for (int i = i0; i < n; i += is) body(i);
            };
            const int f = flip_rounds;
            const int fstep = ++step;
            const int stamp = stamp0 + fstep;
            flip_rounds++;
            const int ab = f & 1;
            const int nitems = f == 0 ? T : ld_int(&hd->n_al[ab]);
            const int* al = m.alist + ab * m.t_cap;
            int* an = m.alist + (ab ^ 1) * m.t_cap;
            if (lead) hd->n_al[ab ^ 1] = 0;
            const unsigned long long tag = (unsigned long long)(0xFFFFFu - (unsigned)fstep) << 44;
            auto tri_of = [&](int i) { return f == 0 ? i : al[i]; };
            // propose
            its(nitems, [&](int i) {
                const int t = tri_of(i);
                if (f == 0 && m.smap[t].x <= stamp0) return;  // untouched this pass: its edges are legal
                const TriRec R = m.tr[t];
                const int4 rt = refs_of(R);
                const int2 a = unpk(R.a.x), b = unpk(R.a.y), c = unpk(R.a.z);
                unsigned long long best = kNoClaim;
                for (int k = 0; k < 3; k++) {
                    const int r = ref_of(rt, k);
                    if (r < 0) continue;
                    const int n = r >> 2;
                    if (incircle_sos(a, b, c, unpk(vtx(m.tr[n].a, r & 3)))) {
                        const unsigned eid = (unsigned)(n < t ? r : mk_ref(t, k));
                        const unsigned long long key = tag | ((unsigned long long)(mix32(eid, fstep) & 0x7FFFFu) << 25) | eid;
                        atomicMin(&m.cl[t].key, key);
                        atomicMin(&m.cl[n].key, key);
                        best = min(best, key);
                    }
                }
                m.cl[t].acc = best;
            });
            sync(solo);
            // flip each winning edge once
            its(nitems, [&](int i) {
                const int t = tri_of(i);
                if (f == 0 && m.smap[t].x <= stamp0) return;
                const ClaimRec ct = m.cl[t];
                const unsigned long long key = ct.key;
                if (ct.acc != key || (key >> 44) != (tag >> 44)) return;  // t did not propose the winner
                const int tm = (int)((key & 0x1FFFFFFull) >> 2), km = (int)(key & 3);
                const int n = t == tm ? get_ref(m, t, km) >> 2 : tm;
                if (m.cl[n].key != key) return;
                if (t != tm) {
                    const ClaimRec cm = m.cl[tm];
                    if (cm.acc == key && cm.key == key) return;  // the lower slot flips it
                }
                const int r = get_ref(m, tm, km);
                flip(m, tm, km, r >> 2, r & 3, stamp);
                const int at = atomicAdd(&hd->n_al[ab ^ 1], 2);
                an[at] = tm;
                an[at + 1] = r >> 2;
                atomicAdd(&hd->flips, 1);
            });
            sync(solo);
            // the flipped triangles link their outer edges (0 and 2); proposers that lost
            // join the next worklist.  The flipped pairs fill the worklist's first
            // 2 x (this round's flips) entries; the count comes from the flip counter,
            // which no block changes in this phase (the worklist's own counter grows
            // here as the losers are appended, so a block reading it late would take
            // losers, or entries not yet written, for flipped triangles)
            const int nfl = 2 * (ld_int(&hd->flips) - flips_seen);
            its(nfl, [&](int i) {
                const int t = an[i];
                relink(m, t, 0, stamp);
                relink(m, t, 2, stamp);
            });
            its(nitems, [&](int i) {
                const int t = tri_of(i);
                if (f == 0 && m.smap[t].x <= stamp0) return;
                if (m.cl[t].acc == kNoClaim || m.smap[t].x == stamp) return;  // no proposal, or flipped
                an[atomicAdd(&hd->n_al[ab ^ 1], 1)] = t;
            });
            sync(solo);
            const int fl = ld_int(&hd->flips);
            const bool none = fl == flips_seen;
            flips_seen = fl;
            return none;
        };
        bool done = false;
        while (!done && flip_rounds < kMaxFlipRounds) {
            if (flip_rounds == 0 || ld_int(&hd->n_al[flip_rounds & 1]) > kSoloItems) {
                done = flip_round(false);
                continue;
            }
            if (rank == 0) {
                bool none;
                do none = flip_round(true);
                while (!none && flip_rounds < kMaxFlipRounds && ld_int(&hd->n_al[flip_rounds & 1]) <= kSoloItems);
                if (lead) {
                    hd->frounds = flip_rounds;
                    hd->step = step;
                    hd->fdone = none ? 1 : 0;
                }
            }
            cl.sync();
            flip_rounds = ld_int(&hd->frounds);
            step = ld_int(&hd->step);
            flips_seen = ld_int(&hd->flips);
            done = ld_int(&hd->fdone) != 0;
        }
        if (!done && lead) hd->err = 3;
    }

    const int n = ld_int(&hd->n), T = ld_int(&hd->T);
    // ---- 4: canonical ranks (the next pass is the last).  Vertex rank = vertex
    // pixels before it in raster order (the bit map's prefix); triangles grouped by
    // their smallest canonical vertex, each group ordered by the other two.
    if (m.canonical) {
        const int nch = scan_chunks(words);
        warp_items(nch, [&](int c) { scan_a(m.occ, words, m.scan, c, Popc()); });
        items(n + 1, [&](int i) { m.gcnt[i] = 0; });
        cl.sync();
        warp_items(1, [&](int) { scan_b(m.scan, nch, nullptr); });
        cl.sync();
        warp_items(nch, [&](int c) { scan_c(m.occ, m.wpre, words, m.scan, c, Popc()); });
        cl.sync();
        // the rank of the vertex at packed position k: vertex pixels before it
        auto rank_of = [&](int k) {
            const int2 q = unpk(k);
            const uint32_t px = (uint32_t)q.y * (uint32_t)m.W + (uint32_t)q.x;
            return (int)m.wpre[px >> 5] + __popc(m.occ[px >> 5] & ((1u << (px & 31)) - 1u));
        };
        items(n, [&](int v) {
            const int2 q = m.pos[v];
            const int r = rank_of(pk(q));
            m.vcanon[r] = make_int4(q.x, q.y, __float_as_int(m.dmap[(size_t)q.y * m.W + q.x]), m.vpass[v]);
            m.tpass[r] = m.vpass[v];
        });
        items(T, [&](int t) {
            const int4 tp = m.tr[t].a;
            int a = rank_of(tp.x), b = rank_of(tp.y), c = rank_of(tp.z);
            if (a > b) { const int x = a; a = b; b = x; }
            if (b > c) { const int x = b; b = c; c = x; }
            if (a > b) { const int x = a; a = b; b = x; }
            m.cl[t].acc = ((unsigned long long)(unsigned)b << 32) | (unsigned)c;
            m.tr[t].b.w = a;
            atomicAdd(m.gcnt + a, 1);
        });
        cl.sync();
        const int nchn = scan_chunks(n);
        warp_items(nchn, [&](int c) { scan_a((const uint32_t*)m.gcnt, n, m.scan, c, Ident()); });
        cl.sync();
        warp_items(1, [&](int) { scan_b(m.scan, nchn, nullptr); });
        cl.sync();
        warp_items(nchn, [&](int c) { scan_c((const uint32_t*)m.gcnt, (uint32_t*)m.gcnt, n, m.scan, c, Ident()); });
        cl.sync();
        items(T, [&](int t) {  // gcnt[i] ends at the start of group i + 1
            m.tperm[atomicAdd(m.gcnt + m.tr[t].b.w, 1)] = t;
        });
        cl.sync();
        items(n, [&](int i) {
            const int lo = i ? m.gcnt[i - 1] : 0, hi = m.gcnt[i];
            for (int x = lo + 1; x < hi; x++) {
                const int t = m.tperm[x];
                const unsigned long long kt = m.cl[t].acc;
                int y = x - 1;
                while (y >= lo && m.cl[m.tperm[y]].acc > kt) {
                    m.tperm[y + 1] = m.tperm[y];
                    y--;
                }
                m.tperm[y + 1] = t;
            }
        });
        cl.sync();
        // the support sets S_1 .. S_iters into the trace, each in canonical order: S_it is the
        // vertices that joined at pass it or before, at their rank among those (a prefix count
        // over the ranks per iteration); S_iters is every vertex, at its rank
        if (m.trace && m.iters >= 1 && m.iters <= kMeshMaxIters) {
            const int nchv = scan_chunks(n);
            int off = 0;  // floats before S_it
            for (int it = 1; it <= m.iters; it++) {
                const bool last = it == m.iters;
                if (!last) {
                    const uint32_t lim = (uint32_t)it;
                    auto le = [lim](uint32_t x) { return (int)(x <= lim); };
                    warp_items(nchv, [&](int c) { scan_a(m.tpass, n, m.scan, c, le); });
                    cl.sync();
                    warp_items(1, [&](int) { scan_b(m.scan, nchv, &hd->s_count[it]); });
                    cl.sync();
                    warp_items(nchv, [&](int c) { scan_c(m.tpass, m.tpos, n, m.scan, c, le); });
                    cl.sync();
                } else if (lead) {
                    hd->s_count[it] = n;
                }
                const int cnt = last ? n : ld_int(&hd->s_count[it]);
                if (off + 3 * cnt > m.trace_cap) {
                    if (lead) hd->err = 1;
                    break;
                }
                items(n, [&](int r) {
                    if (!last && m.tpass[r] > (uint32_t)it) return;
                    const int4 q = m.vcanon[r];
                    float* o = m.trace + off + 3 * (last ? r : (int)m.tpos[r]);
                    o[0] = (float)q.x;
                    o[1] = (float)q.y;
                    o[2] = __int_as_float(q.z);
                });
                off += 3 * cnt;
                // the next iteration's scan rewrites tpos: every write of this one first
                if (!last) cl.sync();
            }
            if (lead) hd->trace_floats = off;
        }
    }

    // ---- 5: the next pass's raster inputs (triangle id = slot, or canonical position)
    items(T, [&](int s) {
        const int t = m.canonical ? m.tperm[s] : s;
        const TriRec R = m.tr[t];
        const int4 tp = pks_of(R);
        int2 P[3] = {unpk(tp.x), unpk(tp.y), unpk(tp.z)};
        // the vertices in canonical (v, u) order, as the plane solve takes them
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2 - a; b++)
                if (vkey(P[b]) > vkey(P[b + 1])) {
                    const int2 x = P[b]; P[b] = P[b + 1]; P[b + 1] = x;
                }
        int32_t* q = m.tri_uv + 6 * (size_t)s;
        q[0] = P[0].x; q[1] = P[0].y; q[2] = P[1].x; q[3] = P[1].y; q[4] = P[2].x; q[5] = P[2].y;
        // Eq. 3 by Cramer's rule in fp64, the host's expression operation by
        // operation (each rounded on its own: no contraction into FMAs)
        const long long u0 = P[0].x, v0 = P[0].y, u1 = P[1].x, v1 = P[1].y, u2 = P[2].x, v2 = P[2].y;
        const long long det = (u1 - u0) * (v2 - v0) - (u2 - u0) * (v1 - v0);
        const double d0 = f2d(m.dmap[v0 * m.W + u0]);
        const double e1 = __dsub_rn(f2d(m.dmap[v1 * m.W + u1]), d0);
        const double e2 = __dsub_rn(f2d(m.dmap[v2 * m.W + u2]), d0);
        const double na = __dsub_rn(__dmul_rn(e1, i2d((int)(v2 - v0))), __dmul_rn(e2, i2d((int)(v1 - v0))));
        const double nb = __dsub_rn(__dmul_rn(i2d((int)(u1 - u0)), e2), __dmul_rn(i2d((int)(u2 - u0)), e1));
        const double A = __ddiv_rn(na, i2d((int)det));
        const double B = __ddiv_rn(nb, i2d((int)det));
        const double C = __dsub_rn(__dsub_rn(d0, __dmul_rn(A, i2d((int)u0))), __dmul_rn(B, i2d((int)v0)));
        m.abc[3 * (size_t)s] = d2f_rn(A);
        m.abc[3 * (size_t)s + 1] = d2f_rn(B);
        m.abc[3 * (size_t)s + 2] = d2f_rn(C);
        // raster lists: small boxes by width class, large ones by work items
        const int x0 = max(0, min(q[0], min(q[2], q[4]))), x1 = min(m.W - 1, max(q[0], max(q[2], q[4])));
        const int y0 = max(0, min(q[1], min(q[3], q[5]))), y1 = min(m.H - 1, max(q[1], max(q[3], q[5])));
        const int area = (x1 < x0 || y1 < y0) ? 0 : (x1 - x0 + 1) * (y1 - y0 + 1);
        if (area <= m.small_area) {
            const int bw = x1 - x0 + 1;
            const int cls = bw <= 1 ? 0 : min(kMeshClasses - 1, 32 - __clz(bw - 1));
            atomicAdd(&hd->cls[cls], 1);
        } else {
            const int li = atomicAdd(&hd->n_large, 1);
            m.large[li] = s;
            m.lrows[li] = ((y1 - y0) / kRasterRows + 1) * ((x1 - x0) / m.cols + 1);
        }
        // hull edges, directed with the interior on the positive side
        const int4 rt = refs_of(R);
        for (int k = 0; k < 3; k++) {
            if (ref_of(rt, k) >= 0) continue;
            const int h = atomicAdd(&hd->n_hull, 1);
            const int2 a = unpk(vtx(tp, k == 2 ? 0 : k + 1)), b = unpk(vtx(tp, k == 0 ? 2 : k - 1));
            if (h < m.n_cap) reinterpret_cast<int4*>(m.hull)[h] = make_int4(a.x, a.y, b.x, b.y);
            else hd->err = 1;
        }
    });
    cl.sync();
    // small list in class order; work-item counts of the large ones summed per chunk
    items(T, [&](int s) {
        const int32_t* q = m.tri_uv + 6 * (size_t)s;
        const int x0 = max(0, min(q[0], min(q[2], q[4]))), x1 = min(m.W - 1, max(q[0], max(q[2], q[4])));
        const int y0 = max(0, min(q[1], min(q[3], q[5]))), y1 = min(m.H - 1, max(q[1], max(q[3], q[5])));
        const int area = (x1 < x0 || y1 < y0) ? 0 : (x1 - x0 + 1) * (y1 - y0 + 1);
        if (area > m.small_area) return;
        const int bw = x1 - x0 + 1;
        const int cls = bw <= 1 ? 0 : min(kMeshClasses - 1, 32 - __clz(bw - 1));
        int off = 0;
        for (int c = 0; c < cls; c++) off += hd->cls[c];
        m.small[off + atomicAdd(&hd->cls_fill[cls], 1)] = s;
    });
    const int nl = ld_int(&hd->n_large);
    const int nchl = scan_chunks(nl);
    warp_items(nchl, [&](int c) { scan_a((const uint32_t*)m.lrows, nl, m.scan, c, Ident()); });
    cl.sync();
    warp_items(1, [&](int) {
        scan_b(m.scan, nchl, &hd->n_items);
        if ((threadIdx.x & 31) == 0) {
            int ns = 0;
            for (int c = 0; c < kMeshClasses; c++) ns += hd->cls[c];
            hd->n_small = ns;
        }
    });
    cl.sync();
    warp_items(nchl, [&](int c) { scan_c((const uint32_t*)m.lrows, (uint32_t*)m.lrows, nl, m.scan, c, Ident()); });
    if (lead) {
        hd->rounds = ins_rounds;
        hd->frounds = flip_rounds;
        hd->stamp = stamp0 + step + 1;
    }
}
}  // namespace

// ---------------------------------------------------------------- launch
cudaError_t prepare_mesh_kernels() {
    // every cluster of the launch is resident at once when np * cluster blocks fit
    // the SMs; larger launches queue clusters, which is fine (they are independent)
    return cudaFuncSetAttribute(k_mesh_pass, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

int mesh_cluster_blocks(int np) {
    int c = 1;
    while (c < 8 && np * c * 2 <= sm_count()) c *= 2;
    return c;
}

cudaError_t launch_mesh_pass(const MeshDev* md, int np, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (np > kMeshBatch) return cudaErrorInvalidValue;
    const int c = mesh_cluster_blocks(np);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(np * c));
    cfg.blockDim = dim3(kMeshThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_mesh_pass, md, np);
}

}  // namespace stereo
