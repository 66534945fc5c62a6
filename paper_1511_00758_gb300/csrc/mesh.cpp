// Host mesh step: Delaunay triangulation of the support points and the
// disparity plane of every triangle (Sec. III-A DelaunayTriangulation,
// Sec. III-B "solving a linear system", Eq. 3).
//
// Triangulation: Guibas-Stolfi divide and conquer on a quad-edge structure
// (Guibas & Stolfi, ACM TOG 1985) with exact int64 predicates, cutting
// alternately along u and v (Dwyer's alternating cuts) so subproblems stay
// near square on wide images.  The points are sorted once in each cut's
// order and every split partitions both lists stably, so no level sorts or
// selects; quad edges live in 32-byte records and removed ones are reused,
// which keeps the structure compact in cache.  Cocircular
// ties resolve by symbolic perturbation of the lifted coordinate u^2 + v^2
// (Edelsbrunner & Muecke 1990): a point of smaller canonical index (support
// points sorted by (v, u)) carries a larger perturbation.  The perturbed
// point set is in general position, so its Delaunay triangulation is unique
// and any correct algorithm returns it.
//
// Compiled with -ffp-contract=off: the plane coefficients are a fixed fp64
// expression rounded to fp32, and contraction would change their bits.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <memory>
#include <utility>
#include <vector>

#include "internal.h"

namespace stereo {
namespace {

// One quad edge: the onext links of its four directed edges (e = 4q + r;
// r = 0, 2 primal, 1, 3 dual), the origins of the two primal ones, a
// liveness flag and, once the mesh is built, which of the two primal
// directions has the outer face on its left (bit r / 2); 32 bytes, so an
// edge's whole record shares a cache line.
struct alignas(32) Quad {
    int32_t nx[4];
    int32_t org[2];
    int32_t dead;
    int32_t outer;
};

struct Mesh {
    const int32_t* P;  // (u, v) of canonical index i at P[2i], P[2i+1]
    const uint32_t* key[2];  // per-frame order keys of the points (see reroot)
    std::unique_ptr<Quad[]> q;
    int nq = 0, cap = 0;
    std::vector<int> freed;  // quad edges removed by a merge, reused first

    static int rot(int e) { return (e & ~3) | ((e + 1) & 3); }
    static int invrot(int e) { return (e & ~3) | ((e + 3) & 3); }
    static int sym(int e) { return e ^ 2; }
    int onext(int e) const { return q[e >> 2].nx[e & 3]; }
    int& nref(int e) { return q[e >> 2].nx[e & 3]; }
    int org(int e) const { return q[e >> 2].org[(e >> 1) & 1]; }
    int dest(int e) const { return q[e >> 2].org[((e >> 1) & 1) ^ 1]; }
    int oprev(int e) const { return rot(onext(rot(e))); }
    int lnext(int e) const { return rot(onext(invrot(e))); }
    int rprev(int e) const { return onext(sym(e)); }

    int64_t orient(int a, int b, int c) const {
        const int64_t ax = P[2 * a], ay = P[2 * a + 1];
        const int64_t bx = P[2 * b], by = P[2 * b + 1];
        const int64_t cx = P[2 * c], cy = P[2 * c + 1];
        return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    }
    bool ccw(int a, int b, int c) const { return orient(a, b, c) > 0; }

    // d strictly inside the circle of the positively oriented (a, b, c) in the
    // perturbed configuration.  At an exact tie the sign is that of the
    // cofactor of the smallest-index point's lifted entry in the 4x4
    // determinant with rows (u, v, u^2 + v^2, 1).
    bool incircle(int a, int b, int c, int d) const {
        if (d == a || d == b || d == c) return false;
        const int64_t dx = P[2 * d], dy = P[2 * d + 1];
        const int64_t ax = P[2 * a] - dx, ay = P[2 * a + 1] - dy;
        const int64_t bx = P[2 * b] - dx, by = P[2 * b + 1] - dy;
        const int64_t cx = P[2 * c] - dx, cy = P[2 * c + 1] - dy;
        const int64_t la = ax * ax + ay * ay, lb = bx * bx + by * by, lc = cx * cx + cy * cy;
        const int64_t det = la * (bx * cy - by * cx) - lb * (ax * cy - ay * cx) + lc * (ax * by - ay * bx);
        if (det != 0) return det > 0;
        // cofactors of the lifted column for rows a, b, c, d, taken in
        // increasing index order until one is non-zero
        int id[4] = {a, b, c, d};
        for (int r = 0; r < 4; r++) {
            int k = 0;
            for (int j = 1; j < 4; j++)
                if (id[j] < id[k]) k = j;
            int64_t cof;
            switch (k) {
                case 0: cof = orient(b, c, d); break;
                case 1: cof = -orient(a, c, d); break;
                case 2: cof = orient(a, b, d); break;
                default: cof = -orient(a, b, c); break;
            }
            if (cof != 0) return cof > 0;
            id[k] = 0x7fffffff;
        }
        return false;
    }

    int make_edge(int a, int b) {
        int k;
        if (!freed.empty()) {
            k = freed.back();
            freed.pop_back();
        } else {
            if (nq == cap) {
                const int nc = std::max(2 * cap, 64);
                std::unique_ptr<Quad[]> g(new Quad[nc]);
                if (nq) std::memcpy(g.get(), q.get(), sizeof(Quad) * (size_t)nq);
                q.swap(g);
                cap = nc;
            }
            k = nq++;
        }
        Quad& Q = q[k];
        const int e = 4 * k;
        Q.nx[0] = e;
        Q.nx[1] = e + 3;
        Q.nx[2] = e + 2;
        Q.nx[3] = e + 1;
        Q.org[0] = a;
        Q.org[1] = b;
        Q.dead = 0;
        return e;
    }
    void splice(int a, int b) {
        const int al = rot(onext(a)), be = rot(onext(b));
        std::swap(nref(a), nref(b));
        std::swap(nref(al), nref(be));
    }
    int connect(int a, int b) {
        const int e = make_edge(dest(a), org(b));
        splice(e, lnext(a));
        splice(sym(e), b);
        return e;
    }
    void remove(int e) {
        splice(e, oprev(e));
        splice(sym(e), oprev(sym(e)));
        q[e >> 2].dead = 1;
        freed.push_back(e >> 2);
    }
    bool rightof(int x, int e) const { return ccw(x, dest(e), org(e)); }
    bool leftof(int x, int e) const { return ccw(x, org(e), dest(e)); }

    // Frame 0 orders points by (u, v) lexicographically; frame 1 is the frame
    // rotated by -90 degrees, (v, -u) lexicographic, as the key
    // (v << 16) | (65535 - u).  A rotation keeps the orientation and
    // in-circle signs, so the merge logic is the same in both frames; only
    // "leftmost" and "rightmost" change.
    //
    // Walk the hull from the clockwise hull edge e (outer face on its left)
    // and return, for frame f, the counter-clockwise hull edge out of the
    // minimum vertex and the clockwise hull edge out of the maximum vertex.
    std::pair<int, int> reroot(int e, int f) const {
        const uint32_t* K = key[f];
        int emin = e, emax = e;
        int pmin = e;
        uint32_t kmin = K[org(e)], kmax = kmin;
        int prev = e, cur = lnext(e);
        for (;;) {
            const uint32_t kv = K[org(cur)];
            if (kv < kmin) {
                kmin = kv;
                emin = cur;
                pmin = prev;
            }
            if (kv > kmax) {
                kmax = kv;
                emax = cur;
            }
            if (cur == e) break;
            prev = cur;
            cur = lnext(cur);
        }
        if (emin == e) {  // find the edge that enters org(e)
            int t = e;
            while (lnext(t) != e) t = lnext(t);
            pmin = t;
        }
        return {sym(pmin), emax};
    }

    // s0, s1: the n vertex ids of this subproblem sorted in frame 0 and in
    // frame 1; both are reordered in place so that the first child's ids
    // come first, each part still sorted in both frames.  tmp: scratch for n
    // ids; side: a per-vertex mark.  Returns, in frame f, the
    // counter-clockwise hull edge out of the minimum vertex and the
    // clockwise hull edge out of the maximum vertex.  Cuts alternate between
    // the two frames so the subproblems stay close to square.
    std::pair<int, int> build(int* s0, int* s1, int n, int f, int* tmp, uint8_t* side) {
        int* sf = f == 0 ? s0 : s1;  // sorted in the cut frame
        if (n <= 3) {
            if (n == 2) {
                const int a = make_edge(sf[0], sf[1]);
                return {a, sym(a)};
            }
            const int a = make_edge(sf[0], sf[1]);
            const int b = make_edge(sf[1], sf[2]);
            splice(sym(a), b);
            if (ccw(sf[0], sf[1], sf[2])) {
                connect(b, a);
                return {a, sym(b)};
            }
            if (ccw(sf[0], sf[2], sf[1])) {
                const int c = connect(b, a);
                return {sym(c), c};
            }
            return {a, sym(b)};
        }
        const int h = n / 2;
        int* so = f == 0 ? s1 : s0;  // sorted in the other frame: split stably
        for (int i = 0; i < h; i++) side[sf[i]] = 0;
        for (int i = h; i < n; i++) side[sf[i]] = 1;
        int nl = 0, nr = h;
        for (int i = 0; i < n; i++) {
            const int v = so[i];
            if (side[v]) tmp[nr++] = v;
            else tmp[nl++] = v;
        }
        std::memcpy(so, tmp, sizeof(int) * (size_t)n);
        const int g = 1 - f;
        auto L = build(s0, s1, h, g, tmp, side);
        auto R = build(s0 + h, s1 + h, n - h, g, tmp, side);
        // hull handles of the children in this frame
        auto Lf = reroot(L.second, f);
        auto Rf = reroot(R.second, f);
        int ldo = Lf.first, ldi = Lf.second, rdi = Rf.first, rdo = Rf.second;
        // lower common tangent
        for (;;) {
            if (leftof(org(rdi), ldi)) ldi = lnext(ldi);
            else if (rightof(org(ldi), rdi)) rdi = rprev(rdi);
            else break;
        }
        int basel = connect(sym(rdi), ldi);
        if (org(ldi) == org(ldo)) ldo = sym(basel);
        if (org(rdi) == org(rdo)) rdo = basel;
        // merge upwards
        for (;;) {
            const int bo = org(basel), bd = dest(basel);
            int lc = onext(sym(basel));
            bool lv = ccw(dest(lc), bd, bo);
            if (lv) {
                int lcn = onext(lc);
                while (incircle(bd, bo, dest(lc), dest(lcn))) {
                    remove(lc);
                    lc = lcn;
                    lcn = onext(lc);
                }
                lv = ccw(dest(lc), bd, bo);
            }
            int rc = oprev(basel);
            bool rv = ccw(dest(rc), bd, bo);
            if (rv) {
                int rcp = oprev(rc);
                while (incircle(bd, bo, dest(rc), dest(rcp))) {
                    remove(rc);
                    rc = rcp;
                    rcp = oprev(rc);
                }
                rv = ccw(dest(rc), bd, bo);
            }
            if (!lv && !rv) break;
            if (!lv || (rv && incircle(dest(lc), org(lc), org(rc), dest(rc))))
                basel = connect(rc, sym(basel));
            else
                basel = connect(sym(basel), sym(lc));
        }
        return {ldo, rdo};
    }
};

}  // namespace

int delaunay(const int32_t* uv, int n, int32_t* tri, int cap) { return delaunay(uv, n, tri, cap, nullptr, nullptr); }

int delaunay(const int32_t* uv, int n, int32_t* tri, int cap, int32_t* hull, int* n_hull) {
    if (n_hull) *n_hull = 0;
    if (n < 3) return 0;
    std::unique_ptr<uint32_t[]> keys(new uint32_t[(size_t)2 * n]);
    for (int i = 0; i < n; i++) {
        const uint32_t u = (uint32_t)uv[2 * i], v = (uint32_t)uv[2 * i + 1];
        keys[i] = (u << 16) | v;
        keys[n + i] = (v << 16) | (0xFFFFu - u);
    }
    Mesh m;
    m.P = uv;
    m.key[0] = keys.get();
    m.key[1] = keys.get() + n;
    m.cap = 3 * n + 16;
    m.q.reset(new Quad[m.cap]);
    m.freed.reserve(n);
    // the vertex ids in both frames' orders: the input is in (v, u) order, so
    // frame 1 (v ascending, u descending) reverses each row's run, and frame
    // 0 (u, then v) is a stable counting sort of the input by u
    std::unique_ptr<int[]> s0(new int[n]), s1(new int[n]), tmp(new int[n]);
    std::unique_ptr<uint8_t[]> side(new uint8_t[n]);
    for (int i = 0; i < n;) {
        int j = i;
        while (j < n && uv[2 * j + 1] == uv[2 * i + 1]) j++;
        for (int k = i; k < j; k++) s1[k] = i + j - 1 - k;
        i = j;
    }
    {
        int umax = 0;
        for (int i = 0; i < n; i++) umax = std::max(umax, (int)uv[2 * i]);
        std::vector<int> cnt((size_t)umax + 2, 0);
        for (int i = 0; i < n; i++) cnt[uv[2 * i] + 1]++;
        for (int u = 0; u <= umax; u++) cnt[u + 1] += cnt[u];
        for (int i = 0; i < n; i++) s0[cnt[uv[2 * i]]++] = i;
    }
    const int ldo = m.build(s0.get(), s1.get(), n, 0, tmp.get(), side.get()).first;
    // the outer face, walked from the reverse of a hull edge: its edges are
    // the hull edges (reported tail-first in the interior's orientation)
    for (int k = 0; k < m.nq; k++) m.q[k].outer = 0;
    int nh = 0;
    {
        const int e0 = Mesh::sym(ldo);
        int e = e0;
        do {
            if (hull && nh < 2 * n) {
                hull[2 * nh] = m.dest(e);
                hull[2 * nh + 1] = m.org(e);
            }
            nh++;
            m.q[e >> 2].outer |= 1 << ((e >> 1) & 1);
            e = m.lnext(e);
        } while (e != e0 && nh <= 4 * n);
    }
    // every other face is a triangle, found once from its directed edge
    // leaving its smallest vertex (edges in memory order, so the loads of
    // the third vertex are independent), then bucketed by that vertex and
    // listed with the other two in increasing order: lexicographic output
    std::unique_ptr<int[]> first(new int[(size_t)n + 1]);
    std::fill(first.get(), first.get() + n + 1, 0);
    std::vector<int32_t> own;
    std::vector<uint64_t> bc;
    own.reserve((size_t)2 * n + 8);
    bc.reserve((size_t)2 * n + 8);
    for (int k = 0; k < m.nq; k++) {
        const Quad& Q = m.q[k];
        if (Q.dead) continue;
        for (int r = 0; r < 2; r++) {
            if ((Q.outer >> r) & 1) continue;
            const int a = Q.org[r], b = Q.org[r ^ 1];
            if (b < a) continue;
            const int c = m.dest(m.lnext(4 * k + 2 * r));
            if (c < a) continue;
            own.push_back(a);
            bc.push_back(((uint64_t)(uint32_t)std::min(b, c) << 32) | (uint32_t)std::max(b, c));
            first[a + 1]++;
        }
    }
    const int T = (int)own.size();
    if (T > cap) return -9;  // STEREO_E_CAP
    for (int i = 0; i < n; i++) first[i + 1] += first[i];
    std::unique_ptr<uint64_t[]> key(new uint64_t[(size_t)T + 1]);
    {
        std::unique_ptr<int[]> pos(new int[n]);
        std::memcpy(pos.get(), first.get(), sizeof(int) * (size_t)n);
        for (int t = 0; t < T; t++) key[pos[own[t]]++] = bc[t];
    }
    for (int a = 0; a < n; a++) {
        for (int i = first[a] + 1; i < first[a + 1]; i++) {  // insertion sort: a vertex owns few triangles
            const uint64_t kk = key[i];
            int j = i;
            for (; j > first[a] && key[j - 1] > kk; j--) key[j] = key[j - 1];
            key[j] = kk;
        }
        for (int t = first[a]; t < first[a + 1]; t++) {
            tri[3 * t] = a;
            tri[3 * t + 1] = (int32_t)(key[t] >> 32);
            tri[3 * t + 2] = (int32_t)(key[t] & 0xFFFFFFFFu);
        }
    }
    if (n_hull) *n_hull = (T > 0 && nh <= 2 * n) ? nh : 0;
    return T;
}


// Disparity plane d = a u + b v + c through the three vertices (Eq. 3), by
// Cramer's rule in fp64 with the vertices in index order, rounded to fp32.
void planes(const int32_t* uv, const float* d, const int32_t* tri, int T, float* abc) {
    for (int t = 0; t < T; t++) {
        const int i0 = tri[3 * t], i1 = tri[3 * t + 1], i2 = tri[3 * t + 2];
        const int64_t u0 = uv[2 * i0], v0 = uv[2 * i0 + 1];
        const int64_t u1 = uv[2 * i1], v1 = uv[2 * i1 + 1];
        const int64_t u2 = uv[2 * i2], v2 = uv[2 * i2 + 1];
        const int64_t det = (u1 - u0) * (v2 - v0) - (u2 - u0) * (v1 - v0);
        const double d0 = (double)d[i0];
        const double e1 = (double)d[i1] - d0;
        const double e2 = (double)d[i2] - d0;
        const double na = e1 * (double)(v2 - v0) - e2 * (double)(v1 - v0);
        const double nb = (double)(u1 - u0) * e2 - (double)(u2 - u0) * e1;
        const double A = na / (double)det;
        const double B = nb / (double)det;
        const double C = d0 - A * (double)u0 - B * (double)v0;
        abc[3 * t] = (float)A;
        abc[3 * t + 1] = (float)B;
        abc[3 * t + 2] = (float)C;
    }
}

int raster_lists(const int32_t* q, int T, int W, int H, int32_t* rows, int32_t* small, int* n_small, int small_area,
                 int cols) {
    // small triangles are listed by box width class, then by box area (a
    // counting sort), so the 32 triangles of a warp have boxes of similar
    // width and size
    std::vector<int> area_of(T, -1);
    constexpr int kClasses = 7;  // box width 1, 2, <=4, <=8, <=16, <=32, wider
    const int kKeys = kClasses * (small_area + 1);
    std::vector<int> cnt(kKeys + 1, 0);
    int s = 0;
    for (int t = 0; t < T; t++, q += 6) {
        rows[t] = s;
        const int x0 = std::max(0, std::min(q[0], std::min(q[2], q[4])));
        const int x1 = std::min(W - 1, std::max(q[0], std::max(q[2], q[4])));
        const int y0 = std::max(0, std::min(q[1], std::min(q[3], q[5])));
        const int y1 = std::min(H - 1, std::max(q[1], std::max(q[3], q[5])));
        const int area = (x1 < x0 || y1 < y0) ? 0 : (x1 - x0 + 1) * (y1 - y0 + 1);
        if (area <= small_area) {
            const int bw = x1 - x0 + 1;
            int cls = 0;
            while (cls < kClasses - 1 && (1 << cls) < bw) cls++;
            area_of[t] = cls * (small_area + 1) + area;
            cnt[area_of[t] + 1]++;
        } else {
            s += ((y1 - y0) / kRasterRows + 1) * ((x1 - x0) / cols + 1);
        }
    }
    rows[T] = s;
    for (int a = 0; a < kKeys; a++) cnt[a + 1] += cnt[a];
    for (int t = 0; t < T; t++)
        if (area_of[t] >= 0) small[cnt[area_of[t]]++] = t;
    *n_small = cnt[kKeys - 1];
    return s;
}

int small_batches(const int32_t* q, const int32_t* small, int n_small, int W, int H, int32_t* batch, int batch_area) {
    int nb = 0, cnt = 0, area = 0;
    for (int i = 0; i < n_small; i++) {
        const int32_t* t = q + 6 * (size_t)small[i];
        const int x0 = std::max(0, std::min(t[0], std::min(t[2], t[4])));
        const int x1 = std::min(W - 1, std::max(t[0], std::max(t[2], t[4])));
        const int y0 = std::max(0, std::min(t[1], std::min(t[3], t[5])));
        const int y1 = std::min(H - 1, std::max(t[1], std::max(t[3], t[5])));
        const int a = (x1 < x0 || y1 < y0) ? 1 : (x1 - x0 + 1) * (y1 - y0 + 1);
        if (cnt == 0 || cnt == 32 || area + a > batch_area) {  // open a new batch
            batch[nb++] = i;
            cnt = 0;
            area = 0;
        }
        cnt++;
        area += a;
    }
    batch[nb] = n_small;
    return nb;
}

void raster_item_tri(const int32_t* rows, int T, int32_t* item_tri) {
    for (int t = 0; t < T; t++)
        for (int i = rows[t]; i < rows[t + 1]; i++) item_tri[i] = t;
}

}  // namespace stereo
