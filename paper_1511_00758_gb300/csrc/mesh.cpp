// Host mesh step: Delaunay triangulation of the support points and the
// disparity plane of every triangle (Sec. III-A DelaunayTriangulation,
// Sec. III-B "solving a linear system", Eq. 3).
//
// Triangulation: Guibas-Stolfi divide and conquer on a quad-edge structure
// (Guibas & Stolfi, ACM TOG 1985) with exact int64 predicates, cutting
// alternately along u and v (Dwyer's alternating cuts) so subproblems stay
// near square on wide images.  Cocircular
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
#include <utility>
#include <vector>

#include "internal.h"

namespace stereo {
namespace {

struct Mesh {
    const int32_t* P;            // (u, v) of canonical index i at P[2i], P[2i+1]
    std::vector<int> nxt;        // onext of directed edge e (4 per quad edge)
    std::vector<int> org;        // origin vertex of primal edges
    std::vector<uint8_t> dead;   // per quad edge

    static int rot(int e) { return (e & ~3) | ((e + 1) & 3); }
    static int invrot(int e) { return (e & ~3) | ((e + 3) & 3); }
    static int sym(int e) { return e ^ 2; }
    int onext(int e) const { return nxt[e]; }
    int oprev(int e) const { return rot(nxt[rot(e)]); }
    int lnext(int e) const { return rot(nxt[invrot(e)]); }
    int rprev(int e) const { return nxt[sym(e)]; }
    int dest(int e) const { return org[sym(e)]; }

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
            for (int q = 1; q < 4; q++)
                if (id[q] < id[k]) k = q;
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

    int ne = 0;  // directed edges in use (4 per quad edge)

    int make_edge(int a, int b) {
        const int e = ne;
        ne += 4;
        if ((size_t)ne > nxt.size()) {
            nxt.resize(std::max<size_t>(2 * nxt.size(), 64));
            org.resize(nxt.size(), -1);
            dead.resize(nxt.size() / 4, 0);
        }
        dead[e >> 2] = 0;
        nxt[e] = e;
        nxt[e + 1] = e + 3;
        nxt[e + 2] = e + 2;
        nxt[e + 3] = e + 1;
        org[e] = a;
        org[e + 2] = b;
        return e;
    }
    void splice(int a, int b) {
        const int al = rot(nxt[a]), be = rot(nxt[b]);
        std::swap(nxt[a], nxt[b]);
        std::swap(nxt[al], nxt[be]);
    }
    int connect(int a, int b) {
        const int e = make_edge(dest(a), org[b]);
        splice(e, lnext(a));
        splice(sym(e), b);
        return e;
    }
    void remove(int e) {
        splice(e, oprev(e));
        splice(sym(e), oprev(sym(e)));
        dead[e >> 2] = 1;
    }
    bool rightof(int x, int e) const { return ccw(x, dest(e), org[e]); }
    bool leftof(int x, int e) const { return ccw(x, org[e], dest(e)); }

    // Order of frame f: frame 0 is (u, v) lexicographic; frame 1 is the
    // frame rotated by -90 degrees, (v, -u) lexicographic.  A rotation keeps
    // the orientation and in-circle signs, so the merge logic is the same in
    // both frames; only "leftmost" and "rightmost" change.
    bool less_f(int a, int b, int f) const {
        const int au = P[2 * a], av = P[2 * a + 1], bu = P[2 * b], bv = P[2 * b + 1];
        if (f == 0) return au != bu ? au < bu : av < bv;
        return av != bv ? av < bv : au > bu;
    }

    // Walk the hull from the clockwise hull edge e (outer face on its left)
    // and return, for frame f, the counter-clockwise hull edge out of the
    // minimum vertex and the clockwise hull edge out of the maximum vertex.
    std::pair<int, int> reroot(int e, int f) const {
        int emin = e, emax = e;   // clockwise edges out of the extreme vertices
        int pmin = e;             // clockwise edge into the minimum vertex
        int prev = e, cur = lnext(e);
        // one full turn around the outer face
        for (;;) {
            const int v = org[cur];
            if (less_f(v, org[emin], f)) { emin = cur; pmin = prev; }
            if (less_f(org[emax], v, f)) emax = cur;
            if (cur == e) break;
            prev = cur;
            cur = lnext(cur);
        }
        if (emin == e) {  // find the edge that enters org[e]
            int q = e;
            while (lnext(q) != e) q = lnext(q);
            pmin = q;
        }
        return {sym(pmin), emax};
    }

    // s: n vertex ids (reordered in place).  Returns, in frame f, the
    // counter-clockwise hull edge out of the minimum vertex and the clockwise
    // hull edge out of the maximum vertex.  Cuts alternate between the two
    // frames so the subproblems stay close to square.
    std::pair<int, int> build(int* s, int n, int f) {
        if (n <= 3) {
            std::sort(s, s + n, [this, f](int a, int b) { return less_f(a, b, f); });
            if (n == 2) {
                const int a = make_edge(s[0], s[1]);
                return {a, sym(a)};
            }
            const int a = make_edge(s[0], s[1]);
            const int b = make_edge(s[1], s[2]);
            splice(sym(a), b);
            if (ccw(s[0], s[1], s[2])) {
                connect(b, a);
                return {a, sym(b)};
            }
            if (ccw(s[0], s[2], s[1])) {
                const int c = connect(b, a);
                return {sym(c), c};
            }
            return {a, sym(b)};
        }
        const int h = n / 2;
        std::nth_element(s, s + h, s + n, [this, f](int a, int b) { return less_f(a, b, f); });
        const int g = 1 - f;
        auto L = build(s, h, g);
        auto R = build(s + h, n - h, g);
        // hull handles of the children in this frame
        auto Lf = reroot(L.second, f);
        auto Rf = reroot(R.second, f);
        int ldo = Lf.first, ldi = Lf.second, rdi = Rf.first, rdo = Rf.second;
        // lower common tangent
        for (;;) {
            if (leftof(org[rdi], ldi)) ldi = lnext(ldi);
            else if (rightof(org[ldi], rdi)) rdi = rprev(rdi);
            else break;
        }
        int basel = connect(sym(rdi), ldi);
        if (org[ldi] == org[ldo]) ldo = sym(basel);
        if (org[rdi] == org[rdo]) rdo = basel;
        // merge upwards
        for (;;) {
            int lc = onext(sym(basel));
            if (rightof(dest(lc), basel)) {
                while (incircle(dest(basel), org[basel], dest(lc), dest(onext(lc)))) {
                    const int t = onext(lc);
                    remove(lc);
                    lc = t;
                }
            }
            int rc = oprev(basel);
            if (rightof(dest(rc), basel)) {
                while (incircle(dest(basel), org[basel], dest(rc), dest(oprev(rc)))) {
                    const int t = oprev(rc);
                    remove(rc);
                    rc = t;
                }
            }
            const bool lv = rightof(dest(lc), basel), rv = rightof(dest(rc), basel);
            if (!lv && !rv) break;
            if (!lv || (rv && incircle(dest(lc), org[lc], org[rc], dest(rc))))
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
    Mesh m;
    m.P = uv;
    m.nxt.resize((size_t)16 * n);  // about 3n quad edges survive; make_edge grows on demand
    m.org.resize((size_t)16 * n, -1);
    m.dead.resize((size_t)4 * n, 0);
    std::vector<int> s(n);
    for (int i = 0; i < n; i++) s[i] = i;
    m.build(s.data(), n, 0);
    // faces: each triangle once, from its directed edge leaving the smallest
    // vertex; bucketed by that vertex, so the output order is lexicographic
    // after sorting the (at most a few) triangles of each bucket
    std::vector<int> first(n + 1, 0);
    std::vector<int32_t> jk;
    std::vector<int> owner;
    jk.reserve((size_t)4 * n);
    owner.reserve((size_t)2 * n);
    const int ne = m.ne;
    int nh = 0;
    for (int e = 0; e < ne; e += 2) {
        if (m.dead[e >> 2]) continue;
        const int a = m.org[e], b = m.dest(e);
        const int e2 = m.lnext(e);
        const int c = m.dest(e2);
        if (m.lnext(m.lnext(e2)) != e || !m.ccw(a, b, c)) {
            // the left face is the outside: b -> a is a hull edge with its
            // triangle on the left
            if (hull && nh < 2 * n) {
                hull[2 * nh] = b;
                hull[2 * nh + 1] = a;
            }
            nh++;
            continue;
        }
        if (!(a < b) || !(a < c)) continue;
        owner.push_back(a);
        jk.push_back(std::min(b, c));
        jk.push_back(std::max(b, c));
        first[a + 1]++;
    }
    const int T = (int)owner.size();
    if (T > cap) return -9;  // STEREO_E_CAP
    if (n_hull) *n_hull = (T > 0 && nh <= 2 * n) ? nh : 0;
    for (int i = 0; i < n; i++) first[i + 1] += first[i];
    std::vector<int> pos(first.begin(), first.end() - 1);
    std::vector<uint64_t> key(T);
    for (int t = 0; t < T; t++) key[pos[owner[t]]++] = ((uint64_t)(uint32_t)jk[2 * t] << 32) | (uint32_t)jk[2 * t + 1];
    for (int a = 0; a < n; a++) {
        std::sort(key.begin() + first[a], key.begin() + first[a + 1]);
        for (int t = first[a]; t < first[a + 1]; t++) {
            tri[3 * t] = a;
            tri[3 * t + 1] = (int32_t)(key[t] >> 32);
            tri[3 * t + 2] = (int32_t)(key[t] & 0xFFFFFFFFu);
        }
    }
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
