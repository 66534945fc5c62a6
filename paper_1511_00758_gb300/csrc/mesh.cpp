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
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
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

// One builder of a triangulation.  The quad records are shared by every
// builder of the same triangulation; each builder hands out fresh records
// from its own range [lo, hi) (so that two halves can be built at the same
// time) and reuses the records it removed first.  The mesh is a planar
// subdivision at every step, so a builder over m points never holds more than
// 3m - 3 live edges, and a range of 3m + 16 records cannot run out; a builder
// that owns the whole array (grow = true) still grows it if it ever did.
struct Mesh {
    const int32_t* P;  // (u, v) of canonical index i at P[2i], P[2i+1]
    const uint32_t* key[2];  // per-frame order keys of the points (see reroot)
    Quad* q = nullptr;
    std::unique_ptr<Quad[]>* store = nullptr;  // the owning array, when this builder may grow it
    int lo = 0, nq = 0, hi = 0;                // fresh records [lo, nq) handed out, up to hi
    bool overflow = false;
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
            if (nq >= hi) {
                if (store && lo == 0) {
                    const int nc = std::max(2 * hi, 64);
                    std::unique_ptr<Quad[]> g(new Quad[nc]);
                    if (nq) std::memcpy(g.get(), q, sizeof(Quad) * (size_t)nq);
                    store->swap(g);
                    q = store->get();
                    hi = nc;
                } else {  // unreachable (see above); keeps every access in bounds
                    overflow = true;
                    nq = hi - 1;
                }
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
        const int h = split(s0, s1, n, f, tmp, side);
        const auto L = build(s0, s1, h, 1 - f, tmp, side);
        const auto R = build(s0 + h, s1 + h, n - h, 1 - f, tmp, side);
        return merge(L, R, f);
    }

    // Splits a subproblem of n > 3 ids at the median of frame f: the first h
    // = n / 2 ids of both lists become the lower half, each part still sorted
    // in both frames.  Returns h.
    static int split(int* s0, int* s1, int n, int f, int* tmp, uint8_t* side) {
        const int h = n / 2;
        int* sf = f == 0 ? s0 : s1;  // sorted in the cut frame
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
        return h;
    }

    // Merges the triangulations of the lower (L) and upper (R) halves of a
    // frame-f split, given by their children's hull handles (in the
    // children's frame), and returns the merged hull handles in frame f.
    std::pair<int, int> merge(std::pair<int, int> L, std::pair<int, int> R, int f) {
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

// Every builder of one triangulation: the shared quad records and a bump
// allocator that gives each builder a range of its own.
struct Builders {
    const int32_t* P;
    const uint32_t* key[2];
    std::unique_ptr<Quad[]> store;
    int total = 0;
    std::atomic<int> next{0};
    std::mutex mu;
    std::vector<std::unique_ptr<Mesh>> all;

    // A builder for a subproblem of m points (grow: it is the only one).
    Mesh* make(int m, bool grow) {
        std::unique_ptr<Mesh> b(new Mesh);
        b->P = P;
        b->key[0] = key[0];
        b->key[1] = key[1];
        b->q = store.get();
        const int len = 3 * m + 16;
        b->lo = b->nq = next.fetch_add(len);
        b->hi = std::min(total, b->lo + len);
        if (grow) b->store = &store;
        Mesh* out = b.get();
        std::lock_guard<std::mutex> g(mu);
        all.push_back(std::move(b));
        return out;
    }
};

// Runs a() on this thread and b() on this thread or on a helper started by
// spawn, and returns when both have finished.  Whichever thread claims b
// first runs it, so nothing waits for a helper that never starts.
void fork_join(const Spawn& spawn, const std::function<void()>& a, const std::function<void()>& b) {
    struct Job {
        std::atomic<bool> claimed{false};
        std::mutex mu;
        std::condition_variable cv;
        bool done = false;
        const std::function<void()>* run = nullptr;
    };
    auto job = std::make_shared<Job>();
    job->run = &b;
    spawn([job] {
        if (job->claimed.exchange(true)) return;
        (*job->run)();
        {
            std::lock_guard<std::mutex> g(job->mu);
            job->done = true;
        }
        job->cv.notify_all();
    });
    a();
    if (!job->claimed.exchange(true)) {
        b();
        return;
    }
    std::unique_lock<std::mutex> g(job->mu);
    job->cv.wait(g, [&] { return job->done; });
}

constexpr int kParallelMin = 2048;  // smallest subproblem worth a second thread

// The divide and conquer, its top `depth` levels forked (the lower half of
// each split on a helper when spawn finds one); *out receives the builder of
// the top merge.  The result is the same as a single-threaded build: the same
// splits and merges, only the quad records differ.
std::pair<int, int> build_parallel(Builders& B, Mesh** out, int* s0, int* s1, int n, int f, int* tmp, uint8_t* side,
                                   int depth, const Spawn& spawn) {
    if (depth <= 0 || n < kParallelMin) {
        Mesh* m = B.make(n, false);
        *out = m;
        return m->build(s0, s1, n, f, tmp, side);
    }
    const int h = Mesh::split(s0, s1, n, f, tmp, side);
    Mesh *ml = nullptr, *mr = nullptr;
    std::pair<int, int> L, R;
    fork_join(
        spawn, [&] { R = build_parallel(B, &mr, s0 + h, s1 + h, n - h, 1 - f, tmp + h, side, depth - 1, spawn); },
        [&] { L = build_parallel(B, &ml, s0, s1, h, 1 - f, tmp, side, depth - 1, spawn); });
    Mesh* m = B.make(n, false);  // reuses the halves' removed records first
    m->freed.swap(ml->freed);
    m->freed.insert(m->freed.end(), mr->freed.begin(), mr->freed.end());
    mr->freed.clear();
    *out = m;
    return m->merge(L, R, f);
}

}  // namespace

int delaunay(const int32_t* uv, int n, int32_t* tri, int cap) { return delaunay(uv, n, tri, cap, nullptr, nullptr); }

int delaunay(const int32_t* uv, int n, int32_t* tri, int cap, int32_t* hull, int* n_hull, int depth,
             const Spawn* spawn) {
    if (n_hull) *n_hull = 0;
    if (n < 3) return 0;
    if (!spawn) depth = 0;
    depth = std::max(0, std::min(depth, 3));
    std::unique_ptr<uint32_t[]> keys(new uint32_t[(size_t)2 * n]);
    for (int i = 0; i < n; i++) {
        const uint32_t u = (uint32_t)uv[2 * i], v = (uint32_t)uv[2 * i + 1];
        keys[i] = (u << 16) | v;
        keys[n + i] = (v << 16) | (0xFFFFu - u);
    }
    Builders B;
    B.P = uv;
    B.key[0] = keys.get();
    B.key[1] = keys.get() + n;
    // one range of 3m + 16 per builder: the leaves of the forked levels cover
    // n points, and so do the merges of each forked level
    B.total = (depth + 1) * (3 * n + 16) + 16 * (2 << depth);
    B.store.reset(new Quad[B.total]);
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
    Mesh* top = nullptr;
    int ldo;
    if (depth == 0) {
        top = B.make(n, true);
        ldo = top->build(s0.get(), s1.get(), n, 0, tmp.get(), side.get()).first;
    } else {
        ldo = build_parallel(B, &top, s0.get(), s1.get(), n, 0, tmp.get(), side.get(), depth, *spawn).first;
    }
    for (const auto& b : B.all)
        if (b->overflow) return -10;  // unreachable: a range outgrown
    const Mesh& m = *top;
    Quad* const q = top->q;  // the top builder sees the array after any growth
    for (const auto& b : B.all)
        for (int k = b->lo; k < b->nq; k++) q[k].outer = 0;
    // the outer face, walked from the reverse of a hull edge: its edges are
    // the hull edges (reported tail-first in the interior's orientation)
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
            q[e >> 2].outer |= 1 << ((e >> 1) & 1);
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
    for (const auto& bl : B.all)
        for (int k = bl->lo; k < bl->nq; k++) {
            const Quad& Q = q[k];
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

void mesh_adjacency(const int32_t* uv, const int32_t* tri, int T, int32_t* ccw, int32_t* opp) {
    // every edge once per side: (smaller vertex, larger vertex) -> (t << 2) | e
    std::vector<std::pair<uint64_t, int32_t>> half((size_t)3 * T);
    for (int t = 0; t < T; t++) {
        int a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        const int64_t o = (int64_t)(uv[2 * b] - uv[2 * a]) * (uv[2 * c + 1] - uv[2 * a + 1]) -
                          (int64_t)(uv[2 * b + 1] - uv[2 * a + 1]) * (uv[2 * c] - uv[2 * a]);
        if (o < 0) std::swap(b, c);  // positive orientation
        const int v[3] = {a, b, c};
        ccw[4 * t] = a;
        ccw[4 * t + 1] = b;
        ccw[4 * t + 2] = c;
        ccw[4 * t + 3] = 0;
        opp[4 * t + 3] = 0;
        for (int e = 0; e < 3; e++) {  // edge e joins v[e + 1] and v[e + 2]
            const uint32_t x = (uint32_t)v[(e + 1) % 3], y = (uint32_t)v[(e + 2) % 3];
            const uint64_t key = x < y ? ((uint64_t)x << 32) | y : ((uint64_t)y << 32) | x;
            half[(size_t)3 * t + e] = {key, (t << 2) | e};
            opp[4 * t + e] = -1;
        }
    }
    std::sort(half.begin(), half.end());
    for (size_t i = 0; i + 1 < half.size(); i++)
        if (half[i].first == half[i + 1].first) {
            const int32_t r0 = half[i].second, r1 = half[i + 1].second;
            opp[4 * (r0 >> 2) + (r0 & 3)] = r1;
            opp[4 * (r1 >> 2) + (r1 & 3)] = r0;
            i++;
        }
}

int raster_lists(const int32_t* q, int T, int W, int H, int32_t* rows, int32_t* small, int* n_small, int small_area,
                 int cols, int32_t* small_box) {
    // small triangles are listed by box width class, then by box area (a
    // counting sort), so the 32 triangles of a warp have boxes of similar
    // width and size
    constexpr int kClasses = 7;  // box width 1, 2, <=4, <=8, <=16, <=32, wider
    const int kKeys = kClasses * (small_area + 1);
    std::unique_ptr<int32_t[]> key(new int32_t[(size_t)T + 1]);  // sort key | area << 16, or -1
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
            const int cls = bw <= 1 ? 0 : std::min(kClasses - 1, 32 - __builtin_clz((unsigned)(bw - 1)));
            const int k = cls * (small_area + 1) + area;
            key[t] = k | (area << 16);
            cnt[k + 1]++;
        } else {
            key[t] = -1;
            s += ((y1 - y0) / kRasterRows + 1) * ((x1 - x0) / cols + 1);
        }
    }
    rows[T] = s;
    for (int a = 0; a < kKeys; a++) cnt[a + 1] += cnt[a];
    for (int t = 0; t < T; t++) {
        const int32_t k = key[t];
        if (k < 0) continue;
        const int pos = cnt[k & 0xFFFF]++;
        small[pos] = t;
        if (small_box) small_box[pos] = std::max(1, k >> 16);
    }
    *n_small = cnt[kKeys - 1];
    return s;
}

int small_batches(const int32_t* small_box, int n_small, int32_t* batch, int batch_area) {
    int nb = 0, cnt = 0, area = 0;
    for (int i = 0; i < n_small; i++) {
        const int a = small_box[i];
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
