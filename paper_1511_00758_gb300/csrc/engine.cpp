// Host runtime of libstereo: the request API of include/stereo.h, a device
// arena, the continuous-batching scheduler and the stage entry points.
//
// A request runs Alg. 1: SparseStereo (census, FAST bins, epipolar match on
// the GPU), then per iteration the host mesh step (Delaunay + planes) and
// the GPU pass (raster, fused validate, resample + match).  The scheduler
// thread gathers every admitted request that is ready for a GPU stage and
// launches each stage kind once for all of them (kernels take a PairBatch);
// host mesh steps run on a worker pool meanwhile, so requests at different
// iterations overlap.  A round's launches are captured into a CUDA graph, one
// executable graph per round shape (seed stage, iteration stage or both)
// updated in place; workers with nothing queued take halves of a large
// triangulation.  max_slots = 1 gives the plain per-pair path.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "../../include/stereo.h"

using namespace stereo;

namespace {

// Default batching window with device meshes: how long a round waits for
// seed host steps still running (a few hundred microseconds each).
constexpr int kSeedWindowUs = 4000;

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Last failing CUDA call of this process (for stereo_last_error).
static std::mutex g_err_mu;
static char g_err[256] = "";
static void note_error(cudaError_t e, const char* what, int line) {
    std::lock_guard<std::mutex> g(g_err_mu);
    std::snprintf(g_err, sizeof(g_err), "%s (%d) at engine.cpp:%d: %s", cudaGetErrorName(e), (int)e, line, what);
}

#define CKQ(x)                                    \
    do {                                          \
        cudaError_t e_ = (x);                     \
        if (e_ != cudaSuccess) return e_;         \
    } while (0)

#define CK(x)                                            \
    do {                                                 \
        cudaError_t e_ = (x);                            \
        if (e_ != cudaSuccess) {                         \
            note_error(e_, #x, __LINE__);                \
            return e_;                                   \
        }                                                \
    } while (0)

// ------------------------------------------------------------------ arena
// First-fit sub-allocator over one device region (caller-provided, e.g. a
// PyTorch tensor, or one cudaMalloc).  Not thread safe: the context mutex
// guards it.
class Arena {
public:
    void init(char* base, size_t size) {
        base_ = base;
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_.clear();
        in_use_ = 0;
    }
    void* alloc(size_t bytes) {
        bytes = align_up(bytes ? bytes : 1, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_[off] = bytes;
                in_use_ += bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(void* p) {
        if (!p) return;
        size_t off = (size_t)((char*)p - base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t bytes = u->second;
        used_.erase(u);
        in_use_ -= bytes;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + bytes == nx->first) {
            bytes += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    size_t in_use() const { return in_use_; }
    size_t size() const { return size_; }

private:
    char* base_ = nullptr;
    size_t size_ = 0, in_use_ = 0;
    std::map<size_t, size_t> free_, used_;
};

// ------------------------------------------------------------------ pinned host buffers
// Pinned host buffers of finished requests, kept for the next ones: page-
// locking memory is slow and freeing it can wait for the device, so requests
// take their staging buffers from here (sizes rounded up to powers of two)
// and give them back at release.  At most kKeep bytes stay idle.
class PinnedPool {
public:
    static constexpr size_t kKeep = (size_t)2 << 30;
    void* get(size_t bytes, size_t* cap) {
        size_t want = 1 << 16;
        while (want < bytes) want <<= 1;
        {
            std::lock_guard<std::mutex> g(mu_);
            auto it = free_.find(want);
            if (it != free_.end()) {
                void* p = it->second;
                free_.erase(it);
                idle_ -= want;
                *cap = want;
                return p;
            }
        }
        void* p = nullptr;
        if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        *cap = want;
        return p;
    }
    void put(void* p, size_t cap) {
        std::lock_guard<std::mutex> g(mu_);
        if (idle_ + cap > kKeep) {
            cudaFreeHost(p);
            return;
        }
        free_.emplace(cap, p);
        idle_ += cap;
    }
    ~PinnedPool() {
        for (auto& kv : free_) cudaFreeHost(kv.second);
    }

private:
    std::mutex mu_;
    std::multimap<size_t, void*> free_;
    size_t idle_ = 0;
};

// Support-set buffers (the trace of a result) of released requests, kept for
// the next ones: a request's trace is a few hundred KB, written once.
class TracePool {
public:
    static constexpr size_t kKeep = 256;
    std::vector<float> get() {
        std::lock_guard<std::mutex> g(mu_);
        if (free_.empty()) return {};
        std::vector<float> v = std::move(free_.back());
        free_.pop_back();
        v.clear();
        return v;
    }
    void put(std::vector<float>&& v) {
        if (v.capacity() == 0) return;
        std::lock_guard<std::mutex> g(mu_);
        if (free_.size() < kKeep) free_.push_back(std::move(v));
    }

private:
    std::mutex mu_;
    std::vector<std::vector<float>> free_;
};

struct Pinned {
    void* p = nullptr;
    size_t cap = 0;
    PinnedPool* pool = nullptr;  // null: allocated and freed directly
    bool ensure(size_t bytes) {
        if (bytes <= cap) return true;
        free();
        if (pool) {
            p = pool->get(bytes, &cap);
            return p != nullptr;
        }
        size_t want = align_up(bytes + bytes / 4, 4096);
        if (cudaHostAlloc(&p, want, cudaHostAllocDefault) != cudaSuccess) {
            p = nullptr;
            return false;
        }
        cap = want;
        return true;
    }
    void free() {
        if (p) {
            if (pool) pool->put(p, cap);
            else cudaFreeHost(p);
        }
        p = nullptr;
        cap = 0;
    }
    template <class T> T* as() { return (T*)p; }
};

struct SupportPoint {
    int32_t u, v;
    float d;
};

enum State { Q_QUEUED, Q_SEED_READY, Q_RUNNING, Q_HOST, Q_ITER_READY, Q_DONE, Q_FAILED };

// Work shapes of the kernels that a context may tune (results do not depend
// on them): the raster's small-triangle threshold, warp batch area and
// large-triangle item width, the fused validate's blocks per SM and launch mode.
struct Tuning {
    int small_area = kSmallArea;
    int batch_area = kBatchArea;
    int raster_cols = kRasterCols;
    int validate_bps = 8;
    int validate_mixed = 1;
};

struct Request {
    uint64_t ticket = 0;
    int stream_id = 0;
    int W = 0, H = 0, dmax = 0, iters = 0, cell = 0;
    int it = 0, sz = 0;
    Tuning tune;              // the context's work shapes when admitted
    State state = Q_QUEUED;
    int status = STEREO_OK;
    double t_submit = 0, t_done = 0, mesh_ms = 0;
    // inputs before admission
    Pinned in_host;           // 2*W*H bytes when the caller gave host pointers
    // the caller's destinations of D_f, C_f and the mask (optional); direct ones are
    // written by the copy kernel (device pointers of page-locked or device memory)
    void* out[3] = {nullptr, nullptr, nullptr};
    bool out_direct[3] = {false, false, false};
    uint8_t* in_dev = nullptr;  // arena copy when the caller gave device pointers
    // device block
    void* block = nullptr;
    PairDev dev{};
    int ncell_max = 0;
    int32_t* pidx_buf = nullptr;  // plane-index map, written on the last pass
    uint32_t* cells_dev = nullptr;  // 4 * ncell_max words of cell records
    // triangle buffers (device) and their capacities
    void* tri_block = nullptr;
    size_t tri_block_bytes = 0;
    // host state
    std::vector<SupportPoint> S;
    std::vector<int32_t> n_support, n_tri;
    std::vector<float> trace;
    TracePool* tpool = nullptr;  // where the trace buffer comes from and goes back to
    int T = 0;
    int raster_items = 0, n_small = 0, n_hull = 0, n_batch = 0;
    Pinned st_tri;            // one mesh, laid out as tri_stage_bytes() describes
    Pinned st_kp;             // kp_uv + kp_d
    Pinned st_cells;          // cg_key, cg_d, cb_key, x_d
    bool resample_now = false;
    // The seed stage's keypoints (a few KB) are written by the kernels
    // straight into the page-locked staging buffer (device-mapped), so a seed
    // round issues no copy back for them; false when the mapping is
    // unavailable and the round copies them instead.  (Writing a pass's cell
    // records to host memory the same way made the resample slower than the
    // copy it saves: many scattered 4-byte writes over the host link.)
    bool direct_kp = false;
    int32_t* kp_dev = nullptr;  // the device block's keypoint region (the copy-back path)
    class Pool* pool = nullptr;  // the context's host workers (idle ones help triangulate)
    // device mesh (re-tessellation on the GPU after the first pass)
    bool dev_mesh = false;      // later passes' meshes are built on the device
    void* mesh_block = nullptr; // arena block of the device mesh
    MeshDev mesh{};             // its arrays (host copy of the descriptor)
    size_t seed_off = 0;        // offset of the seed mesh arrays in the staging blob (pass 1)
    Pinned st_hdr;              // the mesh header after each device pass
    void* hdr_view = nullptr;   // st_hdr's address on the device (null: copied by the copy engine)
    const void* hdr_view_of = nullptr;  // the st_hdr buffer hdr_view belongs to
    Pinned st_trace;            // device mesh: S_1 .. S_iters as (u, v, d) floats, written by the last pass
    bool dev_trace = false;     // st_trace holds the trace (the device wrote it)
    int dev_n = 0;              // vertices after the last device pass
    bool mesh_now = false;      // this round runs the device mesh pass for this request
    bool raster_dev = false;    // this round rasters the device mesh
    long long cohort = -1;      // the seed round it took part in
};

size_t block_bytes(const Request& r, int K) {
    const size_t N = (size_t)r.W * r.H;
    const size_t words = (size_t)r.H * ((r.W + 31) / 32);
    size_t b = 0;
    auto add = [&](size_t x) { b += align_up(x, 256); };
    add(N); add(N);              // L, R
    add(4 * N); add(4 * N);      // cL, cR
    add(4 * words);              // omega
    add(4 * N);                  // planeidx (FAST scores alias it)
    add(4 * N);                  // D_it
    add(4 * N); add(N); add(N);  // Df, Cf, mask
    add((size_t)kFastBins * K * 12);
    add(16 * (size_t)r.ncell_max);
    return b;
}

void carve(Request& r, int K) {
    char* p = (char*)r.block;
    const size_t N = (size_t)r.W * r.H;
    const size_t words = (size_t)r.H * ((r.W + 31) / 32);
    auto take = [&](size_t x) { char* q = p; p += align_up(x, 256); return q; };
    PairDev& d = r.dev;
    d = PairDev{};
    d.L = (const uint8_t*)take(N);
    d.R = (const uint8_t*)take(N);
    d.cL = (uint32_t*)take(4 * N);
    d.cR = (uint32_t*)take(4 * N);
    d.omega = (uint32_t*)take(4 * words);
    d.planeidx = (int32_t*)take(4 * N);
    r.pidx_buf = d.planeidx;
    d.fast_score = (int16_t*)d.planeidx;
    d.Dit = (float*)take(4 * N);
    d.Df = (float*)take(4 * N);
    d.Cf = (uint8_t*)take(N);
    d.mask = (uint8_t*)take(N);
    d.kp_uv = (int32_t*)take((size_t)kFastBins * K * 12);  // (u, v) slots, then the matches
    d.kp_d = d.kp_uv + (size_t)kFastBins * K * 2;
    r.kp_dev = d.kp_uv;
    // cell records: four arrays laid out at the current pass's cell count, so
    // one copy moves them (set per pass by set_cells)
    r.cells_dev = (uint32_t*)take(16 * (size_t)r.ncell_max);
    d.W = r.W;
    d.H = r.H;
    d.dmax = r.dmax;
    d.K = K;
}

int cells_of(int W, int H, int sz) { return ((W + sz - 1) / sz) * ((H + sz - 1) / sz); }

// ------------------------------------------------------------------ worker pool
class Pool {
public:
    void start(int n) {
        for (int i = 0; i < n; i++) th_.emplace_back([this] { loop(); });
    }
    void push(std::function<void()> f) {
        {
            std::lock_guard<std::mutex> g(mu_);
            q_.push_back(std::move(f));
        }
        cv_.notify_one();
    }
    // Many tasks under one lock, every idle worker woken at once (one wake-up per
    // task in turn spread the starts of a round's host steps over 0.2 ms).
    void push_all(std::vector<std::function<void()>>& fs) {
        if (fs.empty()) return;
        {
            std::lock_guard<std::mutex> g(mu_);
            for (auto& f : fs) q_.push_back(std::move(f));
        }
        fs.clear();
        cv_.notify_all();
    }
    // Workers waiting for a task (a hint: it may change at once).
    int idle() const { return idle_.load(std::memory_order_relaxed); }
    void stop() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
        th_.clear();
    }

private:
    void loop() {
        for (;;) {
            std::function<void()> f;
            {
                std::unique_lock<std::mutex> g(mu_);
                idle_++;
                cv_.wait(g, [this] { return stop_ || !q_.empty(); });
                idle_--;
                if (q_.empty()) return;
                f = std::move(q_.front());
                q_.pop_front();
            }
            f();
        }
    }
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<std::function<void()>> q_;
    std::vector<std::thread> th_;
    std::atomic<int> idle_{0};
    bool stop_ = false;
};

}  // namespace

struct stereo_ctx {
    PinnedPool pinned;  // first member, destroyed last (after every request's buffers came back)
    TracePool traces;
    stereo_config cfg{};
    Params prm{};
    int K = 4;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* arena_base = nullptr;
    bool own_arena = false;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1;
    std::thread sched;
    bool stop = false;
    int host_busy = 0;
    long long seed_rounds = 0;                        // seed rounds run (cohort ids)
    std::unordered_map<long long, int> cohort_busy;   // cohort -> members still in their seed host step
    std::atomic<int> mesh_steps{0};  // host mesh steps run (for the failure-injection hook)
    Pool pool;
    Pinned desc_host;
    void* desc_dev = nullptr;
    size_t desc_cap = 0;
    cudaEvent_t ev = nullptr;
    cudaStream_t copy_stream = nullptr;      // submit-time device copies (never captured)
    cudaStream_t capture_stream = nullptr;   // private stream the rounds are captured on
    // executable graphs by round shape (bit 0: seed stage, bit 1: iteration
    // stage, bit 2: timed with events), each updated in place by the next
    // round of its shape
    std::map<int, cudaGraphExec_t> graph_exec;  // by round shape
    long long rounds_seen = 0;  // for timing every profile-th round
    long long iter_rounds = 0;  // rounds with an iteration stage (for the wait-timeout test hook)
    int* err_dev = nullptr;                  // set by a device-side wait that gave up
    Pinned err_host;
    bool bulk_validate = false;              // the bulk-copy validate kernel (else the plain one)
    bool dev_mesh = true;                    // re-tessellate on the device (cfg.host_mesh == 0)
    Tuning tune;                             // kernel work shapes (defaults, or chosen by the autotuner)
    bool tuned = false;                      // tune chosen by the autotuner
    double tune_raster_us = 0, tune_validate_us = 0;
    FILE* launch_log = nullptr;              // per-launch kind and algorithmic bytes, in launch order (diagnostics)
    std::vector<cudaEvent_t> ev_pool;     // timing events of profiled launches
    std::vector<cudaEvent_t> ev_retired;  // events of the last round (still in its graph)
    stereo_stats stats{};
};

bool stereo::valid_size(int w, int h) {
    return w >= 5 && h >= 5 && w <= 8192 && h <= 8192 && (long long)w * h < (1ll << 27);
}

namespace {

bool valid_params(const stereo_config& c) {
    return c.t_lo >= 0 && c.t_lo <= c.t_hi && c.t_hi < 24 && c.t_grad >= 0 && c.t_fast >= 0 &&
           c.kp_per_bin >= 1 && c.kp_per_bin <= kMaxK && c.uniq_margin >= 0;
}

// Staging layout of one mesh: the hull edges (4 int32 each, first so they
// stay 16-byte aligned), tri_uv (6 int32) and abc (3 fp32) per triangle,
// T + 1 work item offsets, the triangle of every raster work item, the
// small triangles, then the n_batch + 1 starts of their warp batches.
size_t tri_stage_bytes(int T, int items, int n_small, int n_hull, int n_batch) {
    return (size_t)n_hull * 16 + (size_t)T * 40 + 4 + (size_t)items * 4 + (size_t)n_small * 4 +
           ((size_t)n_batch + 1) * 4;
}

// Bytes of the request's staging blob: the mesh of tri_stage_bytes(), then,
// for a device mesh, S_1's positions (8 B) and disparities (4 B) per point and
// its triangles' vertices and neighbours (16 B each per triangle).
size_t stage_bytes(const Request& r) {
    const size_t base = tri_stage_bytes(r.T, r.raster_items, r.n_small, r.n_hull, r.n_batch);
    if (!r.dev_mesh || r.seed_off == 0) return base;
    const size_t n = r.n_support.empty() ? 0 : (size_t)r.n_support.back();
    return align_up(r.seed_off + 12 * n, 16) + 32 * (size_t)r.T;
}

// Support set -> triangles, planes and raster inputs in the request's pinned
// staging buffer.  Runs on a pool thread.
int mesh_step(Request& r) {
    const int n = (int)r.S.size();
    std::vector<int32_t> P((size_t)2 * n);
    std::vector<float> D(n);
    for (int i = 0; i < n; i++) {
        P[2 * i] = r.S[i].u;
        P[2 * i + 1] = r.S[i].v;
        D[i] = r.S[i].d;
    }
    const int cap = 2 * n + 8;
    // scratch left uninitialised: every entry read below is written first
    std::unique_ptr<int32_t[]> tri(new int32_t[(size_t)3 * cap]);
    std::unique_ptr<int32_t[]> hull_v(new int32_t[(size_t)4 * n + 4]);
    int n_hull = 0;
    // workers with nothing to do (the end of a burst) take halves of a large
    // triangulation: one idle worker, the top split; three or more, the top two
    const int idle = r.pool ? r.pool->idle() : 0;
    const int depth = n < 4096 || idle == 0 ? 0 : idle >= 3 ? 2 : 1;
    Pool* pool = r.pool;
    const Spawn spawn = [pool](std::function<void()> f) { pool->push(std::move(f)); };
    int T = n >= 3 ? delaunay(P.data(), n, tri.get(), cap, hull_v.get(), &n_hull, depth, depth ? &spawn : nullptr) : 0;
    if (T < 0) return STEREO_E_INTERNAL;
    std::unique_ptr<int32_t[]> tuv_v(new int32_t[(size_t)6 * T + 1]), rows_v(new int32_t[(size_t)T + 1]),
        small_v(new int32_t[(size_t)T + 1]), box_v(new int32_t[(size_t)T + 1]);
    for (int t = 0; t < T; t++)
        for (int k = 0; k < 3; k++) {
            tuv_v[6 * t + 2 * k] = P[2 * tri[3 * t + k]];
            tuv_v[6 * t + 2 * k + 1] = P[2 * tri[3 * t + k] + 1];
        }
    int n_small = 0;
    const int items = raster_lists(tuv_v.get(), T, r.W, r.H, rows_v.get(), small_v.get(), &n_small,
                                   r.tune.small_area, r.tune.raster_cols, box_v.get());
    std::unique_ptr<int32_t[]> batch_v(new int32_t[(size_t)n_small + 1]);
    const int n_batch = small_batches(box_v.get(), n_small, batch_v.get(), r.tune.batch_area);
    // device mesh: S_1's mesh goes up with the first pass (positions, disparities, the triangles
    // in positive orientation and their neighbours), for the device to insert into
    if (T == 0) r.dev_mesh = false;
    const size_t base_bytes = tri_stage_bytes(T, items, n_small, n_hull, n_batch);
    r.seed_off = r.dev_mesh ? align_up(base_bytes, 16) : 0;
    const size_t ccw_off = align_up(r.seed_off + 12 * (size_t)n, 16);
    const size_t all_bytes = r.dev_mesh ? ccw_off + 32 * (size_t)T : base_bytes;
    if (!r.st_tri.ensure(all_bytes)) return STEREO_E_NOMEM;
    if (r.dev_mesh) {
        char* b = r.st_tri.as<char>();
        std::memcpy(b + r.seed_off, P.data(), 8 * (size_t)n);
        std::memcpy(b + r.seed_off + 8 * (size_t)n, D.data(), 4 * (size_t)n);
        mesh_adjacency(P.data(), tri.get(), T, (int32_t*)(b + ccw_off), (int32_t*)(b + ccw_off + 16 * (size_t)T));
    }
    int32_t* hull = r.st_tri.as<int32_t>();
    for (int j = 0; j < n_hull; j++) {
        const int a = hull_v[2 * j], b = hull_v[2 * j + 1];
        hull[4 * j] = P[2 * a];
        hull[4 * j + 1] = P[2 * a + 1];
        hull[4 * j + 2] = P[2 * b];
        hull[4 * j + 3] = P[2 * b + 1];
    }
    int32_t* tuv = hull + (size_t)4 * n_hull;
    float* abc = (float*)(tuv + (size_t)6 * T);
    int32_t* rows = (int32_t*)(abc + (size_t)3 * T);
    int32_t* item_tri = rows + T + 1;
    std::memcpy(tuv, tuv_v.get(), sizeof(int32_t) * 6 * (size_t)T);
    std::memcpy(rows, rows_v.get(), sizeof(int32_t) * ((size_t)T + 1));
    raster_item_tri(rows, T, item_tri);
    std::memcpy(item_tri + items, small_v.get(), sizeof(int32_t) * (size_t)n_small);
    std::memcpy(item_tri + items + n_small, batch_v.get(), sizeof(int32_t) * ((size_t)n_batch + 1));
    planes(P.data(), D.data(), tri.get(), T, abc);
    r.T = T;
    r.raster_items = items;
    r.n_small = n_small;
    r.n_batch = n_batch;
    r.n_hull = n_hull;
    r.n_support.push_back(n);
    r.n_tri.push_back(T);
    if (r.trace.capacity() == 0 && r.tpool) r.trace = r.tpool->get();
    r.trace.reserve(r.trace.size() + 3 * r.S.size());
    for (const auto& s : r.S) {
        r.trace.push_back((float)s.u);
        r.trace.push_back((float)s.v);
        r.trace.push_back(s.d);
    }
    return STEREO_OK;
}

void sort_support(std::vector<SupportPoint>& S) {
    std::sort(S.begin(), S.end(), [](const SupportPoint& a, const SupportPoint& b) {
        return a.v != b.v ? a.v < b.v : a.u < b.u;
    });
}

// Host work after the seeding stage: S_1 from the accepted keypoint matches.
int host_after_seed(stereo_ctx* c, Request& r) {
    const int nk = kFastBins * c->K;
    const int32_t* uv = r.st_kp.as<int32_t>();
    const int32_t* d = uv + 2 * nk;
    r.S.clear();
    for (int i = 0; i < nk; i++)
        if (uv[2 * i] >= 0 && d[i] >= 0) r.S.push_back({uv[2 * i], uv[2 * i + 1], (float)d[i]});
    sort_support(r.S);
    r.S.erase(std::unique(r.S.begin(), r.S.end(), [](const SupportPoint& a, const SupportPoint& b) {
                  return a.u == b.u && a.v == b.v;
              }), r.S.end());
    r.it = 1;
    r.sz = r.cell;
    return mesh_step(r);
}

// Host work after a resampling pass: S_{it+1} = S_it + C_g picks + matched X
// (Alg. 4), an existing point winning over a new one at the same pixel, in
// canonical (v, u) order, then the next mesh.  A cell's picks lie inside the
// cell, so each band of cell rows yields its new points already ordered by u
// within every pixel row; a stable bucket pass by row puts the band in (v, u)
// order, and one linear merge with the sorted old points drops the new points
// that land on an old one.  (C_g needs C < t_lo and X a pixel with C > t_hi,
// so a cell's two picks are never the same pixel.)
int host_after_iter(Request& r) {
    const int W = r.W, H = r.H, sz = r.sz;
    const int Wc = (W + sz - 1) / sz, Hc = (H + sz - 1) / sz;
    const size_t nc = (size_t)Wc * Hc;
    const uint32_t* gk = r.st_cells.as<uint32_t>();  // cg_key, cg_d, cb_key, x_d at stride nc
    const float* gd = (const float*)(gk + nc);
    const uint32_t* bk = gk + 2 * nc;
    const int32_t* xd = (const int32_t*)(gk + 3 * nc);
    std::vector<SupportPoint> fresh, band;
    fresh.reserve(2 * nc);
    band.reserve(2 * (size_t)Wc);
    std::vector<int> row_start(sz + 1);
    for (int by = 0; by < Hc; by++) {
        band.clear();
        for (int bx = 0; bx < Wc; bx++) {
            const size_t c = (size_t)by * Wc + bx;
            SupportPoint q[2];
            int k = 0;
            if (gk[c] != kNoKey) {
                const uint32_t p = gk[c] & kIdxMask;
                q[k++] = {(int32_t)(p % W), (int32_t)(p / W), gd[c]};
            }
            if (bk[c] != kNoKey && xd[c] >= 0) {
                const uint32_t p = bk[c] & kIdxMask;
                q[k++] = {(int32_t)(p % W), (int32_t)(p / W), (float)xd[c]};
            }
            if (k == 2 && q[1].v == q[0].v && q[1].u < q[0].u) std::swap(q[0], q[1]);
            for (int i = 0; i < k; i++) band.push_back(q[i]);
        }
        // stable bucket pass by pixel row within the band
        const int v0 = by * sz;
        std::fill(row_start.begin(), row_start.end(), 0);
        for (const auto& q : band) row_start[q.v - v0 + 1]++;
        for (int i = 0; i < sz; i++) row_start[i + 1] += row_start[i];
        const size_t base = fresh.size();
        fresh.resize(base + band.size());
        for (const auto& q : band) fresh[base + row_start[q.v - v0]++] = q;
    }
    auto key = [](const SupportPoint& q) { return ((int64_t)q.v << 32) | (uint32_t)q.u; };
    std::vector<SupportPoint> S;
    S.reserve(r.S.size() + fresh.size());
    size_t i = 0, j = 0;
    while (i < r.S.size() && j < fresh.size()) {
        const int64_t ki = key(r.S[i]), kj = key(fresh[j]);
        if (ki < kj) S.push_back(r.S[i++]);
        else if (kj < ki) S.push_back(fresh[j++]);
        else {  // an existing point wins
            S.push_back(r.S[i++]);
            j++;
        }
    }
    S.insert(S.end(), r.S.begin() + i, r.S.end());
    S.insert(S.end(), fresh.begin() + j, fresh.end());
    r.S.swap(S);
    r.it += 1;
    r.sz = std::max(1, r.sz / 2);
    return mesh_step(r);
}

void finish(stereo_ctx* c, Request& r, int status) {
    r.status = status;
    r.state = status == STEREO_OK ? Q_DONE : Q_FAILED;
    r.t_done = now_ms();
    c->stats.requests_done++;
    c->stats.host_mesh_ms += r.mesh_ms;
}

// Admit queued requests while the arena has room.  Called with c->mu held.
void admit(stereo_ctx* c) {
    while (!c->queue.empty() && (int)c->active.size() < c->cfg.max_slots) {
        Request* r = c->queue.front();
        size_t need = block_bytes(*r, c->K);
        void* blk = c->arena.alloc(need);
        if (!blk) {
            if (c->active.empty()) {  // cannot ever fit next to nothing
                c->queue.pop_front();
                finish(c, *r, STEREO_E_NOMEM);
                c->cv_done.notify_all();
                continue;
            }
            break;
        }
        if (c->dev_mesh && r->iters >= 2) {  // the device mesh of the passes after the first
            const int n_cap = mesh_vertex_cap(r->W, r->H, kFastBins * c->K, r->iters, r->cell);
            const int p_cap = (int)std::min<long long>(2ll * r->ncell_max, (long long)r->W * r->H);
            const size_t mb = mesh_bytes(r->W, r->H, n_cap, 2 * n_cap + 8, p_cap);
            void* mblk = c->arena.alloc(mb);
            if (!mblk) {
                c->arena.release(blk);
                if (c->active.empty()) {
                    c->queue.pop_front();
                    finish(c, *r, STEREO_E_NOMEM);
                    c->cv_done.notify_all();
                    continue;
                }
                break;
            }
            r->mesh_block = mblk;
            mesh_carve(r->mesh, mblk, r->W, r->H, n_cap, 2 * n_cap + 8, p_cap);
            r->dev_mesh = true;
        }
        c->queue.pop_front();
        r->block = blk;
        r->tune = c->tune;
        carve(*r, c->K);
        const size_t N = (size_t)r->W * r->H;
        if (r->in_dev) {  // the submit's copy is read in place (it stays until release)
            r->dev.L = r->in_dev;
            r->dev.R = r->in_dev + align_up(N, 256);
        } else {
            cudaMemcpyAsync((void*)r->dev.L, r->in_host.p, N, cudaMemcpyHostToDevice, c->stream);
            cudaMemcpyAsync((void*)r->dev.R, (char*)r->in_host.p + N, N, cudaMemcpyHostToDevice, c->stream);
        }
        r->state = Q_SEED_READY;
        c->active.push_back(r);
    }
}

// Descriptor upload for one group of pairs: PairDev[n] then per work kind
// an offset array of n + 1 ints.  Returns device pointers via out params.
// Then, for the pairs whose mesh is on the device: their PairDev and
// MeshDev for the device-mesh raster (pass >= 2), the MeshDev of those that
// re-tessellate this round.
struct Group {
    std::vector<Request*> reqs;
    const PairDev* pd = nullptr;
    const PairDev* hpd = nullptr;  // host copies of the descriptors (as uploaded)
    const int* off[WK_COUNT] = {};
    int total[WK_COUNT] = {};
    int n_mr = 0, n_mp = 0;        // pairs of the device-mesh raster and of the mesh pass
    const PairDev* mr_pd = nullptr;
    const MeshDev* mr_md = nullptr;
    const MeshDev* mp_md = nullptr;
};

void count_mesh(Group& g) {
    g.n_mr = g.n_mp = 0;
    for (Request* r : g.reqs) {
        g.n_mr += r->raster_dev ? 1 : 0;
        g.n_mp += r->mesh_now ? 1 : 0;
    }
}

size_t group_bytes(const Group& g) {
    const size_t n = g.reqs.size();
    return align_up(sizeof(PairDev) * n, 256) + WK_COUNT * align_up(sizeof(int) * (n + 1), 256) +
           align_up(sizeof(PairDev) * g.n_mr, 256) + align_up(sizeof(MeshDev) * g.n_mr, 256) +
           align_up(sizeof(MeshDev) * g.n_mp, 256);
}

void fill_group(Group& g, char* host, char* dev) {
    const size_t n = g.reqs.size();
    PairDev* hp = (PairDev*)host;
    for (size_t i = 0; i < n; i++) {
        hp[i] = g.reqs[i]->dev;
        if (!g.reqs[i]->resample_now) {  // no cell records on a pass that does not resample
            hp[i].cg_key = nullptr;
            hp[i].cb_key = nullptr;
            hp[i].Wc = hp[i].Hc = 0;
        }
    }
    g.pd = (const PairDev*)dev;
    g.hpd = hp;
    size_t off = align_up(sizeof(PairDev) * n, 256);
    for (int k = 0; k < WK_COUNT; k++) {
        int* ho = (int*)(host + off);
        int s = 0;
        for (size_t i = 0; i < n; i++) {
            ho[i] = s;
            s += work_items((WorkKind)k, hp[i]);
        }
        ho[n] = s;
        g.off[k] = (const int*)(dev + off);
        g.total[k] = s;
        off += align_up(sizeof(int) * (n + 1), 256);
    }
    PairDev* mr_pd = (PairDev*)(host + off);
    g.mr_pd = (const PairDev*)(dev + off);
    off += align_up(sizeof(PairDev) * g.n_mr, 256);
    MeshDev* mr_md = (MeshDev*)(host + off);
    g.mr_md = (const MeshDev*)(dev + off);
    off += align_up(sizeof(MeshDev) * g.n_mr, 256);
    MeshDev* mp_md = (MeshDev*)(host + off);
    g.mp_md = (const MeshDev*)(dev + off);
    off += align_up(sizeof(MeshDev) * g.n_mp, 256);
    int a = 0, b = 0;
    for (size_t i = 0; i < n; i++) {
        const Request* r = g.reqs[i];
        if (r->raster_dev) {
            mr_pd[a] = hp[i];
            mr_md[a++] = r->mesh;
        }
        if (r->mesh_now) mp_md[b++] = r->mesh;
    }
}

PairBatch batch_of(const Group& g, WorkKind k) {
    PairBatch b{};
    b.pd = g.pd;
    b.work_off = g.off[k];
    b.npairs = (int)g.reqs.size();
    b.total = g.total[k];
    b.scan_rows = g.reqs.empty() ? 0 : g.reqs[0]->dev.scan_rows;  // set alike for the whole group
    return b;
}


// Launch bookkeeping of one round: counters, algorithmic bytes and (when
// profiling) CUDA events recorded on the launching stream around each launch.
struct Launcher {
    stereo_ctx* c;
    cudaStream_t s;
    stereo_stats delta{};
    struct Timed {
        int kind;
        cudaEvent_t a, b;
        int launches;
    };
    std::vector<Timed> timed;
    int launched = 1;  // kernels issued by the current run() body (a body may set it)
    bool prof = false;  // this round's launches are timed (every profile-th round)

    cudaEvent_t event() {  // the pool is filled before each capture (at most 24 per round)
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    template <class F>
    cudaError_t run(int kind, int npairs, double bytes, F&& f) {
        cudaEvent_t a = nullptr;
        cudaError_t e;
        if (prof) {  // event nodes of the round's graph: timed on the GPU, after it
            a = event();
            if ((e = cudaEventRecordWithFlags(a, s, cudaEventRecordExternal)) != cudaSuccess) {
                note_error(e, "event record before a launch", __LINE__);
                return e;
            }
        }
        if ((e = f()) != cudaSuccess) {
            note_error(e, "kernel launch", __LINE__);
            return e;
        }
        if (prof) {
            cudaEvent_t b = event();
            if ((e = cudaEventRecordWithFlags(b, s, cudaEventRecordExternal)) != cudaSuccess) {
                note_error(e, "event record after a launch", __LINE__);
                return e;
            }
            timed.push_back({kind, a, b, launched});
        }
        if (c->launch_log)  // one line per launch; a run() body's bytes split evenly over its launches
            for (int i = 0; i < launched; i++)
                std::fprintf(c->launch_log, "%d %d %.0f\n", kind, npairs, launched ? bytes / launched : 0.0);
        delta.kernel_launches += launched;
        delta.kind_launches[kind] += launched;
        launched = 1;
        delta.kind_bytes[kind] += bytes;
        delta.batched_pairs += npairs;
        return cudaSuccess;
    }
    // after the round's synchronisation: read this round's durations; the
    // previous round's events are no longer in any graph and return to the pool.
    void collect() {
        for (cudaEvent_t ev : c->ev_retired) c->ev_pool.push_back(ev);
        c->ev_retired.clear();
        for (auto& t : timed) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
                delta.kind_ms[t.kind] += ms;
                delta.kind_timed[t.kind] += t.launches;
            }
            c->ev_retired.push_back(t.a);
            c->ev_retired.push_back(t.b);
        }
        timed.clear();
    }
};

void add_stats(stereo_stats& to, const stereo_stats& d) {
    to.kernel_launches += d.kernel_launches;
    to.batched_pairs += d.batched_pairs;
    to.gpu_rounds += d.gpu_rounds;
    to.round_ms += d.round_ms;
    to.graph_ms += d.graph_ms;
    to.exec_ms += d.exec_ms;
    to.graph_instantiations += d.graph_instantiations;
    for (int k = 0; k < STEREO_K_KINDS; k++) {
        to.kind_launches[k] += d.kind_launches[k];
        to.kind_ms[k] += d.kind_ms[k];
        to.kind_bytes[k] += d.kind_bytes[k];
        to.kind_timed[k] += d.kind_timed[k];
    }
}

// Per-request copies of a round, issued directly on the round's stream
// before and after the graph launch, so that the graph's nodes do not
// depend on how many requests the round holds.
cudaError_t issue_inputs(Group& iter, cudaStream_t s) {
    for (Request* r : iter.reqs)
        if (r->T > 0 && !r->raster_dev)
            CK(cudaMemcpyAsync((void*)r->dev.hull, r->st_tri.p, stage_bytes(*r), cudaMemcpyHostToDevice, s));
    return cudaSuccess;
}

cudaError_t issue_outputs(stereo_ctx* c, Group& seed, Group& iter, cudaStream_t s) {
    for (Request* r : seed.reqs)  // keypoint slots and their matches, one copy
        if (!r->direct_kp)
            CK(cudaMemcpyAsync(r->st_kp.p, r->dev.kp_uv, (size_t)kFastBins * c->K * 12, cudaMemcpyDeviceToHost, s));
    // the results of the requests this round finishes, into the caller's buffers, and the
    // device meshes' headers, into page-locked memory: one gather-copy launch (per
    // kCopyBatch buffers) for those the device can write, a copy each for the others
    CopyList outs{};
    auto gather = [&](const void* src, void* dst, size_t bytes) -> cudaError_t {
        outs.src[outs.count] = (const uint8_t*)src;
        outs.dst[outs.count] = (uint8_t*)dst;
        outs.n[outs.count++] = (long long)bytes;
        if (outs.count < kCopyBatch) return cudaSuccess;
        const cudaError_t e = launch_copy_list(outs, s);
        outs.count = 0;
        return e;
    };
    for (Request* r : iter.reqs) {
        if (r->mesh_now && r->hdr_view) CK(gather(r->mesh.hdr, r->hdr_view, sizeof(MeshHdr)));
        if (r->resample_now) continue;
        const size_t N = (size_t)r->W * r->H;
        const void* src[3] = {r->dev.Df, r->dev.Cf, r->dev.mask};
        const size_t bytes[3] = {4 * N, N, N};
        for (int k = 0; k < 3; k++) {
            if (!r->out[k]) continue;
            if (!r->out_direct[k]) {
                CK(cudaMemcpyAsync(r->out[k], src[k], bytes[k], cudaMemcpyDeviceToHost, s));
                continue;
            }
            CK(gather(src[k], r->out[k], bytes[k]));
        }
    }
    if (outs.count > 0) CK(launch_copy_list(outs, s));
    for (Request* r : iter.reqs) {
        if (r->mesh_now) {  // the device mesh's counters after its re-tessellation (gathered above)
            if (!r->hdr_view) CK(cudaMemcpyAsync(r->st_hdr.p, r->mesh.hdr, sizeof(MeshHdr), cudaMemcpyDeviceToHost, s));
            continue;
        }
        if (!r->resample_now) continue;
        // the four cell arrays of this pass, one copy, for the host mesh step
        const size_t nc = (size_t)r->dev.Wc * r->dev.Hc;
        CK(cudaMemcpyAsync(r->st_cells.p, r->cells_dev, 16 * nc, cudaMemcpyDeviceToHost, s));
    }
    return cudaSuccess;
}

// The kernels of one round, issued on stream s (captured into a graph): the
// seed stage's kernels when the seed group has requests, the iteration
// stage's when the iteration group has.  For a given shape the nodes are the
// same every round (the fused validate is launched a fixed number of times),
// so the previous executable graph of that shape can be updated in place.
cudaError_t record_round(stereo_ctx* c, Group& seed, Group& iter, Launcher& Lr, cudaStream_t s, size_t desc_bytes,
                         double seed_px, double cells_bytes, double raster_bytes, double validate_bytes) {
    CK(cudaMemcpyAsync(c->desc_dev, c->desc_host.p, desc_bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->err_dev, 0, sizeof(int), s));
    Params prm = c->prm;
    prm.err = c->err_dev;
    const int ns = (int)seed.reqs.size(), ni = (int)iter.reqs.size();
    // test hook: this round's bulk validate withholds its copies (its waits run out)
    prm.withhold = ni > 0 && c->bulk_validate && c->cfg.inject_wait_timeout > 0 &&
                   ++c->iter_rounds == c->cfg.inject_wait_timeout;
    if (ns > 0) {
        CKQ(Lr.run(STEREO_K_CENSUS, ns, seed_px * 10.125, [&] { return launch_census(batch_of(seed, WK_CENSUS), prm, s); }));
        CKQ(Lr.run(STEREO_K_FAST_SCORE, ns, seed_px * 3.0, [&] { return launch_fast_score(batch_of(seed, WK_FAST_SCORE), prm, s); }));
        CKQ(Lr.run(STEREO_K_FAST_BINS, ns, 0.0, [&] { return launch_fast_bins(batch_of(seed, WK_FAST_BINS), prm, s); }));
        CKQ(Lr.run(STEREO_K_MATCH_KP, ns, 0.0, [&] { return launch_match_kp(batch_of(seed, WK_MATCH_KP), prm, s); }));
    }
    if (ni == 0) {
        CK(cudaMemcpyAsync(c->err_host.p, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
        return cudaSuccess;
    }
    // the raster also resets this pass's cell records (no launch of their own): meshes
    // listed on the host (every first pass, and every pass of the host-mesh path), then
    // meshes built on the device, kMeshBatch pairs per launch
    const int n_host_raster = ni - iter.n_mr;
    if (n_host_raster > 0)
        CKQ(Lr.run(STEREO_K_RASTER, n_host_raster, raster_bytes + cells_bytes,
                   [&] { return launch_raster(batch_of(iter, WK_RASTER), s); }));
    for (int a = 0; a < iter.n_mr; a += kMeshBatch) {
        PairBatch mb{};
        mb.pd = iter.mr_pd + a;
        mb.npairs = std::min(kMeshBatch, iter.n_mr - a);
        CKQ(Lr.run(STEREO_K_RASTER, mb.npairs, n_host_raster > 0 ? 0.0 : raster_bytes + cells_bytes,
                   [&] { return launch_raster_mesh(mb, iter.mr_md + a, s); }));
    }
    CKQ(Lr.run(STEREO_K_VALIDATE, ni, validate_bytes, [&] {
        if (c->bulk_validate) return launch_validate_bulk(batch_of(iter, WK_VALIDATE_BULK), prm, s);
        const int fixed = (std::max(1, c->cfg.max_slots) + kVBatch - 1) / kVBatch;
        int n = 0, nk = 0;
        if (c->tune.validate_mixed) {
            const cudaError_t ev = launch_validate(iter.hpd, ni, WK_VALIDATE_MIXED, prm, s, &n, fixed, c->tune.validate_bps);
            if (ev != cudaSuccess) return ev;
        } else {  // one launch per cell-side class
            for (WorkKind k : kValidateKinds) {
                const cudaError_t ev = launch_validate(iter.hpd, ni, k, prm, s, &nk, fixed, c->tune.validate_bps);
                if (ev != cudaSuccess) return ev;
                n += nk;
            }
        }
        Lr.launched = n;
        return cudaSuccess;
    }));
    CKQ(Lr.run(STEREO_K_RESAMPLE, ni, 0.0, [&] { return launch_resample(batch_of(iter, WK_RESAMPLE), prm, s); }));
    for (int a = 0; a < iter.n_mp; a += kMeshBatch) {
        const int np = std::min(kMeshBatch, iter.n_mp - a);
        CKQ(Lr.run(STEREO_K_MESH, np, 0.0, [&] { return launch_mesh_pass(iter.mp_md + a, np, s); }));
    }
    CK(cudaMemcpyAsync(c->err_host.p, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    return cudaSuccess;
}

// One GPU round for the seed group and the iteration group: host-side
// preparation (buffers, descriptors), then every copy and launch of the round
// captured as one CUDA graph and replayed (the previous executable graph is
// updated in place when the topology matches), then one synchronisation.
cudaError_t gpu_round(stereo_ctx* c, Group& seed, Group& iter, Launcher& Lr) {
    cudaStream_t s = c->stream;
    double seed_px = 0, validate_bytes = 0, cells_bytes = 0, raster_bytes = 0;
    for (Request* r : seed.reqs) {
        // census and FAST strips: shorter items when few pairs share the launch (more warps)
        r->dev.scan_rows = seed.reqs.size() >= 8 ? 14 : 7;
        seed_px += (double)r->W * r->H;
        if (!r->st_kp.ensure((size_t)kFastBins * c->K * 12)) return cudaErrorMemoryAllocation;
        void* hp = nullptr;
        r->direct_kp = cudaHostGetDevicePointer(&hp, r->st_kp.p, 0) == cudaSuccess && hp;
        if (!r->direct_kp) cudaGetLastError();
        r->dev.kp_uv = r->direct_kp ? (int32_t*)hp : r->kp_dev;
        r->dev.kp_d = r->dev.kp_uv + (size_t)kFastBins * c->K * 2;
    }
    for (Request* r : iter.reqs) {
        r->raster_dev = r->dev_mesh && r->it >= 2;  // the device built this pass's mesh
        r->resample_now = r->it < r->iters;
        r->mesh_now = r->dev_mesh && r->resample_now;
        r->dev.mesh_raster = r->raster_dev ? 1 : 0;
        if (r->raster_dev) {  // raster inputs live in the device mesh
            r->dev.small_batch = nullptr;
            r->dev.n_small = r->dev.raster_items = r->dev.n_batch = 0;
            r->dev.n_hull = -1;
        }
        const size_t tri_bytes = r->raster_dev ? 0 : align_up(stage_bytes(*r) + 64, 256);
        if (!r->raster_dev && tri_bytes > r->tri_block_bytes) {
            std::lock_guard<std::mutex> g(c->mu);
            c->arena.release(r->tri_block);
            r->tri_block = c->arena.alloc(tri_bytes * 5 / 4);
            r->tri_block_bytes = r->tri_block ? tri_bytes * 5 / 4 : 0;
        }
        if (!r->raster_dev && !r->tri_block) return cudaErrorMemoryAllocation;
        char* tb = (char*)r->tri_block;
        if (!r->raster_dev) {
        r->dev.hull = (const int32_t*)tb;
        r->dev.n_hull = r->n_hull;
        tb += (size_t)r->n_hull * 16;
        r->dev.tri_uv = (const int32_t*)tb;
        r->dev.abc = (const float*)(tb + (size_t)r->T * 24);
        r->dev.tri_rows = (int32_t*)(tb + (size_t)r->T * 36);
        r->dev.item_tri = r->dev.tri_rows + r->T + 1;
        r->dev.small_tri = r->dev.tri_rows + r->T + 1 + r->raster_items;
        r->dev.small_batch = r->dev.small_tri + r->n_small;
        r->dev.n_batch = r->n_batch;
        r->dev.raster_cols = r->tune.raster_cols;
        r->dev.raster_items = r->raster_items;
        r->dev.n_small = r->n_small;
        r->dev.T = r->T;
        }
        // the LUT is an output of the last pass, and with a device mesh it locates the new points of every pass
        r->dev.planeidx = r->it == r->iters || r->dev_mesh ? r->pidx_buf : nullptr;
        set_cell_size(r->dev, r->sz);
        r->dev.first_pass = r->it == 1;
        r->dev.Wc = r->resample_now ? (r->W + r->sz - 1) / r->sz : 0;
        r->dev.Hc = r->resample_now ? (r->H + r->sz - 1) / r->sz : 0;
        {
            const size_t nc = (size_t)r->dev.Wc * r->dev.Hc;
            r->dev.cg_key = r->cells_dev;
            r->dev.cg_d = (float*)(r->cells_dev + nc);
            r->dev.cb_key = r->cells_dev + 2 * nc;
            r->dev.x_d = (int32_t*)(r->cells_dev + 3 * nc);
        }
        const double px = (double)r->W * r->H;
        raster_bytes += px * (r->dev.planeidx ? 8.0 : 4.0) + (double)r->T * 36.0;  // each pixel written once; tri_uv + abc read
        validate_bytes += px * (r->dev.first_pass ? 18.125 : 19.125);
        if (r->resample_now) {
            cells_bytes += 8.0 * r->dev.Wc * r->dev.Hc;
            if (!r->mesh_now && !r->st_cells.ensure(16 * (size_t)r->ncell_max)) return cudaErrorMemoryAllocation;
        }
        if (r->raster_dev || r->mesh_now) {  // the device mesh's fields for this pass
            MeshDev& m = r->mesh;
            m.small_area = r->tune.small_area;
            m.cols = r->tune.raster_cols;
            m.planeidx = r->pidx_buf;
            m.seed_n = m.seed_T = 0;
            m.cg_key = nullptr;
            m.ncells = 0;
            if (r->mesh_now) {
                m.cg_key = r->dev.cg_key;
                m.cg_d = r->dev.cg_d;
                m.cb_key = r->dev.cb_key;
                m.x_d = r->dev.x_d;
                m.ncells = r->dev.Wc * r->dev.Hc;
                m.pass = r->it + 1;
                m.canonical = r->it + 1 == r->iters;
                if (r->it == 1) {  // take S_1's mesh over from the staging blob uploaded this round
                    const char* base = (const char*)r->tri_block + r->seed_off;
                    const int n = r->n_support.back();
                    m.seed_pos = (const int32_t*)base;
                    m.seed_d = (const float*)(base + 8 * (size_t)n);
                    m.seed_tri = (const int4*)((const char*)r->tri_block + align_up(r->seed_off + 12 * (size_t)n, 16));
                    m.seed_opp = m.seed_tri + r->T;
                    m.seed_n = n;
                    m.seed_T = r->T;
                }
                if (!r->st_hdr.ensure(sizeof(MeshHdr))) return cudaErrorMemoryAllocation;
                if (r->hdr_view_of != r->st_hdr.p) {  // the device's view of the page-locked header
                    void* hp = nullptr;
                    if (cudaHostGetDevicePointer(&hp, r->st_hdr.p, 0) != cudaSuccess) {
                        cudaGetLastError();
                        hp = nullptr;
                    }
                    r->hdr_view = hp;
                    r->hdr_view_of = r->st_hdr.p;
                }
                m.trace = nullptr;
                m.trace_cap = 0;
                m.iters = r->iters;
                if (m.canonical) {  // the pass writes the trace into page-locked memory: room for
                    // the known S_1 .. S_it and the largest S_iters this pass can make
                    size_t known = 0;
                    for (int k : r->n_support) known += (size_t)k;
                    const size_t grow = std::min((size_t)r->W * r->H, (size_t)r->n_support.back() + 2 * (size_t)m.ncells);
                    const size_t floats = 3 * (known + grow);
                    void* hp = nullptr;
                    if (!r->st_trace.ensure(4 * floats)) return cudaErrorMemoryAllocation;
                    if (cudaHostGetDevicePointer(&hp, r->st_trace.p, 0) != cudaSuccess || !hp) {
                        cudaGetLastError();
                        return cudaErrorMemoryAllocation;
                    }
                    m.trace = (float*)hp;
                    m.trace_cap = (int)std::min(floats, (size_t)INT32_MAX);
                }
            }
        }
    }
    count_mesh(seed);
    count_mesh(iter);
    const size_t bs = group_bytes(seed), bi = group_bytes(iter);
    if (bs + bi > c->desc_cap) {
        if (c->desc_dev) cudaFree(c->desc_dev);
        c->desc_dev = nullptr;
        c->desc_cap = align_up((bs + bi) * 2, 4096);
        CK(cudaMalloc(&c->desc_dev, c->desc_cap));
        if (!c->desc_host.ensure(c->desc_cap)) return cudaErrorMemoryAllocation;
    }
    fill_group(seed, c->desc_host.as<char>(), (char*)c->desc_dev);
    fill_group(iter, c->desc_host.as<char>() + bs, (char*)c->desc_dev + bs);

    // Timing events must exist before the capture that records them.  The
    // last round's events are still referenced by its executable graph until
    // that graph has run, so they are recycled a round later; events are
    // never destroyed while the context lives, and an executable graph is
    // always updated with fresh events before it is launched again.
    // one round in every `profile`, the sampled position rotating (round r is timed when
    // r mod P == (r / P) mod P), so rounds that recur with period P are all sampled
    {
        const long long P = c->cfg.profile, r = c->rounds_seen++;
        Lr.prof = P > 0 && r % P == (r / P) % P;
    }
    if (Lr.prof)
        while (c->ev_pool.size() < 32) {
            cudaEvent_t ev = nullptr;
            CK(cudaEventCreate(&ev));
            c->ev_pool.push_back(ev);
        }
    // capture on a private stream nobody else uses, launch on the context's stream
    cudaStream_t cs = c->capture_stream;
    Lr.s = cs;  // event records belong to the captured stream too
    const double tg0 = now_ms();
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = record_round(c, seed, iter, Lr, cs, bs + bi, seed_px, cells_bytes, raster_bytes, validate_bytes);
    cudaGraph_t graph = nullptr;
    cudaError_t end = cudaStreamEndCapture(cs, &graph);
    if (err == cudaSuccess && end != cudaSuccess) {
        err = end;
        note_error(err, "cudaStreamEndCapture", __LINE__);
    }
    if (err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        for (auto& t : Lr.timed) {
            c->ev_retired.push_back(t.a);
            c->ev_retired.push_back(t.b);
        }
        Lr.timed.clear();
        return err;
    }
    // shape: stages present, timing, the launch counts of the raster kinds and the mesh pass, the
    // cluster size of the last mesh launch and the census / FAST strip rows.  An executable graph is
    // only updated in place from a graph of the same shape: the update carries new kernel arguments
    // and grids, but a mesh launch's cluster size (set from its pair count) is a launch attribute,
    // so graphs whose clusters differ are kept apart.
    const int n_mr_launch = (iter.n_mr + kMeshBatch - 1) / kMeshBatch, n_mp_launch = (iter.n_mp + kMeshBatch - 1) / kMeshBatch;
    const int last_np = iter.n_mp - (n_mp_launch - 1) * kMeshBatch;
    const int cluster = n_mp_launch > 0 ? mesh_cluster_blocks(last_np) : 0;
    const int cluster_bits = cluster >= 8 ? 3 : cluster >= 4 ? 2 : cluster >= 2 ? 1 : 0;
    const int short_strips = !seed.reqs.empty() && seed.reqs[0]->dev.scan_rows == 7 ? 1 : 0;
    const int shape = (seed.reqs.empty() ? 0 : 1) | (iter.reqs.empty() ? 0 : 2) | (Lr.prof ? 4 : 0) |
                      ((int)iter.reqs.size() > iter.n_mr ? 8 : 0) | (n_mr_launch << 4) | (n_mp_launch << 12) |
                      (cluster_bits << 24) | (short_strips << 26);
    cudaGraphExec_t& exec = c->graph_exec[shape];
    bool updated = false;
    if (exec) {
        cudaGraphExecUpdateResultInfo info{};
        updated = cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess;
        if (!updated) {
            cudaGetLastError();
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (!updated) {
        err = cudaGraphInstantiate(&exec, graph, 0);
        Lr.delta.graph_instantiations++;
    }
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        note_error(err, "cudaGraphInstantiate", __LINE__);
        exec = nullptr;
        Lr.timed.clear();
        return err;
    }
    const double tx0 = now_ms();
    Lr.delta.graph_ms += tx0 - tg0;
    CK(issue_inputs(iter, s));
    CK(cudaGraphLaunch(exec, s));
    CK(issue_outputs(c, seed, iter, s));
    CK(cudaEventRecord(c->ev, s));
    CK(cudaEventSynchronize(c->ev));
    Lr.delta.exec_ms += now_ms() - tx0;
    Lr.collect();
    Lr.delta.gpu_rounds++;
    if (*c->err_host.as<int>() != 0) {
        note_error(cudaErrorTimeout, "a bounded device-side wait gave up", __LINE__);
        return cudaErrorTimeout;
    }
    return cudaSuccess;
}

void scheduler(stereo_ctx* c) {
    cudaSetDevice(c->cfg.device);
    for (;;) {
        Group seed, iter;
        {
            std::unique_lock<std::mutex> g(c->mu);
            bool waiting = false;
            std::chrono::steady_clock::time_point deadline;
            for (;;) {
                admit(c);
                seed.reqs.clear();
                iter.reqs.clear();
                for (Request* r : c->active) {
                    if (r->state == Q_SEED_READY) seed.reqs.push_back(r);
                    else if (r->state == Q_ITER_READY) iter.reqs.push_back(r);
                }
                const size_t ready = seed.reqs.size() + iter.reqs.size();
                if (ready > 0) {
                    // batching window: others are still in their host step.  By default, with
                    // device meshes (whose only host steps are the short seed meshes), a request
                    // about to take its first pass waits for the rest of its seed cohort (the
                    // requests of the same seed round): a burst then takes every pass in the same
                    // rounds and each mesh launch serves all of it, while a request that arrived
                    // alone waits for nobody.
                    int window = 0, busy = 0;
                    if (c->cfg.batch_window_us > 0) {
                        window = c->cfg.batch_window_us;
                        busy = c->host_busy;
                    } else if (c->cfg.batch_window_us == 0 && c->dev_mesh) {
                        window = kSeedWindowUs;
                        for (Request* r : iter.reqs) {
                            auto it = c->cohort_busy.find(r->cohort);
                            if (r->it == 1 && it != c->cohort_busy.end()) busy += it->second;
                        }
                    }
                    const auto now = std::chrono::steady_clock::now();
                    if (window > 0 && busy > 0 && !c->stop) {
                        if (!waiting) {
                            waiting = true;
                            deadline = now + std::chrono::microseconds(window);
                        }
                        if (now < deadline) {
                            c->cv_sched.wait_until(g, deadline);
                            continue;
                        }
                    }
                    break;
                }
                if (c->stop && c->queue.empty() && c->host_busy == 0) return;
                c->cv_sched.wait(g);
            }
            for (Request* r : seed.reqs) r->state = Q_RUNNING;
            for (Request* r : iter.reqs) r->state = Q_RUNNING;
        }
        Launcher Lr{c, c->stream};
        const double tr0 = now_ms();
        cudaError_t e = gpu_round(c, seed, iter, Lr);
        Lr.delta.round_ms += now_ms() - tr0;
        if (e != cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            Lr.collect();
        }
        std::lock_guard<std::mutex> g(c->mu);
        add_stats(c->stats, Lr.delta);
        if (e != cudaSuccess) {
            const int rc = e == cudaErrorMemoryAllocation ? STEREO_E_NOMEM
                           : e == cudaErrorTimeout           ? STEREO_E_TIMEOUT
                                                             : STEREO_E_CUDA;
            for (Request* r : seed.reqs) finish(c, *r, rc);
            for (Request* r : iter.reqs) finish(c, *r, rc);
            cudaGetLastError();
            c->cv_done.notify_all();
            continue;
        }
        std::vector<Request*> host;
        const long long cohort = c->seed_rounds++;
        for (Request* r : seed.reqs) {
            r->cohort = cohort;
            host.push_back(r);
        }
        for (Request* r : iter.reqs) {
            if (r->mesh_now) {  // the device built the next pass's mesh: no host step
                const MeshHdr& h = *r->st_hdr.as<MeshHdr>();
                if (h.err != 0) {
                    char what[160];
                    std::snprintf(what, sizeof(what),
                                  "device mesh pass %d failed: code %d (1 capacity, 2 location, 3 round limit, 4 launch shape), "
                                  "n %d T %d new %d inserted %d/%d rounds %d", r->it, h.err, h.n, h.T, h.n_new,
                                  h.inserted, h.total_new, h.rounds);
                    note_error(cudaErrorUnknown, what, __LINE__);
                    finish(c, *r, STEREO_E_INTERNAL);
                    continue;
                }
                // algorithmic bytes of the pass: the cell records read (16 B each), the new
                // points written (16 B), the finished mesh written (72 B per triangle: vertices
                // and neighbours 32 B, raster inputs 40 B)
                c->stats.kind_bytes[STEREO_K_MESH] += 16.0 * r->dev.Wc * r->dev.Hc + 16.0 * h.n_new + 72.0 * h.T;
                c->stats.mesh_passes++;
                c->stats.mesh_insert_rounds += h.rounds;
                c->stats.mesh_flip_rounds += h.frounds;
                c->stats.mesh_flips += h.flips;
                c->stats.mesh_edge_points += h.edge_ins;
                c->stats.mesh_points += h.n - (r->dev_n > 0 ? r->dev_n : r->n_support.back());
                r->dev_n = h.n;
                r->n_support.push_back(h.n);  // S_{it+1}
                r->dev_trace = r->it + 1 == r->iters;  // the last pass wrote S_1 .. S_iters
                r->T = h.T;
                r->n_tri.push_back(h.T);
                r->it += 1;
                r->sz = std::max(1, r->sz / 2);
                r->state = Q_ITER_READY;
                continue;
            }
            if (!r->resample_now) {
                finish(c, *r, STEREO_OK);
                continue;
            }
            host.push_back(r);
        }
        std::vector<std::function<void()>> tasks;
        tasks.reserve(host.size());
        for (Request* r : host) {
            r->state = Q_HOST;
            c->host_busy++;
            const bool is_seed = r->it == 0;
            if (is_seed) c->cohort_busy[r->cohort]++;
            tasks.emplace_back([c, r, is_seed] {
                const double t0 = now_ms();
                int rc = is_seed ? host_after_seed(c, *r) : host_after_iter(*r);
                r->mesh_ms += now_ms() - t0;  // the whole host step
                if (c->cfg.inject_mesh_failure > 0 && ++c->mesh_steps == c->cfg.inject_mesh_failure)
                    rc = STEREO_E_INTERNAL;  // test hook: this host step reports a failure
                std::lock_guard<std::mutex> g2(c->mu);
                c->host_busy--;
                if (is_seed) {
                    auto cb = c->cohort_busy.find(r->cohort);
                    if (cb != c->cohort_busy.end() && --cb->second <= 0) c->cohort_busy.erase(cb);
                }
                if (rc != STEREO_OK) finish(c, *r, rc);
                else r->state = Q_ITER_READY;
                c->cv_sched.notify_all();
                c->cv_done.notify_all();
            });
        }
        c->pool.push_all(tasks);
        c->cv_done.notify_all();
    }
}

}  // namespace

// ====================================================================== C ABI
// ------------------------------------------------------------------ autotuner
// Times the kernels' work-shape candidates on a synthetic round and keeps the
// fastest.  None of the shapes changes a result, so the choice only moves
// time.  The round: 8 pairs of tune_w x tune_h sharing one jittered-lattice
// mesh as dense as a late pass (one point per 6x6 pixels), each with its own
// outputs; for the validate, random census codes with the right image a few
// pixels shifted (so cells get C_g and C_b keys), random Omega_I bits and two
// cell-side classes (8 and 4) in the batch.  Buffers are allocated for the
// tuning only and freed before create returns.
namespace {

struct TuneBuf {
    std::vector<void*> ptrs;
    ~TuneBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    T* alloc(size_t n) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(n * sizeof(T), 256)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return (T*)p;
    }
};

// Minimum over reps timed runs of f (after one untimed run), in microseconds;
// negative on a CUDA error.
template <class F>
double time_runs(cudaStream_t s, cudaEvent_t a, cudaEvent_t b, int reps, F&& f) {
    if (f() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return -1.0;
    double best = 1e30;
    for (int i = 0; i < reps; i++) {
        cudaEventRecord(a, s);
        if (f() != cudaSuccess) return -1.0;
        cudaEventRecord(b, s);
        if (cudaEventSynchronize(b) != cudaSuccess) return -1.0;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, 1e3 * (double)ms);
    }
    return best;
}

}  // namespace

cudaError_t autotune(stereo_ctx* c) {
    const int W = c->cfg.tune_w > 0 ? c->cfg.tune_w : 1242, H = c->cfg.tune_h > 0 ? c->cfg.tune_h : 375;
    if (!valid_size(W, H)) return cudaErrorInvalidValue;
    const size_t N = (size_t)W * H;
    const int NP = (int)std::max<size_t>(1, std::min<size_t>(8, ((size_t)512 << 20) / (N * 32)));
    cudaStream_t s = c->stream;
    // the mesh: canonical (v, u) order, no duplicates
    std::vector<int32_t> P;
    std::vector<float> D;
    uint32_t seed = 0x5EEDu;
    auto rnd = [&]() {
        seed = seed * 1664525u + 1013904223u;
        return seed >> 8;
    };
    std::vector<std::pair<int, int>> pts;
    for (int v = 0; v < H; v += 6)
        for (int u = 0; u < W; u += 6)
            pts.push_back({std::min(H - 1, v + (int)(rnd() % 6)), std::min(W - 1, u + (int)(rnd() % 6))});
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    const int n = (int)pts.size();
    for (auto& q : pts) {
        P.push_back(q.second);
        P.push_back(q.first);
        D.push_back(20.0f + 0.01f * q.second + 0.02f * q.first + 0.001f * (float)(rnd() % 1000));
    }
    const int cap = 2 * n + 8;
    std::vector<int32_t> tri((size_t)3 * cap), hull_v((size_t)4 * n + 4);
    int n_hull = 0;
    const int T = delaunay(P.data(), n, tri.data(), cap, hull_v.data(), &n_hull);
    if (T <= 0) return cudaErrorInvalidValue;
    std::vector<int32_t> tuv((size_t)6 * T);
    for (int t = 0; t < T; t++)
        for (int k = 0; k < 3; k++) {
            tuv[6 * t + 2 * k] = P[2 * tri[3 * t + k]];
            tuv[6 * t + 2 * k + 1] = P[2 * tri[3 * t + k] + 1];
        }
    std::vector<float> abc((size_t)3 * T);
    planes(P.data(), D.data(), tri.data(), T, abc.data());
    std::vector<int32_t> hull((size_t)4 * n_hull);
    for (int j = 0; j < n_hull; j++) {
        const int a = hull_v[2 * j], b = hull_v[2 * j + 1];
        hull[4 * j] = P[2 * a];
        hull[4 * j + 1] = P[2 * a + 1];
        hull[4 * j + 2] = P[2 * b];
        hull[4 * j + 3] = P[2 * b + 1];
    }
    TuneBuf buf;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (cudaEventCreate(&ea) != cudaSuccess || cudaEventCreate(&eb) != cudaSuccess) return cudaErrorUnknown;
    struct Events {
        cudaEvent_t a, b;
        ~Events() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } evs{ea, eb};
    float* dit = buf.alloc<float>(N * NP);
    int32_t* pidx = buf.alloc<int32_t>(N * NP);
    PairDev* desc = buf.alloc<PairDev>(NP);
    int* off = buf.alloc<int>(NP + 1);
    if (!dit || !pidx || !desc || !off) return cudaErrorMemoryAllocation;

    // raster: every (small-triangle threshold, batch area, item width)
    const int kSmall[] = {128, 256, 512}, kBatch[] = {512, 1024, 2048}, kCols[] = {64, 128, 256};
    std::vector<int32_t> rows((size_t)T + 1), small((size_t)T + 1), box((size_t)T + 1), batch((size_t)T + 2);
    std::vector<char> blob;
    char* blob_dev = nullptr;
    size_t blob_cap = 0;
    std::vector<PairDev> pd(NP);
    auto stage = [&](int sa, int ba, int cols) -> cudaError_t {  // host lists + upload + descriptors
        int n_small = 0;
        const int items = raster_lists(tuv.data(), T, W, H, rows.data(), small.data(), &n_small, sa, cols, box.data());
        const int n_batch = small_batches(box.data(), n_small, batch.data(), ba);
        const size_t bytes = tri_stage_bytes(T, items, n_small, n_hull, n_batch);
        blob.assign(bytes, 0);
        char* q = blob.data();
        std::memcpy(q, hull.data(), (size_t)16 * n_hull);
        int32_t* t_uv = (int32_t*)(q + (size_t)16 * n_hull);
        float* t_abc = (float*)(t_uv + (size_t)6 * T);
        int32_t* t_rows = (int32_t*)(t_abc + (size_t)3 * T);
        int32_t* t_item = t_rows + T + 1;
        std::memcpy(t_uv, tuv.data(), (size_t)24 * T);
        std::memcpy(t_abc, abc.data(), (size_t)12 * T);
        std::memcpy(t_rows, rows.data(), (size_t)4 * (T + 1));
        raster_item_tri(t_rows, T, t_item);
        std::memcpy(t_item + items, small.data(), (size_t)4 * n_small);
        std::memcpy(t_item + items + n_small, batch.data(), (size_t)4 * (n_batch + 1));
        if (bytes > blob_cap) {
            blob_dev = buf.alloc<char>(bytes * 2);
            blob_cap = blob_dev ? bytes * 2 : 0;
            if (!blob_dev) return cudaErrorMemoryAllocation;
        }
        cudaError_t e = cudaMemcpy(blob_dev, blob.data(), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
        std::vector<int> o(NP + 1, 0);
        for (int i = 0; i < NP; i++) {
            PairDev p{};
            p.W = W;
            p.H = H;
            p.T = T;
            p.hull = (const int32_t*)blob_dev;
            p.n_hull = n_hull;
            p.tri_uv = (const int32_t*)(blob_dev + (size_t)16 * n_hull);
            p.abc = (const float*)(p.tri_uv + (size_t)6 * T);
            p.tri_rows = (int32_t*)(p.abc + (size_t)3 * T);
            p.item_tri = p.tri_rows + T + 1;
            p.small_tri = p.tri_rows + T + 1 + items;
            p.small_batch = p.small_tri + n_small;
            p.n_small = n_small;
            p.n_batch = n_batch;
            p.raster_items = items;
            p.raster_cols = cols;
            p.planeidx = pidx + N * i;
            p.Dit = dit + N * i;
            pd[i] = p;
            o[i + 1] = o[i] + work_items(WK_RASTER, p);
        }
        if ((e = cudaMemcpy(desc, pd.data(), sizeof(PairDev) * NP, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        return cudaMemcpy(off, o.data(), sizeof(int) * (NP + 1), cudaMemcpyHostToDevice);
    };
    auto raster_batch = [&]() {
        PairBatch b{};
        b.pd = desc;
        b.work_off = off;
        b.npairs = NP;
        int o = 0;
        for (int i = 0; i < NP; i++) o += work_items(WK_RASTER, pd[i]);
        b.total = o;
        return b;
    };
    // A shape replaces the defaults only when it is measurably faster (by kTuneMargin):
    // the candidates often time within noise of each other on the tuning round, and the
    // small-triangle threshold also shapes the lists of the later passes' meshes, which
    // this round does not time.
    // Every candidate is timed in two sweeps over all of them and keeps its better time, so
    // that a drift during one sweep (clocks settling on a fresh device) favours none.
    constexpr double kTuneMargin = 0.97;
    constexpr int kSweeps = 2;
    Tuning best = c->tune;
    double best_r = 1e30, default_r = -1.0;
    std::vector<double> cand_us;
    for (int sweep = 0; sweep < kSweeps; sweep++) {
        int ci = 0;
        for (int sa : kSmall)
            for (int ba : kBatch)
                for (int cols : kCols) {
                    cudaError_t e = stage(sa, ba, cols);
                    if (e != cudaSuccess) return e;
                    const PairBatch b = raster_batch();
                    double us = time_runs(s, ea, eb, 3, [&] { return launch_raster(b, s); });
                    if (us < 0) return cudaErrorUnknown;
                    if (sweep == 0) cand_us.push_back(us);
                    us = cand_us[ci] = std::min(cand_us[ci], us);
                    ci++;
                    if (sweep + 1 < kSweeps) continue;
                    if (sa == kSmallArea && ba == kBatchArea && cols == kRasterCols) default_r = us;
                    if (us < best_r) {
                        best_r = us;
                        best.small_area = sa;
                        best.batch_area = ba;
                        best.raster_cols = cols;
                    }
                }
    }
    if (default_r > 0 && best_r > kTuneMargin * default_r) {
        best.small_area = kSmallArea;
        best.batch_area = kBatchArea;
        best.raster_cols = kRasterCols;
        best_r = default_r;
    }
    cudaError_t e = stage(best.small_area, best.batch_area, best.raster_cols);  // D_it for the validate
    if (e != cudaSuccess) return e;
    {
        const PairBatch b = raster_batch();
        if ((e = launch_raster(b, s)) != cudaSuccess || (e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    // validate: blocks per SM and launch mode, on two cell-side classes
    const int words = (W + 31) / 32;
    const int Wc4 = (W + 3) / 4, Hc4 = (H + 3) / 4;
    uint32_t* cL = buf.alloc<uint32_t>(N * NP);
    uint32_t* cR = buf.alloc<uint32_t>(N * NP);
    uint32_t* om = buf.alloc<uint32_t>((size_t)words * H * NP);
    float* Df = buf.alloc<float>(N * NP);
    uint8_t* Cf = buf.alloc<uint8_t>(N * NP);
    uint8_t* mask = buf.alloc<uint8_t>(N * NP);
    uint32_t* cells = buf.alloc<uint32_t>((size_t)2 * Wc4 * Hc4 * NP);
    if (!cL || !cR || !om || !Df || !Cf || !mask || !cells) return cudaErrorMemoryAllocation;
    {
        std::vector<uint32_t> hl(N), hr(N), ho((size_t)words * H);
        for (size_t i = 0; i < N; i++) hl[i] = rnd() & 0xFFFFFFu;
        for (size_t i = 0; i < N; i++) {  // the right image: a few pixels of shift, some noise
            const size_t u = i % W;
            hr[i] = (u + 3 < (size_t)W && rnd() % 8) ? hl[i + 3] : (rnd() & 0xFFFFFFu);
        }
        for (auto& w : ho) w = rnd() | rnd();
        for (int i = 0; i < NP; i++) {
            if ((e = cudaMemcpy(cL + N * i, hl.data(), 4 * N, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(cR + N * i, hr.data(), 4 * N, cudaMemcpyHostToDevice)) != cudaSuccess ||
                (e = cudaMemcpy(om + (size_t)words * H * i, ho.data(), 4 * ho.size(), cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
                return e;
        }
        if ((e = cudaMemset(Df, 0, 4 * N * NP)) != cudaSuccess || (e = cudaMemset(Cf, 12, N * NP)) != cudaSuccess ||
            (e = cudaMemset(cells, 0xFF, (size_t)8 * Wc4 * Hc4 * NP)) != cudaSuccess)
            return e;
    }
    std::vector<PairDev> pv(NP);
    for (int i = 0; i < NP; i++) {
        PairDev p{};
        p.W = W;
        p.H = H;
        p.cL = cL + N * i;
        p.cR = cR + N * i;
        p.omega = om + (size_t)words * H * i;
        p.Dit = dit + N * i;
        p.Df = Df + N * i;
        p.Cf = Cf + N * i;
        p.mask = mask + N * i;
        const int sz = i % 2 ? 4 : 8;
        set_cell_size(p, sz);
        p.Wc = (W + sz - 1) / sz;
        p.Hc = (H + sz - 1) / sz;
        p.cg_key = cells + (size_t)2 * Wc4 * Hc4 * i;
        p.cb_key = p.cg_key + (size_t)Wc4 * Hc4;
        pv[i] = p;
    }
    Params prm = c->prm;
    prm.err = c->err_dev;
    double best_v = 1e30, default_v = -1.0;
    const Tuning defaults{};
    std::vector<double> vcand_us;
    for (int sweep = 0; sweep < kSweeps; sweep++) {
        int ci = 0;
        for (int mixed = 1; mixed >= 0; mixed--)
            for (int bps : {4, 8, 16}) {
                double us = time_runs(s, ea, eb, 3, [&]() -> cudaError_t {
                    if (mixed) return launch_validate(pv.data(), NP, WK_VALIDATE_MIXED, prm, s, nullptr, 0, bps);
                    for (WorkKind k : kValidateKinds) {
                        const cudaError_t ev = launch_validate(pv.data(), NP, k, prm, s, nullptr, 0, bps);
                        if (ev != cudaSuccess) return ev;
                    }
                    return cudaSuccess;
                });
                if (us < 0) return cudaErrorUnknown;
                if (sweep == 0) vcand_us.push_back(us);
                us = vcand_us[ci] = std::min(vcand_us[ci], us);
                ci++;
                if (sweep + 1 < kSweeps) continue;
                if (mixed == defaults.validate_mixed && bps == defaults.validate_bps) default_v = us;
                if (us < best_v) {
                    best_v = us;
                    best.validate_mixed = mixed;
                    best.validate_bps = bps;
                }
            }
    }
    if (default_v > 0 && best_v > kTuneMargin * default_v) {
        best.validate_mixed = defaults.validate_mixed;
        best.validate_bps = defaults.validate_bps;
        best_v = default_v;
    }
    c->tune = best;
    c->tuned = true;
    c->tune_raster_us = best_r;
    c->tune_validate_us = best_v;
    return cudaSuccess;
}

extern "C" {

int stereo_get_tuning(stereo_ctx* c, stereo_tuning* out) {
    if (!c || !out) return STEREO_E_INVAL;
    out->small_area = c->tune.small_area;
    out->batch_area = c->tune.batch_area;
    out->raster_cols = c->tune.raster_cols;
    out->validate_blocks_per_sm = c->tune.validate_bps;
    out->validate_mixed = c->tune.validate_mixed;
    out->autotuned = c->tuned ? 1 : 0;
    out->raster_us = c->tuned ? c->tune_raster_us : 0.0;
    out->validate_us = c->tuned ? c->tune_validate_us : 0.0;
    return STEREO_OK;
}

void stereo_default_config(stereo_config* cfg) {
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->mem_budget_bytes = (size_t)4 << 30;
    cfg->max_slots = 1;
    cfg->max_queue = 64;
    cfg->t_lo = 4;
    cfg->t_hi = 8;
    cfg->t_grad = 8;
    cfg->t_fast = 20;
    cfg->kp_per_bin = 4;
    cfg->uniq_margin = 2;
    cfg->host_threads = 1;
}

size_t stereo_request_bytes(const stereo_config* cfg, int w, int h, int dmax, int iters, int cell) {
    if (!cfg || !valid_size(w, h) || dmax < 1 || dmax > 256 || iters < 1 || cell < 1 || cfg->kp_per_bin < 1 ||
        cfg->kp_per_bin > kMaxK)
        return 0;
    Request r;
    r.W = w;
    r.H = h;
    r.iters = iters;
    const int sz_min = iters >= 2 ? std::max(1, cell >> (iters - 2)) : 0;
    r.ncell_max = iters >= 2 ? cells_of(w, h, sz_min) : 1;
    size_t b = align_up(block_bytes(r, cfg->kp_per_bin), 256);
    const size_t N = (size_t)w * h;
    const int n_cap = mesh_vertex_cap(w, h, kFastBins * cfg->kp_per_bin, iters, cell);
    if (cfg->host_mesh == 0 && iters >= 2) {
        const int p_cap = (int)std::min<long long>(2ll * r.ncell_max, (long long)N);
        b += align_up(mesh_bytes(w, h, n_cap, 2 * n_cap + 8, p_cap), 256);
        b += align_up((size_t)kFastBins * cfg->kp_per_bin * 140 + (1 << 16), 256);  // S_1's staged mesh
    } else {
        // a staged host mesh: up to 2 triangles per support point, 40 B each plus its
        // raster lists and hull, with the 5/4 headroom the engine keeps
        b += align_up((size_t)n_cap * 2 * 56 * 5 / 4 + (1 << 16), 256);
    }
    b += align_up(align_up(N, 256) + N, 256);  // the submitted inputs awaiting admission
    return b;
}

namespace {
cudaError_t ensure_mesh_kernels();
}

int stereo_create(const stereo_config* cfg, stereo_ctx** out) {
    if (!cfg || !out) return STEREO_E_INVAL;
    if (!valid_params(*cfg) || cfg->max_slots < 1 || cfg->max_queue < 0) return STEREO_E_INVAL;
    *out = nullptr;
    if (cudaSetDevice(cfg->device) != cudaSuccess) return STEREO_E_CUDA;
    stereo_ctx* c = new stereo_ctx();
    c->cfg = *cfg;
    if (c->cfg.mem_budget_bytes == 0) c->cfg.mem_budget_bytes = (size_t)4 << 30;
    c->prm = Params{cfg->t_lo, cfg->t_hi, cfg->t_grad, cfg->t_fast, cfg->kp_per_bin, cfg->uniq_margin};
    c->K = cfg->kp_per_bin;
    if (cfg->stream) {
        c->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return STEREO_E_CUDA;
        }
        c->own_stream = true;
    }
    if (cfg->arena) {
        c->arena_base = (char*)cfg->arena;
    } else {
        if (cudaMalloc((void**)&c->arena_base, c->cfg.mem_budget_bytes) != cudaSuccess) {
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return STEREO_E_NOMEM;
        }
        c->own_arena = true;
    }
    c->arena.init(c->arena_base, c->cfg.mem_budget_bytes);
    // the scheduler thread has a core of its own (the host workers take the
    // others), so it waits for each round by polling rather than sleeping:
    // about 50 us less per round than a blocking wait
    cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming);
    cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (cudaMalloc((void**)&c->err_dev, 256) != cudaSuccess || !c->err_host.ensure(sizeof(int))) {
        stereo_destroy(c);
        return STEREO_E_NOMEM;
    }
    *c->err_host.as<int>() = 0;
    if (const char* v = std::getenv("STEREO_LAUNCH_LOG")) c->launch_log = std::fopen(v, "a");
    if (const char* v = std::getenv("STEREO_VALIDATE")) {
        c->bulk_validate = std::strcmp(v, "bulk") == 0;
        c->tune.validate_mixed = std::strcmp(v, "classes") != 0;
    }
    if (cfg->inject_wait_timeout > 0) c->bulk_validate = true;
    if (prepare_kernels() != cudaSuccess) c->bulk_validate = false;
    c->dev_mesh = cfg->host_mesh == 0;
    if (c->dev_mesh && ensure_mesh_kernels() != cudaSuccess) {
        note_error(cudaGetLastError(), "device mesh kernels unavailable (host meshes kept)", __LINE__);
        c->dev_mesh = false;
    }
    if (cfg->autotune) {  // before the scheduler starts: the tuning round owns the stream
        const Tuning keep = c->tune;
        if (autotune(c) != cudaSuccess) {
            note_error(cudaGetLastError(), "autotune (defaults kept)", __LINE__);
            c->tune = keep;
            c->tuned = false;
        }
    }
    c->pool.start(std::max(1, cfg->host_threads));
    c->sched = std::thread(scheduler, c);
    *out = c;
    return STEREO_OK;
}

namespace {
bool valid_pair(const stereo_pair& p) {
    return p.left && p.right && valid_size(p.w, p.h) && p.dmax >= 1 && p.dmax <= 256 && p.iters >= 1 && p.cell >= 1;
}
}  // namespace

// Submission of n pairs: every argument is checked first (one bad pair
// rejects the batch); the pairs are then taken in order while the queue has
// room, their inputs copied with one synchronisation for the batch, and
// queued under one lock, so the scheduler sees them together.
int stereo_submit_batch(stereo_ctx* c, const stereo_pair* pairs, int n, uint64_t* tickets_out) {
    if (!c || !pairs || n < 1 || !tickets_out) return STEREO_E_INVAL;
    for (int i = 0; i < n; i++)
        if (!valid_pair(pairs[i])) return STEREO_E_INVAL;
    std::vector<Request*> rs;
    rs.reserve(n);
    auto drop_all = [&](int rc) {
        {
            std::lock_guard<std::mutex> g2(c->mu);
            for (Request* r : rs) c->arena.release(r->in_dev);
        }
        for (Request* r : rs) {
            r->in_host.free();
            delete r;
        }
        return rc;
    };
    for (int i = 0; i < n; i++) {
        const stereo_pair& q = pairs[i];
        Request* r = new Request();
        r->in_host.pool = r->st_tri.pool = r->st_kp.pool = r->st_cells.pool = r->st_hdr.pool = r->st_trace.pool =
            &c->pinned;
        r->tpool = &c->traces;
        r->pool = &c->pool;
        r->stream_id = q.stream_id;
        r->W = q.w;
        r->H = q.h;
        r->dmax = q.dmax;
        r->iters = q.iters;
        r->cell = q.cell;
        const int sz_min = q.iters >= 2 ? std::max(1, q.cell >> (q.iters - 2)) : 0;
        r->ncell_max = q.iters >= 2 ? cells_of(q.w, q.h, sz_min) : 1;
        rs.push_back(r);
        if (block_bytes(*r, c->K) > c->cfg.mem_budget_bytes) return drop_all(STEREO_E_NOMEM);
    }
    // where the inputs live: device (or managed) memory and page-locked host memory are
    // copied straight to the arena (one DMA each), pageable memory through pinned staging
    // page-locked memory is read by the same gather-copy kernel through its device
    // pointers (over the CPU-GPU link), like device memory
    std::vector<char> kind(n);  // 'd' device or page-locked (device-readable), 'h' pageable
    std::vector<const uint8_t*> src_l(n), src_r(n);
    auto dev_view = [](const void* p, const void** dp) {  // a pointer the device can use, or none
        cudaPointerAttributes at{};
        const bool known = cudaPointerGetAttributes(&at, p) == cudaSuccess;
        cudaGetLastError();
        if (!known) return false;
        if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
            *dp = p;
            return true;
        }
        if (at.type == cudaMemoryTypeHost && at.devicePointer) {
            *dp = at.devicePointer;
            return true;
        }
        return false;
    };
    for (int i = 0; i < n; i++) {
        const void *dl = nullptr, *dr = nullptr;
        const bool direct = dev_view(pairs[i].left, &dl) && dev_view(pairs[i].right, &dr);
        kind[i] = direct ? 'd' : 'h';
        src_l[i] = (const uint8_t*)dl;
        src_r[i] = (const uint8_t*)dr;
        void* outs[3] = {pairs[i].out_disparity, pairs[i].out_cost, pairs[i].out_mask};
        for (int k = 0; k < 3; k++) {
            Request* r = rs[i];
            if (!outs[k]) continue;
            const void* dp = nullptr;
            r->out_direct[k] = dev_view(outs[k], &dp);
            r->out[k] = r->out_direct[k] ? const_cast<void*>(dp) : outs[k];
        }
    }
    int take = 0;
    {
        std::lock_guard<std::mutex> g(c->mu);
        int queued = (int)c->queue.size();
        for (; take < n; take++) {
            if (queued >= c->cfg.max_queue && (int)c->active.size() >= c->cfg.max_slots) break;
            Request* r = rs[take];
            if (kind[take] == 'd') {
                // the right image starts 256-byte aligned: the gather copy moves whole
                // 16-byte words only between aligned ends (bytes otherwise, about 4x slower)
                const size_t N = (size_t)r->W * r->H;
                r->in_dev = (uint8_t*)c->arena.alloc(align_up(N, 256) + N);
                if (!r->in_dev) break;
            }
            queued++;
        }
    }
    if (take == 0) return drop_all(STEREO_E_BUSY);
    for (int i = take; i < n; i++) delete rs[i];
    rs.resize(take);
    bool copied = false;
    CopyList cl{};  // device inputs: one gather-copy launch per kCopyBatch buffers
    for (int i = 0; i < take; i++) {
        Request* r = rs[i];
        const size_t N = (size_t)r->W * r->H;
        if (kind[i] == 'd') {
            for (int k = 0; k < 2; k++) {
                cl.src[cl.count] = k ? src_r[i] : src_l[i];
                cl.dst[cl.count] = r->in_dev + k * align_up(N, 256);
                cl.n[cl.count++] = (long long)N;
            }
            if (cl.count + 2 > kCopyBatch) {
                if (launch_copy_list(cl, c->copy_stream) != cudaSuccess) return drop_all(STEREO_E_CUDA);
                cl.count = 0;
            }
            copied = true;
        } else {
            if (!r->in_host.ensure(2 * N)) return drop_all(STEREO_E_NOMEM);
            std::memcpy(r->in_host.p, pairs[i].left, N);
            std::memcpy((char*)r->in_host.p + N, pairs[i].right, N);
        }
    }
    if (cl.count > 0 && launch_copy_list(cl, c->copy_stream) != cudaSuccess) return drop_all(STEREO_E_CUDA);
    if (copied && cudaStreamSynchronize(c->copy_stream) != cudaSuccess) {
        cudaGetLastError();
        return drop_all(STEREO_E_CUDA);
    }
    {
        std::lock_guard<std::mutex> g(c->mu);
        const double t = now_ms();
        for (int i = 0; i < take; i++) {
            Request* r = rs[i];
            r->ticket = c->next_ticket++;
            r->t_submit = t;
            c->reqs[r->ticket] = r;
            c->queue.push_back(r);
            tickets_out[i] = r->ticket;
        }
    }
    c->cv_sched.notify_all();
    return take;
}

int stereo_submit(stereo_ctx* c, int stream_id, const uint8_t* left, const uint8_t* right, int w, int h,
                  int dmax, int iters, int cell, uint64_t* ticket_out) {
    const stereo_pair p{stream_id, left, right, w, h, dmax, iters, cell};
    const int rc = stereo_submit_batch(c, &p, 1, ticket_out);
    return rc == 1 ? STEREO_OK : rc;
}

namespace {
// A finished request's result, as stereo_poll reports it.  Called with c->mu held.
void fill_result(const Request* r, stereo_result* out) {
    std::memset(out, 0, sizeof(*out));
    out->status = r->status;
    out->w = r->W;
    out->h = r->H;
    out->iters = r->iters;
    out->latency_ms = r->t_done - r->t_submit;
    out->host_mesh_ms = r->mesh_ms;
    if (r->state == Q_DONE) {
        out->disparity = r->dev.Df;
        out->cost = r->dev.Cf;
        out->mask = r->dev.mask;
        out->planeidx = r->pidx_buf;
        out->n_support = r->n_support.data();
        out->n_tri = r->n_tri.data();
        out->support = r->dev_trace ? const_cast<Pinned&>(r->st_trace).as<float>() : r->trace.data();
    }
}
}  // namespace

int stereo_poll(stereo_ctx* c, uint64_t ticket, stereo_result* out, int timeout_us) {
    if (!c || !out) return STEREO_E_INVAL;
    std::unique_lock<std::mutex> g(c->mu);
    auto it = c->reqs.find(ticket);
    if (it == c->reqs.end()) return STEREO_E_NOTFOUND;
    Request* r = it->second;
    auto ready = [r] { return r->state == Q_DONE || r->state == Q_FAILED; };
    if (!ready()) {
        if (timeout_us == 0) return STEREO_E_PENDING;
        if (timeout_us < 0) c->cv_done.wait(g, ready);
        else if (!c->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), ready)) return STEREO_E_PENDING;
    }
    fill_result(r, out);
    return r->status;
}

int stereo_poll_batch(stereo_ctx* c, const uint64_t* tickets, int n, stereo_result* out, int timeout_us) {
    if (!c || !tickets || !out || n < 1) return STEREO_E_INVAL;
    std::unique_lock<std::mutex> g(c->mu);
    std::vector<Request*> rs((size_t)n);
    for (int i = 0; i < n; i++) {
        auto it = c->reqs.find(tickets[i]);
        if (it == c->reqs.end()) return STEREO_E_NOTFOUND;
        rs[i] = it->second;
    }
    auto all_ready = [&rs] {
        for (const Request* r : rs)
            if (r->state != Q_DONE && r->state != Q_FAILED) return false;
        return true;
    };
    if (!all_ready()) {
        if (timeout_us == 0) return STEREO_E_PENDING;
        if (timeout_us < 0) c->cv_done.wait(g, all_ready);
        else if (!c->cv_done.wait_for(g, std::chrono::microseconds(timeout_us), all_ready)) return STEREO_E_PENDING;
    }
    for (int i = 0; i < n; i++) fill_result(rs[i], out + i);
    return STEREO_OK;
}

int stereo_poll_host(stereo_ctx* c, uint64_t ticket, stereo_result* out, int timeout_us, float* disparity,
                     uint8_t* cost, uint8_t* mask) {
    const int rc = stereo_poll(c, ticket, out, timeout_us);
    if (rc != STEREO_OK) return rc;
    const size_t N = (size_t)out->w * out->h;
    cudaSetDevice(c->cfg.device);
    cudaStream_t s = cudaStreamPerThread;
    cudaError_t e = cudaSuccess;
    if (disparity && e == cudaSuccess) e = cudaMemcpyAsync(disparity, out->disparity, 4 * N, cudaMemcpyDeviceToHost, s);
    if (cost && e == cudaSuccess) e = cudaMemcpyAsync(cost, out->cost, N, cudaMemcpyDeviceToHost, s);
    if (mask && e == cudaSuccess) e = cudaMemcpyAsync(mask, out->mask, N, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return STEREO_E_CUDA;
    }
    return STEREO_OK;
}

namespace {
// Take a done request out of the context (c->mu held): its ticket, slot and arena blocks.
int detach(stereo_ctx* c, uint64_t ticket, Request** out) {
    auto it = c->reqs.find(ticket);
    if (it == c->reqs.end()) return STEREO_E_NOTFOUND;
    Request* r = it->second;
    if (r->state != Q_DONE && r->state != Q_FAILED) return STEREO_E_PENDING;
    c->reqs.erase(it);
    c->active.erase(std::remove(c->active.begin(), c->active.end(), r), c->active.end());
    c->arena.release(r->block);
    c->arena.release(r->tri_block);
    c->arena.release(r->in_dev);
    c->arena.release(r->mesh_block);
    *out = r;
    return STEREO_OK;
}
// Its host buffers back to the pools (c->mu not held).
void free_request(stereo_ctx* c, Request* r) {
    r->in_host.free();
    r->st_tri.free();
    r->st_kp.free();
    r->st_cells.free();
    r->st_hdr.free();
    r->st_trace.free();
    c->traces.put(std::move(r->trace));
    delete r;
}
}  // namespace

int stereo_release(stereo_ctx* c, uint64_t ticket) {
    if (!c) return STEREO_E_INVAL;
    Request* r = nullptr;
    {
        std::lock_guard<std::mutex> g(c->mu);
        const int rc = detach(c, ticket, &r);
        if (rc != STEREO_OK) return rc;
    }
    free_request(c, r);
    c->cv_sched.notify_all();
    return STEREO_OK;
}

int stereo_release_batch(stereo_ctx* c, const uint64_t* tickets, int n) {
    if (!c || !tickets || n < 1) return STEREO_E_INVAL;
    std::vector<Request*> rs;
    rs.reserve((size_t)n);
    int first = STEREO_OK;
    {
        std::lock_guard<std::mutex> g(c->mu);
        for (int i = 0; i < n; i++) {
            Request* r = nullptr;
            const int rc = detach(c, tickets[i], &r);
            if (rc == STEREO_OK) rs.push_back(r);
            else if (first == STEREO_OK) first = rc;
        }
    }
    for (Request* r : rs) free_request(c, r);
    c->cv_sched.notify_all();
    return first;
}

const char* stereo_last_error(void) {
    std::lock_guard<std::mutex> g(g_err_mu);
    static thread_local char copy[256];
    std::memcpy(copy, g_err, sizeof(copy));
    return copy;
}

int stereo_get_stats(stereo_ctx* c, stereo_stats* out) {
    if (!c || !out) return STEREO_E_INVAL;
    std::lock_guard<std::mutex> g(c->mu);
    *out = c->stats;
    return STEREO_OK;
}

void stereo_destroy(stereo_ctx* c) {
    if (!c) return;
    {
        std::lock_guard<std::mutex> g(c->mu);
        for (Request* r : c->queue) {
            finish(c, *r, STEREO_E_INTERNAL);
        }
        c->queue.clear();
        c->stop = true;
    }
    c->cv_sched.notify_all();
    if (c->sched.joinable()) c->sched.join();
    c->pool.stop();
    cudaStreamSynchronize(c->stream);
    for (auto& kv : c->reqs) {
        Request* r = kv.second;
        r->in_host.free();
        r->st_tri.free();
        r->st_kp.free();
        r->st_cells.free();
        r->st_hdr.free();
        r->st_trace.free();
        delete r;
    }
    c->reqs.clear();
    if (c->launch_log) std::fclose(c->launch_log);
    c->desc_host.free();
    if (c->desc_dev) cudaFree(c->desc_dev);
    if (c->own_arena) cudaFree(c->arena_base);
    for (auto& kv : c->graph_exec)
        if (kv.second) cudaGraphExecDestroy(kv.second);
    if (c->err_dev) cudaFree(c->err_dev);
    c->err_host.free();
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->ev) cudaEventDestroy(c->ev);
    for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->ev_retired) cudaEventDestroy(ev);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ---------------------------------------------------------------- stage entry points
static int to_rc(cudaError_t e) { return e == cudaSuccess ? STEREO_OK : STEREO_E_CUDA; }

static PairBatch single(const PairDev& p, WorkKind k) {
    PairBatch b{};
    b.pd = nullptr;
    b.one = p;
    b.npairs = 1;
    b.total = work_items(k, p);
    b.scan_rows = p.scan_rows;
    return b;
}

int stereo_census(const uint8_t* left, const uint8_t* right, int w, int h, int t_grad, uint32_t* cL,
                  uint32_t* cR, uint32_t* omega, void* stream) {
    if (!left || !valid_size(w, h) || t_grad < 0 || (cR && !right)) return STEREO_E_INVAL;
    PairDev p{};
    p.L = left;
    p.R = right ? right : left;
    p.cL = cL;
    p.cR = cR;
    p.omega = omega;
    p.W = w;
    p.H = h;
    p.scan_rows = 7;  // one frame: the shorter strip items (more warps)
    Params prm{0, 0, t_grad, 0, 1, 0};
    return to_rc(launch_census(single(p, WK_CENSUS), prm, (cudaStream_t)stream));
}

int stereo_fast(const uint8_t* left, int w, int h, int t_fast, int K, int16_t* scratch, int32_t* out_uv,
                void* stream) {
    if (!left || !scratch || !out_uv || !valid_size(w, h) || t_fast < 0 || K < 1 || K > kMaxK) return STEREO_E_INVAL;
    PairDev p{};
    p.L = left;
    p.fast_score = scratch;
    p.kp_uv = out_uv;
    p.W = w;
    p.H = h;
    p.K = K;
    p.scan_rows = 7;
    Params prm{0, 0, 0, t_fast, K, 0};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_fast_score(single(p, WK_FAST_SCORE), prm, s);
    if (e == cudaSuccess) e = launch_fast_bins(single(p, WK_FAST_BINS), prm, s);
    return to_rc(e);
}

int stereo_epipolar_match(const uint32_t* cL, const uint32_t* cR, int w, int h, const int32_t* q_uv, int n,
                          int dmax, int t_lo, int margin, int32_t* out_d, void* stream) {
    if (!cL || !cR || (n > 0 && (!q_uv || !out_d)) || !valid_size(w, h) || n < 0 || dmax < 1 || dmax > 256 ||
        t_lo < 0 || margin < 0)
        return STEREO_E_INVAL;
    Params prm{t_lo, 0, 0, 0, 1, margin};
    return to_rc(launch_match_list(cL, cR, w, h, q_uv, n, dmax, prm, out_d, (cudaStream_t)stream));
}

namespace {
int check_canonical(const int32_t* uv, int n, int32_t* tri, int cap) {
    if (n < 0 || (n > 0 && !uv) || cap < 0 || (cap > 0 && !tri)) return STEREO_E_INVAL;
    for (int i = 0; i < n; i++) {
        if (uv[2 * i] < 0 || uv[2 * i + 1] < 0 || uv[2 * i] > 16383 || uv[2 * i + 1] > 16383) return STEREO_E_INVAL;
        if (i > 0) {
            const int a = uv[2 * i - 1], b = uv[2 * i + 1];
            if (b < a || (b == a && uv[2 * i] <= uv[2 * i - 2])) return STEREO_E_INVAL;  // not canonical
        }
    }
    return STEREO_OK;
}
}  // namespace

int stereo_delaunay(const int32_t* uv, int n, int32_t* tri, int cap) {
    const int rc = check_canonical(uv, n, tri, cap);
    return rc != STEREO_OK ? rc : delaunay(uv, n, tri, cap);
}

int stereo_delaunay_parallel(const int32_t* uv, int n, int32_t* tri, int cap, int threads) {
    const int rc = check_canonical(uv, n, tri, cap);
    if (rc != STEREO_OK) return rc;
    if (threads < 1) return STEREO_E_INVAL;
    const int depth = threads >= 8 ? 3 : threads >= 4 ? 2 : threads >= 2 ? 1 : 0;
    std::mutex mu;
    std::vector<std::thread> helpers;  // joined before returning
    const Spawn spawn = [&](std::function<void()> f) {
        std::lock_guard<std::mutex> g(mu);
        helpers.emplace_back(std::move(f));
    };
    int T;
    try {
        T = delaunay(uv, n, tri, cap, nullptr, nullptr, depth, depth ? &spawn : nullptr);
    } catch (...) {  // a helper thread or an allocation refused
        T = STEREO_E_NOMEM;
    }
    for (auto& t : helpers) t.join();
    return T;
}


namespace {
// k_mesh_pass's occupancy, looked up once per device (outside any capture).
std::mutex g_mesh_mu;
unsigned long long g_mesh_ready = 0;  // bit per device ordinal
cudaError_t ensure_mesh_kernels() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(g_mesh_mu);
    if (dev < 64 && (g_mesh_ready >> dev) & 1ull) return cudaSuccess;
    e = prepare_mesh_kernels();
    if (e == cudaSuccess && dev < 64) g_mesh_ready |= 1ull << dev;
    return e;
}
}  // namespace

int stereo_delaunay_insert(const int32_t* uv, int n, const int32_t* tri, int T, const int32_t* uv_new, int m, int w,
                           int h, int32_t* tri_out, int cap) {
    if (!tri || T < 1 || n < 3 || m < 0 || (m > 0 && !uv_new) || !valid_size(w, h) || cap < 0 || (cap > 0 && !tri_out))
        return STEREO_E_INVAL;
    if (check_canonical(uv, n, tri_out, cap) != STEREO_OK) return STEREO_E_INVAL;
    for (int i = 0; i < n; i++)
        if (uv[2 * i] >= w || uv[2 * i + 1] >= h) return STEREO_E_INVAL;
    for (int i = 0; i < m; i++)
        if (uv_new[2 * i] < 0 || uv_new[2 * i + 1] < 0 || uv_new[2 * i] >= w || uv_new[2 * i + 1] >= h)
            return STEREO_E_INVAL;
    for (int i = 0; i < 3 * T; i++)
        if (tri[i] < 0 || tri[i] >= n) return STEREO_E_INVAL;
    std::vector<int32_t> ccw((size_t)4 * T), opp((size_t)4 * T), tuv((size_t)6 * T);
    mesh_adjacency(uv, tri, T, ccw.data(), opp.data());
    for (int t = 0; t < T; t++)
        for (int k = 0; k < 3; k++) {
            tuv[6 * (size_t)t + 2 * k] = uv[2 * tri[3 * t + k]];
            tuv[6 * (size_t)t + 2 * k + 1] = uv[2 * tri[3 * t + k] + 1];
        }
    const int n_cap = n + m, t_cap = 2 * n_cap + 8, p_cap = m > 0 ? m : 1;
    const size_t N = (size_t)w * h;
    const size_t b_mesh = align_up(mesh_bytes(w, h, n_cap, t_cap, p_cap), 256);
    const size_t b_pos = align_up(8 * (size_t)n, 256), b_d = align_up(4 * (size_t)n, 256);
    const size_t b_tri = align_up(16 * (size_t)T, 256), b_list = align_up(8 * (size_t)p_cap, 256);
    const size_t b_tuv = align_up(24 * (size_t)T, 256), b_pidx = align_up(4 * N, 256);
    const size_t b_scr = align_up(4 * raster_list_words(T), 256), b_md = align_up(sizeof(MeshDev), 256);
    const size_t total = b_mesh + b_pos + b_d + 2 * b_tri + b_list + b_tuv + b_pidx + b_scr + b_md + 256;
    if (ensure_mesh_kernels() != cudaSuccess) return STEREO_E_CUDA;
    char* base = nullptr;
    cudaStream_t s = nullptr;
    int rc = STEREO_OK;
    if (cudaMalloc((void**)&base, total) != cudaSuccess) {
        cudaGetLastError();
        return STEREO_E_NOMEM;
    }
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaFree(base);
        cudaGetLastError();
        return STEREO_E_CUDA;
    }
    char* q = base;
    auto take = [&](size_t b) { char* r = q; q += b; return r; };
    char* mesh = take(b_mesh);
    int32_t* d_pos = (int32_t*)take(b_pos);
    float* d_d = (float*)take(b_d);
    int4* d_tri = (int4*)take(b_tri);
    int4* d_opp = (int4*)take(b_tri);
    int32_t* d_list = (int32_t*)take(b_list);
    int32_t* d_tuv = (int32_t*)take(b_tuv);
    int32_t* d_pidx = (int32_t*)take(b_pidx);
    int32_t* d_scr = (int32_t*)take(b_scr);
    MeshDev* d_md = (MeshDev*)take(b_md);
    MeshDev md{};
    mesh_carve(md, mesh, w, h, n_cap, t_cap, p_cap);
    md.seed_pos = d_pos;
    md.seed_d = d_d;
    md.seed_tri = d_tri;
    md.seed_opp = d_opp;
    md.seed_n = n;
    md.seed_T = T;
    md.list_uv = d_list;
    md.list_n = m;
    md.planeidx = d_pidx;
    md.pass = 2;
    md.canonical = 1;
    md.small_area = kSmallArea;
    md.cols = kRasterCols;
    PairDev p{};
    p.W = w;
    p.H = h;
    p.T = T;
    p.tri_uv = d_tuv;
    p.tri_rows = d_scr;
    p.small_tri = d_scr + T + 1;
    p.n_hull = -1;
    p.planeidx = d_pidx;
    PairBatch clear{};
    clear.one = p;
    clear.npairs = 1;
    clear.total = work_items(WK_CLEAR, p);
    cudaError_t e = cudaMemcpyAsync(d_pos, uv, 8 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_d, 0, 4 * (size_t)n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tri, ccw.data(), 16 * (size_t)T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_opp, opp.data(), 16 * (size_t)T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && m > 0) e = cudaMemcpyAsync(d_list, uv_new, 8 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tuv, tuv.data(), 24 * (size_t)T, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_md, &md, sizeof(MeshDev), cudaMemcpyHostToDevice, s);
    // the old mesh's plane-index map locates the new points, as a pass's raster does in the engine
    if (e == cudaSuccess) e = launch_raster_clear(clear, s);
    if (e == cudaSuccess) e = launch_raster_device_lists(p, s);
    if (e == cudaSuccess) e = launch_mesh_pass(d_md, 1, s);
    MeshHdr hd{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hd, md.hdr, sizeof(MeshHdr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        note_error(e, "stereo_delaunay_insert", __LINE__);
        rc = STEREO_E_CUDA;
    } else if (hd.err == 2) {
        rc = STEREO_E_INVAL;  // a new point outside the raster's cover of the old mesh
    } else if (hd.err != 0) {
        rc = STEREO_E_INTERNAL;
    } else if (hd.T > cap) {
        rc = STEREO_E_CAP;
    } else {
        // the canonical triangles as vertex positions (each triple in (v, u) order); a
        // vertex's index is its rank among S = uv + the new points, in (v, u) order
        std::vector<int32_t> tq((size_t)6 * hd.T);
        e = cudaMemcpyAsync(tq.data(), md.tri_uv, 24 * (size_t)hd.T, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            note_error(e, "stereo_delaunay_insert copy back", __LINE__);
            rc = STEREO_E_CUDA;
        } else {
            std::vector<int64_t> keys;
            keys.reserve((size_t)n + m);
            for (int i = 0; i < n; i++) keys.push_back(((int64_t)uv[2 * i + 1] << 32) | uv[2 * i]);
            for (int i = 0; i < m; i++) keys.push_back(((int64_t)uv_new[2 * i + 1] << 32) | uv_new[2 * i]);
            std::sort(keys.begin(), keys.end());
            keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
            auto rank = [&](int32_t u, int32_t v) {
                const int64_t k = ((int64_t)v << 32) | u;
                return (int32_t)(std::lower_bound(keys.begin(), keys.end(), k) - keys.begin());
            };
            for (int i = 0; i < hd.T; i++)
                for (int k = 0; k < 3; k++) tri_out[3 * i + k] = rank(tq[6 * (size_t)i + 2 * k], tq[6 * (size_t)i + 2 * k + 1]);
            rc = hd.T;
        }
    }
    cudaStreamDestroy(s);
    cudaFree(base);
    return rc;
}

int stereo_planes(const int32_t* uv, const float* d, const int32_t* tri, int T, float* abc) {
    if (T < 0 || (T > 0 && (!uv || !d || !tri || !abc))) return STEREO_E_INVAL;
    planes(uv, d, tri, T, abc);
    return STEREO_OK;
}

size_t stereo_raster_scratch_bytes(int T) {
    if (T < 0) return 0;
    return align_up(4 * raster_list_words(T), 256);
}

int stereo_raster(const int32_t* tri_uv, const float* abc, int T, int w, int h, int32_t* planeidx, float* D_it,
                  void* scratch, size_t scratch_bytes, void* stream) {
    if (!valid_size(w, h) || T < 0 || (T > 0 && (!tri_uv || !scratch)) || (!planeidx && !D_it) ||
        (D_it && T > 0 && !abc) || ((uintptr_t)planeidx & 15) != 0 || ((uintptr_t)D_it & 15) != 0)
        return STEREO_E_INVAL;
    if (T > 0 && scratch_bytes < 4 * raster_list_words(T)) return STEREO_E_CAP;
    PairDev p{};
    p.W = w;
    p.H = h;
    p.T = T;
    p.tri_uv = tri_uv;
    p.abc = abc;
    p.tri_rows = (int32_t*)scratch;
    p.small_tri = (int32_t*)scratch + T + 1;
    p.n_hull = -1;  // no hull: the frame is cleared first
    p.planeidx = planeidx;
    p.Dit = D_it;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_raster_clear(single(p, WK_CLEAR), s);
    if (e == cudaSuccess) e = launch_raster_device_lists(p, s);
    return to_rc(e);
}

int stereo_validate(const uint32_t* cL, const uint32_t* cR, const uint32_t* omega, const float* D_it, int w, int h,
                    int sz, int t_lo, int t_hi, int first_pass, float* D_f, uint8_t* C_f, uint8_t* mask,
                    uint32_t* cg_key, uint32_t* cb_key, void* stream) {
    if (!cL || !cR || !omega || !D_it || !D_f || !C_f || !mask || !valid_size(w, h) || sz < 1 ||
        !(0 <= t_lo && t_lo <= t_hi && t_hi < 24) || ((cg_key == nullptr) != (cb_key == nullptr)))
        return STEREO_E_INVAL;
    PairDev p{};
    p.cL = (uint32_t*)cL;
    p.cR = (uint32_t*)cR;
    p.omega = (uint32_t*)omega;
    p.Dit = (float*)D_it;
    p.W = w;
    p.H = h;
    set_cell_size(p, sz);
    p.Wc = (w + sz - 1) / sz;
    p.Hc = (h + sz - 1) / sz;
    p.first_pass = first_pass ? 1 : 0;
    p.Df = D_f;
    p.Cf = C_f;
    p.mask = mask;
    p.cg_key = cg_key;
    p.cb_key = cb_key;
    Params prm{t_lo, t_hi, 0, 0, 1, 0};
    const WorkKind k = validate_kind(p);
    return to_rc(launch_validate(&p, 1, k, prm, (cudaStream_t)stream, nullptr));
}

int stereo_validate_bulk(const uint32_t* cL, const uint32_t* cR, const uint32_t* omega, const float* D_it, int w,
                         int h, int sz, int t_lo, int t_hi, int first_pass, float* D_f, uint8_t* C_f, uint8_t* mask,
                         uint32_t* cg_key, uint32_t* cb_key, int* err_flag, void* stream) {
    if (!cL || !cR || !omega || !D_it || !D_f || !C_f || !err_flag || !valid_size(w, h) || sz < 1 ||
        !(0 <= t_lo && t_lo <= t_hi && t_hi < 24) || ((cg_key == nullptr) != (cb_key == nullptr)))
        return STEREO_E_INVAL;
    if ((((uintptr_t)cL | (uintptr_t)cR | (uintptr_t)omega | (uintptr_t)D_it | (uintptr_t)C_f) & 15) != 0)
        return STEREO_E_INVAL;
    static int prepared_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (prepared_device != dev) {
        if (prepare_kernels() != cudaSuccess) return STEREO_E_CUDA;
        prepared_device = dev;
    }
    PairDev p{};
    p.cL = (uint32_t*)cL;
    p.cR = (uint32_t*)cR;
    p.omega = (uint32_t*)omega;
    p.Dit = (float*)D_it;
    p.W = w;
    p.H = h;
    set_cell_size(p, sz);
    p.Wc = (w + sz - 1) / sz;
    p.Hc = (h + sz - 1) / sz;
    p.first_pass = first_pass ? 1 : 0;
    p.Df = D_f;
    p.Cf = C_f;
    p.mask = mask;
    p.cg_key = cg_key;
    p.cb_key = cb_key;
    Params prm{t_lo, t_hi, 0, 0, 1, 0, err_flag};
    return to_rc(launch_validate_bulk(single(p, WK_VALIDATE_BULK), prm, (cudaStream_t)stream));
}

int stereo_resample_match(const uint32_t* cg_key, const uint32_t* cb_key, int ncells, const float* D_it,
                          const uint32_t* cL, const uint32_t* cR, int w, int h, int dmax, int t_lo, int margin,
                          float* cg_d, int32_t* x_d, void* stream) {
    if (!cg_key || !cb_key || ncells < 0 || !D_it || !cL || !cR || !valid_size(w, h) || dmax < 1 || dmax > 256 ||
        !cg_d || !x_d || t_lo < 0 || margin < 0)
        return STEREO_E_INVAL;
    PairDev p{};
    p.cg_key = (uint32_t*)cg_key;
    p.cb_key = (uint32_t*)cb_key;
    p.Dit = (float*)D_it;
    p.cL = (uint32_t*)cL;
    p.cR = (uint32_t*)cR;
    p.W = w;
    p.H = h;
    p.dmax = dmax;
    p.Wc = ncells;
    p.Hc = 1;
    p.cg_d = cg_d;
    p.x_d = x_d;
    Params prm{t_lo, 0, 0, 0, 1, margin};
    return to_rc(launch_resample(single(p, WK_RESAMPLE), prm, (cudaStream_t)stream));
}

}  // extern "C"
