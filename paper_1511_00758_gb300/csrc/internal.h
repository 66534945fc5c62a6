// Internal declarations shared by the kernels and the host engine of libstereo.
#pragma once

#include <cstddef>
#include <cstdint>
#include <functional>

#include <cuda_runtime.h>

namespace stereo {

constexpr int kFastBins = 120;          // 12 x 10 spatial bins (Sec. III-A)
constexpr int kFastBinsX = 12;
constexpr int kFastBinsY = 10;
constexpr int kMaxK = 32;               // keypoints per bin, upper bound
constexpr int kRasterRows = 8;          // rows of a raster work item of a large triangle
constexpr int kFillCells = 2048;        // cell records reset per block (raster launch or the fill kernel)
constexpr int kRasterCols = 128;        // columns of a raster work item of a large triangle
constexpr int kVBatch = 64;            // pair descriptors per fused-validate launch (about 7 KB of kernel parameters)
constexpr int kBatchArea = 1024;        // box pixels of a warp's batch of small triangles (at most 32)
constexpr int kSmallArea = 256;         // bounding-box pixels of a thread-rasterised triangle
constexpr uint32_t kNoKey = 0xFFFFFFFFu;
constexpr uint32_t kIdxMask = (1u << 27) - 1;

// Device buffers and sizes of one frame pair.  Every kernel reads its pair's
// descriptor from a PairBatch, so one launch can cover many pairs.
struct PairDev {
    const uint8_t* L;
    const uint8_t* R;
    uint32_t* cL;
    uint32_t* cR;
    uint32_t* omega;          // H * ceil(W/32) bit words
    int16_t* fast_score;      // W*H
    int scan_rows;            // census / FAST strip rows per warp item: 7 or 14 (0: 14)
    int32_t* kp_uv;           // 120*K (u, v) slots
    int32_t* kp_d;            // 120*K matches
    const int32_t* tri_uv;    // T * 6
    const float* abc;         // T * 3
    int32_t* tri_rows;        // T + 1: exclusive prefix of work items (8x128 blocks) per large triangle
    const int32_t* item_tri;  // raster_items: triangle of each large-triangle work item
    int32_t* small_tri;       // n_small small triangles
    const int32_t* small_batch;  // n_batch + 1 starts of the warp batches of small_tri (null: 32 each)
    int n_batch;
    int raster_cols;              // columns of a large-triangle work item (0: kRasterCols)
    const int32_t* hull;      // n_hull directed hull edges (ax, ay, bx, by), interior on the positive side
    int n_hull;               // -1: no hull; the caller clears the frame before the raster
    int n_small;
    int32_t* planeidx;        // W*H plane-index map, or null (not needed this pass)
    float* Dit;               // W*H interpolated prior D_it (NaN outside the mesh)
    float* Df;                // W*H
    uint8_t* Cf;              // W*H
    uint8_t* mask;            // W*H or null
    uint32_t* cg_key;         // cells
    uint32_t* cb_key;         // cells
    float* cg_d;              // cells
    int32_t* x_d;             // cells
    int W, H, dmax;
    int T;                    // triangles
    int sz, Wc, Hc;           // current occupancy grid
    int sz_shift;             // log2(sz) when sz is a power of two, else -1
    uint32_t sz_magic;        // floor(2^32 / sz) + 1: x / sz == umulhi(x, magic) for x < 2^18
    int raster_items;         // tri_rows[T] when known on the host
    int first_pass;
    int K;                    // keypoints per bin
    int mesh_raster;          // the pass's mesh is on the device: k_raster_mesh rasters it (no k_raster work)
};

// One launch's pairs: either a single descriptor by value (pd == nullptr)
// or a device array with a prefix of work items per pair.
struct PairBatch {
    const PairDev* pd;        // device array [npairs], or null
    const int* work_off;      // device array [npairs + 1], or null
    int npairs;
    int total;                // work items in this launch
    PairDev one;
    int scan_rows;            // census / FAST strip rows of every pair of the launch (PairDev::scan_rows)
};

struct Params {
    int t_lo, t_hi, t_grad, t_fast, K, margin;
    int* err;  // device flag set when a bounded device-side wait gave up (may be null)
    int withhold;  // testing: the bulk-copy validate's producer issues nothing, so every bounded wait runs out
};

// Work items per pair for each kernel kind.
enum WorkKind { WK_CENSUS = 0, WK_FAST_SCORE, WK_FAST_BINS, WK_MATCH_KP, WK_CLEAR,
                WK_RASTER, WK_VALIDATE, WK_VALIDATE_UNIT, WK_VALIDATE_C4, WK_VALIDATE_C2,
                WK_VALIDATE_ANY, WK_VALIDATE_MIXED, WK_VALIDATE_BULK, WK_RESAMPLE, WK_FILL, WK_COUNT };
int work_items(WorkKind k, const PairDev& p);
// Sets sz and its division helpers.
void set_cell_size(PairDev& p, int sz);

// Kernel launchers (async on stream).  grid_cap limits persistent grids.
cudaError_t launch_census(const PairBatch& b, const Params& prm, cudaStream_t s);
cudaError_t launch_fast_score(const PairBatch& b, const Params& prm, cudaStream_t s);
cudaError_t launch_fast_bins(const PairBatch& b, const Params& prm, cudaStream_t s);
cudaError_t launch_match_kp(const PairBatch& b, const Params& prm, cudaStream_t s);
cudaError_t launch_raster_clear(const PairBatch& b, cudaStream_t s);
cudaError_t launch_raster(const PairBatch& b, cudaStream_t s);
// single pair whose work lists are built on the device (stage entry point):
// tri_rows needs T + 1 entries; small_tri T + 1 entries followed by
// 2 * ceil(T / 1024) entries of block offsets
cudaError_t launch_raster_device_lists(const PairDev& p, cudaStream_t s);
constexpr size_t raster_list_words(int T) { return 2 * ((size_t)T + 1) + 2 * (((size_t)T + 1023) / 1024); }
// Fused validate: one kernel variant per cell-side class; a pair has work
// only under its own class, validate_kind(p): WK_VALIDATE (no cells, or
// 8 | sz), WK_VALIDATE_UNIT (sz 1), WK_VALIDATE_C4 (sz 4), WK_VALIDATE_C2
// (sz 2), WK_VALIDATE_ANY (other sides).  Launch every class with work, or
// WK_VALIDATE_MIXED: one launch in which every pair takes its own class.
constexpr WorkKind kValidateKinds[] = {WK_VALIDATE, WK_VALIDATE_UNIT, WK_VALIDATE_C4, WK_VALIDATE_C2,
                                       WK_VALIDATE_ANY};
WorkKind validate_kind(const PairDev& p);
// Launches class k over pairs[0..n) (pairs without work under k are skipped),
// kVBatch pairs per launch, their descriptors passed in the kernel
// parameters, and at least min_launches launches (empty ones idle);
// *launches (may be null) receives the launch count.
cudaError_t launch_validate(const PairDev* pairs, int n, WorkKind k, const Params& prm, cudaStream_t s,
                            int* launches, int min_launches = 0, int blocks_per_sm = 8);
// Bulk-copy pipelined validate (same results).  Needs 16-byte aligned D_it,
// cL, cR, C_f and Omega_I buffers; sets *prm.err if a bounded wait gave up.
cudaError_t launch_validate_bulk(const PairBatch& b, const Params& prm, cudaStream_t s);
size_t validate_bulk_smem_bytes();
cudaError_t prepare_kernels();  // kernel attributes; call with the device current, outside capture
cudaError_t launch_resample(const PairBatch& b, const Params& prm, cudaStream_t s);
cudaError_t launch_fill_cells(const PairBatch& b, cudaStream_t s);
cudaError_t launch_fill_u32(uint32_t* p, uint32_t value, size_t n, cudaStream_t s);
cudaError_t launch_match_list(const uint32_t* cL, const uint32_t* cR, int W, int H,
                              const int32_t* q, int n, int dmax, const Params& prm,
                              int32_t* out, cudaStream_t s);

// Copies of up to kCopyBatch device buffers in one launch (the inputs of a
// batch submission): entry i copies n[i] bytes from src[i] to dst[i].
constexpr int kCopyBatch = 128;
struct CopyList {
    const uint8_t* src[kCopyBatch];
    uint8_t* dst[kCopyBatch];
    long long n[kCopyBatch];
    int count;
};
cudaError_t launch_copy_list(const CopyList& L, cudaStream_t s);

int sm_count();
// Frame sizes every entry point accepts: 5 <= W, H <= 8192 and W * H < 2^27
// (pixel indices fit the 27-bit index field of the cell keys).
bool valid_size(int w, int h);

// ---------------------------------------------------------------- device mesh (retess.cu)
// The triangulation G(S_it) of a pair kept on the device between passes:
// after a pass's resampling, the new support points are inserted into it and
// the mesh is flipped back to the unique triangulation of reading 6, its
// planes and raster lists are built for the next pass, all on the GPU.
constexpr int kMeshBatch = 64;      // pairs per mesh launch
constexpr int kMeshClasses = 7;     // small-triangle box width classes: 1, 2, <=4, <=8, <=16, <=32, wider
constexpr int kMeshMaxIters = 16;   // iterations a request may take (the trace's support sets)

// Counters of one pair's device mesh (device memory).
struct MeshHdr {
    int n, T;                        // vertices, triangles
    int n_new;                       // points of this pass waiting for insertion (pending entries)
    int n_small, n_large, n_items, n_hull;  // raster lists of the mesh
    int cls[kMeshClasses];           // small triangles per box width class
    int cls_fill[kMeshClasses];
    int stamp;                       // last stamp of the split / flip records
    int err;                         // nonzero: 1 capacity, 2 a point not found in its triangle, 3 round limit,
                                     // 4 a launch whose clusters did not match its pair count
    int rounds, flips;               // insertion rounds and flips of the last pass
    int frounds;                     // flip rounds of the last pass
    int n_pl[2];                     // entries of the two pending worklists (this round's, the next's)
    int n_al[2];                     // entries of the two active-triangle worklists of the flip rounds
    int edge_ins;                    // insertions on an edge (2 -> 4 or hull 1 -> 2) in the last pass
    int total_new, inserted;         // points of the pass to insert, and those inserted (or given up)
    int step;                        // rounds (insertion and flip) taken so far in this pass
    int fdone;                       // the flip rounds ended (a round without flips)
    int s_count[kMeshMaxIters + 1];  // |S_it| of the trace (canonical pass)
    int trace_floats;                // floats written to the trace
};

// A triangle of the device mesh, one 32-byte sector: a = the packed positions
// (v << 14 | u) of its vertices a, b, c (positive orientation) and the
// neighbour ref of edge 0; b = the neighbour refs of edges 1 and 2, the number
// of points pending in it (insertion), and a scratch word (its smallest
// canonical vertex, when ranked).  Edge k runs opposite vertex k; a ref is
// (t << 2) | j, the neighbour's twin edge, or -1 on the hull.  A vertex is
// named by its pixel: the rounds never need a vertex slot.
struct TriRec {
    int4 a, b;
};

// Per triangle: its claim (an insertion claim, then in the flip rounds a flip
// claim whose high bits hold the round, so newer rounds win; all ~0 between
// insertion rounds) and a second word: the sums of the u and v of the points
// pending in it (u << 32 | v) while points are inserted, its own best flip
// proposal in the flip rounds, its canonical key when ranked.
struct ClaimRec {
    unsigned long long key, acc;
};

struct MeshDev {
    // vertices (slot order: as inserted)
    int2* pos;                // (u, v)
    uint8_t* vpass;           // iteration the point joined the support set (1-based)
    int4* vcanon;             // (u, v, d bits, pass) in canonical order, when ranked
    float* dmap;              // W*H: the support disparity at each vertex pixel
    uint32_t* occ;            // W*H bits: pixel holds a vertex
    uint32_t* wpre;           // exclusive prefix of popcount(occ) per word
    // triangles (slot order)
    TriRec* tr;
    ClaimRec* cl;
    int* alist;               // two worklists of triangles to check in the flip rounds (2 * t_cap)
    int4* smap;               // split / flip record: (stamp, new ref of old edge 0, 1, 2)
    int* gcnt;                // triangles per smallest canonical vertex, then their prefix [n_cap + 1]
    int* tperm;               // canonical triangle order: position -> slot
    uint32_t* tpass;          // canonical pass: the pass each vertex joined, by rank
    uint32_t* tpos;           // and its position within S_it (scan scratch)
    int4* plist;              // two worklists (2 * p_cap) of the points still to insert, one record each:
                              // (vertex slot, current triangle, edge code, packed position); the
                              // triangle is -2 - t while the round that inserted it into t links its
                              // pieces; the edge code is -1 inside, else
                              // ((neighbour + 1) << 4) | (twin edge << 2) | edge
    unsigned long long* pkey; // this round's claim key of each worklist entry
    int* scan;                // scan scratch: chunk totals [scan_cap]
    int* large;               // large-triangle list (triangle ids of the raster) and item prefix [t_cap + 1]
    int* lrows;
    // raster inputs of the next pass (triangle id = slot, or canonical position)
    int32_t* tri_uv;          // 6 int32 per triangle
    float* abc;               // 3 fp32 per triangle
    int32_t* small;           // small triangles by width class
    int32_t* hull;            // directed hull edges (ax, ay, bx, by)
    MeshHdr* hdr;
    int n_cap, t_cap, p_cap, scan_cap;
    int W, H;
    // the pass's new points: from cell records (engine) or a point list (stage entry)
    const uint32_t* cg_key;
    const float* cg_d;
    const uint32_t* cb_key;
    const int32_t* x_d;
    int ncells;
    const int32_t* list_uv;
    int list_n;
    const int32_t* planeidx;  // the pass's plane-index map (triangle slot per pixel)
    // seed mesh to take over (first device pass), in the host staging layout
    const int32_t* seed_pos;  // n (u, v)
    const float* seed_d;
    const int4* seed_tri;     // T (a, b, c, -) positive orientation, canonical order
    const int4* seed_opp;
    int seed_n, seed_T;       // > 0: take the seed mesh over first
    int pass;                 // iteration the new points join
    int canonical;            // the next pass is the last: canonical triangle order and vertex ranks
    // canonical pass: the support sets S_1 .. S_iters, each in canonical order as (u, v, d) floats,
    // one after the other, written to trace (the request's page-locked buffer, trace_cap floats)
    float* trace;
    int trace_cap;
    int iters;
    int small_area, cols;     // raster work shapes
};

// Bytes of one pair's device mesh for the given capacities, and the carving
// of a block of that size (256-byte aligned arrays).
size_t mesh_bytes(int W, int H, int n_cap, int t_cap, int p_cap);
void mesh_carve(MeshDev& m, void* block, int W, int H, int n_cap, int t_cap, int p_cap);
// Vertex capacity of a request: the seed keypoints plus two points per cell
// of every pass that resamples, at most one per pixel.
int mesh_vertex_cap(int W, int H, int seed_points, int iters, int cell);
// One pass of mesh work for up to kMeshBatch pairs (device descriptors md[np]):
// take over seed meshes, collect and insert the new points, flip to the
// triangulation, rank canonically where asked, build the next raster inputs.
// One thread-block cluster per pair (mesh_cluster_blocks(np) blocks each).
cudaError_t launch_mesh_pass(const MeshDev* md, int np, cudaStream_t s);
int mesh_cluster_blocks(int np);
// Raster of device meshes: PairBatch b lists the pairs (their PairDev:
// outputs, cells), md the same pairs' meshes (counts read on the device).
cudaError_t launch_raster_mesh(const PairBatch& b, const MeshDev* md, cudaStream_t s);
cudaError_t prepare_mesh_kernels();

// Host mesh step (mesh.cpp).
int delaunay(const int32_t* uv, int n, int32_t* tri, int cap);
// Also returns the directed hull edges (org, dest vertex index pairs, the
// triangles on the left as in a positively oriented triangle) in hull[2 * n]
// and their count in *n_hull (0 when there is no triangle).
// depth > 0 with spawn: the top `depth` levels of the divide and conquer
// (at most 3) fork, the lower half of each split offered to spawn, which runs
// the function it is given on another thread or not at all (the caller then
// runs it itself); the result is the same.
using Spawn = std::function<void(std::function<void()>)>;
int delaunay(const int32_t* uv, int n, int32_t* tri, int cap, int32_t* hull, int* n_hull, int depth = 0,
             const Spawn* spawn = nullptr);
void planes(const int32_t* uv, const float* d, const int32_t* tri, int T, float* abc);
// Positively oriented vertex order (ccw: 4 int32 per triangle, the fourth 0)
// and the neighbour across each edge (opp: 4 int32 per triangle; edge e joins
// vertices e + 1 and e + 2, entry (s << 2) | e' names the twin edge e' of
// triangle s, -1 on the hull) of a triangle list.
void mesh_adjacency(const int32_t* uv, const int32_t* tri, int T, int32_t* ccw, int32_t* opp);
// Raster work lists of a mesh: small[] the triangles whose clipped bounding
// box has at most kSmallArea pixels (returns their count in *n_small), and,
// when small_box is given, each one's box area (at least 1) in the same
// order; rows[T + 1] the exclusive prefix of the 8x128 work items of the
// others (returns the total).
int raster_lists(const int32_t* tri_uv, int T, int W, int H, int32_t* rows, int32_t* small, int* n_small,
                 int small_area = kSmallArea, int cols = kRasterCols, int32_t* small_box = nullptr);
// Warp batches of the (sorted) small list, from its box areas: consecutive
// runs of at most 32 triangles and kBatchArea box pixels (a single larger box
// runs alone); batch[0..n] are their starts plus n_small; returns n.
int small_batches(const int32_t* small_box, int n_small, int32_t* batch, int batch_area = kBatchArea);
// Triangle of every large-triangle work item (items = rows[T] entries).
void raster_item_tri(const int32_t* rows, int T, int32_t* item_tri);

}  // namespace stereo
