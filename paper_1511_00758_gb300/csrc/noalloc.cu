// stereo_raster_noalloc: the plane-index / D_it raster for callers that
// cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocating routine) on the
// path that runs the raster: a real-time loop with a fixed memory plan that
// allocates everything up front, or code running while another component
// owns the device allocator.  stereo_raster needs scratch for
// its per-triangle work lists; this variant takes that scratch from one
// fixed, file-scope device array instead, so the caller passes only its
// inputs and outputs.
//
// The array holds the work lists of up to kNoAllocMaxTriangles triangles
// (2 * (T + 1) + 2 * ceil(T / 1024) int32, just over 2 MiB).  Every GPU that loads the library keeps it
// until the process exits.  All calls share it: two calls whose work
// overlaps on the GPU (different streams, or different threads without
// ordering) race on it and must be serialised by the caller.  Nothing in it
// needs clearing: each call writes every entry it later reads.  The address
// of the array is looked up once per device and kept; a cudaDeviceReset (or
// anything else that destroys the device's primary context) makes it stale,
// so this entry point must not be used after one.
#include <mutex>

#include "internal.h"
#include "../../include/stereo.h"

namespace {

constexpr int kNoAllocMaxTriangles = 262143;
constexpr int kMaxDevices = 64;

// Work lists: work-item offsets of the large triangles (T + 1), the small-triangle list (T + 1),
// then per-block offsets of the list builder.
static __device__ __align__(256) int32_t g_raster_lists[stereo::raster_list_words(kNoAllocMaxTriangles)];
static_assert(sizeof(g_raster_lists) == sizeof(int32_t) * stereo::raster_list_words(kNoAllocMaxTriangles),
              "the array holds the work lists of kNoAllocMaxTriangles triangles");

std::mutex g_mu;
int32_t* g_addr[kMaxDevices] = {};

// Device address of g_raster_lists on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
int lists_address(int32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return STEREO_E_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_raster_lists) != cudaSuccess || !p) {
            cudaGetLastError();
            return STEREO_E_CUDA;
        }
        g_addr[dev] = (int32_t*)p;
    }
    *out = g_addr[dev];
    return STEREO_OK;
}

}  // namespace

extern "C" int stereo_raster_noalloc(const int32_t* tri_uv, const float* abc, int T, int w, int h,
                                     int32_t* planeidx, float* D_it, void* stream) {
    if (!stereo::valid_size(w, h) || T < 0 ||
        (T > 0 && !tri_uv) || (!planeidx && !D_it) || (D_it && T > 0 && !abc) ||
        ((uintptr_t)planeidx & 15) != 0 || ((uintptr_t)D_it & 15) != 0)
        return STEREO_E_INVAL;
    if (T > kNoAllocMaxTriangles) return STEREO_E_CAP;
    int32_t* lists = nullptr;
    const int rc = lists_address(&lists);
    if (rc != STEREO_OK) return rc;
    stereo::PairDev p{};
    p.W = w;
    p.H = h;
    p.T = T;
    p.tri_uv = tri_uv;
    p.abc = abc;
    p.tri_rows = lists;
    p.small_tri = lists + T + 1;
    p.n_hull = -1;  // no hull: the frame is cleared first
    p.planeidx = planeidx;
    p.Dit = D_it;
    stereo::PairBatch b{};
    b.one = p;
    b.npairs = 1;
    b.total = stereo::work_items(stereo::WK_CLEAR, p);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = stereo::launch_raster_clear(b, s);
    if (e == cudaSuccess) e = stereo::launch_raster_device_lists(p, s);
    return e == cudaSuccess ? STEREO_OK : STEREO_E_CUDA;
}
