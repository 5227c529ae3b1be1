// p2m_query_noalloc: the closest-point query for callers that are not allowed to allocate
// device memory.  p2m_query may grow a per-index scratch buffer with cudaMalloc; this entry
// point instead runs the same kernels on a fixed scratch array that is part of the loaded
// library image (a file-scope __device__ array, one copy per GPU, kept until the process
// exits).  It never calls cudaMalloc, cudaFree or any allocating library routine.
#include <mutex>

#include "host.h"

namespace p2m {

int launch_query_on_scratch(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
                            int32_t* d_tri, float* d_bary, int32_t* d_rest, int2* d_long, int* d_cnt, cudaStream_t s);

namespace {

constexpr int64_t kMaxQueries = P2M_NOALLOC_MAX_QUERIES;
constexpr size_t kRestBytes = sizeof(int32_t) * kMaxQueries;  // queries left to the BVH search
constexpr size_t kLongBytes = sizeof(int2) * kMaxQueries;     // (query, site) pairs with long lists
constexpr size_t kScratchBytes = kRestBytes + kLongBytes + 256;

// The scratch itself.  Host code must not use this name as an address: on the host it is
// only a stand-in, so the device address is looked up once per device below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up on first use per device).
int scratch_address(void** out) {
    int dev = 0;
    P2M_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(P2M_ERR_INVALID_ARG, "device id out of range for p2m_query_noalloc");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(P2M_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return P2M_OK;
}

}  // namespace
}  // namespace p2m

using namespace p2m;

extern "C" int p2m_query_noalloc(p2m_index* h, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
                                 int32_t* d_tri, float* d_bary, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_query_noalloc needs a single-mesh index");
    if (n < 0) return fail(P2M_ERR_INVALID_ARG, "n < 0");
    if (n > kMaxQueries)
        return fail(P2M_ERR_LIMIT, "p2m_query_noalloc takes at most " + std::to_string(kMaxQueries) +
                                       " queries per call (got " + std::to_string(n) + "); split the batch");
    if (n == 0) return P2M_OK;
    if (!d_pts || !d_dist) return fail(P2M_ERR_INVALID_ARG, "d_pts and d_dist must be non-NULL");
    // the index's device must be current: the scratch address below is the current device's
    P2M_TRY(check_call(h, n, "p2m_query_noalloc"));
    void* base = nullptr;
    P2M_TRY(scratch_address(&base));
    char* b = static_cast<char*>(base);
    int32_t* d_rest = reinterpret_cast<int32_t*>(b);
    int2* d_long = reinterpret_cast<int2*>(b + kRestBytes);
    int* d_cnt = reinterpret_cast<int*>(b + kRestBytes + kLongBytes);
    return launch_query_on_scratch(h, *h->meshes[0], d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_long, d_cnt,
                                   (cudaStream_t)stream);
}
