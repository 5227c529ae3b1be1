// Query path: nearest site (K2) + interception-list scan (K3), and the BVH search (K5) for
// points outside the clipped domain.
#include "geom.cuh"
#include "host.h"

namespace p2m {

int run_query(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
              int32_t* d_tri, float* d_bary, unsigned long long* counters, cudaStream_t s) {
    (void)counters;
    const MeshView v = m.view();
    return launch_bvh_closest(v, d_pts, nullptr, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

int run_nearest_site(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, int32_t* d_site, cudaStream_t s) {
    (void)h; (void)m; (void)d_pts; (void)n; (void)d_site; (void)s;
    return fail(P2M_ERR_NOT_IMPLEMENTED, "nearest-site search not built yet");
}

}  // namespace p2m
