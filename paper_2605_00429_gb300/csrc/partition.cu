// Build of the site partition and of everything the query reads besides the triangles.
#include "host.h"

namespace p2m {

int build_partition(MeshData& m, const p2m_build_params& prm, p2m_index* h, cudaStream_t s) {
    (void)prm; (void)h; (void)s;
    m.G = 0;  // no grid yet: every query takes the exact BVH search
    return P2M_OK;
}

}  // namespace p2m
