// Query path (Section 3.3 "Distance Query Stage"):
//   K2  nearest site: one grid lookup, an FP32 scan of the cell's candidate sites, and an
//       FP64 re-check when the two best are within 4e-6 (relative, squared) of each other;
//       ties go to the lower site index.
//   K3  list scan: the site's interception list, with bounding-sphere pruning ("Bounding
//       Sphere Pruning"): a triangle is tested exactly only if ||q - c|| - r does not exceed
//       the current bound.  The bound starts at the distance to the site's reference point on
//       the mesh (an upper bound of d(q, M)), so pruning works from the first entry.  The
//       minimum is taken over (squared distance, triangle id).
//   K5  points outside the domain box D (or, defensively, whose list gave no triangle) are
//       compacted and answered by the exact BVH search.
#include "host.h"
#include "query_dev.cuh"

namespace p2m {

// Thread-per-query schedule: fused nearest-site search and list scan.  A query whose list
// is longer than m.long_row is queued (query, site) for the warp-per-query scan.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_query_thread(MeshView m, const float* __restrict__ pts, int64_t n,
                                                     float* __restrict__ dist, float* __restrict__ closest,
                                                     int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                                     int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                                     int2* __restrict__ longq, int* __restrict__ n_long,
                                                     unsigned long long* counters) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        int cell;
        int site = -1;
        if (grid_cell(m, q, cell)) site = nearest_site<COUNT>(m, q, cell, counters);
        if (site >= 0 && __ldg(m.row_off + site + 1) - __ldg(m.row_off + site) > m.long_row) {
            longq[atomicAdd(n_long, 1)] = make_int2((int)i, site);
            continue;
        }
        unsigned long long key = ~0ull;
        float s = 0.0f, t = 0.0f;
        if (site >= 0) key = scan_list<COUNT>(m, q, site, s, t, counters);
        if (key == ~0ull) {
            rest[atomicAdd(n_rest, 1)] = (int32_t)i;
            if (COUNT) atomicAdd(counters + C_OUTSIDE, 1ull);
            continue;
        }
        write_result(m, i, key, s, t, dist, closest, tri_out, bary);
    }
}

// Warp-per-query schedule for the queued long lists.
template <bool COUNT>
__global__ void __launch_bounds__(256, 2) k_query_warp(MeshView m, const float* __restrict__ pts,
                                                   const int2* __restrict__ longq, const int* __restrict__ n_long,
                                                   float* __restrict__ dist, float* __restrict__ closest,
                                                   int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                                   int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                                   unsigned long long* counters) {
    const int lane = threadIdx.x & 31;
    const int nq = *n_long;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nq; k += nwarps) {
        const int2 qs = longq[k];
        const int64_t i = qs.x;
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        unsigned bhi, blo;
        float bs, bt;
        const bool found = warp_scan_list<COUNT>(m, q, qs.y, bhi, blo, bs, bt, counters);
        if (lane == 0) {
            if (!found) rest[atomicAdd(n_rest, 1)] = (int32_t)i;
            else write_result(m, i, ((unsigned long long)bhi << 32) | blo, bs, bt, dist, closest, tri_out, bary);
        }
    }
}

__global__ void k_site_only(MeshView m, const float* __restrict__ pts, int64_t n, int32_t* __restrict__ site_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        int cell;
        site_out[i] = grid_cell(m, q, cell) ? nearest_site<false>(m, q, cell, nullptr) : -1;
    }
}

int query_grid_blocks(int64_t n, int threads) {
    const int64_t want = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, 152LL * 64));
}

int run_query(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
              int32_t* d_tri, float* d_bary, unsigned long long* counters, DevBuf& rest, cudaStream_t s) {
    const MeshView v = m.view();
    if (v.G == 0) return launch_bvh_closest(v, d_pts, nullptr, nullptr, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
    // scratch: rest ids [n], long queue [n] of int2, two counters
    const size_t rest_bytes = ((sizeof(int32_t) * n + 255) / 256) * 256;
    const size_t long_bytes = ((sizeof(int2) * n + 255) / 256) * 256;
    P2M_TRY(rest.ensure(rest_bytes + long_bytes + 256));
    int32_t* d_rest = rest.as<int32_t>();
    int2* d_long = reinterpret_cast<int2*>(rest.as<char>() + rest_bytes);
    int* d_cnt = reinterpret_cast<int*>(rest.as<char>() + rest_bytes + long_bytes);
    P2M_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int), s));
    const int threads = 256;
    const int blocks = query_grid_blocks(n, threads);
    const int wblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152LL * 16));
    if (counters) {
        k_query_thread<true><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                        d_long, d_cnt + 1, counters);
        k_query_warp<true><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                       d_rest, d_cnt, counters);
    } else {
        k_query_thread<false><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                         d_long, d_cnt + 1, nullptr);
        k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                        d_rest, d_cnt, nullptr);
    }
    P2M_CUDA_TRY(cudaGetLastError());
    // the points left over take the exact BVH search; the count stays on the device
    return launch_bvh_closest(v, d_pts, d_rest, d_cnt, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

int run_nearest_site(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, int32_t* d_site, cudaStream_t s) {
    (void)h;
    const MeshView v = m.view();
    if (v.G == 0) return fail(P2M_ERR_INVALID_ARG, "index has no nearest-site grid");
    k_site_only<<<query_grid_blocks(n, 256), 256, 0, s>>>(v, d_pts, n, d_site);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

}  // namespace p2m

namespace p2m {

// The same launch sequence as run_query, on scratch memory the caller provides: d_rest
// holds n int32, d_long n int2, d_cnt two ints.  Nothing is allocated here.
int launch_query_on_scratch(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
                            int32_t* d_tri, float* d_bary, int32_t* d_rest, int2* d_long, int* d_cnt, cudaStream_t s) {
    const MeshView v = m.view();
    if (v.G == 0) return launch_bvh_closest(v, d_pts, nullptr, nullptr, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
    P2M_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int), s));
    const int threads = 256;
    const int blocks = query_grid_blocks(n, threads);
    const int wblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152LL * 16));
    k_query_thread<false><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt, d_long,
                                                     d_cnt + 1, nullptr);
    k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary, d_rest,
                                                    d_cnt, nullptr);
    P2M_CUDA_TRY(cudaGetLastError());
    return launch_bvh_closest(v, d_pts, d_rest, d_cnt, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

}  // namespace p2m
