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
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

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
                                                     unsigned long long* counters, const int32_t* __restrict__ perm,
                                                     int2* __restrict__ cand, unsigned char* __restrict__ flag) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm ? (int64_t)__ldg(perm + k) : k;
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        int cell;
        int site = -1;
        if (grid_cell(m, q, cell)) site = nearest_site<COUNT>(m, q, cell, counters);
        const bool is_long = site >= 0 && __ldg(m.row_off + site + 1) - __ldg(m.row_off + site) > m.long_row;
        if (flag) {
            // sorted order: mark long queries; an order-preserving compaction follows
            flag[k] = is_long;
            cand[k] = make_int2((int)i, site);
        }
        if (is_long) {
            if (!flag) longq[atomicAdd(n_long, 1)] = make_int2((int)i, site);
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

// Warp-per-query pass over the queued long lists.  With `head` given (an order-preserving
// queue, which keeps the queries of one site together), each block claims runs of kSeg
// consecutive entries, so one SM works through one site's queries and reuses its list in L1;
// warps take the run's entries one at a time.  Without `head`, warps stride over the queue.
constexpr int kSeg = 128;

template <bool COUNT>
__device__ __forceinline__ void warp_query_one(const MeshView& m, const float* __restrict__ pts, int2 qs,
                                               float* __restrict__ dist, float* __restrict__ closest,
                                               int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                               int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                               unsigned long long* counters) {
    const int64_t i = qs.x;
    const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    unsigned bhi, blo;
    float bs, bt;
    const bool found = warp_scan_list<COUNT>(m, q, qs.y, bhi, blo, bs, bt, counters);
    if ((threadIdx.x & 31) == 0) {
        if (!found) rest[atomicAdd(n_rest, 1)] = (int32_t)i;
        else write_result(m, i, ((unsigned long long)bhi << 32) | blo, bs, bt, dist, closest, tri_out, bary);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(256) k_query_warp(MeshView m, const float* __restrict__ pts,
                                                   const int2* __restrict__ longq, const int* __restrict__ n_long,
                                                   float* __restrict__ dist, float* __restrict__ closest,
                                                   int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                                   int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                                   unsigned long long* counters, int* __restrict__ head) {
    const int nq = *n_long;
    if (!head) {
        const int nwarps = (gridDim.x * blockDim.x) >> 5;
        for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nq; k += nwarps)
            warp_query_one<COUNT>(m, pts, longq[k], dist, closest, tri_out, bary, rest, n_rest, counters);
        return;
    }
    __shared__ int s_base, s_next;
    const int lane = threadIdx.x & 31;
    while (true) {
        if (threadIdx.x == 0) {
            s_base = atomicAdd(head, kSeg);
            s_next = 0;
        }
        __syncthreads();
        const int base = s_base;
        if (base >= nq) break;  // uniform over the block
        while (true) {
            int j = 0;
            if (lane == 0) j = atomicAdd(&s_next, 1);
            j = __shfl_sync(0xffffffffu, j, 0);
            if (j >= kSeg || base + j >= nq) break;
            warp_query_one<COUNT>(m, pts, longq[base + j], dist, closest, tri_out, bary, rest, n_rest, counters);
        }
        __syncthreads();  // the run is finished before s_base changes
    }
}

// Sort key of a query: the Morton code of its grid cell (8 bits per axis, G <= 256), so that
// neighbouring threads of the sorted order read the same candidate lists, interception lists
// and triangles.  Points outside the domain box sort last.
__device__ __forceinline__ unsigned spread8(unsigned v) {
    v &= 0xffu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_query_keys(MeshView m, const float* __restrict__ pts, int64_t n, unsigned* __restrict__ key,
                             int32_t* __restrict__ idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        const float fx = (q.x - m.lo.x) * m.inv_h.x, fy = (q.y - m.lo.y) * m.inv_h.y, fz = (q.z - m.lo.z) * m.inv_h.z;
        unsigned k = 0xffffffu;
        if (fx >= 0.0f && fy >= 0.0f && fz >= 0.0f && fx < (float)m.G && fy < (float)m.G && fz < (float)m.G)
            k = (spread8((unsigned)fx) << 2) | (spread8((unsigned)fy) << 1) | spread8((unsigned)fz);
        key[i] = k;
        idx[i] = (int32_t)i;
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
    // scratch: rest ids [n], long queue [n] of int2, counters, and for the sorted schedule the
    // sort keys / permutation double buffers, per-query (query, site) pairs and long flags,
    // and the temporary storage of the radix sort and of the compaction
    const bool sorted = m.sorted && n >= 4096 && n <= 0x7fffffff;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t rest_bytes = up(sizeof(int32_t) * n), long_bytes = up(sizeof(int2) * n), cnt_bytes = 256;
    size_t sort_tmp = 0, sel_tmp = 0;
    if (sorted) {
        P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, sort_tmp, (unsigned*)nullptr, (unsigned*)nullptr,
                                                     (int32_t*)nullptr, (int32_t*)nullptr, (int)n, 0, 24, s));
        P2M_CUDA_TRY(cub::DeviceSelect::Flagged(nullptr, sel_tmp, (int2*)nullptr, (unsigned char*)nullptr, (int2*)nullptr,
                                                (int*)nullptr, (int)n, s));
    }
    const size_t a4 = up(sizeof(int32_t) * n);
    const size_t sort_bytes = sorted ? 4 * a4 + up(sizeof(int2) * n) + up(n) + up(std::max(sort_tmp, sel_tmp)) : 0;
    P2M_TRY(rest.ensure(rest_bytes + long_bytes + cnt_bytes + sort_bytes));
    char* base = rest.as<char>();
    int32_t* d_rest = reinterpret_cast<int32_t*>(base);
    int2* d_long = reinterpret_cast<int2*>(base + rest_bytes);
    int* d_cnt = reinterpret_cast<int*>(base + rest_bytes + long_bytes);  // [0] rest, [1] long, [2] head
    P2M_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), s));
    const int threads = 256;
    const int blocks = query_grid_blocks(n, threads);
    const int wblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 152LL * 16));
    const int32_t* perm = nullptr;
    int2* cand = nullptr;
    unsigned char* flag = nullptr;
    void* sel_buf = nullptr;
    if (sorted) {
        char* sb = base + rest_bytes + long_bytes + cnt_bytes;
        unsigned* k0 = reinterpret_cast<unsigned*>(sb);
        unsigned* k1 = reinterpret_cast<unsigned*>(sb + a4);
        int32_t* i0 = reinterpret_cast<int32_t*>(sb + 2 * a4);
        int32_t* i1 = reinterpret_cast<int32_t*>(sb + 3 * a4);
        cand = reinterpret_cast<int2*>(sb + 4 * a4);
        flag = reinterpret_cast<unsigned char*>(sb + 4 * a4 + up(sizeof(int2) * n));
        sel_buf = sb + 4 * a4 + up(sizeof(int2) * n) + up(n);
        k_query_keys<<<blocks, threads, 0, s>>>(v, d_pts, n, k0, i0);
        P2M_CUDA_TRY(cudaGetLastError());
        cub::DoubleBuffer<unsigned> dk(k0, k1);
        cub::DoubleBuffer<int32_t> dv(i0, i1);
        P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(sel_buf, sort_tmp, dk, dv, (int)n, 0, 24, s));
        perm = dv.Current();
    }
    if (counters)
        k_query_thread<true><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                        d_long, d_cnt + 1, counters, perm, cand, flag);
    else
        k_query_thread<false><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                         d_long, d_cnt + 1, nullptr, perm, cand, flag);
    P2M_CUDA_TRY(cudaGetLastError());
    int* head = nullptr;
    if (sorted) {
        // order-preserving compaction of the long queries (count written on the device)
        P2M_CUDA_TRY(cub::DeviceSelect::Flagged(sel_buf, sel_tmp, cand, flag, d_long, d_cnt + 1, (int)n, s));
        head = d_cnt + 2;
    }
    if (counters)
        k_query_warp<true><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                       d_rest, d_cnt, counters, head);
    else
        k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                        d_rest, d_cnt, nullptr, head);
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
                                                     d_cnt + 1, nullptr, nullptr, nullptr, nullptr);
    k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary, d_rest,
                                                    d_cnt, nullptr, nullptr);
    P2M_CUDA_TRY(cudaGetLastError());
    return launch_bvh_closest(v, d_pts, d_rest, d_cnt, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

}  // namespace p2m
