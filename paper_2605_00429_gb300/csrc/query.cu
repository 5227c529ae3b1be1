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
#include "geom.cuh"
#include "host.h"

namespace p2m {

enum { C_OUTSIDE = 0, C_SITES = 1, C_TIES = 2, C_ROWS = 3, C_EXACT = 4 };

__device__ __forceinline__ bool grid_cell(const MeshView& m, float3 q, int& cell) {
    const float fx = (q.x - m.lo.x) * m.inv_h.x;
    const float fy = (q.y - m.lo.y) * m.inv_h.y;
    const float fz = (q.z - m.lo.z) * m.inv_h.z;
    // NaN fails every comparison and lands outside
    if (!(fx >= 0.0f && fy >= 0.0f && fz >= 0.0f && fx < (float)m.G && fy < (float)m.G && fz < (float)m.G)) return false;
    const int ix = min((int)fx, m.G - 1), iy = min((int)fy, m.G - 1), iz = min((int)fz, m.G - 1);
    cell = (iz * m.G + iy) * m.G + ix;
    return true;
}

// Nearest site among the grid cell's candidates.
template <bool COUNT>
__device__ __forceinline__ int nearest_site(const MeshView& m, float3 q, int cell, unsigned long long* counters) {
    const int j0 = __ldg(m.cell_off + cell), j1 = __ldg(m.cell_off + cell + 1);
    float bd = INFINITY, sd = INFINITY;
    int bs = -1;
    for (int j = j0; j < j1; ++j) {
        const int s = __ldg(m.cell_site + j);
        const float4 p = __ldg(m.sites + s);
        const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (d2 < bd || (d2 == bd && s < bs)) {
            sd = bd;
            bd = d2;
            bs = s;
        } else if (d2 < sd) {
            sd = d2;
        }
    }
    if (COUNT) atomicAdd(counters + C_SITES, (unsigned long long)(j1 - j0));
    if (sd <= bd * (1.0f + 4e-6f) + 1e-30f) {
        // near tie: decide in FP64 (differences of FP32 coordinates are exact in FP64)
        if (COUNT) atomicAdd(counters + C_TIES, 1ull);
        const float lim = bd * (1.0f + 8e-6f) + 1e-30f;
        double best = 1e300;
        int bi = -1;
        for (int j = j0; j < j1; ++j) {
            const int s = __ldg(m.cell_site + j);
            const float4 p = __ldg(m.sites + s);
            const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > lim) continue;
            const double ex = (double)q.x - (double)p.x, ey = (double)q.y - (double)p.y, ez = (double)q.z - (double)p.z;
            const double d2 = ex * ex + ey * ey + ez * ez;
            if (d2 < best || (d2 == best && s < bi)) { best = d2; bi = s; }
        }
        bs = bi;
    }
    return bs;
}

constexpr int kChunk = 32;  // list entries per chunk box (matches the list build)

__device__ __forceinline__ float ref_bound(const MeshView& m, float3 q, int site) {
    const float4 ref = __ldg(m.refs + site);
    const float rx = q.x - ref.x, ry = q.y - ref.y, rz = q.z - ref.z;
    const float b = sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz))) + ref.w;
    return fmaf(b, 1.0f + 9.6e-7f, m.prune_abs);
}

__device__ __forceinline__ bool chunk_may_hit(const MeshView& m, int c, float3 q, float bound) {
    const float4 lo = __ldg(m.cbox + 2 * (int64_t)c), hi = __ldg(m.cbox + 2 * (int64_t)c + 1);
    return box_dist2(q, f3(lo), f3(hi)) <= bound * bound;
}

// Thread scan of one interception list, chunk by chunk; returns the (d2, tri) key and the
// (s, t) of the winner.
template <bool COUNT>
__device__ __forceinline__ unsigned long long scan_list(const MeshView& m, float3 q, int site, float& bs, float& bt,
                                                        unsigned long long* counters) {
    const int r0 = __ldg(m.row_off + site), r1 = __ldg(m.row_off + site + 1);
    const int c0 = __ldg(m.chunk_off + site), c1 = __ldg(m.chunk_off + site + 1);
    float bound = ref_bound(m, q, site);
    unsigned long long best = ~0ull;
    int n_exact = 0, n_entries = 0;
    for (int c = c0; c < c1; ++c) {
        if (!chunk_may_hit(m, c, q, bound)) continue;
        const int j0 = r0 + (c - c0) * kChunk, j1 = min(j0 + kChunk, r1);
        if (COUNT) n_entries += j1 - j0;
        for (int j = j0; j < j1; ++j) {
            const int f = __ldg(m.row_tri + j);
            const float4 sp = __ldg(m.tsph + f);
            const float dx = q.x - sp.x, dy = q.y - sp.y, dz = q.z - sp.z;
            const float lim = bound + sp.w;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > lim * lim) continue;
            if (COUNT) ++n_exact;
            const TriRec T = load_tri(m.tri, f);
            float s, t;
            const float d2 = tri_dist2(q, T, s, t);
            const unsigned long long key = dist_key(d2, f);
            if (key < best) {
                best = key;
                bs = s;
                bt = t;
                bound = fminf(bound, fmaf(sqrtf(d2), 1.0f + 9.6e-7f, m.prune_abs));
            }
        }
    }
    if (COUNT) {
        atomicAdd(counters + C_ROWS, (unsigned long long)n_entries);
        atomicAdd(counters + C_EXACT, (unsigned long long)n_exact);
    }
    return best;
}

__device__ __forceinline__ void write_result(const MeshView& m, int64_t i, unsigned long long key, float s, float t,
                                             float* __restrict__ dist, float* __restrict__ closest,
                                             int32_t* __restrict__ tri_out, float* __restrict__ bary) {
    const int f = (int)(key & 0xffffffffu);
    dist[i] = sqrtf(__uint_as_float((unsigned)(key >> 32)));
    if (tri_out) tri_out[i] = f;
    if (closest) {
        const TriRec T = load_tri(m.tri, f);
        const float3 p = tri_point(T, s, t);
        closest[3 * i] = p.x;
        closest[3 * i + 1] = p.y;
        closest[3 * i + 2] = p.z;
    }
    if (bary) {
        bary[3 * i] = 1.0f - s - t;
        bary[3 * i + 1] = s;
        bary[3 * i + 2] = t;
    }
}

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

// Warp-per-query schedule for long lists: lanes test 32 chunk boxes at once (ballot), then
// the entries of each surviving chunk one per lane; the (d2, id) minimum is reduced across
// the warp with two 32-bit redux operations and the bound shrinks after every chunk.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_query_warp(MeshView m, const float* __restrict__ pts,
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
        const int site = qs.y;
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        const int r0 = __ldg(m.row_off + site), r1 = __ldg(m.row_off + site + 1);
        const int c0 = __ldg(m.chunk_off + site), nc = __ldg(m.chunk_off + site + 1) - c0;
        float bound = ref_bound(m, q, site);
        unsigned bhi = 0xffffffffu, blo = 0xffffffffu;  // best (d2 bits, id)
        float bs = 0.0f, bt = 0.0f;
        int n_exact = 0, n_entries = 0;
        for (int cb = 0; cb < nc; cb += 32) {
            const int ch = cb + lane;
            unsigned mask = __ballot_sync(0xffffffffu, ch < nc && chunk_may_hit(m, c0 + ch, q, bound));
            while (mask) {
                const int kk = __ffs(mask) - 1;
                mask &= mask - 1;
                const int c = cb + kk;
                if (!chunk_may_hit(m, c0 + c, q, bound)) continue;  // the bound may have shrunk
                const int j = r0 + c * kChunk + lane;
                unsigned khi = 0xffffffffu, klo = 0xffffffffu;
                float s = 0.0f, t = 0.0f;
                if (j < min(r0 + (c + 1) * kChunk, r1)) {
                    if (COUNT) ++n_entries;
                    const int f = __ldg(m.row_tri + j);
                    const float4 sp = __ldg(m.tsph + f);
                    const float dx = q.x - sp.x, dy = q.y - sp.y, dz = q.z - sp.z;
                    const float lim = bound + sp.w;
                    if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= lim * lim) {
                        if (COUNT) ++n_exact;
                        const TriRec T = load_tri(m.tri, f);
                        const float d2 = tri_dist2(q, T, s, t);
                        khi = __float_as_uint(d2);
                        klo = (unsigned)f;
                    }
                }
                const unsigned mhi = __reduce_min_sync(0xffffffffu, khi);
                const unsigned mlo = __reduce_min_sync(0xffffffffu, khi == mhi ? klo : 0xffffffffu);
                if (mhi < bhi || (mhi == bhi && mlo < blo)) {
                    if (mhi != 0xffffffffu || mlo != 0xffffffffu) {
                        const int owner = __ffs(__ballot_sync(0xffffffffu, khi == mhi && klo == mlo)) - 1;
                        bs = __shfl_sync(0xffffffffu, s, owner);
                        bt = __shfl_sync(0xffffffffu, t, owner);
                        bhi = mhi;
                        blo = mlo;
                        bound = fminf(bound, fmaf(sqrtf(__uint_as_float(mhi)), 1.0f + 9.6e-7f, m.prune_abs));
                    }
                }
            }
        }
        if (COUNT) {
            atomicAdd(counters + C_ROWS, (unsigned long long)n_entries);
            atomicAdd(counters + C_EXACT, (unsigned long long)n_exact);
        }
        if (lane == 0) {
            if (bhi == 0xffffffffu && blo == 0xffffffffu) {
                rest[atomicAdd(n_rest, 1)] = (int32_t)i;
            } else {
                const unsigned long long key = ((unsigned long long)bhi << 32) | blo;
                write_result(m, i, key, bs, bt, dist, closest, tri_out, bary);
            }
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
