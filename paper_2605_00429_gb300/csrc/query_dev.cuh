// Device functions of the query path, shared by the single-mesh kernels (query.cu) and the
// batched persistent kernels (batch.cu).
#pragma once

#include "geom.cuh"
#include "p2m_internal.h"

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

// Warp-cooperative scan of one long list (all 32 lanes call it with the same query): lanes
// test 32 chunk boxes at once (ballot), then the entries of each surviving chunk one per
// lane; the (d2, id) minimum is reduced across the warp with two 32-bit redux operations and
// the bound shrinks after every chunk.  Returns false if no triangle was found.
template <bool COUNT>
__device__ __forceinline__ bool warp_scan_list(const MeshView& m, float3 q, int site, unsigned& bhi, unsigned& blo,
                                               float& bs, float& bt, unsigned long long* counters) {
    const int lane = threadIdx.x & 31;
    const int r0 = __ldg(m.row_off + site), r1 = __ldg(m.row_off + site + 1);
    const int c0 = __ldg(m.chunk_off + site), nc = __ldg(m.chunk_off + site + 1) - c0;
    float bound = ref_bound(m, q, site);
    bhi = 0xffffffffu;
    blo = 0xffffffffu;
    bs = 0.0f;
    bt = 0.0f;
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
            if ((mhi < bhi || (mhi == bhi && mlo < blo)) && (mhi != 0xffffffffu || mlo != 0xffffffffu)) {
                const int owner = __ffs(__ballot_sync(0xffffffffu, khi == mhi && klo == mlo)) - 1;
                bs = __shfl_sync(0xffffffffu, s, owner);
                bt = __shfl_sync(0xffffffffu, t, owner);
                bhi = mhi;
                blo = mlo;
                bound = fminf(bound, fmaf(sqrtf(__uint_as_float(mhi)), 1.0f + 9.6e-7f, m.prune_abs));
            }
        }
    }
    if (COUNT) {
        atomicAdd(counters + C_ROWS, (unsigned long long)n_entries);
        atomicAdd(counters + C_EXACT, (unsigned long long)n_exact);
    }
    return bhi != 0xffffffffu || blo != 0xffffffffu;
}

}  // namespace p2m
