// Device functions of the query path, shared by the single-mesh kernels (query.cu) and the
// batched persistent kernels (batch.cu).
#pragma once

#include "geom.cuh"
#include "p2m_internal.h"

namespace p2m {

enum { C_OUTSIDE = 0, C_SITES = 1, C_TIES = 2, C_ROWS = 3, C_EXACT = 4, C_LONG = 5, C_LONG_ROWS = 6, C_QUERIED = 7 };

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

// Nearest site among the grid cell's candidates: site ids (4 B each) whose positions come
// from the site table, which stays in cache.
template <bool COUNT>
__device__ __forceinline__ int nearest_site(const MeshView& m, float3 q, int cell, unsigned long long* counters) {
    const int j0 = __ldg(m.cell_off + cell), j1 = __ldg(m.cell_off + cell + 1);
    auto cand = [&](int j, int& s) {
        s = __ldg(m.cell_id + j);
        return __ldg(m.sites + s);
    };
    float bd = INFINITY, sd = INFINITY;
    int bs = -1;
    for (int j = j0; j < j1; ++j) {
        int s;
        const float4 p = cand(j, s);
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
            int s;
            const float4 p = cand(j, s);
            const float dx = q.x - p.x, dy = q.y - p.y, dz = q.z - p.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > lim) continue;
            const double ex = (double)q.x - (double)p.x, ey = (double)q.y - (double)p.y, ez = (double)q.z - (double)p.z;
            const double d2 = ex * ex + ey * ey + ez * ez;
            if (d2 < best || (d2 == best && s < bi)) { best = d2; bi = s; }
        }
        bs = bi;
    }
    if (COUNT && bs >= 0)
        atomicAdd(counters + C_QUERIED, (unsigned long long)(__ldg(m.row_off + bs + 1) - __ldg(m.row_off + bs)));
    return bs;
}

constexpr int kChunk = 32;  // list entries per chunk box (matches the list build)

__device__ __forceinline__ float ref_bound(const MeshView& m, float3 q, int site) {
    const float4 ref = __ldg(m.refs + site);
    const float rx = q.x - ref.x, ry = q.y - ref.y, rz = q.z - ref.z;
    const float b = sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz))) + ref.w;
    return fmaf(b, 1.0f + 9.6e-7f, m.prune_abs);
}

// Squared lower bound of the distance from q to the triangles of chunk c: the larger of the
// distance to the chunk's box and the distance to its normal slab {x : hmin <= n.x <= hmax}
// (n = the chunk's mean unit normal, hmin / hmax padded like the box).
__device__ __forceinline__ float chunk_dist2(const MeshView& m, int c, float3 q) {
    const float4* r = m.cbox + 3 * (int64_t)c;
    const float4 lo = __ldg(r), hi = __ldg(r + 1), n = __ldg(r + 2);
    const float h = dot3(f3(n), q);
    const float slab = fmaxf(fmaxf(lo.w - h, h - hi.w), 0.0f);
    return fmaxf(box_dist2(q, f3(lo), f3(hi)), slab * slab);
}

__device__ __forceinline__ bool chunk_may_hit(const MeshView& m, int c, float3 q, float bound) {
    return chunk_dist2(m, c, q) <= bound * bound;
}

// Thread scan of one interception list, chunk by chunk; returns the (d2, tri) key and the
// (s, t) of the winner.
template <bool COUNT>
__device__ __forceinline__ unsigned long long scan_list(const MeshView& m, float3 q, int site, float& bs, float& bt,
                                                        unsigned long long* counters) {
    const int r0 = __ldg(m.row_off + site), r1 = __ldg(m.row_off + site + 1);
    const int c0 = __ldg(m.chunk_off + site), c1 = __ldg(m.chunk_off + site + 1);
    const float4 ref = __ldg(m.refs + site);
    const float rx = q.x - ref.x, ry = q.y - ref.y, rz = q.z - ref.z;
    const float dq = sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
    float bound = fmaf(dq + ref.w, 1.0f + 9.6e-7f, m.prune_abs);
    // a list of at most long_row entries is sorted by key = ||ref - c_f|| - r_f: once
    // key - ||q - ref|| exceeds the bound, so does every later entry's lower bound
    const bool sorted_list = r1 - r0 <= m.long_row;
    const float dq_up = fmaf(dq, 1.0f + 9.6e-7f, m.prune_abs);
    unsigned long long best = ~0ull;
    int n_exact = 0, n_entries = 0;
    bool done = false;
    for (int c = c0; c < c1 && !done; ++c) {
        if (!chunk_may_hit(m, c, q, bound)) continue;
        const int j0 = r0 + (c - c0) * kChunk, j1 = min(j0 + kChunk, r1);
        for (int j = j0; j < j1; ++j) {
            const int2 e = __ldg(m.row_ent + j);
            if (sorted_list && __int_as_float(e.y) > bound + dq_up) {
                done = true;
                break;
            }
            if (COUNT) ++n_entries;
            const int f = e.x;
            const float4 sp = __ldg(m.tsph + f);
            const float dx = q.x - sp.x, dy = q.y - sp.y, dz = q.z - sp.z;
            const float lim = bound + sp.w;
            const float dc2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (dc2 > lim * lim) continue;
            // plane and sphere together give a second, tighter bound from half of the record
            if (tri_lower_bound2(m.tri, f, q, sp, dc2, 8.0f * m.prune_abs) > bound * bound) continue;
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

// The same scan over a list staged in shared memory by the block (see k_query_staged):
// entries ent[0, len), their bounding spheres sph[] and full triangle records rec[][4].  A
// staged list is short, so sorted by key and scanned with the early exit alone (chunk boxes
// of a key-sorted list are shells around the reference point and prune little; testing them
// measured no faster).  Returns the (d2, tri) key and the winner's (s, t) and staged
// position (for its record).
template <bool COUNT>
__device__ __forceinline__ unsigned long long scan_list_staged(const MeshView& m, float3 q, int site, const int2* ent,
                                                               const float4* sph, const float4 (*rec)[4], int len,
                                                               float& bs, float& bt, int& bpos,
                                                               unsigned long long* counters) {
    const float4 ref = __ldg(m.refs + site);
    const float rx = q.x - ref.x, ry = q.y - ref.y, rz = q.z - ref.z;
    const float dq = sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
    float bound = fmaf(dq + ref.w, 1.0f + 9.6e-7f, m.prune_abs);
    const float dq_up = fmaf(dq, 1.0f + 9.6e-7f, m.prune_abs);
    unsigned long long best = ~0ull;
    int n_exact = 0, n_entries = 0;
    for (int j = 0; j < len; ++j) {
        const int2 e = ent[j];
        // every later entry's lower bound exceeds the bound too
        if (__int_as_float(e.y) > bound + dq_up) break;
        if (COUNT) ++n_entries;
        const float4 sp = sph[j];
        const float dx = q.x - sp.x, dy = q.y - sp.y, dz = q.z - sp.z;
        const float lim = bound + sp.w;
        const float dc2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (dc2 > lim * lim) continue;
        if (tri_lower_bound2_rec(rec[j][0], rec[j][1], q, sp, dc2, 8.0f * m.prune_abs) > bound * bound) continue;
        if (COUNT) ++n_exact;
        TriRec T;
        T.r0 = rec[j][0];
        T.r1 = rec[j][1];
        T.r2 = rec[j][2];
        T.r3 = rec[j][3];
        float s, t;
        const float d2 = tri_dist2(q, T, s, t);
        const unsigned long long key = dist_key(d2, e.x);
        if (key < best) {
            best = key;
            bs = s;
            bt = t;
            bpos = j;
            bound = fminf(bound, fmaf(sqrtf(d2), 1.0f + 9.6e-7f, m.prune_abs));
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
    if (tri_out) tri_out[i] = __ldg(m.orig + f);
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

// The same result as one 32-byte record at rec[2i .. 2i+1]: (distance, closest point) and
// (original triangle id bits, barycentrics).  Queries taken in sorted order land at random
// indices; a record fills one whole 32-byte sector, where the four separate outputs would
// each touch a partial sector.  k_split_records turns the records into the output arrays.
__device__ __forceinline__ void write_record(const MeshView& m, float4* __restrict__ rec, int64_t i,
                                             unsigned long long key, float s, float t) {
    const int f = (int)(key & 0xffffffffu);
    const TriRec T = load_tri(m.tri, f);
    const float3 p = tri_point(T, s, t);
    rec[2 * i] = make_float4(sqrtf(__uint_as_float((unsigned)(key >> 32))), p.x, p.y, p.z);
    rec[2 * i + 1] = make_float4(__int_as_float(__ldg(m.orig + f)), 1.0f - s - t, s, t);
}

__device__ __forceinline__ float box2_dist2(const float4* __restrict__ box, int64_t k, float3 q) {
    const float4 lo = __ldg(box + 2 * k), hi = __ldg(box + 2 * k + 1);
    return box_dist2(q, f3(lo), f3(hi));
}

// Warp-cooperative, best-first scan of one long list (all 32 lanes call it with the same
// query).  The list is a sequence of 32-entry chunks, and every 32 chunks have a level-1
// box.  The warp first scans the level-1 box nearest to q, which makes the bound tight
// early; it then visits level-1 boxes, and the chunks inside each, in ascending box
// distance (selected with redux.sync + ballot), stopping at the bound.  Within a chunk the
// entries go one per lane, and the (d2, id) minimum is reduced across the warp with two
// 32-bit redux operations.  Anything skipped has a box farther than the bound at the time
// of the test, and the bound only shrinks, so the result is the list's exact minimum.
// Returns false if no triangle was found.
template <bool COUNT>
__device__ __forceinline__ bool warp_scan_list(const MeshView& m, float3 q, int site, unsigned& bhi, unsigned& blo,
                                               float& bs, float& bt, unsigned long long* counters) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int r0 = __ldg(m.row_off + site), r1 = __ldg(m.row_off + site + 1);
    const int c0 = __ldg(m.chunk_off + site), nc = __ldg(m.chunk_off + site + 1) - c0;
    const int p0 = __ldg(m.l1_off + site), np = __ldg(m.l1_off + site + 1) - p0;
    float bound = ref_bound(m, q, site);
    bhi = 0xffffffffu;
    blo = 0xffffffffu;
    bs = 0.0f;
    bt = 0.0f;
    int n_exact = 0, n_entries = 0;

    // entries of chunk c (warp-uniform), one per lane
    auto do_chunk = [&](int c) {
        const int j = r0 + c * kChunk + lane;
        unsigned khi = 0xffffffffu, klo = 0xffffffffu;
        float s = 0.0f, t = 0.0f;
        if (j < min(r0 + (c + 1) * kChunk, r1)) {
            if (COUNT) ++n_entries;
            // the sphere in list order when the list has it (a coalesced load beside the id)
            const int f = __ldg(&m.row_ent[j].x);
            const float4 sp = m.row_sph ? __ldg(m.row_sph + j) : __ldg(m.tsph + f);
            const float dx = q.x - sp.x, dy = q.y - sp.y, dz = q.z - sp.z;
            const float lim = bound + sp.w;
            const float dc2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (dc2 <= lim * lim && tri_lower_bound2(m.tri, f, q, sp, dc2, 8.0f * m.prune_abs) <= bound * bound) {
                if (COUNT) ++n_exact;
                const TriRec T = load_tri(m.tri, f);
                const float d2 = tri_dist2(q, T, s, t);
                khi = __float_as_uint(d2);
                klo = (unsigned)f;
            }
        }
        const unsigned mhi = __reduce_min_sync(FULL, khi);
        const unsigned mlo = __reduce_min_sync(FULL, khi == mhi ? klo : 0xffffffffu);
        if ((mhi < bhi || (mhi == bhi && mlo < blo)) && (mhi != 0xffffffffu || mlo != 0xffffffffu)) {
            const int owner = __ffs(__ballot_sync(FULL, khi == mhi && klo == mlo)) - 1;
            bs = __shfl_sync(FULL, s, owner);
            bt = __shfl_sync(FULL, t, owner);
            bhi = mhi;
            blo = mlo;
            bound = fminf(bound, fmaf(sqrtf(__uint_as_float(mhi)), 1.0f + 9.6e-7f, m.prune_abs));
        }
    };
    // chunks of level-1 box p, nearest first
    auto do_node = [&](int p) {
        const int ch = 32 * p + lane;
        const float d = ch < nc ? chunk_dist2(m, c0 + ch, q) : INFINITY;
        bool live = d <= bound * bound;
        while (__any_sync(FULL, live)) {
            const unsigned dm = __reduce_min_sync(FULL, live ? __float_as_uint(d) : 0xffffffffu);
            if (__uint_as_float(dm) > bound * bound) break;
            const int owner = __ffs(__ballot_sync(FULL, live && __float_as_uint(d) == dm)) - 1;
            if (lane == owner) live = false;
            do_chunk(32 * p + owner);
        }
    };
    // pre-pass: the nearest level-1 box
    unsigned nd = 0xffffffffu, ni = 0xffffffffu;
    for (int pb = 0; pb < np; pb += 32) {
        const int p = pb + lane;
        const unsigned d = p < np ? __float_as_uint(box2_dist2(m.l1box, p0 + p, q)) : 0xffffffffu;
        const unsigned dmin = __reduce_min_sync(FULL, d);
        const unsigned imin = __reduce_min_sync(FULL, d == dmin ? (unsigned)p : 0xffffffffu);
        if (dmin < nd) { nd = dmin; ni = imin; }
    }
    const int first = (int)ni;
    if (np > 0 && __uint_as_float(nd) <= bound * bound) do_node(first);
    // the other level-1 boxes, nearest first within each group of 32
    for (int pb = 0; pb < np; pb += 32) {
        const int p = pb + lane;
        const float d = (p < np && p != first) ? box2_dist2(m.l1box, p0 + p, q) : INFINITY;
        bool live = d <= bound * bound;
        while (__any_sync(FULL, live)) {
            const unsigned dm = __reduce_min_sync(FULL, live ? __float_as_uint(d) : 0xffffffffu);
            if (__uint_as_float(dm) > bound * bound) break;
            const int owner = __ffs(__ballot_sync(FULL, live && __float_as_uint(d) == dm)) - 1;
            if (lane == owner) live = false;
            do_node(pb + owner);
        }
    }
    if (COUNT) {
        atomicAdd(counters + C_ROWS, (unsigned long long)n_entries);
        atomicAdd(counters + C_EXACT, (unsigned long long)n_exact);
        atomicAdd(counters + C_LONG_ROWS, (unsigned long long)n_entries);
        if (lane == 0) atomicAdd(counters + C_LONG, 1ull);
    }
    return bhi != 0xffffffffu || blo != 0xffffffffu;
}

}  // namespace p2m
