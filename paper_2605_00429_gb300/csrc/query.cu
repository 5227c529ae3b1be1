// Query path (Section 3.3 "Distance Query Stage"):
//   order  the queries are counting-sorted by the Morton code of their grid cell, so that
//       neighbouring threads read the same candidate and interception lists; each result
//       leaves as a 32-byte record at the query's index, split into the outputs at the end.
//   K2  nearest site: one grid lookup, an FP32 scan of the cell's candidate sites, and an
//       FP64 re-check when the two best are within 4e-6 (relative, squared) of each other;
//       ties go to the lower site index.
//   K3  list scan: the site's interception list, with bounding-sphere pruning ("Bounding
//       Sphere Pruning"): a triangle is tested exactly only if ||q - c|| - r, and a tighter
//       bound combining its plane and its sphere, do not exceed the current bound.  The
//       bound starts at the distance to the site's reference point on the mesh (an upper
//       bound of d(q, M)), so pruning works from the first entry; short lists are sorted so
//       the scan can stop early.  The minimum is taken over (squared distance, triangle id).
//   K5  points outside the domain box D (or, defensively, whose list gave no triangle) are
//       compacted and answered by the exact BVH search.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include "host.h"
#include "query_dev.cuh"

namespace p2m {

// Thread-per-query schedule: fused nearest-site search and list scan.  A query whose list
// is longer than m.long_row is queued (query, site) for the warp-per-query scan.
template <bool COUNT>
__global__ void __launch_bounds__(256, 6) k_query_thread(MeshView m, const float* __restrict__ pts, int64_t n,
                                                     float* __restrict__ dist, float* __restrict__ closest,
                                                     int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                                     int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                                     int2* __restrict__ longq, int* __restrict__ n_long,
                                                     unsigned long long* counters, const float4* __restrict__ qs,
                                                     int2* __restrict__ cand, unsigned char* __restrict__ flag,
                                                     float4* __restrict__ rec) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        // sorted order: the points were gathered into qs (xyz, index); else input order
        int64_t i = k;
        float3 q;
        if (qs) {
            const float4 p = __ldg(qs + k);
            i = __float_as_int(p.w);
            q = make_float3(p.x, p.y, p.z);
        } else {
            q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        }
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
        if (rec) write_record(m, rec, i, key, s, t);
        else write_result(m, i, key, s, t, dist, closest, tri_out, bary);
    }
}

// ---------------------------------------------------------------------------------------
// Site-staged schedule (5).  The queries are counting-sorted by their nearest site, so that
// runs of consecutive queries share one interception list; a block of 256 threads takes a
// tile of up to 1024 queries, stages the short lists of its runs (entries, bounding spheres,
// full triangle records) in shared memory, and every thread then scans its lists from there.  The lanes of a warp
// read the same staged entry at the same time (a broadcast), where the thread-per-query
// kernels gather the same data through L1 once per lane.

constexpr int kStage = 384;        // list entries one block stages
constexpr int kStageThreads = 256;
constexpr int kStagePer = 4;       // queries per thread in one block iteration (at most)
constexpr int kDqBuckets = 8;      // distance classes of the queries of one site (see k_site_rank)
constexpr int kStageRuns = 64;     // runs (sites) one tile may span; the rest scan unstaged

// Pass 1, queries in input order: nearest site (K2) and the query's rank among the queries
// of the same key.  The key is site * kDqBuckets + a distance class of the query from the site
// (below 1, 2, 4, ..., 64 site spacings, or beyond): the site's queries then come in order of
// distance,
// so that the lanes of a warp, which scan the same list, have similar bounds and stop at
// similar entries.  A point outside D gets the key n_sites * kDqBuckets.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_site_rank(MeshView m, const float* __restrict__ pts, int64_t n,
                                                  int* __restrict__ key, int* __restrict__ rank,
                                                  int* __restrict__ count, unsigned long long* counters) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        int cell;
        int site = -1;
        if (grid_cell(m, q, cell)) site = nearest_site<COUNT>(m, q, cell, counters);
        int k = m.n_sites * kDqBuckets;
        if (site >= 0) {
            const float4 sp = __ldg(m.sites + site);
            const float dx = q.x - sp.x, dy = q.y - sp.y, dz = q.z - sp.z;
            const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            int b = 0;
            for (float t = m.spacing; b < kDqBuckets - 1 && d >= t; t *= 2.0f) ++b;
            k = site * kDqBuckets + b;
        }
        key[i] = k;
        rank[i] = atomicAdd(count + k, 1);
    }
}

// Pass 2: the points to their slots in site order, as (xyz, input index).
__global__ void k_site_scatter(const float* __restrict__ pts, int64_t n, const int* __restrict__ key,
                               const int* __restrict__ rank, const int* __restrict__ first, float4* __restrict__ qs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = __ldg(key + i);
        const int64_t slot = (int64_t)__ldg(first + k) + __ldg(rank + i);
        qs[slot] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __int_as_float((int)i));
    }
}

// The record of a winner whose triangle record is already in registers.
__device__ __forceinline__ void write_record_tri(const MeshView& m, float4* __restrict__ rec, int64_t i,
                                                 unsigned long long key, float s, float t, const TriRec& T) {
    const int f = (int)(key & 0xffffffffu);
    const float3 p = tri_point(T, s, t);
    rec[2 * i] = make_float4(sqrtf(__uint_as_float((unsigned)(key >> 32))), p.x, p.y, p.z);
    rec[2 * i + 1] = make_float4(__int_as_float(__ldg(m.orig + f)), 1.0f - s - t, s, t);
}

// Pass 3: the list scan over the site-ordered queries, per * 256 per block iteration.  The
// tile's runs (sites) come from the key offsets `first` (first[s * kDqBuckets] = the first
// slot of site s, first[n_sites * kDqBuckets + 1] = n; site n_sites = outside D): a binary
// search finds the site of the
// tile's first query, and the next offsets give the runs.  Whole short lists of the runs
// (entries, bounding spheres, triangle records) are staged while they fit; each thread then
// scans per (1..kStagePer, fewer for small calls so that every SM gets tiles) queries (lanes of a warp take
// consecutive queries, mostly of one site, so their reads of the staged list are broadcasts).
template <bool COUNT>
__global__ void __launch_bounds__(kStageThreads, 5)
    k_query_staged(MeshView m, const float4* __restrict__ qs, const int* __restrict__ first, int64_t n, int per,
                   int32_t* __restrict__ rest, int* __restrict__ n_rest, int2* __restrict__ longq,
                   int* __restrict__ n_long, float4* __restrict__ rec, unsigned long long* counters) {
    __shared__ int2 s_ent[kStage];
    __shared__ float4 s_sph[kStage];
    __shared__ float4 s_rec[kStage][4];
    // runs: site, first slot, list start and length, staged entry offset (-1: not staged)
    __shared__ int s_run_site[kStageRuns], s_run_beg[kStageRuns + 1];
    __shared__ int s_run_row[kStageRuns], s_run_len[kStageRuns];
    __shared__ int s_run_off[kStageRuns];
    __shared__ int s_st_run[kStageRuns], s_st_off[kStageRuns + 1];
    __shared__ int s_nruns, s_nstaged, s_site0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int S = m.n_sites;
    // first slot of site s's queries (all its distance classes); S: the points outside D
    auto site_first = [&](int s) { return s <= S ? __ldg(first + (int64_t)s * kDqBuckets) : (int)n; };
    const int tile = kStageThreads * per;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        const int64_t tend = min(base + (int64_t)tile, n);
        if (tid == 0) {
            // the site of the tile's first query: the last s in [0, S] with first[s] <= base
            int lo = 0, hi = S;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (site_first(mid) <= base) lo = mid;
                else hi = mid - 1;
            }
            s_site0 = lo;
        }
        __syncthreads();
        if (wid == 0) {
            // runs: sites s0, s0 + 1, ... with queries in [base, tend), 32 offsets per step
            int nr = 0, s = s_site0;
            while (nr < kStageRuns && s <= S) {
                const int ss = s + lane;
                const int f0 = site_first(ss);
                const int f1 = site_first(ss + 1);
                const bool has = ss <= S && f1 > f0 && f0 < tend && f1 > base;
                const unsigned hm = __ballot_sync(0xffffffffu, has);
                const int r = nr + __popc(hm & ((1u << lane) - 1u));
                if (has && r < kStageRuns) {
                    s_run_site[r] = ss;
                    s_run_beg[r] = (int)max((int64_t)f0, base);
                }
                nr = min(kStageRuns, nr + __popc(hm));
                const bool past = ss > S || f0 >= tend;
                if (__any_sync(0xffffffffu, past)) break;
                s += 32;
            }
            if (lane == 0) s_nruns = nr;
        }
        __syncthreads();
        const int nr = s_nruns;
        if (tid < nr) {
            const int st = s_run_site[tid];
            int r0 = 0, len = 0;
            if (st < S) {
                r0 = __ldg(m.row_off + st);
                len = __ldg(m.row_off + st + 1) - r0;
            }
            s_run_row[tid] = r0;
            s_run_len[tid] = len;
        }
        __syncthreads();
        if (tid == 0) {
            // stage whole short lists in run order while they fit
            int cum = 0, k = 0;
            for (int r = 0; r < nr; ++r) {
                const int len = s_run_len[r];
                if (s_run_site[r] < S && len > 0 && len <= m.long_row && cum + len <= kStage) {
                    s_run_off[r] = cum;
                    s_st_run[k] = r;
                    s_st_off[k] = cum;
                    cum += len;
                    ++k;
                } else {
                    s_run_off[r] = -1;
                }
            }
            s_st_off[k] = cum;
            s_nstaged = k;
            // queries past the last run (a tile spanning more than kStageRuns sites) scan
            // unstaged; mark where the runs end
            s_run_beg[nr] = nr < kStageRuns ? (int)tend : s_run_beg[nr - 1];
        }
        __syncthreads();
        const int nst = s_nstaged, n_ent = s_st_off[nst];
        for (int e = tid; e < n_ent; e += kStageThreads) {
            int lo = 0, hi = nst - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_st_off[mid] <= e) lo = mid;
                else hi = mid - 1;
            }
            const int2 en = __ldg(m.row_ent + s_run_row[s_st_run[lo]] + (e - s_st_off[lo]));
            s_ent[e] = en;
            s_sph[e] = __ldg(m.tsph + en.x);
            const float4* tp = m.tri + 4 * (int64_t)en.x;
            s_rec[e][0] = __ldg(tp);
            s_rec[e][1] = __ldg(tp + 1);
            s_rec[e][2] = __ldg(tp + 2);
            s_rec[e][3] = __ldg(tp + 3);
        }
        __syncthreads();
        for (int k = 0; k < per; ++k) {
            if (base + k * kStageThreads >= tend) break;  // uniform over the block
            const int64_t j = base + k * kStageThreads + tid;
            const bool valid = j < tend;
            // the run holding slot j (runs are in slot order)
            int run = -1;
            if (valid && nr > 0 && j < s_run_beg[nr]) {
                int lo = 0, hi = nr - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_run_beg[mid] <= j) lo = mid;
                    else hi = mid - 1;
                }
                run = lo;
            }
            float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
            int site = S;
            if (valid) {
                p = __ldg(qs + j);
                if (run >= 0) {
                    site = s_run_site[run];
                } else {
                    // beyond the tile's run table: find the site by binary search of the offsets
                    int lo = 0, hi = S;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (site_first(mid) <= j) lo = mid;
                        else hi = mid - 1;
                    }
                    site = lo;
                }
            }
            const int i = __float_as_int(p.w);
            const float3 q = make_float3(p.x, p.y, p.z);
            const bool inside = valid && site < S;
            const int len = inside ? (run >= 0 ? s_run_len[run] : __ldg(m.row_off + site + 1) - __ldg(m.row_off + site)) : 0;
            const bool is_long = inside && len > m.long_row;
            {
                // long lists go to the long-list pass: one append per warp keeps a warp's
                // queries (mostly one site) together in the queue
                const unsigned lm = __ballot_sync(0xffffffffu, is_long);
                if (lm) {
                    int wbase = 0;
                    if (lane == __ffs(lm) - 1) wbase = atomicAdd(n_long, __popc(lm));
                    wbase = __shfl_sync(0xffffffffu, wbase, __ffs(lm) - 1);
                    if (is_long) longq[wbase + __popc(lm & ((1u << lane) - 1u))] = make_int2(i, site);
                }
            }
            if (!valid || is_long) continue;
            unsigned long long key = ~0ull;
            float bs = 0.0f, bt = 0.0f;
            const int off = run >= 0 ? s_run_off[run] : -1;
            if (inside && off >= 0) {
                int bpos = 0;
                key = scan_list_staged<COUNT>(m, q, site, s_ent + off, s_sph + off, s_rec + off, len, bs, bt, bpos,
                                              counters);
                if (key != ~0ull) {
                    TriRec T;
                    T.r0 = s_rec[off + bpos][0];
                    T.r1 = s_rec[off + bpos][1];
                    T.r2 = s_rec[off + bpos][2];
                    T.r3 = s_rec[off + bpos][3];
                    write_record_tri(m, rec, i, key, bs, bt, T);
                }
            } else if (inside) {
                key = scan_list<COUNT>(m, q, site, bs, bt, counters);
                if (key != ~0ull) write_record(m, rec, i, key, bs, bt);
            }
            if (key == ~0ull) {
                rest[atomicAdd(n_rest, 1)] = i;
                if (COUNT) atomicAdd(counters + C_OUTSIDE, 1ull);
            }
        }
        __syncthreads();  // the staged data and run tables are reused by the next iteration
    }
}

// Batched path, after its radix sort: the points in sorted order with their index in .w,
// so that the query kernels read them coalesced (the random gather runs here, in a
// streaming kernel).
__global__ void k_gather_points(const float* __restrict__ pts, const int32_t* __restrict__ perm, int64_t n,
                                float4* __restrict__ qs) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = __ldg(perm + k);
        qs[k] = make_float4(__ldg(pts + 3 * i), __ldg(pts + 3 * i + 1), __ldg(pts + 3 * i + 2), __int_as_float((int)i));
    }
}

// Sorted order, last step: the 32-byte result records (in input order) to the output arrays,
// coalesced.  Queries left to the BVH search have no record; that search runs afterwards and
// overwrites their outputs.
__global__ void k_split_records(const float4* __restrict__ rec, int64_t n, float* __restrict__ dist,
                                float* __restrict__ closest, int32_t* __restrict__ tri_out, float* __restrict__ bary) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldcs(rec + 2 * i), b = __ldcs(rec + 2 * i + 1);
        dist[i] = a.x;
        if (closest) {
            closest[3 * i] = a.y;
            closest[3 * i + 1] = a.z;
            closest[3 * i + 2] = a.w;
        }
        if (tri_out) tri_out[i] = __float_as_int(b.x);
        if (bary) {
            bary[3 * i] = b.y;
            bary[3 * i + 1] = b.z;
            bary[3 * i + 2] = b.w;
        }
    }
}

// Site-sorted schedule, first pass: the nearest site of every query, taken in Morton order
// (so the grid lookups of neighbouring threads hit the same cells).  The site becomes the key
// of a second radix sort that gathers the queries of each site together (the value is the
// Morton-order position); points outside the domain box get the key n_sites and sort last.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_query_sites(MeshView m, const float4* __restrict__ qs, int64_t n,
                                                    unsigned* __restrict__ skey, int32_t* __restrict__ sval,
                                                    unsigned long long* counters) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(qs + k);
        const float3 q = make_float3(p.x, p.y, p.z);
        int cell;
        int site = -1;
        if (grid_cell(m, q, cell)) site = nearest_site<COUNT>(m, q, cell, counters);
        skey[k] = site >= 0 ? (unsigned)site : (unsigned)m.n_sites;
        sval[k] = (int32_t)k;
    }
}

// Site-sorted schedule, second pass: thread per query over the queries grouped by site, so
// the lanes of a warp mostly scan the same interception list (its entries, spheres and
// triangle records are loaded once for the warp, and trip counts are alike).  Long lists are
// flagged for the order-preserving compaction, as in the Morton-ordered schedule.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_query_scan(MeshView m, const float4* __restrict__ qbuf,
                                                   const unsigned* __restrict__ skey, const int32_t* __restrict__ sval,
                                                   int64_t n, float* __restrict__ dist, float* __restrict__ closest,
                                                   int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                                   int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                                   int2* __restrict__ cand, unsigned char* __restrict__ flag,
                                                   unsigned long long* counters, float4* __restrict__ rec) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float4 p = __ldg(qbuf + __ldg(sval + k));
        const int i = __float_as_int(p.w);
        const float3 q = make_float3(p.x, p.y, p.z);
        const unsigned sk = __ldg(skey + k);
        const int site = sk < (unsigned)m.n_sites ? (int)sk : -1;
        const bool is_long = site >= 0 && __ldg(m.row_off + site + 1) - __ldg(m.row_off + site) > m.long_row;
        flag[k] = is_long;
        cand[k] = make_int2(i, site);
        if (is_long) continue;
        unsigned long long key = ~0ull;
        float s = 0.0f, t = 0.0f;
        if (site >= 0) key = scan_list<COUNT>(m, q, site, s, t, counters);
        if (key == ~0ull) {
            rest[atomicAdd(n_rest, 1)] = (int32_t)i;
            if (COUNT) atomicAdd(counters + C_OUTSIDE, 1ull);
            continue;
        }
        write_record(m, rec, i, key, s, t);
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
                                               unsigned long long* counters, float4* __restrict__ rec) {
    const int64_t i = qs.x;
    const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    unsigned bhi, blo;
    float bs, bt;
    const bool found = warp_scan_list<COUNT>(m, q, qs.y, bhi, blo, bs, bt, counters);
    if ((threadIdx.x & 31) == 0) {
        if (!found) rest[atomicAdd(n_rest, 1)] = (int32_t)i;
        else if (rec) write_record(m, rec, i, ((unsigned long long)bhi << 32) | blo, bs, bt);
        else write_result(m, i, ((unsigned long long)bhi << 32) | blo, bs, bt, dist, closest, tri_out, bary);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(256) k_query_warp(MeshView m, const float* __restrict__ pts,
                                                   const int2* __restrict__ longq, const int* __restrict__ n_long,
                                                   float* __restrict__ dist, float* __restrict__ closest,
                                                   int32_t* __restrict__ tri_out, float* __restrict__ bary,
                                                   int32_t* __restrict__ rest, int* __restrict__ n_rest,
                                                   unsigned long long* counters, int* __restrict__ head,
                                                   float4* __restrict__ rec) {
    const int nq = *n_long;
    if (!head) {
        const int nwarps = (gridDim.x * blockDim.x) >> 5;
        for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nq; k += nwarps)
            warp_query_one<COUNT>(m, pts, longq[k], dist, closest, tri_out, bary, rest, n_rest, counters, rec);
        return;
    }
    __shared__ int s_base, s_next;
    const int lane = threadIdx.x & 31;
    // runs of at most kSeg entries; shorter when the queue is short, so that it spreads over
    // the SMs instead of leaving a few blocks with long serial runs
    const int seg = max(8, min(kSeg, nq / (2 * (int)gridDim.x)));
    while (true) {
        if (threadIdx.x == 0) {
            s_base = atomicAdd(head, seg);
            s_next = 0;
        }
        __syncthreads();
        const int base = s_base;
        if (base >= nq) break;  // uniform over the block
        while (true) {
            int j = 0;
            if (lane == 0) j = atomicAdd(&s_next, 1);
            j = __shfl_sync(0xffffffffu, j, 0);
            if (j >= seg || base + j >= nq) break;
            warp_query_one<COUNT>(m, pts, longq[base + j], dist, closest, tri_out, bary, rest, n_rest, counters,
                                  rec);
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


// Counting sort of the queries by the Morton code of their grid cell (mbits bits per axis,
// G <= 2^mbits; the code shifted right by `shift` bits, i.e. the Morton code of a coarser
// grid, when the call is small): each query takes its rank inside its cell from an atomic counter, an
// exclusive scan of the counters gives each cell's first slot, and the points go straight to
// their slots as (xyz, index).  Points outside the domain box get the last key and go last.
// The order inside a cell is arbitrary; no result depends on it.
__global__ void k_cell_rank(MeshView m, const float* __restrict__ pts, int64_t n, unsigned outside_key, int shift,
                            unsigned* __restrict__ key, int32_t* __restrict__ rank, int* __restrict__ count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        const float fx = (q.x - m.lo.x) * m.inv_h.x, fy = (q.y - m.lo.y) * m.inv_h.y, fz = (q.z - m.lo.z) * m.inv_h.z;
        unsigned k = outside_key;
        if (fx >= 0.0f && fy >= 0.0f && fz >= 0.0f && fx < (float)m.G && fy < (float)m.G && fz < (float)m.G)
            k = ((spread8((unsigned)fx) << 2) | (spread8((unsigned)fy) << 1) | spread8((unsigned)fz)) >> shift;
        key[i] = k;
        rank[i] = atomicAdd(count + k, 1);
    }
}

__global__ void k_cell_scatter(const float* __restrict__ pts, int64_t n, const unsigned* __restrict__ key,
                               const int32_t* __restrict__ rank, const int* __restrict__ first,
                               float4* __restrict__ qs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = (int64_t)__ldg(first + __ldg(key + i)) + __ldg(rank + i);
        qs[slot] = make_float4(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2], __int_as_float((int)i));
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
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * 64));
}

// Site-staged schedule: nearest site + rank, scan, scatter into site order, staged scan,
// compaction of the long-list queries, warp pass, record split, BVH pass for the rest.
static int run_query_staged(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist,
                            float* d_closest, int32_t* d_tri, float* d_bary, unsigned long long* counters,
                            DevBuf& rest, cudaStream_t s) {
    const MeshView v = m.view();
    const int S = v.n_sites;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t scan_tmp = 0;
    const int K = S * kDqBuckets + 2;  // keys 0 .. S * kDqBuckets, and the end
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, scan_tmp, (int*)nullptr, (int*)nullptr, K, s));
    const size_t a4 = up(sizeof(int) * n), a8 = up(sizeof(int2) * n), a16 = up(sizeof(float4) * n);
    const size_t tmp_bytes = up(scan_tmp), site_bytes = up(sizeof(int) * K);
    // rest ids, long queue, counters | key, rank | tmp | qs | rec | site count, first
    const size_t total = a4 + a8 + 256 + 2 * a4 + tmp_bytes + a16 + 2 * a16 + 2 * site_bytes;
    P2M_TRY(rest.ensure(total));
    char* p = rest.as<char>();
    int32_t* d_rest = reinterpret_cast<int32_t*>(p); p += a4;
    int2* d_long = reinterpret_cast<int2*>(p); p += a8;
    int* d_cnt = reinterpret_cast<int*>(p); p += 256;  // [0] rest, [1] long, [2] head
    int* key = reinterpret_cast<int*>(p); p += a4;
    int* rank = reinterpret_cast<int*>(p); p += a4;
    void* tmp = p; p += tmp_bytes;
    float4* qs = reinterpret_cast<float4*>(p); p += a16;
    float4* rec = reinterpret_cast<float4*>(p); p += 2 * a16;
    int* site_count = reinterpret_cast<int*>(p); p += site_bytes;
    int* site_first = reinterpret_cast<int*>(p);
    P2M_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), s));
    P2M_CUDA_TRY(cudaMemsetAsync(site_count, 0, sizeof(int) * K, s));
    const int threads = 256;
    const int blocks = query_grid_blocks(n, threads);
    if (counters)
        k_site_rank<true><<<blocks, threads, 0, s>>>(v, d_pts, n, key, rank, site_count, counters);
    else
        k_site_rank<false><<<blocks, threads, 0, s>>>(v, d_pts, n, key, rank, site_count, nullptr);
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, scan_tmp, site_count, site_first, K, s));
    k_site_scatter<<<blocks, threads, 0, s>>>(d_pts, n, key, rank, site_first, qs);
    P2M_CUDA_TRY(cudaGetLastError());
    // queries per thread: up to kStagePer, fewer when the call would not give every resident
    // block (5 per SM) a tile, and fewer when sites have few queries each, so that a tile
    // spans no more sites than the staging area holds lists of.  Measured on the icosphere(6)
    // at 61 / 122 / 244 queries per site: best with 1 / 2 / 4 queries per thread (0.62 /
    // 1.03 / 1.83 ms, against 0.72 / 1.07 / 1.83 with 4); the cylinder + cone, at 97, is best
    // with 4.
    const int64_t resident = (int64_t)sm_count() * 5;
    const int64_t q_site = n / std::max(S, 1);
    const int64_t by_site = q_site >= 90 ? kStagePer : (q_site >= 70 ? 2 : 1);
    const int per = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(kStagePer, n / (resident * kStageThreads)), by_site));
    const int sblocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + (int64_t)kStageThreads * per - 1) / ((int64_t)kStageThreads * per), resident * 4));
    timing_mark(h, 1, s);
    if (counters)
        k_query_staged<true><<<sblocks, kStageThreads, 0, s>>>(v, qs, site_first, n, per, d_rest, d_cnt, d_long, d_cnt + 1,
                                                               rec, counters);
    else
        k_query_staged<false><<<sblocks, kStageThreads, 0, s>>>(v, qs, site_first, n, per, d_rest, d_cnt, d_long, d_cnt + 1,
                                                                rec, nullptr);
    P2M_CUDA_TRY(cudaGetLastError());
    timing_mark(h, 2, s);
    const int wblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)sm_count() * 16));
    if (counters)
        k_query_warp<true><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                       d_rest, d_cnt, counters, d_cnt + 2, rec);
    else
        k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                        d_rest, d_cnt, nullptr, d_cnt + 2, rec);
    P2M_CUDA_TRY(cudaGetLastError());
    k_split_records<<<blocks, threads, 0, s>>>(rec, n, d_dist, d_closest, d_tri, d_bary);
    P2M_CUDA_TRY(cudaGetLastError());
    return launch_bvh_closest(v, d_pts, d_rest, d_cnt, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

static int run_query_impl(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
                          int32_t* d_tri, float* d_bary, unsigned long long* counters, DevBuf& rest, cudaStream_t s);

int run_query(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
              int32_t* d_tri, float* d_bary, unsigned long long* counters, DevBuf& rest, cudaStream_t s) {
    timing_mark(h, 0, s);
    timing_mark(h, 1, s);  // moved to the list scan by the schedules that have one
    timing_mark(h, 2, s);
    const int rc = run_query_impl(h, m, d_pts, n, d_dist, d_closest, d_tri, d_bary, counters, rest, s);
    timing_mark(h, 3, s);
    return rc;
}

static int run_query_impl(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
                          int32_t* d_tri, float* d_bary, unsigned long long* counters, DevBuf& rest, cudaStream_t s) {
    const MeshView v = m.view();
    if (v.G == 0) return launch_bvh_closest(v, d_pts, nullptr, nullptr, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
    // the site-staged schedule pays when sites have many queries each; a smaller call takes
    // the Morton-ordered thread-per-query path instead
    if (m.site_staged && n >= 4096 && n >= 48 * (int64_t)v.n_sites &&
        (int64_t)v.n_sites * kDqBuckets + 2 <= 0x7fffffffLL)
        return run_query_staged(h, m, d_pts, n, d_dist, d_closest, d_tri, d_bary, counters, rest, s);
    // scratch: rest ids [n], long queue [n] of int2, counters; for the sorted schedules also
    // the sort keys / permutation double buffers [4][n], per-query (query, site) pairs and long
    // flags, the temporary storage of the radix sorts and of the compaction, the points in
    // sorted order [n] float4 and the result records [n][2] float4
    const bool sorted = (m.sorted || m.site_staged) && n >= 4096 && n <= 0x7fffffff;
    const bool by_site = sorted && m.site_sorted;
    int site_bits = 1;
    while ((1u << site_bits) <= (unsigned)v.n_sites) ++site_bits;  // keys 0..n_sites
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t rest_bytes = up(sizeof(int32_t) * n), long_bytes = up(sizeof(int2) * n), cnt_bytes = 256;
    size_t sort_tmp = 0, sel_tmp = 0;
    if (sorted) {
        P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, sort_tmp, (unsigned*)nullptr, (unsigned*)nullptr,
                                                     (int32_t*)nullptr, (int32_t*)nullptr, (int)n, 0, 24, s));
        size_t site_tmp = 0;
        P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, site_tmp, (unsigned*)nullptr, (unsigned*)nullptr,
                                                     (int32_t*)nullptr, (int32_t*)nullptr, (int)n, 0, site_bits, s));
        sort_tmp = std::max(sort_tmp, site_tmp);
        P2M_CUDA_TRY(cub::DeviceSelect::Flagged(nullptr, sel_tmp, (int2*)nullptr, (unsigned char*)nullptr, (int2*)nullptr,
                                                (int*)nullptr, (int)n, s));
    }
    // counting sort over the Morton codes of the grid cells: mbits bits per axis, coarsened by
    // `shift` bits per axis so that the key space (its counters are cleared and scanned on
    // every call) stays within about 2n keys: small calls do not pay for a fine grid
    int mbits = 1;
    while ((1 << mbits) < v.G) ++mbits;
    int shift = 0;
    while (shift < mbits - 1 && ((int64_t)1 << (3 * (mbits - shift))) > std::max<int64_t>(2 * n, 4096)) ++shift;
    const int64_t n_keys = (int64_t)1 << (3 * (mbits - shift));  // key n_keys: outside the domain box
    size_t scan_tmp = 0;
    if (sorted)
        P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, scan_tmp, (int*)nullptr, (int*)nullptr, (int)(n_keys + 1), s));
    const size_t a4 = up(sizeof(int32_t) * n), tmp_bytes = up(std::max(std::max(sort_tmp, sel_tmp), scan_tmp));
    const size_t cell_bytes = up(sizeof(int) * (n_keys + 1));
    const size_t sort_bytes = sorted ? 4 * a4 + up(sizeof(int2) * n) + up(n) + tmp_bytes + up(sizeof(float4) * n) +
                                           up(2 * sizeof(float4) * n) + 2 * cell_bytes
                                     : 0;
    P2M_TRY(rest.ensure(rest_bytes + long_bytes + cnt_bytes + sort_bytes));
    char* base = rest.as<char>();
    int32_t* d_rest = reinterpret_cast<int32_t*>(base);
    int2* d_long = reinterpret_cast<int2*>(base + rest_bytes);
    int* d_cnt = reinterpret_cast<int*>(base + rest_bytes + long_bytes);  // [0] rest, [1] long, [2] head
    P2M_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, 4 * sizeof(int), s));
    const int threads = 256;
    const int blocks = query_grid_blocks(n, threads);
    const int wblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)sm_count() * 16));
    int* head = nullptr;
    float4* rec = nullptr;
    if (sorted) {
        char* sb = base + rest_bytes + long_bytes + cnt_bytes;
        unsigned* k0 = reinterpret_cast<unsigned*>(sb);
        unsigned* k1 = reinterpret_cast<unsigned*>(sb + a4);
        int32_t* i0 = reinterpret_cast<int32_t*>(sb + 2 * a4);
        int32_t* i1 = reinterpret_cast<int32_t*>(sb + 3 * a4);
        char* p = sb + 4 * a4;
        int2* cand = reinterpret_cast<int2*>(p);
        p += up(sizeof(int2) * n);
        unsigned char* flag = reinterpret_cast<unsigned char*>(p);
        p += up(n);
        void* tmp = p;
        p += tmp_bytes;
        float4* qs = reinterpret_cast<float4*>(p);
        p += up(sizeof(float4) * n);
        rec = reinterpret_cast<float4*>(p);
        p += up(2 * sizeof(float4) * n);
        int* cell_count = reinterpret_cast<int*>(p);
        int* cell_first = reinterpret_cast<int*>(p + cell_bytes);
        // queries in grid-cell Morton order, gathered into qs (counting sort)
        P2M_CUDA_TRY(cudaMemsetAsync(cell_count, 0, sizeof(int) * (n_keys + 1), s));
        k_cell_rank<<<blocks, threads, 0, s>>>(v, d_pts, n, (unsigned)n_keys, 3 * shift, k0, i0, cell_count);
        P2M_CUDA_TRY(cudaGetLastError());
        P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp, scan_tmp, cell_count, cell_first, (int)(n_keys + 1), s));
        k_cell_scatter<<<blocks, threads, 0, s>>>(d_pts, n, k0, i0, cell_first, qs);
        P2M_CUDA_TRY(cudaGetLastError());
        cub::DoubleBuffer<unsigned> dk(k0, k1);
        cub::DoubleBuffer<int32_t> dv(i0, i1);
        if (by_site) {
            // nearest sites in Morton order, then a stable sort by site (the Morton keys and the
            // permutation are dead once the points are gathered)
            unsigned* sk = dk.Alternate();
            int32_t* sv = dv.Alternate();
            if (counters)
                k_query_sites<true><<<blocks, threads, 0, s>>>(v, qs, n, sk, sv, counters);
            else
                k_query_sites<false><<<blocks, threads, 0, s>>>(v, qs, n, sk, sv, nullptr);
            P2M_CUDA_TRY(cudaGetLastError());
            cub::DoubleBuffer<unsigned> sk2(sk, dk.Current());
            cub::DoubleBuffer<int32_t> sv2(sv, dv.Current());
            P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, sort_tmp, sk2, sv2, (int)n, 0, site_bits, s));
            if (counters)
                k_query_scan<true><<<blocks, threads, 0, s>>>(v, qs, sk2.Current(), sv2.Current(), n, d_dist, d_closest,
                                                             d_tri, d_bary, d_rest, d_cnt, cand, flag, counters, rec);
            else
                k_query_scan<false><<<blocks, threads, 0, s>>>(v, qs, sk2.Current(), sv2.Current(), n, d_dist, d_closest,
                                                              d_tri, d_bary, d_rest, d_cnt, cand, flag, nullptr, rec);
        } else if (counters) {
            k_query_thread<true><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                            d_long, d_cnt + 1, counters, qs, cand, flag, rec);
        } else {
            timing_mark(h, 1, s);
            k_query_thread<false><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                             d_long, d_cnt + 1, nullptr, qs, cand, flag, rec);
            timing_mark(h, 2, s);
        }
        P2M_CUDA_TRY(cudaGetLastError());
        // order-preserving compaction of the long queries (count written on the device)
        P2M_CUDA_TRY(cub::DeviceSelect::Flagged(tmp, sel_tmp, cand, flag, d_long, d_cnt + 1, (int)n, s));
        head = d_cnt + 2;
    } else if (counters) {
        k_query_thread<true><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                        d_long, d_cnt + 1, counters, nullptr, nullptr, nullptr, nullptr);
    } else {
        k_query_thread<false><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt,
                                                         d_long, d_cnt + 1, nullptr, nullptr, nullptr, nullptr, nullptr);
    }
    P2M_CUDA_TRY(cudaGetLastError());
    if (counters)
        k_query_warp<true><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                       d_rest, d_cnt, counters, head, rec);
    else
        k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary,
                                                        d_rest, d_cnt, nullptr, head, rec);
    P2M_CUDA_TRY(cudaGetLastError());
    if (rec) {
        k_split_records<<<blocks, threads, 0, s>>>(rec, n, d_dist, d_closest, d_tri, d_bary);
        P2M_CUDA_TRY(cudaGetLastError());
    }
    // the points left over take the exact BVH search (after the split, which leaves their
    // outputs undefined); the count stays on the device
    return launch_bvh_closest(v, d_pts, d_rest, d_cnt, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

int launch_gather_points(const float* d_pts, const int32_t* d_perm, int64_t n, float4* d_qs, cudaStream_t s) {
    if (n <= 0) return P2M_OK;
    k_gather_points<<<query_grid_blocks(n, 256), 256, 0, s>>>(d_pts, d_perm, n, d_qs);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

int launch_split_records(const float4* d_rec, int64_t n, float* d_dist, float* d_closest, int32_t* d_tri,
                         float* d_bary, cudaStream_t s) {
    if (n <= 0) return P2M_OK;
    k_split_records<<<query_grid_blocks(n, 256), 256, 0, s>>>(d_rec, n, d_dist, d_closest, d_tri, d_bary);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
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
    const int wblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, (int64_t)sm_count() * 16));
    k_query_thread<false><<<blocks, threads, 0, s>>>(v, d_pts, n, d_dist, d_closest, d_tri, d_bary, d_rest, d_cnt, d_long,
                                                     d_cnt + 1, nullptr, nullptr, nullptr, nullptr, nullptr);
    k_query_warp<false><<<wblocks, threads, 0, s>>>(v, d_pts, d_long, d_cnt + 1, d_dist, d_closest, d_tri, d_bary, d_rest,
                                                    d_cnt, nullptr, nullptr, nullptr);
    P2M_CUDA_TRY(cudaGetLastError());
    return launch_bvh_closest(v, d_pts, d_rest, d_cnt, n, d_dist, d_closest, d_tri, d_bary, index_status(h), s);
}

}  // namespace p2m
