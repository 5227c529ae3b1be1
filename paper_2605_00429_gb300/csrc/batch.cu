// K6: batched queries over many meshes in one persistent launch (not in the paper).
//
// The queries of mesh i are pts[off[i] .. off[i+1]).  They are cut into tiles of `tile`
// queries; a persistent grid (SM count x resident blocks) pulls tiles from an atomic queue
// and answers each query exactly as the single-mesh path does (nearest site, list scan).
// Queries whose list is longer than `long_row` are queued for a persistent warp-per-query
// pass, and the few points outside their mesh's domain box take the BVH search.  Before
// that, every mesh's queries are radix-sorted by (mesh, Morton code of their grid cell) and
// gathered into sort order; results leave as 32-byte records split into the outputs.  The
// whole sequence (counter reset, sort, gather, thread and warp passes, split, BVH pass) is
// captured once in a CUDA graph and replayed.
// An autotuner picks (tile, long_row) by timing the candidates on the caller's own batch.
#include <algorithm>
#include <cstring>

#include <cub/device/device_radix_sort.cuh>

#include "bvh_dev.cuh"
#include "host.h"
#include "query_dev.cuh"

namespace p2m {

struct BatchArgs {
    const MeshView* views;
    const int4* tiles;  // (mesh, begin, end, 0)
    int n_tiles;
    int long_row;
    const float* pts;
    float* dist;
    float* closest;
    int32_t* tri;
    float* bary;
    int4* longq;        // (query, site, mesh, 0)
    int2* rest;         // (query, mesh)
    int* ctr;           // [0] tile head, [1] long count, [2] rest count, [3] long head
    const float4* qs;   // sorted order: the points with their index in .w (NULL: unsorted)
    float4* rec;        // sorted order: 32-byte result records, split after the warp pass
};

__global__ void __launch_bounds__(256, 6) k_batch_thread(BatchArgs a) {
    __shared__ int s_tile;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(a.ctr, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= a.n_tiles) break;
        const int4 tile = __ldg(a.tiles + t);
        const MeshView& m = a.views[tile.x];
        for (int64_t k = (int64_t)tile.y + threadIdx.x; k < tile.z; k += blockDim.x) {
            int64_t i = k;
            float3 q;
            if (a.qs) {
                const float4 p = __ldg(a.qs + k);
                i = __float_as_int(p.w);
                q = make_float3(p.x, p.y, p.z);
            } else {
                q = make_float3(a.pts[3 * i], a.pts[3 * i + 1], a.pts[3 * i + 2]);
            }
            int cell;
            int site = -1;
            if (m.G > 0 && grid_cell(m, q, cell)) site = nearest_site<false>(m, q, cell, nullptr);
            if (site >= 0 && __ldg(m.row_off + site + 1) - __ldg(m.row_off + site) > a.long_row) {
                a.longq[atomicAdd(a.ctr + 1, 1)] = make_int4((int)i, site, tile.x, 0);
                continue;
            }
            unsigned long long key = ~0ull;
            float s = 0.0f, tt = 0.0f;
            if (site >= 0) key = scan_list<false>(m, q, site, s, tt, nullptr);
            if (key == ~0ull) {
                a.rest[atomicAdd(a.ctr + 2, 1)] = make_int2((int)i, tile.x);
                continue;
            }
            if (a.rec) write_record(m, a.rec, i, key, s, tt);
            else write_result(m, i, key, s, tt, a.dist, a.closest, a.tri, a.bary);
        }
    }
}

__global__ void __launch_bounds__(256, 2) k_batch_warp(BatchArgs a) {
    const int lane = threadIdx.x & 31;
    const int nq = *(volatile int*)(a.ctr + 1);
    while (true) {
        int k = 0;
        if (lane == 0) k = atomicAdd(a.ctr + 3, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nq) break;
        const int4 e = a.longq[k];
        const MeshView& m = a.views[e.z];
        const int64_t i = e.x;
        const float3 q = make_float3(a.pts[3 * i], a.pts[3 * i + 1], a.pts[3 * i + 2]);
        unsigned bhi, blo;
        float bs, bt;
        const bool found = warp_scan_list<false>(m, q, e.y, bhi, blo, bs, bt, nullptr);
        if (lane == 0) {
            if (!found) a.rest[atomicAdd(a.ctr + 2, 1)] = make_int2((int)i, e.z);
            else if (a.rec) write_record(m, a.rec, i, ((unsigned long long)bhi << 32) | blo, bs, bt);
            else write_result(m, i, ((unsigned long long)bhi << 32) | blo, bs, bt, a.dist, a.closest, a.tri, a.bary);
        }
    }
}

__global__ void __launch_bounds__(128) k_batch_bvh(BatchArgs a, unsigned* status) {
    const int nr = *(volatile int*)(a.ctr + 2);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nr; k += gridDim.x * blockDim.x) {
        const int2 e = a.rest[k];
        const MeshView& m = a.views[e.y];
        const int64_t i = e.x;
        const float3 q = make_float3(a.pts[3 * i], a.pts[3 * i + 1], a.pts[3 * i + 2]);
        float s = 0.0f, t = 0.0f;
        const unsigned long long key = bvh_closest_key(q, m.bvh, m.bvh_root, m.tri, s, t, status);
        write_result(m, i, key, s, t, a.dist, a.closest, a.tri, a.bary);
    }
}

// Sort key of a query of a batch: (mesh << 24) | Morton code of its cell in that mesh's grid,
// so that sorting keeps every mesh's queries in its own offset range (the tiles stay valid)
// and makes neighbouring threads read the same lists.
__device__ __forceinline__ unsigned spread8b(unsigned v) {
    v &= 0xffu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_batch_keys(BatchArgs a, unsigned long long* __restrict__ key, int32_t* __restrict__ idx) {
    for (int t = blockIdx.x; t < a.n_tiles; t += gridDim.x) {
        const int4 tile = __ldg(a.tiles + t);
        const MeshView& m = a.views[tile.x];
        for (int64_t i = (int64_t)tile.y + threadIdx.x; i < tile.z; i += blockDim.x) {
            const float3 q = make_float3(a.pts[3 * i], a.pts[3 * i + 1], a.pts[3 * i + 2]);
            unsigned mc = 0xffffffu;
            if (m.G > 0) {
                const float fx = (q.x - m.lo.x) * m.inv_h.x, fy = (q.y - m.lo.y) * m.inv_h.y,
                            fz = (q.z - m.lo.z) * m.inv_h.z;
                if (fx >= 0.0f && fy >= 0.0f && fz >= 0.0f && fx < (float)m.G && fy < (float)m.G && fz < (float)m.G)
                    mc = (spread8b((unsigned)fx) << 2) | (spread8b((unsigned)fy) << 1) | spread8b((unsigned)fz);
            }
            key[i] = ((unsigned long long)tile.x << 24) | mc;
            idx[i] = (int32_t)i;
        }
    }
}

static int persistent_blocks(const void* kernel, int threads) {
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return std::max(1, per_sm) * sm_count();
}

// The launch sequence of one batched query (captured into the graph when requested).
static int launch_batch(BatchState& b, const BatchArgs& a0, unsigned* status, cudaStream_t s) {
    BatchArgs a = a0;
    P2M_CUDA_TRY(cudaMemsetAsync(a.ctr, 0, 4 * sizeof(int), s));
    if (b.sort_tmp_bytes) {
        // Morton sort of every mesh's queries inside its own range
        const int64_t N = b.offsets.back();
        unsigned long long* k0 = b.sort_keys.as<unsigned long long>();
        int32_t* i0 = b.sort_idx.as<int32_t>();
        k_batch_keys<<<std::max(1, std::min(a.n_tiles, sm_count() * 32)), 256, 0, s>>>(a, k0, i0);
        P2M_CUDA_TRY(cudaGetLastError());
        cub::DoubleBuffer<unsigned long long> dk(k0, k0 + N);
        cub::DoubleBuffer<int32_t> dv(i0, i0 + N);
        size_t tb = b.sort_tmp_bytes;
        P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(b.sort_tmp.p, tb, dk, dv, (int)N, 0, b.sort_end_bit, s));
        // the points in sorted order; results go out as whole-sector records, split below
        P2M_TRY(launch_gather_points(a.pts, dv.Current(), N, b.qs.as<float4>(), s));
        a.qs = b.qs.as<const float4>();
        a.rec = b.rec.as<float4>();
    }
    k_batch_thread<<<b.grid_thread, 256, 0, s>>>(a);
    k_batch_warp<<<b.grid_warp, 256, 0, s>>>(a);
    P2M_CUDA_TRY(cudaGetLastError());
    // queries left to the BVH search have no record: the split leaves their outputs undefined
    // and the BVH pass writes them afterwards
    if (a.rec) P2M_TRY(launch_split_records(a.rec, b.offsets.back(), a.dist, a.closest, a.tri, a.bary, s));
    k_batch_bvh<<<b.grid_bvh, 128, 0, s>>>(a, status);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

static int make_tiles(BatchState& b, const std::vector<int64_t>& off, int tile) {
    std::vector<int4> tiles;
    const int n = (int)off.size() - 1;
    for (int i = 0; i < n; ++i)
        for (int64_t q = off[i]; q < off[i + 1]; q += tile)
            tiles.push_back(make_int4(i, (int)q, (int)std::min<int64_t>(q + tile, off[i + 1]), 0));
    b.n_tiles = (int)tiles.size();
    P2M_TRY(b.tiles.ensure(sizeof(int4) * std::max<size_t>(tiles.size(), 1)));
    if (!tiles.empty())
        P2M_CUDA_TRY(cudaMemcpy(b.tiles.p, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice));
    b.tile = tile;
    return P2M_OK;
}

int run_batch_query(p2m_index* h, const float* d_pts, const int64_t* h_off, float* d_dist, float* d_closest,
                    int32_t* d_tri, float* d_bary, int mode, int use_graph, cudaStream_t s) {
    const int nm = (int)h->meshes.size();
    std::vector<int64_t> off(h_off, h_off + nm + 1);
    if (off[0] != 0) return fail(P2M_ERR_INVALID_ARG, "offsets must start at 0");
    for (int i = 0; i < nm; ++i)
        if (off[i + 1] < off[i]) return fail(P2M_ERR_INVALID_ARG, "offsets must be non-decreasing");
    const int64_t N = off[nm];
    if (N == 0) return P2M_OK;
    if (N > 0x7fffffffLL) return fail(P2M_ERR_INVALID_ARG, "batch larger than 2^31 queries");
    if (!d_pts || !d_dist) return fail(P2M_ERR_INVALID_ARG, "d_pts and d_dist must be non-NULL");
    if (mode == 1) {
        // plain per-mesh forward: one query call per mesh
        for (int i = 0; i < nm; ++i) {
            const int64_t b0 = off[i], n = off[i + 1] - off[i];
            if (n == 0) continue;
            P2M_TRY(run_query(h, *h->meshes[i], d_pts + 3 * b0, n, d_dist + b0, d_closest ? d_closest + 3 * b0 : nullptr,
                              d_tri ? d_tri + b0 : nullptr, d_bary ? d_bary + 3 * b0 : nullptr, nullptr, h->scratch_idx, s));
        }
        return P2M_OK;
    }
    if (mode != 0) return fail(P2M_ERR_INVALID_ARG, "mode must be 0 or 1");
    BatchState& b = h->batch;
    if (!b.views.p) {
        std::vector<MeshView> v(nm);
        for (int i = 0; i < nm; ++i) v[i] = h->meshes[i]->view();
        P2M_TRY(b.views.alloc(sizeof(MeshView) * nm));
        P2M_CUDA_TRY(cudaMemcpy(b.views.p, v.data(), sizeof(MeshView) * nm, cudaMemcpyHostToDevice));
        P2M_TRY(b.counter.alloc(sizeof(int) * 4));
        b.grid_thread = persistent_blocks((const void*)k_batch_thread, 256);
        b.grid_warp = persistent_blocks((const void*)k_batch_warp, 256);
        b.grid_bvh = persistent_blocks((const void*)k_batch_bvh, 128);
    }
    const bool new_offsets = off != b.offsets;
    if (new_offsets) {
        P2M_TRY(b.longq.ensure(sizeof(int4) * N));
        P2M_TRY(b.rest.ensure(sizeof(int2) * N));
        b.offsets = off;
        b.tuned = false;
        // scratch of the per-mesh Morton sort (double buffers + radix-sort temporaries)
        int mesh_bits = 1;
        while ((1 << mesh_bits) < nm) ++mesh_bits;
        b.sort_end_bit = 24 + mesh_bits;
        P2M_TRY(b.sort_keys.ensure(sizeof(unsigned long long) * 2 * N));
        P2M_TRY(b.sort_idx.ensure(sizeof(int32_t) * 2 * N));
        size_t tb = 0;
        P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                                     (int32_t*)nullptr, (int32_t*)nullptr, (int)N, 0, b.sort_end_bit, s));
        P2M_TRY(b.sort_tmp.ensure(tb + 16));
        b.sort_tmp_bytes = tb;
        P2M_TRY(b.qs.ensure(sizeof(float4) * N));
        P2M_TRY(b.rec.ensure(2 * sizeof(float4) * N));
    }
    BatchArgs a;
    a.views = b.views.as<const MeshView>();
    a.pts = d_pts;
    a.dist = d_dist;
    a.closest = d_closest;
    a.tri = d_tri;
    a.bary = d_bary;
    a.longq = b.longq.as<int4>();
    a.rest = b.rest.as<int2>();
    a.ctr = b.counter.as<int>();
    a.qs = nullptr;
    a.rec = nullptr;
    unsigned* status = index_status(h);
    if (!b.tuned) {
        // autotuner: time each (tile, long_row) candidate on this batch, keep the fastest.
        // long_row starts at the lists' own threshold: the warp pass reads the list-order
        // bounding spheres, which the build stores only for the lists longer than that
        const int tiles[] = {1024, 4096};
        const int64_t lr0 = h->meshes[0]->long_row;
        const int longs[] = {(int)lr0, (int)std::min<int64_t>(4 * lr0, 0x7fffffff),
                             (int)std::min<int64_t>(16 * lr0, 0x7fffffff)};
        Event e0, e1;
        P2M_CUDA_TRY(cudaEventCreate(&e0.e));
        P2M_CUDA_TRY(cudaEventCreate(&e1.e));
        float best = 1e30f;
        int bt = tiles[0], bl = longs[0];
        for (int tile : tiles) {
            P2M_TRY(make_tiles(b, off, tile));
            a.tiles = b.tiles.as<const int4>();
            a.n_tiles = b.n_tiles;
            for (int lr : longs) {
                a.long_row = lr;
                P2M_TRY(launch_batch(b, a, status, s));  // warm
                P2M_CUDA_TRY(cudaEventRecord(e0.e, s));
                for (int r = 0; r < 2; ++r) P2M_TRY(launch_batch(b, a, status, s));
                P2M_CUDA_TRY(cudaEventRecord(e1.e, s));
                P2M_CUDA_TRY(cudaEventSynchronize(e1.e));
                float ms = 0;
                P2M_CUDA_TRY(cudaEventElapsedTime(&ms, e0.e, e1.e));
                if (ms < best) { best = ms; bt = tile; bl = lr; }
            }
        }
        P2M_TRY(make_tiles(b, off, bt));
        b.long_row = bl;
        b.tuned = true;
        b.tune_ms = best / 2;
        if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
    }
    a.tiles = b.tiles.as<const int4>();
    a.n_tiles = b.n_tiles;
    a.long_row = b.long_row;
    if (!use_graph) return launch_batch(b, a, status, s);
    const void* outs[4] = {d_dist, d_closest, d_tri, d_bary};
    const bool same = b.exec && b.graph_pts == d_pts && std::memcmp(outs, b.graph_out, sizeof(outs)) == 0;
    if (!same) {
        if (b.exec) { cudaGraphExecDestroy(b.exec); b.exec = nullptr; }
        // capture on a private stream (the caller's may be the legacy stream, which cannot be
        // captured); the instantiated graph is then launched on the caller's stream
        if (!b.cap) P2M_CUDA_TRY(cudaStreamCreateWithFlags(&b.cap, cudaStreamNonBlocking));
        cudaGraph_t g;
        P2M_CUDA_TRY(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
        const int rc = launch_batch(b, a, status, b.cap);
        const cudaError_t ec = cudaStreamEndCapture(b.cap, &g);
        if (rc != P2M_OK) return rc;
        P2M_CUDA_TRY(ec);
        const cudaError_t ei = cudaGraphInstantiate(&b.exec, g, 0);
        cudaGraphDestroy(g);
        P2M_CUDA_TRY(ei);
        b.graph_pts = d_pts;
        std::memcpy(b.graph_out, outs, sizeof(outs));
    }
    P2M_CUDA_TRY(cudaGraphLaunch(b.exec, s));
    return P2M_OK;
}

}  // namespace p2m
