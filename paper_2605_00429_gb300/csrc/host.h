// Declarations that cross translation units between the C ABI and the build / query code.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <vector>

#include "p2m_internal.h"

struct p2m_index;

namespace p2m {

// State of the batched persistent query (tile queue, autotuned choice, captured graph).
struct BatchState {
    DevBuf views;        // MeshView per mesh (device copy)
    DevBuf tiles;        // int4 work list: (mesh, q_begin, q_end, 0)
    DevBuf counter;      // tile head, long count, rest count, long head
    DevBuf longq, rest;  // queues of the warp pass and of the BVH pass
    DevBuf sort_keys, sort_idx, sort_tmp;  // per-mesh Morton sort of the queries
    DevBuf qs, rec;      // points in sorted order, 32-byte result records
    size_t sort_tmp_bytes = 0;
    int sort_end_bit = 24;
    int n_tiles = 0;
    int tile = 0;        // queries per tile picked by the autotuner
    int long_row = 256;  // lists longer than this take the warp-per-query pass
    bool tuned = false;
    float tune_ms = 0.f;
    int grid_thread = 0, grid_warp = 0, grid_bvh = 0;
    std::vector<int64_t> offsets;  // host offsets the work list was built for
    const void* graph_pts = nullptr;
    const void* graph_out[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;  // private stream the graph is captured on
    ~BatchState() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
    }
};

}  // namespace p2m

// The index object behind the opaque C handle.
struct p2m_index {
    p2m_build_params params{};
    std::vector<std::unique_ptr<p2m::MeshData>> meshes;
    p2m::DevBuf status;        // device status word (ST_* bits)
    p2m::DevBuf scratch_idx;   // compacted list of queries left to the BVH search
    p2m::BatchState batch;     // batched-query state (tile queue, graph)
    int device = 0;
    // host-buffer query pipeline: a copy-in stream, a compute stream and a copy-out stream;
    // kPipe buffer slots, each with its own device buffers and events (copied in, computed,
    // copied out)
    static constexpr int kPipe = 3;
    cudaStream_t streams[kPipe] = {nullptr, nullptr, nullptr};
    p2m::DevBuf pipe[kPipe][5];    // pts, dist, closest, tri, bary
    p2m::DevBuf pipe_rest[kPipe];
    cudaEvent_t pipe_ev[kPipe][3] = {};
    p2m::DevBuf grad_acc;      // fixed-point vertex-gradient accumulator
    // kernel timing (p2m_set_timing): events at the call's start, around its list-scan
    // kernel, and at its end
    bool timing = false;
    bool timed_call = false;
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
    p2m::DevBuf sign_scratch;  // triangle ids / barycentrics for the signed query
    ~p2m_index();
};

namespace p2m {

unsigned* index_status(p2m_index* h);
DevBuf& index_rest(p2m_index* h);  // scratch for the compacted out-of-domain query list
int check_status_word(p2m_index* h, cudaStream_t s, const char* what);
// Checks shared by the entry points that launch work on an index: the device the index was
// built on must be current (its buffers live there), and a call takes at most 2^31 - 1
// points (query positions are int32 inside the kernels).
int check_call(const p2m_index* h, int64_t n, const char* what);
// With timing on, records event k (0 start, 1 before the list scan, 2 after it, 3 end) on s.
void timing_mark(p2m_index* h, int k, cudaStream_t s);

// Sites, Delaunay, augmentation, corner balls, interception lists, nearest-site grid.
int build_partition(MeshData& m, const p2m_build_params& prm, p2m_index* h, cudaStream_t s);
// Angle-weighted pseudonormals of the signed query (host FP64, uploaded to m.d_snorm/d_vnorm).
int build_pseudonormals(MeshData& m);

// Full query of one mesh; counters (8 x u64, may be NULL) accumulate instrumentation.
int run_query(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
              int32_t* d_tri, float* d_bary, unsigned long long* counters, DevBuf& rest, cudaStream_t s);
int run_nearest_site(p2m_index* h, MeshData& m, const float* d_pts, int64_t n, int32_t* d_site, cudaStream_t s);
int run_batch_query(p2m_index* h, const float* d_pts, const int64_t* h_off, float* d_dist, float* d_closest,
                    int32_t* d_tri, float* d_bary, int mode, int use_graph, cudaStream_t s);

}  // namespace p2m
