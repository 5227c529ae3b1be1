// Internal declarations shared by the translation units of libp2mpp.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/p2mpp.h"

namespace p2m {

// ----------------------------------------------------------------------------- errors

void set_error(const std::string& msg);
bool inject_fault(const char* what);  // P2M_FAULT == what (host-side test fault injection)
int fail(int code, const std::string& msg);
// Streaming multiprocessors of the current device (cached per device); launch grids are
// sized in multiples of it.
int sm_count();

#define P2M_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            return ::p2m::fail(P2M_ERR_CUDA, std::string(#expr) + ": " +               \
                                                 cudaGetErrorString(_e));               \
    } while (0)

#define P2M_TRY(expr)                  \
    do {                               \
        int _rc = (expr);              \
        if (_rc != P2M_OK) return _rc; \
    } while (0)

// Device status word bits (written by kernels, read by the host after a sync).
enum : unsigned {
    ST_STACK = 1u,   // a BVH traversal stack overflowed
    ST_LIMIT = 2u,   // an iteration / capacity cap was reached
    ST_BAD = 4u,     // an index check failed
};

// ----------------------------------------------------------------------------- device buffers

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void release() { if (p) cudaFree(p); p = nullptr; bytes = 0; }
    int alloc(size_t nbytes);          // (re)allocate, contents undefined
    int ensure(size_t nbytes);         // grow if smaller
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Owns a CUDA event: destroyed when it goes out of scope, early error returns included.
struct Event {
    cudaEvent_t e = nullptr;
    Event() = default;
    Event(const Event&) = delete;
    Event& operator=(const Event&) = delete;
    ~Event() { if (e) cudaEventDestroy(e); }
};

// ----------------------------------------------------------------------------- BVH

// Binary BVH node holding the boxes of both children (one 64-byte load tests both).
// lo0.w / lo1.w carry the child references as int bits: >= 0 internal node, < 0 leaf ~prim.
struct BNode {
    float4 lo0, hi0, lo1, hi1;
};

struct Bvh {
    DevBuf nodes;      // BNode[n-1]
    int n_prims = 0;
    int root = 0;      // node index, or ~prim when n_prims == 1
};

// ----------------------------------------------------------------------------- one mesh

// Everything the query path of one mesh reads, as raw device pointers (for kernels).
struct MeshView {
    const float4* tri;      // [T][4] triangle records (see geom.cuh), in BVH leaf order
    const int32_t* orig;    // [T] original triangle id of each leaf-order position
    const float4* tsph;     // [T] bounding spheres (c.xyz, r)
    const BNode* bvh;       // triangle BVH
    int bvh_root;
    const float4* sites;    // [S] (x, y, z, 0)
    const float4* refs;     // [S] reference point on the mesh (x, y, z, rounding radius)
    const int32_t* row_off; // [S+1]
    // [nnz] (triangle, key bits), key = ||ref - c_f|| - r_f; lists of <= long_row entries
    // are sorted by key
    const int2* row_ent;
    const float4* row_sph;  // [nnz] the entries' bounding spheres in list order (long lists only), or NULL
    const int32_t* chunk_off;  // [S+1] first 32-entry chunk of each list
    const float4* cbox;     // [n_chunks][3] chunk bounds: (lo, hmin), (hi, hmax), (unit normal, 0)
    const int32_t* l1_off;  // [S+1] first level-1 box (32 chunks = 1024 entries) of each list
    const float4* l1box;    // [n_l1][2]
    const int32_t* cell_off;// [G^3+1] nearest-site grid CSR
    const int32_t* cell_id; // candidate site ids (positions from `sites`)
    int G;                  // grid cells per axis (0 => no grid: every query takes the BVH path)
    float3 lo;              // domain D lower corner
    float3 inv_h;           // 1 / grid cell size
    float3 hi;              // domain D upper corner
    float prune_abs;        // absolute prune slack
    float spacing;          // mean spacing of the vertex sites (sqrt(area / sites))
    int n_tris;
    int n_sites;
    int long_row;           // lists longer than this go to the warp-per-query scan
};

struct MeshData {
    // host copies
    std::vector<float> verts;    // [V*3]
    std::vector<int32_t> tris;   // [T*3]
    int64_t n_verts = 0, n_tris = 0;
    double bb_lo[3], bb_hi[3], diag = 0;
    double dom_lo[3], dom_hi[3];
    // sites (host)
    std::vector<float> site_pos;      // [S*3] float positions used by the queries
    std::vector<double> site_ref;     // [S*3] reference point on the mesh
    std::vector<int32_t> site_kind;   // 0 vertex site, 1 aux site
    std::vector<int64_t> ball_off;    // [S+1]
    std::vector<double> ball_c;       // [B*3]
    std::vector<double> ball_r;       // [B]
    // device
    DevBuf d_verts, d_tris, d_tri, d_tsph, d_tlo, d_thi, d_orig;
    DevBuf d_snorm, d_vnorm;     // pseudonormals for the sign: [T][4] (face, edges 01/12/20), [V]
    std::vector<int32_t> orig;   // host copy of d_orig
    Bvh bvh;
    DevBuf d_sites, d_refs, d_row_off, d_row_tri, d_row_key, d_row_ent, d_row_sph, d_cell_off, d_cell_id, d_chunk_off, d_cbox, d_l1_off, d_l1box;
    int64_t nnz = 0, n_chunks = 0;
    int long_row = 256;
    bool sorted = true;          // process queries in grid-cell Morton order
    bool site_sorted = false;    // then regroup them by nearest site before the list scan
    bool site_staged = false;    // queries counting-sorted by nearest site, lists staged in shared memory
    int G = 0;
    float spacing = 0.0f;
    float3 g_lo{}, g_hi{}, g_inv_h{};
    p2m_stats stats{};
    MeshView view() const;
};

// ----------------------------------------------------------------------------- kernels (launchers)

// K0b: triangle records + bounding spheres.
int launch_tri_precompute(const float* d_verts, const int32_t* d_tris, int n_tris, float4* d_tri,
                          float4* d_tsph, cudaStream_t s);
// K0: LBVH over primitive boxes (lo[i], hi[i]); scene centroid bounds given.
// With order_out, primitives are renumbered in leaf (Morton) order: leaves reference sorted
// positions and order_out[k] receives the original id of position k.
int build_lbvh(const float4* d_lo, const float4* d_hi, int n, float3 c_lo, float3 c_hi, Bvh& out,
               cudaStream_t s, DevBuf* order_out = nullptr);
int gather_f4(DevBuf& buf, const int* d_order, int n, int per, cudaStream_t s);  // buf[k] = buf[order[k]]
int tri_boxes(const float* d_verts, const int32_t* d_tris, int n_tris, float4* lo, float4* hi,
              cudaStream_t s);
// K5: exact closest triangle by BVH branch and bound.  Queries are d_pts[d_idx[k]] for
// k < *d_count (both on the device) when d_idx is given, else d_pts[k] for k < n.  n bounds
// the launch either way.
// Sorted-order helpers of the query path: qs[k] = (pts[perm[k]], perm[k] bits); and the
// 32-byte result records rec[2i..2i+1] split into the output arrays (closest, tri, bary may be
// NULL).
int launch_gather_points(const float* d_pts, const int32_t* d_perm, int64_t n, float4* d_qs, cudaStream_t s);
int launch_split_records(const float4* d_rec, int64_t n, float* d_dist, float* d_closest, int32_t* d_tri,
                         float* d_bary, cudaStream_t s);
int launch_bvh_closest(const MeshView& m, const float* d_pts, const int32_t* d_idx, const int* d_count,
                       int64_t n, float* d_dist, float* d_closest, int32_t* d_tri, float* d_bary,
                       unsigned* d_status, cudaStream_t s);

}  // namespace p2m
