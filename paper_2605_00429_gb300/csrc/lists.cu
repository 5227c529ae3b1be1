// K1: interception lists by corner-sphere vs BVH collision (Section 3.3 "Implementation
// Details").  The list of site v holds every triangle f that meets the union of its balls:
//   vertex site:  balls B(u, ||u - v||) over the corners u of its clipped cell (Eq. 3);
//   aux site:     one ball B(s, r) with r from Eq. 8.
// Ball centres and radii arrive in FP32 with the radius already inflated on the host by the
// build slack plus the FP32 rounding of the centre, so a triangle whose FP64 distance to a
// ball is <= r joins the list (the test is solid ball vs solid triangle).
//
// One warp per (site, subtree) work item; lanes split the site's balls.  The warp walks the
// subtree in lockstep (the traversal stack is warp-uniform); a node is entered if any lane's
// ball overlaps the node box, a triangle is kept if any lane's ball reaches it.  Two passes
// share the code: count, then (after a scan) fill.  Both passes visit triangles in the same
// order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include "geom.cuh"
#include "host.h"

namespace p2m {

constexpr int kListWarps = 4;     // warps per block
constexpr int kChunk = 32;        // list entries per chunk box
constexpr int kListStack = 64;
constexpr int kStash = 512;       // entries of one item a warp keeps in shared memory (first pass)

__device__ __forceinline__ bool any_ball_box(const float4* __restrict__ balls, int nb, float3 lo, float3 hi) {
    bool hit = false;
    for (int k = threadIdx.x & 31; k < nb && !hit; k += 32) {
        const float4 b = __ldg(balls + k);
        hit = box_dist2(f3(b), lo, hi) <= b.w * b.w;
    }
    return __any_sync(0xffffffffu, hit);
}

__device__ __forceinline__ bool any_ball_tri(const float4* __restrict__ balls, int nb, const TriRec& T) {
    bool hit = false;
    for (int k = threadIdx.x & 31; k < nb && !hit; k += 32) {
        const float4 b = __ldg(balls + k);
        float s, t;
        hit = tri_dist2(f3(b), T, s, t) <= b.w * b.w;
    }
    return __any_sync(0xffffffffu, hit);
}

// Work items: (site, subtree).  The BVH is cut at a fixed depth into subtrees, listed left to
// right as (parent node, child 0 or 1); a site's list is the concatenation of its items in that
// order, so one warp never walks the whole tree for a site whose balls cover most of the mesh
// (the cells reaching the corners of D), and such a site's work spreads over its items' warps.
// FILL = false: count every item's triangles (count[it]) and, where they fit, keep them: an
// item of at most kStash triangles is gathered in shared memory and copied to a slot of
// `stash` reserved with one atomic (item_pos[it] = the slot, or -1 for an item that did not
// fit), so that the second pass walks the tree again only for the items it must.
// FILL = true: write every item not kept in the first pass (item_pos[it] < 0) at
// row_tri[item_off[it] ..].
template <bool FILL>
__global__ void __launch_bounds__(32 * kListWarps) k_lists(const float4* __restrict__ balls, const int64_t* __restrict__ ball_off,
                                                            int n_sites, const BNode* __restrict__ nodes, int root,
                                                            const int2* __restrict__ subroots, int n_sub,
                                                            const float4* __restrict__ tri, int64_t* __restrict__ count,
                                                            const int64_t* __restrict__ item_off, int32_t* __restrict__ row_tri,
                                                            int32_t* __restrict__ stash, int64_t stash_cap,
                                                            unsigned long long* __restrict__ stash_top,
                                                            int64_t* __restrict__ item_pos, unsigned* status) {
    __shared__ int stk[kListWarps][kListStack];
    __shared__ int sbuf[FILL ? 1 : kListWarps][FILL ? 1 : kStash];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = gridDim.x * kListWarps;
    const int64_t n_items = (int64_t)n_sites * n_sub;
    for (int64_t it = (int64_t)blockIdx.x * kListWarps + w; it < n_items; it += nwarps) {
        if (FILL && item_pos[it] >= 0) continue;  // kept by the first pass (uniform over the warp)
        const int s = (int)(it / n_sub), r = (int)(it % n_sub);
        const int64_t b0 = ball_off[s];
        const int nb = (int)(ball_off[s + 1] - b0);
        const float4* sb = balls + b0;
        int64_t k = 0;
        const int64_t out = FILL ? item_off[it] : 0;
        auto emit = [&](int f) {
            if (lane == 0) {
                if (FILL) row_tri[out + k] = f;
                else if (k < kStash) sbuf[FILL ? 0 : w][k] = f;
            }
            ++k;
        };
        if (nb > 0) {
            if (root < 0) {
                const TriRec T = load_tri(tri, ~root);
                if (any_ball_tri(sb, nb, T)) emit(~root);
            } else {
                // the item's subtree: child `which` of node `parent`, tested by its box first
                const int2 sr = __ldg(subroots + r);
                const float4* pp = reinterpret_cast<const float4*>(nodes + sr.x) + 2 * sr.y;
                const float4 rlo = __ldg(pp), rhi = __ldg(pp + 1);
                const int rc = __float_as_int(rlo.w);
                int node = -1;
                if (any_ball_box(sb, nb, f3(rlo), f3(rhi))) {
                    if (rc < 0) {
                        const TriRec T = load_tri(tri, ~rc);
                        if (any_ball_tri(sb, nb, T)) emit(~rc);
                    } else {
                        node = rc;
                    }
                }
                int sp = 0;
                while (node >= 0) {
                    const float4* np = reinterpret_cast<const float4*>(nodes + node);
                    const float4 lo0 = __ldg(np), hi0 = __ldg(np + 1), lo1 = __ldg(np + 2), hi1 = __ldg(np + 3);
                    const int c0 = __float_as_int(lo0.w), c1 = __float_as_int(lo1.w);
                    const bool h0 = any_ball_box(sb, nb, f3(lo0), f3(hi0));
                    const bool h1 = any_ball_box(sb, nb, f3(lo1), f3(hi1));
                    int next = -1;
                    if (h0) {
                        if (c0 < 0) {
                            const TriRec T = load_tri(tri, ~c0);
                            if (any_ball_tri(sb, nb, T)) emit(~c0);
                        } else {
                            next = c0;
                        }
                    }
                    if (h1) {
                        if (c1 < 0) {
                            const TriRec T = load_tri(tri, ~c1);
                            if (any_ball_tri(sb, nb, T)) emit(~c1);
                        } else if (next < 0) {
                            next = c1;
                        } else {
                            if (sp < kListStack) {
                                if (lane == 0) stk[w][sp] = c1;
                                ++sp;
                            } else if (lane == 0) {
                                atomicOr(status, ST_STACK);
                            }
                        }
                    }
                    __syncwarp();
                    if (next < 0) {
                        if (sp > 0) {
                            --sp;
                            next = stk[w][sp];
                        }
                    }
                    __syncwarp();
                    node = next;
                }
            }
        }
        if (!FILL) {
            long long pos = -1;
            if (k <= kStash) {
                if (lane == 0) {
                    pos = 0;
                    if (k > 0) {
                        pos = (long long)atomicAdd(stash_top, (unsigned long long)k);
                        if (pos + k > stash_cap) pos = -1;  // the stash is full: the second pass writes it
                    }
                }
                pos = __shfl_sync(0xffffffffu, pos, 0);
                __syncwarp();
                if (pos >= 0)
                    for (int j = lane; j < (int)k; j += 32) stash[pos + j] = sbuf[FILL ? 0 : w][j];
                __syncwarp();
            }
            if (lane == 0) {
                count[it] = k;
                item_pos[it] = pos;
            }
        }
        if (FILL && lane == 0 && k != item_off[it + 1] - item_off[it]) atomicOr(status, ST_BAD);
    }
}

// The items kept by the first pass, from the stash to their places in the lists (a warp per
// item).
__global__ void k_copy_stash(const int32_t* __restrict__ stash, const int64_t* __restrict__ item_pos,
                             const int64_t* __restrict__ item_off, int64_t n_items, int32_t* __restrict__ row_tri) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t it = warp; it < n_items; it += nwarps) {
        const int64_t pos = item_pos[it];
        if (pos < 0) continue;
        const int64_t o = item_off[it], k = item_off[it + 1] - o;
        for (int64_t j = lane; j < k; j += 32) row_tri[o + j] = stash[pos + j];
    }
}

// Site offsets from the item offsets: off64[s] = item_off[s * n_sub].
__global__ void k_site_offsets(const int64_t* __restrict__ item_off, int n_sites, int n_sub, int64_t* __restrict__ off64) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= n_sites; s += gridDim.x * blockDim.x)
        off64[s] = item_off[(int64_t)s * n_sub];
}

// Chunks of 32 consecutive list entries, each with the bounding box of its triangles
// (grown by 2^-20 of the coordinate scale so that FP32 box distances stay lower bounds).
// K1 emits each list in BVH order, so a chunk covers a compact patch of the mesh.
__global__ void k_chunk_count(const int64_t* __restrict__ row_off64, int n_sites, int32_t* __restrict__ nch) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sites; s += gridDim.x * blockDim.x)
        nch[s] = (int32_t)((row_off64[s + 1] - row_off64[s] + kChunk - 1) / kChunk);
}

__global__ void k_chunk_boxes(const int64_t* __restrict__ row_off64, const int32_t* __restrict__ chunk_off, int n_sites,
                              const int32_t* __restrict__ row_tri, const float4* __restrict__ tlo,
                              const float4* __restrict__ thi, const float4* __restrict__ tri, float pad,
                              float4* __restrict__ cbox) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int s = warp; s < n_sites; s += nwarps) {
        const int64_t r0 = row_off64[s], r1 = row_off64[s + 1];
        const int c0 = chunk_off[s], nc = chunk_off[s + 1] - c0;
        for (int k = 0; k < nc; ++k) {
            const int64_t j = r0 + (int64_t)k * kChunk + lane;
            float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
            float3 nsum = make_float3(0.f, 0.f, 0.f);
            int f = -1;
            if (j < r1) {
                f = row_tri[j];
                lo = f3(tlo[f]);
                hi = f3(thi[f]);
                nsum = f3(tri[4 * (int64_t)f]);  // unit normal
            }
            for (int o = 16; o > 0; o >>= 1) {
                lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
                lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
                lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
                hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
                hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
                hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
                nsum.x += __shfl_xor_sync(0xffffffffu, nsum.x, o);
                nsum.y += __shfl_xor_sync(0xffffffffu, nsum.y, o);
                nsum.z += __shfl_xor_sync(0xffffffffu, nsum.z, o);
            }
            // slab of the chunk along its mean normal: extent of n.v over its vertices
            const float nl = sqrtf(dot3(nsum, nsum));
            const float3 n = nl > 0.0f ? (1.0f / nl) * nsum : make_float3(0.f, 0.f, 0.f);
            float hmin = INFINITY, hmax = -INFINITY;
            if (f >= 0) {
                const float4* r = tri + 4 * (int64_t)f;
                const float3 v0 = f3(r[1]), e0 = f3(r[2]), e1 = f3(r[3]);
                const float a = dot3(n, v0), b = dot3(n, e0), c = dot3(n, e1);
                hmin = fminf(a, fminf(a + b, a + c));
                hmax = fmaxf(a, fmaxf(a + b, a + c));
            }
            for (int o = 16; o > 0; o >>= 1) {
                hmin = fminf(hmin, __shfl_xor_sync(0xffffffffu, hmin, o));
                hmax = fmaxf(hmax, __shfl_xor_sync(0xffffffffu, hmax, o));
            }
            if (lane == 0) {
                // a zero normal leaves the slab unbounded (then only the box prunes)
                const bool ok = nl > 0.0f;
                cbox[3 * (int64_t)(c0 + k)] = make_float4(lo.x - pad, lo.y - pad, lo.z - pad, ok ? hmin - 2.0f * pad : -INFINITY);
                cbox[3 * (int64_t)(c0 + k) + 1] = make_float4(hi.x + pad, hi.y + pad, hi.z + pad, ok ? hmax + 2.0f * pad : INFINITY);
                cbox[3 * (int64_t)(c0 + k) + 2] = make_float4(n.x, n.y, n.z, 0.0f);
            }
        }
    }
}

// Level-1 boxes: the union of each run of 32 consecutive chunk boxes of a list.
__global__ void k_count_parents(const int32_t* __restrict__ child_off, int n_sites, int32_t* __restrict__ npar) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sites; s += gridDim.x * blockDim.x)
        npar[s] = (child_off[s + 1] - child_off[s] + 31) / 32;
}

__global__ void k_parent_boxes(const int32_t* __restrict__ child_off, const int32_t* __restrict__ par_off, int n_sites,
                               const float4* __restrict__ cbox, float4* __restrict__ pbox) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int s = warp; s < n_sites; s += nwarps) {
        const int c0 = child_off[s], nc = child_off[s + 1] - c0, p0 = par_off[s];
        for (int k = 0; 32 * k < nc; ++k) {
            const int c = 32 * k + lane;
            float3 lo = make_float3(INFINITY, INFINITY, INFINITY), hi = make_float3(-INFINITY, -INFINITY, -INFINITY);
            if (c < nc) {
                lo = f3(cbox[3 * (int64_t)(c0 + c)]);
                hi = f3(cbox[3 * (int64_t)(c0 + c) + 1]);
            }
            for (int o = 16; o > 0; o >>= 1) {
                lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
                lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
                lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
                hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
                hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
                hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
            }
            if (lane == 0) {
                pbox[2 * (int64_t)(p0 + k)] = make_float4(lo.x, lo.y, lo.z, 0.0f);
                pbox[2 * (int64_t)(p0 + k) + 1] = make_float4(hi.x, hi.y, hi.z, 0.0f);
            }
        }
    }
}

// Key of every list entry: ||ref_s - c_f|| - r_f - (rounding radius of ref_s), a lower bound
// of the distance from the site's reference point to triangle f; q - ref gives, by the
// triangle inequality, key - ||q - ref|| <= ||q - c_f|| - r_f <= d(q, f).
__global__ void k_entry_keys(const int64_t* __restrict__ row_off64, int n_sites, const int32_t* __restrict__ row_tri,
                             const float4* __restrict__ refs, const float4* __restrict__ tsph, float* __restrict__ key) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int s = warp; s < n_sites; s += nwarps) {
        const float4 r = refs[s];
        for (int64_t j = row_off64[s] + lane; j < row_off64[s + 1]; j += 32) {
            const float4 c = tsph[row_tri[j]];
            const float dx = r.x - c.x, dy = r.y - c.y, dz = r.z - c.z;
            const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            // rounded down so that FP32 error never raises a lower bound
            key[j] = (d - c.w - r.w) * (1.0f - 1e-6f) - 1e-30f;
        }
    }
}

// Segment ends for the segmented sort: lists longer than long_row stay in BVH order (an
// empty segment), shorter ones are sorted by key.
__global__ void k_sort_segments(const int64_t* __restrict__ row_off64, int n_sites, int long_row,
                                int* __restrict__ beg, int* __restrict__ end) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sites; s += gridDim.x * blockDim.x) {
        const int64_t b = row_off64[s], e = row_off64[s + 1];
        beg[s] = (int)b;
        end[s] = (e - b <= long_row) ? (int)e : (int)b;
    }
}

// Copies the entries of the long (unsorted) lists from (ki, ti) to (ko, to).
__global__ void k_copy_long(const int64_t* __restrict__ row_off64, int n_sites, int long_row,
                            const float* __restrict__ ki, const int32_t* __restrict__ ti, float* __restrict__ ko,
                            int32_t* __restrict__ to) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int s = warp; s < n_sites; s += nwarps) {
        const int64_t b = row_off64[s], e = row_off64[s + 1];
        if (e - b <= long_row) continue;
        for (int64_t j = b + lane; j < e; j += 32) {
            ko[j] = ki[j];
            to[j] = ti[j];
        }
    }
}

__global__ void k_i64_to_i32(const int64_t* __restrict__ a, int32_t* __restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (int32_t)a[i];
}

// Builds the lists from the device ball table (d_balls, d_ball_off): m.d_row_off, the
// (triangle, key) entries m.d_row_ent (short lists sorted by key), the chunk boxes and the
// level-1 boxes.
// Bounding spheres in list order for the entries of long lists (the warp pass then reads an
// entry's sphere with a coalesced load instead of a gather through its triangle id).
__global__ void k_long_spheres(const int64_t* __restrict__ row_off64, int n_sites, int long_row,
                               const int32_t* __restrict__ row_tri, const float4* __restrict__ tsph,
                               float4* __restrict__ row_sph) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int s = warp; s < n_sites; s += nwarps) {
        const int64_t b = row_off64[s], e = row_off64[s + 1];
        if (e - b <= long_row) continue;
        for (int64_t j = b + lane; j < e; j += 32) row_sph[j] = tsph[row_tri[j]];
    }
}

// List entries as (triangle, key bits) pairs: the thread scan reads both with one 8-byte load.
__global__ void k_pack_entries(const int32_t* __restrict__ row_tri, const float* __restrict__ row_key, int64_t nnz,
                               int2* __restrict__ row_ent) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x)
        row_ent[j] = make_int2(row_tri[j], __float_as_int(row_key[j]));
}

int build_lists(MeshData& m, const float4* d_balls, const int64_t* d_ball_off, int n_sites, unsigned* status,
                cudaStream_t s) {
    const MeshView v = m.view();
    // the subtrees of the work items: the children of the nodes at depth kSplitDepth - 1 (a
    // leaf met earlier stands for itself), left to right
    constexpr int kSplitDepth = 4;
    auto child_ref = [](float w) {
        int r;
        std::memcpy(&r, &w, sizeof(r));
        return r;
    };
    std::vector<int2> sub;
    if (v.bvh_root >= 0) {
        std::vector<int2> level = {make_int2(-1, v.bvh_root)};  // (parent, node) with parent -1: the root
        for (int d = 0; d < kSplitDepth; ++d) {
            std::vector<int2> nextl;
            for (const int2& e : level) {
                if (e.y < 0) {  // a leaf: keep it where it is
                    nextl.push_back(e);
                    continue;
                }
                BNode nd;
                P2M_CUDA_TRY(cudaMemcpy(&nd, v.bvh + e.y, sizeof(BNode), cudaMemcpyDeviceToHost));
                nextl.push_back(make_int2(e.y, child_ref(nd.lo0.w)));
                nextl.push_back(make_int2(e.y, child_ref(nd.lo1.w)));
            }
            level.swap(nextl);
        }
        // (parent, child slot): which child of the parent each subtree root is
        for (const int2& e : level) {
            BNode nd;
            P2M_CUDA_TRY(cudaMemcpy(&nd, v.bvh + e.x, sizeof(BNode), cudaMemcpyDeviceToHost));
            sub.push_back(make_int2(e.x, child_ref(nd.lo0.w) == e.y ? 0 : 1));
        }
    } else {
        sub.push_back(make_int2(0, 0));  // one triangle: the root is the leaf itself
    }
    const int n_sub = (int)sub.size();
    const int64_t n_items = (int64_t)n_sites * n_sub;
    DevBuf d_sub, cnt, item_off, off64, tmp, stash, item_pos, top;
    P2M_TRY(d_sub.alloc(sizeof(int2) * n_sub));
    P2M_CUDA_TRY(cudaMemcpyAsync(d_sub.p, sub.data(), sizeof(int2) * n_sub, cudaMemcpyHostToDevice, s));
    P2M_TRY(cnt.alloc(sizeof(int64_t) * (n_items + 1)));
    P2M_TRY(item_off.alloc(sizeof(int64_t) * (n_items + 1)));
    P2M_TRY(off64.alloc(sizeof(int64_t) * (n_sites + 1)));
    // the first pass's stash: room for 64 entries per item on average, at most 2^28 entries
    const int64_t stash_cap = std::max<int64_t>(1024, std::min<int64_t>(64 * n_items, (int64_t)1 << 28));
    P2M_TRY(stash.alloc(sizeof(int32_t) * stash_cap));
    P2M_TRY(item_pos.alloc(sizeof(int64_t) * std::max<int64_t>(n_items, 1)));
    P2M_TRY(top.alloc(sizeof(unsigned long long)));
    P2M_CUDA_TRY(cudaMemsetAsync(top.p, 0, sizeof(unsigned long long), s));
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n_items + kListWarps - 1) / kListWarps,
                                                                   (int64_t)sm_count() * 16));
    k_lists<false><<<blocks, 32 * kListWarps, 0, s>>>(d_balls, d_ball_off, n_sites, v.bvh, v.bvh_root, d_sub.as<int2>(),
                                                     n_sub, v.tri, cnt.as<int64_t>(), nullptr, nullptr,
                                                     stash.as<int32_t>(), stash_cap, top.as<unsigned long long>(),
                                                     item_pos.as<int64_t>(), status);
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_CUDA_TRY(cudaMemsetAsync(cnt.as<int64_t>() + n_items, 0, sizeof(int64_t), s));
    size_t tb = 0;
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt.as<int64_t>(), item_off.as<int64_t>(), n_items + 1, s));
    P2M_TRY(tmp.alloc(tb + 16));
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp.p, tb, cnt.as<int64_t>(), item_off.as<int64_t>(), n_items + 1, s));
    k_site_offsets<<<std::max(1, std::min((n_sites + 256) / 256, 4096)), 256, 0, s>>>(item_off.as<int64_t>(), n_sites,
                                                                                     n_sub, off64.as<int64_t>());
    P2M_CUDA_TRY(cudaGetLastError());
    int64_t nnz = 0;
    P2M_CUDA_TRY(cudaMemcpyAsync(&nnz, off64.as<int64_t>() + n_sites, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    if (nnz > 0x7fffffffLL)
        return fail(P2M_ERR_LIMIT, "interception lists hold " + std::to_string(nnz) +
                                       " entries (> 2^31); enable site augmentation or coarsen the mesh");
    m.nnz = nnz;
    P2M_TRY(m.d_row_tri.alloc(sizeof(int32_t) * std::max<int64_t>(nnz, 1)));
    P2M_TRY(m.d_row_off.alloc(sizeof(int32_t) * (n_sites + 1)));
    k_copy_stash<<<std::max(1, std::min((int)((n_items + 7) / 8), sm_count() * 16)), 256, 0, s>>>(
        stash.as<int32_t>(), item_pos.as<int64_t>(), item_off.as<int64_t>(), n_items, m.d_row_tri.as<int32_t>());
    P2M_CUDA_TRY(cudaGetLastError());
    k_lists<true><<<blocks, 32 * kListWarps, 0, s>>>(d_balls, d_ball_off, n_sites, v.bvh, v.bvh_root, d_sub.as<int2>(),
                                                    n_sub, v.tri, nullptr, item_off.as<int64_t>(),
                                                    m.d_row_tri.as<int32_t>(), nullptr, 0, nullptr,
                                                    item_pos.as<int64_t>(), status);
    P2M_CUDA_TRY(cudaGetLastError());
    stash.release();
    k_i64_to_i32<<<64, 256, 0, s>>>(off64.as<int64_t>(), m.d_row_off.as<int32_t>(), n_sites + 1);
    P2M_CUDA_TRY(cudaGetLastError());
    // entry keys; lists scanned per thread are sorted by key (nearest first)
    {
        const int kb = std::max(1, std::min((n_sites + 7) / 8, sm_count() * 16));
        P2M_TRY(m.d_row_key.alloc(sizeof(float) * std::max<int64_t>(nnz, 1)));
        k_entry_keys<<<kb, 256, 0, s>>>(off64.as<int64_t>(), n_sites, m.d_row_tri.as<int32_t>(), m.d_refs.as<float4>(),
                                        m.d_tsph.as<float4>(), m.d_row_key.as<float>());
        P2M_CUDA_TRY(cudaGetLastError());
        if (nnz > 0) {
            DevBuf beg, end, key2, tri2, tmp3;
            P2M_TRY(beg.alloc(sizeof(int) * n_sites));
            P2M_TRY(end.alloc(sizeof(int) * n_sites));
            P2M_TRY(key2.alloc(sizeof(float) * nnz));
            P2M_TRY(tri2.alloc(sizeof(int32_t) * nnz));
            k_sort_segments<<<std::max(1, std::min((n_sites + 255) / 256, 4096)), 256, 0, s>>>(
                off64.as<int64_t>(), n_sites, m.long_row, beg.as<int>(), end.as<int>());
            P2M_CUDA_TRY(cudaGetLastError());
            size_t tb3 = 0;
            P2M_CUDA_TRY(cub::DeviceSegmentedSort::StableSortPairs(
                nullptr, tb3, m.d_row_key.as<float>(), key2.as<float>(), m.d_row_tri.as<int32_t>(), tri2.as<int32_t>(),
                (int)nnz, n_sites, beg.as<int>(), end.as<int>(), s));
            P2M_TRY(tmp3.alloc(tb3 + 16));
            P2M_CUDA_TRY(cub::DeviceSegmentedSort::StableSortPairs(
                tmp3.p, tb3, m.d_row_key.as<float>(), key2.as<float>(), m.d_row_tri.as<int32_t>(), tri2.as<int32_t>(),
                (int)nnz, n_sites, beg.as<int>(), end.as<int>(), s));
            k_copy_long<<<kb, 256, 0, s>>>(off64.as<int64_t>(), n_sites, m.long_row, m.d_row_key.as<float>(),
                                           m.d_row_tri.as<int32_t>(), key2.as<float>(), tri2.as<int32_t>());
            P2M_CUDA_TRY(cudaGetLastError());
            P2M_CUDA_TRY(cudaStreamSynchronize(s));
            m.d_row_key = std::move(key2);
            m.d_row_tri = std::move(tri2);
        }
    }
    // chunk boxes
    {
        DevBuf nch;
        P2M_TRY(nch.alloc(sizeof(int32_t) * (n_sites + 1)));
        P2M_TRY(m.d_chunk_off.alloc(sizeof(int32_t) * (n_sites + 1)));
        k_chunk_count<<<std::max(1, std::min((n_sites + 255) / 256, 4096)), 256, 0, s>>>(off64.as<int64_t>(), n_sites,
                                                                                      nch.as<int32_t>());
        P2M_CUDA_TRY(cudaGetLastError());
        P2M_CUDA_TRY(cudaMemsetAsync(nch.as<int32_t>() + n_sites, 0, sizeof(int32_t), s));
        size_t tb2 = 0;
        P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb2, nch.as<int32_t>(), m.d_chunk_off.as<int32_t>(), n_sites + 1, s));
        DevBuf tmp2;
        P2M_TRY(tmp2.alloc(tb2 + 16));
        P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp2.p, tb2, nch.as<int32_t>(), m.d_chunk_off.as<int32_t>(), n_sites + 1, s));
        int32_t nc = 0;
        P2M_CUDA_TRY(cudaMemcpyAsync(&nc, m.d_chunk_off.as<int32_t>() + n_sites, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        P2M_CUDA_TRY(cudaStreamSynchronize(s));
        m.n_chunks = nc;
        P2M_TRY(m.d_cbox.alloc(sizeof(float4) * 3 * std::max<int64_t>(nc, 1)));
        double scale = m.diag;
        for (int k = 0; k < 3; ++k) scale = std::max(scale, std::max(std::fabs(m.bb_lo[k]), std::fabs(m.bb_hi[k])));
        const float pad = (float)(scale * std::ldexp(1.0, -20));
        k_chunk_boxes<<<std::max(1, std::min((n_sites + 7) / 8, sm_count() * 16)), 256, 0, s>>>(
            off64.as<int64_t>(), m.d_chunk_off.as<int32_t>(), n_sites, m.d_row_tri.as<int32_t>(), m.d_tlo.as<float4>(),
            m.d_thi.as<float4>(), m.d_tri.as<float4>(), pad, m.d_cbox.as<float4>());
        P2M_CUDA_TRY(cudaGetLastError());
        // level-1 boxes over 32 chunks
        P2M_TRY(m.d_l1_off.alloc(sizeof(int32_t) * (n_sites + 1)));
        k_count_parents<<<std::max(1, std::min((n_sites + 255) / 256, 4096)), 256, 0, s>>>(m.d_chunk_off.as<int32_t>(),
                                                                                        n_sites, nch.as<int32_t>());
        P2M_CUDA_TRY(cudaGetLastError());
        P2M_CUDA_TRY(cudaMemsetAsync(nch.as<int32_t>() + n_sites, 0, sizeof(int32_t), s));
        P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp2.p, tb2, nch.as<int32_t>(), m.d_l1_off.as<int32_t>(), n_sites + 1, s));
        int32_t n1 = 0;
        P2M_CUDA_TRY(cudaMemcpyAsync(&n1, m.d_l1_off.as<int32_t>() + n_sites, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        P2M_CUDA_TRY(cudaStreamSynchronize(s));
        P2M_TRY(m.d_l1box.alloc(sizeof(float4) * 2 * std::max<int32_t>(n1, 1)));
        k_parent_boxes<<<std::max(1, std::min((n_sites + 7) / 8, sm_count() * 16)), 256, 0, s>>>(
            m.d_chunk_off.as<int32_t>(), m.d_l1_off.as<int32_t>(), n_sites, m.d_cbox.as<float4>(), m.d_l1box.as<float4>());
        P2M_CUDA_TRY(cudaGetLastError());
    }
    // the entries as (triangle, key) pairs; the separate arrays are released
    P2M_TRY(m.d_row_ent.alloc(sizeof(int2) * std::max<int64_t>(nnz, 1)));
    if (nnz > 0) {
        k_pack_entries<<<(int)std::min<int64_t>((nnz + 255) / 256, sm_count() * 32), 256, 0, s>>>(
            m.d_row_tri.as<int32_t>(), m.d_row_key.as<float>(), nnz, m.d_row_ent.as<int2>());
        P2M_CUDA_TRY(cudaGetLastError());
    }
    // row statistics (Table 1 Max / Avg)
    std::vector<int64_t> c(n_sites + 1);
    P2M_CUDA_TRY(cudaMemcpyAsync(c.data(), off64.p, sizeof(int64_t) * (n_sites + 1), cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t mx = 0;
    for (int i = 0; i < n_sites; ++i) mx = std::max(mx, c[i + 1] - c[i]);
    // spheres in list order for the long lists, when there are any
    m.d_row_sph.release();
    if (mx > m.long_row && nnz > 0) {
        P2M_TRY(m.d_row_sph.alloc(sizeof(float4) * nnz));
        k_long_spheres<<<std::max(1, std::min((n_sites + 7) / 8, sm_count() * 16)), 256, 0, s>>>(
            off64.as<int64_t>(), n_sites, m.long_row, m.d_row_tri.as<int32_t>(), m.d_tsph.as<float4>(),
            m.d_row_sph.as<float4>());
        P2M_CUDA_TRY(cudaGetLastError());
        P2M_CUDA_TRY(cudaStreamSynchronize(s));
    }
    m.d_row_tri.release();
    m.d_row_key.release();
    m.stats.nnz = nnz;
    m.stats.max_row = mx;
    m.stats.avg_row = n_sites ? (double)nnz / n_sites : 0.0;
    return P2M_OK;
}

}  // namespace p2m
