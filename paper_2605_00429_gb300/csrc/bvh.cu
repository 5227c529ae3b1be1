// K0b triangle precompute, K0 LBVH (Morton codes, radix sort, Karras hierarchy, bottom-up
// refit) and K5 exact closest-triangle search by BVH branch and bound.
//
// The BVH of the base mesh is what the paper resolves its sphere-mesh intersection tests
// against (Section 3.3 "Implementation Details"); here it is also the exact search for
// queries outside the clipped domain and for proj(s, M) of auxiliary sites (Eq. 8).
#include <cub/device/device_radix_sort.cuh>

#include "bvh_dev.cuh"
#include "p2m_internal.h"

namespace p2m {

// ----------------------------------------------------------------------------- K0b

// One thread per triangle: the 64-byte record of geom.cuh and the minimal enclosing
// sphere (circumcentre for an acute triangle, else the midpoint of the longest edge; the
// radius is measured to the stored vertices and inflated to absorb FP32 rounding).
__global__ void k_tri_precompute(const float* __restrict__ verts, const int32_t* __restrict__ tris, int n_tris,
                                 float4* __restrict__ rec, float4* __restrict__ sph) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_tris) return;
    const int i0 = tris[3 * f], i1 = tris[3 * f + 1], i2 = tris[3 * f + 2];
    const float3 a = make_float3(verts[3 * i0], verts[3 * i0 + 1], verts[3 * i0 + 2]);
    const float3 b = make_float3(verts[3 * i1], verts[3 * i1 + 1], verts[3 * i1 + 2]);
    const float3 c = make_float3(verts[3 * i2], verts[3 * i2 + 1], verts[3 * i2 + 2]);
    const float3 e0 = b - a, e1 = c - a, e2 = c - b;
    const float l0 = dot3(e0, e0), l1 = dot3(e1, e1), l2 = dot3(e2, e2);
    const float3 n = make_float3(dop(e0.y, e1.z, e0.z, e1.y), dop(e0.z, e1.x, e0.x, e1.z), dop(e0.x, e1.y, e0.y, e1.x));
    const float nn = dot3(n, n);
    // Too thin to project onto (sin^2 of the angle at v0 below 1e-12): edges only.
    const bool flat = !(nn > 1e-12f * l0 * l1 && nn > 0.0f);
    const float rn = flat ? 0.0f : rsqrtf(nn);
    float4* r = rec + 4 * (int64_t)f;
    r[0] = make_float4(n.x * rn, n.y * rn, n.z * rn, flat ? __int_as_float(0x7fc00000) : rn);
    r[1] = make_float4(a.x, a.y, a.z, l0 > 0.0f ? 1.0f / l0 : 0.0f);
    r[2] = make_float4(e0.x, e0.y, e0.z, l1 > 0.0f ? 1.0f / l1 : 0.0f);
    r[3] = make_float4(e1.x, e1.y, e1.z, l2 > 0.0f ? 1.0f / l2 : 0.0f);

    // minimal enclosing sphere
    float3 cen;
    const float d_ab_ac = dot3(e0, e1);               // angle at a
    const float d_ba_bc = -dot3(e0, e2);              // angle at b: (a-b).(c-b)
    const float d_ca_cb = dot3(e1, e2);               // angle at c: (a-c).(b-c) = e1.e2
    if (d_ab_ac <= 0.0f || d_ba_bc <= 0.0f || d_ca_cb <= 0.0f || !(nn > 0.0f)) {
        // right/obtuse/degenerate: midpoint of the longest edge
        if (l0 >= l1 && l0 >= l2) cen = 0.5f * (a + b);
        else if (l1 >= l2) cen = 0.5f * (a + c);
        else cen = 0.5f * (b + c);
    } else {
        // circumcentre a + (l1 (n x e0) ... ) standard form: ((|e0|^2 e1 - |e1|^2 e0) x n) / (2|n|^2)
        const float3 t = make_float3(l0 * e1.x - l1 * e0.x, l0 * e1.y - l1 * e0.y, l0 * e1.z - l1 * e0.z);
        const float3 k = cross3(t, n);
        const float s = 0.5f / nn;
        cen = a + s * k;
    }
    float3 da = a - cen, db = b - cen, dc = c - cen;
    float rad = sqrtf(fmaxf(dot3(da, da), fmaxf(dot3(db, db), dot3(dc, dc))));
    const float mag = fmaxf(fabsf(cen.x), fmaxf(fabsf(cen.y), fabsf(cen.z)));
    rad = rad * (1.0f + 4e-7f) + 2.4e-7f * (mag + rad);
    sph[f] = make_float4(cen.x, cen.y, cen.z, rad);
}

int launch_tri_precompute(const float* d_verts, const int32_t* d_tris, int n_tris, float4* d_tri, float4* d_tsph,
                          cudaStream_t s) {
    if (n_tris <= 0) return P2M_OK;
    k_tri_precompute<<<(n_tris + 255) / 256, 256, 0, s>>>(d_verts, d_tris, n_tris, d_tri, d_tsph);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

__global__ void k_tri_boxes(const float* __restrict__ verts, const int32_t* __restrict__ tris, int n,
                            float4* __restrict__ lo, float4* __restrict__ hi) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    float3 mn = make_float3(INFINITY, INFINITY, INFINITY), mx = make_float3(-INFINITY, -INFINITY, -INFINITY);
    for (int k = 0; k < 3; ++k) {
        const int i = tris[3 * f + k];
        const float x = verts[3 * i], y = verts[3 * i + 1], z = verts[3 * i + 2];
        mn.x = fminf(mn.x, x); mn.y = fminf(mn.y, y); mn.z = fminf(mn.z, z);
        mx.x = fmaxf(mx.x, x); mx.y = fmaxf(mx.y, y); mx.z = fmaxf(mx.z, z);
    }
    lo[f] = make_float4(mn.x, mn.y, mn.z, 0.0f);
    hi[f] = make_float4(mx.x, mx.y, mx.z, 0.0f);
}

int tri_boxes(const float* d_verts, const int32_t* d_tris, int n_tris, float4* lo, float4* hi, cudaStream_t s) {
    if (n_tris <= 0) return P2M_OK;
    k_tri_boxes<<<(n_tris + 255) / 256, 256, 0, s>>>(d_verts, d_tris, n_tris, lo, hi);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

// ----------------------------------------------------------------------------- K0 LBVH

__device__ __forceinline__ unsigned spread10(unsigned v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_morton(const float4* __restrict__ lo, const float4* __restrict__ hi, int n, float3 c_lo,
                         float3 c_scale, unsigned* __restrict__ code, int* __restrict__ idx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 a = lo[i], b = hi[i];
    const float x = (0.5f * (a.x + b.x) - c_lo.x) * c_scale.x;
    const float y = (0.5f * (a.y + b.y) - c_lo.y) * c_scale.y;
    const float z = (0.5f * (a.z + b.z) - c_lo.z) * c_scale.z;
    const unsigned ux = (unsigned)fminf(fmaxf(x, 0.0f), 1023.0f);
    const unsigned uy = (unsigned)fminf(fmaxf(y, 0.0f), 1023.0f);
    const unsigned uz = (unsigned)fminf(fmaxf(z, 0.0f), 1023.0f);
    code[i] = (spread10(ux) << 2) | (spread10(uy) << 1) | spread10(uz);
    idx[i] = i;
}

// Length of the common prefix of keys i and j; equal codes fall back to the index bits so
// that every key is distinct (Karras 2012).
__device__ __forceinline__ int delta(const unsigned* __restrict__ code, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    const unsigned a = code[i], b = code[j];
    if (a == b) return 32 + __clz((unsigned)(i ^ j));
    return __clz(a ^ b);
}

// One thread per internal node i in [0, n-2]: the key range it covers and its split.
__global__ void k_karras(const unsigned* __restrict__ code, int n, int* __restrict__ left, int* __restrict__ right,
                         int* __restrict__ parent_int, int* __restrict__ parent_leaf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(code, n, i, i + 1) - delta(code, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = delta(code, n, i, i - d);
    int lmax = 2;
    while (delta(code, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(code, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = delta(code, n, i, j);
    int s = 0;
    for (int t = (l + 1) >> 1;; t = (t + 1) >> 1) {
        if (delta(code, n, i, i + (s + t) * d) > dnode) s += t;
        if (t == 1) break;
    }
    const int g = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    // children: >= 0 internal, < 0 leaf ~sorted position
    const int c0 = (lo == g) ? ~g : g;
    const int c1 = (hi == g + 1) ? ~(g + 1) : g + 1;
    left[i] = c0;
    right[i] = c1;
    if (c0 >= 0) parent_int[c0] = i; else parent_leaf[~c0] = i;
    if (c1 >= 0) parent_int[c1] = i; else parent_leaf[~c1] = i;
}

// Bottom-up refit: each leaf walks up; the second child to arrive at a node finishes it.
__global__ void k_refit(int n, int leaf_sorted, const int* __restrict__ sorted_prim, const float4* __restrict__ plo,
                        const float4* __restrict__ phi, const int* __restrict__ left, const int* __restrict__ right,
                        const int* __restrict__ parent_int, const int* __restrict__ parent_leaf,
                        unsigned* __restrict__ visits, float4* __restrict__ nlo, float4* __restrict__ nhi,
                        BNode* __restrict__ nodes) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int node = parent_leaf[k];
    while (node >= 0) {
        __threadfence();
        if (atomicAdd(&visits[node], 1u) == 0u) return;  // first arrival: sibling not ready
        __threadfence();
        const int c[2] = {left[node], right[node]};
        float4 blo[2], bhi[2];
        for (int h = 0; h < 2; ++h) {
            if (c[h] < 0) {
                const int p = sorted_prim[~c[h]];
                blo[h] = plo[p];
                bhi[h] = phi[p];
                // leaf reference: ~sorted position (primitives renumbered in leaf order) or
                // ~original primitive id
                blo[h].w = __int_as_float(leaf_sorted ? ~(~c[h]) : ~p);
            } else {
                blo[h] = __ldcg(&nlo[c[h]]);
                bhi[h] = __ldcg(&nhi[c[h]]);
                blo[h].w = __int_as_float(c[h]);
            }
        }
        BNode b;
        b.lo0 = blo[0]; b.hi0 = bhi[0]; b.lo1 = blo[1]; b.hi1 = bhi[1];
        b.hi0.w = 0.0f; b.hi1.w = 0.0f;
        nodes[node] = b;
        nlo[node] = make_float4(fminf(blo[0].x, blo[1].x), fminf(blo[0].y, blo[1].y), fminf(blo[0].z, blo[1].z), 0.0f);
        nhi[node] = make_float4(fmaxf(bhi[0].x, bhi[1].x), fmaxf(bhi[0].y, bhi[1].y), fmaxf(bhi[0].z, bhi[1].z), 0.0f);
        node = (node == 0) ? -1 : parent_int[node];
    }
}

int build_lbvh(const float4* d_lo, const float4* d_hi, int n, float3 c_lo, float3 c_hi, Bvh& out, cudaStream_t s,
               DevBuf* order_out) {
    out.n_prims = n;
    if (n <= 0) return fail(P2M_ERR_INVALID_ARG, "BVH over zero primitives");
    if (n == 1) {
        out.root = ~0;
        if (order_out) {
            P2M_TRY(order_out->alloc(sizeof(int)));
            P2M_CUDA_TRY(cudaMemsetAsync(order_out->p, 0, sizeof(int), s));
        }
        return P2M_OK;
    }
    out.root = 0;
    DevBuf code, code2, idx, idx2, left, right, pint, pleaf, visits, nlo, nhi, tmp;
    P2M_TRY(code.alloc(sizeof(unsigned) * n));
    P2M_TRY(code2.alloc(sizeof(unsigned) * n));
    P2M_TRY(idx.alloc(sizeof(int) * n));
    P2M_TRY(idx2.alloc(sizeof(int) * n));
    P2M_TRY(left.alloc(sizeof(int) * n));
    P2M_TRY(right.alloc(sizeof(int) * n));
    P2M_TRY(pint.alloc(sizeof(int) * n));
    P2M_TRY(pleaf.alloc(sizeof(int) * n));
    P2M_TRY(visits.alloc(sizeof(unsigned) * n));
    P2M_TRY(nlo.alloc(sizeof(float4) * n));
    P2M_TRY(nhi.alloc(sizeof(float4) * n));
    P2M_TRY(out.nodes.alloc(sizeof(BNode) * (n - 1)));
    const float ex = fmaxf(c_hi.x - c_lo.x, 1e-30f), ey = fmaxf(c_hi.y - c_lo.y, 1e-30f), ez = fmaxf(c_hi.z - c_lo.z, 1e-30f);
    const float3 sc = make_float3(1023.0f / ex, 1023.0f / ey, 1023.0f / ez);
    k_morton<<<(n + 255) / 256, 256, 0, s>>>(d_lo, d_hi, n, c_lo, sc, code.as<unsigned>(), idx.as<int>());
    P2M_CUDA_TRY(cudaGetLastError());
    size_t tmp_bytes = 0;
    P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, code.as<unsigned>(), code2.as<unsigned>(),
                                                 idx.as<int>(), idx2.as<int>(), n, 0, 30, s));
    P2M_TRY(tmp.alloc(tmp_bytes + 16));
    P2M_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, code.as<unsigned>(), code2.as<unsigned>(),
                                                 idx.as<int>(), idx2.as<int>(), n, 0, 30, s));
    P2M_CUDA_TRY(cudaMemsetAsync(pint.p, 0xff, sizeof(int) * n, s));
    k_karras<<<(n - 1 + 255) / 256, 256, 0, s>>>(code2.as<unsigned>(), n, left.as<int>(), right.as<int>(),
                                                 pint.as<int>(), pleaf.as<int>());
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_CUDA_TRY(cudaMemsetAsync(visits.p, 0, sizeof(unsigned) * n, s));
    k_refit<<<(n + 255) / 256, 256, 0, s>>>(n, order_out ? 1 : 0, idx2.as<int>(), d_lo, d_hi, left.as<int>(), right.as<int>(),
                                            pint.as<int>(), pleaf.as<int>(), visits.as<unsigned>(), nlo.as<float4>(),
                                            nhi.as<float4>(), out.nodes.as<BNode>());
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_CUDA_TRY(cudaStreamSynchronize(s));  // temporaries are released on return
    if (order_out) *order_out = std::move(idx2);
    return P2M_OK;
}

// dst[k] = src[order[k]] for records of `per` float4 each.
__global__ void k_gather_f4(const float4* __restrict__ src, float4* __restrict__ dst, const int* __restrict__ order,
                            int n, int per) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n * per;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / per, j = t % per;
        dst[t] = src[(int64_t)order[k] * per + j];
    }
}

int gather_f4(DevBuf& buf, const int* d_order, int n, int per, cudaStream_t s) {
    DevBuf out;
    P2M_TRY(out.alloc(sizeof(float4) * (size_t)n * per));
    const int64_t tot = (int64_t)n * per;
    k_gather_f4<<<(int)std::min<int64_t>((tot + 255) / 256, sm_count() * 64), 256, 0, s>>>(buf.as<float4>(), out.as<float4>(),
                                                                                   d_order, n, per);
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    buf = std::move(out);
    return P2M_OK;
}

// ----------------------------------------------------------------------------- K5

__global__ void k_bvh_closest(const BNode* __restrict__ nodes, int root, const float4* __restrict__ tri,
                              const float* __restrict__ pts, const int32_t* __restrict__ idx, const int* __restrict__ count,
                              int64_t n, float* __restrict__ dist, float* __restrict__ closest,
                              int32_t* __restrict__ tri_out, float* __restrict__ bary, unsigned* status,
                              const int32_t* __restrict__ orig) {
    const int64_t nn = count ? (int64_t)*count : n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx ? idx[k] : k;
    const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
    float s = 0.0f, t = 0.0f;
    const unsigned long long key = bvh_closest_key(q, nodes, root, tri, s, t, status);
    const int f = (int)(key & 0xffffffffu);
    const float d2 = __uint_as_float((unsigned)(key >> 32));
    dist[i] = sqrtf(d2);
    if (tri_out) tri_out[i] = orig ? __ldg(orig + f) : f;
    if (closest) {
        const TriRec T = load_tri(tri, f);
        const float3 p = tri_point(T, s, t);
        closest[3 * i] = p.x; closest[3 * i + 1] = p.y; closest[3 * i + 2] = p.z;
    }
    if (bary) { bary[3 * i] = 1.0f - s - t; bary[3 * i + 1] = s; bary[3 * i + 2] = t; }
    }
}

int launch_bvh_closest(const MeshView& m, const float* d_pts, const int32_t* d_idx, const int* d_count, int64_t n,
                       float* d_dist, float* d_closest, int32_t* d_tri, float* d_bary, unsigned* d_status,
                       cudaStream_t s) {
    if (n <= 0) return P2M_OK;
    const int bs = 128;
    // with a device-side count the launch is sized for a modest share of n: the grid-stride
    // loop covers the rest
    const int64_t want = (n + bs - 1) / bs;
    const int64_t blocks = d_count ? std::min<int64_t>(want, sm_count() * 8) : std::min<int64_t>(want, sm_count() * 64);
    k_bvh_closest<<<(unsigned)std::max<int64_t>(blocks, 1), bs, 0, s>>>(m.bvh, m.bvh_root, m.tri, d_pts, d_idx, d_count,
                                                                         n, d_dist, d_closest, d_tri, d_bary, d_status,
                                                                         m.orig);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

}  // namespace p2m
