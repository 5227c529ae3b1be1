// K2a: nearest-site grid.  The paper locates a query's cell by a nearest-neighbour search
// over the sites (Section 3.3 "Recursive Nearest Neighbor Search"); here a uniform grid
// over the domain box D stores, per grid cell, every site that can be the nearest site of
// some point of that cell, so a query reads one short candidate list.
//
// Candidates of a grid cell with centre c and half-diagonal h: with d_nn(c) the nearest-
// site distance, site s can win at a point x of the cell only if ||c - s|| <= d_nn(c) + 2h
// (the triangle inequality twice).  Those sites come from a range query on a BVH of the
// sites; each is then dropped if the whole cell is strictly closer to one of the 16 sites
// nearest to c (a linear test over the cell's corners, with a margin so that rounding
// never drops a true candidate).
#include <cub/device/device_scan.cuh>

#include "geom.cuh"
#include "host.h"

namespace p2m {

constexpr int kKnn = 16;
constexpr int kGridStack = 64;
constexpr int kGridSlab = 16;  // candidates a cell keeps from the counting pass (~6 on average)

struct GridParams {
    float3 lo;
    float3 cell;      // cell size per axis
    int G;
    float margin;     // rejection margin of the half-space filter (squared-length units)
};

__device__ __forceinline__ float3 cell_centre(const GridParams& g, int ix, int iy, int iz) {
    return make_float3(g.lo.x + (ix + 0.5f) * g.cell.x, g.lo.y + (iy + 0.5f) * g.cell.y, g.lo.z + (iz + 0.5f) * g.cell.z);
}

// k nearest sites of c by branch and bound (sorted ascending by (d2, id)).
__device__ void knn(float3 c, const BNode* __restrict__ nodes, int root, const float4* __restrict__ sites,
                    float* kd, int* ki, unsigned* status) {
    for (int j = 0; j < kKnn; ++j) { kd[j] = INFINITY; ki[j] = -1; }
    auto offer = [&](int s) {
        const float4 p = __ldg(sites + s);
        const float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        if (d2 > kd[kKnn - 1] || (d2 == kd[kKnn - 1] && s > ki[kKnn - 1])) return;
        int j = kKnn - 1;
        while (j > 0 && (kd[j - 1] > d2 || (kd[j - 1] == d2 && ki[j - 1] > s))) {
            kd[j] = kd[j - 1];
            ki[j] = ki[j - 1];
            --j;
        }
        kd[j] = d2;
        ki[j] = s;
    };
    if (root < 0) { offer(~root); return; }
    int stk[kGridStack];
    float sd[kGridStack];
    int sp = 0, node = root;
    while (true) {
        const float4* np = reinterpret_cast<const float4*>(nodes + node);
        const float4 lo0 = __ldg(np), hi0 = __ldg(np + 1), lo1 = __ldg(np + 2), hi1 = __ldg(np + 3);
        const int cs[2] = {__float_as_int(lo0.w), __float_as_int(lo1.w)};
        const float ds[2] = {box_dist2(c, f3(lo0), f3(hi0)), box_dist2(c, f3(lo1), f3(hi1))};
        const int first = ds[1] < ds[0] ? 1 : 0;
        int next = -1;
        for (int h = 0; h < 2; ++h) {
            const int k = h == 0 ? first : 1 - first;
            if (ds[k] > kd[kKnn - 1]) continue;
            if (cs[k] < 0) offer(~cs[k]);
            else if (next < 0) next = cs[k];
            else if (sp < kGridStack) { stk[sp] = cs[k]; sd[sp] = ds[k]; ++sp; }
            else atomicOr(status, ST_STACK);
        }
        if (next >= 0) { node = next; continue; }
        node = -1;
        while (sp > 0) {
            --sp;
            if (sd[sp] <= kd[kKnn - 1]) { node = stk[sp]; break; }
        }
        if (node < 0) break;
    }
}

// Is the whole box strictly closer to site t than to site s?  max over the box of
// 2 x.(s - t) + |t|^2 - |s|^2 must be < -margin.
__device__ __forceinline__ bool box_closer_to(float3 lo, float3 hi, float3 s, float3 t, float margin) {
    const float ax = 2.0f * (s.x - t.x), ay = 2.0f * (s.y - t.y), az = 2.0f * (s.z - t.z);
    const float m = (ax > 0 ? ax * hi.x : ax * lo.x) + (ay > 0 ? ay * hi.y : ay * lo.y) + (az > 0 ? az * hi.z : az * lo.z);
    const float v = m + (dot3(t, t) - dot3(s, s));
    return v < -margin;
}

// Counting pass (FILL = false): count[cid] = the cell's candidates, the first kGridSlab of
// them kept in slab[cid * kGridSlab ..].  Filling pass (FILL = true): the candidates of the
// cells in `list` (those that overflowed the slab) written to out[off[cid] ..].
template <bool FILL>
__global__ void k_grid(GridParams g, const BNode* __restrict__ nodes, int root, const float4* __restrict__ sites,
                       int n_sites, int64_t* __restrict__ count, float4* __restrict__ slab,
                       const int64_t* __restrict__ list, int64_t n_list, const int64_t* __restrict__ off,
                       float4* __restrict__ out, unsigned* status) {
    const int64_t n_cells = (int64_t)g.G * g.G * g.G;
    const int64_t n_work = FILL ? n_list : n_cells;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_work; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cid = FILL ? list[w] : w;
        const int ix = (int)(cid % g.G), iy = (int)((cid / g.G) % g.G), iz = (int)(cid / ((int64_t)g.G * g.G));
        const float3 c = cell_centre(g, ix, iy, iz);
        // the box is grown by 1% of a cell on every side: a query binned by FP32 rounding into
        // a neighbouring cell still lies inside the box its candidates were chosen for
        const float3 lo = make_float3(g.lo.x + (ix - 0.01f) * g.cell.x, g.lo.y + (iy - 0.01f) * g.cell.y,
                                      g.lo.z + (iz - 0.01f) * g.cell.z);
        const float3 hi = make_float3(g.lo.x + (ix + 1.01f) * g.cell.x, g.lo.y + (iy + 1.01f) * g.cell.y,
                                      g.lo.z + (iz + 1.01f) * g.cell.z);
        const float h = 0.5f * 1.02f * sqrtf(dot3(g.cell, g.cell));
        float kd[kKnn];
        int ki[kKnn];
        knn(c, nodes, root, sites, kd, ki, status);
        // range radius: d_nn + 2h, inflated so FP32 rounding never loses a site
        const float R = (sqrtf(kd[0]) + 2.0f * h) * (1.0f + 1e-5f) + 1e-6f * h;
        const float R2 = R * R;
        int64_t k = 0;
        const int64_t base = FILL ? off[cid] : 0;
        auto consider = [&](int s) {
            const float4 p = __ldg(sites + s);
            const float3 ps = f3(p);
            const float dx = ps.x - c.x, dy = ps.y - c.y, dz = ps.z - c.z;
            if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) > R2) return;
            for (int j = 0; j < kKnn; ++j) {
                const int t = ki[j];
                if (t < 0 || t == s) continue;
                if (box_closer_to(lo, hi, ps, f3(__ldg(sites + t)), g.margin)) return;
            }
            // candidate stored with its coordinates (id in w) so a query reads one contiguous run
            const float4 e = make_float4(ps.x, ps.y, ps.z, __int_as_float(s));
            if (FILL) out[base + k] = e;
            else if (k < kGridSlab) slab[cid * kGridSlab + k] = e;
            ++k;
        };
        if (root < 0) {
            consider(~root);
        } else {
            int stk[kGridStack];
            int sp = 0, node = root;
            while (node >= 0) {
                const float4* np = reinterpret_cast<const float4*>(nodes + node);
                const float4 lo0 = __ldg(np), hi0 = __ldg(np + 1), lo1 = __ldg(np + 2), hi1 = __ldg(np + 3);
                const int cs[2] = {__float_as_int(lo0.w), __float_as_int(lo1.w)};
                const float ds[2] = {box_dist2(c, f3(lo0), f3(hi0)), box_dist2(c, f3(lo1), f3(hi1))};
                int next = -1;
                for (int hh = 0; hh < 2; ++hh) {
                    if (ds[hh] > R2) continue;
                    if (cs[hh] < 0) consider(~cs[hh]);
                    else if (next < 0) next = cs[hh];
                    else if (sp < kGridStack) stk[sp++] = cs[hh];
                    else atomicOr(status, ST_STACK);
                }
                if (next < 0 && sp > 0) next = stk[--sp];
                node = next;
            }
        }
        if (!FILL) count[cid] = k;
        else if (k != off[cid + 1] - off[cid]) atomicOr(status, ST_BAD);
    }
}

__global__ void k_i64_to_i32(const int64_t* __restrict__ a, int32_t* __restrict__ b, int64_t n);

// Copies the slab-held candidates of every cell that fit into the slab to their CSR slots;
// the cells that overflowed are appended to `list` for the filling pass.
__global__ void k_grid_pack(const float4* __restrict__ slab, const int64_t* __restrict__ count,
                            const int64_t* __restrict__ off, int64_t n_cells, float4* __restrict__ out,
                            int64_t* __restrict__ list, unsigned long long* __restrict__ n_list) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = count[c];
        if (k > kGridSlab) {
            list[atomicAdd(n_list, 1ull)] = c;
            continue;
        }
        for (int64_t j = 0; j < k; ++j) out[off[c] + j] = slab[c * kGridSlab + j];
    }
}

int build_grid(MeshData& m, const Bvh& site_bvh, int G, unsigned* status, cudaStream_t s) {
    const int64_t n_cells = (int64_t)G * G * G;
    GridParams g;
    g.G = G;
    g.lo = make_float3((float)m.dom_lo[0], (float)m.dom_lo[1], (float)m.dom_lo[2]);
    g.cell = make_float3((float)((m.dom_hi[0] - m.dom_lo[0]) / G), (float)((m.dom_hi[1] - m.dom_lo[1]) / G),
                         (float)((m.dom_hi[2] - m.dom_lo[2]) / G));
    double scale = 0;
    for (int k = 0; k < 3; ++k) scale = std::max(scale, std::max(std::fabs(m.dom_lo[k]), std::fabs(m.dom_hi[k])));
    g.margin = (float)(64.0 * 1.2e-7 * 4.0 * scale * scale);
    DevBuf cnt, off;
    P2M_TRY(cnt.alloc(sizeof(int64_t) * (n_cells + 1)));
    P2M_TRY(off.alloc(sizeof(int64_t) * (n_cells + 1)));
    const int n_sites = (int)(m.site_pos.size() / 3);
    const BNode* nodes = site_bvh.nodes.as<const BNode>();
    const int blocks = (int)std::min<int64_t>((n_cells + 127) / 128, 152 * 32);
    DevBuf slab;
    P2M_TRY(slab.alloc(sizeof(float4) * kGridSlab * n_cells));
    k_grid<false><<<blocks, 128, 0, s>>>(g, nodes, site_bvh.root, m.d_sites.as<float4>(), n_sites, cnt.as<int64_t>(),
                                         slab.as<float4>(), nullptr, 0, nullptr, nullptr, status);
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_CUDA_TRY(cudaMemsetAsync(cnt.as<int64_t>() + n_cells, 0, sizeof(int64_t), s));
    DevBuf tmp;
    size_t tb = 0;
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt.as<int64_t>(), off.as<int64_t>(), n_cells + 1, s));
    P2M_TRY(tmp.alloc(tb + 16));
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp.p, tb, cnt.as<int64_t>(), off.as<int64_t>(), n_cells + 1, s));
    int64_t total = 0;
    P2M_CUDA_TRY(cudaMemcpyAsync(&total, off.as<int64_t>() + n_cells, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    if (total > 0x7fffffffLL) return fail(P2M_ERR_LIMIT, "nearest-site grid too large");
    P2M_TRY(m.d_cell_site.alloc(sizeof(float4) * std::max<int64_t>(total, 1)));
    P2M_TRY(m.d_cell_off.alloc(sizeof(int32_t) * (n_cells + 1)));
    // cells within the slab are copied; the rest (cells with more than kGridSlab candidates)
    // run the search again, writing straight to their slots
    DevBuf list, n_list;
    P2M_TRY(list.alloc(sizeof(int64_t) * std::max<int64_t>(n_cells, 1)));
    P2M_TRY(n_list.alloc(sizeof(unsigned long long)));
    P2M_CUDA_TRY(cudaMemsetAsync(n_list.p, 0, sizeof(unsigned long long), s));
    k_grid_pack<<<blocks, 128, 0, s>>>(slab.as<float4>(), cnt.as<int64_t>(), off.as<int64_t>(), n_cells,
                                       m.d_cell_site.as<float4>(), list.as<int64_t>(), n_list.as<unsigned long long>());
    P2M_CUDA_TRY(cudaGetLastError());
    unsigned long long n_over = 0;
    P2M_CUDA_TRY(cudaMemcpyAsync(&n_over, n_list.p, sizeof(n_over), cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    slab.release();
    if (n_over > 0) {
        const int ob = (int)std::min<int64_t>(((int64_t)n_over + 127) / 128, 152 * 32);
        k_grid<true><<<ob, 128, 0, s>>>(g, nodes, site_bvh.root, m.d_sites.as<float4>(), n_sites, nullptr, nullptr,
                                        list.as<int64_t>(), (int64_t)n_over, off.as<int64_t>(),
                                        m.d_cell_site.as<float4>(), status);
        P2M_CUDA_TRY(cudaGetLastError());
    }
    k_i64_to_i32<<<256, 256, 0, s>>>(off.as<int64_t>(), m.d_cell_off.as<int32_t>(), n_cells + 1);
    P2M_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> c(n_cells);
    P2M_CUDA_TRY(cudaMemcpyAsync(c.data(), cnt.p, sizeof(int64_t) * n_cells, cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t mx = 0;
    for (int64_t x : c) mx = std::max(mx, x);
    m.G = G;
    m.g_lo = g.lo;
    m.g_hi = make_float3((float)m.dom_hi[0], (float)m.dom_hi[1], (float)m.dom_hi[2]);
    m.g_inv_h = make_float3(1.0f / g.cell.x, 1.0f / g.cell.y, 1.0f / g.cell.z);
    m.stats.grid_res = G;
    m.stats.grid_entries = total;
    m.stats.grid_max = mx;
    return P2M_OK;
}

}  // namespace p2m
