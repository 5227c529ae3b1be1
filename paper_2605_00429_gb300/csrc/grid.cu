// K2a: nearest-site grid.  The paper locates a query's cell by a nearest-neighbour search
// over the sites (Section 3.3 "Recursive Nearest Neighbor Search"); here a uniform grid over
// the domain box D lists, per grid cell, the sites whose Voronoi cells meet that grid cell.
// The nearest site of any point of the grid cell is among them (that point lies in its
// nearest site's cell), so a query scans one short candidate list.
//
// The lists are built site by site, by rasterising each Voronoi cell into the grid.  A warp
// takes one site s (or one piece of the box of a large cell): starting from the grid-index
// box around the cell's corners, it splits
// boxes in two along their longest side and drops a box as soon as the whole box lies
// strictly on the far side of the bisector between s and one of its Delaunay neighbours t
// (every point of the box nearer to t than to s, so no point of cell(s) is in it).  Boxes of
// one grid cell that survive are emitted as candidates.  Dropping uses one plane at a time,
// and at most 96 neighbours' planes, so a box cut off only by two planes together (or by an
// unused neighbour) survives: the lists may hold a few extra sites, never miss one.  Each grid cell is tested grown by 1% of a cell on every side, so a
// query that FP32 rounding bins into a neighbouring cell still finds its nearest site.
//
// Count pass (cells' candidate counts, atomics), scan, fill pass (atomic slots), then each
// cell's list is sorted by site id (the order does not change any result; it makes the grid
// deterministic).  A query reads its cell's run of ids and the sites' positions from the site
// table.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include "geom.cuh"
#include "host.h"
#include "voronoi.h"

namespace p2m {

constexpr int kRasterWarps = 4;     // warps per block, one site each
constexpr int kRasterStack = 768;   // boxes per warp (a 32-wide depth-first walk needs <= 24 x 32)
constexpr int kRasterPlanes = 96;   // bisectors per site staged in shared memory

struct RasterParams {
    float3 lo;     // domain D lower corner
    float3 h;      // grid cell size per axis
    int G;
    float ext;     // extent E of D (largest |coordinate| or diagonal)
    float rel;     // rounding margin of the bisector test, relative (see build_grid)
};

// A box of grid indices [x0, x1] x [y0, y1] x [z0, z1] (inclusive, 10 bits each).
__device__ __forceinline__ unsigned long long pack_box(int x0, int x1, int y0, int y1, int z0, int z1) {
    return (unsigned long long)x0 | ((unsigned long long)x1 << 10) | ((unsigned long long)y0 << 20) |
           ((unsigned long long)y1 << 30) | ((unsigned long long)z0 << 40) | ((unsigned long long)z1 << 50);
}

// Is the whole box (relative to the site: [bl, bh]) strictly nearer to the neighbour at
// offset d = t - s?  A point x' (relative) is nearer to t iff 2 x'.d - |d|^2 > 0; the
// minimum over the box picks each axis's end by the sign of d.  p.w = |d|^2 + margin.
__device__ __forceinline__ bool box_beyond(float3 bl, float3 bh, float4 p) {
    const float mx = p.x > 0.0f ? bl.x * p.x : bh.x * p.x;
    const float my = p.y > 0.0f ? bl.y * p.y : bh.y * p.y;
    const float mz = p.z > 0.0f ? bl.z * p.z : bh.z * p.z;
    return 2.0f * (mx + my + mz) - p.w > 0.0f;
}

// Rasterise the Voronoi cells into the grid, one work item (site, box of grid indices) per
// warp: a site whose box around its cell is large is cut into several items, so that no warp
// walks a huge box alone.  FILL = false: count the candidates of every grid cell (cell_count)
// and of every item (item_count).  FILL = true: write each site into its grid cells' lists
// (out_site at cell_off[c] + an atomic slot).  nb_off / nb_id: the bisector neighbours of
// each site used by the test (at most kRasterPlanes, see build_grid).
template <bool FILL>
__global__ void __launch_bounds__(32 * kRasterWarps)
    k_grid_raster(RasterParams g, const float4* __restrict__ sites, const int32_t* __restrict__ nb_off,
                  const int32_t* __restrict__ nb_id, const int4* __restrict__ items, int n_items,
                  int* __restrict__ cell_count, const int* __restrict__ cell_off, int* __restrict__ out_site,
                  int* __restrict__ item_count, unsigned* status) {
    __shared__ float4 planes[kRasterWarps][kRasterPlanes];
    __shared__ unsigned long long stack[kRasterWarps][kRasterStack];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    for (int it = blockIdx.x * kRasterWarps + w; it < n_items; it += gridDim.x * kRasterWarps) {
        const int4 item = __ldg(items + it);  // (site, x0 | x1 << 16, y0 | y1 << 16, z0 | z1 << 16)
        const int s = item.x;
        const float4 sp = __ldg(sites + s);
        const int n0 = nb_off[s];
        const int nn = nb_off[s + 1] - n0;
        // bisector of (s, t) relative to s: d = t - s (exact for lattice sites), |d|^2 and a
        // margin that covers the FP32 rounding of the test (|x'| <= the domain's extent)
        auto plane_of = [&](int k) {
            const float4 t = __ldg(sites + __ldg(nb_id + n0 + k));
            const float dx = t.x - sp.x, dy = t.y - sp.y, dz = t.z - sp.z;
            const float dd = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            return make_float4(dx, dy, dz, dd + g.rel * fmaf(g.ext, sqrtf(dd), dd));
        };
        const int np = min(nn, kRasterPlanes);
        __syncwarp();
        for (int k = lane; k < np; k += 32) planes[w][k] = plane_of(k);
        __syncwarp();
        auto rejected = [&](int x0, int x1, int y0, int y1, int z0, int z1) {
            const float3 bl = make_float3(fmaf((float)x0 - 0.01f, g.h.x, g.lo.x) - sp.x,
                                          fmaf((float)y0 - 0.01f, g.h.y, g.lo.y) - sp.y,
                                          fmaf((float)z0 - 0.01f, g.h.z, g.lo.z) - sp.z);
            const float3 bh = make_float3(fmaf((float)x1 + 1.01f, g.h.x, g.lo.x) - sp.x,
                                          fmaf((float)y1 + 1.01f, g.h.y, g.lo.y) - sp.y,
                                          fmaf((float)z1 + 1.01f, g.h.z, g.lo.z) - sp.z);
            for (int k = 0; k < np; ++k)
                if (box_beyond(bl, bh, planes[w][k])) return true;
            return false;
        };
        int emitted = 0;
        auto emit = [&](int x, int y, int z) {
            const int64_t c = ((int64_t)z * g.G + y) * g.G + x;
            if (FILL) out_site[cell_off[c] + atomicAdd(cell_count + c, 1)] = s;
            else atomicAdd(cell_count + c, 1);
            ++emitted;
        };
        if (lane == 0)
            stack[w][0] = pack_box(item.y & 0xffff, item.y >> 16, item.z & 0xffff, item.z >> 16, item.w & 0xffff,
                                   item.w >> 16);
        int sp_top = 1;
        __syncwarp();
        while (sp_top > 0) {
            const int take = min(sp_top, 32);
            sp_top -= take;
            unsigned long long b = 0;
            if (lane < take) b = stack[w][sp_top + lane];
            __syncwarp();
            int x0 = (int)(b & 1023), x1 = (int)((b >> 10) & 1023), y0 = (int)((b >> 20) & 1023),
                y1 = (int)((b >> 30) & 1023), z0 = (int)((b >> 40) & 1023), z1 = (int)((b >> 50) & 1023);
            bool split = false;
            if (lane < take && !rejected(x0, x1, y0, y1, z0, z1)) {
                if (x0 == x1 && y0 == y1 && z0 == z1) emit(x0, y0, z0);
                else split = true;
            }
            // children of the surviving boxes go on the stack (two each), as room allows
            const unsigned m = __ballot_sync(FULL, split);
            const int rank = __popc(m & ((1u << lane) - 1u));
            const bool room = sp_top + 2 * (rank + 1) <= kRasterStack;
            if (split && room) {
                const int ex = x1 - x0, ey = y1 - y0, ez = z1 - z0;
                unsigned long long c0, c1;
                if (ex >= ey && ex >= ez) {
                    const int mid = x0 + ex / 2;
                    c0 = pack_box(x0, mid, y0, y1, z0, z1);
                    c1 = pack_box(mid + 1, x1, y0, y1, z0, z1);
                } else if (ey >= ez) {
                    const int mid = y0 + ey / 2;
                    c0 = pack_box(x0, x1, y0, mid, z0, z1);
                    c1 = pack_box(x0, x1, mid + 1, y1, z0, z1);
                } else {
                    const int mid = z0 + ez / 2;
                    c0 = pack_box(x0, x1, y0, y1, z0, mid);
                    c1 = pack_box(x0, x1, y0, y1, mid + 1, z1);
                }
                stack[w][sp_top + 2 * rank] = c0;
                stack[w][sp_top + 2 * rank + 1] = c1;
            } else if (split) {
                // no room: test this box's grid cells one by one (slower, same result)
                for (int z = z0; z <= z1; ++z)
                    for (int y = y0; y <= y1; ++y)
                        for (int x = x0; x <= x1; ++x)
                            if (!rejected(x, x, y, y, z, z)) emit(x, y, z);
            }
            sp_top += 2 * __popc(__ballot_sync(FULL, split && room));
            __syncwarp();
        }
        for (int o = 16; o > 0; o >>= 1) emitted += __shfl_xor_sync(FULL, emitted, o);
        if (lane == 0) {
            if (!FILL) item_count[it] = emitted;
            else if (emitted != item_count[it]) atomicOr(status, ST_BAD);  // both passes walk alike
        }
    }
}

int build_grid(MeshData& m, const SiteSet& ss, int G, unsigned* status, cudaStream_t s) {
    if (G < 1 || G > 1023) return fail(P2M_ERR_INVALID_ARG, "nearest-site grid resolution must be 1..1023");
    const int64_t n_cells = (int64_t)G * G * G;
    const int S = (int)(m.site_pos.size() / 3);
    RasterParams g;
    g.G = G;
    g.lo = make_float3((float)m.dom_lo[0], (float)m.dom_lo[1], (float)m.dom_lo[2]);
    g.h = make_float3((float)((m.dom_hi[0] - m.dom_lo[0]) / G), (float)((m.dom_hi[1] - m.dom_lo[1]) / G),
                      (float)((m.dom_hi[2] - m.dom_lo[2]) / G));
    // The test value 2 x'.d - |d|^2 is at most a few (|x'| |d| + |d|^2) in size, with |x'| up
    // to the extent E of D; each FP32 operation adds a relative 2^-24, the box corners x'
    // carry an absolute error of a few ulp(E).  A margin of 2^-14 (E |d| + |d|^2) is a wide
    // cover (it moves the bisector by at most ~2^-15 E, far below a grid cell).
    double ext = 0;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, std::max(std::fabs(m.dom_lo[k]), std::fabs(m.dom_hi[k])));
    ext = std::max(ext, m.diag);
    g.ext = (float)ext;
    g.rel = (float)std::ldexp(1.0, -14);
    // per site: the box of grid indices around its cell's corners (one cell of margin against
    // rounding), cut into work items of at most kItemSide^3 grid cells; and the bisector
    // neighbours the test uses.  A site with more than kRasterPlanes neighbours (the centre of
    // a co-spherical or co-circular set has hundreds) keeps a subset spread over directions
    // (farthest-point sampling of the unit vectors to them, starting from the nearest), so
    // that its cell stays bounded on every side; fewer planes only add candidates.
    constexpr int kItemSide = 24;
    std::vector<std::vector<int4>> site_items(S);
    std::vector<std::vector<int32_t>> site_nb(S);
    {
        std::atomic<int> next(0);
        auto work = [&]() {
            std::vector<double> dir;
            std::vector<double> mind;
            while (true) {
                const int i0 = next.fetch_add(256);
                if (i0 >= S) break;
                for (int i = i0; i < std::min(S, i0 + 256); ++i) {
                    const int64_t c0 = ss.cell_off[i], c1 = ss.cell_off[i + 1];
                    if (c1 > c0) {
                        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
                        for (int64_t c = c0; c < c1; ++c)
                            for (int k = 0; k < 3; ++k) {
                                lo[k] = std::min(lo[k], ss.cell_xyz[3 * c + k]);
                                hi[k] = std::max(hi[k], ss.cell_xyz[3 * c + k]);
                            }
                        int a[3], b[3];
                        for (int k = 0; k < 3; ++k) {
                            const double hk = (m.dom_hi[k] - m.dom_lo[k]) / G;
                            a[k] = std::max(0, std::min(G - 1, (int)std::floor((lo[k] - m.dom_lo[k]) / hk) - 1));
                            b[k] = std::max(0, std::min(G - 1, (int)std::floor((hi[k] - m.dom_lo[k]) / hk) + 1));
                        }
                        for (int z = a[2]; z <= b[2]; z += kItemSide)
                            for (int y = a[1]; y <= b[1]; y += kItemSide)
                                for (int x = a[0]; x <= b[0]; x += kItemSide) {
                                    const int x1 = std::min(b[0], x + kItemSide - 1), y1 = std::min(b[1], y + kItemSide - 1),
                                              z1 = std::min(b[2], z + kItemSide - 1);
                                    site_items[i].push_back(make_int4(i, x | (x1 << 16), y | (y1 << 16), z | (z1 << 16)));
                                }
                    }
                    const int64_t n0 = ss.nb_off[i], nn = ss.nb_off[i + 1] - n0;
                    std::vector<int32_t>& out = site_nb[i];
                    if (nn <= kRasterPlanes) {
                        out.assign(ss.nb_id.begin() + n0, ss.nb_id.begin() + n0 + nn);
                        continue;
                    }
                    const float* ps = m.site_pos.data();
                    dir.assign(3 * nn, 0.0);
                    for (int64_t k = 0; k < nn; ++k) {
                        const int t = ss.nb_id[n0 + k];
                        double d[3], l = 0;
                        for (int c = 0; c < 3; ++c) {
                            d[c] = (double)ps[3 * t + c] - (double)ps[3 * i + c];
                            l += d[c] * d[c];
                        }
                        l = std::sqrt(std::max(l, 1e-300));
                        for (int c = 0; c < 3; ++c) dir[3 * k + c] = d[c] / l;
                    }
                    mind.assign(nn, 1e300);
                    int64_t pick = 0;  // the nearest neighbour (lists are nearest first)
                    for (int r = 0; r < kRasterPlanes; ++r) {
                        out.push_back(ss.nb_id[n0 + pick]);
                        int64_t far = -1;
                        for (int64_t k = 0; k < nn; ++k) {
                            const double dd = 1.0 - (dir[3 * k] * dir[3 * pick] + dir[3 * k + 1] * dir[3 * pick + 1] +
                                                     dir[3 * k + 2] * dir[3 * pick + 2]);
                            mind[k] = std::min(mind[k], dd);
                            if (mind[k] > 0 && (far < 0 || mind[k] > mind[far])) far = k;
                        }
                        if (far < 0) break;
                        pick = far;
                    }
                }
            }
        };
        std::vector<std::thread> th;
        for (int t = 0; t < std::max(1, std::min(hardware_threads(), (S + 255) / 256)); ++t) th.emplace_back(work);
        for (auto& t : th) t.join();
    }
    std::vector<int4> items;
    std::vector<int32_t> rnb_off(S + 1, 0), rnb;
    for (int i = 0; i < S; ++i) {
        items.insert(items.end(), site_items[i].begin(), site_items[i].end());
        rnb.insert(rnb.end(), site_nb[i].begin(), site_nb[i].end());
        rnb_off[i + 1] = (int32_t)rnb.size();
    }
    const int n_items = (int)items.size();
    DevBuf d_items, d_nboff, d_nb, d_count, d_off, d_item_count, d_ids, d_ids2, tmp;
    P2M_TRY(d_items.alloc(sizeof(int4) * std::max(n_items, 1)));
    P2M_TRY(d_nboff.alloc(sizeof(int32_t) * (S + 1)));
    P2M_TRY(d_nb.alloc(sizeof(int32_t) * std::max<size_t>(rnb.size(), 1)));
    P2M_TRY(d_count.alloc(sizeof(int) * (n_cells + 1)));
    P2M_TRY(d_off.alloc(sizeof(int) * (n_cells + 1)));
    P2M_TRY(d_item_count.alloc(sizeof(int) * std::max(n_items, 1)));
    if (n_items > 0)
        P2M_CUDA_TRY(cudaMemcpyAsync(d_items.p, items.data(), sizeof(int4) * n_items, cudaMemcpyHostToDevice, s));
    P2M_CUDA_TRY(cudaMemcpyAsync(d_nboff.p, rnb_off.data(), sizeof(int32_t) * (S + 1), cudaMemcpyHostToDevice, s));
    if (!rnb.empty())
        P2M_CUDA_TRY(cudaMemcpyAsync(d_nb.p, rnb.data(), sizeof(int32_t) * rnb.size(), cudaMemcpyHostToDevice, s));
    P2M_CUDA_TRY(cudaMemsetAsync(d_count.p, 0, sizeof(int) * (n_cells + 1), s));
    const int blocks = std::max(1, std::min((n_items + kRasterWarps - 1) / kRasterWarps, sm_count() * 16));
    const float4* sites = m.d_sites.as<float4>();
    k_grid_raster<false><<<blocks, 32 * kRasterWarps, 0, s>>>(g, sites, d_nboff.as<int32_t>(), d_nb.as<int32_t>(),
                                                               d_items.as<int4>(), n_items, d_count.as<int>(), nullptr,
                                                               nullptr, d_item_count.as<int>(), status);
    P2M_CUDA_TRY(cudaGetLastError());
    size_t tb = 0, tb2 = 0;
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tb, d_count.as<int>(), d_off.as<int>(), (int)(n_cells + 1), s));
    // the count could exceed int32 only for absurd grids; it is checked below on the int64 sum
    std::vector<int> cnt(n_cells);
    P2M_CUDA_TRY(cudaMemcpyAsync(cnt.data(), d_count.p, sizeof(int) * n_cells, cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t total = 0, mx = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        total += cnt[c];
        mx = std::max<int64_t>(mx, cnt[c]);
    }
    if (total > 0x7fffffffLL) return fail(P2M_ERR_LIMIT, "nearest-site grid too large");
    P2M_CUDA_TRY(cub::DeviceSegmentedSort::SortKeys(nullptr, tb2, (const int*)nullptr, (int*)nullptr, (int)total,
                                                    (int)n_cells, (const int*)nullptr, (const int*)nullptr, s));
    P2M_TRY(tmp.alloc(std::max(tb, tb2) + 16));
    P2M_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp.p, tb, d_count.as<int>(), d_off.as<int>(), (int)(n_cells + 1), s));
    P2M_TRY(d_ids.alloc(sizeof(int) * std::max<int64_t>(total, 1)));
    P2M_TRY(d_ids2.alloc(sizeof(int) * std::max<int64_t>(total, 1)));
    P2M_CUDA_TRY(cudaMemsetAsync(d_count.p, 0, sizeof(int) * (n_cells + 1), s));
    k_grid_raster<true><<<blocks, 32 * kRasterWarps, 0, s>>>(g, sites, d_nboff.as<int32_t>(), d_nb.as<int32_t>(),
                                                              d_items.as<int4>(), n_items, d_count.as<int>(),
                                                              d_off.as<int>(), d_ids.as<int>(), d_item_count.as<int>(),
                                                              status);
    P2M_CUDA_TRY(cudaGetLastError());
    if (total > 0)
        P2M_CUDA_TRY(cub::DeviceSegmentedSort::SortKeys(tmp.p, tb2, d_ids.as<int>(), d_ids2.as<int>(), (int)total,
                                                        (int)n_cells, d_off.as<int>(), d_off.as<int>() + 1, s));
    m.d_cell_off = std::move(d_off);
    m.d_cell_id = std::move(d_ids2);
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    m.G = G;
    m.g_lo = g.lo;
    m.g_hi = make_float3((float)m.dom_hi[0], (float)m.dom_hi[1], (float)m.dom_hi[2]);
    m.g_inv_h = make_float3(1.0f / g.h.x, 1.0f / g.h.y, 1.0f / g.h.z);
    m.stats.grid_res = G;
    m.stats.grid_entries = total;
    m.stats.grid_max = mx;
    return P2M_OK;
}

}  // namespace p2m
