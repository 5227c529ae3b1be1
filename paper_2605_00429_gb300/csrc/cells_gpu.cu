// Voronoi cell clipping on the device (Section 3.3: the corners of each site's cell carry
// the balls of Eq. 3).  The cell of site s is the domain box D cut by the bisector planes
// of its Delaunay neighbours; one thread clips one cell in FP64, with the same neighbour
// order (nearest first, as the neighbour lists are stored), tolerance rule and early stop
// as the host clipper, so both produce the same cell up to rounding.
//
// Representation: the cell's dual.  Each face plane has an index (0..5 for the box, then one
// per cut), and each corner is a triangle of the three planes through it, together with its
// position; the planes themselves need not be kept, since new corners are interpolated.  Keeping the
// triangles consistently oriented (det(n_a, n_b, n_c) > 0 for the box corners, and inherited
// from the removed triangle for new ones) makes every directed edge (a -> b) appear in
// exactly one triangle and (b -> a) in its neighbour, which is all a clip needs:
//   * the corners strictly beyond the plane (value > tol) are removed;
//   * each directed edge (a -> b) of a removed triangle whose neighbour (b -> a) is kept is
//     a polytope edge crossing the plane.  The new corner on it is interpolated between the
//     kept and the removed corner, as the host clipper does (the kept corner itself if it
//     lies within tol of the plane), and the new triangle is (a, b, P);
//   * for a convex cut the crossing edges form one cycle; anything else (rounding in a
//     degenerate configuration) or a cell beyond the fixed capacity hands the cell to the
//     host clipper.
#include <algorithm>
#include <chrono>
#include <cstring>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_run_length_encode.cuh>

#include "host_geom.h"
#include "p2m_internal.h"
#include "voronoi.h"

namespace p2m {

constexpr int kCellPlanes = 64;                 // 6 box planes + up to 58 cutting bisectors
constexpr int kCellTris = 2 * kCellPlanes - 4;  // corners of a cell with kCellPlanes faces
constexpr int kCellCycle = 64;                  // crossing edges of one cut

enum { CELL_OK = 0, CELL_HOST = 1, CELL_EMPTY = 2 };

struct Plane {
    double x, y, z, w;  // n.x <= w
};

__host__ __device__ __forceinline__ int tri_pack(int a, int b, int c) { return a | (b << 8) | (c << 16); }
__host__ __device__ __forceinline__ int tri_at(int t, int k) { return (t >> (8 * k)) & 0xff; }

struct CellPoly {
    int tri[kCellTris];
    double3 pos[kCellTris];
    int np, nt;  // planes used (box + cuts), corners
};

__host__ __device__ __forceinline__ double plane_val(const Plane& p, const double3& x) {
    return fma(p.x, x.x, fma(p.y, x.y, p.z * x.z)) - p.w;
}

__host__ __device__ void cell_box(CellPoly& C, double3 lo, double3 hi) {
    // planes 0..5: x <= hi.x, -x <= -lo.x, y <= hi.y, -y <= -lo.y, z <= hi.z, -z <= -lo.z
    C.np = 6;
    C.nt = 8;
    for (int i = 0; i < 8; ++i) {
        const int a = (i & 1) ? 0 : 1, b = (i & 2) ? 2 : 3, c = (i & 4) ? 4 : 5;
        // det(n_a, n_b, n_c) of signed axes = product of the signs; swap two planes if < 0
        const int sign = ((i & 1) ? 1 : -1) * ((i & 2) ? 1 : -1) * ((i & 4) ? 1 : -1);
        C.tri[i] = sign > 0 ? tri_pack(a, b, c) : tri_pack(a, c, b);
        C.pos[i] = make_double3((i & 1) ? hi.x : lo.x, (i & 2) ? hi.y : lo.y, (i & 4) ? hi.z : lo.z);
    }
}

// Index of the triangle holding the directed edge (u -> v), or -1.
__host__ __device__ __forceinline__ int find_edge(const CellPoly& C, int u, int v) {
    for (int t = 0; t < C.nt; ++t) {
        const int x = C.tri[t];
        const int a = tri_at(x, 0), b = tri_at(x, 1), c = tri_at(x, 2);
        if ((a == u && b == v) || (b == u && c == v) || (c == u && a == v)) return t;
    }
    return -1;
}

// Keep {x : n.x <= d}.  Returns 0 (no corner beyond the plane), 1 (cut), CELL_HOST or
// CELL_EMPTY (as negative values).
__host__ __device__ int cell_clip(CellPoly& C, double3 n, double d, double tol) {
    unsigned rm[(kCellTris + 31) / 32] = {};
    int n_rm = 0;
    const Plane P{n.x, n.y, n.z, d};
    for (int t = 0; t < C.nt; ++t)
        if (plane_val(P, C.pos[t]) > tol) {
            rm[t >> 5] |= 1u << (t & 31);
            ++n_rm;
        }
    if (n_rm == 0) return 0;
    if (n_rm == C.nt) return -CELL_EMPTY;
    if (C.np >= kCellPlanes) return -CELL_HOST;
    const int pid = C.np;
    int bu[kCellCycle], bv[kCellCycle];
    double3 bp[kCellCycle];
    int nb = 0;
    for (int t = 0; t < C.nt; ++t) {
        if (!(rm[t >> 5] >> (t & 31) & 1u)) continue;
        const int x = C.tri[t];
        for (int e = 0; e < 3; ++e) {
            const int u = tri_at(x, e), v = tri_at(x, (e + 1) % 3);
            const int k = find_edge(C, v, u);
            if (k < 0) return -CELL_HOST;                 // not a closed triangulation
            if (rm[k >> 5] >> (k & 31) & 1u) continue;    // both corners removed
            if (nb == kCellCycle) return -CELL_HOST;
            const double vk = plane_val(P, C.pos[k]), vr = plane_val(P, C.pos[t]);
            double3 p = C.pos[k];
            if (vk < -tol) {
                const double s = vk / (vk - vr);
                p = make_double3(fma(s, C.pos[t].x - p.x, p.x), fma(s, C.pos[t].y - p.y, p.y),
                                 fma(s, C.pos[t].z - p.z, p.z));
            }
            bu[nb] = u;
            bv[nb] = v;
            bp[nb] = p;
            ++nb;
        }
    }
    // the crossing edges must form one cycle: every plane starts at most one edge, and
    // following successors from the first edge visits all of them
    for (int i = 0; i < nb; ++i)
        for (int j = i + 1; j < nb; ++j)
            if (bu[i] == bu[j]) return -CELL_HOST;
    int cur = 0, steps = 0;
    do {
        int nxt = -1;
        for (int j = 0; j < nb; ++j)
            if (bu[j] == bv[cur]) { nxt = j; break; }
        if (nxt < 0) return -CELL_HOST;
        cur = nxt;
        ++steps;
    } while (cur != 0 && steps <= nb);
    if (cur != 0 || steps != nb) return -CELL_HOST;
    if (C.nt - n_rm + nb > kCellTris) return -CELL_HOST;
    // compact the kept corners, then append the new ones
    int w = 0;
    for (int t = 0; t < C.nt; ++t) {
        if (rm[t >> 5] >> (t & 31) & 1u) continue;
        C.tri[w] = C.tri[t];
        C.pos[w] = C.pos[t];
        ++w;
    }
    for (int i = 0; i < nb; ++i) {
        C.tri[w] = tri_pack(bu[i], bv[i], pid);
        C.pos[w] = bp[i];
        ++w;
    }
    C.nt = w;
    ++C.np;
    return 1;
}

__host__ __device__ __forceinline__ double cell_radius2(const CellPoly& C, double3 s) {
    double r2 = 0;
    for (int t = 0; t < C.nt; ++t) {
        const double dx = C.pos[t].x - s.x, dy = C.pos[t].y - s.y, dz = C.pos[t].z - s.z;
        r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
    }
    return r2;
}

// Clips the cell of site s and writes its distinct corners (within tol) to o[0 .. 3 * count);
// returns CELL_OK, CELL_HOST or CELL_EMPTY.
__host__ __device__ int clip_site(CellPoly& C, const double* site, int s, const int64_t* nb_off, const int32_t* nb_id,
                                  double3 lo, double3 hi, double tol, int max_clip, double* o, int& count) {
    const double3 ps = make_double3(site[3 * s], site[3 * s + 1], site[3 * s + 2]);
    const int64_t k0 = nb_off[s], k1 = nb_off[s + 1];
    count = 0;
    // a cell with more neighbours than cutting planes fit (the fans and axes of symmetric
    // meshes) goes to the host at once
    if (k1 - k0 > kCellPlanes - 6) return CELL_HOST;
    cell_box(C, lo, hi);
    double r2 = cell_radius2(C, ps);
    int used = 0, st = CELL_OK;
    for (int64_t k = k0; k < k1; ++k) {  // nearest first
        const int t = nb_id[k];
        const double3 pt = make_double3(site[3 * t], site[3 * t + 1], site[3 * t + 2]);
        double3 nrm = make_double3(pt.x - ps.x, pt.y - ps.y, pt.z - ps.z);
        const double d2 = nrm.x * nrm.x + nrm.y * nrm.y + nrm.z * nrm.z;
        if (0.25 * d2 > r2 * (1.0 + 1e-9) + tol * tol) break;
        const double len = sqrt(d2);
        if (!(len > 0)) continue;
        nrm = make_double3(nrm.x / len, nrm.y / len, nrm.z / len);
        const double d = 0.5 * (nrm.x * (pt.x + ps.x) + nrm.y * (pt.y + ps.y) + nrm.z * (pt.z + ps.z));
        const int rc = cell_clip(C, nrm, d, tol);
        if (rc < 0) {
            st = -rc;
            break;
        }
        if (rc == 1) {
            r2 = cell_radius2(C, ps);
            if (++used >= max_clip) break;
        }
    }
    if (st != CELL_OK) return st;
    int nc = 0;
    for (int t = 0; t < C.nt; ++t) {
        const double3 p = C.pos[t];
        bool dup = false;
        for (int j = 0; j < nc && !dup; ++j)
            dup = fabs(o[3 * j] - p.x) <= tol && fabs(o[3 * j + 1] - p.y) <= tol && fabs(o[3 * j + 2] - p.z) <= tol;
        if (dup) continue;
        o[3 * nc] = p.x;
        o[3 * nc + 1] = p.y;
        o[3 * nc + 2] = p.z;
        ++nc;
    }
    count = nc;
    return CELL_OK;
}

// One thread per site: the corners go to out[s * kCellTris ..], or the site is marked for
// the host clipper.
__global__ void __launch_bounds__(64) k_clip_cells(const double* __restrict__ site, int n_sites,
                                                   const int64_t* __restrict__ nb_off, const int32_t* __restrict__ nb_id,
                                                   double3 lo, double3 hi, double tol, int max_clip,
                                                   double* __restrict__ out, int* __restrict__ count,
                                                   int* __restrict__ state) {
    CellPoly C;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sites; s += gridDim.x * blockDim.x) {
        int nc = 0;
        state[s] = clip_site(C, site, s, nb_off, nb_id, lo, hi, tol, max_clip, out + (int64_t)s * kCellTris * 3, nc);
        count[s] = nc;
    }
}

// Packs the per-site corner slots into one CSR array.
__global__ void k_pack_corners(const double* __restrict__ slab, const int* __restrict__ count,
                               const int64_t* __restrict__ off, int n_sites, double* __restrict__ out) {
    for (int s = blockIdx.x; s < n_sites; s += gridDim.x) {
        const int n3 = 3 * count[s];
        const double* src = slab + (int64_t)s * kCellTris * 3;
        double* dst = out + 3 * off[s];
        for (int k = threadIdx.x; k < n3; k += blockDim.x) dst[k] = src[k];
    }
}

int SiteSet::clip_cells_gpu(const double dom_lo[3], const double dom_hi[3], double diag, int n_threads, void* stream,
                            int64_t* n_host, double* ms_kernel, double* ms_host) {
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)pts.size();
    std::vector<double> xyz(3 * (size_t)n);
    for (int i = 0; i < n; ++i) world(i, &xyz[3 * (size_t)i]);
    const int64_t nnb = nb_off[n];
    DevBuf d_site, d_off, d_nb, d_slab, d_count, d_state, d_coff, d_corner;
    if (d_site.alloc(sizeof(double) * 3 * n) || d_off.alloc(sizeof(int64_t) * (n + 1)) ||
        d_nb.alloc(sizeof(int32_t) * std::max<int64_t>(nnb, 1)) ||
        d_slab.alloc(sizeof(double) * 3 * (size_t)kCellTris * n) || d_count.alloc(sizeof(int) * n) ||
        d_state.alloc(sizeof(int) * n) || d_coff.alloc(sizeof(int64_t) * (n + 1)))
        return -2;
    if (cudaMemcpyAsync(d_site.p, xyz.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_off.p, nb_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s) ||
        (nnb > 0 && cudaMemcpyAsync(d_nb.p, nb_id.data(), sizeof(int32_t) * nnb, cudaMemcpyHostToDevice, s)))
        return -2;
    const double tol = clip_tol(diag);
    const int blocks = std::max(1, std::min((n + 63) / 64, sm_count() * 16));
    Event e0, e1;
    if (cudaEventCreate(&e0.e) || cudaEventCreate(&e1.e) || cudaEventRecord(e0.e, s)) return -2;
    k_clip_cells<<<blocks, 64, 0, s>>>(d_site.as<double>(), n, d_off.as<int64_t>(), d_nb.as<int32_t>(),
                                       make_double3(dom_lo[0], dom_lo[1], dom_lo[2]),
                                       make_double3(dom_hi[0], dom_hi[1], dom_hi[2]), tol, kMaxClip,
                                       d_slab.as<double>(), d_count.as<int>(), d_state.as<int>());
    if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1.e, s)) return -2;
    // meanwhile, the host clips the cells the kernel hands over at once (more neighbours
    // than the device polytope has planes for)
    const auto th0 = std::chrono::steady_clock::now();
    std::vector<int> host_sites;
    for (int i = 0; i < n; ++i)
        if (nb_off[i + 1] - nb_off[i] > kCellPlanes - 6) host_sites.push_back(i);
    std::vector<std::vector<double>> hc(n);
    const size_t n_early = host_sites.size();
    if (n_early && clip_some(host_sites.data(), (int)n_early, dom_lo, dom_hi, diag, n_threads, hc)) return -1;
    double host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th0).count();
    std::vector<int> cnt(n), state(n);
    if (cudaMemcpyAsync(cnt.data(), d_count.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(state.data(), d_state.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return -2;
    float kms = 0.f;
    cudaEventElapsedTime(&kms, e0.e, e1.e);
    if (ms_kernel) *ms_kernel = kms;
    // the few cells that overflowed the device polytope or met a degenerate cut
    const auto th1 = std::chrono::steady_clock::now();
    std::vector<int> late;
    for (int i = 0; i < n; ++i) {
        if (state[i] == CELL_EMPTY) return -1;
        if (state[i] == CELL_HOST && hc[i].empty()) late.push_back(i);
    }
    if (!late.empty() && clip_some(late.data(), (int)late.size(), dom_lo, dom_hi, diag, n_threads, hc)) return -1;
    host_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - th1).count();
    if (ms_host) *ms_host = host_ms;
    // final CSR: the device corners are packed into their slots on the device and copied
    // once; the host cells fill the rest
    cell_off.assign(n + 1, 0);
    for (int i = 0; i < n; ++i)
        cell_off[i + 1] = cell_off[i] + (state[i] == CELL_OK ? cnt[i] : (int64_t)(hc[i].size() / 3));
    cell_xyz.resize(3 * (size_t)cell_off[n]);
    if (cell_off[n] > 0) {
        if (d_corner.alloc(sizeof(double) * 3 * cell_off[n]) ||
            cudaMemcpyAsync(d_coff.p, cell_off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s))
            return -2;
        k_pack_corners<<<std::max(1, std::min(n, sm_count() * 32)), 128, 0, s>>>(d_slab.as<double>(), d_count.as<int>(),
                                                                         d_coff.as<int64_t>(), n, d_corner.as<double>());
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(cell_xyz.data(), d_corner.p, sizeof(double) * cell_xyz.size(), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s))
            return -2;
    }
    for (int i = 0; i < n; ++i)
        if (state[i] != CELL_OK && !hc[i].empty())
            std::memcpy(&cell_xyz[3 * (size_t)cell_off[i]], hc[i].data(), sizeof(double) * hc[i].size());
    if (n_host) *n_host = (int64_t)(n_early + late.size());
    return 0;
}

// The augmentation's binning (Section 3.2) on the device: each Voronoi vertex inside D (world
// coordinates w[n][3]) falls into tau-cell (floor((w - lo) / tau)) with key (cz * ncy + cy) *
// ncx + cx; vertices outside D get the key ncx * ncy * ncz and sort last.  A radix sort and a
// run-length encoding give the occupied cells' keys (ascending) and their vertex counts.
__global__ void k_bin_keys(const double* __restrict__ w, int64_t n, double3 lo, double3 hi, double tau, int64_t ncx,
                           int64_t ncy, unsigned long long top, unsigned long long* __restrict__ key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[3 * i], y = w[3 * i + 1], z = w[3 * i + 2];
        const bool in = x >= lo.x && x <= hi.x && y >= lo.y && y <= hi.y && z >= lo.z && z <= hi.z;
        unsigned long long k = top;
        if (in) {
            const int64_t cx = (int64_t)floor((x - lo.x) / tau), cy = (int64_t)floor((y - lo.y) / tau),
                          cz = (int64_t)floor((z - lo.z) / tau);
            k = (unsigned long long)((cz * ncy + cy) * ncx + cx);
        }
        key[i] = k;
    }
}

int bin_points_gpu(const std::vector<double>& w, const double lo[3], const double hi[3], double tau,
                   const int64_t ncell[3], std::vector<uint64_t>& keys, std::vector<int>& counts, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    keys.clear();
    counts.clear();
    const int64_t n = (int64_t)(w.size() / 3);
    if (n == 0) return 0;
    if (n > 0x7fffffffLL) return -1;
    // every key of a cell inside D is below ncx * ncy * ncz (each coordinate stays below its
    // axis count: the counts carry two cells of margin over the extent / tau)
    const unsigned long long top = (unsigned long long)(ncell[0] * ncell[1] * ncell[2]);
    int bits = 1;
    while (bits < 64 && (top >> bits) != 0) ++bits;
    DevBuf d_w, d_k0, d_k1, d_uniq, d_cnt, d_runs, d_tmp;
    size_t t_sort = 0, t_rle = 0;
    if (cub::DeviceRadixSort::SortKeys(nullptr, t_sort, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                       (int)n, 0, bits, s) ||
        cub::DeviceRunLengthEncode::Encode(nullptr, t_rle, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                           (int*)nullptr, (int*)nullptr, (int)n, s))
        return -1;
    if (d_w.alloc(sizeof(double) * w.size()) || d_k0.alloc(sizeof(unsigned long long) * n) ||
        d_k1.alloc(sizeof(unsigned long long) * n) || d_uniq.alloc(sizeof(unsigned long long) * n) ||
        d_cnt.alloc(sizeof(int) * n) || d_runs.alloc(sizeof(int)) || d_tmp.alloc(std::max(t_sort, t_rle) + 16))
        return -1;
    if (cudaMemcpyAsync(d_w.p, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, s)) return -1;
    k_bin_keys<<<(int)std::min<int64_t>((n + 255) / 256, sm_count() * 16), 256, 0, s>>>(
        d_w.as<double>(), n, make_double3(lo[0], lo[1], lo[2]), make_double3(hi[0], hi[1], hi[2]), tau, ncell[0],
        ncell[1], top, d_k0.as<unsigned long long>());
    if (cudaGetLastError() != cudaSuccess) return -1;
    cub::DoubleBuffer<unsigned long long> db(d_k0.as<unsigned long long>(), d_k1.as<unsigned long long>());
    if (cub::DeviceRadixSort::SortKeys(d_tmp.p, t_sort, db, (int)n, 0, bits, s) ||
        cub::DeviceRunLengthEncode::Encode(d_tmp.p, t_rle, db.Current(), d_uniq.as<unsigned long long>(),
                                           d_cnt.as<int>(), d_runs.as<int>(), (int)n, s))
        return -1;
    int runs = 0;
    if (cudaMemcpyAsync(&runs, d_runs.p, sizeof(int), cudaMemcpyDeviceToHost, s) || cudaStreamSynchronize(s)) return -1;
    std::vector<unsigned long long> u(runs);
    counts.resize(runs);
    if (runs > 0 &&
        (cudaMemcpyAsync(u.data(), d_uniq.p, sizeof(unsigned long long) * runs, cudaMemcpyDeviceToHost, s) ||
         cudaMemcpyAsync(counts.data(), d_cnt.p, sizeof(int) * runs, cudaMemcpyDeviceToHost, s) ||
         cudaStreamSynchronize(s)))
        return -1;
    if (runs > 0 && u.back() == top) {  // the vertices outside D
        u.pop_back();
        counts.pop_back();
    }
    keys.assign(u.begin(), u.end());
    return 0;
}

}  // namespace p2m
