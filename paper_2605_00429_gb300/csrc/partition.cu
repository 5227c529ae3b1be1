// Build of the site partition and of everything the query reads besides the triangles:
//   sites (Section 3.1: mesh vertices as proxy sites), their exact Delaunay triangulation,
//   ring-based augmentation (Section 3.2), clipped Voronoi cells, the corner balls of Eq. 3
//   and Eq. 8, the interception lists (K1, lists.cu) and the nearest-site grid (K2a,
//   grid.cu).
#include <algorithm>
#include <thread>
#include <atomic>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "host.h"
#include "host_geom.h"
#include "voronoi.h"

namespace p2m {

int build_lists(MeshData& m, const float4* d_balls, const int64_t* d_ball_off, int n_sites, unsigned* status,
                cudaStream_t s);
int build_grid(MeshData& m, const SiteSet& ss, int G, unsigned* status, cudaStream_t s);

static double ms_now() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// FP64 closest point of a triangle (host; the same parametrisation as the device routine).
static void closest_on_tri_f64(const double q[3], const double a[3], const double b[3], const double c[3], double p[3]) {
    double e0[3], e1[3], w[3], n[3];
    for (int k = 0; k < 3; ++k) { e0[k] = b[k] - a[k]; e1[k] = c[k] - a[k]; w[k] = q[k] - a[k]; }
    n[0] = e0[1] * e1[2] - e0[2] * e1[1]; n[1] = e0[2] * e1[0] - e0[0] * e1[2]; n[2] = e0[0] * e1[1] - e0[1] * e1[0];
    const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    auto dot = [](const double* x, const double* y) { return x[0] * y[0] + x[1] * y[1] + x[2] * y[2]; };
    if (nn > 0) {
        double wx1[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2], w[0] * e1[1] - w[1] * e1[0]};
        double e0xw[3] = {e0[1] * w[2] - e0[2] * w[1], e0[2] * w[0] - e0[0] * w[2], e0[0] * w[1] - e0[1] * w[0]};
        const double s = dot(wx1, n) / nn, t = dot(e0xw, n) / nn;
        if (s >= 0 && t >= 0 && s + t <= 1) {
            for (int k = 0; k < 3; ++k) p[k] = a[k] + s * e0[k] + t * e1[k];
            return;
        }
    }
    const double* A[3] = {a, a, b};
    const double* B[3] = {b, c, c};
    double best = 1e300;
    for (int e = 0; e < 3; ++e) {
        double d[3], r[3];
        for (int k = 0; k < 3; ++k) { d[k] = B[e][k] - A[e][k]; r[k] = q[k] - A[e][k]; }
        const double l = dot(d, d);
        double u = l > 0 ? dot(r, d) / l : 0.0;
        u = std::min(1.0, std::max(0.0, u));
        double x[3];
        for (int k = 0; k < 3; ++k) x[k] = A[e][k] + u * d[k];
        const double dd = (q[0] - x[0]) * (q[0] - x[0]) + (q[1] - x[1]) * (q[1] - x[1]) + (q[2] - x[2]) * (q[2] - x[2]);
        if (dd < best) { best = dd; p[0] = x[0]; p[1] = x[1]; p[2] = x[2]; }
    }
}

// Unit directions of the auxiliary ring: icosahedron (12) or octahedron (6) vertices.
static std::vector<double> ring_dirs(int n) {
    std::vector<double> d;
    if (n == 6) {
        d = {1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1};
        return d;
    }
    const double t = (1.0 + std::sqrt(5.0)) / 2.0, s = 1.0 / std::sqrt(1.0 + t * t);
    const double v[12][3] = {{-1, t, 0}, {1, t, 0}, {-1, -t, 0}, {1, -t, 0}, {0, -1, t}, {0, 1, t},
                             {0, -1, -t}, {0, 1, -t}, {t, 0, -1}, {t, 0, 1}, {-t, 0, -1}, {-t, 0, 1}};
    for (auto& p : v)
        for (int k = 0; k < 3; ++k) d.push_back(p[k] * s);
    return d;
}

// Spatial hash of points for "is any point within r of x" checks on the host.
struct PointHash {
    double cell;
    std::unordered_map<uint64_t, std::vector<int>> m;
    std::vector<double> P;
    static uint64_t key(int64_t x, int64_t y, int64_t z) {
        return ((uint64_t)(x & 0x1fffff) << 42) | ((uint64_t)(y & 0x1fffff) << 21) | (uint64_t)(z & 0x1fffff);
    }
    void add(const double p[3]) {
        const int id = (int)(P.size() / 3);
        P.insert(P.end(), p, p + 3);
        m[key((int64_t)std::floor(p[0] / cell), (int64_t)std::floor(p[1] / cell), (int64_t)std::floor(p[2] / cell))]
            .push_back(id);
    }
    bool near(const double p[3], double r) const {
        const int64_t cx = (int64_t)std::floor(p[0] / cell), cy = (int64_t)std::floor(p[1] / cell),
                      cz = (int64_t)std::floor(p[2] / cell);
        const int64_t k = (int64_t)std::ceil(r / cell);
        for (int64_t dx = -k; dx <= k; ++dx)
            for (int64_t dy = -k; dy <= k; ++dy)
                for (int64_t dz = -k; dz <= k; ++dz) {
                    auto it = m.find(key(cx + dx, cy + dy, cz + dz));
                    if (it == m.end()) continue;
                    for (int id : it->second) {
                        const double* q = &P[3 * id];
                        const double d2 = (q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) + (q[2] - p[2]) * (q[2] - p[2]);
                        if (d2 < r * r) return true;
                    }
                }
        return false;
    }
};

// Section 3.2: bin the Voronoi vertices into a tau-grid, flag dense cells, and add a centre
// site p_c (the centroid of the cell's Voronoi vertices, or the cell's centre) plus a ring
// of auxiliary sites on a sphere about p_c for each; sites that fall near an existing site,
// and ring sites that fall inside a neighbouring dense cell's ring, are dropped.
// Returns the number of auxiliary sites appended to ss.pts.
static int augment(SiteSet& ss, MeshData& m, const p2m_build_params& prm, int64_t& n_dense, cudaStream_t s) {
    n_dense = 0;
    // tau from the mean edge length
    double sum = 0;
    int64_t ne = 0;
    for (int64_t f = 0; f < m.n_tris; ++f)
        for (int k = 0; k < 3; ++k) {
            const float* a = &m.verts[3 * (int64_t)m.tris[3 * f + k]];
            const float* b = &m.verts[3 * (int64_t)m.tris[3 * f + (k + 1) % 3]];
            sum += std::sqrt((double)(a[0] - b[0]) * (a[0] - b[0]) + (double)(a[1] - b[1]) * (a[1] - b[1]) +
                             (double)(a[2] - b[2]) * (a[2] - b[2]));
            ++ne;
        }
    const double tau = prm.tau_scale * sum / std::max<int64_t>(ne, 1);
    if (!(tau > 0)) return 0;
    // the Voronoi vertices (circumcentres of the Delaunay tetrahedra) in world coordinates
    std::vector<double> cc;
    ss.dt.circumcentres(cc);
    for (size_t i = 0; i + 2 < cc.size(); i += 3)
        for (int k = 0; k < 3; ++k) cc[i + k] = (cc[i + k] + (double)ss.lat.c[k]) * ss.lat.h;
    // tau-cells per axis; a cell's key is (cz * ncy + cy) * ncx + cx
    int64_t ncell[3];
    for (int k = 0; k < 3; ++k) ncell[k] = (int64_t)std::ceil((m.dom_hi[k] - m.dom_lo[k]) / tau) + 2;
    const int64_t ncx = ncell[0], ncy = ncell[1];
    // occupied tau-cells and their vertex counts: binned on the device, or on the host
    std::vector<uint64_t> cell_key;
    std::vector<int> cell_count;
    if (prm.gpu_cells) {
        if (bin_points_gpu(cc, m.dom_lo, m.dom_hi, tau, ncell, cell_key, cell_count, s))
            return fail(P2M_ERR_CUDA, "device binning of the Voronoi vertices failed");
    } else {
        std::unordered_map<uint64_t, int> count;
        for (size_t i = 0; i + 2 < cc.size(); i += 3) {
            const double* w = &cc[i];
            bool in = true;
            for (int k = 0; k < 3; ++k) in &= w[k] >= m.dom_lo[k] && w[k] <= m.dom_hi[k];
            if (!in) continue;
            int64_t c[3];
            for (int k = 0; k < 3; ++k) c[k] = (int64_t)std::floor((w[k] - m.dom_lo[k]) / tau);
            count[(uint64_t)((c[2] * ncy + c[1]) * ncx + c[0])]++;
        }
        for (auto& kv : count) {
            cell_key.push_back(kv.first);
            cell_count.push_back(kv.second);
        }
    }
    if (cell_key.empty()) return 0;
    std::vector<int> vals(cell_count);
    std::nth_element(vals.begin(), vals.begin() + vals.size() / 2, vals.end());
    const double median = vals[vals.size() / 2];
    m.stats.aug_cell_median = (int64_t)median;
    m.stats.aug_cell_max = *std::max_element(vals.begin(), vals.end());
    const double thresh = std::max((double)prm.density_min, prm.density_factor * median);
    // dense cells: (geometric centre of the tau-cell, position of p_c)
    std::unordered_map<uint64_t, int> dense_id;
    std::vector<std::array<double, 6>> dense;
    for (size_t j = 0; j < cell_key.size(); ++j) {
        if (cell_count[j] <= thresh) continue;
        const uint64_t k = cell_key[j];
        const int64_t cx = (int64_t)(k % ncx), cy = (int64_t)((k / ncx) % ncy), cz = (int64_t)(k / ((uint64_t)ncx * ncy));
        const double g[3] = {m.dom_lo[0] + (cx + 0.5) * tau, m.dom_lo[1] + (cy + 0.5) * tau,
                             m.dom_lo[2] + (cz + 0.5) * tau};
        dense_id[k] = (int)dense.size();
        dense.push_back({g[0], g[1], g[2], g[0], g[1], g[2]});
    }
    n_dense = (int64_t)dense.size();
    if (dense.empty()) return 0;
    if (prm.aux_centre) {
        // p_c at the centroid of the Voronoi vertices the cell holds (the same binning as above)
        std::vector<double> sum(4 * dense.size(), 0.0);
        for (size_t i = 0; i + 2 < cc.size(); i += 3) {
            const double* w = &cc[i];
            bool in = true;
            for (int k = 0; k < 3; ++k) in &= w[k] >= m.dom_lo[k] && w[k] <= m.dom_hi[k];
            if (!in) continue;
            int64_t c[3];
            for (int k = 0; k < 3; ++k) c[k] = (int64_t)std::floor((w[k] - m.dom_lo[k]) / tau);
            auto it = dense_id.find((uint64_t)((c[2] * ncy + c[1]) * ncx + c[0]));
            if (it == dense_id.end()) continue;
            double* sm = &sum[4 * (size_t)it->second];
            for (int k = 0; k < 3; ++k) sm[k] += w[k];
            sm[3] += 1.0;
        }
        for (size_t j = 0; j < dense.size(); ++j)
            if (sum[4 * j + 3] > 0)
                for (int k = 0; k < 3; ++k) dense[j][3 + k] = sum[4 * j + k] / sum[4 * j + 3];
    }
    std::sort(dense.begin(), dense.end());
    PointHash sites;
    sites.cell = std::max(tau, 1e-30);
    for (int i = 0; i < (int)ss.pts.size(); ++i) {
        double w[3];
        ss.world(i, w);
        sites.add(w);
    }
    PointHash flagged;
    flagged.cell = tau;
    for (auto& c : dense) flagged.add(c.data());
    const double ring_r = prm.ring_radius_scale * tau;
    const double bound_r = 0.5 * std::sqrt(3.0) * tau;  // a flagged cell's bounding sphere
    const std::vector<double> dirs = ring_dirs(prm.ring_sites);
    int added = 0;
    auto try_add = [&](const double* p) {
        bool in = true;
        for (int k = 0; k < 3; ++k) in &= p[k] > m.dom_lo[k] && p[k] < m.dom_hi[k];
        if (!in || sites.near(p, 0.5 * tau)) return false;
        const IPt q = ss.lat.to_lattice(p);
        if (!ss.lat.inside(q)) return false;
        ss.pts.push_back(q);
        sites.add(p);
        ++added;
        return true;
    };
    // the centre sites (a centroid within half a cell of a site already placed is dropped:
    // clusters that straddle cell faces give neighbouring cells nearly the same centroid)
    std::vector<char> placed(dense.size(), 0);
    PointHash centres;
    centres.cell = std::max(ring_r, 1e-30);
    for (size_t j = 0; j < dense.size(); ++j)
        if (try_add(dense[j].data() + 3)) {
            placed[j] = 1;
            centres.add(dense[j].data() + 3);
        }
    for (size_t j = 0; j < dense.size(); ++j) {
        const auto& c = dense[j];
        // with the cells' centres, a ring site inside another flagged cell's bounding sphere is
        // dropped; with centroids, a ring site closer to another centre site than the ring
        // radius is (it lies inside that site's ring).  Either way the rings of adjacent dense
        // cells merge into one around them.
        if (prm.aux_centre && !placed[j]) continue;
        for (size_t d = 0; d < dirs.size(); d += 3) {
            const double p[3] = {c[3] + ring_r * dirs[d], c[4] + ring_r * dirs[d + 1], c[5] + ring_r * dirs[d + 2]};
            if (prm.aux_centre ? centres.near(p, ring_r * (1.0 - 1e-6)) : flagged.near(p, bound_r)) continue;
            try_add(p);
        }
    }
    return added;
}

// At most this many balls per site (4 per lane of the K1 warp); only cells that reach a
// degenerate region (fan centres, symmetry axes) have more corners than this.
constexpr int kMaxBalls = 128;

int build_partition(MeshData& m, const p2m_build_params& prm, p2m_index* h, cudaStream_t s) {
    p2m_stats& st = m.stats;
    unsigned* status = index_status(h);
    double t0 = ms_now();
    SiteSet ss;
    if (!ss.lat.setup(m.dom_lo, m.dom_hi)) return fail(P2M_ERR_DEGENERATE, "domain lattice setup failed");
    // vertex sites: referenced vertices, merged when they share a lattice point
    std::vector<char> used(m.n_verts, 0);
    for (int64_t i = 0; i < m.n_tris * 3; ++i) used[m.tris[i]] = 1;
    std::vector<std::pair<std::array<int64_t, 3>, int>> lv;
    for (int64_t i = 0; i < m.n_verts; ++i) {
        if (!used[i]) continue;
        const double p[3] = {m.verts[3 * i], m.verts[3 * i + 1], m.verts[3 * i + 2]};
        const IPt q = ss.lat.to_lattice(p);
        lv.push_back({{q.x, q.y, q.z}, (int)i});
    }
    std::sort(lv.begin(), lv.end());
    std::vector<int> ref_vertex;
    uint64_t rng = mix64((uint64_t)prm.seed * 0x100000001b3ull + 17);
    for (size_t i = 0; i < lv.size(); ++i) {
        if (i > 0 && lv[i].first == lv[i - 1].first) continue;
        IPt q{lv[i].first[0], lv[i].first[1], lv[i].first[2]};
        // one lattice step of jitter breaks the exact co-planarity / co-sphericity of
        // symmetric meshes; a site is only a partition generator, so any nearby point works
        rng = mix64(rng);
        q.x += (int64_t)(rng % 3) - 1;
        q.y += (int64_t)((rng >> 8) % 3) - 1;
        q.z += (int64_t)((rng >> 16) % 3) - 1;
        ss.pts.push_back(q);
        ref_vertex.push_back(lv[i].second);
    }
    const int n_vsites = (int)ss.pts.size();
    if (n_vsites < 4) {
        // too few sites for a 3D partition: every query takes the exact BVH search
        m.G = 0;
        return P2M_OK;
    }
    std::string err;
    ss.dt.init(ss.lat.R);
    if (ss.triangulate_from(0, (uint64_t)prm.seed, err)) return fail(P2M_ERR_INTERNAL, err);
    if (ss.dt.count_real_tets() == 0) return fail(P2M_ERR_DEGENERATE, "all sites are coplanar");
    double t1 = ms_now();
    st.ms_delaunay = t1 - t0;
    int n_aux = 0;
    int64_t n_dense = 0;
    if (prm.enable_aux) {
        n_aux = augment(ss, m, prm, n_dense, s);
        if (n_aux < 0) return n_aux;
        if (n_aux > 0) {
            // triangulate all sites again in one Morton order: inserting the auxiliary sites
            // into the finished triangulation would open very large cavities around the
            // degenerate interior tetrahedra they are meant to break up
            ss.dt.init(ss.lat.R);
            ss.vid.clear();
            if (ss.triangulate_from(0, (uint64_t)prm.seed + 1, err)) return fail(P2M_ERR_INTERNAL, err);
        }
    }
    double t2 = ms_now();
    st.ms_aug = t2 - t1;
    st.n_dense_cells = n_dense;
    st.n_delaunay_tets = ss.dt.count_real_tets();
    ss.neighbour_csr();  // the Delaunay adjacency, nearest first: counted with the triangulation
    st.ms_delaunay += ms_now() - t2;
    t2 = ms_now();
    if (prm.gpu_cells) {
        int64_t n_host = 0;
        const int rc = ss.clip_cells_gpu(m.dom_lo, m.dom_hi, m.diag, hardware_threads(), s, &n_host,
                                         &st.ms_cells_kernel, &st.ms_cells_fallback);
        if (rc == -2) return fail(P2M_ERR_CUDA, "device cell clipping failed");
        if (rc) return fail(P2M_ERR_INTERNAL, "a Voronoi cell clipped to nothing");
        st.n_cells_host = n_host;
    } else if (ss.clip_cells(m.dom_lo, m.dom_hi, m.diag, hardware_threads())) {
        return fail(P2M_ERR_INTERNAL, "a Voronoi cell clipped to nothing");
    }
    double t3 = ms_now();
    st.ms_cells = t3 - t2;
    const int S = (int)ss.pts.size();
    st.n_sites = S;
    st.n_vertex_sites = n_vsites;
    st.n_aux_sites = S - n_vsites;
    // site positions (FP32-exact) and reference points
    m.site_pos.resize(3 * S);
    m.site_ref.resize(3 * S);
    m.site_kind.assign(S, 0);
    for (int i = 0; i < S; ++i) {
        double w[3];
        ss.world(i, w);
        for (int k = 0; k < 3; ++k) m.site_pos[3 * i + k] = (float)w[k];
        if (i < n_vsites) {
            for (int k = 0; k < 3; ++k) m.site_ref[3 * i + k] = (double)m.verts[3 * (int64_t)ref_vertex[i] + k];
        } else {
            m.site_kind[i] = 1;
        }
    }
    P2M_TRY(m.d_sites.alloc(sizeof(float4) * S));
    {
        std::vector<float4> sp(S);
        for (int i = 0; i < S; ++i) sp[i] = make_float4(m.site_pos[3 * i], m.site_pos[3 * i + 1], m.site_pos[3 * i + 2], 0.f);
        P2M_CUDA_TRY(cudaMemcpyAsync(m.d_sites.p, sp.data(), sizeof(float4) * S, cudaMemcpyHostToDevice, s));
        P2M_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // proj(s, M) of the auxiliary sites: exact BVH search on the device, then the closest
    // point recomputed in FP64 on the winning triangle (so it lies on M)
    if (S > n_vsites) {
        const int na = S - n_vsites;
        DevBuf dd, dt;
        P2M_TRY(dd.alloc(sizeof(float) * na));
        P2M_TRY(dt.alloc(sizeof(int32_t) * na));
        DevBuf pts;
        P2M_TRY(pts.alloc(sizeof(float) * 3 * na));
        P2M_CUDA_TRY(cudaMemcpyAsync(pts.p, m.site_pos.data() + 3 * n_vsites, sizeof(float) * 3 * na,
                                     cudaMemcpyHostToDevice, s));
        const MeshView v = m.view();
        P2M_TRY(launch_bvh_closest(v, pts.as<float>(), nullptr, nullptr, na, dd.as<float>(), nullptr, dt.as<int32_t>(),
                                   nullptr, status, s));
        std::vector<int32_t> tri(na);
        P2M_CUDA_TRY(cudaMemcpyAsync(tri.data(), dt.p, sizeof(int32_t) * na, cudaMemcpyDeviceToHost, s));
        P2M_CUDA_TRY(cudaStreamSynchronize(s));
        for (int a = 0; a < na; ++a) {
            const int i = n_vsites + a;
            const int f = tri[a];
            double q[3], A[3], B[3], C[3], p[3];
            for (int k = 0; k < 3; ++k) {
                q[k] = m.site_pos[3 * i + k];
                A[k] = m.verts[3 * (int64_t)m.tris[3 * f] + k];
                B[k] = m.verts[3 * (int64_t)m.tris[3 * f + 1] + k];
                C[k] = m.verts[3 * (int64_t)m.tris[3 * f + 2] + k];
            }
            closest_on_tri_f64(q, A, B, C, p);
            for (int k = 0; k < 3; ++k) m.site_ref[3 * i + k] = p[k];
        }
    }
    double t4 = ms_now();
    st.ms_proj = t4 - t3;
    // reference points for the query's initial bound: FP32 position + its rounding radius
    {
        std::vector<float4> rf(S);
        for (int i = 0; i < S; ++i) {
            const double* r = &m.site_ref[3 * i];
            const float x = (float)r[0], y = (float)r[1], z = (float)r[2];
            const double e = std::sqrt((x - r[0]) * (x - r[0]) + (y - r[1]) * (y - r[1]) + (z - r[2]) * (z - r[2]));
            rf[i] = make_float4(x, y, z, (float)(e * 1.0001 + 1e-30));
        }
        P2M_TRY(m.d_refs.alloc(sizeof(float4) * S));
        P2M_CUDA_TRY(cudaMemcpyAsync(m.d_refs.p, rf.data(), sizeof(float4) * S, cudaMemcpyHostToDevice, s));
        P2M_CUDA_TRY(cudaStreamSynchronize(s));
    }
    // corner balls (Eq. 3; for auxiliary sites with reference point proj(s, M), or Eq. 8's one
    // enclosing ball when aux_balls = 0); a ball contained in
    // another ball of the same site adds nothing to the union and is dropped.  Sites are
    // independent: threads build each site's balls, which are then concatenated in order.
    m.ball_off.assign(S + 1, 0);
    m.ball_c.clear();
    m.ball_r.clear();
    {
        std::vector<std::vector<double>> site_c(S), site_r(S);
        auto site_balls = [&](int i, std::vector<double>& uc, std::vector<double>& ur, std::vector<char>& keep) {
            std::vector<double>& out_c = site_c[i];
            std::vector<double>& out_r = site_r[i];
            const double* v = &m.site_ref[3 * i];
            const int64_t c0 = ss.cell_off[i], c1 = ss.cell_off[i + 1];
            uc.clear();
            ur.clear();
            // a vertex site, or an auxiliary site with per-corner balls: Eq. 3 with reference
            // point v (its vertex, or proj(s, M)); else the single Eq. 8 ball
            if (m.site_kind[i] == 0 || prm.aux_balls) {
                for (int64_t c = c0; c < c1; ++c) {
                    const double* u = &ss.cell_xyz[3 * c];
                    uc.insert(uc.end(), u, u + 3);
                    ur.push_back(std::sqrt((u[0] - v[0]) * (u[0] - v[0]) + (u[1] - v[1]) * (u[1] - v[1]) + (u[2] - v[2]) * (u[2] - v[2])));
                }
                const int nb = (int)ur.size();
                keep.assign(nb, 1);
                for (int a = 0; a < nb; ++a) {
                    for (int b = 0; b < nb && keep[a]; ++b) {
                        if (a == b || !keep[b]) continue;
                        const double dx = uc[3 * a] - uc[3 * b], dy = uc[3 * a + 1] - uc[3 * b + 1], dz = uc[3 * a + 2] - uc[3 * b + 2];
                        const double d = std::sqrt(dx * dx + dy * dy + dz * dz);
                        // a inside b (ties keep the lower index)
                        if (d + ur[a] < ur[b] || (d + ur[a] == ur[b] && b < a)) keep[a] = 0;
                    }
                }
                std::vector<int> kept;
                for (int a = 0; a < nb; ++a)
                    if (keep[a]) kept.push_back(a);
                if ((int)kept.size() <= kMaxBalls) {
                    for (int a : kept) {
                        out_c.insert(out_c.end(), &uc[3 * a], &uc[3 * a] + 3);
                        out_r.push_back(ur[a]);
                    }
                } else {
                    // Too many corners (cells reaching a degenerate region have hundreds):
                    // merge them into kMaxBalls enclosing balls.  Centres are picked by
                    // farthest-point sampling; each corner joins its nearest centre c and
                    // B(u, r) lies inside B(c, |u - c| + r), so the union only grows and the
                    // list stays complete (any convex superset of the cell is valid for Eq. 3).
                    const int k = (int)kept.size();
                    std::vector<int> centre;
                    std::vector<double> dmin(k, 1e300);
                    int pick = 0;
                    for (int a = 1; a < k; ++a)
                        if (ur[kept[a]] > ur[kept[pick]]) pick = a;
                    for (int c = 0; c < kMaxBalls; ++c) {
                        centre.push_back(pick);
                        const double* pc = &uc[3 * kept[pick]];
                        int far = 0;
                        for (int a = 0; a < k; ++a) {
                            const double* pa = &uc[3 * kept[a]];
                            const double d = std::sqrt((pa[0] - pc[0]) * (pa[0] - pc[0]) + (pa[1] - pc[1]) * (pa[1] - pc[1]) +
                                                       (pa[2] - pc[2]) * (pa[2] - pc[2]));
                            dmin[a] = std::min(dmin[a], d);
                            if (dmin[a] > dmin[far]) far = a;
                        }
                        pick = far;
                    }
                    std::vector<double> R(kMaxBalls, 0.0);
                    for (int a = 0; a < k; ++a) {
                        const double* pa = &uc[3 * kept[a]];
                        int best = 0;
                        double bd = 1e300;
                        for (int c = 0; c < kMaxBalls; ++c) {
                            const double* pc = &uc[3 * kept[centre[c]]];
                            const double d = std::sqrt((pa[0] - pc[0]) * (pa[0] - pc[0]) + (pa[1] - pc[1]) * (pa[1] - pc[1]) +
                                                       (pa[2] - pc[2]) * (pa[2] - pc[2]));
                            if (d < bd) { bd = d; best = c; }
                        }
                        R[best] = std::max(R[best], bd + ur[kept[a]]);
                    }
                    for (int c = 0; c < kMaxBalls; ++c) {
                        const double* pc = &uc[3 * kept[centre[c]]];
                        out_c.insert(out_c.end(), pc, pc + 3);
                        out_r.push_back(R[c]);
                    }
                }
            } else {
                double p[3];
                for (int k = 0; k < 3; ++k) p[k] = m.site_pos[3 * i + k];
                double r = 0;
                for (int64_t c = c0; c < c1; ++c) {
                    const double* u = &ss.cell_xyz[3 * c];
                    const double a = std::sqrt((u[0] - p[0]) * (u[0] - p[0]) + (u[1] - p[1]) * (u[1] - p[1]) + (u[2] - p[2]) * (u[2] - p[2]));
                    const double b = std::sqrt((u[0] - v[0]) * (u[0] - v[0]) + (u[1] - v[1]) * (u[1] - v[1]) + (u[2] - v[2]) * (u[2] - v[2]));
                    r = std::max(r, a + b);
                }
                out_c.insert(out_c.end(), p, p + 3);
                out_r.push_back(r);
            }
        };
        std::atomic<int> next(0);
        auto work = [&]() {
            std::vector<double> uc, ur;
            std::vector<char> keep;
            while (true) {
                const int i0 = next.fetch_add(256);
                if (i0 >= S) break;
                for (int i = i0; i < std::min(S, i0 + 256); ++i) site_balls(i, uc, ur, keep);
            }
        };
        std::vector<std::thread> th;
        for (int t = 0; t < std::max(1, std::min(hardware_threads(), (S + 255) / 256)); ++t) th.emplace_back(work);
        for (auto& t : th) t.join();
        for (int i = 0; i < S; ++i) {
            m.ball_c.insert(m.ball_c.end(), site_c[i].begin(), site_c[i].end());
            m.ball_r.insert(m.ball_r.end(), site_r[i].begin(), site_r[i].end());
            m.ball_off[i + 1] = (int64_t)m.ball_r.size();
        }
    }
    const int64_t B = (int64_t)m.ball_r.size();
    st.n_corners = B;
    // FP32 balls for the device: centre rounded, radius inflated by the build slack, the
    // centre's rounding and the FP32 error of the distance test
    {
        std::vector<float4> bf(B);
        const double slack = (double)prm.build_eps_rel * m.diag;
        for (int64_t b = 0; b < B; ++b) {
            const double* u = &m.ball_c[3 * b];
            const float x = (float)u[0], y = (float)u[1], z = (float)u[2];
            const double e = std::sqrt((x - u[0]) * (x - u[0]) + (y - u[1]) * (y - u[1]) + (z - u[2]) * (z - u[2]));
            const double mag = std::max(std::fabs(u[0]), std::max(std::fabs(u[1]), std::fabs(u[2])));
            const double r = (m.ball_r[b] + e + slack + 4.8e-7 * (mag + m.ball_r[b] + m.diag)) * (1.0 + 1e-6);
            bf[b] = make_float4(x, y, z, (float)r);
        }
        DevBuf d_balls, d_boff;
        P2M_TRY(d_balls.alloc(sizeof(float4) * std::max<int64_t>(B, 1)));
        P2M_TRY(d_boff.alloc(sizeof(int64_t) * (S + 1)));
        P2M_CUDA_TRY(cudaMemcpyAsync(d_balls.p, bf.data(), sizeof(float4) * B, cudaMemcpyHostToDevice, s));
        P2M_CUDA_TRY(cudaMemcpyAsync(d_boff.p, m.ball_off.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));
        const double t5 = ms_now();
        P2M_TRY(build_lists(m, d_balls.as<float4>(), d_boff.as<int64_t>(), S, status, s));
        P2M_TRY(check_status_word(h, s, "interception lists"));
        st.ms_k1 = ms_now() - t5;
    }
    // nearest-site grid over D
    {
        const double t6 = ms_now();
        double area = 0;
        for (int64_t f = 0; f < m.n_tris; ++f) {
            const float* a = &m.verts[3 * (int64_t)m.tris[3 * f]];
            const float* b = &m.verts[3 * (int64_t)m.tris[3 * f + 1]];
            const float* c = &m.verts[3 * (int64_t)m.tris[3 * f + 2]];
            const double e0[3] = {(double)b[0] - a[0], (double)b[1] - a[1], (double)b[2] - a[2]};
            const double e1[3] = {(double)c[0] - a[0], (double)c[1] - a[1], (double)c[2] - a[2]};
            const double n[3] = {e0[1] * e1[2] - e0[2] * e1[1], e0[2] * e1[0] - e0[0] * e1[2], e0[0] * e1[1] - e0[1] * e1[0]};
            area += 0.5 * std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        }
        const double spacing = std::sqrt(std::max(area, 1e-300) / std::max(1, n_vsites));
        m.spacing = (float)spacing;
        int G = prm.nn_grid_res;
        if (G <= 0) {
            double ext = 0;
            for (int k = 0; k < 3; ++k) ext = std::max(ext, m.dom_hi[k] - m.dom_lo[k]);
            // finer cells mean fewer candidate sites per query (config 2: 4.4 at 0.8 spacing,
            // 3.7 at 0.68) for a larger grid; the site search is a fifth of a query pass
            G = (int)std::lround(ext / (0.68 * spacing));
            G = std::max(8, std::min(G, 256));
        }
        P2M_TRY(build_grid(m, ss, G, status, s));
        P2M_TRY(check_status_word(h, s, "nearest-site grid"));
        st.ms_grid = ms_now() - t6;
    }
    return P2M_OK;
}

}  // namespace p2m

// ----------------------------------------------------------------------------- host-only API

static int voronoi_cells(const float* h_sites, int64_t n, const double* dom_lo, const double* dom_hi, int seed,
                         float* h_sites_out, int64_t* h_corner_off, double* h_corners, int64_t* n_corners,
                         bool device, int64_t* n_host, void* stream) {
    using namespace p2m;
    if (!h_sites || n < 4 || !dom_lo || !dom_hi || !n_corners) return fail(P2M_ERR_INVALID_ARG, "bad arguments");
    SiteSet ss;
    if (!ss.lat.setup(dom_lo, dom_hi)) return fail(P2M_ERR_INVALID_ARG, "bad domain");
    uint64_t rng = mix64((uint64_t)seed * 0x100000001b3ull + 17);
    for (int64_t i = 0; i < n; ++i) {
        const double p[3] = {h_sites[3 * i], h_sites[3 * i + 1], h_sites[3 * i + 2]};
        IPt q = ss.lat.to_lattice(p);
        rng = mix64(rng);
        q.x += (int64_t)(rng % 3) - 1;
        q.y += (int64_t)((rng >> 8) % 3) - 1;
        q.z += (int64_t)((rng >> 16) % 3) - 1;
        if (!ss.lat.inside(q)) return fail(P2M_ERR_INVALID_ARG, "site outside the domain");
        ss.pts.push_back(q);
    }
    std::string err;
    ss.dt.init(ss.lat.R);
    if (ss.triangulate_from(0, (uint64_t)seed, err)) return fail(P2M_ERR_INTERNAL, err);
    if (ss.dt.validate(false)) return fail(P2M_ERR_INTERNAL, "triangulation failed its self-check");
    ss.neighbour_csr();
    double diag = 0;
    for (int k = 0; k < 3; ++k) diag += (dom_hi[k] - dom_lo[k]) * (dom_hi[k] - dom_lo[k]);
    if (device) {
        const int rc = ss.clip_cells_gpu(dom_lo, dom_hi, std::sqrt(diag), hardware_threads(), stream, n_host);
        if (rc == -2) return fail(P2M_ERR_CUDA, "device cell clipping failed");
        if (rc) return fail(P2M_ERR_INTERNAL, "empty cell");
    } else if (ss.clip_cells(dom_lo, dom_hi, std::sqrt(diag), hardware_threads())) {
        return fail(P2M_ERR_INTERNAL, "empty cell");
    }
    *n_corners = ss.cell_off[n];
    if (h_sites_out)
        for (int64_t i = 0; i < n; ++i) {
            double w[3];
            ss.world((int)i, w);
            for (int k = 0; k < 3; ++k) h_sites_out[3 * i + k] = (float)w[k];
        }
    if (h_corner_off) std::memcpy(h_corner_off, ss.cell_off.data(), sizeof(int64_t) * (n + 1));
    if (h_corners) std::memcpy(h_corners, ss.cell_xyz.data(), sizeof(double) * ss.cell_xyz.size());
    return P2M_OK;
}

extern "C" int p2m_voronoi_cells(const float* h_sites, int64_t n, const double* dom_lo, const double* dom_hi, int seed,
                                 float* h_sites_out, int64_t* h_corner_off, double* h_corners, int64_t* n_corners) {
    return voronoi_cells(h_sites, n, dom_lo, dom_hi, seed, h_sites_out, h_corner_off, h_corners, n_corners, false,
                         nullptr, nullptr);
}

extern "C" int p2m_voronoi_cells_device(const float* h_sites, int64_t n, const double* dom_lo, const double* dom_hi,
                                        int seed, float* h_sites_out, int64_t* h_corner_off, double* h_corners,
                                        int64_t* n_corners, int64_t* n_host, void* stream) {
    return voronoi_cells(h_sites, n, dom_lo, dom_hi, seed, h_sites_out, h_corner_off, h_corners, n_corners, true,
                         n_host, stream);
}
