// Exact incremental 3D Delaunay triangulation (Bowyer-Watson) of integer lattice points.
//
// P2M++ builds the Voronoi diagram of its sites from a Delaunay triangulation (Section 4,
// "CGAL for constructing the Delaunay triangulation"; Section 4.3: the Voronoi build and the
// site search both rely on it).  This is our own triangulator:
//   * points are integers with |x| <= 2^19 (the caller quantises; the four vertices of an
//     enclosing tetrahedron sit at up to 12 * 2^19), so every orientation and in-sphere
//     determinant is exact in __int128 (|det| < 2^122);
//   * an exact zero of the in-sphere test (co-spherical points) is resolved by symbolically
//     lifting the newest point slightly above the paraboloid: it is then outside every
//     co-spherical circumsphere, which keeps the cavity consistent;
//   * a new tetrahedron that would be flat (the new point coplanar with a cavity face) makes
//     the insertion report failure before anything changes, so the caller can move the
//     point by one lattice step and retry (the sites are only a partition of space, so any
//     nearby position is valid).
#include "host_geom.h"

#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstring>

namespace p2m {

using i128 = __int128;

static inline int sgn(i128 v) { return (v > 0) - (v < 0); }

// Both predicates first evaluate their determinant in double with a static error bound
// and fall back to exact __int128 arithmetic only when the sign is not certain.  All
// coordinate differences are below 2^24 in magnitude (|x| <= 12 * 2^19), so every 2x2 minor
// below is an exact int64 (< 2^49) and converts to double exactly; the double sums then
// carry a relative error below a few units of 2^-53 of the sum of the absolute terms, and
// the bounds used (2^-50 and 2^-49 of those sums) exceed it with margin.

// orient3d(a,b,c,d) = det[b-a, c-a, d-a]: > 0 if d is on the side of plane (a,b,c) that the
// normal (b-a) x (c-a) points to.
static inline int orient3d(const IPt& a, const IPt& b, const IPt& c, const IPt& d) {
    const int64_t bx = b.x - a.x, by = b.y - a.y, bz = b.z - a.z;
    const int64_t cx = c.x - a.x, cy = c.y - a.y, cz = c.z - a.z;
    const int64_t dx = d.x - a.x, dy = d.y - a.y, dz = d.z - a.z;
    const int64_t m0 = cy * dz - cz * dy;
    const int64_t m1 = cz * dx - cx * dz;
    const int64_t m2 = cx * dy - cy * dx;
    const double p0 = (double)bx * (double)m0, p1 = (double)by * (double)m1, p2 = (double)bz * (double)m2;
    const double det = p0 + p1 + p2;
    const double bound = (std::fabs(p0) + std::fabs(p1) + std::fabs(p2)) * 0x1p-50;
    if (det > bound) return 1;
    if (det < -bound) return -1;
    return sgn((i128)bx * m0 + (i128)by * m1 + (i128)bz * m2);
}

// > 0 iff e lies strictly inside the circumsphere of the positively oriented tet (a,b,c,d).
static inline int insphere(const IPt& a, const IPt& b, const IPt& c, const IPt& d, const IPt& e) {
    const int64_t r[4][3] = {{a.x - e.x, a.y - e.y, a.z - e.z}, {b.x - e.x, b.y - e.y, b.z - e.z},
                             {c.x - e.x, c.y - e.y, c.z - e.z}, {d.x - e.x, d.y - e.y, d.z - e.z}};
    int64_t w[4];
    for (int i = 0; i < 4; ++i) w[i] = r[i][0] * r[i][0] + r[i][1] * r[i][1] + r[i][2] * r[i][2];
    // 3x3 minors of the coordinate rows (expansion along the lifted column): the 2x2 minors
    // exactly, the 3x3 value in double with the sum of its absolute terms
    auto m3d = [&](int i, int j, int k, double& perm) -> double {
        const int64_t a0 = r[j][1] * r[k][2] - r[j][2] * r[k][1];
        const int64_t a1 = r[j][2] * r[k][0] - r[j][0] * r[k][2];
        const int64_t a2 = r[j][0] * r[k][1] - r[j][1] * r[k][0];
        const double q0 = (double)r[i][0] * (double)a0, q1 = (double)r[i][1] * (double)a1,
                     q2 = (double)r[i][2] * (double)a2;
        perm = std::fabs(q0) + std::fabs(q1) + std::fabs(q2);
        return q0 + q1 + q2;
    };
    double e0, e1, e2, e3;
    const double n0 = m3d(1, 2, 3, e0), n1 = m3d(0, 2, 3, e1), n2 = m3d(0, 1, 3, e2), n3 = m3d(0, 1, 2, e3);
    const double t0 = (double)w[0] * n0, t1 = (double)w[1] * n1, t2 = (double)w[2] * n2, t3 = (double)w[3] * n3;
    const double detd = -t0 + t1 - t2 + t3;
    const double bound = ((double)w[0] * e0 + (double)w[1] * e1 + (double)w[2] * e2 + (double)w[3] * e3) * 0x1p-49;
    // for a positively oriented tet the determinant is negative for an inside point
    if (detd > bound) return -1;
    if (detd < -bound) return 1;
    auto m3 = [&](int i, int j, int k) -> i128 {
        const i128 a0 = (i128)r[j][1] * r[k][2] - (i128)r[j][2] * r[k][1];
        const i128 a1 = (i128)r[j][2] * r[k][0] - (i128)r[j][0] * r[k][2];
        const i128 a2 = (i128)r[j][0] * r[k][1] - (i128)r[j][1] * r[k][0];
        return (i128)r[i][0] * a0 + (i128)r[i][1] * a1 + (i128)r[i][2] * a2;
    };
    // det of rows (r_i, w_i): sum_i (-1)^(i+3) w_i M_i
    const i128 det = -(i128)w[0] * m3(1, 2, 3) + (i128)w[1] * m3(0, 2, 3) - (i128)w[2] * m3(0, 1, 3) +
                     (i128)w[3] * m3(0, 1, 2);
    return -sgn(det);
}

// Vertex positions (within a tet) of the face opposite vertex i, ordered so that vertex i
// lies on its positive side.
static const int kFace[4][3] = {{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}};

int Delaunay::init(int64_t R) {
    pts.clear();
    tets.clear();
    free_list.clear();
    // Enclosing tetrahedron {x, y, z >= -4R, x + y + z <= 4R}; it holds the cube [-R, R]^3
    // and its vertices are farther from that cube than the cube's diameter.
    const int64_t M = 4 * R;
    pts.push_back({-M, -M, -M});
    pts.push_back({3 * M, -M, -M});
    pts.push_back({-M, 3 * M, -M});
    pts.push_back({-M, -M, 3 * M});
    n_super = 4;
    Tet t;
    t.v[0] = 0; t.v[1] = 1; t.v[2] = 2; t.v[3] = 3;
    if (orient3d(pts[0], pts[1], pts[2], pts[3]) < 0) std::swap(t.v[0], t.v[1]);
    for (int k = 0; k < 4; ++k) t.n[k] = -1;
    t.alive = 1;
    tets.push_back(t);
    last = 0;
    mark.assign(1, 0);
    epoch = 1;
    return 0;
}

int Delaunay::new_tet() {
    if (!free_list.empty()) {
        int t = free_list.back();
        free_list.pop_back();
        return t;
    }
    tets.push_back(Tet());
    mark.push_back(0);
    return (int)tets.size() - 1;
}

bool Delaunay::conflict(int t, const IPt& q) const {
    const Tet& T = tets[t];
    return insphere(pts[T.v[0]], pts[T.v[1]], pts[T.v[2]], pts[T.v[3]], q) > 0;
}

// Visibility walk to a tetrahedron containing q (exact orientations).
int Delaunay::locate(const IPt& q, uint64_t& rng) const {
    int t = last;
    if (t < 0 || t >= (int)tets.size() || !tets[t].alive) {
        t = -1;
        for (int i = (int)tets.size() - 1; i >= 0; --i)
            if (tets[i].alive) { t = i; break; }
    }
    const int64_t cap = 4 * (int64_t)tets.size() + 64;
    for (int64_t step = 0; step < cap; ++step) {
        const Tet& T = tets[t];
        rng = rng * 6364136223846793005ull + 1442695040888963407ull;
        const int start = (int)((rng >> 33) & 3);
        int next = -1;
        for (int h = 0; h < 4; ++h) {
            const int i = (start + h) & 3;
            const int* f = kFace[i];
            if (orient3d(pts[T.v[f[0]]], pts[T.v[f[1]]], pts[T.v[f[2]]], q) < 0) {
                next = T.n[i];
                break;
            }
        }
        if (next < 0) return t;  // inside (or outside the hull: cannot happen inside the super tet)
        t = next;
    }
    return -1;
}

int Delaunay::insert(const IPt& q, uint64_t& rng) {
    int seed = locate(q, rng);
    if (seed < 0 || !conflict(seed, q)) {
        // walk failed or q duplicates a vertex of its tet: search any conflicting tet
        seed = -1;
        for (int i = 0; i < (int)tets.size(); ++i) {
            if (tets[i].alive && conflict(i, q)) { seed = i; break; }
        }
        if (seed < 0) return INSERT_DUPLICATE;
    }
    // cavity: all tets whose circumsphere strictly contains q (connected, star-shaped)
    if (++epoch == 0) { std::fill(mark.begin(), mark.end(), 0u); epoch = 1; }
    cavity.clear();
    boundary.clear();
    stack.clear();
    stack.push_back(seed);
    mark[seed] = epoch;
    while (!stack.empty()) {
        const int t = stack.back();
        stack.pop_back();
        cavity.push_back(t);
        for (int i = 0; i < 4; ++i) {
            const int nb = tets[t].n[i];
            if (nb >= 0 && mark[nb] == epoch) continue;
            if (nb >= 0 && conflict(nb, q)) {
                mark[nb] = epoch;
                stack.push_back(nb);
            } else {
                boundary.push_back({t, i});
            }
        }
    }
    // every new tet (boundary face, q) must be positively oriented
    for (const auto& b : boundary) {
        const Tet& T = tets[b.first];
        const int* f = kFace[b.second];
        if (orient3d(pts[T.v[f[0]]], pts[T.v[f[1]]], pts[T.v[f[2]]], q) <= 0) return INSERT_FLAT;
    }
    const int qi = (int)pts.size();
    pts.push_back(q);
    // create new tets; the boundary faces keep their outer neighbours
    created.clear();
    for (const auto& b : boundary) {
        const Tet T = tets[b.first];
        const int* f = kFace[b.second];
        const int nt = new_tet();
        Tet& N = tets[nt];
        N.v[0] = T.v[f[0]];
        N.v[1] = T.v[f[1]];
        N.v[2] = T.v[f[2]];
        N.v[3] = qi;
        N.n[0] = N.n[1] = N.n[2] = -1;
        N.n[3] = T.n[b.second];
        N.alive = 1;
        created.push_back(nt);
        const int outer = T.n[b.second];
        if (outer >= 0) {
            Tet& O = tets[outer];
            for (int k = 0; k < 4; ++k)
                if (O.n[k] == b.first) { O.n[k] = nt; break; }
        }
    }
    // kill the cavity (after the outer links are rewired: a cavity tet may be reused)
    for (int t : cavity) {
        tets[t].alive = 0;
        free_list.push_back(t);
    }
    // Note: new_tet() above could not reuse cavity tets because they were freed afterwards.
    // link new tets to each other through their edges on the cavity boundary: every such
    // edge is shared by exactly two new tets.  An open-addressing table keyed by the edge
    // pairs them; its slots carry the insertion's stamp, so nothing is cleared per point.
    const size_t need = 4 * 3 * created.size();
    if (htab.size() < need) {
        size_t sz = 64;
        while (sz < need) sz <<= 1;
        htab.assign(sz, HSlot());
        hstamp = 0;
    }
    if (++hstamp == 0) {
        for (HSlot& h : htab) h.stamp = 0;
        hstamp = 1;
    }
    const size_t mask = htab.size() - 1;
    int open_edges = 0;
    for (int nt : created) {
        const Tet& N = tets[nt];
        for (int k = 0; k < 3; ++k) {
            // face opposite N.v[k] contains q and the edge of the other two base vertices
            const int a = N.v[(k + 1) % 3], b = N.v[(k + 2) % 3];
            const uint64_t key = a < b ? ((uint64_t)a << 32 | (uint32_t)b) : ((uint64_t)b << 32 | (uint32_t)a);
            size_t h = (size_t)((key * 0x9E3779B97F4A7C15ull) >> 32) & mask;
            while (htab[h].stamp == hstamp && htab[h].key != key) h = (h + 1) & mask;
            HSlot& e = htab[h];
            if (e.stamp != hstamp) {
                e = {key, nt, k, hstamp, 1};
                ++open_edges;
            } else {
                if (++e.count > 2) return INSERT_BROKEN;
                tets[e.tet].n[e.face] = nt;
                tets[nt].n[k] = e.tet;
                --open_edges;
            }
        }
    }
    if (open_edges != 0) return INSERT_BROKEN;
    last = created.empty() ? last : created.back();
    return qi;
}

void Delaunay::neighbours(int n_real, std::vector<int64_t>& off, std::vector<int32_t>& nb, int n_threads) const {
    // every live tet lists, for each real vertex, its other real vertices; each vertex's list
    // (with repeats: an edge lies in several tets) is then sorted and deduplicated, threads
    // splitting the vertices.  Ids are shifted by n_super.
    std::vector<int64_t> cnt(n_real + 1, 0);
    for (const Tet& T : tets) {
        if (!T.alive) continue;
        int real = 0;
        for (int i = 0; i < 4; ++i) real += T.v[i] >= n_super;
        for (int i = 0; i < 4; ++i)
            if (T.v[i] >= n_super) cnt[T.v[i] - n_super + 1] += real - 1;
    }
    for (int i = 0; i < n_real; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> all(cnt[n_real]);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (const Tet& T : tets) {
        if (!T.alive) continue;
        for (int i = 0; i < 4; ++i) {
            if (T.v[i] < n_super) continue;
            for (int j = 0; j < 4; ++j)
                if (j != i && T.v[j] >= n_super) all[pos[T.v[i] - n_super]++] = T.v[j] - n_super;
        }
    }
    std::vector<int64_t> len(n_real, 0);
    std::atomic<int> next(0);
    auto work = [&]() {
        while (true) {
            const int v0 = next.fetch_add(1024);
            if (v0 >= n_real) break;
            for (int v = v0; v < std::min(n_real, v0 + 1024); ++v) {
                int32_t* b = all.data() + cnt[v];
                int32_t* e = all.data() + cnt[v + 1];
                std::sort(b, e);
                len[v] = std::unique(b, e) - b;
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < std::max(1, n_threads); ++t) th.emplace_back(work);
    for (auto& t : th) t.join();
    off.assign(n_real + 1, 0);
    for (int v = 0; v < n_real; ++v) off[v + 1] = off[v] + len[v];
    nb.resize(off[n_real]);
    for (int v = 0; v < n_real; ++v) std::copy(all.begin() + cnt[v], all.begin() + cnt[v] + len[v], nb.begin() + off[v]);
}

int64_t Delaunay::count_real_tets() const {
    int64_t c = 0;
    for (const Tet& T : tets)
        if (T.alive && T.v[0] >= n_super && T.v[1] >= n_super && T.v[2] >= n_super && T.v[3] >= n_super) ++c;
    return c;
}

// Circumcentres of the real tetrahedra (FP64, lattice units).
void Delaunay::circumcentres(std::vector<double>& out) const {
    out.clear();
    for (const Tet& T : tets) {
        if (!T.alive || T.v[0] < n_super || T.v[1] < n_super || T.v[2] < n_super || T.v[3] < n_super) continue;
        const IPt& a = pts[T.v[0]];
        double e[3][3];
        for (int k = 0; k < 3; ++k) {
            const IPt& b = pts[T.v[k + 1]];
            e[k][0] = (double)(b.x - a.x); e[k][1] = (double)(b.y - a.y); e[k][2] = (double)(b.z - a.z);
        }
        auto cr = [](const double* u, const double* v, double* o) {
            o[0] = u[1] * v[2] - u[2] * v[1]; o[1] = u[2] * v[0] - u[0] * v[2]; o[2] = u[0] * v[1] - u[1] * v[0];
        };
        double c12[3], c20[3], c01[3];
        cr(e[1], e[2], c12); cr(e[2], e[0], c20); cr(e[0], e[1], c01);
        const double den = 2.0 * (e[0][0] * c12[0] + e[0][1] * c12[1] + e[0][2] * c12[2]);
        if (den == 0.0) continue;
        double l[3];
        for (int k = 0; k < 3; ++k) l[k] = e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2];
        for (int c = 0; c < 3; ++c) {
            const double v = (l[0] * c12[c] + l[1] * c20[c] + l[2] * c01[c]) / den;
            out.push_back(v + (c == 0 ? a.x : c == 1 ? a.y : a.z));
        }
    }
}

// Self-check used by the host tests: every live tet positively oriented, neighbour links
// symmetric, and (if full) no vertex strictly inside any circumsphere.
int Delaunay::validate(bool full) const {
    for (int t = 0; t < (int)tets.size(); ++t) {
        const Tet& T = tets[t];
        if (!T.alive) continue;
        if (orient3d(pts[T.v[0]], pts[T.v[1]], pts[T.v[2]], pts[T.v[3]]) <= 0) return 1;
        for (int i = 0; i < 4; ++i) {
            const int nb = T.n[i];
            if (nb < 0) continue;
            if (!tets[nb].alive) return 2;
            int back = 0;
            for (int k = 0; k < 4; ++k) back += tets[nb].n[k] == t;
            if (back != 1) return 3;
        }
        if (full)
            for (int p = 0; p < (int)pts.size(); ++p) {
                if (p == T.v[0] || p == T.v[1] || p == T.v[2] || p == T.v[3]) continue;
                if (insphere(pts[T.v[0]], pts[T.v[1]], pts[T.v[2]], pts[T.v[3]], pts[p]) > 0) return 4;
            }
    }
    return 0;
}

}  // namespace p2m
