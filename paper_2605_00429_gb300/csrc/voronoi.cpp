// Host stage of the build: sites on a lattice, their exact Delaunay triangulation, the
// clipped Voronoi cells (FP64) and the corner balls of Eq. 3 / Eq. 8.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "host_geom.h"
#include "p2m_internal.h"
#include "voronoi.h"

namespace p2m {

static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t morton_key(const IPt& p, int64_t R) {
    auto spread = [](uint64_t v) {
        v &= 0x1fffff;
        v = (v | v << 32) & 0x1f00000000ffffull;
        v = (v | v << 16) & 0x1f0000ff0000ffull;
        v = (v | v << 8) & 0x100f00f00f00f00full;
        v = (v | v << 4) & 0x10c30c30c30c30c3ull;
        v = (v | v << 2) & 0x1249249249249249ull;
        return v;
    };
    return (spread((uint64_t)(p.x + R)) << 2) | (spread((uint64_t)(p.y + R)) << 1) | spread((uint64_t)(p.z + R));
}

void SiteSet::world(int i, double out[3]) const { lat.to_world(pts[i], out); }

int hardware_threads();

// Insert sites [first, pts.size()) into the triangulation in a biased randomized insertion
// order (Amenta, Choi and Rote 2003): each site draws a round, the last round holding about
// half of them, the one before a quarter, and so on; within a round the sites go in Morton
// order.  A pure Morton order sweeps the sites of a surface mesh in space, and the
// triangulation's open front then carries long tetrahedra with huge circumspheres that each
// new site must cut away.  A site whose insertion fails (flat tetrahedron or exact duplicate)
// is moved by one lattice step.
int SiteSet::triangulate_from(int first, uint64_t seed, std::string& err) {
    std::vector<std::pair<uint64_t, int>> order;
    uint64_t rr = mix64(seed ^ 0xb410ull);
    for (int i = first; i < (int)pts.size(); ++i) {
        // round = number of leading one bits of a random word, capped: P(round k) = 2^-(k+1),
        // reversed so that the big rounds come last
        rr = mix64(rr);
        int k = 0;
        while (k < 20 && ((rr >> k) & 1u)) ++k;
        const uint64_t round = (uint64_t)(20 - k);
        order.push_back({(round << 58) | (morton_key(pts[i], lat.R) >> 6), i});
    }
    std::sort(order.begin(), order.end());
    uint64_t rng = mix64(seed ^ 0x5eedull);
    vid.resize(pts.size(), -1);
    for (auto& o : order) {
        const int i = o.second;
        int tries = 0;
        while (true) {
            const int r = inject_fault("delaunay") ? INSERT_BROKEN : dt.insert(pts[i], rng);
            if (r >= 0) { vid[i] = r; break; }
            if (r == INSERT_BROKEN) { err = "Delaunay insertion broke the triangulation"; return -1; }
            if (++tries > 64) { err = "could not place a site after 64 jitters"; return -1; }
            rng = mix64(rng);
            IPt p = pts[i];
            p.x += (int64_t)(rng % 3) - 1;
            p.y += (int64_t)((rng >> 8) % 3) - 1;
            p.z += (int64_t)((rng >> 16) % 3) - 1;
            if (lat.inside(p)) pts[i] = p;
        }
    }
    return 0;
}

void SiteSet::neighbour_csr() {
    // Delaunay vertex ids are 4 + insertion position; map them back to site ids
    std::vector<int> site_of(dt.pts.size(), -1);
    for (int i = 0; i < (int)vid.size(); ++i) site_of[vid[i]] = i;
    std::vector<int64_t> off;
    std::vector<int32_t> nb;
    dt.neighbours((int)dt.pts.size() - dt.n_super, off, nb, hardware_threads());
    const int n = (int)pts.size();
    const int nv = (int)dt.pts.size() - dt.n_super;
    // CSR over sites straight from the CSR over Delaunay vertices
    nb_off.assign(n + 1, 0);
    for (int v = 0; v < nv; ++v) {
        const int s = site_of[v + dt.n_super];
        if (s < 0) continue;
        int64_t c = 0;
        for (int64_t k = off[v]; k < off[v + 1]; ++k) c += site_of[nb[k] + dt.n_super] >= 0;
        nb_off[s + 1] = c;
    }
    for (int s = 0; s < n; ++s) nb_off[s + 1] += nb_off[s];
    nb_id.assign(nb_off[n], 0);
    for (int v = 0; v < nv; ++v) {
        const int s = site_of[v + dt.n_super];
        if (s < 0) continue;
        int64_t w = nb_off[s];
        for (int64_t k = off[v]; k < off[v + 1]; ++k) {
            const int t = site_of[nb[k] + dt.n_super];
            if (t >= 0) nb_id[w++] = t;
        }
    }
    // each site's neighbours nearest first (squared distance, then id): the order both cell
    // clippers cut in
    std::atomic<int> next(0);
    auto work = [&]() {
        std::vector<std::pair<double, int>> order;
        while (true) {
            const int s = next.fetch_add(1);
            if (s >= n) break;
            double ps[3];
            world(s, ps);
            order.clear();
            for (int64_t k = nb_off[s]; k < nb_off[s + 1]; ++k) {
                double pt[3];
                world(nb_id[k], pt);
                const double dx = pt[0] - ps[0], dy = pt[1] - ps[1], dz = pt[2] - ps[2];
                order.push_back({dx * dx + dy * dy + dz * dz, nb_id[k]});
            }
            std::sort(order.begin(), order.end());
            for (size_t k = 0; k < order.size(); ++k) nb_id[nb_off[s] + (int64_t)k] = order[k].second;
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < std::max(1, std::min(hardware_threads(), n)); ++t) th.emplace_back(work);
    for (auto& t : th) t.join();
}

// Corners of site s's cell: D cut by the bisectors of its Delaunay neighbours, nearest
// neighbour first (the neighbour lists are kept in that order).  A neighbour t can cut the
// cell only if its bisector, at distance |s - t| / 2 from s, comes within the cell's radius
// about s.  Only bisectors that remove a corner count towards kMaxClip: a fan centre has
// hundreds of near neighbours whose bisectors are all faces (or redundant), and the far
// neighbours that close its cell must still be reached.  After kMaxClip cutting bisectors
// the clip stops, and the cell is then a superset of the true one, which is still a valid
// region for Eq. 3.  Returns false if the cell clipped to nothing.
bool SiteSet::clip_one(int s, const double dom_lo[3], const double dom_hi[3], double tol, Clipper& C) const {
    double ps[3];
    world(s, ps);
    C.box(dom_lo, dom_hi);
    int used = 0;
    for (int64_t k = nb_off[s]; k < nb_off[s + 1]; ++k) {
        double pt[3];
        world(nb_id[k], pt);
        double nrm[3] = {pt[0] - ps[0], pt[1] - ps[1], pt[2] - ps[2]};
        const double d2 = nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2];
        if (0.25 * d2 > C.radius2_from(ps) * (1.0 + 1e-9) + tol * tol) break;
        const double len = std::sqrt(d2);
        if (!(len > 0)) continue;
        for (double& c : nrm) c /= len;
        const double d = 0.5 * (nrm[0] * (pt[0] + ps[0]) + nrm[1] * (pt[1] + ps[1]) + nrm[2] * (pt[2] + ps[2]));
        if (!C.clip(nrm, d, tol)) return false;
        if (C.cut && ++used >= kMaxClip) break;
    }
    return true;
}

// The cells of all sites (or of the listed ones: `only`), threads splitting the sites.
int SiteSet::clip_cells(const double dom_lo[3], const double dom_hi[3], double diag, int n_threads) {
    const int n = (int)pts.size();
    std::vector<std::vector<double>> corners(n);
    if (clip_some(nullptr, n, dom_lo, dom_hi, diag, n_threads, corners)) return -1;
    cell_off.assign(n + 1, 0);
    for (int s = 0; s < n; ++s) cell_off[s + 1] = cell_off[s] + (int64_t)(corners[s].size() / 3);
    cell_xyz.resize(cell_off[n] * 3);
    for (int s = 0; s < n; ++s) std::copy(corners[s].begin(), corners[s].end(), cell_xyz.begin() + cell_off[s] * 3);
    return 0;
}

int SiteSet::clip_some(const int* only, int count, const double dom_lo[3], const double dom_hi[3], double diag,
                       int n_threads, std::vector<std::vector<double>>& corners) const {
    std::atomic<int> next(0), bad(0);
    const double tol = clip_tol(diag);
    auto work = [&]() {
        Clipper C;
        while (true) {
            const int k = next.fetch_add(1);
            if (k >= count) break;
            const int s = only ? only[k] : k;
            if (!clip_one(s, dom_lo, dom_hi, tol, C)) {
                bad.fetch_add(1);
                continue;
            }
            corners[s] = C.V;
        }
    };
    std::vector<std::thread> th;
    for (int t = 0; t < std::max(1, std::min(n_threads, count)); ++t) th.emplace_back(work);
    for (auto& t : th) t.join();
    return bad.load() ? -1 : 0;
}

int hardware_threads() {
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h, 64u));
}

}  // namespace p2m
