// Host-side geometry of the index build: exact Delaunay triangulation of the sites,
// FP64 Voronoi cell clipping, and site augmentation.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

namespace p2m {

struct IPt {
    int64_t x, y, z;
};

enum { INSERT_DUPLICATE = -1, INSERT_FLAT = -2, INSERT_BROKEN = -3 };

class Delaunay {
public:
    struct Tet {
        int v[4];
        int n[4];  // neighbour opposite v[i], -1 on the enclosing tetrahedron's hull
        int alive = 0;
    };
    std::vector<IPt> pts;  // 4 enclosing vertices first, then inserted points in order
    std::vector<Tet> tets;
    int n_super = 4;

    // Start with the enclosing tetrahedron of the cube [-R, R]^3 (R <= 2^19).
    int init(int64_t R);
    // Insert q; returns its vertex id (>= 4) or INSERT_* on failure (nothing changed for
    // DUPLICATE and FLAT).
    int insert(const IPt& q, uint64_t& rng);
    // Delaunay neighbours of the real points (ids 0..n_real-1 = vertex id - 4), CSR, each
    // list ascending; n_threads threads sort the lists.
    void neighbours(int n_real, std::vector<int64_t>& off, std::vector<int32_t>& nb, int n_threads) const;
    int64_t count_real_tets() const;
    void circumcentres(std::vector<double>& out) const;
    int validate(bool full) const;

private:
    int new_tet();
    bool conflict(int t, const IPt& q) const;
    int locate(const IPt& q, uint64_t& rng) const;
    std::vector<int> free_list, cavity, stack, created;
    std::vector<std::pair<int, int>> boundary;
    std::vector<unsigned> mark;
    unsigned epoch = 1;
    int last = 0;
    struct HSlot {
        uint64_t key = 0;  // cavity-boundary edge (lower vertex id << 32 | higher)
        int tet = 0, face = 0;
        unsigned stamp = 0, count = 0;
    };
    std::vector<HSlot> htab;
    unsigned hstamp = 0;
};

// Convex polytope clipping in FP64: returns the corners of D ∩ {x : (x - m_k) . n_k <= 0}.
struct Clipper {
    std::vector<double> V;                 // xyz
    std::vector<int> fidx, foff;           // faces as cyclic vertex-id lists (CSR)
    void box(const double lo[3], const double hi[3]);
    // keep the half-space n . x <= d; returns false if the polytope became empty.  `cut`
    // tells whether the last call removed a corner.
    bool clip(const double n[3], double d, double tol);
    bool cut = false;
    double radius_from(const double p[3]) const;  // max distance from p to a corner
    double radius2_from(const double p[3]) const;  // its square
    int n_verts() const { return (int)(V.size() / 3); }

private:
    std::vector<double> val, V2;
    std::vector<int> remap, nfidx, nfoff;
    std::vector<std::pair<uint64_t, int>> edge_new;
    std::vector<int> cap;
    std::vector<std::pair<double, int>> ang;
};

// Lattice that maps FP32-exact site positions to small integers: x = (c + k) * h, with
// h a power of two, |k| <= 2^19 over the domain box and |c + k| < 2^24.
struct Lattice {
    double h = 1.0;
    int64_t c[3] = {0, 0, 0};
    int64_t R = 1 << 19;
    bool setup(const double dom_lo[3], const double dom_hi[3]);
    IPt to_lattice(const double p[3]) const;  // rounds to the nearest lattice point, relative to c
    void to_world(const IPt& k, double out[3]) const;
    bool inside(const IPt& k) const { return k.x >= -R && k.x <= R && k.y >= -R && k.y <= R && k.z >= -R && k.z <= R; }
};

}  // namespace p2m
