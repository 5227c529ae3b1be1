// The site set of one mesh and its Voronoi cells (host).
#pragma once

#include <string>
#include <vector>

#include "host_geom.h"

namespace p2m {

struct SiteSet {
    Lattice lat;
    std::vector<IPt> pts;           // lattice coordinates of the sites (after jitter)
    std::vector<int> vid;           // Delaunay vertex id of each site
    Delaunay dt;
    std::vector<int64_t> nb_off;    // Delaunay neighbours (CSR over sites), nearest first
    std::vector<int32_t> nb_id;
    std::vector<int64_t> cell_off;  // cell corners (CSR over sites)
    std::vector<double> cell_xyz;

    // at most this many bisectors cut one cell (the cell is then a superset of the true one)
    static constexpr int kMaxClip = 4096;
    // clipping tolerance: a corner within this distance of a cutting plane is kept
    static double clip_tol(double diag) { return 1e-12 * diag; }

    void world(int i, double out[3]) const;
    int triangulate_from(int first, uint64_t seed, std::string& err);
    void neighbour_csr();
    // host clip of every cell (threads over sites)
    int clip_cells(const double dom_lo[3], const double dom_hi[3], double diag, int n_threads);
    // device clip of every cell; cells beyond its fixed capacity are clipped on the host
    // (ms_kernel / ms_host: the device kernel and the host clip of the rest, may be NULL)
    int clip_cells_gpu(const double dom_lo[3], const double dom_hi[3], double diag, int n_threads, void* stream,
                       int64_t* n_host, double* ms_kernel = nullptr, double* ms_host = nullptr);
    bool clip_one(int s, const double dom_lo[3], const double dom_hi[3], double tol, Clipper& C) const;
    int clip_some(const int* only, int count, const double dom_lo[3], const double dom_hi[3], double diag,
                  int n_threads, std::vector<std::vector<double>>& corners) const;
};

int hardware_threads();

// Voronoi vertices w[n][3] inside [lo, hi] binned into tau-cells on the device (ncell[3]
// cells per axis): the occupied cells' keys (cz * ncy + cy) * ncx + cx, ascending, and their
// counts.  Returns 0, or -1 on a CUDA or allocation failure.
int bin_points_gpu(const std::vector<double>& w, const double lo[3], const double hi[3], double tau,
                   const int64_t ncell[3], std::vector<uint64_t>& keys, std::vector<int>& counts, void* stream);

}  // namespace p2m
