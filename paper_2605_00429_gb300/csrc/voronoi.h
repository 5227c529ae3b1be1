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
    std::vector<int64_t> nb_off;    // Delaunay neighbours (CSR over sites)
    std::vector<int32_t> nb_id;
    std::vector<int64_t> cell_off;  // cell corners (CSR over sites)
    std::vector<double> cell_xyz;

    void world(int i, double out[3]) const;
    int triangulate_from(int first, uint64_t seed, std::string& err);
    void neighbour_csr();
    int clip_cells(const double dom_lo[3], const double dom_hi[3], double diag, int n_threads);
};

int hardware_threads();

}  // namespace p2m
