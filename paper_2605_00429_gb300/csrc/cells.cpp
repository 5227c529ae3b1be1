// FP64 Voronoi cell clipping and the lattice the sites live on.
//
// The interception list of a site is built from the corners of its Voronoi cell
// (Section 3.3, Eq. 3): the cell of site s is the box D cut by the bisector half-spaces of
// its Delaunay neighbours.  Any superset of the cell is still a valid region for Eq. 3 (the
// theorem holds for every convex polytope containing the queries), so rounding here is
// resolved towards keeping points: a vertex within `tol` of a cutting plane is kept.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "host_geom.h"

namespace p2m {

void Clipper::box(const double lo[3], const double hi[3]) {
    V.clear();
    for (int i = 0; i < 8; ++i) {
        V.push_back((i & 1) ? hi[0] : lo[0]);
        V.push_back((i & 2) ? hi[1] : lo[1]);
        V.push_back((i & 4) ? hi[2] : lo[2]);
    }
    static const int kBoxFaces[6][4] = {{0, 2, 6, 4}, {1, 5, 7, 3}, {0, 4, 5, 1}, {2, 3, 7, 6}, {0, 1, 3, 2}, {4, 6, 7, 5}};
    fidx.clear();
    foff.assign(1, 0);
    for (const auto& f : kBoxFaces) {
        fidx.insert(fidx.end(), f, f + 4);
        foff.push_back((int)fidx.size());
    }
}

double Clipper::radius_from(const double p[3]) const { return std::sqrt(radius2_from(p)); }

double Clipper::radius2_from(const double p[3]) const {
    double r2 = 0;
    for (int i = 0; i < n_verts(); ++i) {
        const double dx = V[3 * i] - p[0], dy = V[3 * i + 1] - p[1], dz = V[3 * i + 2] - p[2];
        r2 = std::max(r2, dx * dx + dy * dy + dz * dz);
    }
    return r2;
}

bool Clipper::clip(const double n[3], double d, double tol) {
    const int nv = n_verts();
    val.resize(nv);
    int n_out = 0;
    for (int i = 0; i < nv; ++i) {
        val[i] = n[0] * V[3 * i] + n[1] * V[3 * i + 1] + n[2] * V[3 * i + 2] - d;
        n_out += val[i] > tol;
    }
    cut = n_out > 0;
    if (n_out == 0) return true;
    if (n_out == nv) {
        V.clear();
        fidx.clear();
        foff.assign(1, 0);
        return false;
    }
    edge_new.clear();
    // new vertex on edge (a, b) with a kept and b cut away; shared by the two faces of the edge
    auto cut_vertex = [&](int a, int b) -> int {
        if (val[a] >= -tol) return a;  // a lies on the plane already
        const uint64_t key = a < b ? ((uint64_t)a << 32 | (uint32_t)b) : ((uint64_t)b << 32 | (uint32_t)a);
        for (auto& e : edge_new)
            if (e.first == key) return e.second;
        const double t = val[a] / (val[a] - val[b]);
        const int id = n_verts();
        for (int k = 0; k < 3; ++k) V.push_back(V[3 * a + k] + t * (V[3 * b + k] - V[3 * a + k]));
        val.push_back(0.0);
        edge_new.push_back({key, id});
        return id;
    };
    cap.clear();
    nfidx.clear();
    nfoff.assign(1, 0);
    const int n_faces = (int)foff.size() - 1;
    for (int fi = 0; fi < n_faces; ++fi) {
        const int* f = fidx.data() + foff[fi];
        const int k = foff[fi + 1] - foff[fi];
        // the kept part of the face, consecutive duplicates dropped, straight into nfidx
        const size_t start = nfidx.size();
        auto put = [&](int v) {
            if (nfidx.size() == start || nfidx.back() != v) nfidx.push_back(v);
        };
        for (int j = 0; j < k; ++j) {
            const int a = f[j], b = f[(j + 1) % k];
            const bool ain = val[a] <= tol, bin = val[b] <= tol;
            if (ain) put(a);
            if (ain && !bin) {
                const int c = cut_vertex(a, b);
                if (c != a) put(c);
                cap.push_back(c);
            } else if (!ain && bin) {
                const int c = cut_vertex(b, a);
                if (c != b) put(c);
                cap.push_back(c);
            }
        }
        if (nfidx.size() - start > 1 && nfidx[start] == nfidx.back()) nfidx.pop_back();
        if (nfidx.size() - start >= 3) nfoff.push_back((int)nfidx.size());
        else nfidx.resize(start);
    }
    // the cap face: the cut vertices, ordered by angle about their centroid in the plane
    std::sort(cap.begin(), cap.end());
    cap.erase(std::unique(cap.begin(), cap.end()), cap.end());
    if (cap.size() >= 3) {
        double c[3] = {0, 0, 0};
        for (int v : cap)
            for (int k = 0; k < 3; ++k) c[k] += V[3 * v + k];
        for (int k = 0; k < 3; ++k) c[k] /= (double)cap.size();
        // in-plane basis
        double u[3], w[3];
        const double ax = std::fabs(n[0]), ay = std::fabs(n[1]), az = std::fabs(n[2]);
        double t[3] = {0, 0, 0};
        t[(ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2)] = 1.0;
        u[0] = n[1] * t[2] - n[2] * t[1]; u[1] = n[2] * t[0] - n[0] * t[2]; u[2] = n[0] * t[1] - n[1] * t[0];
        w[0] = n[1] * u[2] - n[2] * u[1]; w[1] = n[2] * u[0] - n[0] * u[2]; w[2] = n[0] * u[1] - n[1] * u[0];
        ang.clear();
        for (int v : cap) {
            const double d0 = V[3 * v] - c[0], d1 = V[3 * v + 1] - c[1], d2 = V[3 * v + 2] - c[2];
            ang.push_back({std::atan2(d0 * w[0] + d1 * w[1] + d2 * w[2], d0 * u[0] + d1 * u[1] + d2 * u[2]), v});
        }
        std::sort(ang.begin(), ang.end());
        for (auto& p : ang) nfidx.push_back(p.second);
        nfoff.push_back((int)nfidx.size());
    }
    // compact: keep vertices used by some face, numbered in order of first use
    const int nv2 = n_verts();
    remap.assign(nv2, -1);
    V2.clear();
    for (int& v : nfidx) {
        if (remap[v] < 0) {
            remap[v] = (int)(V2.size() / 3);
            for (int k = 0; k < 3; ++k) V2.push_back(V[3 * v + k]);
        }
        v = remap[v];
    }
    V.swap(V2);
    fidx.swap(nfidx);
    foff.swap(nfoff);
    return foff.size() > 1;
}

bool Lattice::setup(const double dom_lo[3], const double dom_hi[3]) {
    double half = 0, mid[3];
    for (int k = 0; k < 3; ++k) {
        mid[k] = 0.5 * (dom_lo[k] + dom_hi[k]);
        half = std::max(half, 0.5 * (dom_hi[k] - dom_lo[k]));
    }
    double mag = 0;
    for (int k = 0; k < 3; ++k) mag = std::max(mag, std::fabs(mid[k]) + half);
    // smallest power of two h with half/h <= R - 2 and (|mid| + half)/h < 2^24
    int e = (int)std::ceil(std::log2(std::max(half / (double)(R - 2), mag / 16777000.0)));
    for (;; ++e) {
        h = std::ldexp(1.0, e);
        bool ok = half / h <= (double)(R - 2) && mag / h < 16777000.0;
        if (ok) break;
    }
    for (int k = 0; k < 3; ++k) c[k] = (int64_t)std::llround(mid[k] / h);
    return std::isfinite(h) && h > 0;
}

IPt Lattice::to_lattice(const double p[3]) const {
    return {(int64_t)std::llround(p[0] / h) - c[0], (int64_t)std::llround(p[1] / h) - c[1],
            (int64_t)std::llround(p[2] / h) - c[2]};
}

void Lattice::to_world(const IPt& k, double out[3]) const {
    out[0] = (double)(k.x + c[0]) * h;
    out[1] = (double)(k.y + c[1]) * h;
    out[2] = (double)(k.z + c[2]) * h;
}

}  // namespace p2m
