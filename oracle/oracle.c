/*
 * P2M++ FP64 brute-force oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
 * library.  The product path (paper_2605_00429_gb300) never calls it and shares no code,
 * header, table or helper with it.
 *
 * What it computes (plain definitions, no acceleration structure, no pruning):
 *
 *  orc_closest      d(q, M) = min_f d(q, f) over ALL triangles (the quantity the method
 *                   reaches exactly, Section 3.3 "Distance Query Stage" and Section 3.3
 *                   "Relaxation of Interference Relationships": the relaxed table keeps
 *                   every triangle that can beat the reference point, so the localised
 *                   search returns the global minimum).  Tie between equal FP64 distances:
 *                   smallest triangle id.  Also returns the second-smallest distance so a
 *                   parity test can tell a genuine tie from a wrong answer.
 *  orc_nearest_site argmin_s ||q - s|| over ALL sites (the cell-locate step, Section 3.3
 *                   "Recursive Nearest Neighbor Search"); tie -> lower site index.
 *  orc_ball_margin  for every triangle f, min over a set of balls B(u, r_u) of
 *                   d(u, f) - r_u.  A triangle meets the union of balls iff its margin
 *                   is <= 0 (solid ball vs solid triangle, Section 3.3 "Implementation
 *                   Details", Eq. 3 and Eq. 8).
 *
 * Point-triangle distance, written from the geometry and deliberately unlike the GPU
 * routine: project q onto the supporting plane; if the projection's three signed-area
 * barycentrics are all >= 0 it is the closest point; otherwise the closest point lies on
 * the boundary, so take the best of the three clamped segment projections.  Triangles
 * whose normal vanishes (zero area) use the segment path only.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 crs(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }

/* closest point of segment [a,b] to q; t in [0,1] is the parameter of the result */
static v3 seg_closest(v3 q, v3 a, v3 b, double *t_out) {
    v3 ab = sub(b, a);
    double l2 = dot(ab, ab);
    double t = 0.0;
    if (l2 > 0.0) {
        t = dot(sub(q, a), ab) / l2;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    *t_out = t;
    return add(a, scl(ab, t));
}

/* closest point p on triangle (a,b,c) to q, barycentrics (wa,wb,wc) with p = wa a + wb b + wc c */
static double tri_closest(v3 q, v3 a, v3 b, v3 c, v3 *p_out, double bary[3]) {
    v3 n = crs(sub(b, a), sub(c, a));
    double n2 = dot(n, n);
    double lab = dot(sub(b, a), sub(b, a)), lac = dot(sub(c, a), sub(c, a));
    if (n2 > 1e-24 * lab * lac && n2 > 0.0) {
        /* orthogonal projection onto the supporting plane */
        v3 p = sub(q, scl(n, dot(sub(q, a), n) / n2));
        /* signed sub-triangle areas relative to the full one */
        double wa = dot(crs(sub(c, b), sub(p, b)), n) / n2;
        double wb = dot(crs(sub(a, c), sub(p, c)), n) / n2;
        double wc = dot(crs(sub(b, a), sub(p, a)), n) / n2;
        if (wa >= 0.0 && wb >= 0.0 && wc >= 0.0) {
            *p_out = p;
            bary[0] = wa; bary[1] = wb; bary[2] = wc;
            v3 d = sub(q, p);
            return dot(d, d);
        }
    }
    /* boundary: best of the three edges */
    double best = INFINITY, t;
    v3 e[3][2] = {{a, b}, {b, c}, {c, a}};
    for (int k = 0; k < 3; ++k) {
        v3 p = seg_closest(q, e[k][0], e[k][1], &t);
        v3 d = sub(q, p);
        double d2 = dot(d, d);
        if (d2 < best) {
            best = d2;
            *p_out = p;
            double w[3] = {0, 0, 0};
            w[k] = 1.0 - t;
            w[(k + 1) % 3] = t;
            bary[0] = w[0]; bary[1] = w[1]; bary[2] = w[2];
        }
    }
    return best;
}

static v3 vert(const float *verts, int64_t i) {
    return mk((double)verts[3 * i], (double)verts[3 * i + 1], (double)verts[3 * i + 2]);
}

/* single point-triangle query, exported for closed-form pin tests */
double orc_point_triangle(const double *q, const double *a, const double *b, const double *c,
                          double *closest, double *bary) {
    v3 p;
    double d2 = tri_closest(mk(q[0], q[1], q[2]), mk(a[0], a[1], a[2]), mk(b[0], b[1], b[2]),
                            mk(c[0], c[1], c[2]), &p, bary);
    closest[0] = p.x; closest[1] = p.y; closest[2] = p.z;
    return sqrt(d2);
}

void orc_closest(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                 const float *pts, int64_t n, double *dist, double *closest, int64_t *tri,
                 double *bary, double *dist_second) {
    (void)n_verts;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        v3 q = mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        double best = INFINITY, second = INFINITY, bb[3] = {0, 0, 0};
        int64_t bt = -1;
        v3 bp = mk(0, 0, 0);
        for (int64_t f = 0; f < n_tris; ++f) {
            v3 p;
            double w[3];
            double d2 = tri_closest(q, vert(verts, tris[3 * f]), vert(verts, tris[3 * f + 1]),
                                    vert(verts, tris[3 * f + 2]), &p, w);
            if (d2 < best) {
                second = best;
                best = d2; bt = f; bp = p;
                bb[0] = w[0]; bb[1] = w[1]; bb[2] = w[2];
            } else if (d2 < second) {
                second = d2;
            }
        }
        dist[i] = sqrt(best);
        if (dist_second) dist_second[i] = sqrt(second);
        if (tri) tri[i] = bt;
        if (closest) { closest[3 * i] = bp.x; closest[3 * i + 1] = bp.y; closest[3 * i + 2] = bp.z; }
        if (bary) { bary[3 * i] = bb[0]; bary[3 * i + 1] = bb[1]; bary[3 * i + 2] = bb[2]; }
    }
}

void orc_nearest_site(const double *sites, int64_t n_sites, const double *pts, int64_t n,
                      int64_t *site, double *dist, double *dist_second) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        v3 q = mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        double best = INFINITY, second = INFINITY;
        int64_t bs = -1;
        for (int64_t s = 0; s < n_sites; ++s) {
            v3 d = sub(q, mk(sites[3 * s], sites[3 * s + 1], sites[3 * s + 2]));
            double d2 = dot(d, d);
            if (d2 < best) { second = best; best = d2; bs = s; }
            else if (d2 < second) second = d2;
        }
        site[i] = bs;
        if (dist) dist[i] = sqrt(best);
        if (dist_second) dist_second[i] = sqrt(second);
    }
}

void orc_ball_margin(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                     const double *centres, const double *radii, int64_t n_balls, double *margin) {
    (void)n_verts;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t f = 0; f < n_tris; ++f) {
        v3 a = vert(verts, tris[3 * f]), b = vert(verts, tris[3 * f + 1]), c = vert(verts, tris[3 * f + 2]);
        double m = INFINITY;
        for (int64_t k = 0; k < n_balls; ++k) {
            v3 p;
            double w[3];
            double d = sqrt(tri_closest(mk(centres[3 * k], centres[3 * k + 1], centres[3 * k + 2]), a, b, c, &p, w));
            double g = d - radii[k];
            if (g < m) m = g;
        }
        margin[f] = m;
    }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* d(q, M) with FP64 vertices and queries (no FP32 rounding), for finite differences */
void orc_dist_f64(const double *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris,
                  const double *pts, int64_t n, double *dist) {
    (void)n_verts;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        v3 q = mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        double best = INFINITY;
        for (int64_t f = 0; f < n_tris; ++f) {
            const double *a = verts + 3 * (int64_t)tris[3 * f], *b = verts + 3 * (int64_t)tris[3 * f + 1],
                         *c = verts + 3 * (int64_t)tris[3 * f + 2];
            v3 p;
            double w[3];
            double d2 = tri_closest(q, mk(a[0], a[1], a[2]), mk(b[0], b[1], b[2]), mk(c[0], c[1], c[2]), &p, w);
            if (d2 < best) best = d2;
        }
        dist[i] = sqrt(best);
    }
}

/* Generalized winding number of a closed, outward-oriented triangle mesh at each point:
 * w(q) = sum_f Omega_f(q) / (4 pi), with Omega_f the signed solid angle of triangle f seen
 * from q (van Oosterom & Strackee 1983: tan(Omega/2) = a.(b x c) / (|a||b||c| + (a.b)|c| +
 * (a.c)|b| + (b.c)|a|), a, b, c the vertices relative to q).  w = 1 inside, 0 outside; it
 * is the plain definition of inside/outside that the sign of the signed distance follows. */
void orc_winding(const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris, const float *pts,
                 int64_t n, double *w) {
    (void)n_verts;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        v3 q = mk(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        double sum = 0.0;
        for (int64_t f = 0; f < n_tris; ++f) {
            v3 a = sub(vert(verts, tris[3 * f]), q), b = sub(vert(verts, tris[3 * f + 1]), q),
               c = sub(vert(verts, tris[3 * f + 2]), q);
            double la = sqrt(dot(a, a)), lb = sqrt(dot(b, b)), lc = sqrt(dot(c, c));
            double num = dot(a, crs(b, c));
            double den = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
            sum += 2.0 * atan2(num, den);
        }
        w[i] = sum / (4.0 * 3.14159265358979323846);
    }
}
