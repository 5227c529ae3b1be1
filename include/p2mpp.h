/*
 * p2mpp.h -- C ABI of libp2mpp.so, a GB300 (sm_103a) implementation of the P2M++ query
 * path: Voronoi-localised exact closest-triangle search on a triangle mesh.
 *
 * The method (P2M++, Guo et al.):
 *   * Sites = referenced mesh vertices plus auxiliary sites added where Voronoi vertices
 *     cluster (Section 3.2, "Ring-based Site Augmentation").
 *   * Each site's cell is a convex polytope; its interception list is every triangle that
 *     meets the union of balls B(u, ||u - v||) centred at the cell's corners u, with v the
 *     site's reference point on the mesh (Section 3.3, Eq. 2, Eq. 3 "Vertex Sphere Union").
 *     An off-surface site uses v = proj(s, M): its corner balls, or (aux_balls = 0) the one
 *     ball of radius Eq. 8 around itself that encloses them.
 *   * A query finds its nearest site and scans only that site's list, pruning with each
 *     triangle's bounding sphere (Section 3.3 "Distance Query Stage", "Bounding Sphere
 *     Pruning").  The result is the exact closest point on the mesh.
 *
 * Conventions for every entry point:
 *   * Return value 0 (P2M_OK) on success, else one of the negative P2M_ERR_* codes;
 *     p2m_last_error() then returns a thread-local message.  No entry point aborts or
 *     traps; device-side failures (stack overflow, iteration caps) come back as codes.
 *   * `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Device work is stream-ordered and asynchronous unless the entry point says it
 *     synchronises.
 *   * "d_" pointers are device pointers, "h_" pointers host pointers.  Caller-owned
 *     buffers stay caller-owned; the library never frees them.
 *   * Points and vertices are float32 xyz triples, row-major [n,3].  Triangle ids index
 *     the caller's `tris` array; barycentrics (b0,b1,b2) refer to that triangle's
 *     (v0,v1,v2) so that closest = b0 v0 + b1 v1 + b2 v2.
 *   * Sizes are int64_t.  n == 0 is a successful no-op wherever n appears.  A call takes at
 *     most 2^31 - 1 points (larger n returns P2M_ERR_LIMIT: split the call).
 *   * The device an index was built on must be current when it is used (else
 *     P2M_ERR_INVALID_ARG): its buffers, and the scratch it reuses, live there.
 *   * Calls on one index share its scratch buffers (sort keys, queues, result records, the
 *     host pipeline's staging buffers).  Issue them on one stream, or order them with events:
 *     two calls on the same index whose work overlaps on the GPU race on that scratch.
 *     Different indexes are independent.
 */
#ifndef P2MPP_H
#define P2MPP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define P2M_OK 0
#define P2M_ERR_INVALID_ARG (-1)     /* NULL/NaN/out-of-range input, bad sizes */
#define P2M_ERR_CUDA (-2)            /* a CUDA runtime call failed */
#define P2M_ERR_OOM (-3)             /* device or host allocation failed */
#define P2M_ERR_EMPTY_MESH (-4)      /* no triangle, or no referenced vertex */
#define P2M_ERR_DEGENERATE (-5)      /* all referenced vertices coincide */
#define P2M_ERR_LIMIT (-6)           /* a device work cap or iteration cap was reached */
#define P2M_ERR_STACK (-7)           /* a device BVH traversal stack overflowed */
#define P2M_ERR_NOT_IMPLEMENTED (-8)
#define P2M_ERR_INTERNAL (-9)        /* an internal consistency check failed */

typedef struct p2m_index p2m_index; /* opaque; owns every device structure it builds */

/* Build parameters.  p2m_default_params() fills the defaults given in brackets. */
typedef struct {
    /* Domain box D = mesh bbox scaled by this factor about its centre [1.5].  Cells are
     * clipped to D (the paper is silent on unbounded cells; every cell ∩ D is convex, so
     * Eq. 3 still applies).  Queries outside D take an exact BVH branch-and-bound search. */
    float domain_scale;
    /* Site augmentation of Section 3.2 on/off [1]. */
    int enable_aux;
    /* tau = tau_scale x mean edge length [1.0] (Section 3.2 "Choice of Parameters"). */
    float tau_scale;
    /* A tau-cell is dense when its Voronoi-vertex count exceeds density_factor x the median
     * count of non-empty tau-cells [8.0] and density_min [256].  (Symmetric meshes put
     * thousands of Voronoi vertices in one tau-cell; noise-perturbed ones about a hundred.) */
    float density_factor;
    int density_min;
    /* Auxiliary sites per ring: 12 (icosahedron directions) or 6 (octahedron) [12]. */
    int ring_sites;
    /* Ring radius = ring_radius_scale x tau [0.9: just above sqrt(3) / 2, the radius of the
     * sphere about a tau-cell's centre that encloses the cell]. */
    float ring_radius_scale;
    /* List-membership slack, relative to the bbox diagonal [1e-6]: a triangle joins a list
     * when its distance to a ball is <= radius + slack (conservative). */
    float build_eps_rel;
    /* Nearest-site grid resolution per axis; 0 = automatic [0]. */
    int nn_grid_res;
    /* Query schedule [5]: 5 = queries counting-sorted by nearest site, then each block stages
     * the short lists of the sites of its 1024 queries (entries, bounding spheres, triangle
     * records) in shared memory and scans them thread per query; lists longer
     * than long_list take a warp-cooperative best-first scan (a call with fewer than 48
     * queries per site takes schedule 0 instead); 0 = queries sorted by the Morton code of
     * their grid cell, then thread per query for lists up to long_list entries and the
     * warp-cooperative scan for longer lists; 1 = thread per query for every list; 2 = warp
     * per query for every list; 3 = as 0 without the sort; 4 = as 0, with the queries
     * regrouped by nearest site (a second radix sort) before the list scan.  All give
     * identical results. */
    int schedule;
    /* Deterministic vertex-gradient accumulation (fixed-point integer atomics) [1]. */
    int deterministic;
    /* Seed of the site jitter used to break exact Delaunay degeneracies [1]. */
    int seed;
    /* Lists longer than this take the warp-cooperative scan in schedules 0, 3, 4 and 5; 0 picks
     * the default (256) [0]. */
    int long_list;
    /* Clip the Voronoi cells on the GPU in FP64 [1]; cells beyond the device clipper's fixed
     * capacity (58 cutting planes) are clipped on the host.  0 = every cell on the host. */
    int gpu_cells;
    /* Chunks of the host-buffer query pipeline (p2m_query_host); 0 picks the default (3) [0].
     * More chunks overlap copies and compute better; fewer keep more queries per grid cell
     * in each chunk's Morton order. */
    int pipe_chunks;
    /* Balls of an auxiliary (off-surface) site [1]: 1 = one ball per corner u of its cell with
     * radius ||u - proj(s, M)|| (Eq. 3 with the reference point proj(s, M), merged to at most 128
     * like a vertex site's); 0 = the single enclosing ball of Eq. 8 around s.  Eq. 8's ball
     * contains the corner balls (triangle inequality), so both give exact results; the corner
     * balls give shorter lists where the cell is large. */
    int aux_balls;
    /* Position of the centre site p_c of a dense tau-cell [1]: 1 = the centroid of the
     * Voronoi vertices binned into the cell (the cluster the site is meant to isolate);
     * 0 = the geometric centre of the tau-cell. */
    int aux_centre;
} p2m_build_params;

/* Build statistics (Section 4.1, Table 1: Max / Avg list length) and stage timings. */
typedef struct {
    int64_t n_verts, n_tris;
    int64_t n_sites, n_vertex_sites, n_aux_sites;
    int64_t n_corners;        /* corner balls in the CSR ball table (aux sites count 1) */
    int64_t nnz;              /* total interception-list entries */
    int64_t max_row;          /* Max list length */
    double avg_row;           /* Avg list length */
    int64_t grid_res;         /* nearest-site grid cells per axis */
    int64_t grid_entries;     /* total candidate-site entries in the grid */
    int64_t grid_max;         /* longest candidate-site list */
    int64_t n_delaunay_tets;
    int64_t n_dense_cells;    /* tau-cells flagged dense by the augmentation */
    double domain_lo[3], domain_hi[3];
    double bbox_diag;
    /* stage wall times in milliseconds */
    double ms_upload, ms_tri, ms_lbvh, ms_delaunay, ms_cells, ms_aug, ms_proj, ms_k1, ms_grid, ms_total;
    /* Voronoi vertices per non-empty tau-cell of the augmentation: median and maximum */
    int64_t aug_cell_median, aug_cell_max;
    /* cells clipped on the host although gpu_cells was set (beyond the device capacity) */
    int64_t n_cells_host;
    /* with gpu_cells: the device clip kernel (CUDA events) and the host clip of the rest */
    double ms_cells_kernel, ms_cells_fallback;
} p2m_stats;

/* Per-call query counters (Section 4.1, Table 1 "Queried"). */
typedef struct {
    int64_t n_queries;
    int64_t n_outside;        /* queries outside D (answered by the BVH search) */
    int64_t site_candidates;  /* candidate sites examined by the nearest-site search */
    int64_t tie_rechecks;     /* nearest-site decisions re-checked in FP64 */
    int64_t row_entries;      /* interception-list entries visited */
    int64_t exact_tests;      /* exact point-triangle tests run (after pruning) */
    int64_t long_queries;     /* queries whose list was scanned by the warp-cooperative pass */
    int64_t long_entries;     /* list entries those queries visited (part of row_entries) */
    int64_t queried_list;     /* sum over in-domain queries of the length of their nearest
                                 site's list (over n_queries: the query-weighted average list
                                 length, Table 4's "Queried") */
} p2m_counters;

/* Library version string. */
const char* p2m_version(void);

/* Thread-local message describing the last non-zero return on this thread. */
const char* p2m_last_error(void);

/* Fill *out with the defaults documented in p2m_build_params.  Errors: INVALID_ARG if out
 * is NULL. */
int p2m_default_params(p2m_build_params* out);

/* Build an index over a triangle mesh (the whole preprocessing of Section 3: Voronoi diagram
 * of the sites, augmentation (Section 3.2), corner spheres (Eq. 3, Eq. 8), BVH collision
 * into the interception lists (Section 3.3 "Implementation Details"), and the nearest-site
 * grid).
 *   verts[n_verts*3] float32, tris[n_tris*3] int32 (0-based).  If inputs_on_device != 0
 *   both are device pointers, else host pointers.  The mesh is copied; the caller may free
 *   its arrays when the call returns.  params may be NULL (defaults).
 * A mesh with fewer than 4 distinct vertices gets no site partition: its queries all take
 * the exact BVH search (same results, no localisation).
 * Synchronises `stream`.  On success *out owns the index (release with p2m_destroy).
 * Errors: INVALID_ARG (NULL, NaN/Inf vertex, index out of range, n <= 0), EMPTY_MESH,
 * DEGENERATE, OOM, CUDA, STACK, LIMIT (lists beyond 2^31 entries). */
int p2m_build(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris,
              int inputs_on_device, const p2m_build_params* params, void* stream,
              p2m_index** out);

/* Release an index and all device memory it owns.  NULL is a no-op. */
void p2m_destroy(p2m_index* h);

/* Closest-point query (Section 3.3 "Distance Query Stage"): for each of n points
 * d_pts[n*3], nearest site -> scan of its interception list -> exact closest point.
 *   d_dist[n]      unsigned distance (required)
 *   d_closest[n*3] closest point on the mesh (or NULL)
 *   d_tri[n]       triangle id holding the closest point (or NULL)
 *   d_bary[n*3]    barycentrics of the closest point in that triangle (or NULL)
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA, STACK (checked lazily: the
 * overflow flag of a query is reported by the next synchronising call). */
int p2m_query(p2m_index* h, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
              int32_t* d_tri, float* d_bary, void* stream);

/* Signed distance (an extension: the paper computes unsigned distances): the
 * query of p2m_query, then the sign of (q - p) . n with n the angle-weighted pseudonormal of
 * the feature (face, edge or vertex) holding the closest point p: negative inside, positive
 * outside a closed, outward-oriented mesh (meaningless for an open or inconsistently
 * oriented one).  d_sdist[n] receives the signed distance; d_closest, d_tri, d_bary as in
 * p2m_query (may be NULL; the index then uses its own scratch for d_tri / d_bary).
 * Asynchronous, except that the first call on an index (and the first after
 * p2m_update_vertices) computes the pseudonormals on the host in FP64 and uploads them
 * before it launches anything.  Errors: INVALID_ARG, OOM, CUDA. */
int p2m_query_signed(p2m_index* h, const float* d_pts, int64_t n, float* d_sdist, float* d_closest,
                     int32_t* d_tri, float* d_bary, void* stream);

/* Mesh-to-mesh distance (an extension the paper names as future work, Section 5): mesh B
 * (device arrays d_verts_b[n_verts_b*3], d_tris_b[n_tris_b*3]) is sampled on the
 * barycentric lattice of `subdivisions` (0..64) of every triangle (0 = its vertices), the
 * samples are queried against the index (mesh A), and h_out[3] receives, over the samples,
 * the minimum distance (an upper bound of the distance between the meshes), the maximum
 * (the directed Hausdorff distance B -> A over the samples, a lower bound of the true one)
 * and the mean.  Allocates its sample buffers; synchronises `stream`.  Errors: INVALID_ARG,
 * OOM, CUDA. */
int p2m_mesh_distance(p2m_index* h, const float* d_verts_b, int64_t n_verts_b, const int32_t* d_tris_b,
                      int64_t n_tris_b, int subdivisions, double* h_out, void* stream);

/* Both directions between the meshes of two single-mesh indexes, sampled as in
 * p2m_mesh_distance: h_out[7] = (min, max, mean) of mesh B's samples against A, the same
 * for A's samples against B, and the symmetric Hausdorff distance over the samples,
 * max(h_out[1], h_out[4]).  Allocates its sample buffers; synchronises `stream`.  Errors:
 * INVALID_ARG, OOM, CUDA. */
int p2m_mesh_distance_pair(p2m_index* a, p2m_index* b, int subdivisions, double* h_out, void* stream);

/* The same query from host memory: copies h_pts in chunks to the device, runs the query
 * and copies the results back.  Host buffers may be pageable, but pinned (cudaHostAlloc)
 * buffers are much faster: the chunks (pipe_chunks of the build parameters, 3 by default,
 * at least 1M points each) run on separate streams, so one chunk's copies overlap another
 * chunk's kernels.  Output pointers other than h_dist may be NULL.  Synchronous: returns
 * when the outputs are in host memory.  Errors: INVALID_ARG, OOM, CUDA. */
int p2m_query_host(p2m_index* h, const float* h_pts, int64_t n, float* h_dist, float* h_closest,
                   int32_t* h_tri, float* h_bary, void* stream);

/* Nearest site only (the "Cell Locate" step, Section 3.3 "Recursive Nearest Neighbor
 * Search"): d_site[n] gets the index of the nearest site (ties -> lower index), or -1 for
 * a point outside D.  Asynchronous. */
int p2m_nearest_site(p2m_index* h, const float* d_pts, int64_t n, int32_t* d_site, void* stream);

/* Instrumented query: runs the query and fills *out with counters (Table 1 "Queried").
 * Synchronises `stream`.  d_dist etc. as in p2m_query (d_dist may be NULL here). */
int p2m_query_counters(p2m_index* h, const float* d_pts, int64_t n, float* d_dist,
                       p2m_counters* out, void* stream);

/* Backward of the unsigned distance (not in the paper; the differentiable form).  With p
 * the closest point on triangle (v0,v1,v2), b its barycentrics and g = d_grad_dist[i]:
 *   d_grad_pts[i]   = g (q - p) / ||q - p||          (0 when q lies on the mesh)
 *   d_grad_verts[vk] += -g b_k (q - p) / ||q - p||    for k = 0,1,2
 * p is recomputed from the index's current vertices and d_tri / d_bary of the forward.
 * d_grad_pts may be NULL; d_grad_verts may be NULL; d_grad_verts[n_verts*3] is
 * ACCUMULATED into (zero it first).  With params.deterministic the vertex sums are
 * bit-reproducible: fixed-point integer atomics whose unit 2^-e is picked per call from
 * B = max_i |g_i| max(1, max_k |b_ik|) so that 3 n B 2^e <= 2^62 (no sum can overflow; each
 * contribution is rounded to the unit, an error of at most 3 n B 2^-63).  There a non-finite
 * g or b leaves d_grad_pts and d_grad_verts untouched and makes the next synchronising call
 * on the index return P2M_ERR_LIMIT.  Asynchronous.  Errors: INVALID_ARG, OOM, CUDA. */
int p2m_backward(p2m_index* h, const float* d_pts, int64_t n, const int32_t* d_tri,
                 const float* d_bary, const float* d_grad_dist, float* d_grad_pts,
                 float* d_grad_verts, void* stream);

/* Replace the vertex positions (same topology) and rebuild every structure.  d_verts is a
 * device pointer [n_verts*3].  Synchronises `stream`. */
int p2m_update_vertices(p2m_index* h, const float* d_verts, void* stream);

/* Build statistics (Table 1 Max / Avg, counts, stage times).  Host-only. */
int p2m_get_stats(const p2m_index* h, p2m_stats* out);

/* ---- Batched form (not in the paper): many meshes behind one persistent launch. ------ */

/* Build one index over n_meshes meshes (host pointers verts[i], tris[i]).  Each mesh gets
 * its own sites, lists and grid; all live in shared device arrays with per-mesh offsets.
 * Synchronises.  Errors as p2m_build (the message names the failing mesh). */
int p2m_batch_build(int n_meshes, const float* const* verts, const int64_t* n_verts,
                    const int32_t* const* tris, const int64_t* n_tris,
                    const p2m_build_params* params, void* stream, p2m_index** out);

/* Query a batch: queries of mesh i are d_pts[h_q_offsets[i] .. h_q_offsets[i+1]) (host
 * array of n_meshes+1 offsets, non-decreasing, starting at 0).  Outputs as p2m_query, tri
 * ids local to each mesh.  mode 0: one persistent launch over a tile queue (tile size and
 * schedule picked by the autotuner); with use_graph != 0 that launch is captured once in a
 * CUDA graph per (batch, offsets) and replayed.  mode 1: one launch per mesh (the plain
 * per-mesh forward, for comparison).  Asynchronous.  Errors: INVALID_ARG, CUDA, OOM. */
int p2m_batch_query(p2m_index* batch, const float* d_pts, const int64_t* h_q_offsets,
                    float* d_dist, float* d_closest, int32_t* d_tri, float* d_bary,
                    int mode, int use_graph, void* stream);

/* Number of meshes in an index (1 for p2m_build). */
int p2m_num_meshes(const p2m_index* h);

/* ---- Introspection (tests and tools).  All synchronous; host output buffers. -------- */

/* Sizes of mesh `mesh` of the index: n_sites, nnz (list entries), n_balls (corner balls). */
int p2m_get_sizes(const p2m_index* h, int mesh, int64_t* n_sites, int64_t* nnz, int64_t* n_balls);

/* Sites of mesh `mesh`: h_sites[n_sites*3] float32 positions (the exact partition the
 * queries use), h_ref[n_sites*3] float64 reference points on the mesh (vertex position,
 * or proj(s, M) for an auxiliary site), h_kind[n_sites] 0 = vertex site, 1 = aux site.
 * Any pointer may be NULL. */
int p2m_get_sites(const p2m_index* h, int mesh, float* h_sites, double* h_ref, int32_t* h_kind);

/* Interception lists (CSR) of mesh `mesh`: h_offsets[n_sites+1], h_tri_ids[nnz]. */
int p2m_get_lists(const p2m_index* h, int mesh, int64_t* h_offsets, int32_t* h_tri_ids);

/* Kernel timing of the query path (for benchmarks).  With on != 0, every later query call on
 * the index records CUDA events on its stream: at the start, around its list-scan kernel
 * (k_query_staged, or k_query_thread in the Morton-ordered schedules; the dominant kernel)
 * and at the end.  p2m_query_timing then returns, for the last call, h_ms[0] = the list-scan
 * kernel's milliseconds (0 when the call had none) and h_ms[1] = the whole launch sequence's;
 * it waits for the call's end event.  Errors: INVALID_ARG (NULL, timing off, no timed call),
 * CUDA. */
int p2m_set_timing(p2m_index* h, int on);
int p2m_query_timing(p2m_index* h, double* h_ms);

/* Triangle BVH of mesh `mesh` (the LBVH of Section 3.3 "Implementation Details" that the
 * corner balls are tested against, and the exact search for points outside D uses).
 * *n_nodes = n_tris - 1 internal nodes (0 for a one-triangle mesh); *root = the root node, or
 * ~0 when the only node is a leaf.  h_nodes[n_nodes*16] float32, per node: the box of child 0
 * (lo.xyz, child ref, hi.xyz, 0) then the box of child 1 (same layout); a child ref is int32
 * bits, >= 0 an internal node, < 0 a leaf ~k where k is a leaf position.  h_leaf_tri[n_tris]
 * = the caller's triangle id stored at each leaf position.  Either pointer may be NULL. */
int p2m_get_bvh(const p2m_index* h, int mesh, int64_t* n_nodes, int32_t* root, float* h_nodes, int32_t* h_leaf_tri);

/* Corner balls of mesh `mesh` (Eq. 3, or Eq. 8 for auxiliary sites with aux_balls = 0): h_ball_offsets[n_sites+1] into
 * h_centres[n_balls*3] (float64) and h_radii[n_balls] (float64, before slack). */
int p2m_get_balls(const p2m_index* h, int mesh, int64_t* h_ball_offsets, double* h_centres,
                  double* h_radii);

/* ---- Allocation-free query.  The paper has no counterpart: this is a service entry
 * point for callers that must not allocate device memory. --------------------------------
 *
 * Some callers cannot let a library call cudaMalloc / cudaFree: a framework that owns all
 * device memory through its own pool or arena, a latency-bound loop that cannot afford the
 * device-wide synchronisation those calls imply, or an operator hook that is forbidden to
 * allocate.  p2m_query may grow a scratch buffer of the index on demand; this variant gives
 * the same results as p2m_query (same arguments and outputs) but runs on a fixed scratch
 * array compiled into the library: about 3 MiB of device memory on every GPU where the
 * library is loaded, held until the process exits.  It calls no allocating routine.
 *   * At most P2M_NOALLOC_MAX_QUERIES points per call; a larger n returns P2M_ERR_LIMIT
 *     (split the batch).  The index itself must already exist (p2m_build allocates).
 *   * The first call on each device looks up the scratch array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call before any
 *     stream capture begins.
 *   * Every call on a device shares the one scratch array, and each call resets the parts
 *     that must start at zero.  Calls whose work overlaps on the GPU (different streams, or
 *     other host threads, without ordering between them) race on that array: order them.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, LIMIT, CUDA. */
#define P2M_NOALLOC_MAX_QUERIES 262144
int p2m_query_noalloc(p2m_index* h, const float* d_pts, int64_t n, float* d_dist, float* d_closest,
                      int32_t* d_tri, float* d_bary, void* stream);

/* ---- Host-only stage (no GPU needed). ------------------------------------------------ */

/* The clipped Voronoi cells of a point set exactly as p2m_build computes them (Section 3.3:
 * the cells whose corners carry the balls of Eq. 3): each site is moved to the library's
 * lattice (at most about 2e-6 of the domain size away; the moved positions are returned in
 * h_sites_out[n*3]), the exact Delaunay triangulation gives each site's neighbours, and the
 * box D = [dom_lo, dom_hi] is cut by the neighbours' bisector planes in FP64.
 *   h_sites[n*3] float32 inside D, n >= 4.  Outputs h_corner_off[n+1] (CSR over sites) and
 *   h_corners[n_corners*3] (FP64); call once with h_corners == NULL to learn *n_corners.
 * Errors: INVALID_ARG (NULL, n < 4, a site outside D), INTERNAL. */
int p2m_voronoi_cells(const float* h_sites, int64_t n, const double* dom_lo, const double* dom_hi, int seed,
                      float* h_sites_out, int64_t* h_corner_off, double* h_corners, int64_t* n_corners);

/* The same cells clipped on the GPU (the path p2m_build takes with gpu_cells = 1): the same
 * arguments and outputs, plus *n_host = the cells beyond the device clipper's capacity that
 * were clipped on the host, and the stream the device work runs on.  Corners within 1e-12 of
 * the domain diagonal are merged.  Errors: INVALID_ARG, OOM, CUDA, INTERNAL. */
int p2m_voronoi_cells_device(const float* h_sites, int64_t n, const double* dom_lo, const double* dom_hi, int seed,
                             float* h_sites_out, int64_t* h_corner_off, double* h_corners, int64_t* n_corners,
                             int64_t* n_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* P2MPP_H */
