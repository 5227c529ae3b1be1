"""Pins for the FP64 oracle against facts the mathematics fixes (no GPU).

Each pin is independent of the oracle's own arithmetic: hand-computed closed forms,
analytic distance functions of simple solids, dense sampling, scipy's kd-tree, and finite
differences.
"""
import os

import numpy as np
import pytest

import oracle
import p2m_workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_regions():
    rows = []
    with open(os.path.join(GOLDEN, "triangle_regions.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((np.array(parts[0:3], float), np.array(parts[3:6], float), float(parts[6]),
                         np.array(parts[7:10], float), parts[10]))
    return rows


A, B, C = np.zeros(3), np.array([1.0, 0, 0]), np.array([0, 1.0, 0])


@pytest.mark.parametrize("row", _load_regions(), ids=lambda r: r[4])
def test_triangle_seven_regions(row):
    q, p, d, bary, _ = row
    d_o, p_o, b_o = oracle.point_triangle(q, A, B, C)
    assert abs(d_o - d) < 1e-12
    assert np.allclose(p_o, p, atol=1e-12)
    assert np.allclose(b_o, bary, atol=1e-12)


@pytest.mark.parametrize("perm", [(0, 1, 2), (1, 2, 0), (2, 0, 1), (0, 2, 1)])
def test_triangle_vertex_order_invariance(perm):
    """Distance and closest point do not depend on vertex order; barycentrics permute with it."""
    rng = np.random.default_rng(1)
    tri = rng.normal(size=(3, 3))
    for q in rng.normal(size=(50, 3)) * 2:
        d0, p0, b0 = oracle.point_triangle(q, *tri)
        d1, p1, b1 = oracle.point_triangle(q, *tri[list(perm)])
        assert abs(d0 - d1) < 1e-12 and np.allclose(p0, p1, atol=1e-12)
        assert np.allclose(b1, b0[list(perm)], atol=1e-9)


def test_triangle_against_dense_sampling():
    """min over a dense sample of points of each triangle bounds the oracle from above, and the
    gap is within the sample's resolution."""
    rng = np.random.default_rng(2)
    n = 200
    i, j = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    keep = i + j <= n
    u, v = (i[keep] / n), (j[keep] / n)
    for _ in range(20):
        tri = rng.normal(size=(3, 3))
        pts = (1 - u - v)[:, None] * tri[0] + u[:, None] * tri[1] + v[:, None] * tri[2]
        res = max(np.linalg.norm(tri[1] - tri[0]), np.linalg.norm(tri[2] - tri[0]),
                  np.linalg.norm(tri[2] - tri[1])) / n
        for q in rng.normal(size=(10, 3)) * 1.5:
            d_s = np.min(np.linalg.norm(pts - q, axis=1))
            d_o, p_o, b_o = oracle.point_triangle(q, *tri)
            assert d_o <= d_s + 1e-12
            assert d_s - d_o <= res
            assert np.all(b_o >= -1e-12) and abs(b_o.sum() - 1) < 1e-12
            assert np.allclose(b_o @ tri, p_o, atol=1e-12)


def test_degenerate_triangles():
    """Zero-area triangles reduce to segments / points."""
    q = np.array([0.5, 2.0, 0.0])
    # collinear: segment from (0,0,0) to (1,0,0), with a duplicate point in the middle
    d, p, b = oracle.point_triangle(q, [0, 0, 0], [1, 0, 0], [0.5, 0, 0])
    assert abs(d - 2.0) < 1e-12 and np.allclose(p, [0.5, 0, 0])
    d, p, b = oracle.point_triangle(q, [1, 1, 1], [1, 1, 1], [1, 1, 1])
    assert abs(d - np.linalg.norm(q - 1)) < 1e-12


def test_cube_closed_form():
    """Axis-aligned unit cube: outside d = ||max(|q| - 1/2, 0)||, inside d = 1/2 - max|q_i|."""
    m = W.unit_cube()
    rng = np.random.default_rng(3)
    q = (rng.random((4000, 3)) * 3 - 1.5).astype(np.float32)
    r = oracle.closest(m.verts, m.tris, q)
    a = np.abs(q.astype(np.float64))
    inside = np.all(a <= 0.5, axis=1)
    d_out = np.linalg.norm(np.maximum(a - 0.5, 0), axis=1)
    d_in = 0.5 - a.max(axis=1)
    expect = np.where(inside, d_in, d_out)
    assert np.max(np.abs(r["dist"] - expect)) < 1e-12
    assert np.max(np.abs(np.linalg.norm(q - r["closest"], axis=1) - r["dist"])) < 1e-12


def test_plane_closed_form():
    m = W.square_plane(1.0)
    rng = np.random.default_rng(4)
    q = (rng.random((3000, 3)) * np.array([4, 4, 2]) - np.array([2, 2, 1])).astype(np.float64).astype(np.float32)
    r = oracle.closest(m.verts, m.tris, q)
    qd = q.astype(np.float64)
    dx = np.maximum(np.abs(qd[:, 0]) - 1, 0)
    dy = np.maximum(np.abs(qd[:, 1]) - 1, 0)
    expect = np.sqrt(dx ** 2 + dy ** 2 + qd[:, 2] ** 2)
    assert np.max(np.abs(r["dist"] - expect)) < 1e-12


@pytest.mark.parametrize("mesh", ["ico3", "uv"])
def test_vertex_rays(mesh):
    """For a convex polyhedron inscribed in a sphere, q = t * v/|v| (t > |v|) has closest
    point v: the sphere's tangent plane at v supports the polyhedron."""
    m = W.icosphere(3) if mesh == "ico3" else W.uv_sphere()
    v = m.verts.astype(np.float64)
    rng = np.random.default_rng(5)
    idx = rng.choice(m.n_verts, 200, replace=False)
    t = 1.0 + rng.random(200)
    dirs = v[idx] / np.linalg.norm(v[idx], axis=1, keepdims=True)
    q = (dirs * t[:, None]).astype(np.float32)
    r = oracle.closest(m.verts, m.tris, q)
    expect = np.linalg.norm(q.astype(np.float64) - v[idx], axis=1)
    assert np.max(np.abs(r["dist"] - expect)) < 1e-9
    assert np.max(np.linalg.norm(r["closest"] - v[idx], axis=1)) < 1e-6


def test_whole_result_invariants():
    m, q = W.workload_small(3000)
    r = oracle.closest(m.verts, m.tris, q)
    qd = q.astype(np.float64)
    assert np.max(np.abs(np.linalg.norm(qd - r["closest"], axis=1) - r["dist"])) < 1e-12
    assert np.all(r["bary"] >= -1e-12) and np.max(np.abs(r["bary"].sum(1) - 1)) < 1e-12
    v = m.verts.astype(np.float64)
    tv = v[m.tris[r["tri"]]]
    assert np.max(np.abs(np.einsum("nk,nkc->nc", r["bary"], tv) - r["closest"])) < 1e-12
    assert np.all(r["dist2"] >= r["dist"])
    # 1-Lipschitz
    i = np.arange(len(q) - 1)
    assert np.all(np.abs(r["dist"][i] - r["dist"][i + 1]) <= np.linalg.norm(qd[i] - qd[i + 1], axis=1) + 1e-12)


def test_closest_tie_breaks_to_lowest_id():
    """A point equidistant from two faces gets the lower id."""
    m = W.unit_cube()
    q = np.array([[0.0, 0.0, 0.0]], np.float32)  # centre: all 12 triangles at 1/2
    r = oracle.closest(m.verts, m.tris, q)
    assert r["tri"][0] == 0 and abs(r["dist"][0] - 0.5) < 1e-15 and abs(r["dist2"][0] - 0.5) < 1e-15


def test_nearest_site_against_kdtree():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(6)
    s = rng.normal(size=(500, 3))
    q = rng.normal(size=(5000, 3)) * 1.3
    site, d, d2 = oracle.nearest_site(s, q)
    dk, ik = cKDTree(s).query(q, k=2)
    assert np.array_equal(site, ik[:, 0])
    assert np.allclose(d, dk[:, 0], atol=1e-12) and np.allclose(d2, dk[:, 1], atol=1e-12)


def test_nearest_site_tie_lower_index():
    s = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 1.0, 0]])
    site, d, _ = oracle.nearest_site(s, np.zeros((1, 3)))
    assert site[0] == 0


def test_ball_margin_closed_forms():
    """Ball at the centre of a unit icosphere: radius 1 contains every (chordal) face, radius
    0.5 meets none; the margin at the centre equals the face-plane distance minus r."""
    m = W.icosphere(2)
    mg1 = oracle.ball_margin(m.verts, m.tris, [[0, 0, 0]], [1.0])
    assert np.all(mg1 <= 1e-7)
    mg2 = oracle.ball_margin(m.verts, m.tris, [[0, 0, 0]], [0.5])
    assert np.all(mg2 > 0.4)
    v = m.verts.astype(np.float64)
    a, b, c = v[m.tris[:, 0]], v[m.tris[:, 1]], v[m.tris[:, 2]]
    n = np.cross(b - a, c - a)
    plane = np.abs(np.einsum("ij,ij->i", n, a)) / np.linalg.norm(n, axis=1)
    assert np.max(np.abs(mg2 - (plane - 0.5))) < 1e-12
    # union of two balls = elementwise minimum
    mg3 = oracle.ball_margin(m.verts, m.tris, [[0, 0, 0], [0, 0, 1.5]], [0.5, 0.7])
    mg4 = oracle.ball_margin(m.verts, m.tris, [[0, 0, 1.5]], [0.7])
    assert np.array_equal(mg3, np.minimum(mg2, mg4))
    # a tiny ball at a vertex meets exactly its incident faces
    j = 7
    mg5 = oracle.ball_margin(m.verts, m.tris, [v[j]], [1e-6])
    assert set(np.nonzero(mg5 <= 0)[0]) == set(np.nonzero((m.tris == j).any(1))[0])


def test_aux_radius_eq8():
    u = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)
    r = oracle.aux_radius([0, 0, 0], u, [0, 0, 2])
    assert abs(r - (np.sqrt(3) + np.sqrt(11))) < 1e-12


def test_gradient_analytic_vs_fd():
    """FP64 central differences of L = sum g_i d_i on icosphere(2) (320 tris)."""
    m = W.displace_radial(W.icosphere(2), 0.05, 0)
    rng = np.random.default_rng(7)
    q = W.queries_surface_gauss(m, 300, 0.05, seed=8)
    g = rng.normal(size=q.shape[0])
    res = oracle.closest(m.verts, m.tris, q)
    gq, gv = oracle.grad_analytic(m.verts, m.tris, q, g, res)
    # skip medial ties and on-surface points, where d is not differentiable
    ok = ((res["dist2"] - res["dist"]) > 1e-5) & (res["dist"] > 1e-5)
    qi = np.nonzero(ok)[0][:60]
    h = 1e-7
    fq, _ = oracle.grad_fd(m.verts, m.tris, q, g, h, query_idx=qi, vert_idx=[])
    assert np.max(np.abs(fq - gq[qi])) < 1e-6 * np.max(np.abs(g)) + 1e-7
    # vertex gradient: restrict the loss to well-separated points only
    g2 = np.where(ok, g, 0.0)
    _, gv2 = oracle.grad_analytic(m.verts, m.tris, q, g2, res)
    vi = rng.choice(m.n_verts, 12, replace=False)
    _, fv = oracle.grad_fd(m.verts, m.tris, q, g2, h, query_idx=[], vert_idx=vi)
    assert np.max(np.abs(fv - gv2[vi])) < 1e-5


def test_winding_number_closed_forms():
    """Winding number: 1 inside and 0 outside a closed outward-oriented mesh; on the cube the
    answer is max|q_i| < 1/2, on the icosphere |q| below the inscribed radius / above 1."""
    cube = W.unit_cube()
    rng = np.random.default_rng(9)
    q = (rng.random((3000, 3)) * 1.4 - 0.7).astype(np.float32)
    a = np.abs(q.astype(np.float64)).max(1)
    keep = np.abs(a - 0.5) > 1e-3
    w = oracle.winding(cube.verts, cube.tris, q[keep])
    assert np.allclose(w, (a[keep] < 0.5).astype(float), atol=1e-9)
    ico = W.icosphere(3)
    r = np.linalg.norm(q.astype(np.float64), axis=1) / 0.7 * 1.5
    q2 = (q.astype(np.float64) / np.linalg.norm(q, axis=1, keepdims=True) * r[:, None]).astype(np.float32)
    rr = np.linalg.norm(q2.astype(np.float64), axis=1)
    keep = (rr < 0.98) | (rr > 1.0001)
    w = oracle.winding(ico.verts, ico.tris, q2[keep])
    assert np.allclose(w, (rr[keep] < 0.98).astype(float), atol=1e-9)
    # reversing the orientation negates it
    w_rev = oracle.winding(ico.verts, ico.tris[:, ::-1].copy(), q2[keep][:50])
    assert np.allclose(w_rev, -w[:50], atol=1e-9)


def test_signed_distance_sphere():
    m = W.icosphere(4)
    rng = np.random.default_rng(10)
    q = (rng.normal(size=(2000, 3)) * 0.7).astype(np.float32)
    sd, w = oracle.signed_distance(m.verts, m.tris, q)
    r = np.linalg.norm(q.astype(np.float64), axis=1)
    far = np.abs(r - 1.0) > 0.01
    assert np.all(np.sign(sd[far]) == np.sign(r[far] - 1.0))


def test_voronoi_cell_lattice_closed_form():
    """Sites on a 4x4x4 lattice of spacing h: an interior site's cell is the cube of side h
    centred on it, and a corner site's cell reaches the box corner."""
    h = 0.25
    g = (np.arange(4) + 0.5) * h
    sites = np.array([[x, y, z] for z in g for y in g for x in g])
    lo, hi = np.zeros(3), np.ones(3)
    i = 1 + 4 * 1 + 16 * 2  # (1, 1, 2): interior
    c = oracle.voronoi_cell(sites, i, lo, hi)
    expect = {tuple(np.round(sites[i] + 0.5 * h * np.array([a, b, d]), 12)) for a in (-1, 1) for b in (-1, 1)
              for d in (-1, 1)}
    assert {tuple(np.round(u, 12)) for u in c} == expect
    c0 = oracle.voronoi_cell(sites, 0, lo, hi)
    assert {tuple(np.round(u, 12)) for u in c0} == {(x, y, z) for x in (0, h) for y in (0, h) for z in (0, h)}


def test_voronoi_cell_two_sites_half_boxes():
    s = np.array([[0.3, 0.5, 0.5], [0.7, 0.5, 0.5]])
    c = oracle.voronoi_cell(s, 0, np.zeros(3), np.ones(3))
    assert {tuple(np.round(u, 12)) for u in c} == {(x, y, z) for x in (0.0, 0.5) for y in (0.0, 1.0) for z in (0.0, 1.0)}


def test_voronoi_cells_partition_the_box():
    """Random sites: every corner lies in its closed cell (no other site strictly nearer) and
    in D, and the cell volumes sum to vol(D)."""
    from scipy.spatial import ConvexHull
    rng = np.random.default_rng(11)
    sites = rng.random((150, 3)) * np.array([2.0, 1.0, 0.5])
    lo, hi = np.array([-0.1, -0.1, -0.1]), np.array([2.1, 1.1, 0.6])
    vol = 0.0
    for i in range(len(sites)):
        c = oracle.voronoi_cell(sites, i, lo, hi)
        d_own = np.linalg.norm(c - sites[i], axis=1)
        d_all = np.min(np.linalg.norm(c[:, None, :] - sites[None, :, :], axis=2), axis=1)
        assert np.all(d_own <= d_all + 1e-9)
        assert np.all(c >= lo - 1e-12) and np.all(c <= hi + 1e-12)
        vol += ConvexHull(c).volume
    assert abs(vol - np.prod(hi - lo)) <= 1e-9 * np.prod(hi - lo)


def test_vertex_sphere_union_theorem():
    """Eq. 3 (Vertex Sphere Union): for a convex cell P with corners u and any fixed v, every
    ball B(x, ||x - v||) with x in P lies inside the union of the corner balls B(u, ||u - v||).
    Checked on random cells with random points of the small balls."""
    rng = np.random.default_rng(12)
    sites = rng.random((60, 3))
    for i in range(10):
        c = oracle.voronoi_cell(sites, i, np.zeros(3), np.ones(3))
        v = rng.random(3) * 2 - 0.5
        ru = np.linalg.norm(c - v, axis=1)
        for _ in range(20):
            w = rng.dirichlet(np.ones(len(c)))
            x = w @ c
            r = np.linalg.norm(x - v)
            dirs = rng.normal(size=(200, 3))
            dirs /= np.linalg.norm(dirs, axis=1)[:, None]
            p = x + dirs * (r * rng.random(200) ** (1 / 3))[:, None]
            cover = np.min(np.linalg.norm(p[:, None, :] - c[None, :, :], axis=2) - ru[None, :], axis=1)
            assert np.all(cover <= 1e-12)
