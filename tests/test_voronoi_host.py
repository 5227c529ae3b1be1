"""Host Voronoi stage (exact Delaunay + FP64 cell clipping), checked on the CPU against brute
force: every corner of a site's cell is at least as close to that site as to any other site
(oracle nearest-site search), the cells tile the domain box (volumes sum to vol(D)), and
sampled points lie inside their nearest site's polytope."""
import numpy as np
import pytest

import oracle
import p2m_workloads as W


@pytest.fixture(scope="module")
def p2m():
    from paper_2605_00429_gb300 import build as b
    try:
        b.build()
    except RuntimeError as e:  # pragma: no cover
        pytest.skip(str(e))
    import paper_2605_00429_gb300 as p
    return p


def _cases():
    rng = np.random.default_rng(11)
    uv = W.uv_sphere(16, 8).verts
    ico = W.icosphere(2).verts
    g = np.stack(np.meshgrid(*[np.arange(4.0)] * 3, indexing="ij"), -1).reshape(-1, 3) / 3 - 0.5
    cyl = W.cylinder_cone(24, 6, 3, 2).verts
    # fan centres (cap centre, cone apex) with 300 neighbours each: their cells are closed by
    # far neighbours only after hundreds of near ones have cut them
    fan = W.cylinder_cone(300, 4, 2, 2).verts
    return {
        "cylinder_fan300": fan,
        "random": (rng.random((300, 3)) - 0.5).astype(np.float32),
        "uv_sphere": uv,
        "icosphere": ico,
        "lattice": g.astype(np.float32),
        "cylinder_cone": cyl,
    }


CASES = _cases()


def _domain(p):
    lo, hi = p.min(0).astype(np.float64), p.max(0).astype(np.float64)
    c, h = (lo + hi) / 2, (hi - lo) / 2 * 1.5 + 1e-3
    return c - h, c + h


@pytest.mark.parametrize("name", sorted(CASES))
def test_corners_in_cell_and_volumes(p2m, name):
    from scipy.spatial import ConvexHull
    pts = CASES[name]
    lo, hi = _domain(pts)
    sites, off, cor = p2m.voronoi_cells(pts, lo, hi, seed=3)
    s64 = sites.astype(np.float64)
    diag = np.linalg.norm(hi - lo)
    # moved by at most ~2 lattice steps
    assert np.max(np.abs(s64 - pts)) < 1e-5 * diag
    own = np.repeat(np.arange(len(sites)), np.diff(off))
    _, dmin, _ = oracle.nearest_site(s64, cor)
    down = np.linalg.norm(cor - s64[own], axis=1)
    assert np.max(down - dmin) < 1e-9 * diag, "a corner is closer to another site"
    # corners inside D
    assert np.all(cor >= lo - 1e-9 * diag) and np.all(cor <= hi + 1e-9 * diag)
    vol = 0.0
    for i in range(len(sites)):
        c = cor[off[i]:off[i + 1]]
        assert len(c) >= 4
        vol += ConvexHull(c).volume
    assert abs(vol - np.prod(hi - lo)) < 1e-7 * np.prod(hi - lo)


@pytest.mark.parametrize("name", ["random", "uv_sphere", "lattice"])
def test_samples_inside_nearest_cell(p2m, name):
    from scipy.spatial import ConvexHull
    pts = CASES[name]
    lo, hi = _domain(pts)
    sites, off, cor = p2m.voronoi_cells(pts, lo, hi, seed=5)
    rng = np.random.default_rng(12)
    x = lo + rng.random((3000, 3)) * (hi - lo)
    near, _, _ = oracle.nearest_site(sites.astype(np.float64), x)
    diag = np.linalg.norm(hi - lo)
    hulls = {}
    for j, s in enumerate(near):
        if s not in hulls:
            hulls[s] = ConvexHull(cor[off[s]:off[s + 1]]).equations
        eq = hulls[s]
        assert np.max(eq[:, :3] @ x[j] + eq[:, 3]) < 1e-9 * diag
