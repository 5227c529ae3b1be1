"""Corner balls and interception lists against oracles that share nothing with the build
(Section 3.3, Eq. 2, Eq. 3 "Vertex Sphere Union", Eq. 8, "Implementation Details").

The sites are the index's own (the exact partition its queries use); everything else is
recomputed here from the plain definitions:

* each sampled site's Voronoi cell, clipped to the domain box D, from the bisectors of every
  other site (``oracle.voronoi_cell``);
* a vertex site's balls B(u, ||u - v||) over those corners u, with v its vertex (Eq. 3);
* an auxiliary site's reference point is checked to be a closest point of M (its distance is
  the brute-force d(s, M) and it lies on M); its balls are then, by default, the corner balls
  of Eq. 3 with v = proj(s, M), or (aux_balls = 0) the one ball of radius
  max_u (||s - u|| + ||u - proj||) over the oracle's corners (Eq. 8, ``oracle.aux_radius``);
* the list must contain every triangle that meets the union of the oracle's balls (the lower
  bound of the list sandwich, with balls the product did not make);
* Vertex Sphere Union on sampled points x of the cell: B(x, ||x - v||) meets no triangle
  outside the list.
"""
import numpy as np
import pytest

import oracle
import p2m_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2m():
    from paper_2605_00429_gb300 import build as b
    b.build()
    import paper_2605_00429_gb300 as p
    return p


def _cases():
    return {
        "uv_sphere": lambda: W.uv_sphere(32, 16),
        "noisy_icosphere3": lambda: W.displace_radial(W.icosphere(3), 0.05, 0),
        "cylinder_cone_48x12": lambda: W.cylinder_cone(n_ang=48, n_ax=12, n_cone=8, n_cap=3),
    }


def _site_sample(kind, rng, n_vertex=30, n_aux=30):
    aux = np.nonzero(kind == 1)[0]
    vtx = np.nonzero(kind == 0)[0]
    pick_a = aux if len(aux) <= n_aux else rng.choice(aux, n_aux, replace=False)
    pick_v = vtx if len(vtx) <= n_vertex else rng.choice(vtx, n_vertex, replace=False)
    return np.concatenate([pick_a, pick_v]).astype(np.int64)


@pytest.mark.parametrize("aux_balls", [1, 0])
@pytest.mark.parametrize("name", sorted(_cases()))
def test_balls_and_lists_against_oracle_cells(p2m, name, aux_balls):
    mesh = _cases()[name]()
    idx = p2m.P2MIndex(mesh.verts, mesh.tris, aux_balls=aux_balls)
    st = idx.stats()
    lo, hi = np.array(st["domain_lo"]), np.array(st["domain_hi"])
    diag = mesh.diag()
    sites, ref, kind = idx.sites()
    S = sites.astype(np.float64)
    boff, bc, br = idx.balls()
    off, ids = idx.lists()
    rng = np.random.default_rng(5)
    eps = 1e-6 * diag
    checked_aux = 0
    for s in _site_sample(kind, rng):
        corners = oracle.voronoi_cell(S, int(s), lo, hi)
        pc, pr = bc[boff[s]:boff[s + 1]], br[boff[s]:boff[s + 1]]
        row = set(ids[off[s]:off[s + 1]].tolist())
        if kind[s] == 0:
            v = ref[s]
            # v is the site's own mesh vertex (Section 3.1): a vertex of the mesh within two
            # lattice steps of the site
            assert np.min(np.linalg.norm(mesh.verts.astype(np.float64) - v, axis=1)) == 0.0
        else:
            checked_aux += 1
            d_true = oracle.closest(mesh.verts, mesh.tris, sites[s:s + 1])["dist"][0]
            # the reference point is a closest point of M to s: at the oracle's distance and on
            # M (near an axis of symmetry several points tie, and any of them is proj(s, M))
            assert abs(np.linalg.norm(S[s] - ref[s]) - d_true) <= 1e-6 * diag
            assert oracle.closest(mesh.verts, mesh.tris, ref[s:s + 1])["dist"][0] <= 1e-6 * diag
            v = ref[s]
        if kind[s] == 0 or aux_balls == 1:
            # Eq. 3 with reference point v
            ru = np.linalg.norm(corners - v, axis=1)
            merged = len(pr) > 0 and np.max(np.abs(pr - np.linalg.norm(pc - v, axis=1))) > 1e-12 * diag
            if not merged:
                # every kept ball is an oracle corner ball: centre at a corner, radius ||u - v||
                dc = np.min(np.linalg.norm(pc[:, None, :] - corners[None, :, :], axis=2), axis=1)
                assert np.max(dc) <= 2e-6 * diag, f"site {s}: a ball centre is no corner of the cell"
                assert np.max(np.abs(pr - np.linalg.norm(pc - v, axis=1))) <= 1e-12 * diag
            # every oracle corner ball lies inside some kept ball (dropped balls were contained)
            cover = np.min(np.linalg.norm(corners[:, None, :] - pc[None, :, :], axis=2) + ru[:, None] - pr[None, :],
                           axis=1)
            assert np.max(cover) <= 2e-6 * diag, f"site {s}: corner ball not covered ({np.max(cover):.3e})"
            oc, orad = corners, ru
        else:
            # Eq. 8: one ball around s enclosing the corner balls of reference point proj(s, M)
            r8 = oracle.aux_radius(S[s], corners, v)
            assert len(pr) == 1 and np.linalg.norm(pc[0] - S[s]) == 0.0
            assert abs(pr[0] - r8) <= 2e-6 * diag, f"aux site {s}: radius {pr[0]} vs Eq. 8 {r8}"
            oc, orad = S[s:s + 1], np.array([r8])
        # list lower bound from the oracle's balls (L- of the sandwich)
        mg = oracle.ball_margin(mesh.verts, mesh.tris, oc, orad)
        must = set(np.nonzero(mg <= -eps)[0].tolist())
        assert must <= row, f"site {s}: {len(must - row)} triangles of the oracle's balls missing"
        # Vertex Sphere Union: points x of the cell, B(x, ||x - v||) meets only listed triangles
        w = rng.dirichlet(np.ones(len(corners)) * 0.3, size=24)
        x = np.vstack([w @ corners, corners])
        mx = oracle.ball_margin(mesh.verts, mesh.tris, x, np.linalg.norm(x - v, axis=1))
        inside = set(np.nonzero(mx <= -eps)[0].tolist())
        assert inside <= row, f"site {s}: {len(inside - row)} triangles reached from inside the cell are missing"
    if name == "uv_sphere":
        assert checked_aux > 0, "the co-spherical UV sphere should get auxiliary sites"
