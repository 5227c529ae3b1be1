"""Voronoi cells clipped on the GPU (FP64, one thread per cell) against the host clipper on the
same sites and triangulation, and the index built with device cells against one built with
host cells.  The host clipper is itself checked against brute force in test_voronoi_host.py."""
import numpy as np
import pytest

import oracle
import p2m_workloads as W
from test_voronoi_host import CASES, _domain

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2m():
    from paper_2605_00429_gb300 import build as b
    b.build()
    import paper_2605_00429_gb300 as p
    return p


def _same_region(a, b, tol):
    """Each corner set lies inside the other's convex hull, within tol.  Corner positions
    themselves may differ: where two bisector planes are nearly parallel (sites a lattice
    step apart in direction) the vertex between them is ill-conditioned along the thin edge,
    and the host and device clips place it differently by up to ~1e-6 of the domain while
    both stay on its planes to 1e-17; the regions then agree to ~1e-15."""
    from scipy.spatial import ConvexHull
    for p, q in ((a, b), (b, a)):
        eq = ConvexHull(q).equations
        if (p @ eq[:, :3].T + eq[:, 3]).max() > tol:
            return False
    return True


@pytest.mark.parametrize("name", sorted(CASES) + ["random_large"])
def test_device_cells_match_host(p2m, name):
    if name == "random_large":
        pts = (np.random.default_rng(12).random((20000, 3)) - 0.5).astype(np.float32)
    else:
        pts = CASES[name]
    lo, hi = _domain(pts)
    diag = np.linalg.norm(hi - lo)
    hs, hoff, hcor = p2m.voronoi_cells(pts, lo, hi, seed=3)
    ds, doff, dcor, n_host = p2m.voronoi_cells_device(pts, lo, hi, seed=3)
    np.testing.assert_array_equal(hs, ds)
    if name in ("random", "random_large"):
        assert n_host == 0
    bad = [i for i in range(len(pts))
           if not _same_region(hcor[hoff[i]:hoff[i + 1]], dcor[doff[i]:doff[i + 1]], 1e-9 * diag)]
    assert not bad, f"{len(bad)} cells differ, first {bad[:5]}"
    # every device corner is at least as close to its own site as to any other site
    own = np.repeat(np.arange(len(ds)), np.diff(doff))
    s64 = ds.astype(np.float64)
    _, dmin, _ = oracle.nearest_site(s64, dcor)
    assert np.max(np.linalg.norm(dcor - s64[own], axis=1) - dmin) < 1e-9 * diag


@pytest.mark.parametrize("mesh_name", ["noisy_sphere", "cylinder_cone"])
def test_index_with_device_cells(p2m, mesh_name):
    """The index built with device cells answers every query exactly as the one built with
    host cells (both lists contain the closest triangle; ties go to the lower id)."""
    import torch
    if mesh_name == "noisy_sphere":
        mesh = W.displace_radial(W.icosphere(4), 0.05, 3)
    else:
        mesh = W.cylinder_cone(96, 24, 12, 4)
    q = np.concatenate([W.queries_uniform_box(mesh, 20000, 1.2, 5),
                        W.queries_surface_gauss(mesh, 20000, 0.01 * mesh.diag(), 6)]).astype(np.float32)
    pts = torch.from_numpy(q).cuda()
    a = p2m.P2MIndex(mesh.verts, mesh.tris, gpu_cells=1)
    b = p2m.P2MIndex(mesh.verts, mesh.tris, gpu_cells=0)
    ra, rb = a.query(pts), b.query(pts)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ra[0].cpu().numpy(), rb[0].cpu().numpy())
    np.testing.assert_array_equal(ra[2].cpu().numpy(), rb[2].cpu().numpy())
    sa, sb = a.stats(), b.stats()
    assert sb["n_cells_host"] == 0
    # the augmentation's binning (device with gpu_cells=1, host otherwise) flags the same cells
    for k in ("n_sites", "n_aux_sites", "n_dense_cells", "aug_cell_median", "aug_cell_max", "n_delaunay_tets"):
        assert sa[k] == sb[k], k
    if mesh_name == "cylinder_cone":
        assert sa["n_aux_sites"] > 0


def test_augmentation_binning_elongated_domain(p2m):
    """Full-size cylinder + cone: its domain is 1.75x longer in z than in x, so the tau-grid
    needs a cell count per axis.  Device and host binning must flag the same cells."""
    mesh = W.cylinder_cone(512, 128, 64, 8)
    sa = p2m.P2MIndex(mesh.verts, mesh.tris, gpu_cells=1).stats()
    sb = p2m.P2MIndex(mesh.verts, mesh.tris, gpu_cells=0).stats()
    assert sa["n_dense_cells"] > 0
    for k in ("n_sites", "n_aux_sites", "n_dense_cells", "aug_cell_median", "aug_cell_max", "n_delaunay_tets"):
        assert sa[k] == sb[k], k
