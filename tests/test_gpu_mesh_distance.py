"""Mesh-to-mesh distance on the GPU against the FP64 oracle on the same lattice samples."""
import numpy as np
import pytest

import oracle
import p2m_workloads as W

pytestmark = pytest.mark.gpu


def _samples(mesh, k):
    v = mesh.verts.astype(np.float64)
    a, b, c = v[mesh.tris[:, 0]], v[mesh.tris[:, 1]], v[mesh.tris[:, 2]]
    if k == 0:
        return np.concatenate([a, b, c])
    pts = []
    for i in range(k + 1):
        for j in range(k - i + 1):
            pts.append(((k - i - j) * a + i * b + j * c) / k)
    return np.concatenate(pts)


@pytest.mark.parametrize("k", [0, 3])
def test_mesh_distance_vs_oracle(k):
    from paper_2605_00429_gb300 import build as bld
    bld.build()
    import paper_2605_00429_gb300 as p2m
    a = W.displace_radial(W.icosphere(3), 0.05, 1)
    b = W.capped_cylinder(24, 6)
    b.verts[:] = b.verts * np.float32(0.4) + np.float32(0.3)  # a smaller shape partly inside
    idx = p2m.P2MIndex(a.verts, a.tris)
    mn, mx, mean = idx.mesh_distance(b.verts, b.tris, k)
    ref = oracle.closest(a.verts, a.tris, _samples(b, k).astype(np.float32))["dist"]
    tol = 2e-6 * a.diag()
    assert abs(mn - ref.min()) <= tol and abs(mx - ref.max()) <= tol and abs(mean - ref.mean()) <= tol


def test_mesh_distance_pair_vs_oracle():
    """Both directions and the symmetric Hausdorff distance over the samples."""
    import paper_2605_00429_gb300 as p2m
    a = W.displace_radial(W.icosphere(3), 0.05, 1)
    b = W.capped_cylinder(24, 6)
    b.verts[:] = b.verts * np.float32(0.4) + np.float32(0.3)
    ia, ib = p2m.P2MIndex(a.verts, a.tris), p2m.P2MIndex(b.verts, b.tris)
    k = 2
    r = ia.mesh_distance_pair(ib, k)
    d_ba = oracle.closest(a.verts, a.tris, _samples(b, k).astype(np.float32))["dist"]
    d_ab = oracle.closest(b.verts, b.tris, _samples(a, k).astype(np.float32))["dist"]
    tol = 2e-6 * max(a.diag(), b.diag())
    for got, ref in ((r["b_to_a"], d_ba), (r["a_to_b"], d_ab)):
        assert abs(got[0] - ref.min()) <= tol and abs(got[1] - ref.max()) <= tol and abs(got[2] - ref.mean()) <= tol
    assert abs(r["hausdorff"] - max(d_ba.max(), d_ab.max())) <= tol
