"""GPU parity of the exact BVH branch-and-bound search (K5) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import p2m_workloads as W

pytestmark = pytest.mark.gpu


def _check(mesh, q, dist, closest, tri, bary):
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    tol = 1e-6 * mesh.diag()
    d = dist.astype(np.float64)
    assert np.max(np.abs(d - ref["dist"])) <= tol
    tie = (ref["dist2"] - ref["dist"]) <= tol
    assert np.all((tri == ref["tri"]) | tie)
    assert np.max(np.linalg.norm(closest - ref["closest"], axis=1)[~tie]) <= 2 * tol
    # barycentrics reproduce the closest point on the reported triangle
    v = mesh.verts.astype(np.float64)
    p = np.einsum("nk,nkc->nc", bary.astype(np.float64), v[mesh.tris[tri]])
    assert np.max(np.linalg.norm(p - closest, axis=1)) <= 2 * tol
    assert np.all(bary >= -1e-5)


def test_bvh_closest_small():
    import torch
    import paper_2605_00429_gb300 as p2m
    from paper_2605_00429_gb300 import build as b
    b.build()
    mesh, q = W.workload_small(20000)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    d, c, t, ba = idx.query(torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    _check(mesh, q, d.cpu().numpy(), c.cpu().numpy(), t.cpu().numpy(), ba.cpu().numpy())
