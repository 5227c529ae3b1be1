"""Moving the mesh and the limits of the boundary.

* p2m_update_vertices: the vertices move (same topology), the index is rebuilt from them, and
  queries match the FP64 oracle on the moved mesh;
* the autograd Function refuses vertices that differ from the index's (stale gradients), and
  accepts them again after update_vertices;
* the deterministic vertex-gradient sum stays exact for gradient scales from 1e-20 to 1e12
  (its fixed-point unit is picked per call) and reports a non-finite gradient as LIMIT;
* a call with more than 2^31 - 1 points is refused before anything is launched.
"""
import ctypes

import numpy as np
import pytest

import oracle
import p2m_workloads as W
from test_gpu_query import check_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2m():
    from paper_2605_00429_gb300 import build as b
    b.build()
    import paper_2605_00429_gb300 as p
    return p


def test_update_vertices_parity(p2m):
    import torch
    mesh = W.displace_radial(W.icosphere(3), 0.05, 0)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    moved = W.displace_radial(W.icosphere(3), 0.12, 5)  # same topology, other positions
    moved_v = (moved.verts * np.array([1.3, 0.8, 1.0], np.float32) + np.array([0.2, -0.1, 0.05], np.float32))
    moved = W._mesh(moved_v.astype(np.float32), mesh.tris)
    idx.update_vertices(torch.from_numpy(moved.verts).cuda())
    q = W.queries_uniform_box(moved, 20000, 1.2, seed=9)
    d, c, t, b = idx.query(torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    check_parity(moved, q, (d.cpu().numpy(), c.cpu().numpy(), t.cpu().numpy(), b.cpu().numpy()))
    assert idx.stats()["bbox_diag"] == pytest.approx(moved.diag(), rel=1e-6)


def test_unsigned_distance_refuses_stale_vertices(p2m):
    import torch
    mesh = W.displace_radial(W.icosphere(2), 0.05, 0)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    q = torch.from_numpy(W.queries_surface_gauss(mesh, 500, 0.02, seed=1)).cuda()
    verts = torch.from_numpy(mesh.verts).cuda().requires_grad_(True)
    p2m.unsigned_distance(q, verts, idx).sum().backward()  # same vertices: accepted
    with torch.no_grad():
        verts += 0.01  # moved in place, index not updated
    with pytest.raises(ValueError):
        p2m.unsigned_distance(q, verts, idx)
    idx.update_vertices(verts.detach())
    verts.grad = None
    d = p2m.unsigned_distance(q, verts, idx)
    d.sum().backward()
    torch.cuda.synchronize()
    ref = oracle.closest(verts.detach().cpu().numpy(), mesh.tris, q.cpu().numpy())
    assert np.max(np.abs(d.detach().cpu().numpy() - ref["dist"])) <= 1e-6 * mesh.diag()
    other = torch.from_numpy(mesh.verts).cuda()  # a different tensor with the old positions
    with pytest.raises(ValueError):
        p2m.unsigned_distance(q, other, idx)


@pytest.mark.parametrize("scale", [1e-20, 1.0, 1e12])
def test_deterministic_vertex_sum_scales(p2m, scale):
    """Fixed-point vertex sums at extreme gradient scales: bit-identical on a second call,
    equal to the float-atomic sums of the same contributions up to FP32 summation error, and
    equal to the FP64 analytic gradient up to the closest point's FP32 error."""
    import torch
    mesh, q = W.workload_diff(50_000, k=3)
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    diag = mesh.diag()
    # medial ties and points almost on the surface (ill-conditioned direction) carry no gradient
    ok = ((ref["dist2"] - ref["dist"]) > 1e-6 * diag) & (ref["dist"] > 1e-3 * diag)
    g = np.where(ok, scale * (1.0 + np.random.default_rng(0).random(len(q))), 0.0).astype(np.float32)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    idx_f = p2m.P2MIndex(mesh.verts, mesh.tris, deterministic=0)
    pts = torch.from_numpy(q).cuda()
    _, _, tri, bary = idx.query(pts)
    gd = torch.from_numpy(g).cuda()
    outs = []
    for which in (idx, idx, idx_f):
        gv = torch.zeros(mesh.n_verts, 3, device="cuda")
        which.backward(pts, tri, bary, gd, None, gv)
        torch.cuda.synchronize()
        outs.append(gv.cpu().numpy().astype(np.float64))
    assert np.array_equal(outs[0], outs[1])
    assert np.all(np.isfinite(outs[0]))
    mass = np.zeros(mesh.n_verts)
    tv = mesh.tris[tri.cpu().numpy()]
    b = bary.cpu().numpy().astype(np.float64)
    for k in range(3):
        np.add.at(mass, tv[:, k], np.abs(g.astype(np.float64)) * np.abs(b[:, k]))
    assert np.all(np.abs(outs[0] - outs[2]).max(1) <= 1e-5 * mass)
    _, gv_ref = oracle.grad_analytic(mesh.verts, mesh.tris, q, g.astype(np.float64), ref)
    assert np.all(np.abs(outs[0] - gv_ref).max(1) <= 1e-2 * mass)


def test_nonfinite_gradient_reports_limit(p2m):
    import torch
    mesh, q = W.workload_diff(2000, k=2)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    pts = torch.from_numpy(q).cuda()
    _, _, tri, bary = idx.query(pts)
    g = torch.ones(len(q), device="cuda")
    g[17] = float("nan")
    gv = torch.zeros(mesh.n_verts, 3, device="cuda")
    idx.backward(pts, tri, bary, g, None, gv)
    with pytest.raises(p2m.P2MError) as e:
        idx.counters(pts)  # the next synchronising call reports it
    assert e.value.code == -6
    assert torch.count_nonzero(gv).item() == 0
    idx.counters(pts)  # and the index stays usable


def test_more_than_int32_points_refused(p2m):
    import torch
    mesh = W.uv_sphere(8, 6)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    L = p2m.lib()
    buf = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    n = (1 << 31)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the size check runs before any launch, so the short buffers are never touched
    assert L.p2m_query(idx._h, p, n, p, None, None, None, s) == -6
    assert b"2^31" in L.p2m_last_error()
    assert L.p2m_nearest_site(idx._h, p, n, p, s) == -6
    assert L.p2m_query_signed(idx._h, p, n, p, None, None, None, s) == -6
    d, _, _, _ = idx.query(torch.zeros(3, 3, device="cuda"))
    torch.cuda.synchronize()
    assert np.isfinite(d.cpu().numpy()).all()
