"""GPU backward (K4) and the autograd Function against the FP64 oracle: the analytic gradient
from the oracle's closest points, and central finite differences in FP64."""
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


def _grads(p2m, mesh, q, g, **params):
    import torch
    idx = p2m.P2MIndex(mesh.verts, mesh.tris, **params)
    pts = torch.from_numpy(q).cuda()
    d, _, tri, bary = idx.query(pts)
    gq = torch.empty_like(pts)
    gv = torch.zeros(mesh.n_verts, 3, device="cuda")
    idx.backward(pts, tri, bary, torch.from_numpy(g.astype(np.float32)).cuda(), gq, gv)
    torch.cuda.synchronize()
    return idx, d.cpu().numpy(), tri.cpu().numpy(), gq.cpu().numpy(), gv.cpu().numpy()


def test_backward_vs_analytic(p2m):
    """Config-5 mesh (icosphere(5) + noise), 100k near-surface queries, L = sum d^2."""
    mesh, q = W.workload_diff(100_000)
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    diag = mesh.diag()
    tie = (ref["dist2"] - ref["dist"]) <= 1e-6 * diag
    g = np.where(tie, 0.0, 2.0 * ref["dist"])  # dL/dd for L = sum d^2, ties excluded
    _, d, tri, gq, gv = _grads(p2m, mesh, q, g)
    gq_ref, gv_ref = oracle.grad_analytic(mesh.verts, mesh.tris, q, g, ref)
    # g_q = 2 (q - p): the closest point is within 2e-6 diag
    assert np.max(np.abs(gq - gq_ref)) <= 2 * 2e-6 * diag + 1e-4 * np.max(np.abs(gq_ref))
    # vertex sums: per-vertex tolerance from the mass of the contributions
    mass = np.zeros(mesh.n_verts)
    cnt = np.zeros(mesh.n_verts)
    tv = mesh.tris[ref["tri"]]
    for k in range(3):
        np.add.at(mass, tv[:, k], np.abs(g) * ref["bary"][:, k])
        np.add.at(cnt, tv[:, k], (g != 0).astype(float))
    tol = 1e-4 * mass + 4e-6 * diag * np.sqrt(np.maximum(cnt, 1)) * 2 + 1e-6
    assert np.all(np.abs(gv - gv_ref).max(1) <= tol)


def test_backward_vs_finite_differences(p2m):
    """icosphere(2) + noise (320 tris), 1k points, FP64 central differences."""
    mesh = W.displace_radial(W.icosphere(2), 0.05, 0)
    q = W.queries_surface_gauss(mesh, 1000, 0.01 * mesh.diag(), seed=4)
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    ok = ((ref["dist2"] - ref["dist"]) > 1e-4) & (ref["dist"] > 1e-4)
    g = np.where(ok, 2.0 * ref["dist"], 0.0)
    _, d, tri, gq, gv = _grads(p2m, mesh, q, g)
    qi = np.nonzero(ok)[0][:100]
    fq, _ = oracle.grad_fd(mesh.verts, mesh.tris, q, g, 1e-6, query_idx=qi, vert_idx=[])
    assert np.max(np.abs(gq[qi] - fq)) <= 1e-4 * np.max(np.abs(fq)) + 1e-5
    vi = np.random.default_rng(0).choice(mesh.n_verts, 24, replace=False)
    _, fv = oracle.grad_fd(mesh.verts, mesh.tris, q, g, 1e-6, query_idx=[], vert_idx=vi)
    assert np.max(np.abs(gv[vi] - fv)) <= 1e-4 * np.max(np.abs(fv)) + 1e-4


def test_backward_deterministic(p2m):
    mesh, q = W.workload_diff(200_000)
    g = np.random.default_rng(1).normal(size=len(q))
    a = _grads(p2m, mesh, q, g, deterministic=1)[4]
    b = _grads(p2m, mesh, q, g, deterministic=1)[4]
    assert np.array_equal(a, b)
    c = _grads(p2m, mesh, q, g, deterministic=0)[4]
    assert np.allclose(a, c, atol=1e-3, rtol=1e-4)


def test_autograd_function(p2m):
    import torch
    mesh, q = W.workload_diff(50_000)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    pts = torch.from_numpy(q).cuda().requires_grad_(True)
    verts = torch.from_numpy(mesh.verts).cuda().requires_grad_(True)
    d = p2m.unsigned_distance(pts, verts, idx)
    (d * d).sum().backward()
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    gq_ref = 2.0 * (q.astype(np.float64) - ref["closest"])
    tie = (ref["dist2"] - ref["dist"]) <= 1e-6 * mesh.diag()
    assert np.max(np.abs(pts.grad.cpu().numpy() - gq_ref)[~tie]) <= 4e-6 * mesh.diag()
    assert verts.grad is not None and torch.isfinite(verts.grad).all()


@pytest.mark.parametrize("n_queries,chunks", [(300_000, 0), (2_500_000, 3)])
def test_query_host_matches_device(p2m, n_queries, chunks):
    """The host-buffer pipeline (one chunk, or three 1M-point chunks on three streams) gives
    the device query's answers bit for bit."""
    import torch
    mesh, q = W.workload_large(n_queries, k=4)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris, pipe_chunks=chunks)
    d, c, t, b = idx.query(torch.from_numpy(q).cuda())
    hd = np.empty(len(q), np.float32)
    hc = np.empty((len(q), 3), np.float32)
    ht = np.empty(len(q), np.int32)
    hb = np.empty((len(q), 3), np.float32)
    idx.query_host(q, hd, hc, ht, hb)
    assert np.array_equal(hd, d.cpu().numpy()) and np.array_equal(ht, t.cpu().numpy())
    assert np.array_equal(hc, c.cpu().numpy()) and np.array_equal(hb, b.cpu().numpy())
