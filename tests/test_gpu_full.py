"""Full-size GPU parity: every workload at its full size, built with the default parameters
and queried in the same launch configuration bench.py times, checked against the FP64 oracle
on sampled outputs (the oracle answers a sampled query exactly, one by one)."""
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


def _sampled(p2m, mesh, q, n_check=3000, seed=0):
    import torch
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    out = idx.query(torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    d = out[0].cpu().numpy()
    assert np.all(np.isfinite(d)) and np.all(d >= 0)
    t = out[2].cpu().numpy()
    assert t.min() >= 0 and t.max() < mesh.n_tris
    sel = np.random.default_rng(seed).choice(len(q), n_check, replace=False)
    check_parity(mesh, q[sel], tuple(o.cpu().numpy()[sel] for o in out))
    return idx


def test_full_large(p2m):
    """icosphere(6) + noise, 81,920 tris, 10M queries."""
    mesh, q = W.workload_large()
    idx = _sampled(p2m, mesh, q)
    st = idx.stats()
    assert st["max_row"] < mesh.n_tris


def test_full_symmetric(p2m):
    """cylinder + cone, 203,776 tris, aux sites on, 10M queries (70% near the surface)."""
    mesh, q = W.workload_symmetric()
    assert mesh.n_tris == 203_776
    idx = _sampled(p2m, mesh, q)
    assert idx.stats()["n_aux_sites"] > 0


def test_full_batch(p2m):
    """256 meshes (T log-uniform in [500, 200k]), ~39M queries, one persistent launch."""
    import torch
    meshes, queries = W.workload_batch(256)
    idx = p2m.P2MIndex.batch([(m.verts, m.tris) for m in meshes])
    off = np.concatenate([[0], np.cumsum([len(q) for q in queries])]).astype(np.int64)
    out = idx.batch_query(torch.from_numpy(np.concatenate(queries)).cuda(), off, mode=0, use_graph=True)
    torch.cuda.synchronize()
    d, c, t, b = [o.cpu().numpy() for o in out]
    rng = np.random.default_rng(4)
    for i, (m, q) in enumerate(zip(meshes, queries)):
        sel = rng.choice(len(q), min(25, len(q)), replace=False)
        g = off[i] + sel
        check_parity(m, q[sel], (d[g], c[g], t[g], b[g]))


def test_full_diff(p2m):
    """icosphere(5) + noise, 1M near-surface queries, L = sum d^2: backward to points and to
    vertices checked on a sampled subset (upstream gradient zero elsewhere)."""
    import torch
    mesh, q = W.workload_diff()
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    pts = torch.from_numpy(q).cuda()
    d, _, tri, bary = idx.query(pts)
    sel = np.random.default_rng(5).choice(len(q), 20000, replace=False)
    ref = oracle.closest(mesh.verts, mesh.tris, q[sel])
    diag = mesh.diag()
    ok = (ref["dist2"] - ref["dist"]) > 1e-6 * diag
    g = np.zeros(len(q))
    g[sel[ok]] = 2.0 * ref["dist"][ok]
    gq = torch.empty_like(pts)
    gv = torch.zeros(mesh.n_verts, 3, device="cuda")
    idx.backward(pts, tri, bary, torch.from_numpy(g.astype(np.float32)).cuda(), gq, gv)
    torch.cuda.synchronize()
    gq_ref, gv_ref = oracle.grad_analytic(mesh.verts, mesh.tris, q[sel], g[sel], ref)
    assert np.max(np.abs(gq.cpu().numpy()[sel] - gq_ref)) <= 4e-6 * diag + 1e-4 * np.max(np.abs(gq_ref))
    assert np.max(np.abs(gv.cpu().numpy() - gv_ref)) <= 1e-4 * np.max(np.abs(gv_ref)) + 4e-5 * diag
