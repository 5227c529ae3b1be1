"""GPU parity of the batched persistent query (K6) against the per-mesh forward and the FP64
oracle: graph replay, graph re-capture on new buffers, the per-mesh mode, empty meshes."""
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


@pytest.fixture(scope="module")
def batch(p2m):
    meshes, queries = W.workload_batch(12, seed=3, t_range=(200, 20_000), q_range=(500, 40_000))
    queries[3] = queries[3][:0]  # an empty query set
    idx = p2m.P2MIndex.batch([(m.verts, m.tris) for m in meshes])
    off = np.concatenate([[0], np.cumsum([len(q) for q in queries])]).astype(np.int64)
    pts = np.concatenate(queries, 0)
    return meshes, queries, idx, off, pts


def _run(p2m, idx, pts, off, mode, use_graph, out=None):
    import torch
    t = torch.from_numpy(pts).cuda()
    res = idx.batch_query(t, off, mode=mode, use_graph=use_graph, out=out)
    torch.cuda.synchronize()
    return [r.cpu().numpy() for r in res]


def test_batch_modes_agree(p2m, batch):
    meshes, queries, idx, off, pts = batch
    a = _run(p2m, idx, pts, off, 0, True)
    b = _run(p2m, idx, pts, off, 0, False)
    c = _run(p2m, idx, pts, off, 1, False)
    a2 = _run(p2m, idx, pts, off, 0, True)  # graph replay (new output buffers: re-capture)
    for x in (b, c, a2):
        assert np.array_equal(a[0], x[0]) and np.array_equal(a[2], x[2])


def test_batch_graph_replay_same_buffers(p2m, batch):
    import torch
    meshes, queries, idx, off, pts = batch
    n = len(pts)
    out = (torch.empty(n, device="cuda"), torch.empty(n, 3, device="cuda"),
           torch.empty(n, device="cuda", dtype=torch.int32), torch.empty(n, 3, device="cuda"))
    r1 = _run(p2m, idx, pts, off, 0, True, out)
    for o in out:
        o.zero_()
    r2 = _run(p2m, idx, pts, off, 0, True, out)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[2], r2[2])


def test_batch_vs_oracle(p2m, batch):
    meshes, queries, idx, off, pts = batch
    d, c, t, b = _run(p2m, idx, pts, off, 0, True)
    for i, (m, q) in enumerate(zip(meshes, queries)):
        if len(q) == 0:
            continue
        sl = slice(off[i], off[i] + min(len(q), 1500))
        check_parity(m, q[:1500], (d[sl], c[sl], t[sl], b[sl]))


def test_batch_bad_offsets(p2m, batch):
    import torch
    meshes, queries, idx, off, pts = batch
    t = torch.from_numpy(pts).cuda()
    bad = off.copy()
    bad[2], bad[3] = bad[3], bad[2] - 1
    with pytest.raises(p2m.P2MError):
        idx.batch_query(t, bad)
