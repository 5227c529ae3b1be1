"""The allocation-free query entry point (p2m_query_noalloc), called through the C ABI.

It exists for callers that must not allocate device memory (a framework that owns all
device memory in its own pool, a latency-bound loop, an operator hook that may not
allocate); it runs the query kernels on a fixed scratch array inside the library.  This
file runs last so that a failure here cannot hide the other tests; it also passes alone in
a fresh process.  Two calls in a row must match p2m_query on the same index within the
query tolerance (the scratch array keeps the previous call's contents).  The calls run with
the library's host-side allocation fault injector armed (P2M_FAULT=alloc:1 makes the next
device allocation fail), so any allocation on this path would fail the test."""
import ctypes

import numpy as np
import pytest

import oracle
import p2m_workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_query_on_two_calls(monkeypatch):
    import torch
    from paper_2605_00429_gb300 import build as b
    b.build()
    import paper_2605_00429_gb300 as p2m
    L = p2m.lib()
    mesh, q = W.workload_large(2 * 150_000, k=4)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    tol = 1e-6 * mesh.diag()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, part in enumerate((q[:150_000], q[150_000:])):
        pts = torch.from_numpy(np.ascontiguousarray(part)).cuda()
        n = pts.shape[0]
        d_ref, c_ref, t_ref, b_ref = idx.query(pts)
        d = torch.full((n,), -1.0, device="cuda")
        c = torch.empty(n, 3, device="cuda")
        t = torch.full((n,), -1, device="cuda", dtype=torch.int32)
        bb = torch.empty(n, 3, device="cuda")
        torch.cuda.synchronize()
        # armed injector: the first device allocation from here on fails with P2M_ERR_OOM
        monkeypatch.setenv("P2M_FAULT", "alloc:1")
        rc = L.p2m_query_noalloc(idx._h, ctypes.c_void_p(pts.data_ptr()), n, ctypes.c_void_p(d.data_ptr()),
                                 ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                 ctypes.c_void_p(bb.data_ptr()), stream)
        torch.cuda.synchronize()
        monkeypatch.delenv("P2M_FAULT")
        assert rc == 0, L.p2m_last_error()
        d, d_ref = d.cpu().numpy(), d_ref.cpu().numpy()
        assert np.max(np.abs(d.astype(np.float64) - d_ref)) <= tol, f"call {call}"
        ref = oracle.closest(mesh.verts, mesh.tris, part[:2000])
        tie = (ref["dist2"] - ref["dist"]) <= tol
        tt = t.cpu().numpy()
        assert np.all((tt[:2000] == ref["tri"]) | tie), f"call {call}"
        assert np.max(np.abs(d[:2000] - ref["dist"])) <= tol
        assert np.max(np.abs(c.cpu().numpy() - c_ref.cpu().numpy())) <= 2 * tol
    # beyond the fixed scratch: a clear error, nothing launched
    big = torch.zeros(p2m.NOALLOC_MAX_QUERIES + 1, 3, device="cuda")
    out = torch.empty(big.shape[0], device="cuda")
    rc = L.p2m_query_noalloc(idx._h, ctypes.c_void_p(big.data_ptr()), big.shape[0], ctypes.c_void_p(out.data_ptr()),
                             None, None, None, stream)
    assert rc == -6 and b"at most" in L.p2m_last_error()
