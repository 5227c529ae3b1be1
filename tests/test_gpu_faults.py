"""Failure detection without any GPU fault: host-side injected failures (P2M_FAULT) and bad
inputs come back as error codes, and the library stays usable afterwards."""
import os

import numpy as np
import pytest

import p2m_workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p2m():
    from paper_2605_00429_gb300 import build as b
    b.build()
    import paper_2605_00429_gb300 as p
    return p


@pytest.fixture
def mesh():
    return W.workload_small(10)[0]


def _build(p2m, mesh):
    return p2m.P2MIndex(mesh.verts, mesh.tris)


@pytest.mark.parametrize("k", [1, 3, 7, 15])
def test_injected_allocation_failure(p2m, mesh, monkeypatch, k):
    monkeypatch.setenv("P2M_FAULT", f"alloc:{k}")
    with pytest.raises(p2m.P2MError) as e:
        _build(p2m, mesh)
    assert e.value.code == -3 and "injected" in str(e.value)
    monkeypatch.delenv("P2M_FAULT")
    idx = _build(p2m, mesh)  # recovers
    assert idx.stats()["n_sites"] > 0


def test_injected_triangulation_failure(p2m, mesh, monkeypatch):
    monkeypatch.setenv("P2M_FAULT", "delaunay")
    with pytest.raises(p2m.P2MError) as e:
        _build(p2m, mesh)
    assert e.value.code == -9
    monkeypatch.delenv("P2M_FAULT")
    assert _build(p2m, mesh).stats()["nnz"] > 0


def test_bad_inputs_are_errors(p2m, mesh):
    import torch
    with pytest.raises(p2m.P2MError) as e:
        p2m.P2MIndex(mesh.verts, mesh.tris[:0])
    assert e.value.code == -4
    with pytest.raises(p2m.P2MError):
        p2m.P2MIndex(np.zeros((5, 3), np.float32), np.array([[0, 1, 2]], np.int32))  # all vertices coincide
    with pytest.raises(p2m.P2MError):
        p2m.P2MIndex(mesh.verts, mesh.tris, domain_scale=0.5)
    with pytest.raises(p2m.P2MError):
        p2m.P2MIndex(mesh.verts, mesh.tris, ring_sites=5)
    idx = _build(p2m, mesh)
    with pytest.raises(p2m.P2MError):
        idx.batch_query(torch.zeros(4, 3, device="cuda"), [1, 4])  # offsets must start at 0
    with pytest.raises(p2m.P2MError):
        idx.batch_query(torch.zeros(4, 3, device="cuda"), [0, 4], mode=7)
    # a single-mesh query still works after the errors
    d, _, _, _ = idx.query(torch.zeros(1, 3, device="cuda"))
    torch.cuda.synchronize()
    assert np.isfinite(d.cpu().numpy()).all()
