"""Signed distance (pseudonormal sign at the closest feature) against the FP64 oracle, whose
sign comes from an independent definition: the generalized winding number."""
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


def _signed(p2m, mesh, q):
    import torch
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    sd, _, _, _ = idx.query_signed(torch.from_numpy(np.ascontiguousarray(q)).cuda())
    torch.cuda.synchronize()
    return sd.cpu().numpy().astype(np.float64)


def test_cube_signed_closed_form(p2m):
    cube = W.unit_cube()
    rng = np.random.default_rng(21)
    q = (rng.random((20000, 3)) * 1.6 - 0.8).astype(np.float32)
    a = np.abs(q.astype(np.float64))
    inside = np.all(a < 0.5, 1)
    expect = np.where(inside, -(0.5 - a.max(1)), np.linalg.norm(np.maximum(a - 0.5, 0), axis=1))
    sd = _signed(p2m, cube, q)
    assert np.max(np.abs(sd - expect)) <= 1e-6 * cube.diag()


@pytest.mark.parametrize("name", ["noisy_sphere", "cylinder_cone", "uv_sphere"])
def test_signed_vs_winding_oracle(p2m, name):
    if name == "noisy_sphere":
        mesh, q = W.workload_large(20000, k=4)
    elif name == "cylinder_cone":
        mesh, q = W.workload_symmetric(20000, n_ang=64, n_ax=16)
    else:
        mesh, q = W.workload_small(20000)
    sd = _signed(p2m, mesh, q)
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    sd_ref, w = oracle.signed_distance(mesh.verts, mesh.tris, q, ref)
    diag = mesh.diag()
    assert np.max(np.abs(np.abs(sd) - ref["dist"])) <= 1e-6 * diag
    # the sign is decided where the point is not within rounding of the surface
    clear = ref["dist"] > 1e-5 * diag
    assert np.all(np.sign(sd[clear]) == np.sign(sd_ref[clear])), f"{(np.sign(sd[clear]) != np.sign(sd_ref[clear])).sum()} signs differ"
