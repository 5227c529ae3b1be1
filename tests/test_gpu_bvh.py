"""The triangle LBVH (Section 3.3 "Implementation Details") and the exact BVH search (K5) that
answers every query outside the domain box D.

* K5 in bulk: the paper's query box is 10x the model's bbox (Section 4), where almost every
  point lies outside D (1.5x the bbox) and takes the BVH search instead of the site lists.
  Tens of thousands of such points are checked element by element against the FP64 oracle.
* Structure: every triangle is reachable from the root exactly once, and every child box
  stored in a node contains its whole subtree (the triangle's vertices at a leaf).
"""
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


def _check(mesh, q, dist, closest, tri, bary):
    ref = oracle.closest(mesh.verts, mesh.tris, q)
    diag = mesh.diag()
    # 1e-6 diag; beyond 4 diag the FP32 result's own rounding (2^-22 d) is the bound
    tol = np.maximum(1e-6 * diag, 2.0 ** -22 * ref["dist"])
    err = np.abs(dist.astype(np.float64) - ref["dist"])
    assert np.all(err <= tol), f"distance error {np.max(err - tol):.3e} above tolerance"
    tie = (ref["dist2"] - ref["dist"]) <= tol
    assert np.all((tri == ref["tri"]) | tie), f"{np.sum((tri != ref['tri']) & ~tie)} triangle ids differ"
    assert np.all((np.linalg.norm(closest - ref["closest"], axis=1) <= 2 * tol) | tie)
    v = mesh.verts.astype(np.float64)
    p = np.einsum("nk,nkc->nc", bary.astype(np.float64), v[mesh.tris[tri]])
    assert np.all(np.linalg.norm(p - closest, axis=1) <= 2e-6 * diag + 2.0 ** -22 * ref["dist"])
    assert np.all(bary >= -1e-5)


def _paper_box_queries(mesh, n, seed):
    """Half uniform in the 10x bbox (the paper's query box), half in the 2x-4x shell."""
    far = W.queries_uniform_box(mesh, n // 2, 10.0, seed=seed)
    mid = W.queries_uniform_box(mesh, 4 * n, 4.0, seed=seed + 1)
    c = 0.5 * (mesh.verts.min(0) + mesh.verts.max(0))
    ext = 0.5 * (mesh.verts.max(0) - mesh.verts.min(0))
    shell = mid[np.any(np.abs(mid - c) > 2.0 * ext, axis=1)][: n - n // 2]
    return np.ascontiguousarray(np.concatenate([far, shell]).astype(np.float32))


@pytest.mark.parametrize("name", ["noisy_icosphere4", "cylinder_cone_96x24"])
def test_bvh_search_paper_query_box(p2m, name):
    import torch
    mesh = (W.displace_radial(W.icosphere(4), 0.05, 0) if name == "noisy_icosphere4"
            else W.cylinder_cone(n_ang=96, n_ax=24, n_cone=12, n_cap=4))
    q = _paper_box_queries(mesh, 24_000, seed=3)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    pts = torch.from_numpy(q).cuda()
    c = idx.counters(pts)
    assert c["n_outside"] >= 0.95 * len(q), "these points should almost all lie outside D"
    d, cl, t, b = idx.query(pts)
    torch.cuda.synchronize()
    _check(mesh, q, d.cpu().numpy(), cl.cpu().numpy(), t.cpu().numpy(), b.cpu().numpy())


def test_bvh_search_small_uv_sphere_in_domain(p2m):
    """In-domain queries answered through the site lists, for comparison on the same mesh."""
    import torch
    mesh, q = W.workload_small(20000)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    d, c, t, ba = idx.query(torch.from_numpy(q).cuda())
    torch.cuda.synchronize()
    _check(mesh, q, d.cpu().numpy(), c.cpu().numpy(), t.cpu().numpy(), ba.cpu().numpy())


@pytest.mark.parametrize("name", ["uv_sphere", "cylinder_cone_96x24", "single_triangle"])
def test_lbvh_structure(p2m, name):
    if name == "uv_sphere":
        mesh = W.uv_sphere(32, 16)
    elif name == "single_triangle":
        mesh = W._mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.5]], np.float32), np.array([[0, 1, 2]], np.int32))
    else:
        mesh = W.cylinder_cone(n_ang=96, n_ax=24, n_cone=12, n_cap=4)
    idx = p2m.P2MIndex(mesh.verts, mesh.tris)
    root, nodes, leaf_tri = idx.bvh()
    T = mesh.n_tris
    assert nodes.shape[0] == max(T - 1, 0)
    assert sorted(leaf_tri.tolist()) == list(range(T)), "leaf positions are not a permutation of the triangles"
    v = mesh.verts.astype(np.float32)
    tri_lo = v[mesh.tris].min(1)
    tri_hi = v[mesh.tris].max(1)
    if T == 1:
        assert root == ~0
        return
    child = nodes.view(np.int32)
    seen_leaf = np.zeros(T, np.int64)
    seen_node = np.zeros(T - 1, np.int64)
    stack = [root]
    while stack:
        a = stack.pop()
        assert 0 <= a < T - 1
        seen_node[a] += 1
        for k in range(2):
            lo, hi = nodes[a, 8 * k:8 * k + 3], nodes[a, 8 * k + 4:8 * k + 7]
            ref = int(child[a, 8 * k + 3])
            if ref < 0:
                leaf = ~ref
                seen_leaf[leaf] += 1
                f = leaf_tri[leaf]
                assert np.all(lo <= tri_lo[f]) and np.all(hi >= tri_hi[f]), f"leaf {leaf}: box misses its triangle"
            else:
                # the stored child box contains both boxes the child stores for its children
                for j in range(2):
                    assert np.all(lo <= nodes[ref, 8 * j:8 * j + 3]) and np.all(hi >= nodes[ref, 8 * j + 4:8 * j + 7]), \
                        f"node {a}: child box does not contain node {ref}'s children"
                stack.append(ref)
    assert np.all(seen_leaf == 1), "a triangle is unreachable or reachable twice"
    assert np.all(seen_node == 1), "an internal node is unreachable or shared"
