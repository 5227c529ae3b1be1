"""P2M++ FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA path (``paper_2605_00429_gb300``) and
imports nothing from it.

Contents (each a plain, slow definition; see ``oracle.c`` for the C part):

* ``closest``       brute-force FP64 closest point over all triangles (the result the
                    localised search must reproduce, Section 3.3, Eq. 2).
* ``nearest_site``  brute-force FP64 nearest site (cell locate, Section 3.3).
* ``ball_margin``   per triangle, min over balls of d(u, f) - r_u (Eq. 3, Eq. 8).
* ``aux_radius``    Eq. 8 for an off-surface site.
* ``voronoi_cell``  corners of one site's Voronoi cell clipped to the domain box, from the
                    bisectors of every other site (no neighbour search).
* ``winding``       generalized winding number (inside / outside of a closed mesh), the
                    plain definition behind the sign of the signed distance.
* ``grad_analytic`` gradient of sum_i g_i d(q_i, M) w.r.t. queries and vertices, from the
                    closest-point barycentrics.
* ``grad_fd``       central finite differences of the same loss, FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_oracle.so with gcc (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-shared", "-fPIC", "-std=c11", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int64
        _lib.orc_closest.argtypes = [P, I, P, I, P, I, P, P, P, P, P]
        _lib.orc_nearest_site.argtypes = [P, I, P, I, P, P, P]
        _lib.orc_ball_margin.argtypes = [P, I, P, I, P, P, I, P]
        _lib.orc_point_triangle.argtypes = [P, P, P, P, P, P]
        _lib.orc_point_triangle.restype = ctypes.c_double
        _lib.orc_num_threads.restype = ctypes.c_int
        _lib.orc_dist_f64.argtypes = [P, I, P, I, P, I, P]
        _lib.orc_winding.argtypes = [P, I, P, I, P, I, P]
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(_load().orc_num_threads())


def point_triangle(q, a, b, c):
    """FP64 closest point of one triangle: returns (dist, closest[3], bary[3])."""
    arr = [np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(3)) for x in (q, a, b, c)]
    cl = np.zeros(3)
    ba = np.zeros(3)
    d = _load().orc_point_triangle(*[_ptr(x) for x in arr], _ptr(cl), _ptr(ba))
    return float(d), cl, ba


def closest(verts, tris, pts):
    """Brute force over all triangles.  Returns dict of FP64 dist, closest[n,3], tri (int64),
    bary[n,3] and dist2 (second-best triangle distance)."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    p = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
    n = p.shape[0]
    out = dict(dist=np.empty(n), closest=np.empty((n, 3)), tri=np.empty(n, np.int64),
               bary=np.empty((n, 3)), dist2=np.empty(n))
    _load().orc_closest(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(p), n,
                        _ptr(out["dist"]), _ptr(out["closest"]), _ptr(out["tri"]),
                        _ptr(out["bary"]), _ptr(out["dist2"]))
    return out


def nearest_site(sites, pts):
    """Brute-force nearest site (FP64), lower index on ties.  Returns (site, dist, dist2)."""
    s = np.ascontiguousarray(sites, dtype=np.float64).reshape(-1, 3)
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    n = p.shape[0]
    site = np.empty(n, np.int64)
    d = np.empty(n)
    d2 = np.empty(n)
    _load().orc_nearest_site(_ptr(s), s.shape[0], _ptr(p), n, _ptr(site), _ptr(d), _ptr(d2))
    return site, d, d2


def ball_margin(verts, tris, centres, radii):
    """margin[f] = min_k d(u_k, f) - r_k.  f meets the union of the balls iff margin <= 0."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    m = np.empty(t.shape[0])
    _load().orc_ball_margin(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(c), _ptr(r), c.shape[0], _ptr(m))
    return m


def winding(verts, tris, pts):
    """Generalized winding number (sum of signed solid angles / 4 pi): 1 inside a closed
    outward-oriented mesh, 0 outside."""
    v = np.ascontiguousarray(verts, dtype=np.float32)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    p = np.ascontiguousarray(pts, dtype=np.float32).reshape(-1, 3)
    w = np.empty(p.shape[0])
    _load().orc_winding(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(p), p.shape[0], _ptr(w))
    return w


def signed_distance(verts, tris, pts, res=None):
    """Signed distance of a closed mesh: -d(q, M) inside (winding number > 1/2), +d outside."""
    if res is None:
        res = closest(verts, tris, pts)
    w = winding(verts, tris, pts)
    return np.where(w > 0.5, -res["dist"], res["dist"]), w


def voronoi_cell(sites, i, dom_lo, dom_hi):
    """Corners of the Voronoi cell of site i clipped to the box D = [dom_lo, dom_hi], in FP64.

    The cell is the plain definition {x in D : ||x - s_i|| <= ||x - s_j|| for every j != i}
    (Section 3.1: each site owns the points nearer to it than to any other site).  Squaring
    both sides, each other site gives the half-space 2 x.(s_j - s_i) <= |s_j|^2 - |s_i|^2;
    all of them are used, with the six faces of D.  The vertices of that intersection of
    half-spaces come from Qhull (scipy.spatial.HalfspaceIntersection), a library step, started
    from the interior point s_i.  A vertex where more than three planes meet may be listed more
    than once.  Needs distinct sites and s_i strictly inside D."""
    from scipy.spatial import HalfspaceIntersection
    S = np.asarray(sites, dtype=np.float64).reshape(-1, 3)
    lo = np.asarray(dom_lo, dtype=np.float64).reshape(3)
    hi = np.asarray(dom_hi, dtype=np.float64).reshape(3)
    s = S[i]
    other = np.delete(S, i, axis=0)
    # rows (a, b) of a.x + b <= 0
    bis = np.c_[2.0 * (other - s), -(np.sum(other * other, axis=1) - np.dot(s, s))]
    box = np.array([[-1, 0, 0, lo[0]], [0, -1, 0, lo[1]], [0, 0, -1, lo[2]],
                    [1, 0, 0, -hi[0]], [0, 1, 0, -hi[1]], [0, 0, 1, -hi[2]]], dtype=np.float64)
    hs = HalfspaceIntersection(np.vstack([bis, box]), s)
    return np.asarray(hs.intersections, dtype=np.float64)


def aux_radius(site, corners, proj):
    """Eq. 8: r = max_u (||s - u|| + ||u - proj(s, M)||) over the corners u of the site's cell."""
    s = np.asarray(site, dtype=np.float64).reshape(3)
    u = np.asarray(corners, dtype=np.float64).reshape(-1, 3)
    p = np.asarray(proj, dtype=np.float64).reshape(3)
    return float(np.max(np.linalg.norm(u - s, axis=1) + np.linalg.norm(u - p, axis=1)))


def grad_analytic(verts, tris, pts, grad_dist, res=None):
    """Gradient of L = sum_i g_i d(q_i, M).

    With p the closest point on triangle f = (v0, v1, v2) and p = sum_k b_k v_k, the
    distance d = ||q - p|| has dd/dq = (q - p)/d and dd/dv_k = -b_k (q - p)/d (the
    closest point moves with the triangle; the envelope theorem removes the dependence of
    b on v).  At d = 0 the gradient is taken as 0.
    """
    if res is None:
        res = closest(verts, tris, pts)
    q = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    g = np.asarray(grad_dist, dtype=np.float64).reshape(-1)
    diff = q - res["closest"]
    d = res["dist"]
    unit = np.where(d[:, None] > 0, diff / np.where(d > 0, d, 1.0)[:, None], 0.0)
    gq = g[:, None] * unit
    gv = np.zeros((np.asarray(verts).shape[0], 3))
    tri_v = np.asarray(tris)[res["tri"]]
    for k in range(3):
        np.add.at(gv, tri_v[:, k], -(g * res["bary"][:, k])[:, None] * unit)
    return gq, gv


def _dist_fp64(verts64, tris, pts64):
    """FP64 d(q, M) without any FP32 rounding of inputs (for finite differences)."""
    v = np.ascontiguousarray(verts64, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    q = np.ascontiguousarray(pts64, dtype=np.float64).reshape(-1, 3)
    out = np.empty(q.shape[0])
    _load().orc_dist_f64(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(q), q.shape[0], _ptr(out))
    return out


def grad_fd(verts, tris, pts, grad_dist, h, query_idx=None, vert_idx=None):
    """Central finite differences of L = sum_i g_i d(q_i, M) in FP64 (slow: small meshes only).

    Returns (gq[len(query_idx),3], gv[len(vert_idx),3])."""
    v64 = np.asarray(verts, dtype=np.float64).copy()
    q64 = np.asarray(pts, dtype=np.float64).reshape(-1, 3).copy()
    g = np.asarray(grad_dist, dtype=np.float64).reshape(-1)
    t = np.asarray(tris, dtype=np.int64)
    qi = np.arange(q64.shape[0]) if query_idx is None else np.asarray(query_idx)
    vi = np.arange(v64.shape[0]) if vert_idx is None else np.asarray(vert_idx)
    gq = np.zeros((len(qi), 3))
    for r, i in enumerate(qi):
        for k in range(3):
            qp, qm = q64[i].copy(), q64[i].copy()
            qp[k] += h
            qm[k] -= h
            gq[r, k] = g[i] * (_dist_fp64(v64, t, qp)[0] - _dist_fp64(v64, t, qm)[0]) / (2 * h)
    gv = np.zeros((len(vi), 3))
    for r, j in enumerate(vi):
        for k in range(3):
            vp, vm = v64.copy(), v64.copy()
            vp[j, k] += h
            vm[j, k] -= h
            gv[r, k] = float(np.sum(g * (_dist_fp64(vp, t, q64) - _dist_fp64(vm, t, q64)))) / (2 * h)
    return gq, gv
