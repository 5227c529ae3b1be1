"""Seeded synthetic meshes and query sets shaped like the P2M++ evaluation workloads.

This module generates inputs only. It holds none of the closest-point, Voronoi or
interception-list arithmetic, so both the CUDA path and the FP64 oracle may use it.

The paper measures on Stanford / ABC / "#1-#3" models (Section 4, Fig. 4), which are not
available here. These generators stand in for them:

* ``uv_sphere``         -- latitude/longitude sphere; every vertex is co-spherical, the
                           worst case of Section 3.2 (Fig. 2) and the "Sphere" column of
                           Tables 1-4.
* ``icosphere``         -- subdivided icosahedron on the unit sphere.
* ``geodesic_sphere``   -- frequency-n geodesic subdivision (T = 20 n^2), used for batches.
* ``displace_radial``   -- 3-octave value-noise radial displacement (organic-model stand-in).
* ``cylinder_cone``     -- capped cylinder fused with a cone: a rotationally symmetric
                           stress case like "#1-#3" (Section 4, Table 4).
* ``capped_cylinder``   -- a x b capped cylinder, used for batches.

Query recipes follow Section 4 (points in a box around the model), plus near-surface
recipes for the differentiation and symmetric workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Mesh", "uv_sphere", "icosphere", "geodesic_sphere", "displace_radial",
    "cylinder_cone", "capped_cylinder", "unit_cube", "square_plane",
    "queries_uniform_box", "queries_surface_gauss", "queries_near_surface",
    "workload_small", "workload_large", "workload_symmetric", "workload_batch",
    "workload_diff", "splitmix64",
]


@dataclass
class Mesh:
    verts: np.ndarray  # [V,3] float32
    tris: np.ndarray   # [T,3] int32

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    def bbox(self):
        return self.verts.min(axis=0).astype(np.float64), self.verts.max(axis=0).astype(np.float64)

    def diag(self) -> float:
        lo, hi = self.bbox()
        return float(np.linalg.norm(hi - lo))


def _mesh(verts, tris) -> Mesh:
    return Mesh(np.ascontiguousarray(np.asarray(verts, dtype=np.float32)),
                np.ascontiguousarray(np.asarray(tris, dtype=np.int32)))


# ----------------------------------------------------------------------------- meshes

def uv_sphere(n_lon: int = 32, n_lat: int = 16, radius: float = 1.0) -> Mesh:
    """Two poles plus (n_lat-1) rings of n_lon vertices; 2*n_lon*(n_lat-1) triangles."""
    verts = [(0.0, 0.0, radius)]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * math.pi * j / n_lon
            verts.append((radius * math.sin(th) * math.cos(ph),
                          radius * math.sin(th) * math.sin(ph),
                          radius * math.cos(th)))
    verts.append((0.0, 0.0, -radius))
    south = len(verts) - 1

    def ring(i, j):  # i in [0, n_lat-2]
        return 1 + i * n_lon + (j % n_lon)

    tris = []
    for j in range(n_lon):
        tris.append((0, ring(0, j), ring(0, j + 1)))
    for i in range(n_lat - 2):
        for j in range(n_lon):
            a, b = ring(i, j), ring(i, j + 1)
            c, d = ring(i + 1, j), ring(i + 1, j + 1)
            tris.append((a, c, d))
            tris.append((a, d, b))
    for j in range(n_lon):
        tris.append((south, ring(n_lat - 2, j + 1), ring(n_lat - 2, j)))
    return _mesh(verts, tris)


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
                  (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
                  (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
                  (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
                  (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
                  (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int64)
    return v, f


def icosphere(k: int, radius: float = 1.0) -> Mesh:
    """Icosahedron with k midpoint subdivisions, projected to the sphere: T = 20*4^k, V = 10*4^k + 2."""
    v, f = _icosahedron()
    for _ in range(k):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e.sort(axis=1)
        uniq, inv = np.unique(e, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], 1), np.stack([f[:, 1], m12, m01], 1),
            np.stack([f[:, 2], m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
    return _mesh(v * radius, f)


def geodesic_sphere(freq: int, radius: float = 1.0) -> Mesh:
    """Each icosahedron face split into freq^2 triangles, projected to the sphere: T = 20*freq^2."""
    v0, f0 = _icosahedron()
    n = max(1, int(freq))
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    keep = ii + jj <= n
    ii, jj = ii[keep], jj[keep]
    local = -np.ones((n + 1, n + 1), np.int64)
    local[ii, jj] = np.arange(len(ii))
    # triangles of one face in local grid ids
    a_i, a_j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    up = a_i + a_j <= n - 1
    dn = a_i + a_j <= n - 2
    t_up = np.stack([local[a_i[up], a_j[up]], local[a_i[up] + 1, a_j[up]], local[a_i[up], a_j[up] + 1]], 1)
    t_dn = np.stack([local[a_i[dn] + 1, a_j[dn]], local[a_i[dn] + 1, a_j[dn] + 1], local[a_i[dn], a_j[dn] + 1]], 1)
    tloc = np.concatenate([t_up, t_dn], 0)
    npf = len(ii)
    pts = []
    tris = []
    for k, (a, b, c) in enumerate(f0):
        p = ((n - ii - jj)[:, None] * v0[a] + ii[:, None] * v0[b] + jj[:, None] * v0[c]) / n
        pts.append(p)
        tris.append(tloc + k * npf)
    pts = np.concatenate(pts, 0)
    tris = np.concatenate(tris, 0)
    # points on shared edges / corners coincide exactly up to rounding: merge them
    key = np.round(pts * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    order = np.argsort(first)
    remap = np.empty_like(order)
    remap[order] = np.arange(len(order))
    verts = pts[first[order]]
    verts /= np.linalg.norm(verts, axis=1, keepdims=True)
    return _mesh(verts * radius, remap[inv][tris])


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea & Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _lattice_value(ix, iy, iz, seed, octave):
    with np.errstate(over="ignore"):
        h = splitmix64(ix.astype(np.int64).astype(np.uint64))
        h = splitmix64(h ^ iy.astype(np.int64).astype(np.uint64))
        h = splitmix64(h ^ iz.astype(np.int64).astype(np.uint64))
        h = splitmix64(h ^ np.uint64(seed))
        h = splitmix64(h ^ np.uint64(octave))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 / 2.0 ** 53) - 1.0


def _value_noise(p: np.ndarray, seed: int, octave: int) -> np.ndarray:
    fl = np.floor(p)
    i0 = fl.astype(np.int64)
    f = p - fl
    w = f * f * (3.0 - 2.0 * f)  # smoothstep weights
    out = np.zeros(p.shape[0])
    for dx in (0, 1):
        wx = w[:, 0] if dx else 1.0 - w[:, 0]
        for dy in (0, 1):
            wy = w[:, 1] if dy else 1.0 - w[:, 1]
            for dz in (0, 1):
                wz = w[:, 2] if dz else 1.0 - w[:, 2]
                out += wx * wy * wz * _lattice_value(i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz, seed, octave)
    return out


def fractal_noise(p: np.ndarray, seed: int = 0) -> np.ndarray:
    """N(p) = sum_{k=0..2} 0.5^k vn(2^{k+1} p) / 1.75, values in [-1, 1]."""
    p = np.asarray(p, dtype=np.float64)
    return sum(0.5 ** k * _value_noise(p * 2.0 ** (k + 1), seed, k) for k in range(3)) / 1.75


def displace_radial(mesh: Mesh, amplitude: float = 0.05, seed: int = 0, axis: str | None = None) -> Mesh:
    """Scale each vertex's distance from the origin (or from the z axis if axis == 'z') by 1 + a*N."""
    v = mesh.verts.astype(np.float64)
    n = fractal_noise(v, seed)
    if axis == "z":
        out = v.copy()
        out[:, :2] *= (1.0 + amplitude * n)[:, None]
    else:
        out = v * (1.0 + amplitude * n)[:, None]
    return _mesh(out, mesh.tris)


def _ring(r, z, n):
    a = 2.0 * np.pi * np.arange(n) / n
    return np.stack([r * np.cos(a), r * np.sin(a), np.full(n, z)], 1)


def _strip(ia, ib, n):
    """Quads between two rings of n vertices (ids ia[j], ib[j]), outward-facing if ia is below ib."""
    j = np.arange(n)
    jn = (j + 1) % n
    t1 = np.stack([ia[j], ia[jn], ib[jn]], 1)
    t2 = np.stack([ia[j], ib[jn], ib[j]], 1)
    return np.concatenate([t1, t2], 0)


def cylinder_cone(n_ang: int = 512, n_ax: int = 128, n_cone: int = 64, n_cap: int = 8,
                  radius: float = 1.0, height: float = 2.0, cone_height: float = 1.5) -> Mesh:
    """Watertight capped cylinder (z in [0, height]) fused with a cone (apex at height+cone_height).

    Side: n_ang x n_ax quads; cone: n_cone rings ending in a fan to the apex; bottom cap:
    n_cap concentric rings ending in a fan to the centre.
    """
    verts, tris = [], []
    base = 0
    side_rings = []
    for i in range(n_ax + 1):
        verts.append(_ring(radius, height * i / n_ax, n_ang))
        side_rings.append(base + np.arange(n_ang))
        base += n_ang
    for i in range(n_ax):
        tris.append(_strip(side_rings[i], side_rings[i + 1], n_ang))
    cone_rings = [side_rings[-1]]
    for j in range(1, n_cone):
        verts.append(_ring(radius * (1.0 - j / n_cone), height + cone_height * j / n_cone, n_ang))
        cone_rings.append(base + np.arange(n_ang))
        base += n_ang
    for j in range(n_cone - 1):
        tris.append(_strip(cone_rings[j], cone_rings[j + 1], n_ang))
    verts.append(np.array([[0.0, 0.0, height + cone_height]]))
    apex = base
    base += 1
    jj = np.arange(n_ang)
    last = cone_rings[-1]
    tris.append(np.stack([last[jj], last[(jj + 1) % n_ang], np.full(n_ang, apex)], 1))
    cap_rings = [side_rings[0]]
    for k in range(n_cap - 1, 0, -1):
        verts.append(_ring(radius * k / n_cap, 0.0, n_ang))
        cap_rings.append(base + np.arange(n_ang))
        base += n_ang
    for k in range(len(cap_rings) - 1):
        # the cap faces -z: reverse the winding relative to the side strips
        s = _strip(cap_rings[k + 1], cap_rings[k], n_ang)
        tris.append(s)
    verts.append(np.array([[0.0, 0.0, 0.0]]))
    centre = base
    inner = cap_rings[-1]
    tris.append(np.stack([inner[(jj + 1) % n_ang], inner[jj], np.full(n_ang, centre)], 1))
    return _mesh(np.concatenate(verts, 0), np.concatenate(tris, 0))


def capped_cylinder(n_ang: int, n_ax: int, radius: float = 1.0, height: float = 2.0) -> Mesh:
    """n_ang x n_ax side quads plus a fan cap at each end: T = 2*n_ang*n_ax + 2*n_ang."""
    verts, tris = [], []
    rings = []
    for i in range(n_ax + 1):
        verts.append(_ring(radius, height * i / n_ax - height / 2, n_ang))
        rings.append(i * n_ang + np.arange(n_ang))
    for i in range(n_ax):
        tris.append(_strip(rings[i], rings[i + 1], n_ang))
    nb = (n_ax + 1) * n_ang
    verts.append(np.array([[0.0, 0.0, -height / 2], [0.0, 0.0, height / 2]]))
    j = np.arange(n_ang)
    jn = (j + 1) % n_ang
    r0, r1 = rings[0], rings[-1]
    tris.append(np.stack([r0[jn], r0[j], np.full(n_ang, nb)], 1))
    tris.append(np.stack([r1[j], r1[jn], np.full(n_ang, nb + 1)], 1))
    return _mesh(np.concatenate(verts, 0), np.concatenate(tris, 0))


def unit_cube() -> Mesh:
    """Axis-aligned cube [-1/2, 1/2]^3 as 12 triangles."""
    v = np.array([[x, y, z] for x in (-0.5, 0.5) for y in (-0.5, 0.5) for z in (-0.5, 0.5)])
    quads = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    return _mesh(v, tris)


def square_plane(half: float = 1.0) -> Mesh:
    """Two triangles covering [-half, half]^2 in the z = 0 plane."""
    v = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]])
    return _mesh(v, [(0, 1, 2), (0, 2, 3)])


# ----------------------------------------------------------------------------- queries

def queries_uniform_box(mesh: Mesh, n: int, scale: float = 1.2, seed: int = 0) -> np.ndarray:
    """n points uniform in the bbox scaled by `scale` about its centre."""
    lo, hi = mesh.bbox()
    c, h = (lo + hi) / 2, (hi - lo) / 2 * scale
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray((c + (rng.random((n, 3)) * 2 - 1) * h).astype(np.float32))


def _surface_points(mesh: Mesh, n: int, rng) -> np.ndarray:
    v = mesh.verts.astype(np.float64)
    a, b, c = v[mesh.tris[:, 0]], v[mesh.tris[:, 1]], v[mesh.tris[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    t = np.minimum(np.searchsorted(cdf, rng.random(n)), mesh.n_tris - 1)
    r1 = np.sqrt(rng.random(n))[:, None]
    r2 = rng.random(n)[:, None]
    return (1 - r1) * a[t] + r1 * (1 - r2) * b[t] + r1 * r2 * c[t]


def queries_surface_gauss(mesh: Mesh, n: int, sigma: float, seed: int = 0) -> np.ndarray:
    """Area-weighted surface points plus isotropic N(0, sigma^2 I) offsets."""
    rng = np.random.default_rng(seed)
    p = _surface_points(mesh, n, rng) + rng.normal(0.0, sigma, (n, 3))
    return np.ascontiguousarray(p.astype(np.float32))


def queries_near_surface(mesh: Mesh, n: int, max_dist: float, seed: int = 0) -> np.ndarray:
    """Surface point plus a uniform random direction times U[0, max_dist]."""
    rng = np.random.default_rng(seed)
    p = _surface_points(mesh, n, rng)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = p + d * (rng.random(n) * max_dist)[:, None]
    return np.ascontiguousarray(p.astype(np.float32))


def _mix(parts, seed):
    p = np.concatenate(parts, 0)
    rng = np.random.default_rng(seed + 7919)
    return np.ascontiguousarray(p[rng.permutation(p.shape[0])])


# ----------------------------------------------------------------------------- workloads

def workload_small(n_queries: int = 100_000, seed: int = 0):
    """UV sphere (32 x 16, 960 tris); queries uniform in the 1.2x bbox."""
    m = uv_sphere(32, 16)
    return m, queries_uniform_box(m, n_queries, 1.2, seed)


def workload_large(n_queries: int = 10_000_000, seed: int = 0, k: int = 6):
    """Icosphere(k) with 3-octave noise (amplitude 0.05); half uniform in 1.2x bbox, half
    surface + N(0, (0.01 diag)^2)."""
    m = displace_radial(icosphere(k), 0.05, seed)
    nu = n_queries // 2
    q = _mix([queries_uniform_box(m, nu, 1.2, seed + 1),
              queries_surface_gauss(m, n_queries - nu, 0.01 * m.diag(), seed + 2)], seed)
    return m, q


def workload_symmetric(n_queries: int = 10_000_000, seed: int = 0, n_ang: int = 512, n_ax: int = 128):
    """Cylinder + cone (203,776 tris at 512 x 128); 70% within 0.02 diag of the surface,
    30% uniform in 1.2x bbox."""
    m = cylinder_cone(n_ang, n_ax, max(2, n_ax // 2), 8)
    nn = int(round(n_queries * 0.7))
    q = _mix([queries_near_surface(m, nn, 0.02 * m.diag(), seed + 1),
              queries_uniform_box(m, n_queries - nn, 1.2, seed + 2)], seed)
    return m, q


def workload_diff(n_queries: int = 1_000_000, seed: int = 0, k: int = 5):
    """Icosphere(k) with noise; near-surface queries, surface + N(0, (0.01 diag)^2)."""
    m = displace_radial(icosphere(k), 0.05, seed)
    return m, queries_surface_gauss(m, n_queries, 0.01 * m.diag(), seed + 3)


def workload_batch(n_meshes: int = 256, seed: int = 0, t_range=(500, 200_000), q_range=(1_000, 1_000_000),
                   query_scale: float = 1.0):
    """Alternating noisy geodesic spheres and noisy capped cylinders; triangle and query counts
    log-uniform in the given ranges. Returns (meshes, queries) lists."""
    rng = np.random.default_rng(seed + 104729)
    lt = np.exp(rng.uniform(np.log(t_range[0]), np.log(t_range[1]), n_meshes))
    lq = np.exp(rng.uniform(np.log(q_range[0]), np.log(q_range[1]), n_meshes))
    meshes, queries = [], []
    for i in range(n_meshes):
        t = float(lt[i])
        if i % 2 == 0:
            m = displace_radial(geodesic_sphere(max(2, int(round(math.sqrt(t / 20.0))))), 0.05, seed + i)
        else:
            # T = 2ab + 2a with near-square quads on an r=1, h=2 cylinder: b ~ a / pi
            a = max(8, int(round(math.sqrt(t * math.pi / 2.0))))
            b = max(1, int(round(a / math.pi)))
            m = displace_radial(capped_cylinder(a, b), 0.05, seed + i, axis="z")
        nq = max(1, int(round(lq[i] * query_scale)))
        nu = nq // 2
        q = _mix([queries_uniform_box(m, nu, 1.2, seed + 3 * i + 1),
                  queries_surface_gauss(m, nq - nu, 0.01 * m.diag(), seed + 3 * i + 2)], seed + i)
        meshes.append(m)
        queries.append(q)
    return meshes, queries
