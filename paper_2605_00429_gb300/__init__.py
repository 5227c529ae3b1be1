"""Python binding of libp2mpp.so (P2M++ closest-point queries on GB300).

Argument marshalling only: every step of the build and of the query runs inside the C ABI
(``include/p2mpp.h``).  PyTorch supplies device memory and the current CUDA stream.  There
is no CPU fallback: if the library is missing or no GPU is visible, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libp2mpp.so")

P2M_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "EMPTY_MESH", -5: "DEGENERATE", -6: "LIMIT",
          -7: "STACK", -8: "NOT_IMPLEMENTED", -9: "INTERNAL"}


class P2MError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"p2mpp error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class BuildParams(ctypes.Structure):
    _fields_ = [("domain_scale", ctypes.c_float), ("enable_aux", ctypes.c_int), ("tau_scale", ctypes.c_float),
                ("density_factor", ctypes.c_float), ("density_min", ctypes.c_int), ("ring_sites", ctypes.c_int),
                ("ring_radius_scale", ctypes.c_float), ("build_eps_rel", ctypes.c_float),
                ("nn_grid_res", ctypes.c_int), ("schedule", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("seed", ctypes.c_int), ("long_list", ctypes.c_int), ("gpu_cells", ctypes.c_int),
                ("pipe_chunks", ctypes.c_int), ("aux_balls", ctypes.c_int), ("aux_centre", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_verts", "n_tris", "n_sites", "n_vertex_sites", "n_aux_sites",
                                             "n_corners", "nnz", "max_row")] + \
        [("avg_row", ctypes.c_double)] + \
        [(n, ctypes.c_int64) for n in ("grid_res", "grid_entries", "grid_max", "n_delaunay_tets", "n_dense_cells")] + \
        [("domain_lo", ctypes.c_double * 3), ("domain_hi", ctypes.c_double * 3), ("bbox_diag", ctypes.c_double)] + \
        [(n, ctypes.c_double) for n in ("ms_upload", "ms_tri", "ms_lbvh", "ms_delaunay", "ms_cells", "ms_aug",
                                        "ms_proj", "ms_k1", "ms_grid", "ms_total")] + \
        [("aug_cell_median", ctypes.c_int64), ("aug_cell_max", ctypes.c_int64), ("n_cells_host", ctypes.c_int64),
         ("ms_cells_kernel", ctypes.c_double), ("ms_cells_fallback", ctypes.c_double)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_queries", "n_outside", "site_candidates", "tie_rechecks",
                                             "row_entries", "exact_tests", "long_queries", "long_entries", "queried_list")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
# Every entry point declared in include/p2mpp.h, with its ctypes signature.
_P, _I64, _I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
SIGNATURES = {
    "p2m_version": ([], ctypes.c_char_p),
    "p2m_last_error": ([], ctypes.c_char_p),
    "p2m_default_params": ([_P], _I),
    "p2m_build": ([_P, _I64, _P, _I64, _I, _P, _P, _P], _I),
    "p2m_destroy": ([_P], None),
    "p2m_query": ([_P, _P, _I64, _P, _P, _P, _P, _P], _I),
    "p2m_query_host": ([_P, _P, _I64, _P, _P, _P, _P, _P], _I),
    "p2m_nearest_site": ([_P, _P, _I64, _P, _P], _I),
    "p2m_query_counters": ([_P, _P, _I64, _P, _P, _P], _I),
    "p2m_backward": ([_P, _P, _I64, _P, _P, _P, _P, _P, _P], _I),
    "p2m_update_vertices": ([_P, _P, _P], _I),
    "p2m_get_stats": ([_P, _P], _I),
    "p2m_batch_build": ([_I, _P, _P, _P, _P, _P, _P, _P], _I),
    "p2m_batch_query": ([_P, _P, _P, _P, _P, _P, _P, _I, _I, _P], _I),
    "p2m_num_meshes": ([_P], _I),
    "p2m_get_sizes": ([_P, _I, _P, _P, _P], _I),
    "p2m_get_sites": ([_P, _I, _P, _P, _P], _I),
    "p2m_get_lists": ([_P, _I, _P, _P], _I),
    "p2m_get_balls": ([_P, _I, _P, _P, _P], _I),
    "p2m_get_bvh": ([_P, _I, _P, _P, _P, _P], _I),
    "p2m_set_timing": ([_P, _I], _I),
    "p2m_query_timing": ([_P, _P], _I),
    "p2m_voronoi_cells": ([_P, _I64, _P, _P, _I, _P, _P, _P, _P], _I),
    "p2m_voronoi_cells_device": ([_P, _I64, _P, _P, _I, _P, _P, _P, _P, _P, _P], _I),
    "p2m_query_noalloc": ([_P, _P, _I64, _P, _P, _P, _P, _P], _I),
    "p2m_query_signed": ([_P, _P, _I64, _P, _P, _P, _P, _P], _I),
    "p2m_mesh_distance": ([_P, _P, _I64, _P, _I64, _I, _P, _P], _I),
    "p2m_mesh_distance_pair": ([_P, _P, _I, _P, _P], _I),
}
NOALLOC_MAX_QUERIES = 262144


def lib():
    """Load libp2mpp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                               "(needs nvcc); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc: int):
    if rc != P2M_OK:
        raise P2MError(rc, lib().p2m_last_error().decode())


def default_params(**kw) -> BuildParams:
    p = BuildParams()
    _check(lib().p2m_default_params(ctypes.byref(p)))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown build parameter {k}")
        setattr(p, k, v)
    return p


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _host_arrays(verts, tris):
    try:
        import torch
        if isinstance(verts, torch.Tensor):
            verts = verts.detach().cpu().numpy()
        if isinstance(tris, torch.Tensor):
            tris = tris.detach().cpu().numpy()
    except ImportError:
        pass
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float32).reshape(-1, 3))
    t = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
    return v, t


class P2MIndex:
    """Closest-point index over one triangle mesh (or, from :meth:`batch`, many meshes)."""

    def __init__(self, verts=None, tris=None, _handle=None, **params):
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
            return
        v, t = _host_arrays(verts, tris)
        self.n_verts, self.n_tris = v.shape[0], t.shape[0]
        p = default_params(**params)
        _check(lib().p2m_build(v.ctypes.data_as(_P), v.shape[0], t.ctypes.data_as(_P), t.shape[0], 0,
                               ctypes.byref(p), _stream_ptr(), ctypes.byref(self._h)))
        # the vertices the index was built on (checked by unsigned_distance)
        self._verts = v.copy()
        self._verts_dev = None
        self._vtoken = None

    @classmethod
    def batch(cls, meshes, **params):
        """One index over many meshes (list of (verts, tris)) for :meth:`batch_query`."""
        arrs = [_host_arrays(v, t) for v, t in meshes]
        n = len(arrs)
        vp = (ctypes.c_void_p * n)(*[a[0].ctypes.data for a in arrs])
        tp = (ctypes.c_void_p * n)(*[a[1].ctypes.data for a in arrs])
        nv = (ctypes.c_int64 * n)(*[a[0].shape[0] for a in arrs])
        nt = (ctypes.c_int64 * n)(*[a[1].shape[0] for a in arrs])
        p = default_params(**params)
        h = ctypes.c_void_p()
        _check(lib().p2m_batch_build(n, vp, nv, tp, nt, ctypes.byref(p), _stream_ptr(), ctypes.byref(h)))
        obj = cls(_handle=h)
        obj.n_meshes = n
        obj._arrs = arrs
        return obj

    def close(self):
        if self._h and self._h.value:
            lib().p2m_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- queries
    def query(self, pts, want_closest=True, want_tri=True, want_bary=True, stream=None, out=None):
        """pts: CUDA float32 tensor [n,3].  Returns (dist, closest, tri, bary) CUDA tensors."""
        import torch
        pts = pts.contiguous()
        assert pts.is_cuda and pts.dtype == torch.float32 and pts.dim() == 2 and pts.shape[1] == 3
        n = pts.shape[0]
        if out is None:
            dist = torch.empty(n, device=pts.device, dtype=torch.float32)
            closest = torch.empty(n, 3, device=pts.device, dtype=torch.float32) if want_closest else None
            tri = torch.empty(n, device=pts.device, dtype=torch.int32) if want_tri else None
            bary = torch.empty(n, 3, device=pts.device, dtype=torch.float32) if want_bary else None
        else:
            dist, closest, tri, bary = out
        _check(lib().p2m_query(self._h, _dptr(pts), n, _dptr(dist), _dptr(closest), _dptr(tri), _dptr(bary),
                               _stream_ptr(stream)))
        return dist, closest, tri, bary

    def query_signed(self, pts, stream=None):
        """Signed distance (negative inside a closed outward-oriented mesh): returns
        (sdist, closest, tri, bary) CUDA tensors."""
        import torch
        pts = pts.contiguous()
        n = pts.shape[0]
        sd = torch.empty(n, device=pts.device, dtype=torch.float32)
        cl = torch.empty(n, 3, device=pts.device, dtype=torch.float32)
        tr = torch.empty(n, device=pts.device, dtype=torch.int32)
        ba = torch.empty(n, 3, device=pts.device, dtype=torch.float32)
        _check(lib().p2m_query_signed(self._h, _dptr(pts), n, _dptr(sd), _dptr(cl), _dptr(tr), _dptr(ba),
                                      _stream_ptr(stream)))
        return sd, cl, tr, ba

    def mesh_distance(self, verts_b, tris_b, subdivisions=4, stream=None):
        """(min, max, mean) distance from mesh B's samples (vertices + a barycentric lattice of
        `subdivisions` per triangle) to this index's mesh."""
        import torch
        vb = torch.as_tensor(np.ascontiguousarray(np.asarray(verts_b, np.float32))).cuda()
        tb = torch.as_tensor(np.ascontiguousarray(np.asarray(tris_b, np.int32))).cuda()
        out = np.zeros(3)
        _check(lib().p2m_mesh_distance(self._h, _dptr(vb), vb.shape[0], _dptr(tb), tb.shape[0], int(subdivisions),
                                       out.ctypes.data_as(_P), _stream_ptr(stream)))
        return float(out[0]), float(out[1]), float(out[2])

    def mesh_distance_pair(self, other, subdivisions=4, stream=None):
        """Both directions between this index's mesh (A) and another single-mesh index's (B):
        a dict with (min, max, mean) of B's samples against A ("b_to_a"), of A's against B
        ("a_to_b") and the symmetric Hausdorff distance over the samples ("hausdorff")."""
        out = np.zeros(7)
        _check(lib().p2m_mesh_distance_pair(self._h, other._h, int(subdivisions), out.ctypes.data_as(_P),
                                            _stream_ptr(stream)))
        return {"b_to_a": tuple(out[0:3]), "a_to_b": tuple(out[3:6]), "hausdorff": float(out[6])}

    def query_host(self, pts: np.ndarray, h_dist=None, h_closest=None, h_tri=None, h_bary=None):
        """Host-memory query (copies inside the library).  Arrays may be pinned torch CPU
        tensors or numpy arrays; returns the output arrays."""
        def p(a):
            if a is None:
                return None
            return ctypes.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(_P)
        n = pts.shape[0]
        if h_dist is None:
            h_dist = np.empty(n, np.float32)
        _check(lib().p2m_query_host(self._h, p(pts), n, p(h_dist), p(h_closest), p(h_tri), p(h_bary),
                                    _stream_ptr()))
        return h_dist, h_closest, h_tri, h_bary

    def nearest_site(self, pts, stream=None):
        import torch
        pts = pts.contiguous()
        site = torch.empty(pts.shape[0], device=pts.device, dtype=torch.int32)
        _check(lib().p2m_nearest_site(self._h, _dptr(pts), pts.shape[0], _dptr(site), _stream_ptr(stream)))
        return site

    def counters(self, pts, stream=None) -> dict:
        c = Counters()
        pts = pts.contiguous()
        _check(lib().p2m_query_counters(self._h, _dptr(pts), pts.shape[0], None, ctypes.byref(c),
                                        _stream_ptr(stream)))
        return c.as_dict()

    def backward(self, pts, tri, bary, grad_dist, grad_pts=None, grad_verts=None, stream=None):
        _check(lib().p2m_backward(self._h, _dptr(pts), pts.shape[0], _dptr(tri), _dptr(bary), _dptr(grad_dist),
                                  _dptr(grad_pts), _dptr(grad_verts), _stream_ptr(stream)))

    def update_vertices(self, verts, stream=None):
        src = verts
        verts = verts.detach().contiguous()
        _check(lib().p2m_update_vertices(self._h, _dptr(verts), _stream_ptr(stream)))
        self._verts_dev = verts.float().clone()
        self._verts = None
        self._vtoken = (src.data_ptr(), src._version, tuple(src.shape))

    def check_vertices(self, verts):
        """Raise if `verts` differ from the vertices this index was built on (or last updated
        to).  A tensor seen before and not modified in place since is accepted without a
        comparison; anything else is compared element by element once."""
        import torch
        token = (verts.data_ptr(), verts._version, tuple(verts.shape))
        if token == getattr(self, "_vtoken", None):
            return
        if getattr(self, "_verts_dev", None) is None or self._verts_dev.device != verts.device:
            base = self._verts if self._verts is not None else self._verts_dev.cpu().numpy()
            self._verts_dev = torch.from_numpy(np.ascontiguousarray(base)).to(verts.device)
        if tuple(verts.shape) != tuple(self._verts_dev.shape) or \
                not torch.equal(verts.detach().to(torch.float32), self._verts_dev):
            raise ValueError("the vertices differ from the ones the index was built on: call "
                             "index.update_vertices(verts) after moving them, or the gradients would be stale")
        self._vtoken = token

    def batch_query(self, pts, offsets, mode=0, use_graph=True, out=None, stream=None):
        """pts: CUDA [N,3] (queries of mesh i at offsets[i]:offsets[i+1]); returns CUDA outputs."""
        import torch
        n = pts.shape[0]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        if out is None:
            out = (torch.empty(n, device=pts.device), torch.empty(n, 3, device=pts.device),
                   torch.empty(n, device=pts.device, dtype=torch.int32), torch.empty(n, 3, device=pts.device))
        dist, closest, tri, bary = out
        _check(lib().p2m_batch_query(self._h, _dptr(pts), off.ctypes.data_as(_P), _dptr(dist), _dptr(closest),
                                     _dptr(tri), _dptr(bary), int(mode), int(bool(use_graph)),
                                     _stream_ptr(stream)))
        return out

    def set_timing(self, on=True):
        """Record CUDA events around the list-scan kernel of every later query call."""
        _check(lib().p2m_set_timing(self._h, int(bool(on))))

    def query_timing(self):
        """(list-scan kernel ms, whole call ms) of the last timed query call."""
        out = np.zeros(2)
        _check(lib().p2m_query_timing(self._h, out.ctypes.data_as(_P)))
        return float(out[0]), float(out[1])

    # ---------------------------------------------------------------- introspection
    def stats(self) -> dict:
        s = Stats()
        _check(lib().p2m_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def sizes(self, mesh=0):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().p2m_get_sizes(self._h, mesh, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def sites(self, mesh=0):
        S, _, _ = self.sizes(mesh)
        pos = np.empty((S, 3), np.float32)
        ref = np.empty((S, 3), np.float64)
        kind = np.empty(S, np.int32)
        _check(lib().p2m_get_sites(self._h, mesh, pos.ctypes.data_as(_P), ref.ctypes.data_as(_P),
                                   kind.ctypes.data_as(_P)))
        return pos, ref, kind

    def lists(self, mesh=0):
        S, nnz, _ = self.sizes(mesh)
        off = np.empty(S + 1, np.int64)
        ids = np.empty(max(nnz, 1), np.int32)
        _check(lib().p2m_get_lists(self._h, mesh, off.ctypes.data_as(_P), ids.ctypes.data_as(_P)))
        return off, ids[:nnz]

    def bvh(self, mesh=0):
        """(root, nodes [n_nodes,16] float32 as stored, leaf_tri [n_tris] int32)."""
        nn, root = ctypes.c_int64(), ctypes.c_int32()
        _check(lib().p2m_get_bvh(self._h, mesh, ctypes.byref(nn), ctypes.byref(root), None, None))
        nodes = np.empty((max(nn.value, 1), 16), np.float32)
        n_tris = self.stats()["n_tris"] if getattr(self, "n_meshes", 1) == 1 else None
        if n_tris is None:
            raise ValueError("bvh() of a batch index: use the single-mesh index")
        leaf = np.empty(n_tris, np.int32)
        _check(lib().p2m_get_bvh(self._h, mesh, None, None, nodes.ctypes.data_as(_P), leaf.ctypes.data_as(_P)))
        return root.value, nodes[:nn.value], leaf

    def balls(self, mesh=0):
        S, _, B = self.sizes(mesh)
        off = np.empty(S + 1, np.int64)
        c = np.empty((max(B, 1), 3), np.float64)
        r = np.empty(max(B, 1), np.float64)
        _check(lib().p2m_get_balls(self._h, mesh, off.ctypes.data_as(_P), c.ctypes.data_as(_P),
                                   r.ctypes.data_as(_P)))
        return off, c[:B], r[:B]


def voronoi_cells(sites, dom_lo, dom_hi, seed=1):
    """Host-only: the clipped Voronoi cells the build computes.  Returns (moved sites [n,3]
    float32, corner offsets [n+1], corners [m,3] float64)."""
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.float32).reshape(-1, 3))
    lo = np.ascontiguousarray(np.asarray(dom_lo, dtype=np.float64))
    hi = np.ascontiguousarray(np.asarray(dom_hi, dtype=np.float64))
    n = s.shape[0]
    cnt = ctypes.c_int64()
    _check(lib().p2m_voronoi_cells(s.ctypes.data_as(_P), n, lo.ctypes.data_as(_P), hi.ctypes.data_as(_P), seed,
                                   None, None, None, ctypes.byref(cnt)))
    moved = np.empty((n, 3), np.float32)
    off = np.empty(n + 1, np.int64)
    cor = np.empty((max(cnt.value, 1), 3), np.float64)
    _check(lib().p2m_voronoi_cells(s.ctypes.data_as(_P), n, lo.ctypes.data_as(_P), hi.ctypes.data_as(_P), seed,
                                   moved.ctypes.data_as(_P), off.ctypes.data_as(_P), cor.ctypes.data_as(_P),
                                   ctypes.byref(cnt)))
    return moved, off, cor[:cnt.value]


def voronoi_cells_device(sites, dom_lo, dom_hi, seed=1, stream=None):
    """The same cells clipped on the GPU (the build's default path).  Returns (moved sites,
    corner offsets, corners, number of cells that were clipped on the host instead)."""
    s = np.ascontiguousarray(np.asarray(sites, dtype=np.float32).reshape(-1, 3))
    lo = np.ascontiguousarray(np.asarray(dom_lo, dtype=np.float64))
    hi = np.ascontiguousarray(np.asarray(dom_hi, dtype=np.float64))
    n = s.shape[0]
    cnt, n_host = ctypes.c_int64(), ctypes.c_int64()
    args = (s.ctypes.data_as(_P), n, lo.ctypes.data_as(_P), hi.ctypes.data_as(_P), seed)
    _check(lib().p2m_voronoi_cells_device(*args, None, None, None, ctypes.byref(cnt), ctypes.byref(n_host),
                                          _stream_ptr(stream)))
    moved = np.empty((n, 3), np.float32)
    off = np.empty(n + 1, np.int64)
    cor = np.empty((max(cnt.value, 1), 3), np.float64)
    _check(lib().p2m_voronoi_cells_device(*args, moved.ctypes.data_as(_P), off.ctypes.data_as(_P),
                                          cor.ctypes.data_as(_P), ctypes.byref(cnt), ctypes.byref(n_host),
                                          _stream_ptr(stream)))
    return moved, off, cor[:cnt.value], n_host.value


def _make_function():
    import torch

    class UnsignedDistance(torch.autograd.Function):
        """d(q, M) for query points q with gradients w.r.t. q and the mesh vertices.

        forward(pts [n,3], verts [V,3], index) -> dist [n].  The index must have been built
        on `verts` (rebuild or call ``index.update_vertices`` when they change); other
        vertices raise ValueError instead of giving stale gradients."""

        @staticmethod
        def forward(ctx, pts, verts, index):
            index.check_vertices(verts)
            dist, _, tri, bary = index.query(pts, want_closest=False)
            ctx.save_for_backward(pts, tri, bary)
            ctx.index = index
            ctx.n_verts = verts.shape[0]
            ctx.verts_meta = (verts.device, verts.dtype)
            return dist

        @staticmethod
        def backward(ctx, grad_dist):
            pts, tri, bary = ctx.saved_tensors
            need_q, need_v = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            gq = torch.empty_like(pts) if need_q else None
            gv = torch.zeros(ctx.n_verts, 3, device=pts.device, dtype=torch.float32) if need_v else None
            ctx.index.backward(pts, tri, bary, grad_dist.contiguous().float(), gq, gv)
            return gq, gv, None

    return UnsignedDistance


_UD = None


def unsigned_distance(pts, verts, index):
    """Differentiable unsigned distance (a torch.autograd.Function)."""
    global _UD
    if _UD is None:
        _UD = _make_function()
    return _UD.apply(pts, verts, index)
