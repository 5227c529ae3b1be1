// C ABI of libp2mpp.so: argument checking, index lifecycle, build orchestration and query
// dispatch.  The compute lives in the kernels of bvh.cu / lists.cu / grid.cu / query.cu and
// the host Voronoi code of voronoi.cpp.
#include <array>
#include <atomic>
#include <unordered_map>
#include <cstdlib>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "host.h"
#include "p2m_internal.h"
#include "voronoi.h"

namespace p2m {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

// Host-side fault injection for tests: P2M_FAULT=alloc:K makes the K-th device allocation
// (counted from the last change of the variable) fail as out of memory.
static bool inject_alloc_fault() {
    static std::mutex mu;
    static std::string last;
    static long count = 0;
    const char* e = std::getenv("P2M_FAULT");
    std::lock_guard<std::mutex> lock(mu);
    const std::string v = e ? e : "";
    if (v != last) { last = v; count = 0; }
    if (v.rfind("alloc:", 0) != 0) return false;
    return ++count == std::atol(v.c_str() + 6);
}

int sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 148;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
        cudaGetLastError();
        return 148;
    }
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

bool inject_fault(const char* what) {
    const char* e = std::getenv("P2M_FAULT");
    return e && std::strcmp(e, what) == 0;
}

int DevBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    if (inject_alloc_fault())
        return fail(P2M_ERR_OOM, "cudaMalloc(" + std::to_string(nbytes) + "): injected allocation failure");
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? P2M_ERR_OOM : P2M_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(nbytes) + "): " + cudaGetErrorString(e));
    }
    bytes = nbytes;
    return P2M_OK;
}

int DevBuf::ensure(size_t nbytes) {
    if (p && bytes >= nbytes) return P2M_OK;
    return alloc(nbytes);
}

MeshView MeshData::view() const {
    MeshView v{};
    v.tri = d_tri.as<const float4>();
    v.orig = d_orig.as<const int32_t>();
    v.tsph = d_tsph.as<const float4>();
    v.bvh = bvh.nodes.as<const BNode>();
    v.bvh_root = bvh.root;
    v.sites = d_sites.as<const float4>();
    v.refs = d_refs.as<const float4>();
    v.row_off = d_row_off.as<const int32_t>();
    v.row_ent = d_row_ent.as<const int2>();
    v.row_sph = d_row_sph.as<const float4>();
    v.chunk_off = d_chunk_off.as<const int32_t>();
    v.cbox = d_cbox.as<const float4>();
    v.l1_off = d_l1_off.as<const int32_t>();
    v.l1box = d_l1box.as<const float4>();
    v.long_row = long_row;
    v.cell_off = d_cell_off.as<const int32_t>();
    v.cell_id = d_cell_id.as<const int32_t>();
    v.G = G;
    v.lo = g_lo;
    v.hi = g_hi;
    v.inv_h = g_inv_h;
    v.prune_abs = (float)(diag * std::ldexp(1.0, -22));
    v.spacing = spacing;
    v.n_tris = (int)n_tris;
    v.n_sites = (int)(site_pos.size() / 3);
    return v;
}

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace p2m

using namespace p2m;


namespace p2m {

unsigned* index_status(p2m_index* h) { return h->status.as<unsigned>(); }
DevBuf& index_rest(p2m_index* h) { return h->scratch_idx; }

int check_status_word(p2m_index* h, cudaStream_t s, const char* what) {
    unsigned st = 0;
    P2M_CUDA_TRY(cudaMemcpyAsync(&st, h->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    if (st) {
        P2M_CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(unsigned), s));
        if (st & ST_STACK) return fail(P2M_ERR_STACK, std::string(what) + ": device traversal stack overflow");
        if (st & ST_LIMIT) return fail(P2M_ERR_LIMIT, std::string(what) + ": device capacity or iteration cap reached");
        return fail(P2M_ERR_INTERNAL, std::string(what) + ": device index check failed");
    }
    return P2M_OK;
}

int check_call(const p2m_index* h, int64_t n, const char* what) {
    int dev = -1;
    P2M_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != h->device)
        return fail(P2M_ERR_INVALID_ARG, std::string(what) + ": the index was built on device " + std::to_string(h->device) +
                                             " but device " + std::to_string(dev) + " is current");
    if (n > 0x7fffffffLL)
        return fail(P2M_ERR_LIMIT, std::string(what) + ": " + std::to_string(n) +
                                       " points in one call (at most 2^31 - 1); split the call");
    return P2M_OK;
}

void timing_mark(p2m_index* h, int k, cudaStream_t s) {
    if (!h->timing) return;
    cudaEventRecord(h->tev[k], s);
    if (k == 3) h->timed_call = true;
}

}  // namespace p2m

p2m_index::~p2m_index() {
    for (auto& st : streams)
        if (st) cudaStreamDestroy(st);
    for (auto& slot : pipe_ev)
        for (auto& e : slot)
            if (e) cudaEventDestroy(e);
    for (auto& e : tev)
        if (e) cudaEventDestroy(e);
}

// ----------------------------------------------------------------------------- validation

static int validate_params(const p2m_build_params& p) {
    if (!(p.domain_scale >= 1.0f && p.domain_scale < 1e6f)) return fail(P2M_ERR_INVALID_ARG, "domain_scale must be >= 1");
    if (!(p.tau_scale > 0.0f)) return fail(P2M_ERR_INVALID_ARG, "tau_scale must be > 0");
    if (!(p.density_factor > 0.0f)) return fail(P2M_ERR_INVALID_ARG, "density_factor must be > 0");
    if (p.ring_sites != 6 && p.ring_sites != 12) return fail(P2M_ERR_INVALID_ARG, "ring_sites must be 6 or 12");
    if (!(p.ring_radius_scale > 0.0f)) return fail(P2M_ERR_INVALID_ARG, "ring_radius_scale must be > 0");
    if (!(p.build_eps_rel >= 0.0f && p.build_eps_rel < 1e-2f)) return fail(P2M_ERR_INVALID_ARG, "build_eps_rel out of range");
    if (p.nn_grid_res < 0 || p.nn_grid_res > 1023) return fail(P2M_ERR_INVALID_ARG, "nn_grid_res out of range");
    if (p.schedule < 0 || p.schedule > 5) return fail(P2M_ERR_INVALID_ARG, "schedule must be 0..5");
    if (p.long_list < 0) return fail(P2M_ERR_INVALID_ARG, "long_list must be >= 0");
    if (p.pipe_chunks < 0) return fail(P2M_ERR_INVALID_ARG, "pipe_chunks must be >= 0");
    if (p.aux_balls != 0 && p.aux_balls != 1) return fail(P2M_ERR_INVALID_ARG, "aux_balls must be 0 or 1");
    if (p.aux_centre != 0 && p.aux_centre != 1) return fail(P2M_ERR_INVALID_ARG, "aux_centre must be 0 or 1");
    return P2M_OK;
}

// Copy the mesh to host vectors and check it.
static int load_mesh(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris, int on_device,
                     MeshData& m) {
    if (!verts || !tris) return fail(P2M_ERR_INVALID_ARG, "verts and tris must be non-NULL");
    if (n_verts <= 0 || n_tris <= 0) return fail(P2M_ERR_EMPTY_MESH, "mesh needs at least one vertex and one triangle");
    if (n_verts > (int64_t)1 << 30 || n_tris > (int64_t)1 << 30) return fail(P2M_ERR_INVALID_ARG, "mesh too large (>2^30)");
    m.n_verts = n_verts;
    m.n_tris = n_tris;
    m.verts.resize(n_verts * 3);
    m.tris.resize(n_tris * 3);
    if (on_device) {
        P2M_CUDA_TRY(cudaMemcpy(m.verts.data(), verts, sizeof(float) * 3 * n_verts, cudaMemcpyDeviceToHost));
        P2M_CUDA_TRY(cudaMemcpy(m.tris.data(), tris, sizeof(int32_t) * 3 * n_tris, cudaMemcpyDeviceToHost));
    } else {
        std::memcpy(m.verts.data(), verts, sizeof(float) * 3 * n_verts);
        std::memcpy(m.tris.data(), tris, sizeof(int32_t) * 3 * n_tris);
    }
    for (int64_t i = 0; i < n_verts * 3; ++i)
        if (!std::isfinite(m.verts[i])) return fail(P2M_ERR_INVALID_ARG, "vertex " + std::to_string(i / 3) + " is not finite");
    std::vector<char> used(n_verts, 0);
    for (int64_t i = 0; i < n_tris * 3; ++i) {
        const int32_t v = m.tris[i];
        if (v < 0 || v >= n_verts)
            return fail(P2M_ERR_INVALID_ARG, "triangle " + std::to_string(i / 3) + " has vertex index " + std::to_string(v) +
                                                 " out of range");
        used[v] = 1;
    }
    for (int k = 0; k < 3; ++k) { m.bb_lo[k] = INFINITY; m.bb_hi[k] = -INFINITY; }
    for (int64_t i = 0; i < n_verts; ++i) {
        if (!used[i]) continue;
        for (int k = 0; k < 3; ++k) {
            m.bb_lo[k] = std::min(m.bb_lo[k], (double)m.verts[3 * i + k]);
            m.bb_hi[k] = std::max(m.bb_hi[k], (double)m.verts[3 * i + k]);
        }
    }
    double d2 = 0;
    for (int k = 0; k < 3; ++k) d2 += (m.bb_hi[k] - m.bb_lo[k]) * (m.bb_hi[k] - m.bb_lo[k]);
    m.diag = std::sqrt(d2);
    if (!(m.diag > 0)) return fail(P2M_ERR_DEGENERATE, "all referenced vertices coincide");
    return P2M_OK;
}

// ----------------------------------------------------------------------------- build

// Angle-weighted pseudonormals (FP64, uploaded as float4): the unit face normal, the edge
// normal n_f1 + n_f2 of each edge's two faces (a boundary edge keeps its one face's normal),
// and at every vertex the sum of its faces' normals weighted by their angles there.  The
// sign of (q - p) . n at the feature (face, edge, vertex) holding the closest point p tells
// inside from outside on a closed, outward-oriented mesh.  Built on the first signed query
// (only that entry point reads them), not with the index.
int p2m::build_pseudonormals(MeshData& m) {
    const int64_t T = m.n_tris, V = m.n_verts;
    std::vector<double> fn(3 * T, 0.0), vn(3 * V, 0.0);
    auto vtx = [&](int64_t i, int k) { return (double)m.verts[3 * i + k]; };
    for (int64_t f = 0; f < T; ++f) {
        const int32_t* t = &m.tris[3 * f];
        double e[3][3];
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) e[j][k] = vtx(t[(j + 1) % 3], k) - vtx(t[j], k);  // edge j: v_j -> v_j+1
        double n[3] = {e[0][1] * (-e[2][2]) - e[0][2] * (-e[2][1]), e[0][2] * (-e[2][0]) - e[0][0] * (-e[2][2]),
                       e[0][0] * (-e[2][1]) - e[0][1] * (-e[2][0])};  // (v1 - v0) x (v2 - v0)
        const double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0)) continue;
        for (int k = 0; k < 3; ++k) fn[3 * f + k] = n[k] / len;
        for (int j = 0; j < 3; ++j) {
            // angle at vertex j between edge j (outgoing) and the reversed edge j-1
            const double* a = e[j];
            const double* b = e[(j + 2) % 3];
            const double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            const double lb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
            if (!(la > 0 && lb > 0)) continue;
            const double c = std::max(-1.0, std::min(1.0, -(a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) / (la * lb)));
            const double ang = std::acos(c);
            for (int k = 0; k < 3; ++k) vn[3 * (int64_t)t[j] + k] += ang * fn[3 * f + k];
        }
    }
    std::unordered_map<uint64_t, std::array<double, 3>> en;
    auto ekey = [](int a, int b) { return a < b ? ((uint64_t)a << 32 | (uint32_t)b) : ((uint64_t)b << 32 | (uint32_t)a); };
    for (int64_t f = 0; f < T; ++f)
        for (int j = 0; j < 3; ++j) {
            auto& acc = en[ekey(m.tris[3 * f + j], m.tris[3 * f + (j + 1) % 3])];
            for (int k = 0; k < 3; ++k) acc[k] += fn[3 * f + k];
        }
    auto unit4 = [](const double* v, float4& out) {
        const double l = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        out = l > 0 ? make_float4((float)(v[0] / l), (float)(v[1] / l), (float)(v[2] / l), 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    std::vector<float4> srec(4 * T), vrec(V);
    for (int64_t f = 0; f < T; ++f) {
        unit4(&fn[3 * f], srec[4 * f]);
        for (int j = 0; j < 3; ++j) unit4(en[ekey(m.tris[3 * f + j], m.tris[3 * f + (j + 1) % 3])].data(), srec[4 * f + 1 + j]);
    }
    for (int64_t v = 0; v < V; ++v) unit4(&vn[3 * v], vrec[v]);
    P2M_TRY(m.d_snorm.alloc(sizeof(float4) * 4 * T));
    P2M_TRY(m.d_vnorm.alloc(sizeof(float4) * V));
    P2M_CUDA_TRY(cudaMemcpy(m.d_snorm.p, srec.data(), sizeof(float4) * 4 * T, cudaMemcpyHostToDevice));
    P2M_CUDA_TRY(cudaMemcpy(m.d_vnorm.p, vrec.data(), sizeof(float4) * V, cudaMemcpyHostToDevice));
    return P2M_OK;
}

static int build_mesh(MeshData& m, const p2m_build_params& prm, p2m_index* h, cudaStream_t s) {
    p2m_stats& st = m.stats;
    std::memset(&st, 0, sizeof(st));
    const double t0 = now_ms();
    st.n_verts = m.n_verts;
    st.n_tris = m.n_tris;
    st.bbox_diag = m.diag;
    for (int k = 0; k < 3; ++k) {
        const double c = 0.5 * (m.bb_lo[k] + m.bb_hi[k]);
        const double e = 0.5 * (m.bb_hi[k] - m.bb_lo[k]);
        // a flat axis still gets a slab of half-width diag/4 so that D has volume
        const double ee = std::max(e, 0.25 * m.diag) * prm.domain_scale;
        m.dom_lo[k] = c - ee;
        m.dom_hi[k] = c + ee;
        st.domain_lo[k] = m.dom_lo[k];
        st.domain_hi[k] = m.dom_hi[k];
    }
    // upload + K0b; the pseudonormals of the signed query are rebuilt on its next call
    const int T = (int)m.n_tris;
    m.d_snorm.release();
    m.d_vnorm.release();
    P2M_TRY(m.d_verts.alloc(sizeof(float) * 3 * m.n_verts));
    P2M_TRY(m.d_tris.alloc(sizeof(int32_t) * 3 * m.n_tris));
    P2M_CUDA_TRY(cudaMemcpyAsync(m.d_verts.p, m.verts.data(), sizeof(float) * 3 * m.n_verts, cudaMemcpyHostToDevice, s));
    P2M_CUDA_TRY(cudaMemcpyAsync(m.d_tris.p, m.tris.data(), sizeof(int32_t) * 3 * m.n_tris, cudaMemcpyHostToDevice, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    double t1 = now_ms();
    st.ms_upload = t1 - t0;
    P2M_TRY(m.d_tri.alloc(sizeof(float4) * 4 * T));
    P2M_TRY(m.d_tsph.alloc(sizeof(float4) * T));
    P2M_TRY(launch_tri_precompute(m.d_verts.as<float>(), m.d_tris.as<int32_t>(), T, m.d_tri.as<float4>(),
                                  m.d_tsph.as<float4>(), s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    double t2 = now_ms();
    st.ms_tri = t2 - t1;
    // K0: triangle LBVH
    {
        P2M_TRY(m.d_tlo.alloc(sizeof(float4) * T));
        P2M_TRY(m.d_thi.alloc(sizeof(float4) * T));
        P2M_TRY(tri_boxes(m.d_verts.as<float>(), m.d_tris.as<int32_t>(), T, m.d_tlo.as<float4>(), m.d_thi.as<float4>(), s));
        const float3 clo = make_float3((float)m.bb_lo[0], (float)m.bb_lo[1], (float)m.bb_lo[2]);
        const float3 chi = make_float3((float)m.bb_hi[0], (float)m.bb_hi[1], (float)m.bb_hi[2]);
        P2M_TRY(build_lbvh(m.d_tlo.as<float4>(), m.d_thi.as<float4>(), T, clo, chi, m.bvh, s, &m.d_orig));
        // renumber the triangle data in BVH leaf (Morton) order: list entries, which K1 emits
        // in leaf order, then read mostly contiguous records
        P2M_TRY(gather_f4(m.d_tri, m.d_orig.as<int>(), T, 4, s));
        P2M_TRY(gather_f4(m.d_tsph, m.d_orig.as<int>(), T, 1, s));
        P2M_TRY(gather_f4(m.d_tlo, m.d_orig.as<int>(), T, 1, s));
        P2M_TRY(gather_f4(m.d_thi, m.d_orig.as<int>(), T, 1, s));
        m.orig.resize(T);
        P2M_CUDA_TRY(cudaMemcpy(m.orig.data(), m.d_orig.p, sizeof(int32_t) * T, cudaMemcpyDeviceToHost));
    }
    double t3 = now_ms();
    st.ms_lbvh = t3 - t2;
    // list-scan schedule: 1 = thread per query for every list, 2 = warp per query for every
    // list, 0/3 = thread per query for lists up to long_list entries and warp per query beyond;
    // 0 also processes the queries in grid-cell Morton order, and 4 then regroups them by
    // nearest site.  Known before the lists are built: the lists scanned per thread are
    // stored ordered by their lower bound.
    const int long_list = prm.long_list > 0 ? prm.long_list : 256;
    m.long_row = prm.schedule == 1 ? 0x7fffffff : (prm.schedule == 2 ? 0 : long_list);
    m.sorted = prm.schedule == 0 || prm.schedule == 4;
    m.site_sorted = prm.schedule == 4;
    m.site_staged = prm.schedule == 5;
    // host Voronoi, augmentation, corner balls, lists, nearest-site grid
    P2M_TRY(build_partition(m, prm, h, s));
    st.ms_total = now_ms() - t0;
    return P2M_OK;
}

extern "C" {

const char* p2m_version(void) { return "p2mpp-gb300 0.1 (sm_103a)"; }

const char* p2m_last_error(void) { return g_err.c_str(); }

int p2m_default_params(p2m_build_params* out) {
    if (!out) return fail(P2M_ERR_INVALID_ARG, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    out->domain_scale = 1.5f;
    out->enable_aux = 1;
    out->tau_scale = 1.0f;
    out->density_factor = 8.0f;
    out->density_min = 256;
    out->ring_sites = 12;
    out->ring_radius_scale = 0.9f;  // just above sqrt(3) / 2
    out->build_eps_rel = 1e-6f;
    out->nn_grid_res = 0;
    out->schedule = 5;
    out->deterministic = 1;
    out->seed = 1;
    out->gpu_cells = 1;
    out->aux_balls = 1;
    out->aux_centre = 1;
    return P2M_OK;
}

static int new_index(const p2m_build_params* params, p2m_index** out, std::unique_ptr<p2m_index>& h) {
    if (!out) return fail(P2M_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    h.reset(new p2m_index());
    if (params) h->params = *params;
    else p2m_default_params(&h->params);
    P2M_TRY(validate_params(h->params));
    P2M_CUDA_TRY(cudaGetDevice(&h->device));
    P2M_TRY(h->status.alloc(sizeof(unsigned) * 4));
    P2M_CUDA_TRY(cudaMemset(h->status.p, 0, sizeof(unsigned) * 4));
    return P2M_OK;
}

int p2m_build(const float* verts, int64_t n_verts, const int32_t* tris, int64_t n_tris, int inputs_on_device,
              const p2m_build_params* params, void* stream, p2m_index** out) {
    std::unique_ptr<p2m_index> h;
    P2M_TRY(new_index(params, out, h));
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<MeshData> m(new MeshData());
    P2M_TRY(load_mesh(verts, n_verts, tris, n_tris, inputs_on_device, *m));
    P2M_TRY(build_mesh(*m, h->params, h.get(), s));
    P2M_TRY(check_status_word(h.get(), s, "build"));
    h->meshes.push_back(std::move(m));
    *out = h.release();
    return P2M_OK;
}

void p2m_destroy(p2m_index* h) {
    if (!h) return;
    cudaDeviceSynchronize();
    delete h;
}

int p2m_query(p2m_index* h, const float* d_pts, int64_t n, float* d_dist, float* d_closest, int32_t* d_tri,
              float* d_bary, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_query needs a single-mesh index");
    if (n < 0) return fail(P2M_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return P2M_OK;
    if (!d_pts || !d_dist) return fail(P2M_ERR_INVALID_ARG, "d_pts and d_dist must be non-NULL");
    P2M_TRY(check_call(h, n, "p2m_query"));
    return run_query(h, *h->meshes[0], d_pts, n, d_dist, d_closest, d_tri, d_bary, nullptr, h->scratch_idx,
                     (cudaStream_t)stream);
}

int p2m_query_counters(p2m_index* h, const float* d_pts, int64_t n, float* d_dist, p2m_counters* out,
                       void* stream) {
    if (!h || h->meshes.size() != 1 || !out) return fail(P2M_ERR_INVALID_ARG, "bad index or out");
    if (n < 0 || (n > 0 && !d_pts)) return fail(P2M_ERR_INVALID_ARG, "bad points");
    std::memset(out, 0, sizeof(*out));
    if (n == 0) return P2M_OK;
    P2M_TRY(check_call(h, n, "p2m_query_counters"));
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf cnt, dist;
    P2M_TRY(cnt.alloc(sizeof(unsigned long long) * 8));
    P2M_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long) * 8, s));
    float* dd = d_dist;
    if (!dd) {
        P2M_TRY(dist.alloc(sizeof(float) * n));
        dd = dist.as<float>();
    }
    P2M_TRY(run_query(h, *h->meshes[0], d_pts, n, dd, nullptr, nullptr, nullptr, cnt.as<unsigned long long>(),
                      h->scratch_idx, s));
    unsigned long long c[8];
    P2M_CUDA_TRY(cudaMemcpyAsync(c, cnt.p, sizeof(c), cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    P2M_TRY(check_status_word(h, s, "query"));
    out->n_queries = n;
    out->n_outside = (int64_t)c[0];
    out->site_candidates = (int64_t)c[1];
    out->tie_rechecks = (int64_t)c[2];
    out->row_entries = (int64_t)c[3];
    out->exact_tests = (int64_t)c[4];
    out->long_queries = (int64_t)c[5];
    out->long_entries = (int64_t)c[6];
    out->queried_list = (int64_t)c[7];
    return P2M_OK;
}

int p2m_nearest_site(p2m_index* h, const float* d_pts, int64_t n, int32_t* d_site, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_nearest_site needs a single-mesh index");
    if (n < 0 || (n > 0 && (!d_pts || !d_site))) return fail(P2M_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return P2M_OK;
    P2M_TRY(check_call(h, n, "p2m_nearest_site"));
    return run_nearest_site(h, *h->meshes[0], d_pts, n, d_site, (cudaStream_t)stream);
}

int p2m_get_stats(const p2m_index* h, p2m_stats* out) {
    if (!h || !out || h->meshes.empty()) return fail(P2M_ERR_INVALID_ARG, "bad index or out");
    if (h->meshes.size() == 1) {
        *out = h->meshes[0]->stats;
        return P2M_OK;
    }
    // batch: sums of counts, max of maxima, summed times
    p2m_stats a{};
    double rows = 0;
    for (auto& mp : h->meshes) {
        const p2m_stats& b = mp->stats;
        a.n_verts += b.n_verts; a.n_tris += b.n_tris; a.n_sites += b.n_sites;
        a.n_vertex_sites += b.n_vertex_sites; a.n_aux_sites += b.n_aux_sites; a.n_corners += b.n_corners;
        a.nnz += b.nnz; a.max_row = std::max(a.max_row, b.max_row); a.grid_entries += b.grid_entries;
        a.grid_max = std::max(a.grid_max, b.grid_max); a.grid_res = std::max(a.grid_res, b.grid_res);
        a.n_delaunay_tets += b.n_delaunay_tets; a.n_dense_cells += b.n_dense_cells;
        a.ms_upload += b.ms_upload; a.ms_tri += b.ms_tri; a.ms_lbvh += b.ms_lbvh; a.ms_delaunay += b.ms_delaunay;
        a.ms_cells += b.ms_cells; a.ms_aug += b.ms_aug; a.ms_proj += b.ms_proj; a.ms_k1 += b.ms_k1;
        a.ms_grid += b.ms_grid; a.ms_total += b.ms_total;
        a.n_cells_host += b.n_cells_host; a.ms_cells_kernel += b.ms_cells_kernel;
        a.ms_cells_fallback += b.ms_cells_fallback;
        a.aug_cell_max = std::max(a.aug_cell_max, b.aug_cell_max);
        rows += (double)b.n_sites;
    }
    a.avg_row = rows > 0 ? (double)a.nnz / rows : 0.0;
    *out = a;
    return P2M_OK;
}

int p2m_num_meshes(const p2m_index* h) { return h ? (int)h->meshes.size() : 0; }

static int mesh_of(const p2m_index* h, int mesh, MeshData** m) {
    if (!h || mesh < 0 || mesh >= (int)h->meshes.size()) return fail(P2M_ERR_INVALID_ARG, "bad index or mesh id");
    *m = h->meshes[mesh].get();
    return P2M_OK;
}

int p2m_get_sizes(const p2m_index* h, int mesh, int64_t* n_sites, int64_t* nnz, int64_t* n_balls) {
    MeshData* m;
    P2M_TRY(mesh_of(h, mesh, &m));
    if (n_sites) *n_sites = (int64_t)m->site_kind.size();
    if (nnz) *nnz = m->nnz;
    if (n_balls) *n_balls = (int64_t)m->ball_r.size();
    return P2M_OK;
}

int p2m_get_sites(const p2m_index* h, int mesh, float* h_sites, double* h_ref, int32_t* h_kind) {
    MeshData* m;
    P2M_TRY(mesh_of(h, mesh, &m));
    if (h_sites) std::memcpy(h_sites, m->site_pos.data(), sizeof(float) * m->site_pos.size());
    if (h_ref) std::memcpy(h_ref, m->site_ref.data(), sizeof(double) * m->site_ref.size());
    if (h_kind) std::memcpy(h_kind, m->site_kind.data(), sizeof(int32_t) * m->site_kind.size());
    return P2M_OK;
}

int p2m_get_lists(const p2m_index* h, int mesh, int64_t* h_offsets, int32_t* h_tri_ids) {
    MeshData* m;
    P2M_TRY(mesh_of(h, mesh, &m));
    const int64_t S = (int64_t)m->site_kind.size();
    std::vector<int32_t> off(S + 1);
    if (S > 0 && m->d_row_off.p)
        P2M_CUDA_TRY(cudaMemcpy(off.data(), m->d_row_off.p, sizeof(int32_t) * (S + 1), cudaMemcpyDeviceToHost));
    if (h_offsets)
        for (int64_t i = 0; i <= S; ++i) h_offsets[i] = off[i];
    if (h_tri_ids && m->nnz > 0) {
        std::vector<int2> ent(m->nnz);
        P2M_CUDA_TRY(cudaMemcpy(ent.data(), m->d_row_ent.p, sizeof(int2) * m->nnz, cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < m->nnz; ++k) h_tri_ids[k] = m->orig[ent[k].x];  // caller's triangle ids
    }
    return P2M_OK;
}

int p2m_set_timing(p2m_index* h, int on) {
    if (!h) return fail(P2M_ERR_INVALID_ARG, "NULL index");
    if (on)
        for (auto& e : h->tev)
            if (!e) P2M_CUDA_TRY(cudaEventCreate(&e));
    h->timing = on != 0;
    h->timed_call = false;
    return P2M_OK;
}

int p2m_query_timing(p2m_index* h, double* h_ms) {
    if (!h || !h_ms) return fail(P2M_ERR_INVALID_ARG, "NULL index or output");
    if (!h->timing || !h->timed_call) return fail(P2M_ERR_INVALID_ARG, "timing is off, or no query call was timed");
    P2M_CUDA_TRY(cudaEventSynchronize(h->tev[3]));
    float a = 0.f, b = 0.f;
    P2M_CUDA_TRY(cudaEventElapsedTime(&a, h->tev[1], h->tev[2]));
    P2M_CUDA_TRY(cudaEventElapsedTime(&b, h->tev[0], h->tev[3]));
    h_ms[0] = a;
    h_ms[1] = b;
    return P2M_OK;
}

int p2m_get_bvh(const p2m_index* h, int mesh, int64_t* n_nodes, int32_t* root, float* h_nodes, int32_t* h_leaf_tri) {
    MeshData* m;
    P2M_TRY(mesh_of(h, mesh, &m));
    const int64_t nn = m->bvh.n_prims > 1 ? m->bvh.n_prims - 1 : 0;
    if (n_nodes) *n_nodes = nn;
    if (root) *root = m->bvh.root;
    if (h_nodes && nn > 0)
        P2M_CUDA_TRY(cudaMemcpy(h_nodes, m->bvh.nodes.p, sizeof(BNode) * nn, cudaMemcpyDeviceToHost));
    if (h_leaf_tri) std::memcpy(h_leaf_tri, m->orig.data(), sizeof(int32_t) * m->orig.size());
    return P2M_OK;
}

int p2m_get_balls(const p2m_index* h, int mesh, int64_t* h_ball_offsets, double* h_centres, double* h_radii) {
    MeshData* m;
    P2M_TRY(mesh_of(h, mesh, &m));
    if (h_ball_offsets) std::memcpy(h_ball_offsets, m->ball_off.data(), sizeof(int64_t) * m->ball_off.size());
    if (h_centres) std::memcpy(h_centres, m->ball_c.data(), sizeof(double) * m->ball_c.size());
    if (h_radii) std::memcpy(h_radii, m->ball_r.data(), sizeof(double) * m->ball_r.size());
    return P2M_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- batch and update

extern "C" {

int p2m_batch_build(int n_meshes, const float* const* verts, const int64_t* n_verts, const int32_t* const* tris,
                    const int64_t* n_tris, const p2m_build_params* params, void* stream, p2m_index** out) {
    std::unique_ptr<p2m_index> h;
    P2M_TRY(new_index(params, out, h));
    if (n_meshes <= 0 || !verts || !n_verts || !tris || !n_tris)
        return fail(P2M_ERR_INVALID_ARG, "batch needs n_meshes > 0 and non-NULL arrays");
    h->meshes.resize(n_meshes);
    for (int i = 0; i < n_meshes; ++i) {
        h->meshes[i].reset(new MeshData());
        const int rc = load_mesh(verts[i], n_verts[i], tris[i], n_tris[i], 0, *h->meshes[i]);
        if (rc != P2M_OK) return fail(rc, "mesh " + std::to_string(i) + ": " + p2m_last_error());
    }
    // meshes build concurrently: each worker thread has its own stream and status word
    std::atomic<int> next(0), err_mesh(-1);
    std::mutex mu;
    std::string err_msg;
    int err_code = P2M_OK;
    const int n_workers = std::max(1, std::min(n_meshes, std::max(2, hardware_threads() / 2)));
    auto work = [&]() {
        cudaSetDevice(h->device);
        cudaStream_t ws = nullptr;
        if (cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) return;
        p2m_index local;
        local.params = h->params;
        local.device = h->device;
        if (local.status.alloc(sizeof(unsigned) * 4) == P2M_OK) cudaMemset(local.status.p, 0, sizeof(unsigned) * 4);
        while (err_mesh.load() < 0) {
            const int i = next.fetch_add(1);
            if (i >= n_meshes) break;
            int rc = build_mesh(*h->meshes[i], h->params, &local, ws);
            if (rc == P2M_OK) rc = check_status_word(&local, ws, "build");
            if (rc != P2M_OK) {
                std::lock_guard<std::mutex> lock(mu);
                if (err_mesh.load() < 0) {
                    err_mesh = i;
                    err_code = rc;
                    err_msg = p2m_last_error();
                }
            }
        }
        cudaStreamSynchronize(ws);
        cudaStreamDestroy(ws);
    };
    std::vector<std::thread> th;
    for (int t = 0; t < n_workers; ++t) th.emplace_back(work);
    for (auto& t : th) t.join();
    if (err_mesh.load() >= 0) return fail(err_code, "mesh " + std::to_string(err_mesh.load()) + ": " + err_msg);
    P2M_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *out = h.release();
    return P2M_OK;
}

int p2m_batch_query(p2m_index* batch, const float* d_pts, const int64_t* h_q_offsets, float* d_dist, float* d_closest,
                    int32_t* d_tri, float* d_bary, int mode, int use_graph, void* stream) {
    if (!batch || batch->meshes.empty() || !h_q_offsets) return fail(P2M_ERR_INVALID_ARG, "bad batch or offsets");
    P2M_TRY(check_call(batch, 0, "p2m_batch_query"));
    return run_batch_query(batch, d_pts, h_q_offsets, d_dist, d_closest, d_tri, d_bary, mode, use_graph,
                           (cudaStream_t)stream);
}

int p2m_update_vertices(p2m_index* h, const float* d_verts, void* stream) {
    if (!h || h->meshes.size() != 1 || !d_verts) return fail(P2M_ERR_INVALID_ARG, "p2m_update_vertices needs a single-mesh index");
    P2M_TRY(check_call(h, 0, "p2m_update_vertices"));
    cudaStream_t s = (cudaStream_t)stream;
    MeshData& old = *h->meshes[0];
    std::vector<float> v(old.n_verts * 3);
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    P2M_CUDA_TRY(cudaMemcpy(v.data(), d_verts, sizeof(float) * v.size(), cudaMemcpyDeviceToHost));
    std::unique_ptr<MeshData> m(new MeshData());
    P2M_TRY(load_mesh(v.data(), old.n_verts, old.tris.data(), old.n_tris, 0, *m));
    P2M_TRY(build_mesh(*m, h->params, h, s));
    P2M_TRY(check_status_word(h, s, "update_vertices"));
    h->meshes[0] = std::move(m);
    return P2M_OK;
}

}  // extern "C"
