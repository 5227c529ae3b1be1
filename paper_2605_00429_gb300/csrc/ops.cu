// Host-buffer query pipeline and the backward kernel (K4).
#include <algorithm>
#include <cstring>

#include "geom.cuh"
#include "host.h"

using namespace p2m;

namespace p2m {

// K4: gradient of sum_i g_i d(q_i, M) through the closest point p = sum_k b_k v_k of the
// forward pass:  dd/dq = (q - p)/d,  dd/dv_k = -b_k (q - p)/d  (0 where d = 0).
// Vertex sums either use float atomics, or fixed point in 64-bit integer atomics, whose sum
// does not depend on the order of the additions (bit-reproducible).  The fixed-point unit is
// 2^-e with e chosen per call from bound = max_i |g_i| max_k |b_k|: a contribution is at most
// bound in magnitude (|q - p| / d = 1), a vertex coordinate receives at most 3n of them (three
// per query when a triangle repeats a vertex), and e makes 3n * bound * 2^e <= 2^62, so no
// vertex sum can overflow.  Each contribution is rounded to the unit, an absolute error of at
// most 2^-(e+1) <= 3n * bound * 2^-63.
__global__ void k_grad_bound(const float* __restrict__ gdist, const float* __restrict__ bary, int64_t n,
                             unsigned* __restrict__ bound_bits) {
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float b = fmaxf(fabsf(bary[3 * i]), fmaxf(fabsf(bary[3 * i + 1]), fabsf(bary[3 * i + 2])));
        const float c = fabsf(gdist[i]) * fmaxf(b, 1.0f);
        // NaN is kept (its bits order above infinity) so the caller sees a non-finite bound
        m = (c > m || c != c) ? c : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float x = __shfl_xor_sync(0xffffffffu, m, o);
        m = (x > m || x != x) ? x : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(bound_bits, __float_as_uint(m));  // |x| >= 0: bits order as uint
}

// Exponent e of the fixed-point unit 2^-e for n contributions of magnitude <= bound; 0 when
// every contribution is 0; -1000 when the bound is not finite (the caller flags it).
__device__ __forceinline__ int grad_exponent(unsigned bound_bits, int64_t n) {
    const float bound = __uint_as_float(bound_bits);
    if (!(bound <= 3.0e38f)) return -1000;
    if (bound == 0.0f) return 0;
    int ex;
    frexp((double)bound * (double)n * 1.0001, &ex);  // bound * n * 1.0001 < 2^ex
    return 62 - ex;
}

template <bool DET>
__global__ void k_backward(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                           const float* __restrict__ pts, int64_t n, const int32_t* __restrict__ tri,
                           const float* __restrict__ bary, const float* __restrict__ gdist, float* __restrict__ gpts,
                           float* __restrict__ gverts, unsigned long long* __restrict__ gacc,
                           const unsigned* __restrict__ bound_bits, int n_tris, unsigned* status) {
    double scale = 0.0;
    if (DET) {
        const int e = grad_exponent(*bound_bits, 3 * n);  // a vertex gets at most 3 per query
        if (e == -1000) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_LIMIT);
            return;
        }
        scale = ldexp(1.0, e);
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = tri[i];
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        const float g = gdist[i];
        if (f < 0 || f >= n_tris) {
            if (gpts) { gpts[3 * i] = 0.f; gpts[3 * i + 1] = 0.f; gpts[3 * i + 2] = 0.f; }
            continue;
        }
        const float b[3] = {bary[3 * i], bary[3 * i + 1], bary[3 * i + 2]};
        int vi[3];
        float3 p = make_float3(0.f, 0.f, 0.f);
        for (int k = 0; k < 3; ++k) {
            vi[k] = tris[3 * f + k];
            p.x = fmaf(b[k], verts[3 * vi[k]], p.x);
            p.y = fmaf(b[k], verts[3 * vi[k] + 1], p.y);
            p.z = fmaf(b[k], verts[3 * vi[k] + 2], p.z);
        }
        const float3 d = q - p;
        const float len = sqrtf(dot3(d, d));
        const float s = len > 0.f ? g / len : 0.f;
        const float3 u = s * d;  // g (q - p) / d
        if (gpts) { gpts[3 * i] = u.x; gpts[3 * i + 1] = u.y; gpts[3 * i + 2] = u.z; }
        if (gverts) {
            for (int k = 0; k < 3; ++k) {
                const float c[3] = {-b[k] * u.x, -b[k] * u.y, -b[k] * u.z};
                for (int a = 0; a < 3; ++a) {
                    if (DET) {
                        const long long fx = __double2ll_rn((double)c[a] * scale);
                        atomicAdd(gacc + 3 * (int64_t)vi[k] + a, (unsigned long long)fx);
                    } else {
                        atomicAdd(gverts + 3 * (int64_t)vi[k] + a, c[a]);
                    }
                }
            }
        }
    }
}

__global__ void k_fixed_to_float_add(const unsigned long long* __restrict__ acc, const unsigned* __restrict__ bound_bits,
                                     int64_t n_contrib, float* __restrict__ out, int64_t n) {
    const int e = grad_exponent(*bound_bits, n_contrib);
    if (e == -1000) return;
    const double unit = ldexp(1.0, -e);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] += (float)((double)(long long)acc[i] * unit);
}

// Sign of the distance from the closest feature's pseudonormal.  The feature comes from the
// barycentrics, which the closest-point routine leaves exactly 0 / 1 on edges and vertices:
// two zeros = vertex, one zero = the edge opposite that vertex, none = the face.
__global__ void k_sign(const float* __restrict__ verts, const int32_t* __restrict__ tris, const float4* __restrict__ snorm,
                       const float4* __restrict__ vnorm, const float* __restrict__ pts, int64_t n,
                       const int32_t* __restrict__ tri, const float* __restrict__ bary, float* __restrict__ dist,
                       int n_tris) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = tri[i];
        if (f < 0 || f >= n_tris) continue;
        const float b[3] = {bary[3 * i], bary[3 * i + 1], bary[3 * i + 2]};
        int vi[3];
        float3 p = make_float3(0.f, 0.f, 0.f);
        for (int k = 0; k < 3; ++k) {
            vi[k] = tris[3 * f + k];
            p.x = fmaf(b[k], verts[3 * vi[k]], p.x);
            p.y = fmaf(b[k], verts[3 * vi[k] + 1], p.y);
            p.z = fmaf(b[k], verts[3 * vi[k] + 2], p.z);
        }
        const int nz = (b[0] == 0.0f) + (b[1] == 0.0f) + (b[2] == 0.0f);
        float4 nrm;
        if (nz >= 2) {
            const int k = b[0] != 0.0f ? 0 : (b[1] != 0.0f ? 1 : 2);
            nrm = vnorm[vi[k]];
        } else if (nz == 1) {
            const int k = b[0] == 0.0f ? 0 : (b[1] == 0.0f ? 1 : 2);
            nrm = snorm[4 * (int64_t)f + 1 + (k + 1) % 3];  // edge (v_k+1, v_k+2)
        } else {
            nrm = snorm[4 * (int64_t)f];
        }
        const float3 q = make_float3(pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
        if (dot3(q - p, f3(nrm)) < 0.0f) dist[i] = -dist[i];
    }
}

// Sample points of mesh B: the barycentric lattice ((k-i-j) v0 + i v1 + j v2) / k of every
// triangle (k = subdivisions; k = 0 gives the vertices of each triangle).
__global__ void k_mesh_samples(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t n_tris, int k,
                               float* __restrict__ out) {
    const int per = k == 0 ? 3 : (k + 1) * (k + 2) / 2;
    const int64_t total = n_tris * per;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = t / per;
        int r = (int)(t % per);
        float w0, w1, w2;
        if (k == 0) {
            w0 = r == 0; w1 = r == 1; w2 = r == 2;
        } else {
            int i = 0;  // row i holds k - i + 1 points
            while (r > k - i) { r -= k - i + 1; ++i; }
            const int j = r;
            w1 = (float)i / (float)k;
            w2 = (float)j / (float)k;
            w0 = (float)(k - i - j) / (float)k;
        }
        const int a = tris[3 * f], b = tris[3 * f + 1], c = tris[3 * f + 2];
        for (int d = 0; d < 3; ++d)
            out[3 * t + d] = fmaf(w0, verts[3 * a + d], fmaf(w1, verts[3 * b + d], w2 * verts[3 * c + d]));
    }
}

// min / max / sum of n distances (one block-reduced atomic per block; distances >= 0, so
// their float bits order as unsigned integers)
__global__ void k_dist_stats(const float* __restrict__ d, int64_t n, unsigned* __restrict__ mn, unsigned* __restrict__ mx,
                             double* __restrict__ sum) {
    float lmin = INFINITY, lmax = 0.0f;
    double lsum = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = d[i];
        lmin = fminf(lmin, v);
        lmax = fmaxf(lmax, v);
        lsum += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
        lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mn, __float_as_uint(lmin));
        atomicMax(mx, __float_as_uint(lmax));
        atomicAdd(sum, lsum);
    }
}

}  // namespace p2m

extern "C" {

int p2m_mesh_distance_pair(p2m_index* a, p2m_index* b, int subdivisions, double* h_out, void* stream) {
    if (!a || !b || a->meshes.size() != 1 || b->meshes.size() != 1 || !h_out)
        return fail(P2M_ERR_INVALID_ARG, "p2m_mesh_distance_pair needs two single-mesh indexes and h_out");
    const MeshData& ma = *a->meshes[0];
    const MeshData& mb = *b->meshes[0];
    P2M_TRY(p2m_mesh_distance(a, mb.d_verts.as<const float>(), mb.n_verts, mb.d_tris.as<const int32_t>(), mb.n_tris,
                              subdivisions, h_out, stream));
    P2M_TRY(p2m_mesh_distance(b, ma.d_verts.as<const float>(), ma.n_verts, ma.d_tris.as<const int32_t>(), ma.n_tris,
                              subdivisions, h_out + 3, stream));
    h_out[6] = std::max(h_out[1], h_out[4]);
    return P2M_OK;
}

int p2m_mesh_distance(p2m_index* h, const float* d_verts_b, int64_t n_verts_b, const int32_t* d_tris_b,
                      int64_t n_tris_b, int subdivisions, double* h_out, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_mesh_distance needs a single-mesh index");
    if (!d_verts_b || !d_tris_b || !h_out || n_verts_b <= 0 || n_tris_b <= 0 || subdivisions < 0 || subdivisions > 64)
        return fail(P2M_ERR_INVALID_ARG, "bad mesh B or subdivisions (0..64)");
    cudaStream_t s = (cudaStream_t)stream;
    MeshData& m = *h->meshes[0];
    P2M_TRY(check_call(h, n_tris_b * ((subdivisions + 1) * (subdivisions + 2) / 2 + 3), "p2m_mesh_distance"));
    const int per = subdivisions == 0 ? 3 : (subdivisions + 1) * (subdivisions + 2) / 2;
    const int64_t n = n_tris_b * per;
    DevBuf pts, dist, stats;
    P2M_TRY(pts.alloc(sizeof(float) * 3 * n));
    P2M_TRY(dist.alloc(sizeof(float) * n));
    P2M_TRY(stats.alloc(64));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, sm_count() * 32);
    k_mesh_samples<<<blocks, 256, 0, s>>>(d_verts_b, d_tris_b, n_tris_b, subdivisions, pts.as<float>());
    P2M_CUDA_TRY(cudaGetLastError());
    P2M_TRY(run_query(h, m, pts.as<float>(), n, dist.as<float>(), nullptr, nullptr, nullptr, nullptr, h->scratch_idx, s));
    unsigned init[2] = {0x7f800000u, 0u};
    P2M_CUDA_TRY(cudaMemsetAsync(stats.p, 0, 64, s));
    P2M_CUDA_TRY(cudaMemcpyAsync(stats.p, init, sizeof(init), cudaMemcpyHostToDevice, s));
    unsigned* su = stats.as<unsigned>();
    k_dist_stats<<<blocks, 256, 0, s>>>(dist.as<float>(), n, su, su + 1, reinterpret_cast<double*>(stats.as<char>() + 8));
    P2M_CUDA_TRY(cudaGetLastError());
    unsigned char host[16];
    P2M_CUDA_TRY(cudaMemcpyAsync(host, stats.p, 16, cudaMemcpyDeviceToHost, s));
    P2M_CUDA_TRY(cudaStreamSynchronize(s));
    P2M_TRY(check_status_word(h, s, "mesh distance"));
    unsigned umin, umax;
    double dsum;
    std::memcpy(&umin, host, 4);
    std::memcpy(&umax, host + 4, 4);
    std::memcpy(&dsum, host + 8, 8);
    float fmin, fmax;
    std::memcpy(&fmin, &umin, 4);
    std::memcpy(&fmax, &umax, 4);
    h_out[0] = fmin;
    h_out[1] = fmax;
    h_out[2] = dsum / (double)n;
    (void)n_verts_b;
    return P2M_OK;
}

int p2m_query_signed(p2m_index* h, const float* d_pts, int64_t n, float* d_sdist, float* d_closest, int32_t* d_tri,
                     float* d_bary, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_query_signed needs a single-mesh index");
    if (n < 0) return fail(P2M_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return P2M_OK;
    if (!d_pts || !d_sdist) return fail(P2M_ERR_INVALID_ARG, "d_pts and d_sdist must be non-NULL");
    P2M_TRY(check_call(h, n, "p2m_query_signed"));
    cudaStream_t s = (cudaStream_t)stream;
    MeshData& m = *h->meshes[0];
    if (!m.d_snorm.p) P2M_TRY(build_pseudonormals(m));
    // the sign needs the triangle and barycentrics: use the caller's buffers or scratch
    int32_t* tri = d_tri;
    float* bary = d_bary;
    if (!tri || !bary) {
        P2M_TRY(h->sign_scratch.ensure((sizeof(int32_t) + 3 * sizeof(float)) * n + 256));
        if (!tri) tri = h->sign_scratch.as<int32_t>();
        if (!bary) bary = reinterpret_cast<float*>(h->sign_scratch.as<char>() + ((sizeof(int32_t) * n + 255) / 256) * 256);
    }
    P2M_TRY(run_query(h, m, d_pts, n, d_sdist, d_closest, tri, bary, nullptr, h->scratch_idx, s));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, sm_count() * 32);
    k_sign<<<blocks, 256, 0, s>>>(m.d_verts.as<float>(), m.d_tris.as<int32_t>(), m.d_snorm.as<float4>(),
                                  m.d_vnorm.as<float4>(), d_pts, n, tri, bary, d_sdist, (int)m.n_tris);
    P2M_CUDA_TRY(cudaGetLastError());
    return P2M_OK;
}

int p2m_backward(p2m_index* h, const float* d_pts, int64_t n, const int32_t* d_tri, const float* d_bary,
                 const float* d_grad_dist, float* d_grad_pts, float* d_grad_verts, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_backward needs a single-mesh index");
    if (n < 0) return fail(P2M_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return P2M_OK;
    if (!d_pts || !d_tri || !d_bary || !d_grad_dist) return fail(P2M_ERR_INVALID_ARG, "NULL input");
    P2M_TRY(check_call(h, 0, "p2m_backward"));
    cudaStream_t s = (cudaStream_t)stream;
    MeshData& m = *h->meshes[0];
    const int64_t nv3 = m.n_verts * 3;
    const bool det = h->params.deterministic && d_grad_verts;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, sm_count() * 32);
    unsigned* bound = nullptr;
    if (det) {
        // accumulator [nv3] int64, then the contribution bound word
        P2M_TRY(h->grad_acc.ensure(sizeof(unsigned long long) * nv3 + 16));
        P2M_CUDA_TRY(cudaMemsetAsync(h->grad_acc.p, 0, sizeof(unsigned long long) * nv3 + 16, s));
        bound = reinterpret_cast<unsigned*>(h->grad_acc.as<unsigned long long>() + nv3);
        k_grad_bound<<<blocks, threads, 0, s>>>(d_grad_dist, d_bary, n, bound);
        P2M_CUDA_TRY(cudaGetLastError());
    }
    if (det)
        k_backward<true><<<blocks, threads, 0, s>>>(m.d_verts.as<float>(), m.d_tris.as<int32_t>(), d_pts, n, d_tri, d_bary,
                                                     d_grad_dist, d_grad_pts, d_grad_verts,
                                                     h->grad_acc.as<unsigned long long>(), bound, (int)m.n_tris,
                                                     index_status(h));
    else
        k_backward<false><<<blocks, threads, 0, s>>>(m.d_verts.as<float>(), m.d_tris.as<int32_t>(), d_pts, n, d_tri,
                                                      d_bary, d_grad_dist, d_grad_pts, d_grad_verts, nullptr, nullptr,
                                                      (int)m.n_tris, index_status(h));
    P2M_CUDA_TRY(cudaGetLastError());
    if (det) {
        k_fixed_to_float_add<<<(int)std::min<int64_t>((nv3 + 255) / 256, 4096), 256, 0, s>>>(
            h->grad_acc.as<unsigned long long>(), bound, 3 * n, d_grad_verts, nv3);
        P2M_CUDA_TRY(cudaGetLastError());
    }
    return P2M_OK;
}

int p2m_query_host(p2m_index* h, const float* h_pts, int64_t n, float* h_dist, float* h_closest, int32_t* h_tri,
                   float* h_bary, void* stream) {
    if (!h || h->meshes.size() != 1) return fail(P2M_ERR_INVALID_ARG, "p2m_query_host needs a single-mesh index");
    if (n < 0) return fail(P2M_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return P2M_OK;
    if (!h_pts || !h_dist) return fail(P2M_ERR_INVALID_ARG, "h_pts and h_dist must be non-NULL");
    P2M_TRY(check_call(h, 0, "p2m_query_host"));
    MeshData& m = *h->meshes[0];
    cudaStream_t user = (cudaStream_t)stream;
    constexpr int kSlots = p2m_index::kPipe;
    for (auto& st : h->streams)
        if (!st) P2M_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto& slot : h->pipe_ev)
        for (auto& e : slot)
            if (!e) P2M_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaStream_t s_in = h->streams[0], s_run = h->streams[1], s_out = h->streams[2];
    // the pipeline starts after the caller's earlier work on `stream`
    Event ev;
    P2M_CUDA_TRY(cudaEventCreateWithFlags(&ev.e, cudaEventDisableTiming));
    P2M_CUDA_TRY(cudaEventRecord(ev.e, user));
    for (auto& st : h->streams) P2M_CUDA_TRY(cudaStreamWaitEvent(st, ev.e, 0));
    // Chunks of ~n/k points (at least 1M): chunk c's points go in on the copy-in stream, its
    // query runs on the compute stream, its results go out on the copy-out stream.  The
    // chunks' kernels run one after another, so chunk c's results leave while chunk c+1
    // computes and chunk c+2's points arrive.  A buffer slot is reused once its previous
    // chunk's results are out.
    const int64_t k_chunks = h->params.pipe_chunks > 0 ? h->params.pipe_chunks : 3;
    const int64_t chunk = std::min<int64_t>(n, std::max<int64_t>((int64_t)1 << 20, (n + k_chunks - 1) / k_chunks));
    for (int k = 0; k < kSlots; ++k) {
        P2M_TRY(h->pipe[k][0].ensure(sizeof(float) * 3 * chunk));
        P2M_TRY(h->pipe[k][1].ensure(sizeof(float) * chunk));
        if (h_closest) P2M_TRY(h->pipe[k][2].ensure(sizeof(float) * 3 * chunk));
        if (h_tri) P2M_TRY(h->pipe[k][3].ensure(sizeof(int32_t) * chunk));
        if (h_bary) P2M_TRY(h->pipe[k][4].ensure(sizeof(float) * 3 * chunk));
    }
    int64_t ci = 0;
    for (int64_t b = 0; b < n; b += chunk, ++ci) {
        const int slot = (int)(ci % kSlots);
        const int64_t c = std::min(chunk, n - b);
        DevBuf* P = h->pipe[slot];
        cudaEvent_t* E = h->pipe_ev[slot];  // [0] copied in, [1] computed, [2] copied out
        if (ci >= kSlots) P2M_CUDA_TRY(cudaStreamWaitEvent(s_in, E[2], 0));
        P2M_CUDA_TRY(cudaMemcpyAsync(P[0].p, h_pts + 3 * b, sizeof(float) * 3 * c, cudaMemcpyHostToDevice, s_in));
        P2M_CUDA_TRY(cudaEventRecord(E[0], s_in));
        P2M_CUDA_TRY(cudaStreamWaitEvent(s_run, E[0], 0));
        if (ci >= kSlots) P2M_CUDA_TRY(cudaStreamWaitEvent(s_run, E[2], 0));
        P2M_TRY(run_query(h, m, P[0].as<float>(), c, P[1].as<float>(), h_closest ? P[2].as<float>() : nullptr,
                          h_tri ? P[3].as<int32_t>() : nullptr, h_bary ? P[4].as<float>() : nullptr, nullptr,
                          h->pipe_rest[slot], s_run));
        P2M_CUDA_TRY(cudaEventRecord(E[1], s_run));
        P2M_CUDA_TRY(cudaStreamWaitEvent(s_out, E[1], 0));
        P2M_CUDA_TRY(cudaMemcpyAsync(h_dist + b, P[1].p, sizeof(float) * c, cudaMemcpyDeviceToHost, s_out));
        if (h_closest)
            P2M_CUDA_TRY(cudaMemcpyAsync(h_closest + 3 * b, P[2].p, sizeof(float) * 3 * c, cudaMemcpyDeviceToHost, s_out));
        if (h_tri) P2M_CUDA_TRY(cudaMemcpyAsync(h_tri + b, P[3].p, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, s_out));
        if (h_bary) P2M_CUDA_TRY(cudaMemcpyAsync(h_bary + 3 * b, P[4].p, sizeof(float) * 3 * c, cudaMemcpyDeviceToHost, s_out));
        P2M_CUDA_TRY(cudaEventRecord(E[2], s_out));
    }
    for (auto& st : h->streams) P2M_CUDA_TRY(cudaStreamSynchronize(st));
    return check_status_word(h, h->streams[0], "query");
}

}  // extern "C"
