// Device geometry for the P2M++ query path: triangle records, exact point-triangle
// distance, bounding-sphere pruning bound, box distance.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace p2m {

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(fmaf(a.y, b.z, -a.z * b.y), fmaf(a.z, b.x, -a.x * b.z), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

// a*b - c*d with one rounding error (Kahan's fma difference of products).
__device__ __forceinline__ float dop(float a, float b, float c, float d) {
    float cd = c * d;
    float err = fmaf(-c, d, cd);
    float r = fmaf(a, b, -cd);
    return r + err;
}

// Triangle record, 4 x float4 = 64 bytes; the first 32 bytes alone give a plane bound:
//   r0 = (u.xyz, 1/|n|)         n = e0 x e1 (compensated), u = n/|n| the unit normal
//   r1 = (v0.xyz, 1/|e0|^2)     e0 = v1 - v0
//   r2 = (e0.xyz, 1/|e1|^2)     e1 = v2 - v0
//   r3 = (e1.xyz, 1/|e2|^2)     e2 = v2 - v1
// 1/|n| is NaN and u = 0 for a triangle too thin to project onto (then only the edges are
// used, and the plane bound is 0).  A zero-length edge stores 1/|e|^2 = 0, which clamps its
// parameter to the start vertex.
struct TriRec {
    float4 r0, r1, r2, r3;
};

__device__ __forceinline__ TriRec load_tri(const float4* __restrict__ tri, int f) {
    const float4* p = tri + 4 * (int64_t)f;
    TriRec t;
    t.r0 = __ldg(p + 0);
    t.r1 = __ldg(p + 1);
    t.r2 = __ldg(p + 2);
    t.r3 = __ldg(p + 3);
    return t;
}

// Squared lower bound of the distance from q to triangle f that combines its supporting
// plane with its bounding sphere sp = (c, r).  Every point p of the triangle lies in the plane
// and within r of c, so |q - p|^2 = h^2 + |P(q - p)|^2 >= h^2 + max(0, rho - r)^2, with h the
// plane distance, P the projection onto the plane and rho = |P(q - c)|; this holds wherever
// c sits relative to the plane.  Near a surface it is much tighter than either bound alone:
// a triangle whose disc does not reach below q is pruned even when its plane is as close
// as the answer.  Rounding goes to the safe side: h loses h_slack, and rho^2 loses
// 4e-6 |q - c|^2 (the unit normal is good to a few ulps in direction and length, so the
// computed rho^2 is within about 1.5e-6 |q - c|^2 of the exact one).  dc2 = |q - c|^2.  A
// triangle too thin to project onto has u = 0 and the bound falls back to the sphere's.
// a, b = the first half of the triangle's record.
__device__ __forceinline__ float tri_lower_bound2_rec(float4 a, float4 b, float3 q, float4 sp, float dc2,
                                                      float h_slack) {
    const float3 u = f3(a);
    const float h = fmaxf(fabsf(dot3(u, q - f3(b))) - h_slack, 0.0f);
    const float hc = dot3(u, q - f3(sp));
    const float rho2 = fmaf(-4e-6f, dc2, fmaf(-hc, hc, dc2));
    const float g = fmaxf(sqrtf(fmaxf(rho2, 0.0f)) - sp.w, 0.0f);
    return fmaf(g, g, h * h);
}

__device__ __forceinline__ float tri_lower_bound2(const float4* __restrict__ tri, int f, float3 q, float4 sp,
                                                  float dc2, float h_slack) {
    const float4* p = tri + 4 * (int64_t)f;
    return tri_lower_bound2_rec(__ldg(p), __ldg(p + 1), q, sp, dc2, h_slack);
}

// Exact squared distance from q to the triangle; (s, t) locate the closest point
// p = v0 + s e0 + t e1 (barycentrics (1 - s - t, s, t)).
//
// Interior test by triple products: the projection of q onto the plane has in-plane
// coordinates s = ((w x e1) . u) / |n| and t = ((e0 x w) . u) / |n| with w = q - v0.
// If they lie in the triangle, d^2 = (w . u)^2.  Otherwise the closest point is on an edge
// whose supporting line separates the projection from the triangle; every edge is clamped
// and the best one kept.
__device__ __forceinline__ float tri_dist2(float3 q, const TriRec& T, float& s_out, float& t_out) {
    const float3 u = f3(T.r0), v0 = f3(T.r1), e0 = f3(T.r2), e1 = f3(T.r3);
    const float inv_n = T.r0.w;
    const float3 w = q - v0;
    const float s = dot3(cross3(w, e1), u) * inv_n;
    const float t = dot3(cross3(e0, w), u) * inv_n;
    if (s >= 0.0f && t >= 0.0f && s + t <= 1.0f) {
        const float h = dot3(w, u);
        s_out = s;
        t_out = t;
        return h * h;
    }
    // edge v0 -> v1 (t = 0)
    float k = clamp01(dot3(w, e0) * T.r1.w);
    float3 r = w - k * e0;
    float best = dot3(r, r);
    float bs = k, bt = 0.0f;
    // edge v0 -> v2 (s = 0)
    k = clamp01(dot3(w, e1) * T.r2.w);
    r = w - k * e1;
    float d = dot3(r, r);
    if (d < best) { best = d; bs = 0.0f; bt = k; }
    // edge v1 -> v2 (s + t = 1)
    const float3 w1 = w - e0;
    const float3 e2 = e1 - e0;
    k = clamp01(dot3(w1, e2) * T.r3.w);
    r = w1 - k * e2;
    d = dot3(r, r);
    if (d < best) { best = d; bs = 1.0f - k; bt = k; }
    s_out = bs;
    t_out = bt;
    return best;
}

// Closest point and barycentrics from a record and (s, t).
__device__ __forceinline__ float3 tri_point(const TriRec& T, float s, float t) {
    const float3 v0 = f3(T.r1), e0 = f3(T.r2), e1 = f3(T.r3);
    return make_float3(fmaf(t, e1.x, fmaf(s, e0.x, v0.x)), fmaf(t, e1.y, fmaf(s, e0.y, v0.y)),
                       fmaf(t, e1.z, fmaf(s, e0.z, v0.z)));
}

// Squared distance from q to an axis-aligned box.
__device__ __forceinline__ float box_dist2(float3 q, float3 lo, float3 hi) {
    const float dx = fmaxf(fmaxf(lo.x - q.x, q.x - hi.x), 0.0f);
    const float dy = fmaxf(fmaxf(lo.y - q.y, q.y - hi.y), 0.0f);
    const float dz = fmaxf(fmaxf(lo.z - q.z, q.z - hi.z), 0.0f);
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Ordered 64-bit key of (squared distance, triangle id): the minimum key is the closest
// triangle with ties resolved to the lower id.  d2 >= 0, so its float bits order as uint.
__device__ __forceinline__ unsigned long long dist_key(float d2, int id) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)id;
}

}  // namespace p2m
