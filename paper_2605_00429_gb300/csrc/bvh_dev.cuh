// Exact closest-triangle search by BVH branch and bound (device), shared by the single-mesh
// and the batched query kernels.
#pragma once

#include "geom.cuh"
#include "p2m_internal.h"

namespace p2m {

constexpr int kBvhStack = 64;

// Exact closest triangle of one query by branch and bound over the BVH.  Children are
// visited nearer-first; a subtree is skipped only when its box is farther than the bound
// lim = d_best (1 + 9.6e-7) + slack, padded like the list scan's bound, so every triangle
// whose distance rounds to the best is still compared by id and the result is the same
// (distance, id) minimum the list scan finds.  bound0: a starting bound on d(q, M) (the
// distance to a point of M, padded), or infinity.
__device__ __forceinline__ unsigned long long bvh_closest_key(float3 q, const BNode* __restrict__ nodes, int root,
                                                              const float4* __restrict__ tri, float& bs, float& bt,
                                                              unsigned* status, float bound0 = INFINITY,
                                                              float slack = 0.0f) {
    unsigned long long best = ~0ull;
    float lim = bound0;
    float best_d2 = lim * lim;
    if (root < 0) {
        float s, t;
        const TriRec T = load_tri(tri, ~root);
        const float d2 = tri_dist2(q, T, s, t);
        bs = s; bt = t;
        return dist_key(d2, ~root);
    }
    int stack[kBvhStack];
    float sdist[kBvhStack];
    int sp = 0;
    int node = root;
    while (true) {
        const float4* np = reinterpret_cast<const float4*>(nodes + node);
        const float4 lo0 = __ldg(np), hi0 = __ldg(np + 1), lo1 = __ldg(np + 2), hi1 = __ldg(np + 3);
        const int cs[2] = {__float_as_int(lo0.w), __float_as_int(lo1.w)};
        const float ds[2] = {box_dist2(q, f3(lo0), f3(hi0)), box_dist2(q, f3(lo1), f3(hi1))};
        const int first = (ds[1] < ds[0]) ? 1 : 0;
        int next = -1;
        // nearer child first; a deferred internal child goes on the stack with its box distance
        for (int h = 0; h < 2; ++h) {
            const int k = h == 0 ? first : 1 - first;
            const int c = cs[k];
            if (ds[k] > best_d2) continue;
            if (c < 0) {
                float s, t;
                const TriRec T = load_tri(tri, ~c);
                const float d2 = tri_dist2(q, T, s, t);
                const unsigned long long key = dist_key(d2, ~c);
                if (key < best) {
                    best = key;
                    bs = s;
                    bt = t;
                    lim = fminf(lim, fmaf(sqrtf(d2), 1.0f + 9.6e-7f, slack));
                    best_d2 = lim * lim;
                }
            } else if (next < 0) {
                next = c;
            } else if (sp < kBvhStack) {
                stack[sp] = c;
                sdist[sp] = ds[k];
                ++sp;
            } else {
                atomicOr(status, ST_STACK);
            }
        }
        if (next >= 0) { node = next; continue; }
        node = -1;
        while (sp > 0) {
            --sp;
            if (sdist[sp] <= best_d2) { node = stack[sp]; break; }
        }
        if (node < 0) break;
    }
    return best;
}

}  // namespace p2m
