// Closest-hit / any-hit tracing: stack-based traversal of the quantised BVH2
// (Sec. 3.1) with the Moller-Trumbore ray/triangle test (1997).  GB300 has no
// ray-tracing cores, so traversal is software: one thread per ray, 32-byte
// nodes holding both children's 8-bit boxes, a per-thread stack of
// (node, entry distance) pairs.
//
// Robustness: decoded child boxes are rounded outward (they contain the exact
// boxes), the slab test widens the far distance by 1 + 2*gamma(3) (Ize 2013,
// "Robust BVH Ray Traversal"), and a subtree is dropped only when its entry
// distance exceeds the best hit by more than 2^-16 relative, so traversal
// never loses a triangle that the closest-hit definition would pick.
// Triangle arithmetic is the canonical Moller-Trumbore sequence with explicit
// round-to-nearest intrinsics (built with --fmad=false), so the (t, u, v) of
// a triangle are the same bit patterns on every run and in every ray order.
#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int TRACE_BLOCK = 128;
constexpr int STACK = HCC_TRACE_STACK;
// 1 + 2 * gamma(3), gamma(n) = n u / (1 - n u), u = 2^-24
constexpr float ROBUST_FAR = 1.0000003576279f;
constexpr float PRUNE_SLACK = 1.0f + 1.0f / 65536.0f;

__device__ __forceinline__ float byte_to_float(uint32_t w, uint32_t sel) {
    // 0x4B0000bb as float is 2^23 + bb exactly
    return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, sel)), 8388608.0f);
}
// selectors for byte 0..3 of w combined with bytes of 0x4B000000
constexpr uint32_t SEL0 = 0x7540u, SEL1 = 0x7541u, SEL2 = 0x7542u, SEL3 = 0x7543u;

struct Ray {
    float ox, oy, oz, tmin, dx, dy, dz, tmax, ix, iy, iz;
};

__device__ __forceinline__ float safe_inv(float d) {
    // a zero (or denormal) direction component is replaced by +-1e-30 for the
    // slab test only; this keeps every slab distance a number (no 0 * inf)
    return __frcp_rn(fabsf(d) > 1e-30f ? d : copysignf(1e-30f, d));
}

// Entry / exit distance of the ray through one decoded child box.
__device__ __forceinline__ void slab(const Ray &r, float lox, float loy, float loz, float hix, float hiy, float hiz,
                                     float tcap, float &tn, float &tf) {
    const float ax = __fmul_rn(__fsub_rn(lox, r.ox), r.ix), bx = __fmul_rn(__fsub_rn(hix, r.ox), r.ix);
    const float ay = __fmul_rn(__fsub_rn(loy, r.oy), r.iy), by = __fmul_rn(__fsub_rn(hiy, r.oy), r.iy);
    const float az = __fmul_rn(__fsub_rn(loz, r.oz), r.iz), bz = __fmul_rn(__fsub_rn(hiz, r.oz), r.iz);
    tn = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), r.tmin));
    const float f = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fmaxf(az, bz));
    tf = fminf(__fmul_rn(f, ROBUST_FAR), tcap);
}

// Moller-Trumbore on record k; returns true with (t, u, v) on a hit in
// (tmin, tmax).  Same operation sequence as the definition: p = d x e2,
// det = e1 . p, s = o - v0, u = (s . p) / det, q = s x e1, v = (d . q) / det,
// t = (e2 . q) / det; dot(a, b) = fma(az, bz, fma(ay, by, ax * bx)),
// cross(a, b).x = fma(ay, bz, -(az * by)) and cyclically.
__device__ __forceinline__ bool intersect(const Ray &r, const float4 &A, const float4 &E1, const float4 &E2, float &t,
                                          float &u, float &v) {
    const float px = __fmaf_rn(r.dy, E2.z, -__fmul_rn(r.dz, E2.y));
    const float py = __fmaf_rn(r.dz, E2.x, -__fmul_rn(r.dx, E2.z));
    const float pz = __fmaf_rn(r.dx, E2.y, -__fmul_rn(r.dy, E2.x));
    const float det = __fmaf_rn(E1.z, pz, __fmaf_rn(E1.y, py, __fmul_rn(E1.x, px)));
    if (det == 0.0f) return false;
    const float inv = __frcp_rn(det);
    const float sx = __fsub_rn(r.ox, A.x), sy = __fsub_rn(r.oy, A.y), sz = __fsub_rn(r.oz, A.z);
    u = __fmul_rn(__fmaf_rn(sz, pz, __fmaf_rn(sy, py, __fmul_rn(sx, px))), inv);
    if (u < 0.0f || u > 1.0f) return false;
    const float qx = __fmaf_rn(sy, E1.z, -__fmul_rn(sz, E1.y));
    const float qy = __fmaf_rn(sz, E1.x, -__fmul_rn(sx, E1.z));
    const float qz = __fmaf_rn(sx, E1.y, -__fmul_rn(sy, E1.x));
    v = __fmul_rn(__fmaf_rn(r.dz, qz, __fmaf_rn(r.dy, qy, __fmul_rn(r.dx, qx))), inv);
    if (v < 0.0f || __fadd_rn(u, v) > 1.0f) return false;
    t = __fmul_rn(__fmaf_rn(E2.z, qz, __fmaf_rn(E2.y, qy, __fmul_rn(E2.x, qx))), inv);
    return t > r.tmin && t < r.tmax;
}

// COUNT = true is a diagnostic variant that also adds up internal-node
// visits and triangle tests into a.counts[0..1] (never the timed kernel).
template <bool ANY, bool COUNT>
__global__ void __launch_bounds__(TRACE_BLOCK) k_trace(TraceArgs a) {
    const uint64_t i = (uint64_t)blockIdx.x * TRACE_BLOCK + threadIdx.x;
    uint32_t n_nodes = 0, n_tris = 0;
    if (i >= a.n) return;
    const float4 o4 = __ldcs(a.org + i), d4 = __ldcs(a.dir + i);
    Ray r;
    r.ox = o4.x;
    r.oy = o4.y;
    r.oz = o4.z;
    r.tmin = o4.w;
    r.dx = d4.x;
    r.dy = d4.y;
    r.dz = d4.z;
    r.tmax = d4.w;
    r.ix = safe_inv(d4.x);
    r.iy = safe_inv(d4.y);
    r.iz = safe_inv(d4.z);

    float best_t = r.tmax, best_u = 0.0f, best_v = 0.0f;
    int32_t best_prim = -1;
    float tcap = r.tmax;  // best_t widened by the prune slack
    uint32_t st_ref[STACK];
    float st_t[STACK];
    int sp = 0;
    uint32_t ref = a.root_ref;
    bool overflow = false;

    for (;;) {
        bool have = true;
        // descend through internal nodes until a leaf is reached or the stack runs dry
        while (!(ref & REF_LEAF)) {
            const uint4 A = __ldg(a.nodes + 2 * (size_t)ref);
            const uint4 B = __ldg(a.nodes + 2 * (size_t)ref + 1);
            if (COUNT) ++n_nodes;
            const float ox = __uint_as_float(A.x & 0xFFFFFF00u);
            const float oy = __uint_as_float(A.y & 0xFFFFFF00u);
            const float oz = __uint_as_float(A.z & 0xFFFFFF00u);
            const float sx = __uint_as_float((A.x & 0xFFu) << 23);
            const float sy = __uint_as_float((A.y & 0xFFu) << 23);
            const float sz = __uint_as_float((A.z & 0xFFu) << 23);
            float tn0, tf0, tn1, tf1;
            slab(r, __fmaf_rd(byte_to_float(A.w, SEL0), sx, ox), __fmaf_rd(byte_to_float(A.w, SEL1), sy, oy),
                 __fmaf_rd(byte_to_float(A.w, SEL2), sz, oz), __fmaf_ru(byte_to_float(A.w, SEL3), sx, ox),
                 __fmaf_ru(byte_to_float(B.x, SEL0), sy, oy), __fmaf_ru(byte_to_float(B.x, SEL1), sz, oz), tcap,
                 tn0, tf0);
            slab(r, __fmaf_rd(byte_to_float(B.x, SEL2), sx, ox), __fmaf_rd(byte_to_float(B.x, SEL3), sy, oy),
                 __fmaf_rd(byte_to_float(B.y, SEL0), sz, oz), __fmaf_ru(byte_to_float(B.y, SEL1), sx, ox),
                 __fmaf_ru(byte_to_float(B.y, SEL2), sy, oy), __fmaf_ru(byte_to_float(B.y, SEL3), sz, oz), tcap,
                 tn1, tf1);
            const bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
            if (h0 && h1) {
                const bool first0 = tn0 <= tn1;
                if (sp == STACK) {
                    overflow = true;
                    have = false;
                    break;
                }
                st_ref[sp] = first0 ? B.w : B.z;
                st_t[sp] = first0 ? tn1 : tn0;
                ++sp;
                ref = first0 ? B.z : B.w;
            } else if (h0) {
                ref = B.z;
            } else if (h1) {
                ref = B.w;
            } else {
                // pop the nearest pending subtree that can still hold a closer hit
                have = false;
                while (sp > 0) {
                    --sp;
                    if (st_t[sp] <= tcap) {
                        ref = st_ref[sp];
                        have = true;
                        break;
                    }
                }
                if (!have) break;
            }
        }
        if (!have) break;
        // leaf: test its triangles
        const uint32_t first = ref & REF_TRI_MASK, cnt = ((ref >> 29) & 3u) + 1u;
        bool done = false;
        for (uint32_t k = 0; k < cnt; ++k) {
            const float4 *rec = a.tris + 3 * (size_t)(first + k);
            const float4 A = __ldg(rec), E1 = __ldg(rec + 1), E2 = __ldg(rec + 2);
            if (COUNT) ++n_tris;
            float t, u, v;
            if (!intersect(r, A, E1, E2, t, u, v)) continue;
            const int32_t prim = __float_as_int(A.w);
            if (best_prim < 0 || t < best_t || (t == best_t && prim < best_prim)) {
                best_t = t;
                best_u = u;
                best_v = v;
                best_prim = prim;
                tcap = __fmul_rn(t, PRUNE_SLACK);
            }
            if (ANY) {
                done = true;
                break;
            }
        }
        if (done) break;
        // continue with the nearest pending subtree
        bool popped = false;
        while (sp > 0) {
            --sp;
            if (st_t[sp] <= tcap) {
                ref = st_ref[sp];
                popped = true;
                break;
            }
        }
        if (!popped) break;
    }
    if (overflow) {
        atomicOr(a.err, ERR_STACK);
        best_prim = -1;
    }
    int4 out;
    out.x = best_prim;
    out.y = __float_as_int(best_prim < 0 ? __int_as_float(0x7F800000) : best_t);
    out.z = __float_as_int(best_prim < 0 ? 0.0f : best_u);
    out.w = __float_as_int(best_prim < 0 ? 0.0f : best_v);
    const uint64_t dst = a.scatter ? (uint64_t)a.scatter[i] : i;
    if (dst < a.n)
        a.hits[dst] = out;
    else  // invalid scatter entry: report, never write out of bounds
        atomicOr(a.err, ERR_INDEX);
    if (COUNT) {
        atomicAdd(a.counts, (unsigned long long)n_nodes);
        atomicAdd(a.counts + 1, (unsigned long long)n_tris);
    }
}

}  // namespace

cudaError_t launch_trace(cudaStream_t s, const TraceArgs &a, int any_hit) {
    if (a.n == 0) return cudaSuccess;
    const uint64_t blocks = (a.n + TRACE_BLOCK - 1) / TRACE_BLOCK;
    const bool count = a.counts != nullptr;
    if (any_hit && count)
        k_trace<true, true><<<(unsigned)blocks, TRACE_BLOCK, 0, s>>>(a);
    else if (any_hit)
        k_trace<true, false><<<(unsigned)blocks, TRACE_BLOCK, 0, s>>>(a);
    else if (count)
        k_trace<false, true><<<(unsigned)blocks, TRACE_BLOCK, 0, s>>>(a);
    else
        k_trace<false, false><<<(unsigned)blocks, TRACE_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace hcc
