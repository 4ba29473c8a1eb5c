// Closest-hit / any-hit tracing: stack-based traversal of the BVH2 (Sec. 3.1)
// with the Moller-Trumbore ray/triangle test (1997).  GB300 has no
// ray-tracing cores, so traversal is software: one thread per ray, each
// internal node holding both children's boxes (32-byte 8-bit quantised
// layout, or 64-byte exact FP32 layout), a per-thread stack of
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

constexpr uint32_t REF_NONE = 0xFFFFFFFFu;  // no node (empty stack, no postponed leaf)

// Both children's boxes of an internal node, decoded for the slab test.
struct ChildBoxes {
    float lo0x, lo0y, lo0z, hi0x, hi0y, hi0z, lo1x, lo1y, lo1z, hi1x, hi1y, hi1z;
    uint32_t ref0, ref1;
};

// 32-byte quantised node: bounds are origin + q * 2^E rounded outward.
__device__ __forceinline__ void fetch_quant8(const uint4 *nodes, uint32_t ref, ChildBoxes &c) {
    const uint4 A = __ldg(nodes + 2 * (size_t)ref);
    const uint4 B = __ldg(nodes + 2 * (size_t)ref + 1);
    const float ox = __uint_as_float(A.x & 0xFFFFFF00u);
    const float oy = __uint_as_float(A.y & 0xFFFFFF00u);
    const float oz = __uint_as_float(A.z & 0xFFFFFF00u);
    const float sx = __uint_as_float((A.x & 0xFFu) << 23);
    const float sy = __uint_as_float((A.y & 0xFFu) << 23);
    const float sz = __uint_as_float((A.z & 0xFFu) << 23);
    c.lo0x = __fmaf_rd(byte_to_float(A.w, SEL0), sx, ox);
    c.lo0y = __fmaf_rd(byte_to_float(A.w, SEL1), sy, oy);
    c.lo0z = __fmaf_rd(byte_to_float(A.w, SEL2), sz, oz);
    c.hi0x = __fmaf_ru(byte_to_float(A.w, SEL3), sx, ox);
    c.hi0y = __fmaf_ru(byte_to_float(B.x, SEL0), sy, oy);
    c.hi0z = __fmaf_ru(byte_to_float(B.x, SEL1), sz, oz);
    c.lo1x = __fmaf_rd(byte_to_float(B.x, SEL2), sx, ox);
    c.lo1y = __fmaf_rd(byte_to_float(B.x, SEL3), sy, oy);
    c.lo1z = __fmaf_rd(byte_to_float(B.y, SEL0), sz, oz);
    c.hi1x = __fmaf_ru(byte_to_float(B.y, SEL1), sx, ox);
    c.hi1y = __fmaf_ru(byte_to_float(B.y, SEL2), sy, oy);
    c.hi1z = __fmaf_ru(byte_to_float(B.y, SEL3), sz, oz);
    c.ref0 = B.z;
    c.ref1 = B.w;
}

// 64-byte exact node: the children's FP32 boxes as stored in the input BVH.
__device__ __forceinline__ void fetch_exact(const uint4 *nodes, uint32_t ref, ChildBoxes &c) {
    const float4 *f = reinterpret_cast<const float4 *>(nodes) + 4 * (size_t)ref;
    const float4 n0 = __ldg(f), n1 = __ldg(f + 1), n2 = __ldg(f + 2);
    const uint4 n3 = __ldg(nodes + 4 * (size_t)ref + 3);
    c.lo0x = n0.x;
    c.lo0y = n0.y;
    c.lo0z = n0.z;
    c.hi0x = n0.w;
    c.hi0y = n1.x;
    c.hi0z = n1.y;
    c.lo1x = n1.z;
    c.lo1y = n1.w;
    c.lo1z = n2.x;
    c.hi1x = n2.y;
    c.hi1y = n2.z;
    c.hi1z = n2.w;
    c.ref0 = n3.x;
    c.ref1 = n3.y;
}

// Diagnostic counters of one ray (the COUNT variants only).
struct Counters {
    uint32_t nodes = 0, tris = 0, warp_nodes = 0, warp_leaves = 0;
};

// Traversal loop ("while-while" with postponed leaves, Aila & Laine 2009):
// a lane that reaches a leaf parks it and keeps descending until every lane
// of the warp holds a leaf, so triangle tests run with full warps; the
// nearer child is visited first and the farther one is pushed with its
// entry distance, which lets a pop skip subtrees beyond the best hit.
// Returns the hit record {prim, t, u, v} (prim -1 and t = +inf on a miss);
// sets overflow if the ray needed more than STACK entries.
template <bool ANY, bool COUNT, int LAYOUT>
__device__ __forceinline__ int4 trace_ray(const uint4 *__restrict__ nodes, const float4 *__restrict__ tris,
                                          uint32_t root_ref, const float4 o4, const float4 d4, Counters &cn,
                                          bool &overflow) {
    const uint32_t lane = threadIdx.x & 31;
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
    overflow = false;
    // next pending subtree that can still hold a closer hit, or REF_NONE
    auto pop = [&]() -> uint32_t {
        while (sp > 0) {
            --sp;
            if (st_t[sp] <= tcap) return st_ref[sp];
        }
        return REF_NONE;
    };
    uint32_t node = root_ref, leaf = REF_NONE;
    if (node & REF_LEAF) {
        leaf = node;
        node = REF_NONE;
    }
    while (node != REF_NONE || leaf != REF_NONE) {
        // internal nodes: descend until every lane has a leaf parked
        while (node != REF_NONE && !(node & REF_LEAF)) {
            ChildBoxes c;
            if (LAYOUT == 0)
                fetch_quant8(nodes, node, c);
            else
                fetch_exact(nodes, node, c);
            if (COUNT) {
                ++cn.nodes;  // this lane's node visit; the lowest active lane counts the warp's step
                if (lane == (uint32_t)(__ffs(__activemask()) - 1)) ++cn.warp_nodes;
            }
            float tn0, tf0, tn1, tf1;
            slab(r, c.lo0x, c.lo0y, c.lo0z, c.hi0x, c.hi0y, c.hi0z, tcap, tn0, tf0);
            slab(r, c.lo1x, c.lo1y, c.lo1z, c.hi1x, c.hi1y, c.hi1z, tcap, tn1, tf1);
            const bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
            if (h0 && h1) {
                const bool first0 = tn0 <= tn1;
                if (sp == STACK) {
                    overflow = true;
                    node = leaf = REF_NONE;
                    break;
                }
                st_ref[sp] = first0 ? c.ref1 : c.ref0;
                st_t[sp] = first0 ? tn1 : tn0;
                ++sp;
                node = first0 ? c.ref0 : c.ref1;
            } else if (h0) {
                node = c.ref0;
            } else if (h1) {
                node = c.ref1;
            } else {
                node = pop();
            }
            if (node != REF_NONE && (node & REF_LEAF) && leaf == REF_NONE) {
                leaf = node;
                node = pop();
            }
            if (__all_sync(__activemask(), leaf != REF_NONE)) break;
        }
        // leaves: the parked one, then any leaf that is next on the stack
        while (leaf != REF_NONE) {
            if (COUNT && lane == (uint32_t)(__ffs(__activemask()) - 1)) ++cn.warp_leaves;
            const uint32_t first = leaf & REF_TRI_MASK, cnt = ((leaf >> 29) & 3u) + 1u;
            bool hit_any = false;
            for (uint32_t k = 0; k < cnt; ++k) {
                const float4 *rec = tris + 3 * (size_t)(first + k);
                const float4 A = __ldg(rec), E1 = __ldg(rec + 1), E2 = __ldg(rec + 2);
                if (COUNT) ++cn.tris;
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
                hit_any = true;
                if (ANY) break;
            }
            if (ANY && hit_any) {
                node = leaf = REF_NONE;
                break;
            }
            leaf = REF_NONE;
            if (node != REF_NONE && (node & REF_LEAF)) {
                leaf = node;
                node = pop();
            }
        }
    }
    if (overflow) best_prim = -1;
    int4 out;
    out.x = best_prim;
    out.y = __float_as_int(best_prim < 0 ? __int_as_float(0x7F800000) : best_t);
    out.z = __float_as_int(best_prim < 0 ? 0.0f : best_u);
    out.w = __float_as_int(best_prim < 0 ? 0.0f : best_v);
    return out;
}

// One thread per ray slot i: the ray is org/dir[gather[i]] (or i), its record
// goes to hits[scatter[i]] (or i).  MULTI: the ray's BVH is that of its scene
// in a batch (a.scenes, ray ranges a.offsets).  COUNT = true is a diagnostic
// variant that also adds up work counters into a.counts (never timed).
template <bool ANY, bool COUNT, int LAYOUT, bool MULTI>
__global__ void __launch_bounds__(TRACE_BLOCK) k_trace(TraceArgs a) {
    const uint64_t i = (uint64_t)blockIdx.x * TRACE_BLOCK + threadIdx.x;
    if (i >= a.n) return;
    uint64_t src = i;
    if (a.gather) {
        src = a.gather[i];
        if (src >= a.n) {  // invalid permutation entry: report, never read out of bounds
            atomicOr(a.err, ERR_INDEX);
            return;
        }
    }
    const float4 o4 = __ldcs(a.org + src), d4 = __ldcs(a.dir + src);
    const uint4 *nodes = a.nodes;
    const float4 *tris = a.tris;
    uint32_t root = a.root_ref;
    if (MULTI) {
        const SceneDesc &sc = a.scenes[scene_of(a.offsets, a.num_scenes, src)];
        nodes = sc.nodes;
        tris = sc.tris;
        root = sc.root_ref;
    }
    Counters cn;
    bool overflow;
    const int4 out = trace_ray<ANY, COUNT, LAYOUT>(nodes, tris, root, o4, d4, cn, overflow);
    if (overflow) atomicOr(a.err, ERR_STACK);
    const uint64_t dst = a.scatter ? (uint64_t)a.scatter[i] : i;
    if (dst < a.n)
        __stcs(a.hits + dst, out);
    else  // invalid scatter entry: report, never write out of bounds
        atomicOr(a.err, ERR_INDEX);
    if (COUNT) {
        atomicAdd(a.counts, (unsigned long long)cn.nodes);
        atomicAdd(a.counts + 1, (unsigned long long)cn.tris);
        if (cn.warp_nodes) atomicAdd(a.counts + 2, (unsigned long long)cn.warp_nodes);
        if (cn.warp_leaves) atomicAdd(a.counts + 3, (unsigned long long)cn.warp_leaves);
    }
}

}  // namespace

cudaError_t launch_trace(cudaStream_t s, const TraceArgs &a, int any_hit) {
    if (a.n == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((a.n + TRACE_BLOCK - 1) / TRACE_BLOCK);
    const bool count = a.counts != nullptr, multi = a.scenes != nullptr;
#define HCC_TRACE_LAUNCH(ANY, CNT)                                                  \
    do {                                                                            \
        if (multi) {                                                                \
            if (a.layout == 0)                                                      \
                k_trace<ANY, CNT, 0, true><<<blocks, TRACE_BLOCK, 0, s>>>(a);       \
            else                                                                    \
                k_trace<ANY, CNT, 1, true><<<blocks, TRACE_BLOCK, 0, s>>>(a);       \
        } else {                                                                    \
            if (a.layout == 0)                                                      \
                k_trace<ANY, CNT, 0, false><<<blocks, TRACE_BLOCK, 0, s>>>(a);      \
            else                                                                    \
                k_trace<ANY, CNT, 1, false><<<blocks, TRACE_BLOCK, 0, s>>>(a);      \
        }                                                                           \
    } while (0)
    if (any_hit && count)
        HCC_TRACE_LAUNCH(true, true);
    else if (any_hit)
        HCC_TRACE_LAUNCH(true, false);
    else if (count)
        HCC_TRACE_LAUNCH(false, true);
    else
        HCC_TRACE_LAUNCH(false, false);
#undef HCC_TRACE_LAUNCH
    return cudaGetLastError();
}

}  // namespace hcc
