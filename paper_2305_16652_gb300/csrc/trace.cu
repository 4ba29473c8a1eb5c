// Closest-hit / any-hit tracing: stack-based traversal of the BVH2 (Sec. 3.1)
// with the Moller-Trumbore ray/triangle test (1997).  GB300 has no
// ray-tracing cores, so traversal is software: one thread per ray, each
// internal node holding its children's boxes (32-byte 8-bit quantised
// layout or 64-byte exact FP32 layout of the BVH2, or 128-byte 4-ary nodes
// collapsed from it), a per-thread stack of (node, entry distance) pairs.
//
// Robustness: decoded child boxes are rounded outward (they contain the exact
// boxes), the far slab distance is widened by 1 + 2*gamma(3) to cover the
// rounding of the distances (Ize 2013, "Robust BVH Ray Traversal"; the wide
// nodes' directed-rounding distances leave only the reciprocal's rounding
// to cover), and a subtree is dropped only when its entry
// distance exceeds the best hit by more than 2^-16 relative, so traversal
// never loses a triangle that the closest-hit definition would pick.
// Triangle arithmetic is the canonical Moller-Trumbore sequence with explicit
// round-to-nearest intrinsics (built with --fmad=false), so the (t, u, v) of
// a triangle are the same bit patterns on every run and in every ray order.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int TRACE_BLOCK = 128;
constexpr int STACK = HCC_TRACE_STACK;
// 1 + 2 * gamma(3), gamma(n) = n u / (1 - n u), u = 2^-24
constexpr float ROBUST_FAR = 1.0000003576279f;
constexpr float PRUNE_SLACK = 1.0f + 1.0f / 65536.0f;
// idle lanes that make a warp take new rays: in input order, and in sorted
// order (rays fetched through a permutation), where waiting longer keeps the
// warp's neighbouring rays together (measured faster for each)
constexpr uint32_t REFILL_MIN = 12;
// resident threads per SM the persistent kernel is built for: binary nodes
// (48 registers at 128-thread blocks), and wide nodes or a batch of scenes
// (56); the register cap follows from threads x registers <= 64K
constexpr int POOL_THREADS = 1280;
constexpr int POOL_THREADS_WIDE = 1152;
constexpr uint32_t REFILL_MIN_SORTED = 24;

__device__ __forceinline__ float byte_to_float(uint32_t w, uint32_t sel) {
    // 0x4B0000bb as float is 2^23 + bb exactly
    return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, sel)), 8388608.0f);
}
// selectors for byte 0..3 of w combined with bytes of 0x4B000000
constexpr uint32_t SEL0 = 0x7540u, SEL1 = 0x7541u, SEL2 = 0x7542u, SEL3 = 0x7543u;

// The origin is kept negated and paired, (-ox, -oy) and (-oz, -oz), with the
// reciprocal direction paired alike, so one packed add and one packed
// multiply give two slab distances (lo - o) * inv.
struct Ray {
    float2 nxy, nzz, ixy, izz;
    float tmin, dx, dy, dz, tmax;
    float lx, ly, lz, ux, uy, uz;  // o * (1/d) rounded down and up, per axis
};

__device__ __forceinline__ float safe_inv(float d) {
    // a zero (or denormal) direction component is replaced by +-1e-30 for the
    // slab test only; this keeps every slab distance a number (no 0 * inf)
    return __frcp_rn(fabsf(d) > 1e-30f ? d : copysignf(1e-30f, d));
}

// A child box as pairs: (lo.x, lo.y), (hi.x, hi.y), (lo.z, hi.z).
struct Box2 {
    float2 lxy, hxy, zz;
};

// Entry / exit distance of the ray through one decoded child box of a
// binary node: t = (bound - o) * inv with round-to-nearest, two axes per
// packed add and multiply ((bound + (-o)) * inv, the same results as one at
// a time), near and far by min/max per axis.  Its three roundings make it a
// relative-error estimate, which the far distance widened by 1 + 2*gamma(3)
// covers.
__device__ __forceinline__ void slab(const Ray &r, const Box2 &b, float tcap, float &tn, float &tf) {
    const float2 a = __fmul2_rn(__fadd2_rn(b.lxy, r.nxy), r.ixy);
    const float2 c = __fmul2_rn(__fadd2_rn(b.hxy, r.nxy), r.ixy);
    const float2 z = __fmul2_rn(__fadd2_rn(b.zz, r.nzz), r.izz);
    tn = fmax3(fminf(a.x, c.x), fminf(a.y, c.y), fmaxf(fminf(z.x, z.y), r.tmin));
    const float f = fmin3(fmaxf(a.x, c.x), fmaxf(a.y, c.y), fmaxf(z.x, z.y));
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
    const float sx = __fsub_rn(-r.nxy.x, A.x), sy = __fsub_rn(-r.nxy.y, A.y), sz = __fsub_rn(-r.nzz.x, A.z);
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
    Box2 b0, b1;
    uint32_t ref0, ref1;
};

// One 32-byte read-only load (sm_100+ 256-bit vector load); p must be 32-byte aligned.
__device__ __forceinline__ void ldg256(const void *p, uint4 &a, uint4 &b) {
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
        : "l"(p));
}

__device__ __forceinline__ float2 f2(uint32_t a, uint32_t b) { return make_float2(__uint_as_float(a), __uint_as_float(b)); }

// 32-byte quantised node: bounds are origin + q * 2^E rounded outward.
__device__ __forceinline__ void fetch_quant8(const uint4 *nodes, uint32_t ref, ChildBoxes &c) {
    uint4 A, B;
    ldg256(nodes + 2 * (size_t)ref, A, B);
    const float ox = __uint_as_float(A.x & 0xFFFFFF00u);
    const float oy = __uint_as_float(A.y & 0xFFFFFF00u);
    const float oz = __uint_as_float(A.z & 0xFFFFFF00u);
    const float sx = __uint_as_float((A.x & 0xFFu) << 23);
    const float sy = __uint_as_float((A.y & 0xFFu) << 23);
    const float sz = __uint_as_float((A.z & 0xFFu) << 23);
    c.b0.lxy = make_float2(__fmaf_rd(byte_to_float(A.w, SEL0), sx, ox), __fmaf_rd(byte_to_float(A.w, SEL1), sy, oy));
    c.b0.zz.x = __fmaf_rd(byte_to_float(A.w, SEL2), sz, oz);
    c.b0.hxy = make_float2(__fmaf_ru(byte_to_float(A.w, SEL3), sx, ox), __fmaf_ru(byte_to_float(B.x, SEL0), sy, oy));
    c.b0.zz.y = __fmaf_ru(byte_to_float(B.x, SEL1), sz, oz);
    c.b1.lxy = make_float2(__fmaf_rd(byte_to_float(B.x, SEL2), sx, ox), __fmaf_rd(byte_to_float(B.x, SEL3), sy, oy));
    c.b1.zz.x = __fmaf_rd(byte_to_float(B.y, SEL0), sz, oz);
    c.b1.hxy = make_float2(__fmaf_ru(byte_to_float(B.y, SEL1), sx, ox), __fmaf_ru(byte_to_float(B.y, SEL2), sy, oy));
    c.b1.zz.y = __fmaf_ru(byte_to_float(B.y, SEL3), sz, oz);
    c.ref0 = B.z;
    c.ref1 = B.w;
}

// 64-byte exact node: per child (lo.x, lo.y), (hi.x, hi.y), (lo.z, hi.z) as
// stored in the input BVH, then the two references.
__device__ __forceinline__ void fetch_exact(const uint4 *nodes, uint32_t ref, ChildBoxes &c) {
    uint4 w0, w1, w2, n3;
    ldg256(nodes + 4 * (size_t)ref, w0, w1);
    ldg256(nodes + 4 * (size_t)ref + 2, w2, n3);
    c.b0.lxy = f2(w0.x, w0.y);
    c.b0.hxy = f2(w0.z, w0.w);
    c.b0.zz = f2(w1.x, w1.y);
    c.b1.lxy = f2(w1.z, w1.w);
    c.b1.hxy = f2(w2.x, w2.y);
    c.b1.zz = f2(w2.z, w2.w);
    c.ref0 = n3.x;
    c.ref1 = n3.y;
}

// Child c of a 128-byte wide node (rows of four floats: lo.x hi.x lo.y
// hi.y lo.z hi.z, then the four references) given the ray's near and far
// rows (boxes are stored with lo <= hi, so the near plane of an axis is lo
// for a positive reciprocal direction and hi for a negative one).  Directed
// slab test: the near distance (near - o) * inv is bounded from below by one
// fma rounded down against o * inv rounded up, the far one from above by
// one fma rounded up against o * inv rounded down, so the only error left
// is the relative one of the rounded reciprocal, which the widened far
// distance covers.  t is the child's entry distance if the ray meets it
// (clamped to the largest float, so +inf marks only unused and missed
// slots), else +inf.
__device__ __forceinline__ float wide_child(const Ray &r, float nx, float ny, float nz, float fx, float fy, float fz,
                                            uint32_t ref, float tcap) {
    const float ix = r.ixy.x, iy = r.ixy.y, iz = r.izz.x;
    const float tn = fmax3(__fmaf_rd(nx, ix, -r.ux), __fmaf_rd(ny, iy, -r.uy), fmaxf(__fmaf_rd(nz, iz, -r.uz), r.tmin));
    const float f = fmin3(__fmaf_ru(fx, ix, -r.lx), __fmaf_ru(fy, iy, -r.ly), __fmaf_ru(fz, iz, -r.lz));
    const float tf = fminf(__fmul_rn(f, ROBUST_FAR), tcap);
    return (tn <= tf && ref != 0xFFFFFFFFu) ? fminf(tn, 3.40282347e38f) : __int_as_float(0x7F800000);
}

// Orders two (distance, reference) pairs by distance.
__device__ __forceinline__ void order2(float &ta, uint32_t &ra, float &tb, uint32_t &rb) {
    const bool sw = tb < ta;
    const float t = ta;
    const uint32_t x = ra;
    ta = sw ? tb : ta;
    ra = sw ? rb : ra;
    tb = sw ? t : tb;
    rb = sw ? x : rb;
}

// Diagnostic counters of one ray (the COUNT variants only).
struct Counters {
    uint32_t nodes = 0, tris = 0, warp_nodes = 0, warp_leaves = 0;
};

// Traversal state of one ray: the ray, the best hit so far, the node being
// descended and the parked leaf.  The stack lives beside it in the kernel.
struct RayState {
    Ray r;
    float best_t, best_u, best_v, tcap;  // tcap: best_t widened by the prune slack
    int32_t best_prim;
    int sp;
    uint32_t node, leaf;
    bool overflow;
};

__device__ __forceinline__ void ray_init(RayState &s, const float4 o4, const float4 d4, uint32_t root_ref) {
    s.r.nxy = make_float2(-o4.x, -o4.y);
    s.r.nzz = make_float2(-o4.z, -o4.z);
    s.r.tmin = o4.w;
    s.r.dx = d4.x;
    s.r.dy = d4.y;
    s.r.dz = d4.z;
    s.r.tmax = d4.w;
    const float ix = safe_inv(d4.x), iy = safe_inv(d4.y), iz = safe_inv(d4.z);
    s.r.ixy = make_float2(ix, iy);
    s.r.izz = make_float2(iz, iz);
    s.r.lx = __fmul_rd(o4.x, ix);
    s.r.ly = __fmul_rd(o4.y, iy);
    s.r.lz = __fmul_rd(o4.z, iz);
    s.r.ux = __fmul_ru(o4.x, ix);
    s.r.uy = __fmul_ru(o4.y, iy);
    s.r.uz = __fmul_ru(o4.z, iz);
    s.best_t = s.r.tmax;
    s.best_u = s.best_v = 0.0f;
    s.best_prim = -1;
    s.tcap = s.r.tmax;
    s.sp = 0;
    s.overflow = false;
    s.node = root_ref;
    s.leaf = REF_NONE;
    if (s.node & REF_LEAF) {
        s.leaf = s.node;
        s.node = REF_NONE;
    }
}

__device__ __forceinline__ bool ray_done(const RayState &s) { return s.node == REF_NONE && s.leaf == REF_NONE; }

// Pending subtrees are (node reference, entry distance) entries of a
// STACKN-entry array in local memory, one 8-byte access each.
template <int STACKN>
__device__ __forceinline__ bool ray_push(RayState &s, uint2 *stack, uint2 e) {  // false: no room
    if (s.sp >= STACKN) return false;
    stack[s.sp++] = e;
    return true;
}

// Next pending subtree that can still hold a closer hit, or REF_NONE.
__device__ __forceinline__ uint32_t ray_pop(RayState &s, const uint2 *stack) {
    while (s.sp > 0) {
        const uint2 e = stack[--s.sp];
        if (__uint_as_float(e.y) <= s.tcap) return e.x;
    }
    return REF_NONE;
}

// The node loop of a closest-hit round ends once all but LEAF_SLACK of the
// warp's lanes still descending hold a parked leaf.  Waiting for every lane
// (the plain postponed-leaf rule) kept the others idle behind the last few
// descents: on the room's 16.6M rays a slack of 3 or 4 traced 4.6 %
// (unsorted) and 2 % (HCC order) faster than 0, 6 and 8 slower than 3.
// The leaf loop of a closest-hit round goes on to the next leaf on the stack
// while at least LEAF_MIN lanes have one (4 measured best of 0, 4, 8 and 12:
// 0.6 % faster than chaining leaves while any lane has one).  Any-hit traces
// keep the plain rules (every lane; chain while any lane has a leaf), which
// measured 1-2 % faster for them.
constexpr int LEAF_SLACK = 3;
constexpr int LEAF_MIN = 4;
template <bool ANY>
__device__ __forceinline__ bool leaves_ready(const RayState &s) {
    if (ANY) return __all_sync(__activemask(), s.leaf != REF_NONE);
    const uint32_t active = __activemask();
    const uint32_t parked = __ballot_sync(active, s.leaf != REF_NONE);
    return __popc(parked) + LEAF_SLACK >= __popc(active);
}

// One round of the traversal loop ("while-while" with postponed leaves,
// Aila & Laine 2009): descend internal nodes until (nearly) every lane of
// the warp holds a leaf (a lane that reaches a leaf parks it and keeps
// descending), then test the parked leaf and any leaf that is next on the
// stack; a lane without a leaf yet resumes its descent in the next round.  The
// nearer child is visited first and the farther one is pushed with its
// entry distance, which lets a pop skip subtrees beyond the best hit.
template <bool ANY, bool COUNT, int LAYOUT, int STACKN>
__device__ __forceinline__ void ray_round(RayState &s, uint2 *stack, const uint4 *__restrict__ nodes,
                                          const float4 *__restrict__ tris, Counters &cn) {
    const uint32_t lane = threadIdx.x & 31;
    // wide nodes: the met children sorted by entry distance (a five-exchange
    // network on four pairs), the nearest descended, the others pushed
    // farthest first
    while (LAYOUT == 2 && s.node != REF_NONE && !(s.node & REF_LEAF)) {
        const float4 *nd = reinterpret_cast<const float4 *>(nodes) + 8 * (size_t)s.node;
        if (COUNT) {
            ++cn.nodes;
            if (lane == (uint32_t)(__ffs(__activemask()) - 1)) ++cn.warp_nodes;
        }
        // the near row of an axis is lo for a positive reciprocal direction
        const uint32_t sx = s.r.ixy.x < 0.0f, sy = s.r.ixy.y < 0.0f, sz = s.r.izz.x < 0.0f;
        const float4 nx = __ldg(nd + sx), fx = __ldg(nd + 1 - sx);
        const float4 ny = __ldg(nd + 2 + sy), fy = __ldg(nd + 3 - sy);
        const float4 nz = __ldg(nd + 4 + sz), fz = __ldg(nd + 5 - sz);
        const uint4 rf = __ldg(reinterpret_cast<const uint4 *>(nd + 6));
        uint32_t r0 = rf.x, r1 = rf.y, r2 = rf.z, r3 = rf.w;
        float t0 = wide_child(s.r, nx.x, ny.x, nz.x, fx.x, fy.x, fz.x, r0, s.tcap);
        float t1 = wide_child(s.r, nx.y, ny.y, nz.y, fx.y, fy.y, fz.y, r1, s.tcap);
        float t2 = wide_child(s.r, nx.z, ny.z, nz.z, fx.z, fy.z, fz.z, r2, s.tcap);
        float t3 = wide_child(s.r, nx.w, ny.w, nz.w, fx.w, fy.w, fz.w, r3, s.tcap);
        order2(t0, r0, t1, r1);
        order2(t2, r2, t3, r3);
        order2(t0, r0, t2, r2);
        order2(t1, r1, t3, r3);
        order2(t1, r1, t2, r2);
        const float INF = __int_as_float(0x7F800000);
        const int met = (t0 < INF) + (t1 < INF) + (t2 < INF) + (t3 < INF);
        if (met == 0) {
            s.node = ray_pop(s, stack);
        } else {
            if (s.sp + met - 1 > STACKN) {
                s.overflow = true;
                s.node = s.leaf = REF_NONE;
                break;
            }
            if (met > 3) ray_push<STACKN>(s, stack, make_uint2(r3, __float_as_uint(t3)));
            if (met > 2) ray_push<STACKN>(s, stack, make_uint2(r2, __float_as_uint(t2)));
            if (met > 1) ray_push<STACKN>(s, stack, make_uint2(r1, __float_as_uint(t1)));
            s.node = r0;
        }
        if (s.node != REF_NONE && (s.node & REF_LEAF) && s.leaf == REF_NONE) {
            s.leaf = s.node;
            s.node = ray_pop(s, stack);
        }
        if (leaves_ready<ANY>(s)) break;
    }
    // internal nodes: descend until (nearly) every lane has a leaf parked
    while (LAYOUT != 2 && s.node != REF_NONE && !(s.node & REF_LEAF)) {
        ChildBoxes c;
        if (LAYOUT == 0)
            fetch_quant8(nodes, s.node, c);
        else
            fetch_exact(nodes, s.node, c);
        if (COUNT) {
            ++cn.nodes;  // this lane's node visit; the lowest active lane counts the warp's step
            if (lane == (uint32_t)(__ffs(__activemask()) - 1)) ++cn.warp_nodes;
        }
        float tn0, tf0, tn1, tf1;
        slab(s.r, c.b0, s.tcap, tn0, tf0);
        slab(s.r, c.b1, s.tcap, tn1, tf1);
        const bool h0 = tn0 <= tf0, h1 = tn1 <= tf1;
        if (h0 && h1) {
            const bool first0 = tn0 <= tn1;
            if (!ray_push<STACKN>(s, stack, make_uint2(first0 ? c.ref1 : c.ref0, __float_as_uint(first0 ? tn1 : tn0)))) {
                s.overflow = true;
                s.node = s.leaf = REF_NONE;
                break;
            }
            s.node = first0 ? c.ref0 : c.ref1;
        } else if (h0) {
            s.node = c.ref0;
        } else if (h1) {
            s.node = c.ref1;
        } else {
            s.node = ray_pop(s, stack);
        }
        if (s.node != REF_NONE && (s.node & REF_LEAF) && s.leaf == REF_NONE) {
            s.leaf = s.node;
            s.node = ray_pop(s, stack);
        }
        if (leaves_ready<ANY>(s)) break;
    }
    // leaves: the parked one, then any leaf that is next on the stack
    while (s.leaf != REF_NONE) {
        if (COUNT && lane == (uint32_t)(__ffs(__activemask()) - 1)) ++cn.warp_leaves;
        const uint32_t first = s.leaf & REF_TRI_MASK, cnt = ((s.leaf >> 29) & 3u) + 1u;
        bool hit_any = false;
        for (uint32_t k = 0; k < cnt; ++k) {
            const float4 *rec = tris + 3 * (size_t)(first + k);
            const float4 A = __ldg(rec), E1 = __ldg(rec + 1), E2 = __ldg(rec + 2);
            if (COUNT) ++cn.tris;
            float t, u, v;
            if (!intersect(s.r, A, E1, E2, t, u, v)) continue;
            const int32_t prim = __float_as_int(A.w);
            if (s.best_prim < 0 || t < s.best_t || (t == s.best_t && prim < s.best_prim)) {
                s.best_t = t;
                s.best_u = u;
                s.best_v = v;
                s.best_prim = prim;
                s.tcap = __fmul_rn(t, PRUNE_SLACK);
            }
            hit_any = true;
            if (ANY) break;
        }
        if (ANY && hit_any) {
            s.node = s.leaf = REF_NONE;
            break;
        }
        s.leaf = REF_NONE;
        if (s.node != REF_NONE && (s.node & REF_LEAF)) {
            s.leaf = s.node;
            s.node = ray_pop(s, stack);
        }
        // fewer than LEAF_MIN lanes with a next leaf: keep it parked for
        // the next round rather than hold the warp here for them
        if (!ANY && __popc(__ballot_sync(__activemask(), s.leaf != REF_NONE)) < LEAF_MIN) break;
    }
}

// The hit record {prim, t, u, v} (prim -1 and t = +inf on a miss or a
// stack overflow).
__device__ __forceinline__ int4 ray_result(const RayState &s) {
    const bool miss = s.overflow || s.best_prim < 0;
    int4 out;
    out.x = miss ? -1 : s.best_prim;
    out.y = __float_as_int(miss ? __int_as_float(0x7F800000) : s.best_t);
    out.z = __float_as_int(miss ? 0.0f : s.best_u);
    out.w = __float_as_int(miss ? 0.0f : s.best_v);
    return out;
}

template <bool COUNT>
__device__ __forceinline__ void add_counts(const TraceArgs &a, const Counters &cn) {
    if (COUNT) {
        if (cn.nodes) atomicAdd(a.counts, (unsigned long long)cn.nodes);
        if (cn.tris) atomicAdd(a.counts + 1, (unsigned long long)cn.tris);
        if (cn.warp_nodes) atomicAdd(a.counts + 2, (unsigned long long)cn.warp_nodes);
        if (cn.warp_leaves) atomicAdd(a.counts + 3, (unsigned long long)cn.warp_leaves);
    }
}

// Reads ray slot i: the ray is org/dir[gather[i]] (or i).  Returns false
// (and reports) for an out-of-range permutation entry.
template <bool MULTI>
__device__ __forceinline__ bool fetch_ray(const TraceArgs &a, uint64_t i, float4 &o4, float4 &d4,
                                          const uint4 *&nodes, const float4 *&tris, uint32_t &root) {
    uint64_t src = i;
    if (a.gather) {
        src = a.gather[i];
        if (src >= a.n) {  // invalid permutation entry: report, never read out of bounds
            atomicOr(a.err, ERR_INDEX);
            return false;
        }
    }
    if (a.rec) {  // one 32-byte record: a single access per ray
        asm volatile("ld.global.cs.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                     : "=f"(o4.x), "=f"(o4.y), "=f"(o4.z), "=f"(o4.w), "=f"(d4.x), "=f"(d4.y), "=f"(d4.z), "=f"(d4.w)
                     : "l"(a.org + 2 * src));
    } else {
        o4 = __ldcs(a.org + src * a.rs);
        d4 = __ldcs(a.dir + src * a.rs);
    }
    nodes = a.nodes;
    tris = a.tris;
    root = a.root_ref;
    if (MULTI) {
        const SceneDesc &sc = a.scenes[scene_of(a.offsets, a.num_scenes, src)];
        nodes = sc.nodes;
        tris = sc.tris;
        root = sc.root_ref;
    }
    return true;
}

// Writes the record of ray slot i to hits[scatter[i]] (or i).
__device__ __forceinline__ void store_hit(const TraceArgs &a, uint64_t i, const RayState &s) {
    if (i >= a.n) {  // not a ray slot: report, never index the permutation out of bounds
        atomicOr(a.err, ERR_INDEX);
        return;
    }
    if (s.overflow) atomicOr(a.err, ERR_STACK);
    const uint64_t dst = a.scatter ? (uint64_t)a.scatter[i] : i;
    if (dst < a.n)
        __stcs(a.hits + dst, ray_result(s));
    else  // invalid scatter entry: report, never write out of bounds
        atomicOr(a.err, ERR_INDEX);
}

// One thread per ray slot.  MULTI: the ray's BVH is that of its scene in a
// batch (a.scenes, ray ranges a.offsets).  COUNT = true is a diagnostic
// variant that also adds up work counters into a.counts (never timed).
template <bool ANY, bool COUNT, int LAYOUT, bool MULTI>
__global__ void __launch_bounds__(TRACE_BLOCK) k_trace(TraceArgs a) {
    uint64_t i = (uint64_t)blockIdx.x * TRACE_BLOCK + threadIdx.x;
    if (i >= a.n) return;
    if (a.gather || a.scatter) i = a.n - 1 - i;  // sorted order from its end (blocks start in index order)
    float4 o4, d4;
    const uint4 *nodes;
    const float4 *tris;
    uint32_t root;
    if (!fetch_ray<MULTI>(a, i, o4, d4, nodes, tris, root)) return;
    RayState s;
    uint2 stack[STACK];
    Counters cn;
    ray_init(s, o4, d4, root);
    while (!ray_done(s)) ray_round<ANY, COUNT, LAYOUT, STACK>(s, stack, nodes, tris, cn);
    store_hit(a, i, s);
    add_counts<COUNT>(a, cn);
}

// Persistent variant with ray replacement (Aila & Laine 2009, "replacing
// terminated rays"): each warp takes ray slots from a global counter, runs
// traversal rounds, and after each round the lanes whose ray has finished
// take new slots (all at once, one atomic per warp) as soon as refill_min of
// them are idle or none is busy.  Slots are handed out in counter order,
// so lanes of a warp trace neighbouring slots -- in sorted order, rays with
// equal keys.  Every ray's record is the same as in k_trace: a ray's own
// traversal does not depend on which rays share its warp, except for which
// of several hits an any-hit query returns first.  A trace in sorted order
// (rays fetched through a permutation, or already gathered and their hits
// written back through one) hands out its slots from the end of
// the order, largest keys first: in HCC order those are the rays whose keys
// set the most cut nodes and the longest traversals (the room's 16.6M rays:
// 54.8 node visits per ray in the last tenth of the order, 15.8 in the
// first), and starting them first leaves short rays for the end of the
// launch, where warps run out of work (its HCC trace: 4.08 ms against 4.19
// in ascending order).
// BLOCK threads per block and STACKN stack entries per ray are a shape the
// autotuner may pick.
template <bool ANY, bool COUNT, int LAYOUT, bool MULTI, int BLOCK, int STACKN>
__global__ void __launch_bounds__(BLOCK, ((LAYOUT == 2 || MULTI) ? POOL_THREADS_WIDE : POOL_THREADS) / BLOCK)
    k_trace_pool(TraceArgs a) {
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    RayState s;
    uint2 stack[STACKN];
    Counters cn;
    const uint4 *nodes = a.nodes;
    const float4 *tris = a.tris;
    uint64_t slot = 0;
    bool have = false, exhausted = false;
    const uint32_t refill_min = a.gather ? REFILL_MIN_SORTED : REFILL_MIN;
    for (;;) {
        const bool want = !have && !exhausted;
        const uint32_t need = __ballot_sync(FULL, want);
        const uint32_t busy = __ballot_sync(FULL, have);
        if (need && (busy == 0 || (uint32_t)__popc(need) >= refill_min)) {
            const int leader = __ffs(need) - 1;
            unsigned long long base = 0;
            if ((int)lane == leader) base = atomicAdd(a.work, (unsigned long long)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (want) {
                slot = base + __popc(need & lt);
                if ((a.gather || a.scatter) && slot < a.n) slot = a.n - 1 - slot;  // sorted order from its end
                if (slot < a.n) {
                    float4 o4, d4;
                    uint32_t root;
                    if (fetch_ray<MULTI>(a, slot, o4, d4, nodes, tris, root)) {
                        ray_init(s, o4, d4, root);
                        have = true;
                    }
                } else {
                    exhausted = true;
                }
            }
        }
        if (!__any_sync(FULL, have)) {
            if (__all_sync(FULL, exhausted)) break;
            continue;
        }
        if (have) {
            ray_round<ANY, COUNT, LAYOUT, STACKN>(s, stack, nodes, tris, cn);
            if (ray_done(s)) {
                store_hit(a, slot, s);
                have = false;
            }
        }
    }
    add_counts<COUNT>(a, cn);
}

}  // namespace

namespace {

// Resident blocks per SM of one persistent kernel on the current device
// (queried once per device and kernel).
int resident_blocks(const void *kernel, int block) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, const void *>, int>> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &e : cache)
        if (e.first.first == dev && e.first.second == kernel) return e.second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm <= 0) {
        cudaGetLastError();
        per_sm = 1;
    }
    cache.push_back({{dev, kernel}, per_sm});
    return per_sm;
}

// Persistent grid: every block resident at once.
template <bool ANY, bool CNT, int LAYOUT, bool MULTI, int BLOCK, int STACKN>
cudaError_t launch_pool(cudaStream_t s, const TraceArgs &a) {
    const auto kernel = k_trace_pool<ANY, CNT, LAYOUT, MULTI, BLOCK, STACKN>;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned cap = (unsigned)std::max(1, sms) * (unsigned)resident_blocks((const void *)kernel, BLOCK);
    const unsigned blocks = (unsigned)std::min<uint64_t>((a.n + BLOCK - 1) / BLOCK, cap);
    cudaError_t e = cudaMemsetAsync(a.work, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    kernel<<<blocks, BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

// The closest-hit persistent trace in the shape the context asks for; the
// any-hit and counting variants keep the default shape.
template <bool ANY, bool CNT, int LAYOUT, bool MULTI>
cudaError_t launch_pool_shaped(cudaStream_t s, const TraceArgs &a) {
    if constexpr (ANY || CNT) {
        return launch_pool<ANY, CNT, LAYOUT, MULTI, TRACE_BLOCK, STACK>(s, a);
    } else {
        switch (a.block * 1000 + a.stack) {
            case 64032: return launch_pool<ANY, CNT, LAYOUT, MULTI, 64, 32>(s, a);
            case 64048: return launch_pool<ANY, CNT, LAYOUT, MULTI, 64, 48>(s, a);
            case 64064: return launch_pool<ANY, CNT, LAYOUT, MULTI, 64, 64>(s, a);
            case 128032: return launch_pool<ANY, CNT, LAYOUT, MULTI, 128, 32>(s, a);
            case 128048: return launch_pool<ANY, CNT, LAYOUT, MULTI, 128, 48>(s, a);
            case 256032: return launch_pool<ANY, CNT, LAYOUT, MULTI, 256, 32>(s, a);
            case 256048: return launch_pool<ANY, CNT, LAYOUT, MULTI, 256, 48>(s, a);
            case 256064: return launch_pool<ANY, CNT, LAYOUT, MULTI, 256, 64>(s, a);
            default: return launch_pool<ANY, CNT, LAYOUT, MULTI, TRACE_BLOCK, STACK>(s, a);
        }
    }
}

template <bool ANY, bool CNT, bool MULTI>
cudaError_t launch_layout(cudaStream_t s, const TraceArgs &a, bool pool) {
    if (pool) {
        if (a.layout == 0) return launch_pool_shaped<ANY, CNT, 0, MULTI>(s, a);
        if (a.layout == 1) return launch_pool_shaped<ANY, CNT, 1, MULTI>(s, a);
        return launch_pool_shaped<ANY, CNT, 2, MULTI>(s, a);
    }
    const unsigned blocks = (unsigned)((a.n + TRACE_BLOCK - 1) / TRACE_BLOCK);
    if (a.layout == 0)
        k_trace<ANY, CNT, 0, MULTI><<<blocks, TRACE_BLOCK, 0, s>>>(a);
    else if (a.layout == 1)
        k_trace<ANY, CNT, 1, MULTI><<<blocks, TRACE_BLOCK, 0, s>>>(a);
    else
        k_trace<ANY, CNT, 2, MULTI><<<blocks, TRACE_BLOCK, 0, s>>>(a);
    return cudaGetLastError();
}

template <bool ANY, bool CNT>
cudaError_t launch_multi(cudaStream_t s, const TraceArgs &a, bool pool) {
    return a.scenes ? launch_layout<ANY, CNT, true>(s, a, pool) : launch_layout<ANY, CNT, false>(s, a, pool);
}

}  // namespace

bool trace_shape_supported(uint32_t block, uint32_t stack) {
    const uint32_t shapes[][2] = {{64, 32}, {64, 48}, {64, 64}, {128, 32}, {128, 48}, {128, 64},
                                  {256, 32}, {256, 48}, {256, 64}};
    for (const auto &sh : shapes)
        if (sh[0] == block && sh[1] == stack) return true;
    return false;
}

cudaError_t launch_trace(cudaStream_t s, const TraceArgs &a, int any_hit) {
    if (a.n == 0) return cudaSuccess;
    const bool count = a.counts != nullptr, pool = a.work != nullptr;
    if (any_hit && count) return launch_multi<true, true>(s, a, pool);
    if (any_hit) return launch_multi<true, false>(s, a, pool);
    if (count) return launch_multi<false, true>(s, a, pool);
    return launch_multi<false, false>(s, a, pool);
}

}  // namespace hcc
