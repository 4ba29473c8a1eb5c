// Internal declarations of the hcc library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hcc.h"

namespace hcc {

// Bits of the per-context device error word.
constexpr uint32_t ERR_STACK = 1u;
constexpr uint32_t ERR_TIMEOUT = 2u;
constexpr uint32_t ERR_INDEX = 4u;  // a permutation entry was out of range (access skipped)

// ----------------------------------------------------------------- BVH layout
//
// One internal BVH2 node = 32 bytes = two uint4 (w0..w7):
//   w0..w2  node origin x/y/z: a float whose low 8 mantissa bits are cleared
//           (rounded toward -inf), with the biased exponent E+127 of the
//           quantisation step 2^E of that axis stored in those 8 bits
//   w3      child0 lo.x lo.y lo.z hi.x   (one byte each, low byte first)
//   w4      child0 hi.y hi.z, child1 lo.x lo.y
//   w5      child1 lo.z hi.x hi.y hi.z
//   w6, w7  child references
// A decoded bound is origin + q * 2^E, computed with outward rounding, so the
// decoded box always contains the child's exact box.
// Child reference: bit 31 set = leaf, bits 29..30 = triangle count - 1,
// bits 0..28 = first triangle record; bit 31 clear = internal node index.
constexpr uint32_t REF_LEAF = 0x80000000u;
constexpr uint32_t REF_TRI_MASK = 0x1FFFFFFFu;

// Exact layout: one internal node = 64 bytes = four uint4: the children's
// FP32 boxes as pairs c0.lo.xy c0.hi.xy | c0.lo.z c0.hi.z c1.lo.xy |
// c1.hi.xy c1.lo.z c1.hi.z | ref0 ref1 0 0.
// Wide layout: one 4-ary node = 128 bytes = eight float4 rows, one entry per
// child: lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, references, zeros; an unused
// child has ref 0xFFFFFFFF.  An internal reference indexes wide nodes.

// Triangle record = three float4: (v0.xyz, id bits), (e1.xyz, 0), (e2.xyz, 0)
// with e1 = v1 - v0, e2 = v2 - v0 rounded to float.

// One scene of a batch of wavefronts (device table, read by the fused
// multi-scene kernels): its BVH, its cut (HCC), its key normalisation box and
// the rays [begin, end) of the batch that belong to it.
struct SceneDesc {
    const uint4 *nodes;
    const float4 *tris;
    const float4 *cut;  // (lo, hi) pairs in key order
    const uint32_t *prim_rec;  // triangle id -> triangle record
    uint32_t root_ref;
    uint32_t used;      // cut nodes that drive key bits
    float lo[3], ext[3], L;
    uint32_t num_tris;
    uint32_t cut_ordered;  // every cut box has lo <= hi on every axis
};

// Scene of ray src in a batch: the last s with offsets[s] <= src.
__device__ __forceinline__ uint32_t scene_of(const uint64_t *__restrict__ offsets, uint32_t num_scenes, uint64_t src) {
    uint32_t lo = 0, hi = num_scenes;  // offsets[lo] <= src < offsets[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(offsets + mid) <= src)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Three-input max / min (sm_100+ PTX): like nested fmaxf / fminf, NaN inputs
// are ignored and the result is one of the inputs, so a slab test written
// with them gives the same comparisons in one instruction fewer.
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------------------ launchers
// All return the launch error (cudaSuccess when queued).

cudaError_t launch_encode_hcc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                              const float4 *cut_boxes, uint32_t used, uint32_t key_bits, void *keys);

cudaError_t launch_encode_twopoint(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                   const float lo[3], const float ext[3], float L, uint32_t key_bits, void *keys);

cudaError_t launch_encode_origin(cudaStream_t s, const float4 *org, uint64_t n, uint32_t rs, const float lo[3], const float ext[3],
                                 uint32_t key_bits, void *keys);

cudaError_t launch_encode_origin_dir(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                     const float lo[3], const float ext[3], uint32_t key_bits, void *keys);

// Multi-level HCC: ntop top boxes (at most top_field), ntop * low_field low
// boxes (row r = top node r), (lo, hi) float4 pairs.
cudaError_t launch_encode_mlhcc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                const float4 *top, uint32_t ntop, uint32_t top_field, const float4 *low,
                                uint32_t low_field, uint32_t key_bits, void *keys);

// Prefix path code over the exact-layout nodes; root box given separately.
cudaError_t launch_encode_ppc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs, const uint4 *nodes,
                              uint32_t root_ref, const float root_lo[3], const float root_hi[3], uint32_t key_bits,
                              void *keys);

// Batch of scenes: key of ray i = (scene << key_bits) | its key in its scene.
cudaError_t launch_encode_multi(cudaStream_t s, int method, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                const SceneDesc *scenes, const uint64_t *offsets, uint32_t num_scenes,
                                uint32_t key_bits, uint32_t total_bits, void *keys);

// Next bounce of a batch: diffuse rays from the hit points (see spawn.cu).
cudaError_t launch_spawn(cudaStream_t s, const float4 *in_org, const float4 *in_dir, uint32_t in_rs, const int4 *hits,
                         uint64_t n, const SceneDesc *scenes, const uint64_t *offsets, uint32_t num_scenes,
                         uint64_t seed, float tmin, float4 *out_org, float4 *out_dir, uint32_t out_rs, uint32_t *err);

// cnt[0] += key changes between consecutive sorted positions, cnt[1] += those
// inside groups of 32 positions (cnt zeroed by the caller).
cudaError_t launch_key_stats(cudaStream_t s, const void *keys, uint32_t key_bits, const uint32_t *perm, uint64_t n,
                             unsigned long long *cnt);

// Radix sort scratch bytes for n keys of key_bits bits.
size_t sort_scratch_bytes(uint64_t n, uint32_t key_bits);

// Bounded-wait settings of one sort.
struct SortOptions {
    uint32_t wait_limit = 1u << 22;        // status reads a tile may wait in the look-back before giving up
    uint32_t withhold_tile = 0xFFFFFFFFu;  // test hook: this tile never publishes its counts (none by default)
};

cudaError_t launch_sort(cudaStream_t s, const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm,
                        void *scratch, uint32_t *err_word, const SortOptions &opt = SortOptions());

// Ray i of a stream pair is org[i * rs], dir[i * rs] (rs: the stride in
// float4 units; 1 = two packed float4 arrays, 2 with dir = org + 1 = 32-byte
// records).
cudaError_t launch_gather(cudaStream_t s, const float4 *in_org, const float4 *in_dir, uint32_t in_rs, uint64_t in_n,
                          const uint32_t *perm, float4 *out_org, float4 *out_dir, uint32_t out_rs, uint64_t n,
                          uint32_t *err);

struct TraceArgs {
    const uint4 *nodes = nullptr;  // 2 (quantised), 4 (exact) or 8 (wide) per node
    int layout = 0;          // 0 = 32-byte quantised, 1 = 64-byte exact, 2 = 128-byte wide
    const float4 *tris = nullptr;  // 3 per triangle
    uint32_t root_ref = 0;
    const float4 *org = nullptr;
    const float4 *dir = nullptr;
    uint32_t rs = 1;     // ray i is org/dir[i * rs]
    bool rec = false;    // 32-byte records (rs 2, dir = org + 1, 32-byte aligned): one load per ray
    uint64_t n = 0;
    const uint32_t *gather = nullptr;   // ray j is read from org/dir[gather[j]] (NULL = j)
    const uint32_t *scatter = nullptr;  // its hit goes to hits[scatter[j]] (NULL = j)
    int4 *hits = nullptr;
    uint32_t *err = nullptr;
    unsigned long long *counts = nullptr;  // diagnostic (NULL = off): node visits, triangle tests,
                                 // warp node steps, warp leaf steps
    const SceneDesc *scenes = nullptr;     // batch mode (NULL = single BVH above)
    const uint64_t *offsets = nullptr;     // scene s owns rays [offsets[s], offsets[s+1])
    uint32_t num_scenes = 0;
    unsigned long long *work = nullptr;    // slot counter of the persistent trace (NULL: one thread per slot)
    int block = 128;                       // closest-hit persistent trace: threads per block ...
    int stack = HCC_TRACE_STACK;           // ... and stack entries per ray (a supported shape)
};

cudaError_t launch_trace(cudaStream_t s, const TraceArgs &a, int any_hit);
// The block sizes and stack depths of the closest-hit persistent trace: 64,
// 128 or 256 threads with 32, 48 or 64 stack entries.
bool trace_shape_supported(uint32_t block, uint32_t stack);

}  // namespace hcc
