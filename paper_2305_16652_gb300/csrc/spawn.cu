// Next bounce of a batch of wavefronts: every ray that hit a triangle spawns
// one diffuse ray from its hit point, cosine-weighted about the triangle's
// normal turned toward the incoming ray; a ray that missed becomes an empty
// ray (interval [1, 0]) that every later step skips at once.
//
// This is ray generation between bounces (the shading stage of a wavefront
// path tracer), not part of the reordering method.  Every operation is an
// explicit round-to-nearest step (library built with --fmad=false) and the
// random numbers come from a counter-based generator, so the rays are a
// fixed function of (seed, ray index, hit) that a CPU restatement reproduces
// bit for bit:
//   u_j      = top 24 bits of mix(mix(seed) ^ (64 i + j)) * 2^-24
//              (mix = SplitMix64 finaliser)
//   disk     = first (x, y) = (2 u_2a - 1, 2 u_2a+1 - 1), a = 0..15, with
//              fma(y, y, x x) <= 1 (else (0, 0)); z = sqrt(max(0, 1 - r2))
//   normal   = cross(e1, e2) / |cross(e1, e2)|, flipped if dot(n, d) > 0
//   basis    = Duff et al. 2017, "Building an Orthonormal Basis, Revisited"
//   origin   = o + t d (one fma per axis), direction = x b1 + y b2 + z n
#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int SPAWN_BLOCK = 256;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float uniform24(uint64_t seed_mixed, uint64_t i, uint32_t j) {
    const uint64_t z = mix64(seed_mixed ^ (i * 64u + j));
    return __fmul_rn((float)(uint32_t)(z >> 40), 5.9604644775390625e-08f);  // 2^-24, exact
}

__global__ void __launch_bounds__(SPAWN_BLOCK) k_spawn(const float4 *__restrict__ in_org,
                                                       const float4 *__restrict__ in_dir, uint32_t in_rs,
                                                       const int4 *__restrict__ hits, uint64_t n,
                                                       const SceneDesc *__restrict__ scenes,
                                                       const uint64_t *__restrict__ offsets, uint32_t num_scenes,
                                                       uint64_t seed, float tmin, float4 *__restrict__ out_org,
                                                       float4 *__restrict__ out_dir, uint32_t out_rs, uint32_t *err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t sm = mix64(seed);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = in_org[i * in_rs], d = in_dir[i * in_rs];
        const int4 h = hits[i];
        const int32_t prim = h.x;
        const SceneDesc &sc = scenes[scene_of(offsets, num_scenes, i)];
        if (prim >= 0 && (uint32_t)prim >= sc.num_tris) {  // not a triangle of this scene
            atomicOr(err, ERR_INDEX);
        }
        if (prim < 0 || (uint32_t)prim >= sc.num_tris) {  // miss: an empty ray
            out_org[i * out_rs] = make_float4(o.x, o.y, o.z, 1.0f);
            out_dir[i * out_rs] = make_float4(d.x, d.y, d.z, 0.0f);
            continue;
        }
        const uint32_t rec = __ldg(sc.prim_rec + prim);
        const float4 e1 = __ldg(sc.tris + 3 * (size_t)rec + 1), e2 = __ldg(sc.tris + 3 * (size_t)rec + 2);
        const float t = __int_as_float(h.y);
        const float px = __fmaf_rn(t, d.x, o.x), py = __fmaf_rn(t, d.y, o.y), pz = __fmaf_rn(t, d.z, o.z);
        // geometric normal, unit length, facing the incoming ray
        float nx = __fmaf_rn(e1.y, e2.z, -__fmul_rn(e1.z, e2.y));
        float ny = __fmaf_rn(e1.z, e2.x, -__fmul_rn(e1.x, e2.z));
        float nz = __fmaf_rn(e1.x, e2.y, -__fmul_rn(e1.y, e2.x));
        const float len = __fsqrt_rn(__fmaf_rn(nz, nz, __fmaf_rn(ny, ny, __fmul_rn(nx, nx))));
        if (len > 0.0f) {
            nx = __fdiv_rn(nx, len);
            ny = __fdiv_rn(ny, len);
            nz = __fdiv_rn(nz, len);
        } else {
            nx = 0.0f;
            ny = 0.0f;
            nz = 1.0f;
        }
        if (__fmaf_rn(nz, d.z, __fmaf_rn(ny, d.y, __fmul_rn(nx, d.x))) > 0.0f) {
            nx = -nx;
            ny = -ny;
            nz = -nz;
        }
        // cosine-weighted direction: uniform point of the unit disk by rejection
        float x = 0.0f, y = 0.0f, r2 = 0.0f;
        for (uint32_t a = 0; a < 16; ++a) {
            const float cx = __fsub_rn(__fmul_rn(2.0f, uniform24(sm, i, 2 * a)), 1.0f);
            const float cy = __fsub_rn(__fmul_rn(2.0f, uniform24(sm, i, 2 * a + 1)), 1.0f);
            const float c2 = __fmaf_rn(cy, cy, __fmul_rn(cx, cx));
            if (c2 <= 1.0f) {
                x = cx;
                y = cy;
                r2 = c2;
                break;
            }
        }
        const float z = __fsqrt_rn(fmaxf(0.0f, __fsub_rn(1.0f, r2)));
        // orthonormal basis about n (Duff et al. 2017)
        const float sign = copysignf(1.0f, nz);
        const float aa = __fdiv_rn(-1.0f, __fadd_rn(sign, nz));
        const float bb = __fmul_rn(__fmul_rn(nx, ny), aa);
        const float b1x = __fadd_rn(1.0f, __fmul_rn(__fmul_rn(__fmul_rn(sign, nx), nx), aa));
        const float b1y = __fmul_rn(sign, bb);
        const float b1z = -__fmul_rn(sign, nx);
        const float b2x = bb;
        const float b2y = __fadd_rn(sign, __fmul_rn(__fmul_rn(ny, ny), aa));
        const float b2z = -ny;
        const float wx = __fmaf_rn(z, nx, __fmaf_rn(y, b2x, __fmul_rn(x, b1x)));
        const float wy = __fmaf_rn(z, ny, __fmaf_rn(y, b2y, __fmul_rn(x, b1y)));
        const float wz = __fmaf_rn(z, nz, __fmaf_rn(y, b2z, __fmul_rn(x, b1z)));
        out_org[i * out_rs] = make_float4(px, py, pz, tmin);
        out_dir[i * out_rs] = make_float4(wx, wy, wz, __int_as_float(0x7F800000));
    }
}

}  // namespace

cudaError_t launch_spawn(cudaStream_t s, const float4 *in_org, const float4 *in_dir, uint32_t in_rs, const int4 *hits,
                         uint64_t n, const SceneDesc *scenes, const uint64_t *offsets, uint32_t num_scenes,
                         uint64_t seed, float tmin, float4 *out_org, float4 *out_dir, uint32_t out_rs, uint32_t *err) {
    if (n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (n + SPAWN_BLOCK - 1) / SPAWN_BLOCK;
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    k_spawn<<<(unsigned)blocks, SPAWN_BLOCK, 0, s>>>(in_org, in_dir, in_rs, hits, n, scenes, offsets, num_scenes, seed,
                                                     tmin, out_org, out_dir, out_rs, err);
    return cudaGetLastError();
}

}  // namespace hcc
