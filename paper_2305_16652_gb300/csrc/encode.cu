// Key encoding kernels: hierarchy cut code (Algorithm 1, Sec. 4.2.1), its
// multi-level form (Sec. 4.3), the prefix path code (Sec. 4.1) and the
// TwoPoint, Origin and Origin-Direction baselines (Sec. 3.2, Sec. 5).
//
// Floating point: every rounding step is an explicit round-to-nearest
// intrinsic (scalar, or Blackwell's packed FP32x2 add and multiply, which
// round each half the same way) and the library is built with
// --fmad=false, so each key is the same bit pattern the arithmetic defines,
// whatever the compiler schedules.
#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int ENC_BLOCK = 256;
constexpr uint32_t MAX_CUT_BITS = 64;

int encode_grid(uint64_t n, int block, int per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    uint64_t want = (n + block - 1) / block;
    uint64_t cap = (uint64_t)sms * per_sm;
    return (int)(want < cap ? (want ? want : 1) : cap);
}

// Slab test of one ray against one box: t = (bound - o) * (1/d) per axis,
// tnear = max over axes and tmin, tfar = min over axes and tmax, met when
// tnear <= tfar (fminf/fmaxf ignore the NaN of 0 * inf).
__device__ __forceinline__ bool meets(const float4 &o, const float4 &d, float ix, float iy, float iz, const float4 &lo,
                                      const float4 &hi) {
    const float ax = __fmul_rn(__fsub_rn(lo.x, o.x), ix), bx = __fmul_rn(__fsub_rn(hi.x, o.x), ix);
    const float ay = __fmul_rn(__fsub_rn(lo.y, o.y), iy), by = __fmul_rn(__fsub_rn(hi.y, o.y), iy);
    const float az = __fmul_rn(__fsub_rn(lo.z, o.z), iz), bz = __fmul_rn(__fsub_rn(hi.z, o.z), iz);
    const float tnear = fmax3(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), o.w));
    const float tfar = fmin3(fmaxf(ax, bx), fmaxf(ay, by), fminf(fmaxf(az, bz), d.w));
    return tnear <= tfar;
}

// Algorithm 1: the cut nodes are staged in shared memory once per block
// (line 1); every ray is tested against every cut node and each result sets
// one key bit.  Cut node r drives bit (key_bits - 1 - r).
//
// For a ray whose three reciprocal direction components are finite and a cut
// whose boxes all have lo <= hi, the per-axis min / max of the slab test is
// known from the sign of the reciprocal: with inv > 0, (lo - o) * inv <=
// (hi - o) * inv (rounding is monotonic), and the order flips for inv < 0.
// Those rays read the (near, far) bounds of each axis as one pair by a
// per-lane index and take both distances with one packed add and one packed
// multiply instead of computing both and taking min and max -- the same
// comparisons with six fewer min/max operations per node and half the
// arithmetic instructions.  Other rays (a zero or denormal
// direction component, where 0 * inf makes a NaN that fminf / fmaxf skip) take
// the general test.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_hcc(const float4 *__restrict__ org,
                                                          const float4 *__restrict__ dir, uint64_t n, uint32_t rs,
                                                          const float4 *__restrict__ cut, uint32_t used,
                                                          uint32_t key_bits, K *__restrict__ keys) {
    __shared__ float4 s_lo[MAX_CUT_BITS], s_hi[MAX_CUT_BITS];
    // per node and axis the two orders of its bounds, (lo, hi) and (hi, lo):
    // a ray reads (near, far) of an axis as one pair, by its direction sign
    __shared__ float2 s_p[MAX_CUT_BITS * 6];
    bool ordered = true;
    for (uint32_t r = threadIdx.x; r < used; r += blockDim.x) {
        const float4 lo = cut[2 * r], hi = cut[2 * r + 1];
        s_lo[r] = lo;
        s_hi[r] = hi;
        float2 *b = s_p + 6 * r;
        b[0] = make_float2(lo.x, hi.x);
        b[1] = make_float2(hi.x, lo.x);
        b[2] = make_float2(lo.y, hi.y);
        b[3] = make_float2(hi.y, lo.y);
        b[4] = make_float2(lo.z, hi.z);
        b[5] = make_float2(hi.z, lo.z);
        ordered = ordered && lo.x <= hi.x && lo.y <= hi.y && lo.z <= hi.z;
    }
    ordered = __syncthreads_and(ordered);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i * rs);
        const float4 d = __ldcs(dir + i * rs);
        const float ix = __frcp_rn(d.x), iy = __frcp_rn(d.y), iz = __frcp_rn(d.z);
        K key = 0;
        if (ordered && isfinite(ix) && isfinite(iy) && isfinite(iz)) {
            // (bound + (-o)) * inv for the near and far bound of an axis in one
            // packed add and one packed multiply: the same round-to-nearest
            // results as (bound - o) * inv one at a time
            const float2 *px = s_p + (ix < 0.0f), *py = s_p + 2 + (iy < 0.0f), *pz = s_p + 4 + (iz < 0.0f);
            const float2 nox = make_float2(-o.x, -o.x), noy = make_float2(-o.y, -o.y), noz = make_float2(-o.z, -o.z);
            const float2 ixx = make_float2(ix, ix), iyy = make_float2(iy, iy), izz = make_float2(iz, iz);
#pragma unroll 8
            for (uint32_t r = 0; r < used; ++r) {
                const float2 tx = __fmul2_rn(__fadd2_rn(px[6 * r], nox), ixx);
                const float2 ty = __fmul2_rn(__fadd2_rn(py[6 * r], noy), iyy);
                const float2 tz = __fmul2_rn(__fadd2_rn(pz[6 * r], noz), izz);
                const float tnear = fmax3(tx.x, ty.x, fmaxf(tz.x, o.w));
                const float tfar = fmin3(tx.y, ty.y, fminf(tz.y, d.w));
                key = (key << 1) | (K)(tnear <= tfar);
            }
        } else {
            for (uint32_t r = 0; r < used; ++r) key = (key << 1) | (K)meets(o, d, ix, iy, iz, s_lo[r], s_hi[r]);
        }
        if (used && key_bits > used) key <<= (key_bits - used);  // node r drives bit key_bits - 1 - r
        __stcs(keys + i, key);
    }
}

// TwoPoint: o and t = o + L d (one fused multiply-add per axis) normalised
// to the scene box, quantised to b bits, Morton-interleaved most significant
// level first in the order o.x o.y o.z t.x t.y t.z, left-justified in k bits.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_twopoint(const float4 *__restrict__ org,
                                                               const float4 *__restrict__ dir, uint64_t n, uint32_t rs,
                                                               float lox, float loy, float loz, float ex, float ey,
                                                               float ez, float L, uint32_t key_bits,
                                                               K *__restrict__ keys) {
    const uint32_t b = key_bits / 6;
    const float levels = (float)(1u << b);  // exact power of two (b <= 10)
    const uint32_t qmax = b ? ((1u << b) - 1u) : 0u;
    const uint32_t pad = key_bits - 6 * b;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i * rs);
        const float4 d = __ldcs(dir + i * rs);
        const float p[6] = {o.x, o.y, o.z, __fmaf_rn(L, d.x, o.x), __fmaf_rn(L, d.y, o.y), __fmaf_rn(L, d.z, o.z)};
        const float lo[3] = {lox, loy, loz}, ext[3] = {ex, ey, ez};
        uint32_t q[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const int a = c % 3;
            float u = (ext[a] == 0.0f) ? 0.0f : __fdiv_rn(__fsub_rn(p[c], lo[a]), ext[a]);
            u = fminf(fmaxf(u, 0.0f), 1.0f);
            const uint32_t qi = __float2uint_rz(__fmul_rn(u, levels));
            q[c] = qi < qmax ? qi : qmax;
        }
        K key = 0;
        for (int j = (int)b - 1; j >= 0; --j) {
#pragma unroll
            for (int c = 0; c < 6; ++c) key = (key << 1) | (K)((q[c] >> j) & 1u);
        }
        if (pad) key <<= pad;
        __stcs(keys + i, key);
    }
}

// Normalise p to the box [lo, lo + ext], clamp to [0, 1], quantise to b bits.
__device__ __forceinline__ uint32_t quantise(float p, float lo, float ext, uint32_t b) {
    if (b == 0) return 0u;
    float u = (ext == 0.0f) ? 0.0f : __fdiv_rn(__fsub_rn(p, lo), ext);
    u = fminf(fmaxf(u, 0.0f), 1.0f);
    const uint32_t q = __float2uint_rz(__fmul_rn(u, (float)(1u << b)));
    const uint32_t qmax = (1u << b) - 1u;
    return q < qmax ? q : qmax;
}

// Morton interleave, most significant level first, coordinates in order.
template <typename K, int M>
__device__ __forceinline__ K interleave(const uint32_t (&q)[M], uint32_t b) {
    K key = 0;
    for (int j = (int)b - 1; j >= 0; --j) {
#pragma unroll
        for (int c = 0; c < M; ++c) key = (key << 1) | (K)((q[c] >> j) & 1u);
    }
    return key;
}

// Octahedral map of a direction: L1-normalise, fold the lower hemisphere
// (z < 0) over the diagonals, map [-1, 1]^2 to [0, 1]^2; zero -> centre.
__device__ __forceinline__ void octahedral(const float4 &d, float &u, float &v) {
    u = 0.5f;
    v = 0.5f;
    const float s = __fadd_rn(__fadd_rn(fabsf(d.x), fabsf(d.y)), fabsf(d.z));
    if (s > 0.0f) {
        const float nx = __fdiv_rn(d.x, s), ny = __fdiv_rn(d.y, s), nz = __fdiv_rn(d.z, s);
        float x = nx, y = ny;
        if (nz < 0.0f) {
            x = __fmul_rn(__fsub_rn(1.0f, fabsf(ny)), nx >= 0.0f ? 1.0f : -1.0f);
            y = __fmul_rn(__fsub_rn(1.0f, fabsf(nx)), ny >= 0.0f ? 1.0f : -1.0f);
        }
        u = __fadd_rn(__fmul_rn(x, 0.5f), 0.5f);
        v = __fadd_rn(__fmul_rn(y, 0.5f), 0.5f);
    }
}

// Origin key: 3D Morton code of the origin, floor(k/3) bits per axis,
// left-justified in k bits.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_origin(const float4 *__restrict__ org, uint64_t n, uint32_t rs, float lox,
                                                             float loy, float loz, float ex, float ey, float ez,
                                                             uint32_t key_bits, K *__restrict__ keys) {
    const uint32_t b = key_bits / 3, pad = key_bits - 3 * b;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i * rs);
        const uint32_t q[3] = {quantise(o.x, lox, ex, b), quantise(o.y, loy, ey, b), quantise(o.z, loz, ez, b)};
        K key = interleave<K, 3>(q, b);
        if (pad) key <<= pad;
        __stcs(keys + i, key);
    }
}

// Origin-Direction key: origin Morton code (bo bits per axis) above a Morton
// code of the octahedral map of the direction (bd bits per coordinate),
// bd = floor(k/6), bo = floor((k - 2 bd)/3), left-justified in k bits.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_origin_dir(const float4 *__restrict__ org,
                                                                 const float4 *__restrict__ dir, uint64_t n, uint32_t rs,
                                                                 float lox, float loy, float loz, float ex,
                                                                 float ey, float ez, uint32_t key_bits,
                                                                 K *__restrict__ keys) {
    const uint32_t bd = key_bits / 6, bo = (key_bits - 2 * bd) / 3;
    const uint32_t pad = key_bits - (3 * bo + 2 * bd);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i * rs);
        const float4 d = __ldcs(dir + i * rs);
        float u, v;
        octahedral(d, u, v);
        const uint32_t qo[3] = {quantise(o.x, lox, ex, bo), quantise(o.y, loy, ey, bo), quantise(o.z, loz, ez, bo)};
        const uint32_t qd[2] = {quantise(u, 0.0f, 1.0f, bd), quantise(v, 0.0f, 1.0f, bd)};
        K key = (interleave<K, 3>(qo, bo) << (2 * bd)) | interleave<K, 2>(qd, bd);
        if (pad) key <<= pad;
        __stcs(keys + i, key);
    }
}

// Key statistics over keys in sorted order (keys[perm[j]] ascending):
// cnt[0] += changes of key between consecutive positions, cnt[1] += changes
// inside groups of 32 consecutive positions.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_key_stats(const K *__restrict__ keys, const uint32_t *__restrict__ perm,
                                                         uint64_t n, K mask, unsigned long long *cnt) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long all = 0, inner = 0;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; j < n; j += stride) {
        const uint32_t a = perm[j - 1], b = perm[j];
        if (a < n && b < n && ((keys[a] & mask) != (keys[b] & mask))) {
            ++all;
            if (j % 32 != 0) ++inner;
        }
    }
    if (all) atomicAdd(cnt, all);
    if (inner) atomicAdd(cnt + 1, inner);
}

// TwoPoint / Origin / Origin-Direction keys of one ray (the formulas of the
// single-scene kernels above, as functions of the scene box).
template <typename K>
__device__ __forceinline__ K twopoint_key(const float4 &o, const float4 &d, const SceneDesc &sc, uint32_t key_bits) {
    const uint32_t b = key_bits / 6, pad = key_bits - 6 * b;
    const float p[6] = {o.x, o.y, o.z, __fmaf_rn(sc.L, d.x, o.x), __fmaf_rn(sc.L, d.y, o.y),
                        __fmaf_rn(sc.L, d.z, o.z)};
    uint32_t q[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) q[c] = quantise(p[c], sc.lo[c % 3], sc.ext[c % 3], b);
    K key = interleave<K, 6>(q, b);
    return pad ? (K)(key << pad) : key;
}

template <typename K>
__device__ __forceinline__ K origin_key(const float4 &o, const SceneDesc &sc, uint32_t key_bits) {
    const uint32_t b = key_bits / 3, pad = key_bits - 3 * b;
    const uint32_t q[3] = {quantise(o.x, sc.lo[0], sc.ext[0], b), quantise(o.y, sc.lo[1], sc.ext[1], b),
                           quantise(o.z, sc.lo[2], sc.ext[2], b)};
    K key = interleave<K, 3>(q, b);
    return pad ? (K)(key << pad) : key;
}

template <typename K>
__device__ __forceinline__ K origin_dir_key(const float4 &o, const float4 &d, const SceneDesc &sc, uint32_t key_bits) {
    const uint32_t bd = key_bits / 6, bo = (key_bits - 2 * bd) / 3, pad = key_bits - (3 * bo + 2 * bd);
    float u, v;
    octahedral(d, u, v);
    const uint32_t qo[3] = {quantise(o.x, sc.lo[0], sc.ext[0], bo), quantise(o.y, sc.lo[1], sc.ext[1], bo),
                            quantise(o.z, sc.lo[2], sc.ext[2], bo)};
    const uint32_t qd[2] = {quantise(u, 0.0f, 1.0f, bd), quantise(v, 0.0f, 1.0f, bd)};
    K key = (interleave<K, 3>(qo, bo) << (2 * bd)) | interleave<K, 2>(qd, bd);
    return pad ? (K)(key << pad) : key;
}

// Batch of wavefronts: one launch encodes the rays of every scene against
// that scene's cut or box; the scene index sits above the key so that one
// sort groups rays by scene, then by key.
template <typename K, int METHOD>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_multi(const float4 *__restrict__ org,
                                                            const float4 *__restrict__ dir, uint64_t n, uint32_t rs,
                                                            const SceneDesc *__restrict__ scenes,
                                                            const uint64_t *__restrict__ offsets, uint32_t num_scenes,
                                                            uint32_t key_bits, K *__restrict__ keys) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t s = scene_of(offsets, num_scenes, i);
        const SceneDesc &sc = scenes[s];
        const float4 o = __ldcs(org + i * rs);
        const float4 d = __ldcs(dir + i * rs);
        K key = 0;
        if (METHOD == HCC_METHOD_HCC) {
            const float ix = __frcp_rn(d.x), iy = __frcp_rn(d.y), iz = __frcp_rn(d.z);
            K bit = (K)1 << (key_bits - 1);
            if (sc.cut_ordered && isfinite(ix) && isfinite(iy) && isfinite(iz)) {
                // (near, far) pairs selected by the direction signs and packed
                // arithmetic, as in k_encode_hcc
                const bool sx = ix < 0.0f, sy = iy < 0.0f, sz = iz < 0.0f;
                const float2 nox = make_float2(-o.x, -o.x), noy = make_float2(-o.y, -o.y), noz = make_float2(-o.z, -o.z);
                const float2 ixx = make_float2(ix, ix), iyy = make_float2(iy, iy), izz = make_float2(iz, iz);
                for (uint32_t r = 0; r < sc.used; ++r, bit >>= 1) {
                    const float4 lo = __ldg(sc.cut + 2 * r), hi = __ldg(sc.cut + 2 * r + 1);
                    const float2 px = sx ? make_float2(hi.x, lo.x) : make_float2(lo.x, hi.x);
                    const float2 py = sy ? make_float2(hi.y, lo.y) : make_float2(lo.y, hi.y);
                    const float2 pz = sz ? make_float2(hi.z, lo.z) : make_float2(lo.z, hi.z);
                    const float2 tx = __fmul2_rn(__fadd2_rn(px, nox), ixx);
                    const float2 ty = __fmul2_rn(__fadd2_rn(py, noy), iyy);
                    const float2 tz = __fmul2_rn(__fadd2_rn(pz, noz), izz);
                    if (fmax3(tx.x, ty.x, fmaxf(tz.x, o.w)) <= fmin3(tx.y, ty.y, fminf(tz.y, d.w))) key |= bit;
                }
            } else {
                for (uint32_t r = 0; r < sc.used; ++r, bit >>= 1)
                    if (meets(o, d, ix, iy, iz, __ldg(sc.cut + 2 * r), __ldg(sc.cut + 2 * r + 1))) key |= bit;
            }
        } else if (METHOD == HCC_METHOD_TWOPOINT) {
            key = twopoint_key<K>(o, d, sc, key_bits);
        } else if (METHOD == HCC_METHOD_ORIGIN) {
            key = origin_key<K>(o, sc, key_bits);
        } else {
            key = origin_dir_key<K>(o, d, sc, key_bits);
        }
        if (key_bits < 8 * sizeof(K)) key |= (K)s << key_bits;
        __stcs(keys + i, key);
    }
}

}  // namespace

cudaError_t launch_encode_multi(cudaStream_t s, int method, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                const SceneDesc *scenes, const uint64_t *offsets, uint32_t num_scenes,
                                uint32_t key_bits, uint32_t total_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
#define HCC_ENC_MULTI(K, M) \
    k_encode_multi<K, M><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, scenes, offsets, num_scenes, key_bits, (K *)keys)
#define HCC_ENC_MULTI_K(K)                                                      \
    do {                                                                        \
        if (method == HCC_METHOD_HCC)                                           \
            HCC_ENC_MULTI(K, HCC_METHOD_HCC);                                   \
        else if (method == HCC_METHOD_TWOPOINT)                                 \
            HCC_ENC_MULTI(K, HCC_METHOD_TWOPOINT);                              \
        else if (method == HCC_METHOD_ORIGIN)                                   \
            HCC_ENC_MULTI(K, HCC_METHOD_ORIGIN);                                \
        else                                                                    \
            HCC_ENC_MULTI(K, HCC_METHOD_ORIGIN_DIR);                            \
    } while (0)
    if (total_bits <= 32)
        HCC_ENC_MULTI_K(uint32_t);
    else
        HCC_ENC_MULTI_K(uint64_t);
#undef HCC_ENC_MULTI_K
#undef HCC_ENC_MULTI
    return cudaGetLastError();
}

cudaError_t launch_key_stats(cudaStream_t s, const void *keys, uint32_t key_bits, const uint32_t *perm, uint64_t n,
                             unsigned long long *cnt) {
    if (n < 2) return cudaSuccess;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32) {
        const uint32_t mask = key_bits == 32 ? 0xFFFFFFFFu : ((1u << key_bits) - 1u);
        k_key_stats<uint32_t><<<grid, ENC_BLOCK, 0, s>>>((const uint32_t *)keys, perm, n, mask, cnt);
    } else {
        const uint64_t mask = key_bits == 64 ? ~0ull : ((1ull << key_bits) - 1ull);
        k_key_stats<uint64_t><<<grid, ENC_BLOCK, 0, s>>>((const uint64_t *)keys, perm, n, mask, cnt);
    }
    return cudaGetLastError();
}

cudaError_t launch_encode_origin(cudaStream_t s, const float4 *org, uint64_t n, uint32_t rs, const float lo[3], const float ext[3],
                                 uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_origin<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, n, rs, lo[0], lo[1], lo[2], ext[0], ext[1], ext[2],
                                                             key_bits, (uint32_t *)keys);
    else
        k_encode_origin<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, n, rs, lo[0], lo[1], lo[2], ext[0], ext[1], ext[2],
                                                             key_bits, (uint64_t *)keys);
    return cudaGetLastError();
}

cudaError_t launch_encode_origin_dir(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                     const float lo[3], const float ext[3], uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_origin_dir<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, lo[0], lo[1], lo[2], ext[0], ext[1],
                                                                 ext[2], key_bits, (uint32_t *)keys);
    else
        k_encode_origin_dir<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, lo[0], lo[1], lo[2], ext[0], ext[1],
                                                                 ext[2], key_bits, (uint64_t *)keys);
    return cudaGetLastError();
}

namespace {

// Multi-level HCC (Sec. 4.3): the top field as in Algorithm 1; the first met
// top node (HAD order) is the representative, and its low-level cut fills the
// next low_field bits.  All boxes of both levels are staged in shared memory:
// top boxes first, then the low boxes row by row.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_mlhcc(const float4 *__restrict__ org,
                                                            const float4 *__restrict__ dir, uint64_t n, uint32_t rs,
                                                            const float4 *__restrict__ top, uint32_t ntop,
                                                            uint32_t top_field, const float4 *__restrict__ low,
                                                            uint32_t low_field, uint32_t key_bits,
                                                            K *__restrict__ keys) {
    // per box and axis the two orders of its bounds, (lo, hi) and (hi, lo),
    // as in k_encode_hcc; top boxes, then the low rows
    extern __shared__ float2 s_pair[];
    const uint32_t nbox = ntop + ntop * low_field;
    bool ordered = true;
    for (uint32_t q = threadIdx.x; q < nbox; q += blockDim.x) {
        const float4 lo = q < ntop ? top[2 * q] : low[2 * (q - ntop)];
        const float4 hi = q < ntop ? top[2 * q + 1] : low[2 * (q - ntop) + 1];
        float2 *b = s_pair + 6 * q;
        b[0] = make_float2(lo.x, hi.x);
        b[1] = make_float2(hi.x, lo.x);
        b[2] = make_float2(lo.y, hi.y);
        b[3] = make_float2(hi.y, lo.y);
        b[4] = make_float2(lo.z, hi.z);
        b[5] = make_float2(hi.z, lo.z);
        ordered = ordered && lo.x <= hi.x && lo.y <= hi.y && lo.z <= hi.z;
    }
    ordered = __syncthreads_and(ordered);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i * rs);
        const float4 d = __ldcs(dir + i * rs);
        const float ix = __frcp_rn(d.x), iy = __frcp_rn(d.y), iz = __frcp_rn(d.z);
        // the slab test of box q: (near, far) pairs selected by the direction
        // signs and packed arithmetic when that is exact (see k_encode_hcc),
        // the general test otherwise
        const bool fast = ordered && isfinite(ix) && isfinite(iy) && isfinite(iz);
        const uint32_t sx = ix < 0.0f, sy = 2u + (iy < 0.0f), sz = 4u + (iz < 0.0f);
        const float2 nox = make_float2(-o.x, -o.x), noy = make_float2(-o.y, -o.y), noz = make_float2(-o.z, -o.z);
        const float2 ixx = make_float2(ix, ix), iyy = make_float2(iy, iy), izz = make_float2(iz, iz);
        auto hit = [&](uint32_t q) {
            const float2 *b = s_pair + 6 * q;
            if (fast) {
                const float2 tx = __fmul2_rn(__fadd2_rn(b[sx], nox), ixx);
                const float2 ty = __fmul2_rn(__fadd2_rn(b[sy], noy), iyy);
                const float2 tz = __fmul2_rn(__fadd2_rn(b[sz], noz), izz);
                return fmax3(tx.x, ty.x, fmaxf(tz.x, o.w)) <= fmin3(tx.y, ty.y, fminf(tz.y, d.w));
            }
            return meets(o, d, ix, iy, iz, make_float4(b[0].x, b[2].x, b[4].x, 0.f),
                         make_float4(b[0].y, b[2].y, b[4].y, 0.f));
        };
        K key = 0;
        if (fast) {
            // top bits first (node r at bit ntop - 1 - r of tb), then the low
            // row of the first met top node (the highest set bit of tb)
            uint64_t tb = 0;
#pragma unroll 8
            for (uint32_t r = 0; r < ntop; ++r) tb = (tb << 1) | (uint64_t)hit(r);
            key = ntop ? (K)(tb << (key_bits - ntop)) : (K)0;
            if (tb) {
                const uint32_t rep = ntop - 64u + (uint32_t)__clzll((long long)tb);
                const uint32_t row = ntop + rep * low_field;
                uint64_t lb = 0;
#pragma unroll 8
                for (uint32_t j = 0; j < low_field; ++j) lb = (lb << 1) | (uint64_t)hit(row + j);
                if (low_field) key |= (K)(lb << (key_bits - top_field - low_field));
            }
        } else {
            K bit = (K)1 << (key_bits - 1);
            uint32_t rep = ntop;
            for (uint32_t r = 0; r < ntop; ++r, bit >>= 1)
                if (hit(r)) {
                    key |= bit;
                    rep = min(rep, r);
                }
            if (rep < ntop) {
                const uint32_t row = ntop + rep * low_field;
                K lbit = (K)1 << (key_bits - 1 - top_field);
                for (uint32_t j = 0; j < low_field; ++j, lbit >>= 1)
                    if (hit(row + j)) key |= lbit;
            }
        }
        __stcs(keys + i, key);
    }
}

// Prefix path code (Sec. 4.1): a depth-first, left-child-first walk that
// every ray takes in the same order; each visited node's box test is one key
// bit, a met internal node is entered, a missed subtree skipped, and the walk
// stops after key_bits tests.  The children's exact boxes come from the
// parent's 64-byte node; a parent whose right child is still due waits on a
// stack of node indices (each entry follows a test, so key_bits entries
// suffice).
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_ppc(const float4 *__restrict__ org,
                                                          const float4 *__restrict__ dir, uint64_t n, uint32_t rs,
                                                          const float4 *__restrict__ nodes, uint32_t root_ref,
                                                          float4 root_lo, float4 root_hi, uint32_t key_bits,
                                                          K *__restrict__ keys) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i * rs);
        const float4 d = __ldcs(dir + i * rs);
        const float ix = __frcp_rn(d.x), iy = __frcp_rn(d.y), iz = __frcp_rn(d.z);
        K key = 0;
        uint32_t m = 0;  // tests made
        const bool root_met = meets(o, d, ix, iy, iz, root_lo, root_hi);
        if (root_met) key |= (K)1 << (key_bits - 1);
        m = 1;
        uint32_t stack[64];
        uint32_t sp = 0;
        uint32_t cur = root_ref;
        bool right = false;  // which child of cur is visited next
        bool go = root_met && !(root_ref & REF_LEAF);
        while (go && m < key_bits) {
            const float4 *f = nodes + 4 * (size_t)cur;
            const float4 n0 = __ldg(f), n1 = __ldg(f + 1), n2 = __ldg(f + 2);
            const uint4 n3 = __ldg(reinterpret_cast<const uint4 *>(f + 3));
            float4 lo, hi;
            uint32_t child;
            if (!right) {  // exact node: per child (lo.x, lo.y), (hi.x, hi.y), (lo.z, hi.z)
                lo = make_float4(n0.x, n0.y, n1.x, 0.f);
                hi = make_float4(n0.z, n0.w, n1.y, 0.f);
                child = n3.x;
                stack[sp++] = cur;  // its right child follows the left subtree
            } else {
                lo = make_float4(n1.z, n1.w, n2.z, 0.f);
                hi = make_float4(n2.x, n2.y, n2.w, 0.f);
                child = n3.y;
            }
            const bool met = meets(o, d, ix, iy, iz, lo, hi);
            if (met) key |= (K)1 << (key_bits - 1 - m);
            ++m;
            if (met && !(child & REF_LEAF)) {
                cur = child;
                right = false;
            } else if (sp > 0) {
                cur = stack[--sp];
                right = true;
            } else {
                go = false;
            }
        }
        __stcs(keys + i, key);
    }
}

}  // namespace

cudaError_t launch_encode_mlhcc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                const float4 *top, uint32_t ntop, uint32_t top_field, const float4 *low,
                                uint32_t low_field, uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    if (ntop > top_field || top_field + low_field > MAX_CUT_BITS || top_field + low_field > key_bits)
        return cudaErrorInvalidValue;
    // six float2 per box: at most (32 + 32 * 32) * 48 bytes = 50,688 bytes
    const size_t smem = sizeof(float2) * 6 * ((size_t)ntop + (size_t)ntop * low_field);
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_encode_mlhcc<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_encode_mlhcc<uint32_t><<<grid, ENC_BLOCK, smem, s>>>(org, dir, n, rs, top, ntop, top_field, low, low_field,
                                                              key_bits, (uint32_t *)keys);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_encode_mlhcc<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_encode_mlhcc<uint64_t><<<grid, ENC_BLOCK, smem, s>>>(org, dir, n, rs, top, ntop, top_field, low, low_field,
                                                              key_bits, (uint64_t *)keys);
    }
    return cudaGetLastError();
}

cudaError_t launch_encode_ppc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs, const uint4 *nodes,
                              uint32_t root_ref, const float root_lo[3], const float root_hi[3], uint32_t key_bits,
                              void *keys) {
    if (n == 0) return cudaSuccess;
    if (key_bits < 1 || key_bits > MAX_CUT_BITS) return cudaErrorInvalidValue;
    const float4 lo = make_float4(root_lo[0], root_lo[1], root_lo[2], 0.f);
    const float4 hi = make_float4(root_hi[0], root_hi[1], root_hi[2], 0.f);
    const float4 *f = reinterpret_cast<const float4 *>(nodes);
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_ppc<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, f, root_ref, lo, hi, key_bits,
                                                          (uint32_t *)keys);
    else
        k_encode_ppc<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, f, root_ref, lo, hi, key_bits,
                                                          (uint64_t *)keys);
    return cudaGetLastError();
}

cudaError_t launch_encode_hcc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                              const float4 *cut_boxes, uint32_t used, uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    if (used > MAX_CUT_BITS) used = MAX_CUT_BITS;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_hcc<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, cut_boxes, used, key_bits, (uint32_t *)keys);
    else
        k_encode_hcc<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, cut_boxes, used, key_bits, (uint64_t *)keys);
    return cudaGetLastError();
}

cudaError_t launch_encode_twopoint(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n, uint32_t rs,
                                   const float lo[3], const float ext[3], float L, uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_twopoint<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, lo[0], lo[1], lo[2], ext[0], ext[1],
                                                               ext[2], L, key_bits, (uint32_t *)keys);
    else
        k_encode_twopoint<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, rs, lo[0], lo[1], lo[2], ext[0], ext[1],
                                                               ext[2], L, key_bits, (uint64_t *)keys);
    return cudaGetLastError();
}

}  // namespace hcc
