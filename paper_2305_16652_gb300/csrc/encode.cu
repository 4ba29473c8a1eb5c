// Key encoding kernels: hierarchy cut code (Algorithm 1, Sec. 4.2.1) and the
// TwoPoint baseline (Sec. 3.2, Sec. 5).
//
// Floating point: every rounding step is an explicit round-to-nearest
// intrinsic and the library is built with --fmad=false, so each key is the
// same bit pattern the arithmetic defines, whatever the compiler schedules.
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

// Algorithm 1: the cut nodes are staged in shared memory once per block
// (line 1); every ray is tested against every cut node and each result sets
// one key bit.  Cut node r drives bit (key_bits - 1 - r).  Slab test per
// axis: t = (bound - o) * (1/d), tn = min, tf = max; tnear = max over axes
// and tmin, tfar = min over axes and tmax; the node is met when tnear <= tfar.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_hcc(const float4 *__restrict__ org,
                                                          const float4 *__restrict__ dir, uint64_t n,
                                                          const float4 *__restrict__ cut, uint32_t used,
                                                          uint32_t key_bits, K *__restrict__ keys) {
    __shared__ float4 s_lo[MAX_CUT_BITS], s_hi[MAX_CUT_BITS];
    for (uint32_t r = threadIdx.x; r < used; r += blockDim.x) {
        s_lo[r] = cut[2 * r];
        s_hi[r] = cut[2 * r + 1];
    }
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i);
        const float4 d = __ldcs(dir + i);
        const float ix = __frcp_rn(d.x), iy = __frcp_rn(d.y), iz = __frcp_rn(d.z);
        K key = 0;
        K bit = (K)1 << (key_bits - 1);
        for (uint32_t r = 0; r < used; ++r, bit >>= 1) {
            const float4 lo = s_lo[r], hi = s_hi[r];
            const float ax = __fmul_rn(__fsub_rn(lo.x, o.x), ix), bx = __fmul_rn(__fsub_rn(hi.x, o.x), ix);
            const float ay = __fmul_rn(__fsub_rn(lo.y, o.y), iy), by = __fmul_rn(__fsub_rn(hi.y, o.y), iy);
            const float az = __fmul_rn(__fsub_rn(lo.z, o.z), iz), bz = __fmul_rn(__fsub_rn(hi.z, o.z), iz);
            const float tnear = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, by)), fmaxf(fminf(az, bz), o.w));
            const float tfar = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, by)), fminf(fmaxf(az, bz), d.w));
            if (tnear <= tfar) key |= bit;
        }
        __stcs(keys + i, key);
    }
}

// TwoPoint: o and t = o + L d (one fused multiply-add per axis) normalised
// to the scene box, quantised to b bits, Morton-interleaved most significant
// level first in the order o.x o.y o.z t.x t.y t.z, left-justified in k bits.
template <typename K>
__global__ void __launch_bounds__(ENC_BLOCK) k_encode_twopoint(const float4 *__restrict__ org,
                                                               const float4 *__restrict__ dir, uint64_t n,
                                                               float lox, float loy, float loz, float ex, float ey,
                                                               float ez, float L, uint32_t key_bits,
                                                               K *__restrict__ keys) {
    const uint32_t b = key_bits / 6;
    const float levels = (float)(1u << b);  // exact power of two (b <= 10)
    const uint32_t qmax = b ? ((1u << b) - 1u) : 0u;
    const uint32_t pad = key_bits - 6 * b;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 o = __ldcs(org + i);
        const float4 d = __ldcs(dir + i);
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

}  // namespace

cudaError_t launch_encode_hcc(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n,
                              const float4 *cut_boxes, uint32_t used, uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    if (used > MAX_CUT_BITS) used = MAX_CUT_BITS;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_hcc<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, cut_boxes, used, key_bits, (uint32_t *)keys);
    else
        k_encode_hcc<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, cut_boxes, used, key_bits, (uint64_t *)keys);
    return cudaGetLastError();
}

cudaError_t launch_encode_twopoint(cudaStream_t s, const float4 *org, const float4 *dir, uint64_t n,
                                   const float lo[3], const float ext[3], float L, uint32_t key_bits, void *keys) {
    if (n == 0) return cudaSuccess;
    const int grid = encode_grid(n, ENC_BLOCK, 8);
    if (key_bits <= 32)
        k_encode_twopoint<uint32_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, lo[0], lo[1], lo[2], ext[0], ext[1],
                                                               ext[2], L, key_bits, (uint32_t *)keys);
    else
        k_encode_twopoint<uint64_t><<<grid, ENC_BLOCK, 0, s>>>(org, dir, n, lo[0], lo[1], lo[2], ext[0], ext[1],
                                                               ext[2], L, key_bits, (uint64_t *)keys);
    return cudaGetLastError();
}

}  // namespace hcc
