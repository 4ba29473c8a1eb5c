// Gather of rays into sorted order (Sec. 5: the trace fetches rays through
// the sorted indices): out[j] = in[perm[j]] for both float4 streams.
//
// Each thread moves GATHER_RAYS rays: the permutation entries and the
// output rays are read/written coalesced; the source records are read
// through the read-only path.  When both sides hold 32-byte ray records
// (origin and direction adjacent), a ray moves as one 32-byte load and one
// 32-byte store, so a random source ray costs one DRAM sector rather than
// two in separate streams.  The output is streamed (evict first) because the
// trace reads it once, much later.
#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int GATHER_BLOCK = 256;
constexpr int GATHER_RAYS = 4;

__device__ __forceinline__ void ld_rec(const float4 *p, float4 &o, float4 &d) {
    asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w), "=f"(d.x), "=f"(d.y), "=f"(d.z), "=f"(d.w)
                 : "l"(p));
}
__device__ __forceinline__ void st_rec(float4 *p, const float4 &o, const float4 &d) {
    asm volatile("st.global.cs.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(o.x), "f"(o.y),
                 "f"(o.z), "f"(o.w), "f"(d.x), "f"(d.y), "f"(d.z), "f"(d.w)
                 : "memory");
}

// REC: both sides are 32-byte records (in_dir = in_org + 1, out_dir =
// out_org + 1, 32-byte aligned); otherwise streams with strides in_rs /
// out_rs (float4 units).
template <bool REC>
__global__ void __launch_bounds__(GATHER_BLOCK) k_gather(const float4 *__restrict__ in_org,
                                                         const float4 *__restrict__ in_dir, uint32_t in_rs,
                                                         uint64_t in_n, const uint32_t *__restrict__ perm,
                                                         float4 *__restrict__ out_org, float4 *__restrict__ out_dir,
                                                         uint32_t out_rs, uint64_t n, uint32_t *err) {
    const uint64_t base = (uint64_t)blockIdx.x * (GATHER_BLOCK * GATHER_RAYS) + threadIdx.x;
    uint32_t src[GATHER_RAYS];
#pragma unroll
    for (int k = 0; k < GATHER_RAYS; ++k) {
        const uint64_t j = base + (uint64_t)k * GATHER_BLOCK;
        src[k] = j < n ? __ldcs(perm + j) : 0u;
    }
    float4 o[GATHER_RAYS], d[GATHER_RAYS];
#pragma unroll
    for (int k = 0; k < GATHER_RAYS; ++k) {
        const uint64_t j = base + (uint64_t)k * GATHER_BLOCK;
        if (j < n) {
            if (src[k] < in_n) {
                if (REC) {
                    ld_rec(in_org + 2 * (uint64_t)src[k], o[k], d[k]);
                } else {
                    o[k] = __ldg(in_org + (uint64_t)src[k] * in_rs);
                    d[k] = __ldg(in_dir + (uint64_t)src[k] * in_rs);
                }
            } else {  // invalid permutation entry: report, never read out of bounds
                atomicOr(err, ERR_INDEX);
                o[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                d[k] = o[k];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < GATHER_RAYS; ++k) {
        const uint64_t j = base + (uint64_t)k * GATHER_BLOCK;
        if (j < n) {
            if (REC) {
                st_rec(out_org + 2 * j, o[k], d[k]);
            } else {
                __stcs(out_org + j * out_rs, o[k]);
                __stcs(out_dir + j * out_rs, d[k]);
            }
        }
    }
}

bool is_record(const float4 *org, const float4 *dir, uint32_t rs) {
    return rs == 2 && dir == org + 1 && (reinterpret_cast<uintptr_t>(org) & 31u) == 0;
}

}  // namespace

cudaError_t launch_gather(cudaStream_t s, const float4 *in_org, const float4 *in_dir, uint32_t in_rs, uint64_t in_n,
                          const uint32_t *perm, float4 *out_org, float4 *out_dir, uint32_t out_rs, uint64_t n,
                          uint32_t *err) {
    if (n == 0) return cudaSuccess;
    const uint64_t per_block = (uint64_t)GATHER_BLOCK * GATHER_RAYS;
    const uint64_t blocks = (n + per_block - 1) / per_block;
    if (is_record(in_org, in_dir, in_rs) && is_record(out_org, out_dir, out_rs))
        k_gather<true><<<(unsigned)blocks, GATHER_BLOCK, 0, s>>>(in_org, in_dir, in_rs, in_n, perm, out_org, out_dir,
                                                                 out_rs, n, err);
    else
        k_gather<false><<<(unsigned)blocks, GATHER_BLOCK, 0, s>>>(in_org, in_dir, in_rs, in_n, perm, out_org,
                                                                  out_dir, out_rs, n, err);
    return cudaGetLastError();
}

}  // namespace hcc
