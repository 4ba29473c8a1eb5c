// Gather of rays into sorted order (Sec. 5: the trace fetches rays through
// the sorted indices): out[j] = in[perm[j]] for both float4 streams.
//
// Each thread moves GATHER_RAYS rays: the permutation entries and the
// output rays are read/written coalesced; the two 16-byte source records of a
// ray are read through the read-only path.  The output is streamed (evict
// first) because the trace reads it once, much later.
#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int GATHER_BLOCK = 256;
constexpr int GATHER_RAYS = 4;

__global__ void __launch_bounds__(GATHER_BLOCK) k_gather(const float4 *__restrict__ in_org,
                                                         const float4 *__restrict__ in_dir,
                                                         uint64_t in_n, const uint32_t *__restrict__ perm,
                                                         float4 *__restrict__ out_org, float4 *__restrict__ out_dir,
                                                         uint64_t n, uint32_t *err) {
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
                o[k] = __ldg(in_org + src[k]);
                d[k] = __ldg(in_dir + src[k]);
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
            __stcs(out_org + j, o[k]);
            __stcs(out_dir + j, d[k]);
        }
    }
}

}  // namespace

cudaError_t launch_gather(cudaStream_t s, const float4 *in_org, const float4 *in_dir, uint64_t in_n,
                          const uint32_t *perm, float4 *out_org, float4 *out_dir, uint64_t n, uint32_t *err) {
    if (n == 0) return cudaSuccess;
    const uint64_t per_block = (uint64_t)GATHER_BLOCK * GATHER_RAYS;
    const uint64_t blocks = (n + per_block - 1) / per_block;
    k_gather<<<(unsigned)blocks, GATHER_BLOCK, 0, s>>>(in_org, in_dir, in_n, perm, out_org, out_dir, n, err);
    return cudaGetLastError();
}

}  // namespace hcc
