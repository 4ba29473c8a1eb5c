// hcc_sort_noalloc: the radix sort of hcc_sort for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a host program whose
// device memory is entirely reserved up front by its own allocator (a
// stray cudaMalloc then fails or fragments the pool), or a latency-bound
// loop in which the device-wide synchronisation that cudaMalloc/cudaFree
// may imply is not acceptable.  This entry point needs no context and no
// allocation: its scratch is one fixed-size array in device memory that
// belongs to this file, sized for HCC_SORT_NOALLOC_MAX_N keys of up to 64
// bits (12 MiB, held by every device that loads the library for as long as
// the process lives).
//
// The array is a __device__ symbol, so host code only knows a stand-in for
// it; the real device address is looked up with cudaGetSymbolAddress once
// per device, with that device current, the first time the entry point runs
// on it.  That first call should therefore come before any stream capture.
// Every call uses the same array and leaves its contents behind; the sort
// clears what must start at zero (histograms, look-back words) itself.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and give wrong results.
#include <mutex>

#include "hcc_internal.cuh"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)12 << 20;  // >= sort scratch of HCC_SORT_NOALLOC_MAX_N 64-bit keys
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ uint32_t g_noalloc_err;  // sink for error bits when the caller passes no error word (never read)

std::mutex g_mu;
void *g_scratch_ptr[MAX_DEVICES] = {};
uint32_t *g_err_ptr[MAX_DEVICES] = {};

// Device addresses of this file's arrays on the current device (set up once).
cudaError_t device_arrays(int dev, void **scratch, uint32_t **err) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *s = nullptr, *e = nullptr;
        cudaError_t rc = cudaGetSymbolAddress(&s, g_noalloc_scratch);
        if (rc != cudaSuccess) return rc;
        rc = cudaGetSymbolAddress(&e, g_noalloc_err);
        if (rc != cudaSuccess) return rc;
        g_scratch_ptr[dev] = s;
        g_err_ptr[dev] = static_cast<uint32_t *>(e);
    }
    *scratch = g_scratch_ptr[dev];
    *err = g_err_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" hcc_status hcc_sort_noalloc(const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm,
                                       uint32_t *err_word, void *stream) {
    if (key_bits < 1 || key_bits > 64) return HCC_ERR_INVALID_ARG;
    if (n > HCC_SORT_NOALLOC_MAX_N) return HCC_ERR_INVALID_ARG;
    if (n == 0) return HCC_OK;
    const size_t ksz = key_bits > 32 ? 8 : 4;
    if (!keys || !perm || (reinterpret_cast<uintptr_t>(keys) % ksz) != 0 || (reinterpret_cast<uintptr_t>(perm) % 4) != 0)
        return HCC_ERR_INVALID_ARG;
    if (err_word && (reinterpret_cast<uintptr_t>(err_word) % 4) != 0) return HCC_ERR_INVALID_ARG;
    const uintptr_t k0 = (uintptr_t)keys, k1 = k0 + n * ksz, p0 = (uintptr_t)perm, p1 = p0 + n * 4;
    if (k0 < p1 && p0 < k1) return HCC_ERR_INVALID_ARG;
    if (hcc::sort_scratch_bytes(n, key_bits) > NOALLOC_SCRATCH_BYTES) return HCC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HCC_ERR_CUDA;
    void *scratch = nullptr;
    uint32_t *own_err = nullptr;
    if (device_arrays(dev, &scratch, &own_err) != cudaSuccess) {
        cudaGetLastError();
        return HCC_ERR_CUDA;
    }
    const cudaError_t e = hcc::launch_sort(static_cast<cudaStream_t>(stream), keys, key_bits, n, perm, scratch,
                                           err_word ? err_word : own_err);
    return e == cudaSuccess ? HCC_OK : HCC_ERR_CUDA;
}
