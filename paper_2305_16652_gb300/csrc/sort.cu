// Stable LSD radix sort of ray ids by key (Sec. 4.2.3 "Sorting": keys are
// sorted as natural numbers; Sec. 5: the sort orders ray indices).
//
// Design (one pass per 8-bit digit, "onesweep" structure):
//   k_hist   one read of every key builds the digit histograms of all passes
//   k_plan   exclusive scan of each histogram; passes whose digit is the same
//            for every key are marked inactive (skipping them cannot change a
//            stable result); the ping-pong buffer of every active pass is
//            chosen so that the first active pass reads the caller's keys and
//            synthesises ids, and the last one writes only the permutation
//   k_pass   per 4096-key tile: warp-level ranking (match.any, or a ballot
//            split when a warp's digits are spread), per-digit tile counts
//            published to a decoupled look-back chain (bounded waits), keys
//            reordered in shared memory and written out in runs of equal
//            digits (coalesced)
//   k_ident  perm = identity when no pass is active (all keys equal, n <= 1)
// Tiles take their position from an atomic counter in launch order, so a tile
// only ever waits for tiles that are already running.
#include <algorithm>
#include <atomic>

#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int RADIX = 256;
constexpr int MAX_PASSES = 8;
constexpr int SORT_BLOCK = 256;  // one thread per digit in the scan / look-back
constexpr int SORT_WARPS = SORT_BLOCK / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_BLOCK * SORT_ITEMS;
constexpr uint32_t ST_AGG = 1u << 30;  // tile count of this digit available
constexpr uint32_t ST_INC = 2u << 30;  // inclusive prefix of this digit available
constexpr uint32_t ST_VALUE = (1u << 30) - 1u;
constexpr uint32_t SPIN_LIMIT = 1u << 22;  // total status reads a tile may wait
constexpr int LOOKBACK = 4;                // predecessors read per look-back round
constexpr int MATCH_MAX_DISTINCT = 16;     // distinct digits per warp item below which match.any ranks

enum : int { KB_USER = 0, KB_A = 1, KB_B = 2, KB_NONE = 3 };
enum : int { VB_SYNTH = 0, VB_A = 1, VB_PERM = 2 };

struct PassPlan {
    int active, src_keys, dst_keys, src_vals, dst_vals, pad[3];
};

// Scratch header, followed by the status words [passes][tiles][RADIX] and
// the ping-pong buffers.
struct SortHeader {
    uint32_t hist[MAX_PASSES][RADIX];
    uint32_t start[MAX_PASSES][RADIX];
    PassPlan plan[MAX_PASSES];
    uint32_t tile_counter[MAX_PASSES];
    uint32_t identity;
    uint32_t abort;
    uint32_t pad[14];
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t header, status, ka, kb, va, total;
};

Layout layout(uint64_t n, uint32_t key_bits) {
    const uint32_t passes = (key_bits + 7) / 8;
    const uint64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
    const size_t ksz = key_bits > 32 ? 8 : 4;
    Layout L;
    L.header = 0;
    L.status = align256(sizeof(SortHeader));
    L.ka = L.status + align256((size_t)passes * tiles * RADIX * sizeof(uint32_t));
    L.kb = L.ka + align256(n * ksz);
    L.va = L.kb + align256(n * ksz);
    L.total = L.va + align256(n * sizeof(uint32_t));
    return L;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp whose digit equals this lane's, found with one ballot per
// digit bit (data-independent cost, unlike match.any whose cost grows with
// the number of distinct values).  valid_mask: lanes holding a real item.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, uint32_t dbits, uint32_t valid_mask) {
    uint32_t peers = valid_mask;
    for (uint32_t b = 0; b < dbits; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

template <typename K>
__device__ __forceinline__ K key_mask(uint32_t key_bits) {
    return key_bits >= 8 * sizeof(K) ? (K)~(K)0 : (K)(((K)1 << key_bits) - 1);
}

// One read of all keys: digit histograms of every pass.  Keys of ray
// batches are heavily skewed (one digit value often holds most keys), so
// each warp first picks the most common digit of its first 32 keys for each
// pass and counts that value in a register; every other digit goes to a
// shared-memory atomic, where collisions are then rare.
template <typename K>
__global__ void __launch_bounds__(SORT_BLOCK) k_hist(const K *__restrict__ keys, uint64_t n, uint32_t key_bits,
                                                     int passes, SortHeader *h) {
    __shared__ uint32_t sh[MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const K mask = key_mask<K>(key_bits);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // dominant digit per pass among the warp's first keys
    const K k0 = first < n ? (keys[first] & mask) : (K)0;
    uint32_t dom[MAX_PASSES], cnt[MAX_PASSES];
#pragma unroll
    for (int p = 0; p < MAX_PASSES; ++p) {
        cnt[p] = 0;
        dom[p] = 0;
        if (p < passes) {
            const uint32_t d = (uint32_t)(k0 >> (8 * p)) & 255u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, first < n ? d : 256u + lane);
            uint32_t best = ((uint32_t)__popc(peers) << 9) | d;
            best = __reduce_max_sync(0xFFFFFFFFu, best);
            dom[p] = best & 511u;
        }
    }
    constexpr int UNROLL = 8;  // independent loads in flight per thread
    for (uint64_t base = first; base < n; base += UNROLL * stride) {
        K kk[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const uint64_t i = base + (uint64_t)u * stride;
            kk[u] = i < n ? (__ldcs(keys + i) & mask) : (K)0;
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (base + (uint64_t)u * stride >= n) break;
#pragma unroll
            for (int p = 0; p < MAX_PASSES; ++p) {
                if (p < passes) {
                    const uint32_t d = (uint32_t)(kk[u] >> (8 * p)) & 255u;
                    if (d == dom[p])
                        ++cnt[p];
                    else
                        atomicAdd(&sh[p * RADIX + d], 1u);
                }
            }
        }
    }
#pragma unroll
    for (int p = 0; p < MAX_PASSES; ++p) {
        if (p < passes) {
            const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, cnt[p]);
            if (lane == 0 && c && dom[p] < 256u) atomicAdd(&sh[p * RADIX + dom[p]], c);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&h->hist[0][0] + i, sh[i]);
}

// Exclusive scan per pass, pass activity and buffer plan.  One block.
__global__ void __launch_bounds__(RADIX) k_plan(SortHeader *h, int passes, uint64_t n) {
    __shared__ uint32_t s_scan[RADIX];
    __shared__ int s_trivial[MAX_PASSES];
    const int t = threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        const uint32_t c = h->hist[p][t];
        s_scan[t] = c;
        __syncthreads();
        for (int off = 1; off < RADIX; off <<= 1) {
            const uint32_t v = t >= off ? s_scan[t - off] : 0u;
            __syncthreads();
            s_scan[t] += v;
            __syncthreads();
        }
        h->start[p][t] = s_scan[t] - c;
        if (t == 0) s_trivial[p] = 0;
        __syncthreads();
        if ((uint64_t)c == n) s_trivial[p] = 1;
        __syncthreads();
    }
    if (t == 0) {
        int act[MAX_PASSES], m = 0;
        for (int p = 0; p < passes; ++p) {
            h->plan[p].active = 0;
            if (!s_trivial[p]) act[m++] = p;
        }
        for (int idx = 0; idx < m; ++idx) {
            PassPlan &pl = h->plan[act[idx]];
            pl.active = 1;
            pl.dst_vals = ((m - 1 - idx) % 2 == 0) ? VB_PERM : VB_A;
            pl.dst_keys = (idx == m - 1) ? KB_NONE : (((m - 2 - idx) % 2 == 0) ? KB_A : KB_B);
        }
        for (int idx = 0; idx < m; ++idx) {
            PassPlan &pl = h->plan[act[idx]];
            pl.src_keys = idx == 0 ? KB_USER : h->plan[act[idx - 1]].dst_keys;
            pl.src_vals = idx == 0 ? VB_SYNTH : h->plan[act[idx - 1]].dst_vals;
        }
        h->identity = (m == 0);
    }
}

template <typename K>
struct PassArgs {
    const K *user_keys;
    K *ka, *kb;
    uint32_t *va, *perm;
    uint32_t *status;
    SortHeader *h;
    uint64_t n;
    uint32_t key_bits, num_tiles;
    uint32_t *err;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy count elements of T from global src to shared dst with asynchronous
// copies: 16-byte chunks when the whole tile is present and src is 16-byte
// aligned, element by element otherwise.  Only elements below count are read.
template <typename T>
__device__ __forceinline__ void load_tile_async(T *dst, const T *src, uint32_t count) {
    if (count == SORT_TILE && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        constexpr uint32_t per = 16 / sizeof(T), chunks = SORT_TILE / per;
        for (uint32_t c = threadIdx.x; c < chunks; c += SORT_BLOCK) cp_async16(dst + c * per, src + c * per);
    } else {
        for (uint32_t p = threadIdx.x; p < count; p += SORT_BLOCK) {
            if (sizeof(T) == 8)
                cp_async8(dst + p, src + p);
            else
                cp_async4(dst + p, src + p);
        }
    }
}

// One digit pass.  Persistent blocks (three per SM for 32-bit keys, two for
// 64-bit keys) take tiles of 4096 keys in launch order from an atomic
// counter; while a tile is ranked and written, the next tile's keys and
// values stream into the other shared-memory buffer (cp.async), so the DRAM
// latency of a tile overlaps the work on the previous one.  Per tile:
// warp-level stable ranking (match.any or the ballot bit-split, the group
// leader's atomic returns the group's base), the tile's digit counts
// published at once to the decoupled look-back chain, the tile reordered by
// digit in shared memory, the look-back for the global offsets (bounded
// waits with back-off), and runs of equal digits written out coalesced.
// A block handles its tiles in increasing order, so the lowest unfinished
// tile is always being worked on and every wait ends.
template <typename K>
__global__ void __launch_bounds__(SORT_BLOCK, sizeof(K) == 4 ? 3 : 2) k_pass(PassArgs<K> a, int pass) {
    const PassPlan pl = a.h->plan[pass];
    if (!pl.active) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *in_keys = reinterpret_cast<K *>(smem_raw);                                  // [2][TILE]
    uint32_t *in_vals = reinterpret_cast<uint32_t *>(in_keys + 2 * SORT_TILE);     // [2][TILE]
    __shared__ uint32_t s_whist[SORT_WARPS][RADIX];
    __shared__ uint32_t s_local[RADIX];
    __shared__ uint32_t s_base[RADIX];
    __shared__ uint32_t s_wsum[SORT_WARPS];
    __shared__ uint32_t s_next, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t shift = 8u * (uint32_t)pass;
    const K mask = key_mask<K>(a.key_bits);
    const uint32_t dbits = a.key_bits - shift < 8u ? a.key_bits - shift : 8u;
    const K *kin = pl.src_keys == KB_USER ? a.user_keys : (pl.src_keys == KB_A ? a.ka : a.kb);
    const uint32_t *vin = pl.src_vals == VB_A ? a.va : a.perm;
    const bool synth = pl.src_vals == VB_SYNTH;
    K *kout = pl.dst_keys == KB_A ? a.ka : (pl.dst_keys == KB_B ? a.kb : nullptr);
    uint32_t *vout = pl.dst_vals == VB_A ? a.va : a.perm;
    const uint32_t lt = lanemask_lt();
    const uint32_t wfirst = (uint32_t)warp * (SORT_ITEMS * 32) + lane;  // tile position of this lane's item 0

    auto tile_count = [&](uint32_t t) -> uint32_t {
        const uint64_t b = (uint64_t)t * SORT_TILE;
        return (uint32_t)((a.n - b) < (uint64_t)SORT_TILE ? (a.n - b) : SORT_TILE);
    };
    auto issue = [&](uint32_t t, int buf) {
        if (t < a.num_tiles) {
            const uint64_t b = (uint64_t)t * SORT_TILE;
            const uint32_t cnt = tile_count(t);
            load_tile_async(in_keys + buf * SORT_TILE, kin + b, cnt);
            if (!synth) load_tile_async(in_vals + buf * SORT_TILE, vin + b, cnt);
        }
        cp_async_commit();  // possibly empty group: keeps one group per tile
    };

    if (tid == 0) {
        s_next = atomicAdd(&a.h->tile_counter[pass], 1u);
        s_abort = 0;
    }
    __syncthreads();
    uint32_t cur = s_next;
    int buf = 0;
    issue(cur, buf);
    while (cur < a.num_tiles) {
        __syncthreads();  // everyone is done with the previous tile and has read s_next
        if (tid == 0) s_next = atomicAdd(&a.h->tile_counter[pass], 1u);
        for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_BLOCK) (&s_whist[0][0])[i] = 0;
        __syncthreads();
        const uint32_t nxt = s_next;
        issue(nxt, buf ^ 1);
        cp_async_wait_prev();  // this thread's copies of the current tile have landed
        __syncthreads();       // ... and everyone's

        const uint32_t tile = cur;
        const uint64_t base = (uint64_t)tile * SORT_TILE;
        const uint32_t tile_n = tile_count(tile);
        K *tk = in_keys + buf * SORT_TILE;  // the tile's keys, then (reordered) its staging area
        uint32_t *tv = in_vals + buf * SORT_TILE;

        // this thread's items in registers; the buffer is reused for the reorder
        K kreg[SORT_ITEMS];
        uint32_t vreg[SORT_ITEMS];
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t pos = wfirst + (uint32_t)i * 32;
            kreg[i] = pos < tile_n ? (tk[pos] & mask) : (K)0;
            vreg[i] = synth ? (uint32_t)(base + pos) : (pos < tile_n ? tv[pos] : 0u);
        }

        // warp-level stable ranking: lanes with equal digits found by match.any
        // while the warp's items hold few distinct digits (ray keys do), by
        // the fixed-cost ballot split otherwise; the choice follows the
        // previous item's number of distinct digits
        uint32_t rank[SORT_ITEMS];
        uint32_t *wh = s_whist[warp];
        bool use_match = true;
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t pos = wfirst + (uint32_t)i * 32;
            const bool valid = pos < tile_n;
            const uint32_t d = valid ? (uint32_t)(kreg[i] >> shift) & 255u : 0u;
            const uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
            const uint32_t peers = use_match ? (__match_any_sync(0xFFFFFFFFu, valid ? d : 256u + lane) & vmask)
                                             : digit_peers(d, dbits, vmask);
            const uint32_t leader = __ffs(peers) - 1;
            use_match = __popc(__ballot_sync(0xFFFFFFFFu, valid && (uint32_t)lane == leader)) <= MATCH_MAX_DISTINCT;
            uint32_t prior = 0;
            if (valid && (uint32_t)lane == leader) prior = atomicAdd(&wh[d], (uint32_t)__popc(peers));
            prior = __shfl_sync(0xFFFFFFFFu, prior, valid ? leader : lane);
            rank[i] = prior + __popc(peers & lt);
        }
        __syncthreads();
        // thread tid owns digit tid: warp offsets, tile count, publication
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = s_whist[w][tid];
            s_whist[w][tid] = total;
            total += c;
        }
        uint32_t *st = a.status + ((size_t)pass * a.num_tiles + tile) * RADIX;
        if (tile == 0)
            st_relaxed(st + tid, ST_INC | ((a.h->start[pass][tid] + total) & ST_VALUE));
        else
            st_relaxed(st + tid, ST_AGG | total);
        uint32_t incl = total;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        uint32_t wpre = 0;
        for (int w = 0; w < warp; ++w) wpre += s_wsum[w];
        s_local[tid] = wpre + incl - total;
        __syncthreads();
        // reorder the tile by digit (stable) into its own buffer: every thread
        // read its items before the barriers above
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t pos = wfirst + (uint32_t)i * 32;
            if (pos < tile_n) {
                const uint32_t d = (uint32_t)(kreg[i] >> shift) & 255u;
                const uint32_t o = s_local[d] + wh[d] + rank[i];
                tk[o] = kreg[i];
                tv[o] = vreg[i];
            }
        }
        // decoupled look-back for digit tid
        uint32_t excl;
        if (tile == 0) {
            excl = a.h->start[pass][tid];
        } else {
            excl = 0;
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            bool timed_out = false, done = false;
            const uint32_t *col = a.status + (size_t)pass * a.num_tiles * RADIX + tid;
            while (!done) {
                uint32_t sv[LOOKBACK];
#pragma unroll
                for (int w = 0; w < LOOKBACK; ++w)
                    sv[w] = (j - w >= 0) ? ld_relaxed(col + (size_t)(j - w) * RADIX) : ST_INC;
                int used = 0;
                bool stalled = false;
#pragma unroll
                for (int w = 0; w < LOOKBACK; ++w) {
                    if (done || stalled) continue;
                    const uint32_t flag = sv[w] & ~ST_VALUE;
                    if (flag == 0) {
                        stalled = true;
                        continue;
                    }
                    if (j - w >= 0) excl += sv[w] & ST_VALUE;
                    ++used;
                    if (flag == ST_INC) done = true;
                }
                j -= used;
                if (done) break;
                if (stalled) {
                    if (++spins > SPIN_LIMIT / LOOKBACK || ((spins & 63u) == 0 && ld_relaxed(&a.h->abort))) {
                        timed_out = true;
                        break;
                    }
                    __nanosleep(spins < 8 ? 32u * spins : 256u);
                }
            }
            if (timed_out) {
                atomicOr(a.err, ERR_TIMEOUT);
                atomicExch(&a.h->abort, 1u);
                s_abort = 1;
            }
            st_relaxed(st + tid, ST_INC | ((excl + total) & ST_VALUE));
        }
        s_base[tid] = excl;
        __syncthreads();
        if (s_abort) break;
        // runs of equal digits to their global positions
#pragma unroll 4
        for (uint32_t p = tid; p < tile_n; p += SORT_BLOCK) {
            const K k = tk[p];
            const uint32_t d = (uint32_t)(k >> shift) & 255u;
            const uint32_t g = s_base[d] + (p - s_local[d]);
            if (kout) __stcs(kout + g, k);
            __stcs(vout + g, tv[p]);
        }
        cur = nxt;
        buf ^= 1;
    }
    cp_async_wait_all();
}

__global__ void k_ident(const SortHeader *h, uint32_t *perm, uint64_t n) {
    if (!h->identity) return;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) perm[i] = (uint32_t)i;
}

template <typename K>
cudaError_t run_sort(cudaStream_t s, const K *keys, uint32_t key_bits, uint64_t n, uint32_t *perm,
                     unsigned char *scratch, uint32_t *err) {
    const Layout L = layout(n, key_bits);
    const int passes = (int)((key_bits + 7) / 8);
    const uint32_t tiles = (uint32_t)((n + SORT_TILE - 1) / SORT_TILE);
    SortHeader *h = reinterpret_cast<SortHeader *>(scratch + L.header);
    cudaError_t e = cudaMemsetAsync(scratch, 0, L.ka, s);  // header + status words
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t hblocks = (n + SORT_BLOCK * 8 - 1) / (SORT_BLOCK * 8);
    const uint64_t hcap = (uint64_t)(sms > 0 ? sms : 1) * 4;
    if (hblocks > hcap) hblocks = hcap;
    if (hblocks == 0) hblocks = 1;
    k_hist<K><<<(unsigned)hblocks, SORT_BLOCK, 0, s>>>(keys, n, key_bits, passes, h);
    k_plan<<<1, RADIX, 0, s>>>(h, passes, n);
    PassArgs<K> a;
    a.user_keys = keys;
    a.ka = reinterpret_cast<K *>(scratch + L.ka);
    a.kb = reinterpret_cast<K *>(scratch + L.kb);
    a.va = reinterpret_cast<uint32_t *>(scratch + L.va);
    a.perm = perm;
    a.status = reinterpret_cast<uint32_t *>(scratch + L.status);
    a.h = h;
    a.n = n;
    a.key_bits = key_bits;
    a.num_tiles = tiles;
    a.err = err;
    const size_t dyn = 2 * (sizeof(K) + sizeof(uint32_t)) * SORT_TILE;  // 2 tile buffers (prefetch, current)
    // the shared-memory opt-in is set once per device (so that a sort can be
    // captured in a CUDA graph without any non-stream call)
    static std::atomic<uint64_t> opted{0};
    if (dev >= 0 && dev < 64 && !(opted.load() & (1ull << dev))) {
        e = cudaFuncSetAttribute(k_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        opted.fetch_or(1ull << dev);
    }
    const uint32_t per_sm = sizeof(K) == 4 ? 3u : 2u;  // blocks that fit the shared memory
    const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)(sms > 0 ? sms : 1) * per_sm);
    for (int p = 0; p < passes; ++p) k_pass<K><<<grid, SORT_BLOCK, dyn, s>>>(a, p);
    uint64_t iblocks = (n + 255) / 256;
    if (iblocks > 4096) iblocks = 4096;
    k_ident<<<(unsigned)iblocks, 256, 0, s>>>(h, perm, n);
    return cudaGetLastError();
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n, uint32_t key_bits) { return layout(n, key_bits).total; }

cudaError_t launch_sort(cudaStream_t s, const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm,
                        void *scratch, uint32_t *err_word) {
    if (n == 0) return cudaSuccess;
    unsigned char *sc = static_cast<unsigned char *>(scratch);
    if (key_bits <= 32) return run_sort<uint32_t>(s, (const uint32_t *)keys, key_bits, n, perm, sc, err_word);
    return run_sort<uint64_t>(s, (const uint64_t *)keys, key_bits, n, perm, sc, err_word);
}

}  // namespace hcc
