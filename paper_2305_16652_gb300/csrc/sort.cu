// Stable LSD radix sort of ray ids by key (Sec. 4.2.3 "Sorting": keys are
// sorted as natural numbers; Sec. 5: the sort orders ray indices).
//
// Design (one pass per 8-bit digit, "onesweep" structure):
//   k_hist   one read of every key builds the digit histograms of all passes
//            (warp-private counters, equal digits of a warp merged with
//            match.any); the last block to finish scans them and plans the
//            passes: a pass whose digit is the same for every key is marked
//            inactive (skipping it cannot change a stable result), and the
//            ping-pong buffers are chosen so that the first active pass reads
//            the caller's keys and synthesises ids, and the last one writes
//            only the permutation
//   k_pass   per 4096-key tile: warp-level stable ranking (match.any, or a
//            ballot split when a warp's digits are spread), per-digit tile
//            counts published to a decoupled look-back chain (bounded
//            waits), keys reordered in shared memory and written out in runs
//            of equal digits (coalesced); the last launch writes the
//            identity permutation when no pass is active
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
constexpr int LOOKBACK = 4;                // predecessors read per look-back round
constexpr int MATCH_MAX_DISTINCT = 16;     // distinct digits per warp item below which match.any ranks
constexpr int HIST_BLOCK = 256;
constexpr int HIST_WARPS = HIST_BLOCK / 32;

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
    uint32_t hist_done;  // blocks of k_hist that have added their counts
    uint32_t pad[13];
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
// Highest set lane of a non-zero mask.
__device__ __forceinline__ int top_lane(uint32_t m) { return 31 - __clz(m); }

// Digit `byte` (0..7) of a key: one byte permute of the key word holding it.
__device__ __forceinline__ uint32_t digit_of(uint32_t k, uint32_t byte) { return __byte_perm(k, 0u, 0x4440u | byte); }
__device__ __forceinline__ uint32_t digit_of(uint64_t k, uint32_t byte) {
    const uint32_t w = byte >= 4 ? (uint32_t)(k >> 32) : (uint32_t)k;
    return __byte_perm(w, 0u, 0x4440u | (byte & 3u));
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

// Exclusive scan of each pass's histogram, pass activity and the buffer plan
// (run by one block of RADIX threads: the last k_hist block).
__device__ void plan_passes(SortHeader *h, int passes, uint64_t n) {
    __shared__ uint32_t s_scan[RADIX];
    __shared__ int s_trivial[MAX_PASSES];
    const int t = threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        const uint32_t c = ld_relaxed(&h->hist[p][t]);
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

// One read of all keys: the digit histograms of every pass.  Each warp reads
// runs of consecutive keys (neighbouring rays have similar keys), merges the
// lanes with equal digits with match.any and adds each group's size to its
// own shared-memory counters, so neither warps nor lanes contend.  The
// block's counters then go to the global histograms, and the last block to
// finish plans the passes.
template <typename K>
__global__ void __launch_bounds__(HIST_BLOCK) k_hist(const K *__restrict__ keys, uint64_t n, uint32_t key_bits,
                                                     int passes, SortHeader *h) {
    extern __shared__ uint32_t hsh[];  // [HIST_WARPS][passes][RADIX]
    __shared__ bool s_last;
    const int per_warp = passes * RADIX;
    for (int i = threadIdx.x; i < HIST_WARPS * per_warp; i += blockDim.x) hsh[i] = 0;
    __syncthreads();
    const K mask = key_mask<K>(key_bits);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *wh = hsh + warp * per_warp;
    constexpr int UNROLL = 4;  // keys per lane in flight
    const uint64_t gwarp = (uint64_t)blockIdx.x * HIST_WARPS + warp, nwarps = (uint64_t)gridDim.x * HIST_WARPS;
    for (uint64_t base = gwarp * (32 * UNROLL); base < n; base += nwarps * (32 * UNROLL)) {
        K kk[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const uint64_t i = base + (uint64_t)u * 32 + lane;
            kk[u] = i < n ? (keys[i] & mask) : (K)0;
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const bool valid = base + (uint64_t)u * 32 + lane < n;
#pragma unroll
            for (int p = 0; p < MAX_PASSES; ++p) {
                if (p < passes) {
                    const uint32_t d = digit_of(kk[u], (uint32_t)p);
                    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, valid ? d : 256u + lane);
                    if (valid && (int)lane == top_lane(peers)) wh[p * RADIX + d] += (uint32_t)__popc(peers);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < per_warp; i += blockDim.x) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < HIST_WARPS; ++w) c += hsh[w * per_warp + i];
        if (c) atomicAdd(&h->hist[0][0] + i, c);
    }
    // the last block to finish plans the passes
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&h->hist_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        plan_passes(h, passes, n);
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
    uint32_t wait_limit;     // status reads a tile may wait in the look-back
    uint32_t withhold_tile;  // test hook: this tile never publishes its counts
    int last_launch;         // the last pass launch writes the identity permutation if no pass is active
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
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy count elements of T from global src to shared dst with asynchronous
// copies: 16-byte chunks when the whole tile is present and src is 16-byte
// aligned, element by element otherwise.  Only elements below count are read.
template <typename T>
__device__ __forceinline__ void load_tile_async(T *dst, const T *src, uint32_t count) {
    if (count == SORT_TILE && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
        constexpr uint32_t per = 16 / sizeof(T), chunks = SORT_TILE / per;
#pragma unroll
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

// Stable rank of this thread's items within their digit in the warp's
// running count: lanes with equal digits found by match.any (or by the
// ballot split when the warp's first item shows many distinct digits), the
// highest lane of each group adds the group's size to the warp's counter and
// passes the old value to the group.  FULL: every item of the tile is valid.
template <bool FULL, typename K>
__device__ __forceinline__ void rank_items(const K (&kreg)[SORT_ITEMS], uint32_t (&rank)[SORT_ITEMS], uint32_t *wh,
                                           uint32_t byte, uint32_t dbits, uint32_t wfirst, uint32_t tile_n) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    bool use_match = true;
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        const uint32_t d = digit_of(kreg[i], byte);
        uint32_t peers;
        bool valid = true;
        if (FULL) {
            peers = use_match ? __match_any_sync(0xFFFFFFFFu, d) : digit_peers(d, dbits, 0xFFFFFFFFu);
        } else {
            valid = wfirst + (uint32_t)i * 32 < tile_n;
            const uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
            peers = use_match ? (__match_any_sync(0xFFFFFFFFu, valid ? d : 256u + lane) & vmask)
                              : digit_peers(d, dbits, vmask);
            if (!valid) peers = 0;
        }
        const int leader = valid ? top_lane(peers) : lane;
        if (i == 0)  // the first item's number of distinct digits picks the method for the rest
            use_match = __popc(__ballot_sync(0xFFFFFFFFu, valid && lane == leader)) <= MATCH_MAX_DISTINCT;
        uint32_t prior = 0;
        if (valid && lane == leader) prior = atomicAdd(&wh[d], (uint32_t)__popc(peers));
        prior = __shfl_sync(0xFFFFFFFFu, prior, leader);
        rank[i] = prior + __popc(peers & lt);
    }
}

// One digit pass.  Persistent blocks (three per SM for 32-bit keys, two for
// 64-bit keys) take tiles of 4096 keys in launch order from an atomic
// counter; while a tile is ranked and written, the next tile's keys and
// values stream into the other shared-memory buffer (cp.async), so the DRAM
// latency of a tile overlaps the work on the previous one.  Per tile: the
// warp-level stable ranking, the tile's digit counts published at once to
// the decoupled look-back chain, the tile reordered by digit in shared
// memory, the look-back for the global offsets (bounded waits with
// back-off), and runs of equal digits written out coalesced.  A block
// handles its tiles in increasing order, so the lowest unfinished tile is
// always being worked on and every wait ends.
template <typename K>
__global__ void __launch_bounds__(SORT_BLOCK, sizeof(K) == 4 ? 3 : 2) k_pass(PassArgs<K> a, int pass) {
    const PassPlan pl = a.h->plan[pass];
    if (!pl.active) {
        if (a.last_launch && a.h->identity) {  // no active pass: the permutation is the identity
            const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
            for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
                a.perm[i] = (uint32_t)i;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *in_keys = reinterpret_cast<K *>(smem_raw);                                  // [2][TILE]
    uint32_t *in_vals = reinterpret_cast<uint32_t *>(in_keys + 2 * SORT_TILE);     // [2][TILE]
    // per-warp digit counts of the tile, then each warp's first reorder slot per digit
    __shared__ uint32_t s_wofs[SORT_WARPS][RADIX];
    __shared__ uint32_t s_gofs[RADIX];  // global position of digit d's run minus its first tile slot
    __shared__ uint32_t s_wsum[SORT_WARPS];
    __shared__ uint32_t s_claim, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t byte = (uint32_t)pass;
    const uint32_t shift = 8u * (uint32_t)pass;
    const bool from_user = pl.src_keys == KB_USER;
    const K mask = key_mask<K>(a.key_bits);
    const uint32_t dbits = a.key_bits - shift < 8u ? a.key_bits - shift : 8u;
    const K *kin = from_user ? a.user_keys : (pl.src_keys == KB_A ? a.ka : a.kb);
    const uint32_t *vin = pl.src_vals == VB_A ? a.va : a.perm;
    const bool synth = pl.src_vals == VB_SYNTH;
    K *kout = pl.dst_keys == KB_A ? a.ka : (pl.dst_keys == KB_B ? a.kb : nullptr);
    uint32_t *vout = pl.dst_vals == VB_A ? a.va : a.perm;
    const uint32_t wfirst = (uint32_t)warp * (SORT_ITEMS * 32) + lane;  // tile position of this lane's item 0
    const uint32_t wait_rounds = a.wait_limit / LOOKBACK;

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
        cp_async_commit();
    };

    for (int i = tid; i < SORT_WARPS * RADIX; i += SORT_BLOCK) (&s_wofs[0][0])[i] = 0;
    if (tid == 0) {
        s_claim = atomicAdd(&a.h->tile_counter[pass], 1u);
        s_abort = 0;
    }
    __syncthreads();
    uint32_t cur = s_claim;
    __syncthreads();
    if (tid == 0) s_claim = atomicAdd(&a.h->tile_counter[pass], 1u);
    int buf = 0;
    issue(cur, buf);
    while (cur < a.num_tiles) {
        cp_async_wait_all();
        __syncthreads();  // (1) the tile's data everywhere; the previous tile fully written; s_claim visible
        const uint32_t nxt = s_claim;
        issue(nxt, buf ^ 1);  // prefetch the next tile into the other buffer

        const uint32_t tile = cur;
        const uint64_t base = (uint64_t)tile * SORT_TILE;
        const uint32_t tile_n = tile_count(tile);
        K *tk = in_keys + buf * SORT_TILE;  // the tile's keys, then (reordered) its staging area
        uint32_t *tv = in_vals + buf * SORT_TILE;
        const bool full = tile_n == SORT_TILE;

        K kreg[SORT_ITEMS];
        uint32_t vreg[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            const uint32_t pos = wfirst + (uint32_t)i * 32;
            const bool ok = full || pos < tile_n;
            const K k = ok ? tk[pos] : (K)0;
            kreg[i] = from_user ? (K)(k & mask) : k;
            vreg[i] = synth ? (uint32_t)(base + pos) : (ok ? tv[pos] : 0u);
        }
        uint32_t *wh = s_wofs[warp];
        if (full)
            rank_items<true>(kreg, rank, wh, byte, dbits, wfirst, tile_n);
        else
            rank_items<false>(kreg, rank, wh, byte, dbits, wfirst, tile_n);
        __syncthreads();  // (2) warp counts complete; every thread has read its items and nxt
        if (tid == 0) s_claim = atomicAdd(&a.h->tile_counter[pass], 1u);  // the tile after nxt
        // thread tid owns digit tid: warp offsets, tile count, publication
        uint32_t wpref[SORT_WARPS];
        uint32_t total = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            wpref[w] = total;
            total += s_wofs[w][tid];
        }
        uint32_t *st = a.status + ((size_t)pass * a.num_tiles + tile) * RADIX;
        const bool publish = tile != a.withhold_tile;
        if (publish) {
            if (tile == 0)
                st_relaxed(st + tid, ST_INC | ((a.h->start[pass][tid] + total) & ST_VALUE));
            else
                st_relaxed(st + tid, ST_AGG | total);
        }
        uint32_t incl = total;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();  // (3) per-warp sums of the digit totals
        uint32_t local = incl - total;
        for (int w = 0; w < warp; ++w) local += s_wsum[w];
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) s_wofs[w][tid] = local + wpref[w];
        __syncthreads();  // (4) reorder slots ready
        // reorder the tile by digit (stable) into its own buffer
#pragma unroll
        for (int i = 0; i < SORT_ITEMS; ++i) {
            if (full || wfirst + (uint32_t)i * 32 < tile_n) {
                const uint32_t o = wh[digit_of(kreg[i], byte)] + rank[i];
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
                    if (++spins > wait_rounds || ((spins & 63u) == 0 && ld_relaxed(&a.h->abort))) {
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
            if (publish) st_relaxed(st + tid, ST_INC | ((excl + total) & ST_VALUE));
        }
        s_gofs[tid] = excl - local;
        __syncthreads();  // (5) the tile reordered, global offsets ready
        if (s_abort) break;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) s_wofs[w][tid] = 0;  // counters of the next tile
        // runs of equal digits to their global positions
        if (kout) {
#pragma unroll 4
            for (uint32_t p = tid; p < tile_n; p += SORT_BLOCK) {
                const K k = tk[p];
                const uint32_t g = s_gofs[digit_of(k, byte)] + p;
                kout[g] = k;
                vout[g] = tv[p];
            }
        } else {
#pragma unroll 4
            for (uint32_t p = tid; p < tile_n; p += SORT_BLOCK) {
                const uint32_t g = s_gofs[digit_of(tk[p], byte)] + p;
                __stcs(vout + g, tv[p]);
            }
        }
        cur = nxt;
        buf ^= 1;
    }
    cp_async_wait_all();
}

template <typename K>
cudaError_t run_sort(cudaStream_t s, const K *keys, uint32_t key_bits, uint64_t n, uint32_t *perm,
                     unsigned char *scratch, uint32_t *err, const SortOptions &opt) {
    const Layout L = layout(n, key_bits);
    const int passes = (int)((key_bits + 7) / 8);
    const uint32_t tiles = (uint32_t)((n + SORT_TILE - 1) / SORT_TILE);
    SortHeader *h = reinterpret_cast<SortHeader *>(scratch + L.header);
    cudaError_t e = cudaMemsetAsync(scratch, 0, L.ka, s);  // header + status words
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t hblocks = (n + HIST_BLOCK * 16 - 1) / (HIST_BLOCK * 16);
    const uint64_t hcap = (uint64_t)(sms > 0 ? sms : 1) * 4;
    if (hblocks > hcap) hblocks = hcap;
    if (hblocks == 0) hblocks = 1;
    const size_t dyn = 2 * (sizeof(K) + sizeof(uint32_t)) * SORT_TILE;  // 2 tile buffers (prefetch, current)
    // the shared-memory opt-in is set once per device (so that a sort can be
    // captured in a CUDA graph without any non-stream call)
    static std::atomic<uint64_t> opted{0};
    if (dev >= 0 && dev < 64 && !(opted.load() & (1ull << dev))) {
        e = cudaFuncSetAttribute(k_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_hist<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 HIST_WARPS * MAX_PASSES * RADIX * (int)sizeof(uint32_t));
        if (e != cudaSuccess) return e;
        opted.fetch_or(1ull << dev);
    }
    const size_t hdyn = (size_t)HIST_WARPS * passes * RADIX * sizeof(uint32_t);
    k_hist<K><<<(unsigned)hblocks, HIST_BLOCK, hdyn, s>>>(keys, n, key_bits, passes, h);
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
    a.wait_limit = opt.wait_limit;
    a.withhold_tile = opt.withhold_tile;
    a.last_launch = 0;
    const uint32_t per_sm = sizeof(K) == 4 ? 3u : 2u;  // blocks that fit the shared memory
    const uint32_t grid = std::min<uint32_t>(tiles, (uint32_t)(sms > 0 ? sms : 1) * per_sm);
    for (int p = 0; p < passes; ++p) {
        a.last_launch = p == passes - 1;
        k_pass<K><<<grid, SORT_BLOCK, dyn, s>>>(a, p);
    }
    return cudaGetLastError();
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n, uint32_t key_bits) { return layout(n, key_bits).total; }

cudaError_t launch_sort(cudaStream_t s, const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm,
                        void *scratch, uint32_t *err_word, const SortOptions &opt) {
    if (n == 0) return cudaSuccess;
    unsigned char *sc = static_cast<unsigned char *>(scratch);
    if (key_bits <= 32) return run_sort<uint32_t>(s, (const uint32_t *)keys, key_bits, n, perm, sc, err_word, opt);
    return run_sort<uint64_t>(s, (const uint64_t *)keys, key_bits, n, perm, sc, err_word, opt);
}

}  // namespace hcc
