// Stable LSD radix sort of ray ids by key (Sec. 4.2.3 "Sorting": keys are
// sorted as natural numbers; Sec. 5: the sort orders ray indices).
//
// Design (one pass per 8-bit digit, "onesweep" structure):
//   k_hist   one read of every key builds the digit histograms of all passes
//            (each warp counts its most common digit in a register, the rest
//            with shared-memory atomics); the last block to finish scans them
//            and plans the
//            passes: a pass whose digit is the same for every key is marked
//            inactive (skipping it cannot change a stable result), and the
//            ping-pong buffers are chosen so that the first active pass reads
//            the caller's keys and synthesises ids, and the last one writes
//            only the permutation
//   k_pass   one block per tile of keys: warp-level stable ranking
//            (match.any, or a ballot split when a warp's digits are spread),
//            per-digit tile counts published to a decoupled look-back chain
//            (bounded waits), keys reordered in shared memory and written out
//            in runs of equal digits (coalesced); the last launch writes the
//            identity permutation when no pass is active
// Blocks take their tile from an atomic counter when they start, so a tile
// only ever waits for tiles that are already running.
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "hcc_internal.cuh"

namespace hcc {
namespace {

constexpr int RADIX = 256;
constexpr int MAX_PASSES = 8;
constexpr int SORT_BLOCK = 256;  // one thread per digit in the scan / look-back
constexpr int SORT_WARPS = SORT_BLOCK / 32;
// 14 keys per thread (3584-key tiles) and four resident blocks per SM
// measured fastest among 8-16 keys and 3-6 blocks on 16.6M ray keys
#ifndef SORT_ITEMS_PER_THREAD
#define SORT_ITEMS_PER_THREAD 14
#endif
#ifndef SORT_MIN_BLOCKS
#define SORT_MIN_BLOCKS 4
#endif
constexpr int SORT_ITEMS = SORT_ITEMS_PER_THREAD;
constexpr int SORT_TILE = SORT_BLOCK * SORT_ITEMS;
constexpr uint32_t ST_AGG = 1u << 30;  // tile count of this digit available
constexpr uint32_t ST_INC = 2u << 30;  // inclusive prefix of this digit available
constexpr uint32_t ST_VALUE = (1u << 30) - 1u;
#ifndef SORT_LOOKBACK
#define SORT_LOOKBACK 4
#endif
constexpr int LOOKBACK = SORT_LOOKBACK;    // predecessors read per look-back round
constexpr int MATCH_MAX_DISTINCT = 16;     // distinct digits per warp item below which match.any ranks
constexpr int HIST_BLOCK = 256;

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

// Buffers between passes: for 32-bit keys two ping-pong arrays of (key, id)
// pairs (8 bytes each); for 64-bit keys two key arrays and one id array (the
// permutation is the other id buffer).
Layout layout(uint64_t n, uint32_t key_bits) {
    const uint32_t passes = (key_bits + 7) / 8;
    const uint64_t tiles = (n + SORT_TILE - 1) / SORT_TILE;
    Layout L;
    L.header = 0;
    L.status = align256(sizeof(SortHeader));
    L.ka = L.status + align256((size_t)passes * tiles * RADIX * sizeof(uint32_t));
    L.kb = L.ka + align256(n * 8);
    L.va = L.kb + align256(n * 8);
    L.total = L.va + (key_bits > 32 ? align256(n * sizeof(uint32_t)) : 0);
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

// One read of all keys: the digit histograms of every pass.  Keys of ray
// batches are heavily skewed (one digit value often holds most keys), so
// each warp first picks the most common digit of its first 32 keys for each
// pass and counts that value in a register; every other digit goes to a
// shared-memory add (predicated, not branched around).  Threads read 16
// bytes of keys at a time (VEC keys) where the keys are 16-byte aligned; the
// last n % VEC keys are read one at a time.  The block's counts then go to the
// global histograms, and the last block to finish plans the passes.
template <typename K, int P>
__device__ __forceinline__ void hist_key(K k, const uint32_t (&dom)[P], uint32_t (&cnt)[P], uint32_t sh) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const uint32_t d = digit_of(k, (uint32_t)p);
        cnt[p] += d == dom[p] ? 1u : 0u;
        // a predicated shared-memory add for the other digits, no branch
        asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, %1;\n\t@q red.shared.add.u32 [%2], 1;\n\t}" ::"r"(d),
                     "r"(dom[p]), "r"(sh + (uint32_t)(p * RADIX + d) * 4u)
                     : "memory");
    }
}

// P: the number of digit passes (a template argument, so that the per-key
// loop has no pass test).
template <typename K, int VEC, int P>
__global__ void __launch_bounds__(HIST_BLOCK) k_hist(const K *__restrict__ keys, uint64_t n, uint32_t key_bits,
                                                     SortHeader *h) {
    __shared__ uint32_t sh[MAX_PASSES * RADIX];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < P * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const K mask = key_mask<K>(key_bits);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // dominant digit per pass among the warp's first keys
    const K k0 = first < n ? (keys[first] & mask) : (K)0;
    uint32_t dom[P], cnt[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        cnt[p] = 0;
        const uint32_t d = digit_of(k0, (uint32_t)p);
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, first < n ? d : 256u + lane);
        uint32_t best = ((uint32_t)__popc(peers) << 9) | d;
        best = __reduce_max_sync(0xFFFFFFFFu, best);
        dom[p] = best & 511u;
    }
    constexpr int UNROLL = 4;  // independent 16-byte loads in flight per thread
    using V = typename std::conditional<VEC == 1, K, uint4>::type;
    const V *kv = reinterpret_cast<const V *>(keys);
    const uint32_t shb = (uint32_t)__cvta_generic_to_shared(sh);
    const uint64_t nv = n / VEC;  // whole vectors; the last n % VEC keys follow one at a time
    for (uint64_t base = first; base < nv; base += UNROLL * stride) {
        V x[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const uint64_t v = base + (uint64_t)u * stride;
            x[u] = v < nv ? kv[v] : V{};
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (base + (uint64_t)u * stride >= nv) break;
            if constexpr (VEC == 1) {
                hist_key<K, P>(x[u] & mask, dom, cnt, shb);
            } else if constexpr (sizeof(K) == 4) {
                hist_key<K, P>((K)x[u].x & mask, dom, cnt, shb);
                hist_key<K, P>((K)x[u].y & mask, dom, cnt, shb);
                hist_key<K, P>((K)x[u].z & mask, dom, cnt, shb);
                hist_key<K, P>((K)x[u].w & mask, dom, cnt, shb);
            } else {
                hist_key<K, P>((((K)x[u].y << 32) | x[u].x) & mask, dom, cnt, shb);
                hist_key<K, P>((((K)x[u].w << 32) | x[u].z) & mask, dom, cnt, shb);
            }
        }
    }
    for (uint64_t i = nv * VEC + first; i < n; i += stride) hist_key<K, P>(keys[i] & mask, dom, cnt, shb);
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, cnt[p]);
        if (lane == 0 && c && dom[p] < 256u) atomicAdd(&sh[p * RADIX + dom[p]], c);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&h->hist[0][0] + i, sh[i]);
    // the last block to finish plans the passes
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&h->hist_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) {
        __threadfence();
        plan_passes(h, P, n);
    }
}

// The histogram kernel for `passes` digit passes (1-4 for 32-bit keys, 5-8
// for 64-bit keys) and the keys' alignment.
template <typename K, int VEC>
void launch_hist(cudaStream_t s, unsigned blocks, const K *keys, uint64_t n, uint32_t key_bits, int passes,
                 SortHeader *h) {
    constexpr int LO = sizeof(K) == 4 ? 1 : 5;
    switch (passes - LO) {
        case 0: k_hist<K, VEC, LO><<<blocks, HIST_BLOCK, 0, s>>>(keys, n, key_bits, h); break;
        case 1: k_hist<K, VEC, LO + 1><<<blocks, HIST_BLOCK, 0, s>>>(keys, n, key_bits, h); break;
        case 2: k_hist<K, VEC, LO + 2><<<blocks, HIST_BLOCK, 0, s>>>(keys, n, key_bits, h); break;
        default: k_hist<K, VEC, LO + 3><<<blocks, HIST_BLOCK, 0, s>>>(keys, n, key_bits, h); break;
    }
}

template <typename K>
struct PassArgs {
    const K *user_keys;
    void *buf_a, *buf_b;  // between passes: (key, id) pairs for 32-bit keys, keys for 64-bit keys
    uint32_t *va;         // ids between passes (64-bit keys)
    uint32_t *perm;
    uint32_t *status;
    SortHeader *h;
    uint64_t n;
    uint32_t key_bits, num_tiles;
    uint32_t *err;
    uint32_t wait_limit;     // status reads a tile may wait in the look-back
    uint32_t withhold_tile;  // test hook: this tile never publishes its counts
    int last_launch;         // the last pass launch writes the identity permutation if no pass is active
};

// Decoupled look-back for digit d of tile `tile`: the sum of the digit's
// counts in all earlier tiles, read from their status words newest first
// (LOOKBACK per round) until an inclusive prefix is found.  Each wait is
// bounded: after wait_limit status reads without progress (or once another
// tile has given up) it records a timeout and returns.
template <typename K>
__device__ __forceinline__ uint32_t look_back(const PassArgs<K> &a, int pass, uint32_t tile, uint32_t d,
                                              bool &timed_out) {
    uint32_t excl = 0;
    int64_t j = (int64_t)tile - 1;
    uint32_t spins = 0;
    bool done = false;
    const uint32_t wait_rounds = a.wait_limit / LOOKBACK;
    const uint32_t *col = a.status + (size_t)pass * a.num_tiles * RADIX + d;
    while (!done) {
        uint32_t sv[LOOKBACK];
#pragma unroll
        for (int w = 0; w < LOOKBACK; ++w) sv[w] = (j - w >= 0) ? ld_relaxed(col + (size_t)(j - w) * RADIX) : ST_INC;
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
                atomicOr(a.err, ERR_TIMEOUT);
                atomicExch(&a.h->abort, 1u);
                break;
            }
            __nanosleep(spins < 8 ? 32u * spins : 256u);
        }
    }
    return excl;
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

// One digit pass, one block per tile of SORT_TILE keys.  A block takes its tile
// from an atomic counter when it starts, so tiles are worked on in the order
// blocks start and a tile's predecessors are already running when it looks
// back.  Per tile: each thread loads its 16 items (a warp reads 32
// consecutive elements per item), the warp-level stable ranking, the tile's
// digit counts published at once to the decoupled look-back chain, the tile
// reordered by digit in shared memory, the look-back for the global offsets
// (bounded waits with back-off), and runs of equal digits written out
// coalesced.  32-bit keys travel between passes as (key, id) pairs, so an
// element moves with one 8-byte access; 64-bit keys as separate key and id
// arrays.
template <typename K>
__global__ void __launch_bounds__(SORT_BLOCK, sizeof(K) == 4 ? SORT_MIN_BLOCKS : 2) k_pass(PassArgs<K> a, int pass) {
    constexpr bool PAIRS = sizeof(K) == 4;
    const PassPlan pl = a.h->plan[pass];
    if (!pl.active) {
        if (a.last_launch && a.h->identity) {  // no active pass: the permutation is the identity
            const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
            for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
                a.perm[i] = (uint32_t)i;
        }
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];     // the tile, reordered
    uint2 *tp = reinterpret_cast<uint2 *>(smem_raw);              // pairs (32-bit keys), and ...
    uint32_t *tvs = reinterpret_cast<uint32_t *>(tp + SORT_TILE);  // ... their ids in input order
    K *tk = reinterpret_cast<K *>(smem_raw);                      // keys (64-bit keys) ...
    uint32_t *tv = reinterpret_cast<uint32_t *>(tk + SORT_TILE);  // ... and their ids
    // per-warp digit counts of the tile, then each warp's first reorder slot per digit
    __shared__ uint32_t s_wofs[SORT_WARPS][RADIX];
    __shared__ uint32_t s_gofs[RADIX];  // global position of digit d's run minus its first tile slot
    __shared__ uint32_t s_wsum[SORT_WARPS];
    __shared__ uint32_t s_tile, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t byte = (uint32_t)pass;
    const uint32_t shift = 8u * (uint32_t)pass;
    const bool from_user = pl.src_keys == KB_USER;
    const K mask = key_mask<K>(a.key_bits);
    const uint32_t dbits = a.key_bits - shift < 8u ? a.key_bits - shift : 8u;
    const void *bin = pl.src_keys == KB_A ? a.buf_a : a.buf_b;
    void *bout = pl.dst_keys == KB_A ? a.buf_a : (pl.dst_keys == KB_B ? a.buf_b : nullptr);
    const uint32_t wfirst = (uint32_t)warp * (SORT_ITEMS * 32) + lane;  // tile position of this lane's item 0

#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) s_wofs[w][tid] = 0;
    if (tid == 0) {
        s_tile = atomicAdd(&a.h->tile_counter[pass], 1u);
        s_abort = 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= a.num_tiles) return;  // uniform; the grid has one block per tile, so this never happens
    const uint64_t base = (uint64_t)tile * SORT_TILE;
    const uint32_t tile_n = (uint32_t)((a.n - base) < (uint64_t)SORT_TILE ? (a.n - base) : SORT_TILE);
    const bool full = tile_n == SORT_TILE;

    K kreg[SORT_ITEMS];
    uint32_t vreg[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        const uint32_t pos = wfirst + (uint32_t)i * 32;
        const bool ok = full || pos < tile_n;
        const uint64_t g = base + pos;
        if (from_user) {
            kreg[i] = ok ? (K)(a.user_keys[g] & mask) : (K)0;
            if (!PAIRS) vreg[i] = (uint32_t)g;
        } else if (PAIRS) {  // the id waits in shared memory, not in a register, until the reorder
            const uint2 e = ok ? static_cast<const uint2 *>(bin)[g] : make_uint2(0u, 0u);
            kreg[i] = (K)e.x;
            if (ok) tvs[pos] = e.y;
        } else {
            kreg[i] = ok ? static_cast<const K *>(bin)[g] : (K)0;
            vreg[i] = ok ? (pl.src_vals == VB_A ? a.va : a.perm)[g] : 0u;
        }
    }
    uint32_t *wh = s_wofs[warp];
    if (full)
        rank_items<true>(kreg, rank, wh, byte, dbits, wfirst, tile_n);
    else
        rank_items<false>(kreg, rank, wh, byte, dbits, wfirst, tile_n);
    __syncthreads();  // (1) warp counts complete
    // thread tid owns digit tid: warp offsets, tile count, publication
    uint32_t total = 0;  // the counts become each warp's offset within the digit, in place
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) {
        const uint32_t c = s_wofs[w][tid];
        s_wofs[w][tid] = total;
        total += c;
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
    __syncthreads();  // (2) per-warp sums of the digit totals
    uint32_t local = incl - total;
    for (int w = 0; w < warp; ++w) local += s_wsum[w];
#pragma unroll
    for (int w = 0; w < SORT_WARPS; ++w) s_wofs[w][tid] += local;
    __syncthreads();  // (3) reorder slots ready
    // reorder the tile by digit (stable)
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; ++i) {
        if (full || wfirst + (uint32_t)i * 32 < tile_n) {
            const uint32_t o = wh[digit_of(kreg[i], byte)] + rank[i];
            if (PAIRS) {
                const uint32_t pos = wfirst + (uint32_t)i * 32;
                tp[o] = make_uint2((uint32_t)kreg[i], from_user ? (uint32_t)(base + pos) : tvs[pos]);
            } else {
                tk[o] = kreg[i];
                tv[o] = vreg[i];
            }
        }
    }
    // decoupled look-back for digit tid
    uint32_t excl;
    if (tile == 0) {
        excl = a.h->start[pass][tid];
    } else {
        bool timed_out = false;
        excl = look_back(a, pass, tile, tid, timed_out);
        if (timed_out) s_abort = 1;
        if (publish) st_relaxed(st + tid, ST_INC | ((excl + total) & ST_VALUE));
    }
    s_gofs[tid] = excl - local;
    __syncthreads();  // (4) the tile reordered, global offsets ready
    if (s_abort) return;
    // runs of equal digits to their global positions
    if (PAIRS) {
        if (bout) {
            uint2 *out = static_cast<uint2 *>(bout);
#pragma unroll 4
            for (uint32_t p = tid; p < tile_n; p += SORT_BLOCK) {
                const uint2 e = tp[p];
                out[s_gofs[digit_of(e.x, byte)] + p] = e;
            }
        } else {
#pragma unroll 4
            for (uint32_t p = tid; p < tile_n; p += SORT_BLOCK) {
                const uint2 e = tp[p];
                a.perm[s_gofs[digit_of(e.x, byte)] + p] = e.y;
            }
        }
    } else {
        K *kout = static_cast<K *>(bout);
        uint32_t *vout = pl.dst_vals == VB_A ? a.va : a.perm;
#pragma unroll 4
        for (uint32_t p = tid; p < tile_n; p += SORT_BLOCK) {
            const K k = tk[p];
            const uint32_t g = s_gofs[digit_of(k, byte)] + p;
            if (kout) kout[g] = k;
            vout[g] = tv[p];
        }
    }
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
    uint64_t hblocks = (n + HIST_BLOCK * 8 - 1) / (HIST_BLOCK * 8);
    const uint64_t hcap = (uint64_t)(sms > 0 ? sms : 1) * 4;
    if (hblocks > hcap) hblocks = hcap;
    if (hblocks == 0) hblocks = 1;
    const size_t dyn = (sizeof(K) == 4 ? sizeof(uint2) : sizeof(K)) * SORT_TILE + sizeof(uint32_t) * SORT_TILE;
    // the shared-memory opt-in is set once per device (so that a sort can be
    // captured in a CUDA graph without any non-stream call)
    static std::atomic<uint64_t> opted{0};
    if (dev >= 0 && dev < 64 && !(opted.load() & (1ull << dev))) {
        e = cudaFuncSetAttribute(k_pass<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
        opted.fetch_or(1ull << dev);
    }
    if ((reinterpret_cast<uintptr_t>(keys) & 15u) == 0)
        launch_hist<K, 16 / sizeof(K)>(s, (unsigned)hblocks, keys, n, key_bits, passes, h);
    else
        launch_hist<K, 1>(s, (unsigned)hblocks, keys, n, key_bits, passes, h);
    PassArgs<K> a;
    a.user_keys = keys;
    a.buf_a = scratch + L.ka;
    a.buf_b = scratch + L.kb;
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
    for (int p = 0; p < passes; ++p) {
        a.last_launch = p == passes - 1;
        k_pass<K><<<tiles, SORT_BLOCK, dyn, s>>>(a, p);
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
