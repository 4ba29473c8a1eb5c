/*
 * hcc.h -- C ABI of the GB300 hierarchy-cut-code ray-reordering library.
 *
 * The library implements the reordering hot path of Xiang et al., "Faster
 * Ray Tracing through Hierarchy Cut Code" (arXiv 2305.16652), Sec. 4.2 and
 * Sec. 5: a cut of the BVH is chosen once per scene (Algorithm 2, Eq. 1),
 * every ray gets a key from its intersections with the cut nodes
 * (Algorithm 1), ray indices are sorted by key, the rays are fetched in
 * sorted order and traced.  The paper's NoSort and TwoPoint baselines run
 * behind the same calls.  Every step runs in hand-written CUDA kernels for
 * sm_103a except cut selection, which the paper also performs once per scene
 * on the host.
 *
 * Conventions shared by every call
 *   - Status: every call returns an hcc_status; HCC_OK is 0.  Argument
 *     errors are reported before anything is launched or written.  No call
 *     aborts the process or throws across the ABI.
 *   - Memory: ray, key, permutation and hit buffers are allocated by the
 *     caller on the context's device and passed as plain device pointers;
 *     the library never frees them.  Opaque handles (context, BVH, cut) are
 *     owned by the library and released by their *_destroy call.  The
 *     context owns its scratch memory (sort buffers, error word).
 *   - Execution: calls that take device buffers are asynchronous on the
 *     context's CUDA stream.  Errors found by kernels (traversal-stack
 *     overflow, a bounded wait that gave up) are recorded in a device error
 *     word and returned by the next hcc_sync.
 *   - Threads: a context must not be used by two host threads at once; use
 *     one context per host thread or stream.  BVH and cut handles are
 *     read-only after creation and may be shared by contexts on the same
 *     device.
 *   - Sizes: n = 0 is a valid no-op everywhere.
 */
#ifndef HCC_H
#define HCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hcc_status {
    HCC_OK = 0,
    HCC_ERR_INVALID_ARG = 1,    /* null pointer, bad size, misaligned buffer, bad enum */
    HCC_ERR_OOM = 2,            /* device or host allocation failed */
    HCC_ERR_CUDA = 3,           /* a CUDA runtime call failed; see hcc_last_error */
    HCC_ERR_UNSUPPORTED = 4,    /* valid request this library does not implement */
    HCC_ERR_STACK_OVERFLOW = 5, /* a ray needed more traversal-stack entries than exist */
    HCC_ERR_TIMEOUT = 6         /* a bounded device-side wait gave up */
} hcc_status;

/* Ray-ordering methods (Sec. 5 and Table 1 of the paper). */
typedef enum hcc_method {
    HCC_METHOD_NOSORT = 0,    /* trace in generation order (Table 1, NoSort) */
    HCC_METHOD_HCC = 1,       /* hierarchy cut code (Sec. 4.2) */
    HCC_METHOD_TWOPOINT = 2,  /* origin + estimated termination Morton code (Sec. 3.2, Sec. 5) */
    HCC_METHOD_ORIGIN = 3,    /* Morton code of the origin (Sec. 3.2 "Origin", Table 1) */
    HCC_METHOD_ORIGIN_DIR = 4, /* origin Morton above direction Morton (Sec. 3.2 "Origin-Direction") */
    HCC_METHOD_PPC = 5,        /* prefix path code (Sec. 4.1), an upper bound */
    HCC_METHOD_MLHCC = 6       /* multi-level hierarchy cut code (Sec. 4.3) */
} hcc_method;

typedef struct hcc_ctx hcc_ctx; /* device, stream, scratch, device error word */
typedef struct hcc_bvh hcc_bvh; /* device copy of a BVH2: quantised nodes, triangles */
typedef struct hcc_cut hcc_cut; /* cut nodes in key order and their exact boxes */

/*
 * A BVH2 on the host (Sec. 3.1), read only during hcc_bvh_upload.
 * Nodes are numbered so that node 0 is the root.  left[i] < 0 (and
 * right[i] < 0) marks a leaf that owns order[first[i] .. first[i]+count[i]),
 * 1 <= count <= 4; otherwise left/right are child node ids.  lo/hi: the
 * node's axis-aligned box, 3 floats each, which must contain the node's
 * triangles.  tris: num_tris triangles as 9 floats (v0, v1, v2); order holds
 * triangle ids (indices into tris); hits report these ids.
 */
typedef struct hcc_bvh_desc {
    uint32_t num_nodes;
    const float *lo;       /* [num_nodes * 3] */
    const float *hi;       /* [num_nodes * 3] */
    const int32_t *left;   /* [num_nodes] */
    const int32_t *right;  /* [num_nodes] */
    const uint32_t *first; /* [num_nodes] */
    const uint32_t *count; /* [num_nodes] */
    uint32_t num_tris;
    const float *tris;     /* [num_tris * 9] */
    const uint32_t *order; /* [num_tris] */
} hcc_bvh_desc;

/*
 * n rays on the device as two float4 streams, each 16-byte aligned:
 * org_tmin[i] = (ox, oy, oz, tmin), dir_tmax[i] = (dx, dy, dz, tmax).  A ray
 * covers the parameter interval [tmin, tmax]; tmax = +inf for an unbounded
 * ray.  Directions need not be normalised.
 * stride: bytes from ray i to ray i + 1 in each stream, a multiple of 16
 * (0 means 16).  16 = two packed float4 arrays (structure of arrays); 32
 * with dir_tmax = org_tmin + 4 = one 32-byte record per ray (origin, then
 * direction), which a fetch through a permutation reads as one 32-byte
 * access instead of two 16-byte ones.  Every call that takes rays accepts
 * any stride; outputs of hcc_gather and hcc_batch_spawn are written with
 * their own descriptor's stride.
 */
typedef struct hcc_rays {
    float *org_tmin;
    float *dir_tmax;
    uint64_t n;
    uint64_t stride;
} hcc_rays;

/* One hit record (16 bytes): prim = triangle id or -1 for a miss (then t =
 * +inf); u, v are the barycentric coordinates of the hit on (v0, v1, v2). */
typedef struct hcc_hit {
    int32_t prim;
    float t, u, v;
} hcc_hit;

/* Largest ray count a single sort accepts (the look-back counters are 30-bit). */
#define HCC_MAX_SORT_N ((uint64_t)((1u << 30) - 1u))
/* Traversal-stack entries per ray in hcc_trace. */
#define HCC_TRACE_STACK 64

/* ------------------------------------------------------------- context */

/* Create a context on CUDA device `device` issuing work on `stream` (a
 * cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: INVALID_ARG (out NULL, bad device), CUDA, OOM. */
hcc_status hcc_create(hcc_ctx **out, int device, void *stream);

/* Release the context and its scratch after waiting for its stream. */
hcc_status hcc_destroy(hcc_ctx *ctx);

/* Replace the stream used by later calls. */
hcc_status hcc_set_stream(hcc_ctx *ctx, void *stream);

/* Pre-allocate sort and pipeline scratch for up to max_n rays and keys of
 * up to max_key_bits bits, so that later calls allocate nothing.  Calls that
 * need more scratch than reserved grow it themselves (a synchronising
 * cudaMalloc).  Errors: INVALID_ARG, OOM. */
hcc_status hcc_reserve(hcc_ctx *ctx, uint64_t max_n, uint32_t max_key_bits);

/*
 * How the context's traces schedule rays on warps.  PER_RAY: one thread per
 * ray slot for the whole traversal (the plain tracer).  REFILL: persistent
 * warps take ray slots from a counter in increasing order, and after each
 * traversal round the lanes whose ray has finished take new slots once 12
 * lanes of the warp are idle (24 when the rays are fetched through a sorted
 * permutation) (Aila & Laine 2009, "replacing terminated rays").  AUTO (the
 * default): REFILL for closest-hit traces, PER_RAY for any-hit traces
 * (measured faster for each on GB300).  Results do not depend
 * on the schedule, except which hit an any-hit query reports.
 */
typedef enum hcc_trace_schedule {
    HCC_TRACE_AUTO = 0,
    HCC_TRACE_PER_RAY = 1,
    HCC_TRACE_REFILL = 2
} hcc_trace_schedule;

hcc_status hcc_set_trace_schedule(hcc_ctx *ctx, hcc_trace_schedule schedule);

/*
 * Shape of the context's closest-hit traces that use ray replacement
 * (REFILL, and AUTO for closest hit), single wavefronts and batches: threads
 * per block (64, 128 or 256) and traversal-stack entries per ray (32, 48 or
 * 64).  The paper fixes neither (its tracer follows Aila & Laine 2009); the
 * autotuner picks them by measurement.  A ray whose traversal needs more
 * stack entries than the shape has is reported as HCC_ERR_STACK_OVERFLOW by
 * hcc_sync (its record is a miss): a binary layout needs at most the BVH's
 * depth (hcc_bvh_info), the 4-ary layout up to three entries per 4-ary
 * level.  Results do not depend on the shape otherwise.  (0, 0) restores
 * the default (128, HCC_TRACE_STACK).  Errors: INVALID_ARG for any other
 * pair.
 */
hcc_status hcc_set_trace_shape(hcc_ctx *ctx, uint32_t block_threads, uint32_t stack_entries);

/* The TwoPoint key's estimated ray length as a fraction of the root box's
 * largest extent (App. B sweeps it; Sec. 5 and the default use 0.25), for
 * this context's hcc_encode and hcc_run.  Batches and servers use 0.25.
 * Errors: INVALID_ARG (negative or not finite). */
hcc_status hcc_set_twopoint_distance(hcc_ctx *ctx, float fraction);

/* Bound on the decoupled look-back wait of this context's sorts (Sec. 4.2.3
 * sort; the bound is this library's failure detection): a tile that has
 * read its predecessors' status words status_reads times without finding
 * their counts gives up, marks the sort aborted (so no other tile waits
 * long) and hcc_sync reports HCC_ERR_TIMEOUT; the permutation is then
 * unspecified and the next sort starts afresh.  0 restores the default of
 * 2^22 reads (with back-off, about a quarter of a second), which a sort
 * whose blocks all make progress never reaches. */
hcc_status hcc_set_sort_wait_limit(hcc_ctx *ctx, uint32_t status_reads);

/* Test hook for the bounded wait above (no counterpart in the paper): while
 * set, tile number `tile` (3584 keys each) of every digit pass of this
 * context's sorts never publishes its counts, so the tile after it waits
 * until its limit and the sort reports HCC_ERR_TIMEOUT.  0xFFFFFFFF (the
 * default) withholds nothing.  Never needed outside tests. */
hcc_status hcc_test_sort_withhold_tile(hcc_ctx *ctx, uint32_t tile);

/* Wait for all work queued on the context's stream, then read and clear the
 * device error word: STACK_OVERFLOW or TIMEOUT if a kernel reported one
 * since the last hcc_sync, INVALID_ARG if a gather or scatter met an index
 * out of range, CUDA if the stream failed, else OK. */
hcc_status hcc_sync(hcc_ctx *ctx);

/* Text of the last error recorded on this context ("" if none).  The
 * string is owned by the context and valid until its next call. */
const char *hcc_last_error(const hcc_ctx *ctx);

/* Static name of a status code. */
const char *hcc_status_string(hcc_status s);

/* ----------------------------------------------------------------- BVH */

/* Copy a host BVH2 to the device in the traversal layout: every internal
 * node becomes one 32-byte record holding both children's boxes quantised
 * to 8 bits per bound and rounded outward (a superset of each exact box),
 * triangles become (v0, v1 - v0, v2 - v0) records.  The exact boxes are kept
 * on the host for cut selection.  Synchronous.  Errors: INVALID_ARG
 * (malformed tree, leaf count outside 1..4, ids out of range), OOM, CUDA. */
hcc_status hcc_bvh_upload(hcc_ctx *ctx, const hcc_bvh_desc *desc, hcc_bvh **out);

/* Device layouts of the BVH's internal nodes (each node holds both
 * children's boxes and references). */
typedef enum hcc_bvh_layout {
    HCC_BVH_QUANTISED = 0, /* 32 bytes: 8-bit child bounds on a per-node power-of-two grid, rounded outward */
    HCC_BVH_EXACT = 1,     /* 64 bytes: the children's exact FP32 boxes */
    HCC_BVH_WIDE = 2       /* 128 bytes: a 4-ary node collapsed from the BVH2 (each internal child with
                              the largest surface area replaced by its two children until four are
                              held), the children's exact FP32 boxes as rows of four per bound */
} hcc_bvh_layout;

/* hcc_bvh_upload with a choice of node layout.  Every layout gives the same
 * hits (boxes only decide which triangles are tested, and every box holds
 * the exact box of its BVH2 node); the quantised one halves node memory, the
 * exact one avoids decoding work per node visit, and the wide one visits
 * about half as many nodes per ray.  Cuts are always chosen on the BVH2.
 * Errors: as hcc_bvh_upload, plus INVALID_ARG for an unknown layout. */
hcc_status hcc_bvh_upload_layout(hcc_ctx *ctx, const hcc_bvh_desc *desc, hcc_bvh_layout layout, hcc_bvh **out);

/* Node and triangle counts, tree depth (root = 0) and the root box. Any
 * output pointer may be NULL. */
hcc_status hcc_bvh_info(const hcc_bvh *bvh, uint32_t *num_nodes, uint32_t *num_tris, uint32_t *depth,
                        float *scene_lo3, float *scene_hi3);

hcc_status hcc_bvh_destroy(hcc_bvh *bvh);

/* -------------------------------------------------------- cut selection */

/*
 * Choose the cut (Sec. 4.2.2): compute the hierarchically accumulated
 * density of every node (Eq. 1: TC * SA for a leaf, HAD_left + HAD_right +
 * lambda * SA otherwise, in double), run the priority-queue search of
 * Algorithm 2 with MaxQueueSize = cut_size (a popped leaf joins the cut and
 * lowers MaxQueueSize by one), and order the cut by HAD, descending, ties by
 * lower node id.  Cut node r drives key bit (key_bits - 1 - r) in hcc_encode.
 * If the tree has fewer leaves than cut_size the cut is every leaf.  Runs on
 * the host (once per scene, as in the paper) and copies the cut's exact
 * boxes to the device.  The paper uses lambda = 0.125.
 * Errors: INVALID_ARG (cut_size 0, lambda negative or not finite), OOM, CUDA.
 */
hcc_status hcc_select_cut(hcc_ctx *ctx, const hcc_bvh *bvh, uint32_t cut_size, double lambda, hcc_cut **out);

/* Actual cut size and, if node_ids is not NULL, the cut's node ids in key
 * order (node_ids must hold *size entries; call once with NULL to size it). */
hcc_status hcc_cut_info(const hcc_cut *cut, uint32_t *size, int32_t *node_ids);

hcc_status hcc_cut_destroy(hcc_cut *cut);

/*
 * The two-level cut of the multi-level hierarchy cut code (Sec. 4.3,
 * Algorithm 3).  A node may be a top-level node only if its subtree holds at
 * least low_size leaves (Algorithm 3 discards the others, so that no
 * low-level node is empty).  The top level runs the queue of Algorithm 2 on
 * such nodes: pop the largest-HAD node, push its children that qualify (a
 * child that does not is discarded with its subtree); a node with no
 * qualifying child joins the cut as a leaf does in Algorithm 2; stop at
 * top_size nodes.  Each top node r then gets the Algorithm 2 cut of its own
 * subtree with low_size nodes.  Both levels are ordered by HAD, descending.
 * The result has between 0 and top_size top nodes (0 when the root has fewer
 * than low_size leaves: every key is then 0), each with exactly low_size
 * low-level nodes; hcc_cut_info reports the top level.
 * Errors: INVALID_ARG (a size 0, top_size + low_size > 64, lambda negative
 * or not finite), OOM, CUDA.
 */
hcc_status hcc_select_cut_ml(hcc_ctx *ctx, const hcc_bvh *bvh, uint32_t top_size, uint32_t low_size, double lambda,
                             hcc_cut **out);

/* Two-level cut sizes: *ntop top nodes, the field widths top_size and
 * low_size it was made with, and (if low_ids is not NULL, ntop * low_size
 * entries) the low-level node ids, row r for top node r.  INVALID_ARG for a
 * one-level cut. */
hcc_status hcc_cut_ml_info(const hcc_cut *cut, uint32_t *ntop, uint32_t *top_size, uint32_t *low_size,
                           int32_t *low_ids);

/*
 * Regular grid encoding (Sec. 5): a "cut" of grid cells that divide the
 * BVH's root box evenly, for hcc_encode(HCC).  The cell count is the largest
 * power of two not above max_cells; starting from one cell, the axis whose
 * cells are longest (the first such axis on ties) is halved until that count
 * is reached.  Boundary i of g along an axis is ((g - i) lo + i hi) / g in
 * double, rounded to float, so neighbouring cells share their faces exactly.
 * Cell (i, j, l) is cut node (i gy + j) gz + l.  hcc_cut_info reports the
 * cell count and node ids of -1.  Errors: INVALID_ARG (max_cells not in
 * 1..64), OOM, CUDA.
 */
hcc_status hcc_select_grid(hcc_ctx *ctx, const hcc_bvh *bvh, uint32_t max_cells, hcc_cut **out);

/* Host copy of the boxes behind the key bits (the top level of a two-level
 * cut): lo and hi receive 3 floats per node, min(cut size, 64) nodes. */
hcc_status hcc_cut_boxes(const hcc_cut *cut, float *lo, float *hi);

/* ---------------------------------------------------------------- encode */

/*
 * One sort key per ray.  keys: n uint32_t if key_bits <= 32, else n
 * uint64_t (device, aligned to its type); the key occupies the low key_bits
 * bits, higher bits are 0.  key_bits in 1..64.
 *   HCC (Algorithm 1): bit (key_bits - 1 - r) = [the ray meets cut node r's
 *     box on [tmin, tmax]] for r < min(cut size, key_bits); other bits 0.
 *     Slab test per axis t = (bound - o) * (1 / d) in IEEE float, inclusive
 *     (tnear <= tfar).  Requires cut; bvh may be NULL.
 *   TWOPOINT (Sec. 3.2, Sec. 5): origin and estimated termination point
 *     o + L d, L = 0.25 * largest extent of the root box, each normalised to
 *     the root box and quantised to floor(key_bits / 6) bits, interleaved
 *     most significant level first in the order o.x o.y o.z t.x t.y t.z and
 *     left-justified in key_bits.  Requires bvh; cut may be NULL.
 *   ORIGIN (Sec. 3.2): origin normalised to the root box, floor(k/3) bits
 *     per axis, Morton-interleaved x y z most significant level first,
 *     left-justified.  Requires bvh.
 *   ORIGIN_DIR (Sec. 3.2, after Reis et al.): origin Morton code with
 *     bo = floor((k - 2 bd)/3) bits per axis in the high bits, then a Morton
 *     code (u, v) of the octahedral map of the direction (L1-normalise, fold
 *     z < 0 over the diagonals, map [-1, 1] to [0, 1]) with bd = floor(k/6)
 *     bits per coordinate, left-justified.  Requires bvh.
 *   MLHCC (Sec. 4.3): with a cut from hcc_select_cut_ml of field widths T
 *     and L (T + L <= key_bits): bit (key_bits - 1 - r) = the ray meets top
 *     node r; the representative is the first top node in HAD order that it
 *     meets, and bit (key_bits - 1 - T - j) = the ray meets low-level node j
 *     of the representative.  No top node met: the low field is 0.  The
 *     slab test is HCC's.  Requires a two-level cut.
 *   PPC (Sec. 4.1): the results of the first key_bits box tests of a
 *     depth-first, left-child-first traversal that does not depend on the
 *     ray (a met internal node is entered, a missed node's subtree skipped,
 *     hits never cut it short); test m drives bit (key_bits - 1 - m), bits
 *     after the traversal ends are 0.  HCC's slab test on the exact boxes.
 *     Requires a bvh uploaded with HCC_BVH_EXACT (UNSUPPORTED otherwise).
 *   NOSORT: INVALID_ARG (nothing to encode).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 */
hcc_status hcc_encode(hcc_ctx *ctx, hcc_method method, const hcc_bvh *bvh, const hcc_cut *cut,
                      const hcc_rays *rays, uint32_t key_bits, void *keys);

/*
 * Diagnostic (not on the timed path): statistics of keys in sorted order,
 * i.e. of keys[perm[j]], j = 0..n-1, which must be ascending.  *distinct =
 * number of different keys; *anc = average number of different codes per
 * warp, the groups of 32 consecutive sorted rays (Sec. 6.5, Table 6).
 * Waits for the stream; outputs are valid on return.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
hcc_status hcc_key_stats(hcc_ctx *ctx, const void *keys, uint32_t key_bits, const uint32_t *perm, uint64_t n,
                         double *anc, uint64_t *distinct);

/* ------------------------------------------------------------------ sort */

/*
 * Stable ascending sort of ray ids 0..n-1 by the low key_bits bits of keys
 * (Sec. 4.2.3 "Sorting": keys sorted as natural numbers; Sec. 5: the sort
 * orders ray indices).  perm[j] = id of the j-th ray in sorted order.
 * keys: n uint32_t (key_bits <= 32) or uint64_t (key_bits > 32), device,
 * not modified.  perm: n uint32_t, device, must not overlap keys.
 * LSD radix sort, 8-bit digits; digits that are equal for every key are
 * skipped, which leaves the result unchanged.  Scratch comes from the
 * context (see hcc_reserve).  n <= HCC_MAX_SORT_N.
 * Errors: INVALID_ARG, OOM, CUDA; TIMEOUT at hcc_sync if a bounded
 * inter-block wait gave up (perm is then unspecified).
 */
hcc_status hcc_sort(hcc_ctx *ctx, const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm);

/*
 * hcc_sort without a context and without allocating anything, for callers
 * that cannot let a library allocate device memory: programs whose device
 * memory is reserved up front by their own allocator, and latency-bound
 * loops that cannot take the device synchronisation cudaMalloc/cudaFree
 * may imply.  The paper has no counterpart; this is a service of this
 * library.  Same result as hcc_sort (stable ascending sort of ids by the low
 * key_bits bits).  Scratch is a fixed device array owned by the library,
 * sized for n <= HCC_SORT_NOALLOC_MAX_N keys of up to 64 bits (12 MiB on
 * every device that loads the library, for the life of the process).
 * Runs on the calling thread's current device; stream (a cudaStream_t,
 * NULL = legacy default stream) must belong to it.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array:
 * calls whose work overlaps on the GPU race and give wrong results.
 * err_word: optional device uint32 into which bounded-wait failures are
 * OR-ed (bit value 2); it is never cleared by the library.  With NULL such
 * a failure is not reported anywhere (the permutation is then unspecified),
 * so callers that need to detect it pass a word and read it.
 * Errors (synchronous): INVALID_ARG (n above the maximum, key_bits outside
 * 1..64, NULL/misaligned/overlapping buffers), CUDA.
 */
#define HCC_SORT_NOALLOC_MAX_N 524288u
hcc_status hcc_sort_noalloc(const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm, uint32_t *err_word,
                            void *stream);

/* ---------------------------------------------------------------- gather */

/*
 * out ray j = in ray perm[j] for j < n, both float4 streams, bit for bit
 * (Sec. 5: the trace fetches rays through the sorted indices).  in->n is the
 * number of valid source rays (every perm[j] must be below it); out->n is
 * the count gathered.  in and out must not overlap.  An entry perm[j] >=
 * in->n is never read through: out ray j is then zero and hcc_sync reports
 * INVALID_ARG.
 * Errors: INVALID_ARG, CUDA.
 */
hcc_status hcc_gather(hcc_ctx *ctx, const hcc_rays *in, const uint32_t *perm, const hcc_rays *out);

/* ----------------------------------------------------------------- trace */

/*
 * Closest hit (any_hit = 0) or any hit (any_hit != 0) of every ray against
 * the BVH's triangles by stack-based traversal of the quantised BVH2 and
 * the Moller-Trumbore test (two-sided, no epsilon, hit when tmin < t <
 * tmax).  Closest hit = smallest t, ties to the lower triangle id; it does
 * not depend on traversal order.  Any hit reports some hit of the ray.
 * Result of ray j goes to hits[j], or to hits[scatter[j]] when scatter is
 * not NULL (scatter must then be a permutation of 0..n-1; an entry >= n is
 * skipped and reported as INVALID_ARG by hcc_sync).  hits: n records,
 * device, 16-byte aligned.
 * Errors: INVALID_ARG, CUDA; STACK_OVERFLOW at hcc_sync if some ray needed
 * more than HCC_TRACE_STACK entries (its record is then a miss).
 */
hcc_status hcc_trace(hcc_ctx *ctx, const hcc_bvh *bvh, const hcc_rays *rays, int any_hit,
                     const uint32_t *scatter, hcc_hit *hits);

/*
 * Trace in sorted order without a separate gather (the arrangement of
 * Sec. 5: the trace kernel fetches each ray through the sorted indices).
 * Thread j traces ray perm[j] of rays and writes its record to
 * hits[perm[j]], so hits come out in input order, identical to hcc_trace on
 * the unsorted rays; only the order in which rays are traced changes.
 * perm: n uint32_t, a permutation of 0..n-1 (an entry >= n is skipped and
 * reported as INVALID_ARG by hcc_sync).  Errors: as hcc_trace.
 */
hcc_status hcc_trace_sorted(hcc_ctx *ctx, const hcc_bvh *bvh, const hcc_rays *rays, const uint32_t *perm,
                            int any_hit, hcc_hit *hits);

/*
 * Diagnostic (never on the timed path): trace like hcc_trace (perm NULL) or
 * hcc_trace_sorted (perm given) and count, over all rays: counts[0] internal
 * node visits, counts[1] triangle tests, counts[2] warp-level node steps
 * (loop iterations of a warp in which any lane visits a node), counts[3]
 * warp-level leaf steps.  counts[0] / (32 counts[2]) is the warp execution
 * efficiency of the node loop.  All four depend on which rays share a warp
 * (a lane that has parked a leaf keeps descending until its warp-mates
 * have one too), which is what ray order changes; the hits do not.  Allocates a
 * temporary hit buffer and waits for the stream.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
hcc_status hcc_trace_counts(hcc_ctx *ctx, const hcc_bvh *bvh, const hcc_rays *rays, const uint32_t *perm,
                            int any_hit, uint64_t counts[4]);

/* ---------------------------------------------- batches of wavefronts */

/*
 * A batch: the wavefronts of several scenes traced together.  Scene s owns
 * rays [offsets[s], offsets[s+1]) of the batch's combined ray buffers; its
 * BVH is bvhs[s] and, for HCC keys, its cut is cuts[s] (cuts may be NULL for
 * other methods).  All BVHs must use the same node layout.  offsets (host,
 * num_scenes + 1 entries, offsets[0] = 0, non-decreasing) and the scene table
 * are copied to the device; the handles must outlive the batch.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
typedef struct hcc_batch hcc_batch;
hcc_status hcc_batch_create(hcc_ctx *ctx, uint32_t num_scenes, const hcc_bvh *const *bvhs, const hcc_cut *const *cuts,
                            const uint64_t *offsets, hcc_batch **out);
hcc_status hcc_batch_destroy(hcc_batch *batch);

/*
 * One bounce of every wavefront of the batch with one launch per stage:
 * one encode over all rays (each against its own scene's cut or box, the
 * scene index placed above the key_bits key), one sort of the combined keys
 * (rays grouped by scene, then by key), one trace that fetches each ray
 * through the permutation and traverses its own scene's BVH.  NOSORT traces
 * in input order.  hits[i] is the record of ray i in its scene (triangle ids
 * of that scene).  key_bits plus ceil(log2(num_scenes)) must be <= 64.
 * rays->n must equal offsets[num_scenes].  Asynchronous; no host
 * synchronisation inside (scratch is grown first if needed, see
 * hcc_reserve).  Errors: as hcc_run.
 */
hcc_status hcc_batch_run(hcc_ctx *ctx, const hcc_batch *batch, hcc_method method, const hcc_rays *rays,
                         uint32_t key_bits, int any_hit, hcc_hit *hits);

/*
 * The next bounce of a batch (ray generation between bounces, not part of
 * the reordering method): for every ray i with hits[i].prim >= 0, a diffuse
 * ray leaving its hit point o + t d, cosine-weighted about the hit
 * triangle's normal turned toward the incoming ray, interval [tmin, +inf);
 * a ray that missed becomes the empty ray (interval [1, 0]) at its old
 * origin.  Random numbers: the top 24 bits of SplitMix64(SplitMix64(seed) ^
 * (64 i + j)); the direction is the first point of the unit disk found by
 * rejection among 16 tries (else the centre) lifted to the hemisphere, in
 * the orthonormal basis of Duff et al. 2017; every step is a correctly
 * rounded FP32 operation so the rays are reproducible.  in and out must be
 * different buffers with n = offsets[num_scenes].
 * Errors: INVALID_ARG, CUDA; INVALID_ARG at hcc_sync for a hit whose
 * triangle id is outside its scene (that ray becomes empty).
 */
hcc_status hcc_batch_spawn(hcc_ctx *ctx, const hcc_batch *batch, const hcc_rays *in, const hcc_hit *hits,
                           uint64_t seed, float tmin, const hcc_rays *out);

/*
 * CUDA graph of one batch bounce: reserves the scratch hcc_batch_run needs,
 * captures hcc_batch_run(ctx, batch, method, rays, key_bits, any_hit, hits)
 * on the context's stream (which must not be the legacy default stream) and
 * instantiates it.  hcc_graph_launch replays it on the context's stream with
 * the same buffers; the rays may be rewritten between launches.
 * Errors: INVALID_ARG, OOM, CUDA.
 */
typedef struct hcc_graph hcc_graph;
hcc_status hcc_graph_capture_batch(hcc_ctx *ctx, const hcc_batch *batch, hcc_method method, const hcc_rays *rays,
                                   uint32_t key_bits, int any_hit, hcc_hit *hits, hcc_graph **out);
/* General capture: every hcc call issued on ctx between hcc_graph_begin and
 * hcc_graph_end is recorded (not run) into the graph.  Reserve scratch first
 * (hcc_reserve): a call that would allocate fails inside a capture.  The
 * context's stream must not be the legacy default stream. */
hcc_status hcc_graph_begin(hcc_ctx *ctx);
hcc_status hcc_graph_end(hcc_ctx *ctx, hcc_graph **out);
hcc_status hcc_graph_launch(hcc_ctx *ctx, const hcc_graph *graph);
hcc_status hcc_graph_destroy(hcc_graph *graph);

/* ------------------------------------------------------- whole pipeline */

/*
 * The per-bounce reordering pipeline of Sec. 5 in one call:
 *   NOSORT:   trace(rays) -> hits
 *   HCC:      encode(cut) -> sort -> trace_sorted (fetch through perm) -> hits
 *   TWOPOINT: encode(root box) -> sort -> trace_sorted -> hits
 * hits[i] is always the result of input ray i, so every method produces
 * the same array.  Keys and permutation live in the context's scratch.
 * Device pointers; asynchronous on the context's stream.
 * Errors: as the individual calls.
 */
hcc_status hcc_run(hcc_ctx *ctx, hcc_method method, const hcc_bvh *bvh, const hcc_cut *cut,
                   const hcc_rays *rays, uint32_t key_bits, int any_hit, hcc_hit *hits);

/*
 * hcc_run on host memory: org_tmin and dir_tmax are n float4 each and hits
 * n records, all in host memory (page-locked memory gives asynchronous,
 * full-speed copies).  Copies the rays to device scratch, runs the
 * pipeline, copies the hits back and waits, so the hits are valid on return.
 * Above 2^22 rays, the rays go through in chunks of 2^22 (the first one
 * 2^21, so the first kernels start sooner) that alternate between two
 * internal streams (each chunk encoded, sorted and traced on its own), so
 * that the copies of one chunk overlap the kernels of the other; the hits
 * are the same as hcc_run's.  Errors: as hcc_run, plus those
 * of hcc_sync.
 */
hcc_status hcc_run_host(hcc_ctx *ctx, hcc_method method, const hcc_bvh *bvh, const hcc_cut *cut,
                        const float *org_tmin, const float *dir_tmax, uint64_t n, uint32_t key_bits, int any_hit,
                        hcc_hit *hits);

/* ------------------------------------------------------------ serving loop */

/*
 * A ray-query server over resident scenes.  The paper traces one wavefront
 * at a time (Sec. 5) and has no serving layer; this loop runs the same
 * per-request pipeline as hcc_run_host (encode against the scene's cut, sort,
 * trace through the permutation) for many clients at once.
 *
 * Requests are admitted in arrival order by a dispatcher thread that the
 * server owns, as soon as one of `slots` execution slots is free and the
 * request's device memory fits the budget; each admitted request runs on its
 * slot's own stream, so requests that arrive while others are on the GPU
 * start at once and their kernels and copies overlap.  Request buffers come
 * from a stream-ordered pool that keeps released memory, so steady-state
 * requests allocate nothing from the driver.  slots = 1 is the unbatched
 * per-request path: one request on the GPU at a time.
 *
 * A request's result does not depend on which requests share the GPU with
 * it: its kernels read only its own buffers and the read-only scene data,
 * and its hits equal hcc_run_host's for the same rays bit for bit.
 *
 * The BVH and cut handles given to hcc_server_create must stay alive until
 * hcc_server_destroy.  Host ray and hit buffers should be page-locked:
 * pageable buffers work, but their copies are staged synchronously and
 * serialise the dispatcher.
 */
typedef struct hcc_server hcc_server;

typedef struct hcc_server_config {
    uint32_t slots;       /* requests on the GPU at once, 1..64 */
    hcc_method method;    /* NOSORT, HCC, TWOPOINT, ORIGIN or ORIGIN_DIR */
    uint32_t key_bits;    /* 1..64 (ignored for NOSORT) */
    uint64_t hbm_budget;  /* device bytes for request buffers; 0 = 90% of free memory at creation */
} hcc_server_config;

typedef struct hcc_server_stats {
    uint64_t completed;     /* requests finished with HCC_OK */
    uint64_t failed;        /* requests finished with an error */
    uint64_t rays;          /* rays of the completed requests */
    uint32_t max_in_flight; /* most requests on the GPU at one time */
    uint32_t queued;        /* requests waiting for admission now */
    uint64_t budget;        /* the admission budget in bytes */
    uint64_t peak_bytes;    /* most budget bytes held by admitted requests */
} hcc_server_stats;

/*
 * Creates a server for num_scenes resident scenes (scene s = bvhs[s] and, for
 * HCC, cuts[s]); all BVHs must share one node layout and live on `device`.
 * Starts the dispatcher thread.  Errors: INVALID_ARG (bad config or handles),
 * CUDA (streams, events, the memory pool), OOM (host).
 */
hcc_status hcc_server_create(int device, uint32_t num_scenes, const hcc_bvh *const *bvhs, const hcc_cut *const *cuts,
                             const hcc_server_config *cfg, hcc_server **out);

/*
 * Queues a request of n rays (host float4 arrays org_tmin and dir_tmax, as
 * hcc_rays) against scene `scene`; the n hit records go to host memory
 * `hits`, valid once hcc_server_wait returns HCC_OK for *ticket.  The caller
 * keeps the three buffers alive and unchanged until then.  Thread-safe.
 * Errors: INVALID_ARG (scene index, NULL buffer, n = 0 or above
 * HCC_MAX_SORT_N, server stopping), OOM (the request alone exceeds the
 * budget; it would never be admitted).
 */
hcc_status hcc_server_submit(hcc_server *s, uint32_t scene, const float *org_tmin, const float *dir_tmax, uint64_t n,
                             int any_hit, hcc_hit *hits, uint64_t *ticket);

/* *done = 1 once the request has finished (successfully or not). */
hcc_status hcc_server_query(hcc_server *s, uint64_t ticket, int *done);

/*
 * Blocks until the request finishes, releases its ticket and returns its
 * status (wait once per ticket, from one thread; every wait must return
 * before hcc_server_destroy): OK, STACK_OVERFLOW (a ray's traversal needed more than
 * HCC_TRACE_STACK entries; its record is incomplete), TIMEOUT (a bounded
 * wait in the sort gave up), OOM (the pool could not grow), CUDA.  A failed
 * request does not affect any other.  *latency_ms (may be NULL) = time from
 * submission until the dispatcher saw the request's last copy complete.
 * INVALID_ARG for an unknown ticket.
 */
hcc_status hcc_server_wait(hcc_server *s, uint64_t ticket, double *latency_ms);

hcc_status hcc_server_stats_get(hcc_server *s, hcc_server_stats *out);

/* *bytes = the device memory a request of n rays is charged against the
 * budget (its ray, hit, key, permutation and sort-scratch buffers). */
hcc_status hcc_server_request_bytes(const hcc_server *s, uint64_t n, uint64_t *bytes);

/* Finishes every queued and running request, stops the thread, frees the
 * server (tickets not yet waited for are dropped). */
hcc_status hcc_server_destroy(hcc_server *s);

#ifdef __cplusplus
}
#endif

#endif /* HCC_H */
