// C ABI of the hcc library: argument checking, device memory, the BVH
// upload (quantised and exact BVH2 node layouts, 4-ary nodes collapsed from
// the BVH2), host-side cut selection (Sec. 4.2.2), the per-bounce pipeline
// (Sec. 5), batches of wavefronts and CUDA graphs.  Kernels live in
// encode.cu, sort.cu, gather.cu, trace.cu and spawn.cu; the serving loop in
// serve.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "hcc_internal.cuh"

using namespace hcc;

// ---------------------------------------------------------------- handles

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Rays per chunk and lanes (contexts with their own streams) of the
// pipelined hcc_run_host.
constexpr uint64_t HOST_CHUNK = 1ull << 22;
constexpr uint32_t HOST_LANES = 2;
// The first chunks are a quarter and a half as large, so the first kernels
// start sooner while the next copies catch up (1M, 2M, then 4M rays: 5.81 ms
// for the room's 16.6M rays against 5.88 with 2M then 4M, 5.98 with 1M then 4M).
static uint64_t host_chunk_rays(uint64_t c, uint64_t rem) {
    return std::min(c == 0 ? HOST_CHUNK / 4 : c == 1 ? HOST_CHUNK / 2 : HOST_CHUNK, rem);
}

struct hcc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t *d_err = nullptr;                 // device error word (16-byte allocation) ...
    unsigned long long *d_work = nullptr;      // ... whose second half is the trace's slot counter
    hcc_trace_schedule schedule = HCC_TRACE_AUTO;
    float twopoint_fraction = 0.25f;            // TwoPoint length estimate / largest extent
    hcc::SortOptions sort_opt;                  // bounded-wait settings of this context's sorts
    uint32_t trace_block = 128, trace_stack = HCC_TRACE_STACK;  // shape of the closest-hit persistent trace
    std::string last_error;
    DevBuf sort_scratch;
    DevBuf keys, perm;                          // hcc_run
    DevBuf in_org, in_dir, hits;                // hcc_run_host
    hcc_ctx *lane[HOST_LANES] = {};             // hcc_run_host pipeline: contexts on their own streams
    cudaEvent_t lane_in[HOST_LANES] = {};       // ... and the end of each lane's last input copy
};

struct hcc_bvh {
    int device = 0;
    int layout = HCC_BVH_QUANTISED;
    uint4 *d_nodes = nullptr;
    float4 *d_tris = nullptr;
    uint32_t *d_prim_rec = nullptr;  // triangle id -> record index
    uint32_t num_nodes = 0, num_internal = 0, num_tris = 0, depth = 0;
    uint32_t root_ref = 0;
    // exact tree kept on the host for cut selection
    std::vector<float> lo, hi;
    std::vector<int32_t> left, right;
    std::vector<uint32_t> count;
};

struct hcc_cut {
    int device = 0;
    std::vector<int32_t> ids;   // cut nodes (the top level of a two-level cut), key order; -1 for grid cells
    float4 *d_boxes = nullptr;  // (lo, hi) pairs in key order, at most 64 nodes
    uint32_t on_device = 0;
    std::vector<float> lo, hi;  // host copy of the on-device boxes, 3 floats each
    // two-level cut (MLHCC): field widths, low-level ids and boxes (row r = top node r)
    uint32_t top_field = 0, low_field = 0;
    std::vector<int32_t> low_ids;
    float4 *d_low = nullptr;
};

struct hcc_batch {
    int device = 0;
    int layout = 0;
    uint32_t num_scenes = 0;
    uint32_t scene_bits = 0;  // bits above the key that hold the scene index
    std::vector<uint64_t> offsets;
    hcc::SceneDesc *d_scenes = nullptr;
    uint64_t *d_offsets = nullptr;
};

struct hcc_graph {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr uint32_t MAX_KEY_NODES = 64;
constexpr uint32_t MAX_BATCH_SCENES = 1024;

hcc_status fail(hcc_ctx *ctx, hcc_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

hcc_status cuda_fail(hcc_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(ctx, HCC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(ctx, HCC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Make ctx current on its device for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

hcc_status ensure(hcc_ctx *ctx, DevBuf &b, size_t bytes, const char *what) {
    if (b.bytes >= bytes) return HCC_OK;
    if (b.p) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stream sync before growing scratch");
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 256);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, HCC_ERR_OOM, "cudaMalloc of %zu bytes for %s failed", bytes, what);
    }
    b.p = p;
    b.bytes = bytes;
    return HCC_OK;
}

void release(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

hcc_status check_rays(hcc_ctx *ctx, const hcc_rays *r, const char *name) {
    if (!r) return fail(ctx, HCC_ERR_INVALID_ARG, "%s is NULL", name);
    if (r->stride % 16 != 0 || r->stride > (1u << 20))
        return fail(ctx, HCC_ERR_INVALID_ARG, "%s: the stride must be a multiple of 16 bytes (at most 2^20)", name);
    if (r->n == 0) return HCC_OK;
    if (!r->org_tmin || !r->dir_tmax) return fail(ctx, HCC_ERR_INVALID_ARG, "%s has a NULL stream", name);
    if (!aligned(r->org_tmin, 16) || !aligned(r->dir_tmax, 16))
        return fail(ctx, HCC_ERR_INVALID_ARG, "%s streams must be 16-byte aligned", name);
    if (r->n > (uint64_t)0xFFFFFFFFu) return fail(ctx, HCC_ERR_INVALID_ARG, "%s: n above 2^32-1", name);
    return HCC_OK;
}

// Stride of a ray descriptor in float4 units (0 bytes: packed arrays).
uint32_t ray_rs(const hcc_rays *r) { return r->stride ? (uint32_t)(r->stride / 16) : 1u; }
// One 32-byte record per ray: direction right after the origin, 32-byte aligned.
bool ray_rec(const hcc_rays *r) {
    return ray_rs(r) == 2 && r->dir_tmax == r->org_tmin + 4 && aligned(r->org_tmin, 32);
}

// ------------------------------------------------------ node quantisation

// Round a float toward -inf to a value whose low 8 mantissa bits are zero.
float round_down_24(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    if ((b & 0xFFu) == 0) return x;
    if (!(x < 0.0f))
        b &= ~0xFFu;
    else
        b = (b & ~0xFFu) + 0x100u;
    float y;
    std::memcpy(&y, &b, 4);
    return y;
}

uint32_t float_bits(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    return b;
}

// Quantise the boxes of an internal node's two children (exact boxes lo/hi,
// 3 floats each) into the 32-byte record described in hcc_internal.cuh.
// Every decoded bound origin + q * 2^E is outside (or on) the exact bound.
void quantise_node(const float *lo0, const float *hi0, const float *lo1, const float *hi1, uint32_t ref0,
                   uint32_t ref1, uint32_t w[8]) {
    uint8_t q[2][6];
    for (int a = 0; a < 3; ++a) {
        const float o = round_down_24(std::min(lo0[a], lo1[a]));
        const double od = o;
        const double top = std::max((double)hi0[a], (double)hi1[a]);
        const double ext = top - od;
        int E = -126;
        if (ext > 0) {
            int e2;
            std::frexp(ext / 255.0, &e2);  // ext/255 in [2^(e2-1), 2^e2)
            E = std::max(e2, -126);
            while (E > -126 && std::ldexp(255.0, E - 1) >= ext) --E;
            while (std::ldexp(255.0, E) < ext) ++E;
        }
        const double s = std::ldexp(1.0, E);
        const float *los[2] = {lo0, lo1}, *his[2] = {hi0, hi1};
        for (int c = 0; c < 2; ++c) {
            double ql = std::floor(((double)los[c][a] - od) / s);
            double qh = std::ceil(((double)his[c][a] - od) / s);
            ql = std::min(std::max(ql, 0.0), 255.0);
            qh = std::min(std::max(qh, 0.0), 255.0);
            while (ql > 0 && od + ql * s > (double)los[c][a]) ql -= 1;
            while (qh < 255 && od + qh * s < (double)his[c][a]) qh += 1;
            q[c][a] = (uint8_t)ql;
            q[c][3 + a] = (uint8_t)qh;
        }
        w[a] = (float_bits(o) & 0xFFFFFF00u) | (uint32_t)(E + 127);
    }
    // byte stream: child0 lo.xyz hi.xyz, child1 lo.xyz hi.xyz
    uint8_t bytes[12];
    for (int k = 0; k < 6; ++k) {
        bytes[k] = q[0][k];
        bytes[6 + k] = q[1][k];
    }
    for (int j = 0; j < 3; ++j)
        w[3 + j] = (uint32_t)bytes[4 * j] | ((uint32_t)bytes[4 * j + 1] << 8) | ((uint32_t)bytes[4 * j + 2] << 16) |
                   ((uint32_t)bytes[4 * j + 3] << 24);
    w[6] = ref0;
    w[7] = ref1;
}

// ---------------------------------------------------------- cut selection

// Eq. 1 in double, children before parents (reverse of a pre-order walk).
std::vector<double> compute_had(const hcc_bvh *b, double lambda) {
    const uint32_t n = b->num_nodes;
    std::vector<double> had(n, 0.0);
    std::vector<int32_t> order;
    order.reserve(n);
    std::vector<int32_t> todo{0};
    while (!todo.empty()) {
        int32_t k = todo.back();
        todo.pop_back();
        order.push_back(k);
        if (b->left[k] >= 0) {
            todo.push_back(b->right[k]);
            todo.push_back(b->left[k]);
        }
    }
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
        const int32_t k = *it;
        const double ex = (double)b->hi[3 * k] - (double)b->lo[3 * k];
        const double ey = (double)b->hi[3 * k + 1] - (double)b->lo[3 * k + 1];
        const double ez = (double)b->hi[3 * k + 2] - (double)b->lo[3 * k + 2];
        const double sa = 2.0 * (ex * ey + ey * ez + ez * ex);
        if (b->left[k] < 0)
            had[k] = (double)b->count[k] * sa;
        else
            had[k] = (had[b->left[k]] + had[b->right[k]]) + lambda * sa;
    }
    return had;
}

// Max-heap of node ids by (HAD descending, id ascending).
struct HadHeap {
    const std::vector<double> &had;
    std::vector<int32_t> a;
    explicit HadHeap(const std::vector<double> &h) : had(h) {}
    bool above(int32_t x, int32_t y) const { return had[x] > had[y] || (had[x] == had[y] && x < y); }
    void push(int32_t v) {
        a.push_back(v);
        size_t i = a.size() - 1;
        while (i > 0) {
            size_t p = (i - 1) / 2;
            if (!above(a[i], a[p])) break;
            std::swap(a[i], a[p]);
            i = p;
        }
    }
    int32_t pop() {
        int32_t top = a[0];
        a[0] = a.back();
        a.pop_back();
        size_t i = 0;
        for (;;) {
            size_t l = 2 * i + 1, r = l + 1, m = i;
            if (l < a.size() && above(a[l], a[m])) m = l;
            if (r < a.size() && above(a[r], a[m])) m = r;
            if (m == i) break;
            std::swap(a[i], a[m]);
            i = m;
        }
        return top;
    }
};

}  // namespace

namespace hcc {

// Device views of the handles for the serving loop (serve.cu).
void bvh_view(const hcc_bvh *b, SceneDesc *out, int *layout, int *device) {
    std::memset(out, 0, sizeof *out);
    out->nodes = b->d_nodes;
    out->tris = b->d_tris;
    out->prim_rec = b->d_prim_rec;
    out->root_ref = b->root_ref;
    out->num_tris = b->num_tris;
    for (int a = 0; a < 3; ++a) {
        out->lo[a] = b->lo[a];
        out->ext[a] = b->hi[a] - b->lo[a];
    }
    out->L = 0.25f * std::max(out->ext[0], std::max(out->ext[1], out->ext[2]));
    *layout = b->layout;
    *device = b->device;
}

void cut_view(const hcc_cut *c, const float4 **boxes, uint32_t *on_device, int *device) {
    *boxes = c->d_boxes;
    *on_device = c->on_device;
    *device = c->device;
}

}  // namespace hcc

// Slot counter for the persistent trace, or NULL for one thread per ray.
static unsigned long long *trace_work(const hcc_ctx *ctx, int any_hit) {
    const bool refill = ctx->schedule == HCC_TRACE_REFILL || (ctx->schedule == HCC_TRACE_AUTO && !any_hit);
    return refill ? ctx->d_work : nullptr;
}

// ================================================================== C ABI

extern "C" {

const char *hcc_status_string(hcc_status s) {
    switch (s) {
        case HCC_OK: return "HCC_OK";
        case HCC_ERR_INVALID_ARG: return "HCC_ERR_INVALID_ARG";
        case HCC_ERR_OOM: return "HCC_ERR_OOM";
        case HCC_ERR_CUDA: return "HCC_ERR_CUDA";
        case HCC_ERR_UNSUPPORTED: return "HCC_ERR_UNSUPPORTED";
        case HCC_ERR_STACK_OVERFLOW: return "HCC_ERR_STACK_OVERFLOW";
        case HCC_ERR_TIMEOUT: return "HCC_ERR_TIMEOUT";
    }
    return "HCC_ERR_UNKNOWN";
}

const char *hcc_last_error(const hcc_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "NULL context"; }

hcc_status hcc_create(hcc_ctx **out, int device, void *stream) {
    if (!out) return HCC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
        cudaGetLastError();
        return HCC_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return HCC_ERR_INVALID_ARG;
    hcc_ctx *c = new (std::nothrow) hcc_ctx;
    if (!c) return HCC_ERR_OOM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    DeviceGuard g(device);
    if (cudaMalloc(&c->d_err, 16) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return HCC_ERR_OOM;
    }
    c->d_work = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(c->d_err) + 8);
    if (cudaMemset(c->d_err, 0, 16) != cudaSuccess) {
        cudaFree(c->d_err);
        delete c;
        return HCC_ERR_CUDA;
    }
    *out = c;
    return HCC_OK;
}

hcc_status hcc_set_trace_schedule(hcc_ctx *ctx, hcc_trace_schedule schedule) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (schedule != HCC_TRACE_AUTO && schedule != HCC_TRACE_PER_RAY && schedule != HCC_TRACE_REFILL)
        return fail(ctx, HCC_ERR_INVALID_ARG, "unknown trace schedule");
    ctx->schedule = schedule;
    return HCC_OK;
}

hcc_status hcc_set_twopoint_distance(hcc_ctx *ctx, float fraction) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (!(fraction >= 0.0f) || !std::isfinite(fraction))
        return fail(ctx, HCC_ERR_INVALID_ARG, "the TwoPoint distance must be finite and non-negative");
    ctx->twopoint_fraction = fraction;
    for (hcc_ctx *l : ctx->lane)
        if (l) l->twopoint_fraction = fraction;
    return HCC_OK;
}

hcc_status hcc_set_trace_shape(hcc_ctx *ctx, uint32_t block_threads, uint32_t stack_entries) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (block_threads == 0 && stack_entries == 0) {
        block_threads = 128;
        stack_entries = HCC_TRACE_STACK;
    }
    if (!hcc::trace_shape_supported(block_threads, stack_entries))
        return fail(ctx, HCC_ERR_INVALID_ARG, "unsupported trace shape %u threads x %u stack entries", block_threads,
                    stack_entries);
    ctx->trace_block = block_threads;
    ctx->trace_stack = stack_entries;
    for (hcc_ctx *l : ctx->lane)
        if (l) {
            l->trace_block = block_threads;
            l->trace_stack = stack_entries;
        }
    return HCC_OK;
}

hcc_status hcc_set_sort_wait_limit(hcc_ctx *ctx, uint32_t status_reads) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    ctx->sort_opt.wait_limit = status_reads ? status_reads : hcc::SortOptions().wait_limit;
    for (hcc_ctx *l : ctx->lane)
        if (l) l->sort_opt.wait_limit = ctx->sort_opt.wait_limit;
    return HCC_OK;
}

hcc_status hcc_test_sort_withhold_tile(hcc_ctx *ctx, uint32_t tile) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    ctx->sort_opt.withhold_tile = tile;
    for (hcc_ctx *l : ctx->lane)
        if (l) l->sort_opt.withhold_tile = tile;
    return HCC_OK;
}

hcc_status hcc_destroy(hcc_ctx *ctx) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < HOST_LANES; ++i) {
        hcc_ctx *&l = ctx->lane[i];
        if (l) {
            cudaStream_t s = l->stream;
            hcc_destroy(l);
            DeviceGuard g(ctx->device);
            cudaStreamDestroy(s);
            l = nullptr;
        }
        if (ctx->lane_in[i]) {
            DeviceGuard g(ctx->device);
            cudaEventDestroy(ctx->lane_in[i]);
            ctx->lane_in[i] = nullptr;
        }
    }
    {
        DeviceGuard g(ctx->device);
        cudaStreamSynchronize(ctx->stream);
        for (DevBuf *b : {&ctx->sort_scratch, &ctx->keys, &ctx->perm, &ctx->in_org, &ctx->in_dir, &ctx->hits})
            release(*b);
        if (ctx->d_err) cudaFree(ctx->d_err);
    }
    delete ctx;
    return HCC_OK;
}

hcc_status hcc_set_stream(hcc_ctx *ctx, void *stream) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    return HCC_OK;
}

hcc_status hcc_reserve(hcc_ctx *ctx, uint64_t max_n, uint32_t max_key_bits) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (max_key_bits < 1 || max_key_bits > 64) return fail(ctx, HCC_ERR_INVALID_ARG, "max_key_bits must be 1..64");
    if (max_n > HCC_MAX_SORT_N) return fail(ctx, HCC_ERR_INVALID_ARG, "max_n above HCC_MAX_SORT_N");
    DeviceGuard g(ctx->device);
    const size_t ksz = max_key_bits > 32 ? 8 : 4;
    hcc_status st;
    if ((st = ensure(ctx, ctx->sort_scratch, sort_scratch_bytes(max_n, max_key_bits), "sort scratch")) != HCC_OK)
        return st;
    if ((st = ensure(ctx, ctx->keys, max_n * ksz, "keys")) != HCC_OK) return st;
    if ((st = ensure(ctx, ctx->perm, max_n * 4, "perm")) != HCC_OK) return st;
    return HCC_OK;
}

hcc_status hcc_sync(hcc_ctx *ctx) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    uint32_t err = 0;
    e = cudaMemcpy(&err, ctx->d_err, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the device error word");
    if (err) {
        e = cudaMemset(ctx->d_err, 0, sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "clearing the device error word");
        if (err & ERR_STACK)
            return fail(ctx, HCC_ERR_STACK_OVERFLOW, "a ray needed more than %d traversal-stack entries",
                        HCC_TRACE_STACK);
        if (err & ERR_TIMEOUT) return fail(ctx, HCC_ERR_TIMEOUT, "a bounded wait in the sort gave up");
        if (err & ERR_INDEX)
            return fail(ctx, HCC_ERR_INVALID_ARG, "a permutation or scatter entry was out of range (skipped)");
    }
    return HCC_OK;
}

// ------------------------------------------------------------------- BVH

// 4-ary traversal nodes from a validated BVH2 (root internal): starting
// from a BVH2 node's two children, the internal child with the largest
// surface area is replaced by its two children until four are held or all
// are leaves (the usual collapse of a binary tree into a wide one).  Node i
// is 32 words, eight rows of four (one entry per child): lo.x, hi.x, lo.y,
// hi.y, lo.z, hi.z of the exact boxes of the BVH2 nodes they stand for,
// the references, and zeros; an unused child has reference 0xFFFFFFFF and
// a zero box.  Returns the node count.
static uint32_t collapse_wide(const hcc_bvh_desc *d, std::vector<uint32_t> &words) {
    auto is_leaf = [&](int32_t k) { return d->left[k] < 0; };
    auto leaf_ref = [&](int32_t k) { return REF_LEAF | ((d->count[k] - 1u) << 29) | d->first[k]; };
    auto area = [&](int32_t k) {
        const double ex = (double)d->hi[3 * k] - d->lo[3 * k], ey = (double)d->hi[3 * k + 1] - d->lo[3 * k + 1],
                     ez = (double)d->hi[3 * k + 2] - d->lo[3 * k + 2];
        return ex * ey + ey * ez + ez * ex;
    };
    std::vector<int32_t> order{0};  // BVH2 node of each wide node, in creation order
    std::vector<std::array<int32_t, 4>> slots;
    std::vector<uint32_t> used;
    for (size_t w = 0; w < order.size(); ++w) {
        const int32_t k = order[w];
        std::vector<int32_t> ch{d->left[k], d->right[k]};
        while (ch.size() < 4) {
            int best = -1;
            double best_a = -1.0;
            for (int c = 0; c < (int)ch.size(); ++c)
                if (!is_leaf(ch[c]) && area(ch[c]) > best_a) {
                    best = c;
                    best_a = area(ch[c]);
                }
            if (best < 0) break;
            const int32_t n = ch[best];
            ch[best] = d->left[n];
            ch.insert(ch.begin() + best + 1, d->right[n]);
        }
        std::array<int32_t, 4> sl{-1, -1, -1, -1};
        for (size_t c = 0; c < ch.size(); ++c) sl[c] = ch[c];
        slots.push_back(sl);
        used.push_back((uint32_t)ch.size());
        for (int32_t c : ch)
            if (!is_leaf(c)) order.push_back(c);
    }
    std::vector<int32_t> widx(d->num_nodes, -1);
    for (size_t w = 0; w < order.size(); ++w) widx[order[w]] = (int32_t)w;
    words.assign(order.size() * 32, 0u);
    for (size_t w = 0; w < order.size(); ++w) {
        uint32_t *q = &words[32 * w];
        for (uint32_t c = 0; c < 4; ++c) {
            if (c >= used[w]) {
                q[24 + c] = 0xFFFFFFFFu;
                continue;
            }
            const int32_t k = slots[w][c];
            for (int a = 0; a < 3; ++a) {
                std::memcpy(&q[8 * a + c], d->lo + 3 * (size_t)k + a, 4);
                std::memcpy(&q[8 * a + 4 + c], d->hi + 3 * (size_t)k + a, 4);
            }
            q[24 + c] = is_leaf(k) ? leaf_ref(k) : (uint32_t)widx[k];
        }
    }
    return (uint32_t)order.size();
}

hcc_status hcc_bvh_upload(hcc_ctx *ctx, const hcc_bvh_desc *d, hcc_bvh **out) {
    return hcc_bvh_upload_layout(ctx, d, HCC_BVH_QUANTISED, out);
}

hcc_status hcc_bvh_upload_layout(hcc_ctx *ctx, const hcc_bvh_desc *d, hcc_bvh_layout layout, hcc_bvh **out) {
    if (!ctx || !d || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (layout != HCC_BVH_QUANTISED && layout != HCC_BVH_EXACT && layout != HCC_BVH_WIDE)
        return fail(ctx, HCC_ERR_INVALID_ARG, "unknown BVH layout");
    if (d->num_nodes == 0 || d->num_tris == 0) return fail(ctx, HCC_ERR_INVALID_ARG, "empty BVH");
    if (!d->lo || !d->hi || !d->left || !d->right || !d->first || !d->count || !d->tris || !d->order)
        return fail(ctx, HCC_ERR_INVALID_ARG, "NULL array in hcc_bvh_desc");
    if (d->num_nodes > 0x7FFFFFFFu || d->num_tris > REF_TRI_MASK)
        return fail(ctx, HCC_ERR_INVALID_ARG, "BVH too large for the node layout");
    const uint32_t N = d->num_nodes, T = d->num_tris;
    for (uint32_t k = 0; k < T; ++k)
        if (d->order[k] >= T) return fail(ctx, HCC_ERR_INVALID_ARG, "order[%u] out of range", k);
    // walk the tree from the root: validates structure, numbers internal nodes
    // in pre-order and measures the depth
    std::vector<int32_t> qidx(N, -1);
    std::vector<uint8_t> seen(N, 0);
    std::vector<std::pair<int32_t, uint32_t>> todo{{0, 0u}};
    std::vector<int32_t> internal;
    uint32_t depth = 0;
    while (!todo.empty()) {
        auto [k, dep] = todo.back();
        todo.pop_back();
        if (seen[k]) return fail(ctx, HCC_ERR_INVALID_ARG, "node %d reached twice", k);
        seen[k] = 1;
        depth = std::max(depth, dep);
        const int32_t l = d->left[k], r = d->right[k];
        if (l < 0 || r < 0) {
            if (l >= 0 || r >= 0) return fail(ctx, HCC_ERR_INVALID_ARG, "node %d has one child", k);
            if (d->count[k] < 1 || d->count[k] > 4)
                return fail(ctx, HCC_ERR_INVALID_ARG, "leaf %d holds %u triangles (1..4 allowed)", k, d->count[k]);
            if ((uint64_t)d->first[k] + d->count[k] > T)
                return fail(ctx, HCC_ERR_INVALID_ARG, "leaf %d range out of bounds", k);
            continue;
        }
        if ((uint32_t)l >= N || (uint32_t)r >= N || l == r)
            return fail(ctx, HCC_ERR_INVALID_ARG, "node %d has bad children", k);
        qidx[k] = (int32_t)internal.size();
        internal.push_back(k);
        todo.push_back({r, dep + 1});
        todo.push_back({l, dep + 1});
    }
    auto ref_of = [&](int32_t k) -> uint32_t {
        if (d->left[k] < 0) return REF_LEAF | ((d->count[k] - 1u) << 29) | d->first[k];
        return (uint32_t)qidx[k];
    };
    // node boxes with lo <= hi on every axis (the traversal's slab test picks
    // the near plane by the direction's sign); a box given inverted on an
    // axis means the same slab to a min/max slab test, so it is swapped
    std::vector<float> blo(d->lo, d->lo + 3 * (size_t)N), bhi(d->hi, d->hi + 3 * (size_t)N);
    for (size_t j = 0; j < blo.size(); ++j)
        if (blo[j] > bhi[j]) std::swap(blo[j], bhi[j]);
    hcc_bvh_desc nd = *d;
    nd.lo = blo.data();
    nd.hi = bhi.data();
    std::vector<uint32_t> words;
    uint32_t num_device_nodes = (uint32_t)internal.size();
    if (layout == HCC_BVH_WIDE) {
        if (internal.empty())
            words.assign(32, 0u);  // a leaf root: the traversal reads no node
        else
            num_device_nodes = collapse_wide(&nd, words);
    } else {
        const size_t wpn = layout == HCC_BVH_EXACT ? 16 : 8;  // 32-bit words per node
        words.assign((size_t)std::max<size_t>(internal.size(), 1) * wpn, 0u);
    }
    for (size_t i = 0; layout != HCC_BVH_WIDE && i < internal.size(); ++i) {
        const size_t wpn = layout == HCC_BVH_EXACT ? 16 : 8;
        const int32_t k = internal[i], l = d->left[k], r = d->right[k];
        uint32_t *w = &words[wpn * i];
        if (layout == HCC_BVH_QUANTISED) {
            quantise_node(&blo[3 * l], &bhi[3 * l], &blo[3 * r], &bhi[3 * r], ref_of(l), ref_of(r), w);
        } else {
            // per child (lo.x, lo.y), (hi.x, hi.y), (lo.z, hi.z): the pairs the
            // traversal's packed slab arithmetic takes
            const float f[12] = {blo[3 * l], blo[3 * l + 1], bhi[3 * l], bhi[3 * l + 1],
                                 blo[3 * l + 2], bhi[3 * l + 2], blo[3 * r], blo[3 * r + 1],
                                 bhi[3 * r], bhi[3 * r + 1], blo[3 * r + 2], bhi[3 * r + 2]};
            std::memcpy(w, f, sizeof f);
            w[12] = ref_of(l);
            w[13] = ref_of(r);
        }
    }
    std::vector<float> tri((size_t)T * 12);
    for (uint32_t k = 0; k < T; ++k) {
        const uint32_t id = d->order[k];
        const float *v = d->tris + 9 * (size_t)id;
        float *o = &tri[12 * (size_t)k];
        o[0] = v[0];
        o[1] = v[1];
        o[2] = v[2];
        std::memcpy(&o[3], &id, 4);
        for (int a = 0; a < 3; ++a) {
            o[4 + a] = v[3 + a] - v[a];
            o[8 + a] = v[6 + a] - v[a];
        }
        o[7] = 0.0f;
        o[11] = 0.0f;
    }
    hcc_bvh *b = new (std::nothrow) hcc_bvh;
    if (!b) return fail(ctx, HCC_ERR_OOM, "host allocation");
    b->device = ctx->device;
    b->layout = layout;
    b->num_nodes = N;
    b->num_internal = num_device_nodes;
    b->num_tris = T;
    b->depth = depth;
    b->root_ref = ref_of(0);
    b->lo.assign(d->lo, d->lo + 3 * (size_t)N);
    b->hi.assign(d->hi, d->hi + 3 * (size_t)N);
    b->left.assign(d->left, d->left + N);
    b->right.assign(d->right, d->right + N);
    b->count.assign(d->count, d->count + N);
    DeviceGuard g(ctx->device);
    std::vector<uint32_t> prim_rec(T, 0u);
    for (uint32_t k = 0; k < T; ++k) prim_rec[d->order[k]] = k;
    cudaError_t e = cudaMalloc(&b->d_nodes, words.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tris, tri.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_prim_rec, (size_t)T * 4);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_nodes, words.data(), words.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tris, tri.data(), tri.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_prim_rec, prim_rec.data(), (size_t)T * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hcc_bvh_destroy(b);
        return cuda_fail(ctx, e, "BVH upload");
    }
    *out = b;
    return HCC_OK;
}

hcc_status hcc_bvh_info(const hcc_bvh *b, uint32_t *num_nodes, uint32_t *num_tris, uint32_t *depth, float *lo3,
                        float *hi3) {
    if (!b) return HCC_ERR_INVALID_ARG;
    if (num_nodes) *num_nodes = b->num_nodes;
    if (num_tris) *num_tris = b->num_tris;
    if (depth) *depth = b->depth;
    for (int a = 0; a < 3; ++a) {
        if (lo3) lo3[a] = b->lo[a];
        if (hi3) hi3[a] = b->hi[a];
    }
    return HCC_OK;
}

hcc_status hcc_bvh_destroy(hcc_bvh *b) {
    if (!b) return HCC_ERR_INVALID_ARG;
    {
        DeviceGuard g(b->device);
        if (b->d_nodes) cudaFree(b->d_nodes);
        if (b->d_tris) cudaFree(b->d_tris);
        if (b->d_prim_rec) cudaFree(b->d_prim_rec);
    }
    delete b;
    return HCC_OK;
}

// ------------------------------------------------------------------- cut

// Algorithm 2 on the subtree of `start`: pop the largest-HAD node; a leaf
// joins the cut and lowers the queue limit, an internal node is replaced by
// its children; stop at cut_size nodes (or when the queue empties).  Result
// in key order.
static std::vector<int32_t> cut_of_subtree(const hcc_bvh *bvh, const std::vector<double> &had, int32_t start,
                                           uint32_t cut_size) {
    HadHeap pq(had);
    std::vector<int32_t> cut;
    uint32_t max_queue = cut_size;
    pq.push(start);
    while (!pq.a.empty() && pq.a.size() < max_queue) {
        const int32_t k = pq.pop();
        if (bvh->left[k] < 0) {
            cut.push_back(k);
            --max_queue;
        } else {
            pq.push(bvh->left[k]);
            pq.push(bvh->right[k]);
        }
    }
    cut.insert(cut.end(), pq.a.begin(), pq.a.end());
    std::sort(cut.begin(), cut.end(),
              [&](int32_t x, int32_t y) { return had[x] > had[y] || (had[x] == had[y] && x < y); });
    return cut;
}

static void push_box(std::vector<float4> &boxes, const float *lo, const float *hi) {
    boxes.push_back(make_float4(lo[0], lo[1], lo[2], 0.0f));
    boxes.push_back(make_float4(hi[0], hi[1], hi[2], 0.0f));
}

// Copies (lo, hi) pairs to a new device array (at least one pair).
static cudaError_t upload_boxes(std::vector<float4> boxes, float4 **out) {
    if (boxes.empty()) boxes.resize(2, make_float4(0.f, 0.f, 0.f, 0.f));
    cudaError_t e = cudaMalloc(out, boxes.size() * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemcpy(*out, boxes.data(), boxes.size() * sizeof(float4), cudaMemcpyHostToDevice);
    return e;
}

// Sets the key-driving boxes of a cut (host copy and device array).
static cudaError_t set_key_boxes(hcc_cut *c, const std::vector<float> &lo, const std::vector<float> &hi) {
    const uint32_t m = (uint32_t)std::min<size_t>(lo.size() / 3, MAX_KEY_NODES);
    c->on_device = m;
    c->lo.assign(lo.begin(), lo.begin() + 3 * m);
    c->hi.assign(hi.begin(), hi.begin() + 3 * m);
    std::vector<float4> boxes;
    for (uint32_t r = 0; r < m; ++r) push_box(boxes, &c->lo[3 * r], &c->hi[3 * r]);
    return upload_boxes(boxes, &c->d_boxes);
}

static hcc_status check_lambda(hcc_ctx *ctx, double lambda) {
    if (!(lambda >= 0.0) || !std::isfinite(lambda))
        return fail(ctx, HCC_ERR_INVALID_ARG, "lambda must be finite and non-negative");
    return HCC_OK;
}

hcc_status hcc_select_cut(hcc_ctx *ctx, const hcc_bvh *bvh, uint32_t cut_size, double lambda, hcc_cut **out) {
    if (!ctx || !bvh || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (cut_size == 0) return fail(ctx, HCC_ERR_INVALID_ARG, "cut_size must be positive");
    hcc_status st = check_lambda(ctx, lambda);
    if (st != HCC_OK) return st;
    const std::vector<double> had = compute_had(bvh, lambda);
    const std::vector<int32_t> cut = cut_of_subtree(bvh, had, 0, cut_size);
    hcc_cut *c = new (std::nothrow) hcc_cut;
    if (!c) return fail(ctx, HCC_ERR_OOM, "host allocation");
    c->device = ctx->device;
    c->ids = cut;
    std::vector<float> lo, hi;
    for (int32_t k : cut) {
        lo.insert(lo.end(), &bvh->lo[3 * k], &bvh->lo[3 * k] + 3);
        hi.insert(hi.end(), &bvh->hi[3 * k], &bvh->hi[3 * k] + 3);
    }
    DeviceGuard g(ctx->device);
    cudaError_t e = set_key_boxes(c, lo, hi);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hcc_cut_destroy(c);
        return cuda_fail(ctx, e, "cut upload");
    }
    *out = c;
    return HCC_OK;
}

hcc_status hcc_select_cut_ml(hcc_ctx *ctx, const hcc_bvh *bvh, uint32_t top_size, uint32_t low_size, double lambda,
                             hcc_cut **out) {
    if (!ctx || !bvh || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (top_size == 0 || low_size == 0 || top_size + low_size > MAX_KEY_NODES)
        return fail(ctx, HCC_ERR_INVALID_ARG, "top_size and low_size must be positive with a sum of at most 64");
    hcc_status st = check_lambda(ctx, lambda);
    if (st != HCC_OK) return st;
    const std::vector<double> had = compute_had(bvh, lambda);
    // leaves under every node, children before parents (ids are not assumed ordered)
    const uint32_t n = bvh->num_nodes;
    std::vector<uint32_t> leaves(n, 1);
    {
        std::vector<int32_t> order, todo{0};
        while (!todo.empty()) {
            const int32_t k = todo.back();
            todo.pop_back();
            order.push_back(k);
            if (bvh->left[k] >= 0) {
                todo.push_back(bvh->left[k]);
                todo.push_back(bvh->right[k]);
            }
        }
        for (auto it = order.rbegin(); it != order.rend(); ++it)
            if (bvh->left[*it] >= 0) leaves[*it] = leaves[bvh->left[*it]] + leaves[bvh->right[*it]];
    }
    auto qualifies = [&](int32_t k) { return leaves[k] >= low_size; };
    // Algorithm 3, top level: Algorithm 2 over the nodes that qualify
    HadHeap pq(had);
    std::vector<int32_t> top;
    uint32_t max_queue = top_size;
    if (qualifies(0)) pq.push(0);
    while (!pq.a.empty() && pq.a.size() < max_queue) {
        const int32_t k = pq.pop();
        const bool l = bvh->left[k] >= 0 && qualifies(bvh->left[k]);
        const bool r = bvh->left[k] >= 0 && qualifies(bvh->right[k]);
        if (!l && !r) {
            top.push_back(k);
            --max_queue;
        } else {
            if (l) pq.push(bvh->left[k]);
            if (r) pq.push(bvh->right[k]);
        }
    }
    top.insert(top.end(), pq.a.begin(), pq.a.end());
    std::sort(top.begin(), top.end(),
              [&](int32_t x, int32_t y) { return had[x] > had[y] || (had[x] == had[y] && x < y); });
    hcc_cut *c = new (std::nothrow) hcc_cut;
    if (!c) return fail(ctx, HCC_ERR_OOM, "host allocation");
    c->device = ctx->device;
    c->ids = top;
    c->top_field = top_size;
    c->low_field = low_size;
    std::vector<float> lo, hi;
    std::vector<float4> low_boxes;
    for (int32_t t : top) {
        lo.insert(lo.end(), &bvh->lo[3 * t], &bvh->lo[3 * t] + 3);
        hi.insert(hi.end(), &bvh->hi[3 * t], &bvh->hi[3 * t] + 3);
        const std::vector<int32_t> low = cut_of_subtree(bvh, had, t, low_size);  // exactly low_size nodes
        for (int32_t k : low) {
            c->low_ids.push_back(k);
            push_box(low_boxes, &bvh->lo[3 * k], &bvh->hi[3 * k]);
        }
    }
    DeviceGuard g(ctx->device);
    cudaError_t e = set_key_boxes(c, lo, hi);
    if (e == cudaSuccess) e = upload_boxes(low_boxes, &c->d_low);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hcc_cut_destroy(c);
        return cuda_fail(ctx, e, "cut upload");
    }
    *out = c;
    return HCC_OK;
}

hcc_status hcc_cut_ml_info(const hcc_cut *cut, uint32_t *ntop, uint32_t *top_size, uint32_t *low_size,
                           int32_t *low_ids) {
    if (!cut || !ntop || !top_size || !low_size || cut->low_field == 0) return HCC_ERR_INVALID_ARG;
    *ntop = (uint32_t)cut->ids.size();
    *top_size = cut->top_field;
    *low_size = cut->low_field;
    if (low_ids) std::memcpy(low_ids, cut->low_ids.data(), cut->low_ids.size() * sizeof(int32_t));
    return HCC_OK;
}

hcc_status hcc_select_grid(hcc_ctx *ctx, const hcc_bvh *bvh, uint32_t max_cells, hcc_cut **out) {
    if (!ctx || !bvh || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (max_cells == 0 || max_cells > MAX_KEY_NODES) return fail(ctx, HCC_ERR_INVALID_ARG, "max_cells must be 1..64");
    const float *blo = &bvh->lo[0], *bhi = &bvh->hi[0];  // the root box
    uint32_t g[3] = {1, 1, 1}, cells = 1;
    while (cells * 2 <= max_cells) {
        int axis = 0;
        double longest = -1.0;
        for (int a = 0; a < 3; ++a) {
            const double len = ((double)bhi[a] - (double)blo[a]) / g[a];
            if (len > longest) {
                longest = len;
                axis = a;
            }
        }
        g[axis] *= 2;
        cells *= 2;
    }
    auto boundary = [&](int a, uint32_t i) {
        return (float)(((double)(g[a] - i) * (double)blo[a] + (double)i * (double)bhi[a]) / (double)g[a]);
    };
    std::vector<float> lo, hi;
    for (uint32_t i = 0; i < g[0]; ++i)
        for (uint32_t j = 0; j < g[1]; ++j)
            for (uint32_t l = 0; l < g[2]; ++l) {
                const uint32_t idx[3] = {i, j, l};
                for (int a = 0; a < 3; ++a) {
                    lo.push_back(boundary(a, idx[a]));
                    hi.push_back(boundary(a, idx[a] + 1));
                }
            }
    hcc_cut *c = new (std::nothrow) hcc_cut;
    if (!c) return fail(ctx, HCC_ERR_OOM, "host allocation");
    c->device = ctx->device;
    c->ids.assign(cells, -1);
    DeviceGuard dg(ctx->device);
    cudaError_t e = set_key_boxes(c, lo, hi);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hcc_cut_destroy(c);
        return cuda_fail(ctx, e, "cut upload");
    }
    *out = c;
    return HCC_OK;
}

hcc_status hcc_cut_boxes(const hcc_cut *cut, float *lo, float *hi) {
    if (!cut || !lo || !hi) return HCC_ERR_INVALID_ARG;
    std::memcpy(lo, cut->lo.data(), cut->lo.size() * sizeof(float));
    std::memcpy(hi, cut->hi.data(), cut->hi.size() * sizeof(float));
    return HCC_OK;
}

hcc_status hcc_cut_info(const hcc_cut *cut, uint32_t *size, int32_t *node_ids) {
    if (!cut || !size) return HCC_ERR_INVALID_ARG;
    *size = (uint32_t)cut->ids.size();
    if (node_ids) std::memcpy(node_ids, cut->ids.data(), cut->ids.size() * sizeof(int32_t));
    return HCC_OK;
}

hcc_status hcc_cut_destroy(hcc_cut *cut) {
    if (!cut) return HCC_ERR_INVALID_ARG;
    {
        DeviceGuard g(cut->device);
        if (cut->d_boxes) cudaFree(cut->d_boxes);
        if (cut->d_low) cudaFree(cut->d_low);
    }
    delete cut;
    return HCC_OK;
}

// ---------------------------------------------------------------- encode

hcc_status hcc_encode(hcc_ctx *ctx, hcc_method method, const hcc_bvh *bvh, const hcc_cut *cut,
                      const hcc_rays *rays, uint32_t key_bits, void *keys) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    hcc_status st = check_rays(ctx, rays, "rays");
    if (st != HCC_OK) return st;
    if (key_bits < 1 || key_bits > 64) return fail(ctx, HCC_ERR_INVALID_ARG, "key_bits must be 1..64");
    if (method != HCC_METHOD_HCC && method != HCC_METHOD_TWOPOINT && method != HCC_METHOD_ORIGIN &&
        method != HCC_METHOD_ORIGIN_DIR && method != HCC_METHOD_PPC && method != HCC_METHOD_MLHCC)
        return fail(ctx, HCC_ERR_INVALID_ARG, "hcc_encode needs a method with a key");
    const bool cut_key = method == HCC_METHOD_HCC || method == HCC_METHOD_MLHCC;
    if (cut_key && !cut) return fail(ctx, HCC_ERR_INVALID_ARG, "this key needs a cut");
    if (!cut_key && !bvh) return fail(ctx, HCC_ERR_INVALID_ARG, "this key needs the BVH");
    if (method == HCC_METHOD_MLHCC) {
        if (cut->low_field == 0) return fail(ctx, HCC_ERR_INVALID_ARG, "MLHCC needs a two-level cut");
        if (cut->top_field + cut->low_field > key_bits)
            return fail(ctx, HCC_ERR_INVALID_ARG, "the cut's two fields need %u key bits",
                        cut->top_field + cut->low_field);
    }
    if (method == HCC_METHOD_PPC && bvh->layout != HCC_BVH_EXACT)
        return fail(ctx, HCC_ERR_UNSUPPORTED, "the prefix path code needs a BVH with exact node boxes");
    if (rays->n == 0) return HCC_OK;
    if (!keys || !aligned(keys, key_bits > 32 ? 8 : 4))
        return fail(ctx, HCC_ERR_INVALID_ARG, "keys NULL or misaligned");
    DeviceGuard g(ctx->device);
    const float4 *o = reinterpret_cast<const float4 *>(rays->org_tmin);
    const float4 *d = reinterpret_cast<const float4 *>(rays->dir_tmax);
    const uint32_t rs = ray_rs(rays);
    cudaError_t e;
    if (method == HCC_METHOD_HCC) {
        const uint32_t used = std::min<uint32_t>(cut->on_device, key_bits);
        e = launch_encode_hcc(ctx->stream, o, d, rays->n, rs, cut->d_boxes, used, key_bits, keys);
    } else if (method == HCC_METHOD_MLHCC) {
        e = launch_encode_mlhcc(ctx->stream, o, d, rays->n, rs, cut->d_boxes, cut->on_device, cut->top_field, cut->d_low,
                                cut->low_field, key_bits, keys);
    } else if (method == HCC_METHOD_PPC) {
        e = launch_encode_ppc(ctx->stream, o, d, rays->n, rs, bvh->d_nodes, bvh->root_ref, &bvh->lo[0], &bvh->hi[0],
                              key_bits, keys);
    } else {
        float lo[3], ext[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = bvh->lo[a];
            ext[a] = bvh->hi[a] - bvh->lo[a];
        }
        if (method == HCC_METHOD_TWOPOINT) {
            const float L = ctx->twopoint_fraction * std::max(ext[0], std::max(ext[1], ext[2]));
            e = launch_encode_twopoint(ctx->stream, o, d, rays->n, rs, lo, ext, L, key_bits, keys);
        } else if (method == HCC_METHOD_ORIGIN) {
            e = launch_encode_origin(ctx->stream, o, rays->n, rs, lo, ext, key_bits, keys);
        } else {
            e = launch_encode_origin_dir(ctx->stream, o, d, rays->n, rs, lo, ext, key_bits, keys);
        }
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "encode launch");
    return HCC_OK;
}

hcc_status hcc_key_stats(hcc_ctx *ctx, const void *keys, uint32_t key_bits, const uint32_t *perm, uint64_t n,
                         double *anc, uint64_t *distinct) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (key_bits < 1 || key_bits > 64) return fail(ctx, HCC_ERR_INVALID_ARG, "key_bits must be 1..64");
    if (!anc || !distinct) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL output");
    *anc = 0.0;
    *distinct = 0;
    if (n == 0) return HCC_OK;
    if (!keys || !perm || !aligned(keys, key_bits > 32 ? 8 : 4) || !aligned(perm, 4))
        return fail(ctx, HCC_ERR_INVALID_ARG, "keys/perm NULL or misaligned");
    DeviceGuard g(ctx->device);
    DevBuf tmp;
    hcc_status st = ensure(ctx, tmp, 256, "key statistics");
    if (st != HCC_OK) return st;
    unsigned long long host[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(tmp.p, 0, 2 * sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess)
        e = launch_key_stats(ctx->stream, keys, key_bits, perm, n, static_cast<unsigned long long *>(tmp.p));
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, tmp.p, sizeof host, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    release(tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "key statistics");
    const uint64_t groups = (n + 31) / 32;
    *anc = (double)(groups + host[1]) / (double)groups;
    *distinct = 1 + host[0];
    return HCC_OK;
}

// ------------------------------------------------------------------ sort

hcc_status hcc_sort(hcc_ctx *ctx, const void *keys, uint32_t key_bits, uint64_t n, uint32_t *perm) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (key_bits < 1 || key_bits > 64) return fail(ctx, HCC_ERR_INVALID_ARG, "key_bits must be 1..64");
    if (n > HCC_MAX_SORT_N) return fail(ctx, HCC_ERR_INVALID_ARG, "n above HCC_MAX_SORT_N");
    if (n == 0) return HCC_OK;
    const size_t ksz = key_bits > 32 ? 8 : 4;
    if (!keys || !perm || !aligned(keys, ksz) || !aligned(perm, 4))
        return fail(ctx, HCC_ERR_INVALID_ARG, "keys/perm NULL or misaligned");
    const uintptr_t k0 = (uintptr_t)keys, k1 = k0 + n * ksz, p0 = (uintptr_t)perm, p1 = p0 + n * 4;
    if (k0 < p1 && p0 < k1) return fail(ctx, HCC_ERR_INVALID_ARG, "keys and perm overlap");
    DeviceGuard g(ctx->device);
    hcc_status st = ensure(ctx, ctx->sort_scratch, sort_scratch_bytes(n, key_bits), "sort scratch");
    if (st != HCC_OK) return st;
    cudaError_t e = launch_sort(ctx->stream, keys, key_bits, n, perm, ctx->sort_scratch.p, ctx->d_err, ctx->sort_opt);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sort launch");
    return HCC_OK;
}

// ---------------------------------------------------------------- gather

hcc_status hcc_gather(hcc_ctx *ctx, const hcc_rays *in, const uint32_t *perm, const hcc_rays *out) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    hcc_status st;
    if ((st = check_rays(ctx, in, "in")) != HCC_OK) return st;
    if ((st = check_rays(ctx, out, "out")) != HCC_OK) return st;
    if (out->n == 0) return HCC_OK;
    if (!perm || !aligned(perm, 4)) return fail(ctx, HCC_ERR_INVALID_ARG, "perm NULL or misaligned");
    if (in->n == 0) return fail(ctx, HCC_ERR_INVALID_ARG, "gather from an empty ray set");
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_gather(ctx->stream, reinterpret_cast<const float4 *>(in->org_tmin),
                                  reinterpret_cast<const float4 *>(in->dir_tmax), ray_rs(in), in->n, perm,
                                  reinterpret_cast<float4 *>(out->org_tmin), reinterpret_cast<float4 *>(out->dir_tmax),
                                  ray_rs(out), out->n, ctx->d_err);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather launch");
    return HCC_OK;
}

// ----------------------------------------------------------------- trace

hcc_status hcc_trace(hcc_ctx *ctx, const hcc_bvh *bvh, const hcc_rays *rays, int any_hit, const uint32_t *scatter,
                     hcc_hit *hits) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    hcc_status st = check_rays(ctx, rays, "rays");
    if (st != HCC_OK) return st;
    if (!bvh) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL BVH");
    if (rays->n == 0) return HCC_OK;
    if (!hits || !aligned(hits, 16)) return fail(ctx, HCC_ERR_INVALID_ARG, "hits NULL or not 16-byte aligned");
    if (scatter && !aligned(scatter, 4)) return fail(ctx, HCC_ERR_INVALID_ARG, "scatter misaligned");
    DeviceGuard g(ctx->device);
    TraceArgs a;
    a.nodes = bvh->d_nodes;
    a.layout = bvh->layout;
    a.tris = bvh->d_tris;
    a.root_ref = bvh->root_ref;
    a.org = reinterpret_cast<const float4 *>(rays->org_tmin);
    a.dir = reinterpret_cast<const float4 *>(rays->dir_tmax);
    a.rs = ray_rs(rays);
    a.rec = ray_rec(rays);
    a.n = rays->n;
    a.gather = nullptr;
    a.scatter = scatter;
    a.hits = reinterpret_cast<int4 *>(hits);
    a.err = ctx->d_err;
    a.work = trace_work(ctx, any_hit);
    a.block = (int)ctx->trace_block;
    a.stack = (int)ctx->trace_stack;
    a.counts = nullptr;
    a.scenes = nullptr;
    a.offsets = nullptr;
    a.num_scenes = 0;
    cudaError_t e = launch_trace(ctx->stream, a, any_hit);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace launch");
    return HCC_OK;
}

hcc_status hcc_trace_sorted(hcc_ctx *ctx, const hcc_bvh *bvh, const hcc_rays *rays, const uint32_t *perm,
                            int any_hit, hcc_hit *hits) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    hcc_status st = check_rays(ctx, rays, "rays");
    if (st != HCC_OK) return st;
    if (!bvh) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL BVH");
    if (rays->n == 0) return HCC_OK;
    if (!hits || !aligned(hits, 16)) return fail(ctx, HCC_ERR_INVALID_ARG, "hits NULL or not 16-byte aligned");
    if (!perm || !aligned(perm, 4)) return fail(ctx, HCC_ERR_INVALID_ARG, "perm NULL or misaligned");
    DeviceGuard g(ctx->device);
    TraceArgs a;
    a.nodes = bvh->d_nodes;
    a.layout = bvh->layout;
    a.tris = bvh->d_tris;
    a.root_ref = bvh->root_ref;
    a.org = reinterpret_cast<const float4 *>(rays->org_tmin);
    a.dir = reinterpret_cast<const float4 *>(rays->dir_tmax);
    a.rs = ray_rs(rays);
    a.rec = ray_rec(rays);
    a.n = rays->n;
    a.gather = perm;
    a.scatter = perm;
    a.hits = reinterpret_cast<int4 *>(hits);
    a.err = ctx->d_err;
    a.work = trace_work(ctx, any_hit);
    a.block = (int)ctx->trace_block;
    a.stack = (int)ctx->trace_stack;
    a.counts = nullptr;
    a.scenes = nullptr;
    a.offsets = nullptr;
    a.num_scenes = 0;
    cudaError_t e = launch_trace(ctx->stream, a, any_hit);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace launch");
    return HCC_OK;
}

hcc_status hcc_trace_counts(hcc_ctx *ctx, const hcc_bvh *bvh, const hcc_rays *rays, const uint32_t *perm,
                            int any_hit, uint64_t counts[4]) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    hcc_status st = check_rays(ctx, rays, "rays");
    if (st != HCC_OK) return st;
    if (!bvh || !counts) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < 4; ++k) counts[k] = 0;
    if (rays->n == 0) return HCC_OK;
    if (perm && !aligned(perm, 4)) return fail(ctx, HCC_ERR_INVALID_ARG, "perm misaligned");
    DeviceGuard g(ctx->device);
    DevBuf tmp;
    if ((st = ensure(ctx, tmp, rays->n * sizeof(hcc_hit) + 256, "counting trace output")) != HCC_OK) return st;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(static_cast<char *>(tmp.p) +
                                                                     rays->n * sizeof(hcc_hit));
    cudaError_t e = cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), ctx->stream);
    TraceArgs a;
    a.nodes = bvh->d_nodes;
    a.layout = bvh->layout;
    a.tris = bvh->d_tris;
    a.root_ref = bvh->root_ref;
    a.org = reinterpret_cast<const float4 *>(rays->org_tmin);
    a.dir = reinterpret_cast<const float4 *>(rays->dir_tmax);
    a.rs = ray_rs(rays);
    a.rec = ray_rec(rays);
    a.n = rays->n;
    a.gather = perm;
    a.scatter = perm;
    a.hits = reinterpret_cast<int4 *>(tmp.p);
    a.err = ctx->d_err;
    a.work = trace_work(ctx, any_hit);
    a.block = (int)ctx->trace_block;
    a.stack = (int)ctx->trace_stack;
    a.counts = cnt;
    a.scenes = nullptr;
    a.offsets = nullptr;
    a.num_scenes = 0;
    if (e == cudaSuccess) e = launch_trace(ctx->stream, a, any_hit);
    unsigned long long host[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, cnt, sizeof host, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    release(tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counting trace");
    for (int k = 0; k < 4; ++k) counts[k] = host[k];
    return HCC_OK;
}

// ----------------------------------------------------------------- batch

hcc_status hcc_batch_create(hcc_ctx *ctx, uint32_t num_scenes, const hcc_bvh *const *bvhs, const hcc_cut *const *cuts,
                            const uint64_t *offsets, hcc_batch **out) {
    if (!ctx || !bvhs || !offsets || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (num_scenes == 0 || num_scenes > MAX_BATCH_SCENES)
        return fail(ctx, HCC_ERR_INVALID_ARG, "a batch holds 1..%u scenes", MAX_BATCH_SCENES);
    if (offsets[0] != 0) return fail(ctx, HCC_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (uint32_t s = 0; s < num_scenes; ++s) {
        if (!bvhs[s]) return fail(ctx, HCC_ERR_INVALID_ARG, "scene %u has no BVH", s);
        if (bvhs[s]->layout != bvhs[0]->layout)
            return fail(ctx, HCC_ERR_INVALID_ARG, "all BVHs of a batch need the same node layout");
        if (offsets[s + 1] < offsets[s]) return fail(ctx, HCC_ERR_INVALID_ARG, "offsets must not decrease");
    }
    if (offsets[num_scenes] > HCC_MAX_SORT_N) return fail(ctx, HCC_ERR_INVALID_ARG, "batch above HCC_MAX_SORT_N rays");
    std::vector<hcc::SceneDesc> sd(num_scenes);
    for (uint32_t s = 0; s < num_scenes; ++s) {
        const hcc_bvh *b = bvhs[s];
        hcc::SceneDesc &d = sd[s];
        std::memset(&d, 0, sizeof d);
        d.nodes = b->d_nodes;
        d.tris = b->d_tris;
        d.prim_rec = b->d_prim_rec;
        d.root_ref = b->root_ref;
        d.num_tris = b->num_tris;
        const hcc_cut *c = cuts ? cuts[s] : nullptr;
        d.cut = c ? c->d_boxes : nullptr;
        d.used = c ? c->on_device : 0;
        d.cut_ordered = 1;
        if (c)
            for (size_t q = 0; q < c->lo.size(); ++q) d.cut_ordered &= c->lo[q] <= c->hi[q] ? 1u : 0u;
        for (int a = 0; a < 3; ++a) {
            d.lo[a] = b->lo[a];
            d.ext[a] = b->hi[a] - b->lo[a];
        }
        d.L = 0.25f * std::max(d.ext[0], std::max(d.ext[1], d.ext[2]));
    }
    hcc_batch *bt = new (std::nothrow) hcc_batch;
    if (!bt) return fail(ctx, HCC_ERR_OOM, "host allocation");
    bt->device = ctx->device;
    bt->layout = bvhs[0]->layout;
    bt->num_scenes = num_scenes;
    while ((1u << bt->scene_bits) < num_scenes) ++bt->scene_bits;
    bt->offsets.assign(offsets, offsets + num_scenes + 1);
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaMalloc(&bt->d_scenes, sizeof(hcc::SceneDesc) * num_scenes);
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_offsets, sizeof(uint64_t) * (num_scenes + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(bt->d_scenes, sd.data(), sizeof(hcc::SceneDesc) * num_scenes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(bt->d_offsets, offsets, sizeof(uint64_t) * (num_scenes + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        hcc_batch_destroy(bt);
        return cuda_fail(ctx, e, "batch upload");
    }
    *out = bt;
    return HCC_OK;
}

hcc_status hcc_batch_destroy(hcc_batch *b) {
    if (!b) return HCC_ERR_INVALID_ARG;
    {
        DeviceGuard g(b->device);
        if (b->d_scenes) cudaFree(b->d_scenes);
        if (b->d_offsets) cudaFree(b->d_offsets);
    }
    delete b;
    return HCC_OK;
}

hcc_status hcc_batch_run(hcc_ctx *ctx, const hcc_batch *b, hcc_method method, const hcc_rays *rays, uint32_t key_bits,
                         int any_hit, hcc_hit *hits) {
    if (!ctx || !b) return HCC_ERR_INVALID_ARG;
    hcc_status st = check_rays(ctx, rays, "rays");
    if (st != HCC_OK) return st;
    const uint64_t n = b->offsets[b->num_scenes];
    if (rays->n != n) return fail(ctx, HCC_ERR_INVALID_ARG, "rays->n must equal the batch's last offset");
    if (method == HCC_METHOD_PPC || method == HCC_METHOD_MLHCC)
        return fail(ctx, HCC_ERR_UNSUPPORTED, "batches take NOSORT, HCC, TWOPOINT, ORIGIN or ORIGIN_DIR keys");
    if (method != HCC_METHOD_NOSORT && method != HCC_METHOD_HCC && method != HCC_METHOD_TWOPOINT &&
        method != HCC_METHOD_ORIGIN && method != HCC_METHOD_ORIGIN_DIR)
        return fail(ctx, HCC_ERR_INVALID_ARG, "unknown method");
    if (n == 0) return HCC_OK;
    if (!hits || !aligned(hits, 16)) return fail(ctx, HCC_ERR_INVALID_ARG, "hits NULL or not 16-byte aligned");
    const uint32_t total_bits = key_bits + b->scene_bits;
    if (method != HCC_METHOD_NOSORT && (key_bits < 1 || total_bits > 64))
        return fail(ctx, HCC_ERR_INVALID_ARG, "key_bits plus %u scene bits must fit 64 bits", b->scene_bits);
    DeviceGuard g(ctx->device);
    TraceArgs a;
    a.layout = b->layout;
    a.org = reinterpret_cast<const float4 *>(rays->org_tmin);
    a.dir = reinterpret_cast<const float4 *>(rays->dir_tmax);
    a.rs = ray_rs(rays);
    a.rec = ray_rec(rays);
    a.n = n;
    a.hits = reinterpret_cast<int4 *>(hits);
    a.err = ctx->d_err;
    a.work = trace_work(ctx, any_hit);
    a.block = (int)ctx->trace_block;
    a.stack = (int)ctx->trace_stack;
    a.scenes = b->d_scenes;
    a.offsets = b->d_offsets;
    a.num_scenes = b->num_scenes;
    cudaError_t e;
    if (method != HCC_METHOD_NOSORT) {
        const size_t ksz = total_bits > 32 ? 8 : 4;
        if ((st = ensure(ctx, ctx->keys, n * ksz, "keys")) != HCC_OK) return st;
        if ((st = ensure(ctx, ctx->perm, n * 4, "perm")) != HCC_OK) return st;
        e = launch_encode_multi(ctx->stream, (int)method, a.org, a.dir, n, a.rs, b->d_scenes, b->d_offsets,
                                b->num_scenes, key_bits, total_bits, ctx->keys.p);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch encode launch");
        uint32_t *perm = static_cast<uint32_t *>(ctx->perm.p);
        if ((st = hcc_sort(ctx, ctx->keys.p, total_bits, n, perm)) != HCC_OK) return st;
        a.gather = perm;
        a.scatter = perm;
    }
    e = launch_trace(ctx->stream, a, any_hit);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch trace launch");
    return HCC_OK;
}

hcc_status hcc_batch_spawn(hcc_ctx *ctx, const hcc_batch *b, const hcc_rays *in, const hcc_hit *hits, uint64_t seed,
                           float tmin, const hcc_rays *out) {
    if (!ctx || !b) return HCC_ERR_INVALID_ARG;
    hcc_status st;
    if ((st = check_rays(ctx, in, "in")) != HCC_OK) return st;
    if ((st = check_rays(ctx, out, "out")) != HCC_OK) return st;
    const uint64_t n = b->offsets[b->num_scenes];
    if (in->n != n || out->n != n) return fail(ctx, HCC_ERR_INVALID_ARG, "ray counts must equal the batch's");
    if (n == 0) return HCC_OK;
    if (!hits || !aligned(hits, 16)) return fail(ctx, HCC_ERR_INVALID_ARG, "hits NULL or misaligned");
    if (in->org_tmin == out->org_tmin || in->dir_tmax == out->dir_tmax)
        return fail(ctx, HCC_ERR_INVALID_ARG, "in and out must be different buffers");
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_spawn(ctx->stream, reinterpret_cast<const float4 *>(in->org_tmin),
                                 reinterpret_cast<const float4 *>(in->dir_tmax), ray_rs(in),
                                 reinterpret_cast<const int4 *>(hits), n, b->d_scenes, b->d_offsets, b->num_scenes,
                                 seed, tmin, reinterpret_cast<float4 *>(out->org_tmin),
                                 reinterpret_cast<float4 *>(out->dir_tmax), ray_rs(out), ctx->d_err);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "spawn launch");
    return HCC_OK;
}

// --------------------------------------------------------- graph capture

hcc_status hcc_graph_capture_batch(hcc_ctx *ctx, const hcc_batch *b, hcc_method method, const hcc_rays *rays,
                                   uint32_t key_bits, int any_hit, hcc_hit *hits, hcc_graph **out) {
    if (!ctx || !b || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!ctx->stream) return fail(ctx, HCC_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    // everything the bounce needs must exist before capture: no allocation inside it
    const uint64_t n = b->offsets[b->num_scenes];
    if (method != HCC_METHOD_NOSORT) {
        const uint32_t total_bits = key_bits + b->scene_bits;
        if (key_bits < 1 || total_bits > 64) return fail(ctx, HCC_ERR_INVALID_ARG, "key bits do not fit");
        hcc_status st = hcc_reserve(ctx, n, total_bits);
        if (st != HCC_OK) return st;
    }
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
    hcc_status st = hcc_batch_run(ctx, b, method, rays, key_bits, any_hit, hits);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != HCC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(ctx, e, "graph instantiate");
    }
    hcc_graph *gr = new (std::nothrow) hcc_graph;
    if (!gr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(ctx, HCC_ERR_OOM, "host allocation");
    }
    gr->device = ctx->device;
    gr->graph = graph;
    gr->exec = exec;
    *out = gr;
    return HCC_OK;
}

hcc_status hcc_graph_begin(hcc_ctx *ctx) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (!ctx->stream) return fail(ctx, HCC_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
    return HCC_OK;
}

hcc_status hcc_graph_end(hcc_ctx *ctx, hcc_graph **out) {
    if (!ctx || !out) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    DeviceGuard g(ctx->device);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(ctx, e, "graph instantiate");
    }
    hcc_graph *gr = new (std::nothrow) hcc_graph;
    if (!gr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(ctx, HCC_ERR_OOM, "host allocation");
    }
    gr->device = ctx->device;
    gr->graph = graph;
    gr->exec = exec;
    *out = gr;
    return HCC_OK;
}

hcc_status hcc_graph_launch(hcc_ctx *ctx, const hcc_graph *gr) {
    if (!ctx || !gr) return HCC_ERR_INVALID_ARG;
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaGraphLaunch(gr->exec, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
    return HCC_OK;
}

hcc_status hcc_graph_destroy(hcc_graph *gr) {
    if (!gr) return HCC_ERR_INVALID_ARG;
    {
        DeviceGuard g(gr->device);
        if (gr->exec) cudaGraphExecDestroy(gr->exec);
        if (gr->graph) cudaGraphDestroy(gr->graph);
    }
    delete gr;
    return HCC_OK;
}

// -------------------------------------------------------------- pipeline

hcc_status hcc_run(hcc_ctx *ctx, hcc_method method, const hcc_bvh *bvh, const hcc_cut *cut, const hcc_rays *rays,
                   uint32_t key_bits, int any_hit, hcc_hit *hits) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    hcc_status st = check_rays(ctx, rays, "rays");
    if (st != HCC_OK) return st;
    if (!bvh) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL BVH");
    if (method != HCC_METHOD_NOSORT && method != HCC_METHOD_HCC && method != HCC_METHOD_TWOPOINT &&
        method != HCC_METHOD_ORIGIN && method != HCC_METHOD_ORIGIN_DIR && method != HCC_METHOD_PPC &&
        method != HCC_METHOD_MLHCC)
        return fail(ctx, HCC_ERR_INVALID_ARG, "unknown method");
    if (rays->n == 0) return HCC_OK;
    if (method == HCC_METHOD_NOSORT) return hcc_trace(ctx, bvh, rays, any_hit, nullptr, hits);
    if (key_bits < 1 || key_bits > 64) return fail(ctx, HCC_ERR_INVALID_ARG, "key_bits must be 1..64");
    if ((method == HCC_METHOD_HCC || method == HCC_METHOD_MLHCC) && !cut)
        return fail(ctx, HCC_ERR_INVALID_ARG, "this key needs a cut");
    const uint64_t n = rays->n;
    if (n > HCC_MAX_SORT_N) return fail(ctx, HCC_ERR_INVALID_ARG, "n above HCC_MAX_SORT_N");
    DeviceGuard g(ctx->device);
    const size_t ksz = key_bits > 32 ? 8 : 4;
    if ((st = ensure(ctx, ctx->keys, n * ksz, "keys")) != HCC_OK) return st;
    if ((st = ensure(ctx, ctx->perm, n * 4, "perm")) != HCC_OK) return st;
    if ((st = hcc_encode(ctx, method, bvh, cut, rays, key_bits, ctx->keys.p)) != HCC_OK) return st;
    uint32_t *perm = static_cast<uint32_t *>(ctx->perm.p);
    if ((st = hcc_sort(ctx, ctx->keys.p, key_bits, n, perm)) != HCC_OK) return st;
    return hcc_trace_sorted(ctx, bvh, rays, perm, any_hit, hits);
}

hcc_status hcc_run_host(hcc_ctx *ctx, hcc_method method, const hcc_bvh *bvh, const hcc_cut *cut,
                        const float *org_tmin, const float *dir_tmax, uint64_t n, uint32_t key_bits, int any_hit,
                        hcc_hit *hits) {
    if (!ctx) return HCC_ERR_INVALID_ARG;
    if (n == 0) return HCC_OK;
    if (!org_tmin || !dir_tmax || !hits) return fail(ctx, HCC_ERR_INVALID_ARG, "NULL host buffer");
    if (n > HCC_MAX_SORT_N) return fail(ctx, HCC_ERR_INVALID_ARG, "n above HCC_MAX_SORT_N");
    DeviceGuard g(ctx->device);
    hcc_status st;
    cudaError_t e;
    if (n <= HOST_CHUNK) {
        // one pass on the context's stream
        if ((st = ensure(ctx, ctx->in_org, n * 16, "input rays")) != HCC_OK) return st;
        if ((st = ensure(ctx, ctx->in_dir, n * 16, "input rays")) != HCC_OK) return st;
        if ((st = ensure(ctx, ctx->hits, n * sizeof(hcc_hit), "hits")) != HCC_OK) return st;
        e = cudaMemcpyAsync(ctx->in_org.p, org_tmin, n * 16, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->in_dir.p, dir_tmax, n * 16, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "host-to-device copy of rays");
        hcc_rays r{static_cast<float *>(ctx->in_org.p), static_cast<float *>(ctx->in_dir.p), n};
        if ((st = hcc_run(ctx, method, bvh, cut, &r, key_bits, any_hit, static_cast<hcc_hit *>(ctx->hits.p))) !=
            HCC_OK)
            return st;
        e = cudaMemcpyAsync(hits, ctx->hits.p, n * sizeof(hcc_hit), cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "device-to-host copy of hits");
        return hcc_sync(ctx);
    }
    // Pipelined: chunks of HOST_CHUNK rays take turns on the lane contexts,
    // each with its own stream and scratch, so that one chunk's copies overlap
    // another's kernels.  Each chunk is encoded, sorted and traced on its
    // own; hits do not depend on the order rays are traced in.
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "context stream");
    for (uint32_t i = 0; i < HOST_LANES; ++i) {
        hcc_ctx *&l = ctx->lane[i];
        if (!ctx->lane_in[i] && (e = cudaEventCreateWithFlags(&ctx->lane_in[i], cudaEventDisableTiming)) != cudaSuccess) {
            ctx->lane_in[i] = nullptr;
            return cuda_fail(ctx, e, "pipeline event");
        }
        if (l) continue;
        cudaStream_t s = nullptr;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(ctx, e, "pipeline stream");
        if ((st = hcc_create(&l, ctx->device, s)) != HCC_OK) {
            cudaStreamDestroy(s);
            return fail(ctx, st, "pipeline context");
        }
    }
    for (hcc_ctx *l : ctx->lane) {  // the lanes follow the context's settings
        l->schedule = ctx->schedule;
        l->trace_block = ctx->trace_block;
        l->trace_stack = ctx->trace_stack;
        l->twopoint_fraction = ctx->twopoint_fraction;
        l->sort_opt = ctx->sort_opt;
    }
    hcc_status result = HCC_OK;
    for (uint64_t c0 = 0, c = 0, m = 0; c0 < n && result == HCC_OK; c0 += m, ++c) {
        hcc_ctx *L = ctx->lane[c % HOST_LANES];
        L->schedule = ctx->schedule;
        L->twopoint_fraction = ctx->twopoint_fraction;
        m = host_chunk_rays(c, n - c0);
        if ((st = ensure(L, L->in_org, HOST_CHUNK * 16, "input rays")) != HCC_OK ||
            (st = ensure(L, L->in_dir, HOST_CHUNK * 16, "input rays")) != HCC_OK ||
            (st = ensure(L, L->hits, HOST_CHUNK * sizeof(hcc_hit), "hits")) != HCC_OK) {
            result = st;
            ctx->last_error = L->last_error;
            break;
        }
        // input copies run one chunk after another (a chunk's copy does not
        // share the link with the next one's), overlapping the kernels
        e = c > 0 ? cudaStreamWaitEvent(L->stream, ctx->lane_in[(c - 1) % HOST_LANES], 0) : cudaSuccess;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(L->in_org.p, org_tmin + 4 * c0, m * 16, cudaMemcpyHostToDevice, L->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(L->in_dir.p, dir_tmax + 4 * c0, m * 16, cudaMemcpyHostToDevice, L->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->lane_in[c % HOST_LANES], L->stream);
        if (e != cudaSuccess) {
            result = cuda_fail(ctx, e, "host-to-device copy of rays");
            break;
        }
        hcc_rays r{static_cast<float *>(L->in_org.p), static_cast<float *>(L->in_dir.p), m};
        if ((st = hcc_run(L, method, bvh, cut, &r, key_bits, any_hit, static_cast<hcc_hit *>(L->hits.p))) != HCC_OK) {
            result = st;
            ctx->last_error = L->last_error;
            break;
        }
        e = cudaMemcpyAsync(hits + c0, L->hits.p, m * sizeof(hcc_hit), cudaMemcpyDeviceToHost, L->stream);
        if (e != cudaSuccess) {
            result = cuda_fail(ctx, e, "device-to-host copy of hits");
            break;
        }
    }
    for (hcc_ctx *L : ctx->lane) {  // always drain every lane and read its error word
        st = hcc_sync(L);
        if (st != HCC_OK && result == HCC_OK) {
            result = st;
            ctx->last_error = L->last_error;
        }
    }
    return result;
}

}  // extern "C"
