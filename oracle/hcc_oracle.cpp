// CPU oracle for the hierarchy-cut-code hot path (Xiang et al.,
// "Faster Ray Tracing through Hierarchy Cut Code", arXiv 2305.16652).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
// restatement of what the method computes, written from the paper.  It is
// called only by the tests, by __graft_entry__.smoke() and by the benchmark's
// CPU-baseline / reference leg.  The product library never links, loads or
// calls it, and it shares no code, header or table with the CUDA path.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fno-fast-math (no FMA
// contraction: every fused multiply-add below is an explicit std::fma).
//
// Contents, each citing the passage it follows:
//   oracle_surface_area   SA term of Eq. 1
//   oracle_had            hierarchically accumulated density, Eq. 1 (Sec. 4.2.2)
//   oracle_select_cut     cut-node search, Algorithm 2, ordered by HAD (Sec. 4.2.2)
//   oracle_encode_hcc     hierarchy cut code, Algorithm 1 (Sec. 4.2.1); bit
//                         order as in the worked example of the SpaceAnchor figure
//   oracle_key_margin     distance of a ray from flipping any HCC bit
//   oracle_select_cut_ml  two-level cut of the multi-level HCC, Algorithm 3 (Sec. 4.3)
//   oracle_encode_mlhcc   multi-level hierarchy cut code (Sec. 4.3)
//   oracle_grid_cells     regular grid encoding's cells (Sec. 5; encoded by
//                         oracle_encode_hcc with the cells as the cut)
//   oracle_encode_ppc     prefix path code (Sec. 4.1)
//   oracle_encode_twopoint  TwoPoint key (Sec. 3.2 "Two Point", Sec. 5:
//                         fixed-length termination estimate 0.25 x largest extent)
//   oracle_encode_origin  Origin key: 3D Morton code of the ray origin (Sec. 3.2 "Origin")
//   oracle_encode_origin_dir  Origin-Direction key (Sec. 3.2, after Reis et al.):
//                         origin Morton code in the high bits, a Morton code
//                         of the octahedral parametrisation of the direction
//                         in the low bits
//   oracle_spawn          next-bounce diffuse rays (wavefront path tracing,
//                         Sec. 5 pipeline; the definition is the one stated
//                         for hcc_batch_spawn, restated here independently)
//   oracle_stable_sort    sort keys as natural numbers (Sec. 4.2.3 "Sorting",
//                         Sec. 5: sort of ray indices)
//   oracle_gather         rays fetched through the sorted indices (Sec. 5)
//   oracle_intersect      Moller-Trumbore ray/triangle test (1997)
//   oracle_trace_brute    closest hit by definition: argmin over all triangles
//   oracle_trace_bvh      same result through the BVH2 (Sec. 3.1), as a faster
//                         way to evaluate the definition
//
// Readings where the paper is silent (each also listed in the design notes):
//  * slab test: inclusive (tnear <= tfar) over the ray interval [tmin, tmax];
//    per axis t = (bound - o) * (1/d) with IEEE division, NaN (0 * inf when
//    the origin lies on a slab plane of a zero direction component) ignored
//    by fminf/fmaxf, i.e. touching counts;
//  * HAD in double, evaluated as (HAD_l + HAD_r) + lambda * SA; ties in the
//    priority queue broken by lower node index;
//  * key bit (k-1-r) <- cut node r for r < min(cut size, k); other bits 0;
//  * TwoPoint: b = floor(k/6) bits per coordinate, interleaved MSB-first in
//    the order o.x o.y o.z t.x t.y t.z, left-justified in k bits;
//  * Origin: b = floor(k/3) bits per axis, MSB-first in the order x y z,
//    left-justified; origin normalised to the scene box as for TwoPoint;
//  * Origin-Direction: bd = floor(k/6) bits per direction coordinate, bo =
//    floor((k - 2 bd)/3) bits per origin axis; direction parametrised by the
//    octahedral map (L1-normalise, fold the lower hemisphere), u = x/2 + 1/2;
//  * sort: stable and ascending on all k key bits;
//  * closest hit: lexicographic minimum of (t, triangle id) over every
//    triangle with a Moller-Trumbore hit and tmin < t < tmax.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <queue>
#include <vector>

namespace {

struct V3 {
    float x, y, z;
};

inline V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
// Canonical dot and cross products: the same fused operations in the same
// order on every platform (std::fma is the correctly rounded fused op).
inline float dot(V3 a, V3 b) { return std::fma(a.z, b.z, std::fma(a.y, b.y, a.x * b.x)); }
inline V3 cross(V3 a, V3 b) {
    return {std::fma(a.y, b.z, -(a.z * b.y)), std::fma(a.z, b.x, -(a.x * b.z)), std::fma(a.x, b.y, -(a.y * b.x))};
}

struct Hit {
    int32_t prim;
    float t, u, v;
};

inline bool closer(float t, int32_t prim, const Hit &h) {
    return h.prim < 0 || t < h.t || (t == h.t && prim < h.prim);
}

}  // namespace

extern "C" {

// Surface area of an axis-aligned box, the SA term of Eq. 1, evaluated in
// double from the float extents.
double oracle_surface_area(const float *lo, const float *hi) {
    double ex = (double)hi[0] - (double)lo[0];
    double ey = (double)hi[1] - (double)lo[1];
    double ez = (double)hi[2] - (double)lo[2];
    return 2.0 * (ex * ey + ey * ez + ez * ex);
}

// Eq. 1: HAD_n = TC_n * SA_n for a leaf; HAD_left + HAD_right + lambda * SA_n
// otherwise.  Nodes are given as parallel arrays; left[n] < 0 marks a leaf.
// Children may have any index; the recursion below follows the definition.
static double had_rec(uint32_t n, const float *lo, const float *hi, const int32_t *left, const int32_t *right,
                      const uint32_t *count, double lambda, double *had) {
    double sa = oracle_surface_area(lo + 3 * n, hi + 3 * n);
    double h;
    if (left[n] < 0) {
        h = (double)count[n] * sa;
    } else {
        double hl = had_rec((uint32_t)left[n], lo, hi, left, right, count, lambda, had);
        double hr = had_rec((uint32_t)right[n], lo, hi, left, right, count, lambda, had);
        h = (hl + hr) + lambda * sa;
    }
    had[n] = h;
    return h;
}

void oracle_had(uint32_t num_nodes, const float *lo, const float *hi, const int32_t *left, const int32_t *right,
                const uint32_t *count, double lambda, double *had) {
    if (num_nodes == 0) return;
    had_rec(0, lo, hi, left, right, count, lambda, had);
}

// Algorithm 2 (Sec. 4.2.2), with the priority of Eq. 1:
//   MaxQueueSize <- cut_size; PriorityQueue <- {root}
//   while |PriorityQueue| < MaxQueueSize:
//       pop the head (largest HAD); a leaf goes to the cut list and
//       MaxQueueSize decreases by one; otherwise push both children
//   the cut is the cut list plus everything left in the queue.
// The cut is then ordered by HAD, descending (Sec. 4.2.2, last paragraph), so
// that cut_out[r] is the node behind key bit r counted from the most
// significant end.  The loop also stops when the queue empties (the tree has
// fewer leaves than cut_size).  Returns the cut size.
uint32_t oracle_select_cut(uint32_t num_nodes, const float *lo, const float *hi, const int32_t *left,
                           const int32_t *right, const uint32_t *count, uint32_t cut_size, double lambda,
                           int32_t *cut_out) {
    if (num_nodes == 0 || cut_size == 0) return 0;
    std::vector<double> had(num_nodes);
    oracle_had(num_nodes, lo, hi, left, right, count, lambda, had.data());
    // head of the queue: larger HAD first, then lower node index
    auto lower_priority = [&](int32_t a, int32_t b) {
        if (had[a] != had[b]) return had[a] < had[b];
        return a > b;
    };
    std::priority_queue<int32_t, std::vector<int32_t>, decltype(lower_priority)> pq(lower_priority);
    std::vector<int32_t> cut;
    uint32_t max_queue = cut_size;
    pq.push(0);
    while (!pq.empty() && pq.size() < max_queue) {
        int32_t node = pq.top();
        pq.pop();
        if (left[node] < 0) {
            cut.push_back(node);
            max_queue -= 1;
        } else {
            pq.push(left[node]);
            pq.push(right[node]);
        }
    }
    while (!pq.empty()) {
        cut.push_back(pq.top());
        pq.pop();
    }
    std::sort(cut.begin(), cut.end(), [&](int32_t a, int32_t b) {
        if (had[a] != had[b]) return had[a] > had[b];
        return a < b;
    });
    for (size_t i = 0; i < cut.size(); ++i) cut_out[i] = cut[i];
    return (uint32_t)cut.size();
}

// Ray / box slab test on the ray interval [tmin, tmax]; returns tnear, tfar.
static void slab(const float *o, const float *inv, float tmin, float tmax, const float *lo, const float *hi,
                 float *tnear, float *tfar) {
    float tn[3], tf[3];
    for (int a = 0; a < 3; ++a) {
        float t0 = (lo[a] - o[a]) * inv[a];
        float t1 = (hi[a] - o[a]) * inv[a];
        tn[a] = std::fmin(t0, t1);
        tf[a] = std::fmax(t0, t1);
    }
    *tnear = std::fmax(std::fmax(tn[0], tn[1]), std::fmax(tn[2], tmin));
    *tfar = std::fmin(std::fmin(tf[0], tf[1]), std::fmin(tf[2], tmax));
}

// Algorithm 1 (Sec. 4.2.1): for every ray, intersect it with every cut node
// and record each result as one key bit.  cut_lo/cut_hi hold ncut boxes in
// key order (HAD descending); node r drives bit (key_bits - 1 - r), so node 0
// is the most significant bit, as in the SpaceAnchor figure's worked codes.
// Rays are float4 (ox, oy, oz, tmin) and (dx, dy, dz, tmax).
void oracle_encode_hcc(uint64_t n, const float *org, const float *dir, uint32_t ncut, const float *cut_lo,
                       const float *cut_hi, uint32_t key_bits, uint64_t *keys) {
    uint32_t used = std::min(ncut, key_bits);
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        float inv[3] = {1.0f / d[0], 1.0f / d[1], 1.0f / d[2]};
        uint64_t key = 0;
        for (uint32_t r = 0; r < used; ++r) {
            float tnear, tfar;
            slab(o, inv, o[3], d[3], cut_lo + 3 * r, cut_hi + 3 * r, &tnear, &tfar);
            if (tnear <= tfar) key |= (uint64_t)1 << (key_bits - 1 - r);
        }
        keys[i] = key;
    }
}

// For each ray, the smallest relative gap |tfar - tnear| / max(1, |tnear|,
// |tfar|) over the cut nodes that drive key bits.  A ray whose gap is below
// 1e-6 sits on a box boundary and could flip a bit under any rounding change.
void oracle_key_margin(uint64_t n, const float *org, const float *dir, uint32_t ncut, const float *cut_lo,
                       const float *cut_hi, uint32_t key_bits, double *margin) {
    uint32_t used = std::min(ncut, key_bits);
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        float inv[3] = {1.0f / d[0], 1.0f / d[1], 1.0f / d[2]};
        double m = INFINITY;
        for (uint32_t r = 0; r < used; ++r) {
            float tnear, tfar;
            slab(o, inv, o[3], d[3], cut_lo + 3 * r, cut_hi + 3 * r, &tnear, &tfar);
            if (std::isinf(tnear) || std::isinf(tfar) || std::isnan(tnear) || std::isnan(tfar)) continue;
            double g = std::fabs((double)tfar - (double)tnear) /
                       std::max(1.0, std::max(std::fabs((double)tnear), std::fabs((double)tfar)));
            m = std::min(m, g);
        }
        margin[i] = m;
    }
}

// TwoPoint key (Sec. 3.2; Sec. 5 fixes the termination estimate to a ray
// length of 0.25 of the largest extent of the scene box).  Each of the six
// coordinates of (origin, estimated termination) is normalised to the scene
// box, quantised to b = floor(k/6) bits and the bits are interleaved from the
// most significant level down (Morton order).
// The estimated ray length is `fraction` of the largest extent (App. B
// sweeps it; Sec. 5 uses 0.25, the value oracle_encode_twopoint passes).
void oracle_encode_twopoint_frac(uint64_t n, const float *org, const float *dir, const float *scene_lo,
                                 const float *scene_hi, float fraction, uint32_t key_bits, uint64_t *keys) {
    float ext[3] = {scene_hi[0] - scene_lo[0], scene_hi[1] - scene_lo[1], scene_hi[2] - scene_lo[2]};
    float L = fraction * std::fmax(ext[0], std::fmax(ext[1], ext[2]));
    uint32_t b = key_bits / 6;
    double levels = std::ldexp(1.0, (int)b);
    uint32_t qmax = (b == 0) ? 0u : ((1u << b) - 1u);
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        float p[6] = {o[0], o[1], o[2], std::fma(L, d[0], o[0]), std::fma(L, d[1], o[1]), std::fma(L, d[2], o[2])};
        uint32_t q[6];
        for (int c = 0; c < 6; ++c) {
            int a = c % 3;
            float u = (ext[a] == 0.0f) ? 0.0f : (p[c] - scene_lo[a]) / ext[a];
            u = std::fmin(std::fmax(u, 0.0f), 1.0f);
            float s = u * (float)levels;  // exact: levels is a power of two
            uint32_t qi = (uint32_t)s;
            q[c] = std::min(qi, qmax);
        }
        uint64_t key = 0;
        for (int j = (int)b - 1; j >= 0; --j)
            for (int c = 0; c < 6; ++c) key = (key << 1) | ((q[c] >> j) & 1u);
        if (key_bits > 6 * b) key <<= (key_bits - 6 * b);
        keys[i] = key;
    }
}

void oracle_encode_twopoint(uint64_t n, const float *org, const float *dir, const float *scene_lo,
                            const float *scene_hi, uint32_t key_bits, uint64_t *keys) {
    oracle_encode_twopoint_frac(n, org, dir, scene_lo, scene_hi, 0.25f, key_bits, keys);
}

// ------------------------------------------------ method variants (Sec. 4.1, 4.3, 5)

// Number of leaves under node n.
static uint32_t leaves_under(int32_t n, const int32_t *left, const int32_t *right) {
    if (left[n] < 0) return 1;
    return leaves_under(left[n], left, right) + leaves_under(right[n], left, right);
}

// Algorithm 2 run on the subtree of `start` (the low-level cut of one top
// node of MLHCC): the same queue discipline as oracle_select_cut, result in
// HAD order.
static std::vector<int32_t> cut_of_subtree(int32_t start, uint32_t size, const std::vector<double> &had,
                                           const int32_t *left, const int32_t *right) {
    auto lower_priority = [&](int32_t a, int32_t b) {
        if (had[a] != had[b]) return had[a] < had[b];
        return a > b;
    };
    std::priority_queue<int32_t, std::vector<int32_t>, decltype(lower_priority)> pq(lower_priority);
    std::vector<int32_t> cut;
    uint32_t max_queue = size;
    pq.push(start);
    while (!pq.empty() && pq.size() < max_queue) {
        int32_t node = pq.top();
        pq.pop();
        if (left[node] < 0) {
            cut.push_back(node);
            max_queue -= 1;
        } else {
            pq.push(left[node]);
            pq.push(right[node]);
        }
    }
    while (!pq.empty()) {
        cut.push_back(pq.top());
        pq.pop();
    }
    std::sort(cut.begin(), cut.end(), [&](int32_t a, int32_t b) {
        if (had[a] != had[b]) return had[a] > had[b];
        return a < b;
    });
    return cut;
}

// Two-level cut of the multi-level hierarchy cut code (Sec. 4.3, Algorithm 3).
// A node may be a top-level cut node only if its subtree can supply low_size
// low-level nodes, i.e. it holds at least low_size leaves; Algorithm 3
// discards the others.  Reading: the top level is Algorithm 2 on the tree of
// such eligible nodes -- pop the largest-HAD node, push its eligible children
// (an ineligible child and its subtree are discarded), and a node with no
// eligible child goes to the cut list as a leaf does in Algorithm 2 -- until
// the queue plus the list hold top_size nodes.  Every top node t then gets
// the cut of its own subtree by Algorithm 2 with low_size nodes.  Outputs:
// top_out[r] (HAD order, r < returned count) and low_out[r * low_size + j]
// (node j of top node r's low cut, HAD order).  Returns the number of top
// nodes (0 when the root itself has fewer than low_size leaves).
uint32_t oracle_select_cut_ml(uint32_t num_nodes, const float *lo, const float *hi, const int32_t *left,
                              const int32_t *right, const uint32_t *count, uint32_t top_size, uint32_t low_size,
                              double lambda, int32_t *top_out, int32_t *low_out) {
    if (num_nodes == 0 || top_size == 0 || low_size == 0) return 0;
    std::vector<double> had(num_nodes);
    oracle_had(num_nodes, lo, hi, left, right, count, lambda, had.data());
    auto eligible = [&](int32_t n) { return leaves_under(n, left, right) >= low_size; };
    auto lower_priority = [&](int32_t a, int32_t b) {
        if (had[a] != had[b]) return had[a] < had[b];
        return a > b;
    };
    std::priority_queue<int32_t, std::vector<int32_t>, decltype(lower_priority)> pq(lower_priority);
    std::vector<int32_t> top;
    uint32_t max_queue = top_size;
    if (eligible(0)) pq.push(0);
    while (!pq.empty() && pq.size() < max_queue) {
        int32_t node = pq.top();
        pq.pop();
        std::vector<int32_t> kids;
        if (left[node] >= 0) {
            if (eligible(left[node])) kids.push_back(left[node]);
            if (eligible(right[node])) kids.push_back(right[node]);
        }
        if (kids.empty()) {
            top.push_back(node);
            max_queue -= 1;
        } else {
            for (int32_t c : kids) pq.push(c);
        }
    }
    while (!pq.empty()) {
        top.push_back(pq.top());
        pq.pop();
    }
    std::sort(top.begin(), top.end(), [&](int32_t a, int32_t b) {
        if (had[a] != had[b]) return had[a] > had[b];
        return a < b;
    });
    for (size_t r = 0; r < top.size(); ++r) {
        top_out[r] = top[r];
        std::vector<int32_t> low = cut_of_subtree(top[r], low_size, had, left, right);
        for (uint32_t j = 0; j < low_size; ++j) low_out[r * low_size + j] = low[j];
    }
    return (uint32_t)top.size();
}

// Multi-level hierarchy cut code (Sec. 4.3): the top field (top_field bits,
// most significant) holds one bit per top node as in Algorithm 1; the
// representative is the first top node in HAD order that the ray meets
// (Sec. 4.3: the intersected top node of highest HAD), and the next
// low_field bits hold the ray's results against that node's low-level cut.
// A ray that meets no top node has an empty low field.  ntop top boxes,
// ntop * low_field low boxes (row r = top node r); top_field + low_field <=
// key_bits, remaining low bits 0.
void oracle_encode_mlhcc(uint64_t n, const float *org, const float *dir, uint32_t top_field, uint32_t ntop,
                         const float *top_lo, const float *top_hi, uint32_t low_field, const float *low_lo,
                         const float *low_hi, uint32_t key_bits, uint64_t *keys) {
    uint32_t used_top = std::min(ntop, top_field);
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        float inv[3] = {1.0f / d[0], 1.0f / d[1], 1.0f / d[2]};
        uint64_t key = 0;
        int rep = -1;
        for (uint32_t r = 0; r < used_top; ++r) {
            float tnear, tfar;
            slab(o, inv, o[3], d[3], top_lo + 3 * r, top_hi + 3 * r, &tnear, &tfar);
            if (tnear <= tfar) {
                key |= (uint64_t)1 << (key_bits - 1 - r);
                if (rep < 0) rep = (int)r;
            }
        }
        if (rep >= 0) {
            for (uint32_t j = 0; j < low_field; ++j) {
                const size_t b = (size_t)rep * low_field + j;
                float tnear, tfar;
                slab(o, inv, o[3], d[3], low_lo + 3 * b, low_hi + 3 * b, &tnear, &tfar);
                if (tnear <= tfar) key |= (uint64_t)1 << (key_bits - 1 - top_field - j);
            }
        }
        keys[i] = key;
    }
}

// Regular grid encoding (Sec. 5): the cut boxes of HCC replaced by cells that
// divide the scene box evenly.  Reading: the cell count is the largest power
// of two not above max_cells; starting from one cell, the axis whose cells
// are longest (first axis on ties) is halved until that count is reached.
// Cell boundary i of g along an axis is ((g - i) lo + i hi) / g evaluated in
// double and rounded to float, so the outer boundaries are lo and hi exactly
// and neighbouring cells share their face.  Cell (i, j, l) is number
// (i gy + j) gz + l and drives key bit (k - 1 - number).  Writes the cell
// boxes and dims; returns the cell count.
uint32_t oracle_grid_cells(const float *scene_lo, const float *scene_hi, uint32_t max_cells, float *cell_lo,
                           float *cell_hi, uint32_t *dims) {
    if (max_cells == 0) return 0;
    uint32_t g[3] = {1, 1, 1};
    uint32_t cells = 1;
    while (cells * 2 <= max_cells) {
        int best = 0;
        double best_len = -1.0;
        for (int a = 0; a < 3; ++a) {
            double len = ((double)scene_hi[a] - (double)scene_lo[a]) / g[a];
            if (len > best_len) {
                best_len = len;
                best = a;
            }
        }
        g[best] *= 2;
        cells *= 2;
    }
    auto bound = [&](int a, uint32_t i) {
        return (float)(((double)(g[a] - i) * (double)scene_lo[a] + (double)i * (double)scene_hi[a]) / (double)g[a]);
    };
    uint32_t r = 0;
    for (uint32_t i = 0; i < g[0]; ++i)
        for (uint32_t j = 0; j < g[1]; ++j)
            for (uint32_t l = 0; l < g[2]; ++l, ++r) {
                const uint32_t c[3] = {i, j, l};
                for (int a = 0; a < 3; ++a) {
                    cell_lo[3 * r + a] = bound(a, c[a]);
                    cell_hi[3 * r + a] = bound(a, c[a] + 1);
                }
            }
    for (int a = 0; a < 3; ++a) dims[a] = g[a];
    return cells;
}

// Prefix path code (Sec. 4.1): the results of the first k box tests of a
// traversal that every ray makes in the same fixed order.  Reading: the order
// is depth-first pre-order from the root, left child before right; a node
// whose box the ray meets is followed into its children, a missed node's
// subtree is skipped, and no test is skipped for a found hit (the path does
// not depend on hits).  Test number m drives bit (k - 1 - m); a traversal
// that ends before k tests leaves the remaining bits 0.
static void ppc_visit(int32_t node, const float *o, const float *inv, float tmin, float tmax, const float *lo,
                      const float *hi, const int32_t *left, const int32_t *right, uint32_t key_bits, uint32_t *m,
                      uint64_t *key) {
    if (*m >= key_bits) return;
    float tnear, tfar;
    slab(o, inv, tmin, tmax, lo + 3 * node, hi + 3 * node, &tnear, &tfar);
    const bool met = tnear <= tfar;
    if (met) *key |= (uint64_t)1 << (key_bits - 1 - *m);
    *m += 1;
    if (met && left[node] >= 0) {
        ppc_visit(left[node], o, inv, tmin, tmax, lo, hi, left, right, key_bits, m, key);
        ppc_visit(right[node], o, inv, tmin, tmax, lo, hi, left, right, key_bits, m, key);
    }
}

void oracle_encode_ppc(uint64_t n, const float *org, const float *dir, uint32_t num_nodes, const float *lo,
                       const float *hi, const int32_t *left, const int32_t *right, uint32_t key_bits,
                       uint64_t *keys) {
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        float inv[3] = {1.0f / d[0], 1.0f / d[1], 1.0f / d[2]};
        uint64_t key = 0;
        uint32_t m = 0;
        if (num_nodes > 0) ppc_visit(0, o, inv, o[3], d[3], lo, hi, left, right, key_bits, &m, &key);
        keys[i] = key;
    }
}

// Quantise coordinate p of the scene box [lo, lo + ext] to bits b
// (normalise, clamp to [0, 1], scale by 2^b, truncate, cap at 2^b - 1).
static uint32_t quantise(float p, float lo, float ext, uint32_t b) {
    if (b == 0) return 0;
    float u = (ext == 0.0f) ? 0.0f : (p - lo) / ext;
    u = std::fmin(std::fmax(u, 0.0f), 1.0f);
    uint32_t q = (uint32_t)(u * (float)std::ldexp(1.0, (int)b));
    uint32_t qmax = (1u << b) - 1u;
    return std::min(q, qmax);
}

// Morton interleave of m coordinates of b bits each, most significant level
// first, coordinates in the given order.
static uint64_t interleave(const uint32_t *q, int m, uint32_t b) {
    uint64_t key = 0;
    for (int j = (int)b - 1; j >= 0; --j)
        for (int c = 0; c < m; ++c) key = (key << 1) | ((q[c] >> j) & 1u);
    return key;
}

// Origin key (Sec. 3.2 "Origin"): 3D Morton code of the origin in the scene
// box, b = floor(k/3) bits per axis, left-justified in k bits.
void oracle_encode_origin(uint64_t n, const float *org, const float *scene_lo, const float *scene_hi,
                          uint32_t key_bits, uint64_t *keys) {
    float ext[3] = {scene_hi[0] - scene_lo[0], scene_hi[1] - scene_lo[1], scene_hi[2] - scene_lo[2]};
    uint32_t b = key_bits / 3;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) q[a] = quantise(org[4 * i + a], scene_lo[a], ext[a], b);
        uint64_t key = interleave(q, 3, b);
        if (key_bits > 3 * b) key <<= (key_bits - 3 * b);
        keys[i] = key;
    }
}

// Octahedral parametrisation of a direction onto [0, 1]^2: divide by the L1
// norm, fold the lower hemisphere (z < 0) over the diagonals, map [-1, 1] to
// [0, 1].  A zero direction maps to the centre.
void oracle_octahedral(const float *d, float *u, float *v) {
    float s = (std::fabs(d[0]) + std::fabs(d[1])) + std::fabs(d[2]);
    if (!(s > 0.0f)) {
        *u = 0.5f;
        *v = 0.5f;
        return;
    }
    float nx = d[0] / s, ny = d[1] / s, nz = d[2] / s;
    float x = nx, y = ny;
    if (nz < 0.0f) {
        x = (1.0f - std::fabs(ny)) * (nx >= 0.0f ? 1.0f : -1.0f);
        y = (1.0f - std::fabs(nx)) * (ny >= 0.0f ? 1.0f : -1.0f);
    }
    *u = x * 0.5f + 0.5f;
    *v = y * 0.5f + 0.5f;
}

// Origin-Direction key (Sec. 3.2, Reis et al.): origin Morton code (bo bits
// per axis) in the high bits, direction Morton code (bd bits per octahedral
// coordinate) in the low bits, bd = floor(k/6), bo = floor((k - 2 bd)/3),
// left-justified in k bits.
void oracle_encode_origin_dir(uint64_t n, const float *org, const float *dir, const float *scene_lo,
                              const float *scene_hi, uint32_t key_bits, uint64_t *keys) {
    float ext[3] = {scene_hi[0] - scene_lo[0], scene_hi[1] - scene_lo[1], scene_hi[2] - scene_lo[2]};
    uint32_t bd = key_bits / 6, bo = (key_bits - 2 * bd) / 3;
    for (uint64_t i = 0; i < n; ++i) {
        uint32_t qo[3], qd[2];
        for (int a = 0; a < 3; ++a) qo[a] = quantise(org[4 * i + a], scene_lo[a], ext[a], bo);
        float u, v;
        oracle_octahedral(dir + 4 * i, &u, &v);
        qd[0] = quantise(u, 0.0f, 1.0f, bd);
        qd[1] = quantise(v, 0.0f, 1.0f, bd);
        uint64_t key = (interleave(qo, 3, bo) << (2 * bd)) | interleave(qd, 2, bd);
        uint32_t used = 3 * bo + 2 * bd;
        if (key_bits > used) key <<= (key_bits - used);
        keys[i] = key;
    }
}

// Average number of distinct codes per warp (Sec. 6.5, Table 6): the keys in
// sorted order cut into consecutive groups of 32 rays; the mean number of
// distinct keys per group (the last group may be shorter).
double oracle_anc(uint64_t n, const uint64_t *keys, const uint32_t *perm) {
    if (n == 0) return 0.0;
    uint64_t groups = 0, distinct = 0;
    for (uint64_t g = 0; g < n; g += 32) {
        std::vector<uint64_t> w;
        for (uint64_t j = g; j < std::min<uint64_t>(g + 32, n); ++j) w.push_back(keys[perm[j]]);
        std::sort(w.begin(), w.end());
        distinct += (uint64_t)(std::unique(w.begin(), w.end()) - w.begin());
        ++groups;
    }
    return (double)distinct / (double)groups;
}

static uint64_t splitmix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Uniform number j of ray i: the top 24 bits of SplitMix64(SplitMix64(seed)
// ^ (64 i + j)) scaled by 2^-24.
static float uniform24(uint64_t seed_mixed, uint64_t i, uint32_t j) {
    uint64_t z = splitmix(seed_mixed ^ (i * 64u + j));
    return (float)(uint32_t)(z >> 40) * 5.9604644775390625e-08f;
}

// Next bounce: a ray that hit triangle p at distance t spawns a diffuse ray
// from o + t d, cosine-weighted about the triangle's unit normal turned
// toward the incoming ray (a point of the unit disk by rejection, lifted to
// the hemisphere, in the orthonormal basis of Duff et al. 2017); a miss
// becomes the empty ray [1, 0] at the old origin.  tris: the scene's
// triangles (v0, v1, v2); hits: records {prim, t, u, v}.  Ray k of the call
// is ray first_index + k of its batch (the index keys its random numbers).
void oracle_spawn(uint64_t n, const float *org, const float *dir, const void *hits_in, const float *tris,
                  uint32_t ntris, uint64_t seed, float tmin, uint64_t first_index, float *out_org, float *out_dir) {
    const Hit *hits = (const Hit *)hits_in;
    const uint64_t sm = splitmix(seed);
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        const Hit h = hits[i];
        if (h.prim < 0 || (uint32_t)h.prim >= ntris) {
            out_org[4 * i] = o[0];
            out_org[4 * i + 1] = o[1];
            out_org[4 * i + 2] = o[2];
            out_org[4 * i + 3] = 1.0f;
            out_dir[4 * i] = d[0];
            out_dir[4 * i + 1] = d[1];
            out_dir[4 * i + 2] = d[2];
            out_dir[4 * i + 3] = 0.0f;
            continue;
        }
        const float *T = tris + 9 * (uint64_t)h.prim;
        V3 v0{T[0], T[1], T[2]}, v1{T[3], T[4], T[5]}, v2{T[6], T[7], T[8]};
        V3 nrm = cross(sub(v1, v0), sub(v2, v0));
        float len = std::sqrt(dot(nrm, nrm));
        if (len > 0.0f)
            nrm = {nrm.x / len, nrm.y / len, nrm.z / len};
        else
            nrm = {0.0f, 0.0f, 1.0f};
        V3 dv{d[0], d[1], d[2]};
        if (dot(nrm, dv) > 0.0f) nrm = {-nrm.x, -nrm.y, -nrm.z};
        float x = 0.0f, y = 0.0f, r2 = 0.0f;
        for (uint32_t a = 0; a < 16; ++a) {
            float cx = 2.0f * uniform24(sm, first_index + i, 2 * a) - 1.0f;
            float cy = 2.0f * uniform24(sm, first_index + i, 2 * a + 1) - 1.0f;
            float c2 = std::fma(cy, cy, cx * cx);
            if (c2 <= 1.0f) {
                x = cx;
                y = cy;
                r2 = c2;
                break;
            }
        }
        float z = std::sqrt(std::fmax(0.0f, 1.0f - r2));
        float sign = std::copysign(1.0f, nrm.z);
        float aa = -1.0f / (sign + nrm.z);
        float bb = (nrm.x * nrm.y) * aa;
        V3 b1{1.0f + ((sign * nrm.x) * nrm.x) * aa, sign * bb, -(sign * nrm.x)};
        V3 b2{bb, sign + (nrm.y * nrm.y) * aa, -nrm.y};
        float t = h.t;
        out_org[4 * i] = std::fma(t, d[0], o[0]);
        out_org[4 * i + 1] = std::fma(t, d[1], o[1]);
        out_org[4 * i + 2] = std::fma(t, d[2], o[2]);
        out_org[4 * i + 3] = tmin;
        out_dir[4 * i] = std::fma(z, nrm.x, std::fma(y, b2.x, x * b1.x));
        out_dir[4 * i + 1] = std::fma(z, nrm.y, std::fma(y, b2.y, x * b1.y));
        out_dir[4 * i + 2] = std::fma(z, nrm.z, std::fma(y, b2.z, x * b1.z));
        out_dir[4 * i + 3] = INFINITY;
    }
}

// Rays sorted by key as natural numbers (Sec. 4.2.3), realised as a stable
// sort of ray indices (Sec. 5); equal keys keep their input order.
void oracle_stable_sort(uint64_t n, const uint64_t *keys, uint32_t *perm) {
    std::vector<uint32_t> idx(n);
    for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
    for (uint64_t i = 0; i < n; ++i) perm[i] = idx[i];
}

// The trace fetches rays through the sorted indices (Sec. 5):
// out[j] = in[perm[j]].
void oracle_gather(uint64_t n, const float *in_org, const float *in_dir, const uint32_t *perm, float *out_org,
                   float *out_dir) {
    for (uint64_t j = 0; j < n; ++j) {
        std::memcpy(out_org + 4 * j, in_org + 4 * (uint64_t)perm[j], 16);
        std::memcpy(out_dir + 4 * j, in_dir + 4 * (uint64_t)perm[j], 16);
    }
}

// Moller-Trumbore (Moller & Trumbore 1997), two-sided, no epsilon:
// p = d x e2, det = e1 . p (0 -> miss), s = o - v0, u = (s . p) / det,
// q = s x e1, v = (d . q) / det, t = (e2 . q) / det, hit when u >= 0,
// v >= 0, u + v <= 1 and tmin < t < tmax.  e1, e2 are v1 - v0, v2 - v0
// rounded to float.  Returns 1 on a hit.
int oracle_intersect(const float *o3, const float *d3, float tmin, float tmax, const float *tri, float *t_out,
                     float *u_out, float *v_out) {
    V3 o{o3[0], o3[1], o3[2]}, d{d3[0], d3[1], d3[2]};
    V3 v0{tri[0], tri[1], tri[2]}, v1{tri[3], tri[4], tri[5]}, v2{tri[6], tri[7], tri[8]};
    V3 e1 = sub(v1, v0), e2 = sub(v2, v0);
    V3 p = cross(d, e2);
    float det = dot(e1, p);
    if (det == 0.0f) return 0;
    float inv = 1.0f / det;
    V3 s = sub(o, v0);
    float u = dot(s, p) * inv;
    if (u < 0.0f || u > 1.0f) return 0;
    V3 q = cross(s, e1);
    float v = dot(d, q) * inv;
    if (v < 0.0f || u + v > 1.0f) return 0;
    float t = dot(e2, q) * inv;
    if (!(t > tmin && t < tmax)) return 0;
    *t_out = t;
    *u_out = u;
    *v_out = v;
    return 1;
}

// Closest hit by its definition: every triangle is tested; the hit with the
// smallest t wins, ties to the lower triangle id.  any_hit != 0 stops at the
// first hit in triangle order.  hits: n records {prim, t, u, v}, prim = -1
// and t = +inf for a miss.
void oracle_trace_brute(uint32_t ntris, const float *tri_v, uint64_t n, const float *org, const float *dir,
                        int any_hit, void *hits_out) {
    Hit *hits = (Hit *)hits_out;
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        Hit h{-1, INFINITY, 0.0f, 0.0f};
        for (uint32_t k = 0; k < ntris; ++k) {
            float t, u, v;
            if (!oracle_intersect(o, d, o[3], d[3], tri_v + 9 * (uint64_t)k, &t, &u, &v)) continue;
            if (closer(t, (int32_t)k, h)) h = Hit{(int32_t)k, t, u, v};
            if (any_hit) break;
        }
        hits[i] = h;
    }
}

// Conservative ray/box overlap in double precision: the box is widened by a
// relative 1e-5 and the interval by a relative 1e-4, so that no triangle
// inside the box whose float Moller-Trumbore t lies in the interval is ever
// skipped.  Only used to skip triangles faster; the answer is the same as
// oracle_trace_brute (checked by the tests).
static bool box_maybe_hit(const float *o, const float *d, double t0, double t1, const float *lo, const float *hi,
                          double *tnear_out) {
    double tn = t0, tf = t1;
    for (int a = 0; a < 3; ++a) {
        double pad = 1e-5 * (1.0 + std::max(std::fabs((double)lo[a]), std::fabs((double)hi[a])));
        double l = (double)lo[a] - pad, h = (double)hi[a] + pad;
        double oa = o[a], da = d[a];
        if (da == 0.0) {
            if (oa < l || oa > h) return false;
            continue;
        }
        double ta = (l - oa) / da, tb = (h - oa) / da;
        if (ta > tb) std::swap(ta, tb);
        tn = std::max(tn, ta);
        tf = std::min(tf, tb);
        if (tn > tf) return false;
    }
    *tnear_out = tn;
    return true;
}

// The same closest hit found through the BVH2 (Sec. 3.1): subtrees whose box
// the ray cannot reach before the current best hit are skipped.  Nodes in
// the arrays of oracle_had; order[first .. first+count) are a leaf's
// triangle ids (indices into tri_v).
void oracle_trace_bvh(uint32_t num_nodes, const float *lo, const float *hi, const int32_t *left,
                      const int32_t *right, const uint32_t *first, const uint32_t *count, const uint32_t *order,
                      const float *tri_v, uint64_t n, const float *org, const float *dir, int any_hit,
                      void *hits_out) {
    Hit *hits = (Hit *)hits_out;
    std::vector<int32_t> stack;
    for (uint64_t i = 0; i < n; ++i) {
        const float *o = org + 4 * i, *d = dir + 4 * i;
        Hit h{-1, INFINITY, 0.0f, 0.0f};
        double lo_t = (double)o[3] * (1.0 - 1e-4) - 1e-30;
        stack.clear();
        if (num_nodes) stack.push_back(0);
        bool done = false;
        while (!stack.empty() && !done) {
            int32_t node = stack.back();
            stack.pop_back();
            double hi_t = (h.prim < 0) ? (double)d[3] : (double)h.t;
            hi_t = hi_t * (1.0 + 1e-4) + 1e-30;
            double tn;
            if (!box_maybe_hit(o, d, lo_t, hi_t, lo + 3 * node, hi + 3 * node, &tn)) continue;
            if (left[node] >= 0) {
                stack.push_back(right[node]);
                stack.push_back(left[node]);
                continue;
            }
            for (uint32_t k = 0; k < count[node]; ++k) {
                uint32_t prim = order[first[node] + k];
                float t, u, v;
                if (!oracle_intersect(o, d, o[3], d[3], tri_v + 9 * (uint64_t)prim, &t, &u, &v)) continue;
                if (closer(t, (int32_t)prim, h)) h = Hit{(int32_t)prim, t, u, v};
                if (any_hit) {
                    done = true;
                    break;
                }
            }
        }
        hits[i] = h;
    }
}

}  // extern "C"
