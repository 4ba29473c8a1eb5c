/*
 * Seeded synthetic inputs for the hierarchy-cut-code hot path.
 *
 * This file produces the *inputs* of the method and nothing else: triangle
 * scenes, a binned-SAH BVH2 over them, primary visibility of a pinhole
 * camera (found by z-buffer rasterisation, not by ray tracing), and the
 * secondary (cosine-weighted diffuse bounce) and shadow rays that leave the
 * visible points.  It contains none of the method's arithmetic: no slab
 * test, no key encoding, no sort, no Moller-Trumbore, no BVH traversal.
 *
 * Every random number comes from one counter-based generator keyed by
 * (seed, purpose, index), so any element can be regenerated on its own and
 * the result does not depend on evaluation order or thread count.
 *
 * The scenes stand in for the paper's test scenes (Sec. 6: interiors with
 * dense detail clustered in small regions of a closed space, rendered at
 * 1920x1080 with 8 samples per pixel and two shadow rays per bounce).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ RNG */

/* SplitMix64 finaliser (Steele, Lea, Flood 2014) used as a hash. */
static inline uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t gen_rng_u64(uint64_t seed, uint64_t purpose, uint64_t index) {
    return mix64(mix64(mix64(seed) ^ (purpose * 0xD1B54A32D192ED03ull)) ^ index);
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double u01(uint64_t seed, uint64_t purpose, uint64_t index) {
    return (double)(gen_rng_u64(seed, purpose, index) >> 11) * (1.0 / 9007199254740992.0);
}

/* Standard normal by Box-Muller from two uniforms of the same stream. */
static inline double normal01(uint64_t seed, uint64_t purpose, uint64_t index) {
    double a = u01(seed, purpose, 2 * index);
    double b = u01(seed, purpose, 2 * index + 1);
    return sqrt(-2.0 * log(1.0 - a)) * cos(2.0 * M_PI * b);
}

enum {
    P_TRI_CENTRE = 1,
    P_TRI_DIR = 2,
    P_TRI_LEN = 3,
    P_CLUSTER = 10,
    P_INST_CLUSTER = 11,
    P_INST_TYPE = 12,
    P_INST_SCALE = 13,
    P_INST_YAW = 14,
    P_INST_POS = 15,
    P_INST_STACK = 16,
    P_INST_STACK_ON = 17,
    P_JITTER = 20,
    P_BOUNCE = 21,
    P_LIGHT_PICK = 22,
    P_LIGHT_POINT = 23,
};

/* ---------------------------------------------- scene: random triangles */

/*
 * n triangles whose centroids are uniform in the unit cube; each vertex sits
 * at centroid + l * w with w uniform on the unit sphere and l log-normal
 * (mu, sigma); the three offsets are re-centred so the centroid is exact.
 * out: n * 9 floats (v0, v1, v2).
 */
void gen_random_tris(uint64_t seed, uint32_t n, double mu, double sigma, float *out) {
    for (uint32_t i = 0; i < n; ++i) {
        double c[3], off[3][3], mean[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) c[a] = u01(seed, P_TRI_CENTRE, (uint64_t)i * 3 + a);
        for (int k = 0; k < 3; ++k) {
            uint64_t id = (uint64_t)i * 3 + k;
            double z = 1.0 - 2.0 * u01(seed, P_TRI_DIR, 2 * id);
            double ph = 2.0 * M_PI * u01(seed, P_TRI_DIR, 2 * id + 1);
            double r = sqrt(fmax(0.0, 1.0 - z * z));
            double l = exp(mu + sigma * normal01(seed, P_TRI_LEN, id));
            off[k][0] = l * r * cos(ph);
            off[k][1] = l * r * sin(ph);
            off[k][2] = l * z;
            for (int a = 0; a < 3; ++a) mean[a] += off[k][a] / 3.0;
        }
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) out[(size_t)i * 9 + k * 3 + a] = (float)(c[a] + off[k][a] - mean[a]);
    }
}

/* ------------------------------------------- scene: furnished interior */

typedef struct {
    float *v;      /* output triangles, 9 floats each */
    uint32_t n;    /* triangles written (or counted) */
    uint32_t cap;  /* capacity of v in triangles; writes beyond are counted only */
} TriSink;

static void sink_tri(TriSink *s, const double *a, const double *b, const double *c) {
    if (s->v && s->n < s->cap) {
        float *o = s->v + (size_t)s->n * 9;
        for (int k = 0; k < 3; ++k) {
            o[k] = (float)a[k];
            o[3 + k] = (float)b[k];
            o[6 + k] = (float)c[k];
        }
    }
    s->n++;
}

typedef struct {
    double s, cy, sy, tx, ty, tz; /* uniform scale, yaw (cos, sin), translation */
} Xform;

static void xf(const Xform *x, double px, double py, double pz, double *o) {
    double X = px * x->s, Y = py * x->s, Z = pz * x->s;
    o[0] = x->cy * X + x->sy * Z + x->tx;
    o[1] = Y + x->ty;
    o[2] = -x->sy * X + x->cy * Z + x->tz;
}

static void quad(TriSink *s, const double *a, const double *b, const double *c, const double *d) {
    sink_tri(s, a, b, c);
    sink_tri(s, a, c, d);
}

/* Unit prototypes: each spans y in [0, 1] and |x|, |z| <= 0.5. */

/* UV sphere, 32 segments x 16 rings: 960 triangles. */
static void proto_sphere(TriSink *s, const Xform *x) {
    const int SEG = 32, RING = 16;
    for (int r = 0; r < RING; ++r) {
        double th0 = M_PI * r / RING, th1 = M_PI * (r + 1) / RING;
        for (int g = 0; g < SEG; ++g) {
            double ph0 = 2 * M_PI * g / SEG, ph1 = 2 * M_PI * (g + 1) / SEG;
            double p[4][3];
            double ths[4] = {th0, th0, th1, th1}, phs[4] = {ph0, ph1, ph1, ph0};
            for (int k = 0; k < 4; ++k)
                xf(x, 0.5 * sin(ths[k]) * cos(phs[k]), 0.5 + 0.5 * cos(ths[k]), 0.5 * sin(ths[k]) * sin(phs[k]), p[k]);
            if (r == 0)
                sink_tri(s, p[0], p[2], p[3]);
            else if (r == RING - 1)
                sink_tri(s, p[0], p[1], p[2]);
            else
                quad(s, p[0], p[1], p[2], p[3]);
        }
    }
}

/* Capped cylinder, 32 segments: 128 triangles. */
static void proto_cylinder(TriSink *s, const Xform *x) {
    const int SEG = 32;
    double cb[3], ct[3];
    xf(x, 0, 0, 0, cb);
    xf(x, 0, 1, 0, ct);
    for (int g = 0; g < SEG; ++g) {
        double ph0 = 2 * M_PI * g / SEG, ph1 = 2 * M_PI * (g + 1) / SEG;
        double b0[3], b1[3], t0[3], t1[3];
        xf(x, 0.5 * cos(ph0), 0, 0.5 * sin(ph0), b0);
        xf(x, 0.5 * cos(ph1), 0, 0.5 * sin(ph1), b1);
        xf(x, 0.5 * cos(ph0), 1, 0.5 * sin(ph0), t0);
        xf(x, 0.5 * cos(ph1), 1, 0.5 * sin(ph1), t1);
        quad(s, b0, b1, t1, t0);
        sink_tri(s, cb, b1, b0);
        sink_tri(s, ct, t0, t1);
    }
}

/* Box with every face subdivided 4 x 4: 192 triangles. */
static void proto_box(TriSink *s, const Xform *x) {
    const int D = 4;
    /* face: fixed axis, sign, and the two in-plane axes */
    for (int ax = 0; ax < 3; ++ax)
        for (int sg = 0; sg < 2; ++sg) {
            int u = (ax + 1) % 3, v = (ax + 2) % 3;
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double p[4][3];
                    int du[4] = {0, 1, 1, 0}, dv[4] = {0, 0, 1, 1};
                    for (int k = 0; k < 4; ++k) {
                        double l[3];
                        l[ax] = sg ? 0.5 : -0.5;
                        l[u] = -0.5 + (double)(i + du[k]) / D;
                        l[v] = -0.5 + (double)(j + dv[k]) / D;
                        xf(x, l[0], l[1] + 0.5, l[2], p[k]);
                    }
                    quad(s, p[0], p[1], p[2], p[3]);
                }
        }
}

/* Closed axis-aligned room [0,RX] x [0,RY] x [0,RZ]: 12 triangles. */
static void room_shell(TriSink *s, double RX, double RY, double RZ) {
    double c[8][3];
    for (int k = 0; k < 8; ++k) {
        c[k][0] = (k & 1) ? RX : 0;
        c[k][1] = (k & 2) ? RY : 0;
        c[k][2] = (k & 4) ? RZ : 0;
    }
    quad(s, c[0], c[1], c[3], c[2]); /* z = 0   */
    quad(s, c[4], c[6], c[7], c[5]); /* z = RZ  */
    quad(s, c[0], c[4], c[5], c[1]); /* y = 0   */
    quad(s, c[2], c[3], c[7], c[6]); /* y = RY  */
    quad(s, c[0], c[2], c[6], c[4]); /* x = 0   */
    quad(s, c[1], c[5], c[7], c[3]); /* x = RX  */
}

/*
 * A closed 10 x 3 x 8 m room holding instanced procedural furniture
 * (spheres, capped cylinders, subdivided boxes in a 1:1:1 random mix)
 * placed in n_clusters clusters on the floor: instance positions are normal
 * around a uniform cluster centre (sigma 0.4 m), 30 % are stacked on an
 * earlier instance, scale is log-normal (median 0.25 m, sigma 0.5), yaw is
 * uniform.  Instances are added until at least target_tris triangles exist;
 * instancing is flattened into world-space triangles.
 * Returns the triangle count; writes at most cap triangles into out (out may
 * be NULL to count only).
 */
uint32_t gen_room_tris(uint64_t seed, uint32_t target_tris, uint32_t n_clusters, float *out, uint32_t cap) {
    const double RX = 10.0, RY = 3.0, RZ = 8.0;
    TriSink s = {out, 0, cap};
    room_shell(&s, RX, RY, RZ);
    if (n_clusters == 0) n_clusters = 1;
    /* per-instance records for stacking */
    uint32_t max_inst = target_tris / 128 + 16;
    double *top = (double *)malloc(sizeof(double) * max_inst);
    double *ix = (double *)malloc(sizeof(double) * max_inst);
    double *iz = (double *)malloc(sizeof(double) * max_inst);
    uint32_t ninst = 0;
    while (s.n < target_tris && ninst < max_inst) {
        uint32_t j = ninst;
        uint32_t cl = (uint32_t)(u01(seed, P_INST_CLUSTER, j) * n_clusters);
        if (cl >= n_clusters) cl = n_clusters - 1;
        double ccx = 1.0 + 8.0 * u01(seed, P_CLUSTER, 2 * cl);
        double ccz = 1.0 + 6.0 * u01(seed, P_CLUSTER, 2 * cl + 1);
        int type = (int)(u01(seed, P_INST_TYPE, j) * 3.0);
        if (type > 2) type = 2;
        double sc = exp(log(0.25) + 0.5 * normal01(seed, P_INST_SCALE, j));
        if (sc < 0.04) sc = 0.04;
        if (sc > 1.2) sc = 1.2;
        double yaw = 2.0 * M_PI * u01(seed, P_INST_YAW, j);
        double px = ccx + 0.4 * normal01(seed, P_INST_POS, 2 * (uint64_t)j);
        double pz = ccz + 0.4 * normal01(seed, P_INST_POS, 2 * (uint64_t)j + 1);
        double base = 0.0;
        if (j > 0 && u01(seed, P_INST_STACK, j) < 0.3) {
            uint32_t k = (uint32_t)(u01(seed, P_INST_STACK_ON, j) * j);
            if (k >= j) k = j - 1;
            if (top[k] + sc < RY - 0.05) {
                base = top[k];
                px = ix[k];
                pz = iz[k];
            }
        }
        double m = 0.5 * sc * 1.0000001 + 0.01;
        if (px < m) px = m;
        if (px > RX - m) px = RX - m;
        if (pz < m) pz = m;
        if (pz > RZ - m) pz = RZ - m;
        if (base + sc > RY - 0.01) sc = RY - 0.01 - base;
        Xform x = {sc, cos(yaw), sin(yaw), px, base, pz};
        if (type == 0)
            proto_sphere(&s, &x);
        else if (type == 1)
            proto_cylinder(&s, &x);
        else
            proto_box(&s, &x);
        top[j] = base + sc;
        ix[j] = px;
        iz[j] = pz;
        ninst++;
    }
    free(top);
    free(ix);
    free(iz);
    return s.n;
}

/* ------------------------------------------------- BVH2, binned SAH build */

typedef struct {
    const float *tv;
    uint32_t *order;  /* triangle ids, permuted in place into leaf order */
    float *cen;       /* centroid per triangle id (3 floats) */
    float *tlo, *thi; /* triangle AABB per id */
    float *lo, *hi;
    int32_t *left, *right;
    uint32_t *first, *count;
    uint32_t nnodes, cap;
    int bins, max_leaf;
    uint32_t depth;
    int32_t *bcnt;
    float *blo, *bhi;
} Builder;

static double box_area(const float *lo, const float *hi) {
    double ex = (double)hi[0] - lo[0], ey = (double)hi[1] - lo[1], ez = (double)hi[2] - lo[2];
    if (ex < 0 || ey < 0 || ez < 0) return 0.0;
    return 2.0 * (ex * ey + ey * ez + ez * ex);
}

static uint32_t build_rec(Builder *B, uint32_t b, uint32_t e, uint32_t depth) {
    uint32_t me = B->nnodes++;
    if (depth > B->depth) B->depth = depth;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (uint32_t i = b; i < e; ++i) {
        uint32_t t = B->order[i];
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], B->tlo[t * 3 + a]);
            hi[a] = fmaxf(hi[a], B->thi[t * 3 + a]);
            clo[a] = fminf(clo[a], B->cen[t * 3 + a]);
            chi[a] = fmaxf(chi[a], B->cen[t * 3 + a]);
        }
    }
    memcpy(B->lo + me * 3, lo, sizeof lo);
    memcpy(B->hi + me * 3, hi, sizeof hi);
    uint32_t n = e - b;
    if (n == 1) {
        B->left[me] = B->right[me] = -1;
        B->first[me] = b;
        B->count[me] = n;
        return me;
    }
    /* binned SAH over centroid bounds */
    int nb = B->bins;
    double best = INFINITY;
    int bax = -1, bsplit = -1;
    for (int a = 0; a < 3; ++a) {
        double ext = (double)chi[a] - clo[a];
        if (!(ext > 0)) continue;
        for (int k = 0; k < nb; ++k) {
            B->bcnt[k] = 0;
            for (int q = 0; q < 3; ++q) {
                B->blo[k * 3 + q] = INFINITY;
                B->bhi[k * 3 + q] = -INFINITY;
            }
        }
        for (uint32_t i = b; i < e; ++i) {
            uint32_t t = B->order[i];
            int k = (int)(((double)B->cen[t * 3 + a] - clo[a]) * nb / ext);
            if (k >= nb) k = nb - 1;
            if (k < 0) k = 0;
            B->bcnt[k]++;
            for (int q = 0; q < 3; ++q) {
                B->blo[k * 3 + q] = fminf(B->blo[k * 3 + q], B->tlo[t * 3 + q]);
                B->bhi[k * 3 + q] = fmaxf(B->bhi[k * 3 + q], B->thi[t * 3 + q]);
            }
        }
        /* sweep: cost of splitting after bin k */
        double rarea[64];
        int rcnt[64];
        float rlo[3] = {INFINITY, INFINITY, INFINITY}, rhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        int rc = 0;
        for (int k = nb - 1; k >= 1; --k) {
            for (int q = 0; q < 3; ++q) {
                rlo[q] = fminf(rlo[q], B->blo[k * 3 + q]);
                rhi[q] = fmaxf(rhi[q], B->bhi[k * 3 + q]);
            }
            rc += B->bcnt[k];
            rarea[k] = box_area(rlo, rhi);
            rcnt[k] = rc;
        }
        float llo[3] = {INFINITY, INFINITY, INFINITY}, lhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        int lc = 0;
        for (int k = 0; k < nb - 1; ++k) {
            for (int q = 0; q < 3; ++q) {
                llo[q] = fminf(llo[q], B->blo[k * 3 + q]);
                lhi[q] = fmaxf(lhi[q], B->bhi[k * 3 + q]);
            }
            lc += B->bcnt[k];
            if (lc == 0 || rcnt[k + 1] == 0) continue;
            double cost = box_area(llo, lhi) * lc + rarea[k + 1] * rcnt[k + 1];
            if (cost < best) {
                best = cost;
                bax = a;
                bsplit = k;
            }
        }
    }
    /* SAH termination: a node of at most max_leaf triangles stays a leaf
       unless splitting is cheaper (traversal step 1, triangle test 1). */
    if (n <= (uint32_t)B->max_leaf) {
        double parea = box_area(lo, hi);
        double split_cost = (bax < 0 || !(parea > 0)) ? INFINITY : 1.0 + best / parea;
        if ((double)n <= split_cost) {
            B->left[me] = B->right[me] = -1;
            B->first[me] = b;
            B->count[me] = n;
            return me;
        }
    }
    uint32_t mid;
    if (bax < 0) {
        mid = b + n / 2; /* all centroids coincide: split the range in half */
    } else {
        double ext = (double)chi[bax] - clo[bax];
        uint32_t i = b, j = e;
        while (i < j) {
            uint32_t t = B->order[i];
            int k = (int)(((double)B->cen[t * 3 + bax] - clo[bax]) * nb / ext);
            if (k >= nb) k = nb - 1;
            if (k < 0) k = 0;
            if (k <= bsplit) {
                ++i;
            } else {
                --j;
                B->order[i] = B->order[j];
                B->order[j] = t;
            }
        }
        mid = i;
        if (mid == b || mid == e) mid = b + n / 2;
    }
    B->first[me] = 0;
    B->count[me] = 0;
    int32_t l = (int32_t)build_rec(B, b, mid, depth + 1);
    int32_t r = (int32_t)build_rec(B, mid, e, depth + 1);
    B->left[me] = l;
    B->right[me] = r;
    return me;
}

/*
 * Binned-SAH BVH2 over ntris triangles (tv: 9 floats each): every node is
 * split at the cheapest of the bins-1 candidate planes per axis (surface
 * area heuristic); a node of at most max_leaf triangles becomes a leaf
 * unless the split is cheaper than testing its triangles (traversal and
 * triangle test both cost 1).  Nodes are
 * numbered in depth-first pre-order with the root at 0; a leaf has
 * left = right = -1 and owns order[first .. first+count).  Node boxes are
 * the exact FP32 union of their triangles' vertex bounds.  Arrays must hold
 * 2*ntris nodes (lo/hi 3 floats per node) and ntris order entries.
 * Returns the node count; *depth_out receives the maximum depth (root = 0).
 */
uint32_t gen_build_bvh(const float *tv, uint32_t ntris, int bins, int max_leaf, float *lo, float *hi,
                       int32_t *left, int32_t *right, uint32_t *first, uint32_t *count, uint32_t *order,
                       uint32_t *depth_out) {
    if (ntris == 0) return 0;
    if (bins < 2) bins = 2;
    if (bins > 64) bins = 64;
    if (max_leaf < 1) max_leaf = 1;
    Builder B;
    memset(&B, 0, sizeof B);
    B.tv = tv;
    B.order = order;
    B.cen = (float *)malloc(sizeof(float) * 3 * (size_t)ntris);
    B.tlo = (float *)malloc(sizeof(float) * 3 * (size_t)ntris);
    B.thi = (float *)malloc(sizeof(float) * 3 * (size_t)ntris);
    B.lo = lo;
    B.hi = hi;
    B.left = left;
    B.right = right;
    B.first = first;
    B.count = count;
    B.cap = 2 * ntris;
    B.bins = bins;
    B.max_leaf = max_leaf;
    B.bcnt = (int32_t *)malloc(sizeof(int32_t) * 64);
    B.blo = (float *)malloc(sizeof(float) * 3 * 64);
    B.bhi = (float *)malloc(sizeof(float) * 3 * 64);
    for (uint32_t t = 0; t < ntris; ++t) {
        order[t] = t;
        for (int a = 0; a < 3; ++a) {
            float x0 = tv[(size_t)t * 9 + a], x1 = tv[(size_t)t * 9 + 3 + a], x2 = tv[(size_t)t * 9 + 6 + a];
            float mn = fminf(x0, fminf(x1, x2)), mx = fmaxf(x0, fmaxf(x1, x2));
            B.tlo[t * 3 + a] = mn;
            B.thi[t * 3 + a] = mx;
            B.cen[t * 3 + a] = (float)(0.5 * ((double)mn + mx));
        }
    }
    build_rec(&B, 0, ntris, 0);
    if (depth_out) *depth_out = B.depth;
    free(B.cen);
    free(B.tlo);
    free(B.thi);
    free(B.bcnt);
    free(B.blo);
    free(B.bhi);
    return B.nnodes;
}

/* ------------------------------------- camera, rasterised visibility, rays */

typedef struct {
    double pos[3], f[3], r[3], u[3];
    double tan_half, aspect;
    int W, H, spp;
    uint64_t seed;
} Cam;

static void v3sub(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
static double v3dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v3cross(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void v3norm(double *a) {
    double l = sqrt(v3dot(a, a));
    if (l > 0) {
        a[0] /= l;
        a[1] /= l;
        a[2] /= l;
    }
}

static void cam_setup(Cam *c, const double *pos, const double *target, double vfov_deg, int W, int H, int spp,
                      uint64_t seed) {
    double up[3] = {0, 1, 0};
    memcpy(c->pos, pos, sizeof c->pos);
    v3sub(target, pos, c->f);
    v3norm(c->f);
    v3cross(c->f, up, c->r);
    v3norm(c->r);
    v3cross(c->r, c->f, c->u);
    c->tan_half = tan(0.5 * vfov_deg * M_PI / 180.0);
    c->aspect = (double)W / H;
    c->W = W;
    c->H = H;
    c->spp = spp;
    c->seed = seed;
}

/* Sample s of pixel p sits at (px + jx, py + jy) with jitter in [0, 1)^2. */
static void cam_jitter(const Cam *c, uint64_t sample_id, double *jx, double *jy) {
    *jx = u01(c->seed, P_JITTER, 2 * sample_id);
    *jy = u01(c->seed, P_JITTER, 2 * sample_id + 1);
}

/* Unnormalised world direction through screen point (X, Y). */
static void cam_dir(const Cam *c, double X, double Y, double *d) {
    double nx = (2.0 * X / c->W - 1.0) * c->tan_half * c->aspect;
    double ny = (1.0 - 2.0 * Y / c->H) * c->tan_half;
    for (int a = 0; a < 3; ++a) d[a] = c->f[a] + nx * c->r[a] + ny * c->u[a];
}

typedef struct {
    double x, y;
} P2;

/*
 * Z-buffer rasterisation of every triangle against every sample position
 * (inclusive edge functions in double precision, near-plane clipping in
 * camera space).  Depth is the distance parameter along the sample's
 * unnormalised camera direction to the triangle's plane; the nearest
 * triangle wins, ties to the lower triangle id.  zt/id: one per sample,
 * sample index = pixel * spp + s.
 */
static void rasterise(const Cam *c, const float *tv, uint32_t ntris, double *zt, int32_t *id, const float *jit) {
    const double znear = 1e-4;
    size_t ns = (size_t)c->W * c->H * c->spp;
    for (size_t i = 0; i < ns; ++i) {
        zt[i] = INFINITY;
        id[i] = -1;
    }
    double sx_scale = 0.5 * c->W / (c->tan_half * c->aspect), sy_scale = 0.5 * c->H / c->tan_half;
    for (uint32_t t = 0; t < ntris; ++t) {
        double v[3][3], cs[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) v[k][a] = tv[(size_t)t * 9 + k * 3 + a];
        double e1[3], e2[3], n[3], rel[3];
        v3sub(v[1], v[0], e1);
        v3sub(v[2], v[0], e2);
        v3cross(e1, e2, n);
        if (v3dot(n, n) == 0.0) continue;
        v3sub(v[0], c->pos, rel);
        double nd0 = v3dot(n, rel);
        for (int k = 0; k < 3; ++k) {
            double q[3];
            v3sub(v[k], c->pos, q);
            cs[k][0] = v3dot(q, c->r);
            cs[k][1] = v3dot(q, c->u);
            cs[k][2] = v3dot(q, c->f);
        }
        /* clip the polygon against z >= znear (Sutherland-Hodgman) */
        double poly[4][3];
        int np = 0;
        for (int k = 0; k < 3; ++k) {
            const double *A = cs[k], *Bv = cs[(k + 1) % 3];
            int ina = A[2] >= znear, inb = Bv[2] >= znear;
            if (ina) {
                memcpy(poly[np], A, sizeof poly[np]);
                np++;
            }
            if (ina != inb) {
                double s = (znear - A[2]) / (Bv[2] - A[2]);
                for (int a = 0; a < 3; ++a) poly[np][a] = A[a] + s * (Bv[a] - A[a]);
                poly[np][2] = znear;
                np++;
            }
        }
        if (np < 3) continue;
        P2 sp[4];
        for (int k = 0; k < np; ++k) {
            sp[k].x = (poly[k][0] / poly[k][2]) * sx_scale + 0.5 * c->W;
            sp[k].y = 0.5 * c->H - (poly[k][1] / poly[k][2]) * sy_scale;
        }
        for (int f = 1; f + 1 < np; ++f) {
            P2 a = sp[0], b = sp[f], d = sp[f + 1];
            double area = (b.x - a.x) * (d.y - a.y) - (b.y - a.y) * (d.x - a.x);
            if (area == 0.0) continue;
            double mnx = fmin(a.x, fmin(b.x, d.x)), mxx = fmax(a.x, fmax(b.x, d.x));
            double mny = fmin(a.y, fmin(b.y, d.y)), mxy = fmax(a.y, fmax(b.y, d.y));
            int x0 = (int)floor(mnx), x1 = (int)floor(mxx), y0 = (int)floor(mny), y1 = (int)floor(mxy);
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x1 > c->W - 1) x1 = c->W - 1;
            if (y1 > c->H - 1) y1 = c->H - 1;
            double sg = area > 0 ? 1.0 : -1.0;
            for (int py = y0; py <= y1; ++py)
                for (int px = x0; px <= x1; ++px) {
                    size_t pix = (size_t)py * c->W + px;
                    for (int s = 0; s < c->spp; ++s) {
                        size_t si = pix * c->spp + s;
                        double X = px + jit[2 * si], Y = py + jit[2 * si + 1];
                        double w0 = ((b.x - a.x) * (Y - a.y) - (b.y - a.y) * (X - a.x)) * sg;
                        double w1 = ((d.x - b.x) * (Y - b.y) - (d.y - b.y) * (X - b.x)) * sg;
                        double w2 = ((a.x - d.x) * (Y - d.y) - (a.y - d.y) * (X - d.x)) * sg;
                        if (w0 < 0 || w1 < 0 || w2 < 0) continue;
                        double dir[3];
                        cam_dir(c, X, Y, dir);
                        double nd = v3dot(n, dir);
                        if (nd == 0.0) continue;
                        double tt = nd0 / nd;
                        if (tt > 0 && tt < zt[si]) {
                            zt[si] = tt;
                            id[si] = (int32_t)t;
                        }
                    }
                }
        }
    }
}

/* Orthonormal basis around unit n (Duff et al. 2017, "Building an
 * Orthonormal Basis, Revisited"). */
static void onb(const double *n, double *b1, double *b2) {
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a;
    b1[1] = sign * b;
    b1[2] = -sign * n[0];
    b2[0] = b;
    b2[1] = sign + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/* Concentric square-to-disk map (Shirley & Chiu 1997). */
static void concentric(double u1, double u2, double *x, double *y) {
    double a = 2 * u1 - 1, b = 2 * u2 - 1;
    if (a == 0 && b == 0) {
        *x = *y = 0;
        return;
    }
    double r, ph;
    if (fabs(a) > fabs(b)) {
        r = a;
        ph = (M_PI / 4) * (b / a);
    } else {
        r = b;
        ph = (M_PI / 2) - (M_PI / 4) * (a / b);
    }
    *x = r * cos(ph);
    *y = r * sin(ph);
}

/*
 * Workload of one camera: rasterise the scene, then for every sample that
 * sees a triangle emit
 *   - one secondary ray: origin at the visible point, direction
 *     cosine-weighted about the surface normal turned toward the camera,
 *     interval [tmin, +inf);
 *   - n_shadow shadow rays toward a uniformly picked light quad and a
 *     uniform point on it, interval [tmin, dist * (1 - 1e-4)].
 * Light quads are axis-aligned in y (horizontal): light k is centred at
 * lights[k*3 .. k*3+2] with half size light_half.
 *
 * Samples are visited in the order given by sample_major: 0 = pixel-major
 * (index = pixel * spp + s), 1 = sample-major (index = s * W*H + pixel).
 * At most max_rays secondary rays are emitted (earliest first); shadow rays
 * of secondary i are at 2*i, 2*i+1 (n_shadow = 2) and so on.
 * Rays are written as float4 (ox, oy, oz, tmin) and (dx, dy, dz, tmax).
 * Returns the number of secondary rays written.
 */
uint64_t gen_camera_rays(const float *tv, uint32_t ntris, const double *cam_pos, const double *cam_target,
                         double vfov_deg, int W, int H, int spp, uint64_t seed, int sample_major, uint64_t max_rays,
                         float tmin, float *sec_org, float *sec_dir, int n_shadow, const double *lights,
                         int n_lights, double light_half, float *sh_org, float *sh_dir, int32_t *prim_out) {
    Cam c;
    cam_setup(&c, cam_pos, cam_target, vfov_deg, W, H, spp, seed);
    size_t ns = (size_t)W * H * spp;
    double *zt = (double *)malloc(sizeof(double) * ns);
    int32_t *id = (int32_t *)malloc(sizeof(int32_t) * ns);
    float *jit = (float *)malloc(sizeof(float) * 2 * ns);
    for (size_t i = 0; i < ns; ++i) {
        double jx, jy;
        cam_jitter(&c, i, &jx, &jy);
        jit[2 * i] = (float)jx;
        jit[2 * i + 1] = (float)jy;
    }
    rasterise(&c, tv, ntris, zt, id, jit);
    uint64_t nout = 0;
    size_t npix = (size_t)W * H;
    for (size_t k = 0; k < ns && nout < max_rays; ++k) {
        size_t si = sample_major ? ((k % npix) * spp + k / npix) : k;
        if (id[si] < 0) continue;
        size_t pix = si / spp;
        int px = (int)(pix % W), py = (int)(pix / W);
        double dir[3], p[3];
        cam_dir(&c, px + jit[2 * si], py + jit[2 * si + 1], dir);
        for (int a = 0; a < 3; ++a) p[a] = c.pos[a] + zt[si] * dir[a];
        v3norm(dir);
        const float *T = tv + (size_t)id[si] * 9;
        double e1[3], e2[3], n[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = (double)T[3 + a] - T[a];
            e2[a] = (double)T[6 + a] - T[a];
        }
        v3cross(e1, e2, n);
        v3norm(n);
        if (v3dot(n, dir) > 0) {
            n[0] = -n[0];
            n[1] = -n[1];
            n[2] = -n[2];
        }
        double b1[3], b2[3], lx, ly;
        onb(n, b1, b2);
        concentric(u01(seed, P_BOUNCE, 2 * (uint64_t)si), u01(seed, P_BOUNCE, 2 * (uint64_t)si + 1), &lx, &ly);
        double lz = sqrt(fmax(0.0, 1.0 - lx * lx - ly * ly));
        double w[3];
        for (int a = 0; a < 3; ++a) w[a] = lx * b1[a] + ly * b2[a] + lz * n[a];
        v3norm(w);
        float *o4 = sec_org + nout * 4, *d4 = sec_dir + nout * 4;
        o4[0] = (float)p[0];
        o4[1] = (float)p[1];
        o4[2] = (float)p[2];
        o4[3] = tmin;
        d4[0] = (float)w[0];
        d4[1] = (float)w[1];
        d4[2] = (float)w[2];
        d4[3] = INFINITY;
        if (prim_out) prim_out[nout] = id[si];
        for (int j = 0; j < n_shadow && n_lights > 0 && sh_org; ++j) {
            uint64_t sid = (uint64_t)si * (uint64_t)n_shadow + j;
            int L = (int)(u01(seed, P_LIGHT_PICK, sid) * n_lights);
            if (L >= n_lights) L = n_lights - 1;
            double q[3] = {lights[L * 3 + 0] + light_half * (2 * u01(seed, P_LIGHT_POINT, 2 * sid) - 1),
                           lights[L * 3 + 1],
                           lights[L * 3 + 2] + light_half * (2 * u01(seed, P_LIGHT_POINT, 2 * sid + 1) - 1)};
            double to[3];
            v3sub(q, p, to);
            double dist = sqrt(v3dot(to, to));
            float *so = sh_org + (nout * n_shadow + j) * 4, *sd = sh_dir + (nout * n_shadow + j) * 4;
            so[0] = o4[0];
            so[1] = o4[1];
            so[2] = o4[2];
            so[3] = tmin;
            sd[0] = (float)(to[0] / dist);
            sd[1] = (float)(to[1] / dist);
            sd[2] = (float)(to[2] / dist);
            sd[3] = (float)(dist * (1.0 - 1e-4));
        }
        nout++;
    }
    free(zt);
    free(id);
    free(jit);
    return nout;
}
