/*
 * FP64 CPU oracle for the neural path tracer of "Towards Neural Path Tracing
 * in SRAM" (Pupilli 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; both read the
 * same seeded host arrays and nothing else.
 *
 * Plain, slow, obviously correct: every quantity is computed in double
 * precision from the float32 inputs (promoted), with no blocking, fusion or
 * reordering beyond what the cited definitions state.
 *
 * Parity status of each part (pins live in tests/test_oracle_*.py):
 *   Philox-4x32-10 ........ pinned (published known-answer vectors)
 *   intersections ......... pinned (closed-form roots, brute force, watertightness)
 *   BVH ................... pinned (brute force)
 *   estimator ............. pinned (white-furnace closed forms, energy bounds)
 *   BSDF lobes ............ pinned (cosine moments, Fresnel at normal incidence,
 *                           Snell's law, total internal reflection, Schlick/Smith at h = n;
 *                           GGX metal: mean weight = directional albedo from an independent
 *                           quadrature of the microfacet BRDF, half-vector chi-square)
 *   NIF forward ........... pinned (B = 0, zero weights, relu(x) - relu(-x) = x wiring;
 *                           skip concatenation: a silent skip layer reduces to the
 *                           shorter plain network, features routed around it,
 *                           97.7 KiB parameter count of the paper's network)
 *   NIF backward / Adam ... pinned (central finite differences, Adam closed-form steps)
 *   sky lookup ............ pinned (pixel centres, wrap/clamp, four-centre average)
 *   radiance cache ........ pinned (zero weights, wiring closed forms, fixed-denominator
 *                           finite differences, output-bias closed form, furnace suffix
 *                           radiance and cached-render closed forms)
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Section 3.3 / Fig. 2). */
/* The paper's renderer draws from the IPU's hardware generator (Section     */
/* 3.1.3); here a counter-based generator keyed by (seed, stream) and        */
/* counted by (pixel, sample, vertex, 0) replaces it.                        */
/* ------------------------------------------------------------------------ */
OR_API void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {           /* Weyl key schedule between rounds */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in [0,1): the top 24 bits of a word times 2^-24 (exact in float) */
static double u01(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

static void philox_words(uint32_t seed, uint32_t tag, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                         uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {seed, tag};
    or_philox4x32_10(ctr, key, out);
}

OR_API void or_philox_batch(uint32_t seed, uint32_t tag, int64_t n, const uint32_t* ctr /* n x 4 */, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) philox_words(seed, tag, ctr[4*i], ctr[4*i+1], ctr[4*i+2], ctr[4*i+3], out + 4*i);
}

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
typedef struct { double x, y, z; } V3;
static V3 v3(double x, double y, double z) { V3 r = {x, y, z}; return r; }
static V3 add(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static V3 sub(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static V3 mul(V3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static V3 hadamard(V3 a, V3 b) { return v3(a.x * b.x, a.y * b.y, a.z * b.z); }
static double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static V3 cross(V3 a, V3 b) { return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static V3 normalize(V3 a) { double l = sqrt(dot(a, a)); return mul(a, 1.0 / l); }
static double comp(V3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }
static double maxd(double a, double b) { return a > b ? a : b; }
static double mind(double a, double b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Scene: spheres, axis-aligned quads, triangles (global ID order: spheres,  */
/* quads, triangles) and materials.  Section 4.1 test scenes are stood in    */
/* for by procedural ones with the same primitive kinds.                     */
/* ------------------------------------------------------------------------ */
enum { MAT_LAMBERT = 0, MAT_METAL = 1, MAT_DIELECTRIC = 2 };

typedef struct { double lo[3], hi[3]; int32_t left, right, start, count; } OrNode;

typedef struct {
    int64_t nS, nQ, nT, nM, nPrim;
    double *sph;        /* nS x 4 */
    int32_t *sph_mat;
    double *quad;       /* nQ x 5 */
    int32_t *quad_axis, *quad_mat;
    double *tv;         /* nT x 9 : v0, v1, v2 */
    int32_t *tri_mat;
    int32_t *mat_type;
    double *mat;        /* nM x 8 */
    /* oracle-own BVH (median split, <= 4 prims per leaf) */
    int use_bvh;
    OrNode *nodes;
    int64_t n_nodes;
    int64_t *prim_idx;
    /* scene bounds (for the radiance-cache position encoding) */
    double lo[3], hi[3];
} OrScene;

static void prim_bounds(const OrScene* s, int64_t id, double lo[3], double hi[3])
{
    if (id < s->nS) {
        const double* c = s->sph + 4 * id;
        for (int a = 0; a < 3; ++a) { lo[a] = c[a] - c[3]; hi[a] = c[a] + c[3]; }
    } else if (id < s->nS + s->nQ) {
        int64_t q = id - s->nS;
        int a = s->quad_axis[q], u = (a + 1) % 3, v = (a + 2) % 3;
        const double* p = s->quad + 5 * q;
        lo[a] = hi[a] = p[0];
        lo[u] = p[1]; hi[u] = p[2];
        lo[v] = p[3]; hi[v] = p[4];
    } else {
        const double* t = s->tv + 9 * (id - s->nS - s->nQ);
        for (int a = 0; a < 3; ++a) {
            lo[a] = mind(t[a], mind(t[3 + a], t[6 + a]));
            hi[a] = maxd(t[a], maxd(t[3 + a], t[6 + a]));
        }
    }
}

/* --- oracle BVH: plain median split on the widest centroid axis --------- */
typedef struct { const OrScene* s; double* cen; OrNode* nodes; int64_t n_nodes; } BuildCtx;

static double centroid_key(BuildCtx* b, int64_t prim, int axis) { return b->cen[3 * prim + axis]; }

static void quickselect(BuildCtx* b, int64_t* idx, int64_t lo, int64_t hi, int64_t k, int axis)
{
    /* order idx[lo..hi) so that idx[k] has the k-th smallest key (ties by prim id) */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        double pk = centroid_key(b, idx[mid], axis);
        int64_t pid = idx[mid];
        int64_t i = lo, j = hi - 1;
        while (i <= j) {
            while (1) { double kk = centroid_key(b, idx[i], axis); if (kk < pk || (kk == pk && idx[i] < pid)) ++i; else break; }
            while (1) { double kk = centroid_key(b, idx[j], axis); if (kk > pk || (kk == pk && idx[j] > pid)) --j; else break; }
            if (i <= j) { int64_t t = idx[i]; idx[i] = idx[j]; idx[j] = t; ++i; --j; }
        }
        if (k <= j) hi = j + 1;
        else if (k >= i) lo = i;
        else return;
    }
}

static int64_t build_rec(BuildCtx* b, int64_t* idx, int64_t start, int64_t count)
{
    const OrScene* s = b->s;
    int64_t me = b->n_nodes++;
    OrNode* n = &b->nodes[me];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = start; i < start + count; ++i) {
        double plo[3], phi[3];
        prim_bounds(s, idx[i], plo, phi);
        for (int a = 0; a < 3; ++a) {
            lo[a] = mind(lo[a], plo[a]); hi[a] = maxd(hi[a], phi[a]);
            double c = b->cen[3 * idx[i] + a];
            clo[a] = mind(clo[a], c); chi[a] = maxd(chi[a], c);
        }
    }
    double pad = 1e-9 * (1.0 + maxd(fabs(lo[0]), maxd(fabs(lo[1]), maxd(fabs(lo[2]),
                          maxd(fabs(hi[0]), maxd(fabs(hi[1]), fabs(hi[2])))))));
    for (int a = 0; a < 3; ++a) { n->lo[a] = lo[a] - pad; n->hi[a] = hi[a] + pad; }
    if (count <= 4) {
        n->left = n->right = -1; n->start = (int32_t)start; n->count = (int32_t)count;
        return me;
    }
    int axis = 0;
    double ext = chi[0] - clo[0];
    for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > ext) { ext = chi[a] - clo[a]; axis = a; }
    int64_t half = count / 2;
    quickselect(b, idx, start, start + count, start + half, axis);
    int64_t l = build_rec(b, idx, start, half);
    int64_t r = build_rec(b, idx, start + half, count - half);
    n = &b->nodes[me];
    n->left = (int32_t)l; n->right = (int32_t)r; n->start = -1; n->count = 0;
    return me;
}

static void build_bvh(OrScene* s)
{
    int64_t N = s->nPrim;
    BuildCtx b;
    b.s = s;
    b.cen = (double*)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        double lo[3], hi[3];
        prim_bounds(s, i, lo, hi);
        for (int a = 0; a < 3; ++a) b.cen[3 * i + a] = 0.5 * (lo[a] + hi[a]);
    }
    s->prim_idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) s->prim_idx[i] = i;
    b.nodes = (OrNode*)malloc(sizeof(OrNode) * (size_t)(2 * N + 1));
    b.n_nodes = 0;
    if (N > 0) build_rec(&b, s->prim_idx, 0, N);
    s->nodes = b.nodes;
    s->n_nodes = b.n_nodes;
    free(b.cen);
}

OR_API OrScene* or_scene_create(int64_t nS, const float* sphere, const int32_t* sphere_mat,
                                int64_t nQ, const float* quad, const int32_t* quad_axis, const int32_t* quad_mat,
                                int64_t nV, const float* vert, int64_t nT, const int32_t* tri, const int32_t* tri_mat,
                                int64_t nM, const int32_t* mat_type, const float* mat, int use_bvh)
{
    (void)nV;
    OrScene* s = (OrScene*)calloc(1, sizeof(OrScene));
    s->nS = nS; s->nQ = nQ; s->nT = nT; s->nM = nM; s->nPrim = nS + nQ + nT;
    s->sph = (double*)malloc(sizeof(double) * (size_t)(4 * nS + 1));
    s->sph_mat = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nS + 1));
    for (int64_t i = 0; i < 4 * nS; ++i) s->sph[i] = sphere[i];
    for (int64_t i = 0; i < nS; ++i) s->sph_mat[i] = sphere_mat[i];
    s->quad = (double*)malloc(sizeof(double) * (size_t)(5 * nQ + 1));
    s->quad_axis = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nQ + 1));
    s->quad_mat = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nQ + 1));
    for (int64_t i = 0; i < 5 * nQ; ++i) s->quad[i] = quad[i];
    for (int64_t i = 0; i < nQ; ++i) { s->quad_axis[i] = quad_axis[i]; s->quad_mat[i] = quad_mat[i]; }
    s->tv = (double*)malloc(sizeof(double) * (size_t)(9 * nT + 1));
    s->tri_mat = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nT + 1));
    for (int64_t i = 0; i < nT; ++i) {
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) s->tv[9 * i + 3 * k + a] = vert[3 * (int64_t)tri[3 * i + k] + a];
        s->tri_mat[i] = tri_mat[i];
    }
    s->mat_type = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nM + 1));
    s->mat = (double*)malloc(sizeof(double) * (size_t)(8 * nM + 1));
    for (int64_t i = 0; i < nM; ++i) s->mat_type[i] = mat_type[i];
    for (int64_t i = 0; i < 8 * nM; ++i) s->mat[i] = mat[i];
    for (int a = 0; a < 3; ++a) { s->lo[a] = INFINITY; s->hi[a] = -INFINITY; }
    for (int64_t i = 0; i < s->nPrim; ++i) {
        double lo[3], hi[3];
        prim_bounds(s, i, lo, hi);
        for (int a = 0; a < 3; ++a) { s->lo[a] = mind(s->lo[a], lo[a]); s->hi[a] = maxd(s->hi[a], hi[a]); }
    }
    s->use_bvh = use_bvh;
    if (use_bvh) build_bvh(s);
    return s;
}

OR_API void or_scene_destroy(OrScene* s)
{
    if (!s) return;
    free(s->sph); free(s->sph_mat); free(s->quad); free(s->quad_axis); free(s->quad_mat);
    free(s->tv); free(s->tri_mat); free(s->mat_type); free(s->mat);
    free(s->nodes); free(s->prim_idx);
    free(s);
}

OR_API int64_t or_scene_bvh_nodes(const OrScene* s) { return s->n_nodes; }

OR_API void or_scene_bounds(const OrScene* s, double* lo, double* hi)
{
    for (int a = 0; a < 3; ++a) { lo[a] = s->lo[a]; hi[a] = s->hi[a]; }
}

/* ------------------------------------------------------------------------ */
/* Ray-primitive intersection (Section 3.1.3: slab test, PBRT-style          */
/* watertight triangle test; analytic spheres for the spheres scene).        */
/* Each returns the smallest t > 0 or INFINITY.                              */
/* ------------------------------------------------------------------------ */
static double hit_sphere(const double* c, V3 o, V3 d)
{
    /* roots of |o + t d - c|^2 = r^2 with |d| = 1; discriminant from the
       closest-approach vector, product form for the second root */
    V3 oc = sub(o, v3(c[0], c[1], c[2]));
    double r = c[3];
    double b = dot(oc, d);
    V3 l = sub(oc, mul(d, b));
    double disc = r * r - dot(l, l);
    if (disc < 0.0) return INFINITY;
    double sq = sqrt(disc);
    double q = -b - copysign(sq, b);
    double cc = dot(oc, oc) - r * r;
    double t0 = q, t1 = (q != 0.0) ? cc / q : q;
    double tn = mind(t0, t1), tf = maxd(t0, t1);
    if (tn > 0.0) return tn;
    if (tf > 0.0) return tf;
    return INFINITY;
}

static double hit_quad(const double* p, int a, V3 o, V3 d)
{
    int u = (a + 1) % 3, v = (a + 2) % 3;
    double da = comp(d, a);
    if (da == 0.0) return INFINITY;
    double t = (p[0] - comp(o, a)) / da;
    if (!(t > 0.0)) return INFINITY;
    double pu = comp(o, u) + t * comp(d, u);
    double pv = comp(o, v) + t * comp(d, v);
    if (pu < p[1] || pu > p[2] || pv < p[3] || pv > p[4]) return INFINITY;
    return t;
}

/* Woop, Benthin, Wald, "Watertight Ray/Triangle Intersection", JCGT 2013. */
static double hit_triangle(const double* tv, V3 o, V3 d)
{
    double dd[3] = {d.x, d.y, d.z};
    int kz = 0;
    if (fabs(dd[1]) > fabs(dd[kz])) kz = 1;
    if (fabs(dd[2]) > fabs(dd[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (dd[kz] < 0.0) { int t = kx; kx = ky; ky = t; }
    double Sx = dd[kx] / dd[kz], Sy = dd[ky] / dd[kz], Sz = 1.0 / dd[kz];
    double oo[3] = {o.x, o.y, o.z};
    double A[3], B[3], C[3];
    for (int a = 0; a < 3; ++a) { A[a] = tv[a] - oo[a]; B[a] = tv[3 + a] - oo[a]; C[a] = tv[6 + a] - oo[a]; }
    double Ax = A[kx] - Sx * A[kz], Ay = A[ky] - Sy * A[kz];
    double Bx = B[kx] - Sx * B[kz], By = B[ky] - Sy * B[kz];
    double Cx = C[kx] - Sx * C[kz], Cy = C[ky] - Sy * C[kz];
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0)) return INFINITY;
    double det = U + V + W;
    if (det == 0.0) return INFINITY;
    double T = U * (Sz * A[kz]) + V * (Sz * B[kz]) + W * (Sz * C[kz]);
    double t = T / det;
    if (!(t > 0.0)) return INFINITY;
    return t;
}

static double hit_prim(const OrScene* s, int64_t id, V3 o, V3 d)
{
    if (id < s->nS) return hit_sphere(s->sph + 4 * id, o, d);
    if (id < s->nS + s->nQ) { int64_t q = id - s->nS; return hit_quad(s->quad + 5 * q, s->quad_axis[q], o, d); }
    return hit_triangle(s->tv + 9 * (id - s->nS - s->nQ), o, d);
}

/* closest hit, ties broken towards the smaller primitive ID */
static void consider(const OrScene* s, int64_t id, V3 o, V3 d, double* tb, int64_t* ib)
{
    double t = hit_prim(s, id, o, d);
    if (t < *tb || (t == *tb && t < INFINITY && id < *ib)) { *tb = t; *ib = id; }
}

static int box_hit(const OrNode* n, V3 o, V3 d, double tbest)
{
    double tmin = 0.0, tmax = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double oa = comp(o, a), da = comp(d, a);
        if (da == 0.0) {
            if (oa < n->lo[a] || oa > n->hi[a]) return 0;
            continue;
        }
        double t0 = (n->lo[a] - oa) / da, t1 = (n->hi[a] - oa) / da;
        if (t0 > t1) { double t = t0; t0 = t1; t1 = t; }
        tmin = maxd(tmin, t0);
        tmax = mind(tmax, t1);
    }
    return tmin <= tmax && tmin <= tbest;
}

static void closest_hit(const OrScene* s, V3 o, V3 d, int brute, double* t_out, int64_t* id_out)
{
    double tb = INFINITY;
    int64_t ib = -1;
    if (brute || !s->use_bvh) {
        for (int64_t i = 0; i < s->nPrim; ++i) consider(s, i, o, d, &tb, &ib);
    } else if (s->n_nodes > 0) {
        int64_t stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const OrNode* n = &s->nodes[stack[--sp]];
            if (!box_hit(n, o, d, tb)) continue;
            if (n->left < 0) {
                for (int i = 0; i < n->count; ++i) consider(s, s->prim_idx[n->start + i], o, d, &tb, &ib);
            } else {
                stack[sp++] = n->right;
                stack[sp++] = n->left;
            }
        }
    }
    *t_out = tb;
    *id_out = (tb < INFINITY) ? ib : -1;
}

OR_API void or_closest_hit(const OrScene* s, int64_t n, const double* org, const double* dir, int brute,
                           double* t_out, int64_t* id_out)
{
    for (int64_t i = 0; i < n; ++i) {
        V3 o = v3(org[3 * i], org[3 * i + 1], org[3 * i + 2]);
        V3 d = v3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
        closest_hit(s, o, d, brute, &t_out[i], &id_out[i]);
    }
}

static int prim_material(const OrScene* s, int64_t id)
{
    if (id < s->nS) return s->sph_mat[id];
    if (id < s->nS + s->nQ) return s->quad_mat[id - s->nS];
    return s->tri_mat[id - s->nS - s->nQ];
}

static V3 geometric_normal(const OrScene* s, int64_t id, V3 p)
{
    if (id < s->nS) {
        const double* c = s->sph + 4 * id;
        return normalize(sub(p, v3(c[0], c[1], c[2])));
    }
    if (id < s->nS + s->nQ) {
        int a = s->quad_axis[id - s->nS];
        return v3(a == 0, a == 1, a == 2);
    }
    const double* t = s->tv + 9 * (id - s->nS - s->nQ);
    V3 e1 = v3(t[3] - t[0], t[4] - t[1], t[5] - t[2]);
    V3 e2 = v3(t[6] - t[0], t[7] - t[1], t[8] - t[2]);
    return normalize(cross(e1, e2));
}

/* ------------------------------------------------------------------------ */
/* HDR neural image field (Section 3.2): (u, v) -> Gaussian Fourier         */
/* features [sin 2 pi Bx, cos 2 pi Bx] -> dense ReLU layers -> linear layer  */
/* -> fixed colour matrix -> exp (inverse of the log compression).          */
/* Flat float32 parameter layout: B (F x 2), then per layer W (out x in) and */
/* b (out), then M (3 x 3).                                                  */
/* Skip concatenation (Section 3.2, the paper's network): with skip = s >= 1 */
/* the s-th hidden layer (1-based) has H - 2F outputs, and the input of      */
/* hidden layer s + 1 is those outputs followed by the 2F Fourier features.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int F, H, L;        /* frequencies, hidden width, hidden layers */
    int skip;           /* 0: plain MLP; s: hidden layer s feeds [h_s, features] to layer s + 1 */
    int nl;             /* linear layers = L + 1 */
    int in[9], out[9];
    double *B, *W[9], *b[9], M[9];
} OrNif;

OR_API OrNif* or_nif_create_skip(int F, int H, int L, int skip, const float* flat)
{
    if (L < 1 || L > 8 || skip < 0 || skip >= L || (skip > 0 && H <= 2 * F)) return NULL;
    OrNif* n = (OrNif*)calloc(1, sizeof(OrNif));
    n->F = F; n->H = H; n->L = L; n->skip = skip; n->nl = L + 1;
    const float* p = flat;
    n->B = (double*)malloc(sizeof(double) * 2 * F);
    for (int i = 0; i < 2 * F; ++i) n->B[i] = *p++;
    for (int l = 0; l < n->nl; ++l) {
        n->in[l] = (l == 0) ? 2 * F : H;
        n->out[l] = (l == n->nl - 1) ? 3 : (skip > 0 && l == skip - 1 ? H - 2 * F : H);
        n->W[l] = (double*)malloc(sizeof(double) * n->in[l] * n->out[l]);
        n->b[l] = (double*)malloc(sizeof(double) * n->out[l]);
        for (int i = 0; i < n->in[l] * n->out[l]; ++i) n->W[l][i] = *p++;
        for (int i = 0; i < n->out[l]; ++i) n->b[l][i] = *p++;
    }
    for (int i = 0; i < 9; ++i) n->M[i] = *p++;
    return n;
}

OR_API OrNif* or_nif_create(int F, int H, int L, const float* flat) { return or_nif_create_skip(F, H, L, 0, flat); }

OR_API void or_nif_destroy(OrNif* n)
{
    if (!n) return;
    free(n->B);
    for (int l = 0; l < n->nl; ++l) { free(n->W[l]); free(n->b[l]); }
    free(n);
}

/* number of trainable parameters (all W and b; B and M are fixed) */
OR_API int64_t or_nif_n_trainable(const OrNif* n)
{
    int64_t c = 0;
    for (int l = 0; l < n->nl; ++l) c += (int64_t)n->in[l] * n->out[l] + n->out[l];
    return c;
}

/* write trainable params (double) back to a float32 flat layout copy */
OR_API void or_nif_export(const OrNif* n, double* flat_out)
{
    double* p = flat_out;
    for (int i = 0; i < 2 * n->F; ++i) *p++ = n->B[i];
    for (int l = 0; l < n->nl; ++l) {
        for (int i = 0; i < n->in[l] * n->out[l]; ++i) *p++ = n->W[l][i];
        for (int i = 0; i < n->out[l]; ++i) *p++ = n->b[l][i];
    }
    for (int i = 0; i < 9; ++i) *p++ = n->M[i];
}

/* Forward for one input.  xin receives every linear layer's input vector
   (layer l at xin + l * XW, XW = max(2F, H)): the features for layer 0, the
   previous hidden output otherwise, and for the layer after the skip layer
   that output followed by the features.  pre (optional) receives each hidden
   layer's pre-activation (layer l at pre + l * H); y = final linear output
   (3), z = M y (3). */
static int nif_xw(const OrNif* n) { return 2 * n->F > n->H ? 2 * n->F : n->H; }

static void nif_forward_one(const OrNif* n, double u, double v, double* xin, double* pre, double y[3], double z[3])
{
    const int F = n->F, H = n->H, XW = nif_xw(n);
    double* feat = xin;
    for (int i = 0; i < F; ++i) {
        double ph = n->B[2 * i] * u + n->B[2 * i + 1] * v;
        feat[i] = sin(2.0 * OR_PI * ph);
        feat[F + i] = cos(2.0 * OR_PI * ph);
    }
    for (int l = 0; l < n->L; ++l) {
        const double* x = xin + (size_t)l * XW;
        double* h = xin + (size_t)(l + 1) * XW;   /* the next layer's input */
        for (int j = 0; j < n->out[l]; ++j) {
            double acc = n->b[l][j];
            for (int k = 0; k < n->in[l]; ++k) acc += n->W[l][(size_t)j * n->in[l] + k] * x[k];
            if (pre) pre[(size_t)l * H + j] = acc;
            h[j] = acc > 0.0 ? acc : 0.0;
        }
        if (n->skip > 0 && l == n->skip - 1)
            for (int k = 0; k < 2 * F; ++k) h[n->out[l] + k] = feat[k];
    }
    int lo = n->nl - 1;
    const double* x = xin + (size_t)n->L * XW;
    for (int j = 0; j < 3; ++j) {
        double acc = n->b[lo][j];
        for (int k = 0; k < H; ++k) acc += n->W[lo][(size_t)j * H + k] * x[k];
        y[j] = acc;
    }
    for (int i = 0; i < 3; ++i) z[i] = n->M[3 * i] * y[0] + n->M[3 * i + 1] * y[1] + n->M[3 * i + 2] * y[2];
}

OR_API void or_nif_forward(const OrNif* n, int64_t cnt, const double* uv, double* rgb, double* z_out)
{
    double* xin = (double*)malloc(sizeof(double) * (size_t)(n->L + 1) * nif_xw(n));
    for (int64_t i = 0; i < cnt; ++i) {
        double y[3], z[3];
        nif_forward_one(n, uv[2 * i], uv[2 * i + 1], xin, NULL, y, z);
        for (int c = 0; c < 3; ++c) {
            rgb[3 * i + c] = exp(z[c]);
            if (z_out) z_out[3 * i + c] = z[c];
        }
    }
    free(xin);
}

/* Huber loss (Section 3.2.1): 0.5 r^2 for |r| <= delta, else
   delta (|r| - 0.5 delta); averaged over samples and channels. */
static double huber(double r, double delta)
{
    double a = fabs(r);
    return a <= delta ? 0.5 * r * r : delta * (a - 0.5 * delta);
}
static double huber_grad(double r, double delta)
{
    double a = fabs(r);
    return a <= delta ? r : delta * (r > 0 ? 1.0 : -1.0);
}

/* Loss and gradient of the mean Huber loss between z = M y and the
   log-compressed targets, by the chain rule layer by layer.  Gradient
   layout matches the trainable part of the flat layout: per layer W then b. */
OR_API double or_nif_loss_grad(const OrNif* n, int64_t cnt, const double* uv, const double* target,
                               double delta, double* grad)
{
    int H = n->H, L = n->L, XW = nif_xw(n);
    int64_t nt = or_nif_n_trainable(n);
    memset(grad, 0, sizeof(double) * (size_t)nt);
    double* gW[9]; double* gb[9];
    double* p = grad;
    for (int l = 0; l < n->nl; ++l) { gW[l] = p; p += n->in[l] * n->out[l]; gb[l] = p; p += n->out[l]; }
    double* xin = (double*)malloc(sizeof(double) * (size_t)(L + 1) * XW);
    double* pre = (double*)malloc(sizeof(double) * L * H);
    double* dh = (double*)malloc(sizeof(double) * XW);
    double* dprev = (double*)malloc(sizeof(double) * XW);
    double loss = 0.0;
    double scale = 1.0 / (3.0 * (double)cnt);
    for (int64_t s = 0; s < cnt; ++s) {
        double y[3], z[3], dz[3], dy[3];
        nif_forward_one(n, uv[2 * s], uv[2 * s + 1], xin, pre, y, z);
        for (int c = 0; c < 3; ++c) {
            double r = z[c] - target[3 * s + c];
            loss += huber(r, delta) * scale;
            dz[c] = huber_grad(r, delta) * scale;
        }
        for (int j = 0; j < 3; ++j) dy[j] = n->M[j] * dz[0] + n->M[3 + j] * dz[1] + n->M[6 + j] * dz[2];
        /* output layer */
        int lo = n->nl - 1;
        const double* x_out = xin + (size_t)L * XW;
        for (int j = 0; j < 3; ++j) {
            gb[lo][j] += dy[j];
            for (int k = 0; k < H; ++k) gW[lo][(size_t)j * H + k] += dy[j] * x_out[k];
        }
        for (int k = 0; k < H; ++k) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += n->W[lo][(size_t)j * H + k] * dy[j];
            dh[k] = acc;
        }
        /* hidden layers, last to first; dh holds the gradient at layer l's output (its first out[l]
           entries: at the skip layer the entries of the concatenated features are dropped, B is fixed) */
        for (int l = L - 1; l >= 0; --l) {
            const double* pl = pre + (size_t)l * H;
            const int nout = n->out[l], nin = n->in[l];
            for (int j = 0; j < nout; ++j) dh[j] = pl[j] > 0.0 ? dh[j] : 0.0;
            const double* x = xin + (size_t)l * XW;
            for (int j = 0; j < nout; ++j) {
                gb[l][j] += dh[j];
                for (int k = 0; k < nin; ++k) gW[l][(size_t)j * nin + k] += dh[j] * x[k];
            }
            if (l > 0) {
                for (int k = 0; k < nin; ++k) {
                    double acc = 0.0;
                    for (int j = 0; j < nout; ++j) acc += n->W[l][(size_t)j * nin + k] * dh[j];
                    dprev[k] = acc;
                }
                memcpy(dh, dprev, sizeof(double) * nin);
            }
        }
    }
    free(xin); free(pre); free(dh); free(dprev);
    return loss;
}

/* Adam (Kingma & Ba 2015, Algorithm 1) with bias-corrected moments; the
   paper trains with Adam, lr 1e-3 (Section 3.2.1). */
OR_API void or_adam_step(int64_t n, double* w, const double* g, double* m, double* v, int64_t t,
                         double lr, double beta1, double beta2, double eps)
{
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        w[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* read / write the trainable parameters of a NIF as one double vector */
OR_API void or_nif_get_trainable(const OrNif* n, double* out)
{
    double* p = out;
    for (int l = 0; l < n->nl; ++l) {
        memcpy(p, n->W[l], sizeof(double) * n->in[l] * n->out[l]); p += n->in[l] * n->out[l];
        memcpy(p, n->b[l], sizeof(double) * n->out[l]); p += n->out[l];
    }
}
OR_API void or_nif_set_trainable(OrNif* n, const double* in)
{
    const double* p = in;
    for (int l = 0; l < n->nl; ++l) {
        memcpy(n->W[l], p, sizeof(double) * n->in[l] * n->out[l]); p += n->in[l] * n->out[l];
        memcpy(n->b[l], p, sizeof(double) * n->out[l]); p += n->out[l];
    }
}

/* Bilinear sub-pixel sample of an equirectangular image (Section 3.2.1:
   training samples are uniform in (u, v) with a bilinear filter).  Pixel
   centres sit at ((i + 0.5)/w, (j + 0.5)/h); u wraps, v clamps. */
OR_API void or_sky_bilinear(const float* img, int w, int h, int64_t n, const double* uv, double* rgb)
{
    for (int64_t s = 0; s < n; ++s) {
        double x = uv[2 * s] * w - 0.5, y = uv[2 * s + 1] * h - 0.5;
        double x0 = floor(x), y0 = floor(y);
        double fx = x - x0, fy = y - y0;
        int64_t ix0 = (int64_t)x0, iy0 = (int64_t)y0;
        int64_t xa = ((ix0 % w) + w) % w, xb = (((ix0 + 1) % w) + w) % w;
        int64_t ya = iy0 < 0 ? 0 : (iy0 > h - 1 ? h - 1 : iy0);
        int64_t yb = iy0 + 1 < 0 ? 0 : (iy0 + 1 > h - 1 ? h - 1 : iy0 + 1);
        for (int c = 0; c < 3; ++c) {
            double p00 = img[(ya * w + xa) * 3 + c], p10 = img[(ya * w + xb) * 3 + c];
            double p01 = img[(yb * w + xa) * 3 + c], p11 = img[(yb * w + xb) * 3 + c];
            rgb[3 * s + c] = (1 - fy) * ((1 - fx) * p00 + fx * p10) + fy * ((1 - fx) * p01 + fx * p11);
        }
    }
}

/* uniform training coordinates for step `step`, sample i:
   Philox key (seed, 1), counter (i, step, 0, 0) -> (U(w0), U(w1)) */
OR_API void or_train_uv(uint32_t seed, uint32_t step, int64_t n, double* uv)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t w[4];
        philox_words(seed, 1u, (uint32_t)i, step, 0u, 0u, w);
        uv[2 * i] = u01(w[0]);
        uv[2 * i + 1] = u01(w[1]);
    }
}

/* One training run of the NIF on an HDR image (Section 3.2.1): each step
   draws `batch` uniform (u, v), targets log(max(rgb, 1e-6)) from the
   bilinear sample, takes the Huber-loss gradient and one Adam step. */
OR_API void or_nif_train(OrNif* n, const float* img, int w, int h, uint32_t seed, int64_t steps, int64_t batch,
                         double lr, double beta1, double beta2, double eps, double delta, double* losses)
{
    int64_t nt = or_nif_n_trainable(n);
    double* wts = (double*)malloc(sizeof(double) * nt);
    double* g = (double*)malloc(sizeof(double) * nt);
    double* m = (double*)calloc((size_t)nt, sizeof(double));
    double* v = (double*)calloc((size_t)nt, sizeof(double));
    double* uv = (double*)malloc(sizeof(double) * 2 * batch);
    double* tg = (double*)malloc(sizeof(double) * 3 * batch);
    for (int64_t st = 0; st < steps; ++st) {
        or_train_uv(seed, (uint32_t)st, batch, uv);
        or_sky_bilinear(img, w, h, batch, uv, tg);
        for (int64_t i = 0; i < 3 * batch; ++i) tg[i] = log(maxd(tg[i], 1e-6));
        double loss = or_nif_loss_grad(n, batch, uv, tg, delta, g);
        if (losses) losses[st] = loss;
        or_nif_get_trainable(n, wts);
        or_adam_step(nt, wts, g, m, v, st + 1, lr, beta1, beta2, eps);
        or_nif_set_trainable(n, wts);
    }
    free(wts); free(g); free(m); free(v); free(uv); free(tg);
}

/* ------------------------------------------------------------------------ */
/* Path tracer (Section 3.1): no light sampling; radiance is gathered when a */
/* path hits an emitter or escapes to the environment, whose value comes     */
/* from the NIF at the equirect (u, v) of the escape direction (Section      */
/* 3.3).  Russian roulette is optional.                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double eye[3], fwd[3], right[3], up[3];
    double tan_half, aspect;
} OrCam;

static void make_camera(const float* cam /* eye3 target3 up3 fov */, int W, int H, OrCam* c)
{
    V3 eye = v3(cam[0], cam[1], cam[2]), tgt = v3(cam[3], cam[4], cam[5]), up = v3(cam[6], cam[7], cam[8]);
    V3 f = normalize(sub(tgt, eye));
    V3 r = normalize(cross(f, up));
    V3 u = cross(r, f);
    c->eye[0] = eye.x; c->eye[1] = eye.y; c->eye[2] = eye.z;
    c->fwd[0] = f.x; c->fwd[1] = f.y; c->fwd[2] = f.z;
    c->right[0] = r.x; c->right[1] = r.y; c->right[2] = r.z;
    c->up[0] = u.x; c->up[1] = u.y; c->up[2] = u.z;
    c->tan_half = tan(0.5 * (double)cam[9] * OR_PI / 180.0);
    c->aspect = (double)W / (double)H;
}

static V3 camera_dir(const OrCam* c, int W, int H, int px, int py, double jx, double jy)
{
    double fx = ((px + jx) / W * 2.0 - 1.0) * c->tan_half * c->aspect;
    double fy = (1.0 - (py + jy) / H * 2.0) * c->tan_half;
    V3 d = v3(fx * c->right[0] + fy * c->up[0] + c->fwd[0],
              fx * c->right[1] + fy * c->up[1] + c->fwd[1],
              fx * c->right[2] + fy * c->up[2] + c->fwd[2]);
    return normalize(d);
}

/* primary rays of given slots (for ray-generation parity) */
OR_API void or_primary_rays(const float* cam, int W, int H, uint32_t seed, int64_t n, const int64_t* slots,
                            double* org, double* dir)
{
    OrCam c;
    make_camera(cam, W, H, &c);
    int64_t WH = (int64_t)W * H;
    for (int64_t i = 0; i < n; ++i) {
        int64_t pix = slots[i] % WH, smp = slots[i] / WH;
        uint32_t w[4];
        philox_words(seed, 0u, (uint32_t)pix, (uint32_t)smp, 0u, 0u, w);
        V3 d = camera_dir(&c, W, H, (int)(pix % W), (int)(pix / W), u01(w[0]), u01(w[1]));
        for (int a = 0; a < 3; ++a) org[3 * i + a] = c.eye[a];
        dir[3 * i] = d.x; dir[3 * i + 1] = d.y; dir[3 * i + 2] = d.z;
    }
}

/* Direction -> equirect coordinates: u = 1/2 + atan2(dx, -dz)/(2 pi),
   v = acos(dy)/pi, so v = 0 is the zenith (Section 3.3 states the lookup
   but not the convention). */
static void dir_to_uv(V3 d, double* u, double* v)
{
    *u = 0.5 + atan2(d.x, -d.z) / (2.0 * OR_PI);
    double y = d.y < -1.0 ? -1.0 : (d.y > 1.0 ? 1.0 : d.y);
    *v = acos(y) / OR_PI;
}

OR_API void or_dir_to_uv(int64_t n, const double* dir, double* uv)
{
    for (int64_t i = 0; i < n; ++i) dir_to_uv(v3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]), &uv[2 * i], &uv[2 * i + 1]);
}

/* Orthonormal basis around unit n (Duff et al., JCGT 2017, Listing 3). */
static void onb(V3 n, V3* t, V3* b)
{
    double sign = copysign(1.0, n.z);
    double a = -1.0 / (sign + n.z);
    double bb = n.x * n.y * a;
    *t = v3(1.0 + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    *b = v3(bb, sign + n.y * n.y * a, -n.y);
}

static V3 to_world(V3 l, V3 t, V3 b, V3 n) { return add(add(mul(t, l.x), mul(b, l.y)), mul(n, l.z)); }

/* Sample one bounce.  Returns 0 if the path is absorbed. */
static int sample_bsdf(const OrScene* s, int mat, V3 d, V3 ng, double u1, double u2, double ul, V3* wi, V3* weight)
{
    const double* m = s->mat + 8 * mat;
    int type = s->mat_type[mat];
    V3 alb = v3(m[0], m[1], m[2]);
    if (type == MAT_DIELECTRIC) {
        /* exact unpolarised Fresnel; reflect with probability F, refract otherwise; weight 1 */
        int entering = dot(d, ng) < 0.0;
        V3 n = entering ? ng : mul(ng, -1.0);
        double ei = entering ? 1.0 : m[4], et = entering ? m[4] : 1.0;
        double cosi = -dot(d, n);
        double eta = ei / et;
        double sin2t = eta * eta * (1.0 - cosi * cosi);
        V3 refl = add(d, mul(n, 2.0 * cosi));
        if (sin2t >= 1.0) {
            *wi = normalize(refl);
        } else {
            double cost = sqrt(1.0 - sin2t);
            double rs = (ei * cosi - et * cost) / (ei * cosi + et * cost);
            double rp = (et * cosi - ei * cost) / (et * cosi + ei * cost);
            double F = 0.5 * (rs * rs + rp * rp);
            if (ul < F) *wi = normalize(refl);
            else *wi = normalize(add(mul(d, eta), mul(n, eta * cosi - cost)));
        }
        *weight = v3(1.0, 1.0, 1.0);
        return 1;
    }
    V3 n = dot(ng, d) < 0.0 ? ng : mul(ng, -1.0);
    V3 t, b;
    onb(n, &t, &b);
    if (type == MAT_LAMBERT) {
        /* cosine-weighted hemisphere: pdf cos/pi cancels the BRDF a/pi * cos */
        double r = sqrt(u1), phi = 2.0 * OR_PI * u2;
        V3 l = v3(r * cos(phi), r * sin(phi), sqrt(maxd(0.0, 1.0 - u1)));
        *wi = normalize(to_world(l, t, b, n));
        *weight = alb;
        return 1;
    }
    /* GGX microfacet metal (Walter et al. 2007): sample the normal
       distribution, reflect, weight F G (o.h) / ((n.o)(n.h)), height-
       uncorrelated Smith G = G1(o) G1(i), Schlick F with F0 = albedo. */
    double alpha = m[3] * m[3];
    V3 wo = mul(d, -1.0);
    double no = dot(n, wo);
    if (!(no > 0.0)) return 0;
    double tan2 = alpha * alpha * u1 / (1.0 - u1);
    double ch = 1.0 / sqrt(1.0 + tan2);
    double sh = sqrt(maxd(0.0, 1.0 - ch * ch));
    double phi = 2.0 * OR_PI * u2;
    V3 h = normalize(to_world(v3(sh * cos(phi), sh * sin(phi), ch), t, b, n));
    double oh = dot(wo, h);
    if (!(oh > 0.0)) return 0;
    V3 w = normalize(sub(mul(h, 2.0 * oh), wo));
    double ni = dot(n, w);
    if (!(ni > 0.0)) return 0;
    double nh = dot(n, h);
    double t2o = (1.0 - no * no) / (no * no), t2i = (1.0 - ni * ni) / (ni * ni);
    double G = (2.0 / (1.0 + sqrt(1.0 + alpha * alpha * t2o))) * (2.0 / (1.0 + sqrt(1.0 + alpha * alpha * t2i)));
    double fw = pow(1.0 - oh, 5.0);
    V3 F = v3(alb.x + (1.0 - alb.x) * fw, alb.y + (1.0 - alb.y) * fw, alb.z + (1.0 - alb.z) * fw);
    double k = G * oh / (no * nh);
    *wi = w;
    *weight = mul(F, k);
    return 1;
}

typedef struct {
    const OrScene* s;
    const OrNif* nif;
    const float* env_const;
    OrCam cam;
    int W, H, spp, depth, rr, rr_start;
    uint32_t seed;
    int64_t n_pix;
    const int64_t* pixels;
    double* out;
    double* slot_out;
    int64_t* ids_out;
    int64_t next;
    pthread_mutex_t lock;
} RenderJob;

static V3 env_radiance(const RenderJob* j, V3 d)
{
    if (j->env_const) return v3(j->env_const[0], j->env_const[1], j->env_const[2]);
    if (!j->nif) return v3(0, 0, 0);
    double uv[2], rgb[3];
    dir_to_uv(d, &uv[0], &uv[1]);
    or_nif_forward(j->nif, 1, uv, rgb, NULL);
    return v3(rgb[0], rgb[1], rgb[2]);
}

/* radiance of one path (pixel p, sample s); records the hit ID per bounce */
static V3 trace_path(const RenderJob* j, int64_t pix, int64_t smp, int64_t* ids)
{
    const OrScene* s = j->s;
    uint32_t w[4];
    philox_words(j->seed, 0u, (uint32_t)pix, (uint32_t)smp, 0u, 0u, w);
    V3 o = v3(j->cam.eye[0], j->cam.eye[1], j->cam.eye[2]);
    V3 d = camera_dir(&j->cam, j->W, j->H, (int)(pix % j->W), (int)(pix / j->W), u01(w[0]), u01(w[1]));
    V3 tp = v3(1, 1, 1), L = v3(0, 0, 0);
    if (ids) for (int k = 0; k < j->depth; ++k) ids[k] = -2;
    for (int k = 1; k <= j->depth; ++k) {
        double t;
        int64_t id;
        closest_hit(s, o, d, 0, &t, &id);
        if (ids) ids[k - 1] = id;
        if (id < 0) {
            L = add(L, hadamard(tp, env_radiance(j, d)));
            break;
        }
        V3 p = add(o, mul(d, t));
        int mat = prim_material(s, id);
        const double* m = s->mat + 8 * mat;
        L = add(L, hadamard(tp, v3(m[5], m[6], m[7])));
        if (k == j->depth) break;
        philox_words(j->seed, 0u, (uint32_t)pix, (uint32_t)smp, (uint32_t)k, 0u, w);
        V3 ng = geometric_normal(s, id, p);
        V3 wi, wt;
        if (!sample_bsdf(s, mat, d, ng, u01(w[0]), u01(w[1]), u01(w[2]), &wi, &wt)) break;
        tp = hadamard(tp, wt);
        if (j->rr && k >= j->rr_start) {
            double q = mind(1.0, maxd(tp.x, maxd(tp.y, tp.z)));
            if (u01(w[3]) < q) tp = mul(tp, 1.0 / q);
            else break;
        }
        double eps = 1e-4 * maxd(1.0, maxd(fabs(p.x), maxd(fabs(p.y), fabs(p.z))));
        V3 off = dot(wi, ng) > 0.0 ? ng : mul(ng, -1.0);
        o = add(p, mul(off, eps));
        d = wi;
    }
    return L;
}

static void* render_worker(void* arg)
{
    RenderJob* j = (RenderJob*)arg;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int64_t i = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (i >= j->n_pix) break;
        int64_t pix = j->pixels ? j->pixels[i] : i;
        V3 acc = v3(0, 0, 0);
        for (int smp = 0; smp < j->spp; ++smp) {
            int64_t* ids = j->ids_out ? j->ids_out + (i * j->spp + smp) * j->depth : NULL;
            V3 L = trace_path(j, pix, smp, ids);
            if (j->slot_out) {
                double* so = j->slot_out + 3 * (i * j->spp + smp);
                so[0] = L.x; so[1] = L.y; so[2] = L.z;
            }
            acc = add(acc, L);
        }
        j->out[3 * i] = acc.x / j->spp;
        j->out[3 * i + 1] = acc.y / j->spp;
        j->out[3 * i + 2] = acc.z / j->spp;
    }
    return NULL;
}

/* Render the given pixels (NULL = all W*H).  out: n_pix x 3 mean radiance.
   slot_out (optional): n_pix x spp x 3 per-path radiance.  ids_out
   (optional): n_pix x spp x depth hit primitive IDs (-1 escape, -2 not
   traced). */
OR_API void or_render(const OrScene* s, const OrNif* nif, const float* env_const, const float* cam,
                      int W, int H, int spp, int depth, uint32_t seed, int rr, int rr_start,
                      int64_t n_pix, const int64_t* pixels, double* out, double* slot_out, int64_t* ids_out,
                      int n_threads)
{
    RenderJob j;
    memset(&j, 0, sizeof(j));
    j.s = s; j.nif = nif; j.env_const = env_const;
    make_camera(cam, W, H, &j.cam);
    j.W = W; j.H = H; j.spp = spp; j.depth = depth; j.rr = rr; j.rr_start = rr_start; j.seed = seed;
    j.n_pix = pixels ? n_pix : (int64_t)W * H;
    j.pixels = pixels; j.out = out; j.slot_out = slot_out; j.ids_out = ids_out;
    pthread_mutex_init(&j.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, render_worker, &j);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&j.lock);
}

/* Direct access to one BSDF sample (for closed-form tests of the lobes). */
OR_API int or_sample_bsdf(const OrScene* s, int mat, const double* d, const double* ng, double u1, double u2,
                          double ul, double* wi, double* weight)
{
    V3 w, wt;
    int ok = sample_bsdf(s, mat, v3(d[0], d[1], d[2]), v3(ng[0], ng[1], ng[2]), u1, u2, ul, &w, &wt);
    wi[0] = w.x; wi[1] = w.y; wi[2] = w.z;
    weight[0] = wt.x; weight[1] = wt.y; weight[2] = wt.z;
    if (!ok) { wi[0] = wi[1] = wi[2] = 0.0; weight[0] = weight[1] = weight[2] = 0.0; }
    return ok;
}

/* n independent draws of or_sample_bsdf for one incident direction and
   normal: u is n x 3 (u1, u2, lobe), wi and weight n x 3, ok n flags */
OR_API void or_sample_bsdf_batch(const OrScene* s, int mat, const double* d, const double* ng, int64_t n,
                                 const double* u, double* wi, double* weight, int32_t* ok)
{
    for (int64_t i = 0; i < n; ++i)
        ok[i] = or_sample_bsdf(s, mat, d, ng, u[3 * i], u[3 * i + 1], u[3 * i + 2], wi + 3 * i, weight + 3 * i);
}

/* ------------------------------------------------------------------------ */
/* Neural radiance cache (cited in Section 2.1, Mueller et al. 2021): an MLP */
/* from (position, direction, normal) to outgoing radiance, queried where   */
/* paths terminate early and trained online on the radiance of longer       */
/* training paths.  Encoding: position normalised to the cache's box, then  */
/* [sin(2^j pi p_a) (j < J), cos(2^j pi p_a) (j < J)] per axis a, then the   */
/* direction and the normal (3 + 3).  Hidden ReLU layers, linear output.    */
/* Flat parameters: per layer W (out x in), b (out).                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int J, H, L, nl, in0;
    int in[10], out[10];
    double *W[10], *b[10];
    double lo[3], hi[3];
} OrCache;

OR_API OrCache* or_cache_create(int J, int H, int L, const float* flat, const float* bounds /* lo3 hi3 */)
{
    if (L < 1 || L > 9) return NULL;
    OrCache* c = (OrCache*)calloc(1, sizeof(OrCache));
    c->J = J; c->H = H; c->L = L; c->nl = L + 1; c->in0 = 6 * J + 6;
    const float* p = flat;
    for (int l = 0; l < c->nl; ++l) {
        c->in[l] = l == 0 ? c->in0 : H;
        c->out[l] = l == c->nl - 1 ? 3 : H;
        c->W[l] = (double*)malloc(sizeof(double) * c->in[l] * c->out[l]);
        c->b[l] = (double*)malloc(sizeof(double) * c->out[l]);
        for (int i = 0; i < c->in[l] * c->out[l]; ++i) c->W[l][i] = *p++;
        for (int i = 0; i < c->out[l]; ++i) c->b[l][i] = *p++;
    }
    for (int a = 0; a < 3; ++a) { c->lo[a] = bounds[a]; c->hi[a] = bounds[3 + a]; }
    return c;
}

OR_API void or_cache_destroy(OrCache* c)
{
    if (!c) return;
    for (int l = 0; l < c->nl; ++l) { free(c->W[l]); free(c->b[l]); }
    free(c);
}

OR_API int64_t or_cache_n_params(const OrCache* c)
{
    int64_t n = 0;
    for (int l = 0; l < c->nl; ++l) n += (int64_t)c->in[l] * c->out[l] + c->out[l];
    return n;
}

OR_API void or_cache_get_params(const OrCache* c, double* out)
{
    double* p = out;
    for (int l = 0; l < c->nl; ++l) {
        memcpy(p, c->W[l], sizeof(double) * c->in[l] * c->out[l]); p += c->in[l] * c->out[l];
        memcpy(p, c->b[l], sizeof(double) * c->out[l]); p += c->out[l];
    }
}
OR_API void or_cache_set_params(OrCache* c, const double* in)
{
    const double* p = in;
    for (int l = 0; l < c->nl; ++l) {
        memcpy(c->W[l], p, sizeof(double) * c->in[l] * c->out[l]); p += c->in[l] * c->out[l];
        memcpy(c->b[l], p, sizeof(double) * c->out[l]); p += c->out[l];
    }
}

/* query = (x, direction, normal) -> encoding e [in0] */
static void cache_encode(const OrCache* c, const double* q, double* e)
{
    int k = 0;
    for (int a = 0; a < 3; ++a) {
        double p = (q[a] - c->lo[a]) / (c->hi[a] - c->lo[a]);
        for (int j = 0; j < c->J; ++j) e[k + j] = sin(ldexp(1.0, j) * OR_PI * p);
        for (int j = 0; j < c->J; ++j) e[k + c->J + j] = cos(ldexp(1.0, j) * OR_PI * p);
        k += 2 * c->J;
    }
    for (int i = 0; i < 6; ++i) e[k + i] = q[3 + i];
}

static void cache_forward_one(const OrCache* c, const double* q, double* enc, double* hid, double* pre, double y[3])
{
    cache_encode(c, q, enc);
    const double* x = enc;
    for (int l = 0; l < c->L; ++l) {
        double* h = hid + (size_t)l * c->H;
        for (int j = 0; j < c->H; ++j) {
            double acc = c->b[l][j];
            for (int k = 0; k < c->in[l]; ++k) acc += c->W[l][(size_t)j * c->in[l] + k] * x[k];
            if (pre) pre[(size_t)l * c->H + j] = acc;
            h[j] = acc > 0.0 ? acc : 0.0;
        }
        x = h;
    }
    int lo = c->nl - 1;
    for (int j = 0; j < 3; ++j) {
        double acc = c->b[lo][j];
        for (int k = 0; k < c->H; ++k) acc += c->W[lo][(size_t)j * c->H + k] * x[k];
        y[j] = acc;
    }
}

OR_API void or_cache_forward(const OrCache* c, int64_t n, const double* q /* n x 9 */, double* out /* n x 3 */)
{
    double* enc = (double*)malloc(sizeof(double) * c->in0);
    double* hid = (double*)malloc(sizeof(double) * c->L * c->H);
    for (int64_t i = 0; i < n; ++i) cache_forward_one(c, q + 9 * i, enc, hid, NULL, out + 3 * i);
    free(enc); free(hid);
}

/* Relative L2 loss (Mueller et al. 2021): mean over samples and channels of
   (y - t)^2 / (sg(y)^2 + 0.01), where sg() holds the prediction constant in
   the gradient.  denom (optional, n x 3) replaces sg(y)^2 + 0.01 by fixed
   values, which makes the loss an ordinary function of the weights.  mask
   (optional, n) excludes samples; the mean is over all n x 3 entries. */
OR_API double or_cache_loss_grad(const OrCache* c, int64_t n, const double* q, const double* target,
                                 const double* denom, const int32_t* mask, double* grad)
{
    int H = c->H, L = c->L;
    int64_t np = or_cache_n_params(c);
    memset(grad, 0, sizeof(double) * (size_t)np);
    double* gW[10]; double* gb[10];
    double* p = grad;
    for (int l = 0; l < c->nl; ++l) { gW[l] = p; p += c->in[l] * c->out[l]; gb[l] = p; p += c->out[l]; }
    double* enc = (double*)malloc(sizeof(double) * c->in0);
    double* hid = (double*)malloc(sizeof(double) * L * H);
    double* pre = (double*)malloc(sizeof(double) * L * H);
    double* dh = (double*)malloc(sizeof(double) * H);
    double* dprev = (double*)malloc(sizeof(double) * H);
    double loss = 0.0, scale = 1.0 / (3.0 * (double)n);
    for (int64_t s = 0; s < n; ++s) {
        if (mask && !mask[s]) continue;
        double y[3], dy[3];
        cache_forward_one(c, q + 9 * s, enc, hid, pre, y);
        for (int ch = 0; ch < 3; ++ch) {
            double d = denom ? denom[3 * s + ch] : y[ch] * y[ch] + 0.01;
            double r = y[ch] - target[3 * s + ch];
            loss += r * r / d * scale;
            dy[ch] = 2.0 * r / d * scale;
        }
        int lo = c->nl - 1;
        const double* xin = hid + (size_t)(L - 1) * H;
        for (int j = 0; j < 3; ++j) {
            gb[lo][j] += dy[j];
            for (int k = 0; k < H; ++k) gW[lo][(size_t)j * H + k] += dy[j] * xin[k];
        }
        for (int k = 0; k < H; ++k) {
            double acc = 0.0;
            for (int j = 0; j < 3; ++j) acc += c->W[lo][(size_t)j * H + k] * dy[j];
            dh[k] = acc;
        }
        for (int l = L - 1; l >= 0; --l) {
            const double* pl = pre + (size_t)l * H;
            for (int j = 0; j < H; ++j) dh[j] = pl[j] > 0.0 ? dh[j] : 0.0;
            const double* x = (l == 0) ? enc : hid + (size_t)(l - 1) * H;
            int nin = c->in[l];
            for (int j = 0; j < H; ++j) {
                gb[l][j] += dh[j];
                for (int k = 0; k < nin; ++k) gW[l][(size_t)j * nin + k] += dh[j] * x[k];
            }
            if (l > 0) {
                for (int k = 0; k < H; ++k) {
                    double acc = 0.0;
                    for (int j = 0; j < H; ++j) acc += c->W[l][(size_t)j * nin + k] * dh[j];
                    dprev[k] = acc;
                }
                memcpy(dh, dprev, sizeof(double) * H);
            }
        }
    }
    free(enc); free(hid); free(pre); free(dh); free(dprev);
    return loss;
}

/* Path with the cache: like trace_path, but a hit at vertex cache_vertex
   adds tp * max(cache(x, -d, n), 0) and ends the path (n faces the incoming
   ray).  Records at rec_vertex (rec, 16 doubles: x, -d, n, tp, gathered
   radiance before the vertex, valid) when rec is given. */
static V3 trace_path_ex(const RenderJob* j, int64_t pix, int64_t smp, int64_t* ids, const OrCache* cache,
                        int cache_vertex, int rec_vertex, double* rec)
{
    const OrScene* s = j->s;
    uint32_t w[4];
    philox_words(j->seed, 0u, (uint32_t)pix, (uint32_t)smp, 0u, 0u, w);
    V3 o = v3(j->cam.eye[0], j->cam.eye[1], j->cam.eye[2]);
    V3 d = camera_dir(&j->cam, j->W, j->H, (int)(pix % j->W), (int)(pix / j->W), u01(w[0]), u01(w[1]));
    V3 tp = v3(1, 1, 1), L = v3(0, 0, 0);
    if (ids) for (int k = 0; k < j->depth; ++k) ids[k] = -2;
    if (rec) for (int k = 0; k < 16; ++k) rec[k] = 0.0;
    for (int k = 1; k <= j->depth; ++k) {
        double t;
        int64_t id;
        closest_hit(s, o, d, 0, &t, &id);
        if (ids) ids[k - 1] = id;
        if (id < 0) {
            L = add(L, hadamard(tp, env_radiance(j, d)));
            break;
        }
        V3 p = add(o, mul(d, t));
        V3 ng = geometric_normal(s, id, p);
        V3 nf = dot(ng, d) < 0.0 ? ng : mul(ng, -1.0);
        if (rec && k == rec_vertex) {
            double v[16] = {p.x, p.y, p.z, -d.x, -d.y, -d.z, nf.x, nf.y, nf.z, tp.x, tp.y, tp.z, L.x, L.y, L.z, 1.0};
            memcpy(rec, v, sizeof v);
        }
        if (cache && k == cache_vertex) {
            double q[9] = {p.x, p.y, p.z, -d.x, -d.y, -d.z, nf.x, nf.y, nf.z}, y[3];
            or_cache_forward(cache, 1, q, y);
            L = add(L, hadamard(tp, v3(maxd(y[0], 0.0), maxd(y[1], 0.0), maxd(y[2], 0.0))));
            break;
        }
        int mat = prim_material(s, id);
        const double* m = s->mat + 8 * mat;
        L = add(L, hadamard(tp, v3(m[5], m[6], m[7])));
        if (k == j->depth) break;
        philox_words(j->seed, 0u, (uint32_t)pix, (uint32_t)smp, (uint32_t)k, 0u, w);
        V3 wi, wt;
        if (!sample_bsdf(s, mat, d, ng, u01(w[0]), u01(w[1]), u01(w[2]), &wi, &wt)) break;
        tp = hadamard(tp, wt);
        if (j->rr && k >= j->rr_start) {
            double qq = mind(1.0, maxd(tp.x, maxd(tp.y, tp.z)));
            if (u01(w[3]) < qq) tp = mul(tp, 1.0 / qq);
            else break;
        }
        double eps = 1e-4 * maxd(1.0, maxd(fabs(p.x), maxd(fabs(p.y), fabs(p.z))));
        V3 off = dot(wi, ng) > 0.0 ? ng : mul(ng, -1.0);
        o = add(p, mul(off, eps));
        d = wi;
    }
    return L;
}

/* Paths (pixel[i], sample[i]) with an optional cache at cache_vertex (0 =
   none) and vertex records at rec_vertex (0 = none): L_out [n][3], rec_out
   [n][16] (nullable), ids_out [n][depth] (nullable).  Single-threaded. */
OR_API void or_trace_paths(const OrScene* s, const OrNif* nif, const float* env_const, const float* cam, int W, int H,
                           int depth, uint32_t seed, int64_t n, const int64_t* pixels, const int64_t* samples,
                           const OrCache* cache, int cache_vertex, int rec_vertex, double* L_out, double* rec_out,
                           int64_t* ids_out)
{
    RenderJob j;
    memset(&j, 0, sizeof(j));
    j.s = s; j.nif = nif; j.env_const = env_const;
    make_camera(cam, W, H, &j.cam);
    j.W = W; j.H = H; j.spp = 1; j.depth = depth; j.seed = seed;
    for (int64_t i = 0; i < n; ++i) {
        V3 L = trace_path_ex(&j, pixels[i], samples[i], ids_out ? ids_out + i * depth : NULL, cache, cache_vertex,
                             rec_vertex, rec_out ? rec_out + 16 * i : NULL);
        L_out[3 * i] = L.x; L_out[3 * i + 1] = L.y; L_out[3 * i + 2] = L.z;
    }
}
