// Device helpers of the path tracer: counter-based RNG, small vector math,
// ray-primitive tests and BVH traversal.  FP32 throughout.
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

#include "pt_internal.h"

namespace ptk {

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with a Weyl-sequence key schedule.  It stands in
// for the IPU's hardware generator (Section 3.1.3).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// uniform in [0, 1): top 24 bits times 2^-24 (exact)
__device__ __forceinline__ float u01(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 norm3(float3 a) { return a * rsqrtf(dot3(a, a)); }
__device__ __forceinline__ float comp3(float3 a, int i) { return i == 0 ? a.x : (i == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Fourier features with an error-free phase (Section 3.2's positional
// embedding evaluated in FP32): t = B0 u + B1 v is carried as an unevaluated
// sum hi + lo (exact products via fma, exact sum via TwoSum), the integer
// part is removed exactly, and sinpi/cospi of 2r give sin(2 pi t) and
// cos(2 pi t) to ~1e-7 absolute even for |t| ~ 100 turns.
__device__ __forceinline__ void fourier_feature(float b0, float b1, float u, float v, float& s, float& c)
{
    const float p0 = b0 * u, e0 = fmaf(b0, u, -p0);
    const float p1 = b1 * v, e1 = fmaf(b1, v, -p1);
    const float hi = p0 + p1;
    const float bp = hi - p0;
    const float es = (p0 - (hi - bp)) + (p1 - bp);
    const float lo = e0 + e1 + es;
    const float n = rintf(hi);
    const float r = (hi - n) + lo;
    sincospif(2.f * r, &s, &c);
}

// Radiance-cache position encoding (frequency encoding of Mueller et al.
// 2021): p = (q - lo) / ext carried as a float pair ph + pl (TwoSum for the
// numerator, ext = eh + el exact, one correction step for the quotient), so
// that the top frequencies 2^j p keep a phase error of ~1e-7 instead of
// 2^j ulp(p).  Writes sin(2^j pi p) to s[j] and cos(2^j pi p) to c[j].
__device__ __forceinline__ void cache_axis_features(float q, float lo, float eh, float el, int J, float* s, int s_stride,
                                                    float* c, int c_stride)
{
    const float d = q - lo;
    const float bv = d - q;
    const float e = (q - (d - bv)) + (-lo - bv);           // q - lo = d + e exactly
    const float ph = __fdiv_rn(d, eh);
    const float rem = fmaf(-ph, eh, d) + e - ph * el;      // first term exact
    const float pl = __fdiv_rn(rem, eh);
    float sc = 1.f;
    for (int j = 0; j < J; ++j) {
        const float x = ph * sc;                            // exact: power-of-two scale
        const float xr = x - 2.f * floorf(0.5f * x);        // exact removal of whole turns
        float sv, cv;
        sincospif(xr + pl * sc, &sv, &cv);
        s[j * s_stride] = sv;
        c[j * c_stride] = cv;
        sc *= 2.f;
    }
}

// ---------------------------------------------------------------------------
// Ray-primitive tests (Section 3.1.3).  Each returns t > 0 or +inf.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float isect_sphere(float4 s, float3 o, float3 d)
{
    // closest-approach discriminant, product form for the second root
    const float3 oc = o - f3(s.x, s.y, s.z);
    const float b = dot3(oc, d);
    const float3 l = oc - d * b;
    const float disc = s.w * s.w - dot3(l, l);
    if (disc < 0.f) return INFINITY;
    const float sq = sqrtf(disc);
    const float q = -b - copysignf(sq, b);
    const float cc = dot3(oc, oc) - s.w * s.w;
    const float t0 = q, t1 = cc / q;
    const float tn = fminf(t0, t1), tf = fmaxf(t0, t1);
    return tn > 0.f ? tn : (tf > 0.f ? tf : INFINITY);
}

__device__ __forceinline__ float isect_quad(float4 q0, float4 q1, float3 o, float3 d)
{
    const int a = __float_as_int(q1.y);
    const int u = a == 2 ? 0 : a + 1, v = a == 0 ? 2 : a - 1;  // (a+1)%3, (a+2)%3
    const float t = (q0.x - comp3(o, a)) / comp3(d, a);
    if (!(t > 0.f) || !(t < INFINITY)) return INFINITY;
    const float pu = comp3(o, u) + t * comp3(d, u);
    const float pv = comp3(o, v) + t * comp3(d, v);
    if (pu < q0.y || pu > q0.z || pv < q0.w || pv > q1.x) return INFINITY;
    return t;
}

// Per-ray set-up of the watertight triangle test (Woop, Benthin, Wald 2013).
struct TriRay {
    int kx, ky, kz;
    float Sx, Sy, Sz;
    float ox, oy, oz;   // origin permuted
};

__device__ __forceinline__ TriRay tri_setup(float3 o, float3 d)
{
    TriRay r;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dz = comp3(d, kz);
    if (dz < 0.f) { int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.Sx = comp3(d, kx) / dz;
    r.Sy = comp3(d, ky) / dz;
    r.Sz = 1.f / dz;
    r.ox = comp3(o, kx); r.oy = comp3(o, ky); r.oz = comp3(o, kz);
    return r;
}

// Edge functions are evaluated with explicitly rounded products so that the
// two triangles sharing an edge compute exactly negated values (no FMA
// contraction), which is what makes the test watertight.
__device__ __forceinline__ float edge_fn(float ax, float ay, float bx, float by)
{
    return __fsub_rn(__fmul_rn(ax, by), __fmul_rn(ay, bx));
}

__device__ __forceinline__ float isect_tri(const TriRay& r, float4 v0, float4 v1, float4 v2)
{
    const float3 p0 = f3(v0.x, v0.y, v0.z), p1 = f3(v1.x, v1.y, v1.z), p2 = f3(v2.x, v2.y, v2.z);
    const float Az = comp3(p0, r.kz) - r.oz, Bz = comp3(p1, r.kz) - r.oz, Cz = comp3(p2, r.kz) - r.oz;
    const float Ax = __fsub_rn(comp3(p0, r.kx) - r.ox, __fmul_rn(r.Sx, Az));
    const float Ay = __fsub_rn(comp3(p0, r.ky) - r.oy, __fmul_rn(r.Sy, Az));
    const float Bx = __fsub_rn(comp3(p1, r.kx) - r.ox, __fmul_rn(r.Sx, Bz));
    const float By = __fsub_rn(comp3(p1, r.ky) - r.oy, __fmul_rn(r.Sy, Bz));
    const float Cx = __fsub_rn(comp3(p2, r.kx) - r.ox, __fmul_rn(r.Sx, Cz));
    const float Cy = __fsub_rn(comp3(p2, r.ky) - r.oy, __fmul_rn(r.Sy, Cz));
    float U = edge_fn(Cx, Cy, Bx, By);
    float V = edge_fn(Ax, Ay, Cx, Cy);
    float W = edge_fn(Bx, By, Ax, Ay);
    if (U == 0.f || V == 0.f || W == 0.f) {
        // exactly on an edge in float: decide in double (as PBRT-v3 does)
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return INFINITY;
    const float det = U + V + W;
    if (det == 0.f) return INFINITY;
    const float T = U * (r.Sz * Az) + V * (r.Sz * Bz) + W * (r.Sz * Cz);
    const float t = T / det;
    return (t > 0.f && t < INFINITY) ? t : INFINITY;
}

// ---------------------------------------------------------------------------
// Closest hit through the packed BVH with a per-thread short stack.
// ---------------------------------------------------------------------------
struct Hit { float t; int32_t prim; };

// Traversal work of one ray: child-pair node fetches and primitive tests by
// kind (the algorithmic work behind the traversal roofline).
struct Work { uint32_t nodes = 0, sph = 0, quad = 0, tri = 0; };

__device__ __forceinline__ void isect_prim(const DevScene& sc, uint32_t id, float3 o, float3 d, const TriRay& tr,
                                           float& tbest, int32_t& best, Work& w)
{
    float t;
    if (id < sc.nS) {
        ++w.sph;
        t = isect_sphere(__ldg(&sc.sph[id]), o, d);
    } else if (id < sc.nS + sc.nQ) {
        ++w.quad;
        const uint32_t q = id - sc.nS;
        t = isect_quad(__ldg(&sc.quad[2 * q]), __ldg(&sc.quad[2 * q + 1]), o, d);
    } else {
        ++w.tri;
        const uint32_t q = id - sc.nS - sc.nQ;
        t = isect_tri(tr, __ldg(&sc.tri[3 * q]), __ldg(&sc.tri[3 * q + 1]), __ldg(&sc.tri[3 * q + 2]));
    }
    if (t < tbest || (t == tbest && t < INFINITY && (int32_t)id < best)) { tbest = t; best = (int32_t)id; }
}

__device__ __forceinline__ float half_bits_to_float(uint32_t bits16) { return __half2float(__ushort_as_half((unsigned short)bits16)); }

// slab test of one child box [lo, hi]; returns entry distance or +inf
__device__ __forceinline__ float slab_box(float3 lo, float3 hi, float3 o, float3 inv, float tbest)
{
    const float tx0 = (lo.x - o.x) * inv.x, tx1 = (hi.x - o.x) * inv.x;
    const float ty0 = (lo.y - o.y) * inv.y, ty1 = (hi.y - o.y) * inv.y;
    const float tz0 = (lo.z - o.z) * inv.z, tz1 = (hi.z - o.z) * inv.z;
    const float tmin = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.f));
    float tmax = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
    tmax *= 1.0000004f;  // 1 + 2 gamma_3 (PBRT): rounding can never drop a true hit
    return (tmin <= tmax && tmin <= tbest) ? tmin : INFINITY;
}
// the same for a box stored as lo + extent (hi = lo + ext rounded in FP32)
__device__ __forceinline__ float slab(float3 lo, float3 ext, float3 o, float3 inv, float tbest)
{
    return slab_box(lo, lo + ext, o, inv, tbest);
}

__device__ __forceinline__ float safe_inv(float d) { return 1.f / (fabsf(d) > 1e-30f ? d : copysignf(1e-30f, d)); }

// Resumable closest-hit traversal: trav_init sets up a ray, trav_step
// visits one node (both children's boxes, leaf children intersected right
// away, near child first, far child stacked with its entry distance).  Both
// return true once the ray's closest hit is final.
struct Trav {
    float3 o, d, inv;
    TriRay tr;
    Hit h;
    uint32_t cur, iters;
    int sp;
};

__device__ __forceinline__ bool trav_init(const DevScene& sc, float3 o, float3 d, Trav& s, Work& w)
{
    s.o = o;
    s.d = d;
    s.h = Hit{INFINITY, -1};
    s.cur = sc.root;
    s.sp = 0;
    s.iters = 0;
    if (s.cur == kEmptyRef) return true;
    if (sc.nT) s.tr = tri_setup(o, d);  // only triangles use the sheared ray
    if (s.cur & kLeafBit) {
        isect_prim(sc, s.cur & ~kLeafBit, o, d, s.tr, s.h.t, s.h.prim, w);
        return true;
    }
    s.inv = f3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    return false;
}

// node forms the traversal reads (DevScene: nodes, wnodes, qnodes)
constexpr int kNodesPacked = 0, kNodesWide = 1, kNodesQuant = 2;

// byte k (0..3) of w as a float
__device__ __forceinline__ float byte_f(uint32_t w, int k) { return (float)((w >> (8 * k)) & 0xFFu); }

// Node `cur`'s two child references and the entry distances of the ray
// (origin o, reciprocal direction inv) into their boxes, +inf for a box
// missed or entered beyond tbest.
template <int kForm>
__device__ __forceinline__ void node_children(const DevScene& sc, uint32_t cur, float3 o, float3 inv, float tbest,
                                              uint32_t& cl, uint32_t& cr, float& tl, float& trr)
{
    if (kForm == kNodesQuant) {
        // 8-bit grid boxes: bound = origin + q * 2^(e - 127 - d_axis), exact product, one rounding
        const uint4* np = sc.qnodes + 2 * (size_t)cur;
        const uint4 q0 = __ldg(np), q1 = __ldg(np + 1);
        const float3 org = f3(__uint_as_float(q0.x), __uint_as_float(q0.y), __uint_as_float(q0.z));
        const uint32_t meta = q0.w, e = meta & 0xFFu;
        const float3 step = f3(__uint_as_float((e - ((meta >> 8) & 3u)) << 23),
                               __uint_as_float((e - ((meta >> 10) & 3u)) << 23),
                               __uint_as_float((e - ((meta >> 12) & 3u)) << 23));
        cl = ((meta >> 16) | ((q1.x & 0xFFu) << 16)) | ((meta & (1u << 14)) ? kLeafBit : 0u);
        cr = (q1.x >> 8) | ((meta & (1u << 15)) ? kLeafBit : 0u);
        const float3 lo_l = f3(fmaf(byte_f(q1.y, 0), step.x, org.x), fmaf(byte_f(q1.y, 1), step.y, org.y),
                               fmaf(byte_f(q1.y, 2), step.z, org.z));
        const float3 hi_l = f3(fmaf(byte_f(q1.y, 3), step.x, org.x), fmaf(byte_f(q1.z, 0), step.y, org.y),
                               fmaf(byte_f(q1.z, 1), step.z, org.z));
        const float3 lo_r = f3(fmaf(byte_f(q1.z, 2), step.x, org.x), fmaf(byte_f(q1.z, 3), step.y, org.y),
                               fmaf(byte_f(q1.w, 0), step.z, org.z));
        const float3 hi_r = f3(fmaf(byte_f(q1.w, 1), step.x, org.x), fmaf(byte_f(q1.w, 2), step.y, org.y),
                               fmaf(byte_f(q1.w, 3), step.z, org.z));
        tl = slab_box(lo_l, hi_l, o, inv, tbest);
        trr = slab_box(lo_r, hi_r, o, inv, tbest);
    } else if (kForm == kNodesWide) {
        // decoded boxes: the same bounds the packed form decodes to, without the fp16 conversions
        const uint4* np = sc.wnodes + 4 * (size_t)cur;
        const uint4 q0 = __ldg(np), q1 = __ldg(np + 1), q2 = __ldg(np + 2), q3 = __ldg(np + 3);
        const float3 lo_l = f3(__uint_as_float(q0.x), __uint_as_float(q0.y), __uint_as_float(q0.z));
        const float3 hi_l = f3(__uint_as_float(q0.w), __uint_as_float(q1.x), __uint_as_float(q1.y));
        const float3 lo_r = f3(__uint_as_float(q1.z), __uint_as_float(q1.w), __uint_as_float(q2.x));
        const float3 hi_r = f3(__uint_as_float(q2.y), __uint_as_float(q2.z), __uint_as_float(q2.w));
        cl = q3.x;
        cr = q3.y;
        tl = slab_box(lo_l, hi_l, o, inv, tbest);
        trr = slab_box(lo_r, hi_r, o, inv, tbest);
    } else {
        const uint4* np = sc.nodes + 3 * (size_t)cur;
        const uint4 q0 = __ldg(np), q1 = __ldg(np + 1), q2 = __ldg(np + 2);
        const float3 lo_l = f3(__uint_as_float(q0.x), __uint_as_float(q0.y), __uint_as_float(q0.z));
        const float3 lo_r = f3(__uint_as_float(q0.w), __uint_as_float(q1.x), __uint_as_float(q1.y));
        const float3 ext_l = f3(half_bits_to_float(q1.z & 0xFFFFu), half_bits_to_float(q1.z >> 16),
                                half_bits_to_float(q1.w & 0xFFFFu));
        const float3 ext_r = f3(half_bits_to_float(q1.w >> 16), half_bits_to_float(q2.x & 0xFFFFu),
                                half_bits_to_float(q2.x >> 16));
        cl = q2.y;
        cr = q2.z;
        tl = slab(lo_l, ext_l, o, inv, tbest);
        trr = slab(lo_r, ext_r, o, inv, tbest);
    }
}

template <int kForm>
__device__ __forceinline__ bool trav_step(const DevScene& sc, Trav& s, uint32_t* stack_ref, float* stack_t,
                                          uint32_t* err, Work& w)
{
    if (++s.iters > kIterCap) { atomicOr(err, PT_ERR_ITER_CAP); return true; }
    if (s.cur >= sc.n_nodes) { atomicOr(err, PT_ERR_BAD_NODE); return true; }  // never fetch outside the node array
    uint32_t cl, cr;
    float tl, trr;
    node_children<kForm>(sc, s.cur, s.o, s.inv, s.h.t, cl, cr, tl, trr);
    ++w.nodes;
    // leaf children are intersected right away
    if ((cl & kLeafBit) && tl < INFINITY) {
        isect_prim(sc, cl & ~kLeafBit, s.o, s.d, s.tr, s.h.t, s.h.prim, w);
        tl = INFINITY;
    }
    if ((cr & kLeafBit) && trr < INFINITY) {
        isect_prim(sc, cr & ~kLeafBit, s.o, s.d, s.tr, s.h.t, s.h.prim, w);
        trr = INFINITY;
    }
    // a child is entered only if its box was hit (finite entry) no later than the best hit
    const bool hl = tl < INFINITY && tl <= s.h.t, hr = trr < INFINITY && trr <= s.h.t;
    if (hl && hr) {
        const bool left_first = tl <= trr;
        if (s.sp >= kStackSize) { atomicOr(err, PT_ERR_STACK_OVERFLOW); return true; }
        stack_ref[s.sp] = left_first ? cr : cl;
        stack_t[s.sp] = left_first ? trr : tl;
        ++s.sp;
        s.cur = left_first ? cl : cr;
        return false;
    }
    if (hl) { s.cur = cl; return false; }
    if (hr) { s.cur = cr; return false; }
    while (s.sp > 0) {
        --s.sp;
        if (stack_t[s.sp] <= s.h.t) { s.cur = stack_ref[s.sp]; return false; }
    }
    return true;
}

__device__ __forceinline__ Hit trace_closest(const DevScene& sc, float3 o, float3 d, uint32_t* err, Work& w)
{
    Trav s;
    if (trav_init(sc, o, d, s, w)) return s.h;
    uint32_t stack_ref[kStackSize];
    float stack_t[kStackSize];
    while (!trav_step<kNodesPacked>(sc, s, stack_ref, stack_t, err, w)) {
    }
    return s.h;
}

}  // namespace ptk
