// Wavefront path tracing kernels (Section 3.1): camera rays from Philox
// words, closest-hit traversal, BSDF sampling of the next bounce, and
// warp-aggregated compaction of surviving rays and environment escapes.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace ptk {

namespace {

constexpr float kPi = 3.14159265358979323846f;

struct PathState {
    float3 o, d, tp, L;
    uint32_t slot;
};

__device__ __forceinline__ void slot_to_pixel(const BounceParams& p, uint32_t j, uint32_t& pix, uint32_t& smp)
{
    // a call renders fewer than 2^32 paths (checked on the host), so 32-bit arithmetic is exact
    const uint32_t g = (uint32_t)(p.chunk_first + j);
    const uint32_t s = g / p.n_pix;
    const uint32_t i = g - s * p.n_pix;
    smp = s + (p.first_sample_dev ? __ldg(p.first_sample_dev) : p.first_sample);
    pix = p.pixels ? (uint32_t)p.pixels[i] : i;
}

// Order in which the camera rays of a chunk are taken: the j-th ray is the
// path of slot tile_slot(j).  For a whole image with W % 8 == 0 and
// H % 4 == 0, 32 consecutive rays cover an 8 x 4 pixel tile of one sample
// instead of 32 pixels of one row (more coherent warps); a bijection of the
// chunk's slots, so every path is traced once and keeps its own slot.
__device__ __forceinline__ uint32_t tile_slot(const BounceParams& p, uint32_t j)
{
    if (!p.tiled) return j;
    const uint32_t s = j / p.n_pix, q = j - s * p.n_pix;
    const uint32_t b = q >> 5, l = q & 31u;
    const uint32_t per_band = (uint32_t)p.W >> 3;
    const uint32_t band = b / per_band, bx = b - band * per_band;
    return s * p.n_pix + (band * 4u + (l >> 3)) * (uint32_t)p.W + bx * 8u + (l & 7u);
}

__device__ __forceinline__ float3 camera_dir(const DevScene& sc, int W, int H, uint32_t pix, float jx, float jy)
{
    const float x = (float)(pix % (uint32_t)W), y = (float)(pix / (uint32_t)W);
    const float fx = ((x + jx) / (float)W * 2.f - 1.f) * sc.tan_half * sc.aspect;
    const float fy = (1.f - (y + jy) / (float)H * 2.f) * sc.tan_half;
    const float3 d = f3(fx * sc.right[0] + fy * sc.up[0] + sc.fwd[0], fx * sc.right[1] + fy * sc.up[1] + sc.fwd[1],
                        fx * sc.right[2] + fy * sc.up[2] + sc.fwd[2]);
    return norm3(d);
}

__device__ __forceinline__ float3 geometric_normal(const DevScene& sc, uint32_t id, float3 p)
{
    if (id < sc.nS) {
        const float4 s = __ldg(&sc.sph[id]);
        return norm3(p - f3(s.x, s.y, s.z));
    }
    if (id < sc.nS + sc.nQ) {
        const int a = __float_as_int(__ldg(&sc.quad[2 * (id - sc.nS) + 1]).y);
        return f3(a == 0 ? 1.f : 0.f, a == 1 ? 1.f : 0.f, a == 2 ? 1.f : 0.f);
    }
    const uint32_t q = id - sc.nS - sc.nQ;
    const float4 v0 = __ldg(&sc.tri[3 * q]), v1 = __ldg(&sc.tri[3 * q + 1]), v2 = __ldg(&sc.tri[3 * q + 2]);
    return norm3(cross3(f3(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z), f3(v2.x - v0.x, v2.y - v0.y, v2.z - v0.z)));
}

// Orthonormal basis around unit n (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b)
{
    const float sign = copysignf(1.f, n.z);
    const float a = -1.f / (sign + n.z);
    const float bb = n.x * n.y * a;
    t = f3(1.f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    b = f3(bb, sign + n.y * n.y * a, -n.y);
}

// Sample the next direction at a hit; false = absorbed.
__device__ __forceinline__ bool sample_bsdf(const DevScene& sc, int32_t mat, float3 d, float3 ng, float u1, float u2,
                                            float ul, float3& wi, float3& wt)
{
    const float4 m0 = __ldg(&sc.mat[2 * mat]), m1 = __ldg(&sc.mat[2 * mat + 1]);
    const int type = __ldg(&sc.mat_type[mat]);
    if (type == 2) {  // dielectric: exact unpolarised Fresnel, reflect w.p. F, weight 1
        const bool entering = dot3(d, ng) < 0.f;
        const float3 n = entering ? ng : ng * -1.f;
        const float ei = entering ? 1.f : m1.x, et = entering ? m1.x : 1.f;
        const float cosi = -dot3(d, n);
        const float eta = ei / et;
        const float sin2t = eta * eta * (1.f - cosi * cosi);
        const float3 refl = d + n * (2.f * cosi);
        if (sin2t >= 1.f) {
            wi = norm3(refl);
        } else {
            const float cost = sqrtf(1.f - sin2t);
            const float rs = (ei * cosi - et * cost) / (ei * cosi + et * cost);
            const float rp = (et * cosi - ei * cost) / (et * cosi + ei * cost);
            const float F = 0.5f * (rs * rs + rp * rp);
            wi = (ul < F) ? norm3(refl) : norm3(d * eta + n * (eta * cosi - cost));
        }
        wt = f3(1.f, 1.f, 1.f);
        return true;
    }
    const float3 n = dot3(ng, d) < 0.f ? ng : ng * -1.f;
    float3 t, b;
    onb(n, t, b);
    if (type == 0) {  // Lambertian, cosine-weighted hemisphere
        const float r = sqrtf(u1);
        float sp, cp;
        sincospif(2.f * u2, &sp, &cp);
        const float lz = sqrtf(fmaxf(0.f, 1.f - u1));
        wi = norm3(t * (r * cp) + b * (r * sp) + n * lz);
        wt = f3(m0.x, m0.y, m0.z);
        return true;
    }
    // GGX metal: sample the normal distribution (Walter et al. 2007), reflect
    const float alpha = m0.w * m0.w;
    const float3 wo = d * -1.f;
    const float no = dot3(n, wo);
    if (!(no > 0.f)) return false;
    const float tan2 = alpha * alpha * u1 / (1.f - u1);
    const float ch = rsqrtf(1.f + tan2);
    const float sh = sqrtf(fmaxf(0.f, 1.f - ch * ch));
    float sp, cp;
    sincospif(2.f * u2, &sp, &cp);
    const float3 h = norm3(t * (sh * cp) + b * (sh * sp) + n * ch);
    const float oh = dot3(wo, h);
    if (!(oh > 0.f)) return false;
    const float3 w = norm3(h * (2.f * oh) - wo);
    const float ni = dot3(n, w);
    if (!(ni > 0.f)) return false;
    const float nh = dot3(n, h);
    const float t2o = (1.f - no * no) / (no * no), t2i = (1.f - ni * ni) / (ni * ni);
    const float a2 = alpha * alpha;
    const float G = (2.f / (1.f + sqrtf(1.f + a2 * t2o))) * (2.f / (1.f + sqrtf(1.f + a2 * t2i)));
    const float x = 1.f - oh, x2 = x * x, fw = x2 * x2 * x;
    const float k = G * oh / (no * nh);
    wi = w;
    wt = f3((m0.x + (1.f - m0.x) * fw) * k, (m0.y + (1.f - m0.y) * fw) * k, (m0.z + (1.f - m0.z) * fw) * k);
    return true;
}

// Warp-aggregated append: returns this lane's index in the queue.
__device__ __forceinline__ uint32_t warp_append(bool pred, uint32_t* counter)
{
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (mask) {
        const int leader = __ffs(mask) - 1;
        if (lane == leader) base = atomicAdd(counter, (uint32_t)__popc(mask));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
    }
    return base + __popc(mask & ((1u << lane) - 1u));
}

__device__ __forceinline__ void store_L(float* slot_L, uint32_t slot, float3 L, uint32_t* err)
{
    if (!(isfinite(L.x) && isfinite(L.y) && isfinite(L.z))) atomicOr(err, PT_ERR_NONFINITE);
    slot_L[3 * (size_t)slot] = L.x;
    slot_L[3 * (size_t)slot + 1] = L.y;
    slot_L[3 * (size_t)slot + 2] = L.z;
}

// Closest hits of every ray of the input queue (vertex k) into p.hits.
// Persistent warps keep their lanes busy: whenever at least kRefillMin lanes
// have finished, the idle lanes take the next ray indices from a range the
// warp claimed with one atomic (kFetchRange indices at a time), so a warp no
// longer waits for its slowest ray before starting new ones.  Trees in the
// decoded form (small enough for L2; the node step is issue-bound) refill
// in larger groups than large packed trees (the node step waits on memory).
#ifndef PT_TRACE_REFILL_MIN
#define PT_TRACE_REFILL_MIN 12
#endif
#ifndef PT_TRACE_REFILL_MIN_WIDE
#define PT_TRACE_REFILL_MIN_WIDE 20
#endif
#ifndef PT_TRACE_STEPS
#define PT_TRACE_STEPS 3
#endif
#ifndef PT_TRACE_RANGE_DIV
#define PT_TRACE_RANGE_DIV 4096
#endif
constexpr int kRefillMinPacked = PT_TRACE_REFILL_MIN;
constexpr int kRefillMinWide = PT_TRACE_REFILL_MIN_WIDE;
constexpr int kStepsPerCheck = PT_TRACE_STEPS;

#ifndef PT_TRACE_MIN_BLOCKS
#define PT_TRACE_MIN_BLOCKS 4
#endif
template <int kForm>
__global__ void __launch_bounds__(256, PT_TRACE_MIN_BLOCKS) k_trace(const BounceParams p)
{
    const uint32_t count = (p.k == 1) ? p.n_chunk : min(*p.count_in, p.cap);
    const uint32_t lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    // indices claimed per atomic: 128 when every warp has many rays, down to 32 for short queues so that
    // the work still spreads over all warps
    const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
    const uint32_t per_warp = count / n_warps;
    const uint32_t kFetchRange = per_warp >= PT_TRACE_RANGE_DIV ? 128u : (per_warp >= PT_TRACE_RANGE_DIV / 4 ? 64u : 32u);
    Work work;
    Trav t;
    uint32_t stack_ref[kStackSize];
    float stack_t[kStackSize];
    bool live = false, exhausted = false;
    uint32_t ri = 0;
    uint32_t rnext = 0, rend = 0;   // the warp's claimed index range (warp-uniform)
    while (true) {
        const unsigned idle = __ballot_sync(0xFFFFFFFFu, !live);
        constexpr int kRefillMin = kForm == kNodesWide ? kRefillMinWide : kRefillMinPacked;
        if (idle && !exhausted && (__popc(idle) >= kRefillMin || idle == 0xFFFFFFFFu)) {
            const uint32_t n = __popc(idle), rank = __popc(idle & lanes_below);
            const uint32_t avail = rend - rnext;
            uint32_t idx = rnext + rank;
            if (avail < n) {
                uint32_t nb = 0;
                if (lane == 0) nb = atomicAdd(p.fetch, kFetchRange);
                nb = __shfl_sync(0xFFFFFFFFu, nb, 0);
                if (rank >= avail) idx = nb + (rank - avail);
                rnext = nb + (n - avail);
                rend = nb + kFetchRange;
            } else {
                rnext += n;
            }
            exhausted = rnext >= count;   // claims only grow: nothing below count is left for this warp
            if (!live && idx < count) {
                float3 o, d;
                if (p.k == 1) {
                    ri = tile_slot(p, idx);   // camera rays: hits are stored per slot
                    uint32_t pix, smp;
                    slot_to_pixel(p, ri, pix, smp);
                    const uint4 w = philox4x32_10(make_uint4(pix, smp, 0u, 0u), p.seed, 0u);
                    o = f3(p.sc.eye[0], p.sc.eye[1], p.sc.eye[2]);
                    d = camera_dir(p.sc, p.W, p.H, pix, u01(w.x), u01(w.y));
                } else {
                    const float4 o4 = p.qin.o[idx], d4 = p.qin.d[idx];
                    o = f3(o4.x, o4.y, o4.z);
                    d = f3(d4.x, d4.y, d4.z);
                    ri = idx;
                }
                if (trav_init(p.sc, o, d, t, work)) p.hits[ri] = make_int2(__float_as_int(t.h.t), t.h.prim);
                else live = true;
            }
        }
        if (!__any_sync(0xFFFFFFFFu, live)) {
            if (exhausted) break;
            continue;
        }
#pragma unroll 1
        for (int st = 0; st < kStepsPerCheck; ++st) {
            if (live && trav_step<kForm>(p.sc, t, stack_ref, stack_t, p.err, work)) {
                p.hits[ri] = make_int2(__float_as_int(t.h.t), t.h.prim);
                live = false;
            }
        }
    }
    // traversal work, one atomic per warp
    for (int off = 16; off > 0; off >>= 1) {
        work.nodes += __shfl_down_sync(0xFFFFFFFFu, work.nodes, off);
        work.sph += __shfl_down_sync(0xFFFFFFFFu, work.sph, off);
        work.quad += __shfl_down_sync(0xFFFFFFFFu, work.quad, off);
        work.tri += __shfl_down_sync(0xFFFFFFFFu, work.tri, off);
    }
    if (lane == 0 && p.work && work.nodes + work.sph + work.quad + work.tri) {
        atomicAdd(&p.work[0], (unsigned long long)work.nodes);
        atomicAdd(&p.work[1], (unsigned long long)work.sph);
        atomicAdd(&p.work[2], (unsigned long long)work.quad);
        atomicAdd(&p.work[3], (unsigned long long)work.tri);
    }
}

// Camera rays (vertex 1) of a whole image traced as warp packets.  The 32
// rays a warp takes together are an 8 x 4 pixel tile of one sample
// (tile_slot), close enough in origin and direction to walk the upper tree
// together: the warp visits every node that any of its rays enters, fetching
// each once for all lanes, and each lane tests its own ray against the node's
// two child boxes.  The near child is the one most of the lanes that enter a
// child reach first; the other is stacked with each lane's own entry
// distance, and a stacked node is visited while any lane still needs it.
// Once fewer than PT_PACKET_MIN_LANES lanes enter the current node (the rays
// part near the leaves of a large tree), each lane finishes on its own from
// that state with the per-ray step.  The closest hit does not depend on the
// order of the visits (boxes are entered at equal distance, equal distances
// go to the lower primitive ID), and a lane only finds hits inside every box
// above them, so the hits equal those of the per-ray traversal bit for bit.
// Work counts only the nodes a lane's own ray entered.
#ifndef PT_TRACE_CAMERA_PACKETS
#define PT_TRACE_CAMERA_PACKETS 1
#endif
// below this many lanes entering the current node, each lane goes on alone
#ifndef PT_PACKET_MIN_LANES
#define PT_PACKET_MIN_LANES 24
#endif
constexpr uint32_t kCameraClaim = 128;   // camera rays claimed per warp atomic (four packets)

template <int kForm>
__global__ void __launch_bounds__(256, PT_TRACE_MIN_BLOCKS) k_trace_camera(const BounceParams p)
{
    const uint32_t count = p.n_chunk;
    const uint32_t lane = threadIdx.x & 31;
    Work work;
    uint32_t stack_ref[kStackSize];
    float stack_t[kStackSize];
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(p.fetch, kCameraClaim);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= count) break;
        for (uint32_t pk = base; pk < base + kCameraClaim && pk < count; pk += 32) {
            const uint32_t idx = pk + lane;
            const bool valid = idx < count;
            uint32_t ri = 0;
            float3 o = f3(p.sc.eye[0], p.sc.eye[1], p.sc.eye[2]), d = f3(0.f, 0.f, 1.f);
            if (valid) {
                ri = tile_slot(p, idx);   // hits are stored per slot
                uint32_t pix, smp;
                slot_to_pixel(p, ri, pix, smp);
                const uint4 w = philox4x32_10(make_uint4(pix, smp, 0u, 0u), p.seed, 0u);
                d = camera_dir(p.sc, p.W, p.H, pix, u01(w.x), u01(w.y));
            }
            Trav t;
            bool done = trav_init(p.sc, o, d, t, work);   // the same for every lane: empty tree or one leaf
            if (!valid) t.h.t = -1.f;                      // a lane without a ray enters no box
            uint32_t cur = t.cur;
            int sp = 0;
            uint32_t iters = 0;
            bool need = valid;   // this lane's ray entered `cur`
            bool split = false;  // too few lanes left on one path: each lane goes on alone
            while (!done) {
                if (__popc(__ballot_sync(0xFFFFFFFFu, need)) < PT_PACKET_MIN_LANES) { split = true; break; }
                if (++iters > kIterCap) { if (lane == 0) atomicOr(p.err, PT_ERR_ITER_CAP); break; }
                if (cur >= p.sc.n_nodes) { if (lane == 0) atomicOr(p.err, PT_ERR_BAD_NODE); break; }
                uint32_t cl, cr;
                float tl, trr;
                node_children<kForm>(p.sc, cur, t.o, t.inv, t.h.t, cl, cr, tl, trr);
                if (need) ++work.nodes;
                if ((cl & kLeafBit) && tl < INFINITY) {
                    isect_prim(p.sc, cl & ~kLeafBit, t.o, t.d, t.tr, t.h.t, t.h.prim, work);
                    tl = INFINITY;
                }
                if ((cr & kLeafBit) && trr < INFINITY) {
                    isect_prim(p.sc, cr & ~kLeafBit, t.o, t.d, t.tr, t.h.t, t.h.prim, work);
                    trr = INFINITY;
                }
                const bool hl = tl < INFINITY && tl <= t.h.t, hr = trr < INFINITY && trr <= t.h.t;
                const unsigned bl = __ballot_sync(0xFFFFFFFFu, hl), br = __ballot_sync(0xFFFFFFFFu, hr);
                if (bl && br) {
                    const unsigned pref = __ballot_sync(0xFFFFFFFFu, hl && (!hr || tl <= trr));
                    const bool left_first = 2 * __popc(pref) >= __popc(bl | br);
                    if (sp >= kStackSize) { if (lane == 0) atomicOr(p.err, PT_ERR_STACK_OVERFLOW); break; }
                    stack_ref[sp] = left_first ? cr : cl;
                    stack_t[sp] = left_first ? (hr ? trr : INFINITY) : (hl ? tl : INFINITY);
                    ++sp;
                    cur = left_first ? cl : cr;
                    need = left_first ? hl : hr;
                } else if (bl) {
                    cur = cl;
                    need = hl;
                } else if (br) {
                    cur = cr;
                    need = hr;
                } else {
                    done = true;
                    while (sp > 0) {
                        --sp;
                        const bool want = stack_t[sp] <= t.h.t;
                        if (__any_sync(0xFFFFFFFFu, want)) {
                            cur = stack_ref[sp];
                            need = want;
                            done = false;
                            break;
                        }
                    }
                }
            }
            if (split && valid) {
                // the rest of this lane's traversal on its own: from `cur` if its ray entered it, else from
                // the nearest stacked node it still needs (the stack holds its own entry distances)
                bool alive = need;
                while (!alive && sp > 0) {
                    --sp;
                    if (stack_t[sp] <= t.h.t) { cur = stack_ref[sp]; alive = true; }
                }
                if (alive) {
                    t.cur = cur;
                    t.sp = sp;
                    t.iters = iters;
                    while (!trav_step<kForm>(p.sc, t, stack_ref, stack_t, p.err, work)) {
                    }
                }
            }
            if (valid) p.hits[ri] = make_int2(__float_as_int(t.h.t), t.h.prim);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        work.nodes += __shfl_down_sync(0xFFFFFFFFu, work.nodes, off);
        work.sph += __shfl_down_sync(0xFFFFFFFFu, work.sph, off);
        work.quad += __shfl_down_sync(0xFFFFFFFFu, work.quad, off);
        work.tri += __shfl_down_sync(0xFFFFFFFFu, work.tri, off);
    }
    if (lane == 0 && p.work && work.nodes + work.sph + work.quad + work.tri) {
        atomicAdd(&p.work[0], (unsigned long long)work.nodes);
        atomicAdd(&p.work[1], (unsigned long long)work.sph);
        atomicAdd(&p.work[2], (unsigned long long)work.quad);
        atomicAdd(&p.work[3], (unsigned long long)work.tri);
    }
}

// Lanes that arrive here together take consecutive slots of a queue with one
// atomic; returns this lane's slot.
__device__ __forceinline__ uint32_t active_append(uint32_t* counter)
{
    const unsigned m = __activemask();
    const uint32_t lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if ((int)lane == leader) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(m, base, leader);
    return base + __popc(m & ((1u << lane) - 1u));
}

__device__ __forceinline__ void push_escape(const BounceParams& p, uint32_t ei, const PathState& s, float eu, float ev)
{
    if (ei < p.cap) {
        p.esc.uv[ei] = make_float2(eu, ev);
        p.esc.tp[ei] = make_float4(s.tp.x, s.tp.y, s.tp.z, __uint_as_float(s.slot));
    } else {
        atomicOr(p.err, PT_ERR_QUEUE_OVERFLOW);
    }
}

struct VertexOut {
    bool survive, escape_nif;
    float eu, ev;
};

// Shading of path vertex k given its closest hit h (Section 3.1): the hit
// record, the record row and the cache query at their vertices, emission, the
// environment or the NIF escape (Section 3.3), BSDF sampling of the next
// direction with the Philox words of (pixel, sample, k) and Russian roulette.
// A path that ends here has its radiance stored, unless a later kernel stores
// it (cache query; NIF escape without emitters); a surviving path continues
// from s.o along s.d.  Shared by the wavefront step and the path-per-thread
// kernel, which therefore compute the same paths.
__device__ __forceinline__ VertexOut shade_vertex(const BounceParams& p, int k, PathState& s, uint32_t pix,
                                                  uint32_t smp, Hit h)
{
    VertexOut v{false, false, 0.f, 0.f};
    if (p.hit_ids) p.hit_ids[(p.chunk_first + s.slot) * (uint64_t)p.max_depth + (k - 1)] = h.prim;
    if (h.prim < 0) {
        if (p.sc.env_is_nif) {
            // Section 3.3: direction -> equirect (u, v), shaded later by the NIF
            v.eu = 0.5f + atan2f(s.d.x, -s.d.z) * (0.5f / kPi);
            v.ev = acosf(fminf(1.f, fmaxf(-1.f, s.d.y))) * (1.f / kPi);
            v.escape_nif = true;
            // without emitters the NIF kernel stores the path's whole radiance itself
            if (p.sc.has_emission) store_L(p.slot_L, s.slot, s.L, p.err);
        } else {
            s.L = s.L + s.tp * f3(p.sc.env[0], p.sc.env[1], p.sc.env[2]);
            store_L(p.slot_L, s.slot, s.L, p.err);
        }
        return v;
    }
    const float3 hp = s.o + s.d * h.t;
    const int32_t mat = __ldg(&p.sc.prim_mat[h.prim]);
    bool cache_q = false;
    if (p.rec_vertex == k || p.cache_vertex == k) {
        // state at this vertex: position, direction to the previous vertex, normal facing it,
        // throughput reaching it and radiance gathered before it
        const float3 ng0 = geometric_normal(p.sc, (uint32_t)h.prim, hp);
        const float3 nf = dot3(ng0, s.d) < 0.f ? ng0 : ng0 * -1.f;
        float* row = nullptr;
        float last = 1.f;   // record: valid
        if (p.rec_vertex == k) row = p.rec + 16 * (p.chunk_first + s.slot);
        if (p.cache_vertex == k) {
            // the path ends here; its query row goes to the cache queue
            cache_q = true;
            const uint32_t ci = active_append(p.cache_count);
            if (ci < p.cap) row = p.cache_rows + 16 * (size_t)ci;
            else atomicOr(p.err, PT_ERR_QUEUE_OVERFLOW);
            last = __uint_as_float(s.slot);
        }
        if (row) {
            float4* r = reinterpret_cast<float4*>(row);
            r[0] = make_float4(hp.x, hp.y, hp.z, -s.d.x);
            r[1] = make_float4(-s.d.y, -s.d.z, nf.x, nf.y);
            r[2] = make_float4(nf.z, s.tp.x, s.tp.y, s.tp.z);
            r[3] = make_float4(s.L.x, s.L.y, s.L.z, last);
        }
    }
    if (p.sc.has_emission && !cache_q) {
        const float4 m1 = __ldg(&p.sc.mat[2 * mat + 1]);
        s.L = s.L + s.tp * f3(m1.y, m1.z, m1.w);
    }
    bool alive = k < p.max_depth && !cache_q;
    if (alive) {
        const uint4 w = philox4x32_10(make_uint4(pix, smp, (uint32_t)k, 0u), p.seed, 0u);
        const float3 ng = geometric_normal(p.sc, (uint32_t)h.prim, hp);
        float3 wi, wt;
        alive = sample_bsdf(p.sc, mat, s.d, ng, u01(w.x), u01(w.y), u01(w.z), wi, wt);
        if (alive) {
            s.tp = s.tp * wt;
            if (p.rr && k >= p.rr_start) {
                const float q = fminf(1.f, fmaxf(s.tp.x, fmaxf(s.tp.y, s.tp.z)));
                if (u01(w.w) < q) s.tp = s.tp * (1.f / q);
                else alive = false;
            }
        }
        if (alive) {
            const float eps = 1e-4f * fmaxf(1.f, fmaxf(fabsf(hp.x), fmaxf(fabsf(hp.y), fabsf(hp.z))));
            const float3 off = dot3(wi, ng) > 0.f ? ng : ng * -1.f;
            s.o = hp + off * eps;
            s.d = wi;
        }
    }
    if (alive) v.survive = true;
    else if (!cache_q) store_L(p.slot_L, s.slot, s.L, p.err);   // a cache query writes it later
    return v;
}

__device__ __forceinline__ void camera_ray(const BounceParams& p, uint32_t pix, uint32_t smp, PathState& s)
{
    const uint4 w = philox4x32_10(make_uint4(pix, smp, 0u, 0u), p.seed, 0u);
    s.o = f3(p.sc.eye[0], p.sc.eye[1], p.sc.eye[2]);
    s.d = camera_dir(p.sc, p.W, p.H, pix, u01(w.x), u01(w.y));
    s.tp = f3(1.f, 1.f, 1.f);
    s.L = f3(0.f, 0.f, 0.f);
}

__device__ __forceinline__ void add_work(const BounceParams& p, Work work)
{
    for (int off = 16; off > 0; off >>= 1) {
        work.nodes += __shfl_down_sync(0xFFFFFFFFu, work.nodes, off);
        work.sph += __shfl_down_sync(0xFFFFFFFFu, work.sph, off);
        work.quad += __shfl_down_sync(0xFFFFFFFFu, work.quad, off);
        work.tri += __shfl_down_sync(0xFFFFFFFFu, work.tri, off);
    }
    if ((threadIdx.x & 31) == 0 && p.work && work.nodes + work.sph + work.quad + work.tri) {
        atomicAdd(&p.work[0], (unsigned long long)work.nodes);
        atomicAdd(&p.work[1], (unsigned long long)work.sph);
        atomicAdd(&p.work[2], (unsigned long long)work.quad);
        atomicAdd(&p.work[3], (unsigned long long)work.tri);
    }
}

// One wavefront step at vertex k for every ray of the input queue: shading of
// the hits k_trace found, next-bounce sampling and compaction.
__global__ void __launch_bounds__(256, 4) k_bounce(const BounceParams p)
{
    const uint32_t count = (p.k == 1) ? p.n_chunk : min(*p.count_in, p.cap);  // counters may pass cap on overflow
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    uint32_t traced = 0;
    for (uint32_t base = warp * 32; base < count; base += n_warps * 32) {
        const uint32_t i = base + lane;
        const bool active = i < count;
        PathState s;
        uint32_t pix = 0, smp = 0;
        if (active) {
            if (p.k == 1) {
                // camera paths in the traversal's tile order, so that the survivors' queue (the rays of
                // vertex 2) keeps neighbouring pixels together
                s.slot = tile_slot(p, i);
                slot_to_pixel(p, s.slot, pix, smp);
                camera_ray(p, pix, smp, s);
            } else {
                const float4 o = p.qin.o[i], d = p.qin.d[i], tp = p.qin.tp[i];
                s.o = f3(o.x, o.y, o.z);
                s.slot = __float_as_uint(o.w);
                s.d = f3(d.x, d.y, d.z);
                s.tp = f3(tp.x, tp.y, tp.z);
                if (p.sc.has_emission) {
                    const float4 L = p.qin.L[i];
                    s.L = f3(L.x, L.y, L.z);
                } else {
                    s.L = f3(0.f, 0.f, 0.f);
                }
                slot_to_pixel(p, s.slot, pix, smp);
            }
        }
        VertexOut v{false, false, 0.f, 0.f};
        if (active) {
            ++traced;
            const int2 hv = p.hits[p.k == 1 ? s.slot : i];   // camera-ray hits are stored per slot
            v = shade_vertex(p, p.k, s, pix, smp, Hit{__int_as_float(hv.x), hv.y});
        }
        // compaction: survivors into the next queue, escapes into the NIF queue
        const uint32_t qi = warp_append(v.survive, p.count_out);
        if (v.survive) {
            if (qi < p.cap) {
                p.qout.o[qi] = make_float4(s.o.x, s.o.y, s.o.z, __uint_as_float(s.slot));
                p.qout.d[qi] = make_float4(s.d.x, s.d.y, s.d.z, 0.f);
                p.qout.tp[qi] = make_float4(s.tp.x, s.tp.y, s.tp.z, 0.f);
                if (p.sc.has_emission) p.qout.L[qi] = make_float4(s.L.x, s.L.y, s.L.z, 0.f);
            } else {
                atomicOr(p.err, PT_ERR_QUEUE_OVERFLOW);
            }
        }
        const uint32_t ei = warp_append(v.escape_nif, p.esc_count);
        if (v.escape_nif) push_escape(p, ei, s, v.eu, v.ev);
    }
    // k_trace of this vertex has finished: its claim counter starts the next vertex at zero
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.fetch = 0;
    // per-vertex ray count, one atomic per warp
    for (int off = 16; off > 0; off >>= 1) traced += __shfl_down_sync(0xFFFFFFFFu, traced, off);
    if (lane == 0 && traced) atomicAdd(&p.stats[p.k - 1], (unsigned long long)traced);
}

// Path-per-thread schedule for wavefronts smaller than one resident wave of
// threads: each thread follows its paths through every vertex in one launch
// (traversal, then shade_vertex), so a call pays for its slowest path once
// instead of for the slowest ray of every vertex, with no queues between
// vertices.  Same Philox counters, records, NIF escape queue and cache queue
// as the wavefront schedule; only the order of the queues differs, and every
// consumer of a queue entry addresses the path by its slot.
// Small blocks spread a small chunk over every SM (a latency-bound launch
// runs fastest with the fewest warps per SM).
constexpr int kPathsBlock = 64;
template <int kForm>
__global__ void __launch_bounds__(kPathsBlock, 12) k_paths(const BounceParams p)
{
    const uint32_t lane = threadIdx.x & 31;
    const int k_end = p.cache_vertex ? min(p.max_depth, p.cache_vertex) : p.max_depth;
    Work work;
    uint32_t stack_ref[kStackSize];
    float stack_t[kStackSize];
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < p.n_chunk; j += gridDim.x * blockDim.x) {
        PathState s;
        uint32_t pix, smp;
        s.slot = tile_slot(p, j);
        slot_to_pixel(p, s.slot, pix, smp);
        camera_ray(p, pix, smp, s);
        for (int k = 1; k <= k_end; ++k) {
            {   // rays traced at vertex k: one atomic per group of lanes at the same vertex
                const unsigned m = __match_any_sync(__activemask(), k);
                if ((int)lane == __ffs(m) - 1) atomicAdd(&p.stats[k - 1], (unsigned long long)__popc(m));
            }
            Trav t;
            if (!trav_init(p.sc, s.o, s.d, t, work)) {
                while (!trav_step<kForm>(p.sc, t, stack_ref, stack_t, p.err, work)) {
                }
            }
            const VertexOut v = shade_vertex(p, k, s, pix, smp, t.h);
            if (v.escape_nif) push_escape(p, active_append(p.esc_count), s, v.eu, v.ev);
            if (!v.survive) break;
        }
    }
    add_work(p, work);
}

// image[i] (+)= sum over the chunk's samples in sample order; scaled at the end
__global__ void k_reduce(const float* __restrict__ slot_L, float* __restrict__ pix, uint32_t n_pix, uint32_t s_count,
                         int first, float scale)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pix) return;
    float r = first ? 0.f : pix[3 * (size_t)i], g = first ? 0.f : pix[3 * (size_t)i + 1],
          b = first ? 0.f : pix[3 * (size_t)i + 2];
    for (uint32_t s = 0; s < s_count; ++s) {
        const size_t o = 3 * ((size_t)s * n_pix + i);
        r += slot_L[o];
        g += slot_L[o + 1];
        b += slot_L[o + 2];
    }
    pix[3 * (size_t)i] = r * scale;
    pix[3 * (size_t)i + 1] = g * scale;
    pix[3 * (size_t)i + 2] = b * scale;
}

__global__ void k_fill_i32(int32_t* p, int64_t n, int32_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_philox(uint32_t seed, uint32_t tag, int64_t n, const uint4* __restrict__ ctr, uint4* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(ctr[i], seed, tag);
}

__global__ void k_primary(const DevScene sc, int W, int H, uint32_t seed, uint32_t first_sample, int64_t first, int64_t n,
                          float* org, float* dir)
{
    const int64_t WH = (int64_t)W * H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = first + i;
        const uint32_t pix = (uint32_t)(g % WH), smp = (uint32_t)(g / WH) + first_sample;
        const uint4 w = philox4x32_10(make_uint4(pix, smp, 0u, 0u), seed, 0u);
        const float3 d = camera_dir(sc, W, H, pix, u01(w.x), u01(w.y));
        org[3 * i] = sc.eye[0]; org[3 * i + 1] = sc.eye[1]; org[3 * i + 2] = sc.eye[2];
        dir[3 * i] = d.x; dir[3 * i + 1] = d.y; dir[3 * i + 2] = d.z;
    }
}

__global__ void __launch_bounds__(256) k_trace_rays(const DevScene sc, int64_t n, const float* __restrict__ org,
                                                     const float* __restrict__ dir, float* t, int32_t* prim,
                                                     uint32_t* err)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 o = f3(org[3 * i], org[3 * i + 1], org[3 * i + 2]);
        const float3 d = f3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
        Work w;
        const Hit h = trace_closest(sc, o, d, err, w);
        t[i] = h.t;
        prim[i] = h.prim;
    }
}

int grid_for(int64_t n, int block, int sm_count, int per_sm)
{
    int64_t g = (n + block - 1) / block;
    const int64_t cap = (int64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_trace(const BounceParams& p, int sm_count, cudaStream_t s)
{
    // traversal: persistent, 4 resident blocks of 256 threads per SM; camera rays as warp packets
    const int grid = sm_count * PT_TRACE_MIN_BLOCKS;
    if (PT_TRACE_CAMERA_PACKETS && p.k == 1 && p.tiled) {
        if (p.sc.qnodes) k_trace_camera<kNodesQuant><<<grid, 256, 0, s>>>(p);
        else if (p.sc.wnodes) k_trace_camera<kNodesWide><<<grid, 256, 0, s>>>(p);
        else k_trace_camera<kNodesPacked><<<grid, 256, 0, s>>>(p);
    } else if (p.sc.qnodes) {
        k_trace<kNodesQuant><<<grid, 256, 0, s>>>(p);
    } else if (p.sc.wnodes) {
        k_trace<kNodesWide><<<grid, 256, 0, s>>>(p);
    } else {
        k_trace<kNodesPacked><<<grid, 256, 0, s>>>(p);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_shade(const BounceParams& p, int sm_count, cudaStream_t s)
{
    // shading: grid-stride over the queue
    k_bounce<<<sm_count * 8, 256, 0, s>>>(p); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_bounce(const BounceParams& p, int sm_count, cudaStream_t s)
{
    const cudaError_t e = launch_trace(p, sm_count, s);
    return e != cudaSuccess ? e : launch_shade(p, sm_count, s);
}

int paths_resident_threads(int form, int sm_count)
{
    int per_sm = 0;
    const cudaError_t e =
        form == kNodesQuant  ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_paths<kNodesQuant>, kPathsBlock, 0)
        : form == kNodesWide ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_paths<kNodesWide>, kPathsBlock, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_paths<kNodesPacked>, kPathsBlock, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sm_count * kPathsBlock;
}

cudaError_t launch_paths(const BounceParams& p, int resident_threads, cudaStream_t s)
{
    // one thread per path while they fit in one resident wave, grid-stride beyond
    const int cap = resident_threads;
    int64_t blocks = ((int64_t)p.n_chunk + kPathsBlock - 1) / kPathsBlock;
    if (cap > 0 && blocks > cap / kPathsBlock) blocks = cap / kPathsBlock;
    if (blocks < 1) blocks = 1;
    if (p.sc.qnodes) k_paths<kNodesQuant><<<(int)blocks, kPathsBlock, 0, s>>>(p);
    else if (p.sc.wnodes) k_paths<kNodesWide><<<(int)blocks, kPathsBlock, 0, s>>>(p);
    else k_paths<kNodesPacked><<<(int)blocks, kPathsBlock, 0, s>>>(p);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_reduce(const float* slot_L, float* pix, uint32_t n_pix, uint32_t s_count, int first, float scale,
                          cudaStream_t s)
{
    k_reduce<<<(n_pix + 255) / 256, 256, 0, s>>>(slot_L, pix, n_pix, s_count, first, scale); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fill_i32(int32_t* p, int64_t n, int32_t v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_fill_i32<<<grid_for(n, 256, 152, 16), 256, 0, s>>>(p, n, v); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_philox(uint32_t seed, uint32_t tag, int64_t n, const uint32_t* ctr, uint32_t* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_philox<<<grid_for(n, 256, 152, 16), 256, 0, s>>>(seed, tag, n, reinterpret_cast<const uint4*>(ctr),
                                                      reinterpret_cast<uint4*>(out)); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_primary(const DevScene& sc, int W, int H, uint32_t seed, uint32_t first_sample, int64_t first,
                           int64_t n, float* org, float* dir, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_primary<<<grid_for(n, 256, 152, 16), 256, 0, s>>>(sc, W, H, seed, first_sample, first, n, org, dir); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_trace_rays(const DevScene& sc, int64_t n, const float* org, const float* dir, float* t,
                              int32_t* prim, uint32_t* err, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_trace_rays<<<grid_for(n, 256, 152, 16), 256, 0, s>>>(sc, n, org, dir, t, prim, err); count_launch();
    return cudaGetLastError();
}

}  // namespace ptk

namespace ptk {
namespace {
__global__ void k_set_u32(uint32_t* dst, uint32_t value) { *dst = value; }
}  // namespace
cudaError_t launch_set_u32(uint32_t* dst, uint32_t value, cudaStream_t s)
{
    k_set_u32<<<1, 1, 0, s>>>(dst, value); count_launch();
    return cudaGetLastError();
}
}  // namespace ptk
