// Host BVH builder: binned SAH, one primitive per leaf, nodes packed for the
// device with the two children's boxes stored in the parent.  The upper
// levels hand their left subtrees to other threads (node lists merged with
// an index offset), so large meshes build on all host cores.
//
// Section 3.1.4 builds a BVH-2 on the host, compacts it into pointer-less
// nodes with the first child stored next in the array, and stores box
// extents in fp16 with a rounding that never shrinks the box.  The layout
// here keeps the fp32 origin + fp16 extent rounded up and a depth-first order
// within each subtree, but stores both child references and both child boxes
// in the parent, so one node fetch tests two boxes and subtrees can be built
// apart and placed anywhere.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include <cuda_fp16.h>

#include "pt_internal.h"

namespace ptk {

namespace {

struct Box {
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const float* l, const float* h)
    {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], l[a]);
            hi[a] = std::max(hi[a], h[a]);
        }
    }
    void grow(const Box& b) { grow(b.lo, b.hi); }
    double area() const
    {
        if (lo[0] > hi[0]) return 0.0;
        const double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

constexpr int kBins = 16;

// One primitive's centroid, bounds and input index.  The builder reorders
// these records themselves (not indices into the input), so every pass over
// a range reads memory in order.
struct Prim {
    float cen[3], lo[3], hi[3];
    uint32_t id;
};

struct Builder {
    std::vector<Prim>& prims;        // shared by the builders of one tree (each works on its own range)
    std::vector<PackedNode> nodes;
    int32_t max_depth = 0;
    int par_depth = 0;               // subtrees above this depth may be built on other threads
    std::string error;

    explicit Builder(std::vector<Prim>& pr) : prims(pr) {}

    Box range_box(int64_t b, int64_t e) const
    {
        Box bx;
        for (int64_t i = b; i < e; ++i) bx.grow(prims[i].lo, prims[i].hi);
        return bx;
    }

    // choose a split of idx[b, e) (count >= 2): binned SAH over the three axes
    // (one pass fills the bins of all axes); returns the midpoint and, when
    // the split came from the bins, the two children's exact boxes
    int64_t split(int64_t b, int64_t e, Box* bl, Box* br, bool* boxes_known)
    {
        const int64_t n = e - b;
        *boxes_known = false;
        if (n == 2) {
            // two leaves whatever the split; the binned sweep below would order them by centroid along the
            // first axis where the centroids differ (ties: as listed), which this reproduces without the bins
            for (int a = 0; a < 3; ++a) {
                const float c0 = prims[b].cen[a], c1 = prims[b + 1].cen[a];
                if (c0 != c1) {
                    if (c1 < c0) std::swap(prims[b], prims[b + 1]);
                    break;
                }
            }
            bl->grow(prims[b].lo, prims[b].hi);
            br->grow(prims[b + 1].lo, prims[b + 1].hi);
            *boxes_known = true;
            return b + 1;
        }
        float clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t i = b; i < e; ++i)
            for (int a = 0; a < 3; ++a) {
                const float c = prims[i].cen[a];
                clo[a] = std::min(clo[a], c);
                chi[a] = std::max(chi[a], c);
            }
        float scale[3];
        bool live[3];
        for (int a = 0; a < 3; ++a) {
            const float ext = chi[a] - clo[a];
            live[a] = ext > 0.f;
            scale[a] = live[a] ? kBins / ext : 0.f;
        }
        Box bb[3][kBins];
        int64_t cnt[3][kBins] = {};
        for (int64_t i = b; i < e; ++i) {
            const Prim& q = prims[i];
            for (int a = 0; a < 3; ++a) {
                if (!live[a]) continue;
                int k = (int)((q.cen[a] - clo[a]) * scale[a]);
                k = std::min(std::max(k, 0), kBins - 1);
                cnt[a][k]++;
                bb[a][k].grow(q.lo, q.hi);
            }
        }
        double best_cost = INFINITY;
        int best_axis = -1, best_bin = -1;
        for (int a = 0; a < 3; ++a) {
            if (!live[a]) continue;
            // an empty bin leaves the running box and count unchanged, so its area is carried over
            // instead of recomputed (same values, fewer operations on small ranges)
            double left_area[kBins];
            int64_t left_cnt[kBins];
            Box acc;
            int64_t c = 0;
            double area = 0.0;
            for (int k = 0; k < kBins - 1; ++k) {
                if (cnt[a][k]) {
                    acc.grow(bb[a][k]);
                    c += cnt[a][k];
                    area = acc.area();
                }
                left_area[k] = area;
                left_cnt[k] = c;
            }
            Box racc;
            int64_t rc = 0;
            double rarea = 0.0;
            for (int k = kBins - 1; k >= 1; --k) {
                if (cnt[a][k]) {
                    racc.grow(bb[a][k]);
                    rc += cnt[a][k];
                    rarea = racc.area();
                }
                const int64_t lc = left_cnt[k - 1];
                if (lc == 0 || rc == 0) continue;
                const double cost = left_area[k - 1] * (double)lc + rarea * (double)rc;
                if (cost < best_cost) { best_cost = cost; best_axis = a; best_bin = k; }
            }
        }
        int64_t mid;
        if (best_axis >= 0) {
            const int a = best_axis;
            auto it = std::partition(prims.begin() + b, prims.begin() + e, [&](const Prim& q) {
                int k = (int)((q.cen[a] - clo[a]) * scale[a]);
                k = std::min(std::max(k, 0), kBins - 1);
                return k < best_bin;
            });
            mid = it - prims.begin();
            if (mid > b && mid < e) {
                Box l, r;
                for (int k = 0; k < kBins; ++k) (k < best_bin ? l : r).grow(bb[a][k]);
                *bl = l;
                *br = r;
                *boxes_known = true;
                return mid;
            }
        }
        return b + n / 2;   // no usable split (all centroids coincide): halve the list
    }

    // build idx[b, e); returns the child reference
    uint32_t build(int64_t b, int64_t e, int depth)
    {
        max_depth = std::max(max_depth, depth);
        if (e - b == 1) return kLeafBit | prims[b].id;
        const uint32_t me = (uint32_t)nodes.size();
        nodes.emplace_back();
        Box bl, br;
        bool known = false;
        const int64_t mid = split(b, e, &bl, &br, &known);
        if (!known) {
            bl = range_box(b, mid);
            br = range_box(mid, e);
        }
        uint32_t cl, cr;
        if (depth < par_depth && e - b >= (int64_t)1 << 14) {
            // the left subtree on another thread into its own node list, appended after the right one
            Builder sub(prims);
            sub.par_depth = par_depth;
            sub.nodes.reserve((size_t)(mid - b));
            uint32_t sub_root = kEmptyRef;
            std::thread th([&] { sub_root = sub.build(b, mid, depth + 1); });
            cr = build(mid, e, depth + 1);
            th.join();
            const uint32_t off = (uint32_t)nodes.size();
            for (PackedNode nd : sub.nodes) {
                for (int c = 9; c <= 10; ++c)
                    if (!(nd.w[c] & kLeafBit)) nd.w[c] += off;
                nodes.push_back(nd);
            }
            cl = (sub_root & kLeafBit) ? sub_root : sub_root + off;
            max_depth = std::max(max_depth, sub.max_depth);
            if (!sub.error.empty()) error = sub.error;
        } else {
            cl = build(b, mid, depth + 1);
            cr = build(mid, e, depth + 1);
        }
        if (!error.empty()) return kEmptyRef;
        uint16_t el[3], er[3];
        for (int a = 0; a < 3; ++a) {
            if (!round_up_half_extent(bl.lo[a], bl.hi[a], &el[a]) || !round_up_half_extent(br.lo[a], br.hi[a], &er[a])) {
                error = "BVH box extent exceeds the fp16 range";
                return kEmptyRef;
            }
        }
        PackedNode& nd = nodes[me];
        std::memset(&nd, 0, sizeof(nd));
        std::memcpy(&nd.w[0], &bl.lo[0], 4);
        std::memcpy(&nd.w[1], &bl.lo[1], 4);
        std::memcpy(&nd.w[2], &bl.lo[2], 4);
        std::memcpy(&nd.w[3], &br.lo[0], 4);
        std::memcpy(&nd.w[4], &br.lo[1], 4);
        std::memcpy(&nd.w[5], &br.lo[2], 4);
        nd.w[6] = (uint32_t)el[0] | ((uint32_t)el[1] << 16);
        nd.w[7] = (uint32_t)el[2] | ((uint32_t)er[0] << 16);
        nd.w[8] = (uint32_t)er[1] | ((uint32_t)er[2] << 16);
        nd.w[9] = cl;
        nd.w[10] = cr;
        nd.w[11] = 0;
        return me;
    }
};

}  // namespace

// Smallest fp16 extent h >= 0 such that lo + float(h), evaluated in fp32,
// is >= hi: the decoded box then contains [lo, hi] ("round-to-nearest-not-
// lower").  Fails if no finite half qualifies.
bool round_up_half_extent(float lo, float hi, uint16_t* out_bits)
{
    const double ext = std::max(0.0, (double)hi - (double)lo);
    if (!(ext <= 65504.0)) return false;
    __half h = __float2half_rn((float)ext);
    uint16_t bits;
    std::memcpy(&bits, &h, 2);
    for (int guard = 0; guard < 64; ++guard) {
        __half hh;
        std::memcpy(&hh, &bits, 2);
        const float e = __half2float(hh);
        if (!std::isfinite(e)) return false;
        volatile float top = lo + e;  // fp32 addition as the device performs it
        if ((double)e >= ext && top >= hi) {
            *out_bits = bits;
            return true;
        }
        bits = (uint16_t)(bits + 1);  // next larger half (positive values)
    }
    return false;
}

void decode_packed_boxes(const PackedNode& n, float box[12])
{
    const uint16_t ext[6] = {(uint16_t)(n.w[6] & 0xFFFFu), (uint16_t)(n.w[6] >> 16), (uint16_t)(n.w[7] & 0xFFFFu),
                             (uint16_t)(n.w[7] >> 16), (uint16_t)(n.w[8] & 0xFFFFu), (uint16_t)(n.w[8] >> 16)};
    for (int c = 0; c < 2; ++c)
        for (int a = 0; a < 3; ++a) {
            float lo;
            std::memcpy(&lo, &n.w[3 * c + a], 4);
            __half h;
            std::memcpy(&h, &ext[3 * c + a], 2);
            volatile float top = lo + __half2float(h);   // fp32 addition as the device performs it
            box[6 * c + a] = lo;
            box[6 * c + 3 + a] = top;
        }
}

namespace {

// fp32 value of origin + q * 2^(E - 127), as the device computes it (exact product, one rounding)
float grid_value(float origin, int q, int E)
{
    volatile float step = std::ldexp(1.0f, E - 127);
    volatile float prod = (float)q * step;
    volatile float sum = origin + prod;
    return sum;
}

// 8-bit codes of [lo, hi] on the grid origin + q * 2^(E - 127): lo rounded down, hi rounded up, each
// checked in the device's fp32 arithmetic; false if hi needs a code above 255
bool quantize_interval(float origin, float lo, float hi, int E, int* qlo, int* qhi)
{
    const double step = std::ldexp(1.0, E - 127);
    int a = (int)std::floor(((double)lo - (double)origin) / step);
    int b = (int)std::ceil(((double)hi - (double)origin) / step);
    a = std::min(std::max(a, 0), 255);
    while (a > 0 && grid_value(origin, a, E) > lo) --a;
    while (a < 255 && grid_value(origin, a + 1, E) <= lo) ++a;   // the tightest code that still contains lo
    b = std::max(b, a);
    while (b <= 255 && grid_value(origin, b, E) < hi) ++b;
    if (b > 255) return false;
    while (b > a && grid_value(origin, b - 1, E) >= hi) --b;
    if (grid_value(origin, a, E) > lo) return false;
    *qlo = a;
    *qhi = b;
    return true;
}

}  // namespace

bool quantize_bvh(const std::vector<PackedNode>& in, std::vector<QuantNode>& out, std::string* error)
{
    out.assign(in.size(), QuantNode{});
    for (size_t i = 0; i < in.size(); ++i) {
        const PackedNode& n = in[i];
        float box[12];
        decode_packed_boxes(n, box);
        const uint32_t refs[2] = {n.w[9], n.w[10]};
        for (uint32_t r : refs)
            if ((r & ~kLeafBit) >= kQuantRefLimit) {
                if (error) *error = "BVH too large for 24-bit references of quantised nodes";
                return false;
            }
        float origin[3];
        int e_axis[3];
        for (int a = 0; a < 3; ++a) {
            origin[a] = std::min(box[a], box[6 + a]);
            const double span = std::max((double)box[3 + a], (double)box[9 + a]) - (double)origin[a];
            // smallest grid step 2^k with 255 steps covering the span (with a little slack for the rounding)
            int k = span > 0.0 ? (int)std::ceil(std::log2(span * (1.0 + 1e-6) / 255.0)) : -126;
            e_axis[a] = std::min(std::max(k + 127, 4), 254);
        }
        int e = std::max(e_axis[0], std::max(e_axis[1], e_axis[2]));
        int q[12];
        for (int guard = 0;; ++guard) {
            int d[3];
            bool ok = e <= 254;
            for (int a = 0; a < 3 && ok; ++a) {
                d[a] = std::min(3, e - e_axis[a]);
                for (int c = 0; c < 2 && ok; ++c)
                    ok = quantize_interval(origin[a], box[6 * c + a], box[6 * c + 3 + a], e - d[a], &q[6 * c + a],
                                           &q[6 * c + 3 + a]);
            }
            if (ok) {
                QuantNode& o = out[i];
                for (int a = 0; a < 3; ++a) std::memcpy(&o.w[a], &origin[a], 4);
                const uint32_t cl = refs[0] & ~kLeafBit, cr = refs[1] & ~kLeafBit;
                o.w[3] = (uint32_t)e | ((uint32_t)d[0] << 8) | ((uint32_t)d[1] << 10) | ((uint32_t)d[2] << 12) |
                         ((refs[0] & kLeafBit) ? 1u << 14 : 0u) | ((refs[1] & kLeafBit) ? 1u << 15 : 0u) |
                         ((cl & 0xFFFFu) << 16);
                o.w[4] = (cl >> 16) | (cr << 8);
                for (int j = 0; j < 3; ++j)
                    o.w[5 + j] = (uint32_t)q[4 * j] | ((uint32_t)q[4 * j + 1] << 8) | ((uint32_t)q[4 * j + 2] << 16) |
                                 ((uint32_t)q[4 * j + 3] << 24);
                break;
            }
            if (guard > 8 || e >= 254) {
                if (error) *error = "BVH box does not fit an 8-bit grid";
                return false;
            }
            ++e;   // a coarser grid
        }
    }
    return true;
}

bool build_bvh(const BuildInput& in, BuildOutput& out)
{
    out.nodes.clear();
    out.depth = 0;
    if (in.n_prims == 0) {
        out.root = kEmptyRef;
        return true;
    }
    std::vector<Prim> prims((size_t)in.n_prims);
    for (int64_t i = 0; i < in.n_prims; ++i) {
        Prim& q = prims[(size_t)i];
        for (int a = 0; a < 3; ++a) {
            q.cen[a] = in.cen[3 * i + a];
            q.lo[a] = in.lo[3 * i + a];
            q.hi[a] = in.hi[3 * i + a];
        }
        q.id = (uint32_t)i;
    }
    Builder bd(prims);
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    while ((1u << bd.par_depth) < 2 * hw && bd.par_depth < 8) ++bd.par_depth;   // about two subtrees per core
    bd.nodes.reserve((size_t)std::max<int64_t>(in.n_prims - 1, 1));
    out.root = bd.build(0, in.n_prims, 0);
    if (!bd.error.empty()) {
        out.error = bd.error;
        return false;
    }
    out.nodes = std::move(bd.nodes);
    out.depth = bd.max_depth;
    return true;
}

}  // namespace ptk
