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
// ranges of at least this many primitives run their split passes on several threads
constexpr int64_t kParallelPass = (int64_t)1 << 16;
// ranges of at least this many primitives (above par_depth) hand their left subtree to another thread
constexpr int64_t kParallelSubtree = (int64_t)1 << 14;

// One primitive's bounds and input index; its centroid is the box midpoint.
// The builder moves these records themselves (not indices into the input),
// so every pass over a range reads memory in order.
struct Prim {
    float lo[3], hi[3];
    uint32_t id;
    float cen(int a) const { return 0.5f * (lo[a] + hi[a]); }
};

struct CenBounds {
    float lo[3] = {INFINITY, INFINITY, INFINITY};
    float hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const Prim& q)
    {
        for (int a = 0; a < 3; ++a) {
            const float c = q.cen(a);
            lo[a] = std::min(lo[a], c);
            hi[a] = std::max(hi[a], c);
        }
    }
    void grow(const CenBounds& o)   // o may be empty (lo = +inf, hi = -inf)
    {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], o.lo[a]);
            hi[a] = std::max(hi[a], o.hi[a]);
        }
    }
};

// Bins of one split, filled lazily: a bin's box and count are valid only
// where its bit in `used` is set, so a split of a few primitives does not
// initialise 48 boxes.
struct Bins {
    Box bb[3][kBins];
    int64_t cnt[3][kBins];
    uint32_t used[3] = {0, 0, 0};
    void add(int a, int k, const Prim& q)
    {
        const uint32_t bit = 1u << k;
        if (used[a] & bit) {
            cnt[a][k]++;
            bb[a][k].grow(q.lo, q.hi);
        } else {
            used[a] |= bit;
            cnt[a][k] = 1;
            bb[a][k] = Box();
            bb[a][k].grow(q.lo, q.hi);
        }
    }
    void merge(const Bins& o)   // exact: integer counts, min and max
    {
        for (int a = 0; a < 3; ++a)
            for (uint32_t m = o.used[a]; m; m &= m - 1) {
                const int k = __builtin_ctz(m);
                if (used[a] & (1u << k)) {
                    cnt[a][k] += o.cnt[a][k];
                    bb[a][k].grow(o.bb[a][k]);
                } else {
                    used[a] |= 1u << k;
                    cnt[a][k] = o.cnt[a][k];
                    bb[a][k] = o.bb[a][k];
                }
            }
    }
};

// What the builders of one tree share.  Each works on its own range [b, e)
// of the two record buffers and writes its own nodes: a subtree over m
// primitives holds exactly m - 1 nodes, so where each subtree's nodes go
// follows from the split counts alone.
struct Tree {
    std::vector<Prim, NoInitAlloc<Prim>> buf[2];
    NodeVec nodes;
    int par_depth = 0;       // subtrees above this depth may be built on other threads
    unsigned threads = 1;
};

struct Builder {
    Tree& tr;
    int32_t max_depth = 0;
    std::string error;

    explicit Builder(Tree& t) : tr(t) {}

    // threads for the passes over a range: the 2^depth ranges of one level above par_depth are split at
    // the same time, so each takes its share
    int pass_threads(int64_t n, int depth) const
    {
        if (n < kParallelPass || depth >= 16) return 1;
        return std::max(1, (int)(tr.threads >> depth));
    }

    static Box range_box(const Prim* P, int64_t b, int64_t e)
    {
        Box bx;
        for (int64_t i = b; i < e; ++i) bx.grow(P[i].lo, P[i].hi);
        return bx;
    }

    static CenBounds range_centroids(const Prim* P, int64_t b, int64_t e)
    {
        CenBounds c;
        for (int64_t i = b; i < e; ++i) c.grow(P[i]);
        return c;
    }

    // choose a split of [b, e) (count >= 2), whose records are in *src: binned SAH over the three axes
    // (one pass fills the bins of all axes; cb holds the range's centroid bounds), then a partition that
    // also takes the children's centroid bounds.  Ranges of kParallelPass records or more are partitioned
    // stably into the other buffer (on several threads where the level has them to spare), which then
    // holds the children's records (*src is swapped with *dst); smaller ranges in place.  Returns the
    // midpoint and, when the split came from the bins, the two children's exact boxes and centroid bounds.
    int64_t split(int64_t b, int64_t e, int depth, const CenBounds& cb, Prim** src, Prim** dst, Box* bl,
                  Box* br, CenBounds* cl, CenBounds* cr, bool* known)
    {
        Prim* P = *src;
        const int64_t n = e - b;
        *known = false;
        if (n == 2) {
            // two leaves whatever the split; the binned sweep below would order them by centroid along the
            // first axis where the centroids differ (ties: as listed), which this reproduces without the bins
            for (int a = 0; a < 3; ++a) {
                const float c0 = P[b].cen(a), c1 = P[b + 1].cen(a);
                if (c0 != c1) {
                    if (c1 < c0) std::swap(P[b], P[b + 1]);
                    break;
                }
            }
            bl->grow(P[b].lo, P[b].hi);
            br->grow(P[b + 1].lo, P[b + 1].hi);
            cl->grow(P[b]);
            cr->grow(P[b + 1]);
            *known = true;
            return b + 1;
        }
        const int T = pass_threads(n, depth);
        float scale[3];
        bool live[3];
        for (int a = 0; a < 3; ++a) {
            const float ext = cb.hi[a] - cb.lo[a];
            live[a] = ext > 0.f;
            scale[a] = live[a] ? kBins / ext : 0.f;
        }
        // bin index along axis a (kept in locals: stores to the bins could otherwise alias cb and scale)
        struct BinOf {
            float o[3], s[3];
            int operator()(const Prim& q, int a) const
            {
                const int k = (int)((q.cen(a) - o[a]) * s[a]);
                return std::min(std::max(k, 0), kBins - 1);
            }
        };
        const BinOf bin_of{{cb.lo[0], cb.lo[1], cb.lo[2]}, {scale[0], scale[1], scale[2]}};
        // bins per chunk, merged in chunk order (exact: integer counts, min and max)
        Bins bins;
        {
            std::vector<Bins> part(T > 1 ? (size_t)T : 0);
            for_chunks(b, e, T, [&](int t, int64_t lo, int64_t hi) {
                Bins& acc = T > 1 ? part[t] : bins;
                const BinOf bo = bin_of;
                const bool lv[3] = {live[0], live[1], live[2]};
                for (int64_t i = lo; i < hi; ++i) {
                    const Prim q = P[i];   // a copy: the bin updates cannot change it
                    for (int a = 0; a < 3; ++a)
                        if (lv[a]) acc.add(a, bo(q, a), q);
                }
            });
            for (const Bins& p : part) bins.merge(p);
        }
        // SAH over the split positions between non-empty bins: every position between two neighbouring
        // non-empty bins gives the same two children and the same cost, so the sweep visits one per
        // group (the highest, where a sweep over all 15 positions from the top meets each group first)
        double best_cost = INFINITY;
        int best_axis = -1, best_bin = -1;
        for (int a = 0; a < 3; ++a) {
            if (!live[a]) continue;
            int ks[kBins], nk = 0;   // the non-empty bins, ascending
            for (uint32_t m = bins.used[a]; m; m &= m - 1) ks[nk++] = __builtin_ctz(m);
            double left_area[kBins];
            int64_t left_cnt[kBins];
            Box acc;
            int64_t c = 0;
            for (int j = 0; j + 1 < nk; ++j) {
                acc.grow(bins.bb[a][ks[j]]);
                c += bins.cnt[a][ks[j]];
                left_area[j] = acc.area();
                left_cnt[j] = c;
            }
            Box racc;
            int64_t rc = 0;
            for (int j = nk - 1; j >= 1; --j) {
                racc.grow(bins.bb[a][ks[j]]);
                rc += bins.cnt[a][ks[j]];
                const double cost = left_area[j - 1] * (double)left_cnt[j - 1] + racc.area() * (double)rc;
                if (cost < best_cost) { best_cost = cost; best_axis = a; best_bin = ks[j]; }
            }
        }
        if (best_axis < 0) return b + n / 2;   // no usable split (all centroids coincide): halve the list
        const int a = best_axis;
        int64_t n_left = 0;
        for (uint32_t m = bins.used[a] & ((1u << best_bin) - 1u); m; m &= m - 1) n_left += bins.cnt[a][__builtin_ctz(m)];
        const int64_t mid = b + n_left;
        struct Left {
            float o, s;
            int a, bin;
            bool operator()(const Prim& q) const
            {
                const int k = (int)((q.cen(a) - o) * s);
                return std::min(std::max(k, 0), kBins - 1) < bin;
            }
        };
        const Left left{bin_of.o[a], bin_of.s[a], a, best_bin};
        if (n < kParallelPass) {
            // in place: swap the first right record from the front with the last left one from the back
            CenBounds gl, gr;
            int64_t i = b, j = e - 1;
            for (;;) {
                while (i <= j && left(P[i])) gl.grow(P[i++]);
                while (i <= j && !left(P[j])) gr.grow(P[j--]);
                if (i >= j) break;
                std::swap(P[i], P[j]);
                gl.grow(P[i++]);
                gr.grow(P[j--]);
            }
            *cl = gl;
            *cr = gr;
        } else {
            // stable, into the other buffer: chunk t's left records go to [b + L_t, ...) and its right
            // records to [mid + R_t, ...), L_t and R_t the counts in the chunks before it
            Prim* D = *dst;
            std::vector<int64_t> nl((size_t)T, 0), lo_at((size_t)T), ro_at((size_t)T);
            if (T > 1)
                for_chunks(b, e, T, [&](int t, int64_t lo, int64_t hi) {
                    int64_t c = 0;
                    for (int64_t i = lo; i < hi; ++i) c += left(P[i]);
                    nl[t] = c;
                });
            else
                nl[0] = n_left;
            int64_t l = 0, r = 0;
            for (int t = 0; t < T; ++t) {
                lo_at[t] = b + l;
                ro_at[t] = mid + r;
                l += nl[t];
                r += n * (t + 1) / T - n * t / T - nl[t];
            }
            std::vector<CenBounds> pl((size_t)T), pr((size_t)T);
            for_chunks(b, e, T, [&](int t, int64_t lo, int64_t hi) {
                int64_t wl = lo_at[t], wr = ro_at[t];
                CenBounds gl, gr;
                for (int64_t i = lo; i < hi; ++i) {
                    const Prim q = P[i];
                    if (left(q)) {
                        D[wl++] = q;
                        gl.grow(q);
                    } else {
                        D[wr++] = q;
                        gr.grow(q);
                    }
                }
                pl[t] = gl;
                pr[t] = gr;
            });
            for (int t = 0; t < T; ++t) {
                cl->grow(pl[t]);
                cr->grow(pr[t]);
            }
            std::swap(*src, *dst);
        }
        for (uint32_t m = bins.used[a]; m; m &= m - 1) {
            const int k = __builtin_ctz(m);
            (k < best_bin ? *bl : *br).grow(bins.bb[a][k]);
        }
        *known = true;
        return mid;
    }

    // build [b, e) (records in src, centroid bounds cb; dst the other buffer) with its first node, if it
    // has one, at index `at`; returns the child reference.  The nodes are in depth-first order, left
    // subtree first, whichever thread builds which subtree.
    uint32_t build(int64_t b, int64_t e, int depth, uint32_t at, const CenBounds& cb, Prim* src, Prim* dst)
    {
        max_depth = std::max(max_depth, depth);
        if (e - b == 1) return kLeafBit | src[b].id;
        Box bl, br;
        CenBounds cbl, cbr;
        bool known = false;
        const int64_t mid = split(b, e, depth, cb, &src, &dst, &bl, &br, &cbl, &cbr, &known);
        if (!known) {
            bl = range_box(src, b, mid);
            br = range_box(src, mid, e);
            cbl = range_centroids(src, b, mid);
            cbr = range_centroids(src, mid, e);
        }
        uint32_t cl, cr;
        if (depth < tr.par_depth && e - b >= kParallelSubtree) {
            Builder sub(tr);
            uint32_t sub_root = kEmptyRef;
            auto left = [&] {
                try {
                    sub_root = sub.build(b, mid, depth + 1, at + 1, cbl, src, dst);
                } catch (...) {
                    sub.error = "host allocation failed in the BVH build";
                }
            };
            std::thread th;
            try {
                th = std::thread(left);
            } catch (...) {
                // no thread to spare: the left subtree is built here, after the right one
            }
            cr = build(mid, e, depth + 1, at + (uint32_t)(mid - b), cbr, src, dst);
            if (th.joinable()) th.join();
            else left();
            cl = sub_root;
            max_depth = std::max(max_depth, sub.max_depth);
            if (!sub.error.empty()) error = sub.error;
        } else {
            cl = build(b, mid, depth + 1, at + 1, cbl, src, dst);
            cr = build(mid, e, depth + 1, at + (uint32_t)(mid - b), cbr, src, dst);
        }
        if (!error.empty()) return kEmptyRef;
        uint16_t el[3], er[3];
        for (int a = 0; a < 3; ++a) {
            if (!round_up_half_extent(bl.lo[a], bl.hi[a], &el[a]) || !round_up_half_extent(br.lo[a], br.hi[a], &er[a])) {
                error = "BVH box extent exceeds the fp16 range";
                return kEmptyRef;
            }
        }
        PackedNode& nd = tr.nodes[at];
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
        return at;
    }
};

}  // namespace

// Smallest fp16 extent h >= 0 such that lo + float(h), evaluated in fp32,
// is >= hi: the decoded box then contains [lo, hi] ("round-to-nearest-not-
// lower").  Fails if no finite half qualifies.
// IEEE 754 binary16, non-negative values only (1 sign bit, 5 exponent bits
// biased by 15, 10 fraction bits; exponent field 0: subnormal m * 2^-24,
// field 31: infinity or NaN).
float half_bits_to_float(uint16_t h)
{
    const uint32_t e = (h >> 10) & 0x1Fu, m = h & 0x3FFu;
    if (e == 0) return (float)m * 5.9604644775390625e-8f;   // m * 2^-24, exact in fp32
    if (e == 31) return INFINITY;
    const uint32_t bits = ((e - 15u + 127u) << 23) | (m << 13);
    float f;
    std::memcpy(&f, &bits, 4);
    return f;
}

namespace {

// the smallest binary16 value >= x, for 0 <= x <= 65504, from the bits of the double
uint16_t half_at_least(double x)
{
    if (!(x > 0.0)) return 0;
    uint64_t b;
    std::memcpy(&b, &x, 8);
    const int ex = (int)((b >> 52) & 0x7FFu) - 1023;
    if (ex < -1022) return 1;                                          // double subnormal: far below 2^-24
    const uint64_t sig = (b & ((1ull << 52) - 1)) | (1ull << 52);     // x = sig * 2^(ex - 52)
    if (ex < -14) {
        // half subnormal: ceil(x 2^24) = ceil(sig / 2^(28 - ex)); 1024 is the smallest normal half's pattern
        const int sh = 28 - ex;
        if (sh >= 64) return 1;
        return (uint16_t)((sig >> sh) + ((sig & ((1ull << sh) - 1)) != 0));
    }
    uint64_t m = (sig >> 42) + ((sig & ((1ull << 42) - 1)) != 0);   // 1 + 10 fraction bits, rounded up
    int E = ex;
    if (m == 2048) {
        m = 1024;
        ++E;
    }
    return (uint16_t)(((uint32_t)(E + 15) << 10) | (uint32_t)(m - 1024));
}

}  // namespace

bool round_up_half_extent(float lo, float hi, uint16_t* out_bits)
{
    const double ext = std::max(0.0, (double)hi - (double)lo);
    if (!(ext <= 65504.0)) return false;
    uint16_t bits = half_at_least(ext);   // every smaller half is below the exact extent
    for (int guard = 0; guard < 64; ++guard) {
        const float e = half_bits_to_float(bits);
        if (!std::isfinite(e)) return false;
        const float top = lo + e;  // fp32 addition as the device performs it
        if (top >= hi) {
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
            const float top = lo + half_bits_to_float(ext[3 * c + a]);   // fp32 addition as the device performs it
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

namespace {

// one node's quantised form; nullptr, or the reason it has none
const char* quantize_node(const PackedNode& n, QuantNode& o)
{
    float box[12];
    decode_packed_boxes(n, box);
    const uint32_t refs[2] = {n.w[9], n.w[10]};
    for (uint32_t r : refs)
        if ((r & ~kLeafBit) >= kQuantRefLimit) return "BVH too large for 24-bit references of quantised nodes";
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
            for (int a = 0; a < 3; ++a) std::memcpy(&o.w[a], &origin[a], 4);
            const uint32_t cl = refs[0] & ~kLeafBit, cr = refs[1] & ~kLeafBit;
            o.w[3] = (uint32_t)e | ((uint32_t)d[0] << 8) | ((uint32_t)d[1] << 10) | ((uint32_t)d[2] << 12) |
                     ((refs[0] & kLeafBit) ? 1u << 14 : 0u) | ((refs[1] & kLeafBit) ? 1u << 15 : 0u) |
                     ((cl & 0xFFFFu) << 16);
            o.w[4] = (cl >> 16) | (cr << 8);
            for (int j = 0; j < 3; ++j)
                o.w[5 + j] = (uint32_t)q[4 * j] | ((uint32_t)q[4 * j + 1] << 8) | ((uint32_t)q[4 * j + 2] << 16) |
                             ((uint32_t)q[4 * j + 3] << 24);
            return nullptr;
        }
        if (guard > 8 || e >= 254) return "BVH box does not fit an 8-bit grid";
        ++e;   // a coarser grid
    }
}

}  // namespace

bool quantize_bvh(const PackedNode* in, size_t n, QuantVec& out, std::string* error)
{
    out.resize(n);
    const int T = host_pass_threads((int64_t)n);
    std::vector<int64_t> bad((size_t)T, -1);   // each chunk's first failing node
    std::vector<const char*> why((size_t)T, nullptr);
    for_chunks(0, (int64_t)n, T, [&](int t, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i)
            if (const char* w = quantize_node(in[i], out[(size_t)i])) {
                bad[t] = i;
                why[t] = w;
                return;
            }
    });
    for (int t = 0; t < T; ++t)
        if (bad[t] >= 0) {
            if (error) *error = why[t];
            return false;
        }
    return true;
}

bool build_bvh(const BuildInput& in, BuildOutput& out, unsigned threads)
{
    out.nodes.clear();
    out.depth = 0;
    if (in.n_prims == 0) {
        out.root = kEmptyRef;
        return true;
    }
    const int64_t n = in.n_prims;
    Tree tr;
    tr.threads = threads ? threads : std::max(1u, std::thread::hardware_concurrency());
    while ((1u << tr.par_depth) < 2 * tr.threads && tr.par_depth < 8) ++tr.par_depth;   // about two subtrees per core
    tr.buf[0].resize((size_t)n);
    tr.buf[1].resize((size_t)n);
    tr.nodes.resize((size_t)std::max<int64_t>(n - 1, 0));
    const int T = n >= kParallelPass ? (int)tr.threads : 1;
    std::vector<CenBounds> part((size_t)T);
    for_chunks(0, n, T, [&](int t, int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            Prim& q = tr.buf[0][(size_t)i];
            for (int a = 0; a < 3; ++a) {
                q.lo[a] = in.lo[3 * i + a];
                q.hi[a] = in.hi[3 * i + a];
            }
            q.id = (uint32_t)i;
            part[t].grow(q);
        }
    });
    CenBounds cb;
    for (const CenBounds& p : part) cb.grow(p);
    Builder bd(tr);
    out.root = bd.build(0, n, 0, 0, cb, tr.buf[0].data(), tr.buf[1].data());
    if (!bd.error.empty()) {
        out.error = bd.error;
        return false;
    }
    out.nodes = std::move(tr.nodes);
    out.depth = bd.max_depth;
    return true;
}

}  // namespace ptk
