"""The traversal's work counters (node fetches and primitive tests, the
algorithmic work behind the bench's traversal roofline) against an
independent count: the same packed BVH, downloaded from the device, walked
on the host by a plain Python restatement of the closest-hit traversal (near
child first, far child stacked with its entry distance, leaf children
intersected when their box is entered, stacked entries culled once the best
hit is nearer) with the same FP32 slab arithmetic; primitive distances in
FP64.  Camera rays of a pixel sample, one vertex each, on the sphere field
(255 nodes) and on the 10M-triangle heightfield (packed nodes, beyond L2):
scattered pixels, traced ray by ray, and the whole image, whose camera rays
walk the tree as warp packets of 8 x 4 pixels."""
import numpy as np
import pytest
import torch

from paper_2305_20061_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LEAF = 0x80000000
f32 = np.float32


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


def _children(nd):
    lo = nd[0:6].view(np.float32).reshape(2, 3)
    ext = np.array([nd[6] & 0xFFFF, nd[6] >> 16, nd[7] & 0xFFFF, nd[7] >> 16, nd[8] & 0xFFFF, nd[8] >> 16],
                   np.uint32).astype(np.uint16).view(np.float16).astype(np.float32).reshape(2, 3)
    return lo, (lo + ext).astype(np.float32), (int(nd[9]), int(nd[10]))


def _slab(lo, hi, o, inv, tbest):
    t0 = (lo - o) * inv
    t1 = (hi - o) * inv
    tmin = max(max(min(t0[0], t1[0]), min(t0[1], t1[1])), max(min(t0[2], t1[2]), f32(0)))
    tmax = f32(min(min(max(t0[0], t1[0]), max(t0[1], t1[1])), max(t0[2], t1[2])) * f32(1.0000004))
    return tmin if (tmin <= tmax and tmin <= tbest) else f32(np.inf)


def _isect(sc, pid, o, d):
    """Distance to primitive pid (FP64), +inf on a miss."""
    o, d = o.astype(np.float64), d.astype(np.float64)
    nS = len(sc.sphere)
    if pid < nS:
        c, r = sc.sphere[pid, :3].astype(np.float64), float(sc.sphere[pid, 3])
        oc = o - c
        b = oc @ d
        disc = b * b - (oc @ oc - r * r)
        if disc < 0:
            return np.inf
        s = np.sqrt(disc)
        for t in (-b - s, -b + s):
            if t > 0:
                return t
        return np.inf
    v = sc.vert[sc.tri[pid - nS]].astype(np.float64)
    e1, e2 = v[1] - v[0], v[2] - v[0]
    p = np.cross(d, e2)
    det = e1 @ p
    if det == 0:
        return np.inf
    s = o - v[0]
    u = (s @ p) / det
    q = np.cross(s, e1)
    w = (d @ q) / det
    t = (e2 @ q) / det
    return t if (u >= 0 and w >= 0 and u + w <= 1 and t > 0) else np.inf


def _inv(d):
    return np.array([f32(1) / (x if abs(x) > 1e-30 else np.copysign(f32(1e-30), x)) for x in d], np.float32)


def _leaf_tests(sc, refs_t, o, d, best_t, best):
    """Leaf children whose box was entered: (tests, best_t, best)."""
    n = 0
    for ref, tch in refs_t:
        if (ref & LEAF) and np.isfinite(tch):
            n += 1
            t = _isect(sc, ref & ~LEAF, o, d)
            if t < best_t or (t == best_t and (ref & ~LEAF) < best):
                best_t, best = t, ref & ~LEAF
    return n, best_t, best


def reference_work(sc, nodes, root, o, d, start=None):
    """(node fetches, primitive tests, closest primitive) of one ray; with
    start = (cur, stack, best_t, best), the rest of a traversal from that state
    (cur None: resume from the stack)."""
    inv = _inv(d)
    best_t, best = np.inf, -1
    n_nodes = n_prims = 0
    stack, cur = [], root
    if start is not None:
        cur, stack, best_t, best = start
        stack = list(stack)
        if cur is None:
            while stack:
                ref, t = stack.pop()
                if t <= (f32(best_t) if np.isfinite(best_t) else f32(np.inf)):
                    cur = ref
                    break
            else:
                return 0, 0, best
    elif root & LEAF:
        return 0, 1, root & ~LEAF
    while True:
        n_nodes += 1
        lo, hi, (cl, cr) = _children(nodes[cur])
        tb = f32(best_t) if np.isfinite(best_t) else f32(np.inf)
        tl, tr = _slab(lo[0], hi[0], o, inv, tb), _slab(lo[1], hi[1], o, inv, tb)
        k, best_t, best = _leaf_tests(sc, ((cl, tl), (cr, tr)), o, d, best_t, best)
        n_prims += k
        tl = f32(np.inf) if cl & LEAF else tl
        tr = f32(np.inf) if cr & LEAF else tr
        bt = f32(best_t) if np.isfinite(best_t) else f32(np.inf)
        hl, hr = np.isfinite(tl) and tl <= bt, np.isfinite(tr) and tr <= bt
        if hl and hr:
            near, far, tfar = (cl, cr, tr) if tl <= tr else (cr, cl, tl)
            stack.append((far, tfar))
            cur = near
            continue
        if hl or hr:
            cur = cl if hl else cr
            continue
        while stack:
            ref, t = stack.pop()
            if t <= bt:
                cur = ref
                break
        else:
            return n_nodes, n_prims, best


@pytest.mark.parametrize("config,n", [("C2", 600), ("C4", 300)])
def test_traversal_work_matches_an_independent_count(pt, ctx, config, n):
    sc = I.make_scene(config)
    cfg0 = I.CONFIGS[config]["cfg"]
    s = pt.Scene(ctx, sc, node_format="packed")
    nodes, root = s.download_bvh()
    rng = np.random.default_rng(3)
    pix = np.sort(rng.choice(cfg0.width * cfg0.height, n, replace=False)).astype(np.int64)
    cfg = I.RenderCfg(cfg0.width, cfg0.height, 1, 1)
    _, _, ids = pt.render_pixels(ctx, s, None if sc.env_const is not None else pt.Nif(ctx, I.nif_init()), cfg,
                                 torch.from_numpy(pix).cuda(), want_ids=True)
    ctx.check()
    work = pt.last_render_work(ctx)
    org, dirs = pt.primary_rays(ctx, s, cfg, 0, cfg.width * cfg.height)
    org, dirs = org.cpu().numpy()[pix], dirs.cpu().numpy()[pix]
    ref_nodes = ref_prims = agree = 0
    gids = ids.cpu().numpy().reshape(-1)
    for i in range(n):
        a, b, best = reference_work(sc, nodes, root, org[i].astype(np.float32), dirs[i].astype(np.float32))
        ref_nodes += a
        ref_prims += b
        agree += int(best == gids[i])
    gpu_prims = work["sphere"] + work["quad"] + work["triangle"]
    print({config: {"gpu": work, "reference_nodes": ref_nodes, "reference_prims": ref_prims, "ids_agree": agree}})
    assert agree >= n - 1
    assert abs(work["nodes"] - ref_nodes) <= 1e-3 * ref_nodes + 2
    assert abs(gpu_prims - ref_prims) <= 1e-3 * ref_prims + 2


PACKET_MIN_LANES = 24   # the traversal kernel's switch from a warp packet to single rays


def packet_work(sc, nodes, root, org, dirs):
    """(node fetches, primitive tests, closest primitives) of one warp packet
    of camera rays: the warp visits every node that one of its rays entered,
    each ray testing the node's child boxes, a node counted for the rays that
    entered it; the near child is the one most entering rays reach first; a
    stacked node is visited while a ray still needs it; below
    PACKET_MIN_LANES entering rays each ray goes on alone from that state."""
    n = len(org)
    inv = [_inv(d) for d in dirs]
    bt = [np.inf] * n
    best = [-1] * n
    need = [True] * n
    stack, cur = [], root
    n_nodes = n_prims = 0

    def f(t):
        return f32(t) if np.isfinite(t) else f32(np.inf)

    while True:
        if sum(need) < PACKET_MIN_LANES:
            for i in range(n):
                lane_stack = [(ref, ts[i]) for ref, ts in stack]
                a, b, best[i] = reference_work(sc, nodes, root, org[i], dirs[i],
                                               start=(cur if need[i] else None, lane_stack, bt[i], best[i]))
                n_nodes += a
                n_prims += b
            return n_nodes, n_prims, best
        lo, hi, (cl, cr) = _children(nodes[cur])
        n_nodes += sum(need)
        tl, tr, hl, hr = [], [], [], []
        for i in range(n):
            a = _slab(lo[0], hi[0], org[i], inv[i], f(bt[i]))
            b = _slab(lo[1], hi[1], org[i], inv[i], f(bt[i]))
            k, bt[i], best[i] = _leaf_tests(sc, ((cl, a), (cr, b)), org[i], dirs[i], bt[i], best[i])
            n_prims += k
            a = f32(np.inf) if cl & LEAF else a
            b = f32(np.inf) if cr & LEAF else b
            tl.append(a)
            tr.append(b)
            hl.append(bool(np.isfinite(a) and a <= f(bt[i])))
            hr.append(bool(np.isfinite(b) and b <= f(bt[i])))
        if any(hl) and any(hr):
            pref = sum(hl[i] and (not hr[i] or tl[i] <= tr[i]) for i in range(n))
            left_first = 2 * pref >= sum(hl[i] or hr[i] for i in range(n))
            far_t = [(tr[i] if hr[i] else f32(np.inf)) if left_first else (tl[i] if hl[i] else f32(np.inf))
                     for i in range(n)]
            stack.append((cr if left_first else cl, far_t))
            cur, need = (cl, hl) if left_first else (cr, hr)
        elif any(hl):
            cur, need = cl, hl
        elif any(hr):
            cur, need = cr, hr
        else:
            while stack:
                ref, ts = stack.pop()
                want = [ts[i] <= f(bt[i]) for i in range(n)]
                if any(want):
                    cur, need = ref, want
                    break
            else:
                return n_nodes, n_prims, best


def tile_order(W, H):
    """The pixels of one sample in the order the camera rays of a whole image
    are taken: 8 x 4 pixel tiles, row by row within a tile (W % 8 == H % 4 == 0)."""
    out = np.empty(W * H, np.int64)
    for j in range(W * H):
        b, l = j >> 5, j & 31
        band, bx = divmod(b, W >> 3)
        out[j] = (band * 4 + (l >> 3)) * W + bx * 8 + (l & 7)
    return out


@pytest.mark.parametrize("config,W,H", [("C2", 64, 32), ("C4", 48, 24)])
def test_packet_traversal_work_matches_an_independent_count(pt, ctx, config, W, H):
    """Camera rays of a whole image (wavefront schedule, one vertex): the
    work counters of the warp packets against the host walk of the same
    packets, and the closest hits against it."""
    sc = I.make_scene(config)
    s = pt.Scene(ctx, sc, node_format="packed")
    nodes, root = s.download_bvh()
    cfg = I.RenderCfg(W, H, 1, 1)
    nif = None if sc.env_const is not None else pt.Nif(ctx, I.nif_init())
    _, _, ids = pt.render_pixels(ctx, s, nif, cfg, None, want_ids=True, schedule="wavefront")
    ctx.check()
    work = pt.last_render_work(ctx)
    org, dirs = pt.primary_rays(ctx, s, cfg, 0, W * H)
    org, dirs = org.cpu().numpy().astype(np.float32), dirs.cpu().numpy().astype(np.float32)
    gids = ids.cpu().numpy().reshape(-1)
    order = tile_order(W, H)
    ref_nodes = ref_prims = agree = 0
    for p0 in range(0, W * H, 32):
        pix = order[p0:p0 + 32]
        a, b, best = packet_work(sc, nodes, root, org[pix], dirs[pix])
        ref_nodes += a
        ref_prims += b
        agree += int(np.sum(np.array(best) == gids[pix]))
    gpu_prims = work["sphere"] + work["quad"] + work["triangle"]
    print({config: {"gpu": work, "reference_nodes": ref_nodes, "reference_prims": ref_prims, "ids_agree": agree}})
    assert agree >= W * H - 1
    assert abs(work["nodes"] - ref_nodes) <= 1e-3 * ref_nodes + 2
    assert abs(gpu_prims - ref_prims) <= 1e-3 * ref_prims + 2
