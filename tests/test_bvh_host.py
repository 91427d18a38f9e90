"""The scene builder's BVH step on the CPU (pt_build_bvh_host, the same
builder pt_create_scene runs before its upload): every primitive in exactly
one leaf, every stored child box (fp32 origin + fp16 extent, Section 3.1.4)
containing its subtree after the FP32 add the traversal performs, each fp16
extent the smallest that does, the reported depth, determinism and the
argument errors."""
import numpy as np
import pytest

from paper_2305_20061_gb300 import inputs as I

LEAF = 0x80000000


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


def _half(bits):
    return np.array([bits], np.uint16).view(np.float16).astype(np.float32)[0]


def _children(nd):
    """(ref, origin[3], extent bits[3]) of the left and right child."""
    w = nd.astype(np.uint64)
    ext = [int(w[6] & 0xFFFF), int(w[6] >> 16), int(w[7] & 0xFFFF), int(w[7] >> 16), int(w[8] & 0xFFFF),
           int(w[8] >> 16)]
    lo_l = nd[0:3].view(np.float32)
    lo_r = nd[3:6].view(np.float32)
    return [(int(nd[9]), lo_l, ext[0:3]), (int(nd[10]), lo_r, ext[3:6])]


def check_tree(nodes, root, depth, lo, hi):
    n = len(lo)
    assert len(nodes) == max(n - 1, 0)
    if n == 1:
        assert root == LEAF and depth == 0
        return
    seen_leaves, seen_nodes = [], []

    def visit(ref, d):
        """Bounds of the subtree, checking every stored box on the way."""
        if ref & LEAF:
            seen_leaves.append(ref & ~LEAF)
            return lo[ref & ~LEAF].astype(np.float64), hi[ref & ~LEAF].astype(np.float64), d
        seen_nodes.append(ref)
        blo, bhi, dmax = np.full(3, np.inf), np.full(3, -np.inf), d
        for cref, origin, ext in _children(nodes[ref]):
            clo, chi, cd = visit(cref, d + 1)
            dmax = max(dmax, cd)
            for a in range(3):
                e = _half(ext[a])
                top = np.float32(origin[a]) + e            # the FP32 add of the traversal
                assert origin[a] <= clo[a] and top >= chi[a], (ref, a)
                if ext[a] > 0:                             # one fp16 step less would not contain the subtree
                    e1 = _half(ext[a] - 1)
                    assert float(e1) < chi[a] - float(origin[a]) or np.float32(origin[a]) + e1 < chi[a]
            blo, bhi = np.minimum(blo, clo), np.maximum(bhi, chi)
        return blo, bhi, dmax

    _, _, dmax = visit(root, 0)
    assert sorted(seen_leaves) == list(range(n))
    assert sorted(seen_nodes) == list(range(n - 1))
    assert dmax == depth


def _sphere_bounds(sc):
    s = sc.sphere.astype(np.float64)
    lo = np.nextafter((s[:, :3] - s[:, 3:]).astype(np.float32), -np.inf)
    hi = np.nextafter((s[:, :3] + s[:, 3:]).astype(np.float32), np.inf)
    return lo, hi


def _tri_bounds(sc):
    v = sc.vert[sc.tri]                                     # [n, 3 vertices, 3]
    return v.min(1), v.max(1)


@pytest.mark.parametrize("case", ["spheres", "heightfield", "coincident", "two", "one"])
def test_tree_invariants(pt, case):
    if case == "spheres":
        lo, hi = _sphere_bounds(I.spheres_scene(256))
    elif case == "heightfield":
        lo, hi = _tri_bounds(I.heightfield_scene(24))
    elif case == "coincident":                              # many equal centroids: the halving fallback
        c = np.repeat(np.arange(5, dtype=np.float32), 40)[:, None] * np.ones((1, 3), np.float32)
        lo, hi = c - 0.25, c + 0.25
    elif case == "two":
        lo = np.array([[1, 0, 0], [0, 0, 0]], np.float32)
        hi = lo + 0.5
    else:
        lo = np.zeros((1, 3), np.float32)
        hi = np.ones((1, 3), np.float32)
    nodes, root, depth = pt.build_bvh_host(lo, hi)
    check_tree(nodes, root, depth, lo, hi)
    again = pt.build_bvh_host(lo, hi)
    assert np.array_equal(nodes, again[0]) and root == again[1] and depth == again[2]


def test_two_primitives_ordered_by_centroid(pt):
    """Two primitives: the lower centroid along the first axis where they
    differ is the left child."""
    lo = np.array([[0, 2, 0], [0, 1, 0]], np.float32)
    nodes, root, _ = pt.build_bvh_host(lo, lo + 0.5)
    assert int(nodes[root][9]) == LEAF | 1 and int(nodes[root][10]) == LEAF | 0


def test_empty_and_errors(pt):
    nodes, root, depth = pt.build_bvh_host(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    assert len(nodes) == 0 and root == 0xFFFFFFFF and depth == 0
    bad = np.array([[0, 0, 0], [np.nan, 0, 0]], np.float32)
    with pytest.raises(pt.PTError) as e:
        pt.build_bvh_host(bad, bad + 1)
    assert e.value.status == pt.PT_EINVAL
    huge_lo = np.array([[0, 0, 0], [1, 1, 1]], np.float32)
    huge_hi = np.array([[1e5, 1, 1], [2, 2, 2]], np.float32)   # an extent past the fp16 range
    with pytest.raises(pt.PTError) as e:
        pt.build_bvh_host(huge_lo, huge_hi)
    assert e.value.status == pt.PT_EUNSUPPORTED


def test_inverted_box_is_refused(pt):
    """A box with lo > hi on some axis would pack negative extents: refused."""
    lo = np.array([[0, 0, 0], [1, 1, 1]], np.float32)
    hi = np.array([[1, 1, 1], [2, 0.5, 2]], np.float32)   # second box inverted in y
    with pytest.raises(pt.PTError) as e:
        pt.build_bvh_host(lo, hi)
    assert e.value.status == pt.PT_EINVAL
    # a flat box (lo == hi) is fine
    nodes, root, _ = pt.build_bvh_host(lo, np.array([[1, 1, 1], [2, 1, 2]], np.float32))
    assert len(nodes) == 1


def _check_large_tree(nodes, root, depth, lo, hi):
    """check_tree for large inputs: children follow their parent (depth-first
    order), every primitive and node is reached once, and each stored child
    box, decoded as the traversal decodes it, contains its subtree."""
    n = len(lo)
    assert len(nodes) == n - 1 and root == 0
    refs = nodes[:, 9:11].astype(np.int64)
    leaf = (refs & LEAF) != 0
    idx = refs & ~LEAF
    assert np.array_equal(np.sort(idx[leaf]), np.arange(n))
    assert np.array_equal(np.sort(idx[~leaf]), np.arange(1, n - 1))
    parent = np.repeat(np.arange(n - 1), 2).reshape(-1, 2)
    assert np.all(idx[~leaf] > parent[~leaf])
    assert np.all(idx[:, 0][~leaf[:, 0]] == np.arange(n - 1)[~leaf[:, 0]] + 1)   # left subtree first
    origin = nodes[:, 0:6].view(np.float32).reshape(-1, 2, 3)
    ext = np.stack([nodes[:, 6] & 0xFFFF, nodes[:, 6] >> 16, nodes[:, 7] & 0xFFFF, nodes[:, 7] >> 16,
                    nodes[:, 8] & 0xFFFF, nodes[:, 8] >> 16], 1).astype(np.uint16).view(np.float16)
    top = origin + ext.astype(np.float32).reshape(-1, 2, 3)       # the FP32 add of the traversal
    sub_lo = np.zeros((n - 1, 3), np.float32)
    sub_hi = np.zeros((n - 1, 3), np.float32)
    dep = np.zeros(n - 1, np.int64)
    for i in range(n - 2, -1, -1):                                 # children have larger indices
        blo, bhi, d = np.full(3, np.inf, np.float32), np.full(3, -np.inf, np.float32), 0
        for c in range(2):
            j = idx[i, c]
            clo, chi, cd = (lo[j], hi[j], 0) if leaf[i, c] else (sub_lo[j], sub_hi[j], dep[j])
            assert np.all(origin[i, c] <= clo) and np.all(top[i, c] >= chi), (i, c)
            blo, bhi, d = np.minimum(blo, clo), np.maximum(bhi, chi), max(d, cd + 1)
        sub_lo[i], sub_hi[i], dep[i] = blo, bhi, d
    assert dep[0] == depth


@pytest.mark.parametrize("case", ["heightfield", "coincident"])
def test_large_inputs_split_on_several_threads(pt, case):
    """Inputs above 2^16 primitives, whose upper splits bin and partition on
    several host threads into a second record buffer: a valid tree in
    depth-first order, the same on every call."""
    if case == "heightfield":
        lo, hi = _tri_bounds(I.heightfield_scene(200))            # 80,000 triangles
    else:                                                          # the halving fallback on large ranges
        c = np.repeat(np.float32([0, 1]), [70000, 30000])[:, None] * np.ones((1, 3), np.float32)
        lo, hi = c - 0.25, c + 0.25
    nodes, root, depth = pt.build_bvh_host(lo, hi)
    _check_large_tree(nodes, root, depth, lo, hi)
    again = pt.build_bvh_host(lo, hi)
    assert np.array_equal(nodes, again[0]) and root == again[1] and depth == again[2]
