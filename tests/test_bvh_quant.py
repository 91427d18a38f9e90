"""The quantised BVH node form (8-bit grid per node, 32 bytes; the paper's
quarter-precision outlook, Section 5) on the CPU: pt_quantize_bvh_host turns
the builder's packed tree into the form the traversal reads, and every
decoded child box (origin + q * 2^(e - 127 - d) in fp32, the device's
arithmetic) contains the packed tree's decoded fp16-extent box and so the
whole subtree; references are preserved; codes are tight (one grid step less
would not contain); oversized references are refused."""
import numpy as np
import pytest

from paper_2305_20061_gb300 import inputs as I

from test_bvh_host import LEAF, _half, _sphere_bounds, _tri_bounds


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


def packed_boxes(nd):
    """Decoded child boxes of a packed node: [2, 2, 3] (child, lo/hi, axis) as fp32."""
    ext = np.array([nd[6] & 0xFFFF, nd[6] >> 16, nd[7] & 0xFFFF, nd[7] >> 16, nd[8] & 0xFFFF, nd[8] >> 16],
                   np.uint32).astype(np.uint16).view(np.float16).astype(np.float32)
    lo = nd[0:6].view(np.float32).reshape(2, 3)
    return np.stack([lo, (lo + ext.reshape(2, 3)).astype(np.float32)], 1)


def quant_fields(q):
    w = q.astype(np.uint64)
    origin = q[0:3].view(np.float32)
    meta = int(w[3])
    e = meta & 0xFF
    d = [(meta >> 8) & 3, (meta >> 10) & 3, (meta >> 12) & 3]
    leaf = [(meta >> 14) & 1, (meta >> 15) & 1]
    refs = [(meta >> 16) | ((int(w[4]) & 0xFF) << 16), int(w[4]) >> 8]
    codes = np.concatenate([np.array([(int(x) >> (8 * k)) & 0xFF for k in range(4)]) for x in w[5:8]])
    return origin, e, d, leaf, refs, codes.reshape(2, 2, 3)   # child, lo/hi, axis


def decode(origin, e, d, codes):
    step = np.array([np.ldexp(np.float32(1), e - 127 - d[a]) for a in range(3)], np.float32)
    return (origin[None, None, :] + (codes.astype(np.float32) * step[None, None, :])).astype(np.float32), step


def check_quantised(nodes, q):
    assert q.shape == (len(nodes), 8)
    for nd, qq in zip(nodes, q):
        origin, e, d, leaf, refs, codes = quant_fields(qq)
        pb = packed_boxes(nd)
        box, step = decode(origin, e, d, codes)
        assert np.all(box[:, 0] <= pb[:, 0]) and np.all(box[:, 1] >= pb[:, 1])
        # tight: the next code inwards would not contain the packed box
        for c in range(2):
            for a in range(3):
                if codes[c, 0, a] < 255:
                    inner = np.float32(origin[a] + np.float32((codes[c, 0, a] + 1) * step[a]))
                    assert inner > pb[c, 0, a]
                if codes[c, 1, a] > 0:
                    inner = np.float32(origin[a] + np.float32((codes[c, 1, a] - 1) * step[a]))
                    assert inner < pb[c, 1, a]
        for c, ref in enumerate((int(nd[9]), int(nd[10]))):
            assert leaf[c] == (1 if ref & LEAF else 0) and refs[c] == ref & ~LEAF
        assert np.all(origin == np.minimum(pb[0, 0], pb[1, 0]))


@pytest.mark.parametrize("case", ["spheres", "heightfield", "random_tris"])
def test_quantised_boxes_contain_the_packed_boxes(pt, case):
    if case == "spheres":
        lo, hi = _sphere_bounds(I.spheres_scene())
    elif case == "heightfield":
        lo, hi = _tri_bounds(I.heightfield_scene(40))
    else:
        lo, hi = _tri_bounds(I.random_triangles_scene(3000, seed=4))
    nodes, root, depth = pt.build_bvh_host(lo, hi)
    q = pt.quantize_bvh_host(nodes)
    check_quantised(nodes, q)
    # and therefore every primitive: walk the tree with the quantised boxes
    def visit(ref):
        if ref & LEAF:
            return lo[ref & ~LEAF], hi[ref & ~LEAF]
        origin, e, d, leaf, refs, codes = quant_fields(q[ref])
        box, _ = decode(origin, e, d, codes)
        blo, bhi = np.full(3, np.inf, np.float32), np.full(3, -np.inf, np.float32)
        for c in range(2):
            clo, chi = visit(refs[c] | (LEAF if leaf[c] else 0))
            assert np.all(box[c, 0] <= clo) and np.all(box[c, 1] >= chi)
            blo, bhi = np.minimum(blo, clo), np.maximum(bhi, chi)
        return blo, bhi
    if case != "random_tris":   # the deep random tree is covered by the node-by-node check above
        visit(root)


def test_quantised_codes_use_the_grid(pt):
    """A node whose children span the grid: the larger child reaches code 255 or close, and an axis much
    thinner than the others gets a finer step (d > 0)."""
    lo = np.array([[0, 0, 0], [5, 0, 0]], np.float32)
    hi = np.array([[4, 0.01, 1], [9, 0.02, 1]], np.float32)
    nodes, root, _ = pt.build_bvh_host(lo, hi)
    origin, e, d, leaf, refs, codes = quant_fields(pt.quantize_bvh_host(nodes)[0])
    assert leaf == [1, 1] and sorted(refs) == [0, 1]
    assert codes[:, 1, 0].max() >= 128          # x spans the grid
    assert d[1] == 3 and d[0] == 0               # y is 100x thinner: the finest offset


def test_quantise_refuses_wide_references(pt):
    nodes = np.zeros((1, 12), np.uint32)
    nodes[0, 9] = LEAF | (1 << 24)               # a primitive ID past 24 bits
    nodes[0, 10] = LEAF | 0
    with pytest.raises(pt.PTError) as e:
        pt.quantize_bvh_host(nodes)
    assert e.value.status == pt.PT_EUNSUPPORTED
    assert pt.quantize_bvh_host(np.zeros((0, 12), np.uint32)).shape == (0, 8)
