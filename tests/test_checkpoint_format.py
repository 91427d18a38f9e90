"""The checkpoint file format of include/pt.h, pinned on the CPU: a file
written here from the documented layout (with FNV-1a from its published
definition: offset basis 14695981039346656037, prime 1099511628211) is read
back by the library's host-only reader; corrupted, truncated, foreign and
future-version files are refused.  No GPU is needed."""
import os
import struct

import numpy as np
import pytest


def fnv1a(data: bytes) -> int:
    h = 14695981039346656037
    for b in data:
        h ^= b
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _file(kind=2, version=1, dims=(3, 8, 2, 0), box=(-1, -2, -3, 1, 2, 3), params=None, m=None, v=None, adam_t=7):
    params = np.arange(11, dtype=np.float32) * 0.5 if params is None else params
    m = np.zeros(0, np.float32) if m is None else m
    v = np.zeros(0, np.float32) if v is None else v
    head = b"PTCKPT01" + struct.pack("<II4i6fqqq", kind, version, *dims, *box, params.size, m.size, adam_t)
    assert len(head) == 80
    body = head + params.astype("<f4").tobytes() + m.astype("<f4").tobytes() + v.astype("<f4").tobytes()
    return body + struct.pack("<Q", fnv1a(body))


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


def test_reads_the_documented_layout(pt, tmp_path):
    f = tmp_path / "a.ckpt"
    m = np.full(11, 0.25, np.float32)
    f.write_bytes(_file(params=np.linspace(-1, 1, 11).astype(np.float32), m=m, v=m * 2, adam_t=42))
    info = pt.checkpoint_info(str(f))
    assert info["kind"] == "cache" and info["version"] == 1 and info["dims"] == [3, 8, 2, 0]
    assert info["lo"] == [-1.0, -2.0, -3.0] and info["hi"] == [1.0, 2.0, 3.0]
    assert info["n_params"] == 11 and info["n_adam"] == 11 and info["adam_t"] == 42


def test_fnv1a_known_values():
    # published test vectors of 64-bit FNV-1a
    assert fnv1a(b"") == 0xCBF29CE484222325
    assert fnv1a(b"a") == 0xAF63DC4C8601EC8C
    assert fnv1a(b"foobar") == 0x85944171F73967E8


@pytest.mark.parametrize("damage", ["flip", "truncate", "magic", "sizes", "missing"])
def test_damaged_files_are_refused_with_eio(pt, tmp_path, damage):
    f = tmp_path / "b.ckpt"
    data = bytearray(_file())
    if damage == "flip":
        data[90] ^= 0x01               # a parameter byte: the hash no longer matches
    elif damage == "truncate":
        data = data[:-5]
    elif damage == "magic":
        data[0:8] = b"PTCKPT00"
    elif damage == "sizes":
        data = bytearray(_file(params=np.zeros(12, np.float32)))
        data[56:64] = struct.pack("<q", 13)   # n_params says 13: the file length disagrees
    if damage != "missing":
        f.write_bytes(bytes(data))
    with pytest.raises(pt.PTError) as e:
        pt.checkpoint_info(str(f))
    assert e.value.status == pt.PT_EIO


def test_future_version_is_refused_with_einval(pt, tmp_path):
    f = tmp_path / "c.ckpt"
    f.write_bytes(_file(version=2))
    with pytest.raises(pt.PTError) as e:
        pt.checkpoint_info(str(f))
    assert e.value.status == pt.PT_EINVAL
