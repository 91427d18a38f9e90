"""The measurement helpers behind the roofline denominators: the FP32 FMA
rate and the L2 read bandwidth, each within the bounds the GB300's
documented unit counts and clocks allow, and their argument checks."""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


def test_ffma_rate_is_below_the_unit_count_peak(pt):
    # 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz = 80.5 TFLOP/s at most
    rate = pt.ffma_rate_tflops(0)
    print({"ffma_tflops": rate})
    assert 20.0 < rate <= 81.0


def test_l2_read_rate(pt):
    """A buffer inside L2 read again and again: faster than HBM (the
    measured copy bandwidth is about 6.7 TB/s) and below 128 B per SM per
    clock (about 40 TB/s)."""
    rate = pt.l2_read_rate_gbs(0)
    print({"l2_read_gbs": rate})
    assert 6000.0 < rate < 41000.0


def test_l2_read_rejects_bad_arguments(pt):
    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = C.c_double(0)
    lib = pt.lib()
    p = C.c_void_p(buf.data_ptr())
    s = C.c_void_p(sink.data_ptr())
    assert lib.pt_microbench_l2_read(C.c_void_p(buf.data_ptr() + 4), 4096, 1, s, C.byref(out), None) == pt.PT_EINVAL
    assert lib.pt_microbench_l2_read(p, 8, 1, s, C.byref(out), None) == pt.PT_EINVAL
    assert lib.pt_microbench_l2_read(p, 4096, 0, s, C.byref(out), None) == pt.PT_EINVAL
    assert lib.pt_microbench_l2_read(p, 4096, 2, s, C.byref(out), None) == pt.PT_OK
    torch.cuda.synchronize()
    assert out.value == 8192.0
