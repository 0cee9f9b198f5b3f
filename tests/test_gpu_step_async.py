"""Stream-ordered coarse steps (amrmhd_step_async) and amrmhd_sync: the steps
queued without waiting give the state and dt history of amrmhd_step bit for
bit, interleaved with stream-ordered state I/O through device pointers; a
non-physical state is reported by the next synchronising call, not by the
queuing one, and the error word is cleared once reported."""
import ctypes as C

import numpy as np
import pytest

from paper_1110_1616_gb300 import amrmhd as A
from paper_1110_1616_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_1616_gb300 import build
    build.build()


def make(pb, precision):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_async_steps_equal_steps(precision):
    pb = inputs.orszag_tang(64, 16, refine=True)
    a, b = make(pb, precision), make(pb, precision)
    a.step_async(3)
    a.step_async(2)
    a.sync()
    b.step(5)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)
    assert np.array_equal(a.step(2), b.step(2))  # the dt sequence goes on the same


def test_async_steps_with_device_state_io():
    """Queue: load the state from a device buffer, two async steps, store the
    state into another device buffer; equal to the synchronous calls."""
    import torch
    pb = inputs.blast_3d(32, 16)
    a, b = make(pb, A.MIXED), make(pb, A.MIXED)
    n = sum(int(a.packed_size(f)) for f in range(8))
    src = torch.empty(n, dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    lib = A.lib()
    assert lib.amrmhd_get_state_all_f32(a.h, C.c_void_p(src.data_ptr()), 1) == 0
    torch.cuda.synchronize()
    assert lib.amrmhd_set_state_all_f32(a.h, C.c_void_p(src.data_ptr()), 1) == 0
    a.step_async(2)
    assert lib.amrmhd_get_state_all_f32(a.h, C.c_void_p(dst.data_ptr()), 1) == 0
    a.sync()
    b.step(2)
    ref = torch.empty_like(src)
    assert lib.amrmhd_get_state_all_f32(b.h, C.c_void_p(ref.data_ptr()), 1) == 0
    torch.cuda.synchronize()
    assert torch.equal(dst, ref)


def test_nonphysical_state_reported_by_sync():
    pb = inputs.orszag_tang(32, 8, refine=False)
    pb.state[0][4] = pb.state[0][4].copy()
    pb.state[0][4][0, 3, 3] = -1.0  # negative total energy -> negative pressure
    ctx = make(pb, A.FP64)
    ctx.step_async(1)  # queued: no report yet
    with pytest.raises(A.AmrmhdError) as e:
        ctx.sync()
    assert e.value.status == A.ENONPHYS
    ctx.sync()  # reported once: the error word is clear
