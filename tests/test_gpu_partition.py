"""SM partitions (amrmhd_sm_partition_create): a context whose stream belongs
to a partition of the GPU's SMs gives, bit for bit, the result of the same
steps on an ordinary stream (only where the kernels run changes)."""
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


def run(pb, stream):
    import torch
    ctx = A.context_for(pb, precision=A.MIXED, stream=stream)
    ctx.set_option(A.OPT_CONCURRENT, 0)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    dts = ctx.step(3)
    return ctx.read_state(), dts


def test_partition_stream_gives_the_same_result():
    import torch
    pb = inputs.cylinder_3d_tiled((1, 1, 1), 32, 16)
    part = A.SmPartition(16)
    try:
        assert 16 <= part.sms <= torch.cuda.get_device_properties(0).multi_processor_count
        sa, da = run(pb, part.stream)
        sb, db = run(pb, torch.cuda.Stream().cuda_stream)
    finally:
        torch.cuda.synchronize()
        part.close()
    assert np.array_equal(da, db)
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)
