"""Direct halo reads of the fused 3D advance (AMRMHD_OPT_DIRECT_HALO): on a
level of equal patches tiling the periodic domain with no finer level, the
advance reads its halo from the neighbour patches and the same-level ghost
fill is skipped. The results must equal the fill-then-read path bit for bit
in the strict FP64 build (same inputs to the same arithmetic, no contraction)
and within FP32 rounding in mixed precision (the two are separate kernel
instances, whose multiply-adds the compiler may contract differently), with
1, 2, 4 and 6 patches per dimension (a patch that is its own neighbour,
neighbours -1 and +1 the same patch, distinct neighbours), and the strict FP64
result must equal the oracle."""
import numpy as np
import pytest

from helpers import compare_states, gpu_level_arrays, max_err, oracle_for
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


def run(pb, precision, steps, direct, fused=True):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    if fused:
        ctx.set_option(A.OPT_ADVANCE, 3)
    ctx.set_option(A.OPT_DIRECT_HALO, 1 if direct else 0)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    l0 = ctx.query(A.Q_KERNEL_LAUNCHES)
    dts = ctx.step(steps)
    launches = ctx.query(A.Q_KERNEL_LAUNCHES) - l0
    return ctx, dts, launches


@pytest.mark.parametrize("n,psize", [(16, 16), (32, 16), (64, 16), (48, 8)])
@pytest.mark.parametrize("precision", [A.MIXED, A.FP64])
def test_direct_halo_equals_fill(n, psize, precision):
    pb = inputs.blast_3d(n, psize)
    a, da, la = run(pb, precision, 4, True)
    b, db, lb = run(pb, precision, 4, False)
    if precision == A.FP64:
        assert np.array_equal(da, db)
    else:
        assert np.allclose(da, db, rtol=1e-5, atol=0.0)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            x, y = sa[f][p], sb[f][p]
            if precision == A.FP64:
                assert np.array_equal(x, y), (f, p)
            else:
                assert np.all(np.isfinite(x)) and np.abs(x - y).sum() <= 1e-5 * np.abs(y).sum() + 1e-12, (f, p)
    assert la < lb, (la, lb)  # the fills are not launched


def test_direct_halo_fp64_equals_oracle():
    pb = inputs.mhd_wave(3, 32, "fast", amp=1e-2, v0=(0.3, -0.2, 0.25), psize=8)
    ctx, dts, _ = run(pb, A.FP64, 5, True)
    o = oracle_for(pb)
    odts = np.array([o.step() for _ in range(5)])
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_levels_with_children_keep_their_fills():
    """Level 0 of a two-level hierarchy has a finer level (its ghosts feed the
    prolongation), and level 1 does not tile the domain: the option changes
    nothing there."""
    base = (16, 16, 16)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 24, 24), 8, 3)
    st = {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]}
    pb = inputs.Problem("b3", 3, base, patches, 2, st)
    a, _, la = run(pb, A.MIXED, 3, True)
    b, _, lb = run(pb, A.MIXED, 3, False)
    assert la == lb
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)
