"""The multi-level queue advance (AMRMHD_OPT_QUEUE): one persistent launch per
sub-step of the finest level takes the finest level's same-level ghost copies
and every starting level's advance tiles from a device queue, finest level
first, with per-patch counters between the copies and the tiles.

* Strict FP64: bit for bit equal to the level-by-level launches (the same
  formulas on the same inputs in the same data flow), and equal to the oracle.
* Mixed precision: within FP32 rounding of the level-by-level launches.
* A withheld fill signal (test switch) makes a wait run out: amrmhd_step
  returns AMRMHD_ETIMEOUT within a bounded time, nothing hangs, and the context
  steps correctly afterwards.
"""
import time

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


def three_level_3d():
    """16^3 base in 8^3 patches, random properly nested levels 1 and 2 (seeded),
    a smooth finite-amplitude wave on every level."""
    patches = inputs.random_hierarchy(3, 5, base=16, psize0=8, nlev=3)
    nlev = max(p[0] for p in patches) + 1
    st = {l: inputs.mhd_wave(3, 16 << l, "fast", amp=1e-2, v0=(0.3, -0.2, 0.25)).state[0] for l in range(nlev)}
    return inputs.Problem("rand3d", 3, (16, 16, 16), patches, nlev, st)


def run(pb, precision, steps, queue, **opts):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    ctx.set_option(A.OPT_ADVANCE, 3)
    ctx.set_option(A.OPT_QUEUE, 1 if queue else 0)
    for k, v in opts.items():
        ctx.set_option(getattr(A, k), v)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx, ctx.step(steps)


def test_queue_hierarchy_has_three_levels():
    assert three_level_3d().nlev == 3


@pytest.mark.parametrize("tile,balance", [(3, 1), (2, 1), (3, 0)])
def test_queue_equals_level_launches_fp64(tile, balance):
    """Tile variants and both ways of sharing out the coarser levels' tiles
    (work-balanced or equal counts) give the level-by-level result."""
    pb = three_level_3d()
    a, da = run(pb, A.FP64, 3, True, OPT_QUEUE_TILE=tile, OPT_QUEUE_BALANCE=balance)
    b, db = run(pb, A.FP64, 3, False)
    assert np.array_equal(da, db)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)


def test_queue_fp64_equals_oracle():
    pb = three_level_3d()
    ctx, dts = run(pb, A.FP64, 3, True)
    o = oracle_for(pb)
    odts = np.array([o.step() for _ in range(3)])
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_queue_mixed_close_to_level_launches():
    pb = three_level_3d()
    a, _ = run(pb, A.MIXED, 3, True)
    b, _ = run(pb, A.MIXED, 3, False)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            x, y = sa[f][p], sb[f][p]
            assert np.all(np.isfinite(x))
            assert np.abs(x - y).sum() <= 1e-5 * np.abs(y).sum() + 1e-12, (f, p)


def test_withheld_signal_times_out_and_the_context_recovers():
    pb = three_level_3d()
    ctx, _ = run(pb, A.FP64, 0, True, OPT_QUEUE_WITHHOLD=1)
    t0 = time.time()
    with pytest.raises(A.AmrmhdError) as e:
        ctx.step(1)
    assert e.value.status == A.ETIMEOUT
    assert time.time() - t0 < 30.0
    # the switch off, the initial state back: the next steps are correct
    ctx.set_option(A.OPT_QUEUE_WITHHOLD, 0)
    ctx.load_state(pb.state)
    d1 = ctx.step(2)
    b, d2 = run(pb, A.FP64, 2, False)
    assert np.array_equal(d1, d2)
    sa, sb = ctx.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)
