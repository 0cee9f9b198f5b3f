"""Density and pressure floors (amrmhd_set_floors): never raised on a problem
that does not need them (the down-scaled shock clump, bitwise the same result
as without floors), raised and counted where a pressure is negative (a state
that otherwise stops with AMRMHD_ENONPHYS), refused by the adjoint."""
import numpy as np
import pytest

from helpers import gpu_level_arrays, owned_mask
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


def ctx_for(pb, precision, floors=None):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    if floors:
        ctx.set_floors(*floors)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


@pytest.mark.parametrize("precision", [A.MIXED, A.FP64])
def test_floors_silent_where_not_needed(precision):
    pb = inputs.shock_clump_3d_small(16, 3)
    a = ctx_for(pb, precision, floors=(1e-8, 1e-8))
    b = ctx_for(pb, precision)
    da, db = a.step(4), b.step(4)
    assert np.array_equal(da, db)
    assert a.query(A.Q_FLOOR_EVENTS) == 0
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)


@pytest.mark.parametrize("precision", [A.MIXED, A.FP64])
def test_floors_raise_a_negative_pressure(precision):
    pb = inputs.blast_3d(32, 16)
    e = pb.state[0][4].copy()
    e[5, 6, 7] = 0.05  # below the magnetic energy 1/2: negative pressure
    pb.state[0][4] = e
    bad = ctx_for(pb, precision)
    with pytest.raises(A.AmrmhdError) as err:
        bad.step(1)
    assert err.value.status == A.ENONPHYS
    ctx = ctx_for(pb, precision, floors=(1e-6, 1e-3))
    ctx.step(2)
    assert ctx.query(A.Q_FLOOR_EVENTS) > 0
    g = gpu_level_arrays(ctx, pb)
    for f in range(8):
        assert np.all(np.isfinite(g[0][f][owned_mask(pb, 0, f)])), f


def test_adjoint_refuses_floors():
    import torch
    pb = inputs.orszag_tang(32, 8, refine=False)
    ctx = ctx_for(pb, A.FP64, floors=(1e-8, 1e-8))
    n = sum(ctx.packed_size(f) for f in range(8))
    g = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(A.AmrmhdError) as err:
        ctx.backward(np.array([1e-3]), g, torch.zeros_like(g), 1)
    assert err.value.status == A.ESTATE
