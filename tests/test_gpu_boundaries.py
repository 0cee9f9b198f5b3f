"""GPU parity with physical boundaries (zero-gradient outflow and fixed
inflow): the CUDA path through the C ABI against the CPU oracle on bounded
domains whose fine patches touch the boundaries. FP64 (strict build) within
1e-12 relative L1 per field with a bitwise dt sequence; the mixed path on a
smooth bounded flow within 1e-5."""
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


def gpu_for(pb, precision=A.FP64, advance=None):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    if advance is not None:
        ctx.set_option(A.OPT_ADVANCE, advance)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


def run_both(pb, nsteps, precision=A.FP64, advance=None):
    ctx = gpu_for(pb, precision, advance)
    dts = ctx.step(nsteps)
    o = oracle_for(pb)
    odts = np.array([o.step() for _ in range(nsteps)])
    return ctx, dts, o, odts


def edge_hierarchy_2d():
    return inputs.tile(0, (0, 0, 0), (32, 32, 1), 8, 2) + [
        (1, (0, 8, 0), (16, 40, 1)), (1, (48, 0, 0), (64, 24, 1)), (2, (0, 24, 0), (16, 56, 1))]


def corner_hierarchy_3d():
    return inputs.tile(0, (0, 0, 0), (16, 16, 16), 8, 3) + [
        (1, (0, 0, 0), (16, 16, 16)), (1, (16, 0, 16), (32, 8, 32)), (1, (24, 24, 0), (32, 32, 8))]


@pytest.mark.parametrize("dim,n,steps", [(2, 64, 30), (3, 64, 8)])
def test_stationary_shock_fp64(dim, n, steps):
    """Mach-10 inflow at x-low, outflow at x-high, level 1 over the shock
    and both x boundaries."""
    pb = inputs.stationary_shock(dim, n=n, refine=True)
    ctx, dts, o, odts = run_both(pb, steps)
    assert np.array_equal(dts, odts), np.abs(dts - odts).max()
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("mirrored", [False, True])
def test_smooth_bounded_fp64(mirrored):
    pb = inputs.smooth_bounded_2d(32, refine=True, seed=4, mirrored=mirrored)
    ctx, dts, o, odts = run_both(pb, 8)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("bc", [(2, 1, 0, 0, 0, 0), (1, 2, 2, 1, 0, 0)])
def test_random_smooth_on_edge_hierarchy_fp64(bc):
    """Three levels whose fine patches touch the bounded sides; inflow state
    differing from the interior so the inflow ghosts matter."""
    st = inputs.random_smooth_2d(32, 3, seed=9)
    inflow = inputs.conserved((1.1, 0.4, -0.1, 0.05, 0.9, 0.3, 0.2, 0.1))
    pb = inputs.Problem("edge2", 2, (32, 32, 1), edge_hierarchy_2d(), 3, st, bc=bc, inflow=inflow)
    ctx, dts, o, odts = run_both(pb, 6)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("advance", [2, 3])
def test_corner_hierarchy_3d_fp64(advance):
    """3D blast on a bounded box (inflow, outflow and periodic sides mixed),
    level-1 patches in three corners; staged (2) and fused (3) advance."""
    base = (16, 16, 16)
    st = {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]}
    inflow = inputs.conserved((1.0, 0.5, 0.0, 0.0, 0.1) + (1 / 3 ** 0.5,) * 3)
    pb = inputs.Problem("corner3", 3, base, corner_hierarchy_3d(), 2, st, bc=(2, 1, 1, 1, 0, 0), inflow=inflow)
    ctx, dts, o, odts = run_both(pb, 6, advance=advance)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_uniform_flow_preserved_3d(precision):
    pb = inputs.uniform_flow(3, (16, 16, 16), corner_hierarchy_3d(), 2, (2, 1, 1, 2, 1, 1), seed=3)
    ctx = gpu_for(pb, precision)
    g0 = gpu_level_arrays(ctx, pb)
    ctx.step(3)
    g = gpu_level_arrays(ctx, pb)
    for l in range(pb.nlev):
        for f in range(8):
            m = ~np.isnan(g0[l][f])
            assert np.array_equal(g[l][f][m], g0[l][f][m]), (l, f)


def test_mixed_smooth_bounded_within_1e5():
    pb = inputs.smooth_bounded_2d(64, refine=True, seed=2)
    ctx, dts, o, odts = run_both(pb, 20, precision=A.MIXED)
    assert np.allclose(dts, odts, rtol=1e-5)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-5, res
