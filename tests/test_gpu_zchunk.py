"""The fused 3D advance split along z (AMRMHD_OPT_ZCHUNK: n planes per CTA)
gives the unsplit result bit for bit: every chunk restarts the z march two
planes below its first output plane and recomputes the same primitives,
predicted states, fluxes and EMFs there, and a face or edge plane that two
chunks share is captured for the registers by one of them. Chunk lengths 1,
3 and 8 cut the columns of 8^3 to 16^3 patches (12 to 20 planes with the two
extended ghost layers of sub-step 1) into full and ragged chunks."""
import numpy as np
import pytest

from paper_1110_1616_gb300 import amrmhd as A
from paper_1110_1616_gb300 import inputs
from helpers import oracle_for, gpu_level_arrays, compare_states, max_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_1616_gb300 import build
    build.build()


def three_level_3d():
    """16^3 base in 8^3 patches, random properly nested levels 1 and 2 (seeded;
    patch widths 8 to 16), a finite-amplitude fast wave on every level."""
    patches = inputs.random_hierarchy(3, 5, base=16, psize0=8, nlev=3)
    nlev = max(p[0] for p in patches) + 1
    st = {l: inputs.mhd_wave(3, 16 << l, "fast", amp=1e-2, v0=(0.3, -0.2, 0.25)).state[0] for l in range(nlev)}
    return inputs.Problem("rand3d", 3, (16, 16, 16), patches, nlev, st)


def run(pb, precision, steps, **opts):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    ctx.set_option(A.OPT_ADVANCE, 3)
    for k, v in opts.items():
        ctx.set_option(getattr(A, k), v)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    dts = ctx.step(steps)
    return ctx, np.asarray(dts)


def assert_same(pb, a, b):
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
@pytest.mark.parametrize("zlen", [1, 3, 8])
def test_zchunk_equals_whole_column(precision, zlen):
    pb = three_level_3d()
    assert pb.nlev == 3
    ref, dref = run(pb, precision, 3, OPT_ZCHUNK=0)
    got, dgot = run(pb, precision, 3, OPT_ZCHUNK=zlen)
    assert np.array_equal(dref, dgot)
    assert_same(pb, ref, got)
    for l in range(pb.nlev):
        for kind in (0, 1):
            t, z = got.tile_choice(l, kind)
            assert z == zlen and 0 <= t <= 4


def test_zchunk_strict_fp64_against_oracle():
    """Chunks of 3 planes in strict FP64 against the oracle (<= 1e-12), dt
    sequence equal bit for bit."""
    pb = three_level_3d()
    ctx, dts = run(pb, A.FP64, 3, OPT_ZCHUNK=3)
    o = oracle_for(pb)
    odts = np.array([o.step() for _ in range(3)])
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("tile", [2, 3, 4])
def test_zchunk_direct_halo_and_tiles(tile):
    """A one-level periodic level of equal patches (halo read straight from the
    neighbour patches) with chunks of 5 planes, per tile variant, mixed
    precision: the unsplit result bit for bit."""
    pb = inputs.blast_3d(32, 16)
    ref, dref = run(pb, A.MIXED, 3, OPT_TILE=tile, OPT_ZCHUNK=0)
    got, dgot = run(pb, A.MIXED, 3, OPT_TILE=tile, OPT_ZCHUNK=5)
    assert np.array_equal(dref, dgot)
    assert_same(pb, ref, got)


def test_autotune_chooses_a_chunk_and_keeps_results():
    """The autotuner's (tile, z chunk) choice per level and sub-step kind is a
    listed pair, and stepping with it gives the result of the 16x8 tile
    (the same as any z chunk) within FP32 rounding."""
    pb = three_level_3d()
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=A.MIXED, stream=s.cuda_stream)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    ctx.autotune(2)
    for l in range(pb.nlev):
        for kind in ((0, 1) if l > 0 else (0,)):
            t, z = ctx.tile_choice(l, kind)
            assert 0 <= t <= 4 and z in (0, -2, 4, 8, 16), (l, kind, t, z)
    ctx.step(3)
    ref, _ = run(pb, A.MIXED, 3, OPT_TILE=2, OPT_ZCHUNK=0)
    sa, sb = ctx.read_state(), ref.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            x, y = sa[f][p], sb[f][p]
            assert np.abs(x - y).sum() <= 1e-5 * np.abs(y).sum() + 1e-12, (f, p)


def test_tile_choice_errors():
    pb = three_level_3d()
    ctx, _ = run(pb, A.MIXED, 1)
    with pytest.raises(A.AmrmhdError):
        ctx.tile_choice(pb.nlev, 0)
    with pytest.raises(A.AmrmhdError):
        ctx.tile_choice(0, 2)
    with pytest.raises(A.AmrmhdError):
        ctx.set_option(A.OPT_ZCHUNK, -3)
    fp64 = A.context_for(pb, precision=A.FP64)
    assert fp64.tile_choice(0, 0) == (-1, 0)  # staged kernels by default in FP64


@pytest.mark.parametrize("zlen", [3, 8])
def test_zchunk_bounded_domain_with_floors(zlen):
    """The down-scaled shock clump (inflow and outflow boundaries, 3 levels,
    floors on: the recovery's floor instances of the fused kernel), mixed
    precision: chunks give the whole-column result bit for bit, and the floor
    counts agree."""
    pb = inputs.shock_clump_3d_small(16, 3)

    def make(z):
        import torch
        s = torch.cuda.Stream()
        ctx = A.context_for(pb, precision=A.MIXED, strict_fp64=True, stream=s.cuda_stream)
        ctx.set_option(A.OPT_ZCHUNK, z)
        ctx.set_floors(1e-8, 1e-8)
        ctx.alloc_arena()
        torch.cuda.synchronize()
        ctx.load_state(pb.state)
        return ctx

    a, b = make(0), make(zlen)
    da, db = a.step(3), b.step(3)
    assert np.array_equal(da, db)
    assert a.query(A.Q_FLOOR_EVENTS) == b.query(A.Q_FLOOR_EVENTS)
    assert_same(pb, a, b)


def test_tail_halves_uniform_blast_128():
    """AMRMHD_OPT_ZCHUNK -2 on the 128^3 blast (1024 columns of the 16x8 tile,
    3.4 waves at two CTAs per SM): the columns of the last partial wave run as
    two halves each; the result is the whole-column one bit for bit."""
    pb = inputs.blast_3d(128, 16)
    ref, dref = run(pb, A.MIXED, 2, OPT_TILE=2, OPT_ZCHUNK=0)
    got, dgot = run(pb, A.MIXED, 2, OPT_TILE=2, OPT_ZCHUNK=-2)
    assert np.array_equal(dref, dgot)
    assert_same(pb, ref, got)
    assert got.tile_choice(0, 0) == (2, -2)


def test_tail_halves_with_boundary_capture():
    """A refined level of 64 patches of 16^3 (384 columns in its extended
    sub-step, so a partial last wave): the halved columns' boundary fluxes and
    EMFs reach the registers once; the result is the whole-column one bit for
    bit."""
    base = (64, 64, 64)
    p3 = inputs.tile(0, (0, 0, 0), base, 16, 3) + inputs.tile(1, (32, 32, 32), (96, 96, 96), 16, 3)
    pb = inputs.Problem("b3", 3, base, p3, 2, {0: inputs.blast_3d(64, 16).state[0], 1: inputs.blast_3d(128, 16).state[0]})
    ref, dref = run(pb, A.MIXED, 2, OPT_TILE=2, OPT_ZCHUNK=0)
    got, dgot = run(pb, A.MIXED, 2, OPT_TILE=2, OPT_ZCHUNK=-2)
    assert np.array_equal(dref, dgot)
    assert_same(pb, ref, got)
