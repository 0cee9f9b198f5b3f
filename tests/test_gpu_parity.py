"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs, plus properties that hold at any size.

Tolerances: FP64 (strict build, no FMA contraction) must match the oracle to
1e-12 relative L1 per field (it is expected to be bitwise identical; the dt
sequence must be bitwise identical since the CFL maximum is order-free). The
mixed FP32 path must be within 1e-5 relative L1 per field on smooth problems.
"""
import math

import numpy as np
import pytest

from helpers import compare_states, gpu_level_arrays, max_err, oracle_for, owned_mask
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


def gpu_for(pb, precision=A.FP64, strict=True, graph=True, baseline=False):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=strict, stream=s.cuda_stream)
    if not graph:
        ctx.set_option(A.OPT_GRAPH, 0)
    if baseline:
        ctx.set_option(A.OPT_ADVANCE, 1)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


def run_both(pb, nsteps, precision=A.FP64, strict=True):
    ctx = gpu_for(pb, precision, strict)
    dts = ctx.step(nsteps)
    o = oracle_for(pb)
    odts = np.array([o.step() for _ in range(nsteps)])
    return ctx, dts, o, odts


def test_ot_amr_fp64_config1_full():
    """2D Orszag-Tang, 64^2 base in 16^2 patches + one refined level over the
    central 32^2 base cells, seeded noise 1e-3, 50 coarse steps, FP64."""
    pb = inputs.orszag_tang(64, 16, refine=True, noise=1e-3, seed=1)
    ctx, dts, o, odts = run_both(pb, 50)
    assert np.array_equal(dts, odts), np.abs(dts - odts).max()
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("case", ["ot2d_one_128_patch", "ot2d_amr_64_patches", "blast3d_one_64_patch"])
def test_wide_patches(case):
    """Patches wider than a fill chunk (64 positions): ghost rows of more than
    64 cells are split into several chunks along x, and a single periodic patch
    is its own neighbour on every side. FP64 strict against the oracle."""
    if case == "ot2d_one_128_patch":
        pb, n = inputs.orszag_tang(128, 128, refine=False), 10
    elif case == "ot2d_amr_64_patches":
        pb, n = inputs.orszag_tang(128, 64, refine=True), 4
    else:
        pb, n = inputs.blast_3d(64, 64), 3
    ctx, dts, o, odts = run_both(pb, n)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_blast3d_fp64_reduced():
    """3D blast (config-2 physics) at 32^3 in 16^3 patches, 30 steps, FP64."""
    pb = inputs.blast_3d(32, 16)
    ctx, dts, o, odts = run_both(pb, 30)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_3d_amr_fp64():
    base = (16, 16, 16)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3) \
        + inputs.tile(1, (8, 16, 8), (16, 24, 16), 8, 3)
    st = {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]}
    pb = inputs.Problem("blast3d_amr", 3, base, patches, 2, st)
    ctx, dts, o, odts = run_both(pb, 8)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_hierarchy_2d_fp64(seed):
    patches = inputs.random_hierarchy(2, seed, base=32, nlev=3)
    nlev = max(p[0] for p in patches) + 1
    pb = inputs.Problem("rand2d", 2, (32, 32, 1), patches, nlev, inputs.random_smooth_2d(32, nlev, seed=seed))
    ctx, dts, o, odts = run_both(pb, 6)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_random_hierarchy_3d_fp64():
    patches = inputs.random_hierarchy(3, 10, base=16, nlev=2)
    st = {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]}
    pb = inputs.Problem("rand3d", 3, (16, 16, 16), patches, 2, st)
    ctx, dts, o, odts = run_both(pb, 4)
    assert np.array_equal(dts, odts)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_ot_amr_fp64_fast_build():
    """FP64 with FMA contraction allowed: still within 1e-12 of the oracle."""
    pb = inputs.orszag_tang(64, 16, refine=True)
    ctx, dts, o, odts = run_both(pb, 20, strict=False)
    assert np.allclose(dts, odts, rtol=1e-13, atol=0)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_mixed_smooth_amr_within_1e5():
    """Mixed precision (FP32 stencil, FP64 recovery/registers/dt) against the
    FP64 oracle on a smooth 2D problem with a refined quadrant across the
    periodic seam: relative L1 per field <= 1e-5."""
    base = (64, 64, 1)
    patches = inputs.tile(0, (0, 0, 0), base, 16, 2) + inputs.tile(1, (0, 0, 0), (64, 64, 1), 16, 2)
    pb = inputs.Problem("smooth_quadrant", 2, base, patches, 2, inputs.random_smooth_2d(64, 2, seed=3))
    ctx, dts, o, odts = run_both(pb, 20, precision=A.MIXED)
    assert np.allclose(dts, odts, rtol=1e-5)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-5, res


def test_mixed_alfven_within_1e5():
    """A finite-amplitude (0.1) circularly polarised Alfven wave: smooth, and
    every field's magnitude is set by the wave rather than by round-off."""
    pb = inputs.alfven_2d(64, 16, amp=1e-1)
    ctx, dts, o, odts = run_both(pb, 40, precision=A.MIXED)
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-5, res


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_uniform_state_preserved(precision):
    pb = inputs.orszag_tang(32, 8, refine=True)
    pb.state = inputs.uniform_state(2, pb.base, pb.patches, pb.nlev, seed=4)
    ctx = gpu_for(pb, precision)
    ctx.step(3)
    g = gpu_level_arrays(ctx, pb)
    for l in range(pb.nlev):
        for f in range(8):
            a = g[l][f][owned_mask(pb, l, f)]
            v = pb.state[l][f].flat[0]
            if precision == A.MIXED:
                v = np.float32(v)
            assert a.size > 0 and np.all(a == v), (l, f)


def composite(ctx, pb):
    g = gpu_level_arrays(ctx, pb)[0]
    vol = 1.0 / g[0].size
    return np.array([np.nansum(g[f]) * vol for f in range(5)])


def test_conservation_across_cf_boundaries_fp64():
    pb = inputs.orszag_tang(64, 16, refine=True)
    ctx = gpu_for(pb, A.FP64, strict=False)
    ctx.step(1)
    ref = composite(ctx, pb)
    ctx.step(10)
    tot = composite(ctx, pb)
    scale = np.abs(ref).max()
    assert np.all(np.abs(tot - ref) <= 1e-13 * scale), tot - ref


def test_divb_roundoff_gpu():
    pb = inputs.orszag_tang(64, 16, refine=True)
    for precision, tol in ((A.FP64, 1e-13), (A.MIXED, 1e-5)):
        ctx = gpu_for(pb, precision)
        ctx.step(10)
        per = ctx.read_state()
        for p, (l, lo, hi) in enumerate(pb.patches):
            bx, by = per[5][p][0], per[6][p][0]
            n = 64 << l
            d = (bx[:, 1:] - bx[:, :-1]) * n + (by[1:, :] - by[:-1, :]) * n
            bmax = max(np.abs(bx).max(), np.abs(by).max())
            assert np.abs(d).max() <= tol * bmax * n, (precision, p)


def test_graph_equals_direct_calls():
    """The captured coarse step equals the same sequence of C-ABI calls
    (fill, advance, reflux/restrict in the order 0,1,1) bitwise."""
    pb = inputs.orszag_tang(32, 8, refine=True)
    a = gpu_for(pb, A.FP64)
    a.step(3)
    b = gpu_for(pb, A.FP64)
    for _ in range(3):
        dt = b.cfl_dt()
        b.fill_ghosts(0, 1)
        b.advance_level(0, dt, 1)
        b.fill_ghosts(1, 1)
        b.advance_level(1, dt * 0.5, 1)
        b.fill_ghosts(1, 2)
        b.advance_level(1, dt * 0.5, 2)
        b.reflux_restrict(1)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)


def test_one_patch_per_launch_baseline_equals_batched():
    pb = inputs.orszag_tang(32, 8, refine=True)
    a = gpu_for(pb, A.FP64)
    a.step(3)
    b = gpu_for(pb, A.FP64, baseline=True, graph=False)
    b.step(3)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)


def test_nonphysical_state_reported():
    pb = inputs.orszag_tang(32, 8, refine=False)
    pb.state[0][4] = pb.state[0][4].copy()
    pb.state[0][4][0, 3, 3] = -1.0  # negative total energy -> negative pressure
    ctx = gpu_for(pb, A.FP64)
    with pytest.raises(A.AmrmhdError) as e:
        ctx.cfl_dt()
    assert e.value.status == A.ENONPHYS


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_blast3d_full_size_sampled(precision):
    """Config-2 size (128^3, 512 patches of 16^3) in the launch configuration
    the benchmark times: after one graph step, sampled cells (interior, patch
    corners and edges, across the periodic seam) equal the oracle's one-by-one
    update of those cells from the same state and dt."""
    pb = inputs.blast_3d(128, 16)
    ctx = gpu_for(pb, precision, strict=True)
    dt = ctx.step(1)[0]
    g = gpu_level_arrays(ctx, pb)[0]
    rng = np.random.default_rng(0)
    pts = [(0, 0, 0), (127, 127, 127), (15, 16, 17), (63, 64, 64), (64, 63, 50), (31, 0, 127), (50, 50, 50)]
    pts += [tuple(int(x) for x in rng.integers(0, 128, 3)) for _ in range(40)]
    o = oracle_for(pb)
    o.step_targets(dt, pts)
    ost = o.get_state()[0]
    tol = 1e-12 if precision == A.FP64 else 1e-5
    for (i, j, k) in pts:
        for f in range(5):
            ov, gv = ost[f][k, j, i], g[f][k, j, i]
            assert abs(gv - ov) <= tol * (abs(ov) + 1e-30) + (0 if precision == A.FP64 else 1e-6), (i, j, k, f, gv, ov)
        for f, (a, b, c) in ((5, (i, j, k)), (6, (i, j, k)), (7, (i, j, k))):
            ov, gv = ost[f][c, b, a], g[f][c, b, a]
            assert abs(gv - ov) <= tol * (abs(ov) + 1e-30) + (0 if precision == A.FP64 else 1e-6), (i, j, k, f, gv, ov)


def test_blast3d_full_size_invariants():
    """Config-2 size in the benchmark's launch configuration (mixed precision,
    fused advance reading its halo from the neighbour patches, one graph per
    coarse step), 10 coarse steps: every stored value finite, mass, momentum
    and energy conserved on the periodic domain to FP32 round-off, and div B
    of every cell at round-off (properties that hold at any size; the sampled
    test above compares values with the oracle)."""
    pb = inputs.blast_3d(128, 16)
    ctx = gpu_for(pb, A.MIXED, strict=True)
    ctx.step(1)
    g0 = gpu_level_arrays(ctx, pb)[0]
    ctx.step(10)
    g = gpu_level_arrays(ctx, pb)[0]
    for f in range(8):
        assert np.all(np.isfinite(g[f])), f
    n = 128
    for f in range(5):
        t0, t1 = np.sum(g0[f], dtype=np.float64), np.sum(g[f], dtype=np.float64)
        scale = np.sum(np.abs(g0[f]), dtype=np.float64) + np.sum(np.abs(g0[0]), dtype=np.float64) * 1e-3
        assert abs(t1 - t0) <= 2e-6 * scale, (f, t0, t1)
    bx, by, bz = g[5], g[6], g[7]  # face arrays (z, y, x+1), (z, y+1, x), (z+1, y, x)
    d = (bx[:, :, 1:] - bx[:, :, :-1]) + (by[:, 1:, :] - by[:, :-1, :]) + (bz[1:, :, :] - bz[:-1, :, :])
    bmax = max(np.abs(bx).max(), np.abs(by).max(), np.abs(bz).max())
    assert np.abs(d).max() <= 1e-5 * bmax, np.abs(d).max() / bmax


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_fused_equals_staged_3d_amr(precision):
    """The fused 3D advance (option 3) and the staged kernels (option 2) give
    the same result on a 3D AMR hierarchy: bitwise in the strict FP64 build
    (registers recomputed from the state vs read from the staged scratch),
    within FP32 rounding in mixed precision."""
    base = (16, 16, 16)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3) \
        + inputs.tile(1, (8, 16, 8), (16, 24, 16), 8, 3)
    st = {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]}
    pb = inputs.Problem("blast3d_amr", 3, base, patches, 2, st)
    import torch
    out = []
    for opt in (3, 2):
        s = torch.cuda.Stream()
        ctx = A.Context(A.make_config(3, base, precision=precision, strict_fp64=True), s.cuda_stream)
        ctx.set_option(A.OPT_ADVANCE, opt)
        ctx.set_hierarchy(patches)
        ctx.alloc_arena()
        torch.cuda.synchronize()
        ctx.load_state(pb.state)
        ctx.step(4)
        out.append(ctx.read_state())
    for f in range(8):
        for p in range(len(patches)):
            a, b = out[0][f][p], out[1][f][p]
            if precision == A.FP64:
                assert np.array_equal(a, b), (f, p, np.abs(a - b).max())
            else:
                assert np.abs(a - b).sum() <= 1e-5 * np.abs(b).sum() + 1e-12, (f, p)


def run_opts(pb, precision, steps, **opts):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    for k, v in opts.items():
        ctx.set_option(getattr(A, k), v)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


@pytest.mark.parametrize("graph", [1, 0])
def test_concurrent_levels_equal_serial(graph):
    """Running each finer level's sub-steps concurrently with the coarser
    advance (side streams, joined before the reflux) changes nothing, bitwise:
    3-level 2D FP64 and 2-level 3D mixed precision."""
    patches = inputs.random_hierarchy(2, 1, base=32, nlev=3)
    nlev = max(p[0] for p in patches) + 1
    pb2 = inputs.Problem("rand3", 2, (32, 32, 1), patches, nlev, inputs.random_smooth_2d(32, nlev, seed=2))
    base = (16, 16, 16)
    p3 = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3)
    pb3 = inputs.Problem("b3", 3, base, p3, 2, {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]})
    for pb, prec in ((pb2, A.FP64), (pb3, A.MIXED)):
        a = run_opts(pb, prec, 4, OPT_CONCURRENT=1, OPT_GRAPH=graph)
        b = run_opts(pb, prec, 4, OPT_CONCURRENT=0, OPT_GRAPH=graph)
        a.step(4)
        b.step(4)
        sa, sb = a.read_state(), b.read_state()
        for f in range(8):
            for p in range(len(pb.patches)):
                assert np.array_equal(sa[f][p], sb[f][p]), (pb.name, f, p)


def test_autotune_picks_a_tile_per_level_and_keeps_results():
    base = (16, 16, 16)
    p3 = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3)
    pb = inputs.Problem("b3", 3, base, p3, 2, {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]})
    a = run_opts(pb, A.MIXED, 3)
    tiles = a.autotune(3)
    assert len(tiles) == 2 and all(0 <= t <= 4 for t in tiles)
    b = run_opts(pb, A.MIXED, 3)
    a.step(3)
    b.step(3)
    sa, sb = a.read_state(), b.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            x, y = sa[f][p], sb[f][p]
            assert np.abs(x - y).sum() <= 1e-5 * np.abs(y).sum() + 1e-12, (f, p)


@pytest.mark.parametrize("tile", [0, 1, 3, 4])
def test_fused_tile_variants_agree(tile):
    """Every fused tile variant (16x16/256, 16x16/512, 8x8, 12x12) gives the
    16x8 variant's result on a 3D AMR hierarchy of 8^3 patches (extended
    sub-steps and partial tiles included): bit for bit with the fused kernel
    in strict FP64 (no FMA contraction), within FP32 rounding in mixed
    precision (the compiler may contract multiply-adds differently per
    variant)."""
    base = (16, 16, 16)
    p3 = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3)
    pb = inputs.Problem("b3", 3, base, p3, 2, {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]})
    for precision in (A.FP64, A.MIXED):
        a = run_opts(pb, precision, 3, OPT_ADVANCE=3, OPT_TILE=tile)
        b = run_opts(pb, precision, 3, OPT_ADVANCE=3, OPT_TILE=2)
        a.step(3)
        b.step(3)
        sa, sb = a.read_state(), b.read_state()
        for f in range(8):
            for p in range(len(pb.patches)):
                x, y = sa[f][p], sb[f][p]
                if precision == A.FP64:
                    assert np.array_equal(x, y), (f, p)
                else:
                    assert np.abs(x - y).sum() <= 1e-5 * np.abs(y).sum() + 1e-12, (f, p)


def test_whole_state_packed_io_round_trip():
    """amrmhd_set_state_all / get_state_all (host pointers) move the same
    values as the per-field packed calls."""
    import ctypes as C
    pb = inputs.orszag_tang(32, 8, refine=True)
    ctx = gpu_for(pb, A.FP64)
    ref = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
    out = np.empty_like(ref)
    ctx._check(A.lib().amrmhd_get_state_all(ctx.h, out.ctypes.data_as(C.c_void_p), 0), "get_all")
    assert np.array_equal(out, ref)
    new = ref * 1.5
    ctx._check(A.lib().amrmhd_set_state_all(ctx.h, new.ctypes.data_as(C.c_void_p), 0), "set_all")
    back = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
    assert np.array_equal(back, new)


@pytest.mark.parametrize("precision", [A.FP64, A.MIXED])
def test_whole_state_io_page_locked_host_memory(precision):
    """With page-locked host buffers (read and written by the packing kernels
    directly, no staging copy) the whole-state I/O moves the same values as
    with ordinary host memory (through the staging buffer)."""
    import ctypes as C
    import torch
    pb = inputs.orszag_tang(32, 8, refine=True)
    ctx = gpu_for(pb, precision)
    ref = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
    pinned = torch.empty(ref.size, dtype=torch.float64).pin_memory()
    ctx._check(A.lib().amrmhd_get_state_all(ctx.h, C.c_void_p(pinned.data_ptr()), 0), "get_all")
    assert np.array_equal(pinned.numpy(), ref)
    new = ref * 1.25
    pinned.copy_(torch.from_numpy(new))
    ctx._check(A.lib().amrmhd_set_state_all(ctx.h, C.c_void_p(pinned.data_ptr()), 0), "set_all")
    back = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
    expect = new if precision == A.FP64 else new.astype(np.float32).astype(np.float64)
    assert np.array_equal(back, expect)


@pytest.mark.parametrize("where", ["device", "pinned"])
def test_whole_state_io_3d_ragged(where):
    """3D, three levels of patches 8 to 16 cells wide (face fields one longer
    along their normal, rows of 8 to 17 elements, row counts not multiples of
    the packing kernel's row batch): the whole-state calls (device pointers, or
    page-locked host memory) move the values of the per-field packed calls,
    both ways."""
    import ctypes as C
    import torch
    patches = inputs.random_hierarchy(3, 5, base=16, psize0=8, nlev=3)
    nlev = max(p[0] for p in patches) + 1
    st = {l: inputs.mhd_wave(3, 16 << l, "fast", amp=1e-2).state[0] for l in range(nlev)}
    pb = inputs.Problem("rand3d", 3, (16, 16, 16), patches, nlev, st)
    ctx = gpu_for(pb, A.FP64)
    ref = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
    if where == "device":
        buf = torch.empty(ref.size, dtype=torch.float64, device="cuda")
        on_dev = 1
    else:
        buf = torch.empty(ref.size, dtype=torch.float64).pin_memory()
        on_dev = 0
    ctx._check(A.lib().amrmhd_get_state_all(ctx.h, C.c_void_p(buf.data_ptr()), on_dev), "get_all")
    torch.cuda.synchronize()
    assert np.array_equal(buf.cpu().numpy(), ref)
    new = ref * 1.5 + 0.25
    buf.copy_(torch.from_numpy(new))
    torch.cuda.synchronize()
    ctx._check(A.lib().amrmhd_set_state_all(ctx.h, C.c_void_p(buf.data_ptr()), on_dev), "set_all")
    back = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
    assert np.array_equal(back, new)


@pytest.mark.parametrize("pinned,staged", [(False, 0), (True, 0), (True, 1)])
def test_whole_state_io_float_elements(pinned, staged):
    """amrmhd_set_state_all_f32 / get_state_all_f32 move the stored FP32 values
    of a mixed-precision context unchanged (page-locked or ordinary host
    memory, in place or through the staging buffer), and round / widen those
    of an FP64 context."""
    import ctypes as C
    import torch
    pb = inputs.orszag_tang(32, 8, refine=True)
    for precision in (A.MIXED, A.FP64):
        ctx = gpu_for(pb, precision)
        ctx.set_option(A.OPT_HOST_IO, staged)
        ref = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
        buf = torch.empty(ref.size, dtype=torch.float32)
        if pinned:
            buf = buf.pin_memory()
        ctx._check(A.lib().amrmhd_get_state_all_f32(ctx.h, C.c_void_p(buf.data_ptr()), 0), "get_all_f32")
        assert np.array_equal(buf.numpy(), ref.astype(np.float32))
        new = (ref * 1.25).astype(np.float32)
        buf.copy_(torch.from_numpy(new))
        ctx._check(A.lib().amrmhd_set_state_all_f32(ctx.h, C.c_void_p(buf.data_ptr()), 0), "set_all_f32")
        back = np.concatenate([ctx.get_field_packed(f) for f in range(8)])
        assert np.array_equal(back, new.astype(np.float64))
