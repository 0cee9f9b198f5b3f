"""CPU-only checks of the C-ABI library: it builds, loads and exports every
entry point the header declares; the host-side hierarchy builder (neighbours by
inheritance, Sec. 3.1) reproduces the oracle's brute-force integer maps bit for
bit; malformed hierarchies return the documented error codes. No kernel runs."""
import ctypes

import numpy as np
import pytest

from oracle import build_map
from paper_1110_1616_gb300 import amrmhd as A
from paper_1110_1616_gb300 import build as B
from paper_1110_1616_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def test_exports_every_declared_symbol():
    names = A.declared_symbols()
    assert len(names) >= 18
    L = ctypes.CDLL(A.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n


def ctx_for(dim, base, patches, max_level=10, bc=None):
    cfg = A.make_config(dim, base, max_level=max_level, bc=bc)
    c = A.Context(cfg)
    c.set_hierarchy(patches)
    return c


def hierarchies():
    out = [
        ("ot_amr", 2, (32, 32, 1), inputs.orszag_tang(32, 8, refine=True).patches),
        ("seam_quadrant", 2, (32, 32, 1), inputs.tile(0, (0, 0, 0), (32, 32, 1), 8, 2) + inputs.tile(1, (0, 0, 0), (32, 32, 1), 8, 2)),
        ("single_patch_levels", 2, (16, 16, 1), [(0, (0, 0, 0), (16, 16, 1)), (1, (8, 8, 0), (24, 24, 1))]),
        ("everywhere_refined", 2, (16, 16, 1), inputs.tile(0, (0, 0, 0), (16, 16, 1), 8, 2) + [(1, (0, 0, 0), (32, 32, 1))]),
        ("3d_two_boxes", 3, (16, 16, 16), inputs.tile(0, (0, 0, 0), (16, 16, 16), 8, 3)
         + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3) + inputs.tile(1, (8, 16, 8), (16, 24, 16), 8, 3)),
    ]
    for seed in range(4):
        out.append(("rand2d_%d" % seed, 2, (32, 32, 1), inputs.random_hierarchy(2, seed, base=32, nlev=3)))
    for seed in range(2):
        out.append(("rand3d_%d" % seed, 3, (16, 16, 16), inputs.random_hierarchy(3, 10 + seed, base=16, nlev=2)))
    return out


def boundary_hierarchies():
    """Hierarchies whose fine patches touch non-periodic domain sides; bc is
    (x-low, x-high, y-low, y-high, z-low, z-high) with 0 periodic, 1 outflow,
    2 inflow."""
    edge2 = inputs.tile(0, (0, 0, 0), (32, 32, 1), 8, 2) + [
        (1, (0, 8, 0), (16, 40, 1)), (1, (48, 0, 0), (64, 24, 1)), (2, (0, 24, 0), (16, 56, 1))]
    corner3 = inputs.tile(0, (0, 0, 0), (16, 16, 16), 8, 3) + [
        (1, (0, 0, 0), (16, 16, 16)), (1, (16, 0, 16), (32, 8, 32)), (1, (24, 24, 0), (32, 32, 8))]
    out = [
        ("edge2_inflow_outflow", 2, (32, 32, 1), edge2, (2, 1, 0, 0, 0, 0)),
        ("edge2_all_outflow", 2, (32, 32, 1), edge2, (1, 1, 1, 1, 0, 0)),
        ("edge2_y_inflow", 2, (32, 32, 1), edge2, (1, 2, 2, 1, 0, 0)),
        ("corner3_mixed", 3, (16, 16, 16), corner3, (2, 1, 1, 1, 0, 0)),
        ("corner3_all", 3, (16, 16, 16), corner3, (1, 2, 2, 1, 1, 2)),
    ]
    for seed in range(3):
        out.append(("rand2d_bc_%d" % seed, 2, (32, 32, 1), inputs.random_hierarchy(2, 20 + seed, base=32, nlev=3),
                    (2, 1, 1, 1, 0, 0)))
    out.append(("rand3d_bc", 3, (16, 16, 16), inputs.random_hierarchy(3, 30, base=16, nlev=2), (2, 1, 0, 0, 1, 1)))
    return out


HIERS = [h + (None,) for h in hierarchies()] + boundary_hierarchies()


@pytest.mark.parametrize("name,dim,base,patches,bc", HIERS, ids=[h[0] for h in HIERS])
def test_maps_bit_exact_vs_oracle(name, dim, base, patches, bc):
    c = ctx_for(dim, base, patches, bc=bc)
    for which in A.MAPS:
        got = c.export_map(which)
        exp = build_map(dim, base, patches, which, bc=bc)
        assert got.shape == exp.shape, (which, got.shape, exp.shape)
        assert np.array_equal(got, exp), which
    if bc is not None:
        g = c.export_map("ghost_cells")
        assert (g[:, 2] >= 2).any()
        assert ((g[:, 2] == 3).any()) == (2 in bc[:2 * dim])


def test_boundary_config_errors():
    base = (32, 32, 1)
    lvl0 = inputs.tile(0, (0, 0, 0), base, 16, 2)
    for bad in [(0, 1, 0, 0, 0, 0), (3, 1, 0, 0, 0, 0), (-1, -1, 0, 0, 0, 0)]:
        with pytest.raises(A.AmrmhdError) as e:
            ctx_for(2, base, lvl0, bc=bad)
        assert e.value.status == A.EINVAL


def test_error_codes():
    base = (32, 32, 1)
    lvl0 = inputs.tile(0, (0, 0, 0), base, 16, 2)
    # misaligned fine patch
    with pytest.raises(A.AmrmhdError) as e:
        ctx_for(2, base, lvl0 + [(1, (21, 20, 0), (30, 30, 1))])
    assert e.value.status == A.EINVAL
    # overlap on level 1
    with pytest.raises(A.AmrmhdError) as e:
        ctx_for(2, base, lvl0 + [(1, (20, 20, 0), (30, 30, 1)), (1, (24, 24, 0), (34, 34, 1))])
    assert e.value.status == A.EOVERLAP
    # nesting: level 2 box touching the edge of the level-1 region
    with pytest.raises(A.AmrmhdError) as e:
        ctx_for(2, base, lvl0 + [(1, (20, 20, 0), (40, 40, 1)), (2, (40, 40, 0), (48, 48, 1))])
    assert e.value.status == A.ENEST
    # level 0 must tile the domain
    with pytest.raises(A.AmrmhdError) as e:
        ctx_for(2, base, lvl0[:-1])
    assert e.value.status == A.EINVAL
    # level gap
    with pytest.raises(A.AmrmhdError) as e:
        ctx_for(2, base, lvl0 + [(2, (40, 40, 0), (48, 48, 1))])
    assert e.value.status == A.EINVAL
    # an empty patch list
    with pytest.raises(A.AmrmhdError) as e:
        A.Context(A.make_config(2, base)).set_hierarchy([])
    assert e.value.status == A.EINVAL
    # a patch over 2^28 elements per field (rejected before any map is built)
    with pytest.raises(A.AmrmhdError) as e:
        ctx_for(3, (1024, 512, 512), [(0, (0, 0, 0), (1024, 512, 512))])
    assert e.value.status == A.EINVAL and "too large" in str(e.value)
    # calls out of order
    c = A.Context(A.make_config(2, base))
    with pytest.raises(A.AmrmhdError) as e:
        c.fill_ghosts(0, 1)
    assert e.value.status == A.ESTATE
    c.set_hierarchy(lvl0)
    with pytest.raises(A.AmrmhdError) as e:
        c.advance_level(0, 1e-3, 1)
    assert e.value.status == A.ESTATE


def test_nesting_matches_oracle_validation():
    """The library's nesting check and the oracle's agree on random boxes."""
    from oracle import OracleSim
    rng = np.random.default_rng(5)
    base = (32, 32, 1)
    lvl0 = inputs.tile(0, (0, 0, 0), base, 16, 2)
    l1 = [(1, (16, 16, 0), (48, 48, 1))]
    agree = 0
    for _ in range(40):
        a = int(rng.integers(14, 44)) * 2
        b = int(rng.integers(14, 44)) * 2
        w = int(rng.integers(2, 8)) * 2
        p2 = [(2, (a, b, 0), (min(a + w, 128), min(b + w, 128), 1))]
        try:
            OracleSim(2, base, lvl0 + l1 + p2)
            ok_o = True
        except ValueError:
            ok_o = False
        try:
            ctx_for(2, base, lvl0 + l1 + p2)
            ok_l = True
        except A.AmrmhdError:
            ok_l = False
        assert ok_o == ok_l, p2
        agree += 1
    assert agree == 40


def test_query_counts():
    pb = inputs.orszag_tang(64, 16, refine=True)
    c = A.context_for(pb)
    assert c.query(A.Q_NPATCH) == 32
    assert c.query(A.Q_NLEVEL) == 2
    assert c.query(A.Q_CELLS) == 64 * 64 + 64 * 64
    assert c.query(A.Q_CELL_UPDATES_PER_STEP) == 64 * 64 + 2 * 64 * 64
    assert c.query(A.Q_ARENA_BYTES) > 0


def regrid_cases():
    out = []
    rng = np.random.default_rng(12)
    for seed in range(3):
        patches = inputs.random_hierarchy(2, 40 + seed, base=32, nlev=3)
        out.append(("rand2d_%d" % seed, 2, (32, 32, 1), patches, None))
    out.append(("clumps2d", 2, (32, 32, 1), inputs.clumps_2d(32, 3).patches, None))
    out.append(("bounded2d", 2, (32, 32, 1), inputs.clumps_2d(32, 3).patches, (2, 1, 1, 1, 0, 0)))
    out.append(("rand3d", 3, (16, 16, 16), inputs.random_hierarchy(3, 50, base=16, nlev=2), None))
    # fine levels well inside the domain: the clustering works on the region's
    # bounding box there
    out.append(("clumps3d", 3, (32, 32, 32), inputs.clumps_3d_small(32, 3).patches, None))
    out.append(("clumps3d_bounded", 3, (32, 32, 32), inputs.clumps_3d_small(32, 3).patches, (1, 1, 2, 1, 1, 1)))
    return out


@pytest.mark.parametrize("name,dim,base,patches,bc", regrid_cases(), ids=[c[0] for c in regrid_cases()])
def test_regrid_clustering_bit_exact_vs_oracle(name, dim, base, patches, bc):
    """The library's host clustering (steps 2-4 of the regrid) and the oracle's
    give the same boxes, in the same order, for the same flagged cells: random
    sparse flags, clustered flags and all-flagged levels."""
    from oracle import OracleSim
    c = ctx_for(dim, base, patches, bc=bc)
    o = OracleSim(dim, base, patches, bc=bc)
    nlev = max(p[0] for p in patches) + 1
    rng = np.random.default_rng(hash(name) % 1000)
    for l in range(nlev):
        n = [base[d] << l if d < dim else 1 for d in range(3)]
        sets = [np.stack([rng.integers(0, n[d], size=40) for d in range(3)], axis=1)]
        centre = [rng.integers(0, n[d]) for d in range(3)]
        blob = np.array([[(centre[0] + a) % n[0], (centre[1] + b) % n[1], (centre[2] + cc) % n[2] if dim == 3 else 0]
                         for a in range(-6, 7) for b in range(-6, 7) for cc in (range(-3, 4) if dim == 3 else [0])])
        sets.append(blob)
        full = np.array([[i, j, k] for k in range(n[2]) for j in range(n[1]) for i in range(n[0])])
        sets.append(full)
        for fl in sets:
            fl = fl.astype(np.int32)
            if dim == 2:
                fl[:, 2] = 0
            got = c.regrid_boxes(l, fl)
            exp = o.regrid_boxes(l, fl)
            assert np.array_equal(got, exp), (l, got[:4], exp[:4])


def test_launch_shape_options_and_async_calls_on_the_host():
    """The fused advance's launch shape as the options set it (no device
    needed: the choice is host state), and the stream-ordered step and sync
    refused before an arena is bound."""
    base = (32, 32, 32)
    patches = inputs.tile(0, (0, 0, 0), base, 16, 3) + inputs.tile(1, (16, 16, 16), (48, 48, 48), 16, 3)
    c = A.Context(A.make_config(3, base, precision=A.MIXED))
    with pytest.raises(A.AmrmhdError) as e:
        c.tile_choice(0, 0)  # no hierarchy yet
    assert e.value.status == A.ESTATE
    c.set_hierarchy(patches)
    assert c.tile_choice(0, 0) == (2, 0) and c.tile_choice(1, 1) == (2, 0)  # 16x8, whole columns
    c.set_option(A.OPT_TILE, 3)
    c.set_option(A.OPT_ZCHUNK, -2)
    assert c.tile_choice(1, 0) == (3, -2)
    c.set_option(A.OPT_ZCHUNK, 8)
    assert c.tile_choice(1, 1) == (3, 8)
    for bad in ((2, 0), (0, 2), (-1, 0)):
        with pytest.raises(A.AmrmhdError) as e:
            c.tile_choice(*bad)
        assert e.value.status == A.EINVAL
    for bad in (-3, 4097):
        with pytest.raises(A.AmrmhdError) as e:
            c.set_option(A.OPT_ZCHUNK, bad)
        assert e.value.status == A.EINVAL
    with pytest.raises(A.AmrmhdError) as e:
        c.step_async(1)
    assert e.value.status == A.ESTATE
    with pytest.raises(A.AmrmhdError) as e:
        c.sync()
    assert e.value.status == A.ESTATE
    f = A.Context(A.make_config(3, base))  # FP64: the staged kernels by default
    f.set_hierarchy(patches)
    assert f.tile_choice(0, 0) == (-1, 0)
    f.set_option(A.OPT_ADVANCE, 3)  # the fused kernel in FP64: the 8x8 tile by default
    assert f.tile_choice(0, 0) == (3, 0)
