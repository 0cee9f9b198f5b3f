"""Ghost-fill, register, reflux and restriction maps built on the device
(AMRMHD_OPT_DEVICE_MAPS): the rows equal the host builder's and the oracle's
brute-force maps bit for bit and in the same order, on 2D and 3D hierarchies,
periodic and bounded (outflow and inflow sides), with patches that are their
own periodic neighbours, ghost faces held by two neighbours and coarse-fine
edges shared by several coarse patches; a strict FP64 run on device-built maps
equals the run on host-built maps bit for bit."""
import numpy as np
import pytest

from oracle import build_map
from paper_1110_1616_gb300 import amrmhd as A
from paper_1110_1616_gb300 import inputs
from test_library_cpu import HIERS

pytestmark = pytest.mark.gpu

REGISTER_MAPS = ["cf_faces", "cf_edges", "emf_faces", "restrict_cells", "restrict_faces", "reflux_cells"]
ALL_MAPS = ["ghost_cells", "ghost_faces"] + REGISTER_MAPS


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_1616_gb300 import build
    build.build()


def ctx(dim, base, patches, bc, device):
    c = A.Context(A.make_config(dim, base, max_level=10, bc=bc))
    c.set_option(A.OPT_DEVICE_MAPS, 1 if device else 0)
    c.set_hierarchy(patches)
    return c


def extra_hierarchies():
    three = inputs.random_hierarchy(3, 5, base=16, psize0=8, nlev=3)
    out = [
        ("clumps3d_small", 3, (32, 32, 32), inputs.clumps_3d_small(32, 3).patches, None),
        ("rand3d_3lev", 3, (16, 16, 16), three, None),
        ("rand3d_3lev_bounded", 3, (16, 16, 16), three, (2, 1, 1, 1, 1, 2)),
        ("clumps2d", 2, (32, 32, 1), inputs.clumps_2d(32, 3).patches, None),
    ]
    for seed in range(4):
        out.append(("rand2d_deep_%d" % seed, 2, (16, 16, 1), inputs.random_hierarchy(2, 60 + seed, base=16, nlev=4),
                    None))
    return out


CASES = HIERS + extra_hierarchies()
ORACLE_CASES = {h[0] for h in HIERS}


@pytest.mark.parametrize("name,dim,base,patches,bc", CASES, ids=[h[0] for h in CASES])
def test_device_maps_equal_host_and_oracle(name, dim, base, patches, bc):
    cd = ctx(dim, base, patches, bc, True)
    ch = ctx(dim, base, patches, bc, False)
    nonempty = 0
    for which in ALL_MAPS:
        got, exp = cd.export_map(which), ch.export_map(which)
        assert got.shape == exp.shape, (which, got.shape, exp.shape)
        assert np.array_equal(got, exp), which
        nonempty += len(got) > 0
        if name in ORACLE_CASES:  # (the oracle's brute-force maps are slow on the larger cases)
            assert np.array_equal(got, build_map(dim, base, patches, which, bc=bc)), which
    nlev = max(p[0] for p in patches) + 1
    # restricted cells and faces exist wherever a level has a finer one; the
    # coarse-fine lists wherever the finer level does not cover it all
    assert nonempty >= (4 if nlev > 1 else 2)
    assert cd.query(A.Q_ARENA_BYTES) == ch.query(A.Q_ARENA_BYTES)


def test_single_level_has_no_register_rows():
    c = ctx(3, (16, 16, 16), inputs.tile(0, (0, 0, 0), (16, 16, 16), 8, 3), None, True)
    for which in REGISTER_MAPS:
        assert len(c.export_map(which)) == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_run_on_device_maps_equals_host_maps(dim):
    import torch
    if dim == 3:
        patches = inputs.random_hierarchy(3, 5, base=16, psize0=8, nlev=3)
        nlev = max(p[0] for p in patches) + 1
        st = {l: inputs.mhd_wave(3, 16 << l, "fast", amp=1e-2, v0=(0.3, -0.2, 0.25)).state[0] for l in range(nlev)}
        pb = inputs.Problem("rand3d", 3, (16, 16, 16), patches, nlev, st)
    else:
        pb = inputs.orszag_tang(32, 8, refine=True)
    res = []
    for device in (True, False):
        s = torch.cuda.Stream()
        c = A.context_for(pb, precision=A.FP64, strict_fp64=True, stream=s.cuda_stream)
        c.set_option(A.OPT_DEVICE_MAPS, 1 if device else 0)
        c.set_hierarchy(pb.patches)
        c.alloc_arena()
        torch.cuda.synchronize()
        c.load_state(pb.state)
        res.append((c.step(4), c.read_state()))
    (da, sa), (db, sb) = res
    assert np.array_equal(da, db)
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(sa[f][p], sb[f][p]), (f, p)
