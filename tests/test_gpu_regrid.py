"""GPU regrid (amrmhd_regrid) against the oracle's regrid on the same states:
the new patch lists are identical (integer work, bit-exact) and the
transferred states and the states after further steps agree within 1e-12
relative L1 per field (FP64 strict build); mixed precision conserves the
composite totals and keeps div B at round-off."""
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


def gpu_for(pb, precision=A.FP64):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


def as_problem(pb, patches):
    nlev = max(p[0] for p in patches) + 1
    return inputs.Problem(pb.name, pb.dim, pb.base, [(l, tuple(lo), tuple(hi)) for (l, lo, hi) in patches], nlev,
                          pb.state, gamma=pb.gamma, cfl=pb.cfl, lo=pb.lo, hi=pb.hi, bc=pb.bc, inflow=pb.inflow)


def norm_patches(ps):
    return [(int(l), tuple(int(v) for v in lo), tuple(int(v) for v in hi)) for (l, lo, hi) in ps]


@pytest.mark.parametrize("device_cluster", [1, 0])
@pytest.mark.parametrize("case", ["clumps_2d", "clumps_2d_bounded", "clumps_3d"])
def test_regrid_matches_oracle_fp64(case, device_cluster):
    if case == "clumps_3d":
        pb = inputs.clumps_3d_small(16, 2)
        maxl = 3
    else:
        pb = inputs.clumps_2d(32, 3, b_pert=0.3)
        maxl = 3
        if case == "clumps_2d_bounded":
            pb.bc = (2, 1, 1, 1, 0, 0)
            pb.inflow = inputs.conserved((1.0, 1.0, 0.0, 0.0, 1.0, 2 ** 0.5, 0.0, 0.0))
    ctx = gpu_for(pb)
    # the device path (clustering and maps on the device) and the host path
    ctx.set_option(A.OPT_DEVICE_CLUSTER, device_cluster)
    ctx.set_option(A.OPT_DEVICE_MAPS, -1 if device_cluster else 0)
    o = oracle_for(pb)
    for rnd in range(2):
        dts = ctx.step(2)
        odts = [o.step() for _ in range(2)]
        assert np.array_equal(dts, np.array(odts))
        gp = norm_patches(ctx.regrid(0.1, maxl))
        op = norm_patches(o.regrid(0.1, maxl))
        assert gp == op, (rnd, len(gp), len(op))
        cur = as_problem(pb, gp)
        res = compare_states(gpu_level_arrays(ctx, cur), o.get_state(), cur)
        assert max_err(res) <= 1e-12, (rnd, res)
    dts = ctx.step(2)
    odts = [o.step() for _ in range(2)]
    res = compare_states(gpu_level_arrays(ctx, cur), o.get_state(), cur)
    assert max_err(res) <= 1e-12, res


def test_regrid_mixed_conserves_and_keeps_divb():
    pb = inputs.clumps_2d(32, 3, b_pert=0.3)
    ctx = gpu_for(pb, A.MIXED)
    ctx.step(2)

    def totals(c, p):
        g = gpu_level_arrays(c, p)[0]
        return np.array([np.nansum(g[f]) for f in range(5)]) / g[0].size

    t0 = totals(ctx, pb)
    ps = norm_patches(ctx.regrid(0.1, 3))
    cur = as_problem(pb, ps)
    t1 = totals(ctx, cur)
    scale = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    assert np.all(np.abs(t1 - t0) <= 1e-6 * scale), t1 - t0
    g = gpu_level_arrays(ctx, cur)
    for l in range(cur.nlev):
        n = 32 << l
        bx, by = g[l][5][0], g[l][6][0]
        d = (bx[:, 1:] - bx[:, :-1]) * n + (by[1:, :] - by[:-1, :]) * n
        d = d[~np.isnan(d)]
        assert np.abs(d).max() <= 1e-5 * n * 2, l
    ctx.step(2)


@pytest.mark.parametrize("case", ["clumps3d_32", "clumps3d_32_bounded", "clumps2d_64"])
def test_device_clustering_equals_host(case):
    """The device clustering (flag test, buffer and block marks on the GPU)
    and the host clustering (flag list copied back) give the same patches and
    the same transferred state, for several thresholds, through three levels."""
    if case.startswith("clumps3d"):
        pb = inputs.clumps_3d_small(32, 3)
        if case.endswith("bounded"):
            pb.bc = (1, 1, 2, 1, 1, 1)
            pb.inflow = inputs.conserved((1.0, 1.0, 0.0, 0.0, 1.0, 2 ** 0.5, 0.0, 0.0))
    else:
        pb = inputs.clumps_2d(64, 3, b_pert=0.3)
    for theta in (0.05, 0.1, 0.3):
        res = []
        for dev in (1, 0):
            ctx = gpu_for(pb, A.MIXED)
            ctx.set_option(A.OPT_DEVICE_CLUSTER, dev)
            ctx.step(1)
            ps = norm_patches(ctx.regrid(theta, 4))
            res.append((ps, ctx.read_state()))
        (pa, sa), (pb_, sb) = res
        assert pa == pb_, (theta, len(pa), len(pb_))
        assert len(pa) > len(pb.patches) // 4
        for f in range(8):
            for p in range(len(pa)):
                assert np.array_equal(sa[f][p], sb[f][p]), (theta, f, p)
