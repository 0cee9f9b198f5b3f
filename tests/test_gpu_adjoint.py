"""GPU discrete adjoint (amrmhd_backward) against the oracle's own adjoint
(a reverse sweep over its operation tape) and against central differences of
the GPU forward; checkpointing, state restoration and torch.autograd.

Tolerances: FP64 (strict build) relative L2 <= 1e-10 against the oracle over
the stored values of all levels; central differences (h = 1e-6 |U0| / |v|,
then h/4 and h/16 when a difference straddles a branch change) within 1e-6
relative.
"""
import numpy as np
import pytest

from helpers import levels_to_packed_seed, oracle_for, packed_grad_to_levels
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


def quadrant_2d(n=16, seed=3):
    base = (n, n, 1)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 2) + inputs.tile(1, (0, 0, 0), (n, n, 1), 8, 2)
    return inputs.Problem("quadrant", 2, base, patches, 2, inputs.random_smooth_2d(n, 2, seed=seed))


def three_level_2d():
    patches = inputs.random_hierarchy(2, 1, base=16, nlev=3, psize0=8)
    nlev = max(p[0] for p in patches) + 1
    return inputs.Problem("rand3", 2, (16, 16, 1), patches, nlev, inputs.random_smooth_2d(16, nlev, seed=6))


def small_3d():
    base = (8, 8, 8)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + [(1, (4, 4, 4), (12, 12, 12))]
    st = {0: inputs.blast_3d(8, 8).state[0], 1: inputs.blast_3d(16, 8).state[0]}
    for l in st:
        st[l][4] = np.where(st[l][4] > 10, st[l][4] * 0.05 + 0.5, st[l][4])
    return inputs.Problem("small3d", 3, base, patches, 2, st)


def bounded_2d():
    return inputs.smooth_bounded_2d(16, refine=True, seed=2)


PROBLEMS = {"quadrant_2d": quadrant_2d, "three_level_2d": three_level_2d, "small_3d": small_3d,
            "bounded_2d": bounded_2d}


def gpu_ctx(pb, precision=A.FP64):
    import torch
    s = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=True, stream=s.cuda_stream)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    return ctx


def gpu_backward(ctx, pb, dts, lam, ckpt):
    import torch
    seed = torch.tensor(levels_to_packed_seed(ctx, pb, lam), dtype=torch.float64, device="cuda")
    g0 = torch.empty_like(seed)
    torch.cuda.synchronize()
    ctx.backward(dts, seed, g0, ckpt)
    return g0.cpu().numpy()


def stored_mask(ctx, pb):
    m = packed_grad_to_levels(ctx, pb, np.ones(ctx.packed_total()))
    return {l: [~np.isnan(a) for a in m[l]] for l in m}


def random_lam(pb, rng, mask):
    return {l: [np.where(mask[l][f], rng.normal(size=a.shape), 0.0) for f, a in enumerate(pb.state[l])]
            for l in pb.state}


def rel_l2(g, o, mask):
    num = den = 0.0
    for l in g:
        for f in range(8):
            m = mask[l][f]
            num += float(((g[l][f][m] - o[l][f][m]) ** 2).sum())
            den += float((o[l][f][m] ** 2).sum())
    return np.sqrt(num / den)


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_adjoint_matches_oracle_fp64(name):
    pb = PROBLEMS[name]()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(3)]
    ctx = gpu_ctx(pb)
    mask = stored_mask(ctx, pb)
    lam = random_lam(pb, np.random.default_rng(7), mask)
    g = packed_grad_to_levels(ctx, pb, gpu_backward(ctx, pb, dts, lam, 2))
    go = oracle_for(pb).backward(dts, lam)
    err = rel_l2(g, go, mask)
    assert err <= 1e-10, err


def test_checkpoint_interval_does_not_change_the_gradient():
    pb = quadrant_2d()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(5)]
    ctx = gpu_ctx(pb)
    mask = stored_mask(ctx, pb)
    lam = random_lam(pb, np.random.default_rng(3), mask)
    res = [gpu_backward(ctx, pb, dts, lam, k) for k in (1, 2, 5)]
    for r in res[1:]:
        assert np.abs(r - res[0]).max() <= 1e-12 * np.abs(res[0]).max()


@pytest.mark.parametrize("name,ckpt", [("quadrant_2d", 2), ("three_level_2d", 5), ("small_3d", 1)])
def test_recorded_backward_equals_backward(name, ckpt):
    """amrmhd_step_dt_ckpt + amrmhd_backward_recorded (the forward's own
    checkpoints, no second forward pass) give amrmhd_backward's gradient (to
    the round-off of the adjoint's atomic accumulations, whose order varies
    from run to run) and leave the initial state; a state change drops the
    record."""
    import torch
    pb = PROBLEMS[name]()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(4)]
    ctx = gpu_ctx(pb)
    before = ctx.read_state()
    mask = stored_mask(ctx, pb)
    lam = random_lam(pb, np.random.default_rng(11), mask)
    g_ref = gpu_backward(ctx, pb, dts, lam, ckpt)
    seed = torch.tensor(levels_to_packed_seed(ctx, pb, lam), dtype=torch.float64, device="cuda")
    g0 = torch.empty_like(seed)
    ctx.step_dt_ckpt(dts, ckpt)
    assert ctx.backward_recorded(seed, g0)
    g_rec = g0.cpu().numpy()
    assert np.abs(g_rec - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
    after = ctx.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(before[f][p], after[f][p])
    # the record is used once, and any state change drops it
    assert not ctx.backward_recorded(seed, g0)
    ctx.step_dt_ckpt(dts, ckpt)
    ctx.step_dt(dts[:1])
    assert not ctx.backward_recorded(seed, g0)
    ctx.step_dt_ckpt(dts, ckpt)
    ctx.load_state(pb.state)
    assert not ctx.backward_recorded(seed, g0)


def test_backward_restores_the_initial_state():
    pb = quadrant_2d()
    ctx = gpu_ctx(pb)
    before = ctx.read_state()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(3)]
    mask = stored_mask(ctx, pb)
    gpu_backward(ctx, pb, dts, random_lam(pb, np.random.default_rng(1), mask), 2)
    after = ctx.read_state()
    for f in range(8):
        for p in range(len(pb.patches)):
            assert np.array_equal(before[f][p], after[f][p])


def test_step_dt_matches_oracle_steps():
    pb = quadrant_2d()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(3)]
    ctx = gpu_ctx(pb)
    ctx.step_dt(dts)
    from helpers import compare_states, gpu_level_arrays, max_err
    res = compare_states(gpu_level_arrays(ctx, pb), o.get_state(), pb)
    assert max_err(res) <= 1e-12, res


def test_central_differences_of_the_gpu_forward():
    import torch
    pb = quadrant_2d()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(3)]
    ctx = gpu_ctx(pb)
    mask = stored_mask(ctx, pb)
    rng = np.random.default_rng(9)
    lam = random_lam(pb, rng, mask)
    seed = levels_to_packed_seed(ctx, pb, lam)
    u0 = np.concatenate([ctx.pack(pb.state, f) for f in range(8)])
    g = gpu_backward(ctx, pb, dts, lam, 3)

    def loss(u):
        t = torch.tensor(u, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ctx.load_packed_all(t)
        ctx.step_dt(dts)
        out = torch.empty_like(t)
        ctx.read_packed_all(out)
        torch.cuda.synchronize()
        return float((out.cpu().numpy() * seed).sum())

    checked = 0
    seen = []
    for trial in range(6):
        # a smooth direction given as whole-level arrays, packed (copies of a face agree)
        vlev = {}
        for l in pb.state:
            vlev[l] = []
            for f, a in enumerate(pb.state[l]):
                idx = np.indices(a.shape, dtype=np.float64)
                ph = rng.uniform(0, 2 * np.pi, size=3)
                k = rng.integers(1, 3, size=3)
                w = np.ones(a.shape)
                for dd in range(3):
                    w = w * np.cos(2 * np.pi * k[dd] * idx[dd] / max(a.shape[dd], 1) + ph[dd])
                vlev[l].append(w * np.abs(a).mean())
        v = np.concatenate([ctx.pack(vlev, f) for f in range(8)])
        h = 1e-6 * np.linalg.norm(u0) / np.linalg.norm(v)
        ad = float((g * v).sum())
        # central differences at h, h/4, h/16: the first two consecutive ones
        # that agree did not straddle a branch change (minmod or HLLD switch)
        fds = [(loss(u0 + hh * v) - loss(u0 - hh * v)) / (2 * hh) for hh in (h, h / 4, h / 16)]
        seen.append((fds, ad))
        for a_, b_ in zip(fds, fds[1:]):
            if abs(a_ - b_) <= 1e-7 * abs(b_):
                assert abs(b_ - ad) <= 1e-6 * abs(ad), (trial, fds, ad)
                checked += 1
                break
    assert checked >= 3, seen


def test_autograd_function_gradient_of_a_density_loss():
    """torch.autograd through amrmhd_backward: loss 0.5 sum over level-0 cells
    of (rho - rho_target)^2, gradient w.r.t. the packed initial state against
    the oracle adjoint of the same loss."""
    import torch
    from paper_1110_1616_gb300.autograd import advance
    pb = quadrant_2d()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(4)]
    final = o.get_state()
    ctx = gpu_ctx(pb)
    u0 = torch.tensor(np.concatenate([ctx.pack(pb.state, f) for f in range(8)]), dtype=torch.float64,
                      device="cuda", requires_grad=True)
    n0 = ctx.packed_size(0)
    # rho of the level-0 patches: the first entries of field 0's packed array
    nl0 = sum(int(np.prod([hi[d] - lo[d] for d in range(2)])) for (l, lo, hi) in pb.patches if l == 0)
    target = torch.tensor(ctx.pack(final, 0)[:nl0] * 1.01, dtype=torch.float64, device="cuda")
    uf = advance(ctx, u0, dts, ckpt_every=2)
    loss = 0.5 * ((uf[:nl0] - target) ** 2).sum()
    loss.backward()
    g = packed_grad_to_levels(ctx, pb, u0.grad.detach().cpu().numpy())
    # the same loss seeded into the oracle adjoint
    lam = {l: [np.zeros_like(a) for a in pb.state[l]] for l in pb.state}
    lam[0][0] = final[0][0] - 1.01 * final[0][0]
    go = oracle_for(pb).backward(dts, lam)
    mask = stored_mask(ctx, pb)
    assert rel_l2(g, go, mask) <= 1e-10
    assert n0 > nl0


def test_mixed_precision_adjoint_close_to_fp64():
    pb = quadrant_2d()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(3)]
    ctx = gpu_ctx(pb, A.MIXED)
    mask = stored_mask(ctx, pb)
    lam = random_lam(pb, np.random.default_rng(7), mask)
    g = packed_grad_to_levels(ctx, pb, gpu_backward(ctx, pb, dts, lam, 2))
    go = oracle_for(pb).backward(dts, lam)
    err = rel_l2(g, go, mask)
    assert err <= 1e-4, err


def test_velocity_gradient_against_central_differences():
    """dL/dv0 (amrmhd_grad_velocity: the backward's dL/dU0 pushed through the
    initial state's dependence on the velocity, rho, p and B held) against
    central differences of the forward in v0: moving v0 by h dv changes the
    momentum by rho h dv and the total energy by rho (h v.dv + h^2 |dv|^2 / 2)."""
    import torch
    from paper_1110_1616_gb300.autograd import velocity_gradient
    pb = quadrant_2d()
    o = oracle_for(pb)
    dts = [o.step() for _ in range(3)]
    ctx = gpu_ctx(pb)
    rng = np.random.default_rng(21)
    n = ctx.packed_size(0)
    u0 = np.concatenate([ctx.pack(pb.state, f) for f in range(8)])
    seed = np.zeros_like(u0)
    seed[:n] = rng.normal(size=n)  # a loss linear in the final density
    s_t = torch.tensor(seed, dtype=torch.float64, device="cuda")
    g0 = torch.empty_like(s_t)
    torch.cuda.synchronize()
    ctx.backward(dts, s_t, g0, 3)
    gv = velocity_gradient(torch.tensor(u0, device="cuda"), g0, n).cpu().numpy()

    def loss(u):
        t = torch.tensor(u, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ctx.load_packed_all(t)
        ctx.step_dt(dts)
        out = torch.empty_like(t)
        ctx.read_packed_all(out)
        torch.cuda.synchronize()
        return float((out.cpu().numpy() * seed).sum())

    rho = u0[:n]
    v = [u0[(1 + c) * n:(2 + c) * n] / rho for c in range(3)]

    def moved(dv, h):
        u = u0.copy()
        for c in range(3):
            u[(1 + c) * n:(2 + c) * n] += rho * h * dv[c]
        u[4 * n:5 * n] += rho * sum(h * v[c] * dv[c] + 0.5 * h * h * dv[c] * dv[c] for c in range(3))
        return u

    checked = 0
    seen = []
    for trial in range(10):
        x = np.arange(n, dtype=np.float64)
        dv = [np.cos(2 * np.pi * (rng.integers(1, 4) * x / n) + rng.uniform(0, 2 * np.pi)) for _ in range(3)]
        # |h dv| up to 1e-6 (velocities of order 0.3); a direction whose
        # differences at h, h/4, h/16 disagree crosses a limiter or HLLD branch
        # change of some cell and is not used
        h = 1e-6 / max(np.abs(np.concatenate(dv)).max(), 1e-30)
        ad = float(sum((gv[c * n:(c + 1) * n] * dv[c]).sum() for c in range(3)))
        fds = [(loss(moved(dv, hh)) - loss(moved(dv, -hh))) / (2 * hh) for hh in (h, h / 4, h / 16)]
        seen.append((fds, ad))
        for a_, b_ in zip(fds, fds[1:]):
            if abs(a_ - b_) <= 1e-6 * abs(b_):
                assert abs(b_ - ad) <= 1e-6 * abs(ad), (trial, fds, ad)
                checked += 1
                break
        if checked >= 3:
            break
    assert checked >= 3, seen
