"""Pins of the oracle's whole advance against what the physics fixes; CPU only.

* a uniform state is preserved exactly on any hierarchy;
* second-order convergence on a linear Alfven wave (closed-form solution);
* constrained transport keeps the discrete div B at round-off on every level;
* composite conservation at round-off across coarse/fine boundaries after reflux;
* Orszag-Tang point symmetry;
* an everywhere-refined hierarchy equals the uniform fine grid bitwise.
"""
import math

import numpy as np
import pytest

from oracle import OracleSim
from paper_1110_1616_gb300 import inputs


def sim_from(pb):
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, gamma=pb.gamma, cfl=pb.cfl)
    s.set_state(pb.state)
    return s


def div_b(st, dim):
    n = st[0].shape[2]
    dx = 1.0 / n
    d = (st[5][:, :, 1:] - st[5][:, :, :-1]) / dx + (st[6][:, 1:, :] - st[6][:, :-1, :]) / dx
    if dim == 3:
        d = d + (st[7][1:, :, :] - st[7][:-1, :, :]) / dx
    return d


def test_uniform_state_preserved_2d_amr():
    pb = inputs.orszag_tang(32, 8, refine=True)
    pb.state = inputs.uniform_state(2, pb.base, pb.patches, pb.nlev, seed=4)
    s = sim_from(pb)
    for _ in range(3):
        s.step()
    st = s.get_state()
    for l in range(pb.nlev):
        dist, _ = s.masks(l)
        reg = dist == 0
        for f in range(5):
            a = st[l][f]
            assert np.all(a[reg] == pb.state[l][f][reg]), (l, f)
        assert np.all(st[l][5][:, :, :-1][reg] == pb.state[l][5][0, 0, 0])
        assert np.all(st[l][6][:, :-1, :][reg] == pb.state[l][6][0, 0, 0])
        assert np.all(st[l][7][reg] == pb.state[l][7][reg])


def test_uniform_state_preserved_3d_amr():
    base = (16, 16, 16)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 24, 24), 8, 3)
    state = inputs.uniform_state(3, base, patches, 2, seed=5)
    s = OracleSim(3, base, patches, 2)
    s.set_state(state)
    for _ in range(2):
        s.step()
    st = s.get_state()
    for l in range(2):
        dist, _ = s.masks(l)
        reg = dist == 0
        for f in range(5):
            assert np.all(st[l][f][reg] == state[l][f][reg]), (l, f)
        for f in (5, 6, 7):
            v = state[l][f].flat[0]
            sl = st[l][f]
            # faces touching the region
            if f == 5:
                m = reg
                assert np.all(sl[:, :, :-1][m] == v)
            elif f == 6:
                assert np.all(sl[:, :-1, :][reg] == v)
            else:
                assert np.all(sl[:-1, :, :][reg] == v)


def alfven_error(n, amp=1e-6, flags=0):
    """Sum over vx, vy, vz, Bz of the L1 error / amplitude after one period."""
    pb = inputs.alfven_2d(n, n // 2, amp)
    s = sim_from(pb)
    s.set_flags(flags)
    T = 1.0 / math.sqrt(2.0)
    t = 0.0
    while t < T * (1 - 1e-14):
        dt = min(s.cfl_dt(), T - t)
        s.step(dt)
        t += dt
    st = s.get_state()[0]
    ex = inputs.alfven_2d_state(n, amp, T)
    err = 0.0
    for f in (1, 2, 3):
        err += np.abs(st[f] / st[0] - ex[f] / ex[0]).mean()
    err += np.abs(st[7] - ex[7]).mean()
    return err / amp


def test_alfven_second_order_unlimited_slopes():
    """With the limiter replaced by the centred slope (oracle switch), the
    predictor + HLLD + CT advance converges at second order on the linear
    Alfven wave (closed-form solution: the translated eigenmode)."""
    e = [alfven_error(n, flags=2) for n in (16, 32, 64)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert min(orders) >= 1.9, (e, orders)


@pytest.mark.slow
def test_alfven_minmod_converges_towards_second_order():
    """With minmod the extrema are clipped, so the L1 order approaches 2 from
    below as the wave is resolved (observed 1.5 at N=32->64, 1.8 at 64->128)."""
    e = [alfven_error(n) for n in (32, 64, 128)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[0] >= 1.4 and orders[1] >= 1.75 and orders[1] > orders[0], (e, orders)


def test_divb_roundoff_ot_amr():
    pb = inputs.orszag_tang(32, 8, refine=True)
    s = sim_from(pb)
    for _ in range(10):
        s.step()
        st = s.get_state()
        for l in range(pb.nlev):
            dist, _ = s.masks(l)
            n = 32 << l
            d = div_b(st[l], 2)
            bmax = max(np.abs(st[l][5]).max(), np.abs(st[l][6]).max())
            assert np.abs(d[dist == 0]).max() <= 1e-13 * bmax * n, l


def test_divb_roundoff_3d_amr():
    base = (16, 16, 16)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 24, 24), 8, 3)
    pb = inputs.blast_3d(16, 8)
    st0 = {0: pb.state[0], 1: inputs.blast_3d(32, 8).state[0]}
    s = OracleSim(3, base, patches, 2)
    s.set_state(st0)
    for _ in range(3):
        s.step()
    st = s.get_state()
    for l in range(2):
        dist, _ = s.masks(l)
        d = div_b(st[l], 3)
        assert np.abs(d[dist == 0]).max() <= 1e-13 * 16 * (2 ** l) * 2


def composite_totals(s, dim):
    st = s.get_state()[0]
    vol = 1.0 / st[0].size
    return np.array([st[f].sum() * vol for f in range(5)])


@pytest.mark.parametrize("refined_seam", [False, True])
def test_composite_conservation_2d(refined_seam):
    """Sum over base cells (after restriction) of rho, m, E is conserved to
    round-off across coarse/fine boundaries thanks to reflux."""
    if not refined_seam:
        pb = inputs.orszag_tang(32, 8, refine=True)
    else:
        # fine quadrant [0, 1/2)^2 touching the periodic seam, smooth random data
        base = (32, 32, 1)
        patches = inputs.tile(0, (0, 0, 0), base, 8, 2) + inputs.tile(1, (0, 0, 0), (32, 32, 1), 8, 2)
        pb = inputs.Problem("seam", 2, base, patches, 2, inputs.random_smooth_2d(32, 2, seed=7))
    s = sim_from(pb)
    s.step()
    ref = composite_totals(s, 2)
    for _ in range(6):
        s.step()
    tot = composite_totals(s, 2)
    scale = np.array([abs(ref[0]), abs(ref[0]), abs(ref[0]), abs(ref[0]), abs(ref[4])])
    assert np.all(np.abs(tot - ref) <= 1e-13 * scale + 1e-15), (tot - ref)


def test_composite_conservation_3d():
    base = (16, 16, 16)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + inputs.tile(1, (8, 8, 8), (24, 16, 24), 8, 3) \
        + inputs.tile(1, (8, 16, 8), (16, 24, 16), 8, 3)
    st0 = {0: inputs.blast_3d(16, 8).state[0], 1: inputs.blast_3d(32, 8).state[0]}
    s = OracleSim(3, base, patches, 2)
    s.set_state(st0)
    s.step()
    ref = composite_totals(s, 3)
    for _ in range(3):
        s.step()
    tot = composite_totals(s, 3)
    assert np.all(np.abs(tot - ref) <= 1e-13 * np.abs(ref).max()), tot - ref


def test_conservation_pin_detects_missing_reflux():
    """Control for the conservation pin: with the cell reflux switched off in
    the oracle (a planted mistake) the composite totals drift far above
    round-off, so the pin is not vacuous."""
    pb = inputs.orszag_tang(32, 8, refine=True)
    s = sim_from(pb)
    s.set_flags(1)
    s.step()
    ref = composite_totals(s, 2)
    for _ in range(4):
        s.step()
    tot = composite_totals(s, 2)
    assert np.abs(tot - ref)[[1, 2, 4]].max() > 1e-9


def test_ot_point_symmetry():
    pb = inputs.orszag_tang(32, 8, refine=True, noise=0.0)
    s = sim_from(pb)
    for _ in range(20):
        s.step()
    st = s.get_state()
    for l in range(pb.nlev):
        rho = st[l][0][0]
        dist, _ = s.masks(l)
        reg = dist[0] == 0
        rrot = rho[::-1, ::-1]
        assert np.abs((rho - rrot)[reg & reg[::-1, ::-1]]).max() <= 1e-10 * rho.max()
        mx = st[l][1][0]
        assert np.abs((mx + mx[::-1, ::-1])[reg & reg[::-1, ::-1]]).max() <= 1e-10 * np.abs(mx).max()
        bx = st[l][5][0][:, :-1]
        # x-face i maps to x-face n - i under the point reflection
        n = bx.shape[1]
        bx_rot = np.roll(bx[::-1, ::-1], 1, axis=1)
        assert np.abs((bx + bx_rot)[reg & reg[::-1, ::-1]]).max() <= 1e-10 * np.abs(bx).max()
        del n


def test_everywhere_refined_equals_uniform():
    """A level 1 that covers the whole periodic domain evolves exactly like a
    uniform fine grid stepped with the same dt/2 sequence (bitwise)."""
    n = 16
    base = (n, n, 1)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 2) + inputs.tile(1, (0, 0, 0), (2 * n, 2 * n, 1), 8, 2)
    state = inputs.random_smooth_2d(n, 2, seed=11)
    s = OracleSim(2, base, patches, 2)
    s.set_state(state)
    u = OracleSim(2, (2 * n, 2 * n, 1), inputs.tile(0, (0, 0, 0), (2 * n, 2 * n, 1), 8, 2), 1)
    u.set_state({0: state[1]})
    for _ in range(4):
        dt0 = s.step()
        u.step(0.5 * dt0)
        u.step(0.5 * dt0)
    a, b = s.get_state()[1], u.get_state()[0]
    for f in range(8):
        assert np.array_equal(a[f], b[f]), f
