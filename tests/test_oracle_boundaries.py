"""Pins of the oracle's physical boundaries (zero-gradient outflow and fixed
inflow) against what the physics fixes; CPU only.

* a uniform moving state with matching inflow is preserved exactly on
  hierarchies whose fine patches touch the boundaries (2D and 3D);
* a stationary Mach-10 shock (Rankine-Hugoniot jump, closed form) stays in
  place: the supersonic upstream keeps the inflow state exactly and the
  downstream holds the jump state;
* a flow and its mirror image about x = 1/2 (outflow on both sides) stay
  mirror images (a low/high side mix-up in the boundary fill breaks it);
* constrained transport keeps div B at round-off up to the boundaries;
* a planted mistake (inflow state off by one part in 10^3) fails the uniform
  pin, so the pin is not vacuous.
"""
import numpy as np
import pytest

from oracle import OracleSim
from paper_1110_1616_gb300 import inputs


def sim_from(pb, inflow=None):
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, lo=pb.lo, hi=pb.hi, gamma=pb.gamma, cfl=pb.cfl, bc=pb.bc,
                  inflow=pb.inflow if inflow is None else inflow)
    s.set_state(pb.state)
    return s


def edge_hierarchy_2d():
    return inputs.tile(0, (0, 0, 0), (32, 32, 1), 8, 2) + [
        (1, (0, 8, 0), (16, 40, 1)), (1, (48, 0, 0), (64, 24, 1)), (2, (0, 24, 0), (16, 56, 1))]


def corner_hierarchy_3d():
    return inputs.tile(0, (0, 0, 0), (16, 16, 16), 8, 3) + [
        (1, (0, 0, 0), (16, 16, 16)), (1, (16, 0, 16), (32, 8, 32)), (1, (24, 24, 0), (32, 32, 8))]


def uniform_deviation(pb, s, steps):
    for _ in range(steps):
        s.step()
    st = s.get_state()
    dev = 0.0
    for l in range(pb.nlev):
        dist, _ = s.masks(l)
        reg = dist == 0
        for f in range(5):
            ref = pb.state[l][f].flat[0]
            dev = max(dev, np.abs(st[l][f][reg] - ref).max() / max(abs(ref), 1.0))
    return dev


@pytest.mark.parametrize("bc", [(2, 1, 0, 0, 0, 0), (1, 2, 2, 1, 0, 0), (2, 2, 1, 1, 0, 0)])
def test_uniform_flow_preserved_2d(bc):
    pb = inputs.uniform_flow(2, (32, 32, 1), edge_hierarchy_2d(), 3, bc, seed=sum(bc))
    assert uniform_deviation(pb, sim_from(pb), 3) == 0.0


def test_uniform_flow_preserved_3d():
    pb = inputs.uniform_flow(3, (16, 16, 16), corner_hierarchy_3d(), 2, (2, 1, 1, 2, 1, 1), seed=3)
    assert uniform_deviation(pb, sim_from(pb), 2) == 0.0


def test_uniform_pin_detects_wrong_inflow():
    pb = inputs.uniform_flow(2, (32, 32, 1), edge_hierarchy_2d(), 3, (2, 1, 0, 0, 0, 0), seed=2)
    bad = np.array(pb.inflow) * (1.0 + 1e-3)
    assert uniform_deviation(pb, sim_from(pb, inflow=bad), 3) > 1e-5


def totals(st, dim):
    return np.array([st[f].sum() for f in range(5)]) / st[0].size


@pytest.mark.parametrize("dim", [2, 3])
def test_stationary_shock_rankine_hugoniot(dim):
    """The jump of the closed-form Rankine-Hugoniot relations is (up to a
    startup transient of a few per cent) a steady state: the shock keeps its
    cell, the supersonic upstream keeps the inflow state bit for bit, and the
    composite totals stay constant to round-off because the inflow and outflow
    face fluxes of mass, momentum and energy balance across the jump."""
    n = 64 if dim == 2 else 32
    pb = inputs.stationary_shock(dim, n=n, mach=10.0, refine=True)
    s = sim_from(pb)
    ref = totals(s.get_state()[0], dim)
    for _ in range(30 if dim == 2 else 12):
        s.step()
    st = s.get_state()[0]
    rho1, u1, p1 = pb.meta["upstream"]
    rho2, u2, p2 = pb.meta["downstream"]
    rho = st[0][0, 0]
    vx = (st[1] / st[0])[0, 0]
    x = (np.arange(n) + 0.5) / n
    up = x < 0.4
    down = x > 0.5 + 1.0 / n
    assert np.all(rho[up] == rho1) and np.all(vx[up] == u1)
    assert np.abs(rho[down] / rho2 - 1).max() < 5e-2
    assert np.abs(vx[down] / u2 - 1).max() < 3e-2
    # the shock keeps its cell: the one cell between the two states is n/2 - 1
    assert np.all(rho[: n // 2 - 1] == rho1) and np.all(rho[n // 2:] > 0.9 * rho2)
    # the last cells still hold the jump state, so the boundary fluxes balance
    assert np.abs(rho[-4:] / rho2 - 1).max() < 1e-6
    tot = totals(st, dim)
    assert np.all(np.abs(tot - ref) <= 1e-13 * np.abs(ref).max()), tot - ref
    # planar problem: uniform across y (and z)
    assert np.abs(st[0] - st[0][..., :1, :]).max() <= 1e-12 * rho2


def mirror_pair(refine, steps, seed=4, flags=0):
    pa = inputs.smooth_bounded_2d(32, refine=refine, seed=seed)
    pb = inputs.smooth_bounded_2d(32, refine=refine, seed=seed, mirrored=True)
    sa, sb = sim_from(pa), sim_from(pb)
    sa.set_flags(flags)
    sb.set_flags(flags)
    for _ in range(steps):
        dt = sa.step()
        sb.step(dt)
    return pa, sa, sb


def mirror_deviation(flags=0):
    pa, sa, sb = mirror_pair(True, 8, flags=flags)
    A, B = sa.get_state(), sb.get_state()
    sign = (1, -1, 1, 1, 1, -1, 1, 1)
    worst = 0.0
    for l in range(pa.nlev):
        dist, _ = sa.masks(l)
        reg = dist == 0
        for f in range(8):
            a, b = A[l][f], sign[f] * B[l][f][..., ::-1]
            m = reg if a.shape == reg.shape else None
            if f == 5:
                m = np.zeros(a.shape, bool)
                m[..., :-1] |= reg
                m[..., 1:] |= reg
            elif f == 6:
                m = np.zeros(a.shape, bool)
                m[:, :-1, :] |= reg
                m[:, 1:, :] |= reg
            worst = max(worst, np.abs(a - b)[m].max() / np.abs(a).max())
    return worst


def test_mirror_pair_outflow():
    """A flow and its mirror image about x = 1/2 stay mirror images: the
    outflow side of one run is the low-x side of the other, so a low/high
    mix-up in the boundary fill, the boundary faces or the prolongation at the
    boundary breaks the pair."""
    assert mirror_deviation() <= 1e-12


def test_mirror_pin_detects_high_side_face_offset():
    """Control: with an off-by-one planted in the oracle's high-side boundary
    faces the pair separates far above round-off."""
    assert mirror_deviation(flags=4) > 1e-6


def test_mirror_pair_sees_the_boundary():
    """The mirror pin is not vacuous: the flow crosses both x boundaries
    during the test, changing the cells next to them."""
    pa, sa, _ = mirror_pair(False, 8)
    st = sa.get_state()[0]
    assert np.abs(st[0][0][:, 0] - pa.state[0][0][0][:, 0]).max() > 1e-4
    assert np.abs(st[0][0][:, -1] - pa.state[0][0][0][:, -1]).max() > 1e-4


def test_divb_roundoff_bounded():
    pb = inputs.smooth_bounded_2d(32, refine=True, seed=1)
    s = sim_from(pb)
    for _ in range(5):
        s.step()
    for l, st in s.get_state().items():
        dist, _ = s.masks(l)
        n = 32 << l
        d = (st[5][:, :, 1:] - st[5][:, :, :-1]) * n + (st[6][:, 1:, :] - st[6][:, :-1, :]) * n
        bmax = max(np.abs(st[5]).max(), np.abs(st[6]).max())
        assert np.abs(d[dist == 0]).max() <= 1e-13 * bmax * n, l
