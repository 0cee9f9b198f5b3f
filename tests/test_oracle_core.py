"""Pins of the oracle's per-face and per-cell formulas against what the
mathematics fixes (closed forms, exact solutions, symmetries); CPU only.

The paper prints no worked example for the advance, so every pin here comes
from a property the method is defined to have.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import oracle as O

G = 5.0 / 3.0


def rand_state(rng, bn_scale=1.0):
    # rotated state: rho, un, ut, uu, p, bt, bu
    q = np.array([rng.uniform(0.3, 3), rng.normal(), rng.normal(), rng.normal(), rng.uniform(0.1, 3),
                  rng.normal(), rng.normal()])
    return q


def test_minmod_cases():
    mm = oracle.minmod
    assert mm(1.0, 2.0) == 1.0
    assert mm(2.0, 1.0) == 1.0
    assert mm(-1.0, -3.0) == -1.0
    assert mm(-3.0, -1.0) == -1.0
    assert mm(1.0, -1.0) == 0.0
    assert mm(0.0, 5.0) == 0.0
    assert mm(-2.0, 0.0) == 0.0
    assert mm(1.5, 1.5) == 1.5


def test_fast_speed_limits():
    # no field: sound speed
    assert math.isclose(oracle.fast_speed(2.0, 3.0, 0, 0, 0), math.sqrt(G * 3.0 / 2.0), rel_tol=1e-15)
    # purely transverse field: sqrt((g p + B^2)/rho)
    assert math.isclose(oracle.fast_speed(2.0, 3.0, 0, 1.0, 2.0), math.sqrt((G * 3 + 5.0) / 2.0), rel_tol=1e-15)
    # field along the normal: max(c_s, v_A)
    cs = math.sqrt(G * 0.5 / 1.0)
    assert math.isclose(oracle.fast_speed(1.0, 0.5, 3.0, 0, 0), 3.0, rel_tol=1e-14)
    assert math.isclose(oracle.fast_speed(1.0, 0.5, 0.1, 0, 0), cs, rel_tol=1e-14)


def test_hlld_consistency():
    """F(U, U) = F(U) for any state (consistency of the Riemann solver)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        q = rand_state(rng)
        bn = rng.normal()
        f = oracle.hlld(q, q, bn)
        fe = oracle.mhd_flux(q, bn)
        assert np.allclose(f, fe, rtol=1e-13, atol=1e-13 * np.abs(fe).max())


def test_hlld_supersonic_upwind():
    q = np.array([1.0, 10.0, 0.1, 0.2, 1.0, 0.3, 0.1])
    qr = np.array([0.5, 9.0, -0.1, 0.0, 0.7, -0.2, 0.4])
    assert np.array_equal(oracle.hlld(q, qr, 0.5), oracle.mhd_flux(q, 0.5))
    q2, qr2 = q.copy(), qr.copy()
    q2[1], qr2[1] = -10.0, -9.0
    assert np.array_equal(oracle.hlld(q2, qr2, 0.5), oracle.mhd_flux(qr2, 0.5))


def test_hlld_stationary_contact_exact():
    """An isolated stationary contact (density jump only, Bn != 0) is resolved
    exactly: the flux equals the physical flux of either side."""
    ql = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.7, -0.3])
    qr = np.array([0.125, 0.0, 0.0, 0.0, 1.0, 0.7, -0.3])
    f = oracle.hlld(ql, qr, 0.9)
    fe = oracle.mhd_flux(ql, 0.9)
    assert np.allclose(f, fe, rtol=0, atol=1e-14)
    assert np.allclose(fe, oracle.mhd_flux(qr, 0.9), atol=1e-15)


def test_hlld_stationary_tangential_exact():
    """An isolated stationary tangential discontinuity (Bn = 0, total pressure
    balanced) is resolved exactly."""
    ql = np.array([1.0, 0.0, 0.5, -0.2, 1.0, 1.0, 0.0])
    # p_R + Bt_R^2/2 = p_L + Bt_L^2/2 = 1.5
    qr = np.array([0.3, 0.0, -0.4, 0.8, 1.5 - 0.5 * (0.2 ** 2 + 0.6 ** 2), 0.2, 0.6])
    f = oracle.hlld(ql, qr, 0.0)
    assert np.allclose(f, [0, 1.5, 0, 0, 0, 0, 0], atol=1e-14)


def test_hlld_stationary_rotational_exact():
    """An isolated stationary rotational (Alfven) discontinuity is resolved
    exactly: v_t = -B_t/sqrt(rho), u_n = -Bn/sqrt(rho), |B_t| equal."""
    bn = 1.0
    ql = np.array([1.0, -1.0, -1.0, 0.0, 1.0, 1.0, 0.0])
    qr = np.array([1.0, -1.0, 0.0, -1.0, 1.0, 0.0, 1.0])
    fl, fr = oracle.mhd_flux(ql, bn), oracle.mhd_flux(qr, bn)
    assert np.allclose(fl, fr, atol=1e-15)
    f = oracle.hlld(ql, qr, bn)
    assert np.allclose(f, fl, atol=1e-13)


def test_hlld_mirror_symmetry():
    """x -> -x maps (u, Bn) -> (-u, -Bn); the flux of rho, m_t, E, B_t changes
    sign and the normal momentum flux does not."""
    rng = np.random.default_rng(1)
    sgn = np.array([-1, 1, -1, -1, -1, -1, -1.0])
    for _ in range(200):
        ql, qr = rand_state(rng), rand_state(rng)
        bn = rng.normal()
        f = oracle.hlld(ql, qr, bn)
        mr, ml = qr.copy(), ql.copy()
        mr[1] *= -1
        ml[1] *= -1
        g = oracle.hlld(mr, ml, -bn)
        assert np.allclose(g, sgn * f, rtol=1e-12, atol=1e-12 * np.abs(f).max())


def test_hlld_flux_between_hll_bounds():
    """HLLD's density flux for a Riemann problem lies within the HLL wave-speed
    envelope: it reduces to the physical flux in supersonic states and is
    continuous in Bn through the Bn -> 0 switch."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        ql, qr = rand_state(rng), rand_state(rng)
        f0 = oracle.hlld(ql, qr, 0.0)
        f1 = oracle.hlld(ql, qr, 1e-7)
        assert np.allclose(f0, f1, rtol=1e-4, atol=1e-5)


def test_gs_edge_reduces_to_average_and_linear():
    # uniform: all EMFs equal -> that value
    a = np.full(12, 0.7)
    a[8:] = [1.0, -1.0, 0.0, 2.0]
    assert math.isclose(oracle.gs_edge(a), 0.7, rel_tol=1e-15)
    # E varies linearly in b (cells at integer b, faces at half-integers):
    # the edge value at b - 1/2 is exact whatever the mass fluxes
    beta, b = 0.37, 3.0
    ea_lo, ea_hi = beta * (b - 1), beta * b
    eb = beta * (b - 0.5)
    r00, r10, r01, r11 = beta * (b - 1), beta * (b - 1), beta * b, beta * b
    for fl in [(1, 1, 1, 1), (-1, 2, 0, -3), (0, 0, 0, 0)]:
        v = oracle.gs_edge([ea_lo, ea_hi, eb, eb, r00, r10, r01, r11, *fl])
        assert math.isclose(v, beta * (b - 0.5), rel_tol=1e-14)


def test_gs_edge_upwinding_selects_side():
    """With all mass fluxes positive the derivative terms come from the low
    cells; flipping the high-side references must not change the edge EMF."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        a = rng.normal(size=12)
        a[8:] = [1, 1, 1, 1]
        v1 = oracle.gs_edge(a)
        b = a.copy()
        b[7] += 5.0  # r11 only enters through the high-side (negative-flux) branches
        assert v1 == oracle.gs_edge(b)


def _one_level(dim, n, state):
    base = (n, n, n if dim == 3 else 1)
    from paper_1110_1616_gb300 import inputs
    pt = inputs.tile(0, (0, 0, 0), base, n, dim)
    s = oracle.OracleSim(dim, base, pt, 1)
    s.set_state({0: state})
    return s


def _random_divfree_2d(n, rng):
    """Random cell fields and face B from a random corner potential (div-free)."""
    az = rng.normal(size=(n + 1, n + 1))
    az[-1, :] = az[0, :]
    az[:, -1] = az[:, 0]
    dx = 1.0 / n
    bx = ((az[1:, :] - az[:-1, :]) / dx)[None]
    by = (-(az[:, 1:] - az[:, :-1]) / dx)[None]
    cells = [rng.uniform(0.5, 2.0, size=(1, n, n)) for _ in range(5)] + [None, None, rng.normal(size=(1, n, n))]
    return [cells[0], cells[1], cells[2], cells[3], cells[4], bx, by, cells[7]]


def _random_divfree_3d(n, rng):
    dx = 1.0 / n
    # vector potential on edges; B = curl A on faces (periodic)
    ax = rng.normal(size=(n, n, n))  # A_x at (i, j-1/2, k-1/2) stored [k, j, i]
    ay = rng.normal(size=(n, n, n))
    az = rng.normal(size=(n, n, n))
    r = lambda a, ax_: np.roll(a, -1, axis=ax_)
    bx = (r(az, 1) - az) / dx - (r(ay, 0) - ay) / dx  # at (i-1/2, j, k)
    by = (r(ax, 0) - ax) / dx - (r(az, 2) - az) / dx
    bz = (r(ay, 2) - ay) / dx - (r(ax, 1) - ax) / dx
    pad = lambda a, axis: np.concatenate([a, np.take(a, [0], axis=axis)], axis=axis)
    cells = [rng.uniform(0.5, 2.0, size=(n, n, n)) for _ in range(5)]
    return cells + [pad(bx, 2), pad(by, 1), pad(bz, 0)]


def _div(state, dim, n):
    dx = 1.0 / n
    bx, by, bz = state[5], state[6], state[7]
    d = (bx[:, :, 1:] - bx[:, :, :-1]) / dx + (by[:, 1:, :] - by[:, :-1, :]) / dx
    if dim == 3:
        d = d + (bz[1:, :, :] - bz[:-1, :, :]) / dx
    return d


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_conservative_and_divfree(dim):
    """Children average to the parent (conserved fields and face flux through
    each coarse face), and prolonged face B of a div-free coarse field is
    div-free in every child."""
    rng = np.random.default_rng(10 + dim)
    n = 8
    st = _random_divfree_2d(n, rng) if dim == 2 else _random_divfree_3d(n, rng)
    assert np.abs(_div(st, dim, n)).max() < 1e-10
    c = _one_level(dim, n, st)
    blank = [np.zeros_like(a) for a in (_random_divfree_2d(2 * n, rng) if dim == 2 else _random_divfree_3d(2 * n, rng))]
    f = _one_level(dim, 2 * n, blank)
    O.prolong_all(c, f)
    fs = [f.get_field(0, k) for k in range(8)]
    cs = [c.get_field(0, k) for k in range(8)]
    cell_fields = [0, 1, 2, 3, 4] + ([7] if dim == 2 else [])
    for k in cell_fields:
        a = fs[k]
        if dim == 2:
            avg = 0.25 * (a[0, 0::2, 0::2] + a[0, 0::2, 1::2] + a[0, 1::2, 0::2] + a[0, 1::2, 1::2])
            assert np.allclose(avg, cs[k][0], rtol=1e-14, atol=1e-14)
        else:
            avg = sum(a[z::2, y::2, x::2] for z in (0, 1) for y in (0, 1) for x in (0, 1)) / 8
            assert np.allclose(avg, cs[k], rtol=1e-14, atol=1e-14)
    # fine faces on a coarse face average to it
    if dim == 2:
        assert np.allclose(0.5 * (fs[5][0, 0::2, 0:-1:2] + fs[5][0, 1::2, 0:-1:2]), cs[5][0, :, :-1], atol=1e-12)
        assert np.allclose(0.5 * (fs[6][0, 0:-1:2, 0::2] + fs[6][0, 0:-1:2, 1::2]), cs[6][0, :-1, :], atol=1e-12)
    scale = max(np.abs(fs[5]).max(), np.abs(fs[6]).max()) * 2 * n
    assert np.abs(_div(fs, dim, 2 * n)).max() < 1e-12 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_exact_for_linear(dim):
    """A linear (monotone) field is reproduced exactly by the limited linear
    prolongation when the limiter is inactive (away from the periodic seam)."""
    n = 8
    rng = np.random.default_rng(20 + dim)
    g = rng.uniform(0.5, 1.5, size=3)
    shp = (1, n, n) if dim == 2 else (n, n, n)
    z, y, x = np.meshgrid(*[np.arange(s) + 0.5 for s in shp], indexing="ij")
    lin = 3.0 + g[0] * x + g[1] * y + (g[2] * z if dim == 3 else 0)
    st = [lin.copy() for _ in range(5)]
    if dim == 2:
        st += [np.zeros((1, n, n + 1)), np.zeros((1, n + 1, n)), lin.copy()]
    else:
        st += [np.zeros((n, n, n + 1)), np.zeros((n, n + 1, n)), np.zeros((n + 1, n, n))]
    c = _one_level(dim, n, st)
    fshp = (1, 2 * n, 2 * n) if dim == 2 else (2 * n,) * 3
    blank = [np.zeros(fshp) for _ in range(5)]
    blank += [np.zeros(fshp[:-1] + (fshp[-1] + 1,)), np.zeros((fshp[0], fshp[1] + 1, fshp[2]))]
    blank += [np.zeros(fshp)] if dim == 2 else [np.zeros((fshp[0] + 1, fshp[1], fshp[2]))]
    f = _one_level(dim, 2 * n, blank)
    O.prolong_all(c, f)
    a = f.get_field(0, 0)
    zf, yf, xf = np.meshgrid(*[(np.arange(s) + 0.5) / (2 if s > 1 else 1) for s in fshp], indexing="ij")
    exact = 3.0 + g[0] * xf + g[1] * yf + (g[2] * zf if dim == 3 else 0)
    inner = (slice(None) if dim == 2 else slice(2, -2), slice(2, -2), slice(2, -2))
    assert np.allclose(a[inner], exact[inner], rtol=1e-14, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_is_mean(dim):
    rng = np.random.default_rng(30 + dim)
    n = 4
    fst = _random_divfree_2d(2 * n, rng) if dim == 2 else _random_divfree_3d(2 * n, rng)
    cst = _random_divfree_2d(n, rng) if dim == 2 else _random_divfree_3d(n, rng)
    c = _one_level(dim, n, cst)
    f = _one_level(dim, 2 * n, fst)
    O.restrict_all(c, f)
    rho = c.get_field(0, 0)
    a = f.get_field(0, 0)
    if dim == 2:
        exp = 0.25 * (a[0, 0::2, 0::2] + a[0, 0::2, 1::2] + a[0, 1::2, 0::2] + a[0, 1::2, 1::2])
        assert np.allclose(rho[0], exp, rtol=1e-15)
    else:
        exp = sum(a[z::2, y::2, x::2] for z in (0, 1) for y in (0, 1) for x in (0, 1)) / 8
        assert np.allclose(rho, exp, rtol=1e-15)
    # restricted face B of a div-free fine field is div-free
    cs = [c.get_field(0, k) for k in range(8)]
    scale = np.abs(cs[5]).max() * n
    assert np.abs(_div(cs, dim, n)).max() < 1e-12 * scale


def test_golden_closed_forms_used_by_inputs():
    import json
    import os
    from paper_1110_1616_gb300 import inputs
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
    pb = inputs.orszag_tang(16, 8, refine=False, noise=0.0)
    assert pb.state[0][0].flat[0] == g["orszag_tang_rho"]["value"]
    f = oracle.hlld([1.0, 0.0, 0.5, -0.2, 1.0, 1.0, 0.0], [0.3, 0.0, -0.4, 0.8, 1.3, 0.2, 0.6], 0.0)
    assert abs(f[1] - g["stationary_tangential_total_pressure"]["value"]) < 1e-14
