"""Pins of the oracle's time step (reading R6: dt0 = CFL / max_l (2^-l max over
the level's cells of sum_d (|v_d| + c_f,d) / dx_d)) and of its
conservative-to-primitive recovery; CPU only.

The fast speed c_f,d is taken here as the largest characteristic speed of
the primitive quasi-linear matrix A_d(W) minus v_d: the matrix is probed
column by column from the oracle's predictor (whose eigenstructure is pinned
to the closed forms in test_oracle_waves.py) and its eigenvalues computed by
numpy, so the expected dt does not use the oracle's fast-speed formula.
The recovery is pinned by a round trip through the definition of the total
energy, E = p / (gamma - 1) + rho |v|^2 / 2 + |B|^2 / 2, on random states, and
by one cell computed by hand (tests/golden/closed_forms.json).
"""
import json
import math
import os

import numpy as np

from oracle import OracleSim
from oracle import oracle as O
from paper_1110_1616_gb300 import inputs

GAMMA = 5.0 / 3.0
HERE = os.path.dirname(os.path.abspath(__file__))


def a_matrix(w, d):
    """A_d(w) (8 x 8), column j = A_d(w) e_j from the predictor with s_d = e_j."""
    A = np.zeros((8, 8))
    for j in range(8):
        x = np.zeros(8 + 8 * 3)
        x[:8] = w
        x[8 + 8 * d + j] = 1.0
        h = [0.0, 0.0, 0.0]
        h[d] = 1.0
        A[:, j] = w - O.predict(3, x, h)
    return A


def rate(w, dx, dim):
    """sum_d (|v_d| + c_f,d) / dx_d with c_f,d = max eigenvalue of A_d - v_d."""
    r = 0.0
    for d in range(dim):
        lam = np.linalg.eigvals(a_matrix(w, d)).real.max()
        r += (abs(w[1 + d]) + (lam - w[1 + d])) / dx[d]
    return r


def prim(rho, v, p, b):
    return np.array([rho, v[0], v[1], v[2], p, b[0], b[1], b[2]], dtype=np.float64)


def test_fast_speed_is_the_largest_characteristic_speed():
    rng = np.random.default_rng(3)
    for _ in range(20):
        w = prim(rng.uniform(0.1, 5), rng.uniform(-2, 2, 3), rng.uniform(0.01, 3), rng.uniform(-2, 2, 3))
        for d in range(3):
            t, u = (d + 1) % 3, (d + 2) % 3
            lam = np.linalg.eigvals(a_matrix(w, d)).real.max()
            cf = O.fast_speed(w[0], w[4], w[5 + d], w[5 + t], w[5 + u], GAMMA)
            assert abs((lam - w[1 + d]) - cf) <= 1e-12 * cf


def set_uniform(s, dim, base, nlev, w, overrides=()):
    """Whole-level arrays of the uniform primitive state w on every level;
    overrides: (level, (i, j, k), w_cell) changes the cell fields of one cell
    (same B, so the faces stay uniform)."""
    state = inputs.uniform_state(dim, base, [], nlev)
    for l in range(nlev):
        for f in range(8):
            state[l][f] = np.array(state[l][f], dtype=np.float64)
        u = inputs.conserved(w)
        for f in range(5):
            state[l][f][...] = u[f]
        for f in range(5, 8):
            state[l][f][...] = w[f]
    for (l, (i, j, k), wc) in overrides:
        u = inputs.conserved(wc)
        for f in range(5):
            state[l][f][k, j, i] = u[f]
    s.set_state(state)


def test_cfl_uniform_state_closed_form():
    w = prim(1.2, (0.4, -0.7, 0.2), 0.8, (0.6, -0.3, 0.9))
    for dim, base in ((2, (32, 16, 1)), (3, (16, 8, 8))):
        patches = inputs.tile(0, (0, 0, 0), base, 8, dim)
        s = OracleSim(dim, base, patches, 1, cfl=0.4)
        set_uniform(s, dim, base, 1, w)
        dx = [1.0 / base[d] for d in range(3)]
        expect = 0.4 / rate(w, dx, dim)
        assert abs(s.cfl_dt() - expect) <= 1e-13 * expect


def test_cfl_two_states_on_two_levels():
    """The maximum runs over every valid cell of every level with the level's
    rate scaled by 2^-l; a faster state in one fine cell sets dt as if it were
    a coarse cell of the same state, and values outside the fine region do not
    count."""
    dim, base = 2, (16, 16, 1)
    patches = inputs.tile(0, (0, 0, 0), base, 8, dim) + inputs.tile(1, (8, 8, 0), (24, 24, 1), 8, dim)
    wa = prim(1.0, (0.2, 0.1, 0.0), 0.6, (0.5, 0.4, 0.3))
    wb = prim(0.7, (-1.5, 0.8, 0.3), 2.5, (0.5, 0.4, 0.3))   # faster, inside the fine region
    wc = prim(0.1, (9.0, 9.0, 0.0), 50.0, (0.5, 0.4, 0.3))   # fastest, outside the fine region
    dx0 = [1.0 / 16, 1.0 / 16, 1.0]
    dx1 = [1.0 / 32, 1.0 / 32, 1.0]
    # fine cell (10, 12) is inside [8, 24)^2; fine cell (2, 3) is not
    s = OracleSim(dim, base, patches, 2, cfl=0.4)
    set_uniform(s, dim, base, 2, wa, overrides=[(1, (10, 12, 0), wb), (1, (2, 3, 0), wc)])
    expect = 0.4 / max(rate(wa, dx0, dim), 0.5 * rate(wb, dx1, dim))
    assert abs(s.cfl_dt() - expect) <= 1e-13 * expect
    assert abs(0.5 * rate(wb, dx1, dim) - rate(wb, dx0, dim)) <= 1e-13 * rate(wb, dx0, dim)
    # the same fast state in a covered coarse cell counts as well
    s2 = OracleSim(dim, base, patches, 2, cfl=0.4)
    set_uniform(s2, dim, base, 2, wa, overrides=[(0, (5, 6, 0), wc)])
    expect2 = 0.4 / rate(wc, dx0, dim)
    assert abs(s2.cfl_dt() - expect2) <= 1e-13 * expect2


def test_recovery_round_trip():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        rho = math.exp(rng.uniform(-4, 4))
        v = rng.uniform(-3, 3, 3)
        p = math.exp(rng.uniform(-4, 3))
        b = rng.uniform(-3, 3, 3)
        u = np.array([rho, rho * v[0], rho * v[1], rho * v[2],
                      p / (GAMMA - 1.0) + 0.5 * rho * (v @ v) + 0.5 * (b @ b)])
        w = O.recover(u, b, GAMMA)
        assert w[0] == rho
        assert np.all(np.abs(w[1:4] - v) <= 4e-16 * np.abs(v) + 1e-300)
        assert np.array_equal(w[5:8], b)
        # the energy balance cancels: the error is a few ulp of E
        assert abs(w[4] - p) <= 8 * 2.0 ** -52 * (GAMMA - 1.0) * u[4], (w[4], p, u[4])


def test_recovery_hand_computed_cell():
    g = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))["recovery_cell"]
    w = O.recover(g["u"], g["bc"], g["gamma"])
    assert np.allclose(w, g["w"], rtol=1e-15, atol=0.0), (w, g["w"])
