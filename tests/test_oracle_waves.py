"""Pins of the oracle's half-step predictor (the primitive quasi-linear
matrices A_d(W) of the ideal-MHD equations) and of its whole advance on
compressive waves; CPU only.

* Eigenstructure: for a plane wave along a unit vector n through a uniform
  state, sum_d n_d A_d(W) r = lam r for every characteristic family (fast,
  slow, Alfven, entropy; both directions) with the closed-form speeds and
  eigenvectors of the linearised ideal-MHD equations (inputs.mhd_wave_mode),
  along each axis and along an oblique n, with a background flow: every
  coefficient of every row of A_x, A_y and A_z, including the compressive rows
  (continuity, gamma p div v, total-pressure gradient, B_t dv_n) and the
  z-direction terms, is fixed by these identities.
* Convergence: the advance with the unlimited centred slope (oracle switch)
  converges at second order in L1 on linear fast and slow magnetosonic waves,
  2D oblique and 3D oblique (wave vector 2 pi (1,1,1), background flow), against
  the closed-form solution (the translated eigenmode).
* Controls: a planted mistake in a compressive row (p div v for gamma p div v)
  or in a z-only term (the sign of B_t dv_z/dz, or a dropped dp/dz) makes the
  convergence pin fail, in 3D only for the z-only mistakes.
"""
import math

import numpy as np
import pytest

from oracle import OracleSim
from oracle import oracle as O
from paper_1110_1616_gb300 import inputs

W0 = np.array([1.3, 0.2, -0.3, 0.1, 0.7, 0.9, 0.45, -0.3])  # rho, v, p, B (oblique field)
DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 2, -1.5)]


def a_times(w, khat, r):
    """sum_d khat_d A_d(w) r from the oracle's predictor: with slopes s_d =
    khat_d r and factors h_d = 1, the predictor returns w - sum_d A_d(w) s_d."""
    x = np.concatenate([w, khat[0] * r, khat[1] * r, khat[2] * r])
    return w - O.predict(3, x, [1.0, 1.0, 1.0])


@pytest.mark.parametrize("family", ["fast", "slow", "alfven", "entropy"])
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("khat", DIRS)
def test_predictor_matrix_eigenstructure(family, sign, khat):
    n = np.asarray(khat, dtype=np.float64)
    n = n / np.linalg.norm(n)
    lam, r = inputs.mhd_wave_mode(family, W0[0], W0[4], W0[5:8], n, W0[1:4], sign)
    lhs = a_times(W0, n, r)
    assert np.abs(lhs - lam * r).max() <= 1e-12 * np.abs(r).max() * (abs(lam) + 1.0), (lhs, lam * r)


def test_predictor_matrix_eigenvalues_2d():
    """In 2D (two directions) the in-plane matrices carry the same speeds."""
    for khat in ((1, 0, 0), (0, 1, 0), (0.6, 0.8, 0)):
        n = np.asarray(khat, dtype=np.float64)
        for family in ("fast", "slow", "alfven"):
            lam, r = inputs.mhd_wave_mode(family, W0[0], W0[4], W0[5:8], n, W0[1:4], 1)
            x = np.concatenate([W0, n[0] * r, n[1] * r])
            lhs = W0 - O.predict(2, x, [1.0, 1.0, 0.0])
            assert np.abs(lhs - lam * r).max() <= 1e-12 * np.abs(r).max() * (abs(lam) + 1.0)


def wave_error(dim, n, family, flags=2, v0=(0.0, 0.0, 0.0), frac=0.5):
    """L1 error (sum over the 8 stored fields of the mean |U - U_exact|) per unit
    amplitude after `frac` of a wave period, against the closed-form solution."""
    amp = 1e-6
    pb = inputs.mhd_wave(dim, n, family, amp=amp, v0=v0)
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, gamma=pb.gamma, cfl=pb.cfl)
    s.set_state(pb.state)
    s.set_flags(flags)
    T = frac * 2.0 * math.pi / abs(pb.meta["omega"])
    t = 0.0
    while t < T * (1.0 - 1e-14):
        dt = min(s.cfl_dt(), T - t)
        s.step(dt)
        t += dt
    st = s.get_state()[0]
    ex = inputs.mhd_wave(dim, n, family, amp=amp, t=T, v0=v0).state[0]
    return sum(np.abs(st[f] - ex[f]).mean() for f in range(8)) / amp


def orders(dim, family, ns, flags=2, v0=(0.0, 0.0, 0.0)):
    e = [wave_error(dim, n, family, flags, v0) for n in ns]
    return e, [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]


V2 = (0.3, -0.2, 0.1)
V3 = (0.3, -0.2, 0.25)


@pytest.mark.parametrize("family", ["fast", "slow"])
def test_magnetosonic_second_order_2d_oblique(family):
    """Observed orders (N = 16, 32, 64): fast 2.6, 2.4; slow 2.4, 2.1."""
    e, o = orders(2, family, (16, 32, 64), v0=V2)
    assert min(o) >= 1.9, (e, o)


@pytest.mark.parametrize("family", ["fast", "slow"])
def test_magnetosonic_second_order_3d_oblique(family):
    """Wave vector 2 pi (1,1,1), oblique field, background flow: every
    z-direction term is active. Observed orders (N = 8, 16, 32): fast 2.7,
    2.6; slow 2.6, 2.5."""
    e, o = orders(3, family, (8, 16, 32), v0=V3)
    assert o[-1] >= 1.9, (e, o)


def test_pin_detects_wrong_pressure_coefficient():
    """Control: p div v in place of gamma p div v in the predictor's pressure
    row (oracle flag bit 4) drops the 2D fast wave to first order (observed
    1.0, 0.8), so the pin above fails; the incompressible Alfven wave (div v =
    0) could not see this mistake."""
    e, o = orders(2, "fast", (16, 32, 64), flags=2 | 16, v0=V2)
    assert min(o) < 1.5, (e, o)


@pytest.mark.parametrize("flag", [32, 64])
def test_pin_detects_z_only_mistakes(flag):
    """Controls for the z-direction terms: the sign of the B_t dv_z/dz terms of
    the induction rows flipped (bit 5) or the dp/dz term of the z-momentum
    row dropped (bit 6) leaves every 2D pin unchanged (z terms are inactive
    there) but fails the 3D pin (observed last orders 1.3 and 1.6)."""
    e2, o2 = orders(2, "fast", (16, 32), flags=2 | flag, v0=V2)
    e2r, _ = orders(2, "fast", (16, 32), flags=2, v0=V2)
    assert e2 == e2r  # bitwise: the planted z-term never runs in 2D
    e, o = orders(3, "fast", (8, 16, 32), flags=2 | flag, v0=V3)
    assert o[-1] < 1.7, (e, o)
