"""Pins of the oracle's transposed Jacobians of single formulas (the HLLD flux
of Sec. 4's hyperbolic advance and the half-step primitive predictor), which
the GPU test of the adjoint's hand-written transposes compares against.

Independent route: central differences of the oracle's own forward formulas
(oc_hlld, oc_predict) in every direction, g . (f(x + h e_i) - f(x - h e_i)) / 2h.
HLLD is only piecewise smooth: a row counts where the difference quotients at
h and h/4 agree (no branch switch within the stencil) and the two normal
velocities differ (at a tie the wave-speed min/max has a kink that a central
difference averages); every HLLD case with a nonzero-measure region must keep
rows, so a mistake confined to one case (a dropped term, a wrong sign in the
double-star state) still fails. Degenerate star states occur on a set of
measure zero (|e| within 1e-12 of 0), where no difference quotient stays in
the case: there the derivative is the one of the formula the forward takes,
and the GPU test compares the adjoint's transposes with this tape. The predictor is smooth (polynomial in w, s
and 1/rho), so every row counts."""
import numpy as np
import pytest

from oracle import oracle as O
from local_vjp_cases import hlld_branch, hlld_cases, predict_cases


def _hlld(x):
    return O.hlld(x[:7], x[7:14], x[14])


def _fd(fun, x, g, h):
    out = np.zeros(x.size)
    for i in range(x.size):
        e = np.zeros(x.size)
        e[i] = h * max(1.0, abs(x[i]))
        out[i] = g @ (fun(x + e) - fun(x - e)) / (2 * e[i])
    return out


def test_hlld_vjp_matches_central_differences_in_every_case():
    x, g = hlld_cases(600, seed=11)
    kept = np.zeros(6, dtype=int)
    for xi, gi in zip(x, g):
        if xi[1] == xi[8]:
            continue
        a = _fd(_hlld, xi, gi, 1e-5)
        b = _fd(_hlld, xi, gi, 2.5e-6)
        scale = max(1.0, np.abs(b).max())
        if np.abs(a - b).max() > 1e-6 * scale:
            continue  # a branch switch inside the stencil
        r = O.hlld_vjp(xi, gi)
        assert np.abs(r - b).max() <= 2e-7 * scale, (hlld_branch(xi), r, b)
        kept[hlld_branch(xi)] += 1
    assert (kept[:5] >= 20).all(), kept


def test_hlld_vjp_supersonic_is_the_physical_flux_transpose():
    """In the supersonic cases the flux is the upwind state's physical flux,
    so the transpose is zero on the other state and on nothing else."""
    x, g = hlld_cases(120, seed=5)
    for xi, gi in zip(x, g):
        b = hlld_branch(xi)
        if b > 1:
            continue
        r = O.hlld_vjp(xi, gi)
        other = r[7:14] if b == 0 else r[:7]
        assert np.all(other == 0.0)
        side = xi[:7] if b == 0 else xi[7:14]

        def flux_of_side(y):
            return O.mhd_flux(y[:7], y[7])
        ref = _fd(flux_of_side, np.r_[side, xi[14]], gi, 1e-6)
        got = np.r_[r[:7] if b == 0 else r[7:14], r[14]]
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("dim", [2, 3])
def test_predict_vjp_matches_central_differences(dim):
    x, g, h = predict_cases(dim, 60, seed=7)
    for xi, gi in zip(x, g):
        ref = _fd(lambda y: O.predict(dim, y, h), xi, gi, 1e-6)
        r = O.predict_vjp(dim, xi, h, gi)
        assert np.allclose(r, ref, rtol=1e-7, atol=1e-8 * np.abs(ref).max())


def test_predict_is_identity_without_slopes():
    """Zero slopes: wh = w, so J^T g on w is g plus only the terms that
    multiply a slope (none), and the slope part is A_d(w)^T (-h_d g)."""
    x, g, h = predict_cases(3, 5, seed=2)
    for xi, gi in zip(x, g):
        y = xi.copy()
        y[8:] = 0.0
        assert np.array_equal(O.predict(3, y, h), y[:8])
        r = O.predict_vjp(3, y, h, gi)
        assert np.allclose(r[:8], gi, rtol=0, atol=0)
