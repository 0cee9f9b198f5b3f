"""The adjoint's transposed Jacobians of the HLLD flux and of the half-step
predictor (amrmhd_local_vjp: the hand-written transposes that amrmhd_backward
applies at every face and cell, and the same formulas with forward-mode dual
numbers) against the oracle's tape of its own formulas, row by row, on seeded
states that cover every HLLD case (supersonic, single star with and without a
normal field, double star, degenerate star states).

Tolerance: both sides evaluate the same FP64 formulas without FMA contraction;
the transposes sum the same terms in a different order, so they agree to a few
ulps of the largest term: 1e-12 relative to the row's largest entry. The FP32
transposes of the mixed-precision adjoint (inputs rounded to FP32, the FP32
forward's degenerate-state threshold 1e-6) agree to 1e-4 relative: a few
hundred FP32 operations of unit roundoff 6e-8 give ~1e-6 on most rows, and
the differences of nearly equal wave speeds and star states in the
double-star case amplify that by up to ~20 on these states (1.4e-5)."""
import numpy as np
import pytest

from oracle import oracle as O
from local_vjp_cases import hlld_branch, hlld_cases, predict_cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def A():
    from paper_1110_1616_gb300 import build
    build.build()
    from paper_1110_1616_gb300 import amrmhd
    return amrmhd


def _rel(a, r):
    return np.abs(a - r).max(axis=1) / np.maximum(np.abs(r).max(axis=1), 1e-300)


TOL = {0: 1e-12, 1: 1e-12, 2: 1e-4}


@pytest.mark.parametrize("method", [0, 1, 2])
def test_hlld_transpose_matches_oracle_tape_in_every_case(A, method):
    x, g = hlld_cases(6000, seed=21)
    got = A.local_vjp(0, x, g, method=method)
    ref = np.array([O.hlld_vjp(xi, gi) for xi, gi in zip(x, g)])
    br = np.array([hlld_branch(xi) for xi in x])
    assert (np.bincount(br, minlength=6) >= 200).all(), np.bincount(br, minlength=6)
    err = _rel(got, ref)
    for b in range(6):
        assert err[br == b].max() <= TOL[method], (b, err[br == b].max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("method", [0, 1, 2])
def test_predictor_transpose_matches_oracle_tape(A, dim, method):
    x, g, h = predict_cases(dim, 4000, seed=22 + dim)
    got = A.local_vjp(1, x, g, dim=dim, h=h, method=method)
    ref = np.array([O.predict_vjp(dim, xi, h, gi) for xi, gi in zip(x, g)])
    assert _rel(got, ref).max() <= TOL[method]


def test_local_vjp_rejects_bad_arguments(A):
    x, g = hlld_cases(6, seed=1)
    with pytest.raises(RuntimeError):
        A.local_vjp(2, x, g)
    with pytest.raises(RuntimeError):
        A.local_vjp(1, np.zeros((2, 24)), np.zeros((2, 8)), dim=1, h=[0.1])
    with pytest.raises(RuntimeError):
        A.local_vjp(0, x, g, gamma=1.0)
    assert A.local_vjp(0, np.zeros((0, 15)), np.zeros((0, 7))).shape == (0, 15)
