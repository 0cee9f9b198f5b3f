"""Pins of the oracle's discrete adjoint (the transpose of the linearised
forward map of whole coarse steps for a fixed dt sequence); CPU only.

The oracle differentiates its own forward code: a reverse sweep over an
operation tape (oracle/ad.hpp) and, independently of it, forward-mode tangents.

* dot-product test: <J v, lam> = <v, J^T lam> to round-off on 2D and 3D AMR
  hierarchies, periodic and bounded;
* central finite differences of the plain FP64 forward along random smooth
  directions match <v, J^T lam> to 1e-6 relative (a direction whose
  differences at h and h/4 disagree straddles a branch change and is redrawn);
* uniform directions: a uniform state stays uniform, so J c = c for a
  direction c that is constant per field on every level, and summing J^T lam
  over such a direction gives the sum of lam;
* the adjoint is linear in lam and zero for lam = 0.
"""
import numpy as np
import pytest

from oracle import OracleSim
from paper_1110_1616_gb300 import inputs

from helpers import oracle_for


def quadrant_2d(n=16, seed=3):
    base = (n, n, 1)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 2) + inputs.tile(1, (0, 0, 0), (n, n, 1), 8, 2)
    return inputs.Problem("quadrant", 2, base, patches, 2, inputs.random_smooth_2d(n, 2, seed=seed))


def small_3d():
    base = (8, 8, 8)
    patches = inputs.tile(0, (0, 0, 0), base, 8, 3) + [(1, (4, 4, 4), (12, 12, 12))]
    st = {0: inputs.blast_3d(8, 8).state[0], 1: inputs.blast_3d(16, 8).state[0]}
    for l in st:  # soften the blast so the problem is smooth
        st[l][4] = np.where(st[l][4] > 10, st[l][4] * 0.05 + 0.5, st[l][4])
    return inputs.Problem("small3d", 3, base, patches, 2, st)


def bounded_2d():
    return inputs.smooth_bounded_2d(16, refine=True, seed=2)


PROBLEMS = {"quadrant_2d": quadrant_2d, "small_3d": small_3d, "bounded_2d": bounded_2d}


def dts_for(pb, n):
    o = oracle_for(pb)
    return [o.step() for _ in range(n)]


def random_like(pb, rng, smooth=False):
    out = {}
    for l, arrs in pb.state.items():
        out[l] = []
        for a in arrs:
            if smooth:
                # low-frequency pattern, plus a small random part
                idx = np.indices(a.shape, dtype=np.float64)
                ph = rng.uniform(0, 2 * np.pi, size=3)
                k = rng.integers(1, 3, size=3)
                v = np.ones(a.shape)
                for d in range(3):
                    v = v * np.cos(2 * np.pi * k[d] * idx[d] / max(a.shape[d], 1) * (1 << 0) + ph[d])
                out[l].append(v * np.abs(a).mean() + 1e-3 * rng.normal(size=a.shape) * np.abs(a).mean())
            else:
                out[l].append(rng.normal(size=a.shape))
    return out


def dot(pb, a, b, dedup):
    """Sum over levels and fields; with dedup the entry N of a periodic face
    array (a copy of entry 0) is left out."""
    per = [True] * 3 if pb.bc is None else [pb.bc[2 * d] == 0 for d in range(3)]
    s = 0.0
    for l in a:
        for f in range(8):
            x, y = a[l][f], b[l][f]
            if dedup and f >= 5 and not (pb.dim == 2 and f == 7) and per[f - 5]:
                sl = [slice(None)] * 3
                sl[2 - (f - 5)] = slice(0, -1)
                x, y = x[tuple(sl)], y[tuple(sl)]
            s += float((x * y).sum())
    return s


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_dot_product(name):
    pb = PROBLEMS[name]()
    dts = dts_for(pb, 2)
    rng = np.random.default_rng(11)
    lam, v = random_like(pb, rng), random_like(pb, rng)
    o = oracle_for(pb)
    g = o.backward(dts, lam)
    jv = o.tangent(dts, v)
    lhs, rhs = dot(pb, jv, lam, False), dot(pb, v, g, True)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0), (lhs, rhs)


def loss_along(pb, dts, lam, v, h):
    st = {l: [a + h * b for a, b in zip(pb.state[l], v[l])] for l in pb.state}
    o = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, lo=pb.lo, hi=pb.hi, gamma=pb.gamma, cfl=pb.cfl, bc=pb.bc,
                  inflow=pb.inflow)
    o.set_state(st)
    for dt in dts:
        o.step(dt)
    return dot(pb, o.get_state(), lam, False)


@pytest.mark.parametrize("name", ["quadrant_2d", "bounded_2d"])
def test_central_differences(name):
    pb = PROBLEMS[name]()
    dts = dts_for(pb, 3)
    rng = np.random.default_rng(5)
    lam = random_like(pb, rng)
    g = oracle_for(pb).backward(dts, lam)
    checked = 0
    for trial in range(6):
        v = random_like(pb, rng, smooth=True)
        norm = np.sqrt(sum(float((x * x).sum()) for l in v for x in v[l]))
        h = 1e-6 * np.sqrt(sum(float((x * x).sum()) for l in pb.state for x in pb.state[l])) / norm
        fd = (loss_along(pb, dts, lam, v, h) - loss_along(pb, dts, lam, v, -h)) / (2 * h)
        fd4 = (loss_along(pb, dts, lam, v, h / 4) - loss_along(pb, dts, lam, v, -h / 4)) / (h / 2)
        if abs(fd - fd4) > 1e-7 * abs(fd):
            continue  # the +-h interval crosses a branch change (a minmod or HLLD switch): redraw
        ad = dot(pb, v, g, True)
        assert abs(fd - ad) <= 1e-6 * abs(ad), (trial, fd, ad)
        checked += 1
    assert checked >= 3


@pytest.mark.parametrize("name", ["quadrant_2d", "small_3d"])
def test_uniform_direction_is_identity(name):
    pb = PROBLEMS[name]()
    pb.state = inputs.uniform_state(pb.dim, pb.base, pb.patches, pb.nlev, seed=8)
    dts = dts_for(pb, 2)
    o = oracle_for(pb)
    for f in range(8):
        c = {l: [np.full(a.shape, 1.0 if k == f else 0.0) for k, a in enumerate(pb.state[l])] for l in pb.state}
        jc = o.tangent(dts, c)
        for l in pb.state:
            for k in range(8):
                assert np.allclose(jc[l][k], c[l][k], rtol=0, atol=1e-12), (f, l, k)
    rng = np.random.default_rng(2)
    lam = random_like(pb, rng)
    g = o.backward(dts, lam)
    for f in range(8):
        c = {l: [np.full(a.shape, 1.0 if k == f else 0.0) for k, a in enumerate(pb.state[l])] for l in pb.state}
        lhs, rhs = dot(pb, c, g, True), dot(pb, c, lam, True)
        # the periodic copies of lam add into the one stored face value
        rhs_full = dot(pb, c, lam, False)
        assert abs(lhs - rhs_full) <= 1e-10 * max(abs(rhs_full), 1.0), (f, lhs, rhs, rhs_full)


def test_linear_in_lambda():
    pb = quadrant_2d()
    dts = dts_for(pb, 2)
    rng = np.random.default_rng(4)
    a, b = random_like(pb, rng), random_like(pb, rng)
    o = oracle_for(pb)
    ga, gb = o.backward(dts, a), o.backward(dts, b)
    ab = {l: [2.0 * x - 3.0 * y for x, y in zip(a[l], b[l])] for l in a}
    gab = o.backward(dts, ab)
    for l in a:
        for f in range(8):
            assert np.allclose(gab[l][f], 2.0 * ga[l][f] - 3.0 * gb[l][f], rtol=1e-12, atol=1e-12)
    zero = {l: [np.zeros_like(x) for x in a[l]] for l in a}
    gz = o.backward(dts, zero)
    assert all(np.all(x == 0) for l in gz for x in gz[l])
