"""Pins of the oracle's regrid (reading R18: flag, buffer, blocks, proper
nesting, greedy merge into 8-32 cell boxes, transfer by copy where the old fine
level covered the parent cell, else by prolongation, with a divergence-free
closure where copied and prolonged fine faces meet); CPU only.

* the new boxes are aligned to 8 fine cells, 8-32 cells per side, disjoint,
  properly nested (the oracle accepts the hierarchy), and cover every cell
  whose density gradient exceeds the threshold (with margin) wherever nesting
  allows a box;
* composite totals of rho, m, E are unchanged by a regrid (round-off);
* div B stays at round-off on every level after regrids (a control with the
  closure switched off in the oracle breaks it);
* a uniform state stays exactly uniform;
* a second regrid without a step in between reproduces boxes and state bitwise;
* a threshold above every gradient drops the fine levels, conserving the totals.
"""
import numpy as np
import pytest

from oracle import OracleSim
from paper_1110_1616_gb300 import inputs


def clump_sim(nlev=3, steps=2):
    pb = inputs.clumps_2d(32, nlev, b_pert=0.3)
    o = OracleSim(2, pb.base, pb.patches, nlev)
    o.set_state(pb.state)
    for _ in range(steps):
        o.step()
    return pb, o


def totals(o):
    st = o.get_state()[0]
    return np.array([st[f].sum() for f in range(5)]) / st[0].size


def divb_max(o, n0=32):
    out = []
    for l, st in o.get_state().items():
        dist, _ = o.masks(l)
        n = n0 << l
        d = (st[5][:, :, 1:] - st[5][:, :, :-1]) * n + (st[6][:, 1:, :] - st[6][:, :-1, :]) * n
        bmax = max(np.abs(st[5]).max(), np.abs(st[6]).max())
        out.append(np.abs(d[dist == 0]).max() / (bmax * n))
    return max(out)


def test_boxes_are_aligned_sized_disjoint_nested_and_cover_the_flags():
    pb, o = clump_sim()
    theta = 0.1
    before = o.get_state()
    masks = {l: o.masks(l)[0] for l in range(o.nlev)}
    ps = o.regrid(theta, max_levels=3)
    fine = [p for p in ps if p[0] > 0]
    assert fine
    for (l, lo, hi) in fine:
        for d in range(2):
            assert lo[d] % 8 == 0 and hi[d] % 8 == 0
            assert 8 <= hi[d] - lo[d] <= 32
    occ = {}
    for (l, lo, hi) in fine:
        for j in range(lo[1], hi[1]):
            for i in range(lo[0], hi[0]):
                assert (l, i, j) not in occ
                occ[(l, i, j)] = True
    OracleSim(2, pb.base, ps, max(p[0] for p in ps) + 1)  # nesting accepted
    # level-0 cells with a clear gradient far from the level-0 boundary: refined
    rho = before[0][0][0]
    g = np.zeros_like(rho)
    for ax in (0, 1):
        g = np.maximum(g, np.abs(np.roll(rho, -1, ax) - np.roll(rho, 1, ax)) / (2 * rho))
    for j, i in np.argwhere(g > 2 * theta):
        assert (1, 2 * i, 2 * j) in occ


def test_regrid_conserves_composite_totals():
    pb, o = clump_sim()
    for _ in range(3):
        t0 = totals(o)
        o.regrid(0.1, max_levels=3)
        t1 = totals(o)
        scale = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
        assert np.all(np.abs(t1 - t0) <= 1e-14 * scale), t1 - t0
        o.step()
        o.step()


def test_regrid_keeps_divb_at_roundoff():
    pb, o = clump_sim()
    for _ in range(3):
        o.regrid(0.1, max_levels=3)
        assert divb_max(o) <= 1e-14
        o.step()
        o.step()
        assert divb_max(o) <= 1e-14


def test_divb_pin_detects_a_missing_closure():
    pb, o = clump_sim(steps=4)
    o.set_flags(8)
    worst = 0.0
    for _ in range(3):
        o.regrid(0.1, max_levels=3)
        worst = max(worst, divb_max(o))
        o.step()
        o.step()
    assert worst > 1e-8


def test_uniform_state_stays_uniform():
    pb = inputs.clumps_2d(32, 3)
    st = inputs.uniform_state(2, pb.base, pb.patches, 3, seed=2)
    o = OracleSim(2, pb.base, pb.patches, 3)
    o.set_state(st)
    o.step()
    # seed some refinement: regrid keeps the levels (threshold 0 flags nothing in a uniform state)
    o.regrid(-1.0, max_levels=3)
    out = o.get_state()
    for l in out:
        dist, _ = o.masks(l)
        for f in range(5):
            assert np.all(out[l][f][dist == 0] == st[0][f].flat[0])


def test_second_regrid_reproduces_boxes_and_state():
    pb, o = clump_sim()
    p1 = o.regrid(0.1, max_levels=3)
    s1 = o.get_state()
    p2 = o.regrid(0.1, max_levels=3)
    s2 = o.get_state()
    assert p1 == p2
    for l in s1:
        dist, _ = o.masks(l)
        for f in range(8):
            a, b = s1[l][f], s2[l][f]
            if a.shape == dist.shape:
                assert np.array_equal(a[dist == 0], b[dist == 0])


def test_high_threshold_drops_fine_levels():
    pb, o = clump_sim()
    t0 = totals(o)
    ps = o.regrid(1e9, max_levels=3)
    assert all(p[0] == 0 for p in ps) and o.nlev == 1
    assert np.allclose(totals(o), t0, rtol=0, atol=1e-14 * np.abs(t0).max())
