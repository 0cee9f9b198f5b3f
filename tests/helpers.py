"""Shared helpers for the parity tests (no method arithmetic: running the two
implementations on the same inputs and comparing their outputs)."""
import numpy as np

from oracle import OracleSim


def oracle_for(pb):
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, lo=pb.lo, hi=pb.hi, gamma=pb.gamma, cfl=pb.cfl,
                  bc=pb.bc, inflow=pb.inflow)
    s.set_state(pb.state)
    return s


def gpu_level_arrays(ctx, pb):
    """Places the library's per-patch interiors into whole-level arrays (NaN
    where no patch owns the cell or face)."""
    per = ctx.read_state()
    out = {}
    for l in range(pb.nlev):
        n = pb.level_n(l)
        arrs = []
        for f in range(8):
            shp = [n[2], n[1], n[0]]
            fd = f - 5 if (f >= 5 and not (pb.dim == 2 and f == 7)) else -1
            if fd >= 0:
                shp[2 - fd] += 1
            arrs.append(np.full(shp, np.nan))
        out[l] = arrs
    for p, (l, lo, hi) in enumerate(pb.patches):
        for f in range(8):
            fd = f - 5 if (f >= 5 and not (pb.dim == 2 and f == 7)) else -1
            ext = [1 if d == fd else 0 for d in range(3)]
            sl = tuple(slice(lo[d], hi[d] + ext[d]) for d in (2, 1, 0))
            out[l][f][sl] = per[f][p]
    return out


def rel_l1(a, b):
    """Relative L1 difference over entries where both are defined."""
    m = ~np.isnan(a) & ~np.isnan(b)
    den = np.abs(b[m]).sum()
    num = np.abs(a[m] - b[m]).sum()
    return num / den if den > 0 else num


def compare_states(g, o, pb):
    """Per level and field: relative L1 of the GPU arrays g against the oracle
    arrays o on the cells/faces the GPU owns. Periodic face copies: the oracle's
    face N equals face 0."""
    res = {}
    for l in range(pb.nlev):
        for f in range(8):
            res[(l, f)] = rel_l1(g[l][f], o[l][f])
    return res


def max_err(res):
    return max(res.values())
