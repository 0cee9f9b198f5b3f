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


def owned_mask(pb, l, f):
    """Entries of the whole-level array of field f on level l that some patch
    of the hierarchy stores: the patch interiors for cell fields, their own
    faces (n_d + 1 along the field's direction d) for face fields. Derived
    from the patch list alone, never from the values."""
    n = pb.level_n(l)
    fd = f - 5 if (f >= 5 and not (pb.dim == 2 and f == 7)) else -1
    shp = [n[2], n[1], n[0]]
    if fd >= 0:
        shp[2 - fd] += 1
    m = np.zeros(shp, dtype=bool)
    for (pl, lo, hi) in pb.patches:
        if pl != l:
            continue
        ext = [1 if d == fd else 0 for d in range(3)]
        m[tuple(slice(lo[d], hi[d] + ext[d]) for d in (2, 1, 0))] = True
    return m


def rel_l1(a, b, mask=None):
    """Relative L1 difference of a against b over the entries of mask (every
    entry if None). A NaN or infinity in either array inside the mask gives
    infinity, so a kernel that leaves non-finite values in owned cells cannot
    pass a tolerance."""
    if mask is None:
        mask = np.ones(np.shape(b), dtype=bool)
    x, y = a[mask], b[mask]
    if not (np.all(np.isfinite(x)) and np.all(np.isfinite(y))):
        return float("inf")
    den = np.abs(y).sum()
    num = np.abs(x - y).sum()
    return num / den if den > 0 else num


def compare_states(g, o, pb):
    """Per level and field: relative L1 of the GPU arrays g against the oracle
    arrays o over the cells/faces the patch list owns (owned_mask); any NaN
    there fails. Periodic face copies: the oracle's face N equals face 0."""
    res = {}
    for l in range(pb.nlev):
        for f in range(8):
            res[(l, f)] = rel_l1(g[l][f], o[l][f], owned_mask(pb, l, f))
    return res


def max_err(res):
    return max(res.values())


# ---- adjoint comparisons: whole-level arrays <-> the packed per-patch layout
def _field_dir(pb, f):
    return f - 5 if (f >= 5 and not (pb.dim == 2 and f == 7)) else -1


def _periodic(pb):
    return [True] * 3 if pb.bc is None else [pb.bc[2 * d] == 0 for d in range(3)]


def _unique_index(pb, l, f):
    """For every entry of a whole-level array of field f, the index of the
    stored value behind it (a periodic face array's entry N is entry 0)."""
    n = list(pb.level_n(l))
    fd = _field_dir(pb, f)
    shp = [n[2], n[1], n[0]]
    if fd >= 0:
        shp[2 - fd] += 1
    idx = np.arange(int(np.prod(shp))).reshape(shp)
    if fd >= 0 and _periodic(pb)[fd]:
        sl_last = [slice(None)] * 3
        sl_first = [slice(None)] * 3
        sl_last[2 - fd] = slice(-1, None)
        sl_first[2 - fd] = slice(0, 1)
        idx[tuple(sl_last)] = idx[tuple(sl_first)]
    return idx


def levels_to_packed_seed(ctx, pb, lam):
    """A packed seed (all 8 fields) whose loss sum(seed * copies) equals
    sum over the whole-level arrays of lam * U: the lam of every level-array
    entry that shows the same stored value (a periodic face array's entries 0
    and N) is summed and given to exactly one stored copy (the first patch
    storing it)."""
    parts = []
    for f in range(8):
        fd = _field_dir(pb, f)
        tot, claimed = {}, {}
        for l in lam:
            idx = _unique_index(pb, l, f)
            tot[l] = np.bincount(idx.ravel(), weights=np.asarray(lam[l][f], dtype=np.float64).ravel(),
                                 minlength=idx.size)
            claimed[l] = np.zeros(idx.size, bool)
        for (l, lo, hi) in pb.patches:
            idx = _unique_index(pb, l, f)
            ext = [1 if d == fd else 0 for d in range(3)]
            sl = tuple(slice(lo[d], hi[d] + ext[d]) for d in (2, 1, 0))
            ii = idx[sl].ravel()
            # one copy per stored value: the first occurrence, also within a
            # patch that spans a periodic dimension (it stores faces 0 and N)
            take = np.zeros(ii.size, bool)
            take[np.unique(ii, return_index=True)[1]] = True
            take &= ~claimed[l][ii]
            v = np.where(take, tot[l][ii], 0.0)
            claimed[l][ii] = True
            parts.append(v)
    return np.concatenate(parts)


def packed_grad_to_levels(ctx, pb, g):
    """Sums the per-copy gradients of a packed vector into whole-level arrays
    (every entry holding the derivative with respect to its stored value;
    NaN where no patch stores it)."""
    out = {}
    o = 0
    acc = {}
    for f in range(8):
        fd = _field_dir(pb, f)
        for l in range(pb.nlev):
            idx = _unique_index(pb, l, f)
            acc[(l, f)] = (np.zeros(idx.size), np.zeros(idx.size, bool), idx)
        for (l, lo, hi) in pb.patches:
            ext = [1 if d == fd else 0 for d in range(3)]
            sl = tuple(slice(lo[d], hi[d] + ext[d]) for d in (2, 1, 0))
            tot, seen, idx = acc[(l, f)]
            ii = idx[sl].ravel()
            n = ii.size
            np.add.at(tot, ii, g[o:o + n])
            seen[ii] = True
            o += n
    for l in range(pb.nlev):
        out[l] = []
        for f in range(8):
            tot, seen, idx = acc[(l, f)]
            a = np.where(seen[idx], tot[idx], np.nan)
            out[l].append(a)
    return out
