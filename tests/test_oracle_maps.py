"""Checks of the oracle's brute-force integer maps against their definitions on
tiny hierarchies (CPU only): every same-level source holds the ghost cell's
position, every prolongation source holds the parent cell, neighbour relations
are symmetric, register lists match the covered masks."""
import numpy as np
import pytest

from oracle import build_map, OracleSim
from paper_1110_1616_gb300 import inputs


def ext(p, dim):
    return [(p[2][d] - p[1][d]) + 9 if d < dim else 1 for d in range(3)]


def unloc(p, L, dim):
    e = ext(p, dim)
    a = L % e[0]
    b = (L // e[0]) % e[1]
    c = L // (e[0] * e[1])
    return [p[1][0] + a - 4, p[1][1] + b - 4, (p[1][2] + c - 4) if dim == 3 else 0]


HIER = [
    (2, (32, 32, 1), inputs.orszag_tang(32, 8, refine=True).patches),
    (2, (32, 32, 1), inputs.random_hierarchy(2, 3, base=32, nlev=3)),
    (3, (16, 16, 16), inputs.tile(0, (0, 0, 0), (16, 16, 16), 8, 3) + inputs.tile(1, (8, 8, 8), (24, 24, 16), 8, 3)),
]


@pytest.mark.parametrize("dim,base,patches", HIER)
def test_ghost_cell_sources(dim, base, patches):
    ok = OracleSim(dim, base, patches)
    assert ok.status == 0
    m = build_map(dim, base, patches, "ghost_cells")
    for (p, Ld, kind, src, Ls) in m:
        P, S = patches[p], patches[src]
        g = unloc(P, Ld, dim)
        gs = unloc(S, Ls, dim)
        lvl = P[0]
        n = [base[d] << lvl if d < dim else 1 for d in range(3)]
        if kind == 0:
            assert S[0] == lvl
            assert all((g[d] - gs[d]) % n[d] == 0 for d in range(dim))
            assert all(S[1][d] <= gs[d] < S[2][d] for d in range(dim))
        else:
            assert kind == 1 and S[0] == lvl - 1
            assert all(((g[d] % n[d]) >> 1) == gs[d] for d in range(dim))
    # count: every patch has (n+8)^dim - n^dim ghost cells
    for p, P in enumerate(patches):
        e = [(P[2][d] - P[1][d]) for d in range(dim)]
        tot = np.prod([x + 8 for x in e]) - np.prod(e)
        assert (m[:, 0] == p).sum() == tot


@pytest.mark.parametrize("dim,base,patches", HIER)
def test_neighbors_symmetric(dim, base, patches):
    m = build_map(dim, base, patches, "neighbors")
    s = set(map(tuple, m.tolist()))
    for (a, b, sx, sy, sz) in s:
        assert (b, a, -sx, -sy, -sz) in s


@pytest.mark.parametrize("dim,base,patches", HIER)
def test_register_lists_match_masks(dim, base, patches):
    sim = OracleSim(dim, base, patches)
    faces = build_map(dim, base, patches, "cf_faces")
    rc = build_map(dim, base, patches, "restrict_cells")
    nl = max(p[0] for p in patches) + 1
    for l in range(1, nl):
        _, cov = sim.masks(l - 1)
        # restriction rows = covered coarse cells (each exactly once)
        assert (rc[:, 0] == l).sum() == cov.sum()
        # C/F faces = faces between covered and uncovered coarse cells
        n = 0
        for d in range(dim):
            ax = 2 - d
            n += (cov != np.roll(cov, 1, axis=ax)).sum()
        assert (faces[:, 0] == l).sum() == n
    refl = build_map(dim, base, patches, "reflux_cells")
    # every C/F face appears in exactly one reflux row
    used = refl[:, 3:].ravel()
    used = used[used >= 0]
    assert sorted(used.tolist()) == list(range(len(faces)))
