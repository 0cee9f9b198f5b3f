"""The allocation-free one-patch advance (amrmhd_advance_patch_noalloc) gives
the same result as the regular entry points on two calls in a row.

Callers that cannot allocate device memory (a memory pool that forbids new
allocations, a real-time loop, a library handed only the state pointers) use
that entry point: it keeps its intermediate arrays in a fixed device array of
the library. The reference here is a one-patch periodic hierarchy advanced
with amrmhd_fill_ghosts + amrmhd_advance_level in mixed precision; the
tolerance is the mixed-precision parity tolerance of the other GPU tests
(1e-5 relative L1 per field). With w = 2 the entry point also updates the two
ghost layers around the interior; on a periodic patch their exact values are
the periodic images of the updated interior, which the regular path gives.
Every element of the output outside the updated region must keep its initial
contents. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1110_1616_gb300 import amrmhd as A
from paper_1110_1616_gb300 import inputs

pytestmark = pytest.mark.gpu


def _fdir(f, dim):
    return f - 5 if (f >= 5 and not (dim == 2 and f == 7)) else -1


def ghosted(interior_fields, dim):
    """Builds the single-patch ghosted layout (extent n+9 per dimension) of a
    periodic patch from its interior cells and owned faces (n+1 faces along d):
    every ghost position takes the value of its periodic image."""
    out = []
    n = interior_fields[0].shape[::-1]  # (nx, ny, nz)
    for f, a in enumerate(interior_fields):
        idx = []
        for d in (2, 1, 0):  # numpy axis order z, y, x
            if d >= dim:
                idx.append(np.zeros(1, dtype=int))
                continue
            idx.append(np.mod(np.arange(-4, n[d] + 5), n[d]))
        out.append(np.ascontiguousarray(a[np.ix_(*idx)]))
    return out


def region(n, dim, f, w):
    """Slices of the ghosted box covering the cells of the interior widened by
    w layers and, for a face field, their faces (one more along its direction)."""
    fd = _fdir(f, dim)
    sl = []
    for d in (2, 1, 0):
        if d >= dim:
            sl.append(slice(0, 1))
        else:
            sl.append(slice(4 - w, 4 + n[d] + w + (1 if d == fd else 0)))
    return tuple(sl)


def periodic_extension(a, n, dim, f, w):
    """The periodic images of the regular path's interior result (cells, or
    faces 0..n_d along d) at the positions of region(n, dim, f, w)."""
    fd = _fdir(f, dim)
    idx = []
    for d in (2, 1, 0):
        if d >= dim:
            idx.append(np.zeros(1, dtype=int))
            continue
        pos = np.arange(-w, n[d] + w + (1 if d == fd else 0))
        idx.append(np.mod(pos, n[d]))
    return a[np.ix_(*idx)]


@pytest.mark.parametrize("w", [0, 2])
@pytest.mark.parametrize("dim", [3, 2])
def test_noalloc_matches_regular_entry_points_two_calls(dim, w):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_1616_gb300 import build
    build.build()
    if dim == 3:
        pb = inputs.blast_3d(16, 16)
    else:
        pb = inputs.orszag_tang(32, 32, refine=False, noise=1e-3, seed=7)
    stream = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=A.MIXED, stream=stream.cuda_stream)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    n = [pb.base[d] for d in range(dim)]
    dx = [1.0 / pb.base[d] for d in range(dim)]
    # current state of the single patch (interior cells, both boundary faces)
    cur = [ctx.get_field(0, f) for f in range(8)]
    for call in range(2):
        dt = ctx.cfl_dt()
        # regular path
        ctx.fill_ghosts(0, 1)
        ctx.advance_level(0, dt, 1)
        torch.cuda.synchronize()
        ref = [ctx.get_field(0, f) for f in range(8)]
        # allocation-free path from the same state; the output buffer starts as
        # a marked copy so that untouched elements can be recognised
        g = ghosted(cur, dim)
        u_in = torch.from_numpy(np.concatenate([x.astype(np.float32).ravel() for x in g])).cuda()
        u_out = torch.full_like(u_in, -12345.0)
        init = u_out.cpu().numpy().copy()
        A.advance_patch_noalloc(u_in, u_out, dim, n, dx, pb.gamma, dt, w, stream.cuda_stream)
        stream.synchronize()
        out = u_out.cpu().numpy()
        fsz = g[0].size
        for f in range(8):
            a = out[f * fsz:(f + 1) * fsz].reshape(g[0].shape).astype(np.float64)
            a0 = init[f * fsz:(f + 1) * fsz].reshape(g[0].shape)
            sl = region(n, dim, f, w)
            got = a[sl]
            exp = periodic_extension(ref[f], n, dim, f, w)
            assert np.all(np.isfinite(got)), (call, f)
            den = np.abs(exp).sum()
            err = np.abs(got - exp).sum() / den if den > 0 else np.abs(got).sum()
            assert err <= 1e-5, (call, f, w, err)
            # nothing outside the updated region is written
            mask = np.ones(a.shape, dtype=bool)
            mask[sl] = False
            assert np.array_equal(a.astype(np.float32)[mask], a0[mask]), (call, f, w)
        cur = ref
