"""The allocation-free one-patch advance (amrmhd_advance_patch_noalloc) gives
the same result as the regular entry points on two calls in a row.

Callers that cannot allocate device memory (a memory pool that forbids new
allocations, a real-time loop, a library handed only the state pointers) use
that entry point: it keeps its intermediate arrays in a fixed device array of
the library. The reference here is a one-patch periodic hierarchy advanced
with amrmhd_fill_ghosts + amrmhd_advance_level in mixed precision; the
tolerance is the mixed-precision parity tolerance of the other GPU tests
(1e-5 relative L1 per field). This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1110_1616_gb300 import amrmhd as A
from paper_1110_1616_gb300 import inputs

pytestmark = pytest.mark.gpu


def ghosted(interior_fields, dim):
    """Builds the single-patch ghosted layout (extent n+9 per dimension) of a
    periodic patch from its interior cells and owned faces (n+1 faces along d)."""
    out = []
    n = interior_fields[0].shape[::-1]  # (nx, ny, nz)
    for f, a in enumerate(interior_fields):
        fd = f - 5 if (f >= 5 and not (dim == 2 and f == 7)) else -1
        idx = []
        for axis, d in ((0, 2), (1, 1), (2, 0)):  # numpy axis -> dimension
            if d >= dim:
                idx.append(np.zeros(1, dtype=int))
                continue
            pos = np.arange(-4, n[d] + 5)
            idx.append(np.mod(pos, n[d]))
        g = a[np.ix_(*idx)] if fd < 0 else a[np.ix_(*idx)]
        # face arrays: positions wrap with period n (entry n equals entry 0)
        out.append(np.ascontiguousarray(g))
    return out


@pytest.mark.parametrize("dim", [3, 2])
def test_noalloc_matches_regular_entry_points_two_calls(dim):
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
        # allocation-free path from the same state
        g = ghosted([c[:, :, :] for c in cur], dim)
        u_in = torch.from_numpy(np.concatenate([x.astype(np.float32).ravel() for x in g])).cuda()
        u_out = u_in.clone()
        A.advance_patch_noalloc(u_in, u_out, dim, n, dx, pb.gamma, dt, 0, stream.cuda_stream)
        stream.synchronize()
        out = u_out.cpu().numpy().astype(np.float64)
        fsz = g[0].size
        got = []
        for f in range(8):
            a = out[f * fsz:(f + 1) * fsz].reshape(g[0].shape)
            fd = f - 5 if (f >= 5 and not (dim == 2 and f == 7)) else -1
            sl = []
            for axis, d in ((0, 2), (1, 1), (2, 0)):
                if d >= dim:
                    sl.append(slice(0, 1))
                else:
                    sl.append(slice(4, 4 + n[d] + (1 if d == fd else 0)))
            got.append(a[tuple(sl)])
        for f in range(8):
            den = np.abs(ref[f]).sum()
            err = np.abs(got[f] - ref[f]).sum() / den if den > 0 else np.abs(got[f]).sum()
            assert err <= 1e-5, (call, f, err)
        cur = ref
