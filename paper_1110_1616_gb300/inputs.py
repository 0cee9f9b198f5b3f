"""Seeded synthetic inputs: patch hierarchies and initial states.

This module holds the workloads only (patch layouts, initial conditions, random
draws); it contains none of the advance's arithmetic. Both the CUDA path and the
CPU oracle take their inputs from here, so each sees identical arrays.

State format: ``{level: [rho, mx, my, mz, E, bx, by, bz]}``; each entry is a
whole-level numpy float64 array over the domain at that level's resolution,
x fastest: cell fields have shape (Nz, Ny, Nx); the face field along d has one
extra entry along d (in a periodic dimension entry N_d repeats entry 0; in a
bounded one it is the high boundary face). In 2D, Nz = 1 and bz is a cell
field.

Boundaries: ``Problem.bc`` lists (x-low, x-high, y-low, y-high, z-low,
z-high) with 0 periodic, 1 zero-gradient outflow, 2 fixed inflow of the
conserved state ``Problem.inflow``; None means periodic everywhere.

Patches are ``(level, lo, hi)`` with half-open level-l cell index boxes
(2D: lo[2] = 0, hi[2] = 1). Patch ids are list positions.
"""
from dataclasses import dataclass, field
import math

import numpy as np

GAMMA = 5.0 / 3.0


@dataclass
class Problem:
    name: str
    dim: int
    base: tuple
    patches: list
    nlev: int
    state: dict
    gamma: float = GAMMA
    cfl: float = 0.4
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    meta: dict = field(default_factory=dict)
    bc: tuple = None      # 6 ints (x-low, x-high, ...): 0 periodic, 1 outflow, 2 inflow
    inflow: tuple = None  # conserved inflow state (rho, mx, my, mz, E, Bx, By, Bz)

    def level_n(self, level):
        return tuple(self.base[d] << level if d < self.dim else 1 for d in range(3))

    def cells_per_coarse_step(self):
        """Work per coarse step: sum over levels of cells x 2^level."""
        tot = 0
        for (l, lo, hi) in self.patches:
            n = 1
            for d in range(self.dim):
                n *= hi[d] - lo[d]
            tot += n << l
        return tot


# ----------------------------------------------------------------- layouts
def tile(level, lo, hi, psize, dim):
    """Tiles the box [lo, hi) of level `level` with patches of edge psize
    (z, y, x order of creation)."""
    out = []
    rng = [range(lo[d], hi[d], psize) if d < dim else range(0, 1) for d in range(3)]
    for k in rng[2]:
        for j in rng[1]:
            for i in rng[0]:
                plo = (i, j, k if dim == 3 else 0)
                phi = (min(i + psize, hi[0]), min(j + psize, hi[1]), min(k + psize, hi[2]) if dim == 3 else 1)
                out.append((level, plo, phi))
    return out


def _cell_centres(n, lo, hi, dim):
    xs = [lo[d] + (np.arange(n[d]) + 0.5) * (hi[d] - lo[d]) / n[d] for d in range(3)]
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return x, y, z


def _faces_from_cells_periodic(a, axis):
    """Face array along `axis` (one extra entry repeating entry 0)."""
    first = np.take(a, [0], axis=axis)
    return np.concatenate([a, first], axis=axis)


def _energy(rho, vx, vy, vz, p, bcx, bcy, bcz, gamma):
    return p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bcx * bcx + bcy * bcy + bcz * bcz)


def _cell_b_from_faces(bx, by, bz, dim):
    bcx = 0.5 * (bx[:, :, :-1] + bx[:, :, 1:])
    bcy = 0.5 * (by[:, :-1, :] + by[:, 1:, :])
    bcz = 0.5 * (bz[:-1, :, :] + bz[1:, :, :]) if dim == 3 else bz
    return bcx, bcy, bcz


def _b_from_az_2d(az_corner, n, dx, dy, periodic=(True, True)):
    """Face B from a corner vector potential A_z of shape (Ny+1, Nx+1). In a
    periodic dimension the copy (entry N along the face normal) is set to
    entry 0 exactly, so that both stored copies of a seam face agree bit for
    bit."""
    bx = (az_corner[1:, :] - az_corner[:-1, :]) / dy  # (Ny, Nx+1)
    by = -(az_corner[:, 1:] - az_corner[:, :-1]) / dx  # (Ny+1, Nx)
    if periodic[0]:
        bx[:, -1] = bx[:, 0]
    if periodic[1]:
        by[-1, :] = by[0, :]
    return bx[None], by[None]


def _state_2d(n, rho, vx, vy, vz, p, bx, by, bz, gamma):
    bcx, bcy, bcz = _cell_b_from_faces(bx, by, bz, 2)
    e = _energy(rho, vx, vy, vz, p, bcx, bcy, bcz, gamma)
    return [rho, rho * vx, rho * vy, rho * vz, e, bx, by, bz]


# ----------------------------------------------------------------- problems
def orszag_tang(n_base=64, psize=16, refine=True, noise=1e-3, seed=1, gamma=GAMMA):
    """2D Orszag-Tang vortex on periodic [0,1]^2 with seeded density noise
    rho (1 + noise U(-1,1)); one static refined level over the central half of
    the base grid (in base cells [n/4, 3n/4)), ratio 2."""
    rng = np.random.default_rng(seed)
    patches = tile(0, (0, 0, 0), (n_base, n_base, 1), psize, 2)
    nlev = 1
    if refine:
        a, b = n_base // 2, 3 * n_base // 2  # level-1 indices of the central half
        patches += tile(1, (a, a, 0), (b, b, 1), psize, 2)
        nlev = 2
    b0 = 1.0 / math.sqrt(4.0 * math.pi)
    state = {}
    for l in range(nlev):
        n = (n_base << l, n_base << l, 1)
        dx = 1.0 / n[0]
        x, y, _ = _cell_centres(n, (0, 0, 0), (1, 1, 1), 2)
        rho = np.full(x.shape, 25.0 / (36.0 * math.pi))
        if noise:
            rho = rho * (1.0 + noise * rng.uniform(-1.0, 1.0, size=x.shape))
        p = np.full(x.shape, 5.0 / (12.0 * math.pi))
        vx = -np.sin(2 * math.pi * y)
        vy = np.sin(2 * math.pi * x)
        vz = np.zeros_like(x)
        xc = np.arange(n[0] + 1) * dx
        yc = np.arange(n[1] + 1) * dx
        Y, X = np.meshgrid(yc, xc, indexing="ij")
        az = b0 * (np.cos(4 * math.pi * X) / (4 * math.pi) + np.cos(2 * math.pi * Y) / (2 * math.pi))
        bx, by = _b_from_az_2d(az, n, dx, dx)
        bz = np.zeros_like(x)
        state[l] = _state_2d(n, rho, vx, vy, vz, p, bx, by, bz, gamma)
    return Problem("orszag_tang_2d", 2, (n_base, n_base, 1), patches, nlev, state, gamma=gamma,
                   meta={"seed": seed, "noise": noise})


def alfven_2d(n=32, psize=16, amp=1e-6, t=0.0, gamma=GAMMA):
    """Circularly polarised linear Alfven wave on periodic [0,1]^2 travelling
    along k = 2 pi (1,1) with B0 = (1,1)/sqrt(2), rho = 1, p = 1/gamma; the
    in-plane perturbation comes from a vector potential so face B is
    divergence-free. The exact solution at time t is the initial state with
    the phase shifted by omega t, omega = |k| v_A, v_A = 1 (period 1/sqrt 2)."""
    patches = tile(0, (0, 0, 0), (n, n, 1), psize, 2)
    state = {0: alfven_2d_state(n, amp, t, gamma)}
    return Problem("alfven_2d", 2, (n, n, 1), patches, 1, state, gamma=gamma, meta={"amp": amp})


def alfven_2d_state(n, amp, t=0.0, gamma=GAMMA):
    k = 2 * math.pi
    omega = 2 * math.pi * math.sqrt(2.0)
    b0 = 1.0 / math.sqrt(2.0)
    dx = 1.0 / n
    x, y, _ = _cell_centres((n, n, 1), (0, 0, 0), (1, 1, 1), 2)
    ph = k * (x + y) - omega * t
    rho = np.ones_like(x)
    p = np.full_like(x, 1.0 / gamma)
    s2 = 1.0 / math.sqrt(2.0)
    vx = amp * np.cos(ph) * s2
    vy = -amp * np.cos(ph) * s2
    vz = -amp * np.sin(ph)
    bz = amp * np.sin(ph)
    xc = np.arange(n + 1) * dx
    Y, X = np.meshgrid(xc, xc, indexing="ij")
    phc = k * (X + Y) - omega * t
    az = -amp * np.sin(phc) / (2 * math.pi * math.sqrt(2.0))
    bx, by = _b_from_az_2d(az, (n, n, 1), dx, dx)
    bx = bx + b0
    by = by + b0
    return _state_2d((n, n, 1), rho, vx, vy, vz, p, bx, by, bz, gamma)


def mhd_wave_mode(family, rho, p, b, khat, v0=(0.0, 0.0, 0.0), sign=1, gamma=GAMMA):
    """Right eigenvector of the linearised ideal-MHD equations in primitive
    variables W = (rho, vx, vy, vz, p, Bx, By, Bz) for a plane wave along the
    unit vector khat through the uniform state (rho, v0, p, b): family
    'fast', 'slow', 'alfven' or 'entropy'; sign +1 or -1 for the wave moving
    along +khat or -khat relative to the flow. Returns (lam, r) with lam =
    khat.v0 + sign c the characteristic speed (c the family's phase speed):
    W + a r cos(k.x - |k| lam t) solves the linearised equations.

    Closed forms (a^2 = gamma p / rho, b_n = b.khat, b_t the rest of b, t its
    direction, u = khat x t): fast / slow c^2 = ((a^2 + |b|^2/rho) +- sqrt((a^2 +
    |b|^2/rho)^2 - 4 a^2 b_n^2 / rho)) / 2, with dv_n = 1, drho = rho / c',
    dp = gamma p / c', dv_t = -b_n |b_t| / (rho c'^2 - b_n^2), dB_t = rho c' |b_t| /
    (rho c'^2 - b_n^2) (c' = sign c); Alfven c = |b_n| / sqrt(rho), dv_u = 1,
    dB_u = -b_n / c'; entropy c = 0, drho = 1. Needs b_t != 0 for the
    magnetosonic and Alfven families."""
    n = np.asarray(khat, dtype=np.float64)
    n = n / np.linalg.norm(n)
    bv = np.asarray(b, dtype=np.float64)
    v0 = np.asarray(v0, dtype=np.float64)
    bn = float(bv @ n)
    bt_vec = bv - bn * n
    bt = float(np.linalg.norm(bt_vec))
    r = np.zeros(8)
    if family == "entropy":
        r[0] = 1.0
        return float(n @ v0), r
    if bt == 0.0:
        raise ValueError("field along the wave vector: degenerate eigenvectors")
    t = bt_vec / bt
    u = np.cross(n, t)
    if family == "alfven":
        c = sign * abs(bn) / math.sqrt(rho)
        r[1:4] = u
        r[5:8] = -bn / c * u
        return float(n @ v0) + c, r
    a2 = gamma * p / rho
    s2 = a2 + (bv @ bv) / rho
    disc = math.sqrt(s2 * s2 - 4.0 * a2 * bn * bn / rho)
    c2 = 0.5 * (s2 + disc) if family == "fast" else 0.5 * (s2 - disc)
    c = sign * math.sqrt(c2)
    den = rho * c * c - bn * bn
    r[0] = rho / c
    r[1:4] = n - (bn * bt / den) * t
    r[4] = gamma * p / c
    r[5:8] = (rho * c * bt / den) * t
    return float(n @ v0) + c, r


def mhd_wave(dim, n, family, amp=1e-6, t=0.0, k=(1, 1, 1), rho=1.0, p=None, b=(0.9, 0.45, 0.3),
             v0=(0.0, 0.0, 0.0), sign=1, psize=16, gamma=GAMMA):
    """Linear MHD wave of one family (mhd_wave_mode) on periodic [0,1]^dim,
    n^dim cells in psize^dim patches, wave vector 2 pi k (integers; k_z = 0 in
    2D): the exact solution of the linearised equations at time t, W(x) =
    W0 + amp r cos(2 pi k.x - omega t), omega = 2 pi |k| lam. Cell fields are
    point values at the cell centres; face B is the uniform b plus the
    discrete curl of the vector potential amp (r_B x K) / |K|^2 sin(phase)
    (K = 2 pi k) sampled at edge midpoints (corners in 2D), so it is
    divergence-free to round-off; in 2D Bz is a cell field. p defaults to
    1/gamma (sound speed 1)."""
    if p is None:
        p = 1.0 / gamma
    kk = np.array([k[d] if d < dim else 0 for d in range(3)], dtype=np.float64)
    K = 2.0 * math.pi * kk
    kn = float(np.linalg.norm(K))
    lam, r = mhd_wave_mode(family, rho, p, b, K / kn, v0, sign, gamma)
    omega = kn * lam
    nn = tuple(n if d < dim else 1 for d in range(3))
    dx = 1.0 / n
    x, y, z = _cell_centres(nn, (0, 0, 0), (1, 1, 1), dim)
    ph = K[0] * x + K[1] * y + K[2] * z - omega * t
    cph = np.cos(ph)
    rho_a = rho + amp * r[0] * cph
    v = [v0[c] + amp * r[1 + c] * cph for c in range(3)]
    p_a = p + amp * r[4] * cph
    avec = amp * np.cross(r[5:8], K) / (kn * kn)  # vector potential amplitude
    if dim == 2:
        xc = np.arange(n + 1) * dx
        Y, X = np.meshgrid(xc, xc, indexing="ij")
        az = avec[2] * np.sin(K[0] * X + K[1] * Y - omega * t)
        bx, by = _b_from_az_2d(az, nn, dx, dx)
        bx = bx + b[0]
        by = by + b[1]
        bz = b[2] + amp * r[7] * cph
        patches = tile(0, (0, 0, 0), nn, psize, 2)
        st = _state_2d(nn, rho_a, v[0], v[1], v[2], p_a, bx, by, bz, gamma)
        return Problem("mhd_wave_%s_2d" % family, 2, nn, patches, 1, {0: st}, gamma=gamma,
                       meta={"amp": amp, "lam": lam, "omega": omega, "r": r})
    ii = np.arange(n + 1)
    ic = (np.arange(n) + 0.5) * dx  # centres
    ie = ii * dx                    # low edges / faces (n + 1 entries)

    def A(c, X, Y, Z):
        return avec[c] * np.sin(K[0] * X + K[1] * Y + K[2] * Z - omega * t)

    # A_x on x-edges (x centre; y, z low corners), A_y on y-edges, A_z on z-edges;
    # arrays indexed [z, y, x] with n + 1 entries along the corner directions
    Zx, Yx, Xx = np.meshgrid(ie, ie, ic, indexing="ij")
    Ax = A(0, Xx, Yx, Zx)                         # (n+1, n+1, n)
    Zy, Yy, Xy = np.meshgrid(ie, ic, ie, indexing="ij")
    Ay = A(1, Xy, Yy, Zy)                         # (n+1, n, n+1)
    Zz, Yz, Xz = np.meshgrid(ic, ie, ie, indexing="ij")
    Az = A(2, Xz, Yz, Zz)                         # (n, n+1, n+1)
    bx = (Az[:, 1:, :] - Az[:, :-1, :]) / dx - (Ay[1:, :, :] - Ay[:-1, :, :]) / dx   # (n, n, n+1)
    by = (Ax[1:, :, :] - Ax[:-1, :, :]) / dx - (Az[:, :, 1:] - Az[:, :, :-1]) / dx   # (n, n+1, n)
    bz = (Ay[:, :, 1:] - Ay[:, :, :-1]) / dx - (Ax[:, 1:, :] - Ax[:, :-1, :]) / dx   # (n+1, n, n)
    bx = bx + b[0]
    by = by + b[1]
    bz = bz + b[2]
    # the periodic copies (entry n along the normal) equal entry 0 exactly
    bx[:, :, -1] = bx[:, :, 0]
    by[:, -1, :] = by[:, 0, :]
    bz[-1, :, :] = bz[0, :, :]
    bcx, bcy, bcz = _cell_b_from_faces(bx, by, bz, 3)
    e = _energy(rho_a, v[0], v[1], v[2], p_a, bcx, bcy, bcz, gamma)
    st = [rho_a, rho_a * v[0], rho_a * v[1], rho_a * v[2], e, bx, by, bz]
    patches = tile(0, (0, 0, 0), nn, psize, 3)
    return Problem("mhd_wave_%s_3d" % family, 3, nn, patches, 1, {0: st}, gamma=gamma,
                   meta={"amp": amp, "lam": lam, "omega": omega, "r": r})


def blast_3d(n=128, psize=16, gamma=GAMMA):
    """3D blast wave on periodic [0,1]^3: rho = 1, p = 0.1, p = 10 for cell
    centres with r^2 < 0.01 around (1/2,1/2,1/2), v = 0, uniform
    B = (1,1,1)/sqrt(3)."""
    patches = tile(0, (0, 0, 0), (n, n, n), psize, 3)
    nn = (n, n, n)
    x, y, z = _cell_centres(nn, (0, 0, 0), (1, 1, 1), 3)
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
    rho = np.ones_like(x)
    p = np.where(r2 < 0.01, 10.0, 0.1)
    b = 1.0 / math.sqrt(3.0)
    bx = np.full((n, n, n + 1), b)
    by = np.full((n, n + 1, n), b)
    bz = np.full((n + 1, n, n), b)
    zero = np.zeros_like(x)
    e = _energy(rho, zero, zero, zero, p, b, b, b, gamma)
    state = {0: [rho, zero.copy(), zero.copy(), zero.copy(), e, bx, by, bz]}
    return Problem("blast_3d", 3, nn, patches, 1, state, gamma=gamma)


def cylinder_3d(n=64, psize=16, contrast=10.0, radius=0.1, gamma=GAMMA):
    """The paper's workload shape (Sec. 6: an advected magnetized cylinder, one
    refined level over 12.5 % of the domain): periodic [0,1]^3, a dense
    cylinder along z through (1/2, 1/2) (density contrast `contrast`, edge
    smoothed over one coarse cell), pressure 1, flow v = (1, 1/2, 0), uniform
    field B = (sqrt 2, 0, 0) (plasma beta 1). Level 0 is n^3 in psize^3 patches;
    level 1 covers the central (n/2)^3 coarse cells (1/8 of the volume) in
    psize^3 fine patches. Whole-level arrays on both levels."""
    base = (n, n, n)
    patches = tile(0, (0, 0, 0), base, psize, 3) + tile(1, (n // 2,) * 3, (3 * n // 2,) * 3, psize, 3)
    b0 = math.sqrt(2.0)
    state = {}
    for l in range(2):
        m = n << l
        x, y, z = _cell_centres((m, m, m), (0, 0, 0), (1, 1, 1), 3)
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2)
        w = 1.0 / n  # smoothing width: one coarse cell
        rho = 1.0 + (contrast - 1.0) * 0.5 * (1.0 - np.tanh((r - radius) / w))
        vx, vy = 1.0, 0.5
        p = np.ones_like(x)
        bx = np.full((m, m, m + 1), b0)
        by = np.zeros((m, m + 1, m))
        bz = np.zeros((m + 1, m, m))
        e = _energy(rho, vx, vy, 0.0, p, b0, 0.0, 0.0, gamma)
        state[l] = [rho, rho * vx, rho * vy, np.zeros_like(x), e, bx, by, bz]
    return Problem("cylinder_3d", 3, base, patches, 2, state, gamma=gamma)


def cylinder_3d_tiled(reps=(1, 1, 1), n=64, psize=16, contrast=10.0, radius=0.1, gamma=GAMMA):
    """The paper's weak-scaling workload unit (Sec. 6) repeated over a block of
    unit cubes: domain [0, a) x [0, b) x [0, c) for reps = (a, b, c), base
    (a n, b n, c n) in psize^3 patches (n^3 base cells per unit, the paper's 64^3
    per processor), in every unit cube the magnetized cylinder of cylinder_3d
    and a refined level over its central eighth (12.5 % filling per unit).
    Whole-level arrays on both levels."""
    a, b, c = reps
    unit = cylinder_3d(n, psize, contrast, radius, gamma)
    base = (a * n, b * n, c * n)
    patches = tile(0, (0, 0, 0), base, psize, 3)
    for k in range(c):
        for j in range(b):
            for i in range(a):
                lo = (2 * (i * n + n // 4), 2 * (j * n + n // 4), 2 * (k * n + n // 4))
                hi = (2 * (i * n + 3 * n // 4), 2 * (j * n + 3 * n // 4), 2 * (k * n + 3 * n // 4))
                patches += tile(1, lo, hi, psize, 3)
    state = {}
    for l in range(2):
        cells = [np.tile(unit.state[l][f], (c, b, a)) for f in range(5)]
        m = n << l
        b0 = float(unit.state[l][5].flat[0])
        bx = np.full((c * m, b * m, a * m + 1), b0)
        by = np.zeros((c * m, b * m + 1, a * m))
        bz = np.zeros((c * m + 1, b * m, a * m))
        state[l] = cells + [bx, by, bz]
    return Problem("cylinder_3d_tiled_%dx%dx%d" % reps, 3, base, patches, 2, state, gamma=gamma,
                   hi=(float(a), float(b), float(c)), meta={"units": a * b * c})


def uniform_state(dim, base, patches, nlev, seed=0, gamma=GAMMA):
    """A random constant state on every level."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0)
    v = rng.uniform(-1, 1, size=3)
    p = rng.uniform(0.2, 2.0)
    b = rng.uniform(-1, 1, size=3)
    if dim == 2:
        pass
    state = {}
    for l in range(nlev):
        n = tuple(base[d] << l if d < dim else 1 for d in range(3))
        shp = (n[2], n[1], n[0])
        one = np.ones(shp)
        e = _energy(rho, v[0], v[1], v[2], p, b[0], b[1], b[2], gamma)
        bx = np.full((n[2], n[1], n[0] + 1), b[0])
        by = np.full((n[2], n[1] + 1, n[0]), b[1])
        bz = np.full((n[2] + 1, n[1], n[0]), b[2]) if dim == 3 else one * b[2]
        state[l] = [one * rho, one * rho * v[0], one * rho * v[1], one * rho * v[2], one * e, bx, by, bz]
    return state


def random_smooth_2d(n, nlev, seed=0, amp=0.05, gamma=GAMMA):
    """A smooth random 2D state (few Fourier modes) on every level of a
    hierarchy with base n x n; face B from a vector potential."""
    rng = np.random.default_rng(seed)
    modes = [(rng.integers(1, 3), rng.integers(1, 3), rng.uniform(0, 2 * math.pi)) for _ in range(3)]
    coef = rng.normal(size=(7, 3)) * amp
    state = {}
    for l in range(nlev):
        nn = (n << l, n << l, 1)
        dx = 1.0 / nn[0]
        x, y, _ = _cell_centres(nn, (0, 0, 0), (1, 1, 1), 2)

        def f(c, X, Y):
            s = 0.0
            for m, (kx, ky, ph) in enumerate(modes):
                s = s + coef[c, m] * np.sin(2 * math.pi * (kx * X + ky * Y) + ph)
            return s

        rho = 1.0 + f(0, x, y)
        vx = 0.3 + f(1, x, y)
        vy = -0.2 + f(2, x, y)
        vz = f(3, x, y)
        p = 1.0 + f(4, x, y)
        bz = 0.3 + f(5, x, y)
        xc = np.arange(nn[0] + 1) * dx
        Y, X = np.meshgrid(xc, xc, indexing="ij")
        az = f(6, X, Y) / (2 * math.pi) + 0.6 * Y - 0.4 * X
        bx, by = _b_from_az_2d(az, nn, dx, dx)
        state[l] = _state_2d(nn, rho, vx, vy, vz, p, bx, by, bz, gamma)
    return state


def conserved(prim, gamma=GAMMA):
    """Conserved vector (rho, mx, my, mz, E, Bx, By, Bz) of one primitive state
    (rho, vx, vy, vz, p, Bx, By, Bz)."""
    rho, vx, vy, vz, p, bx, by, bz = [float(v) for v in prim]
    return (rho, rho * vx, rho * vy, rho * vz, _energy(rho, vx, vy, vz, p, bx, by, bz, gamma), bx, by, bz)


def rankine_hugoniot(mach, rho1=1.0, p1=None, gamma=GAMMA):
    """Hydrodynamic normal-shock jump in the shock frame for an upstream state
    of sound speed 1 (p1 = rho1 / gamma unless given): returns (rho1, u1, p1,
    rho2, u2, p2). A field along the shock normal leaves the jump unchanged."""
    if p1 is None:
        p1 = rho1 / gamma
    c1 = math.sqrt(gamma * p1 / rho1)
    u1 = mach * c1
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    u2 = u1 * rho1 / rho2
    return rho1, u1, p1, rho2, u2, p2


def _fill_level(n, dim, cells, faces):
    """Whole-level arrays of a state given per-cell primitive arrays
    (rho, vx, vy, vz, p, bz-cell in 2D) and per-face normal B arrays."""
    rho, vx, vy, vz, p = cells[:5]
    bx, by, bz = faces
    bcx, bcy, bcz = _cell_b_from_faces(bx, by, bz, dim)
    e = _energy(rho, vx, vy, vz, p, bcx, bcy, bcz, gamma=cells[5])
    return [rho, rho * vx, rho * vy, rho * vz, e, bx, by, bz]


def stationary_shock(dim=2, n=64, mach=10.0, bn=0.2, refine=True, psize=8, gamma=GAMMA):
    """A stationary planar shock at x = 1/2 (a face of every level) on
    [0,1] x [0,1/8] (x [0,1/8] in 3D): supersonic inflow of the upstream
    state (rho 1, sound speed 1, velocity +mach) at x-low, zero-gradient
    outflow at x-high, periodic in y and z; the downstream state is the
    Rankine-Hugoniot jump; uniform normal field Bx = bn. With refine, level 1
    covers the shock and both x boundaries."""
    rho1, u1, p1, rho2, u2, p2 = rankine_hugoniot(mach, gamma=gamma)
    m = n // 8
    base = (n, m, m if dim == 3 else 1)
    hi = (1.0, 1.0 / 8.0, 1.0 / 8.0 if dim == 3 else 1.0)
    patches = tile(0, (0, 0, 0), base, psize, dim)
    nlev = 1
    if refine:
        fy = (2 * base[1], 2 * base[2] if dim == 3 else 1)
        for x0, x1 in ((0, n // 4), (n - n // 4, n + n // 4), (2 * n - n // 4, 2 * n)):
            patches += tile(1, (x0, 0, 0), (x1, fy[0], fy[1]), psize, dim)
        nlev = 2
    state = {}
    for l in range(nlev):
        nn = tuple(base[d] << l if d < dim else 1 for d in range(3))
        x, _, _ = _cell_centres(nn, (0, 0, 0), hi, dim)
        up = x < 0.5
        rho = np.where(up, rho1, rho2)
        vx = np.where(up, u1, u2)
        p = np.where(up, p1, p2)
        zero = np.zeros_like(x)
        bx = np.full((nn[2], nn[1], nn[0] + 1), bn)
        by = np.zeros((nn[2], nn[1] + 1, nn[0]))
        bz = np.zeros((nn[2] + 1, nn[1], nn[0])) if dim == 3 else zero.copy()
        state[l] = _fill_level(nn, dim, (rho, vx, zero, zero.copy(), p, gamma), (bx, by, bz))
    bc = (2, 1, 0, 0, 0, 0)
    return Problem("stationary_shock_%dd" % dim, dim, base, patches, nlev, state, gamma=gamma, hi=hi, bc=bc,
                   inflow=conserved((rho1, u1, 0, 0, p1, bn, 0, 0), gamma),
                   meta={"mach": mach, "downstream": (rho2, u2, p2), "upstream": (rho1, u1, p1)})


def uniform_flow(dim, base, patches, nlev, bc, seed=0, gamma=GAMMA):
    """A random constant state with a non-zero velocity on every level; the
    inflow state (used on inflow sides) is that same state."""
    rng = np.random.default_rng(seed)
    prim = (rng.uniform(0.5, 2.0), *rng.uniform(0.3, 1.0, size=3) * rng.choice([-1, 1], size=3),
            rng.uniform(0.2, 2.0), *rng.uniform(-1, 1, size=3))
    u = conserved(prim, gamma)
    state = {}
    for l in range(nlev):
        n = tuple(base[d] << l if d < dim else 1 for d in range(3))
        shp = (n[2], n[1], n[0])
        one = np.ones(shp)
        bx = np.full((n[2], n[1], n[0] + 1), u[5])
        by = np.full((n[2], n[1] + 1, n[0]), u[6])
        bz = np.full((n[2] + 1, n[1], n[0]), u[7]) if dim == 3 else one * u[7]
        state[l] = [one * u[0], one * u[1], one * u[2], one * u[3], one * u[4], bx, by, bz]
    return Problem("uniform_flow_%dd" % dim, dim, tuple(base), patches, nlev, state, gamma=gamma, bc=tuple(bc),
                   inflow=u)


def smooth_bounded_2d(n=32, refine=True, seed=0, mirrored=False, gamma=GAMMA):
    """A smooth random 2D flow through a box bounded in x (outflow on both x
    sides, periodic y) with vx in [0.3, 0.9] and vy in [0.15, 0.45], so no face
    mass flux changes sign. mirrored=True gives the exact mirror image about
    x = 1/2 (vx and Bx negated, cells and faces reversed in x), which flows the
    other way. Level 1 covers both x boundaries and the centre, a layout that
    is its own mirror image."""
    rng = np.random.default_rng(seed)
    patches = tile(0, (0, 0, 0), (n, n, 1), 8, 2)
    nlev = 1
    if refine:
        for x0, x1 in ((0, n // 2), (n - n // 4, n + n // 4), (2 * n - n // 2, 2 * n)):
            patches += tile(1, (x0, 0, 0), (x1, 2 * n, 1), 8, 2)
        nlev = 2
    k = [(int(rng.integers(1, 3)), int(rng.integers(1, 3)), rng.uniform(0, 2 * math.pi)) for _ in range(7)]
    a = rng.uniform(0.05, 0.1, size=7)

    def f(c, X, Y):
        kx, ky, ph = k[c]
        return a[c] * np.sin(2 * math.pi * (kx * X + ky * Y) + ph)

    state = {}
    for l in range(nlev):
        nn = (n << l, n << l, 1)
        dx = 1.0 / nn[0]
        x, y, _ = _cell_centres(nn, (0, 0, 0), (1, 1, 1), 2)
        rho = 1.0 + 2.0 * f(0, x, y)
        p = 1.0 + 2.0 * f(1, x, y)
        vx = 0.6 + 3.0 * f(2, x, y)
        vy = 0.3 + 1.5 * f(3, x, y)
        vz = f(4, x, y)
        bz = 0.3 + f(5, x, y)
        Y, X = np.meshgrid(np.arange(nn[1] + 1) * dx, np.arange(nn[0] + 1) * dx, indexing="ij")
        az = 0.4 * Y - 0.2 * X + f(6, X, Y) / (2 * math.pi)
        bx, by = _b_from_az_2d(az, nn, dx, dx, periodic=(False, True))
        st = _state_2d(nn, rho, vx, vy, vz, p, bx, by, bz, gamma)
        if mirrored:
            sign = (1, -1, 1, 1, 1, -1, 1, 1)
            st = [sign[i] * v[..., ::-1] for i, v in enumerate(st)]
        state[l] = [np.ascontiguousarray(v) for v in st]
    return Problem("smooth_bounded_2d", 2, (n, n, 1), patches, nlev, state, gamma=gamma, bc=(1, 1, 0, 0, 0, 0),
                   meta={"seed": seed, "mirrored": mirrored})


def clump_centres(dim, n_clumps=8, seed=3, lo=0.15, hi=0.85):
    """Uniformly placed seeded clump centres (kept away from the periodic seam)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(lo, hi, size=(n_clumps, 3))
    if dim == 2:
        c[:, 2] = 0.5
    return c


def clump_cells(x, y, z, dim, centres, radius, rho_clump=100.0, rho_amb=1.0, p=1.0, v=(1.0, 0.0, 0.0),
                gamma=GAMMA):
    """Cell-centred primitive fields of dense clumps in pressure equilibrium in
    a uniform flow: rho = rho_clump inside any clump (cell centre strictly
    within the radius), rho_amb outside."""
    inside = np.zeros(x.shape, bool)
    for c in centres:
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + ((z - c[2]) ** 2 if dim == 3 else 0.0)
        inside |= r2 < radius * radius
    rho = np.where(inside, rho_clump, rho_amb)
    return rho, np.full(x.shape, v[0]), np.full(x.shape, v[1]), np.full(x.shape, v[2]), np.full(x.shape, p)


def clump_boxes(dim, base, nlev, centres, radius, margin=6, block=8):
    """A properly nested static hierarchy around the clumps: on the finest
    level one box per clump covering its radius plus margin cells, aligned to
    block fine cells; each coarser level holds the coarsened finer boxes grown
    by margin cells; overlapping boxes are merged into their bounding box; boxes
    are split into pieces of at most 32 cells per side."""
    def merge(boxes):
        boxes = [list(map(list, b)) for b in boxes]
        changed = True
        while changed:
            changed = False
            for i in range(len(boxes)):
                for j in range(i + 1, len(boxes)):
                    a, b = boxes[i], boxes[j]
                    if all(a[0][d] < b[1][d] and b[0][d] < a[1][d] for d in range(dim)):
                        boxes[i] = [[min(a[0][d], b[0][d]) for d in range(3)], [max(a[1][d], b[1][d]) for d in range(3)]]
                        del boxes[j]
                        changed = True
                        break
                if changed:
                    break
        return boxes

    def align(lo, hi, n):
        lo = [max(0, (v // block) * block) for v in lo]
        hi = [min(n[d], -((-v) // block) * block) for d, v in enumerate(hi)]
        return lo, hi

    levels = {}
    for l in range(nlev - 1, 0, -1):
        n = [base[d] << l if d < dim else 1 for d in range(3)]
        boxes = []
        for c in centres:
            lo = [int(np.floor((c[d] - radius) * n[d])) - margin if d < dim else 0 for d in range(3)]
            hi = [int(np.ceil((c[d] + radius) * n[d])) + margin if d < dim else 1 for d in range(3)]
            boxes.append(align(lo, hi, n))
        if l + 1 in levels:
            for (lo, hi) in levels[l + 1]:
                clo = [(lo[d] // 2) - margin if d < dim else 0 for d in range(3)]
                chi = [(hi[d] + 1) // 2 + margin if d < dim else 1 for d in range(3)]
                boxes.append(align(clo, chi, n))
        for b in boxes:
            if dim == 2:
                b[0][2], b[1][2] = 0, 1
        levels[l] = merge(boxes)
    patches = []
    for l in range(1, nlev):
        for (lo, hi) in levels[l]:
            for k0 in range(lo[2], hi[2], 32 if dim == 3 else 1):
                for j0 in range(lo[1], hi[1], 32):
                    for i0 in range(lo[0], hi[0], 32):
                        patches.append((l, (i0, j0, k0), (min(i0 + 32, hi[0]), min(j0 + 32, hi[1]),
                                                          min(k0 + 32, hi[2]) if dim == 3 else 1)))
    return patches


def clumps_2d(n=32, nlev=3, n_clumps=4, radius=0.06, seed=3, psize=8, b_pert=0.0, gamma=GAMMA):
    """2D version of the clump workload (whole-level arrays on every level):
    dense clumps (contrast 100) in pressure equilibrium advected by a uniform
    flow v = (1, 0) along a uniform field B = (sqrt 2, 0) (plasma beta 1), plus
    optionally a divergence-free perturbation of amplitude b_pert from the
    vector potential b_pert sin(2 pi x) sin(2 pi y) / (2 pi)."""
    centres = clump_centres(2, n_clumps, seed)
    base = (n, n, 1)
    patches = tile(0, (0, 0, 0), base, psize, 2) + clump_boxes(2, base, nlev, centres, radius)
    b0 = math.sqrt(2.0)
    state = {}
    for l in range(nlev):
        nn = (n << l, n << l, 1)
        x, y, z = _cell_centres(nn, (0, 0, 0), (1, 1, 1), 2)
        rho, vx, vy, vz, p = clump_cells(x, y, z, 2, centres, radius)
        dx = 1.0 / nn[0]
        Y, X = np.meshgrid(np.arange(nn[1] + 1) * dx, np.arange(nn[0] + 1) * dx, indexing="ij")
        az = b_pert * np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y) / (2 * math.pi)
        bx, by = _b_from_az_2d(az, nn, dx, dx)
        bx = bx + b0
        bz = np.zeros_like(x)
        state[l] = _state_2d(nn, rho, vx, vy, vz, p, bx, by, bz, gamma)
    return Problem("clumps_2d", 2, base, patches, nlev, state, gamma=gamma,
                   meta={"centres": centres, "radius": radius, "seed": seed})


def clumps_3d_small(n=16, nlev=2, n_clumps=3, radius=0.1, seed=3, b_pert=0.3, gamma=GAMMA):
    """3D clumps as whole-level arrays on every level (small sizes, for parity
    tests): contrast 100, pressure equilibrium, v = (1, 0, 0), B = (sqrt 2, 0, 0)
    plus a perturbation from the vector potential A_z = b_pert sin(2 pi x)
    sin(2 pi y) / (2 pi)."""
    centres = clump_centres(3, n_clumps, seed, lo=0.3, hi=0.7)
    base = (n, n, n)
    patches = tile(0, (0, 0, 0), base, 8, 3) + clump_boxes(3, base, nlev, centres, radius, margin=4)
    b0 = math.sqrt(2.0)
    state = {}
    for l in range(nlev):
        m = n << l
        x, y, z = _cell_centres((m, m, m), (0, 0, 0), (1, 1, 1), 3)
        rho, vx, vy, vz, p = clump_cells(x, y, z, 3, centres, radius)
        dx = 1.0 / m
        ax = np.arange(m + 1) * dx
        Y, X = np.meshgrid(ax, ax, indexing="ij")
        az = b_pert * np.sin(2 * math.pi * X) * np.sin(2 * math.pi * Y) / (2 * math.pi)
        bx2, by2 = _b_from_az_2d(az, (m, m, 1), dx, dx)
        bx = np.broadcast_to(bx2 + b0, (m, m, m + 1)).copy()
        by = np.broadcast_to(by2, (m, m + 1, m)).copy()
        bz = np.zeros((m + 1, m, m))
        bcx, bcy, bcz = _cell_b_from_faces(bx, by, bz, 3)
        e = _energy(rho, vx, vy, vz, p, bcx, bcy, bcz, gamma)
        state[l] = [rho, rho * vx, rho * vy, rho * vz, e, bx, by, bz]
    return Problem("clumps_3d_small", 3, base, patches, nlev, state, gamma=gamma,
                   meta={"centres": centres, "radius": radius})


def clumps_3d(base=32, nlev=6, n_clumps=8, radius=0.02, seed=3, margin=6, gamma=GAMMA):
    """The deep clump workload: 3D, base^3 level 0 in 16^3 patches, nlev
    levels around 8 seeded dense clumps (contrast 100, radius 0.02, uniformly
    placed) in pressure equilibrium (p = 1), advected by v = (1, 0, 0) along
    B = (sqrt 2, 0, 0) (plasma beta 1). The state is given per patch
    (packed_clumps): whole-level arrays of the finest levels would not fit."""
    centres = clump_centres(3, n_clumps, seed)
    b = (base, base, base)
    patches = tile(0, (0, 0, 0), b, 16, 3) + clump_boxes(3, b, nlev, centres, radius, margin=margin)
    return Problem("clumps_3d", 3, b, patches, nlev, None, gamma=gamma,
                   meta={"centres": centres, "radius": radius, "seed": seed})


def packed_clumps(pb, patches=None):
    """The 8 packed field arrays (field-major; patches in id order; a patch's
    interior cells, or its own faces along the field's direction, x fastest)
    of the clump state of pb on the given patch list."""
    patches = pb.patches if patches is None else patches
    centres, radius = pb.meta["centres"], pb.meta["radius"]
    b0 = math.sqrt(2.0)
    out = [[] for _ in range(8)]
    for (l, lo, hi) in patches:
        n = [pb.base[d] << l for d in range(3)]
        xs = [(np.arange(lo[d], hi[d]) + 0.5) / n[d] for d in range(3)]
        z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        rho, vx, vy, vz, p = clump_cells(x, y, z, 3, centres, radius)
        e = _energy(rho, vx, vy, vz, p, b0, 0.0, 0.0, pb.gamma)
        for f, a in enumerate((rho, rho * vx, rho * vy, rho * vz, e)):
            out[f].append(a.ravel())
        shp = [hi[d] - lo[d] for d in range(3)]
        for d, val in ((0, b0), (1, 0.0), (2, 0.0)):
            s = list(shp)
            s[d] += 1
            out[5 + d].append(np.full(int(np.prod(s)), val))
    return [np.concatenate(a) for a in out]


def adjoint_2d(n=256, psize=32, seed=4, amp=1e-4, kmax=8, rms=1e-4, gamma=GAMMA):
    """The adjoint workload: n^2 periodic base in psize^2 patches plus one
    refined level over the quadrant [0, 1/2)^2 (its C/F boundary crosses the
    periodic seam); the circularly polarised Alfven wave of amplitude amp plus
    a seeded smooth velocity perturbation sum_{|k| <= kmax} a_k cos(2 pi k.x +
    phi_k) per component (a_k ~ N(0,1), phi_k ~ U[0, 2 pi)), rescaled to an rms
    of rms."""
    rng = np.random.default_rng(seed)
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if 0 < kx * kx + ky * ky <= kmax * kmax]
    coef = rng.normal(size=(len(ks), 3))
    phase = rng.uniform(0, 2 * math.pi, size=(len(ks), 3))
    base = (n, n, 1)
    patches = tile(0, (0, 0, 0), base, psize, 2) + tile(1, (0, 0, 0), (n, n, 1), psize, 2)
    state = {}
    scale = None
    for l in range(2):
        m = n << l
        st = alfven_2d_state(m, amp, 0.0, gamma)
        x, y, _ = _cell_centres((m, m, 1), (0, 0, 0), (1, 1, 1), 2)
        dv = np.zeros((3,) + x.shape)
        for i, (kx, ky) in enumerate(ks):
            for c in range(3):
                dv[c] += coef[i, c] * np.cos(2 * math.pi * (kx * x + ky * y) + phase[i, c])
        if scale is None:
            scale = rms / np.sqrt((dv ** 2).mean())
        dv *= scale
        rho = st[0]
        v = [st[1 + c] / rho + dv[c] for c in range(3)]
        ke_old = 0.5 * (st[1] ** 2 + st[2] ** 2 + st[3] ** 2) / rho
        for c in range(3):
            st[1 + c] = rho * v[c]
        st[4] = st[4] - ke_old + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
        state[l] = st
    return Problem("adjoint_2d", 2, base, patches, 2, state, gamma=gamma, meta={"seed": seed})


def fractal_field(n=256, slope=-11.0 / 3.0, seed=7):
    """A periodic Gaussian random field on an n^3 grid with power spectrum
    P(k) ~ k^slope (zero mean, unit variance), by filtering white noise in
    Fourier space."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(n) * n
    kz, ky, kx = np.meshgrid(k, k, np.fft.rfftfreq(n) * n, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(kk)
    amp[kk > 0] = kk[kk > 0] ** (slope / 2.0)
    noise = np.fft.rfftn(rng.normal(size=(n, n, n)))
    g = np.fft.irfftn(noise * amp, s=(n, n, n))
    g -= g.mean()
    return g / g.std()


def _trilinear(g, x, y, z):
    """Periodic trilinear sample of the grid g (cell-centred on [0,1]^3) at points."""
    n = g.shape[0]
    fx, fy, fz = x * n - 0.5, y * n - 0.5, z * n - 0.5
    i0, j0, k0 = np.floor(fx).astype(int), np.floor(fy).astype(int), np.floor(fz).astype(int)
    tx, ty, tz = fx - i0, fy - j0, fz - k0
    out = 0.0
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                wgt = (tx if di else 1 - tx) * (ty if dj else 1 - ty) * (tz if dk else 1 - tz)
                out = out + wgt * g[(k0 + dk) % n, (j0 + dj) % n, (i0 + di) % n]
    return out


def shock_clump_3d(base=64, nlev=5, radius=0.15, centre=(0.5, 0.5, 0.5), mach=10.0, sigma=1.0, contrast=10.0,
                   shock_x=0.1, seed=7, fft_n=256, margin=4, gamma=GAMMA):
    """The shock-clump workload: a Mach-10 planar shock (hydrodynamic
    Rankine-Hugoniot jump; the field B = (sqrt 2, 0, 0) lies along the normal,
    plasma beta 1 with p = 1) at x = shock_x moving into a clump of radius
    0.15 whose density is lognormal, rho = contrast exp(sigma G) / <exp(sigma G)>
    with G a Gaussian random field of spectral slope -11/3 (sampled
    trilinearly from an fft_n^3 grid), in an ambient rho = 1, p = 1 at rest.
    Inflow of the post-shock state at x-low, outflow on every other side.
    Level 0 in 16^3 patches; nested boxes around the clump on the finer levels.
    The state is given per patch (packed_shock_clump)."""
    b = (base, base, base)
    patches = tile(0, (0, 0, 0), b, 16, 3) + clump_boxes(3, b, nlev, [centre], radius, margin=margin)
    c1 = math.sqrt(gamma * 1.0 / 1.0)
    rho1, u1, p1, rho2, u2, p2 = rankine_hugoniot(mach, rho1=1.0, p1=1.0, gamma=gamma)
    us = mach * c1                  # shock speed into the gas at rest
    u2lab = us * (1.0 - rho1 / rho2)  # post-shock gas velocity in the lab frame
    b0 = math.sqrt(2.0)
    post = conserved((rho2, u2lab, 0.0, 0.0, p2, b0, 0.0, 0.0), gamma)
    return Problem("shock_clump_3d", 3, b, patches, nlev, None, gamma=gamma,
                   bc=(2, 1, 1, 1, 1, 1), inflow=post,
                   meta={"radius": radius, "centre": centre, "sigma": sigma, "contrast": contrast, "seed": seed,
                         "fft_n": fft_n, "shock_x": shock_x, "post": (rho2, u2lab, p2), "b0": b0})


def packed_shock_clump(pb, patches=None, field=None):
    """The 8 packed field arrays of the shock-clump state of pb on the given
    patch list (layout as packed_clumps)."""
    patches = pb.patches if patches is None else patches
    m = pb.meta
    g = field if field is not None else fractal_field(m["fft_n"], seed=m["seed"])
    mean_exp = np.exp(m["sigma"] * g).mean()
    rho2, u2, p2 = m["post"]
    b0 = m["b0"]
    out = [[] for _ in range(8)]
    for (l, lo, hi) in patches:
        n = [pb.base[d] << l for d in range(3)]
        xs = [(np.arange(lo[d], hi[d]) + 0.5) / n[d] for d in range(3)]
        z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        r2 = (x - m["centre"][0]) ** 2 + (y - m["centre"][1]) ** 2 + (z - m["centre"][2]) ** 2
        rho = np.ones_like(x)
        inside = r2 < m["radius"] ** 2
        if inside.any():
            rho[inside] = m["contrast"] * np.exp(m["sigma"] * _trilinear(g, x[inside], y[inside], z[inside])) / mean_exp
        p = np.ones_like(x)
        vx = np.zeros_like(x)
        shocked = x < m["shock_x"]
        rho[shocked], vx[shocked], p[shocked] = rho2, u2, p2
        e = _energy(rho, vx, 0.0, 0.0, p, b0, 0.0, 0.0, pb.gamma)
        for f, a in enumerate((rho, rho * vx, np.zeros_like(x), np.zeros_like(x), e)):
            out[f].append(a.ravel())
        shp = [hi[d] - lo[d] for d in range(3)]
        for d, val in ((0, b0), (1, 0.0), (2, 0.0)):
            sh = list(shp)
            sh[d] += 1
            out[5 + d].append(np.full(int(np.prod(sh)), val))
    return [np.concatenate(a) for a in out]


def shock_clump_3d_small(base=16, nlev=3, fft_n=64, **kw):
    """The shock-clump workload down-scaled for parity tests (16^3 base, 3
    levels by default) with whole-level arrays on every level: the same state
    as shock_clump_3d / packed_shock_clump, each level generated as one box
    over its whole domain."""
    pb = shock_clump_3d(base=base, nlev=nlev, fft_n=fft_n, **kw)
    g = fractal_field(fft_n, seed=pb.meta["seed"])
    state = {}
    for l in range(nlev):
        n = [base << l] * 3
        whole = [(l, (0, 0, 0), tuple(n))]
        packed = packed_shock_clump(pb, patches=whole, field=g)
        arrs = []
        for f in range(8):
            shp = [n[2], n[1], n[0]]
            if f >= 5:
                shp[2 - (f - 5)] += 1
            arrs.append(packed[f].reshape(shp))
        state[l] = arrs
    pb.state = state
    return pb


def random_hierarchy(dim, seed, base=32, psize0=16, nlev=2, max_tries=200):
    """A random properly nested periodic hierarchy: level 0 tiled by patches
    of random widths; finer levels a few random boxes aligned to parent cells,
    each at least 3 parent cells inside a parent-level patch (so the nesting
    rule holds), possibly touching each other and the periodic seam."""
    rng = np.random.default_rng(seed)
    # level 0: random cuts per dimension
    cuts = []
    for d in range(3):
        if d >= dim:
            cuts.append([0, 1])
            continue
        c = [0]
        while c[-1] < base:
            w = int(rng.choice([8, 12, 16]))
            c.append(min(base, c[-1] + w))
        if c[-1] - c[-2] < 4:
            c.pop(-2)
        cuts.append(c)
    patches = []
    for k in range(len(cuts[2]) - 1):
        for j in range(len(cuts[1]) - 1):
            for i in range(len(cuts[0]) - 1):
                patches.append((0, (cuts[0][i], cuts[1][j], cuts[2][k]), (cuts[0][i + 1], cuts[1][j + 1], cuts[2][k + 1])))
    for l in range(1, nlev):
        parents = [p for p in patches if p[0] == l - 1]
        n_l = base << l
        made = []
        tries = 0
        while len(made) < 3 and tries < max_tries:
            tries += 1
            par = parents[rng.integers(len(parents))]
            lo, hi = [], []
            ok = True
            for d in range(3):
                if d >= dim:
                    lo.append(0)
                    hi.append(1)
                    continue
                plo, phi = par[1][d] + 3, par[2][d] - 3  # parent cells
                if l - 1 == 0:  # level 0 covers the whole domain
                    plo, phi = 0, base
                if phi - plo < 2:
                    ok = False
                    break
                wmax = 10 if l - 1 == 0 else 6
                a = int(rng.integers(plo, phi - 1))
                b = int(rng.integers(min(a + 4, phi) if l - 1 == 0 else a + 1, min(phi, a + wmax) + 1))
                lo.append(2 * a)
                hi.append(2 * b)
            if not ok:
                continue
            cand = (l, tuple(lo), tuple(hi))
            # reject overlaps with already-made boxes on this level
            clash = False
            for m in made:
                if all(not (cand[2][d] <= m[1][d] or cand[1][d] >= m[2][d]) for d in range(dim)):
                    clash = True
            if clash:
                continue
            made.append(cand)
            _ = n_l
        patches += made
    return patches
