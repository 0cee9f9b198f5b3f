"""Seeded inputs for the pointwise transposed Jacobians (HLLD flux and
half-step predictor) that the adjoint applies at every face and cell, chosen so
that every case of the HLLD solver occurs (Sec. 4's hyperbolic advance, HLLD
of Miyoshi and Kusano): supersonic left/right, single star without a normal
field, single star behind a rotational wave, double star, and degenerate star
states (no tangential field, Alfven speed above the sound speed). No scheme
arithmetic except `hlld_branch`, which only labels the case a row falls in (for
coverage reports), never a value that is compared."""
import numpy as np

GAMMA = 5.0 / 3.0


def _state(rng, n, un=None):
    q = np.empty((n, 7))
    q[:, 0] = rng.uniform(0.3, 3.0, n)
    q[:, 1] = rng.normal(0.0, 0.6, n) if un is None else un
    q[:, 2] = rng.normal(0.0, 0.6, n)
    q[:, 3] = rng.normal(0.0, 0.6, n)
    q[:, 4] = rng.uniform(0.1, 2.0, n)
    q[:, 5] = rng.normal(0.0, 1.0, n)
    q[:, 6] = rng.normal(0.0, 1.0, n)
    return q


def hlld_cases(n, seed=0):
    """n rows x = (ql[7], qr[7], bn) and seeds g[7], six families of n/6 rows."""
    rng = np.random.default_rng(seed)
    m = n // 6
    fam = []
    # generic states (mostly double-star)
    fam.append(np.hstack([_state(rng, m), _state(rng, m), rng.normal(0.0, 1.0, (m, 1))]))
    # supersonic to the right and to the left
    for s in (1.0, -1.0):
        u = s * rng.uniform(5.0, 9.0, m)
        fam.append(np.hstack([_state(rng, m, u), _state(rng, m, u + rng.normal(0, 0.2, m)),
                              rng.normal(0.0, 1.0, (m, 1))]))
    # no normal field: single star states
    fam.append(np.hstack([_state(rng, m), _state(rng, m), np.zeros((m, 1))]))
    # weak normal field and a fast flow: single star behind the rotational wave
    u = rng.choice([-1.0, 1.0], m) * rng.uniform(0.6, 1.2, m)
    fam.append(np.hstack([_state(rng, m, u), _state(rng, m, u + rng.normal(0.0, 0.05, m)),
                          rng.normal(0.0, 0.03, (m, 1))]))
    # degenerate star states: equal states, no tangential field, bn^2 > gamma p
    k = n - 5 * m
    q = _state(rng, k)
    q[:, 5:7] = 0.0
    bn = rng.choice([-1.0, 1.0], k) * np.sqrt(GAMMA * q[:, 4] * rng.uniform(1.5, 4.0, k))
    fam.append(np.hstack([q, q, bn[:, None]]))
    x = np.vstack(fam)
    g = rng.normal(0.0, 1.0, (n, 7))
    return x, g


def hlld_branch(x, gamma=GAMMA, eps=1e-12):
    """Label of the HLLD case at x: 0 supersonic left state, 1 supersonic right,
    2 single star with bn^2 <= eps p_T*, 3 single star outside the rotational
    waves, 4 double star, 5 double star with a degenerate star state."""
    ql, qr, bn = x[:7], x[7:14], x[14]

    def cf(q):
        b2 = bn * bn + q[5] ** 2 + q[6] ** 2
        a = (gamma * q[4] + b2) / q[0]
        d = max(a * a - 4 * gamma * q[4] * bn * bn / q[0] ** 2, 0.0)
        return np.sqrt(0.5 * (a + np.sqrt(d)))

    c = max(cf(ql), cf(qr))
    sl, sr = min(ql[1], qr[1]) - c, max(ql[1], qr[1]) + c
    if sl > 0:
        return 0
    if sr < 0:
        return 1
    ptl = ql[4] + 0.5 * (bn * bn + ql[5] ** 2 + ql[6] ** 2)
    ptr = qr[4] + 0.5 * (bn * bn + qr[5] ** 2 + qr[6] ** 2)
    dl, dr = sl - ql[1], sr - qr[1]
    den = dr * qr[0] - dl * ql[0]
    sm = (dr * qr[0] * qr[1] - dl * ql[0] * ql[1] - ptr + ptl) / den
    pts = (dr * qr[0] * ptl - dl * ql[0] * ptr + ql[0] * qr[0] * dr * dl * (qr[1] - ql[1])) / den
    if bn * bn <= eps * pts:
        return 2
    rs, degen = [], False
    for q, s in ((ql, sl), (qr, sr)):
        rs.append(q[0] * (s - q[1]) / (s - sm))
        e = q[0] * (s - q[1]) * (s - sm) - bn * bn
        degen |= abs(e) <= eps * (abs(q[0] * (s - q[1]) * (s - sm)) + bn * bn)
    if sm - abs(bn) / np.sqrt(rs[0]) >= 0 or sm + abs(bn) / np.sqrt(rs[1]) <= 0:
        return 3
    return 5 if degen else 4


def predict_cases(dim, n, seed=0):
    """n rows x = (w[8], s_0[8], .., s_{dim-1}[8]) of primitive states and
    slopes, seeds g[8], and h[dim] = dt / (2 dx_d)."""
    rng = np.random.default_rng(seed)
    w = np.empty((n, 8))
    w[:, 0] = rng.uniform(0.3, 3.0, n)
    w[:, 1:4] = rng.normal(0.0, 1.0, (n, 3))
    w[:, 4] = rng.uniform(0.1, 2.0, n)
    w[:, 5:8] = rng.normal(0.0, 1.0, (n, 3))
    s = rng.normal(0.0, 0.1, (n, 8 * dim)) * np.tile(np.abs(w), dim)
    g = rng.normal(0.0, 1.0, (n, 8))
    h = rng.uniform(0.05, 0.4, dim)
    return np.hstack([w, s]), g, h
