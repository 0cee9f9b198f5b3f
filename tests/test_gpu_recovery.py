"""The mixed-precision recovery (FP32 stored values; ke = |m|^2/(2 rho) and
me = |B_c|^2/2 as double-float FP32 pairs; the energy balance in FP64; the
pressure rounded to FP32) against the oracle's FP64 recovery of the same FP32
inputs, on random cells: the bound of reading R19 (pressure within 2 FP32 ulp
of p plus 2^-44 (gamma-1)(ke + me); velocity within 4 ulp; B_c within half an
ulp)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1110_1616_gb300 import amrmhd as A

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1110_1616_gb300 import build
    build.build()


def random_cells(n, seed):
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.uniform(-5, 5, n))
    v = rng.uniform(-1, 1, (n, 3)) * np.exp(rng.uniform(-3, 3, (n, 1)))
    p = np.exp(rng.uniform(-6, 4, n))
    bl = rng.uniform(-3, 3, (n, 3))
    br = bl + rng.uniform(-0.3, 0.3, (n, 3))
    bc = 0.5 * (bl + br)
    E = p / (GAMMA - 1.0) + 0.5 * rho * (v * v).sum(1) + 0.5 * (bc * bc).sum(1)
    u = np.column_stack([rho, rho * v[:, 0], rho * v[:, 1], rho * v[:, 2], E])
    return u.astype(np.float32), bl.astype(np.float32), br.astype(np.float32)


def test_mixed_recovery_error_bound():
    u, bl, br = random_cells(20000, 5)
    w = A.recover_mixed(u, bl, br, GAMMA).astype(np.float64)
    u64, bl64, br64 = u.astype(np.float64), bl.astype(np.float64), br.astype(np.float64)
    ulp = 2.0 ** -23
    for i in range(u.shape[0]):
        bc = 0.5 * (bl64[i] + br64[i])  # exact in FP64 from FP32 inputs
        ref = O.recover(u64[i], bc, GAMMA)
        ke = 0.5 * (u64[i, 1:4] @ u64[i, 1:4]) / u64[i, 0]
        me = 0.5 * (bc @ bc)
        assert w[i, 0] == ref[0]
        assert np.all(np.abs(w[i, 1:4] - ref[1:4]) <= 4 * ulp * np.abs(ref[1:4])), (i, w[i], ref)
        assert np.all(np.abs(w[i, 5:8] - ref[5:8]) <= 0.5 * ulp * np.abs(ref[5:8])), (i, w[i], ref)
        if ref[4] > 0:
            tol = 2 * ulp * abs(ref[4]) + 2.0 ** -44 * (GAMMA - 1.0) * (ke + me)
            assert abs(w[i, 4] - ref[4]) <= tol, (i, w[i, 4], ref[4], tol)
