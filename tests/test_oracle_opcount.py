"""The algorithmic FP operation count per cell update (the denominator-side
figure of the ALU roofline) from the oracle's formulas with a counting type."""
from oracle import oracle as O


def test_recovery_count_by_hand():
    # 1/rho; 3 velocities; ke: 3 mul + 2 add + 1 mul; me: same; p: 2 sub + 1 mul
    assert O.flops_recovery() == 19


def test_cell_update_count_range_and_determinism():
    a = O.flops_per_cell_update(3, 2000, 1)
    b = O.flops_per_cell_update(3, 2000, 1)
    assert a == b
    assert 1200 < a < 2200, a
    c = O.flops_per_cell_update(2, 2000, 1)
    assert 700 < c < a, c
