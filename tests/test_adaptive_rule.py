"""Host logic of the consensus-penalty balancing rule (no GPU needed)."""
from paper_2011_00162_gb300 import adaptive


def test_decide_balances_and_clamps():
    assert adaptive.decide(1.0, 1.0, 1.0) == 1.0          # balanced: unchanged
    assert adaptive.decide(1.0, 11.0, 1.0) == 2.0         # primal lags: raise r
    assert adaptive.decide(1.0, 1.0, 11.0) == 0.5         # dual lags: lower r
    assert adaptive.decide(1.0, 10.0, 1.0) == 1.0         # the ratio is strict
    assert adaptive.decide(3e3, 1e3, 1.0, r_max=4e3) == 4e3
    assert adaptive.decide(2e-4, 1.0, 1e3, r_min=1.5e-4) == 1.5e-4
    assert adaptive.decide(1.0, 5.0, 1.0, ratio=4.0, factor=3.0) == 3.0
