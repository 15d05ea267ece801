"""The FP64 oracle against what the paper and mathematics fix (CPU only).

Each pin is documented in ``pins.py``; together they tie every term of the
leapfrog (Eqs. 17-26), the winding and cell-overlap detection (Sec. III.A-B)
and the diagnostics (Eqs. 31-37) to closed forms, invariants, brute force or
an independent ODE solution.
"""
import pytest

import pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()
