"""The CPU oracle against the paper's printed numbers, closed forms, brute
force and library routines (no GPU)."""
import pytest

import oracle_pins


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda f: f.__name__[6:])
def test_oracle_pin(orc, check):
    check(orc)
