"""The CPU oracle against what the paper and mathematics fix (no GPU needed)."""
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def o():
    return oracle.Oracle()


@pytest.mark.parametrize("pin", P.FAST_PINS, ids=lambda f: f.__name__)
def test_fast_pin(o, pin):
    pin(o)


@pytest.mark.parametrize("pin", P.SLOW_PINS, ids=lambda f: f.__name__)
def test_statistical_pin(o, pin):
    pin(o)
