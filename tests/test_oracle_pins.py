"""The oracle checked against the paper and mathematics (CPU only)."""
import pytest

from oracle.oracle import load_oracle
from tests.oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(load_oracle())
