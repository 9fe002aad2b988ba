"""The CPU oracle against its pins (no GPU)."""
import pytest

from oracle import oracle as O
from tests import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__[4:])
def test_pin(pin):
    pin(O)
