"""The oracle of GMRES-SDR against the pins in tests/oracle_pins.py."""
import pytest

import oracle_pins as P
from oracle import sdr


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(sdr)
