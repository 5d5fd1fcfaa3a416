"""The reference decoder against the paper, closed forms, library routines and hand-worked traces."""
import pytest

import oracle as oracle_pkg
import oracle_pins


@pytest.fixture(scope="module")
def O():
    return oracle_pkg.load()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(O, pin):
    pin(O)
