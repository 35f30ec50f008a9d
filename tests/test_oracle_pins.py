"""The CPU oracle against its pins (closed forms, hand-worked examples, brute
force, exact symmetries, special cases of the paper's definitions)."""
import pytest

import oracle
import oracle_pins


@pytest.fixture(scope="module")
def L():
    return oracle.lib()


@pytest.mark.parametrize("pin", oracle_pins.PINS, ids=lambda p: p.__name__)
def test_pin(L, pin):
    pin(L)
