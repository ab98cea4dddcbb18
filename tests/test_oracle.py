"""The CPU oracle against the paper's printed values, closed forms, LTLf
identities and brute force over all syntax trees (see ``tests/pins.py``)."""
import pytest

import oracle
from tests import pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load_library(oracle.build())


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin, lib):
    pin(lib)
