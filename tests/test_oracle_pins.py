"""The FP64 oracle against its pins (closed forms, dense unitaries, Bloch
rotations, finite differences, parameter shift, the paper's parameter count)."""
import pytest

import oracle
import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle.default())


def test_paper_parameter_count():
    P.pin_paper_parameter_count()
