"""The FP64 oracle against closed forms, invariants, finite differences,
CAS-derived kernels and high-precision brute force (no GPU)."""
import pytest

import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin, oracle_lib):
    pin(oracle_lib)


def test_uniform_sphere_field(oracle_lib):
    P.pin_uniform_sphere_field(oracle_lib)


def test_plummer_field(oracle_lib):
    P.pin_plummer_field(oracle_lib)
