"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import json
import os

import pytest

import oracle
from tests import oracle_pins as pins

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle)


def test_oracle_defaults_match_paper_constants():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as f:
        c = json.load(f)
    p = oracle.Params()
    assert p.tau_m == c["mask_gate"]["value"]
    assert p.tau_cons == c["tau_cons"]["value"]
    assert p.gamma == c["gamma_gs"]["value"]
