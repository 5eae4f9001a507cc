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


def test_gradient_fd_at_config4_size():
    """Every pixel with a nonzero analytic gradient (at most 600 per view and
    leaf; a 32^3 grid seen at 1008 x 756 has fewer) plus 100 random pixels per
    view and leaf."""
    checked, excluded = pins.gradient_fd_config4_size(oracle)
    assert checked > 600, (checked, excluded)
