"""The depth-weighting oracle against its pins, and planted mistakes in
copies of it that some pin must catch (CPU)."""
import importlib.util
import os

import pytest

import oracle.weighting as W
from tests.oracle_weighting_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(W.__file__), "weighting.py")

MUTANTS = {
    "rank_k_plus_one": ("return float(s[k] + (r - k) * (s[k + 1] - s[k]))",
                        "return float(s[k + 1])"),
    "q_as_percent": ("d_far = percentile_linear(D, 0.98)", "d_far = percentile_linear(D, 0.99)"),
    "nerf_not_inverted": ("w = np.where(fin, 1.0 - zhat, 0.0)", "w = np.where(fin, zhat, 0.0)"),
    "nerf_max_min_swapped": ("zhat[fin] = (D[fin] - lo) / (hi - lo)",
                             "zhat[fin] = (hi - D[fin]) / (hi - lo)"),
    "centre_dropped": ("[(int(x), int(y)) for x, y in prompts] + [(W // 2, H // 2)]",
                       "[(int(x), int(y)) for x, y in prompts]"),
    "centre_transposed": ("[(W // 2, H // 2)]", "[(H // 2, W // 2)]"),
    "no_clip": ("band = np.clip((dm + dp) / den, 0.0, 1.0)", "band = (dm + dp) / den"),
    "den_from_d_min": ("den = max(d_far - d_max, 1e-6)", "den = max(d_far - d_min, 1e-6)"),
    "lower_side_dropped": ("band = np.clip((dm + dp) / den, 0.0, 1.0)",
                           "band = np.clip(dp / den, 0.0, 1.0)"),
    "nonfinite_kept": ("w = np.where(fin, 1.0 - band, 0.0)",
                       "w = np.where(fin, 1.0 - band, 1.0)"),
}


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_weighting_pin(pin):
    pin(W)


def _mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {name}: the planted line is not unique"
    spec = importlib.util.spec_from_loader(f"weighting_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src.replace(old, new), f"<{name}>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    mod = _mutant(name)
    for pin in ALL_PINS:
        try:
            pin(mod)
        except (AssertionError, IndexError, ValueError, ZeroDivisionError):
            return
    pytest.fail(f"no pin catches the planted mistake {name}")
