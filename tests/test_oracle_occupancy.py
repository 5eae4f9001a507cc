"""The occupancy-construction oracle against its pins, and planted mistakes
in copies of it that some pin must catch (CPU)."""
import importlib.util
import os

import pytest

import oracle.occupancy as O
from tests.oracle_occupancy_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(O.__file__), "occupancy.py")

MUTANTS = {
    "median_as_mean": ("c = [percentile_linear(mu[:, a], 0.5) for a in range(3)]",
                       "c = [float(np.mean(mu[:, a], dtype=np.float64)) for a in range(3)]"),
    "p98_for_p99": ("r_fg = percentile_linear(radial_distances(mu, c), 0.99)",
                    "r_fg = percentile_linear(radial_distances(mu, c), 0.98)"),
    "round_for_ceil": ("b = max(math.ceil(pad * r_fg), 1)", "b = max(round(pad * r_fg), 1)"),
    "pad_dropped": ("b = max(math.ceil(pad * r_fg), 1)", "b = max(math.ceil(r_fg), 1)"),
    "min_for_max": ("h = max(alpha_v * s_bar, beta_v * r_fg / g0)",
                    "h = min(alpha_v * s_bar, beta_v * r_fg / g0)"),
    "scene_term_from_b": ("h = max(alpha_v * s_bar, beta_v * r_fg / g0)",
                          "h = max(alpha_v * s_bar, beta_v * b / g0)"),
    "cap_keeps_h": ("        h = 2.0 * b / g_max\n", "        pass\n"),
    "smaller_scale": ("smax = np.maximum(", "smax = np.minimum("),
    "closed_cube": ("keep = np.all((x >= 0.0) & (x < 2.0 * b), axis=1)",
                    "keep = np.all((x >= 0.0) & (x <= 2.0 * b), axis=1)"),
    "strict_floor": ("active = rho >= tau_tf", "active = rho > tau_tf"),
    "y_for_x_index": ("lin = (idx[:, 2] * g + idx[:, 1]) * g + idx[:, 0]",
                      "lin = (idx[:, 2] * g + idx[:, 0]) * g + idx[:, 1]"),
}


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_occupancy_pin(pin):
    pin(O)


def _mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {name}: the planted line is not unique"
    src = src.replace(old, new).replace("from .weighting import", "from oracle.weighting import")
    spec = importlib.util.spec_from_loader(f"occupancy_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src, f"<{name}>", "exec"), mod.__dict__)
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
