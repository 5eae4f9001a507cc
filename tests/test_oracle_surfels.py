"""The voxel-to-surfel oracle against its pins, and planted mistakes in
copies of it that some pin must catch (CPU)."""
import importlib.util
import os

import pytest

import oracle.surfels as S
from tests.oracle_surfels_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(S.__file__), "surfels.py")

MUTANTS = {
    "three_sigma_box": ("ex = max(abs(a0[0]), abs(a1[0]))", "ex = 3 * max(abs(a0[0]), abs(a1[0]))"),
    "one_sigma_ellipse": ("            if r2 <= 9.0:", "            if r2 <= 1.0:"),
    "mean_over_views": ("kappa[i] = max(kappa[i], msk / max(tot, 1))",
                        "kappa[i] = 0.5 * (kappa[i] + msk / max(tot, 1))"),
    "aspect_inverted": ("return (np.maximum(s[:, 0], s[:, 1]) / (np.minimum(s[:, 0], s[:, 1]) + EPS_ASPECT))",
                        "return (np.minimum(s[:, 0], s[:, 1]) / (np.maximum(s[:, 0], s[:, 1]) + EPS_ASPECT))"),
    "p98": ("tau_a = percentile_linear(a, 0.99)", "tau_a = percentile_linear(a, 0.98)"),
    "gating_ignored": ("if not (int(voxel_bits[i]) >> sidx) & 1 or sidx >= 32:", "if sidx >= 32:"),
    "normal_as_tangent": ("t1 = float(np.float32(s[1])) * R[:, 1]", "t1 = float(np.float32(s[1])) * R[:, 2]"),
    "pixel_corner": ("dx, dy = x + 0.5 - c[0], y + 0.5 - c[1]", "dx, dy = x - c[0], y - c[1]"),
    "tip_not_halved": ("a0 = 0.5 * (proj[1][1] - proj[2][1])", "a0 = proj[1][1] - proj[2][1]"),
    "strict_coverage": ("if msk >= tau_kappa * max(tot, 1):", "if msk > tau_kappa * max(tot, 1):"),
}


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda f: f.__name__)
def test_surfels_pin(pin):
    pin(S)


def _mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutant {name}: the planted line is not unique"
    src = src.replace(old, new).replace("from .weighting import", "from oracle.weighting import")
    spec = importlib.util.spec_from_loader(f"surfels_{name}", loader=None)
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
