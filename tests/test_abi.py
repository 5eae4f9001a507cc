"""The C-ABI library loads and exports every entry point its header declares (CPU)."""
import os
import re
import subprocess

import paper_2601_04860_b300.build as B
from paper_2601_04860_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "divas_fuse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(divas_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    B.build()
    lib = L.load()
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (divas_\w+)", out))
    assert set(names) <= exported
    # the binding knows every declared call
    assert set(names) <= set(L.EXPORTED)


def test_default_params_match_paper_constants():
    import ctypes
    import json
    p = L.DivasParams()
    L.load().divas_default_params(ctypes.byref(p))
    c = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    assert p.tau_mask == c["mask_gate"]["value"]
    assert p.tau_cons == c["tau_cons"]["value"]
    assert p.gamma == c["gamma_gs"]["value"]


def test_default_tuple_params_match_paper_constants():
    import json
    import math
    p = L.load().divas_default_tuple_params()
    c = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    f32 = lambda v: float(__import__("numpy").float32(v))  # noqa: E731
    assert p.beta == f32(c["beta_gs"]["value"])
    assert p.gamma_st == f32(c["gamma_st"]["value"])
    assert p.tau_thin == f32(c["tau_thin"]["value"])
    assert p.rho_cover == f32(c["rho_cover"]["value"])
    assert p.rho_occ == f32(c["rho_occ"]["value"])
    assert p.n_abs == c["n_abs"]["value"]
    assert p.dist_gate == c["dist_gate_hv"]["value"]
    assert p.behind_margin == c["behind_margin_hv"]["value"]
    assert p.k_dg == 0.0 and p.rho_thin == 1.0 and not math.isnan(p.beta)
