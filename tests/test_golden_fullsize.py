"""The stored oracle fixes of the full-size workloads
(``tests/golden/fullsize_fix.json``): every case the GPU tests compare with
is present, converged, written by the committed script, and consistent with
the recipe of its input.  A pin of the oracle itself at full size: the
stored F must lie above the input's F (the steepest descent raises F) and
below 1 (F = 1 only for unit links), and theta must be below 1e-15."""
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "fullsize_fix.json")

CASES = {
    "32^4": ((32, 32, 32, 32), 0, 0.5),
    "48^3x8": ((48, 48, 48, 8), 0, 0.6),
    "48^3x12": ((48, 48, 48, 12), 0, 0.6),
    "batch member 0 16^4": ((16, 16, 16, 16), 0, 0.5),
    "batch member 1 24^3x48": ((24, 24, 24, 48), 1, 0.5),
    "batch member 2 32^3x8": ((32, 32, 32, 8), 2, 0.5),
    "batch member 3 20^4": ((20, 20, 20, 20), 3, 0.5),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_stored_oracle_fix(case):
    with open(GOLDEN) as f:
        data = json.load(f)
    assert "make_fullsize_fix.py" in data["source"]
    rec = data["cases"][case]
    dims, seed, scale = CASES[case]
    assert tuple(rec["dims"]) == dims and rec["seed"] == seed and rec["link_scale"] == scale
    assert rec["gauge_scale"] == 1.0 and rec["alpha"] == 0.08 and rec["theta_tol"] == 1e-15
    assert rec["converged"] and rec["theta"] < 1e-15
    assert rec["F_input"] < rec["F"] < 1.0
    assert 0 < rec["iterations"] < 2000


def test_recipe_matches_the_script():
    """The script that writes the file builds the same cases."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mk", os.path.join(HERE, "golden", "make_fullsize_fix.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    assert {k: (tuple(v[0]), v[1], v[2]) for k, v in mk.CASES.items()} == CASES
