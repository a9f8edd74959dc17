"""The pins must have teeth: plant one plausible mistake at a time in a copy of the
oracle's C source (on the CPU), rebuild it, and check that at least one pin of
test_oracle_pins fails against the mutant.  The real oracle is never modified.
"""
import os
import tempfile

import pytest

import oracle
import test_oracle_pins as P

# (name, original text, mutated text) -- each original must occur in the source
MUTATIONS = [
    ("drop_mass", "sx += m[k] * dx / r2;", "sx += dx / r2;"),
    ("star_y_sign", "sy += m[k] * dy / r2;", "sy -= m[k] * dy / r2;"),
    ("star_y_uses_dx", "sy += m[k] * dy / r2;", "sy += m[k] * dx / r2;"),
    ("r_not_r2", "double r2 = dx * dx + dy * dy;", "double r2 = sqrt(dx * dx + dy * dy);"),
    ("shear1_sign", "double sx = (kc + g1) * tx + g2 * ty;", "double sx = (kc - g1) * tx + g2 * ty;"),
    ("shear2_sign", "double sy = g2 * tx + (kc - g1) * ty;", "double sy = -g2 * tx + (kc - g1) * ty;"),
    ("drop_kappa_c", "double sy = g2 * tx + (kc - g1) * ty;", "double sy = g2 * tx + (-g1) * ty;"),
    ("ray_not_centred", "return g->x0 + ((double)i + 0.5)", "return g->x0 + ((double)i + 0.0)"),
    ("map_transposed", "return (int64_t)uy * s->nx + (int64_t)ux;", "return (int64_t)ux * s->ny + (int64_t)uy;"),
    ("round_not_floor", "double ux = floor((bx - s->x0)", "double ux = round((bx - s->x0)"),
    ("upper_edge_inclusive", "ux >= (double)s->nx", "ux > (double)s->nx"),
    ("pair_drops_lo", "    dl = dl + t;\n", "    dl = dl + 0.0f * t;\n"),
    ("pair_floor_no_fix", "if (p == uh && ul < 0.0f) p = p - 1.0f;", ";"),
]

PINS = [getattr(P, n) for n in dir(P) if n.startswith("test_") and n != "test_sheet_macro_magnification"
        and n != "test_random_field_mean_magnification"]


def _run_pins():
    failed = []
    for t in PINS:
        try:
            t()
        except AssertionError:
            failed.append(t.__name__)
        except Exception as e:  # a crash also counts as caught
            failed.append(f"{t.__name__}:{type(e).__name__}")
    try:
        P.test_sheet_macro_magnification(0.1, -0.25, 0.3)
    except AssertionError:
        failed.append("test_sheet_macro_magnification")
    return failed


@pytest.mark.parametrize("name,orig,mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(name, orig, mut):
    src = oracle.source_text()
    assert orig in src, f"mutation anchor for {name} not found"
    with tempfile.TemporaryDirectory() as d:
        so = oracle.build_variant(src.replace(orig, mut, 1), os.path.join(d, f"mut_{name}.so"))
        with oracle.using(so):
            failed = _run_pins()
    assert failed, f"no pin caught mutation {name}"
