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


# ------------------------------------------- convolution / light-curve oracle (Python)
import importlib.util  # noqa: E402
import inspect  # noqa: E402

import test_oracle_lightcurve as PL  # noqa: E402
from oracle import lightcurve as _LC  # noqa: E402

LC_MUTATIONS = [
    ("gauss_unnormalised", "return w / w.sum()", "return w"),
    ("gauss_axes_swapped", "wx, wy = gaussian_weights(size, dx), gaussian_weights(size, dy)",
     "wx, wy = gaussian_weights(size, dy), gaussian_weights(size, dx)"),
    ("gauss_3_sigma", "k = int(math.ceil(4.0 * sigma / d))", "k = int(math.ceil(3.0 * sigma / d))"),
    ("disk_strict_edge", "<= radius * radius:", "< radius * radius:"),
    ("disk_drops_scale", "f = scale / len(offs)", "f = 1.0 / len(offs)"),
    ("shift_sign", "s[j0:j1, i0:i1] = c[j0 + dj:j1 + dj, i0 + di:i1 + di]",
     "s[j0:j1, i0:i1] = c[j0 - dj:j1 - dj, i0 - di:i1 - di]"),
    ("mu_scale_drops_dy", "return a_lens / (rays.nx * rays.ny * dx * dy)", "return a_lens / (rays.nx * rays.ny * dx * dx)"),
    ("curve_not_centred", "u = (bx - src.x0) / dx - 0.5", "u = (bx - src.x0) / dx"),
    ("curve_fx_fy_swapped", "out[k] = ((1 - fy) * ((1 - fx)", "out[k] = ((1 - fx) * ((1 - fy)"),
]


def _lc_mutant(name, orig, mut):
    src = inspect.getsource(_LC)
    assert orig in src, f"mutation anchor for {name} not found"
    spec = importlib.util.spec_from_loader(f"lc_mut_{name}", loader=None)
    mod = importlib.util.module_from_spec(spec)
    exec(compile(src.replace(orig, mut, 1), f"lc_mut_{name}", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name,orig,mut", LC_MUTATIONS, ids=[m[0] for m in LC_MUTATIONS])
def test_light_curve_pins_catch_planted_mistake(name, orig, mut, monkeypatch):
    monkeypatch.setattr(PL, "LC", _lc_mutant(name, orig, mut))
    failed = []
    for t in [getattr(PL, n) for n in dir(PL) if n.startswith("test_")]:
        params = inspect.signature(t).parameters
        cases = [(PL.LC.GAUSSIAN, 0.3), (PL.LC.DISK, 0.45)] if params else [()]
        for args in cases:
            try:
                t(*args)
            except Exception as e:  # an assertion or a crash
                failed.append(f"{t.__name__}:{type(e).__name__}")
    assert failed, f"no pin caught mutation {name}"
