"""The oracle's pins catch plausible mistakes: each mutant below plants one mistake in a copy of the oracle's C
source (a wrong rounding, tie break, threshold, weight, sign, index or normalisation), compiled on the side; the
pin tests run against it must fail.  The unmutated copy, built the same way, must pass.  CPU only; the mutants are
never written over the real source."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "exw_oracle.c")

# name: (text in exw_oracle.c, replacement)
MUTANTS = {
    # stage (a): target rounding, tie break, axes
    "round_half_down": ("double t = floor(0.5 + d);", "double t = ceil(d - 0.5);"),
    "tie_to_larger_index": ("if (key < keys[q]) keys[q] = key;",
                            "if (key < keys[q] || ((key >> 32) == (keys[q] >> 32) && key > keys[q] && "
                            "keys[q] != ORACLE_EMPTY)) keys[q] = key;"),
    "y_offset_from_x_motion": ("if (!oracle_target_offset(my, k, denom, &oy)) continue;",
                               "if (!oracle_target_offset(mx, k, denom, &oy)) continue;"),
    # stage (b): mask, weights, taps, participation, normalisation
    "crack_at_two_neighbours": ("if (count >= 3) m = MASK_CRACK;", "if (count >= 2) m = MASK_CRACK;"),
    "swapped_weights": ("off[0] = 0; w[0] = 1.0 - fabs(rho); dw[0] = -(double)s;",
                        "off[0] = 0; w[0] = fabs(rho); dw[0] = (double)s;"),
    "tap_on_wrong_side": ("off[1] = s; w[1] = fabs(rho);", "off[1] = -s; w[1] = fabs(rho);"),
    "no_renormalisation": ("out[c * n + q] = num[c] / den;", "out[c * n + q] = num[c];"),
    "participation_tau_1_16": ("return fabs(Dt - Dp) <= Dp / 32.0;", "return fabs(Dt - Dp) <= Dp / 16.0;"),
    # adjoint
    "dropped_quotient_term": ("const double diff = color[c * n + tidx[j]] - outc[c];",
                              "const double diff = color[c * n + tidx[j]];"),
    "adjoint_sign": ("const double scale = -(double)k / (double)denom;",
                     "const double scale = (double)k / (double)denom;"),
    # stage (c)
    "push_from_transposed_parent": ("(size_t)(i >> 1) * Wp + (j >> 1);", "(size_t)(j >> 1) * Wp + (i >> 1);"),
    "pull_first_valid_child_only": ("if (!m[cidx]) continue;", "if (!m[cidx] || cnt > 0) continue;"),
    # motion bounds
    "bounds_without_clamp": ("mx = mx < -65536.0f ? -65536.0f : (mx > 65536.0f ? 65536.0f : mx);", ""),
    # frame statistics
    "variance_divides_by_n_minus_1": ("out[1] = vx / cnt;", "out[1] = vx / (cnt - 1.0);"),
    "variance_y_about_x_mean": ("dy = (double)mv[n + i] - my;", "dy = (double)mv[n + i] - mx;"),
    "mse_over_two_channels": ("const size_t n = 3 * (size_t)W * (size_t)H;\n    double s = 0.0;",
                              "const size_t n = 2 * (size_t)W * (size_t)H;\n    double s = 0.0;"),
    "ssim_sigma_1": ("(2.0 * 1.5 * 1.5)", "(2.0 * 1.0 * 1.0)"),
    "ssim_c2_of_0_02": ("C2 = 0.03 * 0.03", "C2 = 0.02 * 0.02"),
    # recursive warps
    "carry_through_cracks": ("if (mask[q] == 0 && keys[q] != ORACLE_EMPTY) {", "if (keys[q] != ORACLE_EMPTY) {"),
    "carry_y_motion_from_x": ("mv_out[n + q] = mv[n + p];", "mv_out[n + q] = mv[p];"),
}


def _run_pins(lib: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, EXW_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                           "-q", "-p", "no:cacheprovider"], capture_output=True, text=True, env=env, cwd=ROOT,
                          timeout=900)


def test_every_mutant_fails_a_pin(tmp_path):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    orig = open(SRC).read()
    jobs = {"unmutated": orig}
    for name, (old, new) in MUTANTS.items():
        assert orig.count(old) == 1, f"{name}: the mutated text must occur exactly once"
        jobs[name] = orig.replace(old, new)
    libs = {}
    for name, text in jobs.items():
        src = tmp_path / f"{name}.c"
        src.write_text(text)
        libs[name] = oracle.compile_source(str(src), str(tmp_path / f"lib{name}.so"))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(libs, ex.map(_run_pins, libs.values())))
    base = results.pop("unmutated")
    assert base.returncode == 0, base.stdout[-2000:] + base.stderr[-2000:]
    # exit status 1 = tests ran and failed (not a collection or usage error)
    missed = {name: r.returncode for name, r in results.items() if r.returncode != 1}
    assert not missed, f"mutants not caught (pytest exit status): {missed}"


# Mistakes in the oracle's Python compositions (function: (text in its source, replacement)); each mutant function
# is rebuilt from its edited source inside the pin run's process before the pins are collected.
PY_MUTANTS = {
    "extrapolate_without_storage_rounding": ("extrapolate", "stored = out.astype(storage).astype(np.float64)",
                                             "stored = out"),
    "extrapolate_fill_before_warp_rounding": ("extrapolate", "out = fill_holes(stored, mask)",
                                              "out = fill_holes(out, mask)"),
    "psnr_with_20_log10": ("psnr", "10.0 * np.log10(1.0 / mse)", "20.0 * np.log10(1.0 / mse)"),
    "l2_gradient_without_factor_2": ("l2_loss_grad", "2.0 * diff", "diff"),
    "halo_signed": ("halo", "max(abs(target_offset(float(v), k, denom)) for v in frame_bounds)",
                    "max(target_offset(float(v), k, denom) for v in frame_bounds)"),
    "recursive_warp_without_carry": ("warp_recursive", "d, m = carry_motion(keys, mask, d, m)", "pass"),
}

_PY_RUNNER = """
import inspect, sys, textwrap
sys.path.insert(0, {root!r})
import numpy as np
import oracle
import pytest
src = textwrap.dedent(inspect.getsource(getattr(oracle, {fn!r})))
assert src.count({old!r}) == 1
ns = dict(vars(oracle))
exec(compile(src.replace({old!r}, {new!r}), "mutant", "exec"), ns)
setattr(oracle, {fn!r}, ns[{fn!r}])
sys.exit(pytest.main([{pins!r}, "-x", "-q", "-p", "no:cacheprovider"]))
"""


def _run_py_mutant(spec):
    fn, old, new = spec
    code = _PY_RUNNER.format(root=ROOT, fn=fn, old=old, new=new,
                             pins=os.path.join(ROOT, "tests", "test_oracle_pins.py"))
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=900)


def test_every_python_composition_mutant_fails_a_pin():
    specs = dict(PY_MUTANTS)
    specs["unmutated"] = ("psnr", "10.0 * np.log10(1.0 / mse)", "10.0 * np.log10(1.0 / mse)")
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip(specs, ex.map(_run_py_mutant, specs.values())))
    base = results.pop("unmutated")
    assert base.returncode == 0, base.stdout[-2000:] + base.stderr[-2000:]
    missed = {name: r.returncode for name, r in results.items() if r.returncode != 1}
    assert not missed, f"mutants not caught (pytest exit status): {missed}"
