"""Plant plausible mistakes in a copy of the CPU oracle and check that the pins
catch every one of them.  This guards the pins themselves: a pin set that a
dropped term, a wrong sign or a transposed operand survives is too weak.

Mutants are compiled from a text-edited copy of oracle/qca_oracle.c in a
temporary directory; the committed oracle is never modified.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from golden_cases import all_cases
from test_oracle import _closed_form, _prose_link

SRC = os.path.join(os.path.dirname(oracle.__file__), "qca_oracle.c")
SRC_1D = os.path.join(os.path.dirname(SRC), "qca_oracle_1d.c")
SRC_VAR = os.path.join(os.path.dirname(SRC), "qca_oracle_variants.c")
HDR = os.path.join(os.path.dirname(oracle.__file__), "qca_oracle.h")

MUTANTS = {
    "zero_is_smallest_in_force": ("if (mplus == 0) return -1;", "if (mplus == 0) return +1;"),
    "tie_order_reversed": ("(val == bv && sa < bsa)", "(val == bv && sa > bsa)"),
    "feedback_xor_not_or": ("return (xv == 1 || yv == 1) ? 1 : 0;",
                            "return ((xv == 1) != (yv == 1)) ? 1 : 0;"),
    "min_includes_empty": ("if (val > 0 && (best == 0 || val < best)) best = val;",
                           "if (best == 0 || val < best) best = val;"),
    "cap_saturates": ("if (nv > m_max) nv = 0;", "if (nv > m_max) nv = m_max;"),
    "normal_ball_transposed": ("out[j + 1] = site(x, y + j, L); /* normal to x^: vary y */",
                               "out[j + 1] = site(x + j, y, L); /* normal to x^: vary y */"),
    "upstream_sign": ("int ux = x - (a == 1 ? s : 0);", "int ux = x + (a == 1 ? s : 0);"),
    "syndrome_drops_term": ("^ ey[site(x, y, L)] ^\n                   ey[site(x, y - 1, L)];",
                            "^ ey[site(x, y, L)];"),
    "cut_uses_wrong_plane": ("px ^= R[site(0, y, L)];", "px ^= R[LL + site(0, y, L)];"),
    "force_axis_swapped": ("f[(size_t)(a - 1) * LL + r] = (int8_t)force_sign(mp, mm);",
                           "f[(size_t)(2 - a) * LL + r] = (int8_t)force_sign(mp, mm);"),
}


def _battery(mod):
    """Run the pins on the currently loaded oracle library; return the names of
    the pins that failed."""
    failed = []
    for case in all_cases():
        C, steps, flag = mod.decode_shot(case["N"], m_max=case["m_max"],
                                         max_steps=case["max_steps"])
        if steps != case["steps"] or flag != case["flag"] or not np.array_equal(C, case["C"]):
            failed.append("golden:" + case["name"])
    rng = np.random.default_rng(3)
    for L in (5, 7):
        anyon = rng.random((L, L)) < 0.08
        anyon[0, 0] = True
        sigma = np.where(anyon, -1, 1).astype(np.int8)
        m = np.zeros((4, L, L), np.int32)
        for t in range(1, L + 2):
            m = mod.message_substep(sigma, m, m_max=4)
            if not np.array_equal(m, _closed_form(anyon, t, 4)):
                failed.append(f"closed_form:L{L}")
                break
    L, x0, y0 = 5, 2, 2
    sigma = np.ones((L, L), np.int8)
    sigma[y0, x0] = -1
    for vals in [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (2, 2, 3, 0), (1, 2, 1, 3)]:
        m = np.zeros((4, L, L), np.int32)
        m[:, y0, x0] = vals
        F = mod.feedback_links(sigma, mod.forces(sigma, m))
        want = np.zeros((2, L, L), np.uint8)
        mv = _prose_link(*vals)
        if mv is not None:
            a, d = mv
            if a == 1:
                want[0, y0, x0 if d > 0 else x0 - 1] = 1
            else:
                want[1, y0 if d > 0 else y0 - 1, x0] = 1
        if not np.array_equal(F, want):
            failed.append(f"prose_force:{vals}")
    N = np.zeros((2, 6, 6), np.uint8)
    N[0, 2, 4] = 1
    if sorted(zip(*np.nonzero(mod.syndrome(N) == -1))) != [(2, 4), (2, 5)]:
        failed.append("syndrome_single_link")
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/found"
    d = tmp_path / "mut"
    d.mkdir()
    shutil.copy(HDR, d / "qca_oracle.h")
    (d / "qca_oracle.c").write_text(src.replace(old, new))
    lib = d / "libmut.so"
    shutil.copy(SRC_1D, d / "qca_oracle_1d.c")
    shutil.copy(SRC_VAR, d / "qca_oracle_variants.c")
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib),
                    str(d / "qca_oracle.c"), str(d / "qca_oracle_1d.c"),
                    str(d / "qca_oracle_variants.c"), "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: str(lib))
    try:
        failed = _battery(oracle)
    finally:
        oracle._lib = None
    assert failed, f"mutant {name} survived every pin"


def test_unmutated_oracle_passes_battery(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", None)
    try:
        assert _battery(oracle) == []
    finally:
        oracle._lib = None
