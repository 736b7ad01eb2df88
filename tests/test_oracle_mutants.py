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
    "budget_off_by_one": ("if (t >= max_steps) {\n      flag = 2;",
                          "if (t > max_steps) {\n      flag = 2;"),
    "cap_off_by_one": ("if (nv > m_max) nv = 0;", "if (nv >= m_max) nv = 0;"),
    "feedback_one_sided": ("(uint8_t)or_pm(t1, t2);", "(uint8_t)or_pm(t1, 0);"),
    "anyon_test_centre_only": ("if (sigma[C[i]] == -1) anyon = 1;",
                               "if (i == 1 && sigma[C[i]] == -1) anyon = 1;"),
    "one_substep_short": ("for (int i = 0; i < v; ++i) {\n    qo_message_substep",
                          "for (int i = 1; i < v; ++i) {\n    qo_message_substep"),
    "correction_overwritten": ("for (size_t i = 0; i < 2 * LL; ++i) C[i] ^= F[i];",
                               "for (size_t i = 0; i < 2 * LL; ++i) C[i] = F[i];"),
    "literal_key_ties_to_nearer": ("(key == bkey && val > bv)", "(key == bkey && val < bv)"),
    "literal_key_offset_sign": ("key = 3 * (int64_t)val + sa, bkey = 3 * (int64_t)bv + bsa;",
                                "key = 3 * (int64_t)val - sa, bkey = 3 * (int64_t)bv - bsa;"),
    "balanced_draw_sign": ("(int8_t)((u >> 63) ? +1 : -1);", "(int8_t)((u >> 63) ? -1 : +1);"),
    "balanced_draw_drops_step": ("const uint64_t k2 = qo_splitmix64(k1 ^ (uint64_t)(uint32_t)t);\n  for (size_t r = 0; r < LL; ++r) {\n    if (!balanced[r])",
                                 "const uint64_t k2 = k1;\n  for (size_t r = 0; r < LL; ++r) {\n    if (!balanced[r])"),
}


# Planted mistakes in the 1D oracle (Sec. 3.1) and in the open-boundary
# variant (appendix on open boundary conditions), each caught by the pins of
# tests/test_oracle_1d.py or tests/test_oracle_variants.py.
MUTANTS_1D = {
    "1d_empty_is_smallest": ("f[r] = -1; /* sgn(-inf + m^-) */", "f[r] = 1; /* sgn(-inf + m^-) */"),
    "1d_force_sign": ("f[r] = (int8_t)((d > 0) - (d < 0));", "f[r] = (int8_t)((d < 0) - (d > 0));"),
    "1d_feedback_xor_not_or": ("flips[r] = (t1 == 1 || t2 == 1) ? 1 : 0;",
                               "flips[r] = ((t1 == 1) != (t2 == 1)) ? 1 : 0;"),
    "1d_upstream_sign": ("const int u = w1(r - s, L);", "const int u = w1(r + s, L);"),
    "1d_cap_saturates": ("if (nv > m_max) nv = 0;", "if (nv > m_max) nv = m_max;"),
    "1d_syndrome_drops_term": ("sigma[r] = (links[w1(r - 1, L)] ^ links[r]) ? -1 : 1;",
                               "sigma[r] = links[r] ? -1 : 1;"),
}
MUTANTS_OPEN = {
    "open_boundary_not_a_source": ("nv = 1; /* the rough boundary sources messages into the bulk */",
                                   "nv = 0; /* the rough boundary sources messages into the bulk */"),
    "open_syndrome_counts_boundary": ("      if (!is_bdry(x, L)) {\n        if (qo_open_link_exists",
                                      "      if (1) {\n        if (qo_open_link_exists"),
    "open_y_links_on_rough_columns": ("return x >= 1 && x <= L - 2 && y <= L - 2;",
                                      "return x <= L - 2 && y <= L - 2;"),
    "open_feedback_xor_not_or": ("F[a * LL + r] = (t1 == 1 || t2 == 1) ? 1 : 0;",
                                 "F[a * LL + r] = ((t1 == 1) != (t2 == 1)) ? 1 : 0;"),
    "open_cone_drops_transverse": ("for (int j = -1; j <= 1; ++j) {\n            const int xx = ax ? ux : ux + j",
                                   "for (int j = 0; j <= 0; ++j) {\n            const int xx = ax ? ux : ux + j"),
}

MUTANTS_DESYNC = {
    "desync_move_at_message_rate": ("(uint64_t)(2 * i + 1)) < thr_move;",
                                    "(uint64_t)(2 * i + 1)) < thr_msg;"),
    "desync_every_site_updates": ("if (!fire)\n        for (int k = 0; k < 4; ++k)",
                                  "if (0)\n        for (int k = 0; k < 4; ++k)"),
    "desync_one_draw_for_both_clocks": ("(uint64_t)(2 * i + 1)) < thr_move;",
                                        "(uint64_t)(2 * i)) < thr_move;"),
}


# Planted mistakes in the pre-decoder's reference (oracle/net.py), each caught
# by the pins of tests/test_net_oracle.py.
NET_SRC = os.path.join(os.path.dirname(oracle.__file__), "net.py")
MUTANTS_NET = {
    "net_conv_tap_shift_sign": (
        "shifted = np.roll(x, shift=(1 - ky, 1 - kx), axis=(1, 2))\n            out +=",
        "shifted = np.roll(x, shift=(ky - 1, kx - 1), axis=(1, 2))\n            out +="),
    "net_relu_on_logits": ("        x = conv3x3_circular(x, W, b)\n        if i < len(layers) - 1:",
                           "        x = conv3x3_circular(x, W, b)\n        if True:"),
    "net_bf16_truncates": ("u = ((u + 0x7FFF + lsb) >> 16) << 16", "u = (u >> 16) << 16"),
    "net_labels_skip_partner_check": ("if anyon[yn, xn] and d[yn, xn] == back:",
                                      "if anyon[yn, xn]:"),
    "net_labels_y_directions_swapped": ("d[f[1] == -1] = 2\n    d[f[1] == 1] = 3",
                                        "d[f[1] == -1] = 3\n    d[f[1] == 1] = 2"),
    "net_pairing_roll_direction": ("C0[0] = ((prop == 0) & (np.roll(prop, -1, axis=1) == 1))",
                                   "C0[0] = ((prop == 0) & (np.roll(prop, 1, axis=1) == 1))"),
    "net_zero_logit_proposes": ("np.where(best > 0.0, k, 4)", "np.where(best >= 0.0, k, 4)"),
    "net_e4m3_no_saturation": ("q = np.minimum(q, E4M3_MAX)", "q = q"),
    "net_e4m3_no_subnormals": ("e = np.maximum(E - 1, -6)", "e = E - 1"),
    "net_fp8_scale_per_tensor": (
        "amax = np.max(np.abs(W.astype(np.float32)).reshape(W.shape[0], -1), axis=1)",
        "amax = np.full(W.shape[0], np.max(np.abs(W.astype(np.float32))))"),
    "net_label_smoothing_off": ("LABEL_SMOOTHING = 0.1", "LABEL_SMOOTHING = 0.0"),
    "net_fifth_class_logit_one": ("zz = np.concatenate([z, np.zeros((1,) + z.shape[1:])])",
                                  "zz = np.concatenate([z, np.ones((1,) + z.shape[1:])])"),
}


def _run_pins(fns):
    """Call pin functions; return the names of those that failed (a pin that
    raises on a mutant catches it as surely as one whose assertion fails)."""
    failed = []
    for name, fn in fns:
        try:
            fn()
        except Exception:
            failed.append(name)
    return failed


def _battery_1d():
    import test_oracle_1d as t
    fns = [(f"messages_L{L}", (lambda L=L: t.test_messages_are_upstream_distances(L)))
           for L in (5, 7)]
    fns += [(n, getattr(t, n)) for n in (
        "test_force_rule_against_the_prose", "test_feedback_or_and_direction",
        "test_single_error_one_step", "test_gap_of_two_meets_in_the_middle",
        "test_balanced_antipodal_pair_never_moves",
        "test_long_way_round_is_a_logical_error_but_matches_the_majority",
        "test_invariants_on_random_noise",
        "test_gerrymander_flips_the_logical_state_in_about_035_L",
        "test_gerrymander_under_the_message_cap_strands_a_pair")]
    return _run_pins(fns)


def _battery_open():
    import test_oracle_variants as t
    fns = [(f"open_messages_L{L}",
            (lambda L=L: t.test_open_messages_are_distances_to_anyons_or_the_boundary(L)))
           for L in (5, 6)]
    fns += [(n, getattr(t, n)) for n in (
        "test_open_link_set", "test_open_syndrome_ignores_missing_links_and_boundary",
        "test_open_single_boundary_error_absorbed", "test_open_bulk_pair_fuses_in_one_step",
        "test_open_boundary_to_boundary_string_is_a_logical_error",
        "test_open_anyon_prefers_the_nearer_boundary", "test_open_invariants_on_random_noise")]
    return _run_pins(fns)


def _battery_desync():
    import test_oracle_variants as t
    return _run_pins([(n, getattr(t, n)) for n in (
        "test_desync_full_rate_unit_speed_is_the_synchronous_decoder",
        "test_desync_first_tick_fusion_rate", "test_desync_no_moves_never_decodes")])


def _battery(mod):
    """Run the pins on the currently loaded oracle library; return the names of
    the pins that failed."""
    failed = []
    for case in all_cases():
        for tie in case["tie_orders"]:
            C, steps, flag = mod.decode_shot(case["N"], m_max=case["m_max"],
                                             max_steps=case["max_steps"], tie_order=tie)
            if steps != case["steps"] or flag != case["flag"] or not np.array_equal(C, case["C"]):
                failed.append(f"golden:{case['name']}:tie{tie}")
    import test_oracle as t
    failed += _run_pins([("balanced_random_rule", lambda: t.test_balanced_random_rule(mod))])
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


def _mutant_lib(tmp_path, target, old, new):
    """Build the oracle with one source file text-edited; return the library."""
    d = tmp_path / "mut"
    d.mkdir()
    shutil.copy(HDR, d / "qca_oracle.h")
    for src in (SRC, SRC_1D, SRC_VAR):
        text = open(src).read()
        if src == target:
            assert text.count(old) == 1, "mutation anchor not unique/found"
            text = text.replace(old, new)
        (d / os.path.basename(src)).write_text(text)
    lib = d / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(lib)] +
                   [str(d / os.path.basename(src)) for src in (SRC, SRC_1D, SRC_VAR)] + ["-lm"],
                   check=True)
    return lib


def _with_lib(monkeypatch, lib, battery):
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: str(lib))
    try:
        return battery()
    finally:
        oracle._lib = None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    lib = _mutant_lib(tmp_path, SRC, *MUTANTS[name])
    failed = _with_lib(monkeypatch, lib, lambda: _battery(oracle))
    assert failed, f"mutant {name} survived every pin"


@pytest.mark.parametrize("name", sorted(MUTANTS_1D))
def test_1d_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    lib = _mutant_lib(tmp_path, SRC_1D, *MUTANTS_1D[name])
    failed = _with_lib(monkeypatch, lib, _battery_1d)
    assert failed, f"mutant {name} survived every 1D pin"


@pytest.mark.parametrize("name", sorted(MUTANTS_OPEN))
def test_open_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    lib = _mutant_lib(tmp_path, SRC_VAR, *MUTANTS_OPEN[name])
    failed = _with_lib(monkeypatch, lib, _battery_open)
    assert failed, f"mutant {name} survived every open-boundary pin"


@pytest.mark.parametrize("name", sorted(MUTANTS_DESYNC))
def test_desync_pins_catch_planted_mistake(tmp_path, monkeypatch, name):
    lib = _mutant_lib(tmp_path, SRC_VAR, *MUTANTS_DESYNC[name])
    failed = _with_lib(monkeypatch, lib, _battery_desync)
    assert failed, f"mutant {name} survived every desynchronisation pin"


def _battery_net(mod, monkeypatch):
    import test_net_oracle as t
    monkeypatch.setattr(t, "onet", mod)
    fns = [(f"single_tap_{ky}{kx}", (lambda ky=ky, kx=kx: t.test_conv_single_tap_is_a_shift(ky, kx)))
           for ky, kx in ((0, 0), (2, 1))]
    fns += [(n, getattr(t, n)) for n in sorted(dir(t))
            if n.startswith("test_") and n != "test_conv_single_tap_is_a_shift"]
    return _run_pins(fns)


def _net_mutant(old, new):
    import types
    src = open(NET_SRC).read()
    assert src.count(old) == 1, "mutation anchor not unique/found"
    mod = types.ModuleType("net_mutant")
    exec(compile(src.replace(old, new), NET_SRC, "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS_NET))
def test_net_pins_catch_planted_mistake(monkeypatch, name):
    failed = _battery_net(_net_mutant(*MUTANTS_NET[name]), monkeypatch)
    assert failed, f"mutant {name} survived every pre-decoder pin"


def test_unmutated_net_reference_passes_battery(monkeypatch):
    import oracle.net
    assert _battery_net(oracle.net, monkeypatch) == []


def test_unmutated_oracle_passes_battery(monkeypatch):
    monkeypatch.setattr(oracle, "_lib", None)
    try:
        assert _battery(oracle) == []
        assert _battery_1d() == []
        assert _battery_open() == []
        assert _battery_desync() == []
    finally:
        oracle._lib = None
