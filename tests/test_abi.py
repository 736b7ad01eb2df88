"""CPU-side checks of the C ABI: the library loads, exports every function
include/qca.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2506_03266_gb300 as qca

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    qca.build()
    return qca.lib()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(qca_[a-z_0-9]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["qca_decode_batch", "qca_decode_batch_async", "qca_sample_errors",
                 "qca_decode_syndrome_batch", "qca_decode_syndrome_batch_async",
                 "qca_decode_batch_host", "qca_last_error",
                 "qca_free_workspace", "qca_default_config"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_version_and_defaults(lib):
    assert lib.qca_version() >= 100
    c = qca.QcaConfig()
    assert lib.qca_default_config(ctypes.byref(c)) == 0
    assert (c.v, c.m_max, c.p_move, c.shot_offset) == (3, 255, 0.0, 0)
    assert (c.tie_order, c.balance_rule) == (qca.TIE_LEX, qca.BALANCE_STAY)
    assert ctypes.sizeof(qca.QcaConfig) == 32  # the struct layout of include/qca.h
    assert lib.qca_default_config(None) == qca.QCA_ERR_ARG


def test_argument_errors_need_no_gpu(lib):
    dummy = ctypes.c_void_p(16)
    cfg = qca.make_config()
    # L < 3, L too large, negative shots, negative / huge budget, NULL arrays
    assert lib.qca_decode_batch(dummy, 2, 1, 10, 0, dummy, dummy, dummy) == qca.QCA_ERR_ARG
    assert "L = 2" in qca.last_error()
    assert lib.qca_decode_batch(dummy, 2000, 1, 10, 0, dummy, dummy, dummy) == \
        qca.QCA_ERR_UNSUPPORTED
    assert lib.qca_decode_batch(dummy, 16, -1, 10, 0, dummy, dummy, dummy) == qca.QCA_ERR_ARG
    assert lib.qca_decode_batch(dummy, 16, 1, -5, 0, dummy, dummy, dummy) == qca.QCA_ERR_ARG
    assert lib.qca_decode_batch(dummy, 16, 1, qca.QCA_MAX_STEPS + 1, 0, dummy, dummy,
                                dummy) == qca.QCA_ERR_ARG
    assert lib.qca_decode_batch(None, 16, 1, 10, 0, dummy, dummy, dummy) == qca.QCA_ERR_ARG
    assert lib.qca_decode_batch_async(dummy, 16, 1, 10, 0, None, dummy, dummy,
                                      ctypes.byref(cfg), None) == qca.QCA_ERR_ARG
    assert lib.qca_decode_syndrome_batch_async(dummy, 16, 1, 10, 0, dummy, dummy, None, None,
                                               ctypes.byref(cfg), None) == qca.QCA_ERR_ARG
    assert lib.qca_sample_errors(16, 1, 1.5, 0, dummy) == qca.QCA_ERR_ARG
    assert lib.qca_sample_errors(16, 1, 0.1, 0, None) == qca.QCA_ERR_ARG
    assert lib.qca_decode_batch_host(None, 16, 1, 10, 0, None, None, None, None) == \
        qca.QCA_ERR_ARG
    # unsupported options
    bad = qca.make_config(v=0)
    assert lib.qca_decode_batch_async(dummy, 16, 1, 10, 0, dummy, dummy, dummy,
                                      ctypes.byref(bad), None) == qca.QCA_ERR_UNSUPPORTED
    bad = qca.make_config(m_max=256)
    assert lib.qca_decode_batch_async(dummy, 16, 1, 10, 0, dummy, dummy, dummy,
                                      ctypes.byref(bad), None) == qca.QCA_ERR_UNSUPPORTED
    bad = qca.make_config(p_move=-0.1)
    assert lib.qca_decode_batch_async(dummy, 16, 1, 10, 0, dummy, dummy, dummy,
                                      ctypes.byref(bad), None) == qca.QCA_ERR_ARG
    for bad in (qca.make_config(tie_order=2), qca.make_config(balance_rule=-1)):
        assert lib.qca_decode_batch_async(dummy, 16, 1, 10, 0, dummy, dummy, dummy,
                                          ctypes.byref(bad), None) == qca.QCA_ERR_ARG
    assert lib.qca_decode_syndrome_batch(None, 16, 1, 10, 0, dummy, dummy, dummy) == \
        qca.QCA_ERR_ARG
    # zero shots: nothing to do, NULL allowed, no device call
    assert lib.qca_decode_batch_async(None, 16, 0, 10, 0, None, None, None, None, None) == 0
    assert lib.qca_sample_errors_async(16, 0, 0, 0.1, 0, None, None) == 0
    assert lib.qca_probe_peaks(None) == qca.QCA_ERR_ARG
    # an int32 step array off a 4-byte boundary is refused before any launch
    assert lib.qca_decode_batch_async(dummy, 16, 1, 10, 0, dummy, ctypes.c_void_p(18), dummy,
                                      ctypes.byref(cfg), None) == qca.QCA_ERR_ARG
    assert "aligned" in qca.last_error()


def test_band_geometry_covers_every_supported_size(lib):
    # host-side geometry of the on-chip sweep (no GPU needed): every multiple
    # of 4 up to 128 and of 8 up to 256 gets a band height of at least 4 rows
    # that divides the CTA's rows (L up to 128, L / 2 in the two-CTA cluster)
    for L in range(8, 257, 4):
        qca.set_tuning(L, 0, 0)
        path = qca.kernel_path(L)
        if L > 128 and L % 8:
            assert path == 0, L
            continue
        assert path == (1 if L <= 128 else 2), L
        H, div, threads = qca.get_tuning(L)
        rows = L if L <= 128 else L // 2
        assert H >= 4 and rows % H == 0, (L, H)
        assert threads % 32 == 0 and 0 < threads <= (1024 if L <= 128 else 512), (L, threads)
    # sizes with a 4-, 8-, 16- or 32-row band keep the measured rule's choice
    for L, H in [(8, 8), (12, 4), (24, 8), (32, 8), (48, 16), (56, 8), (64, 32), (96, 32),
                 (128, 32), (192, 32), (256, 32)]:
        assert qca.get_tuning(L)[0] == H, L
    # and the others take another divisor of their rows
    for L, H in [(68, 34), (100, 25), (136, 17), (160, 20), (200, 25), (248, 31)]:
        assert qca.get_tuning(L)[0] == H, L


def _band_height_rule(L):
    """The band-height rule of the on-chip sweep restated: among 4-, 8-, 16-
    and 32-row bands that divide the CTA's rows within its warp limit, the one
    whose warp count is nearest the target, the taller on a tie; if none fits,
    any other divisor of at least 5 rows by the same distance, the shorter on
    a tie.  Returns (height, whether a tie decided it)."""
    cl = 2 if L > 128 else 1
    kw = 2 if L // 4 > 32 else 1
    rows = L // cl
    spw = 32 // (L // 4 // kw)  # band segments per warp
    max_warps = 32 if cl == 1 else 16
    target = min(max_warps, 4 if L <= 64 else min(16, L // 8))

    def dist(H):
        return abs(-(-4 * (rows // H) // spw) - target)

    def fits(H):
        return rows % H == 0 and -(-4 * (rows // H) // spw) <= max_warps

    cand = [H for H in (4, 8, 16, 32) if fits(H)]
    if cand:
        best = min(cand, key=lambda H: (dist(H), -H))
    else:
        cand = [H for H in range(5, rows + 1) if fits(H)]
        best = min(cand, key=lambda H: (dist(H), H))
    return best, sum(dist(H) == dist(best) for H in cand) > 1


def test_band_height_follows_its_rule_at_every_size_ties_included(lib):
    ties = {}
    for L in range(8, 257, 4):
        if L > 128 and L % 8:
            continue
        qca.set_tuning(L, 0, 0)
        H, tie = _band_height_rule(L)
        assert qca.get_tuning(L)[0] == H, L
        if tie:
            ties[L] = H
    # taller among the power-of-two bands (8: 4 or 8 rows; 24: 4 or 8), shorter
    # among the others (84: 28 or 42 rows; 100: 25 or 50)
    assert ties == {8: 8, 24: 8, 84: 28, 100: 25}, ties


def test_large_lattice_path_selection(lib):
    # above 256: the large-lattice sweep for multiples of 128, else the generic one
    for L in range(257, 1025):
        assert qca.kernel_path(L) == (3 if L % 128 == 0 else 0), L


def test_kernel_path_table(lib):
    assert qca.kernel_path(16) >= 0
    assert qca.kernel_path(256) >= 0
    assert qca.kernel_path(1024) >= 0
    with pytest.raises(qca.QcaError):
        qca.kernel_path(2)


def test_product_path_does_not_import_oracle():
    """The CUDA path and the oracle share nothing; the package never names it."""
    pkg = os.path.join(ROOT, "paper_2506_03266_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "qca_oracle" not in text, fn
