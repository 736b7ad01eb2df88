"""GPU parity of the decoder's rule options against the CPU oracle.

The tie order of Eq. degbreak (lexicographic, or the printed key 3m + s*a with
equal keys to the larger m) and the rule for a balanced axis (stay, or a
counter draw along +a / -a) are options of qca_config.  Every kernel path of
the torus decoder (generic sweep, one-CTA and two-CTA on-chip sweeps, the
large-lattice sweep) must match the oracle bit for bit under each of them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import oracle_pool  # noqa: E402
import paper_2506_03266_gb300 as qca  # noqa: E402
from golden_cases import all_cases  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qca.build()
    oracle.build()
    qca.lib()
    yield
    for L in (12, 128, 256):
        qca.set_kernel_path(L, -1)
    torch.cuda.synchronize()


def gpu_decode(N_np, max_steps=4096, **kw):
    N = torch.from_numpy(np.ascontiguousarray(N_np)).cuda()
    C, steps, fail = qca.decode_batch(N, max_steps=max_steps, **kw)
    torch.cuda.synchronize()
    return C.cpu().numpy(), steps.cpu().numpy(), fail.cpu().numpy()


def assert_same(gpu, cpu, label=""):
    C, s, f = gpu
    Co, so, fo = cpu
    bad = np.nonzero((s != so) | (f != fo) | (C != Co).reshape(len(s), -1).any(1))[0]
    assert bad.size == 0, f"{label}: {bad.size} shots differ, first {bad[:8].tolist()} " \
                          f"steps gpu {s[bad[:4]].tolist()} cpu {so[bad[:4]].tolist()}"


CASE_TIES = [(c, t) for c in all_cases() for t in c["tie_orders"]]


@pytest.mark.parametrize("path", [-1, 0])
@pytest.mark.parametrize("case,tie_order", CASE_TIES,
                         ids=[f"{c['name']}-tie{t}" for c, t in CASE_TIES])
def test_golden_cases_under_each_tie_order(case, tie_order, path):
    L = case["L"]
    qca.set_kernel_path(L, path)
    try:
        C, s, f = gpu_decode(case["N"][None], max_steps=case["max_steps"], m_max=case["m_max"],
                             tie_order=tie_order)
    finally:
        qca.set_kernel_path(L, -1)
    assert s[0] == case["steps"] and f[0] == case["flag"]
    np.testing.assert_array_equal(C[0], case["C"])


RULES = [(1, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("tie_order,balance_rule", RULES)
@pytest.mark.parametrize("L,path,p,shots", [
    (7, -1, 0.09, 80),     # generic sweep (L not a multiple of 4)
    (16, -1, 0.08, 200),   # one-CTA on-chip sweep
    (32, 0, 0.08, 60),     # generic sweep forced
    (64, -1, 0.085, 40),   # one-CTA on-chip sweep
    (128, -1, 0.08, 12),   # one-CTA on-chip sweep, 32 warps
    (128, 3, 0.08, 12),    # large-lattice sweep forced onto L = 128
    (256, -1, 0.08, 8),    # two-CTA cluster
])
def test_rule_options_bit_exact(tie_order, balance_rule, L, path, p, shots):
    N = oracle.sample_errors(L, shots, p, seed=L + 10 * tie_order + balance_rule)
    qca.set_kernel_path(L, path)
    try:
        gpu = gpu_decode(N, 300, tie_order=tie_order, balance_rule=balance_rule, rng_seed=41,
                         shot_offset=3)
    finally:
        qca.set_kernel_path(L, -1)
    kw = dict(max_steps=300, tie_order=tie_order, balance_rule=balance_rule, seed=41)
    if L >= 128:
        cpu = oracle_pool.decode_many(N, shot0=3, **kw)
    else:
        cpu = oracle.decode_batch(N, shot0=3, **kw)
    assert_same(gpu, cpu, f"L{L} path{path} tie{tie_order} bal{balance_rule}")


def test_balanced_random_frees_stuck_pairs_on_gpu():
    """The antipodal pair of the even torus: stuck under the deterministic rule,
    decoded under the balanced random rule, identically on GPU and oracle."""
    L = 6
    N = np.zeros((4, 2, L, L), np.uint8)
    N[:, 0, 0, 0:3] = 1
    stay = gpu_decode(N, 200)
    assert (stay[2] == 2).all() and (stay[1] == 200).all()
    rnd = gpu_decode(N, 200, balance_rule=1, rng_seed=77)
    assert (rnd[2] != 2).all()
    assert_same(rnd, oracle.decode_batch(N, max_steps=200, balance_rule=1, seed=77), "balanced")


def test_synchronous_syndrome_entry_point():
    """qca_decode_syndrome_batch (synchronous, default options) against the
    oracle's syndrome decoder."""
    L, shots = 20, 40
    N = oracle.sample_errors(L, shots, 0.07, seed=19)
    anyon = np.stack([(oracle.syndrome(n) == -1).astype(np.uint8) for n in N])
    C, steps, cut = qca.decode_syndrome_batch_sync(torch.from_numpy(anyon).cuda(), max_steps=300)
    for s in range(shots):
        Co, so, fo, cuto = oracle.decode_syndrome_shot(anyon[s], max_steps=300)
        assert steps[s].item() == so
        np.testing.assert_array_equal(C[s].cpu().numpy(), Co)
        np.testing.assert_array_equal(cut[s].cpu().numpy(), cuto)


def test_rule_options_rejected_where_unsupported():
    """The open-boundary decoder takes only the default rule; an unknown tie
    order is an argument error everywhere."""
    import ctypes
    N = torch.zeros((1, 2, 8, 8), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(N)
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    fl = torch.empty(1, dtype=torch.uint8, device="cuda")
    cfg = qca.make_config(tie_order=1)
    rc = qca.lib().qca_decode_open_batch_async(
        ctypes.c_void_p(N.data_ptr()), 8, 1, 10, ctypes.byref(cfg), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(st.data_ptr()), ctypes.c_void_p(fl.data_ptr()), None)
    assert rc == qca.QCA_ERR_UNSUPPORTED
    with pytest.raises(qca.QcaError):
        qca.decode_batch(N, tie_order=2)
