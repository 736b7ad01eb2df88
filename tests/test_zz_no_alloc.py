"""The no-allocation entry point, qca_decode_batch_noalloc.

Some callers cannot allocate device memory while they decode (a control loop
that reserved all memory up front, a host whose memory pool owns the device).
For them the library decodes with its state in a fixed device array and
allocates nothing.  These tests call that entry point through the C ABI and
require its results to equal those of qca_decode_batch_async on the same
inputs, for two calls in a row (the second runs on the array the first one
left behind).  The file's name sorts last so that a run stopping at the first
failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2506_03266_gb300 as qca  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qca.build()
    qca.lib()


def _reference(N, max_steps):
    C, steps, fail = qca.decode_batch(N, max_steps=max_steps)
    torch.cuda.synchronize()
    return C.cpu().numpy(), steps.cpu().numpy(), fail.cpu().numpy()


def _noalloc(N, max_steps):
    out = (torch.empty_like(N), torch.empty(N.shape[0], dtype=torch.int32, device="cuda"),
           torch.empty(N.shape[0], dtype=torch.uint8, device="cuda"))
    C, steps, fail = qca.decode_batch_noalloc(N, out, max_steps=max_steps)
    torch.cuda.synchronize()
    return C.cpu().numpy(), steps.cpu().numpy(), fail.cpu().numpy()


def test_noalloc_zero_shot_call_sets_up_the_device():
    """A call with no shots is the documented warm-up: it returns 0 and the
    next call decodes correctly."""
    lib = qca.lib()
    assert lib.qca_decode_batch_noalloc(None, 16, 0, 10, 0, None, None, None, None, None) == 0
    N = qca.sample_errors(16, 50, 0.06, seed=3)
    want = _reference(N, 600)
    got = _noalloc(N, 600)
    for g_arr, w_arr in zip(got, want):
        np.testing.assert_array_equal(g_arr, w_arr)


# L = 384 leaves room for 8 shots at once in the fixed array and L = 1024 for
# one, so these batches take several turns
@pytest.mark.parametrize("L,shots,p", [(16, 300, 0.06), (31, 60, 0.08), (256, 40, 0.05),
                                       (384, 10, 0.05), (1024, 2, 0.05)])
def test_noalloc_matches_existing_entry_point_twice(L, shots, p):
    # two different inputs, decoded one after the other on the shared array
    for seed in (11, 12):
        N = qca.sample_errors(L, shots, p, seed=seed)
        want = _reference(N, 600)
        got = _noalloc(N, 600)
        for g_arr, w_arr in zip(got, want):
            np.testing.assert_array_equal(g_arr, w_arr)


def test_noalloc_rejects_sizes_and_arguments():
    lib = qca.lib()
    dummy = ctypes.c_void_p(16)
    assert lib.qca_decode_batch_noalloc(dummy, 2048, 1, 10, 0, dummy, dummy, dummy, None,
                                        None) == qca.QCA_ERR_UNSUPPORTED
    assert lib.qca_decode_batch_noalloc(None, 16, 1, 10, 0, dummy, dummy, dummy, None,
                                        None) == qca.QCA_ERR_ARG
    assert lib.qca_decode_batch_noalloc(None, 16, 0, 10, 0, None, None, None, None, None) == 0
