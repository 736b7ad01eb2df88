"""Caller arrays off a 4-byte boundary.  The on-chip and large-lattice sweeps
access the input and the correction as 32-bit words; the host sends a
misaligned array, or an uneven batch whose odd-L shots move later blocks off
the boundary, to the byte-access generic sweep.  The results must be those of
the aligned decode, bit for bit."""
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


def _at_offset(src, byte_offset):
    """A contiguous copy of src whose first byte sits byte_offset past a
    256-byte aligned allocation."""
    flat = torch.zeros(src.numel() + 16, dtype=torch.uint8, device="cuda")
    view = flat[byte_offset:byte_offset + src.numel()].view(src.shape)
    view.copy_(src)
    return view


@pytest.mark.parametrize("L,shots,forced_path", [(32, 9, -1), (256, 2, -1), (128, 3, 3)])
def test_misaligned_arrays_decode_like_aligned(L, shots, forced_path):
    N = qca.sample_errors(L, shots, 0.06, seed=L)
    if forced_path >= 0:
        qca.set_kernel_path(L, forced_path)
    try:
        C0, s0, f0 = qca.decode_batch(N, 1024)
        for off_in, off_out in [(1, 0), (0, 2), (3, 1)]:
            Nm = _at_offset(N, off_in)
            Cm = _at_offset(torch.zeros_like(N), off_out)
            sm = torch.empty(shots, dtype=torch.int32, device="cuda")
            fm = torch.empty(shots, dtype=torch.uint8, device="cuda")
            qca.decode_batch(Nm, 1024, out=(Cm, sm, fm))
            torch.cuda.synchronize()
            assert torch.equal(Cm, C0) and torch.equal(sm, s0) and torch.equal(fm, f0)
    finally:
        if forced_path >= 0:
            qca.set_kernel_path(L, -1)


def test_uneven_batch_with_odd_sizes():
    # 2 L^2 is 2 mod 4 for odd L: the L = 32 and L = 24 shots after one of
    # them start off a 4-byte boundary
    L = np.array([5, 32, 7, 32, 24, 9, 24, 32, 6, 32], dtype=np.int32)
    thr = np.full(len(L), int(0.05 * 2.0**64), dtype=np.uint64)
    plan = qca.UnevenPlan(L)
    assert any(plan.offsets[s] % 4 for s in range(len(L)) if L[s] % 4 == 0)
    N = plan.sample(thr, seed=11)
    C, steps, fail = plan.decode(N, max_steps=600)
    torch.cuda.synchronize()
    Nh, Ch = N.cpu().numpy(), C.cpu().numpy()
    steps, fail = steps.cpu().numpy(), fail.cpu().numpy()
    for s in range(len(L)):
        n = 2 * int(L[s]) ** 2
        blk = torch.from_numpy(Nh[plan.offsets[s]:plan.offsets[s] + n].reshape(1, 2, L[s], L[s]))
        Cu, su, fu = qca.decode_batch(blk.cuda(), max_steps=600)
        torch.cuda.synchronize()
        assert steps[s] == int(su[0]) and fail[s] == int(fu[0]), s
        np.testing.assert_array_equal(Ch[plan.offsets[s]:plan.offsets[s] + n],
                                      Cu.cpu().numpy().reshape(-1))
    plan.close()
