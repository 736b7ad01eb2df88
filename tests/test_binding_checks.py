"""Checks the Python binding makes on caller-supplied output tensors before it
calls the library: the kernels write the full extents of correction, steps and
flags, so a tensor of another count, dtype, shape, layout or device is refused
on the host."""
import pytest
import torch

import paper_2506_03266_gb300 as qca

CPU = torch.device("cpu")


def _good(shots=3, L=8, device=CPU):
    return (torch.zeros(shots, 2, L, L, dtype=torch.uint8, device=device),
            torch.zeros(shots, dtype=torch.int32, device=device),
            torch.zeros(shots, dtype=torch.uint8, device=device))


def test_out_tensors_checked_for_count_dtype_shape_layout_device():
    specs = qca._decode_specs(torch, 3, 8)
    C, s, f = _good()
    qca._check_out(torch, (C, s, f), specs, CPU)
    qca._check_out(torch, [C, s, f], specs, CPU)
    strided = torch.zeros(3, 2, 8, 16, dtype=torch.uint8)[..., ::2]
    assert strided.shape == C.shape and not strided.is_contiguous()
    bad = {
        "too few": (C, s),
        "too many": (C, s, f, f),
        "not a tuple": C,
        "steps dtype": (C, s.to(torch.int64), f),
        "flag dtype": (C, s, f.to(torch.int32)),
        "correction dtype": (C.to(torch.int8), s, f),
        "more shots": (torch.zeros(4, 2, 8, 8, dtype=torch.uint8), s, f),
        "larger L": (torch.zeros(3, 2, 9, 9, dtype=torch.uint8), s, f),
        "flat correction": (C.reshape(-1), s, f),
        "steps shape": (C, torch.zeros(3, 1, dtype=torch.int32), f),
        "not contiguous": (strided, s, f),
        "not a tensor": (C, s, [0, 0, 0]),
        "other device": (C.to("meta"), s, f),
    }
    for what, out in bad.items():
        with pytest.raises(ValueError):
            qca._check_out(torch, out, specs, CPU)
        assert what


@pytest.mark.gpu
def test_wrong_out_tensors_raise_before_any_launch():
    """Each wrong buffer here is at least as large as the right one, so nothing
    would be written out of bounds even if a check were missing."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qca.build()
    qca.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    N = qca.sample_errors(16, 4, 0.05, seed=1)
    C, s, f = _good(4, 16, dev)
    big_C, big_s, big_f = _good(5, 16, dev)
    for out in [(big_C, s, f), (C, big_s, f), (C, s, big_f), (C, s.to(torch.int64), f),
                (C.reshape(-1), s, f), (C, s)]:
        with pytest.raises(ValueError):
            qca.decode_batch(N, 100, out=out)
        with pytest.raises(ValueError):
            qca.decode_batch_noalloc(N, out, max_steps=100)
    # the host entry point: host outputs, one of them one shot too large
    Nh = N.cpu()
    Ch, sh, fh = _good(4, 16, CPU)
    with pytest.raises(ValueError):
        qca.decode_batch_host(Nh, 100, out=(Ch, torch.zeros(5, dtype=torch.int32), fh))
    with pytest.raises(ValueError):
        qca.decode_batch_host(Nh.reshape(4, 2, 256), 100)
    # an uneven plan: packed buffers one byte too large
    plan = qca.UnevenPlan([8, 12])
    Np = plan.sample([0, 0], seed=1)
    with pytest.raises(ValueError):
        plan.decode(torch.zeros(plan.total_bytes + 1, dtype=torch.uint8, device=dev), 100)
    with pytest.raises(ValueError):
        plan.decode(Np, 100, out=(torch.zeros(plan.total_bytes + 1, dtype=torch.uint8, device=dev),
                                  torch.zeros(2, dtype=torch.int32, device=dev),
                                  torch.zeros(2, dtype=torch.uint8, device=dev)))
    plan.close()
    # right tensors still decode as without out
    C0, s0, f0 = qca.decode_batch(N, 100)
    qca.decode_batch(N, 100, out=(C, s, f))
    torch.cuda.synchronize()
    assert torch.equal(C, C0) and torch.equal(s, s0) and torch.equal(f, f0)
