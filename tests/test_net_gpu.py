"""GPU checks of the learned pre-decoder through the C ABI.

- labels (integer work): bit-exact against the CPU reference of the
  automaton's first step;
- logits: within 1e-2 of the FP64 CPU forward that applies the same bf16
  (or e4m3) rounding points, checked layer by layer on the kernels' own
  activations; every larger end-to-end difference is traced to a rounding
  the arithmetic leaves undetermined;
- proposals and pairing: bit-exact against the reference rule applied to the
  GPU's own fp32 logits (the float decision is taken in the kernel's
  precision on both sides);
- net + automaton: the automaton part is bit-exact against the oracle run on
  the GPU's residual, and the combined correction clears the syndrome;
- training lowers the loss and the trained net reproduces most labels;
- the logical failure rate of net + automaton is within 2 sigma of the plain
  automaton's below threshold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import oracle.net as onet  # noqa: E402
import paper_2506_03266_gb300 as qca  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qca.build()
    oracle.build()
    qca.lib()
    yield
    torch.cuda.synchronize()


@pytest.fixture(scope="module")
def trained():
    """A net trained on L = 32 crops, p ~ U[0.02, 0.07)."""
    net = qca.Net(seed=1)
    losses = net.train(L=32, iterations=1500, batch=64, p_lo=0.02, p_hi=0.07, seed=1, lr=2e-3)
    yield net, losses
    net.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def anyon_maps(N):
    return np.stack([(oracle.syndrome(n) == -1).astype(np.uint8) for n in N])


# ------------------------------------------------------------------- labels

@pytest.mark.parametrize("L,p,shots", [(4, 0.2, 8), (7, 0.08, 10), (16, 0.05, 12),
                                       (33, 0.03, 6), (256, 0.05, 2)])
def test_labels_bit_exact(L, p, shots):
    N = oracle.sample_errors(L, shots, p, seed=3)
    got = qca.net_labels(dev(N)).cpu().numpy()
    for s in range(shots):
        want = onet.first_step_labels(anyon_maps(N[s:s + 1])[0])
        np.testing.assert_array_equal(got[s], want, err_msg=f"shot {s}")


# ------------------------------------------------------------------- logits

def _gpu_chain(net, Nd):
    """The kernels' own activations of layers 1-3 (as layer k+1 reads them) and
    their logits, as numpy arrays."""
    acts = [net.activations(Nd, k).cpu().numpy().astype(np.float64) for k in (1, 2, 3)]
    z = net.logits(Nd)
    torch.cuda.synchronize()
    net.status()
    return acts, z.cpu().numpy().astype(np.float64)


def _check_net(net, N, fp8=False, scales=None):
    """The pre-decoder's parity, layer by layer and end to end, against the
    FP64 forward with the same rounding points.

    Layer by layer: layer k computed in FP64 from the kernels' own layer k-1
    output must store exactly the kernels' layer k output, except where the
    stored value is not determined by the arithmetic (the FP64 sum lies within
    the fp32 accumulation bound of a rounding boundary); there the kernel's
    value must lie between the values stored at the two ends of that
    interval.  Such elements must be rare.
    Logits from the kernels' own layer 3 are within 1e-2 of FP64 (and within
    the accumulation bound).
    End to end: the FP64 forward with its own rounding points; every logit
    whose receptive field holds no layer-3 difference between the two chains
    is within 1e-2, and every larger difference is traced to such a
    difference, i.e. to a rounding the layer-by-layer check allows.
    Returns (uncertain-and-different count per layer, elements per layer,
    logits beyond 1e-2, traced logits)."""
    Nd = dev(N)
    acts, z_gpu = _gpu_chain(net, Nd)
    if fp8:  # e4m3 values times the layer's scale, in float64
        acts = [a * float(np.float32(scales[k])) for k, a in enumerate(acts)]
    params = net.get_params()
    lw = onet.layer_weights(params, fp8=fp8)
    A = anyon_maps(N)
    flips = [0, 0, 0]
    sizes = [0, 0, 0]
    beyond = traced = 0
    for s in range(N.shape[0]):
        x0 = np.stack([A[s].astype(np.float64), np.ones(A[s].shape)])
        inp = [x0, acts[0][s], acts[1][s], acts[2][s]]
        for k in range(3):
            W, b = lw[k]
            z = onet.conv3x3_circular(inp[k], W, b)
            mag = onet.conv_magnitude(inp[k], W, b)
            sc = None if not fp8 else float(np.float32(scales[k]))
            want = onet.store_activation(z, sc)
            lo, hi = onet.store_interval(z, mag, sc)
            got = inp[k + 1]
            diff = got != want
            ok = (got >= lo) & (got <= hi)
            assert not np.any(diff & ~ok), \
                f"layer {k + 1}: {int(np.sum(diff & ~ok))} outputs outside their rounding interval"
            flips[k] += int(diff.sum())
            sizes[k] += diff.size
        W, b = lw[3]
        z4 = onet.conv3x3_circular(inp[3], W, b)
        mag4 = onet.conv_magnitude(inp[3], W, b)
        d4 = np.abs(z_gpu[s] - z4)
        assert np.all(d4 <= onet.ACC_REL_BOUND * mag4 + 1e-6) and d4.max() <= 1e-2, d4.max()
        # end to end: the FP64 chain with its own rounding points
        x = x0
        for k in range(3):
            W, b = lw[k]
            sc = None if not fp8 else float(np.float32(scales[k]))
            x = onet.store_activation(onet.conv3x3_circular(x, W, b), sc)
        zf = onet.conv3x3_circular(x, *lw[3])
        d = np.abs(z_gpu[s] - zf)
        tainted = onet.dilate(np.any(x != acts[2][s], axis=0), 1)
        assert np.all(d[:, ~tainted] <= 1e-2), d[:, ~tainted].max()
        beyond += int(np.sum(d > 1e-2))
        traced += int(np.sum((d > 1e-2) & tainted[None]))
    for k in range(3):
        assert flips[k] <= 1e-3 * sizes[k] + 2, (k + 1, flips[k], sizes[k])
    assert beyond == traced
    return flips, sizes, beyond, traced


@pytest.mark.parametrize("L,shots", [(16, 3), (21, 3), (5, 7)])
def test_logits_initial_net(L, shots):
    net = qca.Net(seed=7)
    try:
        _check_net(net, oracle.sample_errors(L, shots, 0.08, seed=L))
    finally:
        net.close()


def test_logits_trained_net(trained):
    net, _ = trained
    net.set_precision("bf16")
    _check_net(net, oracle.sample_errors(24, 4, 0.05, seed=9))
    _check_net(net, oracle.sample_errors(19, 2, 0.07, seed=10))


def test_set_get_params_roundtrip():
    net = qca.Net(seed=2)
    try:
        p = net.get_params()
        assert p.shape == (onet.param_count(),) and np.isfinite(p).all()
        q = (np.random.default_rng(0).standard_normal(p.size) * 0.05).astype(np.float32)
        net.set_params(q)
        np.testing.assert_array_equal(net.get_params(), q)
        # the prepared bf16 weights follow set_params
        _check_net(net, oracle.sample_errors(12, 2, 0.1, seed=4))
    finally:
        net.close()


# ------------------------------------------------------- pairing / residual

@pytest.mark.parametrize("L,shots,p", [(16, 20, 0.05), (21, 5, 0.08)])
def test_predecode_pairing_bit_exact(trained, L, shots, p):
    net, _ = trained
    N = oracle.sample_errors(L, shots, p, seed=21)
    Nd = dev(N)
    z = net.logits(Nd).cpu().numpy()          # fp32, the kernel's own values
    R, C0 = net.predecode(Nd)
    torch.cuda.synchronize()
    R, C0 = R.cpu().numpy(), C0.cpu().numpy()
    A = anyon_maps(N)
    paired = 0
    for s in range(shots):
        prop = onet.proposals(A[s], z[s])     # float32 comparisons, same as the kernel
        want = onet.pairing_links(A[s], prop)
        np.testing.assert_array_equal(C0[s], want, err_msg=f"shot {s}")
        paired += int(want.sum())
    np.testing.assert_array_equal(R, N ^ C0)
    assert paired > 0


def test_net_decode_matches_oracle_on_residual(trained):
    net, _ = trained
    L, shots = 16, 60
    N = oracle.sample_errors(L, shots, 0.06, seed=31)
    Nd = dev(N)
    C, steps, fail = net.decode_batch(Nd, max_steps=4096)
    R, C0 = net.predecode(Nd)
    torch.cuda.synchronize()
    C, steps, fail, R, C0 = (t.cpu().numpy() for t in (C, steps, fail, R, C0))
    for s in range(shots):
        Co, so, fo = oracle.decode_shot(R[s], max_steps=4096)
        np.testing.assert_array_equal(C[s], Co ^ C0[s], err_msg=f"shot {s}")
        assert (steps[s], fail[s]) == (so, fo), f"shot {s}"


def test_net_decode_full_size_properties(trained):
    # L = 128, the learned-stage workload's size: every shot that ends within
    # the budget leaves N xor C with an empty syndrome (checked with torch ops)
    net, _ = trained
    L, shots = 128, 400
    N = qca.sample_errors(L, shots, 0.04, seed=0)
    C, steps, fail = net.decode_batch(N, max_steps=4096)
    E = (N ^ C).to(torch.int32)
    ex, ey = E[:, 0], E[:, 1]
    sig = ex ^ torch.roll(ex, 1, dims=2) ^ ey ^ torch.roll(ey, 1, dims=1)
    done = fail != 2
    assert int(done.sum()) == shots
    assert int(sig[done].sum()) == 0
    assert int(steps.min()) >= 0


# ----------------------------------------------------------------- training

def test_training_lowers_loss_and_learns_labels(trained):
    net, losses = trained
    assert np.isfinite(losses).all()
    assert losses[-50:].mean() < 0.5 * losses[:5].mean(), (losses[:5], losses[-50:].mean())
    L, shots = 32, 64
    N = oracle.sample_errors(L, shots, 0.05, seed=77)
    Nd = dev(N)
    lab = qca.net_labels(Nd).cpu().numpy()
    z = net.logits(Nd).cpu().numpy()
    A = anyon_maps(N)
    prop = np.stack([onet.proposals(A[s], z[s]) for s in range(shots)])
    m = lab != 255
    acc = float((prop[m] == lab[m]).mean())
    assert acc > 0.9, acc


def test_training_argument_errors():
    net = qca.Net(seed=0)
    try:
        with pytest.raises(qca.QcaError):
            net.train(L=200, iterations=1, batch=1, p_lo=0.01, p_hi=0.05)
        with pytest.raises(qca.QcaError):
            net.train(L=16, iterations=1, batch=1, p_lo=0.05, p_hi=0.01)
        assert net.train(L=16, iterations=0, batch=1, p_lo=0.01, p_hi=0.05).size == 0
    finally:
        net.close()


# ------------------------------------------------------- statistical target

def test_net_plus_automaton_plog_within_2sigma(trained):
    # below threshold (p = 0.058, about 0.8 of the paper's 7.3 %), L = 32:
    # failure counts of plain and net + automaton on the same noise agree
    # within two standard deviations of their difference
    net, _ = trained
    L, shots = 32, 40000
    N = qca.sample_errors(L, shots, 0.058, seed=0)
    _, _, f_plain = qca.decode_batch(N, max_steps=4096)
    _, _, f_net = net.decode_batch(N, max_steps=4096)
    a = (f_plain == 1).double().mean().item()
    b = (f_net == 1).double().mean().item()
    sigma = np.sqrt((a * (1 - a) + b * (1 - b)) / shots)
    assert a > 0.0 and abs(a - b) <= 2 * sigma + 1e-12, (a, b, sigma)


# ------------------------------------------------------------------- FP8 form

@pytest.fixture(scope="module")
def trained_fp8(trained):
    net, _ = trained
    N = qca.sample_errors(32, 256, 0.05, seed=99)
    scales = net.calibrate_fp8(N)
    assert np.all(scales > 0)
    net.set_precision("fp8")
    yield net, scales
    net.set_precision("bf16")


def test_fp8_needs_scales():
    net = qca.Net(seed=3)
    try:
        with pytest.raises(qca.QcaError):
            net.set_precision("fp8")
        net.set_fp8_scales([0.01, 0.02, 0.03])
        np.testing.assert_array_equal(net.fp8_scales(), np.float32([0.01, 0.02, 0.03]))
        net.set_precision("fp8")
    finally:
        net.close()


def test_fp8_logits_match_fp64_forward(trained_fp8):
    # the same layer-by-layer and end-to-end parity as the bf16 form, with
    # e4m3(relu(z) / s) * s as the stored activations (mma.sync path, L = 24)
    net, scales = trained_fp8
    _check_net(net, oracle.sample_errors(24, 6, 0.05, seed=41), fp8=True, scales=scales)


def test_fp8_pairing_bit_exact(trained_fp8):
    net, _ = trained_fp8
    L, shots = 21, 6
    N = oracle.sample_errors(L, shots, 0.07, seed=42)
    Nd = dev(N)
    z = net.logits(Nd).cpu().numpy()
    R, C0 = net.predecode(Nd)
    torch.cuda.synchronize()
    R, C0 = R.cpu().numpy(), C0.cpu().numpy()
    A = anyon_maps(N)
    for s in range(shots):
        want = onet.pairing_links(A[s], onet.proposals(A[s], z[s]))
        np.testing.assert_array_equal(C0[s], want, err_msg=f"shot {s}")
    np.testing.assert_array_equal(R, N ^ C0)


def test_fp8_tcgen05_matches_mma_path_and_fp64(trained_fp8):
    # L % 128 == 0: the FP8 layers run as tcgen05 kind::f8f6f4 MMAs (one K = 32
    # MMA per tap); against the mma.sync m16n8k32 path and the FP64 reference.
    # The two instructions add the 32 products of a K step in different orders,
    # so fp32 results differ in their last bits (measured: 4 % of the logits,
    # by at most 1.5e-6); where that moves an intermediate activation across an
    # E4M3 rounding boundary (rare), a logit moves by up to |W| times one step.
    net, scales = trained_fp8
    L, shots = 128, 2
    N = oracle.sample_errors(L, shots, 0.05, seed=61)
    Nd = dev(N)
    net.set_tensor_path("tcgen05_ws")
    z_tc = net.logits(Nd).cpu().numpy()
    net.status()
    net.set_tensor_path("mma")
    z_ms = net.logits(Nd).cpu().numpy()
    net.set_tensor_path("tcgen05_ws")
    dm = np.abs(z_tc - z_ms).ravel()
    assert np.mean(dm <= 1e-5) >= 0.999 and dm.max() <= 0.25, (np.mean(dm <= 1e-5), dm.max())
    # the tcgen05 path's own chain against FP64, layer by layer and end to end
    _check_net(net, N, fp8=True, scales=scales)


def test_fp8_tcgen05_pairing_bit_exact(trained_fp8):
    net, _ = trained_fp8
    net.set_tensor_path("tcgen05_ws")
    L, shots = 256, 2
    N = oracle.sample_errors(L, shots, 0.05, seed=62)
    Nd = dev(N)
    z = net.logits(Nd).cpu().numpy()
    R, C0 = net.predecode(Nd)
    torch.cuda.synchronize()
    net.status()
    R, C0 = R.cpu().numpy(), C0.cpu().numpy()
    A = anyon_maps(N)
    for s in range(shots):
        want = onet.pairing_links(A[s], onet.proposals(A[s], z[s]))
        np.testing.assert_array_equal(C0[s], want, err_msg=f"shot {s}")
    np.testing.assert_array_equal(R, N ^ C0)


def test_fp8_net_plus_automaton_plog_within_2sigma(trained_fp8):
    net, _ = trained_fp8
    L, shots = 32, 40000
    N = qca.sample_errors(L, shots, 0.058, seed=1)
    _, _, f_plain = qca.decode_batch(N, max_steps=4096)
    _, _, f_net = net.decode_batch(N, max_steps=4096)
    a = (f_plain == 1).double().mean().item()
    b = (f_net == 1).double().mean().item()
    sigma = np.sqrt((a * (1 - a) + b * (1 - b)) / shots)
    assert a > 0.0 and abs(a - b) <= 2 * sigma + 1e-12, (a, b, sigma)


# ------------------------------------------------ tcgen05 path (L % 128 == 0)

def test_tcgen05_logits_match_fp64_and_mma_path(trained):
    # The tcgen05 and mma.sync paths accumulate the same products in the same
    # order: their logits agree bit for bit.  Against FP64: the layer-by-layer
    # and end-to-end check of _check_net on the tcgen05 path's own chain.
    net, _ = trained
    net.set_precision("bf16")   # the FP8 fixture may still be active in this module
    L, shots = 128, 2
    N = oracle.sample_errors(L, shots, 0.05, seed=51)
    Nd = dev(N)
    net.set_tensor_path("tcgen05")
    z_tc = net.logits(Nd).cpu().numpy()
    net.status()
    net.set_tensor_path("tcgen05_ws")
    z_ws = net.logits(Nd).cpu().numpy()
    net.status()
    net.set_tensor_path("mma")
    z_ms = net.logits(Nd).cpu().numpy()
    net.set_tensor_path("tcgen05_ws")
    np.testing.assert_array_equal(z_tc, z_ms)
    np.testing.assert_array_equal(z_ws, z_ms)
    _check_net(net, N)


def test_tcgen05_warp_specialised_matches_row_synchronous(trained):
    # enough shots that every CTA runs several work units through its ring of
    # staged rows (units = shots * (L / 128) * (L / 64) > twice the SM count)
    net, _ = trained
    net.set_precision("bf16")
    L, shots = 128, 400
    Nd = qca.sample_errors(L, shots, 0.05, seed=53)
    out = {}
    for path in ("tcgen05", "tcgen05_ws"):
        net.set_tensor_path(path)
        z = net.logits(Nd)
        R, C0 = net.predecode(Nd)
        torch.cuda.synchronize()
        net.status()
        out[path] = (z.cpu().numpy(), R.cpu().numpy(), C0.cpu().numpy())
    net.set_tensor_path("tcgen05_ws")
    for a, b in zip(out["tcgen05"], out["tcgen05_ws"]):
        np.testing.assert_array_equal(a, b)


def test_tcgen05_pairing_bit_exact_and_decode(trained):
    net, _ = trained
    net.set_precision("bf16")
    net.set_tensor_path("tcgen05_ws")
    L, shots = 256, 3
    N = oracle.sample_errors(L, shots, 0.05, seed=52)
    Nd = dev(N)
    z = net.logits(Nd).cpu().numpy()
    R, C0 = net.predecode(Nd)
    C, steps, fail = net.decode_batch(Nd)
    net.status()
    R, C0 = R.cpu().numpy(), C0.cpu().numpy()
    A = anyon_maps(N)
    for s in range(shots):
        np.testing.assert_array_equal(C0[s], onet.pairing_links(A[s], onet.proposals(A[s], z[s])))
    np.testing.assert_array_equal(R, N ^ C0)
    Co, so, fo = oracle.decode_shot(R[0], max_steps=4096)
    np.testing.assert_array_equal(C[0].cpu().numpy(), Co ^ C0[0])
    assert (int(steps[0]), int(fail[0])) == (so, fo)


# ------------------------------------------------- training on tensor cores

def test_training_repeats_bit_for_bit():
    # the gradient partial sums are added in a fixed order: two runs from the
    # same initial weights and seed end with the same weights
    a, b = qca.Net(seed=5), qca.Net(seed=5)
    try:
        p0 = a.get_params()
        for net in (a, b):
            net.train(L=16, iterations=40, batch=8, p_lo=0.02, p_hi=0.07, seed=3, lr=2e-3)
        pa, pb = a.get_params(), b.get_params()
        assert np.any(pa != p0)  # the runs did train
        np.testing.assert_array_equal(pa, pb)
    finally:
        a.close()
        b.close()


def test_watchdog_gives_up_and_stops_the_other_waiters():
    # a bounded wait on a barrier that nothing completes gives up after its
    # bound (about 2 s of SM clock) and raises the stop flag, and a second
    # waiter leaves at once; the context stays usable (no fault is involved)
    first, second, t_first, lag = qca.watchdog_selftest()
    assert first and second
    assert 0.5 < t_first < 10.0, t_first
    assert 0.0 <= lag < 0.01, lag
    N = qca.sample_errors(16, 8, 0.05, seed=1)
    C, steps, fail = qca.decode_batch(N, max_steps=4096)
    torch.cuda.synchronize()
    assert int((fail == 3).sum()) == 0


def test_gradients_match_fp64_reference():
    # one training step's gradient (bf16 operands, fp32 accumulation) against
    # the FP64 reference of the same loss: the bf16 rounding of weights and
    # activations bounds the agreement to about 1e-2 relative per layer
    net = qca.Net(seed=4)
    try:
        L, B = 16, 6
        N = oracle.sample_errors(L, B, 0.06, seed=61)
        loss, g = net.gradients(dev(N))
        params = net.get_params()
        A = anyon_maps(N)
        lab = np.stack([onet.first_step_labels(A[b]) for b in range(B)])
        loss_ref, g_ref = onet.loss_and_grads(A, lab, params)
        assert loss == pytest.approx(loss_ref, rel=2e-2)
        o = 0
        for co, ci in onet.LAYERS:
            for n_ in (co * ci * 9, co):
                a, b = g[o:o + n_].astype(np.float64), g_ref[o:o + n_]
                rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
                cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
                assert rel < 5e-2 and cos > 0.998, (co, ci, n_, rel, cos)
                o += n_
        # the weights did not move
        np.testing.assert_array_equal(net.get_params(), params)
    finally:
        net.close()
