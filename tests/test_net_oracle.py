"""Pins of the pre-decoder's CPU reference (oracle/net.py), no GPU needed.

The net is not part of the paper; what pins it is plain mathematics and
library routines: bfloat16 round-to-nearest-even against torch's own
conversion, the circular 3x3 convolution against torch's conv2d with circular
padding and against single-tap shifts worked out by hand, and the labels
against the automaton rule (Def. "D-dimensional message passing automaton",
Eqs. blahdef / degbreak / ddfeedback) on hand-derived configurations and
against the oracle's full decoder step.
"""
import numpy as np
import pytest
import torch

import oracle
import oracle.net as onet


def rng_params(seed, scale=0.3):
    r = np.random.default_rng(seed)
    return (r.standard_normal(onet.param_count()) * scale).astype(np.float32)


# ------------------------------------------------------------- bf16 rounding

def test_bf16_round_hand_values():
    # spacing of bf16 just above 1 is 2^-7; midpoints round to the even neighbour
    x = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, 1 + 2**-7, -(1 + 2**-8) , 1 + 2**-8 + 2**-20])
    want = [1.0, 1.0, 1 + 2**-6, 1 + 2**-7, -1.0, 1 + 2**-7]
    assert list(onet.bf16_round(x)) == want


def test_bf16_round_matches_torch_conversion():
    r = np.random.default_rng(0)
    x = np.concatenate([r.standard_normal(20000) * 10.0 ** r.integers(-6, 6, 20000),
                        np.array([0.0, -0.0, 65504.0, 1e-30])]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(onet.bf16_round(x), want)


# ------------------------------------------------------- circular convolution

@pytest.mark.parametrize("ky,kx", [(0, 0), (0, 2), (2, 1), (1, 1)])
def test_conv_single_tap_is_a_shift(ky, kx):
    # out[y][x] = in[y + ky - 1][x + kx - 1]: a single input 1 at (x0, y0) shows
    # up at (x0 - kx + 1, y0 - ky + 1), wrapped
    L, x0, y0 = 5, 0, 4
    inp = np.zeros((1, L, L))
    inp[0, y0, x0] = 1.0
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, ky, kx] = 2.0
    out = onet.conv3x3_circular(inp, W, np.array([0.5]))
    want = np.full((1, L, L), 0.5)
    want[0, (y0 - ky + 1) % L, (x0 - kx + 1) % L] += 2.0
    np.testing.assert_array_equal(out, want)


def test_conv_matches_torch_circular_conv2d():
    r = np.random.default_rng(1)
    x = r.standard_normal((3, 7, 7))
    W = r.standard_normal((4, 3, 3, 3))
    b = r.standard_normal(4)
    xt = torch.nn.functional.pad(torch.from_numpy(x)[None], (1, 1, 1, 1), mode="circular")
    want = torch.nn.functional.conv2d(xt, torch.from_numpy(W), torch.from_numpy(b))[0].numpy()
    np.testing.assert_allclose(onet.conv3x3_circular(x, W, b), want, rtol=1e-12, atol=1e-12)


def test_forward_matches_torch_net():
    L = 9
    r = np.random.default_rng(2)
    anyon = (r.random((L, L)) < 0.2).astype(np.uint8)
    params = rng_params(3)
    x = torch.from_numpy(np.stack([anyon.astype(np.float64), np.ones((L, L))]))[None]
    for i, (W, b) in enumerate(onet.unpack(params)):
        x = torch.nn.functional.pad(x, (1, 1, 1, 1), mode="circular")
        x = torch.nn.functional.conv2d(x, torch.from_numpy(W), torch.from_numpy(b))
        if i < 3:
            x = torch.relu(x)
    np.testing.assert_allclose(onet.forward(anyon, params, quantize=False), x[0].numpy(),
                               rtol=1e-10, atol=1e-10)


def test_forward_quantized_close_to_exact_and_exact_on_bf16_grid():
    L = 8
    r = np.random.default_rng(4)
    anyon = (r.random((L, L)) < 0.2).astype(np.uint8)
    params = rng_params(5)
    zq = onet.forward(anyon, params, quantize=True)
    z = onet.forward(anyon, params, quantize=False)
    assert np.max(np.abs(zq - z)) < 0.05 * max(1.0, np.max(np.abs(z)))
    # a net whose weights are bf16 values and whose activations stay on the bf16
    # grid (single-layer paths of small integers) is unchanged by quantisation
    p = np.zeros(onet.param_count(), np.float32)
    o = 0
    for li, (co, ci) in enumerate(onet.LAYERS):
        W = np.zeros((co, ci, 3, 3), np.float32)
        W[0, 0, 1, 1] = 1.0  # channel 0 passes through the centre tap
        if li == 0:
            W[0, 0, 1, 2] = 1.0  # plus the anyon to the right
        p[o:o + W.size] = W.ravel()
        o += W.size + co
    zq = onet.forward(anyon, p, quantize=True)
    want = anyon + np.roll(anyon, -1, axis=1)
    np.testing.assert_array_equal(zq[0], want)
    np.testing.assert_array_equal(zq[1:], 0)


def test_param_layout():
    assert onet.param_count() == 32 * 2 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 4 * 32 * 9 + 4
    p = np.arange(onet.param_count(), dtype=np.float32)
    layers = onet.unpack(p)
    assert layers[0][0][0, 0, 0, 0] == 0 and layers[0][1][0] == 576
    assert layers[3][1][-1] == onet.param_count() - 1


# ------------------------------------------------------------------- labels

def noise_with(L, links):
    N = np.zeros((2, L, L), np.uint8)
    for plane, x, y in links:
        N[plane, y % L, x % L] ^= 1
    return N


def anyons_of(N):
    return (oracle.syndrome(N) == -1).astype(np.uint8)


def test_labels_single_x_error():
    # one flipped e_x((3, 2)): anyons at (3, 2) and (4, 2) see each other's
    # message at distance 1 and step toward each other
    L = 9
    lab = onet.first_step_labels(anyons_of(noise_with(L, [(0, 3, 2)])))
    assert lab[2, 3] == 0 and lab[2, 4] == 1
    assert np.count_nonzero(lab != 255) == 2


def test_labels_single_y_error_across_the_seam():
    # e_y((1, L-1)) joins (1, L-1) and (1, 0) through the periodic boundary
    L = 8
    lab = onet.first_step_labels(anyons_of(noise_with(L, [(1, 1, L - 1)])))
    assert lab[L - 1, 1] == 2 and lab[0, 1] == 3


def test_labels_diagonal_pair_is_not_adjacent():
    # two links forming an L: anyons at (2, 2) and (3, 3), diagonal neighbours
    L = 9
    lab = onet.first_step_labels(anyons_of(noise_with(L, [(0, 2, 2), (1, 3, 2)])))
    assert lab[2, 2] == 4 and lab[3, 3] == 4


def test_labels_balanced_middle_anyon_does_not_move():
    # anyons at x = 2, 3, 4 on row 4 plus a distant one: the middle anyon hears
    # distance 1 from both sides of the x axis (balanced: no move, reading R4),
    # so nobody forms a mutual pair with it
    L = 12
    sig = np.zeros((L, L), np.uint8)
    for x, y in [(2, 4), (3, 4), (4, 4), (9, 9)]:
        sig[y, x] = 1
    lab = onet.first_step_labels(sig)
    assert lab[4, 3] == 4
    assert lab[4, 2] == 4 and lab[4, 4] == 4


def test_labels_symmetric_and_realised_by_the_oracle_step():
    # a labelled pair (r, r + a^) is mutual, and the oracle's own first step
    # flips the link between them (a third anyon may still step onto r, so the
    # pair's sites need not end empty)
    r = np.random.default_rng(7)
    for L, p in [(10, 0.05), (16, 0.08), (13, 0.03)]:
        for _ in range(6):
            N = (r.random((2, L, L)) < p).astype(np.uint8)
            sig = oracle.syndrome(N)
            lab = onet.first_step_labels((sig == -1).astype(np.uint8))
            s2 = sig.copy()
            m = np.zeros((4, L, L), np.int32)
            C = np.zeros((2, L, L), np.uint8)
            oracle.step(s2, m, C)
            for y, x in zip(*np.nonzero(lab < 4)):
                k = lab[y, x]
                dx, dy = onet.DIRS[k]
                xn, yn = (x + dx) % L, (y + dy) % L
                assert lab[yn, xn] == k ^ 1
                plane = 0 if k < 2 else 1
                lx, ly = (x, y) if k in (0, 2) else (xn, yn)
                assert C[plane, ly, lx] == 1
            assert np.all((lab == 255) == (sig == 1))


# -------------------------------------------------------- proposals / pairing

def test_proposals_rules():
    L = 3
    anyon = np.array([[1, 1, 0], [1, 1, 1], [0, 0, 1]], np.uint8)
    z = np.zeros((4, L, L))
    z[:, 0, 0] = [0.1, 0.5, 0.5, -1]   # tie between 1 and 2: first index
    z[:, 0, 1] = [-0.1, -0.2, -3, -1]  # nothing positive: no proposal
    z[:, 1, 0] = [0, 0, 0, 0]          # zero is not positive
    z[:, 1, 1] = [0, 0, 0, 2.0]
    z[:, 0, 2] = [9, 9, 9, 9]          # not an anyon
    prop = onet.proposals(anyon, z)
    assert prop[0, 0] == 1 and prop[0, 1] == 4 and prop[1, 0] == 4 and prop[1, 1] == 3
    assert prop[0, 2] == 4


def test_pairing_links_hand_cases_and_wrap():
    L = 5
    prop = np.full((L, L), 4, np.int32)
    prop[1, 4], prop[1, 0] = 0, 1      # across the x seam: link e_x((4, 1))
    prop[3, 2], prop[4, 2] = 2, 3      # e_y((2, 3))
    prop[0, 2], prop[0, 3] = 0, 4      # one-sided: no link
    C0 = onet.pairing_links(np.ones((L, L), np.uint8), prop)
    assert C0[0, 1, 4] == 1 and C0[1, 3, 2] == 1
    assert C0.sum() == 2
    # the syndrome of C0 is exactly the four paired anyons
    s = oracle.syndrome(C0)
    assert set(zip(*np.nonzero(s == -1))) == {(1, 4), (1, 0), (3, 2), (4, 2)}


def test_labels_as_proposals_pair_exactly_the_labelled_anyons():
    r = np.random.default_rng(11)
    L = 14
    N = (r.random((2, L, L)) < 0.06).astype(np.uint8)
    anyon = anyons_of(N)
    lab = onet.first_step_labels(anyon)
    prop = np.where(lab < 4, lab, 4).astype(np.int32)
    C0 = onet.pairing_links(anyon, prop)
    paired = oracle.syndrome(C0) == -1
    np.testing.assert_array_equal(paired, lab < 4)


# --------------------------------------------------------------- FP8 (E4M3)

def test_e4m3_hand_values():
    x = np.array([0.0, 1.0, 1.0625, 1.1875, 448.0, 500.0, -600.0, 2.0**-9, 2.0**-10,
                  3 * 2.0**-10, 240.0, 232.0, 0.3])
    want = [0.0, 1.0, 1.0, 1.25, 448.0, 448.0, -448.0, 2.0**-9, 0.0, 2.0**-8, 240.0, 224.0,
            0.3125]
    np.testing.assert_array_equal(onet.e4m3_round(x), want)


def test_e4m3_matches_torch_conversion_in_range():
    r = np.random.default_rng(5)
    x = (r.standard_normal(50000) * 10.0 ** r.uniform(-3, 2.3, 50000)).astype(np.float32)
    x = x[np.abs(x) < 440]
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(onet.e4m3_round(x), want)


def test_fp8_weights_per_channel_scale():
    r = np.random.default_rng(6)
    W = (r.standard_normal((4, 3, 3, 3)) * np.array([1, 10, 0.01, 0])[:, None, None, None]
         ).astype(np.float32)
    s = onet.fp8_weight_scales(W)
    assert s[3] == 1.0
    Wq = onet.fp8_weights(W)
    # the largest entry of each nonzero channel maps exactly onto +-448 * s
    for c in range(3):
        k = np.argmax(np.abs(W[c]))
        assert abs(Wq[c].ravel()[k]) == pytest.approx(448.0 * float(s[c]), rel=1e-7)
        assert np.max(np.abs(Wq[c] - W[c])) <= np.max(np.abs(W[c])) / 16 + 1e-12
    assert np.all(Wq[3] == 0)


def test_forward_fp8_close_to_bf16_form():
    L = 10
    r = np.random.default_rng(8)
    anyon = (r.random((L, L)) < 0.2).astype(np.uint8)
    params = rng_params(9, scale=0.1)
    zb = onet.forward(anyon, params, quantize=True)
    # activation scales from the exact form's per-layer input maxima
    acts, x = [], np.stack([anyon.astype(np.float64), np.ones((L, L))])
    for i, (W, b) in enumerate(onet.unpack(params)):
        if i > 0:
            acts.append(np.max(x))
        x = np.maximum(onet.conv3x3_circular(x, W, b), 0) if i < 3 else x
    scales = [max(a, 1e-6) / 448.0 for a in acts]
    z8 = onet.forward_fp8(anyon, params, scales)
    assert np.max(np.abs(z8 - zb)) < 0.2 * max(1.0, np.max(np.abs(zb)))
    assert np.max(np.abs(z8 - zb)) > 0  # the FP8 points do change the result


# ---------------------------------------------------------------- training

def test_loss_and_grads_match_torch_autograd():
    r = np.random.default_rng(12)
    B, L = 2, 7
    anyons = (r.random((B, L, L)) < 0.25).astype(np.uint8)
    labels = np.where(anyons == 1, r.integers(0, 5, (B, L, L)), 255).astype(np.uint8)
    params = rng_params(13, scale=0.2)
    loss, g = onet.loss_and_grads(anyons, labels, params)
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.from_numpy(np.stack([anyons.astype(np.float64), np.ones((B, L, L))], axis=1))
    o = 0
    for i, (co, ci) in enumerate(onet.LAYERS):
        W = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        x = torch.nn.functional.conv2d(torch.nn.functional.pad(x, (1, 1, 1, 1), mode="circular"),
                                       W, b)
        if i < 3:
            x = torch.relu(x)
    z = torch.cat([x, torch.zeros(B, 1, L, L, dtype=torch.float64)], dim=1)   # [B][5][L][L]
    lab = torch.from_numpy(labels.astype(np.int64))
    valid = lab != 255
    eps = 0.1   # the training recipe's label smoothing, stated here, not read from the oracle
    assert onet.LABEL_SMOOTHING == eps
    logp = torch.log_softmax(z, dim=1)
    onehot = torch.nn.functional.one_hot(torch.where(valid, lab, 0), 5).permute(0, 3, 1, 2)
    q = eps / 5 + (1 - eps) * onehot.double()
    tl = -(q * logp).sum(dim=1)[valid].mean()
    tl.backward()
    assert loss == pytest.approx(float(tl.detach()), rel=1e-12)
    np.testing.assert_allclose(g, p.grad.numpy(), rtol=1e-9, atol=1e-12)


def test_loss_and_grads_finite_differences():
    r = np.random.default_rng(14)
    B, L = 1, 5
    anyons = (r.random((B, L, L)) < 0.3).astype(np.uint8)
    labels = np.where(anyons == 1, r.integers(0, 5, (B, L, L)), 255).astype(np.uint8)
    params = rng_params(15, scale=0.2).astype(np.float64)
    _, g = onet.loss_and_grads(anyons, labels, params)
    for k in r.choice(onet.param_count(), 12, replace=False):
        h = 1e-5
        pp, pm = params.copy(), params.copy()
        pp[k] += h
        pm[k] -= h
        num = (onet.loss_and_grads(anyons, labels, pp)[0] - onet.loss_and_grads(anyons, labels, pm)[0]) / (2 * h)
        assert num == pytest.approx(g[k], rel=1e-4, abs=1e-9), k
