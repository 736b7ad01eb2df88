"""CPU reference of the learned pre-decoder (TEST INFRASTRUCTURE ONLY).

The pre-decoder is not part of the paper: it is a small convolutional net that
proposes, for every anyon, a move toward an adjacent anyon; links whose two end
anyons propose each other are flipped before the paper's automaton finishes
the shot.  Its labels come from the automaton itself: the direction an anyon
takes in the automaton's first step (Def. "D-dimensional message passing
automaton", Eqs. blahdef, degbreak, ddfeedback, readings R1-R4), kept when the
anyon it moves toward moves back, i.e. when the first step annihilates the pair.

Only the tests may import this module.  It uses numpy in float64; the
quantisation points of the GPU kernels (bf16 weights; bf16 activations at layer
boundaries) are applied explicitly so that the two sides compute the same
arithmetic up to accumulation order and precision.
"""
from __future__ import annotations

import numpy as np

import oracle

# layer shapes (c_out, c_in) of the 3x3 circular convolutions
LAYERS = [(32, 2), (32, 32), (32, 32), (4, 32)]
# logit channel k <-> move direction (code k + 1): +x, -x, +y, -y
DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1)]


def param_count() -> int:
    return sum(co * ci * 9 + co for co, ci in LAYERS)


def unpack(params: np.ndarray):
    """Flat float32 parameters -> [(W[co][ci][3][3], b[co]), ...]."""
    out, o = [], 0
    for co, ci in LAYERS:
        W = params[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = params[o:o + co]
        o += co
        out.append((W.astype(np.float64), b.astype(np.float64)))
    assert o == len(params)
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3_circular(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [ci][L][L], W [co][ci][3][3] (tap (ky, kx) <-> offset (ky-1, kx-1)):
    out[co][y][x] = b[co] + sum W[co][ci][ky][kx] x[ci][y+ky-1][x+kx-1] (periodic)."""
    co = W.shape[0]
    L = x.shape[-1]
    out = np.zeros((co, L, L), dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            # shifted[ci][y][x] = x[ci][y + ky - 1][x + kx - 1]
            shifted = np.roll(x, shift=(1 - ky, 1 - kx), axis=(1, 2))
            out += np.einsum("oc,cyx->oyx", W[:, :, ky, kx], shifted)
    return out + b[:, None, None]


def forward(anyon: np.ndarray, params: np.ndarray, quantize: bool = True) -> np.ndarray:
    """Logits [4][L][L] of one syndrome (anyon indicator [L][L])."""
    layers = unpack(params)
    x = np.stack([anyon.astype(np.float64), np.ones_like(anyon, dtype=np.float64)])
    for i, (W, b) in enumerate(layers):
        if quantize:
            W = bf16_round(W)
            x = bf16_round(x)
        x = conv3x3_circular(x, W, b)
        if i < len(layers) - 1:
            x = np.maximum(x, 0.0)
    return x


def first_step_labels(anyon: np.ndarray) -> np.ndarray:
    """Per site: 255 (no anyon), 4 (anyon not in a first-step annihilating
    adjacent pair) or k in 0..3 (direction DIRS[k] toward its partner)."""
    L = anyon.shape[0]
    sigma = np.where(anyon, -1, 1).astype(np.int8)
    m = np.zeros((4, L, L), np.int32)
    for _ in range(3):
        m = oracle.message_substep(sigma, m)
    f = oracle.forces(sigma, m)
    # direction code per anyon: f^x = -1 -> +x, +1 -> -x; same for y
    d = np.full((L, L), -1, np.int32)
    d[f[0] == -1] = 0
    d[f[0] == 1] = 1
    d[f[1] == -1] = 2
    d[f[1] == 1] = 3
    lab = np.full((L, L), 255, np.uint8)
    for y in range(L):
        for x in range(L):
            if not anyon[y, x]:
                continue
            k = d[y, x]
            lab[y, x] = 4
            if k < 0:
                continue
            dx, dy = DIRS[k]
            xn, yn = (x + dx) % L, (y + dy) % L
            back = {0: 1, 1: 0, 2: 3, 3: 2}[k]
            if anyon[yn, xn] and d[yn, xn] == back:
                lab[y, x] = k
    return lab


def proposals(anyon: np.ndarray, logits: np.ndarray) -> np.ndarray:
    """Per anyon: argmax of the four logits if positive, else 4 (no proposal)."""
    k = np.argmax(logits, axis=0)
    best = np.max(logits, axis=0)
    prop = np.where(best > 0.0, k, 4).astype(np.int32)
    return np.where(anyon.astype(bool), prop, 4)


def pairing_links(anyon: np.ndarray, prop: np.ndarray) -> np.ndarray:
    """Links [2][L][L] flipped by the pre-decoder: e_x(r) iff r proposes +x and
    r + x^ proposes -x; e_y(r) likewise with +y / -y."""
    L = anyon.shape[0]
    C0 = np.zeros((2, L, L), np.uint8)
    C0[0] = ((prop == 0) & (np.roll(prop, -1, axis=1) == 1)).astype(np.uint8)
    C0[1] = ((prop == 2) & (np.roll(prop, -1, axis=0) == 3)).astype(np.uint8)
    return C0


# ---------------------------------------------------------------- FP8 form

E4M3_MAX = 448.0


def e4m3_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest FP8 E4M3 value (ties to even), saturating at +-448.

    E4M3: 4 exponent bits (bias 7), 3 mantissa bits, subnormals down to 2^-9,
    largest finite value 1.75 * 2^8 = 448.  Returned as float64."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    _, E = np.frexp(a)                  # a = m 2^E, m in [0.5, 1)
    e = np.maximum(E - 1, -6)           # binade exponent, subnormals share 2^-6's quantum
    quantum = np.ldexp(1.0, e - 3)
    q = np.round(a / quantum) * quantum  # numpy rounds halves to even
    q = np.minimum(q, E4M3_MAX)
    return np.where(x < 0, -q, q)


def fp8_weight_scales(W: np.ndarray) -> np.ndarray:
    """Per output channel: amax over (c_in, taps) / 448 in float32 (1 if the
    channel is all zero)."""
    amax = np.max(np.abs(W.astype(np.float32)).reshape(W.shape[0], -1), axis=1)
    s = (amax / np.float32(E4M3_MAX)).astype(np.float32)
    return np.where(amax > 0, s, np.float32(1.0)).astype(np.float32)


def fp8_weights(W: np.ndarray) -> np.ndarray:
    """Per-channel scaled E4M3 weights, dequantised: e4m3(W / s_co) * s_co with
    the division in float32."""
    W32 = W.astype(np.float32)
    s = fp8_weight_scales(W32)
    q = e4m3_round((W32 / s[:, None, None, None]).astype(np.float32))
    return q * s.astype(np.float64)[:, None, None, None]


def forward_fp8(anyon: np.ndarray, params: np.ndarray, act_scales) -> np.ndarray:
    """Logits [4][L][L] of the FP8 form: layer 1 as the bf16 form (exact inputs,
    bf16 weights); layers 2-4 with per-channel E4M3 weights and E4M3 inputs
    quantised per layer as e4m3(x / s) * s, s = act_scales[layer - 2]."""
    layers = unpack(params)
    x = np.stack([anyon.astype(np.float64), np.ones_like(anyon, dtype=np.float64)])
    for i, (W, b) in enumerate(layers):
        if i == 0:
            x = conv3x3_circular(x, bf16_round(W), b)
        else:
            s = float(np.float32(act_scales[i - 1]))
            xq = e4m3_round(x / s) * s
            x = conv3x3_circular(xq, fp8_weights(W), b)
        if i < len(layers) - 1:
            x = np.maximum(x, 0.0)
    return x


# ------------------------------------------- rounding of stored activations
# Each layer's output is stored in a narrow format before the next layer reads
# it: bf16(relu(z)) in the bf16 form, e4m3(relu(z) / s) * s in the FP8 form.
# The kernels form z as an fp32 sum of the same terms the FP64 reference adds;
# the two sums differ by at most (number of terms) * 2^-23 times the sum of the
# terms' magnitudes (288 products: below 2^-14 of that sum).  Where the stored
# value is not constant over that interval around the FP64 z, either rounding
# is a correct result of the kernel's arithmetic.

ACC_REL_BOUND = 2.0 ** -14


def layer_weights(params: np.ndarray, fp8: bool = False):
    """[(W, b)] as each layer multiplies them: bf16-rounded weights (bf16 form;
    also layer 1 of the FP8 form) or dequantised per-channel e4m3 weights
    (layers 2-4 of the FP8 form)."""
    out = []
    for i, (W, b) in enumerate(unpack(params)):
        out.append((fp8_weights(W) if (fp8 and i > 0) else bf16_round(W), b))
    return out


def conv_magnitude(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Sum of the magnitudes of the terms of each output of conv3x3_circular:
    |b| + sum |W| |x| over taps and input channels."""
    return conv3x3_circular(np.abs(x), np.abs(W), np.abs(b))


def store_activation(z: np.ndarray, scale: float = None) -> np.ndarray:
    """The stored form of relu(z): bf16 (scale None) or e4m3(relu(z) / scale) * scale."""
    r = np.maximum(z, 0.0)
    if scale is None:
        return bf16_round(r)
    return e4m3_round(r / scale) * scale


def store_interval(z: np.ndarray, mag: np.ndarray, scale: float = None,
                   rel: float = ACC_REL_BOUND):
    """Stored values at the two ends of [z - rel*mag, z + rel*mag]: the
    rounding is monotone, so every sum within the interval stores a value
    between them (inclusive), and where they agree exactly that value."""
    d = rel * mag
    return store_activation(z - d, scale), store_activation(z + d, scale)


def dilate(mask: np.ndarray, steps: int) -> np.ndarray:
    """Circular 3x3 dilation of a boolean [..., L, L] map, `steps` times."""
    m = mask.copy()
    for _ in range(steps):
        acc = m.copy()
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                acc |= np.roll(m, shift=(dy, dx), axis=(-2, -1))
        m = acc
    return m


# ------------------------------------------------------------- training

LABEL_SMOOTHING = 0.1


def loss_and_grads(anyons: np.ndarray, labels: np.ndarray, params: np.ndarray):
    """Mean smoothed cross-entropy over the labelled sites of a batch and its
    gradient with respect to the flat parameters, in float64 without
    quantisation.  anyons: uint8 [B][L][L]; labels: uint8 [B][L][L] (0..3
    direction, 4 no move, 255 ignored).  The fifth class has logit 0; the
    target puts 1 - eps + eps/5 on the label and eps/5 elsewhere.

    Backward pass of the four circular 3x3 convolutions written out: for
    out = conv(x, W) + b, dW[o][c][ky][kx] = sum_s dout[o][s] x[c][s + (ky-1, kx-1)],
    db[o] = sum_s dout[o][s], dx[c][s] = sum_{o,ky,kx} W[o][c][ky][kx]
    dout[o][s - (ky-1, kx-1)]; ReLU passes the gradient where its output is
    positive."""
    layers = unpack(params)
    B = anyons.shape[0]
    grads = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
    loss = 0.0
    n = int(np.sum(labels != 255))
    if n == 0:
        return 0.0, np.zeros(param_count())
    q_off = LABEL_SMOOTHING / 5.0
    q_on = 1.0 - LABEL_SMOOTHING + q_off
    for bi in range(B):
        a = anyons[bi]
        xs = [np.stack([a.astype(np.float64), np.ones_like(a, dtype=np.float64)])]
        for i, (W, b) in enumerate(layers):
            y = conv3x3_circular(xs[-1], W, b)
            xs.append(np.maximum(y, 0.0) if i < len(layers) - 1 else y)
        z = xs[-1]                                   # [4][L][L]
        lab = labels[bi]
        zz = np.concatenate([z, np.zeros((1,) + z.shape[1:])])   # fifth class
        m = zz.max(axis=0)
        lse = m + np.log(np.exp(zz - m).sum(axis=0))
        p = np.exp(zz - lse)
        q = np.full_like(zz, q_off)
        valid = lab != 255
        for k in range(5):
            q[k][lab == k] = q_on
        loss += float(np.sum((q * (lse - zz))[:, valid]))
        dz = ((p - q)[:4]) * valid / n
        d = dz
        for i in range(len(layers) - 1, -1, -1):
            W, b = layers[i]
            x = xs[i]
            gW, gb = grads[i]
            for ky in range(3):
                for kx in range(3):
                    shifted = np.roll(x, shift=(1 - ky, 1 - kx), axis=(1, 2))
                    gW[:, :, ky, kx] += np.einsum("oyx,cyx->oc", d, shifted)
            gb += d.sum(axis=(1, 2))
            if i == 0:
                break
            dx = np.zeros_like(x)
            for ky in range(3):
                for kx in range(3):
                    contrib = np.einsum("oc,oyx->cyx", W[:, :, ky, kx], d)
                    dx += np.roll(contrib, shift=(ky - 1, kx - 1), axis=(1, 2))
            d = dx * (x > 0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss / n, flat
