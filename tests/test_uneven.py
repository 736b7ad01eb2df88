"""Uneven batches (shots of mixed lattice sizes) through the C ABI.

The per-shot draw of (L, p) is host code and is checked here against the
oracle's independent implementation; the GPU tests check the packed sampler and
decoder against the oracle shot by shot, against the uniform entry point per
size, and under CUDA-graph capture and replay.
"""
import numpy as np
import pytest

import oracle
import paper_2506_03266_gb300 as qca


@pytest.fixture(scope="module")
def built():
    qca.build()
    oracle.build()
    return qca.lib()


def test_uneven_draw_matches_oracle(built):
    L, thr = qca.uneven_draw(20000, 7)
    Lo, thro = oracle.uneven_draw(20000, 7)
    np.testing.assert_array_equal(L, Lo)
    np.testing.assert_array_equal(thr, thro)


def test_uneven_draw_distribution(built):
    n = 200000
    L, thr = qca.uneven_draw(n, 0)
    want = {24: 0.30, 48: 0.25, 64: 0.20, 96: 0.12, 128: 0.08, 192: 0.05}
    assert set(np.unique(L)) == set(want)
    for size, w in want.items():
        f = (L == size).mean()
        assert abs(f - w) < 5 * np.sqrt(w * (1 - w) / n), (size, f)
    p = thr.astype(np.float64) / 2.0**64
    assert p.min() >= 0.01 - 1e-12 and p.max() < 0.07
    assert abs(p.mean() - 0.04) < 5 * 0.06 / np.sqrt(12 * n)


torch = pytest.importorskip("torch")


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.gpu
def test_uneven_sampler_and_decoder_against_oracle(built):
    _cuda()
    shots = 400
    L, thr = qca.uneven_draw(shots, 3)
    plan = qca.UnevenPlan(L)
    N = plan.sample(thr, seed=3)
    C, steps, fail = plan.decode(N, max_steps=800)
    torch.cuda.synchronize()
    Nh, Ch = N.cpu().numpy(), C.cpu().numpy()
    steps, fail = steps.cpu().numpy(), fail.cpu().numpy()
    # every shot's noise equals the oracle's draw for that shot index
    for s in range(0, shots, 7):
        n = 2 * int(L[s]) ** 2
        blk = Nh[plan.offsets[s]:plan.offsets[s] + n].reshape(2, L[s], L[s])
        np.testing.assert_array_equal(
            blk, oracle.sample_errors(int(L[s]), 1, 0.0, seed=3, shot0=s, thr=int(thr[s]))[0])
    # decode: small shots all against the oracle, every shot per size against
    # the uniform entry point
    small = [s for s in range(shots) if L[s] <= 48][:60]
    for s in small:
        n = 2 * int(L[s]) ** 2
        blk = Nh[plan.offsets[s]:plan.offsets[s] + n].reshape(2, L[s], L[s])
        Co, so, fo = oracle.decode_shot(blk, max_steps=800)
        assert steps[s] == so and fail[s] == fo, s
        np.testing.assert_array_equal(Ch[plan.offsets[s]:plan.offsets[s] + n].reshape(Co.shape), Co)
    for size in np.unique(L):
        idx = np.nonzero(L == size)[0]
        blocks = np.stack([Nh[plan.offsets[s]:plan.offsets[s] + 2 * size * size].reshape(
            2, size, size) for s in idx])
        Cu, su, fu = qca.decode_batch(torch.from_numpy(blocks).cuda(), max_steps=800)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(su.cpu().numpy(), steps[idx])
        np.testing.assert_array_equal(fu.cpu().numpy(), fail[idx])
        Cus = Cu.cpu().numpy()
        for k, s in enumerate(idx):
            np.testing.assert_array_equal(
                Ch[plan.offsets[s]:plan.offsets[s] + 2 * size * size].reshape(2, size, size),
                Cus[k])
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["per_size", "mixed"])
def test_uneven_decode_in_cuda_graph(built, mode):
    _cuda()
    shots = 600
    L, thr = qca.uneven_draw(shots, 5)
    plan = qca.UnevenPlan(L)
    plan.set_mode(mode)
    N = plan.sample(thr, seed=5)
    C0, s0, f0 = plan.decode(N, max_steps=800)  # uncaptured call sizes the workspaces
    torch.cuda.synchronize()
    out = (torch.zeros_like(N), torch.zeros(shots, dtype=torch.int32, device="cuda"),
           torch.zeros(shots, dtype=torch.uint8, device="cuda"))
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        plan.decode(N, max_steps=800, out=out, stream=stream)
    for _ in range(2):
        out[1].zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out[1], s0) and torch.equal(out[2], f0) and torch.equal(out[0], C0)
    plan.close()


@pytest.mark.gpu
@pytest.mark.parametrize("tie_order,balance_rule", [(0, 0), (1, 1)])
def test_mixed_launch_matches_per_size_launches(built, tie_order, balance_rule):
    """The single mixed-size launch (pairs of CTAs for L > 192, one CTA per shot
    for 64 < L <= 192, several groups per CTA below) against one launch per
    size, bit for bit, on nine on-chip sizes (the ninth and smallest runs in a
    launch of its own: the queue takes eight) and two odd sizes packed last
    (byte-access sweep); the small sizes also against the oracle."""
    _cuda()
    rng = np.random.default_rng(11)
    even = [256, 192, 136, 128, 80, 64, 40, 24, 12]
    L = np.array(rng.permutation(np.repeat(even, [3, 4, 4, 6, 8, 10, 12, 14, 16])).tolist()
                 + [33, 33, 21, 21], dtype=np.int32)
    thr = np.full(len(L), oracle.prob_threshold(0.06), dtype=np.uint64)
    plan = qca.UnevenPlan(L)
    N = plan.sample(thr, seed=9)
    kw = dict(max_steps=400, rng_seed=13, tie_order=tie_order, balance_rule=balance_rule)
    plan.set_mode("mixed")
    mixed = [t.cpu().numpy() for t in plan.decode(N, **kw)]
    plan.set_mode("per_size")
    per = [t.cpu().numpy() for t in plan.decode(N, **kw)]
    for a, b in zip(mixed, per):
        np.testing.assert_array_equal(a, b)
    Nh = N.cpu().numpy()
    for s in [i for i in range(len(L)) if L[i] <= 40][:30]:
        n = 2 * int(L[s]) ** 2
        blk = Nh[plan.offsets[s]:plan.offsets[s] + n].reshape(2, L[s], L[s])
        Co, so, fo = oracle.decode_shot(blk, max_steps=400, tie_order=tie_order,
                                        balance_rule=balance_rule, seed=13, shot=s)
        assert mixed[1][s] == so and mixed[2][s] == fo, s
        np.testing.assert_array_equal(
            mixed[0][plan.offsets[s]:plan.offsets[s] + n].reshape(Co.shape), Co)
    plan.close()
