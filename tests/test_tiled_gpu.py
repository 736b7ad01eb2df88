"""GPU parity of the large-lattice kernel (8-CTA cluster per shot, state in
global memory, bulk-copy staged bands) against the CPU oracle.

The kernel takes L > 256 (multiples of 128) by default; `qca_set_kernel_path`
forces it onto L = 128 and 256 so that many shots can be checked against the
oracle quickly.  Bit-exact correction, steps and flag for every shot.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2506_03266_gb300 as qca  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qca.build()
    oracle.build()
    qca.lib()
    yield
    for L in (128, 256):
        qca.set_kernel_path(L, -1)
    torch.cuda.synchronize()


def gpu_decode(N_np, max_steps=4096, **kw):
    N = torch.from_numpy(np.ascontiguousarray(N_np)).cuda()
    C, steps, fail = qca.decode_batch(N, max_steps=max_steps, **kw)
    torch.cuda.synchronize()
    return C.cpu().numpy(), steps.cpu().numpy(), fail.cpu().numpy()


def oracle_decode(N_np, max_steps=4096, **kw):
    out = [oracle.decode_shot(n, max_steps=max_steps, **kw) for n in N_np]
    return (np.stack([o[0] for o in out]), np.array([o[1] for o in out], np.int32),
            np.array([o[2] for o in out], np.uint8))


def assert_same(gpu, cpu, label=""):
    C, s, f = gpu
    Co, so, fo = cpu
    bad = np.nonzero((s != so) | (f != fo) | (C != Co).reshape(len(s), -1).any(1))[0]
    assert bad.size == 0, f"{label}: {bad.size} shots differ, first {bad[:8].tolist()} " \
                          f"steps gpu {s[bad[:4]].tolist()} cpu {so[bad[:4]].tolist()} " \
                          f"flags gpu {f[bad[:4]].tolist()} cpu {fo[bad[:4]].tolist()}"


def test_path_selection():
    assert qca.kernel_path(384) == 3 and qca.kernel_path(1024) == 3
    assert qca.kernel_path(256) == 2 and qca.kernel_path(320) == 0
    qca.set_kernel_path(128, 3)
    assert qca.kernel_path(128) == 3
    qca.set_kernel_path(128, -1)
    assert qca.kernel_path(128) == 1
    with pytest.raises(qca.QcaError):
        qca.set_kernel_path(96, 3)


@pytest.mark.parametrize("p,shots,budget", [(0.05, 120, 4096), (0.09, 30, 300), (0.02, 60, 4096)])
def test_forced_L128_bit_exact(p, shots, budget):
    # above threshold (p = 0.09) many shots run long: a 300-step budget keeps
    # the oracle quick and still checks exhausted shots
    qca.set_kernel_path(128, 3)
    try:
        N = oracle.sample_errors(128, shots, p, seed=11)
        assert_same(gpu_decode(N, max_steps=budget), oracle_decode(N, max_steps=budget),
                    f"L=128 p={p}")
    finally:
        qca.set_kernel_path(128, -1)


def test_forced_L128_budget_and_options():
    qca.set_kernel_path(128, 3)
    try:
        N = oracle.sample_errors(128, 24, 0.08, seed=12)
        for kw in [dict(max_steps=3), dict(max_steps=0), dict(m_max=7, max_steps=400),
                   dict(p_move=0.2, rng_seed=5, max_steps=400)]:
            ms = kw.pop("max_steps", 4096)
            okw = {}
            if "m_max" in kw:
                okw["m_max"] = kw["m_max"]
            if "p_move" in kw:
                okw["move_thr"] = int(np.floor(kw["p_move"] * 2.0**64))
                okw["seed"] = kw["rng_seed"]
            want = [oracle.decode_shot(n, max_steps=ms, shot=i, **okw) for i, n in enumerate(N)]
            want = (np.stack([w[0] for w in want]), np.array([w[1] for w in want], np.int32),
                    np.array([w[2] for w in want], np.uint8))
            assert_same(gpu_decode(N, max_steps=ms, **kw), want, f"L=128 {kw} max_steps={ms}")
    finally:
        qca.set_kernel_path(128, -1)


def test_forced_L256_matches_oracle_and_onchip_kernel():
    N = oracle.sample_errors(256, 400, 0.05, seed=13)
    onchip = gpu_decode(N)
    qca.set_kernel_path(256, 3)
    try:
        tiled = gpu_decode(N)
    finally:
        qca.set_kernel_path(256, -1)
    assert_same(tiled, onchip, "L=256 tiled vs on-chip")
    assert_same((tiled[0][:16], tiled[1][:16], tiled[2][:16]), oracle_decode(N[:16]),
                "L=256 tiled vs oracle")


@pytest.mark.parametrize("L,shots,p", [(384, 3, 0.06), (512, 1, 0.05)])
def test_default_sizes_bit_exact(L, shots, p):
    N = oracle.sample_errors(L, shots, p, seed=14)
    assert_same(gpu_decode(N), oracle_decode(N), f"L={L}")


def test_syndrome_entry_L384():
    L, shots = 384, 3
    N = oracle.sample_errors(L, shots, 0.06, seed=15)
    sig = np.stack([(oracle.syndrome(n) == -1).astype(np.uint8) for n in N])
    C, steps, cut, exh = qca.decode_syndrome_batch(torch.from_numpy(sig).cuda())
    torch.cuda.synchronize()
    Co, so, fo = oracle_decode(N)
    np.testing.assert_array_equal(C.cpu().numpy(), Co)
    np.testing.assert_array_equal(steps.cpu().numpy(), so)
    np.testing.assert_array_equal(exh.cpu().numpy(), (fo == 2).astype(np.uint8))


@pytest.mark.parametrize("p,n_sampled", [(0.05, 4), (0.07, 2)])
def test_L1024_sampled_shots_and_full_batch_properties(p, n_sampled):
    # the large-lattice workload's size: one launch over 64 shots; every shot
    # checked for an empty final syndrome, and sampled shots (the longest one
    # among them) against the oracle, decoded in parallel worker processes
    import oracle_pool
    L, shots = 1024, 64
    N = qca.sample_errors(L, shots, p, seed=0)
    C, steps, fail = qca.decode_batch(N, max_steps=4096)
    torch.cuda.synchronize()
    assert int((fail == 3).sum()) == 0
    E = (N ^ C).to(torch.int32)
    ex, ey = E[:, 0], E[:, 1]
    sig = ex ^ torch.roll(ex, 1, dims=2) ^ ey ^ torch.roll(ey, 1, dims=1)
    done = (fail != 2)
    assert int(sig[done].sum()) == 0
    steps_c = steps.cpu().numpy()
    rng = np.random.default_rng(int(p * 1000))
    pick = [int(np.argmax(steps_c))] + \
        rng.choice(np.setdiff1d(np.arange(shots), [np.argmax(steps_c)]), n_sampled - 1,
                   replace=False).tolist()
    Nh = N[pick].cpu().numpy()
    Co, so, fo = oracle_pool.decode_many(Nh, max_steps=4096)
    for i, s in enumerate(pick):
        assert int(steps[s]) == so[i] and int(fail[s]) == fo[i], s
        np.testing.assert_array_equal(C[s].cpu().numpy(), Co[i])
