"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Every automaton quantity is an exact integer, so the bar is bit-exact equality
of the correction, the step count and the failure flag for every shot.
Inputs come from the oracle's own noise sampler (never from the CUDA path).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
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


# ------------------------------------------------------------------ sampler --

@pytest.mark.parametrize("L,p,shot0", [(3, 0.3, 0), (16, 0.05, 0), (33, 0.1, 7), (256, 0.05, 123)])
def test_sampler_bit_exact(L, p, shot0):
    shots = 4 if L == 256 else 40
    want = oracle.sample_errors(L, shots, p, seed=5, shot0=shot0)
    got = qca.sample_errors(L, shots, p, seed=5, shot0=shot0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), want)


# ------------------------------------------------------------ worked cases --

LEX_CASES = [c for c in all_cases() if 0 in c["tie_orders"]]


@pytest.mark.parametrize("case", LEX_CASES, ids=[c["name"] for c in LEX_CASES])
def test_golden_cases_on_gpu(case):
    # default options (lexicographic ties); tests/test_rules_gpu.py runs every
    # case under each tie order it is written for
    C, s, f = gpu_decode(case["N"][None], max_steps=case["max_steps"], m_max=case["m_max"])
    assert s[0] == case["steps"] and f[0] == case["flag"]
    np.testing.assert_array_equal(C[0], case["C"])


# -------------------------------------------------------------- parity ----

def test_small_config_full_parity():
    """L = 16, p = 0.05, 1000 shots, seed 0, budget 4096: every shot."""
    N = oracle.sample_errors(16, 1000, 0.05, seed=0)
    assert_same(gpu_decode(N, 4096), oracle.decode_batch(N, max_steps=4096), "L16")


@pytest.mark.parametrize("L", [3, 4, 5, 6, 7, 8, 9, 12, 13, 20, 24, 31, 32, 36, 48, 64, 68, 80, 96,
                               100, 112])
@pytest.mark.parametrize("p", [0.03, 0.09])
def test_parity_across_sizes(L, p):
    shots = 120 if L <= 32 else 40
    N = oracle.sample_errors(L, shots, p, seed=L)
    ms = 600
    assert_same(gpu_decode(N, ms), oracle.decode_batch(N, max_steps=ms), f"L{L} p{p}")


# 136, 160, 200 and 248 (like 68 and 100 above) sweep bands of a height other
# than 4, 8, 16 or 32 rows (17, 20, 25 and 31)
@pytest.mark.parametrize("L", [128, 136, 160, 192, 200, 248, 256])
def test_parity_large_lattices_sampled(L):
    shots = 6
    N = oracle.sample_errors(L, shots, 0.06, seed=3)
    assert_same(gpu_decode(N, 300), oracle.decode_batch(N, max_steps=300), f"L{L}")


@pytest.mark.parametrize("L", [136, 160, 192, 200, 248, 256])
def test_four_cta_clusters_bit_exact(L):
    """Clusters of four CTAs (a quarter of the rows each, two clusters per SM
    pair) against two-CTA clusters and the oracle, with the rule options on."""
    shots = 16
    N = oracle.sample_errors(L, shots, 0.07, seed=L + 5)
    kw = dict(tie_order=1, balance_rule=1, rng_seed=3)
    two = gpu_decode(N, 300, **kw)
    qca.set_cluster_ctas(L, 4)
    try:
        assert qca.get_tuning(L)[2] == 256  # the four-CTA form, not a fallback
        four = gpu_decode(N, 300, **kw)
    finally:
        qca.set_cluster_ctas(L, 2)
    assert_same(four, two, f"L{L}")
    import oracle_pool
    cpu = oracle_pool.decode_many(N[:6], max_steps=300, tie_order=1, balance_rule=1, seed=3)
    assert_same((four[0][:6], four[1][:6], four[2][:6]), cpu, f"L{L} oracle")


@pytest.mark.parametrize("p", [0.08, 0.09])
def test_cluster_path_near_and_above_threshold(p):
    """The two-CTA cluster (L = 256) against the oracle where decoding is hard:
    16 shots at p = 0.08 and 0.09, budget 300; among them shots that exhaust
    the budget (flag 2), a case the bench workload never reaches."""
    import oracle_pool
    L = 256
    assert qca.kernel_path(L) == 2
    N = oracle.sample_errors(L, 16, p, seed=21)
    cpu = oracle_pool.decode_many(N, max_steps=300)
    assert (cpu[2] == 2).any() and (cpu[2] == 1).any()
    assert_same(gpu_decode(N, 300), cpu, f"L256 p{p}")


@pytest.mark.parametrize("v,m_max", [(1, 255), (2, 255), (4, 255), (3, 7), (3, 40), (5, 20)])
def test_parity_options(v, m_max):
    L = 20
    N = oracle.sample_errors(L, 60, 0.06, seed=v * 100 + m_max)
    assert_same(gpu_decode(N, 400, v=v, m_max=m_max),
                oracle.decode_batch(N, max_steps=400, v=v, m_max=m_max), f"v{v} m{m_max}")


@pytest.mark.parametrize("L", [12, 32])
def test_parity_random_moves(L):
    N = oracle.sample_errors(L, 40, 0.05, seed=1)
    thr = oracle.prob_threshold(0.1)
    gpu = gpu_decode(N, 400, p_move=0.1, rng_seed=77, shot_offset=5)
    cpu = oracle.decode_batch(N, max_steps=400, move_thr=thr, seed=77, shot0=5)
    assert_same(gpu, cpu, "p_move")


def test_syndrome_entry_point():
    L = 24
    N = oracle.sample_errors(L, 30, 0.06, seed=8)
    anyon = np.stack([(oracle.syndrome(N[s]) == -1).astype(np.uint8) for s in range(30)])
    C, steps, cut, exh = qca.decode_syndrome_batch(torch.from_numpy(anyon).cuda(), max_steps=300)
    torch.cuda.synchronize()
    for s in range(30):
        Co, so, fo, cuto = oracle.decode_syndrome_shot(anyon[s], max_steps=300)
        assert steps[s].item() == so
        np.testing.assert_array_equal(C[s].cpu().numpy(), Co)
        np.testing.assert_array_equal(cut[s].cpu().numpy(), cuto)
        assert exh[s].item() == (1 if fo == 2 else 0)


def test_host_entry_point_matches_device():
    L = 32
    N = oracle.sample_errors(L, 50, 0.06, seed=9)
    Nh = torch.from_numpy(N).pin_memory()
    C, s, f = qca.decode_batch_host(Nh, max_steps=500)
    assert_same((C.numpy(), s.numpy(), f.numpy()), oracle.decode_batch(N, max_steps=500), "host")


@pytest.mark.parametrize("L,shots", [(256, 1100), (1024, 70)])
def test_host_entry_point_in_several_chunks(L, shots):
    """Batches of three 64 MiB chunks: the host-buffer decode's pipelined copies
    (two buffer sets on two streams for the on-chip sweep, one set for the
    large-lattice sweep) give the device entry point's outputs."""
    N = qca.sample_errors(L, shots, 0.05, seed=4)
    Cd, sd, fd = qca.decode_batch(N, max_steps=600)
    torch.cuda.synchronize()
    C, s, f = qca.decode_batch_host(N.cpu().pin_memory(), max_steps=600)
    assert torch.equal(s, sd.cpu()) and torch.equal(f, fd.cpu())
    assert torch.equal(C, Cd.cpu())


# -------------------------------------------------------------- edges -----

def test_edge_cases():
    # zero shots
    C, s, f = qca.decode_batch(torch.empty((0, 2, 8, 8), dtype=torch.uint8, device="cuda"))
    assert C.shape[0] == 0
    # empty noise and noise that is a closed loop: zero steps
    N = np.zeros((2, 2, 9, 9), np.uint8)
    N[1, 0, 4, :] = 1  # row of e_x: wraps x
    C, s, f = gpu_decode(N)
    assert s.tolist() == [0, 0] and f.tolist() == [0, 1] and not C.any()
    # budget 0 with anyons: exhausted immediately
    N = oracle.sample_errors(10, 5, 0.1, seed=2)
    C, s, f = gpu_decode(N, max_steps=0)
    has = np.array([(oracle.syndrome(N[i]) == -1).any() for i in range(5)])
    assert (f[has] == 2).all() and (s == 0).all() and not C.any()
    # an unsupported size is refused without a fault
    with pytest.raises(qca.QcaError):
        qca.decode_batch(torch.zeros((1, 2, 2, 2), dtype=torch.uint8, device="cuda"))


def test_full_size_properties_and_sampled_parity():
    """The configuration the bench times (L = 256, p = 0.05, 100 000 shots,
    sampled on the device): properties that hold at any size for every shot,
    and oracle parity on sampled shots."""
    L, shots, p = 256, 100_000, 0.05
    N = qca.sample_errors(L, shots, p, seed=0)
    C, steps, fail = qca.decode_batch(N, max_steps=4096)
    torch.cuda.synchronize()
    fail_c = fail.cpu().numpy()
    steps_c = steps.cpu().numpy()
    assert set(np.unique(fail_c)) <= {0, 1, 2}
    assert (steps_c >= 0).all() and (steps_c <= 4096).all()
    assert (steps_c[fail_c == 2] == 4096).all()
    # residual of successful shots is a cycle: zero syndrome (checked on a slice)
    idx = torch.arange(0, shots, 997, device="cuda")
    R = (N[idx] ^ C[idx]).to(torch.int32)
    ex, ey = R[:, 0], R[:, 1]
    par = ex ^ torch.roll(ex, 1, dims=2) ^ ey ^ torch.roll(ey, 1, dims=1)
    ok = torch.from_numpy(fail_c != 2).cuda()[idx]
    assert int(par[ok].sum()) == 0
    # sampled shots against the oracle (noise regenerated by the oracle's sampler)
    rng = np.random.default_rng(0)
    short = np.nonzero(steps_c < 150)[0]  # keep the CPU side to seconds per shot
    for s in sorted(rng.choice(short, 4, replace=False).tolist()):
        Nn = oracle.sample_errors(L, 1, p, seed=0, shot0=s)[0]
        np.testing.assert_array_equal(N[s].cpu().numpy(), Nn)
        Co, so, fo = oracle.decode_shot(Nn, max_steps=4096)
        assert steps_c[s] == so and fail_c[s] == fo, s
        np.testing.assert_array_equal(C[s].cpu().numpy(), Co)
