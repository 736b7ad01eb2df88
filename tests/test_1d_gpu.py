"""GPU parity of the 1D decoder (repetition code on a ring; Sec. 3.1,
Def. "message passing automaton, 1D"; Sec. 7.1) against the CPU oracle:
bit-exact correction, steps, flag and majority flag for every shot."""
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
    torch.cuda.synchronize()


def run(N, **kw):
    C, s, f, m = qca.decode_1d_batch(torch.from_numpy(np.ascontiguousarray(N)).cuda(), **kw)
    torch.cuda.synchronize()
    return C.cpu().numpy(), s.cpu().numpy(), f.cpu().numpy(), m.cpu().numpy()


def check(N, max_steps=4096, v=3, m_max=255, p_move=0.0, rng_seed=0, label=""):
    C, s, f, m = run(N, max_steps=max_steps, v=v, m_max=m_max, p_move=p_move, rng_seed=rng_seed)
    thr = oracle.prob_threshold(p_move) if p_move > 0 else 0
    for i, n in enumerate(N):
        Co, so, fo, mo = oracle.decode_shot_1d(n, v=v, m_max=m_max, max_steps=max_steps,
                                                move_thr=thr, seed=rng_seed, shot=i)
        assert (s[i], f[i], m[i]) == (so, fo, mo), (label, i, s[i], so, f[i], fo)
        np.testing.assert_array_equal(C[i], Co, err_msg=f"{label} shot {i}")


def test_sampler_bit_exact():
    for L, p, shot0 in [(3, 0.4, 0), (100, 0.1, 7), (4097, 0.3, 0)]:
        got = qca.sample_errors_1d(L, 20, p, seed=4, shot0=shot0).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.sample_errors_1d(L, 20, p, seed=4, shot0=shot0))


@pytest.mark.parametrize("L", [3, 4, 5, 8, 31, 64, 257, 1000])
def test_sizes_and_rates(L):
    for p in (0.05, 0.2, 0.45):
        check(oracle.sample_errors_1d(L, 60, p, seed=L), label=f"L={L} p={p}")


@pytest.mark.parametrize("v,m_max", [(1, 255), (2, 255), (3, 2), (5, 4), (8, 255), (3, 1)])
def test_speeds_and_caps(v, m_max):
    check(oracle.sample_errors_1d(40, 80, 0.2, seed=v), v=v, m_max=m_max, label=f"v={v} m={m_max}")


def test_random_moves_and_budget():
    N = oracle.sample_errors_1d(64, 100, 0.3, seed=9)
    check(N, p_move=0.1, rng_seed=3, label="p_move")
    check(N, max_steps=2, label="budget 2")
    check(N, max_steps=0, label="budget 0")


def test_large_ring_and_full_batch_properties():
    L, shots = 16384, 256
    N = qca.sample_errors_1d(L, shots, 0.3, seed=0)
    C, s, f, m = qca.decode_1d_batch(N)
    R = (N ^ C)
    done = f != 2
    assert bool(((R.max(1).values == R.min(1).values) | ~done).all())
    Nh = N[:2].cpu().numpy()
    for i in range(2):
        Co, so, fo, mo = oracle.decode_shot_1d(Nh[i])
        assert (int(s[i]), int(f[i]), int(m[i])) == (so, fo, mo)
        np.testing.assert_array_equal(C[i].cpu().numpy(), Co)


def fractal_noise(n, k, m):
    # the gerrymandering pattern of Sec. 5.3: link i of the ring of n^m links
    # is flipped iff every base-n digit of i is below k
    x = np.arange(n ** m)
    keep = np.ones(n ** m, bool)
    for _ in range(m):
        keep &= (x % n) < k
        x //= n
    return keep.astype(np.uint8)


@pytest.mark.parametrize("n,k,m,v", [(6, 5, 3, 3), (5, 4, 4, 4), (5, 4, 4, 3), (6, 5, 4, 3)])
def test_gerrymander_patterns_bit_exact(n, k, m, v):
    # structured inputs from the paper: driven to the flipped logical state
    # (6, 5, 3 at v = 3; 5, 4, 4 at v = 4), decoded correctly (5, 4, 4 at
    # v = 3), and a pair stranded beyond the 8-bit messages' reach (6, 5, 4)
    N = fractal_noise(n, k, m)[None, :]
    check(N, max_steps=2000, v=v, label=f"fractal n={n} m={m} v={v}")
