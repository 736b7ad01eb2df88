"""GPU parity of the 2D variants (open boundaries; uncoordinated
desynchronisation, Sec. 7.3) against the CPU oracle: bit-exact correction,
steps / ticks and flag for every shot."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("L,p", [(3, 0.2), (5, 0.1), (8, 0.05), (17, 0.08), (32, 0.04), (48, 0.06)])
def test_open_bit_exact(L, p):
    N = oracle.sample_errors(L, 40, p, seed=L)      # entries of absent links are ignored
    C, s, f = qca.decode_open_batch(dev(N))
    torch.cuda.synchronize()
    C, s, f = C.cpu().numpy(), s.cpu().numpy(), f.cpu().numpy()
    for i, n in enumerate(N):
        Co, so, fo = oracle.open_decode_shot(n)
        np.testing.assert_array_equal(C[i], Co, err_msg=f"L={L} shot {i}")
        assert (s[i], f[i]) == (so, fo), (L, i)


def test_open_options():
    N = oracle.sample_errors(20, 30, 0.07, seed=3)
    for kw in [dict(v=1), dict(v=5), dict(m_max=4), dict(max_steps=2)]:
        ms = kw.pop("max_steps", 4096)
        C, s, f = qca.decode_open_batch(dev(N), max_steps=ms, **kw)
        torch.cuda.synchronize()
        for i, n in enumerate(N):
            Co, so, fo = oracle.open_decode_shot(n, max_steps=ms, **kw)
            np.testing.assert_array_equal(C[i].cpu().numpy(), Co)
            assert (int(s[i]), int(f[i])) == (so, fo), (kw, i)


@pytest.mark.parametrize("L,p,q,v", [(8, 0.06, 0.3, 3), (16, 0.05, 0.1, 3), (13, 0.08, 1.0, 1),
                                      (24, 0.04, 0.5, 2)])
def test_desync_bit_exact(L, p, q, v):
    N = oracle.sample_errors(L, 30, p, seed=L + 1)
    C, t, f = qca.decode_desync_batch(dev(N), q, max_ticks=20000, rng_seed=11, v=v,
                                      shot_offset=4)
    torch.cuda.synchronize()
    C, t, f = C.cpu().numpy(), t.cpu().numpy(), f.cpu().numpy()
    for i, n in enumerate(N):
        Co, to, fo = oracle.desync_decode_shot(n, q, v=v, max_ticks=20000, seed=11, shot=4 + i)
        np.testing.assert_array_equal(C[i], Co, err_msg=f"L={L} q={q} shot {i}")
        assert (t[i], f[i]) == (to, fo), (L, q, i)


def test_desync_full_rate_matches_synchronous_v1_on_gpu():
    N = qca.sample_errors(64, 2000, 0.05, seed=0)
    C1, t1, f1 = qca.decode_desync_batch(N, 1.0, max_ticks=4096, v=1)
    C2, t2, f2 = qca.decode_batch(N, max_steps=4096, v=1)
    assert torch.equal(C1, C2) and torch.equal(t1, t2) and torch.equal(f1, f2)
