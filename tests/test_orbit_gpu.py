"""Shots in periodic orbits: the on-chip sweep's fast-forward against the oracle.

With the deterministic rules a shot whose anyon set repeats with period P over
the message lifetime never ends; the on-chip sweep stops it early at a step
whose state equals that of the step budget and reports what a run to the budget
reports.  The oracle always runs to the budget, so every case below checks the
shortcut bit for bit: correction, step count and flag.

The shots come from the mixed-size draw (qca_uneven_draw, seed 1000); the
oracle, run over all 200 000 of its shots, finds 429 that never end within
4096 steps.  One shot per kind of orbit is taken: a pair that does not move
(period 1), pairs chasing around the torus with periods L, 2L, 4L/3, 7L/6, 9/8 L,
7L, 9L and 15L, two four-anyon orbits, sizes 24 to 192 (one-CTA and two-CTA
sweeps), and one L = 128 shot with no period the sweep's ring can hold (it runs
to the budget).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import oracle_pool  # noqa: E402
import paper_2506_03266_gb300 as qca  # noqa: E402

SEED = 1000
# (shot index in the draw, L, period found by the oracle; 0 = none up to 3900)
ORBITS = [
    (30062, 24, 1), (1616, 24, 24), (180305, 24, 24), (18968, 24, 32), (1170, 24, 48),
    (1476, 48, 48), (50470, 48, 56), (10860, 48, 336), (2553, 64, 64), (26849, 64, 64),
    (7946, 64, 72), (32764, 64, 576), (4878, 48, 720), (3668, 96, 96), (97881, 128, 128),
    (22942, 128, 0), (179038, 192, 192),
]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    qca.build()
    oracle.build()
    qca.lib()


@pytest.fixture(scope="module")
def noise():
    Ls, thr = oracle.uneven_draw(200000, SEED)
    out = {}
    for s, L, _ in ORBITS:
        assert Ls[s] == L
        out[s] = oracle.sample_errors(L, 1, 0.0, seed=SEED, shot0=s, thr=int(thr[s]))[0]
    return out


def _budgets(L):
    return (4096, 4095, 1001, 777) if L <= 64 else ((4096, 1001) if L <= 128 else (4096,))


def test_orbit_shots_match_the_oracle_at_several_budgets(noise):
    jobs, keys = [], []
    for s, L, _ in ORBITS:
        for b in _budgets(L):
            jobs.append((noise[s], dict(max_steps=b)))
            keys.append((s, L, b))
    want = oracle_pool.run_many("decode_shot", jobs)
    for (s, L, b), (Co, so, fo) in zip(keys, want):
        assert fo == 2 and so == b, (s, b)  # the oracle confirms the shot never ends
        N = torch.from_numpy(noise[s][None]).cuda()
        C, steps, fail = qca.decode_batch(N, max_steps=b)
        torch.cuda.synchronize()
        assert int(steps[0]) == so and int(fail[0]) == fo, (s, L, b)
        np.testing.assert_array_equal(C[0].cpu().numpy(), Co, err_msg=f"shot {s} L {L} budget {b}")


def test_orbit_shots_from_their_syndromes(noise):
    """The syndrome entry point: correction, step count, cut parities and the
    exhausted flag of orbit shots against the oracle's syndrome decoder."""
    picks = [(s, L) for s, L, _ in ORBITS if L in (24, 48)][:5]
    jobs = []
    for s, L in picks:
        anyon = (oracle.syndrome(noise[s]) < 0).astype(np.uint8)
        jobs.append((anyon, dict(max_steps=999)))
    want = oracle_pool.run_many("decode_syndrome_shot", jobs)
    for (s, L), (anyon, _), (Co, so, fo, cut) in zip(picks, jobs, want):
        assert fo == 2
        sig = torch.from_numpy(anyon[None]).cuda()
        C, steps, cutg, exh = qca.decode_syndrome_batch(sig, max_steps=999)
        torch.cuda.synchronize()
        assert int(steps[0]) == so and int(exh[0]) == 1, s
        np.testing.assert_array_equal(cutg[0].cpu().numpy(), np.asarray(cut, np.uint8))
        np.testing.assert_array_equal(C[0].cpu().numpy(), Co)


def test_orbit_shots_in_the_mixed_size_launch(noise):
    """The orbit shots of sizes up to 192 in one uneven batch (one mixed-size
    launch: a 512-thread CTA per L = 192 shot, smaller groups below) against
    the oracle."""
    shots = [(s, L) for s, L, _ in ORBITS]
    Ls = np.array([L for _, L in shots], dtype=np.int32)
    plan = qca.UnevenPlan(Ls)
    plan.set_mode("mixed")
    flat = np.zeros(max(int(plan.offsets[i]) + 2 * L * L for i, (_, L) in enumerate(shots)),
                    dtype=np.uint8)
    for i, (s, L) in enumerate(shots):
        flat[plan.offsets[i]:plan.offsets[i] + 2 * L * L] = noise[s].ravel()
    N = torch.from_numpy(flat).cuda()
    C, steps, fail = plan.decode(N, max_steps=1001)
    torch.cuda.synchronize()
    want = oracle_pool.run_many("decode_shot", [(noise[s], dict(max_steps=1001))
                                                for s, _ in shots])
    Ch, st, fl = C.cpu().numpy(), steps.cpu().numpy(), fail.cpu().numpy()
    for i, ((s, L), (Co, so, fo)) in enumerate(zip(shots, want)):
        assert st[i] == so and fl[i] == fo, s
        np.testing.assert_array_equal(Ch[plan.offsets[i]:plan.offsets[i] + 2 * L * L],
                                      Co.ravel(), err_msg=f"shot {s}")
    plan.close()


@pytest.mark.parametrize("L,p", [(32, 0.08), (48, 0.075)])
def test_near_threshold_batch_with_long_budget(L, p):
    """Every shot of a near-threshold batch against the oracle at a 1500-step
    budget: the shots that end keep their own outcome (no orbit is claimed for
    them) and the 3-4 % that never end match the budget's outcome."""
    n = 1500
    N_np = oracle.sample_errors(L, n, p, seed=77)
    Co, so, fo = oracle_pool.decode_many(N_np, max_steps=1500)
    assert (fo == 2).sum() > 20 and (fo != 2).sum() > 1000  # both kinds occur
    C, steps, fail = qca.decode_batch(torch.from_numpy(N_np).cuda(), max_steps=1500)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(steps.cpu().numpy(), so)
    np.testing.assert_array_equal(fail.cpu().numpy(), fo)
    np.testing.assert_array_equal(C.cpu().numpy(), Co)
