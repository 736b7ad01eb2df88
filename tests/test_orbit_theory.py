"""The premise of the on-chip sweep's periodic-orbit stop, checked on the oracle.

With the deterministic rules the message fields after a step's update depend
only on the syndromes of the last 86 steps (a message grows by 3 per step and
is gone after 85).  So once the anyon sets of 89 consecutive steps repeat those
P steps earlier, the whole state repeats with period P and the correction with
period 2P.  These tests run the oracle step by step on shots of the mixed-size
draw (qca_uneven_draw, seed 1000) that never end and check each part of that
claim on the oracle's own state: the message fields, the syndrome, and the
correction's differences.  They also check the sufficiency direction on a
shot that ends: its anyon sets never show such a repeat.
"""
import numpy as np
import pytest

import oracle

SEED = 1000
WINDOW = 89  # anyon sets compared (the kernels' kOrbitWindow + 1)


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def _run(shot, L, steps):
    Ls, thr = oracle.uneven_draw(200000, SEED)
    assert Ls[shot] == L
    N = oracle.sample_errors(L, 1, 0.0, seed=SEED, shot0=shot, thr=int(thr[shot]))[0]
    sigma = oracle.syndrome(N)
    m = np.zeros((4, L, L), dtype=np.int32)
    C = np.zeros((2, L, L), dtype=np.uint8)
    sets, fields, corr = [], [], []
    for t in range(steps):
        sets.append(tuple(np.flatnonzero(sigma.ravel() != 1)))
        fields.append(m.copy())
        corr.append(C.copy())
        n, _ = oracle.step(sigma, m, C, t=t, shot=shot)
        if n == 0:
            break
    return sets, fields, corr


def _first_repeat(sets, P):
    """First step t at which the anyon sets of steps t - WINDOW + 1 .. t equal
    those P steps earlier, or None."""
    run = 0
    for t in range(P, len(sets)):
        run = run + 1 if sets[t] == sets[t - P] else 0
        if run >= WINDOW:
            return t
    return None


@pytest.mark.parametrize("shot,L,P", [(30062, 24, 1), (1616, 24, 24), (1170, 24, 48),
                                      (18968, 24, 32)])
def test_repeating_anyon_sets_make_the_state_periodic(shot, L, P):
    sets, fields, corr = _run(shot, L, 600)
    assert len(sets) == 600  # the shot never ends
    t0 = _first_repeat(sets, P)
    assert t0 is not None
    for t in range(t0, len(sets)):
        # fields at the start of step t are those after step t - 1's update
        assert sets[t] == sets[t - P]
        np.testing.assert_array_equal(fields[t], fields[t - P], err_msg=f"step {t}")
    # the flips repeat with period P, so every window of P steps adds the same
    # links to the correction, and the correction repeats with period 2P
    d0 = corr[t0 + P] ^ corr[t0]
    for t in range(t0, len(sets) - P):
        np.testing.assert_array_equal(corr[t + P] ^ corr[t], d0, err_msg=f"step {t}")
    for t in range(t0, len(sets) - 2 * P):
        np.testing.assert_array_equal(corr[t + 2 * P], corr[t], err_msg=f"step {t}")
    if P > 1:
        assert d0.any()  # a chasing pair drags its links along: a period is not trivial


def test_a_shot_that_ends_shows_no_repeat():
    # shot 0 of the draw is an ordinary shot (it ends within a few dozen steps)
    sets, _, _ = _run(0, int(oracle.uneven_draw(1, SEED)[0][0]), 4096)
    assert len(sets) < 200
    for P in range(1, len(sets)):
        assert _first_repeat(sets, P) is None
