"""Pins of the 1D oracle (repetition code; Sec. 3.1, Def. "message passing
automaton, 1D"; Sec. 7.1), each derived from the definition by hand or brute
force rather than from the oracle itself."""
import numpy as np
import pytest

import oracle


def sigma_of(L, anyons):
    s = np.ones(L, np.int8)
    for r in anyons:
        s[r % L] = -1
    return s


def noise_of(L, links):
    N = np.zeros(L, np.uint8)
    for r in links:
        N[r % L] ^= 1
    return N


# ---------------------------------------------------------------- messages

@pytest.mark.parametrize("L", [3, 4, 5, 7, 9])
def test_messages_are_upstream_distances(L):
    # from empty fields with sigma frozen, after t sub-steps m^+_r is the
    # smallest d <= min(t, m_max) with an anyon at r - d (0 if none); m^- the
    # same toward r + d
    rng = np.random.default_rng(L)
    for trial in range(20):
        sig = np.where(rng.random(L) < 0.3, -1, 1).astype(np.int8)
        m_max = int(rng.integers(1, 6))
        m = np.zeros((2, L), np.int32)
        for t in range(1, 7):
            m = oracle.substep_1d(sig, m, m_max=m_max)
            for r in range(L):
                for k, s in ((0, 1), (1, -1)):
                    want = 0
                    for d in range(1, min(t, m_max) + 1):
                        if sig[(r - s * d) % L] == -1:
                            want = d
                            break
                    assert m[k, r] == want, (L, trial, t, r, k)


# ------------------------------------------------------------------ forces

def test_force_rule_against_the_prose():
    # an anyon moves toward the only message it hears, or toward the smaller of
    # two; it stays if they are equal or it hears nothing (R1 with the feedback
    # operator: f = -1 moves right, +1 moves left)
    L = 5
    sig = sigma_of(L, [2])
    for mp in range(5):
        for mm in range(5):
            m = np.zeros((2, L), np.int32)
            m[0, 2], m[1, 2] = mp, mm
            f = oracle.forces_1d(sig, m)[2]
            right = mm != 0 and (mp == 0 or mm < mp)
            left = mp != 0 and (mm == 0 or mp < mm)
            assert f == (-1 if right else (1 if left else 0)), (mp, mm, f)
    # non-anyon sites feel no force
    m = np.full((2, L), 3, np.int32)
    m[0, 0] = 1
    assert oracle.forces_1d(sig, m)[0] == 0


def test_feedback_or_and_direction():
    L = 6
    sig = sigma_of(L, [1, 2, 4])
    f = np.zeros(L, np.int8)
    f[1], f[2], f[4] = -1, 1, 1   # 1 moves right, 2 and 4 move left
    F = oracle.feedback_1d(sig, f)
    # <1,2> crossed from both ends flips once; <3,4> by the anyon at 4
    np.testing.assert_array_equal(F, [0, 1, 0, 1, 0, 0])
    f2 = np.zeros(L, np.int8)
    f2[0] = -1  # not an anyon: no move
    assert oracle.feedback_1d(sig, f2).sum() == 0


# -------------------------------------------------------------- hand cases

def test_single_error_one_step():
    N = noise_of(11, [4])
    C, steps, flag, maj = oracle.decode_shot_1d(N)
    np.testing.assert_array_equal(C, N)
    assert (steps, flag, maj) == (1, 0, 0)


def test_gap_of_two_meets_in_the_middle():
    # links 3, 4 flipped: anyons at 3 and 5 step toward each other and meet at 4
    N = noise_of(12, [3, 4])
    C, steps, flag, _ = oracle.decode_shot_1d(N)
    np.testing.assert_array_equal(C, N)
    assert (steps, flag) == (1, 0)


def test_balanced_antipodal_pair_never_moves():
    # even ring, anyons at 0 and 4 of 8: equal messages from both sides forever
    N = noise_of(8, [0, 1, 2, 3])
    C, steps, flag, maj = oracle.decode_shot_1d(N, max_steps=50)
    assert (steps, flag, maj) == (50, 2, 2)
    assert C.sum() == 0


def test_long_way_round_is_a_logical_error_but_matches_the_majority():
    # odd ring of 9: five flipped links (0..4) make anyons at 0 and 5; the
    # decoder closes the shorter gap (links 5..8), so N xor C is all ones:
    # flag 1 against the encoded 0, yet equal to the majority of N (5 of 9)
    N = noise_of(9, [0, 1, 2, 3, 4])
    C, steps, flag, maj = oracle.decode_shot_1d(N)
    np.testing.assert_array_equal(C, noise_of(9, [5, 6, 7, 8]))
    assert flag == 1 and maj == 0


# -------------------------------------------------------------- invariants

def test_invariants_on_random_noise():
    rng = np.random.default_rng(3)
    for L in (10, 17, 32):
        for p in (0.1, 0.3):
            for shot in range(10):
                N = (rng.random(L) < p).astype(np.uint8)
                sig = oracle.syndrome_1d(N)
                m = np.zeros((2, L), np.int32)
                C = np.zeros(L, np.uint8)
                n = int((sig == -1).sum())
                assert n % 2 == 0
                for t in range(200):
                    if n == 0:
                        break
                    n = oracle.step_1d(sig, m, C, t=t)
                    assert n % 2 == 0
                    np.testing.assert_array_equal(sig, oracle.syndrome_1d(N ^ C))
                if n == 0:
                    R = N ^ C
                    assert R.min() == R.max()


def test_random_moves_keep_parity_and_agree_with_decode():
    rng = np.random.default_rng(4)
    thr = oracle.prob_threshold(0.1)
    for shot in range(8):
        N = (rng.random(21) < 0.2).astype(np.uint8)
        C, steps, flag, _ = oracle.decode_shot_1d(N, move_thr=thr, seed=9, shot=shot)
        if flag != 2:
            R = N ^ C
            assert R.min() == R.max() and flag == R[0]


# -------------------------------------------------------------- statistics

def test_threshold_toward_one_half():
    # below p = 1/2 the failure rate falls with L (Sec. 7.1, p_c -> 1/2)
    def plog(L, p, shots):
        N = oracle.sample_errors_1d(L, shots, p, seed=1)
        return np.mean([oracle.decode_shot_1d(n)[2] != 0 for n in N])
    a, b = plog(15, 0.25, 3000), plog(61, 0.25, 3000)
    assert b < a, (a, b)


def test_majority_criterion_below_one_half_at_half():
    # at p = 1/2 the majority-vote criterion leaves p_log below 1/2 (Sec. 7.1)
    N = oracle.sample_errors_1d(15, 3000, 0.5, seed=2)
    maj = np.array([oracle.decode_shot_1d(n)[3] for n in N])
    rate = np.mean(maj[maj != 2] == 1)
    assert rate < 0.5, rate


def test_sampler_rate_and_counter_structure():
    N = oracle.sample_errors_1d(64, 2000, 0.2, seed=5)
    assert abs(N.mean() - 0.2) < 0.01
    sub = oracle.sample_errors_1d(64, 10, 0.2, seed=5, shot0=37)
    np.testing.assert_array_equal(sub, N[37:47])


# ---------------------------------------------------------- gerrymandering

def fractal_noise(n, k, m):
    """The substitution S_{n,k}(X) = X^{(x) k} (x) 1^{(x) (n-k)} iterated m times
    on one X (the gerrymandering construction of Sec. 5.3): link i of the ring
    of n^m links is flipped iff every base-n digit of i is below k (k^m flips)."""
    x = np.arange(n ** m)
    keep = np.ones(n ** m, bool)
    for _ in range(m):
        keep &= (x % n) < k
        x //= n
    return keep.astype(np.uint8)


UNCAPPED = 1 << 30  # the numerics of Sec. 7 set no cap on the messages


def test_gerrymander_flips_the_logical_state_in_about_035_L():
    # Sec. 5.3: with n = 6 (k = 5) and v = 3 the decoder drives the fractal
    # pattern to the flipped logical state, although from m = 4 on the pattern
    # flips a minority of the links (5^m < 6^m / 2): a logical failure by the
    # majority criterion too; its decoding time approaches 0.35 L as L grows
    ratios = []
    for m in (2, 3, 4, 5):
        N = fractal_noise(6, 5, m)
        L = N.size
        C, steps, flag, maj = oracle.decode_shot_1d(N, v=3, m_max=UNCAPPED, max_steps=200000)
        R = N ^ C
        assert R.min() == R.max() == 1 and flag == 1, (m, steps, flag)
        assert maj == (1 if 2 * int(N.sum()) < L else 0), (m, maj)
        ratios.append(steps / L)
    assert all(a < b for a, b in zip(ratios, ratios[1:])), ratios
    assert 0.33 <= ratios[-1] <= 0.36, ratios


def test_gerrymander_with_n5_needs_v5():
    # Sec. 5.3: for n = 5 the pattern is driven to the flipped state only if
    # v >= 5 (at m = 6, L = 15625; smaller m still flip at v = 4)
    N = fractal_noise(5, 4, 6)
    outcomes = {v: oracle.decode_shot_1d(N, v=v, m_max=UNCAPPED, max_steps=200000)[2]
                for v in (3, 4, 5)}
    assert outcomes == {3: 0, 4: 0, 5: 1}, outcomes


def test_gerrymander_under_the_message_cap_strands_a_pair():
    # with 8-bit messages (m_max = 255) the m = 4 pattern leaves one pair 440
    # links apart, beyond any message's reach: it never moves again (R5, R10)
    N = fractal_noise(6, 5, 4)
    C, steps, flag, _ = oracle.decode_shot_1d(N, v=3, m_max=255, max_steps=2000)
    assert (steps, flag) == (2000, 2)
    R = N ^ C
    anyons = np.nonzero(R ^ np.roll(R, 1))[0]
    assert anyons.size == 2
    gap = int(anyons[1] - anyons[0])
    assert min(gap, N.size - gap) > 255
