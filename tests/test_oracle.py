"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form, a worked example derived by hand from the paper's text
(tests/golden), an invariant of the dynamics, or a published test vector.
"""
import os

import numpy as np
import pytest

from golden_cases import GOLDEN, all_cases

CASES = all_cases()


# ------------------------------------------------------------------ noise --

def test_splitmix64_reference_vectors(oracle_mod):
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for z, want in rows:
        # the generator seeded with state z returns splitmix64(z) as its first output
        assert oracle_mod.splitmix64(int(z)) == int(want, 16)


def test_probability_threshold(oracle_mod):
    assert oracle_mod.prob_threshold(0.0) == 0
    assert oracle_mod.prob_threshold(0.5) == 2**63
    assert oracle_mod.prob_threshold(0.25) == 2**62
    assert oracle_mod.prob_threshold(1.0) == 2**64 - 1
    assert oracle_mod.prob_threshold(-0.3) == 0


@pytest.mark.parametrize("p", [0.01, 0.05, 0.2])
def test_noise_rate_and_anyon_density(oracle_mod, p):
    """i.i.d. flips (Sec. 7): the edge rate is p and, because a vertex sees four
    independent links, the anyon density is (1 - (1 - 2p)^4) / 2."""
    L, shots = 32, 100
    N = oracle_mod.sample_errors(L, shots, p, seed=11)
    n = N.size
    rate = N.mean()
    assert abs(rate - p) < 5 * np.sqrt(p * (1 - p) / n)
    anyons = np.array([(oracle_mod.syndrome(N[s]) == -1).mean() for s in range(shots)])
    rho = (1 - (1 - 2 * p) ** 4) / 2
    m = shots * L * L
    assert abs(anyons.mean() - rho) < 6 * np.sqrt(rho * (1 - rho) / m)


def test_noise_extremes_and_counter_structure(oracle_mod):
    assert oracle_mod.sample_errors(8, 3, 0.0, 5).sum() == 0
    assert oracle_mod.sample_errors(8, 3, 1.0, 5).min() == 1
    full = oracle_mod.sample_errors(10, 8, 0.1, 3)
    part = oracle_mod.sample_errors(10, 5, 0.1, 3, shot0=3)
    assert np.array_equal(full[3:], part)  # counter-based: shot index is a key
    other = oracle_mod.sample_errors(10, 8, 0.1, 4)
    assert not np.array_equal(full, other)
    # coupled across p: a lower p flips a subset of a higher p's links
    lo = oracle_mod.sample_errors(10, 8, 0.05, 3)
    assert np.all(lo <= full)


# --------------------------------------------------------------- syndrome --

def test_syndrome_of_single_link_and_loops(oracle_mod):
    L = 6
    N = np.zeros((2, L, L), np.uint8)
    N[0, 2, 4] = 1  # e_x((4,2)) = <(4,2),(5,2)>
    s = oracle_mod.syndrome(N)
    assert sorted(zip(*np.nonzero(s == -1))) == [(2, 4), (2, 5)]
    N = np.zeros((2, L, L), np.uint8)
    N[1, 5, 0] = 1  # e_y((0,5)) wraps to (0,0)
    s = oracle_mod.syndrome(N)
    assert sorted(zip(*np.nonzero(s == -1))) == [(0, 0), (5, 0)]
    # a plaquette boundary and a non-contractible loop have empty syndromes
    P = np.zeros((2, L, L), np.uint8)
    P[0, 1, 1] = P[0, 2, 1] = P[1, 1, 1] = P[1, 1, 2] = 1
    assert (oracle_mod.syndrome(P) == 1).all()
    R = np.zeros((2, L, L), np.uint8)
    R[1, :, 3] = 1
    assert (oracle_mod.syndrome(R) == 1).all()


# --------------------------------------------------------------- messages --

def _closed_form(anyon, t, m_max):
    """Infinity-norm cone distance (Sec. 3.2 text around the cone C^{+-a}, and
    Fig. construction (b)): m^{s a}_r after t sub-steps from m = 0 with sigma
    frozen equals the smallest d in [1, min(t, m_max)] such that an anyon sits at
    r - s d a^ + j b^ for some |j| <= d (periodic), else 0."""
    L = anyon.shape[0]
    out = np.zeros((4, L, L), np.int32)
    for k, (s, a) in enumerate([(1, 0), (-1, 0), (1, 1), (-1, 1)]):
        for y in range(L):
            for x in range(L):
                best = 0
                for d in range(1, min(t, m_max) + 1):
                    hit = False
                    for j in range(-d, d + 1):
                        if a == 0:
                            xx, yy = x - s * d, y + j
                        else:
                            xx, yy = x + j, y - s * d
                        if anyon[yy % L, xx % L]:
                            hit = True
                            break
                    if hit:
                        best = d
                        break
                out[k, y, x] = best
    return out


@pytest.mark.parametrize("L,density,m_max", [(3, 0.2, 255), (4, 0.1, 255), (5, 0.08, 255),
                                             (7, 0.05, 255), (8, 0.03, 255), (9, 0.04, 4)])
def test_messages_equal_cone_distance(oracle_mod, L, density, m_max):
    rng = np.random.default_rng(L * 101 + m_max)
    for trial in range(3):
        anyon = rng.random((L, L)) < density
        if not anyon.any():
            anyon[rng.integers(L), rng.integers(L)] = True
        sigma = np.where(anyon, -1, 1).astype(np.int8)
        m = np.zeros((4, L, L), np.int32)
        for t in range(1, 2 * L + 3):
            m = oracle_mod.message_substep(sigma, m, m_max=m_max)
            np.testing.assert_array_equal(m, _closed_form(anyon, t, m_max), err_msg=f"t={t}")


def test_single_anyon_message_values(oracle_mod):
    """Sec. 3.1: a message's value is the time it has propagated.  A lone anyon
    at the centre of a 15 x 15 torus: after 3 sub-steps m^{+x} = 1, 2, 3 on the
    columns x0+1..x0+3 inside the cone |dy| <= dx, and 0 elsewhere."""
    L, x0, y0 = 15, 7, 7
    sigma = np.ones((L, L), np.int8)
    sigma[y0, x0] = -1
    m = np.zeros((4, L, L), np.int32)
    for _ in range(3):
        m = oracle_mod.message_substep(sigma, m)
    want = np.zeros((L, L), np.int32)
    for dx in (1, 2, 3):
        for dy in range(-dx, dx + 1):
            want[y0 + dy, x0 + dx] = dx
    np.testing.assert_array_equal(m[0], want)
    np.testing.assert_array_equal(m[1], want[:, ::-1])  # (-,x) mirror image
    np.testing.assert_array_equal(m[2], want.T)  # (+,y) transposed
    np.testing.assert_array_equal(m[3], want.T[::-1, :])  # (-,y)


# ------------------------------------------------------- forces, feedback --

def _printed_key_link(mpx, mmx, mpy, mmy):
    """Expected move under the option that takes Eq. degbreak as printed: the
    axis of argmin over the nonzero fields of m + s*a/(D+1), D = 2, evaluated
    in exact rationals; where two keys are equal the larger m wins.  Then, as
    in the prose, the anyon moves toward the smaller field of that axis (an
    empty field counts as +infinity) and stays when the two are equal."""
    from fractions import Fraction
    vals = {(1, 1): mpx, (-1, 1): mmx, (1, 2): mpy, (-1, 2): mmy}
    cands = [(v + Fraction(s * a, 3), -v, (s, a)) for (s, a), v in vals.items() if v > 0]
    if not cands:
        return None
    _, _, (s, a) = min(cands)
    mp, mm = vals[(1, a)] or 10**9, vals[(-1, a)] or 10**9
    if mp == mm:
        return None
    return (a, -1) if mp < mm else (a, +1)


def _prose_link(mpx, mmx, mpy, mmy):
    """Expected move of an anyon from the prose of Sec. 1 and Sec. 3.1/3.2: it
    moves one link toward the source of its smallest nonzero message (m^{+a}
    comes from an anyon on the -a side, so it moves -a); among equal smallest
    messages the degeneracy breaking prefers the smaller s*a; it stays put when
    the two messages on the chosen axis are equal.  Returns (axis, +-1) or None."""
    vals = {(1, 1): mpx, (-1, 1): mmx, (1, 2): mpy, (-1, 2): mmy}
    cands = [(v, s * a, (s, a)) for (s, a), v in vals.items() if v > 0]
    if not cands:
        return None
    v, _, (s, a) = min(cands)
    opp = vals[(-s, a)]
    if opp == v:
        return None
    return (a, -s)


@pytest.mark.parametrize("tie_order", [0, 1])
def test_forces_and_feedback_follow_prose(oracle_mod, tie_order):
    """Tie order 0 against the prose reading; tie order 1 against the printed
    key of Eq. degbreak.  Fields 0..4 cover every exact key tie (values one
    apart) and every plain tie."""
    L, x0, y0 = 5, 2, 2
    sigma = np.ones((L, L), np.int8)
    sigma[y0, x0] = -1
    vals = range(0, 5)
    expect = _prose_link if tie_order == 0 else _printed_key_link
    for mpx in vals:
        for mmx in vals:
            for mpy in vals:
                for mmy in vals:
                    m = np.zeros((4, L, L), np.int32)
                    m[:, y0, x0] = (mpx, mmx, mpy, mmy)
                    f = oracle_mod.forces(sigma, m, tie_order=tie_order)
                    F = oracle_mod.feedback_links(sigma, f)
                    want = np.zeros((2, L, L), np.uint8)
                    mv = expect(mpx, mmx, mpy, mmy)
                    if mv is not None:
                        a, d = mv
                        if a == 1:
                            want[0, y0, x0 if d > 0 else x0 - 1] = 1
                        else:
                            want[1, y0 if d > 0 else y0 - 1, x0] = 1
                    np.testing.assert_array_equal(F, want, err_msg=str((mpx, mmx, mpy, mmy)))


def test_non_anyon_sites_never_move(oracle_mod):
    """Reading R2: feedback acts on anyons only; messages at empty sites are
    inert."""
    L = 6
    sigma = np.ones((L, L), np.int8)
    m = np.random.default_rng(1).integers(0, 5, (4, L, L)).astype(np.int32)
    f = oracle_mod.forces(sigma, m)
    assert not f.any()
    assert not oracle_mod.feedback_links(sigma, f).any()


def test_feedback_or_flips_shared_link_once(oracle_mod):
    """The OR of Def. 1d_msg_passing: two anyons crossing the same link flip it
    once (they annihilate instead of swapping)."""
    L = 6
    sigma = np.ones((L, L), np.int8)
    sigma[3, 1] = sigma[3, 2] = -1
    f = np.zeros((2, L, L), np.int8)
    f[0, 3, 1] = -1  # anyon at (1,3) moves +x
    f[0, 3, 2] = +1  # anyon at (2,3) moves -x
    F = oracle_mod.feedback_links(sigma, f)
    assert F.sum() == 1 and F[0, 3, 1] == 1


# ------------------------------------------------------- worked examples --

CASE_TIES = [(c, t) for c in CASES for t in c["tie_orders"]]


@pytest.mark.parametrize("case,tie_order", CASE_TIES,
                         ids=[f"{c['name']}-tie{t}" for c, t in CASE_TIES])
def test_golden_worked_examples(oracle_mod, case, tie_order):
    C, steps, flag = oracle_mod.decode_shot(case["N"], m_max=case["m_max"],
                                            max_steps=case["max_steps"], tie_order=tie_order)
    assert steps == case["steps"]
    assert flag == case["flag"]
    np.testing.assert_array_equal(C, case["C"])


def test_tie_golden_cases_discriminate(oracle_mod):
    """Each case written for one tie order fails under the other, so the two
    options really differ on them."""
    for c in CASES:
        if len(c["tie_orders"]) != 1:
            continue
        other = 1 - c["tie_orders"][0]
        C, steps, flag = oracle_mod.decode_shot(c["N"], m_max=c["m_max"],
                                                max_steps=c["max_steps"], tie_order=other)
        assert not np.array_equal(C, c["C"]), c["name"]


def test_balanced_random_rule(oracle_mod):
    """Balance rule 1 (R4 option): the antipodal pair of an even torus, a
    steady state of the deterministic rule, gets moving.  Anyons at (0,0) and
    (3,0) on L = 6 hear m^{+x} = m^{-x} = 3 after the first step (wrap), so
    their axis x is balanced; each moves +x when the top bit of its draw
    sm(sm(sm(sm(seed ^ BALANCE) ^ shot) ^ t) ^ r) is 0, else -x."""
    L = 6
    N = np.zeros((2, L, L), np.uint8)
    N[0, 0, 0:3] = 1  # e_x((0,0)), e_x((1,0)), e_x((2,0)): anyons at (0,0), (3,0)
    sm = oracle_mod.splitmix64
    seed, shot = 77, 5
    k = sm(sm(sm(seed ^ 0x42414C414E4345) ^ shot) ^ 0)
    want = np.zeros((2, L, L), np.uint8)
    for x in (0, 3):
        bit = sm(k ^ x) >> 63  # site index r = y*L + x with y = 0
        want[0, 0, x if bit == 0 else (x - 1) % L] ^= 1
    C, steps, flag = oracle_mod.decode_shot(N, max_steps=1, balance_rule=1, seed=seed, shot=shot)
    np.testing.assert_array_equal(C, want)
    # deterministic rule: stuck until the budget; random rule: the pair meets
    _, steps0, flag0 = oracle_mod.decode_shot(N, max_steps=200)
    assert (steps0, flag0) == (200, 2)
    for sh in range(8):
        _, st, fl = oracle_mod.decode_shot(N, max_steps=200, balance_rule=1, seed=seed, shot=sh)
        assert fl != 2 and st < 200


# -------------------------------------------------------------- invariants --

@pytest.mark.parametrize("L,p", [(8, 0.05), (9, 0.08), (12, 0.1), (6, 0.15)])
def test_step_invariants(oracle_mod, L, p):
    N = oracle_mod.sample_errors(L, 6, p, seed=L)
    for s in range(N.shape[0]):
        sigma = oracle_mod.syndrome(N[s])
        m = np.zeros((4, L, L), np.int32)
        C = np.zeros((2, L, L), np.uint8)
        for t in range(200):
            n_before = int((sigma == -1).sum())
            if n_before == 0:
                break
            assert n_before % 2 == 0  # anyons are created and removed in pairs
            anyon_before = sigma == -1
            n_after, F = oracle_mod.step(sigma, m, C, t=t)
            # every flipped link touches an anyon (no vacuum moves, R2)
            ex_ok = anyon_before | np.roll(anyon_before, -1, axis=1)
            ey_ok = anyon_before | np.roll(anyon_before, -1, axis=0)
            assert not (F[0].astype(bool) & ~ex_ok).any()
            assert not (F[1].astype(bool) & ~ey_ok).any()
            assert F.sum() <= n_before  # at most one link per anyon
            # sigma <- sigma * sigma_F agrees with measuring N xor C afresh
            np.testing.assert_array_equal(sigma, oracle_mod.syndrome(N[s] ^ C))
            assert n_after == int((sigma == -1).sum())
            assert n_after % 2 == 0
            assert (m >= 0).all() and (m <= 255).all()


def test_success_leaves_homologically_consistent_cycle(oracle_mod):
    L = 12
    N = oracle_mod.sample_errors(L, 40, 0.06, seed=2)
    C, steps, flags = oracle_mod.decode_batch(N, max_steps=500)
    for s in range(N.shape[0]):
        if flags[s] == 2:
            continue
        R = N[s] ^ C[s]
        assert (oracle_mod.syndrome(R) == 1).all()
        # a closed loop crosses every vertical cut with one parity, every
        # horizontal cut with one parity
        col = [int(R[0, :, c].sum() % 2) for c in range(L)]
        row = [int(R[1, r, :].sum() % 2) for r in range(L)]
        assert len(set(col)) == 1 and len(set(row)) == 1
        assert flags[s] == int(col[0] or row[0])


def test_empty_input_is_fixed_point(oracle_mod):
    for L in (3, 4, 16):
        N = np.zeros((2, L, L), np.uint8)
        C, steps, flag = oracle_mod.decode_shot(N)
        assert steps == 0 and flag == 0 and not C.any()


@pytest.mark.parametrize("dx,dy", [(1, 0), (0, 3), (5, 7)])
def test_translation_covariance(oracle_mod, dx, dy):
    """The rules depend on neither r nor t (Def. synch_ccqs, Eq. localcond)."""
    L = 11
    N = oracle_mod.sample_errors(L, 12, 0.07, seed=9)
    C, steps, flags = oracle_mod.decode_batch(N, max_steps=300)
    Ns = np.roll(N, shift=(dy, dx), axis=(2, 3))
    Cs, steps_s, flags_s = oracle_mod.decode_batch(Ns, max_steps=300)
    np.testing.assert_array_equal(steps, steps_s)
    np.testing.assert_array_equal(flags, flags_s)
    np.testing.assert_array_equal(np.roll(C, shift=(dy, dx), axis=(2, 3)), Cs)


def test_syndrome_entry_matches_noise_entry(oracle_mod):
    """Decoding sees only sigma (footnote of Def. plogandtdec); failure is the
    cut parity of N xor C = cut(N) xor cut(C)."""
    L = 10
    N = oracle_mod.sample_errors(L, 15, 0.06, seed=4)
    for s in range(N.shape[0]):
        C, steps, flag = oracle_mod.decode_shot(N[s], max_steps=300)
        anyon = (oracle_mod.syndrome(N[s]) == -1).astype(np.uint8)
        C2, steps2, flag2, cut = oracle_mod.decode_syndrome_shot(anyon, max_steps=300)
        np.testing.assert_array_equal(C, C2)
        assert steps == steps2
        if flag != 2:
            wx, wy = oracle_mod.cut_parity(N[s])
            assert flag == int((wx ^ cut[0]) or (wy ^ cut[1]))
        else:
            assert flag2 == 2


def test_random_moves_option(oracle_mod):
    L = 10
    N = oracle_mod.sample_errors(L, 6, 0.05, seed=5)
    base = oracle_mod.decode_batch(N, max_steps=300)
    zero = oracle_mod.decode_batch(N, max_steps=300, move_thr=0, seed=99)
    for a, b in zip(base, zero):
        np.testing.assert_array_equal(a, b)  # p_move = 0: the seed is unused
    # always-random moves still preserve anyon parity and sigma consistency
    sigma = oracle_mod.syndrome(N[0])
    m = np.zeros((4, L, L), np.int32)
    C = np.zeros((2, L, L), np.uint8)
    for t in range(20):
        n, F = oracle_mod.step(sigma, m, C, move_thr=2**64 - 1, seed=3, t=t)
        assert n % 2 == 0
        np.testing.assert_array_equal(sigma, oracle_mod.syndrome(N[0] ^ C))


# -------------------------------------------------------------- statistics --

def test_logical_failure_ordering_and_high_noise_limit(oracle_mod):
    """Sec. 7.2: well below p_c ~ 7.3% failures are rare, above it they are
    common, and at p = 1/2 the residual is a uniformly random homology class,
    so p_log -> 3/4 (either cycle counts)."""
    L = 16
    lo = oracle_mod.decode_batch(oracle_mod.sample_errors(L, 300, 0.02, seed=1), max_steps=600)[2]
    hi = oracle_mod.decode_batch(oracle_mod.sample_errors(L, 300, 0.12, seed=1), max_steps=600)[2]
    p_lo, p_hi = (lo > 0).mean(), (hi > 0).mean()
    assert p_lo < 0.02
    assert p_hi > 0.3
    half = oracle_mod.decode_batch(oracle_mod.sample_errors(L, 300, 0.5, seed=1), max_steps=600)[2]
    p_half = (half > 0).mean()
    assert abs(p_half - 0.75) < 4 * np.sqrt(0.75 * 0.25 / 300) + 0.02
