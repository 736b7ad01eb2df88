"""Pins of the 2D variant oracles: open boundaries (Appendix "Open boundary
conditions", Def. "message passing automaton with open boundaries") and
uncoordinated desynchronisation (Sec. 7.3), each derived from the definitions
by hand, by brute force, or by reduction to the synchronous decoder."""
import numpy as np
import pytest

import oracle


def links(L, items):
    N = np.zeros((2, L, L), np.uint8)
    for a, x, y in items:
        N[a, y, x] ^= 1
    return N


# ------------------------------------------------------------ open lattice

def test_open_link_set():
    L = 6
    m = oracle.open_link_mask(L)
    assert m[0, :, : L - 1].all() and not m[0, :, L - 1].any()   # x links up to x = L-2
    assert not m[1, :, 0].any() and not m[1, :, L - 1].any()     # no y links on the rough columns
    assert m[1, : L - 1, 1 : L - 1].all() and not m[1, L - 1].any()


def test_open_syndrome_ignores_missing_links_and_boundary():
    L = 7
    E = np.ones((2, L, L), np.uint8)   # every entry set, existing or not
    s = oracle.open_syndrome(E)
    assert (s[:, 0] == 1).all() and (s[:, L - 1] == 1).all()    # boundary sites never anyons
    # interior degree: 2 x links + 2 y links inside, 3 on the top and bottom rows
    assert (s[1:-1, 1:-1] == 1).all()
    assert (s[0, 1:-1] == -1).all() and (s[L - 1, 1:-1] == -1).all()


@pytest.mark.parametrize("L", [5, 6, 9])
def test_open_messages_are_distances_to_anyons_or_the_boundary(L):
    # after t sub-steps from empty fields with sigma frozen: m^{s a}_r is the
    # smallest d <= t with an anyon on the cone section r - s d a^ + j b^
    # (|j| <= d, inside the lattice) or, for the x fields, the rough column at
    # distance d along -s x^; boundary sites hold nothing
    rng = np.random.default_rng(L)
    for trial in range(12):
        sig = np.where(rng.random((L, L)) < 0.12, -1, 1).astype(np.int8)
        sig[:, 0] = sig[:, L - 1] = 1
        m = np.zeros((4, L, L), np.int32)
        for t in range(1, 6):
            m = oracle.open_substep(sig, m, m_max=255)
            for k in range(4):
                s = 1 if k % 2 == 0 else -1
                ax = k < 2
                for y in range(L):
                    for x in range(L):
                        want = 0
                        if 0 < x < L - 1:
                            for d in range(1, t + 1):
                                hit = False
                                if ax:
                                    xb = x - s * d
                                    if xb in (0, L - 1):
                                        hit = True
                                for j in range(-d, d + 1):
                                    xx, yy = (x - s * d, y + j) if ax else (x + j, y - s * d)
                                    if 0 <= xx < L and 0 <= yy < L and sig[yy, xx] == -1:
                                        hit = True
                                if hit:
                                    want = d
                                    break
                        assert m[k, y, x] == want, (L, trial, t, k, x, y)


def test_open_single_boundary_error_absorbed():
    L = 9
    N = links(L, [(0, 0, 4)])        # e_x(0, 4): one anyon at (1, 4)
    C, steps, flag = oracle.open_decode_shot(N)
    np.testing.assert_array_equal(C, N)
    assert (steps, flag) == (1, 0)
    N = links(L, [(0, L - 2, 2)])    # next to the right boundary
    C, steps, flag = oracle.open_decode_shot(N)
    np.testing.assert_array_equal(C, N)
    assert (steps, flag) == (1, 0)


def test_open_bulk_pair_fuses_in_one_step():
    # e_x(4, 4) on L = 9: anyons at (4, 4) and (5, 4), one link apart and three
    # or more from the rough columns, so each hears its partner first and both
    # mark the link between them, which flips once (the OR of the feedback)
    L = 9
    N = links(L, [(0, 4, 4)])
    C, steps, flag = oracle.open_decode_shot(N)
    np.testing.assert_array_equal(C, N)
    assert (steps, flag) == (1, 0)


def test_open_boundary_to_boundary_string_is_a_logical_error():
    L = 8
    N = links(L, [(0, x, 3) for x in range(L - 1)])
    C, steps, flag = oracle.open_decode_shot(N)
    assert (steps, flag) == (0, 1) and C.sum() == 0


def test_open_anyon_prefers_the_nearer_boundary():
    # chain e_x(1..3, 4): anyons at (1, 4) (one link from the left boundary)
    # and (4, 4); the first goes to the boundary instead of its partner
    # (distance 1 against 3); its partner steps toward where it was.  After
    # the first step the boundary link is flipped, not the link toward the
    # partner
    L = 11
    N = links(L, [(0, 1, 4), (0, 2, 4), (0, 3, 4)])
    C, steps, flag = oracle.open_decode_shot(N, max_steps=1)
    assert (steps, flag) == (1, 2)
    np.testing.assert_array_equal(C, links(L, [(0, 0, 4), (0, 3, 4)]))
    C, steps, flag = oracle.open_decode_shot(N)
    assert flag == 0 and (oracle.open_syndrome(N ^ C) == 1).all()


def test_open_invariants_on_random_noise():
    rng = np.random.default_rng(2)
    for L in (7, 12):
        mask = oracle.open_link_mask(L)
        for p in (0.03, 0.08):
            for _ in range(6):
                N = (rng.random((2, L, L)) < p).astype(np.uint8) & mask
                C, steps, flag = oracle.open_decode_shot(N)
                assert not (C & (1 - mask)).any()          # only existing links
                if flag != 2:
                    assert (oracle.open_syndrome(N ^ C) == 1).all()


# ------------------------------------------------------- desynchronisation

def test_desync_full_rate_unit_speed_is_the_synchronous_decoder():
    # q = 1, v = 1: every site fires every tick, i.e. A^(D) once and the
    # feedback once per tick, which is the synchronous decoder with v = 1
    for L, p in [(8, 0.06), (13, 0.09), (16, 0.04)]:
        N = oracle.sample_errors(L, 25, p, seed=L)
        for i, n in enumerate(N):
            Cd, td, fd = oracle.desync_decode_shot(n, 1.0, v=1, seed=3, shot=i, max_ticks=4096)
            Cs, ts, fs = oracle.decode_shot(n, v=1)
            np.testing.assert_array_equal(Cd, Cs)
            assert (td, fd) == (ts, fs)


def test_desync_first_tick_fusion_rate():
    # one e_x error on the torus: its two anyons are adjacent.  From empty
    # fields, an anyon's only nonzero field after its first message update
    # points at its partner, so in the first tick it steps onto the link
    # between them iff its message update fired (probability min(1, v q)) and
    # its move fired (probability q), two independent draws.  The pair fuses
    # in that tick iff at least one of the two did: 1 - (1 - min(1, v q) q)^2,
    # 0.2256 at v = 3, q = 0.2
    L, v, q, shots = 8, 3, 0.2, 4000
    N = links(L, [(0, 3, 3)])
    fused = 0
    for s in range(shots):
        C, t, f = oracle.desync_decode_shot(N, q, v=v, seed=1, shot=s, max_ticks=1)
        assert t == 1
        if f != 2:
            np.testing.assert_array_equal(C, N)
            fused += 1
    want = 1 - (1 - min(1.0, v * q) * q) ** 2
    sigma = np.sqrt(want * (1 - want) / shots)
    assert abs(fused / shots - want) < 4 * sigma, (fused / shots, want)


def test_desync_no_moves_never_decodes():
    N = oracle.sample_errors(8, 5, 0.1, seed=1)
    for n in N:
        if (oracle.syndrome(n) == -1).any():
            C, t, f = oracle.desync_decode_shot(n, 0.0, max_ticks=40)
            assert (t, f) == (40, 2) and C.sum() == 0


def test_desync_invariants_and_determinism():
    N = oracle.sample_errors(12, 12, 0.05, seed=5)
    for i, n in enumerate(N):
        C, t, f = oracle.desync_decode_shot(n, 0.2, seed=9, shot=i)
        C2, t2, f2 = oracle.desync_decode_shot(n, 0.2, seed=9, shot=i)
        np.testing.assert_array_equal(C, C2)
        assert (t, f) == (t2, f2)
        if f != 2:
            assert (oracle.syndrome(n ^ C) == 1).all()
    # another seed draws other clocks
    ts = [oracle.desync_decode_shot(n, 0.2, seed=10, shot=i)[1] for i, n in enumerate(N)]
    assert ts != [oracle.desync_decode_shot(n, 0.2, seed=9, shot=i)[1] for i, n in enumerate(N)]
