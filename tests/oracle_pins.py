"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees. ``tests/test_oracle_pins.py`` runs them on the oracle;
``tests/test_oracle_mutants.py`` plants plausible mistakes in a copy of the
oracle's C source and checks that at least one pin fails for each.
"""
from __future__ import annotations

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TWO32 = 1 << 32


# --------------------------------------------------------------------------- #
# Philox4x32-10: published known-answer vectors (Random123 / Salmon et al.)    #
# --------------------------------------------------------------------------- #
def load_kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def pin_philox_kat(o):
    for ctr, key, want in load_kat():
        got = [int(x) for x in o.philox(ctr, key)]
        assert got == want, (ctr, key, [hex(g) for g in got], [hex(w) for w in want])


# --------------------------------------------------------------------------- #
# Payoffs, Eq. (1)-(2): hand-worked values and brute-force group membership    #
# --------------------------------------------------------------------------- #
def pattern_lattice(L: int, name: str) -> np.ndarray:
    lat = np.zeros((L, L), dtype=np.uint8)
    if name == "lone_c":
        lat[0, 0] = 1
    elif name == "pair_c":
        lat[0, 0] = 1
        lat[0, 1] = 1
    elif name == "row_c":
        lat[0, :] = 1
    elif name == "all_c":
        lat[:] = 1
    elif name == "all_d":
        pass
    else:
        raise ValueError(name)
    return lat


def load_hand_worked():
    rows = []
    with open(os.path.join(GOLDEN, "payoffs_hand_worked.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            L, r, pat, i, j, S, pay = line.split()
            rows.append((int(L), float(r), pat, int(i), int(j), int(S), float(pay)))
    return rows


def pin_payoff_hand_worked(o):
    for L, r, pat, i, j, S, pay in load_hand_worked():
        lat = pattern_lattice(L, pat)
        s = int(lat[i, j])
        assert o.group_count_total(lat, i, j) == S, (L, pat, i, j)
        assert abs(o.payoff_groups(lat, i, j, r) - pay) < 1e-12, (L, pat, i, j, "groups")
        assert abs(o.payoff_total(s, S, r) - pay) < 1e-12, (L, pat, i, j, "total")


def brute_force_payoffs(lat: np.ndarray, r: float):
    """Payoffs by explicit group membership: build every group G_z (centre z plus
    its four neighbours, as a list with multiplicity), then give each player the
    Eq. (1)-(2) share of every group it is a member of."""
    L = lat.shape[0]
    groups = {}
    for zi in range(L):
        for zj in range(L):
            groups[(zi, zj)] = [(zi, zj), ((zi + 1) % L, zj), ((zi - 1) % L, zj),
                                (zi, (zj + 1) % L), (zi, (zj - 1) % L)]
    pay = np.zeros((L, L))
    tot = np.zeros((L, L), dtype=np.int64)
    for z, members in groups.items():
        nc = sum(int(lat[m]) for m in members)
        for x in set(members):
            s = int(lat[x])
            share = r * nc / 5.0 - (1.0 if s else 0.0)
            pay[x] += share
            tot[x] += nc
    return pay, tot


def pin_payoff_brute_force(o):
    rng = np.random.default_rng(1234)
    for L in (3, 4, 5, 8):
        for trial in range(3):
            lat = (rng.random((L, L)) < 0.5).astype(np.uint8)
            r = float(rng.uniform(1.5, 5.5))
            pay, tot = brute_force_payoffs(lat, r)
            for i in range(L):
                for j in range(L):
                    assert o.group_count_total(lat, i, j) == tot[i, j], (L, i, j)
                    assert abs(o.payoff_groups(lat, i, j, r) - pay[i, j]) < 1e-9, (L, i, j)
                    s = int(lat[i, j])
                    assert abs(o.payoff_total(s, int(tot[i, j]), r) - pay[i, j]) < 1e-9


def pin_payoff_closed_forms(o):
    # all cooperators: every group has N_C = G = 5, payoff 5 (r - 1); all defectors: 0.
    for r in (1.5, 3.74, 4.0, 5.0, 7.25):
        L = 8
        assert abs(o.payoff_groups(pattern_lattice(L, "all_c"), 3, 4, r) - 5 * (r - 1)) < 1e-12
        assert o.payoff_groups(pattern_lattice(L, "all_d"), 3, 4, r) == 0.0
        # the maximum count is G^2 = 25
        assert o.group_count_total(pattern_lattice(L, "all_c"), 0, 0) == 25


# --------------------------------------------------------------------------- #
# Fermi rule, Eq. (3): symmetry, tie, K -> 0 and K -> inf limits, one value    #
# --------------------------------------------------------------------------- #
def pin_fermi_threshold(o):
    # W(D) + W(-D) = 1, so floor(W 2^32) + floor((1-W) 2^32) is 2^32 or 2^32 - 1
    for d in np.linspace(-12.0, 12.0, 97):
        for K in (0.1, 0.5, 2.0):
            t1 = o.threshold(float(d), 0.0, K)
            t2 = o.threshold(0.0, float(d), K)
            assert t1 + t2 in (TWO32 - 1, TWO32), (d, K, t1, t2)
    # tie: W = 1/2 exactly
    for a in (-3.0, 0.0, 1.6, 15.0):
        for K in (0.01, 0.5, 100.0):
            assert o.threshold(a, a, K) == 1 << 31
    # K -> 0: x copies y iff Pi_y > Pi_x (Section III, after Eq. (3))
    K0 = 1e-6
    assert o.threshold(0.0, 0.4, K0) == TWO32 - 1
    assert o.threshold(0.4, 0.0, K0) == 0
    # K -> inf: a coin flip
    t = o.threshold(-7.0, 9.0, 1e12)
    assert abs(t - (1 << 31)) < 1 << 12
    # the better-paid neighbour is imitated with probability above 1/2
    assert o.threshold(1.6, -1.0, 0.5) < 1 << 31 < o.threshold(-1.0, 1.6, 0.5)
    # one value: a defector next to a lone cooperator (payoffs 1.6 and -1.0 at
    # r = 4, hand-worked) with K = 0.5: W = 1 / (1 + e^5.2) = 0.0054863...
    t = o.threshold(1.6, -1.0, 0.5)
    assert abs(t / TWO32 - 0.00548629) < 1e-7, t / TWO32
    # monotone in Pi_y - Pi_x
    ts = [o.threshold(0.0, float(d), 0.5) for d in np.linspace(-5, 5, 41)]
    assert all(b >= a for a, b in zip(ts, ts[1:]))


def pin_adoption_comparator(o):
    # lone cooperator at (0,0); x = (0,1) a defector, y = (0,0) (direction 1: j - 1)
    r, K = 4.0, 0.5
    lat = pattern_lattice(8, "lone_c")
    t = o.threshold(1.6, -1.0, K)
    assert t > 0
    a = lat.copy()
    assert o.elementary_update(a, 0, 1, 1, t - 1, r, K) == 1 and a[0, 1] == 1
    a = lat.copy()
    assert o.elementary_update(a, 0, 1, 1, t, r, K) == 0 and a[0, 1] == 0
    # same strategy: never changes
    a = lat.copy()
    assert o.elementary_update(a, 0, 3, 0, 0, r, K) == 0 and a.sum() == 1
    # the cooperator next to three... direction codes: 0 j+1, 1 j-1, 2 i+1, 3 i-1
    a = pattern_lattice(8, "lone_c")
    assert o.elementary_update(a, 1, 0, 3, 0, r, K) == 1 and a[1, 0] == 1   # y = (0, 0)
    a = pattern_lattice(8, "lone_c")
    assert o.elementary_update(a, 7, 0, 2, 0, r, K) == 1 and a[7, 0] == 1   # y = (0, 0) wrapped
    a = pattern_lattice(8, "lone_c")
    assert o.elementary_update(a, 0, 7, 0, 0, r, K) == 1 and a[0, 7] == 1   # y = (0, 0) wrapped
    a = pattern_lattice(8, "lone_c")
    assert o.elementary_update(a, 0, 1, 0, 0, r, K) == 0                    # y = (0, 2), a D


# --------------------------------------------------------------------------- #
# Dynamics: initial density, absorbing states, schedule coverage, order        #
# --------------------------------------------------------------------------- #
def pin_init_density(o):
    for p in (0.0, 0.2, 0.5, 0.8, 1.0):
        lat = o.init(128, 99, p)
        frac = lat.mean()
        assert abs(frac - p) < 0.01, (p, frac)
    assert o.init(64, 1, 0.5).sum() != o.init(64, 2, 0.5).sum() or \
        not np.array_equal(o.init(64, 1, 0.5), o.init(64, 2, 0.5))


def pin_absorbing_states(o):
    # s_y = s_x everywhere: Eq. (3) is never applied, the lattice never changes
    for name in ("all_c", "all_d"):
        for seed, r, K in ((1, 3.0, 0.5), (7, 5.0, 0.1), (3, 4.2, 10.0)):
            lat = pattern_lattice(16, name)
            ref = lat.copy()
            counts = o.run(lat, r, K, seed, 0, 5)
            assert np.array_equal(lat, ref)
            assert all(int(c) == int(ref.sum()) for c in counts)


def pin_counts_match_lattice(o):
    lat = o.init(32, 5, 0.5)
    counts = o.run(lat, 4.2, 0.5, 5, 0, 3)
    assert int(counts[-1]) == int(lat.sum())
    assert o.count(lat) == int(lat.sum())


def pin_schedule_coverage(o):
    """Every site takes part: with K huge (coin-flip adoption, Section III) the
    sixteen (i mod 4, j mod 4) classes change strategy at equal rates."""
    L = 32
    lat = o.init(L, 17, 0.5)
    changes = np.zeros((L, L))
    for k in range(16 * 24):
        before = lat.copy()
        o.sublattice_step(lat, 4.0, 1e9, 17, k)
        changes += (lat != before)
    per_class = np.array([changes[a::4, b::4].sum() for a in range(4) for b in range(4)])
    mean = per_class.mean()
    assert per_class.min() > 0.6 * mean, per_class
    # and a step changes only sites of one class
    lat2 = o.init(L, 3, 0.5)
    before = lat2.copy()
    o.sublattice_step(lat2, 4.0, 1e9, 3, 5)
    diff = np.argwhere(lat2 != before)
    assert len(diff) > 0
    assert len({(int(i) % 4, int(j) % 4) for i, j in diff}) == 1


def pin_order_independence(o):
    for L, seed in ((16, 2), (40, 9)):
        a = o.init(L, seed, 0.5)
        b = a.copy()
        c = a.copy()
        ca = o.run(a, 3.9, 0.5, seed, 0, 6)
        cb = o.run(b, 3.9, 0.5, seed, 0, 6, reverse=True)
        cc = o.run(c, 3.9, 0.5, seed, 0, 6, threads=3)
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert np.array_equal(ca, cb) and np.array_equal(ca, cc)


def pin_stream_uniformity(o):
    seed = 42
    offs = np.array([o.offset(seed, k) for k in range(16 * 400)])
    hist = np.bincount(offs, minlength=16)
    exp = len(offs) / 16
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 45.0, (chi2, hist)    # 15 dof, p ~ 1e-4
    dirs = np.array([o.dir(seed, 3, a, b) for a in range(8) for b in range(128)])
    hist = np.bincount(dirs, minlength=4)
    chi2 = float(((hist - len(dirs) / 4) ** 2 / (len(dirs) / 4)).sum())
    assert chi2 < 25.0, (chi2, hist)
    us = np.array([o.u(seed, 3, a, b) for a in range(16) for b in range(64)], dtype=np.float64)
    assert abs(us.mean() / TWO32 - 0.5) < 0.03


# --------------------------------------------------------------------------- #
# The random-stream layout                                                      #
# --------------------------------------------------------------------------- #
# The paper names no generator, so the counter layout of the draws is this library's convention
# and no outside value fixes it. These pins write the documented layout out over the Philox
# primitive (itself pinned by the published known-answer vectors), require the oracle's draws to
# follow it, and replay whole sublattice steps from it with brute-force payoffs.
M32 = 0xFFFFFFFF


def _key(seed: int):
    return (seed & M32, (seed >> 32) & M32)


def layout_offset(o, seed: int, k: int) -> int:
    """Offset of step k: call (m_lo, m_hi, 0, tag 2), m = k >> 5; nibble k & 7 of word (k >> 3) & 3."""
    m = k >> 5
    w = o.philox((m & M32, m >> 32, 0, 2 << 24), _key(seed))
    return (int(w[(k >> 3) & 3]) >> (4 * (k & 7))) & 15


def layout_dir(o, seed: int, k: int, a: int, b: int) -> int:
    """Direction of sublattice site (a, b) at step k: call (b >> 6, a, k_lo, k_hi | tag 3);
    2-bit field b & 15 of word (b >> 4) & 3."""
    w = o.philox((b >> 6, a, k & M32, (k >> 32) | (3 << 24)), _key(seed))
    return (int(w[(b >> 4) & 3]) >> (2 * (b & 15))) & 3


def layout_u(o, seed: int, k: int, a: int, b: int) -> int:
    """Adoption draw of sublattice site (a, b) at step k: word b & 3 of call (b >> 2, a, k_lo, k_hi | tag 4)."""
    w = o.philox((b >> 2, a, k & M32, (k >> 32) | (4 << 24)), _key(seed))
    return int(w[b & 3])


def layout_init(o, L: int, seed: int, p: float) -> np.ndarray:
    """Initial state: site x = i L + j is C iff word x & 3 of call (q_lo, q_hi, 0, tag 1),
    q = x >> 2, is below floor(p 2^32) (2^32 for p = 1)."""
    thr = TWO32 if p >= 1.0 else int(math.floor(p * TWO32))
    lat = np.zeros((L, L), dtype=np.uint8)
    for x in range(L * L):
        q = x >> 2
        w = o.philox((q & M32, q >> 32, 0, 1 << 24), _key(seed))
        lat.flat[x] = 1 if int(w[x & 3]) < thr else 0
    return lat


def pin_stream_layout(o):
    rng = np.random.default_rng(2024)
    seeds = [0, 1, 42, (1 << 32) + 5, (1 << 64) - 1] + [int(x) for x in rng.integers(0, 1 << 63, 3)]
    steps = [0, 1, 7, 8, 31, 32, 33, 255, M32, (1 << 32) + 17, (1 << 56) - 1] + \
        [int(x) for x in rng.integers(0, 1 << 56, 4)]
    sites = [(0, 0), (0, 3), (0, 4), (0, 15), (0, 16), (0, 63), (0, 64), (5, 17), (1023, 4095)] + \
        [(int(a), int(b)) for a, b in rng.integers(0, 2048, (6, 2))]
    for seed in seeds:
        for k in steps:
            assert o.offset(seed, k) == layout_offset(o, seed, k), (seed, k)
            for a, b in sites:
                assert o.dir(seed, k, a, b) == layout_dir(o, seed, k, a, b), (seed, k, a, b)
                assert o.u(seed, k, a, b) == layout_u(o, seed, k, a, b), (seed, k, a, b)
    for L, seed, p in ((8, 3, 0.5), (12, (1 << 40) + 1, 0.3), (4, 9, 1.0), (4, 9, 0.0), (16, 77, 0.5)):
        assert np.array_equal(o.init(L, seed, p), layout_init(o, L, seed, p)), (L, seed, p)


def replay_step(o, lat: np.ndarray, r: float, K: float, seed: int, k: int) -> np.ndarray:
    """One group-game sublattice step written out from the stream layout, with payoffs from
    brute_force_payoffs (all sites of a step are independent)."""
    L = lat.shape[0]
    NB = [(0, 1), (0, -1), (1, 0), (-1, 0)]
    pays, _ = brute_force_payoffs(lat, r)
    out = lat.copy()
    off = layout_offset(o, seed, k)
    for a in range(L // 4):
        for b in range(L // 4):
            i, j = 4 * a + (off >> 2), 4 * b + (off & 3)
            d = layout_dir(o, seed, k, a, b)
            yi, yj = (i + NB[d][0]) % L, (j + NB[d][1]) % L
            if lat[i, j] == lat[yi, yj]:
                continue
            t = o.threshold(float(pays[i, j]), float(pays[yi, yj]), K)
            if layout_u(o, seed, k, a, b) < t:
                out[i, j] = lat[yi, yj]
    return out


def pin_step_brute_force(o):
    for L, r, K, seed in ((8, 3.8, 0.5, 5), (12, 4.4, 0.2, 6), (8, 2.9, 1.5, (1 << 33) + 7)):
        lat = layout_init(o, L, seed, 0.5)
        for k in range(24):
            want = replay_step(o, lat, r, K, seed, k)
            o.sublattice_step(lat, r, K, seed, k)
            assert np.array_equal(lat, want), (L, r, k)


# --------------------------------------------------------------------------- #
# Statistical pins against the paper's reported physics (Section V)            #
# --------------------------------------------------------------------------- #
def stationary_density(o, L, r, K, seed, n_mcs, window, classic=False, threads=4):
    lat = o.init(L, seed, 0.5)
    if classic:
        c = o.classic_run(lat, r, K, seed, 0, n_mcs)
    else:
        c = o.run(lat, r, K, seed, 0, n_mcs, threads=threads)
    return float(c[-window:].mean()) / (L * L)


def pin_paper_density_r398(o):
    # Fig. 5 caption: with K = 0.5 and r = 3.98 the stationary fraction of
    # cooperators is 1/2.
    vals = [stationary_density(o, 128, 3.98, 0.5, s, 1200, 400) for s in (21, 22)]
    assert abs(np.mean(vals) - 0.5) < 0.03, vals


def pin_extinction_below_rc(o):
    # Section V: below r_c = 3.7443 the system falls into the absorbing all-D phase.
    for seed in (31, 32):
        rho = stationary_density(o, 64, 3.5, 0.5, seed, 1200, 10)
        assert rho == 0.0, rho
    # above it cooperators survive
    assert stationary_density(o, 64, 4.2, 0.5, 33, 600, 100) > 0.3


def pin_schedules_agree(o):
    # the sublattice schedule and the classic random-sequential one (Section III)
    # give the same stationary density
    for r in (4.5, 5.0):
        sub = np.mean([stationary_density(o, 96, r, 0.5, s, 1000, 400) for s in (41, 42)])
        cla = np.mean([stationary_density(o, 96, r, 0.5, s, 1000, 400, classic=True)
                       for s in (43, 44)])
        assert abs(sub - cla) < 0.03, (r, sub, cla)


def pin_payoff_consistency_during_run(o):
    o.clear_errors()
    lat = o.init(24, 8, 0.5)
    o.run(lat, 4.1, 0.5, 8, 0, 4)
    assert o.errors() == 0


# --------------------------------------------------------------------------- #
# The pairwise game of Section VI (pay = (R, S, T, P))                          #
# --------------------------------------------------------------------------- #
PAIR_MATRICES = [(1.0, 0.0, 1.5, 0.0), (3.0, -1.0, 5.0, 0.5), (1.0, 0.25, 1.75, 0.0),
                 (0.7, -0.3, 1.9, 0.1)]


def load_pair_hand_worked():
    rows = []
    with open(os.path.join(GOLDEN, "pair_payoffs_hand_worked.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            L, R, S, T, Pp, pat, i, j, n, pay = line.split()
            rows.append((int(L), (float(R), float(S), float(T), float(Pp)), pat, int(i), int(j),
                         int(n), float(pay)))
    return rows


def pin_pair_payoff_hand_worked(o):
    for L, pay, pat, i, j, n, want in load_pair_hand_worked():
        lat = pattern_lattice(L, pat)
        s = int(lat[i, j])
        assert o.pair_neighbour_cooperators(lat, i, j) == n, (L, pat, i, j)
        assert abs(o.pair_payoff_games(lat, i, j, pay) - want) < 1e-12, (L, pay, pat, i, j, "games")
        assert abs(o.pair_payoff_total(s, n, pay) - want) < 1e-12, (L, pay, pat, i, j, "total")


def brute_force_pair_payoffs(lat: np.ndarray, pay):
    """Payoffs by enumerating every bond of the torus once (each horizontal bond
    (i, j)-(i, j+1) and each vertical bond (i, j)-(i+1, j)); both ends of a bond
    collect their side of the 2x2 game."""
    R, S, T, Pp = pay
    M = {(1, 1): R, (1, 0): S, (0, 1): T, (0, 0): Pp}
    L = lat.shape[0]
    out = np.zeros((L, L))
    ncoop = np.zeros((L, L), dtype=np.int64)
    for i in range(L):
        for j in range(L):
            for (a, b) in (((i, j), (i, (j + 1) % L)), ((i, j), ((i + 1) % L, j))):
                sa, sb = int(lat[a]), int(lat[b])
                out[a] += M[(sa, sb)]
                out[b] += M[(sb, sa)]
                ncoop[a] += sb
                ncoop[b] += sa
    return out, ncoop


def pin_pair_brute_force(o):
    rng = np.random.default_rng(4321)
    for L in (3, 4, 5, 8):
        for pay in PAIR_MATRICES:
            lat = (rng.random((L, L)) < 0.5).astype(np.uint8)
            want, ncoop = brute_force_pair_payoffs(lat, pay)
            for i in range(L):
                for j in range(L):
                    assert o.pair_neighbour_cooperators(lat, i, j) == ncoop[i, j], (L, i, j)
                    assert abs(o.pair_payoff_games(lat, i, j, pay) - want[i, j]) < 1e-9, (L, pay, i, j)
                    s = int(lat[i, j])
                    assert abs(o.pair_payoff_total(s, int(ncoop[i, j]), pay) - want[i, j]) < 1e-9


def pin_pair_closed_forms(o):
    for pay in PAIR_MATRICES:
        R, S, T, Pp = pay
        assert abs(o.pair_payoff_games(pattern_lattice(8, "all_c"), 2, 6, pay) - 4 * R) < 1e-12
        assert abs(o.pair_payoff_games(pattern_lattice(8, "all_d"), 2, 6, pay) - 4 * Pp) < 1e-12
        for n in range(5):
            assert abs(o.pair_payoff_total(1, n, pay) - (n * R + (4 - n) * S)) < 1e-12
            assert abs(o.pair_payoff_total(0, n, pay) - (n * T + (4 - n) * Pp)) < 1e-12
    assert o.pair_neighbour_cooperators(pattern_lattice(8, "all_c"), 0, 0) == 4


def torus_distance(L, a, b):
    di = abs(a[0] - b[0]) % L
    dj = abs(a[1] - b[1]) % L
    return min(di, L - di) + min(dj, L - dj)


def pin_pair_read_set(o):
    """Section VI: a pairwise update needs one line less in every direction than the
    group game, i.e. the decision for x reads only sites within distance 2 of x
    (x's and y's neighbours); a site at distance 2 (beyond y) does matter."""
    rng = np.random.default_rng(77)
    L, K = 12, 0.5
    pay = (3.0, -1.0, 5.0, 0.5)
    NB = [(0, 1), (0, -1), (1, 0), (-1, 0)]
    checked = far_influence = 0
    for trial in range(12):
        lat = (rng.random((L, L)) < 0.5).astype(np.uint8)
        i, j = int(rng.integers(L)), int(rng.integers(L))
        for d in range(4):
            yi, yj = (i + NB[d][0]) % L, (j + NB[d][1]) % L
            if lat[i, j] == lat[yi, yj]:
                assert o.pair_update_threshold(lat, i, j, d, pay, K) == 0
                continue
            t0 = o.pair_update_threshold(lat, i, j, d, pay, K)
            for zi in range(L):
                for zj in range(L):
                    dist = torus_distance(L, (i, j), (zi, zj))
                    if dist < 2:
                        continue
                    lat[zi, zj] ^= 1
                    t1 = o.pair_update_threshold(lat, i, j, d, pay, K)
                    lat[zi, zj] ^= 1
                    if dist > 2:
                        assert t1 == t0, (trial, i, j, d, zi, zj)
                    elif t1 != t0:
                        far_influence += 1
            checked += 1
    assert checked >= 10 and far_influence > 0, (checked, far_influence)


def replay_pair_step(o, lat: np.ndarray, pay, K: float, seed: int, k: int) -> np.ndarray:
    """One pairwise sublattice step written out from the stream layout, with bond-by-bond
    payoffs from brute_force_pair_payoffs (all sites of a step are independent)."""
    L = lat.shape[0]
    NB = [(0, 1), (0, -1), (1, 0), (-1, 0)]
    pays, _ = brute_force_pair_payoffs(lat, pay)
    out = lat.copy()
    off = layout_offset(o, seed, k)
    for a in range(L // 4):
        for b in range(L // 4):
            i, j = 4 * a + (off >> 2), 4 * b + (off & 3)
            d = layout_dir(o, seed, k, a, b)
            yi, yj = (i + NB[d][0]) % L, (j + NB[d][1]) % L
            if lat[i, j] == lat[yi, yj]:
                continue
            t = o.threshold(float(pays[i, j]), float(pays[yi, yj]), K)
            if layout_u(o, seed, k, a, b) < t:
                out[i, j] = lat[yi, yj]
    return out


def pin_pair_step_brute_force(o):
    for L, pay, K, seed in ((8, (1.0, 0.0, 1.5, 0.0), 0.1, 5), (12, (3.0, -1.0, 5.0, 0.5), 2.0, 6),
                            (8, (0.7, -0.3, 1.9, 0.1), 0.5, 7)):
        lat = o.init(L, seed, 0.5)
        for k in range(24):
            want = replay_pair_step(o, lat, pay, K, seed, k)
            o.pair_sublattice_step(lat, pay, K, seed, k)
            assert np.array_equal(lat, want), (L, pay, k)


def pin_pair_equal_payoffs(o):
    # R = S = T = P: every payoff difference is 0, so every adoption is a fair coin
    # flip (W = 1/2 exactly, Eq. (3))
    rng = np.random.default_rng(5)
    for c in (0.0, 2.0, -1.5):
        pay = (c, c, c, c)
        lat = (rng.random((8, 8)) < 0.5).astype(np.uint8)
        for i in range(8):
            for j in range(8):
                for d in range(4):
                    t = o.pair_update_threshold(lat, i, j, d, pay, 0.3)
                    yi, yj = (i + (0, 0, 1, -1)[d]) % 8, (j + (1, -1, 0, 0)[d]) % 8
                    assert t == (0 if lat[i, j] == lat[yi, yj] else 1 << 31)


def pin_pair_absorbing_and_order(o):
    for name in ("all_c", "all_d"):
        lat = pattern_lattice(16, name)
        ref = lat.copy()
        counts = o.pair_run(lat, (1.0, 0.0, 1.5, 0.0), 0.1, 3, 0, 4)
        assert np.array_equal(lat, ref) and all(int(c) == int(ref.sum()) for c in counts)
    for L, seed in ((16, 2), (28, 9)):
        a = o.init(L, seed, 0.5)
        b, c = a.copy(), a.copy()
        pay = (1.0, 0.5, 1.5, 0.0)
        ca = o.pair_run(a, pay, 0.5, seed, 0, 5)
        cb = o.pair_run(b, pay, 0.5, seed, 0, 5, reverse=True)
        cc = o.pair_run(c, pay, 0.5, seed, 0, 5, threads=3)
        assert np.array_equal(a, b) and np.array_equal(a, c)
        assert np.array_equal(ca, cb) and np.array_equal(ca, cc)
        assert int(ca[-1]) == int(a.sum())


def pin_pair_payoff_consistency_during_run(o):
    o.clear_errors()
    lat = o.init(24, 8, 0.5)
    o.pair_run(lat, (0.7, -0.3, 1.9, 0.1), 0.5, 8, 0, 4)
    assert o.errors() == 0


def pin_pair_schedules_agree(o):
    # the sublattice schedule and the classic random-sequential one give the same
    # stationary density for the pairwise game as well (snowdrift matrix: both
    # strategies coexist robustly)
    pay, K, L = (1.0, 0.5, 1.5, 0.0), 0.5, 96
    sub, cla = [], []
    for s in (51, 52):
        lat = o.init(L, s, 0.5)
        sub.append(float(o.pair_run(lat, pay, K, s, 0, 800, threads=4)[-400:].mean()) / (L * L))
        lat = o.init(L, s + 10, 0.5)
        cla.append(float(o.pair_classic_run(lat, pay, K, s + 10, 0, 800)[-400:].mean()) / (L * L))
    assert abs(np.mean(sub) - np.mean(cla)) < 0.02, (sub, cla)
    assert 0.2 < np.mean(sub) < 0.6, sub


FAST_PINS = [pin_philox_kat, pin_payoff_hand_worked, pin_payoff_brute_force,
             pin_payoff_closed_forms, pin_fermi_threshold, pin_adoption_comparator,
             pin_init_density, pin_absorbing_states, pin_counts_match_lattice,
             pin_schedule_coverage, pin_order_independence, pin_stream_uniformity,
             pin_stream_layout, pin_step_brute_force,
             pin_payoff_consistency_during_run, pin_pair_payoff_hand_worked, pin_pair_brute_force,
             pin_pair_closed_forms, pin_pair_read_set, pin_pair_step_brute_force,
             pin_pair_equal_payoffs, pin_pair_absorbing_and_order,
             pin_pair_payoff_consistency_during_run]
SLOW_PINS = [pin_paper_density_r398, pin_extinction_below_rc, pin_schedules_agree,
             pin_pair_schedules_agree]
