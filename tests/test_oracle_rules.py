"""Pins of the oracle against what the paper and the mathematics fix.

Each test names what fixes its expected value: the paper's printed W^2(L,0),
closed forms of deterministic parameter corners, invariants of height
functions (periodicity, zero curl, parity), library routines (numpy, scipy,
Python's Fraction) or binomial statistics.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _heights_y_first(X, Y, H0):
    """Heights along the other path: down column 0 first, then along each row."""
    sx = 2 * X.astype(np.int64) - 1
    sy = 2 * Y.astype(np.int64) - 1
    L = X.shape[0]
    col0 = H0 + np.concatenate([[0], np.cumsum(sy[:-1, 0])])
    h = np.zeros((L, L), np.int64)
    h[:, 0] = col0
    h[:, 1:] = col0[:, None] + np.cumsum(sx[:, :-1], axis=1)
    return h


def _check_invariants(sim):
    X, Y, L = sim.X, sim.Y, sim.L
    sx = 2 * X.astype(np.int64) - 1
    sy = 2 * Y.astype(np.int64) - 1
    # periodic heights: every row of sigma_x and every column of sigma_y sums to 0
    assert np.all(sx.sum(axis=1) == 0)
    assert np.all(sy.sum(axis=0) == 0)
    # zero curl on every plaquette: sx(x,y) + sy(x+1,y) == sy(x,y) + sx(x,y+1)
    assert np.array_equal(sx + np.roll(sy, -1, axis=1), sy + np.roll(sx, -1, axis=0))
    # half of the bonds of each plane point up
    assert int(X.sum()) == L * L // 2 and int(Y.sum()) == L * L // 2
    h = sim.heights()
    # the two summation paths of Eq. (3) agree
    assert np.array_equal(h, _heights_y_first(X, Y, sim.H0))
    # height parity is conserved: h == x + y (mod 2)
    yy, xx = np.mgrid[0:L, 0:L]
    assert np.all((h - xx - yy) % 2 == 0)
    return h


@pytest.mark.parametrize("p,q,s_sel,k_max,want", [
    (1.0, 0.0, 0.5, 32, (1, 1, 0)),
    (1.0, 0.0, 1.0, 32, (0, 1, 0)),
    (0.0, 0.0, 0.5, 32, (0, 0, 0)),
    (0.75, 0.25, 0.5, 32, (3, 3, 1)),
    (0.5, 0.5, 0.5, 32, (2, 1, 1)),
    (0.5, 0.5, 1.0, 32, (1, 1, 1)),
])
def test_thresholds_dyadic(orc, p, q, s_sel, k_max, want):
    assert orc.thresholds(p, q, s_sel, k_max) == want


@pytest.mark.parametrize("p,q,s_sel,k_max", [
    (0.95, 0.05, 0.5, 32), (0.9, 0.1, 1.0, 32), (0.3, 0.7, 0.5, 12), (1 / 3, 0.0, 1.0, 7)])
def test_thresholds_rounded(orc, p, q, s_sel, k_max):
    """Non-dyadic probabilities: k = k_max, P = round-half-even(p_eff * 2^k), done
    here with exact rationals (Fraction) and Python's round."""
    k, P, Q = orc.thresholds(p, q, s_sel, k_max)
    pe = Fraction(s_sel * p)  # the double product, exactly
    qe = Fraction(s_sel * q)
    assert k == k_max
    assert P == round(pe * 2**k_max) and Q == round(qe * 2**k_max)


def test_thresholds_reject_out_of_range(orc):
    for args in [(1.5, 0, 0.5, 32), (-0.1, 0, 0.5, 32), (1, 0, 0.0, 32), (1, 0, 0.5, 33)]:
        with pytest.raises(ValueError):
            orc.thresholds(*args)


def test_flat_start_width_is_one_quarter(orc):
    """Sec. III: the striped start has W^2(L,0) = 1/4 (golden fixture)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "flat_start.txt"))
            if l.strip() and not l.startswith("#")]
    for L, w2 in rows:
        sim = orc.Sim(int(L), 1.0, 0.0, 1)
        assert sim.width2() == float(w2)
        h = sim.heights()
        yy, xx = np.mgrid[0:int(L), 0:int(L)]
        assert np.array_equal(h, (xx + yy) % 2)


@pytest.mark.parametrize("L,p,q,s_sel,seed", [
    (32, 1.0, 0.0, 0.5, 1), (30, 0.75, 0.25, 0.5, 2), (64, 0.95, 0.05, 0.5, 3),
    (16, 0.5, 0.5, 1.0, 4), (48, 0.3, 0.6, 0.8, 5)])
def test_invariants_and_local_changes(orc, L, p, q, s_sel, seed):
    sim = orc.Sim(L, p, q, seed, s_sel=s_sel)
    h = _check_invariants(sim)
    yy, xx = np.mgrid[0:L, 0:L]
    for _ in range(25):
        for s in (0, 1):
            before = h
            hb = np.pad(before, 1, mode="wrap")
            nbrs = np.stack([hb[1:-1, :-2], hb[1:-1, 2:], hb[:-2, 1:-1], hb[2:, 1:-1]])
            is_min = np.all(nbrs == before + 1, axis=0)
            is_max = np.all(nbrs == before - 1, axis=0)
            sim.halfsweep(s)
            h = _check_invariants(sim)
            d = h - before
            # only active sites change; minima by +2, maxima by -2
            assert np.all(d[(xx + yy) % 2 != s] == 0)
            assert np.all(np.isin(d, (-2, 0, 2)))
            assert np.all(is_min[d == 2]) and np.all(is_max[d == -2])
        sim.t += 1


def test_closed_form_deterministic_growth(orc):
    """s_sel = 1, p = 1, q = 0: every minimum rises each half-sweep, so the
    surface moves up by 2 per sweep: S1 = N/2 + 2Nt and W^2 = 1/4 for all t."""
    L = 32
    N = L * L
    sim = orc.Sim(L, 1.0, 0.0, 5, s_sel=1.0)
    for t in range(1, 12):
        sim.sweep(1)
        S1, _ = sim.sums()
        assert S1 == N // 2 + 2 * N * t
        assert sim.width2() == 0.25


def test_closed_form_deterministic_etching(orc):
    """s_sel = 1, p = 0, q = 1: half-sweep 0 of sweep 1 finds only minima and
    does nothing; from then on every maximum drops, so after t >= 1 sweeps even
    sites sit at -2(t-1) and odd sites at 1 - 2t: S1 = 3N/2 - 2Nt, W^2 = 1/4."""
    L = 16
    N = L * L
    sim = orc.Sim(L, 0.0, 1.0, 9, s_sel=1.0)
    for t in range(1, 10):
        sim.sweep(1)
        S1, _ = sim.sums()
        assert S1 == 3 * N // 2 - 2 * N * t
        assert sim.width2() == 0.25


def test_closed_form_frozen(orc):
    """p = q = 0: nothing ever changes."""
    sim = orc.Sim(32, 0.0, 0.0, 3)
    X0, Y0 = sim.X.copy(), sim.Y.copy()
    sim.sweep(5)
    assert np.array_equal(sim.X, X0) and np.array_equal(sim.Y, Y0) and sim.H0 == 0


def test_order_independence(orc):
    """Sites of one sublattice share no bond: any visiting order gives the same state."""
    rng = np.random.default_rng(0)
    a = orc.Sim(24, 0.75, 0.25, 11)
    a.sweep(7)
    for s in (0, 1):
        b = orc.Sim(24, 0.75, 0.25, 11)
        b.X, b.Y, b.H0, b.t = a.X.copy(), a.Y.copy(), a.H0, a.t
        active = np.array([y * 24 + x for y in range(24) for x in range(24)
                           if (x + y) % 2 == s], np.int64)
        order = rng.permutation(active)
        import ctypes
        H0 = ctypes.c_int64(b.H0)
        assert orc.lib().orc_halfsweep_ordered(b.L, b.X, b.Y, ctypes.byref(H0), b.seed,
                                               b.t, s, b.k, b.P, b.Q, order,
                                               len(order)) == 0
        a.halfsweep(s)
        assert np.array_equal(a.X, b.X) and np.array_equal(a.Y, b.Y) and a.H0 == H0.value


@pytest.mark.parametrize("p,q,s_sel", [(0.75, 0.25, 0.5), (0.95, 0.05, 0.5), (1.0, 0.0, 0.5)])
def test_acceptance_rates(orc, p, q, s_sel):
    """Fractions of active minima (maxima) that move match s_sel*p (s_sel*q)
    within 5 binomial standard deviations."""
    L = 128
    sim = orc.Sim(L, p, q, 21, s_sel=s_sel)
    sim.sweep(20)
    nmin = nmin_acc = nmax = nmax_acc = 0
    yy, xx = np.mgrid[0:L, 0:L]
    for _ in range(30):
        for s in (0, 1):
            h = sim.heights()
            hb = np.pad(h, 1, mode="wrap")
            nbrs = np.stack([hb[1:-1, :-2], hb[1:-1, 2:], hb[:-2, 1:-1], hb[2:, 1:-1]])
            act = (xx + yy) % 2 == s
            is_min = np.all(nbrs == h + 1, axis=0) & act
            is_max = np.all(nbrs == h - 1, axis=0) & act
            sim.halfsweep(s)
            d = sim.heights() - h
            nmin += int(is_min.sum())
            nmin_acc += int((d[is_min] == 2).sum())
            nmax += int(is_max.sum())
            nmax_acc += int((d[is_max] == -2).sum())
        sim.t += 1
    for n, a, pr in [(nmin, nmin_acc, s_sel * p), (nmax, nmax_acc, s_sel * q)]:
        if pr in (0.0, 1.0):
            assert a == (n if pr == 1.0 else 0)
        else:
            assert n > 1000
            assert abs(a - n * pr) < 5 * np.sqrt(n * pr * (1 - pr))


def test_width_and_moments_match_numpy_scipy(orc):
    from scipy import stats
    sim = orc.Sim(64, 0.75, 0.25, 4)
    sim.sweep(40)
    h = sim.heights().astype(np.float64)
    assert sim.width2() == pytest.approx(np.var(h), rel=1e-12)
    sk, ku = sim.skew_kurt()
    assert sk == pytest.approx(stats.skew(h, axis=None), rel=1e-9, abs=1e-12)
    assert ku == pytest.approx(stats.kurtosis(h, axis=None), rel=1e-9, abs=1e-12)
    S = sim.power_sums()
    d = sim.heights() - sim.H0
    assert S == [int((d.astype(object) ** n).sum()) for n in range(1, 5)]


def test_sums_are_exact_beyond_int64(orc):
    """A surface raised by ~2^30 keeps exact 128-bit sums (S2 ~ 2^72)."""
    sim = orc.Sim(64, 1.0, 0.0, 1)
    sim.sweep(3)
    h = sim.heights()
    sim.H0 += 2 ** 31  # shift the whole surface (heights are anchored at H0)
    S1, S2 = sim.sums()
    hh = (h + 2 ** 31).astype(object)
    assert S1 == int(hh.sum()) and S2 == int((hh * hh).sum())
    assert sim.width2() == pytest.approx(np.var(h.astype(np.float64)), rel=1e-12)


def test_sample_times(orc):
    for T, n in [(1000, 20), (10000, 40), (8192, 40), (50, 40)]:
        ts = orc.sample_times(T, n)
        assert ts[0] == 0 and ts[-1] == T and len(ts) == n + 1
        assert all(b > a for a, b in zip(ts, ts[1:]))
        # away from the forced +1 steps the times follow T^(j/(n-1))
        for j in range(n):
            v = round(T ** (j / (n - 1)))
            assert ts[j + 1] >= v
            if v > n:
                assert ts[j + 1] == v
    with pytest.raises(ValueError):
        orc.sample_times(10, 40)


def test_random_sequential_variant(orc):
    """The random-sequential dynamics keeps the height-function invariants, and
    with p = 1, q = 0 every accepted move raises a minimum by 2."""
    sim = orc.Sim(32, 1.0, 0.0, 8)
    for _ in range(10):
        S1_before, _ = sim.sums()
        sim.rs_sweep(1)
        _check_invariants(sim)
        S1, _ = sim.sums()
        assert S1 > S1_before and (S1 - S1_before) % 2 == 0
    sim = orc.Sim(32, 0.5, 0.5, 8)
    sim.rs_sweep(20)
    _check_invariants(sim)


def _p32(p):
    """round-half-even(p * 2^32) from the exact rational value of the double p."""
    return round(Fraction(p) * 2 ** 32)


@pytest.mark.parametrize("p", [0.0, 1.0, 0.5, 0.75, 0.25, 2.0 ** -32,  # dyadic
                               0.1, 0.95, 0.05, 1.0 / 3.0, 0.3141592653589793,  # rounded
                               2.0 ** -33, 3 * 2.0 ** -33, 5 * 2.0 ** -33,  # exactly half-way
                               1.0 - 2.0 ** -33, 0.5 + 2.0 ** -33])
def test_rs_threshold_rounds_half_to_even(orc, p):
    """The 32-bit threshold of the random-sequential rule is p * 2^32 rounded to
    the nearest integer, ties to even (2^-33 -> 0, 3*2^-33 -> 2, 5*2^-33 -> 2),
    against Python's exact Fraction arithmetic."""
    want = _p32(p)
    assert orc.rs_threshold(p) == want
    if p == 5 * 2.0 ** -33:
        assert want == 2
    if p == 3 * 2.0 ** -33:
        assert want == 2


def _rs_by_hand(orc, h, L, p, q, seed, t):
    """One random-sequential sweep on a height array, written from the rule:
    attempt a = 0 .. L*L-1 in order draws Philox4x32-10 at counter
    (a mod 2^32, a div 2^32, t, 256), picks x = floor(r0 * L / 2^32),
    y = floor(r1 * L / 2^32), and moves a minimum up (maximum down) by 2 when
    r2 is below the 32-bit threshold of p (of q)."""
    P32, Q32 = _p32(p), _p32(q)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    sites = []
    for a in range(L * L):
        r = orc.philox4x32_10([a & 0xFFFFFFFF, a >> 32, t, 256], key)
        x, y = (int(r[0]) * L) >> 32, (int(r[1]) * L) >> 32
        sites.append((x, y))
        nb = [h[y, (x - 1) % L], h[y, (x + 1) % L], h[(y - 1) % L, x], h[(y + 1) % L, x]]
        if all(v == h[y, x] + 1 for v in nb) and int(r[2]) < P32:
            h[y, x] += 2
        elif all(v == h[y, x] - 1 for v in nb) and int(r[2]) < Q32:
            h[y, x] -= 2
    return h, sites


@pytest.mark.parametrize("L,p,q,seed", [(2, 1.0, 1.0, 17), (4, 1.0, 0.0, 3), (6, 0.75, 0.25, 4),
                                         (8, 0.5, 0.5, 5), (10, 1.0, 1.0, 6)])
def test_random_sequential_sweep_by_hand(orc, L, p, q, seed):
    """orc_rs_sweeps equals the rule applied attempt by attempt to a height
    array in Python (site decode by multiply-high, strict threshold compare),
    over three sweeps, for power-of-two and other even L (on the 2 x 2 torus
    every site starts as an extremum, so with p = q = 1 the first attempt
    always moves its decoded site); the picked sites stay in [0, L)."""
    sim = orc.Sim(L, p, q, seed)
    h = sim.heights()
    for t in range(3):
        sim.rs_sweep(1)
        h, sites = _rs_by_hand(orc, h, L, p, q, seed, t)
        assert np.array_equal(sim.heights(), h), (L, t)
        xs, ys = zip(*sites)
        assert min(xs) >= 0 and max(xs) < L and min(ys) >= 0 and max(ys) < L


def test_domain_decomposed_random_sequential(orc):
    """The blocked random-sequential dynamics keeps every height-function
    invariant; every move changes a height by 2, and with p = 1, q = 0 the
    surface only rises."""
    sim = orc.Sim(64, 1.0, 0.0, 12)
    for _ in range(6):
        before, _ = sim.sums()
        sim.ddrs_sweep(1)
        _check_invariants(sim)
        after, _ = sim.sums()
        assert after > before and (after - before) % 2 == 0
    sim = orc.Sim(96, 0.5, 0.5, 13)
    sim.ddrs_sweep(10)
    _check_invariants(sim)
    with pytest.raises(ValueError):
        orc.Sim(96, 1.0, 0.0, 1).ddrs_sweep(1, C=64)  # 64 does not divide 96


def _ddrs_by_hand(orc, h, L, C, p, q, seed, t, cell_order):
    """One blocked random-sequential sweep on a height array, written from
    the definition: random origin, C x C cells, C*C attempts per cell from
    the cell's own Philox stream, first column and first row dead."""
    P32, Q32 = orc.rs_threshold(p), orc.rs_threshold(q)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    o = orc.philox4x32_10([0, 0, t, 768], key)
    ox, oy = int(o[0]) % C, int(o[1]) % C
    n = L // C
    for c in cell_order:
        x0, y0 = (ox + (c % n) * C) % L, (oy + (c // n) * C) % L
        for a in range(C * C):
            r = orc.philox4x32_10([c, a // 2, t, 1024], key)
            first, u = (int(r[0]), int(r[1])) if a % 2 == 0 else (int(r[2]), int(r[3]))
            lx, ly = first % C, (first >> 16) % C
            if lx == 0 or ly == 0:
                continue
            x, y = (x0 + lx) % L, (y0 + ly) % L
            nb = [h[y, (x - 1) % L], h[y, (x + 1) % L], h[(y - 1) % L, x], h[(y + 1) % L, x]]
            if all(v == h[y, x] + 1 for v in nb) and u < P32:
                h[y, x] += 2
            elif all(v == h[y, x] - 1 for v in nb) and u < Q32:
                h[y, x] -= 2
    return h


def test_domain_decomposed_cells_are_independent(orc):
    """The oracle's blocked sweep equals the definition applied to heights by
    hand, with the cells taken in reverse order (they share no flipped bond),
    for one cell covering the lattice and for 2 x 2 cells."""
    for L, C, seed in [(16, 16, 5), (32, 16, 6), (32, 8, 9)]:
        sim = orc.Sim(L, 0.75, 0.25, seed)
        h = orc.Sim(L, 0.75, 0.25, seed).heights()
        for t in range(3):
            sim.ddrs_sweep(1, C=C)
            h = _ddrs_by_hand(orc, h, L, C, 0.75, 0.25, seed, t,
                              reversed(range((L // C) ** 2)))
            assert np.array_equal(sim.heights(), h), (L, C, t)


@pytest.mark.parametrize("L,p,q,s_sel,n", [(64, 1.0, 0.0, 0.5, 6), (96, 0.75, 0.25, 0.5, 5),
                                           (64, 1.0, 1.0, 0.5, 7), (128, 0.95, 0.05, 0.5, 4)])
def test_window_mode_matches_full_lattice(orc, L, p, q, s_sel, n):
    """The light-cone window simulation (used to check the largest lattices
    site by site) reproduces the full-lattice oracle on every site farther
    than 2n + 1 from the window's edges, for windows inside the lattice,
    across the periodic wrap in x, in y and at the corner, and one covering
    more than the whole lattice; sites near the window edges are allowed to
    differ (and do, somewhere, for the last one)."""
    ref = orc.Sim(L, p, q, 23, s_sel=s_sel)
    ref.sweep(n)
    m = 2 * n + 2
    for (x0, y0, w, h) in [(5, 9, 2 * m + 20, 2 * m + 11), (L - m - 3, 17, 2 * m + 9, 2 * m + 4),
                           (3, L - m - 6, 2 * m + 8, 2 * m + 12),
                           (L - m - 2, L - m - 5, 2 * m + 7, 2 * m + 10),
                           (L - 7, L - 3, L + 2 * m, L + 2 * m)]:
        WX, WY = orc.window_flat_sweeps(L, x0, y0, w, h, p, q, 23, n, s_sel=s_sel)
        ys = (np.arange(h) + y0) % L
        xs = (np.arange(w) + x0) % L
        RX = ref.X[np.ix_(ys, xs)]
        RY = ref.Y[np.ix_(ys, xs)]
        assert np.array_equal(WX[m:h - m, m:w - m], RX[m:h - m, m:w - m]), (x0, y0)
        assert np.array_equal(WY[m:h - m, m:w - m], RY[m:h - m, m:w - m]), (x0, y0)
    # the frozen edges of the window are not the lattice's (the margin matters)
    assert not (np.array_equal(WX, RX) and np.array_equal(WY, RY))
