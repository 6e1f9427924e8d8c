"""Pins of the pricing step (Section 2.2.2): best opening per MLC row, CP
price, best CP, and the leaf-travel windows (Eq. 2 compatibility reading)."""
import itertools

import numpy as np
import pytest

import oracle
import synth


def window_prefix(row, lo, hi):
    """Running float64 sum over the columns lo .. hi - 1 only, by an explicit loop."""
    P = [0.0]
    for c, p in enumerate(row):
        P.append(P[-1] + float(p) if lo <= c < hi else P[-1])
    return P


def brute_best_opening(row, Lmin, Lmax, Rmin, Rmax):
    """All feasible [L, R) by explicit loops; key (v desc, width, centredness, L)."""
    N = len(row)
    P = window_prefix(row, Lmin, Rmax)
    best = None
    for L in range(N + 1):
        for R in range(L, N + 1):
            if not (Lmin <= L <= Lmax and Rmin <= R <= Rmax):
                continue
            key = (-(P[R] - P[L]), R - L, abs(L + R - N), L)
            if best is None or key < best[0]:
                best = (key, P[R] - P[L], L, R)
    if best is None:
        return None, -1, -1
    return best[1], best[2], best[3]


def test_worked_row():
    # [1, 3) collects 2 + 3 = 5; [4, 5) gives 4; [1, 5) gives 4
    assert oracle.best_opening(np.float32([-1, 2, 3, -5, 4]), 0, 5, 0, 5) == (5.0, 1, 3)


def test_all_negative_row_closes_centred():
    v, L, R = oracle.best_opening(np.float32([-1, -2, -3, -4, -5]), 0, 5, 0, 5)
    assert (v, L, R) == (0.0, 2, 2)
    assert oracle.best_opening(np.zeros(4, np.float32), 0, 4, 0, 4) == (0.0, 2, 2)


def test_equal_value_prefers_narrow():
    # [0, 1) = 2 and [0, 3) = 2: the narrower wins
    assert oracle.best_opening(np.float32([2, -1, 1]), 0, 3, 0, 3) == (2.0, 0, 1)


def test_windows_can_force_negative_row():
    # L forced to 0 and R forced to >= 2 around a negative region
    v, L, R = oracle.best_opening(np.float32([-1, -1, 3, -1]), 0, 0, 2, 4)
    assert (L, R) == (0, 3) and v == 1.0


def test_prefix_sum_is_sequential():
    rng = np.random.default_rng(1)
    row = rng.normal(size=97).astype(np.float32) * np.float32(1e3)
    P = oracle.prefix_sums(row)
    acc = 0.0
    for c, p in enumerate(row):
        acc = acc + float(p)
        assert P[c + 1] == acc  # bitwise: same order of float64 additions


@pytest.mark.parametrize("lo,hi", [(0, 97), (13, 60), (40, 41), (50, 50), (70, 20), (96, 97)])
def test_window_prefix_sum(lo, hi):
    """Zero up to the window, sequential inside it, constant after it; nothing
    outside the window is read (NaN there changes nothing)."""
    rng = np.random.default_rng(2)
    row = (rng.normal(size=97) * 10.0 ** rng.integers(-6, 6, size=97)).astype(np.float32)
    P = oracle.prefix_sums(row, lo, hi)
    assert list(P) == window_prefix(row, lo, hi)
    assert np.all(P[:lo + 1] == 0.0)
    if hi > lo:
        assert np.all(P[hi:] == P[hi])
    poisoned = row.copy()
    poisoned[:lo] = np.nan
    poisoned[max(hi, lo):] = np.nan
    assert np.array_equal(oracle.prefix_sums(poisoned, lo, hi), P)


@pytest.mark.parametrize("seed", range(4))
def test_prices_outside_the_window_never_matter(seed):
    """A row's choice, and a CP's aperture with neighbours placed, are unchanged
    when every price outside the leaf-travel windows is replaced by NaN."""
    rng = np.random.default_rng(10 + seed)
    N = 16
    for _ in range(30):
        row = (rng.normal(size=N) * 10.0 ** rng.integers(-7, 7, size=N)).astype(np.float32)
        a, b = sorted(rng.integers(0, N + 1, 2))
        c, d = sorted(rng.integers(0, N + 1, 2))
        got = oracle.best_opening(row, a, b, c, d)
        poisoned = row.copy()
        poisoned[:a] = np.nan
        poisoned[max(d, a):] = np.nan
        assert oracle.best_opening(poisoned, a, b, c, d) == got
    mlc = synth.MLC(9, 4, 12, np.array([0], np.int32), 2)
    mlc_id = synth.MLC(9, 4, 12, np.array([0], np.int32), 2, interdigitation=True)
    pi = (rng.normal(size=mlc.K * 4 * 12) * 10.0 ** rng.integers(-5, 5, size=mlc.K * 4 * 12)).astype(np.float32)
    occupied = np.zeros(mlc.K, bool)
    leaves = np.zeros((mlc.K, 4, 2), np.int64)
    for k in (2, 6):
        occupied[k] = True
        Ls = rng.integers(0, 9, size=4)
        leaves[k] = np.stack([Ls, Ls + rng.integers(0, 4, size=4)], axis=1)
    for k in range(mlc.K):
        if occupied[k]:
            continue
        Lmin, _, _, Rmax = oracle.leaf_windows(mlc, occupied, leaves, k)
        poisoned = pi.copy()
        for r in range(4):
            seg = poisoned[(k * 4 + r) * 12:(k * 4 + r + 1) * 12]
            seg[:Lmin[r]] = np.nan
            seg[max(Rmax[r], Lmin[r]):] = np.nan
        for m, price_cp in ((mlc, oracle.price_cp), (mlc_id, oracle.price_cp_interdig)):
            p0, l0 = price_cp(m, pi, occupied, leaves, k)
            p1, l1 = price_cp(m, poisoned, occupied, leaves, k)
            assert p0 == p1 and ((l0 is None and l1 is None) or np.array_equal(l0, l1))


@pytest.mark.parametrize("seed", range(6))
def test_best_opening_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(1, 13))
    for _ in range(40):
        row = rng.integers(-3, 4, size=N).astype(np.float32)   # small integers: many ties
        if rng.random() < 0.5:
            a, b = sorted(rng.integers(0, N + 1, 2))
            c, d = sorted(rng.integers(0, N + 1, 2))
        else:
            a, b, c, d = 0, N, 0, N
        got = oracle.best_opening(row, a, b, c, d)
        want = brute_best_opening(row, a, b, c, d)
        assert got == want


def tiny_mlc(K=6, n_rows=3, n_cols=4, arcs=(0,), travel=1):
    return synth.MLC(K, n_rows, n_cols, np.array(arcs, np.int32), travel)


def test_cp_price_is_best_over_all_aperture_combinations():
    mlc = tiny_mlc()
    rng = np.random.default_rng(7)
    pi = rng.integers(-4, 5, size=mlc.K * mlc.n_rows * mlc.n_cols).astype(np.float32)
    occupied = np.zeros(mlc.K, bool)
    leaves = np.zeros((mlc.K, mlc.n_rows, 2), np.int64)
    N = mlc.n_cols
    openings = [(L, R) for L in range(N + 1) for R in range(L, N + 1)]
    for k in range(mlc.K):
        price, lv = oracle.price_cp(mlc, pi, occupied, leaves, k)
        best = -np.inf
        for combo in itertools.product(openings, repeat=mlc.n_rows):
            tot = 0.0
            for r, (L, R) in enumerate(combo):
                base = (k * mlc.n_rows + r) * N
                tot += float(np.sum(pi[base + L: base + R].astype(np.float64)))
            best = max(best, tot)
        assert price == best
        tot = sum(float(np.sum(pi[(k * mlc.n_rows + r) * N + L:(k * mlc.n_rows + r) * N + R].astype(np.float64)))
                  for r, (L, R) in enumerate(lv))
        assert tot == price


def test_leaf_windows_reading():
    mlc = tiny_mlc(K=6, n_rows=2, n_cols=8, travel=1)
    occupied = np.zeros(6, bool)
    leaves = np.zeros((6, 2, 2), np.int64)
    occupied[1] = True
    leaves[1] = [[2, 5], [0, 8]]
    Lmin, Lmax, Rmin, Rmax = oracle.leaf_windows(mlc, occupied, leaves, 3)   # distance 2
    assert list(Lmin) == [0, 0] and list(Lmax) == [4, 2]
    assert list(Rmin) == [3, 6] and list(Rmax) == [7, 8]
    occupied[4] = True
    leaves[4] = [[3, 4], [1, 2]]
    Lmin, Lmax, Rmin, Rmax = oracle.leaf_windows(mlc, occupied, leaves, 3)   # plus distance 1 on the right
    assert list(Lmin) == [2, 0] and list(Lmax) == [4, 2]
    assert list(Rmin) == [3, 6] and list(Rmax) == [5, 3]


def test_windows_stop_at_arc_boundary():
    mlc = tiny_mlc(K=6, n_rows=1, n_cols=8, arcs=(0, 3), travel=1)
    occupied = np.zeros(6, bool)
    leaves = np.zeros((6, 1, 2), np.int64)
    occupied[2] = True
    leaves[2] = [[4, 4]]
    assert [int(a[0]) for a in oracle.leaf_windows(mlc, occupied, leaves, 3)] == [0, 8, 0, 8]
    assert [int(a[0]) for a in oracle.leaf_windows(mlc, occupied, leaves, 1)] == [3, 5, 3, 5]


def test_best_cp_ties_pick_smallest_index():
    mlc = tiny_mlc(K=4, n_rows=1, n_cols=3)
    pi = np.float32([1, 1, 0,  0, 2, 0,  2, 0, 0,  0, 0, 0])
    occupied = np.zeros(4, bool)
    leaves = np.zeros((4, 1, 2), np.int64)
    k, lv, price = oracle.price_apertures(mlc, pi, occupied, leaves)
    assert (k, price) == (0, 2.0) and list(lv[0]) == [0, 2]
    occupied[0] = True
    leaves[0] = [[0, 2]]
    k, lv, price = oracle.price_apertures(mlc, pi, occupied, leaves)
    # CP 1 (distance 1, travel 1): L in [0, 1], R in [1, 3] -> [1, 2) = 2; CP 2: [0, 1) = 2
    assert (k, price) == (1, 2.0) and list(lv[0]) == [1, 2]


# ---------------------------------------------------------------------------- interdigitation (reading R10)

def _interdig_ok(lv):
    """L_r <= min(R_{r-1}, R_{r+1}) for every row."""
    for r in range(len(lv)):
        for q in (r - 1, r + 1):
            if 0 <= q < len(lv) and lv[r][0] > lv[q][1]:
                return False
    return True


def _brute_interdig(mlc, pi, occupied, leaves, k):
    """Every combination of feasible row openings obeying the constraint; the
    largest sequential float64 sum of the row values."""
    Lmin, Lmax, Rmin, Rmax = oracle.leaf_windows(mlc, occupied, leaves, k)
    N = mlc.n_cols
    states, vals = [], []
    for r in range(mlc.n_rows):
        row = pi[(k * mlc.n_rows + r) * N:(k * mlc.n_rows + r + 1) * N]
        P = window_prefix(row, Lmin[r], Rmax[r])
        st = [(L, R) for L in range(N + 1) for R in range(L, N + 1)
              if Lmin[r] <= L <= Lmax[r] and Rmin[r] <= R <= Rmax[r]]
        states.append(st)
        vals.append({s: P[s[1]] - P[s[0]] for s in st})
    best = None
    for combo in itertools.product(*states):
        if not _interdig_ok(combo):
            continue
        tot = 0.0
        for r, s in enumerate(combo):
            tot = tot + vals[r][s]
        if best is None or tot > best:
            best = tot
    return best


@pytest.mark.parametrize("seed", range(6))
def test_interdig_dp_matches_exhaustive_enumeration(seed):
    rng = np.random.default_rng(seed)
    mlc = synth.MLC(4, 3, 4, np.array([0], np.int32), 1, interdigitation=True)
    # small integers make exact ties common; some rows strongly negative
    pi = rng.integers(-3, 4, size=mlc.K * mlc.n_rows * mlc.n_cols).astype(np.float32)
    if seed % 2:
        pi = (pi * rng.uniform(0.1, 1.0, size=pi.shape)).astype(np.float32)
    occupied = np.zeros(mlc.K, bool)
    leaves = np.zeros((mlc.K, mlc.n_rows, 2), np.int64)
    if seed >= 3:  # a neighbour CP with interdigitated leaves narrows the windows
        occupied[1] = True
        leaves[1] = [[1, 3], [0, 2], [2, 4]]
    for k in range(mlc.K):
        if occupied[k]:
            continue
        ref = _brute_interdig(mlc, pi, occupied, leaves, k)
        price, lv = oracle.price_cp_interdig(mlc, pi, occupied, leaves, k)
        if ref is None:
            assert price is None
            continue
        assert price == ref
        assert _interdig_ok(lv)
        Lmin, Lmax, Rmin, Rmax = oracle.leaf_windows(mlc, occupied, leaves, k)
        tot = 0.0
        for r in range(mlc.n_rows):
            assert Lmin[r] <= lv[r][0] <= Lmax[r] and Rmin[r] <= lv[r][1] <= Rmax[r] and lv[r][0] <= lv[r][1]
            P = window_prefix(pi[(k * mlc.n_rows + r) * 4:(k * mlc.n_rows + r + 1) * 4], Lmin[r], Rmax[r])
            tot = tot + (P[lv[r][1]] - P[lv[r][0]])
        assert tot == price


def test_interdig_equals_independent_rows_when_unconstrained():
    # openings that already interlock (every row open over the same columns): the
    # constraint is inactive and the chain price is the row-by-row price
    mlc_free = synth.MLC(3, 4, 6, np.array([0], np.int32), 3)
    mlc_id = synth.MLC(3, 4, 6, np.array([0], np.int32), 3, interdigitation=True)
    pi = np.full(3 * 4 * 6, -1.0, np.float32)
    pi.reshape(3, 4, 6)[:, :, 2:4] = 2.0
    occupied = np.zeros(3, bool)
    leaves = np.zeros((3, 4, 2), np.int64)
    for k in range(3):
        p_free, lv_free = oracle.price_cp(mlc_free, pi, occupied, leaves, k)
        p_id, lv_id = oracle.price_cp_interdig(mlc_id, pi, occupied, leaves, k)
        assert p_id == p_free == 16.0
        assert np.array_equal(lv_id, lv_free)


def test_interdig_constraint_binds():
    # row 0 wants [0, 1), row 1 wants [5, 6): they do not interlock, so the chain
    # gives up value; the row-by-row optimum is infeasible under the constraint
    mlc_id = synth.MLC(1, 2, 6, np.array([0], np.int32), 3, interdigitation=True)
    mlc_free = synth.MLC(1, 2, 6, np.array([0], np.int32), 3)
    pi = np.float32([5, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 5])
    occupied = np.zeros(1, bool)
    leaves = np.zeros((1, 2, 2), np.int64)
    p_free, lv_free = oracle.price_cp(mlc_free, pi, occupied, leaves, 0)
    assert p_free == 10.0 and not _interdig_ok(lv_free)
    p_id, lv_id = oracle.price_cp_interdig(mlc_id, pi, occupied, leaves, 0)
    assert _interdig_ok(lv_id) and p_id == _brute_interdig(mlc_id, pi, occupied, leaves, 0) and p_id < 10.0


# ------------------------------------------------ interdigitation: the chosen leaves (reading R10's order)

def _chains(states, n_rows):
    """Every combination of one state per row in which adjacent rows interlock
    (L_r <= R_{r-1} and L_{r-1} <= R_r), by depth-first extension row by row."""
    out = []

    def extend(prefix):
        if len(prefix) == n_rows:
            out.append(tuple(prefix))
            return
        for s in states[len(prefix)]:
            if prefix and not (s[0] <= prefix[-1][1] and prefix[-1][0] <= s[1]):
                continue
            extend(prefix + [s])

    extend([])
    return out


def _brute_interdig_aperture(mlc, pi, occupied, leaves, k):
    """The aperture R10 selects, by enumeration: of every feasible interlocking
    combination of row openings, the first in R10's order on whole apertures.
    That order compares the total (the sequential float64 sum of the row values),
    larger first; then the last row's opening by the R8 key (width, |L + R - N|,
    L); then the partial sum through the row before it, larger first, and that
    row's opening by the R8 key; and so on down to the first row.
    Returns (price, leaves) or (None, None)."""
    Lmin, Lmax, Rmin, Rmax = oracle.leaf_windows(mlc, occupied, leaves, k)
    N = mlc.n_cols
    states, vals = [], []
    for r in range(mlc.n_rows):
        row = pi[(k * mlc.n_rows + r) * N:(k * mlc.n_rows + r + 1) * N]
        P = window_prefix(row, Lmin[r], Rmax[r])
        st = [(L, R) for L in range(N + 1) for R in range(L, N + 1)
              if Lmin[r] <= L <= Lmax[r] and Rmin[r] <= R <= Rmax[r]]
        states.append(st)
        vals.append({s: P[s[1]] - P[s[0]] for s in st})
    best = None
    for combo in _chains(states, mlc.n_rows):
        assert _interdig_ok(combo)
        partial, tot = [], 0.0
        for r, s in enumerate(combo):
            tot = tot + vals[r][s]
            partial.append(tot)
        key = []
        for r in range(mlc.n_rows - 1, -1, -1):
            L, R = combo[r]
            key += [-partial[r], R - L, abs(L + R - N), L]
        key = tuple(key)
        if best is None or key < best[0]:
            best = (key, tot, combo)
    if best is None:
        return None, None
    return best[1], np.array(best[2], np.int64)


def _interdig_case(seed, n_rows, n_cols, K=4):
    """Prices with many exact ties (small integers), or ties broken by rounding
    (values of very different size), and an occupied neighbour on some seeds."""
    rng = np.random.default_rng(seed)
    mlc = synth.MLC(K, n_rows, n_cols, np.array([0], np.int32), 1 + seed % 2, interdigitation=True)
    J = K * n_rows * n_cols
    kind = seed % 3
    if kind == 0:
        pi = rng.integers(-2, 3, size=J).astype(np.float32)
    elif kind == 1:
        pi = (rng.integers(-3, 4, size=J) * rng.uniform(0.1, 1.0, size=J)).astype(np.float32)
    else:  # 2^25 + small: partial sums round, so distinct chains reach equal totals
        pi = np.where(rng.random(J) < 0.3, 2.0 ** 25, rng.integers(-2, 3, size=J)).astype(np.float32)
    occupied = np.zeros(K, bool)
    leaves = np.zeros((K, n_rows, 2), np.int64)
    if seed % 4 >= 2:
        occupied[1] = True
        L = rng.integers(0, n_cols + 1, size=n_rows)
        R = np.minimum(n_cols, L + rng.integers(0, n_cols + 1, size=n_rows))
        leaves[1] = np.stack([L, R], axis=1)
    return mlc, pi, occupied, leaves


# 5 x 6 only with an occupied neighbour (seed % 4 >= 2), whose windows keep the enumeration short
@pytest.mark.parametrize("n_rows,n_cols,seed", [(3, 6, s) for s in range(6)] + [(4, 5, s) for s in range(6)] +
                         [(5, 4, s) for s in range(6)] + [(5, 6, s) for s in (2, 3, 6, 7)])
def test_interdig_plain_dp_leaves_match_enumeration(n_rows, n_cols, seed):
    mlc, pi, occupied, leaves = _interdig_case(seed, n_rows, n_cols, K=3 if n_rows * n_cols >= 30 else 4)
    for k in range(mlc.K):
        if occupied[k]:
            continue
        p_ref, lv_ref = _brute_interdig_aperture(mlc, pi, occupied, leaves, k)
        price, lv = oracle.price_cp_interdig_plain(mlc, pi, occupied, leaves, k)
        if p_ref is None:
            assert price is None
            continue
        assert np.float64(price).view(np.uint64) == np.float64(p_ref).view(np.uint64)
        assert np.array_equal(lv, lv_ref), (k, lv, lv_ref)


@pytest.mark.parametrize("seed", range(8))
def test_interdig_fast_form_matches_plain_dp(seed):
    """price_cp_interdig (prefix/suffix dominance passes) against the plain DP,
    leaves and price, on 12 x 12 rows with occupied neighbours and ties."""
    rng = np.random.default_rng(100 + seed)
    K, NR, N = 10, 12, 12
    mlc = synth.MLC(K, NR, N, np.array([0, 6], np.int32), 2 + seed % 3, interdigitation=True)
    J = K * NR * N
    if seed % 2:
        pi = rng.integers(-2, 3, size=J).astype(np.float32)
    else:
        pi = (rng.normal(size=J) * 5.0).astype(np.float32)
        pi[rng.random(J) < 0.4] = 0.0
    occupied = np.zeros(K, bool)
    occupied[[2, 7]] = True
    leaves = np.zeros((K, NR, 2), np.int64)
    for kk in (2, 7):
        L = rng.integers(0, N // 2 + 1, size=NR)
        leaves[kk] = np.stack([L, np.minimum(N, L + rng.integers(0, N // 2 + 1, size=NR))], axis=1)
    for k in range(K):
        if occupied[k]:
            continue
        p_ref, lv_ref = oracle.price_cp_interdig_plain(mlc, pi, occupied, leaves, k)
        price, lv = oracle.price_cp_interdig(mlc, pi, occupied, leaves, k)
        if p_ref is None:
            assert price is None
            continue
        assert np.float64(price).view(np.uint64) == np.float64(p_ref).view(np.uint64)
        assert np.array_equal(lv, lv_ref), (k, lv, lv_ref)


def _planted(monkeypatch, which):
    """Plant one mistake in the oracle's interdigitation order (CPU only)."""
    if which == "tie_L":  # L ascending flipped in the dominance passes
        def bad(va, La, Ra, vb, Lb, Rb, N):
            wa, wb = Ra - La, Rb - Lb
            ca, cb = np.abs(La + Ra - N), np.abs(Lb + Rb - N)
            return (va > vb) | ((va == vb) & ((wa < wb) | ((wa == wb) & ((ca < cb) | ((ca == cb) & (La > Lb))))))
        monkeypatch.setattr(oracle.vmat_oracle, "_better", bad)
    elif which == "tie_width":  # wider first
        def bad(va, La, Ra, vb, Lb, Rb, N):
            wa, wb = Ra - La, Rb - Lb
            ca, cb = np.abs(La + Ra - N), np.abs(Lb + Rb - N)
            return (va > vb) | ((va == vb) & ((wa > wb) | ((wa == wb) & ((ca < cb) | ((ca == cb) & (La < Lb))))))
        monkeypatch.setattr(oracle.vmat_oracle, "_better", bad)
    elif which == "final_key":  # the last row's state chosen without the centredness term
        monkeypatch.setattr(oracle.vmat_oracle, "_state_order", lambda val, L, R, N: (L, R - L, -val))


@pytest.mark.parametrize("which", ["tie_L", "tie_width", "final_key"])
def test_interdig_planted_order_mistakes_are_caught(monkeypatch, which):
    """Each planted mistake in the fast form's order changes a chosen aperture on
    the tie-heavy cases above, so the pins would fail."""
    _planted(monkeypatch, which)
    caught = False
    for seed in range(6):
        mlc, pi, occupied, leaves = _interdig_case(seed, 4, 5)
        for k in range(mlc.K):
            if occupied[k]:
                continue
            p_ref, lv_ref = oracle.price_cp_interdig_plain(mlc, pi, occupied, leaves, k)
            price, lv = oracle.price_cp_interdig(mlc, pi, occupied, leaves, k)
            if p_ref is not None and (price != p_ref or not np.array_equal(lv, lv_ref)):
                caught = True
    assert caught
