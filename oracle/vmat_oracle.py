"""FP64 CPU oracle for the column-generation VMAT hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import or run this module.  The
product path (the CUDA library ``libvmat`` and its Python binding) never calls
it, and this module imports nothing from that path.

Plain numpy/scipy in float64, written from Tian et al., "Multi-GPU
implementation of a VMAT treatment plan optimization algorithm"
(arXiv:1503.01721):

* Eq. 1            voxel objective F(z) and Eq. 4 g = -grad F
* Eq. 3            beamlet price pi = D^T g
* Section 2.1      z = D x (dose from beamlet fluence)
* Section 2.2.2    per-MLC-row best opening, per-CP aperture price, best CP
* Eq. 5            aperture dose vector DA = sum of D's columns in the aperture
* Eq. 6-10         master problem by Barzilai-Borwein steps with the
                   subspace (bound) scheme; Section 2.1 stopping rules
* Eq. 2, 6         fluence-rate bounds from gantry-speed, dose-rate and leaf-speed limits
* Section 2.1      column-generation loop (PP <-> MP)

Readings where the paper is silent or ambiguous (each is repeated where used):

R1  Eq. 7-10 sign: the BB step lengths are formed from the gradient of F in
    the fluence domain, G = grad_y F = -DA^T g, so both step lengths are
    positive; Eq. 9-10, written for g_A = -G, freeze y at its lower bound when
    G > 0 and at its upper bound when G < 0.
R2  After each step y is projected onto its box (projected BB).
R3  First step: Cauchy step delta0 = G.G / (2 sum_i w_i (DA G)_i^2), w_i the
    active penalty weight of voxel i (w+ if z>T, w- if z<T, 0 if z=T).
    Then BB1 = s.s/s.r on even iterations, BB2 = s.r/r.r on odd ones; if
    s.r <= 0 the step is delta_max.  Steps are clamped to
    [delta_min, delta_max] * delta0.
R4  Stopping: |F_{t-5} - F_t| <= rel_tol5 * F_t, or
    max|y_t - y_{t-1}| <= step_tol * max(1, max|y_t|), or t = max_iter - 1.
R5  Warm start: the previous y is kept, the new aperture starts at 0.
R6  Fluence bounds [lo, hi] per aperture, default [0, +inf).
R7  Neighbour compatibility (Eq. 2, Section 2.1): for the nearest occupied CP
    on each side within the same arc, at distance m, every leaf stays within
    m * travel_cols columns of that CP's leaf.  No wrap across arc ends.
R8  Ties: a row opening [L, R) is chosen by (value desc, width asc,
    |L + R - n_cols| asc, L asc); CPs by (price desc, index asc).  Row values
    are P_R - P_L with P the sequential float64 prefix sum of the float32
    prices over the row's window [Lmin, Rmax) of R7 (P_c = 0 up to Lmin,
    constant after Rmax): the price of an opening is the sum of its
    beamlets' prices, and only beamlets inside the window can be in an
    opening, so prices outside it never enter a value.  The CP price is the
    sequential float64 sum over rows.
R9  The loop stops when the best CP price is <= 0 (no aperture lowers F) or
    when n_apertures have been generated.
R11 Delivery limits (Eq. 2, 6).  Gantry speed s_k of an occupied CP is the
    speed over the interval that starts at k and ends at the next occupied CP
    k' of the same arc, m = k' - k CP steps of cp_step degrees.  Its leaves move
    at most d = max over rows of |L_k - L_k'|, |R_k - R_k'| columns in that
    interval, so s_k <= S^U_{k,k'} = m cp_step leaf_speed / d (no limit when
    d = 0 or k is the last occupied CP of its arc).  Speed changes between
    consecutive occupied CPs are at most m Delta S.  The updated bounds of
    Eq. 6 are the extreme speeds these constraints allow at k:
    S^U_k = min over occupied j of the arc of (min(S^U, S^U_{j,j'}) + Delta S |k - j|),
    S^L_k = S^L; then R^L / S^U_k <= y_k <= R^U / S^L_k, in float64, rounded to
    float32 for the master problem.  Bounds are recomputed after every new
    aperture.  The travel window (R7) must not exceed what the leaves can do at
    the slowest gantry speed (travel_cols S^L <= cp_step leaf_speed), which
    keeps S^U_k >= S^L.
R10 Interdigitation (Section 2.2.2, second variant): the left leaf of a row may
    not pass the right leaf of an adjacent row, L_r <= min(R_{r-1}, R_{r+1}).
    The best aperture of a CP is then a chain over the rows: the sequential
    float64 sum of row values, maximised by dynamic programming over the row
    states (L, R) in row order (the sum is monotone in the partial sum, so the
    optimum of each prefix extends to the optimum of the next).  A state's
    predecessor is the compatible state of the previous row with the largest
    partial sum, ties by the row key of R8; the last row's state likewise.
    Backtracking from it gives the aperture.  ``price_cp_interdig_plain``
    is this reading written out state by state (every compatible pair of
    states visited); ``price_cp_interdig`` reaches the same states, sums and
    predecessors with prefix/suffix passes over the row states and is the
    form used at clinical sizes.  Both are checked against an enumeration of
    every interlocking aperture under R10's order on whole apertures (total,
    then the last row's key, then the partial sum before it and that row's
    key, down to the first row), prices and leaves.
R12 FP32 refinement of a BF16 / FP8 plan (the precision form): the apertures
    stay as chosen on the stored values; their dose vectors are recomputed from
    the float32 values, the master problem is solved again from the plan's y,
    and the final dose comes from the float32 values.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

F64 = np.float64


# ----------------------------------------------------------------------------
# DDC matrix and the two sparse products
# ----------------------------------------------------------------------------

def ddc_matrix(V: int, J: int, vox, blt, val):
    """D (V voxels x J beamlets) from COO, float64 CSR (Section 2.2.2 storage).

    Duplicate (voxel, beamlet) pairs are summed.
    """
    return sp.csr_matrix((np.asarray(val, F64), (np.asarray(vox, np.int64), np.asarray(blt, np.int64))),
                         shape=(V, J))


def dose_forward(D, x):
    """z = D x, z_i = sum_j D_ij x_j (Section 2.1, dose of a beamlet fluence)."""
    return D @ np.asarray(x, F64)


def beamlet_price(D, g):
    """pi = D^T g, pi_j = sum_i g_i D_ij (Eq. 3)."""
    return D.T @ np.asarray(g, F64)


# ----------------------------------------------------------------------------
# Objective (Eq. 1) and its negative gradient (Eq. 4)
# ----------------------------------------------------------------------------

def objective_grad(z, struct_id, T, w_over, w_under):
    """F(z) = sum_i w+_i max(0, z_i - T_i)^2 + w-_i max(0, T_i - z_i)^2 (Eq. 1)
    and g = -grad F = -2 w+ max(0, z - T) + 2 w- max(0, T - z) (Eq. 4)."""
    sid = np.asarray(struct_id, np.int64)
    Tv = np.asarray(T, F64)[sid]
    wo = np.asarray(w_over, F64)[sid]
    wu = np.asarray(w_under, F64)[sid]
    z = np.asarray(z, F64)
    over = np.maximum(0.0, z - Tv)
    under = np.maximum(0.0, Tv - z)
    F = float(np.sum(wo * over * over + wu * under * under))
    g = -2.0 * wo * over + 2.0 * wu * under
    return F, g


def active_weight(z, struct_id, T, w_over, w_under):
    """Curvature weight of each voxel's penalty at z: w+ if z > T, w- if z < T, else 0."""
    sid = np.asarray(struct_id, np.int64)
    Tv = np.asarray(T, F64)[sid]
    z = np.asarray(z, F64)
    return np.where(z > Tv, np.asarray(w_over, F64)[sid], np.where(z < Tv, np.asarray(w_under, F64)[sid], 0.0))


# ----------------------------------------------------------------------------
# Pricing problem, second step (Section 2.2.2; readings R7, R8)
# ----------------------------------------------------------------------------

def arc_of(mlc, k: int):
    """(first CP, one past the last CP) of the arc containing CP k."""
    first = [int(a) for a in mlc.arc_first_cp] + [int(mlc.K)]
    for a in range(len(first) - 1):
        if first[a] <= k < first[a + 1]:
            return first[a], first[a + 1]
    raise ValueError("CP outside every arc")


def leaf_windows(mlc, occupied, leaves, k: int):
    """Per-row feasible ranges (Lmin, Lmax, Rmin, Rmax) at CP k (reading R7)."""
    N = mlc.n_cols
    nr = mlc.n_rows
    Lmin = np.zeros(nr, np.int64)
    Lmax = np.full(nr, N, np.int64)
    Rmin = np.zeros(nr, np.int64)
    Rmax = np.full(nr, N, np.int64)
    a0, a1 = arc_of(mlc, k)
    for step in (-1, 1):
        kk = k + step
        while a0 <= kk < a1 and not occupied[kk]:
            kk += step
        if a0 <= kk < a1:
            m = abs(k - kk)
            reach = m * mlc.travel_cols
            Ln = np.asarray(leaves[kk][:, 0], np.int64)
            Rn = np.asarray(leaves[kk][:, 1], np.int64)
            Lmin = np.maximum(Lmin, Ln - reach)
            Lmax = np.minimum(Lmax, Ln + reach)
            Rmin = np.maximum(Rmin, Rn - reach)
            Rmax = np.minimum(Rmax, Rn + reach)
    return Lmin, Lmax, Rmin, Rmax


def prefix_sums(pi_row, lo: int = 0, hi=None):
    """Float64 prefix sums over the columns [lo, hi) of a row (reading R8):
    P_c = 0 for c <= lo, P_{c+1} = P_c + pi_c for lo <= c < hi, accumulated in
    column order, and P_c = P_hi for c > hi.  Entries outside [lo, hi) are not read."""
    N = len(pi_row)
    hi = N if hi is None else hi
    P = np.zeros(N + 1, F64)
    if hi > lo:
        np.cumsum(np.asarray(pi_row[lo:hi], F64), out=P[lo + 1:hi + 1])
        P[hi + 1:] = P[hi]
    return P


def best_opening(pi_row, Lmin: int, Lmax: int, Rmin: int, Rmax: int):
    """Best open interval [L, R) of one MLC row: max of P_R - P_L over the
    feasible pairs, ties by (width asc, |L + R - N| asc, L asc) (reading R8).

    Returns (value, L, R), or (None, -1, -1) if no pair is feasible.
    """
    N = len(pi_row)
    P = prefix_sums(pi_row, Lmin, Rmax)
    L, R = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    feas = (L <= R) & (L >= Lmin) & (L <= Lmax) & (R >= Rmin) & (R <= Rmax)
    if not feas.any():
        return None, -1, -1
    Lf, Rf = L[feas], R[feas]
    v = P[Rf] - P[Lf]
    order = np.lexsort((Lf, np.abs(Lf + Rf - N), Rf - Lf, -v))
    b = order[0]
    return float(v[b]), int(Lf[b]), int(Rf[b])


def price_cp(mlc, pi, occupied, leaves, k: int):
    """Best aperture at CP k: per-row best openings and their sequential sum."""
    Lmin, Lmax, Rmin, Rmax = leaf_windows(mlc, occupied, leaves, k)
    N = mlc.n_cols
    base = k * mlc.n_rows * N
    out = np.zeros((mlc.n_rows, 2), np.int64)
    price = 0.0
    for r in range(mlc.n_rows):
        row = pi[base + r * N: base + (r + 1) * N]
        v, Lb, Rb = best_opening(row, int(Lmin[r]), int(Lmax[r]), int(Rmin[r]), int(Rmax[r]))
        if v is None:
            return None, None
        price = price + v
        out[r] = (Lb, Rb)
    return price, out


def _state_order(val, L, R, N):
    """Sort key arrays for 'better first': value desc, width asc, centredness asc, L asc."""
    return (L, np.abs(L + R - N), R - L, -val)


def _better(va, La, Ra, vb, Lb, Rb, N):
    """Elementwise: is state a strictly better than state b (R8 order on the partial sums)?"""
    wa, wb = Ra - La, Rb - Lb
    ca, cb = np.abs(La + Ra - N), np.abs(Lb + Rb - N)
    return (va > vb) | ((va == vb) & ((wa < wb) | ((wa == wb) & ((ca < cb) | ((ca == cb) & (La < Lb))))))


def price_cp_interdig(mlc, pi, occupied, leaves, k: int, with_leaves: bool = True):
    """Best aperture at CP k under the interdigitation constraint (reading R10).

    Row states are the feasible (L, R) of R7 with L <= R; S_r(L, R) = S_{r-1}(pred)
    + (P_R - P_L) in float64, S_0 = P_R - P_L.  Compatible predecessors of (L', R')
    are the states (L, R) with L <= R' and L' <= R.  Returns (price, leaves) or
    (None, None) when no chain is feasible.

    The best compatible predecessor of every state is found with two sweeps
    instead of a scan per state: over R from n_cols down (the best state with
    R >= b for each L), then over L upward (the best of those with L <= a), so
    M[a][b] is the best state with L <= a and R >= b, and the predecessor of
    (L', R') is M[R'][L'].  The result equals ``price_cp_interdig_plain``.
    """
    Lmin, Lmax, Rmin, Rmax = leaf_windows(mlc, occupied, leaves, k)
    N = mlc.n_cols
    base = k * mlc.n_rows * N
    Lg, Rg = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    NEG = -np.inf
    S = None
    preds = []
    for r in range(mlc.n_rows):
        P = prefix_sums(pi[base + r * N: base + (r + 1) * N], int(Lmin[r]), int(Rmax[r]))
        feas = (Lg <= Rg) & (Lg >= Lmin[r]) & (Lg <= Lmax[r]) & (Rg >= Rmin[r]) & (Rg <= Rmax[r])
        v = np.where(feas, P[Rg] - P[Lg], NEG)
        if S is None:
            S_new = v
            preds.append(None)
        else:
            # C[L][b]: best state (L, R) with R >= b (suffix over R), then M[a][b]: best of
            # C[L][b] over L <= a (prefix over L); pred of (L', R') = M[R'][L']
            bestL = np.tile(np.arange(N + 1)[:, None], (1, N + 1))
            bestR = np.full((N + 1, N + 1), N, np.int64)
            bestV = S[:, N].copy()[:, None].repeat(N + 1, axis=1)
            cL = np.arange(N + 1)
            cR = np.full(N + 1, N, np.int64)
            cV = S[:, N].copy()
            for b in range(N, -1, -1):
                if b < N:
                    cand = _better(S[:, b], cL, np.full(N + 1, b), cV, cL, cR, N)
                    cV = np.where(cand, S[:, b], cV)
                    cR = np.where(cand, b, cR)
                bestV[:, b], bestR[:, b] = cV, cR
            mV = np.empty((N + 1, N + 1))
            mL = np.empty((N + 1, N + 1), np.int64)
            mR = np.empty((N + 1, N + 1), np.int64)
            pV, pL, pR = bestV[0].copy(), np.zeros(N + 1, np.int64), bestR[0].copy()
            for a in range(N + 1):
                if a > 0:
                    cand = _better(bestV[a], np.full(N + 1, a), bestR[a], pV, pL, pR, N)
                    pV = np.where(cand, bestV[a], pV)
                    pL = np.where(cand, a, pL)
                    pR = np.where(cand, bestR[a], pR)
                mV[a], mL[a], mR[a] = pV, pL, pR
            predV, predL, predR = mV[Rg, Lg], mL[Rg, Lg], mR[Rg, Lg]
            S_new = np.where(feas & (predV > NEG), predV + v, NEG)
            preds.append((predL, predR))
        S = S_new
    flat = np.argwhere(S > NEG)
    if len(flat) == 0:
        return None, None
    Lf, Rf = flat[:, 0], flat[:, 1]
    o = np.lexsort(_state_order(S[Lf, Rf], Lf, Rf, N))
    L, R = int(Lf[o[0]]), int(Rf[o[0]])
    price = float(S[L, R])
    if not with_leaves:
        return price, None
    out = np.zeros((mlc.n_rows, 2), np.int64)
    for r in range(mlc.n_rows - 1, -1, -1):
        out[r] = (L, R)
        if r > 0:
            L, R = int(preds[r][0][L, R]), int(preds[r][1][L, R])
    return price, out


def price_cp_interdig_plain(mlc, pi, occupied, leaves, k: int):
    """Reading R10 written out state by state: the reference form of
    ``price_cp_interdig``, slow (every pair of states of adjacent rows is
    visited), for small MLCs and for checking the fast form.

    Row r's states are its feasible openings (L, R) of R7 with value P_R - P_L
    (R8 prefix sums).  For each state of row r, every state (L, R) of row r - 1
    that has a chain and is compatible with it (L <= R' and L' <= R: each left
    leaf stays left of the neighbouring right leaf) is visited, and the best by
    (partial sum desc, R - L asc, |L + R - n_cols| asc, L asc) becomes its
    predecessor; its partial sum is that predecessor's plus its own value, in
    float64.  The last row's state is chosen by the same key; the aperture is
    read back through the predecessors.  Returns (price, leaves [n_rows, 2]) or
    (None, None) when no chain is feasible.
    """
    Lmin, Lmax, Rmin, Rmax = leaf_windows(mlc, occupied, leaves, k)
    N = mlc.n_cols
    base = k * mlc.n_rows * N

    def key(st):  # st = (L, R, partial sum, predecessor index)
        L, R, S = st[0], st[1], st[2]
        return (-S, R - L, abs(L + R - N), L)

    rows = []  # per row: the list of states that have a chain
    for r in range(mlc.n_rows):
        P = prefix_sums(pi[base + r * N: base + (r + 1) * N], int(Lmin[r]), int(Rmax[r]))
        cur = []
        for L in range(int(Lmin[r]), int(Lmax[r]) + 1):
            for R in range(max(L, int(Rmin[r])), int(Rmax[r]) + 1):
                v = float(P[R] - P[L])
                if r == 0:
                    cur.append((L, R, v, -1))
                    continue
                best = -1
                for q, prev in enumerate(rows[r - 1]):
                    if prev[0] <= R and L <= prev[1]:
                        if best < 0 or key(prev) < key(rows[r - 1][best]):
                            best = q
                if best >= 0:
                    cur.append((L, R, rows[r - 1][best][2] + v, best))
        if not cur:
            return None, None
        rows.append(cur)
    last = min(range(len(rows[-1])), key=lambda q: key(rows[-1][q]))
    price = rows[-1][last][2]
    out = np.zeros((mlc.n_rows, 2), np.int64)
    q = last
    for r in range(mlc.n_rows - 1, -1, -1):
        out[r] = rows[r][q][:2]
        q = rows[r][q][3]
    return price, out


def price_apertures(mlc, pi, occupied, leaves):
    """Best CP over the unoccupied ones and its aperture (Section 2.2.2).

    ``pi`` holds the float32 beamlet prices (converted exactly to float64).
    Returns (k, leaves [n_rows, 2], price); k = -1 when no CP is feasible.
    """
    pi = np.asarray(pi)
    best_k, best_leaves, best_price = -1, None, -np.inf
    interdig = bool(getattr(mlc, "interdigitation", False))
    for k in range(mlc.K):
        if occupied[k]:
            continue
        if interdig:
            price, lv = price_cp_interdig(mlc, pi, occupied, leaves, k)
        else:
            price, lv = price_cp(mlc, pi, occupied, leaves, k)
        if price is None:
            continue
        if best_k < 0 or price > best_price:
            best_k, best_leaves, best_price = k, lv, price
    return best_k, best_leaves, best_price


# ----------------------------------------------------------------------------
# Apertures <-> beamlets (Eq. 5 and the fluence map of a set of apertures)
# ----------------------------------------------------------------------------

def aperture_beamlets(mlc, k: int, leaves):
    """Beamlet indices inside the aperture at CP k ([L, R) per row)."""
    idx = []
    for r in range(mlc.n_rows):
        L, R = int(leaves[r][0]), int(leaves[r][1])
        base = (k * mlc.n_rows + r) * mlc.n_cols
        idx.extend(range(base + L, base + R))
    return np.array(idx, np.int64)


def aperture_indicator(mlc, k: int, leaves):
    x = np.zeros(mlc.K * mlc.n_rows * mlc.n_cols, F64)
    x[aperture_beamlets(mlc, k, leaves)] = 1.0
    return x


def aperture_dose(D, mlc, k: int, leaves):
    """DA(A_k) = sum_{j in A_k} D_{:, j} (Eq. 5)."""
    return D @ aperture_indicator(mlc, k, leaves)


def aperture_fluence(mlc, cps, leaves, y):
    """x = A y: x_j = sum over apertures n containing beamlet j of y_n."""
    x = np.zeros(mlc.K * mlc.n_rows * mlc.n_cols, F64)
    for n, k in enumerate(cps):
        x[aperture_beamlets(mlc, int(k), leaves[n])] += float(y[n])
    return x


def aperture_grad(mlc, cps, leaves, pi):
    """A^T pi: entry n is the sum of pi over the beamlets of aperture n."""
    pi = np.asarray(pi, F64)
    return np.array([float(np.sum(pi[aperture_beamlets(mlc, int(k), leaves[n])])) for n, k in enumerate(cps)], F64)


# ----------------------------------------------------------------------------
# Fluence-rate bounds from the delivery limits (Eq. 2, 6; reading R11)
# ----------------------------------------------------------------------------

def gantry_speed_bounds(mlc, machine, cps, leaves):
    """Largest gantry speed S^U_k allowed at each placed CP (reading R11).

    Returns (S_hat, S_U) per placed aperture, in the order of ``cps``: S_hat is
    min(S^U, S^U_{k,k'}) of the aperture's own interval, S_U the updated bound
    after the speed-change limit."""
    n = len(cps)
    cps = [int(k) for k in cps]
    lv = [np.asarray(l, np.int64).reshape(mlc.n_rows, 2) for l in leaves]
    S_hat = np.full(n, float(machine.speed_max), F64)
    for t, k in enumerate(cps):
        a0, a1 = arc_of(mlc, k)
        later = [(kk, u) for u, kk in enumerate(cps) if k < kk < a1]
        if not later:
            continue
        k2, u = min(later)
        d = int(np.max(np.abs(lv[t] - lv[u])))
        if d > 0:
            m = k2 - k
            S_hat[t] = min(S_hat[t], (float(m) * machine.cp_step_deg) * machine.leaf_speed_cols / float(d))
    S_U = np.empty(n, F64)
    for t, k in enumerate(cps):
        a0, a1 = arc_of(mlc, k)
        S_U[t] = min(S_hat[u] + machine.speed_step_max * float(abs(k - kk))
                     for u, kk in enumerate(cps) if a0 <= kk < a1)
    return S_hat, S_U


def fluence_bounds(mlc, machine, cps, leaves):
    """Eq. 6 bounds R^L / S^U_k <= y_k <= R^U / S^L of each placed aperture, as
    float32 (reading R11).  Without a machine: [0, +inf)."""
    n = len(cps)
    if machine is None:
        return np.zeros(n, np.float32), np.full(n, np.inf, np.float32)
    _, S_U = gantry_speed_bounds(mlc, machine, cps, leaves)
    lo = machine.rate_min / S_U
    hi = np.full(n, machine.rate_max / machine.speed_min if machine.speed_min > 0 else np.inf, F64)
    return lo.astype(np.float32), hi.astype(np.float32)


# ----------------------------------------------------------------------------
# Master problem (Eq. 6-10; readings R1-R6)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class BBOptions:
    max_iter: int = 500
    rel_tol5: float = 1e-6
    step_tol: float = 1e-9
    delta_min: float = 1e-12
    delta_max: float = 1e12


STOP_REL, STOP_STEP, STOP_MAXIT, STOP_GRAD0, STOP_FLAT = 1, 2, 3, 4, 5


def mp_bb_solve(DA, struct_id, T, w_over, w_under, y0, lo=None, hi=None, opts: BBOptions | None = None,
                F_offset: float = 0.0):
    """min F(DA y) over lo <= y <= hi by BB steps with the subspace scheme.

    DA: float64 [V, n].  Returns (y, z, F, iters, stop_reason, F_history).
    Iteration t (t = 0, 1, ...): z = DA y, G = -DA^T g(z), Eq. 9-10 freeze,
    stopping tests (R4), step length (R3), projected update (R2).
    """
    opts = opts or BBOptions()
    DA = np.asarray(DA, F64)
    n = DA.shape[1]
    lo = np.zeros(n, F64) if lo is None else np.asarray(lo, F64)
    hi = np.full(n, np.inf, F64) if hi is None else np.asarray(hi, F64)
    y = np.clip(np.asarray(y0, F64), lo, hi)
    y_prev = G_prev = None
    delta0 = None
    hist = []
    reason = STOP_MAXIT
    for t in range(opts.max_iter):
        z = DA @ y
        F, g = objective_grad(z, struct_id, T, w_over, w_under)
        F += F_offset
        G = -(DA.T @ g)
        at_lo = (y <= lo) & (G > 0)
        at_hi = (y >= hi) & (G < 0)
        y = np.where(at_lo, lo, np.where(at_hi, hi, y))
        G = np.where(at_lo | at_hi, 0.0, G)
        hist.append(F)
        if t >= 5 and abs(hist[t - 5] - F) <= opts.rel_tol5 * F:
            reason = STOP_REL
            break
        if t >= 1 and np.max(np.abs(y - y_prev)) <= opts.step_tol * max(1.0, float(np.max(np.abs(y)))):
            reason = STOP_STEP
            break
        if t == opts.max_iter - 1:
            reason = STOP_MAXIT
            break
        if t == 0:
            gg = float(G @ G)
            if gg == 0.0:
                reason = STOP_GRAD0
                break
            w = active_weight(z, struct_id, T, w_over, w_under)
            q = DA @ G
            curv = 2.0 * float(np.sum(w * q * q))
            if curv == 0.0:
                reason = STOP_FLAT
                break
            delta0 = gg / curv
            delta = delta0
        else:
            s = y - y_prev
            r = G - G_prev
            sr = float(s @ r)
            if sr <= 0.0:
                delta = opts.delta_max * delta0
            elif t % 2 == 1:
                delta = sr / float(r @ r)
            else:
                delta = float(s @ s) / sr
            delta = min(max(delta, opts.delta_min * delta0), opts.delta_max * delta0)
        y_prev, G_prev = y.copy(), G.copy()
        y = np.clip(y - delta * G, lo, hi)
    return y, z, F, t + 1, reason, hist


# ----------------------------------------------------------------------------
# Column-generation loop (Section 2.1; reading R9)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class PlanResult:
    cps: list
    leaves: list           # [n_ap] arrays [n_rows, 2]
    y: np.ndarray
    dose: np.ndarray       # final D (A y)
    F: float
    prices: list           # best CP price at each generated aperture
    bb_iters: list
    stop: str


def cg_plan(D, mlc, structs, n_apertures: int, opts: BBOptions | None = None, price_fn=None):
    """Column generation: PP (Eq. 3 + row openings) then MP (Eq. 6-10), repeated.

    ``price_fn(g) -> pi`` may replace the float64 price (used by lockstep
    tests); by default pi = D^T g in float64.
    """
    sid, T, wo, wu = structs.struct_id, structs.T, structs.w_over, structs.w_under
    V, J = D.shape
    z = np.zeros(V, F64)
    occupied = np.zeros(mlc.K, bool)
    leaves_all = np.zeros((mlc.K, mlc.n_rows, 2), np.int64)
    cps, lvs, cols, prices, iters = [], [], [], [], []
    y = np.zeros(0, F64)
    stop = "count"
    for _ in range(n_apertures):
        _, g = objective_grad(z, sid, T, wo, wu)
        pi = price_fn(g) if price_fn is not None else beamlet_price(D, g)
        k, lv, price = price_apertures(mlc, pi, occupied, leaves_all)
        if k < 0 or not price > 0.0:
            stop = "price"
            break
        occupied[k] = True
        leaves_all[k] = lv
        cps.append(k)
        lvs.append(lv)
        prices.append(price)
        cols.append(aperture_dose(D, mlc, k, lv))
        y = np.concatenate([y, [0.0]])
        lo, hi = fluence_bounds(mlc, getattr(mlc, "machine", None), cps, lvs)
        y, z, _, it, _, _ = mp_bb_solve(np.stack(cols, axis=1), sid, T, wo, wu, y, lo, hi, opts=opts)
        iters.append(it)
    x = aperture_fluence(mlc, cps, lvs, y) if cps else np.zeros(J, F64)
    dose = dose_forward(D, x)
    F, _ = objective_grad(dose, sid, T, wo, wu)
    return PlanResult(cps, lvs, y, dose, F, prices, iters, stop)


def refine_plan(D, mlc, structs, cps, leaves, y, opts: BBOptions | None = None):
    """FP32 refinement of a plan chosen on lower-precision values (reading R12):
    with D holding the float32 values, each placed aperture's dose vector
    DA = sum of D's columns in the aperture (Eq. 5), the master problem of
    Eq. 6-10 again from the plan's y, and the final dose D (A y).

    Returns (y, dose, F, bb_iters).
    """
    s = structs
    DA = np.stack([aperture_dose(D, mlc, int(k), lv) for k, lv in zip(cps, leaves)], axis=1)
    yr, _, _, iters, _, _ = mp_bb_solve(DA, s.struct_id, s.T, s.w_over, s.w_under, np.asarray(y, F64), opts=opts)
    dose = dose_forward(D, aperture_fluence(mlc, cps, leaves, yr))
    F, _ = objective_grad(dose, s.struct_id, s.T, s.w_over, s.w_under)
    return yr, dose, F, iters


# ----------------------------------------------------------------------------
# Lower-precision DDC storage
# ----------------------------------------------------------------------------

def bf16_codes(x32):
    """Round float32 to bfloat16, round-to-nearest-even (finite inputs)."""
    b = np.asarray(x32, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return b.astype(np.uint16)


def bf16_values(codes):
    return (np.asarray(codes, np.uint16).astype(np.uint32) << 16).view(np.float32)


def _e4m3_table():
    """Values of the 127 finite non-negative E4M3 (fn) codes 0x00..0x7E."""
    vals = np.zeros(127, F64)
    for c in range(127):
        e = (c >> 3) & 0xF
        m = c & 0x7
        vals[c] = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return vals


_E4M3 = _e4m3_table()


def e4m3_codes(x):
    """Round to E4M3 (fn): nearest finite code, ties to even code, saturating at 448."""
    x = np.asarray(x, F64)
    a = np.minimum(np.abs(x), 448.0)
    hi = np.searchsorted(_E4M3, a, side="left").clip(0, 126)
    lo = (hi - 1).clip(0, 126)
    dlo = a - _E4M3[lo]
    dhi = _E4M3[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    c = np.where(pick_hi, hi, lo).astype(np.uint8)
    return np.where(x < 0, c | 0x80, c).astype(np.uint8)


def e4m3_values(codes):
    c = np.asarray(codes, np.uint8)
    v = _E4M3[(c & 0x7F).clip(0, 126)]
    return np.where(c & 0x80, -v, v)


def e4m3_scale(col_max):
    """Per-beamlet power-of-two scale s = 2^e, e the least integer with 448 s >= max.

    Zero columns get s = 1.  Division by s is then exact.
    """
    m = np.asarray(col_max, F64)
    e = np.where(m > 0, np.ceil(np.log2(np.where(m > 0, m, 1.0) / 448.0)), 0.0)
    e = np.where((m > 0) & (448.0 * np.exp2(e - 1) >= m), e - 1, e)
    e = np.where((m > 0) & (448.0 * np.exp2(e) < m), e + 1, e)
    return np.exp2(e)


def quantize_ddc(J, blt, val, dtype: str):
    """Stored value of every COO entry after quantisation, as float64.

    'f32' keeps the value; 'bf16' rounds to bfloat16; 'fp8' stores
    E4M3(val / s_j) with the per-beamlet scale s_j, and the value is s_j * code.
    Returns (dequantised values, per-beamlet scales or None).
    """
    val = np.asarray(val, np.float32)
    if dtype == "f32":
        return val.astype(F64), None
    if dtype == "bf16":
        return bf16_values(bf16_codes(val)).astype(F64), None
    if dtype == "fp8":
        mx = np.zeros(J, F64)
        np.maximum.at(mx, np.asarray(blt, np.int64), np.abs(val.astype(F64)))
        s = e4m3_scale(mx)
        q = e4m3_codes(val.astype(F64) / s[blt])
        return e4m3_values(q) * s[blt], s
    raise ValueError(dtype)
