"""Pins of the global-grid oracle (Eq. 4.3 on the cuboid grid of Sec. 5.2,
direction set R^1_1 of Eq. 5.1, trees of Algorithm 2 evaluated by
Algorithm 3): the grid sizes and the convergence history printed for the
Sec. 6.1 study, brute-force hulls on a tiny grid, the double well's closed
form, monotonicity and discrete rank-one convexity at convergence, and the
tree's consistency with the interpolated W^K."""
import itertools

import numpy as np
import pytest

NH61 = dict(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3)  # Table tab:2Dconvexification, NH row
BETA61 = 0.06
# Figure fig:convergence, NH, R^1_1 column: largest decrease of rows k = 2 .. 15
# (row 1, 2.84696, is printed for both direction sets and is not a decrease of
# this iteration; see the reading of the grid study)
PRINTED_NH_R11 = [1.62022, 1.14215, 0.09311, 0.01674, 0.00401, 0.00182, 0.00084, 0.00056,
                  0.00042, 0.00031, 0.00027, 0.00020, 0.00013, 0.00011]


def test_grid_sizes_of_the_sec61_study(orc):
    """Table tab:2Dconvexification: |N| = 648,025 (NH: delta 0.15, diagonal
    [0.1, 3.4], off-diagonal [-2.55, 2.55]) and 672,400 (STVK: delta 0.1,
    [0.1, 2.0], [-2.0, 2.0])."""
    g1 = orc.Grid.from_bounds((0.1, 3.4), (-2.55, 2.55), (0.15, 0.15))
    g2 = orc.Grid.from_bounds((0.1, 2.0), (-2.0, 2.0), (0.1, 0.1))
    assert g1.count == 648025 and g2.count == 672400
    P = g1.points()
    assert P.shape == (648025, 4)
    np.testing.assert_allclose(P[0], [0.1, -2.55, -2.55, 0.1])
    np.testing.assert_allclose(P[-1], [3.4, 2.55, 2.55, 3.4])


def test_r11_has_sixteen_distinct_rank_one_directions(orc):
    """Eq. (5.1): a (x) b with a, b in {-1, 0, 1}^2, |a|_inf = |b|_inf = 1, up
    to sign: 16 distinct directions, every one of rank one."""
    off = orc.r11_directions()
    assert off.shape == (16, 4)
    seen = set()
    for o in off:
        assert o[0] * o[3] - o[1] * o[2] == 0 and np.abs(o).max() == 1
        key = tuple(o) if tuple(o) > tuple(-o) else tuple(-o)
        assert key not in seen
        seen.add(key)
    # every admissible a (x) b is one of them up to sign
    vecs = [v for v in itertools.product((-1, 0, 1), repeat=2) if max(map(abs, v)) == 1]
    for a, b in itertools.product(vecs, vecs):
        r = np.outer(a, b).reshape(4)
        key = tuple(r) if tuple(r) > tuple(-r) else tuple(-r)
        assert key in seen


def test_convergence_history_of_the_sec61_nh_study(orc):
    """Figure fig:convergence (NH, R^1_1): the largest decrease per iteration
    on the 648,025-point grid of the Sec. 6.1 study.  With ln|det F| for
    det F < 0 (the reading of the grid study) the computed history follows
    the printed rows 2 .. 15: the first three within 1 %, every one within
    30 % (beta_k = 0.06 is printed rounded), and the iteration stops at the
    tolerance 1e-4 right after the last printed row.  Excluding det F <= 0
    instead gives a first decrease below 0.1, far from the printed 1.62."""
    mat = orc.Material(**NH61)
    g = orc.Grid.from_bounds((0.1, 3.4), (-2.55, 2.55), (0.15, 0.15))
    off = orc.r11_directions()
    _, _, decs = orc.grid_convexify(mat, g, BETA61, off, kmax=20, tol=1e-4, abs_det=True)
    assert len(decs) == len(PRINTED_NH_R11) + 1 and decs[-1] <= 1e-4
    rel = np.abs(np.array(decs[:-1]) - PRINTED_NH_R11) / np.array(PRINTED_NH_R11)
    assert rel[:3].max() < 0.01 and rel.max() < 0.3
    W0 = orc.grid_energy(mat, g, BETA61, abs_det=False)
    _, _, _, _, dec = orc.grid_step(g, off, W0)
    assert dec < 0.1


def _brute_step(g, off, W):
    """W^{k+1} by brute force: every pair of finite line points l- < 0 < l+
    (chord at 0), and the point itself."""
    n = g.n
    out = W.copy()
    idx = np.arange(g.count).reshape(n)
    for flat in range(g.count):
        i = np.array(np.unravel_index(flat, n))
        best = W[flat]
        if not np.isfinite(best):
            continue
        for o in off:
            pts = {}
            for l in range(-max(n), max(n) + 1):
                ii = i + l * o
                if np.all(ii >= 0) and np.all(ii < np.array(n)):
                    v = W[idx[tuple(ii)]]
                    if np.isfinite(v):
                        pts[l] = v
            for a, b in itertools.product([l for l in pts if l < 0], [l for l in pts if l > 0]):
                best = min(best, (b * pts[a] - a * pts[b]) / (b - a))
        out[flat] = best
    return out


def test_one_step_against_brute_force_hulls(orc):
    """A 4 x 3 x 3 x 4 grid around the identity, damage energy, three steps:
    Algorithm 1's hull value at every point equals the smallest chord over all
    pairs of line points on both sides (within rounding)."""
    mat = orc.Material(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3)
    g = orc.Grid((4, 3, 3, 4), (0.4, -0.6, -0.6, 0.4), (0.5, 0.6, 0.6, 0.5))
    off = orc.r11_directions()
    W = orc.grid_energy(mat, g, 0.06)
    for _ in range(3):
        Wn, d, lm, lp, dec = orc.grid_step(g, off, W)
        Wb = _brute_step(g, off, W)
        fin = np.isfinite(Wb)
        np.testing.assert_array_equal(np.isfinite(Wn), fin)
        assert np.max(np.abs(Wn[fin] - Wb[fin]) / (1 + np.abs(Wb[fin]))) < 1e-14
        assert np.all(Wn[fin] <= W[fin])
        split = d >= 0
        assert np.all((lm[split] < 0) & (lp[split] > 0)) and np.all(lm[~split] == 0)
        W = Wn


def test_double_well_grid_reaches_the_closed_form_in_one_step(orc):
    """Separable double well (F11^2 - 1)^2 + F12^2 + F21^2 + (F22 - 1)^2 on a
    grid with F11 = -1.5 .. 1.5 step 0.25 (the wells are grid points): the
    rank-one convex envelope replaces (F11^2 - 1)^2 by 0 on |F11| <= 1; one
    step along e1 (x) e1 reaches it exactly, the next changes nothing."""
    mat = orc.Material(energy=1)
    g = orc.Grid((13, 3, 3, 5), (-1.5, -0.25, -0.25, 0.5), (0.25, 0.25, 0.25, 0.25))
    off = orc.r11_directions()
    W0 = orc.grid_energy(mat, g, 0.0)
    W1, d, lm, lp, dec = orc.grid_step(g, off, W0)
    P = g.points()
    a = np.where(np.abs(P[:, 0]) <= 1.0, 0.0, (P[:, 0] ** 2 - 1.0) ** 2)
    exact = a + P[:, 1] ** 2 + P[:, 2] ** 2 + (P[:, 3] - 1.0) ** 2
    np.testing.assert_allclose(W1, exact, rtol=0, atol=1e-14)
    inner = np.abs(P[:, 0]) < 1.0
    assert np.all(d[inner] == 0)  # direction (1,0) (x) (1,0): offset (1, 0, 0, 0)
    np.testing.assert_array_equal(orc.r11_directions()[0], [1, 0, 0, 0])
    _, _, _, _, dec2 = orc.grid_step(g, off, W1)
    assert dec2 == 0.0


def test_converged_grid_is_rank_one_convex_and_trees_are_consistent(orc):
    """Damage energy on a 7 x 5 x 5 x 7 grid iterated until nothing changes:
    W^k never increases, the limit has nonnegative second differences along
    every direction of the set (discrete rank-one convexity), and at random
    points the tree of Algorithm 2 evaluated by Algorithm 3 gives the
    interpolated W^K, with leaf weights summing to one."""
    mat = orc.Material(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3)
    g = orc.Grid((7, 5, 5, 7), (0.4, -0.6, -0.6, 0.4), (0.2, 0.3, 0.3, 0.2))
    off = orc.r11_directions()
    W, forest, decs = orc.grid_convexify(mat, g, 0.06, off, kmax=40, tol=0.0, abs_det=True)
    assert decs[-1] == 0.0 and len(decs) < 40
    for a, b in zip(W[:-1], W[1:]):
        assert np.all(b <= a)
    Wk = W[-1].reshape(g.n)
    worst = 0.0
    for o in off:
        for flat in range(g.count):
            i = np.array(np.unravel_index(flat, g.n))
            lo, hi = i - o, i + o
            nn = np.array(g.n)
            if np.all((lo >= 0) & (lo < nn) & (hi >= 0) & (hi < nn)):
                worst = min(worst, Wk[tuple(lo)] + Wk[tuple(hi)] - 2 * Wk[tuple(i)])
    assert worst > -1e-13
    rng = np.random.default_rng(4)
    P = g.points()
    F = rng.uniform(P.min(0), P.max(0), size=(64, 4))
    wi, wt, Pq, nl = orc.grid_query(mat, g, 0.06, off, W[-1], forest, F, abs_det=True)
    np.testing.assert_allclose(wt, wi, rtol=1e-13, atol=1e-13)
    assert np.all(nl >= 1)
    # a grid point that never split is its own leaf: P is the stress there
    detP = P[:, 0] * P[:, 3] - P[:, 1] * P[:, 2]
    never = np.nonzero(np.all(orc.forest_array(forest)[:, :, 0] < 0, axis=0) & (detP > 0))[0]
    q = never[0]
    _, _, Pg, nlg = orc.grid_query(mat, g, 0.06, off, W[-1], forest, P[q:q + 1], abs_det=True)
    assert nlg[0] == 1
    np.testing.assert_allclose(Pg[0], orc.stress(mat, P[q], 0.06), rtol=1e-14)
