"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of the expected values comes from
the CUDA path: they are the paper's printed numbers (tests/golden, cited in the
file headers), closed forms, invariants or brute force on tiny inputs.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import load_golden

# Material of Tables tab:biaxialperturbation / tab:3Dconvexification (NH rows).
MU, LAM, D0, DINF = 1.0, 0.5, 0.3, 0.9


def _fit_beta(orc, mat, W_identity):
    """beta_k is not printed (or printed rounded): fit it from W(I) = -(1 - D_k) beta_k
    by bisection (W(I) is monotone in beta_k)."""
    lo, hi = 1e-9, 1.0
    f = lambda b: orc.energy(mat, [1, 0, 0, 1], b) - W_identity  # noqa: E731
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (f(lo) > 0) == (f(mid) > 0):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_energy_2d_printed_lines(orc):
    """Eq. (2.9), plane strain: the printed W along diag(s, 1) and diag(s, s)
    (Sec. 6.6, NH biaxial figures) with one fitted constant beta_k."""
    g = load_golden("nh2d_biaxial_lines.txt")
    mat = orc.Material(MU, LAM, DINF, D0)
    beta = _fit_beta(orc, mat, g[0, 1])
    for s, w1, _, w2, _ in g[1:]:
        assert abs(orc.energy(mat, [s, 0, 0, 1], beta) - w1) < 1e-14
        assert abs(orc.energy(mat, [s, 0, 0, s], beta) - w2) < 1e-14


def test_energy_3d_printed_paths(orc):
    """Eq. (2.9) in 3-D invariants along the uni/bi/triaxial paths of Sec. 6.8
    (figure 3dconvexification-lines).  Uniaxial diag(s,1,1) and biaxial
    diag(s,s,1) coincide with plane strain diag(s,1), diag(s,s); triaxial uses
    I1 = 3 s^2, J = s^3 in Eq. (2.3).  The fitted beta_k must round to the
    printed 0.0625 (Table tab:3Dconvexification)."""
    g = load_golden("nh3d_paths.txt")
    mat = orc.Material(MU, LAM, DINF, D0)
    beta = _fit_beta(orc, mat, g[0, 1])
    assert abs(beta - 0.0625) < 5e-5
    for s, wu, _, wb, _, wt, _ in g:
        assert abs(orc.energy(mat, [s, 0, 0, 1], beta) - wu) < 1e-14
        assert abs(orc.energy(mat, [s, 0, 0, s], beta) - wb) < 1e-14
        psi = orc.psi0_nh(3 * s * s, s ** 3, MU, LAM)
        assert abs(orc.W_of_psi0(psi, beta, DINF, D0) - wt) < 1e-14


def test_alg1_reproduces_printed_uniaxial_hull(orc):
    """Algorithm 1 on the printed uniaxial W samples gives the printed relaxed
    curve (the uniaxial path is a rank-one line, Sec. 6.8)."""
    g = load_golden("nh3d_paths.txt")
    x, w, wrc = g[:, 0], g[:, 1], g[:, 2]
    v = orc.lower_hull(x, w)
    assert list(np.round(x[v], 2)) == [1.0, 1.15, 3.1, 3.25, 3.4]
    interp = np.interp(x, x[v], w[v])
    # the printed curve carries ~1e-12 of the paper's own interpolation noise
    assert np.max(np.abs(interp - wrc)) < 5e-12


def test_line_scan_reproduces_printed_rank_one_relaxation(orc):
    """Per-point line scan (Eq. 4.4 + Alg. 1 + value at l = 0) along e1 (x) e1
    on the grid delta = 0.15, F11 in [1.0, 3.4] gives the printed W^15 on the
    rank-one line diag(s, 1) (Sec. 6.6).  Beyond the grid the paper's values
    are unrelaxed."""
    g = load_golden("nh2d_biaxial_lines.txt")
    mat = orc.Material(MU, LAM, DINF, D0)
    beta = _fit_beta(orc, mat, g[0, 1])
    R = np.array([1.0, 0.0, 0.0, 0.0])
    half = 16
    L = 2 * half + 1
    worst = 0.0
    for s, w_plain, w15, _, _ in g:
        if s > 3.4 + 1e-9:
            assert abs(w15 - w_plain) < 1e-14
            continue
        w, valid = orc.sample_line(mat, [s, 0, 0, 1], beta, R, L, 0.15 * half)
        f11 = s + 0.15 * (np.arange(L) - half)
        valid &= (f11 > 1.0 - 1e-9) & (f11 < 3.4 + 1e-9)
        h, mm, mp, _ = orc.line_bridge(w, valid)
        worst = max(worst, abs(h - w15))
    assert worst < 1e-9


def _brute_vertices(x, w):
    """Strict lower-hull vertices by definition: the end points, and every k
    that lies strictly below every chord (i, j) with i < k < j."""
    n = len(x)
    out = []
    for k in range(n):
        ok = True
        for i in range(k):
            for j in range(k + 1, n):
                chord = (w[i] * (x[j] - x[k]) + w[j] * (x[k] - x[i])) / (x[j] - x[i])
                if not w[k] < chord:
                    ok = False
                    break
            if not ok:
                break
        if ok:
            out.append(k)
    return out


@pytest.mark.parametrize("seed", range(40))
def test_alg1_matches_brute_force_vertices(orc, seed):
    """Algorithm 1 returns exactly the strict lower-hull vertices (O(n^3) brute
    force).  Small integer values make collinear triples frequent, so the ">="
    pop rule is exercised; the arithmetic is exact."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 25))
    x = np.sort(rng.choice(np.arange(-30, 31), size=n, replace=False)).astype(float)
    w = rng.integers(-4, 5, size=n).astype(float)
    assert list(orc.lower_hull(x, w)) == _brute_vertices(x, w)


def test_hull_arrays_are_convex_minorants(orc):
    """Every hull array of Algorithm 1 on sampled NH lines, interpolated on the
    whole grid: below the samples, equal to them at its vertices, with
    nonnegative second differences (a convex minorant)."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(20, seed=12, lam_hi=1.8)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(6, 6)
    rng = np.random.default_rng(4)
    lines = 0
    for p in range(20):
        for j in rng.choice(36, 6, replace=False):
            w, v = orc.sample_line(mat, F[p], beta[p], orc.rank_one(dirs[j]), 161, 0.6)
            idx = np.nonzero(v)[0]
            x = idx.astype(np.float64)
            wv = w[idx]
            vt = orc.lower_hull(x, wv)
            hull = np.interp(x, x[vt], wv[vt])
            scale = np.max(np.abs(wv))
            assert np.all(hull <= wv + 1e-13 * scale)
            np.testing.assert_array_equal(hull[vt], wv[vt])
            d2 = hull[2:] - 2 * hull[1:-1] + hull[:-2]
            assert np.all(d2 >= -1e-13 * scale), d2.min()
            assert vt[0] == 0 and vt[-1] == len(x) - 1
            lines += 1
    assert lines == 120


@pytest.mark.parametrize("seed", range(40))
def test_bridge_is_min_over_pairs(orc, seed):
    """Value of the hull at x = 0 equals min(w_0, min over pairs a < 0 < b of
    the chord at 0) (Caratheodory in 1-D); the bridge vertices attain it."""
    rng = np.random.default_rng(1000 + seed)
    L = int(rng.integers(1, 21)) * 2 + 1
    m0 = (L - 1) // 2
    w = rng.normal(size=L) + 0.02 * (np.arange(L) - m0) ** 2
    valid = rng.random(L) > 0.2
    valid[m0] = True
    h, mm, mp, margin = orc.line_bridge(w, valid)
    best = w[m0]
    for a in range(m0):
        for b in range(m0 + 1, L):
            if valid[a] and valid[b]:
                xa, xb = a - m0, b - m0
                best = min(best, (xb * w[a] - xa * w[b]) / (xb - xa))
    assert abs(h - best) < 1e-12
    if mm != mp:
        xa, xb = mm - m0, mp - m0
        assert abs((xb * w[mm] - xa * w[mp]) / (xb - xa) - best) < 1e-12
        assert margin >= 0
    else:
        assert mm == m0 and abs(best - w[m0]) < 1e-12


def test_margin_certifies_decision(orc):
    """The bridge margin is a certificate: perturbing each sample by less than
    it never changes the bridge (random perturbations, many trials)."""
    rng = np.random.default_rng(7)
    L = 41
    m0 = 20
    checked = 0
    for trial in range(200):
        w = rng.normal(size=L) * 0.3 + 0.01 * (np.arange(L) - m0) ** 2
        h, mm, mp, margin = orc.line_bridge(w)
        if not (0 < margin < 10):
            continue
        for _ in range(20):
            d = rng.uniform(-0.999, 0.999, size=L) * margin
            _, mm2, mp2, _ = orc.line_bridge(w + d)
            assert (mm2, mp2) == (mm, mp)
        checked += 1
    assert checked > 50


def _dw_scan(orc, Na=8, L=301, t_half=1.5, depth=1):
    return orc.Scan(orc.angle_directions(Na, Na), L, t_half, depth)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_double_well_closed_form_at_origin(orc, depth):
    """Double well W = (F11^2-1)^2 + F12^2 + F21^2 + (F22-1)^2: at F = diag(0, 1)
    the rank-one convex envelope is 0, reached by the laminate diag(+-1, 1) with
    xi = 1/2 along e1 (x) e1 (direction 0), and P = 0 for every depth."""
    mat = orc.Material(energy=1)
    sc = _dw_scan(orc, depth=depth)
    WR, P, tree, st = orc.convexify(mat, sc, np.array([[0.0, 0, 0, 1]]), np.zeros(1))
    assert abs(WR[0]) < 1e-15 and np.max(np.abs(P[0])) < 1e-12
    root = tree[0, 0]
    assert root["dir"] == 0 and root["flags"] & orc.LAMINATED
    assert abs(root["xi"] - 0.5) < 1e-15
    np.testing.assert_allclose(tree[0, 1]["F"], [-1, 0, 0, 1], atol=1e-14)
    np.testing.assert_allclose(tree[0, 2]["F"], [1, 0, 0, 1], atol=1e-14)


def test_double_well_separable_envelope(orc):
    """Closed form away from the origin: for |F11| <= 1 on the line grid,
    W^rc = F12^2 + F21^2 + (F22 - 1)^2 (convex envelope of the separable double
    well, both wells inside the line window); for |F11| > 1 the point is on the
    convex part and W^R = W."""
    mat = orc.Material(energy=1)
    sc = _dw_scan(orc, depth=2)
    F = np.array([[0.3, 0.1, -0.2, 1.2], [-0.4, 0.0, 0.05, 0.9], [1.2, 0.1, 0.0, 1.0]])
    WR, P, tree, st = orc.convexify(mat, sc, F, np.zeros(3))
    rest = F[:, 1] ** 2 + F[:, 2] ** 2 + (F[:, 3] - 1) ** 2
    assert abs(WR[0] - rest[0]) < 1e-12 and abs(WR[1] - rest[1]) < 1e-12
    assert abs(WR[2] - orc.energy(mat, F[2], 0.0)) < 1e-12


def test_stress_is_gradient_of_energy(orc):
    """Eq. (2.12): P = dW/dF against central differences of Eq. (2.9), on both
    branches of the history (s < beta_k and s > beta_k); P(I) = 0."""
    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    rng = np.random.default_rng(3)
    for trial in range(60):
        F = np.array([1, 0, 0, 1.0]) + rng.normal(0, 0.25, 4)
        if F[0] * F[3] - F[1] * F[2] < 0.3:
            continue
        beta = rng.choice([0.0, 0.05, 0.4, 3.0])
        P = orc.stress(mat, F, beta)
        s = orc.psi0_F(mat, F)
        e = 1e-6
        for k in range(4):
            Fp, Fm = F.copy(), F.copy()
            Fp[k] += e
            Fm[k] -= e
            if (orc.psi0_F(mat, Fp) - beta) * (orc.psi0_F(mat, Fm) - beta) < 0:
                continue  # kink of max(s, beta_k) inside the stencil
            fd = (orc.energy(mat, Fp, beta) - orc.energy(mat, Fm, beta)) / (2 * e)
            assert abs(fd - P[k]) < 1e-7 * max(1.0, abs(P[k])), (F, beta, k, fd, P[k], s)
    assert np.max(np.abs(orc.stress(mat, [1, 0, 0, 1], 0.2))) < 1e-15


def test_tangent_is_gradient_of_stress(orc):
    """A = dP/dF against central differences of the (pinned) stress, on both
    history branches; A is symmetric (a Hessian); double well exactly."""
    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    rng = np.random.default_rng(5)
    checked = 0
    for trial in range(60):
        F = np.array([1, 0, 0, 1.0]) + rng.normal(0, 0.25, 4)
        if F[0] * F[3] - F[1] * F[2] < 0.3:
            continue
        beta = rng.choice([0.0, 0.05, 0.4, 3.0])
        A = orc.tangent(mat, F, beta)
        np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-13 * max(1.0, np.max(np.abs(A))))
        e = 1e-6
        for k in range(4):
            Fp, Fm = F.copy(), F.copy()
            Fp[k] += e
            Fm[k] -= e
            if (orc.psi0_F(mat, Fp) - beta) * (orc.psi0_F(mat, Fm) - beta) < 0:
                continue
            fd = (orc.stress(mat, Fp, beta) - orc.stress(mat, Fm, beta)) / (2 * e)
            assert np.max(np.abs(fd - A[:, k])) < 1e-6 * max(1.0, np.max(np.abs(A))), (F, beta, k)
            checked += 1
    assert checked > 100
    dw = orc.Material(energy=1)
    F = np.array([0.7, 0.2, -0.1, 1.3])
    np.testing.assert_allclose(orc.tangent(dw, F, 0.0),
                               np.diag([12 * 0.49 - 4, 2.0, 2.0, 2.0]), rtol=1e-15, atol=0)


def test_newton_split_is_the_exact_common_tangent_of_the_double_well(orc):
    """Double well along e1 (x) e1 from F = diag(0.3, 1): the common tangent of
    (x^2 - 1)^2 touches at x = +-1, i.e. t- = -1.3, t+ = 0.7, neither on the
    line grid (h = 0.015); the refined split lands there, W^R = 0 and
    xi = 1.3 / 2."""
    mat = orc.Material(energy=1)
    F = np.array([[0.3, 0.0, 0.0, 1.0]])
    grid = orc.Scan(orc.angle_directions(8, 8), 201, 1.5, 1)
    WRg, _, trg, _ = orc.convexify(mat, grid, F, np.zeros(1))
    assert WRg[0] > 1e-6 and not trg[0, 0]["flags"] & orc.NEWTON
    sc = orc.Scan(orc.angle_directions(8, 8), 201, 1.5, 1, newton=True)
    WR, P, tr, st = orc.convexify(mat, sc, F, np.zeros(1))
    root = tr[0, 0]
    assert root["dir"] == 0 and root["flags"] & orc.NEWTON
    np.testing.assert_allclose(tr[0, 1]["F"], [-1, 0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(tr[0, 2]["F"], [1, 0, 0, 1], atol=1e-12)
    assert abs(root["xi"] - 0.65) < 1e-12
    assert abs(WR[0]) < 1e-13 and np.max(np.abs(P[0])) < 1e-11
    assert WR[0] <= WRg[0]


def test_newton_split_satisfies_tangency_by_differences(orc):
    """NH with damage: at every refined split the line function's slope at
    both ends (central differences of W alone) equals the chord slope, and the
    refined chord value at 0 is not above the grid bridge's."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(24, seed=11, lam_hi=1.8)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(12, 12)
    # with this damage law the tangent points lie near |t| = 7..10, so the
    # window must reach beyond them for a split to be interior
    g = orc.Scan(dirs, 301, 12.0, 1)
    sc = orc.Scan(dirs, 301, 12.0, 1, newton=True)
    WRg, _, trg, _ = orc.convexify(mat, g, F, beta)
    WR, _, tr, _ = orc.convexify(mat, sc, F, beta)
    refined = 0
    for p in range(F.shape[0]):
        r = tr[p, 0]
        if not r["flags"] & orc.NEWTON:
            continue
        refined += 1
        R = np.outer(dirs[r["dir"], :2], dirs[r["dir"], 2:]).reshape(4)
        k = np.argmax(np.abs(R))
        tm = (tr[p, 1]["F"][k] - F[p, k]) / R[k]
        tp = (tr[p, 2]["F"][k] - F[p, k]) / R[k]
        gfun = lambda t: orc.energy(mat, F[p] + t * R, beta[p])  # noqa: E731
        slope = (gfun(tp) - gfun(tm)) / (tp - tm)
        e = 1e-6
        for t in (tm, tp):
            d = (gfun(t + e) - gfun(t - e)) / (2 * e)
            assert abs(d - slope) < 1e-6 * max(1.0, abs(slope)), (p, t, d, slope)
        assert r["h"] <= trg[p, 0]["h"] + 1e-15
        assert WR[p] <= WRg[p] + 1e-15
        assert abs(r["xi"] - (0 - tm) / (tp - tm)) < 1e-12
    assert refined >= 5


def test_undamaged_neo_hooke_is_not_relaxed(orc):
    """With D_inf = 0, W = psi0 - beta_k is convex along every rank-one line
    where ln J <= 1 + mu/lam (second derivative along the line is
    mu|R|^2 + (c_J/J)^2 (mu + lam (1 - ln J)) >= 0), so W^R = W exactly."""
    mat = orc.Material(1.0, 5.0, 0.0, 0.5)
    F = np.array([[1.3, 0.1, -0.05, 0.9], [1.1, 0.0, 0.0, 1.1], [0.95, 0.2, 0.1, 1.05]])
    sc = orc.Scan(orc.angle_directions(8, 8), 101, 0.5, 2)
    for p in range(len(F)):
        for d in sc.dirs:
            R = orc.rank_one(d)
            t = np.linspace(-0.5, 0.5, 101)
            J = np.array([np.linalg.det((F[p] + ti * R).reshape(2, 2)) for ti in t])
            assert np.all(np.log(J[J > 0]) <= 1.0 + 1.0 / 5.0)
    WR, P, tree, st = orc.convexify(mat, sc, F, np.zeros(3))
    for p in range(3):
        assert WR[p] == orc.energy(mat, F[p], 0.0)
        assert not tree[p, 0]["flags"] & orc.LAMINATED


def _tree_leaves(orc, tr):
    leaves = []

    def rec(i):
        if tr[i]["flags"] & orc.LAMINATED:
            rec(2 * i + 1)
            rec(2 * i + 2)
        else:
            leaves.append(i)

    rec(0)
    return leaves


def test_tree_invariants_and_depth_chain(orc):
    """Lamination tree (Sec. 4.3, Alg. 2): leaves form an H_M sequence (Eq. 3.4):
    weights sum to 1, the weighted mean of the leaves is F, every split is
    rank-one and lies on the chosen line; and the depth chain
    W^R(K=3) <= W^R(K=2) <= W^R(K=1) <= W (Eq. 3.3)."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(16, seed=5)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(8, 8)
    prev = np.array([orc.energy(mat, F[p], beta[p]) for p in range(16)])
    for K in (1, 2, 3):
        sc = orc.Scan(dirs, 101, 0.5, K)
        WR, P, tree, st = orc.convexify(mat, sc, F, beta)
        assert np.all(WR <= prev + 1e-14)
        prev = WR
        for p in range(16):
            tr = tree[p]
            leaves = _tree_leaves(orc, tr)
            wsum = sum(tr[i]["weight"] for i in leaves)
            assert abs(wsum - 1.0) < 1e-14
            mean = sum(tr[i]["weight"] * tr[i]["F"] for i in leaves)
            np.testing.assert_allclose(mean, F[p], atol=1e-13)
            for i in range(len(tr)):
                if tr[i]["flags"] & orc.LAMINATED:
                    d = (tr[2 * i + 2]["F"] - tr[2 * i + 1]["F"]).reshape(2, 2)
                    assert abs(np.linalg.det(d)) < 1e-13
                    R = orc.rank_one(dirs[tr[i]["dir"]])
                    tp = (tr[i]["m_plus"] - sc.m0) * sc.h
                    np.testing.assert_allclose(tr[2 * i + 2]["F"], tr[i]["F"] + tp * R, atol=1e-14)
            Wsum = sum(tr[i]["weight"] * orc.energy(mat, tr[i]["F"], beta[p]) for i in leaves)
            assert abs(Wsum - WR[p]) < 1e-13


def _exact_lamination(orc, mat, dirs, L, t_half, K, F, beta):
    """Bottom-up discrete lamination by brute force on a tiny grid:
    W^0 = W, W^K(F) = min over R of hull_t[W^{K-1}(F + t_m R)](0)."""
    if K == 0:
        return orc.energy(mat, F, beta)
    m0 = (L - 1) // 2
    h = 2 * t_half / (L - 1)
    best = math.inf
    for d in dirs:
        R = orc.rank_one(d)
        w = np.full(L, np.nan)
        valid = np.zeros(L, dtype=bool)
        for m in range(L):
            G = F + (m - m0) * h * R
            if G[0] * G[3] - G[1] * G[2] > 0:
                valid[m] = True
                w[m] = _exact_lamination(orc, mat, dirs, L, t_half, K - 1, G, beta)
        hv, _, _, _ = orc.line_bridge(np.where(valid, w, 0.0), valid)
        best = min(best, hv)
    return best


def test_top_down_bounds_exact_lamination(orc):
    """Eq. (3.3) chain on tiny grids: W^2_exact <= V_2 <= V_1 = W^1_exact <= W,
    where V_K is the top-down per-point value and W^K_exact the bottom-up
    discrete lamination computed by brute force."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(6, seed=11, lam_lo=1.2, lam_hi=1.6)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(2, 2)
    L, t_half = 7, 0.5
    V = {}
    for K in (1, 2):
        V[K] = orc.convexify(mat, orc.Scan(dirs, L, t_half, K), F, beta)[0]
    for p in range(6):
        W = orc.energy(mat, F[p], beta[p])
        e1 = _exact_lamination(orc, mat, dirs, L, t_half, 1, F[p], beta[p])
        e2 = _exact_lamination(orc, mat, dirs, L, t_half, 2, F[p], beta[p])
        assert abs(V[1][p] - e1) < 1e-14
        assert e2 <= V[2][p] + 1e-14 and V[2][p] <= V[1][p] + 1e-14 and V[1][p] <= W + 1e-14


def test_history_update(orc):
    """Eq. (2.5): beta_new = max(beta_k, psi0(F))."""
    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F = np.array([[1.3, 0, 0, 1.0], [1.0, 0, 0, 1.0]])
    b = orc.history_update(mat, F, np.array([0.0, 0.3]))
    assert abs(b[0] - orc.psi0_F(mat, F[0])) < 1e-15 and b[1] == 0.3


def test_directions_cover_half_circle(orc):
    """Angle grid: a_i = (cos pi i/Na, sin pi i/Na), |a| = |b| = 1 (so |R|_F = 1),
    index j = i Nb + j."""
    d = orc.angle_directions(4, 3)
    assert d.shape == (12, 4)
    np.testing.assert_allclose(d[:, 0] ** 2 + d[:, 1] ** 2, 1.0, atol=1e-15)
    np.testing.assert_allclose(d[5], [math.cos(math.pi / 4), math.sin(math.pi / 4),
                                      math.cos(2 * math.pi / 3), math.sin(2 * math.pi / 3)])


def _stable(orc, t0, t1):
    """Same lamination decisions (directions, bridge indices, flags)."""
    return (np.array_equal(t0["dir"], t1["dir"]) and np.array_equal(t0["m_minus"], t1["m_minus"])
            and np.array_equal(t0["m_plus"], t1["m_plus"])
            and np.array_equal(t0["flags"], t1["flags"]))


def test_relaxed_stress_and_tangent_are_derivatives_of_the_relaxation(orc):
    """With the laminate fixed, W^R(F) = sum_leaves xi_path W(F + t_leaf R) (the
    leaves move with F), so P = dW^R/dF (Eq. 5.2, Algorithm 3) and the tree
    tangent A = dP/dF (the same recursion on second derivatives): central
    differences of the oracle's own W^R and P, at points whose decisions do
    not change under the perturbation, match P and A; A is symmetric and at
    depth 0 it is the tangent of W."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(24, seed=61, lam_hi=1.8)
    beta = orc.history_update(mat, Fp)
    sc = orc.Scan(orc.angle_directions(12, 12), 151, 0.5, 2)
    WR, P, tr, _ = orc.convexify(mat, sc, F, beta)
    A = orc.tree_tangent(mat, 2, tr, beta)
    np.testing.assert_allclose(A, np.transpose(A, (0, 2, 1)), rtol=1e-12, atol=1e-12)
    d = 1e-6
    checked = 0
    for p in range(F.shape[0]):
        if not tr[p, 0]["flags"] & orc.LAMINATED:
            continue
        ok = True
        dW, dP = np.zeros(4), np.zeros((4, 4))
        for k in range(4):
            Fs = np.repeat(F[p:p + 1], 2, axis=0)
            Fs[0, k] += d
            Fs[1, k] -= d
            W2, P2, t2, _ = orc.convexify(mat, sc, Fs, np.repeat(beta[p:p + 1], 2))
            if not (_stable(orc, t2[0], tr[p]) and _stable(orc, t2[1], tr[p])):
                ok = False
                break
            dW[k] = (W2[0] - W2[1]) / (2 * d)
            dP[:, k] = (P2[0] - P2[1]) / (2 * d)
        if not ok:
            continue
        np.testing.assert_allclose(dW, P[p], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(dP, A[p], rtol=1e-5, atol=1e-6)
        checked += 1
    assert checked >= 5
    sc0 = orc.Scan(orc.angle_directions(12, 12), 151, 0.5, 0)
    _, _, t0, _ = orc.convexify(mat, sc0, F[:4], beta[:4])
    A0 = orc.tree_tangent(mat, 0, t0, beta[:4])
    for p in range(4):
        np.testing.assert_array_equal(A0[p], orc.tangent(mat, F[p], beta[p]))


def test_adaptive_window_reaches_the_double_well_envelope(orc):
    """Adaptive line window (Sec. 4.1: the radius must be sufficiently large):
    the double well's split of F = diag(0, 1) has its ends at F11 = -1 and 1,
    outside a window of t_half = 0.25.  Without doublings the split ends on
    the line's ends and W^R > 0; with doublings allowed the window grows to
    t_half = 2 (the ends at t = +-1 are then interior samples, at 1 the ends
    would still be on the line's ends), and the result is the closed form:
    W^R = 0, F+- = diag(+-1, 1), xi = 1/2."""
    dw = orc.Material(energy=1)
    F = np.array([[0.0, 0.0, 0.0, 1.0]])
    sc0 = orc.Scan(orc.angle_directions(4, 4), 101, 0.25, 1)
    W0, _, t0, _ = orc.convexify(dw, sc0, F, np.zeros(1))
    assert t0[0, 0]["m_minus"] == 0 and t0[0, 0]["m_plus"] == 100 and W0[0] > 0.1
    sc = orc.Scan(orc.angle_directions(4, 4), 101, 0.25, 1, adaptive=5)
    W, P, t, _ = orc.convexify(dw, sc, F, np.zeros(1))
    r = t[0, 0]
    assert r["wexp"] == 3 and (r["m_minus"], r["m_plus"]) == (25, 75) and r["xi"] == 0.5
    assert abs(W[0]) < 1e-12 and np.max(np.abs(P[0])) < 1e-12
    np.testing.assert_allclose(t[0, 1]["F"], [-1, 0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(t[0, 2]["F"], [1, 0, 0, 1], atol=1e-12)
    assert t[0, 1]["wexp"] == 3  # children start from their parent's window


def test_adaptive_window_splits_are_interior_or_at_the_cap(orc):
    """NH with damage: with doublings allowed every split has both ends inside
    its line unless the node used all its doublings, and with none allowed
    (the default) the result is the plain method's."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(16, seed=81, lam_hi=1.8)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(8, 8)
    W0, _, t0, _ = orc.convexify(mat, orc.Scan(dirs, 101, 0.5, 2), F, beta)
    Wz, _, tz, _ = orc.convexify(mat, orc.Scan(dirs, 101, 0.5, 2, adaptive=0), F, beta)
    np.testing.assert_array_equal(W0, Wz)
    W, _, t, _ = orc.convexify(mat, orc.Scan(dirs, 101, 0.5, 2, adaptive=5), F, beta)
    lam = (t["flags"] & orc.LAMINATED) > 0
    assert lam.sum() >= 8
    edge = (t["m_minus"] == 0) | (t["m_plus"] == 100)
    assert np.all(~lam | ~edge | (t["wexp"] == 5))
    assert np.any(lam & (t["wexp"] > 0))
