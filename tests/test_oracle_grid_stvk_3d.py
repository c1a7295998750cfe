"""Pins of the oracle's St. Venant-Kirchhoff energy (Eq. 2.2) and of the
three-dimensional global-grid study (Sec. 6.8, Table tab:3Dconvexification):
closed forms of the invariants and of Eq. (2.2), stresses by central
differences, the 169 directions of R^1_1 for d = 3 (Eq. 5.1), brute-force
chords on a small nine-dimensional grid, the printed STVK convergence history
of Sec. 6.1 and the printed bi- and triaxial relaxed curves of Sec. 6.8."""
import itertools

import numpy as np
import pytest

from conftest import load_golden

MAT = dict(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3)  # Tables tab:2Dconvexification / tab:3Dconvexification
# Figure fig:convergence, STVK, R^1_1 column, rows k = 3 .. 11 (rows 1 and 2,
# 1000.00 and 1000.04, carry the paper's starting value 1000; see the reading)
PRINTED_STVK_R11 = [0.18478, 0.07939, 0.01625, 0.00237, 0.00132, 0.00075, 0.00045, 0.00037,
                    0.00014]


def _mat(orc, energy):
    return orc.Material(MAT["mu"], MAT["lam"], MAT["Dinf"], MAT["D0"], energy=energy)


def _embed(F):
    """F in R^{2x2} as the plane-strain 3 x 3 deformation."""
    G = np.eye(3)
    G[:2, :2] = np.asarray(F).reshape(2, 2)
    return G


def _random_F(rng, d, n=20):
    out = []
    while len(out) < n:
        F = np.eye(d) + 0.35 * rng.standard_normal((d, d))
        if np.linalg.det(F) > 0.2:
            out.append(F)
    return out


def test_invariants_and_stvk_closed_forms(orc):
    """I1 = tr C, I2 = (I1^2 - tr C^2) / 2 (the sum of the principal minors of
    C), J = det F, plane strain through the 3 x 3 embedding; Eq. (2.2) equals
    the textbook form lam/2 (tr E)^2 + mu tr E^2, E = (C - 1)/2; both
    energies vanish at F = 1."""
    rng = np.random.default_rng(0)
    for d in (2, 3):
        for F in _random_F(rng, d):
            G = _embed(F) if d == 2 else F
            C = G.T @ G
            I1, I2, J = orc.invariants(F)
            assert abs(I1 - np.trace(C)) < 1e-13
            assert abs(I2 - 0.5 * (np.trace(C) ** 2 - np.trace(C @ C))) < 1e-12
            assert abs(J - np.linalg.det(F)) < 1e-13
            E = 0.5 * (C - np.eye(3))
            ref = 0.5 * MAT["lam"] * np.trace(E) ** 2 + MAT["mu"] * np.trace(E @ E)
            assert abs(orc.psi0_stvk(I1, I2, MAT["mu"], MAT["lam"]) - ref) < 1e-12
    assert orc.psi0_stvk(3.0, 3.0, 1.0, 0.5) == 0.0
    assert orc.energy_dim(_mat(orc, 2), np.eye(3), 0.0) == 0.0
    assert orc.energy_dim(_mat(orc, 0), np.eye(3), 0.0) == 0.0


@pytest.mark.parametrize("energy,d", [(2, 2), (2, 3), (0, 3), (0, 2)])
def test_stresses_are_derivatives_of_the_energies(orc, energy, d):
    """P = dW/dF (Eq. 2.12) for Eq. (2.2) in plane strain and in 3-D and for
    Eq. (2.3) in 3-D: central differences of W, with beta_k below and above
    psi0 (damage loading and unloading)."""
    rng = np.random.default_rng(1 + energy + d)
    mat = _mat(orc, energy)
    h = 1e-6
    for F in _random_F(rng, d, 8):
        f = F.reshape(-1)
        I1, I2, J = orc.invariants(f)
        s = orc.psi0_stvk(I1, I2, MAT["mu"], MAT["lam"]) if energy == 2 else orc.psi0_nh(
            I1, J, MAT["mu"], MAT["lam"])
        for beta in (0.5 * s, 2.0 * s + 0.1):
            P = orc.stress_dim(mat, f, beta)
            fd = np.zeros_like(f)
            for c in range(f.size):
                e = np.zeros_like(f)
                e[c] = h
                fd[c] = (orc.energy_dim(mat, f + e, beta) - orc.energy_dim(mat, f - e, beta)) / (2 * h)
            assert np.max(np.abs(P - fd)) < 1e-7 * (1 + np.max(np.abs(P)))
    if energy == 2 and d == 2:  # the per-point energy and stress are the same functions
        F = _random_F(rng, 2, 1)[0].reshape(-1)
        assert orc.energy(mat, F, 0.1) == orc.energy_dim(mat, F, 0.1)
        assert np.array_equal(orc.stress(mat, F, 0.1), orc.stress_dim(mat, F, 0.1))


def test_r11_for_three_dimensions(orc):
    """Eq. (5.1) with d = 3: a (x) b, a, b in {-1, 0, 1}^3, |a|_inf = |b|_inf = 1,
    up to sign: 169 distinct rank-one directions, and every admissible a (x) b
    is one of them up to sign."""
    off = orc.r11_directions(3)
    assert off.shape == (169, 9)
    seen = set()
    for o in off:
        assert np.linalg.matrix_rank(o.reshape(3, 3)) == 1 and np.abs(o).max() == 1
        key = tuple(o) if tuple(o) > tuple(-o) else tuple(-o)
        assert key not in seen
        seen.add(key)
    vecs = [v for v in itertools.product((-1, 0, 1), repeat=3) if max(map(abs, v)) == 1]
    for a, b in itertools.product(vecs, vecs):
        r = np.outer(a, b).reshape(9)
        key = tuple(r) if tuple(r) > tuple(-r) else tuple(-r)
        assert key in seen


def test_nine_dimensional_step_against_brute_force_chords(orc):
    """A 3^3 x 2^6 grid around the identity (3-D NH), two steps: at every
    point the value of Algorithm 1's hull equals the smallest chord over all
    pairs of line points on both sides, along the 169 directions."""
    mat = _mat(orc, 0)
    n = (3, 2, 2, 2, 3, 2, 2, 2, 3)
    lo = (0.7, -0.1, -0.1, -0.1, 0.7, -0.1, -0.1, -0.1, 0.7)
    de = (0.4, 0.2, 0.2, 0.2, 0.4, 0.2, 0.2, 0.2, 0.4)
    g = orc.Grid(n, lo, de)
    off = orc.r11_directions(3)
    W = orc.grid_energy(mat, g, 0.05)
    idx = np.array(np.unravel_index(np.arange(g.count), n)).T
    nn = np.array(n)
    for _ in range(2):
        Wn, d, lm, lp, dec = orc.grid_step(g, off, W)
        best = W.copy()
        for o in off:
            pts = {}
            for l in (-2, -1, 1, 2):
                ii = idx + l * o
                ok = np.all((ii >= 0) & (ii < nn), axis=1)
                v = np.full(g.count, np.nan)
                v[ok] = W[np.ravel_multi_index(ii[ok].T, n)]
                pts[l] = v
            for a, b in itertools.product((-2, -1), (1, 2)):
                ch = (b * pts[a] - a * pts[b]) / (b - a)
                m = np.isfinite(ch)
                best[m] = np.minimum(best[m], ch[m])
        assert np.max(np.abs(Wn - best) / (1 + np.abs(best))) < 1e-14
        assert np.all(Wn <= W)
        W = Wn


@pytest.mark.slow
def test_stvk_convergence_history_of_the_sec61_study(orc):
    """Figure fig:convergence (STVK, R^1_1) on the 672,400-point grid of Table
    tab:2Dconvexification (delta 0.1, diagonal [0.1, 2.0], off-diagonal
    [-2.0, 2.0], beta_k 0.07) with Eq. (2.2) kept where det F <= 0 (it is a
    polynomial): the run takes the printed number of steps (11), and steps
    2 .. 10 follow the printed rows 3 .. 11, the first three within 5 %, all
    within 15 % (beta_k is printed rounded).  Excluding det F <= 0 instead
    ends after 10 steps with a first decrease of 0.12."""
    mat = _mat(orc, 2)
    g = orc.Grid.from_bounds((0.1, 2.0), (-2.0, 2.0), (0.1, 0.1))
    assert g.count == 672400
    off = orc.r11_directions()
    _, _, decs = orc.grid_convexify(mat, g, 0.07, off, kmax=20, tol=1e-4, rule=1,
                                    keep_all=False)
    assert len(decs) == 11 and decs[-1] <= 1e-4 and decs[-2] > 1e-4
    rel = np.abs(np.array(decs[1:10]) - PRINTED_STVK_R11) / np.array(PRINTED_STVK_R11)
    assert rel[:3].max() < 0.05 and rel.max() < 0.15
    _, _, decs0 = orc.grid_convexify(mat, g, 0.07, off, kmax=20, tol=1e-4, rule=0,
                                     keep_all=False)
    assert len(decs0) == 10 and decs0[0] < 0.13


def _fit_beta(orc, mat, W_identity):
    lo, hi = 1e-9, 1.0
    f = lambda b: orc.energy(mat, [1, 0, 0, 1], b) - W_identity  # noqa: E731
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (f(lo) > 0) == (f(mid) > 0):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.slow
def test_3d_study_reproduces_the_printed_relaxed_curves(orc):
    """Sec. 6.8 (figure 3dconvexification-lines): the nine-dimensional grid of
    Table tab:3Dconvexification (NH; diagonal [1.0, 3.4], off-diagonal
    [-0.15, 0.15], delta 0.15: 3,581,577 points), R^1_1 for d = 3, tol 1e-4.
    W^0 at the path points equals the printed unrelaxed curves; W^K at
    diag(s, s, 1) and diag(s, s, s) equals the printed relaxed curves within
    1e-5 (exactly, 1e-14, where the paper's curve is not relaxed), after the
    5 steps the stopping rule takes."""
    g = load_golden("nh3d_paths.txt")
    mat = _mat(orc, 0)
    beta = _fit_beta(orc, mat, g[0, 1])
    G = orc.Grid.from_bounds((1.0, 3.4), (-0.15, 0.15), (0.15, 0.15), dim=3)
    assert G.count == 3581577
    st = np.ones(9, dtype=np.int64)
    for c in range(7, -1, -1):
        st[c] = st[c + 1] * G.n[c + 1]
    bi = np.array([np.dot([k, 1, 1, 1, k, 1, 1, 1, 0], st) for k in range(17)])
    tri = np.array([np.dot([k, 1, 1, 1, k, 1, 1, 1, k], st) for k in range(17)])
    W, _, decs = orc.grid_convexify(mat, G, beta, orc.r11_directions(3), kmax=20, tol=1e-4,
                                    keep_all=False)
    assert np.max(np.abs(W[0][bi] - g[:, 3])) < 1e-14
    assert np.max(np.abs(W[0][tri] - g[:, 5])) < 1e-14
    assert len(decs) == 5 and decs[-1] <= 1e-4
    for col, ix in ((4, bi), (6, tri)):
        err = np.abs(W[-1][ix] - g[:, col])
        assert err.max() < 1e-5
        flat = g[:, col] == g[:, col - 1]  # printed as not relaxed
        assert flat.sum() >= 8 and err[flat].max() < 1e-14


@pytest.mark.parametrize("energy,d,rule", [(0, 2, 0), (0, 2, 1), (2, 2, 1), (2, 3, 0), (0, 3, 0),
                                           (1, 2, 0)])
def test_tangents_are_derivatives_of_the_stresses(orc, energy, d, rule):
    """A = dP/dF (Algorithm 3's third output) for Eq. (2.3) (with ln|det F|
    under rule 1, det F < 0 included), Eq. (2.2) and the double well, in two
    and three dimensions: central differences of P, symmetric, with beta_k
    below and above psi0; in plane strain the NH tangent equals the
    per-point oracle's."""
    rng = np.random.default_rng(10 + 3 * energy + d + rule)
    mat = _mat(orc, energy)
    h = 1e-6
    Fs = _random_F(rng, d, 6)
    if rule == 1:  # mirror images with det F < 0
        Fs += [np.diag([-1.0] + [1.0] * (d - 1)) @ F for F in Fs[:3]]
    for F in Fs:
        f = F.reshape(-1)
        for beta in (0.01, 3.0):
            A = orc.tangent_dim(mat, f, beta, rule)
            fd = np.zeros_like(A)
            for c in range(f.size):
                e = np.zeros_like(f)
                e[c] = h
                fd[:, c] = (orc.stress_dim(mat, f + e, beta, rule) -
                            orc.stress_dim(mat, f - e, beta, rule)) / (2 * h)
            assert np.max(np.abs(A - fd)) < 2e-6 * (1 + np.max(np.abs(A)))
            assert np.max(np.abs(A - A.T)) < 1e-12 * (1 + np.max(np.abs(A)))
            if energy in (0, 1) and d == 2 and np.linalg.det(F) > 0:
                np.testing.assert_allclose(A, orc.tangent(mat, f, beta), rtol=1e-12, atol=1e-12)


def test_query_tangent_is_the_leaf_tangent_and_symmetric(orc):
    """Algorithm 3's tangent over the tree: a grid point that no iteration
    split is its own leaf (A = the tangent there); at random points A is
    symmetric and, where every corner's tree is a leaf, the interpolation of
    the corner tangents."""
    mat = orc.Material(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3)
    g = orc.Grid((7, 5, 5, 7), (0.4, -0.6, -0.6, 0.4), (0.2, 0.3, 0.3, 0.2))
    off = orc.r11_directions()
    W, forest, decs = orc.grid_convexify(mat, g, 0.06, off, kmax=40, tol=0.0, abs_det=True)
    P = g.points()
    fa = orc.forest_array(forest)
    detP = P[:, 0] * P[:, 3] - P[:, 1] * P[:, 2]
    never = np.nonzero(np.all(fa[:, :, 0] < 0, axis=0) & (detP > 0))[0]
    q = never[:8]
    _, _, _, nl, A = orc.grid_query(mat, g, 0.06, off, W[-1], forest, P[q], abs_det=True,
                                    want_A=True)
    assert np.all(nl == 1)
    for k, i in enumerate(q):
        np.testing.assert_allclose(A[k], orc.tangent_dim(mat, P[i], 0.06, 1), rtol=1e-14,
                                   atol=1e-14)
    rng = np.random.default_rng(3)
    F = rng.uniform(P.min(0), P.max(0), size=(32, 4))
    _, _, _, _, A = orc.grid_query(mat, g, 0.06, off, W[-1], forest, F, abs_det=True,
                                   want_A=True)
    assert np.max(np.abs(A - np.transpose(A, (0, 2, 1)))) < 1e-12
