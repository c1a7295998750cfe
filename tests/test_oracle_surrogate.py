"""Pins of the surrogate-proposed oracle (oracle/surrogate.py) against the
plain oracle (oracle.c): when every node falls back, or when a fixed network
proposes the full scan's own direction, the proposed form must reproduce the
plain method; the window enumerates (2w + 1)^2 wrapped grid cells."""
import math

import numpy as np
import pytest

from oracle import mlp
from oracle import surrogate as osur

MAT = (1.0, 5.0, 0.99, 0.5)


def _points(orc, n, seed):
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(*MAT)
    F, Fp = inputs.material_points(n, seed=seed)
    return mat, F, orc.history_update(mat, Fp)


def test_window_indices_wrap():
    idx = osur.window_indices(0, 7, 1, 8, 8)
    assert len(idx) == 9 and len(set(idx.tolist())) == 9
    rows = sorted({int(i) // 8 for i in idx})
    cols = sorted({int(i) % 8 for i in idx})
    assert rows == [0, 1, 7] and cols == [0, 6, 7]
    assert len(set(osur.window_indices(3, 3, 3, 7, 7).tolist())) == 49


def test_zero_tolerance_falls_back_everywhere_and_equals_plain(orc):
    """gap_tol = 0: every scanned node falls back, so the proposed form is the
    plain method node for node (W^R and P bit-identical)."""
    mat, F, beta = _points(orc, 10, 31)
    flat = mlp.init_params(2)
    mean, std = np.zeros(6), np.ones(6)
    WR, P, trees = osur.propose_convexify(orc, mat, 8, 8, 101, 0.5, 2, 1, 0.0, flat, mean, std,
                                          F, beta)
    sc = orc.Scan(orc.angle_directions(8, 8), 101, 0.5, 2)
    WRo, Po, tro, _ = orc.convexify(mat, sc, F, beta)
    np.testing.assert_allclose(WR, WRo, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(P, Po, rtol=1e-12, atol=1e-14)
    for t in trees:
        for rec in t.values():
            if rec["flags"] & orc.SCANNED:
                assert rec["flags"] & osur.FALLBACK


def _constant_net(theta_a, theta_b, xi, jump):
    parts = [np.zeros(s) for s in mlp.SHAPES]
    parts[9] = np.array([theta_a, theta_b, math.log(xi / (1 - xi)), *jump])
    return mlp.flatten(parts)


def test_window_around_the_true_direction_reproduces_the_full_scan(orc):
    """Depth 1: a network that outputs exactly the full scan's own laminate
    (angles of its direction, its xi and jump) centres the window on that
    direction, which is then the window's best and not on its border; the
    energy gap is zero, nothing falls back, and the result is the plain one."""
    mat, F, beta = _points(orc, 8, 32)
    Na = Nb = 12
    dirs = orc.angle_directions(Na, Nb)
    sc = orc.Scan(dirs, 151, 0.5, 1)
    WRo, Po, tro, _ = orc.convexify(mat, sc, F, beta)
    checked = 0
    for p in range(F.shape[0]):
        r = tro[p, 0]
        if not r["flags"] & orc.LAMINATED:
            continue
        d = int(r["dir"])
        jump = tro[p, 2]["F"] - tro[p, 1]["F"]
        flat = _constant_net(math.pi * (d // Nb) / Na, math.pi * (d % Nb) / Nb, r["xi"], jump)
        WR, P, trees = osur.propose_convexify(orc, mat, Na, Nb, 151, 0.5, 1, 2, 1e-9, flat,
                                              np.zeros(6), np.ones(6), F[p:p + 1], beta[p:p + 1])
        rec = trees[0][0]
        assert rec["center"] == (d // Nb, d % Nb)
        assert not rec["flags"] & osur.FALLBACK
        assert rec["dir"] == d and rec["gap"] < 1e-9
        assert WR[0] == WRo[p]
        np.testing.assert_array_equal(P[0], Po[p])
        checked += 1
    assert checked >= 4


def test_one_sided_gap_falls_back_on_a_subset(orc):
    """One-sided gap test: a node falls back on the border or when
    V - E_pred > gap_tol (1e-8 + |V|); its fallbacks are a subset of the
    two-sided test's, and a proposal that is worse than the window's value
    never falls back through the gap (a fixed network with a small jump;
    NaN proposals fall back in both modes)."""
    mat, F, beta = _points(orc, 8, 33)
    parts = [np.zeros(s) for s in mlp.SHAPES]
    parts[9] = np.array([0.3, 0.2, 0.0, 0.05, -0.04, 0.03, 0.02])
    flat = mlp.flatten(parts)
    kw = dict(Na=8, Nb=8, L=101, t_half=0.5, K=2, w=1, gap_tol=1e-6, flat=flat,
              mean=np.zeros(6), std=np.ones(6), F=F, beta=beta)
    _, _, t1 = osur.propose_convexify(orc, mat, one_sided=True, **kw)
    _, _, t2 = osur.propose_convexify(orc, mat, one_sided=False, **kw)
    seen = 0
    for a, b in zip(t1, t2):
        r1, r2 = a[0], b[0]  # the roots see the same proposal in both modes
        fb1, fb2 = bool(r1["flags"] & osur.FALLBACK), bool(r2["flags"] & osur.FALLBACK)
        assert not fb1 or fb2
        g = r1["gap"]
        gd, (ia, ib) = r1["window_dir"], r1["center"]
        border = bool(r1["window_lam"]) and (abs(osur._offset(gd // 8, ia, 8)) >= 1 or
                                             abs(osur._offset(gd % 8, ib, 8)) >= 1)
        if np.isfinite(g):
            assert fb1 == (g > 1e-6 or border)
            if g < 0:
                assert fb1 == border
                seen += 1
    assert seen >= 1


def test_recentring_walks_to_the_full_scan_direction(orc):
    """A fixed network proposing a cell several cells away from the full
    scan's direction, window half-width 1: without re-centring the window's
    best lies on its border and the node falls back; with enough re-centrings
    the window walks to the full scan's direction (a local descent over the
    angle grid), does not fall back, and the result is the plain method's."""
    mat, F, beta = _points(orc, 12, 36)
    Na = Nb = 12
    sc = orc.Scan(orc.angle_directions(Na, Nb), 151, 0.5, 1)
    WRo, Po, tro, _ = orc.convexify(mat, sc, F, beta)
    walked = 0
    for p in range(F.shape[0]):
        r = tro[p, 0]
        if not r["flags"] & orc.LAMINATED or r["margin"] < 1e-9:
            continue
        d = int(r["dir"])
        ia, ib = d // Nb, d % Nb
        jump = tro[p, 2]["F"] - tro[p, 1]["F"]
        off = ((ia + 3) % Na, ib)  # three cells away along theta_a
        flat = _constant_net(math.pi * off[0] / Na, math.pi * off[1] / Nb, r["xi"], jump)
        kw = dict(Na=Na, Nb=Nb, L=151, t_half=0.5, K=1, w=1, gap_tol=1e30, flat=flat,
                  mean=np.zeros(6), std=np.ones(6), F=F[p:p + 1], beta=beta[p:p + 1])
        _, _, t0 = osur.propose_convexify(orc, mat, recentre=0, **kw)
        WR, P, t6 = osur.propose_convexify(orc, mat, recentre=6, **kw)
        rec0, rec6 = t0[0][0], t6[0][0]
        assert rec0["center"] == off and rec6["center"] == off
        if rec0["flags"] & osur.FALLBACK and not rec6["flags"] & osur.FALLBACK:
            assert rec6["recentred"] >= 1 and rec6["dir"] == d
            assert WR[0] == WRo[p]
            np.testing.assert_array_equal(P[0], Po[p])
            walked += 1
        # a result without fallback always is the window's own interior minimum
        if not rec6["flags"] & osur.FALLBACK and rec6["flags"] & orc.LAMINATED:
            ca, cb = rec6["last_center"]
            assert abs(osur._offset(rec6["dir"] // Nb, ca, Na)) < 1
            assert abs(osur._offset(rec6["dir"] % Nb, cb, Nb)) < 1
    assert walked >= 2


def test_mirror_angles_keep_the_energy(orc):
    """The reflection of a rank-one direction about the principal axes of F
    keeps W on every point of the line (isotropy: I1 and J unchanged); a
    mirror that pairs the axes the wrong way round does not."""
    from paper_2211_14318_gb300 import inputs

    mat, F, beta = _points(orc, 24, 41)
    rng = np.random.default_rng(3)
    F = F + 0.1 * rng.standard_normal(F.shape) * np.array([0, 1, 1, 0])  # break the symmetry of F
    worst, wrong = 0.0, 0.0
    for p in range(F.shape[0]):
        if F[p, 0] * F[p, 3] - F[p, 1] * F[p, 2] <= 0.2:
            continue
        ta, tb = rng.uniform(0, math.pi, 2)
        ma, mb = osur.mirror_angles(F[p], ta, tb)
        p1, p2 = osur.principal_angles(F[p])
        for t in (-0.4, -0.1, 0.05, 0.3):
            def w(a, b):
                R = np.outer([math.cos(a), math.sin(a)], [math.cos(b), math.sin(b)]).reshape(4)
                return orc.energy(mat, F[p] + t * R, beta[p])
            w0 = w(ta, tb)
            if not np.isfinite(w0):
                continue
            worst = max(worst, abs(w(ma, mb) - w0) / (1 + abs(w0)))
            wrong = max(wrong, abs(w(2 * p2 - ta, 2 * p1 - tb) - w0) / (1 + abs(w0)))
    assert worst < 1e-12
    assert wrong > 1e-4


def test_mirror_cell_of_a_diagonal_F():
    """For a diagonal F the principal axes are the coordinate axes, so the
    mirror of cell (ia, ib) is (-ia, -ib) mod N, half a cell from any
    rounding boundary."""
    for F in (np.array([1.3, 0.0, 0.0, 0.9]), np.array([0.8, 0.0, 0.0, 1.2])):
        for gd in (0, 5, 7 * 16 + 3, 255):
            mc, dist = osur.mirror_cell(F, gd, 16, 16)
            assert mc == ((-(gd // 16)) % 16, (-(gd % 16)) % 16)
            assert dist == pytest.approx(0.5)


def test_mirror_window_recovers_the_twin_basin(orc):
    """Load-path nodes whose hull value over the angles has two mirrored
    basins (one the full scan's direction d, the other its twin near the
    mirror cell of d): a fixed network proposing the mirror cell of d makes
    the window settle in the twin basin, and only the mirror window brings
    the result back to the plain method's, bit for bit."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(*MAT)
    path = inputs.load_path(16, n_steps=20, stretch_end=1.8, seed=7)
    beta = None
    for k in range(9):
        beta = orc.history_update(mat, path[k], beta)
    Na = Nb = 32
    dirs = orc.angle_directions(Na, Nb)
    F0, b0 = path[9][:24], beta[:24]
    _, _, tr, _ = orc.convexify(mat, orc.Scan(dirs, 151, 0.5, 3), F0, b0)
    # the level-2 nodes as points of their own (depth 1)
    F = np.array([tr[p, 6]["F"] for p in range(24) if tr[p, 6]["flags"] & orc.LAMINATED])
    b = np.array([b0[p] for p in range(24) if tr[p, 6]["flags"] & orc.LAMINATED])
    sc = orc.Scan(dirs, 151, 0.5, 1)
    WRo, Po, tro, _ = orc.convexify(mat, sc, F, b)
    recovered = 0
    for p in range(F.shape[0]):
        r = tro[p, 0]
        if not r["flags"] & orc.LAMINATED or r["margin"] < 1e-9:
            continue
        d = int(r["dir"])
        mc, _ = osur.mirror_cell(F[p], d, Na, Nb)
        flat = _constant_net(math.pi * mc[0] / Na, math.pi * mc[1] / Nb, r["xi"],
                             tro[p, 2]["F"] - tro[p, 1]["F"])
        kw = dict(Na=Na, Nb=Nb, L=151, t_half=0.5, K=1, w=1, gap_tol=1e30, flat=flat,
                  mean=np.zeros(6), std=np.ones(6), F=F[p:p + 1], beta=b[p:p + 1], recentre=4)
        W0, _, t0 = osur.propose_convexify(orc, mat, mirror=False, **kw)
        W1, P1, t1 = osur.propose_convexify(orc, mat, mirror=True, **kw)
        rec0, rec1 = t0[0][0], t1[0][0]
        if rec0["flags"] & osur.FALLBACK or rec1["flags"] & osur.FALLBACK:
            continue
        if rec0["dir"] != d:  # the window settled in the twin basin
            assert W0[0] > WRo[p]
            assert rec1["mirror_won"] and not rec1["mirror_inside"]
            assert rec1["dir"] == d
            assert W1[0] == WRo[p]
            np.testing.assert_array_equal(P1[0], Po[p])
            recovered += 1
        else:
            assert rec1["dir"] == d and W1[0] == WRo[p]
    assert recovered >= 5
