"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Decision precision: the kernel screens every direction with FP32 samples of W
and then takes each node's direction and split decision on FP64 samples of
the few directions that pass the screen; the oracle decides on FP64 samples
throughout.  The two sides' FP64 samples differ only by the last-bit
differences of the two libm's exp/log, so a decision is compared bit-exactly
wherever the oracle's certified margin (the largest sample perturbation that
cannot change it) exceeds TIE; elsewhere the GPU's choice is checked for
validity.  The FP32 screen itself relies on SAMPLE_EPS, pinned by
test_sample_error_bound.  Bars: indices bit-exact on untied nodes, W^R within
1e-6 relative (gamma = 1e-8, the paper's error measure of Sec. 6.2), P within
1e-5 relative.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SAMPLE_EPS = 4e-7   # max |W_gpu - W| / max(1, |W|) of FP32 line samples (measured 3.1e-7)
TIE = 1e-11         # node margins (FP64 decisions) at or below this are ties
MAT = dict(mu=1.0, lambda_L=5.0, D_inf=0.99, D0=0.5)


@pytest.fixture(scope="module")
def cv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api

    c = api.Convexifier(0)
    yield c
    c.close()


def _omat(orc, energy=0, **kw):
    m = dict(MAT)
    m.update(kw)
    return orc.Material(m["mu"], m["lambda_L"], m["D_inf"], m["D0"], energy=energy)


def _rel(a, b, gamma=1e-8):
    return np.abs(a - b) / (gamma + np.abs(b))


def _compare_trees(orc, api, tree_g, tree_o, L):
    """Walk both trees; returns (n_compared_nodes, untied_point_mask)."""
    n, NT = tree_o.shape
    untied = np.ones(n, dtype=bool)
    compared = 0
    for p in range(n):
        stack = [0]
        while stack:
            i = stack.pop()
            fo = tree_o[p, i]["flags"]
            if not fo & orc.SCANNED:
                continue
            if tree_o[p, i]["margin"] <= TIE:
                untied[p] = False
                continue
            compared += 1
            g, o = tree_g[p, i], tree_o[p, i]
            assert g["flags"] & api.NODE_SCANNED
            lam_o = bool(fo & orc.LAMINATED)
            assert bool(g["flags"] & api.NODE_LAMINATED) == lam_o, (p, i)
            if lam_o:
                assert (g["dir"], g["m_minus"], g["m_plus"]) == (o["dir"], o["m_minus"], o["m_plus"]), (p, i)
                np.testing.assert_array_equal(g["F"], o["F"])
                stack += [2 * i + 1, 2 * i + 2]
    return compared, untied


def test_energy_stress_history(cv, orc):
    """Eqs. (2.5), (2.9), (2.12) in FP64 on the GPU against the oracle."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(300, seed=3, lam_hi=2.0)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    beta[::3] = 0.0
    beta[1::5] = 2.0
    p = api.Params(**MAT)
    W, P = cv.energy(p, F, beta)
    Wo = np.array([orc.energy(mat, F[i], beta[i]) for i in range(300)])
    Po = np.array([orc.stress(mat, F[i], beta[i]) for i in range(300)])
    assert np.max(_rel(W.cpu().numpy(), Wo, 1e-12)) < 1e-11
    assert np.max(np.abs(P.cpu().numpy() - Po)) < 1e-12
    bg = cv.history_update(p, Fp, beta).cpu().numpy()
    np.testing.assert_allclose(bg, orc.history_update(mat, Fp, beta), rtol=1e-14, atol=1e-15)
    # det F <= 0 -> NaN
    W2, P2 = cv.energy(p, np.array([[1.0, 0, 0, -1.0]]), np.zeros(1))
    assert math.isnan(W2.item()) and np.all(np.isnan(P2.cpu().numpy()))


@pytest.mark.parametrize("L", [201, 1025, 2049])
def test_sample_error_bound(cv, orc, L):
    """FP32 line samples (Eq. 4.4 per point) against FP64: the error bound that
    defines a tie (SAMPLE_EPS), and the same validity (det > 0) pattern."""
    from paper_2211_14318_gb300 import api, inputs

    mat = _omat(orc)
    F, Fp = inputs.surrogate_inputs(200, seed=L)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(64, 64)
    idx = np.random.default_rng(L).integers(0, 4096, size=200)
    p = api.Params(n_theta_a=64, n_theta_b=64, line_points=L, **MAT)
    w = cv.sample_lines(p, F, beta, idx).cpu().numpy()
    worst = 0.0
    for i in range(200):
        wo, v = orc.sample_line(mat, F[i], beta[i], orc.rank_one(dirs[idx[i]]), L, 0.5)
        fin = np.isfinite(w[i])
        assert np.all(fin[v] | (np.abs(wo[v]) > 1e3))  # only near det = 0 may differ
        ok = v & fin
        worst = max(worst, np.max(np.abs(w[i][ok] - wo[ok])) / max(1.0, np.max(np.abs(wo[ok]))))
    assert worst < SAMPLE_EPS, worst


def _random_lines(rng, L, n):
    m0 = (L - 1) // 2
    x = np.arange(L) - m0
    sc = max(m0, 1)
    out = []
    for i in range(n):
        kind = i % 5
        if kind == 0:
            v = 0.3 * np.sin(x / (3 + 40 * rng.random())) + 1e-5 * x ** 2 * rng.random() + 0.01 * rng.normal(size=L)
        elif kind == 1:
            v = rng.integers(-3, 4, size=L).astype(float)  # many collinear triples
        elif kind == 2:
            v = (x / sc) ** 4 - (x / sc) ** 2 * rng.random() + 1e-7 * rng.normal(size=L)
        elif kind == 3:
            v = np.abs(x) * 0.001 + 0.001 * rng.normal(size=L)
        else:
            v = np.full(L, 0.25) + (x == 0) * rng.choice([-1.0, 0.0, 1.0])  # flat lines
        v = v.astype(np.float32)
        if i % 3 == 0:
            lo, hi = rng.integers(0, m0 + 1), rng.integers(m0, L)
            v[:lo] = np.nan
            v[hi + 1:] = np.nan
        out.append(v)
    return np.array(out, dtype=np.float32)


@pytest.mark.parametrize("L", [3, 5, 41, 201, 513, 1025, 2049, 2079])
def test_hull_bridge_bit_exact(cv, orc, L):
    """Algorithm 1 + value at l = 0 on identical FP32 samples: bridge indices
    and the FP64 value are bit-identical to the oracle (the kernel's hull is
    exact for its FP32 inputs)."""
    import torch

    rng = np.random.default_rng(L)
    ws = _random_lines(rng, L, 300)
    mm, mp, h = cv.hull_bridge(torch.from_numpy(ws))
    mm, mp, h = mm.cpu().numpy(), mp.cpu().numpy(), h.cpu().numpy()
    for i in range(len(ws)):
        valid = np.isfinite(ws[i])
        ho, a, b, _ = orc.line_bridge(np.where(valid, ws[i].astype(np.float64), 0.0), valid)
        assert (mm[i], mp[i]) == (a, b), (L, i)
        assert h[i] == ho, (L, i)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_double_well_closed_form(cv, depth):
    """Test energy with a closed-form envelope: at F = diag(0, 1) the relaxed
    energy is 0, split into diag(+-1, 1) with xi = 1/2 along e1 (x) e1, P = 0."""
    from paper_2211_14318_gb300 import api

    p = api.Params(energy=api.ENERGY_DOUBLE_WELL, n_theta_a=8, n_theta_b=8, line_points=301,
                   t_half=1.5, depth=depth)
    out = cv.convexify_points(p, np.array([[0.0, 0, 0, 1]]), np.zeros(1), want_tree=True,
                              want_root=True)
    assert abs(out["W_R"].item()) < 1e-15
    assert np.max(np.abs(out["P"].cpu().numpy())) < 1e-12
    r = api.root_numpy(out["root"], 1)[0]
    assert r["laminated"] == 1 and r["dir"] == 0 and r["xi"] == 0.5
    np.testing.assert_array_equal(r["F_plus"], [1, 0, 0, 1])
    np.testing.assert_array_equal(r["F_minus"], [-1, 0, 0, 1])


def _parity(cv, orc, F, beta, p, dirs_o, sample_idx=None):
    from paper_2211_14318_gb300 import api

    out = cv.convexify_points(p, F, beta, want_tree=True, want_root=True)
    n = F.shape[0]
    tree_g = api.tree_numpy(out["tree"], n, p.tree_size)
    WR = out["W_R"].cpu().numpy()
    P = out["P"].cpu().numpy()
    st = out["status"].cpu().numpy()
    idx = np.arange(n) if sample_idx is None else np.asarray(sample_idx)
    mat = _omat(orc, energy=p.energy, mu=p.mu, lambda_L=p.lambda_L, D_inf=p.D_inf, D0=p.D0)
    sc = orc.Scan(dirs_o, p.line_points, p.t_half, p.depth, round32=False)
    WRo, Po, tro, sto = orc.convexify(mat, sc, F[idx], beta[idx])
    compared, untied = _compare_trees(orc, api, tree_g[idx], tro, p.line_points)
    assert np.all((st[idx] & 1) == (sto & 1))
    u = untied
    assert np.max(_rel(WR[idx][u], WRo[u]), initial=0) < 1e-6
    Pn = np.linalg.norm(Po, axis=1)
    assert np.max(np.linalg.norm(P[idx][u] - Po[u], axis=1) / (1e-8 + Pn[u]), initial=0) < 1e-5
    # tied points: the GPU's W^R is the oracle's energy summed over the GPU's
    # own tree leaves, and its root choice is within the tie tolerance of the
    # oracle's best direction
    for k in np.nonzero(~u)[0]:
        p0 = idx[k]
        tr = tree_g[p0]
        leaf = (tr["flags"] & api.NODE_EXISTS > 0) & (tr["flags"] & api.NODE_LAMINATED == 0)
        Wl = sum(tr[i]["weight"] * orc.energy(mat, tr[i]["F"], beta[p0]) for i in np.nonzero(leaf)[0])
        assert abs(WR[p0] - Wl) <= 1e-11 * (1 + abs(Wl))
        if tree_g[p0, 0]["dir"] >= 0 and tro[k, 0]["flags"] & orc.SCANNED:
            info = orc.scan_node(mat, sc, F[p0], beta[p0], per_direction=True)
            hj = info["h_dir"][tree_g[p0, 0]["dir"]]
            assert hj <= info["h"] + 2 * TIE * max(1.0, abs(info["h"]))
    return compared, u.mean()


def test_config1_parity(cv, orc):
    """64 material points (rotated stretch + noise, history from one prior
    step), 16 x 16 angles, L = 201, t in [-0.5, 0.5], depth 2."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(64, seed=0)
    beta = orc.history_update(_omat(orc), Fp)
    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, t_half=0.5, depth=2, **MAT)
    compared, frac = _parity(cv, orc, F, beta, p, orc.angle_directions(16, 16))
    assert compared >= 100 and frac > 0.8


def test_ragged_sizes_and_direction_blocks(cv, orc):
    """A point count that is no multiple of anything, directions split over
    several work items, and an odd line length with a partial last slot."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(37, seed=9, lam_hi=1.8)
    beta = orc.history_update(_omat(orc), Fp)
    p = api.Params(n_theta_a=7, n_theta_b=9, line_points=77, t_half=0.6, depth=3, **MAT)
    cv.set_tuning(4, 5)
    try:
        compared, frac = _parity(cv, orc, F, beta, p, orc.angle_directions(7, 9))
    finally:
        cv.set_tuning(8, 0)
    assert compared > 37


def test_reduced_direction_set(cv, orc):
    """The reduced set R^1_1 of Eq. (5.1) as a custom list: a, b in {-1,0,1}^2,
    one of each +- pair, unnormalised (16 directions)."""
    from paper_2211_14318_gb300 import api, inputs

    vecs = [(1, 0), (0, 1), (1, 1), (1, -1)]
    dirs = np.array([[a[0], a[1], b[0], b[1]] for a in vecs for b in vecs], dtype=np.float64)
    F, Fp = inputs.material_points(24, seed=4)
    beta = orc.history_update(_omat(orc), Fp)
    p = api.Params(line_points=101, t_half=0.4, depth=2, dirs=dirs, **MAT)
    compared, frac = _parity(cv, orc, F, beta, p, dirs)
    assert compared >= 24


def test_edge_cases(cv, orc):
    """n = 0, det F <= 0 (NaN, status bit), depth 0 (W^R = W, P = dW/dF),
    L = 3, a single direction, undamaged Neo-Hooke (no split anywhere)."""
    import torch

    from paper_2211_14318_gb300 import api, inputs

    p = api.Params(**MAT)
    out = cv.convexify_points(p, np.zeros((0, 4)), np.zeros(0))
    assert out["W_R"].numel() == 0
    F = np.array([[1.0, 0, 0, -1.0], [1.2, 0.1, 0, 0.9]])
    out = cv.convexify_points(p, F, np.zeros(2))
    st = out["status"].cpu().numpy()
    assert st[0] & api.PT_NONPOS_DET and math.isnan(out["W_R"][0].item())
    assert not st[1] & api.PT_NONPOS_DET
    F, Fp = inputs.material_points(20, seed=2)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    out = cv.convexify_points(api.Params(depth=0, **MAT), F, beta)
    Wo = np.array([orc.energy(mat, F[i], beta[i]) for i in range(20)])
    np.testing.assert_allclose(out["W_R"].cpu().numpy(), Wo, rtol=1e-11)
    for L in (3, 5):
        pp = api.Params(line_points=L, n_theta_a=4, n_theta_b=4, depth=2, **MAT)
        _parity(cv, orc, F, beta, pp, orc.angle_directions(4, 4))
    p1 = api.Params(n_theta_a=1, n_theta_b=1, depth=2, **MAT)
    _parity(cv, orc, F, beta, p1, orc.angle_directions(1, 1))
    und = dict(MAT, D_inf=0.0)
    pu = api.Params(n_theta_a=8, n_theta_b=8, line_points=101, depth=2, **und)
    out = cv.convexify_points(pu, F, np.zeros(20), want_tree=True)
    Wu = np.array([orc.energy(_omat(orc, D_inf=0.0), F[i], 0.0) for i in range(20)])
    np.testing.assert_allclose(out["W_R"].cpu().numpy(), Wu, rtol=1e-11)
    tr = api.tree_numpy(out["tree"], 20, pu.tree_size)
    assert not np.any(tr["flags"][:, 0] & api.NODE_LAMINATED)
    torch.cuda.synchronize()


def test_tree_invariants_full_size(cv, orc):
    """On the full 65,536-point mesh workload (128 x 128 Q1 x 4 Gauss points,
    64 x 64 angles, L = 1025, depth 3), properties that hold at any size: leaf
    weights sum to 1, the weighted leaf mean is F (an H_M sequence, Eq. 3.4),
    every split is rank-one along its chosen direction, and
    W^R = sum of weighted leaf energies <= W."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.mesh_points(128, stretch=1.3, seed=0)
    p = api.Params(n_theta_a=64, n_theta_b=64, line_points=1025, t_half=0.5, depth=3, **MAT)
    beta = cv.history_update(p, Fp)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    n = F.shape[0]
    tr = api.tree_numpy(out["tree"], n, p.tree_size)
    WR = out["W_R"].cpu().numpy()
    W, _ = cv.energy(p, F, beta)
    assert np.all(WR <= W.cpu().numpy() + 1e-15)
    leaf = (tr["flags"] & api.NODE_EXISTS > 0) & (tr["flags"] & api.NODE_LAMINATED == 0)
    wsum = np.sum(np.where(leaf, tr["weight"], 0.0), axis=1)
    assert np.max(np.abs(wsum - 1.0)) < 1e-13
    mean = np.sum(np.where(leaf[..., None], tr["weight"][..., None] * tr["F"], 0.0), axis=1)
    assert np.max(np.abs(mean - F)) < 1e-12
    lam = tr["flags"] & api.NODE_LAMINATED > 0
    pi, ni = np.nonzero(lam)
    d = tr["F"][pi, 2 * ni + 2] - tr["F"][pi, 2 * ni + 1]
    det = d[:, 0] * d[:, 3] - d[:, 1] * d[:, 2]
    assert np.max(np.abs(det)) < 1e-13
    assert lam.sum() > n  # the workload does laminate


def test_full_size_sampled_parity(cv, orc):
    """Full 65,536-point workload in the launch configuration bench.py times;
    the oracle recomputes 16 sampled points (spread over the mesh, including
    the shear band) one by one."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.mesh_points(128, stretch=1.3, seed=0)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    p = api.Params(n_theta_a=64, n_theta_b=64, line_points=1025, t_half=0.5, depth=3, **MAT)
    idx = np.linspace(0, F.shape[0] - 1, 16).astype(int)
    compared, frac = _parity(cv, orc, F, beta, p, orc.angle_directions(64, 64), sample_idx=idx)
    assert compared >= 16 and frac >= 0.9


@pytest.mark.parametrize("step", [5, 10])
def test_load_path_fine_grid_parity(cv, orc, step):
    """The configuration the proposed form is judged against (128 x 128
    angles, L = 2049, depth 3) on 4,096 points of the load path at a low and
    a medium load:
    enough points that every node is a single work item of 16,384 directions,
    as in bench.py's surrogate checks.  The oracle recomputes 8 sampled
    points."""
    from paper_2211_14318_gb300 import api, inputs

    mat = _omat(orc)
    path = inputs.load_path(128, n_steps=20, stretch_end=1.8, seed=7)
    beta = np.zeros(path[0].shape[0])
    for k in range(step - 1):  # history of the earlier load steps
        beta = orc.history_update(mat, path[k], beta)
    sub = np.linspace(0, path[0].shape[0] - 1, 4096).astype(int)
    F, b = path[step - 1][sub], beta[sub]
    p = api.Params(n_theta_a=128, n_theta_b=128, line_points=2049, t_half=0.5, depth=3, **MAT)
    idx = np.linspace(0, F.shape[0] - 1, 8).astype(int)
    compared, frac = _parity(cv, orc, F, b, p, orc.angle_directions(128, 128), sample_idx=idx)
    assert compared >= 8 and frac >= 0.9


def test_stats_account_for_the_work(cv, orc):
    """Counters: lines = scanned nodes x directions; valid samples <= lines x L."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(50, seed=1)
    p = api.Params(n_theta_a=12, n_theta_b=12, line_points=301, depth=2, **MAT)
    beta = cv.history_update(p, Fp)
    cv.stats(reset=True)
    cv.convexify_points(p, F, beta)
    s = cv.stats(reset=True)
    assert s["points"] == 50
    assert s["lines"] == s["nodes_scanned"] * 144
    assert 0.9 * s["lines"] * 301 <= s["valid_samples"] <= s["lines"] * 301
    # an uncertified node (more than 16 directions inside the FP32 screening
    # band, whose decision is then within 2.25 eps of the FP64 minimum: the
    # golden tests check that bar against the oracle) is rare at 12 x 12 angles
    assert s["iter_caps"] == 0 and s["overflow"] <= 0.1 * s["nodes_scanned"]
    assert s["laminated"] <= s["refined"] <= 16 * s["nodes_scanned"]


def test_newton_double_well_exact_tangent(cv, orc):
    """CVX_FLAG_REFINE_NEWTON on the double well: the refined split of
    F = diag(0.3, 1) is diag(+-1, 1) (off the line grid), W^R = 0, xi = 0.65."""
    from paper_2211_14318_gb300 import api

    p = api.Params(energy=api.ENERGY_DOUBLE_WELL, n_theta_a=8, n_theta_b=8, line_points=201,
                   t_half=1.5, depth=1, newton=True)
    out = cv.convexify_points(p, np.array([[0.3, 0, 0, 1.0]]), np.zeros(1), want_tree=True)
    tr = api.tree_numpy(out["tree"], 1, p.tree_size)[0]
    assert tr[0]["flags"] & api.NODE_NEWTON and tr[0]["dir"] == 0
    np.testing.assert_allclose(tr[1]["F"], [-1, 0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(tr[2]["F"], [1, 0, 0, 1], atol=1e-12)
    assert abs(tr[0]["xi"] - 0.65) < 1e-12
    assert abs(out["W_R"].item()) < 1e-13


def test_newton_refinement_matches_oracle(cv, orc):
    """NH with damage, a window wide enough for interior splits (|t| <= 12),
    depth 2: the GPU's refined splits against the oracle's (same grid
    decision, refined ends to 1e-9, same acceptance), W^R and P to the bars."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(40, seed=12, lam_hi=1.8)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    p = api.Params(n_theta_a=12, n_theta_b=12, line_points=301, t_half=12.0, depth=2,
                   newton=True, **MAT)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    tg = api.tree_numpy(out["tree"], F.shape[0], p.tree_size)
    sc = orc.Scan(orc.angle_directions(12, 12), 301, 12.0, 2, newton=True)
    WRo, Po, to, sto = orc.convexify(mat, sc, F, beta)
    WR, P = out["W_R"].cpu().numpy(), out["P"].cpu().numpy()
    refined = 0
    good = np.ones(F.shape[0], dtype=bool)
    for q in range(F.shape[0]):
        stack = [0]
        while stack:
            i = stack.pop()
            o, g = to[q, i], tg[q, i]
            if not o["flags"] & orc.SCANNED:
                continue
            if o["margin"] <= TIE:
                good[q] = False
                continue
            lam = bool(o["flags"] & orc.LAMINATED)
            assert bool(g["flags"] & api.NODE_LAMINATED) == lam, (q, i)
            if lam:
                assert (g["dir"], g["m_minus"], g["m_plus"]) == (o["dir"], o["m_minus"], o["m_plus"])
            assert bool(g["flags"] & api.NODE_NEWTON) == bool(o["flags"] & orc.NEWTON), (q, i)
            if o["flags"] & orc.NEWTON:
                refined += 1
                np.testing.assert_allclose(tg[q, 2 * i + 1]["F"], to[q, 2 * i + 1]["F"], atol=1e-9)
                np.testing.assert_allclose(tg[q, 2 * i + 2]["F"], to[q, 2 * i + 2]["F"], atol=1e-9)
                assert abs(g["xi"] - o["xi"]) < 1e-9
            if o["flags"] & orc.LAMINATED:
                stack += [2 * i + 1, 2 * i + 2]
    assert refined >= 10
    assert np.max(_rel(WR[good], WRo[good]), initial=0) < 1e-6
    Pn = np.linalg.norm(Po, axis=1)
    assert np.max(np.linalg.norm(P[good] - Po[good], axis=1) / (1e-8 + Pn[good]), initial=0) < 1e-5


def test_tree_tangent_matches_oracle(cv, orc):
    """Tangent of W^R (Eq. 5.2 / Algorithm 3 on second derivatives, laminate
    held fixed): the GPU over its own tree against the oracle's tangent of W
    summed over the same leaves, and on untied points against the oracle's
    tree tangent of its own tree (pinned by central differences of the
    oracle's P); NaN for det F <= 0."""
    from paper_2211_14318_gb300 import api, inputs

    mat = _omat(orc)
    F, Fp = inputs.material_points(64, seed=70, lam_hi=1.8)
    beta = orc.history_update(mat, Fp)
    F[5] = [1.0, 0.0, 0.0, -1.0]
    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    A = cv.tree_tangent(p, beta, out["tree"], 64).cpu().numpy()
    tree = api.tree_numpy(out["tree"], 64, p.tree_size)
    assert np.all(np.isnan(A[5]))
    for q in range(64):
        if q == 5:
            continue
        leaf = (tree[q]["flags"] & api.NODE_EXISTS > 0) & (tree[q]["flags"] & api.NODE_LAMINATED == 0)
        Ao = sum(tree[q, i]["weight"] * orc.tangent(mat, tree[q, i]["F"], beta[q])
                 for i in np.nonzero(leaf)[0])
        np.testing.assert_allclose(A[q], Ao, rtol=1e-12, atol=1e-12 * np.abs(Ao).max())
    sc = orc.Scan(orc.angle_directions(16, 16), 201, 0.5, 2)
    _, _, tro, _ = orc.convexify(mat, sc, F, beta)
    Aor = orc.tree_tangent(mat, 2, tro, beta)
    compared, untied = _compare_trees(orc, api, tree, tro, 201)
    untied[5] = False
    assert untied.sum() > 40
    np.testing.assert_allclose(A[untied], Aor[untied], rtol=1e-10, atol=1e-10)


def test_adaptive_window_double_well_closed_form(cv):
    """Adaptive line window on the double well (the warp-per-line scan):
    F = diag(0, 1) with t_half = 0.25 needs three doublings before the split
    diag(+-1, 1) is interior; then W^R = 0, xi = 1/2, P = 0."""
    from paper_2211_14318_gb300 import api

    p = api.Params(energy=api.ENERGY_DOUBLE_WELL, n_theta_a=4, n_theta_b=4, line_points=101,
                   t_half=0.25, depth=1, window_doublings=5)
    cv.stats(reset=True)
    out = cv.convexify_points(p, np.array([[0.0, 0, 0, 1.0]]), np.zeros(1), want_tree=True)
    st = cv.stats(reset=True)
    tr = api.tree_numpy(out["tree"], 1, p.tree_size)[0]
    assert tr[0]["window_exp"] == 3 and (tr[0]["m_minus"], tr[0]["m_plus"]) == (25, 75)
    assert tr[0]["xi"] == 0.5 and st["window_doublings"] == 3
    np.testing.assert_allclose(tr[1]["F"], [-1, 0, 0, 1], atol=1e-12)
    np.testing.assert_allclose(tr[2]["F"], [1, 0, 0, 1], atol=1e-12)
    assert abs(out["W_R"].item()) < 1e-12 and np.max(np.abs(out["P"].cpu().numpy())) < 1e-12


def test_adaptive_window_matches_oracle(cv, orc):
    """NH with damage, up to 5 doublings of t_half = 0.5 (|t| up to 16),
    depth 2: decisions, window exponents and split points bit-exact on untied
    nodes, W^R and P to the bars; splits are interior unless the node used
    all its doublings."""
    from paper_2211_14318_gb300 import api, inputs

    mat = _omat(orc)
    F, Fp = inputs.material_points(48, seed=82, lam_hi=1.8)
    beta = orc.history_update(mat, Fp)
    p = api.Params(n_theta_a=12, n_theta_b=12, line_points=151, t_half=0.5, depth=2,
                   window_doublings=5, **MAT)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    tg = api.tree_numpy(out["tree"], F.shape[0], p.tree_size)
    sc = orc.Scan(orc.angle_directions(12, 12), 151, 0.5, 2, adaptive=5)
    WRo, Po, to, _ = orc.convexify(mat, sc, F, beta)
    compared, untied = _compare_trees(orc, api, tg, to, 151)
    scanned = (to["flags"] & orc.SCANNED) > 0
    assert np.all(tg["window_exp"][untied][scanned[untied]] == to["wexp"][untied][scanned[untied]])
    assert compared >= 48 and untied.mean() > 0.8
    WR, P = out["W_R"].cpu().numpy(), out["P"].cpu().numpy()
    assert np.max(_rel(WR[untied], WRo[untied])) < 1e-6
    Pn = np.linalg.norm(Po, axis=1)
    assert np.max(np.linalg.norm(P[untied] - Po[untied], axis=1) / (1e-8 + Pn[untied])) < 1e-5
    lam = (tg["flags"] & api.NODE_LAMINATED) > 0
    edge = (tg["m_minus"] == 0) | (tg["m_plus"] == 150)
    assert np.all(~lam | ~edge | (tg["window_exp"] == 5))
    assert np.any(lam & (tg["window_exp"] > 0))
