"""GPU parity of the global-grid form (Eq. 4.3 iterated on the cuboid grid of
Sec. 5.2 with the directions R^1_1 of Eq. 5.1; Algorithm 1 on every line;
Algorithm 2's trees with interpolation branching evaluated by Algorithm 3)
against the FP64 oracle, through the C ABI.

A step has no transcendental function: hull predicates and chord values are
FP64 expressions with every operation rounded on its own on both sides, so a
step taken from the same input is compared bit for bit (values, laminate
records, the step's largest decrease).  W^0 involves log and exp, whose last
bits differ between CUDA's and the host's libm, so the device's own loop is
compared with tolerances, and its laminate records on the points whose
decision is not a near-tie.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NH61 = dict(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3)  # Table tab:2Dconvexification, NH row
BETA61 = 0.06
DIAG61, OFF61, DELTA61 = (0.1, 3.4), (-2.55, 2.55), (0.15, 0.15)


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


def _params(api, energy=0, **m):
    m = m or NH61
    return api.Params(mu=m.get("mu", 1.0), lambda_L=m.get("lam", 0.5), D_inf=m.get("Dinf", 0.9),
                      D0=m.get("D0", 0.3), energy=energy)


def _both_grids(orc, api, n=None, lo=None, delta=None):
    if n is None:
        go = orc.Grid.from_bounds(DIAG61, OFF61, DELTA61)
        gg = api.GridSpec.from_bounds(DIAG61, OFF61, DELTA61)
    else:
        go, gg = orc.Grid(n, lo, delta), api.GridSpec(n, lo, delta)
    assert tuple(gg.n) == go.n and tuple(gg.lo) == go.lo and tuple(gg.delta) == go.delta
    return go, gg


@pytest.fixture(scope="module")
def study(orc):
    """The oracle's run of the Sec. 6.1 NH study (648,025 points, R^1_1,
    tol 1e-4, kmax 20, ln|det F|): every W^k, the forest and the decreases."""
    mat = orc.Material(**NH61)
    go = orc.Grid.from_bounds(DIAG61, OFF61, DELTA61)
    off = orc.r11_directions()
    W, forest, decs = orc.grid_convexify(mat, go, BETA61, off, kmax=20, tol=1e-4, rule=1)
    return dict(W=W, forest=orc.forest_array(forest), decs=decs, off=off)


def _eq_nan(a, b):
    return np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("abs_det", [False, True])
def test_grid_energy_matches_oracle(cv, orc, abs_det):
    from paper_2211_14318_gb300 import api

    go, gg = _both_grids(orc, api)
    Wg = cv.grid_energy(_params(api), gg, BETA61, int(abs_det)).cpu().numpy()
    Wo = orc.grid_energy(orc.Material(**NH61), go, BETA61, abs_det)
    assert np.array_equal(np.isnan(Wg), np.isnan(Wo))
    f = np.isfinite(Wo)
    # log and exp of the two libms differ in their last bits
    assert np.max(np.abs(Wg[f] - Wo[f]) / (1.0 + np.abs(Wo[f]))) < 1e-13
    if not abs_det:
        assert (~f).sum() > 0  # the grid holds det F <= 0


def test_every_step_of_the_sec61_study_is_bit_exact(cv, study):
    """Each of the 15 steps of the study, from the oracle's W^k: W^{k+1}, the
    laminate records and the step's largest decrease are identical."""
    from paper_2211_14318_gb300 import api

    gg = api.GridSpec.from_bounds(DIAG61, OFF61, DELTA61)
    off = api.grid_r11()
    assert len(study["decs"]) == 15
    for k in range(len(study["decs"])):
        Wn, lam, dec = cv.grid_step(gg, off, study["W"][k])
        assert _eq_nan(Wn.cpu().numpy(), study["W"][k + 1]), f"step {k + 1}: W differs"
        assert np.array_equal(lam.cpu().numpy(), study["forest"][k]), f"step {k + 1}: laminates"
        assert float(dec.cpu()[0]) == study["decs"][k]


RAGGED = [
    # lines up to 45 points (128 lines per CTA)
    ((45, 9, 7, 30), (-0.4, -0.5, -0.45, 0.2), (0.05, 0.125, 0.15, 0.05)),
    # lines up to 300 points (32 lines per CTA)
    ((300, 3, 2, 5), (-0.5, -0.3, -0.2, 0.6), (0.01, 0.3, 0.4, 0.1)),
]


@pytest.mark.parametrize("shape", range(len(RAGGED)))
@pytest.mark.parametrize("chunk_bytes", [None, "1"])
def test_steps_with_excluded_points_long_ragged_lines_and_wider_offsets(cv, orc, chunk_bytes,
                                                                        shape):
    """Ragged grids with long lines, det F <= 0 excluded (NaN holes in the
    lines), R^1_1 plus rank-one offsets of two grid steps; three steps from
    the oracle's iterates, bit for bit.  With a chunk budget of one byte every
    direction is its own chunk (the merge across chunks)."""
    from paper_2211_14318_gb300 import api

    n, lo, delta = RAGGED[shape]
    go, gg = _both_grids(orc, api, n, lo, delta)
    off = np.concatenate([api.grid_r11(), np.array([[2, 1, 0, 0], [0, 0, 2, 1], [2, 2, 1, 1],
                                                    [1, -1, -1, 1], [0, 2, 0, -1]], np.int32)])
    mat = orc.Material(**NH61)
    W = orc.grid_energy(mat, go, BETA61, abs_det=False)
    assert np.isnan(W).sum() > 100
    splits = 0
    old = os.environ.get("CVX_GRID_CHUNK_BYTES")
    try:
        if chunk_bytes:
            os.environ["CVX_GRID_CHUNK_BYTES"] = chunk_bytes
        for _ in range(3):
            Wo, d, lm, lp, dec = orc.grid_step(go, off, W)
            Wn, lam, decg = cv.grid_step(gg, off, W)
            lam = lam.cpu().numpy()
            assert _eq_nan(Wn.cpu().numpy(), Wo)
            assert np.array_equal(lam[:, 0], d) and np.array_equal(lam[:, 1], lm)
            assert np.array_equal(lam[:, 2], lp)
            assert float(decg.cpu()[0]) == dec
            splits += int((d >= 0).sum())
            W = Wo
        assert splits > 0
    finally:
        if old is None:
            os.environ.pop("CVX_GRID_CHUNK_BYTES", None)
        else:
            os.environ["CVX_GRID_CHUNK_BYTES"] = old


def _strides(n):
    s = [1] * len(n)
    for c in range(len(n) - 2, -1, -1):
        s[c] = s[c + 1] * n[c + 1]
    return np.array(s)


def test_device_loop_matches_the_oracle_loop(cv, orc, study):
    """cvx_grid_convexify (W^0 on the device, the stop decided on the device)
    against the oracle's loop: the same number of steps, decreases and W^K
    within 1e-12.  Laminates: the direction is unique where the oracle's
    decision is clear (best and second-best hull values, and the best and the
    point's own value, more than 1e-10 apart) and must agree there.  The
    bridge ends are not unique: W^0 takes log and exp of each side's libm, and
    the iterates hold numerically collinear hull points (a laminate's chord is
    a straight segment of W^k), which Algorithm 1 pops or keeps by the last
    bit.  So a bridge that differs must lie on the oracle's hull: the chord of
    the oracle's W^k through the device's ends gives the oracle's hull value
    at the point within 1e-12."""
    from paper_2211_14318_gb300 import api

    gg = api.GridSpec.from_bounds(DIAG61, OFF61, DELTA61)
    off = api.grid_r11()
    out = cv.grid_convexify(_params(api), gg, BETA61, off, kmax=20, tol=1e-4, det_rule=1)
    K = int(out["iters"].cpu()[0])
    assert K == len(study["decs"]) == 15
    decs = out["decs"].cpu().numpy()
    assert np.max(np.abs(decs[:K] - study["decs"])) < 1e-12
    assert np.all(decs[K:] == 0.0)
    WK = out["W"].cpu().numpy()
    Wo = study["W"][-1]
    assert np.array_equal(np.isnan(WK), np.isnan(Wo))
    f = np.isfinite(Wo)
    assert np.max(np.abs(WK[f] - Wo[f]) / (1.0 + np.abs(Wo[f]))) < 1e-12
    forest = out["forest"].cpu().numpy()[:K]
    go = orc.Grid.from_bounds(DIAG61, OFF61, DELTA61)
    steps = study["off"] @ _strides(go.n)
    idx_all = np.arange(go.count)
    for k in (0, 1, 7, K - 1):
        _, _, _, _, _, h = orc.grid_step(go, study["off"], study["W"][k], want_h=True)
        hs = np.sort(h, axis=1)
        w0 = study["W"][k]
        fin = np.isfinite(w0)
        g, o = forest[k], study["forest"][k]
        # a clear split of the oracle: its best hull value is clear of the
        # point's own value and of the second best; there the direction is
        # unique.  A chord equal to the point's value (the point lies on a
        # segment a previous step made straight) is a tie between splitting
        # and not splitting that the last bit decides, so elsewhere only
        # validity is required: in the oracle's own values the device's
        # choice is within 1e-10 of the best.
        clear = fin & (w0 - hs[:, 0] > 1e-10) & (hs[:, 1] - hs[:, 0] > 1e-10)
        assert clear.sum() > 1000
        assert np.array_equal(g[clear, 0], o[clear, 0]), f"step {k + 1}: directions differ"
        gj = g[fin, 0]
        hg = np.where(gj >= 0, h[fin][np.arange(gj.size), np.maximum(gj, 0)], w0[fin])
        best = np.minimum(w0[fin], hs[fin, 0])
        assert np.max(hg - best) < 1e-10, f"step {k + 1}: a device laminate is not the best"
        split = clear & (g[:, 0] >= 0)
        other = split & np.any(g[:, 1:] != o[:, 1:], axis=1)
        if other.any():
            q = idx_all[other]
            d, lm, lp = g[q, 0], g[q, 1], g[q, 2]
            assert np.all((lm < 0) & (lp > 0))
            wa, wb = w0[q + lm * steps[d]], w0[q + lp * steps[d]]
            chord = (lp * wa - lm * wb) / (lp - lm)
            ho = h[q, d]
            assert np.max(np.abs(chord - ho) / (1 + np.abs(ho))) < 1e-12, f"step {k + 1}"
        assert other.sum() < 0.05 * split.sum() + 1


def test_query_on_the_oracle_forest(cv, orc, study):
    """Algorithms 2 and 3 on the oracle's W^K and forest at random points,
    grid points, cell faces and points outside the grid: the interpolated
    W^K bit for bit, the leaf counts exactly, W, P and the tangent A over the
    tree within 1e-12 (leaf energies use each side's log and exp)."""
    from paper_2211_14318_gb300 import api

    go, gg = _both_grids(orc, api)
    rng = np.random.default_rng(11)
    P = go.points()
    F = np.concatenate([
        rng.uniform(P.min(0), P.max(0), size=(4096, 4)),
        P[rng.integers(0, P.shape[0], 512)],
        np.where(rng.random((512, 4)) < 0.5, P[rng.integers(0, P.shape[0], 512)],
                 rng.uniform(P.min(0), P.max(0), size=(512, 4))),
        rng.uniform(P.min(0) - 1.0, P.max(0) + 1.0, size=(256, 4)),
    ])
    mat = orc.Material(**NH61)
    wi_o, wt_o, P_o, nl_o, A_o = orc.grid_query(mat, go, BETA61, study["off"], study["W"][-1],
                                                study["forest"], F, rule=1, want_A=True)
    wi, wt, Pg, nl, Ag = cv.grid_query(_params(api), gg, BETA61, api.grid_r11(), study["W"][-1],
                                       study["forest"], F, det_rule=1, want_A=True)
    wi, wt, Pg, nl, Ag = (x.cpu().numpy() for x in (wi, wt, Pg, nl, Ag))
    assert _eq_nan(wi, wi_o)
    assert np.array_equal(nl, nl_o)
    inside = np.isfinite(wt_o)
    assert inside.sum() > 4000 and (~inside).sum() > 0
    assert np.array_equal(np.isnan(wt), ~inside)
    assert np.max(np.abs(wt[inside] - wt_o[inside]) / (1 + np.abs(wt_o[inside]))) < 1e-12
    pn = np.linalg.norm(P_o[inside], axis=1)
    assert np.max(np.linalg.norm(Pg[inside] - P_o[inside], axis=1) / (1 + pn)) < 1e-12
    assert nl_o.max() > 16  # trees that branch beyond the interpolation corners
    # Algorithm 3's tangent over the same trees
    an = np.abs(A_o[inside]).reshape(-1, 16).max(axis=1)
    assert np.max(np.abs(Ag[inside] - A_o[inside]).reshape(-1, 16).max(axis=1) / (1 + an)) < 1e-12
    assert np.all(np.isnan(Ag[~inside]))


def test_query_tree_matches_the_interpolated_relaxation(cv):
    """On the device's own run: Algorithm 3 over Algorithm 2's tree gives the
    interpolated W^K (the tree is the laminate that produced the value), and
    a grid point is its own single interpolation corner."""
    from paper_2211_14318_gb300 import api

    gg = api.GridSpec.from_bounds(DIAG61, OFF61, DELTA61)
    off = api.grid_r11()
    out = cv.grid_convexify(_params(api), gg, BETA61, off, kmax=20, tol=1e-4, det_rule=1)
    K = int(out["iters"].cpu()[0])
    rng = np.random.default_rng(5)
    lo = np.array(gg.lo)
    hi = lo + (np.array(gg.n) - 1) * np.array(gg.delta)
    F = rng.uniform(lo, hi, size=(20000, 4))
    wi, wt, P, nl = cv.grid_query(_params(api), gg, BETA61, off, out["W"], out["forest"][:K], F,
                                  det_rule=1)
    wi, wt, nl = wi.cpu().numpy(), wt.cpu().numpy(), nl.cpu().numpy()
    f = np.isfinite(wi)
    assert f.mean() > 0.99
    assert np.max(np.abs(wt[f] - wi[f]) / (1 + np.abs(wi[f]))) < 1e-12
    assert np.all(nl[f] >= 16)  # generic points: 16 corners, each at least one leaf


def test_double_well_reaches_the_closed_form(cv):
    """The separable double well on a grid whose F11 values include the wells
    +-1: one step along e1 (x) e1 (direction 0 of R^1_1) replaces (F11^2 - 1)^2
    by 0 on |F11| <= 1, the second step changes nothing and the loop stops."""
    from paper_2211_14318_gb300 import api

    gg = api.GridSpec((13, 3, 3, 5), (-1.5, -0.25, -0.25, 0.5), (0.25, 0.25, 0.25, 0.25))
    off = api.grid_r11()
    p = api.Params(energy=api.ENERGY_DOUBLE_WELL)
    out = cv.grid_convexify(p, gg, 0.0, off, kmax=10, tol=0.0)
    assert int(out["iters"].cpu()[0]) == 2
    axes = [gg.lo[c] + np.arange(gg.n[c]) * gg.delta[c] for c in range(4)]
    P = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 4)
    a = np.where(np.abs(P[:, 0]) <= 1.0, 0.0, (P[:, 0] ** 2 - 1.0) ** 2)
    exact = a + P[:, 1] ** 2 + P[:, 2] ** 2 + (P[:, 3] - 1.0) ** 2
    np.testing.assert_allclose(out["W"].cpu().numpy(), exact, rtol=0, atol=1e-14)
    f0 = out["forest"].cpu().numpy()[0]
    inner = np.abs(P[:, 0]) < 1.0
    assert np.all(f0[inner, 0] == 0)
    assert out["decs"].cpu().numpy()[1] == 0.0


# ---------------------------------------------------------------- STVK, d = 3

STVK61 = dict(diag=(0.1, 2.0), off=(-2.0, 2.0), delta=(0.1, 0.1), beta=0.07)
GRID3D = dict(diag=(1.0, 3.4), off=(-0.15, 0.15), delta=(0.15, 0.15))


def _load_npz(name):
    import json

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"{name}.npz")
    g = dict(np.load(path))
    g["meta"] = json.loads(str(g["meta"]))
    return g


@pytest.mark.parametrize("case", ["stvk2d", "stvk2d_kept", "nh3d", "stvk3d"])
def test_grid_energies_of_both_dimensions_match_oracle(cv, orc, case):
    """W^0 of Eq. (2.2) (plane strain and 3-D) and of Eq. (2.3) in 3-D, with
    det F <= 0 excluded or kept, against the oracle at every grid point."""
    from paper_2211_14318_gb300 import api

    energy, rule = {"stvk2d": (2, 0), "stvk2d_kept": (2, 1), "nh3d": (0, 0), "stvk3d": (2, 0)}[case]
    if case.endswith("3d"):
        go = orc.Grid.from_bounds(GRID3D["diag"], GRID3D["off"], GRID3D["delta"], dim=3)
        gg = api.GridSpec.from_bounds(GRID3D["diag"], GRID3D["off"], GRID3D["delta"], dim=3)
    else:
        go = orc.Grid.from_bounds(STVK61["diag"], STVK61["off"], STVK61["delta"])
        gg = api.GridSpec.from_bounds(STVK61["diag"], STVK61["off"], STVK61["delta"])
    mat = orc.Material(NH61["mu"], NH61["lam"], NH61["Dinf"], NH61["D0"], energy=energy)
    Wo = orc.grid_energy(mat, go, 0.07, rule=rule)
    Wg = cv.grid_energy(_params(api, energy=energy), gg, 0.07, rule).cpu().numpy()
    assert np.array_equal(np.isnan(Wg), np.isnan(Wo))
    f = np.isfinite(Wo)
    assert f.sum() > 0.4 * f.size
    assert np.max(np.abs(Wg[f] - Wo[f]) / (1.0 + np.abs(Wo[f]))) < 1e-13
    if case == "stvk2d":
        assert (~f).sum() > 0


def test_stvk_study_steps_bit_exact_and_device_loop(cv, orc):
    """The STVK study of Sec. 6.1 (672,400 points, Eq. 2.2 kept where
    det F <= 0): three steps from the oracle's iterates bit for bit, and the
    device loop against the stored oracle run (steps, decreases, W^K)."""
    from paper_2211_14318_gb300 import api

    go = orc.Grid.from_bounds(STVK61["diag"], STVK61["off"], STVK61["delta"])
    gg = api.GridSpec.from_bounds(STVK61["diag"], STVK61["off"], STVK61["delta"])
    mat = orc.Material(NH61["mu"], NH61["lam"], NH61["Dinf"], NH61["D0"], energy=2)
    off = api.grid_r11(2)
    W = orc.grid_energy(mat, go, STVK61["beta"], rule=1)
    for _ in range(3):
        Wo, d, lm, lp, dec = orc.grid_step(go, off, W)
        Wn, lam, decg = cv.grid_step(gg, off, W)
        lam = lam.cpu().numpy()
        assert _eq_nan(Wn.cpu().numpy(), Wo)
        assert np.array_equal(lam, np.stack([d, lm, lp], axis=1))
        assert float(decg.cpu()[0]) == dec
        W = Wo
    gold = _load_npz("stvk61")
    out = cv.grid_convexify(_params(api, energy=2), gg, STVK61["beta"], off, kmax=20, tol=1e-4,
                            det_rule=1)
    K = int(out["iters"].cpu()[0])
    assert K == gold["decs"].size == 11
    assert np.max(np.abs(out["decs"].cpu().numpy()[:K] - gold["decs"])) < 1e-12
    WK = out["W"].cpu().numpy()[gold["idx"]]
    assert np.max(np.abs(WK - gold["W_K"]) / (1 + np.abs(gold["W_K"]))) < 1e-12


def test_nine_dimensional_steps_bit_exact(cv, orc):
    """d = 3: a 5^3 x 3^6 grid on the stretches 1.0 .. 1.6 of the Sec. 6.8
    study (3-D NH and 3-D STVK, where both relax),
    two steps of Eq. (4.3) along the 169 directions from the oracle's
    iterates, bit for bit; one run with a chunk of 7 directions."""
    from paper_2211_14318_gb300 import api

    n = (5, 3, 3, 3, 5, 3, 3, 3, 5)
    lo = (1.0, -0.15, -0.15, -0.15, 1.0, -0.15, -0.15, -0.15, 1.0)
    de = (0.15, 0.15, 0.15, 0.15, 0.15, 0.15, 0.15, 0.15, 0.15)
    go, gg = _both_grids(orc, api, n, lo, de)
    off = api.grid_r11(3)
    assert (off == orc.r11_directions(3)).all()
    old = os.environ.get("CVX_GRID_CHUNK_BYTES")
    try:
        for energy, chunk in ((0, None), (2, str(7 * 12 * go.count))):
            if chunk:
                os.environ["CVX_GRID_CHUNK_BYTES"] = chunk
            mat = orc.Material(NH61["mu"], NH61["lam"], NH61["Dinf"], NH61["D0"], energy=energy)
            W = orc.grid_energy(mat, go, 0.0625)
            splits = 0
            for _ in range(2):
                Wo, d, lm, lp, dec = orc.grid_step(go, off, W)
                Wn, lam, decg = cv.grid_step(gg, off, W)
                lam = lam.cpu().numpy()
                assert _eq_nan(Wn.cpu().numpy(), Wo)
                assert np.array_equal(lam, np.stack([d, lm, lp], axis=1))
                assert float(decg.cpu()[0]) == dec
                splits += int((d >= 0).sum())
                W = Wo
            assert splits > 0
    finally:
        if old is None:
            os.environ.pop("CVX_GRID_CHUNK_BYTES", None)
        else:
            os.environ["CVX_GRID_CHUNK_BYTES"] = old


def test_nine_dimensional_study_reproduces_the_printed_curves(cv, orc):
    """Sec. 6.8 on the device: the 3,581,577-point grid of Table
    tab:3Dconvexification with the 169 directions, to tol 1e-4.  Steps,
    decreases and W^K (4,096 grid points and the uni-, bi- and triaxial paths)
    against the stored oracle run within 1e-12, the paths against the printed
    relaxed curves within 1e-5; Algorithms 2 and 3 at the path points (grid
    points: one corner each) give W^K, and at off-grid points the
    interpolated W^K."""
    from paper_2211_14318_gb300 import api
    from conftest import load_golden

    gold = _load_npz("grid3d")
    printed = load_golden("nh3d_paths.txt")
    gg = api.GridSpec.from_bounds(GRID3D["diag"], GRID3D["off"], GRID3D["delta"], dim=3)
    off = api.grid_r11(3)
    p = _params(api)
    beta = gold["meta"]["beta"]
    out = cv.grid_convexify(p, gg, beta, off, kmax=20, tol=1e-4)
    K = int(out["iters"].cpu()[0])
    assert K == gold["decs"].size == 5
    assert np.max(np.abs(out["decs"].cpu().numpy()[:K] - gold["decs"])) < 1e-12
    WK = out["W"].cpu().numpy()
    for a, b in ((WK[gold["idx"]], gold["W_K"]), (WK[gold["paths"]], gold["W_paths"])):
        assert np.max(np.abs(a - b) / (1 + np.abs(b))) < 1e-12
    assert np.max(np.abs(WK[gold["paths"][1]] - printed[:, 4])) < 1e-5
    assert np.max(np.abs(WK[gold["paths"][2]] - printed[:, 6])) < 1e-5
    # the path points as query points
    axes = [gg.lo[c] + np.arange(gg.n[c]) * gg.delta[c] for c in range(9)]
    ii = np.array(np.unravel_index(gold["paths"].reshape(-1), gg.n)).T
    Fp = np.stack([axes[c][ii[:, c]] for c in range(9)], axis=1)
    wi, wt, P, nl = cv.grid_query(p, gg, beta, off, out["W"], out["forest"][:K], Fp)
    wi, wt = wi.cpu().numpy(), wt.cpu().numpy()
    assert np.array_equal(wi, WK[gold["paths"].reshape(-1)])
    assert np.max(np.abs(wt - wi) / (1 + np.abs(wi))) < 1e-12
    rng = np.random.default_rng(9)
    lo = np.array(gg.lo)
    hi = lo + (np.array(gg.n) - 1) * np.array(gg.delta)
    Fr = rng.uniform(lo, hi, size=(256, 9))
    wi, wt, P, nl = cv.grid_query(p, gg, beta, off, out["W"], out["forest"][:K], Fr)
    wi, wt, nl = wi.cpu().numpy(), wt.cpu().numpy(), nl.cpu().numpy()
    assert np.max(np.abs(wt - wi) / (1 + np.abs(wi))) < 1e-12
    assert np.all(nl >= 512)  # 2^9 interpolation corners
