"""The surrogate network on the tensor cores against the FP64 oracle
(oracle/mlp.py): the tcgen05 GEMM against an FP64 matrix product of the same
bf16 operands, the forward pass and the loss gradient against the oracle with
the same bf16 rounding points, training, save/load.

Tolerances.  GEMM: FP32 accumulation of K products, |err| <= K 2^-24
sum_k |a_k b_k| (bound used with a factor 4).  Forward / gradient: the GPU and
the bf16-emulating oracle round the same operands; they differ by the FP32
vs FP64 accumulation (~1e-6 relative) and by the rare activation whose FP32
value lies within that distance of a bf16 rounding boundary, which moves it
by one bf16 step (2^-8 relative).  Bars: outputs within 2e-3 (1 + |o|);
gradient blocks within 2e-2 relative in norm with cosine > 0.9995."""
import math

import numpy as np
import pytest

from oracle import mlp
from test_gpu_parity import MAT, _omat, cv  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu


def _bf16_tensor(rng, shape, scale=1.0):
    import torch

    return torch.tensor(rng.normal(0, scale, shape), dtype=torch.float32).to(torch.bfloat16)


@pytest.mark.parametrize("M,N,K", [(128, 256, 256), (200, 16, 48), (300, 256, 16), (1, 16, 16),
                                   (129, 300, 64), (513, 7, 272)])
def test_gemm_bf16_matches_fp64_product(cv, M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = _bf16_tensor(rng, (M, K))
    B = _bf16_tensor(rng, (N, K))
    C = cv.gemm_bf16(A, B).cpu().numpy().astype(np.float64)
    a = A.to(dtype=__import__("torch").float64).numpy()
    b = B.to(dtype=__import__("torch").float64).numpy()
    ref = a @ b.T
    bound = 4 * K * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)


def _net_inputs(orc, n, seed):
    from paper_2211_14318_gb300 import inputs

    F, Fp = inputs.material_points(n, seed=seed, lam_hi=2.0)
    beta = orc.history_update(_omat(orc), Fp)
    X = mlp.features(F, beta)
    mean, std = X.mean(axis=0), X.std(axis=0) + 1e-3
    return X, mean.astype(np.float32).astype(np.float64), std.astype(np.float32).astype(np.float64)


def _set(cv, seed):
    flat = mlp.init_params(seed).astype(np.float32).astype(np.float64)
    return flat


def test_forward_matches_oracle(cv, orc):
    X, mean, std = _net_inputs(orc, 300, 21)
    flat = _set(cv, 4)
    cv.surrogate_set_weights(flat, mean, std)
    out = cv.surrogate_forward(X.astype(np.float32)).cpu().numpy().astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    ref, _ = mlp.forward(flat, X32, mean, 1.0 / (1.0 / std.astype(np.float32)).astype(np.float64), bf=True)
    assert np.max(np.abs(out - ref) / (1 + np.abs(ref))) < 2e-3
    ref64, _ = mlp.forward(flat, X32, mean, std)
    assert np.max(np.abs(out - ref64) / (1 + np.abs(ref64))) < 5e-2
    p, m, s = cv.surrogate_get_weights()
    np.testing.assert_array_equal(p, flat.astype(np.float32))


def _labels(rng, n):
    Y = np.column_stack([rng.uniform(0, math.pi, (n, 2)), rng.uniform(0.05, 0.95, n),
                         rng.normal(0, 0.3, (n, 4))])
    Y[::5, :3] = np.nan
    return Y


def test_gradient_matches_oracle(cv, orc):
    X, mean, std = _net_inputs(orc, 400, 22)
    flat = _set(cv, 5)
    cv.surrogate_set_weights(flat, mean, std)
    rng = np.random.default_rng(6)
    Y = _labels(rng, 400)
    loss, grad = cv.surrogate_loss_grad(X.astype(np.float32), Y.astype(np.float32))
    loss = loss.item()
    g = grad.cpu().numpy().astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    istd = (1.0 / std.astype(np.float32)).astype(np.float32).astype(np.float64)
    out, cache = mlp.forward(flat, X32, mean, 1.0 / istd, bf=True)
    L, dout = mlp.loss_and_grad(out, Y.astype(np.float32).astype(np.float64))
    ref = mlp.backward(flat, cache, dout, bf=True)
    assert abs(loss - L) < 1e-3 * (1 + abs(L))
    o = 0
    for shp in mlp.SHAPES:
        k = int(np.prod(shp))
        a, b = g[o:o + k], ref[o:o + k]
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        assert rel < 2e-2 and cos > 0.9995, (shp, rel, cos)
        o += k


def test_training_reduces_loss_and_save_load(cv, orc, tmp_path):
    rng = np.random.default_rng(8)
    n = 4096
    X = np.column_stack([rng.normal(1, 0.2, (n, 4)), rng.uniform(0, 0.3, n), rng.normal(0, 0.1, n)])
    # a smooth target the network can learn
    th = np.mod(np.arctan2(X[:, 2], X[:, 0]) + 1.0, math.pi)
    Y = np.column_stack([th, np.mod(th + 0.3 * X[:, 1], math.pi), 1 / (1 + np.exp(-X[:, 4] * 5)),
                         X[:, :4] - 1.0])
    Y[::7, :3] = np.nan
    log = cv.surrogate_train(X.astype(np.float32), Y.astype(np.float32), epochs=25, batch=512,
                             lr=2e-3, init=True, seed=3)
    assert np.all(np.isfinite(log))
    assert log[-1] < 0.25 * log[0], log
    out1 = cv.surrogate_forward(X[:64].astype(np.float32)).cpu().numpy()
    path = str(tmp_path / "sur.bin")
    cv.surrogate_save(path)
    from paper_2211_14318_gb300 import api

    c2 = api.Convexifier(0)
    c2.surrogate_load(path)
    out2 = c2.surrogate_forward(X[:64].astype(np.float32)).cpu().numpy()
    c2.close()
    np.testing.assert_array_equal(out1, out2)


# ---------------------------------------------------------------- proposals
TIE = 1e-11


def _constant_net(theta_a, theta_b, xi, jump):
    parts = [np.zeros(s) for s in mlp.SHAPES]
    parts[9] = np.array([theta_a, theta_b, math.log(xi / (1 - xi)), *jump])
    return mlp.flatten(parts).astype(np.float32).astype(np.float64)


def test_labels_match_oracle_labels(cv, orc):
    """surrogate_labels on the GPU's trees against oracle.mlp.labels_from_tree
    on the oracle's trees of the same points (untied points only)."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(24, seed=33)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    X, Y = cv.surrogate_labels(p, beta, out["tree"], 24)
    X, Y = X.cpu().numpy(), Y.cpu().numpy()
    sc = orc.Scan(orc.angle_directions(16, 16), 201, 0.5, 2)
    _, _, tro, _ = orc.convexify(mat, sc, F, beta)
    Xo, Yo = mlp.labels_from_tree(tro, F, beta, (16, 16), (orc.SCANNED, orc.LAMINATED))
    tied = np.array([any(tro[q, i]["margin"] <= TIE for i in range(7) if tro[q, i]["flags"] & orc.SCANNED)
                     for q in range(24)])
    tg = api.tree_numpy(out["tree"], 24, 7)
    per_g = [int(np.sum(tg[q]["flags"] & api.NODE_SCANNED > 0)) for q in range(24)]
    per_o = [int(np.sum(tro[q]["flags"] & orc.SCANNED > 0)) for q in range(24)]
    assert X.shape[0] == sum(per_g) and Xo.shape[0] == sum(per_o)
    og = oo = 0
    checked = 0
    for q in range(24):
        if not tied[q]:
            assert per_g[q] == per_o[q]
            sg, so = slice(og, og + per_g[q]), slice(oo, oo + per_o[q])
            np.testing.assert_allclose(X[sg], Xo[so].astype(np.float32), rtol=1e-6, atol=1e-6)
            np.testing.assert_allclose(Y[sg], Yo[so].astype(np.float32), rtol=1e-6, atol=1e-6)
            checked += 1
        og += per_g[q]
        oo += per_o[q]
    assert checked >= 12


def test_propose_zero_tolerance_is_the_full_scan(cv, orc):
    """gap_tol = 0: every node falls back, so the proposed form equals
    convexify_points bit for bit (points without tie / overflow flags)."""
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(64, seed=34)
    beta = orc.history_update(_omat(orc), Fp)
    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    cv.surrogate_set_weights(mlp.init_params(9), np.zeros(6), np.ones(6))
    r = cv.surrogate_propose(p, F, beta, window=2, gap_tol=0.0)
    q = cv.convexify_points(p, F, beta)
    st, st1 = r["status"].cpu().numpy(), q["status"].cpu().numpy()
    clean = ((st | st1) & (2 | 16)) == 0
    assert clean.mean() > 0.5
    np.testing.assert_array_equal(r["W_R"].cpu().numpy()[clean], q["W_R"].cpu().numpy()[clean])
    np.testing.assert_array_equal(r["P"].cpu().numpy()[clean], q["P"].cpu().numpy()[clean])
    assert np.all(r["fell_back"].cpu().numpy() == 1)


def test_propose_constant_network_matches_oracle(cv, orc):
    """A fixed network (biases only) proposing point 0's own full-scan
    laminate: the GPU's window / fallback decisions and results against the
    proposed-form oracle with the same network, depth 1 and 2."""
    from oracle import surrogate as osur
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(12, seed=35)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    Na = Nb = 12
    sc = orc.Scan(orc.angle_directions(Na, Nb), 151, 0.5, 1)
    _, _, tro, _ = orc.convexify(mat, sc, F, beta)
    k = next(q for q in range(12) if tro[q, 0]["flags"] & orc.LAMINATED)
    r0 = tro[k, 0]
    d = int(r0["dir"])
    flat = _constant_net(math.pi * (d // Nb) / Na, math.pi * (d % Nb) / Nb, r0["xi"],
                         tro[k, 2]["F"] - tro[k, 1]["F"])
    cv.surrogate_set_weights(flat, np.zeros(6), np.ones(6))
    for depth, one_sided in ((1, False), (2, False), (2, True)):
        p = api.Params(n_theta_a=Na, n_theta_b=Nb, line_points=151, depth=depth,
                       gap_one_sided=one_sided, **MAT)
        r = cv.surrogate_propose(p, F, beta, window=2, gap_tol=1e-5, want_tree=True)
        WRo, Po, trees = osur.propose_convexify(orc, mat, Na, Nb, 151, 0.5, depth, 2, 1e-5, flat,
                                                np.zeros(6), np.ones(6), F, beta,
                                                one_sided=one_sided)
        tg = api.tree_numpy(r["tree"], 12, p.tree_size)
        WR = r["W_R"].cpu().numpy()
        fb = r["fell_back"].cpu().numpy()
        assert fb[k] == 0 or depth > 1
        for q in range(12):
            clear = all(rec.get("margin", np.inf) > TIE and rec.get("window_margin", np.inf) > TIE
                        and abs(rec.get("gap", 0.0) - 1e-5) > 1e-6 and np.isfinite(rec.get("gap", 0.0))
                        for rec in trees[q].values() if rec["flags"] & orc.SCANNED)
            if not clear:
                continue
            ofb = any(rec["flags"] & osur.FALLBACK for rec in trees[q].values())
            assert bool(fb[q]) == ofb, (depth, q)
            for i, rec in trees[q].items():
                if rec["flags"] & orc.LAMINATED:
                    assert tg[q, i]["dir"] == rec["dir"], (depth, q, i)
                    assert bool(tg[q, i]["flags"] & api.NODE_FALLBACK) == bool(rec["flags"] & osur.FALLBACK)
            assert abs(WR[q] - WRo[q]) <= 1e-6 * (1e-8 + abs(WRo[q]))
        if depth == 1:
            assert fb[k] == 0 and abs(WR[k] - WRo[k]) <= 1e-12 * abs(WRo[k])


def test_trained_network_gains_over_untrained(cv, orc):
    """Train on labels from the GPU's own full scans (points drawn like the
    16 x 16, L = 201 material-point workload with lambda in [1, 2]), then on
    held-out points compare the window-only form (window 2, fallback on the
    border only) with a trained and an untrained network: the trained one
    falls back less and its W^R is closer to the full scan's."""
    from paper_2211_14318_gb300 import api, inputs

    mat = _omat(orc)
    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    F, Fp = inputs.material_points(6000, seed=40, lam_hi=2.0)
    beta = orc.history_update(mat, Fp)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    X, Y = cv.surrogate_labels(p, beta, out["tree"], F.shape[0])
    log = cv.surrogate_train(X, Y, epochs=40, batch=1024, lr=2e-3, init=True, seed=1)
    assert log[-1] < 0.5 * log[0]
    Ft, Fpt = inputs.material_points(512, seed=41, lam_hi=2.0)
    bt = orc.history_update(mat, Fpt)
    ref = cv.convexify_points(p, Ft, bt)["W_R"].cpu().numpy()

    def run():
        cv.stats(reset=True)
        r = cv.surrogate_propose(p, Ft, bt, window=2, gap_tol=1e30)
        s = cv.stats(reset=True)
        err = np.abs(r["W_R"].cpu().numpy() - ref) / (1e-8 + np.abs(ref))
        return r["fell_back"].cpu().numpy().mean(), np.quantile(err, 0.9), s

    fb_t, e_t, s_t = run()
    w, m, sd = cv.surrogate_get_weights()
    cv.surrogate_set_weights(mlp.init_params(123), m, sd)
    fb_u, e_u, s_u = run()
    assert fb_t < fb_u and e_t <= e_u, (fb_t, fb_u, e_t, e_u)
    assert s_t["lines"] < 0.5 * s_u["lines"] + 1, (s_t["lines"], s_u["lines"])


def test_full_size_training_and_held_out_quality(cv, orc):
    """The training workload at full size: 2 M samples labelled by the full
    scan (16 x 16 angles, L = 201, depth 2, lambda in [1, 2]), 10 epochs of
    batch 8,192; on 100,000 held-out points the proposed cell equals the full
    scan's direction on >= 80 % of laminated points and lies within one cell
    on >= 99 %.  (Training accumulates gradients with FP32 atomics, so the
    exact-cell fraction varies from run to run; 0.83 to 0.87 were seen.)"""
    import torch

    from paper_2211_14318_gb300 import api, inputs

    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    F, Fp = inputs.surrogate_inputs(1_000_000, seed=200)
    beta = cv.history_update(p, Fp)
    out = cv.convexify_points(p, F, beta, want_tree=True)
    X, Y = cv.surrogate_labels(p, beta, out["tree"], F.shape[0])
    assert X.shape[0] >= 2_000_000
    log = cv.surrogate_train(X[:2_000_000], Y[:2_000_000], epochs=10, batch=8192, lr=1e-3,
                             init=True, seed=0)
    assert log[-1] < 0.2 * log[0]
    Fh, Fph = inputs.surrogate_inputs(100_000, seed=201)
    bh = cv.history_update(p, Fph)
    Xh = torch.as_tensor(mlp.features(Fh, bh.cpu().numpy()), dtype=torch.float32, device="cuda")
    o = cv.surrogate_forward(Xh).cpu().numpy()
    p1 = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=1, **MAT)
    root = api.root_numpy(cv.convexify_points(p1, Fh, bh, want_root=True)["root"], Fh.shape[0])
    lam = root["laminated"] == 1
    ia, ib, *_ = mlp.decode(o.astype(np.float64), Fh, 16, 16)

    def cdist(x, y):
        d = np.abs(x - y) % 16
        return np.minimum(d, 16 - d)

    da, db = cdist(ia, root["dir"] // 16)[lam], cdist(ib, root["dir"] % 16)[lam]
    assert lam.sum() > 50_000
    assert np.mean((da == 0) & (db == 0)) >= 0.80
    assert np.mean((da <= 1) & (db <= 1)) >= 0.99


def test_propose_recentring_matches_oracle(cv, orc):
    """Window re-centring: a fixed network proposing a cell three cells away
    from point k's full-scan direction, window half-width 1, up to 4
    re-centrings; the GPU's fallback decisions, directions and W^R against
    the proposed-form oracle with the same network and re-centring rule."""
    from oracle import surrogate as osur
    from paper_2211_14318_gb300 import api, inputs

    F, Fp = inputs.material_points(16, seed=37)
    mat = _omat(orc)
    beta = orc.history_update(mat, Fp)
    Na = Nb = 12
    sc = orc.Scan(orc.angle_directions(Na, Nb), 151, 0.5, 1)
    _, _, tro, _ = orc.convexify(mat, sc, F, beta)
    k = next(q for q in range(16) if tro[q, 0]["flags"] & orc.LAMINATED)
    r0 = tro[k, 0]
    d = int(r0["dir"])
    flat = _constant_net(math.pi * ((d // Nb + 3) % Na) / Na, math.pi * (d % Nb) / Nb, r0["xi"],
                         tro[k, 2]["F"] - tro[k, 1]["F"])
    cv.surrogate_set_weights(flat, np.zeros(6), np.ones(6))
    for depth, R in ((1, 4), (2, 4), (2, 0)):
        p = api.Params(n_theta_a=Na, n_theta_b=Nb, line_points=151, depth=depth, recentre=R, **MAT)
        cv.stats(reset=True)
        r = cv.surrogate_propose(p, F, beta, window=1, gap_tol=1e30, want_tree=True)
        st = cv.stats(reset=True)
        WRo, Po, trees = osur.propose_convexify(orc, mat, Na, Nb, 151, 0.5, depth, 1, 1e30, flat,
                                                np.zeros(6), np.ones(6), F, beta, recentre=R)
        tg = api.tree_numpy(r["tree"], 16, p.tree_size)
        WR = r["W_R"].cpu().numpy()
        fb = r["fell_back"].cpu().numpy()
        n_rec = sum(rec.get("recentred", 0) for t in trees for rec in t.values())
        checked = 0
        for q in range(16):
            clear = all(rec.get("margin", np.inf) > TIE and rec.get("window_margin", np.inf) > TIE
                        for rec in trees[q].values() if rec["flags"] & orc.SCANNED)
            if not clear:
                continue
            ofb = any(rec["flags"] & osur.FALLBACK for rec in trees[q].values())
            assert bool(fb[q]) == ofb, (depth, R, q)
            for i, rec in trees[q].items():
                if rec["flags"] & orc.LAMINATED:
                    assert tg[q, i]["dir"] == rec["dir"], (depth, R, q, i)
                    assert bool(tg[q, i]["flags"] & api.NODE_FALLBACK) == bool(rec["flags"] & osur.FALLBACK)
            assert abs(WR[q] - WRo[q]) <= 1e-6 * (1e-8 + abs(WRo[q]))
            checked += 1
        assert checked >= 8
        if R == 0:
            assert st["recentred"] == 0
        else:
            assert st["recentred"] >= 1 and n_rec >= 1


def _twin_nodes(orc, n=48):
    """Level-2 nodes of a 16 x 16 load path at step 10 (with its history)
    whose full-scan hull over a 32 x 32 angle grid has mirrored twin basins
    about four cells apart, as points of their own; with their full-scan
    directions."""
    from paper_2211_14318_gb300 import inputs

    mat = _omat(orc)
    path = inputs.load_path(16, n_steps=20, stretch_end=1.8, seed=7)
    beta = None
    for k in range(9):
        beta = orc.history_update(mat, path[k], beta)
    dirs = orc.angle_directions(32, 32)
    _, _, tr, _ = orc.convexify(mat, orc.Scan(dirs, 151, 0.5, 3), path[9][:n], beta[:n])
    keep = [p for p in range(n) if tr[p, 6]["flags"] & orc.LAMINATED]
    F = np.array([tr[p, 6]["F"] for p in keep])
    b = np.array([beta[p] for p in keep])
    return mat, F, b, np.array([int(tr[p, 6]["dir"]) for p in keep])


def test_propose_mirror_window_matches_oracle(cv, orc):
    """CVX_FLAG_MIRROR_WINDOW: load-path nodes with twin basins, a fixed
    network proposing the mirror cell of the most common full-scan direction
    (so the window settles in the twin basin), window half-width 1 (mirror
    half-width 1), up to 4 re-centrings, depth 1 and 2.  The GPU's mirror
    queue, choices, fallbacks, directions and W^R against the proposed-form
    oracle with the same network; at depth 1 the mirror window returns the
    full scan's result on the nodes where it wins."""
    from oracle import surrogate as osur
    from paper_2211_14318_gb300 import api

    mat, F, b, d = _twin_nodes(orc)
    n = F.shape[0]
    Na = Nb = 32
    vals, cnts = np.unique(d, return_counts=True)
    d0 = int(vals[np.argmax(cnts)])
    k = int(np.nonzero(d == d0)[0][0])
    mc, _ = osur.mirror_cell(F[k], d0, Na, Nb)
    flat = _constant_net(math.pi * mc[0] / Na, math.pi * mc[1] / Nb, 0.5, np.zeros(4))
    cv.surrogate_set_weights(flat, np.zeros(6), np.ones(6))
    plain = cv.convexify_points(api.Params(n_theta_a=Na, n_theta_b=Nb, line_points=151, depth=1,
                                           **MAT), F, b)["W_R"].cpu().numpy()
    for depth in (1, 2):
        p = api.Params(n_theta_a=Na, n_theta_b=Nb, line_points=151, depth=depth, recentre=4,
                       mirror=True, **MAT)
        cv.stats(reset=True)
        r = cv.surrogate_propose(p, F, b, window=1, gap_tol=1e30, want_tree=True)
        st = cv.stats(reset=True)
        WRo, Po, trees = osur.propose_convexify(orc, mat, Na, Nb, 151, 0.5, depth, 1, 1e30, flat,
                                                np.zeros(6), np.ones(6), F, b, recentre=4,
                                                mirror=True)
        tg = api.tree_numpy(r["tree"], n, p.tree_size)
        WR = r["W_R"].cpu().numpy()
        fb = r["fell_back"].cpu().numpy()
        n_mirror = sum(1 for t in trees for rec in t.values()
                       if "mirror_center" in rec and not rec["mirror_inside"])
        n_won = sum(1 for t in trees for rec in t.values() if rec.get("mirror_won"))
        checked = won = 0
        for q in range(n):
            recs = [rec for rec in trees[q].values() if rec["flags"] & orc.SCANNED]
            clear = all(rec.get("margin", np.inf) > TIE and rec.get("window_margin", np.inf) > TIE
                        and rec.get("center_margin", 1.0) > 1e-9
                        and rec.get("mirror_center_margin", 1.0) > 1e-9
                        and rec.get("mirror_gap", np.inf) > TIE for rec in recs)
            if not clear:
                continue
            ofb = any(rec["flags"] & osur.FALLBACK for rec in recs)
            assert bool(fb[q]) == ofb, (depth, q)
            for i, rec in trees[q].items():
                if rec["flags"] & orc.LAMINATED:
                    assert tg[q, i]["dir"] == rec["dir"], (depth, q, i)
            assert abs(WR[q] - WRo[q]) <= 1e-12 * (1e-8 + abs(WRo[q])), (depth, q)
            if depth == 1 and trees[q][0].get("mirror_won") and not ofb:
                assert abs(WR[q] - plain[q]) <= 1e-12 * abs(plain[q])
                won += 1
            checked += 1
        assert checked >= n // 2
        assert abs(st["mirror_windows"] - n_mirror) <= n - checked
        assert abs(st["mirror_won"] - n_won) <= n - checked
        assert n_won >= 5 and st["mirror_won"] >= 5
        if depth == 1:
            assert won >= 5
