"""convexify_batch: several problems of uneven sizes and different parameters
in one pipeline run (a CUDA graph), against the FP64 oracle per problem and
against convexify_points; graph replay; the launch-shape autotuner."""
import os

import numpy as np
import pytest

from test_gpu_parity import MAT, TIE, _omat, _rel, cv  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

HARD = 2 | 16  # status bits TIE | OVERFLOW


def _problems(orc):
    from paper_2211_14318_gb300 import api, inputs

    vecs = [(1, 0), (0, 1), (1, 1), (1, -1)]
    r11 = np.array([[a[0], a[1], b[0], b[1]] for a in vecs for b in vecs], dtype=np.float64)
    mat = _omat(orc)
    specs = [
        (api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT), 53, 0),
        (api.Params(n_theta_a=7, n_theta_b=9, line_points=77, t_half=0.6, depth=3, **MAT), 29, 1),
        (api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT), 0, 2),
        (api.Params(line_points=101, t_half=0.4, depth=1, dirs=r11, **MAT), 17, 3),
        (api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=0, **MAT), 5, 4),
        (api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT), 31, 5),
    ]
    out = []
    for p, n, seed in specs:
        F, Fp = inputs.material_points(max(n, 1), seed=40 + seed, lam_hi=1.9)
        F = F[:n]
        beta = orc.history_update(mat, Fp)[:n]
        out.append((p, F, beta))
    return out


def _oracle(orc, p, F, beta):
    from paper_2211_14318_gb300 import api

    mat = _omat(orc, energy=p.energy)
    dirs = p.dirs if p.dirs is not None else orc.angle_directions(p.n_theta_a, p.n_theta_b)
    sc = orc.Scan(dirs, p.line_points, p.t_half, p.depth, round32=False)
    WRo, Po, tro, sto = orc.convexify(mat, sc, F, beta)
    untied = np.array([all(tro[k, i]["margin"] > TIE for i in range(tro.shape[1])
                           if tro[k, i]["flags"] & orc.SCANNED) for k in range(F.shape[0])],
                      dtype=bool)
    return WRo, Po, sto, untied


def test_batch_matches_oracle_and_single_calls(cv, orc):
    probs = _problems(orc)
    res = cv.convexify_batch(probs)
    for (p, F, beta), r in zip(probs, res):
        n = F.shape[0]
        WR, P, st = (r["W_R"].cpu().numpy(), r["P"].cpu().numpy(), r["status"].cpu().numpy())
        assert WR.shape == (n,)
        if n == 0:
            continue
        WRo, Po, sto, u = _oracle(orc, p, F, beta)
        assert np.all((st & 1) == (sto & 1))
        assert np.max(_rel(WR[u], WRo[u]), initial=0) < 1e-6
        Pn = np.linalg.norm(Po, axis=1)
        assert np.max(np.linalg.norm(P[u] - Po[u], axis=1) / (1e-8 + Pn[u]), initial=0) < 1e-5
        one = cv.convexify_points(p, F, beta)
        st1 = one["status"].cpu().numpy()
        clean = ((st | st1) & HARD) == 0
        np.testing.assert_array_equal(WR[clean], one["W_R"].cpu().numpy()[clean])
        np.testing.assert_array_equal(P[clean], one["P"].cpu().numpy()[clean])
        if p.depth == 0:
            W0, P0 = cv.energy(p, F, beta)
            np.testing.assert_allclose(WR, W0.cpu().numpy(), rtol=1e-11, atol=0)


def test_graph_replay_reads_current_inputs(cv, orc):
    """Second call with the same tensors replays the captured graph; the graph
    reads F and beta_k at replay time, so new values in the same tensors give
    the new results."""
    import torch

    from paper_2211_14318_gb300 import inputs

    probs = _problems(orc)
    dev = torch.device("cuda", 0)
    tens = [(p, torch.as_tensor(F, device=dev), torch.as_tensor(b, device=dev)) for p, F, b in probs]
    outs = cv.convexify_batch(tens)
    first = [o["W_R"].clone() for o in outs]
    cv.convexify_batch(tens, outs=outs)
    for a, o in zip(first, outs):
        assert torch.equal(a, o["W_R"])
    mat = _omat(orc)
    for k, (p, F, b) in enumerate(tens):
        if F.shape[0] == 0:
            continue
        F2, Fp2 = inputs.material_points(F.shape[0], seed=90 + k, lam_hi=1.9)
        F.copy_(torch.as_tensor(F2))
        b.copy_(torch.as_tensor(orc.history_update(mat, Fp2)))
    outs2 = cv.convexify_batch(tens, outs=outs)
    assert all(o2["W_R"].data_ptr() == o["W_R"].data_ptr() for o, o2 in zip(outs, outs2))
    for (p, F, b), o in zip(tens, outs2):
        if F.shape[0] == 0:
            continue
        one = cv.convexify_points(p, F, b)
        st, st1 = o["status"].cpu().numpy(), one["status"].cpu().numpy()
        clean = ((st | st1) & HARD) == 0
        assert clean.mean() > 0.5
        np.testing.assert_array_equal(o["W_R"].cpu().numpy()[clean], one["W_R"].cpu().numpy()[clean])


def test_autotuner_choice_and_cache_file(orc, tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2211_14318_gb300 import api

    path = tmp_path / "tune.json"
    os.environ["CVX_AUTOTUNE_CACHE"] = str(path)
    try:
        probs = _problems(orc)
        c1 = api.Convexifier(0)
        c1.convexify_batch(probs)
        w, cap, cached = c1.batch_tuning()
        # warps 4 or 8: the warp-per-line scan (item caps 256, 1024, none);
        # warps 0: the lane-per-line scan (item caps 64, 128, none)
        assert (w, cap) in {(4, 0), (4, 256), (4, 1024), (8, 0), (8, 256), (8, 1024),
                            (0, 0), (0, 64), (0, 128)} and not cached
        c1.close()
        assert path.exists() and f"[{w}, {cap}]" in path.read_text()
        c2 = api.Convexifier(0)
        c2.convexify_batch(probs)
        assert c2.batch_tuning() == (w, cap, True)
        c2.close()
    finally:
        del os.environ["CVX_AUTOTUNE_CACHE"]


def test_full_size_batch_sampled_against_oracle(cv, orc):
    """The batched workload at full size: 256 meshes with log-uniform point
    counts in [1e3, 1e5] (about 5.5 M points), per-problem stretch in
    [1.1, 1.8], angle grid 32^2 or 64^2, line 513 or 1025, depth 2 or 3, in one
    autotuned, graph-captured run; the oracle recomputes two sampled points
    of each of 12 problems one by one."""
    import torch

    from paper_2211_14318_gb300 import api, inputs

    probs = inputs.batch_problems(256, seed=0)
    mat = _omat(orc)
    dev = torch.device("cuda", 0)
    items, total = [], 0
    for pr in probs:
        p = api.Params(n_theta_a=pr.n_angle, n_theta_b=pr.n_angle, line_points=pr.L,
                       depth=pr.depth, **MAT)
        beta = cv.history_update(p, pr.F_prev)
        items.append((p, torch.as_tensor(pr.F, device=dev), beta))
        total += pr.F.shape[0]
    assert 3_000_000 < total < 9_000_000
    res = cv.convexify_batch(items)
    torch.cuda.synchronize()
    w, cap, cached = cv.batch_tuning()
    assert w in (0, 4, 8)  # 0: the lane-per-line scan
    rng = np.random.default_rng(1)
    checked = 0
    for k in rng.choice(256, 12, replace=False):
        p, F, beta = items[k]
        n = F.shape[0]
        idx = rng.choice(n, 2, replace=False)
        Fh = F.cpu().numpy()[idx]
        bh = beta.cpu().numpy()[idx]
        sc = orc.Scan(orc.angle_directions(p.n_theta_a, p.n_theta_b), p.line_points, p.t_half,
                      p.depth, round32=False)
        WRo, Po, tro, sto = orc.convexify(mat, sc, Fh, bh)
        WR = res[k]["W_R"].cpu().numpy()[idx]
        P = res[k]["P"].cpu().numpy()[idx]
        for j in range(2):
            sc_nodes = tro[j]["flags"] & orc.SCANNED > 0
            if np.any(tro[j]["margin"][sc_nodes] <= TIE):
                continue
            assert _rel(np.array([WR[j]]), np.array([WRo[j]]))[0] < 1e-6, (k, j)
            assert np.linalg.norm(P[j] - Po[j]) / (1e-8 + np.linalg.norm(Po[j])) < 1e-5
            checked += 1
    assert checked >= 16


def test_newton_flag_through_batch_and_static_entry(cv, orc):
    """CVX_FLAG_REFINE_NEWTON reaches the kernels through convexify_batch and
    convexify_points_static: the double well's refined split (exact
    common tangent at x = +-1, off the line grid) comes out of every entry."""
    from paper_2211_14318_gb300 import api

    p = api.Params(energy=api.ENERGY_DOUBLE_WELL, n_theta_a=8, n_theta_b=8, line_points=201,
                   t_half=1.5, depth=1, newton=True)
    F = np.array([[0.3, 0, 0, 1.0], [-0.2, 0, 0, 1.0]])
    one = cv.convexify_points(p, F, np.zeros(2))
    bat = cv.convexify_batch([(p, F, np.zeros(2))], want_root=True)[0]
    sta = api.convexify_points_static(p, F, np.zeros(2))
    for r in (one, bat, sta):
        np.testing.assert_allclose(r["W_R"].cpu().numpy(), [0.0, 0.0], atol=1e-13)
    root = api.root_numpy(bat["root"], 2)
    np.testing.assert_allclose(root["F_plus"][:, 0], [1.0, 1.0], atol=1e-12)
    np.testing.assert_allclose(root["F_minus"][:, 0], [-1.0, -1.0], atol=1e-12)
    np.testing.assert_allclose(root["xi"], [0.65, 0.4], atol=1e-12)


def test_many_tiny_problems(cv, orc):
    """400 problems of 0 to 3 points with alternating parameters in one batch:
    every point's W^R, P and status equal the single-problem call's (the
    problem table's point offsets, empty problems and per-problem depth)."""
    from paper_2211_14318_gb300 import api, inputs

    rng = np.random.default_rng(7)
    F, Fp = inputs.material_points(1200, seed=70)
    beta = orc.history_update(_omat(orc), Fp)
    items, off = [], 0
    for k in range(400):
        m = int(rng.integers(0, 4))
        p = api.Params(n_theta_a=8 + 4 * (k % 2), n_theta_b=8, line_points=61 + 40 * (k % 3),
                       depth=k % 3, **MAT)
        items.append((p, F[off:off + m], beta[off:off + m]))
        off += m
    res = cv.convexify_batch(items)
    for (p, Fk, bk), r in zip(items, res):
        if Fk.shape[0] == 0:
            assert r["W_R"].numel() == 0
            continue
        one = cv.convexify_points(p, Fk, bk)
        st, st1 = r["status"].cpu().numpy(), one["status"].cpu().numpy()
        clean = ((st | st1) & HARD) == 0
        np.testing.assert_array_equal(st[clean], st1[clean])
        np.testing.assert_array_equal(r["W_R"].cpu().numpy()[clean], one["W_R"].cpu().numpy()[clean])
        np.testing.assert_array_equal(r["P"].cpu().numpy()[clean], one["P"].cpu().numpy()[clean])
