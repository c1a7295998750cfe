"""Pins of the FP64 surrogate-network oracle (oracle/mlp.py) against facts
fixed outside it: the normal CDF's tabulated values, bfloat16 rounding as
torch implements it, finite differences, an identity network that reduces to
scalar GELU iterates, and the laminates of oracle lamination trees."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_torch():
    import torch

    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 3, 2000), rng.normal(0, 1e-3, 500),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, 65504.0]])
    x32 = x.astype(np.float32)
    ref = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x32), ref)
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0  # tie -> even


def test_gelu_known_values():
    """gelu(z) = z Phi(z); Phi(1) = 0.8413447460685429, Phi(3) = 0.9986501019683699
    (standard normal table)."""
    z = np.array([0.0, 1.0, -1.0, 3.0])
    expect = np.array([0.0, 0.8413447460685429, -(1 - 0.8413447460685429), 3 * 0.9986501019683699])
    np.testing.assert_allclose(mlp.gelu(z), expect, rtol=1e-15, atol=1e-16)
    zz = np.linspace(-4, 4, 41)
    e = 1e-6
    fd = (mlp.gelu(zz + e) - mlp.gelu(zz - e)) / (2 * e)
    np.testing.assert_allclose(mlp.gelu_grad(zz), fd, rtol=0, atol=1e-9)


def test_identity_network_reduces_to_scalar_gelu_iterates():
    """W0 routes input feature k to unit k, hidden weights are the identity,
    W4 reads unit k into output k, biases zero except b4: every output is the
    fourfold gelu iterate of its standardised input plus its bias."""
    parts = [np.zeros(s) for s in mlp.SHAPES]
    for k in range(6):
        parts[0][k, k] = 1.0
    for l in (2, 4, 6):
        parts[l] = np.eye(256)
    for k in range(6):
        parts[8][k, k] = 1.0
    parts[9] = np.arange(7) * 0.1
    flat = mlp.flatten(parts)
    X = np.array([[0.2, -1.0, 0.5, 1.5, 0.3, 0.1], [1.0, 0.0, -0.4, 2.0, 0.0, -0.3]])
    mean, std = np.full(6, 0.1), np.full(6, 2.0)
    out, _ = mlp.forward(flat, X, mean, std)

    def g(x):
        return 0.5 * x * (1 + math.erf(x / math.sqrt(2)))

    for p in range(2):
        for k in range(6):
            v = (X[p, k] - 0.1) / 2.0
            for _ in range(4):
                v = g(v)
            assert abs(out[p, k] - (v + 0.1 * k)) < 1e-15
        assert out[p, 6] == pytest.approx(0.6, abs=1e-15)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    flat = mlp.init_params(3)
    X = np.column_stack([rng.normal(1, 0.2, (6, 4)), rng.uniform(0, 0.5, 6), rng.normal(0, 0.2, 6)])
    Y = np.column_stack([rng.uniform(0, math.pi, (6, 2)), rng.uniform(0, 1, 6), rng.normal(0, 0.3, (6, 4))])
    Y[1, :3] = np.nan  # a label that does not split
    mean, std = np.zeros(6), np.ones(6)

    def L(f):
        o, _ = mlp.forward(f, X, mean, std)
        return mlp.loss_and_grad(o, Y)[0]

    out, cache = mlp.forward(flat, X, mean, std)
    _, dout = mlp.loss_and_grad(out, Y)
    g = mlp.backward(flat, cache, dout)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS - 1799, 60, replace=False),
                          np.arange(mlp.N_PARAMS - 1799, mlp.N_PARAMS, 97)])
    e = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += e
        fm[i] -= e
        fd = (L(fp) - L(fm)) / (2 * e)
        assert abs(fd - g[i]) < 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_loss_period_and_masks():
    o = np.array([[0.3, 2.0, 0.0, 0.1, 0.2, -0.1, 0.05]])
    y = o.copy()
    y[0, 2] = 0.5  # sigmoid(0) = 0.5
    assert mlp.loss_and_grad(o, y)[0] == pytest.approx(0.0, abs=1e-15)
    y2 = y.copy()
    y2[0, 0] += math.pi  # angles have period pi
    assert mlp.loss_and_grad(o, y2)[0] == pytest.approx(0.0, abs=1e-14)
    y3 = y.copy()
    y3[0, 0] += math.pi / 2  # orthogonal -> 1 - cos(pi) = 2
    assert mlp.loss_and_grad(o, y3)[0] == pytest.approx(2.0, abs=1e-14)
    y4 = y.copy()
    y4[0, :3] = np.nan  # not laminated: only the jump counts
    o4 = o.copy()
    o4[0, :3] = [1.0, 2.0, 3.0]
    L4, g4 = mlp.loss_and_grad(o4, y4)
    assert L4 == pytest.approx(0.0, abs=1e-15) and np.all(g4[0, :3] == 0)


def test_labels_and_decode_reproduce_the_tree_laminates(orc):
    """Labels from oracle trees: the jump F+ - F- is parallel to the chosen
    R = a (x) b (rank one); decoding a label as if it were the network output
    returns the labelled direction's cell and the tree's own F+ and F-."""
    from paper_2211_14318_gb300 import inputs

    mat = orc.Material(1.0, 5.0, 0.99, 0.5)
    F, Fp = inputs.material_points(12, seed=5)
    beta = orc.history_update(mat, Fp)
    dirs = orc.angle_directions(16, 16)
    sc = orc.Scan(dirs, 201, 0.5, 2)
    _, _, tree, _ = orc.convexify(mat, sc, F, beta)
    X, Y = mlp.labels_from_tree(tree, F, beta, (16, 16), (orc.SCANNED, orc.LAMINATED))
    assert X.shape[0] == int(np.sum(tree["flags"] & orc.SCANNED > 0))
    rows, nodes = [], []
    for p in range(12):
        for i in range(tree.shape[1]):
            if tree[p, i]["flags"] & orc.SCANNED:
                rows.append(p)
                nodes.append(i)
    lam = ~np.isnan(Y[:, 0])
    assert lam.sum() > 5
    for r in np.nonzero(lam)[0]:
        p, i = rows[r], nodes[r]
        d = dirs[tree[p, i]["dir"]]
        R = np.outer(d[:2], d[2:]).reshape(4)
        jump = Y[r, 3:]
        np.testing.assert_allclose(jump, (jump @ R) * R, atol=1e-12)
        out = Y[r:r + 1].copy()
        out[0, 2] = math.log(Y[r, 2] / (1 - Y[r, 2]))
        ia, ib, xi, Fplus, Fminus, dist = mlp.decode(out, tree[p, i]["F"], 16, 16)
        assert ia[0] * 16 + ib[0] == tree[p, i]["dir"]
        np.testing.assert_allclose(Fplus[0], tree[p, 2 * i + 2]["F"], atol=1e-12)
        np.testing.assert_allclose(Fminus[0], tree[p, 2 * i + 1]["F"], atol=1e-12)
        np.testing.assert_allclose(X[r, :4], tree[p, i]["F"], rtol=0, atol=0)
        assert X[r, 5] == pytest.approx(math.log(np.linalg.det(tree[p, i]["F"].reshape(2, 2))), abs=1e-14)
