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
