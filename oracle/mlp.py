"""FP64 CPU oracle of the surrogate proposal network (test infrastructure only).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and bench.py's CPU
baseline may use this module.  It shares no code with the CUDA path.

The network (not in the paper; an addition that proposes where the line scan
of Sec. 4.1 should look):

    inputs  x = (F11, F12, F21, F22, beta_k, ln det F), standardised per feature
    hidden  4 layers of width 256, h = gelu(W h + b), gelu(z) = z Phi(z)
    outputs o (7): o0, o1 -> direction angles theta_a, theta_b (period pi),
                   o2 -> volume fraction xi = sigmoid(o2),
                   o3..o6 -> the jump F+ - F- (row-major 2 x 2).

Loss per sample (angle terms only for laminated labels, whose angles are
not NaN; xi term likewise):
    L = sum_{i=0,1} (1 - cos 2 (o_i - theta_i)) + (sigmoid(o2) - xi)^2
        + sum_{j<4} (o_{3+j} - jump_j)^2,
averaged over the batch.

Parameters are one flat FP32-compatible vector in this order:
    W0 (256 x 6), b0 (256), W1 (256 x 256), b1, W2, b2, W3, b3,
    W4 (7 x 256), b4 (7)
(weights row-major as (out, in)).  ``bf16=True`` rounds the GEMM operands
(inputs, weights, hidden activations, back-propagated dz) to bfloat16 at the
places where a BF16 tensor-core implementation must round them, keeping FP64
everywhere else.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

WIDTH = 256
N_IN, N_OUT, N_HIDDEN = 6, 7, 4
SHAPES = [(WIDTH, N_IN), (WIDTH,), (WIDTH, WIDTH), (WIDTH,), (WIDTH, WIDTH), (WIDTH,),
          (WIDTH, WIDTH), (WIDTH,), (N_OUT, WIDTH), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)  # 200,967


def unflatten(flat):
    """Flat vector -> [W0, b0, ..., W4, b4] (views)."""
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == N_PARAMS
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(flat[o:o + k].reshape(s))
        o += k
    return out


def flatten(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])


def init_params(seed: int = 0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        fan_in = s[1] if len(s) == 2 else (N_IN if len(parts) == 1 else WIDTH)
        b = 1.0 / math.sqrt(fan_in)
        parts.append(rng.uniform(-b, b, size=s))
    return flatten(parts)


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), through FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def features(F, beta):
    """(F11, F12, F21, F22, beta_k, ln det F) per point."""
    F = np.asarray(F, dtype=np.float64).reshape(-1, 4)
    J = F[:, 0] * F[:, 3] - F[:, 1] * F[:, 2]
    return np.column_stack([F, np.asarray(beta, dtype=np.float64).reshape(-1), np.log(J)])


def forward(flat, X, mean, std, bf=False):
    """Raw outputs (n, 7) and the cache for backward."""
    W = unflatten(flat)
    r = bf16 if bf else (lambda a: a)
    h = r((np.asarray(X, dtype=np.float64) - mean) / std)
    cache = {"h": [h], "z": []}
    for l in range(N_HIDDEN):
        z = h @ r(W[2 * l]).T + W[2 * l + 1]
        h = r(gelu(z))
        cache["z"].append(z)
        cache["h"].append(h)
    out = h @ r(W[8]).T + W[9]
    return out, cache


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def loss_and_grad(out, Y):
    """Mean loss over the batch and dL/d(out)."""
    out = np.asarray(out, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = out.shape[0]
    g = np.zeros_like(out)
    L = np.zeros(n)
    lam = ~np.isnan(Y[:, 0])
    for i in (0, 1):
        d = out[lam, i] - Y[lam, i]
        L[lam] += 1.0 - np.cos(2.0 * d)
        g[lam, i] = 2.0 * np.sin(2.0 * d)
    hx = ~np.isnan(Y[:, 2])
    s = _sigmoid(out[hx, 2])
    L[hx] += (s - Y[hx, 2]) ** 2
    g[hx, 2] = 2.0 * (s - Y[hx, 2]) * s * (1.0 - s)
    d = out[:, 3:7] - Y[:, 3:7]
    L += np.sum(d * d, axis=1)
    g[:, 3:7] = 2.0 * d
    return float(np.mean(L)), g / n


def backward(flat, cache, dout, bf=False):
    """Flat gradient of the loss whose d(out) is ``dout``."""
    W = unflatten(flat)
    r = bf16 if bf else (lambda a: a)
    grads = [None] * len(SHAPES)
    dz = r(dout)
    grads[8] = dz.T @ cache["h"][N_HIDDEN]
    grads[9] = np.sum(dout, axis=0)
    Wn = r(W[8])
    for l in range(N_HIDDEN - 1, -1, -1):
        da = dz @ Wn
        dz_full = da * gelu_grad(cache["z"][l])
        grads[2 * l + 1] = np.sum(dz_full, axis=0)
        dz = r(dz_full)
        grads[2 * l] = dz.T @ cache["h"][l]
        Wn = r(W[2 * l])
    return flatten(grads)


def labels_from_tree(tree, F, beta, dirs_shape, NODE_flags):
    """Training samples from every scanned node of per-point lamination trees.

    tree: (n, NT) structured nodes with fields F, dir, xi, flags; children of
    node i at 2i+1 (F-) and 2i+2 (F+).  dirs_shape = (Na, Nb) of the angle
    grid.  Returns X (m, 6) and Y (m, 7): angles theta_a = pi i / Na,
    theta_b = pi j / Nb of direction index i Nb + j, xi, jump F+ - F-; for a
    node that does not split, angles and xi are NaN and the jump is 0."""
    Na, Nb = dirs_shape
    SCANNED, LAMINATED = NODE_flags
    X, Y = [], []
    n, NT = tree.shape
    for p in range(n):
        for i in range(NT):
            nd = tree[p, i]
            if not nd["flags"] & SCANNED:
                continue
            Fi = np.asarray(nd["F"], dtype=np.float64)
            X.append(features(Fi, beta[p])[0])
            if nd["flags"] & LAMINATED:
                d = int(nd["dir"])
                jump = tree[p, 2 * i + 2]["F"] - tree[p, 2 * i + 1]["F"]
                Y.append([math.pi * (d // Nb) / Na, math.pi * (d % Nb) / Nb, nd["xi"], *jump])
            else:
                Y.append([np.nan, np.nan, np.nan, 0.0, 0.0, 0.0, 0.0])
    return np.array(X).reshape(-1, 6), np.array(Y).reshape(-1, 7)


def decode(out, F, Na, Nb):
    """Window centres and the proposed laminate from raw outputs.

    Angles are wrapped to [0, pi) and rounded to the nearest grid cell
    (mod Na, Nb); R = a (x) b of the unrounded angles; amp = jump : R;
    F+ = F + (1 - xi) amp R, F- = F - xi amp R.  Returns (ia, ib, xi, Fp, Fm,
    dist) with dist the distance of each scaled angle to the nearest rounding
    boundary (in cells) -- the margin of the integer decision."""
    out = np.asarray(out, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64).reshape(-1, 4)
    ta = np.mod(out[:, 0], math.pi)
    tb = np.mod(out[:, 1], math.pi)
    ua, ub = ta * Na / math.pi, tb * Nb / math.pi
    ia = np.mod(np.floor(ua + 0.5), Na).astype(int)
    ib = np.mod(np.floor(ub + 0.5), Nb).astype(int)
    dist = np.minimum(np.abs(ua + 0.5 - np.round(ua + 0.5)), np.abs(ub + 0.5 - np.round(ub + 0.5)))
    a = np.column_stack([np.cos(ta), np.sin(ta)])
    b = np.column_stack([np.cos(tb), np.sin(tb)])
    R = np.einsum("ni,nj->nij", a, b).reshape(-1, 4)
    xi = _sigmoid(out[:, 2])
    amp = np.sum(out[:, 3:7] * R, axis=1)
    Fp = F + ((1.0 - xi) * amp)[:, None] * R
    Fm = F - (xi * amp)[:, None] * R
    return ia, ib, xi, Fp, Fm, dist
