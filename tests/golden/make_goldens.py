"""Writes the oracle-only expected values of the full-size parity tests.

Every value stored here comes from the FP64 CPU oracle (``oracle/``) run on
seeded inputs from ``paper_2211_14318_gb300.inputs``; nothing is read from the
CUDA path.  Each file holds a fixed subsample of 4,096 points of one workload:
the inputs themselves (F, beta_k, so that the GPU side convexifies exactly the
same numbers on any host), and the oracle's W^R, P, status and lamination
tree (per node: flags, decision margin, direction, bridge indices, F).

Workloads (the sizes the benchmark runs, subsampled evenly):

* ``mesh128``: 128 x 128 Q1 mesh x 4 Gauss points (65,536 points), stretch
  1.3, seed 0, history from the previous load step (0.9 x the displacement);
  64 x 64 angles, L = 1025, t in [-0.5, 0.5], depth 3.
* ``material1m_l201``: 1,048,576 material points (F = Q diag(lam, lam^-0.3)
  Q^T + N(0, 0.02^2), lam ~ U[1, 2], seed 201, history from one prior step);
  16 x 16 angles, L = 201, t in [-0.5, 0.5], depth 2.
* ``loadpath512_sKK``: 512 x 512 Q1 mesh x 4 Gauss points (1,048,576
  points), load path stretch 1.0 -> 1.8 in 20 steps (seed 7), load step KK
  in {1, 10, 20} with the history of the earlier steps (Eq. 2.5);
  128 x 128 angles, L = 2049, t in [-0.5, 0.5], depth 3.

* ``grid61``: the global-grid study of Sec. 6.1 (Table tab:2Dconvexification,
  NH row: mu = 1, lambda = 0.5, D_inf = 0.9, D_0 = 0.3, beta_k = 0.06; grid
  delta 0.15, diagonal [0.1, 3.4], off-diagonal [-2.55, 2.55]: 648,025
  points; R^1_1; tol 1e-4, kmax 20; ln|det F|): the decrease of every step,
  W^K at 4,096 evenly spaced grid points, and Algorithms 2 and 3 over the
  forest at 1,024 points drawn uniformly from the grid's box (seed 61).

* ``grid3d``: the nine-dimensional study of Sec. 6.8 (Table
  tab:3Dconvexification, NH: beta_k fitted to the printed W(1), diagonal
  [1.0, 3.4], off-diagonal [-0.15, 0.15], delta 0.15: 3,581,577 points;
  R^1_1 for d = 3, 169 directions; tol 1e-4, kmax 20): the decreases, W^K at
  4,096 evenly spaced grid points and on the uni-, bi- and triaxial paths.
* ``stvk61``: the STVK study of Sec. 6.1 (beta_k 0.07, delta 0.1, diagonal
  [0.1, 2.0], off-diagonal [-2.0, 2.0]: 672,400 points; R^1_1; Eq. (2.2)
  kept where det F <= 0): the decreases and W^K at 4,096 grid points.

Usage: python tests/golden/make_goldens.py [--only NAME ...] [--threads N]
The load-path files take hours of CPU time (the oracle is plain FP64 C).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2211_14318_gb300 import inputs  # noqa: E402

N_SUB = 4096
MAT = dict(mu=1.0, lam=5.0, Dinf=0.99, D0=0.5)
LOAD_STEPS = (1, 10, 20)


def subsample(n: int) -> np.ndarray:
    return np.linspace(0, n - 1, N_SUB).astype(np.int64)


def workloads():
    """name -> (description, angles, L, t_half, depth, thunk returning (idx, F, beta))."""
    mat = oracle.Material(**MAT)
    out = {}

    def mesh128():
        F, Fp = inputs.mesh_points(128, stretch=1.3, seed=0)
        idx = subsample(F.shape[0])
        return idx, F[idx], oracle.history_update(mat, Fp[idx])

    out["mesh128"] = ("128x128 Q1 mesh x 4 Gauss points, stretch 1.3, seed 0", 64, 1025, 0.5, 3,
                      mesh128)

    def material():
        F, Fp = inputs.surrogate_inputs(1 << 20, seed=201)
        idx = subsample(F.shape[0])
        return idx, F[idx], oracle.history_update(mat, Fp[idx])

    out["material1m_l201"] = ("1,048,576 material points, lam ~ U[1, 2], seed 201", 16, 201, 0.5,
                              2, material)

    for k in LOAD_STEPS:
        def lp(k=k):
            path = inputs.load_path(512, n_steps=20, stretch_end=1.8, seed=7)
            idx = subsample(path[0].shape[0])
            beta = np.zeros(N_SUB)
            for j in range(k - 1):  # history of the earlier load steps
                beta = oracle.history_update(mat, path[j][idx], beta)
            return idx, path[k - 1][idx], beta

        out[f"loadpath512_s{k:02d}"] = (
            f"512x512 Q1 mesh x 4 Gauss points, load path 1.0 -> 1.8 in 20 steps (seed 7), step {k}",
            128, 2049, 0.5, 3, lp)
    return out


def write(name, desc, na, L, t_half, depth, thunk, threads):
    mat = oracle.Material(**MAT)
    idx, F, beta = thunk()
    sc = oracle.Scan(oracle.angle_directions(na, na), L, t_half, depth)
    t0 = time.perf_counter()
    WR, P, tree, st = oracle.convexify(mat, sc, F, beta, nthreads=threads)
    dt = time.perf_counter() - t0
    meta = dict(workload=desc, angles=[na, na], line_points=L, t_half=t_half, depth=depth,
                material=MAT, points=N_SUB, oracle_seconds=dt, threads=threads)
    path = os.path.join(HERE, f"{name}.npz")
    np.savez_compressed(
        path, meta=np.array(json.dumps(meta)), idx=idx, F=F, beta=beta, W_R=WR, P=P, status=st,
        flags=tree["flags"].astype(np.int8), margin=tree["margin"], dir=tree["dir"].astype(np.int16),
        m_minus=tree["m_minus"].astype(np.int16), m_plus=tree["m_plus"].astype(np.int16),
        node_F=tree["F"])
    print(f"{name}: {N_SUB} points in {dt:.0f} s -> {path}", flush=True)


GRID61 = dict(mat=dict(mu=1.0, lam=0.5, Dinf=0.9, D0=0.3), beta=0.06, diag=(0.1, 3.4),
              off=(-2.55, 2.55), delta=(0.15, 0.15), kmax=20, tol=1e-4)


def write_grid61(threads):
    c = GRID61
    mat = oracle.Material(**c["mat"])
    g = oracle.Grid.from_bounds(c["diag"], c["off"], c["delta"])
    off = oracle.r11_directions()
    t0 = time.perf_counter()
    W, forest, decs = oracle.grid_convexify(mat, g, c["beta"], off, kmax=c["kmax"], tol=c["tol"],
                                            abs_det=True, nthreads=threads)
    dt = time.perf_counter() - t0
    idx = subsample(g.count)
    P = g.points()
    Fq = inputs.cuboid_points(P.min(0), P.max(0), 1024, seed=61)
    wi, wt, Pq, nl = oracle.grid_query(mat, g, c["beta"], off, W[-1], forest, Fq, abs_det=True,
                                       nthreads=threads)
    meta = dict(workload="Sec. 6.1 NH grid study, 648,025 points, R^1_1, tol 1e-4, kmax 20, "
                "ln|det F|", **{k: v for k, v in c.items() if k != "mat"}, material=c["mat"],
                oracle_seconds=dt, threads=threads, iterations=len(decs))
    path = os.path.join(HERE, "grid61.npz")
    np.savez_compressed(path, meta=np.array(json.dumps(meta)), decs=np.array(decs), idx=idx,
                        W_K=W[-1][idx], F_query=Fq, W_interp=wi, W_tree=wt, P=Pq, leaves=nl)
    print(f"grid61: {len(decs)} iterations in {dt:.1f} s -> {path}", flush=True)


def _fit_beta_identity(mat, W_identity):
    """beta_k from W(1) = -(1 - D(beta_k)) beta_k by bisection (monotone)."""
    lo, hi = 1e-9, 1.0
    f = lambda b: oracle.energy(mat, [1, 0, 0, 1], b) - W_identity  # noqa: E731
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (f(lo) > 0) == (f(mid) > 0):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def write_grid3d(threads):
    mat = oracle.Material(**GRID61["mat"])
    rows = [[float(v) for v in ln.split()] for ln in open(os.path.join(HERE, "nh3d_paths.txt"))
            if ln.strip() and not ln.startswith("#")]
    beta = _fit_beta_identity(mat, rows[0][1])
    g = oracle.Grid.from_bounds((1.0, 3.4), (-0.15, 0.15), (0.15, 0.15), dim=3)
    t0 = time.perf_counter()
    W, _, decs = oracle.grid_convexify(mat, g, beta, oracle.r11_directions(3), kmax=20,
                                       tol=1e-4, nthreads=threads, keep_all=False)
    dt = time.perf_counter() - t0
    st = np.ones(9, dtype=np.int64)
    for c in range(7, -1, -1):
        st[c] = st[c + 1] * g.n[c + 1]
    paths = np.array([[np.dot([k, 1, 1, 1, 1, 1, 1, 1, 0], st) for k in range(17)],
                      [np.dot([k, 1, 1, 1, k, 1, 1, 1, 0], st) for k in range(17)],
                      [np.dot([k, 1, 1, 1, k, 1, 1, 1, k], st) for k in range(17)]])
    idx = subsample(g.count)
    meta = dict(workload="Sec. 6.8 nine-dimensional NH study, 3,581,577 points, R^1_1 (d = 3), "
                "tol 1e-4, kmax 20", beta=beta, material=GRID61["mat"], oracle_seconds=dt,
                threads=threads, iterations=len(decs))
    path = os.path.join(HERE, "grid3d.npz")
    np.savez_compressed(path, meta=np.array(json.dumps(meta)), decs=np.array(decs), idx=idx,
                        W_K=W[-1][idx], paths=paths, W_paths=W[-1][paths], W0_paths=W[0][paths])
    print(f"grid3d: {len(decs)} iterations in {dt:.1f} s -> {path}", flush=True)


def write_stvk61(threads):
    m = GRID61["mat"]
    mat = oracle.Material(m["mu"], m["lam"], m["Dinf"], m["D0"], energy=2)
    g = oracle.Grid.from_bounds((0.1, 2.0), (-2.0, 2.0), (0.1, 0.1))
    t0 = time.perf_counter()
    W, _, decs = oracle.grid_convexify(mat, g, 0.07, oracle.r11_directions(), kmax=20, tol=1e-4,
                                       rule=1, nthreads=threads, keep_all=False)
    dt = time.perf_counter() - t0
    idx = subsample(g.count)
    meta = dict(workload="Sec. 6.1 STVK grid study, 672,400 points, R^1_1, tol 1e-4, kmax 20, "
                "Eq. (2.2) kept where det F <= 0", beta=0.07, material=m, oracle_seconds=dt,
                threads=threads, iterations=len(decs))
    path = os.path.join(HERE, "stvk61.npz")
    np.savez_compressed(path, meta=np.array(json.dumps(meta)), decs=np.array(decs), idx=idx,
                        W_K=W[-1][idx])
    print(f"stvk61: {len(decs)} iterations in {dt:.1f} s -> {path}", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    oracle.build()
    for name, (desc, na, L, t_half, depth, thunk) in workloads().items():
        if a.only and name not in a.only:
            continue
        write(name, desc, na, L, t_half, depth, thunk, a.threads or oracle.cores())
    if not a.only or "grid61" in a.only:
        write_grid61(a.threads or oracle.cores())
    if not a.only or "stvk61" in a.only:
        write_stvk61(a.threads or oracle.cores())
    if not a.only or "grid3d" in a.only:
        write_grid3d(a.threads or oracle.cores())


if __name__ == "__main__":
    main()
