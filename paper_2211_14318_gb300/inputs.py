"""Seeded synthetic inputs for the per-point convexification path.

This module holds no arithmetic of the method: it only draws deformation
gradients F (row-major F11, F12, F21, F22) and the deformation of the previous
load step, from which each side computes its own history variable with its
own implementation of Eq. (2.5).  It imports nothing from the CUDA binding or
from the oracle, and both sides may use it.

Workloads (shapes and distributions follow the paper's 2-D material-point and
boundary-value studies, Secs. 6.1, 6.6; parameters are fixed here):

* ``material_points``: F = Q(phi) diag(lam, lam^-0.3) Q(phi)^T + N(0, 0.02^2)
  per entry, phi ~ U[0, pi), lam ~ U[lo, hi], redrawn while det F <= 0; the
  previous step is the same rotation with stretch max(1, lam - 0.1), no noise.
* ``mesh_points``: a Q1 mesh of nx x nx elements on [0, 1]^2 with 2 x 2 Gauss
  points; the displacement is an affine stretch (stretch - 1) X1 plus a seeded
  smooth field of 8 Fourier modes (amplitude 0.05) plus a 45 degree shear band
  of width 4 elements; F = I + grad u of the Q1 interpolant at the Gauss
  points.  The previous step uses the same field at 0.9 times the displacement.
* ``batch_problems``: many meshes of log-uniform point counts with their own
  stretch, angle grid, line length and depth.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np


def material_points(n: int, seed: int = 0, lam_lo: float = 1.0, lam_hi: float = 1.6,
                    noise: float = 0.02) -> Tuple[np.ndarray, np.ndarray]:
    """(F, F_prev), each (n, 4) float64."""
    rng = np.random.default_rng(seed)
    F = np.zeros((n, 4))
    Fp = np.zeros((n, 4))
    todo = np.arange(n)
    while todo.size:
        m = todo.size
        phi = rng.uniform(0.0, math.pi, size=m)
        lam = rng.uniform(lam_lo, lam_hi, size=m)
        eps = rng.normal(0.0, noise, size=(m, 4))
        c, s = np.cos(phi), np.sin(phi)
        l2 = lam ** -0.3
        # Q diag(l1, l2) Q^T with Q = [[c, -s], [s, c]]
        A = np.stack([c * c * lam + s * s * l2, c * s * (lam - l2),
                      c * s * (lam - l2), s * s * lam + c * c * l2], axis=1)
        G = A + eps
        ok = G[:, 0] * G[:, 3] - G[:, 1] * G[:, 2] > 0.0
        lp = np.maximum(1.0, lam - 0.1)
        lp2 = lp ** -0.3
        Ap = np.stack([c * c * lp + s * s * lp2, c * s * (lp - lp2),
                       c * s * (lp - lp2), s * s * lp + c * c * lp2], axis=1)
        F[todo[ok]] = G[ok]
        Fp[todo[ok]] = Ap[ok]
        todo = todo[~ok]
    return F, Fp


def _displacement(X: np.ndarray, Y: np.ndarray, stretch: float, seed: int, nx: int,
                  n_modes: int = 8, amp: float = 0.05, band_width_el: float = 4.0,
                  band_amp: float = 0.1) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    ux = (stretch - 1.0) * X
    uy = np.zeros_like(Y)
    for _ in range(n_modes):
        p = rng.integers(1, 5, size=2)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        c = np.array([math.cos(ang), math.sin(ang)])
        ph = rng.uniform(0.0, 2.0 * math.pi)
        arg = 2.0 * math.pi * (p[0] * X + p[1] * Y) + ph
        sn = np.sin(arg) / (2.0 * math.pi * np.hypot(p[0], p[1]))
        ux = ux + amp * c[0] * sn
        uy = uy + amp * c[1] * sn
    # shear band: tangential slip that ramps across a band normal to n = (1,-1)/sqrt2
    hx = 1.0 / nx
    nrm = np.array([1.0, -1.0]) / math.sqrt(2.0)
    tng = np.array([1.0, 1.0]) / math.sqrt(2.0)
    z = X * nrm[0] + Y * nrm[1]
    half = 0.5 * band_width_el * hx
    ramp = np.clip((z + half) / (2.0 * half), 0.0, 1.0) * (2.0 * half)
    ux = ux + band_amp * tng[0] * ramp
    uy = uy + band_amp * tng[1] * ramp
    return ux, uy


def mesh_points(nx: int, stretch: float = 1.3, seed: int = 0, load: float = 1.0,
                prev_load: float = 0.9) -> Tuple[np.ndarray, np.ndarray]:
    """(F, F_prev) at the 4 Gauss points of each Q1 element, (4 nx^2, 4) float64.

    Point order: element (i, j) row-major (j fastest), Gauss points in the
    order (-,-), (+,-), (-,+), (+,+)."""
    xs = np.linspace(0.0, 1.0, nx + 1)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    ux, uy = _displacement(X, Y, stretch, seed, nx)
    hx = 1.0 / nx
    g = 1.0 / math.sqrt(3.0)
    out = []
    for lf in (load, prev_load):
        Fs = np.zeros((nx, nx, 4, 4))
        for q, (xi, eta) in enumerate(((-g, -g), (g, -g), (-g, g), (g, g))):
            # Q1 shape-function gradients on the reference square, mapped by 2/h
            dN = [((-(1 - eta)) / 4, (-(1 - xi)) / 4), (((1 - eta)) / 4, (-(1 + xi)) / 4),
                  (((1 + eta)) / 4, ((1 + xi)) / 4), ((-(1 + eta)) / 4, ((1 - xi)) / 4)]
            corners = [(0, 0), (1, 0), (1, 1), (0, 1)]
            G = np.zeros((nx, nx, 2, 2))
            for (dx, dy), (ci, cj) in zip(dN, corners):
                uxa = ux[ci:ci + nx, cj:cj + nx] * lf
                uya = uy[ci:ci + nx, cj:cj + nx] * lf
                G[..., 0, 0] += uxa * dx * 2.0 / hx
                G[..., 0, 1] += uxa * dy * 2.0 / hx
                G[..., 1, 0] += uya * dx * 2.0 / hx
                G[..., 1, 1] += uya * dy * 2.0 / hx
            Fs[:, :, q, 0] = 1.0 + G[..., 0, 0]
            Fs[:, :, q, 1] = G[..., 0, 1]
            Fs[:, :, q, 2] = G[..., 1, 0]
            Fs[:, :, q, 3] = 1.0 + G[..., 1, 1]
        out.append(Fs.reshape(-1, 4).copy())
    return out[0], out[1]


def load_path(nx: int, n_steps: int = 20, stretch_end: float = 1.8, seed: int = 0) -> List[np.ndarray]:
    """F at every load step k = 1..n_steps of a monotone path from stretch 1.0
    to ``stretch_end``: the full displacement field scaled by k / n_steps."""
    F_full, _ = mesh_points(nx, stretch=stretch_end, seed=seed, load=1.0, prev_load=0.0)
    I = np.array([1.0, 0.0, 0.0, 1.0])
    G = F_full - I
    return [I + G * (k / n_steps) for k in range(1, n_steps + 1)]


@dataclass
class Problem:
    """One mesh of a batch: its points and its own parameters."""
    F: np.ndarray
    F_prev: np.ndarray
    stretch: float
    n_angle: int
    L: int
    depth: int


def batch_problems(n_problems: int = 256, seed: int = 0, n_lo: int = 1000, n_hi: int = 100000,
                   angles=(32, 64), lines=(513, 1025), depths=(2, 3)) -> List[Problem]:
    """Problems with log-uniform point counts (rounded to whole Q1 meshes of
    4 Gauss points per element) and per-problem stretch, angle grid, line and depth."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(n_problems):
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        nx = max(1, int(round(math.sqrt(n_target / 4.0))))
        stretch = float(rng.uniform(1.1, 1.8))
        na = int(angles[rng.integers(0, len(angles))])
        L = int(lines[rng.integers(0, len(lines))])
        K = int(depths[rng.integers(0, len(depths))])
        F, Fp = mesh_points(nx, stretch=stretch, seed=seed * 100003 + p)
        out.append(Problem(F, Fp, stretch, na, L, K))
    return out


def surrogate_inputs(n: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Training / held-out points for the learned proposal: material points
    with lam ~ U[1, 2]."""
    return material_points(n, seed=seed, lam_lo=1.0, lam_hi=2.0)


def cuboid_points(lo, hi, n: int, seed: int = 0) -> np.ndarray:
    """(n, 4) deformation gradients drawn uniformly from the box lo <= F <= hi
    (per entry F11, F12, F21, F22): query points of the global-grid form."""
    rng = np.random.default_rng(seed)
    return rng.uniform(np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64),
                       size=(n, 4))
