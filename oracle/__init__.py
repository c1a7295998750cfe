"""FP64 CPU oracle for per-point rank-one convexification (arXiv 2211.14318).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The CUDA product path never imports
it, and it shares no code with that path.

The arithmetic lives in ``oracle.c`` (plain C, FP64, one function per step of
the paper); this module compiles it with gcc and exposes it through ctypes.
Functions marked "parity unpinned" in their docstring have no external pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")

NODE_DTYPE = np.dtype(
    [
        ("F", "<f8", (4,)),
        ("w", "<f8"),
        ("h", "<f8"),
        ("xi", "<f8"),
        ("weight", "<f8"),
        ("margin", "<f8"),
        ("dir", "<i4"),
        ("m_minus", "<i4"),
        ("m_plus", "<i4"),
        ("flags", "<i4"),
        ("wexp", "<i4"),
        ("pad", "<i4"),
    ]
)
EXISTS, SCANNED, LAMINATED, LEAF, NEWTON = 1, 2, 4, 8, 16


class _Material(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("Dinf", ctypes.c_double),
        ("D0", ctypes.c_double),
        ("energy", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class _Scan(ctypes.Structure):
    _fields_ = [
        ("n_dir", ctypes.c_int32),
        ("L", ctypes.c_int32),
        ("dir", ctypes.POINTER(ctypes.c_double)),
        ("t_half", ctypes.c_double),
        ("depth", ctypes.c_int32),
        ("round32", ctypes.c_int32),
        ("newton", ctypes.c_int32),
        ("adaptive", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_liboracle.so`` (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
        "-o", tmp, _SRC, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        vp = ctypes.c_void_p
        L.orc_psi0_nh.restype = d
        L.orc_psi0_nh.argtypes = [d, d, d, d]
        L.orc_damage.restype = d
        L.orc_damage.argtypes = [d, d, d]
        L.orc_W_of_psi0.restype = d
        L.orc_W_of_psi0.argtypes = [d, d, d, d]
        L.orc_energy.restype = d
        L.orc_energy.argtypes = [vp, vp, d]
        L.orc_stress.restype = None
        L.orc_stress.argtypes = [vp, vp, d, vp]
        L.orc_psi0_F.restype = d
        L.orc_tangent.argtypes = [vp, vp, d, vp]
        L.orc_tangent.restype = None
        L.orc_newton_tangent.argtypes = [vp, vp, d, vp, d, d, d, d, vp, vp, vp]
        L.orc_newton_tangent.restype = i32
        L.orc_psi0_F.argtypes = [vp, vp]
        L.orc_history_update.restype = None
        L.orc_history_update.argtypes = [vp, i64, vp, vp, vp]
        L.orc_angle_directions.restype = None
        L.orc_angle_directions.argtypes = [i32, i32, vp]
        L.orc_sample_line.restype = None
        L.orc_sample_line.argtypes = [vp, vp, d, vp, i32, d, i32, vp, vp]
        L.orc_lower_hull.restype = i32
        L.orc_lower_hull.argtypes = [i32, vp, vp, vp]
        L.orc_line_bridge.restype = d
        L.orc_line_bridge.argtypes = [i32, vp, vp, vp, vp, vp]
        L.orc_scan_node.restype = i32
        L.orc_scan_node.argtypes = [vp, vp, vp, d, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_convexify.restype = None
        L.orc_convexify.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, vp, i32]
        L.orc_tree_tangent.restype = None
        L.orc_tree_tangent.argtypes = [vp, i32, i64, vp, vp, vp]
        L.orc_tree_size.restype = i32
        L.orc_tree_size.argtypes = [i32]
        L.orc_node_size.restype = i32
        L.orc_node_size.argtypes = []
        L.orc_grid_count.restype = i64
        L.orc_grid_count.argtypes = [vp]
        L.orc_grid_point.restype = None
        L.orc_grid_point.argtypes = [vp, i64, vp]
        L.orc_r11_directions.restype = None
        L.orc_r11_directions.argtypes = [vp]
        L.orc_r11_directions3.restype = None
        L.orc_r11_directions3.argtypes = [vp]
        L.orc_psi0_stvk.restype = d
        L.orc_psi0_stvk.argtypes = [d, d, d, d]
        L.orc_invariants.restype = None
        L.orc_invariants.argtypes = [i32, vp, vp, vp, vp]
        L.orc_energy_dim.restype = d
        L.orc_energy_dim.argtypes = [vp, i32, vp, d, i32]
        L.orc_stress_dim.restype = None
        L.orc_stress_dim.argtypes = [vp, i32, vp, d, i32, vp]
        L.orc_grid_energy.restype = None
        L.orc_grid_energy.argtypes = [vp, vp, d, i32, vp, i32]
        L.orc_grid_query.restype = None
        L.orc_grid_query.argtypes = [vp, vp, d, i32, vp, i32, vp, vp, i64, vp, vp, vp, vp, vp, vp,
                                     i32]
        L.orc_tangent_dim.restype = None
        L.orc_tangent_dim.argtypes = [vp, i32, vp, d, i32, vp]
        L.orc_grid_step.restype = d
        L.orc_grid_step.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, i32]
        assert L.orc_node_size() == NODE_DTYPE.itemsize, "node layout mismatch"
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


class Material:
    """Material of Sec. 2: Lame (mu, lam), damage (D_inf, D_0); energy 0 = NH
    with damage (Eqs. 2.3, 2.9), 1 = separable double-well test energy,
    2 = St. Venant-Kirchhoff with damage (Eqs. 2.2, 2.9)."""

    def __init__(self, mu=1.0, lam=5.0, Dinf=0.99, D0=0.5, energy=0):
        self.mu, self.lam, self.Dinf, self.D0, self.energy = mu, lam, Dinf, D0, energy
        self._c = _Material(mu, lam, Dinf, D0, energy, 0)

    @property
    def ref(self):
        return ctypes.byref(self._c)


def psi0_nh(I1: float, J: float, mu: float, lam: float) -> float:
    """Eq. (2.3) in the invariants."""
    return lib().orc_psi0_nh(I1, J, mu, lam)


def psi0_stvk(I1: float, I2: float, mu: float, lam: float) -> float:
    """Eq. (2.2) in the invariants."""
    return lib().orc_psi0_stvk(I1, I2, mu, lam)


def invariants(F) -> tuple:
    """(I1, I2, J) of C = F^T F for F in R^{2x2} (plane strain) or R^{3x3}
    (row-major)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    d = 2 if F.size == 4 else 3
    out = np.zeros(3)
    lib().orc_invariants(d, _p(F), _p(out[0:]), _p(out[1:]), _p(out[2:]))
    return float(out[0]), float(out[1]), float(out[2])


def energy_dim(mat: Material, F, beta_k: float, rule: int = 0) -> float:
    """W(F), Eq. (2.9), for F in R^{2x2} (plane strain) or R^{3x3} under a grid
    rule for det F <= 0 (0 excluded, 1 kept; see grid_energy)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    return lib().orc_energy_dim(mat.ref, 2 if F.size == 4 else 3, _p(F), beta_k, int(rule))


def stress_dim(mat: Material, F, beta_k: float, rule: int = 0) -> np.ndarray:
    """P = dW/dF (row-major, d x d entries) of energy_dim."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    P = np.zeros(F.size)
    lib().orc_stress_dim(mat.ref, 2 if F.size == 4 else 3, _p(F), beta_k, int(rule), _p(P))
    return P


def tangent_dim(mat: Material, F, beta_k: float, rule: int = 0) -> np.ndarray:
    """d^2 W / dF dF (D x D, row-major entries of F) of energy_dim."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    A = np.zeros(F.size * F.size)
    lib().orc_tangent_dim(mat.ref, 2 if F.size == 4 else 3, _p(F), beta_k, int(rule), _p(A))
    return A.reshape(F.size, F.size)


def W_of_psi0(s: float, beta_k: float, Dinf: float, D0: float) -> float:
    """Eq. (2.9) as a function of s = psi0."""
    return lib().orc_W_of_psi0(s, beta_k, Dinf, D0)


def damage(beta: float, Dinf: float, D0: float) -> float:
    """Eq. (2.6)."""
    return lib().orc_damage(beta, Dinf, D0)


def energy(mat: Material, F, beta_k: float) -> float:
    """W(F), Eq. (2.9), plane strain."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    return lib().orc_energy(mat.ref, _p(F), beta_k)


def stress(mat: Material, F, beta_k: float) -> np.ndarray:
    """P = dW/dF, Eq. (2.12)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    P = np.zeros(4)
    lib().orc_stress(mat.ref, _p(F), beta_k, _p(P))
    return P


def tangent(mat: Material, F, beta_k: float) -> np.ndarray:
    """A = d^2 W / dF dF as a 4 x 4 matrix over the row-major entries of F."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    A = np.zeros(16)
    lib().orc_tangent(mat.ref, _p(F), beta_k, _p(A))
    return A.reshape(4, 4)


def newton_tangent(mat: Material, F, beta_k: float, R, t_half: float, tm: float, tp: float,
                   h_grid: float):
    """Common-tangent Newton refinement of a split; (t-, t+, chord value at 0)
    or None when the refinement is not accepted."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(4)
    out = np.zeros(3)
    ok = lib().orc_newton_tangent(mat.ref, _p(F), beta_k, _p(R), t_half, tm, tp, h_grid,
                                  _p(out[0:]), _p(out[1:]), _p(out[2:]))
    return (out[0], out[1], out[2]) if ok else None


def psi0_F(mat: Material, F) -> float:
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    return lib().orc_psi0_F(mat.ref, _p(F))


def history_update(mat: Material, F: np.ndarray, beta_in: Optional[np.ndarray] = None) -> np.ndarray:
    """Eq. (2.5): beta_new = max(beta_in, psi0(F)) per point (beta_in = 0 if None)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 4)
    n = F.shape[0]
    out = np.zeros(n)
    bi = None
    if beta_in is not None:
        bi = np.ascontiguousarray(beta_in, dtype=np.float64).reshape(n)
    lib().orc_history_update(mat.ref, n, _p(F), _p(bi) if bi is not None else None, _p(out))
    return out


def angle_directions(Na: int, Nb: int) -> np.ndarray:
    """(Na*Nb, 4) table of (a1, a2, b1, b2), a_i = (cos pi i/Na, sin pi i/Na)."""
    d = np.zeros((Na * Nb, 4))
    lib().orc_angle_directions(Na, Nb, _p(d))
    return d


class Scan:
    """Direction set, line (L samples on [-t_half, t_half]) and depth K."""

    def __init__(self, dirs: np.ndarray, L: int, t_half: float, depth: int, round32: bool = False,
                 newton: bool = False, adaptive: int = 0):
        self.dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 4)
        self.L, self.t_half, self.depth, self.round32 = int(L), float(t_half), int(depth), bool(round32)
        self.newton = bool(newton)
        self.adaptive = int(adaptive)  # window doublings allowed per node
        self._c = _Scan(
            self.dirs.shape[0], self.L,
            self.dirs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            self.t_half, self.depth, int(self.round32), int(self.newton), self.adaptive,
        )

    @property
    def ref(self):
        return ctypes.byref(self._c)

    @property
    def m0(self) -> int:
        return (self.L - 1) // 2

    @property
    def h(self) -> float:
        return 2.0 * self.t_half / (self.L - 1)


def rank_one(d) -> np.ndarray:
    d = np.asarray(d, dtype=np.float64)
    return np.array([d[0] * d[2], d[0] * d[3], d[1] * d[2], d[1] * d[3]])


def sample_line(mat: Material, F, beta_k: float, R, L: int, t_half: float, round32: bool = False):
    """Samples of W along F + t R (Eq. 4.4 restated per point); returns (w, valid)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(4)
    w = np.zeros(L)
    v = np.zeros(L, dtype=np.uint8)
    lib().orc_sample_line(mat.ref, _p(F), beta_k, _p(R), L, t_half, int(round32), _p(w), _p(v))
    return w, v.astype(bool)


def lower_hull(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Algorithm 1: indices of the strict lower-hull vertices of (x, w)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    vtx = np.zeros(max(len(x), 1), dtype=np.int32)
    k = lib().orc_lower_hull(len(x), _p(x), _p(w), _p(vtx))
    return vtx[:k].copy()


def line_bridge(w: np.ndarray, valid: Optional[np.ndarray] = None):
    """Hull at x = 0 of samples at integer abscissae m - m0.

    Returns (h, m_minus, m_plus, margin)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    L = w.shape[0]
    v = np.ones(L, dtype=np.uint8) if valid is None else np.ascontiguousarray(valid, dtype=np.uint8)
    mm = np.zeros(1, dtype=np.int32)
    mp = np.zeros(1, dtype=np.int32)
    mg = np.zeros(1)
    h = lib().orc_line_bridge(L, _p(w), _p(v), _p(mm), _p(mp), _p(mg))
    return h, int(mm[0]), int(mp[0]), float(mg[0])


def scan_node(mat: Material, sc: Scan, F, beta_k: float, per_direction: bool = False):
    """Min over directions at one node (Eq. 4.3).  Returns a dict."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(4)
    nd = sc.dirs.shape[0]
    hs = np.zeros(nd)
    mm = np.zeros(nd, dtype=np.int32)
    mp = np.zeros(nd, dtype=np.int32)
    mg = np.zeros(nd)
    hb = np.zeros(1)
    a = np.zeros(1, dtype=np.int32)
    b = np.zeros(1, dtype=np.int32)
    margin = np.zeros(1)
    j = lib().orc_scan_node(mat.ref, sc.ref, _p(F), beta_k, _p(hs), _p(mm), _p(mp), _p(mg),
                            _p(hb), _p(a), _p(b), _p(margin))
    out = dict(dir=int(j), h=float(hb[0]), m_minus=int(a[0]), m_plus=int(b[0]),
               margin=float(margin[0]))
    if per_direction:
        out.update(h_dir=hs, m_minus_dir=mm, m_plus_dir=mp, margin_dir=mg)
    return out


def tree_size(depth: int) -> int:
    return (1 << (depth + 1)) - 1


def convexify(mat: Material, sc: Scan, F: np.ndarray, beta_k: np.ndarray, nthreads: int = 0):
    """Per-point W^R, P and lamination tree (Eq. 3.3 top-down, Alg. 2/3).

    Returns (W_R (n,), P (n, 4), tree (n, 2^{K+1}-1) NODE_DTYPE, status (n,))."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 4)
    n = F.shape[0]
    beta_k = np.ascontiguousarray(beta_k, dtype=np.float64).reshape(n)
    WR = np.zeros(n)
    P = np.zeros((n, 4))
    tree = np.zeros((n, tree_size(sc.depth)), dtype=NODE_DTYPE)
    st = np.zeros(n, dtype=np.int32)
    lib().orc_convexify(mat.ref, sc.ref, n, _p(F), _p(beta_k), _p(WR), _p(P), _p(tree), _p(st),
                        int(nthreads))
    return WR, P, tree, st


def tree_tangent(mat: Material, depth: int, tree: np.ndarray, beta_k: np.ndarray) -> np.ndarray:
    """Tangent of W^R, (n, 4, 4) with A[p, i, k] = dP_i / dF_k, by Algorithm 3
    over the given trees (NODE_DTYPE, n x (2^{K+1}-1), xi and weight fields as
    convexify writes them)."""
    tree = np.ascontiguousarray(tree, dtype=NODE_DTYPE)
    n = tree.shape[0]
    beta_k = np.ascontiguousarray(beta_k, dtype=np.float64).reshape(n)
    A = np.zeros((n, 16))
    lib().orc_tree_tangent(mat.ref, int(depth), n, _p(tree), _p(beta_k), _p(A))
    return A.reshape(n, 4, 4)


def cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)


# ---------------------------------------------------------------------------
# Global-grid rank-one convexification: Eq. (4.3) on the cuboid grid of
# Sec. 5.2 with the reduced direction set R^1_1 of Eq. (5.1)
# ---------------------------------------------------------------------------


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 9), ("lo", ctypes.c_double * 9),
                ("delta", ctypes.c_double * 9)]


class Grid:
    """Cuboid grid of Sec. 5.2 for F in R^{d x d}: component c of F (row-major;
    4 components for d = 2, 9 for d = 3) takes lo[c] + i delta[c],
    i = 0 .. n[c] - 1 (flat index with the last component fastest)."""

    def __init__(self, n, lo, delta):
        self.n = tuple(int(x) for x in n)
        self.lo = tuple(float(x) for x in lo)
        self.delta = tuple(float(x) for x in delta)
        D = len(self.n)
        assert D in (4, 9) and len(self.lo) == D and len(self.delta) == D
        self.dim = 2 if D == 4 else 3
        pad = (0,) * (9 - D)
        self._c = _Grid(self.dim, (ctypes.c_int32 * 9)(*(self.n + pad)),
                        (ctypes.c_double * 9)(*(self.lo + (0.0,) * (9 - D))),
                        (ctypes.c_double * 9)(*(self.delta + (0.0,) * (9 - D))))

    @property
    def D(self) -> int:
        return len(self.n)

    @classmethod
    def from_bounds(cls, diag, off, delta, dim: int = 2):
        """Grid with the same bounds (lo, hi) on every diagonal entry and the
        same on every off-diagonal entry, spacing delta (diagonal,
        off-diagonal); hi is a grid value (Tables tab:2Dconvexification,
        tab:3Dconvexification)."""
        (dlo, dhi), (olo, ohi) = diag, off
        dd, do = delta
        nd = int(round((dhi - dlo) / dd)) + 1
        no = int(round((ohi - olo) / do)) + 1
        n, lo, de = [], [], []
        for i in range(dim):
            for j in range(dim):
                n.append(nd if i == j else no)
                lo.append(dlo if i == j else olo)
                de.append(dd if i == j else do)
        return cls(n, lo, de)

    @property
    def ref(self):
        return ctypes.byref(self._c)

    @property
    def count(self) -> int:
        return int(lib().orc_grid_count(self.ref))

    def points(self) -> np.ndarray:
        """(N, D) grid points in flat-index order."""
        axes = [self.lo[c] + np.arange(self.n[c]) * self.delta[c] for c in range(self.D)]
        return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, self.D)


def r11_directions(dim: int = 2) -> np.ndarray:
    """Grid-index offsets of the directions of Eq. (5.1): (16, 4) for d = 2,
    (169, 9) for d = 3."""
    if dim == 2:
        off = np.zeros((16, 4), dtype=np.int32)
        lib().orc_r11_directions(_p(off))
    else:
        off = np.zeros((169, 9), dtype=np.int32)
        lib().orc_r11_directions3(_p(off))
    return off


def _rule(abs_det: bool, rule):
    return int(rule) if rule is not None else (1 if abs_det else 0)


def grid_energy(mat: Material, grid: Grid, beta_k: float, abs_det: bool = False,
                nthreads: int = 0, rule=None) -> np.ndarray:
    """W^0 on the grid.  rule (det F <= 0): 0 excluded (NaN); 1 (abs_det=True)
    ln|det F| for Eq. (2.3), and Eq. (2.2) kept everywhere."""
    W = np.empty(grid.count)
    lib().orc_grid_energy(mat.ref, grid.ref, float(beta_k), _rule(abs_det, rule), _p(W),
                          int(nthreads))
    return W


def grid_step(grid: Grid, off: np.ndarray, W: np.ndarray, want_h: bool = False,
              nthreads: int = 0):
    """One iteration of Eq. (4.3): (W_next, dir, l_minus, l_plus, decrease[, h])."""
    off = np.ascontiguousarray(off, dtype=np.int32).reshape(-1, grid.D)
    W = np.ascontiguousarray(W, dtype=np.float64)
    N = grid.count
    Wn = np.empty(N)
    d = np.empty(N, dtype=np.int32)
    lm = np.empty(N, dtype=np.int32)
    lp = np.empty(N, dtype=np.int32)
    h = np.empty((N, off.shape[0])) if want_h else None
    dec = lib().orc_grid_step(grid.ref, off.shape[0], _p(off), _p(W), _p(Wn), _p(d), _p(lm),
                              _p(lp), _p(h) if want_h else None, int(nthreads))
    out = (Wn, d, lm, lp, float(dec))
    return out + (h,) if want_h else out


def grid_convexify(mat: Material, grid: Grid, beta_k: float, off: np.ndarray, kmax: int = 20,
                   tol: float = 1e-4, abs_det: bool = False, nthreads: int = 0, rule=None,
                   keep_all: bool = True):
    """The global iteration (Sec. 4.1): W^0 = W on the grid, W^{k+1} by
    Eq. (4.3), stopped after kmax iterations or once the largest decrease is
    at most tol (Sec. 6).  Returns (W^k list, forest, decreases) with forest[k]
    = (dir, l_minus, l_plus) of iteration k + 1 (keep_all=False: only W^0 and
    W^K are kept)."""
    W = [grid_energy(mat, grid, beta_k, abs_det, nthreads, rule)]
    forest, decs = [], []
    for _ in range(kmax):
        Wn, d, lm, lp, dec = grid_step(grid, off, W[-1], nthreads=nthreads)
        if keep_all or len(W) < 2:
            W.append(Wn)
        else:
            W[-1] = Wn
        forest.append((d, lm, lp))
        decs.append(dec)
        if dec <= tol:
            break
    return W, forest, decs


def forest_array(forest) -> np.ndarray:
    """(K, N, 3) int32 records (dir, l_minus, l_plus) from grid_convexify's forest."""
    return np.ascontiguousarray(np.stack([np.stack(f, axis=-1) for f in forest]), dtype=np.int32)


def grid_query(mat: Material, grid: Grid, beta_k: float, off: np.ndarray, WK: np.ndarray, forest,
               F: np.ndarray, abs_det: bool = False, nthreads: int = 0, rule=None,
               want_A: bool = False):
    """(W_interp, W_tree, P, leaves[, A]) at points F (n x D) after
    K = len(forest) iterations: the multilinear interpolation of W^K, and
    Algorithm 3 over Algorithm 2's tree (A: n x D x D tangent)."""
    D = grid.D
    off = np.ascontiguousarray(off, dtype=np.int32).reshape(-1, D)
    fa = forest_array(forest) if not isinstance(forest, np.ndarray) else np.ascontiguousarray(forest, dtype=np.int32)
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, D)
    n = F.shape[0]
    wi, wt, P = np.empty(n), np.empty(n), np.empty((n, D))
    nl = np.empty(n, dtype=np.int64)
    A = np.empty((n, D, D)) if want_A else None
    lib().orc_grid_query(mat.ref, grid.ref, float(beta_k), _rule(abs_det, rule), _p(off),
                         fa.shape[0], _p(np.ascontiguousarray(WK, dtype=np.float64)), _p(fa), n,
                         _p(F), _p(wi), _p(wt), _p(P), _p(A) if want_A else None, _p(nl),
                         int(nthreads))
    return (wi, wt, P, nl, A) if want_A else (wi, wt, P, nl)
