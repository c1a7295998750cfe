"""Python binding of libconvexify (C ABI in include/convexify.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors; calls are enqueued on the current
torch stream.  There is no CPU fallback: if the library is missing or no GPU
is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libconvexify.so")

CVX_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "TIMEOUT", -5: "NOT_TRAINED",
          -6: "UNSUPPORTED"}
ENERGY_NH_DAMAGE, ENERGY_DOUBLE_WELL, ENERGY_STVK_DAMAGE = 0, 1, 2
PT_NONPOS_DET, PT_TIE, PT_EDGE, PT_ITER_CAP, PT_OVERFLOW, PT_FALLBACK = 1, 2, 4, 8, 16, 32
NODE_EXISTS, NODE_SCANNED, NODE_LAMINATED, NODE_LEAF, NODE_TIE, NODE_EDGE = 1, 2, 4, 8, 16, 32
NODE_ITER_CAP, NODE_OVERFLOW, NODE_NEWTON, NODE_FALLBACK = 64, 128, 256, 512
FLAG_REFINE_NEWTON = 1

NODE_DTYPE = np.dtype([
    ("F", "<f8", (4,)), ("w", "<f8"), ("h", "<f8"), ("xi", "<f8"), ("weight", "<f8"),
    ("dir", "<i4"), ("m_minus", "<i4"), ("m_plus", "<i4"), ("flags", "<i4"),
    ("gap", "<f4"), ("window_exp", "<i4"),
])
LAMINATE_DTYPE = np.dtype([
    ("laminated", "<i4"), ("dir", "<i4"), ("m_minus", "<i4"), ("m_plus", "<i4"),
    ("xi", "<f8"), ("h", "<f8"), ("F_plus", "<f8", (4,)), ("F_minus", "<f8", (4,)),
])


class CvxError(RuntimeError):
    pass


class _Params(ctypes.Structure):
    _fields_ = [
        ("mu", ctypes.c_double), ("lambda_L", ctypes.c_double), ("D_inf", ctypes.c_double),
        ("D0", ctypes.c_double), ("t_half", ctypes.c_double),
        ("dirs", ctypes.POINTER(ctypes.c_double)),
        ("energy", ctypes.c_int32), ("n_theta_a", ctypes.c_int32), ("n_theta_b", ctypes.c_int32),
        ("n_dirs", ctypes.c_int32), ("line_points", ctypes.c_int32), ("depth", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("recentre", ctypes.c_int32),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "points", "nodes_scanned", "lines", "valid_samples", "laminated", "fp64_checks",
        "full_passes", "rare_paths", "ties", "iter_caps", "window_steps", "rounds", "fp64_window",
        "fp64_rare", "fp64_center", "refined", "overflow", "window_nodes", "fallbacks", "refine_full", "lines_bounded",
        "lines_flat", "recentred", "lines_certified", "edge_splits", "window_doublings",
        "mirror_windows", "mirror_won")]


class _Problem(ctypes.Structure):
    _fields_ = [
        ("params", _Params), ("n", ctypes.c_int64),
        ("F", ctypes.c_void_p), ("beta_k", ctypes.c_void_p), ("W_R", ctypes.c_void_p),
        ("P", ctypes.c_void_p), ("status", ctypes.c_void_p), ("root", ctypes.c_void_p),
    ]


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n", ctypes.c_int32 * 9), ("lo", ctypes.c_double * 9),
                ("delta", ctypes.c_double * 9)]


class _TrainCfg(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("init", ctypes.c_int32), ("seed", ctypes.c_uint64)]


SURROGATE_PARAMS = 200967

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Load libconvexify.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise CvxError(f"{LIB_PATH} is missing: build it with paper_2211_14318_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sigs = {
        "cvx_create": [ctypes.POINTER(vp), ctypes.c_int],
        "cvx_destroy": [vp],
        "cvx_last_error": [ctypes.c_char_p, ctypes.c_size_t],
        "cvx_get_stats": [vp, ctypes.POINTER(_Stats), ctypes.c_int],
        "cvx_set_tuning": [vp, ctypes.c_int, ctypes.c_int],
        "cvx_struct_size": [ctypes.c_int],
        "cvx_set_profiling": [vp, ctypes.c_int],
        "cvx_get_scan_timing": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                ctypes.c_int],
        "cvx_energy": [vp, ctypes.POINTER(_Params), i64, vp, vp, vp, vp, vp],
        "cvx_history_update": [vp, ctypes.POINTER(_Params), i64, vp, vp, vp, vp],
        "cvx_sample_lines": [vp, ctypes.POINTER(_Params), i64, vp, vp, vp, vp, vp],
        "cvx_hull_bridge": [vp, i64, i32, vp, vp, vp, vp, vp],
        "convexify_points": [vp, ctypes.POINTER(_Params), i64, vp, vp, vp, vp, vp, vp, vp, vp],
        "convexify_points_static": [ctypes.POINTER(_Params), i64, vp, vp, vp, vp, vp, vp],
        "cvx_tree_tangent": [vp, ctypes.POINTER(_Params), i64, vp, vp, vp, vp],
        "convexify_batch": [vp, ctypes.c_int, ctypes.POINTER(_Problem), vp],
        "surrogate_set_weights": [vp, vp, vp, vp],
        "surrogate_get_weights": [vp, vp, vp, vp],
        "surrogate_forward": [vp, i64, vp, vp, vp],
        "surrogate_loss_grad": [vp, i64, vp, vp, vp, vp, vp],
        "surrogate_train": [vp, i64, vp, vp, ctypes.POINTER(_TrainCfg), vp, vp],
        "surrogate_save": [vp, ctypes.c_char_p],
        "surrogate_load": [vp, ctypes.c_char_p],
        "cvx_gemm_bf16": [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp],
        "surrogate_labels": [vp, ctypes.POINTER(_Params), i64, vp, vp, vp, vp,
                             ctypes.POINTER(ctypes.c_int64), vp],
        "surrogate_propose": [vp, ctypes.POINTER(_Params), i64, vp, vp, ctypes.c_int,
                              ctypes.c_double, vp, vp, vp, vp, vp, vp, vp],
        "cvx_get_batch_tuning": [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)],
        "cvx_grid_r11": [i32, vp],
        "cvx_grid_energy": [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Grid), ctypes.c_double,
                            i32, vp, vp],
        "cvx_grid_step": [vp, ctypes.POINTER(_Grid), i32, vp, vp, vp, vp, vp, vp],
        "cvx_grid_convexify": [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Grid), ctypes.c_double,
                               i32, i32, vp, i32, ctypes.c_double, vp, vp, vp, vp, vp],
        "cvx_grid_query": [vp, ctypes.POINTER(_Params), ctypes.POINTER(_Grid), ctypes.c_double,
                           i32, i32, vp, i32, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = L
    return L


def exported_symbols() -> Sequence[str]:
    return ("cvx_create", "cvx_destroy", "cvx_last_error", "cvx_get_stats", "cvx_struct_size",
            "cvx_set_tuning", "cvx_set_profiling", "cvx_get_scan_timing",
            "cvx_energy", "cvx_history_update", "cvx_sample_lines", "cvx_hull_bridge",
            "convexify_points", "convexify_points_static", "convexify_batch", "cvx_tree_tangent",
            "cvx_get_batch_tuning", "surrogate_set_weights", "surrogate_get_weights",
            "surrogate_forward", "surrogate_loss_grad", "surrogate_train", "surrogate_save",
            "surrogate_load", "cvx_gemm_bf16", "surrogate_labels", "surrogate_propose",
            "cvx_grid_r11", "cvx_grid_energy", "cvx_grid_step", "cvx_grid_convexify",
            "cvx_grid_query")


def _check(rc: int, what: str):
    if rc != CVX_OK:
        buf = ctypes.create_string_buffer(512)
        lib().cvx_last_error(buf, 512)
        raise CvxError(f"{what}: {ERRORS.get(rc, rc)}: {buf.value.decode(errors='replace')}")


@dataclass
class Params:
    """cvx_params: material (Sec. 2), directions, line, depth."""
    mu: float = 1.0
    lambda_L: float = 5.0
    D_inf: float = 0.99
    D0: float = 0.5
    n_theta_a: int = 16
    n_theta_b: int = 16
    line_points: int = 201
    t_half: float = 0.5
    depth: int = 2
    energy: int = ENERGY_NH_DAMAGE
    dirs: Optional[np.ndarray] = None  # custom (n, 4) rows (a1, a2, b1, b2)
    newton: bool = False  # CVX_FLAG_REFINE_NEWTON
    gap_one_sided: bool = False  # CVX_FLAG_GAP_ONE_SIDED (surrogate_propose)
    recentre: int = 0  # surrogate_propose: window re-centrings (0..8)
    window_doublings: int = 0  # adaptive line window: doublings per node (0..8)
    mirror: bool = False  # CVX_FLAG_MIRROR_WINDOW (surrogate_propose)
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Params:
        p = _Params()
        p.mu, p.lambda_L, p.D_inf, p.D0, p.t_half = self.mu, self.lambda_L, self.D_inf, self.D0, self.t_half
        p.energy, p.n_theta_a, p.n_theta_b = self.energy, self.n_theta_a, self.n_theta_b
        p.line_points, p.depth, p.recentre = self.line_points, self.depth, self.recentre
        p.flags = ((FLAG_REFINE_NEWTON if self.newton else 0) | (2 if self.gap_one_sided else 0)
                   | (4 if self.mirror else 0) | (int(self.window_doublings) << 8))
        if self.dirs is not None:
            d = np.ascontiguousarray(self.dirs, dtype=np.float64).reshape(-1, 4)
            self._keep = [d]
            p.dirs = d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            p.n_dirs = d.shape[0]
        else:
            p.dirs = None
            p.n_dirs = 0
        return p

    @property
    def n_dirs(self) -> int:
        return self.dirs.shape[0] if self.dirs is not None else self.n_theta_a * self.n_theta_b

    @property
    def tree_size(self) -> int:
        return (1 << (self.depth + 1)) - 1


@dataclass
class GridSpec:
    """cvx_grid: the cuboid deformation-gradient grid of Sec. 5.2; the D = d^2
    components of F (row-major; D = 4 for d = 2, 9 for d = 3) take
    lo[c] + i delta[c], i = 0 .. n[c] - 1 (flat index with the last component
    fastest)."""
    n: tuple
    lo: tuple
    delta: tuple

    @classmethod
    def from_bounds(cls, diag, off, delta, dim: int = 2):
        """Every diagonal entry on diag = (lo, hi), every off-diagonal entry on
        off = (lo, hi), spacings delta = (diagonal, off-diagonal); hi is a grid
        value (the parametrisation of Tables tab:2Dconvexification and
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
        return cls(tuple(n), tuple(lo), tuple(de))

    @property
    def D(self) -> int:
        return len(self.n)

    @property
    def dim(self) -> int:
        return 2 if self.D == 4 else 3

    @property
    def count(self) -> int:
        return int(np.prod(self.n))

    def c(self) -> _Grid:
        pad = 9 - self.D
        return _Grid(self.dim, (ctypes.c_int32 * 9)(*([int(x) for x in self.n] + [0] * pad)),
                     (ctypes.c_double * 9)(*([float(x) for x in self.lo] + [0.0] * pad)),
                     (ctypes.c_double * 9)(*([float(x) for x in self.delta] + [0.0] * pad)))


def grid_r11(dim: int = 2) -> np.ndarray:
    """Grid-index offsets of the directions of Eq. (5.1): (16, 4) int32 for
    d = 2, (169, 9) for d = 3."""
    off = np.zeros((16, 4) if dim == 2 else (169, 9), dtype=np.int32)
    _check(lib().cvx_grid_r11(int(dim), off.ctypes.data), "cvx_grid_r11")
    return off


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream=None) -> Optional[int]:
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Convexifier:
    """A library handle bound to one CUDA device."""

    def __init__(self, device: int = 0):
        import torch

        if not torch.cuda.is_available():
            raise CvxError("no CUDA device: the convexification path has no CPU fallback")
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().cvx_create(ctypes.byref(h), device), "cvx_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().cvx_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ utilities
    def stats(self, reset: bool = False) -> dict:
        s = _Stats()
        _check(lib().cvx_get_stats(self._h, ctypes.byref(s), int(reset)), "cvx_get_stats")
        return {n: int(getattr(s, n)) for n, _ in _Stats._fields_}

    def set_tuning(self, warps_per_cta: int = 8, dirs_per_item: int = 0):
        _check(lib().cvx_set_tuning(self._h, warps_per_cta, dirs_per_item), "cvx_set_tuning")

    def set_profiling(self, enable: bool = True):
        _check(lib().cvx_set_profiling(self._h, int(enable)), "cvx_set_profiling")

    def scan_timing(self, reset: bool = True):
        """(total ms, launches) of the line-scan kernel since the last reset."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(lib().cvx_get_scan_timing(self._h, ctypes.byref(ms), ctypes.byref(n), int(reset)),
               "cvx_get_scan_timing")
        return ms.value, n.value

    def _dev(self, t, dtype):
        import torch

        t = torch.as_tensor(t, dtype=dtype)
        return t.to(f"cuda:{self.device}").contiguous()

    # -------------------------------------------------------- single steps
    def energy(self, p: Params, F, beta, want_P: bool = True, stream=None):
        import torch

        F = self._dev(F, torch.float64).reshape(-1, 4)
        beta = self._dev(beta, torch.float64).reshape(-1)
        n = F.shape[0]
        W = torch.empty(n, dtype=torch.float64, device=F.device)
        P = torch.empty(n, 4, dtype=torch.float64, device=F.device) if want_P else None
        c = p.c()
        _check(lib().cvx_energy(self._h, ctypes.byref(c), n, _ptr(F), _ptr(beta), _ptr(W), _ptr(P),
                                _stream(stream)), "cvx_energy")
        return W, P

    def history_update(self, p: Params, F, beta_in=None, stream=None):
        import torch

        F = self._dev(F, torch.float64).reshape(-1, 4)
        n = F.shape[0]
        bi = None if beta_in is None else self._dev(beta_in, torch.float64).reshape(n)
        out = torch.empty(n, dtype=torch.float64, device=F.device)
        c = p.c()
        _check(lib().cvx_history_update(self._h, ctypes.byref(c), n, _ptr(F), _ptr(bi), _ptr(out),
                                        _stream(stream)), "cvx_history_update")
        return out

    def sample_lines(self, p: Params, F, beta, dirs, stream=None):
        import torch

        F = self._dev(F, torch.float64).reshape(-1, 4)
        n = F.shape[0]
        beta = self._dev(beta, torch.float64).reshape(n)
        d = self._dev(dirs, torch.int32).reshape(n)
        w = torch.empty(n, p.line_points, dtype=torch.float32, device=F.device)
        c = p.c()
        _check(lib().cvx_sample_lines(self._h, ctypes.byref(c), n, _ptr(F), _ptr(beta), _ptr(d),
                                      _ptr(w), _stream(stream)), "cvx_sample_lines")
        return w

    def hull_bridge(self, w, stream=None):
        import torch

        w = self._dev(w, torch.float32)
        n, L = w.shape
        mm = torch.empty(n, dtype=torch.int32, device=w.device)
        mp = torch.empty(n, dtype=torch.int32, device=w.device)
        h = torch.empty(n, dtype=torch.float64, device=w.device)
        _check(lib().cvx_hull_bridge(self._h, n, L, _ptr(w), _ptr(mm), _ptr(mp), _ptr(h),
                                     _stream(stream)), "cvx_hull_bridge")
        return mm, mp, h

    # ----------------------------------------------------------- hot path
    def convexify_points(self, p: Params, F, beta, want_tree: bool = False,
                         want_root: bool = False, out: Optional[dict] = None, stream=None):
        """W^R, P (and optionally the tree / root laminate) for n points.

        ``out`` may hold preallocated tensors (W_R, P, status, tree, root)."""
        import torch

        F = self._dev(F, torch.float64).reshape(-1, 4)
        n = F.shape[0]
        beta = self._dev(beta, torch.float64).reshape(n)
        dev = F.device
        o = dict(out) if out else {}
        W_R = o.get("W_R") if o.get("W_R") is not None else torch.empty(n, dtype=torch.float64, device=dev)
        P = o.get("P") if o.get("P") is not None else torch.empty(n, 4, dtype=torch.float64, device=dev)
        st = o.get("status") if o.get("status") is not None else torch.empty(n, dtype=torch.int32, device=dev)
        tree = None
        if want_tree:
            tree = o.get("tree")
            if tree is None:
                tree = torch.empty(n * p.tree_size * NODE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        root = None
        if want_root:
            root = o.get("root")
            if root is None:
                root = torch.empty(n * LAMINATE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        c = p.c()
        _check(lib().convexify_points(self._h, ctypes.byref(c), n, _ptr(F), _ptr(beta), _ptr(W_R),
                                      _ptr(P), _ptr(root), _ptr(tree), _ptr(st), _stream(stream)),
               "convexify_points")
        return dict(W_R=W_R, P=P, status=st, tree=tree, root=root)

    def tree_tangent(self, p: Params, beta, tree, n: int, stream=None):
        """Tangent of W^R (n, 4, 4) over a tree output (Algorithm 3 on second
        derivatives)."""
        import torch

        beta = self._dev(beta, torch.float64).reshape(n)
        A = torch.empty(n, 4, 4, dtype=torch.float64, device=beta.device)
        c = p.c()
        _check(lib().cvx_tree_tangent(self._h, ctypes.byref(c), n, _ptr(beta), _ptr(tree), _ptr(A),
                                      _stream(stream)), "cvx_tree_tangent")
        return A

    def convexify_batch(self, problems, outs: Optional[list] = None, want_root: bool = False,
                        stream=None):
        """Several problems (a list of (Params, F, beta_k)) in one pipeline run.

        The library captures the run as a CUDA graph and replays it while the
        problems, parameters and tensors stay the same; pass ``outs`` (the list
        this call returns) back in to keep the output tensors fixed."""
        import torch

        arr = (_Problem * len(problems))()
        res = []
        keep = []
        for i, (p, F, beta) in enumerate(problems):
            F = self._dev(F, torch.float64).reshape(-1, 4)
            n = F.shape[0]
            beta = self._dev(beta, torch.float64).reshape(n)
            dev = F.device
            o = dict(outs[i]) if outs else {}
            if o.get("W_R") is None:
                o["W_R"] = torch.empty(n, dtype=torch.float64, device=dev)
            if o.get("P") is None:
                o["P"] = torch.empty(n, 4, dtype=torch.float64, device=dev)
            if o.get("status") is None:
                o["status"] = torch.empty(n, dtype=torch.int32, device=dev)
            if want_root and o.get("root") is None:
                o["root"] = torch.empty(n * LAMINATE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
            q = arr[i]
            q.params = p.c()
            keep.append((p, F, beta))
            q.n = n
            q.F, q.beta_k = _ptr(F), _ptr(beta)
            q.W_R, q.P, q.status = _ptr(o["W_R"]), _ptr(o["P"]), _ptr(o["status"])
            q.root = _ptr(o.get("root"))
            res.append(o)
        _check(lib().convexify_batch(self._h, len(problems), arr, _stream(stream)),
               "convexify_batch")
        return res

    # ----------------------------------------------------- surrogate network
    def gemm_bf16(self, A, B, stream=None):
        """C = A B^T (FP32) on the tensor cores; A (M x K), B (N x K) bf16."""
        import torch

        A = A.to(device=f"cuda:{self.device}", dtype=torch.bfloat16).contiguous()
        B = B.to(device=f"cuda:{self.device}", dtype=torch.bfloat16).contiguous()
        M, K = A.shape
        N = B.shape[0]
        C = torch.empty(M, N, dtype=torch.float32, device=A.device)
        _check(lib().cvx_gemm_bf16(self._h, M, N, K, _ptr(A), _ptr(B), _ptr(C), _stream(stream)),
               "cvx_gemm_bf16")
        return C

    def surrogate_set_weights(self, params, mean, std):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(SURROGATE_PARAMS)
        m = np.ascontiguousarray(mean, dtype=np.float32).reshape(6)
        sd = np.ascontiguousarray(std, dtype=np.float32).reshape(6)
        _check(lib().surrogate_set_weights(self._h, p.ctypes.data, m.ctypes.data, sd.ctypes.data),
               "surrogate_set_weights")

    def surrogate_get_weights(self):
        p = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
        m = np.zeros(6, dtype=np.float32)
        sd = np.zeros(6, dtype=np.float32)
        _check(lib().surrogate_get_weights(self._h, p.ctypes.data, m.ctypes.data, sd.ctypes.data),
               "surrogate_get_weights")
        return p, m, sd

    def surrogate_forward(self, X, stream=None):
        import torch

        X = self._dev(X, torch.float32).reshape(-1, 6)
        out = torch.empty(X.shape[0], 7, dtype=torch.float32, device=X.device)
        _check(lib().surrogate_forward(self._h, X.shape[0], _ptr(X), _ptr(out), _stream(stream)),
               "surrogate_forward")
        return out

    def surrogate_loss_grad(self, X, Y, stream=None):
        import torch

        X = self._dev(X, torch.float32).reshape(-1, 6)
        Y = self._dev(Y, torch.float32).reshape(-1, 7)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        grad = torch.empty(SURROGATE_PARAMS, dtype=torch.float32, device=X.device)
        _check(lib().surrogate_loss_grad(self._h, X.shape[0], _ptr(X), _ptr(Y), _ptr(loss),
                                         _ptr(grad), _stream(stream)), "surrogate_loss_grad")
        return loss, grad

    def surrogate_train(self, X, Y, epochs: int, batch: int = 8192, lr: float = 1e-3,
                        init: bool = True, seed: int = 0, stream=None):
        import torch

        X = self._dev(X, torch.float32).reshape(-1, 6)
        Y = self._dev(Y, torch.float32).reshape(-1, 7)
        cfg = _TrainCfg(epochs, batch, lr, 1 if init else 0, seed)
        log = np.zeros(max(epochs, 1), dtype=np.float32)
        _check(lib().surrogate_train(self._h, X.shape[0], _ptr(X), _ptr(Y), ctypes.byref(cfg),
                                     log.ctypes.data, _stream(stream)), "surrogate_train")
        return log[:epochs]

    def surrogate_labels(self, p: Params, beta, tree, n: int, stream=None):
        """(X, Y) training samples from the scanned nodes of n trees."""
        import torch

        beta = self._dev(beta, torch.float64).reshape(n)
        cap = max(1, n * p.tree_size)
        X = torch.empty(cap, 6, dtype=torch.float32, device=beta.device)
        Y = torch.empty(cap, 7, dtype=torch.float32, device=beta.device)
        cnt = ctypes.c_int64()
        c = p.c()
        _check(lib().surrogate_labels(self._h, ctypes.byref(c), n, _ptr(beta), _ptr(tree), _ptr(X),
                                      _ptr(Y), ctypes.byref(cnt), _stream(stream)),
               "surrogate_labels")
        return X[:cnt.value], Y[:cnt.value]

    def surrogate_propose(self, p: Params, F, beta, window: int = 4, gap_tol: float = 1e-6,
                          want_tree: bool = False, want_root: bool = False,
                          out: Optional[dict] = None, stream=None):
        """W^R, P, status and fell_back (uint8) by the surrogate-proposed form."""
        import torch

        F = self._dev(F, torch.float64).reshape(-1, 4)
        n = F.shape[0]
        beta = self._dev(beta, torch.float64).reshape(n)
        dev = F.device
        o = dict(out) if out else {}
        W_R = o.get("W_R") if o.get("W_R") is not None else torch.empty(n, dtype=torch.float64, device=dev)
        P = o.get("P") if o.get("P") is not None else torch.empty(n, 4, dtype=torch.float64, device=dev)
        st = o.get("status") if o.get("status") is not None else torch.empty(n, dtype=torch.int32, device=dev)
        fb = o.get("fell_back") if o.get("fell_back") is not None else torch.empty(n, dtype=torch.uint8, device=dev)
        tree = None
        if want_tree:
            tree = o.get("tree")
            if tree is None:
                tree = torch.empty(n * p.tree_size * NODE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        root = None
        if want_root:
            root = o.get("root")
            if root is None:
                root = torch.empty(n * LAMINATE_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        c = p.c()
        _check(lib().surrogate_propose(self._h, ctypes.byref(c), n, _ptr(F), _ptr(beta), window,
                                       gap_tol, _ptr(W_R), _ptr(P), _ptr(root), _ptr(tree),
                                       _ptr(fb), _ptr(st), _stream(stream)), "surrogate_propose")
        return dict(W_R=W_R, P=P, status=st, fell_back=fb, tree=tree, root=root)

    def surrogate_save(self, path: str):
        _check(lib().surrogate_save(self._h, path.encode()), "surrogate_save")

    def surrogate_load(self, path: str):
        _check(lib().surrogate_load(self._h, path.encode()), "surrogate_load")

    # ------------------------------------------------------ global-grid form
    def grid_energy(self, p: Params, grid: GridSpec, beta_k: float, det_rule: int = 0,
                    stream=None):
        """W^0 on the grid (N values, flat order)."""
        import torch

        W = torch.empty(grid.count, dtype=torch.float64, device=f"cuda:{self.device}")
        c, g = p.c(), grid.c()
        _check(lib().cvx_grid_energy(self._h, ctypes.byref(c), ctypes.byref(g), float(beta_k),
                                     int(det_rule), _ptr(W), _stream(stream)), "cvx_grid_energy")
        return W

    def grid_step(self, grid: GridSpec, off, W_in, stream=None):
        """One iteration of Eq. (4.3): (W_out, lam (N x 3 int32), dec (device scalar))."""
        import torch

        off = np.ascontiguousarray(off, dtype=np.int32).reshape(-1, grid.D)
        W_in = self._dev(W_in, torch.float64).reshape(-1)
        W_out = torch.empty_like(W_in)
        lam = torch.empty(grid.count, 3, dtype=torch.int32, device=W_in.device)
        dec = torch.empty(1, dtype=torch.float64, device=W_in.device)
        g = grid.c()
        _check(lib().cvx_grid_step(self._h, ctypes.byref(g), off.shape[0], off.ctypes.data,
                                   _ptr(W_in), _ptr(W_out), _ptr(lam), _ptr(dec),
                                   _stream(stream)), "cvx_grid_step")
        return W_out, lam, dec

    def grid_convexify(self, p: Params, grid: GridSpec, beta_k: float, off, kmax: int = 20,
                       tol: float = 1e-4, det_rule: int = 0, want_forest: bool = True,
                       out: Optional[dict] = None, stream=None):
        """The global iteration of Sec. 4.1 on the device: dict with W (= W^K),
        forest (kmax x N x 3, rows >= K unwritten), decs (kmax) and iters (a
        device int32; read it to get K).  ``out`` may hold preallocated
        tensors with those names."""
        import torch

        off = np.ascontiguousarray(off, dtype=np.int32).reshape(-1, grid.D)
        dev = f"cuda:{self.device}"
        N = grid.count
        o = dict(out) if out else {}
        W = o.get("W") if o.get("W") is not None else torch.empty(N, dtype=torch.float64, device=dev)
        forest = None
        if want_forest:
            forest = o.get("forest")
            if forest is None:
                forest = torch.empty(kmax, N, 3, dtype=torch.int32, device=dev)
        decs = o.get("decs") if o.get("decs") is not None else torch.empty(kmax, dtype=torch.float64, device=dev)
        iters = o.get("iters") if o.get("iters") is not None else torch.empty(1, dtype=torch.int32, device=dev)
        c, g = p.c(), grid.c()
        _check(lib().cvx_grid_convexify(self._h, ctypes.byref(c), ctypes.byref(g), float(beta_k),
                                        int(det_rule), off.shape[0], off.ctypes.data, int(kmax),
                                        float(tol), _ptr(W), _ptr(forest), _ptr(decs),
                                        _ptr(iters), _stream(stream)), "cvx_grid_convexify")
        return dict(W=W, forest=forest, decs=decs, iters=iters)

    def grid_query(self, p: Params, grid: GridSpec, beta_k: float, off, WK, forest, F,
                   det_rule: int = 0, K: Optional[int] = None, want_A: bool = False,
                   stream=None):
        """(W_interp, W_tree, P (n x D), leaves[, A (n x D x D)]) at points F
        (n x D) from W^K and the first K forest rows (K = len(forest) unless
        given)."""
        import torch

        off = np.ascontiguousarray(off, dtype=np.int32).reshape(-1, grid.D)
        WK = self._dev(WK, torch.float64).reshape(-1)
        fa = self._dev(forest, torch.int32).reshape(-1, grid.count, 3)
        K = fa.shape[0] if K is None else int(K)
        F = self._dev(F, torch.float64).reshape(-1, grid.D)
        n = F.shape[0]
        wi = torch.empty(n, dtype=torch.float64, device=F.device)
        wt = torch.empty(n, dtype=torch.float64, device=F.device)
        P = torch.empty(n, grid.D, dtype=torch.float64, device=F.device)
        nl = torch.empty(n, dtype=torch.int64, device=F.device)
        A = torch.empty(n, grid.D, grid.D, dtype=torch.float64, device=F.device) if want_A else None
        c, g = p.c(), grid.c()
        _check(lib().cvx_grid_query(self._h, ctypes.byref(c), ctypes.byref(g), float(beta_k),
                                    int(det_rule), off.shape[0], off.ctypes.data, K, _ptr(WK),
                                    _ptr(fa), n, _ptr(F), _ptr(wi), _ptr(wt), _ptr(P), _ptr(A),
                                    _ptr(nl), _stream(stream)), "cvx_grid_query")
        return (wi, wt, P, nl, A) if want_A else (wi, wt, P, nl)

    def batch_tuning(self):
        """(warps per CTA, directions-per-item cap, taken from the cache) of the
        last convexify_batch launch-shape choice."""
        w, d, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().cvx_get_batch_tuning(self._h, ctypes.byref(w), ctypes.byref(d),
                                          ctypes.byref(c)), "cvx_get_batch_tuning")
        return w.value, d.value, bool(c.value)


def tree_numpy(tree_bytes, n: int, tree_size: int) -> np.ndarray:
    """Device tree bytes -> (n, tree_size) structured array (host)."""
    return tree_bytes.cpu().numpy().view(NODE_DTYPE).reshape(n, tree_size)


def root_numpy(root_bytes, n: int) -> np.ndarray:
    return root_bytes.cpu().numpy().view(LAMINATE_DTYPE).reshape(n)


def convexify_points_static(p: Params, F, beta, stream=None):
    """The allocation-free entry point (fixed library scratch, no handle): W^R,
    P and status for points already on the current CUDA device."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    F = torch.as_tensor(F, dtype=torch.float64).to(dev).reshape(-1, 4).contiguous()
    n = F.shape[0]
    beta = torch.as_tensor(beta, dtype=torch.float64).to(dev).reshape(n).contiguous()
    W_R = torch.empty(n, dtype=torch.float64, device=dev)
    P = torch.empty(n, 4, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    c = p.c()
    _check(lib().convexify_points_static(ctypes.byref(c), n, _ptr(F), _ptr(beta), _ptr(W_R),
                                         _ptr(P), _ptr(st), _stream(stream)),
           "convexify_points_static")
    return dict(W_R=W_R, P=P, status=st)
