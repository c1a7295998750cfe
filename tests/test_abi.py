"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
function include/convexify.h declares, its struct layouts match the binding,
and argument validation rejects bad input before any CUDA call.  No compute
call is made here (there is no GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "convexify.h")


def _declared():
    txt = open(HEADER).read()
    return re.findall(r"^int\s+(\w+)\s*\(", txt, flags=re.M)


@pytest.fixture(scope="module")
def cvxlib():
    from paper_2211_14318_gb300 import api, build

    build.build()
    api._lib = None
    return api.lib()


def test_header_declares_the_boundary():
    names = set(_declared())
    for n in ("convexify_points", "cvx_create", "cvx_destroy", "cvx_last_error",
              "cvx_hull_bridge", "cvx_sample_lines", "cvx_energy", "cvx_history_update"):
        assert n in names


def test_library_exports_every_declared_symbol(cvxlib):
    from paper_2211_14318_gb300 import api

    for n in _declared():
        assert hasattr(cvxlib, n), n
    assert set(api.exported_symbols()) <= set(_declared())


def test_struct_layouts_match_binding(cvxlib):
    from paper_2211_14318_gb300 import api

    assert cvxlib.cvx_struct_size(0) == ctypes.sizeof(api._Params)
    assert cvxlib.cvx_struct_size(1) == api.NODE_DTYPE.itemsize
    assert cvxlib.cvx_struct_size(2) == api.LAMINATE_DTYPE.itemsize
    assert cvxlib.cvx_struct_size(3) == ctypes.sizeof(api._Stats)
    assert cvxlib.cvx_struct_size(4) == ctypes.sizeof(api._Problem)
    assert cvxlib.cvx_struct_size(7) == -1


def _err(cvxlib):
    buf = ctypes.create_string_buffer(256)
    cvxlib.cvx_last_error(buf, 256)
    return buf.value.decode()


@pytest.mark.parametrize("field,value,msg", [
    ("line_points", 200, "line_points"),
    ("line_points", 1, "line_points"),
    ("line_points", 4001, "line_points"),
    ("depth", 9, "depth"),
    ("depth", -1, "depth"),
    ("t_half", 0.0, "t_half"),
    ("D_inf", 1.0, "material"),
    ("mu", -1.0, "material"),
    ("energy", 7, "energy"),
    ("n_theta_a", 0, "angle grid"),
    ("flags", 8, "flags"),
])
def test_invalid_params_rejected_before_cuda(cvxlib, field, value, msg):
    from paper_2211_14318_gb300 import api

    p = api.Params(line_points=201, depth=2)
    c = p.c()
    setattr(c, field, value)
    rc = cvxlib.convexify_points(None, ctypes.byref(c), 4, None, None, None, None, None, None, None,
                                 None)
    assert rc == -1
    assert msg in _err(cvxlib)


def test_null_handle_and_arrays_rejected(cvxlib):
    from paper_2211_14318_gb300 import api

    c = api.Params().c()
    assert cvxlib.convexify_points(None, ctypes.byref(c), 4, None, None, None, None, None, None,
                                   None, None) == -1
    assert "handle" in _err(cvxlib)
    assert cvxlib.cvx_hull_bridge(None, 1, 4, None, None, None, None, None) == -1
    assert "odd" in _err(cvxlib)
    assert cvxlib.cvx_set_tuning(None, 8, 0) == -1
    assert cvxlib.cvx_energy(None, None, 1, None, None, None, None, None) == -1
    assert "params" in _err(cvxlib)


def _problems(*params_and_n):
    from paper_2211_14318_gb300 import api

    arr = (api._Problem * len(params_and_n))()
    for q, (p, n) in zip(arr, params_and_n):
        q.params = p.c()
        q.n = n
    return arr


def test_batch_validation_before_cuda(cvxlib):
    from paper_2211_14318_gb300 import api

    ok = api.Params(line_points=201, depth=2)
    assert cvxlib.convexify_batch(None, 0, None, None) == -1
    assert "problems" in _err(cvxlib)
    bad = api.Params(line_points=200)
    assert cvxlib.convexify_batch(None, 2, _problems((ok, 0), (bad, 0)), None) == -1
    assert "line_points" in _err(cvxlib)
    dw = api.Params(energy=api.ENERGY_DOUBLE_WELL)
    assert cvxlib.convexify_batch(None, 2, _problems((ok, 0), (dw, 0)), None) == -1
    assert "same energy" in _err(cvxlib)
    assert cvxlib.convexify_batch(None, 1, _problems((ok, 5)), None) == -1
    assert "NULL array" in _err(cvxlib)
    assert cvxlib.convexify_batch(None, 1, _problems((ok, -1)), None) == -1
    assert cvxlib.convexify_batch(None, 1, _problems((ok, 0)), None) == -1
    assert "handle" in _err(cvxlib)
    w, d, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert cvxlib.cvx_get_batch_tuning(None, ctypes.byref(w), ctypes.byref(d), ctypes.byref(c)) == -1


def test_create_without_gpu_fails_cleanly(cvxlib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = cvxlib.cvx_create(ctypes.byref(h), 0)
    assert rc in (-1, -2) and not h.value


def test_binding_refuses_cpu_fallback():
    import torch

    from paper_2211_14318_gb300 import api

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(api.CvxError):
        api.Convexifier(0)


@pytest.mark.parametrize("na,nb,msg", [
    (65536, 65536, "angle grid"),   # 2^32 directions: wraps to 0 in 32-bit arithmetic
    (46341, 46341, "angle grid"),   # wraps to a negative count in 32-bit arithmetic
    (200, 200, "16384"),            # valid grid, above the static limit
])
def test_static_entry_rejects_direction_counts_before_cuda(cvxlib, na, nb, msg):
    from paper_2211_14318_gb300 import api

    c = api.Params(n_theta_a=na, n_theta_b=nb, line_points=201, depth=2).c()
    rc = cvxlib.convexify_points_static(ctypes.byref(c), 4, None, None, None, None, None, None)
    assert rc == -1
    assert msg in _err(cvxlib)


def test_grid_struct_and_r11_table(cvxlib, orc):
    """cvx_grid's layout matches the binding, and the library's table of the
    directions of Eq. (5.1) is the same reading, in the same order, as the
    oracle's (the order decides ties between directions)."""
    from paper_2211_14318_gb300 import api

    assert cvxlib.cvx_struct_size(5) == ctypes.sizeof(api._Grid)
    np_off = api.grid_r11()
    assert np_off.shape == (16, 4)
    assert (np_off == orc.r11_directions()).all()
    g = api.GridSpec.from_bounds((0.1, 3.4), (-2.55, 2.55), (0.15, 0.15))
    assert g.count == 648025 and g.n == (23, 35, 35, 23)
    off3 = api.grid_r11(3)
    assert off3.shape == (169, 9) and (off3 == orc.r11_directions(3)).all()
    g3 = api.GridSpec.from_bounds((1.0, 3.4), (-0.15, 0.15), (0.15, 0.15), dim=3)
    assert g3.count == 3581577 and g3.D == 9


@pytest.mark.parametrize("n,off,msg", [
    ((0, 3, 3, 3), None, "grid points"),
    ((3, 3, 3, 600), None, "grid points"),
    ((3, 3, 3, 3), [[0, 0, 0, 0]], "zero"),
    ((3, 3, 3, 3), [[1, 1, 0, 1]], "rank-one"),
    ((3, 3, 3, 3), [[1000, 0, 0, 0]], "offset"),
])
def test_grid_validation_before_cuda(cvxlib, n, off, msg):
    import numpy as np

    from paper_2211_14318_gb300 import api

    g = api.GridSpec(n, (0.0,) * 4, (0.1,) * 4).c()
    o = np.ascontiguousarray(off if off is not None else api.grid_r11(2), dtype=np.int32)
    rc = cvxlib.cvx_grid_step(None, ctypes.byref(g), o.shape[0], o.ctypes.data, None, None,
                              None, None, None)
    assert rc == -1
    assert msg in _err(cvxlib)


def test_grid_calls_reject_bad_arguments_before_cuda(cvxlib):
    import numpy as np

    from paper_2211_14318_gb300 import api

    g = api.GridSpec((3, 3, 3, 3), (0.5,) * 4, (0.25,) * 4).c()
    c = api.Params().c()
    o = api.grid_r11()
    assert cvxlib.cvx_grid_convexify(None, ctypes.byref(c), ctypes.byref(g), 0.0, 0, 16,
                                     o.ctypes.data, 0, 1e-4, None, None, None, None, None) == -1
    assert "kmax" in _err(cvxlib)
    assert cvxlib.cvx_grid_convexify(None, ctypes.byref(c), ctypes.byref(g), 0.0, 0, 16,
                                     o.ctypes.data, 20, float("nan"), None, None, None, None,
                                     None) == -1
    assert "tol" in _err(cvxlib)
    assert cvxlib.cvx_grid_convexify(None, ctypes.byref(c), ctypes.byref(g), 0.0, 0, 16,
                                     o.ctypes.data, 20, 1e-4, None, None, None, None, None) == -1
    assert "handle" in _err(cvxlib)
    assert cvxlib.cvx_grid_query(None, ctypes.byref(c), ctypes.byref(g), 0.0, 0, 16,
                                 o.ctypes.data, 65, None, None, 1, None, None, None, None, None,
                                 None, None) == -1
    assert "K must" in _err(cvxlib)
    assert cvxlib.cvx_grid_step(None, ctypes.byref(g), 0, o.ctypes.data, None, None, None, None,
                                None) == -1
    assert "direction count" in _err(cvxlib)
    assert cvxlib.cvx_grid_energy(None, ctypes.byref(c), ctypes.byref(g), float("inf"), 0, None,
                                  None) == -1
    assert "handle" in _err(cvxlib) or "beta" in _err(cvxlib)
    assert cvxlib.cvx_grid_r11(2, None) == -1
    buf = np.zeros(64, dtype=np.int32)
    assert cvxlib.cvx_grid_r11(4, buf.ctypes.data) == -1
    assert "dim" in _err(cvxlib)
    g.dim = 4
    assert cvxlib.cvx_grid_step(None, ctypes.byref(g), 16, o.ctypes.data, None, None, None, None,
                                None) == -1
    assert "dim" in _err(cvxlib)
    g.dim = 2
    assert cvxlib.cvx_grid_energy(None, ctypes.byref(c), ctypes.byref(g), 0.0, 2, None,
                                  None) == -1
    assert "det_rule" in _err(cvxlib)
    g3 = api.GridSpec((3,) * 9, (0.5,) * 9, (0.25,) * 9).c()
    dw = api.Params(energy=api.ENERGY_DOUBLE_WELL).c()
    assert cvxlib.cvx_grid_energy(None, ctypes.byref(dw), ctypes.byref(g3), 0.0, 0, None,
                                  None) == -1
    assert "two-dimensional" in _err(cvxlib)
    # a rank-two offset in nine components
    o3 = np.zeros((1, 9), dtype=np.int32)
    o3[0, 0] = o3[0, 4] = 1
    assert cvxlib.cvx_grid_step(None, ctypes.byref(g3), 1, o3.ctypes.data, None, None, None,
                                None, None) == -1
    assert "rank-one" in _err(cvxlib)


def test_stvk_energy_is_grid_only(cvxlib):
    """Eq. (2.2) is built for the global-grid calls; the per-point calls say
    so before any CUDA call."""
    from paper_2211_14318_gb300 import api

    c = api.Params(energy=api.ENERGY_STVK_DAMAGE).c()
    assert cvxlib.convexify_points(None, ctypes.byref(c), 4, None, None, None, None, None, None,
                                   None, None) == -6
    assert "global-grid" in _err(cvxlib)
    assert cvxlib.convexify_points_static(ctypes.byref(c), 4, None, None, None, None, None,
                                          None) == -6
