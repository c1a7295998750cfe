"""The stored oracle results under tests/golden/*.npz: present, shaped as the
GPU parity tests expect, inputs equal to what the seeded generators give on
this host, and the oracle's trees consistent (a split's children lie on its
chosen rank-one line, W^R <= W).  CPU only."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ["material1m_l201", "mesh128", "loadpath512_s01", "loadpath512_s10", "loadpath512_s20"]
MAT = dict(mu=1.0, lam=5.0, Dinf=0.99, D0=0.5)


def _load(name):
    path = os.path.join(HERE, "golden", f"{name}.npz")
    assert os.path.exists(path), f"missing {path}: run tests/golden/make_goldens.py"
    g = dict(np.load(path))
    g["meta"] = json.loads(str(g["meta"]))
    return g


@pytest.mark.parametrize("name", NAMES)
def test_golden_file_shapes(name):
    g = _load(name)
    m = g["meta"]
    n, NT = 4096, (1 << (m["depth"] + 1)) - 1
    assert g["idx"].shape == (n,) and g["F"].shape == (n, 4) and g["beta"].shape == (n,)
    assert g["W_R"].shape == (n,) and g["P"].shape == (n, 4) and g["status"].shape == (n,)
    for k in ("flags", "margin", "dir", "m_minus", "m_plus"):
        assert g[k].shape == (n, NT), k
    assert g["node_F"].shape == (n, NT, 4)
    assert np.all(np.isfinite(g["W_R"][g["status"] == 0]))


@pytest.mark.parametrize("name", NAMES)
def test_golden_trees_consistent(orc, name):
    g = _load(name)
    m = g["meta"]
    mat = orc.Material(**MAT)
    dirs = orc.angle_directions(*m["angles"])
    m0 = (m["line_points"] - 1) // 2
    h = 2.0 * m["t_half"] / (m["line_points"] - 1)
    lam = (g["flags"] & orc.LAMINATED) > 0
    pi, ni = np.nonzero(lam)
    for p, i in zip(pi[:2000], ni[:2000]):
        R = orc.rank_one(dirs[g["dir"][p, i]])
        Fn = g["node_F"][p, i]
        np.testing.assert_allclose(g["node_F"][p, 2 * i + 1], Fn + (g["m_minus"][p, i] - m0) * h * R,
                                   atol=1e-14)
        np.testing.assert_allclose(g["node_F"][p, 2 * i + 2], Fn + (g["m_plus"][p, i] - m0) * h * R,
                                   atol=1e-14)
    W = np.array([orc.energy(mat, g["F"][p], g["beta"][p]) for p in range(0, 4096, 8)])
    assert np.all(g["W_R"][::8] <= W + 1e-15)


def test_golden_inputs_match_generators():
    """The stored inputs are the seeded generators' output (to rounding of the
    host's libm), so the full-size GPU runs place them at the right rows."""
    from paper_2211_14318_gb300 import inputs

    g = _load("mesh128")
    F, _ = inputs.mesh_points(128, stretch=1.3, seed=0)
    np.testing.assert_allclose(F[g["idx"]], g["F"], rtol=0, atol=1e-14)
    g = _load("material1m_l201")
    F, _ = inputs.surrogate_inputs(1 << 20, seed=201)
    np.testing.assert_allclose(F[g["idx"]], g["F"], rtol=0, atol=1e-14)


def test_uncertified_node_bar_rejects_a_worse_direction(orc):
    """The GPU tests' bar for an uncertified node (test_gpu_golden's
    overflow_node), applied to the oracle's own tree at load step 20 with the
    node relabelled as a GPU decision: the oracle's direction and a direction
    whose hull value lies 5e-8 above it (inside 2.25 eps) pass with their own
    bridges; the same direction with another bridge index, and direction
    8000 with its own (unsplit) bridge, 4.2e-6 above the minimum, fail."""
    import sys

    sys.path.insert(0, HERE)
    import test_gpu_golden as T
    from paper_2211_14318_gb300 import api

    g = T.load("loadpath512_s20")
    t = np.zeros((), dtype=[("flags", "<i4"), ("dir", "<i4"), ("m_minus", "<i4"),
                            ("m_plus", "<i4")])
    t["flags"] = api.NODE_SCANNED | api.NODE_LAMINATED | api.NODE_OVERFLOW
    for d, mm, mp, ok in [(0, 0, 1086, True), (516, 0, 1085, True), (516, 0, 1086, False),
                          (8000, 1024, 1024, False)]:
        t["dir"], t["m_minus"], t["m_plus"] = d, mm, mp
        if ok:
            assert T.overflow_node(orc, g, 300, 6, t) == pytest.approx(1.1e-6)
        else:
            with pytest.raises(AssertionError):
                T.overflow_node(orc, g, 300, 6, t)
