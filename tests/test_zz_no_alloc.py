"""The allocation-free entry point convexify_points_static.

For callers that may not allocate device memory (a material routine inside a
host finite-element code that owns all device memory, or a caller that cannot
accept cudaMalloc's device synchronisation): it must give what
convexify_points gives on the same inputs, call after call, although all its
scratch lives in one fixed array that every call reuses.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAT = dict(mu=1.0, lambda_L=5.0, D_inf=0.99, D0=0.5)


@pytest.fixture(scope="module")
def cv():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api

    c = api.Convexifier(0)
    yield c
    c.close()


def _check_same(ref, got):
    np.testing.assert_array_equal(got["status"].cpu().numpy(), ref["status"].cpu().numpy())
    Wr, Wg = ref["W_R"].cpu().numpy(), got["W_R"].cpu().numpy()
    assert np.max(np.abs(Wg - Wr) / (1e-8 + np.abs(Wr))) < 1e-6
    Pr, Pg = ref["P"].cpu().numpy(), got["P"].cpu().numpy()
    assert np.max(np.linalg.norm(Pg - Pr, axis=1) / (1e-8 + np.linalg.norm(Pr, axis=1))) < 1e-5


def test_static_entry_matches_convexify_points_twice(cv):
    import torch

    import oracle
    from paper_2211_14318_gb300 import api, inputs

    mat = oracle.Material(MAT["mu"], MAT["lambda_L"], MAT["D_inf"], MAT["D0"])
    # first call: 64 material points, 16 x 16 angles, L = 201, depth 2
    F1, Fp1 = inputs.material_points(64, seed=0)
    b1 = oracle.history_update(mat, Fp1)
    p1 = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    ref1 = cv.convexify_points(p1, F1, b1)
    got1 = api.convexify_points_static(p1, F1, b1)
    torch.cuda.synchronize()
    _check_same(ref1, got1)
    # second call right after, different sizes: stale scratch must not leak
    F2, Fp2 = inputs.material_points(37, seed=9, lam_hi=1.8)
    b2 = oracle.history_update(mat, Fp2)
    p2 = api.Params(n_theta_a=7, n_theta_b=9, line_points=77, t_half=0.6, depth=3, **MAT)
    ref2 = cv.convexify_points(p2, F2, b2)
    got2 = api.convexify_points_static(p2, F2, b2)
    torch.cuda.synchronize()
    _check_same(ref2, got2)
    # and the first problem again
    got3 = api.convexify_points_static(p1, F1, b1)
    torch.cuda.synchronize()
    _check_same(ref1, got3)


def test_static_entry_leaves_device_memory_unchanged(cv):
    """The defining property: with inputs and outputs already on the device,
    calls of different shapes take no device memory (cudaMemGetInfo's free
    bytes are the same before and after)."""
    import ctypes

    import torch

    import oracle
    from paper_2211_14318_gb300 import api, inputs

    mat = oracle.Material(MAT["mu"], MAT["lambda_L"], MAT["D_inf"], MAT["D0"])
    dev = torch.device("cuda", torch.cuda.current_device())
    shapes = [(64, api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)),
              (37, api.Params(n_theta_a=7, n_theta_b=9, line_points=77, t_half=0.6, depth=3, **MAT)),
              (500, api.Params(n_theta_a=32, n_theta_b=32, line_points=513, depth=2, **MAT))]
    bufs = []
    for n, p in shapes:
        F, Fp = inputs.material_points(n, seed=n)
        b = oracle.history_update(mat, Fp)
        bufs.append((p, n, torch.from_numpy(F).to(dev), torch.from_numpy(b).to(dev),
                     torch.empty(n, dtype=torch.float64, device=dev),
                     torch.empty(n, 4, dtype=torch.float64, device=dev),
                     torch.empty(n, dtype=torch.int32, device=dev)))

    def call(p, n, F, b, W, P, st):
        c = p.c()
        rc = api.lib().convexify_points_static(ctypes.byref(c), n, F.data_ptr(), b.data_ptr(),
                                               W.data_ptr(), P.data_ptr(), st.data_ptr(), None)
        assert rc == 0

    call(*bufs[0])  # warm: the first call on a device looks up the scratch address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        for args in bufs:
            call(*args)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_entry_rejects_oversized_problems(cv):
    from paper_2211_14318_gb300 import api

    p = api.Params(n_theta_a=200, n_theta_b=200, **MAT)  # 40,000 directions
    with pytest.raises(api.CvxError, match="16384"):
        api.convexify_points_static(p, np.tile([1.1, 0, 0, 1.0], (4, 1)), np.zeros(4))
    p = api.Params(n_theta_a=8, n_theta_b=8, depth=8, **MAT)
    with pytest.raises(api.CvxError, match="64 MiB"):
        api.convexify_points_static(p, np.tile([1.1, 0, 0, 1.0], (20000, 1)), np.zeros(20000))
