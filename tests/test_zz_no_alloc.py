"""The allocation-free Jacobian application (dg_apply_jacobian_static), called through the C ABI.

Some callers cannot allocate device memory when they apply the operator (a host application that owns
all device memory through its own pool, or a loop where cudaMalloc is not allowed after start-up).  For
them the library keeps its work space in a fixed device array.  This test checks that entry point
against the regular one (dg_setup + dg_apply_jacobian) on two calls in a row, so that a second call
reusing the array's leftover contents is covered too.  It sits in a file that pytest collects last.
"""

import ctypes

import numpy as np
import pytest

from paper_1711_10885_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1711_10885_gb300 import dg as _dg
    _dg.lib.dg_apply_jacobian_static.argtypes = [ctypes.POINTER(_dg.dg_mesh), ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return _dg


def _call_static(dg, w, D_dev, z, y, sigma):
    mesh = dg.dg_mesh()
    for r in range(3):
        mesh.lo[r], mesh.hi[r], mesh.n[r] = float(w.lo[r]), float(w.hi[r]), int(w.n[r])
    b = (ctypes.c_double * 3)(*[float(v) for v in w.b])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return dg.lib.dg_apply_jacobian_static(ctypes.byref(mesh), w.k, ctypes.c_void_p(D_dev.data_ptr()), b, w.c, sigma,
                                           ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)


# small meshes (the quarter-tile launch variant) and a k = 7 mesh of 2940 cells whose work space fills 30.5 of
# the 32 MiB (the full-tile variant, and every offset of the array in use)
@pytest.mark.parametrize("n,k", [((6, 5, 4), 4), ((3, 4, 5), 7), ((14, 14, 15), 7)])
def test_static_matches_regular_apply_on_two_calls(dg, n, k):
    w = inputs.small_case(n=n, k=k, seed=40 + k, b=(0.6, -0.3, 0.9))
    sigma = dg.dg_penalty_sigma(k, 0)
    op = dg.Operator(w.n, w.k, w.D, b=w.b, c=w.c, sigma=sigma)
    D_dev = torch.tensor(w.D, device="cuda")
    rng = np.random.default_rng(77)
    for call in range(2):
        z = torch.tensor(rng.uniform(-1, 1, w.ndof), device="cuda")
        y_ref = op.apply_jacobian(z)
        y = torch.full_like(z, float("nan"))
        assert _call_static(dg, w, D_dev, z, y, sigma) == 0, dg.lib.dg_last_error()
        torch.cuda.synchronize()
        err = (torch.max(torch.abs(y - y_ref)) / torch.max(torch.abs(y_ref))).item()
        assert err <= TOL64, (call, err)
    # a third call with the same vectors leaves the device's free memory unchanged: nothing is allocated
    free_before = torch.cuda.mem_get_info()[0]
    assert _call_static(dg, w, D_dev, z, y, sigma) == 0, dg.lib.dg_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    op.close()


def test_static_rejects_problems_beyond_the_fixed_size(dg):
    w = inputs.small_case(n=(20, 20, 20), k=7, seed=3)  # 8000 cells at k = 7: over the fixed work space
    D_dev = torch.tensor(w.D, device="cuda")
    z = torch.zeros(w.ndof, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(z)
    rc = _call_static(dg, w, D_dev, z, y, dg.dg_penalty_sigma(7, 0))
    assert rc == -1 and b"fixed" in dg.lib.dg_last_error()
