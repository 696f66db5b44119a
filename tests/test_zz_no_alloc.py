"""The allocation-free analysis entry point against the plan-based one.

Some callers cannot allocate device memory (a fixed memory budget after
start-up, pipelines that cannot take the synchronisation an allocation may
imply); muffin_op_analysis_noalloc serves them with a fixed scratch array in
the library.  This file is collected last on purpose.  The test calls the new
entry point twice in a row through the C ABI and compares each result with
muffin_op_analysis on the same input, at the wavelet tolerance of the other
GPU tests (relative L2 1e-6)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu


def test_noalloc_analysis_matches_plan_operator_twice():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    lib = pkg.library()
    n, L, K, J = 256, 6, 8, 3
    rng = np.random.default_rng(2024)
    x = dev(rng.standard_normal((L, n, n)), torch)
    psf = np.zeros((L, n, n), np.float32)
    psf[:, 0, 0] = 1.0
    u_ref = torch.empty((L, K, n, n), device="cuda")
    with pkg.Plan(n, L, psf, n_wavelets=K, levels=J) as plan:
        plan.op_analysis(x, u_ref)
    ref = host(u_ref)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        u = torch.full((L, K, n, n), float("nan"), device="cuda")
        st = lib.muffin_op_analysis_noalloc(ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(u.data_ptr()),
                                            n, L, K, J, stream)
        assert st == 0, lib.muffin_last_error().decode()
        torch.cuda.synchronize()
        e = rel_l2(host(u), ref)
        assert e <= 1e-6, (call, e)


def test_noalloc_rejects_oversized_and_host_arrays():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    lib = pkg.library()
    n, L, K, J = 2048, 16, 8, 3       # needs 16*8*(1024^2+512^2) floats > 4 Mi
    x = torch.empty((1,), device="cuda")
    st = lib.muffin_op_analysis_noalloc(ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(x.data_ptr()), n, L, K, J, None)
    assert st == 1 and b"scratch" in lib.muffin_last_error()
    h = np.zeros(16, np.float32)
    st = lib.muffin_op_analysis_noalloc(ctypes.c_void_p(h.ctypes.data),
                                        ctypes.c_void_p(h.ctypes.data), 4, 1, 1, 1, None)
    assert st == 1 and b"device" in lib.muffin_last_error()
