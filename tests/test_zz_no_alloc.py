"""The allocation-free analysis entry point against the plan-based one and
against the FP64 oracle.

Some callers cannot allocate device memory (a fixed memory budget after
start-up, pipelines that cannot take the synchronisation an allocation may
imply); muffin_op_analysis_noalloc serves them with a fixed scratch array in
the library.  This file is collected last on purpose.  Each case calls the
new entry point twice in a row through the C ABI and compares each result
with muffin_op_analysis on the same input and with the oracle's W_s
(oracle/wavelets.py), at the wavelet tolerance of the other GPU tests
(relative L2 1e-6).  The cases cover the analysis kernels specialised for
512 and 1024 px sides, J = 0 (identity bases) and J = 1 (no scratch used),
a deep transform, and a cube whose scratch need is exactly the maximum."""
import ctypes

import numpy as np
import pytest

from oracle import daubechies, wavelets
from tests.gpu_util import cuda, dev, host, rel_l2

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = 4 << 20


def scratch_need(n, L, K, J):
    return L * K * sum((n >> j) ** 2 for j in range(1, J))


def call(lib, x, u, n, L, K, J, stream):
    return lib.muffin_op_analysis_noalloc(ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(u.data_ptr()), n, L, K, J, stream)


@pytest.mark.parametrize("n,L,K,J", [(256, 6, 8, 3), (512, 4, 8, 3), (1024, 1, 8, 3),
                                     (256, 3, 8, 1), (256, 3, 4, 0), (64, 2, 8, 6),
                                     (1024, 2, 8, 2)])
def test_noalloc_analysis_matches_plan_operator_and_oracle_twice(n, L, K, J):
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    lib = pkg.library()
    assert scratch_need(n, L, K, J) <= SCRATCH_FLOATS
    rng = np.random.default_rng(2024 + n + L + K + J)
    xh = rng.standard_normal((L, n, n))
    x = dev(xh, torch)
    psf = np.zeros((L, n, n), np.float32)
    psf[:, 0, 0] = 1.0
    u_ref = torch.empty((L, K, n, n), device="cuda")
    with pkg.Plan(n, L, psf, n_wavelets=K, levels=J) as plan:
        plan.op_analysis(x, u_ref)
    ref = host(u_ref)
    orc = wavelets.Ws(host(x), daubechies.filter_bank(K), J)
    assert rel_l2(ref, orc) <= 1e-6
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for c in range(2):
        u = torch.full((L, K, n, n), float("nan"), device="cuda")
        st = call(lib, x, u, n, L, K, J, stream)
        assert st == 0, lib.muffin_last_error().decode()
        torch.cuda.synchronize()
        got = host(u)
        e_plan, e_orc = rel_l2(got, ref), rel_l2(got, orc)
        assert e_plan <= 1e-6, (c, e_plan)
        assert e_orc <= 1e-6, (c, e_orc)


def test_noalloc_rejects_oversized_overlapping_and_host_arrays():
    torch = cuda()
    import paper_1905_08468_gb300 as pkg
    lib = pkg.library()
    x = torch.empty((1,), device="cuda")
    # one band more than the largest accepted 1024^2 x 2 x 8 bases, J = 2 cube
    assert scratch_need(1024, 3, 8, 2) > SCRATCH_FLOATS
    st = call(lib, x, x, 1024, 3, 8, 2, None)
    assert st == 1 and b"scratch" in lib.muffin_last_error()
    n, L, K, J = 64, 1, 2, 2
    buf = torch.zeros(((K + 1) * n * n,), device="cuda")
    st = call(lib, buf, buf[n * n // 2:], n, L, K, J, None)
    assert st == 1 and b"overlap" in lib.muffin_last_error()
    h = np.zeros(16, np.float32)
    st = lib.muffin_op_analysis_noalloc(ctypes.c_void_p(h.ctypes.data),
                                        ctypes.c_void_p(h.ctypes.data), 4, 1, 1, 1, None)
    assert st == 1 and b"device" in lib.muffin_last_error()
