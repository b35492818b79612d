"""ccg_matvec_h_noalloc: the allocation-free A^H x.

Callers that cannot allocate device memory (their memory is owned by their
own pool allocator, or they cannot accept the device-wide synchronisation of
cudaMalloc/cudaFree) use this entry point instead of a handle.  Its result
must match the handle path's ccg_matvec(trans = 1) within the tolerance the
other operator tests use, on two calls in a row (the second call reuses the
fixed scratch array the first one filled).  This file is collected last so
that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    L = C.lib()
    L.ccg_matvec_h_noalloc.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    L.ccg_matvec_h_noalloc.restype = ctypes.c_int
    return C


def noalloc(ccg, code, A, lda, x, y, stream):
    return ccg.lib().ccg_matvec_h_noalloc(code, x.numel(), ctypes.c_void_p(A.data_ptr()), lda,
                                          ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
@pytest.mark.parametrize("n", [1, 1000, 4099])
def test_noalloc_matches_handle_path_twice(ccg, dtype, n):
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    code = ccg.C128 if dtype == np.complex128 else ccg.C64
    A, _ = W.dense_system(n, 1.0, n + 7, dtype=dtype)
    Ad = torch.from_numpy(A).cuda()
    stream = torch.cuda.current_stream()
    h = ccg.Handle(stream)
    op = h.op_dense(Ad)
    tol = 1e-12 if dtype == np.complex128 else 2e-5
    for call in range(2):                       # two calls in a row, different x
        x = torch.from_numpy(W.random_vector(n, 100 + call, dtype)).cuda()
        ref = torch.empty(n, dtype=tdt, device="cuda")
        h.matvec(op, x, ref, trans=True)
        y = torch.full((n,), complex(float("nan"), 0.0), dtype=tdt, device="cuda")
        assert noalloc(ccg, code, Ad, n, x, y, stream) == ccg.OK
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), y.cpu().numpy()
        assert np.abs(g - r).max() <= tol * max(np.abs(r).max(), 1e-300), (n, call)


def test_noalloc_rejects_oversize(ccg):
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    L = ccg.lib()
    big = 65536 + 1
    st = L.ccg_matvec_h_noalloc(ccg.C128, big, ctypes.c_void_p(x.data_ptr()), big, ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == ccg.ERR_INVALID
    assert b"maximum" in L.ccg_last_error()
