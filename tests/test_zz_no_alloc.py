"""ccg_matvec_h_noalloc: the allocation-free A^H x.

Callers that cannot allocate device memory (their memory is owned by their
own pool allocator, or they cannot accept the device-wide synchronisation of
cudaMalloc/cudaFree) use this entry point instead of a handle.  Its result
must match the handle path's ccg_matvec(trans = 1) within the tolerance the
other operator tests use, on two calls in a row (the second call reuses the
fixed scratch array the first one filled), and the oracle's A^H x.  Padded
matrices (lda > n) check the row stride, and for complex64 both load widths
(an odd lda forces single-element loads).  This file is collected last so
that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MAX_N = 65536   # CCG_NOALLOC_MAX_N


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


def noalloc(ccg, code, n, Aptr, lda, xptr, yptr, stream):
    return ccg.lib().ccg_matvec_h_noalloc(code, n, ctypes.c_void_p(Aptr), lda, ctypes.c_void_p(xptr),
                                          ctypes.c_void_p(yptr), ctypes.c_void_p(stream.cuda_stream))


def padded(A, pad):
    """A as the leading n x n block of an n x (n + pad) device buffer (the
    padding holds NaN, which must never be read)."""
    n = A.shape[0]
    buf = torch.full((n, n + pad), complex(float("nan"), float("nan")),
                     dtype=torch.complex128 if A.dtype == np.complex128 else torch.complex64, device="cuda")
    buf[:, :n] = torch.from_numpy(A).cuda()
    return buf


def check_twice(ccg, dtype, A, pad):
    n = A.shape[0]
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    code = ccg.C128 if dtype == np.complex128 else ccg.C64
    buf = padded(A, pad)
    lda = n + pad
    stream = torch.cuda.current_stream()
    h = ccg.Handle(stream)
    op = h.op_dense(buf[:, :n])           # leading dimension n + pad
    oop = O.DenseOp(A)
    tol = 1e-12 if dtype == np.complex128 else 2e-5
    for call in range(2):                       # two calls in a row, different x
        xh = W.random_vector(n, 100 + call, dtype)
        x = torch.from_numpy(xh).cuda()
        ref = torch.empty(n, dtype=tdt, device="cuda")
        h.matvec(op, x, ref, trans=True)
        y = torch.full((n,), complex(float("nan"), 0.0), dtype=tdt, device="cuda")
        assert noalloc(ccg, code, n, buf.data_ptr(), lda, x.data_ptr(), y.data_ptr(), stream) == ccg.OK
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), y.cpu().numpy()
        assert np.abs(g - r).max() <= tol * max(np.abs(r).max(), 1e-300), (n, pad, call)
        o = oop.matvec(xh, trans=True)
        assert np.abs(g - o).max() <= tol * max(np.abs(o).max(), 1e-300), (n, pad, call)


@pytest.mark.parametrize("dtype", [np.complex128, np.complex64])
@pytest.mark.parametrize("n", [1, 1000, 4099])
def test_noalloc_matches_handle_path_and_oracle_twice(ccg, dtype, n):
    A, _ = W.dense_system(n, 1.0, n + 7, dtype=dtype)
    check_twice(ccg, dtype, A, 0)


@pytest.mark.parametrize("dtype,pad", [(np.complex128, 3), (np.complex64, 2), (np.complex64, 3)])
@pytest.mark.parametrize("n", [257, 1000])
def test_noalloc_padded_rows(ccg, dtype, pad, n):
    A, _ = W.dense_system(n, 1.0, n + 11, dtype=dtype)
    check_twice(ccg, dtype, A, pad)


@pytest.mark.parametrize("dtype,n", [(np.complex64, MAX_N), (np.complex128, 46341)])
def test_noalloc_largest_sizes(ccg, dtype, n):
    """The size cap (complex64, 34 GB) and a ragged complex128 size of the
    same bytes: full result against the handle path, sampled columns against
    a plain double-precision sum on the host."""
    tdt = torch.complex128 if dtype == np.complex128 else torch.complex64
    code = ccg.C128 if dtype == np.complex128 else ccg.C64
    g = torch.Generator(device="cuda")
    g.manual_seed(n)
    Ad = torch.randn((n, n), dtype=tdt, device="cuda", generator=g)
    stream = torch.cuda.current_stream()
    h = ccg.Handle(stream)
    op = h.op_dense(Ad)
    cols = np.random.default_rng(1).choice(n, 24, replace=False)
    cols[0], cols[1] = 0, n - 1
    Acols = Ad[:, torch.from_numpy(cols).cuda()].cpu().numpy().astype(np.complex128)
    tol = 1e-12 if dtype == np.complex128 else 2e-5
    for call in range(2):
        xh = W.random_vector(n, 300 + call, dtype)
        x = torch.from_numpy(xh).cuda()
        ref = torch.empty(n, dtype=tdt, device="cuda")
        h.matvec(op, x, ref, trans=True)
        y = torch.full((n,), complex(float("nan"), 0.0), dtype=tdt, device="cuda")
        assert noalloc(ccg, code, n, Ad.data_ptr(), n, x.data_ptr(), y.data_ptr(), stream) == ccg.OK
        torch.cuda.synchronize()
        r, gy = ref.cpu().numpy(), y.cpu().numpy()
        assert np.abs(gy - r).max() <= tol * np.abs(r).max()
        exact = np.conj(Acols).T @ xh.astype(np.complex128)
        scale = np.abs(Acols).T @ np.abs(xh.astype(np.complex128))
        assert np.all(np.abs(gy[cols] - exact) <= 4 * tol * scale * (1 if dtype == np.complex128 else 8))
    del op, Ad
    torch.cuda.empty_cache()


def test_noalloc_rejects_bad_arguments(ccg):
    """Every refusal returns CCG_ERR_INVALID with a message and launches
    nothing (y keeps its contents)."""
    x = torch.zeros(16, dtype=torch.complex128, device="cuda")
    y = torch.full((16,), 5.0 + 0j, dtype=torch.complex128, device="cuda")
    A = torch.zeros((16, 16), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream()
    L = ccg.lib()
    big = MAX_N + 1
    cases = [
        ((ccg.C128, big, A.data_ptr(), big, x.data_ptr(), y.data_ptr()), b"maximum"),
        ((ccg.C128, 16, A.data_ptr(), 15, x.data_ptr(), y.data_ptr()), b"lda"),
        ((ccg.C128, 16, A.data_ptr() + 8, 16, x.data_ptr(), y.data_ptr()), b"aligned"),
        ((ccg.C128, 15, A.data_ptr(), 16, x.data_ptr() + 8, y.data_ptr()), b"aligned"),
        ((7, 16, A.data_ptr(), 16, x.data_ptr(), y.data_ptr()), b"dtype"),
        ((ccg.C128, 0, A.data_ptr(), 16, x.data_ptr(), y.data_ptr()), b"n >= 1"),
        ((ccg.C128, 16, 0, 16, x.data_ptr(), y.data_ptr()), b"NULL"),
    ]
    for args, msg in cases:
        st = noalloc(ccg, *args, stream)
        assert st == ccg.ERR_INVALID, args
        assert msg in L.ccg_last_error(), (args, L.ccg_last_error())
    torch.cuda.synchronize()
    assert torch.all(y == 5.0).item()
