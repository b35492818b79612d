"""Multi-right-hand-side block products through the C ABI: the tcgen05
tensor-core path (complex64, split-bf16 operands, fp32 accumulation) and the
CUDA-core path, against the product of the same single-precision data
computed in double on the host (the manual's `matvec`, Sec. 5, applied to a
block of right-hand sides).

Tolerances (largest entry error over the largest entry): tensor cores
2e-5 up to K = 2n = 2048 and in proportion to K beyond (measured on GB300 for
both two- and three-term splits: 5e-6 at K = 512, 1.7e-5 at K = 2048,
5e-5 at K = 8192 -- their fp32 accumulation, not the operand split, sets the
error); CUDA-core complex64 sums 2e-5 up to n = 8192 (fp32 accumulation over
n terms); complex128 1e-13.
"""
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
    return C


def colmajor(a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def product(ccg, mode, A, X, terms=3):
    h = ccg.Handle()
    h.set_option(ccg.OPT_TENSOR_CORES, mode)
    h.set_option(ccg.OPT_TC_SPLIT, terms)
    op = h.op_dense(torch.from_numpy(A).cuda())
    Y = colmajor(np.zeros(X.shape, A.dtype))
    h.block_matvec(op, colmajor(X), Y)
    torch.cuda.synchronize()
    return Y.cpu().numpy()


def tc_bound(n):
    return 2e-5 * max(1.0, 2 * n / 2048)


def err(got, A, X):
    ref = A.astype(np.complex128) @ X.astype(np.complex128)
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("terms", [2, 3])
def test_tensor_core_small(ccg, terms):
    n, k = 256, 8
    A, _ = W.dense_system(n, 1.0, 1, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=2, dtype=np.complex64)
    e = err(product(ccg, 1, A, X, terms), A, X)
    assert e < tc_bound(n), e


@pytest.mark.parametrize("n,k", [(132, 1), (1000, 37), (512, 256), (4096, 130)])
def test_tensor_core_ragged(ccg, n, k):
    A, _ = W.dense_system(n, 1.0, n, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=k, dtype=np.complex64)
    tc2 = product(ccg, 1, A, X, 2)
    tc3 = product(ccg, 1, A, X, 3)
    cc = product(ccg, 0, A, X)
    assert err(tc2, A, X) < tc_bound(n)
    assert err(tc3, A, X) < tc_bound(n)
    assert err(cc, A, X) < 2e-5


def test_tensor_core_full_size(ccg):
    """n = 8192, 256 right-hand sides (the multi-right-hand-side workload)."""
    A, _ = W.dense_system(8192, 3.0, 0, dtype=np.complex64)
    X = W.dense_rhs_block(8192, 256, seed=1, dtype=np.complex64)
    ref = A.astype(np.complex128) @ X.astype(np.complex128)
    for terms in (2, 3):
        tc = product(ccg, 1, A, X, terms)
        # the relative error of every column
        col = np.linalg.norm(tc - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert col.max() < tc_bound(8192), (terms, col.max())


@pytest.mark.parametrize("n,k", [(2048, 256), (8192, 1), (4099, 200), (640, 24)])
def test_tensor_core_stream_k(ccg, n, k):
    """Shapes whose stream-K ranges cut tiles into two to four pieces (partial
    tiles of lower ranges added by the range holding the tile's last K block)
    or give one CTA several row blocks: every product within the bound, and
    two runs bitwise equal (the partial tiles are added in a fixed order)."""
    A, _ = W.dense_system(n, 1.0, n + k, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=k + 3, dtype=np.complex64)
    for terms in (2, 3):
        a = product(ccg, 1, A, X, terms)
        b = product(ccg, 1, A, X, terms)
        assert err(a, A, X) < tc_bound(n), (terms, err(a, A, X))
        assert np.array_equal(a, b)


def test_complex128_block_product(ccg):
    n, k = 300, 17
    A, _ = W.dense_system(n, 1.0, 3)
    X = W.dense_rhs_block(n, k, seed=4)
    assert err(product(ccg, 1, A, X), A, X) < 1e-13


def test_refined_same_with_and_without_tensor_cores(ccg):
    n, k = 640, 24
    A, _ = W.dense_system(n, 3.0, 0)
    Y = W.dense_rhs_block(n, k, seed=1)
    out = []
    for mode in (0, 1):
        h = ccg.Handle()
        h.set_option(ccg.OPT_TENSOR_CORES, mode)
        Ad = torch.from_numpy(A).cuda()
        op64, op32 = h.op_dense(Ad), h.op_dense(Ad.to(torch.complex64))
        X = colmajor(np.zeros((n, k), np.complex128))
        st, outer, inner, sts, rr = h.solve_batched_refined("bicgstab", op64, op32, colmajor(Y), X, tol=1e-10)
        assert st == 0 and np.all(rr <= 1e-10)
        Xh = X.cpu().numpy()
        assert np.all(np.linalg.norm(Y - A @ Xh, axis=0) / np.linalg.norm(Y, axis=0) <= 1e-10)
        out.append(Xh)
    assert np.linalg.norm(out[0] - out[1]) / np.linalg.norm(out[0]) < 1e-9


@pytest.mark.parametrize("prec", ["complex64", "complex128"])
def test_pipeline_wait_runs_out(ccg, prec):
    """The tensor-core pipelines' bounded waits: with the test hook a CTA's
    producer never issues its first stage's copies, so the MMA issuer's wait
    on that stage runs out (a short CCG_OPT_WAIT_LIMIT); the call returns
    CCG_ERR_TIMEOUT after every CTA drained its work and freed its tensor
    memory, and the next product on the same handle is correct (complex64:
    the split-bf16 pipeline; complex128: the integer-slice one)."""
    dt = np.complex64 if prec == "complex64" else np.complex128
    n, k = 512, 64
    A, _ = W.dense_system(n, 1.0, 4, dtype=dt)
    X = W.dense_rhs_block(n, k, seed=5, dtype=dt)
    h = ccg.Handle()
    op = h.op_dense(torch.from_numpy(A).cuda())
    Y = colmajor(np.zeros(X.shape, dt))
    h.block_matvec(op, colmajor(X), Y)             # the operator's tensor-core copies, made normally
    h.set_option(ccg.OPT_WAIT_LIMIT, 64)           # 64 Ki cycles, ~30 us
    h.set_option(ccg.OPT_TEST_WITHHOLD, 1)
    for _ in range(2):
        with pytest.raises(ccg.CcgError) as e:
            h.block_matvec(op, colmajor(X), Y)
        assert e.value.status == ccg.ERR_TIMEOUT
    h.set_option(ccg.OPT_TEST_WITHHOLD, 0)
    h.set_option(ccg.OPT_WAIT_LIMIT, 0)
    Y = colmajor(np.zeros(X.shape, dt))
    h.block_matvec(op, colmajor(X), Y)
    torch.cuda.synchronize()
    bound = tc_bound(n) if dt == np.complex64 else 1e-13
    assert err(Y.cpu().numpy(), A, X) <= bound


def test_stream_k_partial_wait_runs_out(ccg):
    """The split-bf16 product's stream-K flag wait: with the test hook the
    first K range keeps its partial tile unpublished, so the CTA that
    finishes that tile waits for it until the (short) limit runs out; the
    call returns CCG_ERR_TIMEOUT, and the next product on the same handle is
    correct.  n = 1000, k = 37: 8 row blocks of 63 K blocks in 15 ranges, so
    the first range ends inside row block 0."""
    n, k = 1000, 37
    A, _ = W.dense_system(n, 1.0, 6, dtype=np.complex64)
    X = W.dense_rhs_block(n, k, seed=7, dtype=np.complex64)
    h = ccg.Handle()
    op = h.op_dense(torch.from_numpy(A).cuda())
    Y = colmajor(np.zeros(X.shape, np.complex64))
    h.block_matvec(op, colmajor(X), Y)
    h.set_option(ccg.OPT_WAIT_LIMIT, 64)           # 64 Ki cycles, ~30 us
    h.set_option(ccg.OPT_TEST_WITHHOLD, 2)
    with pytest.raises(ccg.CcgError) as e:
        h.block_matvec(op, colmajor(X), Y)
    assert e.value.status == ccg.ERR_TIMEOUT
    h.set_option(ccg.OPT_TEST_WITHHOLD, 0)
    h.set_option(ccg.OPT_WAIT_LIMIT, 0)
    Y = colmajor(np.zeros(X.shape, np.complex64))
    h.block_matvec(op, colmajor(X), Y)
    torch.cuda.synchronize()
    assert err(Y.cpu().numpy(), A, X) <= tc_bound(n)
