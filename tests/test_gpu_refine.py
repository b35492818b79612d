"""GPU parity of the mixed-precision refinement (complex128 residual and
update around complex64 inner Krylov solves) against the CPU oracle's
refinement, through the C ABI.

The inner complex64 iterates differ from the oracle's by rounding order, so
parity is judged on what the method fixes: the final residual, recomputed in
complex128 (<= 1e-10), and the solution, which must agree with the oracle's
complex128 solution to within the forward error that residual allows
(cond(A) * 1e-10; the systems here have cond < 10).
"""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


@pytest.fixture(scope="module")
def h(ccg):
    return ccg.Handle()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ops(h, A, symmetric=False):
    Ad = dev(A)
    return h.op_dense(Ad, symmetric=symmetric), h.op_dense(Ad.to(torch.complex64), symmetric=symmetric), Ad


def relres(A, x, y):
    return np.linalg.norm(y - A @ x) / np.linalg.norm(y)


@pytest.mark.parametrize("method", ["bicgstab", "cgnr", "qmr", "cocg", "cocr", "bicg", "gmres", "cgs", "cgne", "tfqmr", "bicgstabl"])
@pytest.mark.parametrize("n", [256, 1000])
def test_refined_matches_oracle(h, method, n):
    A, y = W.dense_system(n, 3.0, 17)
    sym = method in ("cocg", "cocr")
    if sym:
        A = (A + A.T) / 2
    op64, op32, _keep = ops(h, A, sym)
    xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
    st, info, hist, inner = h.solve_refined(method, op64, op32, dev(y), xd, tol=1e-10, max_outer=30,
                                            inner_tol=1e-5, inner_maxit=300)
    x = xd.cpu().numpy()
    assert st == 0
    assert relres(A, x, y) <= 1e-10
    assert abs(info["relres"] - relres(A, x, y)) <= 1e-12
    assert hist[-1] <= 1e-10 and np.all(np.diff(hist) < 0)
    ox, outer, ost, oinner, ohist = O.refine(O.DenseOp(A, symmetric=sym),
                                             O.DenseOp(A.astype(np.complex64), symmetric=sym), method, y,
                                             tol=1e-10, max_outer=30, inner_tol=1e-5, inner_maxit=300)
    assert ost == 0
    assert abs(info["iters"] - outer) <= 1
    assert np.linalg.norm(x - ox) / np.linalg.norm(ox) < 1e-8
    assert 0 < inner <= 300 * info["iters"]


def test_refined_edge_cases(h, ccg):
    n = 128
    A, y = W.dense_system(n, 3.0, 5)
    op64, op32, _keep = ops(h, A)
    # y = 0: x = 0, no corrections
    xd = dev(W.random_vector(n, 1))
    st, info, hist, inner = h.solve_refined("bicgstab", op64, op32, torch.zeros_like(xd), xd)
    assert st == 0 and info["iters"] == 0 and inner == 0 and torch.count_nonzero(xd).item() == 0
    # x0 already the solution: converged before any correction
    xs = np.linalg.solve(A, y)
    xd = dev(xs)
    st, info, hist, inner = h.solve_refined("qmr", op64, op32, dev(y), xd, tol=1e-10)
    assert st == 0 and info["iters"] == 0 and inner == 0
    # no corrections allowed
    xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
    st, info, hist, inner = h.solve_refined("bicgstab", op64, op32, dev(y), xd, max_outer=0)
    assert st == ccg.NOT_CONVERGED and info["iters"] == 0
    # one correction, capped inner solve
    st, info, hist, inner = h.solve_refined("bicgstab", op64, op32, dev(y), xd, max_outer=1, inner_maxit=2)
    assert st == ccg.NOT_CONVERGED and info["iters"] == 1 and inner == 2 and len(hist) == 2
    assert hist[1] < hist[0]
    # host buffers equal device buffers
    xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
    h.solve_refined("cgnr", op64, op32, dev(y), xd)
    xh = np.zeros(n, dtype=np.complex128)
    st, info, _, _ = h.solve_refined("cgnr", op64, op32, y.copy(), xh)
    assert st == 0 and np.array_equal(xh, xd.cpu().numpy())
    # argument checks
    with pytest.raises(ccg.CcgError):
        h.solve_refined("bicgstab", op32, op64, dev(y), xd)            # precisions swapped
    with pytest.raises(ccg.CcgError):
        h.solve_refined("cocg", op64, op32, dev(y), xd)                # not flagged symmetric
