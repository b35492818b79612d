"""Many dense systems of uneven sizes in one persistent launch
(ccg_solve_multi, ccg_solve_multi_refined) through the C ABI.

Each system of a batch must give bitwise the result of its own solve on the
kernel-per-step loop (the launch runs the same sweeps and fused updates and
reduces them in the same order, whatever the size of the system's block
group), and match the oracle (iterates to 1e-9 relative, equal iteration
counts in complex128).  Refined batches give each system bitwise the
result of its own ccg_solve_refined.
"""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [1, 64, 300, 513, 1000, 2048, 97, 4096]
# complex64 systems of one launch share a load width (16-byte pairs only when
# every system allows them), so the bitwise comparison with single solves
# takes sizes of one parity
SIZES_EVEN = [2, 64, 300, 514, 1000, 2048, 98, 4096]


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


def systems(sizes, sym=False, dtype=np.complex128, seed=0):
    out = []
    for i, n in enumerate(sizes):
        A, y = W.dense_system(n, 3.0, seed + 31 * i + n)
        if sym:
            A = (A + A.T) / 2
        out.append((A.astype(dtype), y.astype(dtype)))
    return out


def single(ccg, method, A, y, sym, tol, maxit, dtype):
    h = ccg.Handle()
    h.set_option(ccg.OPT_PERSISTENT, 0)
    op = h.op_dense(torch.from_numpy(A).cuda(), symmetric=sym)
    xd = torch.zeros(A.shape[0], dtype=dtype, device="cuda")
    st, info, _ = h.solve(method, op, torch.from_numpy(y).cuda(), xd, tol=tol, maxit=maxit)
    return st, info, xd.cpu().numpy()


@pytest.mark.parametrize("method,sym", [("bicgstab", False), ("cgnr", False), ("qmr", False), ("cocg", True)])
@pytest.mark.parametrize("prec", ["complex128", "complex64"])
def test_multi_equals_single_solves(ccg, method, sym, prec):
    dt = np.complex128 if prec == "complex128" else np.complex64
    tdt = getattr(torch, prec)
    tol = 1e-10 if prec == "complex128" else 1e-6
    sizes = SIZES if prec == "complex128" else SIZES_EVEN
    sys_ = systems(sizes, sym, dt)
    h = ccg.Handle()
    Ads = [torch.from_numpy(A).cuda() for A, _ in sys_]
    ops = [h.op_dense(Ad, symmetric=sym) for Ad in Ads]
    ys = [torch.from_numpy(y).cuda() for _, y in sys_]
    xs = [torch.zeros(len(y), dtype=tdt, device="cuda") for _, y in sys_]
    st, iters, sts, rr = h.solve_multi(method, ops, ys, xs, tol=tol, maxit=400)
    assert st == 0 and np.all(sts == 0)
    for k, (A, y) in enumerate(sys_):
        s1, info, x1 = single(ccg, method, A, y, sym, tol, 400, tdt)
        assert s1 == 0 and iters[k] == info["iters"], (k, iters[k], info["iters"])
        assert np.array_equal(xs[k].cpu().numpy(), x1), (method, prec, sizes[k])
        assert rr[k] <= (1e-10 if prec == "complex128" else 3e-6)
        assert abs(rr[k] - info["true_relres"]) <= 1e-6 * max(rr[k], 1e-30) + 1e-15
        if prec == "complex128":
            ref = O.solve(O.DenseOp(A, symmetric=sym), method, y, tol=tol, maxit=400)
            assert ref.iters == iters[k]
            assert np.linalg.norm(xs[k].cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_multi_shared_operator_and_start_vectors(ccg):
    """Several right-hand sides of one matrix (the same operator in every
    slot), one with a nonzero start vector, one zero right-hand side."""
    n = 700
    A, _ = W.dense_system(n, 3.0, 2)
    h = ccg.Handle()
    op = h.op_dense(torch.from_numpy(A).cuda())
    Y = [W.random_vector(n, s) for s in range(5)]
    Y[3] = np.zeros(n, dtype=np.complex128)
    x0 = W.random_vector(n, 99)
    xs = [torch.zeros(n, dtype=torch.complex128, device="cuda") for _ in Y]
    xs[1] = torch.from_numpy(x0.copy()).cuda()
    st, iters, sts, rr = h.solve_multi("bicgstab", [op] * 5, [torch.from_numpy(y).cuda() for y in Y], xs,
                                       tol=1e-10, maxit=300)
    assert st == 0 and np.all(sts == 0)
    assert iters[3] == 0 and torch.count_nonzero(xs[3]).item() == 0
    for k, y in enumerate(Y):
        if k == 3:
            continue
        ref = O.solve(O.DenseOp(A), "bicgstab", y, x0=x0 if k == 1 else None, tol=1e-10, maxit=300)
        assert iters[k] == ref.iters
        assert np.linalg.norm(xs[k].cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def test_multi_refined_equals_single(ccg):
    sizes = [128, 1000, 2048, 514, 300]
    sys_ = systems(sizes, seed=7)
    h = ccg.Handle()
    keep = []
    ops64, ops32 = [], []
    for A, _ in sys_:
        Ad = torch.from_numpy(A).cuda()
        A32 = Ad.to(torch.complex64)
        keep += [Ad, A32]
        ops64.append(h.op_dense(Ad))
        ops32.append(h.op_dense(A32))
    tols = [1e-10, 1e-6, 1e-10, 1e-8, 1e-10]
    ys = [torch.from_numpy(y).cuda() for _, y in sys_]
    xs = [torch.zeros(len(y), dtype=torch.complex128, device="cuda") for _, y in sys_]
    st, outer, inner, sts, rr = h.solve_multi_refined("bicgstab", ops64, ops32, ys, xs, tol=tols, max_outer=30,
                                                      inner_tol=1e-5, inner_maxit=200)
    assert st == 0 and np.all(sts == 0)
    for k, (A, y) in enumerate(sys_):
        assert rr[k] <= tols[k]
        h1 = ccg.Handle()
        h1.set_option(ccg.OPT_PERSISTENT, 0)
        o64 = h1.op_dense(keep[2 * k])
        o32 = h1.op_dense(keep[2 * k + 1])
        xd = torch.zeros(len(y), dtype=torch.complex128, device="cuda")
        s1, info, _, inn = h1.solve_refined("bicgstab", o64, o32, ys[k], xd, tol=tols[k], max_outer=30,
                                            inner_tol=1e-5, inner_maxit=200)
        assert s1 == 0 and info["iters"] == outer[k] and inn == inner[k]
        assert np.array_equal(xd.cpu().numpy(), xs[k].cpu().numpy()), sizes[k]
        ref = O.solve(O.DenseOp(A), "bicgstab", y, tol=1e-12, maxit=300)
        assert np.linalg.norm(xs[k].cpu().numpy() - ref.x) <= max(10 * tols[k], 1e-9) * np.linalg.norm(ref.x)


def test_multi_limits(ccg):
    h = ccg.Handle()
    A, y = W.dense_system(16, 3.0, 1)
    op = h.op_dense(torch.from_numpy(A).cuda())
    yd = torch.from_numpy(y).cuda()
    # as many systems as the launch has blocks: every group is one block
    cap = 0
    for c in (456, 304, 152):
        try:
            xs = [torch.zeros(16, dtype=torch.complex128, device="cuda") for _ in range(c)]
            st, iters, sts, rr = h.solve_multi("qmr", [op] * c, [yd] * c, xs, tol=1e-12, maxit=100)
            cap = c
            break
        except ccg.CcgError as e:
            assert e.status == ccg.ERR_INVALID and "count" in str(e)
    assert cap > 0 and np.all(sts == 0)
    assert len({tuple(x.cpu().numpy()) for x in xs}) == 1
    with pytest.raises(ccg.CcgError) as e:
        h.solve_multi("qmr", [op] * 5000, [yd] * 5000,
                      [torch.zeros(16, dtype=torch.complex128, device="cuda")] * 5000, tol=1e-12, maxit=10)
    assert e.value.status == ccg.ERR_INVALID
    with pytest.raises(ccg.CcgError) as e:
        h.solve_multi("gmres", [op], [yd], [torch.zeros_like(yd)], tol=1e-12, maxit=10)
    assert e.value.status == ccg.ERR_UNSUPPORTED


def test_multi_barrier_wait_runs_out(ccg):
    """A withheld block makes its group's barrier waits expire; the call
    returns CCG_ERR_TIMEOUT and the handle then solves the batch."""
    sys_ = systems([300, 1000, 2048], seed=3)
    h = ccg.Handle()
    ops = [h.op_dense(torch.from_numpy(A).cuda()) for A, _ in sys_]
    ys = [torch.from_numpy(y).cuda() for _, y in sys_]
    h.set_option(ccg.OPT_WAIT_LIMIT, 64)
    h.set_option(ccg.OPT_TEST_WITHHOLD, 1)
    xs = [torch.zeros(len(y), dtype=torch.complex128, device="cuda") for _, y in sys_]
    with pytest.raises(ccg.CcgError) as e:
        h.solve_multi("bicgstab", ops, ys, xs, tol=1e-10, maxit=100)
    assert e.value.status == ccg.ERR_TIMEOUT
    h.set_option(ccg.OPT_TEST_WITHHOLD, 0)
    h.set_option(ccg.OPT_WAIT_LIMIT, 0)
    xs = [torch.zeros(len(y), dtype=torch.complex128, device="cuda") for _, y in sys_]
    st, iters, sts, rr = h.solve_multi("bicgstab", ops, ys, xs, tol=1e-10, maxit=100)
    assert st == 0 and np.all(rr <= 1e-10)
