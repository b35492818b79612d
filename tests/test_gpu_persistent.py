"""The persistent solve (one cooperative launch per solve, grid barriers in
place of kernel boundaries) against the kernel-per-step loop and the
oracle, through the C ABI; and its bounded barrier wait.

The two paths run the same phase and sweep code, and the persistent launch
reduces each vector phase over the same virtual blocks as the phase
kernels, so the results are bitwise equal (both precisions), and both match
the oracle's iterates (1e-9, the tolerance of the other parity tests).
"""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

METHODS = [("bicgstab", False), ("cgnr", False), ("qmr", False), ("cocg", True)]


@pytest.fixture(scope="module")
def ccg():
    from paper_1208_4869_gb300 import build as B
    B.build()
    from paper_1208_4869_gb300 import ccg as C
    return C


def system(n, shift, seed, symmetric, dtype=np.complex128):
    A, y = W.dense_system(n, shift, seed)
    if symmetric:
        A = (A + A.T) / 2
    return A.astype(dtype), y.astype(dtype)


def solve_both(ccg, method, A, y, sym, tol, maxit):
    out = []
    for persistent in (1, 0):
        h = ccg.Handle()
        h.set_option(ccg.OPT_PERSISTENT, persistent)
        Ad = torch.from_numpy(A).cuda()
        op = h.op_dense(Ad, symmetric=sym)
        xd = torch.zeros(A.shape[0], dtype=Ad.dtype, device="cuda")
        launches = h.launch_count()
        st, info, hist = h.solve(method, op, torch.from_numpy(y).cuda(), xd, tol=tol, maxit=maxit)
        out.append((st, info, hist, xd.cpu().numpy(), h.launch_count() - launches))
    return out


@pytest.mark.parametrize("method,sym", METHODS)
@pytest.mark.parametrize("n", [1, 7, 255, 1000, 4099])
def test_persistent_matches_kernel_loop_fp64(ccg, method, sym, n):
    A, y = system(n, 3.0, n + 3, sym)
    (s1, i1, h1, x1, l1), (s0, i0, h0, x0, l0) = solve_both(ccg, method, A, y, sym, 1e-10, 300)
    assert s1 == s0 == 0 and i1["iters"] == i0["iters"]
    assert np.array_equal(x1, x0) and np.array_equal(h1, h0)
    assert i1["true_relres"] <= 1e-10
    # the whole iteration is one launch (plus the true residual's kernels and,
    # in complex128, the operator's digit copy on its first product)
    assert l1 <= 5 < l0


@pytest.mark.parametrize("method,sym", METHODS)
def test_persistent_iterates_match_oracle(ccg, method, sym):
    A, y = system(300, 3.0, 5, sym)
    h = ccg.Handle()
    h.set_option(ccg.OPT_PERSISTENT, 1)
    op = h.op_dense(torch.from_numpy(A).cuda(), symmetric=sym)
    oop = O.DenseOp(A, symmetric=sym)
    for k in (1, 2, 5, 9):
        xd = torch.zeros(300, dtype=torch.complex128, device="cuda")
        st, info, hist = h.solve(method, op, torch.from_numpy(y).cuda(), xd, tol=0.0, maxit=k)
        ref = O.solve(oop, method, y, tol=0.0, maxit=k)
        assert info["iters"] == ref.iters == k
        x = xd.cpu().numpy()
        assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x), (method, k)


@pytest.mark.parametrize("method,sym", METHODS)
@pytest.mark.parametrize("n", [255, 4098])
def test_persistent_fp32(ccg, method, sym, n):
    A, y = system(n, 3.0, n, sym, np.complex64)
    (s1, i1, _, x1, _), (s0, i0, _, x0, _) = solve_both(ccg, method, A, y, sym, 1e-6, 300)
    assert s1 == s0 == 0 and i1["iters"] == i0["iters"] and np.array_equal(x1, x0)
    A64, y64 = A.astype(np.complex128), y.astype(np.complex128)
    assert np.linalg.norm(y64 - A64 @ x1.astype(np.complex128)) / np.linalg.norm(y64) < 3e-6


def test_persistent_start_vector_and_edge_cases(ccg):
    n = 300
    A, y = system(n, 3.0, 9, False)
    h = ccg.Handle()
    h.set_option(ccg.OPT_PERSISTENT, 1)
    op = h.op_dense(torch.from_numpy(A).cuda())
    # nonzero start vector: the product A x0 is formed
    x0 = W.random_vector(n, 4)
    xd = torch.from_numpy(x0.copy()).cuda()
    st, info, _ = h.solve("bicgstab", op, torch.from_numpy(y).cuda(), xd, tol=1e-10, maxit=300)
    ref = O.solve(O.DenseOp(A), "bicgstab", y, x0=x0, tol=1e-10, maxit=300)
    assert st == 0 and info["iters"] == ref.iters
    assert np.linalg.norm(xd.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    # y = 0, maxit = 0, the solution as the start vector
    for m in ("bicgstab", "cgnr", "qmr"):
        xd = torch.from_numpy(W.random_vector(n, 1)).cuda()
        st, info, _ = h.solve(m, op, torch.zeros(n, dtype=torch.complex128, device="cuda"), xd, 1e-10, 50)
        assert st == 0 and info["iters"] == 0 and torch.count_nonzero(xd).item() == 0
        xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
        st, info, _ = h.solve(m, op, torch.from_numpy(y).cuda(), xd, 1e-10, 0)
        assert st == ccg.NOT_CONVERGED and info["iters"] == 0
        xd = torch.from_numpy(np.linalg.solve(A, y)).cuda()
        st, info, _ = h.solve(m, op, torch.from_numpy(y).cuda(), xd, 1e-10, 10)
        assert st == 0 and info["iters"] == 0


def test_persistent_barrier_wait_runs_out(ccg):
    """A block that never arrives makes the others' bounded waits expire:
    the solve returns CCG_ERR_TIMEOUT, and the same handle then solves
    correctly (the device stays usable)."""
    n = 2048
    A, y = system(n, 3.0, 11, False)
    h = ccg.Handle()
    h.set_option(ccg.OPT_PERSISTENT, 1)
    op = h.op_dense(torch.from_numpy(A).cuda())
    yd = torch.from_numpy(y).cuda()
    h.set_option(ccg.OPT_WAIT_LIMIT, 64)           # 64 Ki cycles, ~30 us
    h.set_option(ccg.OPT_TEST_WITHHOLD, 1)
    for m in ("bicgstab", "cgnr", "qmr"):
        xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
        with pytest.raises(ccg.CcgError) as e:
            h.solve(m, op, yd, xd, tol=1e-10, maxit=100)
        assert e.value.status == ccg.ERR_TIMEOUT
    h.set_option(ccg.OPT_TEST_WITHHOLD, 0)
    h.set_option(ccg.OPT_WAIT_LIMIT, 0)
    xd = torch.zeros(n, dtype=torch.complex128, device="cuda")
    st, info, _ = h.solve("bicgstab", op, yd, xd, tol=1e-10, maxit=100)
    ref = O.solve(O.DenseOp(A), "bicgstab", y, tol=1e-10, maxit=100)
    assert st == 0 and info["iters"] == ref.iters
    assert np.linalg.norm(xd.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("prec", ["complex128", "complex64"])
def test_programmatic_dependent_launch_same_results(ccg, prec):
    """The kernel-per-step loop with and without programmatic dependent
    launch: the same kernels in the same order, so bitwise the same solves."""
    dt = np.complex128 if prec == "complex128" else np.complex64
    A, y = system(1500, 3.0, 13, False, dt)
    outs = []
    for pdl in (1, 0):
        h = ccg.Handle()
        h.set_option(ccg.OPT_PERSISTENT, 0)
        h.set_option(ccg.OPT_PDL, pdl)
        op = h.op_dense(torch.from_numpy(A).cuda())
        for m in ("bicgstab", "cgnr", "qmr"):
            xd = torch.zeros(1500, dtype=getattr(torch, prec), device="cuda")
            st, info, hist = h.solve(m, op, torch.from_numpy(y).cuda(), xd, tol=1e-10 if dt == np.complex128 else 1e-6,
                                     maxit=300)
            outs.append((m, pdl, xd.cpu().numpy(), hist))
    for (m1, _, x1, h1), (m0, _, x0, h0) in zip(outs[:3], outs[3:]):
        assert m1 == m0 and np.array_equal(x1, x0) and np.array_equal(h1, h0), m1


@pytest.mark.parametrize("L,prec", [(32, "complex64"), (12, "complex128"), (64, "complex64")])
def test_programmatic_dependent_launch_dipole(ccg, L, prec):
    """Dipole solves (the fused three-kernel application at L = 32 and 64 in
    complex64, the five-pass one in complex128) with and without
    programmatic dependent launch: bitwise the same."""
    occ = W.sphere_occupancy(L)
    y = W.plane_wave_rhs(occ, W.DIPOLE_CFG["kd"]).astype(np.complex128 if prec == "complex128" else np.complex64)
    outs = []
    for pdl in (1, 0):
        h = ccg.Handle()
        h.set_option(ccg.OPT_PDL, pdl)
        op = h.op_dipole(occ, W.DIPOLE_CFG["kd"], W.DIPOLE_CFG["m"], dtype=prec)
        for m in ("cocg", "bicgstab"):
            xd = torch.zeros(len(y), dtype=getattr(torch, prec), device="cuda")
            st, info, hist = h.solve(m, op, torch.from_numpy(y).cuda(), xd, tol=1e-5, maxit=40)
            outs.append((m, xd.cpu().numpy(), hist))
    for (m1, x1, h1), (m0, x0, h0) in zip(outs[:2], outs[2:]):
        assert m1 == m0 and np.array_equal(x1, x0) and np.array_equal(h1, h0), m1
