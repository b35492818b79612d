"""Pins of the oracle's mixed-precision refinement: single-precision inner
Krylov solves inside a double-precision residual/update loop (no GPU).
Pinned by LAPACK solutions and by the double-precision residual."""
import numpy as np
import pytest

import oracle as O
from paper_1208_4869_gb300 import workloads as W


@pytest.mark.parametrize("method", ["bicgstab", "qmr", "cgnr"])
def test_refine_dense_reaches_fp64_accuracy(method):
    n = 128
    A, y = W.dense_system(n, 3.0, 13)
    xs = np.linalg.solve(A, y)
    op64 = O.DenseOp(A)
    op32 = O.DenseOp(A.astype(np.complex64))
    x, outer, st, inner, hist = O.refine(op64, op32, method, y, tol=1e-10, max_outer=30, inner_tol=1e-4,
                                         inner_maxit=50)
    assert st == O.OK
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(y - A @ x) / np.linalg.norm(y) <= 1e-10
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    # each outer step gains at least ~3 digits at inner_tol 1e-4
    assert outer <= 5
    assert np.all(np.diff(hist) < 0)


def test_refine_dipole_cocg():
    occ = W.sphere_occupancy(6)
    op = O.DipoleOp(occ, 0.5, 1.5 + 0.01j)
    y = W.plane_wave_rhs(occ, 0.5)
    x, outer, st, inner, hist = O.refine(op, O.view(op, np.complex64), "cocg", y, tol=1e-8, max_outer=20,
                                         inner_tol=1e-4, inner_maxit=200)
    assert st == O.OK and hist[-1] <= 1e-8
    ref = O.solve(op, "cocg", y, tol=1e-12, maxit=500)
    assert np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x) < 1e-7


def test_refine_zero_rhs_and_already_converged():
    A, y = W.dense_system(16, 3.0, 1)
    op64, op32 = O.DenseOp(A), O.DenseOp(A.astype(np.complex64))
    x, outer, st, inner, hist = O.refine(op64, op32, "bicgstab", np.zeros(16, complex), tol=1e-10)
    assert st == O.OK and outer == 0 and np.all(x == 0)
    xs = np.linalg.solve(A, y)
    x, outer, st, inner, hist = O.refine(op64, op32, "bicgstab", y, x0=xs, tol=1e-10)
    assert st == O.OK and outer == 0 and inner == 0
