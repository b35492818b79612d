"""Pins of the CPU oracle's discrete-dipole operator (the DDSCAT application of
the manual's Sec. 1) and of its FFT (no GPU).

The manual does not define the operator, so each pin comes from physics or
an independent route:
  * G(r) equals the field of a dipole derived symbolically by sympy as
    k^2 G0 I + Hessian(G0), G0 = exp(ikr)/r (Jackson, curl curl of p G0);
  * the static limit of the whole system reproduces the closed-form
    polarizability of a dielectric sphere, a^3 (m^2 - 1)/(m^2 + 2);
  * the FFT convolution equals the direct sum; the oracle FFT equals numpy's;
  * one dipole gives P = alpha E; two dipoles solve a 2x2-by-symmetry system;
  * A = A^T; A^H x = conj(A) x against an explicitly assembled matrix.
"""
import numpy as np
import pytest
import sympy as sp

import oracle as O
from paper_1208_4869_gb300 import workloads as W

M_CFG = 1.5 + 0.01j


def sympy_green():
    x, y, z, k = sp.symbols("x y z k", real=True)
    r = sp.sqrt(x ** 2 + y ** 2 + z ** 2)
    G0 = sp.exp(sp.I * k * r) / r
    X = [x, y, z]
    comps = [[k ** 2 * G0 * (1 if a == b else 0) + sp.diff(G0, X[a], X[b]) for b in range(3)] for a in range(3)]
    return sp.lambdify((k, x, y, z), sp.Matrix(comps), "numpy")


@pytest.fixture(scope="module")
def green_ref():
    return sympy_green()


@pytest.mark.parametrize("kd", [0.0, 0.5, 1.3])
@pytest.mark.parametrize("r", [(1, 0, 0), (0, 0, 1), (1, 2, -3), (-4, 1, 1), (5, -5, 2)])
def test_green_tensor_matches_symbolic_dipole_field(green_ref, kd, r):
    ref = np.array(green_ref(kd, *[float(v) for v in r]), dtype=np.complex128)
    got = O.green(kd, r)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.allclose(got, got.T, rtol=0, atol=0)
    assert np.allclose(O.green(kd, [-v for v in r]), got, rtol=1e-15, atol=0)


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 12, 10), (48, 4, 3), (5, 7, 9), (1, 1, 16)])
def test_oracle_fft_matches_numpy(shape):
    g = W.complex_normal(np.random.default_rng(3), shape)
    assert np.abs(O.fft3d(g, -1) - np.fft.fftn(g)).max() < 1e-12 * g.size
    assert np.abs(O.fft3d(g, +1) - np.fft.ifftn(g) * g.size).max() < 1e-12 * g.size


def sphere_or_box(kind, L):
    if kind == "sphere":
        return W.sphere_occupancy(L)
    rng = np.random.default_rng(L)
    occ = (rng.random((L, L + 1, L - 1)) < 0.6).astype(np.uint8)   # ragged, non-cubic, holes
    return occ


@pytest.mark.parametrize("kind,L", [("sphere", 4), ("sphere", 7), ("sphere", 10), ("box", 5), ("box", 6)])
def test_fft_convolution_equals_direct_sum(kind, L):
    occ = sphere_or_box(kind, L)
    d = O.DipoleOp(occ, 0.5, M_CFG)
    f = O.DipoleOp(occ, 0.5, M_CFG, use_fft=True)
    x = W.random_vector(d.n, 5)
    a, b = d.matvec(x), f.matvec(x)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def assemble(op):
    n = op.n
    A = np.empty((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1
        A[:, j] = op.matvec(e)
    return A


def test_dipole_matrix_symmetric_and_adjoint():
    op = O.DipoleOp(W.sphere_occupancy(4), 0.5, M_CFG)
    A = assemble(op)
    assert np.abs(A - A.T).max() < 1e-15 * np.abs(A).max()
    x = W.random_vector(op.n, 9)
    assert np.abs(op.matvec(x, trans=True) - A.conj().T @ x).max() < 1e-13 * np.abs(A).max()
    u = W.random_vector(op.n, 10)
    assert abs(u @ op.matvec(x) - x @ op.matvec(u)) < 1e-12 * np.abs(A).max()
    # diagonal blocks are 1/alpha I (no self term)
    N = op.nsites
    for s in range(N):
        blk = A[[s, N + s, 2 * N + s]][:, [s, N + s, 2 * N + s]]
        assert np.allclose(blk, np.eye(3) / op.alpha, rtol=1e-14, atol=0)


def test_single_dipole_polarization():
    occ = np.zeros((3, 3, 3), np.uint8)
    occ[1, 1, 1] = 1
    op = O.DipoleOp(occ, 0.5, M_CFG)
    E = np.array([1.0, 0.3j, -0.2], dtype=np.complex128)
    r = O.solve(op, "cocg", E, tol=1e-14, maxit=5)
    assert np.allclose(r.x, op.alpha * E, rtol=1e-14, atol=0)


def test_two_dipoles_along_z(green_ref):
    """Two sites one spacing apart along z, x-polarised field: by symmetry
    P_1 = P_2 = P x^ with P (1/alpha - G_xx(d)) = 1."""
    kd = 0.5
    occ = np.zeros((1, 1, 2), np.uint8)
    occ[0, 0, :] = 1
    op = O.DipoleOp(occ, kd, M_CFG)
    y = np.zeros(6, dtype=np.complex128)
    y[:2] = 1.0
    r = O.solve(op, "bicgstab", y, tol=1e-14, maxit=20)
    Gxx = complex(np.array(green_ref(kd, 0.0, 0.0, 1.0), dtype=np.complex128)[0, 0])
    P = 1.0 / (1.0 / op.alpha - Gxx)
    assert np.allclose(r.x[:2], P, rtol=1e-12, atol=0)
    assert np.abs(r.x[2:]).max() < 1e-13


def test_static_limit_sphere_polarizability():
    """k -> 0 with a uniform field: the lattice of Clausius-Mossotti dipoles
    in a sphere of volume N (unit spacing) has total dipole close to that of
    a dielectric sphere, a^3 (m^2 - 1)/(m^2 + 2) with a^3 = 3N/(4 pi).
    A sign slip in G or in the polarizability moves this by far more than
    the 1.5% allowed for lattice discretisation."""
    occ = W.sphere_occupancy(8)
    op = O.DipoleOp(occ, 1e-5, M_CFG, use_fft=True)
    N = op.nsites
    y = np.zeros(3 * N, complex)
    y[:N] = 1.0
    r = O.solve(op, "cocg", y, tol=1e-12, maxit=500)
    assert r.status == O.OK
    P = r.x[:N].sum()
    exact = 3 * N / (4 * np.pi) * (M_CFG ** 2 - 1) / (M_CFG ** 2 + 2)
    assert abs(P - exact) / abs(exact) < 0.015
    # by the sphere's mirror symmetry the y and z components cancel in the sum
    assert abs(r.x[N:2 * N].sum()) < 1e-8 * abs(P) and abs(r.x[2 * N:].sum()) < 1e-8 * abs(P)


def test_direct_rows_subset():
    occ = W.sphere_occupancy(6)
    op = O.DipoleOp(occ, 0.5, M_CFG)
    x = W.random_vector(op.n, 2)
    full = op.matvec(x).reshape(3, op.nsites)
    sel = np.array([0, 5, 17, op.nsites - 1])
    assert np.allclose(op.rows(x, sel), full[:, sel], rtol=1e-14, atol=1e-14)


def test_lattice_site_counts_and_order():
    assert W.sphere_occupancy(64).sum() == 137376
    assert W.sphere_occupancy(16).sum() == 2176
    occ = W.sphere_occupancy(6)
    op = O.DipoleOp(occ, 0.5, M_CFG)
    assert np.array_equal(op.sites(), W.occupied_sites(occ))


@pytest.mark.parametrize("method", ["cocg", "bicgstab", "qmr", "cgnr"])
def test_dipole_solvers_converge_to_lapack(method):
    occ = W.sphere_occupancy(4)
    op = O.DipoleOp(occ, 0.5, M_CFG)
    A = assemble(op)
    y = W.plane_wave_rhs(occ, 0.5)
    xs = np.linalg.solve(A, y)
    r = O.solve(op, method, y, tol=1e-12, maxit=500)
    assert r.status == O.OK
    assert np.linalg.norm(r.x - xs) / np.linalg.norm(xs) < 1e-10
