"""Seeded synthetic inputs shared by the GPU library's tests, the benchmark and
the CPU oracle's tests.

This module holds none of the solvers' arithmetic: it only draws matrices,
right-hand sides and lattice geometries.  All random draws use numpy's
PCG64 ``default_rng(seed)``, which gives the same stream on every platform.
A complex normal number is (N(0,1) + i N(0,1)) / sqrt(2): the real parts of
the whole array are drawn first, then the imaginary parts.

Workloads (the problem statement is the manual's Sec. 1, A x = y):
  * dense: A = (shift + 0.5 + 0.5i) I + G / sqrt(n), G iid complex normal
    drawn row-major as one (n, n) array, then y from the same generator;
    shift 8 for the small n=256 case, shift 3 for the n=8192 case.
  * dipole: the occupied sites of an L^3 cubic lattice inside the inscribed
    sphere |(i,j,l) - c|^2 <= (L/2)^2, c = ((L-1)/2,)*3, and the incident
    plane wave along z, x-polarised, E_s = x^ exp(i kd l_s) (phase origin at
    l = 0, unit lattice spacing), in the site-fastest layout v[a*N + s].
"""
import numpy as np

DENSE_SMALL = dict(n=256, shift=8.0, seed=0)
DENSE_LARGE = dict(n=8192, shift=3.0, seed=0)
DIPOLE_CFG = dict(L=64, kd=0.5, m=1.5 + 0.01j)


def complex_normal(rng, shape, dtype=np.complex128):
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    out = np.empty(shape, dtype=dtype)
    out.real = re
    out.imag = im
    out *= 1.0 / np.sqrt(2.0)
    return out


def dense_system(n, shift=8.0, seed=0, dtype=np.complex128):
    """(A, y): A row-major (n, n); y an n-vector, both from default_rng(seed)."""
    rng = np.random.default_rng(seed)
    A = complex_normal(rng, (n, n), np.complex128)
    A *= 1.0 / np.sqrt(n)
    A[np.diag_indices(n)] += complex(shift + 0.5, 0.5)
    y = complex_normal(rng, (n,), np.complex128)
    if dtype != np.complex128:
        return A.astype(dtype), y.astype(dtype)
    return A, y


def dense_rhs_block(n, k, seed=1, dtype=np.complex128):
    """k right-hand sides as an (n, k) column-major block (column j contiguous)."""
    rng = np.random.default_rng(seed)
    Y = complex_normal(rng, (k, n), np.complex128)   # row j of this array is column j of the block
    return np.asfortranarray(Y.T).astype(dtype, copy=False)


def sphere_occupancy(L):
    """uint8 (L, L, L) mask of lattice sites inside the inscribed sphere."""
    c = (L - 1) / 2.0
    i = np.arange(L, dtype=np.float64) - c
    d2 = i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2
    return (d2 <= (L / 2.0) ** 2).astype(np.uint8)


def occupied_sites(occ):
    """(N, 3) int32 coordinates of occupied sites, lexicographic, last axis fastest."""
    return np.argwhere(occ != 0).astype(np.int32)


def plane_wave_rhs(occ, kd, dtype=np.complex128):
    """Incident field x^ exp(i kd z) at the occupied sites, layout v[a*N + s]."""
    sites = occupied_sites(occ)
    N = len(sites)
    y = np.zeros(3 * N, dtype=np.complex128)
    y[:N] = np.exp(1j * kd * sites[:, 2].astype(np.float64))
    return y.astype(dtype, copy=False)


def random_vector(n, seed, dtype=np.complex128):
    return complex_normal(np.random.default_rng(seed), (n,), dtype)
