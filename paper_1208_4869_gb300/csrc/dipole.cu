// Discrete-dipole operator (the DDSCAT application of the manual, Sec. 1):
//     (A p)_s = p_s / alpha - sum_{t != s} G(r_s - r_t) p_t
// over the occupied sites of an nx x ny x nz lattice with unit spacing, G the
// field tensor of an oscillating point dipole (Gaussian units),
//     G(r) = exp(ikr)/r^3 [ (kr)^2 (I - u u^T) + (1 - ikr)(3 u u^T - I) ],
// and the Clausius-Mossotti polarizability alpha = (3/4pi)(m^2-1)/(m^2+2).
//
// The sum is a convolution on the lattice, applied by FFT on a grid of
// M = 2n points per axis (circulant embedding: grid index q < n is
// displacement q, q > n is q - M, q = n and the origin carry zero).  One
// application is five kernels, pruned to the nonzero input octant and the
// needed output octant, with the scatter, the 3x3 tensor multiply and the
// gather fused into FFT passes:
//   K1 scatter p into z-lines (i < nx, j < ny) + forward FFT along z
//   K2 forward FFT along y for i < nx (input j < ny)
//   K3 forward FFT along x (input i < nx), Y_a = sum_b Ghat_ab X_b, inverse
//      FFT along x (output i < nx), all three components in one block
//   K4 inverse FFT along y for i < nx (output j < ny)
//   K5 inverse FFT along z + gather + diagonal term into y
// Ghat (six symmetric components, scaled by 1/(Mx My Mz)) is computed once
// per operator in double precision with the same FFT passes.  Reflecting one
// axis of the lattice flips the sign of the components with exactly one index
// along it (xy, xz odd in x; xy, yz odd in y; xz, yz odd in z; the diagonal
// ones are even), and the circulant embedding maps displacement q to -q as
// grid index q -> M - q, so Ghat(M - k) along that axis is Ghat(k) times the
// same sign.  Only the octant 0 <= k <= M/2 per axis is kept (1/8 of the
// tensor: 13 MB instead of 101 MB at M = 128 in complex64, which stays in
// L2 between applications).  Unknowns are
// ordered v[a * N + s] (component a = x, y, z; sites lexicographic, z
// fastest).  A is complex symmetric, so A^H p = conj(A conj(p)).
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace ccg {

struct DipGeom {
  int nx, ny, nz;
  int Mx, My, Mz;
  int64_t G;  // Mx * My * Mz
  int64_t N;  // occupied sites
  int Hy, Hz; // octant extents along y and z (M/2 + 1)
  int64_t H;  // octant points (Mx/2 + 1)(My/2 + 1)(Mz/2 + 1)
};

template <class R> static bool dipole_fused(const DipGeom& g);

static DipGeom geom(const ccg_operator* op) {
  DipGeom g;
  g.nx = op->dip.nx; g.ny = op->dip.ny; g.nz = op->dip.nz;
  g.Mx = 2 * g.nx; g.My = 2 * g.ny; g.Mz = 2 * g.nz;
  g.G = (int64_t)g.Mx * g.My * g.Mz;
  g.N = op->dip.nsites;
  g.Hy = g.ny + 1;
  g.Hz = g.nz + 1;
  g.H = (int64_t)(g.nx + 1) * g.Hy * g.Hz;
  return g;
}

__device__ __forceinline__ bool skip_state(const SolveState* st) {
  return st != nullptr && (st->poll.done || st->half || st->skip_mv);
}

// ---------------------------------------------------------------------------
// Runtime-length kernels (FFT lengths without a register factorisation):
// shared-memory Stockham transforms, bl lines per block.

// K1: gather the lattice z-line (i, j) of component q from the site vector,
// zero-pad to Mz, forward FFT, store grid[q][i][j][:].
template <class R>
__global__ void __launch_bounds__(kBlock) dip_fwd_z(const cx<R>* __restrict__ x, cx<R>* __restrict__ grid,
                                                    const int* __restrict__ idx, DipGeom g, int bl,
                                                    const cx<R>* __restrict__ W, int conj_in,
                                                    const SolveState* __restrict__ st, int* skip_rec) {
  pdl_wait();
  pdl_launch();
  if (sweep_skipped(st, skip_rec)) return;
  extern __shared__ unsigned char smem_raw[];
  const int Mz = g.Mz, ls = g.Mz;
  cx<R>* buf0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf1 = buf0 + bl * ls;
  const int q = blockIdx.y;
  const int64_t nlines = (int64_t)g.nx * g.ny;
  const int64_t l0 = (int64_t)blockIdx.x * bl;
  const cx<R>* xq = x + (int64_t)q * g.N;
  for (int t = threadIdx.x; t < bl * Mz; t += blockDim.x) {
    const int b = t / Mz, l = t - b * Mz;
    const int64_t line = l0 + b;
    cx<R> v = mk<R>(0, 0);
    if (line < nlines && l < g.nz) {
      const int s = __ldg(&idx[line * g.nz + l]);
      if (s >= 0) {
        v = xq[s];
        if (conj_in) v = cconj(v);
      }
    }
    buf0[b * ls + l] = v;
  }
  __syncthreads();
  const cx<R>* res = block_fft<R>(buf0, buf1, Mz, bl, W, -1);
  cx<R>* gq = grid + (int64_t)q * g.G;
  for (int t = threadIdx.x; t < bl * Mz; t += blockDim.x) {
    const int b = t / Mz, kz = t - b * Mz;
    const int64_t line = l0 + b;
    if (line < nlines) {
      const int64_t i = line / g.ny, j = line - i * g.ny;
      gq[(i * g.My + j) * Mz + kz] = res[b * ls + kz];
    }
  }
}

// K3: x-lines (ky, kz0 .. kz0+bl-1) of all three components: forward FFT
// (input i < nx), tensor multiply, inverse FFT, store i < nx.
template <class R>
__global__ void __launch_bounds__(kBlock) dip_x_mul(cx<R>* __restrict__ grid, const cx<R>* __restrict__ ghat,
                                                    DipGeom g, int bl, const cx<R>* __restrict__ W,
                                                    const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (skip_state(st)) return;
  extern __shared__ unsigned char smem_raw[];
  const int Mx = g.Mx, ls = g.Mx;
  const int per = bl * ls;                      // one component's lines
  cx<R>* buf0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf1 = buf0 + 3 * per;
  const int cblocks = (g.Mz + bl - 1) / bl;
  const int ky = blockIdx.x / cblocks;
  const int kz0 = (blockIdx.x - ky * cblocks) * bl;
  const int64_t sx = (int64_t)g.My * g.Mz;      // stride along x
  const int64_t off = (int64_t)ky * g.Mz + kz0;
  for (int t = threadIdx.x; t < 3 * bl * Mx; t += blockDim.x) {
    const int q = t / (bl * Mx), r = t - q * (bl * Mx);
    const int b = r % bl, i = r / bl;
    cx<R> v = mk<R>(0, 0);
    if (i < g.nx && kz0 + b < g.Mz) v = grid[(int64_t)q * g.G + i * sx + off + b];
    buf0[q * per + b * ls + i] = v;
  }
  __syncthreads();
  cx<R>* fw = block_fft<R>(buf0, buf1, Mx, 3 * bl, W, -1);
  cx<R>* other = fw == buf0 ? buf1 : buf0;
  for (int t = threadIdx.x; t < bl * Mx; t += blockDim.x) {
    const int b = t % bl, kx = t / bl;
    const int kz = kz0 + b;
    if (kz < g.Mz) {
      // octant point and the reflection signs of the odd components
      const bool fx = kx > g.nx, fy = ky > g.ny, fz = kz > g.nz;
      const int64_t hi = ((int64_t)(fx ? g.Mx - kx : kx) * g.Hy + (fy ? g.My - ky : ky)) * g.Hz + (fz ? g.Mz - kz : kz);
      cx<R> c[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) c[k] = __ldg(&ghat[(int64_t)k * g.H + hi]);
      if (fx ^ fy) c[1] = cscale((R)-1, c[1]);
      if (fx ^ fz) c[2] = cscale((R)-1, c[2]);
      if (fy ^ fz) c[4] = cscale((R)-1, c[4]);
      const int e = b * ls + kx;
      const cx<R> X0 = fw[e], X1 = fw[per + e], X2 = fw[2 * per + e];
      // components xx, xy, xz, yy, yz, zz
      fw[e] = cfma(c[2], X2, cfma(c[1], X1, cmul(c[0], X0)));
      fw[per + e] = cfma(c[4], X2, cfma(c[3], X1, cmul(c[1], X0)));
      fw[2 * per + e] = cfma(c[5], X2, cfma(c[4], X1, cmul(c[2], X0)));
    }
  }
  __syncthreads();
  const cx<R>* res = block_fft<R>(fw, other, Mx, 3 * bl, W, +1);
  for (int t = threadIdx.x; t < 3 * bl * g.nx; t += blockDim.x) {
    const int q = t / (bl * g.nx), r = t - q * (bl * g.nx);
    const int b = r % bl, i = r / bl;
    if (kz0 + b < g.Mz) grid[(int64_t)q * g.G + i * sx + off + b] = res[q * per + b * ls + i];
  }
}

// K5: inverse FFT of z-line (i, j) of component q, then for occupied sites
// y = x / alpha - (G * x) (conjugated in and out for A^H).
template <class R>
__global__ void __launch_bounds__(kBlock) dip_inv_z(const cx<R>* __restrict__ x, cx<R>* __restrict__ y,
                                                    cx<R>* __restrict__ grid, const int* __restrict__ idx, DipGeom g,
                                                    int bl, const cx<R>* __restrict__ W, cx<R> alpha_inv, int conj,
                                                    const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (skip_state(st)) return;
  extern __shared__ unsigned char smem_raw[];
  const int Mz = g.Mz, ls = g.Mz;
  cx<R>* buf0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf1 = buf0 + bl * ls;
  const int q = blockIdx.y;
  const int64_t nlines = (int64_t)g.nx * g.ny;
  const int64_t l0 = (int64_t)blockIdx.x * bl;
  const cx<R>* gq = grid + (int64_t)q * g.G;
  for (int t = threadIdx.x; t < bl * Mz; t += blockDim.x) {
    const int b = t / Mz, kz = t - b * Mz;
    const int64_t line = l0 + b;
    cx<R> v = mk<R>(0, 0);
    if (line < nlines) {
      const int64_t i = line / g.ny, j = line - i * g.ny;
      v = gq[(i * g.My + j) * Mz + kz];
    }
    buf0[b * ls + kz] = v;
  }
  __syncthreads();
  const cx<R>* res = block_fft<R>(buf0, buf1, Mz, bl, W, +1);
  const cx<R>* xq = x + (int64_t)q * g.N;
  cx<R>* yq = y + (int64_t)q * g.N;
  for (int t = threadIdx.x; t < bl * g.nz; t += blockDim.x) {
    const int b = t / g.nz, l = t - b * g.nz;
    const int64_t line = l0 + b;
    if (line < nlines) {
      const int s = __ldg(&idx[line * g.nz + l]);
      if (s >= 0) {
        cx<R> xi = xq[s];
        if (conj) xi = cconj(xi);
        cx<R> v = csub(cmul(alpha_inv, xi), res[b * ls + l]);
        if (conj) v = cconj(v);
        yq[s] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Register-FFT kernels (lengths with a factorisation in fft.cuh).  BL lattice
// lines per block, one line per lane, so that global accesses along the
// lines' common contiguous axis coalesce.

// Lines per block: 32 (complex64) / 16 (complex128): 256 contiguous bytes per warp access.
template <class R> constexpr int reg_bl() { return sizeof(R) == 4 ? 32 : 16; }
// Shared memory of the z kernels: staging U (N rows of BL + 1, an odd stride
// so the transposes are conflict-free) and the exchange buffer E (N x BL).
template <class R, int N> constexpr size_t z_reg_smem() {
  return (size_t)N * (reg_bl<R>() + 1) * sizeof(cx<R>) + (size_t)N * reg_bl<R>() * sizeof(cx<R>);
}

// K1: gather the z-lines of BL lattice columns (i, j) from the site vector
// into shared memory (coalesced along z), forward z FFT, store the
// transformed lines through shared memory (coalesced along z).
template <class R, int N>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 3 : 2) dip_fwd_z_reg(const cx<R>* __restrict__ x, cx<R>* __restrict__ grid,
                                                        const int* __restrict__ idx, DipGeom g,
                                                        const cx<R>* __restrict__ W, int conj_in,
                                                        const SolveState* __restrict__ st, int* skip_rec) {
  pdl_wait();
  pdl_launch();
  if (sweep_skipped(st, skip_rec)) return;
  constexpr int BL = reg_bl<R>(), LS = BL + 1, NZ = N / 2;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* U = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* E = U + N * LS;
  const int q = blockIdx.y;
  const int64_t nlines = (int64_t)g.nx * g.ny;
  const int64_t l0 = (int64_t)blockIdx.x * BL;
  const cx<R>* xq = x + (int64_t)q * g.N;
#pragma unroll
  for (int t = threadIdx.x; t < BL * NZ; t += kBlock) {
    const int z = t % NZ, b = t / NZ;
    const int64_t line = l0 + b;
    cx<R> v = mk<R>(0, 0);
    if (line < nlines) {
      const int s = __ldg(&idx[line * NZ + z]);
      if (s >= 0) {
        v = xq[s];
        if (conj_in) v = cconj(v);
      }
    }
    U[z * LS + b] = v;
  }
  __syncthreads();
  auto load = [&](int j, int b) { return U[j * LS + b]; };
  auto store = [&](int k, int b, cx<R> v) { U[k * LS + b] = v; };
  fft2<R, N, BL, -1, NZ, N>(load, store, E, W);
  __syncthreads();
  cx<R>* gq = grid + (int64_t)q * g.G;
#pragma unroll 4
  for (int t = threadIdx.x; t < BL * N; t += kBlock) {
    const int kz = t % N, b = t / N;
    const int64_t line = l0 + b;
    if (line < nlines) {
      const int64_t i = line / g.ny, j = line - i * g.ny;
      gq[(i * g.My + j) * N + kz] = U[kz * LS + b];
    }
  }
}

// Class-major z order of the fused kernels (described with them below).
constexpr int kFusedLine = 32;   // z positions per class; lines per block

// z frequency at class-major position pos of a grid of N points per axis
template <int N> __device__ __forceinline__ int fused_kz(int pos) {
  return (N / kFusedLine) * (pos % kFusedLine) + pos / kFusedLine;
}
// class-major position of z frequency kz
template <int N> __device__ __forceinline__ int fused_pos(int kz) {
  return (kz % (N / kFusedLine)) * kFusedLine + kz / (N / kFusedLine);
}
// Index along z of frequency kz <= N/2 in the class-major octant: class 0
// (kz = 0, G, .., N/2: 17 values) first, then classes c = 1 .. G-1 (16 values
// each, kz = G m + c).
__host__ __device__ __forceinline__ int fused_octant_z(int kz, int G) {
  const int c = kz % G, m = kz / G;
  return (c == 0 ? 0 : 16 * c + 1) + m;
}

// K3: x-lines (ky, kz0 .. kz0 + BL - 1) of the three components (with PZ,
// z positions in the fused kernels' class-major order).  Forward
// step 1 over the input i < nx; then each thread, for its (line, k1), takes
// forward step 2, the tensor multiply Y_a = sum_b Ghat_ab X_b at the N2
// frequencies k1 + N1 k2 it holds, and inverse step 1, in place in the
// exchange buffer; inverse step 2 stores the outputs i < nx.
template <class R, int N, bool PZ = false>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 2 : 1) dip_x_mul_reg(cx<R>* __restrict__ grid, const cx<R>* __restrict__ ghat,
                                                        DipGeom g, const cx<R>* __restrict__ W,
                                                        const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (skip_state(st)) return;
  constexpr int BL = reg_bl<R>(), N1 = Fac<N>::N1, N2 = Fac<N>::N2, CS = N * BL;
  static_assert(N1 % 2 == 0, "the input and output halves need an even N1");
  extern __shared__ unsigned char smem_raw[];
  cx<R>* E = reinterpret_cast<cx<R>*>(smem_raw);  // [component][k1][j2][line]
  const int cblocks = (g.Mz + BL - 1) / BL;
  const int ky = blockIdx.x / cblocks;
  const int kz0 = (blockIdx.x - ky * cblocks) * BL;
  const int nb = min(BL, g.Mz - kz0);
  const int64_t sx = (int64_t)g.My * g.Mz;
  const int64_t off = (int64_t)ky * g.Mz + kz0;
#pragma unroll 1
  for (int t = threadIdx.x; t < BL * N2; t += kBlock) {
    const int b = t % BL, j2 = t / BL;
    // the three components' inputs (i < nx: j1 < N1 / 2) are loaded together
    cx<R> in[3][N1 / 2];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const cx<R>* src = grid + (int64_t)q * g.G + off + b;
#pragma unroll
      for (int j1 = 0; j1 < N1 / 2; ++j1) in[q][j1] = b < nb ? src[(int64_t)(N2 * j1 + j2) * sx] : mk<R>(0, 0);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      cx<R> u[N1];
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) u[j1] = j1 < N1 / 2 ? in[q][j1] : mk<R>(0, 0);
      dft<N1, -1, R>(u);
      cx<R>* Eq = E + q * CS;
      Eq[j2 * BL + b] = u[0];
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) Eq[(k1 * N2 + j2) * BL + b] = cmul(u[k1], line_tw<-1, R>(W, j2 * k1));
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int t = threadIdx.x; t < BL * N1; t += kBlock) {
    const int b = t % BL, k1 = t / BL;
    cx<R> X[3][N2];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) X[q][j2] = E[q * CS + (k1 * N2 + j2) * BL + b];
      dft<N2, -1, R>(X[q]);
    }
    if (b < nb) {
      int kz, hz;
      bool fz;
      if constexpr (PZ) {  // class-major z positions and octant (the fused kernels' layout)
        kz = fused_kz<N>(kz0 + b);
        fz = kz > g.nz;
        hz = fused_octant_z(fz ? g.Mz - kz : kz, N / kFusedLine);
      } else {
        kz = kz0 + b;
        fz = kz > g.nz;
        hz = fz ? g.Mz - kz : kz;
      }
      const bool fy = ky > g.ny;
      const int64_t hyz = (int64_t)(fy ? g.My - ky : ky) * g.Hz + hz;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int kx = k1 + N1 * k2;
        const bool fx = kx > g.nx;
        const int64_t hi = (int64_t)(fx ? g.Mx - kx : kx) * g.Hy * g.Hz + hyz;
        cx<R> c[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) c[k] = __ldg(&ghat[(int64_t)k * g.H + hi]);
        if (fx ^ fy) c[1] = cscale((R)-1, c[1]);
        if (fx ^ fz) c[2] = cscale((R)-1, c[2]);
        if (fy ^ fz) c[4] = cscale((R)-1, c[4]);
        const cx<R> X0 = X[0][k2], X1 = X[1][k2], X2 = X[2][k2];
        // components xx, xy, xz, yy, yz, zz
        X[0][k2] = cfma(c[2], X2, cfma(c[1], X1, cmul(c[0], X0)));
        X[1][k2] = cfma(c[4], X2, cfma(c[3], X1, cmul(c[1], X0)));
        X[2][k2] = cfma(c[5], X2, cfma(c[4], X1, cmul(c[2], X0)));
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      dft<N2, +1, R>(X[q]);
      E[q * CS + (k1 * N2) * BL + b] = X[q][0];
#pragma unroll
      for (int n1 = 1; n1 < N2; ++n1) E[q * CS + (k1 * N2 + n1) * BL + b] = cmul(X[q][n1], line_tw<+1, R>(W, k1 * n1));
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int t = threadIdx.x; t < BL * N2; t += kBlock) {
    const int b = t % BL, n1 = t / BL;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      cx<R> v[N1];
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) v[k1] = E[q * CS + (k1 * N2 + n1) * BL + b];
      dft<N1, +1, R>(v);
      if (b < nb) {
        cx<R>* dst = grid + (int64_t)q * g.G + off + b;
#pragma unroll
        for (int n2 = 0; n2 < N1 / 2; ++n2) dst[(int64_t)(n1 + N2 * n2) * sx] = v[n2];
      }
    }
  }
}

// K5: the transformed z-lines of BL lattice columns through shared memory
// (coalesced along z), inverse z FFT, then for occupied sites
// y = x / alpha - (G * x) (conjugated in and out for A^H), coalesced along z.
template <class R, int N>
__global__ void __launch_bounds__(kBlock, sizeof(R) == 4 ? 3 : 2) dip_inv_z_reg(const cx<R>* __restrict__ x, cx<R>* __restrict__ y,
                                                        const cx<R>* __restrict__ grid, const int* __restrict__ idx,
                                                        DipGeom g, const cx<R>* __restrict__ W, cx<R> alpha_inv,
                                                        int conj, const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (skip_state(st)) return;
  constexpr int BL = reg_bl<R>(), LS = BL + 1, NZ = N / 2;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* U = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* E = U + N * LS;
  const int q = blockIdx.y;
  const int64_t nlines = (int64_t)g.nx * g.ny;
  const int64_t l0 = (int64_t)blockIdx.x * BL;
  const cx<R>* gq = grid + (int64_t)q * g.G;
#pragma unroll 4
  for (int t = threadIdx.x; t < BL * N; t += kBlock) {
    const int kz = t % N, b = t / N;
    const int64_t line = l0 + b;
    cx<R> v = mk<R>(0, 0);
    if (line < nlines) {
      const int64_t i = line / g.ny, j = line - i * g.ny;
      v = gq[(i * g.My + j) * N + kz];
    }
    U[kz * LS + b] = v;
  }
  __syncthreads();
  auto load = [&](int j, int b) { return U[j * LS + b]; };
  auto store = [&](int k, int b, cx<R> v) { U[k * LS + b] = v; };
  fft2<R, N, BL, +1, N, NZ>(load, store, E, W);
  __syncthreads();
  const cx<R>* xq = x + (int64_t)q * g.N;
  cx<R>* yq = y + (int64_t)q * g.N;
#pragma unroll 4
  for (int t = threadIdx.x; t < BL * NZ; t += kBlock) {
    const int z = t % NZ, b = t / NZ;
    const int64_t line = l0 + b;
    if (line < nlines) {
      const int s = __ldg(&idx[line * NZ + z]);
      if (s >= 0) {
        cx<R> xi = xq[s];
        if (conj) xi = cconj(xi);
        cx<R> v = csub(cmul(alpha_inv, xi), U[z * LS + b]);
        if (conj) v = cconj(v);
        yq[s] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Fused z-and-y kernels for cubic lattices (nx = ny = nz = N / 2): one block
// transforms one x-plane of one component in a class of 32 lines in both
// directions, so the z and y passes of each direction become one kernel (3
// kernels per application instead of 5) and the half-transformed plane never
// leaves shared memory.
//
// The classes come from decimation in frequency, so that no block repeats
// another's work.  Forward, with G = N / 32: the z frequencies kz = G m + r
// (m < 32) of class r are a 32-point DFT of the folded line
//     f_r(z') = sum_{p < G/2} x(z' + 32 p) W_N^(r (z' + 32 p)),   z' < 32
// (x is zero for z >= N/2), so each block transforms its plane's N/2
// z-lines at length 32 and then the 32 kz-lines of its class along y.  The
// grid keeps the z frequencies class-major: position r 32 + m holds
// kz = G m + r, so every block writes whole 256-byte rows; the x pass and
// the field-tensor octant follow that order (fused_kz, fused_octant_z).
// Inverse, with Gy = N / 64: the outputs j = Gy m + g (m < 32) of the
// inverse y transform are a 64-point inverse DFT (its first 32 outputs) of
//     h_g(ky') = sum_{p < Gy} X(ky' + 64 p) W_N^(-g (ky' + 64 p)),  ky' < 64,
// so each block transforms the plane's N kz-lines at length 64, then its 32
// j-lines along z (reading the class-major positions in frequency order).
// ---------------------------------------------------------------------------
template <class R, int N> constexpr size_t fwd_zy_smem() {
  // P (N/2 x (N/2 + 1)) -- reused as the y transform's exchange buffer
  // (N x 32) --, T (N/2 x 33), the z transform's exchange buffer (32 x N/2)
  constexpr size_t NH = N / 2, P = NH * (NH + 1), EY = (size_t)N * kFusedLine;
  return ((P > EY ? P : EY) + NH * (kFusedLine + 1) + (size_t)kFusedLine * NH) * sizeof(cx<R>);
}
template <class R, int N> constexpr size_t inv_yz_smem() {
  // Vb (32 x (N + 1)), then the exchange buffer (N x 32)
  return ((size_t)kFusedLine * (N + 1) + (size_t)N * kFusedLine) * sizeof(cx<R>);
}
// Lengths with the fused kernels: complex64 (complex128 keeps the five
// passes: its FP64 pipe makes the in-block transforms slower than the
// passes they save), register-FFT lengths whose half is a multiple of the
// class size, forward buffers that fit in shared memory.
template <class R, int N> constexpr bool fused_ok() {
  return sizeof(R) == 4 && reg_bl<R>() == kFusedLine && Fac<N>::N1 > 0 && (N / 2) % kFusedLine == 0 &&
         fwd_zy_smem<R, N>() <= 200 * 1024;
}

// Forward: gather the (j, z) plane i of component q from the site vector,
// the length-32 z transforms of class r for its N/2 j-lines, then the y FFT
// of those 32 kz-lines (input j < N/2), written to grid[q][i][ky][r 32 ..].
template <class R, int N>
__global__ void __launch_bounds__(kBlock) dip_fwd_zy(const cx<R>* __restrict__ x, cx<R>* __restrict__ grid,
                                                     const int* __restrict__ idx, DipGeom g,
                                                     const cx<R>* __restrict__ Wz, const cx<R>* __restrict__ Wy,
                                                     int conj_in, const SolveState* __restrict__ st,
                                                     int* skip_rec) {
  pdl_wait();
  pdl_launch();
  if (sweep_skipped(st, skip_rec)) return;
  constexpr int BL = kFusedLine, NH = N / 2, G = N / BL;
  constexpr int PS = NH + 1, TS = BL + 1;  // odd strides: conflict-free transposes
  constexpr size_t PE = (size_t)NH * PS > (size_t)N * BL ? (size_t)NH * PS : (size_t)N * BL;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* P = reinterpret_cast<cx<R>*>(smem_raw);  // P[z * PS + j]; then the y exchange buffer
  cx<R>* T = P + PE;                               // T[j * TS + m], kz = G m + r
  cx<R>* EZ = T + NH * TS;                         // z exchange buffer (BL x NH)
  const int q = blockIdx.y;
  const int i = blockIdx.x / G;
  const int r = blockIdx.x - i * G;
  const cx<R>* xq = x + (int64_t)q * g.N;
#pragma unroll 4
  for (int t = threadIdx.x; t < NH * NH; t += kBlock) {
    const int z = t % NH, j = t / NH;
    const int sidx = __ldg(&idx[((int64_t)i * NH + j) * NH + z]);
    cx<R> v = mk<R>(0, 0);
    if (sidx >= 0) {
      v = xq[sidx];
      if (conj_in) v = cconj(v);
    }
    P[z * PS + j] = v;
  }
  __syncthreads();
  {
    // all N/2 j-lines at once: the fold of class r, then a 32-point DFT
    auto load = [&](int zp, int b) {
      cx<R> f = mk<R>(0, 0);
#pragma unroll
      for (int p = 0; p < G / 2; ++p) {
        const int z = zp + BL * p;
        f = cfma(P[z * PS + b], line_tw<-1, R>(Wz, (r * z) % N), f);
      }
      return f;
    };
    auto store = [&](int m, int b, cx<R> v) { T[b * TS + m] = v; };
    fft2<R, BL, NH, -1, BL, BL, G>(load, store, EZ, Wz);
  }
  __syncthreads();  // T complete; P is free for the y exchange buffer
  cx<R>* gq = grid + (int64_t)q * g.G + (int64_t)i * N * N + r * BL;
  auto load = [&](int j, int b) { return T[j * TS + b]; };
  auto store = [&](int ky, int b, cx<R> v) { gq[(int64_t)ky * N + b] = v; };
  fft2<R, N, BL, -1, NH, N>(load, store, P, Wy);
}

// Inverse: the length-64 inverse y transforms of class g for the plane's N
// kz-lines (in batches of 32), keeping the outputs j = Gy m + g (m < 32);
// the inverse z FFT of those 32 j-lines (input in class-major positions,
// output z < N/2); then y = x / alpha - conv on the occupied sites
// (conjugated for A^H).
template <class R, int N>
__global__ void __launch_bounds__(kBlock) dip_inv_yz(const cx<R>* __restrict__ x, cx<R>* __restrict__ y,
                                                     const cx<R>* __restrict__ grid, const int* __restrict__ idx,
                                                     DipGeom g, const cx<R>* __restrict__ Wz,
                                                     const cx<R>* __restrict__ Wy, cx<R> alpha_inv, int conj,
                                                     const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (skip_state(st)) return;
  constexpr int BL = kFusedLine, NH = N / 2, GY = NH / BL, LY = N / GY;  // LY = 64
  constexpr int VS = N + 1, OS = BL + 1;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* Vb = reinterpret_cast<cx<R>*>(smem_raw);  // Vb[m * VS + pos]
  cx<R>* E = Vb + BL * VS;
  cx<R>* O = Vb;                                     // O[z * OS + m], written after Vb's last read
  const int q = blockIdx.y;
  const int i = blockIdx.x / GY;
  const int gc = blockIdx.x - i * GY;
  const cx<R>* gq = grid + (int64_t)q * g.G + (int64_t)i * N * N;
  for (int kb = 0; kb < N; kb += BL) {
    auto load = [&](int kyp, int b) {
      cx<R> f = mk<R>(0, 0);
#pragma unroll
      for (int p = 0; p < GY; ++p) {
        const int ky = kyp + LY * p;
        f = cfma(gq[(int64_t)ky * N + kb + b], line_tw<+1, R>(Wy, (gc * ky) % N), f);
      }
      return f;
    };
    auto store = [&](int m, int b, cx<R> v) { Vb[m * VS + kb + b] = v; };
    fft2<R, LY, BL, +1, LY, BL, GY>(load, store, E, Wy);
    __syncthreads();
  }
  {
    auto load = [&](int kz, int b) { return Vb[b * VS + fused_pos<N>(kz)]; };
    auto store = [&](int z, int b, cx<R> v) { O[z * OS + b] = v; };
    fft2<R, N, BL, +1, N, NH>(load, store, E, Wz);
  }
  __syncthreads();
  const cx<R>* xq = x + (int64_t)q * g.N;
  cx<R>* yq = y + (int64_t)q * g.N;
#pragma unroll 4
  for (int t = threadIdx.x; t < BL * NH; t += kBlock) {
    const int z = t % NH, m = t / NH;
    const int j = GY * m + gc;
    const int sidx = __ldg(&idx[((int64_t)i * NH + j) * NH + z]);
    if (sidx >= 0) {
      cx<R> xi = xq[sidx];
      if (conj) xi = cconj(xi);
      cx<R> v = csub(cmul(alpha_inv, xi), O[z * OS + m]);
      if (conj) v = cconj(v);
      yq[sidx] = v;
    }
  }
}

// One-time setup: the circulant-embedded field tensor on the grid (double).
__global__ void dip_green(double2* __restrict__ g6, DipGeom g, double k) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.G; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = p / ((int64_t)g.My * g.Mz);
    const int64_t rem = p - a * (int64_t)g.My * g.Mz;
    const int64_t b = rem / g.Mz, c = rem - b * g.Mz;
    double2 out[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) out[q] = make_double2(0.0, 0.0);
    const bool excluded = a == g.nx || b == g.ny || c == g.nz || (a == 0 && b == 0 && c == 0);
    if (!excluded) {
      const double dx = a < g.nx ? (double)a : (double)(a - g.Mx);
      const double dy = b < g.ny ? (double)b : (double)(b - g.My);
      const double dz = c < g.nz ? (double)c : (double)(c - g.Mz);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double u[3] = {dx / r, dy / r, dz / r};
      double sn, cs;
      sincos(k * r, &sn, &cs);
      const double r3 = r * r * r;
      const double2 e = make_double2(cs / r3, sn / r3);   // exp(ikr)/r^3
      const double kr2 = (k * r) * (k * r);               // multiplies (I - u u^T)
      const double2 bb = make_double2(1.0, -k * r);       // 1 - ikr, multiplies (3 u u^T - I)
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const double uu = u[ia[q]] * u[ib[q]];
        const double d = ia[q] == ib[q] ? 1.0 : 0.0;
        const double2 inner = make_double2(kr2 * (d - uu) + bb.x * (3.0 * uu - d), bb.y * (3.0 * uu - d));
        out[q] = cmul(e, inner);
      }
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) g6[(int64_t)q * g.G + p] = out[q];
  }
}

// The octant 0 <= k <= M/2 of each transformed component, scaled and
// rounded to R.
// With zclass = G > 0 the z index runs over the class-major octant order of
// the fused kernels (fused_octant_z).
template <class R>
__global__ void dip_octant(const double2* __restrict__ src, cx<R>* __restrict__ dst, DipGeom g, double scale,
                           int zclass) {
  const int64_t count = 6 * g.H;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < count; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = p / g.H, h = p - q * g.H;
    const int64_t kx = h / ((int64_t)g.Hy * g.Hz), rem = h - kx * g.Hy * g.Hz;
    const int64_t ky = rem / g.Hz, hz = rem - ky * g.Hz;
    int64_t kz = hz;
    if (zclass > 0) kz = hz <= 16 ? zclass * hz : zclass * ((hz - 1) % 16) + (hz - 1) / 16;
    const double2 v = src[q * g.G + (kx * g.My + ky) * g.Mz + kz];
    dst[p] = mk<R>((R)(v.x * scale), (R)(v.y * scale));
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
#define DIP_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return CCG_ERR_CUDA;                                                             \
    }                                                                                  \
  } while (0)

static bool fft_size_ok(int n) {
  if (n < 2 || n > kFftMaxN) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

// Lines per block of a pass: 16 for complex64, 8 for complex128 (8 for the
// three-component x pass of complex128 too, keeping shared memory <= 96 KB
// at M = 128).
template <class R> static int lines_per_block(int M) {
  int bl = sizeof(R) == 4 ? 16 : 8;
  while (bl > 1 && (size_t)3 * 2 * bl * M * sizeof(cx<R>) > 200 * 1024) bl /= 2;
  return bl;
}

template <class R> static int set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) DIP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return CCG_OK;
}

template <class R> static std::vector<cx<R>> twiddles(int n) {
  std::vector<cx<R>> w(n);
  for (int t = 0; t < n; ++t) {
    const std::complex<double> z = std::polar(1.0, -2.0 * M_PI * (double)t / (double)n);
    w[t] = mk<R>((R)z.real(), (R)z.imag());
  }
  return w;
}

// Per-operator device data, owned through ccg_operator::dip.
// Uploads go on the creation stream s: a plain cudaMemcpy from pageable
// memory may return before its DMA lands and is not ordered with a
// non-blocking stream's kernels.
template <class R> static int upload_twiddles(ccg_operator* op, const DipGeom& g, cudaStream_t s) {
  const int dims[3] = {g.Mx, g.My, g.Mz};
  for (int a = 0; a < 3; ++a) {
    std::vector<cx<R>> w = twiddles<R>(dims[a]);
    DIP_CUDA(cudaMalloc(&op->dip.tw[a], w.size() * sizeof(cx<R>)));
    DIP_CUDA(cudaMemcpyAsync(op->dip.tw[a], w.data(), w.size() * sizeof(cx<R>), cudaMemcpyHostToDevice, s));
  }
  return CCG_OK;
}

static int strided_launch_d(double2* data, const StridedPass& p, int ncomp, const double2* W, int sign,
                            cudaStream_t s) {
  const int cblocks = (p.nc + p.bl - 1) / p.bl;
  const size_t smem = (size_t)2 * p.bl * p.n * sizeof(double2);
  if (set_smem<double>((const void*)fft_strided<double>, smem) != CCG_OK) return CCG_ERR_CUDA;
  fft_strided<double><<<dim3(p.na * cblocks, ncomp), kBlock, smem, s>>>(data, p, W, sign, nullptr);
  return CCG_OK;
}

// Field tensor on the grid, forward-transformed, scaled and rounded to R.
template <class R> static int build_ghat(ccg_operator* op, const DipGeom& g, cudaStream_t s) {
  double2* g6 = nullptr;
  void* twd[3] = {nullptr, nullptr, nullptr};
  int rc = CCG_OK;
  const int dims[3] = {g.Mx, g.My, g.Mz};
  if (cudaMalloc(&g6, (size_t)6 * g.G * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    set_error("ccg_op_dipole: field-tensor setup allocation failed");
    return CCG_ERR_NOMEM;
  }
  for (int a = 0; a < 3 && rc == CCG_OK; ++a) {
    std::vector<double2> w = twiddles<double>(dims[a]);
    if (cudaMalloc(&twd[a], w.size() * sizeof(double2)) != cudaSuccess ||
        cudaMemcpyAsync(twd[a], w.data(), w.size() * sizeof(double2), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error(std::string("ccg_op_dipole: ") + cudaGetErrorString(cudaGetLastError()));
      rc = CCG_ERR_CUDA;
    }
  }
  if (rc == CCG_OK) {
    const int grid = (int)std::min<int64_t>((g.G + kBlock - 1) / kBlock, 4096);
    dip_green<<<grid, kBlock, 0, s>>>(g6, g, op->dip.kd);
    // z (contiguous lines), then y and x (strided)
    const int blz = 8;
    const size_t smz = (size_t)2 * blz * g.Mz * sizeof(double2);
    if (set_smem<double>((const void*)fft_contig<double>, smz) != CCG_OK) rc = CCG_ERR_CUDA;
    const int nlz = g.Mx * g.My;
    if (rc == CCG_OK)
      fft_contig<double><<<dim3((nlz + blz - 1) / blz, 6), kBlock, smz, s>>>(g6, g.G, g.Mz, nlz, g.Mz, blz,
                                                                             (const double2*)twd[2], -1);
    StridedPass py = {g.G, (int64_t)g.My * g.Mz, g.Mz, g.Mx, g.Mz, g.My, g.My, g.My, 8};
    if (rc == CCG_OK) rc = strided_launch_d(g6, py, 6, (const double2*)twd[1], -1, s);
    StridedPass px = {g.G, g.Mz, (int64_t)g.My * g.Mz, g.My, g.Mz, g.Mx, g.Mx, g.Mx, 8};
    if (rc == CCG_OK) rc = strided_launch_d(g6, px, 6, (const double2*)twd[0], -1, s);
    if (rc == CCG_OK) {
      if (cudaMalloc(&op->dip.ghat, (size_t)6 * g.H * sizeof(cx<R>)) != cudaSuccess) {
        cudaGetLastError();
        set_error("ccg_op_dipole: field-tensor allocation failed");
        rc = CCG_ERR_NOMEM;
      } else {
        const int zclass = dipole_fused<R>(g) ? g.Mz / kFusedLine : 0;
        dip_octant<R><<<2048, kBlock, 0, s>>>(g6, static_cast<cx<R>*>(op->dip.ghat), g, 1.0 / (double)g.G, zclass);
      }
    }
    if (rc == CCG_OK && cudaStreamSynchronize(s) != cudaSuccess) {
      set_error(std::string("ccg_op_dipole: setup failed: ") + cudaGetErrorString(cudaGetLastError()));
      rc = CCG_ERR_CUDA;
    }
  }
  cudaFree(g6);
  for (int a = 0; a < 3; ++a)
    if (twd[a]) cudaFree(twd[a]);
  return rc;
}

template <class R> static int create_t(ccg_operator* op, const uint8_t* occ, cudaStream_t s) {
  const DipGeom g = geom(op);
  // site index grid: idx[(i*ny + j)*nz + l] = site number or -1
  const int64_t cells = (int64_t)g.nx * g.ny * g.nz;
  std::vector<int> idx(cells);
  int64_t count = 0;
  for (int64_t c = 0; c < cells; ++c) idx[c] = occ[c] ? (int)(count++) : -1;
  op->dip.nsites = count;
  op->n = 3 * count;
  DIP_CUDA(cudaMalloc(&op->dip.idx, cells * sizeof(int)));
  DIP_CUDA(cudaMemcpyAsync(op->dip.idx, idx.data(), cells * sizeof(int), cudaMemcpyHostToDevice, s));
  DIP_CUDA(cudaMalloc(&op->dip.work, (size_t)3 * g.G * sizeof(cx<R>)));
  int rc = upload_twiddles<R>(op, geom(op), s);
  if (rc != CCG_OK) return rc;
  rc = build_ghat<R>(op, geom(op), s);
  if (rc != CCG_OK) return rc;
  const int bl = lines_per_block<R>(std::max(g.Mx, std::max(g.My, g.Mz)));
  op->dip.bl = bl;
  // opt in to large dynamic shared memory for the runtime-size kernels
  const int M = std::max(g.Mx, std::max(g.My, g.Mz));
  const size_t sm1 = (size_t)2 * bl * M * sizeof(cx<R>), sm3 = 3 * sm1;
  if (set_smem<R>((const void*)dip_fwd_z<R>, sm1) != CCG_OK) return CCG_ERR_CUDA;
  if (set_smem<R>((const void*)dip_inv_z<R>, sm1) != CCG_OK) return CCG_ERR_CUDA;
  if (set_smem<R>((const void*)fft_strided<R>, sm1) != CCG_OK) return CCG_ERR_CUDA;
  if (set_smem<R>((const void*)dip_x_mul<R>, sm3) != CCG_OK) return CCG_ERR_CUDA;
  // algorithmic bytes of one application (each pass reads and writes its
  // pruned region once; the field-tensor octant is read once)
  const double e = sizeof(cx<R>);
  const double zl = 3.0 * g.nx * g.ny * g.Mz * e;     // z-line region
  const double yl = 3.0 * g.nx * g.My * g.Mz * e;     // after the y pass
  const double vec = 3.0 * count * e;
  op->dip.kernels = dipole_fused<R>(g) ? 3 : 5;
  if (dipole_fused<R>(g))  // gather + one write of the y-transformed region; x pass; one read + scatter
    op->dip.sweep_bytes = (vec + cells * 4.0 + yl) + (yl + 6.0 * g.H * e + yl) + (yl + cells * 4.0 + 2 * vec);
  else
    op->dip.sweep_bytes = (vec + zl) + (zl + yl) + (yl + 6.0 * g.H * e + yl) + (yl + zl) + (zl + 2 * vec) +
                          2.0 * cells * 4.0;
  return CCG_OK;
}

int dipole_create(ccg_operator* op, const uint8_t* occ, cudaStream_t s) {
  const DipGeom g = geom(op);
  if (!fft_size_ok(g.Mx) || !fft_size_ok(g.My) || !fft_size_ok(g.Mz)) {
    set_error("ccg_op_dipole: each of 2*nx, 2*ny, 2*nz must be 2^a 3^b and at most 256");
    return CCG_ERR_INVALID;
  }
  return op->dtype == CCG_C128 ? create_t<double>(op, occ, s) : create_t<float>(op, occ, s);
}

void dipole_free(ccg_operator* op) {
  if (op->dip.idx) cudaFree(op->dip.idx);
  if (op->dip.work) cudaFree(op->dip.work);
  if (op->dip.ghat) cudaFree(op->dip.ghat);
  for (int a = 0; a < 3; ++a)
    if (op->dip.tw[a]) cudaFree(op->dip.tw[a]);
  op->dip.idx = nullptr;
  op->dip.work = op->dip.ghat = nullptr;
}

template <class F> static void smem_opt_in(F* fn, size_t bytes, bool& done) {
  if (!done && bytes > 48 * 1024) cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  done = true;
}

// A kernel of one application: with programmatic dependent launch when the
// caller's loop uses it (every application kernel waits for its predecessor
// first, pdl_wait), else in plain stream order.
template <class... KArgs, class... Args>
static void dlaunch(bool pdl, void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t s, Args... args) {
  if (pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
  } else {
    kern<<<grid, kBlock, smem, s>>>(args...);
  }
}

// Launchers: N > 0 selects the register kernels of that length, N == 0 the
// runtime-length kernels (op->dip.bl lines per block).
template <class R, int N>
static void k1(const cx<R>* x, cx<R>* grid, const ccg_operator* op, const DipGeom& g, const cx<R>* W, int conj,
               const SolveState* st, int* rec, cudaStream_t s, bool pdl) {
  const int64_t nlines = (int64_t)g.nx * g.ny;
  static bool opted = false;
  if constexpr (N > 0) {
    constexpr int BL = reg_bl<R>();
    constexpr size_t sm = z_reg_smem<R, N>();
    smem_opt_in(dip_fwd_z_reg<R, N>, sm, opted);
    dlaunch(pdl, dip_fwd_z_reg<R, N>, dim3((unsigned)((nlines + BL - 1) / BL), 3), sm, s, x, grid,
            (const int*)op->dip.idx, g, W, conj, st, rec);
  } else {
    const int bl = op->dip.bl;
    const size_t sm = (size_t)2 * bl * g.Mz * sizeof(cx<R>);
    dlaunch(pdl, dip_fwd_z<R>, dim3((unsigned)((nlines + bl - 1) / bl), 3), sm, s, x, grid, (const int*)op->dip.idx,
            g, bl, W, conj, st, rec);
  }
}
template <class R, int N>
static void k5(const cx<R>* x, cx<R>* y, cx<R>* grid, const ccg_operator* op, const DipGeom& g, const cx<R>* W,
               cx<R> ainv, int conj, const SolveState* st, cudaStream_t s, bool pdl) {
  const int64_t nlines = (int64_t)g.nx * g.ny;
  static bool opted = false;
  if constexpr (N > 0) {
    constexpr int BL = reg_bl<R>();
    constexpr size_t sm = z_reg_smem<R, N>();
    smem_opt_in(dip_inv_z_reg<R, N>, sm, opted);
    dlaunch(pdl, dip_inv_z_reg<R, N>, dim3((unsigned)((nlines + BL - 1) / BL), 3), sm, s, x, y, (const cx<R>*)grid,
            (const int*)op->dip.idx, g, W, ainv, conj, st);
  } else {
    const int bl = op->dip.bl;
    const size_t sm = (size_t)2 * bl * g.Mz * sizeof(cx<R>);
    dlaunch(pdl, dip_inv_z<R>, dim3((unsigned)((nlines + bl - 1) / bl), 3), sm, s, x, y, grid,
            (const int*)op->dip.idx, g, bl, W, ainv, conj, st);
  }
}
template <class R, int N>
static void ky(cx<R>* grid, const ccg_operator* op, const DipGeom& g, const cx<R>* W, int sign,
               const SolveState* st, cudaStream_t s, bool pdl) {
  static bool opted_f = false, opted_i = false;
  if constexpr (N > 0) {
    constexpr int BL = reg_bl<R>();
    StridedPass p = {g.G, (int64_t)g.My * g.Mz, g.Mz, g.nx, g.Mz, N, 0, 0, BL};
    const int cb = (g.Mz + BL - 1) / BL;
    constexpr size_t sm = (size_t)N * BL * sizeof(cx<R>);
    const dim3 grd((unsigned)(g.nx * cb), 3);
    if (sign < 0) {
      smem_opt_in(fft_strided_reg<R, N, BL, -1, N / 2, N>, sm, opted_f);
      dlaunch(pdl, fft_strided_reg<R, N, BL, -1, N / 2, N>, grd, sm, s, grid, p, W, st);
    } else {
      smem_opt_in(fft_strided_reg<R, N, BL, +1, N, N / 2>, sm, opted_i);
      dlaunch(pdl, fft_strided_reg<R, N, BL, +1, N, N / 2>, grd, sm, s, grid, p, W, st);
    }
  } else {
    const int bl = op->dip.bl;
    StridedPass p = {g.G, (int64_t)g.My * g.Mz, g.Mz, g.nx, g.Mz, g.My, sign < 0 ? g.ny : g.My,
                     sign < 0 ? g.My : g.ny, bl};
    const int cb = (g.Mz + bl - 1) / bl;
    const size_t sm = (size_t)2 * bl * g.My * sizeof(cx<R>);
    dlaunch(pdl, fft_strided<R>, dim3(g.nx * cb, 3), sm, s, grid, p, W, sign, st);
  }
}
template <class R, int N, bool PZ = false>
static void k3(cx<R>* grid, const ccg_operator* op, const DipGeom& g, const cx<R>* W, const SolveState* st,
               cudaStream_t s, bool pdl) {
  static bool opted = false;
  if constexpr (N > 0) {
    constexpr int BL = reg_bl<R>();
    const int cb = (g.Mz + BL - 1) / BL;
    constexpr size_t sm = (size_t)3 * N * BL * sizeof(cx<R>);
    smem_opt_in(dip_x_mul_reg<R, N, PZ>, sm, opted);
    dlaunch(pdl, dip_x_mul_reg<R, N, PZ>, dim3(g.My * cb), sm, s, grid, static_cast<const cx<R>*>(op->dip.ghat), g,
            W, st);
  } else {
    const int bl = op->dip.bl;
    const int cb = (g.Mz + bl - 1) / bl;
    const size_t sm = (size_t)3 * 2 * bl * g.Mx * sizeof(cx<R>);
    dlaunch(pdl, dip_x_mul<R>, dim3(g.My * cb), sm, s, grid, static_cast<const cx<R>*>(op->dip.ghat), g, bl, W, st);
  }
}


// FFT lengths with register kernels; other 2^a 3^b lengths use the runtime
// kernels.
#define CCG_FFT_SIZES(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256)

template <class R, int N>
static void fused_fwd(const cx<R>* x, cx<R>* grid, const ccg_operator* op, const DipGeom& g, const cx<R>* Wz,
                      const cx<R>* Wy, int conj, const SolveState* st, int* rec, cudaStream_t s, bool pdl) {
  static bool opted = false;
  constexpr size_t sm = fwd_zy_smem<R, N>();
  smem_opt_in(dip_fwd_zy<R, N>, sm, opted);
  dlaunch(pdl, dip_fwd_zy<R, N>, dim3((unsigned)(g.nx * (N / kFusedLine)), 3), sm, s, x, grid,
          (const int*)op->dip.idx, g, Wz, Wy, conj, st, rec);
}
template <class R, int N>
static void fused_inv(const cx<R>* x, cx<R>* y, const cx<R>* grid, const ccg_operator* op, const DipGeom& g,
                      const cx<R>* Wz, const cx<R>* Wy, cx<R> ainv, int conj, const SolveState* st, cudaStream_t s,
                      bool pdl) {
  static bool opted = false;
  constexpr size_t sm = inv_yz_smem<R, N>();
  smem_opt_in(dip_inv_yz<R, N>, sm, opted);
  dlaunch(pdl, dip_inv_yz<R, N>, dim3((unsigned)(g.nx * (N / 2 / kFusedLine)), 3), sm, s, x, y, grid,
          (const int*)op->dip.idx, g, Wz, Wy, ainv, conj, st);
}
// Three-kernel application for cubic lattices of a fused length; false if
// the lattice or the length has none.
template <class R, int N>
static bool apply_fused_n(const ccg_operator* op, const DipGeom& g, const cx<R>* x, cx<R>* y, cx<R>* grid,
                          const cx<R>* Wx, const cx<R>* Wy, const cx<R>* Wz, cx<R> ainv, int cj,
                          const SolveState* st, int* rec, cudaStream_t s, bool pdl) {
  if constexpr (fused_ok<R, N>()) {
    fused_fwd<R, N>(x, grid, op, g, Wz, Wy, cj, st, rec, s, pdl);
    k3<R, N, true>(grid, op, g, Wx, st, s, pdl);
    fused_inv<R, N>(x, y, grid, op, g, Wz, Wy, ainv, cj, st, s, pdl);
    return true;
  } else {
    return false;
  }
}
template <class R> static bool dipole_fused(const DipGeom& g) {
  if (!(g.nx == g.ny && g.ny == g.nz)) return false;
  switch (g.Mx) {
#define CCG_FUSED_OK(n) case n: return fused_ok<R, n>();
    CCG_FFT_SIZES(CCG_FUSED_OK)
    default: return false;
  }
}

template <class R>
static int apply_t(const ccg_operator* op, const cx<R>* x, cx<R>* y, bool conj, const SolveState* st, int* rec,
                   cudaStream_t s, bool pdl) {
  const DipGeom g = geom(op);
  cx<R>* grid = static_cast<cx<R>*>(op->dip.work);
  const cx<R>* Wx = static_cast<const cx<R>*>(op->dip.tw[0]);
  const cx<R>* Wy = static_cast<const cx<R>*>(op->dip.tw[1]);
  const cx<R>* Wz = static_cast<const cx<R>*>(op->dip.tw[2]);
  const int cj = conj ? 1 : 0;
  const cx<R> ainv = mk<R>((R)op->dip.alpha_inv[0], (R)op->dip.alpha_inv[1]);
  if (dipole_fused<R>(g)) {
    bool done = false;
    switch (g.Mx) {
#define CCG_CASE_FUSED(n) case n: done = apply_fused_n<R, n>(op, g, x, y, grid, Wx, Wy, Wz, ainv, cj, st, rec, s, pdl); break;
      CCG_FFT_SIZES(CCG_CASE_FUSED)
      default: break;
    }
    if (done) return cudaGetLastError() == cudaSuccess ? CCG_OK : CCG_ERR_CUDA;
  }
#define CCG_CASE_K1(n) case n: k1<R, n>(x, grid, op, g, Wz, cj, st, rec, s, pdl); break;
  switch (g.Mz) { CCG_FFT_SIZES(CCG_CASE_K1) default: k1<R, 0>(x, grid, op, g, Wz, cj, st, rec, s, pdl); }
#define CCG_CASE_KY(n) case n: ky<R, n>(grid, op, g, Wy, sign, st, s, pdl); break;
  for (int sign = -1; sign <= 1; sign += 2) {
    if (sign > 0) {
#define CCG_CASE_K3(n) case n: k3<R, n>(grid, op, g, Wx, st, s, pdl); break;
      switch (g.Mx) { CCG_FFT_SIZES(CCG_CASE_K3) default: k3<R, 0>(grid, op, g, Wx, st, s, pdl); }
    }
    switch (g.My) { CCG_FFT_SIZES(CCG_CASE_KY) default: ky<R, 0>(grid, op, g, Wy, sign, st, s, pdl); }
  }
#define CCG_CASE_K5(n) case n: k5<R, n>(x, y, grid, op, g, Wz, ainv, cj, st, s, pdl); break;
  switch (g.Mz) { CCG_FFT_SIZES(CCG_CASE_K5) default: k5<R, 0>(x, y, grid, op, g, Wz, ainv, cj, st, s, pdl); }
  return cudaGetLastError() == cudaSuccess ? CCG_OK : CCG_ERR_CUDA;
}

int dipole_apply(const ccg_operator* op, const double2* x, double2* y, bool conj, const SolveState* st,
                 cudaStream_t s, int* skip_rec, bool pdl) {
  return apply_t<double>(op, x, y, conj, st, skip_rec, s, pdl);
}
int dipole_apply(const ccg_operator* op, const float2* x, float2* y, bool conj, const SolveState* st,
                 cudaStream_t s, int* skip_rec, bool pdl) {
  return apply_t<float>(op, x, y, conj, st, skip_rec, s, pdl);
}

}  // namespace ccg
