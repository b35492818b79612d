// Shared-memory Stockham FFTs for the discrete-dipole operator.
//
// A thread block transforms `lines` independent 1D sequences of length N
// (N = 2^a 3^b, N <= 256) held line-major in shared memory, with radix-4,
// radix-2 and radix-3 autosort stages (Stockham: every stage reads one
// buffer and writes the other in natural order, so no bit reversal).  For a
// stage of radix R after Ns points have been combined, butterfly j of a line
// reads the R inputs j + r N/R, multiplies input r by the twiddle
// W_N^(r (j mod Ns) N/(Ns R)), takes an R-point DFT and writes its outputs
// to (j div Ns) Ns R + (j mod Ns) + r Ns.  Twiddles come from a table
// W[t] = exp(-2 pi i t / N) in the working precision (conjugated for the
// inverse transform), computed once on the host in double.
#pragma once

#include "common.cuh"

namespace ccg {

constexpr int kFftMaxN = 256;

__host__ __device__ __forceinline__ int fft_radix(int rem) { return (rem % 4 == 0) ? 4 : ((rem % 2 == 0) ? 2 : 3); }

template <class T> __device__ __forceinline__ T mul_i(T v, int sign) {  // (sign * i) * v
  T r;
  if (sign > 0) { r.x = -v.y; r.y = v.x; }
  else { r.x = v.y; r.y = -v.x; }
  return r;
}

template <class R> __device__ __forceinline__ void dft_small(cx<R> (&v)[4], int radix, int sign) {
  if (radix == 4) {
    const cx<R> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const cx<R> c = cadd(v[1], v[3]), d = mul_i(csub(v[1], v[3]), sign);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  } else if (radix == 2) {
    const cx<R> a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else {  // radix 3: W_3 = -1/2 + sign i sqrt(3)/2
    const R h = (R)0.8660254037844386;  // sqrt(3)/2
    const cx<R> s = cadd(v[1], v[2]);
    const cx<R> m = cscale(h, mul_i(csub(v[1], v[2]), sign));
    const cx<R> base = csub(v[0], cscale((R)0.5, s));
    v[0] = cadd(v[0], s);
    v[1] = cadd(base, m);
    v[2] = csub(base, m);
  }
}

// Transform `lines` sequences of length N stored line-major in a; b is a
// scratch buffer of the same size.  Returns the buffer holding the result.
// All threads of the block must call it (it synchronises).
template <class R>
__device__ cx<R>* block_fft(cx<R>* a, cx<R>* b, int N, int lines, const cx<R>* __restrict__ W, int sign) {
  int Ns = 1, rem = N;
  while (rem > 1) {
    const int radix = fft_radix(rem);
    const int nb = N / radix;
    const int tw_step = N / (Ns * radix);
    for (int t = threadIdx.x; t < lines * nb; t += blockDim.x) {
      const int l = t / nb, j = t - l * nb;
      const int k = j % Ns;
      const cx<R>* src = a + l * N;
      cx<R> v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (r < radix) {
          cx<R> e = src[j + r * nb];
          if (r > 0 && k > 0) {
            cx<R> w = __ldg(&W[(r * k * tw_step) % N]);
            if (sign > 0) w = cconj(w);
            e = cmul(e, w);
          }
          v[r] = e;
        }
      }
      dft_small<R>(v, radix, sign);
      cx<R>* dst = b + l * N + (j / Ns) * Ns * radix + k;
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r < radix) dst[r * Ns] = v[r];
    }
    __syncthreads();
    cx<R>* tmp = a;
    a = b;
    b = tmp;
    Ns *= radix;
    rem /= radix;
  }
  return a;
}

// The same transform with N and the number of lines fixed at compile time:
// the radix schedule, loop trip counts and every index division fold into
// constants (the runtime version above serves unusual sizes).  Lines are
// stored LS = N + 1 elements apart so that the line-major <-> element-major
// transposes of the strided passes hit distinct shared-memory banks.
template <int N> constexpr int fft_ls() { return N > 0 ? N + 1 : 0; }

template <class R, int N, int LINES, int NS, int REM>
__device__ __forceinline__ cx<R>* fft_stages(cx<R>* a, cx<R>* b, const cx<R>* __restrict__ W, int sign) {
  if constexpr (REM <= 1) {
    return a;
  } else {
    constexpr int RAD = (REM % 4 == 0) ? 4 : ((REM % 2 == 0) ? 2 : 3);
    constexpr int NB = N / RAD;
    constexpr int TW = N / (NS * RAD);
    constexpr int TOTAL = LINES * NB;
#pragma unroll
    for (int t0 = 0; t0 < TOTAL; t0 += kBlock) {
      const int t = t0 + (int)threadIdx.x;
      if (TOTAL % kBlock == 0 || t < TOTAL) {
        const int l = t / NB, j = t - l * NB;
        const int k = j % NS;
        const cx<R>* src = a + l * fft_ls<N>();
        cx<R> v[4];
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
          cx<R> e = src[j + r * NB];
          if (r > 0 && NS > 1) {
            cx<R> w = __ldg(&W[(r * k * TW) % N]);
            if (sign > 0) w = cconj(w);
            e = cmul(e, w);
          }
          v[r] = e;
        }
        dft_small<R>(v, RAD, sign);
        cx<R>* dst = b + l * fft_ls<N>() + (j / NS) * NS * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) dst[r * NS] = v[r];
      }
    }
    __syncthreads();
    return fft_stages<R, N, LINES, NS * RAD, REM / RAD>(b, a, W, sign);
  }
}

// Dispatch: N > 0 selects the compile-time transform of LINES lines (line
// stride N + 1), N == 0 the runtime one (n, lines given at run time, line
// stride n).
template <class R, int N, int LINES>
__device__ __forceinline__ cx<R>* fft_lines(cx<R>* a, cx<R>* b, int n, int lines, const cx<R>* __restrict__ W,
                                            int sign) {
  if constexpr (N > 0) {
    return fft_stages<R, N, LINES, 1, N>(a, b, W, sign);
  } else {
    return block_fft<R>(a, b, n, lines, W, sign);
  }
}

// Line geometry of a strided pass: element j of line (a, c) of component q
// sits at base + q * comp_stride + a * s_a + j * s_j + c, with c contiguous.
// A block takes `bl` consecutive c for one a, so each of its loads and
// stores touches bl consecutive elements.  Elements j >= in_len read as
// zero; only j < out_len are stored.
struct StridedPass {
  int64_t comp_stride, s_a, s_j;
  int na, nc;
  int n, in_len, out_len;
  int bl;
};

template <class R, int N = 0, int BL = 0>
__global__ void __launch_bounds__(kBlock) fft_strided(cx<R>* __restrict__ data, StridedPass g,
                                                      const cx<R>* __restrict__ W, int sign,
                                                      const SolveState* __restrict__ st) {
  if (st != nullptr && (st->poll.done || st->half || st->skip_mv)) return;
  extern __shared__ unsigned char smem_raw[];
  const int n = N > 0 ? N : g.n;
  const int ls = N > 0 ? fft_ls<N>() : g.n;
  const int bl = BL > 0 ? BL : g.bl;
  cx<R>* buf0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf1 = buf0 + bl * ls;
  const int cblocks = (g.nc + bl - 1) / bl;
  const int a = blockIdx.x / cblocks;
  const int c0 = (blockIdx.x - a * cblocks) * bl;
  cx<R>* base = data + (int64_t)blockIdx.y * g.comp_stride + (int64_t)a * g.s_a + c0;
  for (int t = threadIdx.x; t < bl * n; t += blockDim.x) {
    const int b = t % bl, j = t / bl;
    cx<R> v = mk<R>(0, 0);
    if (j < g.in_len && c0 + b < g.nc) v = base[(int64_t)j * g.s_j + b];
    buf0[b * ls + j] = v;
  }
  __syncthreads();
  const cx<R>* res = fft_lines<R, N, BL>(buf0, buf1, n, bl, W, sign);
  for (int t = threadIdx.x; t < bl * g.out_len; t += blockDim.x) {
    const int b = t % bl, j = t / bl;
    if (c0 + b < g.nc) base[(int64_t)j * g.s_j + b] = res[b * ls + j];
  }
}

// Contiguous pass: line l of component q is data[q * comp_stride + l * s_line + i],
// i < n, all lines full length (used for the one-time field-tensor transform).
template <class R>
__global__ void __launch_bounds__(kBlock) fft_contig(cx<R>* __restrict__ data, int64_t comp_stride, int64_t s_line,
                                                     int nlines, int n, int bl, const cx<R>* __restrict__ W,
                                                     int sign) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* buf0 = reinterpret_cast<cx<R>*>(smem_raw);
  cx<R>* buf1 = buf0 + bl * n;
  const int l0 = blockIdx.x * bl;
  cx<R>* base = data + (int64_t)blockIdx.y * comp_stride;
  for (int t = threadIdx.x; t < bl * n; t += blockDim.x) {
    const int b = t / n, i = t - b * n;
    buf0[t] = (l0 + b < nlines) ? base[(int64_t)(l0 + b) * s_line + i] : mk<R>(0, 0);
  }
  __syncthreads();
  const cx<R>* res = block_fft<R>(buf0, buf1, n, bl, W, sign);
  for (int t = threadIdx.x; t < bl * n; t += blockDim.x) {
    const int b = t / n, i = t - b * n;
    if (l0 + b < nlines) base[(int64_t)(l0 + b) * s_line + i] = res[t];
  }
}

}  // namespace ccg
