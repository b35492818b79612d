// FFTs for the discrete-dipole operator.
//
// Register FFTs (lengths 16 ... 256 with a factorisation below, compiled per
// length): a line of length N = N1 N2 is transformed in two register steps
// with one shared-memory exchange (the four-step factorisation),
//   X[k1 + N1 k2] = sum_{j2 < N2} W_N2^(j2 k2) W_N^(j2 k1)
//                   sum_{j1 < N1} x[N2 j1 + j2] W_N1^(j1 k1),
// W_L = exp(-2 pi i / L) (conjugated for the inverse).  The small DFTs of
// length N1, N2 <= 16 run in registers, factored the same way recursively
// down to radix 2, 3, 4 with their twiddles as compile-time constants; the
// twiddles W_N^(j2 k1) come from a table.  Threads of a block own lines by
// lane (b fastest), so global accesses along b coalesce and the exchange
// buffer, laid out [k1][j2][b], is free of bank conflicts.
//
// Shared-memory Stockham FFTs (any other length N = 2^a 3^b <= 256, and the
// one-time field-tensor setup): a thread block transforms `lines`
// independent sequences held line-major in shared memory, with radix-4,
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

// Stockham transform of `lines` sequences of length N stored line-major in a; b is a
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

template <class R>
__global__ void __launch_bounds__(kBlock) fft_strided(cx<R>* __restrict__ data, StridedPass g,
                                                      const cx<R>* __restrict__ W, int sign,
                                                      const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (st != nullptr && (st->poll.done || st->half || st->skip_mv)) return;
  extern __shared__ unsigned char smem_raw[];
  const int n = g.n, ls = g.n, bl = g.bl;
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
  const cx<R>* res = block_fft<R>(buf0, buf1, n, bl, W, sign);
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

// ---------------------------------------------------------------------------
// Register FFTs.

// cos(2 pi i / 48): the twiddles of every register DFT length (N | 48).
__host__ __device__ constexpr double cos48(int i) {
  i = ((i % 48) + 48) % 48;
  if (i > 24) i = 48 - i;  // even
  const bool neg = i > 12;
  if (neg) i = 24 - i;     // cos(pi - t) = -cos(t)
  double c = 0.0;
  switch (i) {
    case 0: c = 1.0; break;
    case 1: c = 0.991444861373810411145; break;
    case 2: c = 0.96592582628906828675; break;
    case 3: c = 0.923879532511286756128; break;
    case 4: c = 0.866025403784438646764; break;
    case 5: c = 0.79335334029123516458; break;
    case 6: c = 0.707106781186547524401; break;
    case 7: c = 0.608761429008720639416; break;
    case 8: c = 0.5; break;
    case 9: c = 0.382683432365089771728; break;
    case 10: c = 0.258819045102520762349; break;
    case 11: c = 0.130526192220051591548; break;
    default: c = 0.0; break;
  }
  return neg ? -c : c;
}

// v * exp(SIGN 2 pi i m / N), N | 48; m is a constant once loops unroll.
template <int N, int SIGN, class R> __device__ __forceinline__ cx<R> wmul(cx<R> v, int m) {
  m %= N;
  if (m == 0) return v;
  if ((4 * m) % N == 0) {  // quarter turns: -1 or +-i
    const int q = 4 * m / N;
    if (q == 2) return mk<R>(-v.x, -v.y);
    return mul_i(v, q == 1 ? SIGN : -SIGN);
  }
  const int i48 = m * (48 / N);
  const R c = (R)cos48(i48), s = (R)(SIGN * cos48(i48 - 12));
  return mk<R>(v.x * c - v.y * s, v.x * s + v.y * c);
}

// In-place DFT of v[0..N) in registers, sign SIGN (-1 forward).
template <int N, int SIGN, class R> __device__ __forceinline__ void dft(cx<R> (&v)[N]) {
  if constexpr (N == 2) {
    const cx<R> a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if constexpr (N == 3) {
    const R h = (R)0.866025403784438646764;  // sqrt(3)/2
    const cx<R> s = cadd(v[1], v[2]);
    const cx<R> m = cscale(h, mul_i(csub(v[1], v[2]), SIGN));
    const cx<R> base = csub(v[0], cscale((R)0.5, s));
    v[0] = cadd(v[0], s);
    v[1] = cadd(base, m);
    v[2] = csub(base, m);
  } else if constexpr (N == 4) {
    const cx<R> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const cx<R> c = cadd(v[1], v[3]), d = mul_i(csub(v[1], v[3]), SIGN);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  } else if constexpr (N > 4) {
    // N = P Q: P-point DFTs over j1 (stride Q), twiddles, Q-point DFTs
    constexpr int P = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
    constexpr int Q = N / P;
    static_assert(48 % N == 0, "register DFT lengths divide 48");
    cx<R> t[N];
#pragma unroll
    for (int j2 = 0; j2 < Q; ++j2) {
      cx<R> u[P];
#pragma unroll
      for (int j1 = 0; j1 < P; ++j1) u[j1] = v[Q * j1 + j2];
      dft<P, SIGN, R>(u);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) t[k1 * Q + j2] = wmul<N, SIGN, R>(u[k1], j2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      cx<R> w[Q];
#pragma unroll
      for (int j2 = 0; j2 < Q; ++j2) w[j2] = t[k1 * Q + j2];
      dft<Q, SIGN, R>(w);
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = w[k2];
    }
  }
}

// Line lengths with a register transform: N = N1 N2.
template <int N> struct Fac { static constexpr int N1 = 0, N2 = 0; };
template <> struct Fac<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Fac<24> { static constexpr int N1 = 6, N2 = 4; };
template <> struct Fac<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Fac<48> { static constexpr int N1 = 8, N2 = 6; };
template <> struct Fac<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Fac<96> { static constexpr int N1 = 12, N2 = 8; };
template <> struct Fac<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Fac<192> { static constexpr int N1 = 16, N2 = 12; };
template <> struct Fac<256> { static constexpr int N1 = 16, N2 = 16; };

// Twiddle W_N^m of the line transform (m < N) from the table W[t] =
// exp(-2 pi i t / N), conjugated for SIGN > 0.
template <int SIGN, class R> __device__ __forceinline__ cx<R> line_tw(const cx<R>* __restrict__ W, int m) {
  const cx<R> w = __ldg(&W[m]);
  return SIGN > 0 ? cconj(w) : w;
}

// Block-wide transform of BL lines of length N (every thread must call it).
// load(j, b) returns input j of line b; inputs j >= IN are zero and not
// loaded.  store(k, b, v) receives output k of line b for k < OUT.  E is a
// shared buffer of N * BL elements.  load may read, and store may write,
// shared or global memory: every load happens before the block barrier
// that precedes the first store.  W is the twiddle table of a length
// TW * N (entry TW t is W_N^t), so a transform of a divisor of the line
// length can use that line's table.
template <class R, int N, int BL, int SIGN, int IN, int OUT, int TW = 1, class Load, class Store>
__device__ __forceinline__ void fft2(const Load& load, const Store& store, cx<R>* E, const cx<R>* __restrict__ W) {
  constexpr int N1 = Fac<N>::N1, N2 = Fac<N>::N2;
  static_assert(N1 * N2 == N, "no register factorisation for this length");
  constexpr int J1 = IN % N2 == 0 ? IN / N2 : N1;    // j1 bound when IN is a multiple of N2
  constexpr int K2 = OUT % N1 == 0 ? OUT / N1 : N2;  // k2 bound when OUT is a multiple of N1
#pragma unroll 1
  for (int t = threadIdx.x; t < BL * N2; t += kBlock) {
    const int b = t % BL, j2 = t / BL;
    cx<R> u[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int j = N2 * j1 + j2;
      u[j1] = (j1 < J1 && j < IN) ? load(j, b) : mk<R>(0, 0);
    }
    dft<N1, SIGN, R>(u);
    E[j2 * BL + b] = u[0];
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) E[(k1 * N2 + j2) * BL + b] = cmul(u[k1], line_tw<SIGN, R>(W, TW * j2 * k1));
  }
  __syncthreads();
#pragma unroll 1
  for (int t = threadIdx.x; t < BL * N1; t += kBlock) {
    const int b = t % BL, k1 = t / BL;
    cx<R> w[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) w[j2] = E[(k1 * N2 + j2) * BL + b];
    dft<N2, SIGN, R>(w);
#pragma unroll
    for (int k2 = 0; k2 < K2; ++k2) {
      const int k = k1 + N1 * k2;
      if (k < OUT) store(k, b, w[k2]);
    }
  }
}

// Strided pass with the register transform: lines of length N at stride
// g.s_j, g.bl = BL consecutive lines (along c) per block; the input is zero
// beyond IN and outputs beyond OUT are not stored.
template <class R, int N, int BL, int SIGN, int IN, int OUT>
__global__ void __launch_bounds__(kBlock) fft_strided_reg(cx<R>* __restrict__ data, StridedPass g,
                                                          const cx<R>* __restrict__ W,
                                                          const SolveState* __restrict__ st) {
  pdl_wait();
  pdl_launch();
  if (st != nullptr && (st->poll.done || st->half || st->skip_mv)) return;
  extern __shared__ unsigned char smem_raw[];
  cx<R>* E = reinterpret_cast<cx<R>*>(smem_raw);
  const int cblocks = (g.nc + BL - 1) / BL;
  const int a = blockIdx.x / cblocks;
  const int c0 = (blockIdx.x - a * cblocks) * BL;
  const int nb = min(BL, g.nc - c0);
  cx<R>* base = data + (int64_t)blockIdx.y * g.comp_stride + (int64_t)a * g.s_a + c0;
  const int64_t sj = g.s_j;
  auto load = [&](int j, int b) { return b < nb ? base[(int64_t)j * sj + b] : mk<R>(0, 0); };
  auto store = [&](int k, int b, cx<R> v) {
    if (b < nb) base[(int64_t)k * sj + b] = v;
  };
  fft2<R, N, BL, SIGN, IN, OUT>(load, store, E, W);
}

}  // namespace ccg
