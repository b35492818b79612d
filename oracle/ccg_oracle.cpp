// CPU oracle for the complex Krylov solvers of CCGPAK 2.0 (Flatau 2012).
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plainly written reference
// that the GPU library is checked against.  Only the test suite, the smoke
// check and the benchmark's CPU-baseline leg load it; the solver library
// never does, and it shares no code, header or constant with the CUDA path.
//
// The manual (Sec. 1) states the problem only: solve A x = y for complex A,
// unknown x and known right-hand side y, with the matrix-vector products A x
// and A^H x supplied apart from the iteration (Sec. 5, `matvec`/`cmatvec`),
// tolerance `epsilon_err` and iteration cap `maxit` (Sec. 5, `cgmodule`), in
// single or double precision (abstract, Sec. 5 `ddprecision`).  It prints
// no recurrences, so each method below is the unpreconditioned textbook form
// of the source the manual names for it (Sec. 2.1 PIM: BiCGSTAB, CGNR, QMR,
// BiCG (`bigcg`), restarted GMRES (`rgmres`), CGS, CGNE, TFQMR; Sec. 2.2 Sarkar:
// the complex-symmetric CG; Sec. 3.1: BiCGstab(l); Sec. 3.4: COCR of Sogabe
// and Zhang).  Readings where the manual is silent:
//   * stopping rule: ||r_k||_2 / ||y||_2 <= tol on the recurrence residual;
//   * shadow vectors (BiCGSTAB r^, QMR w~_1, BiCG r~_0, CGS r^) equal r_0;
//   * CGNE is Craig's method: CG on A A^H u = y with x = A^H u, residual
//     r = y - A x;
//   * TFQMR (Freund): an iteration is its two half-steps (two products); it
//     keeps no residual vector, so its recorded residual and stopping test
//     use the bound ||r_{m+1}|| <= sqrt(m + 2) tau_{m+1} after half-step m,
//     tested after every half-step (an exit after the first half counts as
//     the iteration); shadow r^ = r_0;
//   * BiCGstab(l) is the vanilla algorithm of Sleijpen and Fokkema (the base
//     form of Fokkema's thesis, Sec. 3.1), without the two enhancements the
//     manual names; an iteration is one cycle of l BiCG steps and the
//     l-dimensional minimal-residual update (2 l products); the residual
//     r^_0 is tested after every BiCG step (an exit there counts as the
//     iteration) and at the cycle end; l (default 2) is a parameter;
//   * complex BiCG pairs A with A^H and conjugated products (the shadow
//     recurrences take conj(alpha), conj(beta));
//   * COCR uses the unconjugated form like COCG and needs A = A^T;
//   * GMRES(m): an iteration is one Arnoldi step (one product); its residual
//     is the least-squares residual |g_{j+1}| the Givens rotations give,
//     the true residual of the cycle's minimiser; x is formed at the end of
//     a cycle (m steps, convergence or the cap), and a cycle restarts from
//     r = y - A x, stopping at once if that residual meets tol; the restart
//     length m (default 30) is a parameter;
//   * BiCGSTAB exits at the half step when ||s|| meets tol (one iteration);
//   * complex QMR uses A^H and conjugated products (the real bilinear form
//     with A^T carried to conjugated vectors);
//   * "Sarkar-style" complex CG = CG with the unconjugated bilinear form
//     [u, v] = sum u_i v_i (COCG), valid for A = A^T;
//   * dot products accumulate in double at both precisions; matrix-vector
//     products accumulate in the working precision;
//   * breakdown when a divisor's modulus is below 1e-300 (double) or 1e-37
//     (single).
//
// The dipole operator (Sec. 1: the DDSCAT application) is not defined by the
// manual; it is the standard discrete-dipole system
//     (A p)_i = p_i / alpha - sum_{j != i} G(r_i - r_j) p_j
// on the occupied sites of a cubic lattice with unit spacing, G the free-space
// field tensor of an oscillating point dipole (Gaussian units, exp(-i w t)):
//     G(r) = exp(ikr)/r^3 [ (kr)^2 (I - u u^T) + (1 - ikr)(3 u u^T - I) ],
// u = r/|r|, and the Clausius-Mossotti polarizability
//     alpha = (3 / 4 pi) (m^2 - 1) / (m^2 + 2).
// Its direct O(N^2) sum is the definition; the FFT form embeds G in a
// circulant of twice the lattice size and applies it with a plain recursive
// mixed-radix FFT written here (used only where the direct sum is too slow).

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <memory>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

template <class R> using C = std::complex<R>;
using Z = std::complex<double>;

enum Status { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_BREAKDOWN = 2, ORC_INVALID = -1 };
enum Method { ORC_BICGSTAB = 0, ORC_CGNR = 1, ORC_QMR = 2, ORC_COCG = 3, ORC_COCR = 4, ORC_BICG = 5, ORC_GMRES = 6,
              ORC_CGS = 7, ORC_CGNE = 8, ORC_TFQMR = 9, ORC_BICGSTABL = 10 };
// Which scalar vanished when a method breaks down.
enum Breakdown { BD_NONE = 0, BD_RHO = 1, BD_SIGMA = 2, BD_TT = 3, BD_OMEGA = 4, BD_GAMMA = 5,
                 BD_WW = 6, BD_XI = 7, BD_DELTA = 8, BD_EPS = 9, BD_BETA = 10, BD_MU = 11, BD_HESS = 12 };

// Restart length of GMRES(m) and degree l of BiCGstab(l), set through
// orc_set_restart and orc_set_bicgstab_l.
int g_restart = 30;
int g_bicgstab_l = 2;

template <class R> double guard();
template <> double guard<double>() { return 1e-300; }
template <> double guard<float>() { return 1e-37; }

template <class R> bool tiny(Z s) { return std::abs(s) < guard<R>(); }
template <class R> bool tiny(double s) { return std::fabs(s) < guard<R>(); }

// ----------------------------------------------------------------------------
// Vector primitives.  Dot products and norms accumulate in double.
// ----------------------------------------------------------------------------
template <class R> Z dotc(int64_t n, const C<R>* u, const C<R>* v) {   // <u,v> = sum conj(u_i) v_i
  Z s = 0;
  for (int64_t i = 0; i < n; ++i) s += std::conj(Z(u[i])) * Z(v[i]);
  return s;
}
template <class R> Z dotu(int64_t n, const C<R>* u, const C<R>* v) {   // [u,v] = sum u_i v_i
  Z s = 0;
  for (int64_t i = 0; i < n; ++i) s += Z(u[i]) * Z(v[i]);
  return s;
}
template <class R> double nrm2(int64_t n, const C<R>* u) {
  double s = 0;
  for (int64_t i = 0; i < n; ++i) s += std::norm(Z(u[i]));
  return std::sqrt(s);
}

// ----------------------------------------------------------------------------
// Operators: y = A x and y = A^H x (the manual's matvec / cmatvec, Sec. 5).
// ----------------------------------------------------------------------------
template <class R> struct Operator {
  int64_t n = 0;
  bool symmetric = false;   // A = A^T
  virtual ~Operator() {}
  virtual void apply(const C<R>* x, C<R>* y) const = 0;
  virtual void apply_h(const C<R>* x, C<R>* y) const = 0;
};

// Dense row-major A with leading dimension lda; plain double loops.  Each
// output element is one sum taken in index order (j for A x, i for A^H x).
// The OpenMP build (liboracle_omp.so, the all-core CPU baseline) only hands
// independent output elements to different threads -- rows of A x, blocks
// of columns of A^H x -- so every sum keeps its order and both builds give
// bit-identical results; the plain build ignores the pragmas.
template <class R> struct Dense : Operator<R> {
  const C<R>* A;
  int64_t lda;
  Dense(int64_t n_, const C<R>* A_, int64_t lda_) : A(A_), lda(lda_) { this->n = n_; }
  void apply(const C<R>* x, C<R>* y) const override {
    const int64_t n = this->n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      C<R> acc = 0;
      for (int64_t j = 0; j < n; ++j) acc += A[i * lda + j] * x[j];
      y[i] = acc;
    }
  }
  void apply_h(const C<R>* x, C<R>* y) const override {
    const int64_t n = this->n, cb = 256;
#pragma omp parallel for schedule(static)
    for (int64_t j0 = 0; j0 < n; j0 += cb) {
      const int64_t j1 = j0 + cb < n ? j0 + cb : n;
      for (int64_t j = j0; j < j1; ++j) y[j] = 0;
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = j0; j < j1; ++j) y[j] += std::conj(A[i * lda + j]) * x[i];
    }
  }
};

// ----------------------------------------------------------------------------
// Plain recursive mixed-radix FFT (decimation in time by the smallest prime
// factor; a direct DFT when the length is prime).  sign = -1 forward,
// +1 inverse (unnormalised).
// ----------------------------------------------------------------------------
void fft_rec(const Z* in, int64_t n, int64_t stride, Z* out, int sign) {
  if (n == 1) { out[0] = in[0]; return; }
  int64_t p = 2;
  while (p * p <= n && n % p) ++p;
  if (n % p) p = n;                       // n is prime
  const int64_t m = n / p;
  if (m == 1) {                           // direct DFT of prime length p
    for (int64_t k = 0; k < n; ++k) {
      Z s = 0;
      for (int64_t j = 0; j < n; ++j) {
        const double ang = sign * 2.0 * M_PI * double((j * k) % n) / double(n);
        s += in[j * stride] * std::polar(1.0, ang);
      }
      out[k] = s;
    }
    return;
  }
  // F_q[k'] = FFT_m of the subsequence in[(p*j + q)], q = 0..p-1.
  std::vector<Z> sub(n);
  for (int64_t q = 0; q < p; ++q) fft_rec(in + q * stride, m, stride * p, sub.data() + q * m, sign);
  // X[k] = sum_q W_n^{q k} F_q[k mod m]
  for (int64_t k = 0; k < n; ++k) {
    Z s = 0;
    for (int64_t q = 0; q < p; ++q) {
      const double ang = sign * 2.0 * M_PI * double((q * k) % n) / double(n);
      s += std::polar(1.0, ang) * sub[q * m + (k % m)];
    }
    out[k] = s;
  }
}

void fft1d(Z* a, int64_t n, int64_t stride, int sign) {
  std::vector<Z> in(n), out(n);
  for (int64_t j = 0; j < n; ++j) in[j] = a[j * stride];
  fft_rec(in.data(), n, 1, out.data(), sign);
  for (int64_t j = 0; j < n; ++j) a[j * stride] = out[j];
}

// 3D transform of g[(a*n1 + b)*n2 + c], each axis in turn.
void fft3d(Z* g, int64_t n0, int64_t n1, int64_t n2, int sign) {
  for (int64_t a = 0; a < n0; ++a)
    for (int64_t b = 0; b < n1; ++b) fft1d(g + (a * n1 + b) * n2, n2, 1, sign);
  for (int64_t a = 0; a < n0; ++a)
    for (int64_t c = 0; c < n2; ++c) fft1d(g + a * n1 * n2 + c, n1, n2, sign);
  for (int64_t b = 0; b < n1; ++b)
    for (int64_t c = 0; c < n2; ++c) fft1d(g + b * n2 + c, n0, n1 * n2, sign);
}

// ----------------------------------------------------------------------------
// Discrete-dipole operator.
// ----------------------------------------------------------------------------
// Field tensor of a point dipole at displacement (dx,dy,dz), unit spacing,
// wavenumber k.  Components in the order xx, xy, xz, yy, yz, zz.
void green(double k, double dx, double dy, double dz, Z G[6]) {
  const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
  const double u[3] = {dx / r, dy / r, dz / r};
  const Z ikr(0.0, k * r);
  const Z e = std::exp(ikr) / (r * r * r);
  const Z a = (k * r) * (k * r);     // multiplies (I - u u^T)
  const Z b = 1.0 - ikr;             // multiplies (3 u u^T - I)
  const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int c = 0; c < 6; ++c) {
    const double uu = u[ia[c]] * u[ib[c]];
    const double d = ia[c] == ib[c] ? 1.0 : 0.0;
    G[c] = e * (a * (d - uu) + b * (3.0 * uu - d));
  }
}

// Index of the symmetric component (a,b) in the xx,xy,xz,yy,yz,zz order.
int sym_index(int a, int b) {
  static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return t[a][b];
}

struct DipoleCore {
  int nx, ny, nz;
  int64_t N;                         // occupied sites
  std::vector<int> si, sj, sl;       // site coordinates, lexicographic with l fastest
  double k;
  Z alpha, alpha_inv;
  bool use_fft;
  int64_t M0, M1, M2;                // FFT grid 2nx x 2ny x 2nz
  std::vector<Z> Ghat[6];

  DipoleCore(int nx_, int ny_, int nz_, const uint8_t* occ, double kd, Z m, bool fft)
      : nx(nx_), ny(ny_), nz(nz_), k(kd), use_fft(fft) {
    for (int i = 0; i < nx; ++i)
      for (int j = 0; j < ny; ++j)
        for (int l = 0; l < nz; ++l)
          if (occ[(int64_t(i) * ny + j) * nz + l]) { si.push_back(i); sj.push_back(j); sl.push_back(l); }
    N = int64_t(si.size());
    const Z m2 = m * m;
    alpha = (3.0 / (4.0 * M_PI)) * (m2 - 1.0) / (m2 + 2.0);
    alpha_inv = 1.0 / alpha;
    M0 = 2 * nx; M1 = 2 * ny; M2 = 2 * nz;
    if (use_fft) build_ghat();
  }

  // Circulant embedding: grid index q in [0, n) is displacement q, q in (n, 2n)
  // is displacement q - 2n, and q = n (a displacement no pair of sites has) and
  // the zero displacement carry the zero tensor.
  void build_ghat() {
    const int64_t G = M0 * M1 * M2;
    for (int c = 0; c < 6; ++c) Ghat[c].assign(G, Z(0));
    for (int64_t a = 0; a < M0; ++a)
      for (int64_t b = 0; b < M1; ++b)
        for (int64_t c = 0; c < M2; ++c) {
          if (a == nx || b == ny || c == nz) continue;
          const double dx = a < nx ? a : a - M0, dy = b < ny ? b : b - M1, dz = c < nz ? c : c - M2;
          if (dx == 0 && dy == 0 && dz == 0) continue;
          Z g[6];
          green(k, dx, dy, dz, g);
          for (int q = 0; q < 6; ++q) Ghat[q][(a * M1 + b) * M2 + c] = g[q];
        }
    for (int q = 0; q < 6; ++q) fft3d(Ghat[q].data(), M0, M1, M2, -1);
  }

  // y_a(s) = x_a(s)/alpha - sum_{t != s} sum_b G_ab(r_s - r_t) x_b(t)  for the
  // listed output sites; x and y in the site-fastest layout v[a*N + s].
  void direct_rows(const Z* x, Z* y, int64_t nsel, const int64_t* sel) const {
    for (int64_t q = 0; q < nsel; ++q) {
      const int64_t s = sel ? sel[q] : q;
      Z acc[3] = {0, 0, 0};
      for (int64_t t = 0; t < N; ++t) {
        if (t == s) continue;
        Z g[6];
        green(k, si[s] - si[t], sj[s] - sj[t], sl[s] - sl[t], g);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc[a] += g[sym_index(a, b)] * x[b * N + t];
      }
      for (int a = 0; a < 3; ++a) y[a * N + q] = alpha_inv * x[a * N + s] - acc[a];
    }
  }

  void fft_apply(const Z* x, Z* y) const {
    const int64_t G = M0 * M1 * M2;
    std::vector<Z> X[3], Y(G);
    for (int b = 0; b < 3; ++b) {
      X[b].assign(G, Z(0));
      for (int64_t s = 0; s < N; ++s) X[b][(int64_t(si[s]) * M1 + sj[s]) * M2 + sl[s]] = x[b * N + s];
      fft3d(X[b].data(), M0, M1, M2, -1);
    }
    for (int a = 0; a < 3; ++a) {
      for (int64_t g = 0; g < G; ++g) {
        Z s = 0;
        for (int b = 0; b < 3; ++b) s += Ghat[sym_index(a, b)][g] * X[b][g];
        Y[g] = s;
      }
      fft3d(Y.data(), M0, M1, M2, +1);
      for (int64_t s = 0; s < N; ++s)
        y[a * N + s] = alpha_inv * x[a * N + s] - Y[(int64_t(si[s]) * M1 + sj[s]) * M2 + sl[s]] / double(G);
    }
  }

  void apply(const Z* x, Z* y) const {
    if (use_fft) fft_apply(x, y);
    else direct_rows(x, y, N, nullptr);
  }
};

// Precision adapter: the dipole arithmetic is carried out in double and the
// result rounded to the working precision.  A is complex symmetric, so
// A^H x = conj(A conj(x)).
template <class R> struct Dipole : Operator<R> {
  std::shared_ptr<DipoleCore> core;
  explicit Dipole(std::shared_ptr<DipoleCore> c) : core(c) { this->n = 3 * c->N; this->symmetric = true; }
  void apply(const C<R>* x, C<R>* y) const override {
    std::vector<Z> xd(this->n), yd(this->n);
    for (int64_t i = 0; i < this->n; ++i) xd[i] = Z(x[i]);
    core->apply(xd.data(), yd.data());
    for (int64_t i = 0; i < this->n; ++i) y[i] = C<R>(yd[i]);
  }
  void apply_h(const C<R>* x, C<R>* y) const override {
    std::vector<Z> xd(this->n), yd(this->n);
    for (int64_t i = 0; i < this->n; ++i) xd[i] = std::conj(Z(x[i]));
    core->apply(xd.data(), yd.data());
    for (int64_t i = 0; i < this->n; ++i) y[i] = C<R>(std::conj(yd[i]));
  }
};

// ----------------------------------------------------------------------------
// Solvers.  Each returns the number of completed iterations and writes
// hist[k] = ||r_k|| / ||y|| for k = 0..iters.  x holds x_0 on entry.
// ----------------------------------------------------------------------------
struct Result { int iters; int status; int detail; };

// Common start: r = y - A x0.  Returns ||y||; y = 0 gives x = 0.
template <class R> double start(const Operator<R>& A, const C<R>* y, C<R>* x, C<R>* r) {
  const int64_t n = A.n;
  const double ynorm = nrm2(n, y);
  if (ynorm == 0) {
    for (int64_t i = 0; i < n; ++i) { x[i] = 0; r[i] = 0; }
    return 0;
  }
  A.apply(x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = y[i] - r[i];
  return ynorm;
}

// BiCGSTAB (van der Vorst 1992; PIM's `bicgstab`, manual Sec. 2.1).
template <class R>
Result bicgstab(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), rh(n), p(n), v(n), s(n), t(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  rh = r;
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  Z rho_old = 1, alpha = 1, omega = 1;
  for (int k = 1; k <= maxit; ++k) {
    const Z rho = dotc(n, rh.data(), r.data());
    if (tiny<R>(rho)) return {k - 1, ORC_BREAKDOWN, BD_RHO};
    if (k == 1) {
      p = r;
    } else {
      const C<R> beta = C<R>((rho / rho_old) * (alpha / omega)), om = C<R>(omega);
      for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - om * v[i]);
    }
    A.apply(p.data(), v.data());
    const Z sigma = dotc(n, rh.data(), v.data());
    if (tiny<R>(sigma)) return {k - 1, ORC_BREAKDOWN, BD_SIGMA};
    alpha = rho / sigma;
    const C<R> al = C<R>(alpha);
    for (int64_t i = 0; i < n; ++i) s[i] = r[i] - al * v[i];
    const double snorm = nrm2(n, s.data()) / ynorm;
    if (snorm <= tol) {                         // half-step exit counts as iteration k
      for (int64_t i = 0; i < n; ++i) x[i] += al * p[i];
      hist[k] = snorm;
      return {k, ORC_OK, BD_NONE};
    }
    A.apply(s.data(), t.data());
    const double tt = dotc(n, t.data(), t.data()).real();
    if (tiny<R>(tt)) return {k - 1, ORC_BREAKDOWN, BD_TT};
    omega = dotc(n, t.data(), s.data()) / tt;
    const C<R> om = C<R>(omega);
    for (int64_t i = 0; i < n; ++i) {
      x[i] += al * p[i] + om * s[i];
      r[i] = s[i] - om * t[i];
    }
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    if (tiny<R>(omega)) return {k, ORC_BREAKDOWN, BD_OMEGA};
    rho_old = rho;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// CGNR: CG on the normal equations A^H A x = A^H y (PIM's `cgnr`, Sec. 2.1).
// The residual tracked and tested is r = y - A x.
template <class R>
Result cgnr(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), z(n), p(n), w(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  A.apply_h(r.data(), z.data());
  p = z;
  double gamma = dotc(n, z.data(), z.data()).real();
  for (int k = 1; k <= maxit; ++k) {
    if (tiny<R>(gamma)) return {k - 1, ORC_BREAKDOWN, BD_GAMMA};
    A.apply(p.data(), w.data());
    const double ww = dotc(n, w.data(), w.data()).real();
    if (tiny<R>(ww)) return {k - 1, ORC_BREAKDOWN, BD_WW};
    const R al = R(gamma / ww);
    for (int64_t i = 0; i < n; ++i) {
      x[i] += al * p[i];
      r[i] -= al * w[i];
    }
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    A.apply_h(r.data(), z.data());
    const double gamma_new = dotc(n, z.data(), z.data()).real();
    const R be = R(gamma_new / gamma);
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
    gamma = gamma_new;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// QMR without look-ahead, coupled two-term recurrences (Freund & Nachtigal;
// PIM's `qmr`, Sec. 2.1), unpreconditioned, complex form with A^H.
// tau (optional) receives the quasi-residual norms tau_0 = rho_1,
// tau_i = tau_{i-1} theta_i gamma_i, for which ||r_i|| <= sqrt(i+1) tau_i.
template <class R>
Result qmr(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist, double* tau) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), vt(n), wt(n), v(n), w(n), p(n), q(n), pt(n), u(n), d(n), s(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; if (tau) tau[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  vt = r;
  wt = r;
  double rho = nrm2(n, vt.data()), xi = nrm2(n, wt.data());
  double gamma_prev = 1.0, theta_prev = 0.0;
  Z eta = -1.0, eps = 0.0;
  if (tau) tau[0] = rho;
  for (int i = 1; i <= maxit; ++i) {
    if (tiny<R>(rho)) return {i - 1, ORC_BREAKDOWN, BD_RHO};
    if (tiny<R>(xi)) return {i - 1, ORC_BREAKDOWN, BD_XI};
    const R rinv = R(1.0 / rho), xinv = R(1.0 / xi);
    for (int64_t j = 0; j < n; ++j) { v[j] = vt[j] * rinv; w[j] = wt[j] * xinv; }
    const Z delta = dotc(n, w.data(), v.data());
    if (tiny<R>(delta)) return {i - 1, ORC_BREAKDOWN, BD_DELTA};
    if (i == 1) {
      p = v;
      q = w;
    } else {
      const C<R> cp = C<R>(xi * delta / eps), cq = C<R>(std::conj(rho * delta / eps));
      for (int64_t j = 0; j < n; ++j) { p[j] = v[j] - cp * p[j]; q[j] = w[j] - cq * q[j]; }
    }
    A.apply(p.data(), pt.data());
    A.apply_h(q.data(), u.data());
    eps = dotc(n, q.data(), pt.data());
    if (tiny<R>(eps)) return {i - 1, ORC_BREAKDOWN, BD_EPS};
    const Z beta = eps / delta;
    if (tiny<R>(beta)) return {i - 1, ORC_BREAKDOWN, BD_BETA};
    const C<R> be = C<R>(beta), bc = C<R>(std::conj(beta));
    for (int64_t j = 0; j < n; ++j) { vt[j] = pt[j] - be * v[j]; wt[j] = u[j] - bc * w[j]; }
    const double rho_next = nrm2(n, vt.data()), xi_next = nrm2(n, wt.data());
    const double theta = rho_next / (gamma_prev * std::abs(beta));
    const double gamma = 1.0 / std::sqrt(1.0 + theta * theta);
    if (tiny<R>(gamma)) return {i - 1, ORC_BREAKDOWN, BD_GAMMA};
    eta = -eta * rho * gamma * gamma / (beta * gamma_prev * gamma_prev);
    const C<R> et = C<R>(eta);
    if (i == 1) {
      for (int64_t j = 0; j < n; ++j) { d[j] = et * p[j]; s[j] = et * pt[j]; }
    } else {
      const R c = R((theta_prev * gamma) * (theta_prev * gamma));
      for (int64_t j = 0; j < n; ++j) { d[j] = et * p[j] + c * d[j]; s[j] = et * pt[j] + c * s[j]; }
    }
    for (int64_t j = 0; j < n; ++j) { x[j] += d[j]; r[j] -= s[j]; }
    hist[i] = nrm2(n, r.data()) / ynorm;
    if (tau) tau[i] = tau[i - 1] * theta * gamma;
    if (hist[i] <= tol) return {i, ORC_OK, BD_NONE};
    rho = rho_next;
    xi = xi_next;
    gamma_prev = gamma;
    theta_prev = theta;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// Complex-symmetric CG with the unconjugated form (COCG; the manual's Sarkar
// family, Sec. 2.2).  Requires A = A^T.
template <class R>
Result cocg(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), p(n), q(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  p = r;
  Z rho = dotu(n, r.data(), r.data());
  for (int k = 1; k <= maxit; ++k) {
    if (tiny<R>(rho)) return {k - 1, ORC_BREAKDOWN, BD_RHO};
    A.apply(p.data(), q.data());
    const Z mu = dotu(n, p.data(), q.data());
    if (tiny<R>(mu)) return {k - 1, ORC_BREAKDOWN, BD_MU};
    const C<R> al = C<R>(rho / mu);
    for (int64_t i = 0; i < n; ++i) { x[i] += al * p[i]; r[i] -= al * q[i]; }
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    const Z rho_new = dotu(n, r.data(), r.data());
    const C<R> be = C<R>(rho_new / rho);
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + be * p[i];
    rho = rho_new;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// COCR: conjugate A-orthogonal conjugate residual (Sogabe & Zhang 2007; the
// manual's Sec. 3.4), unconjugated form, one product A r per iteration with
// q = A p carried by recurrence.  Requires A = A^T.
template <class R>
Result cocr(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), p(n), q(n), w(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  A.apply(r.data(), w.data());  // w = A r
  p = r;
  q = w;                        // q = A p
  Z rho = dotu(n, r.data(), w.data());
  for (int k = 1; k <= maxit; ++k) {
    if (tiny<R>(rho)) return {k - 1, ORC_BREAKDOWN, BD_RHO};
    const Z mu = dotu(n, q.data(), q.data());
    if (tiny<R>(mu)) return {k - 1, ORC_BREAKDOWN, BD_MU};
    const C<R> al = C<R>(rho / mu);
    for (int64_t i = 0; i < n; ++i) { x[i] += al * p[i]; r[i] -= al * q[i]; }
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    A.apply(r.data(), w.data());
    const Z rho_new = dotu(n, r.data(), w.data());
    const C<R> be = C<R>(rho_new / rho);
    for (int64_t i = 0; i < n; ++i) { p[i] = r[i] + be * p[i]; q[i] = w[i] + be * q[i]; }
    rho = rho_new;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// BiCG (Fletcher; PIM's `bigcg`, Sec. 2.1), complex form: the shadow
// system runs with A^H, products are conjugated, shadow r~_0 = r_0.
template <class R>
Result bicg(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), rt(n), p(n), pt(n), q(n), qt(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  rt = r;
  Z rho = dotc(n, rt.data(), r.data());
  for (int k = 1; k <= maxit; ++k) {
    if (tiny<R>(rho)) return {k - 1, ORC_BREAKDOWN, BD_RHO};
    if (k == 1) {
      p = r;
      pt = rt;
    }
    A.apply(p.data(), q.data());
    A.apply_h(pt.data(), qt.data());
    const Z sigma = dotc(n, pt.data(), q.data());
    if (tiny<R>(sigma)) return {k - 1, ORC_BREAKDOWN, BD_SIGMA};
    const Z alpha = rho / sigma;
    const C<R> al = C<R>(alpha), alc = C<R>(std::conj(alpha));
    for (int64_t i = 0; i < n; ++i) {
      x[i] += al * p[i];
      r[i] -= al * q[i];
      rt[i] -= alc * qt[i];
    }
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    const Z rho_new = dotc(n, rt.data(), r.data());
    const Z beta = rho_new / rho;
    const C<R> be = C<R>(beta), bec = C<R>(std::conj(beta));
    for (int64_t i = 0; i < n; ++i) { p[i] = r[i] + be * p[i]; pt[i] = rt[i] + bec * pt[i]; }
    rho = rho_new;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// CGS (Sonneveld 1989; PIM's `cgs`, Sec. 2.1), complex form with
// conjugated products and shadow r^ = r_0: two products per iteration, the
// BiCG polynomial applied twice.
template <class R>
Result cgs(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), rh(n), u(n), p(n), q(n), v(n), uh(n), qh(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  rh = r;
  Z rho_old = 1.0;
  for (int k = 1; k <= maxit; ++k) {
    const Z rho = dotc(n, rh.data(), r.data());
    if (tiny<R>(rho)) return {k - 1, ORC_BREAKDOWN, BD_RHO};
    if (k == 1) {
      u = r;
      p = u;
    } else {
      const C<R> be = C<R>(rho / rho_old);
      for (int64_t i = 0; i < n; ++i) {
        u[i] = r[i] + be * q[i];
        p[i] = u[i] + be * (q[i] + be * p[i]);
      }
    }
    A.apply(p.data(), v.data());
    const Z sigma = dotc(n, rh.data(), v.data());
    if (tiny<R>(sigma)) return {k - 1, ORC_BREAKDOWN, BD_SIGMA};
    const C<R> al = C<R>(rho / sigma);
    for (int64_t i = 0; i < n; ++i) {
      q[i] = u[i] - al * v[i];
      uh[i] = u[i] + q[i];
      x[i] += al * uh[i];
    }
    A.apply(uh.data(), qh.data());
    for (int64_t i = 0; i < n; ++i) r[i] -= al * qh[i];
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    rho_old = rho;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// CGNE (Craig's method; PIM's `cgne`, Sec. 2.1): CG on A A^H u = y with
// x = A^H u, carried in x directly; the residual is r = y - A x.
template <class R>
Result cgne(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), p(n), w(n), z(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  A.apply_h(r.data(), p.data());
  double gamma = dotc(n, r.data(), r.data()).real();
  for (int k = 1; k <= maxit; ++k) {
    const double pp = dotc(n, p.data(), p.data()).real();
    if (tiny<R>(pp)) return {k - 1, ORC_BREAKDOWN, BD_WW};
    const R al = R(gamma / pp);
    A.apply(p.data(), w.data());
    for (int64_t i = 0; i < n; ++i) {
      x[i] += al * p[i];
      r[i] -= al * w[i];
    }
    hist[k] = nrm2(n, r.data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    const double gamma_new = dotc(n, r.data(), r.data()).real();
    const R be = R(gamma_new / gamma);
    A.apply_h(r.data(), z.data());
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
    gamma = gamma_new;
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// TFQMR (Freund 1993; PIM's `tfqmr`, Sec. 2.1), complex form: two
// half-steps per iteration, w the BiCG-squared residual, d the QMR search
// direction, tau the quasi-residual norm, conjugated products with r^ = r_0.
template <class R>
Result tfqmr(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), w(n), u(n), un(n), v(n), uh(n), d(n), rh(n);
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, r.data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  w = r;
  u = r;
  rh = r;
  A.apply(u.data(), uh.data());  // uh = A u_0
  v = uh;
  double tau = nrm2(n, r.data()), theta = 0.0;
  Z eta = 0.0, alpha = 0.0;
  Z rho = dotc(n, rh.data(), r.data());
  for (int k = 1; k <= maxit; ++k) {
    for (int half = 0; half < 2; ++half) {
      const int m = 2 * (k - 1) + half;
      if (half == 0) {
        const Z sigma = dotc(n, rh.data(), v.data());
        if (tiny<R>(sigma)) return {k - 1, ORC_BREAKDOWN, BD_SIGMA};
        alpha = rho / sigma;
        const C<R> al = C<R>(alpha);
        for (int64_t i = 0; i < n; ++i) un[i] = u[i] - al * v[i];
      }
      const std::vector<C<R>>& um = half == 0 ? u : un;  // u_m; uh holds A u_m
      const C<R> al = C<R>(alpha), f = C<R>(theta * theta / alpha * eta);
      for (int64_t i = 0; i < n; ++i) {
        w[i] -= al * uh[i];
        d[i] = um[i] + f * d[i];
      }
      theta = nrm2(n, w.data()) / tau;
      const double c = 1.0 / std::sqrt(1.0 + theta * theta);
      tau = tau * theta * c;
      eta = c * c * alpha;
      const C<R> et = C<R>(eta);
      for (int64_t i = 0; i < n; ++i) x[i] += et * d[i];
      hist[k] = tau * std::sqrt(m + 2.0) / ynorm;
      if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
      if (half == 0) {
        A.apply(un.data(), uh.data());  // A u_{m+1}
      } else {
        const Z rho_new = dotc(n, rh.data(), w.data());
        if (tiny<R>(rho_new)) return {k, ORC_BREAKDOWN, BD_RHO};
        const C<R> be = C<R>(rho_new / rho), be2 = be * be;
        rho = rho_new;
        for (int64_t i = 0; i < n; ++i) {
          u[i] = w[i] + be * un[i];
          v[i] = be * uh[i] + be2 * v[i];
        }
        A.apply(u.data(), uh.data());   // A u_{m+1}
        for (int64_t i = 0; i < n; ++i) v[i] += uh[i];
      }
    }
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// BiCGstab(l) (Sleijpen & Fokkema 1993, vanilla form; manual Sec. 3.1),
// complex: l BiCG steps on the vectors r^_0..r^_l, u^_0..u^_l, then the
// minimal-residual polynomial of degree l by modified Gram-Schmidt on
// r^_1..r^_l.  Shadow r~ = r_0, <a, b> = sum conj(a_i) b_i.
template <class R>
Result bicgstabl(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist, int L) {
  const int64_t n = A.n;
  std::vector<std::vector<C<R>>> rh(L + 1, std::vector<C<R>>(n)), uh(L + 1, std::vector<C<R>>(n));
  std::vector<C<R>> rt(n);
  const double ynorm = start(A, y, x, rh[0].data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  hist[0] = nrm2(n, rh[0].data()) / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  rt = rh[0];
  Z rho0 = 1.0, alpha = 0.0, omega = 1.0;
  std::vector<Z> tau((size_t)(L + 1) * (L + 1)), gp(L + 1), g(L + 1), gpp(L + 1);
  std::vector<double> sigma(L + 1);
  auto T = [&](int i, int j) -> Z& { return tau[(size_t)i * (L + 1) + j]; };
  for (int k = 1; k <= maxit; ++k) {
    rho0 = -omega * rho0;
    for (int j = 0; j < L; ++j) {  // BiCG part
      const Z rho1 = dotc(n, rt.data(), rh[j].data());
      if (tiny<R>(rho0)) return {k - 1, ORC_BREAKDOWN, BD_RHO};
      const C<R> be = C<R>(alpha * rho1 / rho0);
      rho0 = rho1;
      for (int i = 0; i <= j; ++i)
        for (int64_t e = 0; e < n; ++e) uh[i][e] = rh[i][e] - be * uh[i][e];
      A.apply(uh[j].data(), uh[j + 1].data());
      const Z gam = dotc(n, rt.data(), uh[j + 1].data());
      if (tiny<R>(gam)) return {k - 1, ORC_BREAKDOWN, BD_SIGMA};
      alpha = rho0 / gam;
      const C<R> al = C<R>(alpha);
      for (int i = 0; i <= j; ++i)
        for (int64_t e = 0; e < n; ++e) rh[i][e] -= al * uh[i + 1][e];
      for (int64_t e = 0; e < n; ++e) x[e] += al * uh[0][e];
      const double rel = nrm2(n, rh[0].data()) / ynorm;
      if (rel <= tol) {
        hist[k] = rel;
        return {k, ORC_OK, BD_NONE};
      }
      A.apply(rh[j].data(), rh[j + 1].data());
    }
    for (int j = 1; j <= L; ++j) {  // minimal-residual part
      for (int i = 1; i < j; ++i) {
        T(i, j) = dotc(n, rh[i].data(), rh[j].data()) / sigma[i];
        const C<R> t = C<R>(T(i, j));
        for (int64_t e = 0; e < n; ++e) rh[j][e] -= t * rh[i][e];
      }
      sigma[j] = dotc(n, rh[j].data(), rh[j].data()).real();
      if (tiny<R>(sigma[j])) return {k - 1, ORC_BREAKDOWN, BD_MU};
      gp[j] = dotc(n, rh[j].data(), rh[0].data()) / sigma[j];
    }
    g[L] = gp[L];
    omega = g[L];
    for (int j = L - 1; j >= 1; --j) {
      Z t = gp[j];
      for (int i = j + 1; i <= L; ++i) t -= T(j, i) * g[i];
      g[j] = t;
    }
    for (int j = 1; j < L; ++j) {
      Z t = g[j + 1];
      for (int i = j + 1; i < L; ++i) t += T(j, i) * g[i + 1];
      gpp[j] = t;
    }
    {
      const C<R> g1 = C<R>(g[1]), gpl = C<R>(gp[L]), gl = C<R>(g[L]);
      for (int64_t e = 0; e < n; ++e) {
        x[e] += g1 * rh[0][e];
        rh[0][e] -= gpl * rh[L][e];
        uh[0][e] -= gl * uh[L][e];
      }
    }
    for (int j = 1; j < L; ++j) {
      const C<R> gj = C<R>(g[j]), gppj = C<R>(gpp[j]), gpj = C<R>(gp[j]);
      for (int64_t e = 0; e < n; ++e) {
        uh[0][e] -= gj * uh[j][e];
        x[e] += gppj * rh[j][e];
        rh[0][e] -= gpj * rh[j][e];
      }
    }
    hist[k] = nrm2(n, rh[0].data()) / ynorm;
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    if (tiny<R>(omega)) return {k, ORC_BREAKDOWN, BD_OMEGA};
  }
  return {maxit, ORC_NOT_CONVERGED, BD_NONE};
}

// Restarted GMRES(m) (Saad & Schultz 1986; PIM's `rgmres`, Sec. 2.1),
// complex form: Arnoldi with modified Gram-Schmidt in <u, v> = sum conj(u_i)
// v_i, the Hessenberg least-squares problem reduced by complex Givens
// rotations G = [c, s; -conj(s), c] (c real) as columns arrive.
template <class R>
Result gmres(const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist, int m) {
  const int64_t n = A.n;
  std::vector<C<R>> r(n), w(n);
  std::vector<std::vector<C<R>>> V(m + 1, std::vector<C<R>>(n));
  std::vector<Z> H((size_t)(m + 1) * m), g(m + 1), sn(m), yv(m);
  std::vector<double> cs(m);
  auto h = [&](int i, int c) -> Z& { return H[(size_t)i * m + c]; };
  const double ynorm = start(A, y, x, r.data());
  if (ynorm == 0) { hist[0] = 0; return {0, ORC_OK, BD_NONE}; }
  double beta = nrm2(n, r.data());
  hist[0] = beta / ynorm;
  if (hist[0] <= tol) return {0, ORC_OK, BD_NONE};
  int k = 0;
  for (;;) {
    const R binv = R(1.0 / beta);
    for (int64_t e = 0; e < n; ++e) V[0][e] = r[e] * binv;
    std::fill(g.begin(), g.end(), Z(0.0));
    g[0] = beta;
    int cols = 0;
    for (int j = 0; j < m; ++j) {
      ++k;
      A.apply(V[j].data(), w.data());
      for (int i = 0; i <= j; ++i) {
        const Z hij = dotc(n, V[i].data(), w.data());
        h(i, j) = hij;
        const C<R> hc = C<R>(hij);
        for (int64_t e = 0; e < n; ++e) w[e] -= hc * V[i][e];
      }
      const double eta = nrm2(n, w.data());
      for (int i = 0; i < j; ++i) {  // earlier rotations on the new column
        const Z a = h(i, j), b = h(i + 1, j);
        h(i, j) = cs[i] * a + sn[i] * b;
        h(i + 1, j) = -std::conj(sn[i]) * a + cs[i] * b;
      }
      const Z a = h(j, j);
      const double nu = std::sqrt(std::norm(a) + eta * eta);
      if (nu == 0.0) return {k - 1, ORC_BREAKDOWN, BD_HESS};
      if (std::abs(a) == 0.0) {
        cs[j] = 0.0;
        sn[j] = 1.0;
        h(j, j) = eta;
      } else {
        const Z ph = a / std::abs(a);
        cs[j] = std::abs(a) / nu;
        sn[j] = ph * (eta / nu);
        h(j, j) = ph * nu;
      }
      h(j + 1, j) = 0.0;
      g[j + 1] = -std::conj(sn[j]) * g[j];
      g[j] = cs[j] * g[j];
      hist[k] = std::abs(g[j + 1]) / ynorm;
      cols = j + 1;
      if (hist[k] <= tol || k == maxit) break;
      const R einv = R(1.0 / eta);
      for (int64_t e = 0; e < n; ++e) V[j + 1][e] = w[e] * einv;
    }
    for (int i = cols - 1; i >= 0; --i) {  // R y = g by back substitution
      Z t = g[i];
      for (int l = i + 1; l < cols; ++l) t -= h(i, l) * yv[l];
      yv[i] = t / h(i, i);
    }
    for (int i = 0; i < cols; ++i) {
      const C<R> yi = C<R>(yv[i]);
      for (int64_t e = 0; e < n; ++e) x[e] += yi * V[i][e];
    }
    if (hist[k] <= tol) return {k, ORC_OK, BD_NONE};
    if (k == maxit) return {k, ORC_NOT_CONVERGED, BD_NONE};
    A.apply(x, r.data());
    for (int64_t e = 0; e < n; ++e) r[e] = y[e] - r[e];
    beta = nrm2(n, r.data());
    if (beta / ynorm <= tol) return {k, ORC_OK, BD_NONE};
  }
}

template <class R>
Result solve(int method, const Operator<R>& A, const C<R>* y, C<R>* x, double tol, int maxit, double* hist,
             double* tau) {
  switch (method) {
    case ORC_BICGSTAB: return bicgstab(A, y, x, tol, maxit, hist);
    case ORC_CGNR: return cgnr(A, y, x, tol, maxit, hist);
    case ORC_QMR: return qmr(A, y, x, tol, maxit, hist, tau);
    case ORC_COCG:
      if (!A.symmetric) return {0, ORC_INVALID, BD_NONE};
      return cocg(A, y, x, tol, maxit, hist);
    case ORC_COCR:
      if (!A.symmetric) return {0, ORC_INVALID, BD_NONE};
      return cocr(A, y, x, tol, maxit, hist);
    case ORC_BICG: return bicg(A, y, x, tol, maxit, hist);
    case ORC_GMRES: return gmres(A, y, x, tol, maxit, hist, g_restart);
    case ORC_CGS: return cgs(A, y, x, tol, maxit, hist);
    case ORC_CGNE: return cgne(A, y, x, tol, maxit, hist);
    case ORC_TFQMR: return tfqmr(A, y, x, tol, maxit, hist);
    case ORC_BICGSTABL: return bicgstabl(A, y, x, tol, maxit, hist, g_bicgstab_l);
  }
  return {0, ORC_INVALID, BD_NONE};
}

// Mixed-precision iterative refinement: the residual r = y - A x and the
// update x += d in double; the correction A d = r solved in single precision
// to a loose relative tolerance.
Result refine(int method, const Operator<double>& A64, const Operator<float>& A32, const Z* y, Z* x, double tol,
              int max_outer, double inner_tol, int inner_maxit, double* hist_outer, int* inner_total) {
  const int64_t n = A64.n;
  std::vector<Z> r(n);
  std::vector<C<float>> r32(n), d32(n);
  std::vector<double> ih(inner_maxit + 1);
  *inner_total = 0;
  const double ynorm = nrm2(n, y);
  if (ynorm == 0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0;
    hist_outer[0] = 0;
    return {0, ORC_OK, BD_NONE};
  }
  for (int outer = 0;; ++outer) {
    A64.apply(x, r.data());
    for (int64_t i = 0; i < n; ++i) r[i] = y[i] - r[i];
    hist_outer[outer] = nrm2(n, r.data()) / ynorm;
    if (hist_outer[outer] <= tol) return {outer, ORC_OK, BD_NONE};
    if (outer == max_outer) return {outer, ORC_NOT_CONVERGED, BD_NONE};
    for (int64_t i = 0; i < n; ++i) { r32[i] = C<float>(r[i]); d32[i] = 0; }
    const Result in = solve<float>(method, A32, r32.data(), d32.data(), inner_tol, inner_maxit, ih.data(), nullptr);
    *inner_total += in.iters;
    if (in.status < 0) return {outer, in.status, in.detail};
    if (in.iters == 0 && in.status == ORC_BREAKDOWN) return {outer, ORC_BREAKDOWN, in.detail};
    for (int64_t i = 0; i < n; ++i) x[i] += Z(d32[i]);
  }
}

struct OpBox {
  std::unique_ptr<Operator<double>> z;
  std::unique_ptr<Operator<float>> c;
  std::shared_ptr<DipoleCore> dip;
};

}  // namespace

// ============================================================================
// C exports (ctypes).  Complex arrays are interleaved (re, im) in the
// working precision.
// ============================================================================
extern "C" {

int orc_abi_version() { return 1; }
// Threads the dense products may use: 1 in the plain build.
int orc_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Restart length m of GMRES(m) for later solves (1 <= m <= 256).
void orc_set_restart(int m) { g_restart = m < 1 ? 1 : (m > 256 ? 256 : m); }
// Degree l of BiCGstab(l) for later solves (1 <= l <= 8).
void orc_set_bicgstab_l(int l) { g_bicgstab_l = l < 1 ? 1 : (l > 8 ? 8 : l); }

// symmetric != 0 asserts A = A^T (checked by the caller), which COCG and COCR require.
void* orc_op_dense_c128(int64_t n, int64_t lda, const void* A, int symmetric) {
  auto* b = new OpBox;
  b->z.reset(new Dense<double>(n, static_cast<const Z*>(A), lda));
  b->z->symmetric = symmetric != 0;
  return b;
}
void* orc_op_dense_c64(int64_t n, int64_t lda, const void* A, int symmetric) {
  auto* b = new OpBox;
  b->c.reset(new Dense<float>(n, static_cast<const C<float>*>(A), lda));
  b->c->symmetric = symmetric != 0;
  return b;
}
void* orc_op_dipole(int nx, int ny, int nz, const uint8_t* occ, double kd, double m_re, double m_im, int use_fft) {
  auto* b = new OpBox;
  b->dip = std::make_shared<DipoleCore>(nx, ny, nz, occ, kd, Z(m_re, m_im), use_fft != 0);
  b->z.reset(new Dipole<double>(b->dip));
  b->c.reset(new Dipole<float>(b->dip));
  return b;
}
void orc_op_destroy(void* op) { delete static_cast<OpBox*>(op); }
int64_t orc_op_n(void* op) {
  auto* b = static_cast<OpBox*>(op);
  return b->z ? b->z->n : b->c->n;
}
int64_t orc_dipole_nsites(void* op) { return static_cast<OpBox*>(op)->dip->N; }
void orc_dipole_alpha(void* op, double* out) {
  const Z a = static_cast<OpBox*>(op)->dip->alpha;
  out[0] = a.real();
  out[1] = a.imag();
}
void orc_dipole_sites(void* op, int32_t* ijl) {
  auto& d = *static_cast<OpBox*>(op)->dip;
  for (int64_t s = 0; s < d.N; ++s) { ijl[3 * s] = d.si[s]; ijl[3 * s + 1] = d.sj[s]; ijl[3 * s + 2] = d.sl[s]; }
}
// Direct-sum rows of A x for the listed output unknown sites (sel may be
// null: all sites).  y has layout y[a*nsel + q].
void orc_dipole_rows(void* op, const void* x, void* y, int64_t nsel, const int64_t* sel) {
  auto& d = *static_cast<OpBox*>(op)->dip;
  // direct_rows writes y[a*N + q]; stage through a full-size buffer.
  std::vector<Z> out(3 * d.N);
  const Z* xz = static_cast<const Z*>(x);
  d.direct_rows(xz, out.data(), nsel, sel);
  Z* yz = static_cast<Z*>(y);
  for (int a = 0; a < 3; ++a)
    for (int64_t q = 0; q < nsel; ++q) yz[a * nsel + q] = out[a * d.N + q];
}
void orc_green(double kd, double dx, double dy, double dz, double* out12) {
  Z g[6];
  green(kd, dx, dy, dz, g);
  for (int c = 0; c < 6; ++c) { out12[2 * c] = g[c].real(); out12[2 * c + 1] = g[c].imag(); }
}

void orc_matvec_c128(void* op, int trans, const void* x, void* y) {
  auto* b = static_cast<OpBox*>(op);
  if (trans) b->z->apply_h(static_cast<const Z*>(x), static_cast<Z*>(y));
  else b->z->apply(static_cast<const Z*>(x), static_cast<Z*>(y));
}
void orc_matvec_c64(void* op, int trans, const void* x, void* y) {
  auto* b = static_cast<OpBox*>(op);
  auto* xx = static_cast<const C<float>*>(x);
  auto* yy = static_cast<C<float>*>(y);
  if (trans) b->c->apply_h(xx, yy);
  else b->c->apply(xx, yy);
}

// out3 = {iters, status, breakdown detail}
void orc_solve_c128(void* op, int method, const void* y, void* x, double tol, int maxit, int* out3, double* hist,
                    double* tau) {
  auto* b = static_cast<OpBox*>(op);
  const Result res = solve<double>(method, *b->z, static_cast<const Z*>(y), static_cast<Z*>(x), tol, maxit, hist, tau);
  out3[0] = res.iters; out3[1] = res.status; out3[2] = res.detail;
}
void orc_solve_c64(void* op, int method, const void* y, void* x, double tol, int maxit, int* out3, double* hist,
                   double* tau) {
  auto* b = static_cast<OpBox*>(op);
  const Result res = solve<float>(method, *b->c, static_cast<const C<float>*>(y), static_cast<C<float>*>(x), tol,
                                  maxit, hist, tau);
  out3[0] = res.iters; out3[1] = res.status; out3[2] = res.detail;
}
// op64 and op32 describe the same matrix in double and single precision.
// out4 = {outer steps, status, breakdown detail, inner iterations in total}
void orc_refine(void* op64, void* op32, int method, const void* y, void* x, double tol, int max_outer,
                double inner_tol, int inner_maxit, int* out4, double* hist_outer) {
  auto* a = static_cast<OpBox*>(op64);
  auto* c = static_cast<OpBox*>(op32);
  int inner_total = 0;
  const Result res = refine(method, *a->z, *c->c, static_cast<const Z*>(y), static_cast<Z*>(x), tol, max_outer,
                            inner_tol, inner_maxit, hist_outer, &inner_total);
  out4[0] = res.iters; out4[1] = res.status; out4[2] = res.detail; out4[3] = inner_total;
}

void orc_fft3d(void* g, int64_t n0, int64_t n1, int64_t n2, int sign) {
  fft3d(static_cast<Z*>(g), n0, n1, n2, sign);
}

}  // extern "C"
