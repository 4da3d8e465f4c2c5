// FP64 CPU oracle in plain C++ -- TEST INFRASTRUCTURE ONLY.
//
// The staggered Dslash, the normal operator M = m^2 - D_eo D_oe, its CG solve and the SU(3)
// routines of Table 1 of arXiv:1309.0551 (Srinivasan, "Optimizing the performance of
// Lattice Gauge Theory simulations with Streaming SIMD extensions"), written as plain loops
// over std::complex<double>, parallel over sites with OpenMP.  Only the tests,
// __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs load it; the GPU
// library never does, and this file shares no code, header or table with it.
//
// The paper names the routines (Table 1) and writes out one component of the adjoint
// mat-vec (Eqs. (1.1)-(2.3)); it does not write the operator, which follows the readings
// the numpy oracle states too:
//   (D chi)(x) = sum_mu eta_mu(x) [ U_mu(x) chi(x+mu) - U_mu(x-mu)^dag chi(x-mu) ],
//   no factor 1/2, periodic, eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y),
//   eta_t = (-1)^(x+y+z); lex = x + Lx (y + Ly (z + Lz t)), parity (x+y+z+t) mod 2,
//   checkerboard index cb = lex >> 1 (every extent even).
// Layouts: U[mu][lex][a][b] complex (interleaved re, im doubles); a colour vector on one
// parity v[cb][a].
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

using cd = std::complex<double>;

namespace {

struct Lattice {
  int L[4];
  long V;
  explicit Lattice(const int* d) {
    for (int i = 0; i < 4; ++i) L[i] = d[i];
    V = (long)L[0] * L[1] * L[2] * L[3];
  }
  void coords(long lex, int c[4]) const {
    c[0] = (int)(lex % L[0]);
    lex /= L[0];
    c[1] = (int)(lex % L[1]);
    lex /= L[1];
    c[2] = (int)(lex % L[2]);
    c[3] = (int)(lex / L[2]);
  }
  long lex(const int c[4]) const { return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3])); }
  long hop(long x, int mu, int step) const {
    int c[4];
    coords(x, c);
    c[mu] = (c[mu] + step + L[mu]) % L[mu];
    return lex(c);
  }
  int parity(long x) const {
    int c[4];
    coords(x, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
  }
  // the site of parity p whose checkerboard index is cb: one of lex 2cb, 2cb + 1 (Lx even)
  long site(long cb, int p) const { return parity(2 * cb) == p ? 2 * cb : 2 * cb + 1; }
};

int eta(int mu, long x, const Lattice& g) {
  int c[4];
  g.coords(x, c);
  const int s = mu == 0 ? 0 : mu == 1 ? c[0] : mu == 2 ? c[0] + c[1] : c[0] + c[1] + c[2];
  return (s & 1) ? -1 : 1;
}

const cd* link(const double* U, const Lattice& g, int mu, long x) {
  return reinterpret_cast<const cd*>(U) + ((size_t)mu * g.V + x) * 9;
}

// c = A b (mult_su3_mat_vec) and c = A^dag b (mult_adj_su3_mat_vec, Eqs. (1.1)-(2.3)).
void mat_vec(const cd* A, const cd* b, cd* c) {
  for (int i = 0; i < 3; ++i) {
    cd s = 0.0;
    for (int j = 0; j < 3; ++j) s += A[3 * i + j] * b[j];
    c[i] = s;
  }
}
void adj_mat_vec(const cd* A, const cd* b, cd* c) {
  for (int i = 0; i < 3; ++i) {
    cd s = 0.0;
    for (int k = 0; k < 3; ++k) s += std::conj(A[3 * k + i]) * b[k];
    c[i] = s;
  }
}

void dslash(const Lattice& g, const double* U, const cd* in, cd* out, int out_parity, int nthreads) {
  const long Vh = g.V / 2;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (long cb = 0; cb < Vh; ++cb) {
    const long x = g.site(cb, out_parity);
    cd acc[3] = {0.0, 0.0, 0.0};
    for (int mu = 0; mu < 4; ++mu) {
      const long xf = g.hop(x, mu, +1), xb = g.hop(x, mu, -1);
      cd f[3], b[3];
      mat_vec(link(U, g, mu, x), in + 3 * (xf >> 1), f);
      adj_mat_vec(link(U, g, mu, xb), in + 3 * (xb >> 1), b);
      const double e = eta(mu, x, g);
      for (int a = 0; a < 3; ++a) acc[a] += e * (f[a] - b[a]);
    }
    for (int a = 0; a < 3; ++a) out[3 * cb + a] = acc[a];
  }
}

void normal(const Lattice& g, const double* U, const cd* p, cd* out, double mass, int nthreads,
            std::vector<cd>& tmp) {
  const long n = 3 * (g.V / 2);
  tmp.resize(n);
  dslash(g, U, p, tmp.data(), 1, nthreads);
  dslash(g, U, tmp.data(), out, 0, nthreads);
  for (long i = 0; i < n; ++i) out[i] = mass * mass * p[i] - out[i];
}

double norm2(const std::vector<cd>& v) {
  double s = 0.0;
  for (const cd& z : v) s += std::norm(z);
  return s;
}
double redot(const std::vector<cd>& a, const std::vector<cd>& b) {   // Re <a, b>
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += (std::conj(a[i]) * b[i]).real();
  return s;
}

}  // namespace

extern "C" {

int ora_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// c[i] = op(A[i]) b[i], op = adjoint when adj (Table 1: mult_su3_mat_vec, mult_adj_su3_mat_vec).
void ora_su3_mat_vec(long n, const double* A, const double* b, double* c, int adj) {
  const cd* a = reinterpret_cast<const cd*>(A);
  const cd* v = reinterpret_cast<const cd*>(b);
  cd* w = reinterpret_cast<cd*>(c);
  for (long i = 0; i < n; ++i) {
    if (adj) adj_mat_vec(a + 9 * i, v + 3 * i, w + 3 * i);
    else mat_vec(a + 9 * i, v + 3 * i, w + 3 * i);
  }
}

// C[i] = op(A[i]) op(B[i]) (Table 1: mult_su3_nn, mult_su3_an, mult_su3_na).
void ora_su3_mul(long n, const double* A, const double* B, double* C, int adjA, int adjB) {
  const cd* a = reinterpret_cast<const cd*>(A);
  const cd* b = reinterpret_cast<const cd*>(B);
  cd* c = reinterpret_cast<cd*>(C);
  for (long m = 0; m < n; ++m)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        cd s = 0.0;
        for (int k = 0; k < 3; ++k) {
          const cd x = adjA ? std::conj(a[9 * m + 3 * k + i]) : a[9 * m + 3 * i + k];
          const cd y = adjB ? std::conj(b[9 * m + 3 * j + k]) : b[9 * m + 3 * k + j];
          s += x * y;
        }
        c[9 * m + 3 * i + j] = s;
      }
}

// out = D in on the sites of parity out_parity (in on the other parity), [Vh][3] complex.
void ora_dslash_eo(const int* dims, const double* U, const double* in, double* out, int out_parity,
                   int nthreads) {
  Lattice g(dims);
  dslash(g, U, reinterpret_cast<const cd*>(in), reinterpret_cast<cd*>(out), out_parity, nthreads);
}

// out = M p = m^2 p - D_eo D_oe p on the even sites.
void ora_normal_op(const int* dims, const double* U, const double* p, double* out, double mass, int nthreads) {
  Lattice g(dims);
  std::vector<cd> tmp;
  normal(g, U, reinterpret_cast<const cd*>(p), reinterpret_cast<cd*>(out), mass, nthreads, tmp);
}

// FP64 CG on M x = b from x = 0 (Hestenes-Stiefel).  The iterated residual only triggers the
// stop: the true residual ||b - M x|| / ||b|| is then recomputed; if it is above tol the
// residual is replaced by it (at most max_restarts times) with beta in the Polak-Ribiere
// form max(0, Re<r_new, r_new - r_k>) / ||r_k||^2, and the iteration continues.
// Returns the iterations; *true_rel receives the final true relative residual.
int ora_cg(const int* dims, const double* U, const double* b_in, double* x_out, double mass, double tol,
           int maxiter, int max_restarts, int nthreads, double* true_rel) {
  Lattice g(dims);
  const long n = 3 * (g.V / 2);
  const cd* bp = reinterpret_cast<const cd*>(b_in);
  std::vector<cd> b(bp, bp + n), x(n, 0.0), r(b), p(b), Ap(n), rk(n), tmp;
  const double bb = norm2(b);
  double rr = norm2(r);
  int it = 0, restarts = 0;
  if (bb == 0.0) {
    for (long i = 0; i < n; ++i) reinterpret_cast<cd*>(x_out)[i] = 0.0;
    *true_rel = 0.0;
    return 0;
  }
  while (it < maxiter) {
    rk = r;
    normal(g, U, p.data(), Ap.data(), mass, nthreads, tmp);
    const double alpha = rr / redot(p, Ap);
    for (long i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    double rr_new = norm2(r);
    ++it;
    double beta = rr_new / rr;
    if (rr_new <= tol * tol * bb) {
      normal(g, U, x.data(), Ap.data(), mass, nthreads, tmp);
      for (long i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
      const double tr = norm2(r);
      if (std::sqrt(tr / bb) <= tol || restarts >= max_restarts) break;
      ++restarts;
      rr_new = tr;
      const double pr = (tr - redot(rk, r)) / rr;
      beta = pr > 0.0 ? pr : 0.0;
    }
    for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
  }
  normal(g, U, x.data(), Ap.data(), mass, nthreads, tmp);
  double tr = 0.0;
  for (long i = 0; i < n; ++i) tr += std::norm(b[i] - Ap[i]);
  *true_rel = std::sqrt(tr / bb);
  for (long i = 0; i < n; ++i) reinterpret_cast<cd*>(x_out)[i] = x[i];
  return it;
}

}  // extern "C"
