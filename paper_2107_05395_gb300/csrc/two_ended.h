// Host data of the two-ended ("burn at both ends") form of the banded sweeps:
// every system is eliminated from its first row downwards and from its last row
// upwards at the same time, so each thread carries two independent recurrences
// instead of one.  Exact up to rounding.  This is this library's own form (the
// paper sweeps each system from one end, sections 3.1 and 4.1); on GB300 the
// FP64 sweep of a 65536-system batch has too few independent recurrences per SM to
// keep the FP64 pipe full, and this doubles them without adding arithmetic.
//
// For half bandwidth P (1: tridiagonal, 2: pentadiagonal) and split row s:
//  * top: the usual LU elimination of rows 0..s-1 (the first s rows of A = LU),
//    giving   u_i = F0_i b_i - F1_i u_{i-1} - F2_i u_{i-2}   (F = {1/alpha, beta/alpha,
//    eps/alpha}) and the equations  x_i + B1_i x_{i+1} + B2_i x_{i+2} = u_i;
//  * bottom: the same elimination of the reversed matrix J A J (J reverses the
//    order of the unknowns), i.e. rows N-1 down to s, giving
//    u_i = F0'_i b_i - F1'_i u_{i+1} - F2'_i u_{i+2}  and
//    x_i + B1'_i x_{i-1} + B2'_i x_{i-2} = u_i;
//  * interface: the 2P equations of rows s-P..s-1 (top) and s..s+P-1 (bottom)
//    involve only z = (x_{s-P}, ..., x_{s+P-1}); z = Minv (u_{s-P}, ..., u_{s+P-1}),
//    with the 2P x 2P inverse computed here in FP64 once;
//  * back substitution outwards: top rows s-P-1 .. 0, bottom rows s+P .. N-1.
// Both the top and the bottom rows are valid equations of the original system
// (row operations within rows 0..s-1 and within rows s..N-1 respectively), so the
// solution is A^{-1} b.
#pragma once

#include <cmath>
#include <cstdint>
#include <vector>

namespace sb {

struct TwoEnded {
  int P = 0;
  int N = 0;
  int s = 0;                // split row: top rows 0..s-1, bottom rows s..N-1
  std::vector<double> fw;   // N rows of P+1: F0, F1[, F2] (top rows, then bottom rows)
  std::vector<double> bw;   // N rows of P+1: 1, B1[, B2]
  std::vector<double> minv; // (2P) x (2P), row-major
};

// Smallest N the two-ended form takes: 4P rows (two chains of at least 2P rows).
inline int two_ended_min_n(int P) { return 4 * P; }

// LU elimination rows 0..n-1 of the banded matrix given by its diagonals
// d(o, i) = A[i][i+o], o = -P..P, with out-of-range entries zero (the recurrence of
// section 4.1 with the outer diagonals zero when P = 1).  Writes forward rows
// {1/alpha_i, beta_i/alpha_i[, eps_i/alpha_i]} and backward rows {1, gamma_i[, delta_i]}
// for i < n into fw[W*i], bw[W*i] (W = P+1).  False on a zero or non-finite pivot.
template <typename Diag>
bool two_ended_eliminate(int P, int N, int n, Diag d, double* fw, double* bw) {
  const int W = P + 1;
  std::vector<double> ga(n, 0.0), de(n, 0.0);
  auto G = [&](int j) { return j >= 0 ? ga[j] : 0.0; };
  auto D = [&](int j) { return j >= 0 ? de[j] : 0.0; };
  for (int i = 0; i < n; ++i) {
    const double ai = (P == 2 && i >= 2) ? d(-2, i) : 0.0;
    const double bi = (i >= 1) ? d(-1, i) : 0.0;
    const double di = (i + 1 < N) ? d(1, i) : 0.0;
    const double ei = (P == 2 && i + 2 < N) ? d(2, i) : 0.0;
    const double be = bi - ai * G(i - 2);
    const double al = d(0, i) - ai * D(i - 2) - be * G(i - 1);
    if (al == 0.0 || !std::isfinite(al)) return false;
    ga[i] = (di - be * D(i - 1)) / al;
    de[i] = ei / al;
    fw[W * i + 0] = 1.0 / al;
    fw[W * i + 1] = be / al;
    bw[W * i + 0] = 1.0;
    bw[W * i + 1] = ga[i];
    if (P == 2) {
      fw[W * i + 2] = ai / al;
      bw[W * i + 2] = de[i];
    }
  }
  return true;
}

// Sweep rows of the whole reversed matrix J A J (the bottom half of the two-ended
// form, extended to every row), stored at the index of the row of A they act on.
// With them A x = b is solved from the other end: the forward sweep runs from row
// N-1 down, u_i = F0_i b_i - F1_i u_{i+1} - F2_i u_{i+2}, and the backward sweep
// from row 0 up, x_i = u_i - B1_i x_{i-1} - B2_i x_{i-2}.  Refinement passes that
// alternate their direction use them.  diag as for build_two_ended.  False on a
// zero or non-finite pivot of J A J.
inline bool reversed_rows(int P, int N, const double* diag, std::vector<double>& fw,
                          std::vector<double>& bw) {
  const int W = P + 1;
  // reversed matrix: R[i][i+o] = A[N-1-i][N-1-i-o]
  auto rev = [&](int o, int i) { return diag[(size_t)(P - o) * N + (N - 1 - i)]; };
  std::vector<double> rf((size_t)W * N), rb((size_t)W * N);
  if (!two_ended_eliminate(P, N, N, rev, rf.data(), rb.data())) return false;
  fw.assign((size_t)W * N, 0.0);
  bw.assign((size_t)W * N, 0.0);
  for (int j = 0; j < N; ++j)  // reversed row j is row N-1-j of A
    for (int k = 0; k < W; ++k) {
      fw[(size_t)W * (N - 1 - j) + k] = rf[(size_t)W * j + k];
      bw[(size_t)W * (N - 1 - j) + k] = rb[(size_t)W * j + k];
    }
  return true;
}

// Inverse of the n x n row-major matrix m (Gauss-Jordan with partial pivoting, FP64).
// False if a pivot is zero or the result is not finite.
inline bool two_ended_invert(int n, std::vector<double> m, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(m[(size_t)r * n + c]) > std::fabs(m[(size_t)p * n + c])) p = r;
    if (m[(size_t)p * n + c] == 0.0) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(m[(size_t)p * n + k], m[(size_t)c * n + k]);
        std::swap(inv[(size_t)p * n + k], inv[(size_t)c * n + k]);
      }
    const double q = 1.0 / m[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      m[(size_t)c * n + k] *= q;
      inv[(size_t)c * n + k] *= q;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double t = m[(size_t)r * n + c];
      if (t == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        m[(size_t)r * n + k] -= t * m[(size_t)c * n + k];
        inv[(size_t)r * n + k] -= t * inv[(size_t)c * n + k];
      }
    }
  }
  for (double v : inv)
    if (!std::isfinite(v)) return false;
  return true;
}

// Builds the two-ended data of the matrix with diagonals diag[(o + P) * N + i] =
// A[i][i+o].  The split is s = ceil(N / 2).  False for N < 4P, a zero pivot on either
// side, or a singular interface.
inline bool build_two_ended(int P, int N, const double* diag, TwoEnded& t) {
  if ((P != 1 && P != 2) || N < two_ended_min_n(P)) return false;
  const int W = P + 1;
  t.P = P;
  t.N = N;
  t.s = (N + 1) / 2;
  t.fw.assign((size_t)W * N, 0.0);
  t.bw.assign((size_t)W * N, 0.0);
  auto top = [&](int o, int i) { return diag[(size_t)(o + P) * N + i]; };
  // reversed matrix: R[i][i+o] = A[N-1-i][N-1-i-o]
  auto rev = [&](int o, int i) { return diag[(size_t)(P - o) * N + (N - 1 - i)]; };
  if (!two_ended_eliminate(P, N, t.s, top, t.fw.data(), t.bw.data())) return false;
  const int nb = N - t.s;
  std::vector<double> rf((size_t)W * nb), rb((size_t)W * nb);
  if (!two_ended_eliminate(P, N, nb, rev, rf.data(), rb.data())) return false;
  for (int j = 0; j < nb; ++j)  // reversed row j is original row N-1-j
    for (int k = 0; k < W; ++k) {
      t.fw[(size_t)W * (N - 1 - j) + k] = rf[(size_t)W * j + k];
      t.bw[(size_t)W * (N - 1 - j) + k] = rb[(size_t)W * j + k];
    }
  // interface rows: z_j = x_{s-P+j}, j = 0..2P-1
  const int n = 2 * P, z0 = t.s - P;
  std::vector<double> m((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    const int i = z0 + j;
    m[(size_t)j * n + j] = 1.0;
    for (int q = 1; q <= P; ++q) {
      const int col = (i < t.s) ? i + q : i - q;  // top rows look down, bottom rows up
      m[(size_t)j * n + (col - z0)] = t.bw[(size_t)W * i + q];
    }
  }
  return two_ended_invert(n, m, t.minv);
}

// Device image: [fw (W N) | bw (W N) | minv (4 P^2)], FP64.
inline std::vector<double> two_ended_image(const TwoEnded& t) {
  std::vector<double> img(t.fw);
  img.insert(img.end(), t.bw.begin(), t.bw.end());
  img.insert(img.end(), t.minv.begin(), t.minv.end());
  return img;
}

// Reference application to one system (stride 1), in the order the device kernel
// uses: both forward chains, the interface, both backward chains.  The forward
// scaling F0 * b is an FP64 product here.
inline void two_ended_apply(const TwoEnded& t, const double* b, double* x) {
  const int P = t.P, N = t.N, s = t.s, W = P + 1;
  std::vector<double> u(N);
  double v1 = 0, v2 = 0;
  for (int i = 0; i < s; ++i) {  // top, downwards
    const double* c = &t.fw[(size_t)W * i];
    double r = c[0] * b[i] - c[1] * v1;
    if (P == 2) r -= c[2] * v2;
    u[i] = r;
    v2 = v1;
    v1 = r;
  }
  v1 = v2 = 0;
  for (int i = N - 1; i >= s; --i) {  // bottom, upwards
    const double* c = &t.fw[(size_t)W * i];
    double r = c[0] * b[i] - c[1] * v1;
    if (P == 2) r -= c[2] * v2;
    u[i] = r;
    v2 = v1;
    v1 = r;
  }
  const int n = 2 * P, z0 = s - P;
  for (int j = 0; j < n; ++j) {
    double z = 0.0;
    for (int k = 0; k < n; ++k) z += t.minv[(size_t)j * n + k] * u[z0 + k];
    x[z0 + j] = z;
  }
  for (int i = z0 - 1; i >= 0; --i) {  // top, back up to row 0
    const double* c = &t.bw[(size_t)W * i];
    double r = u[i] - c[1] * x[i + 1];
    if (P == 2) r -= c[2] * x[i + 2];
    x[i] = r;
  }
  for (int i = s + P; i < N; ++i) {  // bottom, down to row N-1
    const double* c = &t.bw[(size_t)W * i];
    double r = u[i] - c[1] * x[i - 1];
    if (P == 2) r -= c[2] * x[i - 2];
    x[i] = r;
  }
}

}  // namespace sb
