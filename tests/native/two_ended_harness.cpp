// Host build of the two-ended sweep data (paper_2107_05395_gb300/csrc/two_ended.h)
// for CPU unit tests (compiled by tests/test_two_ended_host.py).
#include <vector>

#include "../../paper_2107_05395_gb300/csrc/two_ended.h"

using namespace sb;

extern "C" {

// Solves A x_m = b_m (transpose = 0) or A^T x_m = b_m (transpose = 1) for the M
// systems of the interleaved array b (row i of system m at i * M + m) with the
// two-ended reference application.  diag: 2P+1 diagonals, diagonal-major, row-indexed
// (diag[(o + P) * N + i] = A[i][i+o]).  Returns the split row, or -1 when the data
// cannot be built.
int h_two_ended_solve(int P, int N, const double* diag, int transpose, long M, const double* b, double* x) {
  std::vector<double> dt;
  const double* d = diag;
  if (transpose) {  // A^T[i][i+o] = A[i+o][i]
    dt.assign((size_t)(2 * P + 1) * N, 0.0);
    for (int o = -P; o <= P; ++o)
      for (int i = 0; i < N; ++i) {
        const int j = i + o;
        if (j >= 0 && j < N) dt[(size_t)(o + P) * N + i] = diag[(size_t)(P - o) * N + j];
      }
    d = dt.data();
  }
  TwoEnded t;
  if (!build_two_ended(P, N, d, t)) return -1;
  std::vector<double> bm(N), xm(N);
  for (long m = 0; m < M; ++m) {
    for (int i = 0; i < N; ++i) bm[i] = b[(long)i * M + m];
    two_ended_apply(t, bm.data(), xm.data());
    for (int i = 0; i < N; ++i) x[(long)i * M + m] = xm[i];
  }
  return t.s;
}

// Solves A x_m = b_m from the other end with the rows of J A J (reversed_rows):
// forward sweep from row N-1 down, backward sweep from row 0 up.  Layout as for
// h_two_ended_solve.  Returns 0, or -1 when J A J has a zero pivot.  rows (may be
// NULL) receives [forward rows | backward rows], (P+1) values per row.
int h_reversed_solve(int P, int N, const double* diag, long M, const double* b, double* x, double* rows) {
  std::vector<double> fw, bw;
  if (!reversed_rows(P, N, diag, fw, bw)) return -1;
  const int W = P + 1;
  if (rows) {
    for (size_t k = 0; k < fw.size(); ++k) rows[k] = fw[k];
    for (size_t k = 0; k < bw.size(); ++k) rows[fw.size() + k] = bw[k];
  }
  std::vector<double> u(N);
  for (long m = 0; m < M; ++m) {
    for (int i = N - 1; i >= 0; --i) {
      double v = fw[(size_t)W * i] * b[(long)i * M + m];
      if (i + 1 < N) v -= fw[(size_t)W * i + 1] * u[i + 1];
      if (P == 2 && i + 2 < N) v -= fw[(size_t)W * i + 2] * u[i + 2];
      u[i] = v;
    }
    for (int i = 0; i < N; ++i) {
      double v = u[i];
      if (i >= 1) v -= bw[(size_t)W * i + 1] * x[(long)(i - 1) * M + m];
      if (P == 2 && i >= 2) v -= bw[(size_t)W * i + 2] * x[(long)(i - 2) * M + m];
      x[(long)i * M + m] = v;
    }
  }
  return 0;
}

// The device image [fw | bw | minv]; returns its length, or -1 when it cannot be
// built or does not fit in cap.
int h_two_ended_image(int P, int N, const double* diag, double* out, int cap) {
  TwoEnded t;
  if (!build_two_ended(P, N, diag, t)) return -1;
  const std::vector<double> img = two_ended_image(t);
  if ((int)img.size() > cap) return -1;
  for (size_t k = 0; k < img.size(); ++k) out[k] = img[k];
  return (int)img.size();
}

}  // extern "C"
