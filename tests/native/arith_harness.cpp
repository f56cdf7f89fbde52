// Host build of the library's arithmetic header for CPU unit tests (compiled by
// tests/test_arith_host.py with -ffp-contract=off so float operations round like
// the device's __f*_rn intrinsics).
#include <vector>

#include "../../paper_2107_05395_gb300/csrc/arith.cuh"
#include "../../paper_2107_05395_gb300/csrc/narrow.cuh"

using namespace sb;

extern "C" {

void h_double_to_df(const double* v, float* h, float* l, long n) {
  for (long i = 0; i < n; ++i) {
    const df d = double_to_df(v[i]);
    h[i] = d.h;
    l[i] = d.l;
  }
}

void h_f64_to_f32_trunc(const double* v, float* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = f64_to_f32_trunc(v[i]);
}

void h_df_to_double(const float* h, const float* l, double* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = df_to_double(df{h[i], l[i]});
}

// One step out = c0*in - c1*v1 - c2*v2 in df arithmetic; all inputs given as
// (hi, lo) pairs; c0one skips the c0 product.  P = 1 ignores c2/v2.
void h_df_step(int P, int c0one, const float* c, const float* in, const float* v1,
               const float* v2, float* out) {
  const df cc[3] = {{c[0], c[1]}, {c[2], c[3]}, {c[4], c[5]}};
  const df a{in[0], in[1]}, b{v1[0], v1[1]}, d{v2[0], v2[1]};
  df r;
  if (P == 1)
    r = c0one ? DFArith::step<1, true>(cc, a, b, d) : DFArith::step<1, false>(cc, a, b, d);
  else
    r = c0one ? DFArith::step<2, true>(cc, a, b, d) : DFArith::step<2, false>(cc, a, b, d);
  out[0] = r.h;
  out[1] = r.l;
}

// The kernel's two recurrences for one system with prescaled coefficient rows
// (forward rows then backward rows, P+1 values per row), in df arithmetic with
// FP64 input and output, exactly as the device code orders them.
void h_df_sweep(int P, int fone, int bone, long N, const double* coef, const double* rhs,
                double* x) {
  const int W = P + 1;
  std::vector<df> c(2 * W * N);
  for (long k = 0; k < 2 * W * N; ++k) {
    const float hi = (float)coef[k];
    c[k] = df{hi, (float)(coef[k] - (double)hi)};
  }
  std::vector<df> mid(N);
  df u1{0.f, 0.f}, u2{0.f, 0.f};
  for (long i = 0; i < N; ++i) {
    const df in = double_to_df(rhs[i]);
    const df* row = &c[W * i];
    df u;
    if (P == 1)
      u = fone ? DFArith::step<1, true>(row, in, u1, u2) : DFArith::step<1, false>(row, in, u1, u2);
    else
      u = fone ? DFArith::step<2, true>(row, in, u1, u2) : DFArith::step<2, false>(row, in, u1, u2);
    mid[i] = u;
    u2 = u1;
    u1 = u;
  }
  df x1{0.f, 0.f}, x2{0.f, 0.f};
  for (long i = N - 1; i >= 0; --i) {
    const df* row = &c[W * N + W * i];
    df xi;
    if (P == 1)
      xi = bone ? DFArith::step<1, true>(row, mid[i], x1, x2)
                : DFArith::step<1, false>(row, mid[i], x1, x2);
    else
      xi = bone ? DFArith::step<2, true>(row, mid[i], x1, x2)
                : DFArith::step<2, false>(row, mid[i], x1, x2);
    x[i] = df_to_double(xi);
    x2 = x1;
    x1 = xi;
  }
}
}

extern "C" void h_dmul_int(const double* a, const double* b, double* out, long n) {
  for (long i = 0; i < n; ++i) out[i] = dmul_int(a[i], b[i]);
}
