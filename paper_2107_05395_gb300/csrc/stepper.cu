// Implicit time steppers with the shared matrix: diffusion and hyperdiffusion
// (backward Euler or Crank-Nicolson, sections 3.2 and 4.2) and the semi-implicit
// Cahn-Hilliard scheme of section 5.1.
//
// One step of every scheme is  A C^{n+1} = B C^n + E phi(C^n)  with band matrices
// A (shared, factorised once), B (identity for backward Euler, I - sigma K for
// Crank-Nicolson) and E (alpha D2_N for Cahn-Hilliard, phi(C) = C^3 - C).
//
// The fused kernel builds each right-hand-side row while the forward sweep
// consumes it: a window of the state rows i-2 .. i+2 (and phi of rows i-1 .. i+1)
// is kept in registers, fed by the same double-buffered row prefetch as the plain
// sweep, so the step reads the state once and writes it once (the paper computes
// the right-hand side with a separate stencil kernel every step).  Intermediates
// go in place into the state array behind the window; the backward sweep then
// overwrites them with C^{n+1}.  The time loop is captured into a CUDA graph.
#include <algorithm>
#include <cstring>
#include <map>
#include <type_traits>
#include <mutex>
#include <tuple>

#include "arith.cuh"
#include "sb_internal.h"

namespace sb {
namespace {

template <class A, typename T>
struct StConv;
template <>
struct StConv<NativeArith<double>, double> {
  static __device__ __forceinline__ double in(double v) { return v; }
  static __device__ __forceinline__ double out(double v) { return v; }
};
template <>
struct StConv<DFArith, double> {
  static __device__ __forceinline__ df in(double v) { return double_to_df(v); }
  static __device__ __forceinline__ double out(df v) { return df_to_double(v); }
};

// rcoef rows: if NB > 0, NB values per row (B at offsets -(NB/2)..NB/2), then if
// HAS_E, 3 values per row (E at offsets -1..1).  Out-of-matrix entries are 0.
// CYC: periodic ends: the window wraps (rows -2, -1 are rows N-2, N-1; rows N, N+1
// are rows 0, 1) and the solve applies the factor's correction: rank 1 (the
// tridiagonal matrix of section 3.3, rows cyc = (w_i, -z_i), scalars alpha, beta)
// or rank 2 (cyclic pentadiagonal, rows (w0_i, w1_i, -z0_i, -z1_i) and 12 scalars
// after them); see sweep_tile.cuh.
__host__ __device__ constexpr int step_cyc_len(int rank, int N) {
  return rank == 1 ? 2 * N : rank == 2 ? 4 * N + 12 : 0;
}

// Fifth-order Hamilton-Jacobi WENO derivative (Jiang and Peng's scheme, the one the
// paper takes for its advection term, section 6.1) at the centre of the window
// c[0..6] = C_{i-3..i+3}, grid spacing 1.  SIDE = -1: the stencil biased toward
// lower rows (differences D_{i-3}..D_{i+1}, D_j = C_{j+1} - C_j); SIDE = +1: toward
// higher rows (D_{i+2}..D_{i-2}).  Three third-order candidates, smoothness
// indicators S_k, eps = 1e-6 max q^2 + 1e-99 and weights (0.1, 0.6, 0.3)/(S_k+eps)^2
// normalised.  GB300's FP64 pipe is the bound here, so what needs no FP64
// arithmetic runs on the integer pipe: max |q| and max_k (S_k + eps) compare bit
// patterns (non-negative doubles order like their bits), and the (S_k + eps) are
// scaled by the power of two that brings their maximum into [1, 2) (built from its
// exponent field; exact), which keeps every product of the weights in range (each
// ratio is at least ~1e-8) with one division in all.  The result equals the
// normalised form up to rounding.
__device__ __forceinline__ double max_bits(double a, double b) {
  return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ double abs_bits(double a) {
  return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffLL);
}
template <int SIDE>
__device__ __forceinline__ double weno5(const double (&c)[7]) {
  double q1, q2, q3, q4, q5;
  if constexpr (SIDE < 0) {
    q1 = c[1] - c[0]; q2 = c[2] - c[1]; q3 = c[3] - c[2]; q4 = c[4] - c[3]; q5 = c[5] - c[4];
  } else {
    q1 = c[6] - c[5]; q2 = c[5] - c[4]; q3 = c[4] - c[3]; q4 = c[3] - c[2]; q5 = c[2] - c[1];
  }
  const double p1 = q1 * (1.0 / 3.0) - q2 * (7.0 / 6.0) + q3 * (11.0 / 6.0);
  const double p2 = -q2 * (1.0 / 6.0) + q3 * (5.0 / 6.0) + q4 * (1.0 / 3.0);
  const double p3 = q3 * (1.0 / 3.0) + q4 * (5.0 / 6.0) - q5 * (1.0 / 6.0);
  const double d1 = q1 - 2.0 * q2 + q3, e1 = q1 - 4.0 * q2 + 3.0 * q3;
  const double d2 = q2 - 2.0 * q3 + q4, e2 = q2 - q4;
  const double d3 = q3 - 2.0 * q4 + q5, e3 = 3.0 * q3 - 4.0 * q4 + q5;
  const double s1 = (13.0 / 12.0) * d1 * d1 + 0.25 * e1 * e1;
  const double s2 = (13.0 / 12.0) * d2 * d2 + 0.25 * e2 * e2;
  const double s3 = (13.0 / 12.0) * d3 * d3 + 0.25 * e3 * e3;
  const double qa = max_bits(max_bits(max_bits(abs_bits(q1), abs_bits(q2)), max_bits(abs_bits(q3), abs_bits(q4))),
                             abs_bits(q5));
  const double eps = fma(1e-6, qa * qa, 1e-99);
  const double t1 = s1 + eps, t2 = s2 + eps, t3 = s3 + eps;
  // 2^-(e - 1023) for the exponent field e of max t (t >= 1e-99, finite unless the
  // data is; the clamp only keeps the bit pattern well formed then)
  const long long ef = (__double_as_longlong(max_bits(max_bits(t1, t2), t3)) >> 52) & 0x7ff;
  const double scale = __longlong_as_double((2046LL - min(max(ef, 1LL), 2045LL)) << 52);
  const double r1 = t1 * scale, r2 = t2 * scale, r3 = t3 * scale;
  const double r12 = r1 * r2, r13 = r1 * r3, r23 = r2 * r3;
  const double w1 = 0.1 * (r23 * r23), w2 = 0.6 * (r13 * r13), w3 = 0.3 * (r12 * r12);
  return (w1 * p1 + w2 * p2 + w3 * p3) / (w1 + w2 + w3);
}

// STATS: each system's new state also gives ell_m = 1 / (1 - <C^2>), <C^2> the mean
// of C_i^2 over its N rows (section 5.3's coarsening length), written to ellm[m].
// GC: the coefficient rows do not fit in shared memory (large N) and are read from
// their device copies directly (warp-uniform loads, served by L1/L2).
// ADV (periodic Cahn-Hilliard, native FP64 only): the travelling-wave forced scheme
// of section 6.1 adds adv * W(C^n) + amp[m] * g[i] to the right-hand side, with W
// the fifth-order Hamilton-Jacobi WENO derivative biased toward lower rows (ADV = -1,
// rows i-3..i+2) or higher rows (ADV = +1, rows i-2..i+3); the state window then
// spans rows i-3..i+3 instead of i-2..i+2.
template <class A, int P, int NB, bool HAS_E, int R, int CYC, bool STATS = false, bool GC = false,
          int ADV = 0>
__global__ void __launch_bounds__(512)
fused_step_kernel(const typename A::C* __restrict__ coef, const typename A::C* __restrict__ rcoef,
                  int N, int64_t M, int64_t ld, const double* src, double* state, int64_t ntiles,
                  const typename A::C* __restrict__ cyc, typename A::C alpha, typename A::C beta,
                  double* __restrict__ ellm = nullptr, const double* __restrict__ gprof = nullptr,
                  const double* __restrict__ amp = nullptr, double adv = 0.0) {
  using V = typename A::V;
  using C = typename A::C;
  using S = typename A::S;
  constexpr int W = P + 1;
  constexpr int NE = HAS_E ? 3 : 0;
  constexpr int RW = NB + NE;  // rhs coefficients per row
  constexpr int LA = ADV != 0 ? 3 : 2;  // rows of look-ahead (and look-behind) in the window
  constexpr int LW = 2 * LA + 1;
  static_assert(ADV == 0 || (std::is_same_v<V, double> && CYC == 2 && HAS_E),
                "the forced scheme is periodic Cahn-Hilliard in native FP64");
  static_assert(R >= LA, "the look-ahead must fit in one prefetch batch");

  const C* fw;
  const C* rc;
  const C* cy;
  const double* gp;
  if constexpr (GC) {
    fw = coef;
    rc = rcoef;
    cy = cyc;
    gp = gprof;
  } else {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* cs = reinterpret_cast<C*>(smem_raw);
    const int n = 2 * W * N;
    for (int k = threadIdx.x; k < n; k += blockDim.x) cs[k] = coef[k];
    for (int k = threadIdx.x; k < RW * N; k += blockDim.x) cs[n + k] = rcoef[k];
    if constexpr (CYC != 0)
      for (int k = threadIdx.x; k < step_cyc_len(CYC, N); k += blockDim.x) cs[n + RW * N + k] = cyc[k];
    double* gs = reinterpret_cast<double*>(cs + n + RW * N + step_cyc_len(CYC, N));
    if constexpr (ADV != 0)
      for (int k = threadIdx.x; k < N; k += blockDim.x) gs[k] = gprof[k];
    __syncthreads();
    fw = cs;
    rc = cs + n;
    cy = rc + RW * N;
    gp = gs;
  }
  const C* bw = fw + W * N;

  const int lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5); tile < ntiles;
       tile += (int64_t)gridDim.x * nw) {
    const int64_t m = tile * 32 + lane;
    if (m >= M) continue;
    double* y = state + m;     // intermediates and the new state
    const double* c = src + m;  // the old state (may be the same array as y)

    // window: cw[k] = C_{i-LA+k}, pw[k] = phi(C_{i-1+k}) for the row i being built
    V cw[LW], pw[3];
#pragma unroll
    for (int k = 0; k < LW; ++k) cw[k] = A::zero();
#pragma unroll
    for (int k = 0; k < 3; ++k) pw[k] = A::zero();
    double va[R], vb[R];
    auto load_rows = [&](double (&buf)[R], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (i0 + j < N) buf[j] = c[(int64_t)(i0 + j) * ld];
    };
    // push raw row k (value v, already 0 when k >= N) into the windows
    auto push = [&](double v) {
#pragma unroll
      for (int k = 0; k < LW - 1; ++k) cw[k] = cw[k + 1];
      cw[LW - 1] = StConv<A, double>::in(v);
      if constexpr (HAS_E) {
        pw[0] = pw[1];
        pw[1] = pw[2];
        pw[2] = A::cubic(cw[LA + 1]);  // phi(C_{i+1}) once C_{i+1} entered the window
      }
    };
    double fm = 0.0;  // this system's forcing amplitude
    if constexpr (ADV != 0) fm = amp[m];
    V u1 = A::zero(), u2 = A::zero(), dot = A::zero(), dot1 = A::zero();
    auto build_and_sweep = [&](int i) {
      V r;
      if constexpr (NB > 0) {
        const C* b = rc + RW * i;
        r = A::mulc(b[0], cw[LA - NB / 2]);
#pragma unroll
        for (int k = 1; k < NB; ++k) r = A::fmac(b[k], cw[LA - NB / 2 + k], r);
      } else {
        r = cw[LA];
      }
      if constexpr (HAS_E) {
        const C* e = rc + RW * i + NB;
        r = A::fmac(e[0], pw[0], r);
        r = A::fmac(e[1], pw[1], r);
        r = A::fmac(e[2], pw[2], r);
      }
      if constexpr (ADV != 0) {
        r = fma(adv, weno5<ADV>(cw), r);
        r = fma(fm, gp[i], r);
      }
      const V u = A::template step<P, false>(fw + W * i, r, u1, u2);
      if constexpr (CYC == 1) dot = A::fmac(cy[2 * i], r, dot);
      if constexpr (CYC == 2) {
        dot = A::fmac(cy[4 * i], r, dot);
        dot1 = A::fmac(cy[4 * i + 1], r, dot1);
      }
      *reinterpret_cast<S*>(y + (int64_t)i * ld) = A::to_store(u);
      u2 = u1;
      u1 = u;
    };
    // prime: rows 0 and 1 enter the window before row 0 is built (rows -2, -1 are 0,
    // or with periodic ends row -1 is row N-1; both wrapped rows are read before the
    // forward sweep overwrites anything)
    load_rows(va, 0);
    load_rows(vb, R);
    double cpre[LA];  // rows 0..LA-1, which wrap in as rows N..N+LA-1
#pragma unroll
    for (int k = 0; k < LA; ++k) cpre[k] = 0.0;
    if constexpr (CYC != 0) {
#pragma unroll
      for (int k = 0; k < LA; ++k) cpre[k] = va[k];  // N >= 3 (rank 1) or 5 (rank 2), R >= LA
      // LA + 1 pushes (rows 0..LA) precede the build of row 0 and each shifts the
      // window left by one, so the last LA slots end up holding rows -LA..-1
#pragma unroll
      for (int k = 0; k < LA; ++k)
        cw[LW - LA + k] = StConv<A, double>::in(c[(int64_t)(N - LA + k) * ld]);
    }
#pragma unroll
    for (int k = 0; k < LA; ++k) push(N > k ? va[k] : 0.0);
    // row i needs raw row i + LA: from the current buffer or the next one
    auto ahead = [&](int i, double v) { return (i + LA < N) ? v : (CYC != 0 ? cpre[i + LA - N] : 0.0); };
    for (int i0 = 0; i0 < N; i0 += 2 * R) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int i = i0 + j;
        if (i < N) {
          const int k = j + LA;
          push(ahead(i, k < R ? va[k] : vb[k - R]));
          build_and_sweep(i);
        }
      }
      load_rows(va, i0 + 2 * R);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int i = i0 + R + j;
        if (i < N) {
          const int k = j + LA;
          push(ahead(i, k < R ? vb[k] : va[k - R]));
          build_and_sweep(i);
        }
      }
      load_rows(vb, i0 + 3 * R);
    }

    // backward sweep (B0 == 1 for the primal factors)
    V x1 = A::zero(), x2 = A::zero(), fc = A::zero(), g1 = A::zero();
    double sq = 0.0;
    auto emit = [&](int row, V v) {
      const double o = StConv<A, double>::out(v);
      y[(int64_t)row * ld] = o;
      if constexpr (STATS) sq = fma(o, o, sq);
    };
    S sa[R], sb_[R];
    auto load_mid = [&](S (&buf)[R], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (i0 - j >= 0) buf[j] = *reinterpret_cast<const S*>(y + (int64_t)(i0 - j) * ld);
    };
    auto bwd = [&](S (&buf)[R], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int i = i0 - j;
        if (i >= 0) {
          const V xi = A::template step<P, true>(bw + W * i, A::from_store(buf[j]), x1, x2);
          if constexpr (CYC == 1) {
            if (i == N - 1) fc = A::mulc(beta, A::fmac(alpha, xi, dot));
            emit(i, A::fmac(cy[2 * i + 1], fc, xi));
          } else if constexpr (CYC == 2) {
            if (i < N - 2) {
              emit(i, A::fmac(cy[4 * i + 3], g1, A::fmac(cy[4 * i + 2], fc, xi)));
            } else if (i == N - 2) {  // x1 holds y_{N-1}
              const C* sc = cy + 4 * N;
              const V t0 = A::fmac(sc[0], dot, A::fmac(sc[1], dot1, A::fmac(sc[4], xi, A::mulc(sc[5], x1))));
              const V t1 = A::fmac(sc[2], dot, A::fmac(sc[3], dot1, A::fmac(sc[6], xi, A::mulc(sc[7], x1))));
              fc = A::fmac(sc[8], t0, A::mulc(sc[9], t1));
              g1 = A::fmac(sc[10], t0, A::mulc(sc[11], t1));
              const int j1 = N - 1;
              emit(j1, A::fmac(cy[4 * j1 + 3], g1, A::fmac(cy[4 * j1 + 2], fc, x1)));
              emit(i, A::fmac(cy[4 * i + 3], g1, A::fmac(cy[4 * i + 2], fc, xi)));
            }
          } else {
            emit(i, xi);
          }
          x2 = x1;
          x1 = xi;
        }
      }
    };
    load_mid(sa, N - 1);
    for (int i0 = N - 1; i0 >= 0; i0 -= 2 * R) {
      load_mid(sb_, i0 - R);
      bwd(sa, i0);
      load_mid(sa, i0 - 2 * R);
      bwd(sb_, i0 - R);
    }
    if constexpr (STATS) ellm[m] = 1.0 / (1.0 - sq / (double)N);
  }
}

// Fixed-shape deterministic mean of the per-system values: kMeanBlocks partial sums
// over fixed index ranges (fixed strided order, fixed shared-memory tree), then one
// block sums the partials and scales by 1/M.
constexpr int kMeanBlocks = 256;
constexpr int kMeanThreads = 256;

__global__ void __launch_bounds__(kMeanThreads) mean_partials(const double* v, int64_t n, double* part) {
  __shared__ double sh[kMeanThreads];
  const int64_t chunk = (n + kMeanBlocks - 1) / kMeanBlocks;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kMeanThreads) acc += v[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kMeanThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kMeanThreads) mean_final(const double* part, int64_t n, double* out) {
  __shared__ double sh[kMeanThreads];
  sh[threadIdx.x] = (threadIdx.x < kMeanBlocks) ? part[threadIdx.x] : 0.0;
  __syncthreads();
  for (int w = kMeanThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] / (double)n;
}

// Unfused right-hand side (the paper's separate stencil pass): f = B C + E phi(C);
// CYC: periodic ends (row -1 is row N-1, row N is row 0).
template <class A, int NB, bool HAS_E, bool CYC>
__global__ void rhs_kernel(const typename A::C* __restrict__ rcoef, int N, int64_t M, int64_t ld,
                           const double* __restrict__ C_in, double* __restrict__ f) {
  using V = typename A::V;
  using C = typename A::C;
  constexpr int RW = NB + (HAS_E ? 3 : 0);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (m >= M || i >= N) return;
  auto val = [&](int k) -> V {
    if constexpr (CYC) k = k < 0 ? k + N : (k >= N ? k - N : k);
    return (k >= 0 && k < N) ? StConv<A, double>::in(C_in[(int64_t)k * ld + m]) : A::zero();
  };
  const C* row = rcoef + RW * i;
  V r;
  if constexpr (NB > 0) {
    r = A::mulc(row[0], val(i - NB / 2));
#pragma unroll
    for (int k = 1; k < NB; ++k) r = A::fmac(row[k], val(i - NB / 2 + k), r);
  } else {
    r = val(i);
  }
  if constexpr (HAS_E) {
#pragma unroll
    for (int k = 0; k < 3; ++k) r = A::fmac(row[NB + k], A::cubic(val(i - 1 + k)), r);
  }
  f[(int64_t)i * ld + m] = StConv<A, double>::out(r);
}

}  // namespace
}  // namespace sb

// ------------------------------------------------------------------ host side



namespace sb {
namespace {

constexpr int kStepRows = 8;
constexpr int kGraphSteps = 64;  // steps per captured graph

// Periodic correction data of a factor for an arithmetic policy (see sweep.cu).
template <class A>
struct StepCyc;
template <>
struct StepCyc<NativeArith<double>> {
  static const double* rows(const sb_factor* f) { return f->cyc64; }
  static double coef(double v) { return v; }
};
template <>
struct StepCyc<DFArith> {
  static const df* rows(const sb_factor* f) { return reinterpret_cast<const df*>(f->cycdf); }
  static df coef(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
  }
};

template <class A, int P, int NB, bool HAS_E, int CYC, bool STATS = false, int ADV = 0>
int launch_fused(const sb_stepper* st, const typename A::C* coef, const typename A::C* rc,
                 const double* src, double* state, int64_t M, int64_t ld, cudaStream_t stream,
                 double* ellm = nullptr, const double* amp = nullptr) {
  const sb_factor* f = st->fac;
  const int N = (int)f->N;
  constexpr int RW = NB + (HAS_E ? 3 : 0);
  size_t smem =
      ((size_t)2 * (P + 1) * N + (size_t)RW * N + (size_t)step_cyc_len(CYC, N)) * sizeof(typename A::C) +
      (ADV != 0 ? (size_t)N * sizeof(double) : 0);
  auto k = fused_step_kernel<A, P, NB, HAS_E, kStepRows, CYC, STATS, false, ADV>;
  if (smem > (size_t)kMaxDynSmem) {
    // FP64 coefficients of a large N are read from device memory
    if constexpr (std::is_same_v<A, NativeArith<double>>) {
      k = fused_step_kernel<A, P, NB, HAS_E, kStepRows, CYC, STATS, true, ADV>;
      smem = 0;
    } else {
      return fail(SB_ERR_UNSUPPORTED,
                  "N=%d too large for the fused step's shared memory (only FP64 steps read the "
                  "coefficients from device memory)", N);
    }
  }
  const int threads = 256;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> occ;
  int nb = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(reinterpret_cast<const void*>(k), (int)smem);
    auto it = occ.find(key);
    if (it == occ.end()) {
      SB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
      SB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem));
      occ[key] = nb;
    } else {
      nb = it->second;
    }
  }
  if (nb < 1) return fail(SB_ERR_UNSUPPORTED, "fused step kernel cannot be resident");
  const int64_t ntiles = (M + 31) / 32;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
  const typename A::C* cy = CYC ? StepCyc<A>::rows(f) : nullptr;  // primal rows (op 0)
  k<<<(unsigned)grid, threads, smem, stream>>>(coef, rc, N, M, ld, src, state, ntiles, cy,
                                              StepCyc<A>::coef(CYC ? f->cyc_alpha[0] : 0.0),
                                              StepCyc<A>::coef(CYC ? f->cyc_beta[0] : 0.0), ellm,
                                              ADV != 0 ? st->g64 : nullptr, amp, st->adv);
  return cuda_check(cudaGetLastError(), "fused step launch");
}

// One forced step (periodic Cahn-Hilliard with the travelling-wave terms), in place.
int one_step_forced(const sb_stepper* st, double* state, const double* amp, int64_t M, int64_t ld,
                    cudaStream_t stream) {
  using A = NativeArith<double>;
  return st->adv >= 0.0
             ? launch_fused<A, 2, 0, true, 2, false, -1>(st, st->fac->coef64, st->r64, state, state, M,
                                                         ld, stream, nullptr, amp)
             : launch_fused<A, 2, 0, true, 2, false, +1>(st, st->fac->coef64, st->r64, state, state, M,
                                                         ld, stream, nullptr, amp);
}

template <class A, int NB, bool HAS_E, bool CYC>
int launch_rhs(const sb_stepper* st, const typename A::C* rc, const double* in, double* out,
               int64_t M, int64_t ld, cudaStream_t stream) {
  const int N = (int)st->N;
  dim3 grid((unsigned)((M + 255) / 256), (unsigned)N);
  rhs_kernel<A, NB, HAS_E, CYC><<<grid, 256, 0, stream>>>(rc, N, M, ld, in, out);
  return cuda_check(cudaGetLastError(), "rhs launch");
}

template <class A>
int one_step(const sb_stepper* st, const typename A::C* coef, const typename A::C* rc,
             const double* src, double* state, int64_t M, int64_t ld, cudaStream_t stream) {
  const int P = st->fac->P;
  const bool per = st->fac->periodic;
  if (st->has_e)
    return per ? launch_fused<A, 2, 0, true, 2>(st, coef, rc, src, state, M, ld, stream)
               : launch_fused<A, 2, 0, true, 0>(st, coef, rc, src, state, M, ld, stream);
  if (P == 1 && per)
    return st->NB == 3 ? launch_fused<A, 1, 3, false, 1>(st, coef, rc, src, state, M, ld, stream)
                       : launch_fused<A, 1, 0, false, 1>(st, coef, rc, src, state, M, ld, stream);
  if (P == 1)
    return st->NB == 3 ? launch_fused<A, 1, 3, false, 0>(st, coef, rc, src, state, M, ld, stream)
                       : launch_fused<A, 1, 0, false, 0>(st, coef, rc, src, state, M, ld, stream);
  if (per)
    return st->NB == 5 ? launch_fused<A, 2, 5, false, 2>(st, coef, rc, src, state, M, ld, stream)
                       : launch_fused<A, 2, 0, false, 2>(st, coef, rc, src, state, M, ld, stream);
  return st->NB == 5 ? launch_fused<A, 2, 5, false, 0>(st, coef, rc, src, state, M, ld, stream)
                     : launch_fused<A, 2, 0, false, 0>(st, coef, rc, src, state, M, ld, stream);
}

// A fused Cahn-Hilliard step that also writes each system's coarsening length.
template <class A>
int one_step_stats(const sb_stepper* st, const typename A::C* coef, const typename A::C* rc,
                   double* state, int64_t M, int64_t ld, cudaStream_t stream, double* ellm) {
  if (!st->has_e) return fail(SB_ERR_UNSUPPORTED, "the coarsening statistic needs a Cahn-Hilliard stepper");
  return st->fac->periodic
             ? launch_fused<A, 2, 0, true, 2, true>(st, coef, rc, state, state, M, ld, stream, ellm)
             : launch_fused<A, 2, 0, true, 0, true>(st, coef, rc, state, state, M, ld, stream, ellm);
}

template <class A>
int one_rhs(const sb_stepper* st, const typename A::C* rc, const double* in, double* out,
            int64_t M, int64_t ld, cudaStream_t stream) {
  const bool per = st->fac->periodic;
  if (st->has_e)
    return per ? launch_rhs<A, 0, true, true>(st, rc, in, out, M, ld, stream)
               : launch_rhs<A, 0, true, false>(st, rc, in, out, M, ld, stream);
  if (st->NB == 3)
    return per ? launch_rhs<A, 3, false, true>(st, rc, in, out, M, ld, stream)
               : launch_rhs<A, 3, false, false>(st, rc, in, out, M, ld, stream);
  if (st->NB == 5)
    return per ? launch_rhs<A, 5, false, true>(st, rc, in, out, M, ld, stream)
               : launch_rhs<A, 5, false, false>(st, rc, in, out, M, ld, stream);
  return launch_rhs<A, 0, false, false>(st, rc, in, out, M, ld, stream);
}

}  // namespace

// One fused step from `src` into `dst` (the same array for an in-place step).
int stepper_step(const sb_stepper* st, const double* src, double* dst, int64_t M, int64_t ld,
                 sb_arith arith, cudaStream_t stream) {
  if (arith == SB_ARITH_DF32)
    return one_step<DFArith>(st, reinterpret_cast<const df*>(st->fac->coefdf),
                             reinterpret_cast<const df*>(st->rdf), src, dst, M, ld, stream);
  return one_step<NativeArith<double>>(st, st->fac->coef64, st->r64, src, dst, M, ld, stream);
}

namespace {
int step_fused(const sb_stepper* st, double* state, int64_t M, int64_t ld, sb_arith arith,
               cudaStream_t stream) {
  return stepper_step(st, state, state, M, ld, arith, stream);
}
}  // namespace
}  // namespace sb

namespace sb {
namespace {
// the FP64 right-hand side of a refined step, rounded up so the FP32 scratch after it
// stays 16-byte aligned
size_t refined_f_bytes(size_t elems) { return ((elems * sizeof(double) + 255) / 256) * 256; }

// Runs `nsteps` steps of `step` on stream s: as replays of a captured graph of
// kGraphSteps steps (cached in `cache` under `key`) and the remainder launched
// directly.  Direct launches are used for every step when the mode asks for them,
// on the legacy stream, inside a caller's capture, or for fewer than kGraphSteps
// steps.
template <typename K, typename Step>
int run_graphed(sb_stepper* st, GraphCache<K>& cache, const K& key, int mode, int64_t nsteps,
                cudaStream_t s, Step step) {
  bool capturing = false;
  if (mode == SB_RUN_GRAPH && s != nullptr) {
    cudaStreamCaptureStatus cs;
    SB_CUDA(cudaStreamIsCapturing(s, &cs));
    capturing = (cs != cudaStreamCaptureStatusNone);
  }
  if (mode != SB_RUN_GRAPH || s == nullptr || capturing || nsteps < kGraphSteps) {
    for (int64_t n = 0; n < nsteps; ++n) SB_TRY(step());
    return SB_OK;
  }
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lk(st->mu);
    exec = cache.find(key);
    if (exec == nullptr) {
      cudaGraph_t graph = nullptr;
      SB_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      int rc = SB_OK;
      for (int n = 0; n < kGraphSteps && rc == SB_OK; ++n) rc = step();
      cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (rc != SB_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      SB_CUDA(e);
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      SB_CUDA(e);
      cache.put(key, exec);
    }
  }
  int64_t n = 0;
  for (; n + kGraphSteps <= nsteps; n += kGraphSteps) SB_CUDA(cudaGraphLaunch(exec, s));
  for (; n < nsteps; ++n) SB_TRY(step());
  return SB_OK;
}
}  // namespace
}  // namespace sb

using namespace sb;

extern "C" {

int sb_stepper_create(int kind, int scheme, int bc, int64_t N, double coef, double dt,
                      sb_stepper** out) {
  clear_error();
  if (!out) return fail(SB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 1) return fail(SB_ERR_INVALID_ARG, "N must be >= 1");
  if (!std::isfinite(coef) || !std::isfinite(dt)) return fail(SB_ERR_INVALID_ARG, "non-finite coefficient");
  int mat = 0;
  double acoef = coef;
  if (kind == SB_STEP_DIFFUSION) {
    if (bc != SB_BC_DIRICHLET && bc != SB_BC_PERIODIC)
      return fail(SB_ERR_INVALID_ARG, "diffusion supports SB_BC_DIRICHLET or SB_BC_PERIODIC");
    if (bc == SB_BC_PERIODIC && N < 3) return fail(SB_ERR_INVALID_ARG, "periodic ends need N >= 3");
    mat = bc == SB_BC_PERIODIC ? SB_MAT_DIFFUSION_PERIODIC : SB_MAT_DIFFUSION_DIRICHLET;
  } else if (kind == SB_STEP_HYPERDIFFUSION) {
    if (bc != SB_BC_HINGED && bc != SB_BC_TRUNCATED && bc != SB_BC_PERIODIC)
      return fail(SB_ERR_INVALID_ARG,
                  "hyperdiffusion supports SB_BC_HINGED, SB_BC_TRUNCATED or SB_BC_PERIODIC");
    if (bc == SB_BC_PERIODIC && N < 5) return fail(SB_ERR_INVALID_ARG, "periodic ends need N >= 5");
    mat = bc == SB_BC_HINGED ? SB_MAT_HYPER_HINGED
                             : (bc == SB_BC_TRUNCATED ? SB_MAT_HYPER_TRUNCATED : SB_MAT_CH_PERIODIC);
  } else if (kind == SB_STEP_CAHN_HILLIARD) {
    if (bc != SB_BC_NOFLUX && bc != SB_BC_PERIODIC)
      return fail(SB_ERR_INVALID_ARG, "Cahn-Hilliard supports SB_BC_NOFLUX or SB_BC_PERIODIC");
    if (bc == SB_BC_PERIODIC && N < 5) return fail(SB_ERR_INVALID_ARG, "periodic ends need N >= 5");
    if (scheme != SB_SCHEME_BE)
      return fail(SB_ERR_INVALID_ARG, "Cahn-Hilliard uses the semi-implicit scheme (SB_SCHEME_BE)");
    if (!(dt > 0.0)) return fail(SB_ERR_INVALID_ARG, "dt must be > 0");
    mat = bc == SB_BC_PERIODIC ? SB_MAT_CH_PERIODIC : SB_MAT_CH_NOFLUX;
    acoef = dt * coef;
  } else {
    return fail(SB_ERR_INVALID_ARG, "unknown stepper kind %d", kind);
  }
  if (scheme != SB_SCHEME_BE && scheme != SB_SCHEME_CN)
    return fail(SB_ERR_INVALID_ARG, "unknown scheme %d", scheme);

  std::vector<double> adiag;
  int P = 0;
  SB_TRY(build_matrix(mat, N, acoef, adiag, &P));
  sb_stepper* st = new (std::nothrow) sb_stepper();
  if (!st) return fail(SB_ERR_ALLOC, "host allocation failed");
  st->kind = kind;
  st->scheme = scheme;
  st->bc = bc;
  st->N = N;
  st->coef = coef;
  st->dt = dt;
  int rc;
  if (P == 1 && mat == SB_MAT_DIFFUSION_PERIODIC)
    rc = sb_factor_shared_tri_periodic(N, adiag.data(), adiag.data() + N, adiag.data() + 2 * N,
                                       &st->fac);
  else if (P == 1)
    rc = sb_factor_shared_tri(N, adiag.data(), adiag.data() + N, adiag.data() + 2 * N, &st->fac);
  else if (mat == SB_MAT_CH_PERIODIC)
    rc = sb_factor_shared_penta_periodic(N, adiag.data(), adiag.data() + N, adiag.data() + 2 * N,
                                         adiag.data() + 3 * N, adiag.data() + 4 * N, &st->fac);
  else
    rc = sb_factor_shared_penta(N, adiag.data(), adiag.data() + N, adiag.data() + 2 * N,
                                adiag.data() + 3 * N, adiag.data() + 4 * N, &st->fac);
  if (rc != SB_OK) {
    delete st;
    return rc;
  }
  // right-hand-side rows
  std::vector<double> rows;
  if (kind == SB_STEP_CAHN_HILLIARD) {
    st->has_e = true;
    rows.assign(3 * N, 0.0);  // dt * D2_N (cell-centred no-flux closure) or dt * D2_P
    const bool per = bc == SB_BC_PERIODIC;
    for (int64_t i = 0; i < N; ++i) {
      const bool first = (i == 0) && !per, last = (i == N - 1) && !per;
      rows[3 * i + 0] = first ? 0.0 : dt;
      rows[3 * i + 1] = dt * (-2.0 + (first ? 1.0 : 0.0) + (last ? 1.0 : 0.0));
      rows[3 * i + 2] = last ? 0.0 : dt;
    }
  } else if (scheme == SB_SCHEME_CN) {
    std::vector<double> bdiag;
    int PB = 0;
    rc = build_matrix(mat, N, -coef, bdiag, &PB);  // B = I - sigma K
    if (rc != SB_OK) {
      sb_stepper_destroy(st);
      return rc;
    }
    st->NB = 2 * PB + 1;
    rows.assign((size_t)st->NB * N, 0.0);
    for (int64_t i = 0; i < N; ++i)
      for (int k = 0; k < st->NB; ++k) rows[(size_t)st->NB * i + k] = bdiag[(size_t)k * N + i];
  }
  if (!rows.empty()) {
    std::vector<float> rdf(2 * rows.size());
    for (size_t k = 0; k < rows.size(); ++k) {
      rdf[2 * k] = (float)rows[k];
      rdf[2 * k + 1] = (float)(rows[k] - (double)rdf[2 * k]);
    }
    DeviceGuard g(st->fac->device);
    rc = cuda_check(cudaMalloc(&st->r64, rows.size() * sizeof(double)), "cudaMalloc");
    if (rc == SB_OK) rc = cuda_check(cudaMalloc(&st->rdf, rdf.size() * sizeof(float)), "cudaMalloc");
    if (rc == SB_OK)
      rc = cuda_check(cudaMemcpy(st->r64, rows.data(), rows.size() * sizeof(double),
                                 cudaMemcpyHostToDevice), "cudaMemcpy");
    if (rc == SB_OK)
      rc = cuda_check(cudaMemcpy(st->rdf, rdf.data(), rdf.size() * sizeof(float),
                                 cudaMemcpyHostToDevice), "cudaMemcpy");
    if (rc != SB_OK) {
      sb_stepper_destroy(st);
      return rc;
    }
  }
  *out = st;
  return SB_OK;
}

void sb_stepper_destroy(sb_stepper* st) {
  if (!st) return;
  if (st->fac) {
    DeviceGuard g(st->fac->device);
    st->graphs.clear();
    st->forced_graphs.clear();
    st->refined_graphs.clear();
    if (st->g64) cudaFree(st->g64);
    if (st->r64) cudaFree(st->r64);
    if (st->rdf) cudaFree(st->rdf);
    sb_factor_destroy(st->fac);
  }
  delete st;
}

const sb_factor* sb_stepper_factor(const sb_stepper* st) { return st ? st->fac : nullptr; }

int sb_stepper_set_forcing(sb_stepper* st, double adv, const double* profile) {
  clear_error();
  if (!st || !profile) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (st->kind != SB_STEP_CAHN_HILLIARD || st->bc != SB_BC_PERIODIC)
    return fail(SB_ERR_UNSUPPORTED, "the travelling-wave forcing needs a periodic Cahn-Hilliard stepper");
  if (!std::isfinite(adv)) return fail(SB_ERR_INVALID_ARG, "non-finite advection coefficient");
  const int64_t N = st->N;
  for (int64_t i = 0; i < N; ++i)
    if (!std::isfinite(profile[i])) return fail(SB_ERR_INVALID_ARG, "non-finite forcing at row %lld", (long long)i);
  DeviceGuard g(st->fac->device);
  SB_TRY(g.rc);
  std::lock_guard<std::mutex> lk(st->mu);
  if (!st->g64) SB_CUDA(cudaMalloc(&st->g64, (size_t)N * sizeof(double)));
  // captured graphs read the old values through the same pointer, so they stay valid;
  // the advection coefficient is a launch argument, so they are rebuilt
  SB_CUDA(cudaDeviceSynchronize());
  SB_CUDA(cudaMemcpy(st->g64, profile, (size_t)N * sizeof(double), cudaMemcpyHostToDevice));
  st->forced_graphs.clear();
  st->adv = adv;
  st->forced = true;
  return SB_OK;
}

int sb_stepper_run_forced(sb_stepper* st, double* state, const double* amp, int64_t M, int64_t ld,
                          int64_t nsteps, int mode, void* stream) {
  clear_error();
  if (!st) return fail(SB_ERR_INVALID_ARG, "stepper is NULL");
  if (!st->forced) return fail(SB_ERR_INVALID_ARG, "the stepper has no forcing (sb_stepper_set_forcing)");
  if (nsteps < 0) return fail(SB_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (mode != SB_RUN_GRAPH && mode != SB_RUN_DIRECT)
    return fail(SB_ERR_INVALID_ARG, "forced runs support SB_RUN_GRAPH and SB_RUN_DIRECT");
  const sb_factor* f = st->fac;
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  if (M < 0 || ld < M || ld < 1) return fail(SB_ERR_INVALID_ARG, "bad M or ld");
  if (M == 0 || nsteps == 0) return SB_OK;
  const size_t bytes = (size_t)((f->N - 1) * ld + M) * sizeof(double);
  SB_TRY(check_device_range(state, bytes, sizeof(double), f->device, "state"));
  SB_TRY(check_device_range(amp, (size_t)M * sizeof(double), sizeof(double), f->device, "amp"));
  SB_TRY(check_alias(state, bytes, amp, (size_t)M * sizeof(double), "state", "amp"));
  cudaStream_t s = (cudaStream_t)stream;
  const auto key = std::make_tuple(reinterpret_cast<uintptr_t>(state), reinterpret_cast<uintptr_t>(amp), M, ld);
  return run_graphed(st, st->forced_graphs, key, mode, nsteps, s,
                     [&]() { return one_step_forced(st, state, amp, M, ld, s); });
}

int sb_stepper_refined_workspace_bytes(const sb_stepper* st, int64_t M, int64_t ld, size_t* bytes) {
  clear_error();
  if (!st || !bytes) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (M < 0 || ld < M) return fail(SB_ERR_INVALID_ARG, "bad M or ld");
  const size_t elems = (size_t)((st->N - 1) * ld + M);
  *bytes = refined_f_bytes(elems) + elems * sizeof(float);
  return SB_OK;
}

int sb_stepper_run_refined(sb_stepper* st, double* state, int64_t M, int64_t ld, int n_refine,
                           sb_arith residual_arith, int64_t nsteps, int mode, void* work,
                           size_t work_bytes, void* stream) {
  clear_error();
  if (!st) return fail(SB_ERR_INVALID_ARG, "stepper is NULL");
  if (st->forced) return fail(SB_ERR_INVALID_ARG, "a forced stepper runs through sb_stepper_run_forced");
  if (st->fac->periodic)
    return fail(SB_ERR_UNSUPPORTED, "the refined steps do not support periodic ends");
  if (nsteps < 0) return fail(SB_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (n_refine < 0 || n_refine > 16) return fail(SB_ERR_INVALID_ARG, "n_refine must be in [0, 16]");
  if (residual_arith != SB_ARITH_NATIVE && residual_arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown residual arithmetic mode %d", (int)residual_arith);
  if (mode != SB_RUN_GRAPH && mode != SB_RUN_DIRECT)
    return fail(SB_ERR_INVALID_ARG, "refined runs support SB_RUN_GRAPH and SB_RUN_DIRECT");
  const sb_factor* f = st->fac;
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  if (M < 0 || ld < M || ld < 1) return fail(SB_ERR_INVALID_ARG, "bad M or ld");
  if (M == 0 || nsteps == 0) return SB_OK;
  const size_t elems = (size_t)((f->N - 1) * ld + M);
  const size_t need = refined_f_bytes(elems) + elems * sizeof(float);
  SB_TRY(check_device_range(state, elems * sizeof(double), sizeof(double), f->device, "state"));
  if (work == nullptr || work_bytes < need)
    return fail(SB_ERR_INVALID_ARG, "the refined run needs a workspace of %zu bytes", need);
  SB_TRY(check_device_range(work, need, 16, f->device, "work"));
  SB_TRY(check_alias(state, elems * sizeof(double), work, need, "state", "work"));
  double* fbuf = static_cast<double*>(work);
  void* scratch = static_cast<char*>(work) + refined_f_bytes(elems);
  cudaStream_t s = (cudaStream_t)stream;
  // one step: f = B C + E phi(C) in FP64, then C = A^{-1} f by FP32 sweeps of f and
  // n_refine passes r = f - A C (residual in FP64 or double-float), d = A_32^{-1} r,
  // C += d; one kernel per step, each tile taken through all of it in turn
  auto step = [&]() -> int {
    return refined_step(f, st->r64, st->NB, st->has_e, state, fbuf, static_cast<float*>(scratch), M, ld,
                        n_refine, residual_arith, s);
  };
  const auto key = std::make_tuple(reinterpret_cast<uintptr_t>(state), reinterpret_cast<uintptr_t>(work), M, ld,
                                   n_refine * 2 + (residual_arith == SB_ARITH_DF32 ? 1 : 0));
  return run_graphed(st, st->refined_graphs, key, mode, nsteps, s, [&]() { return step(); });
}

int sb_stepper_run_coarsening(sb_stepper* st, double* state, int64_t M, int64_t ld, sb_arith arith,
                              int64_t nsteps, double* ell, void* work, size_t work_bytes,
                              void* stream) {
  clear_error();
  if (!st) return fail(SB_ERR_INVALID_ARG, "stepper is NULL");
  if (st->kind != SB_STEP_CAHN_HILLIARD || st->forced)
    return fail(SB_ERR_UNSUPPORTED, "the coarsening statistic needs an unforced Cahn-Hilliard stepper");
  if (nsteps < 0) return fail(SB_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (arith != SB_ARITH_NATIVE && arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown arithmetic mode %d", (int)arith);
  const sb_factor* f = st->fac;
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  if (M < 1 || ld < M) return fail(SB_ERR_INVALID_ARG, "need M >= 1 and ld >= M");
  if (nsteps == 0) return SB_OK;
  const size_t bytes = (size_t)((f->N - 1) * ld + M) * sizeof(double);
  SB_TRY(check_device_range(state, bytes, sizeof(double), f->device, "state"));
  SB_TRY(check_device_range(ell, (size_t)nsteps * sizeof(double), sizeof(double), f->device, "ell"));
  const size_t need = ((size_t)M + kMeanBlocks) * sizeof(double);
  if (work == nullptr || work_bytes < need)
    return fail(SB_ERR_INVALID_ARG, "the coarsening run needs a workspace of %zu bytes", need);
  SB_TRY(check_device_range(work, need, sizeof(double), f->device, "work"));
  SB_TRY(check_alias(state, bytes, work, need, "state", "work"));
  SB_TRY(check_alias(ell, (size_t)nsteps * sizeof(double), work, need, "ell", "work"));
  SB_TRY(check_alias(ell, (size_t)nsteps * sizeof(double), state, bytes, "ell", "state"));
  double* ellm = static_cast<double*>(work);
  double* part = ellm + M;
  cudaStream_t s = (cudaStream_t)stream;
  for (int64_t n = 0; n < nsteps; ++n) {
    if (arith == SB_ARITH_DF32)
      SB_TRY(one_step_stats<DFArith>(st, reinterpret_cast<const df*>(f->coefdf),
                                     reinterpret_cast<const df*>(st->rdf), state, M, ld, s, ellm));
    else
      SB_TRY(one_step_stats<NativeArith<double>>(st, f->coef64, st->r64, state, M, ld, s, ellm));
    mean_partials<<<kMeanBlocks, kMeanThreads, 0, s>>>(ellm, M, part);
    mean_final<<<1, kMeanThreads, 0, s>>>(part, M, ell + n);
    SB_CUDA(cudaGetLastError());
  }
  return SB_OK;
}

int sb_stepper_workspace_bytes(const sb_stepper* st, int64_t M, int64_t ld, size_t* bytes) {
  clear_error();
  if (!st || !bytes) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (M < 0 || ld < M) return fail(SB_ERR_INVALID_ARG, "bad M or ld");
  *bytes = (size_t)((st->N - 1) * ld + M) * sizeof(double);
  return SB_OK;
}

int sb_stepper_run(sb_stepper* st, double* state, int64_t M, int64_t ld, sb_arith arith,
                   int64_t nsteps, int mode, void* work, size_t work_bytes, void* stream) {
  clear_error();
  if (!st) return fail(SB_ERR_INVALID_ARG, "stepper is NULL");
  if (st->forced) return fail(SB_ERR_INVALID_ARG, "a forced stepper runs through sb_stepper_run_forced");
  if (nsteps < 0) return fail(SB_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (arith != SB_ARITH_NATIVE && arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown arithmetic mode %d", (int)arith);
  if (mode != SB_RUN_GRAPH && mode != SB_RUN_DIRECT && mode != SB_RUN_UNFUSED)
    return fail(SB_ERR_INVALID_ARG, "unknown run mode %d", mode);
  const sb_factor* f = st->fac;
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  if (M < 0 || ld < M || ld < 1) return fail(SB_ERR_INVALID_ARG, "bad M or ld");
  if (M == 0 || nsteps == 0) return SB_OK;
  const size_t bytes = (size_t)((f->N - 1) * ld + M) * sizeof(double);
  SB_TRY(check_device_range(state, bytes, sizeof(double), f->device, "state"));
  cudaStream_t s = (cudaStream_t)stream;

  if (mode == SB_RUN_UNFUSED) {
    if (work == nullptr || work_bytes < bytes)
      return fail(SB_ERR_INVALID_ARG, "the unfused run needs a workspace of %zu bytes", bytes);
    SB_TRY(check_device_range(work, bytes, sizeof(double), f->device, "work"));
    SB_TRY(check_alias(state, bytes, work, bytes, "state", "work"));
    double* w = static_cast<double*>(work);
    for (int64_t n = 0; n < nsteps; ++n) {
      if (st->NB == 0 && !st->has_e) {
        SB_TRY(launch_sweep(f, OP_PRIMAL, state, SB_F64, state, SB_F64, M, ld, arith,
                            shape_for(f, arith, SB_F64, SB_F64), s));
        continue;
      }
      if (arith == SB_ARITH_DF32)
        SB_TRY(one_rhs<DFArith>(st, reinterpret_cast<const df*>(st->rdf), state, w, M, ld, s));
      else
        SB_TRY(one_rhs<NativeArith<double>>(st, st->r64, state, w, M, ld, s));
      SB_TRY(launch_sweep(f, OP_PRIMAL, w, SB_F64, state, SB_F64, M, ld, arith,
                          shape_for(f, arith, SB_F64, SB_F64), s));
    }
    return SB_OK;
  }

  // graphs of kGraphSteps fused steps, replayed; the remainder launched directly
  const auto key = std::make_tuple(reinterpret_cast<uintptr_t>(state), M, ld, (int)arith, kGraphSteps);
  return run_graphed(st, st->graphs, key, mode, nsteps, s,
                     [&]() { return step_fused(st, state, M, ld, arith, s); });
}

}  // extern "C"
