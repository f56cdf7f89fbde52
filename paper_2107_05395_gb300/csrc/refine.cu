// Mixed precision with iterative refinement and multi-group batching.
//
// Refinement (FP32 right-hand sides, FP64 solution):
//   x_0 = sweep32(b);   for k = 1..n:  r = b - A x_{k-1} (FP64, or double-float),
//                                      d = sweep32(r),  x_k = x_{k-1} + d.
// The factorisation of A is the FP64 one rounded to FP32 for the sweeps; the
// residual uses A's original FP64 entries.  A correction pass's forward sweep
// builds r_i from a window of x (rows i-P .. i+P, prefetched in batches) and
// writes the FP32 intermediate to a caller-provided workspace (x must stay intact
// until every residual row is built); its backward sweep adds d_i to x_i.  One
// launch runs every pass: each warp takes a tile through the FP32 pass and all
// correction passes before its next tile.
//
// Forms, chosen by what fits in shared memory: (1) separate passes, their rows
// staged through a shared-memory ring or prefetched into registers; (2) merged
// passes, each correction pass run inside the backward sweep of the pass before it
// (passes alternate between eliminating from the top and from the bottom, with
// the rows of J A J); (3) for two passes with the FP64 residual, the merged passes
// with two tiles per warp two sweeps apart, so that every loop has FP64 work.
//
// Groups: several shared-LHS factors (different N) are solved by one launch.  The
// persistent CTAs are split between the groups in proportion to N*M; a CTA stages
// its own group's coefficients once.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "sb_internal.h"
#include "narrow.cuh"
#include "sweep_tile.cuh"

namespace sb {
namespace {

constexpr int kMaxGroups = 8;

template <typename CT, typename TI, typename TO>
struct Groups {
  int G;
  int cta_begin[kMaxGroups + 1];
  const CT* coef[kMaxGroups];   // sweep rows [forward | backward]
  const CT* rcoef[kMaxGroups];  // the same for J A J, at A's row indices (fused refinement only)
  const void* arow[kMaxGroups]; // A row by row (refinement passes only)
  int N[kMaxGroups];
  int64_t M[kMaxGroups], ld[kMaxGroups], ntiles[kMaxGroups];
  const TI* rhs[kMaxGroups];
  TO* x[kMaxGroups];
  float* work[kMaxGroups];
};

__device__ __forceinline__ int group_of(const int* cta_begin, int G) {
  int g = 0;
  while (g + 1 < G && (int)blockIdx.x >= cta_begin[g + 1]) ++g;
  return g;
}

// ---------------------------------------------------------- grouped sweep

template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO>
__global__ void __launch_bounds__(512)
grouped_sweep_kernel(const __grid_constant__ Groups<typename A::C, TI, TO> a) {
  using C = typename A::C;
  constexpr int W = P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* cs = reinterpret_cast<C*>(smem_raw);
  const int g = group_of(a.cta_begin, a.G);
  const int N = a.N[g];
  stage(cs, a.coef[g], 2 * W * N);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  const int ctas = a.cta_begin[g + 1] - a.cta_begin[g];
  for (int64_t tile = (blockIdx.x - a.cta_begin[g]) + (int64_t)ctas * (threadIdx.x >> 5);
       tile < a.ntiles[g]; tile += (int64_t)ctas * nw)
    sweep_tile<A, P, F_ONE, B_ONE, TI, TO, 1, kRows>(cs, cs + W * N, N, a.M[g], a.ld[g],
                                                     a.rhs[g], a.x[g], tile);
}

// ------------------------------------------------------- refinement pass

// FP64 residual -> FP32 right-hand side of the correction sweep (truncation with
// integer operations; see f64_to_f32_trunc).
__device__ __forceinline__ float narrow_trunc(double v) { return f64_to_f32_trunc(v); }

template <bool DFRES>
struct Residual;

__device__ __forceinline__ double to_f64(float b) { return widen_f32(b); }
__device__ __forceinline__ double to_f64(double b) { return b; }
__device__ __forceinline__ df to_df(float b) { return {b, 0.f}; }
__device__ __forceinline__ df to_df(double b) { return double_to_df(b); }

template <>
struct Residual<false> {  // FP64 residual: r = b - sum_k a_k x_{i+k} with FMAs
  using X = double;
  using AC = double;
  static __device__ __forceinline__ X in(double v) { return v; }
  template <int NB, typename TB>
  static __device__ __forceinline__ float eval(const AC* a, const X* xw, TB b) {
    double r = to_f64(b);
#pragma unroll
    for (int k = 0; k < NB; ++k) r = fma(-a[k], xw[k], r);
    return narrow_trunc(r);
  }
};

template <>
struct Residual<true> {  // the same residual in double-float arithmetic
  using X = df;
  using AC = df;
  static __device__ __forceinline__ X in(double v) { return double_to_df(v); }
  template <int NB, typename TB>
  static __device__ __forceinline__ float eval(const AC* a, const X* xw, TB b) {
    df r = to_df(b);
#pragma unroll
    for (int k = 0; k < NB; ++k) r = DFArith::fmac(df{-a[k].h, -a[k].l}, xw[k], r);
    return r.h;
  }
};

// TB: the stored right-hand side, FP32 (the mixed-precision solve) or FP64 (a
// right-hand side built in FP64, e.g. by a time step).
template <int P, bool DFRES, int R, typename TB>
__device__ __forceinline__ void refine_tile(const float* fw, const float* bw,
                                            const typename Residual<DFRES>::AC* arow, int N,
                                            int64_t M, int64_t ld, const TB* b, double* x,
                                            float* g, int64_t tile) {
  using RS = Residual<DFRES>;
  using X = typename RS::X;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  const int64_t m = tile * 32 + (threadIdx.x & 31);
  if (m >= M) return;
  const TB* bp = b + m;
  double* xp = x + m;
  float* gp = g + m;

  // ---- forward: r_i = b_i - (A x)_i, FP32 forward sweep, intermediate to g
  X xw[NB];  // x_{i-P} .. x_{i+P}
#pragma unroll
  for (int k = 0; k < NB; ++k) xw[k] = RS::in(0.0);
  double xa[R], xb[R];
  TB ba[R], bb[R];
  auto load = [&](double (&xs)[R], TB (&bs)[R], int i0) {
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (i0 + j < N) {
        xs[j] = xp[(int64_t)(i0 + j) * ld];
        bs[j] = ld_stream(bp + (int64_t)(i0 + j) * ld);
      }
  };
  auto push = [&](double v) {
#pragma unroll
    for (int k = 0; k < NB - 1; ++k) xw[k] = xw[k + 1];
    xw[NB - 1] = RS::in(v);
  };
  float u1 = 0.f, u2 = 0.f;
  auto row = [&](int i, TB bi) {
    const float r = RS::template eval<NB>(arow + NB * i, xw, bi);
    const float u = NativeArith<float>::step<P, false>(fw + W * i, r, u1, u2);
    gp[(int64_t)i * ld] = u;
    u2 = u1;
    u1 = u;
  };
  load(xa, ba, 0);
  load(xb, bb, R);
#pragma unroll
  for (int k = 0; k < P; ++k) push(k < N ? xa[k] : 0.0);  // rows 0 .. P-1 enter first
  for (int i0 = 0; i0 < N; i0 += 2 * R) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = i0 + j;
      if (i < N) {
        const int k = j + P;
        push(i + P < N ? (k < R ? xa[k] : xb[k - R]) : 0.0);
        row(i, ba[j]);
      }
    }
    load(xa, ba, i0 + 2 * R);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = i0 + R + j;
      if (i < N) {
        const int k = j + P;
        push(i + P < N ? (k < R ? xb[k] : xa[k - R]) : 0.0);
        row(i, bb[j]);
      }
    }
    load(xb, bb, i0 + 3 * R);
  }

  // ---- backward: FP32 back sweep of g, x_i += d_i
  float d1 = 0.f, d2 = 0.f;
  float ga[R], gb[R];
  double ya[R], yb[R];
  auto loadb = [&](float (&gs)[R], double (&ys)[R], int i0) {
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (i0 - j >= 0) {
        gs[j] = gp[(int64_t)(i0 - j) * ld];
        ys[j] = xp[(int64_t)(i0 - j) * ld];
      }
  };
  auto bwd = [&](float (&gs)[R], double (&ys)[R], int i0) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = i0 - j;
      if (i >= 0) {
        const float d = NativeArith<float>::step<P, true>(bw + W * i, gs[j], d1, d2);
        st_stream(xp + (int64_t)i * ld, ys[j] + widen_f32(d));
        d2 = d1;
        d1 = d;
      }
    }
  };
  loadb(ga, ya, N - 1);
  for (int i0 = N - 1; i0 >= 0; i0 -= 2 * R) {
    loadb(gb, yb, i0 - R);
    bwd(ga, ya, i0);
    loadb(ga, ya, i0 - 2 * R);
    bwd(gb, yb, i0 - R);
  }
}

template <int P, bool DFRES, typename TB>
__global__ void __launch_bounds__(512)
grouped_refine_kernel(const __grid_constant__ Groups<float, TB, double> a) {
  using AC = typename Residual<DFRES>::AC;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = group_of(a.cta_begin, a.G);
  const int N = a.N[g];
  AC* as = reinterpret_cast<AC*>(smem_raw);  // A rows first (8-byte aligned)
  float* cs = reinterpret_cast<float*>(as + NB * N);
  stage(as, static_cast<const AC*>(a.arow[g]), NB * N);
  stage(cs, a.coef[g], 2 * W * N);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  const int ctas = a.cta_begin[g + 1] - a.cta_begin[g];
  for (int64_t tile = (blockIdx.x - a.cta_begin[g]) + (int64_t)ctas * (threadIdx.x >> 5);
       tile < a.ntiles[g]; tile += (int64_t)ctas * nw)
    refine_tile<P, DFRES, kRows, TB>(cs, cs + W * N, as, N, a.M[g], a.ld[g], a.rhs[g], a.x[g],
                                     a.work[g], tile);
}

// ------------------------------------------------ staged refinement pass
//
// The same correction pass with its row streams staged through shared memory by
// cp.async: kStageRows rows of each stream are in flight per thread without
// holding them in registers.  The register-prefetched form above keeps 4 to 8 rows
// in flight per warp, and the fused solve was bound by the latency of those loads
// (more warps with fewer rows each, or fewer with more, ran no faster).  Each lane
// copies, and later reads, only its own system's values, so the thread's own
// cp.async.wait_group is the only ordering needed; a slot is refilled after the row
// read from it has been computed and its result stored.
constexpr int kStageRows = 16;
constexpr int kStageBatch = 4;  // rows taken per wait in the correction passes
constexpr int kStagedThreads = 512;  // one CTA per SM: its registers fill the SM
constexpr bool kRefinedStepStaged = true;

// Shared-memory bytes of the staging ring of a block of `threads` threads: D slots
// of an FP64 value and of a right-hand-side value per thread.
template <typename TB>
constexpr size_t stage_ring_bytes(int threads) {
  return (size_t)kStageRows * threads * (sizeof(double) + sizeof(TB));
}

template <int P, bool DFRES, typename TB>
__device__ __forceinline__ void refine_tile_staged(const float* fw, const float* bw,
                                                   const typename Residual<DFRES>::AC* arow, int N,
                                                   int64_t M, int64_t ld, const TB* b, double* x,
                                                   float* g, int64_t tile, unsigned char* ring) {
  using RS = Residual<DFRES>;
  using X = typename RS::X;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  constexpr int D = kStageRows;
  constexpr int K = kStageBatch;
  static_assert((D & (D - 1)) == 0 && D % K == 0, "the ring length is a power of two and a multiple of K");
  const int64_t m = tile * 32 + (threadIdx.x & 31);
  if (m >= M) return;
  const TB* bp = b + m;
  double* xp = x + m;
  float* gp = g + m;
  const int T = blockDim.x;
  // slot s of this thread: rx[s * T] (FP64) and rb[s * T] (a right-hand-side value,
  // or the FP32 intermediate in the backward sweep)
  double* rx = reinterpret_cast<double*>(ring) + threadIdx.x;
  TB* rb = reinterpret_cast<TB*>(ring + (size_t)D * T * sizeof(double)) + threadIdx.x;
  __threadfence_block();  // this thread's stores of x (earlier passes) before the copies read them

  // ---- forward: iteration i takes x_{i+P} (the window's new row) and b_i
  X xw[NB];  // x_{i-P} .. x_{i+P}
#pragma unroll
  for (int k = 0; k < NB; ++k) xw[k] = RS::in(0.0);
  auto push = [&](double v) {
#pragma unroll
    for (int k = 0; k < NB - 1; ++k) xw[k] = xw[k + 1];
    xw[NB - 1] = RS::in(v);
  };
#pragma unroll
  for (int k = 0; k < P; ++k) push(k < N ? xp[(int64_t)k * ld] : 0.0);  // rows 0 .. P-1 enter first
  auto issue_f = [&](int k) {
    const int s = (k & (D - 1)) * T;
    if (k + P < N) cp_async<8>(rx + s, xp + (int64_t)(k + P) * ld);
    if (k < N) cp_async<sizeof(TB)>(rb + s, bp + (int64_t)k * ld);
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue_f(k);
  // rows in batches of K: the K residuals are independent of each other and of the
  // FP32 recurrence, so their FP64 FMA chains overlap; then the K sweep steps
  float u1 = 0.f, u2 = 0.f;
  for (int i0 = 0; i0 < N; i0 += K) {
    cp_wait<D - K>();  // the groups of rows i0 .. i0+K-1 are complete
    float r[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int i = i0 + j;
      const int s = (i & (D - 1)) * T;
      push(i + P < N ? rx[s] : 0.0);
      r[j] = i < N ? RS::template eval<NB>(arow + NB * i, xw, rb[s]) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int i = i0 + j;
      if (i < N) {
        const float u = NativeArith<float>::step<P, false>(fw + W * i, r[j], u1, u2);
        gp[(int64_t)i * ld] = u;
        u2 = u1;
        u1 = u;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) issue_f(i0 + D + j);  // refills the K slots used above
  }
  cp_wait<0>();           // every group left is empty (rows past N)
  __threadfence_block();  // the stores of g before the copies that read them back

  // ---- backward: iteration k takes row i = N-1-k of g and of x; x_i += d_i
  auto issue_b = [&](int k) {
    const int i = N - 1 - k;
    const int s = (k & (D - 1)) * T;
    if (i >= 0) {
      cp_async<4>(reinterpret_cast<float*>(rb + s), gp + (int64_t)i * ld);
      cp_async<8>(rx + s, xp + (int64_t)i * ld);
    }
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue_b(k);
  float d1 = 0.f, d2 = 0.f;
  for (int k0 = 0; k0 < N; k0 += K) {
    cp_wait<D - K>();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int k = k0 + j;
      const int i = N - 1 - k;
      const int s = (k & (D - 1)) * T;
      if (i >= 0) {
        const float d =
            NativeArith<float>::step<P, true>(bw + W * i, *reinterpret_cast<const float*>(rb + s), d1, d2);
        st_stream(xp + (int64_t)i * ld, rx[s] + widen_f32(d));
        d2 = d1;
        d1 = d;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) issue_b(k0 + D + j);
  }
  cp_wait<0>();
}

// The FP32 pass x_0 = sweep32(b) with the same staging: the forward sweep streams b
// and stores its FP32 intermediate densely in the workspace g (4 bytes per element;
// the unstaged pass keeps it in x's 8-byte slots), the backward sweep streams it
// back and stores x_0 widened to FP64.  The arithmetic is that of
// sweep_tile<NativeArith<float>, P, false, true>.
template <int P, typename TB>
__device__ __forceinline__ void sweep32_tile_staged(const float* fw, const float* bw, int N, int64_t M,
                                                    int64_t ld, const TB* b, double* x, float* g,
                                                    int64_t tile, unsigned char* ring) {
  using A = NativeArith<float>;
  constexpr int W = P + 1;
  constexpr int D = kStageRows;
  const int64_t m = tile * 32 + (threadIdx.x & 31);
  if (m >= M) return;
  const TB* bp = b + m;
  double* xp = x + m;
  float* gp = g + m;
  const int T = blockDim.x;
  TB* rb = reinterpret_cast<TB*>(ring + (size_t)D * T * sizeof(double)) + threadIdx.x;
  __threadfence_block();  // this thread's earlier stores of g before the copies below

  auto issue_f = [&](int k) {
    if (k < N) cp_async<sizeof(TB)>(rb + (k & (D - 1)) * T, bp + (int64_t)k * ld);
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue_f(k);
  float u1 = 0.f, u2 = 0.f;
  for (int i = 0; i < N; ++i) {
    cp_wait<D - 1>();
    const float u = A::step<P, false>(fw + W * i, Conv<A, TB>::in(rb[(i & (D - 1)) * T]), u1, u2);
    gp[(int64_t)i * ld] = u;
    u2 = u1;
    u1 = u;
    issue_f(i + D);
  }
  cp_wait<0>();
  __threadfence_block();  // the stores of g before the copies that read them back

  auto issue_b = [&](int k) {
    const int i = N - 1 - k;
    if (i >= 0) cp_async<4>(reinterpret_cast<float*>(rb + (k & (D - 1)) * T), gp + (int64_t)i * ld);
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue_b(k);
  float x1 = 0.f, x2 = 0.f;
  for (int k = 0; k < N; ++k) {
    cp_wait<D - 1>();
    const int i = N - 1 - k;
    const float xi = A::step<P, true>(bw + W * i, *reinterpret_cast<const float*>(rb + (k & (D - 1)) * T), x1, x2);
    st_stream(xp + (int64_t)i * ld, widen_f32(xi));
    x2 = x1;
    x1 = xi;
    issue_b(k + D);
  }
  cp_wait<0>();
}

// All passes in one launch: each warp takes a tile and runs the FP32 pass (x_0 into
// x) and then the n_refine correction passes on it, before its next tile.  Tiles are
// independent, so no pass waits for another tile; warps drift into different passes,
// so the FP64 residual arithmetic of some overlaps the memory phases of others.
// Rows per prefetch batch of the fused kernel: 4 (not kRows) keeps every pass within
// 128 registers, so two 256-thread CTAs share an SM.
constexpr int kFusedRows = 4;

// STAGED: the correction passes stream their rows through a shared-memory ring
// (refine_tile_staged; 512 threads, one CTA per SM) placed after the coefficients at
// ring_off bytes; otherwise the register-prefetched passes (256 threads, two CTAs).
template <int P, bool DFRES, typename TB, bool STAGED>
__global__ void __launch_bounds__(STAGED ? kStagedThreads : 256, STAGED ? 1 : 2)
grouped_refined_solve_kernel(const __grid_constant__ Groups<float, TB, double> a, int n_refine,
                             unsigned ring_off) {
  using AC = typename Residual<DFRES>::AC;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = group_of(a.cta_begin, a.G);
  const int N = a.N[g];
  AC* as = reinterpret_cast<AC*>(smem_raw);  // A rows first (8-byte aligned)
  float* cs = reinterpret_cast<float*>(as + NB * N);
  stage(as, static_cast<const AC*>(a.arow[g]), NB * N);
  stage(cs, a.coef[g], 2 * W * N);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  const int ctas = a.cta_begin[g + 1] - a.cta_begin[g];
  for (int64_t tile = (blockIdx.x - a.cta_begin[g]) + (int64_t)ctas * (threadIdx.x >> 5);
       tile < a.ntiles[g]; tile += (int64_t)ctas * nw) {
    if constexpr (STAGED)
      sweep32_tile_staged<P, TB>(cs, cs + W * N, N, a.M[g], a.ld[g], a.rhs[g], a.x[g], a.work[g], tile,
                                 smem_raw + ring_off);
    else
      sweep_tile<NativeArith<float>, P, false, true, TB, double, 1, kFusedRows>(cs, cs + W * N, N, a.M[g],
                                                                              a.ld[g], a.rhs[g], a.x[g], tile);
    for (int k = 0; k < n_refine; ++k) {
      if constexpr (STAGED)
        refine_tile_staged<P, DFRES, TB>(cs, cs + W * N, as, N, a.M[g], a.ld[g], a.rhs[g], a.x[g], a.work[g],
                                         tile, smem_raw + ring_off);
      else
        refine_tile<P, DFRES, kFusedRows, TB>(cs, cs + W * N, as, N, a.M[g], a.ld[g], a.rhs[g], a.x[g],
                                              a.work[g], tile);
    }
  }
}

// ------------------------------------------------ fused refinement passes
//
// The same solve with each correction pass's residual and forward sweep merged
// into the backward sweep of the pass before it, which already delivers x row by
// row.  For that, pass k eliminates from the top (the rows of A = LU) when k is
// even and from the bottom (the rows of J A J, J the exchange matrix) when k is
// odd, so that its forward sweep runs in the direction in which pass k-1's backward
// sweep produces x:
//   pass 0:              forward sweep of b into g (rows 0 .. N-1)
//   merged pass k >= 1:  pass k-1's backward sweep of g gives d_i and
//                        x_{k-1,i} = x_{k-2,i} + d_i (stored); P rows behind it the
//                        residual r_j = b_j - (A x_{k-1})_j and pass k's forward step
//                        at row j, into the row of g that was read P iterations before
//   last:                pass n's backward sweep, x_n = x_{n-1} + d.
// Bytes per element with n = 2: 4 + 4, then 4 + 8 + 4 + 4 (k = 1: x_0 is not read),
// 4 + 8 + 8 + 4 + 4 and 4 + 8 + 8: 76, against 92 for separate passes.  The FP64
// work (the residuals and the additions to x) is the same.  Each lane copies and
// reads only its own system's values, as in the staged passes above.

// One merged pass (k >= 1): DOWN when pass k-1 eliminated from the top, i.e. its
// backward sweep runs from row N-1 down.  bw: backward rows of pass k-1; fw: forward
// rows of pass k (both at A's row indices); FIRST: k == 1 (x_0 = d, nothing to add).
template <int P, bool DFRES, typename TB, int D, bool DOWN, bool FIRST>
__device__ __forceinline__ void fused_merged_pass(const float* bw, const float* fw,
                                                  const typename Residual<DFRES>::AC* arow, int N, int64_t ld,
                                                  const TB* bp, double* xp, float* gp, double* rx, float* rg,
                                                  TB* rb, int T) {
  using RS = Residual<DFRES>;
  using X = typename RS::X;
  using F = NativeArith<float>;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  constexpr int K = kStageBatch;
  // iteration s takes row(s) of g (and of x_{k-2}) and row(s - P) of b
  auto row = [&](int s) { return DOWN ? N - 1 - s : s; };
  auto issue = [&](int s) {
    const int sl = (s & (D - 1)) * T;
    if (s < N) {
      const int i = row(s);
      cp_async<4>(rg + sl, gp + (int64_t)i * ld);
      if (!FIRST) cp_async<8>(rx + sl, xp + (int64_t)i * ld);
    }
    if (s >= P && s < N + P) cp_async<sizeof(TB)>(rb + sl, bp + (int64_t)row(s - P) * ld);
    cp_commit();
  };
  // window x_{j-P} .. x_{j+P} of the residual's row j: the newest value enters at
  // the low end going down and at the high end going up; rows outside 0..N-1 are 0
  X xw[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) xw[q] = RS::in(0.0);
  auto push = [&](double v) {
    if constexpr (DOWN) {
#pragma unroll
      for (int q = NB - 1; q > 0; --q) xw[q] = xw[q - 1];
      xw[0] = RS::in(v);
    } else {
#pragma unroll
      for (int q = 0; q < NB - 1; ++q) xw[q] = xw[q + 1];
      xw[NB - 1] = RS::in(v);
    }
  };
#pragma unroll
  for (int s = 0; s < D; ++s) issue(s);
  float d1 = 0.f, d2 = 0.f, u1 = 0.f, u2 = 0.f;
  // rows s0 .. s0+K-1; GUARD: test them against 0 .. N-1 and the lag
  auto batch = [&](int s0, auto guard) {
    constexpr bool GUARD = decltype(guard)::value;
    cp_wait<D - K>();  // the groups of iterations s0 .. s0+K-1 are complete
    float r[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int s = s0 + q;
      const int sl = (s & (D - 1)) * T;
      double xi = 0.0;
      if (!GUARD || s < N) {
        const int i = row(s);
        const float d = F::step<P, true>(bw + W * i, rg[sl], d1, d2);
        d2 = d1;
        d1 = d;
        xi = FIRST ? widen_f32(d) : rx[sl] + widen_f32(d);
        st_stream(xp + (int64_t)i * ld, xi);
      }
      push(xi);
      r[q] = (!GUARD || (s >= P && s < N + P)) ? RS::template eval<NB>(arow + NB * row(s - P), xw, rb[sl]) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int s = s0 + q;
      if (!GUARD || (s >= P && s < N + P)) {
        const int j = row(s - P);
        const float u = F::step<P, false>(fw + W * j, r[q], u1, u2);
        gp[(int64_t)j * ld] = u;
        u2 = u1;
        u1 = u;
      }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) issue(s0 + D + q);  // refills the K slots used above
  };
  static_assert(K >= P, "the first batch covers the P rows of lag");
  batch(0, std::true_type{});
  int s0 = K;
  for (; s0 + K <= N; s0 += K) batch(s0, std::false_type{});
  for (; s0 < N + P; s0 += K) batch(s0, std::true_type{});
  cp_wait<0>();
  __threadfence_block();  // the stores of g and x before the copies of the next pass
}

// The last backward sweep: x_i = x_{n-1,i} + d_i (x_i = d_i when FIRST, n = 0).
template <int P, int D, bool DOWN, bool FIRST>
__device__ __forceinline__ void fused_last_pass(const float* bw, int N, int64_t ld, double* xp, float* gp,
                                                double* rx, float* rg, int T) {
  using F = NativeArith<float>;
  constexpr int W = P + 1;
  constexpr int K = kStageBatch;
  auto row = [&](int s) { return DOWN ? N - 1 - s : s; };
  auto issue = [&](int s) {
    const int sl = (s & (D - 1)) * T;
    if (s < N) {
      const int i = row(s);
      cp_async<4>(rg + sl, gp + (int64_t)i * ld);
      if (!FIRST) cp_async<8>(rx + sl, xp + (int64_t)i * ld);
    }
    cp_commit();
  };
#pragma unroll
  for (int s = 0; s < D; ++s) issue(s);
  float d1 = 0.f, d2 = 0.f;
  auto batch = [&](int s0, auto guard) {
    constexpr bool GUARD = decltype(guard)::value;
    cp_wait<D - K>();
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int s = s0 + q;
      if (!GUARD || s < N) {
        const int sl = (s & (D - 1)) * T;
        const int i = row(s);
        const float d = F::step<P, true>(bw + W * i, rg[sl], d1, d2);
        d2 = d1;
        d1 = d;
        st_stream(xp + (int64_t)i * ld, FIRST ? widen_f32(d) : rx[sl] + widen_f32(d));
      }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) issue(s0 + D + q);
  };
  int s0 = 0;
  for (; s0 + K <= N; s0 += K) batch(s0, std::false_type{});
  for (; s0 < N; s0 += K) batch(s0, std::true_type{});
  cp_wait<0>();
}

// Shared-memory bytes of the fused form's ring: D slots per thread of an FP64 value,
// an FP32 intermediate and a right-hand-side value.
template <typename TB>
constexpr size_t fused_ring_bytes(int D, int threads) {
  return (size_t)D * threads * (sizeof(double) + sizeof(float) + sizeof(TB));
}

// cf: rows [forward | backward] of A = LU; cr: the same of J A J at A's row indices.
template <int P, bool DFRES, typename TB, int D>
__device__ __forceinline__ void refine_fused_tile(const float* cf, const float* cr,
                                                  const typename Residual<DFRES>::AC* arow, int N, int64_t M,
                                                  int64_t ld, const TB* b, double* x, float* g, int64_t tile,
                                                  unsigned char* ring, int n_refine) {
  using F = NativeArith<float>;
  constexpr int W = P + 1;
  static_assert((D & (D - 1)) == 0 && D % kStageBatch == 0, "the ring length is a power of two and a multiple of K");
  const int64_t m = tile * 32 + (threadIdx.x & 31);
  if (m >= M) return;
  const TB* bp = b + m;
  double* xp = x + m;
  float* gp = g + m;
  const int T = blockDim.x;
  double* rx = reinterpret_cast<double*>(ring) + threadIdx.x;
  float* rg = reinterpret_cast<float*>(ring + (size_t)D * T * sizeof(double)) + threadIdx.x;
  TB* rb = reinterpret_cast<TB*>(ring + (size_t)D * T * (sizeof(double) + sizeof(float))) + threadIdx.x;
  __threadfence_block();  // this thread's stores of an earlier tile before the copies below

  // pass 0: forward sweep of b (from the top) into g
  {
    auto issue = [&](int k) {
      if (k < N) cp_async<sizeof(TB)>(rb + (k & (D - 1)) * T, bp + (int64_t)k * ld);
      cp_commit();
    };
#pragma unroll
    for (int k = 0; k < D; ++k) issue(k);
    float u1 = 0.f, u2 = 0.f;
    for (int i = 0; i < N; ++i) {
      cp_wait<D - 1>();
      const float u = F::step<P, false>(cf + W * i, Conv<F, TB>::in(rb[(i & (D - 1)) * T]), u1, u2);
      gp[(int64_t)i * ld] = u;
      u2 = u1;
      u1 = u;
      issue(i + D);
    }
    cp_wait<0>();
    __threadfence_block();
  }
  const float* lu_f = cf;
  const float* lu_b = cf + W * N;
  const float* ul_f = cr;
  const float* ul_b = cr + W * N;
  for (int k = 1; k <= n_refine; ++k) {
    if (k == 1)
      fused_merged_pass<P, DFRES, TB, D, true, true>(lu_b, ul_f, arow, N, ld, bp, xp, gp, rx, rg, rb, T);
    else if (k & 1)
      fused_merged_pass<P, DFRES, TB, D, true, false>(lu_b, ul_f, arow, N, ld, bp, xp, gp, rx, rg, rb, T);
    else
      fused_merged_pass<P, DFRES, TB, D, false, false>(ul_b, lu_f, arow, N, ld, bp, xp, gp, rx, rg, rb, T);
  }
  if (n_refine == 0)
    fused_last_pass<P, D, true, true>(lu_b, N, ld, xp, gp, rx, rg, T);
  else if (n_refine & 1)
    fused_last_pass<P, D, false, false>(ul_b, N, ld, xp, gp, rx, rg, T);
  else
    fused_last_pass<P, D, true, false>(lu_b, N, ld, xp, gp, rx, rg, T);
}

template <int P, bool DFRES, typename TB, int D>
__global__ void __launch_bounds__(kStagedThreads, 1)
grouped_refined_fused_kernel(const __grid_constant__ Groups<float, TB, double> a, int n_refine,
                             unsigned ring_off) {
  using AC = typename Residual<DFRES>::AC;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = group_of(a.cta_begin, a.G);
  const int N = a.N[g];
  AC* as = reinterpret_cast<AC*>(smem_raw);  // A rows first (8-byte aligned)
  float* cs = reinterpret_cast<float*>(as + NB * N);
  float* crs = cs + 2 * W * N;
  stage(as, static_cast<const AC*>(a.arow[g]), NB * N);
  stage(cs, a.coef[g], 2 * W * N);
  stage(crs, a.rcoef[g], 2 * W * N);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  const int ctas = a.cta_begin[g + 1] - a.cta_begin[g];
  for (int64_t tile = (blockIdx.x - a.cta_begin[g]) + (int64_t)ctas * (threadIdx.x >> 5);
       tile < a.ntiles[g]; tile += (int64_t)ctas * nw)
    refine_fused_tile<P, DFRES, TB, D>(cs, crs, as, N, a.M[g], a.ld[g], a.rhs[g], a.x[g], a.work[g], tile,
                                       smem_raw + ring_off, n_refine);
}

// ------------------------------------------- paired tiles, two refinements
//
// With two correction passes a tile goes through four sweeps: pass 0's forward
// sweep (up, no FP64 work), the first merged pass (down, 3 FP64 operations per
// element for a tridiagonal A), the second (up, 4) and the last backward sweep
// (down, 1).  A warp whose tiles all sit in the same sweep leaves the FP64 pipe
// idle in the first and the last one.  Here a warp carries two tiles two sweeps
// apart, so every loop runs sweeps 0 and 2, or 1 and 3, of two different tiles
// side by side: both in the same direction, with 4 FP64 operations per element
// pair in every loop (and 36 or 40 bytes).  Tile k of the warp runs its sweep p in step
// 2k + p; steps 0, 1 and the last two carry a single tile.

struct TileRef {
  const float* b;
  double* x;
  float* g;
  bool ok;  // this lane's system exists (the last tile may be ragged)
};

// Shared-memory bytes of the paired form's ring: D slots per thread of an FP64
// value and three FP32 values.
constexpr size_t pair_ring_bytes(int D, int threads) {
  return (size_t)D * threads * (sizeof(double) + 3 * sizeof(float));
}

// One step: ODD == false runs sweep 0 of tile A and sweep 2 of tile B (upwards),
// ODD == true sweep 1 of A and sweep 3 of B (downwards); HA / HB: the warp has tile
// A / B in this step.  Ring use per slot: even steps b of A (f1), g and x of B (f2,
// rx) and B's b, P rows behind (f3); odd steps g of A (f1), A's b, P rows behind
// (f2), g and x of B (f3, rx).  The batches between the first and the last take
// every row without the range tests.
template <int P, bool DFRES, int D, bool ODD, bool HA, bool HB>
__device__ __forceinline__ void pair_step(const float* cf, const float* cr,
                                          const typename Residual<DFRES>::AC* arow, int N, int64_t ld,
                                          const TileRef& A, const TileRef& B, double* rx, float* f1, float* f2,
                                          float* f3, int T) {
  using RS = Residual<DFRES>;
  using X = typename RS::X;
  using F = NativeArith<float>;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  constexpr int K = kStageBatch;
  static_assert(K >= P, "the first batch covers the P rows of lag");
  constexpr bool RES = ODD ? HA : HB;  // the tile in a merged sweep
  const float* lu_f = cf;
  const float* lu_b = cf + W * N;
  const float* ul_f = cr;
  const float* ul_b = cr + W * N;
  const bool a = HA && A.ok, b = HB && B.ok;  // this lane copies and stores
  auto row = [&](int s) { return ODD ? N - 1 - s : s; };
  auto issue = [&](int s) {
    const int sl = (s & (D - 1)) * T;
    if (s < N) {
      const int64_t i = row(s);
      if (!ODD) {
        if (a) cp_async<4>(f1 + sl, A.b + i * ld);
        if (b) {
          cp_async<4>(f2 + sl, B.g + i * ld);
          cp_async<8>(rx + sl, B.x + i * ld);
        }
      } else {
        if (a) cp_async<4>(f1 + sl, A.g + i * ld);
        if (b) {
          cp_async<4>(f3 + sl, B.g + i * ld);
          cp_async<8>(rx + sl, B.x + i * ld);
        }
      }
    }
    if (RES && s >= P && s < N + P) {
      const int64_t j = row(s - P);
      if (!ODD && b) cp_async<4>(f3 + sl, B.b + j * ld);
      if (ODD && a) cp_async<4>(f2 + sl, A.b + j * ld);
    }
    cp_commit();
  };
  // the residual's window (of B going up, of A going down); rows outside are 0
  X xw[NB];
#pragma unroll
  for (int q = 0; q < NB; ++q) xw[q] = RS::in(0.0);
  auto push = [&](double v) {
    if constexpr (ODD) {
#pragma unroll
      for (int q = NB - 1; q > 0; --q) xw[q] = xw[q - 1];
      xw[0] = RS::in(v);
    } else {
#pragma unroll
      for (int q = 0; q < NB - 1; ++q) xw[q] = xw[q + 1];
      xw[NB - 1] = RS::in(v);
    }
  };
#pragma unroll
  for (int s = 0; s < D; ++s) issue(s);
  float ua1 = 0.f, ua2 = 0.f, da1 = 0.f, da2 = 0.f;  // tile A: forward, backward recurrences
  float ub1 = 0.f, ub2 = 0.f, db1 = 0.f, db2 = 0.f;  // tile B
  // rows s0 .. s0+K-1; GUARD: test them against 0 .. N-1 and the lag
  auto batch = [&](int s0, auto guard) {
    constexpr bool GUARD = decltype(guard)::value;
    cp_wait<D - K>();  // the groups of iterations s0 .. s0+K-1 are complete
    float r[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int s = s0 + q;
      const int sl = (s & (D - 1)) * T;
      double xi = 0.0;
      if (!GUARD || s < N) {
        const int64_t i = row(s);
        if constexpr (!ODD) {
          if constexpr (HA) {  // A, sweep 0: forward from the top
            const float u = F::step<P, false>(lu_f + W * i, f1[sl], ua1, ua2);
            ua2 = ua1;
            ua1 = u;
            if (a) A.g[i * ld] = u;
          }
          if constexpr (HB) {  // B, sweep 2: backward of pass 1 (bottom elimination), x_1 = x_0 + d
            const float d = F::step<P, true>(ul_b + W * i, f2[sl], db1, db2);
            db2 = db1;
            db1 = d;
            xi = rx[sl] + widen_f32(d);
            if (b) st_stream(B.x + i * ld, xi);
          }
        } else {
          if constexpr (HB) {  // B, sweep 3: backward of pass 2, x_2 = x_1 + d
            const float d = F::step<P, true>(lu_b + W * i, f3[sl], db1, db2);
            db2 = db1;
            db1 = d;
            if (b) st_stream(B.x + i * ld, rx[sl] + widen_f32(d));
          }
          if constexpr (HA) {  // A, sweep 1: backward of pass 0, x_0 = d
            const float d = F::step<P, true>(lu_b + W * i, f1[sl], da1, da2);
            da2 = da1;
            da1 = d;
            xi = widen_f32(d);
            if (a) st_stream(A.x + i * ld, xi);
          }
        }
      }
      if constexpr (RES) {
        push(xi);
        r[q] = (!GUARD || (s >= P && s < N + P))
                   ? RS::template eval<NB>(arow + NB * row(s - P), xw, ODD ? f2[sl] : f3[sl])
                   : 0.f;
      }
    }
    if constexpr (RES) {
#pragma unroll
      for (int q = 0; q < K; ++q) {
        const int s = s0 + q;
        if (!GUARD || (s >= P && s < N + P)) {
          const int64_t j = row(s - P);
          if constexpr (!ODD) {  // B: pass 2's forward step (top elimination)
            const float u = F::step<P, false>(lu_f + W * j, r[q], ub1, ub2);
            ub2 = ub1;
            ub1 = u;
            if (b) B.g[j * ld] = u;
          } else {  // A: pass 1's forward step (bottom elimination)
            const float u = F::step<P, false>(ul_f + W * j, r[q], ua1, ua2);
            ua2 = ua1;
            ua1 = u;
            if (a) A.g[j * ld] = u;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) issue(s0 + D + q);  // refills the K slots used above
  };
  const int last = RES ? N + P : N;  // iterations of this step
  batch(0, std::true_type{});
  int s0 = K;
  for (; s0 + K <= N; s0 += K) batch(s0, std::false_type{});
  for (; s0 < last; s0 += K) batch(s0, std::true_type{});
  cp_wait<0>();
  __threadfence_block();  // the stores of g and x before the copies of the next step
}

template <int P, bool DFRES, int D>
__global__ void __launch_bounds__(kStagedThreads, 1)
grouped_refined_pair_kernel(const __grid_constant__ Groups<float, float, double> a, unsigned ring_off) {
  using AC = typename Residual<DFRES>::AC;
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = group_of(a.cta_begin, a.G);
  const int N = a.N[g];
  AC* as = reinterpret_cast<AC*>(smem_raw);  // A rows first (8-byte aligned)
  float* cs = reinterpret_cast<float*>(as + NB * N);
  float* crs = cs + 2 * W * N;
  stage(as, static_cast<const AC*>(a.arow[g]), NB * N);
  stage(cs, a.coef[g], 2 * W * N);
  stage(crs, a.rcoef[g], 2 * W * N);
  __syncthreads();
  const int T = blockDim.x;
  unsigned char* ring = smem_raw + ring_off;
  double* rx = reinterpret_cast<double*>(ring) + threadIdx.x;
  float* f1 = reinterpret_cast<float*>(ring + (size_t)D * T * sizeof(double)) + threadIdx.x;
  float* f2 = f1 + D * T;
  float* f3 = f2 + D * T;
  const int nw = blockDim.x >> 5;
  const int ctas = a.cta_begin[g + 1] - a.cta_begin[g];
  const int64_t first = (blockIdx.x - a.cta_begin[g]) + (int64_t)ctas * (threadIdx.x >> 5);
  const int64_t stride = (int64_t)ctas * nw;
  const int64_t ntiles = a.ntiles[g];
  const int64_t nt = first < ntiles ? (ntiles - first + stride - 1) / stride : 0;  // this warp's tiles
  const int64_t M = a.M[g], ld = a.ld[g];
  auto ref = [&](int64_t k) {
    const int64_t m = (first + k * stride) * 32 + (threadIdx.x & 31);
    return TileRef{a.rhs[g] + m, a.x[g] + m, a.work[g] + m, m < M};
  };
  for (int64_t s = 0; nt > 0 && s < 2 * nt + 2; ++s) {
    const int64_t ka = s >> 1, kb = ka - 1;  // tile in sweep s % 2, tile in sweep s % 2 + 2
    const bool hasA = ka < nt, hasB = kb >= 0;
    const TileRef A = ref(hasA ? ka : 0), B = ref(hasB ? kb : 0);
    if (s & 1) {
      if (hasA && hasB)
        pair_step<P, DFRES, D, true, true, true>(cs, crs, as, N, ld, A, B, rx, f1, f2, f3, T);
      else if (hasA)
        pair_step<P, DFRES, D, true, true, false>(cs, crs, as, N, ld, A, B, rx, f1, f2, f3, T);
      else
        pair_step<P, DFRES, D, true, false, true>(cs, crs, as, N, ld, A, B, rx, f1, f2, f3, T);
    } else {
      if (hasA && hasB)
        pair_step<P, DFRES, D, false, true, true>(cs, crs, as, N, ld, A, B, rx, f1, f2, f3, T);
      else if (hasA)
        pair_step<P, DFRES, D, false, true, false>(cs, crs, as, N, ld, A, B, rx, f1, f2, f3, T);
      else
        pair_step<P, DFRES, D, false, false, true>(cs, crs, as, N, ld, A, B, rx, f1, f2, f3, T);
    }
  }
}

// ---------------------------------------------------- refined time step

// Right-hand side of a time step for one tile, in FP64, in the same order of
// operations as the stepper's right-hand-side kernel: f_i = sum_k B_ik C_k (NB
// values per row at offsets -(NB/2)..NB/2; f_i = C_i when NB == 0) plus, with
// HAS_E, sum_k E_ik (C_k^3 - C_k) over offsets -1..1.  Rows outside the matrix
// are 0.  C is read ahead in double-buffered batches of R rows.
template <int NB, bool HAS_E, int R>
__device__ __forceinline__ void rhs_tile(const double* rc, int N, int64_t M, int64_t ld, const double* Cin,
                                         double* f, int64_t tile) {
  using A = NativeArith<double>;
  constexpr int RW = NB + (HAS_E ? 3 : 0);
  const int64_t m = tile * 32 + (threadIdx.x & 31);
  if (m >= M) return;
  const double* cp = Cin + m;
  double* fp = f + m;
  auto row_c = [&](int k) { return (k >= 0 && k < N) ? ld_stream(cp + (int64_t)k * ld) : 0.0; };
  double w[5] = {0.0, 0.0, row_c(0), row_c(1), row_c(2)};  // rows i-2 .. i+2
  double na[R], nb[R];
  auto load = [&](double (&b)[R], int i0) {
#pragma unroll
    for (int j = 0; j < R; ++j) b[j] = row_c(i0 + 3 + j);
  };
  auto rows = [&](const double (&b)[R], int i0) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int i = i0 + j;
      if (i < N) {
        const double* rw = rc + RW * i;
        double r;
        if constexpr (NB > 0) {
          r = A::mulc(rw[0], w[2 - NB / 2]);
#pragma unroll
          for (int k = 1; k < NB; ++k) r = A::fmac(rw[k], w[2 - NB / 2 + k], r);
        } else {
          r = w[2];
        }
        if constexpr (HAS_E) {
#pragma unroll
          for (int k = 0; k < 3; ++k) r = A::fmac(rw[NB + k], A::cubic(w[1 + k]), r);
        }
        fp[(int64_t)i * ld] = r;
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = w[k + 1];
        w[4] = b[j];
      }
    }
  };
  load(na, 0);
  for (int i0 = 0; i0 < N; i0 += 2 * R) {
    load(nb, i0 + R);
    rows(na, i0);
    load(na, i0 + 2 * R);
    rows(nb, i0 + R);
  }
}

// One FP32 + refinement time step in one launch: each warp takes a tile of the
// state C through its right-hand side f (FP64, into the workspace), the FP32 solve
// of f into C (in place: the tile's C is read completely first) and n_refine
// correction passes with the FP64 f.  a.G == 1, a.rhs[0] == f, a.x[0] == C.
// STAGED: the FP32 pass and the correction passes stream their rows through the
// shared-memory ring at ring_off (512 threads, one CTA per SM), as in the grouped
// refined solve.
// FORM 0: register-prefetched passes (256 threads, two CTAs per SM); 1: passes
// staged through the shared-memory ring; 2: the merged passes of
// refine_fused_tile with a ring of D rows (the rows of J A J staged after the
// FP32 sweep rows).
template <int P, bool DFRES, int NB, bool HAS_E, int FORM, int D = 16>
__global__ void __launch_bounds__(FORM > 0 ? kStagedThreads : 256, FORM > 0 ? 1 : 2)
refined_step_kernel(const __grid_constant__ Groups<float, double, double> a, double* f,
                    const double* __restrict__ rcoef, int n_refine, unsigned ring_off) {
  using AC = typename Residual<DFRES>::AC;
  constexpr bool STAGED = FORM == 1;
  constexpr int W = P + 1;
  constexpr int NBA = 2 * P + 1;
  constexpr int RW = NB + (HAS_E ? 3 : 0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = a.N[0];
  AC* as = reinterpret_cast<AC*>(smem_raw);          // A rows (8-byte values)
  float* cs = reinterpret_cast<float*>(as + NBA * N);  // FP32 sweep rows
  float* crs = cs + 2 * W * N;                         // the same of J A J (FORM 2)
  double* rs = reinterpret_cast<double*>(cs + (FORM == 2 ? 4 : 2) * W * N);  // right-hand-side rows (8-byte aligned)
  stage(as, static_cast<const AC*>(a.arow[0]), NBA * N);
  stage(cs, a.coef[0], 2 * W * N);
  if constexpr (FORM == 2) stage(crs, a.rcoef[0], 2 * W * N);
  stage(rs, rcoef, RW * N);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5); tile < a.ntiles[0];
       tile += (int64_t)gridDim.x * nw) {
    rhs_tile<NB, HAS_E, kFusedRows>(rs, N, a.M[0], a.ld[0], a.x[0], f, tile);
    if constexpr (FORM == 2) {
      refine_fused_tile<P, DFRES, double, D>(cs, crs, as, N, a.M[0], a.ld[0], f, a.x[0], a.work[0], tile,
                                             smem_raw + ring_off, n_refine);
    } else if constexpr (STAGED) {
      sweep32_tile_staged<P, double>(cs, cs + W * N, N, a.M[0], a.ld[0], f, a.x[0], a.work[0], tile,
                                     smem_raw + ring_off);
      for (int k = 0; k < n_refine; ++k)
        refine_tile_staged<P, DFRES, double>(cs, cs + W * N, as, N, a.M[0], a.ld[0], f, a.x[0], a.work[0], tile,
                                             smem_raw + ring_off);
    } else {
      sweep_tile<NativeArith<float>, P, false, true, double, double, 1, kFusedRows>(cs, cs + W * N, N, a.M[0],
                                                                                  a.ld[0], f, a.x[0], tile);
      for (int k = 0; k < n_refine; ++k)
        refine_tile<P, DFRES, kFusedRows, double>(cs, cs + W * N, as, N, a.M[0], a.ld[0], f, a.x[0], a.work[0],
                                                  tile);
    }
  }
}

// ------------------------------------------------------------------ host

constexpr int kThreads = 256;

template <typename K>
int resident_ctas(K kernel, int device, size_t smem, int* total, int threads = kThreads) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, size_t, int>, int> cache;
  int nb = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(reinterpret_cast<const void*>(kernel), smem, threads);
    auto it = cache.find(key);
    if (it != cache.end()) {
      nb = it->second;
    } else {
      SB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
      SB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem));
      cache[key] = nb;
    }
  }
  if (nb < 1) return fail(SB_ERR_UNSUPPORTED, "grouped kernel cannot be resident (%zu B smem)", smem);
  *total = nb * sm_count(device);
  return SB_OK;
}

// Splits `total` CTAs over the groups in proportion to N*M (each group gets at
// least one CTA and no more than it has tiles for).  Returns the grid size.
template <typename GA>
int plan(GA& a, const std::vector<const sb_factor*>& f, int total) {
  double work = 0.0;
  for (int g = 0; g < a.G; ++g) work += (double)f[g]->N * (double)a.M[g];
  int begin = 0;
  for (int g = 0; g < a.G; ++g) {
    const int64_t need = a.ntiles[g];
    int64_t share = (int64_t)std::llround(total * ((double)f[g]->N * (double)a.M[g]) / work);
    share = std::max<int64_t>(1, std::min<int64_t>(share, need));
    a.cta_begin[g] = begin;
    begin += (int)share;
  }
  a.cta_begin[a.G] = begin;
  return begin;
}

template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO>
int launch_grouped_sweep(const std::vector<const sb_factor*>& f, Op op,
                         const std::vector<const void*>& rhs, const std::vector<void*>& x,
                         const std::vector<int64_t>& M, const std::vector<int64_t>& ld,
                         const typename A::C* const* coefs, cudaStream_t stream) {
  using C = typename A::C;
  Groups<C, TI, TO> a{};
  a.G = (int)f.size();
  size_t smem = 0;
  for (int g = 0; g < a.G; ++g) {
    a.coef[g] = coefs[g] + (op == OP_PRIMAL ? 0 : op_block_len(P, f[g]->N));
    a.N[g] = (int)f[g]->N;
    a.M[g] = M[g];
    a.ld[g] = ld[g];
    a.ntiles[g] = (M[g] + 31) / 32;
    a.rhs[g] = static_cast<const TI*>(rhs[g]);
    a.x[g] = static_cast<TO*>(x[g]);
    smem = std::max(smem, (size_t)2 * (P + 1) * f[g]->N * sizeof(C));
  }
  if (smem > 227 * 1024) return fail(SB_ERR_UNSUPPORTED, "a group's factors exceed shared memory");
  auto k = grouped_sweep_kernel<A, P, F_ONE, B_ONE, TI, TO>;
  int total = 0;
  SB_TRY(resident_ctas(k, f[0]->device, smem, &total));
  const int grid = plan(a, f, total);
  k<<<grid, kThreads, smem, stream>>>(a);
  return cuda_check(cudaGetLastError(), "grouped sweep launch");
}

template <int P, bool DFRES, typename TB>
int launch_grouped_refined_solve(const std::vector<const sb_factor*>& f, const std::vector<const void*>& rhs,
                                 const std::vector<void*>& x, const std::vector<int64_t>& M,
                                 const std::vector<int64_t>& ld, const std::vector<void*>& work, int n_refine,
                                 cudaStream_t stream) {
  using AC = typename Residual<DFRES>::AC;
  Groups<float, TB, double> a{};
  a.G = (int)f.size();
  size_t smem = 0;
  for (int g = 0; g < a.G; ++g) {
    a.coef[g] = f[g]->coef32;  // primal block
    a.arow[g] = DFRES ? static_cast<const void*>(f[g]->arowdf) : static_cast<const void*>(f[g]->arow64);
    a.N[g] = (int)f[g]->N;
    a.M[g] = M[g];
    a.ld[g] = ld[g];
    a.ntiles[g] = (M[g] + 31) / 32;
    a.rhs[g] = static_cast<const TB*>(rhs[g]);
    a.x[g] = static_cast<double*>(x[g]);
    a.work[g] = static_cast<float*>(work[g]);
    smem = std::max(smem, (size_t)(2 * P + 1) * f[g]->N * sizeof(AC) +
                              (size_t)2 * (P + 1) * f[g]->N * sizeof(float));
  }
  if (smem > 227 * 1024) return fail(SB_ERR_UNSUPPORTED, "a group's factors exceed shared memory");
  // the fused passes (FP32 right-hand sides) when every group has the rows of J A J
  // and both coefficient sets and a ring of 16, else 8, rows fit in shared memory
  if constexpr (std::is_same<TB, float>::value) {
    bool fused = n_refine > 0;
    size_t fsmem = 0;
    for (int g = 0; g < a.G; ++g) {
      fused = fused && f[g]->coef32_rev != nullptr;
      a.rcoef[g] = f[g]->coef32_rev;
      fsmem = std::max(fsmem, (size_t)(2 * P + 1) * f[g]->N * sizeof(AC) +
                                  (size_t)4 * (P + 1) * f[g]->N * sizeof(float));
    }
    const size_t foff = (fsmem + 15) / 16 * 16;
    // two refinements with the FP64 residual: tiles paired two sweeps apart, with an
    // 8-row ring and as many threads (256 to 512) as fit beside the coefficients.
    // (A 16-row ring spills registers: 21.0 against 16.3 ms on the 3-group
    // workload.  The double-float residual leaves the FP64 pipe idle anyway and is
    // bound by instruction issue, which the paired loops raise: it takes the
    // single-tile form below.)
    if (!DFRES && fused && n_refine == 2 && foff < (size_t)kMaxDynSmem) {
      const size_t room = (size_t)kMaxDynSmem - foff;
      const int threads = (int)std::min<size_t>(kStagedThreads, room / pair_ring_bytes(8, 1) / 32 * 32);
      if (threads >= 256) {
        const size_t total_smem = foff + pair_ring_bytes(8, threads);
        auto k = grouped_refined_pair_kernel<P, false, 8>;
        int total = 0;
        SB_TRY(resident_ctas(k, f[0]->device, total_smem, &total, threads));
        const int grid = plan(a, f, total);
        k<<<grid, threads, total_smem, stream>>>(a, (unsigned)foff);
        return cuda_check(cudaGetLastError(), "paired refined solve launch");
      }
    }
    if (fused && foff < (size_t)kMaxDynSmem) {
      // a 16-row ring when 512 threads fit with it beside the coefficients, else an
      // 8-row ring with as many threads (256 to 512) as fit; else the passes below.
      // (For the double-float residual, which is bound by instruction issue, 512
      // threads with 8 rows beat 448 with 16: 16.0 against 17.5 ms on the 3-group
      // workload.)
      const size_t room = (size_t)kMaxDynSmem - foff;
      auto fit = [&](int D) { return (int)std::min<size_t>(kStagedThreads, room / fused_ring_bytes<TB>(D, 1) / 32 * 32); };
      int D = 16, threads = fit(16);
      if (threads < kStagedThreads) {
        D = 8;
        threads = fit(8);
      }
      if (threads >= 256) {
        const size_t total_smem = foff + fused_ring_bytes<TB>(D, threads);
        auto k = D == 16 ? grouped_refined_fused_kernel<P, DFRES, TB, 16> : grouped_refined_fused_kernel<P, DFRES, TB, 8>;
        int total = 0;
        SB_TRY(resident_ctas(k, f[0]->device, total_smem, &total, threads));
        const int grid = plan(a, f, total);
        k<<<grid, threads, total_smem, stream>>>(a, n_refine, (unsigned)foff);
        return cuda_check(cudaGetLastError(), "fused refined solve launch");
      }
    }
  }
  // the staged passes when their ring fits beside the coefficients
  const size_t ring_off = (smem + 15) / 16 * 16;
  const bool staged = n_refine > 0 && ring_off + stage_ring_bytes<TB>(kStagedThreads) <= (size_t)kMaxDynSmem;
  auto k = staged ? grouped_refined_solve_kernel<P, DFRES, TB, true> : grouped_refined_solve_kernel<P, DFRES, TB, false>;
  const int threads = staged ? kStagedThreads : kThreads;
  if (staged) smem = ring_off + stage_ring_bytes<TB>(kStagedThreads);
  int total = 0;
  SB_TRY(resident_ctas(k, f[0]->device, smem, &total, threads));
  const int grid = plan(a, f, total);
  k<<<grid, threads, smem, stream>>>(a, n_refine, (unsigned)ring_off);
  return cuda_check(cudaGetLastError(), "refined solve launch");
}

template <int P, bool DFRES, int NB, bool HAS_E>
int launch_refined_step(const sb_factor* f, const double* rcoef, double* state, double* fbuf, float* scratch,
                        int64_t M, int64_t ld, int n_refine, cudaStream_t stream) {
  using AC = typename Residual<DFRES>::AC;
  Groups<float, double, double> a{};
  a.G = 1;
  a.coef[0] = f->coef32;
  a.arow[0] = DFRES ? static_cast<const void*>(f->arowdf) : static_cast<const void*>(f->arow64);
  a.N[0] = (int)f->N;
  a.M[0] = M;
  a.ld[0] = ld;
  a.ntiles[0] = (M + 31) / 32;
  a.rhs[0] = fbuf;
  a.x[0] = state;
  a.work[0] = scratch;
  constexpr int RW = NB + (HAS_E ? 3 : 0);
  const size_t smem = (size_t)(2 * P + 1) * f->N * sizeof(AC) + (size_t)2 * (P + 1) * f->N * sizeof(float) +
                      (size_t)RW * f->N * sizeof(double);
  if (smem > 227 * 1024) return fail(SB_ERR_UNSUPPORTED, "N=%lld: the step's coefficients exceed shared memory",
                                     (long long)f->N);
  // with the FP64 residual, the merged passes when the rows of J A J exist and,
  // with them, a 16-row ring for 512 threads fits beside the coefficients (CH
  // N = 256, 2^20 systems, two passes: 10.3 -> 9.9 ms; with the double-float
  // residual they were slower, 8.2 -> 8.5 ms, and are not used)
  a.rcoef[0] = f->coef32_rev;
  const size_t foff = (smem + (size_t)2 * (P + 1) * f->N * sizeof(float) + 15) / 16 * 16;
  if (!DFRES && n_refine > 0 && f->coef32_rev &&
      foff + fused_ring_bytes<double>(16, kStagedThreads) <= (size_t)kMaxDynSmem) {
    auto k = refined_step_kernel<P, false, NB, HAS_E, 2, 16>;
    const size_t smem_all = foff + fused_ring_bytes<double>(16, kStagedThreads);
    int total = 0;
    SB_TRY(resident_ctas(k, f->device, smem_all, &total, kStagedThreads));
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ntiles[0], total));
    a.cta_begin[0] = 0;
    a.cta_begin[1] = (int)grid;
    k<<<(unsigned)grid, kStagedThreads, smem_all, stream>>>(a, fbuf, rcoef, n_refine, (unsigned)foff);
    return cuda_check(cudaGetLastError(), "refined step launch");
  }
  // the staged passes when their ring fits beside the coefficients
  const size_t ring_off = (smem + 15) / 16 * 16;
  const bool staged = kRefinedStepStaged && n_refine > 0 &&
                      ring_off + stage_ring_bytes<double>(kStagedThreads) <= (size_t)kMaxDynSmem;
  auto k = staged ? refined_step_kernel<P, DFRES, NB, HAS_E, 1> : refined_step_kernel<P, DFRES, NB, HAS_E, 0>;
  const int threads = staged ? kStagedThreads : kThreads;
  const size_t smem_all = staged ? ring_off + stage_ring_bytes<double>(kStagedThreads) : smem;
  int total = 0;
  SB_TRY(resident_ctas(k, f->device, smem_all, &total, threads));
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.ntiles[0], total));
  a.cta_begin[0] = 0;
  a.cta_begin[1] = (int)grid;
  k<<<(unsigned)grid, threads, smem_all, stream>>>(a, fbuf, rcoef, n_refine, (unsigned)ring_off);
  return cuda_check(cudaGetLastError(), "refined step launch");
}

template <bool DFRES>
int refined_step_dispatch(const sb_factor* f, const double* rcoef, int NB, bool has_e, double* state,
                          double* fbuf, float* scratch, int64_t M, int64_t ld, int n_refine, cudaStream_t s) {
  if (f->P == 1 && !has_e && NB == 0)
    return launch_refined_step<1, DFRES, 0, false>(f, rcoef, state, fbuf, scratch, M, ld, n_refine, s);
  if (f->P == 1 && !has_e && NB == 3)
    return launch_refined_step<1, DFRES, 3, false>(f, rcoef, state, fbuf, scratch, M, ld, n_refine, s);
  if (f->P == 2 && !has_e && NB == 0)
    return launch_refined_step<2, DFRES, 0, false>(f, rcoef, state, fbuf, scratch, M, ld, n_refine, s);
  if (f->P == 2 && !has_e && NB == 5)
    return launch_refined_step<2, DFRES, 5, false>(f, rcoef, state, fbuf, scratch, M, ld, n_refine, s);
  if (f->P == 2 && has_e && NB == 0)
    return launch_refined_step<2, DFRES, 0, true>(f, rcoef, state, fbuf, scratch, M, ld, n_refine, s);
  return fail(SB_ERR_UNSUPPORTED, "no refined step for half bandwidth %d with this right-hand side", f->P);
}

template <class A, typename TI, typename TO>
int grouped_sweep_dispatch(const std::vector<const sb_factor*>& f, Op op,
                           const std::vector<const void*>& rhs, const std::vector<void*>& x,
                           const std::vector<int64_t>& M, const std::vector<int64_t>& ld,
                           const typename A::C* const* coefs, cudaStream_t s) {
  if (f[0]->P == 1)
    return op == OP_PRIMAL
               ? launch_grouped_sweep<A, 1, false, true, TI, TO>(f, op, rhs, x, M, ld, coefs, s)
               : launch_grouped_sweep<A, 1, true, false, TI, TO>(f, op, rhs, x, M, ld, coefs, s);
  return op == OP_PRIMAL
             ? launch_grouped_sweep<A, 2, false, true, TI, TO>(f, op, rhs, x, M, ld, coefs, s)
             : launch_grouped_sweep<A, 2, true, false, TI, TO>(f, op, rhs, x, M, ld, coefs, s);
}

size_t dsize(sb_dtype t) { return t == SB_F64 ? 8 : (t == SB_F32 ? 4 : 0); }

}  // namespace

int solve_groups(int G, const sb_factor* const* fs, const void* const* rhs, void* const* x,
                 const int64_t* M, const int64_t* ld, sb_dtype rt, sb_dtype xt, sb_arith arith,
                 int n_refine, sb_arith res_arith, void* const* work, const size_t* work_bytes,
                 cudaStream_t stream, bool fp32_sweeps) {
  if (G < 1 || G > kMaxGroups)
    return fail(SB_ERR_INVALID_ARG, "number of groups must be in [1, %d]", kMaxGroups);
  if (!fs || !rhs || !x || !M || !ld) return fail(SB_ERR_INVALID_ARG, "NULL array argument");
  if (n_refine < 0 || n_refine > 16) return fail(SB_ERR_INVALID_ARG, "n_refine must be in [0, 16]");
  if (dsize(rt) == 0 || dsize(xt) == 0) return fail(SB_ERR_INVALID_ARG, "unknown dtype");
  if (arith != SB_ARITH_NATIVE && arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown arithmetic mode");
  if (res_arith != SB_ARITH_NATIVE && res_arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown residual arithmetic mode");
  std::vector<const sb_factor*> f;
  std::vector<const void*> r;
  std::vector<void*> xs, ws;
  std::vector<int64_t> Ms, lds;
  for (int g = 0; g < G; ++g) {
    if (!fs[g]) return fail(SB_ERR_INVALID_ARG, "factor %d is NULL", g);
    if (fs[g]->periodic)
      return fail(SB_ERR_UNSUPPORTED, "factor %d is periodic: use sb_solve_batched_ex", g);
    if (fs[g]->P != fs[0]->P)
      return fail(SB_ERR_UNSUPPORTED, "all groups of one call must have the same bandwidth");
    if (fs[g]->device != fs[0]->device)
      return fail(SB_ERR_INVALID_ARG, "all groups of one call must live on one device");
    if (M[g] < 1 || ld[g] < M[g])
      return fail(SB_ERR_INVALID_ARG, "group %d: need M >= 1 and ld >= M", g);
    if (ld[g] > ((int64_t)1 << 40) / fs[g]->N) return fail(SB_ERR_INVALID_ARG, "N*ld too large");
    const size_t elems = (size_t)((fs[g]->N - 1) * ld[g] + M[g]);
    SB_TRY(check_device_range(rhs[g], elems * dsize(rt), dsize(rt), fs[g]->device, "rhs"));
    SB_TRY(check_device_range(x[g], elems * dsize(xt), dsize(xt), fs[g]->device, "x"));
    if (rhs[g] == x[g] && rt != xt) return fail(SB_ERR_INVALID_ARG, "x may alias rhs only with equal dtypes");
    SB_TRY(check_alias(rhs[g], elems * dsize(rt), x[g], elems * dsize(xt), "rhs", "x"));
    if (n_refine > 0) {
      if (!work || !work_bytes || !work[g] || work_bytes[g] < elems * sizeof(float))
        return fail(SB_ERR_INVALID_ARG, "group %d: refinement needs a workspace of %zu bytes", g,
                    elems * sizeof(float));
      SB_TRY(check_device_range(work[g], elems * sizeof(float), 4, fs[g]->device, "work"));
      SB_TRY(check_alias(work[g], elems * sizeof(float), x[g], elems * dsize(xt), "work", "x"));
      SB_TRY(check_alias(work[g], elems * sizeof(float), rhs[g], elems * dsize(rt), "work", "rhs"));
      ws.push_back(work[g]);
    }
    f.push_back(fs[g]);
    r.push_back(rhs[g]);
    xs.push_back(x[g]);
    Ms.push_back(M[g]);
    lds.push_back(ld[g]);
  }
  if (n_refine > 0 && (xt != SB_F64 || arith != SB_ARITH_NATIVE))
    return fail(SB_ERR_UNSUPPORTED,
                "refinement takes FP32 or FP64 right-hand sides, FP64 solutions and FP32 sweeps (native)");
  if (n_refine > 0)
    for (int g = 0; g < G; ++g)
      if (rhs[g] == x[g]) return fail(SB_ERR_INVALID_ARG, "refinement needs x separate from rhs");

  DeviceGuard dg(f[0]->device);
  SB_TRY(dg.rc);
  std::vector<const float*> c32(G);
  std::vector<const double*> c64(G);
  std::vector<const df*> cdf(G);
  for (int g = 0; g < G; ++g) {
    c32[g] = f[g]->coef32;
    c64[g] = f[g]->coef64;
    cdf[g] = reinterpret_cast<const df*>(f[g]->coefdf);
  }
  int rc;
  if (n_refine > 0) {
    // the FP32 pass and every correction pass of a tile in one launch
    const bool dfr = res_arith == SB_ARITH_DF32;
    if (rt == SB_F64) {
      if (f[0]->P == 1)
        rc = dfr ? launch_grouped_refined_solve<1, true, double>(f, r, xs, Ms, lds, ws, n_refine, stream)
                 : launch_grouped_refined_solve<1, false, double>(f, r, xs, Ms, lds, ws, n_refine, stream);
      else
        rc = dfr ? launch_grouped_refined_solve<2, true, double>(f, r, xs, Ms, lds, ws, n_refine, stream)
                 : launch_grouped_refined_solve<2, false, double>(f, r, xs, Ms, lds, ws, n_refine, stream);
    } else {
      if (f[0]->P == 1)
        rc = dfr ? launch_grouped_refined_solve<1, true, float>(f, r, xs, Ms, lds, ws, n_refine, stream)
                 : launch_grouped_refined_solve<1, false, float>(f, r, xs, Ms, lds, ws, n_refine, stream);
      else
        rc = dfr ? launch_grouped_refined_solve<2, true, float>(f, r, xs, Ms, lds, ws, n_refine, stream)
                 : launch_grouped_refined_solve<2, false, float>(f, r, xs, Ms, lds, ws, n_refine, stream);
    }
    return rc;
  }
  // the whole solve in one pass
  if (arith == SB_ARITH_DF32) {
    if (rt == SB_F64 && xt == SB_F64)
      rc = grouped_sweep_dispatch<DFArith, double, double>(f, OP_PRIMAL, r, xs, Ms, lds, cdf.data(), stream);
    else if (rt == SB_F32 && xt == SB_F64)
      rc = grouped_sweep_dispatch<DFArith, float, double>(f, OP_PRIMAL, r, xs, Ms, lds, cdf.data(), stream);
    else
      rc = fail(SB_ERR_UNSUPPORTED, "double-float sweeps write FP64 solutions");
  } else if (rt == SB_F64 && xt == SB_F64 && (n_refine > 0 || fp32_sweeps)) {
    // mixed precision with an FP64 right-hand side: FP32 sweeps of b rounded to FP32
    rc = grouped_sweep_dispatch<NativeArith<float>, double, double>(f, OP_PRIMAL, r, xs, Ms, lds, c32.data(), stream);
  } else if (rt == SB_F64 && xt == SB_F64) {
    rc = grouped_sweep_dispatch<NativeArith<double>, double, double>(f, OP_PRIMAL, r, xs, Ms, lds, c64.data(), stream);
  } else if (rt == SB_F32 && xt == SB_F32) {
    rc = grouped_sweep_dispatch<NativeArith<float>, float, float>(f, OP_PRIMAL, r, xs, Ms, lds, c32.data(), stream);
  } else if (rt == SB_F32 && xt == SB_F64) {
    rc = grouped_sweep_dispatch<NativeArith<float>, float, double>(f, OP_PRIMAL, r, xs, Ms, lds, c32.data(), stream);
  } else {
    rc = fail(SB_ERR_UNSUPPORTED, "unsupported dtype combination");
  }
  SB_TRY(rc);
  return SB_OK;
}

int refined_step(const sb_factor* f, const double* rcoef, int NB, bool has_e, double* state, double* fbuf,
                 float* scratch, int64_t M, int64_t ld, int n_refine, sb_arith residual_arith,
                 cudaStream_t stream) {
  if (f->periodic) return fail(SB_ERR_UNSUPPORTED, "the refined steps do not support periodic ends");
  return residual_arith == SB_ARITH_DF32
             ? refined_step_dispatch<true>(f, rcoef, NB, has_e, state, fbuf, scratch, M, ld, n_refine, stream)
             : refined_step_dispatch<false>(f, rcoef, NB, has_e, state, fbuf, scratch, M, ld, n_refine, stream);
}

}  // namespace sb

using namespace sb;

extern "C" {

int sb_refine_workspace_bytes(const sb_factor* f, int64_t M, int64_t ld, size_t* bytes) {
  clear_error();
  if (!f || !bytes) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (M < 0 || ld < M) return fail(SB_ERR_INVALID_ARG, "bad M or ld");
  *bytes = M == 0 ? 0 : (size_t)((f->N - 1) * ld + M) * sizeof(float);
  return SB_OK;
}

int sb_solve_batched_refined(const sb_factor* f, const float* rhs, double* x, int64_t M,
                             int64_t ld, int n_refine, sb_arith residual_arith, void* work,
                             size_t work_bytes, void* stream) {
  clear_error();
  if (!f) return fail(SB_ERR_INVALID_ARG, "factor handle is NULL");
  if (M == 0) return SB_OK;
  const void* r = rhs;
  void* xx = x;
  return solve_groups(1, &f, &r, &xx, &M, &ld, SB_F32, SB_F64, SB_ARITH_NATIVE, n_refine,
                      residual_arith, &work, &work_bytes, (cudaStream_t)stream);
}

int sb_solve_batched_groups(int G, const sb_factor* const* f, const void* const* rhs,
                            void* const* x, const int64_t* M, const int64_t* ld,
                            sb_dtype rhs_dtype, sb_dtype x_dtype, sb_arith arith, int n_refine,
                            sb_arith residual_arith, void* const* work, const size_t* work_bytes,
                            void* stream) {
  clear_error();
  return solve_groups(G, f, rhs, x, M, ld, rhs_dtype, x_dtype, arith, n_refine, residual_arith,
                      work, work_bytes, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Refined solve without any allocation by the caller.
//
// Some callers cannot allocate device memory at the point where they solve: code
// running inside a framework whose memory pool owns every allocation, real-time
// loops that must not call into the allocator, or plain C callers with no
// allocator of their own.  For them sb_solve_batched_refined_noalloc takes its
// FP32 scratch from the array below instead of a caller workspace.  The array is
// a file-scope device variable, so every GPU that loads this library holds it
// (16 MiB) until the process exits.  Every call uses the same array: calls that
// overlap on the GPU (different streams, or different host threads) race on it.
// The refinement pass writes each scratch element before reading it, so nothing
// needs clearing between calls.
namespace sb {
namespace {

constexpr size_t kNoAllocScratchElems = (size_t)4 << 20;  // 4 Mi FP32 values = 16 MiB
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device `dev` (looked up
// once per device; the host symbol itself is not a device address).
int noalloc_scratch(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SB_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    SB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SB_OK;
}

// One launch of kernel k over a single group, sized from the occupancy query
// (no caches, so no host containers grow).
template <typename K, typename GA>
int launch_one_group(K k, GA& a, int64_t N, int64_t M, size_t smem, int device,
                     cudaStream_t stream) {
  SB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
  int nb = 0;
  SB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kThreads, smem));
  if (nb < 1) return fail(SB_ERR_UNSUPPORTED, "kernel cannot be resident (%zu B smem)", smem);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.ntiles[0], (int64_t)nb * sm_count(device)));
  a.G = 1;
  a.cta_begin[0] = 0;
  a.cta_begin[1] = grid;
  (void)N;
  (void)M;
  k<<<grid, kThreads, smem, stream>>>(a);
  return cuda_check(cudaGetLastError(), "kernel launch");
}

template <int P>
int noalloc_refined(const sb_factor* f, const float* rhs, double* x, int64_t M, int64_t ld,
                    int n_refine, sb_arith res, float* scratch, cudaStream_t stream) {
  const int N = (int)f->N;
  // first pass: FP32 sweeps of the FP32 right-hand side into the FP64 solution
  {
    Groups<float, float, double> a{};
    a.coef[0] = f->coef32;
    a.N[0] = N;
    a.M[0] = M;
    a.ld[0] = ld;
    a.ntiles[0] = (M + 31) / 32;
    a.rhs[0] = rhs;
    a.x[0] = x;
    const size_t smem = (size_t)2 * (P + 1) * N * sizeof(float);
    SB_TRY(launch_one_group(grouped_sweep_kernel<NativeArith<float>, P, false, true, float, double>,
                            a, N, M, smem, f->device, stream));
  }
  for (int k = 0; k < n_refine; ++k) {
    Groups<float, float, double> a{};
    a.coef[0] = f->coef32;
    a.arow[0] = res == SB_ARITH_DF32 ? static_cast<const void*>(f->arowdf)
                                     : static_cast<const void*>(f->arow64);
    a.N[0] = N;
    a.M[0] = M;
    a.ld[0] = ld;
    a.ntiles[0] = (M + 31) / 32;
    a.rhs[0] = rhs;
    a.x[0] = x;
    a.work[0] = scratch;
    const size_t smem = (size_t)(2 * P + 1) * N * 8 + (size_t)2 * (P + 1) * N * sizeof(float);
    if (res == SB_ARITH_DF32)
      SB_TRY(launch_one_group(grouped_refine_kernel<P, true, float>, a, N, M, smem, f->device, stream));
    else
      SB_TRY(launch_one_group(grouped_refine_kernel<P, false, float>, a, N, M, smem, f->device, stream));
  }
  return SB_OK;
}

}  // namespace
}  // namespace sb

extern "C" int sb_solve_batched_refined_noalloc(const sb_factor* f, const float* rhs, double* x,
                                                int64_t M, int64_t ld, int n_refine,
                                                sb_arith residual_arith, void* stream) {
  clear_error();
  if (f == nullptr) return fail(SB_ERR_INVALID_ARG, "factor handle is NULL");
  if (f->periodic) return fail(SB_ERR_UNSUPPORTED, "periodic factors are not refined: use sb_solve_batched_ex");
  if (M < 0 || ld < M || ld < 1)
    return fail(SB_ERR_INVALID_ARG, "need M >= 0 and ld >= max(M, 1)");
  if (n_refine < 0 || n_refine > 16) return fail(SB_ERR_INVALID_ARG, "n_refine must be in [0, 16]");
  if (residual_arith != SB_ARITH_NATIVE && residual_arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown residual arithmetic mode");
  if (M == 0) return SB_OK;
  if (ld > ((int64_t)1 << 40) / f->N) return fail(SB_ERR_INVALID_ARG, "N*ld too large");
  const size_t elems = (size_t)((f->N - 1) * ld + M);
  if (elems > kNoAllocScratchElems)
    return fail(SB_ERR_INVALID_ARG,
                "(N-1)*ld + M = %zu elements exceeds the allocation-free scratch of %zu elements "
                "(16 MiB); use sb_solve_batched_refined with a workspace instead",
                elems, kNoAllocScratchElems);
  const size_t smem = (size_t)(2 * f->P + 1) * f->N * 8 + (size_t)2 * (f->P + 1) * f->N * 4;
  if (smem > 227 * 1024) return fail(SB_ERR_UNSUPPORTED, "N too large for shared memory");
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  SB_TRY(check_device_range(rhs, elems * sizeof(float), sizeof(float), f->device, "rhs"));
  SB_TRY(check_device_range(x, elems * sizeof(double), sizeof(double), f->device, "x"));
  SB_TRY(check_alias(rhs, elems * sizeof(float), x, elems * sizeof(double), "rhs", "x"));
  if ((const void*)rhs == (const void*)x) return fail(SB_ERR_INVALID_ARG, "x must not alias rhs");
  float* scratch = nullptr;
  SB_TRY(noalloc_scratch(f->device, &scratch));
  cudaStream_t s = (cudaStream_t)stream;
  return f->P == 1 ? noalloc_refined<1>(f, rhs, x, M, ld, n_refine, residual_arith, scratch, s)
                   : noalloc_refined<2>(f, rhs, x, M, ld, n_refine, residual_arith, scratch, s);
}
