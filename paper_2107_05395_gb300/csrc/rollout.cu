// Discrete adjoint of an implicit rollout with a shared matrix (no counterpart in
// the paper, which only runs forward).
//
// Rollout: x_{n+1} = A(p)^{-1} F(x_n), n = 0 .. T-1, with F = identity for the
// backward-Euler diffusion / hyperdiffusion steppers and F(x) = x + E (x^3 - x),
// E = dt D2_N, for Cahn-Hilliard; p is the stepper's coefficient (r, or gamma).
// Given gbar_T = dL/dx_T, the reverse sweep is
//     mu = A^{-T} gbar_{n+1};   dL/dp -= mu . (dA/dp) x_{n+1};   gbar_n = J_F(x_n)^T mu
// with J_F(x)^T mu = mu + (3 x^2 - 1) * (E^T mu).
//
// Memory: the forward pass keeps a checkpoint every k steps in the caller's
// workspace; the backward pass recomputes each k-step segment from its checkpoint
// (out-of-place fused steps, bitwise the states of the forward pass) and walks it
// backwards.  One fused kernel per backward step runs both adjoint sweeps, and in
// the back sweep (rows N-1 .. 0) accumulates the per-system parameter gradient and
// writes gbar_n in place over gbar_{n+1}.  The per-system gradients are summed
// over the batch by a fixed-shape two-level reduction, so the scalar does not
// depend on scheduling.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "arith.cuh"
#include "sb_internal.h"

namespace sb {
namespace {

constexpr int kAdjRows = 8;
constexpr int kAdjThreads = 256;
constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

// coef: adjoint block [forward rows | backward rows], (P+1) per row;
// dA: (2P+1) per row (offsets -P..P); E: 3 per row (offsets -1..1), CH only.
template <int P, bool CH, int R>
__global__ void __launch_bounds__(kAdjThreads)
adjoint_step_kernel(const double* __restrict__ coef, const double* __restrict__ dA,
                    const double* __restrict__ E, int N, int64_t M, int64_t ld, double* G,
                    const double* __restrict__ Xn1, const double* __restrict__ Xn, double* dp,
                    int64_t ntiles) {
  constexpr int W = P + 1;
  constexpr int NB = 2 * P + 1;
  extern __shared__ __align__(16) double sm[];
  double* fw = sm;
  double* bw = sm + W * N;
  double* da = sm + 2 * W * N;
  double* e = da + NB * N;
  for (int k = threadIdx.x; k < 2 * W * N; k += blockDim.x) sm[k] = coef[k];
  for (int k = threadIdx.x; k < NB * N; k += blockDim.x) da[k] = dA[k];
  if constexpr (CH)
    for (int k = threadIdx.x; k < 3 * N; k += blockDim.x) e[k] = E[k];
  __syncthreads();

  const int nw = blockDim.x >> 5;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5); tile < ntiles;
       tile += (int64_t)gridDim.x * nw) {
    const int64_t m = tile * 32 + (threadIdx.x & 31);
    if (m >= M) continue;
    double* g = G + m;
    const double* x1p = Xn1 + m;
    const double* x0p = Xn + m;

    // ---- forward adjoint sweep: w_i = g_i - F1 w_{i-1} - F2 w_{i-2} (in place)
    {
      double w1 = 0.0, w2 = 0.0;
      double va[R], vb[R];
      auto load = [&](double (&b)[R], int i0) {
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (i0 + j < N) b[j] = g[(int64_t)(i0 + j) * ld];
      };
      auto fwd = [&](double (&b)[R], int i0) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int i = i0 + j;
          if (i < N) {
            const double* c = fw + W * i;
            double w = fma(-c[1], w1, b[j]);
            if constexpr (P == 2) w = fma(-c[2], w2, w);
            g[(int64_t)i * ld] = w;
            w2 = w1;
            w1 = w;
          }
        }
      };
      load(va, 0);
      for (int i0 = 0; i0 < N; i0 += 2 * R) {
        load(vb, i0 + R);
        fwd(va, i0);
        load(va, i0 + 2 * R);
        fwd(vb, i0 + R);
      }
    }

    // ---- backward adjoint sweep with the gradient terms, rows N-1 .. 0
    double mu1 = 0.0, mu2 = 0.0;    // mu_{i+1}, mu_{i+2}
    double xw[NB];                  // x_{n+1} rows i-P .. i+P
#pragma unroll
    for (int k = 0; k < NB; ++k) xw[k] = 0.0;
    double xn_next = 0.0;           // x_n row i+1 (CH)
    double acc = 0.0;               // sum_i mu_i (dA x_{n+1})_i
    double wa[R], wb[R], ya[R], yb[R], za[R], zb[R];
    auto load = [&](double (&w)[R], double (&y)[R], double (&z)[R], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (i0 - j >= 0) {
          w[j] = g[(int64_t)(i0 - j) * ld];
          y[j] = x1p[(int64_t)(i0 - j) * ld];
          if constexpr (CH) z[j] = x0p[(int64_t)(i0 - j) * ld];
        }
    };
    auto push = [&](double v) {  // insert x_{n+1} row i-P at the bottom of the window
#pragma unroll
      for (int k = NB - 1; k > 0; --k) xw[k] = xw[k - 1];
      xw[0] = v;
    };
    // finalize gbar_n at row r = i + 1 once mu_i is known (CH): mu window (mu_i, mu_r, mu_{r+1})
    auto emit_ch = [&](int r, double mu_lo, double mu_r, double mu_hi, double xr) {
      const double* er = e + 3 * r;
      const double s = fma(er[0], mu_lo, fma(er[1], mu_r, er[2] * mu_hi));
      g[(int64_t)r * ld] = fma(fma(3.0 * xr, xr, -1.0), s, mu_r);
    };
    auto bwd = [&](double (&w)[R], double (&y)[R], double (&z)[R], double (&yn)[R], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int i = i0 - j;
        if (i >= 0) {
          const int k = j + P;  // x_{n+1} row i - P
          push(i - P >= 0 ? (k < R ? y[k] : yn[k - R]) : 0.0);
          const double* c = bw + W * i;
          double mu = dmul_int(c[0], w[j]);  // off the chain: integer pipe, bit-identical
          mu = fma(-c[1], mu1, mu);
          if constexpr (P == 2) mu = fma(-c[2], mu2, mu);
          const double* a = da + NB * i;
          double t = a[0] * xw[0];
#pragma unroll
          for (int q = 1; q < NB; ++q) t = fma(a[q], xw[q], t);
          acc = fma(mu, t, acc);
          if constexpr (CH) {
            if (i + 1 < N) emit_ch(i + 1, mu, mu1, mu2, xn_next);
            xn_next = z[j];
          } else {
            g[(int64_t)i * ld] = mu;
          }
          mu2 = mu1;
          mu1 = mu;
        }
      }
    };
    load(wa, ya, za, N - 1);
    load(wb, yb, zb, N - 1 - R);
#pragma unroll
    for (int k = 0; k < P; ++k) push(N - 1 - k >= 0 ? ya[k] : 0.0);  // rows N-1 .. N-P
    for (int i0 = N - 1; i0 >= 0; i0 -= 2 * R) {
      bwd(wa, ya, za, yb, i0);
      load(wa, ya, za, i0 - 2 * R);
      bwd(wb, yb, zb, ya, i0 - R);
      load(wb, yb, zb, i0 - 3 * R);
    }
    if constexpr (CH) emit_ch(0, 0.0, mu1, mu2, xn_next);
    dp[m] -= acc;
  }
}

// Fixed-shape deterministic sum: kRedBlocks partial sums over fixed index ranges,
// each a fixed strided order and a fixed shared-memory tree, then one block.
__global__ void __launch_bounds__(kRedThreads) reduce_partials(const double* v, int64_t n,
                                                               double* part) {
  __shared__ double s[kRedThreads];
  const int64_t chunk = (n + kRedBlocks - 1) / kRedBlocks;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) acc += v[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void __launch_bounds__(kRedThreads) reduce_final(const double* part, double* out) {
  __shared__ double s[kRedThreads];
  s[threadIdx.x] = (threadIdx.x < kRedBlocks) ? part[threadIdx.x] : 0.0;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

struct Layout {
  size_t S;       // doubles per state (N * ld)
  int64_t nckpt;  // checkpoints
  int64_t k;
  size_t bytes;
};

Layout layout(const sb_stepper* st, int64_t M, int64_t ld, int64_t T, int64_t k) {
  Layout L;
  L.S = (size_t)st->N * (size_t)ld;
  L.k = k;
  L.nckpt = (T + k - 1) / k;
  L.bytes = ((size_t)L.nckpt + (size_t)k + 2) * L.S * sizeof(double) +
            (size_t)M * sizeof(double) + kRedBlocks * sizeof(double);
  return L;
}

int ensure_dA(sb_stepper* st) {
  std::lock_guard<std::mutex> lk(st->mu);
  if (st->dA64) return SB_OK;
  int mat = 0;
  double scale = 1.0;
  if (st->kind == SB_STEP_DIFFUSION) mat = SB_MAT_DIFFUSION_DIRICHLET;
  else if (st->kind == SB_STEP_HYPERDIFFUSION)
    mat = st->bc == SB_BC_HINGED ? SB_MAT_HYPER_HINGED : SB_MAT_HYPER_TRUNCATED;
  else {
    mat = SB_MAT_CH_NOFLUX;
    scale = st->dt;  // A = I + dt * gamma * D4_N, so dA/dgamma = dt * D4_N
  }
  std::vector<double> diag;
  int P = 0;
  SB_TRY(build_matrix(mat, st->N, scale, diag, &P));  // I + scale K
  const int64_t N = st->N, nb = 2 * P + 1;
  std::vector<double> rows((size_t)nb * N);
  for (int64_t i = 0; i < N; ++i)
    for (int64_t q = 0; q < nb; ++q)
      rows[(size_t)nb * i + q] = diag[(size_t)q * N + i] - (q == P ? 1.0 : 0.0);  // remove I
  DeviceGuard g(st->fac->device);
  SB_TRY(g.rc);
  double* d = nullptr;
  SB_CUDA(cudaMalloc(&d, rows.size() * sizeof(double)));
  const cudaError_t e = cudaMemcpy(d, rows.data(), rows.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return cuda_check(e, "cudaMemcpy");
  }
  st->dA64 = d;
  return SB_OK;
}

int copy_state(double* dst, const double* src, int64_t N, int64_t M, int64_t ld, cudaStream_t s) {
  if (dst == src) return SB_OK;
  return cuda_check(cudaMemcpy2DAsync(dst, ld * sizeof(double), src, ld * sizeof(double),
                                      M * sizeof(double), N, cudaMemcpyDeviceToDevice, s),
                    "cudaMemcpy2DAsync");
}

template <int P, bool CH>
int launch_adjoint(const sb_stepper* st, double* G, const double* Xn1, const double* Xn, double* dp,
                   int64_t M, int64_t ld, cudaStream_t s) {
  const int N = (int)st->N;
  const size_t smem = ((size_t)2 * (P + 1) * N + (size_t)(2 * P + 1) * N + (CH ? 3 * (size_t)N : 0)) *
                      sizeof(double);
  if (smem > 227 * 1024) return fail(SB_ERR_UNSUPPORTED, "N=%d too large for the adjoint kernel", N);
  auto k = adjoint_step_kernel<P, CH, kAdjRows>;
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> occ;
  int nb = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(reinterpret_cast<const void*>(k), smem);
    auto it = occ.find(key);
    if (it == occ.end()) {
      SB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
      SB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kAdjThreads, smem));
      occ[key] = nb;
    } else {
      nb = it->second;
    }
  }
  if (nb < 1) return fail(SB_ERR_UNSUPPORTED, "adjoint kernel cannot be resident");
  const int64_t ntiles = (M + 31) / 32;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(st->fac->device)));
  const double* coef = st->fac->coef64 + op_block_len(P, N);  // adjoint block
  k<<<(unsigned)grid, kAdjThreads, smem, s>>>(coef, st->dA64, st->r64, N, M, ld, G, Xn1, Xn, dp, ntiles);
  return cuda_check(cudaGetLastError(), "adjoint step launch");
}

int adjoint_step(const sb_stepper* st, double* G, const double* Xn1, const double* Xn, double* dp,
                 int64_t M, int64_t ld, cudaStream_t s) {
  if (st->kind == SB_STEP_CAHN_HILLIARD) return launch_adjoint<2, true>(st, G, Xn1, Xn, dp, M, ld, s);
  if (st->fac->P == 1) return launch_adjoint<1, false>(st, G, Xn1, Xn, dp, M, ld, s);
  return launch_adjoint<2, false>(st, G, Xn1, Xn, dp, M, ld, s);
}

int check_rollout(const sb_stepper* st, int64_t M, int64_t ld, int64_t T, int64_t k, sb_arith arith,
                  void* work, size_t work_bytes, Layout* L) {
  if (!st) return fail(SB_ERR_INVALID_ARG, "stepper is NULL");
  if (st->scheme != SB_SCHEME_BE)
    return fail(SB_ERR_UNSUPPORTED, "the rollout adjoint supports backward-Euler and Cahn-Hilliard steppers");
  if (st->fac->periodic)
    return fail(SB_ERR_UNSUPPORTED, "the rollout adjoint does not support periodic ends");
  if (M < 1 || ld < M) return fail(SB_ERR_INVALID_ARG, "need M >= 1 and ld >= M");
  if (T < 1 || k < 1) return fail(SB_ERR_INVALID_ARG, "need nsteps >= 1 and ckpt_every >= 1");
  if (arith != SB_ARITH_NATIVE && arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown arithmetic mode");
  *L = layout(st, M, ld, T, k);
  if (!work || work_bytes < L->bytes)
    return fail(SB_ERR_INVALID_ARG, "the rollout needs a workspace of %zu bytes", L->bytes);
  return check_device_range(work, L->bytes, 8, st->fac->device, "work");
}

}  // namespace
}  // namespace sb

using namespace sb;

extern "C" {

int sb_rollout_workspace_bytes(const sb_stepper* st, int64_t M, int64_t ld, int64_t nsteps,
                               int64_t ckpt_every, size_t* bytes) {
  clear_error();
  if (!st || !bytes) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (M < 1 || ld < M || nsteps < 1 || ckpt_every < 1) return fail(SB_ERR_INVALID_ARG, "bad sizes");
  *bytes = layout(st, M, ld, nsteps, ckpt_every).bytes;
  return SB_OK;
}

int sb_rollout_forward(sb_stepper* st, const double* C0, double* CT, int64_t M, int64_t ld,
                       int64_t nsteps, int64_t ckpt_every, sb_arith arith, void* work,
                       size_t work_bytes, void* stream) {
  clear_error();
  Layout L;
  SB_TRY(check_rollout(st, M, ld, nsteps, ckpt_every, arith, work, work_bytes, &L));
  DeviceGuard g(st->fac->device);
  SB_TRY(g.rc);
  const size_t bytes = (size_t)((st->N - 1) * ld + M) * sizeof(double);
  SB_TRY(check_device_range(C0, bytes, 8, st->fac->device, "C0"));
  SB_TRY(check_device_range(CT, bytes, 8, st->fac->device, "CT"));
  SB_TRY(check_alias(C0, bytes, CT, bytes, "C0", "CT"));
  SB_TRY(check_alias(CT, bytes, work, L.bytes, "CT", "work"));
  cudaStream_t s = (cudaStream_t)stream;
  double* ck = static_cast<double*>(work);
  SB_TRY(copy_state(ck, C0, st->N, M, ld, s));
  SB_TRY(copy_state(CT, C0, st->N, M, ld, s));
  for (int64_t n = 0; n < nsteps; ++n) {
    SB_TRY(stepper_step(st, CT, CT, M, ld, arith, s));
    if ((n + 1) % ckpt_every == 0 && n + 1 < nsteps)
      SB_TRY(copy_state(ck + ((n + 1) / ckpt_every) * L.S, CT, st->N, M, ld, s));
  }
  return SB_OK;
}

int sb_rollout_backward(sb_stepper* st, const double* grad_CT, double* grad_C0,
                        double* grad_param_per_system, double* grad_param, int64_t M, int64_t ld,
                        int64_t nsteps, int64_t ckpt_every, sb_arith arith, void* work,
                        size_t work_bytes, void* stream) {
  clear_error();
  Layout L;
  SB_TRY(check_rollout(st, M, ld, nsteps, ckpt_every, arith, work, work_bytes, &L));
  DeviceGuard g(st->fac->device);
  SB_TRY(g.rc);
  const int dev = st->fac->device;
  const size_t bytes = (size_t)((st->N - 1) * ld + M) * sizeof(double);
  SB_TRY(check_device_range(grad_CT, bytes, 8, dev, "grad_CT"));
  SB_TRY(check_device_range(grad_C0, bytes, 8, dev, "grad_C0"));
  SB_TRY(check_alias(grad_C0, bytes, work, L.bytes, "grad_C0", "work"));
  if (grad_param_per_system)
    SB_TRY(check_device_range(grad_param_per_system, M * sizeof(double), 8, dev, "grad_param_per_system"));
  if (grad_param) SB_TRY(check_device_range(grad_param, sizeof(double), 8, dev, "grad_param"));
  SB_TRY(ensure_dA(st));
  cudaStream_t s = (cudaStream_t)stream;
  double* base = static_cast<double*>(work);
  double* ck = base;
  double* seg = base + L.nckpt * L.S;
  double* gbar = seg + (L.k + 1) * L.S;
  double* dp = gbar + L.S;
  double* part = dp + M;
  SB_TRY(copy_state(gbar, grad_CT, st->N, M, ld, s));
  SB_CUDA(cudaMemsetAsync(dp, 0, M * sizeof(double), s));
  for (int64_t sgm = L.nckpt - 1; sgm >= 0; --sgm) {
    const int64_t start = sgm * L.k, end = std::min(nsteps, start + L.k);
    SB_TRY(copy_state(seg, ck + sgm * L.S, st->N, M, ld, s));
    for (int64_t j = 0; j < end - start; ++j)
      SB_TRY(stepper_step(st, seg + j * L.S, seg + (j + 1) * L.S, M, ld, arith, s));
    for (int64_t n = end - 1; n >= start; --n)
      SB_TRY(adjoint_step(st, gbar, seg + (n + 1 - start) * L.S, seg + (n - start) * L.S, dp, M, ld, s));
  }
  SB_TRY(copy_state(grad_C0, gbar, st->N, M, ld, s));
  if (grad_param_per_system)
    SB_CUDA(cudaMemcpyAsync(grad_param_per_system, dp, M * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (grad_param) {
    reduce_partials<<<kRedBlocks, kRedThreads, 0, s>>>(dp, M, part);
    SB_CUDA(cudaGetLastError());
    reduce_final<<<1, kRedThreads, 0, s>>>(part, grad_param);
    SB_CUDA(cudaGetLastError());
  }
  return SB_OK;
}

}  // extern "C"
