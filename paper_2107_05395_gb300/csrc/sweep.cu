// Batched forward/backward sweeps with one shared factor (Algorithms 2 and 4),
// native arithmetic in the storage type (FP64 or FP32).
//
// One thread owns one system m; a warp therefore touches 32 consecutive
// systems, and every row access i*ld + m is one coalesced 256 B (FP64) or 128 B
// (FP32) transaction per warp.  The shared coefficients (one copy on the device,
// section 2) are staged once per CTA into shared memory and read as broadcasts.
// The forward result u is written into x and read back by the backward sweep
// (in place, as in Algorithm 2); the same thread reads what it wrote, so no
// synchronisation is needed.  Rows are fetched R at a time into registers so
// that R independent loads are in flight per thread.
#include <algorithm>
#include <mutex>
#include <unordered_map>

#include "sb_internal.h"

namespace sb {
namespace {

constexpr int kThreads = 128;  // threads per CTA (4 warps)
constexpr int kRows = 8;       // rows fetched ahead per batch

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// coef: [forward rows][backward rows], (P + 1) values per row (see sb_internal.h).
template <typename T, int P, bool SCALE_FWD, bool SCALE_BWD, bool SMEM>
__global__ void __launch_bounds__(kThreads)
banded_sweep_kernel(const T* __restrict__ coef, int N, int64_t M, int64_t ld,
                    const T* rhs, T* x, int64_t tiles) {
  constexpr int W = P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const T* cf;
  if constexpr (SMEM) {
    T* s = reinterpret_cast<T*>(smem_raw);
    const int n = 2 * W * N;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s[k] = coef[k];
    __syncthreads();
    cf = s;
  } else {
    cf = coef;
  }
  const T* fw = cf;
  const T* bw = cf + (int64_t)W * N;

  for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int64_t m = tile * kThreads + threadIdx.x;
    if (m >= M) continue;
    const T* r = rhs + m;
    T* y = x + m;

    // forward: u_i = (r_i - p1 u_{i-1} - p2 u_{i-2}) * s_i
    T u1 = T(0), u2 = T(0);
    for (int i0 = 0; i0 < N; i0 += kRows) {
      T v[kRows];
#pragma unroll
      for (int j = 0; j < kRows; ++j)
        if (i0 + j < N) v[j] = ld_stream(r + (int64_t)(i0 + j) * ld);
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        const int i = i0 + j;
        if (i < N) {
          const T* c = fw + W * i;
          T u = v[j] - c[0] * u1;
          if constexpr (P == 2) u -= c[1] * u2;
          if constexpr (SCALE_FWD) u *= c[P];
          y[(int64_t)i * ld] = u;
          if constexpr (P == 2) u2 = u1;
          u1 = u;
        }
      }
    }
    // backward: x_i = (u_i - q1 x_{i+1} - q2 x_{i+2}) * t_i
    T x1 = T(0), x2 = T(0);
    for (int i0 = N - 1; i0 >= 0; i0 -= kRows) {
      T v[kRows];
#pragma unroll
      for (int j = 0; j < kRows; ++j)
        if (i0 - j >= 0) v[j] = y[(int64_t)(i0 - j) * ld];
#pragma unroll
      for (int j = 0; j < kRows; ++j) {
        const int i = i0 - j;
        if (i >= 0) {
          const T* c = bw + W * i;
          T xi = v[j] - c[0] * x1;
          if constexpr (P == 2) xi -= c[1] * x2;
          if constexpr (SCALE_BWD) xi *= c[P];
          st_stream(y + (int64_t)i * ld, xi);
          if constexpr (P == 2) x2 = x1;
          x1 = xi;
        }
      }
    }
  }
}

struct LaunchInfo {
  int blocks_per_sm = 0;
};

std::mutex g_occ_mu;
std::unordered_map<uint64_t, LaunchInfo> g_occ;

template <typename K>
int prepare_kernel(K kernel, int device, size_t smem, int* blocks_per_sm) {
  const uint64_t key = (reinterpret_cast<uint64_t>(reinterpret_cast<const void*>(kernel)) << 8) ^
                       ((uint64_t)smem << 1) ^ (uint64_t)device * 0x9E3779B97F4A7C15ull;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
      *blocks_per_sm = it->second.blocks_per_sm;
      return SB_OK;
    }
  }
  if (smem > 48 * 1024)
    SB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int nb = 0;
  SB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, smem));
  if (nb < 1) return fail(SB_ERR_UNSUPPORTED, "kernel cannot be resident with %zu B smem", smem);
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ[key].blocks_per_sm = nb;
  *blocks_per_sm = nb;
  return SB_OK;
}

template <typename T, int P, bool SF, bool SB_>
int launch_typed(const sb_factor* f, const T* coef, const T* rhs, T* x, int64_t M, int64_t ld,
                 cudaStream_t stream) {
  const int N = (int)f->N;
  const size_t coef_bytes = (size_t)2 * (P + 1) * N * sizeof(T);
  const int64_t tiles = (M + kThreads - 1) / kThreads;
  const int sms = sm_count(f->device);
  int nb = 0;
  // Shared-memory staging when the coefficients fit beside a useful occupancy.
  if (coef_bytes <= 200 * 1024) {
    auto k = banded_sweep_kernel<T, P, SF, SB_, true>;
    SB_TRY(prepare_kernel(k, f->device, coef_bytes, &nb));
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)nb * sms);
    k<<<(unsigned)grid, kThreads, coef_bytes, stream>>>(coef, N, M, ld, rhs, x, tiles);
  } else {
    auto k = banded_sweep_kernel<T, P, SF, SB_, false>;
    SB_TRY(prepare_kernel(k, f->device, 0, &nb));
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)nb * sms);
    k<<<(unsigned)grid, kThreads, 0, stream>>>(coef, N, M, ld, rhs, x, tiles);
  }
  return cuda_check(cudaGetLastError(), "banded sweep launch");
}

}  // namespace

int launch_banded_sweep(const sb_factor* f, Op op, const void* rhs, void* x, int64_t M,
                        int64_t ld, sb_dtype dtype, cudaStream_t stream) {
  const int64_t blk = op_block_len(f->P, f->N);
  if (dtype == SB_F64) {
    const double* c = f->coef64 + (op == OP_PRIMAL ? 0 : blk);
    const double* r = static_cast<const double*>(rhs);
    double* y = static_cast<double*>(x);
    if (f->P == 1)
      return op == OP_PRIMAL ? launch_typed<double, 1, true, false>(f, c, r, y, M, ld, stream)
                             : launch_typed<double, 1, false, true>(f, c, r, y, M, ld, stream);
    return op == OP_PRIMAL ? launch_typed<double, 2, true, false>(f, c, r, y, M, ld, stream)
                           : launch_typed<double, 2, false, true>(f, c, r, y, M, ld, stream);
  }
  const float* c = f->coef32 + (op == OP_PRIMAL ? 0 : blk);
  const float* r = static_cast<const float*>(rhs);
  float* y = static_cast<float*>(x);
  if (f->P == 1)
    return op == OP_PRIMAL ? launch_typed<float, 1, true, false>(f, c, r, y, M, ld, stream)
                           : launch_typed<float, 1, false, true>(f, c, r, y, M, ld, stream);
  return op == OP_PRIMAL ? launch_typed<float, 2, true, false>(f, c, r, y, M, ld, stream)
                         : launch_typed<float, 2, false, true>(f, c, r, y, M, ld, stream);
}

}  // namespace sb
