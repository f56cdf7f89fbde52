// Batched forward/backward sweeps with one shared factor (Algorithms 2 and 4, and
// the transposed solve), for every arithmetic policy of arith.cuh.
//
// Mapping.  One thread owns one system m; a warp owns 32 consecutive systems (a
// "tile"), so every row access i*ld + m is one coalesced transaction per warp.
// CTAs are persistent: each stages the shared coefficients into shared memory
// once (the single device copy of section 2, broadcast from shared memory instead
// of the caches) and its warps then take tiles round-robin over the grid.
//
// Per system: the forward sweep reads the right-hand side and writes its
// intermediate (A::S, at most the size of an output element) in place into x; the
// backward sweep reads it back (the same thread, so no synchronisation) and
// writes the solution over it.  Rows are fetched R at a time into registers with
// double buffering: the next batch is in flight while the current one is swept.
#include <algorithm>
#include <type_traits>
#include <mutex>
#include <unordered_map>

#include "sb_internal.h"
#include "sweep_tile.cuh"

namespace sb {
namespace {

// Per-op length of a periodic factor's correction data (rank 1 or 2).
__host__ __device__ constexpr int cyc_len(int rank, int N) { return rank == 1 ? 2 * N : rank == 2 ? 4 * N + 12 : 0; }

// Single-factor kernel: persistent CTAs stage the coefficients once, then their
// warps take tiles round-robin over the grid.  CYC: periodic matrices (rank-1
// tridiagonal of section 3.3, rank-2 cyclic pentadiagonal); the correction data is
// staged after the coefficients.  GC: the factors do not fit in shared memory
// (large N), so the sweeps read the single device copy directly (warp-uniform
// loads, served by L1/L2) instead of a staged one.
template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO, int SPT, int R,
          int CYC, bool GC = false>
__global__ void __launch_bounds__(512)
sweep_kernel(const typename A::C* __restrict__ coef, int N, int64_t M, int64_t ld,
             const TI* rhs, TO* x, int64_t ntiles, const typename A::C* __restrict__ cyc,
             typename A::C alpha, typename A::C beta) {
  using C = typename A::C;
  constexpr int W = P + 1;
  const C* fw;
  const C* cy;
  if constexpr (GC) {
    fw = coef;
    cy = cyc;
  } else {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* cs = reinterpret_cast<C*>(smem_raw);
    stage(cs, coef, 2 * W * N);
    if constexpr (CYC) stage(cs + 2 * W * N, cyc, cyc_len(CYC, N));
    __syncthreads();
    fw = cs;
    cy = cs + 2 * W * N;
  }
  const int nw = blockDim.x >> 5;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5); tile < ntiles;
       tile += (int64_t)gridDim.x * nw)
    sweep_tile<A, P, F_ONE, B_ONE, TI, TO, SPT, R, CYC>(fw, fw + W * N, N, M, ld, rhs, x, tile,
                                                         cy, alpha, beta);
}

// Staged single-factor kernel (SB_ALGO_STAGED): the coefficients as above, then a
// ring of kStagedRows slots per thread for the rows in flight (sweep_tile_staged),
// so that up to 1024 threads per CTA fit in the registers (512 in double-float
// arithmetic, whose values take two registers).
constexpr int kStagedRows = 8;
constexpr int kStagedBatch = 4;

template <class A>
__host__ __device__ constexpr int staged_max_threads() {
  return std::is_same_v<A, DFArith> ? 512 : 1024;
}

template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO>
__global__ void __launch_bounds__(staged_max_threads<A>())
sweep_staged_kernel(const typename A::C* __restrict__ coef, int N, int64_t M, int64_t ld, const TI* rhs,
                    TO* x, int64_t ntiles, unsigned ring_off) {
  using C = typename A::C;
  constexpr int W = P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* cs = reinterpret_cast<C*>(smem_raw);
  stage(cs, coef, 2 * W * N);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5); tile < ntiles;
       tile += (int64_t)gridDim.x * nw)
    sweep_tile_staged<A, P, F_ONE, B_ONE, TI, TO, kStagedRows, kStagedBatch>(cs, cs + W * N, N, M, ld, rhs, x,
                                                                            tile, smem_raw + ring_off);
}

// Two-ended kernel (SB_ALGO_TWO_ENDED; FP64 rhs and x, native arithmetic): every
// system is eliminated from both ends at once (two_ended.h).  A warp takes 16
// systems: lane l < 16 runs the top half of system l (rows 0 .. s-1 down, then back
// up from the interface) and lane l + 16 its bottom half (rows N-1 .. s up, then back
// down), so a batch gives twice as many warps, each with all 32 lanes busy; with
// 65536 systems that is 6.7 warps per scheduler instead of 3.4, and the FP64 pipe
// of the scheduler with the most warps no longer sets the time alone.  The two
// halves of a system meet in the 2P x 2P interface system through one warp shuffle.
// Each lane's rows go through a ring of kTwoRows slots in shared memory, as in the
// staged sweeps.  Image in shared memory: fw (W N) | bw (W N) | the (2P)^2 interface
// inverse.
constexpr int kTwoRows = 8;
constexpr int kTwoBatch = 4;

template <int P>
__device__ __forceinline__ void two_ended_tile(const double* fw, const double* bw, const double* minv, int N,
                                               int s, int64_t M, int64_t ld, const double* rhs, double* x,
                                               int64_t tile, unsigned char* ring) {
  using A = NativeArith<double>;
  constexpr int W = P + 1;
  constexpr int D = kTwoRows;
  constexpr int K = kTwoBatch;
  constexpr int NZ = 2 * P;
  static_assert((D & (D - 1)) == 0 && D % K == 0, "the ring length is a power of two and a multiple of K");
  const int lane = threadIdx.x & 31;
  const bool top = lane < 16;
  const int64_t m = tile * 16 + (lane & 15);
  // lanes l and l + 16 hold the same system, so both are in the mask or neither
  const unsigned mask = __ballot_sync(0xffffffffu, m < M);
  if (m >= M) return;
  const double* r = rhs + m;
  double* y = x + m;
  const int T = blockDim.x;
  double* rs = reinterpret_cast<double*>(ring) + threadIdx.x;  // slot k at rs[k * T]
  __threadfence_block();  // this thread's stores of the previous tile before the copies below

  // ---- forward: step t is row t (top) or row N-1-t (bottom); u in place in x
  const int nf = top ? s : N - s;
  const int TF = s > N - s ? s : N - s;
  auto issue_f = [&](int t) {
    if (t < nf) cp_async<8>(rs + (t & (D - 1)) * T, r + (int64_t)(top ? t : N - 1 - t) * ld);
    cp_commit();
  };
#pragma unroll
  for (int t = 0; t < D; ++t) issue_f(t);
  double v1 = 0.0, v2 = 0.0;
  for (int t0 = 0; t0 < TF; t0 += K) {
    cp_wait<D - K>();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int t = t0 + j;
      if (t < nf) {
        const int i = top ? t : N - 1 - t;
        const double u = A::step<P, false>(fw + W * i, rs[(t & (D - 1)) * T], v1, v2);
        y[(int64_t)i * ld] = u;
        v2 = v1;
        v1 = u;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) issue_f(t0 + D + j);
  }
  cp_wait<0>();
  __threadfence_block();  // the stores of u before the copies that read them back

  // ---- interface: z = (x_{s-P} .. x_{s+P-1}) = Minv (u_{s-P} .. u_{s+P-1}); the top
  // lane ends at u_{s-1} (v1), u_{s-2} (v2), the bottom lane at u_s (v1), u_{s+1} (v2)
  const double o1 = __shfl_xor_sync(mask, v1, 16);
  const double o2 = __shfl_xor_sync(mask, v2, 16);
  double uz[NZ];
  if constexpr (P == 2) {
    uz[0] = top ? v2 : o2;
    uz[1] = top ? v1 : o1;
    uz[2] = top ? o1 : v1;
    uz[3] = top ? o2 : v2;
  } else {
    uz[0] = top ? v1 : o1;
    uz[1] = top ? o1 : v1;
  }
  const int j0 = top ? 0 : P;  // this lane's interface rows: s-P .. s-1 (top), s .. s+P-1
  double z[P];
#pragma unroll
  for (int jj = 0; jj < P; ++jj) {
    const int j = j0 + jj;
    double v = 0.0;
#pragma unroll
    for (int q = 0; q < NZ; ++q) v = fma(minv[j * NZ + q], uz[q], v);
    z[jj] = v;
    st_stream(y + (int64_t)(s - P + j) * ld, v);
  }

  // ---- backward: rows s-P-1 .. 0 (top) or s+P .. N-1 (bottom)
  const int nbk = top ? s - P : N - s - P;
  const int TB = s > N - s ? s - P : N - s - P;
  auto issue_b = [&](int t) {
    if (t < nbk) cp_async<8>(rs + (t & (D - 1)) * T, y + (int64_t)(top ? s - P - 1 - t : s + P + t) * ld);
    cp_commit();
  };
#pragma unroll
  for (int t = 0; t < D; ++t) issue_b(t);
  // the two nearest solved rows: x_{i+1}, x_{i+2} (top) or x_{i-1}, x_{i-2} (bottom)
  double x1 = top ? z[0] : z[P - 1];
  double x2 = P == 2 ? (top ? z[P - 1] : z[0]) : 0.0;
  for (int t0 = 0; t0 < TB; t0 += K) {
    cp_wait<D - K>();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int t = t0 + j;
      if (t < nbk) {
        const int i = top ? s - P - 1 - t : s + P + t;
        const double xi = A::step<P, true>(bw + W * i, rs[(t & (D - 1)) * T], x1, x2);
        st_stream(y + (int64_t)i * ld, xi);
        x2 = x1;
        x1 = xi;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) issue_b(t0 + D + j);
  }
  cp_wait<0>();
}

template <int P>
__global__ void __launch_bounds__(1024)
sweep_two_ended_kernel(const double* __restrict__ img, int N, int s, int64_t M, int64_t ld, const double* rhs,
                       double* x, int64_t ntiles, unsigned ring_off) {
  constexpr int W = P + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* cs = reinterpret_cast<double*>(smem_raw);
  stage(cs, img, 2 * W * N + 4 * P * P);
  __syncthreads();
  const int nw = blockDim.x >> 5;
  for (int64_t tile = blockIdx.x + (int64_t)gridDim.x * (threadIdx.x >> 5); tile < ntiles;
       tile += (int64_t)gridDim.x * nw)
    two_ended_tile<P>(cs, cs + W * N, cs + 2 * W * N, N, s, M, ld, rhs, x, tile, smem_raw + ring_off);
}

// The periodic correction data of a factor for an arithmetic policy: (w_i, -z_i)
// rows of op `o` and the scalars alpha, beta as coefficients.
template <class A>
struct CycData;
template <>
struct CycData<NativeArith<double>> {
  static const double* rows(const sb_factor* f, int o) {
    return f->cyc64 ? f->cyc64 + cyc_len(f->periodic_rank, (int)f->N) * o : nullptr;
  }
  static double coef(double v) { return v; }
};
template <>
struct CycData<NativeArith<float>> {
  static const float* rows(const sb_factor* f, int o) {
    return f->cyc32 ? f->cyc32 + cyc_len(f->periodic_rank, (int)f->N) * o : nullptr;
  }
  static float coef(double v) { return (float)v; }
};
template <>
struct CycData<DFArith> {
  static const df* rows(const sb_factor* f, int o) {
    return f->cycdf ? reinterpret_cast<const df*>(f->cycdf) + cyc_len(f->periodic_rank, (int)f->N) * o
                    : nullptr;
  }
  static df coef(double v) {
    const float h = (float)v;
    return df{h, (float)(v - (double)h)};
  }
};

// ----------------------------------------------------------------- launching

template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO, int SPT, int R,
          int CYC>
int launch(const sb_factor* f, const typename A::C* coef, const void* rhs, void* x, int64_t M,
           int64_t ld, const SweepShape& shape, cudaStream_t stream, int op) {
  using C = typename A::C;
  const int N = (int)f->N;
  size_t smem = ((size_t)2 * (P + 1) * N + (size_t)cyc_len(CYC, N)) * sizeof(C);
  auto k = sweep_kernel<A, P, F_ONE, B_ONE, TI, TO, SPT, R, CYC>;
  if (smem > (size_t)kMaxDynSmem) {
    // FP64 factors of a large N are read from device memory; the other policies
    // keep the staged form only
    if constexpr (std::is_same_v<A, NativeArith<double>> && std::is_same_v<TI, double> &&
                  std::is_same_v<TO, double>) {
      k = sweep_kernel<A, P, F_ONE, B_ONE, TI, TO, SPT, R, CYC, true>;
      smem = 0;
    } else {
      return fail(SB_ERR_UNSUPPORTED,
                  "N=%d: the shared factors (%zu B) exceed the shared memory of one CTA "
                  "(only FP64 solves read them from device memory)", N, smem);
    }
  }
  const int threads = shape.threads;
  if (threads < 32 || threads > 512 || threads % 32 != 0)
    return fail(SB_ERR_INVALID_ARG, "threads per CTA must be a multiple of 32 in [32, 512]");
  int nb = 0;
  SB_TRY(kernel_occupancy(reinterpret_cast<const void*>(k), f->device, threads, smem, &nb));
  if (shape.ctas_per_sm > 0) nb = std::min(nb, shape.ctas_per_sm);
  const int64_t ntiles = (M + 32 * SPT - 1) / (32 * SPT);
  // one CTA per resident slot at most, tiles dealt round-robin over the CTAs first
  // (tile = block + grid * warp) so that every SM gets an equal share
  const int64_t grid =
      std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
  const C* cyc = CYC ? CycData<A>::rows(f, op) : nullptr;
  const C alpha = CycData<A>::coef(CYC ? f->cyc_alpha[op] : 0.0);
  const C beta = CycData<A>::coef(CYC ? f->cyc_beta[op] : 0.0);
  k<<<(unsigned)grid, threads, smem, stream>>>(coef, N, M, ld, static_cast<const TI*>(rhs),
                                              static_cast<TO*>(x), ntiles, cyc, alpha, beta);
  return cuda_check(cudaGetLastError(), "sweep kernel launch");
}

// The staged sweeps; *applied = false (nothing launched, SB_OK) where they do not
// apply: periodic factors, or coefficients and ring beyond one CTA's shared memory.
template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO, int CYC>
int launch_staged(const sb_factor* f, const typename A::C* coef, const void* rhs, void* x, int64_t M,
                  int64_t ld, const SweepShape& shape, cudaStream_t stream, bool* applied) {
  using C = typename A::C;
  *applied = false;
  if constexpr (CYC != 0) {
    return SB_OK;
  } else {
    const int N = (int)f->N;
    const int threads = shape.threads;
    if (threads < 32 || threads > staged_max_threads<A>() || threads % 32 != 0)
      return fail(SB_ERR_INVALID_ARG, "threads per CTA must be a multiple of 32 in [32, %d] for the staged sweeps",
                  staged_max_threads<A>());
    const size_t ring_off = ((size_t)2 * (P + 1) * N * sizeof(C) + 15) / 16 * 16;
    const size_t smem =
        ring_off + (size_t)kStagedRows * threads * staged_slot_bytes<TI, typename A::S>();
    if (smem > (size_t)kMaxDynSmem) return SB_OK;
    *applied = true;
    auto k = sweep_staged_kernel<A, P, F_ONE, B_ONE, TI, TO>;
    int nb = 0;
    SB_TRY(kernel_occupancy(reinterpret_cast<const void*>(k), f->device, threads, smem, &nb));
    if (shape.ctas_per_sm > 0) nb = std::min(nb, shape.ctas_per_sm);
    const int64_t ntiles = (M + 31) / 32;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
    k<<<(unsigned)grid, threads, smem, stream>>>(coef, N, M, ld, static_cast<const TI*>(rhs),
                                                static_cast<TO*>(x), ntiles, (unsigned)ring_off);
    return cuda_check(cudaGetLastError(), "staged sweep kernel launch");
  }
}

// The two-ended sweeps of op (A or A^T); *applied = false (nothing launched, SB_OK)
// where they do not apply: no image (periodic factor, N < 4P, a zero pivot or a
// singular interface), or image and ring beyond one CTA's shared memory.
int launch_two_ended(const sb_factor* f, Op op, const void* rhs, void* x, int64_t M, int64_t ld,
                     const SweepShape& shape, cudaStream_t stream, bool* applied) {
  *applied = false;
  const double* img = f->two_img[op == OP_PRIMAL ? 0 : 1];
  if (img == nullptr) return SB_OK;
  const int N = (int)f->N, P = f->P, threads = shape.threads;
  if (threads < 32 || threads > 1024 || threads % 32 != 0)
    return fail(SB_ERR_INVALID_ARG, "threads per CTA must be a multiple of 32 in [32, 1024] for the two-ended sweeps");
  const size_t ring_off = (((size_t)2 * (P + 1) * N + 4 * P * P) * sizeof(double) + 15) / 16 * 16;
  const size_t smem = ring_off + (size_t)kTwoRows * threads * sizeof(double);
  if (smem > (size_t)kMaxDynSmem) return SB_OK;
  *applied = true;
  auto k = P == 1 ? sweep_two_ended_kernel<1> : sweep_two_ended_kernel<2>;
  int nb = 0;
  SB_TRY(kernel_occupancy(reinterpret_cast<const void*>(k), f->device, threads, smem, &nb));
  if (shape.ctas_per_sm > 0) nb = std::min(nb, shape.ctas_per_sm);
  const int64_t ntiles = (M + 15) / 16;  // 16 systems per warp
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
  k<<<(unsigned)grid, threads, smem, stream>>>(img, N, f->two_s, M, ld, static_cast<const double*>(rhs),
                                              static_cast<double*>(x), ntiles, (unsigned)ring_off);
  return cuda_check(cudaGetLastError(), "two-ended sweep kernel launch");
}

template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO, int CYC>
int launch_spt(const sb_factor* f, const typename A::C* coef, const void* rhs, void* x, int64_t M,
               int64_t ld, const SweepShape& shape, cudaStream_t stream, int op) {
  if (shape.algo == SB_ALGO_STAGED) {
    bool applied = false;
    const int rc = launch_staged<A, P, F_ONE, B_ONE, TI, TO, CYC>(f, coef, rhs, x, M, ld, shape, stream, &applied);
    if (rc != SB_OK || applied) return rc;
    // where the staged sweeps do not apply, the sequential ones with the default shape
    const sb_arith arith = std::is_same_v<A, DFArith> ? SB_ARITH_DF32 : SB_ARITH_NATIVE;
    return launch_spt<A, P, F_ONE, B_ONE, TI, TO, CYC>(f, coef, rhs, x, M, ld, default_shape(f, arith), stream, op);
  }
  if (shape.spt == 2)
    return launch<A, P, F_ONE, B_ONE, TI, TO, 2, 4, CYC>(f, coef, rhs, x, M, ld, shape, stream, op);
  if (shape.spt != 1) return fail(SB_ERR_INVALID_ARG, "systems per thread must be 1 or 2");
  return launch<A, P, F_ONE, B_ONE, TI, TO, 1, kRows, CYC>(f, coef, rhs, x, M, ld, shape, stream, op);
}

template <class A, typename TI, typename TO>
int dispatch_pb(const sb_factor* f, Op op, const typename A::C* base, const void* rhs, void* x,
                int64_t M, int64_t ld, const SweepShape& shape, cudaStream_t stream) {
  const typename A::C* c = base + (op == OP_PRIMAL ? 0 : op_block_len(f->P, f->N));
  const int o = op == OP_PRIMAL ? 0 : 1;
  if (f->P == 1) {
    if (f->periodic)
      return op == OP_PRIMAL
                 ? launch_spt<A, 1, false, true, TI, TO, 1>(f, c, rhs, x, M, ld, shape, stream, o)
                 : launch_spt<A, 1, true, false, TI, TO, 1>(f, c, rhs, x, M, ld, shape, stream, o);
    return op == OP_PRIMAL
               ? launch_spt<A, 1, false, true, TI, TO, 0>(f, c, rhs, x, M, ld, shape, stream, o)
               : launch_spt<A, 1, true, false, TI, TO, 0>(f, c, rhs, x, M, ld, shape, stream, o);
  }
  if (f->periodic)
    return op == OP_PRIMAL
               ? launch_spt<A, 2, false, true, TI, TO, 2>(f, c, rhs, x, M, ld, shape, stream, o)
               : launch_spt<A, 2, true, false, TI, TO, 2>(f, c, rhs, x, M, ld, shape, stream, o);
  return op == OP_PRIMAL
             ? launch_spt<A, 2, false, true, TI, TO, 0>(f, c, rhs, x, M, ld, shape, stream, o)
             : launch_spt<A, 2, true, false, TI, TO, 0>(f, c, rhs, x, M, ld, shape, stream, o);
}

}  // namespace

namespace {
std::mutex g_occ_mu;
std::unordered_map<uint64_t, int> g_occ;
}  // namespace

int kernel_occupancy(const void* kernel, int device, int threads, size_t smem, int* blocks_per_sm) {
  const uint64_t key = (reinterpret_cast<uint64_t>(kernel) * 31u) ^ ((uint64_t)smem << 20) ^
                       ((uint64_t)threads << 8) ^ (uint64_t)device;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
      *blocks_per_sm = it->second;
      return SB_OK;
    }
  }
  SB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
  int nb = 0;
  SB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem));
  if (nb < 1)
    return fail(SB_ERR_UNSUPPORTED, "kernel cannot be resident (%d threads, %zu B smem)", threads, smem);
  std::lock_guard<std::mutex> lk(g_occ_mu);
  g_occ[key] = nb;
  *blocks_per_sm = nb;
  return SB_OK;
}

SweepShape default_shape(const sb_factor* f, sb_arith arith) {
  SweepShape s;
  s.threads = (arith == SB_ARITH_DF32) ? 128 : 256;
  s.ctas_per_sm = 0;  // occupancy limit
  s.spt = 1;
  (void)f;
  return s;
}

int launch_sweep(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype, void* x,
                 sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, const SweepShape& shape,
                 cudaStream_t stream) {
  if (shape.algo == SB_ALGO_PARTITIONED && shape.threads == kPart64Threads) {
    if (partitioned64_applies(f, op, rhs_dtype, x_dtype, M, arith))
      return launch_partitioned64(f, op, rhs, x, M, ld, shape, stream);
    return launch_sweep(f, op, rhs, rhs_dtype, x, x_dtype, M, ld, arith, default_shape(f, arith),
                        stream);
  }
  if (shape.algo == SB_ALGO_PARTITIONED) {
    if (partitioned_applies(f, op, rhs, rhs_dtype, x_dtype, M, ld, arith, shape.threads))
      return launch_partitioned(f, op, rhs, rhs_dtype, x, x_dtype, M, ld, arith, shape, stream);
    // where the partition does not apply (sizes, dtypes, alignment) the sequential
    // sweeps run with their default shape
    return launch_sweep(f, op, rhs, rhs_dtype, x, x_dtype, M, ld, arith, default_shape(f, arith),
                        stream);
  }
  if (shape.algo == SB_ALGO_TWO_ENDED) {
    if (arith == SB_ARITH_NATIVE && rhs_dtype == SB_F64 && x_dtype == SB_F64) {
      bool applied = false;
      const int rc = launch_two_ended(f, op, rhs, x, M, ld, shape, stream, &applied);
      if (rc != SB_OK || applied) return rc;
    }
    // where the two-ended sweeps do not apply, the sequential ones with the default shape
    return launch_sweep(f, op, rhs, rhs_dtype, x, x_dtype, M, ld, arith, default_shape(f, arith), stream);
  }
  if (shape.algo != SB_ALGO_SEQUENTIAL && shape.algo != SB_ALGO_STAGED)
    return fail(SB_ERR_INVALID_ARG, "unknown algorithm %d", shape.algo);
  if (arith == SB_ARITH_NATIVE) {
    if (rhs_dtype == SB_F64 && x_dtype == SB_F64)
      return dispatch_pb<NativeArith<double>, double, double>(f, op, f->coef64, rhs, x, M, ld,
                                                              shape, stream);
    if (rhs_dtype == SB_F32 && x_dtype == SB_F32)
      return dispatch_pb<NativeArith<float>, float, float>(f, op, f->coef32, rhs, x, M, ld, shape,
                                                           stream);
    if (rhs_dtype == SB_F32 && x_dtype == SB_F64)
      return dispatch_pb<NativeArith<float>, float, double>(f, op, f->coef32, rhs, x, M, ld,
                                                            shape, stream);
  } else if (arith == SB_ARITH_DF32) {
    const df* c = reinterpret_cast<const df*>(f->coefdf);
    if (rhs_dtype == SB_F64 && x_dtype == SB_F64)
      return dispatch_pb<DFArith, double, double>(f, op, c, rhs, x, M, ld, shape, stream);
    if (rhs_dtype == SB_F32 && x_dtype == SB_F64)
      return dispatch_pb<DFArith, float, double>(f, op, c, rhs, x, M, ld, shape, stream);
  }
  return fail(SB_ERR_UNSUPPORTED, "unsupported combination: rhs dtype %d, x dtype %d, arith %d",
              (int)rhs_dtype, (int)x_dtype, (int)arith);
}

}  // namespace sb
