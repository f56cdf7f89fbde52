// Internal declarations of the sbsolve library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cstdio>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/sbsolve.h"

namespace sb {

// ---------------------------------------------------------------- errors
// Records a message for sb_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
// Clears the message (called at the start of every ABI entry point).
void clear_error();
// Turns a CUDA error into SB_ERR_CUDA with the call site; returns SB_OK on success.
int cuda_check(cudaError_t e, const char* what);

#define SB_CUDA(call)                                              \
  do {                                                             \
    int rc_ = ::sb::cuda_check((call), #call);                     \
    if (rc_ != SB_OK) return rc_;                                  \
  } while (0)

#define SB_TRY(expr)                                               \
  do {                                                             \
    int rc_ = (expr);                                              \
    if (rc_ != SB_OK) return rc_;                                  \
  } while (0)

// ----------------------------------------------------- coefficient blocks
// Both solves (A and A^T) run the same two recurrences over the interleaved
// array, with P = half bandwidth (1 tridiagonal, 2 pentadiagonal) and the
// coefficients prescaled by the reciprocal pivot on the host:
//   forward : u_i = F0_i r_i - F1_i u_{i-1} - F2_i u_{i-2}
//   backward: x_i = B0_i u_i - B1_i x_{i+1} - B2_i x_{i+2}
// For A (primal) F0 is the reciprocal pivot and B0 = 1; for A^T (adjoint)
// F0 = 1 and B0 is the reciprocal pivot.  Each row stores (P + 1) values
// (F0, F1[, F2]).  Coefficients that reach outside the matrix are exactly 0, so
// the sweeps need no edge cases.
// One "op" block = [forward rows 0..N-1][backward rows 0..N-1].
inline int64_t op_block_len(int P, int64_t N) { return 2 * (P + 1) * N; }

// Every kernel's dynamic shared-memory limit is raised once to the opt-in maximum
// of a GB300 CTA (227 KB), never to the size of one launch: a limit lowered for a
// small-N launch would make a later, larger launch of the same kernel fail.
constexpr int kMaxDynSmem = 227 * 1024;

enum Op { OP_PRIMAL = 0, OP_ADJOINT = 1 };

// Launch shape of the sweep kernel (chosen by default_shape or the autotuner).
struct SweepShape {
  int threads = 256;     // threads per CTA (multiple of 32)
  int ctas_per_sm = 0;   // cap on resident CTAs per SM (0 = occupancy limit)
  int spt = 1;           // systems per thread (1 or 2)
  int algo = SB_ALGO_SEQUENTIAL;  // sequential sweeps or the partitioned solve
};

// Partitioned-solve variants: variant v cuts the rows into part_chunks(v) chunks:
// 0 = 16 chunks, one warp each (512 threads); 1 = 32 chunks (1024 threads); 2 = 16
// chunks, half a warp each with two systems per thread (256 threads, paired image).
constexpr int kPartVariants = 3;
inline int part_chunks(int v) { return v == 1 ? 32 : 16; }

// Captured CUDA graphs keyed by the pointers and sizes they were captured with.  A
// caller that passes fresh buffers on every run would otherwise make the cache grow
// without bound, so at most kCap executables are kept and the least recently used
// one is destroyed first (CUDA frees an executable that is still running when it
// completes).  Not thread-safe: the owner holds its lock around every call.
template <typename K>
struct GraphCache {
  static constexpr size_t kCap = 8;
  std::list<std::pair<K, cudaGraphExec_t>> items;  // most recently used first

  cudaGraphExec_t find(const K& key) {
    for (auto it = items.begin(); it != items.end(); ++it)
      if (it->first == key) {
        items.splice(items.begin(), items, it);
        return items.front().second;
      }
    return nullptr;
  }
  void put(const K& key, cudaGraphExec_t exec) {
    items.emplace_front(key, exec);
    while (items.size() > kCap) {
      cudaGraphExecDestroy(items.back().second);
      items.pop_back();
    }
  }
  void clear() {
    for (auto& kv : items) cudaGraphExecDestroy(kv.second);
    items.clear();
  }
  size_t size() const { return items.size(); }
};

}  // namespace sb

struct sb_factor {
  int P = 0;                 // half bandwidth
  int64_t N = 0;
  int device = -1;
  double* coef64 = nullptr;  // device: [primal block | adjoint block], FP64
  float* coef32 = nullptr;   // device: same values rounded to FP32
  float* coefdf = nullptr;   // device: same values as (hi, lo) FP32 pairs
  double* diag64 = nullptr;  // device: the original 2P+1 diagonals, diagonal-major (d * N + i)
  double* arow64 = nullptr;  // device: A row by row, (2P+1) entries per row (offsets -P..P)
  // device images (FP32) of the partitioned solve (partition.h) of A and A^T per
  // variant v (part_chunks(v) chunks of part_L[v] rows); null where it does not apply
  float* part_img[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
  int part_L[3] = {0, 0, 0}, part_NL[3] = {0, 0, 0};
  // FP64 images (block Thomas form) of the small-tile FP64 partitioned solve of A and
  // A^T: 16 chunks of part64_L rows; null where it does not apply
  double* part64_img[2] = {nullptr, nullptr};
  int part64_L = 0;
  // FP64 images of the two-ended sweeps (two_ended.h) of A and A^T: N forward rows,
  // N backward rows, the (2P)^2 interface inverse; split row two_s; null where they
  // do not apply (periodic factors, N < 4P, a zero pivot or a singular interface)
  double* two_img[2] = {nullptr, nullptr};
  int two_s = 0;
  float* arowdf = nullptr;   // device: the same as (hi, lo) FP32 pairs
  // device: FP32 sweep rows [forward | backward] of the primal solve by way of the
  // reversed matrix J A J (J the exchange matrix), row i holding the coefficients
  // used at A's row i: the forward sweep runs from row N-1 down to row 0 and the
  // backward sweep from row 0 up.  Used by refinement passes that alternate their
  // direction; null for periodic factors or when J A J has a zero pivot.
  float* coef32_rev = nullptr;
  std::vector<double> h_coef;  // host copy of coef64
  std::vector<double> h_diag;  // host copy of diag64 (of A' for a periodic factor)
  // Periodic tridiagonal (section 3.3): the factors above are those of A' and each
  // solve applies the Sherman-Morrison correction x = y - f z with
  // f = beta (y_0 + alpha y_{N-1}) and y_0 = w . rhs accumulated in the forward
  // sweep.  Per op (A, A^T): rows (w_i, -z_i) on the device, alpha and beta on the host.
  // Cyclic pentadiagonal (rank 2): per op, rows (w0_i, w1_i, -z0_i, -z1_i) and then
  // 12 scalars P, Q, S^{-1} (2 x 2 each): g = S^{-1} (P (y_0, y_1) + Q (y_{N-2}, y_{N-1})),
  // x = y - z0 g_0 - z1 g_1.
  bool periodic = false;
  int periodic_rank = 0;    // 1 (tridiagonal) or 2 (pentadiagonal)
  double* cyc64 = nullptr;  // device: per op, N rows (2 or 4 values) [+ 12 scalars], FP64
  float* cyc32 = nullptr;   // device: the same rounded to FP32
  float* cycdf = nullptr;   // device: the same as (hi, lo) FP32 pairs
  double cyc_alpha[2] = {0.0, 0.0}, cyc_beta[2] = {0.0, 0.0};
};

struct sb_stepper {
  // stepper.cu: scheme, factor of A and right-hand-side rows; rollout.cu: dA rows
  int kind = 0, scheme = 0, bc = 0;
  int64_t N = 0;
  double coef = 0.0, dt = 0.0;
  sb_factor* fac = nullptr;
  int NB = 0;            // B band width (0 = identity)
  bool has_e = false;
  double* r64 = nullptr;  // device rhs coefficient rows, FP64
  float* rdf = nullptr;   // same as (hi, lo) pairs
  double* dA64 = nullptr;  // d A / d coef row by row ((2P+1) per row), for the rollout adjoint
  // travelling-wave forcing (section 6.1): adv * W(C) + amp[m] * g[i] on the right-hand side
  bool forced = false;
  double adv = 0.0;
  double* g64 = nullptr;  // device forcing profile, N values
  std::mutex mu;
  // captured step graphs: fused steps (state, M, ld, arith, steps), forced steps
  // (state, amp, M, ld) and FP32 + refinement steps (state, work, M, ld,
  // n_refine * 2 + residual mode)
  sb::GraphCache<std::tuple<uintptr_t, int64_t, int64_t, int, int>> graphs;
  sb::GraphCache<std::tuple<uintptr_t, uintptr_t, int64_t, int64_t>> forced_graphs;
  sb::GraphCache<std::tuple<uintptr_t, uintptr_t, int64_t, int64_t, int>> refined_graphs;
};

namespace sb {

// ------------------------------------------------------------ validation
// Checks that [p, p + bytes) is device/managed memory of `device`, aligned to
// `align`.  Host pointers and out-of-allocation ranges are rejected.
int check_device_range(const void* p, size_t bytes, size_t align, int device, const char* name);
// Rejects overlap of [a, a+abytes) and [b, b+bbytes) unless a == b.
int check_alias(const void* a, size_t abytes, const void* b, size_t bbytes, const char* na,
                const char* nb);

// RAII guard that makes `device` current and restores the previous device.
struct DeviceGuard {
  int prev = -1;
  int rc = SB_OK;
  explicit DeviceGuard(int device);
  ~DeviceGuard();
};

int sm_count(int device);

// Resident CTAs per SM of `kernel` at (threads, smem); raises the kernel's
// dynamic shared-memory limit to kMaxDynSmem the first time (cached).
int kernel_occupancy(const void* kernel, int device, int threads, size_t smem, int* blocks_per_sm);

// Diagonals of a workload matrix (sb_build_matrix); sets *P to 1 or 2.
int build_matrix(int kind, int64_t N, double coef, std::vector<double>& diags, int* P);

// Launchers implemented in sweep.cu.
SweepShape default_shape(const sb_factor* f, sb_arith arith);
// Tuned shape for (device, P, N, arith, dtypes) or the default (tune.cpp).
SweepShape shape_for(const sb_factor* f, sb_arith arith, sb_dtype rt, sb_dtype xt);
// One fused stepper step from src into dst (stepper.cu).
int stepper_step(const sb_stepper* st, const double* src, double* dst, int64_t M, int64_t ld,
                 sb_arith arith, cudaStream_t stream);
// The partitioned solve (partition.cu); shape.algo == SB_ALGO_PARTITIONED.
// The small-tile FP64 partitioned solve (partition64.cu): 128-thread CTAs, 16 chunks.
constexpr int kPart64Threads = 128;
constexpr int kPart64Chunks = 16;
constexpr int kPart64Levels = 4;  // cyclic-reduction levels for its 15 chunk boundaries
bool partitioned64_applies(const sb_factor* f, Op op, sb_dtype rhs_dtype, sb_dtype x_dtype,
                           int64_t M, sb_arith arith);
int launch_partitioned64(const sb_factor* f, Op op, const void* rhs, void* x, int64_t M, int64_t ld,
                         const SweepShape& shape, cudaStream_t stream);
// Variant of a partitioned shape (threads 512 -> 0, 1024 -> 1, 256 -> 2, else -1).
int part_variant(int threads);
bool partitioned_applies(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype,
                         sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, int threads);
// Reads and resets the count of partitioned-solve CTAs that timed out on `device`.
int partition_timeouts(int device, unsigned* count);
int launch_partitioned(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype, void* x,
                       sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith,
                       const SweepShape& shape, cudaStream_t stream);
int launch_sweep(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype, void* x,
                 sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, const SweepShape& shape,
                 cudaStream_t stream);
// refine.cu: grouped (and refined) solves, G groups in one launch per pass.
// fp32_sweeps: an FP64 right-hand side is swept in FP32 even with n_refine == 0 (by
// default an FP64 right-hand side gets FP64 sweeps unless refinement is asked for).
int solve_groups(int G, const sb_factor* const* fs, const void* const* rhs, void* const* x,
                 const int64_t* M, const int64_t* ld, sb_dtype rt, sb_dtype xt, sb_arith arith,
                 int n_refine, sb_arith res_arith, void* const* work, const size_t* work_bytes,
                 cudaStream_t stream, bool fp32_sweeps = false);
// One FP32 + refinement time step in one launch (refine.cu): per tile, the FP64
// right-hand side f = B C + E phi(C) of the state (rows rcoef: NB B values then, if
// has_e, 3 E values per row) into fbuf, the FP32 solve of f into the state and
// n_refine correction passes (residual in FP64 or double-float).
int refined_step(const sb_factor* f, const double* rcoef, int NB, bool has_e, double* state, double* fbuf,
                 float* scratch, int64_t M, int64_t ld, int n_refine, sb_arith residual_arith,
                 cudaStream_t stream);
}  // namespace sb
