// Launch-shape table and autotuner for the batched solves.
//
// A shape (threads per CTA, resident CTAs per SM, systems per thread, algorithm) is looked up
// per (device, half bandwidth, N, arithmetic, rhs dtype, x dtype).  Entries come
// from sb_shape_set (e.g. a persisted tuning cache) or from sb_autotune, which
// times every candidate shape on the caller's buffers with CUDA events and keeps
// the fastest.  Without an entry, FP32 right-hand sides in native arithmetic use the
// partitioned solve where it applies and everything else the default of sweep.cu.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "sb_internal.h"

namespace sb {
namespace {

using Key = std::tuple<int, int, int64_t, int, int, int>;
std::mutex g_mu;
std::map<Key, SweepShape> g_table;

Key make_key(const sb_factor* f, sb_arith arith, sb_dtype rt, sb_dtype xt) {
  return Key(f->device, f->P, f->N, (int)arith, (int)rt, (int)xt);
}

}  // namespace

SweepShape shape_for(const sb_factor* f, sb_arith arith, sb_dtype rt, sb_dtype xt) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(make_key(f, arith, rt, xt));
  if (it != g_table.end()) return it->second;
  // FP32 right-hand sides in native arithmetic default to the partitioned solve where
  // the factor has its data (the launcher falls back to the sweeps per call where it
  // does not apply)
  if (arith == SB_ARITH_NATIVE && rt == SB_F32 && (f->part_img[0][0] || f->part_img[1][0])) {
    SweepShape s;
    // two systems per thread (variant 2) where the factor has its image
    s.threads = (f->part_img[0][2] || f->part_img[1][2]) ? 256 : 512;
    s.ctas_per_sm = 0;
    s.spt = 1;
    s.algo = SB_ALGO_PARTITIONED;
    return s;
  }
  return default_shape(f, arith);
}

}  // namespace sb

using namespace sb;

extern "C" {

int sb_shape_get(const sb_factor* f, sb_arith arith, sb_dtype rhs_dtype, sb_dtype x_dtype,
                 sb_shape* out) {
  clear_error();
  if (!f || !out) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  const SweepShape s = shape_for(f, arith, rhs_dtype, x_dtype);
  out->threads = s.threads;
  out->ctas_per_sm = s.ctas_per_sm;
  out->systems_per_thread = s.spt;
  out->algorithm = s.algo;
  return SB_OK;
}

int sb_shape_set(const sb_factor* f, sb_arith arith, sb_dtype rhs_dtype, sb_dtype x_dtype,
                 const sb_shape* shape) {
  clear_error();
  if (!f || !shape) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (shape->algorithm != SB_ALGO_SEQUENTIAL && shape->algorithm != SB_ALGO_PARTITIONED &&
      shape->algorithm != SB_ALGO_STAGED && shape->algorithm != SB_ALGO_TWO_ENDED)
    return fail(SB_ERR_INVALID_ARG, "unknown algorithm %d", shape->algorithm);
  if (shape->ctas_per_sm < 0 || shape->ctas_per_sm > 32)
    return fail(SB_ERR_INVALID_ARG, "ctas_per_sm must be in [0, 32]");
  if (shape->algorithm == SB_ALGO_SEQUENTIAL) {
    if (shape->threads < 32 || shape->threads > 512 || shape->threads % 32 != 0)
      return fail(SB_ERR_INVALID_ARG, "threads must be a multiple of 32 in [32, 512]");
    if (shape->systems_per_thread != 1 && shape->systems_per_thread != 2)
      return fail(SB_ERR_INVALID_ARG, "systems_per_thread must be 1 or 2");
  } else if (shape->algorithm == SB_ALGO_STAGED || shape->algorithm == SB_ALGO_TWO_ENDED) {
    const int cap = (arith == SB_ARITH_DF32 && shape->algorithm == SB_ALGO_STAGED) ? 512 : 1024;
    if (shape->threads < 32 || shape->threads > cap || shape->threads % 32 != 0)
      return fail(SB_ERR_INVALID_ARG, "threads must be a multiple of 32 in [32, %d] for this algorithm", cap);
    if (shape->systems_per_thread != 1)
      return fail(SB_ERR_INVALID_ARG, "the staged and two-ended sweeps take systems_per_thread = 1");
  } else {
    if (part_variant(shape->threads) < 0 && shape->threads != kPart64Threads)
      return fail(SB_ERR_INVALID_ARG, "the partitioned solve runs 128, 256, 512 or 1024 threads per CTA");
    if (shape->systems_per_thread != 1 || shape->ctas_per_sm > 1)
      return fail(SB_ERR_INVALID_ARG,
                  "the partitioned solve takes systems_per_thread = 1 and ctas_per_sm 0 or 1");
  }
  SweepShape s;
  s.threads = shape->threads;
  s.ctas_per_sm = shape->ctas_per_sm;
  s.spt = shape->systems_per_thread;
  s.algo = shape->algorithm;
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[make_key(f, arith, rhs_dtype, x_dtype)] = s;
  return SB_OK;
}

int sb_autotune(const sb_factor* f, int transpose, const void* rhs, sb_dtype rhs_dtype, void* x,
                sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, void* stream,
                sb_shape* best, float* best_ms) {
  clear_error();
  if (!f) return fail(SB_ERR_INVALID_ARG, "factor handle is NULL");
  if (M < 1) return fail(SB_ERR_INVALID_ARG, "autotuning needs M >= 1");
  if (rhs == x) return fail(SB_ERR_INVALID_ARG, "autotuning needs rhs and x to be different arrays");
  // Validate once through the normal path (also rejects unsupported combinations).
  SB_TRY(sb_solve_batched_ex(f, transpose, rhs, rhs_dtype, x, x_dtype, M, ld, arith, stream));
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  cudaStream_t st = (cudaStream_t)stream;
  const Op op = transpose ? OP_ADJOINT : OP_PRIMAL;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SB_CUDA(cudaEventCreate(&e0));
  int rc = cuda_check(cudaEventCreate(&e1), "cudaEventCreate");
  if (rc != SB_OK) {
    cudaEventDestroy(e0);
    return rc;
  }
  SweepShape winner = default_shape(f, arith);
  float winner_ms = 1e30f;
  std::vector<SweepShape> cands;
  for (int spt : {1, 2})
    for (int threads : {64, 128, 256, 512})
      for (int cps : {0, 1, 2}) {
        SweepShape s;
        s.threads = threads;
        s.ctas_per_sm = cps;
        s.spt = spt;
        cands.push_back(s);
      }
  for (int threads : {256, 512, 768, 1024})
    if (threads <= 512 || arith != SB_ARITH_DF32) {
      SweepShape s;
      s.threads = threads;
      s.ctas_per_sm = 0;
      s.algo = SB_ALGO_STAGED;
      cands.push_back(s);
    }
  if (f->two_img[op == OP_PRIMAL ? 0 : 1] && arith == SB_ARITH_NATIVE && rhs_dtype == SB_F64 &&
      x_dtype == SB_F64)
    for (int threads : {256, 512, 768, 1024}) {
      SweepShape s;
      s.threads = threads;
      s.ctas_per_sm = 0;
      s.algo = SB_ALGO_TWO_ENDED;
      cands.push_back(s);
    }
  if (partitioned64_applies(f, op, rhs_dtype, x_dtype, M, arith)) {
    SweepShape s;
    s.threads = kPart64Threads;
    s.ctas_per_sm = 0;
    s.algo = SB_ALGO_PARTITIONED;
    cands.push_back(s);
  }
  for (int threads : {256, 512, 1024})
    if (partitioned_applies(f, op, rhs, rhs_dtype, x_dtype, M, ld, arith, threads)) {
      SweepShape s;
      s.threads = threads;
      s.ctas_per_sm = 0;
      s.algo = SB_ALGO_PARTITIONED;
      cands.push_back(s);
    }
  for (const SweepShape& s : cands) {
    // one warm-up launch, then the best of three timed launches
    if (launch_sweep(f, op, rhs, rhs_dtype, x, x_dtype, M, ld, arith, s, st) != SB_OK) {
      clear_error();
      continue;
    }
    float ms_best = 1e30f;
    bool good = true;
    for (int rep = 0; rep < 3 && good; ++rep) {
      good = cudaEventRecord(e0, st) == cudaSuccess &&
             launch_sweep(f, op, rhs, rhs_dtype, x, x_dtype, M, ld, arith, s, st) == SB_OK &&
             cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      if (good && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) ms_best = std::min(ms_best, ms);
    }
    if (!good) {
      cudaGetLastError();
      clear_error();
      continue;
    }
    if (ms_best < winner_ms) {
      winner_ms = ms_best;
      winner = s;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (winner_ms >= 1e30f) return fail(SB_ERR_CUDA, "no candidate shape could be launched");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[make_key(f, arith, rhs_dtype, x_dtype)] = winner;
  }
  if (best) {
    best->threads = winner.threads;
    best->ctas_per_sm = winner.ctas_per_sm;
    best->systems_per_thread = winner.spt;
    best->algorithm = winner.algo;
  }
  if (best_ms) *best_ms = winner_ms;
  return SB_OK;
}

}  // extern "C"
