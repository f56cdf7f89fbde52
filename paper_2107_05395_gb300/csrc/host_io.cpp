// Solves of batches that live in host memory: the batch is cut into chunks of
// systems (column ranges of the interleaved layout); each chunk's host->device
// copy, solve and device->host copy go on one of kSlots internal streams, so the
// two copy directions and the solves of neighbouring chunks overlap.  The call is
// ordered after prior work on the caller's stream and the caller's stream waits
// for all of it; the host thread does not block.
#include <algorithm>
#include <mutex>

#include "host_layout.h"
#include "sb_internal.h"

namespace sb {
namespace {

constexpr int kSlots = kHostSlots;
constexpr int kMaxDev = 64;

struct DevStreams {
  cudaStream_t s[kSlots] = {nullptr, nullptr, nullptr};
  cudaEvent_t start = nullptr;
  cudaEvent_t done[kSlots] = {nullptr, nullptr, nullptr};
};
std::mutex g_mu;
DevStreams g_dev[kMaxDev];

int streams_for(int dev, DevStreams** out) {
  if (dev < 0 || dev >= kMaxDev) return fail(SB_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  DevStreams& d = g_dev[dev];
  if (d.s[0] == nullptr) {
    for (int k = 0; k < kSlots; ++k) {
      SB_CUDA(cudaStreamCreateWithFlags(&d.s[k], cudaStreamNonBlocking));
      SB_CUDA(cudaEventCreateWithFlags(&d.done[k], cudaEventDisableTiming));
    }
    SB_CUDA(cudaEventCreateWithFlags(&d.start, cudaEventDisableTiming));
  }
  *out = &d;
  return SB_OK;
}

size_t esize(sb_dtype t) { return t == SB_F64 ? 8 : (t == SB_F32 ? 4 : 0); }

// Chunk width: about eight chunks, but every copied row at least 128 KB wide
// (strided copies of narrower rows lose bandwidth on GB300's host link: 64 KB
// rows measured 131 GB/s against 208 GB/s for 128 KB rows), in whole 64-system
// tiles.
int64_t auto_chunk(int64_t M, size_t elem_bytes) {
  int64_t c = std::max<int64_t>((M + 7) / 8, (int64_t)(131072 / elem_bytes));
  c = ((c + 63) / 64) * 64;
  return std::max<int64_t>(1, std::min<int64_t>(c, M));
}

}  // namespace
}  // namespace sb

using namespace sb;

extern "C" {

int sb_host_workspace_bytes(const sb_factor* f, int64_t M, int64_t chunk_systems, sb_dtype rhs_dtype,
                            sb_dtype x_dtype, size_t* bytes) {
  clear_error();
  if (!f || !bytes) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  if (M < 0 || chunk_systems < 0) return fail(SB_ERR_INVALID_ARG, "bad sizes");
  if (esize(rhs_dtype) == 0 || esize(x_dtype) == 0) return fail(SB_ERR_INVALID_ARG, "unknown dtype");
  const int64_t c = chunk_systems > 0 ? std::min(chunk_systems, std::max<int64_t>(M, 1))
                                       : auto_chunk(std::max<int64_t>(M, 1), std::min(esize(rhs_dtype), esize(x_dtype)));
  *bytes = (size_t)kSlots * host_slot_bytes(f->N, c, esize(rhs_dtype), esize(x_dtype));
  return SB_OK;
}

int sb_solve_batched_host(const sb_factor* f, int transpose, const void* rhs_host, sb_dtype rhs_dtype,
                          void* x_host, sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith,
                          int64_t chunk_systems, void* work, size_t work_bytes, void* stream) {
  clear_error();
  if (!f) return fail(SB_ERR_INVALID_ARG, "factor handle is NULL");
  if (transpose != 0 && transpose != 1) return fail(SB_ERR_INVALID_ARG, "transpose must be 0 or 1");
  const size_t rs = esize(rhs_dtype), xs = esize(x_dtype);
  if (rs == 0 || xs == 0) return fail(SB_ERR_INVALID_ARG, "unknown dtype");
  if (M < 0 || ld < M || ld < 1) return fail(SB_ERR_INVALID_ARG, "need M >= 0 and ld >= max(M, 1)");
  if (M == 0) return SB_OK;
  if (!rhs_host || !x_host) return fail(SB_ERR_INVALID_ARG, "NULL host array");
  if (chunk_systems < 0) return fail(SB_ERR_INVALID_ARG, "chunk_systems must be >= 0");
  const int64_t C = chunk_systems > 0 ? std::min(chunk_systems, M) : auto_chunk(M, std::min(rs, xs));
  size_t need = 0;
  SB_TRY(sb_host_workspace_bytes(f, M, C, rhs_dtype, x_dtype, &need));
  if (!work || work_bytes < need)
    return fail(SB_ERR_INVALID_ARG, "the host-memory solve needs a device workspace of %zu bytes", need);
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  SB_TRY(check_device_range(work, need, 8, f->device, "work"));
  // host arrays: must not be device memory
  for (const void* p : {rhs_host, (const void*)x_host}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (a.type == cudaMemoryTypeDevice) return fail(SB_ERR_INVALID_ARG, "rhs_host / x_host must be host memory");
  }
  DevStreams* ds = nullptr;
  SB_TRY(streams_for(f->device, &ds));
  cudaStream_t caller = (cudaStream_t)stream;
  SB_CUDA(cudaEventRecord(ds->start, caller));
  for (int k = 0; k < kSlots; ++k) SB_CUDA(cudaStreamWaitEvent(ds->s[k], ds->start, 0));

  const int64_t N = f->N;
  const size_t slot = host_slot_bytes(N, C, rs, xs), x_off = host_slot_x_offset(N, C, rs);
  const Op op = transpose ? OP_ADJOINT : OP_PRIMAL;
  const SweepShape shape = shape_for(f, arith, rhs_dtype, x_dtype);
  int64_t chunk = 0;
  for (int64_t m0 = 0; m0 < M; m0 += C, ++chunk) {
    const int64_t Mc = std::min(C, M - m0);
    const int k = (int)(chunk % kSlots);
    cudaStream_t s = ds->s[k];
    char* base = static_cast<char*>(work) + (size_t)k * slot;
    void* d_rhs = base;
    void* d_x = base + x_off;
    SB_CUDA(cudaMemcpy2DAsync(d_rhs, (size_t)Mc * rs, static_cast<const char*>(rhs_host) + (size_t)m0 * rs,
                              (size_t)ld * rs, (size_t)Mc * rs, (size_t)N, cudaMemcpyHostToDevice, s));
    SB_TRY(launch_sweep(f, op, d_rhs, rhs_dtype, d_x, x_dtype, Mc, Mc, arith, shape, s));
    SB_CUDA(cudaMemcpy2DAsync(static_cast<char*>(x_host) + (size_t)m0 * xs, (size_t)ld * xs, d_x,
                              (size_t)Mc * xs, (size_t)Mc * xs, (size_t)N, cudaMemcpyDeviceToHost, s));
  }
  for (int k = 0; k < kSlots; ++k) {
    SB_CUDA(cudaEventRecord(ds->done[k], ds->s[k]));
    SB_CUDA(cudaStreamWaitEvent(caller, ds->done[k], 0));
  }
  return SB_OK;
}

}  // extern "C"
