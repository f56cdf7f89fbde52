// Host side of the sbsolve C ABI: errors, argument checks, the FP64 shared-matrix
// factorisations, and the device copy of their coefficients.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <mutex>
#include <new>

#include <cuda.h>

#include "partition.h"
#include "sb_internal.h"
#include "two_ended.h"

namespace sb {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SB_OK;
  cudaGetLastError();  // clear the sticky-free error state of the runtime
  return fail(e == cudaErrorMemoryAllocation ? SB_ERR_ALLOC : SB_ERR_CUDA, "%s failed: %s", what,
              cudaGetErrorString(e));
}

DeviceGuard::DeviceGuard(int device) {
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  if (device >= 0 && device != prev) rc = cuda_check(cudaSetDevice(device), "cudaSetDevice");
}

DeviceGuard::~DeviceGuard() {
  int cur = -1;
  if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

int sm_count(int device) {
  static std::mutex mu;
  static int cache[64] = {0};
  if (device < 0 || device >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[device] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cache[device] = v;
  }
  return cache[device];
}

// cuMemGetAddressRange, looked up through the runtime so that the library does
// not link the driver library directly (it then loads on machines without one).
typedef CUresult (*RangeFn)(CUdeviceptr*, size_t*, CUdeviceptr);
static RangeFn range_fn() {
  static RangeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<RangeFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

int check_device_range(const void* p, size_t bytes, size_t align, int device, const char* name) {
  if (p == nullptr) return fail(SB_ERR_INVALID_ARG, "%s is NULL", name);
  if (align > 1 && (reinterpret_cast<uintptr_t>(p) % align) != 0)
    return fail(SB_ERR_INVALID_ARG, "%s is not aligned to %zu bytes", name, align);
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SB_ERR_INVALID_ARG, "%s is not a pointer known to CUDA (%s)", name,
                cudaGetErrorString(e));
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(SB_ERR_INVALID_ARG, "%s must be device or managed memory (got a host pointer)",
                name);
  if (attr.type == cudaMemoryTypeDevice && attr.device != device)
    return fail(SB_ERR_INVALID_ARG, "%s lives on device %d, the factor on device %d", name,
                attr.device, device);
  if (attr.type == cudaMemoryTypeDevice && bytes > 0) {
    // The whole range [p, p + bytes) must lie inside one allocation.
    CUdeviceptr base = 0;
    size_t size = 0;
    RangeFn fn = range_fn();
    if (fn == nullptr) return fail(SB_ERR_CUDA, "cuMemGetAddressRange is unavailable");
    CUresult r = fn(&base, &size, reinterpret_cast<CUdeviceptr>(p));
    if (r != CUDA_SUCCESS)
      return fail(SB_ERR_INVALID_ARG, "%s: cannot query its allocation (CUresult %d)", name,
                  (int)r);
    uintptr_t lo = reinterpret_cast<uintptr_t>(p);
    if (lo + bytes > static_cast<uintptr_t>(base) + size)
      return fail(SB_ERR_INVALID_ARG,
                  "%s: %zu bytes from the pointer run past the end of its allocation "
                  "(%zu bytes left)",
                  name, bytes, (size_t)(static_cast<uintptr_t>(base) + size - lo));
  }
  return SB_OK;
}

int check_alias(const void* a, size_t abytes, const void* b, size_t bbytes, const char* na,
                const char* nb) {
  if (a == b || abytes == 0 || bbytes == 0) return SB_OK;
  uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  if (x < y + bbytes && y < x + abytes)
    return fail(SB_ERR_INVALID_ARG, "%s and %s overlap without being the same array", na, nb);
  return SB_OK;
}

// ------------------------------------------------------ factorisations (FP64)

static bool finite_all(const double* v, int64_t lo, int64_t hi) {
  for (int64_t i = lo; i < hi; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

// Section 3.1 / Algorithm 1: bh_0 = b_0, ch_0 = c_0/b_0, bh_i = b_i - a_i ch_{i-1},
// ch_i = c_i / bh_i.  Fills the primal and adjoint coefficient rows (P = 1).
static int factor_tri_host(int64_t N, const double* a, const double* b, const double* c,
                           std::vector<double>& coef) {
  std::vector<double> bh(N), ch(N, 0.0);
  for (int64_t i = 0; i < N; ++i) {
    bh[i] = (i == 0) ? b[0] : b[i] - a[i] * ch[i - 1];
    if (bh[i] == 0.0 || !std::isfinite(bh[i]))
      return fail(SB_ERR_SINGULAR, "zero or non-finite pivot at row %lld", (long long)i);
    if (i + 1 < N) ch[i] = c[i] / bh[i];
  }
  const int64_t W = 2;  // P + 1; rows prescaled by the reciprocal pivot
  coef.assign(2 * op_block_len(1, N), 0.0);
  double* pf = coef.data();  // primal forward  {1/bh_i, a_i/bh_i}
  double* pb = pf + W * N;   // primal backward {1, ch_i}
  double* af = pb + W * N;   // adjoint forward {1, ch_{i-1}}
  double* ab = af + W * N;   // adjoint backward {1/bh_i, a_{i+1}/bh_i}
  for (int64_t i = 0; i < N; ++i) {
    pf[W * i + 0] = 1.0 / bh[i];
    pf[W * i + 1] = (i > 0) ? a[i] / bh[i] : 0.0;
    pb[W * i + 0] = 1.0;
    pb[W * i + 1] = (i + 1 < N) ? ch[i] : 0.0;
    af[W * i + 0] = 1.0;
    af[W * i + 1] = (i > 0) ? ch[i - 1] : 0.0;
    ab[W * i + 0] = 1.0 / bh[i];
    ab[W * i + 1] = (i + 1 < N) ? a[i + 1] / bh[i] : 0.0;
  }
  return SB_OK;
}

// Section 4.1 (Algorithm 3 read with the section's equations), as one recurrence
// with out-of-range terms zero:
//   beta_i  = b_i - a_i gamma_{i-2};  alpha_i = c_i - a_i delta_{i-2} - beta_i gamma_{i-1}
//   gamma_i = (d_i - beta_i delta_{i-1}) / alpha_i;  delta_i = e_i / alpha_i;  eps_i = a_i
static int factor_penta_host(int64_t N, const double* a, const double* b, const double* c,
                             const double* d, const double* e, std::vector<double>& coef) {
  std::vector<double> al(N), be(N, 0.0), ga(N, 0.0), de(N, 0.0), ep(N, 0.0);
  auto G = [&](int64_t j) { return j >= 0 ? ga[j] : 0.0; };
  auto D = [&](int64_t j) { return j >= 0 ? de[j] : 0.0; };
  for (int64_t i = 0; i < N; ++i) {
    const double ai = (i >= 2) ? a[i] : 0.0;
    const double bi = (i >= 1) ? b[i] : 0.0;
    const double di = (i + 1 < N) ? d[i] : 0.0;
    const double ei = (i + 2 < N) ? e[i] : 0.0;
    be[i] = bi - ai * G(i - 2);
    al[i] = c[i] - ai * D(i - 2) - be[i] * G(i - 1);
    if (al[i] == 0.0 || !std::isfinite(al[i]))
      return fail(SB_ERR_SINGULAR, "zero or non-finite pivot at row %lld", (long long)i);
    ga[i] = (di - be[i] * D(i - 1)) / al[i];
    de[i] = ei / al[i];
    ep[i] = ai;
  }
  const int64_t W = 3;  // rows prescaled by the reciprocal pivot
  coef.assign(2 * op_block_len(2, N), 0.0);
  double* pf = coef.data();  // primal forward  {1/alpha_i, beta_i/alpha_i, eps_i/alpha_i}
  double* pb = pf + W * N;   // primal backward {1, gamma_i, delta_i}
  double* af = pb + W * N;   // adjoint forward {1, gamma_{i-1}, delta_{i-2}}
  double* ab = af + W * N;   // adjoint backward {1/alpha_i, beta_{i+1}/alpha_i, eps_{i+2}/alpha_i}
  for (int64_t i = 0; i < N; ++i) {
    pf[W * i + 0] = 1.0 / al[i];
    pf[W * i + 1] = be[i] / al[i];
    pf[W * i + 2] = ep[i] / al[i];
    pb[W * i + 0] = 1.0;
    pb[W * i + 1] = ga[i];
    pb[W * i + 2] = de[i];
    af[W * i + 0] = 1.0;
    af[W * i + 1] = (i >= 1) ? ga[i - 1] : 0.0;
    af[W * i + 2] = (i >= 2) ? de[i - 2] : 0.0;
    ab[W * i + 0] = 1.0 / al[i];
    ab[W * i + 1] = (i + 1 < N) ? be[i + 1] / al[i] : 0.0;
    ab[W * i + 2] = (i + 2 < N) ? ep[i + 2] / al[i] : 0.0;
  }
  return SB_OK;
}

static int upload_factor(sb_factor* f) {
  const size_t nc = f->h_coef.size(), nd = f->h_diag.size();
  SB_CUDA(cudaMalloc(&f->coef64, nc * sizeof(double)));
  SB_CUDA(cudaMalloc(&f->coef32, nc * sizeof(float)));
  SB_CUDA(cudaMalloc(&f->coefdf, 2 * nc * sizeof(float)));
  SB_CUDA(cudaMalloc(&f->diag64, nd * sizeof(double)));
  std::vector<float> c32(nc), cdf(2 * nc);
  for (size_t k = 0; k < nc; ++k) {
    const double v = f->h_coef[k];
    c32[k] = static_cast<float>(v);
    cdf[2 * k] = static_cast<float>(v);  // hi: v rounded to FP32
    cdf[2 * k + 1] = static_cast<float>(v - static_cast<double>(cdf[2 * k]));  // lo
  }
  SB_CUDA(cudaMemcpy(f->coefdf, cdf.data(), 2 * nc * sizeof(float), cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(f->coef64, f->h_coef.data(), nc * sizeof(double), cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(f->coef32, c32.data(), nc * sizeof(float), cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(f->diag64, f->h_diag.data(), nd * sizeof(double), cudaMemcpyHostToDevice));
  // row-major copy of A for residuals: arow[(2P+1)*i + k] = entry at offset k - P of row i
  const int64_t nb = 2 * f->P + 1, N = f->N;
  std::vector<double> arow((size_t)nb * N);
  std::vector<float> arowdf(2 * (size_t)nb * N);
  for (int64_t i = 0; i < N; ++i)
    for (int64_t k = 0; k < nb; ++k) {
      const double v = f->h_diag[(size_t)k * N + i];
      arow[(size_t)nb * i + k] = v;
      arowdf[2 * ((size_t)nb * i + k)] = (float)v;
      arowdf[2 * ((size_t)nb * i + k) + 1] = (float)(v - (double)(float)v);
    }
  SB_CUDA(cudaMalloc(&f->arow64, arow.size() * sizeof(double)));
  SB_CUDA(cudaMalloc(&f->arowdf, arowdf.size() * sizeof(float)));
  SB_CUDA(cudaMemcpy(f->arow64, arow.data(), arow.size() * sizeof(double), cudaMemcpyHostToDevice));
  SB_CUDA(cudaMemcpy(f->arowdf, arowdf.data(), arowdf.size() * sizeof(float), cudaMemcpyHostToDevice));
  // FP32 sweep rows of J A J (the rows and columns of A in reverse order) for the
  // refinement passes that eliminate from the bottom, stored at the index of the
  // row of A they act on (two_ended.h).  A zero pivot of J A J only disables them.
  if (!f->periodic) {
    std::vector<double> rfw, rbw;
    if (reversed_rows(f->P, (int)N, f->h_diag.data(), rfw, rbw)) {
      std::vector<float> rev(rfw.size() + rbw.size());
      for (size_t k = 0; k < rfw.size(); ++k) rev[k] = (float)rfw[k];
      for (size_t k = 0; k < rbw.size(); ++k) rev[rfw.size() + k] = (float)rbw[k];
      SB_CUDA(cudaMalloc(&f->coef32_rev, rev.size() * sizeof(float)));
      SB_CUDA(cudaMemcpy(f->coef32_rev, rev.data(), rev.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  // images of the partitioned solve of A and A^T (FP32) for each variant: chunks of
  // the shortest L that covers N (16/32/64 rows for 16 chunks, 8/16/32 for 32), N >= 64;
  // variant 2 holds variant 0's rows with each pair of chunks interleaved
  for (int v = 0; v < kPartVariants && !f->periodic; ++v) {
    const int P = part_chunks(v);
    int L = 0;
    const int lens[3] = {v == 1 ? 8 : 16, v == 1 ? 16 : 32, v == 1 ? 32 : 64};
    for (int cand : lens)
      if (L == 0 && (int64_t)cand * P >= N) L = cand;
    if (N < 64 || L == 0) continue;
    for (int o = 0; o < 2; ++o) {
      std::vector<double> dt;
      const double* d = f->h_diag.data();
      if (o == 1) {
        dt = transpose_diagonals(f->P, (int)N, d);
        d = dt.data();
      }
      Partition part;
      if (!build_partition(f->P, (int)N, d, L, P, part)) continue;  // a zero pivot
      const std::vector<double> img = v == 2 ? partition_image_paired(part) : partition_image(part);
      std::vector<float> img32(img.size());
      for (size_t k = 0; k < img.size(); ++k) img32[k] = (float)img[k];
      SB_CUDA(cudaMalloc(&f->part_img[o][v], img32.size() * sizeof(float)));
      SB_CUDA(cudaMemcpy(f->part_img[o][v], img32.data(), img32.size() * sizeof(float),
                         cudaMemcpyHostToDevice));
      f->part_L[v] = L;
      f->part_NL[v] = part.NL;
    }
  }
  // FP64 images (block-Thomas factors and cyclic-reduction matrices) of the
  // small-tile FP64 partitioned solve: kPart64Chunks
  // chunks of the shortest L in {8, 16, 32} that covers N, for N >= 32
  {
    int L64 = 0;
    for (int cand : {8, 16, 32})
      if (L64 == 0 && (int64_t)cand * kPart64Chunks >= N) L64 = cand;
    if (N >= 32 && L64 > 0 && !f->periodic) {
      for (int o = 0; o < 2; ++o) {
        std::vector<double> dt;
        const double* d = f->h_diag.data();
        if (o == 1) {
          dt = transpose_diagonals(f->P, (int)N, d);
          d = dt.data();
        }
        Partition part;
        if (!build_partition(f->P, (int)N, d, L64, kPart64Chunks, part)) continue;
        if (part.NL != kPart64Levels) continue;  // (cannot happen for 16 chunks)
        const std::vector<double> img = partition_image_thomas(part);
        SB_CUDA(cudaMalloc(&f->part64_img[o], img.size() * sizeof(double)));
        SB_CUDA(cudaMemcpy(f->part64_img[o], img.data(), img.size() * sizeof(double),
                           cudaMemcpyHostToDevice));
        f->part64_L = L64;
      }
    }
  }
  // FP64 images of the two-ended sweeps of A and A^T
  if (!f->periodic && N >= two_ended_min_n(f->P)) {
    for (int o = 0; o < 2; ++o) {
      std::vector<double> dt;
      const double* d = f->h_diag.data();
      if (o == 1) {
        dt = transpose_diagonals(f->P, (int)N, d);
        d = dt.data();
      }
      TwoEnded t;
      if (!build_two_ended(f->P, (int)N, d, t)) continue;
      const std::vector<double> img = two_ended_image(t);
      SB_CUDA(cudaMalloc(&f->two_img[o], img.size() * sizeof(double)));
      SB_CUDA(cudaMemcpy(f->two_img[o], img.data(), img.size() * sizeof(double), cudaMemcpyHostToDevice));
      f->two_s = t.s;
    }
  }
  return SB_OK;
}

static void free_factor(sb_factor* f) {
  if (!f) return;
  if (f->device >= 0) {
    DeviceGuard g(f->device);
    if (f->coef64) cudaFree(f->coef64);
    if (f->coef32) cudaFree(f->coef32);
    if (f->coefdf) cudaFree(f->coefdf);
    if (f->diag64) cudaFree(f->diag64);
    if (f->arow64) cudaFree(f->arow64);
    if (f->arowdf) cudaFree(f->arowdf);
    if (f->coef32_rev) cudaFree(f->coef32_rev);
    if (f->cyc64) cudaFree(f->cyc64);
    for (auto& per_op : f->part_img)
      for (float* p : per_op)
        if (p) cudaFree(p);
    for (double* p : f->part64_img)
      if (p) cudaFree(p);
    for (double* p : f->two_img)
      if (p) cudaFree(p);
  }
  delete f;
}

static int make_factor(int P, int64_t N, const double* const* diags, sb_factor** out,
                       bool periodic = false) {
  if (out == nullptr) return fail(SB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 1) return fail(SB_ERR_INVALID_ARG, "N must be >= 1 (got %lld)", (long long)N);
  if (N > (int64_t)1 << 28) return fail(SB_ERR_INVALID_ARG, "N too large (%lld)", (long long)N);
  const int nd = 2 * P + 1;
  for (int k = 0; k < nd; ++k) {
    if (diags[k] == nullptr) return fail(SB_ERR_INVALID_ARG, "diagonal %d is NULL", k);
    const int off = k - P;  // offset of this diagonal
    const int64_t lo = off < 0 ? -off : 0, hi = off > 0 ? N - off : N;
    if (hi > lo && !finite_all(diags[k], lo, hi))
      return fail(SB_ERR_INVALID_ARG, "diagonal at offset %d has a non-finite entry", off);
  }
  sb_factor* f = new (std::nothrow) sb_factor();
  if (!f) return fail(SB_ERR_ALLOC, "host allocation failed");
  f->P = P;
  f->N = N;
  f->periodic = periodic;
  int rc = (P == 1) ? factor_tri_host(N, diags[0], diags[1], diags[2], f->h_coef)
                    : factor_penta_host(N, diags[0], diags[1], diags[2], diags[3], diags[4],
                                        f->h_coef);
  if (rc != SB_OK) {
    delete f;
    return rc;
  }
  f->h_diag.assign((size_t)nd * N, 0.0);
  for (int k = 0; k < nd; ++k) {
    const int off = k - P;
    for (int64_t i = 0; i < N; ++i) {
      const int64_t j = i + off;
      f->h_diag[(size_t)k * N + i] = (j >= 0 && j < N) ? diags[k][i] : 0.0;
    }
  }
  if (cudaGetDevice(&f->device) != cudaSuccess) {
    cudaGetLastError();
    delete f;
    return fail(SB_ERR_CUDA, "no CUDA device is available");
  }
  rc = upload_factor(f);
  if (rc != SB_OK) {
    free_factor(f);
    return rc;
  }
  *out = f;
  return SB_OK;
}

// Square of a tridiagonal operator T given row-wise by (lo, mid, up):
// (T T)[i][i+o] = sum over k = i-1..i+1 of T[i][k] T[k][i+o], o = -2..2.
static void square_tridiagonal(int64_t N, const std::vector<double>& lo,
                               const std::vector<double>& mid, const std::vector<double>& up,
                               std::vector<double>& out /* 5*N, diagonal-major */) {
  auto T = [&](int64_t i, int64_t k) -> double {
    if (i < 0 || i >= N || k < 0 || k >= N) return 0.0;
    if (k == i) return mid[i];
    if (k == i - 1) return lo[i];
    if (k == i + 1) return up[i];
    return 0.0;
  };
  out.assign(5 * N, 0.0);
  for (int64_t i = 0; i < N; ++i)
    for (int o = -2; o <= 2; ++o) {
      const int64_t j = i + o;
      if (j < 0 || j >= N) continue;
      double s = 0.0;
      for (int64_t k = i - 1; k <= i + 1; ++k) s += T(i, k) * T(k, j);
      out[(o + 2) * N + i] = s;
    }
}

int build_matrix(int kind, int64_t N, double coef, std::vector<double>& diags, int* P) {
  if (N < 1) return fail(SB_ERR_INVALID_ARG, "N must be >= 1 (got %lld)", (long long)N);
  if (!std::isfinite(coef)) return fail(SB_ERR_INVALID_ARG, "coefficient is not finite");
  std::vector<double> lo(N, 1.0), mid(N, -2.0), up(N, 1.0), K;
  lo[0] = 0.0;
  up[N - 1] = 0.0;
  switch (kind) {
    case SB_MAT_DIFFUSION_DIRICHLET:
      *P = 1;
      diags.assign(3 * N, 0.0);
      for (int64_t i = 0; i < N; ++i) {
        diags[i] = (i > 0) ? -coef : 0.0;
        diags[N + i] = 1.0 + 2.0 * coef;
        diags[2 * N + i] = (i + 1 < N) ? -coef : 0.0;
      }
      return SB_OK;
    case SB_MAT_DIFFUSION_PERIODIC:
      if (N < 3) return fail(SB_ERR_INVALID_ARG, "the periodic matrix needs N >= 3");
      *P = 1;
      diags.assign(3 * N, -coef);  // the corners a[0], c[N-1] included
      for (int64_t i = 0; i < N; ++i) diags[N + i] = 1.0 + 2.0 * coef;
      return SB_OK;
    case SB_MAT_CH_PERIODIC: {
      if (N < 5) return fail(SB_ERR_INVALID_ARG, "the periodic matrix needs N >= 5");
      *P = 2;
      const double st[5] = {1.0, -4.0, 6.0, -4.0, 1.0};  // D2_P D2_P, wrapping around
      diags.assign(5 * N, 0.0);
      for (int k = 0; k < 5; ++k)
        for (int64_t i = 0; i < N; ++i) diags[k * N + i] = (k == 2 ? 1.0 : 0.0) + coef * st[k];
      return SB_OK;
    }
    case SB_MAT_HYPER_HINGED:
      square_tridiagonal(N, lo, mid, up, K);
      break;
    case SB_MAT_HYPER_TRUNCATED: {
      const double st[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
      K.assign(5 * N, 0.0);
      for (int o = -2; o <= 2; ++o)
        for (int64_t i = 0; i < N; ++i)
          if (i + o >= 0 && i + o < N) K[(o + 2) * N + i] = st[o + 2];
      break;
    }
    case SB_MAT_CH_NOFLUX:
      mid[0] += 1.0;      // ghost cell C_{-1} = C_0
      mid[N - 1] += 1.0;  // ghost cell C_N = C_{N-1}
      square_tridiagonal(N, lo, mid, up, K);
      break;
    default:
      return fail(SB_ERR_INVALID_ARG, "unknown matrix kind %d", kind);
  }
  *P = 2;
  diags.assign(5 * N, 0.0);
  for (int k = 0; k < 5; ++k)
    for (int64_t i = 0; i < N; ++i)
      diags[k * N + i] = (k == 2 ? 1.0 : 0.0) + coef * K[k * N + i];
  for (int k = 0; k < 5; ++k)  // exact zeros outside the matrix
    for (int64_t i = 0; i < N; ++i)
      if (i + (k - 2) < 0 || i + (k - 2) >= N) diags[k * N + i] = 0.0;
  return SB_OK;
}

static size_t dtype_size(sb_dtype t) { return t == SB_F64 ? 8 : (t == SB_F32 ? 4 : 0); }

// Common checks of a batched solve.
static int check_solve_args(const sb_factor* f, const void* rhs, sb_dtype rt, const void* x,
                            sb_dtype xt, int64_t M, int64_t ld) {
  if (f == nullptr) return fail(SB_ERR_INVALID_ARG, "factor handle is NULL");
  const size_t rs = dtype_size(rt), xs = dtype_size(xt);
  if (rs == 0) return fail(SB_ERR_INVALID_ARG, "unknown rhs dtype %d", (int)rt);
  if (xs == 0) return fail(SB_ERR_INVALID_ARG, "unknown x dtype %d", (int)xt);
  if (M < 0) return fail(SB_ERR_INVALID_ARG, "M must be >= 0 (got %lld)", (long long)M);
  if (ld < M || ld < 1)
    return fail(SB_ERR_INVALID_ARG, "ld must be >= max(M, 1) (got ld=%lld, M=%lld)",
                (long long)ld, (long long)M);
  if (ld > ((int64_t)1 << 40) / f->N) return fail(SB_ERR_INVALID_ARG, "N*ld too large");
  if (M == 0) return SB_OK;
  const size_t elems = (size_t)((f->N - 1) * ld + M);
  SB_TRY(check_device_range(rhs, elems * rs, rs, f->device, "rhs"));
  SB_TRY(check_device_range(x, elems * xs, xs, f->device, "x"));
  if (rhs == x && rt != xt)
    return fail(SB_ERR_INVALID_ARG, "x may alias rhs only when both have the same dtype");
  SB_TRY(check_alias(rhs, elems * rs, x, elems * xs, "rhs", "x"));
  return SB_OK;
}

static int solve_common(const sb_factor* f, Op op, const void* rhs, sb_dtype rt, void* x,
                        sb_dtype xt, int64_t M, int64_t ld, sb_arith arith, void* stream) {
  if (f == nullptr) return fail(SB_ERR_INVALID_ARG, "factor handle is NULL");
  if (arith != SB_ARITH_NATIVE && arith != SB_ARITH_DF32)
    return fail(SB_ERR_INVALID_ARG, "unknown arithmetic mode %d", (int)arith);
  DeviceGuard g(f->device);
  SB_TRY(g.rc);
  SB_TRY(check_solve_args(f, rhs, rt, x, xt, M, ld));
  if (M == 0) return SB_OK;
  return launch_sweep(f, op, rhs, rt, x, xt, M, ld, arith, shape_for(f, arith, rt, xt),
                      (cudaStream_t)stream);
}

}  // namespace sb

using namespace sb;

extern "C" {

int sb_factor_shared_tri(int64_t N, const double* a, const double* b, const double* c,
                         sb_factor** out) {
  clear_error();
  const double* d[3] = {a, b, c};
  return make_factor(1, N, d, out);
}

// Plain Thomas solve of the tridiagonal (a, b, c) (a[0], c[N-1] unused), or of its
// transpose, for the periodic correction vectors (host, FP64, once per factor).
static bool thomas_host(const std::vector<double>& a, const std::vector<double>& b,
                        const std::vector<double>& c, std::vector<double> r, bool transpose,
                        std::vector<double>& x) {
  const int64_t N = (int64_t)b.size();
  std::vector<double> lo(N, 0.0), up(N, 0.0);  // sub- and super-diagonal of the solved matrix
  for (int64_t i = 0; i < N; ++i) {
    lo[i] = transpose ? (i > 0 ? c[i - 1] : 0.0) : (i > 0 ? a[i] : 0.0);
    up[i] = transpose ? (i + 1 < N ? a[i + 1] : 0.0) : (i + 1 < N ? c[i] : 0.0);
  }
  std::vector<double> cp(N, 0.0);
  for (int64_t i = 0; i < N; ++i) {
    const double piv = b[i] - (i > 0 ? lo[i] * cp[i - 1] : 0.0);
    if (piv == 0.0 || !std::isfinite(piv)) return false;
    cp[i] = up[i] / piv;
    r[i] = (r[i] - (i > 0 ? lo[i] * r[i - 1] : 0.0)) / piv;
  }
  x.assign(N, 0.0);
  for (int64_t i = N - 1; i >= 0; --i) x[i] = r[i] - (i + 1 < N ? cp[i] * x[i + 1] : 0.0);
  return true;
}

int sb_factor_shared_tri_periodic(int64_t N, const double* a, const double* b, const double* c,
                                  sb_factor** out) {
  clear_error();
  if (out == nullptr) return fail(SB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 3) return fail(SB_ERR_INVALID_ARG, "a periodic tridiagonal matrix needs N >= 3 (got %lld)",
                         (long long)N);
  if (!a || !b || !c) return fail(SB_ERR_INVALID_ARG, "a diagonal is NULL");
  if (!finite_all(a, 0, N) || !finite_all(b, 0, N) || !finite_all(c, 0, N))
    return fail(SB_ERR_INVALID_ARG, "a diagonal has a non-finite entry");
  if (b[0] == 0.0) return fail(SB_ERR_SINGULAR, "b[0] = 0: the rank-one split of section 3.3 needs b[0] != 0");
  // A = A' + u v^T, u = (-b_0, 0.., c_{N-1}), v = (1, 0.., -a_0/b_0)  (section 3.3)
  std::vector<double> ap(a, a + N), bp(b, b + N), cp(c, c + N), u(N, 0.0), v(N, 0.0);
  u[0] = -b[0];
  u[N - 1] = c[N - 1];
  v[0] = 1.0;
  v[N - 1] = -a[0] / b[0];
  ap[0] = 0.0;
  cp[N - 1] = 0.0;
  bp[0] = b[0] - u[0] * v[0];
  bp[N - 1] = b[N - 1] - u[N - 1] * v[N - 1];
  const double* d[3] = {ap.data(), bp.data(), cp.data()};
  sb_factor* f = nullptr;
  SB_TRY(make_factor(1, N, d, &f, true));
  f->periodic_rank = 1;
  // correction data, per op: rows (w_i, -z_i), alpha, beta (see sb_factor)
  std::vector<double> e0(N, 0.0), z, w, zt, wt;
  e0[0] = 1.0;
  bool ok = thomas_host(ap, bp, cp, u, false, z) && thomas_host(ap, bp, cp, e0, true, w) &&
            thomas_host(ap, bp, cp, v, true, zt) && thomas_host(ap, bp, cp, e0, false, wt);
  double vz = 0.0, uzt = 0.0;
  for (int64_t i = 0; ok && i < N; ++i) {
    vz += v[i] * z[i];
    uzt += u[i] * zt[i];
  }
  if (!ok || 1.0 + vz == 0.0 || 1.0 + uzt == 0.0 || !std::isfinite(vz) || !std::isfinite(uzt)) {
    sb_factor_destroy(f);
    return fail(SB_ERR_SINGULAR, "the periodic matrix is singular (1 + v.A'^{-1}u = 0)");
  }
  // primal: f = (v.y)/(1 + v.z), v.y = y_0 + v_{N-1} y_{N-1}
  f->cyc_alpha[0] = v[N - 1];
  f->cyc_beta[0] = 1.0 / (1.0 + vz);
  // adjoint: f = (u.y)/(1 + u.z'), u.y = u_0 (y_0 + (u_{N-1}/u_0) y_{N-1})
  f->cyc_alpha[1] = u[N - 1] / u[0];
  f->cyc_beta[1] = u[0] / (1.0 + uzt);
  std::vector<double> h(4 * N);
  for (int64_t i = 0; i < N; ++i) {
    h[2 * i] = w[i];
    h[2 * i + 1] = -z[i];
    h[2 * N + 2 * i] = wt[i];
    h[2 * N + 2 * i + 1] = -zt[i];
  }
  std::vector<float> h32(4 * N), hdf(8 * N);
  for (int64_t k = 0; k < 4 * N; ++k) {
    h32[k] = (float)h[k];
    hdf[2 * k] = (float)h[k];
    hdf[2 * k + 1] = (float)(h[k] - (double)hdf[2 * k]);
  }
  int rc = SB_OK;
  {
    DeviceGuard g(f->device);
    rc = g.rc;
    void* mem = nullptr;
    if (rc == SB_OK) rc = cuda_check(cudaMalloc(&mem, 4 * N * 8 + 4 * N * 4 + 8 * N * 4), "cudaMalloc");
    if (rc == SB_OK) {
      f->cyc64 = static_cast<double*>(mem);
      f->cyc32 = reinterpret_cast<float*>(f->cyc64 + 4 * N);
      f->cycdf = f->cyc32 + 4 * N;
      rc = cuda_check(cudaMemcpy(f->cyc64, h.data(), 4 * N * 8, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    if (rc == SB_OK)
      rc = cuda_check(cudaMemcpy(f->cyc32, h32.data(), 4 * N * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (rc == SB_OK)
      rc = cuda_check(cudaMemcpy(f->cycdf, hdf.data(), 8 * N * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  }
  if (rc != SB_OK) {
    sb_factor_destroy(f);
    return rc;
  }
  *out = f;
  return SB_OK;
}

// Solve of a pentadiagonal matrix given diagonal-major (5 N values, offsets -2..2),
// by the section 4.1 recurrence (host, FP64, for the periodic correction vectors).
static bool penta_solve_host(int64_t N, const std::vector<double>& dg, std::vector<double> r,
                             std::vector<double>& x) {
  auto D = [&](int k, int64_t i) { return dg[(size_t)k * N + i]; };
  std::vector<double> al(N), be(N), ga(N, 0.0), de(N, 0.0), ep(N);
  for (int64_t i = 0; i < N; ++i) {
    const double ai = i >= 2 ? D(0, i) : 0.0, bi = i >= 1 ? D(1, i) : 0.0;
    const double di = i + 1 < N ? D(3, i) : 0.0, ei = i + 2 < N ? D(4, i) : 0.0;
    be[i] = bi - ai * (i >= 2 ? ga[i - 2] : 0.0);
    al[i] = D(2, i) - ai * (i >= 2 ? de[i - 2] : 0.0) - be[i] * (i >= 1 ? ga[i - 1] : 0.0);
    if (al[i] == 0.0 || !std::isfinite(al[i])) return false;
    ga[i] = (di - be[i] * (i >= 1 ? de[i - 1] : 0.0)) / al[i];
    de[i] = ei / al[i];
    ep[i] = ai;
  }
  for (int64_t i = 0; i < N; ++i)
    r[i] = (r[i] - (i >= 1 ? be[i] * r[i - 1] : 0.0) - (i >= 2 ? ep[i] * r[i - 2] : 0.0)) / al[i];
  x.assign(N, 0.0);
  for (int64_t i = N - 1; i >= 0; --i)
    x[i] = r[i] - (i + 1 < N ? ga[i] * x[i + 1] : 0.0) - (i + 2 < N ? de[i] * x[i + 2] : 0.0);
  return true;
}

int sb_factor_shared_penta_periodic(int64_t N, const double* a, const double* b, const double* c,
                                    const double* d, const double* e, sb_factor** out) {
  clear_error();
  if (out == nullptr) return fail(SB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (N < 5)
    return fail(SB_ERR_INVALID_ARG, "a cyclic pentadiagonal matrix needs N >= 5 (got %lld)", (long long)N);
  const double* in[5] = {a, b, c, d, e};
  for (int k = 0; k < 5; ++k) {
    if (!in[k]) return fail(SB_ERR_INVALID_ARG, "diagonal %d is NULL", k);
    if (!finite_all(in[k], 0, N)) return fail(SB_ERR_INVALID_ARG, "diagonal %d has a non-finite entry", k);
  }
  // corner blocks (row-major 2 x 2): TL rows/cols 0,1; TR rows 0,1 x cols N-2,N-1;
  // BL rows N-2,N-1 x cols 0,1
  const double TL[4] = {c[0], d[0], b[1], c[1]};
  const double TR[4] = {a[0], b[0], 0.0, a[1]};
  const double BL[4] = {e[N - 2], 0.0, d[N - 1], e[N - 1]};
  // X = -TL, W = X^{-1} TR; U = [X; 0; BL], V = [I; 0; W^T] (rank 2)
  const double X[4] = {-TL[0], -TL[1], -TL[2], -TL[3]};
  const double detX = X[0] * X[3] - X[1] * X[2];
  if (detX == 0.0 || !std::isfinite(detX))
    return fail(SB_ERR_SINGULAR, "the top-left 2 x 2 block is singular: the rank-2 split needs it invertible");
  const double Xi[4] = {X[3] / detX, -X[1] / detX, -X[2] / detX, X[0] / detX};
  double W[4], BW[4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) W[2 * i + j] = Xi[2 * i] * TR[j] + Xi[2 * i + 1] * TR[2 + j];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) BW[2 * i + j] = BL[2 * i] * W[j] + BL[2 * i + 1] * W[2 + j];
  // A' = A - U V^T: corners removed, top-left block 2 TL, bottom-right block BR - BL W
  std::vector<double> dg((size_t)5 * N);
  for (int k = 0; k < 5; ++k)
    for (int64_t i = 0; i < N; ++i) {
      const int64_t j = i + (k - 2);
      dg[(size_t)k * N + i] = (j >= 0 && j < N) ? in[k][i] : 0.0;
    }
  auto at = [&](int off, int64_t i) -> double& { return dg[(size_t)(off + 2) * N + i]; };
  at(0, 0) = 2.0 * c[0];
  at(1, 0) = 2.0 * d[0];
  at(-1, 1) = 2.0 * b[1];
  at(0, 1) = 2.0 * c[1];
  at(0, N - 2) -= BW[0];
  at(1, N - 2) -= BW[1];
  at(-1, N - 1) -= BW[2];
  at(0, N - 1) -= BW[3];
  const double* dp[5] = {&dg[0], &dg[N], &dg[2 * N], &dg[3 * N], &dg[4 * N]};
  sb_factor* f = nullptr;
  SB_TRY(make_factor(2, N, dp, &f, true));
  f->periodic_rank = 2;
  // U and V as N x 2 (column-major vectors)
  std::vector<double> U0(N, 0.0), U1(N, 0.0), V0(N, 0.0), V1(N, 0.0), e0(N, 0.0), e1(N, 0.0);
  U0[0] = X[0]; U1[0] = X[1]; U0[1] = X[2]; U1[1] = X[3];
  U0[N - 2] = BL[0]; U1[N - 2] = BL[1]; U0[N - 1] = BL[2]; U1[N - 1] = BL[3];
  V0[0] = 1.0; V1[1] = 1.0;
  // V[N-2:N, :] = W^T: V_k[N-2+r] = W[k][r]
  V0[N - 2] = W[0]; V1[N - 2] = W[2]; V0[N - 1] = W[1]; V1[N - 1] = W[3];
  e0[0] = 1.0;
  e1[1] = 1.0;
  const std::vector<double> dgT = transpose_diagonals(2, (int)N, dg.data());
  std::vector<double> z0, z1, w0, w1, zt0, zt1, wt0, wt1;
  const bool ok = penta_solve_host(N, dg, U0, z0) && penta_solve_host(N, dg, U1, z1) &&
                  penta_solve_host(N, dgT, e0, w0) && penta_solve_host(N, dgT, e1, w1) &&
                  penta_solve_host(N, dgT, V0, zt0) && penta_solve_host(N, dgT, V1, zt1) &&
                  penta_solve_host(N, dg, e0, wt0) && penta_solve_host(N, dg, e1, wt1);
  // per op: rows (w0, w1, -z0, -z1) and 12 scalars P (2x2), Q (2x2), S^{-1} (2x2) with
  // g = S^{-1} (P (y_0, y_1) + Q (y_{N-2}, y_{N-1})), x = y - z0 g_0 - z1 g_1
  auto dot = [&](const std::vector<double>& p, const std::vector<double>& q) {
    double t = 0.0;
    for (int64_t i = 0; i < N; ++i) t += p[i] * q[i];
    return t;
  };
  double S[4], St[4];
  if (ok) {
    S[0] = 1.0 + dot(V0, z0); S[1] = dot(V0, z1); S[2] = dot(V1, z0); S[3] = 1.0 + dot(V1, z1);
    St[0] = 1.0 + dot(U0, zt0); St[1] = dot(U0, zt1); St[2] = dot(U1, zt0); St[3] = 1.0 + dot(U1, zt1);
  }
  const double dS = ok ? S[0] * S[3] - S[1] * S[2] : 0.0, dSt = ok ? St[0] * St[3] - St[1] * St[2] : 0.0;
  if (!ok || dS == 0.0 || dSt == 0.0 || !std::isfinite(dS) || !std::isfinite(dSt)) {
    sb_factor_destroy(f);
    return fail(SB_ERR_SINGULAR, "the cyclic matrix is singular (I + V^T A'^{-1} U)");
  }
  const size_t per_op = 4 * (size_t)N + 12;
  std::vector<double> h(2 * per_op, 0.0);
  auto fill = [&](double* o, const std::vector<double>& wa, const std::vector<double>& wb,
                  const std::vector<double>& za, const std::vector<double>& zb, const double* P,
                  const double* Q, const double* Sm, double det) {
    for (int64_t i = 0; i < N; ++i) {
      o[4 * i] = wa[i];
      o[4 * i + 1] = wb[i];
      o[4 * i + 2] = -za[i];
      o[4 * i + 3] = -zb[i];
    }
    double* sc = o + 4 * N;
    for (int k = 0; k < 4; ++k) {
      sc[k] = P[k];
      sc[4 + k] = Q[k];
    }
    sc[8] = Sm[3] / det;
    sc[9] = -Sm[1] / det;
    sc[10] = -Sm[2] / det;
    sc[11] = Sm[0] / det;
  };
  // primal: V^T y = (y_0, y_1) + W (y_{N-2}, y_{N-1})
  const double Ip[4] = {1.0, 0.0, 0.0, 1.0};
  fill(h.data(), w0, w1, z0, z1, Ip, W, S, dS);
  // adjoint: U^T y = X^T (y_0, y_1) + BL^T (y_{N-2}, y_{N-1})
  const double XT[4] = {X[0], X[2], X[1], X[3]}, BLT[4] = {BL[0], BL[2], BL[1], BL[3]};
  fill(h.data() + per_op, wt0, wt1, zt0, zt1, XT, BLT, St, dSt);
  std::vector<float> h32(h.size()), hdf(2 * h.size());
  for (size_t k = 0; k < h.size(); ++k) {
    h32[k] = (float)h[k];
    hdf[2 * k] = (float)h[k];
    hdf[2 * k + 1] = (float)(h[k] - (double)hdf[2 * k]);
  }
  int rc = SB_OK;
  {
    DeviceGuard g(f->device);
    rc = g.rc;
    void* mem = nullptr;
    const size_t n = h.size();
    if (rc == SB_OK) rc = cuda_check(cudaMalloc(&mem, n * 8 + n * 4 + 2 * n * 4), "cudaMalloc");
    if (rc == SB_OK) {
      f->cyc64 = static_cast<double*>(mem);
      f->cyc32 = reinterpret_cast<float*>(f->cyc64 + n);
      f->cycdf = f->cyc32 + n;
      rc = cuda_check(cudaMemcpy(f->cyc64, h.data(), n * 8, cudaMemcpyHostToDevice), "cudaMemcpy");
    }
    if (rc == SB_OK) rc = cuda_check(cudaMemcpy(f->cyc32, h32.data(), n * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (rc == SB_OK) rc = cuda_check(cudaMemcpy(f->cycdf, hdf.data(), 2 * n * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  }
  if (rc != SB_OK) {
    sb_factor_destroy(f);
    return rc;
  }
  *out = f;
  return SB_OK;
}

int sb_factor_shared_penta(int64_t N, const double* a, const double* b, const double* c,
                           const double* d, const double* e, sb_factor** out) {
  clear_error();
  const double* g[5] = {a, b, c, d, e};
  return make_factor(2, N, g, out);
}

void sb_factor_destroy(sb_factor* f) { free_factor(f); }

int sb_factor_info(const sb_factor* f, int* half_bandwidth, int64_t* N) {
  clear_error();
  if (!f || !half_bandwidth || !N) return fail(SB_ERR_INVALID_ARG, "NULL argument");
  *half_bandwidth = f->P;
  *N = f->N;
  return SB_OK;
}

int sb_solve_batched(const sb_factor* f, const void* rhs, void* x, int64_t M, int64_t ld,
                     sb_dtype dtype, void* stream) {
  clear_error();
  return solve_common(f, OP_PRIMAL, rhs, dtype, x, dtype, M, ld, SB_ARITH_NATIVE, stream);
}

int sb_solve_batched_adjoint(const sb_factor* f, const void* rhs, void* x, int64_t M,
                             int64_t ld, sb_dtype dtype, void* stream) {
  clear_error();
  return solve_common(f, OP_ADJOINT, rhs, dtype, x, dtype, M, ld, SB_ARITH_NATIVE, stream);
}

int sb_solve_batched_ex(const sb_factor* f, int transpose, const void* rhs, sb_dtype rhs_dtype,
                        void* x, sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith,
                        void* stream) {
  clear_error();
  if (transpose != 0 && transpose != 1)
    return fail(SB_ERR_INVALID_ARG, "transpose must be 0 or 1");
  return solve_common(f, transpose ? OP_ADJOINT : OP_PRIMAL, rhs, rhs_dtype, x, x_dtype, M, ld,
                      arith, stream);
}

int sb_build_matrix(int kind, int64_t N, double coef, double* diags) {
  clear_error();
  if (diags == nullptr) return fail(SB_ERR_INVALID_ARG, "diags is NULL");
  std::vector<double> v;
  int P = 0;
  SB_TRY(build_matrix(kind, N, coef, v, &P));
  std::memcpy(diags, v.data(), v.size() * sizeof(double));
  return SB_OK;
}

int sb_device_timeouts(int device, unsigned* count) {
  clear_error();
  if (count == nullptr) return fail(SB_ERR_INVALID_ARG, "count is NULL");
  return partition_timeouts(device, count);
}

const char* sb_last_error(void) { return g_last_error.c_str(); }

const char* sb_version(void) { return "sbsolve 0.1 (sm_103a)"; }

}  // extern "C"
