// Partitioned batched solve in FP64 for latency-bound batches (SB_ALGO_PARTITIONED
// with 128-thread CTAs; the math is in partition.h).
//
// A small batch (say 1024 systems of 256 unknowns) gives the sequential sweeps one
// warp per 32 systems: a few dozen SMs, each walking 2N dependent rows.  Here a
// 128-thread CTA takes a tile of only 8 systems and cuts its rows into 16 chunks of
// L rows, so the same batch spreads over 128 CTAs and every thread walks 2L rows:
//   - lane l of warp w owns system l % 8 of the tile and chunk 4w + l / 8, and loads
//     its chunk's rows straight into registers (8 lanes read one 64 B row segment);
//   - each chunk is swept forward and back with its own factors (y_c = A_c^{-1} b_c);
//   - the chunk heads and tails go to shared memory and the block-tridiagonal
//     boundary system is solved either by block Thomas, 8 threads (one per system)
//     walking the 15 boundaries (the least FP64 work; factors E, H, J from A alone),
//     or, when every CTA has a single tile so the solve is latency-bound, by cyclic
//     reduction with all 128 threads: 16 lanes per system, lane k holding boundary
//     k, four levels with warp shuffles (matrices T0, M from A alone);
//   - every thread corrects its rows, x_c = y_c - W_c lam_c - V_c rho_c, and stores
//     them.
// The partition image is staged into shared memory once per CTA; CTAs are
// persistent over the tiles.  There are no waits other than block barriers.
#include <algorithm>

#include "partition.h"
#include "sb_internal.h"
#include "sweep_tile.cuh"

namespace sb {
namespace {

constexpr int kPS = 8;                // systems per tile
constexpr int kWarps = 4;
constexpr int kChunks = kWarps * 4;   // four chunks per warp
constexpr int kThreads = kWarps * 32;

template <typename T, int n>
struct alignas(sizeof(T) * n) Row {
  T v[n];
};

constexpr int kLevels = kPart64Levels;  // cyclic-reduction levels for kChunks - 1 boundaries
static_assert(kChunks == kPart64Chunks && (1 << kLevels) >= kChunks - 1 && (1 << (kLevels - 1)) < kChunks - 1,
              "the image's chunk and level counts must match the kernel's");

template <int PB, int L>
__global__ void __launch_bounds__(kThreads)
part64_kernel(const double* __restrict__ image, PartLayoutT lay, int N, int64_t M, int64_t ld,
              const double* rhs, double* x, int64_t ntiles, bool pcr) {
  constexpr int Q = 2 * PB, FW = PB == 2 ? 4 : 2, K = kChunks - 1;
  using RF = Row<double, FW>;
  using RB = Row<double, PB>;
  using RC = Row<double, Q>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* img = reinterpret_cast<double*>(smem_raw);
  double* tips = img + lay.total;         // [kChunks][Q][kPS]: heads then tails
  double* zb = tips + kChunks * Q * kPS;  // [K][Q][kPS]: q_k, then z_k
  {
    const double2* s2 = reinterpret_cast<const double2*>(image);
    double2* d2 = reinterpret_cast<double2*>(img);
    for (int k = threadIdx.x; k < lay.total / 2; k += kThreads) d2[k] = s2[k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int s = lane & (kPS - 1);
  const int c = (threadIdx.x >> 5) * 4 + (lane >> 3);
  const int r0 = c * L;
  const bool full_chunk = r0 + L <= N;
  const RF* fw = reinterpret_cast<const RF*>(img + lay.fwd) + r0;
  const RB* bw = reinterpret_cast<const RB*>(img + lay.bwd) + r0;
  const RC* cw = reinterpret_cast<const RC*>(img + lay.cor) + r0;
  const double* E = img + lay.E;
  const double* Hm = img + lay.H;
  const double* J = img + lay.J;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t m = tile * kPS + s;
    const bool act = m < M;
    double y[L];
    {
      const double* src = rhs + (int64_t)r0 * ld + m;
      if (act && full_chunk) {
#pragma unroll
        for (int j = 0; j < L; ++j) y[j] = ld_stream(src + (int64_t)j * ld);
      } else {
#pragma unroll
        for (int j = 0; j < L; ++j) y[j] = (act && r0 + j < N) ? ld_stream(src + (int64_t)j * ld) : 0.0;
      }
    }
    // chunk sweeps (padding rows are identity rows with a zero right-hand side)
    {
      double u1 = 0.0, u2 = 0.0;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const RF f = fw[j];
        double t = y[j] * f.v[0];
        if constexpr (PB == 2) t = fma(-f.v[2], u2, t);
        const double u = fma(-f.v[1], u1, t);
        y[j] = u;
        u2 = u1;
        u1 = u;
      }
      double x1 = 0.0, x2 = 0.0;
#pragma unroll
      for (int j = L - 1; j >= 0; --j) {
        const RB b = bw[j];
        double t = y[j];
        if constexpr (PB == 2) t = fma(-b.v[1], x2, t);
        const double v = fma(-b.v[0], x1, t);
        y[j] = v;
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      tips[(c * Q + u) * kPS + s] = y[u];                 // head of chunk c
      tips[(c * Q + PB + u) * kPS + s] = y[L - PB + u];  // tail of chunk c
    }
    __syncthreads();
    if (pcr) {
      // boundary system by cyclic reduction: lanes 16 ss .. 16 ss + 15 serve system
      // ss, lane k boundary k (slot 15 holds none)
      const int ss = threadIdx.x >> 4, k = threadIdx.x & 15;
      double d[Q];
      {
        double r[Q];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          r[u] = k < K ? tips[(k * Q + PB + u) * kPS + ss] : 0.0;         // tail of chunk k
          r[PB + u] = k < K ? tips[((k + 1) * Q + u) * kPS + ss] : 0.0;   // head of chunk k+1
        }
        const double* T0 = img + lay.T0 + k;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          double t = 0.0;
#pragma unroll
          for (int j = 0; j < Q; ++j) t = fma(T0[(i * Q + j) * kChunks], r[j], t);
          d[i] = t;
        }
      }
      const double* Mb = img + lay.M + k;
#pragma unroll
      for (int l = 0; l < kLevels; ++l) {
        const int st = 1 << l;
        double dl[PB], dr[PB];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          dl[u] = __shfl_up_sync(0xffffffffu, d[u], st, 16);
          dr[u] = __shfl_down_sync(0xffffffffu, d[PB + u], st, 16);
        }
        const bool has_l = k >= st, has_r = k + st < K;
        const double* M0 = Mb;
        const double* M1 = Mb + Q * Q * kChunks;
        const double* M2 = M1 + Q * PB * kChunks;
        double nd[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          double t = 0.0;
#pragma unroll
          for (int j = 0; j < Q; ++j) t = fma(M0[(i * Q + j) * kChunks], d[j], t);
#pragma unroll
          for (int j = 0; j < PB; ++j) {
            if (has_l) t = fma(-M1[(i * PB + j) * kChunks], dl[j], t);
            if (has_r) t = fma(-M2[(i * PB + j) * kChunks], dr[j], t);
          }
          nd[i] = t;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = nd[i];
        Mb += (Q * Q + 2 * Q * PB) * kChunks;
      }
      if (k < K) {
#pragma unroll
        for (int i = 0; i < Q; ++i) zb[(k * Q + i) * kPS + ss] = d[i];
      }
    } else if (threadIdx.x < kPS) {
      // boundary system by block Thomas, one thread per system
      const int ss = threadIdx.x;
      double qp[Q];
#pragma unroll
      for (int t = 0; t < Q; ++t) qp[t] = 0.0;
      for (int k = 0; k < K; ++k) {  // q_k = r_k - E_k q_{k-1}
        double q[Q];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          q[u] = tips[(k * Q + PB + u) * kPS + ss];
          q[PB + u] = tips[((k + 1) * Q + u) * kPS + ss];
        }
#pragma unroll
        for (int u = 0; u < PB; ++u)
#pragma unroll
          for (int t = 0; t < Q; ++t) q[u] = fma(-E[(k * PB + u) * Q + t], qp[t], q[u]);
#pragma unroll
        for (int u = 0; u < Q; ++u) {
          zb[(k * Q + u) * kPS + ss] = q[u];
          qp[u] = q[u];
        }
      }
      double zn[PB];
#pragma unroll
      for (int u = 0; u < PB; ++u) zn[u] = 0.0;
      for (int k = K - 1; k >= 0; --k) {  // z_k = H_k q_k - J_k z_{k+1}[PB:Q]
        double q[Q], z[Q];
#pragma unroll
        for (int u = 0; u < Q; ++u) q[u] = zb[(k * Q + u) * kPS + ss];
#pragma unroll
        for (int u = 0; u < Q; ++u) {
          double t = 0.0;
#pragma unroll
          for (int v = 0; v < Q; ++v) t = fma(Hm[(k * Q + u) * Q + v], q[v], t);
#pragma unroll
          for (int v = 0; v < PB; ++v) t = fma(-J[(k * Q + u) * PB + v], zn[v], t);
          z[u] = t;
        }
#pragma unroll
        for (int u = 0; u < Q; ++u) zb[(k * Q + u) * kPS + ss] = z[u];
#pragma unroll
        for (int u = 0; u < PB; ++u) zn[u] = z[PB + u];
      }
    }
    __syncthreads();
    // correction x_j = y_j - W_j lam - V_j rho
    {
      double lam[PB], rho[PB];
#pragma unroll
      for (int u = 0; u < PB; ++u) {
        lam[u] = c > 0 ? zb[((c - 1) * Q + u) * kPS + s] : 0.0;
        rho[u] = c < K ? zb[(c * Q + PB + u) * kPS + s] : 0.0;
      }
      double* dst = x + (int64_t)r0 * ld + m;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const RC w = cw[j];
        double v = y[j];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          v = fma(-w.v[u], lam[u], v);
          v = fma(-w.v[PB + u], rho[u], v);
        }
        if (act && (full_chunk || r0 + j < N)) st_stream(dst + (int64_t)j * ld, v);
      }
    }
    // No barrier here: the next tile writes `tips` only after every thread has
    // passed this tile's second barrier (so block Thomas has read them), and `zb`
    // only after its own first barrier (so every correction has read it).
  }
}

template <int PB, int L>
int launch(const sb_factor* f, const double* image, const void* rhs, void* x, int64_t M, int64_t ld,
           const SweepShape& shape, cudaStream_t stream) {
  const PartLayoutT lay = part_layout_thomas(PB, L, kChunks, kLevels);
  constexpr int Q = 2 * PB;
  const size_t smem = ((size_t)lay.total + (size_t)(2 * kChunks - 1) * Q * kPS) * sizeof(double);
  if (smem > (size_t)kMaxDynSmem)
    return fail(SB_ERR_UNSUPPORTED, "partitioned FP64 solve: %zu B of shared memory needed", smem);
  auto k = part64_kernel<PB, L>;
  int nb = 0;
  SB_TRY(kernel_occupancy(reinterpret_cast<const void*>(k), f->device, kThreads, smem, &nb));
  if (shape.ctas_per_sm > 0) nb = std::min(nb, shape.ctas_per_sm);
  const int64_t ntiles = (M + kPS - 1) / kPS;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
  // one tile per CTA: the boundary solve is on the critical path of the whole launch,
  // so take the parallel form; otherwise the one with the least FP64 work
  const bool pcr = ntiles <= grid;
  k<<<(unsigned)grid, kThreads, smem, stream>>>(image, lay, (int)f->N, M, ld,
                                                static_cast<const double*>(rhs), static_cast<double*>(x),
                                                ntiles, pcr);
  return cuda_check(cudaGetLastError(), "partitioned FP64 solve launch");
}

template <int PB>
int dispatch(const sb_factor* f, const double* image, const void* rhs, void* x, int64_t M,
             int64_t ld, const SweepShape& shape, cudaStream_t stream) {
  switch (f->part64_L) {
    case 8: return launch<PB, 8>(f, image, rhs, x, M, ld, shape, stream);
    case 16: return launch<PB, 16>(f, image, rhs, x, M, ld, shape, stream);
    case 32: return launch<PB, 32>(f, image, rhs, x, M, ld, shape, stream);
    default: return fail(SB_ERR_UNSUPPORTED, "partitioned FP64 solve: chunk length %d", f->part64_L);
  }
}

}  // namespace

bool partitioned64_applies(const sb_factor* f, Op op, sb_dtype rhs_dtype, sb_dtype x_dtype,
                           int64_t M, sb_arith arith) {
  return arith == SB_ARITH_NATIVE && rhs_dtype == SB_F64 && x_dtype == SB_F64 && M >= 1 &&
         f->part64_img[op == OP_PRIMAL ? 0 : 1] != nullptr;
}

int launch_partitioned64(const sb_factor* f, Op op, const void* rhs, void* x, int64_t M, int64_t ld,
                         const SweepShape& shape, cudaStream_t stream) {
  const double* image = f->part64_img[op == OP_PRIMAL ? 0 : 1];
  if (image == nullptr) return fail(SB_ERR_UNSUPPORTED, "the partitioned FP64 solve does not apply");
  return f->P == 1 ? dispatch<1>(f, image, rhs, x, M, ld, shape, stream)
                   : dispatch<2>(f, image, rhs, x, M, ld, shape, stream);
}

}  // namespace sb
