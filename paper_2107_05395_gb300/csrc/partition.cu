// Partitioned batched solve (SB_ALGO_PARTITIONED; the math is in partition.h).
//
// The sequential sweeps keep the forward intermediate of every system in flight in
// x: with a whole batch in flight that intermediate leaves the chip and comes back,
// doubling the HBM traffic of an FP32 solve.  Here a CTA keeps a tile of 32
// systems on chip from the read of b to the write of x, so each element of b is
// read once and each element of x written once:
//   - the tile (32 systems x P L rows, FP32) arrives in shared memory by TMA
//     (cp.async.bulk.tensor, completion on an mbarrier); rows >= N and systems >= M
//     are filled with zeros by the copy;
//   - warp c owns chunk c (L rows) and lane s owns system s: each thread copies its
//     L values into registers (conflict-free: a warp reads one 128 B row), and once
//     every thread has its copy the next tile's TMA is issued into the same buffer,
//     so the HBM read of tile t+1 overlaps all the arithmetic of tile t;
//   - each chunk is swept forward and back with its own factors (y_c = A_c^{-1} b_c);
//     the coefficient rows are warp-uniform shared-memory broadcasts;
//   - the chunk heads and tails go to shared memory, then warp w solves the
//     boundary system of system w by parallel cyclic reduction with lane k holding
//     boundary k (neighbours exchanged with warp shuffles, no block barriers);
//   - every thread corrects its rows, x_c = y_c - W_c lam_c - V_c rho_c, and stores
//     them to x straight from registers (one 128 B row per warp and store).
// The partition image (chunk factors, spikes, reduction matrices) is staged into
// shared memory once per CTA; CTAs are persistent over the tiles.  Every wait on the
// mbarrier is bounded: on a timeout the CTA records it in a device flag (read with
// sb_device_timeouts), waits once more (bounded) for its copy in flight and returns.
#include <algorithm>
#include <mutex>

#include <cuda.h>

#include "partition.h"
#include "sb_internal.h"
#include "sweep_tile.cuh"

namespace sb {

__device__ unsigned int g_partition_timeouts = 0;

namespace {

constexpr int kTile = 32;              // systems per tile (one per lane)
constexpr int kSpinLimit = 1 << 20;    // bounded mbarrier polling (well under a second)

// cyclic-reduction levels for NW - 1 boundaries
__host__ __device__ constexpr int levels_for(int NW) { return NW == 16 ? 4 : 5; }

template <typename T, int n>
struct alignas(sizeof(T) * n) Row {
  T v[n];
};

template <typename TO>
struct OutCvt;
template <>
struct OutCvt<float> {
  static __device__ __forceinline__ float cvt(float v) { return v; }
};
template <>
struct OutCvt<double> {  // exact widening on the integer pipes
  static __device__ __forceinline__ double cvt(float v) { return widen_f32(v); }
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(phase)
      : "memory");
  return done != 0;
}

// Bounded wait for the completion of `phase` of the mbarrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (int i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, phase)) return true;
    if (i >= 8) __nanosleep(128);
  }
  return false;
}

// Thread 0: announce the tile's bytes on the mbarrier and issue its TMA copies
// (nbox boxes of 32 systems x box_rows rows, stacked in the buffer).
__device__ __forceinline__ void issue_tile(const CUtensorMap* tmap, uint32_t bar, float* buf,
                                           int64_t tile, int nbox, int box_rows) {
  const uint32_t bytes = (uint32_t)nbox * (uint32_t)box_rows * 32u * 4u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  const int x0 = (int)(tile * 32);
  for (int b = 0; b < nbox; ++b) {
    const uint32_t dst = smem_addr(buf + (size_t)b * box_rows * 32);
    const int y0 = b * box_rows;
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0), "r"(bar)
        : "memory");
  }
}

// NW warps = NW chunks of L rows; the CTA has NW * 32 threads.
template <typename TO, int PB, int L, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
part_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ image,
            PartLayout lay, int N, int64_t M, int64_t ld, TO* x, int64_t ntiles, int nbox,
            int box_rows) {
  constexpr int kThreads = NW * 32, kLevels = levels_for(NW);
  constexpr int Q = 2 * PB, FW = PB == 2 ? 4 : 2, K = NW - 1;
  constexpr int ZS = Q * 32 + 1;  // padded stride of a chunk / boundary in zt
  using RF = Row<float, FW>;
  using RB = Row<float, PB>;
  using RC = Row<float, Q>;
  extern __shared__ unsigned char smem_raw[];
  // buffer first, 1024-byte aligned; then the image, the head/tail/z array, the mbarrier
  float* buf = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* img = buf + (size_t)nbox * box_rows * 32;
  float* zt = img + lay.total;  // [NW][ZS]: chunk heads/tails, then boundary unknowns z
  uint64_t* barp = reinterpret_cast<uint64_t*>(zt + ((NW * ZS + 3) & ~3));  // 16-byte aligned
  const uint32_t bar = smem_addr(barp);
  const int tid = threadIdx.x;
  const int c = tid >> 5, s = tid & 31;

  {
    const float4* s4 = reinterpret_cast<const float4*>(image);
    float4* d4 = reinterpret_cast<float4*>(img);
    for (int k = tid; k < lay.total / 4; k += kThreads) d4[k] = s4[k];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) issue_tile(&tmap, bar, buf, blockIdx.x, nbox, box_rows);

  const RF* fw = reinterpret_cast<const RF*>(img + lay.fwd) + c * L;
  const RB* bw = reinterpret_cast<const RB*>(img + lay.bwd) + c * L;
  const RC* cw = reinterpret_cast<const RC*>(img + lay.cor) + c * L;
  const bool full_chunk = (c + 1) * L <= N;
  uint32_t phase = 0;

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const bool ok = mbar_wait(bar, phase);
    float y[L];
    if (ok) {
      const float* src = buf + (size_t)c * L * 32 + s;
#pragma unroll
      for (int j = 0; j < L; ++j) y[j] = src[j * 32];
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicAdd(&g_partition_timeouts, 1u);
        mbar_wait(bar, phase);  // bounded: let a late copy land before the CTA exits
      }
      return;
    }
    phase ^= 1u;
    // every thread has its rows: the buffer takes the next tile
    if (tid == 0 && tile + gridDim.x < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_tile(&tmap, bar, buf, tile + gridDim.x, nbox, box_rows);
    }
    // chunk sweeps: u_j = F0 b_j - F1 u_{j-1} - F2 u_{j-2};  y_j = u_j - B1 y_{j+1} - B2 y_{j+2}
    {
      float u1 = 0.f, u2 = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const RF f = fw[j];
        float t = y[j] * f.v[0];
        if constexpr (PB == 2) t = fmaf(-f.v[2], u2, t);
        const float u = fmaf(-f.v[1], u1, t);
        y[j] = u;
        u2 = u1;
        u1 = u;
      }
      float x1 = 0.f, x2 = 0.f;
#pragma unroll
      for (int j = L - 1; j >= 0; --j) {
        const RB b = bw[j];
        float t = y[j];
        if constexpr (PB == 2) t = fmaf(-b.v[1], x2, t);
        const float v = fmaf(-b.v[0], x1, t);
        y[j] = v;
        x2 = x1;
        x1 = v;
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      zt[c * ZS + u * 32 + s] = y[u];                 // head of chunk c
      zt[c * ZS + (PB + u) * 32 + s] = y[L - PB + u];  // tail of chunk c
    }
    __syncthreads();
    // boundary systems by cyclic reduction: warp w serves the 32 / NW systems
    // w + NW h, one per group of NW lanes; lane k of a group holds boundary k
    {
      const int k = s % NW, w = c + NW * (s / NW);
      float d[Q];
      {
        float r[Q];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          r[u] = k < K ? zt[k * ZS + (PB + u) * 32 + w] : 0.f;       // tail of chunk k
          r[PB + u] = k < K ? zt[(k + 1) * ZS + u * 32 + w] : 0.f;   // head of chunk k+1
        }
        const float* T0 = img + lay.T0 + k;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          float t = 0.f;
#pragma unroll
          for (int j = 0; j < Q; ++j) t = fmaf(T0[(i * Q + j) * NW], r[j], t);
          d[i] = t;
        }
      }
      const float* Mb = img + lay.M + k;
#pragma unroll 1
      for (int l = 0; l < kLevels; ++l) {
        const int st = 1 << l;
        float dl[PB], dr[PB];
#pragma unroll
        for (int u = 0; u < PB; ++u) {
          dl[u] = __shfl_up_sync(0xffffffffu, d[u], st, NW);
          dr[u] = __shfl_down_sync(0xffffffffu, d[PB + u], st, NW);
        }
        const bool has_l = k >= st, has_r = k + st < K;
        const float* M0 = Mb;
        const float* M1 = Mb + Q * Q * NW;
        const float* M2 = M1 + Q * PB * NW;
        float nd[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          float t = 0.f;
#pragma unroll
          for (int j = 0; j < Q; ++j) t = fmaf(M0[(i * Q + j) * NW], d[j], t);
#pragma unroll
          for (int j = 0; j < PB; ++j) {
            if (has_l) t = fmaf(-M1[(i * PB + j) * NW], dl[j], t);
            if (has_r) t = fmaf(-M2[(i * PB + j) * NW], dr[j], t);
          }
          nd[i] = t;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = nd[i];
        Mb += (Q * Q + 2 * Q * PB) * NW;
      }
      __syncwarp();  // every lane has read its heads and tails before any z is written
      if (k < K) {
#pragma unroll
        for (int i = 0; i < Q; ++i) zt[k * ZS + i * 32 + w] = d[i];
      }
    }
    __syncthreads();
    // correction x_j = y_j - W_j lam - V_j rho, stored straight to x
    {
      float lam[PB], rho[PB];
#pragma unroll
      for (int u = 0; u < PB; ++u) {
        lam[u] = c > 0 ? zt[(c - 1) * ZS + u * 32 + s] : 0.f;
        rho[u] = c < K ? zt[c * ZS + (PB + u) * 32 + s] : 0.f;
      }
      const int64_t m = tile * 32 + s;
      TO* dst = x + (int64_t)c * L * ld + m;
      if (m < M) {
        if (full_chunk) {
#pragma unroll
          for (int j = 0; j < L; ++j) {
            const RC wv = cw[j];
            float v = y[j];
#pragma unroll
            for (int u = 0; u < PB; ++u) {
              v = fmaf(-wv.v[u], lam[u], v);
              v = fmaf(-wv.v[PB + u], rho[u], v);
            }
            st_stream(dst + (int64_t)j * ld, OutCvt<TO>::cvt(v));
          }
        } else {
#pragma unroll
          for (int j = 0; j < L; ++j) {
            if (c * L + j < N) {
              const RC wv = cw[j];
              float v = y[j];
#pragma unroll
              for (int u = 0; u < PB; ++u) {
                v = fmaf(-wv.v[u], lam[u], v);
                v = fmaf(-wv.v[PB + u], rho[u], v);
              }
              st_stream(dst + (int64_t)j * ld, OutCvt<TO>::cvt(v));
            }
          }
        }
      }
    }
    // No barrier here: the next tile writes zt only after its __syncthreads_or, which
    // every thread reaches after finishing this tile's correction.
  }
}

// ------------------------------------------------------------------ host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

size_t smem_bytes(const PartLayout& lay, int nbox, int box_rows, int PB, int NW) {
  const int ZS = 2 * PB * 32 + 1;
  return 1024 + ((size_t)nbox * box_rows * 32 + lay.total + (size_t)((NW * ZS + 3) & ~3)) * 4 + 8;
}

template <typename TO, int PB, int L, int NW>
int launch_part(const sb_factor* f, const float* image, const CUtensorMap& tmap, void* x,
                int64_t M, int64_t ld, cudaStream_t stream) {
  const int N = (int)f->N;
  const int P = NW;
  const PartLayout lay = part_layout(PB, L, P, levels_for(NW));
  const int box_rows = std::min(256, P * L), nbox = (P * L) / box_rows;
  const size_t smem = smem_bytes(lay, nbox, box_rows, PB, NW);
  if (smem > (size_t)kMaxDynSmem)
    return fail(SB_ERR_UNSUPPORTED, "partitioned solve: %zu B of shared memory needed", smem);
  auto k = part_kernel<TO, PB, L, NW>;
  int nb = 0;
  SB_TRY(kernel_occupancy(reinterpret_cast<const void*>(k), f->device, NW * 32, smem, &nb));
  const int64_t ntiles = (M + 31) / 32;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
  k<<<(unsigned)grid, NW * 32, smem, stream>>>(tmap, image, lay, N, M, ld, static_cast<TO*>(x),
                                                ntiles, nbox, box_rows);
  return cuda_check(cudaGetLastError(), "partitioned solve launch");
}

template <typename TO, int PB>
int dispatch_l(const sb_factor* f, int v, const float* image, const CUtensorMap& tmap, void* x,
               int64_t M, int64_t ld, cudaStream_t stream) {
  const int L = f->part_L[v];
  if (v == 0) {
    switch (L) {
      case 16: return launch_part<TO, PB, 16, 16>(f, image, tmap, x, M, ld, stream);
      case 32: return launch_part<TO, PB, 32, 16>(f, image, tmap, x, M, ld, stream);
      case 64: return launch_part<TO, PB, 64, 16>(f, image, tmap, x, M, ld, stream);
      default: break;
    }
  } else {
    switch (L) {
      case 8: return launch_part<TO, PB, 8, 32>(f, image, tmap, x, M, ld, stream);
      case 16: return launch_part<TO, PB, 16, 32>(f, image, tmap, x, M, ld, stream);
      case 32: return launch_part<TO, PB, 32, 32>(f, image, tmap, x, M, ld, stream);
      default: break;
    }
  }
  return fail(SB_ERR_UNSUPPORTED, "partitioned solve: chunk length %d", L);
}

}  // namespace

int part_variant(int threads) { return threads == 512 ? 0 : (threads == 1024 ? 1 : -1); }

bool partitioned_applies(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype,
                         sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, int threads) {
  const int o = op == OP_PRIMAL ? 0 : 1, v = part_variant(threads);
  return v >= 0 && arith == SB_ARITH_NATIVE && rhs_dtype == SB_F32 &&
         (x_dtype == SB_F32 || x_dtype == SB_F64) && f->part_img[o][v] != nullptr &&
         f->part_NL[v] == levels_for(part_chunks(v)) && M >= 1 &&
         (reinterpret_cast<uintptr_t>(rhs) % 16) == 0 && ((ld * 4) % 16) == 0 &&
         ld * 4 < ((int64_t)1 << 40) && encode_fn() != nullptr;
}

int launch_partitioned(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype, void* x,
                       sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith,
                       const SweepShape& shape, cudaStream_t stream) {
  if (!partitioned_applies(f, op, rhs, rhs_dtype, x_dtype, M, ld, arith, shape.threads))
    return fail(SB_ERR_UNSUPPORTED, "the partitioned solve does not apply to this call");
  const int o = op == OP_PRIMAL ? 0 : 1, v = part_variant(shape.threads);
  const int box_rows = std::min(256, part_chunks(v) * f->part_L[v]);
  CUtensorMap tmap;
  const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)f->N};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(rhs), dims,
                                 strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SB_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  const float* image = f->part_img[o][v];
  if (f->P == 1)
    return x_dtype == SB_F32 ? dispatch_l<float, 1>(f, v, image, tmap, x, M, ld, stream)
                             : dispatch_l<double, 1>(f, v, image, tmap, x, M, ld, stream);
  return x_dtype == SB_F32 ? dispatch_l<float, 2>(f, v, image, tmap, x, M, ld, stream)
                           : dispatch_l<double, 2>(f, v, image, tmap, x, M, ld, stream);
}

int partition_timeouts(int device, unsigned* count) {
  DeviceGuard g(device);
  SB_TRY(g.rc);
  unsigned v = 0, zero = 0;
  SB_CUDA(cudaMemcpyFromSymbol(&v, g_partition_timeouts, sizeof(v)));
  SB_CUDA(cudaMemcpyToSymbol(g_partition_timeouts, &zero, sizeof(zero)));
  *count = v;
  return SB_OK;
}

}  // namespace sb
