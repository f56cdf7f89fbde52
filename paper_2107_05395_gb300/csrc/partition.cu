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
//   - warp c owns chunk c (L rows) and lane s owns system s: each thread holds its
//     L values in registers (a warp reads one 128 B row of the tile at a time);
//   - each chunk is swept forward and back with its own factors (y_c = A_c^{-1} b_c);
//     the coefficient rows are warp-uniform shared-memory broadcasts;
//   - the chunk heads and tails go to shared memory, then warp w solves the
//     boundary system of system w by parallel cyclic reduction with lane k holding
//     boundary k (neighbours exchanged with warp shuffles, no block barriers);
//   - every thread corrects its rows, x_c = y_c - W_c lam_c - V_c rho_c, and stores
//     them to x straight from registers (one 128 B row per warp and store).
// The next tile's TMA load is issued as soon as every thread has copied the current
// tile to registers, so it overlaps all of the current tile's arithmetic; the
// 256-thread form also spreads its FP32 stores over the next tile through tensor
// memory (see part_kernel2).  (Staging
// x back through the buffer for TMA stores was measured slower: it doubles the
// shared-memory instructions per element and makes the next load wait for the
// store to have read the buffer.)
// The partition image (chunk factors, spikes, reduction matrices) is staged into
// shared memory once per CTA; CTAs are persistent over the tiles.  Every wait on an
// mbarrier is bounded: on a timeout the CTA records it in a device flag (read with
// sb_device_timeouts), waits once more (bounded) for its copy in flight and returns.
#include <algorithm>
#include <mutex>
#include <type_traits>

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

// Two adjacent output values as one vector store.
template <typename TO>
struct Vec2;
template <>
struct Vec2<float> {
  using T = float2;
};
template <>
struct Vec2<double> {
  using T = double2;
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

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Announce the tile's bytes on the mbarrier and issue its TMA loads (nbox boxes of
// 32 systems x box_rows rows, stacked in the buffer).
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

// ------------------------------------------------------------ the solve's steps

// Chunk sweeps in registers, y <- A_c^{-1} y:
//   u_j = F0 b_j - F1 u_{j-1} - F2 u_{j-2};  y_j = u_j - B1 y_{j+1} - B2 y_{j+2}
template <int PB, int L, typename RF, typename RB>
__device__ __forceinline__ void chunk_solve(float (&y)[L], const RF* fw, const RB* bw) {
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

// Head (first PB rows) and tail (last PB rows) of chunk c of system s into zt.
template <int PB, int L, int ZS>
__device__ __forceinline__ void put_heads_tails(float* zt, const float (&y)[L], int c, int s) {
#pragma unroll
  for (int u = 0; u < PB; ++u) {
    zt[c * ZS + u * 32 + s] = y[u];
    zt[c * ZS + (PB + u) * 32 + s] = y[L - PB + u];
  }
}

// The boundary systems by cyclic reduction, in place in zt: warp c serves the
// 32 / NW systems c + NW h, one per group of NW lanes; lane k of a group holds
// boundary k.  Reads the heads and tails of its systems and overwrites them with the
// boundary unknowns z (each warp touches only its own systems' columns).
template <int PB, int NW, int ZS>
__device__ __forceinline__ void boundary_solve(float* zt, const float* img, const PartLayout& lay,
                                               int c, int s) {
  constexpr int Q = 2 * PB, K = NW - 1, kLevels = levels_for(NW);
  using RQ = Row<float, Q>;
  using RP = Row<float, PB>;
  const int k = s % NW, w = c + NW * (s / NW);
  float d[Q];
  {
    float r[Q];
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      r[u] = k < K ? zt[k * ZS + (PB + u) * 32 + w] : 0.f;      // tail of chunk k
      r[PB + u] = k < K ? zt[(k + 1) * ZS + u * 32 + w] : 0.f;  // head of chunk k+1
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

// The same reduction with two systems per lane (the 256-thread kernel): warp w
// serves systems sa = 4w + 2g and sa + 1 with the 16 lanes of group g = lane / 16,
// lane k of a group holding boundary k; each matrix entry is read once for both.
template <int PB, int ZS>
__device__ __forceinline__ void boundary_solve2(float* zt, const float* img, const PartLayout& lay, int w,
                                                int lane) {
  constexpr int NW = 16, Q = 2 * PB, K = NW - 1, kLevels = levels_for(NW);
  const int k = lane & 15, sa = 4 * w + 2 * (lane >> 4);
  float d[2][Q];
  {
    float r[2][Q];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int u = 0; u < PB; ++u) {
        r[e][u] = k < K ? zt[k * ZS + (PB + u) * 32 + sa + e] : 0.f;       // tail of chunk k
        r[e][PB + u] = k < K ? zt[(k + 1) * ZS + u * 32 + sa + e] : 0.f;   // head of chunk k+1
      }
    const float* T0 = img + lay.T0 + k;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float t0 = 0.f, t1 = 0.f;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const float a = T0[(i * Q + j) * NW];
        t0 = fmaf(a, r[0][j], t0);
        t1 = fmaf(a, r[1][j], t1);
      }
      d[0][i] = t0;
      d[1][i] = t1;
    }
  }
  const float* Mb = img + lay.M + k;
#pragma unroll 1
  for (int l = 0; l < kLevels; ++l) {
    const int st = 1 << l;
    float dl[2][PB], dr[2][PB];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
      for (int u = 0; u < PB; ++u) {
        dl[e][u] = __shfl_up_sync(0xffffffffu, d[e][u], st, NW);
        dr[e][u] = __shfl_down_sync(0xffffffffu, d[e][PB + u], st, NW);
      }
    const bool has_l = k >= st, has_r = k + st < K;
    const float* M0 = Mb;
    const float* M1 = Mb + Q * Q * NW;
    const float* M2 = M1 + Q * PB * NW;
    float nd[2][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float t0 = 0.f, t1 = 0.f;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const float a = M0[(i * Q + j) * NW];
        t0 = fmaf(a, d[0][j], t0);
        t1 = fmaf(a, d[1][j], t1);
      }
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        if (has_l) {
          const float a = M1[(i * PB + j) * NW];
          t0 = fmaf(-a, dl[0][j], t0);
          t1 = fmaf(-a, dl[1][j], t1);
        }
        if (has_r) {
          const float a = M2[(i * PB + j) * NW];
          t0 = fmaf(-a, dr[0][j], t0);
          t1 = fmaf(-a, dr[1][j], t1);
        }
      }
      nd[0][i] = t0;
      nd[1][i] = t1;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      d[0][i] = nd[0][i];
      d[1][i] = nd[1][i];
    }
    Mb += (Q * Q + 2 * Q * PB) * NW;
  }
  __syncwarp();  // every lane has read its heads and tails before any z is written
  if (k < K) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      zt[k * ZS + i * 32 + sa] = d[0][i];
      zt[k * ZS + i * 32 + sa + 1] = d[1][i];
    }
  }
}

// The boundary unknowns next to chunk c of system s: lam (last PB of chunk c-1) and
// rho (first PB of chunk c+1), zero at the ends.
template <int PB, int NW, int ZS>
__device__ __forceinline__ void neighbours(const float* zt, int c, int s, float (&lam)[PB], float (&rho)[PB]) {
#pragma unroll
  for (int u = 0; u < PB; ++u) {
    lam[u] = c > 0 ? zt[(c - 1) * ZS + u * 32 + s] : 0.f;
    rho[u] = c < NW - 1 ? zt[c * ZS + (PB + u) * 32 + s] : 0.f;
  }
}

// Corrected row: x_j = y_j - W_j lam - V_j rho.
template <int PB, typename RC>
__device__ __forceinline__ float corrected(float y, const RC& wv, const float (&lam)[PB], const float (&rho)[PB]) {
  float v = y;
#pragma unroll
  for (int u = 0; u < PB; ++u) {
    v = fmaf(-wv.v[u], lam[u], v);
    v = fmaf(-wv.v[PB + u], rho[u], v);
  }
  return v;
}

// ------------------------------------------------------------------ the kernels

// Shared-memory carve-up: the tile buffer first (1024-byte aligned), then the image,
// the head/tail/z array (NW * ZS floats), the mbarrier and the word that receives a
// tensor-memory address.
struct PartSmem {
  float* buf;
  float* img;
  float* zt;
  uint64_t* bar;
};

template <int PB, int NW>
__device__ __forceinline__ PartSmem carve(unsigned char* raw, const PartLayout& lay, int nbox, int box_rows) {
  constexpr int ZS = 2 * PB * 32 + 1;
  PartSmem m;
  m.buf = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  m.img = m.buf + (size_t)nbox * box_rows * 32;
  m.zt = m.img + lay.total;
  m.bar = reinterpret_cast<uint64_t*>(m.zt + ((NW * ZS + 3) & ~3));  // 16-byte aligned
  return m;
}

size_t smem_bytes(const PartLayout& lay, int nbox, int box_rows, int PB, int NW) {
  const int ZS = 2 * PB * 32 + 1;
  return 1024 + ((size_t)nbox * box_rows * 32 + lay.total + (size_t)((NW * ZS + 3) & ~3)) * 4 + 16;
}

// NW warps = NW chunks of L rows.
template <typename TO, int PB, int L, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
part_kernel(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ image,
            PartLayout lay, int N, int64_t M, int64_t ld, TO* x, int64_t ntiles, int nbox,
            int box_rows) {
  constexpr int kThreads = NW * 32;
  constexpr int Q = 2 * PB, FW = PB == 2 ? 4 : 2;
  constexpr int ZS = Q * 32 + 1;  // padded stride of a chunk / boundary in zt
  using RF = Row<float, FW>;
  using RB = Row<float, PB>;
  using RC = Row<float, Q>;
  extern __shared__ unsigned char smem_raw[];
  const PartSmem sm = carve<PB, NW>(smem_raw, lay, nbox, box_rows);
  float* const buf = sm.buf;
  float* const zt = sm.zt;
  const uint32_t bar = smem_addr(sm.bar);
  const int tid = threadIdx.x;
  const int c = tid >> 5, s = tid & 31;

  {
    const float4* s4 = reinterpret_cast<const float4*>(image);
    float4* d4 = reinterpret_cast<float4*>(sm.img);
    for (int k = tid; k < lay.total / 4; k += kThreads) d4[k] = s4[k];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) issue_tile(&tmap, bar, buf, blockIdx.x, nbox, box_rows);

  const RF* fw = reinterpret_cast<const RF*>(sm.img + lay.fwd) + c * L;
  const RB* bw = reinterpret_cast<const RB*>(sm.img + lay.bwd) + c * L;
  const RC* cw = reinterpret_cast<const RC*>(sm.img + lay.cor) + c * L;
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
    chunk_solve<PB, L>(y, fw, bw);
    put_heads_tails<PB, L, ZS>(zt, y, c, s);
    __syncthreads();
    boundary_solve<PB, NW, ZS>(zt, sm.img, lay, c, s);
    __syncthreads();
    float lam[PB], rho[PB];
    neighbours<PB, NW, ZS>(zt, c, s, lam, rho);
    const int64_t m = tile * 32 + s;
    TO* dst = x + (int64_t)c * L * ld + m;
    if (m < M) {
      if (full_chunk) {
#pragma unroll
        for (int j = 0; j < L; ++j)
          st_stream(dst + (int64_t)j * ld, OutCvt<TO>::cvt(corrected<PB>(y[j], cw[j], lam, rho)));
      } else {
#pragma unroll
        for (int j = 0; j < L; ++j)
          if (c * L + j < N)
            st_stream(dst + (int64_t)j * ld, OutCvt<TO>::cvt(corrected<PB>(y[j], cw[j], lam, rho)));
      }
    }
    // No barrier here: the next tile writes zt only after its __syncthreads_or, which
    // every thread reaches after finishing this tile's correction.
  }
}

// Two systems per thread: 256 threads, 16 chunks of L rows.  Warp w holds chunks
// 2w (lanes 0-15) and 2w + 1 (lanes 16-31); lane l holds the adjacent systems
// s0 = 2 (l % 16) and s0 + 1 of its chunk, so every coefficient read from shared
// memory serves two systems, the tile is copied with 64-bit loads and x leaves with
// 64-bit (FP32) or 128-bit (FP64) stores.  `image` is the paired image
// (partition_image_paired): the two half-warps' coefficient rows are neighbours.
// vec: x is aligned for the paired stores (else each system is stored alone).  The
// CTAs take tiles tile0 .. ntiles - 1 round-robin; those with one tile fewer than
// the others start delay_ns later (they have that time to spare), so that their
// store phases interleave with the others' compute.
template <typename TO, int PB, int L>
__global__ void __launch_bounds__(256, 1)
part_kernel2(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ image,
             PartLayout lay, int N, int64_t M, int64_t ld, TO* x, int64_t tile0, int64_t ntiles, int nbox,
             int box_rows, bool vec, int delay_ns) {
  constexpr int NW = 16, kThreads = 256;
  constexpr int Q = 2 * PB, FW = PB == 2 ? 4 : 2;
  constexpr int ZS = Q * 32 + 1;
  using RF = Row<float, FW>;
  using RB = Row<float, PB>;
  using RC = Row<float, Q>;
  using T2 = typename Vec2<TO>::T;
  extern __shared__ unsigned char smem_raw[];
  const PartSmem sm = carve<PB, NW>(smem_raw, lay, nbox, box_rows);
  float* const buf = sm.buf;
  float* const zt = sm.zt;
  const uint32_t bar = smem_addr(sm.bar);
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31, h = lane >> 4;
  const int c = 2 * w + h, s0 = 2 * (lane & 15);

  {
    const float4* s4 = reinterpret_cast<const float4*>(image);
    float4* d4 = reinterpret_cast<float4*>(sm.img);
    for (int k = tid; k < lay.total / 4; k += kThreads) d4[k] = s4[k];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const int64_t first = tile0 + blockIdx.x;
  if (tid == 0 && first < ntiles) {
    const int64_t rem = (ntiles - tile0) % gridDim.x;
    if (rem != 0 && (int64_t)blockIdx.x >= rem)
      for (int t = 0; t < delay_ns; t += 256) __nanosleep(256);
    issue_tile(&tmap, bar, buf, first, nbox, box_rows);
  }

  // row j of chunk c at paired row w 2L + 2j + h
  const RF* fw = reinterpret_cast<const RF*>(sm.img + lay.fwd) + w * 2 * L + h;
  const RB* bw = reinterpret_cast<const RB*>(sm.img + lay.bwd) + w * 2 * L + h;
  const RC* cw = reinterpret_cast<const RC*>(sm.img + lay.cor) + w * 2 * L + h;
  const int rows = min(L, N - c * L);  // rows of chunk c inside the matrix (may be <= 0)
  uint32_t phase = 0;

  for (int64_t tile = first; tile < ntiles; tile += gridDim.x) {
    const bool ok = mbar_wait(bar, phase);
    float y0[L], y1[L];
    if (ok) {
      const float2* src = reinterpret_cast<const float2*>(buf + (size_t)c * L * 32 + s0);
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const float2 v = src[j * 16];
        y0[j] = v.x;
        y1[j] = v.y;
      }
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicAdd(&g_partition_timeouts, 1u);
        mbar_wait(bar, phase);  // bounded: let a late copy land before the CTA exits
      }
      return;
    }
    phase ^= 1u;
    if (tid == 0 && tile + gridDim.x < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_tile(&tmap, bar, buf, tile + gridDim.x, nbox, box_rows);
    }
    // chunk sweeps of both systems with the same coefficient rows
    {
      float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const RF f = fw[2 * j];
        float ta = y0[j] * f.v[0], tb = y1[j] * f.v[0];
        if constexpr (PB == 2) {
          ta = fmaf(-f.v[2], a2, ta);
          tb = fmaf(-f.v[2], b2, tb);
        }
        const float ua = fmaf(-f.v[1], a1, ta), ub = fmaf(-f.v[1], b1, tb);
        y0[j] = ua;
        y1[j] = ub;
        a2 = a1;
        a1 = ua;
        b2 = b1;
        b1 = ub;
      }
      a1 = a2 = b1 = b2 = 0.f;
#pragma unroll
      for (int j = L - 1; j >= 0; --j) {
        const RB b = bw[2 * j];
        float ta = y0[j], tb = y1[j];
        if constexpr (PB == 2) {
          ta = fmaf(-b.v[1], a2, ta);
          tb = fmaf(-b.v[1], b2, tb);
        }
        const float va = fmaf(-b.v[0], a1, ta), vb = fmaf(-b.v[0], b1, tb);
        y0[j] = va;
        y1[j] = vb;
        a2 = a1;
        a1 = va;
        b2 = b1;
        b1 = vb;
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      zt[c * ZS + u * 32 + s0] = y0[u];
      zt[c * ZS + u * 32 + s0 + 1] = y1[u];
      zt[c * ZS + (PB + u) * 32 + s0] = y0[L - PB + u];
      zt[c * ZS + (PB + u) * 32 + s0 + 1] = y1[L - PB + u];
    }
    __syncthreads();
    boundary_solve2<PB, ZS>(zt, sm.img, lay, w, lane);
    __syncthreads();
    float lam0[PB], rho0[PB], lam1[PB], rho1[PB];
    neighbours<PB, NW, ZS>(zt, c, s0, lam0, rho0);
    neighbours<PB, NW, ZS>(zt, c, s0 + 1, lam1, rho1);
    const int64_t m = tile * 32 + s0;
    TO* dst = x + (int64_t)c * L * ld + m;
    if (vec && m + 1 < M && rows == L) {
#pragma unroll
      for (int j = 0; j < L; ++j) {
        const RC wv = cw[2 * j];
        T2 v;
        v.x = OutCvt<TO>::cvt(corrected<PB>(y0[j], wv, lam0, rho0));
        v.y = OutCvt<TO>::cvt(corrected<PB>(y1[j], wv, lam1, rho1));
        st_stream(reinterpret_cast<T2*>(dst + (int64_t)j * ld), v);
      }
    } else if (m < M) {
#pragma unroll
      for (int j = 0; j < L; ++j)
        if (j < rows) {
          const RC wv = cw[2 * j];
          st_stream(dst + (int64_t)j * ld, OutCvt<TO>::cvt(corrected<PB>(y0[j], wv, lam0, rho0)));
          if (m + 1 < M) st_stream(dst + (int64_t)j * ld + 1, OutCvt<TO>::cvt(corrected<PB>(y1[j], wv, lam1, rho1)));
        }
    }
    // No barrier here: the next tile writes zt only after its __syncthreads_or.
  }
}

// Tensor memory (TMEM) used as plain storage: an SM's 512 columns x 128 lanes of
// 32-bit words, reached from registers with tcgen05.st / tcgen05.ld (no MMA).  Warp w
// may touch only lanes 32 (w % 4) .. 32 (w % 4) + 31, its thread t lane 32 (w % 4) + t.
__device__ __forceinline__ void tm_st16(uint32_t ta, const float (&v)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};"
               :: "r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
                  "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
                  "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                  "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
               : "memory");
}
__device__ __forceinline__ void tm_ld2(uint32_t ta, uint32_t& a, uint32_t& b) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "r"(ta) : "memory");
}
// The loaded registers are valid only after the wait; they are operands of it so that
// no use of them is scheduled before it.
__device__ __forceinline__ void tm_wait_ld(uint32_t& a, uint32_t& b) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(a), "+r"(b) :: "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// The 256-thread form for FP32 x with its stores spread over the next tile.  With
// direct stores every SM writes its tile's x in one burst at the end of the tile,
// all SMs at once, while DRAM idles through the other phases.  Here the corrected
// rows go to tensor memory (two slots of 2L columns per warp, alternating by tile),
// and while the next tile is copied, swept and corrected each thread takes one row
// pair of the previous tile back every few rows and stores it, so DRAM sees reads and
// writes throughout; the last tile's rows leave after the loop.  The arithmetic is
// part_kernel2's, so the results are the same bits.  Every tile must be whole (32
// systems, N = 16 L rows) and x aligned for paired stores; the launcher sends a
// partial last tile to part_kernel2.  CTAs with one tile fewer start delay_ns later.
template <int PB, int L>
__global__ void __launch_bounds__(256, 1)
part_kernel2s(const __grid_constant__ CUtensorMap tmap, const float* __restrict__ image,
             PartLayout lay, int N, int64_t M, int64_t ld, float* x, int64_t ntiles, int nbox, int box_rows,
             int delay_ns) {
  constexpr int NW = 16, kThreads = 256;
  constexpr int Q = 2 * PB, FW = PB == 2 ? 4 : 2;
  constexpr int ZS = Q * 32 + 1;
  // TMEM columns: two slots of 2L per warp, two warps per lane quadrant (a power of
  // two; every CTA that can share an SM fits in the 512)
  constexpr int kCols = 8 * L;
  static_assert(kCols >= 32 && kCols <= 512 && (kCols & (kCols - 1)) == 0, "TMEM allocation size");
  using RF = Row<float, FW>;
  using RB = Row<float, PB>;
  using RC = Row<float, Q>;
  extern __shared__ unsigned char smem_raw[];
  const PartSmem sm = carve<PB, NW>(smem_raw, lay, nbox, box_rows);
  float* const buf = sm.buf;
  float* const zt = sm.zt;
  const uint32_t bar = smem_addr(sm.bar);
  const int tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31, h = lane >> 4;
  const int c = 2 * w + h, s0 = 2 * (lane & 15);
  {
    const float4* s4 = reinterpret_cast<const float4*>(image);
    float4* d4 = reinterpret_cast<float4*>(sm.img);
    for (int k = tid; k < lay.total / 4; k += kThreads) d4[k] = s4[k];
  }
  if (w == 0) {  // the TMEM address goes to the word after the mbarrier
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(sm.bar + 1)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(sm.bar + 1);
  const uint32_t tw0 = tbase + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)((w >> 2) * 4 * L);
  uint32_t tw = tw0;        // stash slot of the current tile
  uint32_t tprev = tw0;     // slot of the previous tile (being drained)
  if (tid == 0 && (int64_t)blockIdx.x < ntiles) {
    const int64_t rem = ntiles % gridDim.x;
    if (rem != 0 && (int64_t)blockIdx.x >= rem)  // one tile fewer than CTAs 0 .. rem - 1
      for (int t = 0; t < delay_ns; t += 256) __nanosleep(256);
    issue_tile(&tmap, bar, buf, blockIdx.x, nbox, box_rows);
  }

  const RF* fw = reinterpret_cast<const RF*>(sm.img + lay.fwd) + w * 2 * L + h;
  const RB* bw = reinterpret_cast<const RB*>(sm.img + lay.bwd) + w * 2 * L + h;
  const RC* cw = reinterpret_cast<const RC*>(sm.img + lay.cor) + w * 2 * L + h;
  uint32_t phase = 0;
  bool has_prev = false;
  float* pdst = nullptr;  // row c L of the previous tile's systems s0, s0 + 1
  uint32_t da = 0, db = 0;

  // drain step r = 0 .. L of the previous tile: store its row pair r - 1, load pair r
  auto drain = [&](int r) {
    if (r > 0) {
      tm_wait_ld(da, db);
      st_stream(reinterpret_cast<float2*>(pdst + (int64_t)(r - 1) * ld), make_float2(__uint_as_float(da), __uint_as_float(db)));
    }
    if (r < L) tm_ld2(tprev + 2 * r, da, db);
  };

  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const bool ok = mbar_wait(bar, phase);
    float y0[L], y1[L];
    {  // unconditional, so that the warp-wide drains stay uniform; a tile whose wait
       // timed out is discarded below
      const float2* src = reinterpret_cast<const float2*>(buf + (size_t)c * L * 32 + s0);
#pragma unroll
      for (int j = 0; j < L; ++j) {
        if (has_prev && (j & 3) == 0) drain(j / 4);
        const float2 v = src[j * 16];
        y0[j] = v.x;
        y1[j] = v.y;
      }
    }
    tm_fence_before();
    const bool bad = __syncthreads_or(!ok);
    tm_fence_after();
    if (bad) {
      tm_wait_ld(da, db);  // no tensor-memory access may be in flight when it is freed
      tm_fence_before();
      __syncthreads();
      tm_fence_after();
      if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols) : "memory");
      if (tid == 0) {
        atomicAdd(&g_partition_timeouts, 1u);
        mbar_wait(bar, phase);  // bounded: let a late copy land before the CTA exits
      }
      return;
    }
    phase ^= 1u;
    if (tid == 0 && tile + gridDim.x < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_tile(&tmap, bar, buf, tile + gridDim.x, nbox, box_rows);
    }
    {
      float a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
#pragma unroll
      for (int j = 0; j < L; ++j) {
        if (has_prev && (j & 3) == 0) drain(L / 4 + j / 4);
        const RF f = fw[2 * j];
        float ta = y0[j] * f.v[0], tb = y1[j] * f.v[0];
        if constexpr (PB == 2) {
          ta = fmaf(-f.v[2], a2, ta);
          tb = fmaf(-f.v[2], b2, tb);
        }
        const float ua = fmaf(-f.v[1], a1, ta), ub = fmaf(-f.v[1], b1, tb);
        y0[j] = ua;
        y1[j] = ub;
        a2 = a1;
        a1 = ua;
        b2 = b1;
        b1 = ub;
      }
      a1 = a2 = b1 = b2 = 0.f;
#pragma unroll
      for (int j = L - 1; j >= 0; --j) {
        const int t = L - 1 - j;
        if (has_prev && (t & 3) == 0) drain(L / 2 + t / 4);
        const RB b = bw[2 * j];
        float ta = y0[j], tb = y1[j];
        if constexpr (PB == 2) {
          ta = fmaf(-b.v[1], a2, ta);
          tb = fmaf(-b.v[1], b2, tb);
        }
        const float va = fmaf(-b.v[0], a1, ta), vb = fmaf(-b.v[0], b1, tb);
        y0[j] = va;
        y1[j] = vb;
        a2 = a1;
        a1 = va;
        b2 = b1;
        b1 = vb;
      }
    }
#pragma unroll
    for (int u = 0; u < PB; ++u) {
      zt[c * ZS + u * 32 + s0] = y0[u];
      zt[c * ZS + u * 32 + s0 + 1] = y1[u];
      zt[c * ZS + (PB + u) * 32 + s0] = y0[L - PB + u];
      zt[c * ZS + (PB + u) * 32 + s0 + 1] = y1[L - PB + u];
    }
    __syncthreads();
    boundary_solve2<PB, ZS>(zt, sm.img, lay, w, lane);
    __syncthreads();
    float lam0[PB], rho0[PB], lam1[PB], rho1[PB];
    neighbours<PB, NW, ZS>(zt, c, s0, lam0, rho0);
    neighbours<PB, NW, ZS>(zt, c, s0 + 1, lam1, rho1);
    // this tile's rows into the current slot (eight row pairs per store) while the
    // previous tile's last quarter drains from the other
#pragma unroll
    for (int j0 = 0; j0 < L; j0 += 8) {
      if (has_prev) {
        drain(3 * L / 4 + j0 / 8 * 2);
        drain(3 * L / 4 + j0 / 8 * 2 + 1);
      }
      float v[16];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const RC wv = cw[2 * (j0 + j)];
        v[2 * j] = corrected<PB>(y0[j0 + j], wv, lam0, rho0);
        v[2 * j + 1] = corrected<PB>(y1[j0 + j], wv, lam1, rho1);
      }
      tm_st16(tw + 2 * j0, v);
    }
    if (has_prev) drain(L);
    tm_wait_st();
    has_prev = true;
    tprev = tw;
    tw = (tw == tw0) ? tw0 + 2 * L : tw0;
    pdst = x + (int64_t)c * L * ld + tile * 32 + s0;
  }
  if (has_prev)
    for (int r = 0; r <= L; ++r) drain(r);
  tm_fence_before();
  __syncthreads();
  tm_fence_after();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(kCols) : "memory");
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

// Tensor map of an N x ld interleaved FP32 array (M systems used), boxes of 32
// systems x box_rows rows.
int encode_tile_map(CUtensorMap* tmap, const void* base, int64_t N, int64_t M, int64_t ld, int box_rows) {
  const cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)N};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = encode_fn()(tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SB_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return SB_OK;
}

int box_rows_for(int P, int L) { return std::min(256, P * L); }

// Persistent grid: one CTA per resident slot, at most one per tile.
int part_grid(const void* kernel, const sb_factor* f, int threads, size_t smem, int64_t ntiles, int64_t* grid) {
  int nb = 0;
  SB_TRY(kernel_occupancy(kernel, f->device, threads, smem, &nb));
  if (nb < 1) return fail(SB_ERR_UNSUPPORTED, "partitioned solve: the kernel does not fit on an SM");
  *grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)nb * sm_count(f->device)));
  return SB_OK;
}

template <typename TO, int PB, int L, int NW>
int launch_part(const sb_factor* f, const float* image, const CUtensorMap& tmap, void* x,
                int64_t M, int64_t ld, cudaStream_t stream) {
  const int N = (int)f->N;
  const PartLayout lay = part_layout(PB, L, NW, levels_for(NW));
  const int box_rows = box_rows_for(NW, L), nbox = (NW * L) / box_rows;
  const size_t smem = smem_bytes(lay, nbox, box_rows, PB, NW);
  if (smem > (size_t)kMaxDynSmem)
    return fail(SB_ERR_UNSUPPORTED, "partitioned solve: %zu B of shared memory needed", smem);
  auto k = part_kernel<TO, PB, L, NW>;
  const int64_t ntiles = (M + 31) / 32;
  int64_t grid = 0;
  SB_TRY(part_grid(reinterpret_cast<const void*>(k), f, NW * 32, smem, ntiles, &grid));
  k<<<(unsigned)grid, NW * 32, smem, stream>>>(tmap, image, lay, N, M, ld, static_cast<TO*>(x), ntiles, nbox,
                                                box_rows);
  return cuda_check(cudaGetLastError(), "partitioned solve launch");
}

template <typename TO, int PB, int L>
int launch_part2(const sb_factor* f, const float* image, const CUtensorMap& tmap, void* x,
                 int64_t M, int64_t ld, cudaStream_t stream) {
  constexpr int NW = 16;
  const int N = (int)f->N;
  const PartLayout lay = part_layout(PB, L, NW, levels_for(NW));
  const int box_rows = box_rows_for(NW, L), nbox = (NW * L) / box_rows;
  const size_t smem = smem_bytes(lay, nbox, box_rows, PB, NW);
  if (smem > (size_t)kMaxDynSmem)
    return fail(SB_ERR_UNSUPPORTED, "partitioned solve: %zu B of shared memory needed", smem);
  const int64_t ntiles = (M + 31) / 32;
  // paired stores need x aligned to two elements (rows start aligned: ld % 4 == 0)
  const bool vec = (reinterpret_cast<uintptr_t>(x) % (2 * sizeof(TO))) == 0;
  // CTAs with one tile fewer start ~2 ns per row later (about a third of a tile)
  const int delay_ns = 2 * N;
  int64_t done = 0;  // tiles handled by the stashing kernel
  if constexpr (std::is_same<TO, float>::value) {
    if (vec && N == NW * L && M >= 32) {
      done = M / 32;
      auto ks = part_kernel2s<PB, L>;
      int64_t grid = 0;
      SB_TRY(part_grid(reinterpret_cast<const void*>(ks), f, 256, smem, done, &grid));
      ks<<<(unsigned)grid, 256, smem, stream>>>(tmap, image, lay, N, M, ld, static_cast<float*>(x), done, nbox,
                                                box_rows, delay_ns);
      SB_TRY(cuda_check(cudaGetLastError(), "partitioned solve launch"));
      if (done == ntiles) return SB_OK;
    }
  }
  // every tile, or the partial last one after the stashing kernel
  auto k = part_kernel2<TO, PB, L>;
  int64_t grid = 0;
  SB_TRY(part_grid(reinterpret_cast<const void*>(k), f, 256, smem, ntiles - done, &grid));
  k<<<(unsigned)grid, 256, smem, stream>>>(tmap, image, lay, N, M, ld, static_cast<TO*>(x), done, ntiles, nbox,
                                           box_rows, vec, delay_ns);
  return cuda_check(cudaGetLastError(), "partitioned solve launch");
}

template <typename TO, int PB>
int dispatch_l(const sb_factor* f, int v, const float* image, const CUtensorMap& tmap, void* x,
               int64_t M, int64_t ld, cudaStream_t stream) {
  const int L = f->part_L[v];
  if (v == 2) {
    switch (L) {
      case 16: return launch_part2<TO, PB, 16>(f, image, tmap, x, M, ld, stream);
      case 32: return launch_part2<TO, PB, 32>(f, image, tmap, x, M, ld, stream);
      case 64: return launch_part2<TO, PB, 64>(f, image, tmap, x, M, ld, stream);
      default: break;
    }
  } else if (v == 0) {
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

int part_variant(int threads) {
  return threads == 512 ? 0 : threads == 1024 ? 1 : threads == 256 ? 2 : -1;
}

bool partitioned_applies(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype,
                         sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith, int threads) {
  const int o = op == OP_PRIMAL ? 0 : 1, v = part_variant(threads);
  // M bounded so that every TMA x coordinate (tile * 32) fits in 32 bits
  return v >= 0 && arith == SB_ARITH_NATIVE && rhs_dtype == SB_F32 &&
         (x_dtype == SB_F32 || x_dtype == SB_F64) && f->part_img[o][v] != nullptr &&
         f->part_NL[v] == levels_for(part_chunks(v)) && M >= 1 && M <= (int64_t)INT32_MAX &&
         (reinterpret_cast<uintptr_t>(rhs) % 16) == 0 && ((ld * 4) % 16) == 0 &&
         ld * 4 < ((int64_t)1 << 40) && encode_fn() != nullptr;
}

int launch_partitioned(const sb_factor* f, Op op, const void* rhs, sb_dtype rhs_dtype, void* x,
                       sb_dtype x_dtype, int64_t M, int64_t ld, sb_arith arith,
                       const SweepShape& shape, cudaStream_t stream) {
  if (!partitioned_applies(f, op, rhs, rhs_dtype, x_dtype, M, ld, arith, shape.threads))
    return fail(SB_ERR_UNSUPPORTED, "the partitioned solve does not apply to this call");
  const int o = op == OP_PRIMAL ? 0 : 1, v = part_variant(shape.threads);
  CUtensorMap tmap;
  SB_TRY(encode_tile_map(&tmap, rhs, f->N, M, ld, box_rows_for(part_chunks(v), f->part_L[v])));
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
