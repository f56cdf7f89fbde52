// Per-tile body of the batched sweeps, shared by the single-factor and the
// multi-group kernels (see sweep.cu for the mapping and the memory scheme).
#pragma once

#include "arith.cuh"

namespace sb {

constexpr int kRows = 8;  // rows per prefetch batch

// Conversions between the storage types and an arithmetic policy's values.
template <class A, typename T>
struct Conv;

template <typename T>
struct Conv<NativeArith<T>, T> {
  static __device__ __forceinline__ T in(T v) { return v; }
  static __device__ __forceinline__ T out(T v) { return v; }
};
template <>
struct Conv<NativeArith<float>, double> {  // FP32 arithmetic on FP64 data
  // input: the FP64 value truncated to FP32 with integer operations (the leading
  // part of its double-float split; a refined solve corrects the rest)
  static __device__ __forceinline__ float in(double v) { return double_to_df(v).h; }
  static __device__ __forceinline__ double out(float v) { return widen_f32(v); }  // exact widening
};
template <>
struct Conv<DFArith, double> {
  static __device__ __forceinline__ df in(double v) { return double_to_df(v); }
  static __device__ __forceinline__ double out(df v) { return df_to_double(v); }
};
template <>
struct Conv<DFArith, float> {
  static __device__ __forceinline__ df in(float v) { return {v, 0.f}; }
};

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ void st_stream(T* p, T v) { __stcs(p, v); }

// Copies n coefficients into shared memory (all threads of the CTA take part).
template <typename C>
__device__ __forceinline__ void stage(C* dst, const C* __restrict__ src, int n) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = src[k];
}

// Per-lane asynchronous copies global -> shared (cp.async, 4 or 8 bytes), their
// commit groups, and the wait until at most K groups of this thread are pending.
__device__ __forceinline__ uint32_t shared_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  static_assert(B == 4 || B == 8, "per-lane copies of 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(shared_addr(dst)),
               "l"(__cvta_generic_to_global(src)), "n"(B)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

// Solves the tile `tile` (32 * SPT consecutive systems) with coefficient rows
// fw (forward) and bw (backward).  CYC = 1: the periodic tridiagonal matrix of
// section 3.3: rows cy = (w_i, -z_i) and scalars alpha, beta give the
// Sherman-Morrison correction x = y - f z, f = beta (w . rhs + alpha y_{N-1}),
// applied as x is written.  CYC = 2: the cyclic pentadiagonal matrix (rank-2
// correction): rows cy = (w0_i, w1_i, -z0_i, -z1_i) and, after the N rows, 12
// scalars P, Q, S^{-1}; g = S^{-1} (P (y_0, y_1) + Q (y_{N-2}, y_{N-1})) with
// y_0 = w0 . rhs and y_1 = w1 . rhs, x = y - z0 g_0 - z1 g_1; rows N-1 and N-2 are
// written once g is known.
//   forward  u_i = F0 r_i - F1 u_{i-1} - F2 u_{i-2}      (F0 == 1 when F_ONE)
//   backward x_i = B0 u_i - B1 x_{i+1} - B2 x_{i+2}      (B0 == 1 when B_ONE)
// The intermediate u is stored in place in x; SPT systems per thread (m and
// m + 32, ...) interleave independent recurrences; R rows per prefetch batch.
template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO, int SPT, int R,
          int CYC = 0>
__device__ __forceinline__ void sweep_tile(const typename A::C* fw, const typename A::C* bw, int N,
                                           int64_t M, int64_t ld, const TI* rhs, TO* x,
                                           int64_t tile, const typename A::C* cy = nullptr,
                                           typename A::C alpha = typename A::C(),
                                           typename A::C beta = typename A::C()) {
  using V = typename A::V;
  using C = typename A::C;
  using S = typename A::S;
  static_assert(sizeof(S) <= sizeof(TO), "intermediate must fit in an output element");
  constexpr int W = P + 1;
  const int lane = threadIdx.x & 31;
  do {
    const int64_t m0 = tile * (32 * SPT) + lane;
    if (m0 >= M) break;
    bool ok[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) ok[s] = (m0 + 32 * s) < M;
    const TI* r = rhs + m0;
    TO* y = x + m0;
    auto slot = [&](int i, int s) {
      return reinterpret_cast<S*>(y + (int64_t)i * ld + 32 * s);
    };

    // ---- forward sweep
    V u1[SPT], u2[SPT], dot[SPT], dot1[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) u1[s] = u2[s] = dot[s] = dot1[s] = A::zero();
    TI va[R][SPT], vb[R][SPT];
    auto load_in = [&](TI (&buf)[R][SPT], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j)
#pragma unroll
        for (int s = 0; s < SPT; ++s)
          if (i0 + j < N && ok[s]) buf[j][s] = ld_stream(r + (int64_t)(i0 + j) * ld + 32 * s);
    };
    auto fwd = [&](TI (&buf)[R][SPT], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int i = i0 + j;
        if (i < N) {
          const C* c = fw + W * i;
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            const V in = Conv<A, TI>::in(buf[j][s]);
            const V u = A::template step<P, F_ONE>(c, in, u1[s], u2[s]);
            if constexpr (CYC == 1) dot[s] = A::fmac(cy[2 * i], in, dot[s]);
            if constexpr (CYC == 2) {
              dot[s] = A::fmac(cy[4 * i], in, dot[s]);
              dot1[s] = A::fmac(cy[4 * i + 1], in, dot1[s]);
            }
            if (ok[s]) *slot(i, s) = A::to_store(u);
            u2[s] = u1[s];
            u1[s] = u;
          }
        }
      }
    };
    load_in(va, 0);
    for (int i0 = 0; i0 < N; i0 += 2 * R) {
      load_in(vb, i0 + R);
      fwd(va, i0);
      load_in(va, i0 + 2 * R);
      fwd(vb, i0 + R);
    }

    // ---- backward sweep
    V x1[SPT], x2[SPT], fc[SPT], g1[SPT];
#pragma unroll
    for (int s = 0; s < SPT; ++s) x1[s] = x2[s] = fc[s] = g1[s] = A::zero();
    S sa[R][SPT], sb_[R][SPT];
    auto load_mid = [&](S (&buf)[R][SPT], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j)
#pragma unroll
        for (int s = 0; s < SPT; ++s)
          if (i0 - j >= 0 && ok[s]) buf[j][s] = *slot(i0 - j, s);
    };
    auto bwd = [&](S (&buf)[R][SPT], int i0) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int i = i0 - j;
        if (i >= 0) {
          const C* c = bw + W * i;
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            const V xi = A::template step<P, B_ONE>(c, A::from_store(buf[j][s]), x1[s], x2[s]);
            if constexpr (CYC == 1) {
              if (i == N - 1) fc[s] = A::mulc(beta, A::fmac(alpha, xi, dot[s]));
              if (ok[s]) st_stream(y + (int64_t)i * ld + 32 * s, Conv<A, TO>::out(A::fmac(cy[2 * i + 1], fc[s], xi)));
            } else if constexpr (CYC == 2) {
              if (i < N - 2) {
                if (ok[s])
                  st_stream(y + (int64_t)i * ld + 32 * s,
                            Conv<A, TO>::out(A::fmac(cy[4 * i + 3], g1[s], A::fmac(cy[4 * i + 2], fc[s], xi))));
              } else if (i == N - 2) {
                // x1 holds y_{N-1}: g = S^{-1} (P (y_0, y_1) + Q (y_{N-2}, y_{N-1}))
                const C* sc = cy + 4 * N;
                const V yl = x1[s];
                const V t0 = A::fmac(sc[0], dot[s], A::fmac(sc[1], dot1[s], A::fmac(sc[4], xi, A::mulc(sc[5], yl))));
                const V t1 = A::fmac(sc[2], dot[s], A::fmac(sc[3], dot1[s], A::fmac(sc[6], xi, A::mulc(sc[7], yl))));
                fc[s] = A::fmac(sc[8], t0, A::mulc(sc[9], t1));
                g1[s] = A::fmac(sc[10], t0, A::mulc(sc[11], t1));
                if (ok[s]) {
                  const int j1 = N - 1;
                  st_stream(y + (int64_t)j1 * ld + 32 * s,
                            Conv<A, TO>::out(A::fmac(cy[4 * j1 + 3], g1[s], A::fmac(cy[4 * j1 + 2], fc[s], yl))));
                  st_stream(y + (int64_t)i * ld + 32 * s,
                            Conv<A, TO>::out(A::fmac(cy[4 * i + 3], g1[s], A::fmac(cy[4 * i + 2], fc[s], xi))));
                }
              }
            } else {
              if (ok[s]) st_stream(y + (int64_t)i * ld + 32 * s, Conv<A, TO>::out(xi));
            }
            x2[s] = x1[s];
            x1[s] = xi;
          }
        }
      }
    };
    load_mid(sa, N - 1);
    for (int i0 = N - 1; i0 >= 0; i0 -= 2 * R) {
      load_mid(sb_, i0 - R);
      bwd(sa, i0);
      load_mid(sa, i0 - 2 * R);
      bwd(sb_, i0 - R);
    }
  } while (false);
}

// The same sweeps (plain matrices, one system per thread) with both row streams
// staged through shared memory: a ring of D slots per thread (slot s of thread t at
// ring + (s * blockDim.x + t) * E, E = max(sizeof(TI), sizeof(S))) holds the next D
// rows of the right-hand side in the forward sweep and of the intermediate in the
// backward sweep, so the rows in flight cost shared memory instead of registers and
// a block can run more warps.  Each lane copies, and later reads, only its own
// system's values, so the thread's own cp.async.wait_group is the only ordering; a
// slot is refilled after the row read from it has been computed and stored.  Rows
// are taken K per wait.  Same arithmetic as sweep_tile with SPT = 1, CYC = 0.
template <typename TI, typename S>
__host__ __device__ constexpr int staged_slot_bytes() {
  return sizeof(TI) > sizeof(S) ? (int)sizeof(TI) : (int)sizeof(S);
}

template <class A, int P, bool F_ONE, bool B_ONE, typename TI, typename TO, int D, int K>
__device__ __forceinline__ void sweep_tile_staged(const typename A::C* fw, const typename A::C* bw, int N,
                                                  int64_t M, int64_t ld, const TI* rhs, TO* x, int64_t tile,
                                                  unsigned char* ring) {
  using V = typename A::V;
  using S = typename A::S;
  static_assert(sizeof(S) <= sizeof(TO), "intermediate must fit in an output element");
  static_assert((D & (D - 1)) == 0 && D % K == 0, "the ring length is a power of two and a multiple of K");
  constexpr int W = P + 1;
  constexpr int E = staged_slot_bytes<TI, S>();
  const int64_t m = tile * 32 + (threadIdx.x & 31);
  if (m >= M) return;
  const TI* r = rhs + m;
  TO* y = x + m;
  const int T = blockDim.x;
  unsigned char* mine = ring + (size_t)threadIdx.x * E;
  auto slot = [&](int k) { return mine + (size_t)(k & (D - 1)) * T * E; };
  __threadfence_block();  // this thread's stores of the previous tile before the copies below

  // ---- forward sweep: u_i from rhs_i, stored in place in x
  auto issue_f = [&](int k) {
    if (k < N) cp_async<sizeof(TI)>(slot(k), r + (int64_t)k * ld);
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue_f(k);
  V u1 = A::zero(), u2 = A::zero();
  for (int i0 = 0; i0 < N; i0 += K) {
    cp_wait<D - K>();  // the groups of rows i0 .. i0+K-1 are complete
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int i = i0 + j;
      if (i < N) {
        const V u = A::template step<P, F_ONE>(fw + W * i, Conv<A, TI>::in(*reinterpret_cast<const TI*>(slot(i))),
                                               u1, u2);
        *reinterpret_cast<S*>(y + (int64_t)i * ld) = A::to_store(u);
        u2 = u1;
        u1 = u;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) issue_f(i0 + D + j);
  }
  cp_wait<0>();           // every group left is empty (rows past N)
  __threadfence_block();  // the stores of u before the copies that read them back

  // ---- backward sweep: iteration k takes row i = N-1-k of u and writes x_i over it
  auto issue_b = [&](int k) {
    const int i = N - 1 - k;
    if (i >= 0) cp_async<sizeof(S)>(slot(k), reinterpret_cast<const S*>(y + (int64_t)i * ld));
    cp_commit();
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue_b(k);
  V x1 = A::zero(), x2 = A::zero();
  for (int k0 = 0; k0 < N; k0 += K) {
    cp_wait<D - K>();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int k = k0 + j;
      const int i = N - 1 - k;
      if (i >= 0) {
        const V xi = A::template step<P, B_ONE>(bw + W * i, A::from_store(*reinterpret_cast<const S*>(slot(k))),
                                                x1, x2);
        st_stream(y + (int64_t)i * ld, Conv<A, TO>::out(xi));
        x2 = x1;
        x1 = xi;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) issue_b(k0 + D + j);
  }
  cp_wait<0>();
}

}  // namespace sb
