// Host-side data of the partitioned solve (host C++ only, no CUDA).  The paper's
// solvers sweep each system sequentially, one thread per system; this partitioned
// form of the same solve (a SPIKE-type decomposition followed by parallel cyclic
// reduction, exact up to rounding) is this library's own, so that one CTA can keep
// a tile of systems on chip.
//
// Rows are cut into P chunks of L rows, chunk c = rows [cL, cL + L); rows >= N
// (when P L > N) are identity rows with a zero right-hand side, decoupled from A, so
// every chunk has exactly L rows.  With A_c the diagonal block of chunk c (half
// bandwidth PB):
//     x_c = A_c^{-1} b_c - W_c lam_c - V_c rho_c
// where lam_c are the last PB unknowns of chunk c-1, rho_c the first PB unknowns of
// chunk c+1, and the "spikes" W_c = A_c^{-1} Lc_c, V_c = A_c^{-1} Rc_c (L x PB) are
// A_c^{-1} applied to the coupling columns of A.  Because A is shared, the spikes
// and everything below depend on A only and are computed once here, in FP64.
//
// The unknowns z_k = (last PB of chunk k, first PB of chunk k+1), k = 0..K-1 with
// K = P - 1, satisfy a block-tridiagonal system with Q x Q blocks (Q = 2 PB):
//     Lo_k z_{k-1} + D_k z_k + Up_k z_{k+1} = r_k,   r_k = (tail of y_k, head of y_{k+1})
//     D_k  = [[I, Vb_k], [Wt_{k+1}, I]],  Lo_k = [[Wb_k, 0], [0, 0]],  Up_k = [[0, 0], [0, Vt_{k+1}]]
// (Wb/Vb: the last PB rows of W_k/V_k; Wt/Vt: the first PB rows of W_{k+1}/V_{k+1};
// y_c = A_c^{-1} b_c).  It is solved by parallel cyclic reduction.  Normalised,
//     z_k + a_k z_{k-1} + c_k z_{k+1} = d_k,   a_k = D_k^{-1} Lo_k, c_k = D_k^{-1} Up_k,
//     d_k = T0_k r_k with T0_k = D_k^{-1};
// a level with stride s replaces equation k by
//     G_k (eq_k - a_k eq_{k-s} - c_k eq_{k+s}),   G_k = (I - a_k c_{k-s} - c_k a_{k+s})^{-1},
// so that per system d_k <- M0_k d_k - M1_k d_{k-s}[0:PB] - M2_k d_{k+s}[PB:Q] with
// M0 = G, M1 = (G a_k)[:, 0:PB], M2 = (G c_k)[:, PB:Q] (a_k only has non-zero columns
// 0..PB-1 and c_k only PB..Q-1, at every level).  After NL levels (2^NL >= K) every
// coupling reaches outside 0..K-1 and z_k = d_k.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace sb {

struct Partition {
  int PB = 0, N = 0, L = 0, P = 0, NL = 0;
  // per padded row i < P L, local factor rows in the sweep kernels' format:
  // forward  u_i = F0 r_i - F1 u_{i-1} - F2 u_{i-2},  backward x_i = u_i - B1 x_{i+1} - B2 x_{i+2},
  // restarted at each chunk (coefficients reaching outside the chunk are 0)
  std::vector<double> fw;      // (PB+1) per row: F0, F1[, F2]
  std::vector<double> bw;      // PB per row: B1[, B2]
  std::vector<double> W, V;    // PB per row
  // reduced system, per boundary k < K: T0 (Q x Q); per level l and boundary k:
  // M0 (Q x Q), M1 (Q x PB), M2 (Q x PB); all row-major, k-major within a level
  std::vector<double> T0, M0, M1, M2;
  // the same reduced system factored for block Thomas (block LU without pivoting),
  // per boundary k: E_k = Lo_k G_{k-1}^{-1} (its first PB rows, PB x Q), H_k = G_k^{-1}
  // (Q x Q) and J_k = G_k^{-1} Up_k (its last PB columns, Q x PB), G_0 = D_0,
  // G_k = D_k - E_k Up_{k-1}; per system q_k = r_k - E_k q_{k-1} (rows 0..PB-1),
  // then z_{K-1} = H q, z_k = H_k q_k - J_k z_{k+1}[PB:Q]
  std::vector<double> E, H, J;
  int Q() const { return 2 * PB; }
  int K() const { return P - 1; }
};

namespace part_detail {

// Dense small-matrix inverse by Gauss-Jordan elimination with partial pivoting.
inline bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int pr = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r * n + c]) > std::fabs(a[pr * n + c])) pr = r;
    if (pr != c)
      for (int j = 0; j < n; ++j) {
        std::swap(a[c * n + j], a[pr * n + j]);
        std::swap(inv[c * n + j], inv[pr * n + j]);
      }
    const double piv = a[c * n + c];
    if (piv == 0.0 || !std::isfinite(piv)) return false;
    for (int j = 0; j < n; ++j) {
      a[c * n + j] /= piv;
      inv[c * n + j] /= piv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[r * n + j] -= f * a[c * n + j];
        inv[r * n + j] -= f * inv[c * n + j];
      }
    }
  }
  a = inv;
  return true;
}

inline std::vector<double> matmul(const std::vector<double>& a, const std::vector<double>& b, int n) {
  std::vector<double> c(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j) c[i * n + j] += a[i * n + k] * b[k * n + j];
  return c;
}

inline bool all_finite(const std::vector<double>& v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace part_detail

// diag: the 2PB+1 diagonals of A, diagonal-major (diag[k*N + i] is row i at offset k - PB),
// zero outside the matrix.  Chunks of L rows, P chunks (P L >= N, L >= PB).  Returns
// false on a zero pivot of a chunk or of the reduced system, or a non-finite value.
inline bool build_partition(int PB, int N, const double* diag, int L, int P, Partition& out) {
  using namespace part_detail;
  Partition& p = out;
  p = Partition();
  if (PB < 1 || PB > 2 || N < 1 || L < PB || P < 1 || (int64_t)P * L < N) return false;
  p.PB = PB;
  p.N = N;
  p.L = L;
  p.P = P;
  const int NP = P * L, Q = 2 * PB, W = PB + 1, K = P - 1;
  auto A = [&](int i, int j) -> double {  // entry (i, j) of A (0 outside)
    const int off = j - i;
    if (i < 0 || i >= N || j < 0 || j >= N || off < -PB || off > PB) return 0.0;
    return diag[(size_t)(off + PB) * N + i];
  };
  p.fw.assign((size_t)W * NP, 0.0);
  p.bw.assign((size_t)PB * NP, 0.0);
  p.W.assign((size_t)PB * NP, 0.0);
  p.V.assign((size_t)PB * NP, 0.0);
  for (int i = std::min(N, NP); i < NP; ++i) p.fw[(size_t)W * i] = 1.0;  // identity padding
  for (int c = 0; c < P; ++c) {
    const int s = c * L, e = std::min(c * L + L, N), n = e - s;
    if (n <= 0) continue;
    // factorisation of A_c: the pentadiagonal recurrence of section 4.1 (the
    // tridiagonal one of section 3.1 when PB = 1) restarted at row s, with the
    // entries outside the block dropped
    std::vector<double> al(n), be(n, 0.0), ga(n, 0.0), de(n, 0.0), ep(n, 0.0);
    for (int r = 0; r < n; ++r) {
      const int i = s + r;
      const double ai = (PB == 2 && r >= 2) ? A(i, i - 2) : 0.0;
      const double bi = (r >= 1) ? A(i, i - 1) : 0.0;
      const double di = (r + 1 < n) ? A(i, i + 1) : 0.0;
      const double ei = (PB == 2 && r + 2 < n) ? A(i, i + 2) : 0.0;
      const double g2 = r >= 2 ? ga[r - 2] : 0.0, d2 = r >= 2 ? de[r - 2] : 0.0;
      const double g1 = r >= 1 ? ga[r - 1] : 0.0, d1 = r >= 1 ? de[r - 1] : 0.0;
      be[r] = bi - ai * g2;
      al[r] = A(i, i) - ai * d2 - be[r] * g1;
      if (al[r] == 0.0 || !std::isfinite(al[r])) return false;
      ga[r] = (di - be[r] * d1) / al[r];
      de[r] = ei / al[r];
      ep[r] = ai;
      double* f = &p.fw[(size_t)W * i];
      f[0] = 1.0 / al[r];
      f[1] = be[r] / al[r];
      if (PB == 2) f[2] = ep[r] / al[r];
      p.bw[(size_t)PB * i] = ga[r];
      if (PB == 2) p.bw[(size_t)PB * i + 1] = de[r];
    }
    auto local_solve = [&](std::vector<double> v) {  // A_c^{-1} v
      std::vector<double> g(n);
      for (int r = 0; r < n; ++r) {
        const double t = v[r] - (r >= 1 ? be[r] * g[r - 1] : 0.0) - (r >= 2 ? ep[r] * g[r - 2] : 0.0);
        g[r] = t / al[r];
      }
      std::vector<double> x(n);
      for (int r = n - 1; r >= 0; --r)
        x[r] = g[r] - (r + 1 < n ? ga[r] * x[r + 1] : 0.0) - (r + 2 < n ? de[r] * x[r + 2] : 0.0);
      return x;
    };
    // spikes: the coupling columns to x_{s-PB+j} (left) and x_{s+L+j} (right), j < PB
    for (int j = 0; j < PB; ++j) {
      std::vector<double> lc(n, 0.0), rc(n, 0.0);
      for (int r = 0; r < n; ++r) {
        lc[r] = A(s + r, s - PB + j);
        rc[r] = A(s + r, s + L + j);
      }
      const std::vector<double> w = local_solve(lc), v = local_solve(rc);
      for (int r = 0; r < n; ++r) {
        p.W[(size_t)PB * (s + r) + j] = w[r];
        p.V[(size_t)PB * (s + r) + j] = v[r];
      }
    }
  }
  if (!all_finite(p.fw) || !all_finite(p.bw) || !all_finite(p.W) || !all_finite(p.V)) return false;
  // reduced system and its cyclic reduction
  p.NL = 0;
  while ((1 << p.NL) < K) ++p.NL;
  const size_t Kz = (size_t)std::max(K, 0);
  p.T0.assign(Kz * Q * Q, 0.0);
  p.M0.assign((size_t)p.NL * Kz * Q * Q, 0.0);
  p.M1.assign((size_t)p.NL * Kz * Q * PB, 0.0);
  p.M2.assign((size_t)p.NL * Kz * Q * PB, 0.0);
  std::vector<std::vector<double>> a(Kz, std::vector<double>(Q * Q, 0.0)), cc = a;
  p.E.assign(Kz * PB * Q, 0.0);
  p.H.assign(Kz * Q * Q, 0.0);
  p.J.assign(Kz * Q * PB, 0.0);
  std::vector<double> Ginv_prev, Up_prev;
  for (int k = 0; k < K; ++k) {
    const int ek = (k + 1) * L;  // first row of chunk k+1
    std::vector<double> D(Q * Q, 0.0), Lo(Q * Q, 0.0), Up(Q * Q, 0.0);
    for (int u = 0; u < PB; ++u) {
      const int rt = ek - PB + u, rh = ek + u;  // tail row of chunk k, head row of chunk k+1
      D[u * Q + u] = 1.0;
      D[(PB + u) * Q + PB + u] = 1.0;
      for (int v = 0; v < PB; ++v) {
        D[u * Q + PB + v] = p.V[(size_t)PB * rt + v];          // Vb_k
        D[(PB + u) * Q + v] = p.W[(size_t)PB * rh + v];        // Wt_{k+1}
        Lo[u * Q + v] = p.W[(size_t)PB * rt + v];              // Wb_k on z_{k-1}[0:PB]
        Up[(PB + u) * Q + PB + v] = p.V[(size_t)PB * rh + v];  // Vt_{k+1} on z_{k+1}[PB:Q]
      }
    }
    {  // block Thomas factors
      std::vector<double> G = D;
      if (k > 0) {
        const std::vector<double> Ek = matmul(Lo, Ginv_prev, Q), EU = matmul(Ek, Up_prev, Q);
        for (int t = 0; t < Q * Q; ++t) G[t] -= EU[t];
        for (int u = 0; u < PB; ++u)
          for (int v = 0; v < Q; ++v) p.E[((size_t)k * PB + u) * Q + v] = Ek[u * Q + v];
      }
      if (!invert(G, Q)) return false;
      const std::vector<double> GU = matmul(G, Up, Q);
      std::copy(G.begin(), G.end(), p.H.begin() + (size_t)k * Q * Q);
      for (int u = 0; u < Q; ++u)
        for (int v = 0; v < PB; ++v) p.J[((size_t)k * Q + u) * PB + v] = GU[u * Q + PB + v];
      Ginv_prev = G;
      Up_prev = Up;
    }
    if (!invert(D, Q)) return false;
    std::copy(D.begin(), D.end(), p.T0.begin() + (size_t)k * Q * Q);
    a[k] = matmul(D, Lo, Q);
    cc[k] = matmul(D, Up, Q);
  }
  for (int l = 0; l < p.NL; ++l) {
    const int s = 1 << l;
    std::vector<std::vector<double>> na(Kz, std::vector<double>(Q * Q, 0.0)), nc = na;
    for (int k = 0; k < K; ++k) {
      std::vector<double> S(Q * Q, 0.0);
      for (int i = 0; i < Q; ++i) S[i * Q + i] = 1.0;
      if (k - s >= 0) {
        const std::vector<double> t = matmul(a[k], cc[k - s], Q);
        for (int i = 0; i < Q * Q; ++i) S[i] -= t[i];
      }
      if (k + s < K) {
        const std::vector<double> t = matmul(cc[k], a[k + s], Q);
        for (int i = 0; i < Q * Q; ++i) S[i] -= t[i];
      }
      if (!invert(S, Q)) return false;  // S now holds G
      const std::vector<double> Ga = matmul(S, a[k], Q), Gc = matmul(S, cc[k], Q);
      const size_t b0 = ((size_t)l * K + k) * Q * Q, b1 = ((size_t)l * K + k) * Q * PB;
      std::copy(S.begin(), S.end(), p.M0.begin() + b0);
      for (int i = 0; i < Q; ++i)
        for (int j = 0; j < PB; ++j) {
          p.M1[b1 + i * PB + j] = Ga[i * Q + j];
          p.M2[b1 + i * PB + j] = Gc[i * Q + PB + j];
        }
      if (k - s >= 0) {
        const std::vector<double> t = matmul(Ga, a[k - s], Q);
        for (int i = 0; i < Q * Q; ++i) na[k][i] = -t[i];
      }
      if (k + s < K) {
        const std::vector<double> t = matmul(Gc, cc[k + s], Q);
        for (int i = 0; i < Q * Q; ++i) nc[k][i] = -t[i];
      }
    }
    a = na;
    cc = nc;
  }
  return all_finite(p.T0) && all_finite(p.M0) && all_finite(p.M1) && all_finite(p.M2) &&
         all_finite(p.E) && all_finite(p.H) && all_finite(p.J);
}

// Reference application of the partitioned solve to one right-hand side (length N),
// in FP64 and in the order of operations of the device kernels (host tests); the
// boundary system by cyclic reduction, or by block Thomas when `thomas`.
inline void partition_solve_ref(const Partition& p, const double* b, double* x, bool thomas = false) {
  const int PB = p.PB, P = p.P, L = p.L, Q = 2 * PB, W = PB + 1, K = P - 1, NP = P * L;
  std::vector<double> y(NP, 0.0);
  for (int i = 0; i < p.N; ++i) y[i] = b[i];
  for (int c = 0; c < P; ++c) {
    const int s = c * L, e = s + L;
    double u1 = 0, u2 = 0;
    for (int i = s; i < e; ++i) {
      const double* f = &p.fw[(size_t)W * i];
      double t = y[i] * f[0];
      if (PB == 2) t = std::fma(-f[2], u2, t);
      const double u = std::fma(-f[1], u1, t);
      y[i] = u;
      u2 = u1;
      u1 = u;
    }
    double x1 = 0, x2 = 0;
    for (int i = e - 1; i >= s; --i) {
      const double* g = &p.bw[(size_t)PB * i];
      double t = y[i];
      if (PB == 2) t = std::fma(-g[1], x2, t);
      const double v = std::fma(-g[0], x1, t);
      y[i] = v;
      x2 = x1;
      x1 = v;
    }
  }
  std::vector<double> d((size_t)std::max(K, 0) * Q, 0.0);
  if (thomas) {
    for (int k = 0; k < K; ++k) {  // q_k = r_k - E_k q_{k-1}
      const int ek = (k + 1) * L;
      double q[4];
      for (int u = 0; u < PB; ++u) {
        q[u] = y[ek - PB + u];
        q[PB + u] = y[ek + u];
      }
      if (k > 0)
        for (int u = 0; u < PB; ++u)
          for (int t = 0; t < Q; ++t)
            q[u] = std::fma(-p.E[((size_t)k * PB + u) * Q + t], d[(size_t)(k - 1) * Q + t], q[u]);
      for (int u = 0; u < Q; ++u) d[(size_t)k * Q + u] = q[u];
    }
    for (int k = K - 1; k >= 0; --k) {  // z_k = H_k q_k - J_k z_{k+1}[PB:Q]
      double z[4];
      for (int u = 0; u < Q; ++u) {
        double t = 0;
        for (int v = 0; v < Q; ++v) t = std::fma(p.H[((size_t)k * Q + u) * Q + v], d[(size_t)k * Q + v], t);
        if (k + 1 < K)
          for (int v = 0; v < PB; ++v)
            t = std::fma(-p.J[((size_t)k * Q + u) * PB + v], d[(size_t)(k + 1) * Q + PB + v], t);
        z[u] = t;
      }
      for (int u = 0; u < Q; ++u) d[(size_t)k * Q + u] = z[u];
    }
  } else {
  for (int k = 0; k < K; ++k) {
    const int ek = (k + 1) * L;
    double r[4];
    for (int u = 0; u < PB; ++u) {
      r[u] = y[ek - PB + u];
      r[PB + u] = y[ek + u];
    }
    for (int i = 0; i < Q; ++i) {
      double t = 0;
      for (int j = 0; j < Q; ++j) t = std::fma(p.T0[((size_t)k * Q + i) * Q + j], r[j], t);
      d[(size_t)k * Q + i] = t;
    }
  }
  for (int l = 0; l < p.NL; ++l) {
    const int s = 1 << l;
    std::vector<double> nd(d.size(), 0.0);
    for (int k = 0; k < K; ++k) {
      const size_t b0 = ((size_t)l * K + k) * Q * Q, b1 = ((size_t)l * K + k) * Q * PB;
      for (int i = 0; i < Q; ++i) {
        double t = 0;
        for (int j = 0; j < Q; ++j) t = std::fma(p.M0[b0 + i * Q + j], d[(size_t)k * Q + j], t);
        if (k - s >= 0)
          for (int j = 0; j < PB; ++j) t = std::fma(-p.M1[b1 + i * PB + j], d[(size_t)(k - s) * Q + j], t);
        if (k + s < K)
          for (int j = 0; j < PB; ++j) t = std::fma(-p.M2[b1 + i * PB + j], d[(size_t)(k + s) * Q + PB + j], t);
        nd[(size_t)k * Q + i] = t;
      }
    }
    d = nd;
  }
  }
  for (int c = 0; c < P; ++c) {
    const int s = c * L;
    double lam[2] = {0, 0}, rho[2] = {0, 0};
    if (c > 0)
      for (int u = 0; u < PB; ++u) lam[u] = d[(size_t)(c - 1) * Q + u];
    if (c < K)
      for (int u = 0; u < PB; ++u) rho[u] = d[(size_t)c * Q + PB + u];
    for (int i = s; i < s + L && i < p.N; ++i) {
      double v = y[i];
      for (int u = 0; u < PB; ++u) {
        v = std::fma(-p.W[(size_t)PB * i + u], lam[u], v);
        v = std::fma(-p.V[(size_t)PB * i + u], rho[u], v);
      }
      x[i] = v;
    }
  }
}

// Device image of a partition, rounded to FP32 and staged into shared memory by the
// partitioned kernel.  Sections, each starting on a multiple of 4 elements:
//   fwd  P L rows of FW = (PB == 2 ? 4 : 2) values: F0, F1[, F2, 0]
//   bwd  P L rows of PB values: B1[, B2]
//   cor  P L rows of Q values: W_0[, W_1], V_0[, V_1]
//   T0   Q*Q entries x P boundary slots (entry-major, boundary fastest; slots >= K are 0)
//   M    per level: M0 (Q*Q entries), M1 (Q*PB), M2 (Q*PB), each x P boundary slots
// The boundary-fastest order lets lane k of a warp read boundary k's entries
// without bank conflicts.
struct PartLayout {
  int fwd, bwd, cor, T0, M, total;
};

inline int round4(int v) { return (v + 3) & ~3; }

inline PartLayout part_layout(int PB, int L, int P, int NL) {
  const int Q = 2 * PB, FW = PB == 2 ? 4 : 2, NP = P * L;
  PartLayout l;
  int o = 0;
  l.fwd = o;
  o = round4(o + NP * FW);
  l.bwd = o;
  o = round4(o + NP * PB);
  l.cor = o;
  o = round4(o + NP * Q);
  l.T0 = o;
  o = round4(o + Q * Q * P);
  l.M = o;
  o += NL * (Q * Q + 2 * Q * PB) * P;
  l.total = round4(o);
  return l;
}

inline std::vector<double> partition_image(const Partition& p) {
  const int PB = p.PB, W = PB + 1, FW = PB == 2 ? 4 : 2, Q = 2 * PB, K = p.K(), P = p.P;
  const int NP = P * p.L;
  const PartLayout l = part_layout(p.PB, p.L, P, p.NL);
  std::vector<double> img(l.total, 0.0);
  for (int i = 0; i < NP; ++i) {
    for (int k = 0; k < W; ++k) img[l.fwd + i * FW + k] = p.fw[(size_t)W * i + k];
    for (int k = 0; k < PB; ++k) {
      img[l.bwd + i * PB + k] = p.bw[(size_t)PB * i + k];
      img[l.cor + i * Q + k] = p.W[(size_t)PB * i + k];
      img[l.cor + i * Q + PB + k] = p.V[(size_t)PB * i + k];
    }
  }
  for (int k = 0; k < K; ++k)
    for (int e = 0; e < Q * Q; ++e) img[l.T0 + e * P + k] = p.T0[(size_t)k * Q * Q + e];
  const int per_level = (Q * Q + 2 * Q * PB) * P;
  for (int lv = 0; lv < p.NL; ++lv) {
    const int base = l.M + lv * per_level;
    for (int k = 0; k < K; ++k) {
      const size_t b0 = ((size_t)lv * K + k) * Q * Q, b1 = ((size_t)lv * K + k) * Q * PB;
      for (int e = 0; e < Q * Q; ++e) img[base + e * P + k] = p.M0[b0 + e];
      for (int e = 0; e < Q * PB; ++e) {
        img[base + (Q * Q + e) * P + k] = p.M1[b1 + e];
        img[base + (Q * Q + Q * PB + e) * P + k] = p.M2[b1 + e];
      }
    }
  }
  return img;
}

// The same image with the rows of each pair of chunks (2w, 2w + 1) interleaved, for
// the kernel whose warp w holds both chunks (half a warp each): in the fwd, bwd and
// cor sections row j of chunk c sits at padded row (c / 2) 2L + 2j + c % 2, so the
// two half-warps read neighbouring records; the reduction sections are unchanged.
// Needs an even number of chunks.
inline std::vector<double> partition_image_paired(const Partition& p) {
  const PartLayout l = part_layout(p.PB, p.L, p.P, p.NL);
  const std::vector<double> plain = partition_image(p);
  std::vector<double> img = plain;
  const int FW = p.PB == 2 ? 4 : 2, Q = 2 * p.PB, L = p.L;
  for (int c = 0; c < p.P; ++c)
    for (int j = 0; j < L; ++j) {
      const int from = c * L + j, to = (c / 2) * 2 * L + 2 * j + c % 2;
      for (int e = 0; e < FW; ++e) img[l.fwd + to * FW + e] = plain[l.fwd + from * FW + e];
      for (int e = 0; e < p.PB; ++e) img[l.bwd + to * p.PB + e] = plain[l.bwd + from * p.PB + e];
      for (int e = 0; e < Q; ++e) img[l.cor + to * Q + e] = plain[l.cor + from * Q + e];
    }
  return img;
}

// Diagonals of A^T in the same diagonal-major format: A^T(i, i+o) = A(i+o, i).
inline std::vector<double> transpose_diagonals(int PB, int N, const double* diag) {
  std::vector<double> t((size_t)(2 * PB + 1) * N, 0.0);
  for (int o = -PB; o <= PB; ++o)
    for (int i = 0; i < N; ++i) {
      const int j = i + o;
      if (j >= 0 && j < N) t[(size_t)(o + PB) * N + i] = diag[(size_t)(PB - o) * N + j];
    }
  return t;
}

// FP64 image for the small-tile FP64 kernel (scalar records, both forms of the
// boundary solve: block Thomas factors and the cyclic-reduction matrices).
// Sections, each starting on a multiple of 4 elements:
//   fwd  P L rows of FW = (PB == 2 ? 4 : 2): F0, F1[, F2, 0];  bwd  P L rows of PB: B1[, B2]
//   cor  P L rows of Q: W_0[, W_1], V_0[, V_1]
//   E    K x PB x Q;  H  K x Q x Q;  J  K x Q x PB  (row-major, boundary-major)
//   T0, M  as in PartLayout (entry-major, P boundary slots, NL levels)
struct PartLayoutT {
  int fwd, bwd, cor, E, H, J, T0, M, total;
};

inline PartLayoutT part_layout_thomas(int PB, int L, int P, int NL) {
  const int Q = 2 * PB, FW = PB == 2 ? 4 : 2, NP = P * L, K = P - 1;
  PartLayoutT l;
  int o = 0;
  l.fwd = o;
  o = round4(o + NP * FW);
  l.bwd = o;
  o = round4(o + NP * PB);
  l.cor = o;
  o = round4(o + NP * Q);
  l.E = o;
  o = round4(o + K * PB * Q);
  l.H = o;
  o = round4(o + K * Q * Q);
  l.J = o;
  o = round4(o + K * Q * PB);
  l.T0 = o;
  o = round4(o + Q * Q * P);
  l.M = o;
  o += NL * (Q * Q + 2 * Q * PB) * P;
  l.total = round4(o);
  return l;
}

inline std::vector<double> partition_image_thomas(const Partition& p) {
  const int PB = p.PB, W = PB + 1, FW = PB == 2 ? 4 : 2, Q = 2 * PB, NP = p.P * p.L;
  const PartLayoutT l = part_layout_thomas(PB, p.L, p.P, p.NL);
  std::vector<double> img(l.total, 0.0);
  for (int i = 0; i < NP; ++i) {
    for (int k = 0; k < W; ++k) img[l.fwd + i * FW + k] = p.fw[(size_t)W * i + k];
    for (int k = 0; k < PB; ++k) {
      img[l.bwd + i * PB + k] = p.bw[(size_t)PB * i + k];
      img[l.cor + i * Q + k] = p.W[(size_t)PB * i + k];
      img[l.cor + i * Q + PB + k] = p.V[(size_t)PB * i + k];
    }
  }
  std::copy(p.E.begin(), p.E.end(), img.begin() + l.E);
  std::copy(p.H.begin(), p.H.end(), img.begin() + l.H);
  std::copy(p.J.begin(), p.J.end(), img.begin() + l.J);
  // the cyclic-reduction sections, laid out as in partition_image
  const std::vector<double> pcr = partition_image(p);
  const PartLayout lp = part_layout(PB, p.L, p.P, p.NL);
  std::copy(pcr.begin() + lp.T0, pcr.begin() + lp.total, img.begin() + l.T0);
  return img;
}

}  // namespace sb
