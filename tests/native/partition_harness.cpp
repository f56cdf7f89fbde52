// Host build of the partitioned-solve data (paper_2107_05395_gb300/csrc/partition.h)
// for CPU unit tests (compiled by tests/test_partition_host.py).
#include <vector>

#include "../../paper_2107_05395_gb300/csrc/partition.h"

using namespace sb;

extern "C" {

// Solves A x_m = b_m (transpose = 0) or A^T x_m = b_m (transpose = 1) for the M
// systems of the interleaved array b (row i of system m at i * M + m) with P chunks
// of L rows.  diag: 2PB+1 diagonals, diagonal-major.  Returns the number of cyclic
// reduction levels, or -1 when the partition cannot be built.  thomas != 0 solves the
// boundary system with the block Thomas factors instead of cyclic reduction.
int h_partition_solve(int PB, int N, const double* diag, int L, int P, int transpose, long M,
                      const double* b, double* x, int thomas) {
  std::vector<double> dt;
  const double* d = diag;
  if (transpose) {
    dt = transpose_diagonals(PB, N, diag);
    d = dt.data();
  }
  Partition p;
  if (!build_partition(PB, N, d, L, P, p)) return -1;
  std::vector<double> bm(N), xm(N);
  for (long m = 0; m < M; ++m) {
    for (int i = 0; i < N; ++i) bm[i] = b[(long)i * M + m];
    partition_solve_ref(p, bm.data(), xm.data(), thomas != 0);
    for (int i = 0; i < N; ++i) x[(long)i * M + m] = xm[i];
  }
  return p.NL;
}

// The device image (partition_image) and its layout (6 ints: fwd, bwd, cor, T0, M,
// total).  Returns the image length, or -1 when it cannot be built / does not fit.
int h_partition_image(int PB, int N, const double* diag, int L, int P, double* out, int cap,
                      int* layout) {
  Partition p;
  if (!build_partition(PB, N, diag, L, P, p)) return -1;
  const PartLayout l = part_layout(PB, L, P, p.NL);
  const std::vector<double> img = partition_image(p);
  if ((int)img.size() != l.total || l.total > cap) return -1;
  for (int k = 0; k < l.total; ++k) out[k] = img[k];
  const int lv[6] = {l.fwd, l.bwd, l.cor, l.T0, l.M, l.total};
  for (int k = 0; k < 6; ++k) layout[k] = lv[k];
  return l.total;
}

// The paired image (partition_image_paired); same layout as h_partition_image.
int h_partition_image_paired(int PB, int N, const double* diag, int L, int P, double* out, int cap) {
  Partition p;
  if (!build_partition(PB, N, diag, L, P, p)) return -1;
  const std::vector<double> img = partition_image_paired(p);
  if ((int)img.size() > cap) return -1;
  for (size_t k = 0; k < img.size(); ++k) out[k] = img[k];
  return (int)img.size();
}

// The FP64 small-tile image: block-Thomas factors and cyclic-reduction sections;
// layout = fwd, bwd, cor, E, H, J, T0, M, total.
int h_partition_image_thomas(int PB, int N, const double* diag, int L, int P, double* out, int cap,
                             int* layout) {
  Partition p;
  if (!build_partition(PB, N, diag, L, P, p)) return -1;
  const PartLayoutT l = part_layout_thomas(PB, L, P, p.NL);
  const std::vector<double> img = partition_image_thomas(p);
  if ((int)img.size() != l.total || l.total > cap) return -1;
  for (int k = 0; k < l.total; ++k) out[k] = img[k];
  const int lv[9] = {l.fwd, l.bwd, l.cor, l.E, l.H, l.J, l.T0, l.M, l.total};
  for (int k = 0; k < 9; ++k) layout[k] = lv[k];
  return l.total;
}

}  // extern "C"
