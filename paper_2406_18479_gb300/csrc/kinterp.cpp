// Wannier-like k-space interpolation (Sec. 2.5): X(R) = (1/N_k) sum_k X(k) e^{-i k R} on the mesh,
// X(k') = sum_R w_R X(R) e^{i k' R} anywhere. Both sums are linear in X, so
//   X(k') = sum_k T(k', k) X(k),   T(k', k) = (1/N_k) sum_R w_R e^{i (k' - k) R},
// T (nkf x nk, small) is built on the host and applied to every element of X by one FP64
// complex GEMM over k. R runs over the lattice vectors nearest the origin, R_d in
// [-N_d/2, N_d/2], the two boundary vectors of an even N_d sharing one term (weight 1/2 each),
// which makes the interpolation exact on the mesh and keeps X(-k) = X(k)^dagger symmetric.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <vector>

#include "gw_internal.h"

using namespace gwi;

namespace {

// (R, weight) along one direction of an N-point mesh
std::vector<std::pair<int, double>> axis_vectors(int n) {
  std::vector<std::pair<int, double>> a;
  if (n % 2 == 1) {
    for (int r = -(n / 2); r <= n / 2; ++r) a.push_back({r, 1.0});
  } else {
    for (int r = -(n / 2) + 1; r < n / 2; ++r) a.push_back({r, 1.0});
    a.push_back({-(n / 2), 0.5});
    a.push_back({n / 2, 0.5});
  }
  return a;
}

}  // namespace

extern "C" {

int gw_k_interpolate(const int nk3[3], const gw_c128* X_dev, long long nelem, int nkf, const double* f_host,
                     gw_c128* Xf_dev, void* cuda_stream) {
  if (!nk3 || !X_dev || !Xf_dev || (nkf > 0 && !f_host) || nelem < 0 || nkf < 0)
    return fail(GW_EINVAL, "gw_k_interpolate: bad argument");
  if (nk3[0] < 1 || nk3[1] < 1 || nk3[2] < 1 || (long long)nk3[0] * nk3[1] * nk3[2] > 4096 || nelem > (1LL << 30))
    return fail(GW_EINVAL, "gw_k_interpolate: sizes out of range");
  if (nkf == 0 || nelem == 0) return GW_OK;
  const int nk = nk3[0] * nk3[1] * nk3[2];
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // T(k', k) = (1/N_k) prod_d sum_{R_d} w e^{2 pi i (f'_d - f_d) R_d}: the R sum factorises by direction
  std::vector<std::vector<std::pair<int, double>>> ax(3);
  for (int d = 0; d < 3; ++d) ax[d] = axis_vectors(nk3[d]);
  std::vector<gw_c128> T((size_t)nkf * nk);
  for (int a = 0; a < nkf; ++a)
    for (int k = 0; k < nk; ++k) {
      const int n[3] = {k / (nk3[1] * nk3[2]), (k / nk3[2]) % nk3[1], k % nk3[2]};
      std::complex<double> t = 1.0 / nk;
      for (int d = 0; d < 3; ++d) {
        const double df = f_host[3 * a + d] - (double)n[d] / nk3[d];
        std::complex<double> s = 0.0;
        for (const auto& rw : ax[d]) {
          const double ph = 2.0 * M_PI * df * rw.first;
          s += rw.second * std::complex<double>(std::cos(ph), std::sin(ph));
        }
        t *= s;
      }
      T[(size_t)a * nk + k] = gw_c128{t.real(), t.imag()};
    }
  double2* Td = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&Td), T.size() * sizeof(double2), st) != cudaSuccess) {
    cudaGetLastError();
    return fail(GW_ENOMEM, "gw_k_interpolate: device allocation failed");
  }
  int rc = GW_OK;
  if (cudaMemcpyAsync(Td, T.data(), T.size() * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = fail(GW_ECUDA, "gw_k_interpolate: copy");
  // Xf[k'][e] = sum_k T[k'][k] X[k][e], in column blocks of at most 2^30 / 32 elements per launch
  const long long nb = 1LL << 24;
  for (long long e0 = 0; rc == GW_OK && e0 < nelem; e0 += nb) {
    ZGemm g;
    g.M = nkf;
    g.N = (int)std::min(nb, nelem - e0);
    g.K = nk;
    g.A = Td;
    g.va.rs_in = nk;
    g.va.ks_in = 1;
    g.B = reinterpret_cast<const double2*>(X_dev) + e0;
    g.vb.rs_in = 1;
    g.vb.ks_in = nelem;
    g.C = reinterpret_cast<double2*>(Xf_dev) + e0;
    g.vc.rs_in = nelem;
    g.vc.ks_in = 1;
    g.slot = SLOT_ELEMENTWISE;
    rc = zgemm_fp64(g, st);
  }
  cudaFreeAsync(Td, st);
  return rc;
}

}  // extern "C"
