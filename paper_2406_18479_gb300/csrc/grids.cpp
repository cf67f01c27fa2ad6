// Host-side construction of the Chebyshev tau grid and the tau <-> i w
// transform matrices (Fourier integral of Sec. 2.3, Eq. P0t_to_P0w, and its
// fermionic counterpart used by Eq. dyson).
//
// A function X(tau) on [0, beta] is represented by its Chebyshev interpolant
// through the first-kind nodes. F maps node values to the exact Fourier
// integrals of that interpolant at the sampled Matsubara frequencies; B is the
// least-squares left inverse of F (Householder QR), so B F = I.
//
// The Fourier integral of each Chebyshev polynomial is evaluated in the angle
// variable x = cos(theta):
//   int_{-1}^{1} T_l(x) e^{i a x} dx = int_0^pi cos(l theta) e^{i a cos theta} sin(theta) dtheta,
// whose integrand is entire; a composite 20-point Gauss-Legendre rule with
// panels spanning at most 8 radians of phase integrates it to rounding.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "gw_internal.h"

namespace gwi {

using cd = std::complex<double>;

int sample_count(int ntau, int stat) {
  if (ntau < 1 || (stat != 0 && stat != 1)) return -1;
  const bool want_odd = (stat == 0);
  return ((ntau % 2 == 1) == want_odd) ? ntau : ntau + 1;
}

// Sampled Matsubara indices, symmetric under w -> -w:
//   n <= 5: the n smallest |w|;
//   else M = n/3, core |w| <= w_M (bosonic m in [-M, M], fermionic [-M-1, M]),
//   K = (n - core)/2 tail points per side uniform in 1/m:
//   m_j = round_half_up(M (2K+3) / (2K+3-2j)), mirrored to -m_j - stat.
std::vector<int64_t> matsubara_indices(int n, int stat) {
  std::vector<int64_t> out;
  if (n <= 5) {
    // smallest |2m + stat|, symmetric pairs
    for (int64_t r = 0; (int)out.size() < n; ++r) {
      if (stat == 0) {
        if (r == 0) out.push_back(0);
        else { out.push_back(r); out.push_back(-r); }
      } else {
        out.push_back(r); out.push_back(-r - 1);
      }
    }
    out.resize(n);
  } else {
    const int64_t M = n / 3;
    for (int64_t m = -M - stat; m <= M; ++m) out.push_back(m);
    const int64_t K = (n - (int64_t)out.size()) / 2;
    for (int64_t j = 1; j <= K; ++j) {
      const int64_t num = M * (2 * K + 3), den = 2 * K + 3 - 2 * j;
      const int64_t t = (2 * num + den) / (2 * den);
      out.push_back(t);
      out.push_back(-t - stat);
    }
  }
  std::sort(out.begin(), out.end());
  return out;
}

static void gauss_legendre20(double* x, double* w) {
  const int n = 20;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1; p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1; p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Householder QR least-squares left inverse of A (m x n, m >= n, row-major).
bool lsq_left_inverse(const std::vector<cd>& A_in, int m, int n, std::vector<cd>& Binv) {
  std::vector<cd> A = A_in;                  // m x n
  std::vector<cd> Qt(m * (size_t)m, 0.0);    // accumulates Q^H, m x m
  for (int i = 0; i < m; ++i) Qt[(size_t)i * m + i] = 1.0;
  for (int j = 0; j < n; ++j) {
    double norm2 = 0;
    for (int i = j; i < m; ++i) norm2 += std::norm(A[(size_t)i * n + j]);
    double norm = std::sqrt(norm2);
    if (norm == 0) return false;
    cd x0 = A[(size_t)j * n + j];
    cd alpha = (std::abs(x0) > 0) ? -x0 / std::abs(x0) * norm : cd(-norm, 0);
    std::vector<cd> v(m - j);
    for (int i = j; i < m; ++i) v[i - j] = A[(size_t)i * n + j];
    v[0] -= alpha;
    double vn2 = 0;
    for (auto& e : v) vn2 += std::norm(e);
    if (vn2 == 0) continue;
    // H = I - 2 v v^H / (v^H v), applied from the left to A and Qt
    for (int c = j; c < n; ++c) {
      cd s = 0;
      for (int i = j; i < m; ++i) s += std::conj(v[i - j]) * A[(size_t)i * n + c];
      s *= 2.0 / vn2;
      for (int i = j; i < m; ++i) A[(size_t)i * n + c] -= v[i - j] * s;
    }
    for (int c = 0; c < m; ++c) {
      cd s = 0;
      for (int i = j; i < m; ++i) s += std::conj(v[i - j]) * Qt[(size_t)i * m + c];
      s *= 2.0 / vn2;
      for (int i = j; i < m; ++i) Qt[(size_t)i * m + c] -= v[i - j] * s;
    }
  }
  // Solve R B = Qt[:n, :]  (R upper triangular n x n in A)
  Binv.assign((size_t)n * m, 0.0);
  for (int c = 0; c < m; ++c) {
    for (int i = n - 1; i >= 0; --i) {
      cd s = Qt[(size_t)i * m + c];
      for (int k = i + 1; k < n; ++k) s -= A[(size_t)i * n + k] * Binv[(size_t)k * m + c];
      cd d = A[(size_t)i * n + i];
      if (std::abs(d) == 0) return false;
      Binv[(size_t)i * m + c] = s / d;
    }
  }
  return true;
}

int grid_build(int ntau, double beta, int stat, double* tau, int64_t* idx, gw_c128* F, gw_c128* B) {
  const int nw = sample_count(ntau, stat);
  if (nw < 0 || !(beta > 0) || ntau > 4096) return GW_EINVAL;
  const int N = ntau;
  std::vector<double> th(N), x(N);
  for (int j = 0; j < N; ++j) {
    th[j] = M_PI * (j + 0.5) / N;
    // x_j = 2 tau_j / beta - 1 = -cos(theta_j)
    x[j] = -std::cos(th[j]);
    if (tau) tau[j] = 0.5 * beta * (1.0 - std::cos(th[j]));
  }
  std::vector<int64_t> m = matsubara_indices(nw, stat);
  if (idx) for (int n = 0; n < nw; ++n) idx[n] = m[n];
  if (!F && !B) return GW_OK;
  // C[l][t] = (2 - delta_l0)/N T_l(x_t), T_l(x_t) = T_l(-cos th_t) = (-1)^l cos(l th_t)
  std::vector<double> C((size_t)N * N);
  for (int l = 0; l < N; ++l)
    for (int t = 0; t < N; ++t)
      C[(size_t)l * N + t] = (l == 0 ? 1.0 : 2.0) / N * ((l % 2) ? -1.0 : 1.0) * std::cos(l * th[t]);
  // T[n][l] = int_0^beta T_l(2 tau/beta - 1) e^{i w_n tau} dtau
  //         = (beta/2) e^{i a} int_{-1}^{1} T_l(x) e^{i a x} dx,  a = w_n beta / 2
  double gx[20], gwt[20];
  gauss_legendre20(gx, gwt);
  std::vector<cd> T((size_t)nw * N);
  for (int n = 0; n < nw; ++n) {
    const double a = 0.5 * (double)(2 * m[n] + stat) * M_PI;   // w_n beta / 2
    const double fastest = std::fabs(a) + N;                     // phase rate in theta
    // at most 8 radians of phase per 20-point panel: the rule's error is then below 1e-17
    const int panels = 4 + (int)std::ceil(fastest * M_PI / 8.0);
    const double h = M_PI / panels;
    std::vector<cd> acc(N, 0.0);
    for (int p = 0; p < panels; ++p) {
      for (int g = 0; g < 20; ++g) {
        const double t = h * (p + 0.5 * (gx[g] + 1.0));
        const double wq = 0.5 * h * gwt[g] * std::sin(t);
        const double ct = std::cos(t);
        const cd e = std::polar(wq, a * ct);
        double c0 = 1.0, c1 = ct;                 // cos(l t) by the Chebyshev recurrence
        acc[0] += e;
        if (N > 1) acc[1] += e * c1;
        for (int l = 2; l < N; ++l) {
          const double c2 = 2.0 * ct * c1 - c0;
          acc[l] += e * c2;
          c0 = c1; c1 = c2;
        }
      }
    }
    const cd pre = 0.5 * beta * std::polar(1.0, a);
    for (int l = 0; l < N; ++l) T[(size_t)n * N + l] = pre * acc[l];
  }
  std::vector<cd> Fm((size_t)nw * N, 0.0);
  for (int n = 0; n < nw; ++n)
    for (int l = 0; l < N; ++l) {
      const cd tnl = T[(size_t)n * N + l];
      for (int t = 0; t < N; ++t) Fm[(size_t)n * N + t] += tnl * C[(size_t)l * N + t];
    }
  if (F)
    for (size_t i = 0; i < Fm.size(); ++i) F[i] = gw_c128{Fm[i].real(), Fm[i].imag()};
  if (B) {
    std::vector<cd> Bm;
    if (!lsq_left_inverse(Fm, nw, N, Bm)) return GW_EINVAL;
    for (size_t i = 0; i < Bm.size(); ++i) B[i] = gw_c128{Bm[i].real(), Bm[i].imag()};
  }
  return GW_OK;
}

}  // namespace gwi
