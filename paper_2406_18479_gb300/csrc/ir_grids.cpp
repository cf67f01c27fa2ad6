// Intermediate-representation (IR) tau grids and transforms, built on the host.
//
// The logistic kernel K(x, y) = exp(-Lambda y (x + 1) / 2) / (1 + exp(-Lambda y)) (x = 2 tau /
// beta - 1, y = omega / omega_max, Lambda = beta omega_max) has the singular value expansion
// K = sum_l s_l U_l(x) V_l(y); the IR basis is u_l(tau) = sqrt(2 / beta) U_l(x) for the L
// functions with s_l / s_0 > eps. Steps:
//   1. K on composite 16-point Gauss-Legendre panels (x refined towards +-1, y towards 0), with
//      square roots of the weights on both sides, so that its SVD gives U_l at the x nodes;
//   2. the SVD through a randomised range (k columns, k above the rank at 1e-16) and one-sided
//      Jacobi on the k x ny projection; parity U_l(-x) = (-1)^l U_l(x) imposed, U_l(1) > 0;
//   3. U_l as a Legendre series on every panel;
//   4. tau nodes: the L roots of U_L, mirrored exactly;
//   5. Matsubara samples: where the non-vanishing part of u^_L(i nu_n) changes sign (n >= 0, the
//      side of smaller magnitude), mirrored, trimmed or padded to the library's symmetric count
//      (padding: a gap's log-midpoint or half again beyond the last, the candidate with the
//      smallest ||F||_F ||F^+||_F); u^_l(i nu) through int P_m(t) e^{i kappa t} dt = 2 i^m j_m(kappa);
//   6. F = u^(samples) U_tau^{-1}, B its least-squares left inverse; for the bosonic set the
//      mirror symmetry F[nw-1-n][L-1-t] = F[n][t] (and the same for B) is imposed exactly.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#include "gw_internal.h"

namespace gwi {
namespace {

using cd = std::complex<double>;
constexpr int kNgl = 16;

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), p0 = 1, p1 = z, dp = 1;
    for (int it = 0; it < 100; ++it) {
      p0 = 1.0;
      p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    p0 = 1.0;
    p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;                                   // ascending
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void legendre_values(double t, double* P) {
  P[0] = 1.0;
  P[1] = t;
  for (int m = 1; m + 1 < kNgl; ++m) P[m + 1] = ((2 * m + 1) * t * P[m] - m * P[m - 1]) / (m + 1);
}

// j_m(kappa), m = 0..kNgl-1: upward recurrence above the order, Miller's downward recurrence below
void spherical_bessel(double k, double* j) {
  const double ak = std::fabs(k);
  if (ak < 1e-8) {
    j[0] = 1.0;
    for (int m = 1; m < kNgl; ++m) j[m] = 0.0;
    return;
  }
  if (ak > kNgl) {
    j[0] = std::sin(ak) / ak;
    j[1] = std::sin(ak) / (ak * ak) - std::cos(ak) / ak;
    for (int m = 1; m + 1 < kNgl; ++m) j[m + 1] = (2 * m + 1) / ak * j[m] - j[m - 1];
  } else {
    const int top = kNgl + 30 + (int)ak;           // ak <= kNgl: top + 2 <= 64
    double f[64] = {0.0};
    f[top + 1] = 0.0;
    f[top] = 1e-280;
    for (int m = top; m >= 1; --m) {
      f[m - 1] = (2 * m + 1) / ak * f[m] - f[m + 1];
      if (std::fabs(f[m - 1]) > 1e250) {   // rescale
        for (int q = m - 1; q <= top + 1; ++q) f[q] *= 1e-250;
      }
    }
    const double j0 = std::sin(ak) / ak, j1 = std::sin(ak) / (ak * ak) - std::cos(ak) / ak;
    const double scale = std::fabs(j0) > std::fabs(j1) ? j0 / f[0] : j1 / f[1];
    for (int m = 0; m < kNgl; ++m) j[m] = f[m] * scale;
  }
  if (k < 0)
    for (int m = 1; m < kNgl; m += 2) j[m] = -j[m];
}

double logistic(double x, double y, double lam) {
  if (y >= 0) return std::exp(-0.5 * lam * y * (x + 1.0)) / (1.0 + std::exp(-lam * y));
  return std::exp(0.5 * lam * y * (1.0 - x)) / (1.0 + std::exp(lam * y));
}

struct IrBasis {
  std::vector<double> edges;   // x panels
  int L = 0;
  std::vector<double> c;       // [panel][m][l], l = 0..L
  int nl = 0;                  // L + 1

  double eval(int l, double x) const {
    const int np = (int)edges.size() - 1;
    int p = (int)(std::upper_bound(edges.begin(), edges.end(), x) - edges.begin()) - 1;
    p = std::max(0, std::min(np - 1, p));
    const double a = edges[p], b = edges[p + 1], t = (2 * x - a - b) / (b - a);
    double P[kNgl];
    legendre_values(t, P);
    double s = 0;
    for (int m = 0; m < kNgl; ++m) s += c[((size_t)p * kNgl + m) * nl + l] * P[m];
    return s;
  }

  // int_{-1}^{1} e^{i nb (x + 1) / 2} U_l(x) dx for l in [0, lmax]
  void fourier(double nb, int lmax, cd* out) const {
    for (int l = 0; l <= lmax; ++l) out[l] = 0.0;
    double j[kNgl];
    for (size_t p = 0; p + 1 < edges.size(); ++p) {
      const double a = edges[p], b = edges[p + 1];
      const double kappa = nb * (b - a) / 4.0, ph = nb * ((a + b) / 2.0 + 1.0) / 2.0;
      spherical_bessel(kappa, j);
      const cd phase(std::cos(ph), std::sin(ph));
      cd I[kNgl];
      cd im(1.0, 0.0);
      for (int m = 0; m < kNgl; ++m) {
        I[m] = 2.0 * im * j[m] * ((b - a) / 2.0) * phase;
        im *= cd(0.0, 1.0);
      }
      for (int m = 0; m < kNgl; ++m) {
        const double* cm = &c[((size_t)p * kNgl + m) * nl];
        for (int l = 0; l <= lmax; ++l) out[l] += I[m] * cm[l];
      }
    }
  }
};

// Randomised SVD of the weighted kernel: U_l at the x nodes (nx x nl, l = 0..L) and s.
bool build_basis(double lam, double eps, IrBasis& B) {
  const int J = (int)std::ceil(std::log2(std::max(lam, 2.0))) + 1;
  std::vector<double> ex = {-1.0, 0.0, 1.0}, ey = {0.0};
  for (int j = 1; j <= J; ++j) {
    ex.push_back(1.0 - std::ldexp(1.0, -j));
    ex.push_back(-(1.0 - std::ldexp(1.0, -j)));
  }
  for (int j = 0; j <= J; ++j) {
    ey.push_back(std::ldexp(1.0, -j));
    ey.push_back(-std::ldexp(1.0, -j));
  }
  std::sort(ex.begin(), ex.end());
  ex.erase(std::unique(ex.begin(), ex.end()), ex.end());
  std::sort(ey.begin(), ey.end());
  ey.erase(std::unique(ey.begin(), ey.end()), ey.end());
  std::vector<double> gt, gw;
  gauss_legendre(kNgl, gt, gw);
  auto nodes = [&](const std::vector<double>& e, std::vector<double>& x, std::vector<double>& w) {
    for (size_t p = 0; p + 1 < e.size(); ++p)
      for (int i = 0; i < kNgl; ++i) {
        x.push_back(0.5 * (e[p + 1] - e[p]) * (gt[i] + 1.0) + e[p]);
        w.push_back(0.5 * (e[p + 1] - e[p]) * gw[i]);
      }
  };
  std::vector<double> x, wx, y, wy;
  nodes(ex, x, wx);
  nodes(ey, y, wy);
  const int nx = (int)x.size(), ny = (int)y.size();
  std::vector<double> A((size_t)nx * ny);
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) A[(size_t)i * ny + j] = std::sqrt(wx[i]) * logistic(x[i], y[j], lam) * std::sqrt(wy[j]);
  // range: Y = A Omega, k columns (deterministic Gaussian-like draws), orthonormalised twice
  const int k = std::min({nx, ny, 40 + (int)(35.0 * std::log10(std::max(lam, 10.0)))});
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto uni = [&]() {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  };
  std::vector<double> Om((size_t)ny * k);
  for (auto& v : Om) v = std::sqrt(-2.0 * std::log(uni())) * std::cos(2.0 * M_PI * uni());
  std::vector<double> Q((size_t)nx * k, 0.0);
  for (int i = 0; i < nx; ++i)
    for (int j = 0; j < ny; ++j) {
      const double a = A[(size_t)i * ny + j];
      for (int c = 0; c < k; ++c) Q[(size_t)i * k + c] += a * Om[(size_t)j * k + c];
    }
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < k; ++c) {
      for (int d = 0; d < c; ++d) {
        double s = 0;
        for (int i = 0; i < nx; ++i) s += Q[(size_t)i * k + d] * Q[(size_t)i * k + c];
        for (int i = 0; i < nx; ++i) Q[(size_t)i * k + c] -= s * Q[(size_t)i * k + d];
      }
      double n2 = 0;
      for (int i = 0; i < nx; ++i) n2 += Q[(size_t)i * k + c] * Q[(size_t)i * k + c];
      const double n = std::sqrt(n2);
      if (!(n > 0)) return false;
      for (int i = 0; i < nx; ++i) Q[(size_t)i * k + c] /= n;
    }
  // W = (Q^T A)^T (ny x k): one-sided Jacobi orthogonalises its columns, V (k x k) collects the
  // rotations; Q^T A = V S W'^T, so the left singular vectors of A are Q V
  std::vector<double> W((size_t)ny * k, 0.0), V((size_t)k * k, 0.0);
  for (int i = 0; i < nx; ++i)
    for (int c = 0; c < k; ++c) {
      const double q = Q[(size_t)i * k + c];
      if (q == 0) continue;
      for (int j = 0; j < ny; ++j) W[(size_t)j * k + c] += q * A[(size_t)i * ny + j];
    }
  for (int c = 0; c < k; ++c) V[(size_t)c * k + c] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        double alpha = 0, beta = 0, gamma = 0;
        for (int j = 0; j < ny; ++j) {
          const double a = W[(size_t)j * k + p], b = W[(size_t)j * k + q];
          alpha += a * a;
          beta += b * b;
          gamma += a * b;
        }
        if (gamma == 0 || std::fabs(gamma) <= 1e-17 * std::sqrt(alpha * beta)) continue;
        off = std::max(off, std::fabs(gamma) / std::sqrt(alpha * beta));
        const double zeta = (beta - alpha) / (2 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1 + zeta * zeta));
        const double cs = 1 / std::sqrt(1 + t * t), sn = cs * t;
        for (int j = 0; j < ny; ++j) {
          const double a = W[(size_t)j * k + p], b = W[(size_t)j * k + q];
          W[(size_t)j * k + p] = cs * a - sn * b;
          W[(size_t)j * k + q] = sn * a + cs * b;
        }
        for (int r = 0; r < k; ++r) {
          const double a = V[(size_t)r * k + p], b = V[(size_t)r * k + q];
          V[(size_t)r * k + p] = cs * a - sn * b;
          V[(size_t)r * k + q] = sn * a + cs * b;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> s(k);
  for (int c = 0; c < k; ++c) {
    double n2 = 0;
    for (int j = 0; j < ny; ++j) n2 += W[(size_t)j * k + c] * W[(size_t)j * k + c];
    s[c] = std::sqrt(n2);
  }
  std::vector<int> ord(k);
  for (int c = 0; c < k; ++c) ord[c] = c;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return s[a] > s[b]; });
  if (!(s[ord[0]] > 0)) return false;
  int L = 0;
  while (L < k && s[ord[L]] / s[ord[0]] > eps) ++L;
  if (L + 1 > k || s[ord[k - 1]] / s[ord[0]] > 1e-14) return false;   // the range missed part of the basis
  B.L = L;
  B.nl = L + 1;
  B.edges = ex;
  // U_l at the nodes: (Q V)[:, ord[l]] / sqrt(wx), parity, sign
  std::vector<double> U((size_t)nx * B.nl);
  for (int l = 0; l <= L; ++l)
    for (int i = 0; i < nx; ++i) {
      double u = 0;
      for (int c = 0; c < k; ++c) u += Q[(size_t)i * k + c] * V[(size_t)c * k + ord[l]];
      U[(size_t)i * B.nl + l] = u / std::sqrt(wx[i]);
    }
  for (int l = 0; l <= L; ++l) {
    const double sg = U[(size_t)(nx - 1) * B.nl + l] < 0 ? -1.0 : 1.0;
    const double par = (l % 2) ? -1.0 : 1.0;
    for (int i = 0; i < nx / 2; ++i) {
      const double a = sg * U[(size_t)i * B.nl + l], b = sg * U[(size_t)(nx - 1 - i) * B.nl + l];
      U[(size_t)i * B.nl + l] = 0.5 * (a + par * b);
      U[(size_t)(nx - 1 - i) * B.nl + l] = 0.5 * (b + par * a);
    }
  }
  // Legendre coefficients per panel
  const int np = (int)ex.size() - 1;
  B.c.assign((size_t)np * kNgl * B.nl, 0.0);
  for (int p = 0; p < np; ++p)
    for (int i = 0; i < kNgl; ++i) {
      double P[kNgl];
      legendre_values(gt[i], P);
      for (int m = 0; m < kNgl; ++m) {
        const double f = (2 * m + 1) / 2.0 * gw[i] * P[m];
        for (int l = 0; l <= L; ++l) B.c[((size_t)p * kNgl + m) * B.nl + l] += f * U[((size_t)p * kNgl + i) * B.nl + l];
      }
    }
  return true;
}

// roots of U_l on (-1, 1), ascending, mirrored exactly
std::vector<double> roots(const IrBasis& B, int l) {
  std::vector<double> xs;
  for (size_t p = 0; p + 1 < B.edges.size(); ++p)
    for (int i = 0; i < 64; ++i) xs.push_back(B.edges[p] + (B.edges[p + 1] - B.edges[p]) * i / 64.0);
  xs.push_back(1.0);
  std::vector<double> v(xs.size()), out;
  for (size_t i = 0; i < xs.size(); ++i) v[i] = B.eval(l, xs[i]);
  for (size_t i = 0; i + 1 < xs.size(); ++i) {
    if (!((v[i] < 0 && v[i + 1] > 0) || (v[i] > 0 && v[i + 1] < 0))) continue;
    double a = xs[i], b = xs[i + 1], fa = v[i];
    for (int it = 0; it < 60; ++it) {
      const double m = 0.5 * (a + b), fm = B.eval(l, m);
      if ((fm < 0) == (fa < 0)) {
        a = m;
        fa = fm;
      } else {
        b = m;
      }
    }
    out.push_back(0.5 * (a + b));
  }
  const size_t n = out.size();
  std::vector<double> sym(n);
  for (size_t i = 0; i < n; ++i) sym[i] = 0.5 * (out[i] - out[n - 1 - i]);
  return sym;
}

// real Gauss-Jordan inverse with partial pivoting (n x n, row-major)
bool invert(std::vector<double> a, int n, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    if (!(std::fabs(a[(size_t)p * n + c]) > 0)) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)p * n + j], a[(size_t)c * n + j]);
        std::swap(inv[(size_t)p * n + j], inv[(size_t)c * n + j]);
      }
    const double d = a[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      a[(size_t)c * n + j] /= d;
      inv[(size_t)c * n + j] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)r * n + j] -= f * a[(size_t)c * n + j];
        inv[(size_t)r * n + j] -= f * inv[(size_t)c * n + j];
      }
    }
  }
  return true;
}

// ||F||_F ||F^+||_F of an nw x L transform (the padding criterion); +inf when F^+ does not exist
double conditioning(const std::vector<cd>& F, int nw, int L) {
  std::vector<cd> Fp;
  if (nw >= L) {
    if (!lsq_left_inverse(F, nw, L, Fp)) return INFINITY;
  } else {   // fewer rows than columns: the same product through the transpose
    std::vector<cd> Ft((size_t)L * nw);
    for (int r = 0; r < nw; ++r)
      for (int c = 0; c < L; ++c) Ft[(size_t)c * nw + r] = F[(size_t)r * L + c];
    if (!lsq_left_inverse(Ft, L, nw, Fp)) return INFINITY;
  }
  double a = 0, b = 0;
  for (const cd& v : F) a += std::norm(v);
  for (const cd& v : Fp) b += std::norm(v);
  return std::sqrt(a * b);
}

// Matsubara samples, F and B of one statistics (stat 0 bosonic, 1 fermionic) on the tau nodes
// whose basis values inverse is Uinv (L x L)
bool stat_grid(const IrBasis& B, double lam, double beta, int stat, const std::vector<double>& Uinv,
               std::vector<int64_t>& m, std::vector<cd>& F, std::vector<cd>& Bm) {
  const int L = B.L, nw = sample_count(L, stat);
  auto nub = [&](int64_t n) { return stat == 1 ? (2.0 * n + 1.0) * M_PI : 2.0 * n * M_PI; };
  // sign changes of the non-vanishing part of u^_L on n >= 0
  const int64_t nmax = (int64_t)std::ceil(4.0 * lam / (2.0 * M_PI)) + 2 * L;
  std::vector<cd> f(B.nl);
  std::vector<double> re(nmax), im(nmax);
  double mre = 0, mim = 0;
  for (int64_t n = 0; n < nmax; ++n) {
    B.fourier(nub(n), L, f.data());
    re[n] = f[L].real();
    im[n] = f[L].imag();
    mre = std::max(mre, std::fabs(re[n]));
    mim = std::max(mim, std::fabs(im[n]));
  }
  const std::vector<double>& g = mim > mre ? im : re;
  std::vector<int64_t> sel;
  for (int64_t i = 0; i + 1 < nmax; ++i)
    if ((g[i] < 0 && g[i + 1] > 0) || (g[i] > 0 && g[i + 1] < 0)) sel.push_back(std::fabs(g[i]) < std::fabs(g[i + 1]) ? i : i + 1);
  if (stat == 0) sel.push_back(0);
  std::sort(sel.begin(), sel.end());
  sel.erase(std::unique(sel.begin(), sel.end()), sel.end());
  auto full = [&](const std::vector<int64_t>& s) {
    std::vector<int64_t> o;
    for (int64_t k : s) {
      o.push_back(k);
      o.push_back(stat == 1 ? -k - 1 : -k);
    }
    std::sort(o.begin(), o.end());
    o.erase(std::unique(o.begin(), o.end()), o.end());
    return o;
  };
  auto transform = [&](const std::vector<int64_t>& mm, std::vector<cd>& T) {
    const int n = (int)mm.size();
    T.assign((size_t)n * L, 0.0);
    std::vector<cd> u(B.nl);
    for (int r = 0; r < n; ++r) {
      B.fourier(nub(mm[r]), L - 1, u.data());
      for (int j = 0; j < L; ++j) {
        cd acc = 0;
        for (int l = 0; l < L; ++l) acc += u[l] * Uinv[(size_t)l * L + j];
        T[(size_t)r * L + j] = std::sqrt(beta / 2.0) * acc;      // u^_l = sqrt(2 / beta) (beta / 2) int ...
      }
    }
  };
  m = full(sel);
  while ((int)m.size() > nw) {
    sel.pop_back();
    m = full(sel);
  }
  std::vector<cd> T;
  while ((int)m.size() < nw) {
    std::vector<int64_t> pos;
    for (int64_t k : sel)
      if (k > 0) pos.push_back(k);
    if (pos.empty()) pos.push_back(0);
    std::vector<int64_t> cands;
    for (size_t i = 0; i + 1 < pos.size(); ++i)
      if (pos[i + 1] - pos[i] > 1)
        cands.push_back((int64_t)std::llround(std::sqrt((pos[i] + 1.0) * (pos[i + 1] + 1.0)) - 1.0));
    cands.push_back((int64_t)(1.5 * pos.back()) + 1);
    double best = INFINITY;
    int64_t pick = -1;
    for (int64_t cnd : cands) {
      if (std::find(sel.begin(), sel.end(), cnd) != sel.end()) continue;
      std::vector<int64_t> trial = sel;
      trial.push_back(cnd);
      std::sort(trial.begin(), trial.end());
      const std::vector<int64_t> mm = full(trial);
      transform(mm, T);
      const double cval = conditioning(T, (int)mm.size(), L);
      if (cval < best || (cval == best && cnd < pick)) {
        best = cval;
        pick = cnd;
      }
    }
    if (pick < 0) return false;
    sel.push_back(pick);
    std::sort(sel.begin(), sel.end());
    m = full(sel);
  }
  transform(m, F);
  // the bosonic set maps the mirrored node to the mirrored frequency: F[nw-1-n][L-1-t] = F[n][t]
  // holds to rounding amplified by U_tau^{-1}; impose it (and so for B) exactly
  auto mirror = [](std::vector<cd>& X, int r, int c) {
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < c; ++j) {
        const size_t a = (size_t)i * c + j, b = (size_t)(r - 1 - i) * c + (c - 1 - j);
        if (a < b) X[a] = X[b] = 0.5 * (X[a] + X[b]);
      }
  };
  if (stat == 0) mirror(F, nw, L);
  if (!lsq_left_inverse(F, nw, L, Bm)) return false;
  if (stat == 0) mirror(Bm, L, nw);
  return true;
}

}  // namespace
}  // namespace gwi

using namespace gwi;

extern "C" {

int gw_ir_grids(double beta, double lambda, double eps, int cap, int* ntau_out, double* tau_host, gw_c128* Fb_host,
                gw_c128* Bb_host, gw_c128* Ff_host, gw_c128* Bf_host, double* omega_b_host, double* omega_f_host) {
  if (!ntau_out || !(beta > 0) || !(lambda >= 1.0 && lambda <= 1e6) || !(eps >= 1e-15 && eps <= 1e-2) || cap < 0)
    return fail(GW_EINVAL, "gw_ir_grids: beta > 0, 1 <= lambda <= 1e6, 1e-15 <= eps <= 1e-2 required");
  *ntau_out = 0;
  IrBasis B;
  if (!build_basis(lambda, eps, B)) return fail(GW_EINVAL, "gw_ir_grids: the singular value expansion failed");
  const int L = B.L;
  *ntau_out = L;
  if (!tau_host) return GW_OK;                    // size query
  if (L > cap || !Fb_host || !Bb_host || !Ff_host || !Bf_host)
    return fail(GW_EINVAL, "gw_ir_grids: %d tau nodes do not fit the capacity %d", L, cap);
  const std::vector<double> x = roots(B, L);
  if ((int)x.size() != L) return fail(GW_EINVAL, "gw_ir_grids: U_L has %zu roots, not %d", x.size(), L);
  std::vector<double> Ut((size_t)L * L), Uinv;
  for (int j = 0; j < L; ++j)
    for (int l = 0; l < L; ++l) Ut[(size_t)j * L + l] = std::sqrt(2.0 / beta) * B.eval(l, x[j]);
  if (!invert(Ut, L, Uinv)) return fail(GW_EINVAL, "gw_ir_grids: singular sampling matrix");
  for (int stat = 0; stat < 2; ++stat) {
    std::vector<int64_t> m;
    std::vector<cd> F, Bm;
    if (!stat_grid(B, lambda, beta, stat, Uinv, m, F, Bm))
      return fail(GW_EINVAL, "gw_ir_grids: Matsubara sampling failed (statistics %d)", stat);
    gw_c128* Fo = stat == 0 ? Fb_host : Ff_host;
    gw_c128* Bo = stat == 0 ? Bb_host : Bf_host;
    double* wo = stat == 0 ? omega_b_host : omega_f_host;
    for (size_t i = 0; i < F.size(); ++i) Fo[i] = gw_c128{F[i].real(), F[i].imag()};
    for (size_t i = 0; i < Bm.size(); ++i) Bo[i] = gw_c128{Bm[i].real(), Bm[i].imag()};
    if (wo)
      for (size_t n = 0; n < m.size(); ++n) wo[n] = (stat == 1 ? 2.0 * m[n] + 1.0 : 2.0 * m[n]) * M_PI / beta;
  }
  for (int j = 0; j < L; ++j) tau_host[j] = 0.5 * beta * (x[j] + 1.0);
  return GW_OK;
}

}  // extern "C"
