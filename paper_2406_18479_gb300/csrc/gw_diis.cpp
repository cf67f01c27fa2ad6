// Pulay's direct inversion in the iterative subspace for the self-energy (Sec. 5.3).
//
// Each push stores the output Sigma[G_i] of an iteration and its residual, either
// r_i = Sigma[G_i] - Sigma_i (Sigma_i: the self-energy G_i was built from) or one the caller
// computed (the commutator variant passes [G_i(i w), H + Sigma[G_i](i w)]), and
// extends the matrix B_ij = Re <r_i, r_j> by one row from device reductions in a
// fixed order. Extrapolation solves the bordered system for the coefficients c
// minimising |sum_i c_i r_i|^2 with sum_i c_i = 1 (partial pivoting, on the host)
// and forms sum_i c_i Sigma[G_i] on the device. When the subspace is full the
// oldest vector leaves.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "gw_internal.h"

using namespace gwi;

struct gw_diis {
  cudaStream_t stream = nullptr;
  long long n = 0, nres = 0;     // elements of a self-energy vector and of a residual
  int max_vec = 0;
  std::vector<double2*> f, r;     // slots; order[] lists the live ones, oldest first
  std::vector<int> order;
  std::vector<double> B;          // [max_vec][max_vec] over slots
  double* scal = nullptr;         // reduction partials + one result
};

namespace {

int solve_bordered(const std::vector<double>& Bsub, int m, std::vector<double>& c) {
  // [B -1; -1 0] [c; l] = [0; -1]
  const int n = m + 1;
  std::vector<double> a((size_t)n * (n + 1), 0.0);
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) a[(size_t)i * (n + 1) + j] = Bsub[(size_t)i * m + j];
    a[(size_t)i * (n + 1) + m] = -1.0;
    a[(size_t)m * (n + 1) + i] = -1.0;
  }
  a[(size_t)m * (n + 1) + n] = -1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * (n + 1) + col]) > std::fabs(a[(size_t)piv * (n + 1) + col])) piv = i;
    if (!(std::fabs(a[(size_t)piv * (n + 1) + col]) > 0.0)) return fail(GW_ENOTFINITE, "gw_diis: singular subspace");
    if (piv != col)
      for (int j = 0; j <= n; ++j) std::swap(a[(size_t)col * (n + 1) + j], a[(size_t)piv * (n + 1) + j]);
    for (int i = 0; i < n; ++i) {
      if (i == col) continue;
      const double f = a[(size_t)i * (n + 1) + col] / a[(size_t)col * (n + 1) + col];
      for (int j = col; j <= n; ++j) a[(size_t)i * (n + 1) + j] -= f * a[(size_t)col * (n + 1) + j];
    }
  }
  c.assign(m, 0.0);
  for (int i = 0; i < m; ++i) c[i] = a[(size_t)i * (n + 1) + n] / a[(size_t)i * (n + 1) + i];
  for (double x : c)
    if (!std::isfinite(x)) return fail(GW_ENOTFINITE, "gw_diis: non-finite coefficients");
  return GW_OK;
}

}  // namespace

namespace {

// Takes the next slot (the oldest leaves when the subspace is full), stores the output there
// and has fill(r) write the residual; then adds its row of B.
template <class Fill>
int push_common(gw_diis* d, const gw_c128* sigma_out_dev, Fill fill) {
  int slot;
  if ((int)d->order.size() < d->max_vec) {
    std::vector<bool> used(d->max_vec, false);
    for (int s : d->order) used[s] = true;
    slot = 0;
    while (used[slot]) ++slot;
  } else {
    slot = d->order.front();
    d->order.erase(d->order.begin());
  }
  const double2* fo = reinterpret_cast<const double2*>(sigma_out_dev);
  if (cudaMemcpyAsync(d->f[slot], fo, d->n * sizeof(double2), cudaMemcpyDeviceToDevice, d->stream) != cudaSuccess)
    return fail(GW_ECUDA, "gw_diis_push: copy");
  const int rc = fill(d->r[slot]);
  if (rc != GW_OK) return rc;
  d->order.push_back(slot);
  for (int j : d->order) {
    const int r2 = dot_re_fp64(d->r[slot], d->r[j], d->nres, d->scal, d->scal + kDotBlocks, d->stream);
    if (r2 != GW_OK) return r2;
    double v = 0.0;
    if (cudaMemcpyAsync(&v, d->scal + kDotBlocks, sizeof(double), cudaMemcpyDeviceToHost, d->stream) != cudaSuccess ||
        cudaStreamSynchronize(d->stream) != cudaSuccess)
      return fail(GW_ECUDA, "gw_diis_push: reduction");
    d->B[(size_t)slot * d->max_vec + j] = d->B[(size_t)j * d->max_vec + slot] = v;
  }
  return GW_OK;
}

}  // namespace

extern "C" {

int gw_diis_create(gw_diis** out, long long n_elem, long long n_residual, int max_vectors, void* cuda_stream) {
  if (!out || n_elem < 1 || n_residual < 0 || max_vectors < 1 || max_vectors > 16)
    return fail(GW_EINVAL, "gw_diis_create: bad arguments");
  *out = nullptr;
  gw_diis* d = new gw_diis();
  d->stream = (cudaStream_t)cuda_stream;
  d->n = n_elem;
  d->nres = n_residual > 0 ? n_residual : n_elem;
  d->max_vec = max_vectors;
  d->f.assign(max_vectors, nullptr);
  d->r.assign(max_vectors, nullptr);
  d->B.assign((size_t)max_vectors * max_vectors, 0.0);
  bool ok = cudaMalloc(reinterpret_cast<void**>(&d->scal), (kDotBlocks + 1) * sizeof(double)) == cudaSuccess;
  for (int i = 0; i < max_vectors && ok; ++i)
    ok = cudaMalloc(reinterpret_cast<void**>(&d->f[i]), n_elem * sizeof(double2)) == cudaSuccess &&
         cudaMalloc(reinterpret_cast<void**>(&d->r[i]), d->nres * sizeof(double2)) == cudaSuccess;
  if (!ok) {
    gw_diis_destroy(d);
    return fail(GW_ENOMEM, "gw_diis_create: device allocation failed");
  }
  *out = d;
  return GW_OK;
}

int gw_diis_destroy(gw_diis* d) {
  if (!d) return GW_OK;
  if (d->stream) cudaStreamSynchronize(d->stream);
  for (double2* p : d->f)
    if (p) cudaFree(p);
  for (double2* p : d->r)
    if (p) cudaFree(p);
  if (d->scal) cudaFree(d->scal);
  delete d;
  return GW_OK;
}


int gw_diis_push(gw_diis* d, const gw_c128* sigma_in_dev, const gw_c128* sigma_out_dev) {
  if (!d || !sigma_in_dev || !sigma_out_dev) return fail(GW_EINVAL, "gw_diis_push: null argument");
  if (d->nres != d->n) return fail(GW_EINVAL, "gw_diis_push: this subspace takes explicit residuals");
  const double2* vv[2] = {reinterpret_cast<const double2*>(sigma_out_dev),
                          reinterpret_cast<const double2*>(sigma_in_dev)};
  return push_common(d, sigma_out_dev, [&](double2* r) {
    const double cc[2] = {1.0, -1.0};
    return lincomb_fp64(vv, cc, 2, r, d->n, d->stream);
  });
}

int gw_diis_push_residual(gw_diis* d, const gw_c128* sigma_out_dev, const gw_c128* residual_dev) {
  if (!d || !sigma_out_dev || !residual_dev) return fail(GW_EINVAL, "gw_diis_push_residual: null argument");
  return push_common(d, sigma_out_dev, [&](double2* r) {
    return cudaMemcpyAsync(r, residual_dev, d->nres * sizeof(double2), cudaMemcpyDeviceToDevice, d->stream) ==
                   cudaSuccess
               ? GW_OK
               : fail(GW_ECUDA, "gw_diis_push_residual: copy");
  });
}

int gw_diis_extrapolate(gw_diis* d, gw_c128* out_dev, double* coeffs_host, int* nvec_host) {
  if (!d || !out_dev) return fail(GW_EINVAL, "gw_diis_extrapolate: null argument");
  const int m = (int)d->order.size();
  if (m == 0) return fail(GW_EINVAL, "gw_diis_extrapolate: no vectors pushed");
  std::vector<double> Bsub((size_t)m * m), c;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Bsub[(size_t)i * m + j] = d->B[(size_t)d->order[i] * d->max_vec + d->order[j]];
  const int rc = solve_bordered(Bsub, m, c);
  if (rc != GW_OK) return rc;
  std::vector<const double2*> v(m);
  for (int i = 0; i < m; ++i) v[i] = d->f[d->order[i]];
  const int r2 = lincomb_fp64(v.data(), c.data(), m, reinterpret_cast<double2*>(out_dev), d->n, d->stream);
  if (r2 != GW_OK) return r2;
  if (coeffs_host)
    for (int i = 0; i < m; ++i) coeffs_host[i] = c[i];
  if (nvec_host) *nvec_host = m;
  return GW_OK;
}

}  // extern "C"
