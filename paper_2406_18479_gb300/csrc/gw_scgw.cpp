// The self-consistency loop of Sec. 2.4 on one context: static and dynamic (GW, GF2, or none for
// Hartree-Fock) self-energy,
// acceleration (iteration mixing, or DIIS with the difference or the commutator residual,
// Sec. 5.3), the chemical-potential search and
// the Dyson update, until max |Sigma_n - Sigma_{n-1}| < tol.
//
// The pair (Sigma^inf, Sigma~) lives in one buffer [nk][nao][nao] + [nk][ntau][nao][nao], so
// that mixing, DIIS and the stopping test act on it as one vector. Every step runs on the
// context's stream; the host only reads the norms and the particle counts that steer the loop.
#include <cuda_runtime.h>

#include <cmath>

#include "gw_internal.h"

using namespace gwi;

namespace gwi {

size_t scgw_device_bytes(const gw_config* cfg, const gw_scgw_options* opt) {
  const size_t nk = (size_t)cfg->nk[0] * cfg->nk[1] * cfg->nk[2], nao2 = (size_t)cfg->nao * cfg->nao;
  const size_t nall = nk * nao2 * (1 + (size_t)cfg->ntau);
  // Sigma_{n-1}, F_n, H + Sigma^inf, two flags
  size_t b = sizeof(gw_c128) * (2 * nall + nk * nao2) + 256;
  if (opt && opt->diis_size > 0) {
    // the subspace: outputs and residuals; the commutator variant's residuals live on the
    // fermionic samples, plus one buffer to compute them in
    const bool comm = opt->diis_kind == 1;
    const size_t nres = comm ? nk * (size_t)sample_count(cfg->ntau, 1) * nao2 : nall;
    b += sizeof(gw_c128) * ((size_t)opt->diis_size * (nall + nres) + (comm ? nres : 0)) +
         (kDotBlocks + 1) * sizeof(double);
  }
  return b;
}

}  // namespace gwi

extern "C" {

size_t gw_scgw_bytes(const gw_config* cfg, const gw_scgw_options* opt) {
  return cfg ? scgw_device_bytes(cfg, opt) : 0;
}

int gw_scgw(gw_ctx* ctx, const gw_c128* H_dev, gw_c128* G_dev, gw_c128* Sigma_dev, gw_c128* SigInf_dev,
            const gw_scgw_options* o, gw_scgw_result* res) {
  if (!ctx || !H_dev || !G_dev || !o || !res) return fail(GW_EINVAL, "gw_scgw: null argument");
  if (!(o->alpha > 0.0 && o->alpha < 2.0) || !(o->tol >= 0.0) || o->itermax < 1 || o->diis_size < 0 ||
      o->diis_size > 16 || (o->diis_size > 0 && o->diis_start < 2) || o->diis_kind < 0 || o->diis_kind > 1 ||
      o->method < 0 || o->method > 2 || o->resume < 0 || o->resume > 1 ||
      (o->resume && (!Sigma_dev || (o->static_part && !SigInf_dev))) ||
      (o->n_electrons > 0.0 && !(o->mu_lo < o->mu_hi && o->mu_tol > 0.0)))
    return fail(GW_EINVAL, "gw_scgw: options out of range");
  const CtxInfo ci = ctx_info(ctx);
  cudaStream_t st = (cudaStream_t)ci.stream;
  const long long nst = (long long)ci.nk * ci.nao * ci.nao, ndyn = nst * ci.ntau, nall = nst + ndyn;
  const long long off = o->static_part ? 0 : nst;   // the vector starts at Sigma^inf only when it is used
  const long long nvec = nall - off;
  const size_t cb = sizeof(double2);
  const bool comm = o->diis_size > 0 && o->diis_kind == 1;
  const long long nres = comm ? (long long)ci.nk * ci.nwf * ci.nao * ci.nao : 0;
  double2 *S = nullptr, *F = nullptr, *Heff = nullptr, *E = nullptr;
  void* flags = nullptr;
  gw_diis* diis = nullptr;
  auto cleanup = [&]() {
    if (diis) gw_diis_destroy(diis);
    cudaStreamSynchronize(st);
    for (void* p : {(void*)S, (void*)F, (void*)Heff, (void*)E, flags})
      if (p) cudaFree(p);
  };
  if (cudaMalloc((void**)&S, nall * cb) != cudaSuccess || cudaMalloc((void**)&F, nall * cb) != cudaSuccess ||
      cudaMalloc((void**)&Heff, nst * cb) != cudaSuccess || cudaMalloc(&flags, 16) != cudaSuccess ||
      (comm && cudaMalloc((void**)&E, nres * cb) != cudaSuccess)) {
    cleanup();
    return fail(GW_ENOMEM, "gw_scgw: device allocation failed");
  }
  double* maxdiff = reinterpret_cast<double*>(flags);
  int* nonfinite = reinterpret_cast<int*>(reinterpret_cast<char*>(flags) + 8);
  int rc = GW_OK;
  double d = 0.0, mu = ci.mu;
  int it = 1;
  bool converged = false;
  do {
    if (o->diis_size > 0 && (rc = gw_diis_create(&diis, nvec, nres, o->diis_size, st)) != GW_OK) break;
    if (!o->static_part) {
      cudaMemsetAsync(S, 0, nst * cb, st);
      cudaMemsetAsync(F, 0, nst * cb, st);
    }
    if (o->resume) {   // Sigma_{n-1} of the loop being continued
      cudaMemcpyAsync(S + nst, Sigma_dev, ndyn * cb, cudaMemcpyDeviceToDevice, st);
      if (o->static_part) cudaMemcpyAsync(S, SigInf_dev, nst * cb, cudaMemcpyDeviceToDevice, st);
    }
    for (it = 1; it <= o->itermax; ++it) {
      NvtxRange _nr("gw_scgw iteration");
      // (1) the output F_n of G_{n-1}
      if (o->static_part && (rc = gw_sigma_inf(ctx, G_dev, reinterpret_cast<gw_c128*>(F))) != GW_OK) break;
      if (o->method == 2)        // Hartree-Fock: no dynamic part
        rc = cudaMemsetAsync(F + nst, 0, ndyn * cb, st) == cudaSuccess ? GW_OK : fail(GW_ECUDA, "gw_scgw: memset");
      else if (o->method == 1)
        rc = gw_gf2_self_energy(ctx, G_dev, reinterpret_cast<gw_c128*>(F + nst));
      else
        rc = gw_sigma_eval(ctx, G_dev, reinterpret_cast<gw_c128*>(F + nst));
      if (rc != GW_OK) break;
      // (2) Sigma_n from F_n and the history
      if (it == 1 && !o->resume) {
        if (cudaMemcpyAsync(S, F, nall * cb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
          rc = fail(GW_ECUDA, "gw_scgw: copy");
          break;
        }
      } else {
        double alpha = o->alpha;
        if (comm) {
          // residual of G_{n-1} (still in G_dev) against its own output F_n
          if ((rc = gw_commutator_residual(ctx, H_dev, o->static_part ? reinterpret_cast<gw_c128*>(F) : nullptr,
                                           reinterpret_cast<gw_c128*>(F + nst), G_dev,
                                           reinterpret_cast<gw_c128*>(E))) != GW_OK ||
              (rc = gw_diis_push_residual(diis, reinterpret_cast<gw_c128*>(F + off), reinterpret_cast<gw_c128*>(E))) !=
                  GW_OK)
            break;
        } else if (diis) {
          if ((rc = gw_diis_push(diis, reinterpret_cast<gw_c128*>(S + off), reinterpret_cast<gw_c128*>(F + off))) !=
              GW_OK)
            break;
        }
        if (diis && it >= o->diis_start) {
          // the extrapolation replaces F_n and is taken whole (alpha = 1)
          if ((rc = gw_diis_extrapolate(diis, reinterpret_cast<gw_c128*>(F + off), nullptr, nullptr)) != GW_OK) break;
          alpha = 1.0;
        }
        cudaMemsetAsync(flags, 0, 16, st);
        if ((rc = mix_fp64(F + off, S + off, alpha, nvec, maxdiff, nonfinite, st)) != GW_OK) break;
        int bad = 0;
        if (cudaMemcpyAsync(&d, maxdiff, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&bad, nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          rc = fail(GW_ECUDA, "gw_scgw: norm");
          break;
        }
        if (bad) {
          rc = fail(GW_ENOTFINITE, "gw_scgw: non-finite self-energy at iteration %d", it);
          break;
        }
      }
      // (3), (4) mu and G_n from H + Sigma^inf_n and Sigma~_n
      const gw_c128* H = H_dev;
      if (o->static_part) {
        if ((rc = add_fp64(reinterpret_cast<const double2*>(H_dev), S, Heff, nst, st)) != GW_OK) break;
        H = reinterpret_cast<const gw_c128*>(Heff);
      }
      const gw_c128* Sd = reinterpret_cast<const gw_c128*>(S + nst);
      if (o->n_electrons > 0.0)
        rc = gw_find_mu(ctx, H, Sd, o->n_electrons, o->mu_lo, o->mu_hi, o->mu_tol, G_dev, &mu);
      else
        rc = gw_dyson_G(ctx, H, Sd, G_dev);
      if (rc != GW_OK) break;
      if ((it > 1 || o->resume) && d < o->tol) {
        converged = true;
        break;
      }
    }
    if (rc != GW_OK) break;
    res->iterations = converged ? it : o->itermax;
    res->max_abs_dsigma = d;
    res->mu = mu;
    if ((rc = gw_particle_number(ctx, G_dev, &res->n_electrons)) != GW_OK) break;
    if (Sigma_dev && cudaMemcpyAsync(Sigma_dev, S + nst, ndyn * cb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      rc = fail(GW_ECUDA, "gw_scgw: output copy");
      break;
    }
    if (SigInf_dev && cudaMemcpyAsync(SigInf_dev, S, nst * cb, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
      rc = fail(GW_ECUDA, "gw_scgw: output copy");
      break;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(GW_ECUDA, "gw_scgw: sync");
      break;
    }
    if (!converged) rc = fail(GW_ENOTCONV, "gw_scgw: no convergence in %d iterations", o->itermax);
  } while (false);
  cleanup();
  return rc;
}

}  // extern "C"
