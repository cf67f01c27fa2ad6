// C ABI of the GW self-energy library: context, grids, k-mesh gather tables
// and the FP64 stages (arXiv 2406.18479, Sec. 2.3 and Eq. dyson).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gw_internal.h"
#include "gw_mixed.h"

namespace gwi {

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

struct Prof {
  bool on = false;
  long long launches = 0;
  long long slot_launches[SLOT_COUNT] = {};
  double slot_flops[SLOT_COUNT] = {}, slot_bytes[SLOT_COUNT] = {}, slot_ms[SLOT_COUNT] = {};
  cudaEvent_t open[SLOT_COUNT] = {};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[SLOT_COUNT];
  std::vector<cudaEvent_t> pool;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (int s = 0; s < SLOT_COUNT; ++s) {
      for (auto& pr : pending[s]) {
        float ms = 0.f;
        cudaEventSynchronize(pr.second);
        cudaEventElapsedTime(&ms, pr.first, pr.second);
        slot_ms[s] += ms;
        pool.push_back(pr.first);
        pool.push_back(pr.second);
      }
      pending[s].clear();
    }
  }
  void reset() {
    drain();
    for (int s = 0; s < SLOT_COUNT; ++s) {
      slot_launches[s] = 0;
      slot_flops[s] = slot_bytes[s] = slot_ms[s] = 0.0;
    }
    launches = 0;
  }
  ~Prof() {
    drain();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

static thread_local Prof* t_prof = nullptr;

const char* prof_slot_name(int slot) {
  static const char* names[SLOT_COUNT] = {
      "vg_fp64", "p0_gemm_fp64", "r_gemm_fp64", "sigma_gemm_fp64", "transform_fp64", "inverse_fp64",
      "elementwise", "slice_planes", "vg_gemm_tc", "p0_gemm_tc", "r_gemm_tc", "sigma_gemm_tc", "reduce",
      "static_fp64", "gf2_exchange_fp64", "gf2_outer_tc"};
  return (slot >= 0 && slot < SLOT_COUNT) ? names[slot] : "";
}

void prof_begin(int slot, cudaStream_t s) {
  Prof* p = t_prof;
  if (!p) return;
  p->launches++;
  p->slot_launches[slot]++;
  if (p->on) {
    p->open[slot] = p->get();
    cudaEventRecord(p->open[slot], s);
  }
}

void prof_end(int slot, cudaStream_t s, double flops, double bytes) {
  Prof* p = t_prof;
  if (!p) return;
  p->slot_flops[slot] += flops;
  p->slot_bytes[slot] += bytes;
  if (p->on && p->open[slot]) {
    cudaEvent_t e = p->get();
    cudaEventRecord(e, s);
    p->pending[slot].push_back({p->open[slot], e});
    p->open[slot] = nullptr;
  }
}

struct ProfScope {
  Prof* saved;
  explicit ProfScope(Prof* p) : saved(t_prof) { t_prof = p; }
  ~ProfScope() { t_prof = saved; }
};

}  // namespace gwi

using namespace gwi;

struct gw_ctx {
  gw_config cfg{};
  cudaStream_t stream = nullptr;
  bool dry = false;                       // size-only build: count bytes, allocate and copy nothing
  int nk = 0, nao = 0, naux = 0, ntau = 0, nwb = 0, nwf = 0, nt = 1;
  long long nao2 = 0, naux2 = 0, pair = 0;
  double2 *Fb = nullptr, *Bb = nullptr, *Ff = nullptr, *Bf = nullptr;
  double* wf = nullptr;                   // fermionic frequencies (device)
  long long* tabs = nullptr;              // 6 tables [nq][nk]
  long long *tab_kkpq = nullptr, *tab_kpqk = nullptr, *tab_gkpq = nullptr;
  long long *tab_kkmq = nullptr, *tab_kmqk = nullptr, *tab_gkmq = nullptr;
  double2* work = nullptr;                // contraction intermediates, nt * 2 * nk * pair
  double2 *P0t = nullptr, *Pw = nullptr, *Pt = nullptr;
  double2* dyson_ws = nullptr;            // nk * nwf * nao2
  std::vector<int> mq;                    // index of -q for every q
  int* mq_dev = nullptr;
  int* wlist = nullptr;                   // canonical (q, n) matrices of P~(i Omega), as q * nwb + n
  int* wlist_q = nullptr;                 // (q, n) matrices of a q range (gw_sigma_eval_q)
  std::vector<int> wlist_host;            // host copy of wlist (the items of a grouped inversion)
  int nwlist = 0;
  int* status = nullptr;                  // device flags: [0] singular matrix
  double* maxdiff = nullptr;
  int* nonfinite = nullptr;
  const double2* V = nullptr;             // full-layout V: the caller's, or the unpacked copy Vfull
  const double2* Vp = nullptr;            // the caller's packed V (cfg.v_packed)
  double2* Vfull = nullptr;               // FP64 precision with a packed V: the full working copy
  bool coulomb = false;                   // gw_set_coulomb has been called
  size_t bytes = 0;
  MixedState* mixed = nullptr;
  // static part and loop helpers
  double* wbeta = nullptr;                // weights of the interpolant at tau = beta, [ntau]
  double2* gamma = nullptr;               // density matrix, [nk][nao][nao]
  double2* rho = nullptr;                 // Hartree density in the auxiliary basis, [naux]
  double2* xinf = nullptr;                // exchange intermediate of one k, [nk][naux][nao][nao]
  double2* gw_w = nullptr;                // G on the fermionic samples, [nk][nwf][nao][nao]
  double2* heff = nullptr;                // H + Sigma^inf, [nk][nao][nao]
  const double2* S = nullptr;             // overlap of Eq. dyson (borrowed; null: identity)
  double2* cw_tmp = nullptr;              // commutator with an overlap: one product, [nk][nwf][nao][nao]
  double2* gf2_ws = nullptr;              // GF2 exchange intermediates (allocated on first use)
  size_t gf2_n = 0;
  double* scal = nullptr;                 // reduction partials and results
  std::vector<unsigned char*> guards;     // guard zones of the workspaces allocated by dev_alloc
  Prof prof;
};

namespace {

int kshift(const int nk3[3], int k, int q, int sign) {
  const int k1 = k / (nk3[1] * nk3[2]), k2 = (k / nk3[2]) % nk3[1], k3 = k % nk3[2];
  const int q1 = q / (nk3[1] * nk3[2]), q2 = (q / nk3[2]) % nk3[1], q3 = q % nk3[2];
  const int a = ((k1 + sign * q1) % nk3[0] + nk3[0]) % nk3[0];
  const int b = ((k2 + sign * q2) % nk3[1] + nk3[1]) % nk3[1];
  const int c = ((k3 + sign * q3) % nk3[2] + nk3[2]) % nk3[2];
  return (a * nk3[1] + b) * nk3[2] + c;
}

template <class T>
int dev_alloc(gw_ctx* c, T** p, size_t count) {
  if (count == 0) count = 1;
  const size_t bytes = count * sizeof(T);
  if (c->dry) {
    *p = nullptr;
    c->bytes += bytes + kGuardBytes;
    return GW_OK;
  }
  const cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes + kGuardBytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(GW_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  unsigned char* guard = reinterpret_cast<unsigned char*>(*p) + bytes;
  cudaMemsetAsync(guard, kGuardByte, kGuardBytes, c->stream);   // ordered before the context's work
  c->guards.push_back(guard);
  c->bytes += bytes + kGuardBytes;
  return GW_OK;
}

// host -> device copy of a table; nothing in a size-only build
void upload(const gw_ctx* c, void* dst, const void* src, size_t bytes) {
  if (!c->dry) cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
}

int cuda_check(const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GW_TRY(x)                 \
  do {                            \
    const int _rc = (x);          \
    if (_rc != GW_OK) return _rc; \
  } while (0)

void free_ctx(gw_ctx* c) {
  if (!c) return;
  mixed_destroy(c->mixed);
  void* ptrs[] = {c->Fb, c->Bb, c->Ff, c->Bf, c->wf, c->tabs, c->mq_dev, c->wlist, c->wlist_q, c->work, c->P0t, c->Pw,
                  c->Pt, c->dyson_ws, c->status, c->maxdiff, c->nonfinite, c->wbeta, c->gamma, c->rho,
                  c->xinf, c->scal, c->gw_w, c->heff, c->gf2_ws, c->Vfull, c->cw_tmp};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

int upload_grid(gw_ctx* c, int stat, double2** F, double2** B, int* nw_out) {
  const int nw = sample_count(c->ntau, stat);
  std::vector<gw_c128> hF((size_t)nw * c->ntau), hB((size_t)c->ntau * nw);
  std::vector<int64_t> idx(nw);
  GW_TRY(grid_build(c->ntau, c->cfg.beta, stat, nullptr, idx.data(), hF.data(), hB.data()));
  GW_TRY(dev_alloc(c, F, hF.size()));
  GW_TRY(dev_alloc(c, B, hB.size()));
  upload(c, *F, hF.data(), hF.size() * sizeof(double2));
  upload(c, *B, hB.data(), hB.size() * sizeof(double2));
  if (stat == 1) {
    std::vector<double> w(nw);
    for (int n = 0; n < nw; ++n) w[n] = (2.0 * (double)idx[n] + 1.0) * M_PI / c->cfg.beta;
    GW_TRY(dev_alloc(c, &c->wf, nw));
    upload(c, c->wf, w.data(), nw * sizeof(double));
  }
  *nw_out = nw;
  return c->dry ? GW_OK : cuda_check("grid upload");
}

// ---- FP64 stages ------------------------------------------------------------------------

// Canonical tau range of q: all nodes if q < -q, the first half if q = -q, none if q > -q;
// the rest follows from P0^q(beta - tau) = P0^{-q}(tau)^T (mirror_fill).
int canonical_end(const gw_ctx* c, int q, int T) { return c->mq[q] < q ? 0 : (c->mq[q] == q ? (T + 1) / 2 : T); }

// The same within a q range [q0, q1): a q whose -q lies outside the range takes every index.
int canonical_end(const gw_ctx* c, int q, int T, int q0, int q1) {
  return (c->mq[q] < q0 || c->mq[q] >= q1) ? T : canonical_end(c, q, T);
}

int polarization_fp64(gw_ctx* c, const double2* G, double2* P0t, int q0, int q1) {
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau;
  const long long nao2 = c->nao2, pair = c->pair;
  for (int q = q0; q < q1; ++q) {
    const int tend = canonical_end(c, q, ntau, q0, q1);
    for (int t0 = 0; t0 < tend; t0 += c->nt) {
      const int nt = std::min(c->nt, tend - t0);
      double2* Abuf = c->work;
      double2* Bbuf = c->work + (long long)c->nt * nk * pair;
      {  // A^Q_{db}(k,t) = sum_a V^{k,k+q}_da(Q) G^{k+q}_ab(t)
        ZGemm g;
        g.M = naux * nao; g.N = nao; g.K = nao; g.nbatch = nt * nk; g.bin = nk;
        g.A = c->V; g.va.rs_in = nao; g.va.ks_in = 1; g.ba.tab = c->tab_kkpq + (long long)q * nk;
        g.B = G + (long long)t0 * nao2; g.vb.rs_in = 1; g.vb.ks_in = nao;
        g.bb.tab = c->tab_gkpq + (long long)q * nk; g.bb.bs_out = nao2;
        g.C = Abuf; g.vc.rs_in = nao; g.vc.ks_in = 1; g.bc.bs_in = pair; g.bc.bs_out = (long long)nk * pair;
        g.slot = SLOT_VG_FP64;
        GW_TRY(zgemm_fp64(g, c->stream));
      }
      {  // B^{Q'}_{bd}(k,t) = sum_c V^{k+q,k}_bc(Q') G^k_cd(beta - t), stored as [Q'][d][b]
        ZGemm g;
        g.M = naux * nao; g.N = nao; g.K = nao; g.nbatch = nt * nk; g.bin = nk;
        g.A = c->V; g.va.rs_in = nao; g.va.ks_in = 1; g.ba.tab = c->tab_kpqk + (long long)q * nk;
        g.B = G + (long long)(ntau - 1 - t0) * nao2; g.vb.rs_in = 1; g.vb.ks_in = nao;
        g.bb.bs_in = (long long)ntau * nao2; g.bb.bs_out = -nao2;
        g.C = Bbuf; g.vc.rin = nao; g.vc.rs_in = 1; g.vc.rs_out = nao2; g.vc.ks_in = nao;
        g.bc.bs_in = pair; g.bc.bs_out = (long long)nk * pair;
        g.slot = SLOT_VG_FP64;
        GW_TRY(zgemm_fp64(g, c->stream));
      }
      {  // P0^q_QQ'(t) = -(s/N_k) sum_{k,d,b} A^Q_{db} B^{Q'}_{bd}
        ZGemm g;
        g.M = naux; g.N = naux; g.K = nk * (int)nao2; g.nbatch = nt;
        g.A = Abuf; g.va.rs_in = nao2; g.va.kin = (int)nao2; g.va.ks_in = 1; g.va.ks_out = pair;
        g.ba.bs_in = (long long)nk * pair;
        g.B = Bbuf; g.vb = g.va; g.bb = g.ba;
        g.C = P0t + ((long long)q * ntau + t0) * c->naux2; g.vc.rs_in = naux; g.vc.ks_in = 1;
        g.bc.bs_in = c->naux2;
        g.alpha = -c->cfg.spin_factor / nk;
        g.slot = SLOT_P0_FP64;
        GW_TRY(zgemm_fp64(g, c->stream));
      }
    }
  }
  return GW_OK;
}

int self_energy_fp64(gw_ctx* c, const double2* G, const double2* Pt, double2* Sig, int q0, int q1) {
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau;
  const long long nao2 = c->nao2, pair = c->pair;
  if (cudaMemsetAsync(Sig, 0, (size_t)nk * ntau * nao2 * sizeof(double2), c->stream) != cudaSuccess)
    return cuda_check("memset Sigma");
  for (int q = q0; q < q1; ++q) {
    for (int t0 = 0; t0 < ntau; t0 += c->nt) {
      const int nt = std::min(c->nt, ntau - t0);
      double2* Rbuf = c->work;
      double2* Zbuf = c->work + (long long)c->nt * nk * pair;
      {  // R^Q_{bj}(k,t) = sum_Q' P~^q_QQ'(t) V^{k-q,k}_bj(Q')
        ZGemm g;
        g.M = naux; g.N = (int)nao2; g.K = naux; g.nbatch = nt * nk; g.bin = nk;
        g.A = Pt + ((long long)q * ntau + t0) * c->naux2; g.va.rs_in = naux; g.va.ks_in = 1;
        g.ba.bs_out = c->naux2;
        g.B = c->V; g.vb.rs_in = 1; g.vb.ks_in = nao2; g.bb.tab = c->tab_kmqk + (long long)q * nk;
        g.C = Rbuf; g.vc.rs_in = nao2; g.vc.ks_in = 1; g.bc.bs_in = pair; g.bc.bs_out = (long long)nk * pair;
        g.slot = SLOT_R_FP64;
        GW_TRY(zgemm_fp64(g, c->stream));
      }
      {  // Z^Q_{ib}(k,t) = sum_a V^{k,k-q}_ia(Q) G^{k-q}_ab(t)
        ZGemm g;
        g.M = naux * nao; g.N = nao; g.K = nao; g.nbatch = nt * nk; g.bin = nk;
        g.A = c->V; g.va.rs_in = nao; g.va.ks_in = 1; g.ba.tab = c->tab_kkmq + (long long)q * nk;
        g.B = G + (long long)t0 * nao2; g.vb.rs_in = 1; g.vb.ks_in = nao;
        g.bb.tab = c->tab_gkmq + (long long)q * nk; g.bb.bs_out = nao2;
        g.C = Zbuf; g.vc.rs_in = nao; g.vc.ks_in = 1; g.bc.bs_in = pair; g.bc.bs_out = (long long)nk * pair;
        g.slot = SLOT_VG_FP64;
        GW_TRY(zgemm_fp64(g, c->stream));
      }
      {  // Sigma^k_ij(t) += -(1/N_k) sum_{Q,b} Z^Q_{ib} R^Q_{bj}
        ZGemm g;
        g.M = nao; g.N = nao; g.K = naux * nao; g.nbatch = nt * nk; g.bin = nk;
        g.A = Zbuf; g.va.rs_in = nao; g.va.kin = nao; g.va.ks_in = 1; g.va.ks_out = nao2;
        g.ba.bs_in = pair; g.ba.bs_out = (long long)nk * pair;
        g.B = Rbuf; g.vb.rs_in = 1; g.vb.kin = nao; g.vb.ks_in = nao; g.vb.ks_out = nao2;
        g.bb = g.ba;
        g.C = Sig + (long long)t0 * nao2; g.vc.rs_in = nao; g.vc.ks_in = 1;
        g.bc.bs_in = (long long)ntau * nao2; g.bc.bs_out = nao2;
        g.alpha = -1.0 / nk;
        g.accumulate = 1;
        g.slot = SLOT_SIGMA_FP64;
        GW_TRY(zgemm_fp64(g, c->stream));
      }
    }
  }
  return GW_OK;
}

int transform(gw_ctx* c, int stat, bool forward, const double2* in, double2* out, int nbatch,
              long long nelem) {
  const int nw = stat == 0 ? c->nwb : c->nwf;
  const int nin = forward ? c->ntau : nw, nout = forward ? nw : c->ntau;
  const double2* Mtx = forward ? (stat == 0 ? c->Fb : c->Ff) : (stat == 0 ? c->Bb : c->Bf);
  if (nelem > (1LL << 30)) return fail(GW_EINVAL, "transform: nelem %lld too large", nelem);
  for (int b0 = 0; b0 < nbatch; b0 += 65535) {
    const int nb = std::min(65535, nbatch - b0);
    ZGemm g;
    g.M = nout; g.N = (int)nelem; g.K = nin; g.nbatch = nb;
    g.A = Mtx; g.va.rs_in = nin; g.va.ks_in = 1;
    g.B = in + (long long)b0 * nin * nelem; g.vb.rs_in = 1; g.vb.ks_in = nelem; g.bb.bs_in = nin * nelem;
    g.C = out + (long long)b0 * nout * nelem; g.vc.rs_in = nelem; g.vc.ks_in = 1; g.bc.bs_in = nout * nelem;
    g.slot = SLOT_TRANSFORM_FP64;
    GW_TRY(zgemm_fp64(g, c->stream));
  }
  return GW_OK;
}

// Rows [row0, row0 + nrows) of the transform of the q-th block.
int transform_q(gw_ctx* c, int stat, bool forward, const double2* in, double2* out, int q, int row0, int nrows,
                long long nelem) {
  const int nw = stat == 0 ? c->nwb : c->nwf;
  const int nin = forward ? c->ntau : nw, nout = forward ? nw : c->ntau;
  const double2* Mtx = forward ? (stat == 0 ? c->Fb : c->Ff) : (stat == 0 ? c->Bb : c->Bf);
  if (nrows <= 0) return GW_OK;
  ZGemm g;
  g.M = nrows; g.N = (int)nelem; g.K = nin; g.nbatch = 1;
  g.A = Mtx + (long long)row0 * nin; g.va.rs_in = nin; g.va.ks_in = 1;
  g.B = in + (long long)q * nin * nelem; g.vb.rs_in = 1; g.vb.ks_in = nelem;
  g.C = out + ((long long)q * nout + row0) * nelem; g.vc.rs_in = nelem; g.vc.ks_in = 1;
  g.slot = SLOT_TRANSFORM_FP64;
  return zgemm_fp64(g, c->stream);
}

int aux_dyson(gw_ctx* c, const double2* P0w, double2* Pw) {
  const long long n2 = c->naux2;
  const int nb = c->nk * c->nwb;
  if (Pw != P0w &&
      cudaMemcpyAsync(Pw, P0w, (size_t)nb * n2 * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess)
    return cuda_check("aux_dyson copy");
  GW_TRY(add_identity_fp64(Pw, c->naux, n2, nb, -1.0, 1.0, c->stream));   // I - P0
  GW_TRY(batched_inverse_fp64(Pw, c->naux, n2, nb, c->status, c->stream));
  GW_TRY(add_identity_fp64(Pw, c->naux, n2, nb, 1.0, -1.0, c->stream));   // (I - P0)^-1 - I
  return GW_OK;
}

int screened(gw_ctx* c, const double2* P0t, double2* Pt) {
  GW_TRY(transform(c, 0, true, P0t, c->Pw, c->nk, c->naux2));
  GW_TRY(aux_dyson(c, c->Pw, c->Pw));
  GW_TRY(transform(c, 0, false, c->Pw, Pt, c->nk, c->naux2));
  return GW_OK;
}

// The same for a P0t that satisfies P0^q(beta - tau) = P0^{-q}(tau)^T exactly (as gw_polarization
// writes it). Then P0^q(i W_n) = P0^{-q}(-i W_n)^T, the aux Dyson equation commutes with the
// transpose, and P~ inherits both relations: only canonical (q, n) and (q, t) are computed,
// the rest is filled by transposition. The frequency samples are symmetric (index j <-> nw-1-j).
//
// With a q range [q0, q1) only the q of the range are transformed and solved; a q whose -q lies
// outside the range takes every frequency and tau node (its mirror partner is not computed).
int screened_sym_pre(gw_ctx* c, const double2* P0t, int q0, int q1, const int** list_out, int* nlist_out) {
  const long long n2 = c->naux2;
  const bool full = q0 == 0 && q1 == c->nk;
  for (int q = q0; q < q1; ++q) {
    if (canonical_end(c, q, c->nwb, q0, q1) == 0) continue;
    GW_TRY(transform_q(c, 0, true, P0t, c->Pw, q, 0, c->nwb, n2));
  }
  // all canonical (q, n) matrices of the range in one launch each
  int nlist = c->nwlist;
  const int* list = c->wlist;
  if (!full) {
    std::vector<int> wl;
    for (int q = q0; q < q1; ++q)
      for (int n = 0; n < canonical_end(c, q, c->nwb, q0, q1); ++n) wl.push_back(q * c->nwb + n);
    nlist = (int)wl.size();
    if (nlist > 0 && cudaMemcpyAsync(c->wlist_q, wl.data(), wl.size() * sizeof(int), cudaMemcpyHostToDevice,
                                     c->stream) != cudaSuccess)
      return cuda_check("q-range frequency list");
    list = c->wlist_q;
  }
  if (nlist > 0) GW_TRY(add_identity_fp64(c->Pw, c->naux, n2, nlist, -1.0, 1.0, c->stream, list));   // I - P0
  *list_out = list;
  *nlist_out = nlist;
  return GW_OK;
}

int screened_sym_post(gw_ctx* c, double2* Pt, int q0, int q1, const int* list, int nlist) {
  const long long n2 = c->naux2;
  if (nlist > 0) GW_TRY(add_identity_fp64(c->Pw, c->naux, n2, nlist, 1.0, -1.0, c->stream, list));   // (I - P0)^-1 - I
  GW_TRY(mirror_fill(c->Pw, c->nk, c->nwb, c->naux, c->mq_dev, c->stream, q0, q1));
  for (int q = q0; q < q1; ++q)
    GW_TRY(transform_q(c, 0, false, c->Pw, Pt, q, 0, canonical_end(c, q, c->ntau, q0, q1), n2));
  return mirror_fill(Pt, c->nk, c->ntau, c->naux, c->mq_dev, c->stream, q0, q1);
}

int screened_sym(gw_ctx* c, const double2* P0t, double2* Pt, int q0 = 0, int q1 = -1) {
  if (q1 < 0) q1 = c->nk;
  const int* list = nullptr;
  int nlist = 0;
  GW_TRY(screened_sym_pre(c, P0t, q0, q1, &list, &nlist));
  if (nlist > 0) GW_TRY(batched_inverse_fp64(c->Pw, c->naux, c->naux2, nlist, c->status, c->stream, list));
  return screened_sym_post(c, Pt, q0, q1, list, nlist);
}

}  // namespace

// ---- ABI ----------------------------------------------------------------------------------

extern "C" {

const char* gw_version(void) { return "gw-gb300 0.1.0 (sm_103a)"; }

const char* gw_last_error(void) { return g_last_error.c_str(); }

int gw_sample_count(int ntau, int stat) { return sample_count(ntau, stat); }

int gw_grid_build(int ntau, double beta, int stat, double* tau_host, int64_t* idx_host, gw_c128* F_host,
                  gw_c128* B_host) {
  if (sample_count(ntau, stat) < 0 || !(beta > 0)) return fail(GW_EINVAL, "gw_grid_build: bad arguments");
  return grid_build(ntau, beta, stat, tau_host, idx_host, F_host, B_host);
}

}  // extern "C"

namespace gwi {
namespace {

bool config_ok(const gw_config* cfg) {
  const long long nk = (long long)cfg->nk[0] * cfg->nk[1] * cfg->nk[2];
  return !(cfg->nk[0] < 1 || cfg->nk[1] < 1 || cfg->nk[2] < 1 || nk > 4096 || cfg->nao < 1 || cfg->nao > 512 ||
           cfg->naux < 1 || cfg->naux > 4096 || cfg->ntau < 1 || cfg->ntau > 512 || !(cfg->beta > 0) ||
           cfg->precision < GW_FP64 || cfg->precision > GW_MIXED_BF16X4 || cfg->v_slices < GW_V_AUTO ||
           cfg->v_slices > GW_V_PER_Q || cfg->v_packed < 0 || cfg->v_packed > 1 || cfg->slice_pass < 0 ||
           cfg->slice_pass > 1 ||
           !(cfg->tile_n == 0 || cfg->tile_n == 56 || cfg->tile_n == 72 || cfg->tile_n == 80));
}

// Weights w_j with p(beta) = sum_j w_j f(tau_j) for the polynomial p of degree n - 1 through the
// n nodes (all inside (0, beta)): the barycentric form w_j = (lambda_j / (beta - tau_j)) /
// sum_i lambda_i / (beta - tau_i), lambda_j = 1 / prod_{i != j} (tau_j - tau_i), taken in
// logarithms of x = 2 tau / beta - 1 so that no product over- or underflows. For the
// first-kind Chebyshev nodes p is the Chebyshev series of the nodes evaluated at tau = beta.
static void weights_at_beta(const double* tau, int n, double beta, std::vector<double>& w) {
  std::vector<double> lg(n), sg(n);
  double top = -INFINITY;
  for (int j = 0; j < n; ++j) {
    const double xj = 2.0 * tau[j] / beta - 1.0;
    double l = -std::log(1.0 - xj), sgn = 1.0;
    for (int i = 0; i < n; ++i) {
      if (i == j) continue;
      const double d = xj - (2.0 * tau[i] / beta - 1.0);
      l -= std::log(std::fabs(d));
      if (d < 0) sgn = -sgn;
    }
    lg[j] = l;
    sg[j] = sgn;
    top = std::max(top, l);
  }
  w.assign(n, 0.0);
  double norm = 0.0;
  for (int j = 0; j < n; ++j) norm += (w[j] = sg[j] * std::exp(lg[j] - top));
  for (double& x : w) x /= norm;
}

// Grids, gather tables and workspaces of a context; in a size-only build (c->dry)
// the same sequence only sums the bytes it would allocate.
int ctx_build(gw_ctx* c, const gw_config* cfg) {
  const int nk = cfg->nk[0] * cfg->nk[1] * cfg->nk[2];
  c->cfg = *cfg;
  c->nk = nk;
  c->nao = cfg->nao;
  c->naux = cfg->naux;
  c->ntau = cfg->ntau;
  c->nao2 = (long long)c->nao * c->nao;
  c->naux2 = (long long)c->naux * c->naux;
  c->pair = (long long)c->naux * c->nao2;
  int rc = GW_OK;
  do {
    if ((rc = upload_grid(c, 0, &c->Fb, &c->Bb, &c->nwb)) != GW_OK) break;
    if ((rc = upload_grid(c, 1, &c->Ff, &c->Bf, &c->nwf)) != GW_OK) break;
    // k-mesh gather tables (element offsets), [q][k]
    std::vector<long long> t(6 * (size_t)nk * nk);
    const long long gk = (long long)c->ntau * c->nao2;
    for (int q = 0; q < nk; ++q)
      for (int k = 0; k < nk; ++k) {
        const int kp = kshift(cfg->nk, k, q, +1), km = kshift(cfg->nk, k, q, -1);
        const size_t i = (size_t)q * nk + k, s = (size_t)nk * nk;
        t[0 * s + i] = ((long long)k * nk + kp) * c->pair;
        t[1 * s + i] = ((long long)kp * nk + k) * c->pair;
        t[2 * s + i] = (long long)kp * gk;
        t[3 * s + i] = ((long long)k * nk + km) * c->pair;
        t[4 * s + i] = ((long long)km * nk + k) * c->pair;
        t[5 * s + i] = (long long)km * gk;
      }
    if ((rc = dev_alloc(c, &c->tabs, t.size())) != GW_OK) break;
    upload(c, c->tabs, t.data(), t.size() * sizeof(long long));
    const size_t s = (size_t)nk * nk;
    c->tab_kkpq = c->tabs;
    c->tab_kpqk = c->tabs + s;
    c->tab_gkpq = c->tabs + 2 * s;
    c->tab_kkmq = c->tabs + 3 * s;
    c->tab_kmqk = c->tabs + 4 * s;
    c->tab_gkmq = c->tabs + 5 * s;
    c->mq.resize(nk);
    for (int q = 0; q < nk; ++q) c->mq[q] = kshift(cfg->nk, 0, q, -1);
    if ((rc = dev_alloc(c, &c->mq_dev, nk)) != GW_OK) break;
    upload(c, c->mq_dev, c->mq.data(), nk * sizeof(int));
    {
      std::vector<int> wl;
      for (int q = 0; q < nk; ++q)
        for (int n = 0; n < canonical_end(c, q, c->nwb); ++n) wl.push_back(q * c->nwb + n);
      c->nwlist = (int)wl.size();
      c->wlist_host = wl;
      if ((rc = dev_alloc(c, &c->wlist, wl.size())) != GW_OK) break;
      upload(c, c->wlist, wl.data(), wl.size() * sizeof(int));
      // the (q, n) list of a q range (gw_sigma_eval_q): at most every (q, n)
      if ((rc = dev_alloc(c, &c->wlist_q, (size_t)nk * c->nwb)) != GW_OK) break;
    }
    // tau chunk: intermediates of 2 * nk * pair complex per tau node, capped at 4 GiB
    const double per_t = 2.0 * nk * (double)c->pair * sizeof(double2);
    int nt = cfg->tau_chunk > 0 ? cfg->tau_chunk : (int)std::max(1.0, std::floor(4294967296.0 / per_t));
    c->nt = std::min(nt, c->ntau);
    if (cfg->precision == GW_FP64) {
      if ((rc = dev_alloc(c, &c->work, (size_t)c->nt * 2 * nk * c->pair)) != GW_OK) break;
      if (cfg->v_packed && (rc = dev_alloc(c, &c->Vfull, (size_t)nk * nk * c->pair)) != GW_OK) break;
    }
    if ((rc = dev_alloc(c, &c->P0t, (size_t)nk * c->ntau * c->naux2)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->Pw, (size_t)nk * c->nwb * c->naux2)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->Pt, (size_t)nk * c->ntau * c->naux2)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->dyson_ws, (size_t)nk * c->nwf * c->nao2)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->status, 4)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->maxdiff, 1)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->nonfinite, 1)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->gamma, (size_t)nk * c->nao2)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->rho, (size_t)c->naux)) != GW_OK) break;
    // exchange partials of the fused kernel, or the per-k intermediate of the GEMM path (nao above its limit)
    // (plus, with only the packed V resident, room for the two unpacked blocks V^{kk'} and V^{k'k})
    const bool unpack_exchange = cfg->v_packed && cfg->precision != GW_FP64;
    const size_t nxinf = c->nao <= kExchangeMaxNao ? (size_t)nk * nk * exchange_chunks(nk, c->naux) * c->nao2
                                                   : (size_t)(unpack_exchange ? nk + 2 : nk) * c->pair;
    if ((rc = dev_alloc(c, &c->xinf, nxinf)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->scal, (size_t)kDotBlocks + 8)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->gw_w, (size_t)nk * c->nwf * c->nao2)) != GW_OK) break;
    if ((rc = dev_alloc(c, &c->heff, (size_t)nk * c->nao2)) != GW_OK) break;
    {
      std::vector<double> w, tau(c->ntau);
      for (int j = 0; j < c->ntau; ++j) {
        const double th = M_PI * (c->ntau - j - 0.5) / c->ntau;   // ascending first-kind Chebyshev nodes
        tau[j] = 0.5 * cfg->beta * (1.0 + std::cos(th));
      }
      weights_at_beta(tau.data(), c->ntau, cfg->beta, w);
      if ((rc = dev_alloc(c, &c->wbeta, (size_t)c->ntau)) != GW_OK) break;
      upload(c, c->wbeta, w.data(), w.size() * sizeof(double));
    }
    if (!c->dry) cudaMemset(c->status, 0, 4 * sizeof(int));
    if (cfg->precision != GW_FP64) {
      MixedDims d;
      d.nk3[0] = cfg->nk[0]; d.nk3[1] = cfg->nk[1]; d.nk3[2] = cfg->nk[2];
      d.nk = nk; d.nao = c->nao; d.naux = c->naux; d.ntau = c->ntau; d.precision = cfg->precision;
      d.tau_chunk = cfg->tau_chunk;
      d.v_slices = cfg->v_slices;
      d.v_packed = cfg->v_packed;
      d.fuse = cfg->slice_pass == 0;
      d.tile_n = cfg->tile_n;
      d.mq = c->mq;
      if ((rc = mixed_create(&c->mixed, d, c->stream, c->status, &c->bytes, c->dry)) != GW_OK) break;
    }
    if (!c->dry) rc = cuda_check("gw_create");
  } while (false);
  return rc;
}

}  // namespace

CtxInfo ctx_info(const gw_ctx* c) { return CtxInfo{c->stream, c->nk, c->ntau, c->nao, c->nwf, c->cfg.mu}; }

size_t job_device_bytes(const gw_config* cfg) {
  if (!config_ok(cfg)) return 0;
  gw_ctx c;
  c.dry = true;
  if (ctx_build(&c, cfg) != GW_OK) return 0;
  const size_t nk = (size_t)cfg->nk[0] * cfg->nk[1] * cfg->nk[2], nao2 = (size_t)cfg->nao * cfg->nao;
  // V, H (and an overlap of its size), G and the Sigma output of the job, and the loop's buffers
  // with its default options
  gw_scgw_options o{};
  const size_t vblocks = cfg->v_packed ? (size_t)packed_pairs((int)nk) : nk * nk;
  return c.bytes + sizeof(gw_c128) * (vblocks * cfg->naux * nao2 + 2 * nk * nao2 + 2 * nk * cfg->ntau * nao2) +
         scgw_device_bytes(cfg, &o);
}

}  // namespace gwi

extern "C" {

int gw_create(gw_ctx** out, const gw_config* cfg, void* cuda_stream) {
  if (!out || !cfg) return fail(GW_EINVAL, "gw_create: null argument");
  *out = nullptr;
  if (!config_ok(cfg)) return fail(GW_EINVAL, "gw_create: configuration out of range");
  gw_ctx* c = new gw_ctx();
  c->stream = (cudaStream_t)cuda_stream;
  const int rc = ctx_build(c, cfg);
  if (rc != GW_OK) {
    free_ctx(c);
    return rc;
  }
  *out = c;
  return GW_OK;
}

int gw_destroy(gw_ctx* ctx) {
  if (!ctx) return GW_OK;
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
  return GW_OK;
}

size_t gw_workspace_bytes(const gw_ctx* ctx) { return ctx ? ctx->bytes : 0; }

int gw_set_grids(gw_ctx* ctx, const double* tau_host, const gw_c128* Fb_host, const gw_c128* Bb_host,
                 const gw_c128* Ff_host, const gw_c128* Bf_host, const double* omega_b_host,
                 const double* omega_f_host) {
  if (!ctx || !tau_host || !Fb_host || !Bb_host || !Ff_host || !Bf_host || !omega_f_host)
    return fail(GW_EINVAL, "gw_set_grids: null argument");
  const int T = ctx->ntau, nb = ctx->nwb, nf = ctx->nwf;
  const double beta = ctx->cfg.beta;
  for (int t = 0; t < T; ++t) {
    if (!(tau_host[t] > 0.0 && tau_host[t] < beta) || (t > 0 && !(tau_host[t] > tau_host[t - 1])))
      return fail(GW_EINVAL, "gw_set_grids: tau must ascend inside (0, beta)");
    if (std::fabs(tau_host[t] + tau_host[T - 1 - t] - beta) > 1e-12 * beta)
      return fail(GW_EINVAL, "gw_set_grids: tau must be symmetric (tau[T-1-t] = beta - tau[t])");
  }
  if (omega_b_host) {
    double wmax = 0.0;
    for (int n = 0; n < nb; ++n) wmax = std::max(wmax, std::fabs(omega_b_host[n]));
    for (int n = 0; n < nb; ++n)
      if (std::fabs(omega_b_host[n] + omega_b_host[nb - 1 - n]) > 1e-12 * wmax)
        return fail(GW_EINVAL, "gw_set_grids: bosonic frequencies must be symmetric");
  }
  // the bosonic transforms must map the mirrored node to the mirrored frequency (what the
  // canonical-index shortcut of P0, P~ relies on): F[nb-1-n][T-1-t] = F[n][t], likewise B
  double fmax = 0.0, bmax = 0.0, fd = 0.0, bd = 0.0;
  for (int n = 0; n < nb; ++n)
    for (int t = 0; t < T; ++t) {
      const gw_c128 f = Fb_host[(size_t)n * T + t], fm = Fb_host[(size_t)(nb - 1 - n) * T + (T - 1 - t)];
      const gw_c128 b = Bb_host[(size_t)t * nb + n], bm = Bb_host[(size_t)(T - 1 - t) * nb + (nb - 1 - n)];
      fmax = std::max(fmax, std::hypot(f.re, f.im));
      bmax = std::max(bmax, std::hypot(b.re, b.im));
      fd = std::max(fd, std::hypot(f.re - fm.re, f.im - fm.im));
      bd = std::max(bd, std::hypot(b.re - bm.re, b.im - bm.im));
    }
  if (!(fd <= 1e-10 * fmax) || !(bd <= 1e-10 * bmax))
    return fail(GW_EINVAL, "gw_set_grids: bosonic F and B must map mirrored nodes to mirrored frequencies");
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check("gw_set_grids");
  const size_t sb = (size_t)nb * T * sizeof(double2), sf = (size_t)nf * T * sizeof(double2);
  if (cudaMemcpy(ctx->Fb, Fb_host, sb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->Bb, Bb_host, sb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->Ff, Ff_host, sf, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->Bf, Bf_host, sf, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(ctx->wf, omega_f_host, (size_t)nf * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_check("gw_set_grids copy");
  std::vector<double> w;
  weights_at_beta(tau_host, T, beta, w);
  if (cudaMemcpy(ctx->wbeta, w.data(), (size_t)T * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return cuda_check("gw_set_grids copy");
  return GW_OK;
}

int gw_set_coulomb(gw_ctx* ctx, const gw_c128* V_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  if (!ctx || !V_dev) return fail(GW_EINVAL, "gw_set_coulomb: null argument");
  const double2* V = reinterpret_cast<const double2*>(V_dev);
  ctx->coulomb = false;
  if (ctx->cfg.v_packed) {
    ctx->Vp = V;
    if (!ctx->mixed) {   // FP64: one full working copy
      VPairs L;
      L.all = 1;
      GW_TRY(unpack_v_fp64(V, ctx->nk, ctx->nao, ctx->pair, L, ctx->nk * ctx->nk, ctx->Vfull, ctx->stream));
      ctx->V = ctx->Vfull;
    } else {
      ctx->V = nullptr;
      GW_TRY(mixed_set_coulomb(ctx->mixed, nullptr, V));
    }
  } else {
    ctx->V = V;
    ctx->Vp = nullptr;
    if (ctx->mixed) GW_TRY(mixed_set_coulomb(ctx->mixed, V));
  }
  ctx->coulomb = true;
  return GW_OK;
}

int gw_polarization(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* P0t_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_polarization");
  if (!ctx || !G_dev || !P0t_dev) return fail(GW_EINVAL, "gw_polarization: null argument");
  if (!ctx->coulomb) return fail(GW_EINVAL, "gw_polarization: call gw_set_coulomb first");
  const double2* G = reinterpret_cast<const double2*>(G_dev);
  double2* P = reinterpret_cast<double2*>(P0t_dev);
  // only canonical (q, tau) are contracted; the rest is P0^q(beta - tau) = P0^{-q}(tau)^T
  if (ctx->mixed)
    GW_TRY(mixed_polarization(ctx->mixed, G, P, ctx->cfg.spin_factor, 0, ctx->nk));
  else
    GW_TRY(polarization_fp64(ctx, G, P, 0, ctx->nk));
  return mirror_fill(P, ctx->nk, ctx->ntau, ctx->naux, ctx->mq_dev, ctx->stream);
}

int gw_to_matsubara(gw_ctx* ctx, int stat, const gw_c128* in_dev, gw_c128* out_dev, int nbatch,
                    long long nelem) {
  if (!ctx || !in_dev || !out_dev || (stat != 0 && stat != 1) || nbatch < 0 || nelem < 0)
    return fail(GW_EINVAL, "gw_to_matsubara: bad argument");
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  return transform(ctx, stat, true, reinterpret_cast<const double2*>(in_dev),
                   reinterpret_cast<double2*>(out_dev), nbatch, nelem);
}

int gw_to_tau(gw_ctx* ctx, int stat, const gw_c128* in_dev, gw_c128* out_dev, int nbatch, long long nelem) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  if (!ctx || !in_dev || !out_dev || (stat != 0 && stat != 1) || nbatch < 0 || nelem < 0)
    return fail(GW_EINVAL, "gw_to_tau: bad argument");
  return transform(ctx, stat, false, reinterpret_cast<const double2*>(in_dev),
                   reinterpret_cast<double2*>(out_dev), nbatch, nelem);
}

int gw_aux_dyson(gw_ctx* ctx, const gw_c128* P0w_dev, gw_c128* Pw_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_aux_dyson");
  if (!ctx || !P0w_dev || !Pw_dev) return fail(GW_EINVAL, "gw_aux_dyson: null argument");
  return aux_dyson(ctx, reinterpret_cast<const double2*>(P0w_dev), reinterpret_cast<double2*>(Pw_dev));
}

int gw_screened_interaction(gw_ctx* ctx, const gw_c128* P0t_dev, gw_c128* Pt_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_screened_interaction");
  if (!ctx || !P0t_dev || !Pt_dev) return fail(GW_EINVAL, "gw_screened_interaction: null argument");
  return screened(ctx, reinterpret_cast<const double2*>(P0t_dev), reinterpret_cast<double2*>(Pt_dev));
}

int gw_self_energy(gw_ctx* ctx, const gw_c128* G_dev, const gw_c128* Pt_dev, gw_c128* Sig_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_self_energy");
  if (!ctx || !G_dev || !Pt_dev || !Sig_dev) return fail(GW_EINVAL, "gw_self_energy: null argument");
  if (!ctx->coulomb) return fail(GW_EINVAL, "gw_self_energy: call gw_set_coulomb first");
  const double2* G = reinterpret_cast<const double2*>(G_dev);
  const double2* P = reinterpret_cast<const double2*>(Pt_dev);
  double2* S = reinterpret_cast<double2*>(Sig_dev);
  if (ctx->mixed) return mixed_self_energy(ctx->mixed, G, P, S, 0, ctx->nk);
  return self_energy_fp64(ctx, G, P, S, 0, ctx->nk);
}

int gw_sigma_eval(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* Sig_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_sigma_eval");
  if (!ctx || !G_dev || !Sig_dev) return fail(GW_EINVAL, "gw_sigma_eval: null argument");
  GW_TRY(gw_polarization(ctx, G_dev, reinterpret_cast<gw_c128*>(ctx->P0t)));
  GW_TRY(screened_sym(ctx, ctx->P0t, ctx->Pt));
  return gw_self_energy(ctx, G_dev, reinterpret_cast<const gw_c128*>(ctx->Pt), Sig_dev);
}

}  // extern "C"

namespace gwi {

int sigma_eval_part(gw_ctx* ctx, const double2* G, double2* Sig, int part) {
  if (part == 0) {
    GW_TRY(gw_polarization(ctx, reinterpret_cast<const gw_c128*>(G), reinterpret_cast<gw_c128*>(ctx->P0t)));
    ProfScope _ps(&ctx->prof);
    const int* list = nullptr;
    int nlist = 0;
    return screened_sym_pre(ctx, ctx->P0t, 0, ctx->nk, &list, &nlist);
  }
  {
    ProfScope _ps(&ctx->prof);
    GW_TRY(screened_sym_post(ctx, ctx->Pt, 0, ctx->nk, ctx->wlist, ctx->nwlist));
  }
  return gw_self_energy(ctx, reinterpret_cast<const gw_c128*>(G), reinterpret_cast<const gw_c128*>(ctx->Pt),
                        reinterpret_cast<gw_c128*>(Sig));
}

void inverse_items(gw_ctx* ctx, std::vector<GjItem>* items) {
  for (int w : ctx->wlist_host) items->push_back(GjItem{ctx->Pw + (long long)w * ctx->naux2, ctx->naux, ctx->status});
}

}  // namespace gwi

extern "C" {

int gw_sigma_eval_q(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* Sig_dev, int q_begin, int q_end,
                    gw_c128* P0t_dev, gw_c128* Pt_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_sigma_eval_q");
  if (!ctx || !G_dev || !Sig_dev) return fail(GW_EINVAL, "gw_sigma_eval_q: null argument");
  if (q_begin < 0 || q_end > ctx->nk || q_begin > q_end)
    return fail(GW_EINVAL, "gw_sigma_eval_q: range [%d, %d) is not within [0, %d)", q_begin, q_end, ctx->nk);
  if (!ctx->coulomb) return fail(GW_EINVAL, "gw_sigma_eval_q: call gw_set_coulomb first");
  const double2* G = reinterpret_cast<const double2*>(G_dev);
  double2* S = reinterpret_cast<double2*>(Sig_dev);
  if (ctx->mixed)
    GW_TRY(mixed_polarization(ctx->mixed, G, ctx->P0t, ctx->cfg.spin_factor, q_begin, q_end));
  else
    GW_TRY(polarization_fp64(ctx, G, ctx->P0t, q_begin, q_end));
  GW_TRY(mirror_fill(ctx->P0t, ctx->nk, ctx->ntau, ctx->naux, ctx->mq_dev, ctx->stream, q_begin, q_end));
  GW_TRY(screened_sym(ctx, ctx->P0t, ctx->Pt, q_begin, q_end));
  // the range's blocks, for a caller that checks the stages
  const size_t blk = (size_t)(q_end - q_begin) * ctx->ntau * ctx->naux2 * sizeof(double2);
  const size_t off = (size_t)q_begin * ctx->ntau * ctx->naux2;
  if (P0t_dev && blk && cudaMemcpyAsync(P0t_dev, ctx->P0t + off, blk, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
    return cuda_check("gw_sigma_eval_q: P0 copy");
  if (Pt_dev && blk && cudaMemcpyAsync(Pt_dev, ctx->Pt + off, blk, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess)
    return cuda_check("gw_sigma_eval_q: P~ copy");
  if (ctx->mixed) return mixed_self_energy(ctx->mixed, G, ctx->Pt, S, q_begin, q_end);
  return self_energy_fp64(ctx, G, ctx->Pt, S, q_begin, q_end);
}

int gw_dyson_G(gw_ctx* ctx, const gw_c128* H_dev, const gw_c128* Sig_dev, gw_c128* G_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_dyson_G");
  if (!ctx || !H_dev || !Sig_dev || !G_dev) return fail(GW_EINVAL, "gw_dyson_G: null argument");
  const double2* H = reinterpret_cast<const double2*>(H_dev);
  const double2* S = reinterpret_cast<const double2*>(Sig_dev);
  double2* G = reinterpret_cast<double2*>(G_dev);
  GW_TRY(transform(ctx, 1, true, S, ctx->dyson_ws, ctx->nk, ctx->nao2));
  GW_TRY(build_g_dyson_fp64(ctx->dyson_ws, H, ctx->S, ctx->wf, ctx->cfg.mu, ctx->nk, ctx->nwf, ctx->nao,
                            ctx->stream));
  GW_TRY(batched_inverse_fp64(ctx->dyson_ws, ctx->nao, ctx->nao2, ctx->nk * ctx->nwf, ctx->status, ctx->stream));
  GW_TRY(transform(ctx, 1, false, ctx->dyson_ws, G, ctx->nk, ctx->nao2));
  return GW_OK;
}

int gw_density(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* gamma_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_density");
  if (!ctx || !G_dev || !gamma_dev) return fail(GW_EINVAL, "gw_density: null argument");
  return density_fp64(reinterpret_cast<const double2*>(G_dev), ctx->wbeta, reinterpret_cast<double2*>(gamma_dev),
                      ctx->nk, ctx->ntau, ctx->nao, ctx->stream);
}

int gw_sigma_inf(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* SigInf_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_sigma_inf");
  if (!ctx || !G_dev || !SigInf_dev) return fail(GW_EINVAL, "gw_sigma_inf: null argument");
  if (!ctx->coulomb) return fail(GW_EINVAL, "gw_sigma_inf: call gw_set_coulomb first");
  const int nk = ctx->nk, nao = ctx->nao, naux = ctx->naux;
  double2* S = reinterpret_cast<double2*>(SigInf_dev);
  GW_TRY(density_fp64(reinterpret_cast<const double2*>(G_dev), ctx->wbeta, ctx->gamma, nk, ctx->ntau, nao, ctx->stream));
  // Hartree: (s / N_k) sum_Q V^{kk}_ij(Q) rho_Q
  // the full-layout V when there is one, else the packed one (mixed precisions with cfg.v_packed)
  const double2* Vs = ctx->V ? ctx->V : ctx->Vp;
  const int packed = ctx->V ? 0 : 1;
  GW_TRY(hartree_fp64(Vs, ctx->gamma, ctx->rho, S, nk, naux, nao, ctx->cfg.spin_factor / nk, packed, ctx->stream));
  // exchange: -(1 / N_k) sum_{k'} sum_{Q b} X^{k'}_{Q i b} V^{k'k}_bj(Q), X^{k'}_{Q i b} = sum_a V^{kk'}_ia(Q) gamma^{k'}_ab
  if (nao <= kExchangeMaxNao)
    return exchange_fp64(Vs, ctx->gamma, ctx->xinf, S, nk, naux, nao, -1.0 / nk, packed, ctx->stream);
  // per k: X^{k'} = V^{kk'} gamma^{k'} for every k' (one batched product), then S^k -= X^{k'} V^{k'k}
  // summed over k' in order. With only the packed V resident, V^{kk'} and V^{k'k} are unpacked
  // into two scratch blocks per (k, k') and the first product runs one k' at a time (the same
  // arithmetic per element as the batched product).
  double2* vx = ctx->xinf + (long long)nk * ctx->pair;
  auto first = [&](const double2* A, long long a_stride, const double2* B, double2* C, int nbatch) {
    ZGemm a;
    a.M = naux * nao;
    a.N = nao;
    a.K = nao;
    a.nbatch = nbatch;
    a.A = A;
    a.ba.bs_in = a_stride;
    a.va.rs_in = nao;
    a.va.ks_in = 1;
    a.B = B;
    a.bb.bs_in = ctx->nao2;
    a.vb.rs_in = 1;
    a.vb.ks_in = nao;
    a.C = C;
    a.bc.bs_in = ctx->pair;
    a.vc.rs_in = nao;
    a.vc.ks_in = 1;
    a.slot = SLOT_STATIC_FP64;
    return zgemm_fp64(a, ctx->stream);
  };
  auto second = [&](const double2* X, const double2* Vb, int k) {
    ZGemm b;
    b.M = nao;
    b.N = nao;
    b.K = naux * nao;
    b.A = X;
    b.va.rs_in = nao;
    b.va.kin = nao;
    b.va.ks_in = 1;
    b.va.ks_out = ctx->nao2;
    b.B = Vb;
    b.vb.rs_in = 1;
    b.vb.kin = nao;
    b.vb.ks_in = nao;
    b.vb.ks_out = ctx->nao2;
    b.C = S + (long long)k * ctx->nao2;
    b.vc.rs_in = nao;
    b.vc.ks_in = 1;
    b.alpha = -1.0 / nk;
    b.accumulate = 1;
    b.slot = SLOT_STATIC_FP64;
    return zgemm_fp64(b, ctx->stream);
  };
  if (packed) {
    for (int k = 0; k < nk; ++k)
      for (int kp = 0; kp < nk; ++kp) {
        VPairs L;
        L.k1[0] = k;
        L.k2[0] = kp;
        L.k1[1] = kp;
        L.k2[1] = k;
        GW_TRY(unpack_v_fp64(ctx->Vp, nk, nao, ctx->pair, L, 2, vx, ctx->stream));
        GW_TRY(first(vx, 0, ctx->gamma + (long long)kp * ctx->nao2, ctx->xinf, 1));
        GW_TRY(second(ctx->xinf, vx + ctx->pair, k));
      }
    return GW_OK;
  }
  for (int k = 0; k < nk; ++k) {
    GW_TRY(first(ctx->V + (long long)k * nk * ctx->pair, ctx->pair, ctx->gamma, ctx->xinf, nk));
    for (int kp = 0; kp < nk; ++kp)
      GW_TRY(second(ctx->xinf + (long long)kp * ctx->pair, ctx->V + ((long long)kp * nk + k) * ctx->pair, k));
  }
  return GW_OK;
}

int gw_commutator_residual(gw_ctx* ctx, const gw_c128* H_dev, const gw_c128* SigInf_dev, const gw_c128* Sig_dev,
                           const gw_c128* G_dev, gw_c128* e_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_commutator_residual");
  if (!ctx || !H_dev || !Sig_dev || !G_dev || !e_dev) return fail(GW_EINVAL, "gw_commutator_residual: null argument");
  const int nk = ctx->nk, nao = ctx->nao, nw = ctx->nwf;
  const double2* H = reinterpret_cast<const double2*>(H_dev);
  if (SigInf_dev) {
    GW_TRY(add_fp64(H, reinterpret_cast<const double2*>(SigInf_dev), ctx->heff, (long long)nk * ctx->nao2,
                    ctx->stream));
    H = ctx->heff;
  }
  double2* Fw = ctx->dyson_ws;
  GW_TRY(transform(ctx, 1, true, reinterpret_cast<const double2*>(G_dev), ctx->gw_w, nk, ctx->nao2));
  GW_TRY(transform(ctx, 1, true, reinterpret_cast<const double2*>(Sig_dev), Fw, nk, ctx->nao2));
  // Fw <- (i w_n + mu) S - H - Sigma~(i w_n). Without an overlap the multiple of I commutes exactly
  // and e = Fw G - G Fw = [G, H + Sigma~]; with one, e = Fw G S - S G Fw = S G F - F G S.
  GW_TRY(build_g_dyson_fp64(Fw, H, ctx->S, ctx->wf, ctx->cfg.mu, nk, nw, nao, ctx->stream));
  double2* e = reinterpret_cast<double2*>(e_dev);
  // C = alpha X Y (+ C), X and Y per (k, n) or, for the overlap, per k (batch b = k nw + n)
  auto mul = [&](const double2* X, bool x_per_k, const double2* Y, bool y_per_k, double2* C, double alpha,
                 int acc) {
    ZGemm g;
    g.M = g.N = g.K = nao;
    g.nbatch = nk * nw;
    g.bin = nw;
    g.A = X;
    g.B = Y;
    g.C = C;
    g.ba.bs_in = x_per_k ? 0 : ctx->nao2;
    g.ba.bs_out = x_per_k ? ctx->nao2 : (long long)nw * ctx->nao2;
    g.bb.bs_in = y_per_k ? 0 : ctx->nao2;
    g.bb.bs_out = y_per_k ? ctx->nao2 : (long long)nw * ctx->nao2;
    g.bc.bs_in = ctx->nao2;
    g.bc.bs_out = (long long)nw * ctx->nao2;
    g.va.rs_in = nao;                  // A(m, k) = X[m][k]
    g.va.ks_in = 1;
    g.vb.rs_in = 1;                    // B(n, k) = Y[k][n]
    g.vb.ks_in = nao;
    g.vc.rs_in = nao;
    g.vc.ks_in = 1;
    g.alpha = alpha;
    g.accumulate = acc;
    g.slot = SLOT_STATIC_FP64;
    return zgemm_fp64(g, ctx->stream);
  };
  if (!ctx->S) {
    GW_TRY(mul(Fw, false, ctx->gw_w, false, e, 1.0, 0));
    return mul(ctx->gw_w, false, Fw, false, e, -1.0, 1);
  }
  if (!ctx->cw_tmp &&
      cudaMalloc(reinterpret_cast<void**>(&ctx->cw_tmp), (size_t)nk * nw * ctx->nao2 * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(GW_ENOMEM, "gw_commutator_residual: no room for the overlap products");
  }
  GW_TRY(mul(Fw, false, ctx->gw_w, false, ctx->cw_tmp, 1.0, 0));        // Fw G
  GW_TRY(mul(ctx->cw_tmp, false, ctx->S, true, e, 1.0, 0));             // e = Fw G S
  GW_TRY(mul(ctx->gw_w, false, Fw, false, ctx->cw_tmp, 1.0, 0));        // G Fw
  return mul(ctx->S, true, ctx->cw_tmp, false, e, -1.0, 1);             // e -= S G Fw
}

int gw_check_guards(gw_ctx* ctx) {
  if (!ctx) return fail(GW_EINVAL, "gw_check_guards: null context");
  std::vector<unsigned char*> all = ctx->guards;
  if (ctx->mixed) mixed_guards(ctx->mixed, &all);
  int first = -1;
  const int bad = check_guards(all.data(), (int)all.size(), &first, ctx->stream);
  if (bad < 0) return fail(GW_ECUDA, "gw_check_guards: the check did not run");
  if (bad > 0) return fail(GW_ECUDA, "gw_check_guards: %d of %zu workspace guards overwritten (first: %d)", bad,
                           all.size(), first);
  return GW_OK;
}

int gw_debug_mark_guard(gw_ctx* ctx, int index) {
  if (!ctx || index < 0 || index >= (int)ctx->guards.size()) return fail(GW_EINVAL, "gw_debug_mark_guard: bad index");
  // one byte inside the allocation's own guard zone: what a write past the workspace would leave
  return cudaMemset(ctx->guards[index] + kGuardBytes / 2, 0, 1) == cudaSuccess ? GW_OK
                                                                            : fail(GW_ECUDA, "gw_debug_mark_guard");
}

int gw_selftest_bounded_wait(double limit_s, int* code_out, void* cuda_stream) {
  if (!code_out || !(limit_s >= 1e-3 && limit_s <= 10.0)) return fail(GW_EINVAL, "gw_selftest_bounded_wait: bad argument");
  *code_out = 0;
  return mixed_wait_selftest(limit_s, code_out, (cudaStream_t)cuda_stream);
}

int gw_set_overlap(gw_ctx* ctx, const gw_c128* S_dev) {
  if (!ctx) return fail(GW_EINVAL, "gw_set_overlap: null context");
  ctx->S = reinterpret_cast<const double2*>(S_dev);
  return GW_OK;
}

// Exchange term of Eq. sigma2 for every k and tau node, added to S with weight alpha:
//   S^k(t) += alpha sum_{k1 k2} X, X_ij = sum_{Q R q m l} A_iq(Q) D_qm(R) B_ml(Q) V^{k2 k}_lj(R),
//   A(Q) = V^{k k1}(Q) G^{k1}(t), D(R) = V^{k1 k3}(R) G^{k3}(beta - t), B(Q) = V^{k3 k2}(Q) G^{k2}(t),
//   k3 = k1 + k2 - k. Contracted over the auxiliary indices first:
//   Y[(i q)][(m l)] = sum_Q A_iq(Q) B_ml(Q),  W[(q m)][(l j)] = sum_R D_qm(R) V^{k2 k}_lj(R),
//   X_ij = sum_{q m l} Y[(i q)][(m l)] W[(q m)][(l j)],
// 2 nao^4 naux + nao^5 complex MACs per (k, k1, k2, t) (2 naux^2 nao^3 the other way round). The
// last product is split over q into partial sums (its output is only nao x nao) and reduced in
// a fixed order.
static int gf2_exchange(gw_ctx* c, const double2* G, double2* S, double alpha) {
  const int nk = c->nk, nao = c->nao, naux = c->naux, T = c->ntau;
  const long long n2 = c->nao2, pair = c->pair, n3 = n2 * nao, n4 = n2 * n2;
  const double per_t = (3.0 * pair + 2.0 * n4 + n3) * sizeof(double2);   // A, D, B, Y, W, partials
  int nt = (int)std::min<double>(T, std::max(1.0, std::floor(2147483648.0 / per_t)));
  nt = std::max(1, std::min(nt, 65535 / nao));               // batch count of the split last product
  if (c->cfg.tau_chunk > 0) nt = std::min(nt, c->cfg.tau_chunk);
  const bool unpack = c->V == nullptr;    // packed V without a full copy: four blocks per (k, k1, k2)
  const size_t need = (size_t)nt * (3 * pair + 2 * n4 + n3) + (unpack ? 4 * (size_t)pair : 0);
  if (c->gf2_n < need) {
    if (c->gf2_ws) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->gf2_ws);
    }
    c->gf2_ws = nullptr;
    c->gf2_n = 0;
    if (cudaMalloc(reinterpret_cast<void**>(&c->gf2_ws), need * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(GW_ENOMEM, "gf2 exchange: cannot allocate %zu bytes", need * sizeof(double2));
    }
    c->gf2_n = need;
  }
  double2* A = c->gf2_ws;
  double2* D = A + (size_t)nt * pair;
  double2* B = D + (size_t)nt * pair;
  double2* Y = B + (size_t)nt * pair;
  double2* W = Y + (size_t)nt * n4;
  double2* part = W + (size_t)nt * n4;
  double2* vblk = part + (size_t)nt * n3;   // the unpacked blocks (k k1), (k1 k3), (k3 k2), (k2 k)
  // out[t][Q][i][b] = sum_a V[Q][i][a] Gt[a][b], Gt = g0 + t * gstep
  auto vg = [&](const double2* Vb, const double2* g0, long long gstep, int m, double2* out) {
    ZGemm g;
    g.M = naux * nao;
    g.N = nao;
    g.K = nao;
    g.nbatch = m;
    g.A = Vb;
    g.va.rs_in = nao;
    g.va.ks_in = 1;
    g.B = g0;
    g.vb.rs_in = 1;
    g.vb.ks_in = nao;
    g.bb.bs_in = gstep;
    g.C = out;
    g.vc.rs_in = nao;
    g.vc.ks_in = 1;
    g.bc.bs_in = pair;
    g.slot = SLOT_GF2_FP64;
    return zgemm_fp64(g, c->stream);
  };
  // out[t][(a b)][(c d)] = sum_Q X[t][Q][a][b] Z[t][Q][c][d]   (Z's batch stride may be 0)
  auto outer_q = [&](const double2* X, const double2* Z, long long zstep, int m, double2* out) {
    ZGemm g;
    g.M = (int)n2;
    g.N = (int)n2;
    g.K = naux;
    g.nbatch = m;
    g.A = X;
    g.va.rs_in = 1;
    g.va.ks_in = n2;
    g.ba.bs_in = pair;
    g.B = Z;
    g.vb.rs_in = 1;
    g.vb.ks_in = n2;
    g.bb.bs_in = zstep;
    g.C = out;
    g.vc.rs_in = n2;
    g.vc.ks_in = 1;
    g.bc.bs_in = n4;
    g.slot = SLOT_GF2_FP64;
    return zgemm_fp64(g, c->stream);
  };
  for (int k = 0; k < nk; ++k)
    for (int k1 = 0; k1 < nk; ++k1)
      for (int k2 = 0; k2 < nk; ++k2) {
        const int k3 = kshift(c->cfg.nk, kshift(c->cfg.nk, k1, k2, +1), k, -1);
        const int pa[4] = {k, k1, k3, k2}, pb[4] = {k1, k3, k2, k};
        const double2* vb[4];
        if (unpack) {
          VPairs L;
          for (int i = 0; i < 4; ++i) {
            L.k1[i] = pa[i];
            L.k2[i] = pb[i];
            vb[i] = vblk + i * pair;
          }
          GW_TRY(unpack_v_fp64(c->Vp, nk, nao, pair, L, 4, vblk, c->stream));
        } else {
          for (int i = 0; i < 4; ++i) vb[i] = c->V + ((long long)pa[i] * nk + pb[i]) * pair;
        }
        for (int t0 = 0; t0 < T; t0 += nt) {
          const int m = std::min(nt, T - t0);
          GW_TRY(vg(vb[0], G + ((long long)k1 * T + t0) * n2, n2, m, A));
          GW_TRY(vg(vb[1], G + ((long long)k3 * T + (T - 1 - t0)) * n2, -n2, m, D));
          GW_TRY(vg(vb[2], G + ((long long)k2 * T + t0) * n2, n2, m, B));
          if (c->mixed) {   // the two nao^4 naux products on the tensor cores
            GW_TRY(mixed_outer_q(c->mixed, A, pair, B, pair, m, (int)n2, Y, n4));
            GW_TRY(mixed_outer_q(c->mixed, D, pair, vb[3], 0, m, (int)n2, W, n4));
          } else {
            GW_TRY(outer_q(A, B, pair, m, Y));                                          // Y = sum_Q A B
            GW_TRY(outer_q(D, vb[3], 0, m, W));                                         // W = sum_R D V
          }
          if (c->mixed) {
            GW_TRY(mixed_gf2_last(c->mixed, Y, W, m, nao, part));
          } else {  // part[t][q][i][j] = sum_{(m l)} Y[t][(i q)][(m l)] W[t][(q m)][(l j)], batch (t, q)
            ZGemm g;
            g.M = nao;
            g.N = nao;
            g.K = (int)n2;
            g.nbatch = m * nao;
            g.bin = nao;
            g.A = Y;
            g.va.rs_in = n3;
            g.va.ks_in = 1;
            g.ba.bs_in = n2;
            g.ba.bs_out = n4;
            g.B = W;
            g.vb.rs_in = 1;
            g.vb.ks_in = nao;
            g.bb.bs_in = n3;
            g.bb.bs_out = n4;
            g.C = part;
            g.vc.rs_in = nao;
            g.vc.ks_in = 1;
            g.bc.bs_in = n2;
            g.bc.bs_out = n3;
            g.slot = SLOT_GF2_FP64;
            GW_TRY(zgemm_fp64(g, c->stream));
          }
          GW_TRY(reduce_partials_fp64(part, S + ((long long)k * T + t0) * n2, m, (int)n2, nao, alpha, c->stream));
        }
      }
  return GW_OK;
}

int gw_gf2_exchange(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* SigX_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_gf2_exchange");
  if (!ctx || !G_dev || !SigX_dev) return fail(GW_EINVAL, "gw_gf2_exchange: null argument");
  if (!ctx->coulomb) return fail(GW_EINVAL, "gw_gf2_exchange: call gw_set_coulomb first");
  double2* S = reinterpret_cast<double2*>(SigX_dev);
  if (cudaMemsetAsync(S, 0, (size_t)ctx->nk * ctx->ntau * ctx->nao2 * sizeof(double2), ctx->stream) != cudaSuccess)
    return cuda_check("gw_gf2_exchange memset");
  return gf2_exchange(ctx, reinterpret_cast<const double2*>(G_dev), S, 1.0 / ((double)ctx->nk * ctx->nk));
}

int gw_gf2_self_energy(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* Sig_dev) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_gf2_self_energy");
  if (!ctx || !G_dev || !Sig_dev) return fail(GW_EINVAL, "gw_gf2_self_energy: null argument");
  if (!ctx->coulomb) return fail(GW_EINVAL, "gw_gf2_self_energy: call gw_set_coulomb first");
  // direct term: the GW self-energy contraction with P0 in place of P~
  GW_TRY(gw_polarization(ctx, G_dev, reinterpret_cast<gw_c128*>(ctx->P0t)));
  GW_TRY(gw_self_energy(ctx, G_dev, reinterpret_cast<const gw_c128*>(ctx->P0t), Sig_dev));
  return gf2_exchange(ctx, reinterpret_cast<const double2*>(G_dev), reinterpret_cast<double2*>(Sig_dev),
                      -1.0 / ((double)ctx->nk * ctx->nk));
}

int gw_set_mu(gw_ctx* ctx, double mu) {
  if (!ctx || !std::isfinite(mu)) return fail(GW_EINVAL, "gw_set_mu: bad argument");
  ctx->cfg.mu = mu;
  return GW_OK;
}

int gw_particle_number(gw_ctx* ctx, const gw_c128* G_dev, double* n_host) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  NvtxRange _nr("gw_particle_number");
  if (!ctx || !G_dev || !n_host) return fail(GW_EINVAL, "gw_particle_number: null argument");
  GW_TRY(density_fp64(reinterpret_cast<const double2*>(G_dev), ctx->wbeta, ctx->gamma, ctx->nk, ctx->ntau, ctx->nao,
                      ctx->stream));
  GW_TRY(trace_fp64(ctx->gamma, ctx->S, ctx->nk, ctx->nao, ctx->scal, ctx->stream));
  double tr = 0.0;
  if (cudaMemcpyAsync(&tr, ctx->scal, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return cuda_check("gw_particle_number");
  *n_host = ctx->cfg.spin_factor * tr / ctx->nk;
  return GW_OK;
}

int gw_find_mu(gw_ctx* ctx, const gw_c128* Heff_dev, const gw_c128* Sig_dev, double n_target, double mu_lo,
               double mu_hi, double tol, gw_c128* G_dev, double* mu_host) {
  NvtxRange _nr("gw_find_mu");
  if (!ctx || !Heff_dev || !Sig_dev || !G_dev || !mu_host || !(mu_lo < mu_hi) || !(tol > 0))
    return fail(GW_EINVAL, "gw_find_mu: bad argument");
  auto number = [&](double mu, double* n) {
    ctx->cfg.mu = mu;
    GW_TRY(gw_dyson_G(ctx, Heff_dev, Sig_dev, G_dev));
    return gw_particle_number(ctx, G_dev, n);
  };
  // f(mu) = N(mu) - n_target grows with mu. Regula falsi with the Illinois modification (the
  // retained end's value is halved when the same end is kept twice), and a bisection step
  // whenever two steps have not halved the bracket; stops once the bracket is below tol or f
  // vanishes. G_dev holds the solution at the returned mu, the last point evaluated.
  double f_lo = 0.0, f_hi = 0.0;
  GW_TRY(number(mu_lo, &f_lo));
  GW_TRY(number(mu_hi, &f_hi));
  f_lo -= n_target;
  f_hi -= n_target;
  if (!(f_lo <= 0.0 && f_hi >= 0.0))
    return fail(GW_EINVAL, "gw_find_mu: target %.6g outside [N(mu_lo), N(mu_hi)] = [%.6g, %.6g]", n_target,
                f_lo + n_target, f_hi + n_target);
  double mu = mu_hi;                   // G_dev holds the solution at mu_hi now
  if (f_lo == 0.0) {
    mu = mu_lo;
    GW_TRY(number(mu, &f_lo));
  } else if (f_hi != 0.0) {
    int kept = 0;                        // -1: the low end was kept last, +1: the high end
    double width_ref = mu_hi - mu_lo;
    for (int it = 0; it < 200; ++it) {
      double m = (mu_lo * f_hi - mu_hi * f_lo) / (f_hi - f_lo);
      if (it % 2 == 1) {
        if (mu_hi - mu_lo > 0.5 * width_ref) m = 0.5 * (mu_lo + mu_hi);
        width_ref = mu_hi - mu_lo;
      }
      if (!(m > mu_lo && m < mu_hi)) m = 0.5 * (mu_lo + mu_hi);
      double f = 0.0;
      GW_TRY(number(m, &f));
      f -= n_target;
      mu = m;
      if (f == 0.0) break;
      if (f < 0.0) {
        mu_lo = m;
        f_lo = f;
        if (kept == +1) f_hi *= 0.5;
        kept = +1;
      } else {
        mu_hi = m;
        f_hi = f;
        if (kept == -1) f_lo *= 0.5;
        kept = -1;
      }
      if (mu_hi - mu_lo < tol) break;
    }
  }
  *mu_host = mu;
  return GW_OK;
}

int gw_mix(gw_ctx* ctx, const gw_c128* Sig_new_dev, gw_c128* Sig_inout_dev, double alpha,
           double* max_abs_diff_host) {
  ProfScope _ps(ctx ? &ctx->prof : nullptr);
  if (!ctx || !Sig_new_dev || !Sig_inout_dev) return fail(GW_EINVAL, "gw_mix: null argument");
  const long long n = (long long)ctx->nk * ctx->ntau * ctx->nao2;
  cudaMemsetAsync(ctx->maxdiff, 0, sizeof(double), ctx->stream);
  cudaMemsetAsync(ctx->nonfinite, 0, sizeof(int), ctx->stream);
  GW_TRY(mix_fp64(reinterpret_cast<const double2*>(Sig_new_dev), reinterpret_cast<double2*>(Sig_inout_dev),
                  alpha, n, ctx->maxdiff, ctx->nonfinite, ctx->stream));
  double md = 0;
  int bad = 0;
  cudaMemcpyAsync(&md, ctx->maxdiff, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  cudaMemcpyAsync(&bad, ctx->nonfinite, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check("gw_mix sync");
  if (max_abs_diff_host) *max_abs_diff_host = md;
  if (bad) return fail(GW_ENOTFINITE, "gw_mix: non-finite self-energy");
  return GW_OK;
}

int gw_profile_enable(gw_ctx* ctx, int on) {
  if (!ctx) return fail(GW_EINVAL, "gw_profile_enable: null context");
  ctx->prof.reset();
  ctx->prof.on = on != 0;
  return GW_OK;
}

long long gw_launch_count(const gw_ctx* ctx) { return ctx ? ctx->prof.launches : -1; }

int gw_profile_slots(void) { return SLOT_COUNT; }

int gw_profile_read(gw_ctx* ctx, int slot, char* name, int name_cap, long long* launches, double* total_ms,
                    double* flops, double* bytes) {
  if (!ctx || slot < 0 || slot >= SLOT_COUNT) return fail(GW_EINVAL, "gw_profile_read: bad argument");
  ctx->prof.drain();
  if (name && name_cap > 0) {
    std::strncpy(name, prof_slot_name(slot), (size_t)name_cap - 1);
    name[name_cap - 1] = 0;
  }
  if (launches) *launches = ctx->prof.slot_launches[slot];
  if (total_ms) *total_ms = ctx->prof.slot_ms[slot];
  if (flops) *flops = ctx->prof.slot_flops[slot];
  if (bytes) *bytes = ctx->prof.slot_bytes[slot];
  return GW_OK;
}

int gw_synchronize(gw_ctx* ctx) {
  if (!ctx) return fail(GW_EINVAL, "gw_synchronize: null context");
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_check("gw_synchronize");
  int st[4] = {0, 0, 0, 0};
  cudaMemcpy(st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (st[0] || st[1] || st[2] || st[3]) {
    cudaMemset(ctx->status, 0, sizeof(st));
    if (st[1]) return fail(GW_EDEVTIMEOUT, "a device-side wait gave up (code %d)", st[1]);
    if (st[0]) return fail(GW_EINVAL, "a Dyson matrix was singular");
    return fail(GW_ECUDA, "device status %d %d", st[2], st[3]);
  }
  return cuda_check("gw_synchronize");
}

}  // extern "C"
