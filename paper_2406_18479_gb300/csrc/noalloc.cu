// P0(tau) without any device allocation: gw_polarization_noalloc.
//
// For callers that cannot allocate device memory at the time of the call: a host that
// reserved all its device memory at start-up for its own pools, an embedding runtime that
// forbids allocation after initialisation, or a latency-critical loop that cannot take the
// synchronisation cudaMalloc may imply. Those callers pass inputs and outputs only; the
// intermediates of the V.G products live in one file-scope device array of fixed size.
//
// The computation is the FP64 path of gw_polarization (same kernels), with the k sum split
// into chunks that fit the array and accumulated into P0t.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <utility>

#include "gw_internal.h"

namespace gwi {

namespace {

// 64 MiB of scratch (4 Mi complex FP64 elements), held by every GPU that loads the library.
constexpr long long kScratchElems = 4LL * 1024 * 1024;
static __device__ __align__(256) double2 g_noalloc_scratch[kScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double2* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on device dev (looked up once per device and kept: the
// address stays valid until the device is reset, which callers must not do between calls).
int scratch_address(int dev, double2** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(GW_ECUDA, "gw_polarization_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(GW_ECUDA, "gw_polarization_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return GW_OK;
}

// GW_OK if p is device memory of device dev (a pointer from another device, host memory or an
// unknown address would make the kernels fault)
int check_device_ptr(const void* p, int dev, const char* what) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return fail(GW_EINVAL, "gw_polarization_noalloc: %s is not a CUDA pointer", what);
  }
  if (a.type != cudaMemoryTypeDevice || a.device != dev)
    return fail(GW_EINVAL, "gw_polarization_noalloc: %s is not device memory of the current device %d", what, dev);
  return GW_OK;
}

int kshift_na(const int nk3[3], int k, int q, int sign) {
  const int k1 = k / (nk3[1] * nk3[2]), k2 = (k / nk3[2]) % nk3[1], k3 = k % nk3[2];
  const int q1 = q / (nk3[1] * nk3[2]), q2 = (q / nk3[2]) % nk3[1], q3 = q % nk3[2];
  const int a = ((k1 + sign * q1) % nk3[0] + nk3[0]) % nk3[0];
  const int b = ((k2 + sign * q2) % nk3[1] + nk3[1]) % nk3[1];
  const int c = ((k3 + sign * q3) % nk3[2] + nk3[2]) % nk3[2];
  return (a * nk3[1] + b) * nk3[2] + c;
}

}  // namespace

}  // namespace gwi

using namespace gwi;

extern "C" int gw_polarization_noalloc(const int nk3[3], int nao, int naux, int ntau, double spin_factor,
                                       const gw_c128* V_dev, const gw_c128* G_dev, gw_c128* P0t_dev,
                                       void* cuda_stream) {
  if (!nk3 || !V_dev || !G_dev || !P0t_dev) return fail(GW_EINVAL, "gw_polarization_noalloc: null argument");
  if (nk3[0] < 1 || nk3[1] < 1 || nk3[2] < 1 || nao < 1 || naux < 1 || ntau < 1)
    return fail(GW_EINVAL, "gw_polarization_noalloc: sizes must be positive");
  const long long nk_ll = (long long)nk3[0] * nk3[1] * nk3[2];
  if (nk_ll > 65535) return fail(GW_EINVAL, "gw_polarization_noalloc: nk = %lld above 65535", nk_ll);
  const int nk = (int)nk_ll;
  const long long nao2 = (long long)nao * nao, pair = (long long)naux * nao2, naux2 = (long long)naux * naux;
  // one (tau, k) unit needs the A and B~ blocks of one k-point pair: 2 * naux * nao^2 elements
  if (2 * pair > kScratchElems)
    return fail(GW_EINVAL,
                "gw_polarization_noalloc: 2*naux*nao^2 = %lld complex elements exceed the fixed scratch of %lld "
                "(64 MiB); use gw_polarization with a context",
                2 * pair, kScratchElems);
  if ((long long)naux * nao > (1LL << 30)) return fail(GW_EINVAL, "gw_polarization_noalloc: problem too large");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(GW_ECUDA, "gw_polarization_noalloc: no usable current device");
  }
  for (const auto& pw : {std::make_pair((const void*)V_dev, "V_dev"), std::make_pair((const void*)G_dev, "G_dev"),
                         std::make_pair((const void*)P0t_dev, "P0t_dev")}) {
    const int rc = check_device_ptr(pw.first, dev, pw.second);
    if (rc != GW_OK) return rc;
  }
  double2* scratch = nullptr;
  const int rc0 = scratch_address(dev, &scratch);
  if (rc0 != GW_OK) return rc0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double2* V = reinterpret_cast<const double2*>(V_dev);
  const double2* G = reinterpret_cast<const double2*>(G_dev);
  double2* P0t = reinterpret_cast<double2*>(P0t_dev);
  // units per round: nt taus x kc k-points, with 2 * nt * kc * pair <= scratch
  const long long units = kScratchElems / (2 * pair);
  const int kc = (int)std::min<long long>(nk, units);
  const int nt = (int)std::max<long long>(1, std::min<long long>(ntau, units / kc));
  double2* Abuf = scratch;
  double2* Bbuf = scratch + (long long)nt * kc * pair;
  for (int q = 0; q < nk; ++q) {
    for (int t0 = 0; t0 < ntau; t0 += nt) {
      const int ntc = std::min(nt, ntau - t0);
      for (int k0 = 0; k0 < nk; k0 += kc) {
        const int kcc = std::min(kc, nk - k0);
        for (int kk = 0; kk < kcc; ++kk) {
          const int k = k0 + kk, kp = kshift_na(nk3, k, q, +1);
          {  // A^Q_{db}(k,t) = sum_a V^{k,k+q}_da(Q) G^{k+q}_ab(t), into Abuf[t][kk]
            ZGemm g;
            g.M = naux * nao; g.N = nao; g.K = nao; g.nbatch = ntc;
            g.A = V + ((long long)k * nk + kp) * pair; g.va.rs_in = nao; g.va.ks_in = 1;
            g.B = G + ((long long)kp * ntau + t0) * nao2; g.vb.rs_in = 1; g.vb.ks_in = nao; g.bb.bs_in = nao2;
            g.C = Abuf + (long long)kk * pair; g.vc.rs_in = nao; g.vc.ks_in = 1; g.bc.bs_in = (long long)kc * pair;
            g.slot = SLOT_VG_FP64;
            const int rc = zgemm_fp64(g, st);
            if (rc != GW_OK) return rc;
          }
          {  // B^{Q'}_{bd}(k,t) = sum_c V^{k+q,k}_bc(Q') G^k_cd(beta - t), stored [Q'][d][b]
            ZGemm g;
            g.M = naux * nao; g.N = nao; g.K = nao; g.nbatch = ntc;
            g.A = V + ((long long)kp * nk + k) * pair; g.va.rs_in = nao; g.va.ks_in = 1;
            g.B = G + ((long long)k * ntau + (ntau - 1 - t0)) * nao2; g.vb.rs_in = 1; g.vb.ks_in = nao;
            g.bb.bs_in = -nao2;
            g.C = Bbuf + (long long)kk * pair; g.vc.rin = nao; g.vc.rs_in = 1; g.vc.rs_out = nao2; g.vc.ks_in = nao;
            g.bc.bs_in = (long long)kc * pair;
            g.slot = SLOT_VG_FP64;
            const int rc = zgemm_fp64(g, st);
            if (rc != GW_OK) return rc;
          }
        }
        {  // P0^q_QQ'(t) (+)= -(s/N_k) sum_{k in chunk, d, b} A^Q_{db} B^{Q'}_{bd}
          ZGemm g;
          g.M = naux; g.N = naux; g.K = kcc * (int)nao2; g.nbatch = ntc;
          g.A = Abuf; g.va.rs_in = nao2; g.va.kin = (int)nao2; g.va.ks_in = 1; g.va.ks_out = pair;
          g.ba.bs_in = (long long)kc * pair;
          g.B = Bbuf; g.vb = g.va; g.bb = g.ba;
          g.C = P0t + ((long long)q * ntau + t0) * naux2; g.vc.rs_in = naux; g.vc.ks_in = 1; g.bc.bs_in = naux2;
          g.alpha = -spin_factor / nk;
          g.accumulate = k0 > 0;       // the first k chunk overwrites: nothing in P0t must start at zero
          g.slot = SLOT_P0_FP64;
          const int rc = zgemm_fp64(g, st);
          if (rc != GW_OK) return rc;
        }
      }
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "gw_polarization_noalloc: %s", cudaGetErrorString(e));
}
