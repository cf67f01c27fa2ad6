// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <string>
#include <complex>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <vector_types.h>

#include "gw.h"

namespace gwi {

// ---- host utilities (grids.cpp, errors in gw_api.cu)
int sample_count(int ntau, int stat);
// Householder QR least-squares left inverse of A (m x n, m >= n, row-major complex): B A = I
bool lsq_left_inverse(const std::vector<std::complex<double>>& A, int m, int n, std::vector<std::complex<double>>& B);
std::vector<int64_t> matsubara_indices(int n, int stat);
int grid_build(int ntau, double beta, int stat, double* tau, int64_t* idx, gw_c128* F, gw_c128* B);
int fail(int code, const char* fmt, ...);

// Guard zones: every workspace allocation carries kGuardBytes of kGuardByte after its end, checked
// by gw_check_guards; an out-of-bounds write past a workspace shows up there.
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;
// number of guards of [guards, guards + n) that differ from the pattern; *first <- index of the first
int check_guards(unsigned char* const* guards, int n, int* first, void* stream);

// NVTX range over a scope (a no-op unless a tracing tool is attached): the ABI's stages show up
// by name on a timeline
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Device bytes of one scGW job: its context's workspaces (counted by running the
// context build in size-only mode) plus V, H, G and two Sigma buffers. 0 for an
// invalid configuration.
size_t job_device_bytes(const gw_config* cfg);

// ---- kernel timing and launch counting (gw_api.cu)
//
// Every kernel launch goes through prof_begin/prof_end with a slot naming the
// kernel. The launch counter always runs; when the context's profiling is on,
// CUDA events on the launching stream bracket each launch and the slot
// accumulates its algorithmic flops and bytes.
enum ProfSlot {
  SLOT_VG_FP64 = 0, SLOT_P0_FP64, SLOT_R_FP64, SLOT_SIGMA_FP64, SLOT_TRANSFORM_FP64, SLOT_INVERSE_FP64,
  SLOT_ELEMENTWISE, SLOT_LIMBS, SLOT_VG_MIXED, SLOT_P0_TC, SLOT_R_TC, SLOT_SIGMA_MIXED, SLOT_REDUCE,
  SLOT_STATIC_FP64, SLOT_GF2_FP64, SLOT_GF2_TC, SLOT_COUNT
};
const char* prof_slot_name(int slot);
void prof_begin(int slot, cudaStream_t s);
void prof_end(int slot, cudaStream_t s, double flops, double bytes);

// ---- batched complex FP64 GEMM (k_fp64.cu)
//
// Operand view: element (r, k) of a matrix sits at
//   base + (r / rin) * rs_out + (r % rin) * rs_in + (k / kin) * ks_out + (k % kin) * ks_in.
// Two-level row and k indices express the (k-point, orbital) and (Q, orbital)
// flattenings of the GW contractions without copies.
struct ZView {
  long long rs_in = 0, rs_out = 0;
  long long ks_in = 0, ks_out = 0;
  int rin = 1 << 30, kin = 1 << 30;
};

// Batch index b -> (bo, bi) = (b / bin, b % bin); the operand's offset is
//   (tab ? tab[bi] : bi * bs_in) + bo * bs_out.
struct ZBatch {
  const long long* tab = nullptr;
  long long bs_in = 0, bs_out = 0;
};

struct ZGemm {
  int M = 0, N = 0, K = 0, nbatch = 1, bin = 1 << 30;
  const double2* A = nullptr;    // A(m, k)
  const double2* B = nullptr;    // B(n, k)
  double2* C = nullptr;          // C(m, n): rows per C.rs_*, columns with stride C.ks_in
  ZView va, vb, vc;
  ZBatch ba, bb, bc;
  double alpha = 1.0;            // C = alpha * sum_k A(m,k) B(n,k) (+ C if accumulate)
  int accumulate = 0;
  int slot = SLOT_VG_FP64;       // profiling slot of this launch
};

int zgemm_fp64(const ZGemm& g, void* stream);

// In-place Gauss-Jordan inversion with partial pivoting of nbatch n x n matrices
// (matrix b at base + b * stride). diag_shift: before inverting, M <- diag_sign*M + shift(b)*I
// is applied by the callers' build kernels instead; here only the inversion.
// list (optional, device): the matrix indices to process, nbatch of them.
int batched_inverse_fp64(double2* base, int n, long long stride, int nbatch, int* status_dev,
                         void* stream, const int* list = nullptr);

// One matrix of a grouped inversion: its pointer (n x n, row-major), size and status word.
// largest matrix the blocked Gauss-Jordan inversion takes with a 16-column panel and with an
// 8-column panel (its shared-memory footprint); larger ones take the unblocked kernel
constexpr int kGjBlockedMaxN16 = 430;
constexpr int kGjBlockedMaxN8 = 800;
struct GjItem {
  double2* M;
  int n;
  int* status;
};
// Gauss-Jordan inversion of a ragged list of matrices (items in device memory, count of them,
// the largest n at most 800) in one launch, one block per item in list order; flops for the
// profile. The panel width follows max_n (16 up to 430, else 8), as batched_inverse_fp64's does
// for one n, so a matrix gets bit for bit what a lone inversion of its size gives when both
// take the same panel width.
int batched_inverse_group_fp64(const GjItem* items_dev, int count, int max_n, double flops, void* stream);

// Aux Dyson pieces: M <- I - M; and after inversion M <- M - I.
int add_identity_fp64(double2* base, int n, long long stride, int nbatch, double scale_m,
                      double shift, void* stream, const int* list = nullptr);

// G Dyson build: A[k][n] = (i w_n + mu) S[k] - H[k] - Sw[k][n] (S = I when null; in place over Sw)
int build_g_dyson_fp64(double2* sw, const double2* H, const double2* S, const double* wn, double mu, int nk, int nw,
                       int nao, void* stream);

// Index pairs related by P0^q(beta - tau) = P0^{-q}(tau)^T (and the same for the frequency
// samples, which are symmetric): X[q][t] <- X[mq[q]][T-1-t]^T for every (q, t) that is not
// canonical; canonical (q, t): q < mq[q], or q == mq[q] and t <= T-1-t. X is [nk][T][n][n].
// With a range [q0, q1) (q1 < 0: nk) only q in the range whose -q is also in it are filled
// (a q whose -q lies outside was computed at every node).
int mirror_fill(double2* X, int nk, int T, int n, const int* mq_dev, void* stream, int q0 = 0, int q1 = -1);

// Static part and loop helpers (Eq. sigma_inf, Sec. 2.4, Sec. 5.3), all FP64:
//   density:  gamma^k = -sum_t w_t G^k(tau_t)          (w: weights of the interpolant at tau = beta)
//   hartree:  out^k = scale sum_Q V^{kk}(Q) rho_Q, rho_Q = sum_{k'ab} gamma^{k'}_ab V^{k'k'}_ba(Q)
//   trace:    *out = sum_k Re Tr gamma^k S^k (S = I when null);  add: c = a + b
//   dot_re:   *out = Re <x, y> (kDotBlocks partial sums, in a fixed order);  lincomb: out = sum_i c_i v_i
constexpr int kDotBlocks = 512;
int density_fp64(const double2* G, const double* w, double2* gamma, int nk, int ntau, int nao, void* stream);
int hartree_fp64(const double2* V, const double2* gamma, double2* rho, double2* out, int nk, int naux, int nao,
                 double scale, int packed, void* stream);
//   exchange: out^k += scale sum_{k'Q b} (V^{kk'}(Q) gamma^{k'})_ib V^{k'k}_bj(Q), for nao <= kExchangeMaxNao,
//             through part [nk][nk][exchange_chunks][nao][nao]
constexpr int kExchangeMaxNao = 52;
// out[o][e] += scale sum_{p < nparts} part[(o nparts + p)][e], e < n2, summed in the order of p
int reduce_partials_fp64(const double2* part, double2* out, int nouter, int n2, int nparts, double scale,
                         void* stream);
int exchange_chunks(int nk, int naux);
int exchange_fp64(const double2* V, const double2* gamma, double2* part, double2* out, int nk, int naux, int nao,
                  double scale, int packed, void* stream);

// The packed Coulomb factor (gw_config.v_packed): blocks k1 <= k2 only, in row order of the upper
// triangle; V^{k2 k1}_ij(Q) = conj V^{k1 k2}_ji(Q). unpack_v_fp64 writes full-layout blocks
// dst[b] = V^{k1 k2} for a list of pairs: decoded from full-layout offsets tab[b] (a device
// table), every pair in order (all), or up to four given pairs.
struct VPairs {
  const long long* tab = nullptr;
  int all = 0;
  int k1[4] = {0, 0, 0, 0}, k2[4] = {0, 0, 0, 0};
};
inline long long packed_pairs(int nk) { return (long long)nk * (nk + 1) / 2; }
int unpack_v_fp64(const double2* Vp, int nk, int nao, long long pair, const VPairs& L, int nblocks, double2* dst,
                  void* stream);
int trace_fp64(const double2* gamma, const double2* S, int nk, int nao, double* out_dev, void* stream);
int add_fp64(const double2* a, const double2* b, double2* c, long long n, void* stream);
int dot_re_fp64(const double2* x, const double2* y, long long n, double* partial_dev, double* out_dev, void* stream);
int lincomb_fp64(const double2* const* v, const double* c, int m, double2* out, long long n, void* stream);

// gw_sigma_eval in two parts around the aux Dyson inversions (for batches that invert the
// matrices of many systems in one launch): part 0 is P0, the forward transforms and I - P0 of
// the canonical (q, n); then the caller inverts the matrices inverse_items lists (in place, as
// batched_inverse_fp64 does); part 1 is (I - P0)^{-1} - I, the mirror fills, the back transforms
// and Sigma. Together they issue exactly the launches of gw_sigma_eval, in its order.
int sigma_eval_part(gw_ctx* ctx, const double2* G, double2* Sig, int part);
void inverse_items(gw_ctx* ctx, std::vector<GjItem>* items);

// sizes, stream and mu of a context (for host code outside the file that defines gw_ctx)
struct CtxInfo {
  void* stream;
  int nk, ntau, nao, nwf;
  double mu;
};
CtxInfo ctx_info(const gw_ctx* ctx);

// device bytes of the scGW loop's own buffers; job_device_bytes plus these for a serving job
size_t scgw_device_bytes(const gw_config* cfg, const gw_scgw_options* opt);

// Sig_inout = alpha*new + (1-alpha)*old; *maxdiff (device double) = max |change|; nonfinite flag
int mix_fp64(const double2* s_new, double2* s_inout, double alpha, long long n, double* maxdiff_dev,
             int* nonfinite_dev, void* stream);

}  // namespace gwi
