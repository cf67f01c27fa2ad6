/*
 * gw.h -- C ABI of the GB300 (sm_103a) GW self-energy library.
 *
 * The library evaluates the dynamical GW self-energy of fully self-consistent
 * finite-temperature GW with density-fitted Coulomb integrals
 * (arXiv 2406.18479, Sec. 2.3, Eqs. tilde_P0_tau, P0t_to_P0w, tilde_P_omega,
 * tilde_W_DF2, sigma_gw) and the Dyson update of G (Sec. 2.5, Eq. dyson), and the
 * rest of the self-consistency loop around them (Sec. 2.4: the static part,
 * Eq. sigma_inf; the chemical potential; mixing, DIIS and CDIIS, Sec. 5.3), the
 * second-order self-energy (Eq. sigma2), Hartree-Fock, IR and Chebyshev grids and
 * the k-space interpolation of Sec. 2.5.
 *
 * Conventions shared by every call
 * --------------------------------
 * Complex numbers are interleaved (re, im) doubles (gw_c128). All arrays are
 * row-major and dense:
 *   V    [nk][nk][naux][nao][nao]   V[k1][k2][Q][i][j] = V_{k1 i, k2 j}(Q)   (Eq. CoulombDF)
 *   G    [nk][ntau][nao][nao]       G^k_ij(tau_t), tau_t first-kind Chebyshev nodes on [0, beta]
 *   H    [nk][nao][nao]
 *   P0t, Pt   [nk][ntau][naux][naux]      bosonic, indexed by q
 *   P0w, Pw   [nk][nw_b][naux][naux]      nw_b = gw_sample_count(ntau, 0)
 *   Sig  [nk][ntau][nao][nao]
 * k is the flat index (n1*N2 + n2)*N3 + n3 of the Gamma-centred mesh
 * k = 2 pi (n1/N1, n2/N2, n3/N3); k +- q is taken modulo the mesh.
 * With gw_config.v_packed = 1, V holds only the pairs k1 <= k2,
 *   Vp   [nk (nk + 1) / 2][naux][nao][nao]  in the order (0,0), (0,1), .., (0,nk-1), (1,1), ..,
 * and the library takes V^{k2 k1}_ij(Q) = conj V^{k1 k2}_ji(Q) (the k1 <-> k2 symmetry of the
 * density-fitted Coulomb factor, Eq. CoulombDF with real auxiliary functions): about half the
 * memory of V for solids.
 *
 * Pointers named *_dev are device pointers owned by the caller (for example
 * torch tensors); the library never frees them and reads or writes them only
 * on the context's stream, so results are valid in stream order. Pointers
 * named *_host are host memory, read or written synchronously. The library
 * owns its own workspaces, allocated in gw_create.
 *
 * Every call returns a gw_status. On failure the call leaves its outputs
 * undefined and gw_last_error() returns a thread-local message. Nothing is
 * thrown across the ABI.
 *
 * Threads: a context, a DIIS subspace or a batch is used by one thread at a time
 * (its calls are ordered on its stream); different objects may be used from
 * different threads at once. The server's calls (gw_submit, gw_poll, ...) may come
 * from any thread. Host-only calls (gw_grid_build, gw_ir_grids, gw_checkpoint_*,
 * gw_sample_count, the *_bytes queries) need no device.
 */
#ifndef GW_GB300_H
#define GW_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } gw_c128;

typedef enum {
  GW_OK = 0,
  GW_EINVAL = 1,        /* bad argument (null pointer, size out of range) */
  GW_ENOMEM = 2,        /* workspace does not fit the budget or cudaMalloc failed */
  GW_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  GW_ETIMEOUT = 4,      /* host-side wait ran out of time */
  GW_EDEVTIMEOUT = 5,   /* a device-side bounded wait gave up; the kernel returned early */
  GW_ENOTFINITE = 6,    /* a non-finite value was found where the call checks for one */
  GW_ENOTCONV = 7,      /* iteration limit reached without convergence */
  GW_EAGAIN = 8,        /* result not ready yet */
  GW_ENOTIMPL = 9       /* not implemented for this configuration */
} gw_status;

typedef enum {
  GW_FP64 = 0,          /* every contraction in FP64 */
  GW_MIXED_BF16X4 = 1,  /* V.G.V contractions on tcgen05 tensor cores: each operand row is cut,
                           per chunk of at most 256 k, into four bf16 slices on one power-of-two
                           alignment; slice products of order 0 and 1 sum exactly in their own
                           FP32 accumulators, orders 2-3 share a third, higher orders are dropped
                           (2^-32 relative); transforms, Dyson solves and the Sigma accumulation
                           stay FP64 */
  GW_MIXED_BF16X3 = 1   /* former name of GW_MIXED_BF16X4 (the scheme always had four slices) */
} gw_precision;
/* Value 2 (a single FP16 operand per tile with a power-of-two scale) is not a precision of this
 * library: its error, about 1e-4 of max|Sigma|, is five orders of magnitude above the 1e-6 Ha
 * target; gw_create rejects it with GW_EINVAL. */

/*
 * Where the mixed precisions keep the bf16 slices of V: for all nk^2 (k1, k2) pairs, made
 * once by gw_set_coulomb (GW_V_ALL_PAIRS), or for the 4 nk pairs of one q at a time, made
 * before each q from V (GW_V_PER_Q: about nk times less memory, V read again per q).
 * GW_V_AUTO takes all pairs when they need at most 24 GiB. Results are the same either way.
 */
enum { GW_V_AUTO = 0, GW_V_ALL_PAIRS = 1, GW_V_PER_Q = 2 };

typedef struct {
  int nk[3];            /* k-mesh N1, N2, N3 (1,1,1 for a molecule) */
  int nao;              /* orbitals, 1..512 */
  int naux;             /* auxiliary functions, 1..4096 */
  int ntau;             /* Chebyshev tau nodes, 1..512 */
  double beta;          /* inverse temperature (1/Ha), > 0 */
  double mu;            /* chemical potential (Ha), used by gw_dyson_G */
  double spin_factor;   /* spin sum of Eq. tilde_P0_tau: 2 for spin-restricted G */
  int precision;        /* gw_precision */
  int tau_chunk;        /* tau nodes per batch in the contractions; 0 = automatic */
  int v_slices;         /* mixed precisions: GW_V_AUTO, GW_V_ALL_PAIRS or GW_V_PER_Q */
  int v_packed;         /* 1: V holds the pairs k1 <= k2 only (layout above). FP64 keeps a full
                           working copy in the context; the mixed precisions unpack the blocks
                           they slice (all pairs once, through a transient buffer, or the nk
                           blocks of one q at a time) and keep no FP64 copy */
  int slice_pass;       /* mixed precisions: 0 = the V.G products and R write the next
                           contraction's bf16 slices from their epilogue where the sizes allow
                           (nao % 4 == 0, nao <= 56, naux % 40 == 0), 1 = always through FP64-range
                           intermediates and a separate slicing pass. Both meet the same error
                           bound; their results differ by rounding order (the chunks differ). */
  int tile_n;           /* mixed precisions: output columns per tile of the P0, R and V.G GEMMs
                           whose width the slice-output layout does not fix: 0 = automatic (72
                           where that pads the columns less than 80, else 80), or 56, 72 or 80.
                           Results are the same for every width (gw_batch_autotune times them). */
} gw_config;

/* Library version string. */
const char* gw_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char* gw_last_error(void);

/*
 * Number of sampled Matsubara frequencies for an ntau-node grid: ntau, or ntau+1
 * where the parity differs from that of a set symmetric under w -> -w (odd for
 * bosons, stat = 0; even for fermions, stat = 1). Returns -1 on bad input.
 */
int gw_sample_count(int ntau, int stat);

/*
 * Host-only grid builder for the Fourier integral of Eq. P0t_to_P0w (bosonic,
 * w_n = 2 n pi / beta, Sec. 2.3) or of G and Sigma (fermionic,
 * w_n = (2n+1) pi / beta, Eq. dyson). Writes, for nw = gw_sample_count(ntau, stat):
 *   tau_host[ntau]      Chebyshev nodes (beta/2)(1 - cos(pi (j + 1/2)/ntau))
 *   idx_host[nw]        sampled Matsubara indices n (ascending, symmetric in w)
 *   F_host[nw][ntau]    X(i w_n) = sum_t F_nt X(tau_t) for the Chebyshev interpolant
 *   B_host[ntau][nw]    least-squares left inverse of F (B F = I)
 * Any output pointer may be NULL. Needs no GPU.
 */
int gw_grid_build(int ntau, double beta, int stat, double* tau_host, int64_t* idx_host,
                  gw_c128* F_host, gw_c128* B_host);

typedef struct gw_ctx gw_ctx;

/*
 * Creates a context for one problem size on the current CUDA device, bound to
 * cuda_stream (a cudaStream_t; NULL = the legacy default stream). Builds the
 * bosonic and fermionic grids and allocates every workspace. *out is NULL on
 * failure.
 */
int gw_create(gw_ctx** out, const gw_config* cfg, void* cuda_stream);

/* Synchronizes the context's stream and frees its workspaces. NULL is a no-op. */
int gw_destroy(gw_ctx* ctx);

/* Bytes of device memory the context owns. */
size_t gw_workspace_bytes(const gw_ctx* ctx);

/*
 * Intermediate-representation (IR) grids for gw_set_grids (the paper runs on IR grids with
 * Lambda = beta omega_max = 1e4; its grid files are not available and are built here, on the
 * host): the basis u_l(tau) = sqrt(2/beta) U_l(2 tau / beta - 1) of the singular value
 * expansion of the logistic kernel exp(-Lambda y (x + 1) / 2) / (1 + exp(-Lambda y)), the
 * L = *ntau_out functions with s_l / s_0 > eps; tau nodes at the L roots of U_L (mirror
 * symmetric); Matsubara samples where the transform of u_L changes sign, mirrored and trimmed
 * or padded to gw_sample_count(L, stat) (padding by the smallest ||F||_F ||F^+||_F);
 * F = u^(samples) U_tau^{-1} maps node values to Matsubara values, B is its least-squares
 * left inverse. Both statistics share the tau nodes. Output layouts as gw_set_grids takes
 * them, for T = L, nb = gw_sample_count(T, 0), nf = gw_sample_count(T, 1): tau [T],
 * Fb [nb][T], Bb [T][nb], Ff [nf][T], Bf [T][nf], omega_b [nb], omega_f [nf] (host buffers of
 * at least those sizes for T = cap; omega_* may be NULL). tau_host = NULL: only *ntau_out.
 * 1 <= lambda <= 1e6, 1e-15 <= eps <= 1e-2; GW_EINVAL if L > cap. Seconds of host time at
 * Lambda = 1e4 (one SVD per call).
 */
int gw_ir_grids(double beta, double lambda, double eps, int cap, int* ntau_out, double* tau_host, gw_c128* Fb_host,
                gw_c128* Bb_host, gw_c128* Ff_host, gw_c128* Bf_host, double* omega_b_host, double* omega_f_host);

/*
 * Replaces the context's grids (built by gw_create from the Chebyshev interpolant, see
 * gw_grid_build) with the caller's, for example transforms of another basis (the paper's
 * grid files, Sec. 2.3 and Eq. P0t_to_P0w). Host arrays, copied; sizes as gw_create made
 * them: T = ntau nodes, nb = gw_sample_count(ntau, 0), nf = gw_sample_count(ntau, 1):
 *   tau_host[T], Fb_host[nb][T], Bb_host[T][nb] (bosonic), Ff_host[nf][T], Bf_host[T][nf]
 *   and omega_f_host[nf] (fermionic, used by gw_dyson_G), omega_b_host[nb] (optional, checked only).
 * G(beta - tau) is read at the mirrored node and only canonical (q, tau), (q, n) are computed,
 * so the grids must be symmetric: tau ascending in (0, beta) with tau[T-1-t] = beta - tau[t],
 * omega_b[nb-1-n] = -omega_b[n], and Fb[nb-1-n][T-1-t] = Fb[n][t], Bb[T-1-t][nb-1-n] = Bb[t][n]
 * (relative 1e-10); GW_EINVAL otherwise. Synchronizes the context's stream first.
 */
int gw_set_grids(gw_ctx* ctx, const double* tau_host, const gw_c128* Fb_host, const gw_c128* Bb_host,
                 const gw_c128* Ff_host, const gw_c128* Bf_host, const double* omega_b_host,
                 const double* omega_f_host);

/*
 * Borrows the Coulomb factor V (layout above, Eq. CoulombDF; packed when cfg.v_packed). The
 * caller keeps V_dev alive and unchanged until gw_destroy or the next gw_set_coulomb. In the
 * mixed precisions this call also cuts V into its bf16 slices (a device workspace), or,
 * with per-q slices, only records V. A packed V is unpacked here into the context's FP64
 * copy (FP64 precision) or, for all-pair slices, into a transient buffer.
 */
int gw_set_coulomb(gw_ctx* ctx, const gw_c128* V_dev);

/*
 * Step (a), Eq. tilde_P0_tau (Sec. 2.3):
 *   P0^q_QQ'(tau) = -(s/N_k) sum_k sum_abcd V^{k,k+q}_da(Q) G^k_cd(beta - tau)
 *                                          G^{k+q}_ab(tau) V^{k+q,k}_bc(Q'),
 * where G(beta - tau_t) is the mirrored node G[ntau-1-t] and s = spin_factor.
 * Reads G_dev, writes P0t_dev.
 */
int gw_polarization(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* P0t_dev);

/*
 * Grid transforms along the time axis of a batch of nbatch blocks:
 *   to_matsubara:  out[b][n][e] = sum_t F_nt in[b][t][e]   (in: [nbatch][ntau][nelem])
 *   to_tau:        out[b][t][e] = sum_n B_tn in[b][n][e]   (in: [nbatch][nw][nelem])
 * stat = 0 bosonic (Eq. P0t_to_P0w), 1 fermionic (Eq. dyson).
 */
int gw_to_matsubara(gw_ctx* ctx, int stat, const gw_c128* in_dev, gw_c128* out_dev,
                    int nbatch, long long nelem);
int gw_to_tau(gw_ctx* ctx, int stat, const gw_c128* in_dev, gw_c128* out_dev,
              int nbatch, long long nelem);

/*
 * Step (c), Eq. tilde_P_omega: Pw = (I - P0w)^{-1} P0w for every (q, n), by
 * Gauss-Jordan inversion with partial pivoting, Pw = (I - P0w)^{-1} - I.
 * P0w_dev and Pw_dev may be the same buffer.
 */
int gw_aux_dyson(gw_ctx* ctx, const gw_c128* P0w_dev, gw_c128* Pw_dev);

/* Steps (b)+(c)+back-transform: Pt = B (I - F P0t)^{-1} (F P0t). */
int gw_screened_interaction(gw_ctx* ctx, const gw_c128* P0t_dev, gw_c128* Pt_dev);

/*
 * Step (d), Eqs. sigma_gw and tilde_W_DF2 (Sec. 2.3):
 *   Sigma^k_ij(tau) = -(1/N_k) sum_q sum_QQ'ab V^{k,k-q}_ia(Q) G^{k-q}_ab(tau)
 *                                             P~^q_QQ'(tau) V^{k-q,k}_bj(Q').
 * W~ is never formed. Overwrites Sig_dev.
 */
int gw_self_energy(gw_ctx* ctx, const gw_c128* G_dev, const gw_c128* Pt_dev, gw_c128* Sig_dev);

/* One self-energy evaluation, steps (a)-(d), with P0 and P~ in context workspaces. */
int gw_sigma_eval(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* Sig_dev);

/*
 * The part of one evaluation that comes from the momentum transfers q in [q_begin, q_end).
 * Eq. sigma_gw is a sum over q, and P0^q (Eq. tilde_P0_tau), P~^q (Eq. tilde_P_omega) and the
 * transforms are computed per q, so the partial sums of disjoint ranges add up to the full
 * Sigma (up to rounding order): this is the unit by which the path shards over GPUs (each
 * rank a range, one sum of Sig over ranks), and the unit of sampled accuracy checks.
 *   Sig_dev [nk][ntau][nao][nao] is overwritten with
 *   -(1/N_k) sum_{q in range} sum_QQ'ab V^{k,k-q}_ia(Q) G^{k-q}_ab(tau) P~^q_QQ'(tau) V^{k-q,k}_bj(Q').
 * A q whose -q lies in the range uses the symmetry P0^q(beta - tau) = P0^{-q}(tau)^T as
 * gw_sigma_eval does; a q whose -q lies outside is computed at every tau node and frequency.
 * [0, nk) gives the result of gw_sigma_eval bit for bit. P0t_dev and Pt_dev (optional, null to
 * skip; device, [q_end - q_begin][ntau][naux][naux], caller-owned) receive P0^q(tau) and
 * P~^q(tau) of the range. GW_EINVAL for a range outside [0, nk) or with q_begin > q_end (an
 * empty range writes Sig = 0).
 */
int gw_sigma_eval_q(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* Sig_dev, int q_begin, int q_end,
                    gw_c128* P0t_dev, gw_c128* Pt_dev);

/*
 * Dyson equation, Eq. dyson (Sec. 2.5) with S = I and Sigma^inf = 0:
 *   G^k(i w_n) = [(i w_n + mu) I - H^k - Sigma^k(i w_n)]^{-1},
 * with Sigma(i w) = F^f Sigma(tau) and G(tau) = B^f G(i w) on the fermionic grid.
 * Reads H_dev [nk][nao][nao] and Sig_dev, writes G_dev.
 */
int gw_dyson_G(gw_ctx* ctx, const gw_c128* H_dev, const gw_c128* Sig_dev, gw_c128* G_dev);

/*
 * Overlap S^k of a non-orthogonal orbital basis, Eq. dyson: S_dev [nk][nao][nao] Hermitian positive
 * definite, borrowed (kept alive and unchanged by the caller), or NULL for S = I (the default).
 * With an overlap, gw_dyson_G solves G^k(i w_n) = [(i w_n + mu) S^k - H^k - Sigma^k(i w_n)]^{-1},
 * gw_particle_number counts (s/N_k) sum_k Re Tr gamma^k S^k, gw_find_mu uses both, and
 * gw_commutator_residual returns S G F - F G S (Pulay's F D S - S D F up to sign).
 */
int gw_set_overlap(gw_ctx* ctx, const gw_c128* S_dev);

/*
 * Iteration mixing (Sec. 5.3): Sig_inout <- alpha Sig_new + (1 - alpha) Sig_inout, and
 * *max_abs_diff_host = max |Sig_inout(after) - Sig_inout(before)| over all elements.
 * Synchronizes the stream to return the norm. Returns GW_ENOTFINITE if the
 * mixed self-energy holds a NaN or infinity.
 */
int gw_mix(gw_ctx* ctx, const gw_c128* Sig_new_dev, gw_c128* Sig_inout_dev, double alpha,
           double* max_abs_diff_host);

/*
 * Kernel accounting. Every kernel launch of a context is counted. With
 * profiling on, CUDA events on the context's stream also bracket each launch,
 * and each kernel class ("slot") accumulates its device time and its
 * algorithmic flops and bytes. gw_profile_enable resets all counters.
 * gw_profile_read synchronizes the recorded events; name receives the slot's
 * kernel name (at most name_cap bytes with the terminator).
 */
int gw_profile_enable(gw_ctx* ctx, int on);
long long gw_launch_count(const gw_ctx* ctx);
int gw_profile_slots(void);
int gw_profile_read(gw_ctx* ctx, int slot, char* name, int name_cap, long long* launches,
                    double* total_ms, double* flops, double* bytes);

/*
 * P0(tau) of gw_polarization (FP64) for callers that cannot allocate device memory when they
 * call. Some hosts reserve all the device memory they will use at start-up and hand it to
 * their own pools (a serving runtime sized to the GPU's HBM), so a later cudaMalloc fails or
 * would break their accounting; some embedding runtimes forbid allocation after
 * initialisation; and some latency-critical loops cannot afford the device-wide
 * synchronisation that cudaMalloc and cudaFree may imply. This entry point has no counterpart
 * in the paper; it is an allocation-free form of step (a).
 *
 * Needs no context: sizes, spin factor, V_dev, G_dev and the output P0t_dev (layouts as above,
 * device memory of the current device, owned by the caller) are passed directly; work is
 * queued on cuda_stream (a cudaStream_t, NULL = legacy default stream). GW_EINVAL when a pointer
 * is null or not device memory of the current device. The V.G intermediates live in one fixed
 * 64 MiB device array inside the library, which every GPU that loads the library holds until
 * the process exits. The call rejects, with GW_EINVAL and a message, problems whose one
 * (tau, k) unit needs more than that array (2 * naux * nao^2 complex elements > 4 Mi); larger
 * problems split the k sum into chunks that fit and accumulate them into P0t_dev.
 *
 * The first call on a device looks up the array's device address (once per device, then kept
 * for the process): make that first call before any stream capture, and do not reset the
 * device between calls (a reset would move the array). All calls share the one array and
 * nothing in it needs to start at zero, so calls whose work overlaps on the GPU (different
 * streams or threads without ordering) race on it; order them on one stream. P0t_dev is
 * overwritten.
 */
int gw_polarization_noalloc(const int nk3[3], int nao, int naux, int ntau, double spin_factor,
                            const gw_c128* V_dev, const gw_c128* G_dev, gw_c128* P0t_dev,
                            void* cuda_stream);

/*
 * Checks the guard zones (256 bytes of 0xA5 after every workspace allocation of the context):
 * GW_ECUDA if any was overwritten, i.e. some kernel wrote past the end of a workspace. Synchronous.
 */
int gw_check_guards(gw_ctx* ctx);
/* Test hook: changes one byte of the index-th guard zone of the context (inside that allocation),
 * as a write past the end of the workspace would, so that gw_check_guards must report it. */
int gw_debug_mark_guard(gw_ctx* ctx, int index);

/*
 * Failure detection self-test (no counterpart in the paper): one thread waits, with the same
 * bounded mbarrier wait the tensor-core GEMM uses, on a phase that nothing completes. The wait
 * gives up after limit_s seconds (1e-3..10), records its code (*code_out = 99) and the kernel
 * returns: the call returns GW_EDEVTIMEOUT and the device stays usable. Synchronous.
 */
int gw_selftest_bounded_wait(double limit_s, int* code_out, void* cuda_stream);

/* Waits for all work queued on the context's stream. */
int gw_synchronize(gw_ctx* ctx);

/*
 * Second-order (GF2) self-energy, Eq. sigma2 (Sec. 2.2), with G^{k3}(-tau) = -G^{k3}(beta - tau)
 * (the mirrored node) and the momentum delta normalised to N_k:
 *   Sigma^k_ij(tau) = (1/N_k^2) sum_{k1 k2} sum_{QQ' klmnpq}
 *       [ s V^{k1 k}_qj(Q') V^{k2 k3}_ln(Q') - V^{k2 k}_lj(Q') V^{k1 k3}_qn(Q') ]
 *       V^{k k1}_ip(Q) V^{k3 k2}_mk(Q) G^{k1}_pq(tau) G^{k2}_kl(tau) G^{k3}_nm(beta - tau),
 * k3 = k1 + k2 - k, s = spin_factor. The direct (first) term is the GW self-energy contraction
 * with P0 in place of P~ (gw_polarization then gw_self_energy, in the context's precision); the
 * exchange term runs in FP64, contracted over Q and Q' first (2 nao^4 naux + nao^5 complex MACs
 * per (k, k1, k2, tau)), through a device workspace of at most about 2 GiB (fewer tau nodes per
 * batch with cfg.tau_chunk), allocated on first use. Writes Sig_dev [nk][ntau][nao][nao];
 * uses the context's P0 buffer. gw_gf2_exchange writes the exchange term alone,
 * (1/N_k^2) sum ... V^{k2 k}_lj(Q') V^{k1 k3}_qn(Q') ..., so that Sigma = direct - exchange.
 */
int gw_gf2_self_energy(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* Sig_dev);
int gw_gf2_exchange(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* SigX_dev);

/*
 * Density matrix gamma^k = G^k(0^-) = -G^k(beta^-), the G(0^-) of Eq. sigma_inf (Sec. 2.2).
 * The tau nodes exclude beta, so G(beta^-) is the polynomial through the ntau node values
 * evaluated at tau = beta: the Chebyshev series on the default grid, the interpolant of the
 * nodes given to gw_set_grids otherwise. Writes gamma_dev [nk][nao][nao].
 */
int gw_density(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* gamma_dev);

/*
 * Static self-energy, Eq. sigma_inf (Sec. 2.2), with gamma from G as in gw_density:
 *   Sigma^inf,k_ij = (s/N_k) sum_{k'Q ab} V^{kk}_ij(Q) gamma^{k'}_ab V^{k'k'}_ba(Q)
 *                  - (1/N_k) sum_{k'Q ab} V^{kk'}_ia(Q) gamma^{k'}_ab V^{k'k}_bj(Q),
 * s = spin_factor on the Hartree term only. FP64 in every precision. Writes SigInf_dev
 * [nk][nao][nao]. In the Dyson equation it enters like H: pass H + Sigma^inf to gw_dyson_G.
 */
int gw_sigma_inf(gw_ctx* ctx, const gw_c128* G_dev, gw_c128* SigInf_dev);

/*
 * Error vector of the commutator variant of DIIS (Sec. 5.3; Pulay's SCF commutator
 * F D S - S D F): with F = H^k + Sigma^inf,k + Sigma~^k(i w_n) on the fermionic samples,
 * e^k(i w_n) = [G^k(i w_n), F] = G F - F G, or S G F - F G S with an overlap (gw_set_overlap);
 * G(i w) = F^f G(tau), Sigma~(i w) = F^f Sigma~(tau). It vanishes when G solves the Dyson
 * equation with this (Sigma^inf, Sigma~) (and S). SigInf_dev may be NULL (zero).
 * Writes e_dev [nk][nw_f][nao][nao] (nw_f from gw_grid_build, statistics 1).
 */
int gw_commutator_residual(gw_ctx* ctx, const gw_c128* H_dev, const gw_c128* SigInf_dev, const gw_c128* Sig_dev,
                           const gw_c128* G_dev, gw_c128* e_dev);

/*
 * Wannier-like k-space interpolation (Sec. 2.5, without the maximally localised basis):
 *   X(R) = (1/N_k) sum_k X(k) e^{-i k R},   X(k') = sum_R w_R X(R) e^{i k' R},
 * k on the nk3 Gamma-centred mesh (flat order as everywhere), k' = 2 pi f' for the nkf
 * fractional coordinates f_host [nkf][3] (host, any values). R runs over the lattice vectors
 * nearest the origin, R_d in [-N_d/2, N_d/2]; for even N_d the two boundary vectors share one
 * term (w = 1/2 each, weights multiply over directions), so the interpolation is exact on the
 * mesh. X_dev [nk][nelem] -> Xf_dev [nkf][nelem] (any per-k block: Sigma~ [ntau][nao][nao],
 * Sigma^inf [nao][nao], ...), FP64, on cuda_stream (stream-ordered; no context needed). The
 * paper interpolates Sigma^inf and Sigma~ this way and evaluates H on the finer k set directly,
 * then solves the Dyson equation there (gw_dyson_G on a context whose nk equals nkf).
 */
int gw_k_interpolate(const int nk3[3], const gw_c128* X_dev, long long nelem, int nkf, const double* f_host,
                     gw_c128* Xf_dev, void* cuda_stream);

/* Sets the chemical potential used by gw_dyson_G. */
int gw_set_mu(gw_ctx* ctx, double mu);

/* Electrons per cell (s/N_k) sum_k Re Tr gamma^k S^k of G (S = I without an overlap; synchronous). */
int gw_particle_number(gw_ctx* ctx, const gw_c128* G_dev, double* n_host);

/*
 * Sec. 2.4 step 3: the chemical potential in [mu_lo, mu_hi] whose Dyson solution
 * G = Dyson(Heff, Sigma, mu) (Heff = H + Sigma^inf) holds n_target electrons per cell,
 * to tol (the particle number grows with mu): a bracketing search, regula falsi with the Illinois
 * modification and a bisection step whenever two steps have not halved the bracket. Writes
 * G_dev (the solution at the returned mu), *mu_host, and sets the context's mu. GW_EINVAL if
 * n_target lies outside [N(mu_lo), N(mu_hi)]. Synchronous; every step is one gw_dyson_G.
 */
int gw_find_mu(gw_ctx* ctx, const gw_c128* Heff_dev, const gw_c128* Sig_dev, double n_target, double mu_lo,
               double mu_hi, double tol, gw_c128* G_dev, double* mu_host);

/*
 * Convergence acceleration by direct inversion in the iterative subspace (Sec. 5.3), the
 * Pulay form: push the self-energy Sigma_i an iteration's G was built from and the one
 * computed from that G, Sigma[G_i]; extrapolate gives sum_i c_i Sigma[G_i] with c minimising
 * |sum_i c_i r_i|^2 subject to sum_i c_i = 1, r_i = Sigma[G_i] - Sigma_i (real c, inner
 * products Re <r_i, r_j> over all complex entries). With n_residual > 0 the residuals are the
 * caller's, n_residual entries each, given to gw_diis_push_residual (the commutator variant
 * passes gw_commutator_residual); n_residual = 0 takes r_i = Sigma[G_i] - Sigma_i through
 * gw_diis_push. At most max_vectors (1..16) are kept, the oldest leaves first. Vectors are
 * copied; work runs on cuda_stream (a push synchronizes it).
 */
typedef struct gw_diis gw_diis;
int gw_diis_create(gw_diis** out, long long n_elem, long long n_residual, int max_vectors, void* cuda_stream);
int gw_diis_destroy(gw_diis* diis);
int gw_diis_push(gw_diis* diis, const gw_c128* sigma_in_dev, const gw_c128* sigma_out_dev);
int gw_diis_push_residual(gw_diis* diis, const gw_c128* sigma_out_dev, const gw_c128* residual_dev);
/* coeffs_host (optional, max_vectors doubles) and *nvec_host (optional) receive c, oldest first. */
int gw_diis_extrapolate(gw_diis* diis, gw_c128* out_dev, double* coeffs_host, int* nvec_host);

/*
 * The self-consistency loop of Sec. 2.4 on one context. Iteration n takes G_{n-1} and
 *   (1) evaluates the output F_n = (Sigma^inf[G], Sigma~[G]) (gw_sigma_inf, and gw_sigma_eval or
 *       gw_gf2_self_energy by method; Sigma^inf = 0 with static_part = 0);
 *   (2) accelerates (Sec. 5.3): Sigma_1 = F_1; then Sigma_n = alpha F_n + (1 - alpha) Sigma_{n-1},
 *       or with diis_size > 0 Pulay's extrapolation over the newest diis_size pairs
 *       (Sigma_{i-1}, F_i) from iteration diis_start on (earlier iterations mix and fill the
 *       subspace; gw_diis_*), with the residual F_i - Sigma_{i-1} or the commutator of G_{i-1}
 *       and F_i (diis_kind);
 *   (3) with n_electrons > 0, finds mu in [mu_lo, mu_hi] (to mu_tol) whose Dyson solution holds
 *       n_electrons per cell (gw_find_mu); otherwise keeps the context's mu;
 *   (4) G_n = Dyson(H + Sigma^inf_n, Sigma~_n, mu) (gw_dyson_G).
 * (Sigma^inf, Sigma~) is one vector for mixing, DIIS and the stop test max |Sigma_n - Sigma_{n-1}|
 * < tol. G_dev holds G_0 on entry and the last G on return; Sigma_dev [nk][ntau][nao][nao] and
 * SigInf_dev [nk][nao][nao] receive the last Sigma_n (either may be NULL). The loop allocates
 * gw_scgw_bytes() of device memory for its duration and synchronizes the context's stream.
 * GW_ENOTCONV after itermax evaluations without convergence (outputs and *res still written).
 */
typedef struct {
  double alpha;               /* mixing weight in (0, 2) */
  double tol;                 /* stop threshold on max |dSigma| (Ha), >= 0 */
  int itermax;                /* self-energy evaluations at most, >= 1 */
  int static_part;            /* 1: include Sigma^inf (Eq. sigma_inf) */
  int diis_size;              /* 0: mixing only; 1..16: DIIS subspace size */
  int diis_start;             /* first extrapolating iteration, >= 2 */
  double n_electrons;         /* > 0: search mu each iteration for this many electrons per cell */
  double mu_lo, mu_hi, mu_tol;   /* bracket and tolerance of that search */
  int diis_kind;              /* 0: residual F_i - Sigma_{i-1}; 1: commutator (gw_commutator_residual
                                 of G_{i-1} and F_i) */
  int method;                 /* dynamic self-energy: 0 GW (gw_sigma_eval), 1 GF2 (gw_gf2_self_energy),
                                 2 none (Hartree-Fock: Sigma~ = 0, use with static_part = 1) */
  int resume;                 /* 1: Sigma_dev (and SigInf_dev with the static part) hold Sigma_{n-1}
                                 of a loop being continued and G_dev the G built from it; the first
                                 iteration then mixes with it (the DIIS subspace starts empty) */
} gw_scgw_options;

typedef struct {
  int iterations;             /* self-energy evaluations done */
  double max_abs_dsigma;      /* last max |dSigma| (0 after a single evaluation) */
  double mu;                  /* chemical potential of the last G */
  double n_electrons;         /* electrons per cell of the last G */
} gw_scgw_result;

size_t gw_scgw_bytes(const gw_config* cfg, const gw_scgw_options* opt);
int gw_scgw(gw_ctx* ctx, const gw_c128* H_dev, gw_c128* G_dev, gw_c128* Sigma_dev, gw_c128* SigInf_dev,
            const gw_scgw_options* opt, gw_scgw_result* res);

/*
 * Checkpoint files (host memory): a one-line JSON header with the sizes of cfg, beta, the spin
 * factor, mu and the iteration, and the names and element counts of narrays complex arrays,
 * followed by their raw little-endian complex128 values. Names: 1..64 of [A-Za-z0-9_].
 * gw_checkpoint_read fills the arrays it is asked for by name (each must be stored with exactly
 * that count; others are skipped) and the header fields (cfg_out keeps its precision, tau_chunk,
 * v_slices and v_packed); GW_EINVAL for a missing, malformed or truncated file. A loop is
 * continued from saved G, Sigma~ and Sigma^inf through gw_scgw's resume option.
 */
int gw_checkpoint_write(const char* path, const gw_config* cfg, double mu, int iteration, int narrays,
                        const char* const* names, const gw_c128* const* data_host, const long long* counts);
int gw_checkpoint_read(const char* path, gw_config* cfg_out, double* mu, int* iteration, int narrays,
                       const char* const* names, gw_c128* const* data_host, const long long* counts);

/*
 * Batched self-energy evaluation of many independent systems (molecules or k-meshes of
 * uneven size). One context per system on one of max_streams CUDA streams (chosen by
 * predicted cost, longest first onto the least-loaded stream). Modes of gw_batch_sigma_eval:
 *   GW_BATCH_SERIAL   one system after another (the per-system launch loop),
 *   GW_BATCH_STREAMS  all systems enqueued at once on their streams,
 *   GW_BATCH_GRAPH    the same work captured once into a CUDA graph and replayed as one
 *                     graph launch; recaptured when the G or Sigma pointers change (the
 *                     first call after creation or gw_batch_set_coulomb runs uncaptured),
 *   GW_BATCH_GROUPED  every system's evaluation up to the aux Dyson equation (Eq.
 *                     tilde_P_omega) on its stream, then the inversions of all systems'
 *                     (I - P0(i Omega)) matrices as launches over the ragged list of matrices,
 *                     one block per matrix, largest first (one launch for n <= 430, one for
 *                     430 < n <= 800; a system with naux > 800 inverts its own matrices
 *                     within its evaluation), then the rest of every evaluation on its stream,
 *   GW_BATCH_GROUPED_GRAPH  the grouped work captured into a graph as GW_BATCH_GRAPH does.
 * Every mode computes, per system, exactly what gw_sigma_eval computes alone. Calls are
 * asynchronous: the batch starts after the work queued on cuda_stream and cuda_stream waits
 * for the batch. V, G and Sigma are caller-owned device arrays per system, laid out as for
 * gw_sigma_eval; the pointer arrays themselves are host arrays of n entries, read during
 * the call.
 */
typedef struct gw_batch gw_batch;
enum { GW_BATCH_SERIAL = 0, GW_BATCH_STREAMS = 1, GW_BATCH_GRAPH = 2, GW_BATCH_GROUPED = 3, GW_BATCH_GROUPED_GRAPH = 4 };

/*
 * GW_EINVAL for n outside 1..4096 or max_streams outside 1..64. Systems whose tau_chunk is 0
 * get the largest equal tau batch whose device bytes fit their share of hbm_budget: each
 * system's need with all tau nodes in one batch, scaled by one common factor so that the
 * needs add up to the budget, and at least 256 MiB (hbm_budget 0 = 128 GiB).
 */
int gw_batch_create(gw_batch** out, const gw_config* cfgs, int n, int max_streams, size_t hbm_budget,
                    void* cuda_stream);
int gw_batch_destroy(gw_batch* batch);
int gw_batch_set_coulomb(gw_batch* batch, const gw_c128* const* V_dev);
int gw_batch_sigma_eval(gw_batch* batch, const gw_c128* const* G_dev, gw_c128* const* Sig_dev, int mode);
/*
 * Per-system tuner: times one evaluation of each system for equal tau batches of
 * ntau / {1, 2, 3, 4, 6, 8} nodes (the grid of the GEMM launches) that fit the system's
 * budget share, keeps the fastest; then, in the mixed precisions, times the tile widths
 * 0 (automatic), 56, 72 and 80 of gw_config.tile_n at that batch and keeps the fastest.
 * Systems of the same shape (mesh, nao, naux, ntau, precision, V layout, budget share) take
 * the choice of the first one tuned. Rebuilds the contexts. chosen (optional, n ints) receives
 * the tau batch sizes; gw_batch_tuned reports both choices. Blocks until done; Sigma_dev is
 * used as scratch. Every choice gives the same results.
 */
int gw_batch_autotune(gw_batch* batch, const gw_c128* const* G_dev, gw_c128* const* Sig_dev, int* chosen);
/* The tau batch and tile width system i runs with (after gw_batch_autotune: the tuned ones). */
int gw_batch_tuned(const gw_batch* batch, int i, int* tau_chunk, int* tile_n);
/* Waits for the batch and reports any device-side failure of its contexts. */
int gw_batch_synchronize(gw_batch* batch);

/*
 * Request loop for scGW jobs (the self-consistency loop of Sec. 2.4, gw_scgw).
 *
 * A job runs gw_scgw on its own context, CUDA stream and device buffers, with the options
 * in gw_job: with the loop options all zero, at fixed mu without the static part,
 *   it = 1:  Sigma = Sigma[G0]                              (gw_sigma_eval)
 *   it > 1:  Sigma <- alpha Sigma[G] + (1 - alpha) Sigma     (iteration mixing, Sec. 5.3)
 *   then     G = Dyson(H, Sigma)                            (gw_dyson_G, Eq. dyson)
 * and stops when max |dSigma| < tol (it > 1) or after itermax evaluations; the options add
 * the static part, the mu search, DIIS or CDIIS, and GF2 in place of GW.
 *
 * gw_server_create starts max_slots worker threads on the current device. A
 * submitted job waits in arrival order until a slot is free and its device
 * memory (gw_job_bytes) fits in what is left of hbm_budget; jobs are admitted
 * while others run (continuous batching) and their kernels overlap on the GPU.
 * A job computes exactly what it computes alone. The host buffers named in
 * gw_job are borrowed until the job has finished (gw_poll returned GW_OK).
 */
typedef struct gw_server gw_server;

typedef struct {
  gw_config cfg;              /* sizes, beta, mu, spin factor, precision, tau chunk */
  const gw_c128* H_host;      /* [nk][nao][nao] */
  const gw_c128* V_host;      /* [nk][nk][naux][nao][nao], or packed with cfg.v_packed */
  const gw_c128* G0_host;     /* [nk][ntau][nao][nao], the starting Green's function */
  gw_c128* Sigma_out_host;    /* [nk][ntau][nao][nao] final Sigma, or NULL */
  gw_c128* G_out_host;        /* [nk][ntau][nao][nao] final G, or NULL */
  double alpha;               /* mixing weight in (0, 2) */
  double tol;                 /* convergence threshold on max |dSigma| (Ha) */
  int itermax;                /* self-energy evaluations at most, >= 1 */
  /* the rest of the loop of gw_scgw; all zero: fixed mu, no static part, mixing only */
  int static_part;
  int diis_size;
  int diis_start;
  double n_electrons;
  double mu_lo, mu_hi, mu_tol;
  int diis_kind;
  int method;
  const gw_c128* S_host;      /* [nk][nao][nao] overlap of Eq. dyson, or NULL for S = I */
} gw_job;

typedef struct {
  int status;                 /* GW_OK, GW_ENOTCONV (itermax reached), or the failing call's status */
  int iterations;             /* self-energy evaluations done */
  double max_abs_dsigma;      /* last max |dSigma| (0 after a single evaluation) */
  double t_submit, t_start, t_end;   /* seconds on the library's monotonic clock */
  double mu;                  /* chemical potential of the final G */
} gw_job_result;

/* Device bytes a job holds while it runs with the loop options all zero (0 for an invalid
 * configuration); gw_submit also counts the DIIS subspace a job's options ask for. */
size_t gw_job_bytes(const gw_config* cfg);

/* GW_EINVAL for max_slots outside 1..64 or a zero budget. */
int gw_server_create(gw_server** out, size_t hbm_budget, int max_slots);

/* Finishes the running jobs, drops the waiting ones, joins the workers, frees everything. */
int gw_server_destroy(gw_server* srv);

/* Non-blocking. GW_ENOMEM if the job can never fit the budget. */
int gw_submit(gw_server* srv, const gw_job* job, uint64_t* job_id);

/*
 * Result of a job. timeout_us = 0: does not wait (GW_EAGAIN while the job runs or
 * waits); > 0: waits at most that long (GW_ETIMEOUT); < 0: waits until it finishes.
 * GW_OK once the job has finished: *out then holds its status and timings.
 */
int gw_poll(gw_server* srv, uint64_t job_id, gw_job_result* out, int timeout_us);

#ifdef __cplusplus
}
#endif
#endif /* GW_GB300_H */
