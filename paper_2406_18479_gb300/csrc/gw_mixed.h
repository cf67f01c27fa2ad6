// Mixed-precision contractions (tcgen05 tensor cores) of the GW path.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

namespace gwi {

struct MixedDims {
  int nk3[3] = {1, 1, 1};
  int nk = 1, nao = 0, naux = 0, ntau = 0, precision = 0, tau_chunk = 0, v_slices = 0, v_packed = 0;
  int fuse = 1;
  int tile_n = 0;                 // tile width of the free-width GEMMs (0: automatic)           // 1: slice-output epilogues where the sizes allow (nao % 4 == 0, nao <= 56, naux % 40 == 0)
  std::vector<int> mq;    // index of -q for every q
};

struct MixedState;

// status: the context's device status words (status[1] receives device-side wait failures).
// dry: count the workspace bytes into *bytes only; *out stays null.
int mixed_create(MixedState** out, const MixedDims& d, cudaStream_t stream, int* status, size_t* bytes,
                 bool dry = false);
void mixed_destroy(MixedState* s);
// appends the guard zones of the state's workspaces
void mixed_guards(const MixedState* s, std::vector<unsigned char*>* out);
// V: the full-layout Coulomb factor, or null with Vp the packed one (pairs k1 <= k2)
int mixed_set_coulomb(MixedState* s, const double2* V, const double2* Vp = nullptr);
// P0 of the q in [q0, q1): canonical tau nodes of the q whose -q is in the range too, every node
// of the others. Sigma from the q in [q0, q1) (Sig is overwritten with that partial sum).
int mixed_polarization(MixedState* s, const double2* G, double2* P0t, double spin_factor, int q0, int q1);
int mixed_self_energy(MixedState* s, const double2* G, const double2* Pt, double2* Sig, int q0, int q1);
// out[b][(a c)][(d e)] = sum_Q X[b][Q][a][c] Z[b][Q][d][e] on the tensor cores (FP64 output), for nb
// batches of n2 = nao^2 rows, K = naux; z_bs = 0: one Z for every batch.
int mixed_outer_q(MixedState* s, const double2* X, long long x_bs, const double2* Z, long long z_bs, int nb,
                  int n2, double2* out, long long out_bs);
// part[b][q][i][j] = sum_{m l} Y[b][(i q)][(m l)] W[b][(q m)][(l j)] on the tensor cores (FP64 output):
// the last product of the GF2 exchange, split over q, for nb batches.
int mixed_gf2_last(MixedState* s, const double2* Y, const double2* W, int nb, int nao, double2* part);
// launches the bounded-wait self-test (see gw_selftest_bounded_wait); *code receives the wait's code
int mixed_wait_selftest(double limit_s, int* code, cudaStream_t st);

}  // namespace gwi
