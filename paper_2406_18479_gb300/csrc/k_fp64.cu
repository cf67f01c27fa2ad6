// FP64 kernels of the GW self-energy path (the all-FP64 precision and the FP64
// stages of the mixed precisions).
//
// GB300 runs FP64 at about 2 DFMA per clock per SM, so these kernels are bound
// by the FP64 pipe: a 32x32 output tile per 256-thread block, staged through
// shared memory, keeps that pipe busy without deeper register blocking.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "gw_internal.h"

namespace gwi {

namespace {

constexpr int TM = 32, TN = 32, TK = 16;
constexpr long long kInvalid = LLONG_MIN;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ long long view_row(const ZView& v, int r) {
  return (long long)(r / v.rin) * v.rs_out + (long long)(r % v.rin) * v.rs_in;
}

__device__ __forceinline__ long long view_k(const ZView& v, int k) {
  return (long long)(k / v.kin) * v.ks_out + (long long)(k % v.kin) * v.ks_in;
}

__device__ __forceinline__ long long batch_off(const ZBatch& b, int bo, int bi) {
  return (b.tab ? b.tab[bi] : (long long)bi * b.bs_in) + (long long)bo * b.bs_out;
}

__global__ void __launch_bounds__(256) zgemm_fp64_kernel(const ZGemm g) {
  __shared__ double2 As[TK][TM + 1];
  __shared__ double2 Bs[TK][TN + 1];
  __shared__ long long rowA[TM], rowB[TN], kA[TK], kB[TK];

  const int b = blockIdx.z;
  const int bo = b / g.bin, bi = b % g.bin;
  const double2* A = g.A + batch_off(g.ba, bo, bi);
  const double2* B = g.B + batch_off(g.bb, bo, bi);
  double2* C = g.C + batch_off(g.bc, bo, bi);
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;

  if (tid < TM) {
    const int r = m0 + tid;
    rowA[tid] = r < g.M ? view_row(g.va, r) : kInvalid;
  } else if (tid < TM + TN) {
    const int r = n0 + tid - TM;
    rowB[tid - TM] = r < g.N ? view_row(g.vb, r) : kInvalid;
  }
  const bool a_kfast = g.va.ks_in == 1;
  const bool b_kfast = g.vb.ks_in == 1;

  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);

  for (int k0 = 0; k0 < g.K; k0 += TK) {
    __syncthreads();
    if (tid < TK) {
      const int k = k0 + tid;
      kA[tid] = k < g.K ? view_k(g.va, k) : kInvalid;
    } else if (tid < 2 * TK) {
      const int k = k0 + tid - TK;
      kB[tid - TK] = k < g.K ? view_k(g.vb, k) : kInvalid;
    }
    __syncthreads();
    for (int e = tid; e < TM * TK; e += 256) {
      const int mm = a_kfast ? e / TK : e % TM;
      const int kk = a_kfast ? e % TK : e / TM;
      const long long ro = rowA[mm], ko = kA[kk];
      As[kk][mm] = (ro != kInvalid && ko != kInvalid) ? A[ro + ko] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < TN * TK; e += 256) {
      const int nn = b_kfast ? e / TK : e % TN;
      const int kk = b_kfast ? e % TK : e / TN;
      const long long ro = rowB[nn], ko = kB[kk];
      Bs[kk][nn] = (ro != kInvalid && ko != kInvalid) ? B[ro + ko] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < TK; ++kk) {
      const double2 a0 = As[kk][2 * ty], a1 = As[kk][2 * ty + 1];
      const double2 b0 = Bs[kk][2 * tx], b1 = Bs[kk][2 * tx + 1];
      cmac(acc[0][0], a0, b0);
      cmac(acc[0][1], a0, b1);
      cmac(acc[1][0], a1, b0);
      cmac(acc[1][1], a1, b1);
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int m = m0 + 2 * ty + i;
    if (m >= g.M) continue;
    const long long ro = view_row(g.vc, m);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = n0 + 2 * tx + j;
      if (n >= g.N) continue;
      double2* c = C + ro + (long long)n * g.vc.ks_in;
      double2 v = make_double2(g.alpha * acc[i][j].x, g.alpha * acc[i][j].y);
      if (g.accumulate) {
        const double2 old = *c;
        v.x += old.x;
        v.y += old.y;
      }
      *c = v;
    }
  }
}

// One block per matrix; the matrix stays in global memory (L2), the pivot
// column and the scaled pivot row in shared memory.
__global__ void __launch_bounds__(256) gj_inverse_kernel(double2* base, int n, long long stride,
                                                         const int* list, int* status) {
  extern __shared__ double2 sm[];
  double2* f = sm;
  double2* row = sm + n;
  int* piv = reinterpret_cast<int*>(sm + 2 * n);
  __shared__ double red_v[8];
  __shared__ int red_i[8];
  __shared__ int s_p;
  __shared__ int s_bad;
  double2* M = base + (long long)(list ? list[blockIdx.x] : (int)blockIdx.x) * stride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_bad = 0;

  for (int j = 0; j < n; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + tid; i < n; i += blockDim.x) {
      const double2 v = M[(long long)i * n + j];
      const double a = v.x * v.x + v.y * v.y;
      if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bb = red_v[0];
      int ii = red_i[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
      s_p = ii;
      if (!(bb > 0.0)) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) break;
    const int p = s_p;
    if (p != j) {
      for (int c = tid; c < n; c += blockDim.x) {
        const double2 t = M[(long long)j * n + c];
        M[(long long)j * n + c] = M[(long long)p * n + c];
        M[(long long)p * n + c] = t;
      }
    }
    if (tid == 0) piv[j] = p;
    __syncthreads();
    const double2 pv = M[(long long)j * n + j];
    const double den = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = make_double2(pv.x / den, -pv.y / den);
    for (int c = tid; c < n; c += blockDim.x) {
      row[c] = (c == j) ? inv : cmul(M[(long long)j * n + c], inv);
      f[c] = M[(long long)c * n + j];
    }
    __syncthreads();
    for (int c = tid; c < n; c += blockDim.x) M[(long long)j * n + c] = row[c];
    const long long nn = (long long)n * n;
    for (long long e = tid; e < nn; e += blockDim.x) {
      const int i = (int)(e / n), c = (int)(e % n);
      if (i == j) continue;
      double2 v = (c == j) ? make_double2(0.0, 0.0) : M[e];
      const double2 t = cmul(f[i], row[c]);
      v.x -= t.x;
      v.y -= t.y;
      M[e] = v;
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) atomicExch(status, 1);
    return;
  }
  for (int j = n - 1; j >= 0; --j) {
    const int p = piv[j];
    if (p != j) {
      for (int r = tid; r < n; r += blockDim.x) {
        const double2 t = M[(long long)r * n + j];
        M[(long long)r * n + j] = M[(long long)r * n + p];
        M[(long long)r * n + p] = t;
      }
    }
    __syncthreads();
  }
}

// Blocked form of the same inversion (same pivots, same result up to rounding order), for
// n <= kGjBlockedMaxN[B]. Columns are taken in panels of B (16, or 8 for larger n, where two
// 16-column panels no longer fit in shared memory): the panel (n x B) is
// eliminated in shared memory with partial pivoting (explicit row swaps), written back, the
// panel's row swaps are applied to the other columns, and those columns receive the panel's
// effect as one rank-B update,
//   A[i][c] <- (i in the panel's pivot rows ? 0 : A[i][c]) + sum_t P[i][t] A_old[k0 + t][c],
// so the matrix is read and written once per panel instead of once per column. The column
// swaps that undo the row interchanges are applied at the end through one permutation.
// The size limits (kGjBlockedMaxN16, kGjBlockedMaxN8) keep the dynamic shared memory,
// n * (2 * B * 16 + 16 + 8) bytes, plus the kernel's static shared memory within 227 KB.

template <int B>
size_t gj_blocked_smem(int n) {
  return (size_t)n * (2 * B * sizeof(double2) + sizeof(double2) + 2 * sizeof(int));
}

// One matrix per block: matrix blockIdx.x of base (through list when given), or, with items,
// the item blockIdx.x (its own pointer, size and status word: a ragged list of matrices from
// several systems in one launch; the dynamic shared memory is sized for the largest).
template <int B>
__global__ void __launch_bounds__(256) gj_inverse_blocked_kernel(double2* base, int n, long long stride,
                                                                 const int* list, int* status,
                                                                 const GjItem* items) {
  extern __shared__ double2 sm[];
  __shared__ double red_v[8];
  __shared__ int red_i[8];
  __shared__ int s_p, s_bad;
  __shared__ double2 rowc[B];
  double2* M;
  if (items) {
    M = items[blockIdx.x].M;
    n = items[blockIdx.x].n;
    status = items[blockIdx.x].status;
  } else {
    M = base + (long long)(list ? list[blockIdx.x] : (int)blockIdx.x) * stride;
  }
  double2* P = sm;                         // [n][B]  panel
  double2* AK = P + (size_t)n * B;         // [B][n]  pivot rows at the panel start; staging at the end
  double2* fcol = AK + (size_t)n * B;      // [n]     pivot column of one step
  int* swp = reinterpret_cast<int*>(fcol + n);   // [n] row swapped with row c at step c
  int* pi = swp + n;                       // [n]     final column permutation
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_bad = 0;
  __syncthreads();

  for (int k0 = 0; k0 < n; k0 += B) {
    const int kb = min(B, n - k0);
    for (int e = tid; e < n * B; e += blockDim.x) {
      const int i = e / B, j = e % B;
      P[e] = j < kb ? M[(long long)i * n + k0 + j] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    // ---- elimination of the panel, column by column
    for (int j = 0; j < kb; ++j) {
      const int c = k0 + j;
      double best = -1.0;
      int bi = c;
      for (int i = c + tid; i < n; i += blockDim.x) {
        const double2 v = P[i * B + j];
        const double a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
      __syncthreads();
      if (tid == 0) {
        double bb = red_v[0];
        int ii = red_i[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
          if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
        s_p = ii;
        swp[c] = ii;
        if (!(bb > 0.0)) s_bad = 1;
      }
      __syncthreads();
      if (s_bad) break;
      const int p = s_p;
      if (p != c && tid < B) {
        const double2 t = P[c * B + tid];
        P[c * B + tid] = P[p * B + tid];
        P[p * B + tid] = t;
      }
      __syncthreads();
      const double2 pv = P[c * B + j];
      const double den = pv.x * pv.x + pv.y * pv.y;
      const double2 inv = make_double2(pv.x / den, -pv.y / den);
      for (int i = tid; i < n; i += blockDim.x) fcol[i] = P[i * B + j];
      if (tid < B) rowc[tid] = (tid == j) ? inv : cmul(P[c * B + tid], inv);
      __syncthreads();
      for (int e = tid; e < n * B; e += blockDim.x) {
        const int i = e / B, jj = e % B;
        if (jj >= kb) continue;
        if (i == c) {
          P[e] = rowc[jj];
        } else {
          const double2 f = fcol[i];
          if (jj == j) {
            const double2 t = cmul(f, inv);
            P[e] = make_double2(-t.x, -t.y);
          } else {
            const double2 t = cmul(f, rowc[jj]);
            P[e] = make_double2(P[e].x - t.x, P[e].y - t.y);
          }
        }
      }
      __syncthreads();
    }
    if (s_bad) break;
    // ---- panel back; its row swaps on the other columns (each thread keeps its columns)
    for (int e = tid; e < n * B; e += blockDim.x) {
      const int i = e / B, j = e % B;
      if (j < kb) M[(long long)i * n + k0 + j] = P[e];
    }
    for (int j = 0; j < kb; ++j) {
      const int c = k0 + j, p = swp[c];
      if (p == c) continue;
      for (int col = tid; col < n; col += blockDim.x) {
        if (col >= k0 && col < k0 + kb) continue;
        const double2 t = M[(long long)c * n + col];
        M[(long long)c * n + col] = M[(long long)p * n + col];
        M[(long long)p * n + col] = t;
      }
    }
    __syncthreads();
    for (int e = tid; e < B * n; e += blockDim.x) {
      const int t = e / n, col = e % n;
      AK[e] = t < kb ? M[(long long)(k0 + t) * n + col] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    // ---- rank-kb update of the other columns: one warp per row, lanes along the columns
    for (int i = warp; i < n; i += (int)(blockDim.x >> 5)) {
      const bool pivot_row = i >= k0 && i < k0 + kb;
      double2 pr[B];
#pragma unroll
      for (int t = 0; t < B; ++t) pr[t] = P[i * B + t];
      for (int col = lane; col < n; col += 32) {
        if (col >= k0 && col < k0 + kb) continue;
        double2 v = pivot_row ? make_double2(0.0, 0.0) : M[(long long)i * n + col];
#pragma unroll
        for (int t = 0; t < B; ++t) {
          const double2 a = AK[t * n + col];
          v.x = fma(pr[t].x, a.x, v.x);
          v.x = fma(-pr[t].y, a.y, v.x);
          v.y = fma(pr[t].x, a.y, v.y);
          v.y = fma(pr[t].y, a.x, v.y);
        }
        M[(long long)i * n + col] = v;
      }
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) atomicExch(status, 1);
    return;
  }
  // ---- undo the row interchanges as column swaps in reverse order, composed into one permutation
  if (tid == 0) {
    for (int i = 0; i < n; ++i) pi[i] = i;
    for (int c = n - 1; c >= 0; --c) {
      const int r = swp[c];
      if (r != c) {
        const int t = pi[c];
        pi[c] = pi[r];
        pi[r] = t;
      }
    }
  }
  __syncthreads();
  for (int r0 = 0; r0 < n; r0 += B) {
    const int rb = min(B, n - r0);
    for (int e = tid; e < rb * n; e += blockDim.x) AK[e] = M[(long long)r0 * n + e];
    __syncthreads();
    for (int e = tid; e < rb * n; e += blockDim.x) {
      const int t = e / n, y = e % n;
      M[(long long)(r0 + t) * n + y] = AK[t * n + pi[y]];
    }
    __syncthreads();
  }
}

__global__ void add_identity_kernel(double2* base, int n, long long stride, int nbatch, const int* list,
                                    double scale_m, double shift) {
  const long long nn = (long long)n * n;
  const long long total = nn * nbatch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long bl = e / nn, r = e % nn;
    const long long b = list ? list[bl] : bl;
    double2* p = base + b * stride + r;
    double2 v = *p;
    v.x *= scale_m;
    v.y *= scale_m;
    if (r / n == r % n) v.x += shift;
    *p = v;
  }
}

__global__ void build_g_dyson_kernel(double2* sw, const double2* H, const double2* S, const double* wn, double mu,
                                     int nk, int nw, int nao) {
  const long long nn = (long long)nao * nao;
  const long long total = nn * nw * nk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % nn;
    const long long kn = e / nn;
    const int n = (int)(kn % nw), k = (int)(kn / nw);
    const double2 h = H[(long long)k * nn + r];
    double2 s = sw[e];
    double2 v = make_double2(-h.x - s.x, -h.y - s.y);
    if (S) {   // (mu + i w_n) S^k
      const double2 o = S[(long long)k * nn + r];
      v.x += mu * o.x - wn[n] * o.y;
      v.y += mu * o.y + wn[n] * o.x;
    } else if (r / nao == r % nao) {
      v.x += mu;
      v.y += wn[n];
    }
    sw[e] = v;
  }
}

__global__ void mix_kernel(const double2* s_new, double2* s_inout, double alpha, long long n,
                           unsigned long long* maxbits, int* nonfinite) {
  double local = 0.0;
  int bad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 a = s_new[e], o = s_inout[e];
    const double2 v = make_double2(alpha * a.x + (1.0 - alpha) * o.x, alpha * a.y + (1.0 - alpha) * o.y);
    if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
    const double dx = v.x - o.x, dy = v.y - o.y;
    const double d = sqrt(dx * dx + dy * dy);
    if (d > local) local = d;
    s_inout[e] = v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local = fmax(local, __shfl_down_sync(0xffffffffu, local, o));
  if ((threadIdx.x & 31) == 0 && local > 0.0)
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(local));
  if (bad) atomicExch(nonfinite, 1);
}

// X[q][t] = X[mq[q]][T-1-t]^T for the (q, t) that are not canonical, where
// canonical means q < mq[q], or q == mq[q] and t <= T-1-t. One 32x32 tile per block.
__global__ void __launch_bounds__(256) mirror_fill_kernel(double2* X, int nk, int T, int n, const int* mq, int q0,
                                                          int q1) {
  __shared__ double2 tile[32][33];
  const int tiles_1d = (n + 31) / 32;
  long long b = blockIdx.x;
  const int tj = (int)(b % tiles_1d);
  b /= tiles_1d;
  const int ti = (int)(b % tiles_1d);
  b /= tiles_1d;
  const int t = (int)(b % T);
  const int q = (int)(b / T);
  const int p = mq[q];
  // q outside [q0, q1), or its partner -q outside (then every node of q was computed): nothing to fill
  if (q < q0 || q >= q1 || p < q0 || p >= q1) return;
  const bool canonical = q < p || (q == p && t <= T - 1 - t);
  if (canonical) return;
  const long long nn = (long long)n * n;
  const double2* src = X + ((long long)p * T + (T - 1 - t)) * nn;
  double2* dst = X + ((long long)q * T + t) * nn;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // read src rows tj*32.., columns ti*32.. (coalesced), write dst rows ti*32.., columns tj*32..
  for (int r = ty; r < 32; r += 8) {
    const int i = tj * 32 + r, j = ti * 32 + tx;
    if (i < n && j < n) tile[r][tx] = src[(long long)i * n + j];
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = ti * 32 + r, j = tj * 32 + tx;
    if (i < n && j < n) dst[(long long)i * n + j] = tile[tx][r];
  }
}

// ---- static part and loop helpers (Eq. sigma_inf, Sec. 2.4, Sec. 5.3)

// gamma^k = -sum_t w_t G^k(tau_t): minus the interpolant of G at tau = beta (w: extrapolation weights)
__global__ void density_kernel(const double2* G, const double* w, double2* gamma, int nk, int ntau, long long nao2) {
  const long long total = (long long)nk * nao2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / nao2, r = e % nao2;
    const double2* g = G + k * ntau * nao2 + r;
    double2 acc = make_double2(0.0, 0.0);
    for (int t = 0; t < ntau; ++t) {
      const double2 v = g[(long long)t * nao2];
      acc.x = fma(w[t], v.x, acc.x);
      acc.y = fma(w[t], v.y, acc.y);
    }
    gamma[e] = make_double2(-acc.x, -acc.y);
  }
}

// rho_Q = sum_{k'} sum_ab gamma^{k'}_ab V^{k'k'}_ba(Q); one block per Q
// Packed Coulomb factor: only the pairs k1 <= k2, in the order (0,0), (0,1), .., (0,nk-1), (1,1), ..;
// V^{k2 k1}_ij(Q) = conj V^{k1 k2}_ji(Q). Block of the pair (a, b), a <= b:
__device__ __forceinline__ long long packed_block(int a, int b, int nk) {
  return (long long)a * nk - (long long)a * (a - 1) / 2 + (b - a);
}

// Offset of element (Q, i, j) of V^{k1 k2} and whether it is conjugated: the full layout, or the
// packed one (the transposed element of the stored pair for k1 > k2).
__device__ __forceinline__ long long v_elem(int k1, int k2, int Q, int i, int j, int nk, int nao, long long pair,
                                            int packed, bool* conj) {
  const long long n2 = (long long)nao * nao;
  if (!packed) {
    *conj = false;
    return ((long long)k1 * nk + k2) * pair + Q * n2 + (long long)i * nao + j;
  }
  if (k1 <= k2) {
    *conj = false;
    return packed_block(k1, k2, nk) * pair + Q * n2 + (long long)i * nao + j;
  }
  *conj = true;
  return packed_block(k2, k1, nk) * pair + Q * n2 + (long long)j * nao + i;
}

__device__ __forceinline__ double2 v_load(const double2* V, int k1, int k2, int Q, int i, int j, int nk, int nao,
                                          long long pair, int packed) {
  bool cj;
  const double2 v = V[v_elem(k1, k2, Q, i, j, nk, nao, pair, packed, &cj)];
  return cj ? make_double2(v.x, -v.y) : v;
}

// dst[b] = V^{k1 k2} (full layout [naux][nao][nao]) from the packed V, for the blocks b of a list:
// pairs decoded from full-layout offsets tab[b] = (k1 nk + k2) pair, or every pair in order
// (all = 1), or up to four given pairs.
__global__ void unpack_v_kernel(const double2* __restrict__ Vp, int nk, int nao, long long pair, VPairs L,
                                int nblocks, double2* __restrict__ dst) {
  const long long n2 = (long long)nao * nao;
  for (int b = blockIdx.y; b < nblocks; b += gridDim.y) {
    int k1, k2;
    if (L.tab) {
      const long long kk = L.tab[b] / pair;
      k1 = (int)(kk / nk);
      k2 = (int)(kk % nk);
    } else if (L.all) {
      k1 = b / nk;
      k2 = b % nk;
    } else {
      k1 = L.k1[b];
      k2 = L.k2[b];
    }
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < pair;
         e += (long long)gridDim.x * blockDim.x) {
      const int Q = (int)(e / n2), r = (int)(e % n2), i = r / nao, j = r % nao;
      dst[(long long)b * pair + e] = v_load(Vp, k1, k2, Q, i, j, nk, nao, pair, 1);
    }
  }
}

__global__ void __launch_bounds__(256) hartree_rho_kernel(const double2* V, const double2* gamma, double2* rho, int nk,
                                                          int naux, int nao, int packed) {
  const int Q = blockIdx.x;
  const long long nao2 = (long long)nao * nao, pair = (long long)naux * nao2;
  double2 acc = make_double2(0.0, 0.0);
  for (long long e = threadIdx.x; e < (long long)nk * nao2; e += blockDim.x) {
    const int kp = (int)(e / nao2);
    const int a = (int)((e % nao2) / nao), b = (int)(e % nao);
    const double2 g = gamma[(long long)kp * nao2 + (long long)a * nao + b];
    const long long blk = packed ? packed_block(kp, kp, nk) : (long long)kp * nk + kp;
    const double2 v = V[blk * pair + (long long)Q * nao2 + (long long)b * nao + a];
    cmac(acc, g, v);
  }
  __shared__ double sx[256], sy[256];
  sx[threadIdx.x] = acc.x;
  sy[threadIdx.x] = acc.y;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sx[threadIdx.x] += sx[threadIdx.x + o];
      sy[threadIdx.x] += sy[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) rho[Q] = make_double2(sx[0], sy[0]);
}

// out^k_ij = scale sum_Q V^{kk}_ij(Q) rho_Q
__global__ void hartree_j_kernel(const double2* V, const double2* rho, double2* out, int nk, int naux, int nao,
                                 double scale, int packed) {
  const long long nao2 = (long long)nao * nao, pair = (long long)naux * nao2;
  const long long total = (long long)nk * nao2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / nao2, r = e % nao2;
    const double2* v = V + (packed ? packed_block((int)k, (int)k, nk) : k * nk + k) * pair + r;
    double2 acc = make_double2(0.0, 0.0);
    for (int Q = 0; Q < naux; ++Q) cmac(acc, v[(long long)Q * nao2], rho[Q]);
    out[e] = make_double2(scale * acc.x, scale * acc.y);
  }
}

// Exchange term of Eq. sigma_inf, fused per (k, k', chunk c of the auxiliary index):
//   part[(k nk + k') qc + c]_ij = sum_{Q in c} sum_b X_ib(Q) V^{k'k}_bj(Q),
//   X(Q) = V^{kk'}(Q) gamma^{k'},
// with gamma^{k'}, V^{kk'}(Q), X(Q) and V^{k'k}(Q) staged in shared memory one Q at a time and
// each thread holding up to kExMaxPerThread entries of the 'ij' block in registers.
constexpr int kExThreads = 256;
constexpr int kExMaxPerThread = 11;    // nao^2 <= 256 * 11: nao <= kExchangeMaxNao
__global__ void __launch_bounds__(kExThreads) exchange_partial_kernel(const double2* __restrict__ V,
                                                                      const double2* __restrict__ gamma,
                                                                      double2* __restrict__ part, int nk, int naux,
                                                                      int nao, int qc, int packed) {
  extern __shared__ double2 ex_sm[];
  const int n2 = nao * nao;
  double2* g = ex_sm;
  double2* v1 = g + n2;
  double2* x = v1 + n2;
  double2* v2 = x + n2;
  const int c = blockIdx.x % qc, kp = (blockIdx.x / qc) % nk, k = blockIdx.x / (qc * nk);
  const int q0 = (int)((long long)naux * c / qc), q1 = (int)((long long)naux * (c + 1) / qc);
  const long long pair = (long long)naux * n2;
  for (int e = threadIdx.x; e < n2; e += kExThreads) g[e] = gamma[(long long)kp * n2 + e];
  double2 acc[kExMaxPerThread];
#pragma unroll
  for (int t = 0; t < kExMaxPerThread; ++t) acc[t] = make_double2(0.0, 0.0);
  for (int Q = q0; Q < q1; ++Q) {
    __syncthreads();
    for (int e = threadIdx.x; e < n2; e += kExThreads) {
      const int i = e / nao, j = e - i * nao;
      v1[e] = v_load(V, k, kp, Q, i, j, nk, nao, pair, packed);
      v2[e] = v_load(V, kp, k, Q, i, j, nk, nao, pair, packed);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2; e += kExThreads) {
      const int i = e / nao, b = e - i * nao;
      double2 s = make_double2(0.0, 0.0);
      for (int a = 0; a < nao; ++a) cmac(s, v1[i * nao + a], g[a * nao + b]);
      x[e] = s;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kExMaxPerThread; ++t) {
      const int e = threadIdx.x + t * kExThreads;
      if (e < n2) {
        const int i = e / nao, j = e - i * nao;
        for (int b = 0; b < nao; ++b) cmac(acc[t], x[i * nao + b], v2[b * nao + j]);
      }
    }
  }
  double2* out = part + (long long)blockIdx.x * n2;
#pragma unroll
  for (int t = 0; t < kExMaxPerThread; ++t) {
    const int e = threadIdx.x + t * kExThreads;
    if (e < n2) out[e] = acc[t];
  }
}

// out[o][e] += scale sum_{p < nparts} part[o nparts + p][e], summed in the order of p (the exchange
// of Eq. sigma_inf: o = k, p = (k', c); the GF2 exchange: o = tau node, p = orbital q)
__global__ void exchange_reduce_kernel(const double2* __restrict__ part, double2* __restrict__ out, int nouter,
                                       int n2, int nparts, double scale) {
  const long long total = (long long)nouter * n2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const long long o = e / n2, r = e % n2;
    const double2* p = part + o * nparts * n2 + r;
    double2 s = make_double2(0.0, 0.0);
    for (int u = 0; u < nparts; ++u) {
      const double2 v = p[(long long)u * n2];
      s.x += v.x;
      s.y += v.y;
    }
    out[e].x += scale * s.x;
    out[e].y += scale * s.y;
  }
}

// *out = sum_k sum_i Re gamma^k_ii (one block)
__global__ void __launch_bounds__(256) trace_kernel(const double2* gamma, const double2* S, int nk, int nao,
                                                    double* out) {
  double acc = 0.0;
  if (!S) {
    for (long long e = threadIdx.x; e < (long long)nk * nao; e += blockDim.x) {
      const long long k = e / nao, i = e % nao;
      acc += gamma[(k * nao + i) * nao + i].x;
    }
  } else {   // sum_k Re Tr gamma^k S^k = sum_{k i j} Re gamma^k_ij S^k_ji
    const long long nn = (long long)nao * nao;
    for (long long e = threadIdx.x; e < (long long)nk * nn; e += blockDim.x) {
      const long long k = e / nn, r = e % nn, i = r / nao, j = r % nao;
      const double2 a = gamma[e], b = S[k * nn + j * nao + i];
      acc += a.x * b.x - a.y * b.y;
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// c = a + b elementwise
__global__ void add_kernel(const double2* a, const double2* b, double2* c, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    c[e] = make_double2(a[e].x + b[e].x, a[e].y + b[e].y);
}

// partial[block] = sum over the block's share of Re(conj(x_e) y_e), in a fixed order
__global__ void __launch_bounds__(256) dot_re_kernel(const double2* x, const double2* y, long long n, double* partial) {
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    acc = fma(x[e].x, y[e].x, fma(x[e].y, y[e].y, acc));
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// one block sums the partials
__global__ void __launch_bounds__(256) sum_kernel(const double* partial, int m, double* out) {
  double acc = 0.0;
  for (int e = threadIdx.x; e < m; e += blockDim.x) acc += partial[e];
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// out = sum_i c_i v_i (m <= 16 vectors, coefficients in constant-size parameter)
struct LinComb {
  const double2* v[16];
  double c[16];
  int m;
};
__global__ void lincomb_kernel(const LinComb lc, double2* out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < lc.m; ++i) {
      const double2 x = lc.v[i][e];
      acc.x = fma(lc.c[i], x.x, acc.x);
      acc.y = fma(lc.c[i], x.y, acc.y);
    }
    out[e] = acc;
  }
}

inline int grid_for(long long total, int block) {
  long long g = (total + block - 1) / block;
  if (g > 152LL * 32) g = 152LL * 32;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

int zgemm_fp64(const ZGemm& g, void* stream) {
  if (g.M <= 0 || g.N <= 0 || g.nbatch <= 0) return GW_OK;
  if (g.nbatch > 65535) return fail(GW_EINVAL, "zgemm_fp64: batch %d too large", g.nbatch);
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.nbatch);
  if (grid.y > 65535) return fail(GW_EINVAL, "zgemm_fp64: M=%d too large", g.M);
  prof_begin(g.slot, (cudaStream_t)stream);
  zgemm_fp64_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(g);
  prof_end(g.slot, (cudaStream_t)stream, 8.0 * g.M * (double)g.N * g.K * g.nbatch,
           16.0 * ((double)g.M * g.K + (double)g.N * g.K + (double)g.M * g.N) * g.nbatch);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "zgemm_fp64 launch: %s", cudaGetErrorString(e));
}

namespace {
template <int B>
bool gj_blocked_attr() {
  static const bool ok = [] {
    const int maxn = B == 16 ? kGjBlockedMaxN16 : kGjBlockedMaxN8;
    const bool r = cudaFuncSetAttribute(gj_inverse_blocked_kernel<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)gj_blocked_smem<B>(maxn)) == cudaSuccess;
    cudaGetLastError();
    return r;
  }();
  return ok;
}

template <int B>
int launch_gj_blocked(double2* base, int n, long long stride, int nblocks, int* status_dev, cudaStream_t st,
                      const int* list, const GjItem* items, double flops, double bytes) {
  if (!gj_blocked_attr<B>()) return fail(GW_ECUDA, "gj_inverse_blocked: shared memory attribute refused");
  prof_begin(SLOT_INVERSE_FP64, st);
  gj_inverse_blocked_kernel<B><<<nblocks, 256, gj_blocked_smem<B>(n), st>>>(base, n, stride, list, status_dev, items);
  prof_end(SLOT_INVERSE_FP64, st, flops, bytes);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "gj_inverse_blocked launch: %s", cudaGetErrorString(e));
}
}  // namespace

int batched_inverse_fp64(double2* base, int n, long long stride, int nbatch, int* status_dev,
                         void* stream, const int* list) {
  if (nbatch <= 0) return GW_OK;
  const double flops = 8.0 * (double)n * n * n * nbatch, bytes = 32.0 * (double)n * n * nbatch;
  if (n <= kGjBlockedMaxN16)
    return launch_gj_blocked<16>(base, n, stride, nbatch, status_dev, (cudaStream_t)stream, list, nullptr, flops,
                                 bytes);
  if (n <= kGjBlockedMaxN8)
    return launch_gj_blocked<8>(base, n, stride, nbatch, status_dev, (cudaStream_t)stream, list, nullptr, flops,
                                bytes);
  const size_t smem = 2 * (size_t)n * sizeof(double2) + (size_t)n * sizeof(int);
  if (smem > 200 * 1024) return fail(GW_EINVAL, "batched_inverse_fp64: n=%d too large", n);
  static const bool attr_set = [] {   // once, also when several threads launch
    cudaFuncSetAttribute(gj_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr_set;
  prof_begin(SLOT_INVERSE_FP64, (cudaStream_t)stream);
  gj_inverse_kernel<<<nbatch, 256, smem, (cudaStream_t)stream>>>(base, n, stride, list, status_dev);
  prof_end(SLOT_INVERSE_FP64, (cudaStream_t)stream, 8.0 * (double)n * n * n * nbatch,
           32.0 * (double)n * n * nbatch);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "gj_inverse launch: %s", cudaGetErrorString(e));
}

int add_identity_fp64(double2* base, int n, long long stride, int nbatch, double scale_m,
                      double shift, void* stream, const int* list) {
  const long long total = (long long)n * n * nbatch;
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  add_identity_kernel<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(base, n, stride, nbatch, list,
                                                                              scale_m, shift);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 2.0 * total, 32.0 * total);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "add_identity launch: %s", cudaGetErrorString(e));
}

int build_g_dyson_fp64(double2* sw, const double2* H, const double2* S, const double* wn, double mu, int nk, int nw,
                       int nao, void* stream) {
  const long long total = (long long)nao * nao * nw * nk;
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  build_g_dyson_kernel<<<grid_for(total, 256), 256, 0, (cudaStream_t)stream>>>(sw, H, S, wn, mu, nk, nw,
                                                                               nao);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 4.0 * total, 32.0 * total);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "build_g_dyson launch: %s", cudaGetErrorString(e));
}

int mirror_fill(double2* X, int nk, int T, int n, const int* mq_dev, void* stream, int q0, int q1) {
  if (q1 < 0) q1 = nk;
  const long long tiles_1d = (n + 31) / 32;
  const long long blocks = (long long)nk * T * tiles_1d * tiles_1d;
  if (blocks == 0 || q1 <= q0) return GW_OK;
  if (blocks > 2147483647LL) return fail(GW_EINVAL, "mirror_fill: too many blocks");
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  mirror_fill_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(X, nk, T, n, mq_dev, q0, q1);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 0.0, 16.0 * (double)nk * T * n * n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "mirror_fill launch: %s", cudaGetErrorString(e));
}

int mix_fp64(const double2* s_new, double2* s_inout, double alpha, long long n, double* maxdiff_dev,
             int* nonfinite_dev, void* stream) {
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  mix_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
      s_new, s_inout, alpha, n, reinterpret_cast<unsigned long long*>(maxdiff_dev), nonfinite_dev);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 8.0 * n, 48.0 * n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "mix launch: %s", cudaGetErrorString(e));
}

int density_fp64(const double2* G, const double* w, double2* gamma, int nk, int ntau, int nao, void* stream) {
  const long long n = (long long)nk * nao * nao;
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  density_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(G, w, gamma, nk, ntau, (long long)nao * nao);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 4.0 * n * ntau, 16.0 * n * (ntau + 1));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "density launch: %s", cudaGetErrorString(e));
}

int hartree_fp64(const double2* V, const double2* gamma, double2* rho, double2* out, int nk, int naux, int nao,
                 double scale, int packed, void* stream) {
  const long long n = (long long)nk * nao * nao;
  prof_begin(SLOT_STATIC_FP64, (cudaStream_t)stream);
  hartree_rho_kernel<<<naux, 256, 0, (cudaStream_t)stream>>>(V, gamma, rho, nk, naux, nao, packed);
  hartree_j_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(V, rho, out, nk, naux, nao, scale, packed);
  prof_end(SLOT_STATIC_FP64, (cudaStream_t)stream, 16.0 * n * naux, 32.0 * n * naux);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "hartree launch: %s", cudaGetErrorString(e));
}

int reduce_partials_fp64(const double2* part, double2* out, int nouter, int n2, int nparts, double scale,
                         void* stream) {
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  exchange_reduce_kernel<<<grid_for((long long)nouter * n2, 256), 256, 0, (cudaStream_t)stream>>>(part, out, nouter,
                                                                                                n2, nparts, scale);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 2.0 * nouter * (double)n2 * nparts,
           16.0 * nouter * (double)n2 * (nparts + 2));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "reduce_partials launch: %s", cudaGetErrorString(e));
}

__global__ void check_guards_kernel(unsigned char* const* guards, int n, int* count, int* first) {
  for (int g = blockIdx.x; g < n; g += gridDim.x) {
    int bad = 0;
    for (int i = threadIdx.x; i < (int)kGuardBytes; i += blockDim.x) bad |= guards[g][i] != kGuardByte;
    if (__syncthreads_or(bad) && threadIdx.x == 0) {
      atomicAdd(count, 1);
      atomicMin(first, g);
    }
  }
}

int check_guards(unsigned char* const* guards, int n, int* first, void* stream) {
  if (n <= 0) return 0;
  unsigned char** dg = nullptr;
  int* flags = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&dg), n * sizeof(void*)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&flags), 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(dg);
    cudaGetLastError();
    return -1;
  }
  int h[2] = {0, 1 << 30};
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyAsync(dg, guards, n * sizeof(void*), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(flags, h, sizeof h, cudaMemcpyHostToDevice, st);
  check_guards_kernel<<<std::min(n, 1024), 128, 0, st>>>(dg, n, flags, flags + 1);
  cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, st);
  const bool ok = cudaStreamSynchronize(st) == cudaSuccess;
  cudaFree(dg);
  cudaFree(flags);
  if (!ok) return -1;
  *first = h[1];
  return h[0];
}

int exchange_chunks(int nk, int naux) {
  // enough blocks for every SM several times over: 4 x 152 at least, when naux allows
  const int want = (608 + nk * nk - 1) / (nk * nk);
  return std::max(1, std::min(want, naux));
}

int exchange_fp64(const double2* V, const double2* gamma, double2* part, double2* out, int nk, int naux, int nao,
                  double scale, int packed, void* stream) {
  if (nao > kExchangeMaxNao) return fail(GW_EINVAL, "exchange_fp64: nao=%d above %d", nao, kExchangeMaxNao);
  static const bool attr = [] {
    const bool ok = cudaFuncSetAttribute(exchange_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         4 * kExchangeMaxNao * kExchangeMaxNao * (int)sizeof(double2)) == cudaSuccess;
    cudaGetLastError();
    return ok;
  }();
  if (!attr) return fail(GW_ECUDA, "exchange_fp64: shared memory attribute refused");
  const int qc = exchange_chunks(nk, naux), n2 = nao * nao;
  const size_t smem = 4 * (size_t)n2 * sizeof(double2);
  prof_begin(SLOT_STATIC_FP64, (cudaStream_t)stream);
  exchange_partial_kernel<<<nk * nk * qc, kExThreads, smem, (cudaStream_t)stream>>>(V, gamma, part, nk, naux, nao,
                                                                                     qc, packed);
  exchange_reduce_kernel<<<grid_for((long long)nk * n2, 256), 256, 0, (cudaStream_t)stream>>>(part, out, nk, n2,
                                                                                             nk * qc, scale);
  prof_end(SLOT_STATIC_FP64, (cudaStream_t)stream, 16.0 * (double)nk * nk * naux * n2 * nao,
           32.0 * (double)nk * nk * naux * n2);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "exchange launch: %s", cudaGetErrorString(e));
}

int unpack_v_fp64(const double2* Vp, int nk, int nao, long long pair, const VPairs& L, int nblocks, double2* dst,
                  void* stream) {
  if (nblocks <= 0) return GW_OK;
  if (!L.tab && !L.all && nblocks > 4) return fail(GW_EINVAL, "unpack_v: at most four listed pairs");
  const int gx = (int)std::min<long long>((pair + 255) / 256, 1024);
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  unpack_v_kernel<<<dim3(gx, std::min(nblocks, 65535)), 256, 0, (cudaStream_t)stream>>>(Vp, nk, nao, pair, L, nblocks,
                                                                                        dst);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 0.0, 32.0 * (double)pair * nblocks);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "unpack_v launch: %s", cudaGetErrorString(e));
}

int trace_fp64(const double2* gamma, const double2* S, int nk, int nao, double* out_dev, void* stream) {
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  trace_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(gamma, S, nk, nao, out_dev);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, (double)nk * nao, 16.0 * nk * nao);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "trace launch: %s", cudaGetErrorString(e));
}

int add_fp64(const double2* a, const double2* b, double2* c, long long n, void* stream) {
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  add_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(a, b, c, n);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 2.0 * n, 48.0 * n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "add launch: %s", cudaGetErrorString(e));
}

int dot_re_fp64(const double2* x, const double2* y, long long n, double* partial_dev, double* out_dev, void* stream) {
  prof_begin(SLOT_REDUCE, (cudaStream_t)stream);
  dot_re_kernel<<<kDotBlocks, 256, 0, (cudaStream_t)stream>>>(x, y, n, partial_dev);
  sum_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(partial_dev, kDotBlocks, out_dev);
  prof_end(SLOT_REDUCE, (cudaStream_t)stream, 4.0 * n, 32.0 * n);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "dot launch: %s", cudaGetErrorString(e));
}

int lincomb_fp64(const double2* const* v, const double* c, int m, double2* out, long long n, void* stream) {
  if (m < 1 || m > 16) return fail(GW_EINVAL, "lincomb: 1..16 vectors");
  LinComb lc{};
  for (int i = 0; i < m; ++i) {
    lc.v[i] = v[i];
    lc.c[i] = c[i];
  }
  lc.m = m;
  prof_begin(SLOT_ELEMENTWISE, (cudaStream_t)stream);
  lincomb_kernel<<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(lc, out, n);
  prof_end(SLOT_ELEMENTWISE, (cudaStream_t)stream, 4.0 * n * m, 16.0 * n * (m + 1));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "lincomb launch: %s", cudaGetErrorString(e));
}

}  // namespace gwi

namespace gwi {

int batched_inverse_group_fp64(const GjItem* items_dev, int count, int max_n, double flops, void* stream) {
  if (count <= 0) return GW_OK;
  if (max_n > kGjBlockedMaxN8) return fail(GW_EINVAL, "batched_inverse_group_fp64: n = %d above %d", max_n, kGjBlockedMaxN8);
  const double bytes = 32.0 * (double)max_n * max_n * count;
  if (max_n <= kGjBlockedMaxN16)
    return launch_gj_blocked<16>(nullptr, max_n, 0, count, nullptr, (cudaStream_t)stream, nullptr, items_dev, flops,
                                 bytes);
  return launch_gj_blocked<8>(nullptr, max_n, 0, count, nullptr, (cudaStream_t)stream, nullptr, items_dev, flops,
                              bytes);
}

}  // namespace gwi
