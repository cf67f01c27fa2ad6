// Mixed-precision contractions of the GW path on tcgen05 tensor cores.
//
// Every V.G.V contraction (Eqs. tilde_P0_tau and sigma_gw) is a complex GEMM
// C = sum_k A(m,k) B(n,k). Each operand is split, per row and per chunk of at
// most 256 k-values, into four bf16 slices that share one power-of-two
// alignment 2^E (E from the chunk's largest |re|, |im|):
//     x = 2^E (s0 + s1 + s2 + s3) + O(2^(E-32)),   s_i = integer_i * 2^-(8i+7), |integer_i| <= 128.
// Products of leading slices are integers times one common quantum, so their
// sum over a chunk (at most 2*256 terms of at most 2^14) is exact in the FP32
// accumulator, and so is the sum of the order-1 products (i + j = 1, at most
// 4*256 terms of at most 2^14 on a quantum 2^-8 smaller) in a second
// accumulator. Orders 2 and 3 share a third accumulator, whose FP32 rounding
// sits 2^-16 below the leading term; products with i + j > 3 are dropped
// (2^-32 relative). Tensor-core FP32 accumulation rounds toward zero, so only
// exact partial sums keep the error from growing with the chunk length. After
// each chunk the six accumulators (three orders x re/im) are combined without
// rounding into an FP32 pair and added to a double-float running sum (FP64 is
// about 1/64 of the FP32 rate on this part, so no FP64 instruction runs per
// chunk); the last chunk writes FP64, or double-float for intermediates that
// are sliced again. A complex slice product is two real MMAs of N = 160 with
// the real and imaginary parts of B stacked along N (see OzShape).
//
// Kernels
//   slice_kernel   FP64 or double-float complex view -> bf16 slice groups
//                  [re | im][k-step][row][4 slices x 16 k]
//   oz_gemm_kernel persistent tcgen05 GEMM over group tiles loaded by TMA
//                  (128-byte swizzle, K-major, one 16-wide k-step per pipeline stage)
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gw_internal.h"
#include "gw_mixed.h"

namespace gwi {

namespace {

#ifndef GW_TRY_INTERNAL
#define GW_TRY_INTERNAL(x)        \
  do {                            \
    const int _rc = (x);          \
    if (_rc != GW_OK) return _rc; \
  } while (0)
#endif

constexpr int kBM = 128;       // rows of an MMA tile (TMEM lanes)
constexpr int kStepK = 16;     // k per MMA (kind::f16)
constexpr int kMaxChunk = 256; // k per exact-accumulation chunk

// ------------------------------------------------------------------------------------------------
// slicer

// Source elements are FP64 complex (double2) or, for intermediates written by
// the GEMM epilogue, double-float complex: float4 (re_hi, re_lo, im_hi, im_lo)
// in the same 16-byte slot. No FP64 instruction runs per element. An FP64
// element scaled to 2^31 / 2^E is rounded to an integer N (|N| <= 2^31) and
// split into four signed base-256 digits. A double-float element (h, l) is
// rounded, level by level, to a multiple of the slice quantum q_i = 2^(E-7-8i)
// by adding and subtracting 1.5 * 2^23 * q_i in FP32 (exact: |h| < 2^22 q_i);
// the remainder h - s_i is exact and is renormalised with l before the next
// level, so every digit stays within 128 and the four slices carry the value
// to within 2^(E-32).

// Division by a fixed divisor d < 2^31 for numerators x < 2^31: x / d = (x * m) >> sh
// with m = ceil(2^sh / d), sh = 31 + ceil(log2 d) (the error of m times x stays below 2^sh).
struct FastDiv {
  unsigned long long m = 1ull << 31;
  int sh = 31, d = 1;
};
__host__ FastDiv make_fastdiv(int d) {
  FastDiv f;
  int l = 0;
  while ((1ll << l) < d) ++l;
  f.d = d;
  f.sh = 31 + l;
  f.m = ((1ull << f.sh) + (unsigned long long)d - 1) / (unsigned long long)d;
  return f;
}
__device__ __forceinline__ int fdiv(int x, const FastDiv& f) {
  return (int)(((unsigned long long)(unsigned)x * f.m) >> f.sh);
}

struct SliceJob {
  const double2* src = nullptr;
  int src_df = 0;          // 1: src holds double-float complex values
  ZView v;                 // row and k view of one batch entry
  ZBatch b;                // per-batch source offset
  int bin = 1 << 30;
  int rows = 0, K = 0, Kc = 0, Kpad = 0, nbatch = 1;
  __nv_bfloat16* dst = nullptr;
  long long dst_rows = 0;       // rows of the destination planes buffer
  long long dst_row0 = 0;       // first destination row of batch 0
  long long dst_rows_per_batch = 0;
  FastDiv kdiv;                 // division by v.kin
};

__device__ __forceinline__ long long s_view_row(const ZView& v, int r) {
  return (long long)(r / v.rin) * v.rs_out + (long long)(r % v.rin) * v.rs_in;
}

// round(x * 2^(31 - E)) for an FP64 bit pattern x with |x| < 2^E (round half up on |x|).
__device__ __forceinline__ long long fixed31_f64(unsigned long long bits, int E) {
  const int eb = (int)((bits >> 52) & 0x7FF);
  if (eb == 0) return 0;
  const long long m = (long long)((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int sh = 1044 + E - eb;          // x = m 2^(eb - 1075); sh >= 22 because |x| < 2^E
  const long long n = sh >= 62 ? 0 : ((m + (1ll << (sh - 1))) >> sh);
  return (bits >> 63) ? -n : n;
}

// Slices of the double-float value h + l (|h + l| < 2^E): s_i, a multiple of q_i with
// |s_i| <= 128 q_i, for i = 0..3 (magic[i] = 1.5 * 2^23 * q_i; q_i = 2^(E-7-8i)).
// The pair is normalised once (an exact two-sum: the epilogue's pairs are not normalised, l
// holding the order 2-3 sum), after which |l| <= 2^(E-25). s_0 and s_1 are cut from h (each
// remainder exact, |h| <= q_1 / 2 = 2^(E-16) after s_1); l joins before s_2, the one rounding
// on the way (at most 2^(E-40), far below q_3 = 2^(E-31)); |remainder| <= q_2 / 2 = 128 q_3
// before s_3. Residual: q_3 / 2 plus that rounding.
__device__ __forceinline__ void df_slices(float h, float l, const float magic[4], float s[4]) {
  {
    const float t = __fadd_rn(h, l);
    const float hv = __fsub_rn(t, l);
    l = __fadd_rn(__fsub_rn(h, hv), __fsub_rn(l, __fsub_rn(t, hv)));
    h = t;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i == 2) h = __fadd_rn(h, l);
    s[i] = __fsub_rn(__fadd_rn(h, magic[i]), magic[i]);   // h rounded to a multiple of q_i
    if (i < 3) h = __fsub_rn(h, s[i]);                    // exact
  }
}

// N (|N| <= 2^31 + 1) -> signed base-256 digits d0..d3, N = d0 2^24 + d1 2^16 + d2 2^8 + d3, |d| <= 128.
__device__ __forceinline__ void split_digits(long long n, int d[4]) {
  d[0] = (int)((n + (1ll << 23)) >> 24);
  int r = (int)(n - ((long long)d[0] << 24));   // |r| <= 2^23: the rest in 32-bit arithmetic
  d[1] = (r + (1 << 15)) >> 16;
  r -= d[1] << 16;
  d[2] = (r + (1 << 7)) >> 8;
  d[3] = r - (d[2] << 8);
}

// One warp per (batch, row, chunk).
template <bool DF>
__global__ void __launch_bounds__(256) slice_kernel(const SliceJob j) {
  const long long warp_global = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nchunk = j.Kpad / j.Kc;
  const long long total = (long long)j.nbatch * j.rows * nchunk;
  if (warp_global >= total) return;
  // consecutive warps take consecutive rows of one chunk: their 128-byte output lines are adjacent
  const int r = (int)(warp_global % j.rows);
  const long long bc = warp_global / j.rows;
  const int c = (int)(bc % nchunk);
  const int b = (int)(bc / nchunk);
  const int bo = b / j.bin, bi = b % j.bin;
  const double2* src = j.src + (j.b.tab ? j.b.tab[bi] : (long long)bi * j.b.bs_in) + (long long)bo * j.b.bs_out +
                       s_view_row(j.v, r);
  // each lane owns element pairs (2 lane + 64 u, +1): bf16x2 stores, half the store instructions
  constexpr int kPairs = kMaxChunk / 64;
  // raw bit patterns of (re, im): FP64 bits, or the two FP32 halves of a double-float
  unsigned long long xr[2 * kPairs], xi[2 * kPairs];
  unsigned long long mbits = 0;          // largest |value| as bits (ordered like the values)
#pragma unroll
  for (int v = 0; v < 2 * kPairs; ++v) {
    const int e = 2 * lane + 64 * (v >> 1) + (v & 1);
    const int k = c * j.Kc + e;
    xr[v] = xi[v] = 0;
    if (e < j.Kc && k < j.K) {
      const int kq = fdiv(k, j.kdiv);
      const long long off = (long long)kq * j.v.ks_out + (long long)(k - kq * j.v.kin) * j.v.ks_in;
      if (DF) {
        const float4 f = reinterpret_cast<const float4*>(src)[off];
        xr[v] = ((unsigned long long)__float_as_uint(f.y) << 32) | __float_as_uint(f.x);
        xi[v] = ((unsigned long long)__float_as_uint(f.w) << 32) | __float_as_uint(f.z);
        mbits = max(mbits, (unsigned long long)max(__float_as_uint(f.x) & 0x7FFFFFFFu, __float_as_uint(f.z) & 0x7FFFFFFFu));
      } else {
        const double2 d = src[off];
        xr[v] = (unsigned long long)__double_as_longlong(d.x);
        xi[v] = (unsigned long long)__double_as_longlong(d.y);
        mbits = max(mbits, max(xr[v] & 0x7FFFFFFFFFFFFFFFull, xi[v] & 0x7FFFFFFFFFFFFFFFull));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mbits = max(mbits, __shfl_xor_sync(0xffffffffu, mbits, o));
  // E: the chunk maximum m = f 2^E with f in [0.5, 1), so every |x| / 2^E < 1
  int E;
  bool zero;
  if (DF) {
    const int eb = (int)((mbits >> 23) & 0xFF);
    zero = eb == 0;
    E = eb - 126;
  } else {
    const int eb = (int)((mbits >> 52) & 0x7FF);
    zero = eb == 0;
    E = eb - 1022;
  }
  const long long row = j.dst_row0 + (long long)b * j.dst_rows_per_batch + r;
  // element k: group g, k-step k / 16, this row, value (slice s, k % 16) at 16 s + k % 16
  const long long kstride = j.dst_rows * 64;                      // between k-steps
  const long long gstride = (long long)(j.Kpad / 16) * kstride;   // between groups
  __nv_bfloat16* out = j.dst + row * 64;
  // chunks whose largest value is below 2^-90 are taken as zero (their slices would be subnormal)
  if (E < -90) zero = true;
  float scale[4], magic[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    scale[s] = ldexpf(1.0f, E - 7 - 8 * s);
    magic[s] = ldexpf(3.0f, E + 15 - 8 * s);      // 1.5 * 2^23 * q_s
  }
#pragma unroll
  for (int u = 0; u < kPairs; ++u) {
    const int e = 2 * lane + 64 * u;
    if (e >= j.Kc) break;                // Kc is a multiple of 16, so e + 1 < Kc as well
    float fr[2][4], fi[2][4];            // slice values, digit * q_s (exact in bf16)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = 2 * u + h;
      if (zero) {
#pragma unroll
        for (int s = 0; s < 4; ++s) fr[h][s] = fi[h][s] = 0.0f;
      } else if (DF) {
        df_slices(__uint_as_float((uint32_t)xr[v]), __uint_as_float((uint32_t)(xr[v] >> 32)), magic, fr[h]);
        df_slices(__uint_as_float((uint32_t)xi[v]), __uint_as_float((uint32_t)(xi[v] >> 32)), magic, fi[h]);
      } else {
        int dr[4], di[4];
        split_digits(fixed31_f64(xr[v], E), dr);
        split_digits(fixed31_f64(xi[v], E), di);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          fr[h][s] = (float)dr[s] * scale[s];
          fi[h][s] = (float)di[s] * scale[s];
        }
      }
    }
    const int k = c * j.Kc + e;          // even: the pair (k, k + 1) shares its k-step
    __nv_bfloat16* o = out + (long long)(k >> 4) * kstride + (k & 15);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      // digit * 2^(E - 7 - 8s) is exact in float and in bf16 (|digit| <= 128)
      *reinterpret_cast<__nv_bfloat162*>(o + 16 * s) = __floats2bfloat162_rn(fr[0][s], fr[1][s]);
      *reinterpret_cast<__nv_bfloat162*>(o + gstride + 16 * s) = __floats2bfloat162_rn(fi[0][s], fi[1][s]);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// tcgen05 GEMM

struct OzParams {
  int M = 0, N = 0, nsteps = 0, steps_per_chunk = 0;
  int mtiles = 0, ntiles = 0, nbatch = 1, bin = 1 << 30;
  long long a_row0 = 0, b_row0 = 0;   // constant first plane row of A and B
  const long long* a_tab = nullptr;   // A row base per inner batch index
  long long a_bs_in = 0, a_bs_out = 0;
  const long long* b_tab = nullptr;
  long long b_bs_in = 0, b_bs_out = 0;
  double2* C = nullptr;
  ZView vc;                           // rows via rin/rs_*, columns via kin/ks_*
  ZBatch bc;
  double alpha = 1.0;
  int accumulate = 0;
  int out_df = 0;                     // 1: write double-float complex (float4) instead of FP64 (alpha 1, no accumulate)
  // block-diagonal batching: each GEMM "batch" is a group of dgroup problems of dblock x dblock
  // outputs stacked along rows and columns (M = N = dgroup * dblock); only diagonal blocks are
  // written, problem index b * dgroup + block, up to dtotal problems (0: off)
  int dblock = 0, dgroup = 1, dtotal = 0;
  float4* ws = nullptr;               // per-CTA running sums across chunks, gridDim.x * 128 * BN
  float4* cw = nullptr;               // per-CTA newest chunk values, same shape
  FastDiv cdiv;                       // division by vc.kin
  int* status = nullptr;              // status[1] <- error code of a device-side wait that gave up
  // column blocks: tile nt covers output columns [nt * nstride, nt * nstride + nstride) of N
  // (B rows from nt * nstride), nstride <= BN; 0: nstride = BN
  int nstride = 0;
  // Slice output (so = 1): instead of C, the tile's final values are written as the bf16 slice
  // groups of the next contraction's operand (planes [group][k-step][row][64] at so_dst, so_rows
  // rows, so_ksteps k-steps of 16). Output (m, n) of batch (bo, bi), with m = m_hi so_mdiv + m_lo
  // and n = n_hi so_ndiv + n_lo, goes to
  //   row   = bo so_row_bs_out + bi so_row_bs_in + m_hi so_rm + n_hi so_rn,
  //   chunk = bo so_ch_bs_out + bi so_ch_bs_in + (n_lo / so_cb) so_ch_cb + m_lo / 4,
  //   k     = chunk (4 so_cb) + 16 ((n_lo % so_cb) / 4) + 4 (m_lo % 4) + n_lo % 4,
  // so that one chunk (4 consecutive rows m_lo x so_cb consecutive columns n_lo) lies in one
  // tile and shares one slice alignment, the largest |value| of the chunk; within a k-step of 16
  // (4 rows x 4 columns) each row's 4 values are contiguous, so that a lane writes its own
  // 8 bytes per slice (every producer of a consumer's two operands uses this order). so_xhalf: a chunk
  // spans both column halves of the tile (their maxima are exchanged). Requires so_mdiv % 4 == 0,
  // so_cb % 4 == 0, 4-aligned column ranges, and no block-diagonal batching.
  int so = 0, so_xhalf = 0;
  __nv_bfloat16* so_dst = nullptr;
  long long so_rows = 0;
  int so_ksteps = 0, so_cb = 0, so_ch_cb = 0, so_mdiv = 1, so_ndiv = 1 << 30;
  FastDiv so_ndivf, so_cbf;            // so_ndiv and so_cb as multiply-high divisors (set at launch)
  long long so_rm = 0, so_rn = 0, so_row_bs_in = 0, so_row_bs_out = 0, so_ch_bs_in = 0, so_ch_bs_out = 0;
};

// Error-free FP32 sum: s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Double-float addition (hi, lo) + (bh, bl), about 2^-44 relative.
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(lo, bl));
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kWaitLimitNs = 4000000000ull;   // 4 s: far beyond any legitimate wait

// Bounded wait. Returns false when the CTA is aborting or the limit passed (and then raises abort).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          int code, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      atomicExch(status + 1, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Instruction descriptor for kind::f16: D f32, A and B bf16, both K-major, M = 128; optionally B negated.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, bool neg_b) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((neg_b ? 1u : 0u) << 14) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kBM >> 4) << 24);
}

// D (TMEM) (+)= A (shared memory, descriptor) * B (shared memory, descriptor)^T
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Output tile 128 x 80. The planes of an operand are stored in groups of four
// slices: group 0 holds the real parts, group 1 the imaginary parts; within a group one
// 128-byte row holds the four slices of 16 consecutive k (slice s at bytes
// [32 s, 32 s + 32)). A stage is one such 128-byte row per operand row and
// group, loaded by one TMA box per group with the 128-byte swizzle; slice s is
// addressed by advancing the descriptor start by 32 s bytes inside the
// swizzle atom. B sits as three consecutive 80-row blocks [Bi; Br; -Bi] (the
// third made from the first by a sign flip in shared memory, by warp 10) so
// that one complex slice product is two MMAs of N = 160:
//   A_r x [Bi; Br]  -> columns [0, 80) += A_r B_i,  [80, 160) += A_r B_r
//   A_i x [Br; -Bi] -> columns [0, 80) += A_i B_r,  [80, 160) -= A_i B_i
// (imaginary part first, real part second). Three orders take 480 TMEM
// columns. After each chunk the epilogue moves the chunk value out of TMEM
// (into the output when the contraction has one chunk, else into per-CTA
// scratch), releases TMEM, and only then merges it into the running sum while
// the next chunk's MMAs run.
template <int BN_>
struct OzShape {
  static constexpr int kBN = BN_;                      // output columns per tile (40, 56, 72 or 80)
  static constexpr int kStages = kBN <= 56 ? 4 : 3;
  static constexpr int kRowBytes = 128;                // four slices x 16 k x bf16
  static constexpr int kAGroup = kBM * kRowBytes;      // bytes of one A group tile
  static constexpr int kBBlock = kBN * kRowBytes;      // bytes of one B group block
  static constexpr uint32_t kStageBytes = 2 * kAGroup + 3 * kBBlock;
  static constexpr uint32_t kTxBytes = 2 * kAGroup + 2 * kBBlock;   // what TMA brings per stage
  static constexpr int kThreads = 352;                 // producer, MMA, 8 epilogue warps, negation warp
  static constexpr int kOrderCols = 2 * kBN;           // [im | re] of one order
  static constexpr int kTmemCols = 512;
  // accumulator sets in TMEM: two where they fit (tiles up to 40 columns), so that the MMAs of
  // the next chunk run while the epilogue drains the last one
  static constexpr int kBufCols = 3 * kOrderCols;
  static constexpr int kBufs = 2 * kBufCols <= kTmemCols ? 2 : 1;
  // slice output: maxima exchanged between column halves (two tiles in flight x 4 lane quarters x
  // 2 halves x 32 lanes)
  static constexpr int kXmaxBytes = 2 * 4 * 2 * 32 * 4;
  static constexpr size_t kSmem = 1024 + (size_t)kStages * kStageBytes + 256 + kXmaxBytes;
  static_assert(3 * kOrderCols <= kTmemCols, "three orders must fit in TMEM");
  static_assert(kStageBytes % 1024 == 0, "stages must keep the 1024-byte swizzle alignment");
  static_assert(kSmem <= 232448, "stages exceed shared memory");
  static_assert((2 * kBN) % 16 == 0, "M = 128 MMAs need N a multiple of 16");
  static constexpr int kG = (kBN / 2) % 8 == 0 ? 8 : 4;   // epilogue column group
};
constexpr int kMaxBN = 80;

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: 8-row atoms of
// 128 bytes, 1024 bytes between 8-row groups; version 1 (bits 46-47); layout
// type 2 (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <int G>
__device__ __forceinline__ void tmem_ldg(uint32_t taddr, float* v) {
  if constexpr (G == 8) tmem_ld8(taddr, v);
  else tmem_ld4(taddr, v);
}

template <int BN_, bool SO>
__global__ void __launch_bounds__(352, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const OzParams p) {
  using S = OzShape<BN_>;
  constexpr int G = S::kG;
  constexpr int BN = S::kBN;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S::kStages * S::kStageBytes);
  uint64_t* full = bars;                           // TMA landed
  uint64_t* empty = bars + S::kStages;             // MMAs done with the stage
  uint64_t* ready = bars + 2 * S::kStages;         // -Bi block written
  uint64_t* acc_full = bars + 3 * S::kStages;      // [2]: chunk done, per accumulator set
  uint64_t* acc_empty = acc_full + 2;              // [2]: accumulator set drained
  uint64_t* drain_bar = acc_full + 4;
  uint64_t* xbar = acc_full + 5;                   // slice output: column-half maxima written
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  uint32_t* xmax = reinterpret_cast<uint32_t*>(smem + (size_t)S::kStages * S::kStageBytes + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
      mbar_init(&ready[s], 1);
    }
    for (int b = 0; b < S::kBufs; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 8);           // one arrival per epilogue warp
    }
    mbar_init(drain_bar, 1);
    mbar_init(xbar, 8);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int tiles_per_batch = p.mtiles * p.ntiles;
  const int total_tiles = p.nbatch * tiles_per_batch;
  const int nstride = p.nstride > 0 ? p.nstride : BN;
  const int nchunks = (p.nsteps + p.steps_per_chunk - 1) / p.steps_per_chunk;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: per k-step A (re, im) and B (im, re) group tiles
      uint32_t step = 0;
      for (int tile = blockIdx.x; tile < total_tiles && !*abort_flag; tile += gridDim.x) {
        const int b = tile / tiles_per_batch, mt = (tile % tiles_per_batch) / p.ntiles, nt = tile % p.ntiles;
        const int bo = b / p.bin, bi = b % p.bin;
        const int arow = (int)(p.a_row0 + (p.a_tab ? p.a_tab[bi] : bi * p.a_bs_in) + bo * p.a_bs_out) + mt * kBM;
        const int brow = (int)(p.b_row0 + (p.b_tab ? p.b_tab[bi] : bi * p.b_bs_in) + bo * p.b_bs_out) + nt * nstride;
        for (int s = 0; s < p.nsteps; ++s, ++step) {
          const int st = step % S::kStages;
          const uint32_t ph = (step / S::kStages) & 1;
          if (!mbar_wait(&empty[st], ph ^ 1, abort_flag, p.status, 11)) break;
          mbar_expect_tx(&full[st], S::kTxBytes);
          uint8_t* sa = smem + (size_t)st * S::kStageBytes;
          uint8_t* sb = sa + 2 * S::kAGroup;
          tma_load_3d(sa, &tmA, 0, arow, s, &full[st]);                                // A re
          tma_load_3d(sa + S::kAGroup, &tmA, 0, arow, p.nsteps + s, &full[st]);        // A im
          tma_load_3d(sb, &tmB, 0, brow, p.nsteps + s, &full[st]);                     // B im
          tma_load_3d(sb + S::kBBlock, &tmB, 0, brow, s, &full[st]);                   // B re
        }
      }
      if (*abort_flag) {
        // let every issued copy land before the CTA exits (bounded)
        const uint64_t t0 = globaltimer();
        for (int k = 0; k < S::kStages && step > 0; ++k) {
          const uint32_t st2 = (step - 1 - k) % S::kStages;
          const uint32_t ph2 = ((step - 1 - k) / S::kStages) & 1;
          while (!mbar_try(&full[st2], ph2) && globaltimer() - t0 < kWaitLimitNs) {
          }
          if (step - 1 - k == 0) break;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      uint32_t step = 0, chunk = 0;
      const uint32_t idesc = idesc_bf16(2 * BN, false);
      const uint64_t desc0 = sw128_desc(smem_u32(smem));
      bool ok = true;
      for (int tile = blockIdx.x; tile < total_tiles && ok; tile += gridDim.x) {
        for (int s = 0; s < p.nsteps && ok; ++s, ++step) {
          const bool chunk_start = (s % p.steps_per_chunk) == 0;
          const uint32_t buf = chunk % S::kBufs;
          if (chunk_start) {
            if (!mbar_wait(&acc_empty[buf], ((chunk / S::kBufs) & 1) ^ 1, abort_flag, p.status, 12)) { ok = false; break; }
            tc_fence_after();
          }
          const int st = step % S::kStages;
          const uint32_t ph = (step / S::kStages) & 1;
          if (!mbar_wait(&ready[st], ph, abort_flag, p.status, 13)) { ok = false; break; }
          tc_fence_after();
          // descriptor start fields (address >> 4) of this stage; shared memory < 256 KB: no carry
          const uint64_t sa = desc0 + (uint64_t)((st * S::kStageBytes) >> 4);
          const uint64_t sb = sa + (uint64_t)((2 * S::kAGroup) >> 4);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              if (i + jj > 3) continue;
              const int acc = (i + jj == 0) ? 0 : (i + jj == 1 ? 1 : 2);
              const uint32_t d = tmem + buf * S::kBufCols + (uint32_t)(acc * S::kOrderCols);
              // first write of each accumulator in a chunk: (0,0), (0,1) and (0,2) in loop order
              const bool first = chunk_start && i == 0 && jj == acc;
              const uint64_t ar = sa + (uint64_t)(2 * i);                          // +32 i bytes
              const uint64_t ai = ar + (uint64_t)(S::kAGroup >> 4);
              const uint64_t b01 = sb + (uint64_t)(2 * jj);                        // [Bi; Br]
              const uint64_t b12 = b01 + (uint64_t)(S::kBBlock >> 4);              // [Br; -Bi]
              mma_bf16(d, ar, b01, idesc, first ? 0u : 1u);
              mma_bf16(d, ai, b12, idesc, 1u);
            }
          }
          mma_commit(&empty[st]);
          if ((s % p.steps_per_chunk) == p.steps_per_chunk - 1 || s == p.nsteps - 1) {
            mma_commit(&acc_full[buf]);
            ++chunk;
          }
        }
      }
      // wait for the last MMAs before the TMEM is released
      mma_commit(drain_bar);
      const uint64_t t0 = globaltimer();
      while (!mbar_try(drain_bar, 0) && globaltimer() - t0 < kWaitLimitNs) {
      }
    }
  } else if (warp == 10) {
    // ---------------- -Bi block of each stage: sign flip of the Bi block (same swizzle phase)
    uint32_t step = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < total_tiles && ok; tile += gridDim.x) {
      for (int s = 0; s < p.nsteps; ++s, ++step) {
        const int st = step % S::kStages;
        const uint32_t ph = (step / S::kStages) & 1;
        int w = 1;
        if (lane == 0) w = mbar_wait(&full[st], ph, abort_flag, p.status, 15);
        if (!__shfl_sync(0xffffffffu, w, 0)) { ok = false; break; }
        const uint4* src = reinterpret_cast<const uint4*>(smem + (size_t)st * S::kStageBytes + 2 * S::kAGroup);
        uint4* dst = const_cast<uint4*>(src) + 2 * S::kBBlock / 16;
        constexpr int kVec = S::kBBlock / 16;          // 640 per block
#pragma unroll 4
        for (int v = lane; v < kVec; v += 32) {
          uint4 x = src[v];
          x.x ^= 0x80008000u;
          x.y ^= 0x80008000u;
          x.z ^= 0x80008000u;
          x.w ^= 0x80008000u;
          dst[v] = x;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&ready[st]);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; TMEM lane quarter = warp % 4, columns [40 half, 40 half + 40)
    const int quarter = warp & 3;
    const int half = (warp - 2) >> 2;
    constexpr int kCols = BN / 2;
    static_assert(kCols % 4 == 0, "the chunk merge takes columns in groups of 4");
    constexpr int kNG4 = kCols / 4;
    // groups whose running sum stays in registers; the rest go through the per-CTA scratch. At the
    // 168-register limit of 352 threads more groups spill: 3 (48 registers) where the kernel has
    // no slice output, 2 for the wide slice-output tiles, none for the narrow ones (the V.G
    // products, whose one-chunk path slows down with any more live registers)
    constexpr int kRGWant = !SO ? 3 : (BN >= 72 ? 2 : 0);
    constexpr int kRG = kNG4 < kRGWant ? kNG4 : kRGWant;
    const int lrow = quarter * 32 + lane;            // TMEM lane = row within the tile
    // per-CTA scratch, column-major so that a warp's 32 rows of one column are contiguous:
    // ws holds the running sum, cw the newest chunk value
    float4* ws = p.ws + (size_t)blockIdx.x * BN * kBM + lrow;
    float4* cw = p.cw + (size_t)blockIdx.x * BN * kBM + lrow;
    uint32_t chunk = 0;
    uint32_t so_tile = 0;                            // slice-output tiles with a column-half exchange
    for (int tile = blockIdx.x; tile < total_tiles; tile += gridDim.x) {
      const int b = tile / tiles_per_batch, mt = (tile % tiles_per_batch) / p.ntiles, nt = tile % p.ntiles;
      int row = mt * kBM + lrow;
      bool row_ok = row < p.M;
      // block-diagonal mode: the tile holds dgroup problems of dblock rows and columns; this
      // row belongs to problem b * dgroup + row / dblock and only its own column block is kept
      int dcol0 = 0, ncols = 1 << 30;
      int ob = b;
      if (p.dblock) {
        const int blk = row / p.dblock;
        ob = b * p.dgroup + blk;
        row_ok = row_ok && ob < p.dtotal;
        dcol0 = blk * p.dblock;
        ncols = p.dblock;
        row -= dcol0;
      }
      const int bo = ob / p.bin, bi = ob % p.bin;
      double2* C = p.C + (p.bc.tab ? p.bc.tab[bi] : (long long)bi * p.bc.bs_in) + (long long)bo * p.bc.bs_out;
      const long long roff = row_ok ? s_view_row(p.vc, row) : 0;
      // output column of tile column cl: nt * nstride + cl - dcol0 (valid if in [0, min(N, ncols)))
      auto col_ok = [&](int cl) {
        const int n = nt * nstride + cl - dcol0;
        return row_ok && cl - dcol0 >= 0 && cl - dcol0 < ncols && cl < nstride && n < p.N;
      };
      auto out_write = [&](int cl, float rh, float rl, float ih, float il) {
        if constexpr (SO) {                           // kept for the slice output below
          cw[(size_t)cl * kBM] = make_float4(rh, rl, ih, il);
          return;
        }
        const int n = nt * nstride + cl - dcol0;
        const int nq = fdiv(n, p.cdiv);
        double2* dst = C + roff + (long long)nq * p.vc.ks_out + (long long)(n - nq * p.vc.kin) * p.vc.ks_in;
        if (p.out_df) {
          *reinterpret_cast<float4*>(dst) = make_float4(rh, rl, ih, il);
        } else {
          double re = p.alpha * ((double)rh + (double)rl);
          double im = p.alpha * ((double)ih + (double)il);
          if (p.accumulate) {
            const double2 o = *dst;
            re += o.x;
            im += o.y;
          }
          *dst = make_double2(re, im);
        }
      };
      bool ok = true;
      // ---- slice output helpers. A chunk of the next contraction is 4 consecutive rows (this
      //      lane and its 3 neighbours) x so_cb columns; its alignment 2^E comes from the largest
      //      |hi| of its re and im parts, as in slice_kernel.
      const int m_so = mt * kBM + lrow;               // producer row within the batch
      const bool mok = m_so < p.M;
      // the row's part of the consumer position (the column part varies per 4-column group)
      const int so_mhi = SO ? m_so / p.so_mdiv : 0, so_mlo = m_so - so_mhi * p.so_mdiv;
      const long long so_row0 = bo * p.so_row_bs_out + bi * p.so_row_bs_in + (long long)so_mhi * p.so_rm;
      const long long so_ch0 = bo * p.so_ch_bs_out + bi * p.so_ch_bs_in + so_mlo / 4;
      uint32_t so_mx = 0;                             // largest |hi| of this thread's values (bits)
      // alignment of this lane group's chunk from the thread maxima; returns true for a chunk
      // taken as zero (largest value below 2^-90: its slices would be subnormal)
      auto so_alignment = [&](uint32_t mx, float* magic) -> bool {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
        if (p.so_xhalf) {
          // the chunk's other columns belong to the warp with the same lanes and the other half
          const uint32_t par = so_tile & 1;
          xmax[((par * 4 + quarter) * 2 + half) * 32 + lane] = mx;
          __syncwarp();
          int w = 1;
          if (lane == 0) {
            mbar_arrive(xbar);
            w = mbar_wait(xbar, par, abort_flag, p.status, 16);
          }
          w = __shfl_sync(0xffffffffu, w, 0);
          __syncwarp();
          if (w) mx = max(mx, xmax[((par * 4 + quarter) * 2 + (half ^ 1)) * 32 + lane]);
          else ok = false;
          ++so_tile;
        }
        const int eb = (int)((mx >> 23) & 0xFF);
        const int E = eb - 126;                       // every |value| / 2^E < 1
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) magic[sl] = ldexpf(3.0f, E + 15 - 8 * sl);   // 1.5 * 2^23 * q_sl
        return eb == 0 || E < -90;
      };
      // slices of 4 columns c0..c0+3 of this row (double-float values f) -> one 16-wide line of the
      // consumer's planes (128 bytes per part), of which this lane writes its row's 8 bytes per slice
      auto so_line = [&](int c0, const float4* f, bool zero, const float* magic) {
        const int n0 = nt * nstride + c0;
        const bool gok = ok && mok && c0 < nstride && n0 < p.N;   // the same for all 4 columns and lanes
        if (!gok) return;
        const int n_hi = fdiv(n0, p.so_ndivf), n_lo = n0 - n_hi * p.so_ndiv;
        const int c_hi = fdiv(n_lo, p.so_cbf), c_lo = n_lo - c_hi * p.so_cb;
        const long long crow = so_row0 + (long long)n_hi * p.so_rn;
        const long long ch = so_ch0 + (long long)c_hi * p.so_ch_cb;
        const long long kstep = ch * (p.so_cb >> 2) + (c_lo >> 2);
        if (crow < 0 || crow >= p.so_rows || kstep < 0 || kstep >= p.so_ksteps) {
          atomicExch(p.status + 1, 17);              // a layout outside the planes: recorded, not written
          return;
        }
        const int j4 = lane & 3;
#pragma unroll
        for (int gr = 0; gr < 2; ++gr) {              // real part, then imaginary part
          float sv[4][4];                             // [column][slice]
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
#pragma unroll
            for (int sl = 0; sl < 4; ++sl) sv[cc][sl] = 0.f;
            if (!zero) df_slices(gr ? f[cc].z : f[cc].x, gr ? f[cc].w : f[cc].y, magic, sv[cc]);
          }
          __nv_bfloat16* dst = p.so_dst + (((long long)gr * p.so_ksteps + kstep) * p.so_rows + crow) * 64 + 4 * j4;
#pragma unroll
          for (int sl = 0; sl < 4; ++sl) {
            // exact: digit x 2^(E-7-8 sl)
            const __nv_bfloat162 lo = __floats2bfloat162_rn(sv[0][sl], sv[1][sl]);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(sv[2][sl], sv[3][sl]);
            uint2 w;
            w.x = *reinterpret_cast<const uint32_t*>(&lo);
            w.y = *reinterpret_cast<const uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(dst + 16 * sl) = w;
          }
        }
      };
      // running sums of the first kRG groups of 4 columns of this warp (chunked contractions)
      float4 rs[kRG > 0 ? kRG : 1][4];
      for (int c = 0; c < nchunks; ++c, ++chunk) {
        const uint32_t buf = chunk % S::kBufs;
        if (!mbar_wait(&acc_full[buf], (chunk / S::kBufs) & 1, abort_flag, p.status, 14)) { ok = false; break; }
        tc_fence_after();
        const bool single = nchunks == 1;
        const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + buf * S::kBufCols;
        if (SO && single) {
          // ---- slice output of a one-chunk contraction straight from TMEM: pass 1 finds the row
          //      maximum, pass 2 slices 4 columns at a time; TMEM is released after pass 2
          uint32_t mx = 0;
#pragma unroll 1
          for (int g = 0; g < kCols / G; ++g) {
            const int cb = half * kCols + g * G;
            float v[2][2][G];                         // orders 0 and 1: the maximum takes the hi word
            const uint32_t taddr = tbase + (uint32_t)cb;
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              tmem_ldg<G>(taddr + o * S::kOrderCols, v[o][0]);
              tmem_ldg<G>(taddr + o * S::kOrderCols + BN, v[o][1]);
            }
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < G; ++u) {
              if (!col_ok(cb + u)) continue;
              float rh, rl, ih, il;
              two_sum(v[0][1][u], v[1][1][u], rh, rl);
              two_sum(v[0][0][u], v[1][0][u], ih, il);
              mx = max(mx, max(__float_as_uint(rh) & 0x7FFFFFFFu, __float_as_uint(ih) & 0x7FFFFFFFu));
            }
          }
          float magic[4];
          const bool zero = so_alignment(mx, magic);
#pragma unroll 1
          for (int g4 = 0; g4 < kCols / 4; ++g4) {
            const int c0 = half * kCols + 4 * g4;
            float v[3][2][4];
            const uint32_t taddr = tbase + (uint32_t)c0;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
              tmem_ld4(taddr + o * S::kOrderCols, v[o][0]);
              tmem_ld4(taddr + o * S::kOrderCols + BN, v[o][1]);
            }
            tmem_wait_ld();
            float4 f[4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              float rh, rl, ih, il;
              two_sum(v[0][1][cc], v[1][1][cc], rh, rl);
              rl = __fadd_rn(rl, v[2][1][cc]);
              two_sum(v[0][0][cc], v[1][0][cc], ih, il);
              il = __fadd_rn(il, v[2][0][cc]);
              f[cc] = make_float4(rh, rl, ih, il);
            }
            so_line(c0, f, zero, magic);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
          continue;
        }
        if (single) {
          // ---- one-chunk contraction: TMEM -> value (an exact FP32 pair per part) -> output
#pragma unroll 1
          for (int g = 0; g < kCols / G; ++g) {
            const int cb = half * kCols + g * G;
            float v[3][2][G];                         // [order][im, re][column]
            const uint32_t taddr = tbase + (uint32_t)cb;
#pragma unroll
            for (int o = 0; o < 3; ++o) {
              tmem_ldg<G>(taddr + o * S::kOrderCols, v[o][0]);
              tmem_ldg<G>(taddr + o * S::kOrderCols + BN, v[o][1]);
            }
            tmem_wait_ld();
            if (g == kCols / G - 1) {
              // this warp's accumulator columns are in registers: release TMEM
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&acc_empty[buf]);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
              const int cl = cb + u;
              if (!col_ok(cl)) continue;
              // orders 0 and 1 are exact, so their sum is exact as a pair
              float rh, rl, ih, il;
              two_sum(v[0][1][u], v[1][1][u], rh, rl);
              rl = __fadd_rn(rl, v[2][1][u]);
              two_sum(v[0][0][u], v[1][0][u], ih, il);
              il = __fadd_rn(il, v[2][0][u]);
              out_write(cl, rh, rl, ih, il);
            }
          }
          continue;
        }
        const bool last = c == nchunks - 1;
        // chunk value of one column (an exact FP32 pair per part: orders 0 and 1 are exact)
        auto chunk_value = [](const float (&v)[3][2][4], int u) {
          float rh, rl, ih, il;
          two_sum(v[0][1][u], v[1][1][u], rh, rl);
          rl = __fadd_rn(rl, v[2][1][u]);
          two_sum(v[0][0][u], v[1][0][u], ih, il);
          il = __fadd_rn(il, v[2][0][u]);
          return make_float4(rh, rl, ih, il);
        };
        auto tmem_group = [&](int cb, float (&v)[3][2][4]) {
          const uint32_t taddr = tbase + (uint32_t)cb;
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            tmem_ld4(taddr + o * S::kOrderCols, v[o][0]);
            tmem_ld4(taddr + o * S::kOrderCols + BN, v[o][1]);
          }
          tmem_wait_ld();
        };
        auto release = [&]() {                        // this warp's columns are out of TMEM
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[buf]);
        };
        // ---- resident columns: the running sum stays in registers from chunk to chunk
#pragma unroll
        for (int g = 0; g < kRG; ++g) {
          const int cb = half * kCols + 4 * g;
          float v[3][2][4];
          tmem_group(cb, v);
          if (g == kNG4 - 1) release();
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 x = chunk_value(v, u);
            float4& a = rs[g][u];
            if (c == 0) {
              a = x;
            } else {
              df_add(a.x, a.y, x.x, x.y);
              df_add(a.z, a.w, x.z, x.w);
            }
            if (last && col_ok(cb + u)) {
              if (SO) so_mx = max(so_mx, max(__float_as_uint(a.x) & 0x7FFFFFFFu, __float_as_uint(a.z) & 0x7FFFFFFFu));
              out_write(cb + u, a.x, a.y, a.z, a.w);
            }
          }
        }
        // ---- the other columns: chunk value to the per-CTA scratch, then TMEM is released
#pragma unroll 1
        for (int g = kRG; g < kNG4; ++g) {
          const int cb = half * kCols + 4 * g;
          float v[3][2][4];
          tmem_group(cb, v);
          if (g == kNG4 - 1) release();
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (col_ok(cb + u)) (c == 0 ? ws : cw)[(size_t)(cb + u) * kBM] = chunk_value(v, u);
        }
        // ---- and merged into their running sum there (overlaps the next chunk's MMAs)
        if (c > 0) {
#pragma unroll 1
          for (int g = kRG; g < kNG4; ++g) {
            const int cb = half * kCols + 4 * g;
            float4 a[4], x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (col_ok(cb + u)) {
                a[u] = ws[(size_t)(cb + u) * kBM];
                x[u] = cw[(size_t)(cb + u) * kBM];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int cl = cb + u;
              if (!col_ok(cl)) continue;
              df_add(a[u].x, a[u].y, x[u].x, x[u].y);
              df_add(a[u].z, a[u].w, x[u].z, x[u].w);
              if (SO && last)
                so_mx = max(so_mx, max(__float_as_uint(a[u].x) & 0x7FFFFFFFu, __float_as_uint(a[u].z) & 0x7FFFFFFFu));
              if (last) out_write(cl, a[u].x, a[u].y, a[u].z, a[u].w);
              else ws[(size_t)cl * kBM] = a[u];
            }
          }
        }
      }
      if (SO && nchunks > 1 && ok) {
        // ---- slice output of a chunked contraction: the final values wait in cw; the next
        //      group's loads are issued before the current group is sliced
        float magic[4];
        const bool zero = so_alignment(so_mx, magic);
        auto load4 = [&](int c0, float4* f) {
          const bool gok = mok && c0 < nstride && nt * nstride + c0 < p.N;
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) f[cc] = gok ? cw[(size_t)(c0 + cc) * kBM] : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        float4 cur[4], nxt[4];
        load4(half * kCols, cur);
#pragma unroll 1
        for (int g4 = 0; g4 < kCols / 4; ++g4) {
          const int c0 = half * kCols + 4 * g4;
          if (g4 + 1 < kCols / 4) load4(c0 + 4, nxt);
          so_line(c0, cur, zero, magic);
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) cur[cc] = nxt[cc];
        }
      }
      if (!ok) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols));
  }
}

// Self-test of the bounded wait: one thread waits, with the production routine, on an mbarrier
// phase that nothing completes (no arrivals); the wait must give up after limit_ns, write its code
// to status[1] and let the kernel return.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = mbar_wait(&bar, 0, &abort_flag, status, 99, limit_ns);
    if (ok) atomicExch(status, 1);        // would mean the phase completed: not expected
  }
}

// ------------------------------------------------------------------------------------------------
// host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// Planes buffer: 2 groups x (Kpad / 16) x rows x 64 bf16. Group 0 holds the real slices,
// group 1 the imaginary ones; the 64 values of (group, k-step, row) are the four slices
// of 16 consecutive k.
struct Planes {
  __nv_bfloat16* ptr = nullptr;
  long long rows = 0;
  int Kpad = 0, Kc = 0;
  int groups = 2;
  size_t elems() const { return (size_t)groups * 4 * rows * Kpad; }
};

int num_sms() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return std::max(v, 1);
  }();
  return n;
}

int make_map(const Planes& P, int box_rows, CUtensorMap* map) {
  auto enc = encode_fn();
  if (!enc) return fail(GW_ECUDA, "cuTensorMapEncodeTiled is not available");
  // (64 values of one row and k-step, rows, group * k-steps); one box: 64 x box_rows x 1
  cuuint64_t dims[3] = {64, (cuuint64_t)P.rows, (cuuint64_t)P.groups * (P.Kpad / kStepK)};
  cuuint64_t strides[2] = {128, (cuuint64_t)P.rows * 128};
  cuuint32_t box[3] = {64, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)P.ptr, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(GW_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GW_OK;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// chunk length and padded K for a contraction of length K
// (equal chunks of at most 256, each a multiple of 16: the padding stays below 16 per chunk)
inline void chunking(int K, int* Kc, int* Kpad) {
  const int nc = (std::max(K, 1) + kMaxChunk - 1) / kMaxChunk;
  *Kc = round_up((std::max(K, 1) + nc - 1) / nc, kStepK);
  *Kpad = nc * *Kc;
}

int launch_slice(const SliceJob& j, cudaStream_t st) {
  const int nchunk = j.Kpad / j.Kc;
  const long long warps = (long long)j.nbatch * j.rows * nchunk;
  if (warps == 0) return GW_OK;
  const long long blocks = (warps + 7) / 8;
  if (blocks > 2147483647LL) return fail(GW_EINVAL, "slice: too many rows");
  prof_begin(SLOT_LIMBS, st);
  if (j.src_df)
    slice_kernel<true><<<(unsigned)blocks, 256, 0, st>>>(j);
  else
    slice_kernel<false><<<(unsigned)blocks, 256, 0, st>>>(j);
  prof_end(SLOT_LIMBS, st, 0.0, (double)warps * j.Kc * (16.0 + 16.0));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "slice launch: %s", cudaGetErrorString(e));
}


template <int BN_>
int launch_oz_bn(const Planes& A, const Planes& B, OzParams p, int slot, cudaStream_t st) {
  using S = OzShape<BN_>;
  if (A.Kpad != B.Kpad || A.Kc != B.Kc) return fail(GW_EINVAL, "oz_gemm: operand chunking differs");
  if (A.groups != 2 || B.groups != 2) return fail(GW_EINVAL, "oz_gemm: operands need two slice groups");
  p.nsteps = A.Kpad / kStepK;
  p.steps_per_chunk = A.Kc / kStepK;
  if (p.nstride < 0 || p.nstride > S::kBN) return fail(GW_EINVAL, "oz_gemm: column stride above the tile width");
  const int nstride = p.nstride > 0 ? p.nstride : S::kBN;
  if (p.so) {
    // a chunk is 4 rows (a lane group) by so_cb columns within one tile, or one column half
    const bool halves_ok = p.so_xhalf ? p.so_cb >= nstride : (S::kBN / 2) % p.so_cb == 0;
    if (p.dblock || !p.so_dst || p.so_mdiv % 4 || p.so_cb % 4 || p.so_cb <= 0 || p.M % 4 || p.N % 4 ||
        nstride % 4 || !halves_ok || p.so_ksteps <= 0 || p.so_rows <= 0)
      return fail(GW_EINVAL, "oz_gemm: slice output layout not supported");
    p.so_ndivf = make_fastdiv(p.so_ndiv);
    p.so_cbf = make_fastdiv(p.so_cb);
  }
  p.mtiles = (p.M + kBM - 1) / kBM;
  p.ntiles = (p.N + nstride - 1) / nstride;
  const long long total = (long long)p.nbatch * p.mtiles * p.ntiles;
  if (total == 0) return GW_OK;
  if (total > 2147483647LL) return fail(GW_EINVAL, "oz_gemm: too many tiles");
  if (!p.ws) return fail(GW_EINVAL, "oz_gemm: no epilogue scratch");
  p.cdiv = make_fastdiv(p.vc.kin);
  p.cw = p.ws + (size_t)num_sms() * kBM * S::kBN;
  CUtensorMap ma, mb;
  GW_TRY_INTERNAL(make_map(A, kBM, &ma));
  GW_TRY_INTERNAL(make_map(B, S::kBN, &mb));
  // one-time setup; function-local statics initialise once even when contexts run on several threads
  static const bool attr = [] {
    cudaFuncSetAttribute(oz_gemm_kernel<BN_, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
    cudaFuncSetAttribute(oz_gemm_kernel<BN_, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kSmem);
    return true;
  }();
  (void)attr;
  const int grid = (int)std::min<long long>(total, num_sms());
  prof_begin(slot, st);
  if (p.so)
    oz_gemm_kernel<BN_, true><<<grid, S::kThreads, S::kSmem, st>>>(ma, mb, p);
  else
    oz_gemm_kernel<BN_, false><<<grid, S::kThreads, S::kSmem, st>>>(ma, mb, p);
  // executed bf16 tensor flops: 10 slice products x 2 real MMAs of 128 x (2 BN) x 16 per k-step
  prof_end(slot, st, 2.0 * 20.0 * (double)total * kBM * (2 * S::kBN) * (double)p.nsteps * kStepK,
           (double)total * p.nsteps * S::kTxBytes);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GW_OK : fail(GW_ECUDA, "oz_gemm launch: %s", cudaGetErrorString(e));
}

// Tile width by the padding of N: 72 columns (MMA N = 144) when that covers N with fewer padded
// columns than 80 (for example N = 200: 216 instead of 240), else 80. Narrower tiles are taken
// only where a launch asks for them: 56 (block-diagonal tiles, column blocks of 52..56) and 40.
// At 40 columns (MMA N = 80) two accumulator sets fit in TMEM and the next tile's MMAs overlap the
// epilogue, but each MMA reads the 128-row A tile from shared memory for half the work, which
// makes long contractions bound by shared-memory bandwidth (measured: P0 and R 25-50% slower);
// it pays only for the one-chunk V.G product of the fused path, whose epilogue dominates.
int oz_tile_width(long long N) {
  const long long pad72 = (N + 71) / 72 * 72, pad80 = (N + 79) / 80 * 80;
  return pad72 < pad80 ? 72 : 80;
}

int launch_oz(const Planes& A, const Planes& B, OzParams p, int slot, cudaStream_t st, int bn = 0) {
  if (bn == 0) bn = oz_tile_width(p.N);
  if (bn == 40) return launch_oz_bn<40>(A, B, p, slot, st);
  if (bn == 56) return launch_oz_bn<56>(A, B, p, slot, st);
  if (bn == 72) return launch_oz_bn<72>(A, B, p, slot, st);
  return launch_oz_bn<80>(A, B, p, slot, st);
}

// Block-diagonal grouping of nao x nao problems: the tile width and the problems per tile that
// make the most of each 128 x BN tile (g problems of nao x nao on its diagonal, g nao <= 128).
void oz_block_diag(int nao, int* bn, int* grp) {
  double best = -1.0;
  for (int w : {80, 72, 56}) {
    const int g = std::max(1, std::min(kBM, w) / nao);
    const double use = (double)g * nao * nao / ((double)kBM * w);
    if (use > best + 1e-12) best = use, *bn = w, *grp = g;
  }
}

// Automatic tau batch (nodes per batch of the contractions). The largest batch whose
// intermediates take at most 12 GiB, unless that leaves the P0 launches (batch x P0 tiles per
// node) under two waves over the SMs: then, within 64 GiB, the batch whose P0 launches fill
// their waves best (over the canonical tau ranges the launches take), the smaller on a tie.
int auto_tau_batch(const MixedDims& d, double per_t) {
  const int ntau = d.ntau;
  const int nt12 = (int)std::min<double>(ntau, std::max(1.0, std::floor(12884901888.0 / per_t)));
  const int sms = 152;                         // the GB300's SM count: the choice must not depend on the device
  const long long p0_tiles = (long long)((d.naux + kBM - 1) / kBM) * ((d.naux + oz_tile_width(d.naux) - 1) /
                                                                       oz_tile_width(d.naux));
  if ((long long)nt12 * p0_tiles >= 2LL * sms) return nt12;
  const int nt64 = (int)std::min<double>(ntau, std::max(1.0, std::floor(68719476736.0 / per_t)));
  // canonical tau counts of the q (all nodes, half of them, or none)
  std::vector<int> tends;
  for (int q = 0; q < d.nk; ++q) {
    const int mq = q < (int)d.mq.size() ? d.mq[q] : q;
    tends.push_back(mq < q ? 0 : (mq == q ? (ntau + 1) / 2 : ntau));
  }
  int best = nt12;
  double best_eff = -1.0;
  for (int nt = nt12; nt <= nt64; ++nt) {
    double work = 0.0, slots = 0.0;
    for (int tend : tends) {
      const int nb = (tend + nt - 1) / nt;
      for (int i = 0; i < nb; ++i) {
        const long long tiles = p0_tiles * ((long long)tend * (i + 1) / nb - (long long)tend * i / nb);
        work += (double)tiles;
        slots += (double)((tiles + sms - 1) / sms * sms);
      }
    }
    const double eff = slots > 0.0 ? work / slots : 0.0;
    if (eff > best_eff + 1e-9) best_eff = eff, best = nt;
  }
  return best;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// the mixed stages

// Plane-row tables, [kTabs][nq][nk]: first plane row of each operand block.
// Plane-row tables T_* index the per-context V slices (all nk^2 pairs) and G slices; in per-q
// mode the V operands come from per-q slices with rows k * naux * nao (T_LOC_V) or k * nao^2
// (T_LOC_VC), staged from V through the element-offset tables E_* before each q.
enum {
  T_VKKPQ = 0, T_VKPQK, T_GKPQ, T_GK, T_VKKMQ, T_GKMQ, T_VCOL_KMQK, T_LOC_V, T_LOC_VC,
  E_KKPQ, E_KPQK, E_KKMQ, E_KMQK, kTabs
};

struct MixedState {
  MixedDims d;
  cudaStream_t stream = nullptr;
  int nt = 1;                   // tau nodes per batch
  long long nao2 = 0, naux2 = 0, pair = 0;
  const double2* V = nullptr;
  const double2* Vp = nullptr;  // packed V (pairs k1 <= k2), when given instead of V
  double2* vscratch = nullptr;  // per-q mode with a packed V: the nk full-layout blocks of one table
  Planes vrow, vcol, gf, gm;    // V rows (Q,i) over orbitals; V rows (j,b) over Q'; G^T forward / mirrored tau
  Planes vrowt;                 // fused path, all pairs: V rows (i,Q) over orbitals (the Z operand)
  bool per_q = false;           // V slices staged per q (vq, vcq) instead of held for all pairs
  Planes vq[2], vcq;            // (fused path: vq[0] holds rows (i,Q) during the self-energy)
  // Fused path: the V.G products and R write the slice groups of the next contraction straight
  // from their epilogue (no FP64 or double-float intermediate, no separate slicing pass); the
  // P0 and Sigma contractions then run over chunks that lie within one producer tile.
  bool fused = false;
  __nv_bfloat16* xs_mem = nullptr;   // operand planes for the batched GEMMs (two buffers)
  __nv_bfloat16* ys_mem = nullptr;
  Planes ps;                    // P~ planes
  double2 *x64 = nullptr, *y64 = nullptr;   // double-float intermediates (16 B per element), nt * nk * pair each
  float4* ws = nullptr;                       // per-CTA running sums of the chunked GEMMs
  long long* rowtabs = nullptr;
  int* status = nullptr;
  int Kc_vg = 0, Kpad_vg = 0, Kc_p0 = 0, Kpad_p0 = 0, Kc_r = 0, Kpad_r = 0, Kc_s = 0, Kpad_s = 0;
  __nv_bfloat16* oq_mem = nullptr;   // planes of mixed_outer_q (allocated on first use), oq_rows rows each
  long long oq_rows = 0;
  __nv_bfloat16* ol_mem = nullptr;   // planes of mixed_gf2_last (allocated on first use)
  size_t ol_elems = 0;
  std::vector<void*> allocs;
  std::vector<unsigned char*> guards;   // guard zone of each allocation, in the order of allocs
  bool dry = false;   // size-only: count bytes, allocate nothing
};

namespace {

template <class T>
int m_alloc(MixedState* s, T** p, size_t count, size_t* bytes) {
  if (count == 0) count = 1;
  const size_t nb = count * sizeof(T);
  if (s->dry) {
    *p = nullptr;
    *bytes += nb + kGuardBytes;
    return GW_OK;
  }
  if (cudaMalloc(reinterpret_cast<void**>(p), nb + kGuardBytes) != cudaSuccess) {
    *p = nullptr;
    return fail(GW_ENOMEM, "mixed workspace: cudaMalloc of %zu bytes failed", nb);
  }
  unsigned char* guard = reinterpret_cast<unsigned char*>(*p) + nb;
  cudaMemsetAsync(guard, kGuardByte, kGuardBytes, s->stream);   // ordered before the state's work
  s->allocs.push_back(*p);
  s->guards.push_back(guard);
  *bytes += nb + kGuardBytes;
  return GW_OK;
}

int alloc_planes(MixedState* s, Planes* P, long long rows, int Kc, int Kpad, int groups, size_t* bytes) {
  P->rows = rows;
  P->Kc = Kc;
  P->Kpad = Kpad;
  P->groups = groups;
  return m_alloc(s, &P->ptr, P->elems(), bytes);
}

Planes view(__nv_bfloat16* mem, long long rows, int Kc, int Kpad, int groups) {
  Planes P;
  P.ptr = mem;
  P.rows = rows;
  P.Kc = Kc;
  P.Kpad = Kpad;
  P.groups = groups;
  return P;
}

int kshift3(const int nk3[3], int k, int q, int sign) {
  const int k1 = k / (nk3[1] * nk3[2]), k2 = (k / nk3[2]) % nk3[1], k3 = k % nk3[2];
  const int q1 = q / (nk3[1] * nk3[2]), q2 = (q / nk3[2]) % nk3[1], q3 = q % nk3[2];
  const int a = ((k1 + sign * q1) % nk3[0] + nk3[0]) % nk3[0];
  const int b = ((k2 + sign * q2) % nk3[1] + nk3[1]) % nk3[1];
  const int c = ((k3 + sign * q3) % nk3[2] + nk3[2]) % nk3[2];
  return (a * nk3[1] + b) * nk3[2] + c;
}

const long long* tab(const MixedState* s, int which, int q) {
  return s->rowtabs + ((size_t)which * s->d.nk + q) * s->d.nk;
}

// Slice a batch of FP64 (or, with src_df, double-float) matrices into planes
// (rows x K, per-row chunk alignment).
int slice(MixedState* s, const double2* src, const ZView& v, long long b_in, long long b_out, int bin, int nbatch,
          int rows, int K, const Planes& P, long long dst_rows_per_batch, int src_df = 0,
          const long long* b_tab = nullptr) {
  SliceJob j;
  j.b.tab = b_tab;
  j.src = src;
  j.src_df = src_df;
  j.v = v;
  j.b.bs_in = b_in;
  j.b.bs_out = b_out;
  j.bin = bin;
  j.rows = rows;
  j.K = K;
  j.Kc = P.Kc;
  j.Kpad = P.Kpad;
  j.nbatch = nbatch;
  j.kdiv = make_fastdiv(v.kin);
  j.dst = P.ptr;
  j.dst_rows = P.rows;
  j.dst_rows_per_batch = dst_rows_per_batch;
  return launch_slice(j, s->stream);
}

int slice_g(MixedState* s, const double2* G) {
  const int nk = s->d.nk, ntau = s->d.ntau, nao = s->d.nao;
  for (int mir = 0; mir < 2; ++mir) {
    ZView v;
    v.rin = nao;
    v.rs_in = 1;                                   // b (or d)
    v.rs_out = mir ? -s->nao2 : s->nao2;           // tau, or mirrored tau
    v.ks_in = nao;                                 // a (or c)
    const double2* src = G + (mir ? (long long)(ntau - 1) * s->nao2 : 0);
    GW_TRY_INTERNAL(slice(s, src, v, (long long)ntau * s->nao2, 0, 1 << 30, nk, ntau * nao, nao, mir ? s->gm : s->gf,
                          (long long)ntau * nao));
  }
  return GW_OK;
}

// V slices with rows (Q, i) over the orbital a, for nb pairs (pair b at element offset tab[b],
// or b * pair without a table)
int stage_vrow(MixedState* s, const double2* V, int nb, const long long* tab, const Planes& P) {
  const int nao = s->d.nao, naux = s->d.naux;
  ZView vr;
  vr.rs_in = nao;
  vr.ks_in = 1;
  return slice(s, V, vr, s->pair, 0, 1 << 30, nb, naux * nao, nao, P, (long long)naux * nao, 0, tab);
}

// V slices with rows (i, Q) over the orbital a: row i * naux + Q reads V[Q][i][a] (the Z operand
// of the fused path, whose output columns must run over Q)
int stage_vrowt(MixedState* s, const double2* V, int nb, const long long* tab, const Planes& P) {
  const int nao = s->d.nao, naux = s->d.naux;
  ZView vr;
  vr.rin = naux;
  vr.rs_in = s->nao2;
  vr.rs_out = nao;
  vr.ks_in = 1;
  return slice(s, V, vr, s->pair, 0, 1 << 30, nb, naux * nao, nao, P, (long long)naux * nao, 0, tab);
}

// V slices with rows (j, b) over Q': row j * nao + b reads V[Q'][b][j]
int stage_vcol(MixedState* s, const double2* V, int nb, const long long* tab, const Planes& P) {
  const int nao = s->d.nao, naux = s->d.naux;
  ZView vc;
  vc.rin = nao;
  vc.rs_in = nao;
  vc.rs_out = 1;
  vc.ks_in = s->nao2;
  return slice(s, V, vc, s->pair, 0, 1 << 30, nb, (int)s->nao2, naux, P, s->nao2, 0, tab);
}

// The V operand for a pair table: the per-context slices, or in per-q mode the staged slices
struct VOp {
  const Planes* P;
  int tab;
};
VOp v_op(const MixedState* s, int which, bool rows_iq = false) {
  if (!s->per_q) return {which == T_VCOL_KMQK ? &s->vcol : (rows_iq ? &s->vrowt : &s->vrow), which};
  if (which == T_VCOL_KMQK) return {&s->vcq, T_LOC_VC};
  return {which == T_VKPQK ? &s->vq[1] : &s->vq[0], T_LOC_V};
}

// Slice output into operand planes P (the consumer's planes, chunks of 4 so_cb)
void so_target(OzParams& p, const Planes& P, int cb, int ch_cb) {
  p.so = 1;
  p.so_dst = P.ptr;
  p.so_rows = P.rows;
  p.so_ksteps = P.Kpad / kStepK;
  p.so_cb = cb;
  p.so_ch_cb = ch_cb;
}

// out[t][k][Q][i][b] = sum_a V^{pair(k)}_ia(Q) G^{kg(k)}_ab(t) for t in [t0, t0+nt) (A and Z), or, with
// transposed, out[t][k][Q'][d][b] = sum_c V^{pair(k)}_bc(Q') G^{kg(k)}_cd(beta - t) (the B operand of P0).
// Both put the innermost output index b on the TMEM lanes, so a warp's stores are contiguous: the first
// as the GEMM rows (t, b) of G^T times columns (Q, i) of V, the second as rows (Q', b) of V times
// columns (t, d) of G.
int vg_gemm(MixedState* s, int pair_tab, int g_tab, const Planes& Gp, int q, int t0, int nt, bool transposed,
            double2* out) {
  const int nk = s->d.nk, nao = s->d.nao, naux = s->d.naux;
  const VOp vo = v_op(s, pair_tab);
  OzParams p;
  p.nbatch = nk;
  p.C = out;
  p.bc.bs_in = s->pair;
  p.status = s->status;
  p.ws = s->ws;
  p.out_df = 1;
  if (!transposed) {
    p.M = nt * nao;                       // (t, b)
    p.N = naux * nao;                     // (Q, i)
    p.a_tab = tab(s, g_tab, q);
    p.a_row0 = (long long)t0 * nao;
    p.b_tab = tab(s, vo.tab, q);
    p.vc.rin = nao;
    p.vc.rs_in = 1;
    p.vc.rs_out = (long long)nk * s->pair;
    p.vc.ks_in = nao;
    return launch_oz(Gp, *vo.P, p, SLOT_VG_MIXED, s->stream, s->d.tile_n);
  }
  p.M = naux * nao;                       // (Q', b)
  p.N = nt * nao;                         // (t, d)
  p.a_tab = tab(s, vo.tab, q);
  p.b_tab = tab(s, g_tab, q);
  p.b_row0 = (long long)t0 * nao;
  p.vc.rin = nao;
  p.vc.rs_in = 1;
  p.vc.rs_out = s->nao2;
  p.vc.kin = nao;
  p.vc.ks_in = nao;
  p.vc.ks_out = (long long)nk * s->pair;
  return launch_oz(*vo.P, Gp, p, SLOT_VG_MIXED, s->stream, s->d.tile_n);
}

// Fused path, P0 operands. The contraction index of P0 runs over (k, d, b) in chunks of 4 b x all
// d: element (k, d, b) at k-position (k (nao/4) + b/4) 4 nao + 4 d + b % 4, for both operands.
//   X^Q_{db}(k,t) = sum_a G^{k+q}_ab(t) V^{k,k+q}_da(Q): rows (t, b) of G^T, one Q per tile (columns d)
//   Y^{Q'}_{bd}(k,t) = sum_c V^{k+q,k}_bc(Q') G^k_cd(beta - t): rows (Q', b) of V, one t per tile (columns d)
// so that a chunk is 4 consecutive rows b of one tile by all its nao columns.
int p0_operands_fused(MixedState* s, int q, int t0, int nt, const Planes& xs, const Planes& ys) {
  const int nk = s->d.nk, nao = s->d.nao, naux = s->d.naux;
  {
    const VOp vo = v_op(s, T_VKKPQ);
    OzParams p;
    p.nbatch = nk;                        // k
    p.M = nt * nao;                       // (t, b)
    p.N = naux * nao;                     // (Q, d)
    p.nstride = nao;
    p.a_tab = tab(s, T_GKPQ, q);
    p.a_row0 = (long long)t0 * nao;
    p.b_tab = tab(s, vo.tab, q);
    so_target(p, xs, nao, nao / 4);
    p.so_xhalf = 1;
    p.so_mdiv = nao;                      // m = t nao + b
    p.so_ndiv = nao;                      // n = Q nao + d
    p.so_rm = naux;                       // row t naux + Q
    p.so_rn = 1;
    p.so_ch_bs_in = nao / 4;              // chunk k (nao/4) + b/4
    p.status = s->status;
    p.ws = s->ws;
    GW_TRY_INTERNAL(launch_oz(s->gf, *vo.P, p, SLOT_VG_MIXED, s->stream, 56));
  }
  const VOp vo = v_op(s, T_VKPQK);
  OzParams p;
  p.nbatch = nk;
  p.M = naux * nao;                       // (Q', b)
  p.N = nt * nao;                         // (t, d)
  p.nstride = nao;
  p.a_tab = tab(s, vo.tab, q);
  p.b_tab = tab(s, T_GK, q);
  p.b_row0 = (long long)t0 * nao;
  so_target(p, ys, nao, nao / 4);
  p.so_xhalf = 1;
  p.so_mdiv = nao;                        // m = Q' nao + b
  p.so_ndiv = nao;                        // n = t nao + d
  p.so_rm = 1;                            // row t naux + Q'
  p.so_rn = naux;
  p.so_ch_bs_in = nao / 4;
  p.status = s->status;
  p.ws = s->ws;
  return launch_oz(*vo.P, s->gm, p, SLOT_VG_MIXED, s->stream, 56);
}

int polarization_chunk(MixedState* s, const double2* G, double2* P0t, double spin, int q, int t0, int nt) {
  const int nk = s->d.nk, nao = s->d.nao, naux = s->d.naux, ntau = s->d.ntau;
  const Planes xs = view(s->xs_mem, (long long)nt * naux, s->Kc_p0, s->Kpad_p0, 2);
  const Planes ys = view(s->ys_mem, (long long)nt * naux, s->Kc_p0, s->Kpad_p0, 2);
  if (s->fused) {
    GW_TRY_INTERNAL(p0_operands_fused(s, q, t0, nt, xs, ys));
  } else {
    GW_TRY_INTERNAL(vg_gemm(s, T_VKKPQ, T_GKPQ, s->gf, q, t0, nt, false, s->x64));
    GW_TRY_INTERNAL(vg_gemm(s, T_VKPQK, T_GK, s->gm, q, t0, nt, true, s->y64));
    ZView v;                               // rows Q, k = (k, d, b)
    v.rs_in = s->nao2;
    v.kin = (int)s->nao2;
    v.ks_in = 1;
    v.ks_out = s->pair;
    GW_TRY_INTERNAL(slice(s, s->x64, v, (long long)nk * s->pair, 0, 1 << 30, nt, naux, nk * (int)s->nao2, xs, naux, 1));
    GW_TRY_INTERNAL(slice(s, s->y64, v, (long long)nk * s->pair, 0, 1 << 30, nt, naux, nk * (int)s->nao2, ys, naux, 1));
  }
  OzParams p;
  p.M = naux;
  p.N = naux;
  p.nbatch = nt;
  p.a_bs_in = naux;
  p.b_bs_in = naux;
  p.C = P0t + ((long long)q * ntau + t0) * s->naux2;
  p.bc.bs_in = s->naux2;
  p.vc.rs_in = naux;
  p.vc.ks_in = 1;
  p.alpha = -spin / nk;
  p.status = s->status;
  p.ws = s->ws;
  (void)nao;
  return launch_oz(xs, ys, p, SLOT_P0_TC, s->stream, s->d.tile_n);
}

int self_energy_chunk(MixedState* s, const double2* G, const double2* Pt, double2* Sig, int q, int t0, int nt) {
  const int nk = s->d.nk, nao = s->d.nao, naux = s->d.naux, ntau = s->d.ntau;
  {  // P~ planes: rows Q over Q'
    ZView v;
    v.rs_in = naux;
    v.ks_in = 1;
    GW_TRY_INTERNAL(slice(s, Pt + ((long long)q * ntau + t0) * s->naux2, v, s->naux2, 0, 1 << 30, nt, naux, naux,
                          s->ps, naux));
  }
  const Planes xs = view(s->xs_mem, (long long)nt * nk * nao, s->Kc_s, s->Kpad_s, 2);
  const Planes ys = view(s->ys_mem, (long long)nt * nk * nao, s->Kc_s, s->Kpad_s, 2);
  {  // R^Q_{bj}(k,t) = sum_Q' P~_QQ'(t) V^{k-q,k}_bj(Q')  -> y64[t][k][Q][j][b], computed as
     // rows (j, b) of V times columns Q of P~ so that the stores of a warp are contiguous
    OzParams p;
    p.M = (int)s->nao2;
    p.N = naux;
    p.nbatch = nt * nk;
    p.bin = nk;
    const VOp vo = v_op(s, T_VCOL_KMQK);
    p.a_tab = tab(s, vo.tab, q);            // per k
    p.b_bs_out = naux;                      // rows t * naux
    p.C = s->y64;
    p.bc.bs_in = s->pair;
    p.bc.bs_out = (long long)nk * s->pair;
    p.vc.rs_in = 1;
    p.vc.ks_in = s->nao2;
    p.status = s->status;
    p.ws = s->ws;
    p.out_df = 1;                           // double-float, sliced again for the Sigma contraction
    if (s->fused) {
      // straight into the Sigma B operand: rows (t, k, j), k-position of (Q, b)
      // ((Q/40) (nao/4) + b/4) 160 + 4 (Q % 40) + b % 4 (chunks of 4 b x 40 Q: one column half
      // of an 80-wide tile)
      so_target(p, ys, 40, nao / 4);
      p.so_mdiv = nao;                      // m = j nao + b
      p.so_rm = 1;                          // row (t nk + k) nao + j
      p.so_row_bs_in = nao;
      p.so_row_bs_out = (long long)nk * nao;
    }
    // the fused chunks are halves of an 80-wide tile
    GW_TRY_INTERNAL(launch_oz(*vo.P, s->ps, p, SLOT_R_TC, s->stream, s->fused ? 80 : s->d.tile_n));
  }
  if (s->fused) {
    // Z^Q_{ib}(k,t) = sum_a G^{k-q}_ab(t) V^{k,k-q}_ia(Q): rows (t, b) of G^T, columns (i, Q) of V,
    // straight into the Sigma A operand (rows (t, k, i), the k-positions of R)
    const VOp vo = v_op(s, T_VKKMQ, true);
    OzParams p;
    p.nbatch = nk;
    p.M = nt * nao;                         // (t, b)
    p.N = nao * naux;                       // (i, Q)
    p.a_tab = tab(s, T_GKMQ, q);
    p.a_row0 = (long long)t0 * nao;
    p.b_tab = tab(s, vo.tab, q);
    so_target(p, xs, 40, nao / 4);
    p.so_xhalf = 1;
    p.so_mdiv = nao;                        // m = t nao + b
    p.so_ndiv = naux;                       // n = i naux + Q
    p.so_rm = (long long)nk * nao;          // row (t nk + k) nao + i
    p.so_rn = 1;
    p.so_row_bs_in = nao;
    p.status = s->status;
    p.ws = s->ws;
    // 40-wide tiles: two accumulator sets, so the next tile's MMAs overlap this one's slice output
    GW_TRY_INTERNAL(launch_oz(s->gf, *vo.P, p, SLOT_VG_MIXED, s->stream, 40));
  } else {
    // Z^Q_{ib}(k,t) = sum_a V^{k,k-q}_ia(Q) G^{k-q}_ab(t) -> x64[t][k][Q][i][b]
    GW_TRY_INTERNAL(vg_gemm(s, T_VKKMQ, T_GKMQ, s->gf, q, t0, nt, false, s->x64));
    ZView vz;                               // rows i, k = (Q, b)
    vz.rs_in = nao;
    vz.kin = nao;
    vz.ks_out = s->nao2;
    vz.ks_in = 1;
    GW_TRY_INTERNAL(slice(s, s->x64, vz, s->pair, 0, 1 << 30, nt * nk, nao, naux * nao, xs, nao, 1));
    // R is stored [Q][j][b]: rows j, k = (Q, b), the same view as Z
    GW_TRY_INTERNAL(slice(s, s->y64, vz, s->pair, 0, 1 << 30, nt * nk, nao, naux * nao, ys, nao, 1));
  }
  OzParams p;                               // Sigma^k_ij(t) += -(1/N_k) sum_{Q,b} Z_{Q,i,b} R_{Q,b,j}
  // (t, k) problems of nao x nao are consecutive plane rows (t * nk + k) * nao; grp of them share one
  // block-diagonal tile, so one MMA of N = grp * nao does the work of grp narrow ones
  int bn = 80, grp = 1;
  oz_block_diag(nao, &bn, &grp);
  const int nprob = nt * nk;
  p.M = grp * nao;
  p.N = grp * nao;
  p.nbatch = (nprob + grp - 1) / grp;
  // group g = bo * nk + bi (bin = nk below) starts at plane row g * grp * nao
  p.a_bs_in = (long long)grp * nao;
  p.a_bs_out = (long long)nk * grp * nao;
  p.b_bs_in = (long long)grp * nao;
  p.b_bs_out = (long long)nk * grp * nao;
  p.dblock = grp > 1 ? nao : 0;
  p.dgroup = grp;
  p.dtotal = nprob;
  p.bin = nk;                               // output problem index -> (t, k) = (ob / nk, ob % nk)
  p.C = Sig + (long long)t0 * s->nao2;
  p.bc.bs_in = (long long)ntau * s->nao2;
  p.bc.bs_out = s->nao2;
  p.vc.rs_in = nao;
  p.vc.ks_in = 1;
  p.alpha = -1.0 / nk;
  p.accumulate = 1;
  p.status = s->status;
  p.ws = s->ws;
  return launch_oz(xs, ys, p, SLOT_SIGMA_MIXED, s->stream, bn);
}

}  // namespace

int mixed_create(MixedState** out, const MixedDims& d, cudaStream_t stream, int* status, size_t* bytes,
                 bool dry) {
  *out = nullptr;
  if (!dry && !encode_fn()) return fail(GW_ECUDA, "cuTensorMapEncodeTiled entry point not found");
  if (d.nao > 512 || d.naux > 4096) return fail(GW_EINVAL, "mixed: nao <= 512 and naux <= 4096 required");
  MixedState* s = new MixedState();
  s->dry = dry;
  s->d = d;
  s->stream = stream;
  s->status = status;
  s->nao2 = (long long)d.nao * d.nao;
  s->naux2 = (long long)d.naux * d.naux;
  s->pair = (long long)d.naux * s->nao2;
  const int nk = d.nk, nao = d.nao, naux = d.naux, ntau = d.ntau;
  chunking(nao, &s->Kc_vg, &s->Kpad_vg);
  chunking(nk * (int)s->nao2, &s->Kc_p0, &s->Kpad_p0);
  chunking(naux, &s->Kc_r, &s->Kpad_r);
  chunking(naux * nao, &s->Kc_s, &s->Kpad_s);
  // Fused path where the chunks fit producer tiles: 4 orbitals x nao (one 56-wide tile) for P0,
  // 4 orbitals x 40 Q (one half of an 80-wide tile) for Sigma
  s->fused = d.fuse && nao % 4 == 0 && nao <= 56 && naux % 40 == 0;
  if (s->fused) {
    s->Kc_p0 = 4 * nao;
    s->Kpad_p0 = nk * (int)s->nao2;
    s->Kc_s = 160;
    s->Kpad_s = naux * nao;
  }
  // tau batch: FP64 intermediates (unfused) plus operand planes per tau node
  const double per_t = (s->fused ? 0.0 : 2.0 * nk * (double)s->pair * 16.0) +
                       (8.0 + 8.0) * std::max((double)naux * s->Kpad_p0, (double)nk * nao * s->Kpad_s) * 2.0 +
                       (double)naux * s->Kpad_r * 8.0 * 2.0;
  s->nt = d.tau_chunk > 0 ? std::min(d.tau_chunk, ntau) : auto_tau_batch(d, per_t);
  int rc = GW_OK;
  do {
    // V slices for every pair when they take at most 24 GiB; else per q (4 nk pairs at a time)
    const double full_v = 16.0 * nk * nk * ((s->fused ? 2.0 : 1.0) * naux * nao * s->Kpad_vg +
                                            (double)s->nao2 * s->Kpad_r);
    s->per_q = d.v_slices == GW_V_PER_Q || (d.v_slices == GW_V_AUTO && full_v > 25769803776.0);
    const long long vpairs = s->per_q ? nk : (long long)nk * nk;
    if (s->per_q) {
      for (int i = 0; i < 2; ++i)
        if ((rc = alloc_planes(s, &s->vq[i], (long long)nk * naux * nao, s->Kc_vg, s->Kpad_vg, 2, bytes))) break;
      if (rc) break;
      if ((rc = alloc_planes(s, &s->vcq, (long long)nk * s->nao2, s->Kc_r, s->Kpad_r, 2, bytes))) break;
      if (d.v_packed && (rc = m_alloc(s, &s->vscratch, (size_t)nk * s->pair, bytes))) break;
    } else {
      // a packed V is unpacked for the slicing through a transient buffer of all pairs
      if (d.v_packed) *bytes += (size_t)nk * nk * s->pair * sizeof(double2);
      if ((rc = alloc_planes(s, &s->vrow, vpairs * naux * nao, s->Kc_vg, s->Kpad_vg, 2, bytes))) break;
      if (s->fused && (rc = alloc_planes(s, &s->vrowt, vpairs * naux * nao, s->Kc_vg, s->Kpad_vg, 2, bytes))) break;
      if ((rc = alloc_planes(s, &s->vcol, vpairs * s->nao2, s->Kc_r, s->Kpad_r, 2, bytes))) break;
    }
    if ((rc = alloc_planes(s, &s->gf, (long long)nk * ntau * nao, s->Kc_vg, s->Kpad_vg, 2, bytes))) break;
    if ((rc = alloc_planes(s, &s->gm, (long long)nk * ntau * nao, s->Kc_vg, s->Kpad_vg, 2, bytes))) break;
    if ((rc = alloc_planes(s, &s->ps, (long long)s->nt * naux, s->Kc_r, s->Kpad_r, 2, bytes))) break;
    // A and B operands (re and im slice groups) of the P0 and Sigma contractions
    const size_t op_elems = 4 * std::max((size_t)s->nt * naux * s->Kpad_p0, (size_t)s->nt * nk * nao * s->Kpad_s);
    if ((rc = m_alloc(s, &s->xs_mem, 2 * op_elems, bytes))) break;
    if ((rc = m_alloc(s, &s->ys_mem, 2 * op_elems, bytes))) break;
    if (!s->fused) {
      if ((rc = m_alloc(s, &s->x64, (size_t)s->nt * nk * s->pair, bytes))) break;
      if ((rc = m_alloc(s, &s->y64, (size_t)s->nt * nk * s->pair, bytes))) break;
    }
    {
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                    cudaSuccess) {
        cudaGetLastError();
        sms = 152;   // size-only build without a device: the GB300's SM count
      }
      // per-CTA running sums and chunk values of the GEMM epilogue
      if ((rc = m_alloc(s, &s->ws, 2 * (size_t)std::max(sms, 1) * kBM * kMaxBN, bytes))) break;
    }
    std::vector<long long> t((size_t)kTabs * nk * nk);
    const long long vrows = (long long)naux * nao;
    for (int q = 0; q < nk; ++q)
      for (int k = 0; k < nk; ++k) {
        const int kp = kshift3(d.nk3, k, q, +1), km = kshift3(d.nk3, k, q, -1);
        auto at = [&](int w) -> long long& { return t[((size_t)w * nk + q) * nk + k]; };
        at(T_VKKPQ) = ((long long)k * nk + kp) * vrows;
        at(T_VKPQK) = ((long long)kp * nk + k) * vrows;
        at(T_GKPQ) = (long long)kp * ntau * nao;
        at(T_GK) = (long long)k * ntau * nao;
        at(T_VKKMQ) = ((long long)k * nk + km) * vrows;
        at(T_GKMQ) = (long long)km * ntau * nao;
        at(T_VCOL_KMQK) = ((long long)km * nk + k) * s->nao2;
        at(T_LOC_V) = (long long)k * vrows;
        at(T_LOC_VC) = (long long)k * s->nao2;
        at(E_KKPQ) = ((long long)k * nk + kp) * s->pair;
        at(E_KPQK) = ((long long)kp * nk + k) * s->pair;
        at(E_KKMQ) = ((long long)k * nk + km) * s->pair;
        at(E_KMQK) = ((long long)km * nk + k) * s->pair;
      }
    if ((rc = m_alloc(s, &s->rowtabs, t.size(), bytes))) break;
    if (!dry) cudaMemcpy(s->rowtabs, t.data(), t.size() * sizeof(long long), cudaMemcpyHostToDevice);
  } while (false);
  if (rc != GW_OK || dry) {
    mixed_destroy(s);
    return rc;
  }
  *out = s;
  return GW_OK;
}

void mixed_guards(const MixedState* s, std::vector<unsigned char*>* out) {
  out->insert(out->end(), s->guards.begin(), s->guards.end());
}

void mixed_destroy(MixedState* s) {
  if (!s) return;
  for (void* p : s->allocs) cudaFree(p);
  delete s;
}

int mixed_set_coulomb(MixedState* s, const double2* V, const double2* Vp) {
  s->V = V;
  s->Vp = Vp;
  if (s->per_q) return GW_OK;               // sliced per q, when used
  const int nk = s->d.nk;
  double2* tmp = nullptr;
  if (Vp) {
    if (cudaMalloc(reinterpret_cast<void**>(&tmp), (size_t)nk * nk * s->pair * sizeof(double2)) != cudaSuccess) {
      cudaGetLastError();
      return fail(GW_ENOMEM, "mixed: no room to unpack V");
    }
    VPairs L;
    L.all = 1;
    int rc = unpack_v_fp64(Vp, nk, s->d.nao, s->pair, L, nk * nk, tmp, s->stream);
    if (rc == GW_OK) rc = stage_vrow(s, tmp, nk * nk, nullptr, s->vrow);
    if (rc == GW_OK && s->fused) rc = stage_vrowt(s, tmp, nk * nk, nullptr, s->vrowt);
    if (rc == GW_OK) rc = stage_vcol(s, tmp, nk * nk, nullptr, s->vcol);
    cudaStreamSynchronize(s->stream);
    cudaFree(tmp);
    return rc;
  }
  GW_TRY_INTERNAL(stage_vrow(s, V, nk * nk, nullptr, s->vrow));
  if (s->fused) GW_TRY_INTERNAL(stage_vrowt(s, V, nk * nk, nullptr, s->vrowt));
  return stage_vcol(s, V, nk * nk, nullptr, s->vcol);
}

namespace {

// Per-q V slices of one pair table: from V through the table, or from the blocks unpacked
// out of a packed V into the scratch. layout: 0 rows (Q, i) over a, 1 rows (j, b) over Q',
// 2 rows (i, Q) over a.
enum { VL_ROW = 0, VL_COL = 1, VL_ROWT = 2 };
int stage_q(MixedState* s, int table, int q, int layout, const Planes& P) {
  const int nk = s->d.nk;
  const double2* src = s->V;
  const long long* t = tab(s, table, q);
  if (s->Vp) {
    VPairs L;
    L.tab = t;
    GW_TRY_INTERNAL(unpack_v_fp64(s->Vp, nk, s->d.nao, s->pair, L, nk, s->vscratch, s->stream));
    src = s->vscratch;
    t = nullptr;
  }
  if (layout == VL_COL) return stage_vcol(s, src, nk, t, P);
  if (layout == VL_ROWT) return stage_vrowt(s, src, nk, t, P);
  return stage_vrow(s, src, nk, t, P);
}

}  // namespace

int mixed_wait_selftest(double limit_s, int* code, cudaStream_t st) {
  int* status = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&status), 2 * sizeof(int)) != cudaSuccess)
    return fail(GW_ENOMEM, "wait self-test: allocation failed");
  int h[2] = {0, 0};
  cudaMemsetAsync(status, 0, 2 * sizeof(int), st);
  wait_selftest_kernel<<<1, 32, 0, st>>>((uint64_t)(limit_s * 1e9), status);
  int rc = GW_OK;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h, status, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    rc = fail(GW_ECUDA, "wait self-test: launch or copy failed");
  cudaFree(status);
  if (rc != GW_OK) return rc;
  *code = h[1];
  if (h[0]) return fail(GW_ECUDA, "wait self-test: a phase that nothing completes was seen complete");
  return h[1] ? fail(GW_EDEVTIMEOUT, "a device-side wait gave up (code %d)", h[1]) : GW_OK;
}

namespace {

// (re)allocates a lazily sized plane buffer of at least elems bf16 values
int ensure_mem(MixedState* s, __nv_bfloat16** mem, size_t* have, size_t elems) {
  if (*have >= elems) return GW_OK;
  if (*mem) {
    cudaStreamSynchronize(s->stream);
    cudaFree(*mem);
    const size_t at = std::find(s->allocs.begin(), s->allocs.end(), (void*)*mem) - s->allocs.begin();
    s->allocs.erase(s->allocs.begin() + at);
    s->guards.erase(s->guards.begin() + at);
    *mem = nullptr;
    *have = 0;
  }
  size_t bytes = 0;
  GW_TRY_INTERNAL(m_alloc(s, mem, elems, &bytes));
  *have = elems;
  return GW_OK;
}

}  // namespace

int mixed_gf2_last(MixedState* s, const double2* Y, const double2* W, int nb, int nao, double2* part) {
  const int n2 = nao * nao;
  int Kc = 0, Kpad = 0;
  chunking(n2, &Kc, &Kpad);
  const long long rows = (long long)nb * n2;              // (t, q, i) for A, (t, q, j) for B
  const Planes shape = view(nullptr, rows, Kc, Kpad, 2);
  GW_TRY_INTERNAL(ensure_mem(s, &s->ol_mem, &s->ol_elems, 2 * shape.elems()));
  const Planes ys = view(s->ol_mem, rows, Kc, Kpad, 2);
  const Planes ws = view(s->ol_mem + shape.elems(), rows, Kc, Kpad, 2);
  const long long n3 = (long long)n2 * nao, n4 = (long long)n2 * n2;
  {  // rows r = (q, i) of Y[t][(i q)][(m l)]: element (r, k) at (i nao + q) n2 + k
    ZView v;
    v.rin = nao;
    v.rs_out = n2;
    v.rs_in = (long long)nao * n2;
    v.ks_in = 1;
    GW_TRY_INTERNAL(slice(s, Y, v, n4, 0, 1 << 30, nb, n2, n2, ys, n2));
  }
  {  // rows r = (q, j) of W[t][(q m)][(l j)], k = (m, l): element at q n3 + m n2 + l nao + j
    ZView v;
    v.rin = nao;
    v.rs_out = n3;
    v.rs_in = 1;
    v.kin = nao;
    v.ks_out = n2;
    v.ks_in = nao;
    GW_TRY_INTERNAL(slice(s, W, v, n4, 0, 1 << 30, nb, n2, n2, ws, n2));
  }
  OzParams p;                     // part[t][q][i][j] = sum_{(m l)} Y_q[i][(m l)] W_q[(m l)][j], batch (t, q)
  p.M = nao;
  p.N = nao;
  p.nbatch = nb * nao;
  p.a_bs_in = nao;
  p.b_bs_in = nao;
  p.C = part;
  p.vc.rs_in = nao;
  p.vc.ks_in = 1;
  p.bc.bs_in = n2;
  p.status = s->status;
  p.ws = s->ws;
  return launch_oz(ys, ws, p, SLOT_GF2_TC, s->stream);
}

int mixed_outer_q(MixedState* s, const double2* X, long long x_bs, const double2* Z, long long z_bs, int nb,
                  int n2, double2* out, long long out_bs) {
  const int naux = s->d.naux;
  const long long rows = (long long)nb * n2;
  const Planes shape = view(nullptr, rows, s->Kc_r, s->Kpad_r, 2);
  if (s->oq_rows < rows) {
    if (s->oq_mem) {
      cudaStreamSynchronize(s->stream);
      cudaFree(s->oq_mem);
      const size_t at = std::find(s->allocs.begin(), s->allocs.end(), (void*)s->oq_mem) - s->allocs.begin();
      s->allocs.erase(s->allocs.begin() + at);
      s->guards.erase(s->guards.begin() + at);
      s->oq_mem = nullptr;
      s->oq_rows = 0;
    }
    size_t bytes = 0;
    GW_TRY_INTERNAL(m_alloc(s, &s->oq_mem, 2 * shape.elems(), &bytes));
    s->oq_rows = rows;
  }
  const Planes xs = view(s->oq_mem, rows, s->Kc_r, s->Kpad_r, 2);
  const Planes zs = view(s->oq_mem + shape.elems(), z_bs ? rows : n2, s->Kc_r, s->Kpad_r, 2);
  ZView v;                                  // rows r = (a b), k = Q: element r + Q n2
  v.rs_in = 1;
  v.ks_in = n2;
  GW_TRY_INTERNAL(slice(s, X, v, x_bs, 0, 1 << 30, nb, n2, naux, xs, n2));
  GW_TRY_INTERNAL(slice(s, Z, v, z_bs, 0, 1 << 30, z_bs ? nb : 1, n2, naux, zs, n2));
  OzParams p;
  p.M = n2;
  p.N = n2;
  p.nbatch = nb;
  p.a_bs_in = n2;
  p.b_bs_in = z_bs ? n2 : 0;
  p.C = out;
  p.vc.rs_in = n2;
  p.vc.ks_in = 1;
  p.bc.bs_in = out_bs;
  p.status = s->status;
  p.ws = s->ws;
  return launch_oz(xs, zs, p, SLOT_GF2_TC, s->stream);
}

int mixed_polarization(MixedState* s, const double2* G, double2* P0t, double spin_factor, int q0, int q1) {
  GW_TRY_INTERNAL(slice_g(s, G));
  for (int q = q0; q < q1; ++q) {
    // canonical tau nodes only (the caller fills P0^q(beta - tau) = P0^{-q}(tau)^T); every node
    // when -q lies outside the range
    const int mq = s->d.mq[q];
    const int tend = (mq < q0 || mq >= q1) ? s->d.ntau : (mq < q ? 0 : (mq == q ? (s->d.ntau + 1) / 2 : s->d.ntau));
    if (tend > 0 && s->per_q) {
      GW_TRY_INTERNAL(stage_q(s, E_KKPQ, q, VL_ROW, s->vq[0]));
      GW_TRY_INTERNAL(stage_q(s, E_KPQK, q, VL_ROW, s->vq[1]));
    }
    // equal batches of at most nt nodes (no short last batch that would leave the GPU half idle)
    const int nb = (tend + s->nt - 1) / s->nt;
    for (int i = 0; i < nb; ++i) {
      const int t0 = (int)((long long)tend * i / nb), t1 = (int)((long long)tend * (i + 1) / nb);
      GW_TRY_INTERNAL(polarization_chunk(s, G, P0t, spin_factor, q, t0, t1 - t0));
    }
  }
  return GW_OK;
}

int mixed_self_energy(MixedState* s, const double2* G, const double2* Pt, double2* Sig, int q0, int q1) {
  if (cudaMemsetAsync(Sig, 0, (size_t)s->d.nk * s->d.ntau * s->nao2 * sizeof(double2), s->stream) != cudaSuccess)
    return fail(GW_ECUDA, "memset Sigma");
  GW_TRY_INTERNAL(slice_g(s, G));
  const int nb = (s->d.ntau + s->nt - 1) / s->nt;      // equal batches of at most nt nodes
  for (int q = q0; q < q1; ++q) {
    if (s->per_q) {
      GW_TRY_INTERNAL(stage_q(s, E_KKMQ, q, s->fused ? VL_ROWT : VL_ROW, s->vq[0]));
      GW_TRY_INTERNAL(stage_q(s, E_KMQK, q, VL_COL, s->vcq));
    }
    for (int i = 0; i < nb; ++i) {
      const int t0 = (int)((long long)s->d.ntau * i / nb), t1 = (int)((long long)s->d.ntau * (i + 1) / nb);
      GW_TRY_INTERNAL(self_energy_chunk(s, G, Pt, Sig, q, t0, t1 - t0));
    }
  }
  return GW_OK;
}

}  // namespace gwi
