// Chain applications of the absorption (Sec. 3.3) with FP64 emulated on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory): the
// precision option HT_PREC_EMU of ht_reduce_ex.
//
// A chain of transforms G_t (regular WY form, Sec. 2.4) is applied to lines
// (rows for a right application, columns for a left one): every line x takes
// x <- x G_t0 G_t0+1 ... in chain order.  Consecutive windows are grouped so
// that the union of their rows is at most 64 wide, and the product of a group's
// transforms, G (w x w, w <= 64), is formed once in FP64 by tc_prep_kernel.
// The sweep then computes the new line x G directly as one product of integers
// on the tensor cores (the slicing idea of Ozaki, Ogita, Oishi and Rump, 2012,
// in fixed point):
//
//  * x is put in fixed point against its own power-of-two bound over the
//    window, Y = round(x 2^(53-E)), |Y| < 2^53, written as 6 balanced base-2^9
//    digits (|d| <= 256); G is put in fixed point against one bound per group,
//    62 bits, 7 digits of the same weights (the transform is shared by every
//    line, so its rounding is kept below that of the lines).
//  * A digit is exact in FP16 and a product of two is at most 2^16, so a K = 64
//    product of one digit pair is at most 2^22 and four pairs of one level can
//    share an FP32 accumulator exactly (level L = a + b of the 1-based digit
//    indices; levels up to 8 are kept, 27 pairs in 10 accumulators).
//  * tcgen05.mma (M = 128 lines, N = 64 output columns, K = 16) accumulates
//    each group in tensor memory; every thread reads back its line's columns
//    (tcgen05.ld), converts them to integers, combines the levels in int64 and
//    writes the new line as FP64, all in integer arithmetic: the sweep issues
//    no FP64 instruction (GB300's FP64 rate is 1/64 of its integer rate).
//
// The error of a line is that of a rounding at 2^-53 relative to the line's
// bound: the normwise accuracy of an FP64 product.
//
// Launch: a persistent grid of CTAs of 512 threads (one per SM) takes work
// units from a counter: a unit is one stripe of 128 lines and a chunk of
// consecutive groups, units of one stripe in chunk order (a unit waits for
// the stripe's previous chunk), so that the grid does not round up to whole
// waves of stripes.  G's digits are staged per group into shared memory with
// a bulk copy (cp.async.bulk, completion on an mbarrier); the MMAs are issued
// by one thread in three commits (levels 2-5, 6-7, 8), the later ones
// overlapping the read-back of the earlier ones.  Every wait is bounded: on
// expiry the kernel raises HT_ERR_TIMEOUT, waits (bounded) for what it has in
// flight, frees its tensor memory and returns.
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "ht_common.cuh"

namespace {

constexpr int TM = 128;                 // lines per CTA (tensor-memory lanes)
constexpr int TW = 64;                  // largest window width (K and N of the product)
constexpr int TTHREADS = 512;           // 16 warps: four per lane quarter, 16 columns of a line each
constexpr int NDX = 6, NDG = 7;         // digits of a line / of G
constexpr int XS = TW + 1;              // leading dimension of the FP64 stripe (odd)
constexpr int XD_PLANE = TM * TW * 2;   // bytes of one digit plane of the lines (K-major core matrices)
constexpr int GD_PLANE = TW * TW * 2;   // bytes of one digit plane of G
constexpr int GD_BYTES = NDG * GD_PLANE;
constexpr int XF_BYTES = TM * XS * 8;
constexpr int OFF_XD = 0;
constexpr int OFF_GD = OFF_XD + NDX * XD_PLANE;
constexpr int OFF_XF = OFF_GD + GD_BYTES;
constexpr int OFF_MISC = OFF_XF + XF_BYTES;
constexpr int MISC_BYTES = 4096;        // barriers, tensor-memory address, line bounds, abort flag
constexpr int SMEM_BYTES = OFF_MISC + MISC_BYTES + 1024;  // + slack to align the base to 1024 bytes
static_assert(SMEM_BYTES <= 232448, "shared memory of one CTA");
constexpr int PREP_SMEM = (TW * TW + TW * 32) * 8;  // G and G(:, window) Vw
constexpr int TMEM_COLS = 512;
constexpr long TC_POLLS = 1L << 24;     // bounded mbarrier waits

// digit pairs (a, b) (0-based: a of the line, b of G), grouped per accumulator
// in level order; 10 groups, at most 4 pairs each, of one level each:
//   g0 L2: (0,0) | g1 L3: (0,1) (1,0) | g2 L4: (0,2) (1,1) (2,0)
//   g3 L5: (0,3) (1,2) (2,1) (3,0) | g4, g5 L6: (0,4) (1,3) (2,2) (3,1); (4,0)
//   g6, g7 L7: (0,5) (1,4) (2,3) (3,2); (4,1) (5,0)
//   g8, g9 L8: (0,6) (1,5) (2,4) (3,3); (4,2) (5,1)
constexpr int NGROUP = 10;

// ---------------------------------------------------------------------------
// Window geometry (that of the FP64 sweeps, ht_apply.cu) and the groups
// ---------------------------------------------------------------------------
__host__ __device__ inline void tc_win_geom(int mode, int p, int k, int t, int* off, int* width, int* limit) {
  int a, b;
  if (mode == 0) {
    ht_ql_window(p, k, t, &a, &b);
    *off = a; *width = b - a; *limit = b;
  } else if (mode == 1) {
    ht_qr_window(p, k, t, &a, &b);
    *off = a; *width = b - a; *limit = a;
  } else if (mode == 2) {
    const int nbr = ht_num_right_blocks(p, k);
    const int bb = nbr - 1 - t;
    int c0, c1, d0, d1;
    ht_right_block(p, k, bb - 1, &c0, &c1);
    ht_right_block(p, k, bb, &d0, &d1);
    *off = c0; *width = d1 - c0; *limit = d0;
  } else {
    const int nlb = ht_num_left_blocks(p, k);
    int r0, r1, e0, e1;
    ht_left_block(p, k, t, &r0, &r1);
    if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
    *off = r0; *width = e1 - r0; *limit = r1;
  }
}
__device__ inline void tc_win_refl(int mode, int p, int k, int t, int* kr) {
  if (mode == 0 || mode == 1) { *kr = k; return; }
  if (mode == 2) {
    const int nbr = ht_num_right_blocks(p, k);
    int d0, d1;
    ht_right_block(p, k, nbr - 1 - t, &d0, &d1);
    *kr = d1 - d0;
    return;
  }
  int r0, r1;
  ht_left_block(p, k, t, &r0, &r1);
  *kr = r1 - r0;
}

// ---------------------------------------------------------------------------
// Fixed point and digits (integer arithmetic on the bit pattern)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int expo(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return e ? e : 1;
}

// round(x 2^(53 + 9 XTRA - (emax - 1022))), emax >= expo(x); |result| < 2^(53 + 9 XTRA)
template <int XTRA>
__device__ __forceinline__ long long to_fixed(double x, int emax) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  long long m = bits & 0xFFFFFFFFFFFFFLL;
  int ee = 1;
  if (e) { m |= 1LL << 52; ee = e; }
  const int sh = emax - ee - 9 * XTRA;
  long long y;
  if (sh <= 0) y = m << (-sh);
  else if (sh >= 62) y = 0;
  else y = (m + (1LL << (sh - 1))) >> sh;
  return bits < 0 ? -y : y;
}

// ND balanced base-512 digits of y (|y| < 2^(9 ND - 1)) as FP16 bit patterns
// biased by 0x6600 (1536 + d): lower digits are bit fields of y + C (C = 256
// in every lower digit), the top digit is the rest.
template <int ND>
__device__ __forceinline__ void digit_bits(long long y, uint32_t h[ND]) {
  long long c = 0;
#pragma unroll
  for (int a = 1; a < ND; ++a) c += 256LL << (9 * (ND - 1 - a));
  const unsigned long long z = (unsigned long long)(y + c);
#pragma unroll
  for (int a = 1; a < ND; ++a) h[a] = 0x6500u + (uint32_t)((z >> (9 * (ND - 1 - a))) & 511u);
  h[0] = (uint32_t)(0x6600 + (int)((long long)z >> (9 * (ND - 1))));
}

// two biased FP16 patterns -> an FP16 pair of the digits (subtracting 1536 is exact)
__device__ __forceinline__ uint32_t unbias2(uint32_t lo, uint32_t hi) {
  union { uint32_t u; __half2 h; } b;
  b.u = lo | (hi << 16);
  b.h = __hsub2(b.h, __halves2half2(__ushort_as_half((unsigned short)0x6600), __ushort_as_half((unsigned short)0x6600)));
  return b.u;
}

// byte offset of element (row, k) of a K-major operand tile without swizzle,
// core matrices of 8 rows x 16 bytes: the row groups of one 8-column K chunk
// are contiguous (stride 128 bytes), so the tensor core reads along M without
// bank conflicts; K chunks are rows / 8 * 128 bytes apart
template <int ROWS>
__host__ __device__ __forceinline__ int kmajor_off(int row, int kcol) {
  return (kcol >> 3) * (ROWS * 16) + (row >> 3) * 128 + (row & 7) * 16 + (kcol & 7) * 2;
}

// exact integer from an FP32 accumulator that holds one (|c| <= 2^24)
__device__ __forceinline__ int f2i(uint32_t u) { return __float2int_rn(__uint_as_float(u)); }

// results below the normal range: the mantissa shifted into a subnormal (or
// zero), above it an infinity (neither the sweep's inputs nor G produce one)
__device__ __noinline__ unsigned long long scaled_tiny(unsigned long long sgn, unsigned long long mant, int be) {
  if (be > 2046) return sgn | (0x7ffull << 52);
  const int sh = 1 - be;
  if (sh > 53) return sgn;
  return sgn | ((mant + (1ull << (sh - 1))) >> sh);
}

// int64 -> double times 2^ex in integer arithmetic (round to nearest even):
// GB300 issues FP64 instructions at 1/64 of its integer rate
__device__ __forceinline__ double scaled_double(long long t, int ex) {
  if (t == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)t & 0x8000000000000000ull;
  unsigned long long a = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
  const int nb = 64 - __clzll((long long)a);
  unsigned long long mant;
  int e2 = nb - 1 + ex;  // exponent of the leading bit
  if (nb <= 53) {
    mant = a << (53 - nb);
  } else {
    const int sh = nb - 53;
    mant = a >> sh;
    const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;
    if (mant >> 53) { mant >>= 1; ++e2; }
  }
  const int be = e2 + 1023;
  if (be >= 1 && be <= 2046)
    return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  return __longlong_as_double((long long)scaled_tiny(sgn, mant, be));
}

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading byte offset (between
// K-adjacent core matrices), stride byte offset (between 8-row groups),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16, D = F32, A = B = F16, both K-major, N = 64, M = 128 (an MMA of
// this shape costs about what one of N = 32 does: the operand reads dominate)
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with parity `parity` to complete
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < TC_POLLS; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// 8-byte asynchronous copy global -> shared (no register round trip, all in flight together)
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}
// bounded wait until *f >= v (acquire); gives up when the error word is set
__device__ bool flag_wait(const int* f, int v, const int* err) {
  for (long it = 0; it < TC_POLLS; ++it) {
    int x;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(x) : "l"(f) : "memory");
    if (x >= v) return true;
    if (*(const volatile int*)err != 0) return false;
    __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t r[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Products of grouped window transforms and their digits: one CTA per group.
// Output per group m: the 7 digit planes of G (B operand of the product, N =
// output column c, K = input column r, K-major core matrices), the exponent
// field bounding G, and the table geo[m] = (offset, width, limit, -).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TTHREADS) tc_prep_kernel(const double* wy, long stride, int mode, int p, int k,
                                                           int g, int t0, int t1, uint16_t* dig, int* exps,
                                                           int4* geo) {
  extern __shared__ double psm[];
  double* G = psm;             // column-major, ld TW
  double* P = psm + TW * TW;   // G(:, window) Vw, ld TW, at most 32 columns
  __shared__ int sq[4];
  __shared__ int fmax;
  const int tid = threadIdx.x;
  const int ta = t0 + blockIdx.x * g, tb = min(t1, ta + g);
  if (tid == 0) {
    int o0 = 1 << 30, e0 = -1, lm = 0;
    for (int t = ta; t < tb; ++t) {
      int off, w, lim;
      tc_win_geom(mode, p, k, t, &off, &w, &lim);
      o0 = min(o0, off);
      e0 = max(e0, off + w);
      lm = (t == ta) ? lim : (mode == 1 ? min(lm, lim) : max(lm, lim));
    }
    sq[0] = o0; sq[1] = e0 - o0; sq[2] = lm;
    fmax = 1;
  }
  for (int e = tid; e < TW * TW; e += blockDim.x) G[e] = ((e % TW) == (e / TW)) ? 1.0 : 0.0;
  __syncthreads();
  const int o0 = sq[0], wu = sq[1];
  for (int t = ta; t < tb; ++t) {
    int off, w, lim, kr;
    tc_win_geom(mode, p, k, t, &off, &w, &lim);
    tc_win_refl(mode, p, k, t, &kr);
    const double* Vw = wy + (size_t)t * stride;
    const double* Ww = Vw + stride / 2;
    const int ro = off - o0;
    // P = G(:, ro:ro+w) Vw  (wu x kr)
    for (int e = tid; e < wu * kr; e += blockDim.x) {
      const int r = e % wu, q = e / wu;
      double s = 0.0;
      for (int c = 0; c < w; ++c) s += G[r + (ro + c) * TW] * Vw[c + (size_t)q * w];
      P[r + q * TW] = s;
    }
    __syncthreads();
    // G(:, ro:ro+w) -= P Ww^T
    for (int e = tid; e < wu * w; e += blockDim.x) {
      const int r = e % wu, c = e / wu;
      double s = G[r + (ro + c) * TW];
      for (int q = 0; q < kr; ++q) s -= P[r + q * TW] * Ww[c + (size_t)q * w];
      G[r + (ro + c) * TW] = s;
    }
    __syncthreads();
  }
  int em = 1;
  for (int e = tid; e < TW * TW; e += blockDim.x) em = max(em, expo(G[e]));
  atomicMax(&fmax, em);
  __syncthreads();
  const int F = fmax;
  // digits: element (r = K, c = N) of plane b at byte kmajor_off<TW>(c, r)
  uint16_t* out = dig + (size_t)blockIdx.x * (GD_BYTES / 2);
  for (int e = tid; e < TW * TW; e += blockDim.x) {
    const int r = e % TW, c = e / TW;
    const double v = (r < wu && c < wu) ? G[r + c * TW] : 0.0;
    uint32_t h[NDG];
    digit_bits<NDG>(to_fixed<1>(v, F), h);
    const int off = kmajor_off<TW>(c, r) >> 1;
#pragma unroll
    for (int b = 0; b < NDG; ++b) {
      union { uint16_t u; __half x; } cv;
      cv.x = __hsub(__ushort_as_half((unsigned short)h[b]), __ushort_as_half((unsigned short)0x6600));
      out[b * (GD_PLANE / 2) + off] = cv.u;
    }
  }
  if (tid == 0) {
    exps[blockIdx.x] = F;
    geo[blockIdx.x] = make_int4(sq[0], sq[1], sq[2], 0);
  }
}

struct TcJob {
  double* X;
  long ldx;
  int right, line0, nlines, origin, use_limit, limit_base, cta0;
};
struct TcBatch {
  TcJob job[HT_SWEEP_MAXJOBS];
  int njobs;
  int ngroups;           // groups of this launch
  const uint16_t* dig;   // GD_BYTES per group
  const int* exps;
  const int4* geo;
  int* err;
  // work units: (chunk c of wpc consecutive groups, line block gl), unit c nlb + gl
  int nlb, wpc, nunits;
  int* sched;            // [0] next unit, [1 + gl] chunks of line block gl done (zeroed per launch)
};

__device__ __forceinline__ bool tc_skip(const TcJob& jb, int lb, int lines, int lim) {
  if (!jb.use_limit) return false;
  return jb.right ? (lb >= jb.limit_base + lim) : (lb + lines <= jb.limit_base + lim);
}

// tensor-memory column of accumulator group gi (64 columns each): groups 0-7
// fill the 512 columns; groups 8-9 (level 8) reuse those of groups 0-1 once
// levels 2 and 3 have been read
__host__ __device__ constexpr uint32_t acc_col(int gi) { return gi < 8 ? 64u * gi : 64u * (gi - 8); }

// The pair table: a, b of pair i, and the first pair of group g (kGs(10) = 27).
__host__ __device__ constexpr int kPa(int i) {
  constexpr int t[27] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5, 0, 1, 2, 3, 4, 5};
  return t[i];
}
__host__ __device__ constexpr int kPb(int i) {
  constexpr int t[27] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0, 6, 5, 4, 3, 2, 1};
  return t[i];
}
__host__ __device__ constexpr int kGs(int i) {
  constexpr int t[11] = {0, 1, 3, 6, 10, 14, 15, 19, 21, 25, 27};
  return t[i];
}

// MMAs of accumulator groups [G0, G1) (N = 64), interleaved across the groups
// (slot s of every group, then slot s + 1) so that consecutive MMAs go to
// different accumulators; slot s of a group is its pair s / 4 at k-step s % 4.
// Fully unrolled: every descriptor is a base descriptor plus a constant (the
// start-address field takes byte offsets / 16 and does not overflow here).
template <int G0, int G1>
__device__ __forceinline__ void issue_groups(uint32_t tbase, uint64_t da, uint64_t db) {
#pragma unroll
  for (int s = 0; s < 16; ++s) {
#pragma unroll
    for (int gi = G0; gi < G1; ++gi) {
      const int pi = kGs(gi) + (s >> 2);
      if (pi < kGs(gi + 1)) {
        const int ks = s & 3;
        mma_f16(tbase + acc_col(gi), da + (uint64_t)((kPa(pi) * XD_PLANE + ks * 2 * (TM * 16)) >> 4),
                db + (uint64_t)((kPb(pi) * GD_PLANE + ks * 2 * (TW * 16)) >> 4), s > 0 ? 1u : 0u);
      }
    }
  }
}

__global__ void __launch_bounds__(TTHREADS, 1) tc_sweep_kernel(TcBatch b) {
  extern __shared__ __align__(1024) unsigned char tsm_raw[];
  unsigned char* tsm = (unsigned char*)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Xd = tsm + OFF_XD;
  unsigned char* Gd = tsm + OFF_GD;
  double* Xf = (double*)(tsm + OFF_XF);
  uint64_t* bars = (uint64_t*)(tsm + OFF_MISC);  // 0: G copy, 1-3: MMAs of levels 2-5, 6-7, 8, 4: free
  uint32_t* tslot = (uint32_t*)(bars + 8);
  int* Es = (int*)(bars + 16);                   // 4 x TM partial line bounds
  volatile int* abort_flag = (volatile int*)(Es + 4 * TM);
  volatile int* m2_issued = abort_flag + 1;      // the level-8 MMAs of the current group are in flight
  volatile int* unit_sl = abort_flag + 2;        // the unit this CTA works on

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quarter = warp & 3, cq = warp >> 2;
  const int li = 32 * quarter + lane;  // this thread's line (tensor-memory lane); cq: its column quarter
  const uint32_t bar_g = smem_u32(bars + 0), bar_m0 = smem_u32(bars + 1), bar_m1 = smem_u32(bars + 2),
                 bar_m2 = smem_u32(bars + 3), bar_free = smem_u32(bars + 4);

  if (tid == 0) {
    mbar_init(bar_g, 1);
    mbar_init(bar_m0, 1);
    mbar_init(bar_m1, 1);
    mbar_init(bar_m2, 1);
    mbar_init(bar_free, TTHREADS);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
    *m2_issued = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  uint32_t phase = 0;
  bool g_pending = false;  // a bulk copy of G digits is in flight
  bool m_pending = false;  // MMAs in flight (for the clean-up after a timeout)
  for (;;) {
  // ---- the next unit: line block gl, groups [tlo, thi) ----
  if (tid == 0) *unit_sl = atomicAdd(b.sched, 1);
  __syncthreads();
  const int u = *unit_sl;
  if (u >= b.nunits) break;
  const int cu = u / b.nlb, gl = u - cu * b.nlb;
  TcJob jb = b.job[0];
#pragma unroll
  for (int i = 1; i < HT_SWEEP_MAXJOBS; ++i)
    if (i < b.njobs && gl >= b.job[i].cta0) jb = b.job[i];
  const int lb = jb.line0 + (gl - jb.cta0) * TM;
  const int lines = min(TM, jb.line0 + jb.nlines - lb);  // >= 1: line blocks cover the jobs' lines
  double* X = jb.X;
  const long ldx = jb.ldx;
  const int tlo = cu * b.wpc, thi = min(b.ngroups, tlo + b.wpc);
  if (cu > 0 && tid == 0) {
    // the stripe's previous chunk (taken earlier by a resident CTA) must be written
    if (!flag_wait(b.sched + 1 + gl, cu, b.err)) { atomicCAS(b.err, 0, HT_ERR_TIMEOUT); *abort_flag = 1; }
  }
  __syncthreads();
  if (*abort_flag) break;
  // the first group this unit takes
  auto next_group = [&](int from) {
    for (int t = from; t < thi; ++t) {
      const int4 gq = b.geo[t];
      if (!tc_skip(jb, lb, lines, gq.z)) return t;
    }
    return thi;
  };
  int t = next_group(tlo);
  if (tid == 0 && t < thi) {
    mbar_expect_tx(bar_g, GD_BYTES);
    bulk_g2s(smem_u32(Gd), b.dig + (size_t)t * (GD_BYTES / 2), GD_BYTES, bar_g);
  }
  g_pending = t < thi;
  // Xf holds the stripe's columns by absolute index a in slot a mod 64 (a
  // window spans at most 64 consecutive columns): the columns that the next
  // window shares stay in shared memory, the others go to X straight from the
  // read-back, and the next window's new columns are loaded into the freed
  // slots while this window's products run
  auto load_cols = [&](int a0, int a1) {
    const int nc = a1 - a0;
    if (nc <= 0) return;
    if (jb.right) {
      for (int e = tid; e < TM * nc; e += TTHREADS) {
        const int l = e % TM, a = a0 + e / TM;
        double* d = Xf + l * XS + (a & (TW - 1));
        if (l < lines) cp_async8(d, X + (size_t)(lb + l) + (size_t)a * ldx);
        else *d = 0.0;
      }
    } else {
      for (int e = tid; e < TM * nc; e += TTHREADS) {
        const int a = a0 + e % nc, l = e / nc;
        double* d = Xf + l * XS + (a & (TW - 1));
        if (l < lines) cp_async8(d, X + (size_t)a + (size_t)(lb + l) * ldx);
        else *d = 0.0;
      }
    }
  };
  bool first = true;
  while (t < thi) {
    const int4 gq = b.geo[t];
    const int off = gq.x, w = gq.y;
    const int o0 = jb.origin + off;
    const int F = b.exps[t];
    const int tn = next_group(t + 1);
    int n0 = 0, n1 = 0;  // the next window's columns (none after the unit's last)
    if (tn < thi) {
      const int4 gn = b.geo[tn];
      n0 = jb.origin + gn.x;
      n1 = n0 + gn.y;
    }
    if (first) load_cols(o0, o0 + w);
    first = false;
    cp_async_wait_all();
    __syncthreads();
    // ---- per-line bound over the window, from the four quarters of the line ----
    const int c0 = 16 * cq;
    auto xval = [&](int c) { return c < w ? Xf[li * XS + ((o0 + c) & (TW - 1))] : 0.0; };
    {
      int em = 1;
#pragma unroll 8
      for (int c = 0; c < 16; ++c) em = max(em, expo(xval(c0 + c)));
      Es[cq * TM + li] = em;
    }
    __syncthreads();
    const int E = max(max(Es[li], Es[TM + li]), max(Es[2 * TM + li], Es[3 * TM + li]));
    // ---- digits of this thread's 16 columns -> the A operand planes ----
#pragma unroll 1
    for (int ch = 0; ch < 2; ++ch) {
      uint32_t hb[8][NDX];
#pragma unroll
      for (int i = 0; i < 8; ++i) digit_bits<NDX>(to_fixed<0>(xval(c0 + 8 * ch + i), E), hb[i]);
      const int boff = kmajor_off<TM>(li, c0 + 8 * ch);
#pragma unroll
      for (int a = 0; a < NDX; ++a) {
        uint4 v;
        v.x = unbias2(hb[0][a], hb[1][a]);
        v.y = unbias2(hb[2][a], hb[3][a]);
        v.z = unbias2(hb[4][a], hb[5][a]);
        v.w = unbias2(hb[6][a], hb[7][a]);
        *(uint4*)(Xd + a * XD_PLANE + boff) = v;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // ---- the next window's new columns into the slots of this one's leaving columns ----
    load_cols(n0, min(n1, o0));
    load_cols(max(n0, o0 + w), n1);
    // ---- MMAs: levels 2-5 (groups 0-3), then levels 6-7 (groups 4-7) ----
    // A: 128 lines, K chunks 2048 bytes apart; B: 64 output columns, K chunks 1024 apart
    const uint64_t da = sdesc(smem_u32(Xd), TM * 16, 128), db = sdesc(smem_u32(Gd), TW * 16, 128);
    if (tid == 0) {
      bool ok = mbar_wait(bar_g, phase);
      g_pending = !ok;
      if (!ok) { atomicCAS(b.err, 0, HT_ERR_TIMEOUT); *abort_flag = 1; }
      tc_fence_after();
      if (ok) {
        issue_groups<0, 4>(tbase, da, db);
        mma_commit(bar_m0);
        issue_groups<4, 8>(tbase, da, db);
        mma_commit(bar_m1);
        m_pending = true;
      }
    }
    __syncthreads();
    if (*abort_flag) break;
    // ---- read back: this thread's 16 output columns [16 cq, 16 cq + 16) ----
    const int ex = E + F - 2099;  // new x = tot 2^ex
    bool ok = mbar_wait(bar_m0, phase);
    if (ok) {
      tc_fence_after();
      long long tot[16], t78[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) { tot[i] = 0; t78[i] = 0; }
      const uint32_t lanebase = tbase + ((uint32_t)(32 * quarter) << 16) + 16u * cq;
#pragma unroll 1
      for (int L = 2; L <= 8 && ok; ++L) {
        const int ga = (L <= 5) ? L - 2 : 4 + 2 * (L - 6), gb = (L <= 5) ? ga + 1 : ga + 2;
        if (L == 6 || L == 8) {
          ok = mbar_wait(L == 6 ? bar_m1 : bar_m2, phase);
          if (!ok) break;
          tc_fence_after();
        }
        // the level's one or two accumulators, both loads in flight before the wait
        int sl[16];
        {
          uint32_t r[16], r2[16];
          tmem_ld16(lanebase + acc_col(ga), r);
          if (gb - ga > 1) tmem_ld16(lanebase + acc_col(ga + 1), r2);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i) sl[i] = f2i(r[i]);
          if (gb - ga > 1) {
#pragma unroll
            for (int i = 0; i < 16; ++i) sl[i] += f2i(r2[i]);
          }
        }
        if (L <= 6) {
          const int sh = 57 - 9 * L;
#pragma unroll
          for (int i = 0; i < 16; ++i) tot[i] += (long long)sl[i] << sh;
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) t78[i] = t78[i] * 512 + sl[i];
        }
        if (L == 3) {
          // levels 2-3 (groups 0-1) read: level 8 (groups 8-9) may take their columns
          tc_fence_before();
          mbar_arrive(bar_free);
          if (tid == 0) {
            bool fok = mbar_wait(bar_free, phase);
            if (!fok) { atomicCAS(b.err, 0, HT_ERR_TIMEOUT); *abort_flag = 1; }
            tc_fence_after();
            if (fok) {
              issue_groups<8, NGROUP>(tbase, da, db);
              mma_commit(bar_m2);
              *m2_issued = 1;
            }
          }
        }
      }
      if (ok) {
        // levels 7 and 8 rounded once: t78 = S7 2^9 + S8, weight 2^-15
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          tot[i] += (t78[i] + (1LL << 14)) >> 15;
          const int c = 16 * cq + i, a = o0 + c;
          if (c >= w) continue;
          const double v = scaled_double(tot[i], ex);
          if (a >= n0 && a < n1) Xf[li * XS + (a & (TW - 1))] = v;  // shared with the next window
          else if (li < lines)
            X[jb.right ? (size_t)(lb + li) + (size_t)a * ldx : (size_t)a + (size_t)(lb + li) * ldx] = v;
        }
      }
    }
    if (!ok) { atomicCAS(b.err, 0, HT_ERR_TIMEOUT); *abort_flag = 1; }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag) break;
    m_pending = false;
    g_pending = false;
    if (tid == 0) *m2_issued = 0;
    // ---- prefetch the next group's digits (all MMAs of this one are done) ----
    if (tid == 0 && tn < thi) {
      mbar_expect_tx(bar_g, GD_BYTES);
      bulk_g2s(smem_u32(Gd), b.dig + (size_t)tn * (GD_BYTES / 2), GD_BYTES, bar_g);
    }
    g_pending = tn < thi;
    phase ^= 1u;
    t = tn;
  }
  if (*abort_flag) break;
  // ---- the unit's lines are written: release its chunk to the next one ----
  if (tid == 0) {
    __threadfence();
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(b.sched + 1 + gl), "r"(cu + 1) : "memory");
  }
  }
  // ---- clean-up: after a timeout, wait (bounded) for what is in flight ----
  cp_async_wait_all();
  if (*abort_flag && tid == 0) {
    if (g_pending) mbar_wait(bar_g, phase);
    if (m_pending) {
      mbar_wait(bar_m0, phase);
      mbar_wait(bar_m1, phase);
    }
    if (*m2_issued) mbar_wait(bar_m2, phase);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TMEM_COLS));
}

cudaError_t tc_attr() {
  static std::mutex mu;
  static unsigned long long done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1ull) return cudaSuccess;
  e = cudaFuncSetAttribute(tc_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tc_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, PREP_SMEM);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

int tc_sm_count() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 0;
  if (sms[dev] == 0 && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    sms[dev] = 0;
    return 0;
  }
  return sms[dev];
}

}  // namespace

// Groups per work unit for nlb stripes of ng groups on `sms` resident CTAs:
// a stripe's units run one after another, so the sweep takes at least ng
// group times, and ceil(nlb nc / sms) rounds of ng / nc group times with nc
// chunks; the fewest chunks (of at least 4 groups) that come within 2% of the
// best bound.
static int tc_chunk(int nlb, int ng, int sms) {
  auto cost = [&](int nc) {
    const int wpc = (ng + nc - 1) / nc;
    const int ncr = (ng + wpc - 1) / wpc;
    const double rounds = (double)(((long)nlb * ncr + sms - 1) / sms);
    return std::max((double)ng, rounds * wpc);
  };
  const int ncmax = std::max(1, std::min(64, ng / 4));
  double best = cost(1);
  for (int nc = 2; nc <= ncmax; ++nc) best = std::min(best, cost(nc));
  for (int nc = 1; nc <= ncmax; ++nc)
    if (cost(nc) <= 1.02 * best) return (ng + nc - 1) / nc;
  return ng;
}

// windows per group: the union of g consecutive windows of a chain with k
// reflectors spans at most (g + 1) k <= 64 rows
int ht_tc_group(int k) { return std::max(1, TW / std::max(k, 1) - 1); }
size_t ht_tc_group_bytes() { return GD_BYTES; }

cudaError_t ht_tc_sweep_multi(cudaStream_t st, const HtSweepJob* jobs, int njobs, const double* wy, long stride,
                              int mode, int p, int k, int t0, int t1, void* dig, int* exps, void* geo, int cap,
                              int* sched, int* err, int max_ctas) {
  if (njobs < 1 || njobs > HT_SWEEP_MAXJOBS) return cudaErrorInvalidValue;
  if (t1 <= t0) return cudaSuccess;
  if (k < 1 || 2 * k > TW) return cudaErrorNotSupported;
  cudaError_t e = tc_attr();
  if (e != cudaSuccess) return e;
  TcBatch bt{};
  int ctas = 0, nj = 0;
  for (int i = 0; i < njobs; ++i) {
    if (jobs[i].nlines <= 0) continue;
    TcJob& d = bt.job[nj++];
    d.X = jobs[i].X; d.ldx = jobs[i].ldx; d.right = jobs[i].right; d.line0 = jobs[i].line0;
    d.nlines = jobs[i].nlines; d.origin = jobs[i].origin; d.use_limit = jobs[i].use_limit;
    d.limit_base = jobs[i].limit_base; d.cta0 = ctas;
    ctas += (jobs[i].nlines + TM - 1) / TM;
  }
  if (nj == 0) return cudaSuccess;
  bt.njobs = nj;
  bt.dig = (const uint16_t*)dig;
  bt.exps = exps;
  bt.geo = (const int4*)geo;
  bt.err = err;
  bt.nlb = ctas;
  bt.sched = sched;
  int sms = tc_sm_count();
  if (sms <= 0) return cudaErrorUnknown;
  if (max_ctas > 0) sms = std::min(sms, max_ctas);
  const int g = ht_tc_group(k);
  const int ng = (t1 - t0 + g - 1) / g;
  for (int m0 = 0; m0 < ng; m0 += cap) {
    const int mc = std::min(cap, ng - m0);
    const int ta = t0 + m0 * g, tb = std::min(t1, ta + mc * g);
    tc_prep_kernel<<<mc, TTHREADS, PREP_SMEM, st>>>(wy, stride, mode, p, k, g, ta, tb, (uint16_t*)dig, exps, (int4*)geo);
    bt.ngroups = mc;
    bt.wpc = tc_chunk(ctas, mc, sms);
    bt.nunits = ctas * ((mc + bt.wpc - 1) / bt.wpc);
    e = cudaMemsetAsync(sched, 0, (size_t)(1 + ctas) * sizeof(int), st);
    if (e != cudaSuccess) return e;
    tc_sweep_kernel<<<std::min(bt.nunits, sms), TTHREADS, SMEM_BYTES, st>>>(bt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
