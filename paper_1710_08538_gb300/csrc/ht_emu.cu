// Chain applications of the absorption (Sec. 3.3) with FP64 emulated on the
// tensor cores: the precision option HT_PREC_EMU of ht_reduce_ex.
//
// The operation is the one of the FP64 sweeps (ht_apply.cu): for each window
// t of a chain, a stripe of lines of X (rows for a right application, columns
// for a left one; "lines" below) is updated as
//     X_s <- X_s - (X_s Vw) Ww^T          (X_s: lines x w, Vw, Ww: w x kr).
// Both products run as sums of exact integer products on FP16 tensor cores
// (the slicing idea of Ozaki, Ogita, Oishi and Rump, in fixed point):
//
//  * Each line of X_s is put in fixed point against its own power-of-two
//    bound, Y = round(x 2^(53-E)) with |x| < 2^E over the window, so |Y| < 2^53,
//    written as EA = 6 balanced base-2^9 digits, x = 2^E sum_a D_a 2^(1-9a),
//    |D_a| <= 256.  Vw and Ww are put in fixed point against one bound per
//    window with 62 bits, EB = 7 digits of the same weights.  The extra digit
//    matters: Vw and Ww are shared by every line, so their rounding is an
//    error of the transform itself (a departure from orthogonality that adds up
//    over the windows in Q and Z), while the rounding of X_s differs per line.
//  * Digits are exact in FP16, a product of two is at most 2^16, and a sum of
//    K products at most K 2^16, so with FP32 accumulation a K = 64 product of
//    one digit pair is exact, and up to 256 / K digit pairs can share one
//    accumulator (checked on GB300: sums of such products are exact to 2^24).
//  * X_s Vw = sum over levels L = a + b <= EA + 2 of 2^(-9L) S_L; every level
//    sum S_L is converted to an integer and added, shifted, into an int64
//    result.  The levels left out are 2^-9 (and less) below the last one
//    kept: keeping L <= EA + 1 only made the error of a window update about
//    7x that of FP64, with L <= EA + 2 it is within 2x (the rounding of X_s
//    to its line's fixed point).
//  * The product P = X_s Vw is re-normalised per line (its own bound), sliced
//    the same way and multiplied by Ww^T; the update X_s - P Ww^T is formed in
//    FP64 from the int64 result.
//
// The error of each product is that of a rounding at 2^-53 relative to the
// line's bound, the normwise accuracy of an FP64 product.  Digits of Vw and Ww
// are formed once per window by emu_prep_kernel and staged into shared
// memory by every CTA; digits of X_s and P are formed on the fly.
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "ht_common.cuh"

namespace {

constexpr int EA = 6;      // digits of X_s and P (53-bit fixed point)
constexpr int EB = 7;      // digits of Vw and Ww (62-bit fixed point)
constexpr int ER = 32;     // lines per CTA
constexpr int ETH = 256;   // threads per CTA (8 warps)

// ---------------------------------------------------------------------------
// Window geometry (the same as the FP64 sweeps; see ht_apply.cu)
// ---------------------------------------------------------------------------
// mode EMU_MERGED: windows of a merged chain, geometry from the table geo
// (offset, width, reflectors, limit) written by emu_merge_kernel.
constexpr int EMU_MERGED = 4;
__device__ __forceinline__ void emu_win_geom(int mode, int p, int k, int t, int* off, int* width, int* nrefl,
                                             int* limit, const int4* geo = nullptr) {
  int a, b;
  if (mode == EMU_MERGED) {
    const int4 g = geo[t];
    *off = g.x; *width = g.y; *nrefl = g.z; *limit = g.w;
  } else if (mode == 0) {
    ht_ql_window(p, k, t, &a, &b);
    *off = a; *width = b - a; *nrefl = k; *limit = b;
  } else if (mode == 1) {
    ht_qr_window(p, k, t, &a, &b);
    *off = a; *width = b - a; *nrefl = k; *limit = a;
  } else if (mode == 2) {
    const int nbr = ht_num_right_blocks(p, k);
    const int bb = nbr - 1 - t;
    int c0, c1, d0, d1;
    ht_right_block(p, k, bb - 1, &c0, &c1);
    ht_right_block(p, k, bb, &d0, &d1);
    *off = c0; *width = d1 - c0; *nrefl = d1 - d0; *limit = d0;
  } else {
    const int nlb = ht_num_left_blocks(p, k);
    int r0, r1, e0, e1;
    ht_left_block(p, k, t, &r0, &r1);
    if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
    *off = r0; *width = e1 - r0; *nrefl = r1 - r0; *limit = r1;
  }
}

// ---------------------------------------------------------------------------
// Fixed point and digits
// ---------------------------------------------------------------------------
// biased exponent field of x, 1 for zeros and subnormals: |x| < 2^(expo - 1022)
__device__ __forceinline__ int expo(double x) {
  const int e = (int)((__double_as_longlong(x) >> 52) & 0x7ff);
  return e ? e : 1;
}

// x in fixed point against the bound 2^E, E = emax - 1022 (emax >= expo(x)):
// round(x 2^(53 + 9 X - E)) for X extra digits, computed on the bit pattern;
// |result| < 2^(53 + 9 X).
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

// ND balanced base-512 digits, d[0] most significant: y = sum_a d[a] 2^(9(ND-1-a));
// |d[0]| <= 256 for |y| < 2^(9 ND - 1)
template <int ND>
__device__ __forceinline__ void digits9(long long y, int d[ND]) {
#pragma unroll
  for (int a = ND - 1; a >= 1; --a) {
    int v = (int)(y & 511);
    v -= (v & 256) << 1;  // [256, 511] -> [-256, -1]
    d[a] = v;
    y = (y - v) >> 9;
  }
  d[0] = (int)y;
}

// two digits (|d| <= 256) as an FP16 pair: 1536 + d is an FP16 with bits
// 0x6600 + d; subtracting 1536 is exact.
__device__ __forceinline__ uint32_t pack2(int lo, int hi) {
  union { uint32_t u; __half2 h; } b;
  b.u = (uint32_t)(0x6600 + lo) | ((uint32_t)(0x6600 + hi) << 16);
  b.h = __hsub2(b.h, __halves2half2(__ushort_as_half((unsigned short)0x6600), __ushort_as_half((unsigned short)0x6600)));
  return b.u;
}

__device__ __forceinline__ void mma16816(float c[4], const uint4& a, const uint2& b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y));
}

// tot += round(c * 2^sh) for the four accumulator entries; c holds exact integers
__device__ __forceinline__ void flush(long long tot[4], float c[4], int sh) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const long long v = (long long)__float2int_rn(c[i]);
    tot[i] += (sh >= 0) ? v * (1LL << sh) : ((v + (1LL << (-sh - 1))) >> (-sh));
    c[i] = 0.f;
  }
}

constexpr int ELMAX = EA + 2;  // highest digit level kept

// One 16 x 8 output tile of sum_{a+b <= ELMAX} 2^(57 - 9(a+b)) A_a B_b (A: EA
// digits, B: EB digits) with K = 16 KS.  A: per-lane pointer to the fragment
// of digit 1, k-step 0 (digit stride adig, k-step stride 32); B: likewise
// (digit stride bdig, k-step stride bks).  Levels share an FP32 accumulator
// for at most 256 / K pairs.
template <int KS>
__device__ __forceinline__ void emu_tile(long long tot[4], const uint4* A, int adig, const uint2* B, int bdig, int bks) {
  constexpr int PPA = (256 / (16 * KS)) > 0 ? 256 / (16 * KS) : 1;
#pragma unroll
  for (int i = 0; i < 4; ++i) tot[i] = 0;
#pragma unroll
  for (int L = 2; L <= ELMAX; ++L) {
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    int cnt = 0;
#pragma unroll
    for (int a = 1; a <= EA; ++a) {
      const int b = L - a;
      if (b < 1 || b > EB) continue;
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) mma16816(c, A[(a - 1) * adig + ks * 32], B[(b - 1) * bdig + ks * bks]);
      if (++cnt == PPA) {
        flush(tot, c, 57 - 9 * L);
        cnt = 0;
      }
    }
    if (cnt) flush(tot, c, 57 - 9 * L);
  }
}

// 2^e as a double: one factor in the normal range, two below it (a product
// that underflows to a subnormal or zero), 0 under 2^-2044 and infinity above
// 2^1023 (neither occurs for finite input: the exponents are bounds of FP64
// values).
__device__ __forceinline__ double pow2i(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  if (e > 1023) return __longlong_as_double(0x7ffLL << 52);
  if (e < -2044) return 0.0;
  return __longlong_as_double(1LL << 52) * __longlong_as_double((long long)(e + 1022 + 1023) << 52);
}

// ---------------------------------------------------------------------------
// Digits of Vw and Ww, one CTA per window.  Layout per window (uint2 units):
//   V: [EB][KS1][NT1][32]  B fragments of X_s Vw   (K = window columns, N = reflectors)
//   W: [EB][KS2][NT2][32]  B fragments of P Ww^T   (K = reflectors, N = window columns)
// with KS1 = 2 KPAD / 16, NT1 = KPAD / 8, KS2 = KPAD / 16, NT2 = 2 KPAD / 8.
// exps[2 t'] / [2 t' + 1]: exponent fields bounding Vw / Ww of window t0 + t'.
// ---------------------------------------------------------------------------
template <int KPAD>
struct EmuDims {
  static constexpr int KS1 = 2 * KPAD / 16, NT1 = KPAD / 8, KS2 = KPAD / 16, NT2 = 2 * KPAD / 8;
  static constexpr int VU = EB * KS1 * NT1 * 32;  // uint2 units of V digits
  static constexpr int WU = EB * KS2 * NT2 * 32;
  static constexpr int WIN = VU + WU;              // uint2 units per window
};

template <int KPAD>
__global__ void __launch_bounds__(ETH) emu_prep_kernel(const double* wy, long stride, int mode, int p, int k, int t0,
                                                       uint2* dig, int* exps, const int4* geo) {
  using D = EmuDims<KPAD>;
  __shared__ int fmax[2];
  const int t = t0 + blockIdx.x;
  int off, w, kr, lim;
  emu_win_geom(mode, p, k, t, &off, &w, &kr, &lim, geo);
  const double* Vw = wy + (size_t)t * stride;
  const double* Ww = Vw + stride / 2;
  if (threadIdx.x < 2) fmax[threadIdx.x] = 1;
  __syncthreads();
  int ev = 1, ew = 1;
  for (int e = threadIdx.x; e < w * kr; e += blockDim.x) {
    ev = max(ev, expo(Vw[e]));
    ew = max(ew, expo(Ww[e]));
  }
  atomicMax(&fmax[0], ev);
  atomicMax(&fmax[1], ew);
  __syncthreads();
  const int fv = fmax[0], fw = fmax[1];
  uint2* out = dig + (size_t)blockIdx.x * D::WIN;
  // V: element (k = window column, n = reflector)
  for (int u = threadIdx.x; u < D::KS1 * D::NT1 * 32; u += blockDim.x) {
    const int lane = u & 31, n = (u >> 5) % D::NT1, ks = (u >> 5) / D::NT1;
    const int g = lane >> 2, tt = lane & 3, q = n * 8 + g;
    int d[4][EB];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int kk = ks * 16 + 2 * tt + (i & 1) + 8 * (i >> 1);
      const double v = (kk < w && q < kr) ? Vw[kk + (size_t)q * w] : 0.0;
      digits9<EB>(to_fixed<EB - EA>(v, fv), d[i]);
    }
#pragma unroll
    for (int a = 0; a < EB; ++a)
      out[((a * D::KS1 + ks) * D::NT1 + n) * 32 + lane] = make_uint2(pack2(d[0][a], d[1][a]), pack2(d[2][a], d[3][a]));
  }
  // W^T: element (k = reflector q, n = window column c) = Ww(c, q)
  uint2* outw = out + D::VU;
  for (int u = threadIdx.x; u < D::KS2 * D::NT2 * 32; u += blockDim.x) {
    const int lane = u & 31, n = (u >> 5) % D::NT2, ks = (u >> 5) / D::NT2;
    const int g = lane >> 2, tt = lane & 3, c = n * 8 + g;
    int d[4][EB];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = ks * 16 + 2 * tt + (i & 1) + 8 * (i >> 1);
      const double v = (c < w && q < kr) ? Ww[c + (size_t)q * w] : 0.0;
      digits9<EB>(to_fixed<EB - EA>(v, fw), d[i]);
    }
#pragma unroll
    for (int a = 0; a < EB; ++a)
      outw[((a * D::KS2 + ks) * D::NT2 + n) * 32 + lane] = make_uint2(pack2(d[0][a], d[1][a]), pack2(d[2][a], d[3][a]));
  }
  if (threadIdx.x == 0) {
    exps[2 * blockIdx.x] = fv;
    exps[2 * blockIdx.x + 1] = fw;
  }
}

}  // namespace

namespace {

struct EmuJob {
  double* X;
  long ldx;
  int right, line0, nlines, origin, use_limit, limit_base, cta0;
};

struct EmuBatch {
  EmuJob job[HT_SWEEP_MAXJOBS];
  int njobs;
  int mode, p, k, t0, t1;
  const uint2* dig;  // digits of windows t0 .. t1-1
  const int* exps;
  const int4* geo;   // window table (mode EMU_MERGED)
};

template <int KPAD>
struct EmuSmem {
  static constexpr int XS = 2 * KPAD + 1;  // odd leading dimension of the FP64 stripe (per line)
  static constexpr size_t XF = (size_t)ER * XS * sizeof(double);
  static constexpr size_t XD = (size_t)EA * 2 * EmuDims<KPAD>::KS1 * 32 * sizeof(uint4);  // X digits; later P
  static constexpr int PLD = KPAD + 1;  // odd leading dimension of the int64 P buffer (no bank conflicts)
  static constexpr size_t PF = (size_t)ER * PLD * sizeof(long long);
  static constexpr size_t PD = (size_t)EA * 2 * EmuDims<KPAD>::KS2 * 32 * sizeof(uint4);
  static constexpr size_t VW = (size_t)EmuDims<KPAD>::WIN * sizeof(uint2);
  static constexpr size_t BYTES = XF + XD + VW + 2 * ER * sizeof(int);
  static_assert(PF + PD <= XD, "P buffers must fit in the X digit area");
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}

template <int KPAD>
__global__ void __launch_bounds__(ETH) emu_sweep_kernel(EmuBatch b) {
  using D = EmuDims<KPAD>;
  using M = EmuSmem<KPAD>;
  constexpr int XS = M::XS, KS1 = D::KS1, NT1 = D::NT1, KS2 = D::KS2, NT2 = D::NT2;
  extern __shared__ __align__(16) unsigned char esm[];
  double* Xf = (double*)esm;
  uint4* Xd = (uint4*)(esm + M::XF);
  long long* Pf = (long long*)(esm + M::XF);  // aliases Xd once X_s Vw is done
  uint4* Pd = (uint4*)((unsigned char*)Xd + M::PF);
  uint2* Vd = (uint2*)(esm + M::XF + M::XD);
  uint2* Wd = Vd + D::VU;
  int* Es = (int*)(esm + M::XF + M::XD + M::VW);
  int* Bs = Es + ER;

  EmuJob jb = b.job[0];
#pragma unroll
  for (int i = 1; i < HT_SWEEP_MAXJOBS; ++i)
    if (i < b.njobs && (int)blockIdx.x >= b.job[i].cta0) jb = b.job[i];
  const int stripe = (int)blockIdx.x - jb.cta0;
  const int lb = jb.line0 + stripe * ER;
  const int lines = min(ER, jb.line0 + jb.nlines - lb);
  if (lines <= 0) return;
  const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
  const int g = lane >> 2, tt = lane & 3;
  double* X = jb.X;
  const long ldx = jb.ldx;

  for (int t = b.t0; t < b.t1; ++t) {
    int off, w, kr, lim;
    emu_win_geom(b.mode, b.p, b.k, t, &off, &w, &kr, &lim, b.geo);
    if (jb.right) {
      if (jb.use_limit && lb >= jb.limit_base + lim) continue;
    } else {
      if (jb.use_limit && lb + lines <= jb.limit_base + lim) continue;
    }
    const int o0 = jb.origin + off;
    // stage the window's digits of Vw, Ww
    {
      const uint4* src = (const uint4*)(b.dig + (size_t)(t - b.t0) * D::WIN);
      uint4* dst = (uint4*)Vd;
      for (int e = tid; e < D::WIN / 2; e += ETH) cp_async16(dst + e, src + e);
      asm volatile("cp.async.commit_group;");
    }
    // FP64 stripe, line-major, zero beyond w
    if (jb.right) {
      for (int e = tid; e < ER * w; e += ETH) {
        const int li = e % ER, c = e / ER;
        Xf[li * XS + c] = (li < lines) ? X[(size_t)(lb + li) + (size_t)(o0 + c) * ldx] : 0.0;
      }
    } else {
      for (int e = tid; e < ER * w; e += ETH) {
        const int c = e % w, li = e / w;
        Xf[li * XS + c] = (li < lines) ? X[(size_t)(o0 + c) + (size_t)(lb + li) * ldx] : 0.0;
      }
    }
    for (int e = tid; e < ER * (2 * KPAD - w); e += ETH) {
      const int li = e / (2 * KPAD - w), c = w + e % (2 * KPAD - w);
      Xf[li * XS + c] = 0.0;
    }
    __syncthreads();
    // per-line bound of X_s
    {
      const int li = tid >> 3, part = tid & 7;
      int em = 1;
      for (int c = part; c < w; c += 8) em = max(em, expo(Xf[li * XS + c]));
      em = max(em, __shfl_xor_sync(0xffffffffu, em, 1));
      em = max(em, __shfl_xor_sync(0xffffffffu, em, 2));
      em = max(em, __shfl_xor_sync(0xffffffffu, em, 4));
      if (part == 0) Es[li] = em;
    }
    __syncthreads();
    // digits of X_s as A fragments: unit (m, ks), lane -> rows g, g+8; cols 2tt.., 2tt+8..
    for (int u = wi; u < 2 * KS1; u += ETH / 32) {
      const int m = u / KS1, ks = u % KS1;
      int d[8][EA];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        // register order: (g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1), (g, 2t+8), (g, 2t+9), (g+8, 2t+8), (g+8, 2t+9)
        const int li = m * 16 + g + 8 * ((i >> 1) & 1);
        const int c = ks * 16 + 2 * tt + (i & 1) + 8 * (i >> 2);
        digits9<EA>(to_fixed<0>(Xf[li * XS + c], Es[li]), d[i]);
      }
#pragma unroll
      for (int a = 0; a < EA; ++a)
        Xd[((a * 2 + m) * KS1 + ks) * 32 + lane] =
            make_uint4(pack2(d[0][a], d[1][a]), pack2(d[2][a], d[3][a]), pack2(d[4][a], d[5][a]),
                       pack2(d[6][a], d[7][a]));
    }
    asm volatile("cp.async.wait_group 0;");
    __syncthreads();
    // P = X_s Vw in fixed point: P = 2^(E + F - 55) Pf
    static_assert(2 * NT1 <= ETH / 32, "one tile of X_s Vw per warp");
    long long tp[4];
    if (wi < 2 * NT1)
      emu_tile<KS1>(tp, Xd + (wi / NT1) * KS1 * 32 + lane, 2 * KS1 * 32, Vd + (wi % NT1) * 32 + lane,
                    KS1 * NT1 * 32, NT1 * 32);
    __syncthreads();
    if (wi < 2 * NT1) {
      const int r0 = (wi / NT1) * 16 + g, q0 = (wi % NT1) * 8 + 2 * tt;
      Pf[r0 * M::PLD + q0] = tp[0];
      Pf[r0 * M::PLD + q0 + 1] = tp[1];
      Pf[(r0 + 8) * M::PLD + q0] = tp[2];
      Pf[(r0 + 8) * M::PLD + q0 + 1] = tp[3];
    }
    __syncthreads();
    // per-line bit length of P
    {
      const int li = tid >> 3, part = tid & 7;
      unsigned long long mx = 0;
      for (int q = part; q < KPAD; q += 8) {
        const long long v = Pf[li * M::PLD + q];
        mx = max(mx, (unsigned long long)(v < 0 ? -v : v));
      }
      mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mx, 1));
      mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mx, 2));
      mx = max(mx, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)mx, 4));
      if (part == 0) Bs[li] = 64 - __clzll((long long)mx);
    }
    __syncthreads();
    // digits of P (normalised per line to |Y| < 2^53) as A fragments
    for (int u = wi; u < 2 * KS2; u += ETH / 32) {
      const int m = u / KS2, ks = u % KS2;
      int d[8][EA];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int li = m * 16 + g + 8 * ((i >> 1) & 1);
        const int q = ks * 16 + 2 * tt + (i & 1) + 8 * (i >> 2);
        const long long v = Pf[li * M::PLD + q];
        const int beta = Bs[li];
        long long y;
        if (beta <= 53) y = v * (1LL << (53 - beta));
        else y = (v + (1LL << (beta - 54))) >> (beta - 53);
        digits9<EA>(y, d[i]);
      }
#pragma unroll
      for (int a = 0; a < EA; ++a)
        Pd[((a * 2 + m) * KS2 + ks) * 32 + lane] =
            make_uint4(pack2(d[0][a], d[1][a]), pack2(d[2][a], d[3][a]), pack2(d[4][a], d[5][a]),
                       pack2(d[6][a], d[7][a]));
    }
    __syncthreads();
    // U = P Ww^T, X_s <- X_s - U
    {
      const int fv = b.exps[2 * (t - b.t0)], fw = b.exps[2 * (t - b.t0) + 1];
      for (int u = wi; u < 2 * NT2; u += ETH / 32) {
        const int m = u / NT2, n = u % NT2;
        long long tu[4];
        emu_tile<KS2>(tu, Pd + m * KS2 * 32 + lane, 2 * KS2 * 32, Wd + n * 32 + lane, KS2 * NT2 * 32, NT2 * 32);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int li = m * 16 + g + 8 * (i >> 1);
          const int c = n * 8 + 2 * tt + (i & 1);
          if (c < w && tu[i] != 0) {
            // U = 2^(E + F + Omega + beta - 110) tu, E = Es - 1022, F = fv - 1022, Omega = fw - 1022
            const int su = Es[li] + fv + fw - 3 * 1022 + Bs[li] - 110;
            Xf[li * XS + c] = fma(-(double)tu[i], pow2i(su), Xf[li * XS + c]);
          }
        }
      }
    }
    __syncthreads();
    if (jb.right) {
      for (int e = tid; e < ER * w; e += ETH) {
        const int li = e % ER, c = e / ER;
        if (li < lines) X[(size_t)(lb + li) + (size_t)(o0 + c) * ldx] = Xf[li * XS + c];
      }
    } else {
      for (int e = tid; e < ER * w; e += ETH) {
        const int c = e % w, li = e / w;
        if (li < lines) X[(size_t)(o0 + c) + (size_t)(lb + li) * ldx] = Xf[li * XS + c];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Merged windows for chains with few reflectors per window (k <= 16).  The
// chain's transforms are applied in order, x <- x G_t G_{t+1} ..., and the
// product of g consecutive ones is again of the form I - V' W'^T on the union
// of their rows: for two, (I - V1 W1^T)(I - V2 W2^T) = I - [V1, V2 - V1 C]
// [W1, W2]^T with C = W1^T V2.  Merging g = floor(32 / k) windows gives
// blocks of at most (g + 1) k <= 48 rows and g k <= 32 columns, which the
// KPAD = 32 kernels apply as one dense window instead of g thin ones.  The
// chain itself (its windows and their order) is the one of Sec. 3.3.
// One CTA per merged window, FP64 in shared memory; output: V' at
// mwy + m * EMU_MSTRIDE (ld = width), W' at + EMU_MSTRIDE / 2, and the table
// geo[m] = (offset, width, columns, limit), the limit being the largest (mode 0)
// or smallest (mode 1) of the merged windows' so that no line the windows
// update is skipped.
// ---------------------------------------------------------------------------
constexpr int EMU_MROWS = 64, EMU_MCOLS = 32;
constexpr long EMU_MSTRIDE = 2L * EMU_MROWS * EMU_MCOLS;

__global__ void __launch_bounds__(ETH) emu_merge_kernel(const double* wy, long stride, int mode, int p, int k, int g,
                                                        int ta0, int t1, double* mwy, int4* geo) {
  __shared__ double Va[EMU_MROWS * EMU_MCOLS], Wa[EMU_MROWS * EMU_MCOLS], Cm[EMU_MCOLS * EMU_MCOLS];
  __shared__ int gq[4];
  const int tid = threadIdx.x;
  const int ta = ta0 + blockIdx.x * g, tb = min(t1, ta + g);
  if (tid == 0) {
    int o0 = 1 << 30, e0 = -1, kt = 0, lm = 0;
    for (int t = ta; t < tb; ++t) {
      int off, w, kr, lim;
      emu_win_geom(mode, p, k, t, &off, &w, &kr, &lim);
      o0 = min(o0, off);
      e0 = max(e0, off + w);
      kt += kr;
      lm = (t == ta) ? lim : (mode == 1 ? min(lm, lim) : max(lm, lim));
    }
    gq[0] = o0; gq[1] = e0 - o0; gq[2] = kt; gq[3] = lm;
  }
  for (int e = tid; e < EMU_MROWS * EMU_MCOLS; e += blockDim.x) { Va[e] = 0.0; Wa[e] = 0.0; }
  __syncthreads();
  const int o0 = gq[0], wp = gq[1], kp = gq[2];
  int r = 0;  // columns merged so far
  for (int t = ta; t < tb; ++t) {
    int off, w, kr, lim;
    emu_win_geom(mode, p, k, t, &off, &w, &kr, &lim);
    const double* Vw = wy + (size_t)t * stride;
    const double* Ww = Vw + stride / 2;
    const int ro = off - o0;
    // C = Wa(:, 0:r)^T V_t (r x kr); V_t lives on rows [ro, ro + w) of the union
    for (int e = tid; e < r * kr; e += blockDim.x) {
      const int i = e % r, c = e / r;
      double acc = 0.0;
      for (int q = 0; q < w; ++q) acc += Wa[(ro + q) + i * EMU_MROWS] * Vw[q + (size_t)c * w];
      Cm[i + c * EMU_MCOLS] = acc;
    }
    __syncthreads();
    for (int e = tid; e < wp * kr; e += blockDim.x) {
      const int row = e % wp, c = e / wp;
      const bool in = row >= ro && row < ro + w;
      double v = in ? Vw[(row - ro) + (size_t)c * w] : 0.0;
      for (int i = 0; i < r; ++i) v -= Va[row + i * EMU_MROWS] * Cm[i + c * EMU_MCOLS];
      Va[row + (r + c) * EMU_MROWS] = v;
      Wa[row + (r + c) * EMU_MROWS] = in ? Ww[(row - ro) + (size_t)c * w] : 0.0;
    }
    __syncthreads();
    r += kr;
  }
  double* Vo = mwy + (size_t)blockIdx.x * EMU_MSTRIDE;
  double* Wo = Vo + EMU_MSTRIDE / 2;
  for (int e = tid; e < wp * kp; e += blockDim.x) {
    const int row = e % wp, c = e / wp;
    Vo[e] = Va[row + c * EMU_MROWS];
    Wo[e] = Wa[row + c * EMU_MROWS];
  }
  if (tid == 0) geo[blockIdx.x] = make_int4(gq[0], gq[1], gq[2], gq[3]);
}

template <int KPAD>
cudaError_t emu_attr() {
  static std::mutex mu;
  static unsigned long long done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1ull) return cudaSuccess;
  e = cudaFuncSetAttribute(emu_sweep_kernel<KPAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)EmuSmem<KPAD>::BYTES);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

template <int KPAD>
cudaError_t emu_run(cudaStream_t st, const HtSweepJob* jobs, int njobs, const double* wy, long stride, int mode, int p,
                    int k, int t0, int t1, uint2* dig, int* exps, int cap, const int4* geo = nullptr) {
  using D = EmuDims<KPAD>;
  cudaError_t e = emu_attr<KPAD>();
  if (e != cudaSuccess) return e;
  EmuBatch b{};
  int ctas = 0, nj = 0;
  for (int i = 0; i < njobs; ++i) {
    if (jobs[i].nlines <= 0) continue;
    EmuJob& d = b.job[nj++];
    d.X = jobs[i].X; d.ldx = jobs[i].ldx; d.right = jobs[i].right; d.line0 = jobs[i].line0;
    d.nlines = jobs[i].nlines; d.origin = jobs[i].origin; d.use_limit = jobs[i].use_limit;
    d.limit_base = jobs[i].limit_base; d.cta0 = ctas;
    ctas += (jobs[i].nlines + ER - 1) / ER;
  }
  if (nj == 0) return cudaSuccess;
  b.njobs = nj; b.mode = mode; b.p = p; b.k = k; b.dig = dig; b.exps = exps; b.geo = geo;
  for (int c0 = t0; c0 < t1; c0 += cap) {
    const int c1 = std::min(t1, c0 + cap);
    emu_prep_kernel<KPAD><<<c1 - c0, ETH, 0, st>>>(wy, stride, mode, p, k, c0, dig, exps, geo);
    b.t0 = c0; b.t1 = c1;
    emu_sweep_kernel<KPAD><<<ctas, ETH, EmuSmem<KPAD>::BYTES, st>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

size_t ht_emu_window_bytes(int nb) {
  (void)nb;  // merged windows of small-k chains use the KPAD = 32 layout
  return (size_t)EmuDims<32>::WIN * sizeof(uint2);
}
size_t ht_emu_merge_doubles(int cap) { return (size_t)cap * EMU_MSTRIDE; }
long ht_merge_stride() { return EMU_MSTRIDE; }
cudaError_t ht_merge_windows(cudaStream_t st, const double* wy, long stride, int mode, int p, int k, int g, int ta,
                             int tb, double* mwy, void* geo) {
  if (tb <= ta) return cudaSuccess;
  const int nm = (tb - ta + g - 1) / g;
  emu_merge_kernel<<<nm, ETH, 0, st>>>(wy, stride, mode, p, k, g, ta, tb, mwy, (int4*)geo);
  return cudaGetLastError();
}

cudaError_t ht_emu_sweep_multi(cudaStream_t st, const HtSweepJob* jobs, int njobs, const double* wy, long stride, int mode,
                               int p, int k, int t0, int t1, void* dig, int* exps, int cap, double* mwy, void* geo) {
  if (njobs < 1 || njobs > HT_SWEEP_MAXJOBS) return cudaErrorInvalidValue;
  if (t1 <= t0) return cudaSuccess;
  const int g = k >= 1 ? 32 / k : 1;
  if (g >= 2 && mwy && geo) {
    // merged windows, at most cap of them per round (the buffers hold cap)
    const int nm = (t1 - t0 + g - 1) / g;
    for (int m0 = 0; m0 < nm; m0 += cap) {
      const int mc = std::min(cap, nm - m0);
      const int ta = t0 + m0 * g, tb = std::min(t1, ta + mc * g);
      cudaError_t e = ht_merge_windows(st, wy, stride, mode, p, k, g, ta, tb, mwy, geo);
      if (e != cudaSuccess) return e;
      e = emu_run<32>(st, jobs, njobs, mwy, EMU_MSTRIDE, EMU_MERGED, p, k, 0, mc, (uint2*)dig, exps, cap,
                      (const int4*)geo);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (k <= 32) return emu_run<32>(st, jobs, njobs, wy, stride, mode, p, k, t0, t1, (uint2*)dig, exps, cap);
  return cudaErrorNotSupported;
}
