// Small Householder factorizations of the absorption (Sec. 3.3): the QL chain
// that reduces V2 to L-hat (eq. (5)), the QR chain that reduces U2 to R-tilde
// (eq. (7)), and the RQ / QR factorizations of the blocks of B in the restore
// chains (Sec. 3.3.1e, 3.3.2f).  Every orthogonal factor is returned in regular
// WY form G = I - Vw Ww^T with Ww = Vw T^T, T grown by the rule of eq. (1)
// over the reflectors in product order.
//
// Launch structure
//   chains_kernel      2 CTAs: CTA 0 runs the QL chain of V2 and CTA 1 the QR
//                      chain of U2 (they are independent); each window's
//                      reflector vectors and coefficients go to the WY store.
//   form_wy_kernel     one CTA per window: T (recursive halving of eq. (1)) and
//                      Ww = Vw T^T, off the sequential path of the chains.
//   restore_kernel     cooperative, one launch per restore chain: CTA 0 factors
//                      the next block of B (RQ right / QR left) and forms its WY
//                      factors; after a grid barrier every CTA applies them to
//                      its stripes of B; a second barrier ends the step.
// An RQ factorization X G = [0 R1] of a k x w block is the QL factorization of
// X^T: X^T = G [0; R1^T].
#include <cooperative_groups.h>

#include <algorithm>

#include "ht_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int MAXW = 2 * HT_NB_MAX;  // largest window height

// Householder scalars of a column with pivot x0 and squared tail norm tail
// (DLARFG rule): alpha = -sign(x0) ||x||, beta = (alpha - x0) / alpha,
// scal = 1 / (x0 - alpha).  With r = 1 / ||x|| (one reciprocal square root),
// beta = 1 + |x0| r; only scal takes a division.  Called by lanes 0 and 1 of
// one warp (lane 0: beta and alpha, lane 1: scal); the chain of dependent FP64
// operations is the critical path of the factorizations.
__device__ __forceinline__ void house_scalars(double x0, double tail, double* sc, int lane) {
  if (tail == 0.0) {
    if (lane == 0) { sc[0] = 0.0; sc[1] = x0; sc[2] = 0.0; }
    return;
  }
  const double s2 = x0 * x0 + tail;
  const double r = rsqrt(s2);
  const double nr = s2 * r;
  const double alpha = (x0 >= 0.0) ? -nr : nr;
  if (lane == 0) { sc[0] = fma(fabs(x0), r, 1.0); sc[1] = alpha; }
  else sc[2] = 1.0 / (x0 - alpha);
}

// Householder QR (ql = false) or QL (ql = true) of the w x kk column-major
// matrix X (shared, ld w) in place.  On return X holds R (upper triangle in
// rows 0..kk-1) or L (lower triangle in rows w-kk..w-1) with exact zeros
// elsewhere, Vs (w x kk) the reflector vectors in product order and tau[q].
// Warp roles: warp 0 carries the critical path (next column, its norm and
// scalars); the FP64 unit of an SM is shared by its four sub-partitions and a
// busy warp on warp 0's own sub-partition slows warp 0's dependent chain the
// most, so the trailing columns go to the warps of sub-partitions 1-3 only
// (warps 1-3, 5-7); warp 4 publishes the reflectors when asked to.
// Look-ahead: warp 0 updates only the next column to reduce and prepares its
// reflector scalars (double-buffered in sc) while warps 1.. update the other
// columns four at a time with a packed cross-lane reduction.  bv (w entries)
// holds beta * v.  Two block barriers per reflector.

// sums of four per-lane partials over a warp, every lane receives all four
__device__ __forceinline__ void warp_sum4(double d[4], int lane) {
  const bool b16 = lane & 16, b8 = lane & 8;
  double s0 = b16 ? d[2] : d[0], s1 = b16 ? d[3] : d[1];
  const double o0 = __shfl_xor_sync(0xffffffffu, b16 ? d[0] : d[2], 16);
  const double o1 = __shfl_xor_sync(0xffffffffu, b16 ? d[1] : d[3], 16);
  s0 += o0;
  s1 += o1;
  double sv = b8 ? s1 : s0;
  sv += __shfl_xor_sync(0xffffffffu, b8 ? s0 : s1, 8);
  sv += __shfl_xor_sync(0xffffffffu, sv, 4);
  sv += __shfl_xor_sync(0xffffffffu, sv, 2);
  sv += __shfl_xor_sync(0xffffffffu, sv, 1);
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = __shfl_sync(0xffffffffu, sv, 16 * (i >> 1) + 8 * (i & 1));
}

// Optional publication of each reflector as soon as it is formed: v_q to
// gV(:, q) (ld w), tau_q to gTau[q], then flag = base + q + 1 (release), all by
// the last warp of the block, which then takes no column updates.
struct HousePub {
  double* gV;
  double* gTau;
  int* flag;
  int base;
};

__device__ void house_factor(double* X, int w, int kk, bool ql, double* Vs, double* tau, double* sc, double* bv,
                             const HousePub* pub = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const bool bulk = (wid & 3) != 0 && wid < 8;       // trailing-column warps (sub-partitions 1-3)
  const int br = wid - 1 - (wid >> 2), nbulk = 6;    // their rank
  for (int e = tid; e < w * kk; e += blockDim.x) Vs[e] = 0.0;
  if (wid == 0) {
    const int c = ql ? kk - 1 : 0, t = ql ? w - kk + c : c;
    const int lo = ql ? 0 : t, hi = ql ? t + 1 : w;
    double s = 0.0;
    for (int r = lo + lane; r < hi; r += 32)
      if (r != t) s += X[r + c * w] * X[r + c * w];
    s = ht_warp_sum(s);
    if (lane < 2) house_scalars(X[t + c * w], s, sc, lane);
  }
  __syncthreads();
  for (int q = 0; q < kk; ++q) {
    const int c = ql ? (kk - 1 - q) : q;
    const int t = ql ? (w - kk + c) : c;
    const int lo = ql ? 0 : t, hi = ql ? t + 1 : w;
    const double* cur = sc + 4 * (q & 1);
    double* nxt = sc + 4 * ((q + 1) & 1);
    const double beta = cur[0], alpha = cur[1], scal = cur[2];
    for (int r = lo + tid; r < hi; r += blockDim.x) {
      const double v = (r == t) ? 1.0 : X[r + c * w] * scal;
      Vs[r + q * w] = v;
      bv[r] = beta * v;
    }
    if (tid == 0) tau[q] = beta;
    __syncthreads();
    if (pub && wid == 4) {
      // publisher warp: reflector q to global memory, then its flag
      for (int r = lane; r < w; r += 32) pub->gV[r + (size_t)q * w] = Vs[r + q * w];
      if (lane == 0) pub->gTau[q] = tau[q];
      __threadfence();
      __syncwarp();
      if (lane == 0) ht_st_release(pub->flag, pub->base + q + 1);
      __syncthreads();
      continue;
    }
    const int cb = ql ? 0 : c + 1, ce = ql ? c : kk;
    const int cnext = (q + 1 < kk) ? (ql ? c - 1 : c + 1) : -1;
    if (wid == 0) {
      if (cnext >= 0) {
        // critical path: update column cnext, then its reflector scalars
        if (beta != 0.0) {
          double d = 0.0;
          for (int r = lo + lane; r < hi; r += 32) d += Vs[r + q * w] * X[r + cnext * w];
          d = ht_warp_sum(d);
          for (int r = lo + lane; r < hi; r += 32) X[r + cnext * w] -= d * bv[r];
        }
        __syncwarp();
        const int t2 = ql ? (w - kk + cnext) : cnext;
        const int lo2 = ql ? 0 : t2, hi2 = ql ? t2 + 1 : w;
        double sq = 0.0;
        for (int r = lo2 + lane; r < hi2; r += 32)
          if (r != t2) sq += X[r + cnext * w] * X[r + cnext * w];
        sq = ht_warp_sum(sq);
        __syncwarp();
        if (lane < 2) house_scalars(X[t2 + cnext * w], sq, nxt, lane);
      }
    } else if (bulk && beta != 0.0) {
      for (int g0 = cb + 4 * br; g0 < ce; g0 += 4 * nbulk) {
        double d[4] = {0.0, 0.0, 0.0, 0.0};
        for (int r = lo + lane; r < hi; r += 32) {
          const double vr = Vs[r + q * w];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (g0 + i < ce && g0 + i != cnext) d[i] += vr * X[r + (g0 + i) * w];
        }
        warp_sum4(d, lane);
        for (int r = lo + lane; r < hi; r += 32) {
          const double br = bv[r];
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (g0 + i < ce && g0 + i != cnext) X[r + (g0 + i) * w] -= d[i] * br;
        }
      }
    }
    for (int r = lo + tid; r < hi; r += blockDim.x) X[r + c * w] = (r == t) ? alpha : 0.0;
    __syncthreads();
  }
}

// T (kk x kk upper, ld kk) with Vs T Vs^T = I - H_0 H_1 ... by recursive
// halving: T = [T1, -T1 (V1^T V2) T2; 0, T2] (eq. (1) applied blockwise).
// Gm (kk x kk) receives V^T V; scr holds kk*kk doubles.  With `pad` (shared,
// MAXW * HT_NB_MAX doubles) the Gram product reads a copy of Vs with the odd
// leading dimension w + 1 when it fits, so that the lanes (consecutive
// columns a) hit distinct banks.
__device__ void form_t_rec(int kk, double* Tm, const double* Gm, double* scr);
__device__ void form_t(const double* Vs, const double* tau, int w, int kk, double* Tm, double* Gm, double* scr,
                       double* pad = nullptr) {
  const int tid = threadIdx.x;
  const bool use_pad = pad && (w + 1) * kk <= MAXW * HT_NB_MAX;
  const int wp = use_pad ? w + 1 : w;
  const double* Vg = use_pad ? pad : Vs;
  if (use_pad) {
    for (int e = tid; e < w * kk; e += blockDim.x) pad[(e % w) + (e / w) * wp] = Vs[e];
    __syncthreads();
  }
  for (int e = tid; e < kk * kk; e += blockDim.x) {
    const int a = e % kk, b = e / kk;
    Tm[e] = (a == b) ? tau[a] : 0.0;
    double d0 = 0.0, d1 = 0.0;
    if (a < b) {
      int r = 0;
      for (; r + 1 < w; r += 2) {
        d0 += Vg[r + a * wp] * Vg[r + b * wp];
        d1 += Vg[r + 1 + a * wp] * Vg[r + 1 + b * wp];
      }
      if (r < w) d0 += Vg[r + a * wp] * Vg[r + b * wp];
    }
    Gm[e] = d0 + d1;
  }
  __syncthreads();
  form_t_rec(kk, Tm, Gm, scr);
}

// The recursion of form_t on a given Gram matrix (strict upper triangle of
// Gm) and a Tm that holds diag(tau) with zeros elsewhere.
__device__ void form_t_rec(int kk, double* Tm, const double* Gm, double* scr) {
  const int tid = threadIdx.x;
  for (int h = 1; h < kk; h *= 2) {
    // pairs (lo block [p0, p0+h), hi block [p0+h, p0+2h)): T12 = -T11 (G12 T22)
    for (int e = tid; e < kk * kk; e += blockDim.x) {
      const int a = e % kk, b = e / kk;
      const int p0 = (a / (2 * h)) * (2 * h);
      const bool in = (a < p0 + h) && (b >= p0 + h) && (b < min(p0 + 2 * h, kk));
      double v = 0.0;
      if (in)
        for (int l = p0 + h; l <= b; ++l) v += Gm[a + l * kk] * Tm[l + b * kk];
      scr[e] = v;
    }
    __syncthreads();
    for (int e = tid; e < kk * kk; e += blockDim.x) {
      const int a = e % kk, b = e / kk;
      const int p0 = (a / (2 * h)) * (2 * h);
      const bool in = (a < p0 + h) && (b >= p0 + h) && (b < min(p0 + 2 * h, kk));
      if (in) {
        double v = 0.0;
        for (int l = a; l < p0 + h; ++l) v += Tm[a + l * kk] * scr[l + b * kk];
        Tm[e] = -v;
      }
    }
    __syncthreads();
  }
}

// Ww = Vs T^T (w x kk, ld w).
__device__ void form_w(const double* Vs, const double* Tm, int w, int kk, double* Ww) {
  for (int e = threadIdx.x; e < w * kk; e += blockDim.x) {
    const int r = e % w, i = e / w;
    double d = 0.0;
    for (int l = i; l < kk; ++l) d += Vs[r + l * w] * Tm[i + l * kk];
    Ww[e] = d;
  }
  __syncthreads();
}

// shared layout: X, Vs (MAXW*HT_NB_MAX each), Tm, Gm, scr (HT_NB_MAX^2 each), tau, sc (32), bv (MAXW)
__host__ __device__ inline size_t factor_smem_doubles() {
  return 2 * (size_t)MAXW * HT_NB_MAX + 3 * (size_t)HT_NB_MAX * HT_NB_MAX + HT_NB_MAX + 32 + MAXW;
}

struct FSm {
  double *X, *Vs, *Tm, *Gm, *scr, *tau, *nrm, *bv;
};
__device__ FSm fsm(double* sm) {
  FSm f;
  f.X = sm;
  f.Vs = f.X + MAXW * HT_NB_MAX;
  f.Tm = f.Vs + MAXW * HT_NB_MAX;
  f.Gm = f.Tm + HT_NB_MAX * HT_NB_MAX;
  f.scr = f.Gm + HT_NB_MAX * HT_NB_MAX;
  f.tau = f.scr + HT_NB_MAX * HT_NB_MAX;
  f.nrm = f.tau + HT_NB_MAX;
  f.bv = f.nrm + 32;
  return f;
}

// QL (mode 0, V2) or QR (mode 1, U2) chain of p x k windows; reflector vectors
// to wy + i*stride (ld = window height), coefficients to wy + i*stride + stride/2.
// The reduced k x k triangle (L-hat_1 bottom / R-tilde_1 top) goes to tri.
__device__ void run_chain(int mode, double* Xg, long ld, int p, int k, double* wy, size_t stride, double* tri,
                          double* sm) {
  FSm f = fsm(sm);
  const int nwin = ht_num_windows(p, k);
  for (int i = 0; i < nwin; ++i) {
    int r0, r1;
    if (mode == 0) ht_ql_window(p, k, i, &r0, &r1);
    else ht_qr_window(p, k, i, &r0, &r1);
    const int w = r1 - r0;
    for (int e = threadIdx.x; e < w * k; e += blockDim.x) {
      const int r = e % w, c = e / w;
      f.X[e] = Xg[(size_t)(r0 + r) + (size_t)c * ld];
    }
    __syncthreads();
    house_factor(f.X, w, k, mode == 0, f.Vs, f.tau, f.nrm, f.bv);
    double* Vw = wy + (size_t)i * stride;
    double* tw = Vw + stride / 2;
    for (int e = threadIdx.x; e < w * k; e += blockDim.x) {
      const int r = e % w, c = e / w;
      Xg[(size_t)(r0 + r) + (size_t)c * ld] = f.X[e];
      Vw[e] = f.Vs[e];
    }
    for (int q = threadIdx.x; q < k; q += blockDim.x) tw[q] = f.tau[q];
    __syncthreads();
  }
  const int tr0 = (mode == 0) ? p - k : 0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int r = e % k, c = e / k;
    tri[e] = Xg[(size_t)(tr0 + r) + (size_t)c * ld];
  }
}

__global__ void __launch_bounds__(HT_THREADS) chains_kernel(double* V2, double* U2, long ld, int p, int k,
                                                             double* wyR, double* wyL, size_t stride, double* L1,
                                                             double* R1) {
  extern __shared__ double sm[];
  if (blockIdx.x == 0) run_chain(0, V2, ld, p, k, wyR, stride, L1, sm);
  else run_chain(1, U2, ld, p, k, wyL, stride, R1, sm);
}

// T and Ww of one window per CTA (grid: nwr windows of wyR, then nwl of wyL)
__global__ void __launch_bounds__(HT_THREADS) form_wy_kernel(double* wyR, double* wyL, size_t stride, int p, int k,
                                                              int nwr, int nwl) {
  extern __shared__ double sm[];
  FSm f = fsm(sm);
  const bool right = (int)blockIdx.x < nwr;
  const int i = right ? (int)blockIdx.x : (int)blockIdx.x - nwr;
  if (!right && i >= nwl) return;
  int r0, r1;
  if (right) ht_ql_window(p, k, i, &r0, &r1);
  else ht_qr_window(p, k, i, &r0, &r1);
  const int w = r1 - r0;
  double* Vw = (right ? wyR : wyL) + (size_t)i * stride;
  double* Ww = Vw + stride / 2;
  for (int e = threadIdx.x; e < w * k; e += blockDim.x) f.Vs[e] = Vw[e];
  for (int q = threadIdx.x; q < k; q += blockDim.x) f.tau[q] = Ww[q];
  __syncthreads();
  form_t(f.Vs, f.tau, w, k, f.Tm, f.Gm, f.scr, f.X);
  form_w(f.Vs, f.Tm, w, k, Ww);
}

// ---------------------------------------------------------------------------
// Restore chains (cooperative).  Right (mode 2): for t = 0.., block b =
// nbr-1-t: RQ of B(block row b, cols of blocks b-1..b) -> [0 R1], then the
// rows above block row b times G.  Left (mode 3): for t = 0.., QR of B(rows of
// blocks t..t+1, col block t) -> [R; 0], then G^T times those rows over the
// columns right of block t.  Block coordinates are relative to j+1.
// ---------------------------------------------------------------------------
struct RestoreArgs {
  int mode, p, k, j, n;
  double* B;
  long ldb;
  double* wy;
  size_t stride;
  double* tstore;  // T factor of each step (k x k, ld k) for the appliers
  unsigned long long* ptime;  // optional timers: [16] factor, [17] T, [18] wait, [19] apply
};

__device__ __forceinline__ unsigned long long rs_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// right: X(lines [l0, l1), o0 .. o0+w) <- X G = X - (X V) T V^T;
// left:  X(o0 .. o0+w, lines) <- G^T X = X - V T^T (V^T X);
// stripes of SRR lines distributed over `nact` CTAs, this one being `rank`
// (stripes rank, rank + nact, ...).  A CTA with stripes first stages V
// (w x kr) and T (kr x kr) in shared memory (Vsm, Tsm) so that the products
// read no global memory in their inner loops.
constexpr int SRR = 8;
__device__ void apply_vt(bool right, double* X, long ldx, int l0, int l1, int o0, int w, int kr, const double* Vw,
                         const double* Tg, double* Xs, double* Ps, double* P2, double* Vsm, double* Tsm, int rank,
                         int nact) {
  const int tid = threadIdx.x;
  const int nstripes = (l1 - l0 + SRR - 1) / SRR;
  if (rank < 0 || rank >= nstripes) return;
  for (int e = tid; e < w * kr; e += blockDim.x) Vsm[e] = __ldcg(Vw + e);
  for (int e = tid; e < kr * kr; e += blockDim.x) Tsm[e] = __ldcg(Tg + e);
  __syncthreads();
  for (int sidx = rank; sidx < nstripes; sidx += nact) {
    const int sb = l0 + sidx * SRR, lines = min(SRR, l1 - sb);
    // stripe in shared memory column-major by line (Xs[li + c * SRR]): the
    // lanes of a warp take consecutive lines, so shared accesses are free of
    // bank conflicts; for left applications each group of SRR lanes reads
    // 32 contiguous bytes of four consecutive rows
    for (int e = tid; e < SRR * w; e += blockDim.x) {
      const int li = e % SRR, c = e / SRR;
      double v = 0.0;
      if (li < lines)
        v = right ? X[(size_t)(sb + li) + (size_t)(o0 + c) * ldx] : X[(size_t)(o0 + c) + (size_t)(sb + li) * ldx];
      Xs[li + c * SRR] = v;
    }
    __syncthreads();
    for (int e = tid; e < SRR * kr; e += blockDim.x) {
      const int li = e % SRR, q = e / SRR;
      double s0 = 0.0, s1 = 0.0;
      int c = 0;
      for (; c + 1 < w; c += 2) {
        s0 += Xs[li + c * SRR] * Vsm[c + q * w];
        s1 += Xs[li + (c + 1) * SRR] * Vsm[c + 1 + q * w];
      }
      if (c < w) s0 += Xs[li + c * SRR] * Vsm[c + q * w];
      Ps[li + q * SRR] = s0 + s1;
    }
    __syncthreads();
    // P2(li, :) = P(li, :) T: right (X V) T; left (T^T (V^T X))^T has the same rows
    for (int e = tid; e < SRR * kr; e += blockDim.x) {
      const int li = e % SRR, q = e / SRR;
      double s0 = 0.0;
      for (int l = 0; l <= q; ++l) s0 += Ps[li + l * SRR] * Tsm[l + q * kr];
      P2[li + q * SRR] = s0;
    }
    __syncthreads();
    for (int e = tid; e < SRR * w; e += blockDim.x) {
      const int li = e % SRR, c = e / SRR;
      if (li >= lines) continue;
      double s0 = Xs[li + c * SRR], s1 = 0.0;
      int q = 0;
      for (; q + 1 < kr; q += 2) {
        s0 -= P2[li + q * SRR] * Vsm[c + q * w];
        s1 -= P2[li + (q + 1) * SRR] * Vsm[c + (q + 1) * w];
      }
      if (q < kr) s0 -= P2[li + q * SRR] * Vsm[c + q * w];
      if (right) X[(size_t)(sb + li) + (size_t)(o0 + c) * ldx] = s0 + s1;
      else X[(size_t)(o0 + c) + (size_t)(sb + li) * ldx] = s0 + s1;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(HT_THREADS, 1) restore_kernel(RestoreArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sm[];
  FSm f = fsm(sm);
  double* Xs = f.Tm;  // stripe buffers reuse Tm, Gm, scr
  double* Ps = Xs + SRR * MAXW;
  double* P2 = Ps + SRR * HT_NB_MAX;
  const int p = a.p, k = a.k, j1 = a.j + 1;
  const bool right = (a.mode == 2);
  const int nsteps = right ? ht_num_right_blocks(p, k) - 1 : ht_num_left_blocks(p, k);
  const int wcta = (gridDim.x > 1) ? 1 : 0;  // forms Ww of the previous step while the others apply
  for (int t = 0; t < nsteps; ++t) {
    int off, width, kr, lim;
    if (right) {
      const int bb = ht_num_right_blocks(p, k) - 1 - t;
      int c0, c1, d0, d1;
      ht_right_block(p, k, bb - 1, &c0, &c1);
      ht_right_block(p, k, bb, &d0, &d1);
      off = c0; width = d1 - c0; kr = d1 - d0; lim = d0;
    } else {
      const int nlb = ht_num_left_blocks(p, k);
      int r0, r1, e0, e1;
      ht_left_block(p, k, t, &r0, &r1);
      if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
      off = r0; width = e1 - r0; kr = r1 - r0; lim = r1;
    }
    double* Vw = a.wy + (size_t)t * a.stride;
    double* Ww = Vw + a.stride / 2;
    double* Tg = a.tstore + (size_t)t * k * k;  // kr x kr, ld kr
    if (blockIdx.x == 0) {
      // right: QL of the transposed block row; left: QR of the block column
      double* blk = right ? a.B + (size_t)(j1 + lim) + (size_t)(j1 + off) * a.ldb
                          : a.B + (size_t)(j1 + off) + (size_t)(j1 + off) * a.ldb;
      const int w = width;
      for (int e = threadIdx.x; e < w * kr; e += blockDim.x) {
        const int r = e % w, c = e / w;
        f.X[e] = right ? blk[(size_t)c + (size_t)r * a.ldb] : blk[(size_t)r + (size_t)c * a.ldb];
      }
      __syncthreads();
      unsigned long long t0 = (a.ptime && threadIdx.x == 0) ? rs_now() : 0ull;
      house_factor(f.X, w, kr, right, f.Vs, f.tau, f.nrm, f.bv);
      unsigned long long t1 = (a.ptime && threadIdx.x == 0) ? rs_now() : 0ull;
      form_t(f.Vs, f.tau, w, kr, f.Tm, f.Gm, f.scr);
      if (a.ptime && threadIdx.x == 0) {
        const unsigned long long t2 = rs_now();
        a.ptime[16] += t1 - t0;
        a.ptime[17] += t2 - t1;
      }
      for (int e = threadIdx.x; e < w * kr; e += blockDim.x) {
        const int r = e % w, c = e / w;
        if (right) blk[(size_t)c + (size_t)r * a.ldb] = f.X[e];
        else blk[(size_t)r + (size_t)c * a.ldb] = f.X[e];
        Vw[e] = f.Vs[e];
      }
      for (int e = threadIdx.x; e < kr * kr; e += blockDim.x) Tg[e] = f.Tm[e];
      __threadfence();
    }
    unsigned long long tw0 = (a.ptime && blockIdx.x == 0 && threadIdx.x == 0) ? rs_now() : 0ull;
    grid.sync();
    if (a.ptime && blockIdx.x == 0 && threadIdx.x == 0) a.ptime[18] += rs_now() - tw0;
    tw0 = (a.ptime && blockIdx.x == 0 && threadIdx.x == 0) ? rs_now() : 0ull;
    if ((int)blockIdx.x == wcta && wcta != 0) {
      // Ww = Vw T^T for the bulk sweeps of A, Z / A, Q (and B's rows above)
      for (int e = threadIdx.x; e < width * kr; e += blockDim.x) f.Vs[e] = __ldcg(Vw + e);
      for (int e = threadIdx.x; e < kr * kr; e += blockDim.x) f.Tm[e] = __ldcg(Tg + e);
      __syncthreads();
      form_w(f.Vs, f.Tm, width, kr, Ww);
    } else {
      // every CTA but the one forming Ww
      const int nact = (wcta != 0) ? (int)gridDim.x - 1 : (int)gridDim.x;
      const int rank = ((int)blockIdx.x > wcta && wcta != 0) ? (int)blockIdx.x - 1 : (int)blockIdx.x;
      if (right) apply_vt(true, a.B, a.ldb, j1, j1 + lim, j1 + off, width, kr, Vw, Tg, Xs, Ps, P2, f.Vs, f.Gm, rank, nact);
      else apply_vt(false, a.B, a.ldb, j1 + lim, a.n, j1 + off, width, kr, Vw, Tg, Xs, Ps, P2, f.Vs, f.Gm, rank, nact);
    }
    grid.sync();
    if (a.ptime && blockIdx.x == 0 && threadIdx.x == 0) a.ptime[19] += rs_now() - tw0;
  }
  if (gridDim.x == 1) {
    // single CTA: form every Ww at the end
    for (int t = 0; t < nsteps; ++t) {
      int width, kr;
      if (right) {
        const int bb = ht_num_right_blocks(p, k) - 1 - t;
        int c0, c1, d0, d1;
        ht_right_block(p, k, bb - 1, &c0, &c1);
        ht_right_block(p, k, bb, &d0, &d1);
        width = d1 - c0; kr = d1 - d0;
      } else {
        const int nlb = ht_num_left_blocks(p, k);
        int r0, r1, e0, e1;
        ht_left_block(p, k, t, &r0, &r1);
        if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
        width = e1 - r0; kr = r1 - r0;
      }
      double* Vw = a.wy + (size_t)t * a.stride;
      for (int e = threadIdx.x; e < width * kr; e += blockDim.x) f.Vs[e] = Vw[e];
      for (int e = threadIdx.x; e < kr * kr; e += blockDim.x) f.Tm[e] = a.tstore[(size_t)t * k * k + e];
      __syncthreads();
      form_w(f.Vs, f.Tm, width, kr, Vw + a.stride / 2);
    }
  }
}

// ---------------------------------------------------------------------------
// Restore chains as a stream of reflectors (grids of >= 19 CTAs).  The step-t
// transform G_t must reach every line on the far side of the factored block
// (rows above for the RQ restore, columns to the right for the QR one), each
// line taking G_0, G_1, ... in order, but step t + 1 only needs it on the
// lines of the next block.  One grid barrier per step; in iteration t:
//   CTA 0   factors step t and publishes every reflector the moment it is
//           formed (V_t column, tau, then a release flag: t * RS_KSTEP + q + 1);
//   CTAs 2..17 (helpers) hold the lines of step t's next block in registers,
//           one line per warp, apply G_{t-1} and then G_t reflector by
//           reflector as the flags arrive, so the next block is up to date
//           when the factorization ends;
//   CTA 1   first finishes T_{t-1} (the recursion on the Gram matrix it built
//           in the previous iteration), raises tflag, then builds the Gram
//           columns of step t as the reflectors arrive; CTA 18 forms Ww_{t-1};
//   others  apply G_{t-1} with T_{t-1} (after tflag) to the lines beyond step
//           t's next block.
// The step time is the factorization alone.  A helper's wait is bounded; on a
// timeout it raises HT_ERR_TIMEOUT and stops, and every CTA keeps joining the
// barriers.
// ---------------------------------------------------------------------------
constexpr int RS_HELP = 16;                   // helper CTAs (two lines each for k = 32)
constexpr int RS_WCTA = 2 + RS_HELP;          // forms Ww of the previous step
constexpr int RS_FIRST_BULK = RS_WCTA + 1;
constexpr int RS_THREADS = HT_THREADS + 32;   // a ninth warp publishes the reflectors
constexpr int RS_KSTEP = 2 * HT_NB_MAX;       // flag values per step (> reflectors per step)

struct SplitArgs {
  int mode, p, k, j, n;
  double* B;
  long ldb;
  double* wy;
  size_t stride;
  double* tstore;
  double* taus;  // tau of step t at taus + t * k
  int* flag;     // [0] reflectors published, [1] T factors formed (zeroed by the launcher)
  int* err;      // device error word
  unsigned long long* ptime;
  long spin;     // polls before a bounded wait gives up
  int ta, tb;    // steps of this launch (a segment of the chain)
  int blo, bhi;  // lines the bulk CTAs update: [blo, bhi) (relative to j + 1)
};

// step s: window [off, off + width), nrefl kr, factored lines start f0, next block [n0, n1)
// (empty when none), lines beyond the next block [b0, b1); all relative to j + 1
struct SplitStep {
  int off, width, kr, f0, n0, n1, b0, b1;
};
__host__ __device__ __forceinline__ SplitStep split_step(bool right, int p, int k, int s) {
  SplitStep g;
  if (right) {
    const int bb = ht_num_right_blocks(p, k) - 1 - s;
    int c0, c1, d0, d1;
    ht_right_block(p, k, bb - 1, &c0, &c1);
    ht_right_block(p, k, bb, &d0, &d1);
    g.off = c0; g.width = d1 - c0; g.kr = d1 - d0; g.f0 = d0;
    g.n0 = c0; g.n1 = c1; g.b0 = 0; g.b1 = c0;
  } else {
    const int nlb = ht_num_left_blocks(p, k);
    int r0, r1, e0, e1;
    ht_left_block(p, k, s, &r0, &r1);
    if (s + 1 < nlb) ht_left_block(p, k, s + 1, &e0, &e1); else { e0 = r1; e1 = r1; }
    g.off = r0; g.width = e1 - r0; g.kr = r1 - r0; g.f0 = r0;
    g.n0 = e0; g.n1 = e1; g.b0 = e1; g.b1 = p;
  }
  return g;
}

// bounded wait of one thread for *p >= v: gives up at once when the error
// word is already set (a wait elsewhere gave up), else after `spin` polls,
// raising HT_ERR_TIMEOUT
__device__ bool split_wait(const int* p, int v, int* err, long spin) {
  if (ht_ld_acquire(p) >= v) return true;
  for (long it = 0; it < spin; ++it) {
    if (*(volatile int*)err != 0) return false;
    __nanosleep(32);
    if (ht_ld_acquire(p) >= v) return true;
  }
  atomicCAS(err, 0, HT_ERR_TIMEOUT);
  return false;
}

// The reflectors of one step (V at gV, ld w; tau at gTau; QL pattern for
// right, QR for left; kk of them in product order) applied to one line held in
// registers by one warp (at most four rows per lane, w <= 128), reflector q
// once flag >= base + q + 1 (SMEM: V and tau already in shared memory, every
// reflector published, no waiting).  Returns false on a timeout.
template <bool SMEM>
__device__ bool split_reflect(bool right, double x[4], int w, int kk, const double* gV, const double* gTau,
                              const int* flag, int base, int* err, long spin) {
  const int lane = threadIdx.x & 31;
  // reflector data: tau and v issued together; while this warp is behind the
  // factorization (the next flag already up) the next reflector is fetched
  // before the current one is applied
  auto fetch = [&](int q, double v[4], double& beta) {
    beta = SMEM ? gTau[q] : __ldcg(gTau + q);
    const int lo = right ? 0 : q, hi = right ? w - q : w;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = lane + 32 * u;
      v[u] = (r >= lo && r < hi) ? (SMEM ? gV[r + q * w] : __ldcg(gV + r + (size_t)q * w)) : 0.0;
    }
  };
  auto ready = [&](int q, bool wait) -> int {  // 1: published, 0: not yet, -1: timeout
    int st = 1;
    if (!SMEM && lane == 0) {
      if (wait) st = split_wait(flag, base + q + 1, err, spin) ? 1 : -1;
      else st = (ht_ld_acquire(flag) >= base + q + 1) ? 1 : 0;
    }
    return __shfl_sync(0xffffffffu, st, 0);
  };
  double v[4], beta = 0.0;
  if (kk <= 0) return true;
  if (ready(0, true) < 0) return false;
  fetch(0, v, beta);
  for (int q = 0; q < kk; ++q) {
    double vn[4] = {0.0, 0.0, 0.0, 0.0}, bn = 0.0;
    int nxt = 0;
    if (q + 1 < kk) {
      nxt = ready(q + 1, false);
      if (nxt > 0) fetch(q + 1, vn, bn);
    }
    if (beta != 0.0) {
      double d = 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) d += v[u] * x[u];
      d = beta * ht_warp_sum(d);
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] -= d * v[u];
    }
    if (q + 1 < kk) {
      if (nxt == 0) {
        if (ready(q + 1, true) < 0) return false;
        fetch(q + 1, vn, bn);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = vn[u];
      beta = bn;
    }
  }
  return true;
}

__global__ void __launch_bounds__(RS_THREADS, 1) restore_split_kernel(SplitArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sm[];
  FSm f = fsm(sm);
  double* Xs = f.Tm;  // stripe buffers of the bulk reuse Tm, Gm, scr
  double* Ps = Xs + SRR * MAXW;
  double* P2 = Ps + SRR * HT_NB_MAX;
  const int p = a.p, k = a.k, j1 = a.j + 1;
  const bool right = (a.mode == 2);
  const int nsteps = right ? ht_num_right_blocks(p, k) - 1 : ht_num_left_blocks(p, k);
  const int cta = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  double* Bt = a.B + (size_t)j1 + (size_t)j1 * a.ldb;
  const int ta = a.ta, tb = min(a.tb, nsteps);
  for (int t = ta; t <= tb; ++t) {
    if (cta == 0) {
      // ---- factorization of step t, reflectors published as they form ----
      if (t < tb) {
        const SplitStep g = split_step(right, p, k, t);
        const int w = g.width, kr = g.kr;
        for (int e = tid; e < w * kr; e += blockDim.x) {
          const int r = e % w, c = e / w;
          f.X[e] = __ldcg(right ? Bt + (size_t)(g.f0 + c) + (size_t)(g.off + r) * a.ldb
                                : Bt + (size_t)(g.off + r) + (size_t)(g.f0 + c) * a.ldb);
        }
        __syncthreads();
        const unsigned long long t0 = (a.ptime && tid == 0) ? rs_now() : 0ull;
        const HousePub pub{a.wy + (size_t)t * a.stride, a.taus + (size_t)t * k, a.flag, t * RS_KSTEP};
        house_factor(f.X, w, kr, right, f.Vs, f.tau, f.nrm, f.bv, &pub);
        if (a.ptime && tid == 0) a.ptime[16] += rs_now() - t0;
        for (int e = tid; e < w * kr; e += blockDim.x) {
          const int r = e % w, c = e / w;
          *(right ? Bt + (size_t)(g.f0 + c) + (size_t)(g.off + r) * a.ldb
                  : Bt + (size_t)(g.off + r) + (size_t)(g.f0 + c) * a.ldb) = f.X[e];
        }
      }
    } else if (cta == 1) {
      const unsigned long long t0 = (a.ptime && tid == 0) ? rs_now() : 0ull;
      if (t > ta) {
        // T_{t-1} from the Gram matrix, tau and V of step t-1 kept in shared memory, then Ww_{t-1}
        const SplitStep g = split_step(right, p, k, t - 1);
        const int kr = g.kr;
        for (int e = tid; e < kr * kr; e += blockDim.x) f.Tm[e] = (e % kr == e / kr) ? f.tau[e % kr] : 0.0;
        __syncthreads();
        form_t_rec(kr, f.Tm, f.Gm, f.scr);
        double* Tg = a.tstore + (size_t)(t - 1) * k * k;
        for (int e = tid; e < kr * kr; e += blockDim.x) Tg[e] = f.Tm[e];
        __threadfence();
        __syncthreads();
        if (tid == 0) ht_st_release(a.flag + 1, t);
      }
      if (t < tb) {
        // Gram columns of step t as the reflectors arrive, without block barriers:
        // warp wi keeps the columns c = wi (mod nw) in shared memory and, for every
        // arriving v_q (fetched by each warp itself, the next one early when its
        // flag is already up), forms Gm(c, q) for its c < q
        const SplitStep g = split_step(right, p, k, t);
        const int w = g.width, kr = g.kr, nw = blockDim.x >> 5;
        const double* gV = a.wy + (size_t)t * a.stride;
        const double* gT = a.taus + (size_t)t * k;
        const int base = t * RS_KSTEP;
        auto ready = [&](int q, bool wait) -> int {
          int st = 0;
          if (lane == 0) {
            if (wait) st = split_wait(a.flag, base + q + 1, a.err, a.spin) ? 1 : -1;
            else st = (ht_ld_acquire(a.flag) >= base + q + 1) ? 1 : 0;
          }
          return __shfl_sync(0xffffffffu, st, 0);
        };
        double v[4];
        auto fetch = [&](int q, double* dst) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = lane + 32 * u;
            dst[u] = (r < w) ? __ldcg(gV + r + (size_t)q * w) : 0.0;
          }
        };
        bool okw = ready(0, true) > 0;
        if (okw) fetch(0, v);
        for (int q = 0; q < kr && okw; ++q) {
          double vn[4] = {0.0, 0.0, 0.0, 0.0};
          int nxt = 0;
          if (q + 1 < kr) {
            nxt = ready(q + 1, false);
            if (nxt > 0) fetch(q + 1, vn);
          }
          for (int c = wid; c < q; c += nw) {
            double d = 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;
              if (r < w) d += f.Vs[r + c * w] * v[u];
            }
            d = ht_warp_sum(d);
            if (lane == 0) f.Gm[c + q * kr] = d;
          }
          if (q % nw == wid) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;
              if (r < w) f.Vs[r + q * w] = v[u];
            }
            if (lane == 0) f.tau[q] = __ldcg(gT + q);
            __syncwarp();
          }
          if (q + 1 < kr) {
            if (nxt == 0) {
              okw = ready(q + 1, true) > 0;
              if (okw) fetch(q + 1, vn);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = vn[u];
          }
        }
        __syncthreads();
      }
      if (a.ptime && tid == 0) a.ptime[17] += rs_now() - t0;
    } else if (cta < 2 + RS_HELP) {
      // ---- helpers: the next block of step t takes G_{t-1} (already applied at a
      // segment's first step, by the previous segment), then G_t as it streams ----
      if (t < tb) {
        const unsigned long long t0 = (a.ptime && cta == 2 && tid == 0) ? rs_now() : 0ull;
        const SplitStep g = split_step(right, p, k, t);
        const int nl = g.n1 - g.n0, per = (nl + RS_HELP - 1) / RS_HELP;
        const int l0 = g.n0 + (cta - 2) * per, l1 = min(g.n1, l0 + per);
        const bool prev = t > ta;
        const SplitStep gp = split_step(right, p, k, prev ? t - 1 : t);
        if (prev && l1 > l0) {
          // the reflectors of step t-1 (all published) from shared memory
          const double* Vp = a.wy + (size_t)(t - 1) * a.stride;
          for (int e = tid; e < gp.width * gp.kr; e += blockDim.x) f.Vs[e] = __ldcg(Vp + e);
          for (int q = tid; q < gp.kr; q += blockDim.x) f.tau[q] = __ldcg(a.taus + (size_t)(t - 1) * k + q);
          __syncthreads();
        }
        for (int line = l0 + wid; line < l1; line += blockDim.x >> 5) {
          double x[4];
          // the line over the union of both windows: right [off_t, off_t + width_t) holds both
          // transforms' columns (step t-1 acts on [off_{t-1}, ...) which is inside); left likewise
          const int lo = min(g.off, gp.off), hi = max(g.off + g.width, gp.off + gp.width);
          const int wu = prev ? hi - lo : g.width, ou = prev ? lo : g.off;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = lane + 32 * u;
            x[u] = (r < wu) ? __ldcg(right ? Bt + (size_t)line + (size_t)(ou + r) * a.ldb
                                           : Bt + (size_t)(ou + r) + (size_t)line * a.ldb)
                            : 0.0;
          }
          bool ok = true;
          if (prev) {
            // G_{t-1} acts on rows [gp.off - ou, ...) of x: shift into its own frame
            double y[4];
            const int sh = gp.off - ou;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;  // row of the window of step t-1
              const int src = r + sh;
              y[u] = 0.0;
#pragma unroll
              for (int v2 = 0; v2 < 4; ++v2) {
                const double xv = __shfl_sync(0xffffffffu, x[v2], src & 31);
                if ((src >> 5) == v2 && src < wu) y[u] = xv;
              }
            }
            ok = split_reflect<true>(right, y, gp.width, gp.kr, f.Vs, f.tau, a.flag, (t - 1) * RS_KSTEP, a.err,
                                    a.spin);
            // back into the union frame
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;  // row of the union
              const int src = r - sh;       // row of step t-1's window
#pragma unroll
              for (int v2 = 0; v2 < 4; ++v2) {
                const double yv = __shfl_sync(0xffffffffu, y[v2], src & 31);
                if (src >= 0 && src < gp.width && (src >> 5) == v2) x[u] = yv;
              }
            }
          }
          if (ok) {
            double y[4];
            const int sh = g.off - ou;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;
              const int src = r + sh;
              y[u] = 0.0;
#pragma unroll
              for (int v2 = 0; v2 < 4; ++v2) {
                const double xv = __shfl_sync(0xffffffffu, x[v2], src & 31);
                if ((src >> 5) == v2 && src < wu) y[u] = xv;
              }
            }
            ok = split_reflect<false>(right, y, g.width, g.kr, a.wy + (size_t)t * a.stride, a.taus + (size_t)t * k, a.flag,
                                      t * RS_KSTEP, a.err, a.spin);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = lane + 32 * u;
              const int src = r - sh;
#pragma unroll
              for (int v2 = 0; v2 < 4; ++v2) {
                const double yv = __shfl_sync(0xffffffffu, y[v2], src & 31);
                if (src >= 0 && src < g.width && (src >> 5) == v2) x[u] = yv;
              }
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int r = lane + 32 * u;
            if (r < wu) *(right ? Bt + (size_t)line + (size_t)(ou + r) * a.ldb : Bt + (size_t)(ou + r) + (size_t)line * a.ldb) = x[u];
          }
        }
        if (a.ptime && cta == 2 && tid == 0) a.ptime[18] += rs_now() - t0;
      }
    } else if (cta == RS_WCTA) {
      if (t > ta) {
        // Ww_{t-1} = V T^T for the later sweeps, once T_{t-1} is formed
        const SplitStep g = split_step(right, p, k, t - 1);
        if (tid == 0) split_wait(a.flag + 1, t, a.err, a.spin);
        __syncthreads();
        const double* Vw = a.wy + (size_t)(t - 1) * a.stride;
        const double* Tg = a.tstore + (size_t)(t - 1) * k * k;
        for (int e = tid; e < g.width * g.kr; e += blockDim.x) f.Vs[e] = __ldcg(Vw + e);
        for (int e = tid; e < g.kr * g.kr; e += blockDim.x) f.Tm[e] = __ldcg(Tg + e);
        __syncthreads();
        form_w(f.Vs, f.Tm, g.width, g.kr, a.wy + (size_t)(t - 1) * a.stride + a.stride / 2);
      }
    } else if (t > ta) {
      // ---- bulk: G_{t-1} with T_{t-1} beyond step t's next block (step t-1's at the
      // end), within the lines [blo, bhi) of this segment ----
      const SplitStep gp = split_step(right, p, k, t - 1);
      int b0, b1;
      if (t < tb) {
        const SplitStep g = split_step(right, p, k, t);
        b0 = g.b0; b1 = g.b1;
      } else {
        b0 = gp.b0; b1 = gp.b1;
      }
      b0 = max(b0, a.blo);
      b1 = min(b1, a.bhi);
      if (b1 > b0 && cta - RS_FIRST_BULK < (b1 - b0 + SRR - 1) / SRR) {
        if (tid == 0) split_wait(a.flag + 1, t, a.err, a.spin);  // T_{t-1} formed (a timeout is reported, work goes on)
        __syncthreads();
      }
      const unsigned long long t0 = (a.ptime && cta == RS_FIRST_BULK && tid == 0) ? rs_now() : 0ull;
      apply_vt(right, a.B, a.ldb, j1 + b0, j1 + b1, j1 + gp.off, gp.width, gp.kr, a.wy + (size_t)(t - 1) * a.stride,
               a.tstore + (size_t)(t - 1) * k * k, Xs, Ps, P2, f.Vs, f.Gm, cta - RS_FIRST_BULK,
               (int)gridDim.x - RS_FIRST_BULK);
      if (a.ptime && cta == RS_FIRST_BULK && tid == 0) a.ptime[19] += rs_now() - t0;
    }
    if (t == tb) break;
    __threadfence();
    grid.sync();
  }
}

}  // namespace

static int g_factor_attr = 0;
static void set_factor_attr() {
  if (g_factor_attr) return;
  const int bytes = (int)(factor_smem_doubles() * sizeof(double));
  cudaFuncSetAttribute(chains_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(form_wy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(restore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(restore_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  g_factor_attr = 1;
}

cudaError_t ht_launch_chains(cudaStream_t st, double* V2, double* U2, long ld, int p, int k, double* wyR, double* wyL,
                             size_t stride, double* L1, double* R1) {
  set_factor_attr();
  chains_kernel<<<2, HT_THREADS, factor_smem_doubles() * sizeof(double), st>>>(V2, U2, ld, p, k, wyR, wyL, stride,
                                                                               L1, R1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nw = ht_num_windows(p, k);
  form_wy_kernel<<<2 * nw, HT_THREADS, factor_smem_doubles() * sizeof(double), st>>>(wyR, wyL, stride, p, k, nw, nw);
  return cudaGetLastError();
}

cudaError_t ht_launch_form_wy(cudaStream_t st, double* wyR, double* wyL, size_t stride, int p, int k) {
  set_factor_attr();
  const int nw = ht_num_windows(p, k);
  form_wy_kernel<<<2 * nw, HT_THREADS, factor_smem_doubles() * sizeof(double), st>>>(wyR, wyL, stride, p, k, nw, nw);
  return cudaGetLastError();
}

int ht_restore_steps(int mode, int p, int k) {
  return (mode == 2) ? ht_num_right_blocks(p, k) - 1 : ht_num_left_blocks(p, k);
}

void ht_restore_band(int mode, int p, int k, int tb, int* blo, int* bhi) {
  // lines beyond the next block of step tb - 1: the ones a segment ending at
  // tb does not need (rows above for the RQ restore, columns right for the QR one)
  const SplitStep g = split_step(mode == 2, p, k, tb - 1);
  *blo = (mode == 2) ? g.b1 : 0;
  *bhi = (mode == 2) ? p : g.b0;
}

cudaError_t ht_launch_restore(cudaStream_t st, int mode, int p, int k, int j, int n, double* B, long ldb, double* wy,
                              size_t stride, double* tstore, double* taus, int* flag, int* err,
                              unsigned long long* ptime, long spin, int ta, int tb, int max_ctas) {
  set_factor_attr();
  const int nsteps = ht_restore_steps(mode, p, k);
  if (nsteps <= 0) return cudaSuccess;
  if (tb < 0 || tb > nsteps) tb = nsteps;
  if (ta < 0) ta = 0;
  if (ta >= tb) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (k <= 32 && sms > RS_FIRST_BULK && flag && err && taus) {  // the helpers hold three blocks of a line
    cudaError_t e = cudaMemsetAsync(flag, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    int blo = 0, bhi = p;
    if (tb < nsteps) ht_restore_band(mode, p, k, tb, &blo, &bhi);
    SplitArgs sa{mode, p, k, j, n, B, ldb, wy, stride, tstore, taus, flag, err, ptime, spin > 0 ? spin : HT_SPIN_LIMIT,
                 ta, tb, blo, bhi};
    void* sargs[] = {&sa};
    const int g = (max_ctas > RS_FIRST_BULK) ? std::min(sms, max_ctas) : sms;
    return cudaLaunchCooperativeKernel((void*)restore_split_kernel, dim3(g), dim3(RS_THREADS), sargs,
                                       factor_smem_doubles() * sizeof(double), st);
  }
  RestoreArgs a{mode, p, k, j, n, B, ldb, wy, stride, tstore, ptime};
  void* args[] = {&a};
  const int g = max_ctas > 0 ? std::min(sms, max_ctas) : sms;
  return cudaLaunchCooperativeKernel((void*)restore_kernel, dim3(g), dim3(HT_THREADS), args,
                                     factor_smem_doubles() * sizeof(double), st);
}
