// Level-3 updates of the absorption (Sec. 3.3) in native FP64.
//
//  sweep_right  X(:, win_t) <- X(:, win_t) G_t for a chain of windows t, each
//               CTA owning a stripe of rows (the chains B Q^_1..Q^_r, Z Q^..,
//               A Q^.. of Sec. 3.3.1c-e and the restore chains).
//  sweep_left   X(win_t, :) <- G_t^T X(win_t, :) over column stripes
//               (Q~_r^T..Q~_1^T B, A of Sec. 3.3.2c,e and the QR restore).
//  rankk_right  X1 -= (X1 V1 + X2 L1) T V1^T, X2 -= (X1 V1 + X2 L1) T L1^T
//               (steps 2-4 of Sec. 3.3.1c/d; with no X2 also Q's update of
//               Sec. 3.3.2d).
//  rankk_left   X(r0:r0+2k, :) -= U~ S^T (U~^T X(r0:r0+2k, :)) (steps 4-5 of
//               Sec. 3.3.2c, step 2-3 of Sec. 3.3.2e), U~ = [U1; R~1].
//  gemm         C = alpha op(A) op(B) + beta C (deferred rows of Y, Remark 3.1;
//               spike update of Sec. 3.3.2c step 1).
// Window geometry is recomputed on the device from (p, k) with the same
// functions the host uses (ht_common.cuh), so no descriptors are copied.
#include <algorithm>
#include <mutex>

#include "ht_common.cuh"

namespace {

constexpr int SR = 32;                  // stripe rows (right sweeps) / columns (left sweeps)
constexpr int SRK = 16;                 // stripe of the fused rank-k kernels
constexpr int MAXW = 2 * HT_NB_MAX;     // widest window

// Geometry of window t of a chain.  Modes:
//   0 QL chain on V2 (right): cols [r0, r1); limit = r1 (rows >= col0+r1 are zero in B)
//   1 QR chain on U2 (left):  rows [r0, r1); limit = r0 (cols < col0+r0 are zero in B)
//   2 RQ restore, step t = block b = nbr-1-t: cols [start(b-1), end(b)); limit = start(b)
//   3 QR restore, step t = block b = t: rows [start(b), end(b+1) or end(b)); limit = end(b)
//   4 single explicit window: offset = p, width = k, nrefl = limit_base (see launchers)
__device__ __forceinline__ void win_geom(int mode, int p, int k, int t, int* off, int* width, int* nrefl,
                                         int* limit) {
  int a, b;
  if (mode == 0) {
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

// One launch applies the same chain to up to HT_SWEEP_MAXJOBS independent
// targets (B, A, Z or Q of one absorption step), each a "job" with its own
// direction and line range; the CTAs of job i are [cta0_i, cta0_{i+1}).
// Fusing the targets fills the GPU even when one target has few stripes.
struct SweepJob {
  double* X;
  long ldx;
  int right;       // 1: X(:, win) <- X(:, win) G;  0: X(win, :) <- G^T X(win, :)
  int line0;       // first row (right) / column (left) swept
  int nlines;      // rows (right) or columns (left) swept
  int origin;      // column (right) or row (left) index of window offset 0
  int use_limit;   // 1: skip stripes the structural limit says are zero
  int limit_base;  // added to the window limit
  int cta0;        // first CTA of the job
};

struct SweepBatch {
  SweepJob job[HT_SWEEP_MAXJOBS];
  int njobs;
  const double* wy;
  long stride;     // doubles between consecutive windows of the WY store (Ww at stride / 2)
  int mode, p, k, t0, t1;
  int ex_off, ex_width, ex_nrefl;  // mode 4
};

// Right application to rows [line0 + stripe*SR, ...) of X, X(:, c) <- X(:, c) G.
// The stripe sits in shared memory column-major (Xs[r + c * SR]) so that the
// lanes of a warp, which take consecutive rows, hit distinct banks; Vw and Ww
// entries are warp-uniform (broadcast loads through L1).
__device__ void sweep_right_body(const SweepBatch& b, const SweepJob& jb, int stripe, double* Xs, double* Ps) {
  const int tid = threadIdx.x;
  const int row_begin = jb.line0 + stripe * SR;
  const int row_end = min(jb.line0 + jb.nlines, row_begin + SR);
  const int rows = row_end - row_begin;
  if (rows <= 0) return;
  double* X = jb.X;
  const long ldx = jb.ldx;
  for (int t = b.t0; t < b.t1; ++t) {
    int off, w, kr, lim;
    if (b.mode == 4) { off = b.ex_off; w = b.ex_width; kr = b.ex_nrefl; lim = 0; }
    else win_geom(b.mode, b.p, b.k, t, &off, &w, &kr, &lim);
    if (jb.use_limit && row_begin >= jb.limit_base + lim) continue;
    const double* Vw = b.wy + (size_t)t * b.stride;
    const double* Ww = Vw + b.stride / 2;
    const int c0 = jb.origin + off;
    for (int e = tid; e < SR * w; e += blockDim.x) {
      const int r = e % SR, c = e / SR;
      Xs[r + c * SR] = (r < rows) ? X[(size_t)(row_begin + r) + (size_t)(c0 + c) * ldx] : 0.0;
    }
    __syncthreads();
    // P = Xs Vw (SR x kr)
    for (int e = tid; e < SR * kr; e += blockDim.x) {
      const int r = e % SR, q = e / SR;
      const double* v = Vw + (size_t)q * w;
      double s0 = 0.0, s1 = 0.0;
      int c = 0;
      for (; c + 1 < w; c += 2) {
        s0 += Xs[r + c * SR] * __ldg(v + c);
        s1 += Xs[r + (c + 1) * SR] * __ldg(v + c + 1);
      }
      if (c < w) s0 += Xs[r + c * SR] * __ldg(v + c);
      Ps[r + q * SR] = s0 + s1;
    }
    __syncthreads();
    // Xs -= P Ww^T, write back
    for (int e = tid; e < SR * w; e += blockDim.x) {
      const int r = e % SR, c = e / SR;
      if (r >= rows) continue;
      double s0 = Xs[r + c * SR], s1 = 0.0;
      int q = 0;
      for (; q + 1 < kr; q += 2) {
        s0 -= Ps[r + q * SR] * __ldg(Ww + (size_t)q * w + c);
        s1 -= Ps[r + (q + 1) * SR] * __ldg(Ww + (size_t)(q + 1) * w + c);
      }
      if (q < kr) s0 -= Ps[r + q * SR] * __ldg(Ww + (size_t)q * w + c);
      X[(size_t)(row_begin + r) + (size_t)(c0 + c) * ldx] = s0 + s1;
    }
    __syncthreads();
  }
}

// Left application to columns [line0 + stripe*SR, ...) of X, X(rows, c) <- G^T X(rows, c).
// Xs is w x SR with the odd leading dimension XLD, so that lanes taking
// consecutive columns hit distinct banks; Ps is nrefl x SR stored Ps[c + q * SR].
constexpr int XLD = MAXW + 1;
__device__ void sweep_left_body(const SweepBatch& b, const SweepJob& jb, int stripe, double* Xs, double* Ps) {
  const int tid = threadIdx.x;
  const int col_begin = jb.line0 + stripe * SR;
  const int col_end = min(jb.line0 + jb.nlines, col_begin + SR);
  const int cols = col_end - col_begin;
  if (cols <= 0) return;
  double* X = jb.X;
  const long ldx = jb.ldx;
  for (int t = b.t0; t < b.t1; ++t) {
    int off, w, kr, lim;
    if (b.mode == 4) { off = b.ex_off; w = b.ex_width; kr = b.ex_nrefl; lim = 0; }
    else win_geom(b.mode, b.p, b.k, t, &off, &w, &kr, &lim);
    if (jb.use_limit && col_end <= jb.limit_base + lim) continue;
    const double* Vw = b.wy + (size_t)t * b.stride;
    const double* Ww = Vw + b.stride / 2;
    const int r0 = jb.origin + off;
    for (int e = tid; e < w * SR; e += blockDim.x) {
      const int r = e % w, c = e / w;
      Xs[r + c * XLD] = (c < cols) ? X[(size_t)(r0 + r) + (size_t)(col_begin + c) * ldx] : 0.0;
    }
    __syncthreads();
    // P = Vw^T Xs (kr x SR): lanes take columns, Vw entries are warp-uniform
    for (int e = tid; e < kr * SR; e += blockDim.x) {
      const int c = e % SR, q = e / SR;
      const double* v = Vw + (size_t)q * w;
      double s0 = 0.0, s1 = 0.0;
      int r = 0;
      for (; r + 1 < w; r += 2) {
        s0 += __ldg(v + r) * Xs[r + c * XLD];
        s1 += __ldg(v + r + 1) * Xs[r + 1 + c * XLD];
      }
      if (r < w) s0 += __ldg(v + r) * Xs[r + c * XLD];
      Ps[c + q * SR] = s0 + s1;
    }
    __syncthreads();
    // Xs -= Ww P, write back
    for (int e = tid; e < w * SR; e += blockDim.x) {
      const int r = e % w, c = e / w;
      if (c >= cols) continue;
      double s0 = Xs[r + c * XLD], s1 = 0.0;
      int q = 0;
      for (; q + 1 < kr; q += 2) {
        s0 -= __ldg(Ww + (size_t)q * w + r) * Ps[c + q * SR];
        s1 -= __ldg(Ww + (size_t)(q + 1) * w + r) * Ps[c + (q + 1) * SR];
      }
      if (q < kr) s0 -= __ldg(Ww + (size_t)q * w + r) * Ps[c + q * SR];
      X[(size_t)(r0 + r) + (size_t)(col_begin + c) * ldx] = s0 + s1;
    }
    __syncthreads();
  }
}

constexpr size_t SWEEP_RIGHT_SMEM = (size_t)SR * MAXW + (size_t)SR * HT_NB_MAX;
constexpr size_t SWEEP_LEFT_SMEM = (size_t)XLD * SR + (size_t)HT_NB_MAX * SR;
constexpr size_t SWEEP_SMEM = sizeof(double) * (SWEEP_RIGHT_SMEM > SWEEP_LEFT_SMEM ? SWEEP_RIGHT_SMEM : SWEEP_LEFT_SMEM);

__global__ void __launch_bounds__(HT_THREADS) sweep_kernel(SweepBatch b) {
  extern __shared__ double sw_sm[];
  // select the job without indexing the parameter array dynamically
  SweepJob jb = b.job[0];
#pragma unroll
  for (int i = 1; i < HT_SWEEP_MAXJOBS; ++i)
    if (i < b.njobs && (int)blockIdx.x >= b.job[i].cta0) jb = b.job[i];
  const int stripe = (int)blockIdx.x - jb.cta0;
  if (jb.right) sweep_right_body(b, jb, stripe, sw_sm, sw_sm + SR * MAXW);
  else sweep_left_body(b, jb, stripe, sw_sm, sw_sm + XLD * SR);
}

// X1 (cols c1..c1+w1) -= W T V1^T, X2 (cols c2..c2+k) -= W T L1^T with
// W = X1 V1 + X2 L1 (X2 absent when c2 < 0).  Row stripes of SRK rows held
// column-major in shared memory (consecutive lanes, consecutive rows).
__global__ void __launch_bounds__(HT_THREADS) rankk_right_kernel(double* X, long ldx, int nrows, int c1, int w1,
                                                                  int c2, int k, const double* V1, int ldv1,
                                                                  const double* L1, int ldl1, const double* Tm,
                                                                  int ldt) {
  __shared__ double X1s[SRK * MAXW];
  __shared__ double X2s[SRK * HT_NB_MAX];
  __shared__ double Ws[SRK * HT_NB_MAX];
  __shared__ double W2s[SRK * HT_NB_MAX];
  const int tid = threadIdx.x;
  const int rb = blockIdx.x * SRK, rows = min(SRK, nrows - rb);
  if (rows <= 0) return;
  for (int e = tid; e < SRK * w1; e += blockDim.x) {
    const int r = e % SRK, c = e / SRK;
    X1s[r + c * SRK] = (r < rows) ? X[(size_t)(rb + r) + (size_t)(c1 + c) * ldx] : 0.0;
  }
  if (c2 >= 0)
    for (int e = tid; e < SRK * k; e += blockDim.x) {
      const int r = e % SRK, c = e / SRK;
      X2s[r + c * SRK] = (r < rows) ? X[(size_t)(rb + r) + (size_t)(c2 + c) * ldx] : 0.0;
    }
  __syncthreads();
  for (int e = tid; e < SRK * k; e += blockDim.x) {
    const int r = e % SRK, q = e / SRK;
    double s0 = 0.0;
    for (int c = 0; c < w1; ++c) s0 += X1s[r + c * SRK] * __ldg(V1 + c + (size_t)q * ldv1);
    if (c2 >= 0)
      for (int c = 0; c < k; ++c) s0 += X2s[r + c * SRK] * __ldg(L1 + c + (size_t)q * ldl1);
    Ws[r + q * SRK] = s0;
  }
  __syncthreads();
  for (int e = tid; e < SRK * k; e += blockDim.x) {
    const int r = e % SRK, q = e / SRK;
    double s0 = 0.0;
    for (int l = 0; l < k; ++l) s0 += Ws[r + l * SRK] * __ldg(Tm + l + (size_t)q * ldt);
    W2s[r + q * SRK] = s0;
  }
  __syncthreads();
  for (int e = tid; e < SRK * w1; e += blockDim.x) {
    const int r = e % SRK, c = e / SRK;
    if (r >= rows) continue;
    double s0 = X1s[r + c * SRK];
    for (int q = 0; q < k; ++q) s0 -= W2s[r + q * SRK] * __ldg(V1 + c + (size_t)q * ldv1);
    X[(size_t)(rb + r) + (size_t)(c1 + c) * ldx] = s0;
  }
  if (c2 >= 0)
    for (int e = tid; e < SRK * k; e += blockDim.x) {
      const int r = e % SRK, c = e / SRK;
      if (r >= rows) continue;
      double s0 = X2s[r + c * SRK];
      for (int q = 0; q < k; ++q) s0 -= W2s[r + q * SRK] * __ldg(L1 + c + (size_t)q * ldl1);
      X[(size_t)(rb + r) + (size_t)(c2 + c) * ldx] = s0;
    }
}

// X(r0:r0+w1, cols) -= Ut (S^T (Ut^T X(r0:r0+w1, cols))), column stripes.
// Xs has an odd leading dimension so that lanes taking consecutive columns
// hit distinct banks; P and P2 are stored as P[c + q * SRK].
__global__ void __launch_bounds__(HT_THREADS) rankk_left_kernel(double* X, long ldx, int col0, int ncols, int r0,
                                                                 int w1, int k, const double* Ut, int ldu,
                                                                 const double* S, int lds) {
  constexpr int LD = MAXW + 1;
  __shared__ double Xs[LD * SRK];
  __shared__ double Ps[HT_NB_MAX * SRK];
  __shared__ double P2[HT_NB_MAX * SRK];
  const int tid = threadIdx.x;
  const int cb = col0 + blockIdx.x * SRK, cols = min(SRK, col0 + ncols - cb);
  if (cols <= 0) return;
  for (int e = tid; e < w1 * SRK; e += blockDim.x) {
    const int r = e % w1, c = e / w1;
    Xs[r + c * LD] = (c < cols) ? X[(size_t)(r0 + r) + (size_t)(cb + c) * ldx] : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < k * SRK; e += blockDim.x) {
    const int c = e % SRK, q = e / SRK;
    double s0 = 0.0;
    for (int r = 0; r < w1; ++r) s0 += __ldg(Ut + r + (size_t)q * ldu) * Xs[r + c * LD];
    Ps[c + q * SRK] = s0;
  }
  __syncthreads();
  for (int e = tid; e < k * SRK; e += blockDim.x) {
    const int c = e % SRK, q = e / SRK;
    double s0 = 0.0;
    for (int l = 0; l < k; ++l) s0 += __ldg(S + l + (size_t)q * lds) * Ps[c + l * SRK];  // S^T
    P2[c + q * SRK] = s0;
  }
  __syncthreads();
  for (int e = tid; e < w1 * SRK; e += blockDim.x) {
    const int r = e % w1, c = e / w1;
    if (c >= cols) continue;
    double s0 = Xs[r + c * LD];
    for (int q = 0; q < k; ++q) s0 -= __ldg(Ut + r + (size_t)q * ldu) * P2[c + q * SRK];
    X[(size_t)(r0 + r) + (size_t)(cb + c) * ldx] = s0;
  }
}

// C = alpha op(A) op(B) + beta C, 64 x 64 tiles, 4 x 4 per thread, K chunks of 16.
constexpr int GT = 64, GK = 16;
// With gridDim.z > 1 (split K) each z-slice writes alpha * (its partial
// product) to part + z * M * N (ld M); a second kernel adds the slices in order.
__global__ void __launch_bounds__(256) gemm_kernel(int ta, int tb, int M, int N, int K, double alpha,
                                                   const double* A, long lda, const double* Bm, long ldb,
                                                   double beta, double* C, long ldc, double* part, int kchunk) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.x * GT, n0 = blockIdx.y * GT;
  double acc[4][4] = {};
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e % GK, mm = e / GK;
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < kend) v = ta ? A[(size_t)gk + (size_t)gm * lda] : A[(size_t)gm + (size_t)gk * lda];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e % GK, nn = e / GK;
      const int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < kend) v = tb ? Bm[(size_t)gn + (size_t)gk * ldb] : Bm[(size_t)gk + (size_t)gn * ldb];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][tx + 16 * i];
#pragma unroll
      for (int jx = 0; jx < 4; ++jx) bv[jx] = Bs[kk][ty + 16 * jx];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) acc[i][jx] += av[i] * bv[jx];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jx = 0; jx < 4; ++jx) {
      const int gm = m0 + tx + 16 * i, gn = n0 + ty + 16 * jx;
      if (gm < M && gn < N) {
        if (part) {
          part[(size_t)blockIdx.z * M * N + gm + (size_t)gn * M] = alpha * acc[i][jx];
        } else {
          double* c = C + (size_t)gm + (size_t)gn * ldc;
          *c = alpha * acc[i][jx] + (beta == 0.0 ? 0.0 : beta * (*c));
        }
      }
    }
}

__global__ void splitk_reduce_kernel(int M, int N, int splits, const double* part, double beta, double* C,
                                     long ldc) {
  const long total = (long)M * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int z = 0; z < splits; ++z) v += part[(size_t)z * total + e];
    const int gm = (int)(e % M), gn = (int)(e / M);
    double* c = C + (size_t)gm + (size_t)gn * ldc;
    *c = v + (beta == 0.0 ? 0.0 : beta * (*c));
  }
}

__global__ void zero_kernel(double* X, long ldx, int rows, int cols, int lower_only) {
  const long total = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e % rows), c = (int)(e / rows);
    if (!lower_only || r > c) X[(size_t)r + (size_t)c * ldx] = 0.0;
  }
}

__global__ void identity_kernel(double* X, long ldx, int n) {
  const long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    X[(size_t)r + (size_t)c * ldx] = (r == c) ? 1.0 : 0.0;
  }
}

__global__ void finite_kernel(const double* X, long ldx, int n, int upper_only, int* err) {
  const long total = (long)n * n;
  int bad = 0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e % n), c = (int)(e / n);
    if (upper_only && r > c) continue;
    if (!isfinite(X[(size_t)r + (size_t)c * ldx])) bad = 1;
  }
  if (bad) atomicCAS(err, 0, HT_ERR_NONFINITE);
}

inline int grid_for(long work, int per) {
  long g = (work + per - 1) / per;
  if (g < 1) g = 1;
  if (g > 8 * 152) g = 8 * 152;
  return (int)g;
}

}  // namespace

cudaError_t ht_gemm_ws(cudaStream_t st, char ta, char tb, int M, int N, int K, double alpha, const double* A,
                       int lda, const double* Bm, int ldb, double beta, double* C, int ldc, double* ws,
                       size_t ws_doubles) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((M + GT - 1) / GT, (N + GT - 1) / GT, 1);
  const long tiles = (long)grid.x * grid.y;
  int splits = 1;
  if (ws && tiles < 2 * 152 && K > 4 * GK) {
    splits = (int)std::min<long>((2 * 152 + tiles - 1) / tiles, (K + 4 * GK - 1) / (4 * GK));
    while (splits > 1 && (size_t)splits * M * N > ws_doubles) --splits;
  }
  if (splits <= 1) {
    gemm_kernel<<<grid, 256, 0, st>>>(ta == 'T', tb == 'T', M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc, nullptr,
                                      K);
    return cudaGetLastError();
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + GK - 1) / GK * GK;
  splits = (K + kchunk - 1) / kchunk;
  grid.z = splits;
  gemm_kernel<<<grid, 256, 0, st>>>(ta == 'T', tb == 'T', M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc, ws, kchunk);
  splitk_reduce_kernel<<<grid_for((long)M * N, 256), 256, 0, st>>>(M, N, splits, ws, beta, C, ldc);
  return cudaGetLastError();
}

cudaError_t ht_gemm(cudaStream_t st, char ta, char tb, int M, int N, int K, double alpha, const double* A, int lda,
                    const double* Bm, int ldb, double beta, double* C, int ldc) {
  return ht_gemm_ws(st, ta, tb, M, N, K, alpha, A, lda, Bm, ldb, beta, C, ldc, nullptr, 0);
}

// The sweep takes more than the default 48 KB of dynamic shared memory: raise
// its limit once per device.
static cudaError_t sweep_attr() {
  static std::mutex mu;
  static unsigned long long done = 0;  // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1ull) return cudaSuccess;
  e = cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_SMEM);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

static cudaError_t launch_batch(cudaStream_t st, SweepBatch& b, const HtSweepJob* jobs, int njobs) {
  if (njobs < 1 || njobs > HT_SWEEP_MAXJOBS) return cudaErrorInvalidValue;
  if (b.t1 <= b.t0) return cudaSuccess;
  int ctas = 0, nj = 0;
  for (int i = 0; i < njobs; ++i) {
    if (jobs[i].nlines <= 0) continue;
    SweepJob& d = b.job[nj++];
    d.X = jobs[i].X; d.ldx = jobs[i].ldx; d.right = jobs[i].right; d.line0 = jobs[i].line0;
    d.nlines = jobs[i].nlines; d.origin = jobs[i].origin; d.use_limit = jobs[i].use_limit;
    d.limit_base = jobs[i].limit_base; d.cta0 = ctas;
    ctas += (jobs[i].nlines + SR - 1) / SR;
  }
  if (nj == 0) return cudaSuccess;
  b.njobs = nj;
  const cudaError_t e = sweep_attr();
  if (e != cudaSuccess) return e;
  sweep_kernel<<<ctas, HT_THREADS, SWEEP_SMEM, st>>>(b);
  return cudaGetLastError();
}

cudaError_t ht_sweep_multi(cudaStream_t st, const HtSweepJob* jobs, int njobs, const double* wy, long stride, int mode,
                           int p, int k, int t0, int t1) {
  SweepBatch b{};
  b.wy = wy; b.stride = stride; b.mode = mode; b.p = p; b.k = k; b.t0 = t0; b.t1 = t1;
  return launch_batch(st, b, jobs, njobs);
}

cudaError_t ht_sweep(cudaStream_t st, int right, double* X, long ldx, int line0, int nlines, int origin,
                     const double* wy, long stride, int mode, int p, int k, int t0, int t1, int use_limit,
                     int limit_base) {
  const HtSweepJob j{X, ldx, right, line0, nlines, origin, use_limit, limit_base};
  return ht_sweep_multi(st, &j, 1, wy, stride, mode, p, k, t0, t1);
}

cudaError_t ht_apply_single(cudaStream_t st, int right, double* X, long ldx, int line0, int nlines, int origin,
                            int width, int nrefl, const double* wy, long stride) {
  SweepBatch b{};
  b.wy = wy; b.stride = stride; b.mode = 4; b.t0 = 0; b.t1 = 1;
  b.ex_off = 0; b.ex_width = width; b.ex_nrefl = nrefl;
  const HtSweepJob j{X, ldx, right, line0, nlines, origin, 0, 0};
  return launch_batch(st, b, &j, 1);
}

cudaError_t ht_launch_rankk_right(cudaStream_t st, double* X, long ldx, int nrows, int c1, int c2, int k,
                                  const double* V1, int ldv1, const double* L1, int ldl1, const double* T, int ldt) {
  if (nrows <= 0) return cudaSuccess;
  rankk_right_kernel<<<(nrows + SRK - 1) / SRK, HT_THREADS, 0, st>>>(X, ldx, nrows, c1, k, c2, k, V1, ldv1, L1, ldl1, T,
                                                                    ldt);
  return cudaGetLastError();
}

cudaError_t ht_rankk_right_w(cudaStream_t st, double* X, long ldx, int nrows, int c1, int w1, int k,
                             const double* V1, int ldv1, const double* T, int ldt) {
  if (nrows <= 0) return cudaSuccess;
  rankk_right_kernel<<<(nrows + SRK - 1) / SRK, HT_THREADS, 0, st>>>(X, ldx, nrows, c1, w1, -1, k, V1, ldv1, nullptr, 0,
                                                                    T, ldt);
  return cudaGetLastError();
}

cudaError_t ht_rankk_left(cudaStream_t st, double* X, long ldx, int col0, int ncols, int r0, int w1, int k,
                          const double* Ut, int ldu, const double* S, int lds) {
  if (ncols <= 0) return cudaSuccess;
  rankk_left_kernel<<<(ncols + SRK - 1) / SRK, HT_THREADS, 0, st>>>(X, ldx, col0, ncols, r0, w1, k, Ut, ldu, S, lds);
  return cudaGetLastError();
}

cudaError_t ht_launch_zero(cudaStream_t st, double* X, long ldx, int rows, int cols, int lower_only) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  zero_kernel<<<grid_for((long)rows * cols, 256), 256, 0, st>>>(X, ldx, rows, cols, lower_only);
  return cudaGetLastError();
}

cudaError_t ht_launch_set_identity(cudaStream_t st, double* X, long ldx, int n) {
  if (n <= 0) return cudaSuccess;
  identity_kernel<<<grid_for((long)n * n, 256), 256, 0, st>>>(X, ldx, n);
  return cudaGetLastError();
}

cudaError_t ht_launch_check_finite(cudaStream_t st, const double* X, long ldx, int n, int upper_only, int* err) {
  if (n <= 0) return cudaSuccess;
  finite_kernel<<<grid_for((long)n * n, 256), 256, 0, st>>>(X, ldx, n, upper_only, err);
  return cudaGetLastError();
}
