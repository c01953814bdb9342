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

struct SweepArgs {
  double* X;
  long ldx;
  int nlines;      // rows (right) or columns (left) of X swept
  int origin;      // column (right) or row (left) index of window offset 0
  const double* wy;
  int mode, p, k, t0, t1;
  int use_limit;   // 1: skip stripes the structural limit says are zero
  int limit_base;  // added to the window limit
  int line0;       // first row (right) / column (left) of the swept range
  int ex_off, ex_width, ex_nrefl;  // mode 4
  long stride;     // doubles between consecutive windows of the WY store (Ww at stride / 2)
};

// Right application: rows [line0 + stripe*SR, ...) of X, X(:, c) <- X(:, c) G.
// The stripe sits in shared memory column-major (Xs[r + c * SR]) so that the
// lanes of a warp, which take consecutive rows, hit distinct banks; Vw and Ww
// entries are warp-uniform (broadcast loads through L1).
__global__ void __launch_bounds__(HT_THREADS) sweep_right_kernel(SweepArgs a) {
  __shared__ double Xs[SR * MAXW];        // SR x w, ld SR
  __shared__ double Ps[SR * HT_NB_MAX];   // SR x nrefl, ld SR
  const int tid = threadIdx.x;
  const int row_begin = a.line0 + blockIdx.x * SR;
  const int row_end = min(a.line0 + a.nlines, row_begin + SR);
  const int rows = row_end - row_begin;
  if (rows <= 0) return;
  for (int t = a.t0; t < a.t1; ++t) {
    int off, w, kr, lim;
    if (a.mode == 4) { off = a.ex_off; w = a.ex_width; kr = a.ex_nrefl; lim = 0; }
    else win_geom(a.mode, a.p, a.k, t, &off, &w, &kr, &lim);
    if (a.use_limit && row_begin >= a.limit_base + lim) continue;
    const double* Vw = a.wy + (size_t)t * a.stride;
    const double* Ww = Vw + a.stride / 2;
    const int c0 = a.origin + off;
    for (int e = tid; e < SR * w; e += blockDim.x) {
      const int r = e % SR, c = e / SR;
      Xs[r + c * SR] = (r < rows) ? a.X[(size_t)(row_begin + r) + (size_t)(c0 + c) * a.ldx] : 0.0;
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
      a.X[(size_t)(row_begin + r) + (size_t)(c0 + c) * a.ldx] = s0 + s1;
    }
    __syncthreads();
  }
}

// Left application: columns [line0 + stripe*SR, ...) of X, X(rows, c) <- G^T X(rows, c).
// Dynamic shared memory: Xs (w x SR, ld XLD, odd so that lanes taking
// consecutive columns hit distinct banks) and Ps (nrefl x SR, Ps[c + q * SR]).
constexpr int XLD = MAXW + 1;
constexpr size_t SWEEP_LEFT_SMEM = sizeof(double) * ((size_t)XLD * SR + (size_t)HT_NB_MAX * SR);
__global__ void __launch_bounds__(HT_THREADS) sweep_left_kernel(SweepArgs a) {
  extern __shared__ double sl_sm[];
  double* Xs = sl_sm;
  double* Ps = sl_sm + XLD * SR;
  const int tid = threadIdx.x;
  const int col_begin = a.line0 + blockIdx.x * SR;
  const int col_end = min(a.line0 + a.nlines, col_begin + SR);
  const int cols = col_end - col_begin;
  if (cols <= 0) return;
  for (int t = a.t0; t < a.t1; ++t) {
    int off, w, kr, lim;
    if (a.mode == 4) { off = a.ex_off; w = a.ex_width; kr = a.ex_nrefl; lim = 0; }
    else win_geom(a.mode, a.p, a.k, t, &off, &w, &kr, &lim);
    if (a.use_limit && col_end <= a.limit_base + lim) continue;
    const double* Vw = a.wy + (size_t)t * a.stride;
    const double* Ww = Vw + a.stride / 2;
    const int r0 = a.origin + off;
    for (int e = tid; e < w * SR; e += blockDim.x) {
      const int r = e % w, c = e / w;
      Xs[r + c * XLD] = (c < cols) ? a.X[(size_t)(r0 + r) + (size_t)(col_begin + c) * a.ldx] : 0.0;
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
      a.X[(size_t)(r0 + r) + (size_t)(col_begin + c) * a.ldx] = s0 + s1;
    }
    __syncthreads();
  }
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

// The left sweep takes more than the default 48 KB of dynamic shared memory:
// raise its limit once per device.
static cudaError_t sweep_left_attr() {
  static std::mutex mu;
  static unsigned long long done = 0;  // bit d: set on device d
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && (done >> dev) & 1ull) return cudaSuccess;
  e = cudaFuncSetAttribute(sweep_left_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SWEEP_LEFT_SMEM);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

static cudaError_t launch_sweep(cudaStream_t st, bool right, SweepArgs a) {
  if (a.nlines <= 0 || a.t1 <= a.t0) return cudaSuccess;
  const int grid = (a.nlines + SR - 1) / SR;
  if (right) {
    sweep_right_kernel<<<grid, HT_THREADS, 0, st>>>(a);
  } else {
    const cudaError_t e = sweep_left_attr();
    if (e != cudaSuccess) return e;
    sweep_left_kernel<<<grid, HT_THREADS, SWEEP_LEFT_SMEM, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t ht_sweep(cudaStream_t st, int right, double* X, long ldx, int line0, int nlines, int origin,
                     const double* wy, long stride, int mode, int p, int k, int t0, int t1, int use_limit,
                     int limit_base) {
  SweepArgs a{};
  a.X = X; a.ldx = ldx; a.nlines = nlines; a.origin = origin; a.wy = wy; a.stride = stride;
  a.mode = mode; a.p = p; a.k = k; a.t0 = t0; a.t1 = t1;
  a.use_limit = use_limit; a.limit_base = limit_base; a.line0 = line0;
  return launch_sweep(st, right != 0, a);
}

cudaError_t ht_apply_single(cudaStream_t st, int right, double* X, long ldx, int line0, int nlines, int origin,
                            int width, int nrefl, const double* wy, long stride) {
  SweepArgs a{};
  a.X = X; a.ldx = ldx; a.nlines = nlines; a.origin = origin; a.wy = wy; a.stride = stride;
  a.mode = 4; a.p = 0; a.k = 0; a.t0 = 0; a.t1 = 1;
  a.ex_off = 0; a.ex_width = width; a.ex_nrefl = nrefl;
  a.use_limit = 0; a.limit_base = 0; a.line0 = line0;
  return launch_sweep(st, right != 0, a);
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
