// Small Householder factorizations of the absorption (Sec. 3.3): the QL chain
// that reduces V2 to L-hat (eq. (5)), the QR chain that reduces U2 to R-tilde
// (eq. (7)), and the RQ / QR factorizations of the blocks of B in the restore
// chains (Sec. 3.3.1e, 3.3.2f).  Each factorization runs on one CTA with the
// block in shared memory and returns its orthogonal factor in regular WY form
// G = I - Vw Ww^T, Ww = Vw T^T, with T grown by the rule of eq. (1)
// (T <- [T, -tau T Vw^T v; 0, tau]) over the reflectors in product order.
//
// An RQ factorization X G = [0 R1] of a k x w block is the QL factorization
// of X^T: X^T = G [0; R1^T].
#include "ht_common.cuh"

namespace {

constexpr int MAXW = 2 * HT_NB_MAX;  // largest window height

// Householder QR (lower=false) or QL (lower=true) of the w x kk column-major
// matrix X (shared, ld w) in place.  On return X holds R (QR: upper triangle
// in rows 0..kk-1) or L (QL: lower triangle in rows w-kk..w-1) with exact zeros
// elsewhere, Vs (shared, w x kk) the reflector vectors in product order and
// tau[q] their coefficients.
__device__ void house_factor(double* X, int w, int kk, bool ql, double* Vs, double* tau, double* red) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < w * kk; e += blockDim.x) Vs[e] = 0.0;
  __syncthreads();
  for (int q = 0; q < kk; ++q) {
    // column c and pivot row t of this reflector
    const int c = ql ? (kk - 1 - q) : q;
    const int t = ql ? (w - kk + c) : c;
    // rows of the reflector: QR [t, w), QL [0, t]
    const int lo = ql ? 0 : t, hi = ql ? t + 1 : w;
    double tail = 0.0;
    if (wid == 0) {
      for (int r = lo + lane; r < hi; r += 32)
        if (r != t) tail += X[r + c * w] * X[r + c * w];
      tail = ht_warp_sum(tail);
      if (lane == 0) {
        const double x0 = X[t + c * w];
        double beta, alpha, scal;
        if (tail == 0.0) {
          beta = 0.0; alpha = x0; scal = 0.0;
        } else {
          const double nrm = sqrt(x0 * x0 + tail);
          alpha = (x0 >= 0.0) ? -nrm : nrm;
          beta = (alpha - x0) / alpha;
          scal = 1.0 / (x0 - alpha);
        }
        red[0] = beta; red[1] = alpha; red[2] = scal;
      }
    }
    __syncthreads();
    const double beta = red[0], alpha = red[1], scal = red[2];
    // reflector vector into Vs(:, q)
    for (int r = lo + tid; r < hi; r += blockDim.x) Vs[r + q * w] = (r == t) ? 1.0 : X[r + c * w] * scal;
    __syncthreads();
    // apply to the other columns still to be reduced: QR columns c+1..kk-1,
    // QL columns 0..c-1 (rows [lo, hi))
    if (beta != 0.0) {
      const int cb = ql ? 0 : c + 1, ce = ql ? c : kk;
      for (int cc = cb + wid; cc < ce; cc += nw) {
        double d = 0.0;
        for (int r = lo + lane; r < hi; r += 32) d += Vs[r + q * w] * X[r + cc * w];
        d = ht_warp_sum(d) * beta;
        for (int r = lo + lane; r < hi; r += 32) X[r + cc * w] -= d * Vs[r + q * w];
      }
    }
    __syncthreads();
    for (int r = lo + tid; r < hi; r += blockDim.x) X[r + c * w] = (r == t) ? alpha : 0.0;
    if (tid == 0) tau[q] = beta;
    __syncthreads();
  }
}

// T (kk x kk, upper, ld kk) of G = H_0 H_1 ... = I - Vs T Vs^T by the growth
// rule of eq. (1), then Ww = Vs T^T (w x kk).  G_ = Vs^T Vs is scratch.
__device__ void form_wy(const double* Vs, const double* tau, int w, int kk, double* Tm, double* Gm, double* Ww) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kk * kk; e += blockDim.x) {
    const int a = e % kk, b = e / kk;
    double d = 0.0;
    if (a < b)
      for (int r = 0; r < w; ++r) d += Vs[r + a * w] * Vs[r + b * w];
    Gm[e] = d;
    Tm[e] = 0.0;
  }
  __syncthreads();
  for (int q = 0; q < kk; ++q) {
    // T(0:q, q) = -tau_q T(0:q, 0:q) (Vs^T v_q)(0:q)
    for (int i = tid; i < q; i += blockDim.x) {
      double d = 0.0;
      for (int l = i; l < q; ++l) d += Tm[i + l * kk] * Gm[l + q * kk];
      Tm[i + q * kk] = -tau[q] * d;
    }
    if (tid == 0) Tm[q + q * kk] = tau[q];
    __syncthreads();
  }
  for (int e = tid; e < w * kk; e += blockDim.x) {
    const int r = e % w, i = e / w;
    double d = 0.0;
    for (int l = i; l < kk; ++l) d += Vs[r + l * w] * Tm[i + l * kk];
    Ww[e] = d;
  }
  __syncthreads();
}

// shared layout: X (MAXW*HT_NB_MAX), Vs (same), Tm, Gm (HT_NB_MAX^2 each), tau, red
__host__ __device__ inline size_t factor_smem_doubles() {
  return 2 * (size_t)MAXW * HT_NB_MAX + 2 * (size_t)HT_NB_MAX * HT_NB_MAX + HT_NB_MAX + 32;
}

// Factor one w x kk window (QR or QL) whose rows are X0[r0 + r] (global, ld),
// write the reduced window back, and store Vw, Ww at wy.
__device__ void factor_window(double* Xg, long ld, int r0, int w, int kk, bool ql, double* wy, size_t stride,
                              double* sm) {
  double* X = sm;
  double* Vs = X + MAXW * HT_NB_MAX;
  double* Tm = Vs + MAXW * HT_NB_MAX;
  double* Gm = Tm + HT_NB_MAX * HT_NB_MAX;
  double* tau = Gm + HT_NB_MAX * HT_NB_MAX;
  double* red = tau + HT_NB_MAX;
  for (int e = threadIdx.x; e < w * kk; e += blockDim.x) {
    const int r = e % w, c = e / w;
    X[e] = Xg[(size_t)(r0 + r) + (size_t)c * ld];
  }
  __syncthreads();
  house_factor(X, w, kk, ql, Vs, tau, red);
  double* Vw = wy;
  double* Ww = wy + ht_wy_half(stride);
  form_wy(Vs, tau, w, kk, Tm, Gm, Ww);
  for (int e = threadIdx.x; e < w * kk; e += blockDim.x) {
    const int r = e % w, c = e / w;
    Xg[(size_t)(r0 + r) + (size_t)c * ld] = X[e];
    Vw[e] = Vs[e];
  }
  __syncthreads();
}

// mode 0: QL chain on V2 (p x k) top to bottom, L-hat_1 -> tri (k x k, ld k)
// mode 1: QR chain on U2 (p x k) bottom to top, R-tilde_1 -> tri
__global__ void __launch_bounds__(HT_THREADS) factor_chain_kernel(int mode, double* X, long ld, int p, int k,
                                                                   double* wy, size_t stride, double* tri) {
  extern __shared__ double sm[];
  const int nwin = ht_num_windows(p, k);
  for (int i = 0; i < nwin; ++i) {
    int r0, r1;
    if (mode == 0) ht_ql_window(p, k, i, &r0, &r1);
    else ht_qr_window(p, k, i, &r0, &r1);
    factor_window(X, ld, r0, r1 - r0, k, mode == 0, wy + (size_t)i * stride, stride, sm);
  }
  // triangular factor: QL -> bottom k rows, QR -> top k rows
  const int tr0 = (mode == 0) ? p - k : 0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int r = e % k, c = e / k;
    tri[e] = X[(size_t)(tr0 + r) + (size_t)c * ld];
  }
}

// mode 2: RQ of a rows x cols block of B (rows <= cols) in place -> [0 R1]
// mode 3: QR of a rows x cols block (rows >= cols) in place -> [R; 0]
__global__ void __launch_bounds__(HT_THREADS) factor_block_kernel(int mode, double* Xg, long ld, int rows, int cols,
                                                                   double* wy, size_t stride) {
  extern __shared__ double sm[];
  double* X = sm;
  double* Vs = X + MAXW * HT_NB_MAX;
  double* Tm = Vs + MAXW * HT_NB_MAX;
  double* Gm = Tm + HT_NB_MAX * HT_NB_MAX;
  double* tau = Gm + HT_NB_MAX * HT_NB_MAX;
  double* red = tau + HT_NB_MAX;
  // work on the w x kk matrix: QR -> the block itself; RQ -> its transpose
  const bool rq = (mode == 2);
  const int w = rq ? cols : rows, kk = rq ? rows : cols;
  for (int e = threadIdx.x; e < w * kk; e += blockDim.x) {
    const int r = e % w, c = e / w;
    X[e] = rq ? Xg[(size_t)c + (size_t)r * ld] : Xg[(size_t)r + (size_t)c * ld];
  }
  __syncthreads();
  house_factor(X, w, kk, rq, Vs, tau, red);
  double* Ww = wy + ht_wy_half(stride);
  form_wy(Vs, tau, w, kk, Tm, Gm, Ww);
  for (int e = threadIdx.x; e < w * kk; e += blockDim.x) {
    const int r = e % w, c = e / w;
    if (rq) Xg[(size_t)c + (size_t)r * ld] = X[e];
    else Xg[(size_t)r + (size_t)c * ld] = X[e];
    wy[e] = Vs[e];
  }
}

}  // namespace

static int g_factor_attr = 0;
static void set_factor_attr() {
  if (g_factor_attr) return;
  const int bytes = (int)(factor_smem_doubles() * sizeof(double));
  cudaFuncSetAttribute(factor_chain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(factor_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  g_factor_attr = 1;
}

cudaError_t ht_launch_factor_chain(cudaStream_t st, int mode, double* X, int ldx, int p, int k, double* wy,
                                   size_t stride, double* out_tri) {
  set_factor_attr();
  factor_chain_kernel<<<1, HT_THREADS, factor_smem_doubles() * sizeof(double), st>>>(mode, X, ldx, p, k, wy, stride,
                                                                                     out_tri);
  return cudaGetLastError();
}

cudaError_t ht_launch_factor_block(cudaStream_t st, int mode, double* X, int ldx, int rows, int cols, double* wy,
                                   size_t stride) {
  set_factor_attr();
  factor_block_kernel<<<1, HT_THREADS, factor_smem_doubles() * sizeof(double), st>>>(mode, X, ldx, rows, cols, wy,
                                                                                     stride);
  return cudaGetLastError();
}
