// Front ends of the HT reduction that need a dense Householder QR:
//
//  * the QZ front end (Sec. 1): a pencil with a general B is brought to the
//    problem statement of Algorithm 1 by B = Q_B R, A <- Q_B^T A, Q <- Q_B;
//  * the preprocessing of Sec. 3.4.1: with l > 1 zero columns in the upper
//    triangular B, a permutation Z_0 moves them to the front (Q_0 = Z_0 when B
//    is diagonal, else I), a QR of the first l columns of Q_0^T A Z_0 makes
//    them upper triangular (those l eigenvalues are infinite and already in
//    generalized Schur form), and only the trailing pencil is reduced.
//
// The QR is blocked: panels of QB columns are factored by one CTA (DLARFG
// rule, Sec. 2.1), each panel's compact WY factor T (H_0 H_1 ... = I - V T V^T,
// eq. (1)) is formed from the Gram matrix V^T V, and the trailing columns, the
// other matrices transformed from the left and the accumulated Q are updated by
// FP64 GEMMs (ht_gemm).  These run once per call, before the reduction.
#include <algorithm>

#include "ht_common.cuh"

namespace {

constexpr int QB = 32;        // panel width
constexpr int QTHREADS = 512;

// Householder QR of the m x kb panel P (ld ldp) in place: R on and above the
// diagonal, exact zeros below; the reflectors (v(q) = 1, zeros above) to Vb
// (m x kb, ld ldv) and their coefficients to tau.
__global__ void __launch_bounds__(QTHREADS) qr_panel_kernel(int m, int kb, double* P, long ldp, double* Vb, int ldv,
                                                            double* tau) {
  __shared__ double red[QTHREADS / 32][QB + 1];
  __shared__ double sc[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < kb; ++q) {
    double* pq = P + (size_t)q * ldp;
    // ---- tail norm of column q, rows q+1 .. m-1 ----
    double s = 0.0;
    for (int r = q + 1 + tid; r < m; r += blockDim.x) s += pq[r] * pq[r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[wid][0] = s;
    __syncthreads();
    if (tid == 0) {
      double tail = 0.0;
      for (int w = 0; w < nw; ++w) tail += red[w][0];
      const double x0 = pq[q];
      double beta = 0.0, alpha = x0, scal = 0.0;
      if (tail != 0.0) {
        const double nrm = sqrt(x0 * x0 + tail);
        alpha = (x0 >= 0.0) ? -nrm : nrm;
        beta = (alpha - x0) / alpha;
        scal = 1.0 / (x0 - alpha);
      }
      sc[0] = beta; sc[1] = alpha; sc[2] = scal;
      tau[q] = beta;
    }
    __syncthreads();
    const double beta = sc[0], alpha = sc[1], scal = sc[2];
    double* vq = Vb + (size_t)q * ldv;
    for (int r = tid; r < m; r += blockDim.x) vq[r] = (r < q) ? 0.0 : (r == q ? 1.0 : pq[r] * scal);
    __syncthreads();
    // ---- the reflector on columns q+1 .. kb-1 of the panel ----
    const int nc = kb - q - 1;
    if (nc > 0 && beta != 0.0) {
      double acc[QB];
#pragma unroll
      for (int c = 0; c < QB; ++c) acc[c] = 0.0;
      for (int r = q + tid; r < m; r += blockDim.x) {
        const double v = vq[r];
#pragma unroll
        for (int c = 0; c < QB; ++c)
          if (c < nc) acc[c] += v * P[r + (size_t)(q + 1 + c) * ldp];
      }
#pragma unroll
      for (int c = 0; c < QB; ++c) {
        double a = acc[c];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0 && c < nc) red[wid][c] = a;
      }
      __syncthreads();
      if (tid < nc) {
        double d = 0.0;
        for (int w = 0; w < nw; ++w) d += red[w][tid];
        red[0][tid] = beta * d;
      }
      __syncthreads();
      for (int e = tid; e < nc * (m - q); e += blockDim.x) {
        const int c = e / (m - q), r = q + e % (m - q);
        P[r + (size_t)(q + 1 + c) * ldp] -= red[0][c] * vq[r];
      }
      __syncthreads();
    }
    // ---- column q: alpha on the diagonal, exact zeros below ----
    for (int r = q + tid; r < m; r += blockDim.x) pq[r] = (r == q) ? alpha : 0.0;
    __syncthreads();
  }
}

// T (kb x kb upper, ld kb) of H_0 ... H_{kb-1} = I - V T V^T from G = V^T V:
// T(i,i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) G(0:i, i) (eq. (1) column by column).
__global__ void qr_tfac_kernel(int kb, const double* G, const double* tau, double* T) {
  const int j = threadIdx.x;  // one lane per row of T
  for (int e = j; e < kb * kb; e += blockDim.x) T[e] = 0.0;
  __syncwarp();
  for (int i = 0; i < kb; ++i) {
    double t = 0.0;
    if (j < i)
      for (int l = j; l < i; ++l) t += T[j + l * kb] * G[l + i * kb];
    __syncwarp();
    if (j < i) T[j + i * kb] = -tau[i] * t;
    if (j == i) T[i + i * kb] = tau[i];
    __syncwarp();
  }
}

// per column c of the upper triangle of B (one warp a column): zc[c] = 1 when
// B(0:c, c) is zero; *offdiag = 1 when some B(r, c), r < c, is not zero
__global__ void zero_columns_kernel(int n, const double* B, long ldb, int* zc, int* offdiag) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= n) return;
  const double* bc = B + (size_t)c * ldb;
  bool nz = false, off = false;
  for (int r = lane; r <= c; r += 32) {
    const bool z = bc[r] == 0.0;
    nz |= !z;
    off |= (!z && r < c);
  }
  nz = __any_sync(0xffffffffu, nz);
  off = __any_sync(0xffffffffu, off);
  if (lane == 0) {
    zc[c] = nz ? 0 : 1;
    if (off) atomicOr(offdiag, 1);
  }
}

// Y(r, i) = X(rows ? p[r] : r, p[i]) (n x n, Y with ld n)
__global__ void permute_kernel(int n, const double* X, long ldx, double* Y, const int* p, int rows) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int r = (int)(e % n), i = (int)(e / n);
  Y[e] = X[(size_t)(rows ? p[r] : r) + (size_t)p[i] * ldx];
}

// X = the permutation matrix with X(p[i], i) = 1
__global__ void perm_matrix_kernel(int n, double* X, long ldx, const int* p) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)n * n) return;
  const int r = (int)(e % n), i = (int)(e / n);
  X[r + (size_t)i * ldx] = (r == p[i]) ? 1.0 : 0.0;
}

// ---- a-posteriori check of a reduction by Gaussian probes ----
// X (n x np): N(0,1) samples from a counter hash (SplitMix64) and Box-Muller;
// the probes only need to be independent of the data
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void gauss_kernel(size_t count, double* X, unsigned long long seed) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const unsigned long long a = splitmix64(seed ^ (2 * e)), b = splitmix64(seed ^ (2 * e + 1));
  const double u1 = ((a >> 11) + 1) * 0x1.0p-53, u2 = (b >> 11) * 0x1.0p-53;
  X[e] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}
// acc[slot] += sum over the m x c block (ld) of (X - Y)^2 (Y null: X^2)
__global__ void sumsq_kernel(int m, int c, const double* X, long ldx, const double* Y, long ldy, double* acc) {
  __shared__ double red[8];
  double s = 0.0;
  const size_t tot = (size_t)m * c;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e % m, j = e / m;
    const double d = X[r + j * ldx] - (Y ? Y[r + j * ldy] : 0.0);
    s += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(acc, t);
  }
}

}  // namespace

cudaError_t ht_launch_gauss(cudaStream_t st, size_t count, double* X, unsigned long long seed) {
  if (count == 0) return cudaSuccess;
  gauss_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, X, seed);
  return cudaGetLastError();
}

cudaError_t ht_launch_sumsq(cudaStream_t st, int m, int c, const double* X, long ldx, const double* Y, long ldy,
                            double* acc) {
  if (m <= 0 || c <= 0) return cudaSuccess;
  sumsq_kernel<<<304, 256, 0, st>>>(m, c, X, ldx, Y, ldy, acc);
  return cudaGetLastError();
}

size_t ht_qr_ws_doubles(int m, int nx, int nq) {
  const size_t w = (size_t)std::max(nx, 1);
  return (size_t)m * QB + QB + 2 * (size_t)QB * QB + 2 * QB * w + 2 * (size_t)std::max(nq, 1) * QB;
}

cudaError_t ht_qr_blocked(cudaStream_t st, int m, int nc, double* M, long ldm, const HtQrTarget* left, int nleft,
                          double* Qm, long ldq, int nq, double* ws) {
  if (m <= 0 || nc <= 0) return cudaSuccess;
  int nxmax = nc;
  for (int t = 0; t < nleft; ++t) nxmax = std::max(nxmax, left[t].ncols);
  double* Vb = ws;
  double* tau = Vb + (size_t)m * QB;
  double* G = tau + QB;
  double* T = G + QB * QB;
  double* W = T + QB * QB;
  double* W2 = W + (size_t)QB * nxmax;
  double* Wq = W2 + (size_t)QB * nxmax;
  double* Wq2 = Wq + (size_t)std::max(nq, 1) * QB;
  cudaError_t e = cudaSuccess;
  // apply (H_r ... )^T = I - V T^T V^T from the left to the mr x nx block X (ld ldx)
  auto left_apply = [&](int mr, int kb, double* X, long ldx, int nx) -> cudaError_t {
    if (nx <= 0) return cudaSuccess;
    cudaError_t r = ht_gemm(st, 'T', 'N', kb, nx, mr, 1.0, Vb, mr, X, (int)ldx, 0.0, W, kb);
    if (r == cudaSuccess) r = ht_gemm(st, 'T', 'N', kb, nx, kb, 1.0, T, kb, W, kb, 0.0, W2, kb);
    if (r == cudaSuccess) r = ht_gemm(st, 'N', 'N', mr, nx, kb, -1.0, Vb, mr, W2, kb, 1.0, X, (int)ldx);
    return r;
  };
  const int npanel = std::min(m, nc);
  for (int r0 = 0; r0 < npanel; r0 += QB) {
    const int kb = std::min(QB, npanel - r0), mr = m - r0;
    double* P = M + (size_t)r0 + (size_t)r0 * ldm;
    qr_panel_kernel<<<1, QTHREADS, 0, st>>>(mr, kb, P, ldm, Vb, mr, tau);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = ht_gemm(st, 'T', 'N', kb, kb, mr, 1.0, Vb, mr, Vb, mr, 0.0, G, kb)) != cudaSuccess) return e;
    qr_tfac_kernel<<<1, 32, 0, st>>>(kb, G, tau, T);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the trailing columns of M and the left targets (their rows r0 .. m-1)
    if ((e = left_apply(mr, kb, M + (size_t)r0 + (size_t)(r0 + kb) * ldm, ldm, nc - r0 - kb)) != cudaSuccess) return e;
    for (int t = 0; t < nleft; ++t)
      if ((e = left_apply(mr, kb, left[t].X + (size_t)r0, left[t].ld, left[t].ncols)) != cudaSuccess) return e;
    // Qm(:, r0:m) <- Qm(:, r0:m) (I - V T V^T)
    if (Qm && nq > 0) {
      double* Qr = Qm + (size_t)r0 * ldq;
      if ((e = ht_gemm(st, 'N', 'N', nq, kb, mr, 1.0, Qr, (int)ldq, Vb, mr, 0.0, Wq, nq)) != cudaSuccess) return e;
      if ((e = ht_gemm(st, 'N', 'N', nq, kb, kb, 1.0, Wq, nq, T, kb, 0.0, Wq2, nq)) != cudaSuccess) return e;
      if ((e = ht_gemm(st, 'N', 'T', nq, mr, kb, -1.0, Wq2, nq, Vb, mr, 1.0, Qr, (int)ldq)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t ht_launch_zero_columns(cudaStream_t st, int n, const double* B, long ldb, int* zc, int* offdiag) {
  cudaError_t e = cudaMemsetAsync(offdiag, 0, sizeof(int), st);
  if (e != cudaSuccess || n <= 0) return e;
  zero_columns_kernel<<<(n + 7) / 8, 256, 0, st>>>(n, B, ldb, zc, offdiag);
  return cudaGetLastError();
}

cudaError_t ht_launch_permute(cudaStream_t st, int n, double* X, long ldx, double* tmp, const int* p, int rows) {
  if (n <= 0) return cudaSuccess;
  const size_t nn = (size_t)n * n;
  permute_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, X, ldx, tmp, p, rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpy2DAsync(X, ldx * sizeof(double), tmp, n * sizeof(double), n * sizeof(double), n,
                           cudaMemcpyDeviceToDevice, st);
}

cudaError_t ht_launch_perm_matrix(cudaStream_t st, int n, double* X, long ldx, const int* p) {
  if (n <= 0) return cudaSuccess;
  const size_t nn = (size_t)n * n;
  perm_matrix_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(n, X, ldx, p);
  return cudaGetLastError();
}
