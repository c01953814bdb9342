// The QL chain that reduces V2 to L-hat (eq. (5), Sec. 3.3.1b) and the QR
// chain that reduces U2 to R-tilde (eq. (7), Sec. 3.3.2b), as a wavefront over
// the windows of each chain.
//
// A chain is a sequence of Householder factorizations of overlapping windows
// (2k rows, overlap k): window i starts from k rows that window i-1 leaves
// behind (its triangle) and k fresh rows.  Column q of window i-1 is final as
// soon as window i-1 has formed its reflector q (the later reflectors act on
// the other columns only), so reflector q of window i needs only (a) column q
// of window i-1 and (b) the reflectors 0..q-1 of window i.  Window i therefore
// runs one reflector behind window i-1 instead of waiting for all of it: the
// chain takes (windows + k) reflector steps instead of windows x k.
//
// Each window is factored by one CTA in a canonical QR frame (a QL window is
// a QR window with rows and columns reversed).  Column q is brought up to date
// with the window's earlier reflectors in one blocked step,
//     x <- (H_0 ... H_{q-1})^T x = x - Y (W^T x),   W = Y T,
// where T is the triangular factor of eq. (1) and W grows by one column per
// reflector, W(:, q) = beta_q (v_q - W (Y^T v_q)).  The reflector then follows
// the DLARFG rule of Sec. 2.1, and rows 0..k-1 of the finished column are
// published for window i+1 (global memory, then a release flag).
//
// Launch: cooperative, G2 CTAs per chain (the two chains are independent),
// CTA c taking windows c, c + G2, ... in order; a window waits only on the one
// before it, which is processed by a co-resident CTA.  The waits are bounded:
// on expiry HT_ERR_TIMEOUT is raised and the CTA carries on with the data it
// has.  Output per window (as the sequential chain kernel writes it):
// reflector vectors (ld = window height, original row order) and coefficients
// in the WY store, the k x k triangle of the last window in tri.
#include <algorithm>
#include <mutex>

#include "ht_common.cuh"

namespace {

constexpr int CK_MAX = 32;           // reflectors per window
constexpr int CW_MAX = 2 * CK_MAX;   // rows per window
constexpr int CTH = 256;             // threads per CTA
constexpr int LDX = CW_MAX;

struct ChainArgs {
  double* X[2];     // V2 (QL, mode 0) and U2 (QR, mode 1), ld
  long ld;
  int p, k;
  double* wy[2];    // WY stores: window i at wy + i * stride (vectors), + stride / 2 (coefficients)
  size_t stride;
  double* tri[2];   // L-hat_1, R-tilde_1 (k x k, ld k)
  double* pub[2];   // published columns: ((i * k) + q) * k + r
  int* flag[2];     // per window: columns published so far (zeroed by the launcher)
  int G2;           // CTAs per chain
  int* err;
  long spin;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// bounded wait of one thread for *f >= v: gives up at once when the error word
// is set, else after `spin` polls, raising HT_ERR_TIMEOUT
__device__ bool cw_wait(const int* f, int v, int* err, long spin) {
  if (ht_ld_acquire(f) >= v) return true;
  for (long it = 0; it < spin; ++it) {
    if (*(volatile int*)err != 0) return false;
    __nanosleep(32);
    if (ht_ld_acquire(f) >= v) return true;
  }
  atomicCAS(err, 0, HT_ERR_TIMEOUT);
  return false;
}

__global__ void __launch_bounds__(CTH, 1) chain_wave_kernel(ChainArgs a) {
  extern __shared__ double csm[];
  double* X = csm;                    // canonical window, column-major, ld LDX
  double* Y = X + CW_MAX * CK_MAX;    // reflector vectors
  double* W = Y + CW_MAX * CK_MAX;    // W = Y T
  double* tau = W + CW_MAX * CK_MAX;  // CK_MAX
  double* sv = tau + CK_MAX;          // CK_MAX: W^T x, then Y^T v
  double* sc = sv + CK_MAX;           // 4: beta, alpha, scal
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int mode = (int)blockIdx.x < a.G2 ? 0 : 1;
  const int cta = (int)blockIdx.x - mode * a.G2;
  const int p = a.p, k = a.k;
  const int nwin = ht_num_windows(p, k);
  double* Xg = a.X[mode];
  double* pub = a.pub[mode];
  int* flag = a.flag[mode];
  for (int i = cta; i < nwin; i += a.G2) {
    int r0, r1;
    if (mode == 0) ht_ql_window(p, k, i, &r0, &r1);
    else ht_qr_window(p, k, i, &r0, &r1);
    const int w = r1 - r0;
    const int nfresh = (i == 0) ? w : w - k;
    // canonical (rho, col) -> element of Xg: QR as is, QL with rows and columns reversed
    auto gidx = [&](int rho, int col) -> size_t {
      const int r = (mode == 1) ? r0 + rho : r1 - 1 - rho;
      const int cc = (mode == 1) ? col : k - 1 - col;
      return (size_t)r + (size_t)cc * a.ld;
    };
    for (int e = tid; e < LDX * k; e += CTH) {
      const int rho = e % LDX, col = e / LDX;
      X[e] = (rho < nfresh) ? Xg[gidx(rho, col)] : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < k; ++q) {
      double* xq = X + (size_t)q * LDX;
      if (i > 0) {
        // rows w-k..w-1 of column q: rows 0..k-1 of column q of window i-1, once final
        if (tid == 0) cw_wait(flag + (i - 1), q + 1, a.err, a.spin);  // a timeout is reported, work goes on
        __syncthreads();
        if (tid < k) xq[w - k + tid] = __ldcg(pub + ((size_t)(i - 1) * k + q) * k + tid);
        __syncthreads();
      }
      if (q > 0) {
        // sv = W(:, 0:q)^T x: warp wi takes columns j = wi, wi + 8, ... four at a time
        for (int j0 = 4 * warp; j0 < q; j0 += 4 * (CTH / 32)) {
          double d[4] = {0.0, 0.0, 0.0, 0.0};
          for (int rho = lane; rho < w; rho += 32) {
            const double xv = xq[rho];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (j0 + u < q) d[u] += W[rho + (j0 + u) * LDX] * xv;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const double s = warp_sum(d[u]);
            if (lane == 0 && j0 + u < q) sv[j0 + u] = s;
          }
        }
        __syncthreads();
        // x -= Y sv: four threads per row, eight-term partial sums, combined by shuffles
        {
          const int rho = tid >> 2, part = tid & 3;
          double t = 0.0;
          if (rho < w)
            for (int j = part; j < q; j += 4) t += Y[rho + j * LDX] * sv[j];
          t += __shfl_xor_sync(0xffffffffu, t, 1);
          t += __shfl_xor_sync(0xffffffffu, t, 2);
          if (rho < w && part == 0) xq[rho] -= t;
        }
        __syncthreads();
      }
      // reflector q on x[q..w) (DLARFG rule): pivot q, tail q+1..w-1
      if (warp == 0) {
        double t = 0.0;
        for (int rho = q + 1 + lane; rho < w; rho += 32) t += xq[rho] * xq[rho];
        t = warp_sum(t);
        if (lane < 2) {
          const double x0 = xq[q];
          if (t == 0.0) {
            if (lane == 0) { sc[0] = 0.0; sc[1] = x0; sc[2] = 0.0; }
          } else {
            // beta = (alpha - x0) / alpha = 1 + |x0| / ||x||, scal = 1 / (x0 - alpha)
            const double s2 = x0 * x0 + t;
            const double r = rsqrt(s2);
            const double nr = s2 * r;
            const double alpha = (x0 >= 0.0) ? -nr : nr;
            if (lane == 0) { sc[0] = fma(fabs(x0), r, 1.0); sc[1] = alpha; }
            else sc[2] = 1.0 / (x0 - alpha);
          }
        }
      }
      __syncthreads();
      const double beta = sc[0], alpha = sc[1], scal = sc[2];
      double* yq = Y + (size_t)q * LDX;
      for (int rho = tid; rho < LDX; rho += CTH) {
        const double xv = xq[rho];
        yq[rho] = (rho < q || rho >= w) ? 0.0 : (rho == q ? 1.0 : xv * scal);
        xq[rho] = (rho < q) ? xv : (rho == q ? alpha : 0.0);
      }
      if (tid == 0) tau[q] = beta;
      __syncthreads();
      // publish rows 0..k-1 of the finished column for window i+1
      if (i + 1 < nwin) {
        if (tid < k) pub[((size_t)i * k + q) * k + tid] = xq[tid];
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          ht_st_release(flag + i, q + 1);
        }
      }
      // W(:, q) = beta (v - W (Y^T v))
      if (q > 0) {
        for (int j0 = 4 * warp; j0 < q; j0 += 4 * (CTH / 32)) {
          double d[4] = {0.0, 0.0, 0.0, 0.0};
          for (int rho = q + lane; rho < w; rho += 32) {
            const double vv = yq[rho];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (j0 + u < q) d[u] += Y[rho + (j0 + u) * LDX] * vv;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const double s = warp_sum(d[u]);
            if (lane == 0 && j0 + u < q) sv[j0 + u] = s;
          }
        }
        __syncthreads();
        {
          const int rho = tid >> 2, part = tid & 3;
          double t = 0.0;
          if (rho < w)
            for (int j = part; j < q; j += 4) t += W[rho + j * LDX] * sv[j];
          t += __shfl_xor_sync(0xffffffffu, t, 1);
          t += __shfl_xor_sync(0xffffffffu, t, 2);
          if (rho < LDX && part == 0) W[rho + q * LDX] = (rho < w) ? beta * (yq[rho] - t) : 0.0;
        }
      } else {
        for (int rho = tid; rho < LDX; rho += CTH) W[rho] = (rho < w) ? beta * yq[rho] : 0.0;
      }
      __syncthreads();
    }
    // reflector vectors (original row order, ld w) and coefficients to the WY store
    double* Vw = a.wy[mode] + (size_t)i * a.stride;
    double* tw = Vw + a.stride / 2;
    for (int e = tid; e < w * k; e += CTH) {
      const int r = e % w, q = e / w;
      const int rho = (mode == 1) ? r : w - 1 - r;
      Vw[e] = Y[rho + q * LDX];
    }
    for (int q = tid; q < k; q += CTH) tw[q] = tau[q];
    if (i == nwin - 1) {
      // the triangle left by the chain: R-tilde_1 (top k rows) or L-hat_1 (bottom k rows)
      double* tri = a.tri[mode];
      for (int e = tid; e < k * k; e += CTH) {
        const int r = e % k, c = e / k;
        tri[e] = (mode == 1) ? X[r + c * LDX] : X[(k - 1 - r) + (k - 1 - c) * LDX];
      }
    }
    __syncthreads();
  }
}

constexpr int CHAIN_SMEM = (3 * CW_MAX * CK_MAX + 2 * CK_MAX + 8) * (int)sizeof(double);

}  // namespace

// Both chains in one cooperative launch (k <= 32); pub: two buffers of p k
// doubles, flags: two arrays of nwin ints.
cudaError_t ht_launch_chains_wave(cudaStream_t st, double* V2, double* U2, long ld, int p, int k, double* wyR,
                                  double* wyL, size_t stride, double* L1, double* R1, double* pubR, double* pubL,
                                  int* flags, int* err, long spin, int max_ctas) {
  if (k < 1 || k > CK_MAX) return cudaErrorNotSupported;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    static std::mutex mu;
    static unsigned long long done = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 64 || !((done >> dev) & 1ull)) {
      e = cudaFuncSetAttribute(chain_wave_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CHAIN_SMEM);
      if (e != cudaSuccess) return e;
      if (dev < 64) done |= 1ull << dev;
    }
  }
  const int nwin = ht_num_windows(p, k);
  e = cudaMemsetAsync(flags, 0, 2 * (size_t)nwin * sizeof(int), st);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int G2 = std::max(1, std::min(sms / 2, nwin));
  if (max_ctas >= 2) G2 = std::min(G2, max_ctas / 2);
  ChainArgs a;
  a.X[0] = V2; a.X[1] = U2; a.ld = ld; a.p = p; a.k = k;
  a.wy[0] = wyR; a.wy[1] = wyL; a.stride = stride;
  a.tri[0] = L1; a.tri[1] = R1;
  a.pub[0] = pubR; a.pub[1] = pubL;
  a.flag[0] = flags; a.flag[1] = flags + nwin;
  a.G2 = G2; a.err = err; a.spin = spin > 0 ? spin : HT_SPIN_LIMIT;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((void*)chain_wave_kernel, dim3(2 * G2), dim3(CTH), args, CHAIN_SMEM, st);
  if (e != cudaSuccess) return e;
  return ht_launch_form_wy(st, wyR, wyL, stride, p, k);
}
