// C ABI of libht: Algorithm 1 (HouseHT) of Bujanovic, Karlsson, Kressner
// (arXiv 1710.08538) driven from the host.  Per panel: one cooperative
// launch reduces up to nb columns (Sec. 3.2) and reports how many reflector
// pairs it produced (fewer on an IR failure); the host then queues the
// absorption of Sec. 3.3 (right reflectors, then left reflectors) and moves
// the panel start s by k.  The only host/device synchronisation is the read
// of that count, once per panel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ht_common.cuh"

namespace {

thread_local int t_last_status = HT_OK;

#define HT_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) {                           \
      std::fprintf(stderr, "libht: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return HT_ERR_CUDA;                              \
    }                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// Workspace pool (keyed by device, order and panel width)
// ---------------------------------------------------------------------------
struct PoolEntry {
  int dev, n, nb;
  bool busy;
  HtWork w;
  void* base;
  PanelStatus* host_status;  // pinned
};
std::mutex g_pool_mu;
std::vector<PoolEntry*> g_pool;

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

int alloc_work(PoolEntry* e, int n, int nb) {
  HtWork& w = e->w;
  std::memset(&w, 0, sizeof(w));
  w.n = n;
  w.nb = nb;
  w.G = ht_panel_max_ctas(nb);
  w.ychunks = 4;
  const int nblk = n / HT_TRSV_BS + 2;
  const size_t nn = (size_t)n;
  size_t total = 0;
  auto take = [&](size_t doubles) { size_t off = total; total += align_up(doubles * sizeof(double)); return off; };
  const size_t oU = take(nn * nb), oV = take(nn * nb), oY = take(nn * nb);
  const size_t oS = take((size_t)nb * nb), oT = take((size_t)nb * nb);
  const size_t oVec = take(nn * HT_NVEC);
  const size_t oPart = take((size_t)2 * w.G * HT_PART_STRIDE);
  const size_t oYp = take((size_t)w.ychunks * nn);
  const size_t oInvd = take(nn);
  const size_t oBn = take(4);
  // a chain with k reflectors has at most p/k + 2 windows of 4k^2 doubles (Vw, Ww)
  w.wy_cap = 4 * nn * nb + 16 * (size_t)nb * nb;
  const size_t oWy = take(4 * w.wy_cap);
  const size_t oL1 = take((size_t)HT_NB_MAX * HT_NB_MAX), oR1 = take((size_t)HT_NB_MAX * HT_NB_MAX);
  const size_t oT1 = take(nn * 2 * nb), oT2 = take(nn * 2 * nb), oT3 = take(nn * 2 * nb);
  const size_t oSmall = take((size_t)4 * 2 * HT_NB_MAX * HT_NB_MAX);
  const size_t oFlags = take((size_t)nblk);  // ints, over-allocated as doubles
  const size_t oExps = take((size_t)nblk);
  const size_t oMisc = take(16);
  void* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) return HT_ERR_NOMEM;
  cudaMemset(base, 0, total);
  char* b = (char*)base;
  w.U = (double*)(b + oU); w.V = (double*)(b + oV); w.Y = (double*)(b + oY);
  w.S = (double*)(b + oS); w.T = (double*)(b + oT);
  w.vec = (double*)(b + oVec);
  w.part = (double*)(b + oPart);
  w.ypart = (double*)(b + oYp);
  w.invd = (double*)(b + oInvd);
  w.bnorm = (double*)(b + oBn);
  w.wyR = (double*)(b + oWy);
  w.wyL = w.wyR + w.wy_cap;
  w.wyRR = w.wyL + w.wy_cap;
  w.wyLR = w.wyRR + w.wy_cap;
  w.L1 = (double*)(b + oL1); w.R1 = (double*)(b + oR1);
  w.tmp1 = (double*)(b + oT1); w.tmp2 = (double*)(b + oT2); w.tmp3 = (double*)(b + oT3);
  w.small = (double*)(b + oSmall);
  w.flags = (int*)(b + oFlags);
  w.exps = (int*)(b + oExps);
  char* misc = b + oMisc;
  w.epoch = (unsigned*)misc;
  w.err = (int*)(misc + 16);
  w.status = (PanelStatus*)(misc + 64);
  w.epoch_host = 1;
  e->base = base;
  if (cudaMallocHost((void**)&e->host_status, sizeof(PanelStatus)) != cudaSuccess) {
    cudaFree(base);
    return HT_ERR_NOMEM;
  }
  return HT_OK;
}

PoolEntry* acquire(int n, int nb, int* rc) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (PoolEntry* e : g_pool)
    if (!e->busy && e->dev == dev && e->n == n && e->nb == nb) {
      e->busy = true;
      *rc = HT_OK;
      return e;
    }
  PoolEntry* e = new PoolEntry();
  e->dev = dev; e->n = n; e->nb = nb; e->busy = true;
  *rc = alloc_work(e, n, nb);
  if (*rc != HT_OK) { delete e; return nullptr; }
  g_pool.push_back(e);
  return e;
}

void release(PoolEntry* e) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  e->busy = false;
}

struct Ctx {
  HtWork* w;
  cudaStream_t st;
  int n;
  double *A, *B, *Q, *Z;
  long lda, ldb, ldq, ldz;
  int want_qz;
  double flops;
};

#define CK(call)                         \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

// Absorption of k right and k left reflectors (Sec. 3.3.1 and 3.3.2).
cudaError_t absorb(Ctx& c, int s, int k) {
  HtWork& w = *c.w;
  cudaStream_t st = c.st;
  const int n = c.n, nb = w.nb, j = s + k, p = n - j - 1, m = n - s - 1;
  double *A = c.A, *B = c.B, *Q = c.Q, *Z = c.Z;
  const long lda = c.lda, ldb = c.ldb, ldq = c.ldq, ldz = c.ldz;
  double* U = w.U;  // local rows, ld n
  double* V = w.V;
  const double dn = n;
  const long wst = 4L * k * k;  // WY store stride of this absorption

  // Remark 3.1: rows 0..s of Y = A V T, from the unmodified rows 0..s of A
  CK(ht_gemm(st, 'N', 'N', s + 1, k, m, 1.0, A + (size_t)(s + 1) * lda, lda, V, n, 0.0, w.tmp1, n));
  CK(ht_gemm(st, 'N', 'N', s + 1, k, k, 1.0, w.tmp1, n, w.T, nb, 0.0, w.Y, n));
  c.flops += 2.0 * (s + 1) * k * (m + k);

  // ---- right reflectors, Sec. 3.3.1 ----
  // deferred rows 0..s of the panel columns s+1..j-1, then column j (step e2)
  if (k > 1) CK(ht_gemm(st, 'N', 'T', s + 1, k - 1, k, -1.0, w.Y, n, V, n, 1.0, A + (size_t)(s + 1) * lda, lda));
  CK(ht_gemm(st, 'N', 'T', n, 1, k, -1.0, w.Y, n, V + (k - 1), n, 1.0, A + (size_t)j * lda, lda));
  // (b) V2 = Q^_1 .. Q^_r L^  (eq. (5))
  const int nwr = ht_num_windows(p, k);
  CK(ht_launch_factor_chain(st, 0, V + k, n, p, k, w.wyR, wst, w.L1));
  // (c)-(e) step 1: B, Z, A columns j+1..n-1 times the chain
  CK(ht_sweep(st, 1, B, ldb, 0, n, j + 1, w.wyR, wst, 0, p, k, 0, nwr, 1, j + 1));
  if (c.want_qz) CK(ht_sweep(st, 1, Z, ldz, 0, n, j + 1, w.wyR, wst, 0, p, k, 0, nwr, 0, 0));
  CK(ht_sweep(st, 1, A, lda, 0, n, j + 1, w.wyR, wst, 0, p, k, 0, nwr, 0, 0));
  c.flops += 4.0 * dn * p * k * 2.0 * (c.want_qz ? 3 : 2);
  // (c)/(d) steps 2-4 and (e) step 3
  CK(ht_launch_rankk_right(st, B, ldb, n, s + 1, n - k, k, V, n, w.L1, k, w.T, nb));
  if (c.want_qz) CK(ht_launch_rankk_right(st, Z, ldz, n, s + 1, n - k, k, V, n, w.L1, k, w.T, nb));
  CK(ht_gemm(st, 'N', 'T', n, k, k, -1.0, w.Y, n, w.L1, k, 1.0, A + (size_t)(n - k) * lda, lda));
  c.flops += (c.want_qz ? 2 : 1) * 8.0 * dn * k * k + 2.0 * dn * k * k;
  // partial restore: RQ chain bottom to top (Sec. 3.3.1e)
  const int nbr = ht_num_right_blocks(p, k);
  for (int t = 0; t + 1 < nbr; ++t) {
    const int bb = nbr - 1 - t;
    int c0, c1, d0, d1;
    ht_right_block(p, k, bb - 1, &c0, &c1);
    ht_right_block(p, k, bb, &d0, &d1);
    const int rows = d1 - d0, width = d1 - c0;
    double* blk = B + (size_t)(j + 1 + d0) + (size_t)(j + 1 + c0) * ldb;
    double* wy = w.wyRR + (size_t)t * wst;
    CK(ht_launch_factor_block(st, 2, blk, ldb, rows, width, wy, wst));
    CK(ht_apply_single(st, 1, B, ldb, 0, j + 1 + d0, j + 1 + c0, width, rows, wy, wst));
    c.flops += 4.0 * (j + 1 + d0) * width * rows;
  }
  if (nbr > 1) {
    CK(ht_sweep(st, 1, A, lda, 0, n, j + 1, w.wyRR, wst, 2, p, k, 0, nbr - 1, 0, 0));
    if (c.want_qz) CK(ht_sweep(st, 1, Z, ldz, 0, n, j + 1, w.wyRR, wst, 2, p, k, 0, nbr - 1, 0, 0));
    c.flops += 4.0 * dn * p * k * 2.0 * (c.want_qz ? 2 : 1);
  }

  // ---- left reflectors, Sec. 3.3.2 ----
  // (c) step 1: spike B(s+1:j, s+1:j) -= U1 S^T (U^T B(s+1:n, s+1:j)); step 2 zeros below
  double* sm0 = w.small;
  double* sm1 = w.small + 2 * HT_NB_MAX * HT_NB_MAX;
  double* Bsp = B + (size_t)(s + 1) + (size_t)(s + 1) * ldb;
  CK(ht_gemm(st, 'T', 'N', k, k, m, 1.0, U, n, Bsp, ldb, 0.0, sm0, k));
  CK(ht_gemm(st, 'T', 'N', k, k, k, 1.0, w.S, nb, sm0, k, 0.0, sm1, k));
  CK(ht_gemm(st, 'N', 'N', k, k, k, -1.0, U, n, sm1, k, 1.0, Bsp, ldb));
  CK(ht_launch_zero(st, B + (size_t)(j + 1) + (size_t)(s + 1) * ldb, ldb, p, k, 0));
  CK(ht_launch_zero(st, Bsp, ldb, k, k, 1));
  c.flops += 2.0 * k * k * (m + 2 * k);
  // (b) U2 = Q~_1 .. Q~_r R~ (eq. (7))
  const int nwl = ht_num_windows(p, k);
  CK(ht_launch_factor_chain(st, 1, U + k, n, p, k, w.wyL, wst, w.R1));
  // (c) step 3, (e) step 1, (d) step 1
  CK(ht_sweep(st, 0, B, ldb, j + 1, p, j + 1, w.wyL, wst, 1, p, k, 0, nwl, 1, j + 1));
  CK(ht_sweep(st, 0, A, lda, j, n - j, j + 1, w.wyL, wst, 1, p, k, 0, nwl, 0, 0));
  if (c.want_qz) CK(ht_sweep(st, 1, Q, ldq, 0, n, j + 1, w.wyL, wst, 1, p, k, 0, nwl, 0, 0));
  c.flops += 4.0 * p * k * 2.0 * (0.5 * p + (n - j) + (c.want_qz ? dn : 0.0));
  // U~ = [U1; R~1] (2k x k) in tmp3 with ld 2k
  double* Ut = w.tmp3;
  CK(cudaMemcpy2DAsync(Ut, 2 * k * sizeof(double), U, n * sizeof(double), k * sizeof(double), k,
                       cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpy2DAsync(Ut + k, 2 * k * sizeof(double), w.R1, k * sizeof(double), k * sizeof(double), k,
                       cudaMemcpyDeviceToDevice, st));
  // (c) steps 4-5, (e) steps 2-3, (d) steps 2-3
  CK(ht_rankk_left(st, B, ldb, j + 1, p, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
  CK(ht_rankk_left(st, A, lda, j, n - j, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
  if (c.want_qz) CK(ht_rankk_right_w(st, Q, ldq, n, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
  c.flops += 8.0 * k * k * (p + (n - j) + (c.want_qz ? dn : 0.0));
  // (f) restore: QR chain top to bottom
  const int nlb = ht_num_left_blocks(p, k);
  for (int t = 0; t < nlb; ++t) {
    int r0, r1, e0, e1;
    ht_left_block(p, k, t, &r0, &r1);
    if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
    const int width = e1 - r0, kc = r1 - r0;
    double* blk = B + (size_t)(j + 1 + r0) + (size_t)(j + 1 + r0) * ldb;
    double* wy = w.wyLR + (size_t)t * wst;
    CK(ht_launch_factor_block(st, 3, blk, ldb, width, kc, wy, wst));
    CK(ht_apply_single(st, 0, B, ldb, j + 1 + r1, n - (j + 1 + r1), j + 1 + r0, width, kc, wy, wst));
    c.flops += 4.0 * (n - (j + 1 + r1)) * width * kc;
  }
  CK(ht_sweep(st, 0, A, lda, j, n - j, j + 1, w.wyLR, wst, 3, p, k, 0, nlb, 0, 0));
  if (c.want_qz) CK(ht_sweep(st, 1, Q, ldq, 0, n, j + 1, w.wyLR, wst, 3, p, k, 0, nlb, 0, 0));
  c.flops += 4.0 * p * k * 2.0 * ((n - j) + (c.want_qz ? dn : 0.0));
  return cudaGetLastError();
}

int check_args(int n, const void* A, int lda, const void* B, int ldb, const void* Q, int ldq, const void* Z,
               int ldz, int want_qz) {
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && !B) return -4;
  if (ldb < std::max(1, n)) return -5;
  if (want_qz && n > 0 && !Q) return -6;
  if (want_qz && ldq < std::max(1, n)) return -7;
  if (want_qz && n > 0 && !Z) return -8;
  if (want_qz && ldz < std::max(1, n)) return -9;
  return HT_OK;
}

int reduce_impl(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz, int want_qz,
                const ht_options* opt, ht_stats* stats, cudaStream_t st) {
  int rc = check_args(n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz);
  if (rc != HT_OK) return rc;
  int nb = 32, max_ir = 10, prec = HT_PREC_FP64;
  double tol_scale = 1.0;
  uint64_t seed = 0;
  if (opt) {
    if (opt->nb > 0) nb = opt->nb;
    if (opt->max_ir > 0) max_ir = opt->max_ir;
    if (opt->max_ir < 0) max_ir = 0;
    if (opt->ir_tol_scale > 0.0) tol_scale = opt->ir_tol_scale;
    if (opt->ir_tol_scale < 0.0) tol_scale = 0.0;
    prec = opt->precision;
    seed = opt->seed;
  }
  if (nb > HT_NB_MAX) return HT_ERR_NOT_IMPLEMENTED;
  if (prec != HT_PREC_FP64) return HT_ERR_NOT_IMPLEMENTED;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  t_last_status = HT_OK;
  if (n == 0) return HT_OK;
  if (want_qz) {
    HT_CUDA(ht_launch_set_identity(st, Q, ldq, n));
    HT_CUDA(ht_launch_set_identity(st, Z, ldz, n));
  }
  if (n <= 2) {
    HT_CUDA(ht_launch_zero(st, B, ldb, n, n, 1));
    HT_CUDA(cudaStreamSynchronize(st));
    return HT_OK;
  }
  PoolEntry* pe = acquire(n, nb, &rc);
  if (!pe) return rc;
  HtWork& w = pe->w;
  w.stream = st;
  Ctx c{&w, st, n, A, B, Q, Z, lda, ldb, ldq, ldz, want_qz, 0.0};
  cudaEvent_t ev[4] = {};
  const bool timing = (stats != nullptr);
  if (timing)
    for (auto& e : ev) cudaEventCreate(&e);
  int result = HT_OK;
  do {
    if (cudaMemsetAsync(w.err, 0, sizeof(int), st) != cudaSuccess) { result = HT_ERR_CUDA; break; }
    if (ht_launch_check_finite(st, A, lda, n, 0, w.err) != cudaSuccess ||
        ht_launch_check_finite(st, B, ldb, n, 1, w.err) != cudaSuccess) { result = HT_ERR_CUDA; break; }
    {
      int derr = 0;
      if (cudaMemcpyAsync(&pe->host_status->error, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      derr = pe->host_status->error;
      if (derr != 0) { result = derr; break; }
    }
    if (ht_launch_prepare_B(w, B, ldb, 0, seed, 1) != cudaSuccess) { result = HT_ERR_CUDA; break; }
    int s = 0;
    while (s <= n - 3) {
      const int kmax = std::min(nb, (n - s - 1) / 2);
      if (cudaMemsetAsync(w.status, 0, sizeof(PanelStatus), st) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      if (ht_launch_prepare_B(w, B, ldb, s, seed, 0) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      if (timing) cudaEventRecord(ev[0], st);
      cudaError_t e = ht_launch_panel(w, A, lda, B, ldb, s, kmax, tol_scale, max_ir);
      if (e != cudaSuccess) {
        std::fprintf(stderr, "libht: panel launch failed: %s\n", cudaGetErrorString(e));
        result = HT_ERR_CUDA;
        break;
      }
      if (timing) cudaEventRecord(ev[1], st);
      if (cudaMemcpyAsync(pe->host_status, w.status, sizeof(PanelStatus), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        result = HT_ERR_CUDA;
        break;
      }
      const PanelStatus ps = *pe->host_status;
      if (ps.error != 0) { result = ps.error; break; }
      int k = ps.k_done;
      if (k < 1) { result = HT_ERR_INTERNAL; break; }
      if (stats) {
        stats->panels += 1;
        stats->early_absorptions += ps.failed;
        stats->ir_steps += ps.ir_steps;
        stats->cols_with_ir += ps.cols_with_ir;
        stats->perturbed_pivots += ps.perturbed;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        stats->ms_panel += ms;
      }
      {
        const int m = n - s - 1;
        // panel flops: per column the Y GEMV (2 m p), solve and residual (~m^2 each), plus corrections
        for (int q = 0; q < k; ++q) {
          const double mm = m, pp = m - q;
          c.flops += 2.0 * mm * pp + 2.0 * mm * mm;
        }
        c.flops += 2.0 * (double)m * m * ps.ir_steps;
      }
      if (timing) cudaEventRecord(ev[2], st);
      e = absorb(c, s, k);
      if (e != cudaSuccess) {
        std::fprintf(stderr, "libht: absorption failed: %s\n", cudaGetErrorString(e));
        result = HT_ERR_CUDA;
        break;
      }
      if (timing) {
        cudaEventRecord(ev[3], st);
        cudaEventSynchronize(ev[3]);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[2], ev[3]);
        stats->ms_absorb += ms;
      }
      s += k;
    }
    if (result != HT_OK) break;
    int derr = 0;
    if (cudaMemcpyAsync(&derr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      result = HT_ERR_CUDA;
      break;
    }
    if (derr != 0) result = derr;
  } while (0);
  if (stats) stats->flops_nominal = c.flops;
  if (timing)
    for (auto& e : ev) cudaEventDestroy(e);
  {
    int derr = 0;
    cudaMemcpy(&derr, w.err, sizeof(int), cudaMemcpyDeviceToHost);
    t_last_status = derr;
  }
  release(pe);
  return result;
}

}  // namespace

extern "C" {

int ht_reduce_ex(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz, int want_qz,
                 const ht_options* opt, ht_stats* stats, ht_stream_t stream) {
  return reduce_impl(n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz, opt, stats, (cudaStream_t)stream);
}

int ht_reduce(int n, double* A, int lda, double* B, int ldb, double* Q, double* Z, int want_qz, ht_stream_t stream) {
  return reduce_impl(n, A, lda, B, ldb, Q, n, Z, n, want_qz, nullptr, nullptr, (cudaStream_t)stream);
}

int ht_reduce_batched(int batch, const int* n, double* const* A, const int* lda, double* const* B, const int* ldb,
                      double* const* Q, double* const* Z, int want_qz, ht_stream_t stream) {
  if (batch < 0) return -1;
  if (batch > 0 && (!n || !A || !lda || !B || !ldb)) return -2;
  if (want_qz && batch > 0 && (!Q || !Z)) return -7;
  std::vector<int> order(batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  for (int i : order) {
    const int rc = reduce_impl(n[i], A[i], lda[i], B[i], ldb[i], want_qz ? Q[i] : nullptr, std::max(1, n[i]),
                               want_qz ? Z[i] : nullptr, std::max(1, n[i]), want_qz, nullptr, nullptr,
                               (cudaStream_t)stream);
    if (rc != HT_OK) return rc;
  }
  return HT_OK;
}

int ht_last_device_status(ht_stream_t stream, int* status) {
  (void)stream;
  if (!status) return -2;
  *status = t_last_status;
  return HT_OK;
}

int ht_finalize(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (PoolEntry* e : g_pool) {
    if (e->busy) continue;
    cudaFree(e->base);
    cudaFreeHost(e->host_status);
    delete e;
  }
  g_pool.erase(std::remove_if(g_pool.begin(), g_pool.end(), [](PoolEntry* e) { return !e->busy ? true : false; }),
               g_pool.end());
  return HT_OK;
}

const char* ht_status_string(int status) {
  switch (status) {
    case HT_OK: return "success";
    case HT_ERR_CUDA: return "a CUDA runtime call failed";
    case HT_ERR_NOMEM: return "device workspace could not be allocated";
    case HT_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case HT_ERR_NONFINITE: return "A or B holds a NaN or an infinity";
    case HT_ERR_NOT_IMPLEMENTED: return "option combination not available";
    case HT_ERR_INTERNAL: return "a device-side consistency check failed";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

const char* ht_version(void) { return "libht 0.1 (sm_103a)"; }

}  // extern "C"
