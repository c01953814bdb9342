// Internal declarations shared by the CUDA translation units of libht.
//
// Index conventions (0-based; the paper is 1-based):
//   s      first unreduced column of A at the start of a panel (Sec. 3.2)
//   k      reflectors accumulated in the panel, j = s + k
//   m      n - s - 1, rows of the trailing system B(s+1:n, s+1:n)
//   p      n - j - 1, rows of V2 and U2 (Sec. 3.3.1a, 3.3.2a)
// Panel factors are stored with "local" rows r = global row - (s + 1):
//   U(r, i), V(r, i)  ld = n, r in [0, m)   (U1 = rows 0..k-1, U2 = rows k..m-1)
//   Y(row, i)         ld = n, global rows   (rows 0..s formed after the panel)
//   S, T              ld = nbmax, upper triangular
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ht.h"

#define HT_THREADS 256
#define HT_TRSV_BS 64          // row tile of the triangular solve / multiply
#define HT_TRMV_CW 1024        // column chunk of the triangular multiply B w (partials per chunk)
#define HT_TRSV_BI 256         // diagonal block of the grid-synchronous solve (explicit inverses)
#define HT_NB_MAX 64           // largest panel width (windows live in shared memory)
#define HT_BIG_EXP 500         // rescale threshold 2^500 of the scaled solve
#define HT_SPIN_LIMIT (1 << 22)  // ~ a few seconds of polling, then HT_ERR_TIMEOUT

// ---------------------------------------------------------------------------
// Window / block layout of the absorption chains (Sec. 3.3, Remark 3.2).
// p rows of V2 (or U2), k reflectors.  The first window has kt rows with
// k < kt <= 2k (or p rows when p <= 2k); the others have 2k rows, overlap k.
// ---------------------------------------------------------------------------
__host__ __device__ inline int ht_first_window(int p, int k) {
  if (p <= 2 * k) return p;
  int q = (p - 2 * k + k - 1) / k;
  return p - k * q;
}
__host__ __device__ inline int ht_num_windows(int p, int k) {
  int kt = ht_first_window(p, k);
  return (kt >= p) ? 1 : 1 + (p - kt) / k;
}
// QL chain on V2, top to bottom: window i covers rows [r0, r1).
__host__ __device__ inline void ht_ql_window(int p, int k, int i, int* r0, int* r1) {
  int kt = ht_first_window(p, k);
  if (i == 0) { *r0 = 0; *r1 = kt; return; }
  *r0 = kt - k + (i - 1) * k;
  *r1 = *r0 + 2 * k;
}
// QR chain on U2, bottom to top: window i covers rows [r0, r1).
__host__ __device__ inline void ht_qr_window(int p, int k, int i, int* r0, int* r1) {
  int kt = ht_first_window(p, k);
  if (i == 0) { *r0 = p - kt; *r1 = p; return; }
  *r1 = p - kt + k - (i - 1) * k;
  *r0 = *r1 - 2 * k;
}
// Column blocks of B(:, j+1:n) after the QL chain (small block first).
__host__ __device__ inline int ht_num_right_blocks(int p, int k) {
  if (p <= k) return 1;
  int b0 = ht_first_window(p, k) - k;
  return 1 + (p - b0) / k;
}
__host__ __device__ inline void ht_right_block(int p, int k, int b, int* c0, int* c1) {
  if (p <= k) { *c0 = 0; *c1 = p; return; }
  int b0 = ht_first_window(p, k) - k;
  if (b == 0) { *c0 = 0; *c1 = b0; return; }
  *c0 = b0 + (b - 1) * k;
  *c1 = *c0 + k;
}
// Row blocks of B(j+1:n, :) after the QR chain (small block last).
__host__ __device__ inline int ht_num_left_blocks(int p, int k) {
  if (p <= k) return 1;
  int bl = ht_first_window(p, k) - k;
  return (p - bl) / k + 1;
}
__host__ __device__ inline void ht_left_block(int p, int k, int b, int* r0, int* r1) {
  if (p <= k) { *r0 = 0; *r1 = p; return; }
  int bl = ht_first_window(p, k) - k;
  int nfull = (p - bl) / k;
  if (b < nfull) { *r0 = b * k; *r1 = *r0 + k; return; }
  *r0 = nfull * k; *r1 = p;
}

// ---------------------------------------------------------------------------
// A chain of orthogonal transforms G_i = I - Vw_i Ww_i^T (regular WY form,
// Sec. 2.4), each acting on `width` consecutive rows/columns starting at
// `offset`.  Vw_i and Ww_i are width x nrefl, column-major, ld = width, at
// wy + i * stride (Vw) and wy + i * stride + HT_WY_HALF(stride) (Ww).
// ---------------------------------------------------------------------------
struct WyWin {
  int offset;  // first row/column acted on, relative to the chain origin
  int width;   // rows/columns acted on
  int nrefl;   // reflectors (columns of Vw, Ww)
  int limit;   // structural bound used by the sweeps (see ht_apply.cu)
};

struct PanelStatus {
  int k_done;        // reflector pairs accumulated by the panel
  int failed;        // 1 when the panel stopped on an IR failure
  int ir_steps;      // correction solves in this panel
  int cols_with_ir;  // columns with >= 1 correction
  int error;         // HT_OK or an HT_ERR_* code raised on the device
  int perturbed;     // zero pivots replaced before the panel
  int pad[2];
};

// Device workspace of one reduction (sizes for order n and panel width nb).
struct HtWork {
  int n, nb, G;            // order, panel width, CTAs of the cooperative panel
  double *U, *V, *Y;       // n x nb each (ld n)
  double *S, *T;           // nb x nb each (ld nb)
  double *vec;             // 8 vectors of length n (see ht_panel.cu)
  double *part;            // G x HT_PART_STRIDE partial sums
  double *ypart;           // ychunks x n partial GEMV sums
  int ychunks;
  double *invd;            // reciprocal of diag(B), length n
  int *flags, *exps;       // TRSV block flags / scale exponents (n / 64 + 1 each)
  unsigned *epoch;         // TRSV epoch counter (device)
  PanelStatus *status;     // device status of the last panel
  double *bnorm;           // ||B||_F (device scalar)
  double *wyR, *wyL;       // WY stores of the QL (V2) and QR (U2) chains
  double *wyRR, *wyLR;     // WY stores of the RQ and QR restore chains
  size_t wy_cap;           // doubles per store (>= (p/k + 2) * 4k^2 for every k <= nb)
  double *L1, *R1;         // L-hat_1 and R-tilde_1 (nb x nb)
  double *V2w, *U2w;       // working copies of V2, U2 (n x nb)
  double *tmp1, *tmp2, *tmp3;  // n x nb scratch
  double *small;           // nb x nb scratch (4 of them)
  int *err;                // device error word
  unsigned epoch_host;     // next TRSV epoch (host shadow)
  unsigned long long* ptime;  // per-phase panel timers (profile mode) or null
  double* Xinv;            // inverses of the diagonal blocks of the trailing B (n x HT_TRSV_BI)
  int* safe;               // per diagonal block: inverse usable
  double* xmax;            // per diagonal block of the solve: 32 partial max |x| slots
  unsigned long long* prog;  // solve progress word per panel CTA (epoch-stamped, look-ahead solve)
  double* nearv;           // update of the next diagonal block of the solve (HT_TRSV_BI)
  double* wpart;           // chunk partials of the triangular multiply
  double* tstore;          // T factors of the restore steps (HT_NB_MAX^2 each)
  int* rcount;             // restore: reflectors published (a step-stamped counter)
  double* rtaus;           // tau of every restore step (n + 2 HT_NB_MAX)
  void* emu_dig;           // digits of the grouped window transforms of the emulated sweeps (emu_cap groups)
  int* emu_exps;           // their exponent bounds (one per group)
  void* emu_geo;           // their table (emu_cap int4)
  int emu_cap;             // windows per launch of the emulated sweeps
  int prec;                // HT_PREC_* of the current call
  long spin;               // polls before a bounded device wait gives up (HT_SPIN_LIMIT by default)
  int* cflags;             // wavefront chains: columns published per window (2 (n + 8) ints)
  int* tc_sched;           // work-unit counters of the tcgen05 sweeps (1 + 3 (n / 128 + 1) ints)
  cudaStream_t stream;
  // Q / Z updates of an absorption on a second stream (null: all on the caller's
  // stream), with their own digit buffers and unit counters; side_ev: the main
  // stream's points the side stream waits for (chains, RQ restore, U-tilde, QR
  // restore) and [4] the side stream done with the absorption
  cudaStream_t side;
  cudaEvent_t side_ev[5];
  // at most this many CTAs (0: the whole GPU) for every launch whose CTAs wait on
  // one another (cooperative panel, chains and restore; the tcgen05 sweeps), so
  // that reductions on concurrent streams are all resident together
  int cap;
  void* emu_dig2;
  int* emu_exps2;
  void* emu_geo2;
  int* tc_sched2;
};
#define HT_PART_STRIDE 80   // >= nb + 8 for nb <= 64 ... plus norms
#define HT_NVEC 8

// ---------------------------------------------------------------------------
// Launchers (each returns a cudaError_t of the launch)
// ---------------------------------------------------------------------------
cudaError_t ht_launch_prepare_B(HtWork& w, double* B, int ldb, int s, uint64_t seed, int first);
cudaError_t ht_launch_panel(HtWork& w, double* A, int lda, const double* B, int ldb, int s, int kmax,
                            double tol_scale, int max_ir);
cudaError_t ht_gemm(cudaStream_t st, char ta, char tb, int M, int N, int K, double alpha, const double* A, int lda,
                    const double* Bm, int ldb, double beta, double* C, int ldc);
// as ht_gemm, splitting K over extra CTAs (partials in ws) when the output has few tiles
cudaError_t ht_gemm_ws(cudaStream_t st, char ta, char tb, int M, int N, int K, double alpha, const double* A,
                       int lda, const double* Bm, int ldb, double beta, double* C, int ldc, double* ws,
                       size_t ws_doubles);
// QL chain of V2 and QR chain of U2 (two CTAs) plus the T / Ww formation of every window
cudaError_t ht_launch_chains(cudaStream_t st, double* V2, double* U2, long ld, int p, int k, double* wyR, double* wyL,
                             size_t stride, double* L1, double* R1);
// the same two chains as a wavefront over their windows (ht_chain.cu, k <= 32):
// pubR, pubL hold p k doubles each, flags 2 (p / k + 2) ints; then T / Ww
cudaError_t ht_launch_chains_wave(cudaStream_t st, double* V2, double* U2, long ld, int p, int k, double* wyR,
                                  double* wyL, size_t stride, double* L1, double* R1, double* pubR, double* pubL,
                                  int* flags, int* err, long spin, int max_ctas = 0);
cudaError_t ht_launch_form_wy(cudaStream_t st, double* wyR, double* wyL, size_t stride, int p, int k);
// restore chain of B (mode 2: RQ right, mode 3: QR left), one cooperative launch
// steps [ta, tb) of it (tb < 0: to the end); a launch that ends before the last
// step leaves the lines outside ht_restore_band(tb) to a later sweep
cudaError_t ht_launch_restore(cudaStream_t st, int mode, int p, int k, int j, int n, double* B, long ldb, double* wy,
                              size_t stride, double* tstore, double* taus, int* flag, int* err,
                              unsigned long long* ptime, long spin, int ta = 0, int tb = -1, int max_ctas = 0);
int ht_restore_steps(int mode, int p, int k);
// lines [blo, bhi) (relative to j + 1) that the steps up to tb - 1 still update themselves
void ht_restore_band(int mode, int p, int k, int tb, int* blo, int* bhi);
// One target of a fused chain application (see ht_apply.cu).
#define HT_SWEEP_MAXJOBS 4
struct HtSweepJob {
  double* X;
  long ldx;
  int right;       // 1: X(:, win) <- X(:, win) G;  0: X(win, :) <- G^T X(win, :)
  int line0;       // first row (right) / column (left) swept
  int nlines;      // rows (right) or columns (left) swept
  int origin;      // column (right) or row (left) index of window offset 0
  int use_limit;   // 1: skip stripes that the structural limit says are zero
  int limit_base;  // added to the window limit
};
cudaError_t ht_sweep_multi(cudaStream_t st, const HtSweepJob* jobs, int njobs, const double* wy, long stride, int mode,
                           int p, int k, int t0, int t1);
// as ht_sweep_multi with FP64 emulated on the tcgen05 tensor cores (ht_tc.cu):
// consecutive windows grouped into products of at most 64 x 64, `cap` groups per
// launch, dig: cap * ht_tc_group_bytes() bytes, exps: cap ints, geo: cap int4,
// sched: 1 + (line blocks of 128 lines of all jobs) ints of scratch; at most
// max_ctas CTAs (0: one per SM);
// k <= 32; a bounded wait that gives up raises HT_ERR_TIMEOUT in *err
cudaError_t ht_tc_sweep_multi(cudaStream_t st, const HtSweepJob* jobs, int njobs, const double* wy, long stride,
                              int mode, int p, int k, int t0, int t1, void* dig, int* exps, void* geo, int cap,
                              int* sched, int* err, int max_ctas = 0);
int ht_tc_group(int k);
size_t ht_tc_group_bytes();
cudaError_t ht_sweep(cudaStream_t st, int right, double* X, long ldx, int line0, int nlines, int origin,
                     const double* wy, long stride, int mode, int p, int k, int t0, int t1, int use_limit,
                     int limit_base);
cudaError_t ht_apply_single(cudaStream_t st, int right, double* X, long ldx, int line0, int nlines, int origin,
                            int width, int nrefl, const double* wy, long stride);
cudaError_t ht_rankk_right_w(cudaStream_t st, double* X, long ldx, int nrows, int c1, int w1, int k,
                             const double* V1, int ldv1, const double* T, int ldt);
cudaError_t ht_rankk_left(cudaStream_t st, double* X, long ldx, int col0, int ncols, int r0, int w1, int k,
                          const double* Ut, int ldu, const double* S, int lds);
int ht_panel_max_ctas(int nb);
// workspace layout (bytes when b is null) and the driver of Algorithm 1 on it
// side: also the buffers of the side stream's sweeps
size_t ht_layout_work(HtWork& w, char* b, int n, int nb, int G, unsigned long long** pt, bool side = false);
int ht_reduce_core(HtWork& w, PanelStatus* host_status, unsigned long long* pt_dev, int n, double* A, int lda,
                   double* B, int ldb, double* Q, int ldq, double* Z, int ldz, int want_qz, int nb, int max_ir,
                   double tol_scale, uint64_t seed, int profile, ht_stats* stats, cudaStream_t st);
cudaError_t ht_launch_rankk_right(cudaStream_t st, double* X, long ldx, int nrows, int c1, int c2, int k,
                                  const double* V1, int ldv1, const double* L1, int ldl1, const double* T, int ldt);
cudaError_t ht_launch_rankk_left(cudaStream_t st, double* X, long ldx, int ncols, int r0, int k, const double* Ut,
                                 int ldu, const double* S, int lds);
cudaError_t ht_launch_zero(cudaStream_t st, double* X, long ldx, int rows, int cols, int lower_only);
cudaError_t ht_launch_set_identity(cudaStream_t st, double* X, long ldx, int n);
cudaError_t ht_launch_check_finite(cudaStream_t st, const double* X, long ldx, int n, int upper_only, int* err);

// Dense Householder QR (ht_qr.cu): M (m x nc) <- R in place (exact zeros below),
// the same reflectors applied from the left to every target (its rows aligned
// with M's) and from the right to Qm (nq rows): Qm <- Qm Q_M.  ws: at least
// ht_qr_ws_doubles(m, max(nc, targets' columns), nq) doubles.
struct HtQrTarget {
  double* X;
  long ld;
  int ncols;
};
size_t ht_qr_ws_doubles(int m, int nx, int nq);
cudaError_t ht_qr_blocked(cudaStream_t st, int m, int nc, double* M, long ldm, const HtQrTarget* left, int nleft,
                          double* Qm, long ldq, int nq, double* ws);
// zc[c] = 1 when column c of the upper triangle of B is zero; *offdiag = 1 when
// B has a nonzero above its diagonal
cudaError_t ht_launch_zero_columns(cudaStream_t st, int n, const double* B, long ldb, int* zc, int* offdiag);
// X <- X(:, p) (and rows X(p, :) when rows != 0) through tmp (n x n, ld n); p on the device
cudaError_t ht_launch_permute(cudaStream_t st, int n, double* X, long ldx, double* tmp, const int* p, int rows);
// N(0,1) probe samples (count doubles) and a sum of squares of X - Y (Y null:
// of X) over an m x c block added to *acc (ht_qr.cu)
cudaError_t ht_launch_gauss(cudaStream_t st, size_t count, double* X, unsigned long long seed);
cudaError_t ht_launch_sumsq(cudaStream_t st, int m, int c, const double* X, long ldx, const double* Y, long ldy,
                            double* acc);
// X <- the permutation matrix with X(p[i], i) = 1
cudaError_t ht_launch_perm_matrix(cudaStream_t st, int n, double* X, long ldx, const int* p);

// WY store helpers
__host__ __device__ inline size_t ht_wy_half(size_t stride) { return stride / 2; }

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ double ht_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double ht_warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Block-wide sum; `red` is shared scratch of >= 32 doubles.  All threads get the result.
__device__ __forceinline__ double ht_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = ht_warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = ht_warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}
__device__ __forceinline__ double ht_block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = ht_warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = ht_warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}
__device__ __forceinline__ int ht_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void ht_st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ht_ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void ht_st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
#endif
