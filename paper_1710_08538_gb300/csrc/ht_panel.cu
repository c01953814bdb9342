// Panel reduction of the Householder HT reduction (Sec. 3.2 of Bujanovic,
// Karlsson, Kressner, arXiv 1710.08538), as ONE cooperative persistent
// launch per panel.  All CTAs walk the columns j = s, s+1, ... together; the
// grid-wide phases of one column are:
//   A/B  column update A(:,j) -= Y V(j,:)^T, A(:,j) -= U S^T U^T A(:,j) (Sec. 3.2.2a)
//   C/D  left reflector (beta, u), S growth (Sec. 3.2.2b), right-hand side
//        c~ = (I - U S U^T)[0; e1] of the enlarged system (Sec. 3.2.2c step 1)
//   E    backward substitution B y~ = sigma c~ (step 2), scaled by powers of two
//   F/G  y = (I - V T V^T)^T y~, x = y(j+1:n) (steps 3-4)
//   H-K  residual r = sigma e1 - B~22 x through (I - V T V^T), B, (I - U S^T U^T)
//   L    iterative-refinement test ||r|| / ||x|| <= 2u||B||_F (Sec. 2.3); a
//        failure after max_ir corrections ends the panel (early absorption)
//   N-P  right reflector (gamma, v), T growth and the new column of
//        Y = A V T (Sec. 3.2.2d); rows 0..s of Y are formed later (Remark 3.1).
// The FP64 work of a column is two passes over the triangle of B (solve,
// residual) and one over A(s+1:n, j+1:n) (the Y column): HBM- and
// DFMA-bound.  The triangular solve works on 256-row diagonal blocks with
// precomputed inverses: a chain of 32 CTAs solves block after block while the
// other CTAs apply each solved block to the rows above, one step behind,
// synchronised through progress words (bounded spins, error word on timeout).
#include <cooperative_groups.h>

#include "ht_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr double kU = 1.1102230246251565e-16;  // unit roundoff 2^-53
constexpr int BS = HT_TRSV_BS;

struct PanelArgs {
  int n, s, kmax, max_ir, nb;
  double tol_scale;
  double* A;
  long lda;
  const double* B;
  long ldb;
  double *U, *V, *Y, *S, *T;
  double *acol, *ctil, *ytil, *x, *res, *w, *w2, *z;
  double* part;
  double* ypart;
  int ychunks;
  const double* invd;
  int* flags;
  int* exps;
  unsigned epoch0;
  PanelStatus* st;
  int* err;
  const double* bnorm;
  int cap;    // staged rows per CTA (>= ceil(m / G)) when stage != 0
  int stage;  // 1: U, V, Y rows of the CTA's chunk are kept in shared memory
  unsigned long long* ptime;  // optional per-phase nanoseconds (CTA 0), 16 slots
  double* Xinv;    // inverses of the BI x BI diagonal blocks of the trailing B (row-major, per block)
  int* safe;       // per block: 1 = solve with the inverse, 0 = scaled substitution
  double* xmax;    // per diagonal block: 32 partial max |x| slots
  unsigned long long* prog;  // per-CTA progress words of the look-ahead solve
  double* nearv;   // B(block i-1, block i) x_i of the look-ahead solve
  double* wpart;   // chunk partials of the triangular multiply (nchunks x n)
  long spin;       // polls before a bounded wait gives up
};

__device__ __forceinline__ unsigned long long ht_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory layout (doubles): S, T (nb*nb each), vz, vh (nb+1 each),
// red (64), tile (BS*BS), red4 (4*BS), acc (BS), rscr (HT_THREADS), and,
// when `stage` is set, this CTA's rows of U, V and Y (cap x nb each).
__host__ __device__ inline size_t smem_base_doubles(int nb) {
  return 2 * (size_t)nb * nb + 2 * (size_t)(nb + 1) + 64 + BS * BS + 4 * BS + BS + HT_THREADS + 32 * HT_TRSV_BI +
         HT_TRSV_BI;
}
__host__ __device__ inline size_t smem_doubles(int nb, int cap) {
  return smem_base_doubles(nb) + 3 * (size_t)cap * nb;
}

// out[i] = sum_{r in [rb, re)} M(r, i) * y[r] for i < kk, one partial per CTA.
// M is in shared memory when m_shared (indexed M[r + i * ld] as well).
__device__ void partial_mty(const double* M, long ld, bool m_shared, int kk, const double* y, int rb, int re,
                            double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < kk; i += HT_THREADS / 32) {
    double acc = 0.0;
    for (int r = rb + lane; r < re; r += 32) {
      const double mv = m_shared ? M[r + (size_t)i * ld] : __ldcg(M + r + (size_t)i * ld);
      acc += mv * __ldcg(y + r);
    }
    acc = ht_warp_sum(acc);
    if (lane == 0) out[i] = acc;
  }
}

// dst[i] = sum over CTAs of part[c * HT_PART_STRIDE + off + i], i < kk.
// Partials are double-buffered: a phase writes buffer (pc & 1) and the next
// phase reads it, so no CTA overwrites a slot another CTA is still reading.
__device__ void reduce_part(const double* part, int off, int kk, double* dst, double* scratch) {
  // thread t sums CTAs c = t / kk, t / kk + nt, ... of column i = t % kk with
  // independent loads in flight; the nt partial sums are then added in order.
  if (kk <= 0) { __syncthreads(); return; }
  const int nt = max(1, (int)blockDim.x / kk);
  const int t = threadIdx.x, i = t % kk, g0 = t / kk;
  if (g0 < nt) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int c = g0;
    const int G = gridDim.x;
    for (; c + 3 * nt < G; c += 4 * nt) {
      s0 += __ldcg(part + (size_t)c * HT_PART_STRIDE + off + i);
      s1 += __ldcg(part + (size_t)(c + nt) * HT_PART_STRIDE + off + i);
      s2 += __ldcg(part + (size_t)(c + 2 * nt) * HT_PART_STRIDE + off + i);
      s3 += __ldcg(part + (size_t)(c + 3 * nt) * HT_PART_STRIDE + off + i);
    }
    for (; c < G; c += nt) s0 += __ldcg(part + (size_t)c * HT_PART_STRIDE + off + i);
    scratch[g0 * kk + i] = (s0 + s1) + (s2 + s3);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kk; q += blockDim.x) {
    double v = 0.0;
    for (int g = 0; g < nt; ++g) v += scratch[g * kk + q];
    dst[q] = v;
  }
  __syncthreads();
}

__device__ double reduce_scalar(const double* part, int off, double* red, bool is_max) {
  double t = is_max ? 0.0 : 0.0;
  for (int c = threadIdx.x; c < (int)gridDim.x; c += blockDim.x) {
    double v = __ldcg(part + (size_t)c * HT_PART_STRIDE + off);
    t = is_max ? fmax(t, v) : t + v;
  }
  return is_max ? ht_block_max(t, red) : ht_block_sum(t, red);
}

// t[r] = sum_c M(r0 + r, c0 + c) * xv[c] for r < rows, c < cols (tile of at
// most BS rows); 4 threads per row, result in red4 reduced into out[r].
__device__ void tile_gemv(const double* M, long ld, int r0, int rows, int c0, int cols, const double* xv,
                          double* red4, double* out) {
  const int r = threadIdx.x % BS, cq = threadIdx.x / BS;
  double a0 = 0.0, a1 = 0.0;
  if (r < rows) {
    const double* p = M + (size_t)(r0 + r) + (size_t)c0 * ld;
    int c = cq;
    for (; c + 4 < cols; c += 8) {
      a0 += p[(size_t)c * ld] * xv[c];
      a1 += p[(size_t)(c + 4) * ld] * xv[c + 4];
    }
    if (c < cols) a0 += p[(size_t)c * ld] * xv[c];
  }
  red4[cq * BS + r] = a0 + a1;
  __syncthreads();
  if (threadIdx.x < BS) out[threadIdx.x] = red4[threadIdx.x] + red4[BS + threadIdx.x] + red4[2 * BS + threadIdx.x] +
                                           red4[3 * BS + threadIdx.x];
  __syncthreads();
}

// Row tile of a GEMV streamed from memory: returns, to thread r < rows (<= 32),
// sum_c M(r0 + r, c0 + c) x[c] over c < cols.  Lanes take rows (coalesced:
// consecutive rows of a column are contiguous), the warps take interleaved
// columns, GU columns per step so that GU loads per thread are in flight
// (with one CTA per SM, 16 x 8 B x 256 threads keeps ~32 KB per SM in flight,
// about what HBM latency x bandwidth per SM asks for); x is read from global memory (XG, every lane the same address) or
// shared memory.  red: blockDim.x doubles of shared scratch.  Two barriers.
constexpr int GU = 16;
template <bool XG>
__device__ double gemv32(const double* M, long ld, int r0, int rows, int c0, int cols, const double* x, double* red) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double a0 = 0.0, a1 = 0.0;
  if (lane < rows) {
    const double* p = M + (size_t)(r0 + lane) + (size_t)c0 * ld;
    // two batches of matrix loads in flight: the next batch is issued before
    // the current one is consumed; x (a broadcast, cache-resident) is read at
    // use
    double mv[GU];
#pragma unroll
    for (int u = 0; u < GU; ++u) {
      const int cc = wi + u * nw;
      mv[u] = (cc < cols) ? __ldcg(p + (size_t)cc * ld) : 0.0;
    }
    for (int c = wi; c < cols; c += GU * nw) {
      const int cn = c + GU * nw;
      double mn[GU];
#pragma unroll
      for (int u = 0; u < GU; ++u) {
        const int cc = cn + u * nw;
        mn[u] = (cc < cols) ? __ldcg(p + (size_t)cc * ld) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < GU; u += 2) {
        const int c0u = c + u * nw, c1u = c0u + nw;
        const double x0 = (c0u < cols) ? (XG ? __ldcg(x + c0u) : x[c0u]) : 0.0;
        const double x1 = (c1u < cols) ? (XG ? __ldcg(x + c1u) : x[c1u]) : 0.0;
        a0 += mv[u] * x0;
        a1 += mv[u + 1] * x1;
      }
#pragma unroll
      for (int u = 0; u < GU; ++u) mv[u] = mn[u];
    }
  }
  red[threadIdx.x] = a0 + a1;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32)
    for (int w2 = 0; w2 < nw; ++w2) t += red[w2 * 32 + threadIdx.x];
  __syncthreads();
  return t;
}

constexpr int BI = HT_TRSV_BI;  // diagonal block of the grid-synchronous solve

// Inverse of the upper triangular bs x bs diagonal block D = B_loc[r0.., r0..]
// by blocked backward substitution on the identity (32-row sub-blocks from the
// bottom; thread t owns column t of X).  X is written row-major (ld bs) and
// the block is marked safe when X is finite and max|X| max|D| <= 2^26; unsafe
// blocks are solved by scaled substitution instead.  Dsm: 32 x bs scratch.
__device__ void invert_block(const double* Bl, long ldb, int r0, int bs, double* X, int* safe, double* Dsm,
                             double* red) {
  const int tid = threadIdx.x;
  const int nsb = (bs + 31) / 32;
  double dmax = 0.0;
  for (int sb = nsb - 1; sb >= 0; --sb) {
    const int R0 = sb * 32, rows = min(32, bs - R0), wcols = bs - R0;
    __syncthreads();
    for (int e = tid; e < 32 * wcols; e += blockDim.x) {
      const int rr = e % 32, cc = e / 32;
      double v = 0.0;
      if (rr < rows && R0 + rr <= R0 + cc) v = Bl[(size_t)(r0 + R0 + rr) + (size_t)(r0 + R0 + cc) * ldb];
      Dsm[rr + cc * 32] = v;
      dmax = fmax(dmax, fabs(v));
    }
    __syncthreads();
    for (int t = tid; t < bs; t += blockDim.x) {
      if (t < R0) {
        for (int rr = 0; rr < rows; ++rr) X[(size_t)(R0 + rr) * bs + t] = 0.0;
        continue;
      }
      double acc[32];
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) acc[rr] = (R0 + rr == t) ? 1.0 : 0.0;
      for (int c = R0 + rows; c <= t; ++c) {
        const double xv = X[(size_t)c * bs + t];
#pragma unroll
        for (int rr = 0; rr < 32; ++rr) acc[rr] -= Dsm[rr + (c - R0) * 32] * xv;
      }
#pragma unroll
      for (int rr = 31; rr >= 0; --rr) {
        if (rr >= rows) continue;
        const double d = Dsm[rr + rr * 32];
        const double xv = (R0 + rr <= t) ? acc[rr] / d : 0.0;
        X[(size_t)(R0 + rr) * bs + t] = xv;
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (q < rr) acc[q] -= Dsm[q + rr * 32] * xv;
      }
    }
  }
  __syncthreads();
  double xm = 0.0;
  bool fin = true;
  for (int e = tid; e < bs * bs; e += blockDim.x) {
    const double v = X[e];
    if (!isfinite(v)) fin = false;
    xm = fmax(xm, fabs(v));
  }
  xm = ht_block_max(fin ? xm : INFINITY, red);
  dmax = ht_block_max(dmax, red);
  if (tid == 0) *safe = (isfinite(xm) && xm * dmax <= 67108864.0) ? 1 : 0;
}

// Scaled substitution of one diagonal block (rows <= BI) by one CTA: acc
// (shared, rows entries, in the frame of the solve) is overwritten by the
// solution; returns (in *shift) the exponent added to the block frame so that
// no |x| exceeds 2^500.  tile: BS x BS scratch, red4: 4*BS scratch.
__device__ void subst_block(const double* Bl, long ldb, const double* invd, int r0, int rows, double* acc,
                            double* tile, double* red4, double* xl, int* shi, int* shift) {
  const int tid = threadIdx.x;
  if (tid == 0) shi[0] = 0;
  const int nsub = (rows + BS - 1) / BS;
  for (int sbk = nsub - 1; sbk >= 0; --sbk) {
    const int q0 = sbk * BS, qr = min(BS, rows - q0);
    __syncthreads();
    for (int e = tid; e < BS * BS; e += blockDim.x) {
      const int rr = e % BS, cc = e / BS;
      double v = 0.0;
      if (rr < qr && cc < qr && rr <= cc) v = Bl[(size_t)(r0 + q0 + rr) + (size_t)(r0 + q0 + cc) * ldb];
      if (rr == cc && rr >= qr) v = 1.0;
      tile[e] = v;
    }
    __syncthreads();
    if (tid < 32) {
      const int lane = tid;
      double a0 = (lane < qr) ? acc[q0 + lane] : 0.0, a1 = (lane + 32 < qr) ? acc[q0 + lane + 32] : 0.0;
      int E = 0;
      for (int c = BS - 1; c >= 0; --c) {
        const double t = __shfl_sync(0xffffffffu, (c >= 32) ? a1 : a0, c & 31);
        const double d = tile[c + c * BS];
        double xc;
        if (c >= qr) {
          xc = 0.0;
        } else if (fabs(t) > ldexp(fabs(d), HT_BIG_EXP)) {
          const int sh = ilogb(t) - ilogb(d) - HT_BIG_EXP + 2;
          a0 = ldexp(a0, -sh);
          a1 = ldexp(a1, -sh);
          E += sh;
          xc = ldexp(t, -sh) * invd[r0 + q0 + c];
        } else {
          xc = t * invd[r0 + q0 + c];
        }
        if (lane == (c & 31)) {
          if (c >= 32) a1 = xc; else a0 = xc;
        }
        if (lane < c) a0 -= tile[lane + c * BS] * xc;
        if (lane + 32 < c) a1 -= tile[lane + 32 + c * BS] * xc;
      }
      if (lane < qr) acc[q0 + lane] = a0;
      if (lane + 32 < qr) acc[q0 + lane + 32] = a1;
      if (lane == 0) shi[1] = E;
    }
    __syncthreads();
    const int sh = shi[1];
    if (sh != 0) {
      // the rest of the block shares the frame: rows outside this sub-block
      for (int r = tid; r < rows; r += blockDim.x)
        if (r < q0 || r >= q0 + qr) acc[r] = ldexp(acc[r], -sh);
      if (tid == 0) shi[0] += sh;
    }
    __syncthreads();
    // update the rows above the sub-block: acc[0:q0] -= B[r0.., r0+q0..] x_sub
    if (q0 > 0) {
      if (tid < BS) xl[tid] = (tid < qr) ? acc[q0 + tid] : 0.0;
      __syncthreads();
      for (int rb = 0; rb < q0; rb += BS) {
        tile_gemv(Bl, ldb, r0 + rb, min(BS, q0 - rb), r0 + q0, qr, xl, red4, red4);
        if (tid < min(BS, q0 - rb)) acc[rb + tid] -= red4[tid];
        __syncthreads();
      }
    }
  }
  __syncthreads();
  if (tid == 0) *shift = shi[0];
  __syncthreads();
}

// Grid-synchronous blocked backward substitution B_loc y = 2^{-E} rhs.  For
// each BI-row diagonal block from the bottom: (S1) x_i from the precomputed
// inverse, spread over up to 32 CTAs, or by scaled substitution on one CTA;
// grid barrier; (S2) all CTAs subtract B(0:r0, block) x_i from their rows of
// the accumulator; grid barrier.  Every CTA tracks the same frame exponent:
// the stored solution of block i is 2^{-exps[i]} times the true one.
template <class Grid>
__device__ void trsv_gs(const PanelArgs& a, Grid& grid, int m, const double* rhs, double* sol, double* accv,
                        bool force_subst, double* tile, double* red4, double* acc, double* xl, double* xs,
                        double* red, int* shi) {
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int nbk = (m + BI - 1) / BI;
  const double* Bl = a.B + (size_t)(a.s + 1) + (size_t)(a.s + 1) * a.ldb;
  const long ldb = a.ldb;
  const int NX = min(G, 32);
  // accumulator = rhs (chunk rows)
  {
    const int ch = (m + G - 1) / G, rb = min(m, cta * ch), re = min(m, rb + ch);
    for (int r = rb + tid; r < re; r += blockDim.x) accv[r] = __ldcg(rhs + r);
  }
  int E = 0;
  grid.sync();
  for (int i = nbk - 1; i >= 0; --i) {
    const int r0 = i * BI, rows = min(BI, m - r0);
    const bool sf = !force_subst && __ldcg(a.safe + i);
    // ---- S1 ----
    if (sf) {
      if (cta < NX) {
        const int per = (rows + NX - 1) / NX;  // rows of x per CTA
        const double* Xb = a.Xinv + (size_t)i * BI * BI;
        double mx = 0.0;
        for (int rr = cta * per + (tid >> 5); rr < min(rows, (cta + 1) * per); rr += blockDim.x / 32) {
          const int lane = tid & 31;
          double t = 0.0;
          for (int q = rr + lane; q < rows; q += 32) t += __ldcg(Xb + (size_t)rr * rows + q) * __ldcg(accv + r0 + q);
          t = ht_warp_sum(t);
          if (lane == 0) sol[r0 + rr] = t;
          mx = fmax(mx, fabs(t));
        }
        mx = ht_block_max(mx, red);
        if (tid == 0) { a.xmax[cta] = mx; if (cta == 0) a.flags[i] = 0; }
      }
    } else if (cta == i % G) {
      for (int r = tid; r < rows; r += blockDim.x) xs[r] = __ldcg(accv + r0 + r);
      __syncthreads();
      int shift = 0;
      subst_block(Bl, ldb, a.invd, r0, rows, xs, tile, red4, xl, shi, &shift);
      double mx = 0.0;
      for (int r = tid; r < rows; r += blockDim.x) { sol[r0 + r] = xs[r]; mx = fmax(mx, fabs(xs[r])); }
      mx = ht_block_max(mx, red);
      if (tid == 0) { a.xmax[0] = mx; a.flags[i] = shift; }
    }
    grid.sync();
    // ---- S2 ----
    double M = 0.0;
    int delta;
    {
      const int nparts = sf ? NX : 1;
      double t = (tid < nparts) ? __ldcg(a.xmax + tid) : 0.0;
      M = ht_block_max(t, red);
      delta = __ldcg(a.flags + i);  // exponent the block added to the frame
    }
    const int Ei = E + delta;
    int En = max(E, Ei);
    if (M > 0.0 && isfinite(M)) {
      const int big = ilogb(M) + (Ei - En);
      if (big > 400) En += big - 300;
    }
    const int sh_acc = E - En, sh_x = Ei - En;
    if (cta == 0 && tid == 0) a.exps[i] = Ei;  // block exponent relative to the start frame
    if (r0 > 0) {
      for (int q = tid; q < BI; q += blockDim.x) xs[q] = (q < rows) ? __ldcg(sol + r0 + q) : 0.0;
      __syncthreads();
      const int ch = (r0 + G - 1) / G, rb = min(r0, cta * ch), re = min(r0, rb + ch);
      for (int tb = rb; tb < re; tb += 32) {
        const int tr = min(32, re - tb);
        const double sum = gemv32<false>(Bl, ldb, tb, tr, r0, rows, xs, red4);
        if (tid < tr) {
          const double av = __ldcg(accv + tb + tid);
          accv[tb + tid] = ldexp(av, sh_acc) - ldexp(sum, sh_x);
        }
      }
    }
    E = En;
    grid.sync();
  }
}

// Bounded wait until the cnt progress words p[idx(0..cnt-1)] are all >=
// target (warp 0 polls with relaxed loads, all of a lane's words in flight
// together, then one acquire fence; the block follows).  Fails at once when
// the error word is already set (a wait elsewhere gave up), else after
// `spin` polls, setting HT_ERR_TIMEOUT; the caller then carries on
// without the data.
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
template <class Idx>
__device__ bool la_wait(const unsigned long long* p, int cnt, Idx idx, unsigned long long target, int* err,
                        long spin) {
  __shared__ int flag[1];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int ok = 0;
    for (long it = 0; it <= spin; ++it) {
      unsigned long long v[4] = {~0ull, ~0ull, ~0ull, ~0ull};
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (lane + 32 * u < cnt) v[u] = ld_relaxed64(p + idx(lane + 32 * u));
      bool mine = (v[0] >= target) && (v[1] >= target) && (v[2] >= target) && (v[3] >= target);
      for (int c = lane + 128; c < cnt; c += 32) mine = mine && (ld_relaxed64(p + idx(c)) >= target);
      if (__all_sync(0xffffffffu, mine)) { ok = 1; break; }
      if (*(volatile int*)err != 0) break;
      __nanosleep(32);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (!ok && lane == 0) atomicCAS(err, 0, HT_ERR_TIMEOUT);
    if (lane == 0) *flag = ok;
  }
  __syncthreads();
  const bool ok = *flag != 0;
  __syncthreads();
  return ok;
}

// la_wait for two groups at once: words p[0..cntA) against targetA and
// p[idxB(0..cntB-1)] (cntB <= 32) against targetB, all loads of a poll in flight together.
template <class IdxB>
__device__ bool la_wait2(const unsigned long long* p, int cntA, unsigned long long targetA, int cntB, IdxB idxB,
                         unsigned long long targetB, int* err, long spin) {
  __shared__ int flag2[1];
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int ok = 0;
    for (long it = 0; it <= spin; ++it) {
      const unsigned long long va = (lane < cntA) ? ld_relaxed64(p + lane) : ~0ull;
      const unsigned long long vb = (lane < cntB) ? ld_relaxed64(p + idxB(lane)) : ~0ull;
      if (__all_sync(0xffffffffu, va >= targetA && vb >= targetB)) { ok = 1; break; }
      if (*(volatile int*)err != 0) break;
      __nanosleep(32);
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (!ok && lane == 0) atomicCAS(err, 0, HT_ERR_TIMEOUT);
    if (lane == 0) *flag2 = ok;
  }
  __syncthreads();
  const bool ok = *flag2 != 0;
  __syncthreads();
  return ok;
}

// Publishes this CTA's progress word after every thread's stores of the step
// (the barrier orders them before the release store of thread 0).
__device__ __forceinline__ void la_publish(unsigned long long* p, unsigned long long v) {
  __syncthreads();
  if (threadIdx.x == 0) ht_st_release64(p, v);
}

// Look-ahead blocked backward substitution B_loc y = 2^{-E} rhs: the same
// arithmetic as trsv_gs (every sum in the same order, so the same result) on
// a schedule without grid barriers.  CTAs [0, LA_ND) form the diagonal chain:
// for block i they (P1) take x_i from the block inverse (or by scaled
// substitution on CTA 0) and then (P2) the update of the next diagonal block,
// B(block i-1, block i) x_i, into nearv.  CTAs [LA_ND, G) subtract
// B(rows above block i-1, block i) x_i from their 32-row tiles of the
// accumulator, running up to one step behind the chain, which needs their
// update of step i+2 only when it reaches block i.  Progress words (release /
// acquire, epoch-stamped, bounded waits) replace the barriers: chain CTA c
// publishes base + 2 s + 1 after P1 and base + 2 s + 2 after P2 of step s (block
// nbk-1-s), the other CTAs base + s + 1 after their update of step s.  Every
// CTA follows the same frame exponent as trsv_gs from the published per-block
// maxima (xmax, 32 slots per block) and frame shifts (flags).
constexpr int LA_ND = 32;
__device__ __forceinline__ void cp_async8(double* smem, const double* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ void trsv_la(const PanelArgs& a, int m, double* accv, double* sol, bool force_subst, unsigned epoch,
                        double* tile, double* red4, double* xl, double* xs, double* red, int* shi, double* Bt) {
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int nbk = (m + BI - 1) / BI;
  const double* Bl = a.B + (size_t)(a.s + 1) + (size_t)(a.s + 1) * a.ldb;
  const long ldb = a.ldb;
  const unsigned long long base = (unsigned long long)epoch << 14;
  const bool chain = cta < LA_ND;
  const int NF = G - LA_ND;
  auto ident = [](int u) { return u; };
  int E = 0;
  // frame of the step that produced block i (identical in every CTA)
  auto frame = [&](int i, int& sh_acc, int& sh_x) {
    const bool sf = !force_subst && __ldcg(a.safe + i);
    const int nparts = sf ? LA_ND : 1;
    const int delta = __ldcg(a.flags + i);
    if (tid < 32) {
      const double t = ht_warp_max((tid < nparts) ? __ldcg(a.xmax + (size_t)i * 32 + tid) : 0.0);
      if (tid == 0) red[0] = t;
    }
    __syncthreads();
    const double M = red[0];
    __syncthreads();
    const int Ei = E + delta;
    int En = max(E, Ei);
    if (M > 0.0 && isfinite(M)) {
      const int big = ilogb(M) + (Ei - En);
      if (big > 400) En += big - 300;
    }
    sh_acc = E - En;
    sh_x = Ei - En;
    E = En;
    return Ei;
  };
  const int tiles = BI / 32;
  const bool nearcta = chain && cta >= LA_ND - tiles;
  // B(block i-1, block i) rows of this CTA's tile of the next diagonal block
  // (B is fixed during the solve) into Bt (32 x BI, column-major), loaded
  // while the step's x_i is being formed
  auto prefetch_near = [&](int i) {
    const int tr = cta - (LA_ND - tiles);
    const int rn = (i - 1) * BI + tr * 32, c0 = i * BI, cols = min(BI, m - c0);
    for (int e = tid; e < 32 * cols; e += blockDim.x) {
      const int r = e & 31, c = e >> 5;
      cp_async8(Bt + e, Bl + (size_t)(rn + r) + (size_t)(c0 + c) * ldb);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (chain) {
    int sa = 0, sx = 0;  // frame shifts of the previous step
    for (int s = 0; s < nbk; ++s) {
      const int i = nbk - 1 - s, r0 = i * BI, rows = min(BI, m - r0);
      if (nearcta && i > 0) prefetch_near(i);
      const bool sf = !force_subst && __ldcg(a.safe + i);
      // this warp's row of the block inverse (B and its inverses are fixed
      // during the panel), loaded before the waits: x_i(rr) = sum_q X(rr, q) acc(q)
      const int per = (rows + LA_ND - 1) / LA_ND;  // <= BI / 32 rows per CTA, one per warp
      const int rr = cta * per + (tid >> 5), lane = tid & 31;
      const bool myrow = sf && (tid >> 5) < per && rr < rows;
      double xr[BI / 32];
      {
        const double* Xr = a.Xinv + (size_t)i * BI * BI + (size_t)rr * rows;
#pragma unroll
        for (int u = 0; u < BI / 32; ++u) {
          const int q = rr + lane + 32 * u;
          xr[u] = (myrow && q < rows) ? __ldcg(Xr + q) : 0.0;
        }
      }
      // the chain's step s-1 and the far CTAs owning the tiles of block i
      // (tile t belongs to CTA LA_ND + t mod NF), which finished step s-2
      if (s > 0)
        la_wait2(a.prog, LA_ND, base + 2 * s, min(NF, BI / 32),
                 [&](int u) { return LA_ND + (i * (BI / 32) + u) % NF; }, s > 1 ? base + s - 1 : 0ull, a.err, a.spin);
      // accumulator of block i in the frame of this step
      for (int q = tid; q < rows; q += blockDim.x) {
        const double av = __ldcg(accv + r0 + q);
        xs[q] = (s == 0) ? av : ldexp(av, sa) - ldexp(__ldcg(a.nearv + q), sx);
      }
      __syncthreads();
      // ---- P1: x_i ----
      if (sf) {
        double mx = 0.0;
        if (myrow) {
          double t = 0.0;
#pragma unroll
          for (int u = 0; u < BI / 32; ++u) {
            const int q = rr + lane + 32 * u;
            if (q < rows) t += xr[u] * xs[q];
          }
          t = ht_warp_sum(t);
          if (lane == 0) sol[r0 + rr] = t;
          mx = fabs(t);
        }
        mx = ht_block_max(mx, red);
        if (tid == 0) { a.xmax[(size_t)i * 32 + cta] = mx; if (cta == 0) a.flags[i] = 0; }
      } else if (cta == 0) {
        int shift = 0;
        subst_block(Bl, ldb, a.invd, r0, rows, xs, tile, red4, xl, shi, &shift);
        double mx = 0.0;
        for (int r = tid; r < rows; r += blockDim.x) { sol[r0 + r] = xs[r]; mx = fmax(mx, fabs(xs[r])); }
        mx = ht_block_max(mx, red);
        if (tid == 0) { a.xmax[(size_t)i * 32] = mx; a.flags[i] = shift; }
      }
      la_publish(a.prog + cta, base + 2 * s + 1);
      la_wait(a.prog, LA_ND, ident, base + 2 * s + 1, a.err, a.spin);
      const int Ei = frame(i, sa, sx);
      if (cta == 0 && tid == 0) a.exps[i] = Ei;
      // ---- P2: nearv = B(block i-1, block i) x_i, one 32-row tile per CTA ----
      if (i > 0 && nearcta) {
        const int tr = cta - (LA_ND - tiles);
        for (int q = tid; q < rows; q += blockDim.x) xs[q] = __ldcg(sol + r0 + q);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const int lane = tid & 31, wi = tid >> 5, nw = blockDim.x >> 5;
        double s0 = 0.0, s1 = 0.0;
        int c = wi;
        for (; c + nw < rows; c += 2 * nw) {
          s0 += Bt[c * 32 + lane] * xs[c];
          s1 += Bt[(c + nw) * 32 + lane] * xs[c + nw];
        }
        if (c < rows) s0 += Bt[c * 32 + lane] * xs[c];
        red4[tid] = s0 + s1;
        __syncthreads();
        if (tid < 32) {
          double t = 0.0;
          for (int w2 = 0; w2 < nw; ++w2) t += red4[w2 * 32 + tid];
          a.nearv[tr * 32 + tid] = t;
        }
      }
      la_publish(a.prog + cta, base + 2 * s + 2);
    }
  } else {
    const int f = cta - LA_ND;
    for (int s = 0; s + 2 < nbk; ++s) {
      const int i = nbk - 1 - s, r0 = i * BI, rows = min(BI, m - r0);
      const int lim = (i - 1) * BI;  // rows above the next diagonal block
      la_wait(a.prog, LA_ND, ident, base + 2 * s + 1, a.err, a.spin);
      int sh_acc, sh_x;
      frame(i, sh_acc, sh_x);
      if (f * 32 < lim) {
        for (int q = tid; q < BI; q += blockDim.x) xs[q] = (q < rows) ? __ldcg(sol + r0 + q) : 0.0;
        __syncthreads();
        for (int tb = f * 32; tb < lim; tb += NF * 32) {
          const double sum = gemv32<false>(Bl, ldb, tb, 32, r0, rows, xs, red4);
          if (tid < 32) {
            const double av = __ldcg(accv + tb + tid);
            accv[tb + tid] = ldexp(av, sh_acc) - ldexp(sum, sh_x);
          }
        }
      }
      la_publish(a.prog + cta, base + s + 1);
    }
  }
}

template <bool STAGE>
__global__ void __launch_bounds__(HT_THREADS, 1) panel_kernel(PanelArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ double sm[];
  const int nb = a.nb;
  double* Ssh = sm;
  double* Tsh = Ssh + (size_t)nb * nb;
  double* vz = Tsh + (size_t)nb * nb;
  double* vh = vz + (nb + 1);
  double* red = vh + (nb + 1);
  double* tile = red + 64;
  double* red4 = tile + BS * BS;
  double* acc = red4 + 4 * BS;
  double* rscr = acc + BS;
  double* Dsm = rscr + HT_THREADS;  // 32 x BI scratch of the block inversion
  double* xs = Dsm + 32 * BI;       // BI entries: x of the current block
  double* Us = xs + BI;             // staged rows [rbeg, rend) of U, V, Y (ld cap)
  double* Vs = Us + (size_t)a.cap * nb;
  double* Ys = Vs + (size_t)a.cap * nb;
  __shared__ int shi[4];
  __shared__ double xl[BS];

  const int n = a.n, s = a.s, m = n - s - 1, G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const long ldn = n;
  const int chunk = (m + G - 1) / G;
  const int rbeg = min(m, cta * chunk), rend = min(m, rbeg + chunk);
  const double tol = a.tol_scale * 2.0 * kU * (*a.bnorm);
  double* Yl = a.Y + (s + 1);
  // rows [rbeg, rend) of U, V, Y: shared-memory copies when STAGE (written
  // through to global memory, which other CTAs and the absorption read)
  const long lds = STAGE ? (long)a.cap : ldn;
  const double* Ub = STAGE ? (Us - rbeg) : a.U;
  const double* Vb = STAGE ? (Vs - rbeg) : a.V;
  const double* Yb = STAGE ? (Ys - rbeg) : Yl;
  auto ldr = [&](const double* p) -> double { return STAGE ? *p : __ldcg(p); };
  int pc = 0;  // phase counter selecting the partial-sum buffer
  auto pbuf = [&](int c) { return a.part + (size_t)(c & 1) * G * HT_PART_STRIDE; };
  auto mypart = [&]() { return pbuf(pc) + (size_t)cta * HT_PART_STRIDE; };

  for (int e = tid; e < nb * nb; e += blockDim.x) { Ssh[e] = 0.0; Tsh[e] = 0.0; }
  __syncthreads();
  // inverses of the diagonal blocks of B(s+1:n, s+1:n); B is fixed for the panel
  {
    const double* Bl0 = a.B + (size_t)(s + 1) + (size_t)(s + 1) * a.ldb;
    const int nbk = (m + BI - 1) / BI;
    for (int b = cta; b < nbk; b += G)
      invert_block(Bl0, a.ldb, b * BI, min(BI, m - b * BI), a.Xinv + (size_t)b * BI * BI, a.safe + b, Dsm, red);
  }
  grid.sync();

  unsigned epoch = a.epoch0;
  int k = 0, failed = 0, ir_total = 0, ir_cols = 0;
  unsigned long long t_last = (a.ptime && cta == 0 && tid == 0) ? ht_now() : 0ull;
#define PHASE_MARK(id)                                              \
  do {                                                              \
    if (a.ptime && cta == 0 && tid == 0) {                          \
      unsigned long long t_ = ht_now();                             \
      a.ptime[id] += t_ - t_last;                                   \
      t_last = t_;                                                  \
    }                                                               \
  } while (0)
  for (k = 0; k < a.kmax; ++k) {
    const int j = s + k;
    double* Aj = a.A + (size_t)j * a.lda + (s + 1);  // local rows of column j
    // ---- Phase A: right update of column j, save it, partial U^T a ----
    for (int i = tid; i < k; i += blockDim.x) vz[i] = __ldcg(a.V + (k - 1) + (size_t)i * ldn);  // V(j, :)
    __syncthreads();
    for (int r = rbeg + tid; r < rend; r += blockDim.x) {
      double xv = Aj[r];
      a.acol[r] = xv;
      double t = 0.0;
#pragma unroll 8
      for (int i = 0; i < k; ++i) t += ldr(Yb + r + (size_t)i * lds) * vz[i];
      Aj[r] = xv - t;
    }
    __syncthreads();
    ++pc;
    partial_mty(Ub, lds, STAGE, k, Aj, rbeg, rend, mypart());
    grid.sync();
    PHASE_MARK(0);
    // ---- Phase B: left update (I - U S^T U^T), tail norm ----
    reduce_part(pbuf(pc), 0, k, vz, rscr);
    for (int i = tid; i < k; i += blockDim.x) {
      double t = 0.0;
      for (int l = 0; l <= i; ++l) t += Ssh[l + (size_t)i * nb] * vz[l];
      vh[i] = t;
    }
    __syncthreads();
    {
      double tail = 0.0;
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        double xv = Aj[r];
#pragma unroll 8
        for (int i = 0; i < k; ++i) xv -= ldr(Ub + r + (size_t)i * lds) * vh[i];
        Aj[r] = xv;
        if (r > k) tail += xv * xv;
      }
      tail = ht_block_sum(tail, red);
      ++pc;
      if (tid == 0) mypart()[0] = tail;
    }
    grid.sync();
    PHASE_MARK(1);
    // ---- Phase C: left reflector (beta, u) of A(j+1:n, j) ----
    double beta, scal, alpha;
    {
      const double tail2 = reduce_scalar(pbuf(pc), 0, red, false);
      const double x0 = __ldcg(Aj + k);
      if (tail2 == 0.0) {
        beta = 0.0; alpha = x0; scal = 0.0;
      } else {
        const double nrm = sqrt(x0 * x0 + tail2);
        alpha = (x0 >= 0.0) ? -nrm : nrm;
        beta = (alpha - x0) / alpha;
        scal = 1.0 / (x0 - alpha);
      }
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        double u = (r < k) ? 0.0 : (r == k) ? 1.0 : __ldcg(Aj + r) * scal;
        a.U[r + (size_t)k * ldn] = u;
        if (STAGE) Us[(r - rbeg) + (size_t)k * lds] = u;
        if (r == k) Aj[r] = alpha;
        else if (r > k) Aj[r] = 0.0;
      }
      __syncthreads();
      ++pc;
      partial_mty(Ub, lds, STAGE, k, a.U + (size_t)k * ldn, rbeg, rend, mypart());
    }
    grid.sync();
    PHASE_MARK(2);
    // ---- Phase D: S growth; first right-hand side c~ = e_k - U (S U(k,:)^T) ----
    reduce_part(pbuf(pc), 0, k, vz, rscr);
    for (int i = tid; i < k; i += blockDim.x) {
      double t = 0.0;
      for (int l = i; l < k; ++l) t += Ssh[i + (size_t)l * nb] * vz[l];
      vh[i] = -beta * t;
    }
    __syncthreads();
    for (int i = tid; i < k; i += blockDim.x) Ssh[i + (size_t)k * nb] = vh[i];
    if (tid == 0) Ssh[k + (size_t)k * nb] = beta;
    __syncthreads();

    int it = 0, sig_exp = 0;
    bool first = true, ok = false, subst_mode = false;
    double nr2 = 0.0, nx2 = 0.0, xtail2 = 0.0;
    while (true) {
      if (first) {
        // U_new(k, i): row k of U (global row j+1)
        for (int i = tid; i <= k; i += blockDim.x) vz[i] = (i == k) ? 1.0 : __ldcg(a.U + k + (size_t)i * ldn);
        __syncthreads();
        for (int i = tid; i <= k; i += blockDim.x) {
          double t = 0.0;
          for (int l = i; l <= k; ++l) t += Ssh[i + (size_t)l * nb] * vz[l];
          vh[i] = t;
        }
        __syncthreads();
        for (int r = rbeg + tid; r < rend; r += blockDim.x) {
          double c = (r == k) ? 1.0 : 0.0;
#pragma unroll 8
          for (int i = 0; i <= k; ++i) c -= ldr(Ub + r + (size_t)i * lds) * vh[i];
          a.ctil[r] = c;
        }
      } else {
        // c~ = (I - U S U^T)[0; res]: partial U^T [0; res]
        ++pc;
        partial_mty(Ub, lds, STAGE, k + 1, a.res, rbeg, rend, mypart());
        grid.sync();
        reduce_part(pbuf(pc), 0, k + 1, vz, rscr);
        for (int i = tid; i <= k; i += blockDim.x) {
          double t = 0.0;
          for (int l = i; l <= k; ++l) t += Ssh[i + (size_t)l * nb] * vz[l];
          vh[i] = t;
        }
        __syncthreads();
        for (int r = rbeg + tid; r < rend; r += blockDim.x) {
          double c = __ldcg(a.res + r);
#pragma unroll 8
          for (int i = 0; i <= k; ++i) c -= ldr(Ub + r + (size_t)i * lds) * vh[i];
          a.ctil[r] = c;
        }
      }
      grid.sync();
      PHASE_MARK(3);
      // ---- Phase E: scaled backward substitution B y~ = 2^-E c~ ----
      if (G >= 2 * LA_ND) {
        {
          const int ch = (m + G - 1) / G, rb = min(m, cta * ch), re = min(m, rb + ch);
          for (int r = rb + tid; r < re; r += blockDim.x) a.w[r] = __ldcg(a.ctil + r);
        }
        grid.sync();
        trsv_la(a, m, a.w, a.ytil, subst_mode, epoch, tile, red4, xl, xs, red, shi, Dsm);
      } else {
        trsv_gs(a, grid, m, a.ctil, a.ytil, a.w, subst_mode, tile, red4, acc, xl, xs, red, shi);
      }
      ++epoch;
      grid.sync();
    PHASE_MARK(4);
      // ---- Phase F: common exponent, partial V^T y~ ----
      const int nblk = (m + BI - 1) / BI;
      int emax;
      {
        int t = -2147483647;
        for (int b = tid; b < nblk; b += blockDim.x) t = max(t, __ldcg(a.exps + b));
        for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
        __shared__ int wmax[HT_THREADS / 32];
        if ((tid & 31) == 0) wmax[tid >> 5] = t;
        __syncthreads();
        if (tid == 0) {
          int mm = wmax[0];
          for (int q = 1; q < (int)(blockDim.x / 32); ++q) mm = max(mm, wmax[q]);
          shi[2] = mm;
        }
        __syncthreads();
        emax = shi[2];
      }
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        const int e = __ldcg(a.exps + r / BI);
        a.ytil[r] = ldexp(__ldcg(a.ytil + r), e - emax);
      }
      __syncthreads();
      ++pc;
      partial_mty(Vb, lds, STAGE, k, a.ytil, rbeg, rend, mypart());
      grid.sync();
    PHASE_MARK(5);
      // ---- Phase G: x = [(I - V T^T V^T) y~](k:m), combine with the IR iterate ----
      reduce_part(pbuf(pc), 0, k, vz, rscr);
      for (int i = tid; i < k; i += blockDim.x) {
        double t = 0.0;
        for (int l = 0; l <= i; ++l) t += Tsh[l + (size_t)i * nb] * vz[l];
        vh[i] = t;
      }
      __syncthreads();
      {
        double mx = 0.0;
        for (int r = rbeg + tid; r < rend; r += blockDim.x) {
          double xv = 0.0;
          if (r >= k) {
            double d = __ldcg(a.ytil + r);
#pragma unroll 8
            for (int i = 0; i < k; ++i) d -= ldr(Vb + r + (size_t)i * lds) * vh[i];
            xv = first ? d : ldexp(__ldcg(a.x + r), -emax) + d;
            mx = fmax(mx, fabs(xv));
            if (!(fabs(xv) <= 1.79e308)) mx = INFINITY;  // NaN/Inf marker
          }
          a.x[r] = xv;
        }
        mx = ht_block_max(mx, red);
        ++pc;
        if (tid == 0) mypart()[0] = mx;
      }
      sig_exp = first ? -emax : sig_exp - emax;
      grid.sync();
    PHASE_MARK(6);
      // ---- Phase H: normalise x to max |x| in [1, 2); partial V^T [0; x] ----
      int sh = 0;
      {
        const double mx = reduce_scalar(pbuf(pc), 0, red, true);
        if (mx > 0.0 && mx <= 1.79e308) sh = -ilogb(mx);
      }
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        if (r >= k) a.x[r] = ldexp(__ldcg(a.x + r), sh);
      }
      sig_exp += sh;
      __syncthreads();
      ++pc;
      partial_mty(Vb, lds, STAGE, k, a.x, rbeg, rend, mypart());
      grid.sync();
    PHASE_MARK(7);
      // ---- Phase I: w = (I - V T V^T)[0; x] ----
      reduce_part(pbuf(pc), 0, k, vz, rscr);
      for (int i = tid; i < k; i += blockDim.x) {
        double t = 0.0;
        for (int l = i; l < k; ++l) t += Tsh[i + (size_t)l * nb] * vz[l];
        vh[i] = t;
      }
      __syncthreads();
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        double wv = __ldcg(a.x + r);
#pragma unroll 8
        for (int i = 0; i < k; ++i) wv -= ldr(Vb + r + (size_t)i * lds) * vh[i];
        a.w[r] = wv;
      }
      grid.sync();
    PHASE_MARK(8);
      // ---- Phase J: w2 = B w as chunk partials over the upper staircase ----
      // items (column chunk ch of CWC columns, row tile rb of 32 rows) with
      // rb * 32 < (ch + 1) * CWC, assigned round-robin to CTAs; wide chunks
      // keep each CTA streaming for long stretches (the diagonal chunks also
      // multiply the zeros below the diagonal: m CWC / 2 extra entries)
      {
        constexpr int CWC = HT_TRMV_CW;
        constexpr int RPC = CWC / 32;  // 32-row tiles per column chunk on the diagonal
        const double* Bl = a.B + (size_t)(s + 1) + (size_t)(s + 1) * a.ldb;
        const int nrb = (m + 31) / 32, nchk = (m + CWC - 1) / CWC;
        int total = 0;
        for (int ch = 0; ch < nchk; ++ch) total += min(nrb, RPC * (ch + 1));
        int ch = 0, base = 0, staged = -1;
        for (int item = cta; item < total; item += G) {
          while (item >= base + min(nrb, RPC * (ch + 1))) { base += min(nrb, RPC * (ch + 1)); ++ch; }
          const int rb = item - base;
          const int r0 = rb * 32, rows = min(32, m - r0);
          const int cc = ch * CWC, cols = min(CWC, m - cc);
          if (ch != staged) {  // w(chunk) into shared memory (the inversion scratch is free here)
            for (int c = tid; c < cols; c += blockDim.x) Dsm[c] = __ldcg(a.w + cc + c);
            __syncthreads();
            staged = ch;
          }
          const double sum = gemv32<false>(Bl, a.ldb, r0, rows, cc, cols, Dsm, red4);
          if (tid < rows) a.wpart[(size_t)ch * n + r0 + tid] = sum;
        }
      }
      grid.sync();
      PHASE_MARK(9);
      // ---- Phase K1: w2 rows of this CTA, partial U^T w2 ----
      {
        constexpr int CWC = HT_TRMV_CW;
        const int nchk = (m + CWC - 1) / CWC;
        for (int r = rbeg + tid; r < rend; r += blockDim.x) {
          double v = 0.0;
          for (int ch = r / CWC; ch < nchk; ++ch) v += __ldcg(a.wpart + (size_t)ch * n + r);
          a.w2[r] = v;
        }
        __syncthreads();
        ++pc;
        partial_mty(Ub, lds, STAGE, k + 1, a.w2, rbeg, rend, mypart());
      }
      grid.sync();
      // ---- Phase K: w3 = (I - U S^T U^T) w2, residual, norms ----
      reduce_part(pbuf(pc), 0, k + 1, vz, rscr);
      for (int i = tid; i <= k; i += blockDim.x) {
        double t = 0.0;
        for (int l = 0; l <= i; ++l) t += Ssh[l + (size_t)i * nb] * vz[l];
        vh[i] = t;
      }
      __syncthreads();
      {
        const double sigma = ldexp(1.0, sig_exp);
        double pr = 0.0, px = 0.0, pt = 0.0;
        for (int r = rbeg + tid; r < rend; r += blockDim.x) {
          if (r < k) continue;
          double w3 = __ldcg(a.w2 + r);
#pragma unroll 8
          for (int i = 0; i <= k; ++i) w3 -= ldr(Ub + r + (size_t)i * lds) * vh[i];
          const double rv = ((r == k) ? sigma : 0.0) - w3;
          a.res[r] = rv;
          const double xv = __ldcg(a.x + r);
          pr += rv * rv;
          px += xv * xv;
          if (r > k) pt += xv * xv;
        }
        for (int r = rbeg + tid; r < rend && r < k; r += blockDim.x) a.res[r] = 0.0;
        pr = ht_block_sum(pr, red);
        px = ht_block_sum(px, red);
        pt = ht_block_sum(pt, red);
        ++pc;
        if (tid == 0) { mypart()[0] = pr; mypart()[1] = px; mypart()[2] = pt; }
      }
      grid.sync();
    PHASE_MARK(10);
      // ---- Phase L: iterative-refinement decision (identical in every CTA) ----
      nr2 = reduce_scalar(pbuf(pc), 0, red, false);
      nx2 = reduce_scalar(pbuf(pc), 1, red, false);
      xtail2 = reduce_scalar(pbuf(pc), 2, red, false);
      ok = isfinite(nr2) && isfinite(nx2) && nx2 > 0.0 && sqrt(nr2) <= tol * sqrt(nx2);
      if (!ok && it >= a.max_ir && k == 0 && !subst_mode) {
        // k = 0: the solve with B alone is backward stable by substitution
        // (Sec. 3.2.2c); redo the column without the block inverses
        subst_mode = true;
        it = 0;
        first = true;
        continue;
      }
      if (ok || it >= a.max_ir) break;
      ++it;
      first = false;
    }
    ir_total += it;
    ir_cols += (it > 0);
    if (!ok && k > 0) {
      // undo the left reflector: restore column j (Algorithm 1) and stop
      for (int r = rbeg + tid; r < rend; r += blockDim.x) Aj[r] = a.acol[r];
      failed = 1;
      break;
    }
    // ---- Phase N: right reflector (gamma, v) of x; V column; partial V^T v; GEMV partials ----
    double gamma, vscal;
    {
      const double x0 = __ldcg(a.x + k);
      if (xtail2 == 0.0 || !isfinite(xtail2)) {
        gamma = 0.0; vscal = 0.0;
      } else {
        const double nrm = sqrt(x0 * x0 + xtail2);
        const double al = (x0 >= 0.0) ? -nrm : nrm;
        gamma = (al - x0) / al;
        vscal = 1.0 / (x0 - al);
      }
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        const double v = (r < k) ? 0.0 : (r == k) ? 1.0 : __ldcg(a.x + r) * vscal;
        a.V[r + (size_t)k * ldn] = v;
        if (STAGE) Vs[(r - rbeg) + (size_t)k * lds] = v;
        a.z[r] = v;
      }
      __syncthreads();
      ++pc;
      partial_mty(Vb, lds, STAGE, k, a.z, rbeg, rend, mypart());
    }
    grid.sync();
    PHASE_MARK(12);
    // ---- Phase O: GEMV partials A(s+1:n, j+1:n) v(k:m) ----
    {
      // items: (32-row block, column chunk), about 8 per CTA for balance
      const int p = m - k;  // columns j+1..n-1
      const int nrb = (m + 31) / 32;
      int nch = (8 * G + nrb - 1) / nrb;
      nch = max(1, min(nch, a.ychunks));
      const int cw = (p + nch - 1) / nch;
      const double* Ab = a.A + (size_t)(s + 1) + (size_t)(j + 1) * a.lda;
      const double* vk = a.z + k;  // v(k + c) for column j+1+c
      int staged = -1;
      for (int item = cta; item < nrb * nch; item += G) {
        const int rb = item % nrb, ch = item / nrb;
        const int r0 = rb * 32, rows = min(32, m - r0);
        const int c0 = ch * cw, cols = max(0, min(cw, p - c0));
        double sum;
        if (cw <= 32 * BI) {  // v(chunk) into shared memory (the inversion scratch is free here)
          if (ch != staged) {
            for (int c = tid; c < cols; c += blockDim.x) Dsm[c] = __ldcg(vk + c0 + c);
            __syncthreads();
            staged = ch;
          }
          sum = gemv32<false>(Ab, a.lda, r0, rows, c0, cols, Dsm, red4);
        } else {
          sum = gemv32<true>(Ab, a.lda, r0, rows, c0, cols, vk + c0, red4);
        }
        if (tid < rows) a.ypart[(size_t)ch * n + r0 + tid] = sum;
      }
      // chunks never visited for a row stay unused: the reduction below reads nch chunks
      if (tid == 0) shi[3] = nch;
    }
    grid.sync();
    PHASE_MARK(13);
    // ---- Phase P: T growth, Y(:, k) = gamma (A v - Y V^T v) on rows s+1..n-1 ----
    {
      reduce_part(pbuf(pc), 0, k, vz, rscr);
      for (int i = tid; i < k; i += blockDim.x) {
        double t = 0.0;
        for (int l = i; l < k; ++l) t += Tsh[i + (size_t)l * nb] * vz[l];
        vh[i] = -gamma * t;
      }
      __syncthreads();
      for (int i = tid; i < k; i += blockDim.x) Tsh[i + (size_t)k * nb] = vh[i];
      if (tid == 0) Tsh[k + (size_t)k * nb] = gamma;
      __syncthreads();
      const int nch = shi[3];
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        double av = 0.0;
#pragma unroll 4
        for (int c = 0; c < nch; ++c) av += __ldcg(a.ypart + (size_t)c * n + r);
        double t = 0.0;
#pragma unroll 8
        for (int i = 0; i < k; ++i) t += ldr(Yb + r + (size_t)i * lds) * vz[i];
        const double yv = gamma * (av - t);
        Yl[r + (size_t)k * ldn] = yv;
        if (STAGE) Ys[(r - rbeg) + (size_t)k * lds] = yv;
      }
    }
    grid.sync();
    PHASE_MARK(14);
  }
#undef PHASE_MARK
  if (cta == 0) {
    for (int e = tid; e < nb * nb; e += blockDim.x) { a.S[e] = Ssh[e]; a.T[e] = Tsh[e]; }
    if (tid == 0) {
      a.st->k_done = k;
      a.st->failed = failed;
      a.st->ir_steps = ir_total;
      a.st->cols_with_ir = ir_cols;
      a.st->error = *a.err;
    }
  }
}

// ---------------------------------------------------------------------------
// Preparation of B before a panel: exact zeros below the diagonal (first
// call), ||B||_F, replacement of zero pivots by 2 u rho ||B||_F (Remark 2.2,
// Sec. 3.2.1) and reciprocals of the trailing diagonal for the solve.
// ---------------------------------------------------------------------------
__global__ void zero_lower_kernel(double* B, long ldb, int n) {
  const long total = (long)n * n;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    if (i > c) B[i + (size_t)c * ldb] = 0.0;
  }
}

__global__ void frob_kernel(const double* B, long ldb, int n, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int c = blockIdx.x; c < n; c += gridDim.x)
    for (int i = threadIdx.x; i <= c; i += blockDim.x) {
      const double v = B[i + (size_t)c * ldb];
      acc += v * v;
    }
  acc = ht_block_sum(acc, red);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

__global__ void sqrt_kernel(double* x) { *x = sqrt(*x); }

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the counter c under the
// key (k0, k1), the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// N(0,1) sample by Box-Muller on words 0 and 1 of the block with counter
// (column, index, 0, 0) and key (seed lo, seed hi).
__device__ double philox_normal(uint64_t seed, uint32_t column, uint32_t index) {
  uint32_t c[4] = {column, index, 0u, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  const double u1 = ((double)c[0] + 1.0) * 2.3283064365386963e-10;
  const double u2 = (double)c[1] * 2.3283064365386963e-10;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// raw blocks: in = (counter[4], key[2]) per item, out = block[4] per item
__global__ void philox_block_kernel(int count, const uint32_t* in, uint32_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint32_t c[4] = {in[6 * i], in[6 * i + 1], in[6 * i + 2], in[6 * i + 3]};
  philox4x32_10(c, in[6 * i + 4], in[6 * i + 5]);
  for (int q = 0; q < 4; ++q) out[4 * i + q] = c[q];
}

__global__ void diag_prepare_kernel(double* B, long ldb, int n, int s, uint64_t seed, const double* bnorm,
                                    double* invd, PanelStatus* st) {
  const int m = n - s - 1;
  int cnt = 0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    const int g = s + 1 + r;
    double d = B[g + (size_t)g * ldb];
    if (d == 0.0) {
      d = 2.0 * kU * philox_normal(seed, (uint32_t)s, (uint32_t)g) * (*bnorm);
      if (d == 0.0) d = 2.0 * kU * (*bnorm);
      if (d == 0.0) d = 1.0;  // B == 0: any nonzero pivot keeps the solve defined
      B[g + (size_t)g * ldb] = d;
      ++cnt;
    }
    invd[r] = 1.0 / d;
  }
  if (cnt) atomicAdd(&st->perturbed, cnt);
}

}  // namespace

cudaError_t ht_launch_prepare_B(HtWork& w, double* B, int ldb, int s, uint64_t seed, int first) {
  cudaStream_t st = w.stream;
  const int n = w.n;
  if (first) {
    zero_lower_kernel<<<4 * 152, 256, 0, st>>>(B, ldb, n);
    cudaMemsetAsync(w.bnorm, 0, sizeof(double), st);
    frob_kernel<<<2 * 152, 256, 0, st>>>(B, ldb, n, w.bnorm);
    sqrt_kernel<<<1, 1, 0, st>>>(w.bnorm);
    return cudaGetLastError();
  }
  const int m = n - s - 1;
  if (m > 0) diag_prepare_kernel<<<(m + 255) / 256, 256, 0, st>>>(B, ldb, n, s, seed, w.bnorm, w.invd, w.status);
  return cudaGetLastError();
}

static int g_panel_smem_set = 0;
static const int kPanelSmemMax = 220 * 1024;

static void set_panel_attr() {
  if (g_panel_smem_set) return;
  cudaFuncSetAttribute(panel_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemMax);
  cudaFuncSetAttribute(panel_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPanelSmemMax);
  g_panel_smem_set = 1;
}

cudaError_t ht_launch_panel(HtWork& w, double* A, int lda, const double* B, int ldb, int s, int kmax,
                            double tol_scale, int max_ir) {
  PanelArgs a;
  a.n = w.n; a.s = s; a.kmax = kmax; a.max_ir = max_ir; a.nb = w.nb;
  a.tol_scale = tol_scale;
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb;
  a.U = w.U; a.V = w.V; a.Y = w.Y; a.S = w.S; a.T = w.T;
  const size_t n = w.n;
  a.acol = w.vec + 0 * n; a.ctil = w.vec + 1 * n; a.ytil = w.vec + 2 * n; a.x = w.vec + 3 * n;
  a.res = w.vec + 4 * n; a.w = w.vec + 5 * n; a.w2 = w.vec + 6 * n; a.z = w.vec + 7 * n;
  a.part = w.part; a.ypart = w.ypart; a.ychunks = w.ychunks;
  a.invd = w.invd; a.flags = w.flags; a.exps = w.exps;
  a.epoch0 = w.epoch_host;
  a.st = w.status; a.err = w.err; a.bnorm = w.bnorm;
  // epochs used: at most kmax * (max_ir + 1) solves
  w.epoch_host += (unsigned)((kmax + 1) * (max_ir + 1) + 1);
  const int m = w.n - s - 1;
  a.cap = (m + w.G - 1) / w.G;
  a.ptime = w.ptime;
  a.spin = w.spin > 0 ? w.spin : HT_SPIN_LIMIT;
  a.Xinv = w.Xinv; a.safe = w.safe; a.xmax = w.xmax; a.prog = w.prog; a.nearv = w.nearv; a.wpart = w.wpart;
  size_t smem = smem_doubles(w.nb, a.cap) * sizeof(double);
  a.stage = smem <= (size_t)kPanelSmemMax - 4096;
  if (!a.stage) smem = smem_base_doubles(w.nb) * sizeof(double);
  set_panel_attr();
  void* args[] = {&a};
  if (a.stage)
    return cudaLaunchCooperativeKernel((void*)panel_kernel<true>, dim3(w.G), dim3(HT_THREADS), args, smem, w.stream);
  return cudaLaunchCooperativeKernel((void*)panel_kernel<false>, dim3(w.G), dim3(HT_THREADS), args, smem, w.stream);
}

int ht_panel_max_ctas(int nb) {
  (void)nb;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  set_panel_attr();
  return sms;  // one CTA per SM: the phases are latency-bound, not occupancy-bound
}

extern "C" int ht_philox4x32_10(int count, const uint32_t* in, uint32_t* out, ht_stream_t stream) {
  if (count < 0) return -1;
  if (count > 0 && !in) return -2;
  if (count > 0 && !out) return -3;
  if (count == 0) return HT_OK;
  philox_block_kernel<<<(count + 127) / 128, 128, 0, (cudaStream_t)stream>>>(count, in, out);
  return cudaGetLastError() == cudaSuccess ? HT_OK : HT_ERR_CUDA;
}
