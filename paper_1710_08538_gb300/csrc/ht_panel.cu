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
// DFMA-bound; the triangular solve is a wavefront over 64-row blocks that
// CTAs publish through flags (bounded spins, error word on timeout).
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
};

// Shared-memory layout (doubles): S, T (nb*nb each), vz, vh (nb+1 each),
// red (64), tile (BS*BS), red4 (4*BS), acc (BS).
__host__ __device__ inline size_t smem_doubles(int nb) {
  return 2 * (size_t)nb * nb + 2 * (size_t)(nb + 1) + 64 + BS * BS + 4 * BS + BS;
}

// out[i] = sum_{r in [rb, re)} M(r, i) * y[r] for i < kk, one partial per CTA.
__device__ void partial_mty(const double* M, long ld, int kk, const double* y, int rb, int re, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = wid; i < kk; i += HT_THREADS / 32) {
    double acc = 0.0;
    for (int r = rb + lane; r < re; r += 32) acc += __ldcg(M + r + (size_t)i * ld) * __ldcg(y + r);
    acc = ht_warp_sum(acc);
    if (lane == 0) out[i] = acc;
  }
}

// dst[i] = sum over CTAs of part[c * HT_PART_STRIDE + off + i], i < kk.
// Partials are double-buffered: a phase writes buffer (pc & 1) and the next
// phase reads it, so no CTA overwrites a slot another CTA is still reading.
__device__ void reduce_part(const double* part, int off, int kk, double* dst) {
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {
    double t = 0.0;
    for (int c = 0; c < (int)gridDim.x; ++c) t += __ldcg(part + (size_t)c * HT_PART_STRIDE + off + i);
    dst[i] = t;
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

// Row blocks of the trailing system owned by this CTA, bottom first, in a
// zigzag over CTAs so that heavy (top) and light (bottom) blocks pair up.
__device__ __forceinline__ int zz_block(int q, int G, int nblk) {
  // position q -> block index (bottom first)
  return nblk - 1 - q;
}
__device__ __forceinline__ int zz_owner(int q, int G) {
  int round = q / G, pos = q % G;
  return (round & 1) ? (G - 1 - pos) : pos;
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

// Scaled backward substitution B_loc y = 2^{-E} rhs over 64-row blocks.  On
// return (before the next grid barrier) sol holds the stored block values and
// exps[b] the block exponents: true solution = sol * 2^{exps[b]}.
__device__ void trsv_blocks(const PanelArgs& a, int m, const double* rhs, double* sol, unsigned epoch, double* tile,
                            double* red4, double* acc, double* xl, int* shi) {
  const int G = gridDim.x, nblk = (m + BS - 1) / BS;
  const double* Bl = a.B + (size_t)(a.s + 1) + (size_t)(a.s + 1) * a.ldb;
  const long ldb = a.ldb;
  for (int q = 0; q < nblk; ++q) {
    if (zz_owner(q, G) != (int)blockIdx.x) continue;
    const int i = zz_block(q, G, nblk);
    const int r0 = i * BS, rows = min(BS, m - r0);
    // diagonal tile (upper part) and right-hand side
    for (int e = threadIdx.x; e < BS * BS; e += blockDim.x) {
      int rr = e % BS, cc = e / BS;
      double v = 0.0;
      if (rr < rows && cc < rows && rr <= cc) v = Bl[(size_t)(r0 + rr) + (size_t)(r0 + cc) * ldb];
      if (rr == cc && rr >= rows) v = 1.0;
      tile[e] = v;
    }
    if (threadIdx.x < BS) acc[threadIdx.x] = (threadIdx.x < rows) ? __ldcg(rhs + r0 + threadIdx.x) : 0.0;
    if (threadIdx.x == 0) shi[0] = 0;  // block exponent E
    __syncthreads();
    for (int l = nblk - 1; l > i; --l) {
      if (threadIdx.x == 0) {
        int spins = 0;
        while (ht_ld_acquire(a.flags + l) != (int)epoch) {
          if (++spins > HT_SPIN_LIMIT || ht_ld_acquire(a.err) != 0) {
            atomicCAS(a.err, 0, HT_ERR_TIMEOUT);
            break;
          }
          __nanosleep(32);
        }
        shi[1] = __ldcg(a.exps + l);
      }
      __syncthreads();
      const int c0 = l * BS, cols = min(BS, m - c0);
      if (threadIdx.x < BS) xl[threadIdx.x] = (threadIdx.x < cols) ? __ldcg(sol + c0 + threadIdx.x) : 0.0;
      __syncthreads();
      tile_gemv(Bl, ldb, r0, rows, c0, cols, xl, red4, red4 + 0);  // result in red4[0..BS)
      // red4[0..BS) now holds the tile product (tile_gemv wrote out == red4)
      const int el = shi[1];
      if (threadIdx.x < BS) {
        int E = shi[0];
        double av = acc[threadIdx.x];
        if (el > E) { av = ldexp(av, E - el); E = el; }
        av -= ldexp(red4[threadIdx.x], el - E);
        acc[threadIdx.x] = av;
      }
      __syncthreads();
      if (threadIdx.x == 0 && el > shi[0]) shi[0] = el;
      __syncthreads();
    }
    // substitution inside the block by warp 0 (rows lane, lane + 32)
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double a0 = acc[lane], a1 = acc[lane + 32];
      int E = shi[0];
      for (int c = BS - 1; c >= 0; --c) {
        const double t = __shfl_sync(0xffffffffu, (c >= 32) ? a1 : a0, c & 31);
        const double d = tile[c + c * BS];
        double xc;
        if (c >= rows) {
          xc = 0.0;
        } else {
          if (fabs(t) > ldexp(fabs(d), HT_BIG_EXP)) {
            // rescale the whole block so that |x_c| stays below 2^500
            int sh = ilogb(t) - ilogb(d) - HT_BIG_EXP + 2;
            a0 = ldexp(a0, -sh);
            a1 = ldexp(a1, -sh);
            E += sh;
            const double t2 = ldexp(t, -sh);
            xc = t2 * a.invd[r0 + c];
          } else {
            xc = t * a.invd[r0 + c];
          }
        }
        if (lane == (c & 31)) {
          if (c >= 32) a1 = xc; else a0 = xc;
        }
        if (lane < c) a0 -= tile[lane + c * BS] * xc;
        if (lane + 32 < c) a1 -= tile[lane + 32 + c * BS] * xc;
      }
      if (lane < rows) sol[r0 + lane] = a0;
      if (lane + 32 < rows) sol[r0 + lane + 32] = a1;
      if (lane == 0) a.exps[i] = E;
      __threadfence();
      __syncwarp();
      if (lane == 0) ht_st_release(a.flags + i, (int)epoch);
    }
    __syncthreads();
  }
}

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
  __shared__ int shi[4];
  __shared__ double xl[BS];

  const int n = a.n, s = a.s, m = n - s - 1, G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const long ldn = n;
  const int chunk = (m + G - 1) / G;
  const int rbeg = min(m, cta * chunk), rend = min(m, rbeg + chunk);
  const double tol = a.tol_scale * 2.0 * kU * (*a.bnorm);
  double* Yl = a.Y + (s + 1);
  int pc = 0;  // phase counter selecting the partial-sum buffer
  auto pbuf = [&](int c) { return a.part + (size_t)(c & 1) * G * HT_PART_STRIDE; };
  auto mypart = [&]() { return pbuf(pc) + (size_t)cta * HT_PART_STRIDE; };

  for (int e = tid; e < nb * nb; e += blockDim.x) { Ssh[e] = 0.0; Tsh[e] = 0.0; }
  __syncthreads();

  unsigned epoch = a.epoch0;
  int k = 0, failed = 0, ir_total = 0, ir_cols = 0;
  for (k = 0; k < a.kmax; ++k) {
    const int j = s + k;
    double* Aj = a.A + (size_t)j * a.lda + (s + 1);  // local rows of column j
    // ---- Phase A: right update of column j, save it, partial U^T a ----
    for (int r = rbeg + tid; r < rend; r += blockDim.x) {
      double xv = Aj[r];
      a.acol[r] = xv;
      double t = 0.0;
      for (int i = 0; i < k; ++i) t += __ldcg(Yl + r + (size_t)i * ldn) * __ldcg(a.V + (k - 1) + (size_t)i * ldn);
      Aj[r] = xv - t;
    }
    __syncthreads();
    ++pc;
    partial_mty(a.U, ldn, k, Aj, rbeg, rend, mypart());
    grid.sync();
    // ---- Phase B: left update (I - U S^T U^T), tail norm ----
    reduce_part(pbuf(pc), 0, k, vz);
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
        for (int i = 0; i < k; ++i) xv -= __ldcg(a.U + r + (size_t)i * ldn) * vh[i];
        Aj[r] = xv;
        if (r > k) tail += xv * xv;
      }
      tail = ht_block_sum(tail, red);
      ++pc;
      if (tid == 0) mypart()[0] = tail;
    }
    grid.sync();
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
        if (r == k) Aj[r] = alpha;
        else if (r > k) Aj[r] = 0.0;
      }
      __syncthreads();
      ++pc;
      partial_mty(a.U, ldn, k, a.U + (size_t)k * ldn, rbeg, rend, mypart());
    }
    grid.sync();
    // ---- Phase D: S growth; first right-hand side c~ = e_k - U (S U(k,:)^T) ----
    reduce_part(pbuf(pc), 0, k, vz);
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
    bool first = true, ok = false;
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
          for (int i = 0; i <= k; ++i) c -= __ldcg(a.U + r + (size_t)i * ldn) * vh[i];
          a.ctil[r] = c;
        }
      } else {
        // c~ = (I - U S U^T)[0; res]: partial U^T [0; res]
        ++pc;
        partial_mty(a.U, ldn, k + 1, a.res, rbeg, rend, mypart());
        grid.sync();
        reduce_part(pbuf(pc), 0, k + 1, vz);
        for (int i = tid; i <= k; i += blockDim.x) {
          double t = 0.0;
          for (int l = i; l <= k; ++l) t += Ssh[i + (size_t)l * nb] * vz[l];
          vh[i] = t;
        }
        __syncthreads();
        for (int r = rbeg + tid; r < rend; r += blockDim.x) {
          double c = __ldcg(a.res + r);
          for (int i = 0; i <= k; ++i) c -= __ldcg(a.U + r + (size_t)i * ldn) * vh[i];
          a.ctil[r] = c;
        }
      }
      grid.sync();
      // ---- Phase E: scaled backward substitution B y~ = 2^-E c~ ----
      trsv_blocks(a, m, a.ctil, a.ytil, epoch, tile, red4, acc, xl, shi);
      ++epoch;
      grid.sync();
      // ---- Phase F: common exponent, partial V^T y~ ----
      const int nblk = (m + BS - 1) / BS;
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
        const int e = __ldcg(a.exps + r / BS);
        a.ytil[r] = ldexp(__ldcg(a.ytil + r), e - emax);
      }
      __syncthreads();
      ++pc;
      partial_mty(a.V, ldn, k, a.ytil, rbeg, rend, mypart());
      grid.sync();
      // ---- Phase G: x = [(I - V T^T V^T) y~](k:m), combine with the IR iterate ----
      reduce_part(pbuf(pc), 0, k, vz);
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
            for (int i = 0; i < k; ++i) d -= __ldcg(a.V + r + (size_t)i * ldn) * vh[i];
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
      partial_mty(a.V, ldn, k, a.x, rbeg, rend, mypart());
      grid.sync();
      // ---- Phase I: w = (I - V T V^T)[0; x] ----
      reduce_part(pbuf(pc), 0, k, vz);
      for (int i = tid; i < k; i += blockDim.x) {
        double t = 0.0;
        for (int l = i; l < k; ++l) t += Tsh[i + (size_t)l * nb] * vz[l];
        vh[i] = t;
      }
      __syncthreads();
      for (int r = rbeg + tid; r < rend; r += blockDim.x) {
        double wv = __ldcg(a.x + r);
        for (int i = 0; i < k; ++i) wv -= __ldcg(a.V + r + (size_t)i * ldn) * vh[i];
        a.w[r] = wv;
      }
      grid.sync();
      // ---- Phase J: w2 = B w (row blocks), partial U^T w2 over owned blocks ----
      {
        const double* Bl = a.B + (size_t)(s + 1) + (size_t)(s + 1) * a.ldb;
        double up = 0.0;
        for (int q = 0; q < nblk; ++q) {
          if (zz_owner(q, G) != cta) continue;
          const int i = zz_block(q, G, nblk);
          const int r0 = i * BS, rows = min(BS, m - r0);
          double accb = 0.0;
          for (int c0 = r0; c0 < m; c0 += BS) {
            const int cols = min(BS, m - c0);
            if (tid < BS) xl[tid] = (tid < cols) ? __ldcg(a.w + c0 + tid) : 0.0;
            __syncthreads();
            tile_gemv(Bl, a.ldb, r0, rows, c0, cols, xl, red4, red4);
            if (tid < BS) accb += red4[tid];
            __syncthreads();
          }
          if (tid < BS) acc[tid] = accb;
          if (tid < rows) a.w2[r0 + tid] = accb;
          __syncthreads();
          // partial U^T w2 over this block: thread i handles column i
          for (int c = tid; c <= k; c += blockDim.x) {
            double t = 0.0;
            for (int rr = 0; rr < rows; ++rr) t += __ldcg(a.U + r0 + rr + (size_t)c * ldn) * acc[rr];
            if (c == tid) up += t;
          }
          __syncthreads();
        }
        ++pc;
        for (int c = tid; c <= k; c += blockDim.x) mypart()[c] = up;
      }
      grid.sync();
      // ---- Phase K: w3 = (I - U S^T U^T) w2, residual, norms ----
      reduce_part(pbuf(pc), 0, k + 1, vz);
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
          for (int i = 0; i <= k; ++i) w3 -= __ldcg(a.U + r + (size_t)i * ldn) * vh[i];
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
      // ---- Phase L: iterative-refinement decision (identical in every CTA) ----
      nr2 = reduce_scalar(pbuf(pc), 0, red, false);
      nx2 = reduce_scalar(pbuf(pc), 1, red, false);
      xtail2 = reduce_scalar(pbuf(pc), 2, red, false);
      ok = isfinite(nr2) && isfinite(nx2) && nx2 > 0.0 && sqrt(nr2) <= tol * sqrt(nx2);
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
        a.z[r] = v;
      }
      __syncthreads();
      ++pc;
      partial_mty(a.V, ldn, k, a.z, rbeg, rend, mypart());
    }
    grid.sync();
    // ---- Phase O: GEMV partials A(s+1:n, j+1:n) v(k:m) ----
    {
      const int p = m - k;  // columns j+1..n-1
      const int nrb = (m + BS - 1) / BS;
      int nch = (2 * G + nrb - 1) / nrb;
      nch = max(1, min(nch, a.ychunks));
      const int cw = (p + nch - 1) / nch;
      const double* Ab = a.A + (size_t)(s + 1) + (size_t)(j + 1) * a.lda;
      const double* vk = a.z + k;  // v(k + c) for column j+1+c
      for (int item = cta; item < nrb * nch; item += G) {
        const int rb = item % nrb, ch = item / nrb;
        const int r0 = rb * BS, rows = min(BS, m - r0);
        const int c0 = ch * cw, cols = min(cw, p - c0);
        double sum = 0.0;
        for (int cc = 0; cc < cols; cc += BS) {
          const int cn = min(BS, cols - cc);
          if (tid < BS) xl[tid] = (tid < cn) ? __ldcg(vk + c0 + cc + tid) : 0.0;
          __syncthreads();
          tile_gemv(Ab, a.lda, r0, rows, c0 + cc, cn, xl, red4, red4);
          if (tid < BS) sum += red4[tid];
          __syncthreads();
        }
        if (tid < rows) a.ypart[(size_t)ch * n + r0 + tid] = (cols > 0) ? sum : 0.0;
      }
      // chunks never visited for a row stay unused: the reduction below reads nch chunks
      if (tid == 0) shi[3] = nch;
    }
    grid.sync();
    // ---- Phase P: T growth, Y(:, k) = gamma (A v - Y V^T v) on rows s+1..n-1 ----
    {
      reduce_part(pbuf(pc), 0, k, vz);
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
        for (int c = 0; c < nch; ++c) av += __ldcg(a.ypart + (size_t)c * n + r);
        double t = 0.0;
        for (int i = 0; i < k; ++i) t += __ldcg(Yl + r + (size_t)i * ldn) * vz[i];
        Yl[r + (size_t)k * ldn] = gamma * (av - t);
      }
    }
    grid.sync();
  }
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

// Philox4x32-10 (Salmon et al., SC'11) and Box-Muller, keyed like the oracle:
// counter (column, index, 0, 0), key (seed lo, seed hi).
__device__ double philox_normal(uint64_t seed, uint32_t column, uint32_t index) {
  uint32_t c0 = column, c1 = index, c2 = 0, c3 = 0;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  const double u1 = ((double)c0 + 1.0) * 2.3283064365386963e-10;
  const double u2 = (double)c1 * 2.3283064365386963e-10;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
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
  w.epoch_host += (unsigned)(kmax * (max_ir + 1) + 1);
  const size_t smem = smem_doubles(w.nb) * sizeof(double);
  if (!g_panel_smem_set) {
    cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    g_panel_smem_set = 1;
  }
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((void*)panel_kernel, dim3(w.G), dim3(HT_THREADS), args, smem, w.stream);
}

int ht_panel_max_ctas(int nb) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  g_panel_smem_set = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, panel_kernel, HT_THREADS, smem_doubles(nb) * sizeof(double));
  if (per < 1) per = 1;
  return sms * 1;  // one CTA per SM: the phases are latency-bound, not occupancy-bound
}
