// C ABI of libht: Algorithm 1 (HouseHT) of Bujanovic, Karlsson, Kressner
// (arXiv 1710.08538) driven from the host.  Per panel: one cooperative
// launch reduces up to nb columns (Sec. 3.2) and reports how many reflector
// pairs it produced (fewer on an IR failure); the host then queues the
// absorption of Sec. 3.3 (right reflectors, then left reflectors) and moves
// the panel start s by k.  The only host/device synchronisation is the read
// of that count, once per panel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <thread>
#include <atomic>
#include <vector>

#include "ht_common.cuh"
#include "ht_tuned.h"

namespace {

// device status word of the last call, per stream (ht_last_device_status)
std::mutex g_status_mu;
std::vector<std::pair<cudaStream_t, int>> g_status;
void set_stream_status(cudaStream_t st, int v) {
  std::lock_guard<std::mutex> lk(g_status_mu);
  for (auto& e : g_status)
    if (e.first == st) { e.second = v; return; }
  g_status.push_back({st, v});
}

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
  int dev, n, nb;             // n: the order the buffer was sized for
  int cur_n;                  // the order its workspace is laid out for now (<= n)
  int G;                      // CTAs of the cooperative panel on the whole GPU
  bool busy;
  HtWork w;
  void* base;
  PanelStatus* host_status;  // pinned
  unsigned long long* pt_dev; // panel phase timers
};
std::mutex g_pool_mu;
std::vector<PoolEntry*> g_pool;

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// Workspace layout for order n, panel width nb and G CTAs in the cooperative
// panel: returns the bytes needed; when b is not null, carves the pointers of
// w (and *pt, the profile timers) out of the buffer at b.
size_t ht_layout_work(HtWork& w, char* b, int n, int nb, int G, unsigned long long** pt, bool side) {
  std::memset(&w, 0, sizeof(w));
  w.n = n;
  w.nb = nb;
  w.G = G;
  w.ychunks = 4;
  w.spin = HT_SPIN_LIMIT;
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
  const size_t oU2w = take(nn * nb);
  const size_t oSmall = take((size_t)4 * 2 * HT_NB_MAX * HT_NB_MAX);
  const size_t oFlags = take((size_t)nblk);  // ints, over-allocated as doubles
  const size_t oExps = take((size_t)nblk);
  const size_t oMisc = take(16);
  const size_t oPt = take(32);
  const int nbi = (n + HT_TRSV_BI - 1) / HT_TRSV_BI + 1;
  const size_t oXinv = take((size_t)nbi * HT_TRSV_BI * HT_TRSV_BI);
  const size_t oSafe = take((size_t)nbi);
  const size_t oXmax = take((size_t)32 * nbi + 256);
  const size_t oProg = take((size_t)G), oNear = take(HT_TRSV_BI);
  const size_t oTst = take(nn * nb + 4 * (size_t)nb * nb);  // (p/k + 1) T factors of k^2 each
  const size_t oWpart = take((size_t)((n + HT_TRMV_CW - 1) / HT_TRMV_CW + 1) * nn);
  // digits of the emulated sweeps: windows of a chain are processed in launches of emu_cap windows
  const size_t emu_win = nb <= 32 ? ht_tc_group_bytes() : 0;
  w.emu_cap = std::min(n / 32 + 4, 1024);
  const size_t oEmu = take(emu_win ? (emu_win * w.emu_cap + sizeof(double) - 1) / sizeof(double) : 0);
  const size_t oEmuE = take((size_t)w.emu_cap);
  const size_t oEmuG = take(2 * (size_t)w.emu_cap);  // int4 = 2 doubles
  const size_t oCf = take((size_t)n + 8);  // 2 (n + 8) ints
  const size_t oRc = take(2);
  const size_t oRt = take(nn + 2 * HT_NB_MAX);
  // work-unit counters of the tcgen05 sweeps: 1 + line blocks of up to HT_SWEEP_MAXJOBS jobs
  const size_t oTs = take((size_t)(1 + HT_SWEEP_MAXJOBS * (n / 128 + 1)) / 2 + 1);
  // the side stream's sweeps: digits, bounds, table, unit counters of their own
  const size_t oEmu2 = side ? take(emu_win ? (emu_win * w.emu_cap + sizeof(double) - 1) / sizeof(double) : 0) : 0;
  const size_t oEmuE2 = side ? take((size_t)w.emu_cap) : 0;
  const size_t oEmuG2 = side ? take(2 * (size_t)w.emu_cap) : 0;
  const size_t oTs2 = side ? take((size_t)(1 + HT_SWEEP_MAXJOBS * (n / 128 + 1)) / 2 + 1) : 0;
  if (!b) return total;
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
  w.U2w = (double*)(b + oU2w);
  w.small = (double*)(b + oSmall);
  w.flags = (int*)(b + oFlags);
  w.exps = (int*)(b + oExps);
  char* misc = b + oMisc;
  w.epoch = (unsigned*)misc;
  w.err = (int*)(misc + 16);
  w.status = (PanelStatus*)(misc + 64);
  w.epoch_host = 1;
  w.ptime = nullptr;
  w.Xinv = (double*)(b + oXinv);
  w.safe = (int*)(b + oSafe);
  w.xmax = (double*)(b + oXmax);
  w.prog = (unsigned long long*)(b + oProg);
  w.nearv = (double*)(b + oNear);
  w.emu_dig = emu_win ? (void*)(b + oEmu) : nullptr;
  w.emu_exps = (int*)(b + oEmuE);
  w.emu_geo = (void*)(b + oEmuG);
  w.rcount = (int*)(b + oRc);
  w.cflags = (int*)(b + oCf);
  w.rtaus = (double*)(b + oRt);
  w.tc_sched = (int*)(b + oTs);
  if (side) {
    w.emu_dig2 = emu_win ? (void*)(b + oEmu2) : nullptr;
    w.emu_exps2 = (int*)(b + oEmuE2);
    w.emu_geo2 = (void*)(b + oEmuG2);
    w.tc_sched2 = (int*)(b + oTs2);
  }
  w.wpart = (double*)(b + oWpart);
  w.tstore = (double*)(b + oTst);
  if (pt) *pt = (unsigned long long*)(b + oPt);
  return total;
}

namespace {

int alloc_work(PoolEntry* e, int n, int nb) {
  HtWork& w = e->w;
  const int G = ht_panel_max_ctas(nb);
  const size_t total = ht_layout_work(w, nullptr, n, nb, G, nullptr, true);
  void* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) return HT_ERR_NOMEM;
  cudaMemset(base, 0, total);
  ht_layout_work(w, (char*)base, n, nb, G, &e->pt_dev, true);
  e->base = base;
  e->G = G;
  e->cur_n = n;
  // the side stream of the Q / Z updates and its events (without them, one stream)
  if (cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking) != cudaSuccess) {
    w.side = nullptr;
    cudaGetLastError();
  }
  for (int i = 0; i < 5 && w.side; ++i)
    if (cudaEventCreateWithFlags(&w.side_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      for (int q = 0; q < i; ++q) cudaEventDestroy(w.side_ev[q]);
      cudaStreamDestroy(w.side);
      w.side = nullptr;
      cudaGetLastError();
    }
  if (cudaMallocHost((void**)&e->host_status, sizeof(PanelStatus)) != cudaSuccess) {
    cudaFree(base);
    return HT_ERR_NOMEM;
  }
  return HT_OK;
}

// A free workspace laid out for order n, or else the smallest free one sized
// for an order in [n, 2n] (laid out again for n, cleared: its epoch-stamped
// progress words start over), or else a new one.
PoolEntry* acquire(int n, int nb, int* rc) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (PoolEntry* e : g_pool)
    if (!e->busy && e->dev == dev && e->cur_n == n && e->nb == nb) {
      e->busy = true;
      *rc = HT_OK;
      return e;
    }
  PoolEntry* best = nullptr;
  for (PoolEntry* e : g_pool)
    if (!e->busy && e->dev == dev && e->nb == nb && e->n >= n && e->n <= 2 * n && (!best || e->n < best->n)) best = e;
  if (best) {
    HtWork& w = best->w;
    const cudaStream_t side = w.side;
    cudaEvent_t ev[5];
    for (int i = 0; i < 5; ++i) ev[i] = w.side_ev[i];
    best->cur_n = -1;  // until the clear below succeeds
    const size_t bytes = ht_layout_work(w, (char*)best->base, n, nb, best->G, &best->pt_dev, true);
    w.side = side;
    for (int i = 0; i < 5; ++i) w.side_ev[i] = ev[i];
    if (cudaMemset(best->base, 0, bytes) != cudaSuccess) {
      *rc = HT_ERR_CUDA;
      return nullptr;
    }
    best->cur_n = n;
    best->busy = true;
    *rc = HT_OK;
    return best;
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

// Optional per-launch timing by class (ht_options.profile): an event pair
// around each launch, resolved after the stream is synchronised.
struct Prof {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  std::vector<cudaEvent_t> pool;
  double ms[HT_NCLASS] = {};
  double flops[HT_NCLASS] = {};
  long long launches[HT_NCLASS] = {};
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  int cls = 0;
  cudaEvent_t cur = nullptr;
  cudaStream_t side = nullptr;  // the side stream (also synchronised by resolve)
  cudaStream_t lst = nullptr;   // stream of the current launch
  void begin(int c, cudaStream_t s = nullptr) {
    cls = c;
    lst = s ? s : st;
    if (!on) return;
    cur = get();
    cudaEventRecord(cur, lst);
  }
  void end(double fl) {
    flops[cls] += fl;
    launches[cls] += 1;
    if (!on) return;
    cudaEvent_t e = get();
    cudaEventRecord(e, lst);
    pending.push_back({cls, {cur, e}});
  }
  void resolve() {
    if (!on) return;
    cudaStreamSynchronize(st);
    if (side) cudaStreamSynchronize(side);
    for (auto& p : pending) {
      float t = 0.f;
      cudaEventElapsedTime(&t, p.second.first, p.second.second);
      ms[p.first] += t;
      pool.push_back(p.second.first);
      pool.push_back(p.second.second);
    }
    pending.clear();
  }
  ~Prof() {
    for (auto& p : pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct Ctx {
  HtWork* w;
  cudaStream_t st;
  int n;
  double *A, *B, *Q, *Z;
  long lda, ldb, ldq, ldz;
  int want_qz;
  double flops;
  Prof* prof;
  // a mode-3 Q sweep left to the side stream of the next absorption (or the end)
  struct { bool on; int p, k, j, nlb; long wst; } pendq;
};

// Launch `expr` as one timed launch of class `cls` with `fl` algorithmic flops.
#define LAUNCH(cls, fl, expr)            \
  do {                                   \
    c.prof->begin(cls);                  \
    cudaError_t e_ = (expr);             \
    if (e_ != cudaSuccess) return e_;    \
    c.prof->end(fl);                     \
    c.flops += (fl);                     \
  } while (0)

// the same on the side stream (class HT_CLASS_SIDE)
#define LAUNCH_SIDE(fl, expr)                     \
  do {                                            \
    c.prof->begin(HT_CLASS_SIDE, c.w->side);      \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return e_;             \
    c.prof->end(fl);                              \
    c.flops += (fl);                              \
  } while (0)

#define CK(call)                         \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) return e_;    \
  } while (0)

// Flop counts of the launches (the algorithmic work each performs).
double fl_gemm(double M, double N, double K) { return 2.0 * M * N * K; }
double fl_window(double w, double k) { return 2.0 * w * k * k - 2.0 / 3.0 * k * k * k + 2.0 * w * k * k; }
double fl_chain(int p, int k) {  // one chain; both chains have the same windows
  double f = 0.0;
  for (int i = 0; i < ht_num_windows(p, k); ++i) {
    int r0, r1;
    ht_ql_window(p, k, i, &r0, &r1);
    f += fl_window(r1 - r0, k);
  }
  return f;
}
// right sweep of chain `mode` over `rows` rows; limit_base >= 0 clips rows to the structural bound
double fl_sweep(int mode, int p, int k, int nwin, double lines, int limit_base, bool left) {
  double f = 0.0;
  for (int t = 0; t < nwin; ++t) {
    int w = 0, kr = 0, lim = 0;
    if (mode == 0) { int a, b; ht_ql_window(p, k, t, &a, &b); w = b - a; kr = k; lim = b; }
    else if (mode == 1) { int a, b; ht_qr_window(p, k, t, &a, &b); w = b - a; kr = k; lim = a; }
    else if (mode == 2) {
      const int nbr = ht_num_right_blocks(p, k), bb = nbr - 1 - t;
      int c0, c1, d0, d1;
      ht_right_block(p, k, bb - 1, &c0, &c1);
      ht_right_block(p, k, bb, &d0, &d1);
      w = d1 - c0; kr = d1 - d0; lim = d0;
    } else {
      const int nlb = ht_num_left_blocks(p, k);
      int r0, r1, e0, e1;
      ht_left_block(p, k, t, &r0, &r1);
      if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
      w = e1 - r0; kr = r1 - r0; lim = r1;
    }
    double L = lines;
    if (limit_base >= 0) L = left ? std::max(0.0, lines - (double)lim) : std::min(lines, (double)(limit_base + lim));
    f += 4.0 * L * w * kr;
  }
  return f;
}

// Overlap of the Q / Z updates (emulated path): the main stream's cooperative
// restore launches take at most RS_MAIN_CTAS CTAs, the side stream's sweeps the
// other SMs, so that both are resident together whatever runs first.
constexpr int RS_MAIN_CTAS = 88;
// CTAs per lane of ht_reduce_batched (at least the restore kernel's 20 roles)
constexpr int BATCH_LANE_CTAS = 25;
int sm_count() {
  static int sms[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (sms[dev] == 0) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  return sms[dev];
}
int side_ctas() { return std::max(1, sm_count() - RS_MAIN_CTAS); }

// One fused chain application, native FP64 or emulated (HT_PREC_EMU).
cudaError_t run_sweep(Ctx& c, const HtSweepJob* jobs, int njobs, const double* wy, long wst, int mode, int p, int k,
                      int t0, int t1, bool on_side = false) {
  if (on_side) {
    // the side stream: its own buffers, at most RS_SIDE_CTAS CTAs (the rest of the
    // GPU stays free for the cooperative restore of the main stream)
    return ht_tc_sweep_multi(c.w->side, jobs, njobs, wy, wst, mode, p, k, t0, t1, c.w->emu_dig2, c.w->emu_exps2,
                             c.w->emu_geo2, c.w->emu_cap, c.w->tc_sched2, c.w->err, side_ctas());
  }
  if (c.w->prec == HT_PREC_EMU)
    return ht_tc_sweep_multi(c.st, jobs, njobs, wy, wst, mode, p, k, t0, t1, c.w->emu_dig, c.w->emu_exps,
                             c.w->emu_geo, c.w->emu_cap, c.w->tc_sched, c.w->err, c.w->cap);
  // the FP64 sweeps take the windows one by one: they are DFMA-bound, and a merged window
  // of g windows multiplies their flops by about g / 2
  return ht_sweep_multi(c.st, jobs, njobs, wy, wst, mode, p, k, t0, t1);
}

// Restore chain on B (mode 2: RQ, Sec. 3.3.1e; mode 3: QR, Sec. 3.3.2f), fl
// flops in all.  seg: in segments of RS_SEG steps, each launch updating only
// the lines its own steps need, followed by an emulated sweep of the
// segment's transforms on the remaining lines of B (rows 0 .. j as well for
// the RQ chain); otherwise one launch.
constexpr int RS_SEG = 64;
// flops of restore steps [ta, tb) whose updates reach the lines [blo, bhi): the
// factorization of each block and its transform on the trailing lines of B
double fl_restore(int mode, int p, int k, int ta, int tb, int blo, int bhi) {
  double f = 0.0;
  for (int t = ta; t < tb; ++t) {
    int w, kr, lim;
    if (mode == 2) {
      const int bb = ht_num_right_blocks(p, k) - 1 - t;
      int c0, c1, d0, d1;
      ht_right_block(p, k, bb - 1, &c0, &c1);
      ht_right_block(p, k, bb, &d0, &d1);
      w = d1 - c0; kr = d1 - d0; lim = d0;
      f += fl_window(w, kr) + 4.0 * std::max(0, lim - blo) * w * kr;
    } else {
      const int nlb = ht_num_left_blocks(p, k);
      int r0, r1, e0, e1;
      ht_left_block(p, k, t, &r0, &r1);
      if (t + 1 < nlb) ht_left_block(p, k, t + 1, &e0, &e1); else e1 = r1;
      w = e1 - r0; kr = r1 - r0; lim = r1;
      f += fl_window(w, kr) + 4.0 * std::max(0, bhi - lim) * w * kr;
    }
  }
  return f;
}

cudaError_t restore_chain(Ctx& c, int mode, int p, int k, int j, double* wy, long wst, bool seg, int max_ctas = 0) {
  HtWork& w = *c.w;
  const int nsteps = ht_restore_steps(mode, p, k);
  if (nsteps <= 0) return cudaSuccess;
  const double* wyc = wy;
  if (!seg) {
    LAUNCH(HT_CLASS_RESTORE, fl_restore(mode, p, k, 0, nsteps, 0, p),
           ht_launch_restore(c.st, mode, p, k, j, c.n, c.B, c.ldb, wy, wst, w.tstore, w.rtaus, w.rcount, w.err,
                             w.ptime, w.spin, 0, -1, max_ctas));
    return cudaSuccess;
  }
  for (int ta = 0; ta < nsteps; ta += RS_SEG) {
    const int tb = std::min(nsteps, ta + RS_SEG);
    int blo0 = 0, bhi0 = p;
    if (tb < nsteps) ht_restore_band(mode, p, k, tb, &blo0, &bhi0);
    LAUNCH(HT_CLASS_RESTORE, fl_restore(mode, p, k, ta, tb, blo0, bhi0),
           ht_launch_restore(c.st, mode, p, k, j, c.n, c.B, c.ldb, wy, wst, w.tstore, w.rtaus, w.rcount, w.err,
                             w.ptime, w.spin, ta, tb, max_ctas));
    int blo = 0, bhi = p;
    if (tb < nsteps) ht_restore_band(mode, p, k, tb, &blo, &bhi);
    if (mode == 2) {
      // rows 0 .. j + blo of B: rows above the segment's band, including rows 0 .. j
      // (only those for the last segment, blo = 0)
      const HtSweepJob job = {c.B, c.ldb, 1, 0, j + 1 + blo, j + 1, 0, 0};
      LAUNCH(HT_CLASS_SWEEP, fl_sweep(2, p, k, tb, j + 1 + blo, -1, false) - fl_sweep(2, p, k, ta, j + 1 + blo, -1, false),
             run_sweep(c, &job, 1, wyc, wst, 2, p, k, ta, tb));
    } else if (mode == 3 && bhi < p) {
      // columns j + 1 + bhi .. n - 1 of B, right of the segment's band
      const HtSweepJob job = {c.B, c.ldb, 0, j + 1 + bhi, p - bhi, j + 1, 0, 0};
      LAUNCH(HT_CLASS_SWEEP, fl_sweep(3, p, k, tb, p - bhi, -1, true) - fl_sweep(3, p, k, ta, p - bhi, -1, true),
             run_sweep(c, &job, 1, wyc, wst, 3, p, k, ta, tb));
    }
  }
  return cudaSuccess;
}

// The deferred last Q sweep (mode 3, Sec. 3.3.2 (d) step 4) of the previous
// absorption, on the side stream; side_ev[3] marks its end (the main stream
// waits for it before the QR restore overwrites its WY store).
cudaError_t flush_pendq(Ctx& c) {
  HtWork& w = *c.w;
  if (c.pendq.on) {
    const auto& d = c.pendq;
    const HtSweepJob jq = {c.Q, c.ldq, 1, 0, c.n, d.j + 1, 0, 0};
    LAUNCH_SIDE(fl_sweep(3, d.p, d.k, d.nlb, c.n, -1, false),
                run_sweep(c, &jq, 1, w.wyLR, d.wst, 3, d.p, d.k, 0, d.nlb, true));
    c.pendq.on = false;
  }
  return cudaEventRecord(w.side_ev[3], w.side);
}

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
  const size_t wsd = (size_t)n * 2 * nb;  // split-K partials live in tmp2
  LAUNCH(HT_CLASS_GEMM, fl_gemm(s + 1, k, m),
         ht_gemm_ws(st, 'N', 'N', s + 1, k, m, 1.0, A + (size_t)(s + 1) * lda, lda, V, n, 0.0, w.tmp1, n, w.tmp2, wsd));
  LAUNCH(HT_CLASS_GEMM, fl_gemm(s + 1, k, k), ht_gemm(st, 'N', 'N', s + 1, k, k, 1.0, w.tmp1, n, w.T, nb, 0.0, w.Y, n));

  // ---- right reflectors, Sec. 3.3.1 ----
  // deferred rows 0..s of the panel columns s+1..j-1, then column j (step e2)
  if (k > 1)
    LAUNCH(HT_CLASS_GEMM, fl_gemm(s + 1, k - 1, k),
           ht_gemm(st, 'N', 'T', s + 1, k - 1, k, -1.0, w.Y, n, V, n, 1.0, A + (size_t)(s + 1) * lda, lda));
  LAUNCH(HT_CLASS_GEMM, fl_gemm(n, 1, k),
         ht_gemm(st, 'N', 'T', n, 1, k, -1.0, w.Y, n, V + (k - 1), n, 1.0, A + (size_t)j * lda, lda));
  // (b) V2 = Q^_1 .. Q^_r L^ (eq. (5)) and, concurrently, U2 = Q~_1 .. Q~_r R~
  // (eq. (7), Sec. 3.3.2b) on a copy of U2 (the spike update needs U2 itself)
  const int nwr = ht_num_windows(p, k);
  LAUNCH(HT_CLASS_OTHER, 0.0,
         cudaMemcpy2DAsync(w.U2w, n * sizeof(double), U + k, n * sizeof(double), p * sizeof(double), k,
                           cudaMemcpyDeviceToDevice, st));
  if (k <= 32)
    LAUNCH(HT_CLASS_CHAIN_FACTOR, 2.0 * fl_chain(p, k),
           ht_launch_chains_wave(st, V + k, w.U2w, n, p, k, w.wyR, w.wyL, wst, w.L1, w.R1, w.tmp1, w.tmp3, w.cflags,
                                 w.err, w.spin, w.cap));
  else
    LAUNCH(HT_CLASS_CHAIN_FACTOR, 2.0 * fl_chain(p, k),
           ht_launch_chains(st, V + k, w.U2w, n, p, k, w.wyR, w.wyL, wst, w.L1, w.R1));
  // Emulated path with a side stream: the Q and Z updates (sweeps and rank-k
  // corrections) go to the side stream, launched when the main stream starts a
  // restore chain, which leaves most of the GPU idle (the restore takes at most
  // RS_MAIN_CTAS CTAs): during the RQ restore the previous absorption's last Q
  // sweep (mode 3) and the Z sweep and rank-k of this one; during the QR restore
  // the Q sweep (mode 1), the second Z sweep (mode 2) and the Q rank-k.  The
  // main stream waits for the side stream before the next panel (the data these
  // read) and for the deferred Q sweep before the QR restore (its WY store).
  const int nbr = ht_num_right_blocks(p, k);
  const int nlb = ht_num_left_blocks(p, k);
  const bool seg = w.prec == HT_PREC_EMU && k <= 32;
  const bool ov = seg && w.side && w.cap == 0;
  const int rs_ctas = ov ? RS_MAIN_CTAS : w.cap;
  const double fl_rk = dn * (4.0 * k * k + 6.0 * k * k);
  const double fl_rkl = 8.0 * k * k + 2.0 * k * k;
  // (c)-(e) step 1: A, Z, B columns j+1..n-1 times the chain, one fused launch
  {
    const HtSweepJob jobs[3] = {{A, lda, 1, 0, n, j + 1, 0, 0},
                                {B, ldb, 1, 0, n, j + 1, 1, j + 1},
                                {Z, ldz, 1, 0, (c.want_qz && !ov) ? n : 0, j + 1, 0, 0}};
    const double fl = fl_sweep(0, p, k, nwr, n, j + 1, false) +
                      ((c.want_qz && !ov) ? 2.0 : 1.0) * fl_sweep(0, p, k, nwr, n, -1, false);
    LAUNCH(HT_CLASS_SWEEP, fl, run_sweep(c, jobs, 3, w.wyR, wst, 0, p, k, 0, nwr));
  }
  // (c)/(d) steps 2-4 and (e) step 3
  LAUNCH(HT_CLASS_RANKK, fl_rk, ht_launch_rankk_right(st, B, ldb, n, s + 1, n - k, k, V, n, w.L1, k, w.T, nb));
  if (c.want_qz && !ov)
    LAUNCH(HT_CLASS_RANKK, fl_rk, ht_launch_rankk_right(st, Z, ldz, n, s + 1, n - k, k, V, n, w.L1, k, w.T, nb));
  LAUNCH(HT_CLASS_GEMM, fl_gemm(n, k, k),
         ht_gemm(st, 'N', 'T', n, k, k, -1.0, w.Y, n, w.L1, k, 1.0, A + (size_t)(n - k) * lda, lda));
  // partial restore: RQ chain bottom to top (Sec. 3.3.1e); on the emulated path in
  // segments, each followed by the segment's transforms on the rows above its band
  // (emulated sweep) instead of FP64 updates inside the restore kernel
  bool waitq = false;  // the deferred Q sweep was launched: the QR restore waits for it
  if (ov && c.want_qz) {
    CK(cudaEventRecord(w.side_ev[0], st));
    CK(cudaStreamWaitEvent(w.side, w.side_ev[0], 0));
    CK(flush_pendq(c));
    waitq = true;
    // Z: (e) step 1 and steps 2-4 of the right reflectors
    const HtSweepJob jz = {Z, ldz, 1, 0, n, j + 1, 0, 0};
    LAUNCH_SIDE(fl_sweep(0, p, k, nwr, n, -1, false), run_sweep(c, &jz, 1, w.wyR, wst, 0, p, k, 0, nwr, true));
    LAUNCH_SIDE(fl_rk, ht_launch_rankk_right(w.side, Z, ldz, n, s + 1, n - k, k, V, n, w.L1, k, w.T, nb));
  }
  if (nbr > 1) CK(restore_chain(c, 2, p, k, j, w.wyRR, wst, seg, rs_ctas));
  if (nbr > 1) {
    // rows 0..j of B (on the emulated path already done with the segments),
    // all rows of A and Z, one fused launch
    const HtSweepJob jobs[3] = {{A, lda, 1, 0, n, j + 1, 0, 0},
                                {Z, ldz, 1, 0, (c.want_qz && !ov) ? n : 0, j + 1, 0, 0},
                                {B, ldb, 1, 0, seg ? 0 : j + 1, j + 1, 0, 0}};
    const double fl = (seg ? 0.0 : fl_sweep(2, p, k, nbr - 1, j + 1, -1, false)) +
                      ((c.want_qz && !ov) ? 2.0 : 1.0) * fl_sweep(2, p, k, nbr - 1, n, -1, false);
    LAUNCH(HT_CLASS_SWEEP, fl, run_sweep(c, jobs, 3, w.wyRR, wst, 2, p, k, 0, nbr - 1));
  }

  // ---- left reflectors, Sec. 3.3.2 ----
  // (c) step 1: spike B(s+1:j, s+1:j) -= U1 S^T (U^T B(s+1:n, s+1:j)); step 2 zeros below
  double* sm0 = w.small;
  double* sm1 = w.small + 2 * HT_NB_MAX * HT_NB_MAX;
  double* Bsp = B + (size_t)(s + 1) + (size_t)(s + 1) * ldb;
  LAUNCH(HT_CLASS_GEMM, fl_gemm(k, k, m),
         ht_gemm_ws(st, 'T', 'N', k, k, m, 1.0, U, n, Bsp, ldb, 0.0, sm0, k, w.tmp2, wsd));
  LAUNCH(HT_CLASS_GEMM, fl_gemm(k, k, k), ht_gemm(st, 'T', 'N', k, k, k, 1.0, w.S, nb, sm0, k, 0.0, sm1, k));
  LAUNCH(HT_CLASS_GEMM, fl_gemm(k, k, k), ht_gemm(st, 'N', 'N', k, k, k, -1.0, U, n, sm1, k, 1.0, Bsp, ldb));
  LAUNCH(HT_CLASS_OTHER, 0.0, ht_launch_zero(st, B + (size_t)(j + 1) + (size_t)(s + 1) * ldb, ldb, p, k, 0));
  LAUNCH(HT_CLASS_OTHER, 0.0, ht_launch_zero(st, Bsp, ldb, k, k, 1));
  const int nwl = ht_num_windows(p, k);
  // (c) step 3, (e) step 1, (d) step 1
  {
    // columns j.. of A and j+1.. of B from the left, all rows of Q from the right, one fused launch
    const HtSweepJob jobs[3] = {{A, lda, 0, j, n - j, j + 1, 0, 0},
                                {Q, ldq, 1, 0, (c.want_qz && !ov) ? n : 0, j + 1, 0, 0},
                                {B, ldb, 0, j + 1, p, j + 1, 1, j + 1}};
    const double fl = fl_sweep(1, p, k, nwl, p, 0, true) + fl_sweep(1, p, k, nwl, n - j, -1, true) +
                      ((c.want_qz && !ov) ? fl_sweep(1, p, k, nwl, n, -1, false) : 0.0);
    LAUNCH(HT_CLASS_SWEEP, fl, run_sweep(c, jobs, 3, w.wyL, wst, 1, p, k, 0, nwl));
  }
  // U~ = [U1; R~1] (2k x k) in tmp3 with ld 2k
  double* Ut = w.tmp3;
  LAUNCH(HT_CLASS_OTHER, 0.0,
         cudaMemcpy2DAsync(Ut, 2 * k * sizeof(double), U, n * sizeof(double), k * sizeof(double), k,
                           cudaMemcpyDeviceToDevice, st));
  LAUNCH(HT_CLASS_OTHER, 0.0,
         cudaMemcpy2DAsync(Ut + k, 2 * k * sizeof(double), w.R1, k * sizeof(double), k * sizeof(double), k,
                           cudaMemcpyDeviceToDevice, st));
  // (c) steps 4-5, (e) steps 2-3, (d) steps 2-3
  LAUNCH(HT_CLASS_RANKK, fl_rkl * p, ht_rankk_left(st, B, ldb, j + 1, p, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
  LAUNCH(HT_CLASS_RANKK, fl_rkl * (n - j), ht_rankk_left(st, A, lda, j, n - j, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
  if (c.want_qz && !ov)
    LAUNCH(HT_CLASS_RANKK, fl_rkl * dn, ht_rankk_right_w(st, Q, ldq, n, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
  if (ov && c.want_qz) {
    CK(cudaEventRecord(w.side_ev[1], st));
    CK(cudaStreamWaitEvent(w.side, w.side_ev[1], 0));
    // Q: (d) step 1 of the left reflectors; Z: (e) step 3 (the RQ restore); Q: (d) steps 2-3
    const HtSweepJob jq = {Q, ldq, 1, 0, n, j + 1, 0, 0};
    LAUNCH_SIDE(fl_sweep(1, p, k, nwl, n, -1, false), run_sweep(c, &jq, 1, w.wyL, wst, 1, p, k, 0, nwl, true));
    if (nbr > 1) {
      const HtSweepJob jz = {Z, ldz, 1, 0, n, j + 1, 0, 0};
      LAUNCH_SIDE(fl_sweep(2, p, k, nbr - 1, n, -1, false),
                  run_sweep(c, &jz, 1, w.wyRR, wst, 2, p, k, 0, nbr - 1, true));
    }
    LAUNCH_SIDE(fl_rkl * dn, ht_rankk_right_w(w.side, Q, ldq, n, s + 1, 2 * k, k, Ut, 2 * k, w.S, nb));
    CK(cudaEventRecord(w.side_ev[4], w.side));
    // (d) step 4, the last Q sweep, goes to the next absorption's RQ window
    c.pendq = {true, p, k, j, nlb, wst};
  }
  // (f) restore: QR chain top to bottom (in segments on the emulated path), after the
  // deferred Q sweep of the previous absorption has read this store
  if (waitq) CK(cudaStreamWaitEvent(st, w.side_ev[3], 0));
  CK(restore_chain(c, 3, p, k, j, w.wyLR, wst, seg, rs_ctas));
  {
    const HtSweepJob jobs[2] = {{A, lda, 0, j, n - j, j + 1, 0, 0},
                                {Q, ldq, 1, 0, (c.want_qz && !ov) ? n : 0, j + 1, 0, 0}};
    const double fl = fl_sweep(3, p, k, nlb, n - j, -1, true) +
                      ((c.want_qz && !ov) ? fl_sweep(3, p, k, nlb, n, -1, false) : 0.0);
    LAUNCH(HT_CLASS_SWEEP, fl, run_sweep(c, jobs, 2, w.wyLR, wst, 3, p, k, 0, nlb));
  }
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

int preprocess_impl(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                    int want_qz, const ht_options* opt, ht_stats* stats, cudaStream_t st, bool* done);
int checked_emu(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                const ht_options* opt, ht_stats* stats, cudaStream_t st);

// keep_q: Q already holds a left transform (a front end's) that the reduction
// multiplies from the right, instead of starting from Q = I
int reduce_impl(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz, int want_qz,
                const ht_options* opt, ht_stats* stats, cudaStream_t st, int cap = 0, bool keep_q = false) {
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
  if (prec != HT_PREC_FP64 && prec != HT_PREC_EMU) return HT_ERR_NOT_IMPLEMENTED;
  // the emulated sweeps: panels of at most 32 reflectors, 6 digits per operand
  if (prec == HT_PREC_EMU && (nb > 32 || (opt && opt->emu_slices != 0 && opt->emu_slices != 6)))
    return HT_ERR_NOT_IMPLEMENTED;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  set_stream_status(st, HT_OK);
  if (n == 0) return HT_OK;
  if (opt && opt->emu_check && prec == HT_PREC_EMU && want_qz && n > 2 && !keep_q && !opt->preprocess)
    return checked_emu(n, A, lda, B, ldb, Q, ldq, Z, ldz, opt, stats, st);
  if (opt && opt->preprocess && n > 2 && !keep_q) {
    bool done = false;
    rc = preprocess_impl(n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz, opt, stats, st, &done);
    if (rc != HT_OK || done) return rc;
  }
  if (want_qz) {
    if (!keep_q) HT_CUDA(ht_launch_set_identity(st, Q, ldq, n));
    HT_CUDA(ht_launch_set_identity(st, Z, ldz, n));
  }
  if (n <= 2) {
    HT_CUDA(ht_launch_zero(st, B, ldb, n, n, 1));
    HT_CUDA(cudaStreamSynchronize(st));
    return HT_OK;
  }
  PoolEntry* pe = acquire(n, nb, &rc);
  if (!pe) return rc;
  pe->w.prec = prec;
  pe->w.cap = cap;
  pe->w.G = cap > 0 ? std::min(pe->G, cap) : pe->G;
  pe->w.spin = (opt && opt->wait_polls > 0) ? (long)opt->wait_polls : (long)HT_SPIN_LIMIT;
  const int result = ht_reduce_core(pe->w, pe->host_status, pe->pt_dev, n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz,
                                    nb, max_ir, tol_scale, seed, opt && opt->profile, stats, st);
  release(pe);
  return result;
}

// Device memory of the front ends (freed on scope exit, after the stream's work)
struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) {
      cudaStreamSynchronize(st);
      cudaFree(p);
    }
  }
  bool alloc(size_t bytes, cudaStream_t s) {
    st = s;
    return cudaMalloc(&p, bytes > 0 ? bytes : 1) == cudaSuccess;
  }
  double* d() const { return (double*)p; }
};

// QZ front end (Sec. 1): B = Q_B R, A <- Q_B^T A, Q <- Q_B (when want_qz), B <- R
int front_end_qr(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, int want_qz, cudaStream_t st) {
  if (n <= 0) return HT_OK;
  DevBuf ws;
  if (!ws.alloc(ht_qr_ws_doubles(n, n, n) * sizeof(double), st)) return HT_ERR_NOMEM;
  if (want_qz) HT_CUDA(ht_launch_set_identity(st, Q, ldq, n));
  const HtQrTarget tg = {A, lda, n};
  HT_CUDA(ht_qr_blocked(st, n, n, B, ldb, &tg, 1, want_qz ? Q : nullptr, ldq, n, ws.d()));
  return HT_OK;
}

// ht_options.emu_check: the emulated reduction, a probe estimate of its
// backward errors with FP64 products, and a rerun in FP64 from a saved copy of
// the pencil when an estimate exceeds the emulated path's stated 1e-12.
int checked_emu(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                const ht_options* opt, ht_stats* stats, cudaStream_t st) {
  constexpr int NP = 8;
  const size_t nn = (size_t)n * n;
  DevBuf mem;
  if (!mem.alloc((2 * nn + 4 * (size_t)n * NP + 8) * sizeof(double), st)) return HT_ERR_NOMEM;
  double* A0 = mem.d();
  double* B0 = A0 + nn;
  double* X = B0 + nn;
  double* Y1 = X + (size_t)n * NP;
  double* Y2 = Y1 + (size_t)n * NP;
  double* Y3 = Y2 + (size_t)n * NP;
  double* acc = Y3 + (size_t)n * NP;  // |A|^2, |B|^2, |dA X|^2, |dB X|^2
  const size_t row = (size_t)n * sizeof(double);
  HT_CUDA(cudaMemcpy2DAsync(A0, row, A, lda * sizeof(double), row, n, cudaMemcpyDeviceToDevice, st));
  HT_CUDA(cudaMemcpy2DAsync(B0, row, B, ldb * sizeof(double), row, n, cudaMemcpyDeviceToDevice, st));
  HT_CUDA(ht_launch_zero(st, B0, n, n, n, 1));  // B is upper triangular: its strictly lower part is ignored
  ht_options o2 = *opt;
  o2.emu_check = 0;
  int rc = reduce_impl(n, A, lda, B, ldb, Q, ldq, Z, ldz, 1, &o2, stats, st);
  if (rc != HT_OK) return rc;
  // ||Q M Z^T X - M0 X||_F over 8 probes estimates ||Q M Z^T - M0||_F sqrt(8)
  HT_CUDA(cudaMemsetAsync(acc, 0, 8 * sizeof(double), st));
  HT_CUDA(ht_launch_sumsq(st, n, n, A0, n, nullptr, 0, acc + 0));
  HT_CUDA(ht_launch_sumsq(st, n, n, B0, n, nullptr, 0, acc + 1));
  HT_CUDA(ht_launch_gauss(st, (size_t)n * NP, X, 0x5EEDull + (unsigned long long)n));
  const double* M[2] = {A, B};
  const int ldm[2] = {lda, ldb};
  const double* M0[2] = {A0, B0};
  for (int t = 0; t < 2; ++t) {
    HT_CUDA(ht_gemm(st, 'T', 'N', n, NP, n, 1.0, Z, ldz, X, n, 0.0, Y1, n));
    HT_CUDA(ht_gemm(st, 'N', 'N', n, NP, n, 1.0, M[t], ldm[t], Y1, n, 0.0, Y2, n));
    HT_CUDA(ht_gemm(st, 'N', 'N', n, NP, n, 1.0, Q, ldq, Y2, n, 0.0, Y3, n));
    HT_CUDA(ht_gemm(st, 'N', 'N', n, NP, n, 1.0, M0[t], n, X, n, 0.0, Y1, n));
    HT_CUDA(ht_launch_sumsq(st, n, NP, Y3, n, Y1, n, acc + 2 + t));
  }
  double h[4] = {0, 0, 0, 0};
  HT_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
  HT_CUDA(cudaStreamSynchronize(st));
  const double ea = h[0] > 0 ? std::sqrt(h[2] / NP / h[0]) : 0.0;
  const double eb = h[1] > 0 ? std::sqrt(h[3] / NP / h[1]) : 0.0;
  const bool fail = !(ea <= 1e-12 && eb <= 1e-12) || opt->emu_check == 2;
  if (fail) {
    HT_CUDA(cudaMemcpy2DAsync(A, lda * sizeof(double), A0, row, row, n, cudaMemcpyDeviceToDevice, st));
    HT_CUDA(cudaMemcpy2DAsync(B, ldb * sizeof(double), B0, row, row, n, cudaMemcpyDeviceToDevice, st));
    o2.precision = HT_PREC_FP64;
    rc = reduce_impl(n, A, lda, B, ldb, Q, ldq, Z, ldz, 1, &o2, stats, st);
    if (rc != HT_OK) return rc;
  }
  if (stats) {
    stats->emu_bwd_est[0] = ea;
    stats->emu_bwd_est[1] = eb;
    stats->emu_fallback = fail ? 1 : 0;
  }
  return HT_OK;
}

// Sec. 3.4.1 (see ht_options.preprocess).  *done = false: nothing to deflate
// (at most one zero column), the caller reduces the pencil as it is.
int preprocess_impl(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                    int want_qz, const ht_options* opt, ht_stats* stats, cudaStream_t st, bool* done) {
  *done = false;
  DevBuf flags;
  if (!flags.alloc((size_t)(n + 1) * sizeof(int), st)) return HT_ERR_NOMEM;
  int* dz = (int*)flags.p;
  HT_CUDA(ht_launch_zero_columns(st, n, B, ldb, dz, dz + n));
  std::vector<int> hz(n + 1);
  HT_CUDA(cudaMemcpyAsync(hz.data(), dz, (size_t)(n + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  HT_CUDA(cudaStreamSynchronize(st));
  std::vector<int> perm;
  for (int c = 0; c < n; ++c)
    if (hz[c]) perm.push_back(c);
  const int l = (int)perm.size();
  if (l <= 1) return HT_OK;
  for (int c = 0; c < n; ++c)
    if (!hz[c]) perm.push_back(c);
  const bool diag = hz[n] == 0;  // B diagonal: Q_0 = Z_0 keeps it so
  *done = true;
  const int m2 = n - l;
  const size_t nn = (size_t)n * n, mm = (size_t)m2 * m2;
  DevBuf mem;
  const size_t ws_d = ht_qr_ws_doubles(n, n, n);
  if (!mem.alloc((nn + 2 * mm + ws_d) * sizeof(double) + (size_t)n * sizeof(int), st)) return HT_ERR_NOMEM;
  double* tmp = mem.d();
  double* Q22 = tmp + nn;
  double* Z22 = Q22 + mm;
  double* ws = Z22 + mm;
  int* dp = (int*)(ws + ws_d);
  HT_CUDA(cudaMemcpyAsync(dp, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, st));
  // A_0 = Q_0^T A Z_0, B_0 = Q_0^T B Z_0; Q = Q_0, Z = Z_0
  HT_CUDA(ht_launch_permute(st, n, A, lda, tmp, dp, diag ? 1 : 0));
  HT_CUDA(ht_launch_permute(st, n, B, ldb, tmp, dp, diag ? 1 : 0));
  if (want_qz) {
    if (diag) HT_CUDA(ht_launch_perm_matrix(st, n, Q, ldq, dp));
    else HT_CUDA(ht_launch_set_identity(st, Q, ldq, n));
    HT_CUDA(ht_launch_perm_matrix(st, n, Z, ldz, dp));
  }
  // QR of the first l columns of A_0: A_1 = [A11 A12; 0 A22], B_1 = [0 B12; 0 B22]
  const HtQrTarget tg[2] = {{A + (size_t)l * lda, lda, m2}, {B, ldb, n}};
  HT_CUDA(ht_qr_blocked(st, n, l, A, lda, tg, 2, want_qz ? Q : nullptr, ldq, n, ws));
  if (m2 == 0) {
    set_stream_status(st, HT_OK);
    HT_CUDA(cudaStreamSynchronize(st));
    return HT_OK;
  }
  // the trailing pencil: QR of B22 (front end), then Algorithm 1 with Q22, Z22
  double* A22 = A + (size_t)l + (size_t)l * lda;
  double* B22 = B + (size_t)l + (size_t)l * ldb;
  HT_CUDA(ht_launch_set_identity(st, Q22, m2, m2));
  {
    const HtQrTarget t22 = {A22, lda, m2};
    HT_CUDA(ht_qr_blocked(st, m2, m2, B22, ldb, &t22, 1, Q22, m2, m2, ws));
  }
  ht_options o2 = *opt;
  o2.preprocess = 0;
  const int rc = reduce_impl(m2, A22, lda, B22, ldb, Q22, m2, Z22, m2, 1, &o2, stats, st, 0, true);
  if (rc != HT_OK) return rc;
  // rows 0 .. l-1 of A and B take Z22 from the right; Q and Z their trailing columns
  auto right_mul = [&](double* X, long ldx, int rows, const double* M) -> cudaError_t {
    if (rows <= 0) return cudaSuccess;
    cudaError_t e = ht_gemm(st, 'N', 'N', rows, m2, m2, 1.0, X, (int)ldx, M, m2, 0.0, tmp, rows);
    if (e != cudaSuccess) return e;
    return cudaMemcpy2DAsync(X, ldx * sizeof(double), tmp, rows * sizeof(double), rows * sizeof(double), m2,
                             cudaMemcpyDeviceToDevice, st);
  };
  HT_CUDA(right_mul(A + (size_t)l * lda, lda, l, Z22));
  HT_CUDA(right_mul(B + (size_t)l * ldb, ldb, l, Z22));
  if (want_qz) {
    HT_CUDA(right_mul(Q + (size_t)l * ldq, ldq, n, Q22));
    HT_CUDA(right_mul(Z + (size_t)l * ldz, ldz, n, Z22));
  }
  HT_CUDA(cudaStreamSynchronize(st));
  return HT_OK;
}

}  // namespace

// The reduction of Algorithm 1 on a prepared workspace (n >= 3, arguments
// checked, Q = Z = I already set when want_qz).  host_status: host memory
// for the per-panel status read-back; pt_dev: profile timers (or null).
int ht_reduce_core(HtWork& w, PanelStatus* host_status, unsigned long long* pt_dev, int n, double* A, int lda,
                   double* B, int ldb, double* Q, int ldq, double* Z, int ldz, int want_qz, int nb, int max_ir,
                   double tol_scale, uint64_t seed, int profile, ht_stats* stats, cudaStream_t st) {
  w.stream = st;
  Prof prof;
  prof.on = profile && pt_dev;
  w.ptime = prof.on ? pt_dev : nullptr;
  if (prof.on) cudaMemsetAsync(pt_dev, 0, 32 * sizeof(unsigned long long), st);
  prof.st = st;
  prof.side = w.side;
  Ctx c{&w, st, n, A, B, Q, Z, lda, ldb, ldq, ldz, want_qz, 0.0, &prof, {}};
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
      if (cudaMemcpyAsync(&host_status->error, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      derr = host_status->error;
      if (derr != 0) { result = derr; break; }
    }
    if (ht_launch_prepare_B(w, B, ldb, 0, seed, 1) != cudaSuccess) { result = HT_ERR_CUDA; break; }
    int s = 0;
    while (s <= n - 3) {
      const int kmax = std::min(nb, (n - s - 1) / 2);
      // the side stream's Q / Z updates of the previous absorption read the panel's
      // outputs (V, T, U, S) and the chains' WY stores: join before overwriting them
      if (w.side && cudaStreamWaitEvent(st, w.side_ev[4], 0) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      if (cudaMemsetAsync(w.status, 0, sizeof(PanelStatus), st) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      if (ht_launch_prepare_B(w, B, ldb, s, seed, 0) != cudaSuccess) { result = HT_ERR_CUDA; break; }
      if (timing) cudaEventRecord(ev[0], st);
      prof.begin(HT_CLASS_PANEL);
      cudaError_t e = ht_launch_panel(w, A, lda, B, ldb, s, kmax, tol_scale, max_ir);
      prof.end(0.0);
      if (e != cudaSuccess) {
        std::fprintf(stderr, "libht: panel launch failed: %s\n", cudaGetErrorString(e));
        result = HT_ERR_CUDA;
        break;
      }
      if (timing) cudaEventRecord(ev[1], st);
      if (cudaMemcpyAsync(host_status, w.status, sizeof(PanelStatus), cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        result = HT_ERR_CUDA;
        break;
      }
      const PanelStatus ps = *host_status;
      if (ps.error != 0) { result = ps.error; break; }
      int k = ps.k_done;
      if (k < 1) { result = HT_ERR_INTERNAL; break; }
      {
        // panel flops: per column the Y GEMV (2 m p) and the solve and residual
        // passes over the triangle of B (m^2 each), plus m^2 per correction
        const int m = n - s - 1;
        double fl = 0.0;
        for (int q = 0; q < k; ++q) fl += 2.0 * (double)m * (m - q) + 2.0 * (double)m * m;
        fl += 2.0 * (double)m * m * ps.ir_steps;
        prof.flops[HT_CLASS_PANEL] += fl;
        c.flops += fl;
      }
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
      prof.resolve();
      s += k;
    }
    if (result != HT_OK) break;
    if (c.pendq.on && flush_pendq(c) != cudaSuccess) { result = HT_ERR_CUDA; break; }
    if (w.side && (cudaEventRecord(w.side_ev[4], w.side) != cudaSuccess ||
                   cudaStreamWaitEvent(st, w.side_ev[4], 0) != cudaSuccess)) {
      result = HT_ERR_CUDA;
      break;
    }
    int derr = 0;
    if (cudaMemcpyAsync(&derr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      result = HT_ERR_CUDA;
      break;
    }
    if (derr != 0) result = derr;
  } while (0);
  if (w.side) {
    // whatever the outcome, the caller's stream follows every side-stream launch
    cudaEventRecord(w.side_ev[4], w.side);
    cudaStreamWaitEvent(st, w.side_ev[4], 0);
  }
  prof.resolve();
  if (stats && prof.on) {
    unsigned long long pt[24];
    cudaMemcpy(pt, pt_dev, sizeof(pt), cudaMemcpyDeviceToHost);
    for (int q = 0; q < 24; ++q) stats->panel_phase_ms[q] = pt[q] * 1e-6;
  }
  if (stats) {
    stats->flops_nominal = c.flops;
    for (int q = 0; q < HT_NCLASS; ++q) {
      stats->ms_by_class[q] = prof.ms[q];
      stats->flops_by_class[q] = prof.flops[q];
      stats->launches_by_class[q] = prof.launches[q];
    }
  }
  if (timing)
    for (auto& e : ev) cudaEventDestroy(e);
  {
    int derr = 0;
    cudaMemcpy(&derr, w.err, sizeof(int), cudaMemcpyDeviceToHost);
    set_stream_status(st, derr);
  }
  return result;
}

extern "C" {

int ht_reduce_ex(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz, int want_qz,
                 const ht_options* opt, ht_stats* stats, ht_stream_t stream) {
  return reduce_impl(n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz, opt, stats, (cudaStream_t)stream);
}

int ht_reduce_general(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                      int want_qz, const ht_options* opt, ht_stats* stats, ht_stream_t stream) {
  int rc = check_args(n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz);
  if (rc != HT_OK) return rc;
  if (opt && opt->preprocess) return HT_ERR_NOT_IMPLEMENTED;  // preprocessing needs an upper triangular B
  cudaStream_t st = (cudaStream_t)stream;
  rc = front_end_qr(n, A, lda, B, ldb, Q, ldq, want_qz, st);
  if (rc != HT_OK) return rc;
  return reduce_impl(n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz, opt, stats, st, 0, true);
}

int ht_reduce(int n, double* A, int lda, double* B, int ldb, double* Q, double* Z, int want_qz, ht_stream_t stream) {
  return reduce_impl(n, A, lda, B, ldb, Q, n, Z, n, want_qz, nullptr, nullptr, (cudaStream_t)stream);
}

int ht_reduce_batched(int batch, const int* n, double* const* A, const int* lda, double* const* B, const int* ldb,
                      double* const* Q, double* const* Z, int want_qz, ht_stream_t stream) {
  if (batch < 0) return -1;
  if (batch > 0 && (!n || !A || !lda || !B || !ldb)) return -2;
  if (want_qz && batch > 0 && (!Q || !Z)) return -7;
  if (batch == 0) return HT_OK;
  // the pointer arrays may be host arrays or device arrays (the cuBLAS-batched
  // convention): device arrays are copied to the host, which plans the lanes
  std::vector<double*> hp[4];
  double* const* parr[4] = {A, B, want_qz ? Q : nullptr, want_qz ? Z : nullptr};
  for (int a = 0; a < 4; ++a) {
    if (!parr[a]) continue;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, parr[a]) != cudaSuccess) {
      cudaGetLastError();
      continue;  // unregistered host memory
    }
    if (at.type == cudaMemoryTypeDevice) {
      hp[a].resize(batch);
      if (cudaMemcpy(hp[a].data(), parr[a], sizeof(double*) * (size_t)batch, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HT_ERR_CUDA;
      parr[a] = hp[a].data();
    }
  }
  A = parr[0]; B = parr[1];
  if (want_qz) { Q = parr[2]; Z = parr[3]; }
  std::vector<int> order(batch);
  for (int i = 0; i < batch; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  cudaStream_t user = (cudaStream_t)stream;
  // the panel width of each pencil's size class (ht_tuned.h, measured by the autotuner)
  auto one = [&](int i, cudaStream_t st, int cap) {
    ht_options o{};
    o.nb = ht_tuned_nb(n[i]);
    return reduce_impl(n[i], A[i], lda[i], B[i], ldb[i], want_qz ? Q[i] : nullptr, std::max(1, n[i]),
                       want_qz ? Z[i] : nullptr, std::max(1, n[i]), want_qz, &o, nullptr, st, cap);
  };
  // Lanes: the pencils are independent, and one reduction of a small pencil
  // leaves most of the GPU idle (its panels and restore chains are latency-
  // bound), so BATCH_LANES host threads each reduce pencils, largest first, on
  // a stream of their own.  Every launch of a lane whose CTAs wait on one
  // another takes at most sms / lanes CTAs, so that those of all lanes are
  // resident together.
  const int sms = sm_count();
  const int lanes = std::min(batch, std::max(1, sms / BATCH_LANE_CTAS));
  if (lanes <= 1) {
    for (int i : order) {
      const int rc = one(i, user, 0);
      if (rc != HT_OK) return rc;
    }
    return HT_OK;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HT_ERR_CUDA;
  const int cap = sms / lanes;
  std::vector<cudaStream_t> ls(lanes, nullptr);
  std::vector<cudaEvent_t> le(lanes + 1, nullptr);
  int rc = HT_OK;
  for (int l = 0; l < lanes && rc == HT_OK; ++l)
    if (cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking) != cudaSuccess) rc = HT_ERR_CUDA;
  for (int l = 0; l <= lanes && rc == HT_OK; ++l)
    if (cudaEventCreateWithFlags(&le[l], cudaEventDisableTiming) != cudaSuccess) rc = HT_ERR_CUDA;
  // the lanes start after the caller's earlier work on `stream`
  if (rc == HT_OK && cudaEventRecord(le[lanes], user) != cudaSuccess) rc = HT_ERR_CUDA;
  for (int l = 0; l < lanes && rc == HT_OK; ++l)
    if (cudaStreamWaitEvent(ls[l], le[lanes], 0) != cudaSuccess) rc = HT_ERR_CUDA;
  if (rc == HT_OK) {
    std::atomic<int> next{0}, err{HT_OK};
    std::vector<std::thread> th;
    auto lane = [&](int l) {
      if (cudaSetDevice(dev) != cudaSuccess) { int z = HT_OK; err.compare_exchange_strong(z, HT_ERR_CUDA); return; }
      for (;;) {
        const int q = next.fetch_add(1);
        if (q >= batch || err.load() != HT_OK) return;
        const int r = one(order[q], ls[l], cap);
        if (r != HT_OK) { int z = HT_OK; err.compare_exchange_strong(z, r); return; }
      }
    };
    // a lane whose thread cannot be started runs in this thread after the others start
    std::vector<int> inline_lanes;
    for (int l = 0; l < lanes; ++l) {
      try {
        th.emplace_back(lane, l);
      } catch (...) {
        inline_lanes.push_back(l);
      }
    }
    for (int l : inline_lanes) lane(l);
    for (auto& t : th) t.join();
    rc = err.load();
    // the caller's stream follows every lane
    for (int l = 0; l < lanes; ++l)
      if (cudaEventRecord(le[l], ls[l]) != cudaSuccess || cudaStreamWaitEvent(user, le[l], 0) != cudaSuccess)
        rc = (rc == HT_OK) ? HT_ERR_CUDA : rc;
  }
  for (auto s2 : ls) if (s2) cudaStreamDestroy(s2);
  for (auto e2 : le) if (e2) cudaEventDestroy(e2);
  // the caller's stream reports the batch: the first device-side error of any pencil
  set_stream_status(user, (rc == HT_ERR_TIMEOUT || rc == HT_ERR_NONFINITE || rc == HT_ERR_INTERNAL) ? rc : HT_OK);
  return rc;
}

int ht_last_device_status(ht_stream_t stream, int* status) {
  if (!status) return -2;
  std::lock_guard<std::mutex> lk(g_status_mu);
  *status = HT_OK;
  for (const auto& e : g_status)
    if (e.first == (cudaStream_t)stream) *status = e.second;
  return HT_OK;
}

int ht_finalize(void) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  std::vector<PoolEntry*> keep;
  for (PoolEntry* e : g_pool) {
    if (e->busy) {
      keep.push_back(e);
      continue;
    }
    if (e->w.side) {
      for (auto ev : e->w.side_ev) cudaEventDestroy(ev);
      cudaStreamDestroy(e->w.side);
    }
    cudaFree(e->base);
    cudaFreeHost(e->host_status);
    delete e;
  }
  g_pool.swap(keep);
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
    case HT_ERR_TOO_LARGE: return "n exceeds the static workspace of ht_reduce_noalloc (n <= 512)";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

const char* ht_version(void) { return "libht 0.1 (sm_103a)"; }

}  // extern "C"
