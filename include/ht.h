/*
 * ht.h -- C ABI of libht, a GB300 (sm_103a) implementation of the
 * Householder-based Hessenberg-triangular (HT) reduction of Bujanovic,
 * Karlsson and Kressner, "A Householder-based algorithm for
 * Hessenberg-triangular reduction" (arXiv 1710.08538).
 *
 * Problem (Sec. 1 and Sec. 3, Algorithm 1): given A (n x n) and B (n x n,
 * upper triangular), compute orthogonal Q and Z such that H = Q^T A Z is upper
 * Hessenberg and T = Q^T B Z is upper triangular; Q and Z start as the
 * identity.  A is overwritten by H and B by T, as LAPACK's DGGHRD does.
 *
 * Conventions for every call below
 *   - All matrices are FP64, column-major, in device memory owned by the
 *     caller (unless a pointer is documented as a host pointer).
 *   - Leading dimensions must be >= max(1, n).
 *   - Only the upper triangle of B is read; its strictly lower part is
 *     written with exact zeros on return.  Entries of H below the first
 *     subdiagonal are exact zeros on return.
 *   - Work is queued on `stream` (a cudaStream_t; NULL is the legacy default
 *     stream).  The calls synchronize `stream` once per panel to read the
 *     number of reflectors the panel produced, so they return after the
 *     reduction has finished.
 *   - Return value: HT_OK, a negative value -i when argument i is invalid
 *     (LAPACK INFO style), or one of the positive error codes below.  A failure
 *     of iterative refinement inside the method is not an error: it triggers
 *     the early absorption of Sec. 3.2.2c.
 *   - Thread safety: calls on different streams may run concurrently from
 *     different host threads; each call uses its own workspace.
 */
#ifndef HT_H
#define HT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ht_stream_t; /* same type as cudaStream_t */

enum {
  HT_OK = 0,
  HT_ERR_CUDA = 1001,            /* a CUDA runtime call failed */
  HT_ERR_NOMEM = 1002,           /* device workspace could not be allocated */
  HT_ERR_TIMEOUT = 1003,         /* a bounded device-side wait gave up */
  HT_ERR_NONFINITE = 1004,       /* A or B holds a NaN or an infinity */
  HT_ERR_NOT_IMPLEMENTED = 1005, /* option combination not available */
  HT_ERR_INTERNAL = 1006,        /* a device-side consistency check failed */
  HT_ERR_TOO_LARGE = 1007        /* n exceeds the static workspace of ht_reduce_noalloc */
};

/* Precision of the bulk (level-3) updates of the absorption, Sec. 3.3. */
enum {
  HT_PREC_FP64 = 0, /* native FP64 (DFMA) */
  HT_PREC_EMU = 1   /* FP64 emulated by exact FP16 digit products on the tensor cores (nb <= 32) */
};

/* Tuning and test options of ht_reduce_ex.  Zero-initialise, then set
 * fields; a zero field takes its default. */
typedef struct ht_options {
  int nb;              /* panel width (Sec. 3.2); default 32 */
  int max_ir;          /* iterative-refinement steps per column (Sec. 2.3); default 10, < 0 means 0 */
  double ir_tol_scale; /* multiplies the IR tolerance 2u||B||_F; default 1.0, < 0 means 0 */
  int precision;       /* HT_PREC_*; default HT_PREC_FP64 */
  int emu_slices;      /* HT_PREC_EMU digits of the line operand: 0 = automatic (6); 6; other values
                          return HT_ERR_NOT_IMPLEMENTED (the WY factors always take 7) */
  uint64_t seed;       /* key of the singular-B perturbation (Remark 2.2) */
  int profile;         /* 1: time every launch by class into ht_stats (adds syncs) */
  int wait_polls;      /* test option: polls before a bounded device-side wait gives up and the call returns
                          HT_ERR_TIMEOUT; 0 = default (2^22 polls, seconds) */
  int preprocess;      /* 1: deflate the zero columns of B first (Sec. 3.4.1): with l > 1 zero columns, a
                          permutation Z_0 moves them to the front (Q_0 = Z_0 when B is diagonal, else I), a QR
                          of the first l columns of Q_0^T A Z_0 makes them upper triangular (l infinite
                          eigenvalues, already in generalized Schur form) and only the trailing pencil, after
                          a QR of its B, is reduced; H and T keep the form of ht_reduce.  Allocates
                          temporaries (about 3 n^2 doubles).  0: off */
  int emu_check;       /* HT_PREC_EMU with want_qz: 1 = after the reduction, estimate the relative backward
                          errors ||Q H Z^T - A||_F / ||A||_F and ||Q T Z^T - B||_F / ||B||_F with 8 Gaussian
                          probes and FP64 products, report them in ht_stats.emu_bwd_est and, when one exceeds
                          1e-12 (the stated accuracy of the emulated path), redo the reduction with
                          HT_PREC_FP64 from a saved copy of A and B (ht_stats.emu_fallback = 1); allocates
                          2 n^2 + 32 n doubles.  2 = the same with the check treated as failed (a test of the
                          fallback).  0: off.  Not applied together with preprocess, nor by
                          ht_reduce_general (their reductions start from a transformed pencil) */
  int reserved[4];
} ht_options;

/* Launch classes of ht_stats.ms_by_class / flops_by_class / launches_by_class. */
enum {
  HT_CLASS_PANEL = 0,        /* cooperative panel reduction (Sec. 3.2) */
  HT_CLASS_CHAIN_FACTOR = 1, /* QL / QR chains of V2 and U2 (Sec. 3.3.1b, 3.3.2b) */
  HT_CLASS_RESTORE = 2,      /* RQ / QR restore steps on B (Sec. 3.3.1e, 3.3.2f) */
  HT_CLASS_SWEEP = 3,        /* chain applications to A, B, Q, Z */
  HT_CLASS_RANKK = 4,        /* rank-k corrections with V1, L1, U1, R1 */
  HT_CLASS_GEMM = 5,         /* deferred Y rows (Remark 3.1), spike update */
  HT_CLASS_OTHER = 6,        /* preparation of B, zeroing, copies */
  HT_CLASS_SIDE = 7,         /* Q and Z updates on the library's second stream, overlapping
                                the others (emulated path; its time is not additive) */
  HT_NCLASS = 8
};

/* Per-call counters, the columns of the paper's Tables 3 and 4 plus time. */
typedef struct ht_stats {
  int panels;              /* panel reductions started */
  int early_absorptions;   /* panels ended by an IR failure (Sec. 3.2.2c) */
  long long ir_steps;      /* correction solves of iterative refinement */
  long long cols_with_ir;  /* columns that needed at least one correction */
  int perturbed_pivots;    /* zero diagonal entries of B replaced (Remark 2.2) */
  double ms_panel;         /* device time of the panel reductions (Sec. 3.2) */
  double ms_absorb;        /* device time of the absorptions (Sec. 3.3) */
  double flops_nominal;    /* flops of the operations launched (counted per launch) */
  double ms_by_class[HT_NCLASS];        /* device time per launch class (profile = 1) */
  double flops_by_class[HT_NCLASS];     /* algorithmic flops per launch class */
  long long launches_by_class[HT_NCLASS];
  double panel_phase_ms[24];            /* panel (0-15) and restore (16-19) time by phase (profile = 1) */
  double emu_bwd_est[2];   /* ht_options.emu_check: probe estimates of the backward errors of A and B */
  int emu_fallback;        /* ht_options.emu_check: 1 when the reduction was redone in FP64 */
} ht_stats;

/*
 * ht_reduce -- HT reduction of one pencil (Algorithm 1, HouseHT).
 *   n        order of the pencil, n >= 0
 *   A, lda   device, n x n; overwritten by H = Q^T A Z
 *   B, ldb   device, n x n upper triangular; overwritten by T = Q^T B Z
 *   Q, Z     device, n x n with leading dimension n; written with the
 *            accumulated transforms when want_qz != 0 (may be NULL otherwise)
 *   want_qz  0: do not form Q and Z
 *   stream   CUDA stream
 * n <= 2 leaves A and B unchanged and sets Q = Z = I (the loop of
 * Algorithm 1 is empty).
 */
int ht_reduce(int n, double* A, int lda, double* B, int ldb, double* Q, double* Z, int want_qz,
              ht_stream_t stream);

/* ht_reduce_ex -- as ht_reduce with leading dimensions for Q and Z, options
 * (NULL = defaults) and counters (NULL = not wanted). */
int ht_reduce_ex(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                 int want_qz, const ht_options* opt, ht_stats* stats, ht_stream_t stream);

/*
 * ht_reduce_general -- the HT reduction of a pencil whose B is a general
 * matrix: the front end of the QZ algorithm (Sec. 1) first computes the QR
 * factorization B = Q_B R (Householder, DLARFG rule of Sec. 2.1), sets
 * A <- Q_B^T A, B <- R, and then runs Algorithm 1 with Q starting from Q_B, so
 * that H = Q^T A Z and T = Q^T B Z hold for the input A and B.
 *   Arguments as ht_reduce_ex; B (device, n x n, ld ldb) need not be upper
 *   triangular.  opt->preprocess is not available here (it needs an upper
 *   triangular B) and returns HT_ERR_NOT_IMPLEMENTED.  Allocates a QR
 *   workspace of about 34 n doubles for the call.
 */
int ht_reduce_general(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                      int want_qz, const ht_options* opt, ht_stats* stats, ht_stream_t stream);

/*
 * ht_reduce_batched -- HT reduction of `batch` independent pencils of
 * (possibly different) orders.
 *   n, lda, ldb   HOST arrays of length batch
 *   A, B, Q, Z    arrays of `batch` device pointers, in host memory or in
 *                 device memory (the cuBLAS-batched convention; a device
 *                 array is copied to the host first); Q[i], Z[i] have
 *                 leading dimension n[i] (ignored when want_qz == 0)
 * Each pencil follows the rules of ht_reduce.  Pencils are independent; the
 * library reduces them largest first on concurrent lanes (host threads with
 * streams of their own, ordered after the caller's earlier work on `stream`;
 * `stream` waits for all of them), each launch whose CTAs wait on one another
 * capped at a share of the SMs so that the lanes' launches are resident
 * together.  Returns the first error of any pencil (the others may be
 * incomplete then); ht_last_device_status(stream) then reports it when it is
 * a device-side condition.  Blocks until every pencil is done.
 */
int ht_reduce_batched(int batch, const int* n, double* const* A, const int* lda, double* const* B,
                      const int* ldb, double* const* Q, double* const* Z, int want_qz, ht_stream_t stream);

/*
 * ht_reduce_noalloc -- ht_reduce (with leading dimensions for Q and Z) for
 * pencils of order n <= HT_NOALLOC_NMAX that allocates no memory: its whole
 * device workspace is a static array of the library (8 MiB per GPU that loads
 * it, held until the process exits).  The paper has no counterpart; this is a
 * service for callers that cannot let a library allocate device memory -
 * applications whose own allocator already holds the GPU's memory, callers
 * that cannot pay for cudaMalloc / cudaFree (cudaFree synchronises the
 * device), environments that forbid allocations outside their own allocator.
 *   Arguments and results are those of ht_reduce (default options).
 *   n > HT_NOALLOC_NMAX returns HT_ERR_TOO_LARGE before any device work.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   All calls share the array, which keeps the last call's contents (each
 *   call clears what it uses first); calls are serialised by a process-wide
 *   lock, and each returns after its work on `stream` has finished, because
 *   calls that overlapped on the GPU would race on the array.
 */
#define HT_NOALLOC_NMAX 512
int ht_reduce_noalloc(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                      int want_qz, ht_stream_t stream);

/*
 * ht_philox4x32_10 -- raw blocks of the device's counter-based generator,
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the generator that draws
 * rho ~ N(0,1) (Box-Muller on words 0 and 1 of the block with counter
 * (panel start s, global diagonal index, 0, 0) and key (seed lo, seed hi)) for
 * the perturbation of a zero diagonal entry of B (Remark 2.2, Sec. 3.2.1).
 * Exposed so that the generator can be checked against its published
 * known-answer vectors.
 *   count  number of blocks, >= 0
 *   in     device, 6 x count uint32: counter[0..3], key[0..1] of each block
 *   out    device, 4 x count uint32: the output words of each block
 * Asynchronous on `stream`; returns -i for an invalid argument i, HT_ERR_CUDA
 * if the launch fails.
 */
int ht_philox4x32_10(int count, const uint32_t* in, uint32_t* out, ht_stream_t stream);

/* ht_last_device_status -- status word written by the device during the
 * last call on `stream` (any host thread; HT_OK, HT_ERR_TIMEOUT,
 * HT_ERR_NONFINITE, HT_ERR_INTERNAL; HT_OK for a stream without calls). */
int ht_last_device_status(ht_stream_t stream, int* status);

/* ht_finalize -- release every cached workspace of this process. */
int ht_finalize(void);

/* ht_status_string -- static description of a return code. */
const char* ht_status_string(int status);

/* ht_version -- library version string. */
const char* ht_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HT_H */
