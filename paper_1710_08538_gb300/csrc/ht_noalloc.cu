// ht_reduce_noalloc: the HT reduction of ht_reduce for small pencils with its
// whole device workspace taken from a file-scope static array, so that the
// call allocates no memory at all.
//
// Who needs it: callers that cannot let a library allocate device memory -
// applications whose own allocator already holds (nearly) all of the GPU's
// memory, so a cudaMalloc from inside a library would fail or fragment their
// pool; latency-sensitive callers that cannot pay for cudaMalloc, and above all
// cudaFree, which synchronises the whole device; and environments whose policy
// forbids allocations outside a designated allocator.  ht_reduce keeps a
// cached workspace per order instead, which it allocates on first use.
//
// The static array (HT_NOALLOC_WORDS doubles, 8 MiB) is held by every GPU that
// loads the library until the process exits.  Its device address is looked
// up once per device, on the first call made with that device current
// (cudaGetSymbolAddress); that first call should therefore come before any
// stream capture.  All calls on a device share the array and it keeps the
// contents of the last call: each call clears the workspace it uses before
// starting.  Calls that overlapped on the GPU would race on the array; this
// entry point serialises its own calls with a process-wide lock and returns
// only after its work on `stream` has finished.
#include <cuda_runtime.h>

#include <mutex>

#include "ht_common.cuh"

#define HT_NOALLOC_WORDS (1u << 20)  // 8 MiB of doubles
#define HT_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_ht_noalloc_scratch[HT_NOALLOC_WORDS];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[HT_NOALLOC_MAX_DEVICES] = {};  // device address of the array, per device
PanelStatus g_noalloc_status;                          // host copy of the panel status (pageable)
}  // namespace

extern "C" int ht_reduce_noalloc(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                                 int want_qz, ht_stream_t stream) {
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < (n > 1 ? n : 1)) return -3;
  if (n > 0 && !B) return -4;
  if (ldb < (n > 1 ? n : 1)) return -5;
  if (want_qz && n > 0 && !Q) return -6;
  if (want_qz && ldq < (n > 1 ? n : 1)) return -7;
  if (want_qz && n > 0 && !Z) return -8;
  if (want_qz && ldz < (n > 1 ? n : 1)) return -9;
  if (n > HT_NOALLOC_NMAX) return HT_ERR_TOO_LARGE;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= HT_NOALLOC_MAX_DEVICES) return HT_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    // set-up, once per device: the host-side name of the array is not a device
    // address; ask the runtime for the address on the current device
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_ht_noalloc_scratch) != cudaSuccess || !p) return HT_ERR_CUDA;
    g_noalloc_ptr[dev] = (double*)p;
  }
  if (n == 0) return HT_OK;
  // the workspace must fit the array before anything is written (its size
  // depends on the device's SM count through the panel's CTA count)
  const int nb = 32;
  const int G = ht_panel_max_ctas(nb);
  HtWork w;
  const size_t bytes = n > 2 ? ht_layout_work(w, nullptr, n, nb, G, nullptr) : 0;
  if (bytes > sizeof(double) * (size_t)HT_NOALLOC_WORDS) return HT_ERR_TOO_LARGE;
  if (want_qz) {
    if (ht_launch_set_identity(st, Q, ldq, n) != cudaSuccess) return HT_ERR_CUDA;
    if (ht_launch_set_identity(st, Z, ldz, n) != cudaSuccess) return HT_ERR_CUDA;
  }
  if (n <= 2) {
    if (ht_launch_zero(st, B, ldb, n, n, 1) != cudaSuccess) return HT_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? HT_OK : HT_ERR_CUDA;
  }
  ht_layout_work(w, (char*)g_noalloc_ptr[dev], n, nb, G, nullptr);
  // the array keeps the previous call's contents: start from zeros
  if (cudaMemsetAsync(g_noalloc_ptr[dev], 0, bytes, st) != cudaSuccess) return HT_ERR_CUDA;
  const int rc = ht_reduce_core(w, &g_noalloc_status, nullptr, n, A, lda, B, ldb, Q, ldq, Z, ldz, want_qz, nb, 10,
                                1.0, 0, 0, nullptr, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return HT_ERR_CUDA;
  return rc;
}
