// Dense Cholesky of a caller-supplied matrix with no device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// factorisation: a solver loop that runs under a fixed memory budget, an
// application whose device memory is all owned by its own pool allocator, or a
// real-time control loop that forbids allocation once it is set up.
// opf_chol_noalloc serves them: the caller passes the matrix and the output
// buffer, and the small scratch the factorisation needs (status word, grid-barrier
// state, inverse diagonal) lives in a file-scope device array, present on every
// GPU that loads this library until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/condipm.h"
#include "common.cuh"

namespace condipm {
namespace {

constexpr int NOALLOC_MAX_N = 4096;
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoAllocScratch {
  int st[ST_WORDS];             // device status word
  unsigned bar[4];              // grid-barrier arrival counter and generation
  double dinv[NOALLOC_MAX_N];   // inverse diagonal of the factor
};

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device (filled by the first call there).
NoAllocScratch* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_noalloc_mu;

int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return OPF_ERR_CUDA;
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return OPF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    NoAllocScratch* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return OPF_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return OPF_OK;
}

}  // namespace
}  // namespace condipm

using namespace condipm;

extern "C" int opf_chol_noalloc(const double* A, int n, double delta_w, double* L, int* fail_col, void* stream) {
  if (fail_col) *fail_col = -1;
  if (!A || !L || n < 1 || n > NOALLOC_MAX_N || !(delta_w >= 0.0)) return OPF_ERR_INVALID_ARG;
  NoAllocScratch* sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc != OPF_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // status and barrier state must start at zero; the inverse diagonal is overwritten
  if (cudaMemsetAsync(sc, 0, sizeof(int) * ST_WORDS + sizeof(unsigned) * 4, s) != cudaSuccess) return OPF_ERR_CUDA;
  if (launch_chol_prepare(s, n, A, delta_w, L) != cudaSuccess) return OPF_ERR_CUDA;
  const int nblocks = chol_grid_cap(n);
  if (launch_chol(s, n, L, sc->dinv, sc->st, sc->bar, 1LL << 26, nblocks) != cudaSuccess) return OPF_ERR_CUDA;
  int st[ST_WORDS] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(st, sc->st, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess) return OPF_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return OPF_ERR_CUDA;
  if (st[ST_TIMEOUT]) return OPF_ERR_TIMEOUT;
  if (st[ST_CODE] == DEV_NOT_PD) {
    if (fail_col) *fail_col = st[ST_INFO];
    return OPF_ERR_NOT_PD;
  }
  return st[ST_CODE] == 0 ? OPF_OK : OPF_ERR_CUDA;
}
