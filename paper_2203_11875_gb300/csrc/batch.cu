// Batched interior-point solves of many independent OPF instances on one GPU.
//
// One instance keeps the GPU far from busy: its kernels are short, several are
// latency-bound level-scheduled solves, and the host loop waits on the device
// at every iteration.  The batch runs many instances at once: every instance
// gets its own non-blocking stream, and a pool of host threads takes instances
// from a shared queue (largest first, so the long solves start early), each
// thread driving one instance's loop at a time.  The kernels of different
// instances then overlap on the SMs, and the host waits of one instance hide
// behind the device work of the others.  No device memory is allocated or freed
// while the batch runs (freeing would synchronise the whole device).
//
// Before the timed solves, opf_batch_autotune picks each instance's multi-RHS
// solve kernel with the GPU to itself (the choice is timed, and timings taken
// while other instances run would be meaningless).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/condipm.h"
#include "internal.h"

struct opf_batch {
  std::vector<opf_handle*> hs;
  std::vector<cudaStream_t> streams;   // owned, one per instance
  std::vector<cudaStream_t> prev;      // the handles' streams before the batch
  std::vector<int> order;              // instances, largest first
  int nthreads = 1;
  int device = 0;
};

namespace condipm {
namespace {

long long work_estimate(const opf_handle* h) {
  // dense condensed work dominates: nu^2 * nx (trsm output) plus nu^3 (Cholesky)
  const long long nu = h->P.nu, nx = h->P.nx;
  return nu * nu * nx + nu * nu * nu;
}

}  // namespace
}  // namespace condipm

using namespace condipm;

extern "C" int opf_batch_create(opf_handle* const* handles, int n, int nthreads, opf_batch** out) {
  if (!handles || n < 1 || !out) return OPF_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!handles[i]) return OPF_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (handles[i] == handles[j]) return OPF_ERR_INVALID_ARG;
  opf_batch* b = new (std::nothrow) opf_batch;
  if (!b) return OPF_ERR_OOM;
  if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return OPF_ERR_CUDA; }
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  b->nthreads = nthreads > 0 ? nthreads : int(std::min<unsigned>(hw, 32u));
  b->nthreads = std::max(1, std::min(b->nthreads, n));
  b->hs.assign(handles, handles + n);
  for (int i = 0; i < n; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      opf_batch_destroy(b);
      return OPF_ERR_CUDA;
    }
    b->streams.push_back(s);
    b->prev.push_back(b->hs[i]->s);
    b->hs[i]->s = s;
    // the interior-point scratch and solve workspace exist before any solve runs
    int rc = ipm_reserve(b->hs[i]);
    if (rc != OPF_OK) { opf_batch_destroy(b); return rc; }
  }
  b->order.resize(n);
  std::iota(b->order.begin(), b->order.end(), 0);
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return work_estimate(b->hs[a]) > work_estimate(b->hs[c]); });
  if (cudaDeviceSynchronize() != cudaSuccess) { opf_batch_destroy(b); return OPF_ERR_CUDA; }
  *out = b;
  return OPF_OK;
}

extern "C" void opf_batch_destroy(opf_batch* b) {
  if (!b) return;
  for (size_t i = 0; i < b->streams.size(); ++i) {
    cudaStreamSynchronize(b->streams[i]);
    if (i < b->prev.size()) b->hs[i]->s = b->prev[i];
    cudaStreamDestroy(b->streams[i]);
  }
  delete b;
}

extern "C" int opf_batch_size(const opf_batch* b, int* n, int* nthreads) {
  if (!b) return OPF_ERR_INVALID_ARG;
  if (n) *n = int(b->hs.size());
  if (nthreads) *nthreads = b->nthreads;
  return OPF_OK;
}

extern "C" int opf_batch_autotune(opf_batch* b) {
  if (!b) return OPF_ERR_INVALID_ARG;
  for (opf_handle* h : b->hs) {
    if (h->trsm_mode >= 0) continue;
    int rc = autotune_at_flat_start(h);
    if (rc != OPF_OK) return rc;
  }
  return OPF_OK;
}

extern "C" int opf_batch_solve(opf_batch* b, const opf_ipm_options* opt, opf_ipm_result* results,
                               double* wall_ms) {
  if (!b || !results) return OPF_ERR_INVALID_ARG;
  const int n = int(b->hs.size());
  std::atomic<int> next{0};
  std::vector<int> rcs(n, OPF_OK);
  const auto t0 = std::chrono::steady_clock::now();
  auto worker = [&]() {
    if (cudaSetDevice(b->device) != cudaSuccess) return;
    for (;;) {
      const int q = next.fetch_add(1);
      if (q >= n) break;
      const int i = b->order[q];
      rcs[i] = opf_solve(b->hs[i], opt, &results[i]);
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < b->nthreads; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (wall_ms) *wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  // the first instance whose loop failed with an error (not merely the iteration cap)
  for (int i = 0; i < n; ++i)
    if (rcs[i] != OPF_OK && rcs[i] != OPF_ERR_NO_CONVERGENCE) return rcs[i];
  for (int i = 0; i < n; ++i)
    if (rcs[i] != OPF_OK) return rcs[i];
  return OPF_OK;
}
