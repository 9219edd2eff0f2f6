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
//
// opf_batch_condense_factor is the batched form of the per-iteration hot path:
// the G_x refactorisation, both multi-RHS solves, K, H = K Z, Kred and the
// Cholesky of every instance run as one launch per phase over device work
// lists -- (instance, row) items in level order for the refactorisation,
// (instance, 32-column block) items for the solves, one thread-block cluster
// per instance for the Cholesky, and block ranges per instance for the
// elementwise phases -- so that the uneven instances fill the GPU together.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
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
  // batched condensation (built on its first call)
  bool bc_ready = false;
  cudaStream_t bs = nullptr;           // the batched launches' stream
  std::vector<cudaEvent_t> ev;         // per instance: its stream's work so far
  cudaEvent_t ev_done = nullptr;
  condipm::BatchInst* dI = nullptr;    // device descriptors
  condipm::BatchInst* hI = nullptr;    // pinned host copy
  int2* lu_items = nullptr;            // (instance, row), level order
  int n_lu_items = 0, lu_blocks = 1, lu_maxlen = 1;
  int2* cbs = nullptr;                 // (instance, column block)
  int ncbs = 0, nsn_max = 1;
  int* boff[condipm::BOFF_KINDS] = {};
  int nb[condipm::BOFF_KINDS] = {};
  int* st_host = nullptr;              // pinned: ST_WORDS per instance
  std::vector<void*> dev_allocs;
  // cluster sizes of the batched solves and Cholesky: 0 until the first call
  // times the candidates on the batch's own instances
  int trsm_cl = 0, chol_cl = 0;
  float tune_trsm_ms[4] = {}, tune_chol_ms[4] = {};   // candidates 2, 4, 8, 16 CTAs
  // once tuned, the whole batched sequence (descriptor upload, every phase,
  // the status read-back) is captured as one CUDA graph and replayed
  cudaGraphExec_t gexec = nullptr;
  bool graph_failed = false;
  long long graph_calls = 0;
  int* st_dev = nullptr;               // the active instances' status words, gathered
  // lockstep solves: the instances' loops meet at every condensation
  int mode = OPF_BATCH_LOCKSTEP;
  std::mutex mu;
  std::condition_variable cv;
  int active = 0, arrived = 0;
  long long generation = 0;
  std::vector<char> waiting;
  std::vector<const double*> rsu, rsx, rss;
  std::vector<int> rstatus;
  long long lockstep_calls = 0;        // batched condensations issued by lockstep solves
};

#define TRY_B(x)                   \
  do {                             \
    int r_ = (x);                  \
    if (r_ != OPF_OK) return r_;   \
  } while (0)

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
  if (b->bs) cudaStreamSynchronize(b->bs);
  for (size_t i = 0; i < b->streams.size(); ++i) {
    cudaStreamSynchronize(b->streams[i]);
    if (i < b->prev.size()) b->hs[i]->s = b->prev[i];
    cudaStreamDestroy(b->streams[i]);
  }
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->bs) cudaStreamDestroy(b->bs);
  for (void* p : b->dev_allocs) cudaFree(p);
  if (b->hI) cudaFreeHost(b->hI);
  if (b->st_host) cudaFreeHost(b->st_host);
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
  // batches run the condensed step (their rendezvous is the batched condensation)
  if (opt && opt->linear_solver != OPF_LINSOLVE_CONDENSED) return OPF_ERR_INVALID_ARG;
  const int n = int(b->hs.size());
  std::vector<int> rcs(n, OPF_OK);
  const auto t0 = std::chrono::steady_clock::now();
  if (b->mode == OPF_BATCH_LOCKSTEP) {
    // one host thread per instance; the loops meet at every condensation, which
    // one batched call serves (instances that have finished are masked)
    for (opf_handle* h : b->hs)
      if (h->opt.route == OPF_ROUTE_EXPLICIT) return OPF_ERR_INVALID_ARG;
    {
      std::lock_guard<std::mutex> lk(b->mu);
      b->active = n;
      b->arrived = 0;
      b->waiting.assign(n, 0);
      b->rsu.assign(n, nullptr);
      b->rsx.assign(n, nullptr);
      b->rss.assign(n, nullptr);
      b->rstatus.assign(n, OPF_OK);
    }
    auto run = [&](int i) {
      opf_handle* h = b->hs[i];
      if (cudaSetDevice(b->device) == cudaSuccess) {
        h->batch = b;
        h->batch_idx = i;
        rcs[i] = opf_solve(h, opt, &results[i]);
        h->batch = nullptr;
        h->batch_idx = -1;
      } else {
        rcs[i] = OPF_ERR_CUDA;
      }
      batch_leave(b);
    };
    std::vector<std::thread> pool;
    for (int i = 1; i < n; ++i) pool.emplace_back(run, i);
    run(0);
    for (auto& th : pool) th.join();
  } else {
    std::atomic<int> next{0};
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
  }
  if (wall_ms) *wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  // the first instance whose loop failed with an error (not merely the iteration cap)
  for (int i = 0; i < n; ++i)
    if (rcs[i] != OPF_OK && rcs[i] != OPF_ERR_NO_CONVERGENCE) return rcs[i];
  for (int i = 0; i < n; ++i)
    if (rcs[i] != OPF_OK) return rcs[i];
  return OPF_OK;
}

// ------------------------------------------------------------------ batched condensation
namespace condipm {
namespace {

constexpr int BATCH_CL_CANDIDATES[4] = {2, 4, 8, 16};

template <class T>
int dev_upload(opf_batch* b, T** dst, const std::vector<T>& v) {
  const size_t n = std::max<size_t>(1, v.size());
  if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess) return OPF_ERR_OOM;
  b->dev_allocs.push_back(*dst);
  if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return OPF_ERR_CUDA;
  return OPF_OK;
}

// work lists and per-instance block ranges of the batched launches
int batch_setup(opf_batch* b) {
  const int n = int(b->hs.size());
  for (opf_handle* h : b->hs)
    if (h->opt.route == OPF_ROUTE_EXPLICIT) return OPF_ERR_INVALID_ARG;
  // refactorisation rows: level by level, instances in order within a level
  std::vector<int2> items;
  int maxlev = 0;
  for (opf_handle* h : b->hs) {
    maxlev = std::max(maxlev, h->P.fwd.nlev);
    b->lu_maxlen = std::max(b->lu_maxlen, h->lu_maxlen);
  }
  for (int l = 0; l < maxlev; ++l)
    for (int i = 0; i < n; ++i) {
      const Levels& L = b->hs[i]->P.fwd;
      if (l >= L.nlev) continue;
      for (int q = L.ptr[l]; q < L.ptr[l + 1]; ++q) items.push_back(make_int2(i, L.rows[q]));
    }
  b->n_lu_items = int(items.size());
  TRY_B(dev_upload(b, &b->lu_items, items));
  const int mb = batch_lu_max_blocks(b->lu_maxlen);
  if (mb < 1) return OPF_ERR_CUDA;
  b->lu_blocks = std::max(1, std::min(mb, (b->n_lu_items + 7) / 8));
  // solve items
  std::vector<int2> cb;
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < (b->hs[i]->P.nu + 31) / 32; ++c) cb.push_back(make_int2(i, c));
  b->ncbs = int(cb.size());
  TRY_B(dev_upload(b, &b->cbs, cb));
  // block ranges: each instance gets blocks in proportion to its elements of
  // that launch shape (BATCH_EW_ITEMS per thread)
  const long long per_block = (long long)BATCH_EW_THREADS * BATCH_EW_ITEMS;
  for (int k = 0; k < BOFF_KINDS; ++k) {
    std::vector<int> off(n + 1, 0);
    for (int i = 0; i < n; ++i) {
      const opf_handle* h = b->hs[i];
      const Plan& P = h->P;
      long long work = 1;
      switch (k) {
        case BOFF_LU: work = std::max<long long>(32LL * P.nx, P.nw); break;
        case BOFF_K: work = std::max<long long>(P.K.nnz(), P.G.nnz()); break;
        case BOFF_X: work = std::max<long long>((long long)P.nx * h->ldp, P.LU.nnz()); break;
        case BOFF_W: work = (long long)P.nw * P.nu; break;
        case BOFF_U: work = (long long)P.nu * P.nu; break;
        case BOFF_F:
          work = std::max(std::max<long long>(P.Lo.nnz(), P.Up.nnz()),
                          std::max(h->stLo.nslots, h->stUp.nslots));
          break;
        default:   // BOFF_D: one warp per (factor, supernode), four warps per block
          work = 2LL * (long long)(P.csL.sn_first.size() + P.csU.sn_first.size()) * per_block / 4;
      }
      const long long nbk = std::max(1LL, std::min(65536LL, (work + per_block - 1) / per_block));
      off[i + 1] = off[i] + int(nbk);
    }
    b->nb[k] = off[n];
    TRY_B(dev_upload(b, &b->boff[k], off));
  }
  for (opf_handle* h : b->hs)
    b->nsn_max = std::max(b->nsn_max, int(std::max(h->P.csL.sn_first.size(), h->P.csU.sn_first.size())));
  if (cudaMalloc(&b->dI, sizeof(BatchInst) * n) != cudaSuccess) return OPF_ERR_OOM;
  b->dev_allocs.push_back(b->dI);
  if (cudaMallocHost(&b->hI, sizeof(BatchInst) * n) != cudaSuccess) return OPF_ERR_OOM;
  if (cudaMallocHost(&b->st_host, sizeof(int) * ST_WORDS * n) != cudaSuccess) return OPF_ERR_OOM;
  if (cudaMalloc(&b->st_dev, sizeof(int) * ST_WORDS * n) != cudaSuccess) return OPF_ERR_OOM;
  b->dev_allocs.push_back(b->st_dev);
  if (cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) != cudaSuccess) return OPF_ERR_CUDA;
  b->ev.resize(n, nullptr);
  for (int i = 0; i < n; ++i)
    if (cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) != cudaSuccess) return OPF_ERR_CUDA;
  if (cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming) != cudaSuccess) return OPF_ERR_CUDA;
  b->bc_ready = true;
  return OPF_OK;
}

BatchInst describe(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s, double delta_w) {
  const Plan& P = h->P;
  BatchInst B{};
  B.nx = P.nx; B.nu = P.nu; B.nw = P.nw; B.m = P.m; B.ld = h->ldp;
  B.nnzG = P.G.nnz(); B.nnzLU = P.LU.nnz(); B.nnzK = P.K.nnz(); B.nnzLo = P.Lo.nnz(); B.nnzUp = P.Up.nnz();
  B.Gx_to_LU = h->Gx_to_LU; B.LU_rp = h->LU_rp; B.LU_ci = h->LU_ci; B.LU_diag = h->LU_diag;
  B.upd_ptr = h->upd_ptr; B.upd_pos = h->upd_pos; B.Gval = h->Gval;
  B.LUval = h->LUval; B.inv_diag = h->inv_diag; B.rmax = h->rmax; B.flags = h->flags; B.st = h->st;
  B.maxlen = h->lu_maxlen;
  B.Lo_map = h->Lo_map; B.Ut_map = h->Ut_map; B.Up_map = h->Up_map; B.Lt_map = h->Lt_map;
  B.Lo_val = h->Lo_val; B.Ut_val = h->Ut_val; B.Up_val = h->Up_val; B.Lt_val = h->Lt_val;
  for (int k = 0; k < 2; ++k) {
    const opf_handle::StBuf& S = k ? h->stUp : h->stLo;
    B.st_nslots[k] = S.nslots;
    B.st_slot[k] = S.slot;
    B.st_src[k] = S.src;
    B.st_a[k] = reinterpret_cast<double*>(S.bytes_a);
    B.st_b[k] = reinterpret_cast<double*>(S.bytes_b);
  }
  const int nl = int(P.csL.sn_first.size()), nuu = int(P.csU.sn_first.size());
  const ColDev& L = h->csL;
  const ColDev& U = h->csU;
  B.dj[0] = DiagInvJob{nl, 0, L.sn_first, L.sn_w, h->bkL.d_off, L.int_beg, h->Lo_val, nullptr, h->D_L};
  B.dj[1] = DiagInvJob{nl, 0, L.sn_first, L.sn_w, h->bkL.d_off, L.int_beg, h->Ut_val, h->inv_diag, h->D_Ut};
  B.dj[2] = DiagInvJob{nuu, 1, U.sn_first, U.sn_w, h->bkU.d_off, U.int_beg, h->Up_val, h->inv_diag, h->D_U};
  B.dj[3] = DiagInvJob{nuu, 1, U.sn_first, U.sn_w, h->bkU.d_off, U.int_beg, h->Lt_val, nullptr, h->D_Lt};
  B.Wval = h->Wval; B.Aval = h->Aval;
  B.KAA_ptr = h->KAA_ptr; B.KAA_r = h->KAA_r; B.KAA_a = h->KAA_a; B.KAA_b = h->KAA_b;
  B.K_diag = h->K_diag; B.perm = h->perm; B.K_rp = h->K_rp; B.K_ci = h->K_ci;
  B.sig_u = sig_u; B.sig_x = sig_x; B.sig_s_in = sig_s;
  B.sig_s = h->sig_s; B.sig_c = h->sig_c; B.Kval = h->Kval;
  B.Zt = h->Zt; B.H = h->H; B.Y = h->ybuf;
  B.PGu_rp = h->PGu_rp; B.PGu_ci = h->PGu_ci; B.PGu_map = h->PGu_map;
  B.GuT_rp = h->GuT_rp; B.GuT_ci = h->GuT_ci; B.GuT_map = h->GuT_map;
  B.bkL = h->bkL; B.bkU = h->bkU; B.Lo_ci = h->Lo_ci; B.Up_ci = h->Up_ci;
  B.D_L = h->D_L; B.D_Ut = h->D_Ut; B.D_U = h->D_U; B.D_Lt = h->D_Lt;
  B.Kred = h->Kred; B.F = h->F; B.Fdinv = h->Fdinv;
  B.delta_w = delta_w;
  return B;
}

}  // namespace
}  // namespace condipm

namespace condipm {

// The batched condensation of the instances with on[i] set (the others are
// masked: their work-list items are skipped on the device).
int batch_condense_subset(opf_batch* b, const std::vector<char>& on, const double* const* sig_u,
                          const double* const* sig_x, const double* const* sig_s, const double* delta_w, int* status,
                          int* fail_col) {
  const int n = int(b->hs.size());
  for (int i = 0; i < n; ++i) {
    if (!on[i]) continue;
    const opf_handle* h = b->hs[i];
    if (!h->have_W || !sig_u[i] || !sig_x[i] || !sig_s[i] || (delta_w && !(delta_w[i] >= 0.0)))
      return OPF_ERR_INVALID_ARG;
    if ((size_t)h->P.nx * h->ldp > h->ybuf_cap) return OPF_ERR_INVALID_ARG;
  }
  if (!b->bc_ready) {
    const int rc = batch_setup(b);
    if (rc != OPF_OK) return rc;
  }
  for (int i = 0; i < n; ++i) {
    if (on[i]) {
      b->hI[i] = describe(b->hs[i], sig_u[i], sig_x[i], sig_s[i], delta_w ? delta_w[i] : 0.0);
      b->hI[i].active = 1;
    } else {
      b->hI[i] = BatchInst{};
      b->hI[i].active = 0;
    }
  }
  // the batched launches follow every instance's work so far (its derivatives)
  for (int i = 0; i < n; ++i) {
    if (!on[i]) continue;
    if (cudaEventRecord(b->ev[i], b->hs[i]->s) != cudaSuccess) return OPF_ERR_CUDA;
    if (cudaStreamWaitEvent(b->bs, b->ev[i], 0) != cudaSuccess) return OPF_ERR_CUDA;
  }
  cudaStream_t s = b->bs;
  const long long spin = b->hs[0]->spin_limit;
  // A5: refactorisation with its prologue and epilogue
  auto front = [&]() {
    cudaError_t e = launch_batch_prologue(s, b->dI, n, b->boff, b->nb);
    if (e == cudaSuccess)
      e = launch_batch_lu(s, b->dI, b->lu_items, b->n_lu_items, b->lu_blocks, b->lu_maxlen, 1u, spin);
    if (e == cudaSuccess)
      e = launch_batch_factor_post(s, b->dI, n, b->boff[BOFF_F], b->nb[BOFF_F], b->boff[BOFF_D], b->nb[BOFF_D]);
    return e;
  };
  // time a launch on the batch's stream (the tuning of the first call)
  cudaEvent_t ta = nullptr, tb = nullptr;
  auto timed = [&](auto&& launch, float* ms) {
    cudaError_t e = cudaEventRecord(ta, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(tb, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(tb);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ta, tb);
    return e;
  };
  auto upload = [&]() {
    return cudaMemcpyAsync(b->dI, b->hI, sizeof(BatchInst) * n, cudaMemcpyHostToDevice, s);
  };
  // the active instances' status words into one pinned buffer
  auto statuses = [&]() {
    cudaError_t e = launch_batch_status(s, b->dI, n, b->st_dev);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->st_host, b->st_dev, sizeof(int) * ST_WORDS * n, cudaMemcpyDeviceToHost, s);
    return e;
  };
  // the tuned sequence, as enqueued (eagerly or into the graph)
  auto tuned_sequence = [&]() {
    cudaError_t e = upload();
    if (e == cudaSuccess) e = launch_batch_prologue(s, b->dI, n, b->boff, b->nb);
    if (e == cudaSuccess)
      e = launch_batch_lu(s, b->dI, b->lu_items, b->n_lu_items, b->lu_blocks, b->lu_maxlen, 1u, spin);
    if (e == cudaSuccess)
      e = launch_batch_factor_post(s, b->dI, n, b->boff[BOFF_F], b->nb[BOFF_F], b->boff[BOFF_D], b->nb[BOFF_D]);
    if (e == cudaSuccess) e = launch_batch_trsm(s, b->dI, b->cbs, b->ncbs, 0, b->trsm_cl);
    if (e == cudaSuccess) e = launch_batch_spmm(s, b->dI, n, b->boff[BOFF_W], b->nb[BOFF_W], 0);
    if (e == cudaSuccess) e = launch_batch_trsm(s, b->dI, b->cbs, b->ncbs, 1, b->trsm_cl);
    if (e == cudaSuccess) e = launch_batch_spmm(s, b->dI, n, b->boff[BOFF_U], b->nb[BOFF_U], 1);
    if (e == cudaSuccess) e = launch_batch_kred(s, b->dI, n, b->boff[BOFF_U], b->nb[BOFF_U]);
    if (e == cudaSuccess) e = launch_batch_chol(s, b->dI, n, b->chol_cl);
    if (e == cudaSuccess) e = statuses();
    return e;
  };
  const bool tune = b->trsm_cl == 0 || b->chol_cl == 0;
  int trsm_cl = b->trsm_cl, chol_cl = b->chol_cl;
  cudaError_t e = cudaSuccess;
  if (!tune) {
    if (!b->gexec && !b->graph_failed) {
      cudaGraph_t g = nullptr;
      bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const cudaError_t ce = tuned_sequence();
        ok = cudaStreamEndCapture(s, &g) == cudaSuccess && ce == cudaSuccess && g &&
             cudaGraphInstantiate(&b->gexec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      if (!ok) {
        b->gexec = nullptr;
        b->graph_failed = true;
      }
      cudaGetLastError();
    }
    if (b->gexec) {
      e = cudaGraphLaunch(b->gexec, s);
      ++b->graph_calls;
    } else {
      e = tuned_sequence();
    }
  }
  if (tune) {
    e = upload();
    if (e == cudaSuccess) e = cudaEventCreate(&ta);
    if (e == cudaSuccess) e = cudaEventCreate(&tb);
  }
  if (tune) {
    // A6 (S_x): with the tuned cluster size, or each candidate after its own
    // refactorisation (the solve works in place; every cluster size gives the
    // same result, each row being summed by one warp in one order)
    if (e == cudaSuccess && trsm_cl == 0) {
      float best = 1e30f;
      for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
        const int cl = BATCH_CL_CANDIDATES[c];
        if (batch_trsm_clusters(cl) < 1) continue;
        e = front();
        float ms = 0.f;
        if (e == cudaSuccess) e = timed([&]() { return launch_batch_trsm(s, b->dI, b->cbs, b->ncbs, 0, cl); }, &ms);
        b->tune_trsm_ms[c] = ms;
        if (ms < best) { best = ms; trsm_cl = cl; }
        if (c < 3 && e == cudaSuccess) e = cudaStreamSynchronize(s);
      }
      // the last candidate's solve stands only if it is the pick: redo otherwise
      if (e == cudaSuccess && trsm_cl != BATCH_CL_CANDIDATES[3]) {
        e = front();
        if (e == cudaSuccess) e = launch_batch_trsm(s, b->dI, b->cbs, b->ncbs, 0, trsm_cl);
      }
    } else if (e == cudaSuccess) {
      e = front();
      if (e == cudaSuccess) e = launch_batch_trsm(s, b->dI, b->cbs, b->ncbs, 0, trsm_cl);
    }
    // A7: H = K Z, Psi = G_x^{-T} H_x, H_u -= G_u^T Psi, Kred and F
    if (e == cudaSuccess) e = launch_batch_spmm(s, b->dI, n, b->boff[BOFF_W], b->nb[BOFF_W], 0);
    if (e == cudaSuccess) e = launch_batch_trsm(s, b->dI, b->cbs, b->ncbs, 1, trsm_cl);
    if (e == cudaSuccess) e = launch_batch_spmm(s, b->dI, n, b->boff[BOFF_U], b->nb[BOFF_U], 1);
    // A9: Cholesky, with the tuned cluster size or each candidate on a fresh F
    if (e == cudaSuccess && chol_cl == 0) {
      float best = 1e30f;
      int last = 0;
      for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
        const int cl = BATCH_CL_CANDIDATES[c];
        if (batch_chol_clusters(cl) < 1) continue;
        e = launch_batch_kred(s, b->dI, n, b->boff[BOFF_U], b->nb[BOFF_U]);
        float ms = 0.f;
        if (e == cudaSuccess) e = timed([&]() { return launch_batch_chol(s, b->dI, n, cl); }, &ms);
        b->tune_chol_ms[c] = ms;
        if (ms < best) { best = ms; chol_cl = cl; }
        last = cl;
      }
      if (e == cudaSuccess && chol_cl != last) {
        e = launch_batch_kred(s, b->dI, n, b->boff[BOFF_U], b->nb[BOFF_U]);
        if (e == cudaSuccess) e = launch_batch_chol(s, b->dI, n, chol_cl);
      }
    } else if (e == cudaSuccess) {
      e = launch_batch_kred(s, b->dI, n, b->boff[BOFF_U], b->nb[BOFF_U]);
      if (e == cudaSuccess) e = launch_batch_chol(s, b->dI, n, chol_cl);
    }
    if (ta) cudaEventDestroy(ta);
    if (tb) cudaEventDestroy(tb);
  }
  if (tune && e == cudaSuccess) e = statuses();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    note_cuda_error(e);
    return OPF_ERR_CUDA;
  }
  int first = OPF_OK;
  if (tune) {
    // keep the picks when every instance factored completely (an early stop on
    // a non-positive pivot makes a candidate look fast); else tune again later
    bool complete = true;
    for (int i = 0; i < n; ++i)
      if (on[i] && (b->st_host[ST_WORDS * i + ST_CODE] != 0 || b->st_host[ST_WORDS * i + ST_TIMEOUT] != 0))
        complete = false;
    if (complete) {
      b->trsm_cl = trsm_cl;
      b->chol_cl = chol_cl;
    }
  }
  for (int i = 0; i < n; ++i) {
    if (!on[i]) continue;
    opf_handle* h = b->hs[i];
    const int* st = b->st_host + ST_WORDS * i;
    int rc = OPF_OK;
    if (st[ST_TIMEOUT]) rc = OPF_ERR_TIMEOUT;
    else if (st[ST_CODE] == DEV_NOT_PD) rc = OPF_ERR_NOT_PD;
    else if (st[ST_CODE] == DEV_SINGULAR) rc = OPF_ERR_SINGULAR;
    else if (st[ST_CODE] != 0) rc = OPF_ERR_CUDA;
    status[i] = rc;
    if (fail_col) fail_col[i] = rc == OPF_ERR_NOT_PD ? st[ST_INFO] : -1;
    // the handle is left as after opf_condense + opf_kkt_factor
    h->epoch = 1;
    h->have_lu = rc == OPF_OK || rc == OPF_ERR_NOT_PD;
    h->have_condense = h->have_lu;
    h->psi_valid = h->have_lu;
    h->have_factor = rc == OPF_OK;
    h->delta_w = delta_w ? delta_w[i] : 0.0;
    h->delta_c = 0.0;
    h->finv_valid = false;
    h->sens_ready = false;
    if (rc != OPF_OK) {
      cudaMemsetAsync(h->st, 0, sizeof(int) * ST_WORDS, s);
      cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, s);
      if (first == OPF_OK) first = rc;
    }
  }
  // later work on each instance's stream follows the batched launches
  if (cudaEventRecord(b->ev_done, s) != cudaSuccess) return OPF_ERR_CUDA;
  for (int i = 0; i < n; ++i)
    if (on[i] && cudaStreamWaitEvent(b->hs[i]->s, b->ev_done, 0) != cudaSuccess) return OPF_ERR_CUDA;
  return first;
}

namespace {
// issue the batched condensation for the instances waiting now (mu held)
void rendezvous_fire(opf_batch* b) {
  const int n = int(b->hs.size());
  std::vector<int> fc(n, -1);
  const int rc = batch_condense_subset(b, b->waiting, b->rsu.data(), b->rsx.data(), b->rss.data(), nullptr,
                                       b->rstatus.data(), fc.data());
  for (int i = 0; i < n; ++i)
    if (b->waiting[i] && rc != OPF_OK && rc != OPF_ERR_NOT_PD && rc != OPF_ERR_SINGULAR && rc != OPF_ERR_TIMEOUT)
      b->rstatus[i] = rc;   // the call itself failed
  std::fill(b->waiting.begin(), b->waiting.end(), 0);
  b->arrived = 0;
  ++b->generation;
  ++b->lockstep_calls;
  b->cv.notify_all();
}
}  // namespace

// A lockstep solve's condensation and first Cholesky attempt: wait until every
// instance still iterating has arrived, then one batched call serves them all.
int batch_join(opf_batch* b, int idx, const double* su, const double* sx, const double* ss) {
  std::unique_lock<std::mutex> lk(b->mu);
  b->rsu[idx] = su;
  b->rsx[idx] = sx;
  b->rss[idx] = ss;
  b->waiting[idx] = 1;
  ++b->arrived;
  const long long g = b->generation;
  if (b->arrived >= b->active) rendezvous_fire(b);
  else b->cv.wait(lk, [&]() { return b->generation != g; });
  return b->rstatus[idx];
}

// An instance's loop has ended: the others no longer wait for it.
void batch_leave(opf_batch* b) {
  std::unique_lock<std::mutex> lk(b->mu);
  --b->active;
  if (b->active > 0 && b->arrived >= b->active) rendezvous_fire(b);
}

}  // namespace condipm

extern "C" int opf_batch_condense_factor(opf_batch* b, const double* const* sig_u, const double* const* sig_x,
                                         const double* const* sig_s, const double* delta_w, int* status,
                                         int* fail_col) {
  if (!b || !sig_u || !sig_x || !sig_s || !status) return OPF_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(b->mu);
  std::vector<char> on(b->hs.size(), 1);
  return batch_condense_subset(b, on, sig_u, sig_x, sig_s, delta_w, status, fail_col);
}

extern "C" int opf_batch_set_mode(opf_batch* b, int mode) {
  if (!b || (mode != OPF_BATCH_CONCURRENT && mode != OPF_BATCH_LOCKSTEP)) return OPF_ERR_INVALID_ARG;
  b->mode = mode;
  return OPF_OK;
}

extern "C" int opf_batch_stats(const opf_batch* b, long long* lockstep_calls, int* trsm_cl, int* chol_cl,
                               float* tune_ms, long long* graph_calls) {
  if (!b) return OPF_ERR_INVALID_ARG;
  if (lockstep_calls) *lockstep_calls = b->lockstep_calls;
  if (graph_calls) *graph_calls = b->graph_calls;
  if (trsm_cl) *trsm_cl = b->trsm_cl;
  if (chol_cl) *chol_cl = b->chol_cl;
  if (tune_ms)
    for (int c = 0; c < 4; ++c) {
      tune_ms[c] = b->tune_trsm_ms[c];
      tune_ms[4 + c] = b->tune_chol_ms[c];
    }
  return OPF_OK;
}

