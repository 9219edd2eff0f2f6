// C ABI of the condensed interior-point hot path (include/condipm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <new>
#include <string>
#include <vector>

#include "../../include/condipm.h"
#include "common.cuh"
#include "internal.h"
#include "opf_handle.h"
#include "plan.h"

using namespace condipm;

#define CK(call)                                                  \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      condipm::note_cuda_error(e_);                               \
      return OPF_ERR_CUDA;                                        \
    }                                                             \
  } while (0)

namespace condipm {
static std::atomic<unsigned long long> g_launches{0};
static std::atomic<int> g_last_cuda_error{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void note_cuda_error(cudaError_t e) { g_last_cuda_error.store(int(e), std::memory_order_relaxed); }
int last_cuda_error() { return g_last_cuda_error.load(std::memory_order_relaxed); }

cudaError_t allow_cluster16(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, fn})) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  done.insert({dev, fn});
  return cudaSuccess;
}

cudaError_t allow_max_smem(const void* fn) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, fn})) return cudaSuccess;
  int mx = 0;
  e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  // the opt-in limit covers static and dynamic shared memory together
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - int(fa.sharedSizeBytes));
  if (e != cudaSuccess) return e;
  done.insert({dev, fn});
  return cudaSuccess;
}
}  // namespace condipm

namespace condipm {

static cudaEvent_t take_event(opf_handle* h) {
  if (!h->evpool.empty()) {
    cudaEvent_t e = h->evpool.back();
    h->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// bracket the launches between ph_begin and ph_end with events (when profiling)
void ph_begin(opf_handle* h, int phase) {
  if (!h->profiling) return;
  h->open_phase = phase;
  h->open_ev = take_event(h);
  cudaEventRecord(h->open_ev, h->s);
}

void ph_end(opf_handle* h) {
  if (!h->profiling || h->open_phase < 0) return;
  cudaEvent_t b = take_event(h);
  cudaEventRecord(b, h->s);
  h->recs.push_back({h->open_phase, h->open_ev, b});
  h->open_phase = -1;
}

}  // namespace condipm

namespace {

template <class T>
int upload(opf_handle* h, T** dst, const std::vector<T>& v) {
  size_t n = std::max<size_t>(v.size(), 1);
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? OPF_ERR_OOM : OPF_ERR_CUDA;
  h->allocs.push_back(*dst);
  if (!v.empty()) {
    e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return OPF_ERR_CUDA;
  }
  return OPF_OK;
}

template <class T>
int alloc(opf_handle* h, T** dst, size_t n) {
  n = std::max<size_t>(n, 1);
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? OPF_ERR_OOM : OPF_ERR_CUDA;
  h->allocs.push_back(*dst);
  e = cudaMemset(*dst, 0, n * sizeof(T));
  return e == cudaSuccess ? OPF_OK : OPF_ERR_CUDA;
}

#define TRY(x)              \
  do {                      \
    int r_ = (x);           \
    if (r_ != OPF_OK) return r_; \
  } while (0)

int pick_cb(int ncols) {
  const int cands[4] = {8, 4, 2, 1};
  for (int c : cands)
    if ((ncols + c - 1) / c >= 300) return c;
  return 1;
}

int upload_all(opf_handle* h) {
  const Plan& P = h->P;
  TRY(upload(h, &h->end_i, P.end_i));
  TRY(upload(h, &h->end_k, P.end_k));
  TRY(upload(h, &h->end_h, P.end_h));
  TRY(upload(h, &h->gs, P.gs));
  TRY(upload(h, &h->bs, P.bs));
  TRY(upload(h, &h->gm, P.gm));
  TRY(upload(h, &h->bm, P.bm));
  TRY(upload(h, &h->bus_end_ptr, P.bus_end_ptr));
  TRY(upload(h, &h->bus_end, P.bus_end));
  TRY(upload(h, &h->g_row_P, P.g_row_P));
  TRY(upload(h, &h->g_row_Q, P.g_row_Q));
  TRY(upload(h, &h->gen_of_bus, P.gen_of_bus));
  TRY(upload(h, &h->th_w, P.th_w));
  TRY(upload(h, &h->vm_w, P.vm_w));
  TRY(upload(h, &h->Pd, P.Pd));
  TRY(upload(h, &h->Qd, P.Qd));
  TRY(upload(h, &h->c2, P.c2));
  TRY(upload(h, &h->c1, P.c1));
  std::vector<int> pg_of_w(P.nw, -1), slackpos(P.nw, -1);
  for (int k = 1; k < P.ng; ++k) pg_of_w[P.pg_w[k]] = k;
  for (int q = P.A.rp[0]; q < P.A.rp[1]; ++q) slackpos[P.A.ci[q]] = q;
  TRY(upload(h, &h->pg_of_w, pg_of_w));
  TRY(upload(h, &h->slackpos, slackpos));
  // evaluation buffers
  TRY(alloc(h, &h->Vm, P.nb));
  TRY(alloc(h, &h->Va, P.nb));
  TRY(alloc(h, &h->pq, 2 * (size_t)P.ne));
  TRY(alloc(h, &h->dsrc, 12 * (size_t)P.ne));
  TRY(alloc(h, &h->hpq, 20 * (size_t)P.ne));
  TRY(alloc(h, &h->hw, 10 * (size_t)P.ne));
  TRY(alloc(h, &h->wP, P.nb));
  TRY(alloc(h, &h->wQ, P.nb));
  TRY(alloc(h, &h->g, P.nx));
  TRY(alloc(h, &h->hv, P.m));
  TRY(alloc(h, &h->f, 1));
  TRY(alloc(h, &h->gradf, P.nw));
  TRY(alloc(h, &h->Pg, P.ng));
  // G, A
  TRY(upload(h, &h->Ggat_ptr, P.Ggat.ptr));
  TRY(upload(h, &h->Ggat_idx, P.Ggat.idx));
  TRY(upload(h, &h->Ggat_cst, P.Ggat.cst));
  TRY(alloc(h, &h->Gval, P.G.nnz()));
  TRY(upload(h, &h->Agat_ptr, P.Agat.ptr));
  TRY(upload(h, &h->Agat_idx, P.Agat.idx));
  TRY(upload(h, &h->Agat_cst, P.Agat.cst));
  TRY(alloc(h, &h->Aval, P.A.nnz()));
  TRY(upload(h, &h->A_rp, P.A.rp));
  TRY(upload(h, &h->A_ci_c, P.A_ci_c));
  // K / W
  TRY(upload(h, &h->K_rp, P.K.rp));
  TRY(upload(h, &h->K_ci, P.K.ci));
  TRY(upload(h, &h->Wgat_ptr, P.Wgat.ptr));
  TRY(upload(h, &h->Wgat_idx, P.Wgat.idx));
  TRY(upload(h, &h->Wgat_cst, P.Wgat.cst));
  TRY(upload(h, &h->Wsl_pos, P.Wslack_pos));
  TRY(upload(h, &h->Wsl_a, P.Wslack_a));
  TRY(upload(h, &h->Wsl_b, P.Wslack_b));
  TRY(upload(h, &h->K_diag, P.K_diag));
  TRY(upload(h, &h->KAA_ptr, P.KAA.ptr));
  TRY(upload(h, &h->KAA_r, P.KAA.r));
  TRY(upload(h, &h->KAA_a, P.KAA.a));
  TRY(upload(h, &h->KAA_b, P.KAA.b));
  TRY(upload(h, &h->Knat_map, P.Knat_map));
  TRY(upload(h, &h->perm, P.perm));
  TRY(upload(h, &h->c2w, P.c2w));
  TRY(alloc(h, &h->Wval, P.K.nnz()));
  TRY(alloc(h, &h->Kval, P.K.nnz()));
  TRY(alloc(h, &h->sig_c, P.nw));
  TRY(alloc(h, &h->sig_s, P.m));
  TRY(alloc(h, &h->sig_se, P.m));
  TRY(alloc(h, &h->ps_sc, P.m));
  // transposes
  TRY(upload(h, &h->AT_rp, P.AT.rp));
  TRY(upload(h, &h->AT_ci, P.AT.ci));
  TRY(upload(h, &h->AT_map, P.AT_map));
  TRY(upload(h, &h->PGu_rp, P.PGu.rp));
  TRY(upload(h, &h->PGu_ci, P.PGu.ci));
  TRY(upload(h, &h->PGu_map, P.PGu_map));
  TRY(upload(h, &h->GuT_rp, P.GuT.rp));
  TRY(upload(h, &h->GuT_ci, P.GuT.ci));
  TRY(upload(h, &h->GuT_map, P.GuT_map));
  TRY(upload(h, &h->Gc_rp, P.Gc.rp));
  TRY(upload(h, &h->Gc_ci, P.Gc.ci));
  TRY(upload(h, &h->Gc_map, P.Gc_map));
  TRY(upload(h, &h->GcT_rp, P.GcT.rp));
  TRY(upload(h, &h->GcT_ci, P.GcT.ci));
  TRY(upload(h, &h->GcT_map, P.GcT_map));
  TRY(upload(h, &h->GTn_rp, P.GTn.rp));
  TRY(upload(h, &h->GTn_ci, P.GTn.ci));
  TRY(upload(h, &h->GTn_map, P.GTn_map));
  TRY(upload(h, &h->ATn_rp, P.ATn.rp));
  TRY(upload(h, &h->ATn_ci, P.ATn.ci));
  TRY(upload(h, &h->ATn_map, P.ATn_map));
  // LU
  TRY(upload(h, &h->LU_rp, P.LU.rp));
  TRY(upload(h, &h->LU_ci, P.LU.ci));
  TRY(upload(h, &h->LU_diag, P.LU_diag));
  TRY(upload(h, &h->Gx_to_LU, P.Gx_to_LU));
  TRY(upload(h, &h->upd_ptr, P.upd_ptr));
  TRY(upload(h, &h->upd_pos, P.upd_pos));
  TRY(alloc(h, &h->LUval, P.LU.nnz()));
  TRY(alloc(h, &h->inv_diag, P.nx));
  TRY(alloc(h, &h->rmax, P.nx));
  TRY(alloc(h, &h->flags, P.nx));
  TRY(upload(h, &h->Lo_rp, P.Lo.rp));
  TRY(upload(h, &h->Lo_ci, P.Lo.ci));
  TRY(upload(h, &h->Lo_map, P.Lo_map));
  TRY(upload(h, &h->Ut_map, P.Ut_map));
  TRY(upload(h, &h->Up_rp, P.Up.rp));
  TRY(upload(h, &h->Up_ci, P.Up.ci));
  TRY(upload(h, &h->Up_map, P.Up_map));
  TRY(upload(h, &h->Lt_map, P.Lt_map));
  TRY(alloc(h, &h->Lo_val, P.Lo.nnz()));
  TRY(alloc(h, &h->Ut_val, P.Lo.nnz()));
  TRY(alloc(h, &h->Up_val, P.Up.nnz()));
  TRY(alloc(h, &h->Lt_val, P.Up.nnz()));
  TRY(upload(h, &h->fwd_ptr, P.fwd.ptr));
  TRY(upload(h, &h->fwd_rows, P.fwd.rows));
  TRY(upload(h, &h->bwd_ptr, P.bwd.ptr));
  TRY(upload(h, &h->bwd_rows, P.bwd.rows));
  h->st_cap = std::max(P.stL.max_chunk, P.stU.max_chunk);
  h->st_cap = (h->st_cap + 15) & ~15;
  for (int k = 0; k < 2; ++k) {
    const SnStream& S = k ? P.stU : P.stL;
    opf_handle::StBuf& D = k ? h->stUp : h->stLo;
    D.nchunks = int(S.chunk_off.size());
    D.nslots = (long long)S.slot.size();
    TRY(upload(h, &D.chunk_off, S.chunk_off));
    TRY(upload(h, &D.chunk_bytes, S.chunk_bytes));
    TRY(upload(h, &D.chunk_big_f, S.chunk_big_f));
    TRY(upload(h, &D.chunk_big_w, S.chunk_big_w));
    TRY(upload(h, &D.int_beg, (k ? P.snU : P.snL).int_beg));
    TRY(upload(h, &D.slot, S.slot));
    TRY(upload(h, &D.src, S.src));
    TRY(upload(h, &D.bytes_a, S.bytes));
    TRY(upload(h, &D.bytes_b, S.bytes));
  }
  for (int k = 0; k < 2; ++k) {
    const ColSched& C = k ? P.csU : P.csL;
    int *a, *b, *c, *d, *e, *f, *g0, *g, *hh, *i, *j, *l;
    TRY(upload(h, &a, C.lvl_ptr)); TRY(upload(h, &b, C.sn_first)); TRY(upload(h, &c, C.sn_w));
    TRY(upload(h, &d, C.lvl_seg_ptr)); TRY(upload(h, &e, C.seg_q0)); TRY(upload(h, &f, C.seg_q1));
    TRY(upload(h, &g0, C.seg_row));
    TRY(upload(h, &g, C.row_seg)); TRY(upload(h, &hh, C.row_nseg)); TRY(upload(h, &i, C.ext_beg));
    TRY(upload(h, &j, C.ext_end)); TRY(upload(h, &l, C.int_beg));
    (k ? h->csU : h->csL) = ColDev{C.nlev, C.maxseg, a, b, c, d, e, f, g0, g, hh, i, j, l};
  }
  // level-blocked schedules: each level's rows with their supernode, and the
  // offsets of the supernodes' dense inverses
  for (int k = 0; k < 2; ++k) {
    const ColSched& C = k ? P.csU : P.csL;
    std::vector<int> rptr(C.nlev + 1, 0), rows, rsn, doff(C.sn_first.size() + 1, 0);
    for (size_t q = 0; q < C.sn_first.size(); ++q) doff[q + 1] = doff[q] + C.sn_w[q] * C.sn_w[q];
    for (int l = 0; l < C.nlev; ++l) {
      for (int q = C.lvl_ptr[l]; q < C.lvl_ptr[l + 1]; ++q)
        for (int r = C.sn_first[q]; r < C.sn_first[q] + C.sn_w[q]; ++r) { rows.push_back(r); rsn.push_back(q); }
      rptr[l + 1] = int(rows.size());
    }
    const ColDev& cd = k ? h->csU : h->csL;
    int *a, *b, *c, *d;
    TRY(upload(h, &a, rptr)); TRY(upload(h, &b, rows)); TRY(upload(h, &c, rsn)); TRY(upload(h, &d, doff));
    (k ? h->bkU : h->bkL) = BlkDev{C.nlev, a, b, c, cd.sn_first, cd.sn_w, d, cd.ext_beg, cd.ext_end, k};
    for (int l = 0; l < C.nlev; ++l) h->lu1s_ymax = std::max(h->lu1s_ymax, rptr[l + 1] - rptr[l]);
    // the one-CTA form's row descriptions
    std::vector<int> ma(4 * rows.size()), mb(4 * rows.size());
    for (size_t q = 0; q < rows.size(); ++q) {
      const int r = rows[q], sn = rsn[q], f = C.sn_first[sn], w = C.sn_w[sn];
      ma[4 * q] = r; ma[4 * q + 1] = C.ext_beg[r]; ma[4 * q + 2] = C.ext_end[r]; ma[4 * q + 3] = 0;
      mb[4 * q] = r; mb[4 * q + 1] = r - f; mb[4 * q + 2] = w; mb[4 * q + 3] = doff[sn] + (r - f) * w;
    }
    int *pa, *pb;
    TRY(upload(h, &pa, ma)); TRY(upload(h, &pb, mb));
    (k ? h->l1U : h->l1L) = Lu1sDev{C.nlev, a, reinterpret_cast<const int4*>(pa), reinterpret_cast<const int4*>(pb)};
    const size_t nd = std::max<size_t>(1, size_t(doff.back()));
    if (k == 0) { TRY(alloc(h, &h->D_L, nd)); TRY(alloc(h, &h->D_Ut, nd)); }
    else { TRY(alloc(h, &h->D_U, nd)); TRY(alloc(h, &h->D_Lt, nd)); }
  }
  // the forward sweep's reach lists per full 32-column block of P G_u
  if (h->opt.dense_forward == 0 && P.nu >= 32) {
    std::vector<int> rptr, rq;
    build_forward_reach(P, P.csL, rptr, rq, h->rch_work);
    int *a, *b;
    TRY(upload(h, &a, rptr));
    TRY(upload(h, &b, rq.empty() ? std::vector<int>(1, 0) : rq));
    h->bkL.rch_ptr = a;
    h->bkL.rch_q = b;
    h->bkL.rch_nblk = P.nu / 32;
  }
  h->lu1s_ok = sizeof(double) * ((size_t)P.nx + (size_t)h->lu1s_ymax) <= trsm_lu1s_max_smem();
  // the cluster form of the one-right-hand-side solve, for 4, 8 and 16 CTAs
  for (int c = 0; c < 3; ++c) {
    const int CL = 4 << c;
    Cl1Dev dv[2];
    int ymax = 0, nlev = 0;
    for (int k = 0; k < 2; ++k) {
      ClSched S;
      if (!build_cl_sched(k ? P.csU : P.csL, CL, S).empty()) return OPF_ERR_INVALID_ARG;
      int *tp, *ta, *tb;
      TRY(upload(h, &tp, S.t_ptr)); TRY(upload(h, &ta, S.ta)); TRY(upload(h, &tb, S.tb));
      dv[k] = Cl1Dev{S.nlev, CL, S.ymax, tp, reinterpret_cast<const int4*>(ta), reinterpret_cast<const int4*>(tb)};
      ymax = std::max(ymax, S.ymax);
      nlev = std::max(nlev, S.nlev);
    }
    h->cl1L[c] = dv[0];
    h->cl1U[c] = dv[1];
    h->cl1_ok[c] = trsm_lu1c_max_clusters(CL, P.nx, ymax, nlev) >= 1;
  }
  h->ldp = (P.nu + 31) / 32 * 32;
  h->cs_ncb_max = std::max((P.nu + 31) / 32, 64);
  // dataflow task lists: phase A then phase B of each level's rows, each row's
  // supernode, and the supernodes its external entries lie in
  size_t nsn_max = 1, nck_max = 1, nchunked_max = 1;
  for (int k = 0; k < 2; ++k) {
    const ColSched& C = k ? P.csU : P.csL;
    const CSR& M = k ? P.Up : P.Lo;
    const int nsn = int(C.sn_first.size());
    nsn_max = std::max(nsn_max, size_t(nsn));
    std::vector<int> sn_of(P.nx, -1), task, dptr(P.nx + 1, 0), dsn, leaf;
    for (int q = 0; q < nsn; ++q)
      for (int r = C.sn_first[q]; r < C.sn_first[q] + C.sn_w[q]; ++r) sn_of[r] = q;
    // narrow supernodes without external entries need no waiting and no Y: a
    // separate pass multiplies them by their inverse blocks
    std::vector<char> is_leaf(nsn, 0);
    for (int q = 0; q < nsn; ++q) {
      bool ext = false;
      for (int r = C.sn_first[q]; r < C.sn_first[q] + C.sn_w[q]; ++r) ext = ext || C.ext_end[r] > C.ext_beg[r];
      if (!ext && C.sn_w[q] <= DF_LEAF_W) { is_leaf[q] = 1; leaf.push_back(q); }
    }
    // long rows: chunks of at most DF_CHUNK external entries, ids in row order
    std::vector<int> ck_row, ck_e0, ck_e1, rw_ck0(P.nx + 1, 0), rw_cidx(P.nx, 0);
    int nchunked = 0;
    for (int r = 0; r < P.nx; ++r) {
      const int e0 = C.ext_beg[r], len = C.ext_end[r] - e0;
      if (len > DF_CHUNK && !is_leaf[sn_of[r]]) {
        const int m = (len + DF_CHUNK - 1) / DF_CHUNK;
        for (int k = 0; k < m; ++k) {
          ck_row.push_back(r);
          ck_e0.push_back(e0 + int((long long)len * k / m));
          ck_e1.push_back(e0 + int((long long)len * (k + 1) / m));
        }
        rw_cidx[r] = nchunked++;
      }
      rw_ck0[r + 1] = int(ck_row.size());
    }
    for (int l = 0; l < C.nlev; ++l) {
      for (int q = C.lvl_ptr[l]; q < C.lvl_ptr[l + 1]; ++q)
        if (!is_leaf[q])
          for (int r = C.sn_first[q]; r < C.sn_first[q] + C.sn_w[q]; ++r) {
            if (rw_ck0[r + 1] > rw_ck0[r])
              for (int k = rw_ck0[r]; k < rw_ck0[r + 1]; ++k) task.push_back(P.nx + k);
            else
              task.push_back(r);
          }
      for (int q = C.lvl_ptr[l]; q < C.lvl_ptr[l + 1]; ++q)
        if (!is_leaf[q] && C.sn_w[q] > DF_INLINE_B)   // narrower supernodes: the last phase-A task does phase B
          for (int r = C.sn_first[q]; r < C.sn_first[q] + C.sn_w[q]; ++r) task.push_back(-1 - r);
    }
    std::vector<int> seen(nsn, -1);
    for (int r = 0; r < P.nx; ++r) {
      for (int e = C.ext_beg[r]; e < C.ext_end[r]; ++e) {
        const int q = sn_of[M.ci[e]];
        if (seen[q] != r) { seen[q] = r; dsn.push_back(q); }
      }
      dptr[r + 1] = int(dsn.size());
    }
    const ColDev& cd = k ? h->csU : h->csL;
    const BlkDev& bd = k ? h->bkU : h->bkL;
    int *a, *b, *c, *d, *e, *f1, *f2, *f3, *f4, *f5;
    TRY(upload(h, &a, task)); TRY(upload(h, &b, sn_of)); TRY(upload(h, &c, dptr)); TRY(upload(h, &d, dsn));
    TRY(upload(h, &e, leaf));
    TRY(upload(h, &f1, ck_row)); TRY(upload(h, &f2, ck_e0)); TRY(upload(h, &f3, ck_e1));
    TRY(upload(h, &f4, rw_ck0)); TRY(upload(h, &f5, rw_cidx));
    (k ? h->dfU : h->dfL) = DfDev{int(task.size()), nsn, a, b, cd.sn_first, cd.sn_w, bd.d_off, cd.ext_beg,
                                  cd.ext_end, c, d, int(leaf.size()), e, P.nx, int(ck_row.size()), nchunked,
                                  f1, f2, f3, f4, f5, k};
    nck_max = std::max(nck_max, ck_row.size());
    nchunked_max = std::max(nchunked_max, size_t(nchunked));
  }
  TRY(alloc(h, &h->df_cnt, (size_t)h->cs_ncb_max * (2 * nsn_max + nchunked_max)));
  TRY(alloc(h, &h->df_part, nck_max * (size_t)h->cs_ncb_max * 32));
  {
    const int maxseg = std::max(1, std::max(P.csL.maxseg, P.csU.maxseg));
    TRY(alloc(h, &h->cs_scratch, (size_t)h->cs_ncb_max * maxseg * 32));
    TRY(alloc(h, &h->cs_bar, (size_t)h->cs_ncb_max));
  }
  // dense
  TRY(alloc(h, &h->Zt, (size_t)P.nw * h->ldp));
  TRY(alloc(h, &h->H, (size_t)P.nw * h->ldp));
  TRY(alloc(h, &h->Kred, (size_t)P.nu * P.nu));
  TRY(alloc(h, &h->F, (size_t)P.nu * P.nu));
  TRY(alloc(h, &h->Fdinv, (size_t)P.nu));
  TRY(alloc(h, &h->st, ST_WORDS));
  TRY(alloc(h, &h->pf_ws, (size_t)P.nx + 1));
  TRY(alloc(h, &h->bar, 4));
  TRY(alloc(h, &h->chol_cnt, 3 * (size_t)((P.nu + 31) / 32 + 1)));
  TRY(alloc(h, &h->Finv, (size_t)std::max(1, (P.nu + 31) / 32) * 32 * 32));
  h->chol_solve_cl = (P.nu + 31) / 32 > 8 ? 16 : 8;
  TRY(alloc(h, &h->cs_tmp, (size_t)P.nu));
  CK(launch_set_identity(0, P.nu, h->Zt, h->ldp));
  // launch shapes
  int maxlen = 1;
  for (int i = 0; i < P.nx; ++i) maxlen = std::max(maxlen, P.LU.rp[i + 1] - P.LU.rp[i]);
  h->lu_maxlen = maxlen;
  h->lu_threads = 256;
  int mb = lu_refactor_max_blocks(h->lu_threads, (size_t)(h->lu_threads / 32) * maxlen * sizeof(double));
  int need = (P.nx + 7) / 8;
  h->lu_blocks = std::max(1, std::min(mb, need));
  h->chol_blocks = chol_grid_cap(P.nu);
  if (h->opt.chol_form == 2) {
    // the dataflow form until the first complete factorisation tunes it: one CTA
    // per SM, a quarter of the first step's panel row groups in the panel group
    const int nb = std::max(2, std::min(chol_df_max_blocks(), device_sms()));
    const int rows0 = (std::max(0, P.nu - 32) + 7) / 8;
    h->chol_df = 1;
    h->chol_blocks = nb;
    h->chol_np = std::max(1, std::min(nb / 3, std::max(8, rows0 / 4)));
  }
  h->cs_ksplit_max = std::max(1, trsm_cols_max_blocks());
  h->blk_max = std::max(1, trsm_blk_max_blocks());
  for (int i = 0; i < 3; ++i) h->blk_max_minb[i] = std::max(1, trsm_blk_max_blocks(BLK_MINB[i]));
  h->df_max = std::max(1, trsm_df_max_blocks());
  if (!ybuf_reserve(h, (size_t)P.nx * h->ldp)) return OPF_ERR_OOM;
  {
    h->sn_cb = trsm_st_max_cb(P.nx, h->st_cap);
  }
  CK(cudaDeviceSynchronize());
  return OPF_OK;
}

}  // namespace

namespace condipm {
// device status -> OPF code (synchronises the stream); clears the word
int read_status(opf_handle* h, int* info) {
  int st[ST_WORDS];
  CK(cudaMemcpyAsync(st, h->st, sizeof(st), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (st[ST_CODE] == 0 && st[ST_TIMEOUT] == 0) return OPF_OK;
  CK(cudaMemsetAsync(h->st, 0, sizeof(int) * ST_WORDS, h->s));
  CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->s));
  if (info) *info = st[ST_INFO];
  if (st[ST_TIMEOUT]) return OPF_ERR_TIMEOUT;
  if (st[ST_CODE] == DEV_NOT_PD) return OPF_ERR_NOT_PD;
  if (st[ST_CODE] == DEV_SINGULAR) return OPF_ERR_SINGULAR;
  return OPF_ERR_CUDA;
}

// A captured graph of the condensation holds the addresses of these buffers:
// when one is reallocated the graph is dropped, so that it is captured again.
static void drop_graph(opf_handle* h) {
  if (h->cf_exec) cudaGraphExecDestroy(h->cf_exec);
  h->cf_exec = nullptr;
}

double* ybuf_reserve(opf_handle* h, size_t n) {
  if (n > h->ybuf_cap) {
    drop_graph(h);
    if (h->ybuf) cudaFree(h->ybuf);
    h->ybuf = nullptr;
    h->ybuf_cap = 0;
    if (cudaMalloc(&h->ybuf, n * sizeof(double)) != cudaSuccess) return nullptr;
    h->ybuf_cap = n;
  }
  return h->ybuf;
}

double* workspace(opf_handle* h, size_t n) {
  if (n > h->ws_cap) {
    drop_graph(h);
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_cap = 0;
    if (cudaMalloc(&h->ws, n * sizeof(double)) != cudaSuccess) return nullptr;
    h->ws_cap = n;
  }
  return h->ws;
}

// Newton-Raphson on g(x, u) = 0 for x at fixed u (Sec. 4.4): residual, its
// max-norm on the host, refactorisation of G_x and one solve per iteration.
int powerflow_impl(opf_handle* h, const double* u, double* x, double tol, int max_iter, int* iters) {
  const Plan& P = h->P;
  double* ws = h->pf_ws;
  int rc = OPF_ERR_PF_FAILED;
  int k = 0;
  for (; k <= max_iter; ++k) {
    int r = eval_impl(h, x, u, nullptr, nullptr, false);
    if (r != OPF_OK) { rc = r; break; }
    double nrm = 0.0;
    if (launch_absmax(h->s, P.nx, h->g, ws + P.nx) != cudaSuccess ||
        cudaMemcpyAsync(&nrm, ws + P.nx, sizeof(double), cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
        cudaStreamSynchronize(h->s) != cudaSuccess) { rc = OPF_ERR_CUDA; break; }
    if (nrm <= tol) { rc = OPF_OK; break; }
    if (!(nrm < 1e10) || k == max_iter) break;
    r = eval_impl(h, x, u, nullptr, nullptr, true);
    if (r == OPF_OK) r = factor_async(h);
    if (r == OPF_OK) r = read_status(h, nullptr);
    if (r == OPF_OK) r = opf_gx_solve(h, 0, h->g, ws, 1);
    if (r != OPF_OK) { rc = r == OPF_ERR_SINGULAR ? OPF_ERR_PF_FAILED : r; break; }
    if (launch_axpby(h->s, P.nx, -1.0, ws, 1.0, x, x) != cudaSuccess) { rc = OPF_ERR_CUDA; break; }
  }
  cudaStreamSynchronize(h->s);
  if (iters) *iters = k;
  h->have_W = false;
  h->have_condense = false;
  h->have_factor = false;
  return rc;
}

// grad_w L = grad f + G^T lam + A^T y at the last derivative evaluation (device, natural order)
int lagrangian_gradient(opf_handle* h, const double* lam, const double* y, double* out) {
  const Plan& P = h->P;
  CK(cudaMemcpyAsync(out, h->gradf, sizeof(double) * P.nw, cudaMemcpyDeviceToDevice, h->s));
  if (lam) CK(launch_spmm(h->s, P.nw, h->GTn_rp, h->GTn_ci, h->Gval, h->GTn_map, lam, 1, 1, out, 1, 1, 1, 1.0, 1.0));
  if (y) CK(launch_spmm(h->s, P.nw, h->ATn_rp, h->ATn_ci, h->Aval, h->ATn_map, y, 1, 1, out, 1, 1, 1, 1.0, 1.0));
  return OPF_OK;
}
}  // namespace condipm


// ============================================================================ internals
namespace condipm {

int eval_impl(opf_handle* h, const double* x, const double* u, const double* lam, const double* y,
              bool derivs) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  h->fr_ready = false;   // a new point: the condensed right-hand side belongs to the old one
  h->fr_have_b = false;
  CK(launch_bus_state(s, P.nb, P.nu, x, u, h->th_w, h->vm_w, h->Vm, h->Va));
  CK(launch_end_eval(s, P.ne, h->end_i, h->end_k, h->end_h, h->gs, h->bs, h->gm, h->bm, h->Vm, h->Va,
                     h->pq, h->dsrc, h->hpq, h->hv, derivs ? 1 : 0));
  CK(launch_bus_sum(s, P.nb, P.ng, P.nu, P.slack, h->bus_end_ptr, h->bus_end, h->pq, h->g_row_P,
                    h->g_row_Q, h->gen_of_bus, h->Pd, h->Qd, u, h->c2, h->c1, derivs ? lam : nullptr, y,
                    h->g, h->hv, h->Pg, h->wP, h->wQ));
  CK(launch_objective(s, P.ng, h->Pg, h->c2, h->c1, h->f));
  if (!derivs) return OPF_OK;
  CK(launch_gather(s, int(P.G.nnz()), h->Ggat_ptr, h->Ggat_idx, h->Ggat_cst, h->dsrc, h->Gval));
  CK(launch_gather(s, int(P.A.nnz()), h->Agat_ptr, h->Agat_idx, h->Agat_cst, h->dsrc, h->Aval));
  CK(launch_gradf(s, P.nw, P.ng, h->pg_of_w, h->slackpos, h->Pg, h->c2, h->c1, h->Aval, h->gradf));
  if (lam && y) {
    CK(launch_end_hess(s, P.ne, h->end_i, h->end_h, h->pq, h->dsrc, h->hpq, h->wP, h->wQ, y, h->hw));
    CK(launch_gather(s, int(P.K.nnz()), h->Wgat_ptr, h->Wgat_idx, h->Wgat_cst, h->hw, h->Wval));
    CK(launch_bilin_fixed(s, int(P.Wslack_pos.size()), h->Wsl_pos, h->Wsl_a, h->Wsl_b, 2.0 * P.c2[0],
                          h->Aval, h->Wval));
  }
  h->have_eval = true;
  h->have_W = lam && y;
  h->sens_ready = false;
  h->psi_valid = false;
  h->have_lu = false;
  h->have_condense = false;
  h->have_factor = false;
  return OPF_OK;
}

// numeric refactorisation, asynchronous (status read by the caller)
int factor_async(opf_handle* h) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  ph_begin(h, OPF_PHASE_REFACTOR);
  CK(cudaMemsetAsync(h->LUval, 0, sizeof(double) * std::max<long long>(1, P.LU.nnz()), s));
  CK(launch_lu_scatter(s, P.G.nnz(), h->Gx_to_LU, h->Gval, h->LUval));
  CK(launch_row_absmax(s, P.nx, h->LU_rp, h->LUval, h->rmax));
  // the row flags restart from zero every refactorisation (one epoch value), so
  // that a captured graph of this sequence can be replayed
  CK(cudaMemsetAsync(h->flags, 0, sizeof(unsigned) * std::max(1, P.nx), s));
  h->epoch = 1;
  CK(launch_lu_refactor(s, P.nx, h->fwd_rows, h->LU_rp, h->LU_ci, h->LU_diag, h->upd_ptr, h->upd_pos,
                        h->LUval, h->inv_diag, h->rmax, h->flags, h->epoch, h->st, h->spin_limit,
                        h->lu_blocks, h->lu_threads, h->lu_maxlen));
  CK(launch_gather_map(s, P.Lo.nnz(), h->Lo_map, h->LUval, h->Lo_val));
  CK(launch_gather_map(s, P.Lo.nnz(), h->Ut_map, h->LUval, h->Ut_val));
  CK(launch_gather_map(s, P.Up.nnz(), h->Up_map, h->LUval, h->Up_val));
  CK(launch_gather_map(s, P.Up.nnz(), h->Lt_map, h->LUval, h->Lt_val));
  CK(launch_fill_stream(s, h->stLo.nslots, h->stLo.slot, h->stLo.src, h->Lo_val, h->inv_diag, 1, h->stLo.bytes_a));
  CK(launch_fill_stream(s, h->stLo.nslots, h->stLo.slot, h->stLo.src, h->Ut_val, h->inv_diag, 0, h->stLo.bytes_b));
  CK(launch_fill_stream(s, h->stUp.nslots, h->stUp.slot, h->stUp.src, h->Up_val, h->inv_diag, 0, h->stUp.bytes_a));
  CK(launch_fill_stream(s, h->stUp.nslots, h->stUp.slot, h->stUp.src, h->Lt_val, h->inv_diag, 1, h->stUp.bytes_b));
  {
    const int nl = int(P.csL.sn_first.size()), nu_ = int(P.csU.sn_first.size());
    const ColDev& L = h->csL;
    const ColDev& U = h->csU;
    const DiagInvJob jobs[4] = {
        {nl, 0, L.sn_first, L.sn_w, h->bkL.d_off, L.int_beg, h->Lo_val, nullptr, h->D_L},
        {nl, 0, L.sn_first, L.sn_w, h->bkL.d_off, L.int_beg, h->Ut_val, h->inv_diag, h->D_Ut},
        {nu_, 1, U.sn_first, U.sn_w, h->bkU.d_off, U.int_beg, h->Up_val, h->inv_diag, h->D_U},
        {nu_, 1, U.sn_first, U.sn_w, h->bkU.d_off, U.int_beg, h->Lt_val, nullptr, h->D_Lt}};
    CK(launch_diag_inv4(s, jobs));
  }
  ph_end(h);
  h->have_lu = true;
  return OPF_OK;
}

// X (perm space, n x ncols, element (i, c) at X[i*xr + c*xc]) <- (LU)^{-1} X or (LU)^{-T} X
int lu_solve_perm(opf_handle* h, int trans, double* X, long long xr, long long xc, int ncols, bool timed,
                  int gu_c0) {
  const Plan& P = h->P;
  // X holds P G_u's columns from gu_c0 on: the level-blocked forward sweep may
  // use the reach lists (its 32-column blocks must line up with G_u's)
  const int rch = (trans == 0 && gu_c0 >= 0 && gu_c0 % 32 == 0 && xc == 1) ? gu_c0 / 32 : -1;
  cudaStream_t s = h->s;
  const double* lov = trans ? h->Ut_val : h->Lo_val;
  const double* upv = trans ? h->Lt_val : h->Up_val;
  const double* dlo = trans ? h->inv_diag : nullptr;
  const double* dup = trans ? nullptr : h->inv_diag;
  const bool cols_ok = ncols >= 32 && xc == 1 && (ncols + 31) / 32 <= h->cs_ncb_max;
  int mode = (ncols >= 32 && xc == 1) ? h->trsm_mode
                                      : (xc == 1 && h->trsm_mode1 >= 64 ? h->trsm_mode1 : 1);
  if (mode < 0) mode = 32;
  if (mode == 65 && ncols == 1 && h->lu1s_ok) {
    if (timed) ph_begin(h, OPF_PHASE_TRSM);
    CK(launch_trsm_lu1s(s, h->lu1s_g, h->l1L, h->Lo_ci, lov, trans ? h->D_Ut : h->D_L, h->l1U, h->Up_ci, upv,
                        trans ? h->D_Lt : h->D_U, X, xr, P.nx, h->lu1s_ymax));
    if (timed) ph_end(h);
    return OPF_OK;
  }
  if (mode == 66 && ncols == 1 && h->cl1_ok[h->cl1_pick]) {
    if (timed) ph_begin(h, OPF_PHASE_TRSM);
    const int c = h->cl1_pick;
    CK(launch_trsm_lu1c(s, h->cl1L[c], h->Lo_ci, lov, trans ? h->D_Ut : h->D_L, h->cl1U[c], h->Up_ci, upv,
                        trans ? h->D_Lt : h->D_U, X, xr, P.nx));
    if (timed) ph_end(h);
    return OPF_OK;
  }
  if (mode == 65 || mode == 66) mode = 64;
  if (mode == 64 && ncols == 1) {
    double* Y = ybuf_reserve(h, (size_t)P.nx * (size_t)xr);
    if (!Y) return OPF_ERR_OOM;
    const int nblk = std::max(1, std::min(h->blk_max, h->blk1_blocks));
    if (timed) ph_begin(h, OPF_PHASE_TRSM);
    CK(launch_trsm_blk1(s, h->bkL, h->Lo_ci, lov, trans ? h->D_Ut : h->D_L, X, Y, xr, nblk, h->cs_bar, h->st,
                        h->spin_limit));
    CK(launch_trsm_blk1(s, h->bkU, h->Up_ci, upv, trans ? h->D_Lt : h->D_U, X, Y, xr, nblk, h->cs_bar, h->st,
                        h->spin_limit));
    if (timed) ph_end(h);
    return OPF_OK;
  }
  if (mode == 96 && ncols >= 32 && xc == 1 && (ncols + 31) / 32 <= h->cs_ncb_max) {
    double* Y = ybuf_reserve(h, (size_t)P.nx * (size_t)xr);
    if (!Y) return OPF_ERR_OOM;
    const int ncb = (ncols + 31) / 32;
    const int kmax = std::max(1, h->df_max / ncb);
    const int ksplit = std::max(1, std::min(kmax, h->df_ksplit > 0 ? h->df_ksplit : 16));
    if (timed) ph_begin(h, OPF_PHASE_TRSM);
    CK(launch_trsm_df(s, h->dfL, h->Lo_ci, lov, trans ? h->D_Ut : h->D_L, X, Y, xr, ncols, ksplit, h->df_cnt, h->df_part,
                      h->st, h->spin_limit));
    if (timed) { ph_end(h); ph_begin(h, OPF_PHASE_TRSM); }
    CK(launch_trsm_df(s, h->dfU, h->Up_ci, upv, trans ? h->D_Lt : h->D_U, X, Y, xr, ncols, ksplit, h->df_cnt, h->df_part,
                      h->st, h->spin_limit));
    if (timed) ph_end(h);
    return OPF_OK;
  }
  if (mode == 96) mode = 64;
  if (mode == 64 && xc == 1 && (ncols + 31) / 32 <= h->cs_ncb_max) {
    double* Y = ybuf_reserve(h, (size_t)P.nx * (size_t)xr);
    if (!Y) return OPF_ERR_OOM;
    const int ncb = (ncols + 31) / 32;
    const int kmax = std::max(1, h->blk_max_minb[h->blk_minb_i] / ncb);
    const int ksplit = std::max(1, std::min(kmax, h->blk_ksplit > 0 ? h->blk_ksplit : 16));
    const int minb = BLK_MINB[h->blk_minb_i];
    if (timed) ph_begin(h, OPF_PHASE_TRSM);
    if (h->blk_cl > 0) {
      // both triangles in one launch of one cluster per column block
      CK(launch_trsm_blkc(s, h->bkL, h->Lo_ci, lov, trans ? h->D_Ut : h->D_L, h->bkU, h->Up_ci, upv,
                          trans ? h->D_Lt : h->D_U, X, Y, xr, ncols, h->blk_cl, rch));
    } else {
      // one launch per triangle (measured faster than both in one launch)
      CK(launch_trsm_blk(s, h->bkL, h->Lo_ci, lov, trans ? h->D_Ut : h->D_L, X, Y, xr, ncols, ksplit, h->cs_bar,
                         h->st, h->spin_limit, minb, rch));
      if (timed) { ph_end(h); ph_begin(h, OPF_PHASE_TRSM); }
      CK(launch_trsm_blk(s, h->bkU, h->Up_ci, upv, trans ? h->D_Lt : h->D_U, X, Y, xr, ncols, ksplit, h->cs_bar,
                         h->st, h->spin_limit, minb));
    }
    if (timed) ph_end(h);
    return OPF_OK;
  }
  if (mode == 64) mode = ncols >= 32 ? 32 : 1;
  if (mode == 32 && cols_ok) {
    const int ncb = (ncols + 31) / 32;
    const int ksplit = std::max(1, std::min(32, h->cs_ksplit_max / ncb));
    if (timed) ph_begin(h, OPF_PHASE_TRSM);
    CK(launch_trsm_cols(s, false, h->csL, h->Lo_ci, lov, dlo, X, xr, ncols, ksplit, h->cs_scratch, h->cs_bar,
                        h->st, h->spin_limit));
    if (timed) { ph_end(h); ph_begin(h, OPF_PHASE_TRSM); }
    CK(launch_trsm_cols(s, true, h->csU, h->Up_ci, upv, dup, X, xr, ncols, ksplit, h->cs_scratch, h->cs_bar,
                        h->st, h->spin_limit));
    if (timed) ph_end(h);
    return OPF_OK;
  }
  int cb = (mode == 32) ? 1 : std::min(mode, h->sn_cb);
  if (h->sn_cb == 0) cb = 0;
  const opf_handle::StBuf& Lb = h->stLo;
  const opf_handle::StBuf& Ub = h->stUp;
  const StDev lo{Lb.nchunks, h->st_cap, Lb.chunk_off, Lb.chunk_bytes, Lb.chunk_big_f, Lb.chunk_big_w,
                 trans ? Lb.bytes_b : Lb.bytes_a, Lb.int_beg, lov, dlo};
  const StDev up{Ub.nchunks, h->st_cap, Ub.chunk_off, Ub.chunk_bytes, Ub.chunk_big_f, Ub.chunk_big_w,
                 trans ? Ub.bytes_b : Ub.bytes_a, Ub.int_beg, upv, dup};
  if (timed) ph_begin(h, OPF_PHASE_TRSM);
  if (cb > 0) CK(launch_trsm_st(s, cb, false, lo, P.nx, X, xr, xc, ncols, h->st, h->spin_limit));
  else CK(launch_trsm(s, 1, P.fwd.nlev, h->fwd_ptr, h->fwd_rows, h->Lo_rp, h->Lo_ci, lov, dlo, X, xr, xc, ncols));
  if (timed) { ph_end(h); ph_begin(h, OPF_PHASE_TRSM); }
  if (cb > 0) CK(launch_trsm_st(s, cb, true, up, P.nx, X, xr, xc, ncols, h->st, h->spin_limit));
  else CK(launch_trsm(s, 1, P.bwd.nlev, h->bwd_ptr, h->bwd_rows, h->Up_rp, h->Up_ci, upv, dup, X, xr, xc, ncols));
  if (timed) ph_end(h);
  return OPF_OK;
}

// S_x <- -P G_u, the rest of its nx x ld block zero (the forward sweep's
// reach lists rely on those exact zeros)
static int scatter_gu(opf_handle* h, double* Sx, long long ld) {
  const Plan& P = h->P;
  CK(cudaMemsetAsync(Sx, 0, sizeof(double) * (size_t)P.nx * ld, h->s));
  CK(launch_scatter_rows(h->s, P.nx, h->PGu_rp, h->PGu_ci, h->PGu_map, h->Gval, -1.0, Sx, ld, 1));
  return OPF_OK;
}

// Pick the fastest multi-RHS solve kernel for this network on the device at hand:
// each candidate solves the real right-hand side (in the H buffer, which the
// condensation overwrites afterwards) twice, the second run timed with events.
int autotune_trsm(opf_handle* h, const double* Sx, long long ld) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx;
  double* trial = h->H + (size_t)nu * ld;
  const int cands[6] = {32, 1, 2, 4, 64, 96};
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  int pick = 1;
  auto time_solve = [&](int ncols, float* out) -> int {
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaMemcpyAsync(trial, Sx, sizeof(double) * (size_t)nx * ld, cudaMemcpyDeviceToDevice, h->s));
      CK(cudaEventRecord(a, h->s));
      TRY(lu_solve_perm(h, 0, trial, ld, 1, ncols, false, 0));
      CK(cudaEventRecord(b, h->s));
      CK(cudaEventSynchronize(b));
      CK(cudaEventElapsedTime(&ms, a, b));
    }
    *out = ms;
    return OPF_OK;
  };
  int best_ks = 0;
  for (int k = 0; k < 6; ++k) {
    const int m = cands[k];
    const bool lanes = m == 32 || m == 64 || m == 96;
    if (!lanes && (h->sn_cb == 0 || m > h->sn_cb)) continue;
    if (lanes && (nu < 32 || (nu + 31) / 32 > h->cs_ncb_max)) continue;
    h->trsm_mode = m;
    if (m == 96) {
      // the dataflow kernel picks its CTAs per column block
      const int kss[6] = {16, 24, 32, 48, 64, 96};
      float bk = 1e30f;
      int bks = 16;
      for (int ks : kss) {
        if (ks > 16 && ks > h->df_max / ((nu + 31) / 32)) continue;
        h->df_ksplit = ks;
        float ms = 0.f;
        TRY(time_solve(nu, &ms));
        if (ms < bk) { bk = ms; bks = ks; }
      }
      h->df_ksplit = bks;
      h->tune_ms[0][5] = bk;
      if (bk < best) { best = bk; pick = m; }
      continue;
    }
    if (m == 64) {
      // the level-blocked kernel also picks its CTAs per column block: a group
      // meeting at a barrier through global memory, or a thread-block cluster
      const int kss[6] = {4, 8, 12, 16, 24, 32};
      const int cls[4] = {2, 4, 8, 16};
      float bk = 1e30f;
      int best_cl = 0;
      h->blk_cl = 0;
      int best_mb = 0;
      for (int mb = 0; mb < 3; ++mb) {
        h->blk_minb_i = mb;
        for (int ks : kss) {
          if (ks > 16 && ks > h->blk_max_minb[mb] / ((nu + 31) / 32)) continue;
          h->blk_ksplit = ks;
          float ms = 0.f;
          TRY(time_solve(nu, &ms));
          if (ms < bk) { bk = ms; best_ks = ks; best_cl = 0; best_mb = mb; }
        }
      }
      h->blk_minb_i = best_mb;
      for (int cl : cls) {
        if (trsm_blkc_clusters(cl) < 1) continue;
        h->blk_cl = cl;
        float ms = 0.f;
        TRY(time_solve(nu, &ms));
        if (ms < bk) { bk = ms; best_cl = cl; }
      }
      h->blk_ksplit = best_ks;
      h->blk_cl = best_cl;
      h->tune_ms[0][k] = bk;
      if (bk < best) { best = bk; pick = m; }
      continue;
    }
    float ms = 0.f;
    TRY(time_solve(nu, &ms));
    h->tune_ms[0][k] = ms;
    if (ms < best) { best = ms; pick = m; }
  }
  // one right-hand side (the step recovery): staged (one CTA), level-blocked
  // over 8 .. 64 CTAs, or level-blocked in one CTA with the vector in shared
  // memory (4 or 8 lanes per row)
  if (h->opt.rhs1_kernel == 0) {
    float b1 = 1e30f;
    int p1 = 1, pb = h->blk1_blocks, pg = h->lu1s_g, pc = h->cl1_pick;
    const int c1[10] = {1, 64, 64, 64, 64, 65, 65, 66, 66, 66};
    const int nb1[10] = {0, 8, 16, 32, 64, 0, 0, 0, 0, 0};
    const int g1[10] = {0, 0, 0, 0, 0, 8, 4, 0, 0, 0};
    const int cl1[10] = {-1, -1, -1, -1, -1, -1, -1, 0, 1, 2};
    for (int k = 0; k < 10; ++k) {
      if (c1[k] == 65 && !h->lu1s_ok) continue;
      if (c1[k] == 66 && !h->cl1_ok[cl1[k]]) continue;
      h->trsm_mode1 = c1[k];
      if (nb1[k]) h->blk1_blocks = nb1[k];
      if (g1[k]) h->lu1s_g = g1[k];
      if (cl1[k] >= 0) h->cl1_pick = cl1[k];
      float ms = 0.f;
      TRY(time_solve(1, &ms));
      h->tune_ms[1][k] = ms;
      if (ms < b1) {
        b1 = ms;
        p1 = c1[k];
        pb = nb1[k] ? nb1[k] : pb;
        pg = g1[k] ? g1[k] : pg;
        pc = cl1[k] >= 0 ? cl1[k] : pc;
      }
    }
    h->trsm_mode1 = p1;
    h->blk1_blocks = pb;
    h->lu1s_g = pg;
    h->cl1_pick = pc;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  h->trsm_mode = pick;
  return OPF_OK;
}

// A7 on the current K and Z = [I; S_x]: H = K Z, then Kred by the handle's route
// (the x rows of H end up holding Psi = G_x^{-T} H_x on the adjoint route)
static int reduce_route(opf_handle* h, int route, int nc) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nx = P.nx;
  const long long ld = h->ldp;
  double* Sx = h->Zt + (size_t)nu * ld;
  double* Hx = h->H + (size_t)nu * ld;
  if (route == OPF_ROUTE_EXPLICIT) {
    const int z = dense_tn_slices(nu, nx);
    double* scratch = nullptr;
    if (z > 1) {
      scratch = workspace(h, (size_t)z * nu * nu);
      if (!scratch) return OPF_ERR_OOM;
    }
    ph_begin(h, OPF_PHASE_KRED);
    CK(launch_dense_tn(s, nu, nx, Sx, Hx, h->H, ld, h->F, scratch, z));
    CK(launch_symmetrize(s, nu, h->F, nu, 1, h->Kred));
    ph_end(h);
  } else {
    // Psi = G_x^{-T} H_x ; Kred = H_u - G_u^T Psi  (nc = nu + 1: the condensed
    // right-hand side's column rides along: phi = G_x^{-T} e_x, r_hat = e_u - G_u^T phi)
    TRY(lu_solve_perm(h, 1, Hx, ld, 1, nc, true));
    ph_begin(h, OPF_PHASE_KRED);
    CK(launch_spmm(s, nu, h->GuT_rp, h->GuT_ci, h->Gval, h->GuT_map, Hx, ld, 1, h->H, ld, 1, nc, -1.0, 1.0));
    CK(launch_symmetrize(s, nu, h->H, ld, 1, h->Kred));
    ph_end(h);
  }
  return OPF_OK;
}

// A7 on the current K and Z = [I; S_x]: H = K Z, then Kred by the handle's route
// (the x rows of H end up holding Psi = G_x^{-T} H_x on the adjoint route).  With
// OPF_ROUTE_AUTO the first call times both routes on this network (the explicit
// one first: it leaves H intact) and keeps the faster; the adjoint route's
// result stands for that call.
static int reduce_async(opf_handle* h, int nc = 0, const double* bt = nullptr) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nw = P.nw;
  const long long ld = h->ldp;
  if (nc <= 0) nc = nu;
  ph_begin(h, OPF_PHASE_SPMM);
  CK(launch_spmm(s, nw, h->K_rp, h->K_ci, h->Kval, nullptr, h->Zt, ld, 1, h->H, ld, 1, nc, 1.0, 0.0));
  // the right-hand side's column: e = b_t - K [0; q]
  if (bt) CK(launch_column_axpby(s, nw, -1.0, h->H + nu, ld, 1.0, bt, 1, h->H + nu, ld));
  ph_end(h);
  if (h->route >= 0) return reduce_route(h, h->route, nc);
  cudaEvent_t ev[3];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], s));
  TRY(reduce_route(h, OPF_ROUTE_EXPLICIT, nc));
  CK(cudaEventRecord(ev[1], s));
  TRY(reduce_route(h, OPF_ROUTE_ADJOINT, nc));
  CK(cudaEventRecord(ev[2], s));
  CK(cudaEventSynchronize(ev[2]));
  CK(cudaEventElapsedTime(&h->route_ms[OPF_ROUTE_EXPLICIT], ev[0], ev[1]));
  CK(cudaEventElapsedTime(&h->route_ms[OPF_ROUTE_ADJOINT], ev[1], ev[2]));
  for (auto& e : ev) cudaEventDestroy(e);
  h->route = h->route_ms[OPF_ROUTE_EXPLICIT] < h->route_ms[OPF_ROUTE_ADJOINT] ? OPF_ROUTE_EXPLICIT : OPF_ROUTE_ADJOINT;
  h->psi_last_adjoint = true;
  return OPF_OK;
}

// the right-hand side of the step into the handle's KB copy, and
// b_t = b_w + A^T (Sigma_s b_y - b_s) (needs h->sig_s)
int fr_reserve(opf_handle* h) {
  if (!h->fr_kb) {
    TRY(alloc(h, &h->fr_kb, kkt_rows(h->P)));
    TRY(alloc(h, &h->fr_bt, (size_t)h->P.nw + h->P.m));
  }
  return OPF_OK;
}

static int fr_prepare(opf_handle* h, const double* rhs) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nw = P.nw, m = P.m, nx = P.nx;
  const size_t N = kkt_rows(P);
  TRY(fr_reserve(h));
  const KB b = kb_at(P, h->fr_kb, 1);
  CK(launch_permute_rows(s, nw, 1, h->c2w, rhs, int(N), 1, b.w, 1, 0, -1.0, 0));
  CK(launch_permute_rows(s, m, 1, nullptr, rhs + nw, int(N), 1, b.s, 1, 0, -1.0, 0));
  CK(launch_permute_rows(s, nx, 1, h->perm, rhs + nw + m, int(N), 1, b.l, 1, 0, -1.0, 0));
  CK(launch_permute_rows(s, m, 1, nullptr, rhs + nw + m + nx, int(N), 1, b.y, 1, 0, -1.0, 0));
  double* U = h->fr_bt + nw;   // Sigma_s b_y - b_s
  CK(launch_scale_rows(s, m, 1, h->sig_s, b.y, U, -1.0, b.s));
  CK(cudaMemcpyAsync(h->fr_bt, b.w, sizeof(double) * nw, cudaMemcpyDeviceToDevice, s));
  CK(launch_spmm(s, nw, h->AT_rp, h->AT_ci, h->Aval, h->AT_map, U, 1, 1, h->fr_bt, 1, 1, 1, 1.0, 1.0));
  h->fr_have_b = true;
  return OPF_OK;
}

// columns per pass of the adjoint-route condensation
static int chunk_width(const opf_handle* h) {
  const int N = h->opt.rhs_width > 0 ? h->opt.rhs_width : h->rhs_width;
  return N > 0 ? N : h->P.nu;
}

// A6-A7 of the adjoint route in column chunks of N (Fig. 2b's batch width):
// per chunk the S_x solve, H = K Z, Psi = G_x^{-T} H_x and H_u - G_u^T Psi;
// the condensed right-hand side's column rides with the last chunk.  S_x holds
// -P G_u (and b_l) on entry; Kred is symmetrised at the end.
static int condense_chunked(opf_handle* h, int N, bool fused) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nw = P.nw;
  const long long ld = h->ldp;
  double* Sx = h->Zt + (size_t)nu * ld;
  double* Hx = h->H + (size_t)nu * ld;
  for (int c0 = 0; c0 < nu; c0 += N) {
    const bool last = c0 + N >= nu;
    const int ncc = std::min(N, nu - c0) + (fused && last ? 1 : 0);
    TRY(lu_solve_perm(h, 0, Sx + c0, ld, 1, ncc, true, c0));
    ph_begin(h, OPF_PHASE_SPMM);
    CK(launch_spmm(s, nw, h->K_rp, h->K_ci, h->Kval, nullptr, h->Zt + c0, ld, 1, h->H + c0, ld, 1, ncc, 1.0, 0.0));
    if (fused && last) CK(launch_column_axpby(s, nw, -1.0, h->H + nu, ld, 1.0, h->fr_bt, 1, h->H + nu, ld));
    ph_end(h);
    TRY(lu_solve_perm(h, 1, Hx + c0, ld, 1, ncc, true));
    ph_begin(h, OPF_PHASE_KRED);
    CK(launch_spmm(s, nu, h->GuT_rp, h->GuT_ci, h->Gval, h->GuT_map, Hx + c0, ld, 1, h->H + c0, ld, 1, ncc, -1.0,
                   1.0));
    ph_end(h);
  }
  ph_begin(h, OPF_PHASE_KRED);
  CK(launch_symmetrize(s, nu, h->H, ld, 1, h->Kred));
  ph_end(h);
  return OPF_OK;
}

// On the first adjoint-route condensation: the products at N = nu, 512, 256,
// 128 (those below nu), each from the same S_x right-hand side (kept in Zt's
// spare rows: re-scattered before every candidate), timed with events; the
// fastest is kept.  The last candidate's results stand.
static int tune_width(opf_handle* h, bool fused) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nx = P.nx;
  const long long ld = h->ldp;
  double* Sx = h->Zt + (size_t)nu * ld;
  const int cand[4] = {nu, 512, 256, 128};
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  int pick = nu, rc = OPF_OK, ran = 0;
  for (int i = 0; i < 4 && rc == OPF_OK; ++i) {
    h->width_ms[i] = 0.f;
    if (i > 0 && cand[i] >= nu) continue;
    if (ran > 0) {
      // the right-hand side again (the previous candidate solved S_x in place)
      rc = scatter_gu(h, Sx, ld);
      if (rc == OPF_OK && fused &&
          launch_column_axpby(s, nx, 1.0, kb_at(P, h->fr_kb, 1).l, 1, 0.0, nullptr, 0, Sx + nu, ld) != cudaSuccess)
        rc = OPF_ERR_CUDA;
    }
    if (rc == OPF_OK && cudaEventRecord(a, s) != cudaSuccess) rc = OPF_ERR_CUDA;
    if (rc == OPF_OK) {
      if (cand[i] >= nu) {
        rc = lu_solve_perm(h, 0, Sx, ld, 1, fused ? nu + 1 : nu, true, 0);
        if (rc == OPF_OK) rc = reduce_async(h, fused ? nu + 1 : nu, fused ? h->fr_bt : nullptr);
      } else {
        rc = condense_chunked(h, cand[i], fused);
      }
    }
    if (rc == OPF_OK && cudaEventRecord(b, s) != cudaSuccess) rc = OPF_ERR_CUDA;
    if (rc == OPF_OK && cudaEventSynchronize(b) != cudaSuccess) rc = OPF_ERR_CUDA;
    float ms = 0.f;
    if (rc == OPF_OK) cudaEventElapsedTime(&ms, a, b);
    h->width_ms[i] = ms;
    ++ran;
    if (rc == OPF_OK && ms < best) { best = ms; pick = cand[i]; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  TRY(rc);
  h->rhs_width = pick;
  return OPF_OK;
}

int condense_async(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s,
                   const double* rhs) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nx = P.nx, nw = P.nw;
  // the right-hand side in the same pass: needs a spare column (ldp > nu) and
  // the adjoint route's Psi
  const bool fused = rhs != nullptr && h->ldp > nu && h->opt.route != OPF_ROUTE_EXPLICIT;
  h->fr_ready = false;
  h->fr_have_b = false;
  h->psi_valid = false;
  h->finv_valid = false;   // the explicit route uses the factor's buffer as scratch
  h->delta_c = 0.0;
  if (!h->have_lu) TRY(factor_async(h));
  CK(cudaMemcpyAsync(h->sig_s, sig_s, sizeof(double) * std::max(1, P.m), cudaMemcpyDeviceToDevice, s));
  // A4: K = W + A^T Sigma_s A + diag(Sigma)
  ph_begin(h, OPF_PHASE_ASSEMBLE);
  CK(launch_assemble_K(s, P.K.nnz(), h->Wval, h->KAA_ptr, h->KAA_r, h->KAA_a, h->KAA_b, h->sig_s, h->Aval,
                       h->Kval));
  CK(launch_add_diag(s, nw, nu, h->K_diag, h->perm, sig_u, sig_x, h->Kval, h->sig_c));
  if (rhs) TRY(fr_prepare(h, rhs));
  ph_end(h);
  // A6: Z = [I; S_x],  S_x = -(P G_x P^T)^{-1} P G_u   (perm rows); Z and H are
  // row-major with leading dimension ldp (nu rounded up to 32): lanes of a warp
  // hold consecutive right-hand-side columns
  const long long ld = h->ldp;
  double* Sx = h->Zt + (size_t)nu * ld;
  TRY(scatter_gu(h, Sx, ld));
  if (h->trsm_mode < 0) TRY(autotune_trsm(h, Sx, ld));
  // the right-hand side's column of the solve: b_l (then q = G_x^{-1} b_l; the
  // identity rows of Zt are zero in this column, so H gets K [0; q])
  const int nc = fused ? nu + 1 : nu;
  if (fused) CK(launch_column_axpby(s, nx, 1.0, kb_at(P, h->fr_kb, 1).l, 1, 0.0, nullptr, 0, Sx + nu, ld));
  h->psi_last_adjoint = false;
  if (h->route == OPF_ROUTE_ADJOINT && h->rhs_width == 0 && h->opt.rhs_width == 0 && !h->profiling) {
    TRY(tune_width(h, fused));
  } else if (h->route == OPF_ROUTE_ADJOINT && chunk_width(h) < nu) {
    TRY(condense_chunked(h, chunk_width(h), fused));
  } else {
    TRY(lu_solve_perm(h, 0, Sx, ld, 1, nc, true, 0));
    TRY(reduce_async(h, nc, fused ? h->fr_bt : nullptr));
  }
  h->have_condense = true;
  h->have_factor = false;
  h->sens_ready = false;
  h->psi_valid = h->route != OPF_ROUTE_EXPLICIT || h->psi_last_adjoint;
  h->fr_ready = fused && h->psi_valid;
  return OPF_OK;
}

// Fold the dual regularisation delta_c of the inequality rows into K and Kred
// of the last condensation: K = W + diag(Sigma_w) + A^T Sigma_t A with
// Sigma_t = (Sigma_s^{-1} + delta_c)^{-1}, then H and Kred again.  The
// refactorisation and S_x do not depend on Sigma and are kept.
int recondense_dc(opf_handle* h, double delta_c) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  h->psi_valid = false;
  h->fr_ready = false;   // K changes: the condensed right-hand side is recomputed by the plain path
  h->finv_valid = false;
  h->have_factor = false;
  const double* sig = h->sig_s;
  if (delta_c > 0.0) {
    CK(launch_sigma_dc(s, P.m, delta_c, h->sig_s, h->sig_se, h->ps_sc));
    sig = h->sig_se;
  }
  ph_begin(h, OPF_PHASE_ASSEMBLE);
  CK(launch_assemble_K(s, P.K.nnz(), h->Wval, h->KAA_ptr, h->KAA_r, h->KAA_a, h->KAA_b, sig, h->Aval, h->Kval));
  CK(launch_add_diag_c(s, P.nw, h->K_diag, h->sig_c, h->Kval));
  ph_end(h);
  h->psi_last_adjoint = false;
  TRY(reduce_async(h));
  h->delta_c = delta_c;
  h->psi_valid = h->route != OPF_ROUTE_EXPLICIT || h->psi_last_adjoint;
  return OPF_OK;
}

// Time the Cholesky with a few grid sizes (fewer CTAs: cheaper grid barriers;
// more: more of the trailing update in flight) and keep the fastest.  The
// factor does not depend on the grid size.
int tune_chol_blocks(opf_handle* h, double delta_w) {
  const Plan& P = h->P;
  const int cap = h->chol_blocks;
  // candidates {form, grid, panel CTAs}, grids in units of the device's SM
  // count: the barrier form at a quarter, a half, one and two CTAs per SM; the
  // dataflow form at a half, one and two CTAs per SM with a small panel group (a
  // quarter of the first step's row groups), and at one and two CTAs per SM with
  // a panel group of one row group per CTA
  const int sm = device_sms();
  const int rows0 = (std::max(0, P.nu - 32) + 7) / 8;   // panel row groups of the first step
  const int df_cap = chol_df_max_blocks();
  const int want = h->opt.chol_form;   // 0 both, 1 barrier form only, 2 dataflow form only
  struct Cand { int form, nb, np; };
  const int q = std::max(1, sm / 4), hf = std::max(1, sm / 2), one = sm, two = 2 * sm, four = 4 * sm;
  const Cand cand[OPF_CHOL_CANDIDATES] = {
      {0, q, 0}, {0, hf, 0}, {0, one, 0}, {0, two, 0},
      {1, hf, std::max(1, std::min(hf / 3, std::max(8, rows0 / 4)))},
      {1, one, std::max(1, std::min(one / 3, std::max(8, rows0 / 4)))},
      {1, two, std::max(1, std::min(two / 3, std::max(8, rows0 / 4)))},
      {1, one, std::max(1, std::min(one / 2, std::max(8, rows0)))},
      {1, two, std::max(1, std::min(two / 2, std::max(8, rows0)))},
      {1, four, std::max(1, std::min(four / 3, std::max(8, rows0 / 4)))},
      {1, four, std::max(1, std::min(four / 2, std::max(8, rows0)))}};
  // time only from a clean status word, and keep the timings only if every
  // candidate factored the whole matrix: a run that stops early on a
  // non-positive pivot (the dataflow form leaves as soon as one is flagged)
  // would look fast, so an indefinite matrix leaves the handle untuned and the
  // next factorisation tries again
  int st0[ST_WORDS];
  CK(cudaMemcpyAsync(st0, h->st, sizeof(st0), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (st0[ST_CODE] != 0 || st0[ST_TIMEOUT] != 0) return OPF_OK;   // untuned; tried again next time
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best = 1e30f;
  int pick = cap, pick_df = 0, pick_np = 0;
  bool complete = true;
  float ms_c[OPF_CHOL_CANDIDATES] = {};
  for (int c = 0; c < OPF_CHOL_CANDIDATES && complete; ++c) {
    const int form = cand[c].form, nb = cand[c].nb, np = cand[c].np;
    if (want != 0 && want != form + 1) continue;
    if (form == 0 && nb > cap) continue;
    if (form == 1 && (nb > df_cap || nb - np < 1)) continue;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && complete; ++rep) {
      CK(cudaMemsetAsync(h->st, 0, sizeof(int) * ST_WORDS, h->s));
      CK(cudaEventRecord(a, h->s));
      CK(launch_chol_prepare(h->s, P.nu, h->Kred, delta_w, h->F));
      if (form == 0) {
        CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->s));
        CK(launch_chol(h->s, P.nu, h->F, h->Fdinv, h->st, h->bar, h->spin_limit, nb));
      } else {
        CK(launch_chol_df(h->s, P.nu, h->F, h->Fdinv, h->st, h->chol_cnt, h->spin_limit, nb, np));
      }
      CK(cudaEventRecord(b, h->s));
      CK(cudaEventSynchronize(b));
      CK(cudaEventElapsedTime(&ms, a, b));
      int stc[ST_WORDS];
      CK(cudaMemcpyAsync(stc, h->st, sizeof(stc), cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
      if (stc[ST_CODE] != 0 || stc[ST_TIMEOUT] != 0) complete = false;
    }
    ms_c[c] = ms;
    if (ms < best) { best = ms; pick = nb; pick_df = form; pick_np = np; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CK(cudaMemsetAsync(h->st, 0, sizeof(int) * ST_WORDS, h->s));
  CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->s));
  if (!complete) return OPF_OK;   // untuned: defaults for this factorisation
  for (int c = 0; c < OPF_CHOL_CANDIDATES; ++c) h->chol_ms[c] = ms_c[c];
  h->chol_blocks = pick;
  h->chol_df = pick_df;
  h->chol_np = pick_np;
  h->chol_tuned = true;
  return OPF_OK;
}

int factor_kred_async(opf_handle* h, double delta_w) {
  const Plan& P = h->P;
  if (!h->chol_tuned) TRY(tune_chol_blocks(h, delta_w));
  ph_begin(h, OPF_PHASE_CHOL);
  CK(launch_chol_prepare(h->s, P.nu, h->Kred, delta_w, h->F));
  CK(cudaMemsetAsync(h->bar, 0, sizeof(unsigned) * 4, h->s));
  if (h->chol_df) {
    CK(launch_chol_df(h->s, P.nu, h->F, h->Fdinv, h->st, h->chol_cnt, h->spin_limit, h->chol_blocks, h->chol_np));
  } else {
    CK(launch_chol(h->s, P.nu, h->F, h->Fdinv, h->st, h->bar, h->spin_limit, h->chol_blocks));
  }
  ph_end(h);
  h->delta_w = delta_w;
  h->sens_ready = false;
  h->finv_valid = false;
  return OPF_OK;
}

// X (row-major nu x k) <- (L L^T)^{-1} X with the current factor: for a few
// columns one cluster per column (tile inverses computed on first use after
// each factorisation), else one CTA per column
int chol_solve_async(opf_handle* h, double* X, int k) {
  const int nu = h->P.nu;
  if (k >= 1 && k <= 8 && h->chol_solve_cl > 0) {
    if (!h->finv_valid) {
      CK(launch_tile_inv(h->s, nu, h->F, h->Fdinv, h->Finv));
      h->finv_valid = true;
    }
    if (k == 1 && !h->cs_tuned && !h->profiling && nu > 8 * 32) {
      // the cluster size: a tile step costs one cluster barrier, a larger
      // cluster shares the update out wider; time 4, 8, 16 CTAs on this
      // right-hand side (restored before each) and keep the fastest
      cudaEvent_t a = nullptr, b = nullptr;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      CK(cudaMemcpyAsync(h->cs_tmp, X, sizeof(double) * nu, cudaMemcpyDeviceToDevice, h->s));
      const int cand[3] = {4, 8, 16};
      float best = 1e30f;
      int pick = h->chol_solve_cl;
      for (int c = 0; c < 3; ++c) {
        CK(cudaMemcpyAsync(X, h->cs_tmp, sizeof(double) * nu, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaEventRecord(a, h->s));
        CK(launch_chol_solve_cl(h->s, nu, h->F, h->Finv, X, 1, cand[c]));
        CK(cudaEventRecord(b, h->s));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        h->cs_ms[c] = ms;
        if (ms < best) { best = ms; pick = cand[c]; }
      }
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      CK(cudaMemcpyAsync(X, h->cs_tmp, sizeof(double) * nu, cudaMemcpyDeviceToDevice, h->s));
      h->chol_solve_cl = pick;
      h->cs_tuned = true;
    }
    CK(launch_chol_solve_cl(h->s, nu, h->F, h->Finv, X, k, h->chol_solve_cl));
    return OPF_OK;
  }
  CK(launch_chol_solve(h->s, nu, h->F, h->Fdinv, X, k));
  return OPF_OK;
}

}  // namespace condipm

// ============================================================================ C ABI
extern "C" {

const char* opf_strerror(int code) {
  switch (code) {
    case OPF_OK: return "ok";
    case OPF_ERR_INVALID_ARG: return "invalid argument or call order";
    case OPF_ERR_CUDA: return "CUDA runtime error";
    case OPF_ERR_NOT_PD: return "condensed matrix not positive definite";
    case OPF_ERR_SINGULAR: return "G_x refactorisation met a tiny pivot";
    case OPF_ERR_PF_FAILED: return "power flow did not converge";
    case OPF_ERR_TIMEOUT: return "a bounded device wait expired";
    case OPF_ERR_OOM: return "device allocation failed";
    case OPF_ERR_NO_CONVERGENCE: return "interior-point iteration cap reached";
    case OPF_ERR_INFEASIBLE: return "feasibility restoration failed (locally infeasible)";
    default: return "unknown status";
  }
}

int opf_create(const opf_network* net, const opf_options* opt, opf_handle** out) {
  if (!net || !out) return OPF_ERR_INVALID_ARG;
  *out = nullptr;
  opf_handle* h = new (std::nothrow) opf_handle();
  if (!h) return OPF_ERR_OOM;
  if (opt) h->opt = *opt;
  if ((h->opt.route != OPF_ROUTE_ADJOINT && h->opt.route != OPF_ROUTE_EXPLICIT && h->opt.route != OPF_ROUTE_AUTO) ||
      h->opt.rhs_width < 0 || h->opt.dense_forward < 0 || h->opt.dense_forward > 1) {
    delete h;
    return OPF_ERR_INVALID_ARG;
  }
  h->route = h->opt.route == OPF_ROUTE_AUTO ? -1 : h->opt.route;
  h->spin_limit = h->opt.spin_limit > 0 ? h->opt.spin_limit : (1LL << 26);
  std::string err = build_plan(h->P, net->nb, net->nl, net->ng, net->slack, net->Pd, net->Qd, net->Vmin,
                               net->Vmax, net->lf, net->lt, net->r, net->x, net->b, net->rate, net->gbus,
                               net->Pmin, net->Pmax, net->Qmin, net->Qmax, net->c2, net->c1);
  if (!err.empty()) {
    delete h;
    return OPF_ERR_INVALID_ARG;
  }
  if (h->opt.chol_form < 0 || h->opt.chol_form > 2) {
    delete h;
    return OPF_ERR_INVALID_ARG;
  }
  int cb = h->opt.rhs_block;
  if (cb != 0 && cb != 1 && cb != 2 && cb != 4 && cb != 32 && cb != 64 && cb != 96 && cb != 128) {
    delete h;
    return OPF_ERR_INVALID_ARG;
  }
  h->trsm_mode = cb == 128 ? 64 : (cb ? cb : -1);
  if (cb == 128) h->blk_cl = 8;
  const int k1 = h->opt.rhs1_kernel;
  if (k1 != 0 && k1 != 1 && k1 != 64 && k1 != 65 && k1 != 66) {
    delete h;
    return OPF_ERR_INVALID_ARG;
  }
  if (k1) h->trsm_mode1 = k1;
  h->cb = pick_cb(h->P.nu);
  int rc = upload_all(h);
  if (rc != OPF_OK) {
    opf_destroy(h);
    return rc;
  }
  *out = h;
  return OPF_OK;
}

int opf_rhs_width(const opf_handle* h, int* width, float* ms) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (width) *width = h->opt.rhs_width > 0 ? std::min(h->opt.rhs_width, h->P.nu) : std::min(h->rhs_width, h->P.nu);
  if (ms) for (int i = 0; i < 4; ++i) ms[i] = h->width_ms[i];
  return OPF_OK;
}

int opf_route_choice(const opf_handle* h, int* route, float* ms) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (route) *route = h->route;
  if (ms) { ms[0] = h->route_ms[0]; ms[1] = h->route_ms[1]; }
  return OPF_OK;
}

int opf_chol_choice(const opf_handle* h, int* form, int* nblocks, float* ms) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (form) *form = h->chol_tuned ? 1 + h->chol_df : 0;
  if (nblocks) *nblocks = h->chol_blocks;
  if (ms) for (int c = 0; c < OPF_CHOL_CANDIDATES; ++c) ms[c] = h->chol_ms[c];
  return OPF_OK;
}

int opf_forward_reach(const opf_handle* h, int* nblocks, double* work) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (nblocks) *nblocks = h->bkL.rch_ptr ? h->bkL.rch_nblk : 0;
  if (work) { work[0] = h->rch_work[0]; work[1] = h->rch_work[1]; }
  return OPF_OK;
}

int opf_chol_solve_choice(const opf_handle* h, int* cluster, float* ms) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (cluster) *cluster = h->chol_solve_cl;
  if (ms) for (int c = 0; c < 3; ++c) ms[c] = h->cs_ms[c];
  return OPF_OK;
}

void opf_destroy(opf_handle* h) {
  if (!h) return;
  for (auto& r : h->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : h->evpool) cudaEventDestroy(e);
  if (h->cf_exec) cudaGraphExecDestroy(h->cf_exec);
  condipm::fs_release(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->ws) cudaFree(h->ws);
  if (h->ybuf) cudaFree(h->ybuf);
  delete h;
}

int opf_last_cuda_error(char* name, int len) {
  const int e = condipm::last_cuda_error();
  if (name && len > 0) {
    std::snprintf(name, size_t(len), "%s", cudaGetErrorName(cudaError_t(e)));
  }
  return e;
}

int opf_sizes(const opf_handle* h, int* nx, int* nu, int* m) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (nx) *nx = h->P.nx;
  if (nu) *nu = h->P.nu;
  if (m) *m = h->P.m;
  return OPF_OK;
}

int opf_stats(const opf_handle* h, long long* nnz_lu, int* levels_fwd, int* levels_bwd, long long* nnz_k,
              long long* lu_flops) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (nnz_lu) *nnz_lu = h->P.LU.nnz();
  if (levels_fwd) *levels_fwd = h->P.fwd.nlev;
  if (levels_bwd) *levels_bwd = h->P.bwd.nlev;
  if (nnz_k) *nnz_k = h->P.K.nnz();
  if (lu_flops) *lu_flops = h->P.lu_flops;
  return OPF_OK;
}

int opf_trsm_choice(const opf_handle* h, int* kernel, float* ms, int* kernel1) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (kernel) *kernel = (h->trsm_mode == 64 && h->blk_cl > 0) ? 128 : h->trsm_mode;
  if (ms)
    for (int k = 0; k < 6; ++k) ms[k] = h->tune_ms[0][k];
  if (kernel1) *kernel1 = h->trsm_mode1;
  return OPF_OK;
}

int opf_set_stream(opf_handle* h, void* stream) {
  if (!h) return OPF_ERR_INVALID_ARG;
  h->s = (cudaStream_t)stream;
  return OPF_OK;
}

int opf_eval_derivatives(opf_handle* h, const double* x, const double* u, const double* lam, const double* y) {
  if (!h || !x || !u || ((lam == nullptr) != (y == nullptr))) return OPF_ERR_INVALID_ARG;
  TRY(eval_impl(h, x, u, lam, y, true));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_eval_functions(opf_handle* h, const double* x, const double* u) {
  if (!h || !x || !u) return OPF_ERR_INVALID_ARG;
  TRY(eval_impl(h, x, u, nullptr, nullptr, false));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_get_vector(opf_handle* h, int which, double* dst) {
  if (!h || !dst) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  const double* src = nullptr;
  size_t n = 0;
  switch (which) {
    case OPF_VEC_F: src = h->f; n = 1; break;
    case OPF_VEC_G: src = h->g; n = P.nx; break;
    case OPF_VEC_H: src = h->hv; n = P.m; break;
    case OPF_VEC_GRADF: src = h->gradf; n = P.nw; break;
    default: return OPF_ERR_INVALID_ARG;
  }
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_get_csr_pattern(const opf_handle* h, int which, int* nrows, int* ncols, long long* nnz, int* rowptr,
                        int* colind) {
  if (!h) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  const std::vector<int>* rp = nullptr;
  const std::vector<int>* ci = nullptr;
  int nr = 0;
  switch (which) {
    case OPF_MAT_G: rp = &P.G.rp; ci = &P.G.ci; nr = P.nx; break;
    case OPF_MAT_A: rp = &P.A.rp; ci = &P.A.ci; nr = P.m; break;
    case OPF_MAT_W:
    case OPF_MAT_K: rp = &P.Knat_rp; ci = &P.Knat_ci; nr = P.nw; break;
    default: return OPF_ERR_INVALID_ARG;
  }
  if (nrows) *nrows = nr;
  if (ncols) *ncols = P.nw;
  if (nnz) *nnz = rp->back();
  if (rowptr) std::memcpy(rowptr, rp->data(), rp->size() * sizeof(int));
  if (colind) std::memcpy(colind, ci->data(), ci->size() * sizeof(int));
  return OPF_OK;
}

int opf_get_csr_values(opf_handle* h, int which, double* dst) {
  if (!h || !dst) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  switch (which) {
    case OPF_MAT_G:
      if (!h->have_eval) return OPF_ERR_INVALID_ARG;
      CK(cudaMemcpyAsync(dst, h->Gval, P.G.nnz() * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
      break;
    case OPF_MAT_A:
      if (!h->have_eval) return OPF_ERR_INVALID_ARG;
      CK(cudaMemcpyAsync(dst, h->Aval, P.A.nnz() * sizeof(double), cudaMemcpyDeviceToDevice, h->s));
      break;
    case OPF_MAT_W:
      if (!h->have_W) return OPF_ERR_INVALID_ARG;
      CK(launch_gather_map(h->s, P.K.nnz(), h->Knat_map, h->Wval, dst));
      break;
    case OPF_MAT_K:
      if (!h->have_condense) return OPF_ERR_INVALID_ARG;
      CK(launch_gather_map(h->s, P.K.nnz(), h->Knat_map, h->Kval, dst));
      break;
    default: return OPF_ERR_INVALID_ARG;
  }
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_gx_factor(opf_handle* h) {
  if (!h || !h->have_eval) return OPF_ERR_INVALID_ARG;
  TRY(factor_async(h));
  int rc = read_status(h);
  if (rc != OPF_OK) h->have_lu = false;
  return rc;
}

int opf_gx_solve(opf_handle* h, int trans, const double* B, double* X, int nrhs) {
  if (!h || !B || !X || nrhs < 1 || !h->have_lu) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  double* ws = workspace(h, (size_t)P.nx * nrhs);
  if (!ws) return OPF_ERR_OOM;
  CK(launch_permute_rows(h->s, P.nx, nrhs, h->perm, B, P.nx, 1, ws, nrhs, 0, 1.0, 0));
  TRY(lu_solve_perm(h, trans ? 1 : 0, ws, nrhs, 1, nrhs));
  CK(launch_permute_rows(h->s, P.nx, nrhs, h->perm, ws, nrhs, 0, X, P.nx, 1, 1.0, 1));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_condense(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s, double* Kred) {
  if (!h || !sig_u || !sig_x || !sig_s || !h->have_W) return OPF_ERR_INVALID_ARG;
  TRY(condense_async(h, sig_u, sig_x, sig_s));
  if (Kred)
    CK(cudaMemcpyAsync(Kred, h->Kred, sizeof(double) * (size_t)h->P.nu * h->P.nu, cudaMemcpyDeviceToDevice,
                       h->s));
  int rc = read_status(h);
  if (rc != OPF_OK) {
    h->have_condense = false;
    h->have_lu = false;
  }
  return rc;
}

int opf_condense_rhs(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s,
                     const double* rhs, double* Kred) {
  if (!h || !sig_u || !sig_x || !sig_s || !rhs || !h->have_W) return OPF_ERR_INVALID_ARG;
  TRY(condense_async(h, sig_u, sig_x, sig_s, rhs));
  if (Kred)
    CK(cudaMemcpyAsync(Kred, h->Kred, sizeof(double) * (size_t)h->P.nu * h->P.nu, cudaMemcpyDeviceToDevice,
                       h->s));
  int rc = read_status(h);
  if (rc != OPF_OK) {
    h->have_condense = false;
    h->have_lu = false;
    h->fr_ready = false;
    h->fr_have_b = false;
  }
  return rc;
}

int opf_kkt_solve_condensed(opf_handle* h, double* step) {
  if (!h || !step || !h->have_factor || !h->fr_have_b) return OPF_ERR_INVALID_ARG;
  TRY(kkt_solve_prepared(h, step));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_kkt_factor(opf_handle* h, double delta_w, double delta_c, int* fail_col) {
  if (fail_col) *fail_col = -1;
  if (!h || !h->have_condense || !(delta_w >= 0.0) || !(delta_c >= 0.0) || !(delta_c < 1e300))
    return OPF_ERR_INVALID_ARG;
  if (delta_c != h->delta_c) {
    TRY(recondense_dc(h, delta_c));
    int rc = condipm::read_status(h);
    if (rc != OPF_OK) {
      h->have_condense = false;
      return rc;
    }
  }
  TRY(factor_kred_async(h, delta_w));
  int info = -1;
  int rc = condipm::read_status(h, &info);
  if (fail_col) *fail_col = rc == OPF_ERR_NOT_PD ? info : -1;
  h->have_factor = rc == OPF_OK;
  return rc;
}

int opf_get_factor(opf_handle* h, double* dst) {
  if (!h || !dst || !h->have_factor) return OPF_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(dst, h->F, sizeof(double) * (size_t)h->P.nu * h->P.nu, cudaMemcpyDeviceToDevice, h->s));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_kkt_solve(opf_handle* h, const double* rhs, double* step, int nrhs) {
  if (!h || !rhs || !step || nrhs < 1 || !h->have_factor) return OPF_ERR_INVALID_ARG;
  TRY(kkt_solve_impl(h, rhs, step, nrhs, 0));
  CK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int opf_kkt_solve_adjoint(opf_handle* h, const double* rhs, double* sol, int nrhs) {
  // K_aug is symmetric (Eq. kktmatrix:normal), so the transposed system is solved
  // by the same reduction and recovery.
  return opf_kkt_solve(h, rhs, sol, nrhs);
}

unsigned long long opf_launch_count(void) { return launch_count(); }

int opf_profile(opf_handle* h, int enable) {
  if (!h) return OPF_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->s));
  for (auto& r : h->recs) { h->evpool.push_back(r.a); h->evpool.push_back(r.b); }
  h->recs.clear();
  for (int p = 0; p < OPF_PHASE_COUNT; ++p) { h->ph_ms[p] = 0.0; h->ph_n[p] = 0; }
  h->profiling = enable != 0;
  return OPF_OK;
}

int opf_phase_times(opf_handle* h, double* ms, long long* launches) {
  if (!h) return OPF_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->s));
  for (auto& r : h->recs) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    h->ph_ms[r.phase] += t;
    h->ph_n[r.phase] += 1;
    h->evpool.push_back(r.a);
    h->evpool.push_back(r.b);
  }
  h->recs.clear();
  for (int p = 0; p < OPF_PHASE_COUNT; ++p) {
    if (ms) ms[p] = h->ph_ms[p];
    if (launches) launches[p] = h->ph_n[p];
  }
  return OPF_OK;
}

int opf_reduced_gradient(opf_handle* h, const double* grad, double* grad_r, double* lam) {
  if (!h || !grad_r || !h->have_eval || !h->have_lu) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const double* g = grad ? grad : h->gradf;
  double* ws = workspace(h, 2 * (size_t)P.nx);
  if (!ws) return OPF_ERR_OOM;
  double* t = ws;                 // elimination order
  double* ln = ws + P.nx;         // natural order
  // lam = -G_x^{-T} grad_x
  CK(launch_permute_rows(s, P.nx, 1, h->perm, g + P.nu, P.nx, 1, t, 1, 0, -1.0, 0));
  TRY(lu_solve_perm(h, 1, t, 1, 1, 1));
  CK(launch_permute_rows(s, P.nx, 1, h->perm, t, 1, 0, ln, P.nx, 1, 1.0, 1));
  // grad_r = grad_u + G_u^T lam  (the first nu rows of G^T in natural order)
  CK(cudaMemcpyAsync(grad_r, g, sizeof(double) * P.nu, cudaMemcpyDeviceToDevice, s));
  CK(launch_spmm(s, P.nu, h->GTn_rp, h->GTn_ci, h->Gval, h->GTn_map, ln, 1, 1, grad_r, 1, 1, 1, 1.0, 1.0));
  if (lam) CK(cudaMemcpyAsync(lam, ln, sizeof(double) * P.nx, cudaMemcpyDeviceToDevice, s));
  return read_status(h);
}

int opf_powerflow(opf_handle* h, const double* u, double* x, double tol, int max_iter, int* iters) {
  if (!h || !u || !x || !(tol > 0.0) || max_iter < 0) return OPF_ERR_INVALID_ARG;
  return condipm::powerflow_impl(h, u, x, tol, max_iter, iters);
}

}  // extern "C"
