// Shared device helpers and kernel declarations of the condensed-IPM library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace condipm {

// device status word: [0] first error code, [1] its detail (row / column),
// [2] a bounded wait expired
enum { ST_CODE = 0, ST_INFO = 1, ST_TIMEOUT = 2, ST_WORDS = 4 };
enum { DEV_OK = 0, DEV_NOT_PD = 1, DEV_SINGULAR = 2, DEV_TIMEOUT = 3 };

__device__ __forceinline__ void set_status(int* st, int code, int info) {
  if (atomicCAS(&st[ST_CODE], 0, code) == 0) atomicExch(&st[ST_INFO], info);
}

// Sense-reversing grid barrier with a bounded spin.  bar[0] counts arrivals,
// bar[1] is the generation.  Returns false (and flags st[ST_TIMEOUT]) when the
// wait exceeds spin_limit polls; callers then leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, long long spin_limit,
                                             int* st) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* vgen = bar + 1;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (++it > spin_limit) {
          atomicExch(&st[ST_TIMEOUT], 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Kernel launches enqueued by this library (all handles, all threads).
void note_launch();
unsigned long long launch_count();
// The last failed CUDA runtime call's error (any thread), for diagnostics.
void note_cuda_error(cudaError_t e);
int last_cuda_error();

// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per kernel and device.  The limit is process-wide per kernel, so it is
// never set per launch: a launch of another handle on another host thread,
// needing more, could otherwise run between the setting and this launch.
cudaError_t allow_max_smem(const void* fn);
// Allow clusters of up to 16 CTAs for a kernel, once per kernel and device
// (the same reasoning: attributes are not set per launch).
cudaError_t allow_cluster16(const void* fn);

// ---------------------------------------------------------------- launchers
// All launchers enqueue on `s` and return the launch error.

// model (A1-A3)
cudaError_t launch_bus_state(cudaStream_t s, int nb, int nu, const double* x, const double* u,
                             const int* th_w, const int* vm_w, double* Vm, double* Va);
cudaError_t launch_end_eval(cudaStream_t s, int ne, const int* end_i, const int* end_k,
                            const int* end_h, const double* gs, const double* bs, const double* gm,
                            const double* bm, const double* Vm, const double* Va, double* pq,
                            double* dsrc, double* hpq, double* h, int want_derivs);
cudaError_t launch_bus_sum(cudaStream_t s, int nb, int ng, int nu, int slack, const int* bus_end_ptr,
                           const int* bus_end, const double* pq, const int* g_row_P,
                           const int* g_row_Q, const int* gen_of_bus, const double* Pd,
                           const double* Qd, const double* u, const double* c2, const double* c1,
                           const double* lam, const double* y, double* g, double* h, double* Pg,
                           double* wP, double* wQ);
cudaError_t launch_objective(cudaStream_t s, int ng, const double* Pg, const double* c2,
                             const double* c1, double* f);
cudaError_t launch_gather(cudaStream_t s, int n, const int* ptr, const int* idx, const double* cst,
                          const double* src, double* out);
cudaError_t launch_gradf(cudaStream_t s, int nw, int ng, const int* pg_of_w, const int* slackpos,
                         const double* Pg, const double* c2, const double* c1, const double* Aval,
                         double* gradf);
cudaError_t launch_end_hess(cudaStream_t s, int ne, const int* end_i, const int* end_h,
                            const double* pq, const double* dsrc, const double* hpq, const double* wP,
                            const double* wQ, const double* y, double* hw);
cudaError_t launch_bilin_fixed(cudaStream_t s, int n, const int* pos, const int* a, const int* b,
                               double coef, const double* A, double* out);

// condensation (A4, A7, A8)
cudaError_t launch_assemble_K(cudaStream_t s, long long nnz, const double* W, const int* ptr,
                              const int* r, const int* a, const int* b, const double* sig_s,
                              const double* Aval, double* K);
cudaError_t launch_add_diag(cudaStream_t s, int nw, int nu, const int* K_diag, const int* perm,
                            const double* sig_u, const double* sig_x, double* K, double* sig_c);
cudaError_t launch_add_diag_c(cudaStream_t s, int nw, const int* K_diag, const double* sig_c, double* K);
cudaError_t launch_sigma_dc(cudaStream_t s, int m, double dc, const double* sig_s, double* sig_t, double* scale);
cudaError_t launch_scatter_rows(cudaStream_t s, int nrows, const int* rp, const int* ci,
                                const int* map, const double* src, double alpha, double* X, long long xr,
                                long long xc);
cudaError_t launch_spmm(cudaStream_t s, int nrows, const int* rp, const int* ci, const double* val,
                        const int* valmap, const double* X, long long xr, long long xc, double* Y,
                        long long yr, long long yc, int ncols, double alpha, double beta);
cudaError_t launch_trsm(cudaStream_t s, int cb, int nlev, const int* lptr, const int* lrows,
                        const int* rp, const int* ci, const double* val, const double* inv_diag,
                        double* X, long long xr, long long xc, int ncols);
cudaError_t launch_symmetrize(cudaStream_t s, int n, const double* A, long long ar, long long ac,
                              double* S);
cudaError_t launch_dense_tn(cudaStream_t s, int nu, int nx, const double* Sx, const double* Hx,
                            const double* Hu, long long ld, double* Kred, double* scratch, int nslices);
// slices of the explicit route's sum over nx (enough CTAs for the device; the
// scratch of nslices nu x nu partial sums at most 256 MB; 1 = no scratch)
int dense_tn_slices(int nu, int nx);

// Staged supernodal multi-RHS triangular solve (device view of an SnStream with
// its values filled for one factor).  big supernodes read int_beg / val /
// inv_diag (NULL = unit diagonal) of the strict pattern in place.
struct StDev {
  int nchunks, cap;
  const long long* chunk_off;
  const int *chunk_bytes, *chunk_big_f, *chunk_big_w;
  const unsigned char* bytes;
  const int* int_beg;
  const double* val;
  const double* inv_diag;
};
// Solve in place on an n x ncols block, element (i, c) at X[i*xr + c*xc]; upper
// selects the backward sweep; cb columns per CTA in shared memory.
cudaError_t launch_trsm_st(cudaStream_t s, int cb, bool upper, const StDev& T, int n, double* X, long long xr,
                           long long xc, int ncols, int* st, long long spin_limit);
int trsm_st_max_cb(int n, int cap);
// Column-parallel multi-RHS triangular solve (device view of a ColSched).
struct ColDev {
  int nlev, maxseg;
  const int *lvl_ptr, *sn_first, *sn_w, *lvl_seg_ptr, *seg_q0, *seg_q1, *seg_row, *row_seg, *row_nseg;
  const int *ext_beg, *ext_end, *int_beg;
};
// X row-major (element (i, c) at X[i*ld + c]); ksplit CTAs per 32 columns, all
// resident (cooperative launch); scratch holds ncb * maxseg * 32 doubles and bar
// ncb counters.
cudaError_t launch_trsm_cols(cudaStream_t s, bool upper, const ColDev& S, const int* ci, const double* val,
                             const double* inv_diag, double* X, long long ld, int ncols, int ksplit,
                             double* scratch, unsigned* bar, int* st, long long spin_limit);
int trsm_cols_max_blocks();

// Level-blocked solve with explicit inverses of the diagonal blocks.  rows /
// row_sn list each level's rows and their (split) supernode; D holds every
// supernode's dense inverse, row-major w x w at d_off[s].
struct BlkDev {
  int nlev;
  const int *lvl_rptr, *rows, *row_sn, *sn_first, *sn_w, *d_off, *ext_beg, *ext_end;
  // the factor's pattern is upper triangular: the diagonal-block inverses D_s
  // are upper triangular (else lower), so row r of D_s is zero left (right) of r
  int upper;
  // forward sweeps on P G_u: per full 32-column block of G_u (rch_nblk of
  // them) the positions in rows of the rows where the solution can be nonzero,
  // nlev + 1 offsets per block into rch_q (null: no lists)
  const int *rch_ptr, *rch_q;
  int rch_nblk;
};
// inverse of every (split) supernode's diagonal block of one factor
struct DiagInvJob {
  int nsn, upper;
  const int *sn_first, *sn_w, *d_off, *int_beg;
  const double *val, *inv_diag;   // inv_diag NULL: unit diagonal
  double* D;
};
cudaError_t launch_diag_inv4(cudaStream_t s, const DiagInvJob* jobs);
// X, Y row-major with leading dimension ld (Y: scratch of the same shape);
// ksplit CTAs per 32 columns, cooperative launch; bar holds ncb counters.
// minb: the register bound's CTAs per SM (5, 6 or 8; see the kernel)
constexpr int BLK_MINB[3] = {5, 6, 8};
// rch_cb0 >= 0: X's columns are those of P G_u from column 32 rch_cb0 on (with
// exact zeros outside its pattern): the full blocks pass by the rows outside
// their reach lists (S.rch_*) and the levels without such rows
cudaError_t launch_trsm_blk(cudaStream_t s, const BlkDev& S, const int* ci, const double* val, const double* D,
                            double* X, double* Y, long long ld, int ncols, int ksplit, unsigned* bar, int* st,
                            long long spin_limit, int minb = 5, int rch_cb0 = -1);
int trsm_blk_max_blocks(int minb = 5);
// the level-blocked solve, both triangles, with one thread-block cluster of cl
// CTAs per 32-column block (cluster barrier between phases); clusters of cl that
// fit at once (0: none)
cudaError_t launch_trsm_blkc(cudaStream_t s, const BlkDev& SL, const int* ciL, const double* valL,
                             const double* DL, const BlkDev& SU, const int* ciU, const double* valU,
                             const double* DU, double* X, double* Y, long long ld, int ncols, int cl,
                             int rch_cb0 = -1);
int trsm_blkc_clusters(int cl);
// Dataflow (barrier-free) form of the level-blocked solve: task list of
// phase-A (row >= 0) and phase-B (-1 - row) warp tasks in level order, each
// row's supernode, and the supernodes each row's external entries lie in.
// supernodes up to this width get no phase-B tasks: the warp whose phase-A
// task completes the supernode multiplies by D_s itself
constexpr int DF_INLINE_B = 4;
struct DfDev {
  int ntask, nsn;
  const int *task, *sn_of, *sn_first, *sn_w, *d_off, *ext_beg, *ext_end, *dep_ptr, *dep_sn;
  // leaf supernodes (no external entries, width <= DF_LEAF_W): solved by a
  // separate pass before the dataflow kernel, their tasks left out of task
  int nleaf;
  const int* leaf;
  // rows with more than DF_CHUNK external entries are split into chunk tasks
  // (task code n + chunk id): chunk k covers entries ck_e0[k] .. ck_e1[k] of
  // row ck_row[k]; row r's chunks are rw_ck0[r] .. rw_ck0[r + 1] (none for
  // short rows) and it counts its finished chunks in slot rw_cidx[r]
  int n, nchunks, nchunked;
  const int *ck_row, *ck_e0, *ck_e1, *rw_ck0, *rw_cidx;
  int upper;   // as in BlkDev: which half of each D_s is zero
};
constexpr int DF_LEAF_W = 8;
constexpr int DF_CHUNK = 24;
// cnt: ncb * (2 nsn + nchunked) counters (zeroed here); Pc: nchunks * 32 ncb
// partial sums of the chunk tasks; cooperative launch of ncb * ksplit CTAs.
cudaError_t launch_trsm_df(cudaStream_t s, const DfDev& S, const int* ci, const double* val, const double* D,
                           double* X, double* Y, long long ld, int ncols, int ksplit, unsigned* cnt,
                           double* Pc, int* st, long long spin_limit);
int trsm_df_max_blocks();
// One right-hand side X[i * xs] (Y: scratch of the same stride); nblocks CTAs,
// cooperative launch; bar holds one counter.
cudaError_t launch_trsm_blk1(cudaStream_t s, const BlkDev& S, const int* ci, const double* val, const double* D,
                             double* X, double* Y, long long xs, int nblocks, unsigned* bar, int* st,
                             long long spin_limit);
// One-CTA level-blocked schedule of one factor: the levels of the level list
// (as in BlkDev) and, per position q in it, the row's descriptions for the
// two phases: ma[q] = {row, first and end external entry, 0}, mb[q] = {row,
// offset of the row in its supernode, supernode width, offset of the row's
// entries in D}.
struct Lu1sDev {
  int nlev;
  const int* lvl_rptr;
  const int4 *ma, *mb;
};
// One right-hand side X[i * xs] through both triangles (L then U) in one CTA
// with the vector and a level's worth of Y (ymax entries) in shared memory;
// g = lanes per row (4 or 8).  The shared memory it needs, (n + ymax) doubles,
// must not exceed trsm_lu1s_max_smem().
cudaError_t launch_trsm_lu1s(cudaStream_t s, int g, const Lu1sDev& L, const int* ciL, const double* valL,
                             const double* DL, const Lu1sDev& U, const int* ciU, const double* valU,
                             const double* DU, double* X, long long xs, int n, int ymax);
size_t trsm_lu1s_max_smem();
// One right-hand side on one thread-block cluster of CL CTAs (CL <= 16), each
// with a full copy of the vector; the schedule of each triangle (layout as the
// host ClSched) shares every level's supernodes out over the CTAs.
struct Cl1Dev {
  int nlev, CL, ymax;
  const int* t_ptr;
  const int4 *ta, *tb;
};
cudaError_t launch_trsm_lu1c(cudaStream_t s, const Cl1Dev& L, const int* ciL, const double* valL,
                             const double* DL, const Cl1Dev& U, const int* ciU, const double* valU,
                             const double* DU, double* X, long long xs, int n);
// clusters of CL CTAs that can be resident at once with the shared memory the
// solve needs, (n + ymax) doubles and nlev + 1 ints (0: it does not fit)
int trsm_lu1c_max_clusters(int CL, int n, int ymax, int nlev);
cudaError_t launch_fill_stream(cudaStream_t s, long long nslots, const long long* slot, const int* src,
                               const double* vals, const double* inv_diag, int unit, unsigned char* stream);

// LU (A5)
cudaError_t launch_lu_scatter(cudaStream_t s, long long nnzG, const int* Gx_to_LU, const double* Gval,
                              double* LU);
cudaError_t launch_row_absmax(cudaStream_t s, int n, const int* rp, const double* val, double* rmax);
cudaError_t launch_lu_refactor(cudaStream_t s, int n, const int* rows, const int* rp, const int* ci,
                               const int* diag, const long long* upd_ptr, const int* upd_pos,
                               double* LU, double* inv_diag, const double* rmax, unsigned* flags,
                               unsigned epoch, int* st, long long spin_limit, int nblocks, int nthreads,
                               int maxlen);
int lu_refactor_max_blocks(int nthreads, size_t smem);
cudaError_t launch_gather_map(cudaStream_t s, long long n, const int* map, const double* src,
                              double* dst);

// dense Cholesky (A9)
cudaError_t launch_chol_prepare(cudaStream_t s, int n, const double* A, double delta, double* F);
cudaError_t launch_chol(cudaStream_t s, int n, double* F, double* dinv, int* st, unsigned* bar,
                        long long spin_limit, int nblocks);
int chol_max_blocks();
// SMs of the current device
int device_sms();
// grid of the barrier-form Cholesky of an n x n matrix before tuning: enough CTAs
// for the first step's tiles, at most two per SM and never more than are resident
int chol_grid_cap(int n);
// Dataflow (barrier-free, look-ahead) Cholesky: np panel CTAs, nblocks - np
// update CTAs (at least one); cnt holds 2 * ceil(n / 32) counters (zeroed here).
int chol_df_max_blocks();
// Finv[I] = inverse of the I-th 32 x 32 diagonal tile of the Cholesky factor
// (zero-padded), for nt = ceil(n / 32) tiles
cudaError_t launch_tile_inv(cudaStream_t s, int n, const double* F, const double* dinv, double* Finv);
// X (row-major n x nrhs) <- (L L^T)^{-1} X, one cluster of CL (<= 16) CTAs per
// column, with the tile inverses of launch_tile_inv
cudaError_t launch_chol_solve_cl(cudaStream_t s, int n, const double* F, const double* Finv, double* X, int nrhs,
                                 int CL);
cudaError_t launch_chol_df(cudaStream_t s, int n, double* F, double* dinv, int* st, unsigned* cnt,
                           long long spin_limit, int nblocks, int np);
cudaError_t launch_chol_solve(cudaStream_t s, int n, const double* F, const double* dinv, double* X, int nrhs);

// vectors
cudaError_t launch_permute_rows(cudaStream_t s, int n, int ncols, const int* idx, const double* src,
                                int ld_src, int src_colmajor, double* dst, int ld_dst, int dst_colmajor,
                                double alpha, int inverse);
cudaError_t launch_axpby(cudaStream_t s, long long n, double a, const double* x, double b,
                         const double* y, double* z);
cudaError_t launch_scale_rows(cudaStream_t s, int n, int ncols, const double* d, const double* x,
                              double* z, double b, const double* y);
cudaError_t launch_absmax(cudaStream_t s, long long n, const double* x, double* out);
cudaError_t launch_fill(cudaStream_t s, long long n, double v, double* x);
cudaError_t launch_set_identity(cudaStream_t s, int n, double* X, int ld);
// dst[i * ldd] = a * src[i * lds] + b * y[i * ldy] for i < n (y may be NULL)
cudaError_t launch_column_axpby(cudaStream_t s, int n, double a, const double* src, long long lds, double b,
                                const double* y, long long ldy, double* dst, long long ldd);

// ----------------------------------------------------------------- batches
// One instance of a batched condensation (opf_batch_condense_factor): the device
// arrays of its handle that the batched phase kernels read and write.  A device
// array of these, one per instance, is what every batched launch indexes.
struct BatchInst {
  int active;   // 0: this instance takes no part in the call (its items are skipped)
  int nx, nu, nw, m, ld;
  long long nnzG, nnzLU, nnzK, nnzLo, nnzUp;
  // G_x refactorisation
  const int *Gx_to_LU, *LU_rp, *LU_ci, *LU_diag;
  const long long* upd_ptr;
  const int* upd_pos;
  const double* Gval;
  double *LUval, *inv_diag, *rmax;
  unsigned* flags;
  int* st;
  int maxlen;
  const int *Lo_map, *Ut_map, *Up_map, *Lt_map;
  double *Lo_val, *Ut_val, *Up_val, *Lt_val;
  // staged-solve byte streams of the lower (0) and upper (1) patterns
  long long st_nslots[2];
  const long long* st_slot[2];
  const int* st_src[2];
  double *st_a[2], *st_b[2];
  DiagInvJob dj[4];
  // K = W + A^T Sigma_s A + diag(Sigma_w)
  const double *Wval, *Aval;
  const int *KAA_ptr, *KAA_r, *KAA_a, *KAA_b, *K_diag, *perm, *K_rp, *K_ci;
  const double *sig_u, *sig_x, *sig_s_in;
  double *sig_s, *sig_c, *Kval;
  // Z = [I; S_x], H = K Z, Psi, Kred
  double *Zt, *H, *Y;
  const int *PGu_rp, *PGu_ci, *PGu_map, *GuT_rp, *GuT_ci, *GuT_map;
  BlkDev bkL, bkU;
  const int *Lo_ci, *Up_ci;
  const double *D_L, *D_Ut, *D_U, *D_Lt;
  // Cholesky of Kred + delta_w I
  double *Kred, *F, *Fdinv;
  double delta_w;
};

// Work of one batched elementwise launch: block b of the launch belongs to the
// instance i with boff[i] <= b < boff[i + 1] (boff[n] = grid size).
__device__ __forceinline__ int batch_instance(const int* __restrict__ boff, int n, int b) {
  int lo = 0, hi = n;   // boff[lo] <= b < boff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (boff[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Batched phase launches (one launch for every instance of the batch; I is the
// device descriptor array, n instances).  Block offsets boff per launch shape:
// BOFF_LU (nnz(LU) and nnz(G) elements), BOFF_K (nnz(K)), BOFF_X (nx rows of Z),
// BOFF_W (nw rows of H), BOFF_U (nu rows of Kred), BOFF_F (factor entries
// nnz(Lo) + nnz(Up) and staged slots), BOFF_D (warps: 2 (supernodes of L +
// supernodes of U), four per block).
enum { BOFF_LU = 0, BOFF_K = 1, BOFF_X = 2, BOFF_W = 3, BOFF_U = 4, BOFF_F = 5, BOFF_D = 6, BOFF_KINDS = 7 };
constexpr int BATCH_EW_THREADS = 256;
constexpr int BATCH_EW_ITEMS = 4;   // elements (rows) per thread and launch of an elementwise phase
// A5 prologue: zero LU, the row flags, the status word and S_x; then scatter
// G_x into LU, -P G_u into S_x, assemble K and copy Sigma_s; then the row
// maxima of LU and diag(Sigma_w) into K
cudaError_t launch_batch_prologue(cudaStream_t s, const BatchInst* I, int n, const int* const* boff,
                                  const int* nblocks);
// A5: the numeric LU of every instance, one cooperative launch over the merged
// row list items (instance, row) in level order
cudaError_t launch_batch_lu(cudaStream_t s, const BatchInst* I, const int2* items, int nitems, int nblocks,
                            int maxlen, unsigned epoch, long long spin_limit);
int batch_lu_max_blocks(int maxlen);
// A5 epilogue: the four factors' gathers and staged streams, then their
// diagonal-block inverses (BOFF_D: one warp per factor and supernode)
cudaError_t launch_batch_factor_post(cudaStream_t s, const BatchInst* I, int n, const int* boffF, int nbF,
                                     const int* boffD, int nbD);
// A6: S_x (trans = 0: L then U) or Psi = G_x^{-T} H_x (trans = 1: U^T then L^T)
// for every instance, one cluster of cl CTAs per (instance, 32-column block) item
cudaError_t launch_batch_trsm(cudaStream_t s, const BatchInst* I, const int2* cbs, int ncbs, int trans, int cl);
// A7: H = K Z (which = 0), then H_u -= G_u^T Psi (which = 1)
cudaError_t launch_batch_spmm(cudaStream_t s, const BatchInst* I, int n, const int* boff, int nblocks, int which);
// A7 / A9: Kred = sym(H_u) and F = tril(Kred) + delta_w I
cudaError_t launch_batch_kred(cudaStream_t s, const BatchInst* I, int n, const int* boffU, int nblocks);
// the active instances' status words into out[ST_WORDS * n] (0 for the others)
cudaError_t launch_batch_status(cudaStream_t s, const BatchInst* I, int n, int* out);
// A9: Cholesky of every instance's F, one thread-block cluster of cl CTAs per instance
cudaError_t launch_batch_chol(cudaStream_t s, const BatchInst* I, int n, int cl);
// clusters of cl CTAs of the batched solve / Cholesky that fit on the device at
// once (0: that cluster size cannot be launched)
int batch_trsm_clusters(int cl);
int batch_chol_clusters(int cl);

}  // namespace condipm
