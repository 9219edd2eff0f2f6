// Internal (non-ABI) entry points shared by the library's translation units.
#pragma once
#include "opf_handle.h"

namespace condipm {

int eval_impl(opf_handle* h, const double* x, const double* u, const double* lam, const double* y, bool derivs);
int factor_async(opf_handle* h);
// rhs (device, natural layout, one right-hand side; may be NULL): condensed in
// the same pass as one extra column (adjoint route; kept in the handle for
// kkt_solve_prepared)
int condense_async(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s,
                   const double* rhs = nullptr);
int factor_kred_async(opf_handle* h, double delta_w);
// fold the dual regularisation delta_c of the inequality rows into K, H and Kred
int recondense_dc(opf_handle* h, double delta_c);
// X (row-major nu x k, device) <- (L L^T)^{-1} X with the current factor
int chol_solve_async(opf_handle* h, double* X, int k);
// K_aug p = -r (external layout), with up to `refine` refinement corrections
int kkt_solve_impl(opf_handle* h, const double* rhs, double* step, int k, int refine);
// K_aug p = -r for the right-hand side given to the last condense_async (from
// its extra column when it is still valid, else by the plain recovery)
int kkt_solve_prepared(opf_handle* h, double* step);
// the buffers of the condensed right-hand side (allocated before any capture)
int fr_reserve(opf_handle* h);
int polish_solution(opf_handle* h, double tol, int max_iter);
int ipm_reserve(opf_handle* h);
int autotune_at_flat_start(opf_handle* h);

// k right-hand sides of K_aug in the internal layout (row-major, k lanes): the w
// block in c-order, s and y natural, lambda in elimination order; contiguous
// blocks [w | s | l | y] when made by kb_at.
struct KB {
  double *w = nullptr, *s = nullptr, *l = nullptr, *y = nullptr;
};
size_t kkt_rows(const Plan& P);
size_t kkt_core_scratch(const Plan& P);
size_t kkt_refine_scratch(const Plan& P, int k);
KB kb_at(const Plan& P, double* base, int k);
// p = K_aug^{-1} b through the condensed system (b_l = 0 may be declared)
int kkt_core(opf_handle* h, int k, const KB& b, const KB& p, bool bl_zero, double* scratch);
// R = b - K_aug z with the full sparse K_aug
// (with delta_w > 0: + delta_w on the u block of K_aug's primal rows)
int kkt_residual(opf_handle* h, int k, const KB& b, const KB& z, const KB& R, double delta_w = 0.0);
// z <- refined solution of K_aug z = b (solve_first: start from the condensed
// solve, else from z); at most max_steps corrections; relative max-norm residual
// and the corrections taken are returned
int kkt_refine(opf_handle* h, int k, const KB& b, const KB& z, bool solve_first, bool bl_zero, int max_steps,
               double* scratch, double* final_res, int* steps, bool fullspace = false);
// the hybrid full-space solver (block LDL^T of the slack-eliminated augmented
// matrix): Sigma of the next factorisations (device, natural order; drops the
// condensed state), the assembly + factorisation + inertia count with
// (delta_w, delta_c) (status word: SINGULAR, TIMEOUT, NOT_PD = wrong inertia),
// the inertia read-back, p = K_aug^{-1} b in the KB layout, the natural-layout
// solve with refinement, and the release of its state
int fs_set_sigma(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s);
int fs_factor_async(opf_handle* h, double delta_w, double delta_c);
int fs_read_inertia(opf_handle* h, int* inertia, double* logdet);
int fs_core(opf_handle* h, int k, const KB& b, const KB& p);
int fs_solve_impl(opf_handle* h, const double* rhs, double* step, int k, int refine, int* steps, double* res);
void fs_release(opf_handle* h);
double fs_delta_w(const opf_handle* h);   // delta_w of the last block factorisation
int read_status(opf_handle* h, int* info = nullptr);
// bracket the launches enqueued between the two calls with events (opf_profile)
void ph_begin(opf_handle* h, int phase);
void ph_end(opf_handle* h);
double* workspace(opf_handle* h, size_t n);
double* ybuf_reserve(opf_handle* h, size_t n);
int lagrangian_gradient(opf_handle* h, const double* lam, const double* y, double* out);
// gu_c0 >= 0 (trans = 0): X's columns are P G_u's from column gu_c0 on, exact
// zeros outside its pattern (the forward sweep's reach lists apply)
int lu_solve_perm(opf_handle* h, int trans, double* X, long long xr, long long xc, int ncols,
                  bool timed = false, int gu_c0 = -1);
int sens_prepare(opf_handle* h, const double* w, const double* lam, const double* y, const double* sig_w,
                 const double* sig_s);
int powerflow_impl(opf_handle* h, const double* u, double* x, double tol, int max_iter, int* iters);
// lockstep batches: the condensation rendezvous of instance idx (returns its
// status), and the end of an instance's loop
int batch_join(opf_batch* b, int idx, const double* su, const double* sx, const double* ss);
void batch_leave(opf_batch* b);

}  // namespace condipm
