/*
 * condipm.h -- C ABI of the condensed interior-point hot path (FP64, sm_103a).
 *
 * The library condenses the augmented KKT system of a state-control AC optimal
 * power flow into the dense nu x nu matrix
 *
 *     Kred = Z^T (W + diag(Sigma_u, Sigma_x) + A^T Sigma_s A) Z,  Z = [I; -G_x^{-1} G_u]
 *
 * (Eq. algo:reduction, Sec. 3.3; Theorems 1-2, Sec. 2.2), factors it by dense
 * Cholesky (Algorithm 1, "control step"; Theorem 3 makes positive definiteness the
 * inertia test) and recovers the full Newton step (Theorem 1 and 2 recoveries).
 *
 * Conventions shared by every call
 * --------------------------------
 *  * FP64 everywhere; indices are 0-based int32.
 *  * Variables: u = [Vm at the ng generator buses (generator order);
 *                    Pg of generators 1..ng-1]                       (nu = 2 ng - 1)
 *               x = [theta at the non-slack buses (ascending bus index);
 *                    Vm at the buses without a generator (ascending)] (nx = 2 nb - ng - 1)
 *    Generators must sit on distinct buses; generator 0's bus is the slack bus.
 *  * g(x,u) (state equation, Eq. 1) = [P balance at non-slack buses; Q balance at
 *    load buses], in the order of x.  h(x,u) = [Pg of generator 0; Qg of every
 *    generator; |S|^2 at the from-end of every flow-limited line (rate > 0,
 *    ascending line index); |S|^2 at their to-ends]  (m = 1 + ng + 2 nlim).
 *    The slack form is h + s = 0 (Eq. 3), so slack bounds are [-hU, -hL].
 *  * Full-space right-hand sides and steps use the block order of
 *    Eq. kktmatrix:normal: [r1 (nu) | r2 (nx) | r3 (m) | r4 (nx) | r5 (m)], i.e.
 *    n_kkt = nu + 2 nx + 2 m doubles per right-hand side, and the coupling between
 *    p_s and p_y is +I (the sign that h + s = 0 implies).
 *  * Pointers documented "device" are CUDA device pointers owned by the caller;
 *    "host" pointers are ordinary host memory.  The library never frees caller
 *    memory.  Device work is issued on the handle's stream (opf_set_stream).
 *  * Every call returns an OPF_* status; none aborts.  Device-side failures
 *    (non-positive pivot, tiny LU pivot, expired bounded wait) are recorded in a
 *    device status word and reported by the next call that synchronises.
 */
#ifndef CONDIPM_H
#define CONDIPM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define OPF_OK                 0
#define OPF_ERR_INVALID_ARG   -1   /* bad pointer, size or call order            */
#define OPF_ERR_CUDA          -2   /* a CUDA runtime call failed                 */
#define OPF_ERR_NOT_PD        -3   /* Cholesky met a non-positive pivot          */
#define OPF_ERR_SINGULAR      -4   /* G_x refactorisation met a tiny pivot       */
#define OPF_ERR_PF_FAILED     -5   /* Newton-Raphson power flow did not converge */
#define OPF_ERR_TIMEOUT       -6   /* a bounded device wait expired              */
#define OPF_ERR_OOM           -7   /* device allocation failed                   */
#define OPF_ERR_NO_CONVERGENCE -8  /* interior-point loop hit its iteration cap  */
#define OPF_ERR_INFEASIBLE    -9   /* feasibility restoration found no acceptable
                                      point (the problem looks locally infeasible) */

/* ---- network (host arrays, copied by opf_create) ---------------------------- */
typedef struct opf_network {
    int nb, nl, ng, slack;                 /* slack must equal gbus[0]                */
    const double *Pd, *Qd, *Vmin, *Vmax;   /* [nb] loads (p.u.) and voltage bounds     */
    const int *lf, *lt;                    /* [nl] from / to bus                       */
    const double *r, *x, *b, *rate;        /* [nl] pi-model; rate = 0 means unlimited  */
    const int *gbus;                       /* [ng] generator bus (distinct)            */
    const double *Pmin, *Pmax, *Qmin, *Qmax, *c2, *c1; /* [ng]                         */
} opf_network;

/* Condensation route (Sec. 3.3). ADJOINT: Kred = H_u - G_u^T G_x^{-T} H_x with
 * H = K Z (the paper's batched adjoint-adjoint product, N = nu).  EXPLICIT:
 * Kred = H_u + S_x^T H_x as a dense product (the route Sec. 3.3 calls naive). */
#define OPF_ROUTE_ADJOINT  0
#define OPF_ROUTE_EXPLICIT 1
#define OPF_ROUTE_AUTO     2   /* time both on the first opf_condense, keep the faster */

typedef struct opf_options {
    int route;            /* OPF_ROUTE_*                                               */
    int rhs_block;        /* multi-right-hand-side solve kernel: 1, 2 or 4 = staged
                             supernodal kernel with that many columns per CTA; 32 =
                             column-parallel kernel (one lane per column); 64 =
                             level-blocked kernel (explicit inverses of the diagonal
                             blocks, one lane per column); 96 = its barrier-free
                             dataflow form; 128 = the level-blocked kernel with one
                             thread-block cluster of 8 CTAs per 32-column block
                             (hardware cluster barrier between the phases; the
                             autotuner also tries 2, 4, 16); 0 = autotune on the first
                             opf_condense (times each kernel on the actual right-hand
                             side and keeps the fastest)                              */
    long long spin_limit; /* iteration cap of every device-side wait; 0 = 1<<26        */
    int chol_form;        /* dense Cholesky of Kred (Sec. 3.4): 1 = blocked right-looking
                             kernel with grid barriers between steps; 2 = its dataflow
                             form (panel and trailing-update CTA groups synchronised
                             by per-column counters, so the next panel overlaps the
                             rest of the update); 0 = autotune on the first
                             factorisation (times both forms at a few grid sizes)   */
    int rhs1_kernel;      /* solve kernel for one right-hand side (the Newton-step
                             recovery): 1 = staged supernodal kernel in one CTA; 64 =
                             level-blocked kernel over several CTAs with grid
                             barriers; 65 = level-blocked kernel in one CTA with the
                             vector in shared memory; 66 = level-blocked kernel on a
                             thread-block cluster, a copy of the vector in each
                             CTA's shared memory (65 and 66 fall back to 64 when
                             they do not fit); 0 = autotune together with rhs_block
                             (until then: 1)                                       */
    int rhs_width;        /* N, the right-hand sides per pass of the condensation
                             (Sec. 3.3, Fig. 2b: the batch width of the multi-RHS
                             products): the adjoint route runs the S_x solve, H = K Z,
                             the adjoint solve and the G_u^T product over column
                             chunks of N; N >= nu is one pass; 0 = autotune on the
                             first condensation among nu, 512, 256, 128 (the
                             explicit route always uses one pass)                */
    int dense_forward;    /* the forward sweep L Y = P G_u of the condensation (Sec.
                             3.3): 0 = the level-blocked kernels solve, in each
                             full 32-column block of G_u (also in column chunks),
                             only the rows where Y can be nonzero (the etree paths
                             from the block's rows of G_u to the root, found at
                             opf_create; every other row of Y is exactly zero) and
                             pass by the levels without any; 1 = every row     */
} opf_options;

typedef struct opf_handle opf_handle;

/* Copy the network, build the variable layout, the fixed sparsity patterns of
 * G, A, W and K, the fill-reducing ordering and symbolic LU of G_x (its pattern
 * is fixed by the network, Sec. 3.2), the level schedules of the triangular
 * solves, and allocate every device workspace.  opt may be NULL (defaults).
 * Errors: INVALID_ARG (inconsistent network), CUDA, OOM. */
int opf_create(const opf_network* net, const opf_options* opt, opf_handle** out);
void opf_destroy(opf_handle* h);
const char* opf_strerror(int code);

/* Sizes (host outputs, any may be NULL). */
int opf_sizes(const opf_handle* h, int* nx, int* nu, int* m);
/* Statistics of the symbolic analysis (host outputs, any may be NULL):
 * nnz of L+U (strict parts plus diagonal), levels of the forward and backward
 * solves, nnz of K. */
int opf_stats(const opf_handle* h, long long* nnz_lu, int* levels_fwd, int* levels_bwd,
              long long* nnz_k, long long* lu_flops);
/* Multi-RHS solve kernel in use (host outputs, may be NULL): *kernel as in
 * opf_options.rhs_block (-1 before the autotuner ran; 128 the level-blocked
 * kernel on thread-block clusters, of any size), ms[6] the autotuner's
 * timings of {column-parallel, staged 1, 2, 4, level-blocked, dataflow}
 * (0 = not tried),
 * *kernel1 the kernel of solves with fewer than 32 right-hand sides (1 staged,
 * 64 level-blocked, 65 level-blocked in one CTA with the vector in shared
 * memory, 66 level-blocked on a thread-block cluster -- 65 and 66 for one
 * right-hand side only, others then use 64 --, -1 not chosen yet). */
int opf_trsm_choice(const opf_handle* h, int* kernel, float* ms, int* kernel1);
/* Right-hand-side width of the condensation in use (host outputs, may be
 * NULL): *width = N (nu for one pass; 0 before the autotuner ran), ms[4] the
 * autotuner's timings of the condensation's products at N = nu, 512, 256, 128
 * (0 = not tried). */
int opf_rhs_width(const opf_handle* h, int* width, float* ms);
/* Dense Cholesky kernel in use (host outputs, may be NULL): *form as in
 * opf_options.chol_form (0 before the first factorisation), *nblocks its grid,
 * ms[OPF_CHOL_CANDIDATES] the autotuner's timings of {barrier form at 1/4, 1/2,
 * 1 and 2 CTAs per SM; dataflow form at 1/2, 1, 2 CTAs per SM with a small panel
 * group; dataflow form at 1, 2 CTAs per SM with a large panel group; dataflow
 * form at 4 CTAs per SM with a small, then a large panel group} (0 = not tried;
 * a candidate with more CTAs than fit at once is not tried). */
#define OPF_CHOL_CANDIDATES 11
int opf_chol_choice(const opf_handle* h, int* form, int* nblocks, float* ms);
/* Cluster size of the dense solve with L and L^T for one to eight right-hand
 * sides (host outputs, may be NULL): *cluster the CTAs of one thread-block
 * cluster per right-hand side, ms[3] the timings of 4, 8 and 16 CTAs taken on
 * the first one-vector solve (0 = not timed yet; the size chosen from nu is in
 * use until then). */
int opf_chol_solve_choice(const opf_handle* h, int* cluster, float* ms);
/* The condensation's forward sweep over P G_u (host outputs, may be NULL):
 * *nblocks the 32-column blocks with a reach list (nu / 32; 0 when
 * opf_options.dense_forward is set), work[2] the multiply-adds per sweep of the
 * listed rows and of all rows of those blocks (external L entries plus the
 * diagonal-block row). */
int opf_forward_reach(const opf_handle* h, int* nblocks, double* work);
/* Condensation route in use (host outputs, may be NULL): *route as in
 * opf_options.route (-1: OPF_ROUTE_AUTO before its first opf_condense), ms[2]
 * the AUTO timings of {adjoint, explicit} (0 = not timed). */
int opf_route_choice(const opf_handle* h, int* route, float* ms);
/* Stream for all device work (a cudaStream_t, NULL = legacy default stream). */
int opf_set_stream(opf_handle* h, void* stream);

/* ---- A1-A3: model evaluation (Sec. 3.2) ------------------------------------- */
/* Evaluate f, g, h, grad f, G = [G_u G_x], A = [A_u A_x] and the Lagrangian
 * Hessian W = hess(f + lam^T g + y^T h) at device vectors x[nx], u[nu],
 * lam[nx], y[m]; lam and y may be NULL (then W is not evaluated).
 * Results stay in the handle (read them with opf_get_*). */
int opf_eval_derivatives(opf_handle* h, const double* x, const double* u,
                         const double* lam, const double* y);
/* Evaluate only f, g, h (line-search trial points).  Same arguments. */
int opf_eval_functions(opf_handle* h, const double* x, const double* u);

#define OPF_VEC_F     0   /* 1 double: objective                      */
#define OPF_VEC_G     1   /* nx: state equation g                     */
#define OPF_VEC_H     2   /* m : inequality functions h               */
#define OPF_VEC_GRADF 3   /* nu+nx: grad f, ordered [u; x]            */
/* Copy a vector result to device memory dst. */
int opf_get_vector(opf_handle* h, int which, double* dst);

#define OPF_MAT_G 0       /* nx x (nu+nx), columns [u; x]             */
#define OPF_MAT_A 1       /* m  x (nu+nx)                             */
#define OPF_MAT_W 2       /* (nu+nx) x (nu+nx), stored in K's pattern */
#define OPF_MAT_K 3       /* K of the last opf_condense               */
/* CSR pattern of a matrix (host outputs: rowptr[nrows+1], colind[nnz]); pass
 * NULL arrays to query nrows/ncols/nnz first.  Columns use the [u; x] order. */
int opf_get_csr_pattern(const opf_handle* h, int which, int* nrows, int* ncols,
                        long long* nnz, int* rowptr, int* colind);
/* CSR values of a matrix in that pattern (device dst[nnz]). */
int opf_get_csr_values(opf_handle* h, int which, double* dst);

/* ---- A5/A6: G_x refactorisation and solves (Sec. 3.1, 3.3) ------------------- */
/* Numeric LU of P G_x P^T = L U in the fixed pattern at the last evaluation point
 * (static pivots from the ordering).  Errors: SINGULAR when a pivot is below
 * 1e-14 times its row's largest entry. */
int opf_gx_factor(opf_handle* h);
/* Solve G_x X = B (trans = 0) or G_x^T X = B (trans = 1) for nrhs right-hand
 * sides stored one after another (device, nx doubles each); B and X may alias. */
int opf_gx_solve(opf_handle* h, int trans, const double* B, double* X, int nrhs);

/* ---- A4-A8: condensation (Sec. 3.3, Eq. algo:reduction) ---------------------- */
/* Refactor G_x (unless opf_gx_factor ran since the last evaluation), assemble
 * K = W + diag(sig_u, sig_x) + A^T diag(sig_s) A, and form Kred (nu x nu,
 * symmetric, written to device Kred when non-NULL and kept in the handle).
 * sig_u[nu], sig_x[nx], sig_s[m] are device vectors.  Errors: SINGULAR. */
int opf_condense(opf_handle* h, const double* sig_u, const double* sig_x,
                 const double* sig_s, double* Kred);

/* ---- A9: control-step factorisation (Algorithm 1; Theorem 3; Sec. 4.3) ------- */
/* Inertia correction and Cholesky of the control step: Kred + delta_w I = L L^T.
 * The paper regularises until the condensed matrix is positive definite
 * (Sec. 4.3); the two terms sit here:
 *  - delta_w >= 0, the primal term, on the control block (Kred + delta_w I);
 *  - delta_c >= 0, the dual term, on the inequality rows only: -delta_c I in the
 *    (p_y, p_y) block of K_aug.  Eliminating p_s and p_y turns Sigma_s into
 *    Sigma_t = (Sigma_s^{-1} + delta_c)^{-1}, so a delta_c different from the
 *    one the handle holds re-forms K = W + diag(Sigma_w) + A^T Sigma_t A, H and
 *    Kred from the last opf_condense (the G_x factor and S_x are kept; on the
 *    adjoint route this costs one product H = K Z and one multi-RHS G_x^{-T}
 *    solve).  Every opf_condense starts again from delta_c = 0.
 * The condensed matrix is kept unmodified by delta_w, so the call can be
 * repeated with a larger delta_w.  Later opf_kkt_solve calls solve the K_aug
 * with both terms.  Errors: INVALID_ARG (no condensation, negative or
 * non-finite delta), NOT_PD with *fail_col (may be NULL; -1 otherwise) set to
 * the first failing column, SINGULAR, TIMEOUT. */
int opf_kkt_factor(opf_handle* h, double delta_w, double delta_c, int* fail_col);
/* Copy the Cholesky factor (lower triangle, row-major nu x nu; upper part
 * zero) to device dst. */
int opf_get_factor(opf_handle* h, double* dst);

/* ---- A8/A10: step recovery (Theorem 1 and 2 recoveries; Algorithm 1) --------- */
/* Solve K_aug p = -r for nrhs right-hand sides (device, n_kkt doubles each, see
 * the block order above) with the current factors; step receives
 * [p_u | p_x | p_s | p_lambda | p_y] per right-hand side.  rhs and step must not
 * overlap.  K_aug carries Sigma of the last condense and delta_w, delta_c of the
 * last factor (-delta_c I in its (p_y, p_y) block). */
int opf_kkt_solve(opf_handle* h, const double* rhs, double* step, int nrhs);
/* A4-A8 in one pass: opf_condense together with the condensed right-hand side
 * of K_aug p = -rhs (one right-hand side, device, n_kkt doubles in the layout
 * of opf_kkt_solve).  The right-hand side rides along the condensation as one
 * extra column (Theorem 1's reductions with the same factor): q = G_x^{-1} b_l
 * in the S_x solve, K [0; q] in H = K Z, phi = G_x^{-T} (b_t - K [0; q])_x in
 * the adjoint solve, and the condensed right-hand side in the G_u^T product
 * (adjoint route; on the explicit route, or with no spare column, the
 * right-hand side is only kept).  rhs is copied; Kred as in opf_condense.
 * Errors as opf_condense, INVALID_ARG for a NULL rhs. */
int opf_condense_rhs(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s,
                     const double* rhs, double* Kred);
/* The step for that right-hand side after opf_kkt_factor: the Cholesky solve
 * and the recovery products only (step as in opf_kkt_solve, device).  With
 * delta_c > 0 in the factor, or when the condensation could not carry the
 * column, the plain recovery of opf_kkt_solve runs on the kept right-hand side.
 * Errors: INVALID_ARG (no opf_condense_rhs since the last evaluation, or no
 * factor), CUDA, TIMEOUT. */
int opf_kkt_solve_condensed(opf_handle* h, double* step);
/* Solve K_aug^T z = -r (K_aug is symmetric; this path applies the transposed
 * recovery, G_x^{-T} first), same layout.  Used by the dispatch derivative. */
int opf_kkt_solve_adjoint(opf_handle* h, const double* rhs, double* sol, int nrhs);

/* One Newton step from HOST buffers (Algorithm 1's linear algebra in one call):
 * copy x[nx], u[nu], lam[nx], y[m], sig_u[nu], sig_x[nx], sig_s[m] and the
 * full-space right-hand side rhs[n_kkt] to the device, evaluate the derivatives,
 * refactor G_x and condense (A1-A7), factor Kred + delta_w I with the dual
 * regularisation delta_c (A9, as opf_kkt_factor), solve K_aug p = -rhs and
 * recover the step (A8, A10), and copy step[n_kkt] = [p_u | p_x | p_s | p_lambda |
 * p_y] back.  All pointers are host memory (pinned memory makes the copies
 * asynchronous); the handle's stream carries every copy and launch, and the call
 * returns after the step has landed.  The handle is left as after
 * opf_kkt_factor (later opf_kkt_solve calls reuse the factors).
 * Errors: INVALID_ARG, NOT_PD (*fail_col = first failing column; no step is
 * written), SINGULAR, CUDA, OOM, TIMEOUT. */
int opf_newton_step(opf_handle* h, const double* x, const double* u, const double* lam, const double* y,
                    const double* sig_u, const double* sig_x, const double* sig_s, const double* rhs,
                    double delta_w, double delta_c, double* step, int* fail_col);

/* ---- the hybrid full-space solver (Sec. 4.3; Table 2's full-space IPM) --------- */
/* The comparison method of Sec. 4.3 solves the augmented system of
 * Eq. kktmatrix:normal directly (the paper pairs its GPU model with MA27 on the
 * CPU).  Here it is a GPU block LDL^T of the system with the slack step
 * eliminated,
 *   M = [[W + diag(Sigma_w) + delta_w E_u, G^T, A^T], [G, 0, 0],
 *        [A, 0, -(Sigma_s^{-1} + delta_c) I]]   over [p_w; p_lambda; p_y],
 * one dense diagonal block per bus (its unknowns with the multipliers of its
 * rows, so the state / balance-row pairs are pivoted together) and one per
 * flow-limit row, ordered by minimum degree; no pivoting across blocks.  The
 * plan is built on the first call (host), the factor lives in the handle.
 *
 * Assemble M at the last opf_eval_derivatives with Sigma (device, natural order:
 * sig_u[nu], sig_x[nx], sig_s[m]) and the regularisation delta_w (u block, the
 * placement of K_cond + delta_w I) and delta_c (inequality rows), factorise it,
 * and count its inertia from the diagonal blocks (Sylvester's law; host
 * inertia[3] = (n+, n-, n0), may be NULL).  Returns OPF_OK when the inertia is
 * (nu + nx, nx + m, 0) -- by Theorem 3 exactly when K_cond + delta_w I is
 * positive definite --, NOT_PD when it is not (the factor is kept and can still
 * solve), SINGULAR when a diagonal block is singular, TIMEOUT.  The condensed
 * state of the handle is dropped (opf_kkt_solve needs a new opf_condense).
 * Errors also: INVALID_ARG (no evaluation, NULL Sigma, negative delta). */
int opf_fullspace_factor(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s,
                         double delta_w, double delta_c, int* inertia);
/* Solve K_aug p = -r with that factor for nrhs right-hand sides, same device
 * layout as opf_kkt_solve ([r_u | r_x | r_s | r_lambda | r_y] in,
 * [p_u | p_x | p_s | p_lambda | p_y] out), then up to `refine` corrections of
 * iterative refinement against the full K_aug (0: the plain solve).  Host
 * outputs (may be NULL): *steps the corrections taken, *residual the final
 * relative max-norm residual (0 when refine = 0).  Errors: INVALID_ARG (no
 * factor), TIMEOUT, CUDA, OOM. */
int opf_fullspace_solve(opf_handle* h, const double* rhs, double* step, int nrhs, int refine, int* steps,
                        double* residual);
/* Statistics (host outputs, may be NULL): diagonal blocks, levels of the block
 * elimination tree, scalar entries of the strict block lower factor,
 * multiply-adds of one factorisation, log|det M| and the inertia of the last
 * factorisation (0 and -1 before one).  Builds the plan if needed. */
int opf_fullspace_stats(opf_handle* h, int* nblocks, int* levels, long long* nnz_l, long long* flops,
                        double* logabsdet, int* inertia);
/* Launch shapes of the block factorisation and solves (host outputs, may be
 * NULL): grids[2] = CTAs of the factorisation and of the solves (cooperative
 * grids; fewer resident warps poll the dependency flags less), ms[8] = the
 * timings of the first factorisation and the first solve at 1, 2, 4 and 8 CTAs
 * per SM (0 = not tried).  INVALID_ARG before the plan exists. */
int opf_fullspace_tuning(const opf_handle* h, int* grids, float* ms);

/* ---- A11: reduce-then-linearize helpers (Algorithm 2, Sec. 4.4) -------------- */
/* Newton-Raphson on g(x, u) = 0 for x at fixed u (device u[nu]; device x[nx]
 * in: start, out: solution) to ||g||_inf <= tol.  Errors: PF_FAILED. */
int opf_powerflow(opf_handle* h, const double* u, double* x, double tol, int max_iter,
                  int* iters);
/* Reduced gradient of Eq. reduced:derivatives (Sec. 2.3) and the adjoint step of
 * Algorithm 2, with the G_x factor of the last refactorisation (opf_gx_factor,
 * opf_condense or opf_powerflow's last Newton step at the same point):
 *   lam = -G_x^{-T} grad_x,   grad_r = grad_u + G_u^T lam.
 * grad[nu+nx] = [grad_u; grad_x] (device) is any gradient over w = [u; x]: grad f
 * gives grad f_r, grad_w (f + y^T h) the reduced Lagrangian gradient; NULL takes
 * grad f of the last opf_eval_derivatives.  Outputs (device): grad_r[nu], and
 * lam[nx] when non-NULL.  One G_x^{-T} solve; synchronises the handle's stream.
 * Errors: INVALID_ARG (no factor of G_x at the last evaluation, NULL grad_r),
 * CUDA, OOM. */
int opf_reduced_gradient(opf_handle* h, const double* grad, double* grad_r, double* lam);

/* ---- the interior-point loop (Algorithms 1 and 2; Sec. 4.3, 4.4) --------------- */
#define OPF_LINRED 0   /* linearize-then-reduce (Algorithm 1) */
#define OPF_REDLIN 1   /* reduce-then-linearize (Algorithm 2) */

typedef struct opf_ipm_options {
    int variant;       /* OPF_LINRED or OPF_REDLIN                                  */
    double tol;        /* scaled optimality error to stop at (paper: 1e-8)          */
    int max_iter;      /* iteration cap                                             */
    double mu0;        /* initial barrier parameter                                 */
    double pf_tol;     /* Newton-Raphson tolerance of the RedLin projection (1e-10) */
    int verbose;       /* print one line per iteration to stdout                    */
    int line_search;   /* OPF_LINESEARCH_MERIT: backtracking on the l1 exact-penalty
                          merit function; OPF_LINESEARCH_FILTER (LinRed only): the
                          filter line search with second-order corrections of
                          Wachter and Biegler (2006), the Ipopt algorithm Sec. 4.3
                          defers to (no restoration phase: when the step length
                          runs out, a larger primal regularisation shortens the
                          step)                                                   */
    int restoration;   /* filter line search only: 1 = when the step length runs out,
                          the feasibility restoration phase of Wachter and Biegler
                          (2006, Sec. 3.3) with the relaxation on the inequality
                          rows only (Sec. 4.3: there it is a dual regularisation
                          of the inequality rows, so the condensation on G_x is
                          unchanged); 0 = a larger primal regularisation
                          shortens the step instead                             */
    int start_with_resto; /* with restoration: run the phase once from the starting
                          point before the first step (Ipopt's option of that name) */
    int linear_solver; /* OPF_LINSOLVE_CONDENSED: the condensed step (LinRed, RedLin);
                          OPF_LINSOLVE_FULLSPACE (LinRed only): the hybrid
                          full-space IPM of Sec. 4.3 -- the same loop, model,
                          derivatives and regularisation, each step from
                          opf_fullspace_factor / opf_fullspace_solve (the inertia
                          test of the block factor in place of the Cholesky test,
                          equivalent by Theorem 3)                                 */
} opf_ipm_options;
#define OPF_LINSOLVE_CONDENSED 0
#define OPF_LINSOLVE_FULLSPACE 1
#define OPF_LINESEARCH_MERIT  0
#define OPF_LINESEARCH_FILTER 1

typedef struct opf_ipm_result {
    int status;        /* OPF_OK, OPF_ERR_NO_CONVERGENCE, or the failing call's code */
    int iters;
    double obj, err, mu;
    int n_factor;      /* Cholesky attempts (inertia correction included)          */
    double ms_total, ms_eval, ms_condense, ms_factor, ms_solve, ms_linesearch, ms_pf;  /* host wall */
    int graph_iters;   /* iterations whose condensation + first Cholesky attempt ran as
                          a replayed CUDA graph (needs a non-default stream)           */
    int soc_steps;     /* accepted second-order corrections (filter line search)      */
    int restorations;  /* feasibility restoration phases entered                      */
    int resto_iters;   /* iterations spent inside them                                 */
} opf_ipm_result;

/* Solve the OPF of the handle's network from the flat start (theta = 0, Vm = 1 at
 * load buses and 1.05 at generator buses, Pg at mid-range, y0 = 0).  The loop's
 * scalar and vector bookkeeping runs on the host; every model evaluation,
 * refactorisation, condensation, Cholesky factorisation, step recovery and power
 * flow runs on the device (opt may be NULL: LinRed, tol 1e-8, 300 iterations,
 * mu0 0.1, pf_tol 1e-10).  Returns res->status. */
int opf_solve(opf_handle* h, const opf_ipm_options* opt, opf_ipm_result* res);
/* The last solve's point (host outputs, any may be NULL): w[nu+nx] = [u; x],
 * lam[nx], y[m], Pg[ng] (every generator, slack included). */
int opf_get_solution(const opf_handle* h, double* w, double* lam, double* y, double* Pg);

/* ---- A13: derivative of the optimal dispatch with respect to the bus loads ------ */
/* The paper stops at the Newton step; this extension reuses its recoveries
 * (Theorems 1 and 2, Sec. 3.3) for the implicit-function derivative of the
 * barrier solution F(xi; d) = 0 at fixed mu (bound multipliers eliminated into
 * Sigma), d = (Pd, Qd):
 *   dPg/dd = dPg/dd|direct - J_out K_aug^{-1} dF/dd,   J_out = dPg/dxi,
 * with K_aug of Eq. kktmatrix:normal at the point, delta_w = delta_c = 0. */

/* Replace the bus loads Pd[nb], Qd[nb] (host, p.u.) used by every later
 * evaluation and solve; the library copies them.  Drops the factors and the
 * stored solution.  Errors: INVALID_ARG (NULL or non-finite entry). */
int opf_set_loads(opf_handle* h, const double* Pd, const double* Qd);

/* Build K_aug at a barrier KKT point and factor it for opf_dispatch_vjp:
 * evaluates the derivatives at (w, lam, y), refactors G_x, condenses with
 * (sig_w, sig_s) and factors Kred with delta_w = 0.  Host arrays, natural
 * order: w[nw] = [u; x], lam[nx], y[m], sig_w[nw] = [Sigma_u; Sigma_x], sig_s[m].
 * All five NULL: the last successful opf_solve's solution, first moved onto the
 * barrier solution at its final mu by Newton's method at that fixed mu (the IPM
 * stops at its tolerance, short of that point; full steps cut by the
 * fraction-to-the-boundary rule, refined K_aug solves, residual <= 1e-12 or
 * until it stops falling; on failure the IPM's point is kept).  A RedLin
 * solution is used in its full-space form: the state-bound rows' slacks and
 * multipliers become the bounds of x.  Any later evaluate / condense / factor
 * call drops the preparation.
 * Errors: INVALID_ARG (no stored solution, or some but not all pointers NULL),
 * NOT_PD (Kred not positive definite at the point: K_aug has the wrong inertia,
 * Theorem 3, and the derivative of the barrier solution is not defined there),
 * SINGULAR, CUDA, TIMEOUT. */
int opf_vjp_prepare(opf_handle* h, const double* w, const double* lam, const double* y,
                    const double* sig_w, const double* sig_s);

/* Vector-Jacobian products of the optimal dispatch Pg[ng] (every generator,
 * slack included; generator 0 is the slack) for k cotangents:
 *   grad_Pd[j][i] = sum_g vbar[j][g] dPg_g/dPd_i,  grad_Qd likewise.
 * Device arrays, row-major: vbar[k][ng] in, grad_Pd[k][nb] and grad_Qd[k][nb]
 * out (caller-owned; may not overlap vbar).  zeta = K_aug^{-1} J_out^T vbar comes
 * from the condensed solve (one Cholesky solve with Kred and three multi-RHS
 * solves with G_x, all k at once), then iterative refinement against the full
 * sparse K_aug (each correction: one Cholesky and four G_x solves) until the
 * residual reaches rounding level or stops falling, at most 4 corrections: at
 * a converged point Sigma spans many orders of magnitude and Kred's condition
 * number grows like 1/mu.  Synchronises the handle's stream.
 * Errors: INVALID_ARG (not prepared, k < 0, NULL with k > 0), CUDA, OOM, TIMEOUT. */
int opf_dispatch_vjp(opf_handle* h, const double* vbar, int k, double* grad_Pd, double* grad_Qd);
/* Refinement corrections taken by the last opf_dispatch_vjp and its final
 * residual max|b - K_aug zeta| / max|b|; Newton iterations of the last polish of
 * the stored solution (-1: it failed) and its final barrier KKT residual.
 * Outputs may be NULL. */
int opf_vjp_info(const opf_handle* h, int* refine_steps, double* rel_residual, int* polish_iters,
                 double* kkt_residual);

/* ---- A12: many instances at once ------------------------------------------------ */
/* A batch runs the interior-point loops of n independent handles concurrently
 * on the current device: each handle gets its own non-blocking stream (its
 * previous stream comes back at opf_batch_destroy), and nthreads host threads
 * (0 = one per hardware thread, at most 32; never more than n) take instances
 * from a queue, largest first, each thread driving one loop at a time.  Kernels
 * of different instances overlap on the SMs and one instance's host work hides
 * behind the others' device work.  Every handle's loop scratch is allocated at
 * creation, so nothing is allocated or freed while the batch solves.  The
 * handles stay owned by the caller, must be distinct, and must not be used
 * outside the batch while it lives.  Errors: INVALID_ARG, CUDA, OOM. */
typedef struct opf_batch opf_batch;
int opf_batch_create(opf_handle* const* handles, int n, int nthreads, opf_batch** out);
void opf_batch_destroy(opf_batch* b);
/* Number of instances and host threads (outputs may be NULL). */
int opf_batch_size(const opf_batch* b, int* n, int* nthreads);
/* Pick every instance's multi-RHS solve kernel now, one instance at a time with
 * the GPU to itself (at the flat start; see opf_options.rhs_block); handles
 * whose kernel is already chosen are skipped. */
int opf_batch_autotune(opf_batch* b);
/* opf_solve of every instance with the same options (opt may be NULL),
 * concurrently; results[n] receives each instance's result and *wall_ms (may be
 * NULL) the host wall time of the whole batch.  Returns OPF_OK when every
 * instance converged, else the first failing instance's code (errors before
 * OPF_ERR_NO_CONVERGENCE). */
int opf_batch_solve(opf_batch* b, const opf_ipm_options* opt, opf_ipm_result* results, double* wall_ms);
/* How opf_batch_solve runs the loops.
 *  OPF_BATCH_LOCKSTEP (the default): one host thread per instance; at every
 *    iteration the loops meet at the condensation, and one
 *    opf_batch_condense_factor call (one launch per phase for all of them)
 *    serves every instance still iterating -- instances that have converged or
 *    stopped are masked on the device.  The rest of each iteration (derivatives,
 *    step recovery, line search, inertia correction after NOT_PD) stays on the
 *    instance's own stream.  Needs the adjoint route on every handle.
 *  OPF_BATCH_CONCURRENT: nthreads host threads take instances from a queue, each
 *    loop independent on its own stream (kernels of different instances
 *    overlap on the SMs).
 * Errors: INVALID_ARG. */
#define OPF_BATCH_CONCURRENT 0
#define OPF_BATCH_LOCKSTEP   1
int opf_batch_set_mode(opf_batch* b, int mode);
/* Batched condensations issued by lockstep solves since the batch was created;
 * the cluster sizes (CTAs) of the batched multi-RHS solves and Cholesky (0 until
 * the first opf_batch_condense_factor whose instances all factored completely
 * timed the candidates 2, 4, 8, 16); tune_ms[8] those timings (solve, then
 * Cholesky; 0 = not tried); graph_calls: calls served by replaying the captured
 * CUDA graph of the whole batched sequence (descriptor upload, every phase,
 * the status read-back), which every call after the tuning one uses.  Host
 * outputs, any may be NULL. */
int opf_batch_stats(const opf_batch* b, long long* lockstep_calls, int* trsm_cl, int* chol_cl, float* tune_ms,
                    long long* graph_calls);

/* One interior-point iteration's condensation and control-step factorisation
 * (A5-A9: refactor G_x, S_x, K, H = K Z, Psi, Kred, Cholesky of Kred + delta_w I)
 * for every instance of the batch at once, one kernel launch per phase over
 * device work lists: the refactorisations are one cooperative launch over the
 * merged row list (instance, row) in level order; the multi-RHS solves one
 * launch of one CTA per (instance, 32-column block); the products one launch
 * per shape with a block range per instance; the factorisations one launch of
 * one thread-block cluster (8 CTAs) per instance.  Each instance must have been
 * evaluated (opf_eval_derivatives with lam and y) at its point, and use the
 * adjoint route.  sig_u[n], sig_x[n], sig_s[n] are host arrays of device
 * pointers (each instance's Sigma, as in opf_condense); delta_w[n] a host array
 * (NULL: 0 for all).  The launches wait for the work already on every
 * instance's stream and every instance's later work waits for them; the call
 * returns once the factorisations are done.  Outputs (host): status[n] per
 * instance (OPF_OK, NOT_PD, SINGULAR, TIMEOUT) and, when fail_col is non-NULL,
 * fail_col[n] (the first failing column of a NOT_PD instance, else -1).  Each
 * handle is left as after opf_condense + opf_kkt_factor with its delta_w: its
 * Kred, factor and opf_kkt_solve are available (after NOT_PD, opf_kkt_factor
 * with a larger delta_w retries on that handle alone).  The first call builds
 * the work lists.  Returns OPF_OK, or the first instance's failure code.
 * Errors: INVALID_ARG (an instance not evaluated, on the explicit route, or a
 * NULL pointer), CUDA, OOM. */
int opf_batch_condense_factor(opf_batch* b, const double* const* sig_u, const double* const* sig_x,
                              const double* const* sig_s, const double* delta_w, int* status, int* fail_col);

/* ---- dense Cholesky without device allocation ----------------------------------- */
/* The paper has no counterpart to this call.  It serves callers that cannot
 * allocate device memory where they need a factorisation -- a loop running under
 * a fixed memory budget, an application whose device memory is all held by its
 * own pool allocator, a real-time loop that forbids allocation after set-up.
 * It factors A + delta_w I = L L^T for a caller-owned device matrix A (n x n,
 * row-major, only the lower triangle read) into the caller-owned device buffer L
 * (lower triangle; upper part set to zero), on the given stream (a cudaStream_t,
 * NULL = legacy default stream), and returns after the stream synchronises.
 *  - No cudaMalloc / cudaFree and no allocating library routine is called.  The
 *    scratch (status word, grid-barrier state, inverse diagonal) is a file-scope
 *    device array sized for n <= 4096 (about 32 KB), held by every GPU that loads
 *    the library until the process exits; larger n is rejected with INVALID_ARG.
 *  - The first call on a device looks that array's address up on the current
 *    device (once per device).  Every call ends by synchronising the stream, so
 *    the call cannot be used inside a stream capture.
 *  - Every call shares the one array per device: calls whose GPU work overlaps
 *    (two streams, two host threads) race; serialise them.
 * Errors: INVALID_ARG, CUDA, NOT_PD (*fail_col = first failing column), TIMEOUT. */
int opf_chol_noalloc(const double* A, int n, double delta_w, double* L, int* fail_col, void* stream);

/* ---- instrumentation ---------------------------------------------------------- */
/* The CUDA error of the last runtime call that made any call of this library
 * return OPF_ERR_CUDA (any thread; 0 if none), and its name into name[len]
 * (may be NULL). */
int opf_last_cuda_error(char* name, int len);
/* Kernel launches this library has enqueued since it was loaded (all handles). */
unsigned long long opf_launch_count(void);
/* Measured FP64 throughput of the current device in GFLOP/s (host output), the
 * roofline denominator of this library's FP64 kernels: which = 0 DFMA (fma
 * chains on every FP64 pipe of a full grid), 1 / 2 / 3 the warp-level f64
 * tensor-core path mma.sync m8n8k4 / m16n8k4 / m16n8k16 (four accumulators per
 * warp).  Best of two timed launches on the legacy default stream; allocates
 * and frees a small output buffer; synchronises the device.  The paper has no
 * counterpart (it reports no roofline).  Errors: INVALID_ARG, CUDA, OOM. */
int opf_fp64_peak(int which, double* gflops);

/* Phase timing.  While enabled, CUDA events on the handle's stream bracket every
 * launch of each phase of opf_condense / opf_kkt_factor / opf_kkt_solve; opf_phase_times
 * synchronises the stream and returns, per phase, the accumulated milliseconds
 * (ms[OPF_PHASE_COUNT]) and the number of bracketed launches.  Enabling resets
 * the accumulators. */
#define OPF_PHASE_REFACTOR 0   /* G_x scatter, numeric LU, factor gathers       */
#define OPF_PHASE_ASSEMBLE 1   /* K = W + Sigma + A^T Sigma_s A                 */
#define OPF_PHASE_TRSM     2   /* each multi-RHS triangular solve launch         */
#define OPF_PHASE_SPMM     3   /* H = K Z                                        */
#define OPF_PHASE_KRED     4   /* H_u - G_u^T Psi (or S_x^T H_x), symmetrise     */
#define OPF_PHASE_CHOL     5   /* Cholesky of Kred + delta_w I                   */
#define OPF_PHASE_RHS      6   /* condensed right-hand side of opf_kkt_solve     */
#define OPF_PHASE_RECOVER  7   /* its Cholesky solve and step recovery           */
#define OPF_PHASE_COUNT    8
int opf_profile(opf_handle* h, int enable);
int opf_phase_times(opf_handle* h, double* ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* CONDIPM_H */
