// Internal state behind the opaque opf_handle of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/condipm.h"
#include "common.cuh"
#include "plan.h"

struct opf_batch;
namespace condipm {
struct FsState;
}

struct opf_handle {
  condipm::Plan P;
  opf_options opt{};
  cudaStream_t s = nullptr;
  long long spin_limit = 1LL << 26;
  std::vector<void*> allocs;
  // topology / network (device)
  int *end_i = nullptr, *end_k = nullptr, *end_h = nullptr, *bus_end_ptr = nullptr, *bus_end = nullptr;
  int *g_row_P = nullptr, *g_row_Q = nullptr, *gen_of_bus = nullptr, *th_w = nullptr, *vm_w = nullptr;
  int *pg_of_w = nullptr, *slackpos = nullptr;
  double *gs = nullptr, *bs = nullptr, *gm = nullptr, *bm = nullptr, *Pd = nullptr, *Qd = nullptr;
  double *c2 = nullptr, *c1 = nullptr;
  // model evaluation
  double *Vm = nullptr, *Va = nullptr, *pq = nullptr, *dsrc = nullptr, *hpq = nullptr, *hw = nullptr;
  double *wP = nullptr, *wQ = nullptr, *g = nullptr, *hv = nullptr, *f = nullptr, *gradf = nullptr;
  double *Pg = nullptr;
  // G, A
  int *Ggat_ptr = nullptr, *Ggat_idx = nullptr;
  double *Ggat_cst = nullptr, *Gval = nullptr;
  int *Agat_ptr = nullptr, *Agat_idx = nullptr, *A_rp = nullptr, *A_ci_c = nullptr;
  double *Agat_cst = nullptr, *Aval = nullptr;
  // K and W (c-order pattern)
  int *K_rp = nullptr, *K_ci = nullptr, *Wgat_ptr = nullptr, *Wgat_idx = nullptr;
  int *Wsl_pos = nullptr, *Wsl_a = nullptr, *Wsl_b = nullptr, *K_diag = nullptr;
  int *KAA_ptr = nullptr, *KAA_r = nullptr, *KAA_a = nullptr, *KAA_b = nullptr, *Knat_map = nullptr;
  int *perm = nullptr, *c2w = nullptr;
  double *Wgat_cst = nullptr, *Wval = nullptr, *Kval = nullptr, *sig_c = nullptr, *sig_s = nullptr;
  // transposes
  int *AT_rp = nullptr, *AT_ci = nullptr, *AT_map = nullptr;
  int *PGu_rp = nullptr, *PGu_ci = nullptr, *PGu_map = nullptr;
  int *GuT_rp = nullptr, *GuT_ci = nullptr, *GuT_map = nullptr;
  int *Gc_rp = nullptr, *Gc_ci = nullptr, *Gc_map = nullptr;
  int *GcT_rp = nullptr, *GcT_ci = nullptr, *GcT_map = nullptr;
  int *GTn_rp = nullptr, *GTn_ci = nullptr, *GTn_map = nullptr;
  int *ATn_rp = nullptr, *ATn_ci = nullptr, *ATn_map = nullptr;
  // LU
  int *LU_rp = nullptr, *LU_ci = nullptr, *LU_diag = nullptr, *Gx_to_LU = nullptr, *upd_pos = nullptr;
  long long* upd_ptr = nullptr;
  double *LUval = nullptr, *inv_diag = nullptr, *rmax = nullptr;
  unsigned* flags = nullptr;
  unsigned epoch = 0;
  int *Lo_rp = nullptr, *Lo_ci = nullptr, *Lo_map = nullptr, *Ut_map = nullptr;
  int *Up_rp = nullptr, *Up_ci = nullptr, *Up_map = nullptr, *Lt_map = nullptr;
  double *Lo_val = nullptr, *Ut_val = nullptr, *Up_val = nullptr, *Lt_val = nullptr;
  int *fwd_ptr = nullptr, *fwd_rows = nullptr, *bwd_ptr = nullptr, *bwd_rows = nullptr;
  // staged supernodal solves: structure per pattern (lower / upper), values per
  // factor (L and U^T on the lower structure, U and L^T on the upper one)
  struct StBuf {
    int nchunks = 0;
    long long* chunk_off = nullptr;
    int *chunk_bytes = nullptr, *chunk_big_f = nullptr, *chunk_big_w = nullptr, *int_beg = nullptr;
    long long* slot = nullptr;
    int* src = nullptr;
    long long nslots = 0;
    unsigned char *bytes_a = nullptr, *bytes_b = nullptr;
  } stLo, stUp;
  int st_cap = 0;
  condipm::ColDev csL{}, csU{};  // column-parallel schedules
  double* cs_scratch = nullptr;  // segment partial sums, ncb_max * maxseg * 32
  unsigned* cs_bar = nullptr;    // per column-block barrier counters
  int cs_ncb_max = 0, cs_ksplit_max = 1;
  int ldp = 32;                  // leading dimension of Zt / H (nu rounded up to 32)
  int sn_cb = 0;                 // columns per CTA of the staged solves (0 = level fallback)
  int trsm_mode = -1;            // multi-RHS solve kernel: -1 autotune, 32 column-parallel,
                                 // 1/2/4 staged with that many columns per CTA
  float tune_ms[3][10] = {};     // autotuner timings per role: multi-RHS {cols, staged 1, 2, 4, blocked,
                                 // dataflow}; one RHS {staged, blocked x 4 grids, one-CTA x 2, cluster x 3}
  int trsm_mode1 = -1;           // kernel of the solves with fewer than 32 right-hand sides
                                 // (-1 autotune, 1 staged, 64 level-blocked)
  condipm::BlkDev bkL{}, bkU{};  // level-blocked schedules of the lower / upper solves
  double rch_work[2] = {};         // forward sweep on P G_u: multiply-adds of the reach lists / of all rows
  double *D_L = nullptr, *D_Ut = nullptr, *D_U = nullptr, *D_Lt = nullptr;  // diagonal-block inverses
  double* ybuf = nullptr;        // level-blocked solve scratch (rows x leading dimension)
  size_t ybuf_cap = 0;
  int blk_max = 1;               // resident CTAs of the level-blocked kernel
  int blk_ksplit = 0;            // its CTAs per 32-column block (0: as many as fit, at most 16)
  int blk_cl = 0;                // > 0: instead, one thread-block cluster of that many CTAs per block
  int blk_minb_i = 0;            // register-bound variant of the level-blocked kernel (index into BLK_MINB)
  int blk_max_minb[3] = {1, 1, 1};  // resident CTAs of each variant
  int blk1_blocks = 32;          // CTAs of the single-right-hand-side level-blocked solve
  condipm::Lu1sDev l1L{}, l1U{}; // the one-CTA single-right-hand-side solve's schedules
  int lu1s_ymax = 0;             // rows of the largest level (the one-CTA solve's Y buffer)
  bool lu1s_ok = false;          // the one-CTA solve's vector and Y fit in shared memory
  int lu1s_g = 8;                // its lanes per row
  condipm::Cl1Dev cl1L[3]{}, cl1U[3]{};   // cluster one-RHS schedules for 4, 8, 16 CTAs
  bool cl1_ok[3] = {false, false, false};  // ... and whether each fits on the device
  int cl1_pick = 2;              // the cluster size in use (index)
  condipm::DfDev dfL{}, dfU{};   // dataflow task lists of the lower / upper solves
  double* df_part = nullptr;     // partial sums of their chunk tasks (chunks x 32 column blocks)
  unsigned* df_cnt = nullptr;    // their supernode counters (2 x column blocks x supernodes)
  int df_max = 1, df_ksplit = 0; // resident CTAs of the dataflow kernel; CTAs per column block
  // dense condensed buffers: Zt = [I; S_x] and H = K Zt (nw x nu, row-major, x rows permuted),
  // Kred (nu x nu, symmetric) and its Cholesky factor F
  double *Zt = nullptr, *H = nullptr, *Kred = nullptr, *F = nullptr, *Fdinv = nullptr;
  // device status word and grid-barrier state
  int* st = nullptr;
  unsigned* bar = nullptr;
  // growable workspace for solves
  double* ws = nullptr;
  size_t ws_cap = 0;
  // launch shapes
  int lu_blocks = 1, lu_threads = 256, lu_maxlen = 1, chol_blocks = 1, cb = 1;
  bool chol_tuned = false;       // Cholesky form and grid size picked by timing (first factorisation)
  int chol_df = 0, chol_np = 0;  // dataflow form (1) and its panel CTAs
  double* Finv = nullptr;        // inverses of the factor's 32 x 32 diagonal tiles (few-RHS solves)
  bool finv_valid = false;       // Finv belongs to the current factor
  int chol_solve_cl = 0;         // cluster size of the few-RHS solve (0: one CTA per column)
  bool cs_tuned = false;         // ... timed at 4, 8, 16 CTAs on the first one-vector solve
  float cs_ms[3] = {};
  double* cs_tmp = nullptr;      // its copy of the right-hand side (nu; in allocs)
  float chol_ms[OPF_CHOL_CANDIDATES] = {};   // tuner timings
  unsigned* chol_cnt = nullptr;  // its step counters (3 x tile columns)
  // condensation + first Cholesky attempt of the interior-point loop as a CUDA
  // graph (inputs in the loop's fixed device buffers)
  cudaGraphExec_t cf_exec = nullptr;
  bool cf_failed = false;        // capture or instantiation was refused: plain launches
  bool cf_rhs = false;           // the captured condensation carries the step's right-hand side
  bool use_graphs = true;
  // condensation route in use: the option, or with OPF_ROUTE_AUTO the faster one
  // on the first condensation (-1 until then), and the two timings
  int route = -1;
  float route_ms[2] = {0.f, 0.f};
  // right-hand sides per pass of the condensation (adjoint route): the option,
  // or the autotuner's pick on the first condensation (0 until then)
  int rhs_width = 0;
  float width_ms[4] = {};
  bool psi_last_adjoint = false;   // the last condensation ended with the adjoint route's Psi
  // set while a lockstep batch solve runs this handle's loop: its condensation
  // and first Cholesky attempt go through the batch's rendezvous
  opf_batch* batch = nullptr;
  int batch_idx = -1;
  // call-order state
  bool have_eval = false, have_W = false, have_lu = false, have_condense = false, have_factor = false;
  bool psi_valid = false;         // Zt holds S_x and H's x rows G_x^{-T} H_x of the last condensation
  // the right-hand side condensed with the last condensation (one extra column
  // of S_x, H and Psi): its KB copy, b_t = b_w + A^T (Sigma_s b_y - b_s), and
  // whether column nu of Zt / H holds q, e - K [0; q] -> (r_hat; phi) for it
  double* fr_kb = nullptr;       // kkt_rows doubles (in allocs)
  double* fr_bt = nullptr;       // nw (in allocs)
  bool fr_have_b = false, fr_ready = false;
  double delta_w = 0.0;
  // dual regularisation of the inequality rows folded into K, H and Kred
  // (-delta_c I in the (p_y, p_y) block of K_aug); 0 after every condensation
  double delta_c = 0.0;
  double* sig_se = nullptr;      // Sigma_s / (1 + delta_c Sigma_s) (m)
  double* ps_sc = nullptr;       // 1 / (1 + delta_c Sigma_s) (m)
  double* pf_ws = nullptr;       // power-flow step and norm (nx + 1)
  double* ipm_buf = nullptr;     // interior-point loop scratch (in allocs)
  double* resto_w0 = nullptr;    // restoration phase: W at zero multipliers (K pattern; in allocs)
  // converged state of the last opf_solve (host), full-space form
  bool have_solution = false;
  std::vector<double> sol_w, sol_lam, sol_y, sol_s, sol_sig_w, sol_sig_s;
  std::vector<double> sol_zwl, sol_zwu, sol_zsl, sol_zsu;   // bound multipliers (full-space form)
  double sol_mu = 0.0, sol_pg0 = 0.0;
  bool polished = false;         // stored solution already moved onto the barrier solution
  int polish_iters = 0;          // fixed-mu Newton iterations of the last polish (-1: failed)
  double polish_res = 0.0;       // its final barrier KKT residual (max-norm)
  bool sens_ready = false;       // K_aug at the solution factored for opf_dispatch_vjp
  double* sens_buf = nullptr;    // dispatch derivative: point, Sigma and a_0 (in allocs)
  int vjp_steps = 0;             // refinement steps and relative residual of the last VJP
  double vjp_res = 0.0;
  int vjp_max_refine = 4;
  int* sens_pq = nullptr;        // [2 nb] elimination position of P_i / Q_i rows, -1 if none (in allocs)
  // the hybrid full-space solver's plan, factor and buffers (built on first use)
  condipm::FsState* fs = nullptr;
  bool ipm_fs = false;           // the running interior-point loop is the hybrid full-space one
  bool ipm_verbose = false;      // ... and prints its progress
  // phase timing (opf_profile)
  bool profiling = false;
  struct PhaseRec { int phase; cudaEvent_t a, b; };
  std::vector<PhaseRec> recs;
  std::vector<cudaEvent_t> evpool;
  int open_phase = -1;
  cudaEvent_t open_ev = nullptr;
  double ph_ms[OPF_PHASE_COUNT] = {};
  long long ph_n[OPF_PHASE_COUNT] = {};
};
