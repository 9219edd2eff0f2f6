// Host-side symbolic analysis of the hybrid full-space system (Sec. 4.3): the
// augmented matrix with the slack step eliminated,
//
//   M = [[W + diag(Sigma_w) + delta_w E_u,  G^T,  A^T                        ],
//        [G,                                0,    0                          ],
//        [A,                                0,    -(Sigma_s^{-1} + delta_c) I]],
//
// unknowns [w; lambda; y] in natural order (w = [u; x] as in the plan, lambda
// over the rows of g, y over the rows of h), factorised as a block LDL^T:
// P M P^T = L D L^T with L block unit lower triangular and D block diagonal.
//
// Blocks.  Each bus is one block holding its unknowns and the multipliers of
// its rows: theta_i, Vm_i, Pg of its generator, the P and Q balance rows and
// the slack-Pg and Qg rows of h.  The state pairs (theta_i, P_i) and (Vm_i, Q_i)
// sit in one block, so the zero (p_lambda, p_lambda) diagonal is never a
// pivot of its own: the block pivot D_I is inverted as a whole (Gauss-Jordan
// with scaled partial pivoting inside the block).  Each flow-limit row of h is
// a block of its own.  The
// block graph is the bus graph (lines), the limit rows joined to both end
// buses, and a clique on the slack bus and its neighbours (the slack cost
// curvature 2 c2_0 grad P_s grad P_s^T couples them in W).  The flow-limit
// blocks come first (their pivots are then exactly -(Sigma_s^{-1} + delta_c):
// near the optimum an active limit has Sigma_s^{-1} close to 0, and a pivot
// formed later as a difference of Schur terms could lose its sign), then the
// buses by weighted minimum degree.
//
// Numeric form (GPU): a block LU without pivoting across blocks in the row
// (IKJ) form, with U = D L^T stored explicitly: for block row I and each L
// block (I, K) in ascending K, L_IK = W_IK D_K^{-1}, then W_IJ -= L_IK U_KJ
// for every U block (K, J) of row K.  D_I is what is left in the diagonal
// block; by Sylvester's law the inertia of M is the sum of the inertias of
// the D_I.
#pragma once
#include <string>
#include <vector>

#include "plan.h"

namespace condipm {

constexpr int FS_BMAX = 8;   // largest diagonal block

struct FsPlan {
  int n = 0;                  // unknowns of M: nw + nx + m
  int nblk = 0, bmax = 0, levels = 0;
  std::vector<int> bptr;      // [nblk+1] first position of each block (elimination order)
  std::vector<int> pos;       // [n] position of each natural unknown
  // block pattern, combined rows: L part (columns < I), diagonal, U part (> I)
  std::vector<int> brp, bci, bdiag;
  std::vector<long long> voff;   // [nnzb+1] offset of each block's values (row-major b_I x b_J)
  std::vector<long long> doff;   // [nblk+1] offset of each inverse diagonal block
  // update map of every L block q = (I, K): U blocks s = (K, J) of row K and
  // the block d = (I, J) of row I that L_IK U_KJ updates
  std::vector<long long> upd_ptr;  // [nnzb+1]
  std::vector<int> upd_src, upd_dst;
  std::vector<int> rows;      // block rows in level order (forward / factor schedule)
  std::vector<int> lvl_ptr;   // [levels+1] ranges of rows
  // assembly: value slot <- source entry
  std::vector<long long> w_slot;   // W: source = position in the plan's K pattern (c-order)
  std::vector<int> w_src;
  std::vector<long long> g_slot;   // G: source = entry of G (two slots per off-diagonal entry)
  std::vector<int> g_src;
  std::vector<long long> a_slot;   // A: source = entry of A
  std::vector<int> a_src;
  std::vector<long long> diag_slot;  // [n] slot of each natural unknown's diagonal entry
  long long nval = 0, ndinv = 0;
  long long nnz_l = 0;        // scalar entries of the strict block lower part
  long long flops = 0;        // multiply-adds of one numeric factorisation
};

// Builds the full-space plan from the network plan; empty string on success.
std::string build_fs_plan(const Plan& P, FsPlan& F);

}  // namespace condipm
