// Host-side symbolic analysis of a network: variable layout, fixed sparsity
// patterns, deterministic gather plans for the derivative kernels, the
// fill-reducing ordering and symbolic LU of G_x, and triangular-solve level
// schedules.  Everything here is computed once per network (the pattern of
// G_x is fixed by the network topology, Sec. 3.2) and uploaded by opf_create.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace condipm {

// val[p] = cst[p] + sum_{q in [ptr[p], ptr[p+1])} src[idx[q]]
struct Gather {
  std::vector<int> ptr, idx;
  std::vector<double> cst;
};

// val[p] += sum_q coef[r[q]] * A[a[q]] * A[b[q]]
struct Bilin {
  std::vector<int> ptr, r, a, b;
};

struct CSR {
  int nrows = 0, ncols = 0;
  std::vector<int> rp, ci;
  long long nnz() const { return rp.empty() ? 0 : rp.back(); }
};

struct Levels {
  int nlev = 0;
  std::vector<int> ptr, rows;  // rows grouped by level, ascending within a level
};

struct Plan {
  // ---- sizes
  int nb = 0, nl = 0, ng = 0, slack = 0, nx = 0, nu = 0, nw = 0, m = 0, nlim = 0, ne = 0;
  // ---- network copy
  std::vector<double> Pd, Qd, Vmin, Vmax, r, x, b, rate, Pmin, Pmax, Qmin, Qmax, c2, c1;
  std::vector<int> lf, lt, gbus;
  // ---- layout (w = [u; x], c = [u; x permuted])
  std::vector<int> th_w;       // [nb] w-index of theta_i, -1 for the slack
  std::vector<int> vm_w;       // [nb] w-index of Vm_i
  std::vector<int> pg_w;       // [ng] w-index of Pg_k, -1 for generator 0
  std::vector<int> gen_of_bus; // [nb] generator at bus or -1
  std::vector<int> w2c;        // [nw] w-index -> c-index
  std::vector<int> c2w;        // [nw]
  std::vector<int> perm;       // [nx] perm[k] = x-index eliminated k-th
  std::vector<int> iperm;      // [nx] x-index -> position
  // bounds of w and of h (+-inf encoded as +-1e300)
  std::vector<double> wl, wu, hl, hu;
  // ---- line ends: e < nl: (lf, lt); e >= nl: (lt, lf)
  std::vector<int> end_i, end_k, end_w;  // end_w: 4 per end (theta_i, theta_k, Vm_i, Vm_k)
  std::vector<int> end_h;                // h-row of the limited end or -1
  std::vector<double> gs, bs, gm, bm;    // self / mutual admittance per end
  std::vector<int> bus_end_ptr, bus_end; // ends leaving each bus, ascending end index
  std::vector<int> g_row_P, g_row_Q;     // [nb] g-row of P_i / Q_i balance or -1
  // ---- G (nx x nw, natural rows/cols) and A (m x nw)
  CSR G, A;
  Gather Ggat;   // src = [dp(4 ne) | dq(4 ne)]
  Gather Agat;   // src = [dp(4 ne) | dq(4 ne) | dS(4 ne)]
  std::vector<int> A_ci_c;  // A column indices in c-order
  // ---- K pattern (c-order rows and cols); W is stored in the same pattern
  CSR K;
  Gather Wgat;                 // src = Hw (10 per end)
  std::vector<int> Wslack_pos, Wslack_a, Wslack_b;   // + 2 c2_0 A[a] A[b]
  std::vector<int> K_diag;     // [nw] position of (c, c)
  Bilin KAA;                   // A^T Sigma_s A terms
  std::vector<int> Knat_rp, Knat_ci, Knat_map;   // natural-order view: map[p_nat] = p_c
  // ---- transposes used in the condense / solve
  CSR AT;                      // nw (c-order rows) x m
  std::vector<int> AT_map;     // AT value q = A value AT_map[q]
  CSR PGu;                     // nx (perm rows) x nu : P G_u
  std::vector<int> PGu_map;    // value map into G
  CSR GuT;                     // nu x nx (perm cols) : (P G_u)^T
  std::vector<int> GuT_map;
  // ---- LU of P G_x P^T (perm space)
  CSR LU;                      // combined rows: L part (cols < i), diag, U part (cols > i)
  std::vector<int> LU_diag;    // position of (i, i)
  std::vector<int> Gx_to_LU;   // [nnz(G)] LU position of a G_x entry, -1 for G_u entries
  std::vector<long long> upd_ptr;  // [nnz(LU)+1] start of the update map of an L entry
  std::vector<int> upd_pos;        // LU positions updated by l_ik * u_kj
  CSR Lo;                      // strict lower pattern (perm space)
  std::vector<int> Lo_map;     // L values  -> LU positions
  std::vector<int> Ut_map;     // U^T values (strict lower pattern) -> LU positions
  CSR Up;                      // strict upper pattern
  std::vector<int> Up_map;     // U values
  std::vector<int> Lt_map;     // L^T values (strict upper pattern)
  Levels fwd, bwd;             // level schedules of the lower / upper solves
  long long lu_flops = 0;      // multiply-adds of one numeric refactorisation
};

// Builds the plan; returns an empty string on success, else the reason.
std::string build_plan(Plan& P, int nb, int nl, int ng, int slack, const double* Pd,
                       const double* Qd, const double* Vmin, const double* Vmax,
                       const int* lf, const int* lt, const double* r, const double* x,
                       const double* b, const double* rate, const int* gbus,
                       const double* Pmin, const double* Pmax, const double* Qmin,
                       const double* Qmax, const double* c2, const double* c1);

}  // namespace condipm
