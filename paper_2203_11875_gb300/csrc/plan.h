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

// Supernodal schedule of one triangular solve (lower = forward, upper = backward).
// Supernodes are runs of consecutive rows whose diagonal block is dense; a row's
// entries split into "internal" ones (inside its supernode's diagonal block) and
// "external" ones (in supernodes solved at earlier levels).  Level 0 runs first.
struct SnSched {
  int nlev = 0;
  std::vector<int> lvl_ptr;   // [nlev+1] range of small supernodes (width <= 32)
  std::vector<int> lvl_gs;    // [nlev] lanes per small supernode (power of two <= 32)
  std::vector<int> lvl_wmax;  // [nlev] widest small supernode of the level
  std::vector<int> lvl_ga;    // [nlev] lanes per row for the external entries (0 = none)
  std::vector<int> lvl_rptr;  // [nlev+1] range of rows (small and big supernodes) in rows
  std::vector<int> rows;      // rows of each level, in level order
  std::vector<int> lvl_bptr;  // [nlev+1] range of big supernodes (width > 32)
  std::vector<int> sn_first, sn_w;    // small supernodes in level order
  std::vector<int> big_first, big_w;  // big supernodes in level order
  std::vector<int> ext_beg, ext_end, int_beg;  // [n] per row
};

// Byte stream of one supernodal triangular solve, cut into chunks that a CTA
// stages into shared memory one ahead of use.  A chunk holds complete
// supernodes of one level: their rows' external entries (phase A) and their
// packed dense diagonal triangles and diagonal inverses (phase B).  Chunk layout
// (byte offsets from the chunk start, every array 16-byte aligned):
//   int hdr[20] = {nA, nB, nE, nI, ga, gs, wmax, 0,
//                  oAptr, oArow, oEci, oEval, oBf, oBw, oBiptr, oBdptr, oIval, oBd, 0, 0}
//   int   Aptr[nA+1]  entry range of each row (chunk-relative)
//   int   Arow[nA]    row index
//   int   Eci[nE]     column of each external entry
//   double Eval[nE]   its value
//   int   Bf[nB], Bw[nB]        first row and width of each supernode
//   int   Biptr[nB+1], Bdptr[nB+1]   offsets into Ival and Bd
//   double Ival[nI]   dense triangles: lower row s holds columns 0..s-1 at s(s-1)/2;
//                     upper row s holds columns s+1..w-1 at s(w-1) - s(s-1)/2
//   double Bd[]       inverse diagonal of each row (1 for a unit diagonal)
// A "big" chunk (width > 32) carries no data: its rows' external entries sit in
// earlier chunks and its diagonal block is read from the factor in place.
struct SnStream {
  std::vector<unsigned char> bytes;   // structure with value slots left zero
  std::vector<long long> chunk_off;   // [nchunks] byte offsets (16-byte aligned)
  std::vector<int> chunk_bytes;       // [nchunks] sizes (multiples of 16)
  std::vector<int> chunk_big_f, chunk_big_w;  // -1 / 0 unless a big chunk
  // value slots: double index into bytes, and the factor position it takes
  // (>= 0: entry of the factor's strict part; -1: 1.0; -2 - i: inverse diagonal of row i)
  std::vector<long long> slot;
  std::vector<int> src;
  int max_chunk = 0;
};

// Schedule of the column-parallel triangular solve (one warp lane per right-hand
// side column): supernodes split to at most 32 rows, level-scheduled; rows whose
// external part is long are cut into segments whose partial dot products run
// on separate warps before the supernode sweep.
struct ColSched {
  int nlev = 0;
  int maxseg = 0;                      // most segments in one level
  std::vector<int> lvl_ptr;            // [nlev+1] supernodes of each level
  std::vector<int> sn_first, sn_w;     // level order, width <= 32
  std::vector<int> lvl_seg_ptr;        // [nlev+1] segments of each level
  std::vector<int> seg_q0, seg_q1;     // entry range of a segment
  std::vector<int> seg_row;            // >= 0: row the segment updates in place; < 0: -1 - scratch slot
  std::vector<int> row_seg;            // [n] first segment slot (level-relative) or -1
  std::vector<int> row_nseg;           // [n] segments in scratch (0: none, -1: applied in place)
  std::vector<int> ext_beg, ext_end, int_beg;  // [n]
};

// Cluster form of the one-right-hand-side level-blocked solve on CL CTAs.  In
// every level the supernodes are shared out over the CTAs by largest work
// first to the least loaded CTA; a CTA computes both phases of the supernodes
// it owns.  For CTA p and level l, entries t_ptr[p * (nlev + 1) + l] .. of
//   ta: {row, first and end external entry, Y slot of the row},
//   tb: {row, Y slot of the supernode's first row, width, offset of the row of
//        D_s};
// a supernode's rows are consecutive, so its Y is consecutive too.
struct ClSched {
  int CL = 0, nlev = 0, ymax = 0;
  std::vector<int> t_ptr;
  std::vector<int> ta, tb;   // 4 ints per row
};
std::string build_cl_sched(const ColSched& C, int CL, ClSched& S);


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
  CSR Gc, GcT;                 // P G (nx perm rows x nw c-order cols) and its transpose
  std::vector<int> Gc_map, GcT_map;
  CSR GTn, ATn;                // G^T (nw x nx) and A^T (nw x m), natural order
  std::vector<int> GTn_map, ATn_map;
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
  std::vector<int> sn_start;   // [nsn+1] fundamental supernodes (perm space)
  SnSched snL, snU;            // supernodal schedules of the lower / upper solves
  SnStream stL, stU;           // staged streams of the lower / upper solves (positions
                               // in the strict pattern: Lo for lower, Up for upper)
  ColSched csL, csU;           // column-parallel schedules of the lower / upper solves
  long long lu_flops = 0;      // multiply-adds of one numeric refactorisation
};

// Chunked stream of a supernodal schedule over strict pattern M (lower or
// upper), unit or non-unit diagonal, chunks of at most budget bytes.
void build_sn_stream(const CSR& M, const SnSched& S, const std::vector<int>& start, bool upper,
                     bool unit, int budget, SnStream& out);

// The forward sweep L Y = P G_u, one 32-column block of G_u at a time (the
// nu / 32 full blocks): the rows where Y can be nonzero in a block's columns
// are the rows of P G_u's pattern there and every row with an L entry in a
// column already reached (the union of the etree paths from those rows up);
// every other row of Y is exactly zero and the solve can pass it by.  Per
// block, the positions of those rows in C's level order (each level's
// supernodes in turn, each supernode's rows in turn), a supernode listed whole
// or not at all; ptr holds nblk x (C.nlev + 1) offsets into q.  work[0] and
// work[1]: multiply-adds per column of the listed rows and of all rows (their
// external L entries plus their row of the diagonal block's inverse).
void build_forward_reach(const Plan& P, const ColSched& C, std::vector<int>& ptr, std::vector<int>& q,
                         double work[2]);

// Minimum-degree ordering of a weighted graph (adjacency lists, weights =
// unknowns per node); ties broken by node index.
std::vector<int> min_degree_order(int n, const std::vector<std::vector<int>>& adj, const std::vector<int>& wt);

// Builds the plan; returns an empty string on success, else the reason.
std::string build_plan(Plan& P, int nb, int nl, int ng, int slack, const double* Pd,
                       const double* Qd, const double* Vmin, const double* Vmax,
                       const int* lf, const int* lt, const double* r, const double* x,
                       const double* b, const double* rate, const int* gbus,
                       const double* Pmin, const double* Pmax, const double* Qmin,
                       const double* Qmax, const double* c2, const double* c1);

}  // namespace condipm
