// A4-A10: sparse LU refactorisation of G_x, multi-right-hand-side triangular
// solves, K assembly and products, the condensed matrix, dense Cholesky and its
// solves.  FP64 throughout.  On GB300 the FP64 pipe (two DFMA per clock per SM,
// about 1.2 TFLOP/s per GPU; the f64 mma.sync path is slower still) bounds
// every kernel here, so the kernels keep every DFMA lane busy with useful work
// and leave data movement to the load/store pipes.
#include "common.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

namespace condipm {
namespace {

namespace cg = cooperative_groups;

inline int nblk(long long n, int t) { return int((n + t - 1) / t); }

// ----------------------------------------------------------------- K assembly
// K[p] = W[p] + sum_q sig_s[r_q] A[a_q] A[b_q]   (A^T Sigma_s A in K's pattern)
__global__ void k_assemble_K(long long nnz, const double* __restrict__ W, const int* __restrict__ ptr,
                             const int* __restrict__ r, const int* __restrict__ a,
                             const int* __restrict__ b, const double* __restrict__ sig_s,
                             const double* __restrict__ Aval, double* __restrict__ K) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= nnz) return;
  double acc = W[p];
  for (int q = ptr[p]; q < ptr[p + 1]; ++q) acc = fma(sig_s[r[q]] * Aval[a[q]], Aval[b[q]], acc);
  K[p] = acc;
}

// K[(c,c)] += sigma_c, sigma in c-order ([u; x permuted])
__global__ void k_add_diag(int nw, int nu, const int* __restrict__ K_diag, const int* __restrict__ perm,
                           const double* __restrict__ sig_u, const double* __restrict__ sig_x,
                           double* __restrict__ K, double* __restrict__ sig_c) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nw) return;
  double s = c < nu ? sig_u[c] : sig_x[perm[c - nu]];
  K[K_diag[c]] += s;
  sig_c[c] = s;
}

// K[(c,c)] += sigma_c from the stored c-order sigma (re-assembly of K at a new
// dual regularisation)
__global__ void k_add_diag_c(int nw, const int* __restrict__ K_diag, const double* __restrict__ sig_c,
                             double* __restrict__ K) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nw) return;
  K[K_diag[c]] += sig_c[c];
}

// Dual regularisation of the inequality rows (-delta_c I in the (p_y, p_y) block
// of K_aug): Sigma_t = Sigma_s / (1 + delta_c Sigma_s) = (Sigma_s^{-1} + delta_c)^{-1}
// and the slack-step scale 1 / (1 + delta_c Sigma_s)
__global__ void k_sigma_dc(int m, double dc, const double* __restrict__ sig_s, double* __restrict__ sig_t,
                           double* __restrict__ scale) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const double d = 1.0 + dc * sig_s[i];
  sig_t[i] = sig_s[i] / d;
  scale[i] = 1.0 / d;
}

// X(i, ci[q]) = alpha * src[map[q]] for the entries q of row i (X zeroed before),
// element (i, c) at X[i*xr + c*xc]
__global__ void k_scatter_rows(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                               const int* __restrict__ map, const double* __restrict__ src, double alpha,
                               double* __restrict__ X, long long xr, long long xc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int q = rp[i]; q < rp[i + 1]; ++q) X[i * xr + ci[q] * xc] = alpha * src[map ? map[q] : q];
}

// Y = alpha * M X + beta * Y, M CSR; element (i, c) of X at X[i*xr + c*xc] and of
// Y at Y[i*yr + c*yc].  rows_fast selects the thread order (row index fastest for
// column-major operands, column index fastest for row-major ones), so
// neighbouring threads touch neighbouring addresses of Y.
__global__ void k_spmm(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ val, const int* __restrict__ valmap,
                       const double* __restrict__ X, long long xr, long long xc, double* __restrict__ Y,
                       long long yr, long long yc, int ncols, double alpha, double beta, int rows_fast) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long total = (long long)nrows * ncols;
  if (t >= total) return;
  int r, c;
  if (rows_fast) { r = int(t % nrows); c = int(t / nrows); }
  else { r = int(t / ncols); c = int(t % ncols); }
  const double* Xc = X + c * xc;
  double acc = 0.0;
  const int e = rp[r + 1];
  if (valmap) {
    for (int q = rp[r]; q < e; ++q) acc = fma(val[valmap[q]], Xc[ci[q] * xr], acc);
  } else {
    for (int q = rp[r]; q < e; ++q) acc = fma(val[q], Xc[ci[q] * xr], acc);
  }
  double* y = Y + r * yr + c * yc;
  *y = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *y);
}

// Multi-right-hand-side sparse triangular solve, level-scheduled inside one CTA.
// CTA b owns columns [b*CB, b*CB + CB); its threads form slots of CB lanes, one
// lane per column, and a slot walks the rows of the current level.  Levels are
// separated by __syncthreads only: the columns are independent, so no CTA ever
// waits for another.  Row i: X_i <- (X_i - sum_q val_q X_{ci_q}) * inv_diag_i
// (inv_diag NULL = unit diagonal).
template <int CB>
__global__ void __launch_bounds__(256) k_trsm(int nlev, const int* __restrict__ lptr,
                                              const int* __restrict__ lrows, const int* __restrict__ rp,
                                              const int* __restrict__ ci, const double* __restrict__ val,
                                              const double* __restrict__ inv_diag, double* X,
                                              long long xr, long long xc, int ncols) {
  const int c = blockIdx.x * CB + (threadIdx.x % CB);
  const int slot = threadIdx.x / CB;
  const int nslots = blockDim.x / CB;
  const bool active = c < ncols;
  double* Xc = X + c * xc;
  for (int lev = 0; lev < nlev; ++lev) {
    const int beg = lptr[lev], end = lptr[lev + 1];
    if (active) {
      for (int t = beg + slot; t < end; t += nslots) {
        const int i = lrows[t];
        double acc = Xc[i * xr];
        const int qe = rp[i + 1];
        for (int q = rp[i]; q < qe; ++q) acc = fma(-val[q], Xc[ci[q] * xr], acc);
        if (inv_diag) acc *= inv_diag[i];
        Xc[i * xr] = acc;
      }
    }
    __syncthreads();
  }
}

// S (n x n, symmetric) = (A + A^T) / 2, element (i, j) of A at A[i*ar + j*ac]
__global__ void k_symmetrize(int n, const double* __restrict__ A, long long ar, long long ac,
                             double* __restrict__ S) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int i = int(t / n), j = int(t % n);
  S[t] = 0.5 * (A[i * ar + j * ac] + A[j * ar + i * ac]);
}

// Kred = Hu + Sx^T Hx (explicit route): C[a][c] = Hu(a, c) + sum_j Sx(j, a) Hx(j, c),
// operands row-major with leading dimension ld; 64x64 output tiles, 16-deep
// k slices staged in shared memory, 4x4 outputs per thread.  The sum over j
// (nx terms, with nu x nu outputs only) is split over gridDim.z slices of the
// j range: slice z writes its partial sums to P + z nu^2 (P = C and Hu added
// when there is one slice); k_dense_tn_sum adds the slices in order.
__global__ void __launch_bounds__(256) k_dense_tn(int nu, int nx, const double* __restrict__ Sx,
                                                  const double* __restrict__ Hx,
                                                  const double* __restrict__ Hu, long long ld,
                                                  double* __restrict__ P, int kchunk) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int a0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int kb = blockIdx.z * kchunk, ke = min(nx, kb + kchunk);
  double acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      int kk = t / 64, j = t % 64;
      int k = k0 + kk;
      As[kk][j] = (k < ke && a0 + j < nu) ? Sx[k * ld + a0 + j] : 0.0;
      Bs[kk][j] = (k < ke && c0 + j < nu) ? Hx[k * ld + c0 + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { av[u] = As[kk][ty * 4 + u]; bv[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
  }
  double* Pz = P + (size_t)blockIdx.z * nu * nu;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int a = a0 + ty * 4 + u, c = c0 + tx * 4 + v;
      if (a < nu && c < nu) Pz[(size_t)a * nu + c] = gridDim.z == 1 ? Hu[a * ld + c] + acc[u][v] : acc[u][v];
    }
}

// C = Hu + the sum of the slices of P, in slice order (deterministic)
__global__ void k_dense_tn_sum(int nu, int nslices, const double* __restrict__ P, const double* __restrict__ Hu,
                               long long ld, double* __restrict__ C) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nu * nu) return;
  const int a = int(t / nu), c = int(t % nu);
  double v = 0.0;
  for (int z = 0; z < nslices; ++z) v += P[(size_t)z * nu * nu + t];
  C[t] = Hu[a * ld + c] + v;
}

// ----------------------------------------------------------------- LU refactor
__global__ void k_lu_scatter(long long nnzG, const int* __restrict__ map, const double* __restrict__ G,
                             double* __restrict__ LU) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= nnzG) return;
  int p = map[q];
  if (p >= 0) LU[p] = G[q];
}

// max_q |v_q| over each row, one warp per row.  Magnitudes are compared as
// integers on the bit patterns with the sign cleared (the order of non-negative
// doubles), so no FP64 instruction is issued; NaN entries count as 0.
__global__ void k_row_absmax(int n, const int* __restrict__ rp, const double* __restrict__ v,
                             double* __restrict__ out) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  unsigned long long m = 0;
  for (int q = rp[i] + lane; q < rp[i + 1]; q += 32) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v[q]) & 0x7FFFFFFFFFFFFFFFULL;
    if (b > 0x7FF0000000000000ULL) b = 0;   // NaN
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long u = __shfl_xor_sync(0xffffffffu, m, o);
    m = u > m ? u : m;
  }
  if (lane == 0) out[i] = __longlong_as_double((long long)m);
}

// Numeric up-looking LU of P G_x P^T in its fixed pattern (static pivots).
// One warp per row, rows taken in level order; a row waits (bounded) on the
// completion flag of each row k it references, so rows of different levels
// overlap instead of meeting at grid-wide barriers.  The row being factored is
// staged in shared memory; rows of other warps are read through L2 (ld.cg).
// Row i: for k in L(i) ascending: l_ik = w_k / u_kk; w_j -= l_ik u_kj (j in U(k)).
// One row i of the up-looking LU, factored by the calling warp into its
// shared-memory row buffer w (the body of k_lu_refactor and of the batched
// refactorisation).  Returns false when a bounded wait expired.
// entries per lane of a dependency row's update fetched at once
constexpr int LU_PF = 4;

// Reciprocal of an LU pivot (either sign) whose magnitude lies in
// [2^-1000, 2^1000]: the hardware estimate rcp.approx.ftz.f64 and one
// third-order step, r (1 + e + e^2) with e = 1 - d r (relative error e^3,
// from the geometric series of 1 / (1 - e)) -- three dependent FP64
// operations where the IEEE division takes a longer sequence, and each row's
// inverse pivot sits on the refactorisation's hand-off chain.  Other
// magnitudes use the division.
__device__ __forceinline__ double lu_rcp(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFULL;
  if (b >= (23ULL << 52) && b < (2023ULL << 52)) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
  }
  return 1.0 / d;
}

__device__ __forceinline__ bool lu_row(int i, const int* __restrict__ rp, const int* __restrict__ ci,
                                       const int* __restrict__ diag, const long long* __restrict__ upd_ptr,
                                       const int* __restrict__ upd_pos, double* LU, double* inv_diag,
                                       const double* __restrict__ rmax, unsigned* flags, unsigned epoch, int* st,
                                       long long spin_limit, double* w, int lane) {
  volatile int* vst = st;
  const int r0 = rp[i], r1 = rp[i + 1], dpos = diag[i];
  // the pivot threshold, off the hand-off chain: non-negative doubles order
  // like their bit patterns, so the test at the end is an integer compare
  const unsigned long long thr_bits = lane == 0 ? (unsigned long long)__double_as_longlong(1e-14 * rmax[i]) : 0ULL;
  for (int j = r0 + lane; j < r1; j += 32) w[j - r0] = __ldcg(&LU[j]);
  __syncwarp();
  for (int q = r0; q < dpos; ++q) {
    const int k = ci[q];
    // the structure of row k's update needs no wait: fetch it first (its first
    // LU_PF x 32 positions), so that after the flag only the values cost a
    // round trip, all of them in flight together
    const int ub = diag[k] + 1, ue = rp[k + 1];
    const long long base = upd_ptr[q];
    const int j0 = ub + lane;
    int pos[LU_PF];
#pragma unroll
    for (int t = 0; t < LU_PF; ++t) pos[t] = j0 + 32 * t < ue ? upd_pos[base + lane + 32 * t] - r0 : 0;
    int expired = 0;
    if (lane == 0) {
      // acquire load: row k's values and inverse pivot are visible once the
      // flag is (its writer fences before publishing the flag)
      long long it = 0;
      unsigned f;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + k) : "memory");
      unsigned ns = 32;
      while (f != epoch) {
        if (++it > spin_limit) { atomicExch(&st[ST_TIMEOUT], 1); expired = 1; break; }
        // another warp's expired wait ends this one too (its row never comes)
        if ((it & 1023) == 0 && vst[ST_TIMEOUT]) { expired = 1; break; }
        __nanosleep(ns);   // back off, leaving issue slots to working warps
        ns = ns < 128 ? 2 * ns : 128;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + k) : "memory");
      }
    }
    if (__shfl_sync(0xffffffffu, expired, 0)) return false;
    __syncwarp();   // orders lane 0's acquire before every lane's loads of row k
    const double dk = __ldcg(&inv_diag[k]);
    double u[LU_PF];
#pragma unroll
    for (int t = 0; t < LU_PF; ++t) u[t] = j0 + 32 * t < ue ? __ldcg(&LU[j0 + 32 * t]) : 0.0;
    const double lik = w[q - r0] * dk;
    __syncwarp();
#pragma unroll
    for (int t = 0; t < LU_PF; ++t)
      if (j0 + 32 * t < ue) w[pos[t]] = fma(-lik, u[t], w[pos[t]]);
    for (int j = j0 + 32 * LU_PF; j < ue; j += 32) {
      const int pos = upd_pos[base + (j - ub)] - r0;
      w[pos] = fma(-lik, __ldcg(&LU[j]), w[pos]);
    }
    if (lane == 0) w[q - r0] = lik;
    __syncwarp();
  }
  for (int j = r0 + lane; j < r1; j += 32) LU[j] = w[j - r0];
  __syncwarp();
  if (lane == 0) {
    const double u = w[dpos - r0];
    const unsigned long long ub = (unsigned long long)__double_as_longlong(u) & 0x7FFFFFFFFFFFFFFFULL;
    double inv = 0.0;
    // |u| <= 1e-14 max|row| (or NaN threshold), or u not finite: singular
    if (!(ub > thr_bits) || ub >= 0x7FF0000000000000ULL || thr_bits > 0x7FF0000000000000ULL)
      set_status(st, DEV_SINGULAR, i);
    else inv = lu_rcp(u);
    inv_diag[i] = inv;
    // release: the row's values (ordered before lane 0 by __syncwarp) and its
    // inverse pivot are visible to whoever acquires the flag
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flags + i), "r"(epoch) : "memory");
  }
  __syncwarp();
  return true;
}

__global__ void k_lu_refactor(int n, const int* __restrict__ rows, const int* __restrict__ rp,
                              const int* __restrict__ ci, const int* __restrict__ diag,
                              const long long* __restrict__ upd_ptr, const int* __restrict__ upd_pos,
                              double* LU, double* inv_diag, const double* __restrict__ rmax,
                              unsigned* flags, unsigned epoch, int* st, long long spin_limit,
                              int maxlen) {
  extern __shared__ double wsh[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  double* w = wsh + (size_t)wib * maxlen;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < n; t += nwarps)
    if (!lu_row(rows[t], rp, ci, diag, upd_ptr, upd_pos, LU, inv_diag, rmax, flags, epoch, st, spin_limit, w, lane))
      return;
}

// The refactorisation of every instance of a batch in one cooperative launch:
// the warps take the merged row list (instance, row), ordered by level and,
// within a level, by instance; each instance's rows keep their level order, so
// the oldest unfinished item can always proceed and every bounded wait is on
// an item earlier in the list.
__global__ void k_b_lu(const BatchInst* __restrict__ I, const int2* __restrict__ items, int nitems, unsigned epoch,
                       long long spin_limit, int maxlen) {
  extern __shared__ double wsh[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  double* w = wsh + (size_t)wib * maxlen;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < nitems; t += nwarps) {
    const int2 it = items[t];
    const BatchInst& B = I[it.x];
    if (!B.active) continue;
    if (!lu_row(it.y, B.LU_rp, B.LU_ci, B.LU_diag, B.upd_ptr, B.upd_pos, B.LUval, B.inv_diag, B.rmax, B.flags,
                epoch, B.st, spin_limit, w, lane))
      return;
  }
}

__global__ void k_gather_map(long long n, const int* __restrict__ map, const double* __restrict__ src,
                             double* __restrict__ dst) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) dst[q] = src[map[q]];
}

// ----------------------------------------------------------------- batched phases
// Elementwise work of one instance inside a batched launch: the blocks
// boff[i] .. boff[i + 1] of the grid serve instance i; lt is this thread's
// index within them and ls their thread count.
struct BatchSlice {
  const BatchInst* B;
  long long lt, ls;
};
__device__ __forceinline__ BatchSlice batch_slice(const BatchInst* I, const int* __restrict__ boff, int n) {
  const int i = batch_instance(boff, n, blockIdx.x);
  BatchSlice sl;
  sl.B = I + i;
  sl.lt = (long long)(blockIdx.x - boff[i]) * blockDim.x + threadIdx.x;
  sl.ls = (long long)(boff[i + 1] - boff[i]) * blockDim.x;
  return sl;
}

// zero LU, the row flags, the status word and S_x (the x rows of Z)
__global__ void k_b_clear(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff) {
  const BatchSlice sl = batch_slice(I, boff, n);
  const BatchInst& B = *sl.B;
  if (!B.active) return;
  for (long long e = sl.lt; e < B.nnzLU; e += sl.ls) B.LUval[e] = 0.0;
  for (long long e = sl.lt; e < B.nx; e += sl.ls) B.flags[e] = 0u;
  if (sl.lt < ST_WORDS) B.st[sl.lt] = 0;
  double* Sx = B.Zt + (size_t)B.nu * B.ld;
  const long long nsx = (long long)B.nx * B.ld;
  for (long long e = sl.lt; e < nsx; e += sl.ls) Sx[e] = 0.0;
}

// G_x into LU; -P G_u into S_x; K = W + A^T Sigma_s A; the handle's copy of Sigma_s
__global__ void k_b_scatter(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff) {
  const BatchSlice sl = batch_slice(I, boff, n);
  const BatchInst& B = *sl.B;
  if (!B.active) return;
  for (long long q = sl.lt; q < B.nnzG; q += sl.ls) {
    const int p = B.Gx_to_LU[q];
    if (p >= 0) B.LUval[p] = B.Gval[q];
  }
  double* Sx = B.Zt + (size_t)B.nu * B.ld;
  for (long long r = sl.lt; r < B.nx; r += sl.ls)
    for (int q = B.PGu_rp[r]; q < B.PGu_rp[r + 1]; ++q)
      Sx[r * B.ld + B.PGu_ci[q]] = -1.0 * B.Gval[B.PGu_map[q]];
  for (long long p = sl.lt; p < B.nnzK; p += sl.ls) {
    double acc = B.Wval[p];
    for (int q = B.KAA_ptr[p]; q < B.KAA_ptr[p + 1]; ++q)
      acc = fma(B.sig_s_in[B.KAA_r[q]] * B.Aval[B.KAA_a[q]], B.Aval[B.KAA_b[q]], acc);
    B.Kval[p] = acc;
  }
  for (long long i = sl.lt; i < B.m; i += sl.ls) B.sig_s[i] = B.sig_s_in[i];
}

// row maxima of LU (one warp per row, on the bit patterns as k_row_absmax) and
// diag(Sigma_w) into K
__global__ void k_b_rowmax(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff) {
  const BatchSlice sl = batch_slice(I, boff, n);
  const BatchInst& B = *sl.B;
  if (!B.active) return;
  const int lane = threadIdx.x & 31;
  for (long long i = sl.lt >> 5; i < B.nx; i += sl.ls >> 5) {
    unsigned long long mx = 0;
    for (int q = B.LU_rp[i] + lane; q < B.LU_rp[i + 1]; q += 32) {
      unsigned long long b = (unsigned long long)__double_as_longlong(B.LUval[q]) & 0x7FFFFFFFFFFFFFFFULL;
      if (b > 0x7FF0000000000000ULL) b = 0;   // NaN
      mx = b > mx ? b : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = u > mx ? u : mx;
    }
    if (lane == 0) B.rmax[i] = __longlong_as_double((long long)mx);
  }
  for (long long c = sl.lt; c < B.nw; c += sl.ls) {
    const double sg = c < B.nu ? B.sig_u[c] : B.sig_x[B.perm[c - B.nu]];
    B.Kval[B.K_diag[c]] += sg;
    B.sig_c[c] = sg;
  }
}

// which = 0: H = K Z (nw rows); which = 1: H_u -= G_u^T Psi, Psi in H's x rows
__global__ void k_b_spmm(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff, int which) {
  const BatchSlice sl = batch_slice(I, boff, n);
  const BatchInst& B = *sl.B;
  if (!B.active) return;
  const long long ld = B.ld;
  const int nu = B.nu;
  const long long total = (long long)(which == 0 ? B.nw : nu) * nu;
  for (long long e = sl.lt; e < total; e += sl.ls) {
    const int r = int(e / nu), c = int(e % nu);
    double acc = 0.0;
    if (which == 0) {
      for (int q = B.K_rp[r]; q < B.K_rp[r + 1]; ++q) acc = fma(B.Kval[q], B.Zt[B.K_ci[q] * ld + c], acc);
      B.H[r * ld + c] = acc;
    } else {
      const double* Hx = B.H + (size_t)nu * ld;
      for (int q = B.GuT_rp[r]; q < B.GuT_rp[r + 1]; ++q)
        acc = fma(B.Gval[B.GuT_map[q]], Hx[B.GuT_ci[q] * ld + c], acc);
      double* y = B.H + r * ld + c;
      *y = fma(-1.0, acc, *y);
    }
  }
}

// Kred = (H_u + H_u^T) / 2 and F = its lower triangle + delta_w I
__global__ void k_b_kred(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff) {
  const BatchSlice sl = batch_slice(I, boff, n);
  const BatchInst& B = *sl.B;
  if (!B.active) return;
  const int nu = B.nu;
  const long long ld = B.ld;
  for (long long e = sl.lt; e < (long long)nu * nu; e += sl.ls) {
    const int i = int(e / nu), j = int(e % nu);
    const double v = 0.5 * (B.H[i * ld + j] + B.H[j * ld + i]);
    B.Kred[e] = v;
    B.F[e] = j > i ? 0.0 : (i == j ? v + B.delta_w : v);
  }
}

// the status words of the active instances, side by side (read back at once)
__global__ void k_b_status(const BatchInst* __restrict__ I, int n, int* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * ST_WORDS) return;
  const BatchInst& B = I[t / ST_WORDS];
  out[t] = B.active ? B.st[t % ST_WORDS] : 0;
}

// ----------------------------------------------------------------- Cholesky
constexpr int CNB = 32;

__global__ void k_chol_prepare(int n, const double* __restrict__ A, double delta, double* __restrict__ F) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int i = int(t / n), j = int(t % n);
  F[t] = j > i ? 0.0 : (i == j ? A[t] + delta : A[t]);
}

// 1/sqrt(d) by Newton-Raphson on f(x) = x^-2 - d (x <- x (3 - d x^2) / 2), seeded
// with the single-precision hardware estimate; two steps take the ~23-bit seed
// to double precision.  Pivots outside the single-precision exponent range use
// the library square root.
__device__ __forceinline__ double rsqrt_nr(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double x = (double)rsqrtf((float)d);
  x = x * fma(-0.5 * d, x * x, 1.5);
  x = x * fma(-0.5 * d, x * x, 1.5);
  return x;
}

// Pairs (i, l), 0 <= l <= i < 32, of a 32x32 lower triangle, ordered by l
// descending: the trailing triangle of column j (l > j) is the prefix of
// length (31 - j)(32 - j) / 2, and the pair (j+1, j+1) is its last but (31 - j)
// entries.  Packed as i << 8 | l.  Filled by each CTA at kernel start.
__device__ __forceinline__ void fill_pairs(unsigned short* pairs) {
  for (int t = threadIdx.x; t < CNB * (CNB + 1) / 2; t += blockDim.x) {
    // q = 31 - l is the largest q with q (q + 1) / 2 <= t
    int q = int((sqrtf(8.0f * float(t) + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) / 2 <= t) ++q;
    while (q * (q + 1) / 2 > t) --q;
    const int l = CNB - 1 - q, i = l + (t - q * (q + 1) / 2);
    pairs[t] = (unsigned short)((i << 8) | l);
  }
}

// Store the lower triangle of a factored diagonal tile (tile column k) into F.
__device__ __forceinline__ void write_tile_back(double* F, int n, const double (*T)[CNB + 1], int k) {
  const int k0 = k * CNB, kb = min(CNB, n - k0);
  for (int t = threadIdx.x; t < CNB * CNB; t += blockDim.x) {
    const int i = t / CNB, j = t % CNB;
    if (i < kb && j <= i) F[(size_t)(k0 + i) * n + k0 + j] = T[i][j];
  }
}

// Reciprocal of a pivot, or 0 when the pivot is not a positive finite number.
// Inside [2^-1000, 2^1000] (tested on the bit pattern, integer compares only:
// on this GPU every FP64 instruction, compares included, goes through the FP64
// pipe at about 64 cycles) it takes the hardware estimate rcp.approx.ftz.f64
// and one third-order Householder step: with e = 1 - d r, 1/d = r / (1 - e) =
// r (1 + e + e^2 + ...), so r (1 + e + e^2) leaves a relative error of e^3 --
// three dependent FP64 operations where the IEEE division takes a longer
// sequence, and the reciprocal of each pivot sits on the factorisation's
// critical path.  Other positive finite pivots use the division.
__device__ __forceinline__ double pivot_rcp(double d) {
  const long long b = __double_as_longlong(d);
  if (b >= (23LL << 52) && b < (2023LL << 52)) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    const double e = fma(-d, r, 1.0);
    return fma(r, fma(e, e, e), r);
  }
  return (b > 0 && b < 0x7FF0000000000000LL) ? 1.0 / d : 0.0;
}

// Cholesky of the 32x32 tile T in shared memory (kb valid rows, the rest an
// identity block), computed as T = U D U^T with the columns of U left unscaled
// (the root-free form) and converted to L = U D^{-1/2} at the end.  Column j:
// every thread takes pairs of the trailing triangle from the table, so each
// rank-1 update T_il -= T_ij T_lj / d_j is spread evenly over all warps (all
// four FP64 pipes of the SM); the thread that updates T_{j+1,j+1} computes the
// next pivot's reciprocal at once, so a column costs one barrier and its
// critical path is a multiply, an FMA and a reciprocal.  The square roots of
// the pivots are taken once, all together, at the end.  Writes 1 / L_jj to
// dv[j]; returns the first failing local column (non-positive or non-finite
// pivot) or -1.
// R (optional, nr = 8, 16 or 24 rows) holds panel rows below the tile: they
// are eliminated along with it, as further rows of the column block, and leave
// as rows of L (R L_kk^T = the rows given), so the panel solve costs no
// separate sequence of dependent steps.
template <int NR>
__device__ __forceinline__ void tile_rows_update(double (*R)[CNB + 1], const double (*T)[CNB + 1], int j, double rj,
                                                 int wk, int nwk) {
  // R_rl -= R_rj T_lj / d_j for l > j (row index fastest)
  for (int q = wk; q < NR * (CNB - 1 - j); q += nwk) {
    const int rr = q % NR, l = j + 1 + q / NR;
    R[rr][l] = fma(-R[rr][j] * rj, T[l][j], R[rr][l]);
  }
}

__device__ int block_chol_tile(double (*T)[CNB + 1], double* dv, int kb, const unsigned short* pairs,
                               double (*R)[CNB + 1] = nullptr, int nr = 0) {
  const int tid = threadIdx.x;
  // worker index of the threads outside sub-partition 0 (warps 1-3, 5-7, ...)
  const int warp = tid >> 5, nwarps = blockDim.x >> 5;
  const bool one_warp = nwarps == 1;   // then every thread is a worker
  const int wk = one_warp ? tid : ((warp & 3) ? (warp - (warp >> 2) - 1) * 32 + (tid & 31) : -1);
  const int nwk = one_warp ? 32 : (nwarps - (nwarps + 3) / 4) * 32;
  // during the loop dv[j] = 1 / d_j, or 0 for a failed pivot; every thread reads
  // it after a barrier, so all leave together on a failure
  if (tid == 0) dv[0] = pivot_rcp(T[0][0]);
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const double rj = dv[j];
    if (__double_as_longlong(rj) <= 0) return j;   // 0 marks a failed pivot
    const int cnt = (CNB - 1 - j) * (CNB - j) / 2;
    const int diag_next = (CNB - 2 - j) * (CNB - 1 - j) / 2;   // position of (j+1, j+1)
    // thread 0 takes the next pivot's pair and its reciprocal alone: warp w
    // runs on sub-partition w mod 4, and the other warps of thread 0's
    // sub-partition stay off the FP64 pipe, so that chain is not queued behind
    // their updates; the warps of the other three sub-partitions share the
    // rest of the pairs
    if (tid == 0 && cnt > 0) {
      const int pr = pairs[diag_next], i = pr >> 8, l = pr & 255;
      const double v = fma(-T[i][j] * rj, T[l][j], T[i][l]);
      T[i][l] = v;
      if (j + 1 < kb) dv[j + 1] = pivot_rcp(v);
    }
    if (wk >= 0) {
      for (int q = 1 + wk; q < cnt; q += nwk) {
        int t = diag_next + q;
        if (t >= cnt) t -= cnt;
        const int pr = pairs[t], i = pr >> 8, l = pr & 255;
        T[i][l] = fma(-T[i][j] * rj, T[l][j], T[i][l]);
      }
    }
    if (nr > 0 && wk >= 0) {
      if (nr == 8) tile_rows_update<8>(R, T, j, rj, wk, nwk);
      else if (nr == 16) tile_rows_update<16>(R, T, j, rj, wk, nwk);
      else tile_rows_update<24>(R, T, j, rj, wk, nwk);
    }
    __syncthreads();
  }
  // L_jj = sqrt(d_j) = d_j / sqrt(d_j), L_ij = U_ij / sqrt(d_j)
  if (tid < kb) {
    const double d = T[tid][tid], s = rsqrt_nr(d);
    dv[tid] = s;
    T[tid][tid] = d * s;
  }
  __syncthreads();
  for (int t = tid; t < CNB * CNB; t += blockDim.x) {
    const int i = t / CNB, j = t % CNB;
    if (j < kb && i > j) T[i][j] *= dv[j];
  }
  if (nr > 0)
    for (int t = tid; t < nr * CNB; t += blockDim.x) {
      const int rr = t / CNB, j = t % CNB;
      if (j < kb) R[rr][j] *= dv[j];
    }
  __syncthreads();
  return -1;
}

// Right-looking blocked Cholesky of the lower triangle of F (row-major n x n),
// 32x32 tiles, one persistent cooperative grid, two phases per block column
// separated by a bounded grid barrier:
//   P. the rows below the diagonal tile are shared out eight per CTA, one per
//      warp; a CTA with rows (and CTA 0, which writes the tile back once the
//      barrier shows every CTA done reading it) factors the diagonal tile
//      itself in shared memory, then each warp solves its row x L_kk^T = a
//      (one column per lane) -- no barrier between the two;
//   U. the trailing update A_ij -= L_ik L_jk^T in 16x16 sub-tiles.
// A non-positive or non-finite pivot records DEV_NOT_PD with its column.  The
// inverse diagonal of L is written to dinv (used by the solves).
// The barrier form's body, for a group of nbk CTAs (this one is rank) that
// sync() brings together: the whole grid of k_chol, or one thread-block
// cluster per instance in the batched factorisation.
template <class Sync>
__device__ __forceinline__ void chol_run(double* F, int n, double* dinv_out, int* st, int rank, unsigned nbk,
                                         Sync&& sync) {
  __shared__ double Ta[CNB][CNB + 1];
  __shared__ double Tb[CNB][CNB + 1];
  __shared__ double dv[CNB];
  __shared__ unsigned short pairs[CNB * (CNB + 1) / 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nt = (n + CNB - 1) / CNB;
  volatile int* vst = st;
  fill_pairs(pairs);
  __syncthreads();
  for (int k = 0; k < nt; ++k) {
    const int k0 = k * CNB, kb = min(CNB, n - k0);
    const int r0 = k0 + kb, nrows = n - r0;              // panel rows r0 .. n-1
    const int row_blocks = (nrows + nwarps - 1) / nwarps;
    // ---- phase P
    if (rank == 0 || rank < row_blocks) {
      for (int t = tid; t < CNB * CNB; t += blockDim.x) {
        const int i = t / CNB, j = t % CNB;
        Ta[i][j] = (i < kb && j <= i) ? F[(size_t)(k0 + i) * n + k0 + j] : (i == j ? 1.0 : 0.0);
      }
      __syncthreads();
      const int fail = block_chol_tile(Ta, dv, kb, pairs);
      if (fail >= 0) {
        if (tid == 0) set_status(st, DEV_NOT_PD, k0 + fail);
      } else {
        if (rank == 0) {
          // the factored tile goes back to F after the barrier: the other panel
          // CTAs may still be reading the unfactored one now
          for (int t = tid; t < CNB * CNB; t += blockDim.x) Tb[t / CNB][t % CNB] = Ta[t / CNB][t % CNB];
          if (tid < kb) dinv_out[k0 + tid] = dv[tid];
        }
        for (int rb = rank; rb < row_blocks; rb += nbk) {
          const int r = r0 + rb * nwarps + warp;
          if (r < n) {
            double a = lane < kb ? F[(size_t)r * n + k0 + lane] : 0.0;
            for (int j = 0; j < kb; ++j) {
              const double xj = __shfl_sync(0xffffffffu, a, j) * dv[j];
              if (lane == j) a = xj;
              else if (lane > j) a = fma(-xj, Ta[lane][j], a);
            }
            if (lane < kb) F[(size_t)r * n + k0 + lane] = a;
          }
        }
      }
    }
    if (!sync()) return;
    if (vst[ST_CODE] != 0) return;
    if (rank == 0) {
      write_tile_back(F, n, Tb, k);
      __syncthreads();   // Tb is reused by the update below
    }
    const int m = nt - k - 1;
    const long long ntile = (long long)m * (m + 1) / 2;
    if (ntile < (long long)nbk) {
      // ---- phase U, few tiles left: 16x16 sub-tiles (four per tile) for more
      // work items than CTAs
      const long long nsub = ntile * 4;
      for (long long tt = rank; tt < nsub; tt += nbk) {
        const long long tile = tt >> 2;
        const int sub = int(tt & 3);
        int ii = int((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
        while ((long long)(ii + 1) * (ii + 2) / 2 <= tile) ++ii;
        while ((long long)ii * (ii + 1) / 2 > tile) --ii;
        const int jj = int(tile - (long long)ii * (ii + 1) / 2);
        if (ii == jj && sub == 1) continue;   // strictly upper quarter of a diagonal tile
        const int i0 = (k + 1 + ii) * CNB + (sub >> 1) * 16;
        const int j0 = (k + 1 + jj) * CNB + (sub & 1) * 16;
        for (int t = tid; t < 16 * CNB; t += blockDim.x) {
          const int rr = t / CNB, l = t % CNB;
          Ta[rr][l] = (i0 + rr < n && l < kb) ? F[(size_t)(i0 + rr) * n + k0 + l] : 0.0;
          Tb[rr][l] = (j0 + rr < n && l < kb) ? F[(size_t)(j0 + rr) * n + k0 + l] : 0.0;
        }
        __syncthreads();
        const int rr = tid >> 4, cc = tid & 15;
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
        for (int l = 0; l < CNB; l += 2) {
          acc0 = fma(Ta[rr][l], Tb[cc][l], acc0);
          acc1 = fma(Ta[rr][l + 1], Tb[cc][l + 1], acc1);
        }
        const int gi = i0 + rr, gj = j0 + cc;
        if (gi < n && gj < n && gj <= gi) F[(size_t)gi * n + gj] -= acc0 + acc1;
        __syncthreads();
      }
    } else {
      // ---- phase U: whole 32x32 tiles of the lower trailing triangle; thread
      // (ty, tx) owns rows {ty, ty + 16} x columns {tx, tx + 16}; the panel tiles
      // of the next tile are fetched into registers while this one is computed
      const int ty = tid >> 4, tx = tid & 15;
      auto tile_ij = [&](long long tile, int& i0, int& j0) {
        int ii = int((sqrtf(8.0f * (float)tile + 1.0f) - 1.0f) * 0.5f);
        while ((long long)(ii + 1) * (ii + 2) / 2 <= tile) ++ii;
        while ((long long)ii * (ii + 1) / 2 > tile) --ii;
        const int jj = int(tile - (long long)ii * (ii + 1) / 2);
        i0 = (k + 1 + ii) * CNB;
        j0 = (k + 1 + jj) * CNB;
      };
      // each thread moves 4 elements of each panel tile: rows (t / 32) + 8 q, column t % 32
      double pa[4], pb[4];
      auto fetch = [&](long long tile) {
        int i0, j0;
        tile_ij(tile, i0, j0);
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = (tid >> 5) + 8 * q, l = tid & 31;
          pa[q] = (i0 + rr < n && l < kb) ? F[(size_t)(i0 + rr) * n + k0 + l] : 0.0;
          pb[q] = (j0 + rr < n && l < kb) ? F[(size_t)(j0 + rr) * n + k0 + l] : 0.0;
        }
      };
      long long tt = rank;
      if (tt < ntile) fetch(tt);
      for (; tt < ntile; tt += nbk) {
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = (tid >> 5) + 8 * q, l = tid & 31;
          Ta[rr][l] = pa[q];
          Tb[rr][l] = pb[q];
        }
        __syncthreads();
        if (tt + nbk < ntile) fetch(tt + nbk);
        int i0, j0;
        tile_ij(tt, i0, j0);
        double c00 = 0.0, c01 = 0.0, c10 = 0.0, c11 = 0.0;
  #pragma unroll 8
        for (int l = 0; l < CNB; ++l) {
          const double a0 = Ta[ty][l], a1 = Ta[ty + 16][l];
          const double b0 = Tb[tx][l], b1 = Tb[tx + 16][l];
          c00 = fma(a0, b0, c00);
          c01 = fma(a0, b1, c01);
          c10 = fma(a1, b0, c10);
          c11 = fma(a1, b1, c11);
        }
        const int r0g = i0 + ty, r1g = i0 + ty + 16, c0g = j0 + tx, c1g = j0 + tx + 16;
        if (r0g < n && c0g <= r0g) F[(size_t)r0g * n + c0g] -= c00;
        if (r0g < n && c1g < n && c1g <= r0g) F[(size_t)r0g * n + c1g] -= c01;
        if (r1g < n && c0g <= r1g) F[(size_t)r1g * n + c0g] -= c10;
        if (r1g < n && c1g < n && c1g <= r1g) F[(size_t)r1g * n + c1g] -= c11;
        __syncthreads();
      }
    }
    if (!sync()) return;
  }
}


__global__ void __launch_bounds__(256) k_chol(double* F, int n, double* dinv_out, int* st, unsigned* bar,
                                              long long spin_limit) {
  chol_run(F, n, dinv_out, st, (int)blockIdx.x, gridDim.x,
           [&]() { return grid_barrier(bar, gridDim.x, spin_limit, st); });
}

// The Cholesky of every instance of a batch in one launch: one thread-block
// cluster per instance (its CTAs are co-scheduled by the hardware, so the
// cluster barrier between the panel and update phases always completes).
__global__ void __launch_bounds__(256) k_b_chol(const BatchInst* __restrict__ I) {
  cg::cluster_group cl = cg::this_cluster();
  const BatchInst& B = I[blockIdx.x / cl.num_blocks()];
  if (!B.active) return;   // the whole cluster leaves together, before any cluster barrier
  chol_run(B.F, B.nu, B.Fdinv, B.st, (int)cl.block_rank(), cl.num_blocks(), [&]() {
    cl.sync();
    return true;
  });
}

// Solve L L^T X = B for the columns of X (row-major n x nrhs); one CTA per column.
// Forward: 32-row tiles, x_I = L_II^{-1}(b_I - L_I,<I x_<I), the GEMV part with warps
// over rows and lanes over columns of L; backward mirrors it with L^T.
__global__ void __launch_bounds__(256) k_chol_solve(int n, const double* __restrict__ F,
                                                    const double* __restrict__ dinv, double* X, int nrhs) {
  extern __shared__ double xs[];   // n entries: the column being solved
  __shared__ double part[8][CNB];
  const int col = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < n; i += blockDim.x) xs[i] = X[(size_t)i * nrhs + col];
  __syncthreads();
  const int nt = (n + CNB - 1) / CNB;
  // forward
  for (int I = 0; I < nt; ++I) {
    const int i0 = I * CNB, ib = min(CNB, n - i0);
    // b_I -= L[I rows][0:i0] x[0:i0]: warp w takes rows i0+w, i0+w+8, ...
    for (int rr = warp; rr < ib; rr += 8) {
      const double* Lr = F + (size_t)(i0 + rr) * n;
      double acc = 0.0;
      for (int j = lane; j < i0; j += 32) acc = fma(Lr[j], xs[j], acc);
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) xs[i0 + rr] -= acc;
    }
    __syncthreads();
    if (warp == 0) {
      double xv = lane < ib ? xs[i0 + lane] : 0.0;
      for (int j = 0; j < ib; ++j) {
        double xj = __shfl_sync(0xffffffffu, xv, j) * dinv[i0 + j];
        if (lane == j) xv = xj;
        else if (lane > j && lane < ib) xv = fma(-xj, F[(size_t)(i0 + lane) * n + i0 + j], xv);
      }
      if (lane < ib) xs[i0 + lane] = xv;
    }
    __syncthreads();
  }
  // backward: L^T x = y
  for (int I = nt - 1; I >= 0; --I) {
    const int i0 = I * CNB, ib = min(CNB, n - i0);
    // y_I -= sum_{r >= i0+ib} L[r][i0 + c] x_r : warps over rows r, lanes over c
    double acc = 0.0;
    for (int r = i0 + ib + warp; r < n; r += 8)
      if (lane < ib) acc = fma(F[(size_t)r * n + i0 + lane], xs[r], acc);
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
      double s = 0.0;
      for (int w2 = 0; w2 < 8; ++w2) s += part[w2][lane];
      double xv = lane < ib ? xs[i0 + lane] - s : 0.0;
      for (int j = ib - 1; j >= 0; --j) {
        double xj = __shfl_sync(0xffffffffu, xv, j) * dinv[i0 + j];
        if (lane == j) xv = xj;
        else if (lane < j) xv = fma(-xj, F[(size_t)(i0 + j) * n + i0 + lane], xv);
      }
      if (lane < ib) xs[i0 + lane] = xv;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) X[(size_t)i * nrhs + col] = xs[i];
}

// ----------------------------------------------------------------- vectors
// Row permutation and layout change of an n x ncols block:
//   inverse = 0: dst(r, c) = alpha * src(idx[r], c);  inverse = 1: dst(idx[r], c) = alpha * src(r, c)
// (idx NULL = identity).  *_colmajor selects element (row, c) at [c*ld + row]
// instead of [row*ld + c].
__global__ void k_permute_rows(int n, int ncols, const int* __restrict__ idx, const double* __restrict__ src,
                               int lds, int scm, double* __restrict__ dst, int ldd, int dcm, double alpha,
                               int inverse) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * ncols) return;
  int r = int(t / ncols), c = int(t % ncols);
  int rs = r, rd = r;
  if (idx) { if (inverse) rd = idx[r]; else rs = idx[r]; }
  double v = scm ? src[(size_t)c * lds + rs] : src[(size_t)rs * lds + c];
  if (dcm) dst[(size_t)c * ldd + rd] = alpha * v;
  else dst[(size_t)rd * ldd + c] = alpha * v;
}

__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ z) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  z[t] = y ? fma(a, x[t], b * y[t]) : a * x[t];
}

// z(r, c) = d[r] * x(r, c) + b * y(r, c)   (row-major, y may be NULL)
__global__ void k_scale_rows(int n, int ncols, const double* __restrict__ d, const double* __restrict__ x,
                             double* __restrict__ z, double b, const double* __restrict__ y) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * ncols) return;
  int r = int(t / ncols);
  z[t] = y ? fma(d[r], x[t], b * y[t]) : d[r] * x[t];
}

__global__ void k_absmax(long long n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[1024];
  double m = 0.0;
  for (long long t = threadIdx.x; t < n; t += blockDim.x) m = fmax(m, fabs(x[t]));
  sh[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_fill(long long n, double v, double* __restrict__ x) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) x[t] = v;
}

// identity in the leading n x n block of a column-major X with leading dimension ld
__global__ void k_set_identity(int n, double* __restrict__ X, int ld) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int i = int(t % n), j = int(t / n);
  X[(size_t)j * ld + i] = i == j ? 1.0 : 0.0;
}

}  // namespace

// ----------------------------------------------------------------- launchers
cudaError_t launch_assemble_K(cudaStream_t s, long long nnz, const double* W, const int* ptr, const int* r,
                              const int* a, const int* b, const double* sig_s, const double* Aval,
                              double* K) {
  k_assemble_K<<<nblk(nnz, 256), 256, 0, s>>>(nnz, W, ptr, r, a, b, sig_s, Aval, K);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_add_diag(cudaStream_t s, int nw, int nu, const int* K_diag, const int* perm,
                            const double* sig_u, const double* sig_x, double* K, double* sig_c) {
  k_add_diag<<<nblk(nw, 256), 256, 0, s>>>(nw, nu, K_diag, perm, sig_u, sig_x, K, sig_c);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_add_diag_c(cudaStream_t s, int nw, const int* K_diag, const double* sig_c, double* K) {
  k_add_diag_c<<<nblk(nw, 256), 256, 0, s>>>(nw, K_diag, sig_c, K);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_sigma_dc(cudaStream_t s, int m, double dc, const double* sig_s, double* sig_t, double* scale) {
  if (m <= 0) return cudaSuccess;
  k_sigma_dc<<<nblk(m, 256), 256, 0, s>>>(m, dc, sig_s, sig_t, scale);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_scatter_rows(cudaStream_t s, int nrows, const int* rp, const int* ci, const int* map,
                                const double* src, double alpha, double* X, long long xr, long long xc) {
  if (nrows <= 0) return cudaSuccess;
  k_scatter_rows<<<nblk(nrows, 256), 256, 0, s>>>(nrows, rp, ci, map, src, alpha, X, xr, xc);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_spmm(cudaStream_t s, int nrows, const int* rp, const int* ci, const double* val,
                        const int* valmap, const double* X, long long xr, long long xc, double* Y,
                        long long yr, long long yc, int ncols, double alpha, double beta) {
  long long total = (long long)nrows * ncols;
  if (total <= 0) return cudaSuccess;
  const int rows_fast = yr == 1 ? 1 : 0;
  k_spmm<<<nblk(total, 256), 256, 0, s>>>(nrows, rp, ci, val, valmap, X, xr, xc, Y, yr, yc, ncols, alpha,
                                          beta, rows_fast);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_trsm(cudaStream_t s, int cb, int nlev, const int* lptr, const int* lrows, const int* rp,
                        const int* ci, const double* val, const double* inv_diag, double* X, long long xr,
                        long long xc, int ncols) {
  if (ncols <= 0 || nlev <= 0) return cudaSuccess;
  const int T = 256;
#define TRSM_CASE(CBV)                                                                           \
  case CBV:                                                                                      \
    k_trsm<CBV><<<nblk(ncols, CBV), T, 0, s>>>(nlev, lptr, lrows, rp, ci, val, inv_diag, X, xr, xc, ncols); \
    break;
  switch (cb) {
    TRSM_CASE(1) TRSM_CASE(2) TRSM_CASE(4) TRSM_CASE(8) TRSM_CASE(16) TRSM_CASE(32)
    default: return cudaErrorInvalidValue;
  }
#undef TRSM_CASE
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_symmetrize(cudaStream_t s, int n, const double* A, long long ar, long long ac,
                              double* S) {
  k_symmetrize<<<nblk((long long)n * n, 256), 256, 0, s>>>(n, A, ar, ac, S);
  note_launch();
  return cudaGetLastError();
}
int dense_tn_slices(int nu, int nx) {
  const int tiles = nblk(nu, 64) * nblk(nu, 64);
  int z = std::max(1, std::min(64, (2 * device_sms() + tiles - 1) / tiles));
  z = std::min(z, std::max(1, nx / 256));   // at least 256 terms per slice
  while (z > 1 && (size_t)z * nu * nu * sizeof(double) > ((size_t)256 << 20)) --z;
  return z;
}
cudaError_t launch_dense_tn(cudaStream_t s, int nu, int nx, const double* Sx, const double* Hx,
                            const double* Hu, long long ld, double* Kred, double* scratch, int nslices) {
  const int z = std::max(1, nslices);
  const int kchunk = (nblk(nx, z) + 15) / 16 * 16;
  dim3 grid(nblk(nu, 64), nblk(nu, 64), z);
  k_dense_tn<<<grid, 256, 0, s>>>(nu, nx, Sx, Hx, Hu, ld, z == 1 ? Kred : scratch, kchunk);
  note_launch();
  if (z > 1) {
    k_dense_tn_sum<<<nblk((long long)nu * nu, 256), 256, 0, s>>>(nu, z, scratch, Hu, ld, Kred);
    note_launch();
  }
  return cudaGetLastError();
}
cudaError_t launch_lu_scatter(cudaStream_t s, long long nnzG, const int* Gx_to_LU, const double* Gval,
                              double* LU) {
  k_lu_scatter<<<nblk(nnzG, 256), 256, 0, s>>>(nnzG, Gx_to_LU, Gval, LU);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_row_absmax(cudaStream_t s, int n, const int* rp, const double* val, double* rmax) {
  k_row_absmax<<<nblk((long long)n * 32, 256), 256, 0, s>>>(n, rp, val, rmax);
  note_launch();
  return cudaGetLastError();
}
int lu_refactor_max_blocks(int nthreads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (smem > 48 * 1024 && allow_max_smem((const void*)k_lu_refactor) != cudaSuccess) return 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_lu_refactor, nthreads, smem);
  return sms * per;
}
// Cooperative launch: every warp of the grid is resident, which the flag waits
// of the sync-free schedule rely on.
cudaError_t launch_lu_refactor(cudaStream_t s, int n, const int* rows, const int* rp, const int* ci,
                               const int* diag, const long long* upd_ptr, const int* upd_pos, double* LU,
                               double* inv_diag, const double* rmax, unsigned* flags, unsigned epoch,
                               int* st, long long spin_limit, int nblocks, int nthreads, int maxlen) {
  size_t smem = (size_t)(nthreads / 32) * maxlen * sizeof(double);
  void* args[] = {&n, &rows, &rp, &ci, &diag, &upd_ptr, &upd_pos, &LU, &inv_diag, &rmax, &flags, &epoch,
                  &st, &spin_limit, &maxlen};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)k_lu_refactor, dim3(nblocks), dim3(nthreads), args, smem, s);
}
cudaError_t launch_gather_map(cudaStream_t s, long long n, const int* map, const double* src, double* dst) {
  if (n <= 0) return cudaSuccess;
  k_gather_map<<<nblk(n, 256), 256, 0, s>>>(n, map, src, dst);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_chol_prepare(cudaStream_t s, int n, const double* A, double delta, double* F) {
  k_chol_prepare<<<nblk((long long)n * n, 256), 256, 0, s>>>(n, A, delta, F);
  note_launch();
  return cudaGetLastError();
}
int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}
int chol_max_blocks() {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol, 256, 0);
  return device_sms() * (per > 0 ? per : 1);
}
int chol_grid_cap(int n) {
  const int ntl = (n + 31) / 32;
  const int need = std::max(1, std::max((ntl - 1) * ntl / 2 * 4, (ntl + 7) / 8));
  return std::max(1, std::min(chol_max_blocks(), std::min(need, 2 * device_sms())));
}
cudaError_t launch_chol(cudaStream_t s, int n, double* F, double* dinv, int* st, unsigned* bar,
                        long long spin_limit, int nblocks) {
  void* args[] = {&F, &n, &dinv, &st, &bar, &spin_limit};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)k_chol, dim3(nblocks), dim3(256), args, 0, s);
}
cudaError_t launch_chol_solve(cudaStream_t s, int n, const double* F, const double* dinv, double* X, int nrhs) {
  if (nrhs <= 0) return cudaSuccess;
  size_t sm = (size_t)n * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = allow_max_smem((const void*)k_chol_solve);
    if (e != cudaSuccess) return e;
  }
  k_chol_solve<<<nrhs, 256, sm, s>>>(n, F, dinv, X, nrhs);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_permute_rows(cudaStream_t s, int n, int ncols, const int* idx, const double* src,
                                int ld_src, int src_colmajor, double* dst, int ld_dst, int dst_colmajor,
                                double alpha, int inverse) {
  long long total = (long long)n * ncols;
  if (total <= 0) return cudaSuccess;
  k_permute_rows<<<nblk(total, 256), 256, 0, s>>>(n, ncols, idx, src, ld_src, src_colmajor, dst, ld_dst,
                                                 dst_colmajor, alpha, inverse);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_axpby(cudaStream_t s, long long n, double a, const double* x, double b, const double* y,
                         double* z) {
  if (n <= 0) return cudaSuccess;
  k_axpby<<<nblk(n, 256), 256, 0, s>>>(n, a, x, b, y, z);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_scale_rows(cudaStream_t s, int n, int ncols, const double* d, const double* x, double* z,
                              double b, const double* y) {
  long long total = (long long)n * ncols;
  if (total <= 0) return cudaSuccess;
  k_scale_rows<<<nblk(total, 256), 256, 0, s>>>(n, ncols, d, x, z, b, y);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_absmax(cudaStream_t s, long long n, const double* x, double* out) {
  k_absmax<<<1, 1024, 0, s>>>(n, x, out);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_fill(cudaStream_t s, long long n, double v, double* x) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<nblk(n, 256), 256, 0, s>>>(n, v, x);
  note_launch();
  return cudaGetLastError();
}
// dst[i * ldd] = a * src[i * lds] + b * y[i * ldy]  (strided columns; y may be NULL)
__global__ void k_column_axpby(int n, double a, const double* __restrict__ src, long long lds, double b,
                               const double* __restrict__ y, long long ldy, double* __restrict__ dst, long long ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = a * src[(long long)i * lds];
  dst[(long long)i * ldd] = y ? fma(b, y[(long long)i * ldy], v) : v;
}
cudaError_t launch_column_axpby(cudaStream_t s, int n, double a, const double* src, long long lds, double b,
                                const double* y, long long ldy, double* dst, long long ldd) {
  if (n <= 0) return cudaSuccess;
  k_column_axpby<<<(n + 255) / 256, 256, 0, s>>>(n, a, src, lds, b, y, ldy, dst, ldd);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_set_identity(cudaStream_t s, int n, double* X, int ld) {
  k_set_identity<<<nblk((long long)n * n, 256), 256, 0, s>>>(n, X, ld);
  note_launch();
  return cudaGetLastError();
}

}  // namespace condipm

// ============================================================================
// Dataflow form of the blocked Cholesky (look-ahead without grid barriers).
// The CTAs split into a panel group (np CTAs) and an update group.  Step k:
//   panel group: wait until tile column k has received the step k-1 update
//     (counter cdone[k-1]), factor the diagonal tile (every panel CTA, in
//     shared memory; CTA 0 writes it back), solve the panel rows below it (one
//     row per warp), count the finished row groups into pdone[k];
//   update group: wait until pdone[k] is complete, then apply the step-k update
//     to the tiles (or 16x16 sub-tiles) it owns -- each tile has one owner CTA
//     for all steps, so a tile's updates stay in order -- doing the tiles of
//     column k+1 first and counting them into cdone[k].
// The next diagonal factorisation therefore starts as soon as its column is
// updated, while the rest of the trailing update proceeds.  Every wait is
// bounded and also ends when the status word reports an error; the panel
// values are read through L2 (ld.cg), since an SM's L1 may hold them from the
// previous step's update.
namespace condipm {
namespace {

__device__ __forceinline__ bool chol_wait(const unsigned* p, unsigned need, long long limit, int* st) {
  volatile int* vst = st;
  long long it = 0;
  unsigned v, ns = 32;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  while (v < need) {
    if (++it > limit) { atomicExch(&st[ST_TIMEOUT], 1); return false; }
    if ((it & 255) == 0 && (vst[ST_TIMEOUT] || vst[ST_CODE])) return false;
    __nanosleep(ns);
    ns = ns < 256 ? 2 * ns : 256;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  }
  return true;
}

__device__ __forceinline__ void red_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// row groups of the panel each panel CTA eliminates along with its diagonal
// tile (the rest are solved by substitution with the factored tile)
constexpr int CHOL_FUSED_GROUPS = 3;

__global__ void __launch_bounds__(256) k_chol_df(double* F, int n, double* dinv_out, int* st, unsigned* cnt,
                                                 int np, int sub_mode, long long spin_limit) {
  __shared__ double Ta[CNB][CNB + 1];
  __shared__ double Tb[CNB][CNB + 1];
  __shared__ double Tr[8 * CHOL_FUSED_GROUPS][CNB + 1];   // the panel rows eliminated with the diagonal tile
  __shared__ double dv[CNB];
  __shared__ unsigned short pairs[CNB * (CNB + 1) / 2];
  __shared__ int ok_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nt = (n + CNB - 1) / CNB;
  unsigned* pdone = cnt;          // [nt]
  unsigned* cdone = cnt + nt;     // [nt]
  unsigned* ccol = cnt + 2 * nt;  // [nt] full-tile mode: tiles of column k+2 updated at step k
  fill_pairs(pairs);
  __syncthreads();
  const bool panel = (int)blockIdx.x < np;
  const int nU = gridDim.x - np, ub = blockIdx.x - np;
  for (int k = 0; k < nt; ++k) {
    const int k0 = k * CNB, kb = min(CNB, n - k0);
    const int r0 = k0 + kb, nrows = n - r0;
    const int row_blocks = (nrows + nwarps - 1) / nwarps;
    const int m = nt - k - 1;
    if (panel) {
      if (tid == 0) {
        int ok = 1;
        if (k > 0) {
          // the 16 x 16 sub-tiles of column k on and below its diagonal,
          // counted at step k-1 (in both modes column k's last update is done
          // in sub-tiles)
          const int g16 = (n + 15) / 16;
          const unsigned need = (unsigned)((g16 - 2 * k) + (g16 - 2 * k - 1));
          ok = chol_wait(cdone + (k - 1), need, spin_limit, st);
        }
        ok_s = ok;
      }
      __syncthreads();
      if (!ok_s) return;
      // every panel CTA has finished with diagonal tile k-1 once column k is updated
      if (blockIdx.x == 0 && k > 0) write_tile_back(F, n, Tb, k - 1);
      if ((int)blockIdx.x == 0 || (int)blockIdx.x < row_blocks) {
        for (int t = tid; t < CNB * CNB; t += blockDim.x) {
          const int i = t / CNB, j = t % CNB;
          Ta[i][j] = (i < kb && j <= i) ? __ldcg(&F[(size_t)(k0 + i) * n + k0 + j]) : (i == j ? 1.0 : 0.0);
        }
        // this CTA's first row groups (groups blockIdx.x + g np, g < 3: rows
        // r0 + 8 (blockIdx.x + g np) ..) ride along in the tile's elimination
        int nfg = 0;
        while (nfg < CHOL_FUSED_GROUPS && (int)blockIdx.x + nfg * np < row_blocks) ++nfg;
        auto frow = [&](int rr) { return r0 + ((int)blockIdx.x + (rr >> 3) * np) * 8 + (rr & 7); };
        for (int t = tid; t < 8 * nfg * CNB; t += blockDim.x) {
          const int rr = t / CNB, j = t % CNB, r = frow(rr);
          Tr[rr][j] = (r < n && j < kb) ? __ldcg(&F[(size_t)r * n + k0 + j]) : 0.0;
        }
        __syncthreads();
        const int fail = block_chol_tile(Ta, dv, kb, pairs, Tr, 8 * nfg);
        if (fail >= 0) {
          if (tid == 0) set_status(st, DEV_NOT_PD, k0 + fail);
          return;
        }
        if (blockIdx.x == 0) {
          // the factored tile goes back to F only at the next step: the other
          // panel CTAs may still be reading the unfactored one now
          for (int t = tid; t < CNB * CNB; t += blockDim.x) Tb[t / CNB][t % CNB] = Ta[t / CNB][t % CNB];
          if (tid < kb) dinv_out[k0 + tid] = dv[tid];
        }
        int mine = nfg;
        for (int t = tid; t < 8 * nfg * CNB; t += blockDim.x) {
          const int rr = t / CNB, j = t % CNB, r = frow(rr);
          if (r < n && j < kb) F[(size_t)r * n + k0 + j] = Tr[rr][j];
        }
        // further row groups: one row per warp, forward substitution with L_kk
        for (int rb = blockIdx.x + nfg * np; rb < row_blocks; rb += np) {
          ++mine;
          const int r = r0 + rb * nwarps + warp;
          if (r < n) {
            double a = lane < kb ? __ldcg(&F[(size_t)r * n + k0 + lane]) : 0.0;
            for (int j = 0; j < kb; ++j) {
              const double xj = __shfl_sync(0xffffffffu, a, j) * dv[j];
              if (lane == j) a = xj;
              else if (lane > j) a = fma(-xj, Ta[lane][j], a);
            }
            if (lane < kb) F[(size_t)r * n + k0 + lane] = a;
          }
        }
        __syncthreads();
        if (tid == 0 && mine > 0) red_add_release(pdone + k, (unsigned)mine);
      }
      continue;
    }
    // ---- update group
    if (m == 0) continue;
    if (tid == 0) ok_s = chol_wait(pdone + k, (unsigned)row_blocks, spin_limit, st);
    __syncthreads();
    if (!ok_s) return;
    // ownership: the (sub-)tiles of the lower triangle are numbered column by
    // column, (sub-)column gj holding (sub-)rows gj .. gmax-1, and tile number t
    // belongs to update CTA t mod nU for every step.  The trailing triangle of a
    // step is a suffix of that numbering, so every CTA gets an equal share of
    // it.  Columns in order, column k+1 first.
    const int g = sub_mode ? 2 : 1;                   // (sub-)tiles per tile side
    const int gmax = sub_mode ? (n + 15) / 16 : nt;   // (sub-)rows in the matrix
    if (!sub_mode) {
      // Column k+1 first, as 16 x 16 sub-tiles shared out over all update CTAs
      // (the next panel waits on it: four CTAs per tile shorten that wait).
      // This is the last update of those entries, so it needs only their
      // owners' step k-1 updates done (counted in ccol[k-1]).
      {
        const int g16 = (n + 15) / 16, sc0 = 2 * (k + 1);
        const int n0 = g16 - sc0, n1 = g16 - sc0 - 1, nsub = n0 + n1;
        if (ub < nsub) {
          __syncthreads();   // every thread has read ok_s of the pdone wait
          if (tid == 0) ok_s = k == 0 || chol_wait(ccol + (k - 1), (unsigned)(nt - k - 1), spin_limit, st);
          __syncthreads();
          if (!ok_s) return;
        }
        for (int sidx = ub; sidx < nsub; sidx += nU) {
          const int sc = sidx < n0 ? sc0 : sc0 + 1;
          const int sr = sidx < n0 ? sc0 + sidx : sc0 + 1 + (sidx - n0);
          const int i0 = sr * 16, j0 = sc * 16;
          for (int t = tid; t < 16 * CNB; t += blockDim.x) {
            const int rr = t / CNB, l = t % CNB;
            Ta[rr][l] = (i0 + rr < n && l < kb) ? __ldcg(&F[(size_t)(i0 + rr) * n + k0 + l]) : 0.0;
            Tb[rr][l] = (j0 + rr < n && l < kb) ? __ldcg(&F[(size_t)(j0 + rr) * n + k0 + l]) : 0.0;
          }
          __syncthreads();
          const int rr = tid >> 4, cc = tid & 15;
          double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
          for (int l = 0; l < CNB; l += 2) {
            acc0 = fma(Ta[rr][l], Tb[cc][l], acc0);
            acc1 = fma(Ta[rr][l + 1], Tb[cc][l + 1], acc1);
          }
          const int gr = i0 + rr, gc = j0 + cc;
          if (gr < n && gc < n && gc <= gr) F[(size_t)gr * n + gc] -= acc0 + acc1;
          __syncthreads();
          if (tid == 0) red_add_release(cdone + k, 1u);
        }
      }
      // whole 32 x 32 tiles of columns k+2 ..: the owned tiles of this step in
      // order (rows of the CTA's residue class), the next tile's panels fetched
      // into registers while this one is computed (each thread moves rows
      // t / 32 + 8 q, column t % 32 of both panels); column k+2's are counted
      // into ccol[k] for the next step's sub-tiles
      auto first_row = [&](int gj) { return gj + (((ub - (gj * gmax - gj * (gj - 1) / 2)) % nU) + nU) % nU; };
      auto advance = [&](int& gi, int& gj) {
        gi += nU;
        while (gi >= gmax) {
          if (++gj >= gmax) return;
          gi = first_row(gj);
        }
      };
      int gj = k + 2, gi = gj < gmax ? first_row(gj) : gmax;
      if (gi >= gmax) { gi -= nU; advance(gi, gj); }
      double pa[4], pb[4];
      auto fetch = [&](int ti, int tj) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = (tid >> 5) + 8 * q, l = tid & 31;
          pa[q] = (ti * CNB + rr < n && l < kb) ? __ldcg(&F[(size_t)(ti * CNB + rr) * n + k0 + l]) : 0.0;
          pb[q] = (tj * CNB + rr < n && l < kb) ? __ldcg(&F[(size_t)(tj * CNB + rr) * n + k0 + l]) : 0.0;
        }
      };
      if (gj < gmax) fetch(gi, gj);
      while (gj < gmax) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rr = (tid >> 5) + 8 * q, l = tid & 31;
          Ta[rr][l] = pa[q];
          Tb[rr][l] = pb[q];
        }
        __syncthreads();
        int ni = gi, nj = gj;
        advance(ni, nj);
        if (nj < gmax) fetch(ni, nj);
        const int i0 = gi * CNB, j0 = gj * CNB;
        const int ty = tid >> 4, tx = tid & 15;
        double c00 = 0.0, c01 = 0.0, c10 = 0.0, c11 = 0.0;
#pragma unroll 8
        for (int l = 0; l < CNB; ++l) {
          const double a0 = Ta[ty][l], a1 = Ta[ty + 16][l];
          const double b0 = Tb[tx][l], b1 = Tb[tx + 16][l];
          c00 = fma(a0, b0, c00);
          c01 = fma(a0, b1, c01);
          c10 = fma(a1, b0, c10);
          c11 = fma(a1, b1, c11);
        }
        const int r0g = i0 + ty, r1g = i0 + ty + 16, c0g = j0 + tx, c1g = j0 + tx + 16;
        if (r0g < n && c0g <= r0g) F[(size_t)r0g * n + c0g] -= c00;
        if (r0g < n && c1g < n && c1g <= r0g) F[(size_t)r0g * n + c1g] -= c01;
        if (r1g < n && c0g <= r1g) F[(size_t)r1g * n + c0g] -= c10;
        if (r1g < n && c1g < n && c1g <= r1g) F[(size_t)r1g * n + c1g] -= c11;
        __syncthreads();
        if (tid == 0 && gj == k + 2) red_add_release(ccol + k, 1u);
        gi = ni;
        gj = nj;
      }
      continue;
    }
    for (int gj = g * (k + 1); gj < gmax; ++gj) {
      const bool col0 = gj < g * (k + 2);
      const int base = gj * gmax - gj * (gj - 1) / 2;   // number of tile (gj, gj)
      int gi = gj + (((ub - base) % nU) + nU) % nU;
      for (; gi < gmax; gi += nU) {
        const int hh = sub_mode ? 16 : CNB;
        const int i0 = gi * hh, j0 = gj * hh;
        if (sub_mode) {
          for (int t = tid; t < 16 * CNB; t += blockDim.x) {
            const int rr = t / CNB, l = t % CNB;
            Ta[rr][l] = (i0 + rr < n && l < kb) ? __ldcg(&F[(size_t)(i0 + rr) * n + k0 + l]) : 0.0;
            Tb[rr][l] = (j0 + rr < n && l < kb) ? __ldcg(&F[(size_t)(j0 + rr) * n + k0 + l]) : 0.0;
          }
          __syncthreads();
          const int rr = tid >> 4, cc = tid & 15;
          double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
          for (int l = 0; l < CNB; l += 2) {
            acc0 = fma(Ta[rr][l], Tb[cc][l], acc0);
            acc1 = fma(Ta[rr][l + 1], Tb[cc][l + 1], acc1);
          }
          const int gr = i0 + rr, gc = j0 + cc;
          if (gr < n && gc < n && gc <= gr) F[(size_t)gr * n + gc] -= acc0 + acc1;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int rr = (tid >> 5) + 8 * q, l = tid & 31;
            Ta[rr][l] = (i0 + rr < n && l < kb) ? __ldcg(&F[(size_t)(i0 + rr) * n + k0 + l]) : 0.0;
            Tb[rr][l] = (j0 + rr < n && l < kb) ? __ldcg(&F[(size_t)(j0 + rr) * n + k0 + l]) : 0.0;
          }
          __syncthreads();
          const int ty = tid >> 4, tx = tid & 15;
          double c00 = 0.0, c01 = 0.0, c10 = 0.0, c11 = 0.0;
#pragma unroll 8
          for (int l = 0; l < CNB; ++l) {
            const double a0 = Ta[ty][l], a1 = Ta[ty + 16][l];
            const double b0 = Tb[tx][l], b1 = Tb[tx + 16][l];
            c00 = fma(a0, b0, c00);
            c01 = fma(a0, b1, c01);
            c10 = fma(a1, b0, c10);
            c11 = fma(a1, b1, c11);
          }
          const int r0g = i0 + ty, r1g = i0 + ty + 16, c0g = j0 + tx, c1g = j0 + tx + 16;
          if (r0g < n && c0g <= r0g) F[(size_t)r0g * n + c0g] -= c00;
          if (r0g < n && c1g < n && c1g <= r0g) F[(size_t)r0g * n + c1g] -= c01;
          if (r1g < n && c0g <= r1g) F[(size_t)r1g * n + c0g] -= c10;
          if (r1g < n && c1g < n && c1g <= r1g) F[(size_t)r1g * n + c1g] -= c11;
        }
        __syncthreads();
        if (tid == 0 && col0) red_add_release(cdone + k, 1u);
      }
    }
  }
  if (blockIdx.x == 0 && nt > 0) write_tile_back(F, n, Tb, nt - 1);
}

}  // namespace

int chol_df_max_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_df, 256, 0);
  return sms * (per > 0 ? per : 1);
}

cudaError_t launch_chol_df(cudaStream_t s, int n, double* F, double* dinv, int* st, unsigned* cnt,
                           long long spin_limit, int nblocks, int np) {
  const int nt = (n + CNB - 1) / CNB;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * 3 * (size_t)nt, s);
  if (e != cudaSuccess) return e;
  const int nU = std::max(1, nblocks - np);
  const int sub_mode = (nt * (nt - 1) / 2 < 2 * nU) ? 1 : 0;
  void* args[] = {&F, &n, &dinv, &st, &cnt, &np, (void*)&sub_mode, &spin_limit};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)k_chol_df, dim3(nblocks), dim3(256), args, 0, s);
}

}  // namespace condipm

// ============================================================================
// Solves with the dense Cholesky factor for a few right-hand sides (the Newton
// step's reduced system, Sec. 3.4).  A column's forward and backward
// substitutions are chains of nt = ceil(n / 32) tile steps; one CTA per column
// leaves each step to one SM and walks the diagonal tile row by row.  Here a
// thread-block cluster takes one column: every CTA keeps a copy of the
// solution in shared memory, the row tiles are shared out over the CTAs, and a
// tile step is x_J = Linv_JJ part_J by the tile's owner (explicit inverses of
// the diagonal tiles, computed once per factorisation), written into every
// copy, one cluster barrier, then every CTA folds x_J into the partial sums of
// its later tiles.
#include <cooperative_groups.h>
namespace condipm {
namespace cgl = cooperative_groups;
namespace {

// Finv[I] = L_II^{-1} (32 x 32, zero outside the tile's kb x kb lower triangle):
// forward substitution on the identity, one row per step, 32 x 32 threads
__global__ void __launch_bounds__(1024) k_tile_inv(int n, const double* __restrict__ F,
                                                   const double* __restrict__ dinv, double* __restrict__ Finv) {
  __shared__ double Lt[CNB][CNB + 1];
  __shared__ double Y[CNB][CNB + 1];
  const int I = blockIdx.x, i0 = I * CNB, kb = min(CNB, n - i0);
  const int r = threadIdx.x / CNB, c = threadIdx.x % CNB;
  Lt[r][c] = (r < kb && c <= r) ? F[(size_t)(i0 + r) * n + i0 + c] : 0.0;
  Y[r][c] = (r == c && r < kb) ? 1.0 : 0.0;
  __syncthreads();
  for (int i = 0; i < kb; ++i) {
    if (r == i) Y[i][c] *= dinv[i0 + i];
    __syncthreads();
    if (r > i && r < kb) Y[r][c] = fma(-Lt[r][i], Y[i][c], Y[r][c]);
    __syncthreads();
  }
  Finv[(size_t)I * CNB * CNB + r * CNB + c] = Y[r][c];
}

// One cluster per right-hand side column (X row-major n x nrhs); CTA p owns
// the row tiles p, p + CL, ...; 32 warps, warp w handles row (or column) w of
// a tile with the lanes over the other index and a shuffle reduction.
__global__ void __launch_bounds__(1024, 1) k_chol_solve_cl(int n, const double* __restrict__ F,
                                                           const double* __restrict__ Finv, double* X, int nrhs) {
  extern __shared__ double smd[];
  __shared__ double* rx[16];
  cgl::cluster_group cl = cgl::this_cluster();
  const int p = int(cl.block_rank()), CL = int(cl.num_blocks());
  const int col = blockIdx.x / CL;
  const int nt = (n + CNB - 1) / CNB, nown = (nt - p + CL - 1) / CL;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* xv = smd;                      // nt * 32: this CTA's copy of the solution
  double* part = smd + (size_t)nt * CNB; // nown * 32: partial sums of the owned tiles
  if (threadIdx.x < CL) rx[threadIdx.x] = cl.map_shared_rank(xv, threadIdx.x);
  for (int i = threadIdx.x; i < nt * CNB; i += blockDim.x) xv[i] = 0.0;
  for (int o = 0; o < nown; ++o) {
    const int g = (p + o * CL) * CNB + lane;
    if (w == 0) part[o * CNB + lane] = g < n ? X[(size_t)g * nrhs + col] : 0.0;
  }
  cl.sync();
  // forward: L x = b
  for (int J = 0; J < nt; ++J) {
    if (J % CL == p) {
      const double* Li = Finv + (size_t)J * CNB * CNB;
      double v = Li[w * CNB + lane] * part[(J / CL) * CNB + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane < CL) rx[lane][J * CNB + w] = v;
    }
    cl.sync();
    // part_I -= L_IJ x_J for the owned tiles I > J (row w of the tile per warp)
    const double xj = xv[J * CNB + lane];
    const int gc = J * CNB + lane;
    for (int o = 0; o < nown; ++o) {
      const int I = p + o * CL;
      if (I <= J) continue;
      const int gr = I * CNB + w;
      double v = (gr < n && gc < n) ? F[(size_t)gr * n + gc] * xj : 0.0;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if (lane == 0) part[o * CNB + w] -= v;
    }
    __syncthreads();
  }
  // backward: L^T x = y, starting from the forward solution
  for (int o = 0; o < nown; ++o)
    if (w == 0) part[o * CNB + lane] = xv[(p + o * CL) * CNB + lane];
  cl.sync();   // no copy is overwritten before every CTA has read its y
  for (int I = nt - 1; I >= 0; --I) {
    if (I % CL == p) {
      const double* Li = Finv + (size_t)I * CNB * CNB;
      double v = Li[lane * CNB + w] * part[(I / CL) * CNB + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane < CL) rx[lane][I * CNB + w] = v;
    }
    cl.sync();
    // part_J -= L_IJ^T x_I for the owned tiles J < I (column w of the tile per warp)
    const int gr = I * CNB + lane;
    const double xi = xv[gr];
    for (int o = 0; o < nown; ++o) {
      const int J = p + o * CL;
      if (J >= I) continue;
      const int gc = J * CNB + w;
      double v = (gr < n && gc < n) ? F[(size_t)gr * n + gc] * xi : 0.0;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if (lane == 0) part[o * CNB + w] -= v;
    }
    __syncthreads();
  }
  if (p == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[(size_t)i * nrhs + col] = xv[i];
}

}  // namespace

cudaError_t launch_tile_inv(cudaStream_t s, int n, const double* F, const double* dinv, double* Finv) {
  const int nt = (n + CNB - 1) / CNB;
  if (nt <= 0) return cudaSuccess;
  k_tile_inv<<<nt, 1024, 0, s>>>(n, F, dinv, Finv);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_chol_solve_cl(cudaStream_t s, int n, const double* F, const double* Finv, double* X, int nrhs,
                                 int CL) {
  const int nt = (n + CNB - 1) / CNB;
  if (nrhs <= 0 || nt <= 0) return cudaSuccess;
  const size_t smem = sizeof(double) * ((size_t)nt * CNB + (size_t)((nt + CL - 1) / CL) * CNB);
  if (CL > 8) {
    cudaError_t e = allow_cluster16((const void*)k_chol_solve_cl);
    if (e != cudaSuccess) return e;
  }
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem((const void*)k_chol_solve_cl);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL * nrhs);
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_chol_solve_cl, n, F, Finv, X, nrhs);
}

}  // namespace condipm

namespace condipm {

cudaError_t launch_batch_prologue(cudaStream_t s, const BatchInst* I, int n, const int* const* boff,
                                  const int* nblocks) {
  if (n <= 0) return cudaSuccess;
  k_b_clear<<<nblocks[BOFF_X], BATCH_EW_THREADS, 0, s>>>(I, n, boff[BOFF_X]);
  note_launch();
  k_b_scatter<<<nblocks[BOFF_K], BATCH_EW_THREADS, 0, s>>>(I, n, boff[BOFF_K]);
  note_launch();
  k_b_rowmax<<<nblocks[BOFF_LU], BATCH_EW_THREADS, 0, s>>>(I, n, boff[BOFF_LU]);
  note_launch();
  return cudaGetLastError();
}

int batch_lu_max_blocks(int maxlen) {
  const size_t smem = (size_t)(256 / 32) * maxlen * sizeof(double);
  if (smem > 48 * 1024 && allow_max_smem((const void*)k_b_lu) != cudaSuccess) return 0;
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_b_lu, 256, smem);
  return device_sms() * per;
}

// cooperative: every warp of the grid is resident, which the flag waits rely on
cudaError_t launch_batch_lu(cudaStream_t s, const BatchInst* I, const int2* items, int nitems, int nblocks,
                            int maxlen, unsigned epoch, long long spin_limit) {
  if (nitems <= 0) return cudaSuccess;
  const size_t smem = (size_t)(256 / 32) * maxlen * sizeof(double);
  void* args[] = {(void*)&I, (void*)&items, (void*)&nitems, (void*)&epoch, (void*)&spin_limit, (void*)&maxlen};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)k_b_lu, dim3(nblocks), dim3(256), args, smem, s);
}

cudaError_t launch_batch_spmm(cudaStream_t s, const BatchInst* I, int n, const int* boff, int nblocks, int which) {
  if (n <= 0) return cudaSuccess;
  k_b_spmm<<<nblocks, BATCH_EW_THREADS, 0, s>>>(I, n, boff, which);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_status(cudaStream_t s, const BatchInst* I, int n, int* out) {
  if (n <= 0) return cudaSuccess;
  k_b_status<<<nblk((long long)n * ST_WORDS, 256), 256, 0, s>>>(I, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_kred(cudaStream_t s, const BatchInst* I, int n, const int* boffU, int nblocks) {
  if (n <= 0) return cudaSuccess;
  k_b_kred<<<nblocks, BATCH_EW_THREADS, 0, s>>>(I, n, boffU);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_chol(cudaStream_t s, const BatchInst* I, int n, int cl) {
  if (n <= 0) return cudaSuccess;
  if (cl > 8) {
    cudaError_t e = allow_cluster16((const void*)k_b_chol);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(n * cl);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_b_chol, I);
}

int batch_chol_clusters(int cl) {
  if (cl > 8 && allow_cluster16((const void*)k_b_chol) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(256);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, (const void*)k_b_chol, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

}  // namespace condipm

