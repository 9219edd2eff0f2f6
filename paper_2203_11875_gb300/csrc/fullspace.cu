// The linear solver of the hybrid full-space IPM (Sec. 4.3): the augmented
// system of Eq. kktmatrix:normal with the slack step eliminated, factorised on
// the GPU as a block LDL^T (fsplan.h describes the blocks, the ordering and
// the row form of the elimination) in place of the CPU MA27 factorisation the
// paper pairs with its GPU model.
//
//   * assembly: the block values are zeroed, W, G and A are scattered in
//     (every slot has one source) and the diagonals of Sigma_w + delta_w E_u
//     and -(Sigma_s^{-1} + delta_c) are added;
//   * factorisation: one warp per block row, rows taken in level order by a
//     cooperative grid (every row waits only on rows earlier in the list, whose
//     warps are resident, so the oldest unfinished row always proceeds); a row
//     waits for each of its L columns' flags (bounded acquire loads), forms
//     L_IK = W_IK D_K^{-1}, applies L_IK U_KJ to its later blocks, then inverts
//     its diagonal block D_I by Gauss-Jordan with partial pivoting inside the
//     block and publishes its flag (release);
//   * inertia: one thread per block, symmetric elimination with Bunch-Parlett
//     pivoting on the symmetrised D_I; the counts are summed (Sylvester's law)
//     and compared with (n_w, n_x + m, 0),
//     the inertia Theorem 3 requires (wrong inertia is reported as NOT_PD, as
//     for the condensed matrix);
//   * solves: forward with the unit block lower factor, backward with U = D L^T
//     and the inverse diagonal blocks, the same sync-free row scheme (the
//     backward pass takes the list in reverse);
//   * refinement against the full K_aug (with the factor's delta_w on the u
//     block) with the library's residual kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fsplan.h"
#include "internal.h"

namespace condipm {

struct FsDev {
  int nblk = 0;
  const int *bptr = nullptr, *brp = nullptr, *bci = nullptr, *bdiag = nullptr, *rows = nullptr;
  const long long *voff = nullptr, *doff = nullptr, *upd_ptr = nullptr;
  const int *upd_src = nullptr, *upd_dst = nullptr;
};

struct FsState {
  FsPlan F;
  FsDev d;
  long long *w_slot = nullptr, *g_slot = nullptr, *a_slot = nullptr, *diag_slot = nullptr;
  int *w_src = nullptr, *g_src = nullptr, *a_src = nullptr;
  int* kbpos = nullptr;          // [nw + nx + m] rows w (c-order) | lambda (elim. order) | y -> position
  double *val = nullptr, *dinv = nullptr, *sig_w = nullptr;
  unsigned* flags = nullptr;
  unsigned epoch = 0;
  int* cnt = nullptr;            // [4] n+, n-, n0 and a spare
  double* ldet = nullptr;        // [1] log|det M|
  double* X = nullptr;           // permuted right-hand sides (n x xcap)
  int xcap = 0;
  // CTAs of the cooperative row kernels (factorisation, solves): fewer resident
  // warps poll the flags less; timed on first use over FS_GRIDS CTAs per SM
  int grid_f = 1, grid_s = 1, per_f = 1, per_s = 1;
  bool tuned_f = false, tuned_s = false;
  float tune_f[4] = {}, tune_s[4] = {};
  bool sigma_set = false, factored = false;
  double delta_w = 0.0, delta_c = 0.0;
  int inertia[3] = {-1, -1, -1};
  double logdet = 0.0;
};

namespace {

constexpr int FS_THREADS = 128;
constexpr int FS_WARPS = FS_THREADS / 32;
constexpr int FS_KC = 4;   // right-hand-side columns per solve pass (FS_BMAX * FS_KC <= 32)
constexpr int FS_GRIDS[4] = {1, 2, 4, 8};   // CTAs per SM tried by the grid tuner
static_assert(FS_BMAX * FS_KC <= 32, "one lane per (row, column) of a block");

// lane 0 waits (bounded) until flags[k] == epoch with acquire semantics;
// false when the wait expired (st[ST_TIMEOUT] set) or another one did
__device__ __forceinline__ bool fs_wait(const unsigned* flags, int k, unsigned epoch, int* st, long long spin_limit,
                                        int lane) {
  int expired = 0;
  if (lane == 0) {
    volatile int* vst = st;
    unsigned f;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + k) : "memory");
    long long it = 0;
    unsigned ns = 32;
    while (f != epoch) {
      if (++it > spin_limit) { atomicExch(&st[ST_TIMEOUT], 1); expired = 1; break; }
      if ((it & 1023) == 0 && vst[ST_TIMEOUT]) { expired = 1; break; }
      __nanosleep(ns);
      ns = ns < 128 ? 2 * ns : 128;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + k) : "memory");
    }
  }
  expired = __shfl_sync(0xffffffffu, expired, 0);
  __syncwarp();   // orders lane 0's acquire before every lane's loads of row k
  return !expired;
}

// every lane's stores of row i are fenced, then lane 0 publishes the flag
__device__ __forceinline__ void fs_publish(unsigned* flags, int i, unsigned epoch, int lane) {
  __threadfence();
  __syncwarp();
  if (lane == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flags + i), "r"(epoch) : "memory");
  __syncwarp();
}

__global__ void k_fs_zero(long long n, double* __restrict__ v) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) v[t] = 0.0;
}

__global__ void k_fs_scatter(long long n, const long long* __restrict__ slot, const int* __restrict__ src,
                             const double* __restrict__ from, double* __restrict__ val) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) val[slot[t]] = from[src[t]];
}

// diagonals: Sigma_w (+ delta_w on u) on the w rows, -(1/Sigma_s + delta_c) on y
__global__ void k_fs_diag(int nw, int nu, int nx, int m, const long long* __restrict__ ds,
                          const double* __restrict__ sig_w, const double* __restrict__ sig_s, double delta_w,
                          double delta_c, double* __restrict__ val) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < nw) val[ds[u]] += sig_w[u] + (u < nu ? delta_w : 0.0);
  else if (u >= nw + nx && u < nw + nx + m) val[ds[u]] = -(1.0 / sig_s[u - nw - nx] + delta_c);
}

__global__ void __launch_bounds__(FS_THREADS) k_fs_factor(FsDev D, double* val, double* dinv, unsigned* flags,
                                                          unsigned epoch, int* st, long long spin_limit) {
  __shared__ double Lsh[FS_WARPS][FS_BMAX * FS_BMAX];
  __shared__ double Ash[FS_WARPS][FS_BMAX][2 * FS_BMAX + 1];
  __shared__ double Rsh[FS_WARPS][FS_BMAX];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // consecutive rows of the list go to different CTAs (different SMs)
  const int gw = blockIdx.x + gridDim.x * wib, nwarp = gridDim.x * FS_WARPS;
  double* L = Lsh[wib];
  double (*Aw)[2 * FS_BMAX + 1] = Ash[wib];
  for (int t = gw; t < D.nblk; t += nwarp) {
    const int I = D.rows[t];
    const int bI = D.bptr[I + 1] - D.bptr[I];
    const int qd = D.bdiag[I];
    // the flags of the next 32 L columns are read at once (one acquire load per
    // lane); only columns not yet published then cost a wait
    unsigned ready = 0;
    int win = -1;
    for (int q = D.brp[I]; q < qd; ++q) {
      const int K = D.bci[q], bK = D.bptr[K + 1] - D.bptr[K];
      if (win < 0 || q >= win + 32) {
        win = q;
        unsigned f = 0;
        if (q + lane < qd)
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + D.bci[q + lane]) : "memory");
        ready = __ballot_sync(0xffffffffu, q + lane < qd && f == epoch);
      }
      if (!((ready >> (q - win)) & 1u)) {
        if (!fs_wait(flags, K, epoch, st, spin_limit, lane)) return;
      } else {
        __syncwarp();   // orders the reading lane's acquire before every lane's loads of row K
      }
      double* Wik = val + D.voff[q];
      const double* Dk = dinv + D.doff[K];
      const int nIK = bI * bK;
      // L_IK = W_IK D_K^{-1}
      for (int e = lane; e < nIK; e += 32) {
        const int r = e / bK, c = e - r * bK;
        double acc = 0.0;
        for (int k = 0; k < bK; ++k) acc = fma(__ldcg(&Wik[r * bK + k]), __ldcg(&Dk[k * bK + c]), acc);
        L[e] = acc;
      }
      __syncwarp();
      for (int e = lane; e < nIK; e += 32) Wik[e] = L[e];
      // W_IJ -= L_IK U_KJ over the U blocks of row K, four updates in flight
      const long long u0 = D.upd_ptr[q], u1 = D.upd_ptr[q + 1];
      for (long long u = u0; u < u1; u += 4) {
        const double* Ub[4];
        double* Wb[4];
        int bJ[4], nE[4];
        int nmax = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (u + i < u1) {
            const int sx = D.upd_src[u + i], dx = D.upd_dst[u + i], J = D.bci[sx];
            bJ[i] = D.bptr[J + 1] - D.bptr[J];
            nE[i] = bI * bJ[i];
            Ub[i] = val + D.voff[sx];
            Wb[i] = val + D.voff[dx];
            nmax = max(nmax, nE[i]);
          } else {
            bJ[i] = 1;
            nE[i] = 0;
            Ub[i] = nullptr;
            Wb[i] = nullptr;
          }
        }
        for (int e = lane; e < nmax; e += 32) {
          double a[4] = {0.0, 0.0, 0.0, 0.0};
          int r[4], c[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            r[i] = e / bJ[i];
            c[i] = e - r[i] * bJ[i];
          }
          for (int k = 0; k < bK; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (e < nE[i]) a[i] = fma(L[r[i] * bK + k], __ldcg(&Ub[i][k * bJ[i] + c[i]]), a[i]);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (e < nE[i]) Wb[i][e] -= a[i];
        }
      }
      __syncwarp();
    }
    // D_I^{-1}: Gauss-Jordan on [D_I | I] with scaled partial pivoting (rows
    // weighted by their largest entry in D_I: the barrier terms make rows of
    // very different size near the optimum), lane c owns column c
    const double* Di = val + D.voff[qd];
    double* rs = Rsh[wib];
    bool singular = false;
#pragma unroll
    for (int r = 0; r < FS_BMAX; ++r) {
      double v = 0.0;
      if (r < bI && lane < 2 * bI) {
        v = lane < bI ? __ldcg(&Di[r * bI + lane]) : (lane - bI == r ? 1.0 : 0.0);
        Aw[r][lane] = v;
      }
      double a = lane < bI ? fabs(v) : 0.0;
      for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      if (r < bI && (!(a > 0.0) || !isfinite(a))) singular = true;
      if (lane == 0) rs[r] = a;
    }
    __syncwarp();
    for (int k = 0; k < bI && !singular; ++k) {
      int p = k;
      double best = -1.0;
      for (int r = k; r < bI; ++r) {
        const double v = fabs(Aw[r][k]) / rs[r];
        if (v > best) { best = v; p = r; }
      }
      if (!(best > 1e-15)) { singular = true; break; }
      __syncwarp();
      if (p != k) {
        if (lane < 2 * bI) {
          const double tmp = Aw[k][lane];
          Aw[k][lane] = Aw[p][lane];
          Aw[p][lane] = tmp;
        }
        if (lane == 0) {
          const double t2 = rs[k];
          rs[k] = rs[p];
          rs[p] = t2;
        }
      }
      __syncwarp();
      const double pinv = 1.0 / Aw[k][k];
      double f[FS_BMAX];
#pragma unroll
      for (int r = 0; r < FS_BMAX; ++r) f[r] = r < bI ? Aw[r][k] : 0.0;
      __syncwarp();
      if (lane < 2 * bI) {
        const double akc = Aw[k][lane] * pinv;
#pragma unroll
        for (int r = 0; r < FS_BMAX; ++r)
          if (r < bI && r != k) Aw[r][lane] = fma(-f[r], akc, Aw[r][lane]);
        Aw[k][lane] = akc;
      }
      __syncwarp();
    }
    if (singular) {
      if (lane == 0) set_status(st, DEV_SINGULAR, I);
    } else {
      double* Dv = dinv + D.doff[I];
      for (int e = lane; e < bI * bI; e += 32) {
        const int r = e / bI, c = e - r * bI;
        Dv[e] = Aw[r][bI + c];
      }
    }
    __syncwarp();
    fs_publish(flags, I, epoch, lane);
  }
}

// inertia and log|det| of each diagonal block by symmetric elimination with
// Bunch and Parlett's complete pivoting (1971) on (D + D^T) / 2, one thread per
// block: a 1 x 1 pivot on the largest diagonal entry when it is at least
// alpha = (1 + sqrt 17) / 8 times the largest off-diagonal one, else a 2 x 2
// pivot on that off-diagonal pair (negative determinant: one eigenvalue of each
// sign).  The Schur complements keep the sign of small pivots next to large
// barrier terms (the 2 x 2 [[Sigma, g], [g, 0]] gives Sigma and -g^2 / Sigma),
// which an absolute-accuracy eigenvalue method would not.
__global__ void k_fs_inertia(FsDev D, const double* __restrict__ val, int* cnt, double* ldet) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= D.nblk) return;
  const int b = D.bptr[I + 1] - D.bptr[I];
  const double* Di = val + D.voff[D.bdiag[I]];
  double a[FS_BMAX][FS_BMAX];
  bool live[FS_BMAX];
  for (int r = 0; r < b; ++r) {
    live[r] = true;
    for (int c = 0; c < b; ++c) a[r][c] = 0.5 * (Di[r * b + c] + Di[c * b + r]);
  }
  const double alpha = 0.6403882032022076;   // (1 + sqrt(17)) / 8
  int np = 0, nn = 0, nz = 0, left = b;
  double ld = 0.0;
  while (left > 0) {
    int k = -1, p = -1, q = -1;
    double dmax = -1.0, omax = 0.0;
    for (int i = 0; i < b; ++i) {
      if (!live[i]) continue;
      if (fabs(a[i][i]) > dmax) { dmax = fabs(a[i][i]); k = i; }
      for (int j = i + 1; j < b; ++j)
        if (live[j] && fabs(a[i][j]) > omax) { omax = fabs(a[i][j]); p = i; q = j; }
    }
    if (!(dmax > 0.0) && !(omax > 0.0)) { nz += left; break; }
    if (left == 1 || dmax >= alpha * omax) {
      const double piv = a[k][k];
      if (!isfinite(piv)) { nz += left; break; }
      if (piv > 0.0) ++np; else ++nn;
      ld += log(fabs(piv));
      live[k] = false;
      --left;
      for (int i = 0; i < b; ++i) {
        if (!live[i]) continue;
        const double f = a[i][k] / piv;
        for (int j = 0; j < b; ++j)
          if (live[j]) a[i][j] -= f * a[k][j];
      }
    } else {
      const double app = a[p][p], aqq = a[q][q], apq = a[p][q];
      const double det = app * aqq - apq * apq;   // < 0 by the pivot choice
      if (!isfinite(det) || !(det != 0.0)) { nz += left; break; }
      ++np;
      ++nn;
      ld += log(fabs(det));
      live[p] = live[q] = false;
      left -= 2;
      for (int i = 0; i < b; ++i) {
        if (!live[i]) continue;
        // [f_p, f_q] = [a_ip, a_iq] E^{-1},  E = [[app, apq], [apq, aqq]]
        const double fp = (a[i][p] * aqq - a[i][q] * apq) / det;
        const double fq = (a[i][q] * app - a[i][p] * apq) / det;
        for (int j = 0; j < b; ++j)
          if (live[j]) a[i][j] -= fp * a[p][j] + fq * a[q][j];
      }
    }
  }
  atomicAdd(&cnt[0], np);
  atomicAdd(&cnt[1], nn);
  atomicAdd(&cnt[2], nz);
  atomicAdd(ldet, ld);
}

// the inertia Theorem 3 asks for is (n_w, n_x + m, 0)
__global__ void k_fs_check(const int* __restrict__ cnt, int want_neg, int* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && (cnt[1] != want_neg || cnt[2] != 0)) set_status(st, DEV_NOT_PD, cnt[1]);
}

// KB rows -> permuted right-hand side of M: w and lambda rows as they are, y rows
// b_y - Sigma_s^{-1} b_s (the slack row folded in); kc of k columns from j0
__global__ void k_fs_gather(int nw, int nx, int m, int k, int j0, int kc, const int* __restrict__ kbpos,
                            const double* __restrict__ bw, const double* __restrict__ bl,
                            const double* __restrict__ by, const double* __restrict__ bs,
                            const double* __restrict__ sig_s, double* __restrict__ X) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rows = nw + nx + m;
  if (t >= (long long)rows * kc) return;
  const int r = int(t / kc), j = int(t % kc);
  double v;
  if (r < nw) v = bw[(long long)r * k + j0 + j];
  else if (r < nw + nx) v = bl[(long long)(r - nw) * k + j0 + j];
  else {
    const int i = r - nw - nx;
    v = by[(long long)i * k + j0 + j] - bs[(long long)i * k + j0 + j] / sig_s[i];
  }
  X[(long long)kbpos[r] * kc + j] = v;
}

// back to KB rows; p_s = Sigma_s^{-1} (b_s - p_y)
__global__ void k_fs_scatter_back(int nw, int nx, int m, int k, int j0, int kc, const int* __restrict__ kbpos,
                                  const double* __restrict__ X, const double* __restrict__ bs,
                                  const double* __restrict__ sig_s, double* __restrict__ pw, double* __restrict__ pl,
                                  double* __restrict__ py, double* __restrict__ ps) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rows = nw + nx + m;
  if (t >= (long long)rows * kc) return;
  const int r = int(t / kc), j = int(t % kc);
  const double v = X[(long long)kbpos[r] * kc + j];
  if (r < nw) pw[(long long)r * k + j0 + j] = v;
  else if (r < nw + nx) pl[(long long)(r - nw) * k + j0 + j] = v;
  else {
    const int i = r - nw - nx;
    const long long o = (long long)i * k + j0 + j;
    py[o] = v;
    ps[o] = (bs[o] - v) / sig_s[i];
  }
}

// lane-level bounded wait on flags[k] == epoch (acquire); false on expiry
__device__ __forceinline__ bool fs_wait_lane(const unsigned* flags, int k, unsigned epoch, int* st,
                                             long long spin_limit) {
  volatile int* vst = st;
  unsigned f;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + k) : "memory");
  long long it = 0;
  unsigned ns = 32;
  while (f != epoch) {
    if (++it > spin_limit) { atomicExch(&st[ST_TIMEOUT], 1); return false; }
    if ((it & 1023) == 0 && vst[ST_TIMEOUT]) return false;
    __nanosleep(ns);
    ns = ns < 256 ? 2 * ns : 256;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + k) : "memory");
  }
  return true;
}

// The two block triangular solves, X row-major n x kc (kc <= KC).  A row's
// dependency blocks are shared out over the lanes (lane t takes blocks t,
// t + 32, ...; each lane waits for its own blocks' flags), every lane keeps
// partial sums for the whole row block, and a butterfly reduction combines
// them.  Forward (unit block lower factor): y_I = x_I - sum_K L_IK y_K.
// Backward (U = D L^T, rows in reverse list order):
// x_I = D_I^{-1} (y_I - sum_J U_IJ x_J).
template <int KC, bool BWD>
__global__ void __launch_bounds__(FS_THREADS) k_fs_trsv(FsDev D, const double* val, const double* dinv, double* X,
                                                        int kc, unsigned* flags, unsigned epoch, int* st,
                                                        long long spin_limit) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x + gridDim.x * wib, nwarp = gridDim.x * FS_WARPS;
  for (int t = gw; t < D.nblk; t += nwarp) {
    const int I = BWD ? D.rows[D.nblk - 1 - t] : D.rows[t];
    const int p0 = D.bptr[I], bI = D.bptr[I + 1] - p0;
    const int q0 = BWD ? D.bdiag[I] + 1 : D.brp[I], q1 = BWD ? D.brp[I + 1] : D.bdiag[I];
    double acc[FS_BMAX][KC];
#pragma unroll
    for (int r = 0; r < FS_BMAX; ++r)
#pragma unroll
      for (int j = 0; j < KC; ++j) acc[r][j] = 0.0;
    bool ok = true;
    for (int q = q0 + lane; q < q1; q += 32) {
      const int K = D.bci[q];
      if (!fs_wait_lane(flags, K, epoch, st, spin_limit)) { ok = false; break; }
      const int pK = D.bptr[K], bK = D.bptr[K + 1] - pK;
      const double* B = val + D.voff[q];
      for (int c = 0; c < bK; ++c) {
        double xv[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) xv[j] = j < kc ? __ldcg(&X[(long long)(pK + c) * kc + j]) : 0.0;
#pragma unroll
        for (int r = 0; r < FS_BMAX; ++r)
          if (r < bI) {
            const double l = __ldcg(&B[r * bK + c]);
#pragma unroll
            for (int j = 0; j < KC; ++j) acc[r][j] = fma(l, xv[j], acc[r][j]);
          }
      }
    }
    if (__any_sync(0xffffffffu, !ok)) return;
    // sums over the lanes; afterwards every lane holds every row's sum
#pragma unroll
    for (int r = 0; r < FS_BMAX; ++r)
      if (r < bI)
#pragma unroll
        for (int j = 0; j < KC; ++j)
          for (int o = 16; o > 0; o >>= 1) acc[r][j] += __shfl_xor_sync(0xffffffffu, acc[r][j], o);
    const int r = lane / kc, j = lane - r * kc;
    const bool mine = r < bI;
    if (!BWD) {
      if (mine) {
        double sum = 0.0;
#pragma unroll
        for (int rr = 0; rr < FS_BMAX; ++rr)
#pragma unroll
          for (int jj = 0; jj < KC; ++jj)
            if (rr == r && jj == j) sum = acc[rr][jj];
        const long long o = (long long)(p0 + r) * kc + j;
        X[o] = __ldcg(&X[o]) - sum;
      }
    } else {
      double x = 0.0;
      if (mine) {
        const double* Dv = dinv + D.doff[I];
#pragma unroll
        for (int c = 0; c < FS_BMAX; ++c)
          if (c < bI) {
            double sc = 0.0;
#pragma unroll
            for (int jj = 0; jj < KC; ++jj)
              if (jj == j) sc = acc[c][jj];
            const double z = __ldcg(&X[(long long)(p0 + c) * kc + j]) - sc;
            x = fma(__ldcg(&Dv[r * bI + c]), z, x);
          }
      }
      __syncwarp();   // every lane has read y_I before it is overwritten
      if (mine) X[(long long)(p0 + r) * kc + j] = x;
    }
    fs_publish(flags, I, epoch, lane);
  }
}

// Sigma_w in c-order for the K_aug residual: sig_c[c] = sig_w[c2w[c]]
__global__ void k_fs_sigc(int nw, const int* __restrict__ c2w, const double* __restrict__ sig_w,
                          double* __restrict__ sig_c) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < nw) sig_c[c] = sig_w[c2w[c]];
}

inline int nb256(long long n) { return int(std::max(1LL, (n + 255) / 256)); }

template <class T>
int fs_upload(opf_handle* h, T** dst, const std::vector<T>& v) {
  const size_t n = std::max<size_t>(v.size(), 1);
  if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess) return OPF_ERR_OOM;
  h->allocs.push_back(*dst);
  if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return OPF_ERR_CUDA;
  return OPF_OK;
}

template <class T>
int fs_alloc(opf_handle* h, T** dst, size_t n) {
  n = std::max<size_t>(n, 1);
  if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess) return OPF_ERR_OOM;
  h->allocs.push_back(*dst);
  return cudaMemset(*dst, 0, n * sizeof(T)) == cudaSuccess ? OPF_OK : OPF_ERR_CUDA;
}

#define FS_TRY(x)                    \
  do {                               \
    const int r_ = (x);              \
    if (r_ != OPF_OK) return r_;     \
  } while (0)
#define FS_CK(x)                                        \
  do {                                                  \
    if ((x) != cudaSuccess) return OPF_ERR_CUDA;        \
  } while (0)

int launched() {
  note_launch();
  return cudaGetLastError() == cudaSuccess ? OPF_OK : OPF_ERR_CUDA;
}

int coop(const void* fn, int grid, void** args, cudaStream_t s) {
  note_launch();
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(FS_THREADS), args, 0, s) == cudaSuccess ? OPF_OK
                                                                                                   : OPF_ERR_CUDA;
}

// a cooperative grid of c CTAs per SM, within the occupancy and the rows
int fs_grid(const FsState* S, int per, int c) {
  const int need = (S->F.nblk + FS_WARPS - 1) / FS_WARPS;
  return std::max(1, std::min(device_sms() * std::min(per, c), need));
}

// the plan, its device copy and the buffers, on first use
int fs_ensure(opf_handle* h) {
  if (h->fs) return OPF_OK;
  FsState* S = new FsState();
  const std::string e = build_fs_plan(h->P, S->F);
  if (!e.empty()) {
    delete S;
    return OPF_ERR_INVALID_ARG;
  }
  h->fs = S;
  const FsPlan& F = S->F;
  const Plan& P = h->P;
  int *bptr, *brp, *bci, *bdiag, *rows, *usrc, *udst;
  long long *voff, *doff, *uptr;
  FS_TRY(fs_upload(h, &bptr, F.bptr));
  FS_TRY(fs_upload(h, &brp, F.brp));
  FS_TRY(fs_upload(h, &bci, F.bci));
  FS_TRY(fs_upload(h, &bdiag, F.bdiag));
  FS_TRY(fs_upload(h, &rows, F.rows));
  FS_TRY(fs_upload(h, &usrc, F.upd_src));
  FS_TRY(fs_upload(h, &udst, F.upd_dst));
  FS_TRY(fs_upload(h, &voff, F.voff));
  FS_TRY(fs_upload(h, &doff, F.doff));
  FS_TRY(fs_upload(h, &uptr, F.upd_ptr));
  S->d.nblk = F.nblk;
  S->d.bptr = bptr; S->d.brp = brp; S->d.bci = bci; S->d.bdiag = bdiag; S->d.rows = rows;
  S->d.voff = voff; S->d.doff = doff; S->d.upd_ptr = uptr; S->d.upd_src = usrc; S->d.upd_dst = udst;
  FS_TRY(fs_upload(h, &S->w_slot, F.w_slot));
  FS_TRY(fs_upload(h, &S->w_src, F.w_src));
  FS_TRY(fs_upload(h, &S->g_slot, F.g_slot));
  FS_TRY(fs_upload(h, &S->g_src, F.g_src));
  FS_TRY(fs_upload(h, &S->a_slot, F.a_slot));
  FS_TRY(fs_upload(h, &S->a_src, F.a_src));
  FS_TRY(fs_upload(h, &S->diag_slot, F.diag_slot));
  // KB rows: w in c-order (natural c2w[c]), lambda in elimination order
  // (natural row perm[i]), y natural
  std::vector<int> kb(P.nw + P.nx + P.m);
  for (int c = 0; c < P.nw; ++c) kb[c] = F.pos[P.c2w[c]];
  for (int i = 0; i < P.nx; ++i) kb[P.nw + i] = F.pos[P.nw + P.perm[i]];
  for (int r = 0; r < P.m; ++r) kb[P.nw + P.nx + r] = F.pos[P.nw + P.nx + r];
  FS_TRY(fs_upload(h, &S->kbpos, kb));
  FS_TRY(fs_alloc(h, &S->val, (size_t)F.nval));
  FS_TRY(fs_alloc(h, &S->dinv, (size_t)F.ndinv));
  FS_TRY(fs_alloc(h, &S->sig_w, (size_t)P.nw));
  FS_TRY(fs_alloc(h, &S->flags, (size_t)F.nblk));
  FS_TRY(fs_alloc(h, &S->cnt, 4));
  FS_TRY(fs_alloc(h, &S->ldet, 1));
  int per = 0, p2 = 0, p3 = 0, p4 = 0, p5 = 0;
  FS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fs_factor, FS_THREADS, 0));
  FS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p2, k_fs_trsv<FS_KC, false>, FS_THREADS, 0));
  FS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p3, k_fs_trsv<FS_KC, true>, FS_THREADS, 0));
  FS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p4, k_fs_trsv<1, false>, FS_THREADS, 0));
  FS_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p5, k_fs_trsv<1, true>, FS_THREADS, 0));
  S->per_f = std::max(1, per);
  S->per_s = std::max(1, std::min(std::min(p2, p3), std::min(p4, p5)));
  S->grid_f = fs_grid(S, S->per_f, 2);
  S->grid_s = fs_grid(S, S->per_s, 2);
  return OPF_OK;
}

int fs_xbuf(opf_handle* h, int kc) {
  FsState* S = h->fs;
  if (kc <= S->xcap) return OPF_OK;
  if (S->X) cudaFree(S->X);
  S->X = nullptr;
  S->xcap = 0;
  if (cudaMalloc(&S->X, sizeof(double) * (size_t)S->F.n * kc) != cudaSuccess) return OPF_ERR_OOM;
  S->xcap = kc;
  return OPF_OK;
}

}  // namespace

double fs_delta_w(const opf_handle* h) { return h->fs ? h->fs->delta_w : 0.0; }

void fs_release(opf_handle* h) {
  if (!h->fs) return;
  if (h->fs->X) cudaFree(h->fs->X);
  delete h->fs;
  h->fs = nullptr;
}

// Sigma of the next factorisations (device, natural order); the condensed
// state of the handle is dropped (its Sigma buffers now hold these)
int fs_set_sigma(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s) {
  FS_TRY(fs_ensure(h));
  FsState* S = h->fs;
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  FS_CK(cudaMemcpyAsync(S->sig_w, sig_u, sizeof(double) * P.nu, cudaMemcpyDeviceToDevice, s));
  FS_CK(cudaMemcpyAsync(S->sig_w + P.nu, sig_x, sizeof(double) * P.nx, cudaMemcpyDeviceToDevice, s));
  if (P.m > 0) FS_CK(cudaMemcpyAsync(h->sig_s, sig_s, sizeof(double) * P.m, cudaMemcpyDeviceToDevice, s));
  k_fs_sigc<<<nb256(P.nw), 256, 0, s>>>(P.nw, h->c2w, S->sig_w, h->sig_c);
  FS_TRY(launched());
  S->sigma_set = true;
  S->factored = false;
  h->have_condense = false;
  h->have_factor = false;
  h->psi_valid = false;
  h->sens_ready = false;
  h->fr_ready = false;
  h->fr_have_b = false;
  return OPF_OK;
}

// assemble M with (delta_w, delta_c), factorise, count the inertia; the device
// status reports SINGULAR, TIMEOUT or NOT_PD (wrong inertia)
namespace {

int fs_assemble(opf_handle* h, double delta_w, double delta_c) {
  FsState* S = h->fs;
  const Plan& P = h->P;
  const FsPlan& F = S->F;
  cudaStream_t s = h->s;
  k_fs_zero<<<nb256(F.nval), 256, 0, s>>>(F.nval, S->val);
  FS_TRY(launched());
  const long long nW = (long long)F.w_slot.size(), nG = (long long)F.g_slot.size(), nA = (long long)F.a_slot.size();
  if (nW) { k_fs_scatter<<<nb256(nW), 256, 0, s>>>(nW, S->w_slot, S->w_src, h->Wval, S->val); FS_TRY(launched()); }
  if (nG) { k_fs_scatter<<<nb256(nG), 256, 0, s>>>(nG, S->g_slot, S->g_src, h->Gval, S->val); FS_TRY(launched()); }
  if (nA) { k_fs_scatter<<<nb256(nA), 256, 0, s>>>(nA, S->a_slot, S->a_src, h->Aval, S->val); FS_TRY(launched()); }
  k_fs_diag<<<nb256(F.n), 256, 0, s>>>(P.nw, P.nu, P.nx, P.m, S->diag_slot, S->sig_w, h->sig_s, delta_w, delta_c,
                                       S->val);
  return launched();
}

int fs_launch_factor(opf_handle* h, int grid) {
  FsState* S = h->fs;
  unsigned ep = ++S->epoch;
  long long spin = h->spin_limit;
  FsDev d = S->d;
  void* args[] = {&d, &S->val, &S->dinv, &S->flags, &ep, &h->st, &spin};
  return coop((const void*)k_fs_factor, grid, args, h->s);
}

// the factorisation at each candidate grid on the same matrix (re-assembled
// before each), timed with events; the fastest is kept
int fs_tune_factor(opf_handle* h, double delta_w, double delta_c) {
  FsState* S = h->fs;
  cudaEvent_t a = nullptr, b = nullptr;
  FS_CK(cudaEventCreate(&a));
  FS_CK(cudaEventCreate(&b));
  float best = 1e30f;
  int pick = S->grid_f;
  int rc = OPF_OK;
  for (int i = 0; i < 4 && rc == OPF_OK; ++i) {
    S->tune_f[i] = 0.f;
    if (FS_GRIDS[i] > S->per_f) continue;
    const int g = fs_grid(S, S->per_f, FS_GRIDS[i]);
    rc = fs_assemble(h, delta_w, delta_c);
    if (rc == OPF_OK && cudaEventRecord(a, h->s) != cudaSuccess) rc = OPF_ERR_CUDA;
    if (rc == OPF_OK) rc = fs_launch_factor(h, g);
    if (rc == OPF_OK && cudaEventRecord(b, h->s) != cudaSuccess) rc = OPF_ERR_CUDA;
    if (rc == OPF_OK && cudaEventSynchronize(b) != cudaSuccess) rc = OPF_ERR_CUDA;
    float ms = 0.f;
    if (rc == OPF_OK) cudaEventElapsedTime(&ms, a, b);
    S->tune_f[i] = ms;
    if (rc == OPF_OK && ms < best) { best = ms; pick = g; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  FS_TRY(rc);
  S->grid_f = pick;
  S->tuned_f = true;
  return OPF_OK;
}

}  // namespace

// assemble M with (delta_w, delta_c), factorise, count the inertia; the device
// status reports SINGULAR, TIMEOUT or NOT_PD (wrong inertia)
int fs_factor_async(opf_handle* h, double delta_w, double delta_c) {
  FsState* S = h->fs;
  if (!S || !S->sigma_set || !h->have_W) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  const FsPlan& F = S->F;
  cudaStream_t s = h->s;
  if (!S->tuned_f && !h->profiling) FS_TRY(fs_tune_factor(h, delta_w, delta_c));
  ph_begin(h, OPF_PHASE_ASSEMBLE);
  FS_TRY(fs_assemble(h, delta_w, delta_c));
  ph_end(h);
  ph_begin(h, OPF_PHASE_CHOL);
  FS_TRY(fs_launch_factor(h, S->grid_f));
  FS_CK(cudaMemsetAsync(S->cnt, 0, sizeof(int) * 4, s));
  FS_CK(cudaMemsetAsync(S->ldet, 0, sizeof(double), s));
  k_fs_inertia<<<nb256(F.nblk), 256, 0, s>>>(S->d, S->val, S->cnt, S->ldet);
  FS_TRY(launched());
  k_fs_check<<<1, 32, 0, s>>>(S->cnt, P.nx + P.m, h->st);
  FS_TRY(launched());
  ph_end(h);
  S->delta_w = delta_w;
  S->delta_c = delta_c;
  // the K_aug residual of the refinement carries the same dual regularisation
  h->delta_c = delta_c;
  S->factored = true;
  return OPF_OK;
}

// inertia and log|det| of the last factorisation (host; synchronises)
int fs_read_inertia(opf_handle* h, int* inertia, double* logdet) {
  FsState* S = h->fs;
  if (!S || !S->factored) return OPF_ERR_INVALID_ARG;
  int c[4];
  double ld = 0.0;
  FS_CK(cudaMemcpyAsync(c, S->cnt, sizeof(c), cudaMemcpyDeviceToHost, h->s));
  FS_CK(cudaMemcpyAsync(&ld, S->ldet, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  FS_CK(cudaStreamSynchronize(h->s));
  for (int i = 0; i < 3; ++i) S->inertia[i] = c[i];
  S->logdet = ld;
  if (inertia) for (int i = 0; i < 3; ++i) inertia[i] = c[i];
  if (logdet) *logdet = ld;
  return OPF_OK;
}

namespace {

int fs_launch_solves(opf_handle* h, int kc, int grid) {
  FsState* S = h->fs;
  long long spin = h->spin_limit;
  FsDev d = S->d;
  unsigned ep = ++S->epoch;
  void* fa[] = {&d, &S->val, &S->dinv, &S->X, &kc, &S->flags, &ep, &h->st, &spin};
  FS_TRY(coop(kc == 1 ? (const void*)k_fs_trsv<1, false> : (const void*)k_fs_trsv<FS_KC, false>, grid, fa, h->s));
  unsigned ep2 = ++S->epoch;
  void* ba[] = {&d, &S->val, &S->dinv, &S->X, &kc, &S->flags, &ep2, &h->st, &spin};
  return coop(kc == 1 ? (const void*)k_fs_trsv<1, true> : (const void*)k_fs_trsv<FS_KC, true>, grid, ba, h->s);
}

int fs_gather(opf_handle* h, int k, int j0, int kc, const KB& b) {
  FsState* S = h->fs;
  const Plan& P = h->P;
  const int rows = P.nw + P.nx + P.m;
  k_fs_gather<<<nb256((long long)rows * kc), 256, 0, h->s>>>(P.nw, P.nx, P.m, k, j0, kc, S->kbpos, b.w, b.l, b.y,
                                                              b.s, h->sig_s, S->X);
  return launched();
}

// the two solves at each candidate grid on the first right-hand side, timed
int fs_tune_solves(opf_handle* h, int k, const KB& b) {
  FsState* S = h->fs;
  const int kc = std::min(FS_KC, k);
  cudaEvent_t a = nullptr, e = nullptr;
  FS_CK(cudaEventCreate(&a));
  FS_CK(cudaEventCreate(&e));
  float best = 1e30f;
  int pick = S->grid_s;
  int rc = OPF_OK;
  for (int i = 0; i < 4 && rc == OPF_OK; ++i) {
    S->tune_s[i] = 0.f;
    if (FS_GRIDS[i] > S->per_s) continue;
    const int g = fs_grid(S, S->per_s, FS_GRIDS[i]);
    rc = fs_gather(h, k, 0, kc, b);
    if (rc == OPF_OK && cudaEventRecord(a, h->s) != cudaSuccess) rc = OPF_ERR_CUDA;
    if (rc == OPF_OK) rc = fs_launch_solves(h, kc, g);
    if (rc == OPF_OK && cudaEventRecord(e, h->s) != cudaSuccess) rc = OPF_ERR_CUDA;
    if (rc == OPF_OK && cudaEventSynchronize(e) != cudaSuccess) rc = OPF_ERR_CUDA;
    float ms = 0.f;
    if (rc == OPF_OK) cudaEventElapsedTime(&ms, a, e);
    S->tune_s[i] = ms;
    if (rc == OPF_OK && ms < best) { best = ms; pick = g; }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(e);
  FS_TRY(rc);
  S->grid_s = pick;
  S->tuned_s = true;
  return OPF_OK;
}

}  // namespace

// p = K_aug^{-1} b for k right-hand sides in the KB layout, through M
int fs_core(opf_handle* h, int k, const KB& b, const KB& p) {
  FsState* S = h->fs;
  if (!S || !S->factored) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int rows = P.nw + P.nx + P.m;
  FS_TRY(fs_xbuf(h, FS_KC));
  if (!S->tuned_s && !h->profiling) FS_TRY(fs_tune_solves(h, k, b));
  ph_begin(h, OPF_PHASE_RECOVER);
  for (int j0 = 0; j0 < k; j0 += FS_KC) {
    const int kc = std::min(FS_KC, k - j0);
    FS_TRY(fs_gather(h, k, j0, kc, b));
    FS_TRY(fs_launch_solves(h, kc, S->grid_s));
    k_fs_scatter_back<<<nb256((long long)rows * kc), 256, 0, s>>>(P.nw, P.nx, P.m, k, j0, kc, S->kbpos, S->X, b.s,
                                                                   h->sig_s, p.w, p.l, p.y, p.s);
    FS_TRY(launched());
  }
  ph_end(h);
  return OPF_OK;
}

// K_aug p = -r for k right-hand sides (col-major n_kkt x k, natural order, as
// opf_kkt_solve) through the block factor, with up to `refine` corrections
int fs_solve_impl(opf_handle* h, const double* rhs, double* step, int k, int refine, int* steps, double* res) {
  FsState* S = h->fs;
  if (!S || !S->factored) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nw = P.nw, m = P.m, nx = P.nx;
  const size_t N = kkt_rows(P);
  const size_t extra = kkt_refine_scratch(P, k);
  double* ws = workspace(h, 2 * N * (size_t)k + extra + 8);
  if (!ws) return OPF_ERR_OOM;
  const KB b = kb_at(P, ws, k);
  const KB p = kb_at(P, ws + N * k, k);
  double* scratch = ws + 2 * N * k;
  FS_CK(launch_permute_rows(s, nw, k, h->c2w, rhs, int(N), 1, b.w, k, 0, -1.0, 0));
  FS_CK(launch_permute_rows(s, m, k, nullptr, rhs + nw, int(N), 1, b.s, k, 0, -1.0, 0));
  FS_CK(launch_permute_rows(s, nx, k, h->perm, rhs + nw + m, int(N), 1, b.l, k, 0, -1.0, 0));
  FS_CK(launch_permute_rows(s, m, k, nullptr, rhs + nw + m + nx, int(N), 1, b.y, k, 0, -1.0, 0));
  int st = 0;
  double fr = 0.0;
  if (refine > 0) FS_TRY(kkt_refine(h, k, b, p, true, false, refine, scratch, &fr, &st, true));
  else FS_TRY(fs_core(h, k, b, p));
  if (steps) *steps = st;
  if (res) *res = fr;
  FS_CK(launch_permute_rows(s, nw, k, h->c2w, p.w, k, 0, step, int(N), 1, 1.0, 1));
  FS_CK(launch_permute_rows(s, m, k, nullptr, p.s, k, 0, step + nw, int(N), 1, 1.0, 0));
  FS_CK(launch_permute_rows(s, nx, k, h->perm, p.l, k, 0, step + nw + m, int(N), 1, 1.0, 1));
  FS_CK(launch_permute_rows(s, m, k, nullptr, p.y, k, 0, step + nw + m + nx, int(N), 1, 1.0, 0));
  return OPF_OK;
}

int fs_tuning(const opf_handle* h, int* grids, float* ms) {
  if (!h->fs) return OPF_ERR_INVALID_ARG;
  if (grids) { grids[0] = h->fs->grid_f; grids[1] = h->fs->grid_s; }
  if (ms) for (int i = 0; i < 4; ++i) { ms[i] = h->fs->tune_f[i]; ms[4 + i] = h->fs->tune_s[i]; }
  return OPF_OK;
}

int fs_plan_stats(const opf_handle* h, int* nblocks, int* levels, long long* nnz_l, long long* flops) {
  if (!h->fs) return OPF_ERR_INVALID_ARG;
  const FsPlan& F = h->fs->F;
  if (nblocks) *nblocks = F.nblk;
  if (levels) *levels = F.levels;
  if (nnz_l) *nnz_l = F.nnz_l;
  if (flops) *flops = F.flops;
  return OPF_OK;
}

}  // namespace condipm

using namespace condipm;

extern "C" int opf_fullspace_factor(opf_handle* h, const double* sig_u, const double* sig_x, const double* sig_s,
                                    double delta_w, double delta_c, int* inertia) {
  if (!h || !sig_u || !sig_x || (h->P.m > 0 && !sig_s) || !(delta_w >= 0.0) || !(delta_c >= 0.0) ||
      !std::isfinite(delta_w) || !std::isfinite(delta_c))
    return OPF_ERR_INVALID_ARG;
  if (!h->have_W) return OPF_ERR_INVALID_ARG;
  FS_TRY(fs_set_sigma(h, sig_u, sig_x, sig_s));
  FS_TRY(fs_factor_async(h, delta_w, delta_c));
  const int rc = read_status(h, nullptr);
  FS_TRY(fs_read_inertia(h, inertia, nullptr));
  if (rc != OPF_OK) h->fs->factored = rc == OPF_ERR_NOT_PD;   // a wrong-inertia factor still solves
  return rc;
}

extern "C" int opf_fullspace_solve(opf_handle* h, const double* rhs, double* step, int nrhs, int refine, int* steps,
                                   double* residual) {
  if (!h || !rhs || !step || nrhs < 1 || refine < 0) return OPF_ERR_INVALID_ARG;
  if (!h->fs || !h->fs->factored) return OPF_ERR_INVALID_ARG;
  FS_TRY(fs_solve_impl(h, rhs, step, nrhs, refine, steps, residual));
  return read_status(h, nullptr);
}

extern "C" int opf_fullspace_stats(opf_handle* h, int* nblocks, int* levels, long long* nnz_l, long long* flops,
                                   double* logabsdet, int* inertia) {
  if (!h) return OPF_ERR_INVALID_ARG;
  FS_TRY(fs_ensure(h));
  FS_TRY(fs_plan_stats(h, nblocks, levels, nnz_l, flops));
  if (logabsdet) *logabsdet = h->fs->factored ? h->fs->logdet : 0.0;
  if (inertia) for (int i = 0; i < 3; ++i) inertia[i] = h->fs->factored ? h->fs->inertia[i] : -1;
  return OPF_OK;
}

extern "C" int opf_fullspace_tuning(const opf_handle* h, int* grids, float* ms) {
  if (!h) return OPF_ERR_INVALID_ARG;
  return fs_tuning(h, grids, ms);
}
