// Solves with the augmented KKT matrix through its condensed form, the residual
// of the full K_aug, and iterative refinement.
//
// K_aug (Eq. kktmatrix:normal with the +I slack coupling of h(x, u) + s = 0):
//   [ W + Sigma_w   0        G^T   A^T ] [p_w]   [b_w]
//   [ 0             Sigma_s  0     I   ] [p_s] = [b_s]
//   [ G             0        0     0   ] [p_l]   [b_l]
//   [ A             I        0     0   ] [p_y]   [b_y]
// Eliminating p_s, p_y (Theorem 2) and then p_x, p_l (Theorem 1):
//   p_s = b_y - A p_w,   p_y = b_s - Sigma_s p_s,
//   bt_w = b_w - A^T (b_s - Sigma_s b_y),   K = W + Sigma_w + A^T Sigma_s A,
//   q = G_x^{-1} b_l,   e = bt_w - K [0; q],
//   Kred p_u = e_u - G_u^T G_x^{-T} e_x,
//   p_x = G_x^{-1} (b_l - G_u p_u),   p_l = G_x^{-T} (bt_w,x - [K p_w]_x).
// Four multi-RHS solves with G_x (three when b_l = 0) and one with Kred.
// With the dual regularisation delta_c of the inequality rows (-delta_c I in the
// (p_y, p_y) block, folded into K by opf_kkt_factor), the same elimination reads
//   p_s = (b_y' - A p_w) / (1 + delta_c Sigma_s),   b_y' = b_y + delta_c b_s,
//   p_y = b_s - Sigma_t (b_y' - A p_w),   Sigma_t = Sigma_s / (1 + delta_c Sigma_s),
// i.e. Sigma_t in place of Sigma_s, b_y' in place of b_y, and a scaled p_s.
//
// Internal layout of k right-hand sides: row-major with k lanes (element (i, j)
// at X[i*k + j]); the w block in c-order ([u; x in elimination order]), the
// lambda block in elimination order, s and y in natural order.
//
// Near the end of an interior-point solve Sigma spans many orders of magnitude
// and Kred's condition number grows like 1/mu, so one condensed solve leaves a
// residual well above rounding.  kkt_refine applies the classic fixed-precision
// iterative refinement: r = b - K_aug z with the full sparse K_aug, z += solve(r).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/condipm.h"
#include "internal.h"

namespace condipm {
namespace {

#define CKK(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      note_cuda_error(e_);                \
      return OPF_ERR_CUDA;                \
    }                                     \
  } while (0)
#define TRYK(x)                  \
  do {                           \
    int r_ = (x);                \
    if (r_ != OPF_OK) return r_; \
  } while (0)

inline int nblk(long long n, int t) { return int((n + t - 1) / t); }

// z = d .* x  (row scaling, k lanes per row), then z = y - z when y is given
__global__ void k_rows_scale_sub(int n, int k, const double* __restrict__ d, const double* __restrict__ x,
                                 const double* __restrict__ y, double* __restrict__ z) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * k) return;
  const double v = d[t / k] * x[t];
  z[t] = y ? y[t] - v : v;
}

// R_s = b_s - Sigma_s z_s - z_y
__global__ void k_res_s(int m, int k, const double* __restrict__ sig, const double* __restrict__ b,
                        const double* __restrict__ zs, const double* __restrict__ zy, double* __restrict__ R) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)m * k) return;
  R[t] = b[t] - fma(sig[t / k], zs[t], zy[t]);
}

// x <- d .* x (k lanes per row)
__global__ void k_rows_scale_inplace(int n, int k, const double* __restrict__ d, double* x) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n * k) return;
  x[t] *= d[t / k];
}

__global__ void k_absmax_partial(long long n, const double* __restrict__ x, double* __restrict__ out) {
  __shared__ double sh[256];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v = fmax(v, fabs(x[i]));
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// out(i, j) = base(i, j) + alpha * sum_c M(i, c) V(c, j)   (i < n, j < k <= 4;
// M row-major with leading dimension ld, V and out row-major with k lanes);
// one warp per row, lanes over c
__global__ void k_dense_rows(int n, int ncol, int k, const double* __restrict__ M, long long ld,
                             const double* __restrict__ V, const double* __restrict__ base, double alpha,
                             double* __restrict__ out) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  // four passes of 32 columns in flight at once (their loads independent), each
  // with its own accumulators, summed at the end
  double acc[4][4] = {};
  const double* Mi = M + (long long)i * ld;
  int cc = lane;
  for (; cc + 96 < ncol; cc += 128) {
    double m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) m[u] = __ldcs(&Mi[cc + 32 * u]);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < k) acc[u][j] = fma(m[u], V[(long long)(cc + 32 * u) * k + j], acc[u][j]);
  }
  for (; cc < ncol; cc += 32) {
    const double m = __ldcs(&Mi[cc]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j < k) acc[0][j] = fma(m, V[(long long)cc * k + j], acc[0][j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j < k) {
      double a = (acc[0][j] + acc[1][j]) + (acc[2][j] + acc[3][j]);
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) out[(long long)i * k + j] = (base ? base[(long long)i * k + j] : 0.0) + alpha * a;
    }
  }
}

// the same for one right-hand side (the interior-point step): eight loads of
// the row in flight per lane, each with its own accumulator
__global__ void __launch_bounds__(256) k_dense_rows1(int n, int ncol, const double* __restrict__ M, long long ld,
                                                     const double* __restrict__ V, const double* __restrict__ base,
                                                     double alpha, double* __restrict__ out) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  double acc[8] = {};
  const double* Mi = M + (long long)i * ld;
  int cc = lane;
  for (; cc + 224 < ncol; cc += 256) {
    double m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = __ldcs(&Mi[cc + 32 * u]);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] = fma(m[u], __ldg(&V[cc + 32 * u]), acc[u]);
  }
  for (; cc < ncol; cc += 32) acc[0] = fma(__ldcs(&Mi[cc]), __ldg(&V[cc]), acc[0]);
  double a = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) out[i] = (base ? base[i] : 0.0) + alpha * a;
}

int launched() {
  note_launch();
  return cudaGetLastError() == cudaSuccess ? OPF_OK : OPF_ERR_CUDA;
}

}  // namespace

size_t kkt_rows(const Plan& P) { return (size_t)P.nw + 2 * (size_t)P.m + P.nx; }
size_t kkt_core_scratch(const Plan& P) { return 3 * (size_t)P.nw + 2 * (size_t)P.m; }
size_t kkt_refine_scratch(const Plan& P, int k) {
  return (2 * kkt_rows(P) + kkt_core_scratch(P)) * (size_t)k + 512;
}

KB kb_at(const Plan& P, double* base, int k) {
  KB b;
  b.w = base;
  b.s = b.w + (size_t)P.nw * k;
  b.l = b.s + (size_t)P.m * k;
  b.y = b.l + (size_t)P.nx * k;
  return b;
}

int kkt_recover(opf_handle* h, int k, const KB& b, const KB& p, bool bl_zero, double* scratch);

int kkt_core(opf_handle* h, int k, const KB& b, const KB& p, bool bl_zero, double* scratch) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  double* Bt = scratch;                   // bt_w  (nw x k)
  double* E = Bt + (size_t)nw * k;        // e     (nw x k)
  double* D0 = E + (size_t)nw * k;        // [0; q](nw x k)
  double* U = D0 + (size_t)nw * k;        // Sigma_s b_y - b_s (m x k)
  double* Byr = U + (size_t)m * k;        // b_y' = b_y + delta_c b_s (m x k, delta_c > 0)
  const bool dc = h->delta_c > 0.0;
  const double* sig = dc ? h->sig_se : h->sig_s;
  const double* by = b.y;
  ph_begin(h, OPF_PHASE_RHS);
  if (dc) {
    CKK(launch_axpby(s, (long long)m * k, 1.0, b.y, h->delta_c, b.s, Byr));
    by = Byr;
  }
  // bt_w = b_w + A^T (Sigma_s b_y - b_s)
  k_rows_scale_sub<<<nblk((long long)m * k, 256), 256, 0, s>>>(m, k, sig, by, nullptr, U);
  TRYK(launched());
  CKK(launch_axpby(s, (long long)m * k, 1.0, U, -1.0, b.s, U));
  CKK(cudaMemcpyAsync(Bt, b.w, sizeof(double) * (size_t)nw * k, cudaMemcpyDeviceToDevice, s));
  CKK(launch_spmm(s, nw, h->AT_rp, h->AT_ci, h->Aval, h->AT_map, U, k, 1, Bt, k, 1, k, 1.0, 1.0));
  CKK(cudaMemcpyAsync(E, Bt, sizeof(double) * (size_t)nw * k, cudaMemcpyDeviceToDevice, s));
  if (!bl_zero) {
    // q = G_x^{-1} b_l ; e = bt_w - K [0; q]
    CKK(cudaMemsetAsync(D0, 0, sizeof(double) * (size_t)nu * k, s));
    CKK(cudaMemcpyAsync(D0 + (size_t)nu * k, b.l, sizeof(double) * (size_t)nx * k, cudaMemcpyDeviceToDevice, s));
    TRYK(lu_solve_perm(h, 0, D0 + (size_t)nu * k, k, 1, k));
    CKK(launch_spmm(s, nw, h->K_rp, h->K_ci, h->Kval, nullptr, D0, k, 1, E, k, 1, k, -1.0, 1.0));
  }
  // rhs_u = e_u - G_u^T G_x^{-T} e_x  (into p_u)
  TRYK(lu_solve_perm(h, 1, E + (size_t)nu * k, k, 1, k));
  CKK(cudaMemcpyAsync(p.w, E, sizeof(double) * (size_t)nu * k, cudaMemcpyDeviceToDevice, s));
  CKK(launch_spmm(s, nu, h->GuT_rp, h->GuT_ci, h->Gval, h->GuT_map, E + (size_t)nu * k, k, 1, p.w, k, 1, k, -1.0,
                  1.0));
  ph_end(h);
  return kkt_recover(h, k, b, p, bl_zero, scratch);
}

// The recovery half of kkt_core: p_u from the condensed right-hand side in p.w
// (Cholesky solves), then p_x, p_s, p_y, p_lambda, with q = G_x^{-1} b_l in
// D0's x rows and phi = G_x^{-T} e_x in E's x rows (the scratch layout of
// kkt_core) when the condensation's products are used
int kkt_recover(opf_handle* h, int k, const KB& b, const KB& p, bool bl_zero, double* scratch) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  double* Bt = scratch;
  double* E = Bt + (size_t)nw * k;
  double* D0 = E + (size_t)nw * k;
  double* U = D0 + (size_t)nw * k;
  double* Byr = U + (size_t)m * k;
  const bool dc = h->delta_c > 0.0;
  const double* sig = dc ? h->sig_se : h->sig_s;
  const double* by = dc ? Byr : b.y;
  ph_begin(h, OPF_PHASE_RECOVER);
  TRYK(chol_solve_async(h, p.w, k));
  double* px = p.w + (size_t)nu * k;
  if (h->psi_valid && k <= 4) {
    // the condensation left S_x = -G_x^{-1} G_u (in Z) and Psi = G_x^{-T} H_x (in
    // H's x rows, H = K Z); with phi = G_x^{-T} e_x (already in E):
    //   p_x = q + S_x p_u,   p_l = phi - Psi p_u       (two products, no solves)
    const long long ld = h->ldp;
    const int nb = (nx * 32 + 127) / 128, nb1 = (nx * 32 + 255) / 256;
    if (k == 1)
      k_dense_rows1<<<nb1, 256, 0, s>>>(nx, nu, h->Zt + (size_t)nu * ld, ld, p.w, bl_zero ? nullptr : D0 + nu, 1.0,
                                         px);
    else
      k_dense_rows<<<nb, 128, 0, s>>>(nx, nu, k, h->Zt + (size_t)nu * ld, ld, p.w,
                                      bl_zero ? nullptr : D0 + (size_t)nu * k, 1.0, px);
    TRYK(launched());
    CKK(launch_spmm(s, m, h->A_rp, h->A_ci_c, h->Aval, nullptr, p.w, k, 1, p.s, k, 1, k, -1.0, 0.0));
    CKK(launch_axpby(s, (long long)m * k, 1.0, by, 1.0, p.s, p.s));
    k_rows_scale_sub<<<nblk((long long)m * k, 256), 256, 0, s>>>(m, k, sig, p.s, b.s, p.y);
    TRYK(launched());
    if (dc) {
      k_rows_scale_inplace<<<nblk((long long)m * k, 256), 256, 0, s>>>(m, k, h->ps_sc, p.s);
      TRYK(launched());
    }
    if (k == 1)
      k_dense_rows1<<<nb1, 256, 0, s>>>(nx, nu, h->H + (size_t)nu * ld, ld, p.w, E + nu, -1.0, p.l);
    else
      k_dense_rows<<<nb, 128, 0, s>>>(nx, nu, k, h->H + (size_t)nu * ld, ld, p.w, E + (size_t)nu * k, -1.0, p.l);
    TRYK(launched());
    ph_end(h);
    return OPF_OK;
  }
  // p_x = G_x^{-1} (b_l - G_u p_u)
  if (bl_zero) CKK(launch_spmm(s, nx, h->PGu_rp, h->PGu_ci, h->Gval, h->PGu_map, p.w, k, 1, px, k, 1, k, -1.0, 0.0));
  else {
    CKK(cudaMemcpyAsync(px, b.l, sizeof(double) * (size_t)nx * k, cudaMemcpyDeviceToDevice, s));
    CKK(launch_spmm(s, nx, h->PGu_rp, h->PGu_ci, h->Gval, h->PGu_map, p.w, k, 1, px, k, 1, k, -1.0, 1.0));
  }
  TRYK(lu_solve_perm(h, 0, px, k, 1, k));
  // p_s = b_y - A p_w ; p_y = b_s - Sigma_s p_s
  CKK(cudaMemcpyAsync(p.s, by, sizeof(double) * (size_t)m * k, cudaMemcpyDeviceToDevice, s));
  CKK(launch_spmm(s, m, h->A_rp, h->A_ci_c, h->Aval, nullptr, p.w, k, 1, p.s, k, 1, k, -1.0, 1.0));
  k_rows_scale_sub<<<nblk((long long)m * k, 256), 256, 0, s>>>(m, k, sig, p.s, b.s, p.y);
  TRYK(launched());
  if (dc) {
    k_rows_scale_inplace<<<nblk((long long)m * k, 256), 256, 0, s>>>(m, k, h->ps_sc, p.s);
    TRYK(launched());
  }
  // p_l = G_x^{-T} (bt_w,x - [K p_w]_x)
  CKK(cudaMemcpyAsync(p.l, Bt + (size_t)nu * k, sizeof(double) * (size_t)nx * k, cudaMemcpyDeviceToDevice, s));
  CKK(launch_spmm(s, nx, h->K_rp + nu, h->K_ci, h->Kval, nullptr, p.w, k, 1, p.l, k, 1, k, -1.0, 1.0));
  TRYK(lu_solve_perm(h, 1, p.l, k, 1, k));
  ph_end(h);
  return OPF_OK;
}

int kkt_residual(opf_handle* h, int k, const KB& b, const KB& z, const KB& R, double delta_w) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nw = P.nw, nx = P.nx, m = P.m;
  // R_w = b_w - (W + Sigma_w + delta_w E_u) z_w - G^T z_l - A^T z_y
  k_rows_scale_sub<<<nblk((long long)nw * k, 256), 256, 0, s>>>(nw, k, h->sig_c, z.w, b.w, R.w);
  TRYK(launched());
  if (delta_w > 0.0) CKK(launch_axpby(s, (long long)P.nu * k, -delta_w, z.w, 1.0, R.w, R.w));
  CKK(launch_spmm(s, nw, h->K_rp, h->K_ci, h->Wval, nullptr, z.w, k, 1, R.w, k, 1, k, -1.0, 1.0));
  CKK(launch_spmm(s, nw, h->GcT_rp, h->GcT_ci, h->Gval, h->GcT_map, z.l, k, 1, R.w, k, 1, k, -1.0, 1.0));
  CKK(launch_spmm(s, nw, h->AT_rp, h->AT_ci, h->Aval, h->AT_map, z.y, k, 1, R.w, k, 1, k, -1.0, 1.0));
  // R_s = b_s - Sigma_s z_s - z_y
  k_res_s<<<nblk((long long)m * k, 256), 256, 0, s>>>(m, k, h->sig_s, b.s, z.s, z.y, R.s);
  TRYK(launched());
  // R_l = b_l - G z_w
  CKK(cudaMemcpyAsync(R.l, b.l, sizeof(double) * (size_t)nx * k, cudaMemcpyDeviceToDevice, s));
  CKK(launch_spmm(s, nx, h->Gc_rp, h->Gc_ci, h->Gval, h->Gc_map, z.w, k, 1, R.l, k, 1, k, -1.0, 1.0));
  // R_y = b_y - A z_w - z_s (+ delta_c z_y)
  CKK(launch_axpby(s, (long long)m * k, 1.0, b.y, -1.0, z.s, R.y));
  CKK(launch_spmm(s, m, h->A_rp, h->A_ci_c, h->Aval, nullptr, z.w, k, 1, R.y, k, 1, k, -1.0, 1.0));
  if (h->delta_c > 0.0) CKK(launch_axpby(s, (long long)m * k, 1.0, R.y, h->delta_c, z.y, R.y));
  return OPF_OK;
}

// max |x_i| over n entries, read back to the host (two-stage reduction; part holds
// ABSMAX_PARTS doubles)
constexpr int ABSMAX_PARTS = 304;
int device_absmax(opf_handle* h, const double* x, long long n, double* part, double* out) {
  const int g = int(std::max(1LL, std::min<long long>(ABSMAX_PARTS, (n + 255) / 256)));
  k_absmax_partial<<<g, 256, 0, h->s>>>(n, x, part);
  TRYK(launched());
  CKK(launch_absmax(h->s, g, part, part + g));
  CKK(cudaMemcpyAsync(out, part + g, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CKK(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

int kkt_refine(opf_handle* h, int k, const KB& b, const KB& z, bool solve_first, bool bl_zero, int max_steps,
               double* scratch, double* final_res, int* steps, bool fullspace) {
  const Plan& P = h->P;
  const size_t N = kkt_rows(P) * (size_t)k;
  double* Rbase = scratch;
  double* Dbase = Rbase + N;
  double* part = Dbase + N;
  double* core = part + ABSMAX_PARTS + 8;
  const KB R = kb_at(P, Rbase, k), D = kb_at(P, Dbase, k);
  if (solve_first) TRYK(fullspace ? fs_core(h, k, b, z) : kkt_core(h, k, b, z, bl_zero, core));
  double bn = 0.0, rn = 0.0, prev = INFINITY;
  TRYK(device_absmax(h, b.w, (long long)N, part, &bn));
  int it = 0;
  for (; it <= max_steps; ++it) {
    TRYK(kkt_residual(h, k, b, z, R, fullspace ? fs_delta_w(h) : 0.0));
    TRYK(device_absmax(h, Rbase, (long long)N, part, &rn));
    if (!(rn > 1e-15 * std::max(bn, 1e-300)) || rn > 0.5 * prev || it == max_steps) break;
    prev = rn;
    TRYK(fullspace ? fs_core(h, k, R, D) : kkt_core(h, k, R, D, false, core));
    CKK(launch_axpby(h->s, (long long)N, 1.0, Dbase, 1.0, z.w, z.w));
  }
  if (final_res) *final_res = bn > 0 ? rn / bn : rn;
  if (steps) *steps = it;
  return OPF_OK;
}

// K_aug p = -r for k right-hand sides (col-major n_kkt x k in, col-major out,
// natural order [r_w; r_s; r_lambda; r_y] with w = [u; x]); refine > 0 adds up
// to that many refinement corrections against the full K_aug
int kkt_solve_impl(opf_handle* h, const double* rhs, double* step, int k, int refine) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nw = P.nw, m = P.m, nx = P.nx;
  const size_t N = kkt_rows(P);
  const size_t extra = refine > 0 ? kkt_refine_scratch(P, k) : kkt_core_scratch(P) * (size_t)k;
  double* ws = workspace(h, 2 * N * (size_t)k + extra + 8);
  if (!ws) return OPF_ERR_OOM;
  const KB b = kb_at(P, ws, k);
  const KB p = kb_at(P, ws + N * k, k);
  double* scratch = ws + 2 * N * k;
  // b = -r, permuted into the internal layout
  CKK(launch_permute_rows(s, nw, k, h->c2w, rhs, int(N), 1, b.w, k, 0, -1.0, 0));
  CKK(launch_permute_rows(s, m, k, nullptr, rhs + nw, int(N), 1, b.s, k, 0, -1.0, 0));
  CKK(launch_permute_rows(s, nx, k, h->perm, rhs + nw + m, int(N), 1, b.l, k, 0, -1.0, 0));
  CKK(launch_permute_rows(s, m, k, nullptr, rhs + nw + m + nx, int(N), 1, b.y, k, 0, -1.0, 0));
  if (refine > 0) TRYK(kkt_refine(h, k, b, p, true, false, refine, scratch, nullptr, nullptr));
  else TRYK(kkt_core(h, k, b, p, false, scratch));
  CKK(launch_permute_rows(s, nw, k, h->c2w, p.w, k, 0, step, int(N), 1, 1.0, 1));
  CKK(launch_permute_rows(s, m, k, nullptr, p.s, k, 0, step + nw, int(N), 1, 1.0, 0));
  CKK(launch_permute_rows(s, nx, k, h->perm, p.l, k, 0, step + nw + m, int(N), 1, 1.0, 1));
  CKK(launch_permute_rows(s, m, k, nullptr, p.y, k, 0, step + nw + m + nx, int(N), 1, 1.0, 0));
  return OPF_OK;
}

// K_aug p = -r for the right-hand side condensed with the last condensation:
// r_hat, q and phi are read from the extra column of H and Zt, so only the
// Cholesky solve and the recovery products remain (the plain path on the kept
// copy of the right-hand side when the column is no longer valid)
int kkt_solve_prepared(opf_handle* h, double* step) {
  const Plan& P = h->P;
  cudaStream_t s = h->s;
  const int nw = P.nw, m = P.m, nx = P.nx, nu = P.nu;
  if (!h->fr_have_b) return OPF_ERR_INVALID_ARG;
  const size_t N = kkt_rows(P);
  double* ws = workspace(h, N + kkt_core_scratch(P) + 8);
  if (!ws) return OPF_ERR_OOM;
  const KB b = kb_at(P, h->fr_kb, 1);
  const KB p = kb_at(P, ws, 1);
  double* scratch = ws + N;
  if (h->fr_ready && h->delta_c == 0.0 && h->psi_valid) {
    const long long ld = h->ldp;
    double* E = scratch + nw;
    double* D0 = E + nw;
    ph_begin(h, OPF_PHASE_RHS);
    CKK(launch_column_axpby(s, nu, 1.0, h->H + nu, ld, 0.0, nullptr, 0, p.w, 1));                        // r_hat
    CKK(launch_column_axpby(s, nx, 1.0, h->Zt + (size_t)nu * ld + nu, ld, 0.0, nullptr, 0, D0 + nu, 1));  // q
    CKK(launch_column_axpby(s, nx, 1.0, h->H + (size_t)nu * ld + nu, ld, 0.0, nullptr, 0, E + nu, 1));     // phi
    ph_end(h);
    TRYK(kkt_recover(h, 1, b, p, false, scratch));
  } else {
    TRYK(kkt_core(h, 1, b, p, false, scratch));
  }
  CKK(launch_permute_rows(s, nw, 1, h->c2w, p.w, 1, 0, step, int(N), 1, 1.0, 1));
  CKK(launch_permute_rows(s, m, 1, nullptr, p.s, 1, 0, step + nw, int(N), 1, 1.0, 0));
  CKK(launch_permute_rows(s, nx, 1, h->perm, p.l, 1, 0, step + nw + m, int(N), 1, 1.0, 1));
  CKK(launch_permute_rows(s, m, 1, nullptr, p.y, 1, 0, step + nw + m + nx, int(N), 1, 1.0, 0));
  return OPF_OK;
}

}  // namespace condipm
