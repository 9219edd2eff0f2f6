// Derivative of the optimal dispatch with respect to the bus loads.
//
// At a solution of the barrier KKT system F(xi; d) = 0 (fixed mu, bound
// multipliers eliminated into Sigma), the implicit-function theorem gives
//   dPg/dd = dPg/dd|_direct - J_out K_aug^{-1} dF/dd,
// with K_aug the augmented matrix of Eq. kktmatrix:normal at the solution and
// J_out = dPg/dxi.  For cotangents vbar, grad_d = vbar^T dPg/dd is evaluated as
// zeta = K_aug^{-1} J_out^T vbar, grad_d = -(dF/dd)^T zeta + direct term, and
// zeta comes from the condensed recovery of Theorems 1 and 2 with the factors
// the interior-point iteration builds (LU of G_x, Cholesky of Kred), refined
// against the full K_aug (at a converged point Kred is ill-conditioned).
//
// The right-hand side J_out^T vbar lives in the primal block only: Pg_k (k >= 1)
// are controls, and the slack generator's Pg_0 = h_0(w) = P_s(w) + Pd_s has
// gradient a_0 = row 0 of A.  With it the first condensed solve needs one
// Cholesky solve and three multi-RHS solves with G_x (b_l = 0).
// dF/dd: g has +Pd_i in the P row of bus i and +Qd_i in the Q row of a load
// bus; h_0 has +Pd_s, h_{1+k} has +Qd at generator k's bus; the objective's
// slack term puts 2 c2_0 a_0 into the gradient row for Pd_s.  So
//   grad_Pd_i = -zeta_lambda[P_i],  grad_Qd_i = -zeta_lambda[Q_i]   (load bus),
//   grad_Qd_i = -zeta_y[1 + k]                                     (generator k),
//   grad_Pd_s = vbar_0 - 2 c2_0 a_0 . zeta_w - zeta_y[0],  a_0 . zeta_w = -zeta_s[0].
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/condipm.h"
#include "internal.h"

namespace condipm {
namespace {

#define CKS(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      note_cuda_error(e_);                \
      return OPF_ERR_CUDA;                \
    }                                     \
  } while (0)
#define TRYS(x)                  \
  do {                           \
    int r_ = (x);                \
    if (r_ != OPF_OK) return r_; \
  } while (0)

inline int nblk(long long n, int t) { return int((n + t - 1) / t); }

// dense copy of one CSR row (column indices already in the destination order)
__global__ void k_row_dense(int q0, int q1, const int* __restrict__ ci, const double* __restrict__ val,
                            double* __restrict__ out) {
  int q = q0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (q < q1) out[ci[q]] = val[q];
}

// b_w (nw x k, c-order rows) = J_out^T vbar: vbar(j, gen of w-entry c) + vbar(j, 0) a_0(c)
__global__ void k_vjp_rhs(int nw, int k, int ng, const int* __restrict__ gen_of_w, const int* __restrict__ c2w,
                          const double* __restrict__ a0, const double* __restrict__ vbar, double* __restrict__ B) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nw * k) return;
  const int c = int(t / k), j = int(t % k);
  const double* v = vbar + (size_t)j * ng;
  double r = v[0] * a0[c];
  const int g = gen_of_w[c2w[c]];
  if (g >= 1) r += v[g];
  B[t] = r;
}

// gradient assembly, one thread per (cotangent, bus)
__global__ void k_vjp_grad(int nb, int k, int ng, int slack, double c2_0, const int* __restrict__ ppos,
                           const int* __restrict__ qpos, const int* __restrict__ gen_of_bus,
                           const double* __restrict__ zs, const double* __restrict__ zl,
                           const double* __restrict__ zy, const double* __restrict__ vbar,
                           double* __restrict__ gPd, double* __restrict__ gQd) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nb * k) return;
  const int j = int(t / nb), i = int(t % nb);
  double gp;
  if (i == slack) gp = fma(2.0 * c2_0, zs[j], vbar[(size_t)j * ng]) - zy[j];
  else gp = -zl[(size_t)ppos[i] * k + j];
  const int g = gen_of_bus[i];
  const double gq = g >= 0 ? -zy[(size_t)(1 + g) * k + j] : -zl[(size_t)qpos[i] * k + j];
  gPd[t] = gp;
  gQd[t] = gq;
}

int sens_alloc(opf_handle* h) {
  if (h->sens_buf) return OPF_OK;
  const Plan& P = h->P;
  // state: x, u, lam, y, sig_u, sig_x, sig_s ; then a_0 (nw, c-order)
  const size_t n = (size_t)P.nx + P.nu + P.nx + P.m + P.nu + P.nx + P.m + P.nw + 8;
  if (cudaMalloc(&h->sens_buf, n * sizeof(double)) != cudaSuccess) { h->sens_buf = nullptr; return OPF_ERR_OOM; }
  h->allocs.push_back(h->sens_buf);
  std::vector<int> pq(2 * (size_t)P.nb, -1);
  for (int i = 0; i < P.nb; ++i) {
    if (P.g_row_P[i] >= 0) pq[i] = P.iperm[P.g_row_P[i]];
    if (P.g_row_Q[i] >= 0) pq[P.nb + i] = P.iperm[P.g_row_Q[i]];
  }
  if (cudaMalloc(&h->sens_pq, pq.size() * sizeof(int)) != cudaSuccess) { h->sens_pq = nullptr; return OPF_ERR_OOM; }
  h->allocs.push_back(h->sens_pq);
  CKS(cudaMemcpy(h->sens_pq, pq.data(), pq.size() * sizeof(int), cudaMemcpyHostToDevice));
  return OPF_OK;
}

}  // namespace

int sens_prepare(opf_handle* h, const double* w, const double* lam, const double* y, const double* sig_w,
                 const double* sig_s) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  TRYS(sens_alloc(h));
  cudaStream_t s = h->s;
  double* d_x = h->sens_buf;
  double* d_u = d_x + nx;
  double* d_lam = d_u + nu;
  double* d_y = d_lam + nx;
  double* d_su = d_y + m;
  double* d_sx = d_su + nu;
  double* d_ss = d_sx + nx;
  double* a0 = d_ss + m;
  auto up = [&](double* dst, const double* src, size_t n) {
    return n == 0 || cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  if (!up(d_u, w, nu) || !up(d_x, w + nu, nx) || !up(d_lam, lam, nx) || !up(d_y, y, m) || !up(d_su, sig_w, nu) ||
      !up(d_sx, sig_w + nu, nx) || !up(d_ss, sig_s, m))
    return OPF_ERR_CUDA;
  TRYS(eval_impl(h, d_x, d_u, d_lam, d_y, true));
  TRYS(condense_async(h, d_su, d_sx, d_ss));
  TRYS(read_status(h, nullptr));
  TRYS(factor_kred_async(h, 0.0));
  TRYS(read_status(h, nullptr));
  h->have_factor = true;
  // a_0 = row 0 of A (the slack generator's Pg) in c-order
  CKS(cudaMemsetAsync(a0, 0, sizeof(double) * nw, s));
  const int q0 = P.A.rp[0], q1 = P.A.rp[1];
  if (q1 > q0) {
    k_row_dense<<<nblk(q1 - q0, 128), 128, 0, s>>>(q0, q1, h->A_ci_c, h->Aval, a0);
    note_launch();
    CKS(cudaGetLastError());
  }
  TRYS(read_status(h, nullptr));
  h->sens_ready = true;
  return OPF_OK;
}

int dispatch_vjp_impl(opf_handle* h, const double* vbar, int k, double* gPd, double* gQd) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m, nb = P.nb, ng = P.ng;
  cudaStream_t s = h->s;
  const double* a0 = h->sens_buf + (size_t)nx + nu + nx + m + nu + nx + m;
  const size_t N = kkt_rows(P) * (size_t)k;
  double* ws = workspace(h, 2 * N + kkt_refine_scratch(P, k));
  if (!ws) return OPF_ERR_OOM;
  const KB b = kb_at(P, ws, k), z = kb_at(P, ws + N, k);
  // b = [J_out^T vbar; 0; 0; 0]
  CKS(cudaMemsetAsync(b.s, 0, sizeof(double) * (N - (size_t)nw * k), s));
  k_vjp_rhs<<<nblk((long long)nw * k, 256), 256, 0, s>>>(nw, k, ng, h->pg_of_w, h->c2w, a0, vbar, b.w);
  note_launch();
  CKS(cudaGetLastError());
  TRYS(kkt_refine(h, k, b, z, true, true, h->vjp_max_refine, ws + 2 * N, &h->vjp_res, &h->vjp_steps));
  k_vjp_grad<<<nblk((long long)nb * k, 256), 256, 0, s>>>(nb, k, ng, P.slack, P.c2[0], h->sens_pq,
                                                         h->sens_pq + nb, h->gen_of_bus, z.s, z.l, z.y, vbar,
                                                         gPd, gQd);
  note_launch();
  CKS(cudaGetLastError());
  return OPF_OK;
}

}  // namespace condipm

using namespace condipm;

extern "C" int opf_set_loads(opf_handle* h, const double* Pd, const double* Qd) {
  if (!h || !Pd || !Qd) return OPF_ERR_INVALID_ARG;
  Plan& P = h->P;
  for (int i = 0; i < P.nb; ++i)
    if (!std::isfinite(Pd[i]) || !std::isfinite(Qd[i])) return OPF_ERR_INVALID_ARG;
  std::copy(Pd, Pd + P.nb, P.Pd.begin());
  std::copy(Qd, Qd + P.nb, P.Qd.begin());
  CKS(cudaMemcpyAsync(h->Pd, P.Pd.data(), sizeof(double) * P.nb, cudaMemcpyHostToDevice, h->s));
  CKS(cudaMemcpyAsync(h->Qd, P.Qd.data(), sizeof(double) * P.nb, cudaMemcpyHostToDevice, h->s));
  CKS(cudaStreamSynchronize(h->s));
  h->have_eval = h->have_W = h->have_lu = h->have_condense = h->have_factor = false;
  h->have_solution = false;
  h->sens_ready = false;
  return OPF_OK;
}

extern "C" int opf_vjp_prepare(opf_handle* h, const double* w, const double* lam, const double* y,
                               const double* sig_w, const double* sig_s) {
  if (!h) return OPF_ERR_INVALID_ARG;
  const int given = (w != nullptr) + (lam != nullptr) + (y != nullptr) + (sig_w != nullptr) + (sig_s != nullptr);
  if (given == 0) {
    if (!h->have_solution) return OPF_ERR_INVALID_ARG;
    // move the stored point onto the barrier solution at its mu (the IPM stops
    // at its tolerance, a little short of it); on failure keep the IPM's point
    if (!h->polished) {
      h->polished = true;
      if (polish_solution(h, 1e-12, 20) != OPF_OK) h->polish_iters = -1;
    }
    return sens_prepare(h, h->sol_w.data(), h->sol_lam.data(), h->sol_y.data(), h->sol_sig_w.data(),
                        h->sol_sig_s.data());
  }
  if (given != 5) return OPF_ERR_INVALID_ARG;
  return sens_prepare(h, w, lam, y, sig_w, sig_s);
}

extern "C" int opf_vjp_info(const opf_handle* h, int* refine_steps, double* rel_residual, int* polish_iters,
                            double* kkt_residual) {
  if (!h) return OPF_ERR_INVALID_ARG;
  if (refine_steps) *refine_steps = h->vjp_steps;
  if (rel_residual) *rel_residual = h->vjp_res;
  if (polish_iters) *polish_iters = h->polish_iters;
  if (kkt_residual) *kkt_residual = h->polish_res;
  return OPF_OK;
}

extern "C" int opf_dispatch_vjp(opf_handle* h, const double* vbar, int k, double* grad_Pd, double* grad_Qd) {
  if (!h || k < 0 || (k > 0 && (!vbar || !grad_Pd || !grad_Qd))) return OPF_ERR_INVALID_ARG;
  if (!h->sens_ready) return OPF_ERR_INVALID_ARG;
  if (k == 0) return OPF_OK;
  TRYS(dispatch_vjp_impl(h, vbar, k, grad_Pd, grad_Qd));
  return read_status(h, nullptr);
}
