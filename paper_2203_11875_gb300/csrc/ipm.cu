// Interior-point driver around the device hot path, and the derivative of the
// optimal dispatch with respect to the bus loads.
//
// The outer loop is the primal-dual barrier method of Wachter and Biegler (2006)
// that the paper defers to (Sec. 4.3): monotone barrier update, fraction to the
// boundary, bound multipliers eliminated into Sigma, scaled optimality error,
// y0 = 0, inertia correction by a primal regularisation of the control block
// until the condensed matrix is positive definite (Theorem 3).  Steps are
// accepted by backtracking on the l1 exact-penalty merit function (Nocedal and
// Wright, Sec. 19.4).  As in the paper (Sec. 3, "only the interior-point routines
// run on the host"), the scalar and vector bookkeeping of the loop is host code;
// every model evaluation, G_x factorisation, condensation, Cholesky factorisation,
// step recovery and power-flow projection runs in the library's kernels.
//   LinRed (Algorithm 1): condensed step of the full-space barrier system.
//   RedLin (Algorithm 2): Newton-Raphson projection onto g(x, u) = 0 at every
//     control (Sec. 4.4), adjoint solve for lambda, state bounds as rows -x of
//     h_r (Eq. reduced:problem); its condensed matrix is the LinRed one with the
//     bound rows' Sigma in place of Sigma_x.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <utility>
#include <vector>

#include "../../include/condipm.h"
#include "internal.h"

namespace condipm {
namespace {

constexpr double TAU_MIN = 0.99, KAPPA_EPS = 10.0, KAPPA_MU = 0.2, THETA_MU = 1.5, ETA = 1e-4;
constexpr double KAPPA_SIGMA = 1e10, SMAX = 100.0;
// filter line search (Wachter and Biegler 2006, their recommended constants)
constexpr double GAMMA_THETA = 1e-5, GAMMA_PHI = 1e-8, SWITCH_DELTA = 1.0, S_THETA = 1.1, S_PHI = 2.3;
constexpr double ETA_PHI = 1e-4, GAMMA_ALPHA = 0.05, KAPPA_SOC = 0.99;
constexpr int SOC_MAX = 4;
// feasibility restoration (Wachter and Biegler 2006, Sec. 3.3)
constexpr double RHO_RESTO = 1000.0, KAPPA_RESTO = 0.9;
constexpr int RESTO_MAX_ITER = 100;

// The filter: a trial (theta, phi) is acceptable when no pair (theta_l, phi_l)
// has theta >= theta_l and phi >= phi_l.  It starts as theta >= theta_max.
struct Filter {
  std::vector<std::pair<double, double>> pairs;
  void reset(double theta_max) { pairs.assign(1, {theta_max, -INFINITY}); }
  bool acceptable(double theta, double phi) const {
    for (const auto& p : pairs)
      if (theta >= p.first && phi >= p.second) return false;
    return true;
  }
};

// acceptance of a trial point reached with step length a (Sec. 2.3 of the
// filter method): returns accepted, sets phi_type for Armijo (phi-type) steps
bool filter_accepts(const Filter& F, double theta0, double phi0, double dphi, double a, double theta_t,
                    double phi_t, double theta_min, bool& phi_type) {
  phi_type = false;
  if (!std::isfinite(phi_t) || !F.acceptable(theta_t, phi_t)) return false;
  const bool switching = dphi < 0 && a * std::pow(-dphi, S_PHI) > SWITCH_DELTA * std::pow(theta0, S_THETA);
  if (switching && theta0 <= theta_min) {
    phi_type = true;
    return phi_t <= phi0 + ETA_PHI * a * dphi;
  }
  return theta_t <= (1.0 - GAMMA_THETA) * theta0 || phi_t <= phi0 - GAMMA_PHI * theta0;
}

double filter_alpha_min(double theta0, double dphi, double theta_min) {
  if (dphi < 0) {
    double a = std::min(GAMMA_THETA, GAMMA_PHI * theta0 / -dphi);
    if (theta0 <= theta_min) a = std::min(a, SWITCH_DELTA * std::pow(theta0, S_THETA) / std::pow(-dphi, S_PHI));
    return GAMMA_ALPHA * a;
  }
  return GAMMA_ALPHA * GAMMA_THETA;
}

using Vec = std::vector<double>;

#define CKD(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      note_cuda_error(e_);                \
      return OPF_ERR_CUDA;                \
    }                                     \
  } while (0)
#define TRYD(x)                    \
  do {                             \
    int r_ = (x);                  \
    if (r_ != OPF_OK) return r_;   \
  } while (0)

inline bool finite_bound(double b) { return std::fabs(b) < 1e299; }

// finite-bound bookkeeping of a vector v with lo <= v <= hi
struct Bounds {
  Vec lo, hi;
  std::vector<char> fl, fu;
  Bounds() = default;
  Bounds(const Vec& l, const Vec& u) : lo(l), hi(u), fl(l.size()), fu(u.size()) {
    for (size_t i = 0; i < l.size(); ++i) { fl[i] = finite_bound(l[i]); fu[i] = finite_bound(u[i]); }
  }
  size_t n() const { return lo.size(); }
  double dl(const Vec& v, size_t i) const { return v[i] - lo[i]; }
  double du(const Vec& v, size_t i) const { return hi[i] - v[i]; }
  void push(Vec& v) const {   // Ipopt's initial bound push (kappa_1 = kappa_2 = 1e-2)
    for (size_t i = 0; i < n(); ++i) {
      double pl = fl[i] ? 1e-2 * std::max(1.0, std::fabs(lo[i])) : 0.0;
      double pu = fu[i] ? 1e-2 * std::max(1.0, std::fabs(hi[i])) : 0.0;
      if (fl[i] && fu[i]) { pl = std::min(pl, 1e-2 * (hi[i] - lo[i])); pu = std::min(pu, 1e-2 * (hi[i] - lo[i])); }
      if (fl[i]) v[i] = std::max(v[i], lo[i] + pl);
      if (fu[i]) v[i] = std::min(v[i], hi[i] - pu);
    }
  }
  void sigma(const Vec& v, const Vec& zl, const Vec& zu, Vec& out) const {
    out.assign(n(), 0.0);
    for (size_t i = 0; i < n(); ++i) {
      if (fl[i]) out[i] += zl[i] / dl(v, i);
      if (fu[i]) out[i] += zu[i] / du(v, i);
    }
  }
  double bgrad(const Vec& v, size_t i, double mu) const {
    double g = 0.0;
    if (fl[i]) g -= mu / dl(v, i);
    if (fu[i]) g += mu / du(v, i);
    return g;
  }
  double barrier(const Vec& v, double mu) const {
    double b = 0.0;
    for (size_t i = 0; i < n(); ++i) {
      if (fl[i]) b -= mu * std::log(dl(v, i));
      if (fu[i]) b -= mu * std::log(du(v, i));
    }
    return b;
  }
  double max_step(const Vec& v, const Vec& dv, double tau) const {
    double a = 1.0;
    for (size_t i = 0; i < n(); ++i) {
      if (fl[i] && dv[i] < 0) a = std::min(a, -tau * dl(v, i) / dv[i]);
      if (fu[i] && dv[i] > 0) a = std::min(a, tau * du(v, i) / dv[i]);
    }
    return a;
  }
  void dz(const Vec& v, const Vec& zl, const Vec& zu, const Vec& dv, double mu, Vec& dzl, Vec& dzu) const {
    dzl.assign(n(), 0.0);
    dzu.assign(n(), 0.0);
    for (size_t i = 0; i < n(); ++i) {
      if (fl[i]) dzl[i] = mu / dl(v, i) - zl[i] - zl[i] / dl(v, i) * dv[i];
      if (fu[i]) dzu[i] = mu / du(v, i) - zu[i] + zu[i] / du(v, i) * dv[i];
    }
  }
  void safeguard(const Vec& v, Vec& zl, Vec& zu, double mu) const {
    for (size_t i = 0; i < n(); ++i) {
      if (fl[i]) zl[i] = std::min(std::max(zl[i], mu / (KAPPA_SIGMA * dl(v, i))), KAPPA_SIGMA * mu / dl(v, i));
      else zl[i] = 0.0;
      if (fu[i]) zu[i] = std::min(std::max(zu[i], mu / (KAPPA_SIGMA * du(v, i))), KAPPA_SIGMA * mu / du(v, i));
      else zu[i] = 0.0;
    }
  }
  // complementarity max-norm and the multiplier l1 sum / count
  double compl_inf(const Vec& v, const Vec& zl, const Vec& zu, double mu, double& zsum, long long& zcnt) const {
    double e = 0.0;
    for (size_t i = 0; i < n(); ++i) {
      if (fl[i]) { e = std::max(e, std::fabs(dl(v, i) * zl[i] - mu)); zsum += std::fabs(zl[i]); ++zcnt; }
      if (fu[i]) { e = std::max(e, std::fabs(du(v, i) * zu[i] - mu)); zsum += std::fabs(zu[i]); ++zcnt; }
    }
    return e;
  }
};

double max_step_z(const Vec& z, const Vec& dz, const std::vector<char>& mask, double tau) {
  double a = 1.0;
  for (size_t i = 0; i < z.size(); ++i)
    if (mask[i] && dz[i] < 0) a = std::min(a, -tau * z[i] / dz[i]);
  return a;
}

double inf_norm(const Vec& v) {
  double m = 0.0;
  for (double x : v) m = std::max(m, std::fabs(x));
  return m;
}
double l1_norm(const Vec& v) {
  double m = 0.0;
  for (double x : v) m += std::fabs(x);
  return m;
}

// Ipopt-style scaled optimality error
double opt_error(double dual_inf, double primal_inf, double compl_inf, double mult_sum, long long mult_cnt) {
  const double sd = std::max(SMAX, mult_sum / std::max(1LL, mult_cnt)) / SMAX;
  return std::max(std::max(dual_inf / sd, primal_inf), compl_inf / sd);
}

// device scratch of the interior-point loop: one allocation per handle, kept
// for the handle's lifetime (freeing device memory would synchronise the whole
// device and serialise concurrent solves on other streams)
struct Dev {
  double *x = nullptr, *u = nullptr, *lam = nullptr, *y = nullptr, *sig_u = nullptr, *sig_x = nullptr,
         *sig_s = nullptr, *rhs = nullptr, *step = nullptr, *grad = nullptr, *tmp = nullptr;
};

int alloc_dev(Dev& d, opf_handle* h) {
  const Plan& P = h->P;
  const size_t nkkt = (size_t)P.nw + 2 * (size_t)P.m + P.nx;
  const size_t sizes[11] = {(size_t)P.nx, (size_t)P.nu, (size_t)P.nx, (size_t)P.m, (size_t)P.nu, (size_t)P.nx,
                            (size_t)P.m, nkkt, nkkt, (size_t)P.nw, (size_t)std::max(P.nw, P.nx)};
  size_t total = 0;
  for (size_t n : sizes) total += std::max<size_t>(n, 1);
  if (!h->ipm_buf) {
    if (cudaMalloc(&h->ipm_buf, total * sizeof(double)) != cudaSuccess) { h->ipm_buf = nullptr; return OPF_ERR_OOM; }
    h->allocs.push_back(h->ipm_buf);
  }
  double** slots[11] = {&d.x, &d.u, &d.lam, &d.y, &d.sig_u, &d.sig_x, &d.sig_s, &d.rhs, &d.step, &d.grad, &d.tmp};
  double* p = h->ipm_buf;
  for (int i = 0; i < 11; ++i) { *slots[i] = p; p += std::max<size_t>(sizes[i], 1); }
  // the single-right-hand-side K_aug solves of the loop use this much workspace
  if (!workspace(h, 2 * nkkt + kkt_refine_scratch(P, 1) + 8)) return OPF_ERR_OOM;
  TRYD(fr_reserve(h));
  return OPF_OK;
}

int h2d(cudaStream_t s, double* dst, const double* src, size_t n) {
  if (n == 0) return OPF_OK;
  return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess ? OPF_OK : OPF_ERR_CUDA;
}
int d2h(cudaStream_t s, double* dst, const double* src, size_t n) {
  if (n == 0) return OPF_OK;
  return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess ? OPF_OK : OPF_ERR_CUDA;
}

using clk = std::chrono::steady_clock;
double ms_since(clk::time_point t0) { return std::chrono::duration<double, std::milli>(clk::now() - t0).count(); }

// f, g, h at (x, u) (device copies made here)
int eval_fgh(opf_handle* h, Dev& d, const Vec& w, double& f, Vec& g, Vec& hv) {
  const Plan& P = h->P;
  TRYD(h2d(h->s, d.u, w.data(), P.nu));
  TRYD(h2d(h->s, d.x, w.data() + P.nu, P.nx));
  TRYD(eval_impl(h, d.x, d.u, nullptr, nullptr, false));
  g.resize(P.nx);
  hv.resize(P.m);
  TRYD(d2h(h->s, &f, h->f, 1));
  TRYD(d2h(h->s, g.data(), h->g, P.nx));
  TRYD(d2h(h->s, hv.data(), h->hv, P.m));
  CKD(cudaStreamSynchronize(h->s));
  return OPF_OK;
}

// The factorisation with primal regularisation d on the u block: the Cholesky
// of Kred + d I, or in the hybrid full-space mode the block LDL^T of the
// augmented matrix with d on its u diagonal (its inertia test reports NOT_PD
// exactly when Kred + d I is not positive definite, Theorem 3)
int factor_delta(opf_handle* h, double d) { return h->ipm_fs ? fs_factor_async(h, d, 0.0) : factor_kred_async(h, d); }

// K_aug p = -r for the loop's one right-hand side: the condensed recovery, or
// the block factor with up to three refinement corrections
int solve_step(opf_handle* h, const double* rhs, double* step) {
  return h->ipm_fs ? fs_solve_impl(h, rhs, step, 1, 3, nullptr, nullptr) : kkt_solve_impl(h, rhs, step, 1, 0);
}

// Cholesky of Kred + delta I with the inertia-correction schedule; delta in/out.
// skip_zero: the attempt with delta = 0 already failed (NOT_PD)
int factor_with_correction(opf_handle* h, double& delta, double delta_last, int& attempts, bool skip_zero = false) {
  attempts = 0;
  double d = 0.0;
  if (skip_zero) d = delta_last > 0.0 ? std::max(1e-20, delta_last / 3.0) : 1e-4;
  for (;;) {
    TRYD(factor_delta(h, d));
    ++attempts;
    int rc = read_status(h, nullptr);
    if (h->ipm_fs && h->ipm_verbose) {
      int in[3];
      double ld = 0.0;
      TRYD(fs_read_inertia(h, in, &ld));
      std::printf("  full-space factor delta_w %.1e: status %d inertia (%d, %d, %d) want (%d, %d, 0)\n", d, rc, in[0],
                  in[1], in[2], h->P.nw, h->P.nx + h->P.m);
    }
    if (rc == OPF_OK) {
      h->have_factor = true;
      delta = d;
      return OPF_OK;
    }
    if (rc != OPF_ERR_NOT_PD) return rc;
    if (d == 0.0) d = delta_last > 0.0 ? std::max(1e-20, delta_last / 3.0) : 1e-4;
    else d *= 8.0;
    if (d > 1e40) return OPF_ERR_NOT_PD;
  }
}

// Condensation and the Cholesky attempt with delta_w = 0, enqueued as one CUDA
// graph: captured once the solve kernels are autotuned, replayed at every
// later iteration (the inputs live in the loop's fixed device buffers; the
// sequence resets its own counters and flags).  Where capture or instantiation
// is refused, or while phases are being profiled, the launches are enqueued
// one by one.  Returns the device status (one synchronisation).
int condense_factor0(opf_handle* h, Dev& d, int* graph_iters, bool with_rhs = false) {
  if (h->ipm_fs) {
    // hybrid full-space mode: assemble and factor the augmented matrix
    TRYD(fs_set_sigma(h, d.sig_u, d.sig_x, d.sig_s));
    TRYD(fs_factor_async(h, 0.0, 0.0));
    const int rc = read_status(h, nullptr);
    h->have_factor = false;
    return rc;
  }
  if (h->batch) {
    // a lockstep batch: one batched call serves every instance still iterating
    h->fr_ready = false;
    h->fr_have_b = false;
    const int rc = batch_join(h->batch, h->batch_idx, d.sig_u, d.sig_x, d.sig_s);
    h->have_factor = rc == OPF_OK;
    return rc;
  }
  const bool graph_ok = h->use_graphs && !h->cf_failed && !h->profiling && h->trsm_mode >= 0 && h->chol_tuned &&
                        h->route >= 0;
  if (h->cf_exec && h->cf_rhs != with_rhs) {
    // captured for the other kind of call: capture again
    cudaGraphExecDestroy(h->cf_exec);
    h->cf_exec = nullptr;
  }
  if (graph_ok && !h->cf_exec) {
    h->cf_rhs = with_rhs;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int rc = condense_async(h, d.sig_u, d.sig_x, d.sig_s, with_rhs ? d.rhs : nullptr);
      if (rc == OPF_OK) rc = factor_kred_async(h, 0.0);
      const cudaError_t e = cudaStreamEndCapture(h->s, &g);
      if (rc == OPF_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&h->cf_exec, g, 0) == cudaSuccess) {
        // captured
      } else {
        h->cf_exec = nullptr;
        h->cf_failed = true;
      }
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    } else {
      h->cf_failed = true;
      cudaGetLastError();
    }
  }
  if (graph_ok && h->cf_exec) {
    if (cudaGraphLaunch(h->cf_exec, h->s) != cudaSuccess) return OPF_ERR_CUDA;
    ++*graph_iters;
    // the host-side state the enqueued sequence stands for
    h->have_lu = true;
    h->have_condense = true;
    h->psi_valid = h->route != OPF_ROUTE_EXPLICIT;
    h->sens_ready = false;
    h->finv_valid = false;
    h->delta_w = 0.0;
    h->delta_c = 0.0;
    // the captured condensation carried the right-hand side's column
    h->fr_have_b = with_rhs;
    h->fr_ready = with_rhs && h->psi_valid && h->ldp > h->P.nu;
  } else {
    TRYD(condense_async(h, d.sig_u, d.sig_x, d.sig_s, with_rhs ? d.rhs : nullptr));
    TRYD(factor_kred_async(h, 0.0));
  }
  const int rc = read_status(h, nullptr);
  h->have_factor = rc == OPF_OK;
  return rc;
}

// Feasibility restoration phase (Wachter and Biegler 2006, Sec. 3.3), the
// relaxation restricted to the inequality rows as Sec. 4.3 describes for
// LinRed:
//   min rho sum(p + n) + zeta/2 |D_R (w - w_R)|^2
//   s.t. g(w) = 0, h(w) + s - p + n = 0, bounds on w and s, p, n >= 0,
// zeta = sqrt(mu), D_R = diag(min(1, 1/|w_R|)).  Its barrier Newton step is the
// condensed step with W replaced by the Hessian of the constraint terms plus
// zeta D_R^2 and the dual regularisation delta_i = 1/Sigma_p,i + 1/Sigma_n,i
// on the inequality rows (dp, dn eliminated).  That regularisation is folded
// into Sigma_t = Sigma_s / (1 + delta Sigma_s) with the slack row's right-hand
// side moved into the inequality rows (the same p_w, p_lambda and p_y), and the
// slack step taken from the slack row: the device path is the ordinary
// condensation.  The constraint-term Hessian is the evaluation at (lambda, y)
// minus the one at (0, 0).  Steps by backtracking on the l1 merit of the
// restoration barrier problem; the phase ends at the first point whose
// violation is at most kappa of the starting one and that the filter (holding
// the starting point) accepts.  Returns OPF_ERR_INFEASIBLE when it does not
// get there.
int restoration(opf_handle* h, Dev& d, const Bounds& bw, const Bounds& bs, const Filter& filt, double mu, Vec& w,
                Vec& s, Vec& lam, Vec& y, Vec& zwl, Vec& zwu, Vec& zsl, Vec& zsu, bool verbose, opf_ipm_result& R) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  const int nkkt = nw + 2 * m + nx;
  const long long nK = P.K.nnz();
  if (!h->resto_w0) {
    if (cudaMalloc(&h->resto_w0, sizeof(double) * std::max<long long>(1, nK)) != cudaSuccess) {
      h->resto_w0 = nullptr;
      return OPF_ERR_OOM;
    }
    h->allocs.push_back(h->resto_w0);
  }
  double f0;
  Vec g, hv;
  TRYD(eval_fgh(h, d, w, f0, g, hv));
  double theta_R = 0.0, cinf = 0.0;
  for (int i = 0; i < nx; ++i) { theta_R += std::fabs(g[i]); cinf = std::max(cinf, std::fabs(g[i])); }
  for (int i = 0; i < m; ++i) {
    theta_R += std::fabs(hv[i] + s[i]);
    cinf = std::max(cinf, std::fabs(hv[i] + s[i]));
  }
  const Vec wR = w;
  const double zeta = std::sqrt(mu), rho = RHO_RESTO;
  Vec dr2(nw);
  for (int i = 0; i < nw; ++i) {
    const double q = std::min(1.0, 1.0 / std::max(std::fabs(wR[i]), 1e-300));
    dr2[i] = q * q;
  }
  double mur = std::max(mu, cinf);
  Vec p(m), n(m), zp(m), zn(m);
  for (int i = 0; i < m; ++i) {
    // p and n minimising the relaxed barrier terms for the current c (closed form)
    const double c = hv[i] + s[i], t = (mur - rho * c) / (2.0 * rho);
    n[i] = t + std::sqrt(t * t + mur * c / (2.0 * rho));
    p[i] = c + n[i];
    zp[i] = mur / p[i];
    zn[i] = mur / n[i];
  }
  std::fill(lam.begin(), lam.end(), 0.0);
  std::fill(y.begin(), y.end(), 0.0);
  for (int i = 0; i < nw; ++i) {
    zwl[i] = bw.fl[i] ? mur / bw.dl(w, i) : 0.0;
    zwu[i] = bw.fu[i] ? mur / bw.du(w, i) : 0.0;
  }
  for (int i = 0; i < m; ++i) {
    zsl[i] = bs.fl[i] ? mur / bs.dl(s, i) : 0.0;
    zsu[i] = bs.fu[i] ? mur / bs.du(s, i) : 0.0;
  }
  double nu_pen = 1.0, delta = 0.0;
  Vec grad(nw), gradf(nw), sw, ss, st(m), sp(m), sn(m), r(nkkt), step(nkkt), rw(nw), rs(m), ry(m), rp(m), rn(m);
  Vec pw(nw), ps(m), pl(nx), py(m), pp(m), pn(m), dzwl, dzwu, dzsl, dzsu, dzp(m), dzn(m), wt(nw), stt(m), pt(m),
      nt(m);
  std::vector<char> all(m, 1);
  for (int it = 0; it < RESTO_MAX_ITER; ++it) {
    ++R.resto_iters;
    // derivatives; W of the constraint terms only: W(lambda, y) - W(0, 0)
    TRYD(h2d(h->s, d.u, w.data(), nu));
    TRYD(h2d(h->s, d.x, w.data() + nu, nx));
    CKD(cudaMemsetAsync(d.lam, 0, sizeof(double) * std::max(1, nx), h->s));
    CKD(cudaMemsetAsync(d.y, 0, sizeof(double) * std::max(1, m), h->s));
    TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
    CKD(cudaMemcpyAsync(h->resto_w0, h->Wval, sizeof(double) * nK, cudaMemcpyDeviceToDevice, h->s));
    TRYD(h2d(h->s, d.lam, lam.data(), nx));
    TRYD(h2d(h->s, d.y, y.data(), m));
    TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
    CKD(launch_axpby(h->s, nK, -1.0, h->resto_w0, 1.0, h->Wval, h->Wval));
    TRYD(lagrangian_gradient(h, d.lam, d.y, d.grad));
    g.resize(nx);
    hv.resize(m);
    TRYD(d2h(h->s, g.data(), h->g, nx));
    TRYD(d2h(h->s, hv.data(), h->hv, m));
    TRYD(d2h(h->s, grad.data(), d.grad, nw));
    TRYD(d2h(h->s, gradf.data(), h->gradf, nw));
    CKD(cudaStreamSynchronize(h->s));
    bw.sigma(w, zwl, zwu, sw);
    bs.sigma(s, zsl, zsu, ss);
    for (int i = 0; i < nw; ++i) {
      sw[i] += zeta * dr2[i];
      rw[i] = zeta * dr2[i] * (w[i] - wR[i]) + (grad[i] - gradf[i]) + bw.bgrad(w, i, mur);
    }
    double dual = 0.0, prim = 0.0;
    for (int i = 0; i < nw; ++i) dual = std::max(dual, std::fabs(rw[i]));
    for (int i = 0; i < nx; ++i) prim = std::max(prim, std::fabs(g[i]));
    for (int i = 0; i < m; ++i) {
      sp[i] = zp[i] / p[i];
      sn[i] = zn[i] / n[i];
      const double dc = 1.0 / sp[i] + 1.0 / sn[i];
      st[i] = ss[i] / (1.0 + dc * ss[i]);
      rs[i] = y[i] + bs.bgrad(s, i, mur);
      ry[i] = hv[i] + s[i] - p[i] + n[i];
      rp[i] = rho - y[i] - mur / p[i];
      rn[i] = rho + y[i] - mur / n[i];
      dual = std::max(dual, std::max(std::fabs(rs[i]), std::max(std::fabs(rp[i]), std::fabs(rn[i]))));
      prim = std::max(prim, std::fabs(ry[i]));
      // the relaxation folded into the inequality row, then the slack row too
      r[nw + m + nx + i] = ry[i] + rp[i] / sp[i] - rn[i] / sn[i] - rs[i] / ss[i];
      r[nw + i] = 0.0;
    }
    for (int i = 0; i < nw; ++i) r[i] = rw[i];
    for (int i = 0; i < nx; ++i) r[nw + m + i] = g[i];
    TRYD(h2d(h->s, d.sig_u, sw.data(), nu));
    TRYD(h2d(h->s, d.sig_x, sw.data() + nu, nx));
    TRYD(h2d(h->s, d.sig_s, st.data(), m));
    TRYD(h2d(h->s, d.rhs, r.data(), nkkt));
    int att = 1, gi = 0;
    {
      const int rc0 = condense_factor0(h, d, &gi, !h->ipm_fs);
      if (rc0 == OPF_OK) delta = 0.0;
      else if (rc0 == OPF_ERR_NOT_PD) { TRYD(factor_with_correction(h, delta, delta, att, true)); ++att; }
      else return rc0;
    }
    R.n_factor += att;
    if (h->fr_have_b && !h->ipm_fs) TRYD(kkt_solve_prepared(h, d.step));
    else TRYD(solve_step(h, d.rhs, d.step));
    TRYD(d2h(h->s, step.data(), d.step, nkkt));
    CKD(cudaStreamSynchronize(h->s));
    std::copy(step.begin(), step.begin() + nw, pw.begin());
    std::copy(step.begin() + nw + m, step.begin() + nw + m + nx, pl.begin());
    std::copy(step.begin() + nw + m + nx, step.end(), py.begin());
    for (int i = 0; i < m; ++i) {
      ps[i] = -(rs[i] + py[i]) / ss[i];    // the slack row of K_aug
      pp[i] = (py[i] - rp[i]) / sp[i];
      pn[i] = (-py[i] - rn[i]) / sn[i];
    }
    const double tau = std::max(TAU_MIN, 1.0 - mur);
    double amax = std::min(bw.max_step(w, pw, tau), bs.max_step(s, ps, tau));
    for (int i = 0; i < m; ++i) {
      if (pp[i] < 0) amax = std::min(amax, -tau * p[i] / pp[i]);
      if (pn[i] < 0) amax = std::min(amax, -tau * n[i] / pn[i]);
    }
    bw.dz(w, zwl, zwu, pw, mur, dzwl, dzwu);
    bs.dz(s, zsl, zsu, ps, mur, dzsl, dzsu);
    for (int i = 0; i < m; ++i) {
      dzp[i] = mur / p[i] - zp[i] - sp[i] * pp[i];
      dzn[i] = mur / n[i] - zn[i] - sn[i] * pn[i];
    }
    const double az = std::min(std::min(std::min(max_step_z(zwl, dzwl, bw.fl, tau), max_step_z(zwu, dzwu, bw.fu, tau)),
                                        std::min(max_step_z(zsl, dzsl, bs.fl, tau), max_step_z(zsu, dzsu, bs.fu, tau))),
                               std::min(max_step_z(zp, dzp, all, tau), max_step_z(zn, dzn, all, tau)));
    double mmax = 0.0;
    for (int i = 0; i < nx; ++i) mmax = std::max(mmax, std::fabs(lam[i] + pl[i]));
    for (int i = 0; i < m; ++i) mmax = std::max(mmax, std::fabs(y[i] + py[i]));
    nu_pen = std::max(nu_pen, 1.1 * mmax);
    // l1 merit of the restoration barrier problem and its directional derivative
    auto merit = [&](const Vec& wv, const Vec& sv, const Vec& pv, const Vec& nv, const Vec& gv, const Vec& hh) {
      double v = bw.barrier(wv, mur) + bs.barrier(sv, mur), c1 = 0.0;
      for (int i = 0; i < nw; ++i) v += 0.5 * zeta * dr2[i] * (wv[i] - wR[i]) * (wv[i] - wR[i]);
      for (int i = 0; i < m; ++i) {
        v += rho * (pv[i] + nv[i]) - mur * (std::log(pv[i]) + std::log(nv[i]));
        c1 += std::fabs(hh[i] + sv[i] - pv[i] + nv[i]);
      }
      for (int i = 0; i < nx; ++i) c1 += std::fabs(gv[i]);
      return v + nu_pen * c1;
    };
    const double psi0 = merit(w, s, p, n, g, hv);
    double dpsi = 0.0, c1 = 0.0;
    for (int i = 0; i < nw; ++i) dpsi += (zeta * dr2[i] * (w[i] - wR[i]) + bw.bgrad(w, i, mur)) * pw[i];
    for (int i = 0; i < m; ++i) {
      dpsi += rho * (pp[i] + pn[i]) + bs.bgrad(s, i, mur) * ps[i] - mur * (pp[i] / p[i] + pn[i] / n[i]);
      c1 += std::fabs(ry[i]);
    }
    for (int i = 0; i < nx; ++i) c1 += std::fabs(g[i]);
    dpsi -= nu_pen * c1;
    double a = amax, ft = 0.0;
    Vec gt, ht;
    for (;;) {
      for (int i = 0; i < nw; ++i) wt[i] = w[i] + a * pw[i];
      for (int i = 0; i < m; ++i) { stt[i] = s[i] + a * ps[i]; pt[i] = p[i] + a * pp[i]; nt[i] = n[i] + a * pn[i]; }
      TRYD(eval_fgh(h, d, wt, ft, gt, ht));
      const double v = merit(wt, stt, pt, nt, gt, ht);
      if ((std::isfinite(v) && v <= psi0 + ETA * a * std::min(dpsi, 0.0)) || a <= 1e-8 * amax) break;
      a *= 0.5;
    }
    w = wt;
    s = stt;
    p = pt;
    n = nt;
    for (int i = 0; i < nx; ++i) lam[i] += a * pl[i];
    for (int i = 0; i < m; ++i) y[i] += a * py[i];
    for (int i = 0; i < nw; ++i) { zwl[i] += az * dzwl[i]; zwu[i] += az * dzwu[i]; }
    for (int i = 0; i < m; ++i) { zsl[i] += az * dzsl[i]; zsu[i] += az * dzsu[i]; }
    bw.safeguard(w, zwl, zwu, mur);
    bs.safeguard(s, zsl, zsu, mur);
    for (int i = 0; i < m; ++i) {
      zp[i] = std::min(std::max(zp[i] + az * dzp[i], mur / (KAPPA_SIGMA * p[i])), KAPPA_SIGMA * mur / p[i]);
      zn[i] = std::min(std::max(zn[i] + az * dzn[i], mur / (KAPPA_SIGMA * n[i])), KAPPA_SIGMA * mur / n[i]);
    }
    double theta = 0.0;
    for (int i = 0; i < nx; ++i) theta += std::fabs(gt[i]);
    for (int i = 0; i < m; ++i) theta += std::fabs(ht[i] + s[i]);
    const double phi = ft + bw.barrier(w, mu) + bs.barrier(s, mu);
    if (verbose)
      std::printf("  resto it %3d theta %.3e (theta_R %.3e) mu_R %.1e a %.2e\n", it, theta, theta_R, mur, a);
    if (theta <= KAPPA_RESTO * theta_R && filt.acceptable(theta, phi)) return OPF_OK;
    if (dual <= KAPPA_EPS * mur && prim <= KAPPA_EPS * mur)
      mur = std::max(0.1 * mu, std::min(KAPPA_MU * mur, std::pow(mur, THETA_MU)));
  }
  return OPF_ERR_INFEASIBLE;
}

// the initial primal point: theta = 0, Vm = 1 at load buses, 1.05 at generator
// buses (clipped to bounds), non-slack Pg at the middle of its range
Vec flat_start(const Plan& P) {
  Vec w(P.nw, 0.0);
  for (int i = 0; i < P.nb; ++i) w[P.vm_w[i]] = 1.0;
  for (int k = 0; k < P.ng; ++k) {
    const int i = P.gbus[k];
    w[P.vm_w[i]] = std::min(std::max(1.05, P.Vmin[i]), P.Vmax[i]);
  }
  for (int k = 1; k < P.ng; ++k) w[P.pg_w[k]] = 0.5 * (P.Pmin[k] + P.Pmax[k]);
  return w;
}

}  // namespace

// ------------------------------------------------------------------ LinRed
int ipm_linred_body(opf_handle* h, const opf_ipm_options& o, opf_ipm_result& R);

int ipm_linred(opf_handle* h, const opf_ipm_options& o, opf_ipm_result& R) {
  h->ipm_fs = o.linear_solver == OPF_LINSOLVE_FULLSPACE;
  h->ipm_verbose = o.verbose != 0;
  const int rc = ipm_linred_body(h, o, R);
  h->ipm_fs = false;
  return rc;
}

int ipm_linred_body(opf_handle* h, const opf_ipm_options& o, opf_ipm_result& R) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  const int nkkt = nw + 2 * m + nx;
  Dev d;
  TRYD(alloc_dev(d, h));
  Vec slo(m), shi(m);
  for (int i = 0; i < m; ++i) { slo[i] = -P.hu[i]; shi[i] = -P.hl[i]; }
  Bounds bw(P.wl, P.wu), bs(slo, shi);
  Vec w = flat_start(P);
  bw.push(w);
  double f;
  Vec g, hv;
  TRYD(eval_fgh(h, d, w, f, g, hv));
  Vec s(m);
  for (int i = 0; i < m; ++i) s[i] = -hv[i];
  bs.push(s);
  Vec lam(nx, 0.0), y(m, 0.0);
  Vec zwl(nw), zwu(nw), zsl(m), zsu(m);
  for (int i = 0; i < nw; ++i) { zwl[i] = bw.fl[i] ? 1.0 : 0.0; zwu[i] = bw.fu[i] ? 1.0 : 0.0; }
  for (int i = 0; i < m; ++i) { zsl[i] = bs.fl[i] ? 1.0 : 0.0; zsu[i] = bs.fu[i] ? 1.0 : 0.0; }
  double mu = o.mu0, nu_pen = 1.0, delta = 0.0, err0 = 1e300;
  Vec grad(nw), gradf(nw), sw, ss, r(nkkt), step(nkkt), dzwl, dzwu, dzsl, dzsu;
  // filter line search: theta_max / theta_min from the starting point's violation
  double theta_init = 0.0;
  for (double v : g) theta_init += std::fabs(v);
  for (int i = 0; i < m; ++i) theta_init += std::fabs(hv[i] + s[i]);
  const double theta_max = 1e4 * std::max(1.0, theta_init), theta_min = 1e-4 * std::max(1.0, theta_init);
  Filter filt;
  double filt_mu = -1.0;
  const auto t_start = clk::now();
  int it = 0;
  R.status = OPF_ERR_NO_CONVERGENCE;
  for (; it <= o.max_iter; ++it) {
    auto t0 = clk::now();
    TRYD(h2d(h->s, d.u, w.data(), nu));
    TRYD(h2d(h->s, d.x, w.data() + nu, nx));
    TRYD(h2d(h->s, d.lam, lam.data(), nx));
    TRYD(h2d(h->s, d.y, y.data(), m));
    TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
    TRYD(lagrangian_gradient(h, d.lam, d.y, d.grad));
    TRYD(d2h(h->s, &f, h->f, 1));
    g.resize(nx);
    hv.resize(m);
    TRYD(d2h(h->s, g.data(), h->g, nx));
    TRYD(d2h(h->s, hv.data(), h->hv, m));
    TRYD(d2h(h->s, grad.data(), d.grad, nw));
    TRYD(d2h(h->s, gradf.data(), h->gradf, nw));
    CKD(cudaStreamSynchronize(h->s));
    R.ms_eval += ms_since(t0);
    // optimality error (mu = 0) and barrier update
    double dual = 0.0, primal = 0.0, zsum = 0.0;
    long long zcnt = 0;
    for (int i = 0; i < nw; ++i) dual = std::max(dual, std::fabs(grad[i] - zwl[i] + zwu[i]));
    for (int i = 0; i < m; ++i) dual = std::max(dual, std::fabs(y[i] - zsl[i] + zsu[i]));
    double pl1 = 0.0;
    for (int i = 0; i < nx; ++i) { primal = std::max(primal, std::fabs(g[i])); pl1 += std::fabs(g[i]); }
    for (int i = 0; i < m; ++i) { primal = std::max(primal, std::fabs(hv[i] + s[i])); pl1 += std::fabs(hv[i] + s[i]); }
    for (double v : lam) zsum += std::fabs(v);
    for (double v : y) zsum += std::fabs(v);
    zcnt += nx + m;
    double zs2 = zsum;
    long long zc2 = zcnt;
    double c0 = std::max(bw.compl_inf(w, zwl, zwu, 0.0, zs2, zc2), bs.compl_inf(s, zsl, zsu, 0.0, zs2, zc2));
    err0 = opt_error(dual, primal, c0, zs2, zc2);
    if (o.verbose) std::printf("linred it %3d obj %.10f err %.2e mu %.1e inf_pr %.2e delta %.1e\n", it, f, err0, mu, primal, delta);
    if (err0 <= o.tol) { R.status = OPF_OK; break; }
    if (it == o.max_iter) break;
    for (;;) {
      double zs3 = zsum;
      long long zc3 = zcnt;
      double cm = std::max(bw.compl_inf(w, zwl, zwu, mu, zs3, zc3), bs.compl_inf(s, zsl, zsu, mu, zs3, zc3));
      double errmu = opt_error(dual, primal, cm, zs3, zc3);
      if (errmu > KAPPA_EPS * mu || mu <= o.tol / 10) break;
      mu = std::max(o.tol / 10, std::min(KAPPA_MU * mu, std::pow(mu, THETA_MU)));
    }
    const double tau = std::max(TAU_MIN, 1.0 - mu);
    if (o.line_search == OPF_LINESEARCH_FILTER && o.restoration && o.start_with_resto && it == 0) {
      // the restoration phase from the starting point, before any step
      filt.reset(theta_max);
      filt_mu = mu;
      filt.pairs.push_back({pl1, f + bw.barrier(w, mu) + bs.barrier(s, mu)});
      TRYD(restoration(h, d, bw, bs, filt, mu, w, s, lam, y, zwl, zwu, zsl, zsu, o.verbose != 0, R));
      ++R.restorations;
      continue;
    }
    bw.sigma(w, zwl, zwu, sw);
    bs.sigma(s, zsl, zsu, ss);
    // right-hand side of the step (it does not depend on the factorisation, so
    // the condensation below carries it as one extra column)
    for (int i = 0; i < nw; ++i) r[i] = grad[i] + bw.bgrad(w, i, mu);
    for (int i = 0; i < m; ++i) r[nw + i] = y[i] + bs.bgrad(s, i, mu);
    for (int i = 0; i < nx; ++i) r[nw + m + i] = g[i];
    for (int i = 0; i < m; ++i) r[nw + m + nx + i] = hv[i] + s[i];
    // condense + factor with inertia correction
    t0 = clk::now();
    TRYD(h2d(h->s, d.sig_u, sw.data(), nu));
    TRYD(h2d(h->s, d.sig_x, sw.data() + nu, nx));
    TRYD(h2d(h->s, d.sig_s, ss.data(), m));
    TRYD(h2d(h->s, d.rhs, r.data(), nkkt));
    // condensation + first Cholesky attempt (one graph); inertia correction
    // only when Kred is not positive definite
    int att = 1;
    {
      const int rc0 = condense_factor0(h, d, &R.graph_iters, !h->ipm_fs);
      R.ms_condense += ms_since(t0);
      t0 = clk::now();
      if (rc0 == OPF_OK) delta = 0.0;
      else if (rc0 == OPF_ERR_NOT_PD) { TRYD(factor_with_correction(h, delta, delta, att, true)); ++att; }
      else return rc0;
    }
    R.n_factor += att;
    R.ms_factor += ms_since(t0);
    Vec pw(nw), ps(m), plam(nx), py(m);
    double amax = 1.0, az = 1.0, a = 1.0;
    bool accepted = false, resto = false;
    for (int attempt = 0; attempt < 40 && !accepted; ++attempt) {
      t0 = clk::now();
      if (h->fr_have_b && !h->ipm_fs) {
        // the right-hand side condensed with the condensation (any refactor
        // since changed delta_w only)
        TRYD(kkt_solve_prepared(h, d.step));
      } else {
        TRYD(h2d(h->s, d.rhs, r.data(), nkkt));
        TRYD(solve_step(h, d.rhs, d.step));
      }
      TRYD(d2h(h->s, step.data(), d.step, nkkt));
      CKD(cudaStreamSynchronize(h->s));
      R.ms_solve += ms_since(t0);
      std::copy(step.begin(), step.begin() + nw, pw.begin());
      std::copy(step.begin() + nw, step.begin() + nw + m, ps.begin());
      std::copy(step.begin() + nw + m, step.begin() + nw + m + nx, plam.begin());
      std::copy(step.begin() + nw + m + nx, step.end(), py.begin());
      bw.dz(w, zwl, zwu, pw, mu, dzwl, dzwu);
      bs.dz(s, zsl, zsu, ps, mu, dzsl, dzsu);
      amax = std::min(bw.max_step(w, pw, tau), bs.max_step(s, ps, tau));
      az = std::min(std::min(max_step_z(zwl, dzwl, bw.fl, tau), max_step_z(zwu, dzwu, bw.fu, tau)),
                    std::min(max_step_z(zsl, dzsl, bs.fl, tau), max_step_z(zsu, dzsu, bs.fu, tau)));
      double mmax = 0.0;
      for (int i = 0; i < nx; ++i) mmax = std::max(mmax, std::fabs(lam[i] + plam[i]));
      for (int i = 0; i < m; ++i) mmax = std::max(mmax, std::fabs(y[i] + py[i]));
      nu_pen = std::max(nu_pen, 1.1 * mmax);
      const double phi0 = f + bw.barrier(w, mu) + bs.barrier(s, mu) + nu_pen * pl1;
      double dphi = -nu_pen * pl1;
      for (int i = 0; i < nw; ++i) dphi += (gradf[i] + bw.bgrad(w, i, mu)) * pw[i];
      for (int i = 0; i < m; ++i) dphi += bs.bgrad(s, i, mu) * ps[i];
      t0 = clk::now();
      a = amax;
      Vec wt(nw), st2(m);
      if (o.line_search == OPF_LINESEARCH_FILTER) {
        // filter line search with second-order corrections (the l1 merit values
        // above are not used); theta0 = |c|_1 at the current point
        if (filt_mu != mu) { filt.reset(theta_max); filt_mu = mu; }
        const double theta0 = pl1, ph0 = f + bw.barrier(w, mu) + bs.barrier(s, mu);
        double dph = 0.0;
        for (int i = 0; i < nw; ++i) dph += (gradf[i] + bw.bgrad(w, i, mu)) * pw[i];
        for (int i = 0; i < m; ++i) dph += bs.bgrad(s, i, mu) * ps[i];
        const double amin = filter_alpha_min(theta0, dph, theta_min);
        bool phi_type = false;
        auto trial = [&](const Vec& wv, const Vec& sv, double& theta, double& phi, Vec& c) -> int {
          double ft;
          Vec gt, ht;
          TRYD(eval_fgh(h, d, wv, ft, gt, ht));
          c.resize(nx + m);
          theta = 0.0;
          for (int i = 0; i < nx; ++i) { c[i] = gt[i]; theta += std::fabs(gt[i]); }
          for (int i = 0; i < m; ++i) { c[nx + i] = ht[i] + sv[i]; theta += std::fabs(c[nx + i]); }
          phi = ft + bw.barrier(wv, mu) + bs.barrier(sv, mu);
          return OPF_OK;
        };
        while (a >= amin && !accepted) {
          for (int i = 0; i < nw; ++i) wt[i] = w[i] + a * pw[i];
          for (int i = 0; i < m; ++i) st2[i] = s[i] + a * ps[i];
          double tht, pht;
          Vec ct;
          TRYD(trial(wt, st2, tht, pht, ct));
          accepted = filter_accepts(filt, theta0, ph0, dph, a, tht, pht, theta_min, phi_type);
          if (!accepted && a == amax && tht >= theta0) {
            // second-order corrections: the constraint part of the right-hand side
            // becomes c_soc = a c(x) + c(x + a d), accumulated; the factors are reused
            Vec csoc(nx + m);
            for (int i = 0; i < nx + m; ++i) csoc[i] = a * r[nw + m + i] + ct[i];
            double th_prev = theta0;
            Vec rs = r, q(nkkt), ws(nw), ssoc(m), cn;
            for (int k = 0; k < SOC_MAX && !accepted; ++k) {
              std::copy(csoc.begin(), csoc.end(), rs.begin() + nw + m);
              TRYD(h2d(h->s, d.rhs, rs.data(), nkkt));
              TRYD(solve_step(h, d.rhs, d.step));
              TRYD(d2h(h->s, q.data(), d.step, nkkt));
              CKD(cudaStreamSynchronize(h->s));
              Vec qw(q.begin(), q.begin() + nw), qs(q.begin() + nw, q.begin() + nw + m);
              const double asoc = std::min(bw.max_step(w, qw, tau), bs.max_step(s, qs, tau));
              for (int i = 0; i < nw; ++i) ws[i] = w[i] + asoc * qw[i];
              for (int i = 0; i < m; ++i) ssoc[i] = s[i] + asoc * qs[i];
              double ths, phs;
              TRYD(trial(ws, ssoc, ths, phs, cn));
              accepted = filter_accepts(filt, theta0, ph0, dph, a, ths, phs, theta_min, phi_type);
              if (accepted) {
                for (int i = 0; i < nw; ++i) pw[i] = asoc * qw[i] / a;   // so that w + a pw = the corrected point
                for (int i = 0; i < m; ++i) ps[i] = asoc * qs[i] / a;
                ++R.soc_steps;
                break;
              }
              if (ths > KAPPA_SOC * th_prev) break;
              th_prev = ths;
              for (int i = 0; i < nx + m; ++i) csoc[i] = asoc * csoc[i] + cn[i];
            }
          }
          if (!accepted) a *= 0.5;
        }
        if (accepted && !phi_type) filt.pairs.push_back({(1.0 - GAMMA_THETA) * theta0, ph0 - GAMMA_PHI * theta0});
        if (!accepted && o.restoration) {
          // out of step length: the current point goes into the filter and the
          // restoration phase takes over
          filt.pairs.push_back({theta0, ph0});
          resto = true;
        }
      } else {
        while (a > 1e-4 * amax) {
          for (int i = 0; i < nw; ++i) wt[i] = w[i] + a * pw[i];
          for (int i = 0; i < m; ++i) st2[i] = s[i] + a * ps[i];
          double ft;
          Vec gt, ht;
          TRYD(eval_fgh(h, d, wt, ft, gt, ht));
          double c1 = 0.0;
          for (double v : gt) c1 += std::fabs(v);
          for (int i = 0; i < m; ++i) c1 += std::fabs(ht[i] + st2[i]);
          const double phit = ft + bw.barrier(wt, mu) + bs.barrier(st2, mu) + nu_pen * c1;
          if (std::isfinite(phit) && phit <= phi0 + ETA * a * std::min(dphi, 0.0)) { accepted = true; break; }
          a *= 0.5;
        }
      }
      R.ms_linesearch += ms_since(t0);
      if (resto) break;
      if (!accepted) {
        // backtracking failed: shorten the step by a larger primal regularisation
        delta = std::max(1e-8, 10.0 * delta);
        TRYD(factor_delta(h, delta));
        ++R.n_factor;
        int rc = read_status(h, nullptr);
        if (rc == OPF_ERR_NOT_PD) { att = 0; TRYD(factor_with_correction(h, delta, delta, att)); R.n_factor += att; }
        else if (rc != OPF_OK) return rc;
      }
    }
    if (resto) {
      TRYD(restoration(h, d, bw, bs, filt, mu, w, s, lam, y, zwl, zwu, zsl, zsu, o.verbose != 0, R));
      ++R.restorations;
      continue;
    }
    for (int i = 0; i < nw; ++i) w[i] += a * pw[i];
    for (int i = 0; i < m; ++i) s[i] += a * ps[i];
    for (int i = 0; i < nx; ++i) lam[i] += a * plam[i];
    for (int i = 0; i < m; ++i) y[i] += a * py[i];
    for (int i = 0; i < nw; ++i) { zwl[i] += az * dzwl[i]; zwu[i] += az * dzwu[i]; }
    for (int i = 0; i < m; ++i) { zsl[i] += az * dzsl[i]; zsu[i] += az * dzsu[i]; }
    bw.safeguard(w, zwl, zwu, mu);
    bs.safeguard(s, zsl, zsu, mu);
  }
  R.iters = it;
  R.obj = f;
  R.err = err0;
  R.mu = mu;
  R.ms_total = ms_since(t_start);
  // the converged state, kept for the dispatch derivative
  h->sol_w = w;
  h->sol_lam = lam;
  h->sol_y = y;
  h->sol_s = s;
  bw.sigma(w, zwl, zwu, h->sol_sig_w);
  bs.sigma(s, zsl, zsu, h->sol_sig_s);
  h->sol_zwl = zwl;
  h->sol_zwu = zwu;
  h->sol_zsl = zsl;
  h->sol_zsu = zsu;
  h->sol_mu = mu;
  h->sol_pg0 = hv.empty() ? 0.0 : hv[0];
  h->have_solution = true;
  h->polished = false;
  return OPF_OK;
}

// ------------------------------------------------------------------ RedLin
int powerflow_impl(opf_handle* h, const double* u, double* x, double tol, int max_iter, int* iters);

int ipm_redlin(opf_handle* h, const opf_ipm_options& o, opf_ipm_result& R) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  const int nkkt = nw + 2 * m + nx;
  Dev d;
  TRYD(alloc_dev(d, h));
  std::vector<int> xb;   // bounded states (Vm at load buses)
  for (int j = 0; j < nx; ++j)
    if (finite_bound(P.wl[nu + j]) || finite_bound(P.wu[nu + j])) xb.push_back(j);
  const int nbnd = int(xb.size());
  const int mr = m + nbnd;
  Vec ulo(P.wl.begin(), P.wl.begin() + nu), uhi(P.wu.begin(), P.wu.begin() + nu);
  Vec slo(mr), shi(mr);
  for (int i = 0; i < m; ++i) { slo[i] = -P.hu[i]; shi[i] = -P.hl[i]; }
  for (int k = 0; k < nbnd; ++k) { slo[m + k] = P.wl[nu + xb[k]]; shi[m + k] = P.wu[nu + xb[k]]; }
  Bounds bu(ulo, uhi), bs(slo, shi);
  Vec w = flat_start(P);
  {
    Bounds bw(P.wl, P.wu);
    bw.push(w);
  }
  auto project = [&](Vec& wt) -> int {   // x <- NR solution at u (device), from wt's x
    TRYD(h2d(h->s, d.u, wt.data(), nu));
    TRYD(h2d(h->s, d.x, wt.data() + nu, nx));
    int its = 0;
    auto t0 = clk::now();
    int rc = powerflow_impl(h, d.u, d.x, o.pf_tol, 30, &its);
    R.ms_pf += ms_since(t0);
    if (rc != OPF_OK) return rc;
    TRYD(d2h(h->s, wt.data() + nu, d.x, nx));
    CKD(cudaStreamSynchronize(h->s));
    return OPF_OK;
  };
  {
    int rc = project(w);
    if (rc != OPF_OK) return rc == OPF_ERR_PF_FAILED ? OPF_ERR_PF_FAILED : rc;
  }
  double f;
  Vec g, hv;
  TRYD(eval_fgh(h, d, w, f, g, hv));
  auto hr_of = [&](const Vec& wt, const Vec& hh, Vec& out) {
    out.resize(mr);
    for (int i = 0; i < m; ++i) out[i] = hh[i];
    for (int k = 0; k < nbnd; ++k) out[m + k] = -wt[nu + xb[k]];
  };
  Vec hr;
  hr_of(w, hv, hr);
  Vec s(mr);
  for (int i = 0; i < mr; ++i) s[i] = -hr[i];
  bs.push(s);
  Vec y(mr, 0.0), lam(nx, 0.0);
  Vec zul(nu), zuu(nu), zsl(mr), zsu(mr);
  for (int i = 0; i < nu; ++i) { zul[i] = bu.fl[i] ? 1.0 : 0.0; zuu[i] = bu.fu[i] ? 1.0 : 0.0; }
  for (int i = 0; i < mr; ++i) { zsl[i] = bs.fl[i] ? 1.0 : 0.0; zsu[i] = bs.fu[i] ? 1.0 : 0.0; }
  double mu = o.mu0, nu_pen = 1.0, delta = 0.0, err0 = 1e300;
  Vec grad0(nw), grad(nw), gradf(nw), su, ss, r(nkkt), step(nkkt), t(nx), dzul, dzuu, dzsl, dzsu;
  const auto t_start = clk::now();
  int it = 0;
  R.status = OPF_ERR_NO_CONVERGENCE;
  for (; it <= o.max_iter; ++it) {
    auto t0 = clk::now();
    Vec yh(y.begin(), y.begin() + m);
    TRYD(h2d(h->s, d.u, w.data(), nu));
    TRYD(h2d(h->s, d.x, w.data() + nu, nx));
    TRYD(h2d(h->s, d.y, yh.data(), m));
    TRYD(eval_impl(h, d.x, d.u, nullptr, nullptr, true));
    TRYD(lagrangian_gradient(h, nullptr, d.y, d.grad));
    TRYD(d2h(h->s, grad0.data(), d.grad, nw));
    TRYD(d2h(h->s, gradf.data(), h->gradf, nw));
    TRYD(d2h(h->s, &f, h->f, 1));
    hv.resize(m);
    TRYD(d2h(h->s, hv.data(), h->hv, m));
    CKD(cudaStreamSynchronize(h->s));
    // adjoint step: lambda = -G_x^{-T} (grad_x f + A_x^T y_h - E_b^T y_b)
    for (int j = 0; j < nx; ++j) t[j] = grad0[nu + j];
    for (int k = 0; k < nbnd; ++k) t[xb[k]] -= y[m + k];
    TRYD(factor_async(h));
    TRYD(read_status(h, nullptr));
    TRYD(h2d(h->s, d.tmp, t.data(), nx));
    TRYD(opf_gx_solve(h, 1, d.tmp, d.lam, 1));
    TRYD(d2h(h->s, lam.data(), d.lam, nx));
    CKD(cudaStreamSynchronize(h->s));
    for (double& v : lam) v = -v;
    TRYD(h2d(h->s, d.lam, lam.data(), nx));
    // Hessian of the Lagrangian at (lambda, y_h); G_x (and its factors) unchanged
    TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
    h->have_lu = true;
    TRYD(lagrangian_gradient(h, d.lam, d.y, d.grad));
    TRYD(d2h(h->s, grad.data(), d.grad, nw));
    CKD(cudaStreamSynchronize(h->s));
    R.ms_eval += ms_since(t0);
    hr_of(w, hv, hr);
    double dual = 0.0, primal = 0.0, zsum = 0.0, pl1 = 0.0;
    long long zcnt = 0;
    for (int i = 0; i < nu; ++i) dual = std::max(dual, std::fabs(grad[i] - zul[i] + zuu[i]));
    for (int i = 0; i < mr; ++i) dual = std::max(dual, std::fabs(y[i] - zsl[i] + zsu[i]));
    for (int i = 0; i < mr; ++i) { primal = std::max(primal, std::fabs(hr[i] + s[i])); pl1 += std::fabs(hr[i] + s[i]); }
    for (double v : y) zsum += std::fabs(v);
    zcnt += mr;
    double zs2 = zsum;
    long long zc2 = zcnt;
    Vec uu(w.begin(), w.begin() + nu);
    double c0 = std::max(bu.compl_inf(uu, zul, zuu, 0.0, zs2, zc2), bs.compl_inf(s, zsl, zsu, 0.0, zs2, zc2));
    err0 = opt_error(dual, primal, c0, zs2, zc2);
    if (o.verbose) std::printf("redlin it %3d obj %.10f err %.2e mu %.1e delta %.1e\n", it, f, err0, mu, delta);
    if (err0 <= o.tol) { R.status = OPF_OK; break; }
    if (it == o.max_iter) break;
    for (;;) {
      double zs3 = zsum;
      long long zc3 = zcnt;
      double cm = std::max(bu.compl_inf(uu, zul, zuu, mu, zs3, zc3), bs.compl_inf(s, zsl, zsu, mu, zs3, zc3));
      double errmu = opt_error(dual, primal, cm, zs3, zc3);
      if (errmu > KAPPA_EPS * mu || mu <= o.tol / 10) break;
      mu = std::max(o.tol / 10, std::min(KAPPA_MU * mu, std::pow(mu, THETA_MU)));
    }
    const double tau = std::max(TAU_MIN, 1.0 - mu);
    bu.sigma(uu, zul, zuu, su);
    bs.sigma(s, zsl, zsu, ss);
    Vec sigx(nx, 0.0);
    for (int k = 0; k < nbnd; ++k) sigx[xb[k]] = ss[m + k];
    t0 = clk::now();
    TRYD(h2d(h->s, d.sig_u, su.data(), nu));
    TRYD(h2d(h->s, d.sig_x, sigx.data(), nx));
    TRYD(h2d(h->s, d.sig_s, ss.data(), m));
    // condensation + first Cholesky attempt (one graph); inertia correction
    // only when Kred is not positive definite
    int att = 1;
    {
      const int rc0 = condense_factor0(h, d, &R.graph_iters);
      R.ms_condense += ms_since(t0);
      t0 = clk::now();
      if (rc0 == OPF_OK) delta = 0.0;
      else if (rc0 == OPF_ERR_NOT_PD) { TRYD(factor_with_correction(h, delta, delta, att, true)); ++att; }
      else return rc0;
    }
    R.n_factor += att;
    R.ms_factor += ms_since(t0);
    // reduced right-hand sides in the full-space layout (r4 = 0)
    Vec r2b(nbnd), r3b(nbnd);
    for (int k = 0; k < nbnd; ++k) {
      r2b[k] = y[m + k] + bs.bgrad(s, m + k, mu);
      r3b[k] = hr[m + k] + s[m + k];
    }
    std::fill(r.begin(), r.end(), 0.0);
    for (int i = 0; i < nu; ++i) r[i] = grad[i] + bu.bgrad(uu, i, mu);
    for (int k = 0; k < nbnd; ++k) r[nu + xb[k]] = -(ss[m + k] * r3b[k] - r2b[k]);
    for (int i = 0; i < m; ++i) r[nw + i] = y[i] + bs.bgrad(s, i, mu);
    for (int i = 0; i < m; ++i) r[nw + m + nx + i] = hv[i] + s[i];
    Vec pu(nu), px(nx), ps(mr), py(mr);
    double amax = 1.0, az = 1.0, a = 1.0;
    bool accepted = false;
    Vec wn;
    for (int attempt = 0; attempt < 40 && !accepted; ++attempt) {
      t0 = clk::now();
      TRYD(h2d(h->s, d.rhs, r.data(), nkkt));
      TRYD(solve_step(h, d.rhs, d.step));
      TRYD(d2h(h->s, step.data(), d.step, nkkt));
      CKD(cudaStreamSynchronize(h->s));
      R.ms_solve += ms_since(t0);
      std::copy(step.begin(), step.begin() + nu, pu.begin());
      std::copy(step.begin() + nu, step.begin() + nw, px.begin());
      for (int i = 0; i < m; ++i) { ps[i] = step[nw + i]; py[i] = step[nw + m + nx + i]; }
      for (int k = 0; k < nbnd; ++k) {
        ps[m + k] = px[xb[k]] - r3b[k];
        py[m + k] = ss[m + k] * (-px[xb[k]] + r3b[k]) - r2b[k];
      }
      bu.dz(uu, zul, zuu, pu, mu, dzul, dzuu);
      bs.dz(s, zsl, zsu, ps, mu, dzsl, dzsu);
      amax = std::min(bu.max_step(uu, pu, tau), bs.max_step(s, ps, tau));
      az = std::min(std::min(max_step_z(zul, dzul, bu.fl, tau), max_step_z(zuu, dzuu, bu.fu, tau)),
                    std::min(max_step_z(zsl, dzsl, bs.fl, tau), max_step_z(zsu, dzsu, bs.fu, tau)));
      double mmax = 0.0;
      for (int i = 0; i < mr; ++i) mmax = std::max(mmax, std::fabs(y[i] + py[i]));
      nu_pen = std::max(nu_pen, 1.1 * mmax);
      const double phi0 = f + bu.barrier(uu, mu) + bs.barrier(s, mu) + nu_pen * pl1;
      double dphi = -nu_pen * pl1;
      for (int i = 0; i < nu; ++i) dphi += (gradf[i] + bu.bgrad(uu, i, mu)) * pu[i];
      for (int j = 0; j < nx; ++j) dphi += gradf[nu + j] * px[j];
      for (int i = 0; i < mr; ++i) dphi += bs.bgrad(s, i, mu) * ps[i];
      t0 = clk::now();
      a = amax;
      Vec st2(mr), hrt;
      while (a > 1e-4 * amax) {
        Vec wt = w;
        for (int i = 0; i < nu; ++i) wt[i] = w[i] + a * pu[i];
        for (int j = 0; j < nx; ++j) wt[nu + j] = w[nu + j] + a * px[j];
        for (int i = 0; i < mr; ++i) st2[i] = s[i] + a * ps[i];
        int rc = project(wt);
        if (rc == OPF_OK) {
          double ft;
          Vec gt, ht;
          TRYD(eval_fgh(h, d, wt, ft, gt, ht));
          hr_of(wt, ht, hrt);
          double c1 = 0.0;
          for (int i = 0; i < mr; ++i) c1 += std::fabs(hrt[i] + st2[i]);
          Vec ut(wt.begin(), wt.begin() + nu);
          const double phit = ft + bu.barrier(ut, mu) + bs.barrier(st2, mu) + nu_pen * c1;
          if (std::isfinite(phit) && phit <= phi0 + ETA * a * std::min(dphi, 0.0)) {
            accepted = true;
            wn = wt;
            break;
          }
        } else if (rc != OPF_ERR_PF_FAILED && rc != OPF_ERR_SINGULAR) {
          return rc;
        }
        a *= 0.5;
      }
      R.ms_linesearch += ms_since(t0);
      if (!accepted) {
        delta = std::max(1e-8, 10.0 * delta);
        TRYD(factor_kred_async(h, delta));
        ++R.n_factor;
        int rc = read_status(h, nullptr);
        if (rc == OPF_ERR_NOT_PD) { att = 0; TRYD(factor_with_correction(h, delta, delta, att)); R.n_factor += att; }
        else if (rc != OPF_OK) return rc;
      }
    }
    if (!accepted) { R.status = OPF_ERR_NO_CONVERGENCE; break; }
    w = wn;
    for (int i = 0; i < mr; ++i) { s[i] += a * ps[i]; y[i] += a * py[i]; }
    for (int i = 0; i < nu; ++i) { zul[i] += az * dzul[i]; zuu[i] += az * dzuu[i]; }
    for (int i = 0; i < mr; ++i) { zsl[i] += az * dzsl[i]; zsu[i] += az * dzsu[i]; }
    Vec un(w.begin(), w.begin() + nu);
    bu.safeguard(un, zul, zuu, mu);
    bs.safeguard(s, zsl, zsu, mu);
  }
  R.iters = it;
  R.obj = f;
  R.err = err0;
  R.mu = mu;
  R.ms_total = ms_since(t_start);
  // the converged state in the full-space form: state-bound rows become Sigma_x
  h->sol_w = w;
  h->sol_lam = lam;
  h->sol_y.assign(y.begin(), y.begin() + m);
  h->sol_s.assign(s.begin(), s.begin() + m);
  Vec uu(w.begin(), w.begin() + nu);
  bu.sigma(uu, zul, zuu, su);
  bs.sigma(s, zsl, zsu, ss);
  h->sol_sig_w.assign(nw, 0.0);
  for (int i = 0; i < nu; ++i) h->sol_sig_w[i] = su[i];
  for (int k = 0; k < nbnd; ++k) h->sol_sig_w[nu + xb[k]] = ss[m + k];
  h->sol_sig_s.assign(ss.begin(), ss.begin() + m);
  // bound multipliers: the state-bound rows' slack multipliers are those of x's bounds
  h->sol_zwl.assign(nw, 0.0);
  h->sol_zwu.assign(nw, 0.0);
  for (int i = 0; i < nu; ++i) { h->sol_zwl[i] = zul[i]; h->sol_zwu[i] = zuu[i]; }
  for (int k = 0; k < nbnd; ++k) { h->sol_zwl[nu + xb[k]] = zsl[m + k]; h->sol_zwu[nu + xb[k]] = zsu[m + k]; }
  h->sol_zsl.assign(zsl.begin(), zsl.begin() + m);
  h->sol_zsu.assign(zsu.begin(), zsu.begin() + m);
  h->polished = false;
  h->sol_mu = mu;
  h->sol_pg0 = hv.empty() ? 0.0 : hv[0];
  h->have_solution = true;
  return OPF_OK;
}

// Device scratch and workspace of the interior-point loop, allocated ahead of
// the solves (opf_batch_create calls it before concurrent solves start).
int ipm_reserve(opf_handle* h) {
  Dev d;
  return alloc_dev(d, h);
}

// Run the multi-RHS solve autotuner at the flat start with zero multipliers and
// unit Sigma: which kernel is fastest depends on the network's sparsity and
// the number of right-hand sides, not on the values.
int autotune_at_flat_start(opf_handle* h) {
  const Plan& P = h->P;
  Dev d;
  TRYD(alloc_dev(d, h));
  Vec w = flat_start(P);
  Bounds(P.wl, P.wu).push(w);
  Vec ones(std::max(P.nw, P.m), 1.0);
  TRYD(h2d(h->s, d.u, w.data(), P.nu));
  TRYD(h2d(h->s, d.x, w.data() + P.nu, P.nx));
  CKD(cudaMemsetAsync(d.lam, 0, sizeof(double) * std::max(1, P.nx), h->s));
  CKD(cudaMemsetAsync(d.y, 0, sizeof(double) * std::max(1, P.m), h->s));
  TRYD(h2d(h->s, d.sig_u, ones.data(), P.nu));
  TRYD(h2d(h->s, d.sig_x, ones.data(), P.nx));
  TRYD(h2d(h->s, d.sig_s, ones.data(), P.m));
  TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
  TRYD(condense_async(h, d.sig_u, d.sig_x, d.sig_s));
  return read_status(h, nullptr);
}

// ------------------------------------------------------------------ polish
// Newton's method on the full-space barrier KKT system at the fixed mu of the
// stored solution, from that solution: the point whose derivative the dispatch
// VJP takes.  Full primal-dual steps cut only by the fraction-to-the-boundary
// rule (tau = 0.995); each K_aug solve is refined against the full matrix.
// Stops when the residual (stationarity, feasibility, perturbed
// complementarity; max-norm) is <= tol or stops falling below 1e-9.
int polish_solution(opf_handle* h, double tol, int max_iter) {
  const Plan& P = h->P;
  const int nu = P.nu, nx = P.nx, nw = P.nw, m = P.m;
  const int nkkt = nw + 2 * m + nx;
  const double mu = h->sol_mu;
  Dev d;
  TRYD(alloc_dev(d, h));
  Vec slo(m), shi(m);
  for (int i = 0; i < m; ++i) { slo[i] = -P.hu[i]; shi[i] = -P.hl[i]; }
  Bounds bw(P.wl, P.wu), bs(slo, shi);
  Vec w = h->sol_w, s = h->sol_s, lam = h->sol_lam, y = h->sol_y;
  Vec zwl = h->sol_zwl, zwu = h->sol_zwu, zsl = h->sol_zsl, zsu = h->sol_zsu;
  Vec g(nx), hv(m), grad(nw), sw, ss, r(nkkt), step(nkkt), dzwl, dzwu, dzsl, dzsu;
  double prev = 1e300, res = 1e300;
  int it = 0;
  for (;; ++it) {
    TRYD(h2d(h->s, d.u, w.data(), nu));
    TRYD(h2d(h->s, d.x, w.data() + nu, nx));
    TRYD(h2d(h->s, d.lam, lam.data(), nx));
    TRYD(h2d(h->s, d.y, y.data(), m));
    TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
    TRYD(lagrangian_gradient(h, d.lam, d.y, d.grad));
    TRYD(d2h(h->s, g.data(), h->g, nx));
    TRYD(d2h(h->s, hv.data(), h->hv, m));
    TRYD(d2h(h->s, grad.data(), d.grad, nw));
    CKD(cudaStreamSynchronize(h->s));
    res = 0.0;
    for (int i = 0; i < nw; ++i) res = std::max(res, std::fabs(grad[i] - zwl[i] + zwu[i]));
    for (int i = 0; i < m; ++i) res = std::max(res, std::fabs(y[i] - zsl[i] + zsu[i]));
    for (int i = 0; i < nx; ++i) res = std::max(res, std::fabs(g[i]));
    for (int i = 0; i < m; ++i) res = std::max(res, std::fabs(hv[i] + s[i]));
    double zs = 0.0;
    long long zc = 0;
    res = std::max(res, std::max(bw.compl_inf(w, zwl, zwu, mu, zs, zc), bs.compl_inf(s, zsl, zsu, mu, zs, zc)));
    if (!std::isfinite(res)) return OPF_ERR_NO_CONVERGENCE;
    if (res <= tol || (res < 1e-9 && res > 0.5 * prev) || it == max_iter) break;
    prev = res;
    bw.sigma(w, zwl, zwu, sw);
    bs.sigma(s, zsl, zsu, ss);
    TRYD(h2d(h->s, d.sig_u, sw.data(), nu));
    TRYD(h2d(h->s, d.sig_x, sw.data() + nu, nx));
    TRYD(h2d(h->s, d.sig_s, ss.data(), m));
    TRYD(condense_async(h, d.sig_u, d.sig_x, d.sig_s));
    TRYD(read_status(h, nullptr));
    TRYD(factor_kred_async(h, 0.0));
    TRYD(read_status(h, nullptr));
    h->have_factor = true;
    for (int i = 0; i < nw; ++i) r[i] = grad[i] + bw.bgrad(w, i, mu);
    for (int i = 0; i < m; ++i) r[nw + i] = y[i] + bs.bgrad(s, i, mu);
    for (int i = 0; i < nx; ++i) r[nw + m + i] = g[i];
    for (int i = 0; i < m; ++i) r[nw + m + nx + i] = hv[i] + s[i];
    TRYD(h2d(h->s, d.rhs, r.data(), nkkt));
    TRYD(kkt_solve_impl(h, d.rhs, d.step, 1, 4));
    TRYD(d2h(h->s, step.data(), d.step, nkkt));
    CKD(cudaStreamSynchronize(h->s));
    Vec pw(step.begin(), step.begin() + nw), ps(step.begin() + nw, step.begin() + nw + m);
    bw.dz(w, zwl, zwu, pw, mu, dzwl, dzwu);
    bs.dz(s, zsl, zsu, ps, mu, dzsl, dzsu);
    double a = std::min(bw.max_step(w, pw, 0.995), bs.max_step(s, ps, 0.995));
    a = std::min(a, std::min(std::min(max_step_z(zwl, dzwl, bw.fl, 0.995), max_step_z(zwu, dzwu, bw.fu, 0.995)),
                             std::min(max_step_z(zsl, dzsl, bs.fl, 0.995), max_step_z(zsu, dzsu, bs.fu, 0.995))));
    for (int i = 0; i < nw; ++i) { w[i] += a * pw[i]; zwl[i] += a * dzwl[i]; zwu[i] += a * dzwu[i]; }
    for (int i = 0; i < m; ++i) {
      s[i] += a * ps[i];
      y[i] += a * step[nw + m + nx + i];
      zsl[i] += a * dzsl[i];
      zsu[i] += a * dzsu[i];
    }
    for (int i = 0; i < nx; ++i) lam[i] += a * step[nw + m + i];
  }
  h->sol_w = w;
  h->sol_s = s;
  h->sol_lam = lam;
  h->sol_y = y;
  h->sol_zwl = zwl;
  h->sol_zwu = zwu;
  h->sol_zsl = zsl;
  h->sol_zsu = zsu;
  bw.sigma(w, zwl, zwu, h->sol_sig_w);
  bs.sigma(s, zsl, zsu, h->sol_sig_s);
  h->sol_pg0 = hv.empty() ? 0.0 : hv[0];
  h->polish_iters = it;
  h->polish_res = res;
  return OPF_OK;
}

}  // namespace condipm

using namespace condipm;

extern "C" int opf_solve(opf_handle* h, const opf_ipm_options* opt, opf_ipm_result* res) {
  if (!h || !res) return OPF_ERR_INVALID_ARG;
  opf_ipm_options o{};
  o.variant = OPF_LINRED;
  o.tol = 1e-8;
  o.max_iter = 300;
  o.mu0 = 0.1;
  o.pf_tol = 1e-10;
  o.line_search = OPF_LINESEARCH_MERIT;
  if (opt) o = *opt;
  if (!(o.tol > 0) || o.max_iter < 0 || !(o.mu0 > 0) || !(o.pf_tol > 0) ||
      (o.variant != OPF_LINRED && o.variant != OPF_REDLIN) ||
      (o.line_search != OPF_LINESEARCH_MERIT && o.line_search != OPF_LINESEARCH_FILTER) ||
      (o.line_search == OPF_LINESEARCH_FILTER && o.variant != OPF_LINRED) ||
      (o.linear_solver != OPF_LINSOLVE_CONDENSED && o.linear_solver != OPF_LINSOLVE_FULLSPACE) ||
      (o.linear_solver == OPF_LINSOLVE_FULLSPACE && o.variant != OPF_LINRED) ||
      ((o.restoration || o.start_with_resto) && o.line_search != OPF_LINESEARCH_FILTER) ||
      (o.start_with_resto && !o.restoration))
    return OPF_ERR_INVALID_ARG;
  *res = opf_ipm_result{};
  h->have_solution = false;
  const int rc = o.variant == OPF_LINRED ? ipm_linred(h, o, *res) : ipm_redlin(h, o, *res);
  if (rc != OPF_OK) { res->status = rc; return rc; }
  return res->status;
}

extern "C" int opf_get_solution(const opf_handle* h, double* w, double* lam, double* y, double* Pg) {
  if (!h || !h->have_solution) return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  if (w) std::copy(h->sol_w.begin(), h->sol_w.end(), w);
  if (lam) std::copy(h->sol_lam.begin(), h->sol_lam.end(), lam);
  if (y) std::copy(h->sol_y.begin(), h->sol_y.end(), y);
  if (Pg) {
    // Pg of the slack generator from the slack row of h at the solution
    for (int k = 1; k < P.ng; ++k) Pg[k] = h->sol_w[P.pg_w[k]];
    Pg[0] = h->sol_pg0;
  }
  return OPF_OK;
}

// One Newton step of the barrier KKT system (Algorithm 1, its linear-algebra
// core) from host buffers: copy in, evaluate (A1-A3), condense (A4-A7), factor
// (A9, with delta_w and delta_c), solve and recover (A8, A10), copy out.  The
// copies run on the handle's stream through the loop's own device buffers.
extern "C" int opf_newton_step(opf_handle* h, const double* x, const double* u, const double* lam,
                               const double* y, const double* sig_u, const double* sig_x,
                               const double* sig_s, const double* rhs, double delta_w, double delta_c,
                               double* step, int* fail_col) {
  if (fail_col) *fail_col = -1;
  if (!h || !x || !u || !lam || !y || !sig_u || !sig_x || !sig_s || !rhs || !step || !(delta_w >= 0.0) ||
      !(delta_c >= 0.0) || !(delta_c < 1e300))
    return OPF_ERR_INVALID_ARG;
  const Plan& P = h->P;
  const size_t nkkt = (size_t)P.nw + 2 * (size_t)P.m + P.nx;
  Dev d;
  TRYD(alloc_dev(d, h));
  TRYD(h2d(h->s, d.x, x, P.nx));
  TRYD(h2d(h->s, d.u, u, P.nu));
  TRYD(h2d(h->s, d.lam, lam, P.nx));
  TRYD(h2d(h->s, d.y, y, P.m));
  TRYD(h2d(h->s, d.sig_u, sig_u, P.nu));
  TRYD(h2d(h->s, d.sig_x, sig_x, P.nx));
  TRYD(h2d(h->s, d.sig_s, sig_s, P.m));
  TRYD(h2d(h->s, d.rhs, rhs, nkkt));
  TRYD(eval_impl(h, d.x, d.u, d.lam, d.y, true));
  // the condensed right-hand side rides along the condensation (one extra column)
  TRYD(condense_async(h, d.sig_u, d.sig_x, d.sig_s, d.rhs));
  if (delta_c > 0.0) TRYD(recondense_dc(h, delta_c));
  TRYD(factor_kred_async(h, delta_w));
  int info = -1;
  const int rc = read_status(h, &info);
  if (rc != OPF_OK) {
    if (rc == OPF_ERR_NOT_PD && fail_col) *fail_col = info;
    if (rc != OPF_ERR_NOT_PD) h->have_condense = false;
    return rc;
  }
  h->have_factor = true;
  TRYD(kkt_solve_prepared(h, d.step));
  TRYD(d2h(h->s, step, d.step, nkkt));
  CKD(cudaStreamSynchronize(h->s));
  return OPF_OK;
}
