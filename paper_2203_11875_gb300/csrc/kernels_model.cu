// A1-A3: polar power-flow residuals, Jacobians and Lagrangian Hessian (Sec. 3.2).
//
// Every line end e = (bus i, other bus k) carries the flow leaving bus i,
//   p = Vi^2 gs + Vi Vk (gm cos t + bm sin t),  q = -Vi^2 bs + Vi Vk (gm sin t - bm cos t),
// t = theta_i - theta_k, with self admittance gs + j bs and mutual admittance
// gm + j bm of the pi-model.  The bus injections P_i, Q_i (and so g, h) are sums
// of end flows, and all first and second derivatives are sums of per-end 4-vector
// and symmetric 4x4 blocks over the local variables (theta_i, theta_k, Vm_i, Vm_k).
// One thread per end evaluates these blocks; the sparse values of G, A and W are
// then formed by fixed-order gathers (a host-built plan), so every value is a
// deterministic sum, computed by its owner without atomics.
#include "common.cuh"

namespace condipm {
namespace {

__global__ void k_bus_state(int nb, int nu, const double* __restrict__ x, const double* __restrict__ u,
                            const int* __restrict__ th_w, const int* __restrict__ vm_w,
                            double* __restrict__ Vm, double* __restrict__ Va) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  int v = vm_w[i];
  Vm[i] = v < nu ? u[v] : x[v - nu];
  int t = th_w[i];
  Va[i] = t < 0 ? 0.0 : x[t - nu];
}

__global__ void k_end_eval(int ne, const int* __restrict__ end_i, const int* __restrict__ end_k,
                           const int* __restrict__ end_h, const double* __restrict__ gs,
                           const double* __restrict__ bs, const double* __restrict__ gm,
                           const double* __restrict__ bm, const double* __restrict__ Vm,
                           const double* __restrict__ Va, double* __restrict__ pq,
                           double* __restrict__ dsrc, double* __restrict__ hpq, double* __restrict__ h,
                           int want) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int i = end_i[e], k = end_k[e], hr = end_h[e];
  const double Vi = Vm[i], Vk = Vm[k];
  double s, c;
  sincos(Va[i] - Va[k], &s, &c);
  const double g_s = gs[e], b_s = bs[e], g_m = gm[e], b_m = bm[e];
  const double a = g_m * c + b_m * s;     // d a / d t = -bb
  const double bb = g_m * s - b_m * c;    // d bb / d t = a
  const double ViVk = Vi * Vk;
  const double p = Vi * Vi * g_s + ViVk * a;
  const double q = -Vi * Vi * b_s + ViVk * bb;
  pq[2 * e] = p;
  pq[2 * e + 1] = q;
  if (hr >= 0) h[hr] = p * p + q * q;
  if (!want) return;
  const double dp[4] = {-ViVk * bb, ViVk * bb, 2.0 * Vi * g_s + Vk * a, Vi * a};
  const double dq[4] = {ViVk * a, -ViVk * a, -2.0 * Vi * b_s + Vk * bb, Vi * bb};
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    dsrc[4 * e + l] = dp[l];
    dsrc[4 * (size_t)ne + 4 * e + l] = dq[l];
    dsrc[8 * (size_t)ne + 4 * e + l] = hr >= 0 ? 2.0 * (p * dp[l] + q * dq[l]) : 0.0;
  }
  // upper triangles of the 4x4 Hessians, order (00,01,02,03,11,12,13,22,23,33)
  double* hp = hpq + 20 * (size_t)e;
  double* hq = hp + 10;
  hp[0] = -ViVk * a; hp[1] = ViVk * a; hp[2] = -Vk * bb; hp[3] = -Vi * bb;
  hp[4] = -ViVk * a; hp[5] = Vk * bb;  hp[6] = Vi * bb;  hp[7] = 2.0 * g_s;
  hp[8] = a;         hp[9] = 0.0;
  hq[0] = -ViVk * bb; hq[1] = ViVk * bb; hq[2] = Vk * a; hq[3] = Vi * a;
  hq[4] = -ViVk * bb; hq[5] = -Vk * a;   hq[6] = -Vi * a; hq[7] = -2.0 * b_s;
  hq[8] = bb;         hq[9] = 0.0;
}

__global__ void k_bus_sum(int nb, int ng, int nu, int slack, const int* __restrict__ bus_end_ptr,
                          const int* __restrict__ bus_end, const double* __restrict__ pq,
                          const int* __restrict__ g_row_P, const int* __restrict__ g_row_Q,
                          const int* __restrict__ gen_of_bus, const double* __restrict__ Pd,
                          const double* __restrict__ Qd, const double* __restrict__ u,
                          const double* __restrict__ c2, const double* __restrict__ c1,
                          const double* __restrict__ lam, const double* __restrict__ y,
                          double* __restrict__ g, double* __restrict__ h, double* __restrict__ Pg,
                          double* __restrict__ wP, double* __restrict__ wQ) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double P = 0.0, Q = 0.0;
  for (int t = bus_end_ptr[i]; t < bus_end_ptr[i + 1]; ++t) {
    int e = bus_end[t];
    P += pq[2 * e];
    Q += pq[2 * e + 1];
  }
  const int kP = g_row_P[i], kQ = g_row_Q[i], gk = gen_of_bus[i];
  const double Pgi = gk >= 1 ? u[ng + gk - 1] : 0.0;
  if (kP >= 0) g[kP] = P - Pgi + Pd[i];
  if (kQ >= 0) g[kQ] = Q + Qd[i];
  double Pg0 = 0.0;
  if (i == slack) {
    Pg0 = P + Pd[i];
    h[0] = Pg0;
    Pg[0] = Pg0;
  }
  if (gk >= 0) h[1 + gk] = Q + Qd[i];
  if (gk >= 1) Pg[gk] = Pgi;
  if (lam != nullptr) {
    double a = kP >= 0 ? lam[kP] : 0.0;
    if (i == slack) a += 2.0 * c2[0] * Pg0 + c1[0] + y[0];
    double b = kQ >= 0 ? lam[kQ] : 0.0;
    if (gk >= 0) b += y[1 + gk];
    wP[i] = a;
    wQ[i] = b;
  }
}

// f = sum_k c2 Pg^2 + c1 Pg by one block with a fixed reduction tree
__global__ void k_objective(int ng, const double* __restrict__ Pg, const double* __restrict__ c2,
                            const double* __restrict__ c1, double* __restrict__ f) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int k = threadIdx.x; k < ng; k += blockDim.x) acc += (c2[k] * Pg[k] + c1[k]) * Pg[k];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *f = sh[0];
}

__global__ void k_gather(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                         const double* __restrict__ cst, const double* __restrict__ src,
                         double* __restrict__ out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double acc = cst[p];
  for (int q = ptr[p]; q < ptr[p + 1]; ++q) acc += src[idx[q]];
  out[p] = acc;
}

__global__ void k_gradf(int nw, int ng, const int* __restrict__ pg_of_w, const int* __restrict__ slackpos,
                        const double* __restrict__ Pg, const double* __restrict__ c2,
                        const double* __restrict__ c1, const double* __restrict__ Aval,
                        double* __restrict__ gradf) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  double v = 0.0;
  int k = pg_of_w[w];
  if (k >= 1) v = 2.0 * c2[k] * Pg[k] + c1[k];
  int sp = slackpos[w];
  if (sp >= 0) v += (2.0 * c2[0] * Pg[0] + c1[0]) * Aval[sp];
  gradf[w] = v;
}

__global__ void k_end_hess(int ne, const int* __restrict__ end_i, const int* __restrict__ end_h,
                           const double* __restrict__ pq, const double* __restrict__ dsrc,
                           const double* __restrict__ hpq, const double* __restrict__ wP,
                           const double* __restrict__ wQ, const double* __restrict__ y,
                           double* __restrict__ hw) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int i = end_i[e], hr = end_h[e];
  const double a = wP[i], b = wQ[i];
  const double* hp = hpq + 20 * (size_t)e;
  const double* hq = hp + 10;
  double out[10];
#pragma unroll
  for (int t = 0; t < 10; ++t) out[t] = a * hp[t] + b * hq[t];
  if (hr >= 0) {
    // y_l * hess(p^2 + q^2) = 2 y_l (dp dp^T + p hp + dq dq^T + q hq)
    const double yl2 = 2.0 * y[hr];
    const double p = pq[2 * e], q = pq[2 * e + 1];
    double dp[4], dq[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      dp[l] = dsrc[4 * e + l];
      dq[l] = dsrc[4 * (size_t)ne + 4 * e + l];
    }
    const int ia[10] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
    const int ib[10] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
#pragma unroll
    for (int t = 0; t < 10; ++t)
      out[t] += yl2 * (dp[ia[t]] * dp[ib[t]] + p * hp[t] + dq[ia[t]] * dq[ib[t]] + q * hq[t]);
  }
  double* o = hw + 10 * (size_t)e;
#pragma unroll
  for (int t = 0; t < 10; ++t) o[t] = out[t];
}

__global__ void k_bilin_fixed(int n, const int* __restrict__ pos, const int* __restrict__ a,
                              const int* __restrict__ b, double coef, const double* __restrict__ A,
                              double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  out[pos[t]] += coef * A[a[t]] * A[b[t]];
}

inline int nblk(long long n, int t) { return int((n + t - 1) / t); }

}  // namespace

cudaError_t launch_bus_state(cudaStream_t s, int nb, int nu, const double* x, const double* u,
                             const int* th_w, const int* vm_w, double* Vm, double* Va) {
  k_bus_state<<<nblk(nb, 256), 256, 0, s>>>(nb, nu, x, u, th_w, vm_w, Vm, Va);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_end_eval(cudaStream_t s, int ne, const int* end_i, const int* end_k,
                            const int* end_h, const double* gs, const double* bs, const double* gm,
                            const double* bm, const double* Vm, const double* Va, double* pq,
                            double* dsrc, double* hpq, double* h, int want_derivs) {
  k_end_eval<<<nblk(ne, 128), 128, 0, s>>>(ne, end_i, end_k, end_h, gs, bs, gm, bm, Vm, Va, pq, dsrc,
                                            hpq, h, want_derivs);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bus_sum(cudaStream_t s, int nb, int ng, int nu, int slack, const int* bus_end_ptr,
                           const int* bus_end, const double* pq, const int* g_row_P,
                           const int* g_row_Q, const int* gen_of_bus, const double* Pd,
                           const double* Qd, const double* u, const double* c2, const double* c1,
                           const double* lam, const double* y, double* g, double* h, double* Pg,
                           double* wP, double* wQ) {
  k_bus_sum<<<nblk(nb, 256), 256, 0, s>>>(nb, ng, nu, slack, bus_end_ptr, bus_end, pq, g_row_P,
                                          g_row_Q, gen_of_bus, Pd, Qd, u, c2, c1, lam, y, g, h, Pg,
                                          wP, wQ);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_objective(cudaStream_t s, int ng, const double* Pg, const double* c2,
                             const double* c1, double* f) {
  k_objective<<<1, 256, 0, s>>>(ng, Pg, c2, c1, f);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather(cudaStream_t s, int n, const int* ptr, const int* idx, const double* cst,
                          const double* src, double* out) {
  if (n <= 0) return cudaSuccess;
  k_gather<<<nblk(n, 256), 256, 0, s>>>(n, ptr, idx, cst, src, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gradf(cudaStream_t s, int nw, int ng, const int* pg_of_w, const int* slackpos,
                         const double* Pg, const double* c2, const double* c1, const double* Aval,
                         double* gradf) {
  k_gradf<<<nblk(nw, 256), 256, 0, s>>>(nw, ng, pg_of_w, slackpos, Pg, c2, c1, Aval, gradf);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_end_hess(cudaStream_t s, int ne, const int* end_i, const int* end_h,
                            const double* pq, const double* dsrc, const double* hpq, const double* wP,
                            const double* wQ, const double* y, double* hw) {
  k_end_hess<<<nblk(ne, 128), 128, 0, s>>>(ne, end_i, end_h, pq, dsrc, hpq, wP, wQ, y, hw);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_bilin_fixed(cudaStream_t s, int n, const int* pos, const int* a, const int* b,
                               double coef, const double* A, double* out) {
  if (n <= 0) return cudaSuccess;
  k_bilin_fixed<<<nblk(n, 256), 256, 0, s>>>(n, pos, a, b, coef, A, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace condipm
