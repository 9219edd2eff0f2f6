// Measured FP64 throughput of the device: the roofline denominator of the FP64
// kernels of this library (the measured-peak file of the GPU pool lists HBM and
// bf16 figures only).
//
//  * DFMA: every thread of a full grid runs independent fma chains; the FP64
//    pipe of each SM sub-partition is the only unit in use.
//  * f64 mma.sync (the warp-level FP64 tensor-core path; tcgen05 has no f64
//    kind): each warp keeps four independent accumulators of one shape in flight.
// Each figure is the better of two timed launches (CUDA events on one stream),
// flop counted as 2 per fused multiply-add.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/condipm.h"
#include "common.cuh"

namespace condipm {
namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_peak_dfma(int iters, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) a[c] = 1e-3 * (t & 63) + 0.1 * c;
  const double b = 0.9999999, d = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += a[c];
  out[t] = s;
}

// shape 0: m8n8k4 (A 1, B 1, C 2 registers per lane); 1: m16n8k4 (2, 1, 4);
// 2: m16n8k16 (8, 4, 4).  Four independent accumulators per warp.
template <int SHAPE>
__global__ void __launch_bounds__(PK_THREADS) k_peak_dmma(int iters, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int NA = SHAPE == 0 ? 1 : (SHAPE == 1 ? 2 : 8);
  constexpr int NB = SHAPE == 2 ? 4 : 1;
  constexpr int NC = SHAPE == 0 ? 2 : 4;
  double A[NA], B[NB], Cc[4][NC];
#pragma unroll
  for (int i = 0; i < NA; ++i) A[i] = 1e-4 * ((t + i) & 15);
#pragma unroll
  for (int i = 0; i < NB; ++i) B[i] = 1e-4 * ((t + 3 * i) & 7);
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < NC; ++i) Cc[q][i] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if constexpr (SHAPE == 0) {
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                     : "+d"(Cc[q][0]), "+d"(Cc[q][1])
                     : "d"(A[0]), "d"(B[0]));
      } else if constexpr (SHAPE == 1) {
        asm volatile("mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                     "{%0,%1,%2,%3};\n"
                     : "+d"(Cc[q][0]), "+d"(Cc[q][1]), "+d"(Cc[q][2]), "+d"(Cc[q][3])
                     : "d"(A[0]), "d"(A[1]), "d"(B[0]));
      } else {
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
                     "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
                     : "+d"(Cc[q][0]), "+d"(Cc[q][1]), "+d"(Cc[q][2]), "+d"(Cc[q][3])
                     : "d"(A[0]), "d"(A[1]), "d"(A[2]), "d"(A[3]), "d"(A[4]), "d"(A[5]), "d"(A[6]), "d"(A[7]),
                       "d"(B[0]), "d"(B[1]), "d"(B[2]), "d"(B[3]));
      }
    }
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < NC; ++i) s += Cc[q][i];
  out[t] = s;
}

}  // namespace
}  // namespace condipm

using namespace condipm;

extern "C" int opf_fp64_peak(int which, double* gflops) {
  if (!gflops || which < 0 || which > 3) return OPF_ERR_INVALID_ARG;
  *gflops = 0.0;
  int per = 0;
  cudaError_t e = which == 0
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peak_dfma, PK_THREADS, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peak_dmma<0>, PK_THREADS, 0);
  if (e != cudaSuccess) return OPF_ERR_CUDA;
  const int blocks = device_sms() * std::max(1, std::min(per, 8));
  const long long threads = (long long)blocks * PK_THREADS;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * threads) != cudaSuccess) return OPF_ERR_OOM;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  // flop per thread and iteration: DFMA 2 per chain; mma 2 M N K per warp per
  // accumulator, i.e. 2 M N K / 32 per lane, four accumulators
  const double mnk[3] = {8.0 * 8 * 4, 16.0 * 8 * 4, 16.0 * 8 * 16};
  const double fl_it = which == 0 ? 2.0 * PK_CHAINS : 4.0 * 2.0 * mnk[which - 1] / 32.0;
  const int iters = which == 0 ? 20000 : (which == 3 ? 2500 : 10000);
  float best = 1e30f;
  int rc = OPF_OK;
  for (int rep = 0; rep < 3 && rc == OPF_OK; ++rep) {
    cudaEventRecord(a, 0);
    switch (which) {
      case 0: k_peak_dfma<<<blocks, PK_THREADS>>>(iters, out); break;
      case 1: k_peak_dmma<0><<<blocks, PK_THREADS>>>(iters, out); break;
      case 2: k_peak_dmma<1><<<blocks, PK_THREADS>>>(iters, out); break;
      default: k_peak_dmma<2><<<blocks, PK_THREADS>>>(iters, out); break;
    }
    note_launch();
    cudaEventRecord(b, 0);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = OPF_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (rc != OPF_OK) return rc;
  *gflops = fl_it * (double)iters * (double)threads / (best * 1e-3) / 1e9;
  return OPF_OK;
}
