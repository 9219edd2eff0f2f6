// A6: supernodal multi-right-hand-side triangular solves with the factors of
// P G_x P^T = L U (Sec. 3.3: G_x^{-1} b = Q U^{-1} L^{-1} P b, applied to all nu
// columns of G_u, and the transposed solves of the adjoint route).
//
// Each CTA owns cb right-hand-side columns and keeps them in shared memory for
// the whole solve, so no CTA ever waits for another.  Rows are grouped into
// fundamental supernodes (runs of rows with a dense diagonal block -- the
// (theta, Vm) pair of a bus, and the separator chains of the ordering); the
// supernodes are level-scheduled and packed, in level order, into a byte stream
// of chunks (plan.h, SnStream).  The CTA streams that data through two
// shared-memory buffers with cp.async.bulk (the TMA bulk-copy engine), issuing
// chunk c+1 while it works on chunk c, so that after the first chunk every
// operand comes from shared memory.  Per chunk:
//   A. every row subtracts its external entries (columns of earlier levels):
//      ga lanes per row, shuffle reduction;
//   B. every supernode sweeps its packed dense diagonal triangle with one lane
//      per row and one shuffle broadcast per column, warp-synchronous.
// Supernodes wider than 32 rows sweep 32-column panels with the whole CTA,
// reading their diagonal block from the factor in place.
#include <algorithm>
#include <cstdint>

#include "common.cuh"

#include <cooperative_groups.h>

namespace condipm {
namespace cg = cooperative_groups;
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TRSM_THREADS = 512;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
}

// thread 0: stage chunk bytes [src, src+bytes) into dst, completion on bar
__device__ __forceinline__ void stage_chunk(void* dst, const void* src, int bytes, uint64_t* bar) {
  const uint32_t b = smem_addr(bar);
  if (bytes > 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(b)
        : "memory");
  } else {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
  }
}

// bounded wait for the given phase parity; false when the limit expires
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t b = smem_addr(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int CB>
__device__ __forceinline__ void chunk_phase_a(const unsigned char* B, double* Xs) {
  const int* hdr = reinterpret_cast<const int*>(B);
  const int nA = hdr[0], ga = hdr[4];
  const int* Aptr = reinterpret_cast<const int*>(B + hdr[8]);
  const int* Arow = reinterpret_cast<const int*>(B + hdr[9]);
  const int* Eci = reinterpret_cast<const int*>(B + hdr[10]);
  const double* Eval = reinterpret_cast<const double*>(B + hdr[11]);
  const int tid = threadIdx.x;
  const int grp = tid / ga, lig = tid % ga, ngrp = blockDim.x / ga;
  for (int base = 0; base < nA; base += ngrp) {
    const int t = base + grp;
    double part[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) part[c] = 0.0;
    int r = -1;
    if (t < nA) {
      r = Arow[t];
      const int qe = Aptr[t + 1];
      for (int q = Aptr[t] + lig; q < qe; q += ga) {
        const double v = Eval[q];
        const int j = Eci[q];
#pragma unroll
        for (int c = 0; c < CB; ++c) part[c] = fma(v, Xs[j * CB + c], part[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < CB; ++c)
      for (int o = ga >> 1; o > 0; o >>= 1) part[c] += __shfl_xor_sync(FULL, part[c], o, ga);
    if (lig == 0 && r >= 0) {
#pragma unroll
      for (int c = 0; c < CB; ++c) Xs[r * CB + c] -= part[c];
    }
  }
}

// narrow supernodes (width <= 4): one lane sweeps a whole supernode, so every
// FP64 instruction of the sweep has all its lanes busy
template <int CB, bool UPPER>
__device__ __forceinline__ void chunk_phase_b_narrow(const unsigned char* B, double* Xs) {
  const int* hdr = reinterpret_cast<const int*>(B);
  const int nB = hdr[1];
  const int* Bf = reinterpret_cast<const int*>(B + hdr[12]);
  const int* Bw = reinterpret_cast<const int*>(B + hdr[13]);
  const int* Biptr = reinterpret_cast<const int*>(B + hdr[14]);
  const int* Bdptr = reinterpret_cast<const int*>(B + hdr[15]);
  const double* Ival = reinterpret_cast<const double*>(B + hdr[16]);
  const double* Bd = reinterpret_cast<const double*>(B + hdr[17]);
  for (int s = threadIdx.x; s < nB; s += blockDim.x) {
    const int f = Bf[s], w = Bw[s];
    const double* tri = Ival + Biptr[s];
    const double* dg = Bd + Bdptr[s];
#pragma unroll
    for (int c = 0; c < CB; ++c) {
      double a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = i < w ? Xs[(f + i) * CB + c] : 0.0;
      if (!UPPER) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (t < w) {
            a[t] *= dg[t];
#pragma unroll
            for (int i = t + 1; i < 4; ++i)
              if (i < w) a[i] = fma(-tri[i * (i - 1) / 2 + t], a[t], a[i]);
          }
        }
      } else {
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
          const int t = 3 - tt;
          if (t < w) {
            a[t] *= dg[t];
#pragma unroll
            for (int i = 0; i < t; ++i) a[i] = fma(-tri[i * (w - 1) - i * (i - 1) / 2 + (t - i - 1)], a[t], a[i]);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i < w) Xs[(f + i) * CB + c] = a[i];
    }
  }
}

template <int CB, bool UPPER, int LV>
__device__ __forceinline__ void chunk_phase_b(const unsigned char* B, double* Xs) {
  const int* hdr = reinterpret_cast<const int*>(B);
  const int nB = hdr[1], gs = hdr[5], wmax = hdr[6];
  const int* Bf = reinterpret_cast<const int*>(B + hdr[12]);
  const int* Bw = reinterpret_cast<const int*>(B + hdr[13]);
  const int* Biptr = reinterpret_cast<const int*>(B + hdr[14]);
  const int* Bdptr = reinterpret_cast<const int*>(B + hdr[15]);
  const double* Ival = reinterpret_cast<const double*>(B + hdr[16]);
  const double* Bd = reinterpret_cast<const double*>(B + hdr[17]);
  const int tid = threadIdx.x;
  const int grp = tid / gs, lig = tid % gs, ngrp = blockDim.x / gs;
  for (int base = 0; base < nB; base += ngrp) {
    const int s = base + grp;
    const bool act = s < nB;
    const int f = act ? Bf[s] : 0;
    const int w = act ? Bw[s] : 0;
    const bool own = lig < w;
    const int r = f + lig;
    const double* tri = Ival + (act ? Biptr[s] : 0) +
                        (UPPER ? (lig * (w - 1) - lig * (lig - 1) / 2) : (lig * (lig - 1) / 2));
    double lv[LV];
#pragma unroll
    for (int t = 0; t < LV; ++t) {
      if (!UPPER) lv[t] = (own && t < lig) ? tri[t] : 0.0;
      else lv[t] = (own && t > lig && t < w) ? tri[t - lig - 1] : 0.0;
    }
    double acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = own ? Xs[r * CB + c] : 0.0;
    const double dinv = own ? Bd[Bdptr[s] + lig] : 1.0;
#pragma unroll
    for (int tt = 0; tt < LV; ++tt) {
      const int t = UPPER ? LV - 1 - tt : tt;
      if (t < wmax) {
        if (own && lig == t) {
#pragma unroll
          for (int c = 0; c < CB; ++c) { acc[c] *= dinv; Xs[r * CB + c] = acc[c]; }
        }
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const double xt = __shfl_sync(FULL, acc[c], t, gs);
          if (own && (UPPER ? lig < t : lig > t)) acc[c] = fma(-lv[t], xt, acc[c]);
        }
      }
    }
  }
}

// supernode wider than 32 rows: 32-column panels with the whole CTA, diagonal
// block read from the factor (int_beg / val / inv_diag of the solve)
template <int CB, bool UPPER>
__device__ __forceinline__ void big_supernode(const StDev& T, int f, int w, double* Xs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int npan = (w + 31) / 32;
  for (int pi = 0; pi < npan; ++pi) {
    const int p0 = UPPER ? max(0, w - 32 * (pi + 1)) : 32 * pi;
    const int pe = UPPER ? w - 32 * pi : min(w, 32 * (pi + 1));
    const int pw = pe - p0;
    if (warp == 0) {
      const bool own = lane < pw;
      const int r = f + p0 + lane;
      double lv[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        if (!UPPER) lv[t] = (own && t < lane) ? T.val[T.int_beg[r] + p0 + t] : 0.0;
        else lv[t] = (own && t > lane && t < pw) ? T.val[T.int_beg[r] + (t - lane - 1)] : 0.0;
      }
      double acc[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) acc[c] = own ? Xs[r * CB + c] : 0.0;
      const double dinv = (own && T.inv_diag) ? T.inv_diag[r] : 1.0;
#pragma unroll
      for (int tt = 0; tt < 32; ++tt) {
        const int t = UPPER ? 31 - tt : tt;
        if (t < pw) {
          if (own && lane == t) {
#pragma unroll
            for (int c = 0; c < CB; ++c) { acc[c] *= dinv; Xs[r * CB + c] = acc[c]; }
          }
#pragma unroll
          for (int c = 0; c < CB; ++c) {
            const double xt = __shfl_sync(FULL, acc[c], t);
            if (own && (UPPER ? lane < t : lane > t)) acc[c] = fma(-lv[t], xt, acc[c]);
          }
        }
      }
    }
    __syncthreads();
    const int rb = UPPER ? 0 : pe, re = UPPER ? p0 : w;
    for (int ri = rb + warp; ri < re; ri += nwarps) {
      const int r = f + ri;
      const bool on = lane < pw;
      const double v = on ? (UPPER ? T.val[T.int_beg[r] + (p0 + lane - ri - 1)] : T.val[T.int_beg[r] + p0 + lane])
                          : 0.0;
      double part[CB];
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        part[c] = on ? v * Xs[(f + p0 + lane) * CB + c] : 0.0;
        for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_xor_sync(FULL, part[c], o);
      }
      if (lane == 0) {
#pragma unroll
        for (int c = 0; c < CB; ++c) Xs[r * CB + c] -= part[c];
      }
    }
    __syncthreads();
  }
}

template <int CB, bool UPPER>
__global__ void __launch_bounds__(TRSM_THREADS) k_trsm_st(StDev T, int n, double* X, long long xr, long long xc,
                                                          int ncols, int* st, long long spin_limit) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* Xs = reinterpret_cast<double*>(smem);
  const size_t xs_bytes = ((size_t)n * CB * sizeof(double) + 15) & ~size_t(15);
  unsigned char* buf0 = smem + xs_bytes;
  unsigned char* buf1 = buf0 + T.cap;
  uint64_t* bars = reinterpret_cast<uint64_t*>(buf1 + T.cap);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int c0 = blockIdx.x * CB;
  if (tid == 0) {
    abort_flag = 0;
    mbar_init(&bars[0]);
    mbar_init(&bars[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && T.nchunks > 0)
    stage_chunk(buf0, T.bytes + T.chunk_off[0], T.chunk_bytes[0], &bars[0]);
  for (int t = tid; t < n * CB; t += nthr) {
    const int i = t / CB, c = t % CB;
    Xs[t] = (c0 + c < ncols) ? X[i * xr + (c0 + c) * xc] : 0.0;
  }
  __syncthreads();
  for (int ch = 0; ch < T.nchunks; ++ch) {
    unsigned char* B = (ch & 1) ? buf1 : buf0;
    if (tid == 0 && ch + 1 < T.nchunks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      stage_chunk((ch & 1) ? buf0 : buf1, T.bytes + T.chunk_off[ch + 1], T.chunk_bytes[ch + 1],
                  &bars[(ch + 1) & 1]);
    }
    if (!mbar_wait(&bars[ch & 1], (ch >> 1) & 1, spin_limit)) {
      atomicExch(&abort_flag, 1);
      atomicExch(&st[ST_TIMEOUT], 1);
    }
    __syncthreads();
    if (abort_flag) {
      // let the copies in flight (this chunk's and the next one's) land in shared
      // memory before the CTA leaves; a bulk copy takes microseconds, so these
      // waits get at least 2^22 polls whatever the caller's limit
      if (tid == 0) {
        const long long lim = spin_limit > (1LL << 22) ? spin_limit : (1LL << 22);
        mbar_wait(&bars[ch & 1], (ch >> 1) & 1, lim);
        if (ch + 1 < T.nchunks) mbar_wait(&bars[(ch + 1) & 1], ((ch + 1) >> 1) & 1, lim);
      }
      __syncthreads();
      return;
    }
    const int bigw = T.chunk_big_w[ch];
    if (bigw > 0) {
      big_supernode<CB, UPPER>(T, T.chunk_big_f[ch], bigw, Xs);
      continue;
    }
    const int* hdr = reinterpret_cast<const int*>(B);
    if (hdr[0] > 0 && hdr[2] > 0) {
      chunk_phase_a<CB>(B, Xs);
      __syncthreads();
    }
    if (hdr[1] > 0) {
      const int wmax = hdr[6];
      if (wmax <= 4) chunk_phase_b_narrow<CB, UPPER>(B, Xs);
      else if (wmax <= 8) chunk_phase_b<CB, UPPER, 8>(B, Xs);
      else if (wmax <= 16) chunk_phase_b<CB, UPPER, 16>(B, Xs);
      else chunk_phase_b<CB, UPPER, 32>(B, Xs);
    }
    __syncthreads();
  }
  for (int t = tid; t < n * CB; t += nthr) {
    const int i = t / CB, c = t % CB;
    if (c0 + c < ncols) X[i * xr + (c0 + c) * xc] = Xs[t];
  }
}

size_t st_smem(int n, int cb, int cap) {
  return (((size_t)n * cb * sizeof(double) + 15) & ~size_t(15)) + 2 * (size_t)cap + 16;
}

template <int CB, bool UPPER>
cudaError_t launch_one(cudaStream_t s, const StDev& T, int n, double* X, long long xr, long long xc, int ncols,
                       int* st, long long spin_limit) {
  const size_t smem = st_smem(n, CB, T.cap);
  cudaError_t e = allow_max_smem((const void*)k_trsm_st<CB, UPPER>);
  if (e != cudaSuccess) return e;
  const int grid = (ncols + CB - 1) / CB;
  k_trsm_st<CB, UPPER><<<grid, TRSM_THREADS, smem, s>>>(T, n, X, xr, xc, ncols, st, spin_limit);
  note_launch();
  return cudaGetLastError();
}

__global__ void k_fill_stream(long long nslots, const long long* __restrict__ slot, const int* __restrict__ src,
                              const double* __restrict__ vals, const double* __restrict__ inv_diag, int unit,
                              double* __restrict__ stream) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= nslots) return;
  const int sidx = src[k];
  double v;
  if (sidx >= 0) v = vals[sidx];
  else if (sidx == -1 || unit) v = 1.0;
  else v = inv_diag[-2 - sidx];
  stream[slot[k]] = v;
}

}  // namespace

int trsm_st_max_cb(int n, int cap) {
  int dev = 0, lim = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  for (int cb : {4, 2, 1})
    if (st_smem(n, cb, cap) + 1024 <= (size_t)lim) return cb;
  return 0;
}

cudaError_t launch_trsm_st(cudaStream_t s, int cb, bool upper, const StDev& T, int n, double* X, long long xr,
                           long long xc, int ncols, int* st, long long spin_limit) {
  if (ncols <= 0 || T.nchunks <= 0) return cudaSuccess;
  switch (cb * 2 + (upper ? 1 : 0)) {
    case 2: return launch_one<1, false>(s, T, n, X, xr, xc, ncols, st, spin_limit);
    case 3: return launch_one<1, true>(s, T, n, X, xr, xc, ncols, st, spin_limit);
    case 4: return launch_one<2, false>(s, T, n, X, xr, xc, ncols, st, spin_limit);
    case 5: return launch_one<2, true>(s, T, n, X, xr, xc, ncols, st, spin_limit);
    case 8: return launch_one<4, false>(s, T, n, X, xr, xc, ncols, st, spin_limit);
    case 9: return launch_one<4, true>(s, T, n, X, xr, xc, ncols, st, spin_limit);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fill_stream(cudaStream_t s, long long nslots, const long long* slot, const int* src,
                               const double* vals, const double* inv_diag, int unit, unsigned char* stream) {
  if (nslots <= 0) return cudaSuccess;
  k_fill_stream<<<int((nslots + 255) / 256), 256, 0, s>>>(nslots, slot, src, vals, inv_diag, unit,
                                                           reinterpret_cast<double*>(stream));
  note_launch();
  return cudaGetLastError();
}

}  // namespace condipm

// ============================================================================
// Column-parallel variant: one warp lane per right-hand-side column, so every
// FP64 instruction carries 32 useful multiply-adds (on GB300 a warp-wide DFMA
// occupies the SM's FP64 pipe for the same time whatever its active mask).  A
// warp solves one supernode (<= 32 rows, one accumulator register per row) for
// its 32 columns; long rows first have their external part cut into segments
// summed by other warps.  The ksplit CTAs that share a 32-column block split
// each level between them and meet at a bounded counter barrier, so the launch
// is cooperative (every CTA resident).  X is row-major: element (i, c) at
// X[i*ld + c], ld a multiple of 32.
namespace condipm {
namespace {

constexpr int COLS_THREADS = 256;

__device__ __forceinline__ bool block_group_barrier(unsigned* ctr, unsigned target, long long limit, int* st) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(ctr, 1u);
    long long it = 0;
    while (atomicAdd(ctr, 0u) < target) {
      if (++it > limit) { atomicExch(&st[ST_TIMEOUT], 1); ok = 0; break; }
      __nanosleep(20);
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <bool UPPER, int WC>
__device__ __forceinline__ void sweep_supernode(const ColDev& S, int f, int w, const double* __restrict__ val,
                                                const double* __restrict__ inv_diag, double* X, long long ld,
                                                int c, bool on, const double* part) {
  double acc[WC];
#pragma unroll
  for (int si = 0; si < WC; ++si) {
    if (si < w) {
      const int r = f + si;
      double a = on ? X[r * ld + c] : 0.0;
      const int ns = S.row_nseg[r];
      if (ns > 0) {
        const int s0 = S.row_seg[r];
        for (int k = 0; k < ns; ++k) a -= part[(long long)(s0 + k) * 32];
      }
      acc[si] = a;
    }
  }
#pragma unroll
  for (int tt = 0; tt < WC; ++tt) {
    const int t = UPPER ? WC - 1 - tt : tt;
    if (t < w) {
      const int rt = f + t;
      if (inv_diag) acc[t] *= inv_diag[rt];
      if (on) X[rt * ld + c] = acc[t];
#pragma unroll
      for (int s2 = 0; s2 < WC; ++s2) {
        if (UPPER ? (s2 < t) : (s2 > t && s2 < w)) {
          const double l = UPPER ? val[S.int_beg[f + s2] + (t - s2 - 1)] : val[S.int_beg[f + s2] + t];
          acc[s2] = fma(-l, acc[t], acc[s2]);
        }
      }
    }
  }
}

template <bool UPPER>
__global__ void __launch_bounds__(COLS_THREADS) k_trsm_cols(ColDev S, const int* __restrict__ ci,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ inv_diag, double* X,
                                                            long long ld, int ncols, int ksplit, double* scratch,
                                                            unsigned* bar, int* st, long long spin_limit) {
  const int cb = blockIdx.x / ksplit, p = blockIdx.x % ksplit;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int c = cb * 32 + lane;
  const bool on = c < ncols;
  const int gw = p * nwarps + warp, W = ksplit * nwarps;
  double* part = scratch + (long long)cb * S.maxseg * 32 + lane;
  unsigned* ctr = bar + cb;
  unsigned nbar = 0;
  for (int lev = 0; lev < S.nlev; ++lev) {
    const int g0 = S.lvl_seg_ptr[lev], g1 = S.lvl_seg_ptr[lev + 1];
    if (g1 > g0) {
      // external entries: one segment (<= 32 entries) per warp; the segment's
      // indices and values are fetched once, one per lane, and broadcast
      for (int g = g0 + gw; g < g1; g += W) {
        const int q0 = S.seg_q0[g], len = S.seg_q1[g] - q0;
        const int myj = lane < len ? ci[q0 + lane] : 0;
        const double myv = lane < len ? val[q0 + lane] : 0.0;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll 4
        for (int k = 0; k < 32; k += 4) {
          if (k < len) {
            const int j0 = __shfl_sync(FULL, myj, k), j1 = __shfl_sync(FULL, myj, k + 1);
            const int j2 = __shfl_sync(FULL, myj, k + 2), j3 = __shfl_sync(FULL, myj, k + 3);
            const double v0 = __shfl_sync(FULL, myv, k), v1 = __shfl_sync(FULL, myv, k + 1);
            const double v2 = __shfl_sync(FULL, myv, k + 2), v3 = __shfl_sync(FULL, myv, k + 3);
            a0 = fma(v0, on ? X[j0 * ld + c] : 0.0, a0);
            if (k + 1 < len) a1 = fma(v1, on ? X[j1 * ld + c] : 0.0, a1);
            if (k + 2 < len) a2 = fma(v2, on ? X[j2 * ld + c] : 0.0, a2);
            if (k + 3 < len) a3 = fma(v3, on ? X[j3 * ld + c] : 0.0, a3);
          }
        }
        const double dot = (a0 + a1) + (a2 + a3);
        const int tr = S.seg_row[g];
        if (tr >= 0) {
          if (on) X[tr * ld + c] -= dot;
        } else {
          part[(long long)(-1 - tr) * 32] = dot;
        }
      }
      if (!block_group_barrier(ctr, ksplit * (++nbar), spin_limit, st)) return;
    }
    for (int s = S.lvl_ptr[lev] + gw; s < S.lvl_ptr[lev + 1]; s += W) {
      const int f = S.sn_first[s], w = S.sn_w[s];
      if (w <= 4) sweep_supernode<UPPER, 4>(S, f, w, val, inv_diag, X, ld, c, on, part);
      else if (w <= 8) sweep_supernode<UPPER, 8>(S, f, w, val, inv_diag, X, ld, c, on, part);
      else if (w <= 16) sweep_supernode<UPPER, 16>(S, f, w, val, inv_diag, X, ld, c, on, part);
      else sweep_supernode<UPPER, 32>(S, f, w, val, inv_diag, X, ld, c, on, part);
    }
    if (!block_group_barrier(ctr, ksplit * (++nbar), spin_limit, st)) return;
  }
}

}  // namespace

int trsm_cols_max_blocks() {
  int dev = 0, sms = 0, a = 0, b = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_trsm_cols<false>, COLS_THREADS, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trsm_cols<true>, COLS_THREADS, 0);
  return sms * std::min(a, b);
}

cudaError_t launch_trsm_cols(cudaStream_t s, bool upper, const ColDev& S, const int* ci, const double* val,
                             const double* inv_diag, double* X, long long ld, int ncols, int ksplit,
                             double* scratch, unsigned* bar, int* st, long long spin_limit) {
  if (ncols <= 0 || S.nlev <= 0) return cudaSuccess;
  const int ncb = (ncols + 31) / 32;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned) * ncb, s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&S, (void*)&ci, (void*)&val, (void*)&inv_diag, (void*)&X, (void*)&ld, (void*)&ncols,
                  (void*)&ksplit, (void*)&scratch, (void*)&bar, (void*)&st, (void*)&spin_limit};
  void* fn = upper ? (void*)k_trsm_cols<true> : (void*)k_trsm_cols<false>;
  note_launch();
  return cudaLaunchCooperativeKernel(fn, dim3(ncb * ksplit), dim3(COLS_THREADS), args, 0, s);
}

}  // namespace condipm

// ============================================================================
// Level-blocked variant with explicit inverses of the diagonal blocks.  The
// supernodes (split to at most 32 rows) of the column schedule keep their
// levels; after every refactorisation each block's dense inverse D_s is formed
// (k_diag_inv, one warp per supernode, one column of D per lane).  A level is
// then two fully parallel phases, with every row of the level given to some
// warp of the ksplit CTAs that share a 32-column block (one lane per column):
//   A. Y_r = X_r - sum_{external k} T_rk X_k      (dot product along the row)
//   B. X_r = sum_{j in s} D_s(r, j) Y_j            (the block's inverse)
// separated by a bounded counter barrier of the group.  Unlike a sweep of the
// dense triangle, no chain of dependent steps runs inside a supernode, and the
// rows of the widest blocks spread over many warps and SMs.
namespace condipm {
namespace {

constexpr int BLK_THREADS = 256;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// group barrier of the CTAs of one column block: arrive with a release, poll
// with acquire loads (bounded), as in block_group_barrier
__device__ __forceinline__ bool group_barrier(unsigned* ctr, unsigned target, long long limit, int* st) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(ctr, 1u);
    long long it = 0;
    while (ld_acquire_u32(ctr) < target) {
      if (++it > limit) { atomicExch(&st[ST_TIMEOUT], 1); ok = 0; break; }
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <bool UPPER, int WM>
__device__ __forceinline__ void diag_inv_w(double (*Ts)[33], int s, int c, const int* __restrict__ sn_first,
                                             const int* __restrict__ sn_w, const int* __restrict__ d_off,
                                             const int* __restrict__ int_beg, const double* __restrict__ val,
                                             const double* __restrict__ inv_diag, double* __restrict__ D) {
  const int f = sn_first[s], w = sn_w[s];
  // the block's strict triangle goes to shared memory first, all loads in
  // flight together (lane c loads entry c of every row), so the substitution
  // below waits on no global load
  const int ib = c < w ? int_beg[f + c] : 0;   // lane r: where row r's entries start
#pragma unroll
  for (int r = 0; r < WM; ++r) {
    const int ibr = __shfl_sync(0xffffffffu, ib, r);
    if (r < w) {
      if (!UPPER) {
        if (c < r) Ts[r][c] = val[ibr + c];
      } else {
        if (c > r && c < w) Ts[r][c] = val[ibr + c - r - 1];
      }
    }
  }
  const double idg = (inv_diag && c < w) ? inv_diag[f + c] : 1.0;
  __syncwarp();
  double d[WM];
#pragma unroll
  for (int r = 0; r < WM; ++r) d[r] = 0.0;
  // row r of the inverse needs the rows before it (after it, for UPPER): a
  // dependent chain; each row's sum is split over four accumulators (by j mod
  // 4), so the chain of a 32-wide block is about a quarter as long
  if (!UPPER) {
#pragma unroll
    for (int r = 0; r < WM; ++r) {
      if (r < w) {
        double a[4] = {(r == c) ? 1.0 : 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < WM; ++j)
          if (j < r) a[j & 3] = fma(-Ts[r][j], d[j], a[j & 3]);
        const double acc = (a[0] + a[1]) + (a[2] + a[3]);
        d[r] = inv_diag ? acc * __shfl_sync(0xffffffffu, idg, r) : acc;
      }
    }
  } else {
#pragma unroll
    for (int rr = 0; rr < WM; ++rr) {
      const int r = WM - 1 - rr;
      if (r < w) {
        double a[4] = {(r == c) ? 1.0 : 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int j = 0; j < WM; ++j)
          if (j > r && j < w) a[j & 3] = fma(-Ts[r][j], d[j], a[j & 3]);
        const double acc = (a[0] + a[1]) + (a[2] + a[3]);
        d[r] = inv_diag ? acc * __shfl_sync(0xffffffffu, idg, r) : acc;
      }
    }
  }
  if (c < w) {
    double* Ds = D + d_off[s];
#pragma unroll
    for (int r = 0; r < WM; ++r)
      if (r < w) Ds[r * w + c] = d[r];
  }
}

// the inverse of supernode s's diagonal block, its loops unrolled to the
// smallest of 4, 8, 32 that covers the block's width (most blocks are narrow)
template <bool UPPER>
__device__ __forceinline__ void diag_inv_one(double (*Ts)[33], int s, int c, const int* __restrict__ sn_first,
                                             const int* __restrict__ sn_w, const int* __restrict__ d_off,
                                             const int* __restrict__ int_beg, const double* __restrict__ val,
                                             const double* __restrict__ inv_diag, double* __restrict__ D) {
  const int w = sn_w[s];
  if (w <= 4) diag_inv_w<UPPER, 4>(Ts, s, c, sn_first, sn_w, d_off, int_beg, val, inv_diag, D);
  else if (w <= 8) diag_inv_w<UPPER, 8>(Ts, s, c, sn_first, sn_w, d_off, int_beg, val, inv_diag, D);
  else diag_inv_w<UPPER, 32>(Ts, s, c, sn_first, sn_w, d_off, int_beg, val, inv_diag, D);
}

// the four factors' diagonal-block inverses in one launch (blockIdx.y picks
// the factor), so that their widest blocks are inverted side by side
__global__ void k_diag_inv4(DiagInvJob j0, DiagInvJob j1, DiagInvJob j2, DiagInvJob j3) {
  __shared__ double Tsh[4][32][33];   // one block per warp (128 threads)
  const DiagInvJob J = blockIdx.y == 0 ? j0 : blockIdx.y == 1 ? j1 : blockIdx.y == 2 ? j2 : j3;
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int c = threadIdx.x & 31;
  if (s >= J.nsn) return;
  double (*Ts)[33] = Tsh[(threadIdx.x >> 5) & 3];
  if (J.upper) diag_inv_one<true>(Ts, s, c, J.sn_first, J.sn_w, J.d_off, J.int_beg, J.val, J.inv_diag, J.D);
  else diag_inv_one<false>(Ts, s, c, J.sn_first, J.sn_w, J.d_off, J.int_beg, J.val, J.inv_diag, J.D);
}

// The factor epilogue of every instance of a batch: the gathers of L, U^T, U,
// L^T out of LU and the staged-solve byte streams (read through the same maps)
__global__ void k_b_gather(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff) {
  const int i = batch_instance(boff, n, blockIdx.x);
  const BatchInst& B = I[i];
  if (!B.active) return;
  const long long lt = (long long)(blockIdx.x - boff[i]) * blockDim.x + threadIdx.x;
  const long long ls = (long long)(boff[i + 1] - boff[i]) * blockDim.x;
  for (long long q = lt; q < B.nnzLo; q += ls) {
    B.Lo_val[q] = B.LUval[B.Lo_map[q]];
    B.Ut_val[q] = B.LUval[B.Ut_map[q]];
  }
  for (long long q = lt; q < B.nnzUp; q += ls) {
    B.Up_val[q] = B.LUval[B.Up_map[q]];
    B.Lt_val[q] = B.LUval[B.Lt_map[q]];
  }
  // streams: lower pattern a = L (unit), b = U^T; upper pattern a = U, b = L^T (unit)
  for (int k = 0; k < 2; ++k) {
    const int* ma = k ? B.Up_map : B.Lo_map;
    const int* mb = k ? B.Lt_map : B.Ut_map;
    for (long long q = lt; q < B.st_nslots[k]; q += ls) {
      const int sidx = B.st_src[k][q];
      double va, vb;
      if (sidx >= 0) {
        va = B.LUval[ma[sidx]];
        vb = B.LUval[mb[sidx]];
      } else if (sidx == -1) {
        va = vb = 1.0;
      } else {
        const double d = B.inv_diag[-2 - sidx];
        va = k ? d : 1.0;
        vb = k ? 1.0 : d;
      }
      B.st_a[k][B.st_slot[k][q]] = va;
      B.st_b[k][B.st_slot[k][q]] = vb;
    }
  }
}

// diagonal-block inverses of the four factors of every instance: one warp per
// (factor, supernode), the blocks boff[i] .. boff[i + 1] serving instance i
__global__ void __launch_bounds__(128, 4) k_b_diag_inv(const BatchInst* __restrict__ I, int n, const int* __restrict__ boff) {
  __shared__ double Tsh[4][32][33];
  const int i = batch_instance(boff, n, blockIdx.x);
  const BatchInst& B = I[i];
  if (!B.active) return;
  const int c = threadIdx.x & 31;
  double (*Ts)[33] = Tsh[(threadIdx.x >> 5) & 3];
  const int nl = B.dj[0].nsn, nuu = B.dj[2].nsn;
  const int nw = (boff[i + 1] - boff[i]) * (blockDim.x >> 5);
  for (int t = ((blockIdx.x - boff[i]) * blockDim.x + threadIdx.x) >> 5; t < 2 * (nl + nuu); t += nw) {
    const int j = t < nl ? 0 : t < 2 * nl ? 1 : t < 2 * nl + nuu ? 2 : 3;
    const int sn = j < 2 ? t - j * nl : t - 2 * nl - (j - 2) * nuu;
    const DiagInvJob& J = B.dj[j];
    if (J.upper) diag_inv_one<true>(Ts, sn, c, J.sn_first, J.sn_w, J.d_off, J.int_beg, J.val, J.inv_diag, J.D);
    else diag_inv_one<false>(Ts, sn, c, J.sn_first, J.sn_w, J.d_off, J.int_beg, J.val, J.inv_diag, J.D);
    __syncwarp();
  }
}

// The level-blocked solve of one 32-column block (columns cb * 32 ..), by the
// ksplit CTAs of its group (this one is p); sync() separates the phases (a
// bounded group barrier, or __syncthreads when one CTA has the block).
// rch_cb0 >= 0: the block is block rch_cb0 + cb of P G_u's columns, and when
// that block has a reach list only the listed rows are solved (the others are
// zero in X and stay so) and the levels without any are passed by (every CTA
// of the group reads the same list, so all of them skip the same barriers).
// Returns false when a barrier wait expired.
template <class Sync>
__device__ __forceinline__ bool blk_solve(const BlkDev& S, const int* __restrict__ ci, const double* __restrict__ val,
                                          const double* __restrict__ D, double* X, double* Y, long long ld,
                                          int ncols, int cb, int p, int ksplit, Sync&& sync, int rch_cb0 = -1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int c = cb * 32 + lane;
  const bool on = c < ncols;
  const int gw = p * nwarps + warp, W = ksplit * nwarps;
  const int rb = rch_cb0 >= 0 && S.rch_ptr ? rch_cb0 + cb : -1;
  const int* __restrict__ rp = rb >= 0 && rb < S.rch_nblk ? S.rch_ptr + (size_t)rb * (S.nlev + 1) : nullptr;
  for (int lev = 0; lev < S.nlev; ++lev) {
    const int q0 = rp ? rp[lev] : S.lvl_rptr[lev], q1 = rp ? rp[lev + 1] : S.lvl_rptr[lev + 1];
    if (q0 == q1) continue;
    // A: Y_r = X_r - external part of row r
    for (int k = q0 + gw; k < q1; k += W) {
      const int q = rp ? S.rch_q[k] : k;
      const int r = S.rows[q];
      const int e0 = S.ext_beg[r], e1 = S.ext_end[r];
      double a0 = on ? X[(long long)r * ld + c] : 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      // 32 entries at a time: one coalesced load of their columns and values,
      // broadcast by shuffles, so the X loads do not wait on index loads
      for (int eb = e0; eb < e1; eb += 32) {
        const int len = min(32, e1 - eb);
        const int myj = lane < len ? ci[eb + lane] : 0;
        const double myv = lane < len ? val[eb + lane] : 0.0;
        int k = 0;
        for (; k + 3 < len; k += 4) {
          const int j0 = __shfl_sync(FULL, myj, k), j1 = __shfl_sync(FULL, myj, k + 1);
          const int j2 = __shfl_sync(FULL, myj, k + 2), j3 = __shfl_sync(FULL, myj, k + 3);
          const double v0 = __shfl_sync(FULL, myv, k), v1 = __shfl_sync(FULL, myv, k + 1);
          const double v2 = __shfl_sync(FULL, myv, k + 2), v3 = __shfl_sync(FULL, myv, k + 3);
          if (on) {
            a0 = fma(-v0, X[(long long)j0 * ld + c], a0);
            a1 = fma(-v1, X[(long long)j1 * ld + c], a1);
            a2 = fma(-v2, X[(long long)j2 * ld + c], a2);
            a3 = fma(-v3, X[(long long)j3 * ld + c], a3);
          }
        }
        for (; k < len; ++k) {
          const int j = __shfl_sync(FULL, myj, k);
          const double v = __shfl_sync(FULL, myv, k);
          if (on) a0 = fma(-v, X[(long long)j * ld + c], a0);
        }
      }
      if (on) Y[(long long)r * ld + c] = (a0 + a1) + (a2 + a3);
    }
    if (!sync()) return false;
    // B: X_r = D_s(r, :) Y_s over the nonzero half of the triangular D_s row
    for (int k = q0 + gw; k < q1; k += W) {
      const int q = rp ? S.rch_q[k] : k;
      const int r = S.rows[q], s = S.row_sn[q];
      const int f = S.sn_first[s], w = S.sn_w[s];
      const double* Dr = D + S.d_off[s] + (r - f) * w;
      const int jb = S.upper ? r - f : 0, je = S.upper ? w : r - f + 1;
      double a0 = 0.0, a1 = 0.0;
      int j = jb;
      if (on) {
        for (; j + 1 < je; j += 2) {
          a0 = fma(Dr[j], Y[(long long)(f + j) * ld + c], a0);
          a1 = fma(Dr[j + 1], Y[(long long)(f + j + 1) * ld + c], a1);
        }
        if (j < je) a0 = fma(Dr[j], Y[(long long)(f + j) * ld + c], a0);
        X[(long long)r * ld + c] = a0 + a1;
      }
    }
    if (!sync()) return false;
  }
  return true;
}

// MINB: CTAs per SM the register allocation must allow (5: 48 registers, no
// spills; 6 and 8 trade a few spilled registers for more resident warps); the
// autotuner times each
template <int MINB>
__global__ void __launch_bounds__(BLK_THREADS, MINB) k_trsm_blk(BlkDev S, const int* __restrict__ ci,
                                                                const double* __restrict__ val,
                                                                const double* __restrict__ D, double* X, double* Y,
                                                                long long ld, int ncols, int ksplit, unsigned* bar,
                                                                int* st, long long spin_limit, int rch_cb0) {
  const int cb = blockIdx.x / ksplit, p = blockIdx.x % ksplit;
  unsigned* ctr = bar + cb;
  unsigned nbar = 0;
  blk_solve(S, ci, val, D, X, Y, ld, ncols, cb, p, ksplit,
            [&]() { return group_barrier(ctr, ksplit * (++nbar), spin_limit, st); }, rch_cb0);
}


// The level-blocked solve (both triangles) with one thread-block cluster per
// 32-column block:
// the cluster's CTAs share out a level's rows and meet at the hardware cluster
// barrier between the phases (in place of k_trsm_blk's bounded group barrier
// through global memory); the hardware co-schedules a cluster, so no wait can
// be left without its partner.
__global__ void __launch_bounds__(BLK_THREADS) k_trsm_blkc(BlkDev SL, const int* __restrict__ ciL,
                                                           const double* __restrict__ valL,
                                                           const double* __restrict__ DL, BlkDev SU,
                                                           const int* __restrict__ ciU,
                                                           const double* __restrict__ valU,
                                                           const double* __restrict__ DU, double* X, double* Y,
                                                           long long ld, int ncols, int rch_cb0) {
  cg::cluster_group cl = cg::this_cluster();
  const int cb = blockIdx.x / cl.num_blocks();
  auto sync = [&]() {
    cl.sync();
    return true;
  };
  blk_solve(SL, ciL, valL, DL, X, Y, ld, ncols, cb, (int)cl.block_rank(), (int)cl.num_blocks(), sync, rch_cb0);
  blk_solve(SU, ciU, valU, DU, X, Y, ld, ncols, cb, (int)cl.block_rank(), (int)cl.num_blocks(), sync);
}

// Both triangles of a multi-RHS solve for every instance of a batch: one
// thread-block cluster per (instance, 32-column block) item, its CTAs sharing
// out a level's rows and the cluster barrier between the phases (the hardware
// co-schedules a cluster's CTAs, so the barrier always completes and any
// number of items can be launched).  trans = 0: S_x <- U^{-1} L^{-1} S_x;
// trans = 1: the x rows of H <- L^{-T} U^{-T} H_x.
__global__ void __launch_bounds__(BLK_THREADS) k_b_trsm(const BatchInst* __restrict__ I, const int2* __restrict__ cbs,
                                                        int trans) {
  cg::cluster_group cl = cg::this_cluster();
  const int2 it = cbs[blockIdx.x / cl.num_blocks()];
  const BatchInst& B = I[it.x];
  if (!B.active) return;   // the whole cluster leaves together, before any barrier
  double* X = (trans ? B.H : B.Zt) + (size_t)B.nu * B.ld;
  const int p = (int)cl.block_rank(), ks = (int)cl.num_blocks();
  auto bar = [&]() {
    cl.sync();
    return true;
  };
  blk_solve(B.bkL, B.Lo_ci, trans ? B.Ut_val : B.Lo_val, trans ? B.D_Ut : B.D_L, X, B.Y, B.ld, B.nu, it.y, p, ks, bar);
  blk_solve(B.bkU, B.Up_ci, trans ? B.Lt_val : B.Up_val, trans ? B.D_Lt : B.D_U, X, B.Y, B.ld, B.nu, it.y, p, ks, bar);
}

// One right-hand side (the Newton-step recovery): the same two phases, with a
// row's entries spread over G lanes (32 / G rows per warp) and a shuffle
// reduction, so the FP64 instructions stay packed without 32 columns.
template <int G>
__global__ void __launch_bounds__(BLK_THREADS) k_trsm_blk1(BlkDev S, const int* __restrict__ ci,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ D, double* X, double* Y,
                                                           long long xs, unsigned* bar, int* st,
                                                           long long spin_limit) {
  constexpr int RPW = 32 / G;   // rows per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int sub = lane / G, gl = lane % G;
  const int gw = blockIdx.x * nwarps + warp, W = gridDim.x * nwarps;
  unsigned nbar = 0;
  for (int lev = 0; lev < S.nlev; ++lev) {
    const int q0 = S.lvl_rptr[lev], q1 = S.lvl_rptr[lev + 1];
    // A: Y_r = X_r - external part of row r
    for (int qb = q0 + gw * RPW; qb < q1; qb += W * RPW) {
      const int q = qb + sub;
      double a = 0.0;
      int r = 0;
      if (q < q1) {
        r = S.rows[q];
        const int e1 = S.ext_end[r];
        for (int e = S.ext_beg[r] + gl; e < e1; e += G) a = fma(val[e], X[(long long)ci[e] * xs], a);
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
      if (q < q1 && gl == 0) Y[(long long)r * xs] = X[(long long)r * xs] - a;
    }
    if (!group_barrier(bar, gridDim.x * (++nbar), spin_limit, st)) return;
    // B: X_r = D_s(r, :) Y_s
    for (int qb = q0 + gw * RPW; qb < q1; qb += W * RPW) {
      const int q = qb + sub;
      double a = 0.0;
      int r = 0;
      if (q < q1) {
        r = S.rows[q];
        const int s = S.row_sn[q], f = S.sn_first[s], w = S.sn_w[s];
        const double* Dr = D + S.d_off[s] + (r - f) * w;
        const int jb = S.upper ? r - f : 0, je = S.upper ? w : r - f + 1;   // nonzero half of the row
        for (int j = jb + gl; j < je; j += G) a = fma(Dr[j], Y[(long long)(f + j) * xs], a);
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
      if (q < q1 && gl == 0) X[(long long)r * xs] = a;
    }
    if (!group_barrier(bar, gridDim.x * (++nbar), spin_limit, st)) return;
  }
}

// One right-hand side in one CTA: the whole vector lives in shared memory (xv)
// together with the current level's Y (yv, indexed by the row's position in
// the level, where a supernode's rows are consecutive), so every gather of X
// and Y is a shared-memory access and the levels are separated by
// __syncthreads alone, with no grid-wide barrier.  Same two phases per level as
// the multi-CTA form (external part with G lanes per row, then the dense
// inverse of the supernode's diagonal block).  Each row's description is one
// int4 per phase (MA: row, external entries; MB: row, offset in its supernode,
// width, offset of its row of D), and a thread's descriptions for the next
// level, and its D entries for this level, are loaded ahead of the barriers, so
// a level waits on global memory about once instead of three times per phase.
template <int G>
__device__ __forceinline__ void lu1s_tri(int nlev, const int* __restrict__ lvl_rptr, const int4* __restrict__ MA,
                                         const int4* __restrict__ MB, const int* __restrict__ ci,
                                         const double* __restrict__ val, const double* __restrict__ D, double* xv,
                                         double* yv) {
  constexpr int RPW = 32 / G;   // rows per warp
  constexpr int ND = 32 / G;    // D entries per lane (supernodes are at most 32 wide)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int sub = lane / G, gl = lane % G;
  const int slot = warp * RPW + sub, nslot = nwarps * RPW;
  const int4 z4 = make_int4(0, 0, 0, 0);
  int4 ma = z4, mb = z4;
  if (nlev > 0 && lvl_rptr[0] + slot < lvl_rptr[1]) { ma = MA[lvl_rptr[0] + slot]; mb = MB[lvl_rptr[0] + slot]; }
  for (int lev = 0; lev < nlev; ++lev) {
    const int q0 = lvl_rptr[lev], q1 = lvl_rptr[lev + 1];
    const bool first_on = q0 + slot < q1;
    // D row of this thread's first-pass row, for phase B
    double dreg[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      const int j = gl + k * G;
      dreg[k] = (first_on && j < mb.z) ? D[mb.w + j] : 0.0;
    }
    // the next level's descriptions of this thread's first-pass row
    int4 na = z4, nb = z4;
    if (lev + 1 < nlev && q1 + slot < lvl_rptr[lev + 2]) { na = MA[q1 + slot]; nb = MB[q1 + slot]; }
    // A: Y_r = X_r - external part of row r
    for (int qb = q0 + warp * RPW, pass = 0; qb < q1; qb += nslot, ++pass) {
      const int q = qb + sub;
      double a0 = 0.0, a1 = 0.0;
      int r = 0;
      if (q < q1) {
        const int4 m = pass == 0 ? ma : MA[q];
        r = m.x;
        int e = m.y + gl;
        for (; e + G < m.z; e += 2 * G) {
          a0 = fma(val[e], xv[ci[e]], a0);
          a1 = fma(val[e + G], xv[ci[e + G]], a1);
        }
        if (e < m.z) a0 = fma(val[e], xv[ci[e]], a0);
      }
      double a = a0 + a1;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
      if (q < q1 && gl == 0) yv[q - q0] = xv[r] - a;
    }
    __syncthreads();
    // B: X_r = D_s(r, :) Y_s
    for (int qb = q0 + warp * RPW, pass = 0; qb < q1; qb += nslot, ++pass) {
      const int q = qb + sub;
      double a = 0.0;
      int r = 0;
      if (q < q1) {
        if (pass == 0) {
          r = mb.x;
          const double* Ys = yv + (q - q0 - mb.y);   // Y of the supernode's first row
#pragma unroll
          for (int k = 0; k < ND; ++k) {
            const int j = gl + k * G;
            if (j < mb.z) a = fma(dreg[k], Ys[j], a);
          }
        } else {
          const int4 m = MB[q];
          r = m.x;
          const double* Ys = yv + (q - q0 - m.y);
          for (int j = gl; j < m.z; j += G) a = fma(D[m.w + j], Ys[j], a);
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
      if (q < q1 && gl == 0) xv[r] = a;
    }
    __syncthreads();
    ma = na;
    mb = nb;
  }
}

template <int G>
__global__ void __launch_bounds__(1024) k_trsm_lu1s(Lu1sDev L, const int* __restrict__ ciL,
                                                    const double* __restrict__ valL, const double* __restrict__ DL,
                                                    Lu1sDev U, const int* __restrict__ ciU,
                                                    const double* __restrict__ valU, const double* __restrict__ DU,
                                                    double* X, long long xs, int n) {
  extern __shared__ double sm1[];
  double* xv = sm1;       // n
  double* yv = sm1 + n;   // the largest level
  for (int i = threadIdx.x; i < n; i += blockDim.x) xv[i] = X[(long long)i * xs];
  __syncthreads();
  lu1s_tri<G>(L.nlev, L.lvl_rptr, L.ma, L.mb, ciL, valL, DL, xv, yv);
  lu1s_tri<G>(U.nlev, U.lvl_rptr, U.ma, U.mb, ciU, valU, DU, xv, yv);
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long long)i * xs] = xv[i];
}

// One right-hand side on a thread-block cluster of CL CTAs: every CTA keeps a
// full copy of the vector in its shared memory, so every gather is a local
// shared-memory access.  The supernodes of each level are shared out over the
// CTAs; a CTA computes Y for the rows of its supernodes (phase A, external
// parts), then X_r = D_s(r, :) Y_s (phase B), writing X_r into every CTA's copy
// (distributed shared memory stores) before the cluster barrier that ends the
// level.  A level's FP64 work spreads over CL SMs and costs one CTA barrier and
// one hardware cluster barrier; a thread's first row of the next level is
// described, its first two external entries and its D row fetched, ahead of
// the barriers.
template <int G>
__device__ __forceinline__ void lu1c_tri(const Cl1Dev& S, int p, int CL, const int* __restrict__ ci,
                                         const double* __restrict__ val, const double* __restrict__ D,
                                         double* xv, double* yv, double* const* rx, int* lv) {
  constexpr int RPW = 32 / G;
  constexpr int ND = 32 / G;   // D entries per lane (supernodes are at most 32 wide)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int sub = lane / G, gl = lane % G;
  const int slot = warp * RPW + sub, nslot = nwarps * RPW;
  const int L1 = S.nlev + 1;
  // this CTA's level boundaries, staged in shared memory (lv: nlev + 1 ints)
  int* tp = lv;
  for (int i = threadIdx.x; i < L1; i += blockDim.x) tp[i] = S.t_ptr[p * L1 + i];
  __syncthreads();
  const int4 z4 = make_int4(0, 0, 0, 0);
  cg::cluster_group cl = cg::this_cluster();
  int4 ma = z4, mb = z4;
  int pc0 = 0, pc1 = 0;   // ... and its first two external entries
  double pv0 = 0.0, pv1 = 0.0;
  if (S.nlev > 0 && tp[0] + slot < tp[1]) {
    ma = S.ta[tp[0] + slot];
    mb = S.tb[tp[0] + slot];
    const int e0 = ma.y + gl, e1 = e0 + G;
    if (e0 < ma.z) { pc0 = ci[e0]; pv0 = val[e0]; }
    if (e1 < ma.z) { pc1 = ci[e1]; pv1 = val[e1]; }
  }
  for (int lev = 0; lev < S.nlev; ++lev) {
    const int t0 = tp[lev], t1 = tp[lev + 1];
    double dreg[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      const int j = gl + k * G;
      dreg[k] = (t0 + slot < t1 && j < mb.z) ? D[mb.w + j] : 0.0;
    }
    int4 na = z4, nb = z4;
    if (lev + 1 < S.nlev && t1 + slot < tp[lev + 2]) {
      na = S.ta[t1 + slot];
      nb = S.tb[t1 + slot];
    }
    // A: Y_r = X_r - external part of row r, G lanes per row
    for (int tb = t0 + warp * RPW, pass = 0; tb < t1; tb += nslot, ++pass) {
      const int t = tb + sub;
      double s0 = 0.0, s1 = 0.0;
      int4 m = z4;
      if (t < t1) {
        m = pass == 0 ? ma : S.ta[t];
        int e = m.y + gl;
        if (pass == 0) {
          if (e < m.z) s0 = pv0 * xv[pc0];
          if (e + G < m.z) s1 = pv1 * xv[pc1];
          e += 2 * G;
        }
        for (; e + G < m.z; e += 2 * G) {
          s0 = fma(val[e], xv[ci[e]], s0);
          s1 = fma(val[e + G], xv[ci[e + G]], s1);
        }
        if (e < m.z) s0 = fma(val[e], xv[ci[e]], s0);
      }
      double a = s0 + s1;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
      if (t < t1 && gl == 0) yv[m.w] = xv[m.x] - a;
    }
    __syncthreads();
    // the next level's first two external entries of this thread's first row
    pc0 = pc1 = 0;
    pv0 = pv1 = 0.0;
    {
      const int e0 = na.y + gl, e1 = e0 + G;
      if (e0 < na.z) { pc0 = ci[e0]; pv0 = val[e0]; }
      if (e1 < na.z) { pc1 = ci[e1]; pv1 = val[e1]; }
    }
    // B: X_r = D_s(r, :) Y_s, written into every CTA's copy
    for (int tb = t0 + warp * RPW, pass = 0; tb < t1; tb += nslot, ++pass) {
      const int t = tb + sub;
      double a = 0.0;
      int r = 0;
      if (t < t1) {
        if (pass == 0) {
          r = mb.x;
#pragma unroll
          for (int k = 0; k < ND; ++k) {
            const int j = gl + k * G;
            if (j < mb.z) a = fma(dreg[k], yv[mb.y + j], a);
          }
        } else {
          const int4 m = S.tb[t];
          r = m.x;
          const double* Dr = D + m.w;
          for (int j = gl; j < m.z; j += G) a = fma(Dr[j], yv[m.y + j], a);
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
      if (t < t1)
        for (int q = gl; q < CL; q += G) rx[q][r] = a;
    }
    cl.sync();   // every X of the level is in every copy
    ma = na;
    mb = nb;
  }
}

constexpr int LU1C_THREADS = 1024;

template <int G>
__global__ void __launch_bounds__(LU1C_THREADS, 1) k_trsm_lu1c(Cl1Dev L, const int* __restrict__ ciL,
                                                               const double* __restrict__ valL,
                                                               const double* __restrict__ DL, Cl1Dev U,
                                                               const int* __restrict__ ciU,
                                                               const double* __restrict__ valU,
                                                               const double* __restrict__ DU, double* X,
                                                               long long xs, int n) {
  extern __shared__ double smc[];
  __shared__ double* rx[16];
  cg::cluster_group cl = cg::this_cluster();
  const int p = int(cl.block_rank()), CL = int(cl.num_blocks());
  double* xv = smc;       // n: this CTA's copy of the vector
  double* yv = smc + n;   // Y of the rows of the supernodes this CTA owns in the current level
  int* lv = reinterpret_cast<int*>(yv + max(L.ymax, U.ymax));   // level boundaries of one triangle
  if (threadIdx.x < CL) rx[threadIdx.x] = cl.map_shared_rank(xv, threadIdx.x);
  for (int i = threadIdx.x; i < n; i += blockDim.x) xv[i] = X[(long long)i * xs];
  cl.sync();   // every copy is loaded before any CTA writes into another's
  lu1c_tri<G>(L, p, CL, ciL, valL, DL, xv, yv, rx, lv);
  lu1c_tri<G>(U, p, CL, ciU, valU, DU, xv, yv, rx, lv);
  if (p == 0)
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long long)i * xs] = xv[i];
}

}  // namespace

int trsm_lu1c_max_clusters(int CL, int n, int ymax, int nlev) {
  const size_t smem = sizeof(double) * ((size_t)n + (size_t)ymax) + sizeof(int) * ((size_t)nlev + 1);
  if (allow_max_smem((const void*)k_trsm_lu1c<8>) != cudaSuccess) return 0;
  if (CL > 8 && allow_cluster16((const void*)k_trsm_lu1c<8>) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(LU1C_THREADS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  if (cudaOccupancyMaxActiveClusters(&ncl, (const void*)k_trsm_lu1c<8>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return ncl;
}

cudaError_t launch_trsm_lu1c(cudaStream_t s, const Cl1Dev& L, const int* ciL, const double* valL,
                             const double* DL, const Cl1Dev& U, const int* ciU, const double* valU,
                             const double* DU, double* X, long long xs, int n) {
  const int CL = L.CL;
  const size_t smem = sizeof(double) * ((size_t)n + (size_t)std::max(L.ymax, U.ymax)) +
                      sizeof(int) * ((size_t)std::max(L.nlev, U.nlev) + 1);
  cudaError_t e = allow_max_smem((const void*)k_trsm_lu1c<8>);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = allow_cluster16((const void*)k_trsm_lu1c<8>);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(LU1C_THREADS);
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
  return cudaLaunchKernelEx(&cfg, k_trsm_lu1c<8>, L, ciL, valL, DL, U, ciU, valU, DU, X, xs, n);
}

size_t trsm_lu1s_max_smem() {
  int dev = 0, mx = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, (const void*)k_trsm_lu1s<8>);
  return mx > int(fa.sharedSizeBytes) ? size_t(mx) - fa.sharedSizeBytes : 0;
}

cudaError_t launch_trsm_lu1s(cudaStream_t s, int g, const Lu1sDev& L, const int* ciL, const double* valL,
                             const double* DL, const Lu1sDev& U, const int* ciU, const double* valU,
                             const double* DU, double* X, long long xs, int n, int ymax) {
  const size_t smem = sizeof(double) * ((size_t)n + (size_t)ymax);
  const void* fn = g == 4 ? (const void*)k_trsm_lu1s<4> : (const void*)k_trsm_lu1s<8>;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_smem(fn);
    if (e != cudaSuccess) return e;
  }
  if (g == 4) k_trsm_lu1s<4><<<1, 1024, smem, s>>>(L, ciL, valL, DL, U, ciU, valU, DU, X, xs, n);
  else k_trsm_lu1s<8><<<1, 1024, smem, s>>>(L, ciL, valL, DL, U, ciU, valU, DU, X, xs, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_trsm_blk1(cudaStream_t s, const BlkDev& S, const int* ci, const double* val, const double* D,
                             double* X, double* Y, long long xs, int nblocks, unsigned* bar, int* st,
                             long long spin_limit) {
  if (S.nlev <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&S, (void*)&ci, (void*)&val, (void*)&D, (void*)&X, (void*)&Y, (void*)&xs,
                  (void*)&bar, (void*)&st, (void*)&spin_limit};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)k_trsm_blk1<8>, dim3(nblocks), dim3(BLK_THREADS), args, 0, s);
}

cudaError_t launch_diag_inv4(cudaStream_t s, const DiagInvJob* jobs) {
  int nmax = 0;
  for (int k = 0; k < 4; ++k) nmax = std::max(nmax, jobs[k].nsn);
  if (nmax <= 0) return cudaSuccess;
  const int threads = 128;
  const dim3 grid((nmax * 32 + threads - 1) / threads, 4);
  k_diag_inv4<<<grid, threads, 0, s>>>(jobs[0], jobs[1], jobs[2], jobs[3]);
  note_launch();
  return cudaGetLastError();
}

static const void* trsm_blk_fn(int minb) {
  return minb >= 8 ? (const void*)k_trsm_blk<8> : minb >= 6 ? (const void*)k_trsm_blk<6> : (const void*)k_trsm_blk<5>;
}
int trsm_blk_max_blocks(int minb) {
  int a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, trsm_blk_fn(minb), BLK_THREADS, 0);
  return device_sms() * std::max(a, 1);
}

static cudaLaunchConfig_t trsm_cluster_config(int nclusters, int cl, cudaStream_t s, cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(nclusters * cl);
  cfg.blockDim = dim3(BLK_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t launch_trsm_blkc(cudaStream_t s, const BlkDev& SL, const int* ciL, const double* valL,
                             const double* DL, const BlkDev& SU, const int* ciU, const double* valU,
                             const double* DU, double* X, double* Y, long long ld, int ncols, int cl,
                             int rch_cb0) {
  if (ncols <= 0) return cudaSuccess;
  if (cl > 8) {
    cudaError_t e = allow_cluster16((const void*)k_trsm_blkc);
    if (e != cudaSuccess) return e;
  }
  const int ncb = (ncols + 31) / 32;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = trsm_cluster_config(ncb, cl, s, at);
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_trsm_blkc, SL, ciL, valL, DL, SU, ciU, valU, DU, X, Y, ld, ncols, rch_cb0);
}

int trsm_blkc_clusters(int cl) {
  if (cl > 8 && allow_cluster16((const void*)k_trsm_blkc) != cudaSuccess) return 0;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = trsm_cluster_config(1, cl, nullptr, at);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, (const void*)k_trsm_blkc, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

cudaError_t launch_trsm_blk(cudaStream_t s, const BlkDev& S, const int* ci, const double* val, const double* D,
                            double* X, double* Y, long long ld, int ncols, int ksplit, unsigned* bar, int* st,
                            long long spin_limit, int minb, int rch_cb0) {
  if (ncols <= 0 || S.nlev <= 0) return cudaSuccess;
  const int ncb = (ncols + 31) / 32;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(unsigned) * ncb, s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&S, (void*)&ci, (void*)&val, (void*)&D, (void*)&X, (void*)&Y, (void*)&ld,
                  (void*)&ncols, (void*)&ksplit, (void*)&bar, (void*)&st, (void*)&spin_limit, (void*)&rch_cb0};
  note_launch();
  return cudaLaunchCooperativeKernel(trsm_blk_fn(minb), dim3(ncb * ksplit), dim3(BLK_THREADS), args, 0, s);
}

}  // namespace condipm

// ============================================================================
// Dataflow variant of the level-blocked solve: no barrier at all.  Every row
// of the solve is two warp tasks, in level order:
//   A(r): wait until every supernode that r's external entries lie in is
//         complete, then Y_r = X_r - external part, and count r into its
//         supernode's A counter;
//   B(r): wait until all rows of r's supernode have passed A, then
//         X_r = D_s(r, :) Y_s and count r into the supernode's B counter
//         (the supernode is complete when it reaches its width).
// Tasks go round-robin to the warps of the ksplit CTAs that share a 32-column
// block (one lane per column); each warp runs its tasks in list order, every
// wait of a task is on tasks earlier in the list, and all warps are resident
// (cooperative launch), so the waits always end.  Compared with the level
// barriers, a row waits only for the supernodes it reads, not for the slowest
// row of the level, and separate branches of the elimination tree proceed
// independently.
namespace condipm {
namespace {

// add with release semantics at GPU scope: the warp's earlier writes (ordered
// before lane 0 by __syncwarp) are visible to whoever acquires the count
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned need, long long limit, int* st) {
  volatile int* vst = st;
  long long it = 0;
  unsigned ns = 32;
  while (ld_acquire_u32(p) < need) {
    if (++it > limit) { atomicExch(&st[ST_TIMEOUT], 1); return false; }
    if ((it & 1023) == 0 && vst[ST_TIMEOUT]) return false;   // another wait expired
    // back off: waiting warps would otherwise take the issue slots of the
    // working warps on the same SM sub-partition
    __nanosleep(ns);
    ns = ns < 256 ? 2 * ns : 256;
  }
  return true;
}

__global__ void __launch_bounds__(BLK_THREADS) k_trsm_df(DfDev S, const int* __restrict__ ci,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ D, double* X, double* Y,
                                                         long long ld, int ncols, int ksplit, unsigned* cntA,
                                                         unsigned* cntB, double* Pc, int* st,
                                                         long long spin_limit) {
  const int cb = blockIdx.x / ksplit, p = blockIdx.x % ksplit;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int c = cb * 32 + lane;
  const bool on = c < ncols;
  const int gw = p * nwarps + warp, W = ksplit * nwarps;
  unsigned* cA = cntA + (size_t)cb * S.nsn;
  unsigned* cB = cntB + (size_t)cb * S.nsn;
  unsigned* cC = cntB + (size_t)gridDim.x / ksplit * S.nsn + (size_t)cb * S.nchunked;
  const long long pld = (long long)(gridDim.x / ksplit) * 32;   // row stride of the chunk partials
  for (int q = gw; q < S.ntask; q += W) {
    const int code = S.task[q];
    if (code >= 0) {
      // a row's external part, or one chunk of a long row's
      const bool chunk = code >= S.n;
      const int ck = chunk ? code - S.n : 0;
      const int r = chunk ? S.ck_row[ck] : code;
      const int d0 = S.dep_ptr[r], d1 = S.dep_ptr[r + 1];
      for (int db = d0; db < d1; db += 32) {
        bool ok = true;
        if (db + lane < d1) {
          const int sd = S.dep_sn[db + lane];
          ok = wait_count(cB + sd, (unsigned)S.sn_w[sd], spin_limit, st);
        }
        if (!__all_sync(FULL, ok)) return;
      }
      __syncwarp();
      const int e0 = chunk ? S.ck_e0[ck] : S.ext_beg[r], e1 = chunk ? S.ck_e1[ck] : S.ext_end[r];
      double a0 = (on && !chunk) ? __ldcg(&X[(long long)r * ld + c]) : 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
      for (int eb = e0; eb < e1; eb += 32) {
        const int len = min(32, e1 - eb);
        const int myj = lane < len ? ci[eb + lane] : 0;
        const double myv = lane < len ? val[eb + lane] : 0.0;
        int k = 0;
        for (; k + 3 < len; k += 4) {
          const int j0 = __shfl_sync(FULL, myj, k), j1 = __shfl_sync(FULL, myj, k + 1);
          const int j2 = __shfl_sync(FULL, myj, k + 2), j3 = __shfl_sync(FULL, myj, k + 3);
          const double v0 = __shfl_sync(FULL, myv, k), v1 = __shfl_sync(FULL, myv, k + 1);
          const double v2 = __shfl_sync(FULL, myv, k + 2), v3 = __shfl_sync(FULL, myv, k + 3);
          if (on) {
            a0 = fma(-v0, __ldcg(&X[(long long)j0 * ld + c]), a0);
            a1 = fma(-v1, __ldcg(&X[(long long)j1 * ld + c]), a1);
            a2 = fma(-v2, __ldcg(&X[(long long)j2 * ld + c]), a2);
            a3 = fma(-v3, __ldcg(&X[(long long)j3 * ld + c]), a3);
          }
        }
        for (; k < len; ++k) {
          const int j = __shfl_sync(FULL, myj, k);
          const double v = __shfl_sync(FULL, myv, k);
          if (on) a0 = fma(-v, __ldcg(&X[(long long)j * ld + c]), a0);
        }
      }
      if (!chunk) {
        if (on) Y[(long long)r * ld + c] = (a0 + a1) + (a2 + a3);
      } else {
        // the chunk's sum (entries subtracted) goes to its slot; the chunk that
        // completes the row adds the slots up in order and goes on as the row
        Pc[(long long)ck * pld + c] = (a0 + a1) + (a2 + a3);
        __syncwarp();
        const int ck0 = S.rw_ck0[r], nch = S.rw_ck0[r + 1] - ck0;
        unsigned old = 0;
        if (lane == 0)
          asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(cC + S.rw_cidx[r]) : "memory");
        old = __shfl_sync(FULL, old, 0);
        if (old + 1 != (unsigned)nch) continue;
        __syncwarp();
        if (on) {
          double y = __ldcg(&X[(long long)r * ld + c]);
          for (int k = 0; k < nch; ++k) y += __ldcg(&Pc[(long long)(ck0 + k) * pld + c]);
          Y[(long long)r * ld + c] = y;
        }
      }
      __syncwarp();
      const int s = S.sn_of[r], w = S.sn_w[s];
      if (w > DF_INLINE_B) {
        if (lane == 0) red_release_add(cA + s, 1u);
      } else {
        // narrow supernode: the warp that completes phase A also does phase B
        unsigned old = 0;
        if (lane == 0)
          asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(cA + s) : "memory");
        old = __shfl_sync(FULL, old, 0);
        if (old + 1 == (unsigned)w) {
          __syncwarp();
          const int f = S.sn_first[s];
          const double* Ds = D + S.d_off[s];
          double yv[DF_INLINE_B];
#pragma unroll
          for (int j = 0; j < DF_INLINE_B; ++j)
            yv[j] = (on && j < w) ? __ldcg(&Y[(long long)(f + j) * ld + c]) : 0.0;
#pragma unroll
          for (int i = 0; i < DF_INLINE_B; ++i) {
            if (i < w) {
              double a = 0.0;
#pragma unroll
              for (int j = 0; j < DF_INLINE_B; ++j)
                if (j < w && (S.upper ? j >= i : j <= i)) a = fma(Ds[i * w + j], yv[j], a);
              if (on) X[(long long)(f + i) * ld + c] = a;
            }
          }
          __syncwarp();
          if (lane == 0) red_release_add(cB + s, (unsigned)w);
        }
      }
    } else {
      const int r = -1 - code, s = S.sn_of[r];
      const int f = S.sn_first[s], w = S.sn_w[s];
      bool ok = true;
      if (lane == 0) ok = wait_count(cA + s, (unsigned)w, spin_limit, st);
      if (!__shfl_sync(FULL, (int)ok, 0)) return;
      __syncwarp();
      const double* Dr = D + S.d_off[s] + (r - f) * w;
      const int jb = S.upper ? r - f : 0, je = S.upper ? w : r - f + 1;   // nonzero half of the row
      double a0 = 0.0, a1 = 0.0;
      if (on) {
        int j = jb;
        for (; j + 1 < je; j += 2) {
          a0 = fma(Dr[j], __ldcg(&Y[(long long)(f + j) * ld + c]), a0);
          a1 = fma(Dr[j + 1], __ldcg(&Y[(long long)(f + j + 1) * ld + c]), a1);
        }
        if (j < je) a0 = fma(Dr[j], __ldcg(&Y[(long long)(f + j) * ld + c]), a0);
        X[(long long)r * ld + c] = a0 + a1;
      }
      __syncwarp();
      if (lane == 0) red_release_add(cB + s, 1u);
    }
  }
}

// The leaf supernodes of the dataflow schedule: X_s <- D_s X_s, one warp per
// (leaf, 32-column block), the supernode's rows held in registers (at most
// DF_LEAF_W); then its completion count is set for the dataflow kernel that
// follows on the stream.
__global__ void __launch_bounds__(256) k_trsm_df_leaf(DfDev S, const double* __restrict__ D, double* X,
                                                      long long ld, int ncols, unsigned* cntB) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int ncb = (ncols + 31) / 32;
  if (gw >= S.nleaf * ncb) return;
  const int l = gw % S.nleaf, cb = gw / S.nleaf;
  const int sn = S.leaf[l], f = S.sn_first[sn], w = S.sn_w[sn];
  const int c = cb * 32 + lane;
  const bool on = c < ncols;
  const double* Ds = D + S.d_off[sn];
  double xr[DF_LEAF_W];
#pragma unroll
  for (int j = 0; j < DF_LEAF_W; ++j) xr[j] = (on && j < w) ? X[(long long)(f + j) * ld + c] : 0.0;
#pragma unroll
  for (int i = 0; i < DF_LEAF_W; ++i) {
    if (i < w) {
      double a = 0.0;
#pragma unroll
      for (int j = 0; j < DF_LEAF_W; ++j)
        if (j < w && (S.upper ? j >= i : j <= i)) a = fma(Ds[i * w + j], xr[j], a);
      if (on) X[(long long)(f + i) * ld + c] = a;
    }
  }
  if (lane == 0) cntB[(size_t)cb * S.nsn + sn] = (unsigned)w;
}

}  // namespace

cudaError_t launch_trsm_df(cudaStream_t s, const DfDev& S, const int* ci, const double* val, const double* D,
                           double* X, double* Y, long long ld, int ncols, int ksplit, unsigned* cnt,
                           double* Pc, int* st, long long spin_limit) {
  if (ncols <= 0 || S.ntask + S.nleaf <= 0) return cudaSuccess;
  const int ncb = (ncols + 31) / 32;
  unsigned* cntA = cnt;
  unsigned* cntB = cnt + (size_t)ncb * S.nsn;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * ((size_t)2 * ncb * S.nsn + (size_t)ncb * S.nchunked), s);
  if (e != cudaSuccess) return e;
  if (S.nleaf > 0) {
    const long long warps = (long long)S.nleaf * ncb;
    k_trsm_df_leaf<<<int((warps * 32 + 255) / 256), 256, 0, s>>>(S, D, X, ld, ncols, cntB);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (S.ntask <= 0) return cudaSuccess;
  void* args[] = {(void*)&S,   (void*)&ci,     (void*)&val,  (void*)&D,    (void*)&X,  (void*)&Y,
                  (void*)&ld,  (void*)&ncols,  (void*)&ksplit, (void*)&cntA, (void*)&cntB, (void*)&Pc,
                  (void*)&st,  (void*)&spin_limit};
  note_launch();
  return cudaLaunchCooperativeKernel((void*)k_trsm_df, dim3(ncb * ksplit), dim3(BLK_THREADS), args, 0, s);
}

int trsm_df_max_blocks() {
  int dev = 0, sms = 0, a = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_trsm_df, BLK_THREADS, 0);
  return sms * std::max(a, 1);
}

}  // namespace condipm

namespace condipm {

cudaError_t launch_batch_factor_post(cudaStream_t s, const BatchInst* I, int n, const int* boffF, int nbF,
                                     const int* boffD, int nbD) {
  if (n <= 0) return cudaSuccess;
  k_b_gather<<<nbF, 256, 0, s>>>(I, n, boffF);
  note_launch();
  k_b_diag_inv<<<nbD, 128, 0, s>>>(I, n, boffD);
  note_launch();
  return cudaGetLastError();
}


cudaError_t launch_batch_trsm(cudaStream_t s, const BatchInst* I, const int2* cbs, int ncbs, int trans, int cl) {
  if (ncbs <= 0) return cudaSuccess;
  if (cl > 8) {
    cudaError_t e = allow_cluster16((const void*)k_b_trsm);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = trsm_cluster_config(ncbs, cl, s, at);
  note_launch();
  return cudaLaunchKernelEx(&cfg, k_b_trsm, I, cbs, trans);
}

int batch_trsm_clusters(int cl) {
  if (cl > 8 && allow_cluster16((const void*)k_b_trsm) != cudaSuccess) return 0;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = trsm_cluster_config(1, cl, nullptr, at);
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, (const void*)k_b_trsm, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

}  // namespace condipm

