// Device helpers shared by the kernels of the multilevel summation library.
#pragma once

#include <cuda_runtime.h>

#include "mls6_internal.h"

namespace mls6 {

// Block coordinates of a kernel body: the hardware block index and grid
// size in a kernel of its own, a work item's block index and block count
// when a persistent kernel runs the body.
struct Blk {
  unsigned x, n;
  static __device__ __forceinline__ Blk self() { return Blk{blockIdx.x, gridDim.x}; }
};

template <typename T> struct Box3 {
  T L[3], invL[3];
};

// i mod n in [0, n).  Indices are nearly always within one period of the
// grid (a node's neighbours), which is tested first; the remainder is taken
// only for grids narrower than the offset (repeated wrapping).
__device__ __forceinline__ int wrapi(int i, int n) {
  if ((unsigned)i < (unsigned)n) return i;
  if (i < 0 && i >= -n) return i + n;
  if (i >= n && i - n < n) return i - n;
  const int m = i % n;
  return m < 0 ? m + n : m;
}

// Position wrapped into [0, L).
template <typename T> __device__ __forceinline__ T wrapx(T x, T L, T invL) {
  T r = x - floor(x * invL) * L;
  if (r < T(0)) r += L;
  if (r >= L) r -= L;
  if (!(r >= T(0) && r < L)) r = T(0);
  return r;
}

// Weights of the four nodes base-1 .. base+2 of Eq. (Phi-Hermite) for an
// atom at fractional offset t in [0,1) from node base -- Phi(1+t), Phi(t),
// Phi(1-t), Phi(2-t) -- and (phi4 only) their derivatives in t.
template <typename T> __device__ __forceinline__ void phi4w(T t, T w[4]) {
  T s = T(1) - t;
  w[0] = T(-0.5) * t * s * s;
  w[1] = s * (T(1) + t - T(1.5) * t * t);
  w[2] = t * (T(1) + s - T(1.5) * s * s);
  w[3] = T(-0.5) * s * t * t;
}

template <typename T> __device__ __forceinline__ void phi4(T t, T w[4], T dw[4]) {
  phi4w(t, w);
  T s = T(1) - t;
  dw[0] = T(-0.5) * s * (T(1) - T(3) * t);
  dw[1] = t * (T(-5) + T(4.5) * t);
  dw[2] = s * (T(5) - T(4.5) * s);
  dw[3] = T(-0.5) * t * (T(2) - T(3) * t);
}

// Order p = 5: the C^1 quintic (even, support |t| < 3, reproducing
// polynomials of degree <= 4; the member whose outer piece continues to a
// root at |t| = 4).  Weights of the six nodes base-2 .. base+3 of an atom at
// offset t in [0,1) from node base -- Phi(2+t), Phi(1+t), Phi(t), Phi(1-t),
// Phi(2-t), Phi(3-t) -- in factored form (no cancellation near the ends of
// the support), and (phi6 only) their derivatives in t.
template <typename T> __device__ __forceinline__ void phi6w(T t, T w[6]) {
  const T s = T(1) - t, tp = T(1) + t, tm = T(2) - t;
  const T k24 = T(1.0 / 24.0), k12 = T(1.0 / 12.0);
  w[0] = k24 * t * s * s * tp * tm;
  w[1] = k24 * t * s * tm * (T(5) * t * t + t - T(8));
  w[2] = k12 * s * tm * tp * (T(6) + T(3) * t - T(5) * t * t);
  w[3] = k12 * t * tm * tp * (T(4) + T(7) * t - T(5) * t * t);
  w[4] = k24 * t * s * tp * (T(5) * t * t - T(11) * t - T(2));
  w[5] = k24 * t * t * s * tm * tp;
}

template <typename T> __device__ __forceinline__ void phi6(T t, T w[6], T dw[6]) {
  phi6w(t, w);
  const T s = T(1) - t;
  const T k24 = T(1.0 / 24.0), k12 = T(1.0 / 12.0);
  dw[0] = k24 * s * (((T(5) * t - T(7)) * t - T(4)) * t + T(2));
  dw[1] = k24 * ((((T(25) * t - T(56)) * t - T(3)) * t + T(52)) * t - T(16));
  dw[2] = -k12 * t * (((T(25) * t - T(52)) * t - T(15)) * t + T(50));
  dw[3] = -k12 * s * (((T(25) * t - T(23)) * t - T(44)) * t - T(8));
  dw[4] = -k24 * ((((T(25) * t - T(44)) * t - T(21)) * t + T(22)) * t + T(2));
  dw[5] = k24 * t * (((T(5) * t - T(8)) * t - T(3)) * t + T(4));
}

// Basis of NP = p + 1 nodes per axis: weights (and derivatives) of nodes
// base - (NP/2 - 1) .. base + NP/2.
template <int NP, typename T> __device__ __forceinline__ void phiw(T t, T* w) {
  if constexpr (NP == 6)
    phi6w(t, w);
  else
    phi4w(t, w);
}
template <int NP, typename T> __device__ __forceinline__ void phid(T t, T* w, T* dw) {
  if constexpr (NP == 6)
    phi6(t, w, dw);
  else
    phi4(t, w, dw);
}

// Restriction / prolongation: Phi at half-integers.  For a fine node at
// coarse position c + 1/2 the NP coarse nodes c - (NP/2 - 1) .. c + NP/2
// weigh Phi(NP/2 - 1/2), ..., Phi(1/2), Phi(1/2), ..., Phi(NP/2 - 1/2);
// restriction takes the same values at fine offsets +-1, +-3, +-5 from 2 mu.
template <int NP, typename T> __device__ __forceinline__ T half_weight(int k) {
  // k = 0: Phi(1/2), 1: Phi(3/2), 2: Phi(5/2)
  if constexpr (NP == 6)
    return k == 0 ? T(150.0 / 256.0) : (k == 1 ? T(-25.0 / 256.0) : T(3.0 / 256.0));
  else
    return k == 0 ? T(0.5625) : T(-0.0625);
}

// Programmatic dependent launch: every kernel of the evaluation chain first
// waits until its predecessor has completed and flushed (wait), then lets
// its successor be scheduled (launch_dependents), so the successor's launch
// overlaps this kernel's work while every memory access still follows plain
// stream order.  Triggering before the wait let whole chains of waiting
// kernels become resident at once, and under CUDA-graph replay a kernel
// then read a value (the fixed-point scale) that two launches earlier had
// not yet written; with the trigger after the wait at most one kernel waits
// ahead of the running one.  Both are no-ops for a kernel launched without
// the programmatic-serialization attribute.
//
// The wait orders memory operations only for the compiler's ordinary loads:
// a load through a `const T* __restrict__` parameter is treated as
// invariant for the whole kernel and may be scheduled above the wait.
// pdl_begin therefore returns a zero produced by an opaque instruction after
// the wait; kernels add it to every such pointer (`p += z`), so no load
// through them can be issued before the wait (the pointers stay based on
// their restrict parameters).
__device__ __forceinline__ long pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  long z;
  asm volatile("mov.b64 %0, 0;" : "=l"(z)::"memory");
  return z;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sums of NV doubles (blockDim.x a multiple of 32, <= 1024);
// results valid in thread 0; fixed reduction order.  sh: >= 32*NV doubles.
template <int NV> __device__ __forceinline__ void block_sum_n(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) v[c] = warp_sum(v[c]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) sh[c * 32 + wid] = v[c];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[c * 32 + w];
      v[c] = s;
    }
}

// Block-wide sums of NV values accumulated in the kernel's precision T:
// each warp sums in T, warp leaders promote to double and thread 0 adds the
// warp totals in double (fixed order).  Keeps FP64 work, which runs at a
// small fraction of the FP32 rate, to NV values per warp.  Results valid in
// thread 0 (out); sh: >= 32*NV doubles.
template <typename T, int NV>
__device__ __forceinline__ void block_sum_lo(T (&v)[NV], double (&out)[NV], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) sh[c * 32 + wid] = (double)v[c];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NV; ++c) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[c * 32 + w];
      out[c] = s;
    }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  double a[1] = {v};
  block_sum_n<1>(a, sh);
  return a[0];
}

// Fixed-order sum, by one block, of the energy partials (ne doubles) and,
// if vir, of the virial partials (nw records of 6) into out[0..6].
// sh: >= 32*7 doubles.
__device__ __forceinline__ void final_reduce(const double* __restrict__ epart, long ne,
                                             const double* __restrict__ wpart, long nw, int vir,
                                             double* __restrict__ out, double* sh) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long k = threadIdx.x; k < ne; k += blockDim.x) v[0] += epart[k];
  if (vir)
    for (long k = threadIdx.x; k < nw; k += blockDim.x)
#pragma unroll
      for (int c = 0; c < 6; ++c) v[1 + c] += wpart[6 * k + c];
  block_sum_n<7>(v, sh);
  if (threadIdx.x == 0)
    for (int c = 0; c < 7; ++c) out[c] = v[c];
}

// Eq. (last-grid-periodic-transformed) for coarsest node mu in FP64, by
// one warp: the lanes stride over nu; e_mu = sum_nu T[(mu - nu) mod n] q_nu
// and the virial record 1/2 q_mu sum_nu V[(mu - nu) mod n] q_nu.  Partial
// sums are combined by shuffles in a fixed order.
template <typename T, bool VIR>
__device__ __forceinline__ void coarsest_node(const T* __restrict__ q, int n0, int n1, int n2,
                                              const double* __restrict__ tT,
                                              const double* __restrict__ tV, T* __restrict__ e,
                                              double* __restrict__ wpart, int mu) {
  const int lane = threadIdx.x & 31;
  const int np = n0 * n1 * n2;
  const int a = mu % n0, b = (mu / n0) % n1, c = mu / (n0 * n1);
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int nu = lane; nu < np; nu += 32) {
    const int a2 = nu % n0, b2 = (nu / n0) % n1, c2 = nu / (n0 * n1);
    int da = a - a2, db = b - b2, dc = c - c2;
    if (da < 0) da += n0;
    if (db < 0) db += n1;
    if (dc < 0) dc += n2;
    const int m = da + n0 * (db + n1 * dc);
    const double qv = (double)q[nu];
    v[0] += tT[m] * qv;
    if (VIR)
#pragma unroll
      for (int k = 0; k < 6; ++k) v[1 + k] += tV[(size_t)k * np + m] * qv;
  }
#pragma unroll
  for (int k = 0; k < (VIR ? 7 : 1); ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0) {
    e[mu] = (T)v[0];
    if (VIR) {
      const double hq = 0.5 * (double)q[mu];
      for (int k = 0; k < 6; ++k) wpart[6 * (size_t)mu + k] = hq * v[1 + k];
    }
  }
}

// Launch with the programmatic-stream-serialization attribute (see
// pdl_begin); same semantics as kernel<<<grid, block, smem, st>>>(args...).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace mls6
