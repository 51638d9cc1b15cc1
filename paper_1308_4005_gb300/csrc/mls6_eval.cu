// Device side of the multilevel summation library for r^-6 dispersion
// (arXiv 1308.4005): one evaluation is a fixed sequence of kernels on the
// plan's stream.
//
//   bin      wrap positions, cell histogram, scan, scatter, per-cell order
//   pair     local part g_0 (Eq. g_0) over the cell list
//   anterp   Eq. (anterpolation) onto the finest grid
//   restrict xi^{k+1} = R xi^k (Sec. II.B, restriction)
//   stencil  Eq. (evaluation) on levels k < l (cutoff 2^k a)
//   top      Eq. (last-grid-periodic-transformed) on level l
//   prolong  e^{k,tot} = e^k + R^T e^{k+1,tot} (Sec. II.B, prolongation)
//   interp   Eq. (interpolation), its gradient (forces), per-atom energy
//   reduce   fixed-order sums of energy and virial partials
#include <math.h>
#include <stdio.h>

#include "mls6_internal.h"

namespace mls6 {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return MLS6_ERR_CUDA; \
  } while (0)

static inline long cdiv(long a, long b) { return (a + b - 1) / b; }

template <typename T> struct Box3 {
  T L[3], invL[3];
};

__device__ __forceinline__ int wrapi(int i, int n) {
  int m = i % n;
  return m < 0 ? m + n : m;
}

template <typename T> __device__ __forceinline__ T wrapx(T x, T L, T invL) {
  T r = x - floor(x * invL) * L;
  if (r < T(0)) r += L;
  if (r >= L) r -= L;
  if (!(r >= T(0) && r < L)) r = T(0);
  return r;
}

// Weights of the four nodes base-1 .. base+2 of Eq. (Phi-Hermite) for an
// atom at fractional offset t in [0,1) from node base, and their
// derivatives with respect to t:  Phi(1+t), Phi(t), Phi(1-t), Phi(2-t).
template <typename T> __device__ __forceinline__ void phi4(T t, T w[4], T dw[4]) {
  T s = T(1) - t;
  w[0] = T(-0.5) * t * s * s;
  w[1] = s * (T(1) + t - T(1.5) * t * t);
  w[2] = t * (T(1) + s - T(1.5) * s * s);
  w[3] = T(-0.5) * s * t * t;
  dw[0] = T(-0.5) * s * (T(1) - T(3) * t);
  dw[1] = t * (T(-5) + T(4.5) * t);
  dw[2] = s * (T(5) - T(4.5) * s);
  dw[3] = T(-0.5) * t * (T(2) - T(3) * t);
}

template <typename T> __device__ __forceinline__ void phi4w(T t, T w[4]) {
  T s = T(1) - t;
  w[0] = T(-0.5) * t * s * s;
  w[1] = s * (T(1) + t - T(1.5) * t * t);
  w[2] = t * (T(1) + s - T(1.5) * s * s);
  w[3] = T(-0.5) * s * t * t;
}

// Block-wide sum of a double (blockDim.x a multiple of 32, <= 1024); the
// result is valid in thread 0.  Fixed reduction order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

// ------------------------------------------------------------------ binning

template <typename T> struct BinArgs {
  Box3<T> box;
  T inv_w[3];
  int nc[3];
};

template <typename T>
__global__ void k_bin(const T* __restrict__ pos, const T* __restrict__ cc, int stride, int N,
                      BinArgs<T> g, Vec4<T>* __restrict__ posw, int* __restrict__ cell_of,
                      int* __restrict__ count, int* __restrict__ flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T* p = pos + (size_t)i * stride;
  T x = p[0], y = p[1], z = p[2];
  T c = cc ? cc[i] : p[3];
  if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(c))) {
    atomicOr(flag, 1);
    x = y = z = c = T(0);
  }
  x = wrapx(x, g.box.L[0], g.box.invL[0]);
  y = wrapx(y, g.box.L[1], g.box.invL[1]);
  z = wrapx(z, g.box.L[2], g.box.invL[2]);
  int cx = min(max((int)(x * g.inv_w[0]), 0), g.nc[0] - 1);
  int cy = min(max((int)(y * g.inv_w[1]), 0), g.nc[1] - 1);
  int cz = min(max((int)(z * g.inv_w[2]), 0), g.nc[2] - 1);
  int cell = cx + g.nc[0] * (cy + g.nc[1] * cz);
  cell_of[i] = cell;
  Vec4<T> v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = c;
  posw[i] = v;
  atomicAdd(&count[cell], 1);
}

constexpr int kScanTile = 2048;  // elements per block in the cell scan

// Phase 1: tile sums.
__global__ void k_scan_tiles(const int* __restrict__ count, long n, int* __restrict__ tsum) {
  __shared__ double sh[32];
  long base = (long)blockIdx.x * kScanTile;
  int s = 0;
  for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
    if (base + t < n) s += count[base + t];
  double tot = block_sum((double)s, sh);
  if (threadIdx.x == 0) tsum[blockIdx.x] = (int)tot;
}

// Phase 2: exclusive scan of the tile sums (single block, serial over the
// few hundred tiles) -> tile offsets; writes the grand total to start[n].
__global__ void k_scan_top(int* __restrict__ tsum, int ntiles, int* __restrict__ start, long n) {
  if (threadIdx.x != 0) return;
  int acc = 0;
  for (int t = 0; t < ntiles; ++t) {
    int v = tsum[t];
    tsum[t] = acc;
    acc += v;
  }
  start[n] = acc;
}

// Phase 3: scan inside each tile (256 threads x 8 consecutive elements),
// write start[], reset count[] for use as fill counters.
__global__ void k_scan_final(int* __restrict__ count, long n, const int* __restrict__ toff,
                             int* __restrict__ start) {
  __shared__ int wsum[32];
  constexpr int PER = kScanTile / 256;
  long base = (long)blockIdx.x * kScanTile + (long)threadIdx.x * PER;
  int v[PER], s = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    v[k] = (base + k < n) ? count[base + k] : 0;
    s += v[k];
  }
  // inclusive scan of s across the block
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int x = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    wsum[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  int excl = incl - s + (wid > 0 ? wsum[wid - 1] : 0) + toff[blockIdx.x];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (base + k < n) {
      start[base + k] = excl;
      count[base + k] = 0;
    }
    excl += v[k];
  }
}

template <typename T>
__global__ void k_scatter(const Vec4<T>* __restrict__ posw, const int* __restrict__ cell_of, int N,
                          const int* __restrict__ start, int* __restrict__ fill,
                          Vec4<T>* __restrict__ sorted, int* __restrict__ sidx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int cell = cell_of[i];
  int slot = start[cell] + atomicAdd(&fill[cell], 1);
  sorted[slot] = posw[i];
  sidx[slot] = i;
}

// Order the atoms of every cell by their input index so that all later
// sums run in a reproducible order (cells above 256 atoms are left as
// scattered; results stay correct, only bitwise reproducibility is lost).
template <typename T>
__global__ void k_cellsort(const int* __restrict__ start, long ncell, Vec4<T>* __restrict__ sorted,
                           int* __restrict__ sidx) {
  long cell = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= ncell) return;
  int b = start[cell], e = start[cell + 1];
  if (e - b < 2 || e - b > 256) return;
  for (int i = b + 1; i < e; ++i) {
    int key = sidx[i];
    Vec4<T> v = sorted[i];
    int j = i - 1;
    while (j >= b && sidx[j] > key) {
      sidx[j + 1] = sidx[j];
      sorted[j + 1] = sorted[j];
      --j;
    }
    sidx[j + 1] = key;
    sorted[j + 1] = v;
  }
}

// ------------------------------------------------------------- local part

template <typename T> struct PairArgs {
  Box3<T> box;
  T inv_w[3];
  int nc[3], R[3];
  T a2, ia2, ia6, ia8;
};

// e0_i = sum_{j,n: r<a} c_j g_0(r)  (Eq. g_0); F_i = -c_i sum c_j g_0'(r)/r d,
// d = x_j - x_i + n L; virial 1/2 c_i sum c_j g_0'(r)/r d (x) d.
// g_0 = r^-6 - a^-6 gamma(r/a) with gamma an even polynomial in r (no sqrt).
template <typename T, bool VIR>
__global__ void __launch_bounds__(kBlock) k_pair(const Vec4<T>* __restrict__ sp,
                                                  const int* __restrict__ start, int N,
                                                  PairArgs<T> g, T* __restrict__ e0,
                                                  T* __restrict__ floc,
                                                  double* __restrict__ wpart) {
  __shared__ double sh[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  T e = 0, fx = 0, fy = 0, fz = 0;
  T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  T ci = 0;
  if (i < N) {
    Vec4<T> pi = sp[i];
    ci = pi.w;
    int cx = min(max((int)(pi.x * g.inv_w[0]), 0), g.nc[0] - 1);
    int cy = min(max((int)(pi.y * g.inv_w[1]), 0), g.nc[1] - 1);
    int cz = min(max((int)(pi.z * g.inv_w[2]), 0), g.nc[2] - 1);
    for (int dz = -g.R[2]; dz <= g.R[2]; ++dz) {
      int z = cz + dz, iz = wrapi(z, g.nc[2]);
      T sz = (T)((z - iz) / g.nc[2]) * g.box.L[2];
      for (int dy = -g.R[1]; dy <= g.R[1]; ++dy) {
        int y = cy + dy, iy = wrapi(y, g.nc[1]);
        T sy = (T)((y - iy) / g.nc[1]) * g.box.L[1];
        int row = g.nc[0] * (iy + g.nc[1] * iz);
        int dx = -g.R[0];
        while (dx <= g.R[0]) {
          int x = cx + dx, ix = wrapi(x, g.nc[0]);
          int wx = (x - ix) / g.nc[0];
          int last = min(g.R[0], dx + (g.nc[0] - 1 - ix));  // same image run
          T sx = (T)wx * g.box.L[0];
          bool same = (wx == 0) && (y == iy) && (z == iz);
          int j0 = start[row + ix], j1 = start[row + ix + (last - dx) + 1];
          for (int j = j0; j < j1; ++j) {
            if (same && j == i) continue;
            Vec4<T> pj = sp[j];
            T ddx = (pj.x - pi.x) + sx, ddy = (pj.y - pi.y) + sy, ddz = (pj.z - pi.z) + sz;
            T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 < g.a2) {
              T inv = T(1) / r2;
              T inv3 = inv * inv * inv;
              T s = r2 * g.ia2, s2 = s * s, s3 = s2 * s, s6 = s3 * s3;
              T s5 = s3 * s2;
              T g0 = inv3 - g.ia6 * (T(1.875) - T(1.25) * s6 + T(0.375) * s6 * s6);
              T gp = T(-6) * inv3 * inv + g.ia8 * s5 * (T(15) - T(9) * s6);
              e += pj.w * g0;
              T cg = pj.w * gp;
              fx += cg * ddx;
              fy += cg * ddy;
              fz += cg * ddz;
              if (VIR) {
                w0 += cg * ddx * ddx;
                w1 += cg * ddy * ddy;
                w2 += cg * ddz * ddz;
                w3 += cg * ddx * ddy;
                w4 += cg * ddx * ddz;
                w5 += cg * ddy * ddz;
              }
            }
          }
          dx = last + 1;
        }
      }
    }
    e0[i] = e;
    floc[3 * (size_t)i + 0] = -ci * fx;
    floc[3 * (size_t)i + 1] = -ci * fy;
    floc[3 * (size_t)i + 2] = -ci * fz;
  }
  if (VIR) {
    double hc = 0.5 * (double)ci;
    double wv[6] = {hc * w0, hc * w1, hc * w2, hc * w3, hc * w4, hc * w5};
    for (int c = 0; c < 6; ++c) {
      double s = block_sum(wv[c], sh);
      if (threadIdx.x == 0) wpart[6 * (size_t)blockIdx.x + c] = s;
    }
  }
}

// ---------------------------------------------------------------- grids

struct GridDims {
  int n[3];
  float inv_h[3];  // unused for FP64 (kept for layout symmetry)
};

// Eq. (anterpolation): q^1_mu += c_j phi_mu(x_j) over the 4x4x4 nodes.
template <typename T>
__global__ void k_anterp(const Vec4<T>* __restrict__ sp, int N, int n0, int n1, int n2, T ih0,
                         T ih1, T ih2, T* __restrict__ q) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  Vec4<T> p = sp[i];
  T u0 = p.x * ih0, u1 = p.y * ih1, u2 = p.z * ih2;
  T f0 = floor(u0), f1 = floor(u1), f2 = floor(u2);
  int b0 = (int)f0, b1 = (int)f1, b2 = (int)f2;
  T wx[4], wy[4], wz[4];
  phi4w(u0 - f0, wx);
  phi4w(u1 - f1, wy);
  phi4w(u2 - f2, wz);
  int ix[4], iy[4], iz[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ix[k] = wrapi(b0 - 1 + k, n0);
    iy[k] = wrapi(b1 - 1 + k, n1);
    iz[k] = wrapi(b2 - 1 + k, n2);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      T wyz = p.w * wy[b] * wz[c];
      long rowi = (long)n0 * (iy[b] + (long)n1 * iz[c]);
#pragma unroll
      for (int a = 0; a < 4; ++a) atomicAdd(&q[rowi + ix[a]], wyz * wx[a]);
    }
}

// Restriction: q^{k+1}_mu = sum_nu prod_d Phi(nu_d/2 - mu_d) q^k_nu; the
// nonzero weights are Phi(0)=1, Phi(1/2)=9/16, Phi(3/2)=-1/16 at fine
// offsets 0, +-1, +-3 from 2 mu.
template <typename T>
__global__ void k_restrict(const T* __restrict__ qf, int f0, int f1, int f2, T* __restrict__ qc,
                           int c0, int c1, int c2) {
  long mu = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long np = (long)c0 * c1 * c2;
  if (mu >= np) return;
  int m0 = (int)(mu % c0), m1 = (int)((mu / c0) % c1), m2 = (int)(mu / ((long)c0 * c1));
  const int off[5] = {-3, -1, 0, 1, 3};
  const T wt[5] = {T(-0.0625), T(0.5625), T(1), T(0.5625), T(-0.0625)};
  T acc = 0;
  for (int c = 0; c < 5; ++c) {
    int z = wrapi(2 * m2 + off[c], f2);
    for (int b = 0; b < 5; ++b) {
      int y = wrapi(2 * m1 + off[b], f1);
      long row = (long)f0 * (y + (long)f1 * z);
      T wyz = wt[b] * wt[c];
      T s = 0;
      for (int a = 0; a < 5; ++a) s += wt[a] * qf[row + wrapi(2 * m0 + off[a], f0)];
      acc += wyz * s;
    }
  }
  qc[mu] = acc;
}

// Periodic copy of a level grid with a halo of p[d] nodes per side.
template <typename T>
__global__ void k_pad(const T* __restrict__ q, int n0, int n1, int n2, int p0, int p1, int p2,
                      T* __restrict__ qp) {
  long P0 = n0 + 2 * p0, P1 = n1 + 2 * p1, P2 = n2 + 2 * p2;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P0 * P1 * P2) return;
  int a = (int)(idx % P0), b = (int)((idx / P0) % P1), c = (int)(idx / (P0 * P1));
  qp[idx] = q[wrapi(a - p0, n0) + (long)n0 * (wrapi(b - p1, n1) + (long)n1 * wrapi(c - p2, n2))];
}

// Eq. (evaluation) on level k < l: e_mu = s_k sum_t g_t q_{mu + m_t}, with
// s_k = 2^(-6(k-1)) and the level-1 taps g_t = g_1(|m_t h_1|).  The strain
// derivative adds 1/2 q_mu s_k sum_t v_t q_{mu+m_t} to the virial.
template <typename T, bool VIR>
__global__ void __launch_bounds__(kBlock) k_stencil(const T* __restrict__ qp,
                                                     const T* __restrict__ q, int n0, int n1,
                                                     int n2, int p0, int p1, int p2,
                                                     const int* __restrict__ toff,
                                                     const T* __restrict__ tg,
                                                     const T* __restrict__ tv, int ntaps,
                                                     T scale, T* __restrict__ e,
                                                     double* __restrict__ wpart) {
  __shared__ double sh[32];
  long np = (long)n0 * n1 * n2;
  long mu = (long)blockIdx.x * blockDim.x + threadIdx.x;
  T acc = 0, v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0, v5 = 0, qmu = 0;
  if (mu < np) {
    int a = (int)(mu % n0), b = (int)((mu / n0) % n1), c = (int)(mu / ((long)n0 * n1));
    long P0 = n0 + 2 * p0, P1 = n1 + 2 * p1;
    long base = (a + p0) + P0 * ((b + p1) + P1 * (c + p2));
    for (int t = 0; t < ntaps; ++t) {
      T qv = qp[base + toff[t]];
      acc += tg[t] * qv;
      if (VIR) {
        const T* vt = tv + 6 * (size_t)t;
        v0 += vt[0] * qv;
        v1 += vt[1] * qv;
        v2 += vt[2] * qv;
        v3 += vt[3] * qv;
        v4 += vt[4] * qv;
        v5 += vt[5] * qv;
      }
    }
    e[mu] = scale * acc;
    qmu = q[mu];
  }
  if (VIR) {
    double hq = 0.5 * (double)qmu * (double)scale;
    double wv[6] = {hq * v0, hq * v1, hq * v2, hq * v3, hq * v4, hq * v5};
    for (int cc = 0; cc < 6; ++cc) {
      double s = block_sum(wv[cc], sh);
      if (threadIdx.x == 0) wpart[6 * (size_t)blockIdx.x + cc] = s;
    }
  }
}

// Coarsest level, all-to-all with the periodic table T (FP64).
template <typename T, bool VIR>
__global__ void __launch_bounds__(kBlock) k_top(const T* __restrict__ q, int n0, int n1, int n2,
                                                 const double* __restrict__ tT,
                                                 const double* __restrict__ tV,
                                                 T* __restrict__ e, double* __restrict__ wpart) {
  __shared__ double sh[32];
  long np = (long)n0 * n1 * n2;
  long mu = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0, v[6] = {0, 0, 0, 0, 0, 0}, qmu = 0;
  if (mu < np) {
    int a = (int)(mu % n0), b = (int)((mu / n0) % n1), c = (int)(mu / ((long)n0 * n1));
    for (long nu = 0; nu < np; ++nu) {
      int a2 = (int)(nu % n0), b2 = (int)((nu / n0) % n1), c2 = (int)(nu / ((long)n0 * n1));
      int da = a - a2, db = b - b2, dc = c - c2;
      if (da < 0) da += n0;
      if (db < 0) db += n1;
      if (dc < 0) dc += n2;
      long m = da + (long)n0 * (db + (long)n1 * dc);
      double qv = (double)q[nu];
      acc += tT[m] * qv;
      if (VIR)
        for (int k = 0; k < 6; ++k) v[k] += tV[k * np + m] * qv;
    }
    e[mu] = (T)acc;
    qmu = (double)q[mu];
  }
  if (VIR) {
    for (int k = 0; k < 6; ++k) {
      double s = block_sum(0.5 * qmu * v[k], sh);
      if (threadIdx.x == 0) wpart[6 * (size_t)blockIdx.x + k] = s;
    }
  }
}

// Prolongation onto the fine level: et_f = e_f + sum_nu prod_d Phi(mu_d/2 - nu_d) et_c.
template <typename T>
__global__ void k_prolong(const T* __restrict__ ef, int f0, int f1, int f2,
                          const T* __restrict__ etc_, int c0, int c1, int c2,
                          T* __restrict__ etf) {
  long mu = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long np = (long)f0 * f1 * f2;
  if (mu >= np) return;
  int m[3] = {(int)(mu % f0), (int)((mu / f0) % f1), (int)(mu / ((long)f0 * f1))};
  int nc[3] = {c0, c1, c2};
  int idx[3][4];
  T wt[3][4];
  int cnt[3];
  for (int d = 0; d < 3; ++d) {
    if ((m[d] & 1) == 0) {
      cnt[d] = 1;
      idx[d][0] = wrapi(m[d] >> 1, nc[d]);
      wt[d][0] = T(1);
    } else {
      cnt[d] = 4;
      int h = (m[d] - 1) >> 1;  // coarse node left of mu
      idx[d][0] = wrapi(h - 1, nc[d]);
      idx[d][1] = wrapi(h, nc[d]);
      idx[d][2] = wrapi(h + 1, nc[d]);
      idx[d][3] = wrapi(h + 2, nc[d]);
      wt[d][0] = T(-0.0625);
      wt[d][1] = T(0.5625);
      wt[d][2] = T(0.5625);
      wt[d][3] = T(-0.0625);
    }
  }
  T acc = 0;
  for (int c = 0; c < cnt[2]; ++c)
    for (int b = 0; b < cnt[1]; ++b) {
      long row = (long)c0 * (idx[1][b] + (long)c1 * idx[2][c]);
      T s = 0;
      for (int a = 0; a < cnt[0]; ++a) s += wt[0][a] * etc_[row + idx[0][a]];
      acc += wt[1][b] * wt[2][c] * s;
    }
  etf[mu] = ef[mu] + acc;
}

// Eq. (interpolation) and its gradient: e_i = sum phi e^{1,tot},
// F_i = F_i^loc + c_i grad e_i; per-atom energy
// -1/2 c_i (e0_i + e_i) + 1/2 c_self c_i^2; energy partial per block.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_interp(
    const Vec4<T>* __restrict__ sp, const int* __restrict__ sidx, int N, const T* __restrict__ et,
    int n0, int n1, int n2, T ih0, T ih1, T ih2, const T* __restrict__ e0,
    const T* __restrict__ floc, double cself, T* __restrict__ forces,
    double* __restrict__ atom_energy, double* __restrict__ epart) {
  __shared__ double sh[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ea = 0.0;
  if (i < N) {
    Vec4<T> p = sp[i];
    T u0 = p.x * ih0, u1 = p.y * ih1, u2 = p.z * ih2;
    T f0 = floor(u0), f1 = floor(u1), f2 = floor(u2);
    int b0 = (int)f0, b1 = (int)f1, b2 = (int)f2;
    T wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    phi4(u0 - f0, wx, dx);
    phi4(u1 - f1, wy, dy);
    phi4(u2 - f2, wz, dz);
    int ix[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) ix[k] = wrapi(b0 - 1 + k, n0);
    T acc = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int z = wrapi(b2 - 1 + c, n2);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int y = wrapi(b1 - 1 + b, n1);
        const T* row = et + (long)n0 * (y + (long)n1 * z);
        T sx = 0, sdx = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          T v = row[ix[a]];
          sx += wx[a] * v;
          sdx += dx[a] * v;
        }
        acc += wy[b] * wz[c] * sx;
        g0 += wy[b] * wz[c] * sdx;
        g1 += dy[b] * wz[c] * sx;
        g2 += wy[b] * dz[c] * sx;
      }
    }
    int o = sidx[i];
    T ci = p.w;
    forces[3 * (size_t)o + 0] = floc[3 * (size_t)i + 0] + ci * g0 * ih0;
    forces[3 * (size_t)o + 1] = floc[3 * (size_t)i + 1] + ci * g1 * ih1;
    forces[3 * (size_t)o + 2] = floc[3 * (size_t)i + 2] + ci * g2 * ih2;
    double cd = (double)ci;
    ea = -0.5 * cd * ((double)e0[i] + (double)acc) + 0.5 * cself * cd * cd;
    if (atom_energy) atom_energy[o] = ea;
  }
  double s = block_sum(ea, sh);
  if (threadIdx.x == 0) epart[blockIdx.x] = s;
}

// Fixed-order reduction of the energy and virial partials (one block).
__global__ void k_reduce(const double* __restrict__ epart, long ne,
                         const double* __restrict__ wpart, long nw, int vir,
                         double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long k = threadIdx.x; k < ne; k += blockDim.x) s += epart[k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
  for (int c = 0; c < 6; ++c) {
    double w = 0.0;
    if (vir)
      for (long k = threadIdx.x; k < nw; k += blockDim.x) w += wpart[6 * k + c];
    w = block_sum(w, sh);
    if (threadIdx.x == 0) out[1 + c] = w;
  }
}

// ------------------------------------------------------------ host side

static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T> static int upload_tables_t(Plan* p) {
  const long N = p->N;
  const size_t e = sizeof(T);
  auto A = [&](void** ptr, size_t bytes) -> int {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(ptr, bytes) == cudaSuccess ? 0 : MLS6_ERR_NOMEM;
  };
  int rc = 0;
  rc |= A(&p->d_pos_w, sizeof(Vec4<T>) * N);
  rc |= A((void**)&p->d_cell_of, sizeof(int) * N);
  rc |= A((void**)&p->d_cell_count, sizeof(int) * p->cg.ncell);
  rc |= A((void**)&p->d_cell_start, sizeof(int) * (p->cg.ncell + 1));
  rc |= A(&p->d_sorted, sizeof(Vec4<T>) * N);
  rc |= A((void**)&p->d_sorted_idx, sizeof(int) * N);
  rc |= A(&p->d_e0, e * N);
  rc |= A(&p->d_floc, 3 * e * N);
  const int l = p->levels;
  long padmax = 0;
  for (int k = 1; k <= l; ++k) {
    rc |= A(&p->d_q[k], e * p->lv[k].np);
    rc |= A(&p->d_e[k], e * p->lv[k].np);
    if (k < l) {
      rc |= A(&p->d_et[k], e * p->lv[k].np);
      long P = 1;
      for (int d = 0; d < 3; ++d) P *= p->lv[k].n[d] + 2 * p->pad[d];
      padmax = std::max(padmax, P);
    }
  }
  if (rc) return MLS6_ERR_NOMEM;
  p->d_et[l] = p->d_e[l];  // alias: e^{l,tot} = e^l
  if (l >= 2) {
    rc |= A(&p->d_qpad, e * padmax);
    rc |= A((void**)&p->d_tap_off, sizeof(int) * p->ntaps * (l - 1));
    rc |= A(&p->d_tap_g, e * p->ntaps);
    rc |= A(&p->d_tap_v, 6 * e * p->ntaps);
  }
  const long np_top = p->lv[l].np;
  rc |= A((void**)&p->d_top_T, sizeof(double) * np_top);
  rc |= A((void**)&p->d_top_V, 6 * sizeof(double) * np_top);
  // partial sums
  p->n_epart = std::max(1L, cdiv(N, kBlock));
  p->n_pair_blocks = std::max(1L, cdiv(N, kBlock));
  p->wpart_pair = 0;
  long nw = p->n_pair_blocks;
  for (int k = 1; k < l; ++k) {
    p->wpart_lvl[k] = nw;
    nw += cdiv(p->lv[k].np, kBlock);
  }
  p->wpart_top = nw;
  nw += cdiv(np_top, kBlock);
  p->n_wpart = nw;
  rc |= A((void**)&p->d_epart, sizeof(double) * p->n_epart);
  rc |= A((void**)&p->d_wpart, 6 * sizeof(double) * p->n_wpart);
  rc |= A((void**)&p->d_out, 8 * sizeof(double));
  rc |= A((void**)&p->d_flag, sizeof(int) * 4);
  rc |= A((void**)&p->d_scan, sizeof(int) * std::max(1L, cdiv(p->cg.ncell, kScanTile)));
  if (rc) return MLS6_ERR_NOMEM;
  if (cudaMallocHost((void**)&p->h_out, 8 * sizeof(double)) != cudaSuccess) return MLS6_ERR_NOMEM;

  // tables
  if (l >= 2) {
    std::vector<int> off((size_t)p->ntaps * (l - 1));
    for (int k = 1; k < l; ++k) {
      long P0 = p->lv[k].n[0] + 2 * p->pad[0], P1 = p->lv[k].n[1] + 2 * p->pad[1];
      for (int t = 0; t < p->ntaps; ++t) {
        const int* m = &p->h_tap_m[3 * t];
        off[(size_t)(k - 1) * p->ntaps + t] = (int)(m[0] + P0 * (m[1] + P1 * m[2]));
      }
    }
    std::vector<T> tg(p->ntaps), tv(6 * (size_t)p->ntaps);
    for (int t = 0; t < p->ntaps; ++t) tg[t] = (T)p->h_tap_g[t];
    for (size_t t = 0; t < tv.size(); ++t) tv[t] = (T)p->h_tap_v[t];
    CK(cudaMemcpy(p->d_tap_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->d_tap_g, tg.data(), e * tg.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->d_tap_v, tv.data(), e * tv.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(p->d_top_T, p->h_top_T.data(), sizeof(double) * np_top, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->d_top_V, p->h_top_V.data(), 6 * sizeof(double) * np_top,
                cudaMemcpyHostToDevice));
  CK(cudaMemset(p->d_flag, 0, sizeof(int) * 4));
  return MLS6_OK;
}

int upload_tables(Plan* p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MLS6_ERR_CUDA;
  }
  return p->prec == MLS6_FP64 ? upload_tables_t<double>(p) : upload_tables_t<float>(p);
}

template <typename T>
static int eval_t(Plan* p, const void* pos_, const void* c_, void* forces_, double* energy,
                  double* virial, double* atom_energy) {
  cudaStream_t st = p->stream;
  const int N = (int)p->N;
  const int l = p->levels;
  const bool vir = virial != nullptr;
  const T* pos = (const T*)pos_;
  const T* cc = (const T*)c_;
  T* forces = (T*)forces_;
  if (N > 0 && (!pos || !forces)) return MLS6_ERR_ARG;

#define MARK(i) \
  do { if (p->prof) CK(cudaEventRecord(p->ev[i], st)); } while (0)
  int nl_ = 0;  // kernels launched
  MARK(0);
  CK(cudaMemsetAsync(p->d_flag, 0, sizeof(int), st));
  CK(cudaMemsetAsync(p->d_q[1], 0, sizeof(T) * p->lv[1].np, st));
  if (N > 0) {
    BinArgs<T> bg;
    for (int d = 0; d < 3; ++d) {
      bg.box.L[d] = (T)p->L[d];
      bg.box.invL[d] = (T)(1.0 / p->L[d]);
      bg.inv_w[d] = (T)p->cg.inv_w[d];
      bg.nc[d] = p->cg.nc[d];
    }
    const long ncell = p->cg.ncell;
    const long ntiles = cdiv(ncell, kScanTile);
    CK(cudaMemsetAsync(p->d_cell_count, 0, sizeof(int) * ncell, st));
    k_bin<T><<<cdiv(N, kBlock), kBlock, 0, st>>>(pos, cc, cc ? 3 : 4, N, bg, (Vec4<T>*)p->d_pos_w,
                                                p->d_cell_of, p->d_cell_count, p->d_flag);
    int* tsum = p->d_scan;
    k_scan_tiles<<<ntiles, kBlock, 0, st>>>(p->d_cell_count, ncell, tsum);
    k_scan_top<<<1, 32, 0, st>>>(tsum, (int)ntiles, p->d_cell_start, ncell);
    k_scan_final<<<ntiles, kBlock, 0, st>>>(p->d_cell_count, ncell, tsum, p->d_cell_start);
    k_scatter<T><<<cdiv(N, kBlock), kBlock, 0, st>>>((const Vec4<T>*)p->d_pos_w, p->d_cell_of, N,
                                                    p->d_cell_start, p->d_cell_count,
                                                    (Vec4<T>*)p->d_sorted, p->d_sorted_idx);
    k_cellsort<T><<<cdiv(ncell, kBlock), kBlock, 0, st>>>(p->d_cell_start, ncell,
                                                         (Vec4<T>*)p->d_sorted, p->d_sorted_idx);
    nl_ += 6;
    MARK(1);
    PairArgs<T> pg;
    for (int d = 0; d < 3; ++d) {
      pg.box.L[d] = (T)p->L[d];
      pg.box.invL[d] = (T)(1.0 / p->L[d]);
      pg.inv_w[d] = (T)p->cg.inv_w[d];
      pg.nc[d] = p->cg.nc[d];
      pg.R[d] = p->cg.R[d];
    }
    pg.a2 = (T)(p->a * p->a);
    pg.ia2 = (T)(1.0 / (p->a * p->a));
    pg.ia6 = (T)std::pow(p->a, -6.0);
    pg.ia8 = (T)std::pow(p->a, -8.0);
    double* wp_pair = p->d_wpart + 6 * p->wpart_pair;
    if (vir)
      k_pair<T, true><<<cdiv(N, kBlock), kBlock, 0, st>>>((const Vec4<T>*)p->d_sorted,
                                                          p->d_cell_start, N, pg, (T*)p->d_e0,
                                                          (T*)p->d_floc, wp_pair);
    else
      k_pair<T, false><<<cdiv(N, kBlock), kBlock, 0, st>>>((const Vec4<T>*)p->d_sorted,
                                                           p->d_cell_start, N, pg, (T*)p->d_e0,
                                                           (T*)p->d_floc, wp_pair);
    nl_ += 1;
    MARK(2);
    const Level& L1 = p->lv[1];
    k_anterp<T><<<cdiv(N, kBlock), kBlock, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, N, L1.n[0], L1.n[1], L1.n[2], (T)(1.0 / L1.h[0]),
        (T)(1.0 / L1.h[1]), (T)(1.0 / L1.h[2]), (T*)p->d_q[1]);
    nl_ += 1;
  } else {
    MARK(1);
    MARK(2);
  }
  MARK(3);
  // restriction
  for (int k = 1; k < l; ++k) {
    const Level &F = p->lv[k], &Cc = p->lv[k + 1];
    k_restrict<T><<<cdiv(Cc.np, kBlock), kBlock, 0, st>>>((const T*)p->d_q[k], F.n[0], F.n[1],
                                                         F.n[2], (T*)p->d_q[k + 1], Cc.n[0],
                                                         Cc.n[1], Cc.n[2]);
    nl_ += 1;
  }
  MARK(4);
  // level stencils
  for (int k = 1; k < l; ++k) {
    const Level& Lk = p->lv[k];
    long P = 1;
    for (int d = 0; d < 3; ++d) P *= Lk.n[d] + 2 * p->pad[d];
    k_pad<T><<<cdiv(P, kBlock), kBlock, 0, st>>>((const T*)p->d_q[k], Lk.n[0], Lk.n[1], Lk.n[2],
                                                p->pad[0], p->pad[1], p->pad[2], (T*)p->d_qpad);
    T scale = (T)std::ldexp(1.0, -6 * (k - 1));
    const int* toff = p->d_tap_off + (size_t)(k - 1) * p->ntaps;
    double* wp = p->d_wpart + 6 * p->wpart_lvl[k];
    if (vir)
      k_stencil<T, true><<<cdiv(Lk.np, kBlock), kBlock, 0, st>>>(
          (const T*)p->d_qpad, (const T*)p->d_q[k], Lk.n[0], Lk.n[1], Lk.n[2], p->pad[0],
          p->pad[1], p->pad[2], toff, (const T*)p->d_tap_g, (const T*)p->d_tap_v, p->ntaps, scale,
          (T*)p->d_e[k], wp);
    else
      k_stencil<T, false><<<cdiv(Lk.np, kBlock), kBlock, 0, st>>>(
          (const T*)p->d_qpad, (const T*)p->d_q[k], Lk.n[0], Lk.n[1], Lk.n[2], p->pad[0],
          p->pad[1], p->pad[2], toff, (const T*)p->d_tap_g, (const T*)p->d_tap_v, p->ntaps, scale,
          (T*)p->d_e[k], wp);
    nl_ += 2;
  }
  MARK(5);
  // coarsest level
  {
    const Level& Lt = p->lv[l];
    double* wp = p->d_wpart + 6 * p->wpart_top;
    if (vir)
      k_top<T, true><<<cdiv(Lt.np, kBlock), kBlock, 0, st>>>((const T*)p->d_q[l], Lt.n[0],
                                                             Lt.n[1], Lt.n[2], p->d_top_T,
                                                             p->d_top_V, (T*)p->d_e[l], wp);
    else
      k_top<T, false><<<cdiv(Lt.np, kBlock), kBlock, 0, st>>>((const T*)p->d_q[l], Lt.n[0],
                                                              Lt.n[1], Lt.n[2], p->d_top_T,
                                                              p->d_top_V, (T*)p->d_e[l], wp);
    nl_ += 1;
  }
  MARK(6);
  // prolongation
  for (int k = l - 1; k >= 1; --k) {
    const Level &F = p->lv[k], &Cc = p->lv[k + 1];
    k_prolong<T><<<cdiv(F.np, kBlock), kBlock, 0, st>>>((const T*)p->d_e[k], F.n[0], F.n[1],
                                                       F.n[2], (const T*)p->d_et[k + 1], Cc.n[0],
                                                       Cc.n[1], Cc.n[2], (T*)p->d_et[k]);
    nl_ += 1;
  }
  MARK(7);
  // interpolation, forces, per-atom energies
  if (N > 0) {
    const Level& L1 = p->lv[1];
    k_interp<T><<<cdiv(N, kBlock), kBlock, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_sorted_idx, N, (const T*)p->d_et[1], L1.n[0], L1.n[1],
        L1.n[2], (T)(1.0 / L1.h[0]), (T)(1.0 / L1.h[1]), (T)(1.0 / L1.h[2]), (const T*)p->d_e0,
        (const T*)p->d_floc, p->c_self, forces, atom_energy, p->d_epart);
    nl_ += 1;
  } else {
    // no atoms: every grid is zero; zero the atom-side partial sums
    CK(cudaMemsetAsync(p->d_epart, 0, sizeof(double) * p->n_epart, st));
    if (vir) CK(cudaMemsetAsync(p->d_wpart, 0, 6 * sizeof(double) * p->n_pair_blocks, st));
  }
  MARK(8);
  k_reduce<<<1, kBlock, 0, st>>>(p->d_epart, p->n_epart, p->d_wpart, p->n_wpart, vir ? 1 : 0,
                                 p->d_out);
  nl_ += 1;
  MARK(9);
#undef MARK
  p->launches = nl_;
  CK(cudaGetLastError());

  bool host_sync = false;
  if (energy) {
    if (is_device_ptr(energy)) {
      CK(cudaMemcpyAsync(energy, p->d_out, sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      host_sync = true;
    }
  }
  if (virial) {
    if (is_device_ptr(virial)) {
      CK(cudaMemcpyAsync(virial, p->d_out + 1, 6 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      host_sync = true;
    }
  }
  if (host_sync) {
    CK(cudaMemcpyAsync(p->h_out, p->d_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, st));
    int* h_flag = reinterpret_cast<int*>(p->h_out + 7);
    CK(cudaMemcpyAsync(h_flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (energy && !is_device_ptr(energy)) *energy = p->h_out[0];
    if (virial && !is_device_ptr(virial))
      for (int c = 0; c < 6; ++c) virial[c] = p->h_out[1 + c];
    if (*h_flag) return MLS6_ERR_NONFINITE;
  }
  return MLS6_OK;
}

int eval_launch(Plan* p, const void* pos, const void* c, void* forces, double* energy,
                double* virial, double* atom_energy) {
  return p->prec == MLS6_FP64 ? eval_t<double>(p, pos, c, forces, energy, virial, atom_energy)
                              : eval_t<float>(p, pos, c, forces, energy, virial, atom_energy);
}

}  // namespace mls6

using namespace mls6;

template <typename T> static int debug_grid_t(Plan* p, int level, int which, double* out) {
  const Level& Lk = p->lv[level];
  const void* src = which == 0 ? p->d_q[level] : which == 1 ? p->d_e[level] : p->d_et[level];
  std::vector<T> tmp((size_t)Lk.np);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MLS6_ERR_CUDA;
  if (cudaMemcpy(tmp.data(), src, sizeof(T) * Lk.np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MLS6_ERR_CUDA;
  for (long k = 0; k < Lk.np; ++k) out[k] = (double)tmp[k];
  return MLS6_OK;
}

static const char* kStageNames[Plan::kStages] = {
    "bin", "pair", "anterpolate", "restrict", "stencil", "coarsest", "prolongate", "interpolate",
    "reduce"};

extern "C" int mls6_profile(mls6_plan_t* plan, int enable) {
  if (!plan) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (enable && !p->ev[0])
    for (int i = 0; i <= Plan::kStages; ++i)
      if (cudaEventCreate(&p->ev[i]) != cudaSuccess) return MLS6_ERR_CUDA;
  p->prof = enable != 0;
  return MLS6_OK;
}

extern "C" int mls6_stage_times(mls6_plan_t* plan, double* ms, int cap, int* launches) {
  if (!plan) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (launches) *launches = p->launches;
  if (!p->ev[0]) return 0;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MLS6_ERR_CUDA;
  for (int i = 0; i < Plan::kStages && i < cap; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev[i], p->ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      t = -1.f;
    }
    if (ms) ms[i] = (double)t;
  }
  return Plan::kStages;
}

extern "C" const char* mls6_stage_name(int i) {
  return (i >= 0 && i < Plan::kStages) ? kStageNames[i] : nullptr;
}

extern "C" int mls6_debug_grid(mls6_plan_t* plan, int level, int which, double* host_out) {
  if (!plan || !host_out) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (level < 1 || level > p->levels || which < 0 || which > 2) return MLS6_ERR_ARG;
  return p->prec == MLS6_FP64 ? debug_grid_t<double>(p, level, which, host_out)
                              : debug_grid_t<float>(p, level, which, host_out);
}
