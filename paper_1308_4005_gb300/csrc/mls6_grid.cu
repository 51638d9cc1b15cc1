// Grid part of multilevel summation (Sec. II.B): anterpolation, restriction,
// evaluation on every level, prolongation and interpolation.
#include <algorithm>
#include <climits>
#include <cmath>

#include "mls6_device.cuh"

namespace mls6 {


// ------------------------------------------------------------ anterpolation

// (1/8) sqrt(binom(6, k)), the Lorentz-Berthelot expansion coefficient
// (Sec. II.D) of channel k.
__device__ __forceinline__ double lb_coef_d(int k) {
  const double b = (k == 0 || k == 6) ? 1.0 : (k == 1 || k == 5) ? 6.0 : (k == 2 || k == 4) ? 15.0
                                                                                           : 20.0;
  return 0.125 * sqrt(b);
}

// Fixed-point accumulation of the anterpolation: 32-bit integers for the
// FP32 modes (sums kept below 2^30), 64-bit for FP64 (below 2^61).  Each
// contribution is rounded to 2^(e-30) (FP32) or 2^(e-61) (FP64), where 2^e
// exceeds the worst-case node sum B of fixed_exponent; B is a conservative
// bound (most atoms in a cell x cells a support box meets x max |c|), so for
// FP32 the step is ~1e-6 of a typical node sum of order 1: tens of FP32
// rounding units per contribution, far below the FP32 path's force error
// but not below FP32 rounding (the bound is tested against the FP64 oracle
// on the 65,536-atom slab).  For FP64 it is ~1e-15 of a node sum.  The
// conversions stay in the kernel's own precision: FP64 arithmetic is slow on
// this GPU.
template <typename T> struct Fixed;
template <> struct Fixed<float> {
  using I = int;
  using U = unsigned int;
  static constexpr int kBits = 30;
  __device__ static float pow2(int s) { return __int_as_float((127 + s) << 23); }
  __device__ static I to_fixed(float v, float scale) { return __float2int_rn(v * scale); }
  __device__ static float from_fixed(I v, float iscale) { return (float)v * iscale; }
};
template <> struct Fixed<double> {
  using I = long long;
  using U = unsigned long long;
  static constexpr int kBits = 61;
  __device__ static double pow2(int s) { return __longlong_as_double((long long)(1023 + s) << 52); }
  __device__ static I to_fixed(double v, double scale) { return __double2ll_rn(v * scale); }
  __device__ static double from_fixed(I v, double iscale) { return (double)v * iscale; }
};

// Scale 2^s with s chosen so that no node sum can exceed 2^kBits in
// magnitude.  |Phi| <= 1, so a node receives at most |c| per atom within 2h
// of it (per axis; with periodic images), and those atoms lie in at most
// `span` cells (cells meeting a box of width 4h), each holding at most
// flag[3] atoms: bound = flag[3] * span * max|c|.
// Lorentz-Berthelot channel m (lbm >= 0): the coefficient is
// xi_m = lbc sigma^m sqrt(2 eps), bounded by lbc sigma_max^m (flag[4..5])
// times the largest sqrt(2 eps) (flag[6..7]).
template <typename T>
__device__ __forceinline__ int fixed_exponent(const int* __restrict__ flag, double span,
                                              int lbm = -1, double lbc = 0.0) {
  double cmax = *reinterpret_cast<const double*>(flag + 4);
  if (lbm >= 0) {
    double sm = 1.0;
    for (int k = 0; k < lbm; ++k) sm *= cmax;
    cmax = lbc * sm * *reinterpret_cast<const double*>(flag + 6);
  }
  const float bound = (float)((double)flag[3] * span * cmax * (1.0 + 1e-6));
  if (!(bound > 0.f)) return 0;
  int e;
  frexpf(bound, &e);  // bound < 2^e
  return min(max(Fixed<T>::kBits - e, -120), 120);
}

// Eq. (anterpolation): q^1_mu += c_j phi_mu(x_j) over the NP^3 nodes of
// every atom (NP = p + 1: 4x4x4 for the cubic, 6x6x6 for the quintic).  The contributions are rounded to the fixed-point grid 2^-s
// and added as integers (Fixed<T>): integer addition is associative, so the
// sums (and everything downstream) do not depend on the order in which the
// atomics land -- results are reproducible bit for bit.
// A block of kBlock cell-sorted atoms touches a compact box of grid nodes:
// when that box fits in shared memory the block first sums its
// contributions there (integer atomics on shared memory) and then adds each
// non-zero node once to the grid, which cuts the global atomics by the
// overlap of the atoms' supports; otherwise its atoms add to the grid
// directly.  Both paths add the same integers, so the grid does not depend
// on the path either.
constexpr int kAnterpBoxBytes = 24 * 1024;

template <typename T, int NP = 4>
__device__ __forceinline__ void k_anterp_body(const Blk bk,
    const Vec4<T>* __restrict__ sp, int N, int n0, int n1, int n2, T ih0, T ih1, T ih2,
    const int* __restrict__ flag, double span, typename Fixed<T>::U* __restrict__ qfx,
    const T* __restrict__ lbw, int lbm, double lbc) {
  using U = typename Fixed<T>::U;
  constexpr int kCap = kAnterpBoxBytes / (int)sizeof(U);
  __shared__ U box[kCap];
  __shared__ int lo[3], hi[3], sexp;
  const long z = pdl_begin();
  sp += z;
  flag += z;
  lbw += z;
  const int i = bk.x * blockDim.x + threadIdx.x;
  const bool valid = i < N;
  if (threadIdx.x < 3) {
    lo[threadIdx.x] = INT_MAX;
    hi[threadIdx.x] = INT_MIN;
  }
  if (threadIdx.x == 0) sexp = fixed_exponent<T>(flag, span, lbm, lbc);
  Vec4<T> p = valid ? sp[i] : Vec4<T>{T(0), T(0), T(0), T(0)};
  if (valid && lbm >= 0) {  // Lorentz-Berthelot channel: xi_m = lbc sigma^m sqrt(2 eps)
    T s = T(1);
    for (int k = 0; k < lbm; ++k) s *= p.w;
    p.w = (T)lbc * s * lbw[i];
  }
  const T u0 = p.x * ih0, u1 = p.y * ih1, u2 = p.z * ih2;
  const T f0 = floor(u0), f1 = floor(u1), f2 = floor(u2);
  const int b0 = (int)f0, b1 = (int)f1, b2 = (int)f2;
  __syncthreads();
  {  // bounding box of the block's supports (unwrapped node indices): warp
     // minima and maxima first, then one shared atomic per warp and axis
    int l0 = valid ? b0 - (NP / 2 - 1) : INT_MAX, l1 = valid ? b1 - (NP / 2 - 1) : INT_MAX;
    int l2 = valid ? b2 - (NP / 2 - 1) : INT_MAX;
    int h0 = valid ? b0 + NP / 2 : INT_MIN, h1 = valid ? b1 + NP / 2 : INT_MIN;
    int h2 = valid ? b2 + NP / 2 : INT_MIN;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      l0 = min(l0, __shfl_xor_sync(0xffffffffu, l0, o));
      l1 = min(l1, __shfl_xor_sync(0xffffffffu, l1, o));
      l2 = min(l2, __shfl_xor_sync(0xffffffffu, l2, o));
      h0 = max(h0, __shfl_xor_sync(0xffffffffu, h0, o));
      h1 = max(h1, __shfl_xor_sync(0xffffffffu, h1, o));
      h2 = max(h2, __shfl_xor_sync(0xffffffffu, h2, o));
    }
    if ((threadIdx.x & 31) == 0 && l0 != INT_MAX) {
      atomicMin(&lo[0], l0);
      atomicMin(&lo[1], l1);
      atomicMin(&lo[2], l2);
      atomicMax(&hi[0], h0);
      atomicMax(&hi[1], h1);
      atomicMax(&hi[2], h2);
    }
  }
  __syncthreads();
  const T scale = Fixed<T>::pow2(sexp);
  const int e0 = hi[0] - lo[0] + 1, e1 = hi[1] - lo[1] + 1, e2 = hi[2] - lo[2] + 1;
  const long vol = (long)e0 * e1 * e2;
  const bool in_box = hi[0] >= lo[0] && vol <= kCap;  // the same for the whole block
  if (in_box)
    for (int t = threadIdx.x; t < (int)vol; t += blockDim.x) box[t] = 0;
  __syncthreads();
  if (valid) {
    constexpr int B0 = NP / 2 - 1;  // first node of the support below base
    T wx[NP], wy[NP], wz[NP];
    phiw<NP>(u0 - f0, wx);
    phiw<NP>(u1 - f1, wy);
    phiw<NP>(u2 - f2, wz);
    if (in_box) {
      const int x0 = b0 - B0 - lo[0], y0 = b1 - B0 - lo[1], z0 = b2 - B0 - lo[2];
#pragma unroll
      for (int c = 0; c < NP; ++c)
#pragma unroll
        for (int b = 0; b < NP; ++b) {
          const T wyz = p.w * wy[b] * wz[c];
          const int row = e0 * ((y0 + b) + e1 * (z0 + c)) + x0;
#pragma unroll
          for (int a = 0; a < NP; ++a)
            atomicAdd(&box[row + a], (U)Fixed<T>::to_fixed(wyz * wx[a], scale));
        }
    } else {
      int ix[NP], iy[NP], iz[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        ix[k] = wrapi(b0 - B0 + k, n0);
        iy[k] = wrapi(b1 - B0 + k, n1);
        iz[k] = wrapi(b2 - B0 + k, n2);
      }
#pragma unroll
      for (int c = 0; c < NP; ++c)
#pragma unroll
        for (int b = 0; b < NP; ++b) {
          const T wyz = p.w * wy[b] * wz[c];
          const long rowi = (long)n0 * (iy[b] + (long)n1 * iz[c]);
#pragma unroll
          for (int a = 0; a < NP; ++a)
            atomicAdd(&qfx[rowi + ix[a]], (U)Fixed<T>::to_fixed(wyz * wx[a], scale));
        }
    }
  }
  if (in_box) {  // flush: one warp per box row (y, z), lanes along x
    __syncthreads();
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < e1 * e2; r += nw) {
      const int y = wrapi(lo[1] + r % e1, n1), zz = wrapi(lo[2] + r / e1, n2);
      const long row = (long)n0 * (y + (long)n1 * zz);
      const U* br = box + (size_t)r * e0;
      for (int x = lane; x < e0; x += 32) {
        const U v = br[x];
        if (v == 0) continue;
        atomicAdd(&qfx[row + wrapi(lo[0] + x, n0)], v);
      }
    }
  }
}

template <typename T, int NP>
__global__ void __launch_bounds__(kBlock) k_anterp(
    const Vec4<T>* __restrict__ sp, int N, int n0, int n1, int n2, T ih0, T ih1, T ih2,
    const int* __restrict__ flag, double span, typename Fixed<T>::U* __restrict__ qfx,
    const T* __restrict__ lbw, int lbm, double lbc) {
  k_anterp_body<T, NP>(Blk::self(), sp, N, n0, n1, n2, ih0, ih1, ih2, flag, span, qfx, lbw, lbm, lbc);
}

// q^1 = fixed-point sums * 2^-s in the plan's precision.
template <typename T>
__device__ __forceinline__ void k_from_fixed_body(const Blk bk,const typename Fixed<T>::U* __restrict__ qfx, long np,
                             const int* __restrict__ flag, double span, T* __restrict__ q,
                             int lbm, double lbc) {
  __shared__ int sexp;
  const long z = pdl_begin();
  qfx += z; flag += z;
  if (threadIdx.x == 0) sexp = fixed_exponent<T>(flag, span, lbm, lbc);
  __syncthreads();
  const long i = (long)bk.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  q[i] = Fixed<T>::from_fixed((typename Fixed<T>::I)qfx[i], Fixed<T>::pow2(-sexp));
}

template <typename T>
__global__ void k_from_fixed(const typename Fixed<T>::U* __restrict__ qfx, long np,
                             const int* __restrict__ flag, double span, T* __restrict__ q,
                             int lbm, double lbc) {
  k_from_fixed_body<T>(Blk::self(), qfx, np, flag, span, q, lbm, lbc);
}

// Cells (with periodic images) that the support of one node's basis
// function (width (p + 1) h) can meet, product over the axes.
static double support_span(const Plan* p) {
  double s = 1.0;
  const double width = p->order + 1.0;
  for (int d = 0; d < 3; ++d) s *= std::ceil(width * p->lv[1].h[d] / p->cg.w[d]) + 1.0;
  return s;
}

// lbm >= 0: Lorentz-Berthelot channel m (coefficients computed from the
// sorted sigma and sqrt(2 eps)); -1: the atoms' own coefficients.
#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
double lb_coef(int m) {
  static const double binom[7] = {1, 6, 15, 20, 15, 6, 1};
  return m < 0 ? 0.0 : 0.125 * std::sqrt(binom[m]);
}
#endif  // MLS6_DEVICE_ONLY

template <typename T> int launch_anterp(Plan* p, cudaStream_t st, int lbm) {
  const Level& L1 = p->lv[1];
  const int N = (int)p->N;
  const double span = support_span(p);
  const double lbc = lb_coef(lbm);
  launch_pdl(p->order == 5 ? k_anterp<T, 6> : k_anterp<T, 4>, cdiv(N, kBlock), kBlock, 0, st,
      (const Vec4<T>*)p->d_sorted, N, L1.n[0], L1.n[1], L1.n[2], (T)(1.0 / L1.h[0]),
      (T)(1.0 / L1.h[1]), (T)(1.0 / L1.h[2]), p->d_flag, span,
      (typename Fixed<T>::U*)p->d_q1fx, (const T*)p->d_lbw, lbm, lbc);
  launch_pdl(k_from_fixed<T>, cdiv(L1.np, kBlock), kBlock, 0, st, 
      (const typename Fixed<T>::U*)p->d_q1fx, L1.np, p->d_flag, span, (T*)p->d_q[1], lbm, lbc);
  return 2;
}

// sqrt(2 eps) of the atoms in sorted order, and its largest value
// (flag[6..7] as a double; one atomic per block on the value's bits, which
// order like the integers for non-negative doubles).
template <typename T>
__global__ void k_lb_weights(const T* __restrict__ eps, const int* __restrict__ sidx, int N,
                             T* __restrict__ lbw, int* __restrict__ flag) {
  const long z = pdl_begin();
  eps += z; sidx += z;
  __shared__ double wmax[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (i < N) {
    const T e = eps[sidx[i]];
    const T w = sqrt(T(2) * (e > T(0) ? e : T(0)));
    lbw[i] = w;
    m = (double)w;
    if (!isfinite(m)) atomicOr(flag, 1);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
    atomicMax(reinterpret_cast<unsigned long long*>(flag + 6),
              (unsigned long long)__double_as_longlong(m));
  }
}

template <typename T> int launch_lb_weights(Plan* p, const T* eps, cudaStream_t st) {
  const int N = (int)p->N;
  launch_pdl(k_lb_weights<T>, cdiv(N, kBlock), kBlock, 0, st, eps, p->d_sorted_idx, N, (T*)p->d_lbw,
                                                     p->d_flag);
  return 1;
}

// -------------------------------------------------------------- restriction

// q^{k+1}_mu = sum_nu prod_d Phi(nu_d/2 - mu_d) q^k_nu; the nonzero weights
// are Phi(0)=1 at fine offset 0 from 2 mu and Phi(1/2), Phi(3/2) (and, for
// the quintic, Phi(5/2)) at offsets +-1, +-3 (+-5): 9/16, -1/16 for the
// cubic, 150/256, -25/256, 3/256 for the quintic.
template <typename T, int NP = 4>
__device__ __forceinline__ void k_restrict_body(const Blk bk,const T* __restrict__ qf, int f0, int f1, int f2, T* __restrict__ qc,
                           int c0, int c1, int c2) {
  const long z = pdl_begin();
  qf += z;
  const long mu = (long)bk.x * blockDim.x + threadIdx.x;
  const long np = (long)c0 * c1 * c2;
  if (mu >= np) return;
  const unsigned u = (unsigned)mu, uc0 = (unsigned)c0, uc1 = (unsigned)c1;  // grids < 2^31 nodes
  const unsigned q0 = u / uc0;
  const int m0 = (int)(u - q0 * uc0), m1 = (int)(q0 % uc1), m2 = (int)(q0 / uc1);
  constexpr int NT = NP + 1, H = NP / 2;  // taps per axis, nonzero half-integer weights
  int off[NT];
  T wt[NT];
#pragma unroll
  for (int k = 0; k < H; ++k) {  // offsets -(2H-1) .. -1 and 1 .. 2H-1
    off[k] = -(2 * (H - 1 - k) + 1);
    wt[k] = half_weight<NP, T>(H - 1 - k);
    off[NT - 1 - k] = -off[k];
    wt[NT - 1 - k] = wt[k];
  }
  off[H] = 0;
  wt[H] = T(1);
  int ix[NT], iy[NT], iz[NT];  // wrapped fine indices per axis
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    ix[k] = wrapi(2 * m0 + off[k], f0);
    iy[k] = wrapi(2 * m1 + off[k], f1);
    iz[k] = wrapi(2 * m2 + off[k], f2);
  }
  T acc = 0;
#pragma unroll
  for (int c = 0; c < NT; ++c) {
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      const T* row = qf + (size_t)f0 * (iy[b] + (size_t)f1 * iz[c]);
      T s = 0;
#pragma unroll
      for (int a = 0; a < NT; ++a) s += wt[a] * row[ix[a]];
      acc += (wt[b] * wt[c]) * s;
    }
  }
  qc[mu] = acc;
}

template <typename T, int NP>
__global__ void k_restrict(const T* __restrict__ qf, int f0, int f1, int f2, T* __restrict__ qc,
                           int c0, int c1, int c2) {
  k_restrict_body<T, NP>(Blk::self(), qf, f0, f1, f2, qc, c0, c1, c2);
}

template <typename T> int launch_restrict(Plan* p, int k, cudaStream_t st) {
  const Level &F = p->lv[k], &C = p->lv[k + 1];
  launch_pdl(p->order == 5 ? k_restrict<T, 6> : k_restrict<T, 4>, cdiv(C.np, kBlock), kBlock, 0, st, (const T*)p->d_q[k], F.n[0], F.n[1],
                                                      F.n[2], (T*)p->d_q[k + 1], C.n[0], C.n[1],
                                                      C.n[2]);
  return 1;
}

// ------------------------------------------------------- level stencils

template <typename T> struct StencilLevel {
  const T* q;
  T* e;
  int n[3];
  int tiles[3];
  long tile_off;
  T scale;  // 2^(-6(k-1))
};

template <typename T> struct StencilArgs {
  StencilLevel<T> lv[kMaxLevels];
  int nlev, P, S, nrows, ntaps;
  int Sx, Sp;           // padded row and plane pitch of the staged tile
  const int4* rows;     // dy, dz, R, first tap
  const Vec4<T>* wv;    // g_1, G, G dx, G dx^2 per tap
  double hc[6];         // h_x^2, h_y^2, h_z^2, h_x h_y, h_x h_z, h_y h_z (level 1)
  // coarsest level, run by the blocks after the stencil tiles (if any)
  long sblocks;         // number of stencil-tile blocks
  const T* qt;
  T* et;
  int nt[3];
  const double* tT;
  const double* tV;
  double* wtop;         // virial partials, one record per coarsest node
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Pitches of the staged S^3 tile: a warp reads 8 y-rows x 4 z-planes at one
// x offset, so an odd row pitch and a plane pitch of 8 mod 16 put its 32
// lanes in 32 different shared-memory banks (for 8-byte values, 16 lanes
// per half-warp in 16 bank pairs).
inline void stencil_pitches(int S, int& Sx, int& Sp) {
  Sx = S | 1;
  Sp = S * Sx;
  while (Sp % 16 != 8) ++Sp;
}

// Eq. (evaluation) on all levels k < l in one launch.  Block = one 8x8x8
// output tile of one level; the tile plus a halo of P nodes (periodic) is
// staged in shared memory together with the tap table.  Each thread owns
// 4 consecutive x nodes and slides a 4-wide register window along every tap
// row (constant dy, dz).  The strain derivative is accumulated per row from
// three row sums of the node/neighbour products (taps G, G dx, G dx^2), so
// the six virial components cost 7 FMAs per tap and thread instead of 24.
// With G > 1, G groups of 128 threads share a tile and each takes every
// G-th tap row (more resident warps for small grids); the groups' partial
// outputs are added in shared memory, their virial terms in the block sum.
template <typename T, bool VIR, int G>
__device__ __forceinline__ void k_stencil_body(const Blk bk, const StencilArgs<T>& A,
                                                                 double* __restrict__ wpart) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32 * 7];
  __shared__ T part[(G > 1 ? G - 1 : 1) * kStencilThreads * kStencilW];
  if ((long)bk.x >= A.sblocks) {  // coarsest level: one warp per node
    const int mu = (int)((long)bk.x - A.sblocks) * (int)(blockDim.x >> 5) +
                   (int)(threadIdx.x >> 5);
    if (mu < A.nt[0] * A.nt[1] * A.nt[2])
      coarsest_node<T, VIR>(A.qt, A.nt[0], A.nt[1], A.nt[2], A.tT, A.tV, A.et, A.wtop, mu);
    return;
  }
  const int S = A.S, P = A.P, S2 = S * S, S3 = S2 * S, Sx = A.Sx, Sp = A.Sp;
  T* tile = reinterpret_cast<T*>(smem_raw);
  Vec4<T>* wv = reinterpret_cast<Vec4<T>*>(smem_raw + align16(sizeof(T) * S * Sp));
  int4* rows = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(wv) +
                                       sizeof(Vec4<T>) * A.ntaps);
  const long b = bk.x;
  int k = 0;
  while (k + 1 < A.nlev && b >= A.lv[k + 1].tile_off) ++k;
  const T* __restrict__ q = A.lv[k].q;
  const int n0 = A.lv[k].n[0], n1 = A.lv[k].n[1], n2 = A.lv[k].n[2];
  const long t = b - A.lv[k].tile_off;
  const int tx = (int)(t % A.lv[k].tiles[0]);
  const int ty = (int)((t / A.lv[k].tiles[0]) % A.lv[k].tiles[1]);
  const int tz = (int)(t / ((long)A.lv[k].tiles[0] * A.lv[k].tiles[1]));
  const int ox = tx * kStencilTile, oy = ty * kStencilTile, oz = tz * kStencilTile;

  for (int i = threadIdx.x; i < A.ntaps; i += blockDim.x) wv[i] = A.wv[i];
  for (int i = threadIdx.x; i < A.nrows; i += blockDim.x) rows[i] = A.rows[i];
  for (int i = threadIdx.x; i < S3; i += blockDim.x) {
    int ix = i % S, iy = (i / S) % S, iz = i / S2;
    int gx = wrapi(ox + ix - P, n0), gy = wrapi(oy + iy - P, n1), gz = wrapi(oz + iz - P, n2);
    tile[iz * Sp + iy * Sx + ix] = q[gx + (long)n0 * (gy + (long)n1 * gz)];
  }
  __syncthreads();

  const int lt = threadIdx.x % kStencilThreads, grp = threadIdx.x / kStencilThreads;
  // a warp: 8 y-rows x 4 z-planes at one x offset (conflict-free pitches)
  const int lx = ((lt >> 6) & 1) * kStencilW, ly = lt & 7, lz = (lt >> 3) & 7;
  const bool row_in = (oy + ly < n1) && (oz + lz < n2);
  T qv[kStencilW];
#pragma unroll
  for (int w = 0; w < kStencilW; ++w)
    qv[w] = (row_in && ox + lx + w < n0) ? tile[(lz + P) * Sp + (ly + P) * Sx + lx + P + w] : T(0);
  T acc[kStencilW];
#pragma unroll
  for (int w = 0; w < kStencilW; ++w) acc[w] = T(0);
  T vxx = 0, vyy = 0, vzz = 0, vxy = 0, vxz = 0, vyz = 0;
  for (int r = grp; r < A.nrows; r += G) {
    const int4 ri = rows[r];
    const T* in = tile + (lz + P + ri.y) * Sp + (ly + P + ri.x) * Sx + (lx + P - ri.z);
    const Vec4<T>* ww = wv + ri.w;
    const int nd = 2 * ri.z + 1;
    T b0 = in[0], b1 = in[1], b2 = in[2];
    T s0 = 0, s1 = 0, s2 = 0;
    for (int d = 0; d < nd; ++d) {
      const T b3 = in[d + 3];
      const Vec4<T> wt = ww[d];
      acc[0] += wt.x * b0;
      acc[1] += wt.x * b1;
      acc[2] += wt.x * b2;
      acc[3] += wt.x * b3;
      if (VIR) {
        const T cd = qv[0] * b0 + qv[1] * b1 + qv[2] * b2 + qv[3] * b3;
        s0 += wt.y * cd;
        s1 += wt.z * cd;
        s2 += wt.w * cd;
      }
      b0 = b1;
      b1 = b2;
      b2 = b3;
    }
    if (VIR) {
      const T dy = (T)ri.x, dz = (T)ri.y;
      vxx += s2;
      vyy += dy * dy * s0;
      vzz += dz * dz * s0;
      vxy += dy * s1;
      vxz += dz * s1;
      vyz += dy * dz * s0;
    }
  }
  const T scale = A.lv[k].scale;
  if (G > 1) {
    if (grp > 0)
#pragma unroll
      for (int w = 0; w < kStencilW; ++w)
        part[((grp - 1) * kStencilThreads + lt) * kStencilW + w] = acc[w];
    __syncthreads();
    if (grp == 0)
      for (int g2 = 1; g2 < G; ++g2)
#pragma unroll
        for (int w = 0; w < kStencilW; ++w)
          acc[w] += part[((g2 - 1) * kStencilThreads + lt) * kStencilW + w];
  }
  if (row_in && grp == 0) {
    T* e = A.lv[k].e + (ox + lx) + (long)n0 * ((oy + ly) + (long)n1 * (oz + lz));
#pragma unroll
    for (int w = 0; w < kStencilW; ++w)
      if (ox + lx + w < n0) e[w] = scale * acc[w];
  }
  if (VIR) {
    T v6[6] = {vxx, vyy, vzz, vxy, vxz, vyz};
    double w6[6];
    block_sum_lo<T, 6>(v6, w6, red);
    if (threadIdx.x == 0) {
      const double hs = 0.5 * (double)scale;
      for (int c = 0; c < 6; ++c) wpart[6 * b + c] = hs * A.hc[c] * w6[c];
    }
  }
}

template <typename T, bool VIR, int G>
__global__ void __launch_bounds__(kStencilThreads * G) k_stencil(StencilArgs<T> A,
                                                                 double* __restrict__ wpart) {
  k_stencil_body<T, VIR, G>(Blk::self(), A, wpart);
}

// Same evaluation without shared-memory staging, for stencils whose tile
// and tap table exceed the shared-memory budget (large 2a/h): one thread per
// node, periodic indices, taps read from global memory (warp-uniform).
template <typename T, bool VIR>
__global__ void __launch_bounds__(kBlock) k_stencil_global(StencilArgs<T> A,
                                                           double* __restrict__ wpart,
                                                           long nodes_total) {
  pdl_begin();
  __shared__ double red[32 * 6];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  // level of this node (levels are concatenated)
  long off = 0;
  int k = 0;
  for (; k < A.nlev; ++k) {
    long np = (long)A.lv[k].n[0] * A.lv[k].n[1] * A.lv[k].n[2];
    if (gid < off + np) break;
    off += np;
  }
  T acc = 0, vxx = 0, vyy = 0, vzz = 0, vxy = 0, vxz = 0, vyz = 0, qmu = 0;
  T scale = 0;
  if (gid < nodes_total) {
    const T* __restrict__ q = A.lv[k].q;
    const int n0 = A.lv[k].n[0], n1 = A.lv[k].n[1], n2 = A.lv[k].n[2];
    const long mu = gid - off;
    const int x = (int)(mu % n0), y = (int)((mu / n0) % n1), z = (int)(mu / ((long)n0 * n1));
    qmu = q[mu];
    for (int r = 0; r < A.nrows; ++r) {
      const int4 ri = A.rows[r];
      const long rowb = (long)n0 * (wrapi(y + ri.x, n1) + (long)n1 * wrapi(z + ri.y, n2));
      T s0 = 0, s1 = 0, s2 = 0;
      for (int d = 0; d <= 2 * ri.z; ++d) {
        const T v = q[rowb + wrapi(x + d - ri.z, n0)];
        const Vec4<T> wt = A.wv[ri.w + d];
        acc += wt.x * v;
        if (VIR) {
          s0 += wt.y * v;
          s1 += wt.z * v;
          s2 += wt.w * v;
        }
      }
      if (VIR) {
        const T dy = (T)ri.x, dz = (T)ri.y;
        vxx += qmu * s2;
        vyy += qmu * dy * dy * s0;
        vzz += qmu * dz * dz * s0;
        vxy += qmu * dy * s1;
        vxz += qmu * dz * s1;
        vyz += qmu * dy * dz * s0;
      }
    }
    scale = A.lv[k].scale;
    A.lv[k].e[mu] = scale * acc;
  }
  if (VIR) {
    // all nodes of a block are on one level unless the block straddles two;
    // fold the level scale per thread (exact power of two) before summing
    T v6[6] = {scale * vxx, scale * vyy, scale * vzz, scale * vxy, scale * vxz, scale * vyz};
    double w6[6];
    block_sum_lo<T, 6>(v6, w6, red);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) wpart[6 * (size_t)blockIdx.x + c] = 0.5 * A.hc[c] * w6[c];
  }
}

template <typename T> static StencilArgs<T> stencil_args(Plan* p) {
  StencilArgs<T> A;
  A.nlev = p->levels - 1;
  A.P = p->P;
  A.S = kStencilTile + 2 * p->P;
  stencil_pitches(A.S, A.Sx, A.Sp);
  A.nrows = p->nrows;
  A.ntaps = p->ntaps;
  A.rows = reinterpret_cast<const int4*>(p->d_rows);
  A.wv = reinterpret_cast<const Vec4<T>*>(p->d_wv);
  const double* h = p->lv[1].h;
  A.hc[0] = h[0] * h[0];
  A.hc[1] = h[1] * h[1];
  A.hc[2] = h[2] * h[2];
  A.hc[3] = h[0] * h[1];
  A.hc[4] = h[0] * h[2];
  A.hc[5] = h[1] * h[2];
  for (int k = 1; k < p->levels; ++k) {
    StencilLevel<T>& L = A.lv[k - 1];
    L.q = (const T*)p->d_q[k];
    L.e = (T*)p->d_e[k];
    for (int d = 0; d < 3; ++d) {
      L.n[d] = p->lv[k].n[d];
      L.tiles[d] = p->tiles[k][d];
    }
    L.tile_off = p->tile_off[k];
    L.scale = (T)std::ldexp(1.0, -6 * (k - 1));
  }
  const int l = p->levels;
  A.sblocks = p->stencil_blocks;
  A.qt = (const T*)p->d_q[l];
  A.et = (T*)p->d_e[l];
  for (int d = 0; d < 3; ++d) A.nt[d] = p->lv[l].n[d];
  A.tT = p->d_top_T;
  A.tV = p->d_top_V;
  A.wtop = p->d_wpart + 6 * p->wpart_top;
  return A;
}

// Whether the coarsest level rides on the stencil launch (extra blocks).
#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
bool stencil_fuses_top(const Plan* p) { return p->levels >= 2 && !p->stencil_global && !p->prof; }
#endif  // MLS6_DEVICE_ONLY

template <typename T> int launch_stencil(Plan* p, bool vir, cudaStream_t st) {
  if (p->levels < 2) return 0;
  if (p->stencil_mma) return launch_stencil_mma(p, vir, stencil_fuses_top(p), st);
  if (p->stencil_tc) return launch_stencil_tc(p, vir, stencil_fuses_top(p), st);
  StencilArgs<T> A = stencil_args<T>(p);
  double* wp = p->d_wpart + 6 * p->wpart_stencil;
  if (p->stencil_global) {
    long nodes = 0;
    for (int k = 1; k < p->levels; ++k) nodes += p->lv[k].np;
    if (vir)
      launch_pdl(k_stencil_global<T, true>, p->stencil_blocks, kBlock, 0, st, A, wp, nodes);
    else
      launch_pdl(k_stencil_global<T, false>, p->stencil_blocks, kBlock, 0, st, A, wp, nodes);
    return 1;
  }
  const int warps = kStencilThreads * p->stencil_groups / 32;
  const long nb = p->stencil_blocks +
                  (stencil_fuses_top(p) ? cdiv(p->lv[p->levels].np, warps) : 0);
  const size_t sm = p->stencil_smem;
  switch (p->stencil_groups * 2 + (vir ? 1 : 0)) {
    case 2 * 4 + 1: launch_pdl(k_stencil<T, true, 4>, nb, kStencilThreads * 4, sm, st, A, wp); break;
    case 2 * 4 + 0: launch_pdl(k_stencil<T, false, 4>, nb, kStencilThreads * 4, sm, st, A, wp); break;
    case 2 * 2 + 1: launch_pdl(k_stencil<T, true, 2>, nb, kStencilThreads * 2, sm, st, A, wp); break;
    case 2 * 2 + 0: launch_pdl(k_stencil<T, false, 2>, nb, kStencilThreads * 2, sm, st, A, wp); break;
    case 2 * 1 + 1: launch_pdl(k_stencil<T, true, 1>, nb, kStencilThreads, sm, st, A, wp); break;
    default: launch_pdl(k_stencil<T, false, 1>, nb, kStencilThreads, sm, st, A, wp); break;
  }
  return 1;
}

// ------------------------------------------------------------ coarsest level

// Coarsest level on its own launch: one warp per node, 4 warps per block.
template <typename T, bool VIR>
__global__ void __launch_bounds__(128) k_top(const T* __restrict__ q, int n0, int n1, int n2,
                                             const double* __restrict__ tT,
                                             const double* __restrict__ tV, T* __restrict__ e,
                                             double* __restrict__ wpart) {
  const long z = pdl_begin();
  q += z; tT += z; tV += z;
  const int mu = (int)blockIdx.x * 4 + (int)(threadIdx.x >> 5);
  if (mu < n0 * n1 * n2) coarsest_node<T, VIR>(q, n0, n1, n2, tT, tV, e, wpart, mu);
}

template <typename T> int launch_top(Plan* p, bool vir, cudaStream_t st) {
  if (stencil_fuses_top(p)) return 0;  // ran as extra blocks of the stencil launch
  const int l = p->levels;
  const Level& Lt = p->lv[l];
  double* wp = p->d_wpart + 6 * p->wpart_top;
  if (vir)
    launch_pdl(k_top<T, true>, cdiv(Lt.np, 4), 128, 0, st, (const T*)p->d_q[l], Lt.n[0], Lt.n[1], Lt.n[2],
                                          p->d_top_T, p->d_top_V, (T*)p->d_e[l], wp);
  else
    launch_pdl(k_top<T, false>, cdiv(Lt.np, 4), 128, 0, st, (const T*)p->d_q[l], Lt.n[0], Lt.n[1], Lt.n[2],
                                           p->d_top_T, p->d_top_V, (T*)p->d_e[l], wp);
  return 1;
}

// -------------------------------------------------------------- prolongation

// e^{k,tot}_mu = e^k_mu + sum_nu prod_d Phi(mu_d/2 - nu_d) e^{k+1,tot}_nu.
// Per axis an even fine index meets one coarse node (weight 1), an odd one
// the NP coarse nodes around it (weights Phi at half-integers).
template <typename T, int NP>
__device__ __forceinline__ int prolong_axis(int m, int nc, int (&idx)[NP], T (&wt)[NP]) {
  constexpr int H = NP / 2;
  if ((m & 1) == 0) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      idx[k] = wrapi(m >> 1, nc);
      wt[k] = k == 0 ? T(1) : T(0);
    }
    return 1;
  }
  const int h = (m - 1) >> 1;  // coarse node left of m
#pragma unroll
  for (int k = 0; k < NP; ++k) {  // coarse nodes h - (H-1) .. h + H
    idx[k] = wrapi(h - (H - 1) + k, nc);
    wt[k] = half_weight<NP, T>(k < H ? H - 1 - k : k - H);
  }
  return NP;
}

template <typename T, int NP = 4>
__device__ __forceinline__ void k_prolong_body(const Blk bk,const T* __restrict__ ef, int f0, int f1, int f2,
                          const T* __restrict__ etc_, int c0, int c1, int c2,
                          T* __restrict__ etf) {
  const long z = pdl_begin();
  ef += z; etc_ += z;
  const long mu = (long)bk.x * blockDim.x + threadIdx.x;
  const long np = (long)f0 * f1 * f2;
  if (mu >= np) return;
  const unsigned u = (unsigned)mu, uf0 = (unsigned)f0, uf1 = (unsigned)f1;  // grids < 2^31 nodes
  const unsigned q0 = u / uf0;
  int ix[NP], iy[NP], iz[NP];
  T wx[NP], wy[NP], wz[NP];
  const int nx = prolong_axis<T, NP>((int)(u - q0 * uf0), c0, ix, wx);
  const int ny = prolong_axis<T, NP>((int)(q0 % uf1), c1, iy, wy);
  const int nz = prolong_axis<T, NP>((int)(q0 / uf1), c2, iz, wz);
  T acc = 0;
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    if (c >= nz) break;
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      if (b >= ny) break;
      const T* row = etc_ + (size_t)c0 * (iy[b] + (size_t)c1 * iz[c]);
      T s = 0;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        if (a >= nx) break;
        s += wx[a] * row[ix[a]];
      }
      acc += wy[b] * wz[c] * s;
    }
  }
  etf[mu] = ef[mu] + acc;
}

template <typename T, int NP>
__global__ void k_prolong(const T* __restrict__ ef, int f0, int f1, int f2,
                          const T* __restrict__ etc_, int c0, int c1, int c2,
                          T* __restrict__ etf) {
  k_prolong_body<T, NP>(Blk::self(), ef, f0, f1, f2, etc_, c0, c1, c2, etf);
}

template <typename T> int launch_prolong(Plan* p, int k, cudaStream_t st) {
  const Level &F = p->lv[k], &C = p->lv[k + 1];
  launch_pdl(p->order == 5 ? k_prolong<T, 6> : k_prolong<T, 4>, cdiv(F.np, kBlock), kBlock, 0, st, (const T*)p->d_e[k], F.n[0], F.n[1],
                                                     F.n[2], (const T*)p->d_et[k + 1], C.n[0],
                                                     C.n[1], C.n[2], (T*)p->d_et[k]);
  return 1;
}

// ------------------------------------------------------------- interpolation

// Eq. (interpolation) and its gradient: e_i = sum phi e^{1,tot},
// F_i = F_i^loc + c_i grad e_i; per-atom energy
// -1/2 c_i (e0_i + e_i) + 1/2 c_self c_i^2; one energy partial per block.
// The last block to finish (ticket counter, reset by that block) sums all
// energy and virial partials in a fixed order into out[0..6].
struct ReduceArgs {
  const double* wpart;
  long nw;
  int vir;
  double* out;
  unsigned* ticket;
  double* gsum;  // ng slice sums of the virial records (6 doubles each)
  int ng;
};

template <typename T, bool SLICES, int NP = 4>
__device__ __forceinline__ void k_interp_body(const Blk bk,
    const Vec4<T>* __restrict__ sp, const int* __restrict__ sidx, int N, const T* __restrict__ et,
    int n0, int n1, int n2, T ih0, T ih1, T ih2, const T* __restrict__ e0,
    const T* __restrict__ floc, double cself, T* __restrict__ forces,
    double* __restrict__ atom_energy, double* __restrict__ epart, ReduceArgs R) {
  const long z = pdl_begin();
  sp += z; sidx += z; et += z; e0 += z; floc += z;
  __shared__ double sh[32 * 7];
  __shared__ bool last;
  int i = bk.x * blockDim.x + threadIdx.x;
  T ea = T(0);
  if (i < N) {
    Vec4<T> p = sp[i];
    T u0 = p.x * ih0, u1 = p.y * ih1, u2 = p.z * ih2;
    T f0 = floor(u0), f1 = floor(u1), f2 = floor(u2);
    int b0 = (int)f0, b1 = (int)f1, b2 = (int)f2;
    constexpr int B0 = NP / 2 - 1;
    T wx[NP], wy[NP], wz[NP], dx[NP], dy[NP], dz[NP];
    phid<NP>(u0 - f0, wx, dx);
    phid<NP>(u1 - f1, wy, dy);
    phid<NP>(u2 - f2, wz, dz);
    int ix[NP], iy[NP], iz[NP];  // wrapped node indices per axis
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      ix[k] = wrapi(b0 - B0 + k, n0);
      iy[k] = wrapi(b1 - B0 + k, n1);
      iz[k] = wrapi(b2 - B0 + k, n2);
    }
    T acc = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
#pragma unroll
      for (int b = 0; b < NP; ++b) {
        const T* row = et + (long)n0 * (iy[b] + (long)n1 * iz[c]);
        T sx = 0, sdx = 0;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
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
    ea = T(-0.5) * ci * (e0[i] + acc) + T(0.5 * cself) * ci * ci;
    if (atom_energy) atom_energy[o] = (double)ea;
  }
  // block sum in the kernel's precision, promoted per warp (FP64 is slow)
  T ev[1] = {ea};
  double s[1];
  block_sum_lo<T, 1>(ev, s, sh);
  // With several waves of blocks, warp 0 of each of the first ng blocks sums
  // one contiguous slice of the virial records (fixed order) and the last
  // block adds the ng slice sums instead of every record (one block summing
  // ~7,600 records in FP64 took 22 us on a 1M-atom cube).  In a single wave
  // the slices would lengthen the kernel instead, and ng is 0.
  if (SLICES && R.vir && (int)bk.x < R.ng && threadIdx.x < 32) {
    const long per = (R.nw + R.ng - 1) / R.ng, k0 = (long)bk.x * per;
    const long k1 = min(R.nw, k0 + per);
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long k = k0 + threadIdx.x; k < k1; k += 32)
#pragma unroll
      for (int c = 0; c < 6; ++c) v[c] += R.wpart[6 * k + c];
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] = warp_sum(v[c]);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) R.gsum[6 * bk.x + c] = v[c];
  }
  if (threadIdx.x == 0) {
    epart[bk.x] = s[0];
    __threadfence();
    last = atomicAdd(R.ticket, 1u) == bk.n - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (SLICES)
      final_reduce(epart, bk.n, R.gsum, R.ng, R.vir, R.out, sh);
    else
      final_reduce(epart, bk.n, R.wpart, R.nw, R.vir, R.out, sh);
    if (threadIdx.x == 0) *R.ticket = 0u;
  }
}

template <typename T, bool SLICES, int NP>
__global__ void __launch_bounds__(kBlock) k_interp(
    const Vec4<T>* __restrict__ sp, const int* __restrict__ sidx, int N, const T* __restrict__ et,
    int n0, int n1, int n2, T ih0, T ih1, T ih2, const T* __restrict__ e0,
    const T* __restrict__ floc, double cself, T* __restrict__ forces,
    double* __restrict__ atom_energy, double* __restrict__ epart, ReduceArgs R) {
  k_interp_body<T, SLICES, NP>(Blk::self(), sp, sidx, N, et, n0, n1, n2, ih0, ih1, ih2, e0, floc, cself, forces, atom_energy, epart, R);
}

// Lorentz-Berthelot interpolation: the seven channel potentials e^{(m),tot}
// (level 1) are combined per node with the atom's xi_{i,6-m} before the
// basis sum (both linear): e_i = sum_m xi_{i,6-m} e^{(m)}(x_i) and
// F_i = F_i^loc + sum_m xi_{i,6-m} grad e^{(m)}(x_i); per-atom energy
// -1/2 (e0_i + e_i) + 1/2 c_self C_ii with C_ii = 2 eps_i sigma_i^6.
template <typename T, int NP>
__global__ void __launch_bounds__(kBlock) k_interp_lb(
    const Vec4<T>* __restrict__ sp, const int* __restrict__ sidx, int N, const T* __restrict__ pot,
    long np, int n0, int n1, int n2, T ih0, T ih1, T ih2, const T* __restrict__ e0,
    const T* __restrict__ floc, const T* __restrict__ lbw, double cself, T* __restrict__ forces,
    double* __restrict__ epart, ReduceArgs R) {
  const long z = pdl_begin();
  sp += z; sidx += z; pot += z; e0 += z; floc += z; lbw += z;
  __shared__ double sh[32 * 7];
  __shared__ bool last;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double ea = 0.0;
  if (i < N) {
    Vec4<T> p = sp[i];
    const T sg = p.w, w = lbw[i];
    T xi[7];
    T s = T(1);
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      xi[k] = (T)lb_coef_d(k) * s * w;
      s *= sg;
    }
    T u0 = p.x * ih0, u1 = p.y * ih1, u2 = p.z * ih2;
    T f0 = floor(u0), f1 = floor(u1), f2 = floor(u2);
    int b0 = (int)f0, b1 = (int)f1, b2 = (int)f2;
    constexpr int B0 = NP / 2 - 1;
    T wx[NP], wy[NP], wz[NP], dx[NP], dy[NP], dz[NP];
    phid<NP>(u0 - f0, wx, dx);
    phid<NP>(u1 - f1, wy, dy);
    phid<NP>(u2 - f2, wz, dz);
    int ix[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) ix[k] = wrapi(b0 - B0 + k, n0);
    T acc = 0, g0 = 0, g1 = 0, g2 = 0;
    for (int c = 0; c < NP; ++c) {
      int z = wrapi(b2 - B0 + c, n2);
      for (int b = 0; b < NP; ++b) {
        int y = wrapi(b1 - B0 + b, n1);
        const long row = (long)n0 * (y + (long)n1 * z);
        T sx = 0, sdx = 0;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          T v = 0;
#pragma unroll
          for (int m = 0; m < 7; ++m) v += xi[6 - m] * pot[m * np + row + ix[a]];
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
    forces[3 * (size_t)o + 0] = floc[3 * (size_t)i + 0] + g0 * ih0;
    forces[3 * (size_t)o + 1] = floc[3 * (size_t)i + 1] + g1 * ih1;
    forces[3 * (size_t)o + 2] = floc[3 * (size_t)i + 2] + g2 * ih2;
    double cii = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) cii += (double)xi[k] * (double)xi[6 - k];
    ea = -0.5 * ((double)e0[i] + (double)acc) + 0.5 * cself * cii;
  }
  double s = block_sum(ea, sh);
  if (threadIdx.x == 0) {
    epart[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(R.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    final_reduce(epart, gridDim.x, R.wpart, R.nw, R.vir, R.out, sh);
    if (threadIdx.x == 0) *R.ticket = 0u;
  }
}

template <typename T> int launch_interp_lb(Plan* p, T* forces, cudaStream_t st) {
  const Level& L1 = p->lv[1];
  const int N = (int)p->N;
  ReduceArgs R = {p->d_wpart, wpart_used(p), 0, p->d_out,
                  reinterpret_cast<unsigned*>(p->d_flag + 1)};
  launch_pdl(p->order == 5 ? k_interp_lb<T, 6> : k_interp_lb<T, 4>, cdiv(N, kBlock), kBlock, 0, st, 
      (const Vec4<T>*)p->d_sorted, p->d_sorted_idx, N, (const T*)p->d_lbpot, L1.np, L1.n[0],
      L1.n[1], L1.n[2], (T)(1.0 / L1.h[0]), (T)(1.0 / L1.h[1]), (T)(1.0 / L1.h[2]),
      (const T*)p->d_e0, (const T*)p->d_floc, (const T*)p->d_lbw, p->c_self, forces, p->d_epart,
      R);
  return 1;
}

template <typename T>
int launch_interp(Plan* p, T* forces, double* atom_energy, bool vir, cudaStream_t st) {
  const Level& L1 = p->lv[1];
  const int N = (int)p->N;
  // slice sums only for interpolations of several waves: the single-wave
  // instantiation keeps the smaller kernel (one final-reduction copy)
  const bool slices = cdiv(N, kBlock) >= 4L * 152;
  ReduceArgs R = {p->d_wpart, wpart_used(p), vir ? 1 : 0, p->d_out,
                  reinterpret_cast<unsigned*>(p->d_flag + 1), p->d_out + 8,
                  slices ? kReduceGroups : 0};
  auto kern = p->order == 5 ? (slices ? k_interp<T, true, 6> : k_interp<T, false, 6>)
                            : (slices ? k_interp<T, true, 4> : k_interp<T, false, 4>);
  launch_pdl(kern, cdiv(N, kBlock), kBlock, 0, st,
      (const Vec4<T>*)p->d_sorted, p->d_sorted_idx, N, (const T*)p->d_et[1], L1.n[0], L1.n[1],
      L1.n[2], (T)(1.0 / L1.h[0]), (T)(1.0 / L1.h[1]), (T)(1.0 / L1.h[2]), (const T*)p->d_e0,
      (const T*)p->d_floc, p->c_self, forces, atom_energy, p->d_epart, R);
  return 1;
}

// Stencil launch configuration, decided before the workspace is sized: the
// tiled kernel (tiles counted in p->stencil_blocks by the caller) when its
// tile and tap table fit in shared memory (opt in above 48 KB), otherwise
// the global-memory kernel with one block per 256 nodes.
template <typename T> int prepare_grid_kernels(Plan* p) {
  if (p->levels < 2) return MLS6_OK;
  const int S = kStencilTile + 2 * p->P;
  int Sx, Sp;
  stencil_pitches(S, Sx, Sp);
  p->stencil_smem = align16(sizeof(T) * S * Sp) + sizeof(Vec4<T>) * p->ntaps +
                    sizeof(int4) * p->nrows;
  p->stencil_global = p->stencil_smem > kStencilSmemMax;
  if (p->stencil_global) {
    long nodes = 0;
    for (int k = 1; k < p->levels; ++k) nodes += p->lv[k].np;
    p->stencil_blocks = cdiv(nodes, kBlock);
    return MLS6_OK;
  }
  // tap-row groups per tile: the smallest of 1, 2, 4 for which the launch
  // has about 24 warps per SM of a 152-SM GPU in total, and the tiles that
  // fit in one SM's 227 KB of shared memory hold at least 24 warps
  // (1M-atom cube, 51 KB tiles: 4 tiles per SM, two groups -> stencil
  // 511 -> 434 us)
  const long tiles_per_sm = std::max(1L, (long)(227 * 1024) / (long)p->stencil_smem);
  p->stencil_groups = 1;
  while (p->stencil_groups < 4 && (p->stencil_blocks * 4 * p->stencil_groups < 152L * 24 ||
                                   tiles_per_sm * 4 * p->stencil_groups < 24))
    p->stencil_groups *= 2;
  // the limit is a property of the kernel, shared by every plan in the
  // process: set it to the budget ceiling, not to this plan's tile size
  const int sm = (int)kStencilSmemMax;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(k_stencil<T, true, 1>, attr, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil<T, false, 1>, attr, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil<T, true, 2>, attr, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil<T, false, 2>, attr, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil<T, true, 4>, attr, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil<T, false, 4>, attr, sm) != cudaSuccess)
    return MLS6_ERR_CUDA;
  return MLS6_OK;
}

#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
#define MLS6_INSTANTIATE(T)                                               \
  template int launch_anterp<T>(Plan*, cudaStream_t, int);                \
  template int launch_lb_weights<T>(Plan*, const T*, cudaStream_t);       \
  template int launch_interp_lb<T>(Plan*, T*, cudaStream_t);              \
  template int launch_restrict<T>(Plan*, int, cudaStream_t);              \
  template int launch_stencil<T>(Plan*, bool, cudaStream_t);              \
  template int launch_top<T>(Plan*, bool, cudaStream_t);                  \
  template int launch_prolong<T>(Plan*, int, cudaStream_t);               \
  template int launch_interp<T>(Plan*, T*, double*, bool, cudaStream_t);  \
  template int prepare_grid_kernels<T>(Plan*);
MLS6_INSTANTIATE(float)
MLS6_INSTANTIATE(double)
#undef MLS6_INSTANTIATE

#endif  // MLS6_DEVICE_ONLY
}  // namespace mls6
