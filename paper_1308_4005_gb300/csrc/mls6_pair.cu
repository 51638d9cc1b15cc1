// Local part of the split (Eq. g_0): pair sum over the cell list.
//   e0_i = sum_{j,n: r<a} c_j g_0(r),   F_i = -c_i sum c_j g_0'(r)/r d,
//   W   += 1/2 c_i sum c_j g_0'(r)/r d (x) d,       d = x_j - x_i + n L,
// with g_0 = r^-6 - a^-6 gamma(r/a); gamma is an even polynomial in r so no
// square root is taken and each pair costs one reciprocal.
#include <algorithm>
#include <cmath>

#include "mls6_device.cuh"

namespace mls6 {

static inline long cdiv(long a, long b) { return (a + b - 1) / b; }

template <typename T> struct PairArgs {
  Box3<T> box;
  T w[3], inv_w[3];
  int nc[3], R[3];
  T a2, ia2, ia6, ia8;
  T margin;  // absolute slack of the row trimming (covers rounding of x, x/w)
};

template <typename T> __device__ __forceinline__ T rcp(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }

// S consecutive lanes share one atom: the (2R+1)^2 rows of neighbour cells
// (constant dy, dz; the dx cells of a row are contiguous in the sorted
// array, split only where the row wraps periodically) are dealt round-robin
// to the S lanes, and the lanes' partial sums are combined by shuffles.
// S > 1 raises the number of resident warps for small systems, where one
// lane per atom leaves the SMs waiting on memory latency.
// Each row is trimmed to the cutoff sphere before its candidates are read:
// a row whose y-z distance d from the atom is >= a is skipped, otherwise
// only the cells within sqrt(a^2 - d^2) in x are scanned.  The trimming is
// conservative (a small slack); the exact test r^2 < a^2 stays per pair, so
// it changes which candidates are read, never the result.
// LB: Lorentz-Berthelot mixing (Sec. II.D): the sorted record carries
// sigma_i in place of c_i and lbw holds sqrt(2 eps_i) in sorted order; the
// pair coefficient is C_ij = lbw_i lbw_j ((sigma_i + sigma_j)/2)^6, and the
// outputs are e0_i = sum_j C_ij g_0 and F_i = -sum_j C_ij g_0'/r d.
template <typename T, bool VIR, int S, bool LB = false>
__global__ void __launch_bounds__(kBlock) k_pair(const Vec4<T>* __restrict__ sp,
                                                  const int* __restrict__ start, int N,
                                                  PairArgs<T> g, T* __restrict__ e0,
                                                  T* __restrict__ floc,
                                                  double* __restrict__ wpart,
                                                  const T* __restrict__ lbw = nullptr) {
  __shared__ double sh[32 * 6];
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = gid / S, sub = gid % S;
  T e = 0, fx = 0, fy = 0, fz = 0;
  T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  T ci = 0, wi = 0;
  if (i < N) {
    const Vec4<T> pi = sp[i];
    ci = pi.w;
    if (LB) wi = lbw[i];
    const int cx = min(max((int)(pi.x * g.inv_w[0]), 0), g.nc[0] - 1);
    const int cy = min(max((int)(pi.y * g.inv_w[1]), 0), g.nc[1] - 1);
    const int cz = min(max((int)(pi.z * g.inv_w[2]), 0), g.nc[2] - 1);
    const int ny = 2 * g.R[1] + 1, nrows = (2 * g.R[2] + 1) * ny;
    for (int r = sub; r < nrows; r += S) {
      const int dz = r / ny - g.R[2], dy = r % ny - g.R[1];
      const int z = cz + dz, iz = wrapi(z, g.nc[2]);
      const T sz = (T)((z - iz) / g.nc[2]) * g.box.L[2];
      const int y = cy + dy, iy = wrapi(y, g.nc[1]);
      const T sy = (T)((y - iy) / g.nc[1]) * g.box.L[1];
      // distance in y and z from the atom to this (unwrapped) row of cells
      const T ylo = (T)y * g.w[1], zlo = (T)z * g.w[2];
      const T dyl = max(T(0), max(ylo - pi.y, pi.y - (ylo + g.w[1])) - g.margin);
      const T dzl = max(T(0), max(zlo - pi.z, pi.z - (zlo + g.w[2])) - g.margin);
      const T d2 = dyl * dyl + dzl * dzl;
      if (d2 >= g.a2) continue;
      const T rx = sqrt(g.a2 - d2) + g.margin;
      const int xlo = max(-g.R[0], (int)floor((pi.x - rx) * g.inv_w[0]) - cx);
      const int xhi = min(g.R[0], (int)floor((pi.x + rx) * g.inv_w[0]) - cx);
      const T py = pi.y - sy, pz = pi.z - sz;
      const int row = g.nc[0] * (iy + g.nc[1] * iz);
      int dx = xlo;
      while (dx <= xhi) {
        const int x = cx + dx, ix = wrapi(x, g.nc[0]);
        const int wx = (x - ix) / g.nc[0];
        const int last = min(xhi, dx + (g.nc[0] - 1 - ix));  // same image run
        const T px = pi.x - (T)wx * g.box.L[0];
        const bool same = (wx == 0) && (y == iy) && (z == iz);
        const int j0 = start[row + ix], j1 = start[row + ix + (last - dx) + 1];
        // candidates four at a time: the four loads are issued together;
        // slots past the run (or the atom itself) are never inside a
        for (int j = j0; j < j1; j += 4) {
          Vec4<T> pj[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) pj[u] = sp[min(j + u, j1 - 1)];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const T ddx = pj[u].x - px, ddy = pj[u].y - py, ddz = pj[u].z - pz;
            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            const bool valid = (j + u < j1) && !(same && j + u == i);
            if (valid && r2 < g.a2) {
              const T inv = rcp(r2);
              const T inv3 = inv * inv * inv;
              const T s = r2 * g.ia2, s2 = s * s, s3 = s2 * s, s6 = s3 * s3;
              const T s5 = s3 * s2;
              const T g0 = inv3 - g.ia6 * (T(1.875) - T(1.25) * s6 + T(0.375) * s6 * s6);
              const T gp = T(-6) * inv3 * inv + g.ia8 * s5 * (T(15) - T(9) * s6);
              T cj = pj[u].w;
              if (LB) {
                const T sg = T(0.5) * (ci + pj[u].w), sg3 = sg * sg * sg;
                cj = wi * lbw[j + u] * sg3 * sg3;
              }
              e += cj * g0;
              const T cg = cj * gp;
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
        }
        dx = last + 1;
      }
    }
  }
#pragma unroll
  for (int o = S / 2; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
    fz += __shfl_xor_sync(0xffffffffu, fz, o);
  }
  if (i < N && sub == 0) {
    const T cf = LB ? T(1) : ci;  // LB: the coefficient is already in the sums
    e0[i] = e;
    floc[3 * (size_t)i + 0] = -cf * fx;
    floc[3 * (size_t)i + 1] = -cf * fy;
    floc[3 * (size_t)i + 2] = -cf * fz;
  }
  if (VIR) {
    // lanes of one atom hold disjoint candidate sets: all contribute
    T wv[6] = {ci * w0, ci * w1, ci * w2, ci * w3, ci * w4, ci * w5};
    double ws[6];
    block_sum_lo<T, 6>(wv, ws, sh);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) wpart[6 * (size_t)blockIdx.x + c] = 0.5 * ws[c];
  }
}

// Lanes per atom: the smallest of 1, 2, 4, 8 that gives about 48 resident
// warps per SM on a 152-SM GPU.
int pair_split(long N) {
  const long want = 152L * 48 * 32;
  int s = 1;
  while (s < 8 && N * s < want) s *= 2;
  return s;
}

template <typename T, int S>
static void launch_s(Plan* p, const PairArgs<T>& pg, bool vir, bool lb, cudaStream_t st) {
  const int N = (int)p->N;
  const long nb = cdiv((long)N * S, kBlock);
  if (lb)
    k_pair<T, false, S, true><<<nb, kBlock, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
        p->d_wpart + 6 * p->wpart_pair, (const T*)p->d_lbw);
  else if (vir)
    k_pair<T, true, S><<<nb, kBlock, 0, st>>>((const Vec4<T>*)p->d_sorted, p->d_cell_start, N,
                                              pg, (T*)p->d_e0, (T*)p->d_floc,
                                              p->d_wpart + 6 * p->wpart_pair);
  else
    k_pair<T, false, S><<<nb, kBlock, 0, st>>>((const Vec4<T>*)p->d_sorted, p->d_cell_start, N,
                                               pg, (T*)p->d_e0, (T*)p->d_floc,
                                               p->d_wpart + 6 * p->wpart_pair);
}

template <typename T> int launch_pair(Plan* p, bool vir, cudaStream_t st, bool lb) {
  PairArgs<T> pg;
  for (int d = 0; d < 3; ++d) {
    pg.box.L[d] = (T)p->L[d];
    pg.box.invL[d] = (T)(1.0 / p->L[d]);
    pg.w[d] = (T)p->cg.w[d];
    pg.inv_w[d] = (T)p->cg.inv_w[d];
    pg.nc[d] = p->cg.nc[d];
    pg.R[d] = p->cg.R[d];
  }
  // slack: 1e-3 of a cell plus 16 rounding units of the largest coordinate
  const double eps = p->prec == MLS6_FP64 ? 1.1e-16 : 6.0e-8;
  const double wmin = std::min(p->cg.w[0], std::min(p->cg.w[1], p->cg.w[2]));
  const double lmax = std::max(p->L[0], std::max(p->L[1], p->L[2]));
  pg.margin = (T)(1e-3 * wmin + 16.0 * eps * lmax);
  pg.a2 = (T)(p->a * p->a);
  pg.ia2 = (T)(1.0 / (p->a * p->a));
  pg.ia6 = (T)std::pow(p->a, -6.0);
  pg.ia8 = (T)std::pow(p->a, -8.0);
  switch (p->pair_split) {
    case 8: launch_s<T, 8>(p, pg, vir, lb, st); break;
    case 4: launch_s<T, 4>(p, pg, vir, lb, st); break;
    case 2: launch_s<T, 2>(p, pg, vir, lb, st); break;
    default: launch_s<T, 1>(p, pg, vir, lb, st); break;
  }
  return 1;
}

template int launch_pair<float>(Plan*, bool, cudaStream_t, bool);
template int launch_pair<double>(Plan*, bool, cudaStream_t, bool);

}  // namespace mls6
