// Local part of the split (Eq. g_0): pair sum over the cell list.
//   e0_i = sum_{j,n: r<a} c_j g_0(r),   F_i = -c_i sum c_j g_0'(r)/r d,
//   W   += 1/2 c_i sum c_j g_0'(r)/r d (x) d,       d = x_j - x_i + n L,
// with g_0 = r^-6 - a^-6 gamma(r/a); gamma is an even polynomial in r so no
// square root is taken and each pair costs one reciprocal.
#include <cmath>

#include "mls6_device.cuh"

namespace mls6 {

static inline long cdiv(long a, long b) { return (a + b - 1) / b; }

template <typename T> struct PairArgs {
  Box3<T> box;
  T inv_w[3];
  int nc[3], R[3];
  T a2, ia2, ia6, ia8;
};

template <typename T> __device__ __forceinline__ T rcp(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float rcp<float>(float x) { return __fdividef(1.0f, x); }

template <typename T, bool VIR>
__global__ void __launch_bounds__(kBlock) k_pair(const Vec4<T>* __restrict__ sp,
                                                  const int* __restrict__ start, int N,
                                                  PairArgs<T> g, T* __restrict__ e0,
                                                  T* __restrict__ floc,
                                                  double* __restrict__ wpart) {
  __shared__ double sh[32 * 6];
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
              T inv = rcp(r2);
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
    block_sum_n<6>(wv, sh);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) wpart[6 * (size_t)blockIdx.x + c] = wv[c];
  }
}

template <typename T> int launch_pair(Plan* p, bool vir, cudaStream_t st) {
  const int N = (int)p->N;
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
  if (vir)
    k_pair<T, true><<<cdiv(N, kBlock), kBlock, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
        p->d_wpart);
  else
    k_pair<T, false><<<cdiv(N, kBlock), kBlock, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
        p->d_wpart);
  return 1;
}

template int launch_pair<float>(Plan*, bool, cudaStream_t);
template int launch_pair<double>(Plan*, bool, cudaStream_t);

}  // namespace mls6
