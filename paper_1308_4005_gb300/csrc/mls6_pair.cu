// Local part of the split (Eq. g_0): pair sum over the cell list.
//   e0_i = sum_{j,n: r<a} c_j g_0(r),   F_i = -c_i sum c_j g_0'(r)/r d,
//   W   += 1/2 c_i sum c_j g_0'(r)/r d (x) d,       d = x_j - x_i + n L,
// with g_0 = r^-6 - a^-6 gamma(r/a); gamma is an even polynomial in r so no
// square root is taken and each pair costs one reciprocal.
#include <algorithm>
#include <climits>
#include <cmath>

#include "mls6_device.cuh"

namespace mls6 {


template <typename T> struct PairArgs {
  Box3<T> box;
  T w[3], inv_w[3];
  int nc[3], R[3];
  T a2, ia2, ia6, ia8;
  T margin;  // absolute slack of the row trimming (covers rounding of x, x/w)
  T Lhi[3], Llo[3];  // box length as an unevaluated sum hi + lo (exact image shifts)
  // smoothing function of continuity other than C^2 (GEN kernels):
  // gamma = sum gc[k] u^k, u = rho^12; gamma'(rho)/rho = -12 rho^10 ... as
  // g_0'/r = -6 r^-8 + a^-8 rho^10 sum gd[k] u^k with gd[k] = -12 (k+1) gc[k+1]
  T gc[5], gd[4];
};

// Eq. (g_0) and g_0'(r)/r from inv = 1/r^2, s1 = (r/a)^2: the C^2 smoothing
// function of Eq. (gamma) with its coefficients inline, or (GEN) the
// coefficients of the plan's smoothing function.
template <typename T, bool GEN>
__device__ __forceinline__ void g0_and_gp(T inv, T s1, const PairArgs<T>& g, T& g0, T& gp) {
  const T inv3 = inv * inv * inv;
  const T s2 = s1 * s1, s3 = s2 * s1, s6 = s3 * s3;
  const T s5 = s3 * s2;
  if (GEN) {
    const T P = g.gc[0] + s6 * (g.gc[1] + s6 * (g.gc[2] + s6 * (g.gc[3] + s6 * g.gc[4])));
    const T D = g.gd[0] + s6 * (g.gd[1] + s6 * (g.gd[2] + s6 * g.gd[3]));
    g0 = inv3 - g.ia6 * P;
    gp = T(-6) * inv3 * inv + g.ia8 * s5 * D;
  } else {
    g0 = inv3 - g.ia6 * (T(1.875) - T(1.25) * s6 + T(0.375) * s6 * s6);
    gp = T(-6) * inv3 * inv + g.ia8 * s5 * (T(15) - T(9) * s6);
  }
}

// i = m n + iw with 0 <= iw < n: the cell iw and periodic image m of an
// unwrapped cell index (|m| is 0 or 1 unless the box is thinner than the
// neighbour range).
__device__ __forceinline__ void wrap_image(int i, int n, int& iw, int& m) {
  iw = i;
  m = 0;
  while (iw < 0) {
    iw += n;
    --m;
  }
  while (iw >= n) {
    iw -= n;
    ++m;
  }
}

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
// Virial: a pair in the zero periodic image is met from both of its atoms,
// with d_ji = -d_ij, so its d (x) d terms over all atoms equal
// -2 sum_i F0_i (x) x_i, F0_i = sum_j c_j g_0'/r d over atom i's zero-image
// pairs (x_i the wrapped position the separations are taken from).  That
// product is formed once per atom; only pairs in a shifted image (runs of
// cells across a periodic face) add their d (x) d terms one by one.  The
// per-atom terms are not the atom's share of the virial, but their sum over
// all atoms is the virial.
template <typename T, bool VIR, int S, bool LB = false, bool GEN = false>
__device__ __forceinline__ void k_pair_body(const Blk bk,const Vec4<T>* __restrict__ sp,
                                                  const int* __restrict__ start, int N,
                                                  PairArgs<T> g, T* __restrict__ e0,
                                                  T* __restrict__ floc,
                                                  double* __restrict__ wpart,
                                                  const T* __restrict__ lbw) {
  const int gid = bk.x * blockDim.x + threadIdx.x;
  const int i = gid / S, sub = gid % S;
  T e = 0, fx = 0, fy = 0, fz = 0;
  T sfx = 0, sfy = 0, sfz = 0;  // force sum over pairs in shifted images
  T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;  // their d (x) d terms
  T ci = 0, wi = 0, xi = 0, yi = 0, zi = 0;
  if (i < N) {
    const Vec4<T> pi = sp[i];
    ci = pi.w;
    xi = pi.x;
    yi = pi.y;
    zi = pi.z;
    if (LB) wi = lbw[i];
    const int cx = min(max((int)(pi.x * g.inv_w[0]), 0), g.nc[0] - 1);
    const int cy = min(max((int)(pi.y * g.inv_w[1]), 0), g.nc[1] - 1);
    const int cz = min(max((int)(pi.z * g.inv_w[2]), 0), g.nc[2] - 1);
    const int ny = 2 * g.R[1] + 1, nrows = (2 * g.R[2] + 1) * ny;
    for (int r = sub; r < nrows; r += S) {
      const int dz = r / ny - g.R[2], dy = r % ny - g.R[1];
      const int z = cz + dz, y = cy + dy;
      int iz, iy, mz, my;
      wrap_image(z, g.nc[2], iz, mz);
      wrap_image(y, g.nc[1], iy, my);
      const T sz = (T)mz * g.box.L[2], sy = (T)my * g.box.L[1];
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
      int dx = xlo, ix, wx;
      wrap_image(cx + xlo, g.nc[0], ix, wx);
      for (; dx <= xhi; ix = 0, ++wx) {  // runs of one image; the next starts at cell 0
        const int last = min(xhi, dx + (g.nc[0] - 1 - ix));
        const T px = pi.x - (T)wx * g.box.L[0];
        const bool shifted = (wx | my | mz) != 0;
        const int j0 = start[row + ix], j1 = start[row + ix + (last - dx) + 1];
        // candidates four at a time: the four loads are issued together (the
        // sorted array has three padding records, so j + u stays in bounds);
        // slots past the run are never inside a, and the atom itself (zero
        // image, r = 0 exactly) is excluded by r^2 > 0
        for (int j = j0; j < j1; j += 4) {
          Vec4<T> pj[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) pj[u] = sp[j + u];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const T ddx = pj[u].x - px, ddy = pj[u].y - py, ddz = pj[u].z - pz;
            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            const bool valid = (j + u < j1) && r2 > T(0);
            if (valid && r2 < g.a2) {
              T g0, gp;
              g0_and_gp<T, GEN>(rcp(r2), r2 * g.ia2, g, g0, gp);
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
              if (VIR && shifted) {  // runs across a periodic face only
                const T cgx = cg * ddx, cgy = cg * ddy, cgz = cg * ddz;
                sfx += cgx;
                sfy += cgy;
                sfz += cgz;
                w0 += cgx * ddx;
                w1 += cgy * ddy;
                w2 += cgz * ddz;
                w3 += cgx * ddy;
                w4 += cgx * ddz;
                w5 += cgy * ddz;
              }
            }
          }
        }
        dx = last + 1;
      }
    }
  }
  // virial terms of this lane, from its own partial sums (before the lanes of
  // the atom exchange them); lanes of one atom hold disjoint candidate sets,
  // and the zero-image term is linear in the lane's partial force sum
  T wv[6];
  if (VIR) {
    const T f0x = fx - sfx, f0y = fy - sfy, f0z = fz - sfz;
    wv[0] = ci * (w0 - T(2) * f0x * xi);
    wv[1] = ci * (w1 - T(2) * f0y * yi);
    wv[2] = ci * (w2 - T(2) * f0z * zi);
    wv[3] = ci * (w3 - (f0x * yi + f0y * xi));
    wv[4] = ci * (w4 - (f0x * zi + f0z * xi));
    wv[5] = ci * (w5 - (f0y * zi + f0z * yi));
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
    // one partial per warp, at its global warp index: the partials, and so
    // the virial, do not depend on the block size the body runs with (a
    // single plan's launch or the persistent kernel of a batch)
#pragma unroll
    for (int c = 0; c < 6; ++c)
      for (int o = 16; o > 0; o >>= 1) wv[c] += __shfl_down_sync(0xffffffffu, wv[c], o);
    if ((threadIdx.x & 31) == 0) {
      const size_t wg = ((size_t)bk.x * blockDim.x + threadIdx.x) >> 5;
#pragma unroll
      for (int c = 0; c < 6; ++c) wpart[6 * wg + c] = 0.5 * (double)wv[c];
    }
  }
}

template <typename T, bool VIR, int S, bool LB = false, bool GEN = false>
__global__ void __launch_bounds__(kBlock) k_pair(const Vec4<T>* __restrict__ sp,
                                                  const int* __restrict__ start, int N,
                                                  PairArgs<T> g, T* __restrict__ e0,
                                                  T* __restrict__ floc,
                                                  double* __restrict__ wpart,
                                                  const T* __restrict__ lbw = nullptr) {
  k_pair_body<T, VIR, S, LB, GEN>(Blk::self(), sp, start, N, g, e0, floc, wpart, lbw);
}

// Warp form of the pair sum (lanes per atom S = 32 / G, G = 1 or 2 atoms
// per warp).  The G consecutive sorted atoms of a warp that share a row of
// cells (constant cy, cz) form a segment; for each segment
//   1. lane t sets up neighbour row t: the row is trimmed against the
//      segment's bounding box (skipped if its y-z distance is >= a, else
//      clipped in x to the box extent +- sqrt(a^2 - d^2)) and split into at
//      most three same-image pieces of contiguous candidates;
//   2. a warp scan turns the pieces into one flattened candidate stream;
//   3. lane (slot js, atom gi) takes every S-th candidate of the stream and
//      evaluates the pair branch-free (a miss adds zero).
// All lanes of a warp run the same number of iterations, and the integer
// work of the row set-up is done once per row, in parallel.  Each lane sums
// its candidates in stream order; the S partial sums of an atom are combined
// by a fixed shuffle tree, so the result is reproducible bit for bit.
// Requires every R <= 2 (at most 25 rows) and nc[0] >= 2 R[0] + 1 (a row's
// x range then spans at most three periodic pieces); pair_cluster_ok().
template <typename T, bool VIR, int G, bool LB = false>
__global__ void __launch_bounds__(kBlock) k_pair_warp(const Vec4<T>* __restrict__ sp,
                                                       const int* __restrict__ start, int N,
                                                       PairArgs<T> g, T* __restrict__ e0,
                                                       T* __restrict__ floc,
                                                       double* __restrict__ wpart,
                                                       const T* __restrict__ lbw = nullptr) {
  constexpr int S = 32 / G;
  constexpr int kW = kBlock / 32;
  constexpr int kP = 3 * 32;  // pieces of one segment: <= 3 per row, <= 32 rows
  constexpr unsigned kAll = 0xffffffffu;
  __shared__ double sh[32 * 6];
  __shared__ int t_end[kW][kP], t_base[kW][kP], t_img[kW][kP];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gi = lane % G, js = lane / G;
  const long il = ((long)blockIdx.x * kW + wid) * G + gi;
  const bool vi = il < N;
  const int i = vi ? (int)il : 0;
  T e = 0, fx = 0, fy = 0, fz = 0;
  T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  T ci = 0, wi = 0;
  Vec4<T> pi = {T(0), T(0), T(0), T(0)};
  int cx = 0, cy = 0, cz = 0, rid = INT_MAX;
  if (vi) {
    pi = sp[i];
    ci = pi.w;
    if (LB) wi = lbw[i];
    cx = min(max((int)(pi.x * g.inv_w[0]), 0), g.nc[0] - 1);
    cy = min(max((int)(pi.y * g.inv_w[1]), 0), g.nc[1] - 1);
    cz = min(max((int)(pi.z * g.inv_w[2]), 0), g.nc[2] - 1);
    rid = cy + g.nc[1] * cz;
  }
  const int ny = 2 * g.R[1] + 1, nrows = (2 * g.R[2] + 1) * ny;
  for (int s = 0; s < G;) {
    const int rs = __shfl_sync(kAll, rid, s);
    if (rs == INT_MAX) break;  // the remaining atoms are past N
    const unsigned seg = __ballot_sync(kAll, lane < G && rid == rs);
    const bool act = (seg >> gi) & 1u;
    // bounding box of the segment's atoms (lanes of one slot hold all G)
    T xmn = act ? pi.x : T(INFINITY), xmx = act ? pi.x : T(-INFINITY);
    T ymn = act ? pi.y : T(INFINITY), ymx = act ? pi.y : T(-INFINITY);
    T zmn = act ? pi.z : T(INFINITY), zmx = act ? pi.z : T(-INFINITY);
    int cxmn = act ? cx : INT_MAX, cxmx = act ? cx : INT_MIN;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      xmn = min(xmn, __shfl_xor_sync(kAll, xmn, o));
      xmx = max(xmx, __shfl_xor_sync(kAll, xmx, o));
      ymn = min(ymn, __shfl_xor_sync(kAll, ymn, o));
      ymx = max(ymx, __shfl_xor_sync(kAll, ymx, o));
      zmn = min(zmn, __shfl_xor_sync(kAll, zmn, o));
      zmx = max(zmx, __shfl_xor_sync(kAll, zmx, o));
      cxmn = min(cxmn, __shfl_xor_sync(kAll, cxmn, o));
      cxmx = max(cxmx, __shfl_xor_sync(kAll, cxmx, o));
    }
    const int scy = __shfl_sync(kAll, cy, s), scz = __shfl_sync(kAll, cz, s);
    // 1. lane t: row t of the (2R+1)^2 neighbour rows
    int np = 0, cnt = 0;
    int pj0[3] = {0, 0, 0}, pn[3] = {0, 0, 0}, pim[3] = {0, 0, 0};
    if (lane < nrows) {
      const int dz = lane / ny - g.R[2], dy = lane % ny - g.R[1];
      const int z = scz + dz, y = scy + dy;
      int iz, iy, mz, my;
      wrap_image(z, g.nc[2], iz, mz);
      wrap_image(y, g.nc[1], iy, my);
      const T ylo = (T)y * g.w[1], zlo = (T)z * g.w[2];
      const T dyl = max(T(0), max(ylo - ymx, ymn - (ylo + g.w[1])) - g.margin);
      const T dzl = max(T(0), max(zlo - zmx, zmn - (zlo + g.w[2])) - g.margin);
      const T d2 = dyl * dyl + dzl * dzl;
      if (d2 < g.a2) {
        const T rx = sqrt(g.a2 - d2) + g.margin;
        const int xl = max(cxmn - g.R[0], (int)floor((xmn - rx) * g.inv_w[0]));
        const int xh = min(cxmx + g.R[0], (int)floor((xmx + rx) * g.inv_w[0]));
        const int row = g.nc[0] * (iy + g.nc[1] * iz);
        // image of the row in y and z, packed with the x image per piece
        const int img_yz = ((my + 8) << 4) | ((mz + 8) << 8);
        int xa = xl, ix, mx;
        wrap_image(xl, g.nc[0], ix, mx);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (xa <= xh) {
            const int xb = min(xh, xa + (g.nc[0] - 1 - ix));
            pj0[q] = start[row + ix];
            pn[q] = start[row + ix + (xb - xa) + 1] - pj0[q];
            pim[q] = img_yz | (mx + 8);
            cnt += pn[q];
            np = q + 1;
            xa = xb + 1;
            ix = 0;
            ++mx;
          }
        }
      }
    }
    // 2. pieces -> one stream: inclusive scans of piece and candidate counts
    int np_inc = np, c_inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(kAll, np_inc, o), b = __shfl_up_sync(kAll, c_inc, o);
      if (lane >= o) {
        np_inc += a;
        c_inc += b;
      }
    }
    const int total = __shfl_sync(kAll, c_inc, 31);
    {
      int slot = np_inc - np, cend = c_inc - cnt;
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (q < np) {
          cend += pn[q];
          t_end[wid][slot] = cend;
          t_base[wid][slot] = pj0[q] - (cend - pn[q]);
          t_img[wid][slot] = pim[q];
          ++slot;
        }
    }
    __syncwarp();
    // 3. every S-th candidate of the stream, two in flight per lane
    int p = -1, pend = 0, pbase = 0;
    T qx = 0, qy = 0, qz = 0;  // the atom's position shifted by the piece's image
    bool same = false;         // piece in the zero image: exclude j == i
    for (int k0 = js; k0 < total; k0 += 2 * S) {
      int ju[2];
      bool ok[2];
      T sx[2], sy[2], sz[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int k = k0 + u * S;
        ok[u] = act && k < total;
        ju[u] = 0;
        if (k < total) {
          if (k >= pend) {
            do {
              ++p;
              pend = t_end[wid][p];
            } while (k >= pend);
            pbase = t_base[wid][p];
            const int im = t_img[wid][p];
            const int mx = (im & 15) - 8, my = ((im >> 4) & 15) - 8, mz = ((im >> 8) & 15) - 8;
            qx = pi.x - (T)mx * g.box.L[0];
            qy = pi.y - (T)my * g.box.L[1];
            qz = pi.z - (T)mz * g.box.L[2];
            same = (mx | my | mz) == 0;
          }
          ju[u] = pbase + k;
          ok[u] = ok[u] && !(same && ju[u] == i);
        }
        sx[u] = qx;
        sy[u] = qy;
        sz[u] = qz;
      }
      Vec4<T> pj[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) pj[u] = sp[ju[u]];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const T ddx = pj[u].x - sx[u], ddy = pj[u].y - sy[u], ddz = pj[u].z - sz[u];
        const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const bool hit = ok[u] && r2 < g.a2;
        const T rr = hit ? r2 : g.a2;  // a miss evaluates at r = a with weight zero
        const T inv = rcp(rr);
        const T inv3 = inv * inv * inv;
        const T s1 = rr * g.ia2, s2 = s1 * s1, s3 = s2 * s1, s6 = s3 * s3;
        const T s5 = s3 * s2;
        const T g0 = inv3 - g.ia6 * (T(1.875) - T(1.25) * s6 + T(0.375) * s6 * s6);
        const T gp = T(-6) * inv3 * inv + g.ia8 * s5 * (T(15) - T(9) * s6);
        T cj = pj[u].w;
        if (LB) {
          const T sg = T(0.5) * (ci + pj[u].w), sg3 = sg * sg * sg;
          cj = wi * lbw[ju[u]] * sg3 * sg3;
        }
        cj = hit ? cj : T(0);
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
    __syncwarp();  // the next segment rewrites the piece table
    s += __popc(seg);
  }
#pragma unroll
  for (int o = G; o < 32; o <<= 1) {
    e += __shfl_xor_sync(kAll, e, o);
    fx += __shfl_xor_sync(kAll, fx, o);
    fy += __shfl_xor_sync(kAll, fy, o);
    fz += __shfl_xor_sync(kAll, fz, o);
  }
  if (vi && js == 0) {
    const T cf = LB ? T(1) : ci;
    e0[i] = e;
    floc[3 * (size_t)i + 0] = -cf * fx;
    floc[3 * (size_t)i + 1] = -cf * fy;
    floc[3 * (size_t)i + 2] = -cf * fz;
  }
  if (VIR) {
    T wv[6] = {ci * w0, ci * w1, ci * w2, ci * w3, ci * w4, ci * w5};
    double ws[6];
    block_sum_lo<T, 6>(wv, ws, sh);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) wpart[6 * (size_t)blockIdx.x + c] = 0.5 * ws[c];
  }
}


// Cluster form (pair_split 1024, FP32): a warp takes the 8 consecutive
// sorted atoms 8w .. 8w+7 as an i-cluster; lane = i slot (lane & 7) x j slot
// (lane >> 3).  The atoms are split into segments of one cell row spanning
// at most 8 cells in x (sorted order keeps a segment contiguous); for each
// segment
//   1. lane t sets up neighbour row t of the (2R+1)^2 rows against the
//      segment's bounding box (skipped if its y-z distance is >= a, else
//      clipped in x to the box extent +- sqrt(a^2 - d^2), at most two
//      same-image runs of contiguous candidates since nc[0] >= 16 exceeds
//      the <= 15 cells of the clipped range) and the runs are compacted into
//      a per-warp table;
//   2. the warp walks the table; per run, candidates j0, j0+4, ... go to the
//      four j slots, so every candidate is loaded once (8 lanes share the
//      load) and paired with all 8 atoms of the segment.
// Every loop bound is uniform over the warp and the pair is evaluated
// branch-free (a miss or the atom itself adds zero), so all 32 lanes do
// useful issue; the price is the misses of the cluster's union of candidate
// cells.  Each lane sums its candidates in table order and the four j slots
// of an atom are combined by a fixed shuffle tree: results are reproducible
// bit for bit.  Requires R <= 2 on every axis and nc[0] >= 16
// (pair_cl_ok()).
constexpr int kClRuns = 2 * 25;

template <bool VIR, bool GEN>
__global__ void __launch_bounds__(kBlock) k_pair_cl(const Vec4<float>* __restrict__ sp,
                                                     const int* __restrict__ start, int N,
                                                     PairArgs<float> g, float* __restrict__ e0,
                                                     float* __restrict__ floc,
                                                     double* __restrict__ wpart) {
  using T = float;
  constexpr int kW = kBlock / 32;
  constexpr unsigned kAll = 0xffffffffu;
  __shared__ double sh[32 * 6];
  __shared__ int4 run_j[kW][kClRuns];     // first, end, zero image (1/0), -
  __shared__ float4 run_s[kW][kClRuns];   // image shift m L
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gi = lane & 7, js = lane >> 3;
  const long il = ((long)blockIdx.x * kW + wid) * 8 + gi;
  const bool vi = il < N;
  const int i = vi ? (int)il : 0;
  T e = 0, fx = 0, fy = 0, fz = 0;
  T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  T ci = 0;
  Vec4<T> pi = {T(0), T(0), T(0), T(0)};
  int cx = 0, cy = 0, cz = 0, rid = INT_MAX;
  if (vi) {
    pi = sp[i];
    ci = pi.w;
    cx = min(max((int)(pi.x * g.inv_w[0]), 0), g.nc[0] - 1);
    cy = min(max((int)(pi.y * g.inv_w[1]), 0), g.nc[1] - 1);
    cz = min(max((int)(pi.z * g.inv_w[2]), 0), g.nc[2] - 1);
    rid = cy + g.nc[1] * cz;
  }
  const int ny = 2 * g.R[1] + 1, nrows = (2 * g.R[2] + 1) * ny;
  for (int s = 0; s < 8;) {
    const int rs = __shfl_sync(kAll, rid, s);
    if (rs == INT_MAX) break;  // the remaining atoms are past N
    const int cxs = __shfl_sync(kAll, cx, s);
    const unsigned seg =
        __ballot_sync(kAll, js == 0 && gi >= s && rid == rs && cx <= cxs + 7);
    const bool act = (seg >> gi) & 1u;
    // bounding box of the segment (the lanes of one j slot hold all 8 atoms)
    T xmn = act ? pi.x : T(INFINITY), xmx = act ? pi.x : T(-INFINITY);
    T ymn = act ? pi.y : T(INFINITY), ymx = act ? pi.y : T(-INFINITY);
    T zmn = act ? pi.z : T(INFINITY), zmx = act ? pi.z : T(-INFINITY);
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      xmn = min(xmn, __shfl_xor_sync(kAll, xmn, o));
      xmx = max(xmx, __shfl_xor_sync(kAll, xmx, o));
      ymn = min(ymn, __shfl_xor_sync(kAll, ymn, o));
      ymx = max(ymx, __shfl_xor_sync(kAll, ymx, o));
      zmn = min(zmn, __shfl_xor_sync(kAll, zmn, o));
      zmx = max(zmx, __shfl_xor_sync(kAll, zmx, o));
    }
    const int scy = __shfl_sync(kAll, cy, s), scz = __shfl_sync(kAll, cz, s);
    // 1. lane t: neighbour row t, at most two same-image runs
    int nr = 0;  // runs of this row: rj0/rs0, then rj1/rs1 (registers, no indexing)
    int4 rj0 = make_int4(0, 0, 0, 0), rj1 = rj0;
    float4 rs0 = make_float4(0.f, 0.f, 0.f, 0.f), rs1 = rs0;
    if (lane < nrows) {
      const int dz = lane / ny - g.R[2], dy = lane % ny - g.R[1];
      const int z = scz + dz, y = scy + dy;
      int iz, iy, mz, my;
      wrap_image(z, g.nc[2], iz, mz);
      wrap_image(y, g.nc[1], iy, my);
      const T ylo = (T)y * g.w[1], zlo = (T)z * g.w[2];
      const T dyl = max(T(0), max(ylo - ymx, ymn - (ylo + g.w[1])) - g.margin);
      const T dzl = max(T(0), max(zlo - zmx, zmn - (zlo + g.w[2])) - g.margin);
      const T d2 = dyl * dyl + dzl * dzl;
      if (d2 < g.a2) {
        const T rx = sqrt(g.a2 - d2) + g.margin;
        const int xl = (int)floor((xmn - rx) * g.inv_w[0]);
        const int xh = (int)floor((xmx + rx) * g.inv_w[0]);
        const int row = g.nc[0] * (iy + g.nc[1] * iz);
        int ix, mx;
        wrap_image(xl, g.nc[0], ix, mx);
        const T sy = (T)my * g.box.L[1], sz = (T)mz * g.box.L[2];
        int xa = xl;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (xa <= xh) {
            const int xb = min(xh, xa + (g.nc[0] - 1 - ix));
            const int j0 = start[row + ix], j1 = start[row + ix + (xb - xa) + 1];
            if (j1 > j0) {
              const int4 a = make_int4(j0, j1, (mx | my | mz) == 0 ? 1 : 0, 0);
              const float4 b = make_float4((T)mx * g.box.L[0], sy, sz, 0.f);
              if (nr == 0) {
                rj0 = a;
                rs0 = b;
              } else {
                rj1 = a;
                rs1 = b;
              }
              ++nr;
            }
            xa = xb + 1;
            ix = 0;
            ++mx;
          }
        }
      }
    }
    // compact the runs of all rows into the warp's table (row order)
    int inc = nr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(kAll, inc, o);
      if (lane >= o) inc += v;
    }
    const int total = __shfl_sync(kAll, inc, 31);
    if (nr > 0) {
      run_j[wid][inc - nr] = rj0;
      run_s[wid][inc - nr] = rs0;
    }
    if (nr > 1) {
      run_j[wid][inc - 1] = rj1;
      run_s[wid][inc - 1] = rs1;
    }
    __syncwarp();
    // 2. all runs, four candidates per step, paired with the 8 atoms
    for (int r = 0; r < total; ++r) {
      const int4 R = run_j[wid][r];
      const float4 S = run_s[wid][r];
      const T qx = pi.x - S.x, qy = pi.y - S.y, qz = pi.z - S.z;
      const int self = (act && R.z) ? i : -1;  // the atom itself: zero image only
      for (int jb = R.x; jb < R.y; jb += 4) {
        const int j = jb + js;
        const bool ok = act && j < R.y && j != self;
        const Vec4<T> pj = sp[min(j, R.y - 1)];
        const T ddx = pj.x - qx, ddy = pj.y - qy, ddz = pj.z - qz;
        const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
        const bool hit = ok && r2 < g.a2;
        const T rr = hit ? r2 : g.a2;  // a miss evaluates at r = a with weight zero
        T g0, gp;
        g0_and_gp<T, GEN>(rcp(rr), rr * g.ia2, g, g0, gp);
        const T cj = hit ? pj.w : T(0);
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
    __syncwarp();  // the next segment rewrites the run table
    s += __popc(seg);
  }
#pragma unroll
  for (int o = 8; o < 32; o <<= 1) {
    e += __shfl_xor_sync(kAll, e, o);
    fx += __shfl_xor_sync(kAll, fx, o);
    fy += __shfl_xor_sync(kAll, fy, o);
    fz += __shfl_xor_sync(kAll, fz, o);
  }
  if (vi && js == 0) {
    e0[i] = e;
    floc[3 * (size_t)i + 0] = -ci * fx;
    floc[3 * (size_t)i + 1] = -ci * fy;
    floc[3 * (size_t)i + 2] = -ci * fz;
  }
  if (VIR) {
    T wv[6] = {ci * w0, ci * w1, ci * w2, ci * w3, ci * w4, ci * w5};
    double ws[6];
    block_sum_lo<T, 6>(wv, ws, sh);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) wpart[6 * (size_t)blockIdx.x + c] = 0.5 * ws[c];
  }
}

// One queued pair of the queue form: displacement with an exact image shift,
// then Eq. (g_0) and its derivative accumulated into the lane's sums.
// en = {j, image code (mx+8) | (my+8) << 4 | (mz+8) << 8}: the neighbour is
// x_j + m L.  The box length is the unevaluated sum Lhi + Llo, and the
// shift is applied to whichever of x_i, x_j lies near the far face
// (x_i - Lhi for m = +1, x_j - Lhi for m = -1), where the subtraction is
// exact: an image pair carries no rounding of the box length or of the
// absolute coordinates.
template <typename T, bool VIR, bool LB>
__device__ __forceinline__ void pair_eval(int2 en, const Vec4<T>* __restrict__ sp,
                                          const T* __restrict__ lbw, const Vec4<T>& pi, T wi,
                                          const PairArgs<T>& g, T& e, T& fx, T& fy, T& fz, T& w0,
                                          T& w1, T& w2, T& w3, T& w4, T& w5) {
  constexpr int kImg0 = 8 | (8 << 4) | (8 << 8);
  const Vec4<T> pj = sp[en.x];
  T ddx = pj.x - pi.x, ddy = pj.y - pi.y, ddz = pj.z - pi.z;
  if (en.y != kImg0) {
    const int m[3] = {(en.y & 15) - 8, ((en.y >> 4) & 15) - 8, ((en.y >> 8) & 15) - 8};
    const T xj[3] = {pj.x, pj.y, pj.z}, xi[3] = {pi.x, pi.y, pi.z};
    T d[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T sh = (T)m[a] * g.Lhi[a];
      const T sj = m[a] < 0 ? xj[a] + sh : xj[a];
      const T si = m[a] > 0 ? xi[a] - sh : xi[a];
      d[a] = (sj - si) + (T)m[a] * g.Llo[a];
    }
    ddx = d[0];
    ddy = d[1];
    ddz = d[2];
  }
  const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
  const T inv = rcp(r2);
  const T inv3 = inv * inv * inv;
  const T s1 = r2 * g.ia2, s2 = s1 * s1, s3 = s2 * s1, s6 = s3 * s3;
  const T s5 = s3 * s2;
  const T g0 = inv3 - g.ia6 * (T(1.875) - T(1.25) * s6 + T(0.375) * s6 * s6);
  const T gp = T(-6) * inv3 * inv + g.ia8 * s5 * (T(15) - T(9) * s6);
  T cj = pj.w;
  if (LB) {
    const T sg = T(0.5) * (pi.w + pj.w), sg3 = sg * sg * sg;
    cj = wi * lbw[en.x] * sg3 * sg3;
  }
  e += cj * g0;
  const T cg = cj * gp;
  fx += cg * ddx;
  fy += cg * ddy;
  fz += cg * ddz;
  if (VIR) {  // virial records carry c_i (the lanes mix atoms)
    const T cv = LB ? cg : pi.w * cg;
    const T cx_ = cv * ddx, cy_ = cv * ddy;
    w0 += cx_ * ddx;
    w1 += cy_ * ddy;
    w2 += cv * ddz * ddz;
    w3 += cx_ * ddy;
    w4 += cx_ * ddz;
    w5 += cy_ * ddz;
  }
}

// Stage candidates c0 .. c0+cn-1 of a warp's stream in shared memory: the
// position shifted by its piece's periodic image (for the cutoff test) and
// {j, image code} (for the evaluation).
template <typename T>
__device__ __forceinline__ void q_stage(int c0, int cn, int lane, const int* t_end,
                                        const int* t_base, const int* t_img,
                                        const Vec4<T>* __restrict__ sp, const PairArgs<T>& g,
                                        Vec4<T>* cpos, int2* cidx) {
  constexpr int kImg0 = 8 | (8 << 4) | (8 << 8);
  int p = -1, pend = 0, pbase = 0, pimg = kImg0;
  T sx = 0, sy = 0, sz = 0;
  for (int u = lane; u < cn; u += 32) {
    const int k = c0 + u;
    if (k >= pend) {
      do {
        ++p;
        pend = t_end[p];
      } while (k >= pend);
      pbase = t_base[p];
      pimg = t_img[p];
      sx = (T)((pimg & 15) - 8) * g.box.L[0];
      sy = (T)(((pimg >> 4) & 15) - 8) * g.box.L[1];
      sz = (T)(((pimg >> 8) & 15) - 8) * g.box.L[2];
    }
    const int j = pbase + k;
    Vec4<T> pj = sp[j];
    pj.x += sx;
    pj.y += sy;
    pj.z += sz;
    cpos[u] = pj;
    cidx[u] = make_int2(j, pimg);
  }
}

// Queue form of the pair sum (pair_split 64 G: G = 2, 4 or 8 atoms per
// warp, kQWarps warps per block).  The G consecutive sorted atoms of a warp
// that share a row of cells form a segment, and the segment's candidate
// stream is built as in the warp form (lane t: neighbour row t trimmed
// against the segment's bounding box, a warp scan flattening the pieces).
// The stream is staged in shared memory (positions shifted by their
// periodic image, chunks of qcap<T>() candidates), so the G atoms read the
// candidates from global memory once.  Each atom then tests the staged
// candidates 32 at a time (0 < r^2 < a^2: the atom itself is the only
// candidate at distance 0), the hits of the 32 lanes are compacted by a
// ballot into a per-warp queue, and whenever 32 hits are queued all 32
// lanes evaluate one each.  The pair arithmetic therefore runs on full warps
// and only on pairs inside the cutoff.  The queue is filled and drained in
// stream order and each lane sums its evaluations in that order, then a
// fixed shuffle tree combines the lanes: results are reproducible bit for
// bit.
constexpr int kQWarps = 4;
template <typename T> __host__ __device__ constexpr int qcap() {
  return sizeof(T) == 4 ? 512 : 256;
}
template <typename T> constexpr size_t q_smem_bytes() {
  return (size_t)kQWarps * qcap<T>() * (sizeof(Vec4<T>) + sizeof(int2));
}

template <typename T, bool VIR, int G, bool LB = false>
__global__ void __launch_bounds__(kQWarps * 32) k_pair_q(const Vec4<T>* __restrict__ sp,
                                                          const int* __restrict__ start, int N,
                                                          PairArgs<T> g, T* __restrict__ e0,
                                                          T* __restrict__ floc,
                                                          double* __restrict__ wpart,
                                                          const T* __restrict__ lbw = nullptr) {
  constexpr int kW = kQWarps;
  constexpr int kP = 3 * 32;   // pieces of one segment: <= 3 per row, <= 32 rows
  constexpr int kQ = 64;       // queued hits: < 32 left over + 32 new
  constexpr int kCap = qcap<T>();
  constexpr unsigned kAll = 0xffffffffu;
  __shared__ double sh[32 * 6];
  __shared__ int t_end[kW][kP], t_base[kW][kP], t_img[kW][kP];
  __shared__ int2 qu[kW][kQ];
  extern __shared__ __align__(16) unsigned char q_dyn[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Vec4<T>* cpos = reinterpret_cast<Vec4<T>*>(q_dyn) + (size_t)wid * kCap;
  int2* cidx = reinterpret_cast<int2*>(q_dyn + (size_t)kW * kCap * sizeof(Vec4<T>)) +
               (size_t)wid * kCap;
  const long i0 = ((long)blockIdx.x * kW + wid) * G;
  const int nat = (int)max(0L, min((long)G, (long)N - i0));  // atoms of this warp
  // lane t < nat holds atom i0 + t
  Vec4<T> pa = {T(0), T(0), T(0), T(0)};
  int cx = 0, cy = 0, cz = 0, rid = INT_MAX;
  if (lane < nat) {
    pa = sp[i0 + lane];
    cx = min(max((int)(pa.x * g.inv_w[0]), 0), g.nc[0] - 1);
    cy = min(max((int)(pa.y * g.inv_w[1]), 0), g.nc[1] - 1);
    cz = min(max((int)(pa.z * g.inv_w[2]), 0), g.nc[2] - 1);
    rid = cy + g.nc[1] * cz;
  }
  T w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
  const int ny = 2 * g.R[1] + 1, nrows = (2 * g.R[2] + 1) * ny;
  for (int s = 0; s < nat;) {
    const int rs = __shfl_sync(kAll, rid, s);
    const unsigned seg = __ballot_sync(kAll, lane < nat && rid == rs);
    const bool act = (seg >> lane) & 1u;
    // bounding box of the segment
    T xmn = act ? pa.x : T(INFINITY), xmx = act ? pa.x : T(-INFINITY);
    T ymn = act ? pa.y : T(INFINITY), ymx = act ? pa.y : T(-INFINITY);
    T zmn = act ? pa.z : T(INFINITY), zmx = act ? pa.z : T(-INFINITY);
    int cxmn = act ? cx : INT_MAX, cxmx = act ? cx : INT_MIN;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {  // over the lanes 0..G-1 that hold atoms
      xmn = min(xmn, __shfl_xor_sync(kAll, xmn, o));
      xmx = max(xmx, __shfl_xor_sync(kAll, xmx, o));
      ymn = min(ymn, __shfl_xor_sync(kAll, ymn, o));
      ymx = max(ymx, __shfl_xor_sync(kAll, ymx, o));
      zmn = min(zmn, __shfl_xor_sync(kAll, zmn, o));
      zmx = max(zmx, __shfl_xor_sync(kAll, zmx, o));
      cxmn = min(cxmn, __shfl_xor_sync(kAll, cxmn, o));
      cxmx = max(cxmx, __shfl_xor_sync(kAll, cxmx, o));
    }
    // every lane sets up a row: broadcast the box from lane 0
    xmn = __shfl_sync(kAll, xmn, 0);
    xmx = __shfl_sync(kAll, xmx, 0);
    ymn = __shfl_sync(kAll, ymn, 0);
    ymx = __shfl_sync(kAll, ymx, 0);
    zmn = __shfl_sync(kAll, zmn, 0);
    zmx = __shfl_sync(kAll, zmx, 0);
    cxmn = __shfl_sync(kAll, cxmn, 0);
    cxmx = __shfl_sync(kAll, cxmx, 0);
    const int scy = __shfl_sync(kAll, cy, s), scz = __shfl_sync(kAll, cz, s);
    // 1. lane t: row t of the (2R+1)^2 neighbour rows, trimmed and split
    //    into at most three same-image pieces
    int np = 0, cnt = 0;
    int pj0[3] = {0, 0, 0}, pn[3] = {0, 0, 0}, pim[3] = {0, 0, 0};
    if (lane < nrows) {
      const int dz = lane / ny - g.R[2], dy = lane % ny - g.R[1];
      const int z = scz + dz, y = scy + dy;
      int iz, iy, mz, my;
      wrap_image(z, g.nc[2], iz, mz);
      wrap_image(y, g.nc[1], iy, my);
      const T ylo = (T)y * g.w[1], zlo = (T)z * g.w[2];
      const T dyl = max(T(0), max(ylo - ymx, ymn - (ylo + g.w[1])) - g.margin);
      const T dzl = max(T(0), max(zlo - zmx, zmn - (zlo + g.w[2])) - g.margin);
      const T d2 = dyl * dyl + dzl * dzl;
      if (d2 < g.a2) {
        const T rx = sqrt(g.a2 - d2) + g.margin;
        const int xl = max(cxmn - g.R[0], (int)floor((xmn - rx) * g.inv_w[0]));
        const int xh = min(cxmx + g.R[0], (int)floor((xmx + rx) * g.inv_w[0]));
        const int row = g.nc[0] * (iy + g.nc[1] * iz);
        const int img_yz = ((my + 8) << 4) | ((mz + 8) << 8);
        int xa = xl, ix, mx;
        wrap_image(xl, g.nc[0], ix, mx);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (xa <= xh) {
            const int xb = min(xh, xa + (g.nc[0] - 1 - ix));
            pj0[q] = start[row + ix];
            pn[q] = start[row + ix + (xb - xa) + 1] - pj0[q];
            pim[q] = img_yz | (mx + 8);
            cnt += pn[q];
            np = q + 1;
            xa = xb + 1;
            ix = 0;
            ++mx;
          }
        }
      }
    }
    // 2. pieces -> one stream
    int np_inc = np, c_inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(kAll, np_inc, o), b = __shfl_up_sync(kAll, c_inc, o);
      if (lane >= o) {
        np_inc += a;
        c_inc += b;
      }
    }
    const int total = __shfl_sync(kAll, c_inc, 31);
    {
      int slot = np_inc - np, cend = c_inc - cnt;
#pragma unroll
      for (int q = 0; q < 3; ++q)
        if (q < np) {
          cend += pn[q];
          t_end[wid][slot] = cend;
          t_base[wid][slot] = pj0[q] - (cend - pn[q]);
          t_img[wid][slot] = pim[q];
          ++slot;
        }
    }
    __syncwarp();
    const bool one = total <= kCap;
    if (one) q_stage<T>(0, total, lane, t_end[wid], t_base[wid], t_img[wid], sp, g, cpos, cidx);
    __syncwarp();
    // 3. every atom of the segment against the stream
    const int send = s + __popc(seg);
    for (; s < send; ++s) {
      const int i = (int)(i0 + s);
      Vec4<T> pi;
      pi.x = __shfl_sync(kAll, pa.x, s);
      pi.y = __shfl_sync(kAll, pa.y, s);
      pi.z = __shfl_sync(kAll, pa.z, s);
      pi.w = __shfl_sync(kAll, pa.w, s);
      T wi = T(0);
      if (LB) wi = lbw[i];
      T e = 0, fx = 0, fy = 0, fz = 0;
      int qn = 0;
      for (int c0 = 0; c0 < total; c0 += kCap) {
        const int cn = min(kCap, total - c0);
        if (!one) {
          __syncwarp();
          q_stage<T>(c0, cn, lane, t_end[wid], t_base[wid], t_img[wid], sp, g, cpos, cidx);
          __syncwarp();
        }
        for (int u0 = 0; u0 < cn; u0 += 32) {
          const int u = u0 + lane;
          bool hit = false;
          if (u < cn) {
            const Vec4<T> pj = cpos[u];
            const T ddx = pj.x - pi.x, ddy = pj.y - pi.y, ddz = pj.z - pi.z;
            const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            hit = r2 < g.a2 && r2 > T(0);
          }
          const unsigned m = __ballot_sync(kAll, hit);
          if (hit) qu[wid][qn + __popc(m & ((1u << lane) - 1u))] = cidx[u];
          qn += __popc(m);
          if (qn >= 32) {
            __syncwarp();
            pair_eval<T, VIR, LB>(qu[wid][lane], sp, lbw, pi, wi, g, e, fx, fy, fz, w0, w1, w2,
                                  w3, w4, w5);
            __syncwarp();
            if (lane < qn - 32) qu[wid][lane] = qu[wid][lane + 32];
            __syncwarp();
            qn -= 32;
          }
        }
      }
      __syncwarp();
      if (lane < qn)
        pair_eval<T, VIR, LB>(qu[wid][lane], sp, lbw, pi, wi, g, e, fx, fy, fz, w0, w1, w2, w3,
                              w4, w5);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(kAll, e, o);
        fx += __shfl_xor_sync(kAll, fx, o);
        fy += __shfl_xor_sync(kAll, fy, o);
        fz += __shfl_xor_sync(kAll, fz, o);
      }
      if (lane == 0) {
        const T cf = LB ? T(1) : pi.w;
        e0[i] = e;
        floc[3 * (size_t)i + 0] = -cf * fx;
        floc[3 * (size_t)i + 1] = -cf * fy;
        floc[3 * (size_t)i + 2] = -cf * fz;
      }
      __syncwarp();  // the queue is reused by the next atom
    }
    __syncwarp();  // the next segment rewrites the piece table and the stage
  }
  if (VIR) {
    T wv[6] = {w0, w1, w2, w3, w4, w5};
    double ws[6];
    block_sum_lo<T, 6>(wv, ws, sh);
    if (threadIdx.x == 0)
      for (int c = 0; c < 6; ++c) wpart[6 * (size_t)blockIdx.x + c] = 0.5 * ws[c];
  }
}

#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
bool pair_cluster_ok(const Plan* p) {
  if (p->sm.n != 2) return false;  // warp and queue forms: Eq. (gamma) only
  for (int d = 0; d < 3; ++d)
    if (p->cg.R[d] > 2) return false;
  return p->cg.nc[0] >= 2 * p->cg.R[0] + 1;
}
#endif  // MLS6_DEVICE_ONLY

#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
// Cluster form: FP32 arithmetic, every neighbour range R <= 2 and at least
// 16 cells along x (a segment's clipped x range then meets at most two
// periodic images).
bool pair_cl_ok(const Plan* p) {
  if (p->prec == MLS6_FP64) return false;
  for (int d = 0; d < 3; ++d)
    if (p->cg.R[d] > 2) return false;
  return p->cg.nc[0] >= 16;
}

long pair_blocks(const Plan* p, int split) {
  const long N = p->N;
  if (N <= 0) return 0;
  if (split == kPairCluster) return cdiv(N, (long)kBlock / 4);  // 8 atoms per warp
  if (split >= 64) return cdiv(cdiv(N, split / 64), kQWarps);
  if (split <= 8) return cdiv(N * split, 32L);  // per-atom kernel: one virial partial per warp
  return cdiv(N * split, kBlock);                // warp form: one per block
}
#endif  // MLS6_DEVICE_ONLY

// Default pair kernel: FP64 the queue form where the cell geometry allows
// it; otherwise the smallest of 1, 2, 4, 8 lanes per atom that gives about
// 48 resident warps per SM on a 152-SM GPU.
#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
int pair_split(const Plan* p) {
  // the cluster form is not a default: on the 1M-atom cube it takes 1.22 ms
  // against 0.757 ms for the per-atom kernel (every atom of a segment is
  // evaluated against the union of the segment's candidate cells, which the
  // full lanes do not make up for)
  return pair_split_atom(p);
}

int pair_split_atom(const Plan* p) {
  // FP64: the queue form with two atoms per warp where the cell geometry
  // allows it (1M-atom cube 24.5 ms against 29.4 ms per atom and 31.2 ms
  // for the warp form); FP32 keeps the per-atom kernel (0.757 ms there
  // against 2.23 ms for the best queue form)
  if (p->prec == MLS6_FP64 && pair_cluster_ok(p)) return 128;
  const long want = 152L * 48 * 32;
  int s = 1;
  while (s < 8 && p->N * s < want) s *= 2;
  return s;
}
#endif  // MLS6_DEVICE_ONLY

// One lane per atom runs in small blocks (kPairAtomBlock): the block's
// warps end at different times (their atoms' candidate counts differ), and a
// small block gives its SM slot back sooner, to the next pair block or to the
// grid chain running beside the pair sum (1M-atom cube: step 1.230 ->
// 1.214 ms against 256-thread blocks, 1.222 ms with 128).
template <typename T, int S>
static void launch_s(Plan* p, const PairArgs<T>& pg, bool vir, bool lb, cudaStream_t st) {
  const int N = (int)p->N;
  const int TB = S == 1 ? kPairAtomBlock : kBlock;
  const long nb = cdiv((long)N * S, TB);
  if (p->sm.n != 2 && !lb) {  // smoothing function other than Eq. (gamma)
    if (vir)
      k_pair<T, true, S, false, true><<<nb, TB, 0, st>>>(
          (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
          p->d_wpart + 6 * p->wpart_pair);
    else
      k_pair<T, false, S, false, true><<<nb, TB, 0, st>>>(
          (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
          p->d_wpart + 6 * p->wpart_pair);
    return;
  }
  if (lb)
    k_pair<T, false, S, true><<<nb, TB, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
        p->d_wpart + 6 * p->wpart_pair, (const T*)p->d_lbw);
  else if (vir)
    k_pair<T, true, S><<<nb, TB, 0, st>>>((const Vec4<T>*)p->d_sorted, p->d_cell_start, N,
                                              pg, (T*)p->d_e0, (T*)p->d_floc,
                                              p->d_wpart + 6 * p->wpart_pair);
  else
    k_pair<T, false, S><<<nb, TB, 0, st>>>((const Vec4<T>*)p->d_sorted, p->d_cell_start, N,
                                               pg, (T*)p->d_e0, (T*)p->d_floc,
                                               p->d_wpart + 6 * p->wpart_pair);
}

template <typename T, int G>
static void launch_w(Plan* p, const PairArgs<T>& pg, bool vir, bool lb, cudaStream_t st) {
  const int N = (int)p->N;
  const long nb = cdiv(cdiv(N, G), kBlock / 32);  // = cdiv(N * (32 / G), kBlock)
  if (lb)
    k_pair_warp<T, false, G, true><<<nb, kBlock, 0, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
        p->d_wpart + 6 * p->wpart_pair, (const T*)p->d_lbw);
  else if (vir)
    k_pair_warp<T, true, G><<<nb, kBlock, 0, st>>>((const Vec4<T>*)p->d_sorted,
                                                   p->d_cell_start, N, pg, (T*)p->d_e0,
                                                   (T*)p->d_floc, p->d_wpart + 6 * p->wpart_pair);
  else
    k_pair_warp<T, false, G><<<nb, kBlock, 0, st>>>((const Vec4<T>*)p->d_sorted,
                                                    p->d_cell_start, N, pg, (T*)p->d_e0,
                                                    (T*)p->d_floc, p->d_wpart + 6 * p->wpart_pair);
}

template <typename T, int G>
static void launch_q(Plan* p, const PairArgs<T>& pg, bool vir, bool lb, cudaStream_t st) {
  const int N = (int)p->N;
  const long nb = pair_blocks(p, 64 * G);
  if (nb == 0) return;
  const size_t sm = q_smem_bytes<T>();
  const int th = kQWarps * 32;
  if (lb)
    k_pair_q<T, false, G, true><<<nb, th, sm, st>>>(
        (const Vec4<T>*)p->d_sorted, p->d_cell_start, N, pg, (T*)p->d_e0, (T*)p->d_floc,
        p->d_wpart + 6 * p->wpart_pair, (const T*)p->d_lbw);
  else if (vir)
    k_pair_q<T, true, G><<<nb, th, sm, st>>>((const Vec4<T>*)p->d_sorted, p->d_cell_start, N,
                                             pg, (T*)p->d_e0, (T*)p->d_floc,
                                             p->d_wpart + 6 * p->wpart_pair);
  else
    k_pair_q<T, false, G><<<nb, th, sm, st>>>((const Vec4<T>*)p->d_sorted, p->d_cell_start, N,
                                              pg, (T*)p->d_e0, (T*)p->d_floc,
                                              p->d_wpart + 6 * p->wpart_pair);
}

template <typename T, int G> static int q_attr() {
  const int sm = (int)q_smem_bytes<T>();
  const auto a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(k_pair_q<T, true, G>, a, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_pair_q<T, false, G>, a, sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_pair_q<T, false, G, true>, a, sm) != cudaSuccess)
    return MLS6_ERR_CUDA;
  return MLS6_OK;
}

// Shared-memory limits of the queue-form instantiations (plan creation,
// outside any stream capture).
template <typename T> int prepare_pair_kernels(Plan*) {
  if (q_attr<T, 2>() || q_attr<T, 4>() || q_attr<T, 8>()) return MLS6_ERR_CUDA;
  return MLS6_OK;
}
#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
template int prepare_pair_kernels<float>(Plan*);
template int prepare_pair_kernels<double>(Plan*);
#endif  // MLS6_DEVICE_ONLY


// Arguments of the pair kernels for a plan.
template <typename T> static PairArgs<T> pair_args(const Plan* p) {
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
  for (int d = 0; d < 3; ++d) {
    pg.Lhi[d] = (T)p->L[d];
    pg.Llo[d] = (T)(p->L[d] - (double)pg.Lhi[d]);
  }
  for (int k = 0; k < 5; ++k) pg.gc[k] = (T)p->sm.c[k];
  for (int k = 0; k < 4; ++k) pg.gd[k] = (T)(-12.0 * (k + 1) * p->sm.c[k + 1]);
  return pg;
}

template <typename T>
static void launch_cl(Plan* p, const PairArgs<T>& pg, bool vir, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    const int N = (int)p->N;
    const long nb = pair_blocks(p, kPairCluster);
    if (nb == 0) return;
    auto k = p->sm.n != 2 ? (vir ? k_pair_cl<true, true> : k_pair_cl<false, true>)
                          : (vir ? k_pair_cl<true, false> : k_pair_cl<false, false>);
    k<<<nb, kBlock, 0, st>>>((const Vec4<float>*)p->d_sorted, p->d_cell_start, N, pg,
                             (float*)p->d_e0, (float*)p->d_floc, p->d_wpart + 6 * p->wpart_pair);
  }
}

template <typename T> int launch_pair(Plan* p, bool vir, cudaStream_t st, bool lb) {
  const PairArgs<T> pg = pair_args<T>(p);
  if (p->pair_split == kPairCluster) {
    // Lorentz-Berthelot and FP64 run the per-atom kernel
    if (lb || sizeof(T) != 4)
      launch_s<T, 1>(p, pg, vir, lb, st);
    else
      launch_cl<T>(p, pg, vir, st);
    return 1;
  }
  switch (p->pair_split) {
    case 512: launch_q<T, 8>(p, pg, vir, lb, st); break;
    case 256: launch_q<T, 4>(p, pg, vir, lb, st); break;
    case 128: launch_q<T, 2>(p, pg, vir, lb, st); break;
    case 32: launch_w<T, 1>(p, pg, vir, lb, st); break;
    case 16: launch_w<T, 2>(p, pg, vir, lb, st); break;
    case 8: launch_s<T, 8>(p, pg, vir, lb, st); break;
    case 4: launch_s<T, 4>(p, pg, vir, lb, st); break;
    case 2: launch_s<T, 2>(p, pg, vir, lb, st); break;
    default: launch_s<T, 1>(p, pg, vir, lb, st); break;
  }
  return 1;
}

#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
template int launch_pair<float>(Plan*, bool, cudaStream_t, bool);
template int launch_pair<double>(Plan*, bool, cudaStream_t, bool);

#endif  // MLS6_DEVICE_ONLY
}  // namespace mls6
