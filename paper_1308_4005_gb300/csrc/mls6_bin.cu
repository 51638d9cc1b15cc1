// Spatial binning of the atoms (the linked-cell structure of Sec. III.D):
// wrap positions into the box, histogram them over cells of width >= a/2,
// exclusive scan of the counts, scatter into cell order, and order each
// cell by input index so that every later sum runs in a reproducible order.
#include <algorithm>
#include <climits>

#include "mls6_device.cuh"

namespace mls6 {


template <typename T> struct BinArgs {
  Box3<T> box;
  T inv_w[3];
  int nc[3];
};

// Also keeps, for the fixed-point anterpolation, the largest |c| in
// flag[4..5] (a double; one atomic maximum per block on its bits, which
// order like the value for non-negative doubles), and, when tsum is given
// (at most kScanDirect tiles), adds the block's atoms per scan tile of
// kScanTile cells to tsum (a shared-memory histogram first, then one
// integer atomic per touched tile).
template <typename T>
__device__ __forceinline__ void k_bin_body(const Blk bk,const T* __restrict__ pos, const T* __restrict__ cc, int stride, int N,
                      BinArgs<T> g, Vec4<T>* __restrict__ posw, int* __restrict__ cell_of,
                      int* __restrict__ count, int* __restrict__ flag, int* __restrict__ tsum,
                      int ntiles) {
  const long z = pdl_begin();
  pos += z; cc += z;
  __shared__ T wmax[32];
  __shared__ int hist[kScanDirect];
  const int i = bk.x * blockDim.x + threadIdx.x;
  if (tsum)
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0;
  __syncthreads();
  T cabs = T(0);
  if (i < N) {
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
    if (tsum) atomicAdd(&hist[cell / kScanTile], 1);
    cabs = fabs(c);
  }
  for (int o = 16; o > 0; o >>= 1) cabs = fmax(cabs, __shfl_xor_sync(0xffffffffu, cabs, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = cabs;
  __syncthreads();
  if (threadIdx.x == 0) {
    T m = T(0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
    atomicMax(reinterpret_cast<unsigned long long*>(flag + 4),
              (unsigned long long)__double_as_longlong((double)m));
  }
  if (tsum)
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
      if (hist[t]) atomicAdd(&tsum[t], hist[t]);
}

template <typename T>
__global__ void k_bin(const T* __restrict__ pos, const T* __restrict__ cc, int stride, int N,
                      BinArgs<T> g, Vec4<T>* __restrict__ posw, int* __restrict__ cell_of,
                      int* __restrict__ count, int* __restrict__ flag, int* __restrict__ tsum,
                      int ntiles) {
  k_bin_body<T>(Blk::self(), pos, cc, stride, N, g, posw, cell_of, count, flag, tsum, ntiles);
}

// Tile pass, for more than kScanDirect tiles: per-tile sums of the cell
// counts; the last block to finish (ticket counter, reset by that block)
// turns them into exclusive tile offsets (block-wide scan, blockDim.x tiles
// at a time with a running carry) and writes the grand total to start[n].
__device__ __forceinline__ void k_scan_tiles_body(const Blk bk,const int* __restrict__ count, long n, int* __restrict__ tsum,
                             int* __restrict__ start, int* __restrict__ flag) {
  const long z = pdl_begin();
  count += z;
  __shared__ int shm[32];
  __shared__ bool last;
  unsigned* ticket = reinterpret_cast<unsigned*>(flag + 2);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const long base = (long)bk.x * kScanTile;
  int s = 0;
  for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
    if (base + t < n) s += count[base + t];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) shm[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < nw; ++w) tot += shm[w];
    tsum[bk.x] = tot;
    __threadfence();
    last = atomicAdd(ticket, 1u) == bk.n - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  int carry = 0;
  for (int t0 = 0; t0 < (int)bk.n; t0 += blockDim.x) {
    const int t = t0 + threadIdx.x;
    const int v = t < (int)bk.n ? ((volatile int*)tsum)[t] : 0;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    __syncthreads();  // shm free (previous chunk / tile sums above)
    if (lane == 31) shm[wid] = incl;
    __syncthreads();
    int wbase = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      const int ws = shm[w];
      if (w < wid) wbase += ws;
      total += ws;
    }
    if (t < (int)bk.n) tsum[t] = carry + wbase + incl - v;
    carry += total;
  }
  if (threadIdx.x == 0) {
    start[n] = carry;
    *ticket = 0u;
  }
}

#ifndef MLS6_DEVICE_ONLY  // non-template kernel, left out where another unit includes this file
__global__ void k_scan_tiles(const int* __restrict__ count, long n, int* __restrict__ tsum,
                             int* __restrict__ start, int* __restrict__ flag) {
  k_scan_tiles_body(Blk::self(), count, n, tsum, start, flag);
}
#else
__global__ void k_scan_tiles(const int* __restrict__ count, long n, int* __restrict__ tsum,
                             int* __restrict__ start, int* __restrict__ flag);
#endif  // MLS6_DEVICE_ONLY

// Scan inside each tile (256 threads x 8 consecutive cells), write start[],
// reset count[] for use as fill counters by the scatter, and keep the
// largest cell population in flag[3] (one atomic maximum per block).  The
// tile's offset is tsum[tile] from the tile pass, or (direct: at most
// kScanDirect tiles, tsum holding the tile sums from the binning) the sum of
// the preceding tiles' sums, formed by each block; the last tile then also
// writes the grand total to start[n].
__device__ __forceinline__ void k_scan_final_body(const Blk bk,int* __restrict__ count, long n, const int* __restrict__ tsum,
                             int* __restrict__ start, int direct, int* __restrict__ flag) {
  const long z = pdl_begin();
  tsum += z;
  __shared__ int wsum[32], wmx[32];
  __shared__ int toff;
  constexpr int PER = kScanTile / 256;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long base = (long)bk.x * kScanTile + (long)threadIdx.x * PER;
  int v[PER], s = 0, mx = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    v[k] = (base + k < n) ? count[base + k] : 0;
    s += v[k];
    mx = max(mx, v[k]);
  }
  int pre = 0;  // direct: this thread's share of the preceding tiles' sums
  if (direct)
    for (int t = threadIdx.x; t < (int)bk.x; t += blockDim.x) pre += tsum[t];
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    pre += __shfl_xor_sync(0xffffffffu, pre, o);
  }
  int incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[wid] = incl;
  if (lane == 0) wmx[wid] = direct ? pre : 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < nw; ++w) acc += wmx[w];
    toff = direct ? acc : tsum[bk.x];
  }
  if (wid == 0) {
    int x = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    wsum[lane] = x;
  }
  __syncthreads();
  if (lane == 0) wmx[wid] = mx;  // wmx read above by thread 0 before this barrier
  int excl = incl - s + (wid > 0 ? wsum[wid - 1] : 0) + toff;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    if (base + k < n) {
      start[base + k] = excl;
      count[base + k] = 0;
    }
    excl += v[k];
  }
  if (direct && threadIdx.x == blockDim.x - 1 && bk.x == bk.n - 1) start[n] = excl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0;
    for (int w = 0; w < nw; ++w) m = max(m, wmx[w]);
    atomicMax(flag + 3, m);
  }
}

#ifndef MLS6_DEVICE_ONLY  // non-template kernel, left out where another unit includes this file
__global__ void k_scan_final(int* __restrict__ count, long n, const int* __restrict__ tsum,
                             int* __restrict__ start, int direct, int* __restrict__ flag) {
  k_scan_final_body(Blk::self(), count, n, tsum, start, direct, flag);
}
#else
__global__ void k_scan_final(int* __restrict__ count, long n, const int* __restrict__ tsum,
                             int* __restrict__ start, int direct, int* __restrict__ flag);
#endif  // MLS6_DEVICE_ONLY

template <typename T>
__device__ __forceinline__ void k_scatter_body(const Blk bk,const Vec4<T>* __restrict__ posw, const int* __restrict__ cell_of, int N,
                          const int* __restrict__ start, int* __restrict__ fill,
                          Vec4<T>* __restrict__ sorted, int* __restrict__ sidx) {
  const long z = pdl_begin();
  posw += z; cell_of += z; start += z;
  int i = bk.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  int cell = cell_of[i];
  int slot = start[cell] + atomicAdd(&fill[cell], 1);
  sorted[slot] = posw[i];
  sidx[slot] = i;
}

template <typename T>
__global__ void k_scatter(const Vec4<T>* __restrict__ posw, const int* __restrict__ cell_of, int N,
                          const int* __restrict__ start, int* __restrict__ fill,
                          Vec4<T>* __restrict__ sorted, int* __restrict__ sidx) {
  k_scatter_body<T>(Blk::self(), posw, cell_of, N, start, fill, sorted, sidx);
}

// Each cell's records sorted by input index, so that every later sum runs
// in an order that does not depend on the scatter's atomics.  Cells of up
// to 8 atoms (nearly all at liquid densities with cells of width a/2) are
// loaded into registers together and sorted by an odd-even transposition
// network; larger cells use an insertion sort in global memory; cells
// above 256 atoms are left in scatter order (results stay correct, only
// bitwise reproducibility is lost for them).  Also returns the cell's
// counter, and the first nreset tile sums, to zero for the next binning.
template <typename T>
__device__ __forceinline__ void k_cellsort_body(const Blk bk,const int* __restrict__ start, long ncell, Vec4<T>* __restrict__ sorted,
                           int* __restrict__ sidx, int* __restrict__ count,
                           int* __restrict__ tsum, int nreset) {
  const long z = pdl_begin();
  start += z;
  long cell = (long)bk.x * blockDim.x + threadIdx.x;
  if (cell < nreset) tsum[cell] = 0;
  if (cell >= ncell) return;
  count[cell] = 0;
  const int b = start[cell], e = start[cell + 1];
  const int n = e - b;
  if (n < 2 || n > 256) return;
  if (n <= 8) {
    int key[8];
    Vec4<T> v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      key[k] = INT_MAX;
      if (k < n) {
        key[k] = sidx[b + k];
        v[k] = sorted[b + k];
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int k = r & 1; k + 1 < 8; k += 2)
        if (key[k] > key[k + 1]) {
          const int tk = key[k];
          key[k] = key[k + 1];
          key[k + 1] = tk;
          const Vec4<T> tv = v[k];
          v[k] = v[k + 1];
          v[k + 1] = tv;
        }
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < n) {
        sidx[b + k] = key[k];
        sorted[b + k] = v[k];
      }
    return;
  }
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

template <typename T>
__global__ void k_cellsort(const int* __restrict__ start, long ncell, Vec4<T>* __restrict__ sorted,
                           int* __restrict__ sidx, int* __restrict__ count,
                           int* __restrict__ tsum, int nreset) {
  k_cellsort_body<T>(Blk::self(), start, ncell, sorted, sidx, count, tsum, nreset);
}

// Arguments of the binning kernel for a plan.
template <typename T> static BinArgs<T> bin_args(const Plan* p) {
  BinArgs<T> bg;
  for (int d = 0; d < 3; ++d) {
    bg.box.L[d] = (T)p->L[d];
    bg.box.invL[d] = (T)(1.0 / p->L[d]);
    bg.inv_w[d] = (T)p->cg.inv_w[d];
    bg.nc[d] = p->cg.nc[d];
  }
  return bg;
}

template <typename T> int launch_bin(Plan* p, const T* pos, const T* cc, cudaStream_t st) {
  const int N = (int)p->N;
  const BinArgs<T> bg = bin_args<T>(p);
  const long ncell = p->cg.ncell;
  const long ntiles = cdiv(ncell, kScanTile);
  // direct: tile sums from the binning (kept zero between binnings by the
  // cell sort; zeroed at plan creation), no tile pass
  const bool direct = ntiles <= kScanDirect;
  // cell counters start at zero: set at plan creation, reset by k_cellsort
  const int nbin = (int)cdiv(N, kBlock);
  launch_pdl(k_bin<T>, nbin, kBlock, 0, st, pos, cc, cc ? 3 : 4, N, bg, (Vec4<T>*)p->d_pos_w,
             p->d_cell_of, p->d_cell_count, p->d_flag, direct ? p->d_scan : (int*)nullptr,
             (int)ntiles);
  if (!direct)
    launch_pdl(k_scan_tiles, ntiles, kBlock, 0, st, (const int*)p->d_cell_count, ncell, p->d_scan,
               p->d_cell_start, p->d_flag);
  launch_pdl(k_scan_final, ntiles, kBlock, 0, st, p->d_cell_count, ncell, (const int*)p->d_scan,
             p->d_cell_start, direct ? 1 : 0, p->d_flag);
  launch_pdl(k_scatter<T>, cdiv(N, kBlock), kBlock, 0, st, (const Vec4<T>*)p->d_pos_w, p->d_cell_of, N,
                                                  p->d_cell_start, p->d_cell_count,
                                                  (Vec4<T>*)p->d_sorted, p->d_sorted_idx);
  launch_pdl(k_cellsort<T>, cdiv(std::max(ncell, ntiles), kBlock), kBlock, 0, st,
             (const int*)p->d_cell_start, ncell, (Vec4<T>*)p->d_sorted, p->d_sorted_idx,
             p->d_cell_count, p->d_scan, direct ? (int)ntiles : 0);
  return direct ? 4 : 5;
}

#ifndef MLS6_DEVICE_ONLY  // host code, left out where another unit includes this file
template int launch_bin<float>(Plan*, const float*, const float*, cudaStream_t);
template int launch_bin<double>(Plan*, const double*, const double*, cudaStream_t);

#endif  // MLS6_DEVICE_ONLY
}  // namespace mls6
