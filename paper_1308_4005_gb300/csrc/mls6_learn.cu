// Learned force correction for a coarse grid (no counterpart in the paper):
// a small network reads, for each atom, the level-1 total potential of a
// coarse multilevel-summation evaluation around the atom and predicts the
// force residual to a finer evaluation; the correction is c_i * s * y_i.
//
//   features   e^{1,tot} and its gradient interpolated (Eq. interpolation,
//              the method's own basis) at x_i + h d for d in {-1,0,1}^3, and
//              sin / cos of 2 pi times the fractional grid coordinate of x_i:
//              114 values, zero-padded to 128, normalised per feature
//              (shift, scale), stored as BF16 (or FP32) rows in input order
//   network    128 -> 64 -> 64 -> 64 -> 8 (outputs 0..2 used), tanh hidden
//              layers; BF16 weights and activations on the tensor cores
//              (mma.m16n8k16, FP32 accumulation); one warp per 16 atoms, the
//              accumulator tiles of a layer are repacked in registers as the
//              A operand of the next
//   training   FP32 backward pass (per-atom activation gradients, per-chunk
//              weight-gradient partials summed in a fixed order, so results
//              are reproducible), Adam update of FP32 master weights, BF16
//              fragments repacked after every step
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "mls6_device.cuh"

namespace mls6 {

#define CK(x)                                    \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return MLS6_ERR_CUDA; \
  } while (0)

static inline long cdiv(long a, long b) { return (a + b - 1) / b; }

constexpr int kNF = 128;                        // feature row (114 used)
constexpr int kH = 64;                          // hidden width
constexpr int kNO = 8;                          // output row (3 used)
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kNF * kH;
constexpr int kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH;
constexpr int kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH;
constexpr int kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + kH * kNO;
constexpr int kNPar = kOffB4 + kNO;             // 17096
// packed B fragments (uint2 per lane): layer 1 8x8 tiles, layers 2-3 4x8, layer 4 4x1
constexpr int kPk1 = 0, kPk2 = kPk1 + 8 * 8 * 32, kPk3 = kPk2 + 4 * 8 * 32,
              kPk4 = kPk3 + 4 * 8 * 32, kPkN = kPk4 + 4 * 1 * 32;
constexpr int kChunk = 512;                     // atoms per weight-gradient partial

struct Mlp {
  float* d_par = nullptr;   // FP32 master weights
  float* d_m = nullptr;     // Adam moments
  float* d_v = nullptr;
  uint2* d_pack = nullptr;  // BF16 B fragments
  float* d_norm = nullptr;  // shift[128], scale[128]
  float out_scale = 1.0f;
  long step = 0;
  cudaStream_t stream = nullptr;
  // work buffers (grown on demand)
  long cap = 0;
  __nv_bfloat16* d_X = nullptr;   // features for mls6_mlp_apply
  float* d_Y = nullptr;           // outputs
  __nv_bfloat16* d_H = nullptr;   // 3 x N x 64 activations (training)
  float* d_D = nullptr;           // 3 x N x 64 activation gradients
  float* d_dY = nullptr;          // N x 8
  float* d_part = nullptr;        // chunks x kNPar partial gradients
  double* d_lpart = nullptr;      // chunks loss partials
  float* d_grad = nullptr;        // kNPar
  double* d_loss = nullptr;
};

__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// ------------------------------------------------------------- features

// One thread per (atom, dz): the 9 offsets (dx, dy) of one dz.  Separable:
// per z row of the basis, an x pass over the 6 y rows of the 6x6 node
// block, then a y pass, then the z weights.  A block (3 x kFA threads)
// assembles the rows of kFA atoms in shared memory and writes each row with
// 16-byte stores (a row per atom in input order, or in sorted order when
// sorted_out is set).
constexpr int kFA = 64;

template <typename T>
__global__ void __launch_bounds__(3 * kFA) k_features(
    const Vec4<T>* __restrict__ sp, const int* __restrict__ sidx, int N, const T* __restrict__ E,
    int n0, int n1, int n2, T ih0, T ih1, T ih2, const float* __restrict__ norm,
    void* __restrict__ out, int f32, int sorted_out) {
  __shared__ __align__(16) float rows[kFA][kNF];
  const int la = threadIdx.x / 3, dz = (int)(threadIdx.x % 3) - 1;
  const int i = blockIdx.x * kFA + la;
  if (i < N) {
    const Vec4<T> p = sp[i];
    const T u0 = p.x * ih0, u1 = p.y * ih1, u2 = p.z * ih2;
    const T f0 = floor(u0), f1 = floor(u1), f2 = floor(u2);
    const int b0 = (int)f0, b1 = (int)f1, b2 = (int)f2;
    T wx[4], dwx[4], wy[4], dwy[4], wz[4], dwz[4];
    phi4(u0 - f0, wx, dwx);
    phi4(u1 - f1, wy, dwy);
    phi4(u2 - f2, wz, dwz);
    T e[9], gx[9], gy[9], gz[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k] = gx[k] = gy[k] = gz[k] = T(0);
    for (int c = 0; c < 4; ++c) {
      const int iz = wrapi(b2 + dz - 1 + c, n2);
      // x pass: rows y = b1-2 .. b1+3, offsets dx = -1..1
      T ax[6][3], bx[6][3];
#pragma unroll
      for (int yy = 0; yy < 6; ++yy) {
        const T* row = E + (long)n0 * (wrapi(b1 - 2 + yy, n1) + (long)n1 * iz);
        T v[6];
#pragma unroll
        for (int xx = 0; xx < 6; ++xx) v[xx] = row[wrapi(b0 - 2 + xx, n0)];
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          T s = 0, ds = 0;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            s += wx[a] * v[dx + a];
            ds += dwx[a] * v[dx + a];
          }
          ax[yy][dx] = s;
          bx[yy][dx] = ds;
        }
      }
      // y pass and z weights
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          T aa = 0, ab = 0, ba = 0;
#pragma unroll
          for (int bb = 0; bb < 4; ++bb) {
            aa += wy[bb] * ax[dy + bb][dx];
            ab += dwy[bb] * ax[dy + bb][dx];
            ba += wy[bb] * bx[dy + bb][dx];
          }
          const int k = dx + 3 * dy;
          e[k] += wz[c] * aa;
          gz[k] += dwz[c] * aa;
          gy[k] += wz[c] * ab;
          gx[k] += wz[c] * ba;
        }
    }
    auto put = [&](int j, float v) { rows[la][j] = (v - norm[j]) * norm[kNF + j]; };
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int idx = k + 9 * (dz + 1);
      put(4 * idx + 0, (float)e[k]);
      put(4 * idx + 1, (float)(gx[k] * ih0));
      put(4 * idx + 2, (float)(gy[k] * ih1));
      put(4 * idx + 3, (float)(gz[k] * ih2));
    }
    if (dz == 0) {
      const float t[3] = {(float)(u0 - f0), (float)(u1 - f1), (float)(u2 - f2)};
      for (int d = 0; d < 3; ++d) {
        float s, co;
        sincospif(2.0f * t[d], &s, &co);
        put(108 + 2 * d, s);
        put(109 + 2 * d, co);
      }
      for (int j = 114; j < kNF; ++j) put(j, 0.0f);
    }
  }
  __syncthreads();
  // rows out: 16-byte chunks (8 bf16 or 4 floats)
  const int per = f32 ? kNF / 4 : kNF / 8;
  for (int t = threadIdx.x; t < kFA * per; t += blockDim.x) {
    const int a = t / per, ch = t % per;
    const int ii = blockIdx.x * kFA + a;
    if (ii >= N) continue;
    const long r = sorted_out ? ii : sidx[ii];
    if (f32) {
      const float4 v = *reinterpret_cast<const float4*>(&rows[a][4 * ch]);
      reinterpret_cast<float4*>(out)[r * (kNF / 4) + ch] = v;
    } else {
      const float* f = &rows[a][8 * ch];
      uint4 v;
      v.x = pack_bf16(f[0], f[1]);
      v.y = pack_bf16(f[2], f[3]);
      v.z = pack_bf16(f[4], f[5]);
      v.w = pack_bf16(f[6], f[7]);
      reinterpret_cast<uint4*>(out)[r * (kNF / 8) + ch] = v;
    }
  }
}

// ----------------------------------------------------------------- network

// B fragment of mma.m16n8k16 for weights W (K x N row-major, row = input):
// lane (g = lane/4, c2 = 2*(lane%4)) holds W[16ks+c2..+1][8nt+g] and
// W[16ks+c2+8..+9][8nt+g].
__global__ void k_mlp_pack(const float* __restrict__ par, uint2* __restrict__ pk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kPkN) return;
  int off, NT, NO, base;
  if (t < kPk2) {
    off = kOffW1; NT = 8; NO = kH; base = kPk1;
  } else if (t < kPk3) {
    off = kOffW2; NT = 8; NO = kH; base = kPk2;
  } else if (t < kPk4) {
    off = kOffW3; NT = 8; NO = kH; base = kPk3;
  } else {
    off = kOffW4; NT = 1; NO = kNO; base = kPk4;
  }
  const int r = t - base, lane = r & 31, tile = r >> 5;
  const int ks = tile / NT, nt = tile % NT;
  const int g = lane >> 2, c2 = (lane & 3) * 2;
  const int n = 8 * nt + g, k = 16 * ks + c2;
  const float* W = par + off;
  uint2 v;
  v.x = pack_bf16(W[(k + 0) * NO + n], W[(k + 1) * NO + n]);
  v.y = pack_bf16(W[(k + 8) * NO + n], W[(k + 9) * NO + n]);
  pk[t] = v;
}

// bias + tanh of accumulator tiles (2 per k-step of the next layer), packed
// as the next layer's A fragments: acc[2ks] gives rows g / g+8 at columns
// c2.., acc[2ks+1] the columns c2+8...
__device__ __forceinline__ void next_a(const float (&acc)[8][4], const float* __restrict__ b,
                                       int c2, uint32_t (&A)[4][4]) {
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int n0 = 16 * ks + c2, n1 = n0 + 8;
    A[ks][0] = pack_bf16(tanh_fast(acc[2 * ks][0] + b[n0]), tanh_fast(acc[2 * ks][1] + b[n0 + 1]));
    A[ks][1] = pack_bf16(tanh_fast(acc[2 * ks][2] + b[n0]), tanh_fast(acc[2 * ks][3] + b[n0 + 1]));
    A[ks][2] = pack_bf16(tanh_fast(acc[2 * ks + 1][0] + b[n1]),
                         tanh_fast(acc[2 * ks + 1][1] + b[n1 + 1]));
    A[ks][3] = pack_bf16(tanh_fast(acc[2 * ks + 1][2] + b[n1]),
                         tanh_fast(acc[2 * ks + 1][3] + b[n1 + 1]));
  }
}

__device__ __forceinline__ void store_act(uint32_t* __restrict__ H, long ra, long rb, bool va,
                                          bool vb, int c2, const uint32_t (&A)[4][4]) {
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int w0 = (16 * ks + c2) >> 1, w1 = (16 * ks + 8 + c2) >> 1;
    if (va) {
      H[ra * (kH / 2) + w0] = A[ks][0];
      H[ra * (kH / 2) + w1] = A[ks][2];
    }
    if (vb) {
      H[rb * (kH / 2) + w0] = A[ks][1];
      H[rb * (kH / 2) + w1] = A[ks][3];
    }
  }
}

__device__ __forceinline__ void hidden_layer(const uint32_t (&A)[4][4], const uint2* __restrict__ sw,
                                             int lane, float (&acc)[8][4]) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[nt][c] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const uint2 b = sw[(ks * 8 + nt) * 32 + lane];
      mma16816(acc[nt], A[ks][0], A[ks][1], A[ks][2], A[ks][3], b.x, b.y);
    }
}

// Forward pass: Y (N x 8) = network(X); with STORE the three hidden
// activations (BF16, N x 64 each) are kept for the backward pass.
template <bool STORE>
__global__ void __launch_bounds__(128) k_mlp_fwd(const __nv_bfloat16* __restrict__ X, long N,
                                                 const uint2* __restrict__ pk,
                                                 const float* __restrict__ par,
                                                 float* __restrict__ Y,
                                                 __nv_bfloat16* __restrict__ H) {
  __shared__ uint2 sw[kPkN];
  __shared__ float sb[3 * kH + kNO];
  for (int i = threadIdx.x; i < kPkN; i += blockDim.x) sw[i] = pk[i];
  for (int i = threadIdx.x; i < kH; i += blockDim.x) {
    sb[i] = par[kOffB1 + i];
    sb[kH + i] = par[kOffB2 + i];
    sb[2 * kH + i] = par[kOffB3 + i];
  }
  if (threadIdx.x < kNO) sb[3 * kH + threadIdx.x] = par[kOffB4 + threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, c2 = (lane & 3) * 2;
  const uint32_t* Xw = reinterpret_cast<const uint32_t*>(X);
  uint32_t* Hw = reinterpret_cast<uint32_t*>(H);
  for (long tile = (long)blockIdx.x * 4 + warp; tile * 16 < N; tile += (long)gridDim.x * 4) {
    const long ra = tile * 16 + g, rb = ra + 8;
    const bool va = ra < N, vb = rb < N;
    // layer 1: K = 128 (8 k-steps), N = 64 (8 tiles)
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[nt][c] = 0.f;
    // all 32 fragment words of the tile's two rows first (loads in flight
    // together), then the 64 products
    uint32_t xa[8][4];
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
      const int w0 = (16 * ks + c2) >> 1, w1 = (16 * ks + 8 + c2) >> 1;
      xa[ks][0] = va ? __ldg(Xw + ra * (kNF / 2) + w0) : 0u;
      xa[ks][1] = vb ? __ldg(Xw + rb * (kNF / 2) + w0) : 0u;
      xa[ks][2] = va ? __ldg(Xw + ra * (kNF / 2) + w1) : 0u;
      xa[ks][3] = vb ? __ldg(Xw + rb * (kNF / 2) + w1) : 0u;
    }
#pragma unroll
    for (int ks = 0; ks < 8; ++ks)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const uint2 b = sw[kPk1 + (ks * 8 + nt) * 32 + lane];
        mma16816(acc[nt], xa[ks][0], xa[ks][1], xa[ks][2], xa[ks][3], b.x, b.y);
      }
    uint32_t A[4][4];
    next_a(acc, sb, c2, A);
    if (STORE) store_act(Hw, ra, rb, va, vb, c2, A);
    hidden_layer(A, sw + kPk2, lane, acc);
    next_a(acc, sb + kH, c2, A);
    if (STORE) store_act(Hw + N * (kH / 2), ra, rb, va, vb, c2, A);
    hidden_layer(A, sw + kPk3, lane, acc);
    next_a(acc, sb + 2 * kH, c2, A);
    if (STORE) store_act(Hw + 2 * N * (kH / 2), ra, rb, va, vb, c2, A);
    // output layer: N = 8 (one tile)
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint2 b = sw[kPk4 + ks * 32 + lane];
      mma16816(o, A[ks][0], A[ks][1], A[ks][2], A[ks][3], b.x, b.y);
    }
    const float* b4 = sb + 3 * kH;
    if (va) {
      Y[ra * kNO + c2] = o[0] + b4[c2];
      Y[ra * kNO + c2 + 1] = o[1] + b4[c2 + 1];
    }
    if (vb) {
      Y[rb * kNO + c2] = o[2] + b4[c2];
      Y[rb * kNO + c2 + 1] = o[3] + b4[c2 + 1];
    }
  }
}

// Backward through the activations (FP32, one thread per atom):
// dY = 2 (y - t) / N on outputs 0..2; dZ3 = (dY W4^T) (1 - h3^2);
// dZ2 = (dZ3 W3^T) (1 - h2^2); dZ1 = (dZ2 W2^T) (1 - h1^2).
__global__ void __launch_bounds__(128) k_mlp_bwd(const float* __restrict__ Y,
                                                 const float* __restrict__ T, long N,
                                                 float inv_n, const __nv_bfloat16* __restrict__ H,
                                                 const float* __restrict__ par,
                                                 float* __restrict__ D, float* __restrict__ dY,
                                                 double* __restrict__ lpart) {
  __shared__ float w2[kH * kH], w3[kH * kH], w4[kH * kNO];
  __shared__ double sh[32];
  for (int i = threadIdx.x; i < kH * kH; i += blockDim.x) {
    w2[i] = par[kOffW2 + i];
    w3[i] = par[kOffW3 + i];
  }
  for (int i = threadIdx.x; i < kH * kNO; i += blockDim.x) w4[i] = par[kOffW4 + i];
  __syncthreads();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < N) {
    float dy[3];
    for (int c = 0; c < 3; ++c) {
      const float r = Y[i * kNO + c] - T[i * 3 + c];
      l += (double)r * r;
      dy[c] = 2.f * r * inv_n;
    }
    for (int c = 0; c < kNO; ++c) dY[i * kNO + c] = c < 3 ? dy[c] : 0.f;
    const __nv_bfloat16* h1 = H + i * kH;
    const __nv_bfloat16* h2 = H + (N + i) * kH;
    const __nv_bfloat16* h3 = H + (2 * N + i) * kH;
    float d3[kH], d2[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      const float h = __bfloat162float(h3[j]);
      d3[j] = (dy[0] * w4[j * kNO] + dy[1] * w4[j * kNO + 1] + dy[2] * w4[j * kNO + 2]) *
              (1.f - h * h);
    }
    for (int j = 0; j < kH; ++j) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kH; ++k) s += d3[k] * w3[j * kH + k];
      const float h = __bfloat162float(h2[j]);
      d2[j] = s * (1.f - h * h);
    }
    float* D1 = D + i * kH;
    float* D2 = D + (N + i) * kH;
    float* D3 = D + (2 * N + i) * kH;
    for (int j = 0; j < kH; ++j) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < kH; ++k) s += d2[k] * w2[j * kH + k];
      const float h = __bfloat162float(h1[j]);
      D1[j] = s * (1.f - h * h);
      D2[j] = d2[j];
      D3[j] = d3[j];
    }
  }
  const double s = block_sum(l, sh);
  if (threadIdx.x == 0) lpart[blockIdx.x] = s;
}

// Weight gradients of one chunk of atoms: dW = sum_i a_i (x) d_i and
// db = sum_i d_i for the four layers (a = X, h1, h2, h3; d = dZ1, dZ2, dZ3,
// dY).  Each thread owns parameters p = tid, tid + blockDim, ...; the
// chunk's rows are staged 16 atoms at a time.
__global__ void __launch_bounds__(256) k_mlp_wgrad(const __nv_bfloat16* __restrict__ X,
                                                   const __nv_bfloat16* __restrict__ H,
                                                   const float* __restrict__ D,
                                                   const float* __restrict__ dY, long N,
                                                   float* __restrict__ part) {
  constexpr int R = 16;
  __shared__ float sa[R][kNF + 3 * kH];   // x, h1, h2, h3
  __shared__ float sd[R][3 * kH + kNO];   // dz1, dz2, dz3, dy
  constexpr int kPer = (kNPar + 255) / 256;
  float acc[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) acc[j] = 0.f;
  const long i0 = (long)blockIdx.x * kChunk, i1 = min(N, i0 + kChunk);
  for (long r0 = i0; r0 < i1; r0 += R) {
    __syncthreads();
    for (int t = threadIdx.x; t < R * (kNF + 3 * kH); t += blockDim.x) {
      const int r = t / (kNF + 3 * kH), c = t % (kNF + 3 * kH);
      const long i = r0 + r;
      float v = 0.f;
      if (i < i1) {
        if (c < kNF)
          v = __bfloat162float(X[i * kNF + c]);
        else {
          const int l = (c - kNF) / kH, j = (c - kNF) % kH;
          v = __bfloat162float(H[((long)l * N + i) * kH + j]);
        }
      }
      sa[r][c] = v;
    }
    for (int t = threadIdx.x; t < R * (3 * kH + kNO); t += blockDim.x) {
      const int r = t / (3 * kH + kNO), c = t % (3 * kH + kNO);
      const long i = r0 + r;
      float v = 0.f;
      if (i < i1) {
        if (c < 3 * kH) {
          const int l = c / kH, j = c % kH;
          v = D[((long)l * N + i) * kH + j];
        } else {
          v = dY[i * kNO + (c - 3 * kH)];
        }
      }
      sd[r][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int p = threadIdx.x + j * 256;
      if (p >= kNPar) break;
      int ac, dc;  // column of a (or -1 for a bias) and of d
      if (p < kOffB1) {
        ac = p / kH; dc = p % kH;
      } else if (p < kOffW2) {
        ac = -1; dc = p - kOffB1;
      } else if (p < kOffB2) {
        ac = kNF + (p - kOffW2) / kH; dc = kH + (p - kOffW2) % kH;
      } else if (p < kOffW3) {
        ac = -1; dc = kH + (p - kOffB2);
      } else if (p < kOffB3) {
        ac = kNF + kH + (p - kOffW3) / kH; dc = 2 * kH + (p - kOffW3) % kH;
      } else if (p < kOffW4) {
        ac = -1; dc = 2 * kH + (p - kOffB3);
      } else if (p < kOffB4) {
        ac = kNF + 2 * kH + (p - kOffW4) / kNO; dc = 3 * kH + (p - kOffW4) % kNO;
      } else {
        ac = -1; dc = 3 * kH + (p - kOffB4);
      }
      float s = 0.f;
      if (ac >= 0)
        for (int r = 0; r < R; ++r) s += sa[r][ac] * sd[r][dc];
      else
        for (int r = 0; r < R; ++r) s += sd[r][dc];
      acc[j] += s;
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int p = threadIdx.x + j * 256;
    if (p < kNPar) part[(long)blockIdx.x * kNPar + p] = acc[j];
  }
}

// Fixed-order sums over the chunks: gradient (FP32 out, summed in FP64)
// and the loss.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nchunk,
                             const double* __restrict__ lpart, int nl, double inv_n,
                             float* __restrict__ grad, double* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNPar) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += (double)part[(long)c * kNPar + p];
    grad[p] = (float)s;
  }
  if (p == 0) {
    double s = 0.0;
    for (int c = 0; c < nl; ++c) s += lpart[c];
    *loss = s * inv_n;
  }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8); outputs 3..7 stay zero.
__global__ void k_adam(float* __restrict__ par, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, float lr, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNPar) return;
  bool frozen = false;
  if (p >= kOffW4 && p < kOffB4) frozen = ((p - kOffW4) % kNO) >= 3;
  if (p >= kOffB4) frozen = (p - kOffB4) >= 3;
  if (frozen) {
    par[p] = 0.f;
    return;
  }
  const float gi = g[p];
  const float mi = 0.9f * m[p] + 0.1f * gi;
  const float vi = 0.999f * v[p] + 0.001f * gi * gi;
  m[p] = mi;
  v[p] = vi;
  par[p] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

// forces_o += c_o * s * y_i for the atom o at sorted position i (outputs in
// sorted order, forces in input order)
template <typename T>
__global__ void k_mlp_correct(const Vec4<T>* __restrict__ sp, const int* __restrict__ sidx,
                              const float* __restrict__ Y, int N, float s, T* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T c = sp[i].w * (T)s;
  const size_t o = (size_t)sidx[i];
  F[3 * o + 0] += c * (T)Y[(size_t)i * kNO + 0];
  F[3 * o + 1] += c * (T)Y[(size_t)i * kNO + 1];
  F[3 * o + 2] += c * (T)Y[(size_t)i * kNO + 2];
}

// ------------------------------------------------------------------ host

static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static int grow(Mlp* m, long N) {
  if (N <= m->cap) return MLS6_OK;
  void* bufs[] = {m->d_X, m->d_Y, m->d_H, m->d_D, m->d_dY, m->d_part, m->d_lpart};
  for (void* b : bufs)
    if (b) cudaFree(b);
  m->d_X = nullptr;
  m->d_Y = nullptr;
  m->d_H = nullptr;
  m->d_D = nullptr;
  m->d_dY = nullptr;
  m->d_part = nullptr;
  m->d_lpart = nullptr;
  m->cap = 0;
  const long nch = cdiv(N, kChunk), nbl = cdiv(N, 128);
  if (cudaMalloc((void**)&m->d_X, sizeof(__nv_bfloat16) * kNF * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_Y, sizeof(float) * kNO * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_H, sizeof(__nv_bfloat16) * 3 * kH * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_D, sizeof(float) * 3 * kH * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_dY, sizeof(float) * kNO * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_part, sizeof(float) * kNPar * nch) != cudaSuccess ||
      cudaMalloc((void**)&m->d_lpart, sizeof(double) * nbl) != cudaSuccess)
    return MLS6_ERR_NOMEM;
  m->cap = N;
  return MLS6_OK;
}

static int repack(Mlp* m) {
  k_mlp_pack<<<cdiv(kPkN, 256), 256, 0, m->stream>>>(m->d_par, m->d_pack);
  CK(cudaGetLastError());
  return MLS6_OK;
}

static int forward(Mlp* m, const void* X, long N, float* Y, bool store) {
  if (N <= 0) return MLS6_OK;
  const long tiles = cdiv(N, 16);
  const long nb = std::min(cdiv(tiles, 4), 152L * 8);
  if (store)
    k_mlp_fwd<true><<<nb, 128, 0, m->stream>>>((const __nv_bfloat16*)X, N, m->d_pack, m->d_par,
                                               Y, m->d_H);
  else
    k_mlp_fwd<false><<<nb, 128, 0, m->stream>>>((const __nv_bfloat16*)X, N, m->d_pack,
                                                m->d_par, Y, nullptr);
  CK(cudaGetLastError());
  return MLS6_OK;
}

static int gradient(Mlp* m, const void* X, const float* T, long N) {
  int rc = grow(m, N);
  if (rc) return rc;
  rc = forward(m, X, N, m->d_Y, true);
  if (rc) return rc;
  const long nbl = cdiv(N, 128), nch = cdiv(N, kChunk);
  k_mlp_bwd<<<nbl, 128, 0, m->stream>>>(m->d_Y, T, N, 1.0f / (float)N, m->d_H, m->d_par, m->d_D,
                                        m->d_dY, m->d_lpart);
  k_mlp_wgrad<<<nch, 256, 0, m->stream>>>((const __nv_bfloat16*)X, m->d_H, m->d_D, m->d_dY, N,
                                          m->d_part);
  k_mlp_reduce<<<cdiv(kNPar, 256), 256, 0, m->stream>>>(m->d_part, (int)nch, m->d_lpart,
                                                       (int)nbl, 1.0 / (double)N, m->d_grad,
                                                       m->d_loss);
  CK(cudaGetLastError());
  return MLS6_OK;
}

static int read_loss(Mlp* m, double* loss) {
  if (!loss) return MLS6_OK;
  CK(cudaMemcpyAsync(loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return MLS6_OK;
}

static void free_mlp(Mlp* m) {
  if (!m) return;
  void* bufs[] = {m->d_par, m->d_m, m->d_v, m->d_pack, m->d_norm, m->d_X, m->d_Y, m->d_H,
                  m->d_D, m->d_dY, m->d_part, m->d_lpart, m->d_grad, m->d_loss};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete m;
}

template <typename T>
static int features_t(Plan* p, Mlp* m, void* out, int f32, bool sorted_out, cudaStream_t st) {
  const Level& L1 = p->lv[1];
  const int N = (int)p->N;
  if (N == 0) return MLS6_OK;
  k_features<T><<<cdiv(N, kFA), 3 * kFA, 0, st>>>(
      (const Vec4<T>*)p->d_sorted, p->d_sorted_idx, N, (const T*)p->d_et[1], L1.n[0], L1.n[1],
      L1.n[2], (T)(1.0 / L1.h[0]), (T)(1.0 / L1.h[1]), (T)(1.0 / L1.h[2]), m->d_norm, out, f32,
      sorted_out ? 1 : 0);
  CK(cudaGetLastError());
  return MLS6_OK;
}

}  // namespace mls6

using namespace mls6;

extern "C" {

int mls6_mlp_n_params(void) { return kNPar; }

int mls6_mlp_create(mls6_mlp_t** out, uint64_t seed) {
  if (!out) return MLS6_ERR_ARG;
  *out = nullptr;
  Mlp* m = new (std::nothrow) Mlp();
  if (!m) return MLS6_ERR_NOMEM;
  if (cudaMalloc((void**)&m->d_par, sizeof(float) * kNPar) != cudaSuccess ||
      cudaMalloc((void**)&m->d_m, sizeof(float) * kNPar) != cudaSuccess ||
      cudaMalloc((void**)&m->d_v, sizeof(float) * kNPar) != cudaSuccess ||
      cudaMalloc((void**)&m->d_grad, sizeof(float) * kNPar) != cudaSuccess ||
      cudaMalloc((void**)&m->d_pack, sizeof(uint2) * kPkN) != cudaSuccess ||
      cudaMalloc((void**)&m->d_norm, sizeof(float) * 2 * kNF) != cudaSuccess ||
      cudaMalloc((void**)&m->d_loss, sizeof(double)) != cudaSuccess) {
    free_mlp(m);
    return MLS6_ERR_NOMEM;
  }
  // Glorot-uniform weights from SplitMix64, zero biases, outputs 3..7 zero
  std::vector<float> p(kNPar, 0.f);
  uint64_t s = seed;
  auto fill = [&](int off, int K, int Nn, int used) {
    const double lim = std::sqrt(6.0 / (K + used));
    for (int k = 0; k < K; ++k)
      for (int n = 0; n < Nn; ++n) {
        const double u = (double)(splitmix64(s) >> 11) * 0x1.0p-53;
        p[off + k * Nn + n] = n < used ? (float)((2.0 * u - 1.0) * lim) : 0.f;
      }
  };
  fill(kOffW1, kNF, kH, kH);
  fill(kOffW2, kH, kH, kH);
  fill(kOffW3, kH, kH, kH);
  fill(kOffW4, kH, kNO, 3);
  std::vector<float> norm(2 * kNF, 0.f);
  for (int j = 0; j < kNF; ++j) norm[kNF + j] = 1.f;
  if (cudaMemcpy(m->d_par, p.data(), sizeof(float) * kNPar, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(m->d_norm, norm.data(), sizeof(float) * 2 * kNF, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemset(m->d_m, 0, sizeof(float) * kNPar) != cudaSuccess ||
      cudaMemset(m->d_v, 0, sizeof(float) * kNPar) != cudaSuccess || repack(m) != MLS6_OK ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    free_mlp(m);
    return MLS6_ERR_CUDA;
  }
  *out = reinterpret_cast<mls6_mlp_t*>(m);
  return MLS6_OK;
}

int mls6_mlp_set_stream(mls6_mlp_t* mm, void* stream) {
  if (!mm) return MLS6_ERR_ARG;
  reinterpret_cast<Mlp*>(mm)->stream = (cudaStream_t)stream;
  return MLS6_OK;
}

int mls6_mlp_get_params(const mls6_mlp_t* mm, float* host, int n) {
  if (!mm || !host || n != kNPar) return MLS6_ERR_ARG;
  const Mlp* m = reinterpret_cast<const Mlp*>(mm);
  CK(cudaStreamSynchronize(m->stream));
  CK(cudaMemcpy(host, m->d_par, sizeof(float) * kNPar, cudaMemcpyDeviceToHost));
  return MLS6_OK;
}

int mls6_mlp_set_params(mls6_mlp_t* mm, const float* host, int n) {
  if (!mm || !host || n != kNPar) return MLS6_ERR_ARG;
  Mlp* m = reinterpret_cast<Mlp*>(mm);
  CK(cudaStreamSynchronize(m->stream));
  CK(cudaMemcpy(m->d_par, host, sizeof(float) * kNPar, cudaMemcpyHostToDevice));
  CK(cudaMemset(m->d_m, 0, sizeof(float) * kNPar));
  CK(cudaMemset(m->d_v, 0, sizeof(float) * kNPar));
  m->step = 0;
  return repack(m);
}

int mls6_mlp_set_norm(mls6_mlp_t* mm, const float* shift, const float* scale, float out_scale) {
  if (!mm || !shift || !scale || !std::isfinite(out_scale)) return MLS6_ERR_ARG;
  Mlp* m = reinterpret_cast<Mlp*>(mm);
  std::vector<float> norm(2 * kNF);
  for (int j = 0; j < kNF; ++j) {
    norm[j] = shift[j];
    norm[kNF + j] = scale[j];
  }
  CK(cudaStreamSynchronize(m->stream));
  CK(cudaMemcpy(m->d_norm, norm.data(), sizeof(float) * 2 * kNF, cudaMemcpyHostToDevice));
  m->out_scale = out_scale;
  return MLS6_OK;
}

int mls6_mlp_features(mls6_plan_t* plan, const mls6_mlp_t* mm, void* out, int fmt) {
  if (!plan || !mm || (fmt != 0 && fmt != 1)) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (p->N > 0 && !out) return MLS6_ERR_ARG;
  Mlp* m = const_cast<Mlp*>(reinterpret_cast<const Mlp*>(mm));
  return p->prec == MLS6_FP64 ? features_t<double>(p, m, out, fmt, false, p->stream)
                              : features_t<float>(p, m, out, fmt, false, p->stream);
}

int mls6_mlp_forward(mls6_mlp_t* mm, const void* X, int64_t N, float* Y) {
  if (!mm || N < 0 || (N > 0 && (!X || !Y))) return MLS6_ERR_ARG;
  return forward(reinterpret_cast<Mlp*>(mm), X, N, Y, false);
}

int mls6_mlp_grad(mls6_mlp_t* mm, const void* X, const float* T, int64_t N, float* grad,
                  double* loss) {
  if (!mm || N < 1 || !X || !T) return MLS6_ERR_ARG;
  Mlp* m = reinterpret_cast<Mlp*>(mm);
  int rc = gradient(m, X, T, N);
  if (rc) return rc;
  if (grad)
    CK(cudaMemcpyAsync(grad, m->d_grad, sizeof(float) * kNPar, cudaMemcpyDeviceToDevice,
                       m->stream));
  return read_loss(m, loss);
}

int mls6_mlp_train_step(mls6_mlp_t* mm, const void* X, const float* T, int64_t N, float lr,
                        double* loss) {
  if (!mm || N < 1 || !X || !T || !(lr > 0.f)) return MLS6_ERR_ARG;
  Mlp* m = reinterpret_cast<Mlp*>(mm);
  int rc = gradient(m, X, T, N);
  if (rc) return rc;
  m->step += 1;
  const float bc1 = 1.f - (float)std::pow(0.9, (double)m->step);
  const float bc2 = 1.f - (float)std::pow(0.999, (double)m->step);
  k_adam<<<cdiv(kNPar, 256), 256, 0, m->stream>>>(m->d_par, m->d_m, m->d_v, m->d_grad, lr, bc1,
                                                  bc2);
  CK(cudaGetLastError());
  rc = repack(m);
  if (rc) return rc;
  return read_loss(m, loss);
}

int mls6_mlp_apply(mls6_plan_t* plan, mls6_mlp_t* mm, void* forces) {
  if (!plan || !mm) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  Mlp* m = reinterpret_cast<Mlp*>(mm);
  const long N = p->N;
  if (N == 0) return MLS6_OK;
  if (!forces) return MLS6_ERR_ARG;
  int rc = grow(m, N);
  if (rc) return rc;
  cudaStream_t saved = m->stream;
  m->stream = p->stream;
  rc = p->prec == MLS6_FP64 ? features_t<double>(p, m, m->d_X, 0, true, p->stream)
                            : features_t<float>(p, m, m->d_X, 0, true, p->stream);
  if (!rc) rc = forward(m, m->d_X, N, m->d_Y, false);
  m->stream = saved;
  if (rc) return rc;
  if (p->prec == MLS6_FP64)
    k_mlp_correct<double><<<cdiv(N, 256), 256, 0, p->stream>>>(
        (const Vec4<double>*)p->d_sorted, p->d_sorted_idx, m->d_Y, (int)N, m->out_scale,
        (double*)forces);
  else
    k_mlp_correct<float><<<cdiv(N, 256), 256, 0, p->stream>>>(
        (const Vec4<float>*)p->d_sorted, p->d_sorted_idx, m->d_Y, (int)N, m->out_scale,
        (float*)forces);
  CK(cudaGetLastError());
  return MLS6_OK;
}

void mls6_mlp_destroy(mls6_mlp_t* mm) { free_mlp(reinterpret_cast<Mlp*>(mm)); }

}  // extern "C"
