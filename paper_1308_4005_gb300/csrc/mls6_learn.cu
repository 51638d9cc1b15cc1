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
//   training   BF16 tensor-core backward pass: activation gradients
//              dZ = (dZ_next W^T) (1 - h^2) per 16-atom warp tile with the
//              transposed weights as B fragments (mma.m16n8k16, FP32
//              accumulation, dZ kept as BF16); weight gradients X^T dZ1,
//              H^T dZ per block of atoms from shared-memory tiles read as
//              transposed fragments (ldmatrix .trans), bias gradients as
//              products with a ones operand; per-block partials summed in a
//              fixed order (results reproducible bit for bit); Adam update of
//              FP32 master weights, BF16 fragments repacked after every step
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
// transposed weights for the backward pass (B[k][n] = W[n][k]): W4^T one
// k-step (K = 8 padded to 16) x 8 tiles, W3^T and W2^T 4 x 8
constexpr int kPkT4 = kPkN, kPkT3 = kPkT4 + 1 * 8 * 32, kPkT2 = kPkT3 + 4 * 8 * 32,
              kPkAll = kPkT2 + 4 * 8 * 32;
// weight gradients: blocks of kWB atoms staged in shared memory, at most
// kWGrid thread blocks (partials), rows padded by 8 BF16 (16 bytes) so the
// eight rows an ldmatrix reads fall in distinct banks
constexpr int kWB = 64, kWGrid = 152;
constexpr int kXS = kNF + 8, kHS = kH + 8;
constexpr int kWStage = kWB * (kXS + 6 * kHS + kNO);  // BF16 elements per stage

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
  __nv_bfloat16* d_D = nullptr;   // 3 x N x 64 activation gradients dZ1..dZ3
  __nv_bfloat16* d_dY = nullptr;  // N x 8 output gradients
  float* d_part = nullptr;        // blocks x kNPar partial gradients
  double* d_lpart = nullptr;      // loss partials, one per backward block
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
    int ixw[6], iyw[6];  // wrapped x and y node indices, b - 2 .. b + 3
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      ixw[k] = wrapi(b0 - 2 + k, n0);
      iyw[k] = wrapi(b1 - 2 + k, n1);
    }
    for (int c = 0; c < 4; ++c) {
      const int iz = wrapi(b2 + dz - 1 + c, n2);
      // x pass: rows y = b1-2 .. b1+3, offsets dx = -1..1
      T ax[6][3], bx[6][3];
#pragma unroll
      for (int yy = 0; yy < 6; ++yy) {
        const T* row = E + (long)n0 * (iyw[yy] + (long)n1 * iz);
        T v[6];
#pragma unroll
        for (int xx = 0; xx < 6; ++xx) v[xx] = row[ixw[xx]];
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
// Transposed (backward) fragments: B[k][n] = W[n][k] for W = W4, W3, W2
// (row = input n, column = output k); k >= the layer's outputs is zero.
__device__ __forceinline__ float wt_at(const float* W, int NO, int k, int n) {
  return k < NO ? W[n * NO + k] : 0.f;
}

__global__ void k_mlp_pack(const float* __restrict__ par, uint2* __restrict__ pk) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kPkAll) return;
  if (t >= kPkN) {
    int off, NO, base;
    if (t < kPkT3) {
      off = kOffW4; NO = kNO; base = kPkT4;
    } else if (t < kPkT2) {
      off = kOffW3; NO = kH; base = kPkT3;
    } else {
      off = kOffW2; NO = kH; base = kPkT2;
    }
    const int r = t - base, lane = r & 31, tile = r >> 5;
    const int ks = tile / 8, nt = tile % 8;
    const int g = lane >> 2, c2 = (lane & 3) * 2;
    const int n = 8 * nt + g, k = 16 * ks + c2;
    const float* W = par + off;
    uint2 v;
    v.x = pack_bf16(wt_at(W, NO, k, n), wt_at(W, NO, k + 1, n));
    v.y = pack_bf16(wt_at(W, NO, k + 8, n), wt_at(W, NO, k + 9, n));
    pk[t] = v;
    return;
  }
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

// Backward through the activations on the tensor cores, one warp per
// 16-atom tile (the forward pass's tiling): dY = 2 (y - t) / N on outputs
// 0..2 (BF16, stored for the weight gradients), then per layer
//   dZ3 = (dY W4^T) (1 - h3^2),  dZ2 = (dZ3 W3^T) (1 - h2^2),
//   dZ1 = (dZ2 W2^T) (1 - h1^2),
// each product an mma over the transposed-weight fragments with FP32
// accumulators; the factor (1 - h^2) uses the stored BF16 activations at
// the accumulator positions, and the result is packed (BF16) both as the
// next layer's A fragments and into D for the weight gradients.  Loss
// partials: one per block, summed in a fixed order by k_mlp_reduce.
__device__ __forceinline__ void act_grad(const float (&acc)[8][4], const uint32_t* __restrict__ Hl,
                                         long ra, long rb, bool va, bool vb, int c2,
                                         uint32_t* __restrict__ Dl, uint32_t (&A)[4][4]) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int w = (8 * nt + c2) >> 1;
    float ha0 = 0.f, ha1 = 0.f, hb0 = 0.f, hb1 = 0.f;
    if (va) {
      const uint32_t u = Hl[ra * (kH / 2) + w];
      const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&u);
      ha0 = __low2float(h);
      ha1 = __high2float(h);
    }
    if (vb) {
      const uint32_t u = Hl[rb * (kH / 2) + w];
      const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&u);
      hb0 = __low2float(h);
      hb1 = __high2float(h);
    }
    const uint32_t pa = pack_bf16(acc[nt][0] * (1.f - ha0 * ha0), acc[nt][1] * (1.f - ha1 * ha1));
    const uint32_t pb = pack_bf16(acc[nt][2] * (1.f - hb0 * hb0), acc[nt][3] * (1.f - hb1 * hb1));
    // tile nt is half (nt & 1) of k-step nt / 2 of the next product
    A[nt >> 1][(nt & 1) * 2 + 0] = pa;
    A[nt >> 1][(nt & 1) * 2 + 1] = pb;
    if (va) Dl[ra * (kH / 2) + w] = pa;
    if (vb) Dl[rb * (kH / 2) + w] = pb;
  }
}

__device__ __forceinline__ void back_product(const uint32_t (&A)[4][4],
                                             const uint2* __restrict__ sw, int lane,
                                             float (&acc)[8][4]) {
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

__global__ void __launch_bounds__(128) k_mlp_bwd(const float* __restrict__ Y,
                                                 const float* __restrict__ T, long N,
                                                 float inv_n, const __nv_bfloat16* __restrict__ H,
                                                 const uint2* __restrict__ pk,
                                                 __nv_bfloat16* __restrict__ D,
                                                 __nv_bfloat16* __restrict__ dYb,
                                                 double* __restrict__ lpart) {
  constexpr int kT = kPkAll - kPkN;
  __shared__ uint2 sw[kT];
  __shared__ double sh[32];
  for (int i = threadIdx.x; i < kT; i += blockDim.x) sw[i] = pk[kPkN + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, c2 = (lane & 3) * 2;
  const uint32_t* Hw = reinterpret_cast<const uint32_t*>(H);
  uint32_t* Dw = reinterpret_cast<uint32_t*>(D);
  uint32_t* dYw = reinterpret_cast<uint32_t*>(dYb);
  double l = 0.0;
  for (long tile = (long)blockIdx.x * 4 + warp; tile * 16 < N; tile += (long)gridDim.x * 4) {
    const long ra = tile * 16 + g, rb = ra + 8;
    const bool va = ra < N, vb = rb < N;
    float dy[4] = {0.f, 0.f, 0.f, 0.f};  // (ra, c2), (ra, c2+1), (rb, c2), (rb, c2+1)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long r = q < 2 ? ra : rb;
      const int c = c2 + (q & 1);
      if ((q < 2 ? va : vb) && c < 3) {
        const float e = Y[r * kNO + c] - T[r * 3 + c];
        l += (double)e * e;
        dy[q] = 2.f * e * inv_n;
      }
    }
    const uint32_t da = pack_bf16(dy[0], dy[1]), db = pack_bf16(dy[2], dy[3]);
    if (va) dYw[ra * (kNO / 2) + (c2 >> 1)] = da;
    if (vb) dYw[rb * (kNO / 2) + (c2 >> 1)] = db;
    // dY W4^T: one k-step, columns 8..15 of A are zero
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
      const uint2 b = sw[(kPkT4 - kPkN) + nt * 32 + lane];
      mma16816(acc[nt], da, db, 0u, 0u, b.x, b.y);
    }
    uint32_t A[4][4];
    act_grad(acc, Hw + 2 * N * (kH / 2), ra, rb, va, vb, c2, Dw + 2 * N * (kH / 2), A);
    back_product(A, sw + (kPkT3 - kPkN), lane, acc);
    act_grad(acc, Hw + N * (kH / 2), ra, rb, va, vb, c2, Dw + N * (kH / 2), A);
    back_product(A, sw + (kPkT2 - kPkN), lane, acc);
    act_grad(acc, Hw, ra, rb, va, vb, c2, Dw, A);
  }
  const double s = block_sum(l, sh);
  if (threadIdx.x == 0) lpart[blockIdx.x] = s;
}

// Weight gradients on the tensor cores.  Thread block c sums the atoms of
// blocks [c per, (c+1) per) of kWB atoms (per = ceil(blocks / kWGrid)):
//   dW1 = X^T dZ1 (128 x 64), dW2 = H1^T dZ2, dW3 = H2^T dZ3 (64 x 64),
//   dW4 = H3^T dY (64 x 8), db = column sums of dZ1, dZ2, dZ3, dY.
// Each block of atoms is copied (cp.async, 16-byte pieces, rows past N
// zero-filled) into one of two shared-memory stages while the other is
// used.  Atoms are the K dimension: the A operand (activations transposed)
// and the B operand (gradients) are both read from row-major [atom][column]
// tiles with ldmatrix .trans.  Warp w owns rows 16w.. of dW1, rows 16w.. of
// dW2 and dW4 (w < 4) or of dW3 (w >= 4); the bias sums are mma products
// with an all-ones A (every row of the result is the column sum), taken by
// warps 0 (b2), 1 (b4), 4 (b1), 5 (b3) from fragments they already hold.
// The partial of block c is written to part[c][*]; k_mlp_reduce sums the
// partials in block order, so the result is reproducible bit for bit.
__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void ldsm2t(uint32_t (&r)[2], const void* p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(a));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}

// A fragments of rows 16 m0.. (the activation columns) for k-step ks of a
// stage tile [atom][column] with row stride S: matrices (atoms 0-7 / 8-15)
// x (columns 0-7 / 8-15) in the order a0 a1 a2 a3 of the mma.
template <int S>
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* t, int ks, int m0,
                                       int lane) {
  const int j = lane >> 3, r = lane & 7;
  ldsm4t(a, t + (16 * ks + r + 8 * (j >> 1)) * S + 16 * m0 + 8 * (j & 1));
}

// B fragments of column tiles nt0, nt0+1 for k-step ks: b[0..1] for nt0,
// b[2..3] for nt0+1.
template <int S>
__device__ __forceinline__ void frag_b2(uint32_t (&b)[4], const __nv_bfloat16* t, int ks, int nt0,
                                        int lane) {
  const int j = lane >> 3, r = lane & 7;
  ldsm4t(b, t + (16 * ks + r + 8 * (j & 1)) * S + 8 * (nt0 + (j >> 1)));
}

__global__ void __launch_bounds__(256) k_mlp_wgrad(const __nv_bfloat16* __restrict__ X,
                                                   const __nv_bfloat16* __restrict__ H,
                                                   const __nv_bfloat16* __restrict__ D,
                                                   const __nv_bfloat16* __restrict__ dY, long N,
                                                   long per, float* __restrict__ part) {
  extern __shared__ __align__(16) __nv_bfloat16 stg[];  // two stages of kWStage
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, c2 = (lane & 3) * 2;
  const long nblk = cdiv(N, (long)kWB);
  const long b0 = (long)blockIdx.x * per, b1 = min(nblk, b0 + per);
  // stage layout: X [kWB][kXS], H1..H3 [kWB][kHS], dZ1..dZ3 [kWB][kHS], dY [kWB][kNO]
  auto sx = [&](int st) { return stg + (size_t)st * kWStage; };
  auto sh = [&](int st, int l) { return sx(st) + kWB * kXS + l * kWB * kHS; };
  auto sd = [&](int st, int l) { return sx(st) + kWB * kXS + (3 + l) * kWB * kHS; };
  auto sy = [&](int st) { return sx(st) + kWB * kXS + 6 * kWB * kHS; };
  auto stage = [&](int st, long blk) {
    const long r0 = blk * kWB;
    constexpr int kPieces = kNF / 8 + 6 * (kH / 8) + 1;  // 16-byte pieces per atom row
    for (int t = threadIdx.x; t < kWB * kPieces; t += blockDim.x) {
      const int r = t / kPieces, q = t % kPieces;
      const long i = r0 + r;
      const bool ok = i < N;
      const long ic = ok ? i : 0;
      const __nv_bfloat16* src;
      __nv_bfloat16* dst;
      if (q < kNF / 8) {
        src = X + ic * kNF + 8 * q;
        dst = sx(st) + r * kXS + 8 * q;
      } else if (q < kNF / 8 + 6 * (kH / 8)) {
        const int u = q - kNF / 8, l = u / (kH / 8), c = u % (kH / 8);
        src = (l < 3 ? H + ((long)l * N + ic) * kH : D + ((long)(l - 3) * N + ic) * kH) + 8 * c;
        dst = (l < 3 ? sh(st, l) : sd(st, l - 3)) + r * kHS + 8 * c;
      } else {
        src = dY + ic * kNO;
        dst = sy(st) + r * kNO;
      }
      cp_async16(dst, src, ok ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  float a1[8][4], a23[8][4], a4[4], ab[8][4];
#pragma unroll
  for (int n = 0; n < 8; ++n)
#pragma unroll
    for (int c = 0; c < 4; ++c) a1[n][c] = a23[n][c] = ab[n][c] = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) a4[c] = 0.f;
  const uint32_t one = 0x3F803F80u;  // two BF16 ones

  if (b0 < b1) stage(0, b0);
  for (long blk = b0; blk < b1; ++blk) {
    const int st = (int)((blk - b0) & 1);
    if (blk + 1 < b1) {
      stage(st ^ 1, blk + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const int l23 = warp < 4 ? 0 : 1;           // dW2 (H1, dZ2) or dW3 (H2, dZ3)
    const int m23 = warp & 3;
#pragma unroll
    for (int ks = 0; ks < kWB / 16; ++ks) {
      uint32_t a[4], b[4][4];
      // dW1 rows 16 warp..: X^T dZ1
      frag_a<kXS>(a, sx(st), ks, warp, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) frag_b2<kHS>(b[q], sd(st, 0), ks, 2 * q, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        mma16816(a1[2 * q], a[0], a[1], a[2], a[3], b[q][0], b[q][1]);
        mma16816(a1[2 * q + 1], a[0], a[1], a[2], a[3], b[q][2], b[q][3]);
      }
      if (warp == 4)  // b1: column sums of dZ1
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          mma16816(ab[2 * q], one, one, one, one, b[q][0], b[q][1]);
          mma16816(ab[2 * q + 1], one, one, one, one, b[q][2], b[q][3]);
        }
      // dW2 (warps 0-3) / dW3 (warps 4-7)
      frag_a<kHS>(a, sh(st, l23), ks, m23, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) frag_b2<kHS>(b[q], sd(st, 1 + l23), ks, 2 * q, lane);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        mma16816(a23[2 * q], a[0], a[1], a[2], a[3], b[q][0], b[q][1]);
        mma16816(a23[2 * q + 1], a[0], a[1], a[2], a[3], b[q][2], b[q][3]);
      }
      if (warp == 0 || warp == 5)  // b2 (dZ2) / b3 (dZ3)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          mma16816(ab[2 * q], one, one, one, one, b[q][0], b[q][1]);
          mma16816(ab[2 * q + 1], one, one, one, one, b[q][2], b[q][3]);
        }
      if (warp < 4) {  // dW4 rows 16 warp..: H3^T dY (one column tile)
        uint32_t by[2];
        {
          const int j = (lane >> 3) & 1, r = lane & 7;
          ldsm2t(by, sy(st) + (16 * ks + r + 8 * j) * kNO);
        }
        frag_a<kHS>(a, sh(st, 2), ks, warp, lane);
        mma16816(a4, a[0], a[1], a[2], a[3], by[0], by[1]);
        if (warp == 1) mma16816(ab[0], one, one, one, one, by[0], by[1]);  // b4
      }
    }
    __syncthreads();  // the stage is refilled two iterations later
  }

  // partial of this block, parameter order of the master weights
  float* P = part + (long)blockIdx.x * kNPar;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = g + 8 * (c >> 1), n = 8 * nt + c2 + (c & 1);
      P[kOffW1 + (16 * warp + m) * kH + n] = a1[nt][c];
      P[(warp < 4 ? kOffW2 : kOffW3) + (16 * (warp & 3) + m) * kH + n] = a23[nt][c];
    }
  if (warp < 4)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      P[kOffW4 + (16 * warp + g + 8 * (c >> 1)) * kNO + c2 + (c & 1)] = a4[c];
  if (g == 0) {  // row 0 of the ones products
    if (warp == 4 || warp == 0 || warp == 5)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int off = warp == 4 ? kOffB1 : (warp == 0 ? kOffB2 : kOffB3);
        P[off + 8 * nt + c2] = ab[nt][0];
        P[off + 8 * nt + c2 + 1] = ab[nt][1];
      }
    if (warp == 1) {
      P[kOffB4 + c2] = ab[0][0];
      P[kOffB4 + c2 + 1] = ab[0][1];
    }
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

// Launch geometry of the training kernels (a function of N only, so the
// partial sums and hence the results do not depend on the device).
static long fwd_blocks(long N) { return std::min(cdiv(cdiv(N, 16L), 4L), 152L * 8); }
static long bwd_blocks(long N) { return fwd_blocks(N); }
static void wgrad_geometry(long N, long& grid, long& per) {
  const long nblk = cdiv(N, (long)kWB);
  per = cdiv(nblk, (long)kWGrid);
  grid = per > 0 ? cdiv(nblk, per) : 0;
}
constexpr size_t kWSmem = 2 * (size_t)kWStage * sizeof(__nv_bfloat16);

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
  const long nbl = bwd_blocks(N);
  if (cudaMalloc((void**)&m->d_X, sizeof(__nv_bfloat16) * kNF * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_Y, sizeof(float) * kNO * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_H, sizeof(__nv_bfloat16) * 3 * kH * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_D, sizeof(__nv_bfloat16) * 3 * kH * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_dY, sizeof(__nv_bfloat16) * kNO * N) != cudaSuccess ||
      cudaMalloc((void**)&m->d_part, sizeof(float) * kNPar * kWGrid) != cudaSuccess ||
      cudaMalloc((void**)&m->d_lpart, sizeof(double) * nbl) != cudaSuccess)
    return MLS6_ERR_NOMEM;
  m->cap = N;
  return MLS6_OK;
}

static int repack(Mlp* m) {
  k_mlp_pack<<<cdiv(kPkAll, 256), 256, 0, m->stream>>>(m->d_par, m->d_pack);
  CK(cudaGetLastError());
  return MLS6_OK;
}

static int forward(Mlp* m, const void* X, long N, float* Y, bool store) {
  if (N <= 0) return MLS6_OK;
  const long nb = fwd_blocks(N);
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
  const long nbl = bwd_blocks(N);
  long nch, per;
  wgrad_geometry(N, nch, per);
  k_mlp_bwd<<<nbl, 128, 0, m->stream>>>(m->d_Y, T, N, 1.0f / (float)N, m->d_H, m->d_pack,
                                        m->d_D, m->d_dY, m->d_lpart);
  k_mlp_wgrad<<<nch, 256, kWSmem, m->stream>>>((const __nv_bfloat16*)X, m->d_H, m->d_D, m->d_dY,
                                               N, per, m->d_part);
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
      cudaMalloc((void**)&m->d_pack, sizeof(uint2) * kPkAll) != cudaSuccess ||
      cudaMalloc((void**)&m->d_norm, sizeof(float) * 2 * kNF) != cudaSuccess ||
      cudaMalloc((void**)&m->d_loss, sizeof(double)) != cudaSuccess) {
    free_mlp(m);
    return MLS6_ERR_NOMEM;
  }
  // two shared-memory stages of the weight-gradient kernel (above 48 KB)
  if (cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kWSmem) != cudaSuccess) {
    free_mlp(m);
    return MLS6_ERR_CUDA;
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
  if (p->order != 3) return MLS6_ERR_ORDER;  // features are defined on the cubic basis
  if (p->N > 0 && !kernel_addressable(out)) return MLS6_ERR_ARG;
  Mlp* m = const_cast<Mlp*>(reinterpret_cast<const Mlp*>(mm));
  return p->prec == MLS6_FP64 ? features_t<double>(p, m, out, fmt, false, p->stream)
                              : features_t<float>(p, m, out, fmt, false, p->stream);
}

int mls6_mlp_forward(mls6_mlp_t* mm, const void* X, int64_t N, float* Y) {
  if (!mm || N < 0 || (N > 0 && (!kernel_addressable(X) || !kernel_addressable(Y))))
    return MLS6_ERR_ARG;
  return forward(reinterpret_cast<Mlp*>(mm), X, N, Y, false);
}

int mls6_mlp_grad(mls6_mlp_t* mm, const void* X, const float* T, int64_t N, float* grad,
                  double* loss) {
  if (!mm || N < 1 || !kernel_addressable(X) || !kernel_addressable(T) ||
      (reinterpret_cast<uintptr_t>(X) & 15))
    return MLS6_ERR_ARG;
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
  if (!mm || N < 1 || !kernel_addressable(X) || !kernel_addressable(T) || !(lr > 0.f) ||
      (reinterpret_cast<uintptr_t>(X) & 15))
    return MLS6_ERR_ARG;
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
  if (p->order != 3) return MLS6_ERR_ORDER;
  const long N = p->N;
  if (N == 0) return MLS6_OK;
  if (!kernel_addressable(forces)) return MLS6_ERR_ARG;
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
