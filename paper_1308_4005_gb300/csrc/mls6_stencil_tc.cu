// Level stencils (Eq. evaluation) on the tensor cores, for the mixed
// precision mode: BF16 split operands (x = x_hi + x_lo), FP32 accumulation.
//
// The cutoff stencil of level k is a single-channel 3D convolution.  Grouped
// by tap rows of constant (dy, dz) it is, along x, a banded Toeplitz matrix
// product: for 16 consecutive outputs x0..x0+15 of a grid line and the 32
// inputs x0-8..x0+23 of the line shifted by (dy, dz),
//     e[x0 + m] += sum_k T[m][k] q[x0 - 8 + k],   T[m][k] = w(k - 8 - m),
// with w(dx) the row's tap weights (zero for |dx| > R_row <= 8).  T is the A
// operand (16 x 32, two k-steps of mma.m16n8k16) and eight grid lines form
// the B operand (32 x 8).  Every product is taken as
//     A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the lo*lo term is below the representation error of the split), which
// keeps about 16 significant bits per product: relative error <= 3 * 2^-18.
//
// Block: 4 warps, output tile 16 (x) x 16 (y) x 8 (z) of one level; the
// tile's input lines (with a halo of P in y and z, a 32-wide x window) are
// staged once in shared memory as BF16 hi and lo copies.  A warp owns four
// groups of 8 lines (8 consecutive y at one z).  Per tap row it builds its A
// fragments from packed weight pairs (5 words per part and channel cover
// both k-steps) and runs, per line group, two ldmatrix.x4 (hi, lo) and six
// mma.  The virial uses three more weight channels (G, G dx, G dx^2) whose
// products with the line group (weights split, q_hi only: four mma) are
// dotted with the centre values q_mu and folded per row as in the FP32
// kernel (Sec. II.B; strain derivative).
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <vector>

#include "mls6_device.cuh"

namespace mls6 {


constexpr int kTcX = 16, kTcY = 16, kTcZ = 8;
// warps per block: 8 for the energy-only kernel (78 registers: two blocks
// of 8 warps per SM), 4 with the virial channels (160 registers) so that the
// A fragments of a tap row serve 4 line groups; measured on the 1M-atom
// cube: 180 vs 238 us without the virial, 422 vs 439 us with it
template <bool VIR> __host__ __device__ constexpr int tc_warps() { return VIR ? 4 : 8; }
// the x window of a tile is 32 nodes (16 outputs and the stencil's halo)
constexpr int kTcPitch = 40;                          // bf16 per staged line (80 B)
constexpr int kTcWords = 64;                          // packed pairs per row, part, channel

struct TcLevel {
  const float* q;
  float* e;
  int n[3];
  int tiles[3];
  long tile_off;
  float scale;
};

struct TcArgs {
  TcLevel lv[kMaxLevels];
  int nlev, P, nrows;
  const int4* rows;      // dy, dz, R, first tap
  const uint32_t* w;     // [row][channel 0..3][hi, lo][64] packed bf16 pairs
  double hc[6];
  long sblocks;
  const float* qt;
  float* et;
  int nt[3];
  const double* tT;
  const double* tV;
  double* wtop;
};

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}

// Weight pairs P(b-8), P(b), P(b+8), P(b+16), P(b+24) of one channel/part:
// A fragment of k-step 0 is {P(b), P(b-8), P(b+8), P(b)}, of k-step 1
// {P(b+16), P(b+8), P(b+24), P(b+16)} (rows g, g+8; columns c2.., c2+8..).
struct Frag5 {
  uint32_t p[5];
};

__device__ __forceinline__ Frag5 load_frag(const uint32_t* __restrict__ wp, int idx0) {
  Frag5 f;
#pragma unroll
  for (int j = 0; j < 5; ++j) f.p[j] = __ldg(wp + idx0 + 8 * j);
  return f;
}

// D += T(channel) * B over both k-steps with the three split products.
__device__ __forceinline__ void toeplitz_mma(float (&d)[4], const Frag5& h, const Frag5& l,
                                             const uint32_t (&bh)[4], const uint32_t (&bl)[4]) {
  mma16816(d, h.p[1], h.p[0], h.p[2], h.p[1], bh[0], bh[1]);
  mma16816(d, h.p[1], h.p[0], h.p[2], h.p[1], bl[0], bl[1]);
  mma16816(d, l.p[1], l.p[0], l.p[2], l.p[1], bh[0], bh[1]);
  mma16816(d, h.p[3], h.p[2], h.p[4], h.p[3], bh[2], bh[3]);
  mma16816(d, h.p[3], h.p[2], h.p[4], h.p[3], bl[2], bl[3]);
  mma16816(d, l.p[3], l.p[2], l.p[4], l.p[3], bh[2], bh[3]);
}

// Virial channels: D += T * B_hi with T split (A_hi + A_lo), two products.
// The dropped T * B_lo term is a per-node relative error <= 2^-9 of q in a
// sum over all nodes (the virial is a global bilinear form), where it
// averages out; the weights stay exact to 2^-18.
__device__ __forceinline__ void toeplitz_mma2(float (&d)[4], const Frag5& h, const Frag5& l,
                                              const uint32_t (&bh)[4]) {
  mma16816(d, h.p[1], h.p[0], h.p[2], h.p[1], bh[0], bh[1]);
  mma16816(d, l.p[1], l.p[0], l.p[2], l.p[1], bh[0], bh[1]);
  mma16816(d, h.p[3], h.p[2], h.p[4], h.p[3], bh[2], bh[3]);
  mma16816(d, l.p[3], l.p[2], l.p[4], l.p[3], bh[2], bh[3]);
}

template <bool VIR>
__global__ void __launch_bounds__(tc_warps<VIR>() * 32) k_stencil_tc(TcArgs A,
                                                                    double* __restrict__ wpart) {
  pdl_begin();
  constexpr int kTcWarps = tc_warps<VIR>();
  constexpr int kTcNG = (kTcY / 8) * kTcZ / kTcWarps;  // line groups per warp
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32 * 7];
  if ((long)blockIdx.x >= A.sblocks) {  // coarsest level: one warp per node
    const int mu = (int)((long)blockIdx.x - A.sblocks) * kTcWarps + (int)(threadIdx.x >> 5);
    if (mu < A.nt[0] * A.nt[1] * A.nt[2])
      coarsest_node<float, VIR>(A.qt, A.nt[0], A.nt[1], A.nt[2], A.tT, A.tV, A.et, A.wtop, mu);
    return;
  }
  const long b = blockIdx.x;
  int k = 0;
  while (k + 1 < A.nlev && b >= A.lv[k + 1].tile_off) ++k;
  const TcLevel& L = A.lv[k];
  const float* __restrict__ q = L.q;
  const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
  const long t = b - L.tile_off;
  const int x0 = (int)(t % L.tiles[0]) * kTcX;
  const int y0 = (int)((t / L.tiles[0]) % L.tiles[1]) * kTcY;
  const int z0 = (int)(t / ((long)L.tiles[0] * L.tiles[1])) * kTcZ;
  const int P = A.P, LY = kTcY + 2 * P, LZ = kTcZ + 2 * P, NL = LY * LZ;
  __nv_bfloat16* th = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* tl = th + (size_t)NL * kTcPitch;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // stage the input lines: one warp per line, lane = x - (x0 - 8)
  for (int line = warp; line < NL; line += kTcWarps) {
    const int ly = line % LY, lz = line / LY;
    const int gy = wrapi(y0 + ly - P, n1), gz = wrapi(z0 + lz - P, n2);
    const int gx = wrapi(x0 - 8 + lane, n0);
    const float v = q[gx + (long)n0 * (gy + (long)n1 * gz)];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    th[line * kTcPitch + lane] = hi;
    tl[line * kTcPitch + lane] = lo;
  }
  __syncthreads();

  const int g = lane >> 2, c2 = (lane & 3) * 2;
  const int idx0 = c2 - g + 24 - 8;  // word index of P(b - 8), b = c2 - g - 8
  // line groups of this warp: yh = grp & 1 (y half), zz = grp >> 1
  int gbase[kTcNG];
#pragma unroll
  for (int j = 0; j < kTcNG; ++j) {
    const int grp = warp * kTcNG + j;
    gbase[j] = ((grp & 1) * 8 + P) + LY * ((grp >> 1) + P);  // line index of y offset 0
  }
  const uint32_t sh_hi = (uint32_t)__cvta_generic_to_shared(th);
  const uint32_t sh_lo = (uint32_t)__cvta_generic_to_shared(tl);
  const int arow = lane & 7, achunk = lane >> 3;

  float acc[kTcNG][4];
  float qmu[kTcNG][4];
#pragma unroll
  for (int j = 0; j < kTcNG; ++j) {
    const int grp = warp * kTcNG + j;
    const int yy = y0 + (grp & 1) * 8, zz = z0 + (grp >> 1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      acc[j][c] = 0.f;
      const int m = g + (c >> 1) * 8, n = c2 + (c & 1);
      const bool in = (x0 + m < n0) && (yy + n < n1) && (zz < n2);
      const int li = gbase[j] + n;
      qmu[j][c] = in ? __bfloat162float(th[li * kTcPitch + 8 + m]) +
                           __bfloat162float(tl[li * kTcPitch + 8 + m])
                     : 0.f;
    }
  }
  float vxx = 0.f, vyy = 0.f, vzz = 0.f, vxy = 0.f, vxz = 0.f, vyz = 0.f;

  for (int r = 0; r < A.nrows; ++r) {
    const int4 ri = __ldg(A.rows + r);
    const uint32_t* wr = A.w + (size_t)r * (4 * 2 * kTcWords);
    const Frag5 h0 = load_frag(wr, idx0), l0 = load_frag(wr + kTcWords, idx0);
    Frag5 h1, l1, h2, l2, h3, l3;
    if (VIR) {
      h1 = load_frag(wr + 2 * kTcWords, idx0);
      l1 = load_frag(wr + 3 * kTcWords, idx0);
      h2 = load_frag(wr + 4 * kTcWords, idx0);
      l2 = load_frag(wr + 5 * kTcWords, idx0);
      h3 = load_frag(wr + 6 * kTcWords, idx0);
      l3 = load_frag(wr + 7 * kTcWords, idx0);
    }
    const int shift = ri.x + LY * ri.y;  // (dy, dz) in staged lines
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll
    for (int j = 0; j < kTcNG; ++j) {
      const uint32_t off = (uint32_t)(((gbase[j] + arow + shift) * kTcPitch + achunk * 8) * 2);
      uint32_t bh[4], bl[4];
      ldsm_x4(bh, sh_hi + off);
      ldsm_x4(bl, sh_lo + off);
      toeplitz_mma(acc[j], h0, l0, bh, bl);
      if (VIR) {
        float u[4] = {0.f, 0.f, 0.f, 0.f};
        toeplitz_mma2(u, h1, l1, bh);
        t0 += u[0] * qmu[j][0] + u[1] * qmu[j][1] + u[2] * qmu[j][2] + u[3] * qmu[j][3];
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        toeplitz_mma2(v, h2, l2, bh);
        t1 += v[0] * qmu[j][0] + v[1] * qmu[j][1] + v[2] * qmu[j][2] + v[3] * qmu[j][3];
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        toeplitz_mma2(s, h3, l3, bh);
        t2 += s[0] * qmu[j][0] + s[1] * qmu[j][1] + s[2] * qmu[j][2] + s[3] * qmu[j][3];
      }
    }
    if (VIR) {
      const float dy = (float)ri.x, dz = (float)ri.y;
      vxx += t2;
      vyy += dy * dy * t0;
      vzz += dz * dz * t0;
      vxy += dy * t1;
      vxz += dz * t1;
      vyz += dy * dz * t0;
    }
  }

  // outputs
#pragma unroll
  for (int j = 0; j < kTcNG; ++j) {
    const int grp = warp * kTcNG + j;
    const int yy = y0 + (grp & 1) * 8, zz = z0 + (grp >> 1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = g + (c >> 1) * 8, n = c2 + (c & 1);
      if ((x0 + m < n0) && (yy + n < n1) && (zz < n2))
        L.e[(x0 + m) + (long)n0 * ((yy + n) + (long)n1 * zz)] = L.scale * acc[j][c];
    }
  }
  if (VIR) {
    float v6[6] = {vxx, vyy, vzz, vxy, vxz, vyz};
    double w6[6];
    block_sum_lo<float, 6>(v6, w6, red);
    if (threadIdx.x == 0) {
      const double hs = 0.5 * (double)L.scale;
      for (int c = 0; c < 6; ++c) wpart[6 * b + c] = hs * A.hc[c] * w6[c];
    }
  }
}

// ------------------------------------------------------------------ host

static uint16_t bf16_bits(float f) {  // round to nearest even
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

static float bf16_value(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

bool stencil_tc_eligible(const Plan* p) {
  if (p->prec != MLS6_MIXED || p->levels < 2 || p->P > 8) return false;
  const size_t sm = tc_smem_bytes(p->P);
  return sm <= kStencilSmemMax;
}

size_t tc_smem_bytes(int P) {
  return (size_t)(kTcY + 2 * P) * (kTcZ + 2 * P) * kTcPitch * 2 * sizeof(uint16_t);
}

// Tile geometry of the tensor-core stencil (replaces the FP32 kernel's).
void tc_geometry(Plan* p) {
  p->stencil_blocks = 0;
  const int T[3] = {kTcX, kTcY, kTcZ};
  for (int k = 1; k < p->levels; ++k) {
    p->tile_off[k] = p->stencil_blocks;
    long nt = 1;
    for (int d = 0; d < 3; ++d) {
      p->tiles[k][d] = (int)cdiv(p->lv[k].n[d], T[d]);
      nt *= p->tiles[k][d];
    }
    p->stencil_blocks += nt;
  }
  p->stencil_smem = tc_smem_bytes(p->P);
}

// Packed split weight pairs per row: word d + 32 holds (w[d], w[d+1]) as
// bf16 (low half first), channels g_1, G, G dx, G dx^2, parts hi and lo.
std::vector<uint32_t> tc_weight_table(const Plan* p) {
  std::vector<uint32_t> out((size_t)p->nrows * 4 * 2 * kTcWords, 0u);
  for (int r = 0; r < p->nrows; ++r) {
    const int R = p->h_rows[4 * r + 2], first = p->h_rows[4 * r + 3];
    for (int ch = 0; ch < 4; ++ch) {
      uint16_t hi[kTcWords + 1] = {}, lo[kTcWords + 1] = {};
      for (int d = -32; d < 32; ++d) {
        if (d < -R || d > R) continue;
        const double w = p->h_wv[4 * (size_t)(first + d + R) + ch];
        const uint16_t h = bf16_bits((float)w);
        hi[d + 32] = h;
        lo[d + 32] = bf16_bits((float)(w - (double)bf16_value(h)));
      }
      uint32_t* oh = &out[(((size_t)r * 4 + ch) * 2 + 0) * kTcWords];
      uint32_t* ol = &out[(((size_t)r * 4 + ch) * 2 + 1) * kTcWords];
      for (int i = 0; i < kTcWords; ++i) {
        oh[i] = (uint32_t)hi[i] | ((uint32_t)hi[i + 1] << 16);
        ol[i] = (uint32_t)lo[i] | ((uint32_t)lo[i + 1] << 16);
      }
    }
  }
  return out;
}

int prepare_stencil_tc(Plan* p) {
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(k_stencil_tc<true>, attr, (int)kStencilSmemMax) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil_tc<false>, attr, (int)kStencilSmemMax) != cudaSuccess)
    return MLS6_ERR_CUDA;
  return MLS6_OK;
}

int launch_stencil_tc(Plan* p, bool vir, bool fuse_top, cudaStream_t st) {
  TcArgs A;
  A.nlev = p->levels - 1;
  A.P = p->P;
  A.nrows = p->nrows;
  A.rows = reinterpret_cast<const int4*>(p->d_rows);
  A.w = p->d_tcw;
  const double* h = p->lv[1].h;
  A.hc[0] = h[0] * h[0];
  A.hc[1] = h[1] * h[1];
  A.hc[2] = h[2] * h[2];
  A.hc[3] = h[0] * h[1];
  A.hc[4] = h[0] * h[2];
  A.hc[5] = h[1] * h[2];
  for (int k = 1; k < p->levels; ++k) {
    TcLevel& L = A.lv[k - 1];
    L.q = (const float*)p->d_q[k];
    L.e = (float*)p->d_e[k];
    for (int d = 0; d < 3; ++d) {
      L.n[d] = p->lv[k].n[d];
      L.tiles[d] = p->tiles[k][d];
    }
    L.tile_off = p->tile_off[k];
    L.scale = (float)std::ldexp(1.0, -6 * (k - 1));
  }
  const int l = p->levels;
  A.sblocks = p->stencil_blocks;
  A.qt = (const float*)p->d_q[l];
  A.et = (float*)p->d_e[l];
  for (int d = 0; d < 3; ++d) A.nt[d] = p->lv[l].n[d];
  A.tT = p->d_top_T;
  A.tV = p->d_top_V;
  A.wtop = p->d_wpart + 6 * p->wpart_top;
  double* wp = p->d_wpart + 6 * p->wpart_stencil;
  const int warps = vir ? tc_warps<true>() : tc_warps<false>();
  const long nb = p->stencil_blocks + (fuse_top ? cdiv(p->lv[l].np, warps) : 0);
  if (vir)
    launch_pdl(k_stencil_tc<true>, nb, warps * 32, p->stencil_smem, st, A, wp);
  else
    launch_pdl(k_stencil_tc<false>, nb, warps * 32, p->stencil_smem, st, A, wp);
  return 1;
}

}  // namespace mls6
