// Level stencils (Eq. evaluation) on the fifth-generation tensor cores
// (tcgen05, accumulators in tensor memory), for the mixed precision mode:
// BF16 split operands (x = x_hi + x_lo), FP32 accumulation.
//
// Grouped by tap rows of constant (dy, dz), the cutoff stencil of level k is
// along x a banded Toeplitz product.  For 16 consecutive outputs x0..x0+15
// on 128 grid lines (8 y x 16 z; a block holds two such halves, y 0..7 and
// 8..15, which share every weight chunk) and one tap row,
//     D[line][c*16 + m] += sum_k A[line][k] B_c[k][m],
//     A[line][k] = q(x0 - 8 + k, y + dy, z + dz),   B_c[k][m] = W_c(k - 8 - m),
// with W_c the row's weights of channel c (zero for |dx| > R_row <= 8): per
// tap row and K step of 16 one M = 128 MMA whose B operand holds the hi and
// the lo weight matrices side by side (N = 2 x 16 x channels, so the q_hi
// operand is read once for both products), plus one N = 16 MMA of q_lo with
// the energy channel's hi weights; D in tensor memory.  The A operand of every tap row is the same staged block of q,
// addressed with a shifted start: the staged layout puts the 8 y-lines of a
// core matrix 16 bytes apart (a shift in y moves the start by 16 B) and the
// z-lines a fixed stride apart (a shift in z moves it by that stride), so
// the tile is staged once and the 100+ tap rows only change descriptors.
//
// Channels: c = 0 the energy weights g_1; with the virial six more,
// G dx^2, G dy^2, G dz^2, G dx dy, G dx dz, G dy dz (G = g_1'/r, lattice
// offsets; the row constants dy, dz are folded into the weights so every
// channel accumulates over all tap rows).  After the last row the tile reads
// D back once: e = scale * D_0 is stored and, for the virial, each channel is
// dotted with the centre values q_mu (strain derivative, Sec. II.B reading);
// each channel is the sum of its hi-weight and lo-weight accumulator columns.
//
// Products (the lo*lo term is below the split's representation error):
// energy q_hi w_hi + q_hi w_lo + q_lo w_hi (relative error <= 3 * 2^-18 per
// product); virial channels q_hi w_hi + q_hi w_lo (the per-node 2^-9 error
// of q averages out in the global bilinear form).
//
// Pipeline per block (128 threads, one 16^3 tile): all threads stage the q block
// (hi and lo, no swizzle, K-major core matrices); thread 32 streams the
// per-row weight matrices B (precomputed at plan time in the core-matrix
// layout) from global memory into a ring of up to kMmaStagesMax buffers with bulk
// copies completing on mbarriers; thread 0 issues the MMAs and commits each
// buffer back to its "empty" mbarrier; the other threads wait at the block
// barrier; the epilogue reads tensor memory with tcgen05.ld.  Every
// wait on an mbarrier is bounded: on timeout the block records an error
// flag, waits (bounded) for its outstanding MMAs, releases its tensor memory
// and returns.
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mls6_device.cuh"

namespace mls6 {


// tile: 16 x-outputs x 16 y x 16 z, two M = 128 halves (y 0..7 and 8..15)
// that share every weight chunk
constexpr int kMmaX = 16, kMmaY = 16, kMmaZ = 16, kMmaHalves = 2;
constexpr int kMmaThreads = 128;
template <bool VIR> __host__ __device__ constexpr int mma_n() { return VIR ? 112 : 16; }
// tap rows per weight chunk: 28 KB (virial) or 8 KB (energy only) per chunk
template <bool VIR> __host__ __device__ constexpr int mma_rows_per_chunk() { return VIR ? 2 : 4; }
// tensor-memory columns per half: 2 x mma_n (hi-weight and lo-weight
// products), rounded to a power of two; the two halves side by side
template <bool VIR> __host__ __device__ constexpr int mma_tmem_cols() { return VIR ? 256 : 32; }
constexpr int kMmaStagesMax = 4;  // weight buffers in flight (fewer when shared memory is short)
// bytes of one tap row's B matrices (per K chunk of 8: hi rows, then lo
// rows) in the core-matrix layout
template <bool VIR> __host__ __device__ constexpr int mma_row_bytes() {
  return 2 * 4 * mma_n<VIR>() * 16;
}
constexpr long kMmaWaitLimit = 1L << 26;  // mbarrier polls before a block gives up

struct MmaLevel {
  const float* q;
  float* e;
  int n[3];
  int tiles[3];
  long tile_off;
  float scale;
};

struct MmaArgs {
  MmaLevel lv[kMaxLevels];
  int nlev, P, nrows, nrows_pad, stages;
  const int4* rows;        // dy, dz, R, first tap (padding rows: dy = dz = 0)
  const uint8_t* B;        // weight matrices, mma_row_bytes per (padded) row
  double hc[6];
  long sblocks;
  const float* qt;
  float* et;
  int nt[3];
  const double* tT;
  const double* tV;
  double* wtop;
  int* err;                // the plan's device flag word: bit 1 set when a wait timed out
};

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle: start, leading-dimension byte
// offset (between core matrices along K), stride byte offset (between core
// matrices along M/N), descriptor version 1.
__device__ __forceinline__ uint64_t mma_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase of the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  for (long it = 0; it < kMmaWaitLimit; ++it)
    if (mbar_try(b, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          su32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
}

// ------------------------------------------------------------------ kernel

template <bool VIR>
__global__ void __launch_bounds__(kMmaThreads) k_stencil_mma(MmaArgs A,
                                                             double* __restrict__ wpart) {
  pdl_begin();
  constexpr int NV = mma_n<VIR>();
  constexpr int RB = mma_rows_per_chunk<VIR>();
  constexpr int RBYTES = mma_row_bytes<VIR>();
  constexpr int CB = RB * RBYTES;  // bytes per B chunk
  constexpr int TCOLS = mma_tmem_cols<VIR>();
  constexpr int TALLOC = kMmaHalves * TCOLS;
  const int NS = A.stages;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kMmaStagesMax], bar_empty[kMmaStagesMax], bar_done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ double red[32 * 7];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if ((long)blockIdx.x >= A.sblocks) {  // coarsest level: one warp per node
    const int mu = (int)((long)blockIdx.x - A.sblocks) * (kMmaThreads / 32) + warp;
    if (mu < A.nt[0] * A.nt[1] * A.nt[2])
      coarsest_node<float, VIR>(A.qt, A.nt[0], A.nt[1], A.nt[2], A.tT, A.tV, A.et, A.wtop, mu);
    return;
  }
  const long b = blockIdx.x;
  int k = 0;
  while (k + 1 < A.nlev && b >= A.lv[k + 1].tile_off) ++k;
  const MmaLevel& L = A.lv[k];
  const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
  const long t = b - L.tile_off;
  const int x0 = (int)(t % L.tiles[0]) * kMmaX;
  const int y0 = (int)((t / L.tiles[0]) % L.tiles[1]) * kMmaY;
  const int z0 = (int)(t / ((long)L.tiles[0] * L.tiles[1])) * kMmaZ;
  const int P = A.P, Ys = kMmaY + 2 * P, Zs = kMmaZ + 2 * P;
  const uint32_t a_lbo = (uint32_t)(Zs * Ys * 16);  // K-chunk stride of the staged block
  const uint32_t a_part = 4u * a_lbo;                // hi -> lo
  unsigned char* sA = smem_raw;
  unsigned char* sB = smem_raw + 2 * a_part;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "r"(TALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // stage q: entry (kc, zz, yy) = 8 consecutive x values of one line, as
  // BF16 hi and lo, 16 bytes each
  const float* __restrict__ q = L.q;
  const int nent = 4 * Zs * Ys;
  for (int idx = tid; idx < nent; idx += kMmaThreads) {
    const int kc = idx & 3, line = idx >> 2;
    const int yy = line % Ys, zz = line / Ys;
    const int gy = wrapi(y0 - P + yy, n1), gz = wrapi(z0 - P + zz, n2);
    const long row = (long)n0 * (gy + (long)n1 * gz);
    const int xs = x0 - 8 + 8 * kc;
    float v[8];
    if (xs >= 0 && xs + 8 <= n0 && ((row + xs) & 3) == 0) {
      const float4 u0 = *reinterpret_cast<const float4*>(q + row + xs);
      const float4 u1 = *reinterpret_cast<const float4*>(q + row + xs + 4);
      v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
      v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = q[row + wrapi(xs + j, n0)];
    }
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float h0 = __bfloat162float(__float2bfloat16_rn(v[2 * j]));
      const float h1 = __bfloat162float(__float2bfloat16_rn(v[2 * j + 1]));
      hw[j] = pack_bf16(h0, h1);
      lw[j] = pack_bf16(v[2 * j] - h0, v[2 * j + 1] - h1);
    }
    const uint32_t off = (uint32_t)(((kc * Zs + zz) * Ys + yy) * 16);
    *reinterpret_cast<uint4*>(sA + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(sA + a_part + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic -> async proxy
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int nchunks = A.nrows_pad / RB;

  // Only two threads work until the accumulators are complete: the other
  // threads wait at the block barrier below instead of polling (polling
  // lanes share warps 0 and 1 with the two workers and would steal their
  // issue slots).
  bool done = true;
  if (tid == 32) {  // weight producer: up to NS chunks in flight
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % NS, use = c / NS;
      if (use > 0 && !mbar_wait(&bar_empty[s], (uint32_t)((use - 1) & 1))) {
        atomicOr(&abort_flag, 1);
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      bulk_g2s(sB + s * CB, A.B + (size_t)c * CB, (uint32_t)CB, &bar_full[s]);
    }
  } else if (tid == 0) {  // MMA issuer
    const uint32_t id2 = mma_idesc(128, 2 * NV), id16 = mma_idesc(128, 16);
    const uint32_t sa = su32(sA), sb = su32(sB);
    const uint32_t a_sbo = (uint32_t)(Ys * 16);
    uint32_t acc = 0;
    bool ok = true;
    for (int c = 0; c < nchunks && ok; ++c) {
      const int s = c % NS;
      if (!mbar_wait(&bar_full[s], (uint32_t)((c / NS) & 1))) {
        atomicOr(&abort_flag, 1);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int rr = 0; rr < RB; ++rr) {
        const int4 ri = __ldg(A.rows + c * RB + rr);
        const uint32_t abase = sa + (uint32_t)(((P + ri.y) * Ys + (P + ri.x)) * 16);
        const uint32_t bbase = sb + (uint32_t)(s * CB + rr * RBYTES);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ak = abase + (uint32_t)(2 * ks) * a_lbo;
          const uint32_t bk = bbase + (uint32_t)(2 * ks * 2 * NV * 16);
          const uint64_t ah = mma_sdesc(ak, a_lbo, a_sbo), al = mma_sdesc(ak + a_part, a_lbo, a_sbo);
          // B: per K chunk 2 NV rows (hi then lo); the first 16 rows are the
          // energy channel's hi weights
          const uint64_t bb = mma_sdesc(bk, 2 * NV * 16, 128);
#pragma unroll
          for (int hh = 0; hh < kMmaHalves; ++hh) {  // half hh: y lines 8 hh .. 8 hh + 7
            const uint32_t dt = tmem + (uint32_t)(hh * TCOLS);
            const uint64_t ahh = ah + (uint64_t)(hh * 8);  // + 8 rows x 16 B, in 16-B units
            const uint64_t alh = al + (uint64_t)(hh * 8);
            mma_f16(dt, ahh, bb, id2, acc);  // q_hi [w_hi | w_lo], every channel
            mma_f16(dt, alh, bb, id16, 1);   // q_lo w_hi, energy channel
          }
          acc = 1;
        }
      }
      mma_commit(&bar_empty[s]);
    }
    mma_commit(&bar_done);
    // wait for the last MMA (bounded; on timeout once more, for the MMAs
    // already issued)
    done = mbar_wait(&bar_done, 0);
    if (!done) {
      atomicOr(&abort_flag, 1);
      done = mbar_wait(&bar_done, 0);
    }
    if (!done) atomicOr(&abort_flag, 2);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  done = (abort_flag & 2) == 0;
  const bool aborted = abort_flag != 0;
  if (aborted && tid == 0) atomicOr(A.err, 2);

  // epilogue: thread = TMEM lane r, i.e. line (y = r % 8 + 8 hh, z = r / 8)
  // of each half hh; 16 outputs along x
  const int r = 32 * warp + lane;
  float w6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int hh = 0; hh < kMmaHalves; ++hh) {
    const int gy = y0 + 8 * hh + (r & 7), gz = z0 + (r >> 3);
    const bool line_in = gy < n1 && gz < n2 && !aborted && done;
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(hh * TCOLS);
    float d[16], dl[16];
    tmem_ld16(taddr, d);
    tmem_ld16(taddr + NV, dl);  // lo-weight products
#pragma unroll
    for (int j = 0; j < 16; ++j) d[j] += dl[j];
    const long obase = (long)n0 * (gy + (long)n1 * gz);
    if (line_in) {
      if (x0 + 16 <= n0 && ((obase + x0) & 3) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(L.e + obase + x0 + j) = make_float4(
              L.scale * d[j], L.scale * d[j + 1], L.scale * d[j + 2], L.scale * d[j + 3]);
      } else {
        for (int j = 0; j < 16; ++j)
          if (x0 + j < n0) L.e[obase + x0 + j] = L.scale * d[j];
      }
    }
    if (VIR) {
      float qc[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) qc[j] = (line_in && x0 + j < n0) ? q[obase + x0 + j] : 0.f;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        float dc[16], dcl[16];
        tmem_ld16(taddr + 16 * (c + 1), dc);
        tmem_ld16(taddr + NV + 16 * (c + 1), dcl);
        float sacc = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) sacc += qc[j] * (dc[j] + dcl[j]);
        w6[c] += sacc;
      }
    }
  }
  if (VIR) {
    double ws[6];
    block_sum_lo<float, 6>(w6, ws, red);
    if (tid == 0) {
      const double hs = 0.5 * (double)L.scale;
      for (int c = 0; c < 6; ++c) wpart[6 * b + c] = hs * A.hc[c] * ws[c];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TALLOC)
                 : "memory");
}

// ------------------------------------------------------------------ host

static uint16_t bf16_bits_rn(float f) {  // round to nearest even
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

static float bf16_to_float(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// Weight buffers: kMmaStagesMax, or fewer when the staged block and the
// ring would exceed the 227 KB a block can use.
template <bool VIR> static int mma_stages(int P) {
  const size_t a = 2 * 4 * (size_t)(kMmaZ + 2 * P) * (kMmaY + 2 * P) * 16;
  const size_t chunk = (size_t)mma_rows_per_chunk<VIR>() * mma_row_bytes<VIR>();
  int s = kMmaStagesMax;
  while (s > 2 && a + s * chunk + 4096 > 227 * 1024) --s;
  return s;
}

template <bool VIR> static size_t mma_smem(int P) {
  const size_t a = 2 * 4 * (size_t)(kMmaZ + 2 * P) * (kMmaY + 2 * P) * 16;
  return a + (size_t)mma_stages<VIR>(P) * mma_rows_per_chunk<VIR>() * mma_row_bytes<VIR>();
}

size_t stencil_mma_smem(const Plan* p, bool vir) {
  return vir ? mma_smem<true>(p->P) : mma_smem<false>(p->P);
}

bool stencil_mma_eligible(const Plan* p) {
  if (p->prec != MLS6_MIXED || p->levels < 2 || p->P > 8) return false;
  return mma_smem<true>(p->P) + 4096 <= 227 * 1024;
}

// Number of 16^3 tiles over the levels k < l.
long stencil_mma_tiles(const Plan* p) {
  long t = 0;
  for (int k = 1; k < p->levels; ++k)
    t += cdiv(p->lv[k].n[0], kMmaX) * cdiv(p->lv[k].n[1], kMmaY) * cdiv(p->lv[k].n[2], kMmaZ);
  return t;
}

// Tile geometry (16 x 16 x 16 nodes per block).
void stencil_mma_geometry(Plan* p) {
  p->stencil_blocks = 0;
  const int T[3] = {kMmaX, kMmaY, kMmaZ};
  for (int k = 1; k < p->levels; ++k) {
    p->tile_off[k] = p->stencil_blocks;
    long nt = 1;
    for (int d = 0; d < 3; ++d) {
      p->tiles[k][d] = (int)cdiv(p->lv[k].n[d], T[d]);
      nt *= p->tiles[k][d];
    }
    p->stencil_blocks += nt;
  }
  p->stencil_smem = mma_smem<true>(p->P);
}

// Weight matrices in the layout of the MMA's B operand: per tap row (padded
// to a multiple of the chunk size with zero rows), K chunk (8 inputs), part
// (hi, lo), column n = channel * 16 + output m, 8 BF16 inputs: 16 bytes.
// Within a K chunk the hi rows and then the lo rows are one operand of
// 2 NV rows.
template <bool VIR> static std::vector<uint8_t> weight_matrices(const Plan* p, int nrows_pad) {
  constexpr int NV = mma_n<VIR>();
  std::vector<uint8_t> out((size_t)nrows_pad * mma_row_bytes<VIR>(), 0);
  for (int r = 0; r < p->nrows; ++r) {
    const int dy = p->h_rows[4 * r], dz = p->h_rows[4 * r + 1];
    const int R = p->h_rows[4 * r + 2], first = p->h_rows[4 * r + 3];
    uint16_t* row = reinterpret_cast<uint16_t*>(out.data() + (size_t)r * mma_row_bytes<VIR>());
    for (int n = 0; n < NV; ++n) {
      const int ch = n / 16, m = n % 16;
      for (int k = 0; k < 32; ++k) {
        const int dx = k - 8 - m;
        if (dx < -R || dx > R) continue;
        const double* wv = &p->h_wv[4 * (size_t)(first + dx + R)];
        double w = 0.0;
        switch (ch) {
          case 0: w = wv[0]; break;                      // g_1
          case 1: w = wv[3]; break;                      // G dx^2
          case 2: w = (double)dy * dy * wv[1]; break;    // G dy^2
          case 3: w = (double)dz * dz * wv[1]; break;    // G dz^2
          case 4: w = (double)dy * wv[2]; break;         // G dx dy
          case 5: w = (double)dz * wv[2]; break;         // G dx dz
          default: w = (double)dy * dz * wv[1]; break;   // G dy dz
        }
        const uint16_t h = bf16_bits_rn((float)w);
        const uint16_t l = bf16_bits_rn((float)(w - (double)bf16_to_float(h)));
        const int kc = k / 8, kk = k % 8;
        row[((kc * 2 + 0) * NV + n) * 8 + kk] = h;
        row[((kc * 2 + 1) * NV + n) * 8 + kk] = l;
      }
    }
  }
  return out;
}

// Upload the weight matrices and the padded row table (plan creation).
int prepare_stencil_mma(Plan* p) {
  const int RBv = mma_rows_per_chunk<true>(), RBe = mma_rows_per_chunk<false>();
  p->mma_rows_pad_v = (int)cdiv(p->nrows, RBv) * RBv;
  p->mma_rows_pad_e = (int)cdiv(p->nrows, RBe) * RBe;
  const int npad = std::max(p->mma_rows_pad_v, p->mma_rows_pad_e);
  std::vector<int> rows(4 * (size_t)npad, 0);
  for (int r = 0; r < p->nrows; ++r)
    for (int j = 0; j < 4; ++j) rows[4 * r + j] = p->h_rows[4 * r + j];
  std::vector<uint8_t> bv = weight_matrices<true>(p, p->mma_rows_pad_v);
  std::vector<uint8_t> be = weight_matrices<false>(p, p->mma_rows_pad_e);
  if (cudaMalloc((void**)&p->d_mma_rows, sizeof(int) * rows.size()) != cudaSuccess ||
      cudaMalloc((void**)&p->d_mma_bv, bv.size()) != cudaSuccess ||
      cudaMalloc((void**)&p->d_mma_be, be.size()) != cudaSuccess)
    return MLS6_ERR_NOMEM;
  if (cudaMemcpy(p->d_mma_rows, rows.data(), sizeof(int) * rows.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_mma_bv, bv.data(), bv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(p->d_mma_be, be.data(), be.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return MLS6_ERR_CUDA;
  const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(k_stencil_mma<true>, attr, (int)mma_smem<true>(p->P)) != cudaSuccess ||
      cudaFuncSetAttribute(k_stencil_mma<false>, attr, (int)mma_smem<false>(p->P)) != cudaSuccess)
    return MLS6_ERR_CUDA;
  return MLS6_OK;
}

int launch_stencil_mma(Plan* p, bool vir, bool fuse_top, cudaStream_t st) {
  MmaArgs A;
  A.nlev = p->levels - 1;
  A.P = p->P;
  A.nrows = p->nrows;
  A.nrows_pad = vir ? p->mma_rows_pad_v : p->mma_rows_pad_e;
  A.stages = vir ? mma_stages<true>(p->P) : mma_stages<false>(p->P);
  A.rows = reinterpret_cast<const int4*>(p->d_mma_rows);
  A.B = vir ? p->d_mma_bv : p->d_mma_be;
  A.err = p->d_flag;
  const double* h = p->lv[1].h;
  A.hc[0] = h[0] * h[0];
  A.hc[1] = h[1] * h[1];
  A.hc[2] = h[2] * h[2];
  A.hc[3] = h[0] * h[1];
  A.hc[4] = h[0] * h[2];
  A.hc[5] = h[1] * h[2];
  for (int k = 1; k < p->levels; ++k) {
    MmaLevel& L = A.lv[k - 1];
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
  const long nb = p->stencil_blocks + (fuse_top ? cdiv(p->lv[l].np, kMmaThreads / 32) : 0);
  if (vir)
    launch_pdl(k_stencil_mma<true>, nb, kMmaThreads, mma_smem<true>(p->P), st, A, wp);
  else
    launch_pdl(k_stencil_mma<false>, nb, kMmaThreads, mma_smem<false>(p->P), st, A, wp);
  return 1;
}

}  // namespace mls6
