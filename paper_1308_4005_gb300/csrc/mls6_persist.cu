// Persistent execution of a batch of replicas: one kernel launch evaluates
// every replica of the batch.  Its blocks take work items -- (stage, replica,
// block) triples -- from a device queue in a fixed order and run the same
// kernel bodies as the per-stage launches (binning, local pair part,
// anterpolation, restriction, level stencils with the coarsest level,
// prolongation, interpolation with the final reduction), so each replica's
// results are those of a single plan evaluated with the same kernel shapes.
//
// Order and dependencies.  Items are numbered stage-major: every replica's
// blocks of stage 0, then of stage 1, and so on (within a stage, replicas in
// decreasing cost).  A block takes the next number with one atomic ticket;
// before running an item it waits until the replica's previous non-empty
// stage has counted all its blocks done (the pair sum and the grid chain
// depend only on the binning and meet at the interpolation), and after
// running it adds one to its own stage's counter.  Every item a block waits on has a smaller number
// and was therefore taken earlier by a block that is running (a block takes
// a number only when it is free), so the item with the smallest outstanding
// number never waits: the queue cannot deadlock, whatever the number of
// resident blocks.
//
// Bounded waits.  A wait polls at most `limit` times (with a short sleep
// between polls); when it runs out the block sets the queue's error word and
// every block leaves the kernel at its next item.  The host reports the word
// as MLS6_ERR_TIMEOUT.  A test hook withholds the completion count of one
// chosen item so that the waits behind it run out.
//
// Memory visibility.  This unit compiles the kernel bodies without the
// __restrict__ qualifiers, so that no load of data written earlier in the
// same launch (by other blocks) can go through the non-coherent read-only
// path; producers publish with a fence before the counter increment, and a
// consumer's polling thread fences after it sees the count, before the
// block barrier.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <numeric>
#include <vector>

#define __restrict__
#define MLS6_DEVICE_ONLY
#include "mls6_bin.cu"
#include "mls6_pair.cu"
#include "mls6_grid.cu"
#undef MLS6_DEVICE_ONLY
#undef __restrict__

namespace mls6 {

enum PStage : int {
  P_ZERO, P_BIN, P_SCAN_TILES, P_SCAN_FINAL, P_SCATTER, P_CELLSORT, P_PAIR, P_ANTERP,
  P_FROM_FIXED, P_RESTRICT, P_STENCIL, P_PROLONG, P_INTERP, P_OUT
};

struct ZeroP { int* a; long na; int* b; long nb; };
struct BinP {
  const float* pos; const float* cc; int stride, N; BinArgs<float> g;
  Vec4<float>* posw; int* cell_of; int* count; int* flag; int* tsum; int ntiles;
};
struct ScanTilesP { const int* count; long n; int* tsum; int* start; int* flag; };
struct ScanFinalP { int* count; long n; const int* tsum; int* start; int direct; int* flag; };
struct ScatterP {
  const Vec4<float>* posw; const int* cell_of; int N; const int* start; int* fill;
  Vec4<float>* sorted; int* sidx;
};
struct CellsortP {
  const int* start; long ncell; Vec4<float>* sorted; int* sidx; int* count; int* tsum;
  int nreset;
};
struct PairP {
  const Vec4<float>* sp; const int* start; int N; PairArgs<float> g; float* e0; float* floc;
  double* wpart; int S;
};
struct AnterpP {
  const Vec4<float>* sp; int N, n0, n1, n2; float ih0, ih1, ih2; const int* flag; double span;
  unsigned* qfx;
};
struct FromFixedP { const unsigned* qfx; long np; const int* flag; double span; float* q; };
struct RestrictP { const float* qf; int f0, f1, f2; float* qc; int c0, c1, c2; };
struct StencilP { StencilArgs<float> A; double* wpart; };
struct ProlongP { const float* ef; int f0, f1, f2; const float* etc_; int c0, c1, c2; float* etf; };
struct InterpP {
  const Vec4<float>* sp; const int* sidx; int N; const float* et; int n0, n1, n2;
  float ih0, ih1, ih2; const float* e0; const float* floc; double cself; float* forces;
  double* epart; ReduceArgs R; int slices;
};
struct OutP { const double* out; const int* flag; double* ew; int* flagdst; };

// One (replica, stage): its body and arguments, its block count and the
// replica's stages it waits for: the previous non-empty stage, except that
// the anterpolation does not wait for the pair sum (the two only read the
// sorted atoms) and the interpolation waits for both the grid chain and the
// pair sum.
struct PStageDesc {
  int kind;
  unsigned nb;
  int dep, dep2;            // stage indices waited for (-1: none)
  unsigned dep_nb, dep2_nb; // their block counts
  union U {
    ZeroP z; BinP bin; ScanTilesP st; ScanFinalP sf; ScatterP sc; CellsortP cs; PairP pair;
    AnterpP an; FromFixedP ff; RestrictP re; StencilP sten; ProlongP pr; InterpP in; OutP out;
    U() {}
  } u;
};

struct PQueue {
  unsigned long long ticket;  // next item
  int error;                  // bit 0: a bounded wait ran out
};

struct PExecArgs {
  const PStageDesc* st;            // [B][S]
  const long long* first;          // [S*B + 1] first item of (stage s, k-th replica in order)
  const int* order;                // replicas in decreasing cost
  unsigned* done;                  // [B][S] blocks completed
  PQueue* q;
  int B, S;
  long long total, limit, withhold;
};

template <bool VIR>
__device__ __forceinline__ void run_stage(const PStageDesc& d, unsigned b) {
  const Blk bk{b, d.nb};
  switch (d.kind) {
    case P_ZERO: {
      const ZeroP& a = d.u.z;
      for (long i = (long)b * blockDim.x + threadIdx.x; i < a.na; i += (long)d.nb * blockDim.x)
        a.a[i] = 0;
      for (long i = (long)b * blockDim.x + threadIdx.x; i < a.nb; i += (long)d.nb * blockDim.x)
        a.b[i] = 0;
      break;
    }
    case P_BIN: {
      const BinP& a = d.u.bin;
      k_bin_body<float>(bk, a.pos, a.cc, a.stride, a.N, a.g, a.posw, a.cell_of, a.count, a.flag,
                        a.tsum, a.ntiles);
      break;
    }
    case P_SCAN_TILES: {
      const ScanTilesP& a = d.u.st;
      k_scan_tiles_body(bk, a.count, a.n, a.tsum, a.start, a.flag);
      break;
    }
    case P_SCAN_FINAL: {
      const ScanFinalP& a = d.u.sf;
      k_scan_final_body(bk, a.count, a.n, a.tsum, a.start, a.direct, a.flag);
      break;
    }
    case P_SCATTER: {
      const ScatterP& a = d.u.sc;
      k_scatter_body<float>(bk, a.posw, a.cell_of, a.N, a.start, a.fill, a.sorted, a.sidx);
      break;
    }
    case P_CELLSORT: {
      const CellsortP& a = d.u.cs;
      k_cellsort_body<float>(bk, a.start, a.ncell, a.sorted, a.sidx, a.count, a.tsum, a.nreset);
      break;
    }
    case P_PAIR: {
      const PairP& a = d.u.pair;
      switch (a.S) {
        case 8:
          k_pair_body<float, VIR, 8, false, false>(bk, a.sp, a.start, a.N, a.g, a.e0, a.floc,
                                                   a.wpart, nullptr);
          break;
        case 4:
          k_pair_body<float, VIR, 4, false, false>(bk, a.sp, a.start, a.N, a.g, a.e0, a.floc,
                                                   a.wpart, nullptr);
          break;
        case 2:
          k_pair_body<float, VIR, 2, false, false>(bk, a.sp, a.start, a.N, a.g, a.e0, a.floc,
                                                   a.wpart, nullptr);
          break;
        default:
          k_pair_body<float, VIR, 1, false, false>(bk, a.sp, a.start, a.N, a.g, a.e0, a.floc,
                                                   a.wpart, nullptr);
          break;
      }
      break;
    }
    case P_ANTERP: {
      const AnterpP& a = d.u.an;
      k_anterp_body<float>(bk, a.sp, a.N, a.n0, a.n1, a.n2, a.ih0, a.ih1, a.ih2, a.flag, a.span,
                           a.qfx, nullptr, -1, 0.0);
      break;
    }
    case P_FROM_FIXED: {
      const FromFixedP& a = d.u.ff;
      k_from_fixed_body<float>(bk, a.qfx, a.np, a.flag, a.span, a.q, -1, 0.0);
      break;
    }
    case P_RESTRICT: {
      const RestrictP& a = d.u.re;
      k_restrict_body<float>(bk, a.qf, a.f0, a.f1, a.f2, a.qc, a.c0, a.c1, a.c2);
      break;
    }
    case P_STENCIL: {
      const StencilP& a = d.u.sten;
      k_stencil_body<float, VIR, 2>(bk, a.A, a.wpart);
      break;
    }
    case P_PROLONG: {
      const ProlongP& a = d.u.pr;
      k_prolong_body<float>(bk, a.ef, a.f0, a.f1, a.f2, a.etc_, a.c0, a.c1, a.c2, a.etf);
      break;
    }
    case P_INTERP: {
      const InterpP& a = d.u.in;
      if (a.slices)
        k_interp_body<float, true>(bk, a.sp, a.sidx, a.N, a.et, a.n0, a.n1, a.n2, a.ih0, a.ih1,
                                   a.ih2, a.e0, a.floc, a.cself, a.forces, nullptr, a.epart, a.R);
      else
        k_interp_body<float, false>(bk, a.sp, a.sidx, a.N, a.et, a.n0, a.n1, a.n2, a.ih0, a.ih1,
                                    a.ih2, a.e0, a.floc, a.cself, a.forces, nullptr, a.epart,
                                    a.R);
      break;
    }
    case P_OUT: {
      const OutP& a = d.u.out;
      if (threadIdx.x < 7) a.ew[threadIdx.x] = a.out[threadIdx.x];
      if (threadIdx.x == 0) *a.flagdst = *a.flag;
      break;
    }
    default: break;
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <bool VIR>
__global__ void __launch_bounds__(kStencilThreads * 2) k_persist(PExecArgs X) {
  __shared__ long long s_t;
  __shared__ int s_go, s_lo;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long t = (long long)atomicAdd(&X.q->ticket, 1ull);
      // the (stage, replica) range that holds item t: first[lo] <= t < first[lo+1]
      int lo = 0, hi = X.S * X.B;
      if (t < X.total)
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (X.first[mid] <= t) lo = mid;
          else hi = mid;
        }
      s_t = t;
      s_lo = lo;
    }
    __syncthreads();
    const long long t = s_t;
    if (t >= X.total) return;
    const int lo = s_lo;
    const int s = lo / X.B, r = X.order[lo % X.B];
    const PStageDesc& d = X.st[(size_t)r * X.S + s];
    const unsigned b = (unsigned)(t - X.first[lo]);
    if (threadIdx.x == 0) {
      int go = *(volatile int*)&X.q->error ? 0 : 1;
      for (int k = 0; k < 2 && go; ++k) {
        const int dep = k ? d.dep2 : d.dep;
        if (dep < 0) continue;
        const unsigned need = k ? d.dep2_nb : d.dep_nb;
        const unsigned* cnt = X.done + (size_t)r * X.S + dep;
        for (long long it = 0;; ++it) {
          if (ld_acquire(cnt) >= need) break;
          if (it >= X.limit || *(volatile int*)&X.q->error) {
            atomicOr(&X.q->error, 1);
            go = 0;
            break;
          }
          __nanosleep(100);
        }
      }
      __threadfence();
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;  // a wait ran out: leave the kernel
    run_stage<VIR>(d, b);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (t != X.withhold) atomicAdd(X.done + (size_t)r * X.S + s, 1u);
    }
  }
}

// ------------------------------------------------------------------ host

struct PersistExec {
  int B = 0, S = 0;
  bool vir = false;
  PStageDesc* d_st = nullptr;
  long long* d_first = nullptr;
  int* d_order = nullptr;
  unsigned* d_done = nullptr;
  PQueue* d_q = nullptr;
  long long total = 0;
  long long limit = 1LL << 22;
  long long withhold = -1;
  int grid = 0;
  size_t smem = 0;
};

bool persist_eligible(const Plan* p) {
  return p->prec == MLS6_FP32 && p->N > 0 && p->levels >= 2 && !p->stencil_global &&
         !p->stencil_mma && !p->stencil_tc && p->pair_split >= 1 && p->pair_split <= 8 &&
         p->sm.n == 2 && p->order == 3 && p->levels <= kMaxLevels;
}

// The stage list of one replica (mirrors the launch sequence of a single
// evaluation with the pair sum before the anterpolation).
static void replica_stages(Plan* p, const float* pos, const float* cc, float* forces,
                           double* ew, int* flagdst, bool vir, int lmax,
                           std::vector<PStageDesc>& out) {
  const int N = (int)p->N, l = p->levels;
  const Level& L1 = p->lv[1];
  auto add = [&](int kind, long nb) -> PStageDesc& {
    out.emplace_back();
    PStageDesc& d = out.back();
    d.kind = kind;
    d.nb = (unsigned)std::max(0L, nb);
    d.dep = d.dep2 = -1;
    d.dep_nb = d.dep2_nb = 0;
    return d;
  };
  {
    PStageDesc& d = add(P_ZERO, cdiv(L1.np, 8L * kBlock));
    d.u.z = ZeroP{p->d_flag, 8, (int*)p->d_q1fx, L1.np};
  }
  const long ncell = p->cg.ncell, ntiles = cdiv(ncell, kScanTile);
  const bool direct = ntiles <= kScanDirect;
  {
    PStageDesc& d = add(P_BIN, cdiv(N, kBlock));
    d.u.bin = BinP{pos, cc, cc ? 3 : 4, N, bin_args<float>(p), (Vec4<float>*)p->d_pos_w,
                   p->d_cell_of, p->d_cell_count, p->d_flag, direct ? p->d_scan : nullptr,
                   (int)ntiles};
  }
  {
    PStageDesc& d = add(P_SCAN_TILES, direct ? 0 : ntiles);
    d.u.st = ScanTilesP{p->d_cell_count, ncell, p->d_scan, p->d_cell_start, p->d_flag};
  }
  {
    PStageDesc& d = add(P_SCAN_FINAL, ntiles);
    d.u.sf = ScanFinalP{p->d_cell_count, ncell, p->d_scan, p->d_cell_start, direct ? 1 : 0,
                        p->d_flag};
  }
  {
    PStageDesc& d = add(P_SCATTER, cdiv(N, kBlock));
    d.u.sc = ScatterP{(const Vec4<float>*)p->d_pos_w, p->d_cell_of, N, p->d_cell_start,
                      p->d_cell_count, (Vec4<float>*)p->d_sorted, p->d_sorted_idx};
  }
  {
    PStageDesc& d = add(P_CELLSORT, cdiv(std::max(ncell, ntiles), kBlock));
    d.u.cs = CellsortP{p->d_cell_start, ncell, (Vec4<float>*)p->d_sorted, p->d_sorted_idx,
                       p->d_cell_count, p->d_scan, direct ? (int)ntiles : 0};
  }
  {
    PStageDesc& d = add(P_PAIR, cdiv((long)N * p->pair_split, kBlock));
    d.u.pair = PairP{(const Vec4<float>*)p->d_sorted, p->d_cell_start, N, pair_args<float>(p),
                     (float*)p->d_e0, (float*)p->d_floc, p->d_wpart + 6 * p->wpart_pair,
                     p->pair_split};
  }
  const double span = support_span(p);
  {
    PStageDesc& d = add(P_ANTERP, cdiv(N, kBlock));
    d.u.an = AnterpP{(const Vec4<float>*)p->d_sorted, N, L1.n[0], L1.n[1], L1.n[2],
                     (float)(1.0 / L1.h[0]), (float)(1.0 / L1.h[1]), (float)(1.0 / L1.h[2]),
                     p->d_flag, span, (unsigned*)p->d_q1fx};
  }
  {
    PStageDesc& d = add(P_FROM_FIXED, cdiv(L1.np, kBlock));
    d.u.ff = FromFixedP{(const unsigned*)p->d_q1fx, L1.np, p->d_flag, span, (float*)p->d_q[1]};
  }
  for (int k = 1; k < lmax; ++k) {  // restriction slots (empty beyond this replica's levels)
    const bool on = k < l;
    PStageDesc& d = add(P_RESTRICT, on ? cdiv(p->lv[k + 1].np, kBlock) : 0);
    if (on) {
      const Level &F = p->lv[k], &C = p->lv[k + 1];
      d.u.re = RestrictP{(const float*)p->d_q[k], F.n[0], F.n[1], F.n[2], (float*)p->d_q[k + 1],
                         C.n[0], C.n[1], C.n[2]};
    }
  }
  {
    const int warps = kStencilThreads * 2 / 32;
    PStageDesc& d = add(P_STENCIL, p->stencil_blocks + cdiv(p->lv[l].np, warps));
    d.u.sten.A = stencil_args<float>(p);
    d.u.sten.wpart = p->d_wpart + 6 * p->wpart_stencil;
  }
  for (int j = 0; j < lmax - 1; ++j) {  // prolongation slots, coarse to fine
    const int k = l - 1 - j;
    const bool on = k >= 1;
    PStageDesc& d = add(P_PROLONG, on ? cdiv(p->lv[k].np, kBlock) : 0);
    if (on) {
      const Level &F = p->lv[k], &C = p->lv[k + 1];
      d.u.pr = ProlongP{(const float*)p->d_e[k], F.n[0], F.n[1], F.n[2],
                        (const float*)p->d_et[k + 1], C.n[0], C.n[1], C.n[2], (float*)p->d_et[k]};
    }
  }
  {
    const bool slices = cdiv(N, kBlock) >= 4L * 152;
    PStageDesc& d = add(P_INTERP, cdiv(N, kBlock));
    ReduceArgs R = {p->d_wpart, wpart_used(p), vir ? 1 : 0, p->d_out,
                    reinterpret_cast<unsigned*>(p->d_flag + 1), p->d_out + 8,
                    slices ? kReduceGroups : 0};
    d.u.in = InterpP{(const Vec4<float>*)p->d_sorted, p->d_sorted_idx, N, (const float*)p->d_et[1],
                     L1.n[0], L1.n[1], L1.n[2], (float)(1.0 / L1.h[0]), (float)(1.0 / L1.h[1]),
                     (float)(1.0 / L1.h[2]), (const float*)p->d_e0, (const float*)p->d_floc,
                     p->c_self, forces, p->d_epart, R, slices ? 1 : 0};
  }
  {
    PStageDesc& d = add(P_OUT, 1);
    d.u.out = OutP{p->d_out, p->d_flag, ew, flagdst};
  }
}

void persist_free(PersistExec* x) {
  if (!x) return;
  void* ptrs[] = {x->d_st, x->d_first, x->d_order, x->d_done, x->d_q};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete x;
}

int persist_build(PersistExec** out, Plan* const* plans, int B, const int64_t* off,
                  const double* cost, const void* pos, const void* c, void* forces, double* ew,
                  int* flags, bool vir) {
  *out = nullptr;
  for (int r = 0; r < B; ++r)
    if (!persist_eligible(plans[r])) return MLS6_ERR_ARG;
  int lmax = 2;
  for (int r = 0; r < B; ++r) lmax = std::max(lmax, plans[r]->levels);
  PersistExec* x = new (std::nothrow) PersistExec();
  if (!x) return MLS6_ERR_NOMEM;
  x->B = B;
  x->vir = vir;
  std::vector<PStageDesc> st;
  for (int r = 0; r < B; ++r) {
    const size_t o = (size_t)off[r];
    const float* pr = (const float*)pos + o * (c ? 3 : 4);
    const float* cr = c ? (const float*)c + o : nullptr;
    float* fr = (float*)forces + o * 3;
    const size_t before = st.size();
    replica_stages(plans[r], pr, cr, fr, ew + 7 * (size_t)r, flags + r, vir, lmax, st);
    x->S = (int)(st.size() - before);
  }
  const int S = x->S;
  // dependencies: the replica's previous non-empty stage; the pair sum runs
  // beside the grid chain (anterpolation waits for the binning only, the
  // interpolation for the prolongation and the pair sum)
  for (int r = 0; r < B; ++r) {
    PStageDesc* row = &st[(size_t)r * S];
    int last = -1, pair = -1, before_pair = -1;
    for (int s = 0; s < S; ++s) {
      PStageDesc& d = row[s];
      d.dep = last;
      if (d.kind == P_ANTERP) d.dep = before_pair;
      if (d.kind == P_INTERP && pair >= 0 && pair != last) d.dep2 = pair;
      d.dep_nb = d.dep >= 0 ? row[d.dep].nb : 0;
      d.dep2_nb = d.dep2 >= 0 ? row[d.dep2].nb : 0;
      if (d.kind == P_PAIR) {
        before_pair = last;
        pair = d.nb > 0 ? s : -1;
      }
      if (d.nb > 0) last = s;
    }
  }
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<long long> first((size_t)S * B + 1, 0);
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < B; ++k) {
      const size_t i = (size_t)s * B + k;
      first[i + 1] = first[i] + st[(size_t)order[k] * S + s].nb;
    }
  x->total = first.back();
  size_t smem = 0;
  for (int r = 0; r < B; ++r) smem = std::max(smem, plans[r]->stencil_smem);
  x->smem = smem;
  int rc = MLS6_OK;
  auto A = [&](void** ptr, size_t bytes) {
    if (cudaMalloc(ptr, std::max(bytes, (size_t)16)) != cudaSuccess) rc = MLS6_ERR_NOMEM;
  };
  A((void**)&x->d_st, sizeof(PStageDesc) * st.size());
  A((void**)&x->d_first, sizeof(long long) * first.size());
  A((void**)&x->d_order, sizeof(int) * B);
  A((void**)&x->d_done, sizeof(unsigned) * (size_t)B * S);
  A((void**)&x->d_q, sizeof(PQueue));
  if (!rc && (cudaMemcpy(x->d_st, st.data(), sizeof(PStageDesc) * st.size(),
                         cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemcpy(x->d_first, first.data(), sizeof(long long) * first.size(),
                         cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemcpy(x->d_order, order.data(), sizeof(int) * B, cudaMemcpyHostToDevice) !=
                  cudaSuccess))
    rc = MLS6_ERR_CUDA;
  const auto kern = vir ? k_persist<true> : k_persist<false>;
  if (!rc && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::max(smem, (size_t)1)) != cudaSuccess)
    rc = MLS6_ERR_CUDA;
  int dev = 0, sms = 0, per_sm = 0;
  if (!rc) {
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kStencilThreads * 2, smem) !=
            cudaSuccess ||
        per_sm < 1)
      rc = MLS6_ERR_CUDA;
  }
  if (rc) {
    cudaGetLastError();
    persist_free(x);
    return rc;
  }
  x->grid = sms * per_sm;
  *out = x;
  return MLS6_OK;
}

int persist_set_wait(PersistExec* x, long long limit, long long withhold) {
  if (!x || limit < 1) return MLS6_ERR_ARG;
  x->limit = limit;
  x->withhold = withhold;
  return MLS6_OK;
}

// Enqueue one execution: reset the queue and the counters, launch the
// persistent kernel.  Returns kernels launched (1) or a negative status.
int persist_launch(PersistExec* x, cudaStream_t st) {
  if (cudaMemsetAsync(x->d_q, 0, sizeof(PQueue), st) != cudaSuccess ||
      cudaMemsetAsync(x->d_done, 0, sizeof(unsigned) * (size_t)x->B * x->S, st) != cudaSuccess)
    return MLS6_ERR_CUDA;
  PExecArgs a{x->d_st, x->d_first, x->d_order, x->d_done, x->d_q, x->B, x->S,
              x->total, x->limit, x->withhold};
  if (x->vir)
    k_persist<true><<<x->grid, kStencilThreads * 2, x->smem, st>>>(a);
  else
    k_persist<false><<<x->grid, kStencilThreads * 2, x->smem, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? 1 : MLS6_ERR_CUDA;
}

const int* persist_error_word(const PersistExec* x) { return &x->d_q->error; }
long long persist_items(const PersistExec* x) { return x->total; }
int persist_grid(const PersistExec* x) { return x->grid; }

}  // namespace mls6
