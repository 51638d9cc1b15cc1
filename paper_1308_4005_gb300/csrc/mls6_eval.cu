// Evaluation sequence of the multilevel summation library for r^-6
// dispersion (arXiv 1308.4005): a fixed order of kernels on the plan's
// stream, workspace allocation and table upload, the fixed-order energy /
// virial reduction, and the profiling and debug entry points.
//
//   bin      wrap positions, cell histogram, scan, scatter, per-cell order
//   pair     local part g_0 (Eq. g_0) over the cell list
//   anterp   Eq. (anterpolation) onto the finest grid
//   restrict xi^{k+1} = R xi^k (Sec. II.B, restriction)
//   stencil  Eq. (evaluation) on levels k < l (cutoff 2^k a)
//   top      Eq. (last-grid-periodic-transformed) on level l
//   prolong  e^{k,tot} = e^k + R^T e^{k+1,tot} (Sec. II.B, prolongation)
//   interp   Eq. (interpolation), its gradient (forces), per-atom energy
//   reduce   fixed-order sums of energy and virial partials
#include <algorithm>
#include <cmath>

#include "mls6_device.cuh"

namespace mls6 {

#define CK(x)                                    \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return MLS6_ERR_CUDA; \
  } while (0)


// Fixed-order reduction of the energy and virial partials (one block).
__global__ void k_reduce(const double* __restrict__ epart, long ne,
                         const double* __restrict__ wpart, long nw, int vir,
                         double* __restrict__ out) {
  const long z = pdl_begin();
  epart += z; wpart += z;
  __shared__ double sh[32 * 7];
  final_reduce(epart, ne, wpart, nw, vir, out, sh);
}

int launch_reduce(Plan* p, bool vir, cudaStream_t st) {
  launch_pdl(k_reduce, 1, kBlock, 0, st, p->d_epart, p->n_epart, p->d_wpart, wpart_used(p), vir ? 1 : 0,
                                 p->d_out);
  return 1;
}

// Status of the device flag word: bit 1 a bounded wait ran out, bit 0 a
// non-finite input.
int flag_status(int f) { return (f & 2) ? MLS6_ERR_TIMEOUT : (f ? MLS6_ERR_NONFINITE : MLS6_OK); }

static bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int dev_of(const Plan*) {
  int dev = 0;
  cudaGetDevice(&dev);
  return dev;
}

template <typename T> static int upload_tables_t(Plan* p) {
  const long N = p->N;
  const size_t e = sizeof(T);
  auto A = [&](void** ptr, size_t bytes) -> int {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(ptr, bytes) == cudaSuccess ? 0 : MLS6_ERR_NOMEM;
  };
  int rc = 0;
  rc |= A(&p->d_pos_w, sizeof(Vec4<T>) * N);
  rc |= A((void**)&p->d_cell_of, sizeof(int) * N);
  rc |= A((void**)&p->d_cell_count, sizeof(int) * p->cg.ncell);
  rc |= A((void**)&p->d_cell_start, sizeof(int) * (p->cg.ncell + 1));
  rc |= A((void**)&p->d_scan, 2 * sizeof(int) * std::max(1L, cdiv(p->cg.ncell, kScanTile)));
  rc |= A(&p->d_sorted, sizeof(Vec4<T>) * (N + 3));  // 3 padding records (pair kernel loads)
  rc |= A((void**)&p->d_sorted_idx, sizeof(int) * N);
  rc |= A(&p->d_e0, e * N);
  rc |= A(&p->d_floc, 3 * e * N);
  p->pair_split = pair_split(p);
  const int l = p->levels;
  for (int k = 1; k <= l; ++k) {
    rc |= A(&p->d_q[k], e * p->lv[k].np);
    rc |= A(&p->d_e[k], e * p->lv[k].np);
    if (k < l) rc |= A(&p->d_et[k], e * p->lv[k].np);
  }
  if (rc) return MLS6_ERR_NOMEM;
  p->d_et[l] = p->d_e[l];  // e^{l,tot} = e^l
  // stencil geometry: 8^3 tiles per level k < l
  p->stencil_blocks = 0;
  for (int k = 1; k < l; ++k) {
    p->tile_off[k] = p->stencil_blocks;
    long nt = 1;
    for (int d = 0; d < 3; ++d) {
      p->tiles[k][d] = (int)cdiv(p->lv[k].n[d], kStencilTile);
      nt *= p->tiles[k][d];
    }
    p->stencil_blocks += nt;
  }
  rc = prepare_grid_kernels<T>(p);  // may switch to the global-memory stencil
  if (rc) return rc;
  rc = prepare_pair_kernels<T>(p);
  if (rc) return rc;
  // mixed precision: tcgen05 stencil tiles, unless the grids give fewer than
  // two tiles per SM (the FP32 kernel's 8^3 tiles fill the device better:
  // 65,536-atom slab 35 vs 61 us) or the caller asked for the CUDA cores
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_of(p));
  const bool want_mma = p->stencil_req == 2 ||
                        (p->stencil_req == 0 && stencil_mma_tiles(p) >= 2L * std::max(sms, 1));
  if (want_mma && stencil_mma_eligible(p)) {
    stencil_mma_geometry(p);
    p->stencil_mma = true;
    p->stencil_global = false;
    rc = prepare_stencil_mma(p);
    if (rc) return rc;
  } else if (p->stencil_req == 2 && stencil_tc_eligible(p)) {  // mma.sync stencil tiles
    tc_geometry(p);
    p->stencil_tc = true;
    p->stencil_global = false;
    rc = prepare_stencil_tc(p);
    if (rc) return rc;
  }
  if (l >= 2) {
    rc |= A((void**)&p->d_rows, sizeof(int) * 4 * p->nrows);
    rc |= A(&p->d_wv, sizeof(Vec4<T>) * p->ntaps);
  }
  const long np_top = p->lv[l].np;
  rc |= A((void**)&p->d_top_T, sizeof(double) * np_top);
  rc |= A((void**)&p->d_top_V, 6 * sizeof(double) * np_top);
  // partial sums: pair blocks | stencil blocks | coarsest nodes
  p->n_epart = std::max(1L, cdiv(N, kBlock));
  // room for the largest lane split, so that the split can be retuned
  // without reallocation; records a smaller split does not write stay zero
  // virial partials of the pair sum: one per warp of the per-atom kernel
  // (<= 8 lanes per atom; every warp of its blocks, up to kBlock-thread
  // blocks, writes one), one per block of the other forms
  p->n_pair_blocks =
      std::max(1L, std::max(cdiv(N * 8, (long)kBlock) * (kBlock / 32), cdiv(N * kPairSplitMax, kBlock)));
  p->wpart_stencil = 0;
  p->wpart_top = p->stencil_blocks;
  p->wpart_pair = p->wpart_top + np_top;
  p->n_wpart = p->wpart_pair + p->n_pair_blocks;
  rc |= A((void**)&p->d_epart, sizeof(double) * p->n_epart);
  rc |= A((void**)&p->d_wpart, 6 * sizeof(double) * p->n_wpart);
  rc |= A((void**)&p->d_out, (8 + 6 * kReduceGroups) * sizeof(double));
  rc |= A((void**)&p->d_flag, sizeof(int) * 8);
  rc |= A(&p->d_q1fx, sizeof(unsigned long long) * p->lv[1].np);
  if (rc) return MLS6_ERR_NOMEM;
  if (cudaMallocHost((void**)&p->h_out, 8 * sizeof(double)) != cudaSuccess) return MLS6_ERR_NOMEM;

  if (l >= 2) {
    std::vector<Vec4<T>> wv((size_t)p->ntaps);
    for (int t = 0; t < p->ntaps; ++t) {
      wv[t].x = (T)p->h_wv[4 * t + 0];
      wv[t].y = (T)p->h_wv[4 * t + 1];
      wv[t].z = (T)p->h_wv[4 * t + 2];
      wv[t].w = (T)p->h_wv[4 * t + 3];
    }
    CK(cudaMemcpy(p->d_rows, p->h_rows.data(), sizeof(int) * p->h_rows.size(),
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->d_wv, wv.data(), sizeof(Vec4<T>) * wv.size(), cudaMemcpyHostToDevice));
  }
  if (p->stencil_tc) {
    std::vector<uint32_t> tw = tc_weight_table(p);
    if (cudaMalloc((void**)&p->d_tcw, sizeof(uint32_t) * tw.size()) != cudaSuccess)
      return MLS6_ERR_NOMEM;
    CK(cudaMemcpy(p->d_tcw, tw.data(), sizeof(uint32_t) * tw.size(), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(p->d_top_T, p->h_top_T.data(), sizeof(double) * np_top, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->d_top_V, p->h_top_V.data(), 6 * sizeof(double) * np_top,
                cudaMemcpyHostToDevice));
  CK(cudaMemset(p->d_flag, 0, sizeof(int) * 8));
  CK(cudaMemset(p->d_cell_count, 0, sizeof(int) * p->cg.ncell));  // reset by each binning
  CK(cudaMemset(p->d_scan, 0, 2 * sizeof(int) * std::max(1L, cdiv(p->cg.ncell, kScanTile))));
  CK(cudaMemset(p->d_wpart, 0, 6 * sizeof(double) * p->n_wpart));
  return MLS6_OK;
}

int upload_tables(Plan* p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MLS6_ERR_CUDA;
  }
  return p->prec == MLS6_FP64 ? upload_tables_t<double>(p) : upload_tables_t<float>(p);
}

// Enqueue one evaluation on the plan's internal streams: the main chain on
// cs, the pair sum on cs2 (forked after binning, joined before the
// interpolation that adds the local forces).  Returns kernels launched or
// a negative status.
template <typename T>
static int enqueue(Plan* p, const T* pos, const T* cc, T* forces, double* energy_dev,
                   double* virial_dev, bool vir, double* atom_energy, bool capturing) {
  // inside a capture, stage events must be external event-record nodes to
  // be timeable after the graph runs
  const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  // Profiling serialises the two branches so that each stage's events time
  // that stage alone.
  cudaStream_t st = p->cs, st2 = p->prof ? p->cs : p->cs2;
  const int N = (int)p->N;
  const int l = p->levels;
#define BEGIN(i, s)                                        \
  do {                                                      \
    if (p->prof) CK(cudaEventRecordWithFlags(p->ev_s[i], s, evf)); \
  } while (0)
#define END(i, s)                                           \
  do {                                                      \
    if (p->prof) CK(cudaEventRecordWithFlags(p->ev_e[i], s, evf)); \
  } while (0)
  int nl = 0;
  BEGIN(0, st);
  // flags, tickets, maxima (see Plan::d_flag); anterpolation sums
  CK(cudaMemsetAsync(p->d_flag, 0, sizeof(int) * 8, st));
  if (N > 0)
    CK(cudaMemsetAsync(p->d_q1fx, 0, sizeof(T) * p->lv[1].np, st));  // int32 or int64 sums
  else
    CK(cudaMemsetAsync(p->d_q[1], 0, sizeof(T) * p->lv[1].np, st));
  if (N > 0) nl += launch_bin<T>(p, pos, cc, st);
  END(0, st);
  if (N > 0) {
    CK(cudaEventRecord(p->ev_fork, st));
    CK(cudaStreamWaitEvent(st2, p->ev_fork, 0));
    BEGIN(1, st2);
    nl += launch_pair<T>(p, vir, st2);
    END(1, st2);
    CK(cudaEventRecord(p->ev_join, st2));
    BEGIN(2, st);
    nl += launch_anterp<T>(p, st);
    END(2, st);
  } else {
    // no atoms: grids stay zero; zero the atom-side partial sums
    CK(cudaMemsetAsync(p->d_epart, 0, sizeof(double) * p->n_epart, st));
    BEGIN(1, st);
    END(1, st);
    BEGIN(2, st);
    END(2, st);
  }
  BEGIN(3, st);
  for (int k = 1; k < l; ++k) nl += launch_restrict<T>(p, k, st);
  END(3, st);
  BEGIN(4, st);
  nl += launch_stencil<T>(p, vir, st);
  END(4, st);
  BEGIN(5, st);
  nl += launch_top<T>(p, vir, st);
  END(5, st);
  BEGIN(6, st);
  for (int k = l - 1; k >= 1; --k) nl += launch_prolong<T>(p, k, st);
  END(6, st);
  if (N > 0) CK(cudaStreamWaitEvent(st, p->ev_join, 0));
  // interpolation; its last block also performs the final reduction
  BEGIN(7, st);
  if (N > 0) nl += launch_interp<T>(p, forces, atom_energy, vir, st);
  END(7, st);
  BEGIN(8, st);
  if (N == 0) nl += launch_reduce(p, vir, st);
  END(8, st);
#undef BEGIN
#undef END
  if (energy_dev)
    CK(cudaMemcpyAsync(energy_dev, p->d_out, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (virial_dev)
    CK(cudaMemcpyAsync(virial_dev, p->d_out + 1, 6 * sizeof(double), cudaMemcpyDeviceToDevice,
                       st));
  return nl;
}

static int ensure_streams(Plan* p) {
  if (p->cs) return MLS6_OK;
  CK(cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&p->cs2, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  return MLS6_OK;
}

template <typename T>
static int eval_t(Plan* p, const void* pos_, const void* c_, void* forces_, double* energy,
                  double* virial, double* atom_energy) {
  const int N = (int)p->N;
  const bool vir = virial != nullptr;
  const T* pos = (const T*)pos_;
  const T* cc = (const T*)c_;
  T* forces = (T*)forces_;
  if (N > 0 && (!pos || !forces)) return MLS6_ERR_ARG;
  // inputs and per-atom outputs: device or page-locked host memory only
  if (N > 0 && (!kernel_addressable(pos) || (cc && !kernel_addressable(cc)) ||
                !kernel_addressable(forces) ||
                (atom_energy && !kernel_addressable(atom_energy))))
    return MLS6_ERR_ARG;
  int rc = ensure_streams(p);
  if (rc) return rc;
  double* energy_dev = (energy && is_device_ptr(energy)) ? energy : nullptr;
  double* virial_dev = (virial && is_device_ptr(virial)) ? virial : nullptr;
  const bool host_sync = (energy && !energy_dev) || (virial && !virial_dev);

  CK(cudaEventRecord(p->ev_in, p->stream));
  CK(cudaStreamWaitEvent(p->cs, p->ev_in, 0));
  if (p->use_graph) {
    Plan::GraphKey key = {pos_, c_, forces_, energy_dev, virial_dev, atom_energy, vir, p->prof};
    if (!p->gexec || !(key == p->gkey)) {
      if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
      }
      CK(cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeThreadLocal));
      int nl = enqueue<T>(p, pos, cc, forces, energy_dev, virial_dev, vir, atom_energy, true);
      cudaGraph_t graph = nullptr;
      cudaError_t ce = cudaStreamEndCapture(p->cs, &graph);
      if (nl < 0 || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return nl < 0 ? nl : MLS6_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&p->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        p->gexec = nullptr;
        return MLS6_ERR_CUDA;
      }
      p->gkey = key;
      p->launches = nl;
    }
    CK(cudaGraphLaunch(p->gexec, p->cs));
  } else {
    int nl = enqueue<T>(p, pos, cc, forces, energy_dev, virial_dev, vir, atom_energy, false);
    if (nl < 0) return nl;
    p->launches = nl;
  }
  CK(cudaGetLastError());
  if (host_sync) {
    CK(cudaMemcpyAsync(p->h_out, p->d_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, p->cs));
    int* h_flag = reinterpret_cast<int*>(p->h_out + 7);
    CK(cudaMemcpyAsync(h_flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, p->cs));
  }
  CK(cudaEventRecord(p->ev_out, p->cs));
  CK(cudaStreamWaitEvent(p->stream, p->ev_out, 0));
  if (host_sync) {
    CK(cudaStreamSynchronize(p->cs));
    if (energy && !energy_dev) *energy = p->h_out[0];
    if (virial && !virial_dev)
      for (int c = 0; c < 6; ++c) virial[c] = p->h_out[1 + c];
    if (const int f = *reinterpret_cast<int*>(p->h_out + 7)) return flag_status(f);
  }
  return MLS6_OK;
}

int plan_streams(Plan* p) { return ensure_streams(p); }

// Lorentz-Berthelot mixing (Sec. II.D): the local part with the exact pair
// coefficients, then the grid part once per channel m = 0..6 (anterpolation
// of xi_m, restriction, level stencils, coarsest level, prolongation; the
// level-1 total potential of each channel kept), and one interpolation that
// pairs channel m with xi_{6-m}.  Launched eagerly on the plan's main stream.
template <typename T>
static int eval_lb_t(Plan* p, const T* pos, const T* sigma, const T* eps, T* forces,
                     double* energy) {
  const long N = p->N;
  double* energy_dev = (energy && is_device_ptr(energy)) ? energy : nullptr;
  if (N == 0) {
    if (energy_dev) CK(cudaMemsetAsync(energy_dev, 0, sizeof(double), p->stream));
    else if (energy) *energy = 0.0;
    return MLS6_OK;
  }
  if (!pos || !sigma || !eps || !forces) return MLS6_ERR_ARG;
  if (!kernel_addressable(pos) || !kernel_addressable(sigma) || !kernel_addressable(eps) ||
      !kernel_addressable(forces))
    return MLS6_ERR_ARG;
  int rc = ensure_streams(p);
  if (rc) return rc;
  const long np1 = p->lv[1].np;
  if (!p->d_lbw) {
    if (cudaMalloc(&p->d_lbw, sizeof(T) * N) != cudaSuccess) return MLS6_ERR_NOMEM;
    if (cudaMalloc(&p->d_lbpot, sizeof(T) * 7 * np1) != cudaSuccess) return MLS6_ERR_NOMEM;
  }
  cudaStream_t st = p->cs;
  const int l = p->levels;
  CK(cudaEventRecord(p->ev_in, p->stream));
  CK(cudaStreamWaitEvent(st, p->ev_in, 0));
  CK(cudaMemsetAsync(p->d_flag, 0, sizeof(int) * 8, st));
  int nl = launch_bin<T>(p, pos, sigma, st);  // records carry sigma as the coefficient
  nl += launch_lb_weights<T>(p, eps, st);
  nl += launch_pair<T>(p, false, st, true);
  for (int m = 0; m < 7; ++m) {
    CK(cudaMemsetAsync(p->d_q1fx, 0, sizeof(T) * np1, st));
    nl += launch_anterp<T>(p, st, m);
    for (int k = 1; k < l; ++k) nl += launch_restrict<T>(p, k, st);
    nl += launch_stencil<T>(p, false, st);
    nl += launch_top<T>(p, false, st);
    for (int k = l - 1; k >= 1; --k) nl += launch_prolong<T>(p, k, st);
    CK(cudaMemcpyAsync((T*)p->d_lbpot + (size_t)m * np1, p->d_et[1], sizeof(T) * np1,
                       cudaMemcpyDeviceToDevice, st));
  }
  nl += launch_interp_lb<T>(p, forces, st);
  CK(cudaGetLastError());
  p->launches = nl;
  if (energy_dev)
    CK(cudaMemcpyAsync(energy_dev, p->d_out, sizeof(double), cudaMemcpyDeviceToDevice, st));
  const bool host = energy && !energy_dev;
  if (host) {
    CK(cudaMemcpyAsync(p->h_out, p->d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(reinterpret_cast<int*>(p->h_out + 7), p->d_flag, sizeof(int),
                       cudaMemcpyDeviceToHost, st));
  }
  CK(cudaEventRecord(p->ev_out, st));
  CK(cudaStreamWaitEvent(p->stream, p->ev_out, 0));
  if (host) {
    CK(cudaStreamSynchronize(st));
    *energy = p->h_out[0];
    if (const int f = *reinterpret_cast<int*>(p->h_out + 7)) return flag_status(f);
  }
  return MLS6_OK;
}

int eval_lb(Plan* p, const void* pos, const void* sigma, const void* eps, void* forces,
            double* energy) {
  if (p->sm.n != 2) return MLS6_ERR_ARG;  // Lorentz-Berthelot: Eq. (gamma) only
  if (p->prec == MLS6_FP64)
    return eval_lb_t<double>(p, (const double*)pos, (const double*)sigma, (const double*)eps,
                             (double*)forces, energy);
  return eval_lb_t<float>(p, (const float*)pos, (const float*)sigma, (const float*)eps,
                          (float*)forces, energy);
}

int enqueue_eval(Plan* p, const void* pos, const void* c, void* forces, double* energy_dev,
                 double* virial_dev, bool vir, bool capturing) {
  if (p->N > 0 && (!pos || !forces)) return MLS6_ERR_ARG;
  if (p->prec == MLS6_FP64)
    return enqueue<double>(p, (const double*)pos, (const double*)c, (double*)forces, energy_dev,
                           virial_dev, vir, nullptr, capturing);
  return enqueue<float>(p, (const float*)pos, (const float*)c, (float*)forces, energy_dev,
                        virial_dev, vir, nullptr, capturing);
}

int eval_launch(Plan* p, const void* pos, const void* c, void* forces, double* energy,
                double* virial, double* atom_energy) {
  return p->prec == MLS6_FP64 ? eval_t<double>(p, pos, c, forces, energy, virial, atom_energy)
                              : eval_t<float>(p, pos, c, forces, energy, virial, atom_energy);
}
}  // namespace mls6

using namespace mls6;

template <typename T> static int debug_grid_t(Plan* p, int level, int which, double* out) {
  const Level& Lk = p->lv[level];
  const void* src = which == 0 ? p->d_q[level] : which == 1 ? p->d_e[level] : p->d_et[level];
  std::vector<T> tmp((size_t)Lk.np);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MLS6_ERR_CUDA;
  if (cudaMemcpy(tmp.data(), src, sizeof(T) * Lk.np, cudaMemcpyDeviceToHost) != cudaSuccess)
    return MLS6_ERR_CUDA;
  for (long k = 0; k < Lk.np; ++k) out[k] = (double)tmp[k];
  return MLS6_OK;
}

extern "C" int mls6_debug_grid(mls6_plan_t* plan, int level, int which, double* host_out) {
  if (!plan || !host_out) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (level < 1 || level > p->levels || which < 0 || which > 2) return MLS6_ERR_ARG;
  return p->prec == MLS6_FP64 ? debug_grid_t<double>(p, level, which, host_out)
                              : debug_grid_t<float>(p, level, which, host_out);
}

static const char* kStageNames[Plan::kStages] = {
    "bin", "pair", "anterpolate", "restrict", "stencil", "coarsest", "prolongate", "interpolate",
    "reduce"};

extern "C" int mls6_profile(mls6_plan_t* plan, int enable) {
  if (!plan) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (enable && !p->ev_s[0])
    for (int i = 0; i < Plan::kStages; ++i)
      if (cudaEventCreate(&p->ev_s[i]) != cudaSuccess ||
          cudaEventCreate(&p->ev_e[i]) != cudaSuccess)
        return MLS6_ERR_CUDA;
  p->prof = enable != 0;
  return MLS6_OK;
}

extern "C" int mls6_set_graph(mls6_plan_t* plan, int enable) {
  if (!plan) return MLS6_ERR_ARG;
  reinterpret_cast<Plan*>(plan)->use_graph = enable != 0;
  return MLS6_OK;
}

extern "C" int mls6_stage_times(mls6_plan_t* plan, double* ms, int cap, int* launches) {
  if (!plan) return MLS6_ERR_ARG;
  Plan* p = reinterpret_cast<Plan*>(plan);
  if (launches) *launches = p->launches;
  if (!p->ev_s[0]) return 0;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MLS6_ERR_CUDA;
  for (int i = 0; i < Plan::kStages && i < cap; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev_s[i], p->ev_e[i]) != cudaSuccess) {
      cudaGetLastError();
      t = -1.f;
    }
    if (ms) ms[i] = (double)t;
  }
  return Plan::kStages;
}

extern "C" const char* mls6_stage_name(int i) {
  return (i >= 0 && i < Plan::kStages) ? kStageNames[i] : nullptr;
}
