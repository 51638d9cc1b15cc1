// Internal definitions shared by the host plan (mls6_plan.cpp), the launch
// sequence (mls6_eval.cu) and the kernel translation units of the multilevel
// summation library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mls6.h"

namespace mls6 {

constexpr int kMaxLevels = 12;
constexpr int kBlock = 256;
constexpr int kScanTile = 2048;   // cells per block in the cell-count scan
constexpr int kReduceGroups = 64; // interpolation blocks that pre-reduce slices of the virial records
// Up to this many scan tiles the binning blocks add their atoms per tile
// (one global atomic per touched tile and block) and the tile pass is
// skipped; beyond it the per-block atomics cost more than the pass
// (65,536-atom slab, 27 tiles: bin stage 23.4 -> 18.0 us; 1M cube, 175 tiles:
// 69 -> 80 us).
constexpr int kScanDirect = 64;
constexpr int kStencilTile = 8;   // output tile edge of the level-stencil kernel
constexpr int kStencilThreads = 128;
constexpr int kStencilW = 4;      // consecutive x outputs per stencil thread
constexpr size_t kStencilSmemMax = 200 * 1024;  // dynamic shared memory of a stencil tile
constexpr double kCellDiv = 2.0;  // cell width >= a / kCellDiv
constexpr int kPairCluster = 1024;  // pair_split code of the cluster form
constexpr int kPairAtomBlock = 64;  // threads per block of the one-lane-per-atom pair kernel
constexpr int kPairSplitMax = 32;  // pair-kernel blocks are at most N * kPairSplitMax / kBlock

__host__ __device__ inline long cdiv(long a, long b) { return (a + b - 1) / b; }

// A caller's array that kernels read or write: device (or managed) memory,
// or page-locked host memory that the device addresses through the same
// pointer (unified addressing; kernels then reach it over the host link).
// The entry points refuse anything else with MLS6_ERR_ARG rather than hand
// it to a kernel.  Host only.
inline bool kernel_addressable(const void* ptr) {
  cudaPointerAttributes at;
  if (!ptr || cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeHost && at.devicePointer == ptr;
}

// 4-wide records: {x, y, z, c} positions, stencil tap weights.
template <typename T> struct alignas(4 * sizeof(T)) Vec4 {
  T x, y, z, w;
};

// Cell list used by the local (g_0) pair sum and for the spatial sort of
// the atoms.  Cells have width >= a/2 per axis, so neighbours within a lie
// at most R = ceil(a / w) cells away.
struct CellGeom {
  int nc[3];        // cells per axis
  int R[3];         // neighbour range per axis
  double w[3];      // cell width
  double inv_w[3];
  long ncell;
};

// Smoothing function gamma of continuity C^n: gamma = sum_k c[k] u^k for
// rho < 1, u = rho^12 (n = 2: Eq. gamma).
struct Smooth {
  int n = 2;
  double c[5] = {1.875, -1.25, 0.375, 0.0, 0.0};
};

// One grid level.
struct Level {
  int n[3];
  long np;
  double h[3];
};

struct Plan {
  // parameters
  double L[3];
  double a;
  int levels;
  int prec;  // mls6_precision
  int64_t N;
  cudaStream_t stream;

  CellGeom cg;
  Level lv[kMaxLevels + 1];  // 1-based
  Smooth sm;                 // smoothing function
  double c_self;             // gamma(0)/a^6
  int order = 3;             // interpolation order p: 3 (cubic) or 5 (quintic)

  // Level-1 stencil: taps m with |m h_1| < 2a, shared by all levels k < l
  // through the scale 2^(-6(k-1)) (Sec. II.A.4).  Taps are grouped in rows
  // of constant (dy, dz) with dx = -R..R contiguous.
  int ntaps = 0;
  int nrows = 0;
  int P = 0;                      // halo: max |m_d| over all taps and axes
  std::vector<int> h_rows;        // 4 per row: dy, dz, R, first tap
  std::vector<double> h_wv;       // 4 per tap: g_1, G = g_1'/r, G dx, G dx^2
  // stencil launch geometry: one block per 8^3 output tile, all levels k < l
  int tiles[kMaxLevels + 1][3] = {};
  long tile_off[kMaxLevels + 1] = {};
  long stencil_blocks = 0;
  size_t stencil_smem = 0;
  bool stencil_global = false;  // tile does not fit in shared memory
  int stencil_groups = 1;       // thread groups (of 128) sharing one tile
  bool stencil_tc = false;      // mma.sync tensor-core stencil (mixed precision)
  uint32_t* d_tcw = nullptr;    // its packed split weight pairs
  bool stencil_mma = false;     // tcgen05 tensor-core stencil (mixed precision)
  int stencil_req = 0;          // mls6_plan_options::stencil
  int mma_rows_pad_v = 0, mma_rows_pad_e = 0;  // tap rows padded to whole chunks
  int* d_mma_rows = nullptr;    // padded row table (int4: dy, dz, R, first)
  uint8_t* d_mma_bv = nullptr;  // B matrices, energy + six virial channels
  uint8_t* d_mma_be = nullptr;  // B matrices, energy channel only
  // coarsest level tables
  std::vector<double> h_top_T, h_top_V;

  // ------------------------------------------------------------ device
  void* d_pos_w = nullptr;     // Vec4<T>[N]: wrapped positions + c, input order
  int* d_cell_of = nullptr;    // int[N]
  int* d_cell_count = nullptr; // int[ncell]
  int* d_cell_start = nullptr; // int[ncell + 1]
  int* d_scan = nullptr;       // tile sums of the cell-count scan
  void* d_sorted = nullptr;    // Vec4<T>[N] sorted by cell
  int* d_sorted_idx = nullptr; // int[N] original index of sorted atom
  int pair_split = 1;          // lanes per atom in the pair kernel
  void* d_e0 = nullptr;        // T[N] local potential (sorted order)
  void* d_floc = nullptr;      // T[3N] local forces (sorted order)
  void* d_q1fx = nullptr;      // int32 (FP32 modes) / int64 (FP64) fixed-point anterpolation sums
  void* d_lbw = nullptr;       // T[N]: sqrt(2 eps) in sorted order (Lorentz-Berthelot)
  void* d_lbpot = nullptr;     // T[7 n_1]: level-1 total potential of each LB channel
  void* d_q[kMaxLevels + 1] = {};
  void* d_e[kMaxLevels + 1] = {};
  void* d_et[kMaxLevels + 1] = {};
  int* d_rows = nullptr;       // int4 per row
  void* d_wv = nullptr;        // Vec4<T> per tap
  double* d_top_T = nullptr;
  double* d_top_V = nullptr;
  double* d_epart = nullptr;   // energy partials (interpolation blocks)
  double* d_wpart = nullptr;   // virial partials: pair blocks | stencil blocks | top nodes
  long n_epart = 0, n_wpart = 0, n_pair_blocks = 0;
  // virial partials, in 6-double records: stencil blocks | coarsest nodes |
  // pair blocks (room for the largest lane split; only the records of the
  // current split are written and summed)
  long wpart_stencil = 0, wpart_top = 0, wpart_pair = 0;
  double* d_out = nullptr;     // [0] energy, [1..6] virial; [8..] kReduceGroups slice sums of 6
  int* d_flag = nullptr;       // [0] bit 0 non-finite, bit 1 wait timeout, [1] interpolation ticket, [2] tile-pass ticket,
                               // [3] max cell population, [4..5] max |c| (double),
                               // [6..7] max sqrt(2 eps) (double, Lorentz-Berthelot)
  double* h_out = nullptr;     // pinned host staging of d_out

  // per-stage event timing (mls6_profile): start/end event per stage
  static constexpr int kStages = 9;
  bool prof = false;
  cudaEvent_t ev_s[kStages] = {}, ev_e[kStages] = {};
  int launches = 0;            // kernels launched by the last evaluation

  // execution: internal non-blocking streams (main chain, pair branch),
  // ordered against the caller's stream by events; optional CUDA graph of
  // the whole evaluation, re-captured when its pointers or options change.
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
  bool use_graph = true;
  cudaGraphExec_t gexec = nullptr;
  struct GraphKey {
    const void *pos, *c, *forces, *energy, *virial, *atom_energy;
    bool vir, prof;
    bool operator==(const GraphKey& o) const {
      return pos == o.pos && c == o.c && forces == o.forces && energy == o.energy &&
             virial == o.virial && atom_energy == o.atom_energy && vir == o.vir && prof == o.prof;
    }
  } gkey = {};

  size_t elem() const { return prec == MLS6_FP64 ? sizeof(double) : sizeof(float); }
};

// host helpers (mls6_plan.cpp)
Smooth smooth_coefficients(int continuity);
double gamma_fn(const Smooth& s, double rho);
double dgamma_over_rho(const Smooth& s, double rho);  // gamma'(rho)/rho
double g_level(const Smooth& s, int k, int l, double a, double r);
double dg_level_over_r(const Smooth& s, int k, int l, double a, double r);

// launch sequence (mls6_eval.cu)
int eval_launch(Plan* p, const void* pos, const void* c, void* forces, double* energy,
                double* virial, double* atom_energy);
int upload_tables(Plan* p);
int plan_streams(Plan* p);  // create the plan's internal streams and events
int eval_lb(Plan* p, const void* pos, const void* sigma, const void* eps, void* forces,
            double* energy);
// Enqueue one evaluation on the plan's internal streams (cs, cs2), no
// ordering against the caller's stream; energy/virial written to device
// pointers if given.  Returns kernels launched or a negative status.
int enqueue_eval(Plan* p, const void* pos, const void* c, void* forces, double* energy_dev,
                 double* virial_dev, bool vir, bool capturing);

// kernel launchers; each returns the number of kernels it launched
template <typename T> int launch_bin(Plan* p, const T* pos, const T* c, cudaStream_t st);
template <typename T> int launch_pair(Plan* p, bool vir, cudaStream_t st, bool lb = false);
template <typename T> int launch_anterp(Plan* p, cudaStream_t st, int lbm = -1);
template <typename T> int launch_lb_weights(Plan* p, const T* eps, cudaStream_t st);
template <typename T> int launch_interp_lb(Plan* p, T* forces, cudaStream_t st);
template <typename T> int launch_restrict(Plan* p, int k, cudaStream_t st);
template <typename T> int launch_stencil(Plan* p, bool vir, cudaStream_t st);
template <typename T> int launch_top(Plan* p, bool vir, cudaStream_t st);
template <typename T> int launch_prolong(Plan* p, int k, cudaStream_t st);
template <typename T>
int launch_interp(Plan* p, T* forces, double* atom_energy, bool vir, cudaStream_t st);
template <typename T> int prepare_grid_kernels(Plan* p);
template <typename T> int prepare_pair_kernels(Plan* p);
int launch_reduce(Plan* p, bool vir, cudaStream_t st);
int flag_status(int flag_word);  // mls6_eval.cu
double lb_coef(int m);           // Lorentz-Berthelot channel coefficient (mls6_grid.cu)
int pair_split(const Plan* p);  // default lanes per atom of the pair kernel (mls6_pair.cu)
int pair_split_atom(const Plan* p);  // the default among the per-atom, warp and queue forms
bool pair_cl_ok(const Plan* p);      // the cluster form (kPairCluster) applies
bool pair_cluster_ok(const Plan* p);  // warp form usable (mls6_pair.cu)
// virial partial records summed by the final reduction
long pair_blocks(const Plan* p, int split);  // blocks of the pair kernel (mls6_pair.cu)
inline long wpart_used(const Plan* p) { return p->wpart_pair + pair_blocks(p, p->pair_split); }
bool stencil_fuses_top(const Plan* p);
// tensor-core stencil (mls6_stencil_tc.cu)
size_t tc_smem_bytes(int P);
bool stencil_tc_eligible(const Plan* p);
void tc_geometry(Plan* p);
std::vector<uint32_t> tc_weight_table(const Plan* p);
int prepare_stencil_tc(Plan* p);
int launch_stencil_tc(Plan* p, bool vir, bool fuse_top, cudaStream_t st);
// persistent batch execution (mls6_persist.cu)
struct PersistExec;
bool persist_eligible(const Plan* p);
int persist_build(PersistExec** out, Plan* const* plans, int B, const int64_t* off,
                  const double* cost, const void* pos, const void* c, void* forces, double* ew,
                  int* flags, bool vir);
int persist_set_wait(PersistExec* x, long long limit, long long withhold);
int persist_launch(PersistExec* x, cudaStream_t st);
void persist_free(PersistExec* x);
const int* persist_error_word(const PersistExec* x);
long long persist_items(const PersistExec* x);
int persist_grid(const PersistExec* x);
// tcgen05 stencil (mls6_stencil_mma.cu)
bool stencil_mma_eligible(const Plan* p);
long stencil_mma_tiles(const Plan* p);
void stencil_mma_geometry(Plan* p);
int prepare_stencil_mma(Plan* p);
int launch_stencil_mma(Plan* p, bool vir, bool fuse_top, cudaStream_t st);

}  // namespace mls6
