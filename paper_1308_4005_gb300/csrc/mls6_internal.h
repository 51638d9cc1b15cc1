// Internal definitions shared by the host plan (mls6_plan.cpp) and the
// device code (mls6_eval.cu) of the multilevel summation library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mls6.h"

namespace mls6 {

constexpr int kMaxLevels = 12;
constexpr int kBlock = 256;

// 4-wide position+coefficient records: float4-like for FP32, 32-byte
// aligned quadruples for FP64.
template <typename T> struct alignas(4 * sizeof(T)) Vec4 {
  T x, y, z, w;
};

// Geometry of the cell list used by the local (g_0) pair sum and by the
// spatial sort of the atoms.  Cells have width >= a/2 per axis, so
// neighbours within a lie at most R = ceil(a / w) cells away.
struct CellGeom {
  int nc[3];        // cells per axis
  int R[3];         // neighbour range per axis
  double w[3];      // cell width
  double inv_w[3];
  long ncell;
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
  double c_self;             // gamma(0)/a^6

  // level-1 stencil (taps with |m h_1| < 2a), shared by all levels k < l
  // through the scale 2^(-6(k-1)) (Sec. II.A.4).
  int ntaps;
  int pad[3];                // halo width per axis of the padded grid copy
  std::vector<int> h_tap_m;  // 3 ints per tap
  std::vector<double> h_tap_g;   // g_1(|m h_1|)
  std::vector<double> h_tap_v;   // 6 per tap: g_1'(r)/r r_a r_b
  // coarsest level tables
  std::vector<double> h_top_T, h_top_V;

  // ------------------------------------------------------------ device
  void* d_pos_w = nullptr;     // Vec4<T>[N]: wrapped positions + c, input order
  int* d_cell_of = nullptr;    // int[N]
  int* d_cell_count = nullptr; // int[ncell]
  int* d_cell_start = nullptr; // int[ncell + 1]
  void* d_sorted = nullptr;    // Vec4<T>[N] sorted by cell
  int* d_sorted_idx = nullptr; // int[N] original index of sorted atom
  void* d_e0 = nullptr;        // T[N] local potential (sorted order)
  void* d_floc = nullptr;      // T[3N] local forces (sorted order)
  void* d_q[kMaxLevels + 1] = {};
  void* d_e[kMaxLevels + 1] = {};
  void* d_et[kMaxLevels + 1] = {};
  void* d_qpad = nullptr;      // padded copy of a level grid (largest level < l)
  int* d_tap_off = nullptr;    // per level: linear offsets in the padded grid
  void* d_tap_g = nullptr;     // T[ntaps]
  void* d_tap_v = nullptr;     // T[6 * ntaps]
  double* d_top_T = nullptr;
  double* d_top_V = nullptr;
  double* d_epart = nullptr;   // energy partials (interpolation blocks)
  double* d_wpart = nullptr;   // virial partials: pair blocks, stencil blocks, top
  long n_epart = 0, n_wpart = 0, n_pair_blocks = 0;
  int* d_scan = nullptr;       // tile sums of the cell-count scan
  long wpart_pair = 0;         // offsets into d_wpart
  long wpart_lvl[kMaxLevels + 1] = {};
  long wpart_top = 0;
  double* d_out = nullptr;     // [0] energy, [1..6] virial
  int* d_flag = nullptr;       // device error flags
  double* h_out = nullptr;     // pinned host staging of d_out

  // per-stage event timing (mls6_profile)
  static constexpr int kStages = 9;
  bool prof = false;
  cudaEvent_t ev[kStages + 1] = {};
  int launches = 0;            // kernels launched by the last evaluation

  size_t elem() const { return prec == MLS6_FP64 ? sizeof(double) : sizeof(float); }
};

// host helpers (mls6_plan.cpp)
double gamma_fn(double rho);
double dgamma_over_rho(double rho);  // gamma'(rho)/rho
double g_level(int k, int l, double a, double r);
double dg_level_over_r(int k, int l, double a, double r);

// device launch sequence (mls6_eval.cu)
int eval_launch(Plan* p, const void* pos, const void* c, void* forces, double* energy,
                double* virial, double* atom_energy);
int upload_tables(Plan* p);

}  // namespace mls6
