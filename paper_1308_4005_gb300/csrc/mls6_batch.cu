// Batches of independent replicas (systems of uneven size, each its own box
// and grid hierarchy) evaluated by one CUDA graph launch.
//
// FP32 batches can run one persistent kernel inside that graph instead
// (mls6_batch_set_mode(b, 1)): a device work queue of (stage, replica, block)
// items with bounded waits (mls6_persist.cu).  By default, and whenever the
// autotuner measures it faster, the graph holds every replica's kernel
// chain:
//
// Every replica is a complete plan (its own workspace and tables); the batch
// captures all their kernel sequences into a single graph whose replicas are
// spread over K independent chains ("branches"), so that kernels of small
// replicas, which cannot fill the GPU alone, run side by side.  Replicas are
// assigned to branches by longest-processing-time-first on a cost model
// (Sec. IV, Eq. cost: C_local (a/d)^3 N + C_grids (a/h)^3 V/h^3, plus the
// per-atom transfers, the coarsest product and a per-launch latency that
// dominate small replicas), and the autotuner picks the branch count and the
// per-replica kernel shapes (pair-kernel lanes per atom, stencil thread
// groups) by timing whole-batch launches.  Each replica runs the same kernels
// as a single plan with the same shapes, so its results are bitwise those of
// mls6_eval on that plan.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>
#include <vector>

#include "mls6_internal.h"

namespace mls6 {

#define CK(x)                                    \
  do {                                           \
    cudaError_t e_ = (x);                        \
    if (e_ != cudaSuccess) return MLS6_ERR_CUDA; \
  } while (0)

struct Batch {
  int B = 0;
  int prec = MLS6_FP64;
  std::vector<Plan*> plans;
  std::vector<int64_t> off;  // first atom of each replica
  std::vector<double> cost;  // model cost (seconds)
  int branches = 1;
  std::vector<int> branch_of;
  cudaStream_t stream = nullptr;  // caller's stream
  cudaStream_t s0 = nullptr;      // capture origin
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_root = nullptr;
  double* d_ew = nullptr;         // 7 per replica: energy, virial (6)
  int* d_flags = nullptr;         // non-finite flag per replica
  const int** d_flag_src = nullptr;
  double* h_ew = nullptr;         // pinned: 7 per replica + flags
  cudaGraphExec_t gexec = nullptr;
  int launches = 0;               // kernels in the captured graph
  int mode = 0;                   // 1: one persistent kernel where eligible, 0: kernel chains
  bool persistent = false;        // the captured graph runs the persistent kernel
  PersistExec* px = nullptr;      // its work queue (rebuilt with the graph)
  long long wait_limit = 1LL << 22, withhold = -1;  // bounded waits, test hook
  int* h_err = nullptr;           // pinned: the queue's error word
  struct Key {
    const void *pos, *c, *forces;
    bool vir;
    bool operator==(const Key& o) const {
      return pos == o.pos && c == o.c && forces == o.forces && vir == o.vir;
    }
  } key = {};
  size_t elem() const { return prec == MLS6_FP64 ? sizeof(double) : sizeof(float); }
};

// Cost model coefficients (seconds), from stage timings of a 65,536-atom
// slab (a = 3, h = 1.25) on GB300: per neighbour-pair volume term, per
// tap x node, per atom (binning, anterpolation, interpolation, transfers),
// per coarsest-node pair, per kernel launch.
static const double kCostDefault[5] = {1.6e-10, 4.0e-11, 1.7e-9, 3.4e-10, 2.5e-6};

static double model_cost(const double box[3], int64_t N, double a, double h, int levels,
                         const double* coef) {
  const double* k = coef ? coef : kCostDefault;
  const double V = box[0] * box[1] * box[2];
  const double local = (double)N * (a * a * a * (double)N / V);  // (a/d)^3 N
  double grids = 0.0, top = 0.0;
  if (levels >= 2) grids = std::pow(a / h, 3) * V / (h * h * h) * 8.0 / 7.0;
  const double nl = V / std::pow(h * std::ldexp(1.0, levels - 1), 3);
  top = nl * nl;
  const int launches = 8 + 2 * (levels - 1);
  return k[0] * local + k[1] * grids + k[2] * (double)N + k[3] * top + k[4] * launches;
}

// Longest processing time first: replicas in decreasing cost, each to the
// least-loaded branch (ties to the lower branch index).
static void lpt(int B, const double* cost, int K, int* branch_of, double* load) {
  std::vector<int> order(B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<double> L(K, 0.0);
  for (int r : order) {
    int best = 0;
    for (int k = 1; k < K; ++k)
      if (L[k] < L[best]) best = k;
    branch_of[r] = best;
    L[best] += cost[r];
  }
  if (load)
    for (int k = 0; k < K; ++k) load[k] = L[k];
}

static void free_batch(Batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  persist_free(b->px);
  if (b->h_err) cudaFreeHost(b->h_err);
  for (Plan* p : b->plans)
    if (p) mls6_destroy(reinterpret_cast<mls6_plan_t*>(p));
  if (b->d_ew) cudaFree(b->d_ew);
  if (b->d_flags) cudaFree(b->d_flags);
  if (b->d_flag_src) cudaFree(b->d_flag_src);
  if (b->h_ew) cudaFreeHost(b->h_ew);
  cudaEvent_t evs[] = {b->ev_in, b->ev_out, b->ev_root};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (b->s0) cudaStreamDestroy(b->s0);
  delete b;
}

// Gathers the replicas' non-finite flags (one word each) into one array.
__global__ void k_gather_flags(const int* const* __restrict__ src, int B, int* __restrict__ dst) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < B) dst[r] = *src[r];
}

static void reset_graph(Batch* b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  if (b->px) {
    persist_free(b->px);
    b->px = nullptr;
  }
  b->persistent = false;
}

static void assign(Batch* b) {
  b->branch_of.assign(b->B, 0);
  lpt(b->B, b->cost.data(), b->branches, b->branch_of.data(), nullptr);
}

// Capture every replica into one graph: K chains from a common root, each
// replica ordered after the previous one of its chain, all chains joined
// before the flag gather.
// The persistent form: one graph of two small resets and one kernel that
// runs every replica's stages from a device work queue (mls6_persist.cu).
static int capture_persistent(Batch* b, const void* pos, const void* c, void* forces, bool vir) {
  // the persistent kernel's blocks have 256 threads: two stencil thread
  // groups per tile; the replicas' plans take that shape too, so that each
  // still equals its own plan bit for bit
  for (Plan* p : b->plans) {
    const int rc = mls6_set_tuning(reinterpret_cast<mls6_plan_t*>(p), 0, 2);
    if (rc) return rc;
  }
  PersistExec* x = nullptr;
  int rc = persist_build(&x, b->plans.data(), b->B, b->off.data(), b->cost.data(), pos, c,
                         forces, b->d_ew, b->d_flags, vir);
  if (rc) return rc;
  persist_set_wait(x, b->wait_limit, b->withhold);
  CK(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal));
  const int nl = persist_launch(x, b->s0);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->s0, &graph);
  if (nl < 0 || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    persist_free(x);
    return nl < 0 ? nl : MLS6_ERR_CUDA;
  }
  ce = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    b->gexec = nullptr;
    persist_free(x);
    return MLS6_ERR_CUDA;
  }
  b->px = x;
  b->persistent = true;
  b->key = {pos, c, forces, vir};
  b->launches = nl;
  return MLS6_OK;
}

static bool persistent_ok(const Batch* b) {
  if (b->mode != 1 || b->prec != MLS6_FP32) return false;
  for (const Plan* p : b->plans)
    if (!persist_eligible(p)) return false;
  return true;
}

static int capture(Batch* b, const void* pos, const void* c, void* forces, bool vir) {
  reset_graph(b);
  if (persistent_ok(b)) return capture_persistent(b, pos, c, forces, vir);
  const size_t e = b->elem();
  const int K = b->branches;
  std::vector<cudaEvent_t> tail(K, b->ev_root);
  int launches = 1;  // the flag gather
  // chain order: by branch, replicas in decreasing cost (as LPT placed them)
  std::vector<int> order(b->B);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->cost[x] > b->cost[y]; });
  CK(cudaStreamBeginCapture(b->s0, cudaStreamCaptureModeThreadLocal));
  int rc = MLS6_OK;
  cudaEventRecord(b->ev_root, b->s0);
  for (int r : order) {
    Plan* p = b->plans[r];
    const int k = b->branch_of[r];
    if (cudaStreamWaitEvent(p->cs, tail[k], 0) != cudaSuccess) {
      rc = MLS6_ERR_CUDA;
      break;
    }
    const size_t o = (size_t)b->off[r];
    const char* pr = (const char*)pos + o * (c ? 3 : 4) * e;
    const char* cr = c ? (const char*)c + o * e : nullptr;
    char* fr = (char*)forces + o * 3 * e;
    int nl = enqueue_eval(p, pr, cr, fr, b->d_ew + 7 * (size_t)r,
                          vir ? b->d_ew + 7 * (size_t)r + 1 : nullptr, vir, true);
    if (nl < 0) {
      rc = nl;
      break;
    }
    launches += nl;
    if (cudaEventRecord(p->ev_out, p->cs) != cudaSuccess) {
      rc = MLS6_ERR_CUDA;
      break;
    }
    tail[k] = p->ev_out;
  }
  if (rc == MLS6_OK)
    for (int k = 0; k < K; ++k)
      if (cudaStreamWaitEvent(b->s0, tail[k], 0) != cudaSuccess) rc = MLS6_ERR_CUDA;
  if (rc == MLS6_OK) {
    k_gather_flags<<<(b->B + 127) / 128, 128, 0, b->s0>>>(b->d_flag_src, b->B, b->d_flags);
    if (cudaGetLastError() != cudaSuccess) rc = MLS6_ERR_CUDA;
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(b->s0, &graph);
  if (rc != MLS6_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != MLS6_OK ? rc : MLS6_ERR_CUDA;
  }
  ce = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    b->gexec = nullptr;
    return MLS6_ERR_CUDA;
  }
  b->key = {pos, c, forces, vir};
  b->launches = launches;
  return MLS6_OK;
}

static bool is_dev(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static bool arrays_ok(const void* pos, const void* c, const void* forces) {
  return pos && forces && kernel_addressable(pos) && kernel_addressable(forces) &&
         (!c || kernel_addressable(c));
}

static int launch(Batch* b, const void* pos, const void* c, void* forces, bool vir) {
  Batch::Key key = {pos, c, forces, vir};
  if (!b->gexec || !(key == b->key)) {
    int rc = capture(b, pos, c, forces, vir);
    if (rc) return rc;
  }
  CK(cudaEventRecord(b->ev_in, b->stream));
  CK(cudaStreamWaitEvent(b->s0, b->ev_in, 0));
  CK(cudaGraphLaunch(b->gexec, b->s0));
  return MLS6_OK;
}

static int eval(Batch* b, const void* pos, const void* c, void* forces, double* energy,
                double* virial) {
  const int64_t ntot = b->off[b->B];
  if (ntot > 0 && !arrays_ok(pos, c, forces)) return MLS6_ERR_ARG;
  const bool vir = virial != nullptr;
  int rc = launch(b, pos, c, forces, vir);
  if (rc) return rc;
  const size_t B = (size_t)b->B;
  // strided copies out of the 7-per-replica record
  const bool host = (energy && !is_dev(energy)) || (virial && !is_dev(virial));
  if (host) {
    CK(cudaMemcpyAsync(b->h_ew, b->d_ew, 7 * sizeof(double) * B, cudaMemcpyDeviceToHost, b->s0));
    CK(cudaMemcpyAsync(b->h_ew + 7 * B, b->d_flags, sizeof(int) * B, cudaMemcpyDeviceToHost,
                       b->s0));
    if (b->persistent)
      CK(cudaMemcpyAsync(b->h_err, persist_error_word(b->px), sizeof(int),
                         cudaMemcpyDeviceToHost, b->s0));
  }
  if (energy && is_dev(energy))
    CK(cudaMemcpy2DAsync(energy, sizeof(double), b->d_ew, 7 * sizeof(double), sizeof(double), B,
                         cudaMemcpyDeviceToDevice, b->s0));
  if (virial && is_dev(virial))
    CK(cudaMemcpy2DAsync(virial, 6 * sizeof(double), b->d_ew + 1, 7 * sizeof(double),
                         6 * sizeof(double), B, cudaMemcpyDeviceToDevice, b->s0));
  CK(cudaEventRecord(b->ev_out, b->s0));
  CK(cudaStreamWaitEvent(b->stream, b->ev_out, 0));
  if (host) {
    CK(cudaStreamSynchronize(b->s0));
    for (size_t r = 0; r < B; ++r) {
      if (energy && !is_dev(energy)) energy[r] = b->h_ew[7 * r];
      if (virial && !is_dev(virial))
        for (int k = 0; k < 6; ++k) virial[6 * r + k] = b->h_ew[7 * r + 1 + k];
    }
    if (b->persistent && *b->h_err) return MLS6_ERR_TIMEOUT;
    const int* fl = reinterpret_cast<const int*>(b->h_ew + 7 * B);
    for (size_t r = 0; r < B; ++r)
      if (fl[r]) return flag_status(fl[r]);
  }
  return MLS6_OK;
}

// Whole-batch time (seconds, median of reps) of the current configuration.
static int time_batch(Batch* b, const void* pos, const void* c, void* forces, int reps,
                      double* sec) {
  int rc = launch(b, pos, c, forces, true);  // capture + warm-up
  if (rc) return rc;
  CK(cudaStreamSynchronize(b->s0));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::vector<float> t;
  for (int i = 0; i < reps && rc == MLS6_OK; ++i) {
    if (cudaEventRecord(e0, b->s0) != cudaSuccess) rc = MLS6_ERR_CUDA;
    if (!rc) rc = launch(b, pos, c, forces, true);
    if (!rc && cudaEventRecord(e1, b->s0) != cudaSuccess) rc = MLS6_ERR_CUDA;
    float ms = 0.f;
    if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = MLS6_ERR_CUDA;
    if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = MLS6_ERR_CUDA;
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  std::sort(t.begin(), t.end());
  *sec = 1e-3 * t[t.size() / 2];
  return MLS6_OK;
}

static int apply_shapes(Batch* b, const std::vector<int>& split, const std::vector<int>& groups) {
  for (int r = 0; r < b->B; ++r) {
    int rc = mls6_set_tuning(reinterpret_cast<mls6_plan_t*>(b->plans[r]), split[r], groups[r]);
    if (rc) return rc;
  }
  reset_graph(b);
  return MLS6_OK;
}

}  // namespace mls6

using namespace mls6;

extern "C" {

int mls6_cost_model(const double box[3], int64_t N, double a, double h, int levels,
                    const double* coef, double* cost) {
  if (!box || !cost || N < 0 || !(a > 0.0) || !(h > 0.0) || levels < 1 || levels > kMaxLevels)
    return MLS6_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (!(box[d] > 0.0)) return MLS6_ERR_BOX;
  *cost = model_cost(box, N, a, h, levels, coef);
  return MLS6_OK;
}

int mls6_lpt_assign(int B, const double* cost, int K, int* branch_of, double* load) {
  if (B < 0 || K < 1 || (B > 0 && (!cost || !branch_of))) return MLS6_ERR_ARG;
  lpt(B, cost, K, branch_of, load);
  return MLS6_OK;
}

int mls6_batch_plan(mls6_batch_t** out, int B, const double* boxes, const int64_t* N, double a,
                    double h, int levels, int order, int precision) {
  if (!out) return MLS6_ERR_ARG;
  *out = nullptr;
  if (B < 1 || !boxes || !N) return MLS6_ERR_ARG;
  Batch* b = new (std::nothrow) Batch();
  if (!b) return MLS6_ERR_NOMEM;
  b->B = B;
  b->prec = precision;
  b->plans.assign(B, nullptr);
  b->off.assign(B + 1, 0);
  b->cost.assign(B, 0.0);
  int rc = MLS6_OK;
  for (int r = 0; r < B && rc == MLS6_OK; ++r) {
    mls6_plan_t* p = nullptr;
    rc = mls6_plan(&p, boxes + 3 * r, N[r], a, h, levels, order, precision);
    if (rc) break;
    b->plans[r] = reinterpret_cast<Plan*>(p);
    // replicas keep the per-atom pair forms (the persistent kernel runs
    // those; the cluster form is for single large systems)
    b->plans[r]->pair_split = pair_split_atom(b->plans[r]);
    rc = plan_streams(b->plans[r]);
    b->off[r + 1] = b->off[r] + N[r];
    double hh = b->plans[r]->lv[1].h[0];
    b->cost[r] = model_cost(boxes + 3 * r, N[r], a, hh, b->plans[r]->levels, nullptr);
  }
  if (rc == MLS6_OK) {
    auto fail = [&](cudaError_t e) {
      if (e != cudaSuccess && rc == MLS6_OK) rc = MLS6_ERR_CUDA;
    };
    fail(cudaStreamCreateWithFlags(&b->s0, cudaStreamNonBlocking));
    fail(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    fail(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    fail(cudaEventCreateWithFlags(&b->ev_root, cudaEventDisableTiming));
    if (cudaMalloc((void**)&b->d_ew, 7 * sizeof(double) * B) != cudaSuccess ||
        cudaMalloc((void**)&b->d_flags, sizeof(int) * B) != cudaSuccess ||
        cudaMalloc((void**)&b->d_flag_src, sizeof(int*) * B) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_ew, (7 * sizeof(double) + sizeof(int)) * B) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_err, sizeof(int)) != cudaSuccess)
      rc = MLS6_ERR_NOMEM;
  }
  if (rc == MLS6_OK) {
    std::vector<const int*> src(B);
    for (int r = 0; r < B; ++r) src[r] = b->plans[r]->d_flag;
    if (cudaMemcpy(b->d_flag_src, src.data(), sizeof(int*) * B, cudaMemcpyHostToDevice) !=
        cudaSuccess)
      rc = MLS6_ERR_CUDA;
  }
  if (rc) {
    free_batch(b);
    return rc;
  }
  // seed: branches from the model (enough chains that the largest replica
  // bounds the makespan), shapes from each plan's own heuristics
  const double total = std::accumulate(b->cost.begin(), b->cost.end(), 0.0);
  const double big = *std::max_element(b->cost.begin(), b->cost.end());
  int K = (int)std::ceil(total / std::max(big, 1e-12));
  b->branches = std::max(1, std::min(std::min(K, 32), B));
  assign(b);
  *out = reinterpret_cast<mls6_batch_t*>(b);
  return MLS6_OK;
}

int mls6_batch_set_stream(mls6_batch_t* batch, void* stream) {
  if (!batch) return MLS6_ERR_ARG;
  reinterpret_cast<Batch*>(batch)->stream = (cudaStream_t)stream;
  return MLS6_OK;
}

int mls6_batch_eval(mls6_batch_t* batch, const void* pos, const void* c, void* forces,
                    double* energy, double* virial) {
  if (!batch) return MLS6_ERR_ARG;
  return eval(reinterpret_cast<Batch*>(batch), pos, c, forces, energy, virial);
}

int mls6_batch_set_config(mls6_batch_t* batch, int branches, const int* split,
                          const int* groups) {
  if (!batch) return MLS6_ERR_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (branches < 0) return MLS6_ERR_ARG;
  if (split || groups) {
    std::vector<int> s(b->B, 0), g(b->B, 0);
    for (int r = 0; r < b->B; ++r) {
      if (split) s[r] = split[r];
      if (groups) g[r] = groups[r];
    }
    int rc = apply_shapes(b, s, g);
    if (rc) return rc;
  }
  if (branches > 0) {
    b->branches = std::min(branches, b->B);
    assign(b);
  }
  reset_graph(b);
  return MLS6_OK;
}

int mls6_batch_info(const mls6_batch_t* batch, int* branches, int* split, int* groups,
                    int* branch_of, double* cost, int* levels, int* launches) {
  if (!batch) return MLS6_ERR_ARG;
  const Batch* b = reinterpret_cast<const Batch*>(batch);
  if (branches) *branches = b->branches;
  if (launches) *launches = b->launches;
  for (int r = 0; r < b->B; ++r) {
    if (split) split[r] = b->plans[r]->pair_split;
    if (groups) groups[r] = b->plans[r]->stencil_groups;
    if (branch_of) branch_of[r] = b->branch_of[r];
    if (cost) cost[r] = b->cost[r];
    if (levels) levels[r] = b->plans[r]->levels;
  }
  return MLS6_OK;
}

// Tune the batch's current launch form (branch count and kernel shapes of
// the chains, or the pair lanes of the persistent kernel); leaves the best
// configuration applied and its time in *best_out.
static int tune_form(Batch* b, const void* pos, const void* c, void* forces, int reps,
                     double* best_out) {
  // seed shapes: each plan's heuristic value
  std::vector<int> s0(b->B), g0(b->B);
  for (int r = 0; r < b->B; ++r) {
    s0[r] = pair_split_atom(b->plans[r]);
    g0[r] = b->plans[r]->stencil_groups;
  }
  auto shaped = [&](int sb, int gb, std::vector<int>& s, std::vector<int>& g) {
    s.resize(b->B);
    g.resize(b->B);
    for (int r = 0; r < b->B; ++r) {
      int x = sb >= 0 ? s0[r] << sb : s0[r] >> -sb;
      // the persistent kernel runs the per-atom pair kernel (1..8 lanes)
      const int smax = (b->mode == 1 || !pair_cluster_ok(b->plans[r])) ? 8 : kPairSplitMax;
      s[r] = std::max(1, std::min(smax, x));
      int y = gb >= 0 ? g0[r] << gb : g0[r] >> -gb;
      g[r] = std::max(1, std::min(4, y));
    }
  };
  std::vector<int> s, g;
  int best_sb = 0, best_gb = 0, best_k = b->branches;
  shaped(0, 0, s, g);
  int rc = apply_shapes(b, s, g);
  if (rc) return rc;
  double best = 0.0;
  rc = time_batch(b, pos, c, forces, reps, &best);
  if (rc) return rc;
  // the persistent kernel has no chains and fixed stencil groups: tune the
  // pair lanes only
  const bool pers = b->persistent;
  // 1. branch count
  const int Ks[] = {1, 2, 4, 8, 16, 32, 64};
  for (int K : Ks) {
    if (pers) break;
    if (K > b->B || K == best_k) continue;
    b->branches = K;
    assign(b);
    reset_graph(b);
    double t;
    rc = time_batch(b, pos, c, forces, reps, &t);
    if (rc) return rc;
    if (t < best) {
      best = t;
      best_k = K;
    }
  }
  b->branches = best_k;
  assign(b);
  // 2. pair lanes, 3. stencil groups: one power of two either way
  for (int pass = 0; pass < (pers ? 1 : 2); ++pass)
    for (int d : {-1, 1}) {
      const int sb = pass == 0 ? best_sb + d : best_sb, gb = pass == 1 ? best_gb + d : best_gb;
      shaped(sb, gb, s, g);
      rc = apply_shapes(b, s, g);
      if (rc) return rc;
      double t;
      rc = time_batch(b, pos, c, forces, reps, &t);
      if (rc) return rc;
      if (t < best) {
        best = t;
        best_sb = sb;
        best_gb = gb;
      }
    }
  shaped(best_sb, best_gb, s, g);
  rc = apply_shapes(b, s, g);
  if (rc) return rc;
  *best_out = best;
  return MLS6_OK;
}

int mls6_batch_tune(mls6_batch_t* batch, const void* pos, const void* c, void* forces, int reps,
                    double* best_sec) {
  if (!batch || reps < 1) return MLS6_ERR_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (b->off[b->B] > 0 && !arrays_ok(pos, c, forces)) return MLS6_ERR_ARG;
  double t0 = 0.0;
  int rc = tune_form(b, pos, c, forces, reps, &t0);
  if (rc) return rc;
  // FP32 batches whose plans the persistent kernel can run: tune the other
  // launch form too and keep the faster
  // (the persistent form is tuned with 1..8 lanes per atom, which it runs)
  bool other = b->prec == MLS6_FP32;
  for (const Plan* p : b->plans)
    other = other && p->N > 0 && p->levels >= 2 && !p->stencil_global && !p->stencil_mma &&
            !p->stencil_tc && p->sm.n == 2 && p->order == 3;
  if (other) {
    const int m0 = b->mode, k0 = b->branches;
    std::vector<int> s0(b->B), g0(b->B);
    for (int r = 0; r < b->B; ++r) {
      s0[r] = b->plans[r]->pair_split;
      g0[r] = b->plans[r]->stencil_groups;
    }
    b->mode = 1 - m0;
    reset_graph(b);
    double t1 = 0.0;
    rc = tune_form(b, pos, c, forces, reps, &t1);
    if (rc) return rc;
    if (t1 < t0) {
      t0 = t1;
    } else {  // back to the first form and its shapes
      b->mode = m0;
      b->branches = k0;
      assign(b);
      rc = apply_shapes(b, s0, g0);
      if (rc) return rc;
      reset_graph(b);
    }
  }
  if (best_sec) *best_sec = t0;
  return MLS6_OK;
}

int mls6_batch_size(const mls6_batch_t* batch, int* B, int64_t* offsets) {
  if (!batch) return MLS6_ERR_ARG;
  const Batch* b = reinterpret_cast<const Batch*>(batch);
  if (B) *B = b->B;
  if (offsets)
    for (int r = 0; r <= b->B; ++r) offsets[r] = b->off[r];
  return MLS6_OK;
}

int mls6_batch_replica(mls6_batch_t* batch, int r, mls6_plan_t** plan) {
  if (!batch || !plan) return MLS6_ERR_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (r < 0 || r >= b->B) return MLS6_ERR_ARG;
  *plan = reinterpret_cast<mls6_plan_t*>(b->plans[r]);
  return MLS6_OK;
}

int mls6_batch_set_mode(mls6_batch_t* batch, int persistent) {
  if (!batch || persistent < 0 || persistent > 1) return MLS6_ERR_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (b->s0 && cudaStreamSynchronize(b->s0) != cudaSuccess) return MLS6_ERR_CUDA;
  b->mode = persistent;
  reset_graph(b);
  return MLS6_OK;
}

int mls6_batch_mode(const mls6_batch_t* batch) {
  if (!batch) return MLS6_ERR_ARG;
  const Batch* b = reinterpret_cast<const Batch*>(batch);
  // the captured graph's form, or the form the next evaluation captures
  return (b->gexec ? b->persistent : persistent_ok(b)) ? 1 : 0;
}

int mls6_batch_set_wait(mls6_batch_t* batch, long long limit, long long withhold) {
  if (!batch || limit < 1) return MLS6_ERR_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (b->s0 && cudaStreamSynchronize(b->s0) != cudaSuccess) return MLS6_ERR_CUDA;
  b->wait_limit = limit;
  b->withhold = withhold;
  reset_graph(b);
  return MLS6_OK;
}

int mls6_batch_last_error(mls6_batch_t* batch) {
  if (!batch) return MLS6_ERR_ARG;
  Batch* b = reinterpret_cast<Batch*>(batch);
  if (b->s0 && cudaStreamSynchronize(b->s0) != cudaSuccess) return MLS6_ERR_CUDA;
  if (b->persistent) {
    int e = 0;
    if (cudaMemcpy(&e, persist_error_word(b->px), sizeof(int), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return MLS6_ERR_CUDA;
    if (e) return MLS6_ERR_TIMEOUT;
  }
  std::vector<int> fl(b->B, 0);
  if (cudaMemcpy(fl.data(), b->d_flags, sizeof(int) * b->B, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return MLS6_ERR_CUDA;
  for (int f : fl)
    if (f) return flag_status(f);
  return MLS6_OK;
}

void mls6_batch_destroy(mls6_batch_t* batch) { free_batch(reinterpret_cast<Batch*>(batch)); }

}  // extern "C"
