// Coarsest-level product without any device allocation.
//
// mls6_coarse_apply_noalloc computes, for a periodic coarsest grid of n
// nodes, e_mu = sum_nu T[(mu - nu) mod n] q_nu and the virial contribution
// 1/2 sum_mu q_mu sum_nu V_c[(mu - nu) mod n] q_nu.  It is the same
// operation as the coarsest-level step of mls6_eval, for callers that may
// not allocate device memory at call time: an MD engine that reserves its
// whole memory footprint up front, code running where cudaMalloc/cudaFree
// would synchronise the device or are not permitted, or a host framework
// whose allocator must not be bypassed.  The per-node virial partials it
// needs live in one file-scope device array of fixed size instead of
// plan-owned workspace.
#include "mls6_device.cuh"

namespace mls6 {

// Scratch: six doubles per coarsest node.  Every GPU that loads the library
// keeps this array (6 x 4096 x 8 bytes = 192 KiB) until the process exits.
constexpr int kNoAllocMaxNodes = 4096;
static __device__ __align__(256) double g_coarse_scratch[6 * kNoAllocMaxNodes];

// Device address of g_coarse_scratch in the current context (the symbol's
// host name is not a device address).  Looked up on every call rather than
// cached: after a device reset or a re-created primary context a cached
// address would point into a dead context.
static int scratch_for_current_device(double** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_coarse_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return MLS6_ERR_CUDA;
  }
  *out = static_cast<double*>(ptr);
  return MLS6_OK;
}

// One block per node mu; the per-node virial terms go to the scratch array.
template <bool VIR>
__global__ void __launch_bounds__(128) k_coarse_static(const double* __restrict__ q, int n0,
                                                       int n1, int n2,
                                                       const double* __restrict__ tT,
                                                       const double* __restrict__ tV,
                                                       double* __restrict__ e,
                                                       double* __restrict__ scratch) {
  __shared__ double red[32 * 7];
  const long np = (long)n0 * n1 * n2;
  const long mu = blockIdx.x;
  const int a = (int)(mu % n0), b = (int)((mu / n0) % n1), c = (int)(mu / ((long)n0 * n1));
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  for (long nu = threadIdx.x; nu < np; nu += blockDim.x) {
    int a2 = (int)(nu % n0), b2 = (int)((nu / n0) % n1), c2 = (int)(nu / ((long)n0 * n1));
    int da = a - a2, db = b - b2, dc = c - c2;
    if (da < 0) da += n0;
    if (db < 0) db += n1;
    if (dc < 0) dc += n2;
    const long m = da + (long)n0 * (db + (long)n1 * dc);
    const double qv = q[nu];
    v[0] += tT[m] * qv;
    if (VIR)
#pragma unroll
      for (int k = 0; k < 6; ++k) v[1 + k] += tV[k * np + m] * qv;
  }
  block_sum_n<7>(v, red);
  if (threadIdx.x == 0) {
    e[mu] = v[0];
    if (VIR)
      for (int k = 0; k < 6; ++k) scratch[6 * mu + k] = 0.5 * q[mu] * v[1 + k];
  }
}

// Fixed-order sum of the per-node partials into the six virial components.
__global__ void k_coarse_static_sum(const double* __restrict__ scratch, long np,
                                    double* __restrict__ virial) {
  __shared__ double red[32 * 6];
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (long k = threadIdx.x; k < np; k += blockDim.x)
#pragma unroll
    for (int c = 0; c < 6; ++c) v[c] += scratch[6 * k + c];
  block_sum_n<6>(v, red);
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; ++c) virial[c] = v[c];
}

}  // namespace mls6

using namespace mls6;

extern "C" int mls6_coarse_apply_noalloc(const double* q, const int n[3], const double* T,
                                         const double* V, double* e, double* virial,
                                         void* stream) {
  if (!n || !q || !T || !e || (virial && !V)) return MLS6_ERR_ARG;
  if (n[0] < 1 || n[1] < 1 || n[2] < 1) return MLS6_ERR_GRID;
  const long np = (long)n[0] * n[1] * n[2];
  if (np > kNoAllocMaxNodes) return MLS6_ERR_SIZE;
  if (!kernel_addressable(q) || !kernel_addressable(T) || !kernel_addressable(e) ||
      (virial && (!kernel_addressable(V) || !kernel_addressable(virial))))
    return MLS6_ERR_ARG;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (virial) {
    k_coarse_static<true><<<np, 128, 0, st>>>(q, n[0], n[1], n[2], T, V, e, scratch);
    k_coarse_static_sum<<<1, kBlock, 0, st>>>(scratch, np, virial);
  } else {
    k_coarse_static<false><<<np, 128, 0, st>>>(q, n[0], n[1], n[2], T, V, e, scratch);
  }
  if (cudaGetLastError() != cudaSuccess) return MLS6_ERR_CUDA;
  return MLS6_OK;
}
