// Local step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that must run under a hard
// device-memory budget fixed up front, or hosts whose memory is handed out by an
// allocator the library cannot reach.  pd_local_step_noalloc serves them: the
// caller passes every input and output array, and the only scratch the
// computation needs (the per-cell corner forces, the block partial sums of the
// energy and a status word) lives in one file-scope device array of fixed size.
// That array exists on every GPU that loads this library, for the life of the
// process.  The status word (det F <= 0 seen, a non-finite gradient entry) is
// copied to the caller's status_flags, when given, at the end of the call.
//
// Limits and rules of use:
//   * at most kMaxCells cells (and at most 8 kMaxCells nodes) per call;
//   * the first call on a device looks up the array's device address there (with
//     that device current); make that first call before any stream capture;
//   * every call shares the array, so calls whose kernels overlap on the GPU
//     (different streams, or concurrent host threads) race; calls on one stream
//     are ordered and safe;
//   * the array keeps the contents of the last call; this call clears what it
//     needs zeroed (the status word) itself.
#include <mutex>
#include <string>

#include "pd_internal.cuh"

namespace pd {

namespace {

constexpr int64_t kMaxCells = PD_NOALLOC_MAX_CELLS;
constexpr int kT = 256;
// one energy partial per block of the element kernel (its block size is shared
// through pd_internal.cuh, so the layout follows it)
constexpr int64_t kMaxElemBlocks = raw_element_blocks(kMaxCells);
constexpr int64_t kMaxNodeBlocks = (kMaxCells * 8 + kT - 1) / kT;
static_assert(kMaxElemBlocks * kElemBlockThreads >= 8 * kMaxCells, "element partials do not cover the cells");
static_assert(PD_LOCAL_FLAG_INVERTED == DEV_ERR_INVERTED && PD_LOCAL_FLAG_NAN == DEV_ERR_NAN,
              "status bits of the header and of the kernels differ");
// layout (in doubles): corner forces (FP64 worst case) | element block partials |
// node block partials | energy accumulator | status word
constexpr int64_t kForcesOff = 0;
constexpr int64_t kElemPartOff = kForcesOff + 24 * kMaxCells;
constexpr int64_t kNodePartOff = kElemPartOff + kMaxElemBlocks;
constexpr int64_t kStatusOff = kNodePartOff + kMaxNodeBlocks;
constexpr int64_t kScratchDoubles = kStatusOff + 2;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_addr_mu;
void* g_addr[256] = {};   // device address of the scratch array, per device ordinal

// grad E over the caller's nodes from the corner forces, plus the contact force
// and per-block contact energy (fixed-order sums)
template <typename T>
__global__ void __launch_bounds__(kT) noalloc_gather_kernel(int64_t n, const int32_t* inc_ptr, const int32_t* inc,
                                                           const T* forces, const double* x, const uint8_t* contact,
                                                           double k, double* grad, double* partials, int* status) {
  const int64_t c = (int64_t)blockIdx.x * kT + threadIdx.x;
  double en = 0;
  if (c < n) {
    double g0 = 0, g1 = 0, g2 = 0;
    for (int32_t q = inc_ptr[c]; q < inc_ptr[c + 1]; ++q) {
      const int64_t slot = (int64_t)inc[q] * 3;
      g0 += (double)forces[slot];
      g1 += (double)forces[slot + 1];
      g2 += (double)forces[slot + 2];
    }
    if (contact && contact[c]) {
      const double z = x[3 * c + 2];
      if (z < 0.0) {
        g2 += k * z;
        en = 0.5 * k * z * z;
      }
    }
    grad[3 * c] = g0;
    grad[3 * c + 1] = g1;
    grad[3 * c + 2] = g2;
    if (!isfinite(g0) || !isfinite(g1) || !isfinite(g2)) atomicOr(status, DEV_ERR_NAN);
  }
  __shared__ double sh[kT / 32];
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) en += __shfl_xor_sync(0xffffffffu, en, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = en;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < kT / 32; ++w) t += sh[w];
    partials[blockIdx.x] = t;
  }
}

// energy = sum of the element block partials + sum of the node block partials
__global__ void __launch_bounds__(kT) noalloc_energy_kernel(const double* ep, int64_t ne_blk, const double* np,
                                                           int64_t nn_blk, double* energy) {
  double a = 0;
  for (int64_t i = threadIdx.x; i < ne_blk; i += kT) a += ep[i];
  for (int64_t i = threadIdx.x; i < nn_blk; i += kT) a += np[i];
  __shared__ double sh[kT];
  sh[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < kT; ++i) t += sh[i];
    *energy = t;
  }
}

pd_status scratch_address(double** out) {
  int dev = -1;
  PD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) {
    set_error("pd_local_step_noalloc: unsupported device ordinal");
    return PD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    // the symbol's host-side name is not a device address: look it up on this device
    PD_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = p;
  }
  *out = static_cast<double*>(g_addr[dev]);
  return PD_OK;
}

}  // namespace

}  // namespace pd

extern "C" pd_status pd_local_step_noalloc(int64_t n_nodes, int64_t n_elems, const int32_t* elems,
                                           const int32_t* inc_ptr, const int32_t* inc, double dx,
                                           const double* x, const double* act, const double* w_corot,
                                           const double* w_vol, const double* w_muscle, const double* fiber,
                                           const uint8_t* contact, double k_contact, int32_t precision,
                                           double* grad_E, double* energy, int32_t* status_flags,
                                           void* stream) {
  using namespace pd;
  if (n_elems <= 0 || n_nodes <= 0) {
    set_error("pd_local_step_noalloc: empty mesh");
    return PD_ERR_INVALID_ARG;
  }
  if (n_elems > kMaxCells || n_nodes > 8 * kMaxCells) {
    set_error("pd_local_step_noalloc: mesh larger than the fixed scratch (" + std::to_string(kMaxCells) +
              " cells, " + std::to_string(8 * kMaxCells) + " nodes)");
    return PD_ERR_INVALID_ARG;
  }
  if (!elems || !inc_ptr || !inc || !x || !grad_E || !(dx > 0)) {
    set_error("pd_local_step_noalloc: elems, inc_ptr, inc, x, grad_E and dx > 0 are required");
    return PD_ERR_INVALID_ARG;
  }
  if (!w_corot && !w_vol && !w_muscle) {
    set_error("pd_local_step_noalloc: at least one energy weight array is required");
    return PD_ERR_INVALID_ARG;
  }
  if (w_muscle && !fiber) {
    set_error("pd_local_step_noalloc: fiber directions are required with w_muscle");
    return PD_ERR_INVALID_ARG;
  }
  if (precision != PD_PREC_FP64 && precision != PD_PREC_MIXED) {
    set_error("pd_local_step_noalloc: unknown precision");
    return PD_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  pd_status st = scratch_address(&scratch);
  if (st != PD_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  int* status = reinterpret_cast<int*>(scratch + kStatusOff);
  PD_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
  PD_CUDA_TRY(launch_element_forces_raw(n_elems, elems, x, act, w_corot, w_vol, w_muscle, fiber, dx, precision,
                                        scratch + kForcesOff, scratch + kElemPartOff, status, s));
  const int64_t ne_blk = raw_element_blocks(n_elems);
  const int64_t nn_blk = (n_nodes + kT - 1) / kT;
  if (precision == PD_PREC_MIXED)
    noalloc_gather_kernel<float><<<(unsigned)nn_blk, kT, 0, s>>>(
        n_nodes, inc_ptr, inc, reinterpret_cast<const float*>(scratch + kForcesOff), x,
        k_contact > 0 ? contact : nullptr, k_contact, grad_E, scratch + kNodePartOff, status);
  else
    noalloc_gather_kernel<double><<<(unsigned)nn_blk, kT, 0, s>>>(
        n_nodes, inc_ptr, inc, scratch + kForcesOff, x, k_contact > 0 ? contact : nullptr, k_contact, grad_E,
        scratch + kNodePartOff, status);
  PD_CUDA_TRY(cudaGetLastError());
  if (energy) {
    noalloc_energy_kernel<<<1, kT, 0, s>>>(scratch + kElemPartOff, ne_blk, scratch + kNodePartOff, nn_blk, energy);
    PD_CUDA_TRY(cudaGetLastError());
  }
  // the status word leaves the shared scratch in stream order (a device-to-device
  // copy of 4 bytes allocates nothing)
  if (status_flags) PD_CUDA_TRY(cudaMemcpyAsync(status_flags, status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  return PD_OK;
}
