// Energy reduction that allocates nothing: gks_energy_noalloc (declared in include/gks.h).
//
// Some callers cannot call cudaMalloc: a framework that has reserved the device memory up
// front for its own pool, a hot loop that cannot afford the latency or the implicit
// synchronisation of an allocation, or a caller that holds no gks context at all.  This entry
// point computes the same energy as gks_energy from device arrays the caller already owns, and
// keeps its only scratch -- the per-block partial sums -- in the fixed array below, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include "gks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int64_t kCellsPerBlock = (int64_t)kThreads * kCellsPerThread;   // 4096
constexpr int kMaxBlocks = 8192;                                          // 64 KiB of partials
constexpr int64_t kMaxCells = kCellsPerBlock * kMaxBlocks;                // 33,554,432

// One FP64 partial sum per block; blocks cover fixed 4096-cell chunks, so the result does not
// depend on the launch and the final sum runs in a fixed order.
static __device__ __align__(256) double g_energy_partials[kMaxBlocks];

template <typename T>
__global__ void energy_chunks_kernel(const T *__restrict__ f, const T *__restrict__ eps,
                                     const T *__restrict__ mu, int64_t n, int ncomp, int ne,
                                     double *__restrict__ partials) {
  const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock;
  double acc = 0.0;
  for (int k = 0; k < kCellsPerThread; ++k) {
    const int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
    if (i >= n) break;
    double se = 0.0, sh = 0.0;
    for (int c = 0; c < ncomp; ++c) {
      const double v = double(f[(int64_t)c * n + i]);
      if (c < ne) se += v * v; else sh += v * v;
    }
    acc += double(eps[i]) * se + (mu ? double(mu[i]) : 1.0) * sh;
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void energy_finish_kernel(const double *__restrict__ partials, int nblocks,
                                     double scale, double *__restrict__ out) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kThreads) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// Device address of g_energy_partials on the current device.  In host code the array's name
// only stands for it; only this address may go to a kernel.  It is looked up on every call, so a
// device reset (after which the module, and the array with it, is loaded again at a new address)
// cannot leave a stale pointer behind.
gks_status partials_for_current_device(double **out) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_energy_partials) != cudaSuccess || !p) return GKS_E_CUDA;
  *out = static_cast<double *>(p);
  return GKS_OK;
}

}  // namespace

extern "C" gks_status gks_energy_noalloc(int32_t precision, int32_t dim, int64_t n_cells,
                                         double cell_volume, const void *fields, const void *eps,
                                         const void *mu, double *out, void *cuda_stream) {
  if (precision != GKS_FP32 && precision != GKS_FP64) return GKS_E_ARG;
  if (dim != 2 && dim != 3) return GKS_E_ARG;
  if (!fields || !eps || !out) return GKS_E_ARG;
  if (n_cells <= 0 || n_cells > kMaxCells) return GKS_E_ARG;   // beyond the scratch capacity
  if (!(cell_volume > 0.0)) return GKS_E_ARG;
  // An error that earlier work left pending on this thread belongs to that work: leave it in
  // place for its owner and launch nothing (launch errors of this call would be hidden by it).
  if (cudaPeekAtLastError() != cudaSuccess) return GKS_E_CUDA;
  double *partials = nullptr;
  gks_status s = partials_for_current_device(&partials);
  if (s != GKS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int ncomp = dim == 2 ? 3 : 6, ne = dim == 2 ? 1 : 3;
  const int blocks = (int)((n_cells + kCellsPerBlock - 1) / kCellsPerBlock);
  if (precision == GKS_FP64)
    energy_chunks_kernel<double><<<blocks, kThreads, 0, st>>>(
        static_cast<const double *>(fields), static_cast<const double *>(eps),
        static_cast<const double *>(mu), n_cells, ncomp, ne, partials);
  else
    energy_chunks_kernel<float><<<blocks, kThreads, 0, st>>>(
        static_cast<const float *>(fields), static_cast<const float *>(eps),
        static_cast<const float *>(mu), n_cells, ncomp, ne, partials);
  energy_finish_kernel<<<1, kThreads, 0, st>>>(partials, blocks, 0.5 * cell_volume, out);
  // no error was pending before the launches, so one pending now is theirs: report and clear it
  return cudaGetLastError() == cudaSuccess ? GKS_OK : GKS_E_CUDA;
}
