// Layout conversion between user order ([ncomp][n_cells], x fastest, FP64) and the padded
// structure-of-arrays state, fills, and the FP64 energy reduction.
#include <cuda_runtime.h>

#include <algorithm>

#include "gks_internal.h"

namespace gks {
namespace {

template <typename T>
__global__ void user_to_cart_kernel(const double *__restrict__ user, T *__restrict__ dst, int nx,
                                    int ny, int nz, int64_t pitch, int64_t cstride, int ncomp) {
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t total = ncell * ncomp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / ncell, cell = i - c * ncell;
    const int64_t x = cell % nx, yz = cell / nx;
    const int64_t y = yz % ny, z = yz / ny;
    dst[c * cstride + (z * ny + y) * pitch + x] = T(user[i]);
  }
}

template <typename T>
__global__ void cart_to_user_kernel(const T *__restrict__ src, double *__restrict__ user, int nx,
                                    int ny, int nz, int64_t pitch, int64_t cstride, int ncomp) {
  const int64_t ncell = (int64_t)nx * ny * nz;
  const int64_t total = ncell * ncomp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / ncell, cell = i - c * ncell;
    const int64_t x = cell % nx, yz = cell / nx;
    const int64_t y = yz % ny, z = yz / ny;
    user[i] = double(src[c * cstride + (z * ny + y) * pitch + x]);
  }
}

// Copy of a box of columns [x0, x0+w) x rows [y0, y0+h) of every component (same offsets in
// src and dst).  Grid x runs over the columns of a row, grid y over the rows of all components
// (component-major), so a thread finds its row with one 32-bit division.
template <typename T>
__global__ void copy_box_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t cstride,
                                int64_t pitch, int x0, int w, int64_t y0, int h, int rows) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= w) return;
  for (int r = blockIdx.y; r < rows; r += gridDim.y) {
    const int c = r / h, y = r - c * h;
    const int64_t o = c * cstride + (y0 + y) * pitch + x0 + x;
    dst[o] = src[o];
  }
}

// dst (one component in the Cartesian layout) = box on columns [x0, x0+w) x rows [y0, y0+h);
// box row-major FP64.
template <typename T>
__global__ void box_to_cart_kernel(const double *__restrict__ box, T *__restrict__ dst, int x0,
                                   int w, int y0, int h, int64_t pitch) {
  const int64_t n = (int64_t)w * h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / w, x = i - y * w;
    dst[(y0 + y) * pitch + x0 + x] = T(box[i]);
  }
}

template <typename T>
__global__ void fill_kernel(T *dst, int64_t n, T v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = v;
}

// Per-block FP64 partial sums of (eps |E|^2 + mu |H|^2 + phi^2 + psi^2) over the cells (the
// potentials only with divergence cleaning), then one block sums the partials in a fixed order
// (deterministic), times |Omega| / 2.  Components [0, ne) are E, [ne, ne + nh) H, the rest the
// potentials.
template <typename T>
__global__ void energy_partial_kernel(const T *__restrict__ V, const T *__restrict__ eps,
                                      const T *__restrict__ mu, int nx, int ny, int nz,
                                      int64_t pitch, int64_t cstride, int ncomp, int ne, int nh,
                                      double *__restrict__ partials) {
  const int64_t ncell = (int64_t)nx * ny * nz;
  double acc = 0.0;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < ncell;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = cell % nx, yz = cell / nx;
    const int64_t y = yz % ny, z = yz / ny;
    const int64_t o = (z * ny + y) * pitch + x;
    double se = 0.0, sh = 0.0, sp = 0.0;
    for (int c = 0; c < ncomp; ++c) {
      const double v = double(V[c * cstride + o]);
      if (c < ne) se += v * v;
      else if (c < ne + nh) sh += v * v;
      else sp += v * v;
    }
    acc += double(eps[o]) * se + (mu ? double(mu[o]) : 1.0) * sh + sp;
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void sum_partials_kernel(const double *__restrict__ partials, int n, double scale,
                                    double *__restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_user_to_cart(const CartGeom &g, int ncomp, const double *user, void *dst,
                                bool fp64, cudaStream_t st) {
  const int64_t total = (int64_t)g.nx * g.ny * g.nz * ncomp;
  if (fp64)
    user_to_cart_kernel<double><<<grid_for(total), 256, 0, st>>>(
        user, static_cast<double *>(dst), g.nx, g.ny, g.nz, g.pitch, g.cstride, ncomp);
  else
    user_to_cart_kernel<float><<<grid_for(total), 256, 0, st>>>(
        user, static_cast<float *>(dst), g.nx, g.ny, g.nz, g.pitch, g.cstride, ncomp);
  return cudaGetLastError();
}

cudaError_t launch_cart_to_user(const CartGeom &g, int ncomp, const void *src, double *user,
                                bool fp64, cudaStream_t st) {
  const int64_t total = (int64_t)g.nx * g.ny * g.nz * ncomp;
  if (fp64)
    cart_to_user_kernel<double><<<grid_for(total), 256, 0, st>>>(
        static_cast<const double *>(src), user, g.nx, g.ny, g.nz, g.pitch, g.cstride, ncomp);
  else
    cart_to_user_kernel<float><<<grid_for(total), 256, 0, st>>>(
        static_cast<const float *>(src), user, g.nx, g.ny, g.nz, g.pitch, g.cstride, ncomp);
  return cudaGetLastError();
}

cudaError_t launch_copy_box(const void *src, void *dst, int ncomp, int64_t cstride, int64_t pitch,
                            int x0, int x1, int64_t y0, int64_t y1, bool fp64, cudaStream_t st) {
  const int w = x1 - x0, h = (int)(y1 - y0);
  if (w <= 0 || h <= 0 || ncomp <= 0) return cudaSuccess;
  const int rows = ncomp * h;
  const dim3 grid((w + 127) / 128, std::min(rows, 65535));
  if (fp64)
    copy_box_kernel<double><<<grid, 128, 0, st>>>(static_cast<const double *>(src),
                                                  static_cast<double *>(dst), cstride, pitch, x0,
                                                  w, y0, h, rows);
  else
    copy_box_kernel<float><<<grid, 128, 0, st>>>(static_cast<const float *>(src),
                                                 static_cast<float *>(dst), cstride, pitch, x0,
                                                 w, y0, h, rows);
  return cudaGetLastError();
}

cudaError_t launch_box_to_cart(const double *box, void *dst, int x0, int w, int y0, int h,
                               int64_t pitch, bool fp64, cudaStream_t st) {
  const int64_t n = (int64_t)w * h;
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  if (fp64)
    box_to_cart_kernel<double><<<blocks, 256, 0, st>>>(box, static_cast<double *>(dst), x0, w, y0,
                                                       h, pitch);
  else
    box_to_cart_kernel<float><<<blocks, 256, 0, st>>>(box, static_cast<float *>(dst), x0, w, y0,
                                                      h, pitch);
  return cudaGetLastError();
}

cudaError_t launch_fill(void *dst, int64_t n, double value, bool fp64, cudaStream_t st) {
  if (fp64)
    fill_kernel<double><<<grid_for(n), 256, 0, st>>>(static_cast<double *>(dst), n, value);
  else
    fill_kernel<float><<<grid_for(n), 256, 0, st>>>(static_cast<float *>(dst), n, (float)value);
  return cudaGetLastError();
}

template <typename T>
__global__ void halo_copy_kernel(const T *__restrict__ src, int64_t sstride, T *__restrict__ dst,
                                 int64_t dstride, int64_t count, int ncomp, bool add) {
  const int c = blockIdx.y;
  if (c >= ncomp) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T v = src[c * sstride + i];
    if (add) dst[c * dstride + i] += v;
    else dst[c * dstride + i] = v;
  }
}

cudaError_t launch_halo_copy(const void *src, int64_t sstride, void *dst, int64_t dstride,
                             int64_t count, int ncomp, bool add, bool fp64, cudaStream_t st) {
  if (count <= 0 || ncomp <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min<int64_t>((count + 255) / 256, 1024), (unsigned)ncomp);
  if (fp64)
    halo_copy_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double *>(src), sstride,
                                                   static_cast<double *>(dst), dstride, count,
                                                   ncomp, add);
  else
    halo_copy_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float *>(src), sstride,
                                                  static_cast<float *>(dst), dstride, count,
                                                  ncomp, add);
  return cudaGetLastError();
}

cudaError_t launch_cart_energy(const CartGeom &g, int ncomp, const void *V, const void *eps,
                               const void *mu, bool fp64, double *partials, int npart,
                               double *out, cudaStream_t st) {
  const int64_t ncell = (int64_t)g.nx * g.ny * g.nz;
  int blocks = grid_for(ncell);
  if (blocks > npart) blocks = npart;
  // E and H components: TM (Ez; Hx, Hy [; psi]) or 3-D (E; H [; phi, psi])
  const int ne = ncomp <= 4 ? 1 : 3, nh = ncomp <= 4 ? 2 : 3;
  double vol = 1.0;
  for (int a = 0; a < g.dim; ++a) vol *= g.h[a];
  if (fp64)
    energy_partial_kernel<double><<<blocks, 256, 0, st>>>(
        static_cast<const double *>(V), static_cast<const double *>(eps),
        static_cast<const double *>(mu), g.nx, g.ny, g.nz, g.pitch, g.cstride, ncomp, ne, nh,
        partials);
  else
    energy_partial_kernel<float><<<blocks, 256, 0, st>>>(
        static_cast<const float *>(V), static_cast<const float *>(eps),
        static_cast<const float *>(mu), g.nx, g.ny, g.nz, g.pitch, g.cstride, ncomp, ne, nh,
        partials);
  sum_partials_kernel<<<1, 256, 0, st>>>(partials, blocks, 0.5 * vol, out);
  return cudaGetLastError();
}

}  // namespace gks
