// GKS step on a tetrahedral mesh (Sec. 3.1): three deterministic passes per step.
//   1. tet_gradient_kernel: Green-Gauss cell gradients, face value = mean of the two cells
//      (a non-reflecting face uses the cell itself), written to a gradient scratch [18][nt].
//   2. tet_face_kernel: every face once -- reconstruct both sides at the face centroid, rotate
//      fields and gradients into the face frame T'(n), evaluate the GKS flux (shared closed
//      form, gks_flux3.cuh), rotate back, times the face area -> flux scratch [6][nf].
//   3. tet_update_kernel: every cell gathers the fluxes of its four faces (no atomics, fixed
//      order) and applies the FV update with the source.
// Geometry (frames, areas, offsets, face weights) is computed in FP64 on the host and stored on
// the device in the context's precision: an FP32 context reads it rounded to FP32 once, on the
// host (the FP64 volumes kept for the energy are the exception).
#include <cuda_runtime.h>

#include "gks_flux3.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

constexpr int TB = 256;

// Reciprocals: FP32 uses the fast hardware reciprocal (about 1 ulp), FP64 divides.
__device__ __forceinline__ float trcp(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double trcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float trcp2(float x) { return __fdividef(2.f, x); }
__device__ __forceinline__ double trcp2(double x) { return 2.0 / x; }

int blocks_for(int64_t n) {
  int64_t b = (n + TB - 1) / TB;
  return (int)(b < 1 ? 1 : b);
}

// The twelve gradient weights n|l|/|Omega| of a cell (its four faces): vector loads.
__device__ __forceinline__ void load_cell_w(const float *p, float w[kTetCellW]) {
#pragma unroll
  for (int k = 0; k < kTetCellW / 4; ++k) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + k);
    w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
  }
}
__device__ __forceinline__ void load_cell_w(const double *p, double w[kTetCellW]) {
#pragma unroll
  for (int k = 0; k < kTetCellW / 2; ++k) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + k);
    w[2 * k] = v.x; w[2 * k + 1] = v.y;
  }
}

template <typename T>
__global__ void tet_gradient_kernel(const T *__restrict__ V, const int32_t *__restrict__ cnb,
                                    const T *__restrict__ cw, int64_t nt, int pec,
                                    T *__restrict__ G) {
  const int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x;
  if (i >= nt) return;
  // every load is issued before the arithmetic: the four neighbour indices in one vector load,
  // then the 24 neighbour values (a wall face reads the cell itself), so that the gathers are in
  // flight together
  const int4 nb4 = __ldg(reinterpret_cast<const int4 *>(cnb) + i);
  const int32_t nb[4] = {nb4.x, nb4.y, nb4.z, nb4.w};
  T vi[6], vn[4][6], w[kTetCellW];
#pragma unroll
  for (int c = 0; c < 6; ++c) vi[c] = V[c * nt + i];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t j = nb[k] >= 0 ? (int64_t)nb[k] : i;
#pragma unroll
    for (int c = 0; c < 6; ++c) vn[k][c] = V[c * nt + j];
  }
  load_cell_w(cw + kTetCellW * i, w);
  T g[3][6];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 6; ++c) g[a][c] = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T vf[6];
    if (nb[k] >= 0) {
#pragma unroll
      for (int c = 0; c < 6; ++c) vf[c] = T(0.5) * (vi[c] + vn[k][c]);
    } else if (pec) {
      // PEC wall: face value (V + P V)/2 of the mirror ghost P V = (-E + 2 (E.n) n, H - 2 (H.n) n),
      // i.e. the normal part of E and the tangential part of H
      const T *wk = w + 3 * k;
      const T inv = T(1) / sqrt(wk[0] * wk[0] + wk[1] * wk[1] + wk[2] * wk[2]);
      const T n[3] = {wk[0] * inv, wk[1] * inv, wk[2] * inv};
      const T en = vi[0] * n[0] + vi[1] * n[1] + vi[2] * n[2];
      const T hn = vi[3] * n[0] + vi[4] * n[1] + vi[5] * n[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        vf[a] = en * n[a];
        vf[3 + a] = vi[3 + a] - hn * n[a];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) vf[c] = vi[c];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T wa = w[3 * k + a];
#pragma unroll
      for (int c = 0; c < 6; ++c) g[a][c] += vf[c] * wa;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 6; ++c) G[(6 * a + c) * nt + i] = g[a][c];
}

// The packed geometry of one face (10 values, 40 or 80 bytes): 8- or 16-byte vector loads.
__device__ __forceinline__ void load_face_geo(const float *p, float q[kTetFaceGeo]) {
#pragma unroll
  for (int k = 0; k < kTetFaceGeo / 2; ++k) {
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p) + k);
    q[2 * k] = v.x; q[2 * k + 1] = v.y;
  }
}
__device__ __forceinline__ void load_face_geo(const double *p, double q[kTetFaceGeo]) {
#pragma unroll
  for (int k = 0; k < kTetFaceGeo / 2; ++k) {
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + k);
    q[2 * k] = v.x; q[2 * k + 1] = v.y;
  }
}

// Side of a face in the frame with rows T (n, t, w): reconstruct V + G.d, then rotate the
// field index of both blocks and the derivative index.
template <typename T>
__device__ __forceinline__ Side3<T> tet_side(const T *__restrict__ V, const T *__restrict__ G,
                                             const T *__restrict__ eps, const T *__restrict__ mu,
                                             int64_t nt, int64_t cell, const T Tm[9],
                                             const T d[3]) {
  T v[6], g[3][6];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 6; ++c) g[a][c] = G[(6 * a + c) * nt + cell];
#pragma unroll
  for (int c = 0; c < 6; ++c)
    v[c] = V[c * nt + cell] + d[0] * g[0][c] + d[1] * g[1][c] + d[2] * g[2][c];
  Side3<T> s;
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T *r = Tm + 3 * k;                         // row k of T'
      s.v[3 * b + k] = r[0] * v[3 * b] + r[1] * v[3 * b + 1] + r[2] * v[3 * b + 2];
      // component k of the derivative along global axis a
      T ga[3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
        ga[a] = r[0] * g[a][3 * b] + r[1] * g[a][3 * b + 1] + r[2] * g[a][3 * b + 2];
      s.dn[3 * b + k] = Tm[0] * ga[0] + Tm[1] * ga[1] + Tm[2] * ga[2];
      s.dt[3 * b + k] = Tm[3] * ga[0] + Tm[4] * ga[1] + Tm[5] * ga[2];
      s.dw[3 * b + k] = Tm[6] * ga[0] + Tm[7] * ga[1] + Tm[8] * ga[2];
    }
  s.eps = eps[cell];
  s.mu = mu ? mu[cell] : T(1);
  return s;
}

// The mirror ghost of a side across a PEC wall, in the face frame (n, t, w): values
// (En, -Et, -Ew, -Hn, Ht, Hw); the normal derivative flips once more.
template <typename T>
__device__ __forceinline__ Side3<T> pec_ghost(const Side3<T> &l) {
  Side3<T> g;
  const T p[6] = {T(1), T(-1), T(-1), T(-1), T(1), T(1)};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    g.v[c] = p[c] * l.v[c];
    g.dn[c] = -p[c] * l.dn[c];
    g.dt[c] = p[c] * l.dt[c];
    g.dw[c] = p[c] * l.dw[c];
  }
  g.eps = l.eps;
  g.mu = l.mu;
  return g;
}

// FP32 with mu = 1: capped at 64 registers (no spills) for 4 CTAs per SM; the gathers' latency is
// hidden by more resident warps (3.7% faster than at 72 registers).
template <typename T, bool HAS_MU>
__global__ void __launch_bounds__(TB, (sizeof(T) == 4 && !HAS_MU) ? 4 : 1)
    tet_face_kernel(const T *__restrict__ V, const T *__restrict__ G,
                                const T *__restrict__ eps, const T *__restrict__ mu,
                                const int32_t *__restrict__ fL, const int32_t *__restrict__ fR,
                                const T *__restrict__ fgeo, int64_t nt, int64_t nf, int pec,
                                const K3<T> K, const F3K<T> FK, T *__restrict__ F) {
  const int64_t f = blockIdx.x * (int64_t)TB + threadIdx.x;
  if (f >= nf) return;
  T q[kTetFaceGeo];
  load_face_geo(fgeo + kTetFaceGeo * f, q);
  // frame rows (n, t, w) from n and 1/(1 + n_1)
  T Tm[9];
  {
    const T n1 = q[0], n2 = q[1], n3 = q[2], a = q[2] * q[3];
    Tm[0] = n1; Tm[1] = n2; Tm[2] = n3;
    Tm[3] = -n2; Tm[4] = n1 + n3 * a; Tm[5] = -n2 * a;
    Tm[6] = -n3; Tm[7] = -n2 * a; Tm[8] = T(1) - n3 * a;
  }
  const T *dl = q + 4, *dr = q + 7;
  const int32_t L = fL[f], R = fR[f];
  const Side3<T> l = tet_side<T>(V, G, eps, mu, nt, L, Tm, dl);
  T loc[6];
  if (R >= 0) {
    const Side3<T> r = tet_side<T>(V, G, eps, mu, nt, R, Tm, dr);
    if (HAS_MU)
      flux3<T, false>(l, r, K, loc);
    else
      flux3_mu1<T>(l, r, FK, trcp2(l.eps + r.eps), loc);
  } else if (pec) {
    const Side3<T> r = pec_ghost(l);
    if (HAS_MU)
      flux3<T, false>(l, r, K, loc);
    else
      flux3_mu1<T>(l, r, FK, trcp(l.eps), loc);
  } else {
    flux3<T, true>(l, l, K, loc);
  }
  // back to global components: Phi = T'^T Phi_local (|l_s| enters through the update weights)
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      F[(3 * b + a) * nf + f] =
          Tm[a] * loc[3 * b] + Tm[3 + a] * loc[3 * b + 1] + Tm[6 + a] * loc[3 * b + 2];
}

// The four update weights sign_k / |Omega| of a cell: one vector load (FP32) or two (FP64).
__device__ __forceinline__ void load_cell_u(const float *p, float w[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
__device__ __forceinline__ void load_cell_u(const double *p, double w[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}

template <typename T>
__global__ void tet_update_kernel(const T *__restrict__ V, T *__restrict__ Vout,
                                  const T *__restrict__ eps, const T *__restrict__ mu,
                                  const T *__restrict__ src, T src_amp,
                                  const int32_t *__restrict__ cface,
                                  const T *__restrict__ cu, const T *__restrict__ F, int64_t nt,
                                  int64_t nf,
                                  int *__restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)TB + threadIdx.x;
  bool bad = false;
  if (i < nt) {
    T w[4];
    load_cell_u(cu + kTetCellU * i, w);
    const int4 fc = __ldg(reinterpret_cast<const int4 *>(cface) + i);
    const int32_t fk[4] = {fc.x, fc.y, fc.z, fc.w};
    T d[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int c = 0; c < 6; ++c) d[c] -= w[k] * F[c * nf + fk[k]];
    if (src) d[2] -= src_amp * src[i];
    const T ie = trcp(eps[i]);
    const T im = mu ? trcp(mu[i]) : T(1);
    T sum = T(0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const T nv = V[c * nt + i] + d[c] * (c < 3 ? ie : im);
      Vout[c * nt + i] = nv;
      sum += nv;
    }
    bad = !isfinite(sum);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

template <typename T>
__global__ void user_to_tet_kernel(const double *__restrict__ user, T *__restrict__ dst,
                                   const int64_t *__restrict__ perm, int64_t nt, int ncomp) {
  const int64_t total = nt * ncomp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / nt, k = i - c * nt;
    dst[i] = T(user[c * nt + perm[k]]);
  }
}

template <typename T>
__global__ void tet_to_user_kernel(const T *__restrict__ src, double *__restrict__ user,
                                   const int64_t *__restrict__ perm, int64_t nt, int ncomp) {
  const int64_t total = nt * ncomp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / nt, k = i - c * nt;
    user[c * nt + perm[k]] = double(src[i]);
  }
}

template <typename T>
__global__ void tet_energy_partial_kernel(const T *__restrict__ V, const T *__restrict__ eps,
                                          const T *__restrict__ mu,
                                          const double *__restrict__ vol, int64_t nt,
                                          double *__restrict__ partials) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
       i += (int64_t)gridDim.x * blockDim.x) {
    double se = 0.0, sh = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double e = double(V[c * nt + i]), h = double(V[(3 + c) * nt + i]);
      se += e * e;
      sh += h * h;
    }
    acc += vol[i] * (double(eps[i]) * se + (mu ? double(mu[i]) : 1.0) * sh);
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

__global__ void tet_sum_partials_kernel(const double *__restrict__ partials, int n,
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
  if (threadIdx.x == 0) *out = 0.5 * red[0];
}

template <typename T>
cudaError_t step_t(const TetDev &g, const void *Vin, void *Vout, const void *eps, const void *mu,
                   const void *src, double src_amp, const double C[5], double c, int *flag,
                   cudaStream_t st) {
  const T *V = static_cast<const T *>(Vin);
  T *G = static_cast<T *>(g.Gscratch);
  T *F = static_cast<T *>(g.Fscratch);
  const T *fgeo = static_cast<const T *>(g.fgeo);
  const T *cw = static_cast<const T *>(g.cw), *cu = static_cast<const T *>(g.cu);
  tet_gradient_kernel<T><<<blocks_for(g.nt), TB, 0, st>>>(V, g.cnb, cw, g.nt, g.pec, G);
  const K3<T> K = make_k3<T>(C, 1.0, c);     // fluxes carry dt (C_i), areas applied per face
  const F3K<T> FK = make_f3k<T>(C, 1.0, c);
  if (mu)
    tet_face_kernel<T, true><<<blocks_for(g.nf), TB, 0, st>>>(
        V, G, static_cast<const T *>(eps), static_cast<const T *>(mu), g.fL, g.fR, fgeo, g.nt,
        g.nf, g.pec, K, FK, F);
  else
    tet_face_kernel<T, false><<<blocks_for(g.nf), TB, 0, st>>>(
        V, G, static_cast<const T *>(eps), nullptr, g.fL, g.fR, fgeo, g.nt, g.nf, g.pec, K, FK, F);
  tet_update_kernel<T><<<blocks_for(g.nt), TB, 0, st>>>(
      V, static_cast<T *>(Vout), static_cast<const T *>(eps), static_cast<const T *>(mu),
      static_cast<const T *>(src), T(src_amp), g.cface, cu, F, g.nt, g.nf, flag);
  return cudaGetLastError();
}

int grid_capped(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_tet_step(const TetDev &g, const void *V, void *Vout, const void *eps,
                            const void *mu, const void *src, double src_amp, const double C[5],
                            double c, int *flag, bool fp64, cudaStream_t st) {
  return fp64 ? step_t<double>(g, V, Vout, eps, mu, src, src_amp, C, c, flag, st)
              : step_t<float>(g, V, Vout, eps, mu, src, src_amp, C, c, flag, st);
}

cudaError_t launch_user_to_tet(const TetDev &g, int ncomp, const double *user, void *dst,
                               bool fp64, cudaStream_t st) {
  if (fp64)
    user_to_tet_kernel<double><<<grid_capped(g.nt * ncomp), 256, 0, st>>>(
        user, static_cast<double *>(dst), g.perm, g.nt, ncomp);
  else
    user_to_tet_kernel<float><<<grid_capped(g.nt * ncomp), 256, 0, st>>>(
        user, static_cast<float *>(dst), g.perm, g.nt, ncomp);
  return cudaGetLastError();
}

cudaError_t launch_tet_to_user(const TetDev &g, int ncomp, const void *src, double *user,
                               bool fp64, cudaStream_t st) {
  if (fp64)
    tet_to_user_kernel<double><<<grid_capped(g.nt * ncomp), 256, 0, st>>>(
        static_cast<const double *>(src), user, g.perm, g.nt, ncomp);
  else
    tet_to_user_kernel<float><<<grid_capped(g.nt * ncomp), 256, 0, st>>>(
        static_cast<const float *>(src), user, g.perm, g.nt, ncomp);
  return cudaGetLastError();
}

cudaError_t launch_tet_energy(const TetDev &g, const void *V, const void *eps, const void *mu,
                              bool fp64, double *partials, int npart, double *out,
                              cudaStream_t st) {
  int blocks = grid_capped(g.nt);
  if (blocks > npart) blocks = npart;
  if (fp64)
    tet_energy_partial_kernel<double><<<blocks, 256, 0, st>>>(
        static_cast<const double *>(V), static_cast<const double *>(eps),
        static_cast<const double *>(mu), g.vol, g.nt, partials);
  else
    tet_energy_partial_kernel<float><<<blocks, 256, 0, st>>>(
        static_cast<const float *>(V), static_cast<const float *>(eps),
        static_cast<const float *>(mu), g.vol, g.nt, partials);
  tet_sum_partials_kernel<<<1, 256, 0, st>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace gks
