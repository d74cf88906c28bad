// Fused 3-D GKS step on a Cartesian grid (fields E, H): cell gradients, face reconstruction,
// the GKS interface flux and the finite-volume update in one pass (Sec. 3.1).
//
// 2.5-D march.  A CTA of BX x BY threads owns the columns x0-1 .. x0+BX-2, y0-1 .. y0+BY-2 of a
// chunk of z-planes (thread (tx, ty) -> x = x0-1+tx, y = y0-1+ty) and updates the inner
// (BX-2) x (BY-2) columns; the outer ring of threads supplies the gradients and faces the inner
// cells need.  Planes are staged in shared memory (x/y neighbours); per plane a thread forms
// the central differences of plane z+1, the x-face x+1/2, the y-face y+1/2 and the z-face z+1/2
// of its cell, publishes them, and after one barrier completes the update of plane z.
//
// Face frames (Sec. 3.1, T'(n)): interior faces use n = +e_x (frame (x, y, z)), n = +e_y
// (frame (y, -x, z)) and n = +e_z (frame (z, y, -x)); boundary faces on the low sides use the
// outward normals -e_x (frame (-x, -y, z)), -e_y (frame (-y, x, z)) and -e_z (frame (-z, y, x)).
// Every frame is a signed permutation of the axes, so rotations cost nothing.  A PEC wall
// (Sec. 5.5) is an interior face against mirror-image cells (index reflected across the wall,
// tangential E and normal H negated).
//
// NC = 6 carries (E, H); NC = 8 the divergence-cleaning system (E, H, phi, psi) of Sec. 2.1,
// whose potentials are scalars in every frame (phi odd and psi even across a PEC wall).
// LIMIT replaces the central differences of the cell gradients by van Leer-limited slopes (the
// discontinuity capturing of Sec. 5.3).
#include <cuda_runtime.h>

#include <type_traits>

#include "gks_flux3.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

constexpr int BX = 32;
constexpr int PX = BX + 2;            // staged plane: one extra ring around the thread grid
// Tile height: FP32 takes 32 x 16 threads (inner 30 x 14 cells, about 200 KB of shared memory,
// one CTA per SM); FP64 32 x 8 (its planes are twice as large).  The eight-component cleaning
// system stages a third more per cell: 32 x 12 (FP32: 199 KB, 168 registers, 12 warps per SM)
// and 32 x 6 (FP64).
template <typename T, int NC>
struct Geo3 {
  static constexpr int BY = NC == 6 ? (sizeof(T) == 4 ? 16 : 8) : (sizeof(T) == 4 ? 12 : 6);
  static constexpr int NTH = BX * BY;
  static constexpr int PY = BY + 2;
  static constexpr int NV = NC + 2;   // staged quantities: the NC fields, eps, mu
};
constexpr int NSLOT = 4;              // staged planes z-1 .. z+2

// Signed-axis face frame: local axis k is sign S_k times global axis A_k.
template <int AN, int SN, int AT, int ST, int AW, int SW>
struct Frame {
  static constexpr int an = AN, sn = SN, at = AT, st = ST, aw = AW, sw = SW;
};
using FrameXp = Frame<0, 1, 1, 1, 2, 1>;
using FrameYp = Frame<1, 1, 0, -1, 2, 1>;
using FrameZp = Frame<2, 1, 1, 1, 0, -1>;
using FrameXm = Frame<0, -1, 1, -1, 2, 1>;
using FrameYm = Frame<1, -1, 0, 1, 2, 1>;
using FrameZm = Frame<2, -1, 1, 1, 0, 1>;

// Global data of one cell: V (Ex..Hz [, phi, psi]), gradients G[axis][comp] (true
// derivatives), materials.
template <typename T, int NC>
struct Cell3 {
  T v[NC];
  T g[3][NC];
  T eps, mu;
};

template <typename T, int NC>
using SideT = typename std::conditional<NC == 6, Side3<T>, Side8<T>>::type;

// Local side of a cell, reconstructed by `shift` along the face's global normal axis
// (V + shift * d/d(axis) V; shift = +-h/2).
template <typename T, typename F, int NC>
__device__ __forceinline__ SideT<T, NC> to_local(const Cell3<T, NC> &c, T shift) {
  SideT<T, NC> s;
  const int ax[3] = {F::an, F::at, F::aw};
  const T sg[3] = {T(F::sn), T(F::st), T(F::sw)};
#pragma unroll
  for (int b = 0; b < 2; ++b) {           // E block, H block
#pragma unroll
    for (int k = 0; k < 3; ++k) {          // local component n, t, w
      const int gc = 3 * b + ax[k];
      const T sgc = sg[k];
      s.v[3 * b + k] = sgc * (c.v[gc] + shift * c.g[F::an][gc]);
      s.dn[3 * b + k] = sgc * T(F::sn) * c.g[F::an][gc];
      s.dt[3 * b + k] = sgc * T(F::st) * c.g[F::at][gc];
      s.dw[3 * b + k] = sgc * T(F::sw) * c.g[F::aw][gc];
    }
  }
#pragma unroll
  for (int k = 6; k < NC; ++k) {          // potentials: scalars
    s.v[k] = c.v[k] + shift * c.g[F::an][k];
    s.dn[k] = T(F::sn) * c.g[F::an][k];
    s.dt[k] = T(F::st) * c.g[F::at][k];
    s.dw[k] = T(F::sw) * c.g[F::aw][k];
  }
  s.eps = c.eps;
  s.mu = c.mu;
  return s;
}

// Back to global components: Phi_global = T'^T Phi_local.
template <typename T, typename F, int NC>
__device__ __forceinline__ void to_global(const T loc[NC], T glob[NC]) {
  const int ax[3] = {F::an, F::at, F::aw};
  const T sg[3] = {T(F::sn), T(F::st), T(F::sw)};
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int k = 0; k < 3; ++k) glob[3 * b + ax[k]] = sg[k] * loc[3 * b + k];
#pragma unroll
  for (int k = 6; k < NC; ++k) glob[k] = loc[k];
}

// Reciprocals: FP32 uses the fast hardware reciprocal (about 1 ulp), FP64 divides.
__device__ __forceinline__ float rcp3(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp3(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp3x2(float x) { return __fdividef(2.f, x); }
__device__ __forceinline__ double rcp3x2(double x) { return 2.0 / x; }

// Face flux in the face frame: the Maxwell closed forms (NC = 6) or the cleaning system's.
template <typename T, bool GHOST>
__device__ __forceinline__ void face_flux(const Side3<T> &l, const Side3<T> &r, const K3<T> &K, T,
                                          T, T out[6]) {
  flux3<T, GHOST>(l, r, K, out);
}
template <typename T, bool GHOST>
__device__ __forceinline__ void face_flux(const Side8<T> &l, const Side8<T> &r, const K3<T> &K,
                                          T chi, T gam, T out[8]) {
  flux3_phm<T, GHOST, true>(l, r, K, chi, gam, out);   // the cleaning system runs with mu = 1
}

// Interior face of frame F between cells L (low side) and R (high side), along +axis.  Maxwell
// without mu uses the sums-and-differences form flux3_mu1.
template <typename T, typename F, bool HAS_MU, int NC>
__device__ __forceinline__ void interior_face(const Cell3<T, NC> &L, const Cell3<T, NC> &R,
                                              T halfh, const K3<T> &K, const F3K<T> &FK,
                                              const F8K<T> &K8, T phi[NC]) {
  T loc[NC];
  if constexpr (NC == 6) {
    if (HAS_MU)
      flux3<T, false>(to_local<T, F>(L, halfh), to_local<T, F>(R, -halfh), K, loc);
    else
      flux3_mu1<T>(to_local<T, F>(L, halfh), to_local<T, F>(R, -halfh), FK,
                   rcp3x2(L.eps + R.eps), loc);
  } else {
    flux3_phm_mu1<T>(to_local<T, F>(L, halfh), to_local<T, F>(R, -halfh), K8, rcp3x2(L.eps + R.eps),
                     loc);
  }
  to_global<T, F, NC>(loc, phi);
}

// High-side boundary face (outward +axis, l = the cell): flux along +axis.
template <typename T, typename F, int NC>
__device__ __forceinline__ void high_boundary_face(const Cell3<T, NC> &L, T halfh, const K3<T> &K,
                                                   T chi, T gam, T phi[NC]) {
  T loc[NC];
  const SideT<T, NC> s = to_local<T, F>(L, halfh);
  face_flux<T, true>(s, s, K, chi, gam, loc);
  to_global<T, F, NC>(loc, phi);
}

// Low-side boundary face (outward -axis, l = the cell): returns the flux along +axis, i.e.
// minus F.n_out.
template <typename T, typename F, int NC>
__device__ __forceinline__ void low_boundary_face(const Cell3<T, NC> &R, T halfh, const K3<T> &K,
                                                  T chi, T gam, T phi[NC]) {
  T loc[NC], g[NC];
  const SideT<T, NC> s = to_local<T, F>(R, -halfh);
  face_flux<T, true>(s, s, K, chi, gam, loc);
  to_global<T, F, NC>(loc, g);
#pragma unroll
  for (int c = 0; c < NC; ++c) phi[c] = -g[c];
}

template <typename T>
struct Cart3DArgs {
  const T *__restrict__ V;
  T *__restrict__ Vout;
  const T *__restrict__ eps;
  const T *__restrict__ mu;
  const T *__restrict__ src;
  int sx0, sx1, sy0, sy1, sz0, sz1;
  T src_amp;
  int nx, ny, nz;
  int64_t pitch, plane, cstride;
  int per[3];
  int pec[6];          // PEC wall on the -x, +x, -y, +y, -z, +z side
  T inv2h[3], halfh[3];
  K3<T> K[3];
  F3K<T> FK[3];
  F8K<T> K8[3];        // folded cleaning-flux constants (NC = 8)
  T chi, gam;          // cleaning speeds (NC = 8)
  int zchunk;
  int *flag;
};

// Cell of index i on an axis of n cells: periodic wrap, PEC mirror (m = true: the entry is the
// mirror image -1-i or 2n-1-i, clamped beyond the stencil) or the non-reflecting clamp.
__device__ __forceinline__ int axis_index3(int i, int n, int periodic, int pec_lo, int pec_hi,
                                           bool &m) {
  m = false;
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  if (i < 0) {
    if (!pec_lo) return 0;
    m = true;
    i = -1 - i;
    return i < n ? i : n - 1;
  }
  if (i >= n) {
    if (!pec_hi) return n - 1;
    m = true;
    i = 2 * n - 1 - i;
    return i >= 0 ? i : 0;
  }
  return i;
}

template <typename T, int NC>
struct Smem3 {
  using G_ = Geo3<T, NC>;
  T V[NSLOT][G_::NV][G_::PY][PX];    // staged planes with one extra ring
  T G[2][3 * NC][G_::BY][BX];        // gradients (axis-major: x comps, y comps, z comps)
  T F[2][2 * NC][G_::BY][BX];        // x-face (0..NC-1) and y-face (NC..) fluxes at the high side
};

// Load one staged entry (x, y, z) of all quantities into registers.
template <typename T, int NC, bool HAS_MU, bool HAS_PEC>
__device__ __forceinline__ void load_entry(const Cart3DArgs<T> &p, int x, int y, int z,
                                           T out[NC + 2]) {
  bool m[3];
  const int xx = axis_index3(x, p.nx, p.per[0], HAS_PEC && p.pec[0], HAS_PEC && p.pec[1], m[0]);
  const int yy = axis_index3(y, p.ny, p.per[1], HAS_PEC && p.pec[2], HAS_PEC && p.pec[3], m[1]);
  const int zz = axis_index3(z, p.nz, p.per[2], HAS_PEC && p.pec[4], HAS_PEC && p.pec[5], m[2]);
  const int64_t o = (int64_t)zz * p.plane + (int64_t)yy * p.pitch + xx;
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c] = __ldg(p.V + c * p.cstride + o);
  // PEC mirror image across the walls of axes a with m[a]: E_c keeps its sign if c == a (normal
  // E) and flips otherwise; H_c flips if c == a (normal H) and keeps it otherwise
  if (HAS_PEC && (m[0] | m[1] | m[2])) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (m[a])
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          if (c == a) out[3 + c] = -out[3 + c];
          else out[c] = -out[c];
        }
    if (NC == 8 && (m[0] ^ m[1] ^ m[2])) out[6] = -out[6];   // phi odd per wall, psi even
  }
  out[NC] = __ldg(p.eps + o);
  out[NC + 1] = HAS_MU ? __ldg(p.mu + o) : T(1);
}

template <typename T, int NC>
__device__ __forceinline__ void stage(Smem3<T, NC> &s, int slot, int py, int px,
                                      const T v[NC + 2]) {
#pragma unroll
  for (int c = 0; c < NC + 2; ++c) s.V[slot][c][py][px] = v[c];
}

// Slope of one component along an axis from the values below (vm), at (v0) and above (vp) the
// cell: the central difference, or with the limiter van Leer's harmonic mean of the one-sided
// differences, 0 where they differ in sign (an extremum).  FP32 divides with the fast hardware
// division (fast_div).
template <bool LIMIT, typename T>
__device__ __forceinline__ T slope(T vm, T v0, T vp, T inv2h) {
  if (!LIMIT) return (vp - vm) * inv2h;
  const T a = vp - v0, b = v0 - vm, ab = a * b;
  return ab > T(0) ? fast_div(T(4) * ab, a + b) * inv2h : T(0);
}

// Gradient of the thread's cell in plane z: x/y neighbours from the staged plane, z neighbours
// from the staged planes below/above.
template <typename T, int NC, bool LIMIT>
__device__ __forceinline__ void gradient(const Smem3<T, NC> &s, int sl, int sdn, int sup, int ty,
                                         int tx, const Cart3DArgs<T> &p, T g[3][NC]) {
  const int py = ty + 1, px = tx + 1;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T v0 = s.V[sl][c][py][px];
    g[0][c] = slope<LIMIT>(s.V[sl][c][py][px - 1], v0, s.V[sl][c][py][px + 1], p.inv2h[0]);
    g[1][c] = slope<LIMIT>(s.V[sl][c][py - 1][px], v0, s.V[sl][c][py + 1][px], p.inv2h[1]);
    g[2][c] = slope<LIMIT>(s.V[sdn][c][py][px], v0, s.V[sup][c][py][px], p.inv2h[2]);
  }
}

template <typename T, int NC>
__device__ __forceinline__ void cell_from(const Smem3<T, NC> &s, int sl, int py, int px,
                                          const T g[3][NC], Cell3<T, NC> &c) {
#pragma unroll
  for (int k = 0; k < NC; ++k) c.v[k] = s.V[sl][k][py][px];
  c.eps = s.V[sl][NC][py][px];
  c.mu = s.V[sl][NC + 1][py][px];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) c.g[a][k] = g[a][k];
}

template <typename T, int NC>
__device__ __forceinline__ void load_grad(const Smem3<T, NC> &s, int gs, int ty, int tx,
                                          T g[3][NC]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < NC; ++k) g[a][k] = s.G[gs][NC * a + k][ty][tx];
}

// One CTA per SM: FP32 512 threads (registers capped at 128), FP64 256; the cleaning system
// 384 (FP32) and 192 (FP64).
template <typename T, int NC, bool HAS_MU, bool HAS_PEC, bool LIMIT>
__global__ void __launch_bounds__(Geo3<T, NC>::NTH, 1)
    cart3d_step_kernel(const Cart3DArgs<T> p) {
  constexpr int BY = Geo3<T, NC>::BY, PY = Geo3<T, NC>::PY, NV = Geo3<T, NC>::NV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem3<T, NC> &s = *reinterpret_cast<Smem3<T, NC> *>(smem_raw);
  const int tid = threadIdx.x;
  const int tx = tid % BX, ty = tid / BX;
  const int x0 = blockIdx.x * (BX - 2), y0 = blockIdx.y * (BY - 2);
  const int z0 = blockIdx.z * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.nz);
  const int x = x0 - 1 + tx, y = y0 - 1 + ty;
  const bool inner = tx >= 1 && tx <= BX - 2 && ty >= 1 && ty <= BY - 2 && x < p.nx && y < p.ny;
  const bool need_xface = ty >= 1 && ty <= BY - 2 && tx <= BX - 2;   // faces x+1/2 of the tile
  const bool need_yface = tx >= 1 && tx <= BX - 2 && ty <= BY - 2;
  // ring entries of the staged plane (84 for 32 x 8) are loaded by threads 0 .. 83
  constexpr int NRING = 2 * PX + 2 * BY;
  int rpx = 0, rpy = 0;
  const bool ringer = tid < NRING;
  if (ringer) {
    if (tid < PX) { rpy = 0; rpx = tid; }
    else if (tid < 2 * PX) { rpy = PY - 1; rpx = tid - PX; }
    else { const int k = tid - 2 * PX; rpy = 1 + (k >> 1); rpx = (k & 1) ? PX - 1 : 0; }
  }
  const int rx = x0 - 2 + rpx, ry = y0 - 2 + rpy;
  // kinetic ghost faces on non-reflecting sides only (PEC walls are interior faces against the
  // mirrored loads)
  const bool xlo = !p.per[0] && !p.pec[0] && x == -1, xhi = !p.per[0] && !p.pec[1] && x == p.nx - 1;
  const bool ylo = !p.per[1] && !p.pec[2] && y == -1, yhi = !p.per[1] && !p.pec[3] && y == p.ny - 1;
  const bool zlo_nr = !p.per[2] && !p.pec[4], zhi_nr = !p.per[2] && !p.pec[5];

  T own[NV], ring[NV];
  // ---------------- prologue: stage planes z0-1, z0, z0+1; gradients of z0-1 and z0
  T ownm2[NV];
  load_entry<T, NC, HAS_MU, HAS_PEC>(p, x, y, z0 - 2, ownm2);
  for (int dz = -1; dz <= 1; ++dz) {
    load_entry<T, NC, HAS_MU, HAS_PEC>(p, x, y, z0 + dz, own);
    stage<T, NC>(s, (z0 + dz + NSLOT) % NSLOT, ty + 1, tx + 1, own);
    if (ringer) {
      load_entry<T, NC, HAS_MU, HAS_PEC>(p, rx, ry, z0 + dz, ring);
      stage<T, NC>(s, (z0 + dz + NSLOT) % NSLOT, rpy, rpx, ring);
    }
  }
  T pf[NV], pfr[NV];
  load_entry<T, NC, HAS_MU, HAS_PEC>(p, x, y, z0 + 2, pf);
  if (ringer) load_entry<T, NC, HAS_MU, HAS_PEC>(p, rx, ry, z0 + 2, pfr);
  __syncthreads();
  T fzb[NC];    // flux along +z through the face below the plane being processed
  {
    const int sm1 = (z0 - 1 + NSLOT) % NSLOT, s0 = z0 % NSLOT, s1 = (z0 + 1) % NSLOT;
    T gm1[3][NC], g0[3][NC];
    // gradient of z0-1: its lower z neighbour is not staged, use the register copy
    {
      const int py = ty + 1, px = tx + 1;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T v0 = s.V[sm1][c][py][px];
        gm1[0][c] = slope<LIMIT>(s.V[sm1][c][py][px - 1], v0, s.V[sm1][c][py][px + 1],
                                 p.inv2h[0]);
        gm1[1][c] = slope<LIMIT>(s.V[sm1][c][py - 1][px], v0, s.V[sm1][c][py + 1][px],
                                 p.inv2h[1]);
        gm1[2][c] = slope<LIMIT>(ownm2[c], v0, s.V[s0][c][py][px], p.inv2h[2]);
      }
    }
    gradient<T, NC, LIMIT>(s, s0, sm1, s1, ty, tx, p, g0);
    Cell3<T, NC> cm1, c0;
    cell_from<T, NC>(s, sm1, ty + 1, tx + 1, gm1, cm1);
    cell_from<T, NC>(s, s0, ty + 1, tx + 1, g0, c0);
    if (z0 == 0 && zlo_nr)
      low_boundary_face<T, FrameZm, NC>(c0, p.halfh[2], p.K[2], p.chi, p.gam, fzb);
    else
      interior_face<T, FrameZp, HAS_MU, NC>(cm1, c0, p.halfh[2], p.K[2], p.FK[2],
                                            p.K8[2], fzb);
    const int gs = z0 & 1;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < NC; ++k) s.G[gs][NC * a + k][ty][tx] = g0[a][k];
  }
  // fluxes of the plane whose update is pending
  T px_[NC], py_[NC], pzb[NC], pzt[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) { px_[c] = py_[c] = pzb[c] = pzt[c] = T(0); }
  bool bad = false;
#pragma unroll 1
  for (int z = z0; z <= z1; ++z) {
    __syncthreads();
    // finish the update of plane z-1
    if (z > z0 && inner) {
      const int fs = (z - 1) & 1;
      const int sl = (z - 1 + NSLOT) % NSLOT;
      const int64_t o = (int64_t)(z - 1) * p.plane + (int64_t)y * p.pitch + x;
      T d[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        d[c] = (s.F[fs][c][ty][tx - 1] - px_[c]) + (s.F[fs][NC + c][ty - 1][tx] - py_[c]) +
               (pzb[c] - pzt[c]);
      if (p.src && x >= p.sx0 && x < p.sx1 && y >= p.sy0 && y < p.sy1 && z - 1 >= p.sz0 &&
          z - 1 < p.sz1)
        d[2] -= p.src_amp * p.src[o];
      const T ie = rcp3(s.V[sl][NC][ty + 1][tx + 1]);
      const T im = HAS_MU ? rcp3(s.V[sl][NC + 1][ty + 1][tx + 1]) : T(1);
      T sum = T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T nv = s.V[sl][c][ty + 1][tx + 1] + d[c] * (c < 3 ? ie : (c < 6 ? im : T(1)));
        p.Vout[c * p.cstride + o] = nv;
        sum += nv;
      }
      bad |= !isfinite(sum);
    }
    if (z == z1) break;
    const int sm = (z - 1 + NSLOT) % NSLOT, s0 = z % NSLOT, s1 = (z + 1) % NSLOT;
    const int s2 = (z + 2) % NSLOT;
    // gradient of plane z+1 (its upper neighbour, plane z+2, is still in registers: stage
    // it first into its slot, which no thread reads before the next barrier except here)
    T g1[3][NC];
    {
      const int py = ty + 1, px = tx + 1;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T v0 = s.V[s1][c][py][px];
        g1[0][c] = slope<LIMIT>(s.V[s1][c][py][px - 1], v0, s.V[s1][c][py][px + 1], p.inv2h[0]);
        g1[1][c] = slope<LIMIT>(s.V[s1][c][py - 1][px], v0, s.V[s1][c][py + 1][px], p.inv2h[1]);
        g1[2][c] = slope<LIMIT>(s.V[s0][c][py][px], v0, pf[c], p.inv2h[2]);
      }
    }
    // faces of plane z
    T g0[3][NC];
    load_grad<T, NC>(s, z & 1, ty, tx, g0);
    Cell3<T, NC> c0;
    cell_from<T, NC>(s, s0, ty + 1, tx + 1, g0, c0);
    T fx[NC], fy[NC], fzt[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) { fx[c] = fy[c] = T(0); }
    if (need_xface) {
      if (xhi) {
        high_boundary_face<T, FrameXp, NC>(c0, p.halfh[0], p.K[0], p.chi, p.gam, fx);
      } else {
        T gr[3][NC];
        load_grad<T, NC>(s, z & 1, ty, tx + 1, gr);
        Cell3<T, NC> cr;
        cell_from<T, NC>(s, s0, ty + 1, tx + 2, gr, cr);
        if (xlo)
          low_boundary_face<T, FrameXm, NC>(cr, p.halfh[0], p.K[0], p.chi, p.gam, fx);
        else
          interior_face<T, FrameXp, HAS_MU, NC>(c0, cr, p.halfh[0], p.K[0], p.FK[0],
                                                p.K8[0], fx);
      }
    }
    if (need_yface) {
      if (yhi) {
        high_boundary_face<T, FrameYp, NC>(c0, p.halfh[1], p.K[1], p.chi, p.gam, fy);
      } else {
        T gu[3][NC];
        load_grad<T, NC>(s, z & 1, ty + 1, tx, gu);
        Cell3<T, NC> cu;
        cell_from<T, NC>(s, s0, ty + 2, tx + 1, gu, cu);
        if (ylo)
          low_boundary_face<T, FrameYm, NC>(cu, p.halfh[1], p.K[1], p.chi, p.gam, fy);
        else
          interior_face<T, FrameYp, HAS_MU, NC>(c0, cu, p.halfh[1], p.K[1], p.FK[1],
                                                p.K8[1], fy);
      }
    }
    if (inner) {
      if (z + 1 == p.nz && zhi_nr) {
        high_boundary_face<T, FrameZp, NC>(c0, p.halfh[2], p.K[2], p.chi, p.gam, fzt);
      } else {
        Cell3<T, NC> c1;
        cell_from<T, NC>(s, s1, ty + 1, tx + 1, g1, c1);
        interior_face<T, FrameZp, HAS_MU, NC>(c0, c1, p.halfh[2], p.K[2], p.FK[2],
                                              p.K8[2], fzt);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) fzt[c] = T(0);
    }
    // publish gradients of z+1, this thread's x/y faces; stage plane z+2; prefetch plane z+3
    {
      const int gs = (z + 1) & 1, fs = z & 1;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < NC; ++k) s.G[gs][NC * a + k][ty][tx] = g1[a][k];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        s.F[fs][c][ty][tx] = fx[c];
        s.F[fs][NC + c][ty][tx] = fy[c];
      }
      stage<T, NC>(s, s2, ty + 1, tx + 1, pf);
      if (ringer) stage<T, NC>(s, s2, rpy, rpx, pfr);
      if (z + 3 <= z1 + 1) {
        load_entry<T, NC, HAS_MU, HAS_PEC>(p, x, y, z + 3, pf);
        if (ringer) load_entry<T, NC, HAS_MU, HAS_PEC>(p, rx, ry, z + 3, pfr);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      px_[c] = fx[c];
      py_[c] = fy[c];
      pzb[c] = fzb[c];
      pzt[c] = fzt[c];
      fzb[c] = fzt[c];
    }
    (void)sm;
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(p.flag, 1);
}

template <typename T, int NC>
cudaError_t launch3_t(const CartGeom &g, const CartStepArgs &a, double chi, double gamma,
                      cudaStream_t st) {
  Cart3DArgs<T> p;
  p.V = static_cast<const T *>(a.V);
  p.Vout = static_cast<T *>(a.Vout);
  p.eps = static_cast<const T *>(a.eps);
  p.mu = static_cast<const T *>(a.mu);
  p.src = static_cast<const T *>(a.src);
  p.sx0 = a.src_box[0]; p.sx1 = a.src_box[1];
  p.sy0 = a.src_box[2]; p.sy1 = a.src_box[3];
  p.sz0 = a.src_box[4]; p.sz1 = a.src_box[5];
  p.src_amp = T(a.src_amp);
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
  p.pitch = g.pitch; p.plane = g.plane; p.cstride = g.cstride;
  for (int d = 0; d < 3; ++d) {
    p.per[d] = g.periodic[d];
    p.pec[2 * d] = g.pec[2 * d];
    p.pec[2 * d + 1] = g.pec[2 * d + 1];
    p.inv2h[d] = T(0.5 / g.h[d]);
    p.halfh[d] = T(0.5 * g.h[d]);
    p.K[d] = make_k3<T>(a.C, g.h[d], a.c);
    p.FK[d] = make_f3k<T>(a.C, g.h[d], a.c);
    p.K8[d] = make_f8k<T>(a.C, g.h[d], a.c, chi, gamma);
  }
  p.chi = T(chi);
  p.gam = T(gamma);
  p.flag = a.flag;
  constexpr int BY = Geo3<T, NC>::BY, NTH = Geo3<T, NC>::NTH;
  const int gx = (g.nx + BX - 3) / (BX - 2), gy = (g.ny + BY - 3) / (BY - 2);
  const int smem = (int)sizeof(Smem3<T, NC>);
  // z chunks: a CTA marches zchunk planes after a two-plane prologue.  Pick the chunk count
  // that fills whole waves of resident CTAs best, counting the prologue as lost work.
  // PEC walls get their own instantiation: without them the mirror bookkeeping folds away
  const bool pec = g.pec[0] || g.pec[1] || g.pec[2] || g.pec[3] || g.pec[4] || g.pec[5];
  // (the cleaning system runs with mu = 1 only)
  constexpr bool MU_OK = NC == 6;
  const bool mu = a.mu && MU_OK, lim = a.limiter != 0;
  void (*kern)(const Cart3DArgs<T>);
  if (lim)
    kern = mu ? (pec ? cart3d_step_kernel<T, NC, MU_OK, true, true>
                     : cart3d_step_kernel<T, NC, MU_OK, false, true>)
              : (pec ? cart3d_step_kernel<T, NC, false, true, true>
                     : cart3d_step_kernel<T, NC, false, false, true>);
  else
    kern = mu ? (pec ? cart3d_step_kernel<T, NC, MU_OK, true, false>
                     : cart3d_step_kernel<T, NC, MU_OK, false, false>)
              : (pec ? cart3d_step_kernel<T, NC, false, true, false>
                     : cart3d_step_kernel<T, NC, false, false, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  static int resident[2][2][2] = {};   // [has_mu][pec][limiter], per instantiation of this launcher
  int &res = resident[mu ? 1 : 0][pec ? 1 : 0][lim ? 1 : 0];
  if (!res) {
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, NTH, smem);
    res = sms * (bps > 0 ? bps : 1);
  }
  const int64_t tiles = (int64_t)gx * gy;
  int zchunks = 1;
  double best = -1.0;
  for (int zc = 1; zc <= 64 && zc <= g.nz; ++zc) {
    const int len = (g.nz + zc - 1) / zc;
    const int nzc = (g.nz + len - 1) / len;
    const int64_t ctas = tiles * nzc;
    const double waves = (double)((ctas + res - 1) / res);
    const double eff = (double)ctas / (waves * res) * (double)g.nz / (double)(nzc * (len + 2));
    if (eff > best + 1e-9) { best = eff; zchunks = nzc; }
  }
  p.zchunk = (g.nz + zchunks - 1) / zchunks;
  zchunks = (g.nz + p.zchunk - 1) / p.zchunk;
  dim3 grid(gx, gy, zchunks);
  kern<<<grid, NTH, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cart3d_step(const CartGeom &g, const CartStepArgs &a, bool fp64,
                               cudaStream_t st) {
  if (cart3d_side_supported(g, a, fp64)) return launch_cart3d_side(g, a, st);
  return fp64 ? launch3_t<double, 6>(g, a, 0.0, 0.0, st) : launch3_t<float, 6>(g, a, 0.0, 0.0, st);
}

cudaError_t launch_cart3d_phm_step(const CartGeom &g, const CartStepArgs &a, double chi,
                                   double gamma, bool fp64, cudaStream_t st) {
  return fp64 ? launch3_t<double, 8>(g, a, chi, gamma, st)
              : launch3_t<float, 8>(g, a, chi, gamma, st);
}

}  // namespace gks
