// Fused 2-D TM GKS step on a Cartesian grid: cell gradients, face reconstruction, the GKS
// interface flux and the finite-volume update in one pass over the state (Sec. 3.1).
//
// Tile scheme: a CTA owns BX x BY cells.  It stages the tile plus a two-cell halo of
// (Ez, Hx, Hy) and a one-cell halo of eps (and mu) in shared memory, computes the central
// difference gradients of the tile plus one ring (Green-Gauss on a uniform grid, face value =
// mean of the two cells), evaluates every face of the tile once, and updates its cells.
// Halo reads come mostly from L2 (neighbouring CTAs read the same lines at about the same
// time), so HBM sees the state once per step.
//
// Face frames (Sec. 3.1, T'(n)): an x-face uses n = e_x (T' = I); a y-face n = e_y with local
// axes (x', y') = (y, -x); the low boundary faces use the outward normals -e_x (T' =
// diag(-1,-1,1)) and -e_y (local (x', y') = (-y, x)).  In 2-D TM the third-moment term of the
// D3Q4 flux vanishes, so the flux of a TM face does not depend on the tangential orientation.
#include <cuda_runtime.h>

#include "gks_internal.h"

namespace gks {
namespace {

constexpr int BX = 32;
constexpr int BY = 16;
constexpr int NT = 256;
constexpr int SX = BX + 4;  // staged columns (two-cell halo)
constexpr int SY = BY + 4;
constexpr int GX = BX + 2;  // gradient ring
constexpr int GY = BY + 2;

// One side of a face in the face frame: reconstructed (Ez, Hx', Hy') = (e, a, b), their
// normal derivatives, the tangential derivatives of a and e, and the material.
template <typename T>
struct Side {
  T e, a, b;
  T ex, ax, bx;
  T ay, ey;
  T eps, mu;
};

template <typename T>
struct Coef {
  T k1, k2, k3, k4, k5;  // C_i / h_normal
  T c, c2, inv2c, halfc, c2half;
};

// Time-integrated GKS flux (Sec. 3.1) of a 2-D TM face in its frame (normal = local x),
// multiplied by dt / h.  Closed form of the per-velocity sums (D2Q4):
//   W0  = (U^l + U^r)/2 + (F_x^l - F_x^r)/(2c),          V0 = W0 / M_s
//   <u g0> = F_x(V0);  <u u.grad g0> = c^2 d_x W0;  <u g_t> = F_x(V0_t),
//   V0_t = -(F_x(d_x V0) + F_y(d_y V0)) / M_s
//   free transport: (F_x^l + F_x^r)/2 - (c/2)(U^r - U^l)
//   free transport gradient: (c^2/2)(d_x U^l + d_x U^r) + (c/2)(S^l - S^r),
//   S = F_x(d_x V) + F_y(d_y V)
// with F_x(e, a, b) = (-b, 0, -e), F_y(e, a, b) = (a, e, 0).  GHOST: the r side is a
// non-reflecting ghost (all its distributions are zero, M_s = M_l).
template <typename T, bool GHOST>
__device__ __forceinline__ void tm_face_flux(const Side<T> &L, const Side<T> &R, const Coef<T> &K,
                                             T &fe, T &fa, T &fb) {
  const T h = T(0.5);
  const T Ue_l = L.eps * L.e, Ua_l = L.mu * L.a, Ub_l = L.mu * L.b;
  const T Dxe_l = L.eps * L.ex, Dxa_l = L.mu * L.ax, Dxb_l = L.mu * L.bx, Dya_l = L.mu * L.ay;
  T Ue_r = 0, Ua_r = 0, Ub_r = 0, Dxe_r = 0, Dxa_r = 0, Dxb_r = 0, Dya_r = 0;
  T re = 0, rb = 0, rex = 0, rbx = 0, ray = 0, rey = 0;
  T ieps, imu;
  if (!GHOST) {
    Ue_r = R.eps * R.e; Ua_r = R.mu * R.a; Ub_r = R.mu * R.b;
    Dxe_r = R.eps * R.ex; Dxa_r = R.mu * R.ax; Dxb_r = R.mu * R.bx; Dya_r = R.mu * R.ay;
    re = R.e; rb = R.b; rex = R.ex; rbx = R.bx; ray = R.ay; rey = R.ey;
    ieps = T(1) / (h * (L.eps + R.eps));
    imu = T(1) / (h * (L.mu + R.mu));
  } else {
    ieps = T(1) / L.eps;
    imu = T(1) / L.mu;
  }
  // interface equilibrium moment and its gradients
  const T We = h * (Ue_l + Ue_r) + (rb - L.b) * K.inv2c;
  const T Wb = h * (Ub_l + Ub_r) + (re - L.e) * K.inv2c;
  const T Dxe = h * (Dxe_l + Dxe_r) + (rbx - L.bx) * K.inv2c;
  const T Dxa = h * (Dxa_l + Dxa_r);
  const T Dxb = h * (Dxb_l + Dxb_r) + (rex - L.ex) * K.inv2c;
  const T Dya = h * (Dya_l + Dya_r);
  // equilibrium part: C1 F_x(V0) + C2 c^2 d_x W0 + C3 F_x(V0_t)
  const T V0e = We * ieps, V0b = Wb * imu;
  const T dV0e = Dxe * ieps;
  const T Wt_e = Dxb * imu - Dya * imu;     // (d_x V0_b - d_y V0_a)
  T oe = -K.k1 * V0b + K.k2 * K.c2 * Dxe - K.k3 * dV0e * imu;
  T oa = K.k2 * K.c2 * Dxa;
  T ob = -K.k1 * V0e + K.k2 * K.c2 * Dxb - K.k3 * Wt_e * ieps;
  // free-transport part: C4 (...) - C5 (...)
  const T t4e = -h * (L.b + rb) - K.halfc * (Ue_r - Ue_l);
  const T t4a = -K.halfc * (Ua_r - Ua_l);
  const T t4b = -h * (L.e + re) - K.halfc * (Ub_r - Ub_l);
  const T t5e = K.c2half * (Dxe_l + Dxe_r) + K.halfc * ((L.ay - L.bx) - (ray - rbx));
  const T t5a = K.c2half * (Dxa_l + Dxa_r) + K.halfc * (L.ey - rey);
  const T t5b = K.c2half * (Dxb_l + Dxb_r) + K.halfc * (rex - L.ex);
  oe += K.k4 * t4e - K.k5 * t5e;
  oa += K.k4 * t4a - K.k5 * t5a;
  ob += K.k4 * t4b - K.k5 * t5b;
  fe = oe;
  fa = oa;
  fb = ob;
}

template <typename T>
struct Cart2DKernelArgs {
  const T *__restrict__ V;
  T *__restrict__ Vout;
  const T *__restrict__ eps;
  const T *__restrict__ mu;
  const T *__restrict__ src;
  int sx0, sx1, sy0, sy1;
  T src_amp;
  int nx, ny;
  int64_t pitch, cstride;
  int perx, pery;
  T inv2hx, inv2hy, halfhx, halfhy;
  Coef<T> Kx, Ky;
  int *flag;
};

__device__ __forceinline__ int wrap_or_clamp(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Shared-memory layout (dynamic): V[3][SY][SX], eps[GY][GX], mu[GY][GX], grad[6][GY][GX]
// (dEz/dx, dEz/dy, dHx/dx, dHx/dy, dHy/dx, dHy/dy), Fx[3][BY][BX+1], Fy[3][BY+1][BX].
template <typename T>
constexpr int smem_elems() {
  return 3 * SY * SX + 2 * GY * GX + 6 * GY * GX + 3 * BY * (BX + 1) + 3 * (BY + 1) * BX;
}

template <typename T, bool HAS_MU>
__global__ void __launch_bounds__(NT) cart2d_step_kernel(const Cart2DKernelArgs<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  T(*sV)[SY][SX] = reinterpret_cast<T(*)[SY][SX]>(sm);
  T(*sEps)[GX] = reinterpret_cast<T(*)[GX]>(sm + 3 * SY * SX);
  T(*sMu)[GX] = reinterpret_cast<T(*)[GX]>(sm + 3 * SY * SX + GY * GX);
  T(*sG)[GY][GX] = reinterpret_cast<T(*)[GY][GX]>(sm + 3 * SY * SX + 2 * GY * GX);
  T(*sFx)[BY][BX + 1] = reinterpret_cast<T(*)[BY][BX + 1]>(sm + 3 * SY * SX + 8 * GY * GX);
  T(*sFy)[BY + 1][BX] =
      reinterpret_cast<T(*)[BY + 1][BX]>(sm + 3 * SY * SX + 8 * GY * GX + 3 * BY * (BX + 1));

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * BX;
  const int y0 = blockIdx.y * BY;
  const int nx = p.nx, ny = p.ny;

  // 1. stage V with a two-cell halo (periodic wrap, or the ghost copy of the boundary cell)
  for (int idx = tid; idx < SY * SX; idx += NT) {
    const int ly = idx / SX, lx = idx - ly * SX;
    const int gx = wrap_or_clamp(x0 + lx - 2, nx, p.perx);
    const int gy = wrap_or_clamp(y0 + ly - 2, ny, p.pery);
    const int64_t o = (int64_t)gy * p.pitch + gx;
    sV[0][ly][lx] = p.V[o];
    sV[1][ly][lx] = p.V[o + p.cstride];
    sV[2][ly][lx] = p.V[o + 2 * p.cstride];
  }
  for (int idx = tid; idx < GY * GX; idx += NT) {
    const int ly = idx / GX, lx = idx - ly * GX;
    const int gx = wrap_or_clamp(x0 + lx - 1, nx, p.perx);
    const int gy = wrap_or_clamp(y0 + ly - 1, ny, p.pery);
    const int64_t o = (int64_t)gy * p.pitch + gx;
    sEps[ly][lx] = p.eps[o];
    if (HAS_MU) sMu[ly][lx] = p.mu[o];
  }
  __syncthreads();

  // 2. cell gradients of the tile and one ring: (V_{i+1} - V_{i-1}) / (2h)
  for (int idx = tid; idx < GY * GX; idx += NT) {
    const int ly = idx / GX, lx = idx - ly * GX;
    const int sy = ly + 1, sx = lx + 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sG[2 * c][ly][lx] = (sV[c][sy][sx + 1] - sV[c][sy][sx - 1]) * p.inv2hx;
      sG[2 * c + 1][ly][lx] = (sV[c][sy + 1][sx] - sV[c][sy - 1][sx]) * p.inv2hy;
    }
  }
  __syncthreads();

  // 3. faces.  x-face (fx, fy): between tile cells fx-1 and fx of row fy.
  for (int idx = tid; idx < BY * (BX + 1); idx += NT) {
    const int fy = idx / (BX + 1), fx = idx - fy * (BX + 1);
    const int gxl = x0 + fx - 1;              // global x of the left cell
    const int gy = y0 + fy;
    T fe = 0, fa = 0, fb = 0;
    if (gy < ny && gxl < nx) {
      const int gl = fx, gr = fx + 1;          // ring coordinates of left / right cells
      const int vy = fy + 2;
      auto side = [&](int g, int sgn) {
        // global frame: e = Ez, a = Hx, b = Hy; reconstruct to the face centre
        Side<T> s;
        const int sx = g + 1, gyy = fy + 1;
        const T dEx = sG[0][gyy][g], dEy = sG[1][gyy][g];
        const T dAx = sG[2][gyy][g], dAy = sG[3][gyy][g];
        const T dBx = sG[4][gyy][g], dBy = sG[5][gyy][g];
        s.e = sV[0][vy][sx] + T(sgn) * p.halfhx * dEx;
        s.a = sV[1][vy][sx] + T(sgn) * p.halfhx * dAx;
        s.b = sV[2][vy][sx] + T(sgn) * p.halfhx * dBx;
        s.ex = dEx; s.ax = dAx; s.bx = dBx; s.ay = dAy; s.ey = dEy;
        (void)dBy;
        s.eps = sEps[gyy][g];
        s.mu = HAS_MU ? sMu[gyy][g] : T(1);
        return s;
      };
      if (gxl >= 0 && gxl + 1 < nx) {
        tm_face_flux<T, false>(side(gl, +1), side(gr, -1), p.Kx, fe, fa, fb);
      } else if (gxl + 1 < nx || p.perx) {
        if (p.perx) {
          tm_face_flux<T, false>(side(gl, +1), side(gr, -1), p.Kx, fe, fa, fb);
        } else {
          // left boundary face, outward normal -e_x: frame T' = diag(-1, -1, 1)
          Side<T> s = side(gr, -1);
          Side<T> q;
          q.e = s.e; q.a = -s.a; q.b = -s.b;
          q.ex = -s.ex; q.ax = s.ax; q.bx = s.bx;
          q.ay = s.ay; q.ey = -s.ey;
          q.eps = s.eps; q.mu = s.mu;
          T oe, oa, ob;
          tm_face_flux<T, true>(q, q, p.Kx, oe, oa, ob);
          // F.n_out = T'^T f;  flux along +x = -F.n_out
          fe = -oe; fa = oa; fb = ob;
        }
      } else {
        if (p.perx) {
          tm_face_flux<T, false>(side(gl, +1), side(gr, -1), p.Kx, fe, fa, fb);
        } else {
          // right boundary face, outward normal +e_x (T' = I), ghost on the right
          Side<T> s = side(gl, +1);
          tm_face_flux<T, true>(s, s, p.Kx, fe, fa, fb);
        }
      }
    }
    sFx[0][fy][fx] = fe;
    sFx[1][fy][fx] = fa;
    sFx[2][fy][fx] = fb;
  }
  // y-face (fx, fy): between tile cells (fx, fy-1) and (fx, fy).
  for (int idx = tid; idx < (BY + 1) * BX; idx += NT) {
    const int fy = idx / BX, fx = idx - fy * BX;
    const int gyl = y0 + fy - 1;
    const int gx = x0 + fx;
    T fe = 0, fa = 0, fb = 0;
    if (gx < nx && gyl < ny) {
      const int vx = fx + 2;
      // local frame of n = +e_y: e = Ez, a = Hy, b = -Hx; d_x' = d_y, d_y' = -d_x
      auto side = [&](int gyy, int sgn) {
        Side<T> s;
        const int sy = gyy + 1, gxx = fx + 1;
        const T dEx = sG[0][gyy][gxx], dEy = sG[1][gyy][gxx];
        const T dHxx = sG[2][gyy][gxx], dHxy = sG[3][gyy][gxx];
        const T dHyx = sG[4][gyy][gxx], dHyy = sG[5][gyy][gxx];
        const T ez = sV[0][sy][vx] + T(sgn) * p.halfhy * dEy;
        const T hx = sV[1][sy][vx] + T(sgn) * p.halfhy * dHxy;
        const T hy = sV[2][sy][vx] + T(sgn) * p.halfhy * dHyy;
        s.e = ez; s.a = hy; s.b = -hx;
        s.ex = dEy; s.ax = dHyy; s.bx = -dHxy;
        s.ay = -dHyx; s.ey = -dEx;
        s.eps = sEps[gyy][gxx];
        s.mu = HAS_MU ? sMu[gyy][gxx] : T(1);
        return s;
      };
      const int ll = fy, rr = fy + 1;  // ring rows of the lower / upper cell
      T oe, oa, ob;
      if ((gyl >= 0 && gyl + 1 < ny) || p.pery) {
        tm_face_flux<T, false>(side(ll, +1), side(rr, -1), p.Ky, oe, oa, ob);
        // back to global: Phi_Ez = f_e, Phi_Hx = -f_b, Phi_Hy = f_a
        fe = oe; fa = -ob; fb = oa;
      } else if (gyl < 0) {
        // bottom boundary, outward normal -e_y: local (x', y') = (-y, x);
        // e = Ez, a = -Hy, b = Hx; d_x' = -d_y, d_y' = d_x
        Side<T> s = side(rr, -1);   // expressed in the +e_y frame: (e, Hy, -Hx), (d_y, -d_x)
        Side<T> q;
        q.e = s.e; q.a = -s.a; q.b = -s.b;
        q.ex = -s.ex; q.ax = s.ax; q.bx = s.bx;
        q.ay = s.ay; q.ey = -s.ey;
        q.eps = s.eps; q.mu = s.mu;
        tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
        // F.n_out: Phi_Ez = f_e, Phi_Hx = f_b, Phi_Hy = -f_a; flux along +y = -F.n_out
        fe = -oe; fa = -ob; fb = oa;
      } else {
        Side<T> s = side(ll, +1);
        tm_face_flux<T, true>(s, s, p.Ky, oe, oa, ob);
        fe = oe; fa = -ob; fb = oa;
      }
    }
    sFy[0][fy][fx] = fe;
    sFy[1][fy][fx] = fa;
    sFy[2][fy][fx] = fb;
  }
  __syncthreads();

  // 4. update: U^{n+1} = U^n - dt/|Omega| sum |l| F + dt S  (fluxes already carry dt/h)
  bool bad = false;
  for (int idx = tid; idx < BY * BX; idx += NT) {
    const int ly = idx / BX, lx = idx - ly * BX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) continue;
    const T ie = T(1) / sEps[ly + 1][lx + 1];
    const T im = HAS_MU ? T(1) / sMu[ly + 1][lx + 1] : T(1);
    T de = -(sFx[0][ly][lx + 1] - sFx[0][ly][lx]) - (sFy[0][ly + 1][lx] - sFy[0][ly][lx]);
    const T da = -(sFx[1][ly][lx + 1] - sFx[1][ly][lx]) - (sFy[1][ly + 1][lx] - sFy[1][ly][lx]);
    const T db = -(sFx[2][ly][lx + 1] - sFx[2][ly][lx]) - (sFy[2][ly + 1][lx] - sFy[2][ly][lx]);
    const int64_t o = (int64_t)gy * p.pitch + gx;
    if (p.src && gx >= p.sx0 && gx < p.sx1 && gy >= p.sy0 && gy < p.sy1) de -= p.src_amp * p.src[o];
    const T ve = sV[0][ly + 2][lx + 2] + de * ie;
    const T va = sV[1][ly + 2][lx + 2] + da * im;
    const T vb = sV[2][ly + 2][lx + 2] + db * im;
    p.Vout[o] = ve;
    p.Vout[o + p.cstride] = va;
    p.Vout[o + 2 * p.cstride] = vb;
    bad |= !(isfinite(ve) && isfinite(va) && isfinite(vb));
  }
  if (__any_sync(0xffffffffu, bad) && (tid & 31) == 0) atomicOr(p.flag, 1);
}

template <typename T>
Coef<T> make_coef(const double C[5], double h, double c) {
  Coef<T> k;
  k.k1 = T(C[0] / h); k.k2 = T(C[1] / h); k.k3 = T(C[2] / h);
  k.k4 = T(C[3] / h); k.k5 = T(C[4] / h);
  k.c = T(c); k.c2 = T(c * c); k.inv2c = T(0.5 / c); k.halfc = T(0.5 * c);
  k.c2half = T(0.5 * c * c);
  return k;
}

template <typename T>
cudaError_t launch_t(const CartGeom &g, const CartStepArgs &a, cudaStream_t st) {
  Cart2DKernelArgs<T> p;
  p.V = static_cast<const T *>(a.V);
  p.Vout = static_cast<T *>(a.Vout);
  p.eps = static_cast<const T *>(a.eps);
  p.mu = static_cast<const T *>(a.mu);
  p.src = static_cast<const T *>(a.src);
  p.sx0 = a.src_box[0]; p.sx1 = a.src_box[1];
  p.sy0 = a.src_box[2]; p.sy1 = a.src_box[3];
  p.src_amp = T(a.src_amp);
  p.nx = g.nx; p.ny = g.ny;
  p.pitch = g.pitch; p.cstride = g.cstride;
  p.perx = g.periodic[0]; p.pery = g.periodic[1];
  p.inv2hx = T(0.5 / g.h[0]); p.inv2hy = T(0.5 / g.h[1]);
  p.halfhx = T(0.5 * g.h[0]); p.halfhy = T(0.5 * g.h[1]);
  p.Kx = make_coef<T>(a.C, g.h[0], a.c);
  p.Ky = make_coef<T>(a.C, g.h[1], a.c);
  p.flag = a.flag;
  const size_t smem = sizeof(T) * smem_elems<T>();
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY);
  if (a.mu) {
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(cart2d_step_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      set = true;
    }
    cart2d_step_kernel<T, true><<<grid, NT, smem, st>>>(p);
  } else {
    static bool set = false;
    if (!set) {
      cudaFuncSetAttribute(cart2d_step_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      set = true;
    }
    cart2d_step_kernel<T, false><<<grid, NT, smem, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cart2d_step(const CartGeom &g, const CartStepArgs &a, bool fp64,
                               cudaStream_t st) {
  return fp64 ? launch_t<double>(g, a, st) : launch_t<float>(g, a, st);
}

}  // namespace gks
