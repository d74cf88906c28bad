// Fused 2-D TM GKS step on a Cartesian grid: cell gradients, face reconstruction, the GKS
// interface flux and the finite-volume update in one pass over the state (Sec. 3.1).
//
// Warp-strip march.  Each warp owns a strip of 64 columns and a chunk of rows and walks up the
// rows on its own (no shared memory, no barriers).  Lane l holds columns X = x0-2+2l and X+1
// of the rows j .. j+2 in registers, with two more rows in flight; x-neighbours come from the
// adjacent lanes by shuffles.  Every gradient and every face is evaluated once: per row a lane
// forms the central differences of row j+1, the x-faces X+1/2 and X+3/2 and the y-faces
// j+1/2 of its two columns, and updates its two cells of row j.
//
// Face frames (Sec. 3.1, T'(n)): an x-face uses n = e_x (T' = I); a y-face n = e_y with local
// axes (x', y') = (y, -x); the low boundary faces use the outward normals -e_x (T' =
// diag(-1,-1,1)) and -e_y (local (x', y') = (-y, x)).  A PEC wall (Sec. 5.5) is an interior face
// against mirror-image cells: the loads reflect the index across the wall and negate the
// tangential E and the normal H, so the ghost's gradient and reconstruction are the mirror of
// the inner cell's.  In 2-D TM the third-moment term of the
// D3Q4 flux vanishes, so a TM face flux does not depend on the tangential orientation.
#include <cuda_runtime.h>

#include "gks_flux2.cuh"
#include "gks_internal.h"
#include "gks_tma.cuh"

namespace gks {
namespace {


// Reciprocals: FP32 uses the fast hardware reciprocal (about 1 ulp), FP64 divides.
__device__ __forceinline__ float rcp1(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp1(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp2(float x) { return __fdividef(2.f, x); }
__device__ __forceinline__ double rcp2(double x) { return 2.0 / x; }

// Scalar form used on boundary faces (rare): the face frame's (Ez, Hx', Hy') = (e, a, b).
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
// multiplied by dt / h.  Closed form of the per-velocity D2Q4 sums:
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
  const T We = h * (Ue_l + Ue_r) + (rb - L.b) * K.inv2c;
  const T Wb = h * (Ub_l + Ub_r) + (re - L.e) * K.inv2c;
  const T Dxe = h * (Dxe_l + Dxe_r) + (rbx - L.bx) * K.inv2c;
  const T Dxa = h * (Dxa_l + Dxa_r);
  const T Dxb = h * (Dxb_l + Dxb_r) + (rex - L.ex) * K.inv2c;
  const T Dya = h * (Dya_l + Dya_r);
  const T V0e = We * ieps, V0b = Wb * imu;
  const T dV0e = Dxe * ieps;
  const T Wt_e = Dxb * imu - Dya * imu;
  T oe = -K.k1 * V0b + K.k2 * K.c2 * Dxe - K.k3 * dV0e * imu;
  T oa = K.k2 * K.c2 * Dxa;
  T ob = -K.k1 * V0e + K.k2 * K.c2 * Dxb - K.k3 * Wt_e * ieps;
  const T t4e = -h * (L.b + rb) - K.halfc * (Ue_r - Ue_l);
  const T t4a = -K.halfc * (Ua_r - Ua_l);
  const T t4b = -h * (L.e + re) - K.halfc * (Ub_r - Ub_l);
  const T t5e = K.c2half * (Dxe_l + Dxe_r) + K.halfc * ((L.ay - L.bx) - (ray - rbx));
  const T t5a = K.c2half * (Dxa_l + Dxa_r) + K.halfc * (L.ey - rey);
  const T t5b = K.c2half * (Dxb_l + Dxb_r) + K.halfc * (rex - L.ex);
  fe = oe + K.k4 * t4e - K.k5 * t5e;
  fa = oa + K.k4 * t4a - K.k5 * t5a;
  fb = ob + K.k4 * t4b - K.k5 * t5b;
}

// One side of an interior face in global components: e = Ez, hn = normal H, ht =
// tangential H (reconstructed at the face), the raw central differences along the normal of
// (Ez, Hn, Ht) (dn_* = V_{+1} - V_{-1}), the raw tangential differences of Hn and Ez, and the
// material.
template <typename T>
struct FSide {
  T e, hn, ht, den, dhn, dht, dat, det, eps, mu;
};

// Interior face flux (times dt/h), global components, from raw differences:
//   Phi_E  = im (a1 S_UB + a2 D_e) + g (S_Uxe/2 + a3 D_xB) + a4 S_B - q2 D_Ue - q3 S_Uxe
//            + a5 D_At + a6 D_xB
//   Phi_Hn = q5 S_Uxa - q2 D_Ua + b1 D_Et
//   Phi_Ht = ie (c1 S_Ue + c2 D_B) + g (S_UxB/2 + c3 D_ex) + c4 ie im S_UAt + c5 S_e - q2 D_UB
//            - q3 S_UxB + c6 D_ex
// with S_* = l + r sums, D_* = r - l differences, U* = M V, ie = 1/eps_s, im = 1/mu_s and
// g = g0 - k3 ie im.  This is tm_face_flux above rewritten in sums and differences, with the
// face-frame signs, the C1..C5 combinations and the 1/(2h) of the central differences folded
// into FaceK (make_face_k).
template <typename T, bool HAS_MU>
__device__ __forceinline__ void face_flux(const FSide<T> &l, const FSide<T> &r, const FaceK<T> &k,
                                          T &fE, T &fHn, T &fHt) {
  const T Ue_l = l.eps * l.e, Ue_r = r.eps * r.e;
  const T Uxe_l = l.eps * l.den, Uxe_r = r.eps * r.den;
  T UB_l = l.ht, UB_r = r.ht, Ua_l = l.hn, Ua_r = r.hn;
  T UxB_l = l.dht, UxB_r = r.dht, Uxa_l = l.dhn, Uxa_r = r.dhn, UAt_l = l.dat, UAt_r = r.dat;
  if (HAS_MU) {
    UB_l *= l.mu; UB_r *= r.mu; Ua_l *= l.mu; Ua_r *= r.mu;
    UxB_l *= l.mu; UxB_r *= r.mu; Uxa_l *= l.mu; Uxa_r *= r.mu; UAt_l *= l.mu; UAt_r *= r.mu;
  }
  const T S_UB = UB_l + UB_r, D_e = r.e - l.e;
  const T S_Uxe = Uxe_l + Uxe_r, D_xB = r.dht - l.dht;
  const T S_B = l.ht + r.ht, D_Ue = Ue_r - Ue_l, D_At = r.dat - l.dat;
  const T S_Uxa = Uxa_l + Uxa_r, D_Ua = Ua_r - Ua_l, D_Et = r.det - l.det;
  const T S_Ue = Ue_l + Ue_r, D_B = r.ht - l.ht, S_UxB = UxB_l + UxB_r;
  const T D_ex = r.den - l.den, S_UAt = UAt_l + UAt_r, S_e = l.e + r.e;
  const T D_UB = UB_r - UB_l;
  const T ie = rcp2(l.eps + r.eps);                 // 1 / ((eps_l + eps_r)/2)
  const T im = HAS_MU ? rcp2(l.mu + r.mu) : T(1);
  const T iem = HAS_MU ? ie * im : ie;
  const T g = k.g0 - k.k3 * iem;
  T fe = k.a1 * S_UB + k.a2 * D_e;
  if (HAS_MU) fe *= im;
  fe += g * (T(0.5) * S_Uxe + k.a3 * D_xB);
  fe += k.a4 * S_B - k.q2 * D_Ue - k.q3 * S_Uxe + k.a5 * D_At + k.a6 * D_xB;
  const T fa = k.q5 * S_Uxa - k.q2 * D_Ua + k.b1 * D_Et;
  T fb = ie * (k.c1 * S_Ue + k.c2 * D_B);
  fb += g * (T(0.5) * S_UxB + k.c3 * D_ex);
  fb += k.c4 * iem * S_UAt + k.c5 * S_e - k.q2 * D_UB - k.q3 * S_UxB + k.c6 * D_ex;
  fE = fe;
  fHn = fa;
  fHt = fb;
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
  int pec[4];          // PEC wall on the -x, +x, -y, +y side
  T inv2hx, inv2hy;
  FaceK<T> fx, fy;     // interior x- and y-faces
  Coef<T> Kx, Ky;      // boundary faces (scalar path)
  int *flag;
};

// Cell of index i on an axis of n cells: periodic wrap, PEC mirror (m = true: the entry is the
// mirror image -1-i or 2n-1-i; indices further out than the two-cell stencil are clamped) or
// the non-reflecting clamp.
__device__ __forceinline__ int axis_index(int i, int n, int periodic, int pec_lo, int pec_hi,
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

// One row of a thread's column: (Ez, Hx, Hy) and the material.
template <typename T>
struct RowV {
  T ez, hx, hy, eps, mu;
};
// Raw central differences of one row: x and y differences of (Ez, Hx, Hy).
template <typename T>
struct RowG {
  T ex, ey, ax, ay, bx, by;
};

// ------------------------------------------------------------------ warp-strip march
// A warp owns a strip of 64 columns x0-2 .. x0+61 (lane l: columns X = x0-2+2l and X+1) and
// updates columns x0 .. x0+59 (lanes 1..30).  x-neighbours come from the adjacent lanes by
// warp shuffles; rows are loaded straight into registers (float2 / double2 per lane, coalesced)
// two rows ahead of use.  No shared memory and no barriers: warps march independently.
constexpr int WARPS = 4;             // warps per CTA
#ifndef GKS_CART2D_MINBLOCKS
#define GKS_CART2D_MINBLOCKS 1           // CTAs per SM the register allocation must allow
#endif
constexpr int WCOLS = 60;            // columns updated per warp
constexpr unsigned FULL = 0xffffffffu;

template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

// Two columns of one row: (Ez, Hx, Hy, eps, mu), and which entries are PEC mirror images
// (xm: of an x-wall, per column; ym: of a y-wall).  The signs of a mirror image are applied by
// apply_mirror when the row enters the working window, not at the load, so that a prefetched
// row is not waited for early.
template <typename T>
struct Row2 {
  T ez[2], hx[2], hy[2], eps[2], mu[2];
  bool xm[2], ym;
};

// PEC mirror image: an x-wall negates Ez and Hx, a y-wall Ez and Hy.
template <typename T>
__device__ __forceinline__ void apply_mirror(Row2<T> &v) {
  if (v.ym | v.xm[0] | v.xm[1]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (v.xm[k] != v.ym) v.ez[k] = -v.ez[k];
      if (v.xm[k]) v.hx[k] = -v.hx[k];
      if (v.ym) v.hy[k] = -v.hy[k];
    }
  }
}

template <typename T, bool HAS_MU, bool HAS_PEC>
__device__ __forceinline__ Row2<T> load_row2(const Cart2DKernelArgs<T> &p, int X, int row) {
  using P = typename Pair2<T>::type;
  Row2<T> v;
  const int r = axis_index(row, p.ny, p.pery, HAS_PEC && p.pec[2], HAS_PEC && p.pec[3], v.ym);
  v.xm[0] = v.xm[1] = false;
  const int64_t ro = (int64_t)r * p.pitch;
  if (X >= 0 && X + 1 < p.nx) {
    const P a = __ldg(reinterpret_cast<const P *>(p.V + ro + X));
    const P b = __ldg(reinterpret_cast<const P *>(p.V + p.cstride + ro + X));
    const P c = __ldg(reinterpret_cast<const P *>(p.V + 2 * p.cstride + ro + X));
    const P e = __ldg(reinterpret_cast<const P *>(p.eps + ro + X));
    v.ez[0] = a.x; v.ez[1] = a.y; v.hx[0] = b.x; v.hx[1] = b.y;
    v.hy[0] = c.x; v.hy[1] = c.y; v.eps[0] = e.x; v.eps[1] = e.y;
    if (HAS_MU) {
      const P m = __ldg(reinterpret_cast<const P *>(p.mu + ro + X));
      v.mu[0] = m.x; v.mu[1] = m.y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t o =
          ro + axis_index(X + k, p.nx, p.perx, HAS_PEC && p.pec[0], HAS_PEC && p.pec[1], v.xm[k]);
      v.ez[k] = __ldg(p.V + o);
      v.hx[k] = __ldg(p.V + p.cstride + o);
      v.hy[k] = __ldg(p.V + 2 * p.cstride + o);
      v.eps[k] = __ldg(p.eps + o);
      if (HAS_MU) v.mu[k] = __ldg(p.mu + o);
    }
  }
  if (!HAS_MU) { v.mu[0] = T(1); v.mu[1] = T(1); }
  return v;
}

template <typename T>
__device__ __forceinline__ RowV<T> col_of(const Row2<T> &v, int k) {
  RowV<T> c;
  c.ez = v.ez[k]; c.hx = v.hx[k]; c.hy = v.hy[k]; c.eps = v.eps[k]; c.mu = v.mu[k];
  return c;
}

// x-face side of a cell (normal x: hn = Hx, ht = Hy; tangential derivatives along y),
// reconstructed by sgn * (h/2) d/dx = sgn * (raw difference)/4.
template <typename T>
__device__ __forceinline__ FSide<T> xface_side(const RowV<T> &v, const RowG<T> &g, T sgn4) {
  FSide<T> s;
  s.e = v.ez + sgn4 * g.ex; s.hn = v.hx + sgn4 * g.ax; s.ht = v.hy + sgn4 * g.bx;
  s.den = g.ex; s.dhn = g.ax; s.dht = g.bx; s.dat = g.ay; s.det = g.ey;
  s.eps = v.eps; s.mu = v.mu;
  return s;
}

// y-face side (normal y: hn = Hy, ht = Hx; tangential derivatives along x).
template <typename T>
__device__ __forceinline__ FSide<T> yface_side(const RowV<T> &v, const RowG<T> &g, T sgn4) {
  FSide<T> s;
  s.e = v.ez + sgn4 * g.ey; s.hn = v.hy + sgn4 * g.by; s.ht = v.hx + sgn4 * g.ay;
  s.den = g.ey; s.dhn = g.by; s.dht = g.ay; s.dat = g.bx; s.det = g.ex;
  s.eps = v.eps; s.mu = v.mu;
  return s;
}

// Boundary sides for the scalar path (derivatives scaled to true gradients).
template <typename T>
__device__ __forceinline__ Side<T> xside_scalar(const RowV<T> &v, const RowG<T> &g, T sgn4, T sx,
                                               T sy) {
  Side<T> s;
  s.e = v.ez + sgn4 * g.ex; s.a = v.hx + sgn4 * g.ax; s.b = v.hy + sgn4 * g.bx;
  s.ex = g.ex * sx; s.ax = g.ax * sx; s.bx = g.bx * sx;
  s.ay = g.ay * sy; s.ey = g.ey * sy;
  s.eps = v.eps; s.mu = v.mu;
  return s;
}

// In the +e_y face frame: e = Ez, a = Hy, b = -Hx; d_x' = d_y, d_y' = -d_x.
template <typename T>
__device__ __forceinline__ Side<T> yside_scalar(const RowV<T> &v, const RowG<T> &g, T sgn4, T sx,
                                               T sy) {
  Side<T> s;
  s.e = v.ez + sgn4 * g.ey;
  s.a = v.hy + sgn4 * g.by;
  s.b = -(v.hx + sgn4 * g.ay);
  s.ex = g.ey * sy; s.ax = g.by * sy; s.bx = -g.ay * sy;
  s.ay = -g.bx * sx; s.ey = -g.ex * sx;
  s.eps = v.eps; s.mu = v.mu;
  return s;
}

// Flux along +x of the low-x boundary face of a cell (outward normal -e_x, frame
// diag(-1,-1,1)), given the cell's x-frame side reconstructed to that face.
template <typename T>
__device__ __forceinline__ void low_boundary_flux(const Side<T> &s, const Coef<T> &K, T &fe, T &fa,
                                                  T &fb) {
  Side<T> q;
  q.e = s.e; q.a = -s.a; q.b = -s.b;
  q.ex = -s.ex; q.ax = s.ax; q.bx = s.bx;
  q.ay = s.ay; q.ey = -s.ey;
  q.eps = s.eps; q.mu = s.mu;
  T oe, oa, ob;
  tm_face_flux<T, true>(q, q, K, oe, oa, ob);
  fe = -oe; fa = oa; fb = ob;
}

// Flux along +y of the face below a cell on the low-y boundary (outward normal -e_y).
template <typename T>
__device__ __forceinline__ void low_y_boundary_flux(const RowV<T> &v, const RowG<T> &g,
                                                    const Cart2DKernelArgs<T> &p, T &fE, T &fHx,
                                                    T &fHy) {
  const Side<T> sq = yside_scalar<T>(v, g, T(-0.25), p.inv2hx, p.inv2hy);
  Side<T> q;
  q.e = sq.e; q.a = -sq.a; q.b = -sq.b;
  q.ex = -sq.ex; q.ax = sq.ax; q.bx = sq.bx;
  q.ay = sq.ay; q.ey = -sq.ey;
  q.eps = sq.eps; q.mu = sq.mu;
  T oe, oa, ob;
  tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
  fE = -oe; fHx = -ob; fHy = oa;
}

// Raw central differences of the lane's two columns in a row (limited slopes with LIMIT):
// x-neighbours by shuffle, the rows below and above from registers.  right_* receive column X+2
// of this row (reused by the x-face of the row).
template <typename T, bool LIMIT>
__device__ __forceinline__ void diffs2(const Row2<T> &c, const Row2<T> &dn, const Row2<T> &up,
                                       RowG<T> g[2], T right[3]) {
  const T lE = __shfl_up_sync(FULL, c.ez[1], 1), rE = __shfl_down_sync(FULL, c.ez[0], 1);
  const T lA = __shfl_up_sync(FULL, c.hx[1], 1), rA = __shfl_down_sync(FULL, c.hx[0], 1);
  const T lB = __shfl_up_sync(FULL, c.hy[1], 1), rB = __shfl_down_sync(FULL, c.hy[0], 1);
  g[0].ex = raw_slope<LIMIT>(lE, c.ez[0], c.ez[1]);
  g[1].ex = raw_slope<LIMIT>(c.ez[0], c.ez[1], rE);
  g[0].ax = raw_slope<LIMIT>(lA, c.hx[0], c.hx[1]);
  g[1].ax = raw_slope<LIMIT>(c.hx[0], c.hx[1], rA);
  g[0].bx = raw_slope<LIMIT>(lB, c.hy[0], c.hy[1]);
  g[1].bx = raw_slope<LIMIT>(c.hy[0], c.hy[1], rB);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    g[k].ey = raw_slope<LIMIT>(dn.ez[k], c.ez[k], up.ez[k]);
    g[k].ay = raw_slope<LIMIT>(dn.hx[k], c.hx[k], up.hx[k]);
    g[k].by = raw_slope<LIMIT>(dn.hy[k], c.hy[k], up.hy[k]);
  }
  right[0] = rE; right[1] = rA; right[2] = rB;
}

template <typename T, bool HAS_MU, bool HAS_PEC, bool LIMIT>
__global__ void __launch_bounds__(WARPS * 32, GKS_CART2D_MINBLOCKS) cart2d_step_kernel(const Cart2DKernelArgs<T> p,
                                                                 int nstrips, int rows,
                                                                 int strip0, int ybeg, int yend) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int strip = strip0 + wid % nstrips, chunk = wid / nstrips;
  const int y0 = ybeg + chunk * rows;
  if (y0 >= yend) return;                             // whole warp leaves together
  const int y1 = min(y0 + rows, yend);
  const int x0 = strip * WCOLS;
  const int X = x0 - 2 + 2 * lane;
  const int xend = min(x0 + WCOLS, p.nx);
  // non-reflecting sides use the kinetic ghost faces; PEC walls are interior faces against the
  // mirrored loads, periodic sides wrap
  const bool xlo_nr = !p.perx && !p.pec[0], xhi_nr = !p.perx && !p.pec[1];
  const bool ylo_nr = !p.pery && !p.pec[2], yhi_nr = !p.pery && !p.pec[3];
  const T q4 = T(0.25), mq4 = T(-0.25);

  // ---------------- prologue: rows y0-2 .. y0+3 loaded, differences of rows y0-1, y0
  Row2<T> vm2 = load_row2<T, HAS_MU, HAS_PEC>(p, X, y0 - 2);
  Row2<T> vm1 = load_row2<T, HAS_MU, HAS_PEC>(p, X, y0 - 1);
  Row2<T> v0 = load_row2<T, HAS_MU, HAS_PEC>(p, X, y0);
  Row2<T> v1 = load_row2<T, HAS_MU, HAS_PEC>(p, X, y0 + 1);
  Row2<T> v2 = load_row2<T, HAS_MU, HAS_PEC>(p, X, y0 + 2);
  Row2<T> pf = load_row2<T, HAS_MU, HAS_PEC>(p, X, y0 + 3);
  if (HAS_PEC) {
    apply_mirror(vm2);
    apply_mirror(vm1);
    apply_mirror(v0);
    apply_mirror(v1);
    apply_mirror(v2);
  }
  RowG<T> g0[2], gm1[2];
  T r0[3], rm1[3];
  diffs2<T, LIMIT>(vm1, vm2, v0, gm1, rm1);
  diffs2<T, LIMIT>(v0, vm1, v1, g0, r0);
  T fbE[2], fbHx[2], fbHy[2];                         // flux along +y below row j
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (y0 == 0 && ylo_nr)
      low_y_boundary_flux<T>(col_of(v0, k), g0[k], p, fbE[k], fbHx[k], fbHy[k]);
    else
      face_flux<T, HAS_MU>(yface_side<T>(col_of(vm1, k), gm1[k], q4),
                           yface_side<T>(col_of(v0, k), g0[k], mq4), p.fy, fbE[k], fbHy[k],
                           fbHx[k]);
  }
  bool bad = false;
#pragma unroll 1
  for (int j = y0; j < y1; ++j) {
    const Row2<T> pf2 = load_row2<T, HAS_MU, HAS_PEC>(p, X, j + 4);   // two rows ahead of use
    RowG<T> g1[2];
    T r1[3];
    diffs2<T, LIMIT>(v1, v0, v2, g1, r1);
    // x-faces of row j: X+1/2 (own columns) and X+3/2 (own X+1, column X+2 of the next lane)
    T fxE[2], fxHx[2], fxHy[2];
    {
      RowV<T> nb;   // column X+2
      nb.ez = r0[0]; nb.hx = r0[1]; nb.hy = r0[2];
      nb.eps = __shfl_down_sync(FULL, v0.eps[0], 1);
      nb.mu = HAS_MU ? __shfl_down_sync(FULL, v0.mu[0], 1) : T(1);
      RowG<T> gn;
      gn.ex = __shfl_down_sync(FULL, g0[0].ex, 1);
      gn.ax = __shfl_down_sync(FULL, g0[0].ax, 1);
      gn.bx = __shfl_down_sync(FULL, g0[0].bx, 1);
      gn.ay = __shfl_down_sync(FULL, g0[0].ay, 1);
      gn.ey = __shfl_down_sync(FULL, g0[0].ey, 1);
      gn.by = T(0);
      const RowV<T> c0 = col_of(v0, 0), c1 = col_of(v0, 1);
      face_flux<T, HAS_MU>(xface_side<T>(c0, g0[0], q4), xface_side<T>(c1, g0[1], mq4), p.fx,
                           fxE[0], fxHx[0], fxHy[0]);
      face_flux<T, HAS_MU>(xface_side<T>(c1, g0[1], q4), xface_side<T>(nb, gn, mq4), p.fx,
                           fxE[1], fxHx[1], fxHy[1]);
      if (xhi_nr) {
        if (X == p.nx - 1) {            // first face on the high-x boundary
          const Side<T> q = xside_scalar<T>(c0, g0[0], q4, p.inv2hx, p.inv2hy);
          tm_face_flux<T, true>(q, q, p.Kx, fxE[0], fxHx[0], fxHy[0]);
        }
        if (X + 1 == p.nx - 1) {        // second face on the high-x boundary
          const Side<T> q = xside_scalar<T>(c1, g0[1], q4, p.inv2hx, p.inv2hy);
          tm_face_flux<T, true>(q, q, p.Kx, fxE[1], fxHx[1], fxHy[1]);
        }
      }
      if (xlo_nr && X == -2) {          // second face is the low-x boundary face of column 0
        low_boundary_flux<T>(xside_scalar<T>(nb, gn, mq4, p.inv2hx, p.inv2hy), p.Kx, fxE[1],
                             fxHx[1], fxHy[1]);
      }
    }
    // y-faces between rows j and j+1
    T ftE[2], ftHx[2], ftHy[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const RowV<T> c = col_of(v0, k);
      if (j + 1 == p.ny && yhi_nr) {
        const Side<T> q = yside_scalar<T>(c, g0[k], q4, p.inv2hx, p.inv2hy);
        T oe, oa, ob;
        tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
        ftE[k] = oe; ftHx[k] = -ob; ftHy[k] = oa;
      } else {
        face_flux<T, HAS_MU>(yface_side<T>(c, g0[k], q4), yface_side<T>(col_of(v1, k), g1[k], mq4),
                             p.fy, ftE[k], ftHy[k], ftHx[k]);
      }
    }
    // update row j: left face of column X is the previous lane's second face
    {
      const T lE = __shfl_up_sync(FULL, fxE[1], 1);
      const T lHx = __shfl_up_sync(FULL, fxHx[1], 1);
      const T lHy = __shfl_up_sync(FULL, fxHy[1], 1);
      T dE[2], dHx[2], dHy[2];
      dE[0] = (lE - fxE[0]) + (fbE[0] - ftE[0]);
      dHx[0] = (lHx - fxHx[0]) + (fbHx[0] - ftHx[0]);
      dHy[0] = (lHy - fxHy[0]) + (fbHy[0] - ftHy[0]);
      dE[1] = (fxE[0] - fxE[1]) + (fbE[1] - ftE[1]);
      dHx[1] = (fxHx[0] - fxHx[1]) + (fbHx[1] - ftHx[1]);
      dHy[1] = (fxHy[0] - fxHy[1]) + (fbHy[1] - ftHy[1]);
      const int64_t ro = (int64_t)j * p.pitch;
      if (p.src && j >= p.sy0 && j < p.sy1) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (X + k >= p.sx0 && X + k < p.sx1) dE[k] -= p.src_amp * p.src[ro + X + k];
      }
      T ne[2], nhx[2], nhy[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        ne[k] = v0.ez[k] + dE[k] * rcp1(v0.eps[k]);
        if (HAS_MU) {
          const T im = rcp1(v0.mu[k]);
          nhx[k] = v0.hx[k] + dHx[k] * im;
          nhy[k] = v0.hy[k] + dHy[k] * im;
        } else {
          nhx[k] = v0.hx[k] + dHx[k];
          nhy[k] = v0.hy[k] + dHy[k];
        }
      }
      const bool ok0 = X >= x0 && X < xend, ok1 = X + 1 >= x0 && X + 1 < xend;
      using P = typename Pair2<T>::type;
      if (ok0 && ok1) {
        P a, b, c;
        a.x = ne[0]; a.y = ne[1]; b.x = nhx[0]; b.y = nhx[1]; c.x = nhy[0]; c.y = nhy[1];
        *reinterpret_cast<P *>(p.Vout + ro + X) = a;
        *reinterpret_cast<P *>(p.Vout + p.cstride + ro + X) = b;
        *reinterpret_cast<P *>(p.Vout + 2 * p.cstride + ro + X) = c;
        bad |= !(isfinite(ne[0]) && isfinite(nhx[0]) && isfinite(nhy[0]) && isfinite(ne[1]) &&
                 isfinite(nhx[1]) && isfinite(nhy[1]));
      } else {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (k == 0 ? ok0 : ok1) {
            p.Vout[ro + X + k] = ne[k];
            p.Vout[p.cstride + ro + X + k] = nhx[k];
            p.Vout[2 * p.cstride + ro + X + k] = nhy[k];
            bad |= !(isfinite(ne[k]) && isfinite(nhx[k]) && isfinite(nhy[k]));
          }
        }
      }
    }
    // rotate the register window
    v0 = v1; v1 = v2; v2 = pf; pf = pf2;
    if (HAS_PEC) apply_mirror(v2);            // the prefetched row takes its mirror signs now
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      g0[k] = g1[k];
      fbE[k] = ftE[k]; fbHx[k] = ftHx[k]; fbHy[k] = ftHy[k];
    }
    r0[0] = r1[0]; r0[1] = r1[1]; r0[2] = r1[2];
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.flag, 1);
}

// ------------------------------------------------------------------ paired FP32 path
// FP32 with mu = 1.  A lane's two x-faces (X+1/2, X+3/2), its two y-faces (columns X, X+1) and
// its two cell updates run the same arithmetic, so they go through Blackwell's paired FP32
// instructions (__fadd2_rn, __fmul2_rn, __ffma2_rn): component x is the first face or column,
// y the second.  Same march, same closed-form face flux as cart2d_step_kernel.
using f2 = float2;
__device__ __forceinline__ f2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 padd(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 psub(f2 a, f2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ f2 pmul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 pfma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

// face_flux constants for mu = 1 (a14 = a1 + a4, n* negated), kept as scalars: a paired FMA
// reads a scalar kernel parameter replicated into both halves straight from the constant bank,
// whereas a float2 parameter costs an extra instruction per use.
struct FaceKP {
  float a14, a2, a3, a5, a6, nq2, nq3, q5, b1, c1, c2, c3, c4, c5, c6, g0, nk3, half;
};
__device__ __forceinline__ f2 rep(float k) { return make_float2(k, k); }

inline FaceKP make_face_kp(const FaceK<float> &k) {
  FaceKP q;
  q.a14 = k.a1 + k.a4; q.a2 = k.a2; q.a3 = k.a3; q.a5 = k.a5; q.a6 = k.a6;
  q.nq2 = -k.q2; q.nq3 = -k.q3; q.q5 = k.q5; q.b1 = k.b1;
  q.c1 = k.c1; q.c2 = k.c2; q.c3 = k.c3; q.c4 = k.c4; q.c5 = k.c5; q.c6 = k.c6;
  q.g0 = k.g0; q.nk3 = -k.k3; q.half = 0.5f;
  return q;
}

// Two face sides (see FSide) with mu = 1.
struct FSideP {
  f2 e, hn, ht, den, dhn, dht, dat, det, eps;
};

// face_flux<float, false> for two faces at once.  The interface factor g multiplies two
// differences per flux; it is folded into their coefficients (g a3 + a6, g/2 - q3, g c3 + c6),
// and each sum is taken in two independent halves.
__device__ __forceinline__ void face_flux_p(const FSideP &l, const FSideP &r, const FaceKP &k,
                                            f2 &fE, f2 &fHn, f2 &fHt) {
  const f2 se = padd(l.eps, r.eps);
  const f2 ie = pk(rcp2(se.x), rcp2(se.y));
  const f2 g = pfma(rep(k.nk3), ie, rep(k.g0));
  const f2 cX = pfma(g, rep(k.a3), rep(k.a6));        // of D_xB in fE
  const f2 cU = pfma(g, rep(k.half), rep(k.nq3));     // of S_Uxe in fE and of S_UxB in fHt
  const f2 cD = pfma(g, rep(k.c3), rep(k.c6));        // of D_ex in fHt
  const f2 Ue_l = pmul(l.eps, l.e), Ue_r = pmul(r.eps, r.e);
  const f2 Uxe_l = pmul(l.eps, l.den), Uxe_r = pmul(r.eps, r.den);
  const f2 S_B = padd(l.ht, r.ht), D_e = psub(r.e, l.e);
  const f2 S_Uxe = padd(Uxe_l, Uxe_r), D_xB = psub(r.dht, l.dht);
  const f2 D_Ue = psub(Ue_r, Ue_l), D_At = psub(r.dat, l.dat);
  const f2 S_Uxa = padd(l.dhn, r.dhn), D_Ua = psub(r.hn, l.hn), D_Et = psub(r.det, l.det);
  const f2 S_Ue = padd(Ue_l, Ue_r), D_B = psub(r.ht, l.ht), S_UxB = padd(l.dht, r.dht);
  const f2 D_ex = psub(r.den, l.den), S_UAt = padd(l.dat, r.dat), S_e = padd(l.e, r.e);
  f2 fe1 = pfma(rep(k.a2), D_e, pmul(rep(k.a14), S_B));
  fe1 = pfma(rep(k.nq2), D_Ue, fe1);
  f2 fe2 = pfma(cX, D_xB, pmul(rep(k.a5), D_At));
  fe2 = pfma(cU, S_Uxe, fe2);
  f2 fa = pmul(rep(k.q5), S_Uxa);
  fa = pfma(rep(k.nq2), D_Ua, fa);
  fa = pfma(rep(k.b1), D_Et, fa);
  f2 u = pmul(rep(k.c1), S_Ue);
  u = pfma(rep(k.c2), D_B, u);
  u = pfma(rep(k.c4), S_UAt, u);
  const f2 fb1 = pfma(ie, u, pmul(rep(k.nq2), D_B));
  f2 fb2 = pfma(cD, D_ex, pmul(rep(k.c5), S_e));
  fb2 = pfma(cU, S_UxB, fb2);
  fE = padd(fe1, fe2);
  fHn = fa;
  fHt = padd(fb1, fb2);
}

// Two columns of one row as pairs, plus the PEC mirror flags (as in Row2).
struct RowP {
  f2 ez, hx, hy, eps;
  bool xm[2], ym;
};
// Raw differences of the two columns (component x: column X, y: column X+1).
struct GP {
  f2 ex, ey, ax, ay, bx, by;
};

__device__ __forceinline__ void apply_mirror_p(RowP &v) {
  if (v.ym | v.xm[0] | v.xm[1]) {
    if (v.xm[0] != v.ym) v.ez.x = -v.ez.x;
    if (v.xm[1] != v.ym) v.ez.y = -v.ez.y;
    if (v.xm[0]) v.hx.x = -v.hx.x;
    if (v.xm[1]) v.hx.y = -v.hx.y;
    if (v.ym) { v.hy.x = -v.hy.x; v.hy.y = -v.hy.y; }
  }
}

template <bool HAS_PEC>
__device__ __forceinline__ RowP load_row_p(const Cart2DKernelArgs<float> &p, int X, int row) {
  RowP v;
  const int r = axis_index(row, p.ny, p.pery, HAS_PEC && p.pec[2], HAS_PEC && p.pec[3], v.ym);
  v.xm[0] = v.xm[1] = false;
  const int64_t ro = (int64_t)r * p.pitch;
  if (X >= 0 && X + 1 < p.nx) {
    v.ez = __ldg(reinterpret_cast<const f2 *>(p.V + ro + X));
    v.hx = __ldg(reinterpret_cast<const f2 *>(p.V + p.cstride + ro + X));
    v.hy = __ldg(reinterpret_cast<const f2 *>(p.V + 2 * p.cstride + ro + X));
    v.eps = __ldg(reinterpret_cast<const f2 *>(p.eps + ro + X));
  } else {
    int64_t o[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
      o[k] = ro + axis_index(X + k, p.nx, p.perx, HAS_PEC && p.pec[0], HAS_PEC && p.pec[1],
                             v.xm[k]);
    v.ez = pk(__ldg(p.V + o[0]), __ldg(p.V + o[1]));
    v.hx = pk(__ldg(p.V + p.cstride + o[0]), __ldg(p.V + p.cstride + o[1]));
    v.hy = pk(__ldg(p.V + 2 * p.cstride + o[0]), __ldg(p.V + 2 * p.cstride + o[1]));
    v.eps = pk(__ldg(p.eps + o[0]), __ldg(p.eps + o[1]));
  }
  return v;
}

__device__ __forceinline__ RowV<float> col_of_p(const RowP &v, int k) {
  RowV<float> c;
  c.ez = k ? v.ez.y : v.ez.x; c.hx = k ? v.hx.y : v.hx.x; c.hy = k ? v.hy.y : v.hy.x;
  c.eps = k ? v.eps.y : v.eps.x; c.mu = 1.f;
  return c;
}
__device__ __forceinline__ RowG<float> grad_of_p(const GP &g, int k) {
  RowG<float> r;
  r.ex = k ? g.ex.y : g.ex.x; r.ey = k ? g.ey.y : g.ey.x; r.ax = k ? g.ax.y : g.ax.x;
  r.ay = k ? g.ay.y : g.ay.x; r.bx = k ? g.bx.y : g.bx.x; r.by = k ? g.by.y : g.by.x;
  return r;
}

// Raw differences of the lane's two columns (limited slopes with LIMIT); right[] receives
// column X+2 of this row.
template <bool LIMIT>
__device__ __forceinline__ void diffs_p(const RowP &c, const RowP &dn, const RowP &up, GP &g,
                                        float right[3]) {
  const float lE = __shfl_up_sync(FULL, c.ez.y, 1), rE = __shfl_down_sync(FULL, c.ez.x, 1);
  const float lA = __shfl_up_sync(FULL, c.hx.y, 1), rA = __shfl_down_sync(FULL, c.hx.x, 1);
  const float lB = __shfl_up_sync(FULL, c.hy.y, 1), rB = __shfl_down_sync(FULL, c.hy.x, 1);
  if (LIMIT) {
    g.ex = pk(raw_slope<true>(lE, c.ez.x, c.ez.y), raw_slope<true>(c.ez.x, c.ez.y, rE));
    g.ax = pk(raw_slope<true>(lA, c.hx.x, c.hx.y), raw_slope<true>(c.hx.x, c.hx.y, rA));
    g.bx = pk(raw_slope<true>(lB, c.hy.x, c.hy.y), raw_slope<true>(c.hy.x, c.hy.y, rB));
    g.ey = pk(raw_slope<true>(dn.ez.x, c.ez.x, up.ez.x), raw_slope<true>(dn.ez.y, c.ez.y, up.ez.y));
    g.ay = pk(raw_slope<true>(dn.hx.x, c.hx.x, up.hx.x), raw_slope<true>(dn.hx.y, c.hx.y, up.hx.y));
    g.by = pk(raw_slope<true>(dn.hy.x, c.hy.x, up.hy.x), raw_slope<true>(dn.hy.y, c.hy.y, up.hy.y));
  } else {
    g.ex = psub(pk(c.ez.y, rE), pk(lE, c.ez.x));
    g.ax = psub(pk(c.hx.y, rA), pk(lA, c.hx.x));
    g.bx = psub(pk(c.hy.y, rB), pk(lB, c.hy.x));
    g.ey = psub(up.ez, dn.ez);
    g.ay = psub(up.hx, dn.hx);
    g.by = psub(up.hy, dn.hy);
  }
  right[0] = rE; right[1] = rA; right[2] = rB;
}

struct Cart2DPackArgs {
  Cart2DKernelArgs<float> b;
  FaceKP fx, fy;
};

template <bool HAS_PEC, bool LIMIT>
__global__ void __launch_bounds__(WARPS * 32, GKS_CART2D_MINBLOCKS)
    cart2d_step_kernel_p(const Cart2DPackArgs P, int nstrips, int rows, int strip0, int ybeg,
                         int yend) {
  const Cart2DKernelArgs<float> &p = P.b;
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int strip = strip0 + wid % nstrips, chunk = wid / nstrips;
  const int y0 = ybeg + chunk * rows;
  if (y0 >= yend) return;                             // whole warp leaves together
  const int y1 = min(y0 + rows, yend);
  const int x0 = strip * WCOLS;
  const int X = x0 - 2 + 2 * lane;
  const int xend = min(x0 + WCOLS, p.nx);
  const bool xlo_nr = !p.perx && !p.pec[0], xhi_nr = !p.perx && !p.pec[1];
  const bool ylo_nr = !p.pery && !p.pec[2], yhi_nr = !p.pery && !p.pec[3];
  const float q4 = 0.25f, mq4 = -0.25f;
  const f2 Q4 = pk(q4, q4), MQ4 = pk(mq4, mq4);

  RowP vm2 = load_row_p<HAS_PEC>(p, X, y0 - 2);
  RowP vm1 = load_row_p<HAS_PEC>(p, X, y0 - 1);
  RowP v0 = load_row_p<HAS_PEC>(p, X, y0);
  RowP v1 = load_row_p<HAS_PEC>(p, X, y0 + 1);
  RowP v2 = load_row_p<HAS_PEC>(p, X, y0 + 2);
  RowP pf = load_row_p<HAS_PEC>(p, X, y0 + 3);
  if (HAS_PEC) {
    apply_mirror_p(vm2);
    apply_mirror_p(vm1);
    apply_mirror_p(v0);
    apply_mirror_p(v1);
    apply_mirror_p(v2);
  }
  GP g0, gm1;
  float r0[3], rm1[3];
  diffs_p<LIMIT>(vm1, vm2, v0, gm1, rm1);
  diffs_p<LIMIT>(v0, vm1, v1, g0, r0);
  // y-face sides of two columns: normal y (hn = Hy, ht = Hx, tangent x)
  auto yside = [](const RowP &v, const GP &g, f2 sgn) {
    FSideP s;
    s.e = pfma(sgn, g.ey, v.ez); s.hn = pfma(sgn, g.by, v.hy); s.ht = pfma(sgn, g.ay, v.hx);
    s.den = g.ey; s.dhn = g.by; s.dht = g.ay; s.dat = g.bx; s.det = g.ex;
    s.eps = v.eps;
    return s;
  };
  f2 fbE, fbHx, fbHy;                                 // flux along +y below row j
  face_flux_p(yside(vm1, gm1, Q4), yside(v0, g0, MQ4), P.fy, fbE, fbHy, fbHx);
  if (y0 == 0 && ylo_nr) {
    float e[2], hx[2], hy[2];
#pragma unroll
    for (int k = 0; k < 2; ++k)
      low_y_boundary_flux<float>(col_of_p(v0, k), grad_of_p(g0, k), p, e[k], hx[k], hy[k]);
    fbE = pk(e[0], e[1]); fbHx = pk(hx[0], hx[1]); fbHy = pk(hy[0], hy[1]);
  }
  bool bad = false;
#pragma unroll 1
  for (int j = y0; j < y1; ++j) {
    const RowP pf2 = load_row_p<HAS_PEC>(p, X, j + 4);   // two rows ahead of use
    GP g1;
    float r1[3];
    diffs_p<LIMIT>(v1, v0, v2, g1, r1);
    // x-faces of row j: X+1/2 (component x) and X+3/2 (component y, column X+2 of the next
    // lane on its right side)
    f2 fxE, fxHx, fxHy;
    {
      const float nb_eps = __shfl_down_sync(FULL, v0.eps.x, 1);
      const float gn_ex = __shfl_down_sync(FULL, g0.ex.x, 1);
      const float gn_ax = __shfl_down_sync(FULL, g0.ax.x, 1);
      const float gn_bx = __shfl_down_sync(FULL, g0.bx.x, 1);
      const float gn_ay = __shfl_down_sync(FULL, g0.ay.x, 1);
      const float gn_ey = __shfl_down_sync(FULL, g0.ey.x, 1);
      FSideP l, r;
      l.e = pfma(Q4, g0.ex, v0.ez); l.hn = pfma(Q4, g0.ax, v0.hx); l.ht = pfma(Q4, g0.bx, v0.hy);
      l.den = g0.ex; l.dhn = g0.ax; l.dht = g0.bx; l.dat = g0.ay; l.det = g0.ey;
      l.eps = v0.eps;
      r.den = pk(g0.ex.y, gn_ex); r.dhn = pk(g0.ax.y, gn_ax); r.dht = pk(g0.bx.y, gn_bx);
      r.dat = pk(g0.ay.y, gn_ay); r.det = pk(g0.ey.y, gn_ey);
      r.e = pfma(MQ4, r.den, pk(v0.ez.y, r0[0]));
      r.hn = pfma(MQ4, r.dhn, pk(v0.hx.y, r0[1]));
      r.ht = pfma(MQ4, r.dht, pk(v0.hy.y, r0[2]));
      r.eps = pk(v0.eps.y, nb_eps);
      face_flux_p(l, r, P.fx, fxE, fxHx, fxHy);
      if (xhi_nr) {
        if (X == p.nx - 1) {            // first face on the high-x boundary
          const Side<float> q = xside_scalar<float>(col_of_p(v0, 0), grad_of_p(g0, 0), q4,
                                                    p.inv2hx, p.inv2hy);
          tm_face_flux<float, true>(q, q, p.Kx, fxE.x, fxHx.x, fxHy.x);
        }
        if (X + 1 == p.nx - 1) {        // second face on the high-x boundary
          const Side<float> q = xside_scalar<float>(col_of_p(v0, 1), grad_of_p(g0, 1), q4,
                                                    p.inv2hx, p.inv2hy);
          tm_face_flux<float, true>(q, q, p.Kx, fxE.y, fxHx.y, fxHy.y);
        }
      }
      if (xlo_nr && X == -2) {          // second face is the low-x boundary face of column 0
        RowV<float> nb;
        nb.ez = r0[0]; nb.hx = r0[1]; nb.hy = r0[2]; nb.eps = nb_eps; nb.mu = 1.f;
        RowG<float> gn;
        gn.ex = gn_ex; gn.ax = gn_ax; gn.bx = gn_bx; gn.ay = gn_ay; gn.ey = gn_ey; gn.by = 0.f;
        low_boundary_flux<float>(xside_scalar<float>(nb, gn, mq4, p.inv2hx, p.inv2hy), p.Kx,
                                 fxE.y, fxHx.y, fxHy.y);
      }
    }
    // y-faces between rows j and j+1
    f2 ftE, ftHx, ftHy;
    face_flux_p(yside(v0, g0, Q4), yside(v1, g1, MQ4), P.fy, ftE, ftHy, ftHx);
    if (j + 1 == p.ny && yhi_nr) {
      float e[2], hx[2], hy[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const Side<float> q = yside_scalar<float>(col_of_p(v0, k), grad_of_p(g0, k), q4,
                                                  p.inv2hx, p.inv2hy);
        float oe, oa, ob;
        tm_face_flux<float, true>(q, q, p.Ky, oe, oa, ob);
        e[k] = oe; hx[k] = -ob; hy[k] = oa;
      }
      ftE = pk(e[0], e[1]); ftHx = pk(hx[0], hx[1]); ftHy = pk(hy[0], hy[1]);
    }
    // update row j: left face of column X is the previous lane's second face
    {
      const float lE = __shfl_up_sync(FULL, fxE.y, 1);
      const float lHx = __shfl_up_sync(FULL, fxHx.y, 1);
      const float lHy = __shfl_up_sync(FULL, fxHy.y, 1);
      f2 dE = padd(psub(pk(lE, fxE.x), fxE), psub(fbE, ftE));
      const f2 dHx = padd(psub(pk(lHx, fxHx.x), fxHx), psub(fbHx, ftHx));
      const f2 dHy = padd(psub(pk(lHy, fxHy.x), fxHy), psub(fbHy, ftHy));
      const int64_t ro = (int64_t)j * p.pitch;
      if (p.src && j >= p.sy0 && j < p.sy1) {
        if (X >= p.sx0 && X < p.sx1) dE.x -= p.src_amp * p.src[ro + X];
        if (X + 1 >= p.sx0 && X + 1 < p.sx1) dE.y -= p.src_amp * p.src[ro + X + 1];
      }
      const f2 ne = pfma(dE, pk(rcp1(v0.eps.x), rcp1(v0.eps.y)), v0.ez);
      const f2 nhx = padd(v0.hx, dHx);
      const f2 nhy = padd(v0.hy, dHy);
      const bool ok0 = X >= x0 && X < xend, ok1 = X + 1 >= x0 && X + 1 < xend;
      if (ok0 && ok1) {
        *reinterpret_cast<f2 *>(p.Vout + ro + X) = ne;
        *reinterpret_cast<f2 *>(p.Vout + p.cstride + ro + X) = nhx;
        *reinterpret_cast<f2 *>(p.Vout + 2 * p.cstride + ro + X) = nhy;
        const f2 sum = padd(padd(ne, nhx), nhy);
        bad |= !(isfinite(sum.x) && isfinite(sum.y));
      } else {
        if (ok0) {
          p.Vout[ro + X] = ne.x;
          p.Vout[p.cstride + ro + X] = nhx.x;
          p.Vout[2 * p.cstride + ro + X] = nhy.x;
          bad |= !(isfinite(ne.x) && isfinite(nhx.x) && isfinite(nhy.x));
        }
        if (ok1) {
          p.Vout[ro + X + 1] = ne.y;
          p.Vout[p.cstride + ro + X + 1] = nhx.y;
          p.Vout[2 * p.cstride + ro + X + 1] = nhy.y;
          bad |= !(isfinite(ne.y) && isfinite(nhx.y) && isfinite(nhy.y));
        }
      }
    }
    // rotate the register window
    v0 = v1; v1 = v2; v2 = pf; pf = pf2;
    if (HAS_PEC) apply_mirror_p(v2);          // the prefetched row takes its mirror signs now
    g0 = g1;
    fbE = ftE; fbHx = ftHx; fbHy = ftHy;
    r0[0] = r1[0]; r0[1] = r1[1]; r0[2] = r1[2];
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(p.flag, 1);
}

// ------------------------------------------------------------------ staged FP32 path
// FP32, mu = 1, no limiter, x not periodic (non-reflecting or PEC sides).  The rows of a strip
// are staged in shared memory by TMA and the two cells of a lane lie 32 columns apart, so that no
// pair ever has to be assembled from two lanes' registers:
//   - a warp owns a strip of W2 = 63 columns x0 .. x0+62; lane l holds the cells A = x0+l and
//     B = x0+32+l as the two halves of a float2 (lane 31's B is the next strip's first column,
//     computed but not stored);
//   - each lane evaluates the LEFT x-faces of A and B.  The 64 faces x0-1/2 .. x0+62+1/2 of the
//     warp are exactly the faces its 63 cells need; a cell's right face is the next lane's
//     left face (a shuffle; for lane 31's A it is lane 0's left face of B);
//   - every value a lane needs (its own cells, the left neighbours A-1, B-1 and their
//     left neighbours, the right neighbours, the rows above and below) is read from the staged
//     rows, two 4-byte shared loads per pair.  Gradients of the left neighbours are recomputed
//     from the staged rows rather than shuffled, so no lane is special;
//   - updated cells go straight to global memory (coalesced 4-byte stores).
// Each warp keeps a ring of NSLOT2 rows (Ez, Hx, Hy as one 3-D box and eps as a 2-D box, one
// mbarrier per row; the box starts at the 16-byte boundary at or below x0-3).  Lane 0 issues
// row j+NSLOT2-1 once row j is done; iteration j reads rows j-1 .. j+2.  Rows past a
// non-reflecting y side are staged from the clamped row (the Green-Gauss ghost copy), a
// periodic y side wraps; columns past a non-reflecting x side are read from the clamped column,
// so the zero-filled entries of a box are never read.  On PEC sides the rows and columns past the
// wall hold mirror images (fix_row).  The march is unrolled by two so that the
// gradients and face-below fluxes alternate between two register sets.
constexpr int W2 = 63;                  // columns updated per warp
constexpr int TW2 = 72;                 // staged columns (x0-3 rounded down to 4, +72)
constexpr int NSLOT2 = 8;               // staged rows per warp
static_assert((NSLOT2 & (NSLOT2 - 1)) == 0, "the ring index masks with NSLOT2 - 1");
constexpr int MINB2 = 4;                // CTAs per SM the register budget allows
struct alignas(128) RowBox2 { float a[3][TW2]; };     // Ez, Hx, Hy
struct alignas(128) EpsBox2 { float e[TW2]; };
struct StagedRow2 { RowBox2 v; EpsBox2 e; };
struct WarpStage2 {
  StagedRow2 row[NSLOT2];
  unsigned long long bar[NSLOT2];
};
constexpr unsigned kRowBytes2 = 4 * TW2 * 4;           // both boxes of one staged row

// Staged columns of a lane's two cells and of their neighbours at offsets -2 .. +1, clamped to
// the grid (non-reflecting x sides).
struct Taps2 {
  int a[4], b[4];       // [k]: column A + k - 2 / B + k - 2
};

// (Ez, Hx, Hy, eps) of the pair at tap k of a staged row; 3 fields only with EPS = false.
template <bool EPS>
__device__ __forceinline__ RowP staged_pair(const StagedRow2 &R, const Taps2 &q, int k) {
  RowP v;
  v.ez = pk(R.v.a[0][q.a[k]], R.v.a[0][q.b[k]]);
  v.hx = pk(R.v.a[1][q.a[k]], R.v.a[1][q.b[k]]);
  v.hy = pk(R.v.a[2][q.a[k]], R.v.a[2][q.b[k]]);
  v.eps = EPS ? pk(R.e.e[q.a[k]], R.e.e[q.b[k]]) : pk(0.f, 0.f);
  v.xm[0] = v.xm[1] = v.ym = false;
  return v;
}

// Raw central differences of the pair at tap k of row `mid` (rows `dn` and `up` below and
// above): x differences of (Ez, Hx, Hy) from taps k-1 and k+1, y differences from the rows.
__device__ __forceinline__ GP staged_diffs(const StagedRow2 &dn, const StagedRow2 &mid,
                                           const StagedRow2 &up, const Taps2 &q, int k) {
  GP g;
  const RowP l = staged_pair<false>(mid, q, k - 1), r = staged_pair<false>(mid, q, k + 1);
  const RowP d = staged_pair<false>(dn, q, k), u = staged_pair<false>(up, q, k);
  g.ex = psub(r.ez, l.ez); g.ax = psub(r.hx, l.hx); g.bx = psub(r.hy, l.hy);
  g.ey = psub(u.ez, d.ez); g.ay = psub(u.hx, d.hx); g.by = psub(u.hy, d.hy);
  return g;
}

// HAS_PEC: some side is a PEC wall (the mirror-image bookkeeping is compiled in only then).
template <bool HAS_PEC>
__global__ void __launch_bounds__(WARPS * 32, MINB2)
    cart2d_step_kernel_s(const __grid_constant__ CUtensorMap tmV,
                         const __grid_constant__ CUtensorMap tmE, const Cart2DPackArgs P,
                         int nstrips, int rows, int strip0, int ybeg, int yend) {
  extern __shared__ __align__(128) unsigned char smem_s[];
  const Cart2DKernelArgs<float> &p = P.b;
  const int lane = threadIdx.x & 31;
  WarpStage2 &w = reinterpret_cast<WarpStage2 *>(smem_s)[threadIdx.x >> 5];
  const int wid = blockIdx.x * WARPS + (threadIdx.x >> 5);
  const int strip = strip0 + wid % nstrips, chunk = wid / nstrips;
  const int y0 = ybeg + chunk * rows;
  if (y0 >= yend) return;                             // whole warp leaves together
  const int y1 = min(y0 + rows, yend);
  const int x0 = strip * W2;
  const int xs = (x0 - 3) & ~3;                       // first staged column (16-byte aligned)
  const int A = x0 + lane, B = x0 + 32 + lane;
  const bool pxl = HAS_PEC && p.pec[0], pxh = HAS_PEC && p.pec[1];
  const bool pyl = HAS_PEC && p.pec[2], pyh = HAS_PEC && p.pec[3];
  const bool ylo_nr = !p.pery && !pyl, yhi_nr = !p.pery && !pyh;
  const float q4 = 0.25f, mq4 = -0.25f;
  const f2 Q4 = pk(q4, q4), MQ4 = pk(mq4, mq4), Z2 = pk(0.f, 0.f);
  // staged column read for grid column c: a non-reflecting side clamps to the edge cell (the
  // Green-Gauss ghost copy); a PEC side reads its two mirror-image columns, which fix_row writes
  // into the staged row, and nothing further out
  auto tap = [&p, pxl, pxh, xs](int c) {
    c = c < 0 ? (pxl ? max(c, -2) : 0) : c;
    c = c >= p.nx ? (pxh ? min(c, p.nx + 1) : p.nx - 1) : c;
    return c - xs;
  };
  Taps2 q;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    q.a[k] = tap(A + k - 2);
    q.b[k] = tap(B + k - 2);
  }
  // boundary x faces (scalar flux) on non-reflecting sides: the left face of column 0 is the
  // low-x face of column 0; the left face of column nx is the high-x face of column nx - 1.
  // PEC wall faces are interior faces against the mirror-image columns.
  const bool loA = !pxl && A == 0, loB = !pxl && B == 0;
  const bool hiA = !pxh && A == p.nx, hiB = !pxh && B == p.nx;
  const bool xedge = __any_sync(FULL, loA || loB || hiA || hiB);
  // PEC x walls: lane g < 4 writes ghost column gc = (-2, -1, nx, nx+1)[g] of each staged row from
  // its mirror column (Ez and Hx negated), if the warp stages that column
  int gcol = lane == 0 ? -2 : lane == 1 ? -1 : lane == 2 ? p.nx : p.nx + 1;
  const int gmir = lane < 2 ? min(-1 - gcol, p.nx - 1) : max(2 * p.nx - 1 - gcol, 0);
  const bool gact = lane < 4 && (lane < 2 ? pxl : pxh) && gcol - xs >= 0 && gcol - xs < TW2;
  const bool xfix = HAS_PEC && __any_sync(FULL, gact);
  const int xend = min(x0 + W2, p.nx);
  const bool stA = A < xend, stB = lane < 31 && B < xend;   // cells this lane stores

  const int first = y0 - 2, last = y1 + 1;            // staged rows
  auto slot = [first](int r) { return (r - first) & (NSLOT2 - 1); };
  auto parity = [first](int r) { return (unsigned)(((r - first) / NSLOT2) & 1); };
  auto grid_row = [&p, pyl, pyh](int r) {
    if (p.pery) return r < 0 ? r + p.ny : (r >= p.ny ? r - p.ny : r);
    if (r < 0) return pyl ? min(-1 - r, p.ny - 1) : 0;
    if (r >= p.ny) return pyh ? max(2 * p.ny - 1 - r, 0) : p.ny - 1;
    return r;
  };
  // mirror images on PEC walls, written into a staged row once it has landed (whole warp): a row
  // past a PEC y wall negates Ez and Hy; then the ghost columns past a PEC x wall take their
  // mirror columns with Ez and Hx negated (corner ghosts get both)
  auto fix_row = [&](int r) {
    if constexpr (!HAS_PEC) return;
    const bool yg = (r < 0 && pyl) || (r >= p.ny && pyh);
    if (!yg && !xfix) return;
    StagedRow2 &R = w.row[slot(r)];
    if (yg)
      for (int c = lane; c < TW2; c += 32) {
        R.v.a[0][c] = -R.v.a[0][c];
        R.v.a[2][c] = -R.v.a[2][c];
      }
    __syncwarp();
    if (gact) {
      const int t = gcol - xs, m = gmir - xs;
      R.v.a[0][t] = -R.v.a[0][m];
      R.v.a[1][t] = -R.v.a[1][m];
      R.v.a[2][t] = R.v.a[2][m];
      R.e.e[t] = R.e.e[m];
    }
    __syncwarp();
  };
  int issued = first - 1;                             // lane 0: the last row whose copy is issued
  auto issue = [&](int r) {                           // lane 0 only
    const int s_ = slot(r), gr = grid_row(r);
    fence_proxy_async();
    mbar_expect_tx(&w.bar[s_], kRowBytes2);
    tma_load_3d(&w.row[s_].v.a[0][0], &tmV, xs, gr, 0, &w.bar[s_]);
    tma_load_2d(&w.row[s_].e.e[0], &tmE, xs, gr, &w.bar[s_]);
    issued = r;
  };
  auto wait_row = [&](int r) {                        // the whole warp; false if it ran out
    return __all_sync(FULL, mbar_wait(&w.bar[slot(r)], parity(r)));
  };
  if (lane == 0) {
    for (int i = 0; i < NSLOT2; ++i) mbar_init(&w.bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    for (int r = first; r <= min(last, first + NSLOT2 - 1); ++r) issue(r);
  }
  __syncwarp();

  auto yside = [](const RowP &v, const GP &g, f2 sgn) {
    FSideP s;
    s.e = pfma(sgn, g.ey, v.ez); s.hn = pfma(sgn, g.by, v.hy); s.ht = pfma(sgn, g.ay, v.hx);
    s.den = g.ey; s.dhn = g.by; s.dht = g.ay; s.dat = g.bx; s.det = g.ex;
    s.eps = v.eps;
    return s;
  };
  auto xside = [](const RowP &v, const GP &g, f2 sgn) {
    FSideP s;
    s.e = pfma(sgn, g.ex, v.ez); s.hn = pfma(sgn, g.ax, v.hx); s.ht = pfma(sgn, g.bx, v.hy);
    s.den = g.ex; s.dhn = g.ax; s.dht = g.bx; s.dat = g.ay; s.det = g.ey;
    s.eps = v.eps;
    return s;
  };

  bool ok = true;
  for (int r = first; r <= y0 + 1; ++r) {
    ok = ok && wait_row(r);
    if (ok) fix_row(r);
  }
  GP g0, g1;                                          // own gradients of the current / next row
  f2 fbE, fbHx, fbHy, ftE, ftHx, ftHy;                // y-face fluxes below / above the row
  if (ok) {
    const StagedRow2 &Rm2 = w.row[slot(y0 - 2)], &Rm1 = w.row[slot(y0 - 1)];
    const StagedRow2 &R0 = w.row[slot(y0)], &R1 = w.row[slot(y0 + 1)];
    const GP gm1 = staged_diffs(Rm2, Rm1, R0, q, 2);
    g0 = staged_diffs(Rm1, R0, R1, q, 2);
    const RowP vm1 = staged_pair<true>(Rm1, q, 2), v0 = staged_pair<true>(R0, q, 2);
    face_flux_p(yside(vm1, gm1, Q4), yside(v0, g0, MQ4), P.fy, fbE, fbHy, fbHx);
    if (y0 == 0 && ylo_nr) {
      float e[2], hx[2], hy[2];
#pragma unroll
      for (int k = 0; k < 2; ++k)
        low_y_boundary_flux<float>(col_of_p(v0, k), grad_of_p(g0, k), p, e[k], hx[k], hy[k]);
      fbE = pk(e[0], e[1]); fbHx = pk(hx[0], hx[1]); fbHy = pk(hy[0], hy[1]);
    }
    __syncwarp();                                     // row y0-2 is read
    if (lane == 0 && first + NSLOT2 <= last) issue(first + NSLOT2);
  }
  f2 acc = Z2;                                        // 0 * (updated values): NaN iff one is not finite

  // one row: own gradients of row j+1 into gn, the y-face above row j into t*, row j updated
  // with the y-face below b*
  auto row = [&](int j, const GP &gc, GP &gn, f2 bE, f2 bHx, f2 bHy, f2 &tE, f2 &tHx,
                 f2 &tHy) -> bool {
    if (!wait_row(j + 2)) return false;
    fix_row(j + 2);
    const StagedRow2 &Rm = w.row[slot(j - 1)], &R0 = w.row[slot(j)];
    const StagedRow2 &R1 = w.row[slot(j + 1)], &R2 = w.row[slot(j + 2)];
    gn = staged_diffs(R0, R1, R2, q, 2);
    const RowP v0 = staged_pair<true>(R0, q, 2), v1 = staged_pair<true>(R1, q, 2);
    // left x-faces of A and B: l side the left neighbours (their gradients recomputed from the
    // staged rows), r side the lane's own cells
    const RowP vl = staged_pair<true>(R0, q, 1);
    const GP gl = staged_diffs(Rm, R0, R1, q, 1);
    f2 fxE, fxHx, fxHy;
    face_flux_p(xside(vl, gl, Q4), xside(v0, gc, MQ4), P.fx, fxE, fxHx, fxHy);
    if (xedge) {
      if (loA)                          // low-x face of column 0 (cell A)
        low_boundary_flux<float>(xside_scalar<float>(col_of_p(v0, 0), grad_of_p(gc, 0), mq4,
                                                     p.inv2hx, p.inv2hy),
                                 p.Kx, fxE.x, fxHx.x, fxHy.x);
      if (hiA) {                        // high-x face of column nx - 1 (left neighbour of A)
        const Side<float> s_ = xside_scalar<float>(col_of_p(vl, 0), grad_of_p(gl, 0), q4,
                                                   p.inv2hx, p.inv2hy);
        tm_face_flux<float, true>(s_, s_, p.Kx, fxE.x, fxHx.x, fxHy.x);
      }
      if (hiB) {                        // the same for B
        const Side<float> s_ = xside_scalar<float>(col_of_p(vl, 1), grad_of_p(gl, 1), q4,
                                                   p.inv2hx, p.inv2hy);
        tm_face_flux<float, true>(s_, s_, p.Kx, fxE.y, fxHx.y, fxHy.y);
      }
    }
    // right faces: the next lane's left faces; for lane 31's A, lane 0's left face of B
    auto right = [lane](f2 f) {
      const float a = __shfl_down_sync(FULL, f.x, 1), b = __shfl_sync(FULL, f.y, 0);
      const float c = __shfl_down_sync(FULL, f.y, 1);
      return pk(lane == 31 ? b : a, c);
    };
    const f2 frE = right(fxE), frHx = right(fxHx), frHy = right(fxHy);
    // y-faces between rows j and j+1
    face_flux_p(yside(v0, gc, Q4), yside(v1, gn, MQ4), P.fy, tE, tHy, tHx);
    if (j + 1 == p.ny && yhi_nr) {
      float e[2], hx[2], hy[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const Side<float> s_ = yside_scalar<float>(col_of_p(v0, k), grad_of_p(gc, k), q4,
                                                   p.inv2hx, p.inv2hy);
        float oe, oa, ob;
        tm_face_flux<float, true>(s_, s_, p.Ky, oe, oa, ob);
        e[k] = oe; hx[k] = -ob; hy[k] = oa;
      }
      tE = pk(e[0], e[1]); tHx = pk(hx[0], hx[1]); tHy = pk(hy[0], hy[1]);
    }
    // update row j
    f2 dE = padd(psub(fxE, frE), psub(bE, tE));
    const f2 dHx = padd(psub(fxHx, frHx), psub(bHx, tHx));
    const f2 dHy = padd(psub(fxHy, frHy), psub(bHy, tHy));
    const int64_t ro = (int64_t)j * p.pitch;
    if (p.src && j >= p.sy0 && j < p.sy1) {
      if (A >= p.sx0 && A < p.sx1) dE.x -= p.src_amp * p.src[ro + A];
      if (B >= p.sx0 && B < p.sx1) dE.y -= p.src_amp * p.src[ro + B];
    }
    const f2 ne = pfma(dE, pk(rcp1(v0.eps.x), rcp1(v0.eps.y)), v0.ez);
    const f2 nhx = padd(v0.hx, dHx);
    const f2 nhy = padd(v0.hy, dHy);
    float *o = p.Vout + ro;
    if (stA) {
      o[A] = ne.x; o[p.cstride + A] = nhx.x; o[2 * p.cstride + A] = nhy.x;
    }
    if (stB) {
      o[B] = ne.y; o[p.cstride + B] = nhx.y; o[2 * p.cstride + B] = nhy.y;
    }
    const f2 sum = padd(padd(ne, nhx), nhy);
    if (stB) acc = pfma(sum, Z2, acc);                 // stB implies stA
    else if (stA) acc.x = fmaf(sum.x, 0.f, acc.x);
    __syncwarp();                                     // row j-1 is read
    if (lane == 0 && j + NSLOT2 - 1 <= last) issue(j + NSLOT2 - 1);
    return true;
  };

  int j = y0;
  if (ok) {
#pragma unroll 1
    for (; j + 1 < y1; j += 2) {
      if (!row(j, g0, g1, fbE, fbHx, fbHy, ftE, ftHx, ftHy) ||
          !row(j + 1, g1, g0, ftE, ftHx, ftHy, fbE, fbHx, fbHy)) {
        ok = false;
        break;
      }
    }
    if (ok && j < y1) ok = row(j, g0, g1, fbE, fbHx, fbHy, ftE, ftHx, ftHy);
  }
  if (lane == 0 && !ok) {
    atomicOr(p.flag, 2);                              // a row never landed
    for (int r = max(first, issued - NSLOT2 + 1); r <= issued; ++r)   // copies in flight
      mbar_wait(&w.bar[slot(r)], parity(r));
  }
  if (__any_sync(FULL, !(isfinite(acc.x) && isfinite(acc.y))) && lane == 0) atomicOr(p.flag, 1);
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

// The staged kernel covers FP32 with mu = 1, no limiter and a non-periodic x axis (a periodic
// y axis needs two rows for the wrap); non-reflecting and PEC sides.
bool staged2_supported(const CartGeom &g, const CartStepArgs &a) {
  if (a.mu || a.limiter || g.periodic[0]) return false;
  if (g.periodic[1] && g.ny < 2) return false;
  return tensor_map_encoder() != nullptr;
}

// Staged launch over the window's columns [wx0, wx1) (strips of W2 columns) and rows [wy0, wy1):
// about four waves of warps (each marching a chunk of at least 8 rows of one strip), so that the
// CTA scheduler evens out the SMs' progress; one wave of long chunks ran 11% slower on the
// 4096^2 grid.
constexpr int kWaves2 = 4;
cudaError_t launch_staged2(const CartGeom &g, const Cart2DPackArgs &P, int wx0, int wx1, int wy0,
                           int wy1, cudaStream_t st) {
  const int smem = WARPS * (int)sizeof(WarpStage2);
  static int per_sm = 0, sms = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(cart2d_step_kernel_s<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    cudaFuncSetAttribute(cart2d_step_kernel_s<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cart2d_step_kernel_s<false>, WARPS * 32,
                                                  smem);
    if (sms < 1) sms = 1;
    if (per_sm < 1) per_sm = 1;
  }
  const int strip0 = wx0 / W2;
  const int nstrips = (wx1 - 1) / W2 - strip0 + 1;
  const int64_t resident = (int64_t)sms * per_sm * WARPS;
  const int wrows = wy1 - wy0;
  const int64_t want = resident * kWaves2 / nstrips;
  int nchunks = (int)(want > 1 ? want : 1);
  int rows = (wrows + nchunks - 1) / nchunks;
  if (rows < 8) rows = 8;
  nchunks = (wrows + rows - 1) / rows;
  const int64_t nwarps = (int64_t)nstrips * nchunks;
  const int grid = (int)((nwarps + WARPS - 1) / WARPS);
  CUtensorMap tmV, tmE;
  const cuuint64_t dim[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 3};
  const cuuint64_t stride[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.cstride * 4};
  const cuuint32_t box[3] = {TW2, 1, 3};
  if (!encode_f32_map(&tmV, P.b.V, 3, dim, stride, box) ||
      !encode_f32_map(&tmE, P.b.eps, 2, dim, stride, box))
    return cudaErrorInvalidValue;
  const bool pec = g.pec[0] || g.pec[1] || g.pec[2] || g.pec[3];
  auto kern = pec ? cart2d_step_kernel_s<true> : cart2d_step_kernel_s<false>;
  kern<<<grid, WARPS * 32, smem, st>>>(tmV, tmE, P, nstrips, rows, strip0, wy0, wy1);
  return cudaGetLastError();
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
  for (int k = 0; k < 4; ++k) p.pec[k] = g.pec[k];
  p.inv2hx = T(0.5 / g.h[0]); p.inv2hy = T(0.5 / g.h[1]);
  p.fx = make_face_k<T>(a.C, g.h[0], g.h[1], a.c, 1.0, 1.0);
  p.fy = make_face_k<T>(a.C, g.h[1], g.h[0], a.c, -1.0, -1.0);
  p.Kx = make_coef<T>(a.C, g.h[0], a.c);
  p.Ky = make_coef<T>(a.C, g.h[1], a.c);
  p.flag = a.flag;
  // window (the whole grid unless a sub-rectangle is asked for): strips covering its columns
  const int wx0 = a.window[0], wx1 = a.window[1], wy0 = a.window[2], wy1 = a.window[3];
  const int strip0 = wx0 / WCOLS;
  const int nstrips = (wx1 - 1) / WCOLS - strip0 + 1;
  const int wrows = wy1 - wy0;
  // rows per warp: enough warps to fill the GPU (about 24 resident per SM), 4 to 256 rows (a
  // warp spends about two rows of work on its prologue, so small windows take short chunks)
  int rows = wrows;
  const int target = 152 * 24;
  if (nstrips < target) {
    const int chunks = (target + nstrips - 1) / nstrips;
    rows = (wrows + chunks - 1) / chunks;
  }
  rows = rows < 4 ? 4 : (rows > 256 ? 256 : rows);
  const int nchunks = (wrows + rows - 1) / rows;
  const int64_t nwarps = (int64_t)nstrips * nchunks;
  const int grid = (int)((nwarps + WARPS - 1) / WARPS);
  // PEC walls and the limiter get their own instantiations: without them the mirror
  // bookkeeping and the limiter fold away
  const bool pec = g.pec[0] || g.pec[1] || g.pec[2] || g.pec[3];
  using K = void (*)(const Cart2DKernelArgs<T>, int, int, int, int, int);
  static const K kern[2][2][2] = {   // [mu][pec][limiter]
      {{cart2d_step_kernel<T, false, false, false>, cart2d_step_kernel<T, false, false, true>},
       {cart2d_step_kernel<T, false, true, false>, cart2d_step_kernel<T, false, true, true>}},
      {{cart2d_step_kernel<T, true, false, false>, cart2d_step_kernel<T, true, false, true>},
       {cart2d_step_kernel<T, true, true, false>, cart2d_step_kernel<T, true, true, true>}}};
  if constexpr (sizeof(T) == 4) {
    if (!a.mu) {                       // FP32 with mu = 1: the paired-instruction kernel
      Cart2DPackArgs P;
      P.b = p;
      P.fx = make_face_kp(p.fx);
      P.fy = make_face_kp(p.fy);
      if (staged2_supported(g, a)) return launch_staged2(g, P, wx0, wx1, wy0, wy1, st);
      using KP = void (*)(const Cart2DPackArgs, int, int, int, int, int);
      static const KP kp[2][2] = {{cart2d_step_kernel_p<false, false>,
                                   cart2d_step_kernel_p<false, true>},
                                  {cart2d_step_kernel_p<true, false>,
                                   cart2d_step_kernel_p<true, true>}};   // [pec][limiter]
      kp[pec ? 1 : 0][a.limiter ? 1 : 0]<<<grid, WARPS * 32, 0, st>>>(P, nstrips, rows, strip0,
                                                                       wy0, wy1);
      return cudaGetLastError();
    }
  }
  kern[a.mu ? 1 : 0][pec ? 1 : 0][a.limiter ? 1 : 0]<<<grid, WARPS * 32, 0, st>>>(
      p, nstrips, rows, strip0, wy0, wy1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cart2d_step(const CartGeom &g, const CartStepArgs &a, bool fp64,
                               cudaStream_t st) {
  return fp64 ? launch_t<double>(g, a, st) : launch_t<float>(g, a, st);
}

}  // namespace gks
