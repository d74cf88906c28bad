// Fused 2-D TM GKS step on a Cartesian grid: cell gradients, face reconstruction, the GKS
// interface flux and the finite-volume update in one pass over the state (Sec. 3.1).
//
// Row-marching scheme.  A CTA of NT threads owns a strip of W = 2 NT - 4 columns and a chunk of
// rows, and walks up the rows with one barrier per row.  Thread t owns the column pair
// (X, X+1), X = x0 - 2 + 2t, and keeps its own columns of the state, eps, gradients and the
// y-face flux in registers; shared memory holds the current rows only for the x-neighbours.
// Every gradient and every face is evaluated once: per row a thread evaluates the gradient pair
// of row j+1, the x-face pair (X+1/2, X+3/2) and the y-face pair (j+1/2) and updates its two
// cells of row j.  FP32 pairs run on the packed FP32x2 pipe (FFMA2 / FADD2 / FMUL2).
//
// Face frames (Sec. 3.1, T'(n)): an x-face uses n = e_x (T' = I); a y-face n = e_y with local
// axes (x', y') = (y, -x); the low boundary faces use the outward normals -e_x (T' =
// diag(-1,-1,1)) and -e_y (local (x', y') = (-y, x)).  In 2-D TM the third-moment term of the
// D3Q4 flux vanishes, so a TM face flux does not depend on the tangential orientation.
#include <cuda_runtime.h>

#include "gks_internal.h"

namespace gks {
namespace {

constexpr int NT = 64;             // threads per CTA
constexpr int W = 2 * NT - 4;      // columns updated per CTA
constexpr int NCOL = 2 * NT + 2;   // staged columns: x0-3 .. x0+W+2
constexpr int ROWS = 64;           // rows per CTA

// ------------------------------------------------------------------ pair arithmetic
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vbc(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 vrcp(float2 a) {
  return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y));
}
__device__ __forceinline__ float2 vmk(float a, float b) { return make_float2(a, b); }

__device__ __forceinline__ double2 vadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 vmul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 vfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 vbc(double s) { return make_double2(s, s); }
__device__ __forceinline__ double2 vrcp(double2 a) { return make_double2(1.0 / a.x, 1.0 / a.y); }
__device__ __forceinline__ double2 vmk(double a, double b) { return make_double2(a, b); }

template <typename T> struct PairOf;
template <> struct PairOf<float> { using type = float2; };
template <> struct PairOf<double> { using type = double2; };

// ------------------------------------------------------------------ flux coefficients
// Combined constants of one face orientation (K_i = C_i / h_normal, c the lattice speed,
// sb / st the signs of the tangential H component and of the tangential derivative in the face
// frame): see face_pair() for how they enter.
template <typename T>
struct FaceK {
  T a1, a2, a3, a4, a5, a6;   // E flux
  T q2, q3, q5, b1;           // normal-H flux (q2, q3 shared)
  T c1, c2, c3, c4, c5, c6;   // tangential-H flux
  T g0, k3;                   // g = g0 - k3 / (eps_s mu_s)
};

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

// One side of an interior face pair in global components: e = Ez, hn = normal H, ht =
// tangential H (reconstructed at the face), their normal derivatives en, hnn, htn, the
// tangential derivatives at = d_t(hn), et = d_t(Ez), and the material.
template <typename P>
struct PSide {
  P e, hn, ht, en, hnn, htn, at, et, eps, mu;
};

// Interior face flux for a pair of faces (times dt/h), in global components:
//   Phi_E  = im (a1 S_UB + a2 D_e) + g (S_Uxe/2 + a3 D_xB) + a4 S_B - q2 D_Ue - q3 S_Uxe
//            + a5 D_At + a6 D_xB
//   Phi_Hn = q5 S_Uxa - q2 D_Ua + b1 D_Et
//   Phi_Ht = ie (c1 S_Ue + c2 D_B) + g (S_UxB/2 + c3 D_ex) + c4 ie im S_UAt + c5 S_e - q2 D_UB
//            - q3 S_UxB + c6 D_ex
// with S_* = l + r sums, D_* = r - l differences, U* = M V, ie = 1/eps_s, im = 1/mu_s and
// g = g0 - k3 ie im.  This is the closed form of tm_face_flux above with the face-frame signs
// and the C1..C5 combinations folded into FaceK (see make_face_k).
template <typename T, typename P, bool HAS_MU>
__device__ __forceinline__ void face_pair(const PSide<P> &l, const PSide<P> &r,
                                          const FaceK<T> &k, P &fE, P &fHn, P &fHt) {
  const P half = vbc(T(0.5));
  const P Ue_l = vmul(l.eps, l.e), Ue_r = vmul(r.eps, r.e);
  const P Uxe_l = vmul(l.eps, l.en), Uxe_r = vmul(r.eps, r.en);
  P UB_l = l.ht, UB_r = r.ht, Ua_l = l.hn, Ua_r = r.hn;
  P UxB_l = l.htn, UxB_r = r.htn, Uxa_l = l.hnn, Uxa_r = r.hnn, UAt_l = l.at, UAt_r = r.at;
  if (HAS_MU) {
    UB_l = vmul(l.mu, l.ht); UB_r = vmul(r.mu, r.ht);
    Ua_l = vmul(l.mu, l.hn); Ua_r = vmul(r.mu, r.hn);
    UxB_l = vmul(l.mu, l.htn); UxB_r = vmul(r.mu, r.htn);
    Uxa_l = vmul(l.mu, l.hnn); Uxa_r = vmul(r.mu, r.hnn);
    UAt_l = vmul(l.mu, l.at); UAt_r = vmul(r.mu, r.at);
  }
  const P S_UB = vadd(UB_l, UB_r), D_e = vsub(r.e, l.e);
  const P S_Uxe = vadd(Uxe_l, Uxe_r), D_xB = vsub(r.htn, l.htn);
  const P S_B = vadd(l.ht, r.ht), D_Ue = vsub(Ue_r, Ue_l), D_At = vsub(r.at, l.at);
  const P S_Uxa = vadd(Uxa_l, Uxa_r), D_Ua = vsub(Ua_r, Ua_l), D_Et = vsub(r.et, l.et);
  const P S_Ue = vadd(Ue_l, Ue_r), D_B = vsub(r.ht, l.ht), S_UxB = vadd(UxB_l, UxB_r);
  const P D_ex = vsub(r.en, l.en), S_UAt = vadd(UAt_l, UAt_r), S_e = vadd(l.e, r.e);
  const P D_UB = vsub(UB_r, UB_l);
  const P ie = vrcp(vmul(half, vadd(l.eps, r.eps)));
  P im = vbc(T(1));
  if (HAS_MU) im = vrcp(vmul(half, vadd(l.mu, r.mu)));
  const P iem = HAS_MU ? vmul(ie, im) : ie;
  const P g = vfma(vbc(-k.k3), iem, vbc(k.g0));
  // E flux
  P t = vfma(vbc(k.a2), D_e, vmul(vbc(k.a1), S_UB));
  P fe = HAS_MU ? vmul(im, t) : t;
  fe = vfma(g, vfma(vbc(k.a3), D_xB, vmul(half, S_Uxe)), fe);
  fe = vfma(vbc(k.a4), S_B, fe);
  fe = vfma(vbc(-k.q2), D_Ue, fe);
  fe = vfma(vbc(-k.q3), S_Uxe, fe);
  fe = vfma(vbc(k.a5), D_At, fe);
  fe = vfma(vbc(k.a6), D_xB, fe);
  // normal-H flux
  P fa = vmul(vbc(k.q5), S_Uxa);
  fa = vfma(vbc(-k.q2), D_Ua, fa);
  fa = vfma(vbc(k.b1), D_Et, fa);
  // tangential-H flux
  P fb = vmul(ie, vfma(vbc(k.c2), D_B, vmul(vbc(k.c1), S_Ue)));
  fb = vfma(g, vfma(vbc(k.c3), D_ex, vmul(half, S_UxB)), fb);
  fb = vfma(vmul(vbc(k.c4), iem), S_UAt, fb);
  fb = vfma(vbc(k.c5), S_e, fb);
  fb = vfma(vbc(-k.q2), D_UB, fb);
  fb = vfma(vbc(-k.q3), S_UxB, fb);
  fb = vfma(vbc(k.c6), D_ex, fb);
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
  T inv2hx, inv2hy, halfhx, halfhy;
  FaceK<T> fx, fy;     // interior x- and y-faces
  Coef<T> Kx, Ky;      // boundary faces (scalar path)
  int *flag;
};

__device__ __forceinline__ int wrap_or_clamp(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

template <typename T>
__device__ __forceinline__ T lane(const typename PairOf<T>::type &p, int k) {
  return k ? p.y : p.x;
}
template <typename T>
__device__ __forceinline__ void set_lane(typename PairOf<T>::type &p, int k, T v) {
  if (k) p.y = v; else p.x = v;
}

// Register state of one row of a thread's column pair.
template <typename P>
struct RowV {
  P ez, hx, hy, eps, mu;
};
// Gradient pair of one row: d/dx and d/dy of (Ez, Hx, Hy).
template <typename P>
struct RowG {
  P ex, ey, ax, ay, bx, by;
};

// Load the pair (X, X+1) of row `row` (wrapped or clamped), all components.
template <typename T, bool HAS_MU>
__device__ __forceinline__ RowV<typename PairOf<T>::type> load_pair(const Cart2DKernelArgs<T> &p,
                                                                   int X, int row) {
  using P = typename PairOf<T>::type;
  RowV<P> v;
  const int r = wrap_or_clamp(row, p.ny, p.pery);
  const int64_t ro = (int64_t)r * p.pitch;
  if (X >= 0 && X + 1 < p.nx) {
    const P *b0 = reinterpret_cast<const P *>(p.V + ro + X);
    v.ez = __ldg(b0);
    v.hx = __ldg(reinterpret_cast<const P *>(p.V + p.cstride + ro + X));
    v.hy = __ldg(reinterpret_cast<const P *>(p.V + 2 * p.cstride + ro + X));
    v.eps = __ldg(reinterpret_cast<const P *>(p.eps + ro + X));
    if (HAS_MU) v.mu = __ldg(reinterpret_cast<const P *>(p.mu + ro + X));
  } else {
    const int c0 = wrap_or_clamp(X, p.nx, p.perx), c1 = wrap_or_clamp(X + 1, p.nx, p.perx);
    v.ez = vmk(__ldg(p.V + ro + c0), __ldg(p.V + ro + c1));
    v.hx = vmk(__ldg(p.V + p.cstride + ro + c0), __ldg(p.V + p.cstride + ro + c1));
    v.hy = vmk(__ldg(p.V + 2 * p.cstride + ro + c0), __ldg(p.V + 2 * p.cstride + ro + c1));
    v.eps = vmk(__ldg(p.eps + ro + c0), __ldg(p.eps + ro + c1));
    if (HAS_MU) v.mu = vmk(__ldg(p.mu + ro + c0), __ldg(p.mu + ro + c1));
  }
  if (!HAS_MU) v.mu = vbc(T(1));
  return v;
}

// One extra staged column (x-halo of the strip) for shared memory.
template <typename T, bool HAS_MU>
__device__ __forceinline__ void load_extra(const Cart2DKernelArgs<T> &p, int col, int row, T out[5]) {
  const int r = wrap_or_clamp(row, p.ny, p.pery);
  const int c = wrap_or_clamp(col, p.nx, p.perx);
  const int64_t o = (int64_t)r * p.pitch + c;
  out[0] = __ldg(p.V + o);
  out[1] = __ldg(p.V + p.cstride + o);
  out[2] = __ldg(p.V + 2 * p.cstride + o);
  out[3] = __ldg(p.eps + o);
  out[4] = HAS_MU ? __ldg(p.mu + o) : T(1);
}

// Shared memory (per CTA): staged rows sV[3][5][NCOL] (Ez, Hx, Hy, eps, mu; three row slots),
// gradients sG[2][5][NCOL] (dEz/dx, dHx/dx, dHy/dx, dHx/dy, dEz/dy; two slots), and the
// second x-face flux of each thread sF[2][3][NT].
template <typename T>
struct Smem {
  T V[3][5][NCOL];
  T G[2][5][NCOL];
  T F[2][3][NT];
};

template <typename T, typename P, bool HAS_MU>
__device__ __forceinline__ void stage_row(Smem<T> &s, int slot, int t, const RowV<P> &v) {
  const int ci = 2 * t + 1;
  s.V[slot][0][ci] = v.ez.x; s.V[slot][0][ci + 1] = v.ez.y;
  s.V[slot][1][ci] = v.hx.x; s.V[slot][1][ci + 1] = v.hx.y;
  s.V[slot][2][ci] = v.hy.x; s.V[slot][2][ci + 1] = v.hy.y;
  s.V[slot][3][ci] = v.eps.x; s.V[slot][3][ci + 1] = v.eps.y;
  if (HAS_MU) { s.V[slot][4][ci] = v.mu.x; s.V[slot][4][ci + 1] = v.mu.y; }
}

// Gradient pair of a row: x-neighbours from the staged slot, y-neighbours from registers.
template <typename T, typename P>
__device__ __forceinline__ RowG<P> grad_pair(const Smem<T> &s, int slot, int t, const RowV<P> &c,
                                            const RowV<P> &dn, const RowV<P> &up, T inv2hx,
                                            T inv2hy) {
  const int ci = 2 * t + 1;
  RowG<P> g;
  const P sx = vbc(inv2hx), sy = vbc(inv2hy);
  g.ex = vmul(sx, vsub(vmk(c.ez.y, s.V[slot][0][ci + 2]), vmk(s.V[slot][0][ci - 1], c.ez.x)));
  g.ax = vmul(sx, vsub(vmk(c.hx.y, s.V[slot][1][ci + 2]), vmk(s.V[slot][1][ci - 1], c.hx.x)));
  g.bx = vmul(sx, vsub(vmk(c.hy.y, s.V[slot][2][ci + 2]), vmk(s.V[slot][2][ci - 1], c.hy.x)));
  g.ey = vmul(sy, vsub(up.ez, dn.ez));
  g.ay = vmul(sy, vsub(up.hx, dn.hx));
  g.by = vmul(sy, vsub(up.hy, dn.hy));
  return g;
}

template <typename T, typename P>
__device__ __forceinline__ void stage_grad(Smem<T> &s, int slot, int t, const RowG<P> &g) {
  const int ci = 2 * t + 1;
  s.G[slot][0][ci] = g.ex.x; s.G[slot][0][ci + 1] = g.ex.y;
  s.G[slot][1][ci] = g.ax.x; s.G[slot][1][ci + 1] = g.ax.y;
  s.G[slot][2][ci] = g.bx.x; s.G[slot][2][ci + 1] = g.bx.y;
  s.G[slot][3][ci] = g.ay.x; s.G[slot][3][ci + 1] = g.ay.y;
  s.G[slot][4][ci] = g.ey.x; s.G[slot][4][ci + 1] = g.ey.y;
}

// Scalar boundary-face sides, built from lane k of a thread's pair.
template <typename T, typename P>
__device__ __forceinline__ Side<T> xside(const RowV<P> &v, const RowG<P> &g, int k, T sgn_halfh) {
  Side<T> s;
  const T ex = lane<T>(g.ex, k), ax = lane<T>(g.ax, k), bx = lane<T>(g.bx, k);
  s.e = lane<T>(v.ez, k) + sgn_halfh * ex;
  s.a = lane<T>(v.hx, k) + sgn_halfh * ax;
  s.b = lane<T>(v.hy, k) + sgn_halfh * bx;
  s.ex = ex; s.ax = ax; s.bx = bx;
  s.ay = lane<T>(g.ay, k); s.ey = lane<T>(g.ey, k);
  s.eps = lane<T>(v.eps, k); s.mu = lane<T>(v.mu, k);
  return s;
}

// In the +e_y face frame: e = Ez, a = Hy, b = -Hx; d_x' = d_y, d_y' = -d_x.
template <typename T, typename P>
__device__ __forceinline__ Side<T> yside(const RowV<P> &v, const RowG<P> &g, int k, T sgn_halfh) {
  Side<T> s;
  const T dEx = lane<T>(g.ex, k), dEy = lane<T>(g.ey, k);
  const T dHxy = lane<T>(g.ay, k), dHyx = lane<T>(g.bx, k), dHyy = lane<T>(g.by, k);
  const T ez = lane<T>(v.ez, k) + sgn_halfh * dEy;
  const T hx = lane<T>(v.hx, k) + sgn_halfh * dHxy;
  const T hy = lane<T>(v.hy, k) + sgn_halfh * dHyy;
  s.e = ez; s.a = hy; s.b = -hx;
  s.ex = dEy; s.ax = dHyy; s.bx = -dHxy;
  s.ay = -dHyx; s.ey = -dEx;
  s.eps = lane<T>(v.eps, k); s.mu = lane<T>(v.mu, k);
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

template <typename T, bool HAS_MU>
__global__ void __launch_bounds__(NT) cart2d_step_kernel(const Cart2DKernelArgs<T> p) {
  using P = typename PairOf<T>::type;
  __shared__ __align__(16) Smem<T> s;
  const int t = threadIdx.x;
  const int x0 = blockIdx.x * W;
  const int y0 = blockIdx.y * ROWS;
  const int y1 = min(y0 + ROWS, p.ny);
  const int X = x0 - 2 + 2 * t;
  const int xend = min(x0 + W, p.nx);
  const bool xlo_nrbc = !p.perx, ylo_nrbc = !p.pery;

  // extra staged columns: ci = 0 (column x0-3) by thread 0, ci = NCOL-1 by thread NT-1
  const bool has_extra = (t == 0) || (t == NT - 1);
  const int extra_col = (t == 0) ? x0 - 3 : x0 + 2 * NT - 2;
  const int extra_ci = (t == 0) ? 0 : NCOL - 1;

  // ---------------- prologue: rows y0-2 .. y0+2 in registers, rows y0-1 .. y0+1 staged
  RowV<P> vm2 = load_pair<T, HAS_MU>(p, X, y0 - 2);
  RowV<P> vm1 = load_pair<T, HAS_MU>(p, X, y0 - 1);
  RowV<P> v0 = load_pair<T, HAS_MU>(p, X, y0);
  RowV<P> v1 = load_pair<T, HAS_MU>(p, X, y0 + 1);
  RowV<P> v2 = load_pair<T, HAS_MU>(p, X, y0 + 2);
  stage_row<T, P, HAS_MU>(s, (y0 + 2) % 3, t, vm1);
  stage_row<T, P, HAS_MU>(s, y0 % 3, t, v0);
  stage_row<T, P, HAS_MU>(s, (y0 + 1) % 3, t, v1);
  if (has_extra) {
    T e[5];
    for (int rr = -1; rr <= 1; ++rr) {
      load_extra<T, HAS_MU>(p, extra_col, y0 + rr, e);
      const int sl = (y0 + rr + 3) % 3;
#pragma unroll
      for (int c = 0; c < 5; ++c) s.V[sl][c][extra_ci] = e[c];
    }
  }
  __syncthreads();
  RowG<P> gm1 = grad_pair<T, P>(s, (y0 + 2) % 3, t, vm1, vm2, v0, p.inv2hx, p.inv2hy);
  RowG<P> g0 = grad_pair<T, P>(s, y0 % 3, t, v0, vm1, v1, p.inv2hx, p.inv2hy);
  // y-face below row y0
  P fbE, fbHx, fbHy;
  {
    if (y0 == 0 && ylo_nrbc) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        // outward normal -e_y: in the +e_y frame quantities, local (x', y') = (-y, x)
        Side<T> sq = yside<T, P>(v0, g0, k, -p.halfhy);
        Side<T> q;
        q.e = sq.e; q.a = -sq.a; q.b = -sq.b;
        q.ex = -sq.ex; q.ax = sq.ax; q.bx = sq.bx;
        q.ay = sq.ay; q.ey = -sq.ey;
        q.eps = sq.eps; q.mu = sq.mu;
        T oe, oa, ob;
        tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
        set_lane<T>(fbE, k, -oe); set_lane<T>(fbHx, k, -ob); set_lane<T>(fbHy, k, oa);
      }
    } else {
      PSide<P> l, r;
      const P hh = vbc(p.halfhy);
      l.e = vfma(hh, gm1.ey, vm1.ez); l.hn = vfma(hh, gm1.by, vm1.hy); l.ht = vfma(hh, gm1.ay, vm1.hx);
      l.en = gm1.ey; l.hnn = gm1.by; l.htn = gm1.ay; l.at = gm1.bx; l.et = gm1.ex;
      l.eps = vm1.eps; l.mu = vm1.mu;
      r.e = vfma(vbc(-p.halfhy), g0.ey, v0.ez); r.hn = vfma(vbc(-p.halfhy), g0.by, v0.hy);
      r.ht = vfma(vbc(-p.halfhy), g0.ay, v0.hx);
      r.en = g0.ey; r.hnn = g0.by; r.htn = g0.ay; r.at = g0.bx; r.et = g0.ex;
      r.eps = v0.eps; r.mu = v0.mu;
      face_pair<T, P, HAS_MU>(l, r, p.fy, fbE, fbHy, fbHx);
    }
  }
  stage_grad<T, P>(s, y0 & 1, t, g0);
  __syncthreads();

  T ex_next[5];
  bool bad = false;
  for (int j = y0; j < y1; ++j) {
    // A. prefetch row j+3
    const RowV<P> pf = load_pair<T, HAS_MU>(p, X, j + 3);
    if (has_extra) load_extra<T, HAS_MU>(p, extra_col, j + 2, ex_next);
    // B. gradient pair of row j+1
    const RowG<P> g1 = grad_pair<T, P>(s, (j + 1) % 3, t, v1, v0, v2, p.inv2hx, p.inv2hy);
    // C. x-face pair of row j: faces X+1/2 (own cells) and X+3/2 (own X+1, neighbour X+2)
    P fxE, fxHx, fxHy;
    {
      const int sl = j % 3, gs = j & 1, ci = 2 * t + 1;
      const T rE = s.V[sl][0][ci + 2], rHx = s.V[sl][1][ci + 2], rHy = s.V[sl][2][ci + 2];
      const T rEps = s.V[sl][3][ci + 2];
      const T rMu = HAS_MU ? s.V[sl][4][ci + 2] : T(1);
      const T rgex = s.G[gs][0][ci + 2], rgax = s.G[gs][1][ci + 2], rgbx = s.G[gs][2][ci + 2];
      const T rgay = s.G[gs][3][ci + 2], rgey = s.G[gs][4][ci + 2];
      const P hh = vbc(p.halfhx), mh = vbc(-p.halfhx);
      PSide<P> l, r;
      l.e = vfma(hh, g0.ex, v0.ez); l.hn = vfma(hh, g0.ax, v0.hx); l.ht = vfma(hh, g0.bx, v0.hy);
      l.en = g0.ex; l.hnn = g0.ax; l.htn = g0.bx; l.at = g0.ay; l.et = g0.ey;
      l.eps = v0.eps; l.mu = v0.mu;
      const P Re = vmk(v0.ez.y, rE), RHx = vmk(v0.hx.y, rHx), RHy = vmk(v0.hy.y, rHy);
      r.en = vmk(g0.ex.y, rgex); r.hnn = vmk(g0.ax.y, rgax); r.htn = vmk(g0.bx.y, rgbx);
      r.at = vmk(g0.ay.y, rgay); r.et = vmk(g0.ey.y, rgey);
      r.e = vfma(mh, r.en, Re); r.hn = vfma(mh, r.hnn, RHx); r.ht = vfma(mh, r.htn, RHy);
      r.eps = vmk(v0.eps.y, rEps); r.mu = vmk(v0.mu.y, rMu);
      face_pair<T, P, HAS_MU>(l, r, p.fx, fxE, fxHx, fxHy);
      if (xlo_nrbc) {
        // face X+1/2 or X+3/2 on the domain's x boundary
        if (X == p.nx - 1) {
          Side<T> q = xside<T, P>(v0, g0, 0, p.halfhx);
          T e_, a_, b_;
          tm_face_flux<T, true>(q, q, p.Kx, e_, a_, b_);
          fxE.x = e_; fxHx.x = a_; fxHy.x = b_;
        }
        if (X + 1 == p.nx - 1) {
          Side<T> q = xside<T, P>(v0, g0, 1, p.halfhx);
          T e_, a_, b_;
          tm_face_flux<T, true>(q, q, p.Kx, e_, a_, b_);
          fxE.y = e_; fxHx.y = a_; fxHy.y = b_;
        }
        if (X == -2) {
          // second face is the low boundary face of column 0: build column 0's side from the
          // staged neighbour values (column X+2 = 0)
          Side<T> q;
          q.ex = rgex; q.ax = rgax; q.bx = rgbx; q.ay = rgay; q.ey = rgey;
          q.e = rE - p.halfhx * rgex; q.a = rHx - p.halfhx * rgax; q.b = rHy - p.halfhx * rgbx;
          q.eps = rEps; q.mu = rMu;
          T e_, a_, b_;
          low_boundary_flux<T>(q, p.Kx, e_, a_, b_);
          fxE.y = e_; fxHx.y = a_; fxHy.y = b_;
        }
      }
    }
    // D. y-face pair between rows j and j+1
    P ftE, ftHx, ftHy;
    if (j + 1 == p.ny && ylo_nrbc) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        Side<T> q = yside<T, P>(v0, g0, k, p.halfhy);
        T oe, oa, ob;
        tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
        set_lane<T>(ftE, k, oe); set_lane<T>(ftHx, k, -ob); set_lane<T>(ftHy, k, oa);
      }
    } else {
      PSide<P> l, r;
      const P hh = vbc(p.halfhy), mh = vbc(-p.halfhy);
      l.e = vfma(hh, g0.ey, v0.ez); l.hn = vfma(hh, g0.by, v0.hy); l.ht = vfma(hh, g0.ay, v0.hx);
      l.en = g0.ey; l.hnn = g0.by; l.htn = g0.ay; l.at = g0.bx; l.et = g0.ex;
      l.eps = v0.eps; l.mu = v0.mu;
      r.e = vfma(mh, g1.ey, v1.ez); r.hn = vfma(mh, g1.by, v1.hy); r.ht = vfma(mh, g1.ay, v1.hx);
      r.en = g1.ey; r.hnn = g1.by; r.htn = g1.ay; r.at = g1.bx; r.et = g1.ex;
      r.eps = v1.eps; r.mu = v1.mu;
      face_pair<T, P, HAS_MU>(l, r, p.fy, ftE, ftHy, ftHx);
    }
    // E. stage row j+2, gradient row j+1, and the second x-face for the right neighbour
    {
      const int sl = (j + 2) % 3;
      stage_row<T, P, HAS_MU>(s, sl, t, v2);
      if (has_extra) {
#pragma unroll
        for (int c = 0; c < 5; ++c) s.V[sl][c][extra_ci] = ex_next[c];
      }
      stage_grad<T, P>(s, (j + 1) & 1, t, g1);
      s.F[j & 1][0][t] = fxE.y;
      s.F[j & 1][1][t] = fxHx.y;
      s.F[j & 1][2][t] = fxHy.y;
    }
    __syncthreads();
    // G. update the pair of row j: U^{n+1} = U^n - sum of face fluxes (carry dt/h) + dt S
    {
      const T lE = t > 0 ? s.F[j & 1][0][t - 1] : T(0);
      const T lHx = t > 0 ? s.F[j & 1][1][t - 1] : T(0);
      const T lHy = t > 0 ? s.F[j & 1][2][t - 1] : T(0);
      // left faces of (X, X+1) = (neighbour's second face, own first face)
      P dE = vadd(vsub(vmk(lE, fxE.x), fxE), vsub(fbE, ftE));
      const P dHx = vadd(vsub(vmk(lHx, fxHx.x), fxHx), vsub(fbHx, ftHx));
      const P dHy = vadd(vsub(vmk(lHy, fxHy.x), fxHy), vsub(fbHy, ftHy));
      if (p.src && j >= p.sy0 && j < p.sy1) {
        const int64_t ro = (int64_t)j * p.pitch;
        if (X >= p.sx0 && X < p.sx1 && X >= 0) dE.x -= p.src_amp * p.src[ro + X];
        if (X + 1 >= p.sx0 && X + 1 < p.sx1 && X + 1 < p.nx) dE.y -= p.src_amp * p.src[ro + X + 1];
      }
      const P ie = vrcp(v0.eps);
      const P ve = vfma(dE, ie, v0.ez);
      P vhx, vhy;
      if (HAS_MU) {
        const P im = vrcp(v0.mu);
        vhx = vfma(dHx, im, v0.hx);
        vhy = vfma(dHy, im, v0.hy);
      } else {
        vhx = vadd(v0.hx, dHx);
        vhy = vadd(v0.hy, dHy);
      }
      const int64_t ro = (int64_t)j * p.pitch;
      const bool ok0 = X >= x0 && X < xend, ok1 = X + 1 >= x0 && X + 1 < xend;
      if (ok0 && ok1) {
        *reinterpret_cast<P *>(p.Vout + ro + X) = ve;
        *reinterpret_cast<P *>(p.Vout + p.cstride + ro + X) = vhx;
        *reinterpret_cast<P *>(p.Vout + 2 * p.cstride + ro + X) = vhy;
        bad |= !(isfinite(ve.x) && isfinite(vhx.x) && isfinite(vhy.x) && isfinite(ve.y) &&
                 isfinite(vhx.y) && isfinite(vhy.y));
      } else {
        if (ok0) {
          p.Vout[ro + X] = ve.x;
          p.Vout[p.cstride + ro + X] = vhx.x;
          p.Vout[2 * p.cstride + ro + X] = vhy.x;
          bad |= !(isfinite(ve.x) && isfinite(vhx.x) && isfinite(vhy.x));
        }
        if (ok1) {
          p.Vout[ro + X + 1] = ve.y;
          p.Vout[p.cstride + ro + X + 1] = vhx.y;
          p.Vout[2 * p.cstride + ro + X + 1] = vhy.y;
          bad |= !(isfinite(ve.y) && isfinite(vhx.y) && isfinite(vhy.y));
        }
      }
    }
    // H. rotate the register window
    v0 = v1; v1 = v2; v2 = pf;
    g0 = g1;
    fbE = ftE; fbHx = ftHx; fbHy = ftHy;
  }
  if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) atomicOr(p.flag, 1);
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

// Constants of face_pair for a face of normal spacing h whose frame has tangential-H sign sb
// and tangential-derivative sign st (x-faces: +1, +1; y-faces: -1, -1).
template <typename T>
FaceK<T> make_face_k(const double C[5], double h, double c, double sb, double st) {
  const double K1 = C[0] / h, K2 = C[1] / h, K3 = C[2] / h, K4 = C[3] / h, K5 = C[4] / h;
  const double inv2c = 0.5 / c;
  const double q1 = 0.5 * K4, q2 = 0.5 * K4 * c, q3 = 0.5 * K5 * c * c, q4 = 0.5 * K5 * c;
  FaceK<T> k;
  k.a1 = T(-0.5 * K1 * sb); k.a2 = T(-K1 * inv2c); k.a3 = T(sb * inv2c);
  k.a4 = T(-q1 * sb); k.a5 = T(q4 * st); k.a6 = T(-q4 * sb);
  k.q2 = T(q2); k.q3 = T(q3); k.q5 = T(0.5 * K2 * c * c - q3); k.b1 = T(q4 * st);
  k.c1 = T(-0.5 * K1 * sb); k.c2 = T(-K1 * inv2c); k.c3 = T(sb * inv2c);
  k.c4 = T(0.5 * K3 * sb * st); k.c5 = T(-sb * q1); k.c6 = T(-sb * q4);
  k.g0 = T(K2 * c * c); k.k3 = T(K3);
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
  p.fx = make_face_k<T>(a.C, g.h[0], a.c, 1.0, 1.0);
  p.fy = make_face_k<T>(a.C, g.h[1], a.c, -1.0, -1.0);
  p.Kx = make_coef<T>(a.C, g.h[0], a.c);
  p.Ky = make_coef<T>(a.C, g.h[1], a.c);
  p.flag = a.flag;
  dim3 grid((g.nx + W - 1) / W, (g.ny + ROWS - 1) / ROWS);
  if (a.mu)
    cart2d_step_kernel<T, true><<<grid, NT, 0, st>>>(p);
  else
    cart2d_step_kernel<T, false><<<grid, NT, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cart2d_step(const CartGeom &g, const CartStepArgs &a, bool fp64,
                               cudaStream_t st) {
  return fp64 ? launch_t<double>(g, a, st) : launch_t<float>(g, a, st);
}

}  // namespace gks
