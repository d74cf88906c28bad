// Time-integrated GKS face flux in a face frame (normal n, tangents t, w), shared by the
// Cartesian 3-D and the tetrahedral kernels.  Device code only.
#pragma once

#include <cuda_runtime.h>

namespace gks {

// Local face quantities of one side (components in the face frame (n, t, w)):
// V = (En, Et, Ew, Hn, Ht, Hw) reconstructed at the face centre, and its derivatives along
// n, t and w.
template <typename T>
struct Side3 {
  T v[6], dn[6], dt[6], dw[6];
  T eps, mu;
};

template <typename T>
struct K3 {
  T k1, k2, k3, k4, k5;  // C_i / h_normal
  T c, c2, inv2c, halfc, c2half;
};

enum { EN = 0, ET = 1, EW = 2, HN = 3, HT = 4, HW = 5 };

// F_1 (flux along the face normal) in the face frame: (0, Hw, -Ht, 0, -Ew, Et).
// Time-integrated GKS flux (Sec. 3.1) in the face frame, times dt/h.  Closed form of the
// D3Q4 sums (s_k = u_k / c; right-moving pair (1,1,1), (1,-1,-1)):
//   W0 = (U^l + U^r)/2 + (F_1^l - F_1^r)/(2c),        V0 = W0 / M_s
//   <u_n g0> = F_1(V0)
//   <u_n u.grad g0> = c^2 d_n W0 + c (F_3(d_t V0) + F_2(d_w V0))
//   <u_n g_t> = F_1(V0_t),  V0_t = -(F_1(d_n V0) + F_2(d_t V0) + F_3(d_w V0)) / M_s
//   free transport = (F_1^l + F_1^r)/2 - (c/2)(U^r - U^l)
//   free-transport gradient = (c^2/2)(M d_n V^l + M d_n V^r)
//       + (c/2)[F_1(d_n V^l) + (F_2 + F_3)(d_t V^l + d_w V^l)]
//       - (c/2)[F_1(d_n V^r) + (F_2 - F_3)(d_t V^r - d_w V^r)]
// where (F_2 + F_3)(p) = (pHt - pHw, -pHn, pHn, pEw - pEt, pEn, -pEn) and
// (F_2 - F_3)(q) = (-qHw - qHt, qHn, qHn, qEw + qEt, -qEn, -qEn).
// GHOST: the r side is a non-reflecting ghost (no distributions; M_s = M_l).
template <typename T, bool GHOST>
__device__ __forceinline__ void flux3(const Side3<T> &l, const Side3<T> &r, const K3<T> &K,
                                      T out[6]) {
  const T h = T(0.5);
  // conserved values and normal derivatives of conserved values
  T Ul[6], Ur[6], Nl[6], Nr[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const T ml = c < 3 ? l.eps : l.mu;
    Ul[c] = ml * l.v[c];
    Nl[c] = ml * l.dn[c];
    if (!GHOST) {
      const T mr = c < 3 ? r.eps : r.mu;
      Ur[c] = mr * r.v[c];
      Nr[c] = mr * r.dn[c];
    } else {
      Ur[c] = T(0);
      Nr[c] = T(0);
    }
  }
  T ie, im;
  if (GHOST) {
    ie = T(1) / l.eps;
    im = T(1) / l.mu;
  } else {
    ie = T(2) / (l.eps + r.eps);
    im = T(2) / (l.mu + r.mu);
  }
  // r-side raw values (zero on a ghost face)
  T rv[6], rdn[6], rdt[6], rdw[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    rv[c] = GHOST ? T(0) : r.v[c];
    rdn[c] = GHOST ? T(0) : r.dn[c];
    rdt[c] = GHOST ? T(0) : r.dt[c];
    rdw[c] = GHOST ? T(0) : r.dw[c];
  }
  const T rmE = GHOST ? T(0) : r.eps, rmH = GHOST ? T(0) : r.mu;
  // interface moment W0 (components Et, Ew, Ht, Hw) -> V0
  const T W_Et = h * (Ul[ET] + Ur[ET]) + (l.v[HW] - rv[HW]) * K.inv2c;
  const T W_Ew = h * (Ul[EW] + Ur[EW]) + (rv[HT] - l.v[HT]) * K.inv2c;
  const T W_Ht = h * (Ul[HT] + Ur[HT]) + (rv[EW] - l.v[EW]) * K.inv2c;
  const T W_Hw = h * (Ul[HW] + Ur[HW]) + (l.v[ET] - rv[ET]) * K.inv2c;
  // d_n W0 (all six)
  T Dn[6];
  Dn[EN] = h * (Nl[EN] + Nr[EN]);
  Dn[ET] = h * (Nl[ET] + Nr[ET]) + (l.dn[HW] - rdn[HW]) * K.inv2c;
  Dn[EW] = h * (Nl[EW] + Nr[EW]) + (rdn[HT] - l.dn[HT]) * K.inv2c;
  Dn[HN] = h * (Nl[HN] + Nr[HN]);
  Dn[HT] = h * (Nl[HT] + Nr[HT]) + (rdn[EW] - l.dn[EW]) * K.inv2c;
  Dn[HW] = h * (Nl[HW] + Nr[HW]) + (l.dn[ET] - rdn[ET]) * K.inv2c;
  // d_t W0 (En, Et, Hn, Ht) and d_w W0 (En, Ew, Hn, Hw)
  const T Dt_En = h * (l.eps * l.dt[EN] + rmE * rdt[EN]);
  const T Dt_Et = h * (l.eps * l.dt[ET] + rmE * rdt[ET]) + (l.dt[HW] - rdt[HW]) * K.inv2c;
  const T Dt_Hn = h * (l.mu * l.dt[HN] + rmH * rdt[HN]);
  const T Dt_Ht = h * (l.mu * l.dt[HT] + rmH * rdt[HT]) + (rdt[EW] - l.dt[EW]) * K.inv2c;
  const T Dw_En = h * (l.eps * l.dw[EN] + rmE * rdw[EN]);
  const T Dw_Ew = h * (l.eps * l.dw[EW] + rmE * rdw[EW]) + (rdw[HT] - l.dw[HT]) * K.inv2c;
  const T Dw_Hn = h * (l.mu * l.dw[HN] + rmH * rdw[HN]);
  const T Dw_Hw = h * (l.mu * l.dw[HW] + rmH * rdw[HW]) + (l.dw[ET] - rdw[ET]) * K.inv2c;
  // derivatives of V0 = W0 / M_s
  const T aEn = Dt_En * ie, aEt = Dt_Et * ie, aHn = Dt_Hn * im, aHt = Dt_Ht * im;
  const T bEn = Dw_En * ie, bEw = Dw_Ew * ie, bHn = Dw_Hn * im, bHw = Dw_Hw * im;
  const T dEt = Dn[ET] * ie, dEw = Dn[EW] * ie, dHt = Dn[HT] * im, dHw = Dn[HW] * im;
  // term 1: F_1(V0)
  T t1[6] = {T(0), W_Hw * im, -W_Ht * im, T(0), -W_Ew * ie, W_Et * ie};
  // term 2: c^2 d_n W0 + c (F_3(a) + F_2(b))
  T X0[6] = {aHt - bHw, -aHn, bHn, bEw - aEt, aEn, -bEn};
  // term 3: F_1(V0_t), V0_t = -(F_1(d) + F_2(a) + F_3(b)) / M_s (components Et, Ew, Ht, Hw)
  const T Vt_Et = -(dHw - bHn) * ie;
  const T Vt_Ew = -(aHn - dHt) * ie;
  const T Vt_Ht = -(bEn - dEw) * im;
  const T Vt_Hw = -(dEt - aEn) * im;
  T t3[6] = {T(0), Vt_Hw, -Vt_Ht, T(0), -Vt_Ew, Vt_Et};
  // term 4: (F_1^l + F_1^r)/2 - (c/2)(U^r - U^l)
  T t4[6];
  t4[EN] = -K.halfc * (Ur[EN] - Ul[EN]);
  t4[ET] = h * (l.v[HW] + rv[HW]) - K.halfc * (Ur[ET] - Ul[ET]);
  t4[EW] = -h * (l.v[HT] + rv[HT]) - K.halfc * (Ur[EW] - Ul[EW]);
  t4[HN] = -K.halfc * (Ur[HN] - Ul[HN]);
  t4[HT] = -h * (l.v[EW] + rv[EW]) - K.halfc * (Ur[HT] - Ul[HT]);
  t4[HW] = h * (l.v[ET] + rv[ET]) - K.halfc * (Ur[HW] - Ul[HW]);
  // term 5: free-transport gradient
  T p[6], q[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    p[c] = l.dt[c] + l.dw[c];
    q[c] = rdt[c] - rdw[c];
  }
  const T SX_l[6] = {p[HT] - p[HW], -p[HN], p[HN], p[EW] - p[ET], p[EN], -p[EN]};
  const T SX_r[6] = {-q[HW] - q[HT], q[HN], q[HN], q[EW] + q[ET], -q[EN], -q[EN]};
  const T F1l[6] = {T(0), l.dn[HW], -l.dn[HT], T(0), -l.dn[EW], l.dn[ET]};
  const T F1r[6] = {T(0), rdn[HW], -rdn[HT], T(0), -rdn[EW], rdn[ET]};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const T t2 = K.c2 * Dn[c] + K.c * X0[c];
    const T t5 = K.c2half * (Nl[c] + Nr[c]) + K.halfc * ((F1l[c] + SX_l[c]) - (F1r[c] + SX_r[c]));
    out[c] = K.k1 * t1[c] + K.k2 * t2 + K.k3 * t3[c] + K.k4 * t4[c] - K.k5 * t5;
  }
}


// Folded constants of flux3 for mu = 1 on both sides (see flux3_mu1); K_i = C_i / h_normal.
template <typename T>
struct F3K {
  T A1, A2, A3, A4, A5, B1, B2, B3, B4, B5, C1, G1;
};

template <typename T>
inline F3K<T> make_f3k(const double C[5], double h, double c) {
  const double k1 = C[0] / h, k2 = C[1] / h, k3 = C[2] / h, k4 = C[3] / h, k5 = C[4] / h;
  F3K<T> f;
  f.A1 = T(0.5 * k2); f.A2 = T(0.5 * c * (k2 - k5)); f.A3 = T(0.5 * c * k5);
  f.A4 = T(0.5 * c * k4); f.A5 = T(0.5 * c * c * (k2 - k5));
  f.B1 = T(0.5 * (k1 + k4)); f.B2 = T(0.5 * k1 / c); f.B3 = T(0.5 * k3);
  f.B4 = T(0.5 * k1); f.B5 = T(0.5 * k4); f.C1 = T(0.5 * c * k2); f.G1 = T(0.5 * k3 / c);
  return f;
}

// flux3 of an interior face with mu = 1 on both sides, rewritten in sums S(x) = x_l + x_r and
// differences D(x) = x_r - x_l of the side quantities (v reconstructed values, n/t/w the
// derivatives along the face frame's axes; eps-weighted where marked e), with ie = 1/eps_s:
//   En = A1 (D tEw + D wEt) + A2 (S tHt - S wHw) + A3 (D wHt - D tHw) - A4 D e.vEn + A5 S e.nEn
//   Et = B1 S vHw - g D nHw - A2 S tHn - A3 D wHn - A4 D e.vEt - B2 D vEt + B3 ie S e.tEn + cg S e.nEt
//   Ew = -B1 S vHt + g D nHt + A2 S wHn + A3 D tHn - A4 D e.vEw - B2 D vEw + B3 ie S e.wEn + cg S e.nEw
//   Hn = -A4 D vHn + A5 S nHn + A3 (S tEt - S wEw + D tEw - D wEt)
//        + ie (C1 (S e.wEw - S e.tEt) + A1 (D tHw + D wHt))
//   Ht = -B4 ie S e.vEw - B5 S vEw + g D nEw - (A4 + B2 ie) D vHt + A3 (D wEn - S tEn)
//        + B3 ie S tHn + cg S nHt + C1 ie S e.tEn
//   Hw = B4 ie S e.vEt + B5 S vEt - g D nEt - (A4 + B2 ie) D vHw + A3 (S wEn - D tEn)
//        + B3 ie S wHn + cg S nHw - C1 ie S e.wEn
// with g = A2 - G1 ie and cg = A5 - B3 ie.  Equal to flux3<T, false> term by term.
template <typename T>
__device__ __forceinline__ void flux3_mu1(const Side3<T> &l, const Side3<T> &r, const F3K<T> &K,
                                          T ie, T out[6]) {
  const T el = l.eps, er = r.eps;
  const T g = K.A2 - K.G1 * ie, cg = K.A5 - K.B3 * ie;
  const T A4B2 = K.A4 + K.B2 * ie;
#define GKS_S(f, c) (l.f[c] + r.f[c])
#define GKS_D(f, c) (r.f[c] - l.f[c])
#define GKS_SE(f, c) (el * l.f[c] + er * r.f[c])
#define GKS_DE(f, c) (er * r.f[c] - el * l.f[c])
  out[EN] = K.A1 * (GKS_D(dt, EW) + GKS_D(dw, ET)) + K.A2 * (GKS_S(dt, HT) - GKS_S(dw, HW)) +
            K.A3 * (GKS_D(dw, HT) - GKS_D(dt, HW)) - K.A4 * GKS_DE(v, EN) + K.A5 * GKS_SE(dn, EN);
  out[ET] = K.B1 * GKS_S(v, HW) - g * GKS_D(dn, HW) - K.A2 * GKS_S(dt, HN) - K.A3 * GKS_D(dw, HN) -
            K.A4 * GKS_DE(v, ET) - K.B2 * GKS_D(v, ET) + K.B3 * ie * GKS_SE(dt, EN) +
            cg * GKS_SE(dn, ET);
  out[EW] = -K.B1 * GKS_S(v, HT) + g * GKS_D(dn, HT) + K.A2 * GKS_S(dw, HN) + K.A3 * GKS_D(dt, HN) -
            K.A4 * GKS_DE(v, EW) - K.B2 * GKS_D(v, EW) + K.B3 * ie * GKS_SE(dw, EN) +
            cg * GKS_SE(dn, EW);
  out[HN] = -K.A4 * GKS_D(v, HN) + K.A5 * GKS_S(dn, HN) +
            K.A3 * ((GKS_S(dt, ET) - GKS_S(dw, EW)) + (GKS_D(dt, EW) - GKS_D(dw, ET))) +
            ie * (K.C1 * (GKS_SE(dw, EW) - GKS_SE(dt, ET)) + K.A1 * (GKS_D(dt, HW) + GKS_D(dw, HT)));
  out[HT] = -K.B4 * ie * GKS_SE(v, EW) - K.B5 * GKS_S(v, EW) + g * GKS_D(dn, EW) -
            A4B2 * GKS_D(v, HT) + K.A3 * (GKS_D(dw, EN) - GKS_S(dt, EN)) +
            K.B3 * ie * GKS_S(dt, HN) + cg * GKS_S(dn, HT) + K.C1 * ie * GKS_SE(dt, EN);
  out[HW] = K.B4 * ie * GKS_SE(v, ET) + K.B5 * GKS_S(v, ET) - g * GKS_D(dn, ET) -
            A4B2 * GKS_D(v, HW) + K.A3 * (GKS_S(dw, EN) - GKS_D(dt, EN)) +
            K.B3 * ie * GKS_S(dw, HN) + cg * GKS_S(dn, HW) - K.C1 * ie * GKS_SE(dw, EN);
#undef GKS_S
#undef GKS_D
#undef GKS_SE
#undef GKS_DE
}

// ---------------------------------------------------------------------------------------------
// Divergence cleaning (PHM system, Sec. 2.1): V = (En, Et, Ew, Hn, Ht, Hw, phi, psi) in the
// face frame.  F_j adds chi phi to E_j and gamma psi to H_j; the phi and psi rows are chi E_j
// and gamma H_j.  M = diag(eps, eps, eps, mu, mu, mu, 1, 1).
enum { PHI = 6, PSI = 7 };

template <typename T>
struct Side8 {
  T v[8], dn[8], dt[8], dw[8];
  T eps, mu;
};

template <typename T>
__device__ __forceinline__ void phm_fn(const T v[8], T chi, T gam, T o[8]) {
  o[EN] = chi * v[PHI]; o[ET] = v[HW]; o[EW] = -v[HT];
  o[HN] = gam * v[PSI]; o[HT] = -v[EW]; o[HW] = v[ET];
  o[PHI] = chi * v[EN]; o[PSI] = gam * v[HN];
}
template <typename T>
__device__ __forceinline__ void phm_ft(const T v[8], T chi, T gam, T o[8]) {
  o[EN] = -v[HW]; o[ET] = chi * v[PHI]; o[EW] = v[HN];
  o[HN] = v[EW]; o[HT] = gam * v[PSI]; o[HW] = -v[EN];
  o[PHI] = chi * v[ET]; o[PSI] = gam * v[HT];
}
template <typename T>
__device__ __forceinline__ void phm_fw(const T v[8], T chi, T gam, T o[8]) {
  o[EN] = v[HT]; o[ET] = -v[HN]; o[EW] = chi * v[PHI];
  o[HN] = -v[ET]; o[HT] = v[EN]; o[HW] = gam * v[PSI];
  o[PHI] = chi * v[EW]; o[PSI] = gam * v[HW];
}

// Time-integrated GKS flux of the cleaning system in the face frame, times dt/h.  The D3Q4
// half-range sums have the same closed form for any linear flux function (right-moving
// velocities c(1,1,1), c(1,-1,-1); sum over them of u_k^j u_k^m = 2c^2 (delta_jm + [jm = tw])):
//   W0 = (U^l + U^r)/2 + (F_n^l - F_n^r)/(2c),  d_j W0 likewise,  V0 = W0 / M_s
//   <u_n g0> = F_n(V0);  <u_n u.grad g0> = c^2 d_n W0 + c (F_t(d_w V0) + F_w(d_t V0))
//   <u_n g_t> = F_n(V0_t),  V0_t = -(F_n(d_n V0) + F_t(d_t V0) + F_w(d_w V0)) / M_s
//   free transport = (F_n^l + F_n^r)/2 - (c/2)(U^r - U^l)
//   free-transport gradient = (c^2/2)(M_l d_n V^l + M_r d_n V^r)
//       + (c/2)[F_n(d_n V^l) + (F_t + F_w)(d_t V^l + d_w V^l)]
//       - (c/2)[F_n(d_n V^r) + (F_t - F_w)(d_t V^r - d_w V^r)]
// GHOST: the r side is a non-reflecting ghost (no distributions; M_s = M_l).  MU1: mu = 1 on
// both sides (the sides' mu fields are not read).  The reciprocals 1/eps_s are the fast ones in
// FP32 (about 1 ulp), as in the Maxwell kernels.
__device__ __forceinline__ float fast_div(float a, float x) { return __fdividef(a, x); }
__device__ __forceinline__ double fast_div(double a, double x) { return a / x; }

template <typename T, bool GHOST, bool MU1 = false>
__device__ __forceinline__ void flux3_phm(const Side8<T> &l, const Side8<T> &r, const K3<T> &K,
                                          T chi, T gam, T out[8]) {
  const T h = T(0.5);
  const T lmu = MU1 ? T(1) : l.mu, rmu = MU1 ? T(1) : r.mu;
  T ml[8], mr[8], ims[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    ml[c] = c < 3 ? l.eps : (c < 6 ? lmu : T(1));
    mr[c] = GHOST ? T(0) : (c < 3 ? r.eps : (c < 6 ? rmu : T(1)));
  }
  const T ie = GHOST ? fast_div(T(1), l.eps) : fast_div(T(2), l.eps + r.eps);
  const T im = MU1 ? T(1) : (GHOST ? T(1) / lmu : T(2) / (lmu + rmu));
#pragma unroll
  for (int c = 0; c < 8; ++c) ims[c] = c < 3 ? ie : (c < 6 ? im : T(1));
  T rv[8], rn[8], rt[8], rw[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    rv[c] = GHOST ? T(0) : r.v[c];
    rn[c] = GHOST ? T(0) : r.dn[c];
    rt[c] = GHOST ? T(0) : r.dt[c];
    rw[c] = GHOST ? T(0) : r.dw[c];
  }
  // interface moment and its derivatives: X0 = (M_l x^l + M_r x^r)/2 + F_n(x^l - x^r)/(2c)
  T dv[8], dn[8], dt[8], dw[8], Fv[8], Fn_[8], Ft_[8], Fw_[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    dv[c] = l.v[c] - rv[c];
    dn[c] = l.dn[c] - rn[c];
    dt[c] = l.dt[c] - rt[c];
    dw[c] = l.dw[c] - rw[c];
  }
  phm_fn(dv, chi, gam, Fv);
  phm_fn(dn, chi, gam, Fn_);
  phm_fn(dt, chi, gam, Ft_);
  phm_fn(dw, chi, gam, Fw_);
  T V0[8], Dn[8], V0n[8], V0t[8], V0w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T W = h * (ml[c] * l.v[c] + mr[c] * rv[c]) + Fv[c] * K.inv2c;
    Dn[c] = h * (ml[c] * l.dn[c] + mr[c] * rn[c]) + Fn_[c] * K.inv2c;
    const T Dt = h * (ml[c] * l.dt[c] + mr[c] * rt[c]) + Ft_[c] * K.inv2c;
    const T Dw = h * (ml[c] * l.dw[c] + mr[c] * rw[c]) + Fw_[c] * K.inv2c;
    V0[c] = W * ims[c];
    V0n[c] = Dn[c] * ims[c];
    V0t[c] = Dt * ims[c];
    V0w[c] = Dw * ims[c];
  }
  T t1[8], a[8], b[8], q[8], t3[8], Vt[8];
  phm_fn(V0, chi, gam, t1);
  phm_ft(V0w, chi, gam, a);
  phm_fw(V0t, chi, gam, b);
  // V0_t
  phm_fn(V0n, chi, gam, q);
  {
    T u[8], w[8];
    phm_ft(V0t, chi, gam, u);
    phm_fw(V0w, chi, gam, w);
#pragma unroll
    for (int c = 0; c < 8; ++c) Vt[c] = -(q[c] + u[c] + w[c]) * ims[c];
  }
  phm_fn(Vt, chi, gam, t3);
  // free transport and its gradient
  T Fl[8], Fr[8], Gl[8], Gr[8], Sl[8], Sr[8];
  phm_fn(l.v, chi, gam, Fl);
  phm_fn(rv, chi, gam, Fr);
  phm_fn(l.dn, chi, gam, Gl);
  phm_fn(rn, chi, gam, Gr);
  {
    T pl[8], pr[8], x1[8], x2[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      pl[c] = l.dt[c] + l.dw[c];
      pr[c] = rt[c] - rw[c];
    }
    phm_ft(pl, chi, gam, x1);
    phm_fw(pl, chi, gam, x2);
#pragma unroll
    for (int c = 0; c < 8; ++c) Sl[c] = x1[c] + x2[c];
    phm_ft(pr, chi, gam, x1);
    phm_fw(pr, chi, gam, x2);
#pragma unroll
    for (int c = 0; c < 8; ++c) Sr[c] = x1[c] - x2[c];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const T t2 = K.c2 * Dn[c] + K.c * (a[c] + b[c]);
    const T t4 = h * (Fl[c] + Fr[c]) - K.halfc * (mr[c] * rv[c] - ml[c] * l.v[c]);
    const T t5 = K.c2half * (ml[c] * l.dn[c] + mr[c] * rn[c]) +
                 K.halfc * ((Gl[c] + Sl[c]) - (Gr[c] + Sr[c]));
    out[c] = K.k1 * t1[c] + K.k2 * t2 + K.k3 * t3[c] + K.k4 * t4 - K.k5 * t5;
  }
}

// flux3_phm with mu = 1 on an interior face, folded (F8K, make_f8k, flux3_phm_mu1): generated
// into gks_phm3.cuh, included at the end of this header.

template <typename T>
K3<T> make_k3(const double C[5], double h, double c) {
  K3<T> k;
  k.k1 = T(C[0] / h); k.k2 = T(C[1] / h); k.k3 = T(C[2] / h);
  k.k4 = T(C[3] / h); k.k5 = T(C[4] / h);
  k.c = T(c); k.c2 = T(c * c); k.inv2c = T(0.5 / c); k.halfc = T(0.5 * c);
  k.c2half = T(0.5 * c * c);
  return k;
}

}  // namespace gks

#include "gks_phm3.cuh"
