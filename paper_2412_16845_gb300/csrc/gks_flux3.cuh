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

// Folded constants of flux3_phm for an interior face with mu = 1 on both sides: k[] multiply a
// sum or difference directly, c_j = a[j] + b[j] ie (ie = 2/(eps_l + eps_r)) the others.
template <typename T>
struct F8K {
  T k[30];
  T a[19], b[19];
};

template <typename T>
inline F8K<T> make_f8k(const double C[5], double h, double c, double chi, double gam) {
  const double k1 = C[0] / h, k2 = C[1] / h, k3 = C[2] / h, k4 = C[3] / h, k5 = C[4] / h;
  F8K<T> f;
  f.k[0] = T(-1.0/2.0*(chi * chi)*k1/c);
  f.k[1] = T(-1.0/2.0*c*k4);
  f.k[2] = T((1.0/2.0)*chi*(k1 + k4));
  f.k[3] = T((1.0/2.0)*k2);
  f.k[4] = T((1.0/2.0)*c*(k2 - k5));
  f.k[5] = T(-1.0/2.0*c*(k2 - k5));
  f.k[6] = T(-1.0/2.0*k1/c);
  f.k[7] = T((1.0/2.0)*(k1 + k4));
  f.k[8] = T((1.0/2.0)*gam*k2);
  f.k[9] = T(-1.0/2.0*(chi * chi)*k2);
  f.k[10] = T(-1.0/2.0*((c * c)*k5 - (gam * gam)*k3)/c);
  f.k[11] = T((1.0/2.0)*c*chi*(k2 - k5));
  f.k[12] = T(-1.0/2.0*gam*k3);
  f.k[13] = T(-1.0/2.0*(k1 + k4));
  f.k[14] = T((1.0/2.0)*((c * c)*k5 - (gam * gam)*k3)/c);
  f.k[15] = T((1.0/2.0)*gam*k3);
  f.k[16] = T(-1.0/2.0*gam*k2);
  f.k[17] = T(-1.0/2.0*((c * c)*k4 + (gam * gam)*k1)/c);
  f.k[18] = T((1.0/2.0)*gam*(k1 + k4));
  f.k[19] = T((1.0/2.0)*((c * c)*k2 - (c * c)*k5 - (gam * gam)*k3));
  f.k[20] = T(-1.0/2.0*gam*((c * c)*k2 - (c * c)*k5 - (gam * gam)*k3)/c);
  f.k[21] = T((1.0/2.0)*c*k5);
  f.k[22] = T(-1.0/2.0*(gam * gam)*k3);
  f.k[23] = T(-1.0/2.0*c*k5);
  f.k[24] = T(-1.0/2.0*k4);
  f.k[25] = T(-1.0/2.0*(gam * gam)*k2);
  f.k[26] = T((1.0/2.0)*c*gam*(k2 - k5));
  f.k[27] = T((1.0/2.0)*k4);
  f.k[28] = T((1.0/2.0)*chi*k4);
  f.k[29] = T(-1.0/2.0*c*chi*k5);
  f.a[0] = T((1.0/2.0)*(c * c)*(k2 - k5));
  f.b[0] = T(-1.0/2.0*(chi * chi)*k3);
  f.a[1] = T(-1.0/2.0*c*chi*(k2 - k5));
  f.b[1] = T((1.0/2.0)*(chi * chi * chi)*k3/c);
  f.a[2] = T(0);
  f.b[2] = T(-1.0/2.0*(chi * chi)*k3);
  f.a[3] = T(-1.0/2.0*c*k5);
  f.b[3] = T((1.0/2.0)*(chi * chi)*k3/c);
  f.a[4] = T((1.0/2.0)*(c * c)*(k2 - k5));
  f.b[4] = T(-1.0/2.0*k3);
  f.a[5] = T(-1.0/2.0*c*(k2 - k5));
  f.b[5] = T((1.0/2.0)*k3/c);
  f.a[6] = T(0);
  f.b[6] = T((1.0/2.0)*k3);
  f.a[7] = T((1.0/2.0)*c*chi*k5);
  f.b[7] = T(-1.0/2.0*chi*k3/c);
  f.a[8] = T(0);
  f.b[8] = T(-1.0/2.0*c*k2);
  f.a[9] = T(0);
  f.b[9] = T((1.0/2.0)*k2);
  f.a[10] = T(0);
  f.b[10] = T(-1.0/2.0*k1);
  f.a[11] = T(-1.0/2.0*c*k4);
  f.b[11] = T(-1.0/2.0*k1/c);
  f.a[12] = T(0);
  f.b[12] = T(-1.0/2.0*chi*k2);
  f.a[13] = T((1.0/2.0)*c*gam*k5);
  f.b[13] = T(-1.0/2.0*gam*k3/c);
  f.a[14] = T(0);
  f.b[14] = T((1.0/2.0)*chi*k3);
  f.a[15] = T(0);
  f.b[15] = T((1.0/2.0)*chi*k1);
  f.a[16] = T(-1.0/2.0*c*k4);
  f.b[16] = T(-1.0/2.0*(chi * chi)*k1/c);
  f.a[17] = T(0);
  f.b[17] = T((1.0/2.0)*c*chi*k2);
  f.a[18] = T(0);
  f.b[18] = T(-1.0/2.0*gam*k3);
  return f;
}

// flux3_phm<T, false, true> of an interior face rewritten in sums S(x) = x_l + x_r, differences
// D(x) = x_r - x_l and their eps-weighted forms SE(x) = eps_l x_l + eps_r x_r,
// DE(x) = eps_r x_r - eps_l x_l of the side quantities (v reconstructed values, n/t/w the
// derivatives along the face frame's axes; components En, Et, Ew, Hn, Ht, Hw, Ph(i), Ps(i)),
// with the coefficients, polynomials in C_i/h, c, chi and gamma (linear in ie), folded on the
// host.  Equal to flux3_phm term by term (checked symbolically and numerically).
template <typename T>
__device__ __forceinline__ void flux3_phm_mu1(const Side8<T> &l, const Side8<T> &r,
                                              const F8K<T> &K, T ie, T out[8]) {
  const T el = l.eps, er = r.eps;
  const T D_nEn = r.dn[0] - l.dn[0];
  const T D_nEt = r.dn[1] - l.dn[1];
  const T D_nEw = r.dn[2] - l.dn[2];
  const T D_nHn = r.dn[3] - l.dn[3];
  const T D_nHt = r.dn[4] - l.dn[4];
  const T D_nHw = r.dn[5] - l.dn[5];
  const T D_nPh = r.dn[6] - l.dn[6];
  const T D_nPs = r.dn[7] - l.dn[7];
  const T D_tEn = r.dt[0] - l.dt[0];
  const T D_tEt = r.dt[1] - l.dt[1];
  const T D_tEw = r.dt[2] - l.dt[2];
  const T D_tHn = r.dt[3] - l.dt[3];
  const T D_tHt = r.dt[4] - l.dt[4];
  const T D_tHw = r.dt[5] - l.dt[5];
  const T D_tPh = r.dt[6] - l.dt[6];
  const T D_tPs = r.dt[7] - l.dt[7];
  const T D_vEn = r.v[0] - l.v[0];
  const T D_vEt = r.v[1] - l.v[1];
  const T D_vEw = r.v[2] - l.v[2];
  const T D_vHn = r.v[3] - l.v[3];
  const T D_vHt = r.v[4] - l.v[4];
  const T D_vHw = r.v[5] - l.v[5];
  const T D_vPh = r.v[6] - l.v[6];
  const T D_vPs = r.v[7] - l.v[7];
  const T D_wEn = r.dw[0] - l.dw[0];
  const T D_wEt = r.dw[1] - l.dw[1];
  const T D_wEw = r.dw[2] - l.dw[2];
  const T D_wHn = r.dw[3] - l.dw[3];
  const T D_wHt = r.dw[4] - l.dw[4];
  const T D_wHw = r.dw[5] - l.dw[5];
  const T D_wPh = r.dw[6] - l.dw[6];
  const T D_wPs = r.dw[7] - l.dw[7];
  const T DE_vEn = er * r.v[0] - el * l.v[0];
  const T DE_vEt = er * r.v[1] - el * l.v[1];
  const T DE_vEw = er * r.v[2] - el * l.v[2];
  const T S_nHn = l.dn[3] + r.dn[3];
  const T S_nHt = l.dn[4] + r.dn[4];
  const T S_nHw = l.dn[5] + r.dn[5];
  const T S_nPh = l.dn[6] + r.dn[6];
  const T S_nPs = l.dn[7] + r.dn[7];
  const T S_tEn = l.dt[0] + r.dt[0];
  const T S_tEt = l.dt[1] + r.dt[1];
  const T S_tEw = l.dt[2] + r.dt[2];
  const T S_tHn = l.dt[3] + r.dt[3];
  const T S_tHt = l.dt[4] + r.dt[4];
  const T S_tHw = l.dt[5] + r.dt[5];
  const T S_tPh = l.dt[6] + r.dt[6];
  const T S_tPs = l.dt[7] + r.dt[7];
  const T S_vEn = l.v[0] + r.v[0];
  const T S_vEt = l.v[1] + r.v[1];
  const T S_vEw = l.v[2] + r.v[2];
  const T S_vHn = l.v[3] + r.v[3];
  const T S_vHt = l.v[4] + r.v[4];
  const T S_vHw = l.v[5] + r.v[5];
  const T S_vPh = l.v[6] + r.v[6];
  const T S_vPs = l.v[7] + r.v[7];
  const T S_wEn = l.dw[0] + r.dw[0];
  const T S_wEt = l.dw[1] + r.dw[1];
  const T S_wEw = l.dw[2] + r.dw[2];
  const T S_wHn = l.dw[3] + r.dw[3];
  const T S_wHt = l.dw[4] + r.dw[4];
  const T S_wHw = l.dw[5] + r.dw[5];
  const T S_wPh = l.dw[6] + r.dw[6];
  const T S_wPs = l.dw[7] + r.dw[7];
  const T SE_nEn = el * l.dn[0] + er * r.dn[0];
  const T SE_nEt = el * l.dn[1] + er * r.dn[1];
  const T SE_nEw = el * l.dn[2] + er * r.dn[2];
  const T SE_tEn = el * l.dt[0] + er * r.dt[0];
  const T SE_tEt = el * l.dt[1] + er * r.dt[1];
  const T SE_tEw = el * l.dt[2] + er * r.dt[2];
  const T SE_vEn = el * l.v[0] + er * r.v[0];
  const T SE_vEt = el * l.v[1] + er * r.v[1];
  const T SE_vEw = el * l.v[2] + er * r.v[2];
  const T SE_wEn = el * l.dw[0] + er * r.dw[0];
  const T SE_wEt = el * l.dw[1] + er * r.dw[1];
  const T SE_wEw = el * l.dw[2] + er * r.dw[2];
  const T c0 = K.a[0] + K.b[0] * ie;
  const T c1 = K.a[1] + K.b[1] * ie;
  const T c2 = K.b[2] * ie;
  const T c3 = K.a[3] + K.b[3] * ie;
  const T c4 = K.a[4] + K.b[4] * ie;
  const T c5 = K.a[5] + K.b[5] * ie;
  const T c6 = K.b[6] * ie;
  const T c7 = K.a[7] + K.b[7] * ie;
  const T c8 = K.b[8] * ie;
  const T c9 = K.b[9] * ie;
  const T c10 = K.b[10] * ie;
  const T c11 = K.a[11] + K.b[11] * ie;
  const T c12 = K.b[12] * ie;
  const T c13 = K.a[13] + K.b[13] * ie;
  const T c14 = K.b[14] * ie;
  const T c15 = K.b[15] * ie;
  const T c16 = K.a[16] + K.b[16] * ie;
  const T c17 = K.b[17] * ie;
  const T c18 = K.b[18] * ie;
  out[0] = K.k[0] * D_vEn +
      K.k[1] * DE_vEn +
      K.k[2] * S_vPh +
      c0 * SE_nEn +
      c1 * D_nPh +
      c2 * SE_tEt +
      K.k[3] * D_tEw +
      K.k[4] * S_tHt +
      c3 * D_tHw +
      K.k[3] * D_wEt +
      c2 * SE_wEw -
      c3 * D_wHt +
      K.k[5] * S_wHw;
  out[1] = K.k[6] * D_vEt +
      K.k[1] * DE_vEt +
      K.k[7] * S_vHw +
      c4 * SE_nEt +
      c5 * D_nHw +
      c6 * SE_tEn +
      K.k[5] * S_tHn +
      c7 * D_tPh +
      K.k[8] * D_tPs +
      K.k[9] * D_wEn +
      K.k[10] * D_wHn +
      K.k[11] * S_wPh +
      K.k[12] * S_wPs;
  out[2] = K.k[6] * D_vEw +
      K.k[1] * DE_vEw +
      K.k[13] * S_vHt +
      c4 * SE_nEw -
      c5 * D_nHt +
      K.k[9] * D_tEn +
      K.k[14] * D_tHn +
      K.k[11] * S_tPh +
      K.k[15] * S_tPs +
      c6 * SE_wEn +
      K.k[4] * S_wHn +
      c7 * D_wPh +
      K.k[16] * D_wPs;
  out[3] = K.k[17] * D_vHn +
      K.k[18] * S_vPs +
      K.k[19] * S_nHn +
      K.k[20] * D_nPs +
      K.k[21] * S_tEt +
      c8 * SE_tEt +
      K.k[14] * D_tEw +
      K.k[22] * S_tHt +
      c9 * D_tHw +
      K.k[10] * D_wEt +
      K.k[23] * S_wEw -
      c8 * SE_wEw +
      c9 * D_wHt +
      K.k[22] * S_wHw;
  out[4] = K.k[24] * S_vEw +
      c10 * SE_vEw +
      c11 * D_vHt -
      c5 * D_nEw +
      c4 * S_nHt +
      K.k[23] * S_tEn -
      c8 * SE_tEn +
      c6 * S_tHn +
      c12 * D_tPh +
      c13 * D_tPs -
      c3 * D_wEn +
      K.k[25] * D_wHn +
      c14 * S_wPh +
      K.k[26] * S_wPs;
  out[5] = K.k[27] * S_vEt -
      c10 * SE_vEt +
      c11 * D_vHw +
      c5 * D_nEt +
      c4 * S_nHw +
      c3 * D_tEn +
      K.k[25] * D_tHn -
      c14 * S_tPh +
      K.k[26] * S_tPs +
      K.k[21] * S_wEn +
      c8 * SE_wEn +
      c6 * S_wHn -
      c12 * D_wPh +
      c13 * D_wPs;
  out[6] = K.k[28] * S_vEn +
      c15 * SE_vEn +
      c16 * D_vPh +
      c1 * D_nEn +
      c0 * S_nPh +
      c7 * D_tEt +
      K.k[29] * S_tEw +
      c17 * SE_tEw -
      c12 * D_tHt +
      c14 * S_tHw +
      K.k[29] * S_wEt +
      c17 * SE_wEt +
      c7 * D_wEw -
      c14 * S_wHt +
      c12 * D_wHw;
  out[7] = K.k[18] * S_vHn +
      K.k[17] * D_vPs +
      K.k[20] * D_nHn +
      K.k[19] * S_nPs +
      K.k[16] * D_tEt +
      c18 * SE_tEw +
      c13 * D_tHt +
      K.k[26] * S_tHw -
      c18 * SE_wEt +
      K.k[8] * D_wEw +
      K.k[26] * S_wHt +
      c13 * D_wHw;
}

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
