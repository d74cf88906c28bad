// GENERATED by paper_2412_16845_gb300/codegen.py from the D3Q4 sums of Sec. 3.1 for the
// divergence-cleaning system of Sec. 2.1; do not edit by hand (regenerate with
// `python -m paper_2412_16845_gb300.codegen`).
//
// Interior-face flux of the cleaning system with mu = 1 in the face frame (components En,
// Et, Ew, Hn, Ht, Hw, phi, psi; times dt/h), folded: every term is a coefficient times a
// sum S(x) = x_l + x_r, a difference D(x) = x_r - x_l or their eps-weighted forms
// SE(x) = eps_l x_l + eps_r x_r, DE(x) = eps_r x_r - eps_l x_l of one side quantity x
// (reconstructed value v, derivative along n, t or w).  A coefficient is a constant k[] or
// a[] + b[] ie with ie = 2/(eps_l + eps_r), both polynomials in C_i/h, c, chi and gamma
// folded on the host.  Included by gks_flux3.cuh after Side8.
#pragma once

#include <cmath>

namespace gks {

template <typename T>
struct F8K {
  T k[23];
  T a[19], b[19];
};

template <typename T>
inline F8K<T> make_f8k(const double C[5], double h, double c, double chi, double gam) {
  const double K1 = C[0] / h, K2 = C[1] / h, K3 = C[2] / h, K4 = C[3] / h, K5 = C[4] / h;
  (void)K1; (void)K2; (void)K3; (void)K4; (void)K5; (void)chi; (void)gam;
  F8K<T> f;
  f.k[0] = T(-1.0/2.0*K1*std::pow(chi, 2)/c);
  f.k[1] = T(-1.0/2.0*K4*c);
  f.k[2] = T((1.0/2.0)*chi*(K1 + K4));
  f.k[3] = T((1.0/2.0)*K2);
  f.k[4] = T((1.0/2.0)*c*(K2 - K5));
  f.k[5] = T(-1.0/2.0*K1/c);
  f.k[6] = T((1.0/2.0)*(K1 + K4));
  f.k[7] = T((1.0/2.0)*K2*gam);
  f.k[8] = T(-1.0/2.0*K2*std::pow(chi, 2));
  f.k[9] = T(-1.0/2.0*(-K3*std::pow(gam, 2) + K5*std::pow(c, 2))/c);
  f.k[10] = T((1.0/2.0)*c*chi*(K2 - K5));
  f.k[11] = T(-1.0/2.0*K3*gam);
  f.k[12] = T(-1.0/2.0*(K1*std::pow(gam, 2) + K4*std::pow(c, 2))/c);
  f.k[13] = T((1.0/2.0)*gam*(K1 + K4));
  f.k[14] = T((1.0/2.0)*(K2*std::pow(c, 2) - K3*std::pow(gam, 2) - K5*std::pow(c, 2)));
  f.k[15] = T(-1.0/2.0*gam*(K2*std::pow(c, 2) - K3*std::pow(gam, 2) - K5*std::pow(c, 2))/c);
  f.k[16] = T((1.0/2.0)*K5*c);
  f.k[17] = T(-1.0/2.0*K3*std::pow(gam, 2));
  f.k[18] = T(-1.0/2.0*K4);
  f.k[19] = T(-1.0/2.0*K2*std::pow(gam, 2));
  f.k[20] = T((1.0/2.0)*c*gam*(K2 - K5));
  f.k[21] = T((1.0/2.0)*K4*chi);
  f.k[22] = T(-1.0/2.0*K5*c*chi);
  f.a[0] = T((1.0/2.0)*std::pow(c, 2)*(K2 - K5));
  f.b[0] = T(-1.0/2.0*K3*std::pow(chi, 2));
  f.a[1] = T(-1.0/2.0*c*chi*(K2 - K5));
  f.b[1] = T((1.0/2.0)*K3*std::pow(chi, 3)/c);
  f.a[2] = T(0);
  f.b[2] = T(-1.0/2.0*K3*std::pow(chi, 2));
  f.a[3] = T(-1.0/2.0*K5*c);
  f.b[3] = T((1.0/2.0)*K3*std::pow(chi, 2)/c);
  f.a[4] = T((1.0/2.0)*std::pow(c, 2)*(K2 - K5));
  f.b[4] = T(-1.0/2.0*K3);
  f.a[5] = T(-1.0/2.0*c*(K2 - K5));
  f.b[5] = T((1.0/2.0)*K3/c);
  f.a[6] = T(0);
  f.b[6] = T((1.0/2.0)*K3);
  f.a[7] = T((1.0/2.0)*K5*c*chi);
  f.b[7] = T(-1.0/2.0*K3*chi/c);
  f.a[8] = T(0);
  f.b[8] = T(-1.0/2.0*K2*c);
  f.a[9] = T(0);
  f.b[9] = T((1.0/2.0)*K2);
  f.a[10] = T(0);
  f.b[10] = T(-1.0/2.0*K1);
  f.a[11] = T(-1.0/2.0*K4*c);
  f.b[11] = T(-1.0/2.0*K1/c);
  f.a[12] = T(0);
  f.b[12] = T(-1.0/2.0*K2*chi);
  f.a[13] = T((1.0/2.0)*K5*c*gam);
  f.b[13] = T(-1.0/2.0*K3*gam/c);
  f.a[14] = T(0);
  f.b[14] = T((1.0/2.0)*K3*chi);
  f.a[15] = T(0);
  f.b[15] = T((1.0/2.0)*K1*chi);
  f.a[16] = T(-1.0/2.0*K4*c);
  f.b[16] = T(-1.0/2.0*K1*std::pow(chi, 2)/c);
  f.a[17] = T(0);
  f.b[17] = T((1.0/2.0)*K2*c*chi);
  f.a[18] = T(0);
  f.b[18] = T(-1.0/2.0*K3*gam);
  return f;
}

template <typename T>
__device__ __forceinline__ void flux3_phm_mu1(const Side8<T> &l, const Side8<T> &r,
                                              const F8K<T> &K, T ie, T out[8]) {
  const T el = l.eps, er = r.eps;
  (void)el; (void)er;
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
  out[0] = K.k[0] * D_vEn + K.k[1] * DE_vEn + K.k[2] * S_vPh + c0 * SE_nEn + c1 * D_nPh + c2 * SE_tEt + K.k[3] * D_tEw + K.k[4] * S_tHt + c3 * D_tHw + K.k[3] * D_wEt + c2 * SE_wEw - c3 * D_wHt - K.k[4] * S_wHw;
  out[1] = K.k[5] * D_vEt + K.k[1] * DE_vEt + K.k[6] * S_vHw + c4 * SE_nEt + c5 * D_nHw + c6 * SE_tEn - K.k[4] * S_tHn + c7 * D_tPh + K.k[7] * D_tPs + K.k[8] * D_wEn + K.k[9] * D_wHn + K.k[10] * S_wPh + K.k[11] * S_wPs;
  out[2] = K.k[5] * D_vEw + K.k[1] * DE_vEw - K.k[6] * S_vHt + c4 * SE_nEw - c5 * D_nHt + K.k[8] * D_tEn - K.k[9] * D_tHn + K.k[10] * S_tPh - K.k[11] * S_tPs + c6 * SE_wEn + K.k[4] * S_wHn + c7 * D_wPh - K.k[7] * D_wPs;
  out[3] = K.k[12] * D_vHn + K.k[13] * S_vPs + K.k[14] * S_nHn + K.k[15] * D_nPs + K.k[16] * S_tEt + c8 * SE_tEt - K.k[9] * D_tEw + K.k[17] * S_tHt + c9 * D_tHw + K.k[9] * D_wEt - K.k[16] * S_wEw - c8 * SE_wEw + c9 * D_wHt + K.k[17] * S_wHw;
  out[4] = K.k[18] * S_vEw + c10 * SE_vEw + c11 * D_vHt - c5 * D_nEw + c4 * S_nHt - K.k[16] * S_tEn - c8 * SE_tEn + c6 * S_tHn + c12 * D_tPh + c13 * D_tPs - c3 * D_wEn + K.k[19] * D_wHn + c14 * S_wPh + K.k[20] * S_wPs;
  out[5] = -K.k[18] * S_vEt - c10 * SE_vEt + c11 * D_vHw + c5 * D_nEt + c4 * S_nHw + c3 * D_tEn + K.k[19] * D_tHn - c14 * S_tPh + K.k[20] * S_tPs + K.k[16] * S_wEn + c8 * SE_wEn + c6 * S_wHn - c12 * D_wPh + c13 * D_wPs;
  out[6] = K.k[21] * S_vEn + c15 * SE_vEn + c16 * D_vPh + c1 * D_nEn + c0 * S_nPh + c7 * D_tEt + K.k[22] * S_tEw + c17 * SE_tEw - c12 * D_tHt + c14 * S_tHw + K.k[22] * S_wEt + c17 * SE_wEt + c7 * D_wEw - c14 * S_wHt + c12 * D_wHw;
  out[7] = K.k[13] * S_vHn + K.k[12] * D_vPs + K.k[15] * D_nHn + K.k[14] * S_nPs - K.k[7] * D_tEt + c18 * SE_tEw + c13 * D_tHt + K.k[20] * S_tHw - c18 * SE_wEt + K.k[7] * D_wEw + K.k[20] * S_wHt + c13 * D_wHw;
}

}  // namespace gks
