// GENERATED by paper_2412_16845_gb300/codegen.py from the D3Q4 sums of Sec. 3.1; do not
// edit by hand (regenerate with `python -m paper_2412_16845_gb300.codegen`).
//
// Side-split face flux of the 3-D Cartesian step with mu = 1.  The flux through the face
// between cells L and R along axis A (global components, times dt/h_A) is
//     F = (Ev_L + Od_L) + (Ev_R - Od_R) + ie [(EvQ_L + OdQ_L) + (EvQ_R - OdQ_R)],
//     ie = 2 / (eps_L + eps_R),
// where Ev, Od, EvQ, OdQ of a cell are linear in its state v, its raw central differences
// d[j] = V(+e_j) - V(-e_j) and the eps-weighted E rows ev = eps E, ed[j] = eps d[j] (E
// rows).  A non-reflecting face takes zero for the ghost's four vectors and ie = 1/eps of
// the cell.
#pragma once

#include <cmath>

namespace gks {

constexpr int kSide3K = 36;   // coefficient slots per axis

// Coefficient slots of axis A (0 = x, 1 = y, 2 = z) from C1..C5 of Sec. 3.1, the cell
// sizes h[3] and the lattice speed c.  Unused slots are zero.
inline void side3_coefficients(const double C[5], const double h[3], double c, int A,
                               double k[kSide3K]) {
  const double K1 = C[0] / h[A], K2 = C[1] / h[A], K3 = C[2] / h[A], K4 = C[3] / h[A],
               K5 = C[4] / h[A];
  const double ih0 = 0.5 / h[0], ih1 = 0.5 / h[1], ih2 = 0.5 / h[2];
  (void)K1; (void)K2; (void)K3; (void)K4; (void)K5; (void)ih0; (void)ih1; (void)ih2;
  for (int i = 0; i < kSide3K; ++i) k[i] = 0.0;
  if (A == 0) {
    k[0] = (1.0/2.0)*c*ih1*(K2 - K5);
    k[1] = -1.0/2.0*c*ih2*(K2 - K5);
    k[2] = (1.0/8.0)*c*(4*K2*c*ih0 + K4 - 4*K5*c*ih0);
    k[3] = (1.0/2.0)*(K1 + K4);
    k[4] = (1.0/8.0)*K1/c;
    k[5] = -1.0/2.0*c*ih1*(K2 - K5);
    k[6] = -1.0/2.0*(K1 + K4);
    k[7] = (1.0/2.0)*c*ih2*(K2 - K5);
    k[8] = (1.0/2.0)*K5*c*ih1;
    k[9] = -1.0/2.0*K5*c*ih2;
    k[10] = -1.0/2.0*K4;
    k[11] = -1.0/2.0*K5*c*ih1;
    k[12] = (1.0/2.0)*K4;
    k[13] = (1.0/2.0)*K5*c*ih2;
    k[14] = -1.0/2.0*K3*ih0;
    k[15] = (1.0/2.0)*K3*ih1;
    k[16] = (1.0/2.0)*K3*ih2;
    k[17] = -1.0/2.0*K2*c*ih1;
    k[18] = (1.0/2.0)*K2*c*ih2;
    k[19] = -1.0/8.0*(-K1 + 4*K3*c*ih0)/c;
    k[20] = -1.0/2.0*K1;
    k[21] = (1.0/2.0)*K2*c*ih1;
    k[22] = (1.0/2.0)*K1;
    k[23] = -1.0/2.0*K2*c*ih2;
    k[24] = -1.0/2.0*K2*ih1;
    k[25] = -1.0/2.0*K2*ih2;
    k[26] = (1.0/2.0)*K4*c;
    k[27] = (1.0/2.0)*K1/c;
    k[28] = (1.0/8.0)*(K1 + 4*K2*c*ih0 + K4 - 4*K5*c*ih0);
    k[29] = -1.0/8.0*(K1 + 4*K2*c*ih0 + K4 - 4*K5*c*ih0);
    k[30] = -1.0/8.0*(4*K2*c*ih0 + K4 - 4*K5*c*ih0);
    k[31] = (1.0/8.0)*(4*K2*c*ih0 + K4 - 4*K5*c*ih0);
    k[32] = -1.0/2.0*K3*ih0/c;
    k[33] = (1.0/2.0)*K3*ih0/c;
    k[34] = -1.0/8.0*K1;
    k[35] = (1.0/8.0)*K1;
  }
  if (A == 1) {
    k[0] = -1.0/2.0*(K1 + K4);
    k[1] = -1.0/2.0*c*ih0*(K2 - K5);
    k[2] = (1.0/8.0)*K1/c;
    k[3] = (1.0/8.0)*c*(4*K2*c*ih1 + K4 - 4*K5*c*ih1);
    k[4] = (1.0/2.0)*c*ih0*(K2 - K5);
    k[5] = -1.0/2.0*c*ih2*(K2 - K5);
    k[6] = (1.0/2.0)*(K1 + K4);
    k[7] = (1.0/2.0)*c*ih2*(K2 - K5);
    k[8] = (1.0/2.0)*K4;
    k[9] = -1.0/2.0*K5*c*ih0;
    k[10] = (1.0/2.0)*K5*c*ih0;
    k[11] = -1.0/2.0*K5*c*ih2;
    k[12] = -1.0/2.0*K4;
    k[13] = (1.0/2.0)*K5*c*ih2;
    k[14] = (1.0/2.0)*K3*ih0;
    k[15] = -1.0/2.0*K3*ih1;
    k[16] = (1.0/2.0)*K3*ih2;
    k[17] = -1.0/8.0*(-K1 + 4*K3*c*ih1)/c;
    k[18] = (1.0/2.0)*K1;
    k[19] = (1.0/2.0)*K2*c*ih0;
    k[20] = -1.0/2.0*K2*c*ih0;
    k[21] = (1.0/2.0)*K2*c*ih2;
    k[22] = -1.0/2.0*K1;
    k[23] = -1.0/2.0*K2*c*ih2;
    k[24] = (1.0/2.0)*K1/c;
    k[25] = -1.0/8.0*(K1 + 4*K2*c*ih1 + K4 - 4*K5*c*ih1);
    k[26] = (1.0/2.0)*K4*c;
    k[27] = (1.0/2.0)*K2*ih0;
    k[28] = (1.0/2.0)*K2*ih2;
    k[29] = (1.0/8.0)*(K1 + 4*K2*c*ih1 + K4 - 4*K5*c*ih1);
    k[30] = (1.0/8.0)*(4*K2*c*ih1 + K4 - 4*K5*c*ih1);
    k[31] = -1.0/8.0*(4*K2*c*ih1 + K4 - 4*K5*c*ih1);
    k[32] = (1.0/2.0)*K3*ih1/c;
    k[33] = -1.0/2.0*K3*ih1/c;
    k[34] = (1.0/8.0)*K1;
    k[35] = -1.0/8.0*K1;
  }
  if (A == 2) {
    k[0] = (1.0/2.0)*(K1 + K4);
    k[1] = (1.0/2.0)*c*ih0*(K2 - K5);
    k[2] = (1.0/8.0)*K1/c;
    k[3] = (1.0/8.0)*c*(4*K2*c*ih2 + K4 - 4*K5*c*ih2);
    k[4] = -1.0/2.0*(K1 + K4);
    k[5] = -1.0/2.0*c*ih1*(K2 - K5);
    k[6] = -1.0/2.0*c*ih0*(K2 - K5);
    k[7] = (1.0/2.0)*c*ih1*(K2 - K5);
    k[8] = -1.0/2.0*K4;
    k[9] = (1.0/2.0)*K5*c*ih0;
    k[10] = (1.0/2.0)*K4;
    k[11] = -1.0/2.0*K5*c*ih1;
    k[12] = -1.0/2.0*K5*c*ih0;
    k[13] = (1.0/2.0)*K5*c*ih1;
    k[14] = (1.0/2.0)*K3*ih0;
    k[15] = -1.0/2.0*K3*ih2;
    k[16] = (1.0/2.0)*K3*ih1;
    k[17] = -1.0/8.0*(-K1 + 4*K3*c*ih2)/c;
    k[18] = -1.0/2.0*K1;
    k[19] = -1.0/2.0*K2*c*ih0;
    k[20] = (1.0/2.0)*K1;
    k[21] = (1.0/2.0)*K2*c*ih1;
    k[22] = (1.0/2.0)*K2*c*ih0;
    k[23] = -1.0/2.0*K2*c*ih1;
    k[24] = (1.0/2.0)*K1/c;
    k[25] = (1.0/8.0)*(K1 + 4*K2*c*ih2 + K4 - 4*K5*c*ih2);
    k[26] = (1.0/2.0)*K4*c;
    k[27] = -1.0/8.0*(K1 + 4*K2*c*ih2 + K4 - 4*K5*c*ih2);
    k[28] = (1.0/2.0)*K2*ih0;
    k[29] = (1.0/2.0)*K2*ih1;
    k[30] = -1.0/8.0*(4*K2*c*ih2 + K4 - 4*K5*c*ih2);
    k[31] = (1.0/8.0)*(4*K2*c*ih2 + K4 - 4*K5*c*ih2);
    k[32] = -1.0/2.0*K3*ih2/c;
    k[33] = (1.0/2.0)*K3*ih2/c;
    k[34] = -1.0/8.0*K1;
    k[35] = (1.0/8.0)*K1;
  }
}

// Ev, Od, EvQ, OdQ of one cell for faces along axis A, returned as the cell's l-side
// vectors (pl, ql: its face at +1/2) and r-side vectors (pr, qr: its face at -1/2).
// OP supplies mul(k, x), fma(k, x, acc), add, sub for the value type T (a scalar or a
// pair of cells); k holds the slots of axis A in the form OP expects.
template <int A, class OP, class T, class KT>
__device__ __forceinline__ void side3(const T v[6], const T d[3][6], const T ev[3],
                                      const T ed[3][3], const KT *k, T pl[6], T pr[6],
                                      T ql[6], T qr[6]) {
  if constexpr (A == 0) {
    T evp0 = OP::mul(k[0], d[1][4]);
    evp0 = OP::fma(k[1], d[2][5], evp0);
    evp0 = OP::fma(k[2], ed[0][0], evp0);
    T odp0 = OP::mul(k[24], d[1][2]);
    odp0 = OP::fma(k[8], d[1][5], odp0);
    odp0 = OP::fma(k[25], d[2][1], odp0);
    odp0 = OP::fma(k[9], d[2][4], odp0);
    odp0 = OP::fma(k[26], ev[0], odp0);
    pl[0] = OP::add(evp0, odp0); pr[0] = OP::sub(evp0, odp0);
    ql[0] = OP::zero(); qr[0] = OP::zero();
    T evp1 = OP::mul(k[3], v[5]);
    evp1 = OP::fma(k[4], d[0][1], evp1);
    evp1 = OP::fma(k[5], d[1][3], evp1);
    evp1 = OP::fma(k[2], ed[0][1], evp1);
    T odp1 = OP::mul(k[27], v[1]);
    odp1 = OP::fma(k[28], d[0][5], odp1);
    odp1 = OP::fma(k[13], d[2][3], odp1);
    odp1 = OP::fma(k[26], ev[1], odp1);
    T evq1 = OP::mul(k[14], ed[0][1]);
    evq1 = OP::fma(k[15], ed[1][0], evq1);
    T odq1 = OP::mul(k[32], d[0][5]);
    pl[1] = OP::add(evp1, odp1); pr[1] = OP::sub(evp1, odp1);
    ql[1] = OP::add(evq1, odq1); qr[1] = OP::sub(evq1, odq1);
    T evp2 = OP::mul(k[6], v[4]);
    evp2 = OP::fma(k[4], d[0][2], evp2);
    evp2 = OP::fma(k[7], d[2][3], evp2);
    evp2 = OP::fma(k[2], ed[0][2], evp2);
    T odp2 = OP::mul(k[27], v[2]);
    odp2 = OP::fma(k[29], d[0][4], odp2);
    odp2 = OP::fma(k[11], d[1][3], odp2);
    odp2 = OP::fma(k[26], ev[2], odp2);
    T evq2 = OP::mul(k[14], ed[0][2]);
    evq2 = OP::fma(k[16], ed[2][0], evq2);
    T odq2 = OP::mul(k[33], d[0][4]);
    pl[2] = OP::add(evp2, odp2); pr[2] = OP::sub(evp2, odp2);
    ql[2] = OP::add(evq2, odq2); qr[2] = OP::sub(evq2, odq2);
    T evp3 = OP::mul(k[2], d[0][3]);
    evp3 = OP::fma(k[8], d[1][1], evp3);
    evp3 = OP::fma(k[9], d[2][2], evp3);
    T odp3 = OP::mul(k[26], v[3]);
    odp3 = OP::fma(k[11], d[1][2], odp3);
    odp3 = OP::fma(k[13], d[2][1], odp3);
    T evq3 = OP::mul(k[17], ed[1][1]);
    evq3 = OP::fma(k[18], ed[2][2], evq3);
    T odq3 = OP::mul(k[24], d[1][5]);
    odq3 = OP::fma(k[25], d[2][4], odq3);
    pl[3] = OP::add(evp3, odp3); pr[3] = OP::sub(evp3, odp3);
    ql[3] = OP::add(evq3, odq3); qr[3] = OP::sub(evq3, odq3);
    T evp4 = OP::mul(k[10], v[2]);
    evp4 = OP::fma(k[2], d[0][4], evp4);
    evp4 = OP::fma(k[11], d[1][0], evp4);
    T odp4 = OP::mul(k[26], v[4]);
    odp4 = OP::fma(k[30], d[0][2], odp4);
    odp4 = OP::fma(k[9], d[2][0], odp4);
    T evq4 = OP::mul(k[19], d[0][4]);
    evq4 = OP::fma(k[15], d[1][3], evq4);
    evq4 = OP::fma(k[20], ev[2], evq4);
    evq4 = OP::fma(k[21], ed[1][0], evq4);
    T odq4 = OP::mul(k[27], v[4]);
    odq4 = OP::fma(k[33], d[0][2], odq4);
    odq4 = OP::fma(k[34], ed[0][2], odq4);
    pl[4] = OP::add(evp4, odp4); pr[4] = OP::sub(evp4, odp4);
    ql[4] = OP::add(evq4, odq4); qr[4] = OP::sub(evq4, odq4);
    T evp5 = OP::mul(k[12], v[1]);
    evp5 = OP::fma(k[2], d[0][5], evp5);
    evp5 = OP::fma(k[13], d[2][0], evp5);
    T odp5 = OP::mul(k[26], v[5]);
    odp5 = OP::fma(k[31], d[0][1], odp5);
    odp5 = OP::fma(k[8], d[1][0], odp5);
    T evq5 = OP::mul(k[19], d[0][5]);
    evq5 = OP::fma(k[16], d[2][3], evq5);
    evq5 = OP::fma(k[22], ev[1], evq5);
    evq5 = OP::fma(k[23], ed[2][0], evq5);
    T odq5 = OP::mul(k[27], v[5]);
    odq5 = OP::fma(k[32], d[0][1], odq5);
    odq5 = OP::fma(k[35], ed[0][1], odq5);
    pl[5] = OP::add(evp5, odp5); pr[5] = OP::sub(evp5, odp5);
    ql[5] = OP::add(evq5, odq5); qr[5] = OP::sub(evq5, odq5);
  }
  if constexpr (A == 1) {
    T evp0 = OP::mul(k[0], v[5]);
    evp0 = OP::fma(k[1], d[0][4], evp0);
    evp0 = OP::fma(k[2], d[1][0], evp0);
    evp0 = OP::fma(k[3], ed[1][0], evp0);
    T odp0 = OP::mul(k[24], v[0]);
    odp0 = OP::fma(k[25], d[1][5], odp0);
    odp0 = OP::fma(k[11], d[2][4], odp0);
    odp0 = OP::fma(k[26], ev[0], odp0);
    T evq0 = OP::mul(k[14], ed[0][1]);
    evq0 = OP::fma(k[15], ed[1][0], evq0);
    T odq0 = OP::mul(k[32], d[1][5]);
    pl[0] = OP::add(evp0, odp0); pr[0] = OP::sub(evp0, odp0);
    ql[0] = OP::add(evq0, odq0); qr[0] = OP::sub(evq0, odq0);
    T evp1 = OP::mul(k[4], d[0][3]);
    evp1 = OP::fma(k[5], d[2][5], evp1);
    evp1 = OP::fma(k[3], ed[1][1], evp1);
    T odp1 = OP::mul(k[27], d[0][2]);
    odp1 = OP::fma(k[9], d[0][5], odp1);
    odp1 = OP::fma(k[28], d[2][0], odp1);
    odp1 = OP::fma(k[13], d[2][3], odp1);
    odp1 = OP::fma(k[26], ev[1], odp1);
    pl[1] = OP::add(evp1, odp1); pr[1] = OP::sub(evp1, odp1);
    ql[1] = OP::zero(); qr[1] = OP::zero();
    T evp2 = OP::mul(k[6], v[3]);
    evp2 = OP::fma(k[2], d[1][2], evp2);
    evp2 = OP::fma(k[7], d[2][4], evp2);
    evp2 = OP::fma(k[3], ed[1][2], evp2);
    T odp2 = OP::mul(k[24], v[2]);
    odp2 = OP::fma(k[10], d[0][4], odp2);
    odp2 = OP::fma(k[29], d[1][3], odp2);
    odp2 = OP::fma(k[26], ev[2], odp2);
    T evq2 = OP::mul(k[15], ed[1][2]);
    evq2 = OP::fma(k[16], ed[2][1], evq2);
    T odq2 = OP::mul(k[33], d[1][3]);
    pl[2] = OP::add(evp2, odp2); pr[2] = OP::sub(evp2, odp2);
    ql[2] = OP::add(evq2, odq2); qr[2] = OP::sub(evq2, odq2);
    T evp3 = OP::mul(k[8], v[2]);
    evp3 = OP::fma(k[9], d[0][1], evp3);
    evp3 = OP::fma(k[3], d[1][3], evp3);
    T odp3 = OP::mul(k[26], v[3]);
    odp3 = OP::fma(k[30], d[1][2], odp3);
    odp3 = OP::fma(k[13], d[2][1], odp3);
    T evq3 = OP::mul(k[14], d[0][4]);
    evq3 = OP::fma(k[17], d[1][3], evq3);
    evq3 = OP::fma(k[18], ev[2], evq3);
    evq3 = OP::fma(k[19], ed[0][1], evq3);
    T odq3 = OP::mul(k[24], v[3]);
    odq3 = OP::fma(k[33], d[1][2], odq3);
    odq3 = OP::fma(k[34], ed[1][2], odq3);
    pl[3] = OP::add(evp3, odp3); pr[3] = OP::sub(evp3, odp3);
    ql[3] = OP::add(evq3, odq3); qr[3] = OP::sub(evq3, odq3);
    T evp4 = OP::mul(k[10], d[0][0]);
    evp4 = OP::fma(k[3], d[1][4], evp4);
    evp4 = OP::fma(k[11], d[2][2], evp4);
    T odp4 = OP::mul(k[26], v[4]);
    odp4 = OP::fma(k[10], d[0][2], odp4);
    odp4 = OP::fma(k[11], d[2][0], odp4);
    T evq4 = OP::mul(k[20], ed[0][0]);
    evq4 = OP::fma(k[21], ed[2][2], evq4);
    T odq4 = OP::mul(k[27], d[0][5]);
    odq4 = OP::fma(k[28], d[2][3], odq4);
    pl[4] = OP::add(evp4, odp4); pr[4] = OP::sub(evp4, odp4);
    ql[4] = OP::add(evq4, odq4); qr[4] = OP::sub(evq4, odq4);
    T evp5 = OP::mul(k[12], v[0]);
    evp5 = OP::fma(k[3], d[1][5], evp5);
    evp5 = OP::fma(k[13], d[2][1], evp5);
    T odp5 = OP::mul(k[26], v[5]);
    odp5 = OP::fma(k[9], d[0][1], odp5);
    odp5 = OP::fma(k[31], d[1][0], odp5);
    T evq5 = OP::mul(k[17], d[1][5]);
    evq5 = OP::fma(k[16], d[2][4], evq5);
    evq5 = OP::fma(k[22], ev[0], evq5);
    evq5 = OP::fma(k[23], ed[2][1], evq5);
    T odq5 = OP::mul(k[24], v[5]);
    odq5 = OP::fma(k[32], d[1][0], odq5);
    odq5 = OP::fma(k[35], ed[1][0], odq5);
    pl[5] = OP::add(evp5, odp5); pr[5] = OP::sub(evp5, odp5);
    ql[5] = OP::add(evq5, odq5); qr[5] = OP::sub(evq5, odq5);
  }
  if constexpr (A == 2) {
    T evp0 = OP::mul(k[0], v[4]);
    evp0 = OP::fma(k[1], d[0][5], evp0);
    evp0 = OP::fma(k[2], d[2][0], evp0);
    evp0 = OP::fma(k[3], ed[2][0], evp0);
    T odp0 = OP::mul(k[24], v[0]);
    odp0 = OP::fma(k[13], d[1][5], odp0);
    odp0 = OP::fma(k[25], d[2][4], odp0);
    odp0 = OP::fma(k[26], ev[0], odp0);
    T evq0 = OP::mul(k[14], ed[0][2]);
    evq0 = OP::fma(k[15], ed[2][0], evq0);
    T odq0 = OP::mul(k[32], d[2][4]);
    pl[0] = OP::add(evp0, odp0); pr[0] = OP::sub(evp0, odp0);
    ql[0] = OP::add(evq0, odq0); qr[0] = OP::sub(evq0, odq0);
    T evp1 = OP::mul(k[4], v[3]);
    evp1 = OP::fma(k[5], d[1][5], evp1);
    evp1 = OP::fma(k[2], d[2][1], evp1);
    evp1 = OP::fma(k[3], ed[2][1], evp1);
    T odp1 = OP::mul(k[24], v[1]);
    odp1 = OP::fma(k[12], d[0][5], odp1);
    odp1 = OP::fma(k[27], d[2][3], odp1);
    odp1 = OP::fma(k[26], ev[1], odp1);
    T evq1 = OP::mul(k[16], ed[1][2]);
    evq1 = OP::fma(k[15], ed[2][1], evq1);
    T odq1 = OP::mul(k[33], d[2][3]);
    pl[1] = OP::add(evp1, odp1); pr[1] = OP::sub(evp1, odp1);
    ql[1] = OP::add(evq1, odq1); qr[1] = OP::sub(evq1, odq1);
    T evp2 = OP::mul(k[6], d[0][3]);
    evp2 = OP::fma(k[7], d[1][4], evp2);
    evp2 = OP::fma(k[3], ed[2][2], evp2);
    T odp2 = OP::mul(k[28], d[0][1]);
    odp2 = OP::fma(k[9], d[0][4], odp2);
    odp2 = OP::fma(k[29], d[1][0], odp2);
    odp2 = OP::fma(k[11], d[1][3], odp2);
    odp2 = OP::fma(k[26], ev[2], odp2);
    pl[2] = OP::add(evp2, odp2); pr[2] = OP::sub(evp2, odp2);
    ql[2] = OP::zero(); qr[2] = OP::zero();
    T evp3 = OP::mul(k[8], v[1]);
    evp3 = OP::fma(k[9], d[0][2], evp3);
    evp3 = OP::fma(k[3], d[2][3], evp3);
    T odp3 = OP::mul(k[26], v[3]);
    odp3 = OP::fma(k[11], d[1][2], odp3);
    odp3 = OP::fma(k[30], d[2][1], odp3);
    T evq3 = OP::mul(k[14], d[0][5]);
    evq3 = OP::fma(k[17], d[2][3], evq3);
    evq3 = OP::fma(k[18], ev[1], evq3);
    evq3 = OP::fma(k[19], ed[0][2], evq3);
    T odq3 = OP::mul(k[24], v[3]);
    odq3 = OP::fma(k[33], d[2][1], odq3);
    odq3 = OP::fma(k[34], ed[2][1], odq3);
    pl[3] = OP::add(evp3, odp3); pr[3] = OP::sub(evp3, odp3);
    ql[3] = OP::add(evq3, odq3); qr[3] = OP::sub(evq3, odq3);
    T evp4 = OP::mul(k[10], v[0]);
    evp4 = OP::fma(k[11], d[1][2], evp4);
    evp4 = OP::fma(k[3], d[2][4], evp4);
    T odp4 = OP::mul(k[26], v[4]);
    odp4 = OP::fma(k[9], d[0][2], odp4);
    odp4 = OP::fma(k[31], d[2][0], odp4);
    T evq4 = OP::mul(k[16], d[1][5]);
    evq4 = OP::fma(k[17], d[2][4], evq4);
    evq4 = OP::fma(k[20], ev[0], evq4);
    evq4 = OP::fma(k[21], ed[1][2], evq4);
    T odq4 = OP::mul(k[24], v[4]);
    odq4 = OP::fma(k[32], d[2][0], odq4);
    odq4 = OP::fma(k[35], ed[2][0], odq4);
    pl[4] = OP::add(evp4, odp4); pr[4] = OP::sub(evp4, odp4);
    ql[4] = OP::add(evq4, odq4); qr[4] = OP::sub(evq4, odq4);
    T evp5 = OP::mul(k[12], d[0][0]);
    evp5 = OP::fma(k[13], d[1][1], evp5);
    evp5 = OP::fma(k[3], d[2][5], evp5);
    T odp5 = OP::mul(k[26], v[5]);
    odp5 = OP::fma(k[12], d[0][1], odp5);
    odp5 = OP::fma(k[13], d[1][0], odp5);
    T evq5 = OP::mul(k[22], ed[0][0]);
    evq5 = OP::fma(k[23], ed[1][1], evq5);
    T odq5 = OP::mul(k[28], d[0][4]);
    odq5 = OP::fma(k[29], d[1][3], odq5);
    pl[5] = OP::add(evp5, odp5); pr[5] = OP::sub(evp5, odp5);
    ql[5] = OP::add(evq5, odq5); qr[5] = OP::sub(evq5, odq5);
  }
}

}  // namespace gks
