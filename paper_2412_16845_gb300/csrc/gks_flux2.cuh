// Combined flux constants of 2-D TM faces, shared by the forward step and its adjoint.
#pragma once

#include <cuda_runtime.h>

namespace gks {

// ------------------------------------------------------------------ flux coefficients
// Combined constants of one face orientation (K_i = C_i / h_normal, c the lattice speed,
// sb / st the signs of the tangential H component and of the tangential derivative in the face
// frame): see face_flux() in gks_cart2d.cu for how they enter.
template <typename T>
struct FaceK {
  T a1, a2, a3, a4, a5, a6;   // E flux
  T q2, q3, q5, b1;           // normal-H flux (q2, q3 shared)
  T c1, c2, c3, c4, c5, c6;   // tangential-H flux
  T g0, k3;                   // g = g0 - k3 / (eps_s mu_s)
};

// Constants of face_flux for a face of normal spacing hn and tangential spacing ht whose frame
// has tangential-H sign sb and tangential-derivative sign st (x-faces: +1, +1; y-faces: -1, -1).
// Differences along the normal carry 1/(2 hn), along the tangent 1/(2 ht).
template <typename T>
inline FaceK<T> make_face_k(const double C[5], double hn, double ht, double c, double sb, double st) {
  const double K1 = C[0] / hn, K2 = C[1] / hn, K3 = C[2] / hn, K4 = C[3] / hn, K5 = C[4] / hn;
  const double sn = 0.5 / hn, stt = 0.5 / ht;
  const double inv2c = 0.5 / c;
  const double q1 = 0.5 * K4, q2 = 0.5 * K4 * c, q3 = 0.5 * K5 * c * c, q4 = 0.5 * K5 * c;
  FaceK<T> k;
  k.a1 = T(-0.5 * K1 * sb); k.a2 = T(-K1 * inv2c); k.a3 = T(sb * inv2c);
  k.a4 = T(-q1 * sb); k.a5 = T(q4 * st * stt); k.a6 = T(-q4 * sb * sn);
  k.q2 = T(q2); k.q3 = T(q3 * sn); k.q5 = T((0.5 * K2 * c * c - q3) * sn); k.b1 = T(q4 * st * stt);
  k.c1 = T(-0.5 * K1 * sb); k.c2 = T(-K1 * inv2c); k.c3 = T(sb * inv2c);
  k.c4 = T(0.5 * K3 * sb * st * stt); k.c5 = T(-sb * q1); k.c6 = T(-sb * q4 * sn);
  k.g0 = T(K2 * c * c * sn); k.k3 = T(K3 * sn);
  return k;
}

// Twice the slope times the cell size, from the values below (vm), at (v0) and above (vp) a
// cell: the raw central difference vp - vm, or with the limiter twice van Leer's harmonic mean
// of the one-sided differences, 4ab/(a + b) where they share a sign and 0 where they do not.
// (FP32 divides with the fast hardware division, about 2 ulp; FP64 divides exactly.)
__device__ __forceinline__ float slope_div(float n, float d) { return __fdividef(n, d); }
__device__ __forceinline__ double slope_div(double n, double d) { return n / d; }

template <bool LIMIT, typename T>
__device__ __forceinline__ T raw_slope(T vm, T v0, T vp) {
  if (!LIMIT) return vp - vm;
  const T a = vp - v0, b = v0 - vm, ab = a * b;
  return ab > T(0) ? slope_div(T(4) * ab, a + b) : T(0);
}

}  // namespace gks
