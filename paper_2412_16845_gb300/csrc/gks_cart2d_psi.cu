// Fused 2-D TM step with divergence cleaning (Sec. 2.1, the PHM system with gamma > 0): the
// state is (Ez, Hx, Hy, psi), psi carrying div B away at speed gamma (phi decouples in TM: E =
// Ez(x, y) is divergence free).  mu = 1; eps per cell.
//
// The same warp-strip march as cart2d_step_kernel (a warp owns 64 columns, 2 per lane, walks up
// its rows with the state in registers, x-neighbours by shuffles).  Every face -- interior, PEC
// wall (mirror-image loads, psi even) and kinetic non-reflecting boundary (a ghost side of zero
// distributions with eps_s of the inner cell) -- goes through face_flux_psi, the closed form of
// the per-velocity flux of Sec. 3.1 for this system in sums and differences of the two sides.
#include <cuda_runtime.h>

#include "gks_flux2.cuh"
#include "gks_internal.h"
#include "gks_tma.cuh"

namespace gks {
namespace {

__device__ __forceinline__ float prcp1(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double prcp1(double x) { return 1.0 / x; }
__device__ __forceinline__ float prcp2(float x) { return __fdividef(2.f, x); }
__device__ __forceinline__ double prcp2(double x) { return 2.0 / x; }

// Constants of the gamma terms of a face (K_i = C_i / h_normal, sn = 1/(2 h_normal),
// stt = 1/(2 h_tangential), sb / st the face frame's signs of H_t and of the tangential
// derivative; see face_flux_psi).
template <typename T>
struct FacePsiK {
  T pe1, pe2;                       // E
  T pa1, pa2, pa3, pa4, pa5, pa6;   // H_n (pa1, pa2, pa4, pa5 shared with psi)
  T h0, h1;                         // sb st stt H = h0 - h1 ie (H_t and psi)
  T pp5;                            // psi
  T pz1, pz2;                       // psi's own kinetic terms (nonzero for tau > 0)
};

template <typename T>
inline FacePsiK<T> make_face_psi(const double C[5], double hn, double ht, double c, double sb,
                                 double st, double g) {
  const double K1 = C[0] / hn, K2 = C[1] / hn, K3 = C[2] / hn, K4 = C[3] / hn, K5 = C[4] / hn;
  const double sn = 0.5 / hn, stt = 0.5 / ht;
  const double G = g * (K2 * c * c - K3 * g * g - K5 * c * c) / (2.0 * c);
  FacePsiK<T> k;
  k.pe1 = T(st * stt * K3 * g / 2.0);
  k.pe2 = T(-st * stt * K3 * g * g / (2.0 * c));
  k.pa1 = T(g * (K1 + K4) / 2.0);
  k.pa2 = T(-K3 * g * g / 2.0 * sn);
  k.pa3 = T(-K3 * g * g / 2.0 * sb * st * stt);
  k.pa4 = T(-K1 * g * g / (2.0 * c));
  k.pa5 = T(-G * sn);
  k.pa6 = T(-K3 * g * g / (2.0 * c) * st * stt);
  k.h0 = T(sb * st * stt * g * c * K5 / 2.0);
  k.h1 = T(sb * st * stt * g * K3 / (2.0 * c));
  k.pp5 = T(-K3 * g / 2.0 * st * stt);
  k.pz1 = T(-K4 * c / 2.0);
  k.pz2 = T(c * c * (K2 - K5) / 2.0 * sn);
  return k;
}

// One side of a face in global components: reconstructed e = Ez, hn, ht, p = psi; raw central
// differences along the normal (den, dhn, dht, dnp), along the tangent (dat of Hn, det of Ez,
// dtp of psi, dtt of Ht); eps.  A kinetic ghost side is all zero.
template <typename T>
struct PSide {
  T e, hn, ht, p, den, dhn, dht, dnp, dat, det, dtp, dtt, eps;
};

// Flux (times dt/h) of a face: the Maxwell part of face_flux (mu = 1) with ie = 1/eps_s given
// (2/(eps_l + eps_r) inside, 1/eps of the inner cell on a non-reflecting face) plus the gamma
// terms, in local quantities (t_x = tangential, n_x = normal true derivatives, S = l + r,
// D = r - l, G = gamma (c^2 (K2 - K5) - K3 gamma^2)/(2c), H = gamma (c^2 K5 - K3 ie)/(2c)):
//   E   += K3 gamma/2 S t_psi - K3 gamma^2/(2c) D t_Hn
//   Hn  += gamma (K1+K4)/2 S psi - K3 gamma^2/2 (S n_Hn + S t_Ht) - K1 gamma^2/(2c) D Hn
//          - G D n_psi - K3 gamma^2/(2c) D t_E
//   Ht  += H D t_psi
//   psi  = gamma (K1+K4)/2 S Hn - K3 gamma^2/2 S n_psi - K1 gamma^2/(2c) D psi - G D n_Hn
//          + H D t_Ht - K3 gamma ie/2 S (eps t_E) - K4 c/2 D psi + c^2 (K2 - K5)/2 S n_psi
// (the last two, present for tau > 0 even at gamma = 0, are the free transport of psi itself).
template <typename T>
__device__ __forceinline__ void face_flux_psi(const PSide<T> &l, const PSide<T> &r,
                                              const FaceK<T> &k, const FacePsiK<T> &q, T ie,
                                              T &fE, T &fHn, T &fHt, T &fP) {
  const T Ue_l = l.eps * l.e, Ue_r = r.eps * r.e;
  const T Uxe_l = l.eps * l.den, Uxe_r = r.eps * r.den;
  const T S_B = l.ht + r.ht, D_e = r.e - l.e;
  const T S_Uxe = Uxe_l + Uxe_r, D_xB = r.dht - l.dht;
  const T D_Ue = Ue_r - Ue_l, D_At = r.dat - l.dat;
  const T S_Uxa = l.dhn + r.dhn, D_Ua = r.hn - l.hn, D_Et = r.det - l.det;
  const T S_Ue = Ue_l + Ue_r, D_B = r.ht - l.ht, S_UxB = l.dht + r.dht;
  const T D_ex = r.den - l.den, S_UAt = l.dat + r.dat, S_e = l.e + r.e;
  const T g = k.g0 - k.k3 * ie;
  T fe = k.a1 * S_B + k.a2 * D_e;
  fe += g * (T(0.5) * S_Uxe + k.a3 * D_xB);
  fe += k.a4 * S_B - k.q2 * D_Ue - k.q3 * S_Uxe + k.a5 * D_At + k.a6 * D_xB;
  T fa = k.q5 * S_Uxa - k.q2 * D_Ua + k.b1 * D_Et;
  T fb = ie * (k.c1 * S_Ue + k.c2 * D_B);
  fb += g * (T(0.5) * S_UxB + k.c3 * D_ex);
  fb += k.c4 * ie * S_UAt + k.c5 * S_e - k.q2 * D_B - k.q3 * S_UxB + k.c6 * D_ex;
  // gamma terms
  const T S_p = l.p + r.p, D_p = r.p - l.p, S_np = l.dnp + r.dnp, D_np = r.dnp - l.dnp;
  const T S_tp = l.dtp + r.dtp, D_tp = r.dtp - l.dtp, S_tt = l.dtt + r.dtt, D_tt = r.dtt - l.dtt;
  const T S_hn = l.hn + r.hn, D_hn_n = r.dhn - l.dhn;
  const T H = q.h0 - q.h1 * ie;
  fe += q.pe1 * S_tp + q.pe2 * D_At;
  fa += q.pa1 * S_p + q.pa2 * S_Uxa + q.pa3 * S_tt + q.pa4 * D_Ua + q.pa5 * D_np + q.pa6 * D_Et;
  fb += H * D_tp;
  const T fp = q.pa1 * S_hn + q.pa2 * S_np + q.pa4 * D_p + q.pa5 * D_hn_n + H * D_tt +
               q.pp5 * ie * (l.eps * l.det + r.eps * r.det) + q.pz1 * D_p + q.pz2 * S_np;
  fE = fe;
  fHn = fa;
  fHt = fb;
  fP = fp;
}

template <typename T>
struct PsiArgs {
  const T *__restrict__ V;
  T *__restrict__ Vout;
  const T *__restrict__ eps;
  const T *__restrict__ src;
  int sx0, sx1, sy0, sy1;
  T src_amp;
  int nx, ny;
  int64_t pitch, cstride;
  int perx, pery;
  int pec[4];
  FaceK<T> fx, fy;
  FacePsiK<T> qx, qy;
  int *flag;
};

__device__ __forceinline__ int psi_axis(int i, int n, int periodic, int pec_lo, int pec_hi,
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

constexpr int PWARPS = 4;
constexpr int PCOLS = 60;
constexpr unsigned PFULL = 0xffffffffu;

template <typename T> struct PPair;
template <> struct PPair<float> { using type = float2; };
template <> struct PPair<double> { using type = double2; };

// Two columns of a row: (Ez, Hx, Hy, psi, eps) and their PEC mirror flags (signs applied when
// the row enters the working window; psi keeps its sign across a PEC wall).
template <typename T>
struct PRow {
  T ez[2], hx[2], hy[2], ps[2], eps[2];
  bool xm[2], ym;
};

template <typename T>
__device__ __forceinline__ void psi_mirror(PRow<T> &v) {
  if (v.ym | v.xm[0] | v.xm[1]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (v.xm[k] != v.ym) v.ez[k] = -v.ez[k];
      if (v.xm[k]) v.hx[k] = -v.hx[k];
      if (v.ym) v.hy[k] = -v.hy[k];
    }
  }
}

template <typename T>
__device__ __forceinline__ PRow<T> psi_load(const PsiArgs<T> &p, int X, int row) {
  using P = typename PPair<T>::type;
  PRow<T> v;
  const int r = psi_axis(row, p.ny, p.pery, p.pec[2], p.pec[3], v.ym);
  v.xm[0] = v.xm[1] = false;
  const int64_t ro = (int64_t)r * p.pitch;
  if (X >= 0 && X + 1 < p.nx) {
    const P a = __ldg(reinterpret_cast<const P *>(p.V + ro + X));
    const P b = __ldg(reinterpret_cast<const P *>(p.V + p.cstride + ro + X));
    const P c = __ldg(reinterpret_cast<const P *>(p.V + 2 * p.cstride + ro + X));
    const P d = __ldg(reinterpret_cast<const P *>(p.V + 3 * p.cstride + ro + X));
    const P e = __ldg(reinterpret_cast<const P *>(p.eps + ro + X));
    v.ez[0] = a.x; v.ez[1] = a.y; v.hx[0] = b.x; v.hx[1] = b.y; v.hy[0] = c.x; v.hy[1] = c.y;
    v.ps[0] = d.x; v.ps[1] = d.y; v.eps[0] = e.x; v.eps[1] = e.y;
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t o = ro + psi_axis(X + k, p.nx, p.perx, p.pec[0], p.pec[1], v.xm[k]);
      v.ez[k] = __ldg(p.V + o);
      v.hx[k] = __ldg(p.V + p.cstride + o);
      v.hy[k] = __ldg(p.V + 2 * p.cstride + o);
      v.ps[k] = __ldg(p.V + 3 * p.cstride + o);
      v.eps[k] = __ldg(p.eps + o);
    }
  }
  return v;
}

// Raw central differences of one column: x and y differences of (Ez, Hx, Hy, psi).
template <typename T>
struct PG {
  T ex, ey, ax, ay, bx, by, px, py;
};

// Differences of the lane's two columns (x-neighbours by shuffle; limited slopes with LIMIT);
// right[] receives column X+2.
template <typename T, bool LIMIT>
__device__ __forceinline__ void psi_diffs(const PRow<T> &c, const PRow<T> &dn, const PRow<T> &up,
                                          PG<T> g[2], T right[4]) {
  const T lE = __shfl_up_sync(PFULL, c.ez[1], 1), rE = __shfl_down_sync(PFULL, c.ez[0], 1);
  const T lA = __shfl_up_sync(PFULL, c.hx[1], 1), rA = __shfl_down_sync(PFULL, c.hx[0], 1);
  const T lB = __shfl_up_sync(PFULL, c.hy[1], 1), rB = __shfl_down_sync(PFULL, c.hy[0], 1);
  const T lP = __shfl_up_sync(PFULL, c.ps[1], 1), rP = __shfl_down_sync(PFULL, c.ps[0], 1);
  g[0].ex = raw_slope<LIMIT>(lE, c.ez[0], c.ez[1]);
  g[1].ex = raw_slope<LIMIT>(c.ez[0], c.ez[1], rE);
  g[0].ax = raw_slope<LIMIT>(lA, c.hx[0], c.hx[1]);
  g[1].ax = raw_slope<LIMIT>(c.hx[0], c.hx[1], rA);
  g[0].bx = raw_slope<LIMIT>(lB, c.hy[0], c.hy[1]);
  g[1].bx = raw_slope<LIMIT>(c.hy[0], c.hy[1], rB);
  g[0].px = raw_slope<LIMIT>(lP, c.ps[0], c.ps[1]);
  g[1].px = raw_slope<LIMIT>(c.ps[0], c.ps[1], rP);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    g[k].ey = raw_slope<LIMIT>(dn.ez[k], c.ez[k], up.ez[k]);
    g[k].ay = raw_slope<LIMIT>(dn.hx[k], c.hx[k], up.hx[k]);
    g[k].by = raw_slope<LIMIT>(dn.hy[k], c.hy[k], up.hy[k]);
    g[k].py = raw_slope<LIMIT>(dn.ps[k], c.ps[k], up.ps[k]);
  }
  right[0] = rE; right[1] = rA; right[2] = rB; right[3] = rP;
}

// x-face side (normal x: hn = Hx, ht = Hy, tangent y), reconstructed by sgn4 * raw difference.
template <typename T>
__device__ __forceinline__ PSide<T> psi_xside(T ez, T hx, T hy, T ps, T eps, const PG<T> &g,
                                              T sgn4) {
  PSide<T> s;
  s.e = ez + sgn4 * g.ex; s.hn = hx + sgn4 * g.ax; s.ht = hy + sgn4 * g.bx; s.p = ps + sgn4 * g.px;
  s.den = g.ex; s.dhn = g.ax; s.dht = g.bx; s.dnp = g.px;
  s.dat = g.ay; s.det = g.ey; s.dtp = g.py; s.dtt = g.by;
  s.eps = eps;
  return s;
}

// y-face side (normal y: hn = Hy, ht = Hx, tangent x).
template <typename T>
__device__ __forceinline__ PSide<T> psi_yside(T ez, T hx, T hy, T ps, T eps, const PG<T> &g,
                                              T sgn4) {
  PSide<T> s;
  s.e = ez + sgn4 * g.ey; s.hn = hy + sgn4 * g.by; s.ht = hx + sgn4 * g.ay; s.p = ps + sgn4 * g.py;
  s.den = g.ey; s.dhn = g.by; s.dht = g.ay; s.dnp = g.py;
  s.dat = g.bx; s.det = g.ex; s.dtp = g.px; s.dtt = g.ax;
  s.eps = eps;
  return s;
}

template <typename T>
__device__ __forceinline__ PSide<T> psi_zero() {
  PSide<T> s;
  s.e = s.hn = s.ht = s.p = s.den = s.dhn = s.dht = s.dnp = T(0);
  s.dat = s.det = s.dtp = s.dtt = s.eps = T(0);
  return s;
}

template <typename T, bool HAS_PEC, bool LIMIT>
__global__ void __launch_bounds__(PWARPS * 32) cart2d_psi_step_kernel(const PsiArgs<T> p,
                                                                      int nstrips, int rows) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * PWARPS + (threadIdx.x >> 5);
  const int strip = wid % nstrips, chunk = wid / nstrips;
  const int y0 = chunk * rows;
  if (y0 >= p.ny) return;                             // whole warp leaves together
  const int y1 = min(y0 + rows, p.ny);
  const int x0 = strip * PCOLS;
  const int X = x0 - 2 + 2 * lane;
  const int xend = min(x0 + PCOLS, p.nx);
  const bool xlo_nr = !p.perx && !p.pec[0], xhi_nr = !p.perx && !p.pec[1];
  const bool ylo_nr = !p.pery && !p.pec[2], yhi_nr = !p.pery && !p.pec[3];
  const T q4 = T(0.25), mq4 = T(-0.25);

  PRow<T> vm2 = psi_load(p, X, y0 - 2), vm1 = psi_load(p, X, y0 - 1), v0 = psi_load(p, X, y0);
  PRow<T> v1 = psi_load(p, X, y0 + 1), v2 = psi_load(p, X, y0 + 2), pf = psi_load(p, X, y0 + 3);
  if (HAS_PEC) {
    psi_mirror(vm2); psi_mirror(vm1); psi_mirror(v0); psi_mirror(v1); psi_mirror(v2);
  }
  PG<T> g0[2], gm1[2];
  T r0[4], rm1[4];
  psi_diffs<T, LIMIT>(vm1, vm2, v0, gm1, rm1);
  psi_diffs<T, LIMIT>(v0, vm1, v1, g0, r0);
  T fbE[2], fbHx[2], fbHy[2], fbP[2];                 // flux along +y below row j
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const PSide<T> up = psi_yside(v0.ez[k], v0.hx[k], v0.hy[k], v0.ps[k], v0.eps[k], g0[k], mq4);
    if (y0 == 0 && ylo_nr)
      face_flux_psi<T>(psi_zero<T>(), up, p.fy, p.qy, prcp1(v0.eps[k]), fbE[k], fbHy[k], fbHx[k], fbP[k]);
    else
      face_flux_psi<T>(psi_yside(vm1.ez[k], vm1.hx[k], vm1.hy[k], vm1.ps[k], vm1.eps[k], gm1[k], q4),
                       up, p.fy, p.qy, prcp2(vm1.eps[k] + v0.eps[k]), fbE[k], fbHy[k], fbHx[k], fbP[k]);
  }
  bool bad = false;
#pragma unroll 1
  for (int j = y0; j < y1; ++j) {
    const PRow<T> pf2 = psi_load(p, X, j + 4);
    PG<T> g1[2];
    T r1[4];
    psi_diffs<T, LIMIT>(v1, v0, v2, g1, r1);
    // x-faces X+1/2 and X+3/2 (column X+2 from the next lane)
    T fxE[2], fxHx[2], fxHy[2], fxP[2];
    {
      const T ne = __shfl_down_sync(PFULL, v0.eps[0], 1);
      PG<T> gn;
      gn.ex = __shfl_down_sync(PFULL, g0[0].ex, 1);
      gn.ax = __shfl_down_sync(PFULL, g0[0].ax, 1);
      gn.bx = __shfl_down_sync(PFULL, g0[0].bx, 1);
      gn.px = __shfl_down_sync(PFULL, g0[0].px, 1);
      gn.ay = __shfl_down_sync(PFULL, g0[0].ay, 1);
      gn.ey = __shfl_down_sync(PFULL, g0[0].ey, 1);
      gn.by = __shfl_down_sync(PFULL, g0[0].by, 1);
      gn.py = __shfl_down_sync(PFULL, g0[0].py, 1);
      const PSide<T> l0 = psi_xside(v0.ez[0], v0.hx[0], v0.hy[0], v0.ps[0], v0.eps[0], g0[0], q4);
      const PSide<T> r1s = psi_xside(v0.ez[1], v0.hx[1], v0.hy[1], v0.ps[1], v0.eps[1], g0[1], mq4);
      const PSide<T> l1 = psi_xside(v0.ez[1], v0.hx[1], v0.hy[1], v0.ps[1], v0.eps[1], g0[1], q4);
      const PSide<T> rn = psi_xside(r0[0], r0[1], r0[2], r0[3], ne, gn, mq4);
      // first face: high boundary if X is the last column
      if (xhi_nr && X == p.nx - 1)
        face_flux_psi<T>(l0, psi_zero<T>(), p.fx, p.qx, prcp1(v0.eps[0]), fxE[0], fxHx[0], fxHy[0], fxP[0]);
      else
        face_flux_psi<T>(l0, r1s, p.fx, p.qx, prcp2(v0.eps[0] + v0.eps[1]), fxE[0], fxHx[0], fxHy[0], fxP[0]);
      // second face: high boundary if X+1 is the last column, low boundary if X+1 = -1
      if (xhi_nr && X + 1 == p.nx - 1)
        face_flux_psi<T>(l1, psi_zero<T>(), p.fx, p.qx, prcp1(v0.eps[1]), fxE[1], fxHx[1], fxHy[1], fxP[1]);
      else if (xlo_nr && X == -2)
        face_flux_psi<T>(psi_zero<T>(), rn, p.fx, p.qx, prcp1(ne), fxE[1], fxHx[1], fxHy[1], fxP[1]);
      else
        face_flux_psi<T>(l1, rn, p.fx, p.qx, prcp2(v0.eps[1] + ne), fxE[1], fxHx[1], fxHy[1], fxP[1]);
    }
    // y-faces j+1/2
    T ftE[2], ftHx[2], ftHy[2], ftP[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const PSide<T> lo = psi_yside(v0.ez[k], v0.hx[k], v0.hy[k], v0.ps[k], v0.eps[k], g0[k], q4);
      if (j + 1 == p.ny && yhi_nr)
        face_flux_psi<T>(lo, psi_zero<T>(), p.fy, p.qy, prcp1(v0.eps[k]), ftE[k], ftHy[k], ftHx[k], ftP[k]);
      else
        face_flux_psi<T>(lo, psi_yside(v1.ez[k], v1.hx[k], v1.hy[k], v1.ps[k], v1.eps[k], g1[k], mq4),
                         p.fy, p.qy, prcp2(v0.eps[k] + v1.eps[k]), ftE[k], ftHy[k], ftHx[k], ftP[k]);
    }
    // update row j
    {
      const T lE = __shfl_up_sync(PFULL, fxE[1], 1), lHx = __shfl_up_sync(PFULL, fxHx[1], 1);
      const T lHy = __shfl_up_sync(PFULL, fxHy[1], 1), lP = __shfl_up_sync(PFULL, fxP[1], 1);
      T dE[2], dHx[2], dHy[2], dP[2];
      dE[0] = (lE - fxE[0]) + (fbE[0] - ftE[0]);
      dHx[0] = (lHx - fxHx[0]) + (fbHx[0] - ftHx[0]);
      dHy[0] = (lHy - fxHy[0]) + (fbHy[0] - ftHy[0]);
      dP[0] = (lP - fxP[0]) + (fbP[0] - ftP[0]);
      dE[1] = (fxE[0] - fxE[1]) + (fbE[1] - ftE[1]);
      dHx[1] = (fxHx[0] - fxHx[1]) + (fbHx[1] - ftHx[1]);
      dHy[1] = (fxHy[0] - fxHy[1]) + (fbHy[1] - ftHy[1]);
      dP[1] = (fxP[0] - fxP[1]) + (fbP[1] - ftP[1]);
      const int64_t ro = (int64_t)j * p.pitch;
      if (p.src && j >= p.sy0 && j < p.sy1) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (X + k >= p.sx0 && X + k < p.sx1) dE[k] -= p.src_amp * p.src[ro + X + k];
      }
      T out[4][2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        out[0][k] = v0.ez[k] + dE[k] * prcp1(v0.eps[k]);
        out[1][k] = v0.hx[k] + dHx[k];
        out[2][k] = v0.hy[k] + dHy[k];
        out[3][k] = v0.ps[k] + dP[k];
      }
      const bool ok0 = X >= x0 && X < xend, ok1 = X + 1 >= x0 && X + 1 < xend;
      using P = typename PPair<T>::type;
      if (ok0 && ok1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          P v;
          v.x = out[c][0]; v.y = out[c][1];
          *reinterpret_cast<P *>(p.Vout + c * p.cstride + ro + X) = v;
          bad |= !(isfinite(out[c][0]) && isfinite(out[c][1]));
        }
      } else {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (k == 0 ? ok0 : ok1)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              p.Vout[c * p.cstride + ro + X + k] = out[c][k];
              bad |= !isfinite(out[c][k]);
            }
      }
    }
    v0 = v1; v1 = v2; v2 = pf; pf = pf2;
    if (HAS_PEC) psi_mirror(v2);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      g0[k] = g1[k];
      fbE[k] = ftE[k]; fbHx[k] = ftHx[k]; fbHy[k] = ftHy[k]; fbP[k] = ftP[k];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) r0[c] = r1[c];
  }
  if (__any_sync(PFULL, bad) && lane == 0) atomicOr(p.flag, 1);
}

// ------------------------------------------------------------------ paired FP32 path
// As cart2d_step_kernel_p for the Maxwell step: a lane's two x-faces, two y-faces and two cell
// updates go through the paired FP32 instructions (component x: first face or column, y: the
// second).  Boundary faces are evaluated by the scalar face_flux_psi and replace their
// component afterwards.
using q2 = float2;
__device__ __forceinline__ q2 qk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ q2 qadd(q2 a, q2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ q2 qsub(q2 a, q2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ q2 qmul(q2 a, q2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ q2 qfma(q2 a, q2 b, q2 c) { return __ffma2_rn(a, b, c); }

// FaceK and FacePsiK constants as pairs (a14 = a1 + a4; n* negated).
struct PsiKP {
  q2 a14, a2, a3, a5, a6, nq2, nq3, q5, b1, c1, c2, c3, c4, c5, c6, g0, nk3, half;
  q2 pe1, pe2, pa1, pa2, pa3, pa4, pa5, pa6, h0, nh1, pp5, pz1, pz2;
};

inline PsiKP make_psi_kp(const FaceK<float> &k, const FacePsiK<float> &q) {
  auto b = [](float v) { return make_float2(v, v); };
  PsiKP r;
  r.a14 = b(k.a1 + k.a4); r.a2 = b(k.a2); r.a3 = b(k.a3); r.a5 = b(k.a5); r.a6 = b(k.a6);
  r.nq2 = b(-k.q2); r.nq3 = b(-k.q3); r.q5 = b(k.q5); r.b1 = b(k.b1);
  r.c1 = b(k.c1); r.c2 = b(k.c2); r.c3 = b(k.c3); r.c4 = b(k.c4); r.c5 = b(k.c5); r.c6 = b(k.c6);
  r.g0 = b(k.g0); r.nk3 = b(-k.k3); r.half = b(0.5f);
  r.pe1 = b(q.pe1); r.pe2 = b(q.pe2); r.pa1 = b(q.pa1); r.pa2 = b(q.pa2); r.pa3 = b(q.pa3);
  r.pa4 = b(q.pa4); r.pa5 = b(q.pa5); r.pa6 = b(q.pa6); r.h0 = b(q.h0); r.nh1 = b(-q.h1);
  r.pp5 = b(q.pp5); r.pz1 = b(q.pz1); r.pz2 = b(q.pz2);
  return r;
}

// Two face sides (see PSide).
struct PSideP {
  q2 e, hn, ht, p, den, dhn, dht, dnp, dat, det, dtp, dtt, eps;
};

// face_flux_psi<float> of two interior faces at once (ie = 2/(eps_l + eps_r) per face).
__device__ __forceinline__ void face_flux_psi_p(const PSideP &l, const PSideP &r, const PsiKP &k,
                                                q2 &fE, q2 &fHn, q2 &fHt, q2 &fP) {
  const q2 Ue_l = qmul(l.eps, l.e), Ue_r = qmul(r.eps, r.e);
  const q2 Uxe_l = qmul(l.eps, l.den), Uxe_r = qmul(r.eps, r.den);
  const q2 S_B = qadd(l.ht, r.ht), D_e = qsub(r.e, l.e);
  const q2 S_Uxe = qadd(Uxe_l, Uxe_r), D_xB = qsub(r.dht, l.dht);
  const q2 D_Ue = qsub(Ue_r, Ue_l), D_At = qsub(r.dat, l.dat);
  const q2 S_Uxa = qadd(l.dhn, r.dhn), D_Ua = qsub(r.hn, l.hn), D_Et = qsub(r.det, l.det);
  const q2 S_Ue = qadd(Ue_l, Ue_r), D_B = qsub(r.ht, l.ht), S_UxB = qadd(l.dht, r.dht);
  const q2 D_ex = qsub(r.den, l.den), S_UAt = qadd(l.dat, r.dat), S_e = qadd(l.e, r.e);
  const q2 se = qadd(l.eps, r.eps);
  const q2 ie = qk(prcp2(se.x), prcp2(se.y));
  const q2 g = qfma(k.nk3, ie, k.g0);
  // Maxwell part (mu = 1)
  q2 fe = qmul(k.a14, S_B);
  fe = qfma(k.a2, D_e, fe);
  fe = qfma(g, qfma(k.a3, D_xB, qmul(k.half, S_Uxe)), fe);
  fe = qfma(k.nq2, D_Ue, fe);
  fe = qfma(k.nq3, S_Uxe, fe);
  fe = qfma(k.a5, D_At, fe);
  fe = qfma(k.a6, D_xB, fe);
  q2 fa = qmul(k.q5, S_Uxa);
  fa = qfma(k.nq2, D_Ua, fa);
  fa = qfma(k.b1, D_Et, fa);
  q2 u = qmul(k.c1, S_Ue);
  u = qfma(k.c2, D_B, u);
  u = qfma(k.c4, S_UAt, u);
  q2 fb = qmul(ie, u);
  fb = qfma(g, qfma(k.c3, D_ex, qmul(k.half, S_UxB)), fb);
  fb = qfma(k.c5, S_e, fb);
  fb = qfma(k.nq2, D_B, fb);
  fb = qfma(k.nq3, S_UxB, fb);
  fb = qfma(k.c6, D_ex, fb);
  // gamma terms and psi's own transport
  const q2 S_p = qadd(l.p, r.p), D_p = qsub(r.p, l.p);
  const q2 S_np = qadd(l.dnp, r.dnp), D_np = qsub(r.dnp, l.dnp);
  const q2 S_tp = qadd(l.dtp, r.dtp), D_tp = qsub(r.dtp, l.dtp);
  const q2 S_tt = qadd(l.dtt, r.dtt), D_tt = qsub(r.dtt, l.dtt);
  const q2 S_hn = qadd(l.hn, r.hn), D_hn_n = qsub(r.dhn, l.dhn);
  const q2 H = qfma(k.nh1, ie, k.h0);
  fe = qfma(k.pe1, S_tp, fe);
  fe = qfma(k.pe2, D_At, fe);
  fa = qfma(k.pa1, S_p, fa);
  fa = qfma(k.pa2, S_Uxa, fa);
  fa = qfma(k.pa3, S_tt, fa);
  fa = qfma(k.pa4, D_Ua, fa);
  fa = qfma(k.pa5, D_np, fa);
  fa = qfma(k.pa6, D_Et, fa);
  fb = qfma(H, D_tp, fb);
  const q2 Edet = qfma(l.eps, l.det, qmul(r.eps, r.det));
  q2 fp = qmul(k.pa1, S_hn);
  fp = qfma(k.pa2, S_np, fp);
  fp = qfma(k.pa4, D_p, fp);
  fp = qfma(k.pa5, D_hn_n, fp);
  fp = qfma(H, D_tt, fp);
  fp = qfma(qmul(k.pp5, ie), Edet, fp);
  fp = qfma(k.pz1, D_p, fp);
  fp = qfma(k.pz2, S_np, fp);
  fE = fe;
  fHn = fa;
  fHt = fb;
  fP = fp;
}

struct PRowP {
  q2 ez, hx, hy, ps, eps;
  bool xm[2], ym;
};
struct PGP {
  q2 ex, ey, ax, ay, bx, by, px, py;
};

__device__ __forceinline__ void psi_mirror_p(PRowP &v) {
  if (v.ym | v.xm[0] | v.xm[1]) {
    if (v.xm[0] != v.ym) v.ez.x = -v.ez.x;
    if (v.xm[1] != v.ym) v.ez.y = -v.ez.y;
    if (v.xm[0]) v.hx.x = -v.hx.x;
    if (v.xm[1]) v.hx.y = -v.hx.y;
    if (v.ym) { v.hy.x = -v.hy.x; v.hy.y = -v.hy.y; }
  }
}

__device__ __forceinline__ PRowP psi_load_p(const PsiArgs<float> &p, int X, int row) {
  PRowP v;
  const int r = psi_axis(row, p.ny, p.pery, p.pec[2], p.pec[3], v.ym);
  v.xm[0] = v.xm[1] = false;
  const int64_t ro = (int64_t)r * p.pitch;
  if (X >= 0 && X + 1 < p.nx) {
    v.ez = __ldg(reinterpret_cast<const q2 *>(p.V + ro + X));
    v.hx = __ldg(reinterpret_cast<const q2 *>(p.V + p.cstride + ro + X));
    v.hy = __ldg(reinterpret_cast<const q2 *>(p.V + 2 * p.cstride + ro + X));
    v.ps = __ldg(reinterpret_cast<const q2 *>(p.V + 3 * p.cstride + ro + X));
    v.eps = __ldg(reinterpret_cast<const q2 *>(p.eps + ro + X));
  } else {
    int64_t o[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) o[k] = ro + psi_axis(X + k, p.nx, p.perx, p.pec[0], p.pec[1], v.xm[k]);
    v.ez = qk(__ldg(p.V + o[0]), __ldg(p.V + o[1]));
    v.hx = qk(__ldg(p.V + p.cstride + o[0]), __ldg(p.V + p.cstride + o[1]));
    v.hy = qk(__ldg(p.V + 2 * p.cstride + o[0]), __ldg(p.V + 2 * p.cstride + o[1]));
    v.ps = qk(__ldg(p.V + 3 * p.cstride + o[0]), __ldg(p.V + 3 * p.cstride + o[1]));
    v.eps = qk(__ldg(p.eps + o[0]), __ldg(p.eps + o[1]));
  }
  return v;
}

// Scalar views of one column (for the boundary faces).
__device__ __forceinline__ PG<float> pg_of(const PGP &g, int k) {
  PG<float> r;
  r.ex = k ? g.ex.y : g.ex.x; r.ey = k ? g.ey.y : g.ey.x; r.ax = k ? g.ax.y : g.ax.x;
  r.ay = k ? g.ay.y : g.ay.x; r.bx = k ? g.bx.y : g.bx.x; r.by = k ? g.by.y : g.by.x;
  r.px = k ? g.px.y : g.px.x; r.py = k ? g.py.y : g.py.x;
  return r;
}
#define GKS_COL(v, f, k) ((k) ? (v).f.y : (v).f.x)

template <bool LIMIT>
__device__ __forceinline__ void psi_diffs_p(const PRowP &c, const PRowP &dn, const PRowP &up,
                                            PGP &g, float right[4]) {
  const float lE = __shfl_up_sync(PFULL, c.ez.y, 1), rE = __shfl_down_sync(PFULL, c.ez.x, 1);
  const float lA = __shfl_up_sync(PFULL, c.hx.y, 1), rA = __shfl_down_sync(PFULL, c.hx.x, 1);
  const float lB = __shfl_up_sync(PFULL, c.hy.y, 1), rB = __shfl_down_sync(PFULL, c.hy.x, 1);
  const float lP = __shfl_up_sync(PFULL, c.ps.y, 1), rP = __shfl_down_sync(PFULL, c.ps.x, 1);
  if (LIMIT) {
    g.ex = qk(raw_slope<true>(lE, c.ez.x, c.ez.y), raw_slope<true>(c.ez.x, c.ez.y, rE));
    g.ax = qk(raw_slope<true>(lA, c.hx.x, c.hx.y), raw_slope<true>(c.hx.x, c.hx.y, rA));
    g.bx = qk(raw_slope<true>(lB, c.hy.x, c.hy.y), raw_slope<true>(c.hy.x, c.hy.y, rB));
    g.px = qk(raw_slope<true>(lP, c.ps.x, c.ps.y), raw_slope<true>(c.ps.x, c.ps.y, rP));
    g.ey = qk(raw_slope<true>(dn.ez.x, c.ez.x, up.ez.x), raw_slope<true>(dn.ez.y, c.ez.y, up.ez.y));
    g.ay = qk(raw_slope<true>(dn.hx.x, c.hx.x, up.hx.x), raw_slope<true>(dn.hx.y, c.hx.y, up.hx.y));
    g.by = qk(raw_slope<true>(dn.hy.x, c.hy.x, up.hy.x), raw_slope<true>(dn.hy.y, c.hy.y, up.hy.y));
    g.py = qk(raw_slope<true>(dn.ps.x, c.ps.x, up.ps.x), raw_slope<true>(dn.ps.y, c.ps.y, up.ps.y));
  } else {
    g.ex = qsub(qk(c.ez.y, rE), qk(lE, c.ez.x));
    g.ax = qsub(qk(c.hx.y, rA), qk(lA, c.hx.x));
    g.bx = qsub(qk(c.hy.y, rB), qk(lB, c.hy.x));
    g.px = qsub(qk(c.ps.y, rP), qk(lP, c.ps.x));
    g.ey = qsub(up.ez, dn.ez);
    g.ay = qsub(up.hx, dn.hx);
    g.by = qsub(up.hy, dn.hy);
    g.py = qsub(up.ps, dn.ps);
  }
  right[0] = rE; right[1] = rA; right[2] = rB; right[3] = rP;
}

// y-face sides of the two columns (normal y: hn = Hy, ht = Hx, tangent x).
__device__ __forceinline__ PSideP psi_yside_p(const PRowP &v, const PGP &g, q2 sgn) {
  PSideP s;
  s.e = qfma(sgn, g.ey, v.ez); s.hn = qfma(sgn, g.by, v.hy); s.ht = qfma(sgn, g.ay, v.hx);
  s.p = qfma(sgn, g.py, v.ps);
  s.den = g.ey; s.dhn = g.by; s.dht = g.ay; s.dnp = g.py;
  s.dat = g.bx; s.det = g.ex; s.dtp = g.px; s.dtt = g.ax;
  s.eps = v.eps;
  return s;
}

struct PsiPackArgs {
  PsiArgs<float> b;
  PsiKP kx, ky;
};

// Three CTAs per SM (registers capped at 170, a few spills): uncapped the kernel takes 188
// registers and runs two CTAs per SM, 18% slower.
template <bool HAS_PEC, bool LIMIT>
__global__ void __launch_bounds__(PWARPS * 32, 3) cart2d_psi_step_kernel_p(const PsiPackArgs P,
                                                                        int nstrips, int rows) {
  const PsiArgs<float> &p = P.b;
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * PWARPS + (threadIdx.x >> 5);
  const int strip = wid % nstrips, chunk = wid / nstrips;
  const int y0 = chunk * rows;
  if (y0 >= p.ny) return;                             // whole warp leaves together
  const int y1 = min(y0 + rows, p.ny);
  const int x0 = strip * PCOLS;
  const int X = x0 - 2 + 2 * lane;
  const int xend = min(x0 + PCOLS, p.nx);
  const bool xlo_nr = !p.perx && !p.pec[0], xhi_nr = !p.perx && !p.pec[1];
  const bool ylo_nr = !p.pery && !p.pec[2], yhi_nr = !p.pery && !p.pec[3];
  const float q4 = 0.25f, mq4 = -0.25f;
  const q2 Q4 = qk(q4, q4), MQ4 = qk(mq4, mq4);

  PRowP vm2 = psi_load_p(p, X, y0 - 2), vm1 = psi_load_p(p, X, y0 - 1), v0 = psi_load_p(p, X, y0);
  PRowP v1 = psi_load_p(p, X, y0 + 1), v2 = psi_load_p(p, X, y0 + 2), pf = psi_load_p(p, X, y0 + 3);
  if (HAS_PEC) {
    psi_mirror_p(vm2); psi_mirror_p(vm1); psi_mirror_p(v0); psi_mirror_p(v1); psi_mirror_p(v2);
  }
  PGP g0, gm1;
  float r0[4], rm1[4];
  psi_diffs_p<LIMIT>(vm1, vm2, v0, gm1, rm1);
  psi_diffs_p<LIMIT>(v0, vm1, v1, g0, r0);
  q2 fbE, fbHx, fbHy, fbP;                            // flux along +y below row j
  face_flux_psi_p(psi_yside_p(vm1, gm1, Q4), psi_yside_p(v0, g0, MQ4), P.ky, fbE, fbHy, fbHx, fbP);
  if (y0 == 0 && ylo_nr) {
    float e[2], hx[2], hy[2], ps[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const PSide<float> up = psi_yside<float>(GKS_COL(v0, ez, k), GKS_COL(v0, hx, k),
                                               GKS_COL(v0, hy, k), GKS_COL(v0, ps, k),
                                               GKS_COL(v0, eps, k), pg_of(g0, k), mq4);
      face_flux_psi<float>(psi_zero<float>(), up, p.fy, p.qy, prcp1(GKS_COL(v0, eps, k)), e[k],
                           hy[k], hx[k], ps[k]);
    }
    fbE = qk(e[0], e[1]); fbHx = qk(hx[0], hx[1]); fbHy = qk(hy[0], hy[1]); fbP = qk(ps[0], ps[1]);
  }
  bool bad = false;
#pragma unroll 1
  for (int j = y0; j < y1; ++j) {
    const PRowP pf2 = psi_load_p(p, X, j + 4);
    PGP g1;
    float r1[4];
    psi_diffs_p<LIMIT>(v1, v0, v2, g1, r1);
    // x-faces X+1/2 (component x) and X+3/2 (component y; column X+2 from the next lane)
    q2 fxE, fxHx, fxHy, fxP;
    {
      const float ne = __shfl_down_sync(PFULL, v0.eps.x, 1);
      PG<float> gn;
      gn.ex = __shfl_down_sync(PFULL, g0.ex.x, 1);
      gn.ax = __shfl_down_sync(PFULL, g0.ax.x, 1);
      gn.bx = __shfl_down_sync(PFULL, g0.bx.x, 1);
      gn.px = __shfl_down_sync(PFULL, g0.px.x, 1);
      gn.ay = __shfl_down_sync(PFULL, g0.ay.x, 1);
      gn.ey = __shfl_down_sync(PFULL, g0.ey.x, 1);
      gn.by = __shfl_down_sync(PFULL, g0.by.x, 1);
      gn.py = __shfl_down_sync(PFULL, g0.py.x, 1);
      PSideP l, r;
      l.e = qfma(Q4, g0.ex, v0.ez); l.hn = qfma(Q4, g0.ax, v0.hx); l.ht = qfma(Q4, g0.bx, v0.hy);
      l.p = qfma(Q4, g0.px, v0.ps);
      l.den = g0.ex; l.dhn = g0.ax; l.dht = g0.bx; l.dnp = g0.px;
      l.dat = g0.ay; l.det = g0.ey; l.dtp = g0.py; l.dtt = g0.by;
      l.eps = v0.eps;
      r.den = qk(g0.ex.y, gn.ex); r.dhn = qk(g0.ax.y, gn.ax); r.dht = qk(g0.bx.y, gn.bx);
      r.dnp = qk(g0.px.y, gn.px); r.dat = qk(g0.ay.y, gn.ay); r.det = qk(g0.ey.y, gn.ey);
      r.dtp = qk(g0.py.y, gn.py); r.dtt = qk(g0.by.y, gn.by);
      r.e = qfma(MQ4, r.den, qk(v0.ez.y, r0[0]));
      r.hn = qfma(MQ4, r.dhn, qk(v0.hx.y, r0[1]));
      r.ht = qfma(MQ4, r.dht, qk(v0.hy.y, r0[2]));
      r.p = qfma(MQ4, r.dnp, qk(v0.ps.y, r0[3]));
      r.eps = qk(v0.eps.y, ne);
      face_flux_psi_p(l, r, P.kx, fxE, fxHx, fxHy, fxP);
      // boundary faces replace their component (rare, divergent)
      if (xhi_nr && X == p.nx - 1) {
        const PSide<float> l0 = psi_xside<float>(v0.ez.x, v0.hx.x, v0.hy.x, v0.ps.x, v0.eps.x,
                                                 pg_of(g0, 0), q4);
        face_flux_psi<float>(l0, psi_zero<float>(), p.fx, p.qx, prcp1(v0.eps.x), fxE.x, fxHx.x,
                             fxHy.x, fxP.x);
      }
      if (xhi_nr && X + 1 == p.nx - 1) {
        const PSide<float> l1 = psi_xside<float>(v0.ez.y, v0.hx.y, v0.hy.y, v0.ps.y, v0.eps.y,
                                                 pg_of(g0, 1), q4);
        face_flux_psi<float>(l1, psi_zero<float>(), p.fx, p.qx, prcp1(v0.eps.y), fxE.y, fxHx.y,
                             fxHy.y, fxP.y);
      } else if (xlo_nr && X == -2) {
        const PSide<float> rn = psi_xside<float>(r0[0], r0[1], r0[2], r0[3], ne, gn, mq4);
        face_flux_psi<float>(psi_zero<float>(), rn, p.fx, p.qx, prcp1(ne), fxE.y, fxHx.y,
                             fxHy.y, fxP.y);
      }
    }
    // y-faces j+1/2
    q2 ftE, ftHx, ftHy, ftP;
    face_flux_psi_p(psi_yside_p(v0, g0, Q4), psi_yside_p(v1, g1, MQ4), P.ky, ftE, ftHy, ftHx, ftP);
    if (j + 1 == p.ny && yhi_nr) {
      float e[2], hx[2], hy[2], ps[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const PSide<float> lo = psi_yside<float>(GKS_COL(v0, ez, k), GKS_COL(v0, hx, k),
                                                 GKS_COL(v0, hy, k), GKS_COL(v0, ps, k),
                                                 GKS_COL(v0, eps, k), pg_of(g0, k), q4);
        face_flux_psi<float>(lo, psi_zero<float>(), p.fy, p.qy, prcp1(GKS_COL(v0, eps, k)), e[k],
                             hy[k], hx[k], ps[k]);
      }
      ftE = qk(e[0], e[1]); ftHx = qk(hx[0], hx[1]); ftHy = qk(hy[0], hy[1]);
      ftP = qk(ps[0], ps[1]);
    }
    // update row j
    {
      const float lE = __shfl_up_sync(PFULL, fxE.y, 1), lHx = __shfl_up_sync(PFULL, fxHx.y, 1);
      const float lHy = __shfl_up_sync(PFULL, fxHy.y, 1), lP = __shfl_up_sync(PFULL, fxP.y, 1);
      q2 dE = qadd(qsub(qk(lE, fxE.x), fxE), qsub(fbE, ftE));
      const q2 dHx = qadd(qsub(qk(lHx, fxHx.x), fxHx), qsub(fbHx, ftHx));
      const q2 dHy = qadd(qsub(qk(lHy, fxHy.x), fxHy), qsub(fbHy, ftHy));
      const q2 dP = qadd(qsub(qk(lP, fxP.x), fxP), qsub(fbP, ftP));
      const int64_t ro = (int64_t)j * p.pitch;
      if (p.src && j >= p.sy0 && j < p.sy1) {
        if (X >= p.sx0 && X < p.sx1) dE.x -= p.src_amp * p.src[ro + X];
        if (X + 1 >= p.sx0 && X + 1 < p.sx1) dE.y -= p.src_amp * p.src[ro + X + 1];
      }
      const q2 out[4] = {qfma(dE, qk(prcp1(v0.eps.x), prcp1(v0.eps.y)), v0.ez), qadd(v0.hx, dHx),
                         qadd(v0.hy, dHy), qadd(v0.ps, dP)};
      const bool ok0 = X >= x0 && X < xend, ok1 = X + 1 >= x0 && X + 1 < xend;
      if (ok0 && ok1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) *reinterpret_cast<q2 *>(p.Vout + c * p.cstride + ro + X) = out[c];
        const q2 sum = qadd(qadd(out[0], out[1]), qadd(out[2], out[3]));
        bad |= !(isfinite(sum.x) && isfinite(sum.y));
      } else {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (k == 0 ? ok0 : ok1)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float v = k ? out[c].y : out[c].x;
              p.Vout[c * p.cstride + ro + X + k] = v;
              bad |= !isfinite(v);
            }
      }
    }
    v0 = v1; v1 = v2; v2 = pf; pf = pf2;
    if (HAS_PEC) psi_mirror_p(v2);
    g0 = g1;
    fbE = ftE; fbHx = ftHx; fbHy = ftHy; fbP = ftP;
#pragma unroll
    for (int c = 0; c < 4; ++c) r0[c] = r1[c];
  }
  if (__any_sync(PFULL, bad) && lane == 0) atomicOr(p.flag, 1);
}
// ------------------------------------------------------------------ staged FP32 path
// The staged march of the 2-D TM step (gks_cart2d.cu: rows staged per warp by TMA, a lane's two
// cells 32 columns apart, 63 columns per warp, left x-faces per lane, every neighbour read from
// the staged rows, coalesced stores) with psi as a fourth field: FP32, no limiter, no PEC wall,
// x not periodic.  (With the limiter the register-window kernel below is faster: the left
// neighbours' limited slopes would be recomputed here rather than shuffled.)
constexpr int PW2 = 63;                 // columns updated per warp
constexpr int PTW2 = 72;                // staged columns (x0-3 rounded down to 4, +72)
constexpr int PNSLOT2 = 8;              // staged rows per warp
static_assert((PNSLOT2 & (PNSLOT2 - 1)) == 0, "the ring index masks with PNSLOT2 - 1");
struct alignas(128) PRowBox2 { float a[4][PTW2]; };   // Ez, Hx, Hy, psi
struct alignas(128) PEpsBox2 { float e[PTW2]; };
struct PStagedRow2 { PRowBox2 v; PEpsBox2 e; };
struct PWarpStage2 {
  PStagedRow2 row[PNSLOT2];
  unsigned long long bar[PNSLOT2];
};
constexpr unsigned kPRowBytes2 = 5 * PTW2 * 4;         // both boxes of one staged row

struct PTaps2 {
  int a[4], b[4];       // [k]: staged column of A + k - 2 / B + k - 2 (clamped to the grid)
};

template <bool EPS>
__device__ __forceinline__ PRowP pstaged_pair(const PStagedRow2 &R, const PTaps2 &q, int k) {
  PRowP v;
  v.ez = qk(R.v.a[0][q.a[k]], R.v.a[0][q.b[k]]);
  v.hx = qk(R.v.a[1][q.a[k]], R.v.a[1][q.b[k]]);
  v.hy = qk(R.v.a[2][q.a[k]], R.v.a[2][q.b[k]]);
  v.ps = qk(R.v.a[3][q.a[k]], R.v.a[3][q.b[k]]);
  v.eps = EPS ? qk(R.e.e[q.a[k]], R.e.e[q.b[k]]) : qk(0.f, 0.f);
  v.xm[0] = v.xm[1] = v.ym = false;
  return v;
}

// Raw central differences of the pair at tap k of row `mid` (rows `dn` and `up` below and above).
__device__ __forceinline__ PGP pstaged_diffs(const PStagedRow2 &dn, const PStagedRow2 &mid,
                                             const PStagedRow2 &up, const PTaps2 &q, int k) {
  PGP g;
  const PRowP l = pstaged_pair<false>(mid, q, k - 1), r = pstaged_pair<false>(mid, q, k + 1);
  const PRowP d = pstaged_pair<false>(dn, q, k), u = pstaged_pair<false>(up, q, k);
  g.ex = qsub(r.ez, l.ez); g.ax = qsub(r.hx, l.hx); g.bx = qsub(r.hy, l.hy);
  g.px = qsub(r.ps, l.ps);
  g.ey = qsub(u.ez, d.ez); g.ay = qsub(u.hx, d.hx); g.by = qsub(u.hy, d.hy);
  g.py = qsub(u.ps, d.ps);
  return g;
}

// x-face side of the pair (normal x: hn = Hx, ht = Hy).
__device__ __forceinline__ PSideP psi_xside_p(const PRowP &v, const PGP &g, q2 sgn) {
  PSideP s;
  s.e = qfma(sgn, g.ex, v.ez); s.hn = qfma(sgn, g.ax, v.hx); s.ht = qfma(sgn, g.bx, v.hy);
  s.p = qfma(sgn, g.px, v.ps);
  s.den = g.ex; s.dhn = g.ax; s.dht = g.bx; s.dnp = g.px;
  s.dat = g.ay; s.det = g.ey; s.dtp = g.py; s.dtt = g.by;
  s.eps = v.eps;
  return s;
}

// Two CTAs per SM: the psi component's flux keeps more values live than the TM step's (at 3
// CTAs per SM, 168 registers, the kernel spills 356 B per thread and runs 28% slower than at 2).
__global__ void __launch_bounds__(PWARPS * 32, 2)
    cart2d_psi_step_kernel_s(const __grid_constant__ CUtensorMap tmV,
                             const __grid_constant__ CUtensorMap tmE, const PsiPackArgs P,
                             int nstrips, int rows) {
  extern __shared__ __align__(128) unsigned char smem_ps[];
  const PsiArgs<float> &p = P.b;
  const int lane = threadIdx.x & 31;
  PWarpStage2 &w = reinterpret_cast<PWarpStage2 *>(smem_ps)[threadIdx.x >> 5];
  const int wid = blockIdx.x * PWARPS + (threadIdx.x >> 5);
  const int strip = wid % nstrips, chunk = wid / nstrips;
  const int y0 = chunk * rows;
  if (y0 >= p.ny) return;                             // whole warp leaves together
  const int y1 = min(y0 + rows, p.ny);
  const int x0 = strip * PW2;
  const int xs = (x0 - 3) & ~3;                       // first staged column (16-byte aligned)
  const int A = x0 + lane, B = x0 + 32 + lane;
  const bool ylo_nr = !p.pery, yhi_nr = !p.pery;
  const float q4 = 0.25f, mq4 = -0.25f;
  const q2 Q4 = qk(q4, q4), MQ4 = qk(mq4, mq4), Z2 = qk(0.f, 0.f);
  PTaps2 q;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    q.a[k] = min(max(A + k - 2, 0), p.nx - 1) - xs;
    q.b[k] = min(max(B + k - 2, 0), p.nx - 1) - xs;
  }
  // boundary x faces (scalar flux): the left face of column 0 is its low-x face, the left face
  // of column nx is the high-x face of column nx - 1
  const bool loA = A == 0, hiA = A == p.nx, hiB = B == p.nx;
  const bool xedge = __any_sync(PFULL, loA || hiA || hiB);
  const int xend = min(x0 + PW2, p.nx);
  const bool stA = A < xend, stB = lane < 31 && B < xend;

  const int first = y0 - 2, last = y1 + 1;            // staged rows
  auto slot = [first](int r) { return (r - first) & (PNSLOT2 - 1); };
  auto parity = [first](int r) { return (unsigned)(((r - first) / PNSLOT2) & 1); };
  auto grid_row = [&p](int r) {
    return p.pery ? (r < 0 ? r + p.ny : (r >= p.ny ? r - p.ny : r)) : min(max(r, 0), p.ny - 1);
  };
  int issued = first - 1;                             // lane 0: the last row whose copy is issued
  auto issue = [&](int r) {                           // lane 0 only
    const int s_ = slot(r), gr = grid_row(r);
    fence_proxy_async();
    mbar_expect_tx(&w.bar[s_], kPRowBytes2);
    tma_load_3d(&w.row[s_].v.a[0][0], &tmV, xs, gr, 0, &w.bar[s_]);
    tma_load_2d(&w.row[s_].e.e[0], &tmE, xs, gr, &w.bar[s_]);
    issued = r;
  };
  auto wait_row = [&](int r) {                        // the whole warp; false if it ran out
    return __all_sync(PFULL, mbar_wait(&w.bar[slot(r)], parity(r)));
  };
  if (lane == 0) {
    for (int i = 0; i < PNSLOT2; ++i) mbar_init(&w.bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    for (int r = first; r <= min(last, first + PNSLOT2 - 1); ++r) issue(r);
  }
  __syncwarp();

  bool ok = true;
  for (int r = first; r <= y0 + 1; ++r) ok = ok && wait_row(r);
  PGP g0, g1;
  q2 fbE, fbHx, fbHy, fbP, ftE, ftHx, ftHy, ftP;
  if (ok) {
    const PStagedRow2 &Rm2 = w.row[slot(y0 - 2)], &Rm1 = w.row[slot(y0 - 1)];
    const PStagedRow2 &R0 = w.row[slot(y0)], &R1 = w.row[slot(y0 + 1)];
    const PGP gm1 = pstaged_diffs(Rm2, Rm1, R0, q, 2);
    g0 = pstaged_diffs(Rm1, R0, R1, q, 2);
    const PRowP vm1 = pstaged_pair<true>(Rm1, q, 2), v0 = pstaged_pair<true>(R0, q, 2);
    face_flux_psi_p(psi_yside_p(vm1, gm1, Q4), psi_yside_p(v0, g0, MQ4), P.ky, fbE, fbHy, fbHx,
                    fbP);
    if (y0 == 0 && ylo_nr) {
      float e[2], hx[2], hy[2], ps[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const PSide<float> up = psi_yside<float>(GKS_COL(v0, ez, k), GKS_COL(v0, hx, k),
                                                 GKS_COL(v0, hy, k), GKS_COL(v0, ps, k),
                                                 GKS_COL(v0, eps, k), pg_of(g0, k), mq4);
        face_flux_psi<float>(psi_zero<float>(), up, p.fy, p.qy, prcp1(GKS_COL(v0, eps, k)), e[k],
                             hy[k], hx[k], ps[k]);
      }
      fbE = qk(e[0], e[1]); fbHx = qk(hx[0], hx[1]); fbHy = qk(hy[0], hy[1]);
      fbP = qk(ps[0], ps[1]);
    }
    __syncwarp();                                     // row y0-2 is read
    if (lane == 0 && first + PNSLOT2 <= last) issue(first + PNSLOT2);
  }
  q2 acc = Z2;                                        // 0 * (updated values): NaN iff one is not finite

  auto row = [&](int j, const PGP &gc, PGP &gn, q2 bE, q2 bHx, q2 bHy, q2 bP, q2 &tE, q2 &tHx,
                 q2 &tHy, q2 &tP) -> bool {
    if (!wait_row(j + 2)) return false;
    const PStagedRow2 &Rm = w.row[slot(j - 1)], &R0 = w.row[slot(j)];
    const PStagedRow2 &R1 = w.row[slot(j + 1)], &R2 = w.row[slot(j + 2)];
    gn = pstaged_diffs(R0, R1, R2, q, 2);
    const PRowP v0 = pstaged_pair<true>(R0, q, 2), v1 = pstaged_pair<true>(R1, q, 2);
    // left x-faces of A and B: l side the left neighbours, r side the lane's own cells
    const PRowP vl = pstaged_pair<true>(R0, q, 1);
    const PGP gl = pstaged_diffs(Rm, R0, R1, q, 1);
    q2 fxE, fxHx, fxHy, fxP;
    face_flux_psi_p(psi_xside_p(vl, gl, Q4), psi_xside_p(v0, gc, MQ4), P.kx, fxE, fxHx, fxHy, fxP);
    if (xedge) {
      if (loA) {                        // low-x face of column 0 (cell A)
        const PSide<float> rn = psi_xside<float>(v0.ez.x, v0.hx.x, v0.hy.x, v0.ps.x, v0.eps.x,
                                                 pg_of(gc, 0), mq4);
        face_flux_psi<float>(psi_zero<float>(), rn, p.fx, p.qx, prcp1(v0.eps.x), fxE.x, fxHx.x,
                             fxHy.x, fxP.x);
      }
      if (hiA) {                        // high-x face of column nx - 1 (left neighbour of A)
        const PSide<float> l0 = psi_xside<float>(vl.ez.x, vl.hx.x, vl.hy.x, vl.ps.x, vl.eps.x,
                                                 pg_of(gl, 0), q4);
        face_flux_psi<float>(l0, psi_zero<float>(), p.fx, p.qx, prcp1(vl.eps.x), fxE.x, fxHx.x,
                             fxHy.x, fxP.x);
      }
      if (hiB) {
        const PSide<float> l1 = psi_xside<float>(vl.ez.y, vl.hx.y, vl.hy.y, vl.ps.y, vl.eps.y,
                                                 pg_of(gl, 1), q4);
        face_flux_psi<float>(l1, psi_zero<float>(), p.fx, p.qx, prcp1(vl.eps.y), fxE.y, fxHx.y,
                             fxHy.y, fxP.y);
      }
    }
    // right faces: the next lane's left faces; for lane 31's A, lane 0's left face of B
    auto right = [lane](q2 f) {
      const float a = __shfl_down_sync(PFULL, f.x, 1), b = __shfl_sync(PFULL, f.y, 0);
      const float c = __shfl_down_sync(PFULL, f.y, 1);
      return qk(lane == 31 ? b : a, c);
    };
    const q2 frE = right(fxE), frHx = right(fxHx), frHy = right(fxHy), frP = right(fxP);
    // y-faces between rows j and j+1
    face_flux_psi_p(psi_yside_p(v0, gc, Q4), psi_yside_p(v1, gn, MQ4), P.ky, tE, tHy, tHx, tP);
    if (j + 1 == p.ny && yhi_nr) {
      float e[2], hx[2], hy[2], ps[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const PSide<float> lo = psi_yside<float>(GKS_COL(v0, ez, k), GKS_COL(v0, hx, k),
                                                 GKS_COL(v0, hy, k), GKS_COL(v0, ps, k),
                                                 GKS_COL(v0, eps, k), pg_of(gc, k), q4);
        face_flux_psi<float>(lo, psi_zero<float>(), p.fy, p.qy, prcp1(GKS_COL(v0, eps, k)), e[k],
                             hy[k], hx[k], ps[k]);
      }
      tE = qk(e[0], e[1]); tHx = qk(hx[0], hx[1]); tHy = qk(hy[0], hy[1]); tP = qk(ps[0], ps[1]);
    }
    // update row j
    q2 dE = qadd(qsub(fxE, frE), qsub(bE, tE));
    const q2 dHx = qadd(qsub(fxHx, frHx), qsub(bHx, tHx));
    const q2 dHy = qadd(qsub(fxHy, frHy), qsub(bHy, tHy));
    const q2 dP = qadd(qsub(fxP, frP), qsub(bP, tP));
    const int64_t ro = (int64_t)j * p.pitch;
    if (p.src && j >= p.sy0 && j < p.sy1) {
      if (A >= p.sx0 && A < p.sx1) dE.x -= p.src_amp * p.src[ro + A];
      if (B >= p.sx0 && B < p.sx1) dE.y -= p.src_amp * p.src[ro + B];
    }
    const q2 out[4] = {qfma(dE, qk(prcp1(v0.eps.x), prcp1(v0.eps.y)), v0.ez), qadd(v0.hx, dHx),
                       qadd(v0.hy, dHy), qadd(v0.ps, dP)};
    float *o = p.Vout + ro;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (stA) o[c * p.cstride + A] = out[c].x;
      if (stB) o[c * p.cstride + B] = out[c].y;
    }
    const q2 sum = qadd(qadd(out[0], out[1]), qadd(out[2], out[3]));
    if (stB) acc = qfma(sum, Z2, acc);                 // stB implies stA
    else if (stA) acc.x = fmaf(sum.x, 0.f, acc.x);
    __syncwarp();                                     // row j-1 is read
    if (lane == 0 && j + PNSLOT2 - 1 <= last) issue(j + PNSLOT2 - 1);
    return true;
  };

  int j = y0;
  if (ok) {
#pragma unroll 1
    for (; j + 1 < y1; j += 2) {
      if (!row(j, g0, g1, fbE, fbHx, fbHy, fbP, ftE, ftHx, ftHy, ftP) ||
          !row(j + 1, g1, g0, ftE, ftHx, ftHy, ftP, fbE, fbHx, fbHy, fbP)) {
        ok = false;
        break;
      }
    }
    if (ok && j < y1) ok = row(j, g0, g1, fbE, fbHx, fbHy, fbP, ftE, ftHx, ftHy, ftP);
  }
  if (lane == 0 && !ok) {
    atomicOr(p.flag, 2);                              // a row never landed
    for (int r = max(first, issued - PNSLOT2 + 1); r <= issued; ++r)   // copies in flight
      mbar_wait(&w.bar[slot(r)], parity(r));
  }
  if (__any_sync(PFULL, !(isfinite(acc.x) && isfinite(acc.y))) && lane == 0) atomicOr(p.flag, 1);
}

#undef GKS_COL

// The staged kernel covers FP32 without the limiter, without PEC walls and with a non-periodic
// x axis (a periodic y axis needs two rows for the wrap); about four waves of chunks of at least
// 8 rows.
bool psi_staged_supported(const CartGeom &g, const CartStepArgs &a) {
  if (a.limiter || g.periodic[0]) return false;
  for (int k = 0; k < 4; ++k)
    if (g.pec[k]) return false;
  if (g.periodic[1] && g.ny < 2) return false;
  return tensor_map_encoder() != nullptr;
}

cudaError_t launch_psi_staged(const CartGeom &g, const PsiPackArgs &P, cudaStream_t st) {
  const int smem = PWARPS * (int)sizeof(PWarpStage2);
  static int per_sm = 0, sms = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(cart2d_psi_step_kernel_s, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cart2d_psi_step_kernel_s, PWARPS * 32,
                                                  smem);
    if (sms < 1) sms = 1;
    if (per_sm < 1) per_sm = 1;
  }
  const int nstrips = (g.nx + PW2 - 1) / PW2;
  const int64_t want = (int64_t)sms * per_sm * PWARPS * 4 / nstrips;
  int nchunks = (int)(want > 1 ? want : 1);
  int rows = (g.ny + nchunks - 1) / nchunks;
  if (rows < 8) rows = 8;
  nchunks = (g.ny + rows - 1) / rows;
  const int64_t nwarps = (int64_t)nstrips * nchunks;
  const int grid = (int)((nwarps + PWARPS - 1) / PWARPS);
  CUtensorMap tmV, tmE;
  const cuuint64_t dim[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 4};
  const cuuint64_t stride[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.cstride * 4};
  const cuuint32_t box[3] = {PTW2, 1, 4};
  if (!encode_f32_map(&tmV, P.b.V, 3, dim, stride, box) ||
      !encode_f32_map(&tmE, P.b.eps, 2, dim, stride, box))
    return cudaErrorInvalidValue;
  cart2d_psi_step_kernel_s<<<grid, PWARPS * 32, smem, st>>>(tmV, tmE, P, nstrips, rows);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_psi_t(const CartGeom &g, const CartStepArgs &a, double gamma,
                         cudaStream_t st) {
  PsiArgs<T> p;
  p.V = static_cast<const T *>(a.V);
  p.Vout = static_cast<T *>(a.Vout);
  p.eps = static_cast<const T *>(a.eps);
  p.src = static_cast<const T *>(a.src);
  p.sx0 = a.src_box[0]; p.sx1 = a.src_box[1];
  p.sy0 = a.src_box[2]; p.sy1 = a.src_box[3];
  p.src_amp = T(a.src_amp);
  p.nx = g.nx; p.ny = g.ny;
  p.pitch = g.pitch; p.cstride = g.cstride;
  p.perx = g.periodic[0]; p.pery = g.periodic[1];
  for (int k = 0; k < 4; ++k) p.pec[k] = g.pec[k];
  p.fx = make_face_k<T>(a.C, g.h[0], g.h[1], a.c, 1.0, 1.0);
  p.fy = make_face_k<T>(a.C, g.h[1], g.h[0], a.c, -1.0, -1.0);
  p.qx = make_face_psi<T>(a.C, g.h[0], g.h[1], a.c, 1.0, 1.0, gamma);
  p.qy = make_face_psi<T>(a.C, g.h[1], g.h[0], a.c, -1.0, -1.0, gamma);
  p.flag = a.flag;
  const int nstrips = (g.nx + PCOLS - 1) / PCOLS;
  int rows = g.ny;
  const int target = 152 * 16;
  if (nstrips < target) {
    const int chunks = (target + nstrips - 1) / nstrips;
    rows = (g.ny + chunks - 1) / chunks;
  }
  rows = rows < 4 ? 4 : (rows > 256 ? 256 : rows);
  const int nchunks = (g.ny + rows - 1) / rows;
  const int64_t nwarps = (int64_t)nstrips * nchunks;
  const int grid = (int)((nwarps + PWARPS - 1) / PWARPS);
  const bool pec = g.pec[0] || g.pec[1] || g.pec[2] || g.pec[3];
  if constexpr (sizeof(T) == 4) {      // FP32: the paired-instruction kernel
    PsiPackArgs P;
    P.b = p;
    P.kx = make_psi_kp(p.fx, p.qx);
    P.ky = make_psi_kp(p.fy, p.qy);
    if (psi_staged_supported(g, a)) return launch_psi_staged(g, P, st);
    using KP = void (*)(const PsiPackArgs, int, int);
    static const KP kp[2][2] = {{cart2d_psi_step_kernel_p<false, false>,
                                 cart2d_psi_step_kernel_p<false, true>},
                                {cart2d_psi_step_kernel_p<true, false>,
                                 cart2d_psi_step_kernel_p<true, true>}};   // [pec][limiter]
    kp[pec ? 1 : 0][a.limiter ? 1 : 0]<<<grid, PWARPS * 32, 0, st>>>(P, nstrips, rows);
    return cudaGetLastError();
  }
  using K = void (*)(const PsiArgs<T>, int, int);
  static const K kern[2][2] = {{cart2d_psi_step_kernel<T, false, false>,
                                cart2d_psi_step_kernel<T, false, true>},
                               {cart2d_psi_step_kernel<T, true, false>,
                                cart2d_psi_step_kernel<T, true, true>}};   // [pec][limiter]
  kern[pec ? 1 : 0][a.limiter ? 1 : 0]<<<grid, PWARPS * 32, 0, st>>>(p, nstrips, rows);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cart2d_psi_step(const CartGeom &g, const CartStepArgs &a, double gamma,
                                   bool fp64, cudaStream_t st) {
  return fp64 ? launch_psi_t<double>(g, a, gamma, st) : launch_psi_t<float>(g, a, gamma, st);
}

}  // namespace gks
