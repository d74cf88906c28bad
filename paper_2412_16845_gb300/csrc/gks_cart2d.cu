// Fused 2-D TM GKS step on a Cartesian grid: cell gradients, face reconstruction, the GKS
// interface flux and the finite-volume update in one pass over the state (Sec. 3.1).
//
// Row-marching scheme.  A CTA of NT threads owns a strip of W = NT - 2 columns and a chunk of
// rows, and walks up the rows with one barrier per row.  Thread t owns column X = x0 - 1 + t
// and keeps its own column of the state, eps, central differences and the y-face flux in
// registers; shared memory holds the current rows only for the x-neighbours.  Every gradient
// and every face is evaluated once: per row a thread forms the differences of row j+1, the
// x-face X - 1/2 and the y-face j + 1/2, and updates its cell of row j.
//
// Face frames (Sec. 3.1, T'(n)): an x-face uses n = e_x (T' = I); a y-face n = e_y with local
// axes (x', y') = (y, -x); the low boundary faces use the outward normals -e_x (T' =
// diag(-1,-1,1)) and -e_y (local (x', y') = (-y, x)).  In 2-D TM the third-moment term of the
// D3Q4 flux vanishes, so a TM face flux does not depend on the tangential orientation.
#include <cuda_runtime.h>

#include "gks_internal.h"

namespace gks {
namespace {

constexpr int NT = 128;            // threads per CTA, one column each
constexpr int W = NT - 2;          // columns updated per CTA
constexpr int ROWS = 64;           // rows per CTA

// Reciprocals: FP32 uses the fast hardware reciprocal (about 1 ulp), FP64 divides.
__device__ __forceinline__ float rcp1(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp1(double x) { return 1.0 / x; }
__device__ __forceinline__ float rcp2(float x) { return __fdividef(2.f, x); }
__device__ __forceinline__ double rcp2(double x) { return 2.0 / x; }

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
  T inv2hx, inv2hy;
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

// ------------------------------------------------------------------ asynchronous row copies
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem));
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

constexpr int NS = 8;      // row slots in the shared-memory ring
constexpr int AHEAD = 4;   // rows in flight beyond the ones being used

// Shared memory (per CTA): a ring of staged rows V[NS][5][NT+2] (Ez, Hx, Hy, eps, mu of
// columns x0-2 .. x0+NT-1, filled by cp.async), raw differences G[2][5][NT] (x-differences of
// Ez, Hx, Hy and y-differences of Hx, Ez of columns x0-1 .. x0+NT-2), and each thread's
// x-face flux F[2][3][NT].
template <typename T>
struct Smem {
  T V[NS][5][NT + 2];
  T G[2][5][NT];
  T F[2][3][NT];
};

// Issue the copies of row `row` (wrapped or clamped) for the own column and, for threads 0 and
// NT-1, the extra column, into ring slot row mod NS.
template <typename T, bool HAS_MU>
__device__ __forceinline__ void issue_row(Smem<T> &s, const Cart2DKernelArgs<T> &p, int t, int X,
                                          bool has_extra, int extra_col, int extra_idx, int row) {
  const int slot = (row + 2 * NS) % NS;
  const int r = wrap_or_clamp(row, p.ny, p.pery);
  const int64_t ro = (int64_t)r * p.pitch;
  {
    const int c = wrap_or_clamp(X, p.nx, p.perx);
    const int64_t o = ro + c;
    cp_async(&s.V[slot][0][t + 1], p.V + o, sizeof(T));
    cp_async(&s.V[slot][1][t + 1], p.V + p.cstride + o, sizeof(T));
    cp_async(&s.V[slot][2][t + 1], p.V + 2 * p.cstride + o, sizeof(T));
    cp_async(&s.V[slot][3][t + 1], p.eps + o, sizeof(T));
    if (HAS_MU) cp_async(&s.V[slot][4][t + 1], p.mu + o, sizeof(T));
  }
  if (has_extra) {
    const int c = wrap_or_clamp(extra_col, p.nx, p.perx);
    const int64_t o = ro + c;
    cp_async(&s.V[slot][0][extra_idx], p.V + o, sizeof(T));
    cp_async(&s.V[slot][1][extra_idx], p.V + p.cstride + o, sizeof(T));
    cp_async(&s.V[slot][2][extra_idx], p.V + 2 * p.cstride + o, sizeof(T));
    cp_async(&s.V[slot][3][extra_idx], p.eps + o, sizeof(T));
    if (HAS_MU) cp_async(&s.V[slot][4][extra_idx], p.mu + o, sizeof(T));
  }
  cp_async_commit();
}

template <typename T, bool HAS_MU>
__device__ __forceinline__ RowV<T> own_cell(const Smem<T> &s, int row, int t) {
  const int slot = (row + 2 * NS) % NS;
  RowV<T> v;
  v.ez = s.V[slot][0][t + 1];
  v.hx = s.V[slot][1][t + 1];
  v.hy = s.V[slot][2][t + 1];
  v.eps = s.V[slot][3][t + 1];
  v.mu = HAS_MU ? s.V[slot][4][t + 1] : T(1);
  return v;
}

// Raw central differences of the own column in row `row` (all neighbours staged).
template <typename T>
__device__ __forceinline__ RowG<T> grad_row(const Smem<T> &s, int row, int t) {
  const int sl = (row + 2 * NS) % NS, dn = (row - 1 + 2 * NS) % NS, up = (row + 1 + 2 * NS) % NS;
  RowG<T> g;
  g.ex = s.V[sl][0][t + 2] - s.V[sl][0][t];
  g.ax = s.V[sl][1][t + 2] - s.V[sl][1][t];
  g.bx = s.V[sl][2][t + 2] - s.V[sl][2][t];
  g.ey = s.V[up][0][t + 1] - s.V[dn][0][t + 1];
  g.ay = s.V[up][1][t + 1] - s.V[dn][1][t + 1];
  g.by = s.V[up][2][t + 1] - s.V[dn][2][t + 1];
  return g;
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

// Row loop.  Iteration j (after one barrier) issues the copies of row j+6, completes the
// update of row j-1, forms the differences of row j+1, the x-face X-1/2 and the y-face j+1/2
// of row j, and publishes the differences and the x-face for the neighbours.  Rows j-1 .. j+2
// are read while rows j+3 .. j+6 are in flight (ring of NS = 8 slots).
template <typename T, bool HAS_MU>
__global__ void __launch_bounds__(NT) cart2d_step_kernel(const Cart2DKernelArgs<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<T> &s = *reinterpret_cast<Smem<T> *>(smem_raw);
  const int t = threadIdx.x;
  const int x0 = blockIdx.x * W;
  const int y0 = blockIdx.y * ROWS;
  const int y1 = min(y0 + ROWS, p.ny);
  const int X = x0 - 1 + t;                         // own column
  const bool upd = t >= 1 && t <= NT - 2 && X < p.nx;
  const bool xnr = !p.perx, ynr = !p.pery;
  const T q4 = T(0.25), mq4 = T(-0.25);
  const bool has_extra = (t == 0) || (t == NT - 1);
  const int extra_col = (t == 0) ? x0 - 2 : x0 + NT - 1;
  const int extra_idx = (t == 0) ? 0 : NT + 1;

  // ---------------- prologue: rows y0-2 .. y0+5 in flight, differences of rows y0-1, y0
#pragma unroll 1
  for (int r = y0 - 2; r <= y0 + AHEAD + 1; ++r)
    issue_row<T, HAS_MU>(s, p, t, X, has_extra, extra_col, extra_idx, r);
  cp_async_wait<AHEAD - 1>();      // rows up to y0+2 landed
  __syncthreads();
  RowG<T> g0 = grad_row<T>(s, y0, t);
  T fbE, fbHx, fbHy;   // flux along +y through the face below the row being processed
  {
    const RowV<T> v0 = own_cell<T, HAS_MU>(s, y0, t);
    if (y0 == 0 && ynr) {
      // outward normal -e_y: from the +e_y frame quantities, local (x', y') = (-y, x)
      const Side<T> sq = yside_scalar<T>(v0, g0, mq4, p.inv2hx, p.inv2hy);
      Side<T> q;
      q.e = sq.e; q.a = -sq.a; q.b = -sq.b;
      q.ex = -sq.ex; q.ax = sq.ax; q.bx = sq.bx;
      q.ay = sq.ay; q.ey = -sq.ey;
      q.eps = sq.eps; q.mu = sq.mu;
      T oe, oa, ob;
      tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
      fbE = -oe; fbHx = -ob; fbHy = oa;
    } else {
      const RowG<T> gm1 = grad_row<T>(s, y0 - 1, t);
      const RowV<T> vm1 = own_cell<T, HAS_MU>(s, y0 - 1, t);
      face_flux<T, HAS_MU>(yface_side<T>(vm1, gm1, q4), yface_side<T>(v0, g0, mq4), p.fy, fbE,
                           fbHy, fbHx);
    }
  }
  {
    const int gs = y0 & 1;
    s.G[gs][0][t] = g0.ex; s.G[gs][1][t] = g0.ax; s.G[gs][2][t] = g0.bx;
    s.G[gs][3][t] = g0.ay; s.G[gs][4][t] = g0.ey;
  }
  // fluxes of the row whose update is pending
  T pxE = 0, pxHx = 0, pxHy = 0, pbE = 0, pbHx = 0, pbHy = 0, ptE = 0, ptHx = 0, ptHy = 0;
  bool bad = false;
#pragma unroll 1
  for (int j = y0; j <= y1; ++j) {
    cp_async_wait<AHEAD - 1>();    // row j+2 landed (this thread's copies)
    __syncthreads();               // ... and everyone's; G and F of the previous row visible
    if (j + AHEAD + 2 < y1 + 3) issue_row<T, HAS_MU>(s, p, t, X, has_extra, extra_col, extra_idx,
                                                    j + AHEAD + 2);
    else cp_async_commit();        // keep the group count uniform
    // finish the update of row j-1
    if (j > y0 && upd) {
      const int fs = (j - 1) & 1;
      const RowV<T> v = own_cell<T, HAS_MU>(s, j - 1, t);
      T dE = (pxE - s.F[fs][0][t + 1]) + (pbE - ptE);
      const T dHx = (pxHx - s.F[fs][1][t + 1]) + (pbHx - ptHx);
      const T dHy = (pxHy - s.F[fs][2][t + 1]) + (pbHy - ptHy);
      const int64_t o = (int64_t)(j - 1) * p.pitch + X;
      if (p.src && j - 1 >= p.sy0 && j - 1 < p.sy1 && X >= p.sx0 && X < p.sx1)
        dE -= p.src_amp * p.src[o];
      const T ve = v.ez + dE * rcp1(v.eps);
      T vhx, vhy;
      if (HAS_MU) {
        const T im = rcp1(v.mu);
        vhx = v.hx + dHx * im;
        vhy = v.hy + dHy * im;
      } else {
        vhx = v.hx + dHx;
        vhy = v.hy + dHy;
      }
      p.Vout[o] = ve;
      p.Vout[p.cstride + o] = vhx;
      p.Vout[2 * p.cstride + o] = vhy;
      bad |= !(isfinite(ve) && isfinite(vhx) && isfinite(vhy));
    }
    if (j == y1) break;
    const RowV<T> v0 = own_cell<T, HAS_MU>(s, j, t);
    const RowG<T> g1 = grad_row<T>(s, j + 1, t);
    // x-face X - 1/2 of row j (left cell X-1 from shared memory)
    T fxE = 0, fxHx = 0, fxHy = 0;
    if (t >= 1) {
      const int sl = j % NS, gs = j & 1;
      RowV<T> lv;
      lv.ez = s.V[sl][0][t]; lv.hx = s.V[sl][1][t]; lv.hy = s.V[sl][2][t];
      lv.eps = s.V[sl][3][t]; lv.mu = HAS_MU ? s.V[sl][4][t] : T(1);
      RowG<T> lg;
      lg.ex = s.G[gs][0][t - 1]; lg.ax = s.G[gs][1][t - 1]; lg.bx = s.G[gs][2][t - 1];
      lg.ay = s.G[gs][3][t - 1]; lg.ey = s.G[gs][4][t - 1]; lg.by = T(0);
      if (xnr && X == 0) {
        low_boundary_flux<T>(xside_scalar<T>(v0, g0, mq4, p.inv2hx, p.inv2hy), p.Kx, fxE, fxHx,
                             fxHy);
      } else if (xnr && X == p.nx) {
        const Side<T> q = xside_scalar<T>(lv, lg, q4, p.inv2hx, p.inv2hy);
        tm_face_flux<T, true>(q, q, p.Kx, fxE, fxHx, fxHy);
      } else {
        face_flux<T, HAS_MU>(xface_side<T>(lv, lg, q4), xface_side<T>(v0, g0, mq4), p.fx, fxE,
                             fxHx, fxHy);
      }
    }
    // y-face between rows j and j+1
    T ftE, ftHx, ftHy;
    if (j + 1 == p.ny && ynr) {
      const Side<T> q = yside_scalar<T>(v0, g0, q4, p.inv2hx, p.inv2hy);
      T oe, oa, ob;
      tm_face_flux<T, true>(q, q, p.Ky, oe, oa, ob);
      ftE = oe; ftHx = -ob; ftHy = oa;
    } else {
      const RowV<T> v1 = own_cell<T, HAS_MU>(s, j + 1, t);
      face_flux<T, HAS_MU>(yface_side<T>(v0, g0, q4), yface_side<T>(v1, g1, mq4), p.fy, ftE,
                           ftHy, ftHx);
    }
    // publish differences of row j+1 and this thread's x-face of row j
    {
      const int gs = (j + 1) & 1, fs = j & 1;
      s.G[gs][0][t] = g1.ex; s.G[gs][1][t] = g1.ax; s.G[gs][2][t] = g1.bx;
      s.G[gs][3][t] = g1.ay; s.G[gs][4][t] = g1.ey;
      s.F[fs][0][t] = fxE; s.F[fs][1][t] = fxHx; s.F[fs][2][t] = fxHy;
    }
    pxE = fxE; pxHx = fxHx; pxHy = fxHy;
    pbE = fbE; pbHx = fbHx; pbHy = fbHy;
    ptE = ftE; ptHx = ftHx; ptHy = ftHy;
    g0 = g1;
    fbE = ftE; fbHx = ftHx; fbHy = ftHy;
  }
  cp_async_wait<0>();
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

// Constants of face_flux for a face of normal spacing hn and tangential spacing ht whose frame
// has tangential-H sign sb and tangential-derivative sign st (x-faces: +1, +1; y-faces: -1, -1).
// Differences along the normal carry 1/(2 hn), along the tangent 1/(2 ht).
template <typename T>
FaceK<T> make_face_k(const double C[5], double hn, double ht, double c, double sb, double st) {
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
  p.fx = make_face_k<T>(a.C, g.h[0], g.h[1], a.c, 1.0, 1.0);
  p.fy = make_face_k<T>(a.C, g.h[1], g.h[0], a.c, -1.0, -1.0);
  p.Kx = make_coef<T>(a.C, g.h[0], a.c);
  p.Ky = make_coef<T>(a.C, g.h[1], a.c);
  p.flag = a.flag;
  dim3 grid((g.nx + W - 1) / W, (g.ny + ROWS - 1) / ROWS);
  const int smem = (int)sizeof(Smem<T>);
  if (a.mu) {
    cudaFuncSetAttribute(cart2d_step_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
    cart2d_step_kernel<T, true><<<grid, NT, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(cart2d_step_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         smem);
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
