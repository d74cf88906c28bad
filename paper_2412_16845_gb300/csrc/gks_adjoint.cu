// Adjoint of the 2-D TM GKS step and the probe objective (not in the paper; the gradient of a
// field-energy objective with respect to per-cell eps).
//
// Forward map of one step (eps fixed): V^{n+1} = L V^n + s^n, with L linear.  With
// J = sum_{n=1}^{N} q(V^n), q(V) = dt sum_{i in P} |Omega_i| Ez_i^2, the adjoint recursion is
//     lambda^N = dq/dV^N,   lambda^n = L^T lambda^{n+1} + [n >= 1] dq/dV^n,
//     dJ/deps_d = sum_{n=0}^{N-1} (d(L V^n + s^n)/d eps_d)^T lambda^{n+1}.
// L^T is the transpose of the fused stencil, taken by hand: the update adds F/M with sign to
// the two cells of each face, so each face receives Fbar = -(lambda_L/M_L - lambda_R/M_R); the
// closed-form face flux (sums and differences of the two sides, see face_flux in
// gks_cart2d.cu) is transposed term by term; the reconstruction V +- d/4 and the central
// differences d = V_{+1} - V_{-1} (with the forward's clamp/wrap ghosts) are transposed last.
// The eps-derivative of a step is the derivative of the face fluxes of the design cell's faces
// plus -lambda_E (E^{n+1} - E^n)/eps from the 1/eps of the update.  mu = 1 only.
#include <cuda_runtime.h>

#include <algorithm>

#include "gks_flux2.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

// Division: FP32 uses the fast hardware reciprocal (about 1 ulp), FP64 divides.
__device__ __forceinline__ float fdv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdv(double a, double b) { return a / b; }

// Adjoint of one interior / boundary face (GH: 0 interior, 1 ghost on the low side, 2 ghost on
// the high side).  Given Fbar = (fe, fa, fb) in the face's component order (Ez, Hn, Ht), returns
// per side the adjoints of the cell values (Ez, Hn, Ht) and of the raw differences
// (den, dhn, dht, dat, det) the forward flux used.
template <typename T>
struct FOut {
  T v[3];
  T d[5];
};

template <typename T, int GH>
__device__ __forceinline__ void face_adj(T epsl, T epsr, const FaceK<T> &k, T fe, T fa, T fb,
                                         FOut<T> &oL, FOut<T> &oR) {
  const T ie = GH == 0 ? fdv(T(2), epsl + epsr) : (GH == 1 ? fdv(T(1), epsr) : fdv(T(1), epsl));
  const T g = k.g0 - k.k3 * ie;
  const T w1 = g * fe;
  const T SUB = k.a1 * fe, De = k.a2 * fe;
  const T SUxe = T(0.5) * w1 - k.q3 * fe, DxB = k.a3 * w1 + k.a6 * fe, SB = k.a4 * fe;
  const T DUe = -k.q2 * fe, DAt = k.a5 * fe;
  const T SUxa = k.q5 * fa, DUa = -k.q2 * fa, DEt = k.b1 * fa;
  const T w2 = ie * fb, w3 = g * fb;
  const T SUe = k.c1 * w2, DB = k.c2 * w2 - k.q2 * fb;
  const T SUxB = T(0.5) * w3 - k.q3 * fb, Dex = k.c3 * w3 + k.c6 * fb;
  const T SUAt = k.c4 * ie * fb, Se = k.c5 * fb;
  // side l: differences enter with -1, reconstruction V + d/4; side r: +1, V - d/4
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    if ((side == 0 && GH == 1) || (side == 1 && GH == 2)) continue;
    const T sg = side == 0 ? T(-1) : T(1);
    const T rho = side == 0 ? T(0.25) : T(-0.25);
    const T eps = side == 0 ? epsl : epsr;
    FOut<T> &o = side == 0 ? oL : oR;
    const T eb = sg * De + Se + eps * (sg * DUe + SUe);
    const T hnb = sg * DUa;
    const T htb = SUB + SB + sg * DB;
    o.v[0] = eb;
    o.v[1] = hnb;
    o.v[2] = htb;
    o.d[0] = eps * SUxe + sg * Dex + rho * eb;
    o.d[1] = SUxa + rho * hnb;
    o.d[2] = sg * DxB + SUxB + rho * htb;
    o.d[3] = sg * DAt + SUAt;
    o.d[4] = sg * DEt;
  }
}

// Cell data for the eps-derivative: cell values (Ez, Hn, Ht), raw differences
// (den, dhn, dht, dat, det) and eps.
template <typename T>
struct FIn {
  T v[3];
  T d[5];
  T eps;
};

// d F / d eps of a face for its low (dl) and high (dr) side, V fixed (forward quantities).
template <typename T, int GH>
__device__ __forceinline__ void face_deps(const FIn<T> &L, const FIn<T> &R, const FaceK<T> &k,
                                          T dl[3], T dr[3]) {
  const bool hasl = GH != 1, hasr = GH != 2;
  const T el = hasl ? L.v[0] + T(0.25) * L.d[0] : T(0);
  const T htl = hasl ? L.v[2] + T(0.25) * L.d[2] : T(0);
  const T er = hasr ? R.v[0] - T(0.25) * R.d[0] : T(0);
  const T htr = hasr ? R.v[2] - T(0.25) * R.d[2] : T(0);
  const T denl = hasl ? L.d[0] : T(0), denr = hasr ? R.d[0] : T(0);
  const T dhtl = hasl ? L.d[2] : T(0), dhtr = hasr ? R.d[2] : T(0);
  const T datl = hasl ? L.d[3] : T(0), datr = hasr ? R.d[3] : T(0);
  const T epl = hasl ? L.eps : T(0), epr = hasr ? R.eps : T(0);
  const T S_Uxe = epl * denl + epr * denr, D_xB = dhtr - dhtl;
  const T S_Ue = epl * el + epr * er, D_B = htr - htl;
  const T S_UxB = dhtl + dhtr, D_ex = denr - denl, S_UAt = datl + datr;
  const T ie = GH == 0 ? fdv(T(2), L.eps + R.eps) : (GH == 1 ? fdv(T(1), R.eps) : fdv(T(1), L.eps));
  const T die = GH == 0 ? -T(0.5) * ie * ie : -ie * ie;
  const T g = k.g0 - k.k3 * ie, dg = -k.k3 * die;
  const T A = dg * (T(0.5) * S_Uxe + k.a3 * D_xB);
  const T B = die * (k.c1 * S_Ue + k.c2 * D_B) + dg * (T(0.5) * S_UxB + k.c3 * D_ex) +
              k.c4 * die * S_UAt;
  dl[0] = hasl ? A + (T(0.5) * g - k.q3) * denl + k.q2 * el : T(0);
  dl[1] = T(0);
  dl[2] = hasl ? B + ie * k.c1 * el : T(0);
  dr[0] = hasr ? A + (T(0.5) * g - k.q3) * denr - k.q2 * er : T(0);
  dr[1] = T(0);
  dr[2] = hasr ? B + ie * k.c1 * er : T(0);
}

template <typename T>
struct AdjArgs {
  const T *__restrict__ lam;      // lambda^{n+1}
  T *__restrict__ lout;           // lambda^n
  const T *__restrict__ eps;
  const T *__restrict__ Vn;       // state at t^n (probe cells; design box for the gradient)
  const T *__restrict__ Vn1;      // state at t^{n+1} (design cells only)
  const int32_t *__restrict__ dslot;   // design slot per cell or -1
  double *__restrict__ grad;      // [nd] += dJ/deps
  const double *__restrict__ pw;  // probe weights over the probe box (row-major) or null
  int px0, px1, py0, py1;         // probe box (half open)
  double dt2;                     // 2 dt
  int dx0, dx1, dy0, dy1;         // design box (half open)
  int nx, ny;
  int64_t pitch, cstride;
  int perx, pery;
  FaceK<T> fx, fy;
};

__device__ __forceinline__ int wc(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Face type relative to the domain: 0 interior, 1 ghost low, 2 ghost high, 3 outside.
__device__ __forceinline__ int face_kind(int lo_cell, int n, int periodic) {
  if (periodic) return 0;
  const int hi_cell = lo_cell + 1;
  if (lo_cell >= 0 && hi_cell < n) return 0;
  if (lo_cell == -1 && hi_cell < n) return 1;
  if (lo_cell == n - 1) return 2;
  return 3;
}

// Face adjoint from the adjoints of its two cells in face components: (qL, aL, bL) =
// (lambda_E / eps, lambda_Hn, lambda_Ht) of the low side, likewise the high side.  The update adds
// +F/M to the low cell and -F/M to the high cell, so Fbar = lambda_R/M_R - lambda_L/M_L.
template <typename T>
__device__ __forceinline__ void face_adj2(T el, T er, const FaceK<T> &k, T qL, T aL, T bL, T qR,
                                          T aR, T bR, FOut<T> &oL, FOut<T> &oR) {
  face_adj<T, 0>(el, er, k, qR - qL, aR - aL, bR - bL, oL, oR);
}

// ------------------------------------------------------------------ lambda^n = L^T lambda^{n+1}
// Warp-strip march, the transpose of the forward's: a warp owns 64 columns x0-2 .. x0+61 (lane
// l: X = x0-2+2l and X+1) and walks up a chunk of rows; lanes 1..30 write columns x0 .. x0+59.
// Per row j a lane evaluates the face adjoints of its x-faces X+1/2, X+3/2 and of the y-faces
// j+1/2 of its two columns, gathers them into the value adjoints and the raw-difference adjoints
// (dbar) of its cells, applies D_x^T (neighbours by shuffle) and pushes the y-difference adjoints
// of row j to rows j-1 (-) and j+1 (+): row j-1 is complete and is written.  No shared memory,
// no barriers.  The probe term is added by adjoint_post_kernel.
constexpr int AWARPS = 4;
constexpr int AWCOLS = 60;
constexpr unsigned AFULL = 0xffffffffu;

template <typename T> struct APair;
template <> struct APair<float> { using type = float2; };
template <> struct APair<double> { using type = double2; };

// lambda (Ez, Hx, Hy), eps and lambda_E / eps of two columns of a row
template <typename T>
struct ARow {
  T e[2], a[2], b[2], ep[2], q[2];
};

// Off the grid (non-periodic axes) the lambda of a cell is zero and its eps is the clamped copy
// of the edge cell: the interior face formula then is the boundary face's (Fbar from the inner
// side only, eps_s = 2 / (eps + eps) = 1 / eps of the inner side), and what it writes to the
// outer side lands on cells that are never stored.
template <typename T>
__device__ __forceinline__ ARow<T> load_arow(const AdjArgs<T> &p, int X, int row) {
  using P = typename APair<T>::type;
  ARow<T> r;
  const bool rin = p.pery || (row >= 0 && row < p.ny);
  const int64_t ro = (int64_t)wc(row, p.ny, p.pery) * p.pitch;
  if (X >= 0 && X + 1 < p.nx) {
    const P e = __ldg(reinterpret_cast<const P *>(p.lam + ro + X));
    const P a = __ldg(reinterpret_cast<const P *>(p.lam + p.cstride + ro + X));
    const P b = __ldg(reinterpret_cast<const P *>(p.lam + 2 * p.cstride + ro + X));
    const P m = __ldg(reinterpret_cast<const P *>(p.eps + ro + X));
    r.e[0] = e.x; r.e[1] = e.y; r.a[0] = a.x; r.a[1] = a.y;
    r.b[0] = b.x; r.b[1] = b.y; r.ep[0] = m.x; r.ep[1] = m.y;
    if (!rin) {
#pragma unroll
      for (int k = 0; k < 2; ++k) r.e[k] = r.a[k] = r.b[k] = T(0);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int64_t o = ro + wc(X + k, p.nx, p.perx);
      const bool in = rin && (p.perx || (X + k >= 0 && X + k < p.nx));
      r.e[k] = in ? __ldg(p.lam + o) : T(0);
      r.a[k] = in ? __ldg(p.lam + p.cstride + o) : T(0);
      r.b[k] = in ? __ldg(p.lam + 2 * p.cstride + o) : T(0);
      r.ep[k] = __ldg(p.eps + o);
    }
  }
  return r;
}

template <typename T>
__device__ __forceinline__ void finish_arow(ARow<T> &r) {
  r.q[0] = fdv(r.e[0], r.ep[0]);
  r.q[1] = fdv(r.e[1], r.ep[1]);
}

// adjoints gathered into one cell: values (E, Hx, Hy) and raw differences
template <typename T>
struct ACell {
  T vE, vA, vB, dEx, dEy, dAx, dAy, dBx, dBy;
};

// x-face components: v (Ez, Hx, Hy), d (dEx, dAx, dBx, dAy, dEy)
template <typename T>
__device__ __forceinline__ void add_xface(ACell<T> &c, const FOut<T> &o) {
  c.vE += o.v[0]; c.vA += o.v[1]; c.vB += o.v[2];
  c.dEx += o.d[0]; c.dAx += o.d[1]; c.dBx += o.d[2]; c.dAy += o.d[3]; c.dEy += o.d[4];
}
// y-face components: v (Ez, Hy, Hx), d (dEy, dBy, dAy, dBx, dEx)
template <typename T>
__device__ __forceinline__ void add_yface(ACell<T> &c, const FOut<T> &o) {
  c.vE += o.v[0]; c.vB += o.v[1]; c.vA += o.v[2];
  c.dEy += o.d[0]; c.dBy += o.d[1]; c.dAy += o.d[2]; c.dBx += o.d[3]; c.dEx += o.d[4];
}
template <typename T>
__device__ __forceinline__ ACell<T> cell_from_yface(const FOut<T> &o) {
  ACell<T> c;
  c.vE = o.v[0]; c.vB = o.v[1]; c.vA = o.v[2];
  c.dEy = o.d[0]; c.dBy = o.d[1]; c.dAy = o.d[2]; c.dBx = o.d[3]; c.dEx = o.d[4];
  c.dAx = T(0);
  return c;
}

template <typename T>
__global__ void __launch_bounds__(AWARPS * 32) adjoint_lambda_kernel(const AdjArgs<T> p, int nstrips,
                                                                     int rows) {
  const int lane = threadIdx.x & 31;
  const int wid = blockIdx.x * AWARPS + (threadIdx.x >> 5);
  const int strip = wid % nstrips, chunk = wid / nstrips;
  const int y0 = chunk * rows;
  if (y0 >= p.ny) return;                              // whole warp leaves together
  const int y1 = min(y0 + rows, p.ny);
  const int x0 = strip * AWCOLS;
  const int X = x0 - 2 + 2 * lane;
  const int xend = min(x0 + AWCOLS, p.nx);
  // D_x^T weights of the lane's two columns (cell i gets cl dbar_{i-1} - cr dbar_{i+1} +
  // cs dbar_i: d_i = V(i+1) - V(i-1) with clamped ends, or wrapped)
  T cl[2], cr[2], cs[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int i = X + k;
    cl[k] = p.perx || i - 1 >= 0 ? T(1) : T(0);
    cr[k] = p.perx || i + 1 < p.nx ? T(1) : T(0);
    cs[k] = p.perx ? T(0) : T((i == p.nx - 1 ? 1 : 0) - (i == 0 ? 1 : 0));
  }

  ARow<T> cur = load_arow(p, X, y0 - 1);
  ARow<T> nxt = load_arow(p, X, y0);
  ARow<T> pf = load_arow(p, X, y0 + 1);
  ACell<T> A[2];                                       // row j, bottom y-face gathered
  {
    ARow<T> rm = load_arow(p, X, y0 - 2);
    finish_arow(rm);
    finish_arow(cur);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      FOut<T> oL, oR;
      face_adj2<T>(rm.ep[k], cur.ep[k], p.fy, rm.q[k], rm.b[k], rm.a[k], cur.q[k],
                      cur.b[k], cur.a[k], oL, oR);
      A[k] = cell_from_yface(oR);
    }
  }
  finish_arow(nxt);
  T pend[3][2], carry[3][2];                           // row j-1 output so far; +dbar_y of j-1
#pragma unroll
  for (int c = 0; c < 3; ++c) { pend[c][0] = pend[c][1] = carry[c][0] = carry[c][1] = T(0); }

#pragma unroll 1
  for (int j = y0 - 1; j <= y1; ++j) {
    const ARow<T> pf2 = load_arow(p, X, j + 3);
    // x-faces of row j: X+1/2 (own columns) and X+3/2 (column X+2 from the next lane)
    {
      const T nq = __shfl_down_sync(AFULL, cur.q[0], 1), na = __shfl_down_sync(AFULL, cur.a[0], 1);
      const T nb = __shfl_down_sync(AFULL, cur.b[0], 1), ne = __shfl_down_sync(AFULL, cur.ep[0], 1);
      FOut<T> oL, oR;
      face_adj2<T>(cur.ep[0], cur.ep[1], p.fx, cur.q[0], cur.a[0], cur.b[0], cur.q[1],
                      cur.a[1], cur.b[1], oL, oR);
      add_xface(A[0], oL);
      add_xface(A[1], oR);
      face_adj2<T>(cur.ep[1], ne, p.fx, cur.q[1], cur.a[1], cur.b[1], nq, na, nb, oL, oR);
      add_xface(A[1], oL);
      // column X is the high side of the previous lane's second face
      FOut<T> l;
#pragma unroll
      for (int c = 0; c < 3; ++c) l.v[c] = __shfl_up_sync(AFULL, oR.v[c], 1);
#pragma unroll
      for (int c = 0; c < 5; ++c) l.d[c] = __shfl_up_sync(AFULL, oR.d[c], 1);
      add_xface(A[0], l);
    }
    // y-faces j+1/2
    ACell<T> B[2];
    {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        FOut<T> oL, oR;
        face_adj2<T>(cur.ep[k], nxt.ep[k], p.fy, cur.q[k], cur.b[k], cur.a[k], nxt.q[k],
                        nxt.b[k], nxt.a[k], oL, oR);
        add_yface(A[k], oL);
        B[k] = cell_from_yface(oR);
      }
    }
    // row j: lambda^{n+1} + value adjoints + D_x^T + the push from row j-1
    T o[3][2];
    {
      const T lEx = __shfl_up_sync(AFULL, A[1].dEx, 1), rEx = __shfl_down_sync(AFULL, A[0].dEx, 1);
      const T lAx = __shfl_up_sync(AFULL, A[1].dAx, 1), rAx = __shfl_down_sync(AFULL, A[0].dAx, 1);
      const T lBx = __shfl_up_sync(AFULL, A[1].dBx, 1), rBx = __shfl_down_sync(AFULL, A[0].dBx, 1);
      o[0][0] = cur.e[0] + A[0].vE + carry[0][0] + (cl[0] * lEx - cr[0] * A[1].dEx + cs[0] * A[0].dEx);
      o[1][0] = cur.a[0] + A[0].vA + carry[1][0] + (cl[0] * lAx - cr[0] * A[1].dAx + cs[0] * A[0].dAx);
      o[2][0] = cur.b[0] + A[0].vB + carry[2][0] + (cl[0] * lBx - cr[0] * A[1].dBx + cs[0] * A[0].dBx);
      o[0][1] = cur.e[1] + A[1].vE + carry[0][1] + (cl[1] * A[0].dEx - cr[1] * rEx + cs[1] * A[1].dEx);
      o[1][1] = cur.a[1] + A[1].vA + carry[1][1] + (cl[1] * A[0].dAx - cr[1] * rAx + cs[1] * A[1].dAx);
      o[2][1] = cur.b[1] + A[1].vB + carry[2][1] + (cl[1] * A[0].dBx - cr[1] * rBx + cs[1] * A[1].dBx);
    }
    // y-difference adjoints of row j: -> row j-1 (-), row j+1 (+), ends (clamped ghosts)
    {
      const bool has = p.pery || (j >= 0 && j < p.ny);
      const T z = T(0);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const T dy[3] = {A[k].dEy, A[k].dAy, A[k].dBy};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const T d = has ? dy[c] : z;
          pend[c][k] -= d;
          carry[c][k] = d;
          if (!p.pery) {
            if (j == p.ny - 1) o[c][k] += d;
            if (j == 0) o[c][k] -= d;
          }
        }
      }
    }
    // row j-1 is complete
    const int jo = j - 1;
    if (jo >= y0 && jo < y1) {
      const int64_t ro = (int64_t)jo * p.pitch;
      const bool ok0 = X >= x0 && X < xend, ok1 = X + 1 >= x0 && X + 1 < xend;
      using P = typename APair<T>::type;
      if (ok0 && ok1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          P v;
          v.x = pend[c][0]; v.y = pend[c][1];
          *reinterpret_cast<P *>(p.lout + c * p.cstride + ro + X) = v;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 2; ++k)
          if (k == 0 ? ok0 : ok1)
#pragma unroll
            for (int c = 0; c < 3; ++c) p.lout[c * p.cstride + ro + X + k] = pend[c][k];
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) { pend[c][0] = o[c][0]; pend[c][1] = o[c][1]; }
    A[0] = B[0]; A[1] = B[1];
    cur = nxt; nxt = pf; pf = pf2;
    finish_arow(nxt);
  }
}

// ------------------------------------------------------------------ probe term and eps-gradient
// After the march, over the box covering the design cells and the probe (32 x 8 tiles, one
// thread per cell):
//  * lambda^n += dq/dV^n = 2 dt |Omega| Ez^n on the probe;
//  * dJ/deps_d += -lambda_E (E^{n+1} - E^n)/eps_d - sum over the cell's faces of
//    mu_f . dF_f/deps_d, mu_f = lambda_L/M_L - lambda_R/M_R (lambda = lambda^{n+1}, V = V^n),
//    with lambda^{n+1}, eps and V^n staged with a two-cell halo.
constexpr int GX = 32, GY = 8;
constexpr int GSX = GX + 4, GSY = GY + 4;

template <typename T>
struct GradSmem {
  T lam[3][GSY][GSX];
  T eps[GSY][GSX];
  T vn[3][GSY][GSX];
};

// Staged raw differences of a cell (sx, sy in the staged region) from V^n.
template <typename T>
__device__ __forceinline__ void staged_diffs(const GradSmem<T> &s, int sx, int sy, T d[6]) {
  d[0] = s.vn[0][sy][sx + 1] - s.vn[0][sy][sx - 1];   // dEx
  d[1] = s.vn[0][sy + 1][sx] - s.vn[0][sy - 1][sx];   // dEy
  d[2] = s.vn[1][sy][sx + 1] - s.vn[1][sy][sx - 1];   // dAx
  d[3] = s.vn[1][sy + 1][sx] - s.vn[1][sy - 1][sx];   // dAy
  d[4] = s.vn[2][sy][sx + 1] - s.vn[2][sy][sx - 1];   // dBx
  d[5] = s.vn[2][sy + 1][sx] - s.vn[2][sy - 1][sx];   // dBy
}

template <typename T>
__device__ __forceinline__ FIn<T> xin(const GradSmem<T> &s, int sx, int sy) {
  T d[6];
  staged_diffs(s, sx, sy, d);
  FIn<T> f;
  f.v[0] = s.vn[0][sy][sx]; f.v[1] = s.vn[1][sy][sx]; f.v[2] = s.vn[2][sy][sx];
  f.d[0] = d[0]; f.d[1] = d[2]; f.d[2] = d[4]; f.d[3] = d[3]; f.d[4] = d[1];
  f.eps = s.eps[sy][sx];
  return f;
}

template <typename T>
__device__ __forceinline__ FIn<T> yin(const GradSmem<T> &s, int sx, int sy) {
  T d[6];
  staged_diffs(s, sx, sy, d);
  FIn<T> f;
  f.v[0] = s.vn[0][sy][sx]; f.v[1] = s.vn[2][sy][sx]; f.v[2] = s.vn[1][sy][sx];
  f.d[0] = d[1]; f.d[1] = d[5]; f.d[2] = d[3]; f.d[3] = d[4]; f.d[4] = d[0];
  f.eps = s.eps[sy][sx];
  return f;
}

template <typename T>
__global__ void __launch_bounds__(GX * GY) adjoint_post_kernel(const AdjArgs<T> p, int bx0, int by0) {
  __shared__ GradSmem<T> s;
  const int tid = threadIdx.x;
  const int x0 = bx0 + blockIdx.x * GX, y0 = by0 + blockIdx.y * GY;
  const int tx = tid % GX, ty = tid / GX;
  const int gx = x0 + tx, gy = y0 + ty;
  const int64_t o = (int64_t)gy * p.pitch + gx;
  if (p.pw && gx >= p.px0 && gx < p.px1 && gy >= p.py0 && gy < p.py1) {
    const double w = p.pw[(int64_t)(gy - p.py0) * (p.px1 - p.px0) + (gx - p.px0)];
    p.lout[o] += T(p.dt2 * w) * p.Vn[o];
  }
  if (!p.grad) return;                                  // uniform over the launch
  // the cell's own loads go out before the staging so that their latencies overlap
  const bool in_box = gx >= p.dx0 && gx < p.dx1 && gy >= p.dy0 && gy < p.dy1;
  const int slot = in_box ? p.dslot[o] : -1;
  const T en1 = slot >= 0 ? p.Vn1[o] : T(0);
  const double g_old = slot >= 0 ? p.grad[slot] : 0.0;
#pragma unroll
  for (int i = tid; i < GSX * GSY; i += GX * GY) {
    const int sy = i / GSX, sx = i - sy * GSX;
    const int gx = wc(x0 - 2 + sx, p.nx, p.perx), gy = wc(y0 - 2 + sy, p.ny, p.pery);
    const int64_t o = (int64_t)gy * p.pitch + gx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s.lam[c][sy][sx] = p.lam[c * p.cstride + o];
      s.vn[c][sy][sx] = p.Vn[c * p.cstride + o];
    }
    s.eps[sy][sx] = p.eps[o];
  }
  __syncthreads();
  if (slot < 0) return;
  const int sx = tx + 2, sy = ty + 2;
  const T ed = s.eps[sy][sx];
  // the step's contribution in the path's precision; the sum over steps is FP64 (grad)
  T gs = -fdv(s.lam[0][sy][sx] * (en1 - s.vn[0][sy][sx]), ed);
  // faces: left x (cell = R), right x (cell = L), bottom y (R), top y (L)
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const bool isx = f < 2;
    const int lsx = isx ? (f == 0 ? sx - 1 : sx) : sx, lsy = isx ? sy : (f == 2 ? sy - 1 : sy);
    const int rsx = isx ? lsx + 1 : sx, rsy = isx ? sy : lsy + 1;
    const int glo = isx ? gx - 1 + (f == 0 ? 0 : 1) : gy - 1 + (f == 2 ? 0 : 1);
    const int kind = isx ? face_kind(glo, p.nx, p.perx) : face_kind(glo, p.ny, p.pery);
    if (kind == 3) continue;
    const FIn<T> L = isx ? xin(s, lsx, lsy) : yin(s, lsx, lsy);
    const FIn<T> R = isx ? xin(s, rsx, rsy) : yin(s, rsx, rsy);
    const FaceK<T> &k = isx ? p.fx : p.fy;
    T dl[3], dr[3];
    if (kind == 0) face_deps<T, 0>(L, R, k, dl, dr);
    else if (kind == 1) face_deps<T, 1>(L, R, k, dl, dr);
    else face_deps<T, 2>(L, R, k, dl, dr);
    const bool is_low = (f == 1 || f == 3);            // the cell is the face's L side
    const T *dd = is_low ? dl : dr;
    // mu_f = lambda_L/M_L - lambda_R/M_R in the face's (Ez, Hn, Ht) order
    const int hn = isx ? 1 : 2, ht = isx ? 2 : 1;
    T mu[3] = {T(0), T(0), T(0)};
    if (kind != 1) { mu[0] += fdv(s.lam[0][lsy][lsx], L.eps); mu[1] += s.lam[hn][lsy][lsx]; mu[2] += s.lam[ht][lsy][lsx]; }
    if (kind != 2) { mu[0] -= fdv(s.lam[0][rsy][rsx], R.eps); mu[1] -= s.lam[hn][rsy][rsx]; mu[2] -= s.lam[ht][rsy][rsx]; }
    gs -= mu[0] * dd[0] + mu[1] * dd[1] + mu[2] * dd[2];
  }
  p.grad[slot] = g_old + double(gs);
}

// dq/dV for q(V) = dt sum_P |Omega| Ez^2: lam_E[probe] (+)= 2 dt |Omega| Ez.
template <typename T>
__global__ void probe_grad_kernel(const T *__restrict__ V, T *__restrict__ lam,
                                  const int64_t *__restrict__ off, const double *__restrict__ w,
                                  int64_t np, double dt, int assign) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= np) return;
  const int64_t o = off[i];
  const T v = T(2.0 * dt * w[i]) * V[o];
  lam[o] = assign ? v : lam[o] + v;
}

// q(V) = dt sum_P |Omega| Ez^2, deterministic: block b sums its contiguous slice of the probe
// list in a fixed tree order into part[b]; the last block to finish (ticket) adds the partials
// in index order and folds dt * sum into the Kahan-compensated running sum acc = (sum, comp).
constexpr int OBJ_T = 256;

template <typename T>
__global__ void __launch_bounds__(OBJ_T) objective_kernel(const T *__restrict__ V,
                                                          const int64_t *__restrict__ off,
                                                          const double *__restrict__ w, int64_t np,
                                                          double dt, double *__restrict__ acc) {
  __shared__ double red[OBJ_T];
  __shared__ int last;
  double *part = acc + 2;
  unsigned *ticket = reinterpret_cast<unsigned *>(acc + 2 + kObjParts);
  const int64_t per = (np + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = min(np, lo + per);
  double a = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += OBJ_T) {
    const double e = double(V[off[i]]);
    a += w[i] * e * e;
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = OBJ_T / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // one warp: lane l adds partials l, l+32 (in that order), then a fixed shuffle tree
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) v += __ldcg(part + b);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) {
    const double term = dt * v;
    const double y = term - acc[1];
    const double t = acc[0] + y;
    acc[1] = (t - acc[0]) - y;
    acc[0] = t;
    *ticket = 0u;
  }
}

template <typename T>
cudaError_t adjoint_t(const CartGeom &g, const AdjointArgs &a, cudaStream_t st) {
  AdjArgs<T> p;
  p.lam = static_cast<const T *>(a.lam_in);
  p.lout = static_cast<T *>(a.lam_out);
  p.eps = static_cast<const T *>(a.eps);
  p.Vn = static_cast<const T *>(a.Vn);
  p.Vn1 = static_cast<const T *>(a.Vn1);
  p.dslot = a.dslot;
  p.grad = a.grad;
  p.pw = a.probe_w;
  p.px0 = a.pbox[0]; p.px1 = a.pbox[1]; p.py0 = a.pbox[2]; p.py1 = a.pbox[3];
  p.dt2 = 2.0 * a.dt;
  p.dx0 = a.dbox[0]; p.dx1 = a.dbox[1]; p.dy0 = a.dbox[2]; p.dy1 = a.dbox[3];
  p.nx = g.nx; p.ny = g.ny;
  p.pitch = g.pitch; p.cstride = g.cstride;
  p.perx = g.periodic[0]; p.pery = g.periodic[1];
  p.fx = make_face_k<T>(a.C, g.h[0], g.h[1], a.c, 1.0, 1.0);
  p.fy = make_face_k<T>(a.C, g.h[1], g.h[0], a.c, -1.0, -1.0);
  // strips of 60 columns; rows per warp chosen so that the warps fit in one wave
  static int resident = 0;   // warps of this kernel resident on the GPU at once
  if (!resident) {
    int dev = 0, sms = 0, bps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, adjoint_lambda_kernel<T>, AWARPS * 32, 0);
    resident = sms * (bps > 0 ? bps : 1) * AWARPS;
  }
  const int nstrips = (g.nx + AWCOLS - 1) / AWCOLS;
  int rows = g.ny;
  const int target = resident;
  if (nstrips < target) {
    const int chunks = (target + nstrips - 1) / nstrips;
    rows = (g.ny + chunks - 1) / chunks;
  }
  rows = rows < 16 ? 16 : (rows > 256 ? 256 : rows);
  const int nchunks = (g.ny + rows - 1) / rows;
  const int64_t nwarps = (int64_t)nstrips * nchunks;
  const int grid = (int)((nwarps + AWARPS - 1) / AWARPS);
  adjoint_lambda_kernel<T><<<grid, AWARPS * 32, 0, st>>>(p, nstrips, rows);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // probe term and eps-gradient over the bounding box of the probe and the design cells
  if (p.grad && (p.dx1 <= p.dx0 || p.dy1 <= p.dy0)) p.grad = nullptr;
  if (!p.grad && !p.pw) return cudaSuccess;
  int b[4] = {g.nx, 0, g.ny, 0};
  if (p.grad) { b[0] = p.dx0; b[1] = p.dx1; b[2] = p.dy0; b[3] = p.dy1; }
  if (p.pw) {
    b[0] = std::min(b[0], p.px0); b[1] = std::max(b[1], p.px1);
    b[2] = std::min(b[2], p.py0); b[3] = std::max(b[3], p.py1);
  }
  dim3 gg((b[1] - b[0] + GX - 1) / GX, (b[3] - b[2] + GY - 1) / GY);
  adjoint_post_kernel<T><<<gg, GX * GY, 0, st>>>(p, b[0], b[2]);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_step(const CartGeom &g, const AdjointArgs &a, bool fp64,
                                cudaStream_t st) {
  return fp64 ? adjoint_t<double>(g, a, st) : adjoint_t<float>(g, a, st);
}

cudaError_t launch_probe_grad(const void *V, void *lam, const int64_t *off, const double *w,
                              int64_t np, double dt, bool assign, bool fp64, cudaStream_t st) {
  const int b = (int)((np + 255) / 256);
  if (np <= 0) return cudaSuccess;
  if (fp64)
    probe_grad_kernel<double><<<b, 256, 0, st>>>(static_cast<const double *>(V),
                                                 static_cast<double *>(lam), off, w, np, dt,
                                                 assign ? 1 : 0);
  else
    probe_grad_kernel<float><<<b, 256, 0, st>>>(static_cast<const float *>(V),
                                                static_cast<float *>(lam), off, w, np, dt,
                                                assign ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_objective(const void *V, const int64_t *off, const double *w, int64_t np,
                             double dt, double *acc, bool fp64, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(kObjParts, (np + OBJ_T - 1) / OBJ_T);
  if (fp64)
    objective_kernel<double><<<blocks, OBJ_T, 0, st>>>(static_cast<const double *>(V), off, w, np,
                                                       dt, acc);
  else
    objective_kernel<float><<<blocks, OBJ_T, 0, st>>>(static_cast<const float *>(V), off, w, np,
                                                      dt, acc);
  return cudaGetLastError();
}

}  // namespace gks
