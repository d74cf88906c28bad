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

#include "gks_flux2.cuh"
#include "gks_internal.h"

namespace gks {
namespace {

// Division: FP32 uses the fast hardware reciprocal (about 1 ulp), FP64 divides.
__device__ __forceinline__ float fdv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdv(double a, double b) { return a / b; }

constexpr int RX = 32, RY = 16;              // ring of threads: tile 30 x 14 plus one cell around
constexpr int TXI = RX - 2, TYI = RY - 2;    // inner (updated) cells
constexpr int SX = RX + 2, SY = RY + 2;      // staged region: two cells around the tile
constexpr int NXF = RX + 1, NYF = RY + 1;    // x-faces per ring row, y-faces per ring column

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
  const T *__restrict__ Vn;       // state at t^n (design tiles only)
  const T *__restrict__ Vn1;      // state at t^{n+1} (design cells only)
  const int32_t *__restrict__ dslot;   // design slot per cell or -1
  double *__restrict__ grad;      // [nd] += dJ/deps
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

template <typename T>
struct AdjSmem {
  T lam[3][SY][SX];
  T eps[SY][SX];
  T vn[3][SY][SX];
  T xf[2][8][RY][NXF];    // x-face adjoints: [side][v(3) d(5)][row][face]
  T yf[2][8][NYF][RX];    // y-face adjoints: [side][...][face][column]
  T db[6][RY][RX];        // raw-difference adjoints of ring cells: dEx dEy dAx dAy dBx dBy
};

// Face type relative to the domain: 0 interior, 1 ghost low, 2 ghost high, 3 outside.
__device__ __forceinline__ int face_kind(int lo_cell, int n, int periodic) {
  if (periodic) return 0;
  const int hi_cell = lo_cell + 1;
  if (lo_cell >= 0 && hi_cell < n) return 0;
  if (lo_cell == -1 && hi_cell < n) return 1;
  if (lo_cell == n - 1) return 2;
  return 3;
}

// Staged raw differences of a cell (sx, sy in the staged region) from V^n.
template <typename T>
__device__ __forceinline__ void staged_diffs(const AdjSmem<T> &s, int sx, int sy, T d[6]) {
  d[0] = s.vn[0][sy][sx + 1] - s.vn[0][sy][sx - 1];   // dEx
  d[1] = s.vn[0][sy + 1][sx] - s.vn[0][sy - 1][sx];   // dEy
  d[2] = s.vn[1][sy][sx + 1] - s.vn[1][sy][sx - 1];   // dAx
  d[3] = s.vn[1][sy + 1][sx] - s.vn[1][sy - 1][sx];   // dAy
  d[4] = s.vn[2][sy][sx + 1] - s.vn[2][sy][sx - 1];   // dBx
  d[5] = s.vn[2][sy + 1][sx] - s.vn[2][sy - 1][sx];   // dBy
}

template <typename T>
__device__ __forceinline__ FIn<T> xin(const AdjSmem<T> &s, int sx, int sy) {
  T d[6];
  staged_diffs(s, sx, sy, d);
  FIn<T> f;
  f.v[0] = s.vn[0][sy][sx]; f.v[1] = s.vn[1][sy][sx]; f.v[2] = s.vn[2][sy][sx];
  f.d[0] = d[0]; f.d[1] = d[2]; f.d[2] = d[4]; f.d[3] = d[3]; f.d[4] = d[1];
  f.eps = s.eps[sy][sx];
  return f;
}

template <typename T>
__device__ __forceinline__ FIn<T> yin(const AdjSmem<T> &s, int sx, int sy) {
  T d[6];
  staged_diffs(s, sx, sy, d);
  FIn<T> f;
  f.v[0] = s.vn[0][sy][sx]; f.v[1] = s.vn[2][sy][sx]; f.v[2] = s.vn[1][sy][sx];
  f.d[0] = d[1]; f.d[1] = d[5]; f.d[2] = d[3]; f.d[3] = d[4]; f.d[4] = d[0];
  f.eps = s.eps[sy][sx];
  return f;
}

template <typename T>
__global__ void __launch_bounds__(RX * RY) adjoint_step_kernel(const AdjArgs<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  AdjSmem<T> &s = *reinterpret_cast<AdjSmem<T> *>(smem_raw);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TXI, y0 = blockIdx.y * TYI;
  const bool design_tile = p.grad && x0 - 2 < p.dx1 && x0 + TXI + 2 > p.dx0 &&
                           y0 - 2 < p.dy1 && y0 + TYI + 2 > p.dy0;
  // 1. stage lambda^{n+1}, eps (and V^n on design tiles) with a two-cell halo
  for (int i = tid; i < SX * SY; i += RX * RY) {
    const int sy = i / SX, sx = i - sy * SX;
    const int gx = wc(x0 - 2 + sx, p.nx, p.perx), gy = wc(y0 - 2 + sy, p.ny, p.pery);
    const int64_t o = (int64_t)gy * p.pitch + gx;
#pragma unroll
    for (int c = 0; c < 3; ++c) s.lam[c][sy][sx] = p.lam[c * p.cstride + o];
    s.eps[sy][sx] = p.eps[o];
    if (design_tile)
#pragma unroll
      for (int c = 0; c < 3; ++c) s.vn[c][sy][sx] = p.Vn[c * p.cstride + o];
  }
  __syncthreads();
  // 2. face adjoints.  x-face k of ring row ry lies between staged columns k and k+1.
  for (int i = tid; i < RY * NXF; i += RX * RY) {
    const int ry = i / NXF, k = i - ry * NXF;
    const int sy = ry + 1, sxl = k, sxr = k + 1;
    const int gy = y0 - 1 + ry, glo = x0 - 2 + k;
    const int kind = (gy >= 0 && gy < p.ny) || p.pery ? face_kind(glo, p.nx, p.perx) : 3;
    FOut<T> oL = {}, oR = {};
    if (kind != 3) {
      const T el = s.eps[sy][sxl], er = s.eps[sy][sxr];
      // Fbar = -(lambda_L / M_L - lambda_R / M_R), components (Ez, Hx, Hy)
      T mu[3] = {T(0), T(0), T(0)};
      if (kind != 1) { mu[0] += fdv(s.lam[0][sy][sxl], el); mu[1] += s.lam[1][sy][sxl]; mu[2] += s.lam[2][sy][sxl]; }
      if (kind != 2) { mu[0] -= fdv(s.lam[0][sy][sxr], er); mu[1] -= s.lam[1][sy][sxr]; mu[2] -= s.lam[2][sy][sxr]; }
      if (kind == 0) face_adj<T, 0>(el, er, p.fx, -mu[0], -mu[1], -mu[2], oL, oR);
      else if (kind == 1) face_adj<T, 1>(el, er, p.fx, -mu[0], -mu[1], -mu[2], oL, oR);
      else face_adj<T, 2>(el, er, p.fx, -mu[0], -mu[1], -mu[2], oL, oR);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) { s.xf[0][c][ry][k] = oL.v[c]; s.xf[1][c][ry][k] = oR.v[c]; }
#pragma unroll
    for (int c = 0; c < 5; ++c) { s.xf[0][3 + c][ry][k] = oL.d[c]; s.xf[1][3 + c][ry][k] = oR.d[c]; }
  }
  // y-face k of ring column rx lies between staged rows k and k+1; components (Ez, Hy, Hx)
  for (int i = tid; i < NYF * RX; i += RX * RY) {
    const int k = i / RX, rx = i - k * RX;
    const int sx = rx + 1, syl = k, syr = k + 1;
    const int gx = x0 - 1 + rx, glo = y0 - 2 + k;
    const int kind = (gx >= 0 && gx < p.nx) || p.perx ? face_kind(glo, p.ny, p.pery) : 3;
    FOut<T> oL = {}, oR = {};
    if (kind != 3) {
      const T el = s.eps[syl][sx], er = s.eps[syr][sx];
      T mu[3] = {T(0), T(0), T(0)};
      if (kind != 1) { mu[0] += fdv(s.lam[0][syl][sx], el); mu[1] += s.lam[2][syl][sx]; mu[2] += s.lam[1][syl][sx]; }
      if (kind != 2) { mu[0] -= fdv(s.lam[0][syr][sx], er); mu[1] -= s.lam[2][syr][sx]; mu[2] -= s.lam[1][syr][sx]; }
      if (kind == 0) face_adj<T, 0>(el, er, p.fy, -mu[0], -mu[1], -mu[2], oL, oR);
      else if (kind == 1) face_adj<T, 1>(el, er, p.fy, -mu[0], -mu[1], -mu[2], oL, oR);
      else face_adj<T, 2>(el, er, p.fy, -mu[0], -mu[1], -mu[2], oL, oR);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) { s.yf[0][c][k][rx] = oL.v[c]; s.yf[1][c][k][rx] = oR.v[c]; }
#pragma unroll
    for (int c = 0; c < 5; ++c) { s.yf[0][3 + c][k][rx] = oL.d[c]; s.yf[1][3 + c][k][rx] = oR.d[c]; }
  }
  __syncthreads();
  // 3. gather per ring cell: value adjoints (registers) and difference adjoints (shared)
  const int rx = tid % RX, ry = tid / RX;
  T vb[3];        // (Ez, Hx, Hy)
  {
    // cell is the R side of its left / bottom face and the L side of its right / top face
#define XL(c) s.xf[1][c][ry][rx]
#define XR(c) s.xf[0][c][ry][rx + 1]
#define YB(c) s.yf[1][c][ry][rx]
#define YT(c) s.yf[0][c][ry + 1][rx]
    vb[0] = XL(0) + XR(0) + YB(0) + YT(0);
    vb[1] = XL(1) + XR(1) + YB(2) + YT(2);
    vb[2] = XL(2) + XR(2) + YB(1) + YT(1);
    // x-face d order: (dEx, dAx, dBx, dAy, dEy); y-face: (dEy, dBy, dAy, dBx, dEx)
    s.db[0][ry][rx] = XL(3) + XR(3) + YB(7) + YT(7);   // dEx
    s.db[1][ry][rx] = XL(7) + XR(7) + YB(3) + YT(3);   // dEy
    s.db[2][ry][rx] = XL(4) + XR(4);                   // dAx
    s.db[3][ry][rx] = XL(6) + XR(6) + YB(5) + YT(5);   // dAy
    s.db[4][ry][rx] = XL(5) + XR(5) + YB(6) + YT(6);   // dBx
    s.db[5][ry][rx] = YB(4) + YT(4);                   // dBy
#undef XL
#undef XR
#undef YB
#undef YT
  }
  __syncthreads();
  // 4. inner cells: lambda^n = lambda^{n+1} + value adjoints + D^T(difference adjoints)
  if (rx >= 1 && rx <= RX - 2 && ry >= 1 && ry <= RY - 2) {
    const int gx = x0 - 1 + rx, gy = y0 - 1 + ry;
    if (gx < p.nx && gy < p.ny) {
      const int sx = rx + 1, sy = ry + 1;
      T out[3];
      const int cx[3] = {0, 2, 4}, cy[3] = {1, 3, 5};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T a = s.lam[c][sy][sx] + vb[c];
        // x: d_j = V(clamp/wrap j+1) - V(clamp/wrap j-1)
        if (p.perx) {
          a += s.db[cx[c]][ry][rx - 1] - s.db[cx[c]][ry][rx + 1];
        } else {
          if (gx - 1 >= 0) a += s.db[cx[c]][ry][rx - 1];
          if (gx + 1 < p.nx) a -= s.db[cx[c]][ry][rx + 1];
          if (gx == p.nx - 1) a += s.db[cx[c]][ry][rx];
          if (gx == 0) a -= s.db[cx[c]][ry][rx];
        }
        if (p.pery) {
          a += s.db[cy[c]][ry - 1][rx] - s.db[cy[c]][ry + 1][rx];
        } else {
          if (gy - 1 >= 0) a += s.db[cy[c]][ry - 1][rx];
          if (gy + 1 < p.ny) a -= s.db[cy[c]][ry + 1][rx];
          if (gy == p.ny - 1) a += s.db[cy[c]][ry][rx];
          if (gy == 0) a -= s.db[cy[c]][ry][rx];
        }
        out[c] = a;
      }
      const int64_t o = (int64_t)gy * p.pitch + gx;
#pragma unroll
      for (int c = 0; c < 3; ++c) p.lout[c * p.cstride + o] = out[c];
      // 5. eps-gradient of a design cell
      if (design_tile && gx >= p.dx0 && gx < p.dx1 && gy >= p.dy0 && gy < p.dy1) {
        const int slot = p.dslot[o];
        if (slot >= 0) {
          const T ed = s.eps[sy][sx];
          double gsum = -double(s.lam[0][sy][sx]) *
                        double(p.Vn1[o] - s.vn[0][sy][sx]) / double(ed);
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
            gsum -= double(mu[0] * dd[0] + mu[1] * dd[1] + mu[2] * dd[2]);
          }
          p.grad[slot] += gsum;
        }
      }
    }
  }
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

// q(V) = dt sum_P |Omega| Ez^2: one block, fixed order (deterministic); the running sum over
// steps is Kahan-compensated in acc = (sum, comp).  1024 threads keep the single block short.
template <typename T>
__global__ void objective_kernel(const T *__restrict__ V, const int64_t *__restrict__ off,
                                 const double *__restrict__ w, int64_t np, double dt,
                                 double *__restrict__ acc) {
  __shared__ double red[1024];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < np; i += blockDim.x) {
    const double e = double(V[off[i]]);
    a += w[i] * e * e;
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double term = dt * red[0];
    const double y = term - acc[1];
    const double t = acc[0] + y;
    acc[1] = (t - acc[0]) - y;
    acc[0] = t;
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
  p.dx0 = a.dbox[0]; p.dx1 = a.dbox[1]; p.dy0 = a.dbox[2]; p.dy1 = a.dbox[3];
  p.nx = g.nx; p.ny = g.ny;
  p.pitch = g.pitch; p.cstride = g.cstride;
  p.perx = g.periodic[0]; p.pery = g.periodic[1];
  p.fx = make_face_k<T>(a.C, g.h[0], g.h[1], a.c, 1.0, 1.0);
  p.fy = make_face_k<T>(a.C, g.h[1], g.h[0], a.c, -1.0, -1.0);
  const int smem = (int)sizeof(AdjSmem<T>);
  cudaFuncSetAttribute(adjoint_step_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  dim3 grid((g.nx + TXI - 1) / TXI, (g.ny + TYI - 1) / TYI);
  adjoint_step_kernel<T><<<grid, RX * RY, smem, st>>>(p);
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
  if (fp64)
    objective_kernel<double><<<1, 1024, 0, st>>>(static_cast<const double *>(V), off, w, np, dt, acc);
  else
    objective_kernel<float><<<1, 1024, 0, st>>>(static_cast<const float *>(V), off, w, np, dt, acc);
  return cudaGetLastError();
}

}  // namespace gks
