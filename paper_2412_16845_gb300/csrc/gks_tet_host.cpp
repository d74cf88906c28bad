// Host-side geometry of a conforming tetrahedral mesh (FP64): face matching, normals, areas,
// centroids, volumes, face frames T'(n) (Sec. 3.1), per-cell face tables and a Morton
// ordering of the cells for locality.  Everything here runs once per mesh.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "gks_internal.h"

namespace gks {
namespace {

struct FaceKey {
  int64_t a, b, c;   // sorted vertex ids
  int64_t owner;     // user tet id
  int opp;           // local index of the opposite vertex
  bool operator<(const FaceKey &o) const {
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    if (c != o.c) return c < o.c;
    return owner < o.owner;
  }
  bool same(const FaceKey &o) const { return a == o.a && b == o.b && c == o.c; }
};

inline void sub3(const double *p, const double *q, double *r) {
  r[0] = p[0] - q[0]; r[1] = p[1] - q[1]; r[2] = p[2] - q[2];
}
inline void cross3(const double *u, const double *v, double *r) {
  r[0] = u[1] * v[2] - u[2] * v[1];
  r[1] = u[2] * v[0] - u[0] * v[2];
  r[2] = u[0] * v[1] - u[1] * v[0];
}
inline double dot3(const double *u, const double *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; }

// Spread the low 21 bits of x to every third bit (Morton interleave).
inline uint64_t spread3(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | (x << 32)) & 0x1f00000000ffffULL;
  x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
  x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
  x = (x | (x << 2)) & 0x1249249249249249ULL;
  return x;
}

}  // namespace

// The face frame of Sec. 3.1: rows (n, t, w) with
//   t = (-n2, n1 + n3^2/(1+n1), -n2 n3/(1+n1)),  w = (-n3, -n2 n3/(1+n1), 1 - n3^2/(1+n1)),
// and diag(-1, -1, 1) for n1 = -1.  For n1 < 0, 1 + n1 is formed as (n2^2 + n3^2)/(1 - n1),
// equal for unit n and free of cancellation near n1 = -1.
void face_frame(const double n[3], double T[9]) {
  const double n1 = n[0], n2 = n[1], n3 = n[2];
  if (n1 == -1.0) {
    const double d[9] = {-1, 0, 0, 0, -1, 0, 0, 0, 1};
    for (int k = 0; k < 9; ++k) T[k] = d[k];
    return;
  }
  const double inv = frame_inv_one_plus(n1, n2, n3);
  T[0] = n1; T[1] = n2; T[2] = n3;
  T[3] = -n2; T[4] = n1 + n3 * n3 * inv; T[5] = -n2 * n3 * inv;
  T[6] = -n3; T[7] = -n2 * n3 * inv; T[8] = 1.0 - n3 * n3 * inv;
}

gks_status build_tet_geometry(const double *vert, int64_t nv, const int64_t *tet, int64_t nt,
                              TetHost &g, std::string &err) {
  if (nv < 4 || nt < 1) { err = "a tet mesh needs at least 4 vertices and 1 tet"; return GKS_E_ARG; }
  if (nt > (int64_t)1 << 30) { err = "too many tets"; return GKS_E_ARG; }
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(vert[i])) { err = "non-finite vertex coordinate"; return GKS_E_ARG; }
  for (int64_t i = 0; i < 4 * nt; ++i)
    if (tet[i] < 0 || tet[i] >= nv) { err = "tet vertex id out of range"; return GKS_E_ARG; }
  g.nt = nt;
  // user-order volumes and centroids
  std::vector<double> vol_u(nt), cen_u(3 * nt);
  for (int64_t t = 0; t < nt; ++t) {
    const double *p[4];
    for (int k = 0; k < 4; ++k) p[k] = vert + 3 * tet[4 * t + k];
    double e1[3], e2[3], e3[3], cr[3];
    sub3(p[1], p[0], e1); sub3(p[2], p[0], e2); sub3(p[3], p[0], e3);
    cross3(e1, e2, cr);
    const double v = std::fabs(dot3(cr, e3)) / 6.0;
    if (!(v > 0.0)) { err = "degenerate tet " + std::to_string(t); return GKS_E_ARG; }
    vol_u[t] = v;
    for (int a = 0; a < 3; ++a) cen_u[3 * t + a] = 0.25 * (p[0][a] + p[1][a] + p[2][a] + p[3][a]);
  }
  // Morton order of the cell centroids (internal order k -> user id perm[k])
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t t = 0; t < nt; ++t)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], cen_u[3 * t + a]);
      hi[a] = std::max(hi[a], cen_u[3 * t + a]);
    }
  std::vector<std::pair<uint64_t, int64_t>> code(nt);
  for (int64_t t = 0; t < nt; ++t) {
    uint64_t m = 0;
    for (int a = 0; a < 3; ++a) {
      const double span = hi[a] > lo[a] ? hi[a] - lo[a] : 1.0;
      const uint64_t q = (uint64_t)std::min(2097151.0, std::floor((cen_u[3 * t + a] - lo[a]) / span * 2097151.0));
      m |= spread3(q) << a;
    }
    code[t] = {m, t};
  }
  std::sort(code.begin(), code.end());
  g.perm.resize(nt);
  g.iperm.resize(nt);
  for (int64_t k = 0; k < nt; ++k) {
    g.perm[k] = code[k].second;
    g.iperm[code[k].second] = k;
  }
  // faces: sorted vertex triples of the 4 faces of every tet, matched by sorting
  static const int opp_face[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  std::vector<FaceKey> keys(4 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int f = 0; f < 4; ++f) {
      int64_t v[3] = {tet[4 * t + opp_face[f][0]], tet[4 * t + opp_face[f][1]],
                      tet[4 * t + opp_face[f][2]]};
      std::sort(v, v + 3);
      keys[4 * t + f] = {v[0], v[1], v[2], t, f};
    }
  std::sort(keys.begin(), keys.end());
  struct Face { int64_t L, R; int64_t a, b, c; };
  std::vector<Face> faces;
  faces.reserve(2 * nt + 16);
  for (size_t i = 0; i < keys.size();) {
    if (i + 1 < keys.size() && keys[i].same(keys[i + 1])) {
      if (i + 2 < keys.size() && keys[i].same(keys[i + 2])) {
        err = "a face is shared by more than two tets";
        return GKS_E_ARG;
      }
      faces.push_back({keys[i].owner, keys[i + 1].owner, keys[i].a, keys[i].b, keys[i].c});
      i += 2;
    } else {
      faces.push_back({keys[i].owner, -1, keys[i].a, keys[i].b, keys[i].c});
      i += 1;
    }
  }
  // face order: by the smaller internal index of the two cells (locality of the face pass)
  std::sort(faces.begin(), faces.end(), [&](const Face &p, const Face &q) {
    const int64_t mp = p.R < 0 ? g.iperm[p.L] : std::min(g.iperm[p.L], g.iperm[p.R]);
    const int64_t mq = q.R < 0 ? g.iperm[q.L] : std::min(g.iperm[q.L], g.iperm[q.R]);
    return mp != mq ? mp < mq : (p.a != q.a ? p.a < q.a : (p.b != q.b ? p.b < q.b : p.c < q.c));
  });
  const int64_t nf = (int64_t)faces.size();
  g.nf = nf;
  g.fL.resize(nf); g.fR.resize(nf); g.farea.resize(nf);
  g.fT.assign(9 * nf, 0.0); g.fdL.assign(3 * nf, 0.0); g.fdR.assign(3 * nf, 0.0);
  g.cnb.assign(4 * nt, -1); g.cface.assign(4 * nt, -1); g.csign.assign(4 * nt, 0.0);
  g.cw.assign(12 * nt, 0.0);
  std::vector<int> fill(nt, 0);
  std::vector<double> perim(nt, 0.0);
  for (int64_t f = 0; f < nf; ++f) {
    const Face &F = faces[f];
    // interior faces point from the smaller to the larger user id; boundary faces outward
    const int64_t L = F.L, R = F.R;
    const double *pa = vert + 3 * F.a, *pb = vert + 3 * F.b, *pc = vert + 3 * F.c;
    double e1[3], e2[3], cr[3], xs[3];
    sub3(pb, pa, e1); sub3(pc, pa, e2); cross3(e1, e2, cr);
    const double nrm = std::sqrt(dot3(cr, cr));
    if (!(nrm > 0.0)) { err = "degenerate face"; return GKS_E_ARG; }
    double n[3] = {cr[0] / nrm, cr[1] / nrm, cr[2] / nrm};
    for (int a = 0; a < 3; ++a) xs[a] = (pa[a] + pb[a] + pc[a]) / 3.0;
    double dl[3];
    sub3(xs, &cen_u[3 * L], dl);
    if (dot3(n, dl) < 0.0) { n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; }
    const double area = 0.5 * nrm;
    const int64_t iL = g.iperm[L], iR = R >= 0 ? g.iperm[R] : -1;
    g.fL[f] = (int32_t)iL;
    g.fR[f] = (int32_t)iR;
    g.farea[f] = area;
    face_frame(n, &g.fT[9 * f]);
    for (int a = 0; a < 3; ++a) g.fdL[3 * f + a] = dl[a];
    if (R >= 0)
      for (int a = 0; a < 3; ++a) g.fdR[3 * f + a] = xs[a] - cen_u[3 * R + a];
    // per-cell tables (internal order): face id, side sign, neighbour, outward n |l| / |Omega|
    const int64_t cells[2] = {iL, iR};
    for (int side = 0; side < 2; ++side) {
      const int64_t ic = cells[side];
      if (ic < 0) continue;
      const int64_t user = side == 0 ? L : R;
      const int k = fill[ic]++;
      if (k >= 4) { err = "a tet has more than four faces"; return GKS_E_ARG; }
      const double sg = side == 0 ? 1.0 : -1.0;
      g.cface[4 * ic + k] = (int32_t)f;
      g.csign[4 * ic + k] = sg;
      g.cnb[4 * ic + k] = (int32_t)(side == 0 ? iR : iL);
      for (int a = 0; a < 3; ++a) g.cw[12 * ic + 3 * k + a] = sg * n[a] * area / vol_u[user];
      perim[ic] += area;
    }
  }
  for (int64_t k = 0; k < nt; ++k)
    if (fill[k] != 4) { err = "a tet does not have four faces"; return GKS_E_ARG; }
  g.vol.resize(nt);
  g.ivol.resize(nt);
  g.min_h = 1e300;
  for (int64_t k = 0; k < nt; ++k) {
    g.vol[k] = vol_u[g.perm[k]];
    g.ivol[k] = 1.0 / g.vol[k];
    g.min_h = std::min(g.min_h, 6.0 * g.vol[k] / perim[k]);
  }
  return GKS_OK;
}

}  // namespace gks
