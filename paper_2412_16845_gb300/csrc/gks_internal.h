// Internal declarations shared by the host API (gks_api.cpp) and the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gks.h"

namespace gks {

// Time-integration coefficients C1..C5 of the GKS flux (Sec. 3.1) for step dt and relaxation
// time tau (tau = 0: the tau -> 0 limit of Sec. 4.1).
void time_coefficients(double dt, double tau, double C[5]);

// Cartesian grid geometry and state layout.  Fields are stored structure-of-arrays,
// [ncomp][nz][ny][pitch] with x fastest; pitch is nx rounded up to a multiple of 32 elements
// (128 B rows in FP32) so that every row starts 128-byte aligned.
struct CartGeom {
  int dim = 2;
  int nx = 1, ny = 1, nz = 1;
  int64_t pitch = 0;    // elements per row
  int64_t plane = 0;    // pitch * ny
  int64_t cstride = 0;  // elements per component: plane * nz
  double h[3] = {1, 1, 1};
  int periodic[3] = {0, 0, 0};
  int pec[6] = {0, 0, 0, 0, 0, 0};   // per side -x,+x,-y,+y,-z,+z: PEC wall (mirror ghost)
};

// Arguments of one Cartesian step launch (precision-independent; kernels cast).
struct CartStepArgs {
  const void *V;        // state at t^n
  void *Vout;           // state at t^{n+1}
  const void *eps;      // [nz][ny][pitch]
  const void *mu;       // same layout, or nullptr (mu = 1)
  const void *src;      // J_z mask, same layout, or nullptr
  int src_box[6];       // i0,i1,j0,j1,k0,k1 (half open) of the non-zero mask
  double src_amp;       // dt * waveform(t^n)
  double C[5];          // C1..C5
  double c;             // lattice speed
  int *flag;            // non-finite flag (device)
  int window[4];        // x0, x1, y0, y1 (half open) of the cells to advance (2-D)
  int limiter = 0;      // GKS_LIMITER_*: slopes of the cell gradients
};

// Tetrahedral mesh geometry on the host (FP64; cells in internal Morton order).
struct TetHost {
  int64_t nt = 0, nf = 0;
  std::vector<int64_t> perm;    // internal cell k -> user cell perm[k]
  std::vector<int64_t> iperm;   // user cell -> internal
  std::vector<double> vol;      // [nt] internal
  std::vector<double> ivol;     // [nt] 1 / vol
  std::vector<int32_t> cnb;     // [nt][4] neighbour (internal) or -1
  std::vector<int32_t> cface;   // [nt][4] face id
  std::vector<double> csign;    // [nt][4] +1 if the cell is the face's L side, -1 if R
  std::vector<double> cw;       // [nt][4][3] outward n |l| / |Omega|
  std::vector<int32_t> fL, fR;  // [nf] internal cells (R = -1 on the boundary)
  std::vector<double> fT;       // [nf][9] face frame rows (n, t, w)
  std::vector<double> farea;    // [nf]
  std::vector<double> fdL, fdR; // [nf][3] face centroid minus cell centroid
  double min_h = 0.0;           // min_i 6 |Omega_i| / sum_s |l_s|
};

gks_status build_tet_geometry(const double *vert, int64_t nv, const int64_t *tet, int64_t nt,
                              TetHost &g, std::string &err);
void face_frame(const double n[3], double T[9]);
// 1 / (1 + n_1) of the face frame, with 1 + n_1 formed as (n_2^2 + n_3^2) / (1 - n_1) for n_1 < 0
inline double frame_inv_one_plus(double n1, double n2, double n3) {
  return 1.0 / (n1 >= 0.0 ? 1.0 + n1 : (n2 * n2 + n3 * n3) / (1.0 - n1));
}

// Device copies of the tet geometry plus the per-step scratch (gradients, face fluxes).  The
// geometry is computed in FP64 on the host; the step kernels read it in the context's precision
// (rounded once on the host for FP32 contexts), packed per face and per cell.
constexpr int kTetFaceGeo = 10;   // per face: n 3, 1/(1+n_1) of the frame, x_s - x_L 3, x_s - x_R 3
constexpr int kTetCellW = 12;     // per cell, gradient pass: n |l| / |Omega| of its 4 faces
constexpr int kTetCellU = 4;      // per cell, update pass: sign_k |l_k| / |Omega| of its 4 faces
struct TetDev {
  int64_t nt = 0, nf = 0;
  int64_t *perm = nullptr;
  double *vol = nullptr;        // FP64 |Omega| (energy)
  int32_t *cnb = nullptr, *cface = nullptr;
  int32_t *fL = nullptr, *fR = nullptr;
  void *fgeo = nullptr;         // [nf][kTetFaceGeo], context precision
  void *cw = nullptr;           // [nt][kTetCellW], context precision
  void *cu = nullptr;           // [nt][kTetCellU], context precision
  void *Gscratch = nullptr;     // [18][nt] gradients
  void *Fscratch = nullptr;     // [6][nf] face fluxes (times dt and |l|)
  int pec = 0;                  // boundary faces are PEC walls (else non-reflecting)
};

cudaError_t launch_tet_step(const TetDev &g, const void *V, void *Vout, const void *eps,
                            const void *mu, const void *src, double src_amp, const double C[5],
                            double c, int *flag, bool fp64, cudaStream_t st);
cudaError_t launch_user_to_tet(const TetDev &g, int ncomp, const double *user, void *dst,
                               bool fp64, cudaStream_t st);
cudaError_t launch_tet_to_user(const TetDev &g, int ncomp, const void *src, double *user,
                               bool fp64, cudaStream_t st);
cudaError_t launch_tet_energy(const TetDev &g, const void *V, const void *eps, const void *mu,
                              bool fp64, double *partials, int npart, double *out,
                              cudaStream_t st);

// Adjoint of the 2-D TM step (see gks_adjoint.cu).
struct AdjointArgs {
  const void *lam_in;       // lambda^{n+1}, state layout
  void *lam_out;            // lambda^n
  const void *eps;
  const void *Vn;           // state at t^n
  const void *Vn1;          // state at t^{n+1}
  const int32_t *dslot;     // design slot per cell (-1 elsewhere), state layout
  double *grad;             // [nd], accumulated
  int dbox[4];              // design box x0, x1, y0, y1 (half open)
  const double *probe_w;    // probe weights |Omega_i| over the probe box (row-major), or null
  int pbox[4];              // probe box x0, x1, y0, y1 (half open)
  double dt;
  double C[5];
  double c;
};
cudaError_t launch_adjoint_step(const CartGeom &g, const AdjointArgs &a, bool fp64,
                                cudaStream_t st);
cudaError_t launch_probe_grad(const void *V, void *lam, const int64_t *off, const double *w,
                              int64_t np, double dt, bool assign, bool fp64, cudaStream_t st);
// The objective buffer: (sum, Kahan compensation), kObjParts per-block partials and a ticket.
constexpr int kObjParts = 64;
constexpr int kObjWords = 2 + kObjParts + 1;
cudaError_t launch_objective(const void *V, const int64_t *off, const double *w, int64_t np,
                             double dt, double *acc, bool fp64, cudaStream_t st);

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_cart2d_step(const CartGeom &g, const CartStepArgs &a, bool fp64,
                               cudaStream_t st);
cudaError_t launch_cart3d_step(const CartGeom &g, const CartStepArgs &a, bool fp64,
                               cudaStream_t st);
// FP32 3-D step with mu = 1, periodic or non-reflecting sides, no limiter (gks_cart3d_side.cu):
// the side-split flux; launch_cart3d_step dispatches to it when cart3d_side_supported().
bool cart3d_side_supported(const CartGeom &g, const CartStepArgs &a, bool fp64);
cudaError_t launch_cart3d_side(const CartGeom &g, const CartStepArgs &a, cudaStream_t st);
// 2-D TM step with divergence cleaning (state Ez, Hx, Hy, psi; mu = 1).
// Divergence-cleaning system on a 3-D grid: V = (E, H, phi, psi), 8 components.
cudaError_t launch_cart3d_phm_step(const CartGeom &g, const CartStepArgs &a, double chi,
                                   double gamma, bool fp64, cudaStream_t st);
cudaError_t launch_cart2d_psi_step(const CartGeom &g, const CartStepArgs &a, double gamma,
                                   bool fp64, cudaStream_t st);
cudaError_t launch_user_to_cart(const CartGeom &g, int ncomp, const double *user, void *dst,
                                bool fp64, cudaStream_t st);
cudaError_t launch_cart_to_user(const CartGeom &g, int ncomp, const void *src, double *user,
                                bool fp64, cudaStream_t st);
cudaError_t launch_fill(void *dst, int64_t n, double value, bool fp64, cudaStream_t st);
// Halo layers of a slab (gks_create_slab): for every component c < ncomp,
// dst[c * dstride + i] = src[c * sstride + i] (add: +=) for i < count.
cudaError_t launch_halo_copy(const void *src, int64_t sstride, void *dst, int64_t dstride,
                             int64_t count, int ncomp, bool add, bool fp64, cudaStream_t st);
// One 2-D component (pitched layout) = a row-major FP64 box of w x h cells at (x0, y0).
cudaError_t launch_box_to_cart(const double *box, void *dst, int x0, int w, int y0, int h,
                               int64_t pitch, bool fp64, cudaStream_t st);
// dst = src on the box of columns [x0, x1) x rows [y0, y1) of every component.
cudaError_t launch_copy_box(const void *src, void *dst, int ncomp, int64_t cstride, int64_t pitch,
                            int x0, int x1, int64_t y0, int64_t y1, bool fp64, cudaStream_t st);
// Energy 1/2 sum |Omega| (eps |E|^2 + mu |H|^2) into *out (device double), FP64 accumulation.
cudaError_t launch_cart_energy(const CartGeom &g, int ncomp, const void *V, const void *eps,
                               const void *mu, bool fp64, double *partials, int npart,
                               double *out, cudaStream_t st);

}  // namespace gks

struct gks_ctx {
  gks_mesh_desc d{};
  cudaStream_t st = nullptr;
  int dim = 2, kind = GKS_CARTESIAN, ncomp = 3;
  bool fp64 = false;
  int64_t ncell = 0;
  size_t esize = 4;
  gks::CartGeom g;
  gks::TetDev tet;              // kind == GKS_TET
  // device buffers
  void *V[2] = {nullptr, nullptr};
  int cur = 0;
  void *eps = nullptr;
  void *mu = nullptr;           // null: mu = 1
  void *src = nullptr;          // J_z mask or null
  int src_box[6] = {0, 0, 0, 0, 0, 0};
  double srcA = 0, srcF0 = 0, srcT0 = 0, srcS = 1;
  int srcKind = 0;              // 0: Gaussian-modulated sine, 1: continuous wave (cosine)
  bool phm = false;             // divergence cleaning (2-D TM: psi is the 4th component)
  double chi = 0.0, gamma = 0.0;
  int limiter = 0;
  int *flag = nullptr;
  double *red = nullptr;        // reduction scratch (partials + result)
  int red_n = 0;
  double *staging = nullptr;    // FP64 user-order staging buffer [ncomp][ncell]
  // time stepping
  double cfl = 0.5, kappa = 0.0, c = 1.0, c_user = 0.0;
  double dt = 0.0, t0 = 0.0;
  int64_t step = 0;
  double C[5] = {0, 0, 0, 0, 0};
  double min_h = 1.0;
  bool fields_written = false;
  int64_t launches = 0;
  // objective / adjoint (2-D Cartesian)
  int64_t *probe_off = nullptr;   // [np] state offsets of the probe cells
  double *probe_w = nullptr;      // [np] |Omega_i|
  int64_t np = 0;
  double *probe_box_w = nullptr;  // probe weights over the probe box (row-major)
  int pbox[4] = {0, 0, 0, 0};     // probe box x0, x1, y0, y1 (half open)
  int32_t *dslot = nullptr;       // state layout, design slot or -1
  int64_t nd = 0;
  int dbox[4] = {0, 0, 0, 0};
  double *obj = nullptr;          // (sum, Kahan compensation)
  // slab of a grid split across ranks (gks_create_slab): layers along the slowest axis (y in
  // 2-D, z in 3-D); the local grid holds two ghost layers beyond each shared side
  bool slab = false;
  int own0 = 0, own1 = 0;         // owned layers [own0, own1) of the local grid
  int shared[2] = {0, 0};         // the low / high side borders another rank
  std::string err;
};
