// Host side of the C ABI declared in include/gks.h: validation, device memory, dt and C1..C5,
// and the step loop.  Every device operation is enqueued on the context's stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gks_internal.h"

namespace gks {

// C1..C5 = integrals over [0, dt] of 1 - e^{-t/tau}, (tau + t)e^{-t/tau} - tau,
// t + tau(e^{-t/tau} - 1), e^{-t/tau}, t e^{-t/tau} (Sec. 3.1).  For x = dt/tau < 2 the closed
// forms cancel badly, so their power series in x are summed (terms alternate and fall fast).
void time_coefficients(double dt, double tau, double C[5]) {
  if (tau == 0.0) {
    C[0] = dt;
    C[1] = 0.0;
    C[2] = 0.5 * dt * dt;
    C[3] = 0.0;
    C[4] = 0.0;
    return;
  }
  const double x = dt / tau;
  if (x >= 2.0) {
    const double E = std::exp(-x);
    const double one_minus_E = -std::expm1(-x);
    C[0] = dt - tau * one_minus_E;
    C[1] = tau * (-dt + 2.0 * tau * one_minus_E - dt * E);
    C[2] = 0.5 * dt * dt - tau * dt + tau * tau * one_minus_E;
    C[3] = tau * one_minus_E;
    C[4] = -tau * dt * E + tau * tau * one_minus_E;
    return;
  }
  // a_n = (-1)^n x^(n-2) / n!  (n >= 1); the five series below are sums of multiples of a_n.
  double s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
  double xp = 1.0 / x;  // x^(n-2) for n = 1
  double fact = 1.0;
  for (int n = 1; n < 60; ++n) {
    fact *= n;
    const double an = ((n & 1) ? -1.0 : 1.0) * xp / fact;
    s4 += -an * x;                    // (1 - E)/x       = sum_{n>=1} -a_n x
    if (n >= 2) {
      s1 += an * x;                   // 1 - (1 - E)/x   = sum_{n>=2} a_n x
      s5 += (n - 1) * an;             // ((1-E) - xE)/x^2
    }
    if (n >= 3) {
      s3 += -an;                      // 1/2 - 1/x + (1-E)/x^2
      s2 += (n - 2) * an;             // (-x + 2(1-E) - xE)/x^2
    }
    xp *= x;
  }
  C[0] = dt * s1;
  C[1] = dt * dt * s2;
  C[2] = dt * dt * s3;
  C[3] = dt * s4;
  C[4] = dt * dt * s5;
}

}  // namespace gks

namespace {

gks_status fail(gks_ctx *ctx, gks_status s, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return s;
}

gks_status cuda_fail(gks_ctx *ctx, cudaError_t e, const char *where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(ctx, GKS_E_CUDA, m);
}

#define GKS_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

bool finite_positive(double v) { return std::isfinite(v) && v > 0.0; }

// Fastest cleaning wave: gamma (psi, div B) and, in 3-D, chi (phi, div E); the 2-D TM system
// carries no phi.  0 without cleaning.
double cleaning_speed(const gks_ctx *ctx) {
  if (!ctx->phm) return 0.0;
  return ctx->dim == 3 ? std::fmax(ctx->chi, ctx->gamma) : ctx->gamma;
}

// dt = CFL h_min / c and C1..C5 with tau = kappa dt.
void refresh_time_step(gks_ctx *ctx) {
  ctx->dt = ctx->cfl * ctx->min_h / ctx->c;
  gks::time_coefficients(ctx->dt, ctx->kappa * ctx->dt, ctx->C);
}

gks_status alloc_dev(gks_ctx *ctx, void **p, size_t bytes) {
  cudaError_t e = cudaMallocAsync(p, bytes, ctx->st);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, GKS_E_NOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  return GKS_OK;
}

gks_status upload_cells(gks_ctx *ctx, const double *host, int ncomp, void *dst) {
  const size_t bytes = sizeof(double) * (size_t)ncomp * (size_t)ctx->ncell;
  GKS_CUDA(cudaMemcpyAsync(ctx->staging, host, bytes, cudaMemcpyHostToDevice, ctx->st));
  if (ctx->kind == GKS_TET)
    GKS_CUDA(gks::launch_user_to_tet(ctx->tet, ncomp, ctx->staging, dst, ctx->fp64, ctx->st));
  else
    GKS_CUDA(gks::launch_user_to_cart(ctx->g, ncomp, ctx->staging, dst, ctx->fp64, ctx->st));
  return GKS_OK;
}

template <typename V>
gks_status upload_vec(gks_ctx *ctx, const std::vector<V> &h, V **d) {
  gks_status s = alloc_dev(ctx, reinterpret_cast<void **>(d), sizeof(V) * (h.size() ? h.size() : 1));
  if (s != GKS_OK) return s;
  if (!h.empty())
    GKS_CUDA(cudaMemcpyAsync(*d, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, ctx->st));
  return GKS_OK;
}

// Build the tet geometry on the host and copy it to the device (kind == GKS_TET).
gks_status setup_tets(gks_ctx *ctx, const gks_mesh_desc *d) {
  gks::TetHost h;
  gks_status s = gks::build_tet_geometry(d->vert_xyz, d->n_vert, d->tet_vert, d->n_tet, h, ctx->err);
  if (s != GKS_OK) return s;
  gks::TetDev &g = ctx->tet;
  g.nt = h.nt;
  g.nf = h.nf;
  g.pec = d->tet_bc == GKS_BC_PEC;
  // packed step geometry (FP64 values, rounded once to FP32 for FP32 contexts)
  std::vector<double> fgeo((size_t)h.nf * gks::kTetFaceGeo);
  std::vector<double> cw((size_t)h.nt * gks::kTetCellW), cu((size_t)h.nt * gks::kTetCellU);
  for (int64_t f = 0; f < h.nf; ++f) {
    double *q = &fgeo[(size_t)f * gks::kTetFaceGeo];
    // the frame's rows t, w follow from n and 1/(1 + n_1) (zero for n_1 = -1, which gives the
    // special frame diag(-1, -1, 1) from the same expressions)
    const double *T = &h.fT[9 * f];
    for (int k = 0; k < 3; ++k) q[k] = T[k];
    q[3] = T[0] == -1.0 ? 0.0 : gks::frame_inv_one_plus(T[0], T[1], T[2]);
    for (int a = 0; a < 3; ++a) { q[4 + a] = h.fdL[3 * f + a]; q[7 + a] = h.fdR[3 * f + a]; }
  }
  for (int64_t i = 0; i < h.nt; ++i) {
    for (int k = 0; k < 12; ++k) cw[(size_t)i * gks::kTetCellW + k] = h.cw[12 * i + k];
    for (int k = 0; k < 4; ++k)   // the face area enters here, not in the face pass
      cu[(size_t)i * gks::kTetCellU + k] =
          h.csign[4 * i + k] * h.farea[h.cface[4 * i + k]] * h.ivol[i];
  }
  if ((s = upload_vec(ctx, h.perm, &g.perm)) != GKS_OK || (s = upload_vec(ctx, h.vol, &g.vol)) != GKS_OK ||
      (s = upload_vec(ctx, h.cnb, &g.cnb)) != GKS_OK || (s = upload_vec(ctx, h.cface, &g.cface)) != GKS_OK ||
      (s = upload_vec(ctx, h.fL, &g.fL)) != GKS_OK || (s = upload_vec(ctx, h.fR, &g.fR)) != GKS_OK)
    return s;
  if (ctx->fp64) {
    double *fd = nullptr, *wd = nullptr, *ud = nullptr;
    s = upload_vec(ctx, fgeo, &fd);
    g.fgeo = fd;
    if (s != GKS_OK || (s = upload_vec(ctx, cw, &wd)) != GKS_OK) return s;
    g.cw = wd;
    if ((s = upload_vec(ctx, cu, &ud)) != GKS_OK) return s;
    g.cu = ud;
  } else {
    std::vector<float> f32(fgeo.begin(), fgeo.end()), w32(cw.begin(), cw.end()),
        u32(cu.begin(), cu.end());
    float *fd = nullptr, *wd = nullptr, *ud = nullptr;
    s = upload_vec(ctx, f32, &fd);
    g.fgeo = fd;
    if (s != GKS_OK || (s = upload_vec(ctx, w32, &wd)) != GKS_OK) return s;
    g.cw = wd;
    if ((s = upload_vec(ctx, u32, &ud)) != GKS_OK) return s;
    g.cu = ud;
    // the pageable host vectors must outlive the copies
    GKS_CUDA(cudaStreamSynchronize(ctx->st));
  }
  if ((s = alloc_dev(ctx, &g.Gscratch, ctx->esize * 18 * (size_t)g.nt)) != GKS_OK ||
      (s = alloc_dev(ctx, &g.Fscratch, ctx->esize * 6 * (size_t)g.nf)) != GKS_OK)
    return s;
  ctx->min_h = h.min_h;
  // host copies are released here; wait so the pageable sources outlive the copies
  GKS_CUDA(cudaStreamSynchronize(ctx->st));
  return GKS_OK;
}

gks_status check_flag(gks_ctx *ctx) {
  int h = 0;
  GKS_CUDA(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  GKS_CUDA(cudaStreamSynchronize(ctx->st));
  // bit 1: a staged kernel's bounded wait for a tensor copy ran out; bit 0: non-finite value
  if (h & 2) return fail(ctx, GKS_E_TIMEOUT, "a kernel's bounded wait for a staged copy ran out");
  if (h) return fail(ctx, GKS_E_NONFINITE, "a non-finite value appeared in the state");
  return GKS_OK;
}

}  // namespace

extern "C" {

gks_status gks_create_mesh(const gks_mesh_desc *d, gks_ctx **out) {
  if (!out) return GKS_E_ARG;
  *out = nullptr;
  if (!d) return GKS_E_ARG;
  if (d->dim != 2 && d->dim != 3) return GKS_E_ARG;
  if (d->precision != GKS_FP32 && d->precision != GKS_FP64) return GKS_E_ARG;
  if (!finite_positive(d->cfl) || !(d->tau_over_dt >= 0.0) || !std::isfinite(d->tau_over_dt))
    return GKS_E_ARG;
  if (d->kind != GKS_CARTESIAN && d->kind != GKS_TET) return GKS_E_ARG;
  if (!(d->chi >= 0.0) || !(d->gamma >= 0.0) || !std::isfinite(d->chi) || !std::isfinite(d->gamma))
    return GKS_E_ARG;
  const bool phm = d->chi > 0.0 || d->gamma > 0.0;
  if (d->limiter != GKS_LIMITER_NONE && d->limiter != GKS_LIMITER_VAN_LEER) return GKS_E_ARG;
  if (d->limiter != GKS_LIMITER_NONE && d->kind != GKS_CARTESIAN) return GKS_E_UNSUPPORTED;
  if (phm && d->kind != GKS_CARTESIAN) return GKS_E_UNSUPPORTED;
  if (d->kind == GKS_TET) {
    if (d->dim != 3 || !d->vert_xyz || !d->tet_vert || d->n_vert < 4 || d->n_tet < 1)
      return GKS_E_ARG;
    if (d->tet_bc != GKS_BC_NONREFLECTING && d->tet_bc != GKS_BC_PEC) return GKS_E_ARG;
  }
  for (int a = 0; a < (d->kind == GKS_TET ? 0 : d->dim); ++a) {
    if (d->n[a] < 1 || d->n[a] > (1 << 24)) return GKS_E_ARG;
    if (!(d->hi[a] > d->lo[a]) || !std::isfinite(d->hi[a] - d->lo[a])) return GKS_E_ARG;
    const int b0 = d->bc[2 * a], b1 = d->bc[2 * a + 1];
    auto known = [](int b) {
      return b == GKS_BC_PERIODIC || b == GKS_BC_NONREFLECTING || b == GKS_BC_PEC;
    };
    if (!known(b0) || !known(b1)) return GKS_E_ARG;
    if ((b0 == GKS_BC_PERIODIC) != (b1 == GKS_BC_PERIODIC)) return GKS_E_ARG;
    if ((b0 == GKS_BC_PEC || b1 == GKS_BC_PEC) && d->n[a] < 2) return GKS_E_ARG;
  }

  gks_ctx *ctx = new (std::nothrow) gks_ctx();
  if (!ctx) return GKS_E_NOMEM;
  ctx->d = *d;
  ctx->d.vert_xyz = nullptr;
  ctx->d.tet_vert = nullptr;
  ctx->st = (cudaStream_t)d->cuda_stream;
  ctx->dim = d->dim;
  ctx->kind = d->kind;
  ctx->ncomp = d->dim == 2 ? (phm ? 4 : 3) : (phm ? 8 : 6);
  ctx->phm = phm;
  ctx->chi = d->chi;
  ctx->gamma = d->gamma;
  ctx->limiter = d->limiter;
  ctx->fp64 = d->precision == GKS_FP64;
  ctx->esize = ctx->fp64 ? 8 : 4;
  ctx->cfl = d->cfl;
  ctx->kappa = d->tau_over_dt;
  ctx->c_user = d->c_lattice;

  gks::CartGeom &g = ctx->g;
  g.dim = d->dim;
  if (d->kind == GKS_TET) {
    gks_status s = setup_tets(ctx, d);
    if (s != GKS_OK) {
      gks_destroy(ctx);
      return s;
    }
    g.nx = (int)ctx->tet.nt; g.ny = 1; g.nz = 1;
    g.pitch = ctx->tet.nt; g.plane = g.pitch; g.cstride = g.pitch;
    ctx->ncell = ctx->tet.nt;
  } else {
    g.nx = (int)d->n[0];
    g.ny = (int)d->n[1];
    g.nz = d->dim == 3 ? (int)d->n[2] : 1;
    g.pitch = ((int64_t)g.nx + 31) / 32 * 32;
    g.plane = g.pitch * g.ny;
    g.cstride = g.plane * g.nz;
    ctx->ncell = (int64_t)g.nx * g.ny * g.nz;
    for (int a = 0; a < d->dim; ++a) {
      g.h[a] = (d->hi[a] - d->lo[a]) / (double)d->n[a];
      g.periodic[a] = d->bc[2 * a] == GKS_BC_PERIODIC;
      g.pec[2 * a] = d->bc[2 * a] == GKS_BC_PEC;
      g.pec[2 * a + 1] = d->bc[2 * a + 1] == GKS_BC_PEC;
    }
    // h_i = 2 dim |Omega| / sum_s |l_s| for a box cell is dim / sum_a (1/h_a); it equals the
    // edge for squares and cubes.
    double sum = 0;
    for (int a = 0; a < d->dim; ++a) sum += 1.0 / g.h[a];
    ctx->min_h = d->dim / sum;
  }
  ctx->c = ctx->c_user > 0 ? ctx->c_user : std::fmax(1.0, cleaning_speed(ctx));

  gks_status s = GKS_OK;
  const size_t fbytes = ctx->esize * (size_t)ctx->ncomp * (size_t)g.cstride;
  const size_t mbytes = ctx->esize * (size_t)g.cstride;
  if ((s = alloc_dev(ctx, &ctx->V[0], fbytes)) != GKS_OK ||
      (s = alloc_dev(ctx, &ctx->V[1], fbytes)) != GKS_OK ||
      (s = alloc_dev(ctx, &ctx->eps, mbytes)) != GKS_OK ||
      (s = alloc_dev(ctx, (void **)&ctx->flag, sizeof(int))) != GKS_OK ||
      (s = alloc_dev(ctx, (void **)&ctx->staging, sizeof(double) * ctx->ncomp * ctx->ncell)) !=
          GKS_OK) {
    gks_destroy(ctx);
    return s;
  }
  ctx->red_n = 2 * 152 * 8;
  if ((s = alloc_dev(ctx, (void **)&ctx->red, sizeof(double) * (ctx->red_n + 1))) != GKS_OK) {
    gks_destroy(ctx);
    return s;
  }
  cudaError_t e;
  if ((e = cudaMemsetAsync(ctx->V[0], 0, fbytes, ctx->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->V[1], 0, fbytes, ctx->st)) != cudaSuccess ||
      (e = cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st)) != cudaSuccess ||
      (e = gks::launch_fill(ctx->eps, g.cstride, 1.0, ctx->fp64, ctx->st)) != cudaSuccess) {
    gks_destroy(ctx);
    return GKS_E_CUDA;
  }
  refresh_time_step(ctx);
  *out = ctx;
  return GKS_OK;
}

gks_status gks_create_slab(const gks_mesh_desc *global, const gks_slab_desc *slab,
                           gks_ctx **out) {
  if (!out) return GKS_E_ARG;
  *out = nullptr;
  if (!global || !slab) return GKS_E_ARG;
  if (global->kind != GKS_CARTESIAN || (global->dim != 2 && global->dim != 3)) return GKS_E_ARG;
  // every rank must step with the same dt and lattice speed: the automatic speed would follow
  // each slab's own materials
  if (!finite_positive(global->c_lattice)) return GKS_E_ARG;
  const int ax = global->dim - 1;                 // slowest axis: y in 2-D, z in 3-D
  const int64_t n = global->n[ax];
  const int lo_sh = slab->shared_lo, hi_sh = slab->shared_hi;
  if ((lo_sh != 0 && lo_sh != 1) || (hi_sh != 0 && hi_sh != 1)) return GKS_E_ARG;
  if (n < 1 || slab->begin < 0 || slab->end > n || slab->begin >= slab->end) return GKS_E_ARG;
  const int64_t own = slab->end - slab->begin;
  if ((lo_sh || hi_sh) && own < 2) return GKS_E_ARG;   // two owned layers go to each neighbour
  const bool per = global->bc[2 * ax] == GKS_BC_PERIODIC;
  if (per && lo_sh != hi_sh) return GKS_E_ARG;         // a periodic axis splits into a ring
  if (!per && ((lo_sh && slab->begin == 0) || (hi_sh && slab->end == n))) return GKS_E_ARG;
  if (!(global->hi[ax] > global->lo[ax]) || !std::isfinite(global->hi[ax] - global->lo[ax]))
    return GKS_E_ARG;
  const double h = (global->hi[ax] - global->lo[ax]) / (double)n;
  const int64_t first = slab->begin - 2 * lo_sh;        // global index of local layer 0
  const int64_t nloc = own + 2 * (lo_sh + hi_sh);
  gks_mesh_desc d = *global;
  d.n[ax] = nloc;
  d.lo[ax] = global->lo[ax] + (double)first * h;
  d.hi[ax] = d.lo[ax] + (double)nloc * h;
  // a shared side's ghost layers are rewritten by gks_halo_import before every step, so the
  // local grid's own boundary there only touches ghost cells
  if (lo_sh || hi_sh) {
    if (lo_sh) d.bc[2 * ax] = GKS_BC_NONREFLECTING;
    if (hi_sh) d.bc[2 * ax + 1] = GKS_BC_NONREFLECTING;
    if (per) d.bc[2 * ax] = d.bc[2 * ax + 1] = GKS_BC_NONREFLECTING;
  }
  gks_status s = gks_create_mesh(&d, out);
  if (s != GKS_OK) return s;
  gks_ctx *ctx = *out;
  ctx->slab = true;
  ctx->own0 = 2 * lo_sh;
  ctx->own1 = ctx->own0 + (int)own;
  ctx->shared[0] = lo_sh;
  ctx->shared[1] = hi_sh;
  // the same cell size (hence dt and C1..C5) as the whole grid, bit for bit
  ctx->g.h[ax] = h;
  double sum = 0;
  for (int a = 0; a < ctx->dim; ++a) sum += 1.0 / ctx->g.h[a];
  ctx->min_h = ctx->dim / sum;
  refresh_time_step(ctx);
  return GKS_OK;
}

namespace {

// Elements of one layer of the slab axis in the state layout (a padded row in 2-D, a plane in
// 3-D), and the first local layer of the two that a halo call moves.
int64_t halo_layer_elems(const gks_ctx *ctx) {
  return ctx->dim == 3 ? ctx->g.plane : ctx->g.pitch;
}

gks_status halo_check(gks_ctx *ctx, int32_t side, int32_t layers, int *first) {
  if (!ctx->slab) return fail(ctx, GKS_E_UNSUPPORTED, "halo calls need a slab context");
  if (side != 0 && side != 1) return fail(ctx, GKS_E_ARG, "side must be 0 (low) or 1 (high)");
  if (!ctx->shared[side]) return fail(ctx, GKS_E_ARG, "that side is not shared with a rank");
  if (layers == GKS_HALO_OWNED)
    *first = side == 0 ? ctx->own0 : ctx->own1 - 2;
  else if (layers == GKS_HALO_GHOST)
    *first = side == 0 ? ctx->own0 - 2 : ctx->own1;
  else
    return fail(ctx, GKS_E_ARG, "layers must be GKS_HALO_OWNED or GKS_HALO_GHOST");
  return GKS_OK;
}

}  // namespace

gks_status gks_halo_bytes(const gks_ctx *ctx, int64_t *bytes) {
  if (!ctx || !bytes) return GKS_E_ARG;
  if (!ctx->slab) return GKS_E_UNSUPPORTED;
  *bytes = (int64_t)ctx->esize * ctx->ncomp * 2 * halo_layer_elems(ctx);
  return GKS_OK;
}

gks_status gks_halo_export(gks_ctx *ctx, int32_t side, int32_t layers, const void *state,
                           void *buf) {
  if (!ctx) return GKS_E_ARG;
  int first = 0;
  gks_status s = halo_check(ctx, side, layers, &first);
  if (s != GKS_OK) return s;
  if (!buf) return fail(ctx, GKS_E_ARG, "buf is NULL");
  const int64_t L = halo_layer_elems(ctx);
  const char *base = static_cast<const char *>(state ? state : ctx->V[ctx->cur]);
  GKS_CUDA(gks::launch_halo_copy(base + (size_t)first * L * ctx->esize, ctx->g.cstride, buf,
                                 2 * L, 2 * L, ctx->ncomp, false, ctx->fp64, ctx->st));
  ctx->launches += 1;
  return GKS_OK;
}

gks_status gks_halo_import(gks_ctx *ctx, int32_t side, int32_t layers, void *state,
                           const void *buf, int32_t add) {
  if (!ctx) return GKS_E_ARG;
  int first = 0;
  gks_status s = halo_check(ctx, side, layers, &first);
  if (s != GKS_OK) return s;
  if (!buf) return fail(ctx, GKS_E_ARG, "buf is NULL");
  if (add != 0 && add != 1) return fail(ctx, GKS_E_ARG, "add must be 0 or 1");
  const int64_t L = halo_layer_elems(ctx);
  char *base = static_cast<char *>(state ? state : ctx->V[ctx->cur]);
  GKS_CUDA(gks::launch_halo_copy(buf, 2 * L, base + (size_t)first * L * ctx->esize,
                                 ctx->g.cstride, 2 * L, ctx->ncomp, add != 0, ctx->fp64, ctx->st));
  ctx->launches += 1;
  return GKS_OK;
}

gks_status gks_set_materials(gks_ctx *ctx, const double *eps, const double *mu) {
  if (!ctx) return GKS_E_ARG;
  if (!eps) return fail(ctx, GKS_E_ARG, "eps is NULL");
  if (mu && ctx->phm) return fail(ctx, GKS_E_UNSUPPORTED, "divergence cleaning needs mu = 1");
  // lattice speed: the fastest wave, light 1/sqrt(eps mu) or a cleaning wave (mu = 1)
  double cmax = cleaning_speed(ctx);
  for (int64_t i = 0; i < ctx->ncell; ++i) {
    const double e = eps[i], m = mu ? mu[i] : 1.0;
    if (!finite_positive(e) || !finite_positive(m))
      return fail(ctx, GKS_E_ARG, "eps and mu must be finite and > 0 (cell " +
                                      std::to_string(i) + ")");
    cmax = std::fmax(cmax, 1.0 / std::sqrt(e * m));
  }
  gks_status s;
  if ((s = upload_cells(ctx, eps, 1, ctx->eps)) != GKS_OK) return s;
  if (mu) {
    if (!ctx->mu) {
      if ((s = alloc_dev(ctx, &ctx->mu, ctx->esize * (size_t)ctx->g.cstride)) != GKS_OK) return s;
    }
    if ((s = upload_cells(ctx, mu, 1, ctx->mu)) != GKS_OK) return s;
  } else if (ctx->mu) {
    GKS_CUDA(cudaFreeAsync(ctx->mu, ctx->st));
    ctx->mu = nullptr;
  }
  ctx->c = ctx->c_user > 0 ? ctx->c_user : cmax;
  refresh_time_step(ctx);
  return GKS_OK;
}

gks_status gks_set_materials_box(gks_ctx *ctx, int64_t x0, int64_t x1, int64_t y0, int64_t y1,
                                 const double *eps_box) {
  if (!ctx) return GKS_E_ARG;
  if (ctx->kind != GKS_CARTESIAN || ctx->dim != 2)
    return fail(ctx, GKS_E_UNSUPPORTED, "a box update of eps needs a 2-D Cartesian grid");
  if (!eps_box || x0 < 0 || y0 < 0 || x1 > ctx->g.nx || y1 > ctx->g.ny || x0 >= x1 || y0 >= y1)
    return fail(ctx, GKS_E_ARG, "eps_box is NULL or the box is empty / outside the grid");
  if (!(ctx->c_user > 0))
    return fail(ctx, GKS_E_STATE, "a box update of eps needs a fixed lattice speed (c_lattice > 0)");
  const int64_t n = (x1 - x0) * (y1 - y0);
  for (int64_t i = 0; i < n; ++i)
    if (!finite_positive(eps_box[i]))
      return fail(ctx, GKS_E_ARG, "eps must be finite and > 0 (box entry " + std::to_string(i) + ")");
  GKS_CUDA(cudaMemcpyAsync(ctx->staging, eps_box, sizeof(double) * (size_t)n,
                           cudaMemcpyHostToDevice, ctx->st));
  GKS_CUDA(gks::launch_box_to_cart(ctx->staging, ctx->eps, (int)x0, (int)(x1 - x0), (int)y0,
                                   (int)(y1 - y0), ctx->g.pitch, ctx->fp64, ctx->st));
  return GKS_OK;
}

gks_status gks_reset_objective(gks_ctx *ctx) {
  if (!ctx) return GKS_E_ARG;
  if (!ctx->obj) return fail(ctx, GKS_E_STATE, "gks_set_objective must come first");
  GKS_CUDA(cudaMemsetAsync(ctx->obj, 0, 2 * sizeof(double), ctx->st));
  return GKS_OK;
}

gks_status gks_write_fields(gks_ctx *ctx, const double *fields, double t0) {
  if (!ctx) return GKS_E_ARG;
  if (!fields) return fail(ctx, GKS_E_ARG, "fields is NULL");
  if (!std::isfinite(t0)) return fail(ctx, GKS_E_ARG, "t0 must be finite");
  gks_status s = upload_cells(ctx, fields, ctx->ncomp, ctx->V[ctx->cur]);
  if (s != GKS_OK) return s;
  GKS_CUDA(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st));
  if (ctx->obj) GKS_CUDA(cudaMemsetAsync(ctx->obj, 0, 2 * sizeof(double), ctx->st));
  ctx->t0 = t0;
  ctx->step = 0;
  ctx->fields_written = true;
  return GKS_OK;
}

namespace {

// Upload a source mask and its bounding box (shared by both waveforms).
gks_status set_source_mask(gks_ctx *ctx, const double *jz_mask) {
  const gks::CartGeom &g = ctx->g;
  int box[6] = {g.nx, -1, g.ny, -1, g.nz, -1};
  for (int64_t i = 0; i < ctx->ncell; ++i) {
    const double v = jz_mask[i];
    if (!std::isfinite(v)) return fail(ctx, GKS_E_ARG, "jz_mask must be finite");
    if (v != 0.0 && ctx->kind == GKS_CARTESIAN) {
      const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((int64_t)g.nx * g.ny));
      box[0] = std::min(box[0], ix); box[1] = std::max(box[1], ix);
      box[2] = std::min(box[2], iy); box[3] = std::max(box[3], iy);
      box[4] = std::min(box[4], iz); box[5] = std::max(box[5], iz);
    }
  }
  gks_status st;
  if (!ctx->src) {
    if ((st = alloc_dev(ctx, &ctx->src, ctx->esize * (size_t)g.cstride)) != GKS_OK) return st;
  }
  if ((st = upload_cells(ctx, jz_mask, 1, ctx->src)) != GKS_OK) return st;
  if (box[1] < 0) {  // all zero
    box[0] = box[2] = box[4] = 0;
    box[1] = box[3] = box[5] = -1;
  }
  ctx->src_box[0] = box[0]; ctx->src_box[1] = box[1] + 1;
  ctx->src_box[2] = box[2]; ctx->src_box[3] = box[3] + 1;
  ctx->src_box[4] = box[4]; ctx->src_box[5] = box[5] + 1;
  return GKS_OK;
}

}  // namespace

gks_status gks_set_source(gks_ctx *ctx, const double *jz_mask, double A, double f0, double t0,
                          double s) {
  if (!ctx) return GKS_E_ARG;
  if (!jz_mask) {
    if (ctx->src) GKS_CUDA(cudaFreeAsync(ctx->src, ctx->st));
    ctx->src = nullptr;
    return GKS_OK;
  }
  if (!std::isfinite(A) || !std::isfinite(f0) || !std::isfinite(t0) || !finite_positive(s))
    return fail(ctx, GKS_E_ARG, "source parameters must be finite and s > 0");
  gks_status st = set_source_mask(ctx, jz_mask);
  if (st != GKS_OK) return st;
  ctx->srcKind = 0;
  ctx->srcA = A;
  ctx->srcF0 = f0;
  ctx->srcT0 = t0;
  ctx->srcS = s;
  return GKS_OK;
}

gks_status gks_set_source_cw(gks_ctx *ctx, const double *jz_mask, double A, double f0, double t0) {
  if (!ctx) return GKS_E_ARG;
  if (!jz_mask) {
    if (ctx->src) GKS_CUDA(cudaFreeAsync(ctx->src, ctx->st));
    ctx->src = nullptr;
    return GKS_OK;
  }
  if (!std::isfinite(A) || !std::isfinite(f0) || !std::isfinite(t0))
    return fail(ctx, GKS_E_ARG, "source parameters must be finite");
  gks_status st = set_source_mask(ctx, jz_mask);
  if (st != GKS_OK) return st;
  ctx->srcKind = 1;
  ctx->srcA = A;
  ctx->srcF0 = f0;
  ctx->srcT0 = t0;
  ctx->srcS = 1.0;
  return GKS_OK;
}

gks_status gks_set_dt(gks_ctx *ctx, double dt) {
  if (!ctx) return GKS_E_ARG;
  if (!finite_positive(dt)) return fail(ctx, GKS_E_ARG, "dt must be finite and > 0");
  ctx->dt = dt;
  gks::time_coefficients(dt, ctx->kappa * dt, ctx->C);
  return GKS_OK;
}

namespace {

// Advance n_steps over the window [x0, x1) x [y0, y1) (2-D) or the whole mesh.
gks_status step_impl(gks_ctx *ctx, int64_t n_steps, const int win[4], bool objective) {
  gks::CartStepArgs a;
  a.eps = ctx->eps;
  a.mu = ctx->mu;
  a.src = ctx->src;
  std::memcpy(a.src_box, ctx->src_box, sizeof(a.src_box));
  std::memcpy(a.C, ctx->C, sizeof(a.C));
  std::memcpy(a.window, win, sizeof(a.window));
  a.c = ctx->c;
  a.flag = ctx->flag;
  a.limiter = ctx->limiter;
  for (int64_t n = 0; n < n_steps; ++n) {
    const double t = ctx->t0 + (double)ctx->step * ctx->dt;
    a.src_amp = 0.0;
    if (ctx->src) {
      const double tt = t - ctx->srcT0;
      if (ctx->srcKind == 1)
        a.src_amp = tt >= 0.0 ? ctx->dt * ctx->srcA * std::cos(2.0 * M_PI * ctx->srcF0 * tt) : 0.0;
      else
        a.src_amp = ctx->dt * ctx->srcA * std::exp(-(tt / ctx->srcS) * (tt / ctx->srcS)) *
                    std::sin(2.0 * M_PI * ctx->srcF0 * tt);
    }
    a.V = ctx->V[ctx->cur];
    a.Vout = ctx->V[ctx->cur ^ 1];
    cudaError_t e;
    if (ctx->kind == GKS_TET) {
      e = gks::launch_tet_step(ctx->tet, a.V, a.Vout, a.eps, a.mu, a.src, a.src_amp, a.C, a.c,
                               a.flag, ctx->fp64, ctx->st);
      ctx->launches += 3;
    } else {
      if (ctx->dim == 2)
        e = ctx->phm ? gks::launch_cart2d_psi_step(ctx->g, a, ctx->gamma, ctx->fp64, ctx->st)
                     : gks::launch_cart2d_step(ctx->g, a, ctx->fp64, ctx->st);
      else
        e = ctx->phm ? gks::launch_cart3d_phm_step(ctx->g, a, ctx->chi, ctx->gamma, ctx->fp64,
                                                   ctx->st)
                     : gks::launch_cart3d_step(ctx->g, a, ctx->fp64, ctx->st);
      ctx->launches += 1;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
    ctx->cur ^= 1;
    ctx->step += 1;
    if (objective && ctx->np > 0) {
      e = gks::launch_objective(ctx->V[ctx->cur], ctx->probe_off, ctx->probe_w, ctx->np, ctx->dt,
                                ctx->obj, ctx->fp64, ctx->st);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "objective launch");
      ctx->launches += 1;
    }
  }
  return GKS_OK;
}

}  // namespace

gks_status gks_step(gks_ctx *ctx, int64_t n_steps) {
  if (!ctx) return GKS_E_ARG;
  if (n_steps < 0) return fail(ctx, GKS_E_ARG, "n_steps must be >= 0");
  if (!ctx->fields_written) return fail(ctx, GKS_E_STATE, "gks_write_fields must come first");
  const int win[4] = {0, ctx->g.nx, 0, ctx->g.ny};
  return step_impl(ctx, n_steps, win, true);
}

gks_status gks_step_window(gks_ctx *ctx, int64_t n_steps, int64_t x0, int64_t x1, int64_t y0,
                           int64_t y1) {
  if (!ctx) return GKS_E_ARG;
  if (ctx->kind != GKS_CARTESIAN || ctx->dim != 2)
    return fail(ctx, GKS_E_UNSUPPORTED, "windowed steps need a 2-D Cartesian grid");
  if (ctx->phm) return fail(ctx, GKS_E_UNSUPPORTED, "windowed steps do not cover divergence cleaning");
  if (n_steps < 0 || x0 < 0 || y0 < 0 || x1 > ctx->g.nx || y1 > ctx->g.ny || x0 >= x1 || y0 >= y1)
    return fail(ctx, GKS_E_ARG, "window outside the grid or empty");
  if (!ctx->fields_written) return fail(ctx, GKS_E_STATE, "gks_write_fields must come first");
  const int win[4] = {(int)x0, (int)x1, (int)y0, (int)y1};
  return step_impl(ctx, n_steps, win, false);
}

gks_status gks_copy_state_box(gks_ctx *ctx, void *dst, int64_t x0, int64_t x1, int64_t y0,
                              int64_t y1) {
  if (!ctx) return GKS_E_ARG;
  if (ctx->kind != GKS_CARTESIAN) return fail(ctx, GKS_E_UNSUPPORTED, "a Cartesian grid is required");
  if (!dst || x0 < 0 || x1 > ctx->g.nx || x0 >= x1 || y0 < 0 ||
      y1 > (int64_t)ctx->g.ny * ctx->g.nz || y0 >= y1)
    return fail(ctx, GKS_E_ARG, "dst is NULL or the box is empty / outside the grid");
  GKS_CUDA(gks::launch_copy_box(ctx->V[ctx->cur], dst, ctx->ncomp, ctx->g.cstride, ctx->g.pitch,
                                 (int)x0, (int)x1, y0, y1, ctx->fp64, ctx->st));
  ctx->launches += 1;
  return GKS_OK;
}

gks_status gks_read_fields(gks_ctx *ctx, double *out) {
  if (!ctx) return GKS_E_ARG;
  if (!out) return fail(ctx, GKS_E_ARG, "out is NULL");
  if (ctx->kind == GKS_TET)
    GKS_CUDA(gks::launch_tet_to_user(ctx->tet, ctx->ncomp, ctx->V[ctx->cur], ctx->staging,
                                     ctx->fp64, ctx->st));
  else
    GKS_CUDA(gks::launch_cart_to_user(ctx->g, ctx->ncomp, ctx->V[ctx->cur], ctx->staging,
                                      ctx->fp64, ctx->st));
  GKS_CUDA(cudaMemcpyAsync(out, ctx->staging, sizeof(double) * ctx->ncomp * ctx->ncell,
                           cudaMemcpyDeviceToHost, ctx->st));
  return check_flag(ctx);
}

gks_status gks_energy(gks_ctx *ctx, double *out) {
  if (!ctx) return GKS_E_ARG;
  if (!out) return fail(ctx, GKS_E_ARG, "out is NULL");
  if (ctx->kind == GKS_TET)
    GKS_CUDA(gks::launch_tet_energy(ctx->tet, ctx->V[ctx->cur], ctx->eps, ctx->mu, ctx->fp64,
                                    ctx->red, ctx->red_n, ctx->red + ctx->red_n, ctx->st));
  else if (ctx->slab) {
    // owned layers only: the ghost layers belong to the neighbouring ranks
    gks::CartGeom g = ctx->g;
    const int64_t off = (int64_t)ctx->own0 * halo_layer_elems(ctx) * (int64_t)ctx->esize;
    (ctx->dim == 3 ? g.nz : g.ny) = ctx->own1 - ctx->own0;
    const char *V = static_cast<const char *>(ctx->V[ctx->cur]) + off;
    const char *eps = static_cast<const char *>(ctx->eps) + off;
    const char *mu = ctx->mu ? static_cast<const char *>(ctx->mu) + off : nullptr;
    GKS_CUDA(gks::launch_cart_energy(g, ctx->ncomp, V, eps, mu, ctx->fp64, ctx->red,
                                     ctx->red_n, ctx->red + ctx->red_n, ctx->st));
  } else
    GKS_CUDA(gks::launch_cart_energy(ctx->g, ctx->ncomp, ctx->V[ctx->cur], ctx->eps, ctx->mu,
                                     ctx->fp64, ctx->red, ctx->red_n, ctx->red + ctx->red_n,
                                     ctx->st));
  GKS_CUDA(cudaMemcpyAsync(out, ctx->red + ctx->red_n, sizeof(double), cudaMemcpyDeviceToHost,
                           ctx->st));
  return check_flag(ctx);
}

gks_status gks_sync(gks_ctx *ctx) {
  if (!ctx) return GKS_E_ARG;
  GKS_CUDA(cudaStreamSynchronize(ctx->st));
  GKS_CUDA(cudaGetLastError());
  return check_flag(ctx);
}


gks_status gks_set_objective(gks_ctx *ctx, const int64_t *probe, int64_t np, const int64_t *design,
                             int64_t nd) {
  if (!ctx) return GKS_E_ARG;
  if (ctx->kind != GKS_CARTESIAN || ctx->dim != 2)
    return fail(ctx, GKS_E_UNSUPPORTED, "the objective and its adjoint need a 2-D Cartesian grid");
  if (np < 0 || nd < 0 || (np > 0 && !probe) || (nd > 0 && !design))
    return fail(ctx, GKS_E_ARG, "probe / design lists");
  const gks::CartGeom &g = ctx->g;
  std::vector<int64_t> off(np);
  std::vector<double> w(np, g.h[0] * g.h[1]);
  int pbox[4] = {g.nx, -1, g.ny, -1};
  for (int64_t i = 0; i < np; ++i) {
    const int64_t c = probe[i];
    if (c < 0 || c >= ctx->ncell) return fail(ctx, GKS_E_ARG, "probe cell out of range");
    off[i] = (c / g.nx) * g.pitch + c % g.nx;          // Ez component of the state layout
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    pbox[0] = std::min(pbox[0], x); pbox[1] = std::max(pbox[1], x + 1);
    pbox[2] = std::min(pbox[2], y); pbox[3] = std::max(pbox[3], y + 1);
  }
  // the same weights over the probe's bounding box (zero off the probe), for the adjoint
  std::vector<double> wbox;
  if (np > 0) {
    const int bw = pbox[1] - pbox[0];
    wbox.assign((size_t)bw * (pbox[3] - pbox[2]), 0.0);
    for (int64_t i = 0; i < np; ++i) {
      const int x = (int)(probe[i] % g.nx), y = (int)(probe[i] / g.nx);
      wbox[(size_t)(y - pbox[2]) * bw + (x - pbox[0])] += w[i];
    }
  }
  std::vector<int32_t> slot((size_t)g.cstride, -1);
  int box[4] = {g.nx, -1, g.ny, -1};
  for (int64_t i = 0; i < nd; ++i) {
    const int64_t c = design[i];
    if (c < 0 || c >= ctx->ncell) return fail(ctx, GKS_E_ARG, "design cell out of range");
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    const int64_t o = (int64_t)y * g.pitch + x;
    if (slot[o] >= 0) return fail(ctx, GKS_E_ARG, "design cell listed twice");
    slot[o] = (int32_t)i;
    box[0] = std::min(box[0], x); box[1] = std::max(box[1], x);
    box[2] = std::min(box[2], y); box[3] = std::max(box[3], y);
  }
  void *bufs[] = {ctx->probe_off, ctx->probe_w, ctx->probe_box_w, ctx->dslot};
  for (void *b : bufs)
    if (b) GKS_CUDA(cudaFreeAsync(b, ctx->st));
  ctx->probe_off = nullptr; ctx->probe_w = nullptr; ctx->probe_box_w = nullptr; ctx->dslot = nullptr;
  gks_status s;
  if ((s = upload_vec(ctx, off, &ctx->probe_off)) != GKS_OK ||
      (s = upload_vec(ctx, w, &ctx->probe_w)) != GKS_OK ||
      (s = upload_vec(ctx, wbox, &ctx->probe_box_w)) != GKS_OK ||
      (s = upload_vec(ctx, slot, &ctx->dslot)) != GKS_OK)
    return s;
  std::memcpy(ctx->pbox, pbox, sizeof(pbox));
  if (!ctx->obj && (s = alloc_dev(ctx, (void **)&ctx->obj, gks::kObjWords * sizeof(double))) != GKS_OK)
    return s;
  GKS_CUDA(cudaMemsetAsync(ctx->obj, 0, gks::kObjWords * sizeof(double), ctx->st));
  GKS_CUDA(cudaStreamSynchronize(ctx->st));   // the host vectors go out of scope
  ctx->np = np;
  ctx->nd = nd;
  if (nd > 0) {
    ctx->dbox[0] = box[0]; ctx->dbox[1] = box[1] + 1; ctx->dbox[2] = box[2]; ctx->dbox[3] = box[3] + 1;
  } else {
    ctx->dbox[0] = ctx->dbox[1] = ctx->dbox[2] = ctx->dbox[3] = 0;
  }
  return GKS_OK;
}

gks_status gks_objective(gks_ctx *ctx, double *J) {
  if (!ctx) return GKS_E_ARG;
  if (!J) return fail(ctx, GKS_E_ARG, "J is NULL");
  if (!ctx->obj) return fail(ctx, GKS_E_STATE, "gks_set_objective must come first");
  double h[2];
  GKS_CUDA(cudaMemcpyAsync(h, ctx->obj, sizeof(h), cudaMemcpyDeviceToHost, ctx->st));
  gks_status s = check_flag(ctx);
  if (s != GKS_OK) return s;
  *J = h[0];
  return GKS_OK;
}

gks_status gks_state_layout(const gks_ctx *ctx, int64_t *elements, int64_t *bytes) {
  if (!ctx) return GKS_E_ARG;
  const int64_t n = (int64_t)ctx->ncomp * ctx->g.cstride;
  if (elements) *elements = n;
  if (bytes) *bytes = n * (int64_t)ctx->esize;
  return GKS_OK;
}

gks_status gks_copy_state(gks_ctx *ctx, void *dst) {
  if (!ctx) return GKS_E_ARG;
  if (!dst) return fail(ctx, GKS_E_ARG, "dst is NULL");
  GKS_CUDA(cudaMemcpyAsync(dst, ctx->V[ctx->cur], ctx->esize * ctx->ncomp * (size_t)ctx->g.cstride,
                           cudaMemcpyDeviceToDevice, ctx->st));
  return GKS_OK;
}

gks_status gks_load_state(gks_ctx *ctx, const void *src, int64_t step) {
  if (!ctx) return GKS_E_ARG;
  if (!src || step < 0) return fail(ctx, GKS_E_ARG, "src is NULL or step < 0");
  GKS_CUDA(cudaMemcpyAsync(ctx->V[ctx->cur], src, ctx->esize * ctx->ncomp * (size_t)ctx->g.cstride,
                           cudaMemcpyDeviceToDevice, ctx->st));
  ctx->step = step;
  ctx->fields_written = true;
  return GKS_OK;
}

gks_status gks_adjoint_seed(gks_ctx *ctx, const void *state, void *adj) {
  if (!ctx) return GKS_E_ARG;
  if (!state || !adj) return fail(ctx, GKS_E_ARG, "state / adj is NULL");
  if (!ctx->obj) return fail(ctx, GKS_E_STATE, "gks_set_objective must come first");
  GKS_CUDA(cudaMemsetAsync(adj, 0, ctx->esize * ctx->ncomp * (size_t)ctx->g.cstride, ctx->st));
  GKS_CUDA(gks::launch_probe_grad(state, adj, ctx->probe_off, ctx->probe_w, ctx->np, ctx->dt, true,
                                  ctx->fp64, ctx->st));
  return GKS_OK;
}

gks_status gks_adjoint_step(gks_ctx *ctx, const void *state_n, const void *state_np1,
                            const void *adj_in, void *adj_out, double *grad_eps,
                            int32_t add_probe) {
  if (!ctx) return GKS_E_ARG;
  if (ctx->kind != GKS_CARTESIAN || ctx->dim != 2)
    return fail(ctx, GKS_E_UNSUPPORTED, "the adjoint needs a 2-D Cartesian grid");
  if (ctx->mu) return fail(ctx, GKS_E_UNSUPPORTED, "the adjoint supports mu = 1 only");
  if (ctx->phm) return fail(ctx, GKS_E_UNSUPPORTED, "the adjoint does not cover divergence cleaning");
  if (ctx->limiter)
    return fail(ctx, GKS_E_UNSUPPORTED, "the limited step is not linear: no adjoint");
  if (ctx->slab)
    return fail(ctx, GKS_E_UNSUPPORTED, "the adjoint step runs on a whole grid, not on a slab");
  for (int k = 0; k < 4; ++k)
    if (ctx->g.pec[k])
      return fail(ctx, GKS_E_UNSUPPORTED, "the adjoint supports periodic and non-reflecting sides only");
  if (!adj_in || !adj_out || adj_in == adj_out) return fail(ctx, GKS_E_ARG, "adj_in / adj_out");
  if (ctx->nd > 0 && (!grad_eps || !state_n || !state_np1))
    return fail(ctx, GKS_E_ARG, "the eps-gradient needs both states and grad_eps");
  if (add_probe && ctx->np > 0 && !state_n) return fail(ctx, GKS_E_ARG, "state_n is NULL");
  gks::AdjointArgs a;
  a.lam_in = adj_in;
  a.lam_out = adj_out;
  a.eps = ctx->eps;
  a.Vn = state_n;
  a.Vn1 = state_np1;
  a.dslot = ctx->dslot;
  a.grad = ctx->nd > 0 ? grad_eps : nullptr;
  std::memcpy(a.dbox, ctx->dbox, sizeof(a.dbox));
  std::memcpy(a.C, ctx->C, sizeof(a.C));
  a.c = ctx->c;
  a.probe_w = add_probe && ctx->np > 0 ? ctx->probe_box_w : nullptr;
  std::memcpy(a.pbox, ctx->pbox, sizeof(a.pbox));
  a.dt = ctx->dt;
  GKS_CUDA(gks::launch_adjoint_step(ctx->g, a, ctx->fp64, ctx->st));
  ctx->launches += a.grad && ctx->dbox[1] > ctx->dbox[0] ? 2 : 1;
  return GKS_OK;
}

gks_status gks_get_info(const gks_ctx *ctx, double *dt, double *t, int64_t *step,
                        int64_t *n_cells, double *c_lattice) {
  if (!ctx) return GKS_E_ARG;
  if (dt) *dt = ctx->dt;
  if (t) *t = ctx->t0 + (double)ctx->step * ctx->dt;
  if (step) *step = ctx->step;
  if (n_cells) *n_cells = ctx->ncell;
  if (c_lattice) *c_lattice = ctx->c;
  return GKS_OK;
}

gks_status gks_get_launch_count(const gks_ctx *ctx, int64_t *launches) {
  if (!ctx || !launches) return GKS_E_ARG;
  *launches = ctx->launches;
  return GKS_OK;
}

const char *gks_last_error(const gks_ctx *ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

void gks_destroy(gks_ctx *ctx) {
  if (!ctx) return;
  const gks::TetDev &t = ctx->tet;
  void *bufs[] = {ctx->V[0], ctx->V[1], ctx->eps, ctx->mu, ctx->src, ctx->flag, ctx->red,
                  ctx->staging, t.perm, t.vol, t.cnb, t.cface, t.fL, t.fR, t.fgeo, t.cw, t.cu,
                  t.Gscratch, t.Fscratch, ctx->probe_off, ctx->probe_w, ctx->probe_box_w,
                  ctx->dslot, ctx->obj};
  for (void *p : bufs)
    if (p) cudaFreeAsync(p, ctx->st);
  cudaStreamSynchronize(ctx->st);
  delete ctx;
}

}  // extern "C"
