/*
 * gks.h -- C ABI of the GB300 (sm_103a) gas-kinetic scheme (GKS) for Maxwell's equations.
 *
 * Method: Pu, Long & Xu, "A Gas-Kinetic Scheme for Maxwell Equations" (arXiv 2412.16845).
 * One call of gks_step advances the cell averages by the finite-volume update of Sec. 3.1,
 *     U_i^{n+1} = U_i^n - dt/|Omega_i| sum_s |l_s| F_s + dt S_i^n,
 * where every interface flux F_s is the time-integrated GKS flux of Sec. 3.1 (D3Q4 / D2Q4
 * equilibrium, upwind interface equilibrium, compatibility time derivative, coefficients
 * C1..C5), evaluated in the face frame T' of Sec. 3.1, with the kinetic non-reflecting boundary
 * of Sec. 3.1 (incoming distributions of ghost cells are zero).
 *
 * Conventions shared by every entry point
 *  - Fields: 2-D TM carries (Ez, Hx, Hy); 3-D carries (Ex, Ey, Ez, Hx, Hy, Hz).  With divergence
 *    cleaning (gks_mesh_desc.chi, gamma) psi follows in 2-D, (phi, psi) in 3-D.  The library
 *    stores the primitive state V = (E, H[, phi, psi]); the conserved state is
 *    U = (eps E, mu H[, phi, psi]).
 *    Units: c = eps0 = mu0 = 1 (Sec. 5) unless a lattice speed is given.
 *  - User order: host arrays are [ncomp][n_cells] in user cell order.  Cartesian cells are
 *    numbered x fastest (i + nx*(j + ny*k)); tetrahedra in the order of tet_vert.  Internal
 *    layouts (padded rows, reordered cells) never show at the API.
 *  - Ownership: host arrays passed in are copied before the call returns; the caller keeps
 *    them.  Device buffers of the context are owned by the context and freed by gks_destroy.
 *    Device pointers passed in (adjoint buffers) stay owned by the caller.
 *  - Errors: every call returns a gks_status; no call aborts, traps or throws.  Arguments are
 *    validated before anything is enqueued.  Asynchronous device errors and the non-finite
 *    flag surface at the next call that synchronises (gks_read_fields, gks_energy,
 *    gks_objective, gks_sync).  gks_last_error() gives a one-line reason.
 *  - Streams: all device work of a context is enqueued on the stream given at creation
 *    (cudaStream_t as void*, NULL = the legacy default stream).  A context is not re-entrant:
 *    one host thread at a time.
 */
#ifndef GKS_H
#define GKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gks_ctx gks_ctx;

typedef enum gks_status {
  GKS_OK = 0,
  GKS_E_ARG = 1,          /* invalid argument (null pointer, bad size, eps <= 0, ...)     */
  GKS_E_NOMEM = 2,        /* device or host allocation failed                              */
  GKS_E_CUDA = 3,         /* a CUDA runtime call failed                                    */
  GKS_E_UNSUPPORTED = 4,  /* valid but not implemented combination                         */
  GKS_E_STATE = 5,        /* call out of order (e.g. step before fields were written)      */
  GKS_E_NONFINITE = 6,    /* a non-finite value appeared in the state                      */
  GKS_E_TIMEOUT = 7       /* a bounded wait ran out                                        */
} gks_status;

enum { GKS_CARTESIAN = 0, GKS_TET = 1 };
enum { GKS_FP32 = 0, GKS_FP64 = 1 };
enum { GKS_BC_PERIODIC = 0, GKS_BC_NONREFLECTING = 1, GKS_BC_PEC = 2 };
enum { GKS_LIMITER_NONE = 0, GKS_LIMITER_VAN_LEER = 1 };

/* Problem description (Sec. 3.1: cells Omega_i, faces l_s with normals n_s).
 *  dim        2 => TM (Ez, Hx, Hy) on an (x, y) grid; 3 => full Maxwell.
 *  kind       GKS_CARTESIAN, or GKS_TET (requires dim == 3).
 *  precision  GKS_FP32 or GKS_FP64: storage of the state and the flux/update arithmetic.
 *  n, lo, hi  Cartesian cells per axis and box (n[2] ignored in 2-D).
 *  bc         per side -x,+x,-y,+y,-z,+z: GKS_BC_PERIODIC (sides paired),
 *             GKS_BC_NONREFLECTING (kinetic boundary of Sec. 3.1) or GKS_BC_PEC (perfect
 *             electric conductor wall, Sec. 5.5: tangential E and normal B vanish, normal E and
 *             tangential H have zero normal derivative; a mirror ghost cell).  A PEC axis needs
 *             at least 2 cells.
 *  vert_xyz   tets: [n_vert][3] doubles (host, copied).
 *  tet_vert   tets: [n_tet][4] int64 vertex ids (host, copied), any orientation.
 *  tet_bc     tets: boundary kind of every face that belongs to one tet only
 *             (GKS_BC_NONREFLECTING or GKS_BC_PEC).
 *  cfl        dt = cfl * h_min / c, h_i = 2 dim |Omega_i| / sum_s |l_s| (edge of a square/cube).
 *  tau_over_dt  kappa = tau/dt of the BGK relaxation time (Sec. 2.2, eq. of the vector BGK
 *             model); 0 selects the tau -> 0 limit coefficients of Sec. 4.1.
 *  c_lattice  lattice speed c of the D3Q4 velocities (Sec. 2.2); <= 0 selects
 *             max_i 1/sqrt(eps_i mu_i) at gks_set_materials (1 in vacuum).
 *  cuda_stream  cudaStream_t of all device work of this context.
 *  chi, gamma   divergence cleaning (the PHM system of Sec. 2.1): correction potentials phi,
 *             psi carry div E and div B errors away at speeds chi c and gamma c.  0 and 0 is
 *             plain Maxwell.  Supported on Cartesian grids with mu = 1 and no adjoint
 *             (GKS_E_UNSUPPORTED otherwise).  2-D TM: the fields become (Ez, Hx, Hy, psi);
 *             chi has no effect there, E being divergence free.  3-D: the fields become
 *             (Ex, Ey, Ez, Hx, Hy, Hz, phi, psi).  With cleaning the step is stable only at
 *             smaller CFL numbers (about 0.4 in 2-D and 0.3 in 3-D for chi, gamma <= 1 at
 *             lattice speed 1).
 *  limiter    GKS_LIMITER_NONE (central-difference cell gradients, the scheme of Sec. 3.1) or
 *             GKS_LIMITER_VAN_LEER: each component's slope along each axis is van Leer's
 *             harmonic mean of its one-sided differences, 0 at extrema, so the step drops to
 *             first order at discontinuities and stays second order in smooth regions (the
 *             limited scheme of Sec. 5.3, whose limiter the paper does not name).
 *             Cartesian grids; GKS_E_UNSUPPORTED on tets.  The limited step is not linear in
 *             the state: the adjoint rejects it.  Other values: GKS_E_ARG.               */
typedef struct gks_mesh_desc {
  int32_t dim;
  int32_t kind;
  int32_t precision;
  int32_t reserved0;
  int64_t n[3];
  double lo[3];
  double hi[3];
  int32_t bc[6];
  int64_t n_vert;
  const double *vert_xyz;
  int64_t n_tet;
  const int64_t *tet_vert;
  int32_t tet_bc;
  int32_t reserved1;
  double cfl;
  double tau_over_dt;
  double c_lattice;
  void *cuda_stream;
  double chi;
  double gamma;
  int32_t limiter;
  int32_t reserved2;
} gks_mesh_desc;

/* Build the geometry (Sec. 3.1: |Omega_i|, |l_s|, n_s, face and cell centroids; T'(n_s) on
 * tets), allocate the state (zero fields, eps = mu = 1) and compute dt and C1..C5.
 * *out receives a new context, or NULL on error.  GKS_E_ARG on an invalid description,
 * GKS_E_NOMEM / GKS_E_CUDA on allocation failure. */
gks_status gks_create_mesh(const gks_mesh_desc *d, gks_ctx **out);

/* Per-cell material eps, mu ([n_cells] doubles, user order, all > 0 and finite; mu == NULL
 * means mu = 1).  The paper has no materials (Sec. 5 uses vacuum); the library uses
 * U = (eps E, mu H) and the interface equilibrium M_s = (M_L + M_R)/2, which reduces to the
 * paper's scheme for eps = mu = 1.  Recomputes the lattice speed (c_lattice <= 0), dt and
 * C1..C5. */
gks_status gks_set_materials(gks_ctx *ctx, const double *eps, const double *mu);

/* Replace eps on the box of columns [x0, x1) x rows [y0, y1) of a 2-D Cartesian grid by eps_box
 * (row-major, (y1 - y0) x (x1 - x0) doubles, host, copied; finite and > 0); the rest of eps and
 * mu stay.  For design loops that change only a region (the update of Sec. 3.1 divides by
 * eps per cell).  Needs a fixed lattice speed (c_lattice > 0 at creation), because dt and C1..C5
 * are kept: GKS_E_STATE otherwise.  GKS_E_UNSUPPORTED on other meshes. */
gks_status gks_set_materials_box(gks_ctx *ctx, int64_t x0, int64_t x1, int64_t y0, int64_t y1,
                                 const double *eps_box);

/* Upload the primitive fields V = (E, H) ([ncomp][n_cells] doubles, user order, host) and set
 * the time to t0 and the step counter to 0.  Converted to the context precision. */
gks_status gks_write_fields(gks_ctx *ctx, const double *fields, double t0);

/* Current-density source of Sec. 2.1, S = (-J, 0), with J = (0, 0, J_z) and
 *     J_z(x_i, t) = jz_mask[i] * A * exp(-((t - t0)/s)^2) * sin(2 pi f0 (t - t0)),
 * evaluated explicitly at t^n.  jz_mask: [n_cells] doubles, user order, or NULL to remove the
 * source.  s must be > 0. */
gks_status gks_set_source(gks_ctx *ctx, const double *jz_mask, double A, double f0, double t0,
                          double s);

/* Continuous-wave current source of the oscillating-dipole workloads (Sec. 5.4), S = (-J, 0):
 *     J_z(x_i, t) = jz_mask[i] * A * cos(2 pi f0 (t - t0))  for t >= t0, 0 before,
 * evaluated explicitly at t^n (the paper's J_z = J_0 cos(2 pi t / T) is A = J_0, f0 = 1/T,
 * t0 = 0).  jz_mask: [n_cells] doubles, user order, or NULL to remove the source.  Replaces a
 * source set by gks_set_source. */
gks_status gks_set_source_cw(gks_ctx *ctx, const double *jz_mask, double A, double f0, double t0);

/* Override dt (> 0) and recompute C1..C5; used to land exactly on a final time. */
gks_status gks_set_dt(gks_ctx *ctx, double dt);

/* Enqueue n_steps >= 0 GKS steps (Sec. 3.1) on the context stream; asynchronous. */
gks_status gks_step(gks_ctx *ctx, int64_t n_steps);

/* Enqueue n_steps steps that advance only the cells of the window [x0, x1) x [y0, y1) (2-D
 * Cartesian grids).  Cells outside the window keep stale values, which act on the window's
 * cells after one step through the stencil (radius two cells): after k windowed steps only the
 * cells at least 2k cells inside the window are exact.  Used to recompute a region's domain of
 * dependence from a checkpoint (adjoint).  Time and step counter advance as in gks_step; the
 * probe objective is not accumulated. */
gks_status gks_step_window(gks_ctx *ctx, int64_t n_steps, int64_t x0, int64_t x1, int64_t y0,
                           int64_t y1);

/* Wait for the stream, then copy the fields to out ([ncomp][n_cells] doubles, user order,
 * host).  GKS_E_NONFINITE if a step produced a non-finite value, GKS_E_TIMEOUT if a staged
 * kernel's bounded wait for its tensor copies ran out. */
gks_status gks_read_fields(gks_ctx *ctx, double *out);

/* Electromagnetic energy 1/2 sum_i |Omega_i| (eps_i |E_i|^2 + mu_i |H_i|^2), accumulated in
 * FP64 on the device; synchronises.  With divergence cleaning the potentials' 1/2 |Omega_i|
 * (phi_i^2 + psi_i^2) is added (the quantity the cleaning system conserves between walls).
 * (Not in the paper: a diagnostic.) */
gks_status gks_energy(gks_ctx *ctx, double *out);

/* Probe objective and design region for the adjoint (2-D TM Cartesian grids; not in the
 * paper).  After every gks_step the device accumulates, in FP64 with Kahan compensation,
 *     J = sum_{n >= 1} dt sum_{i in probe} |Omega_i| Ez_i^n^2
 * (reset by gks_write_fields).  probe: [np] user cell ids; design: [nd] user cell ids, the
 * cells whose eps the gradient is taken with respect to (slot k = design[k]).  Host arrays,
 * copied.  GKS_E_UNSUPPORTED on tets or 3-D grids, GKS_E_ARG on ids out of range or repeated. */
gks_status gks_set_objective(gks_ctx *ctx, const int64_t *probe, int64_t np,
                             const int64_t *design, int64_t nd);

/* Set the accumulated objective J (and its compensation) back to zero, for a run restarted with
 * gks_load_state; asynchronous.  GKS_E_STATE before gks_set_objective. */
gks_status gks_reset_objective(gks_ctx *ctx);

/* Wait for the stream and return the accumulated objective J.  GKS_E_STATE before
 * gks_set_objective. */
gks_status gks_objective(gks_ctx *ctx, double *J);

/* Size of one state buffer in the context's internal layout (ncomp * padded cells) in elements
 * of the context precision and in bytes.  Checkpoints and adjoint buffers use this layout. */
gks_status gks_state_layout(const gks_ctx *ctx, int64_t *elements, int64_t *bytes);

/* Device-to-device copy of the current state into dst (caller-owned, gks_state_layout bytes);
 * asynchronous on the context stream. */
gks_status gks_copy_state(gks_ctx *ctx, void *dst);

/* Copy only the box of columns [x0, x1) and rows [y0, y1) (row index y + ny*z) of every
 * component of the current state into dst at the same offsets of the internal layout (device,
 * gks_state_layout bytes; entries outside the box are left as they are); asynchronous.
 * GKS_E_ARG for an empty box or one outside the grid. */
gks_status gks_copy_state_box(gks_ctx *ctx, void *dst, int64_t x0, int64_t x1, int64_t y0,
                              int64_t y1);

/* Replace the current state by src (device, internal layout) and set the step counter, so that
 * the time is t0 + step * dt (checkpoint restart); asynchronous. */
gks_status gks_load_state(gks_ctx *ctx, const void *src, int64_t step);

/* adj = dq/dV(state) for q(V) = dt sum_probe |Omega| Ez^2: the adjoint of the final step of J.
 * state, adj: device, internal layout. */
gks_status gks_adjoint_seed(gks_ctx *ctx, const void *state, void *adj);

/* One step of the discrete adjoint of gks_step (hand-transposed fused stencil; not in the
 * paper): adj_out = L^T adj_in (+ dq/dV(state_n) if add_probe), and
 * grad_eps[k] += dV^{n+1}/d eps_{design[k]} . adj_in, with V^{n+1} = L(eps) V^n + s^n.
 * state_n = V^n, state_np1 = V^{n+1} (device, internal layout; needed on the design cells and
 * the probe), adj_in = lambda^{n+1}, adj_out = lambda^n (distinct device buffers),
 * grad_eps: device [nd] doubles.  2-D TM, mu = 1.  Asynchronous. */
gks_status gks_adjoint_step(gks_ctx *ctx, const void *state_n, const void *state_np1,
                            const void *adj_in, void *adj_out, double *grad_eps,
                            int32_t add_probe);

/* ---- Domain split across ranks (one process per GPU).  The finite-volume update of Sec. 3.1
 * reaches two cells along every axis (the Green-Gauss gradient of Sec. 3.1, then the face flux
 * between two reconstructed cells), so a grid split into slabs along its slowest axis (y in
 * 2-D, z in 3-D) advances exactly like the whole grid when every rank also holds the two
 * layers of cells beyond each side it shares with another rank (ghost layers) and those layers
 * are refreshed from the neighbour after every step. */

/* Cells [begin, end) of the slowest axis owned by this rank; shared_lo (shared_hi) = 1 when the
 * side below begin (at end) borders another rank, 0 when it is the grid's own boundary.  A
 * periodic axis split over several ranks is a ring: both sides shared. */
typedef struct gks_slab_desc {
  int64_t begin;
  int64_t end;
  int32_t shared_lo;
  int32_t shared_hi;
} gks_slab_desc;

enum { GKS_HALO_OWNED = 0, GKS_HALO_GHOST = 1 };

/* Rank-local context for the slab `slab` of the grid `global` (a Cartesian description as for
 * gks_create_mesh; c_lattice must be > 0 so that every rank steps with the same dt and C1..C5).
 * The local grid is the owned layers plus two ghost layers beyond each shared side: along the
 * slab axis it covers the global cells begin - 2 shared_lo .. end + 2 shared_hi - 1 (wrapped on
 * a periodic axis).  Every user-order array of this context (materials, fields, source mask,
 * probe cells) covers the local grid, x fastest, starting at that first layer.  The cell size,
 * dt and C1..C5 are those of the global grid.  gks_energy sums owned cells only; the adjoint
 * calls return GKS_E_UNSUPPORTED on a slab.  GKS_E_ARG when the slab does not fit the grid, a
 * shared side owns fewer than two layers, a non-periodic grid edge is marked shared, or a
 * periodic axis has one shared side only. */
gks_status gks_create_slab(const gks_mesh_desc *global, const gks_slab_desc *slab,
                           gks_ctx **out);

/* Bytes of one side's halo buffer: ncomp components x 2 layers of the state layout. */
gks_status gks_halo_bytes(const gks_ctx *ctx, int64_t *bytes);

/* Copy two layers of `state` (device, this context's layout; NULL = the context's own current
 * state) next to side 0 (low) or 1 (high) into the caller's device buffer buf
 * (gks_halo_bytes): layers = GKS_HALO_OWNED the two owned layers at that side,
 * GKS_HALO_GHOST the two ghost layers beyond it; increasing global index order.  Asynchronous
 * on the context's stream.  GKS_E_ARG if the side is not shared. */
gks_status gks_halo_export(gks_ctx *ctx, int32_t side, int32_t layers, const void *state,
                           void *buf);

/* The reverse: write (add = 0) or add (add = 1) buf into the two layers of `state` (NULL = the
 * context's state) chosen as in gks_halo_export.  After each step a rank exports its owned
 * layers to each neighbour, which imports them into its ghost layers (add = 0): rank r's high
 * owned layers are rank r+1's low ghost layers.  The transpose of that copy, for adjoint
 * fields, exports ghost layers and adds them into the neighbour's owned layers (add = 1).
 * Asynchronous on the context's stream. */
gks_status gks_halo_import(gks_ctx *ctx, int32_t side, int32_t layers, void *state,
                           const void *buf, int32_t add);

/* Energy 1/2 |Omega| sum_i (eps_i |E_i|^2 + mu_i |H_i|^2) of caller-owned device arrays, for
 * callers that cannot allocate device memory (a framework that reserved the device memory for
 * its own pool, a hot loop that cannot pay for an allocation, or code without a gks context).
 * The paper has no counterpart; it is a variant of the reduction behind gks_energy.
 *  precision    GKS_FP32 or GKS_FP64: element type of fields, eps and mu.
 *  dim          2 (fields = Ez, Hx, Hy) or 3 (Ex, Ey, Ez, Hx, Hy, Hz).
 *  n_cells      1 .. 33,554,432 cells; larger sizes return GKS_E_ARG (the fixed scratch holds
 *               one partial sum per 4096 cells, 8192 partials).
 *  cell_volume  |Omega| of every cell (> 0).
 *  fields       device, [ncomp][n_cells], contiguous; eps, mu device [n_cells] (mu NULL: 1).
 *  out          device pointer to one double, overwritten with the energy.
 *  cuda_stream  stream the two kernels are enqueued on (asynchronous; no synchronisation).
 * Allocates nothing: the partial sums live in a fixed device array of 64 KiB that every GPU
 * loading the library keeps until the process exits.  Every call looks up that array's device
 * address on the current device (a host-side lookup, so a device reset leaves no stale address);
 * the first call on a device also loads the library's device code there, so make it before any
 * stream capture.  All calls share the array, so calls that overlap on the GPU (on different
 * streams) race; serialise them.  GKS_E_ARG on bad arguments; GKS_E_CUDA on a launch error, and
 * (without launching) when an earlier CUDA error is still pending on the calling thread, which
 * is left in place for the work that caused it. */
gks_status gks_energy_noalloc(int32_t precision, int32_t dim, int64_t n_cells, double cell_volume,
                              const void *fields, const void *eps, const void *mu, double *out,
                              void *cuda_stream);

/* Wait for all enqueued work; report asynchronous errors and the non-finite flag. */
gks_status gks_sync(gks_ctx *ctx);

/* dt, current time, steps taken since the last gks_write_fields, cells, and the lattice c. */
gks_status gks_get_info(const gks_ctx *ctx, double *dt, double *t, int64_t *step,
                        int64_t *n_cells, double *c_lattice);

/* Number of kernels this context has launched since it was created (a diagnostic for
 * benchmarks; not in the paper). */
gks_status gks_get_launch_count(const gks_ctx *ctx, int64_t *launches);

/* One-line reason of the last failed call on this context (never NULL). */
const char *gks_last_error(const gks_ctx *ctx);

/* Free every device and host resource of the context (NULL is ignored). */
void gks_destroy(gks_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* GKS_H */
