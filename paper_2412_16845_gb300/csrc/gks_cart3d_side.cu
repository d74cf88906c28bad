// Fused 3-D GKS step on a Cartesian grid in FP32 with mu = 1 (Sec. 3.1): the side-split face
// flux of gks_side3.cuh, paired FP32 arithmetic, planes staged in shared memory.
//
// Flux.  Through the face between cells L and R along axis A the time-integrated flux is
// F = P^l_L + P^r_R + ie (Q^l_L + Q^r_R), ie = 2/(eps_L + eps_R), where the four vectors of a
// cell depend on that cell alone (its state, raw central differences and eps).  A cell computes
// them once per axis; faces combine two cells' vectors.  Non-reflecting faces (Sec. 3.1, last
// paragraph) take zero vectors for the ghost and ie = 1/eps of the cell (the ghost's eps is the
// cell's, through the clamped loads that also give the Green-Gauss ghost copy).
//
// Layout of the work.  A CTA owns 64 columns x NWO rows of a chunk of z-planes.  Each of its
// NWO row warps holds two adjacent cells per lane (columns X0 + 2l, X0 + 2l + 1) as the two
// halves of a float2, so every flux term of both cells is one paired FP32 instruction
// (__ffma2_rn etc.).  Two halo warps complete the tile: H0 owns the row below, H1 the row
// above; they supply the y-face vectors of those rows and, one plane ahead, the x-face vectors
// of the columns left and right of the tile.  Per plane:
//   - x: the right cell's r-side vectors come from the next lane (shuffle), the flux of a lane's
//     left face from the previous lane;
//   - z: the l-side vectors of the plane below stay in registers (march along z), so the face
//     below the plane completes the update of the plane below;
//   - y: every row publishes its r-side vectors in shared memory, forms the face above it and
//     publishes that flux for the row above (two barriers).
// Planes arrive by TMA (cp.async.bulk.tensor) into five shared-memory slots, one plane per slot:
// one thread issues the two tensor copies of plane k+4 (the six fields as one 4-D box, eps as a
// 3-D box) when plane k starts; they complete on the slot's mbarrier, which every thread waits
// for one plane later, so a whole plane of work hides the latency.  Boxes reaching past the
// grid are zero-filled by the copy; in CTAs at the grid's edge the halo warps then write the
// wrapped or clamped values into those entries (the periodic neighbour, or the copy of the
// edge cell that the non-reflecting Green-Gauss ghost takes).
#include <cuda_runtime.h>

#include "gks_internal.h"
#include "gks_side3.cuh"
#include "gks_tma.cuh"

namespace gks {
namespace {

constexpr int NWO = 10;                 // row warps per CTA
constexpr int NWARP = NWO + 2;          // plus the halo warps H0 (below) and H1 (above)
constexpr int NTH = NWARP * 32;
constexpr int TCOLS = 64;               // columns per CTA (two per lane)
constexpr int TW = 72;                  // staged columns X0-4 .. X0+67 (16-byte chunks)
constexpr int NR = NWO + 4;             // staged rows y0-2 .. y0+NWO+1
constexpr int NA = 7;                   // staged arrays: Ex, Ey, Ez, Hx, Hy, Hz, eps
constexpr int NSLOT = 5;
constexpr unsigned FULL = 0xffffffffu;
// wrapped entries of a staged plane on periodic sides: two layers beyond each side, every row
// for columns and every column for rows, all arrays
constexpr int kMaxFix = NA * (4 * NR + 4 * TW);

using f2 = float2;

// Paired FP32 arithmetic (two cells per value).  A coefficient k is a scalar kernel parameter
// replicated into both halves: the paired FMA then reads it straight from the constant bank,
// whereas a float2 parameter costs an extra instruction per use.
struct OpP {
  static __device__ __forceinline__ f2 mul(float k, f2 x) { return __fmul2_rn(make_float2(k, k), x); }
  static __device__ __forceinline__ f2 fma(float k, f2 x, f2 a) {
    return __ffma2_rn(make_float2(k, k), x, a);
  }
  static __device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ f2 sub(f2 a, f2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
  }
  static __device__ __forceinline__ f2 neg(f2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
  static __device__ __forceinline__ f2 zero() { return make_float2(0.f, 0.f); }
};
struct OpS {                            // scalar FP32 arithmetic
  static __device__ __forceinline__ float mul(float k, float x) { return k * x; }
  static __device__ __forceinline__ float fma(float k, float x, float a) { return fmaf(k, x, a); }
  static __device__ __forceinline__ float add(float a, float b) { return a + b; }
  static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
  static __device__ __forceinline__ float neg(float a) { return -a; }
  static __device__ __forceinline__ float zero() { return 0.f; }
};

__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return OpP::sub(a, b); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 pfma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 pk(float a, float b) { return make_float2(a, b); }
// 2 / s (the interface 1/eps_s), fast FP32 division (about 1 ulp), as the other FP32 kernels
__device__ __forceinline__ f2 two_over(f2 s) { return pk(__fdividef(2.f, s.x), __fdividef(2.f, s.y)); }

struct Side3Args {
  const float *__restrict__ V;
  float *__restrict__ Vout;
  const float *__restrict__ eps;
  const float *__restrict__ src;
  int sx0, sx1, sy0, sy1, sz0, sz1;
  float src_amp;
  int nx, ny, nz;
  int64_t pitch, plane, cstride;
  int per[3];
  int zchunk;
  int *flag;
  float k[3][kSide3K];                 // coefficient slots of the x-, y- and z-faces
};

// One staged plane in the TMA box order (array, row, column); slots start 128-byte aligned.
struct alignas(128) PlaneSlot {
  float a[NA][NR][TW];
};

struct SideSmem {
  PlaneSlot V[NSLOT];                  // staged planes
  unsigned long long bar[NSLOT];       // one mbarrier per slot
  int err;                             // a bounded wait ran out (shared by the CTA)
  f2 Y[NWO + 1][11][32];               // r-side y-vectors of each row (P 6, Q without Ey 5)
  f2 F[NWO + 1][6][32];                // flux through the face above each row; [NWO]: below row 0
  float XL[2][NWO][12];                // l-side x-vectors of column X0-1 (P 6, Q without Ex, eps)
  float XR[2][NWO][12];                // r-side x-vectors of column X0+64
  // periodic sides: staged entries past the grid that hold wrapped cells (the TMA box leaves
  // them zero): position in a plane slot (array, row, column) and source offset in a plane
  unsigned short fixd[kMaxFix];
  int fixg[kMaxFix];
  int nfix;
  unsigned tmem;                       // tensor-memory base of the CTA (tcgen05.alloc)
};

__device__ __forceinline__ int wrap_or_clamp(int i, int n, int periodic) {
  if (periodic) {
    i %= n;
    return i < 0 ? i + n : i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

constexpr unsigned kPlaneBytes = NA * NR * TW * 4;   // one staged plane (both tensor boxes)

// Tensor memory as spill space.  Each row warp keeps the l-side z-vectors of the plane below
// (24 values per thread, from one plane to the next) in its lane quarter of the SM's tensor
// memory instead of registers: one tcgen05 store and one load per plane replace the
// registers they would pin through the x- and y-face work.  No tensor-core instruction is
// issued; the memory is only written and read back by the thread that owns each lane.
constexpr unsigned kTmemCols = 128;                 // 3 row warps per lane quarter x 24 columns

__device__ __forceinline__ void tmem_st24(unsigned ta, const f2 a[6], const f2 b[6]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};\n" ::"r"(ta),
      "f"(a[0].x), "f"(a[0].y), "f"(a[1].x), "f"(a[1].y), "f"(a[2].x), "f"(a[2].y), "f"(a[3].x),
      "f"(a[3].y), "f"(a[4].x), "f"(a[4].y), "f"(a[5].x), "f"(a[5].y), "f"(b[0].x), "f"(b[0].y),
      "f"(b[1].x), "f"(b[1].y)
      : "memory");
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(ta + 16),
      "f"(b[2].x), "f"(b[2].y), "f"(b[3].x), "f"(b[3].y), "f"(b[4].x), "f"(b[4].y), "f"(b[5].x),
      "f"(b[5].y)
      : "memory");
}
__device__ __forceinline__ void tmem_ld24(unsigned ta, f2 a[6], f2 b[6]) {
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      : "=f"(a[0].x), "=f"(a[0].y), "=f"(a[1].x), "=f"(a[1].y), "=f"(a[2].x), "=f"(a[2].y),
        "=f"(a[3].x), "=f"(a[3].y), "=f"(a[4].x), "=f"(a[4].y), "=f"(a[5].x), "=f"(a[5].y),
        "=f"(b[0].x), "=f"(b[0].y), "=f"(b[1].x), "=f"(b[1].y)
      : "r"(ta)
      : "memory");
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=f"(b[2].x), "=f"(b[2].y), "=f"(b[3].x), "=f"(b[3].y), "=f"(b[4].x), "=f"(b[4].y),
        "=f"(b[5].x), "=f"(b[5].y)
      : "r"(ta + 16)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// One thread: the tensor copies of plane gz into slot `slot` (fields box, then eps box), both
// completing on the slot's mbarrier.  Earlier generic-proxy reads of the slot are ordered before
// the copies by the CTA barrier that precedes the call and the proxy fence here.
__device__ __forceinline__ void tma_plane(SideSmem &s, const CUtensorMap *tmV,
                                          const CUtensorMap *tmE, int slot, int x, int y,
                                          int gz) {
  unsigned long long *b = &s.bar[slot];
  fence_proxy_async();
  mbar_expect_tx(b, kPlaneBytes);
  tma_load_4d(&s.V[slot].a[0][0][0], tmV, x, y, gz, 0, b);
  tma_load_3d(&s.V[slot].a[6][0][0], tmE, x, y, gz, b);
}

// Periodic sides: the list of staged entries that hold wrapped cells (x = -2, -1, nx, nx+1 on a
// periodic x axis, every row; y = -2, -1, ny, ny+1 on a periodic y axis, every column; all
// arrays).  The tensor copy leaves them zero.  Built once per CTA; non-reflecting sides need no
// entries, their reads are clamped instead.
__device__ __forceinline__ void build_fix_list(SideSmem &s, const Side3Args &a, int X0, int y0,
                                               int tid) {
  unsigned cols = 0, rows = 0;        // up to four tile columns and rows, one byte each
  int nc = 0, nr = 0;
  for (int g = 1; g <= 2; ++g) {
    const int tl = -g - (X0 - 4), th = a.nx - 1 + g - (X0 - 4);
    const int rl = -g - (y0 - 2), rh = a.ny - 1 + g - (y0 - 2);
    if (a.per[0] && tl >= 0 && tl < TW) cols |= (unsigned)tl << (8 * nc++);
    if (a.per[0] && th >= 0 && th < TW) cols |= (unsigned)th << (8 * nc++);
    if (a.per[1] && rl >= 0 && rl < NR) rows |= (unsigned)rl << (8 * nr++);
    if (a.per[1] && rh >= 0 && rh < NR) rows |= (unsigned)rh << (8 * nr++);
  }
  const int n1 = NA * NR * nc, n = n1 + NA * nr * TW;
  for (int i = tid; i < n; i += NTH) {
    int arr, r, t;
    if (i < n1) {
      t = (cols >> (8 * (i % nc))) & 0xff;
      r = (i / nc) % NR;
      arr = i / (nc * NR);
    } else {
      const int j = i - n1;
      t = j % TW;
      r = (rows >> (8 * ((j / TW) % nr))) & 0xff;
      arr = j / (TW * nr);
    }
    const int gx = wrap_or_clamp(X0 - 4 + t, a.nx, a.per[0]);
    const int gy = wrap_or_clamp(y0 - 2 + r, a.ny, a.per[1]);
    s.fixd[i] = (unsigned short)((arr * NR + r) * TW + t);
    s.fixg[i] = gy * (int)a.pitch + gx;
  }
  if (tid == 0) s.nfix = n;
}

// Write the wrapped entries of plane gz into its slot (all threads; four loads in flight each).
__device__ __forceinline__ void fix_plane(SideSmem &s, const Side3Args &a, int slot, int gz,
                                          int tid) {
  const int n = s.nfix;
  float *dst = &s.V[slot].a[0][0][0];
  for (int i0 = tid; i0 < n; i0 += 4 * NTH) {
    float v[4];
    int d[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * NTH;
      d[u] = -1;
      v[u] = 0.f;
      if (i < n) {
        const int dd = s.fixd[i], arr = dd / (NR * TW);
        v[u] = __ldg((arr < 6 ? a.V + arr * a.cstride : a.eps) + (int64_t)gz * a.plane + s.fixg[i]);
        d[u] = dd;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (d[u] >= 0) dst[d[u]] = v[u];
  }
}

// Where a lane reads the staged planes.  On a non-reflecting side the reads are clamped to the
// grid (the Green-Gauss ghost copy), so the zero-filled entries past the grid are never read;
// on a periodic side they are the wrapped entries the fix-up list writes.
struct Taps {
  int r, rm, rp;          // rows of the warp's cells and of their lower / upper neighbours
  int t0, t1;             // columns of the lane's two cells
  int tm, tp;             // left neighbour of the first cell, right neighbour of the second
  bool pair;              // the warp's two cells of every lane are adjacent and aligned
};

// The own pair (both columns of the lane) of one staged row: 6 fields and eps.
__device__ __forceinline__ void load_pair(const SideSmem &s, int slot, const Taps &q, f2 v[7]) {
  if (q.pair) {
#pragma unroll
    for (int m = 0; m < NA; ++m) v[m] = *reinterpret_cast<const f2 *>(&s.V[slot].a[m][q.r][q.t0]);
  } else {
#pragma unroll
    for (int m = 0; m < NA; ++m) v[m] = pk(s.V[slot].a[m][q.r][q.t0], s.V[slot].a[m][q.r][q.t1]);
  }
}

// Raw central differences of the lane's two cells in plane slot s0 (row r, tile column t of
// the first cell), the planes below (vm) and above (vp) in registers; eps-weighted E rows.
__device__ __forceinline__ void differences(const SideSmem &s, int s0, const Taps &q,
                                            const f2 v[7], const f2 vm[7], const f2 vp[7],
                                            f2 d[3][6], f2 ev[3], f2 ed[3][3]) {
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    const float xm = s.V[s0].a[m][q.r][q.tm], xp = s.V[s0].a[m][q.r][q.tp];
    d[0][m] = pk(v[m].y - xm, xp - v[m].x);
    f2 ym, yp;
    if (q.pair) {
      ym = *reinterpret_cast<const f2 *>(&s.V[s0].a[m][q.rm][q.t0]);
      yp = *reinterpret_cast<const f2 *>(&s.V[s0].a[m][q.rp][q.t0]);
    } else {
      ym = pk(s.V[s0].a[m][q.rm][q.t0], s.V[s0].a[m][q.rm][q.t1]);
      yp = pk(s.V[s0].a[m][q.rp][q.t0], s.V[s0].a[m][q.rp][q.t1]);
    }
    d[1][m] = yp - ym;
    d[2][m] = vp[m] - vm[m];
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    ev[m] = v[6] * v[m];
#pragma unroll
    for (int j = 0; j < 3; ++j) ed[j][m] = v[6] * d[j][m];
  }
}

// Scalar x-face vectors of one cell at tile column t, row r of plane slots (sm, s0, sp): the
// columns left and right of the tile, computed by the halo warps.  left: the cell's l-side
// vectors (its face at +1/2), else its r-side vectors.  out: P 6, Q without Ex 5, eps.
__device__ __forceinline__ void halo_x_cell(const SideSmem &s, int sm, int s0, int sp, int r,
                                            int rm, int rp, int t, int tm, int tp,
                                            const float *k, bool left, bool ghost,
                                            float out[12]) {
  float v[6], d[3][6], ev[3], ed[3][3];
  const float e = s.V[s0].a[6][r][t];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    v[m] = s.V[s0].a[m][r][t];
    d[0][m] = s.V[s0].a[m][r][tp] - s.V[s0].a[m][r][tm];
    d[1][m] = s.V[s0].a[m][rp][t] - s.V[s0].a[m][rm][t];
    d[2][m] = s.V[sp].a[m][r][t] - s.V[sm].a[m][r][t];
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    ev[m] = e * v[m];
#pragma unroll
    for (int j = 0; j < 3; ++j) ed[j][m] = e * d[j][m];
  }
  float pl[6], pr[6], ql[6], qr[6];
  side3<0, OpS>(v, d, ev, ed, k, pl, pr, ql, qr);
#pragma unroll
  for (int m = 0; m < 6; ++m) out[m] = ghost ? 0.f : (left ? pl[m] : pr[m]);
#pragma unroll
  for (int m = 1; m < 6; ++m) out[5 + m] = ghost ? 0.f : (left ? ql[m] : qr[m]);
  out[11] = e;
}

__global__ void __launch_bounds__(NTH, 1)
    cart3d_side_kernel(const __grid_constant__ CUtensorMap tmV,
                       const __grid_constant__ CUtensorMap tmE,
                       const __grid_constant__ Side3Args a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SideSmem &s = *reinterpret_cast<SideSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int X0 = blockIdx.x * TCOLS, y0 = blockIdx.y * NWO;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(z0 + a.zchunk, a.nz);
  const bool owned = warp < NWO, h0 = warp == NWO, h1 = warp == NWO + 1;
  const int y = y0 - 2 + (owned ? warp + 2 : (h0 ? 1 : NWO + 2));   // the warp's grid row
  const int x = X0 + 2 * lane;                               // grid column of its first cell
  // non-reflecting ghosts (outside the grid on a non-periodic axis) carry no distributions
  const bool yghost = !a.per[1] && (y < 0 || y >= a.ny);
  const bool xg0 = !a.per[0] && x >= a.nx, xg1 = !a.per[0] && x + 1 >= a.nx;
  const bool st0 = x < a.nx, st1 = x + 1 < a.nx;            // columns this lane stores
  const float *kx = a.k[0], *ky = a.k[1], *kz = a.k[2];
  // read positions: clamped to the grid on non-reflecting sides
  auto trow = [&](int yy) { return (a.per[1] ? yy : min(max(yy, 0), a.ny - 1)) - (y0 - 2); };
  auto tcol = [&](int xx) { return (a.per[0] ? xx : min(max(xx, 0), a.nx - 1)) - (X0 - 4); };
  Taps q;
  q.r = trow(y);
  q.rm = trow(y - 1);
  q.rp = trow(y + 1);
  q.t0 = tcol(x);
  q.t1 = tcol(x + 1);
  q.tm = tcol(x - 1);
  q.tp = tcol(x + 2);
  q.pair = __all_sync(FULL, q.t1 == q.t0 + 1 && (q.t0 & 1) == 0);
  // the halo warps' x-halo cells: row y0 + lane, column X0 - 1 (H0) or X0 + 64 (H1)
  const int hy = y0 + lane;
  const int hr = trow(hy), hrm = trow(hy - 1), hrp = trow(hy + 1);
  const int hx = h0 ? X0 - 1 : X0 + TCOLS;
  const bool hghost = !a.per[0] && (hx < 0 || hx >= a.nx);
  const int ht = tcol(hx), htm = tcol(hx - 1), htp = tcol(hx + 1);

  // ---------------- prologue: planes z0-1 .. z0+2 staged; z-vectors of plane z0-1
  // plane p sits in slot p mod NSLOT; it is that slot's ((p - z0 + 1) / NSLOT)-th load
  auto slot_of = [](int p) { return (p + 2 * NSLOT) % NSLOT; };
  auto parity_of = [z0](int p) { return (unsigned)(((p - z0 + 1) / NSLOT) & 1); };
  auto zidx = [&a](int p) { return wrap_or_clamp(p, a.nz, a.per[2]); };
  const bool issuer = tid == NWO * 32;                       // lane 0 of H0 issues the copies
  const int last_plane = max(z0 + 3, z1 + 1);                // the last plane this CTA loads
  if (tid == 0) {
    for (int i = 0; i < NSLOT; ++i) mbar_init(&s.bar[i], 1);
    s.err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  build_fix_list(s, a, X0, y0, tid);
  __syncthreads();
  if (issuer)
    for (int p = z0 - 1; p <= z0 + 2; ++p)
      tma_plane(s, &tmV, &tmE, slot_of(p), X0 - 4, y0 - 2, zidx(p));
  // own pair at plane z0-2 (wrapped or clamped, always inside the grid), loaded while the
  // staged planes are in flight
  f2 Wm[7];
  {
    const int gz = wrap_or_clamp(z0 - 2, a.nz, a.per[2]);
    const int gy = wrap_or_clamp(y, a.ny, a.per[1]);
    const int c0 = wrap_or_clamp(x, a.nx, a.per[0]), c1 = wrap_or_clamp(x + 1, a.nx, a.per[0]);
    const int64_t o = (int64_t)gz * a.plane + (int64_t)gy * a.pitch;
#pragma unroll
    for (int m = 0; m < NA; ++m) {
      const float *base = (m < 6 ? a.V + m * a.cstride : a.eps) + o;
      Wm[m] = pk(__ldg(base + c0), __ldg(base + c1));
    }
  }
  {
    bool ok = true;
    for (int p = z0 - 1; p <= z0 + 2; ++p) ok &= mbar_wait(&s.bar[slot_of(p)], parity_of(p));
    if (!ok) { s.err = 1; atomicOr(a.flag, 2); }
    for (int p = z0 - 1; p <= z0 + 2; ++p) fix_plane(s, a, slot_of(p), zidx(p), tid);
  }
  __syncthreads();
  if (s.err) return;                                          // nothing else is in flight
  if (issuer) tma_plane(s, &tmV, &tmE, slot_of(z0 + 3), X0 - 4, y0 - 2, zidx(z0 + 3));
  if (warp == NWO + 1) {                                      // H1 owns the tensor memory
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&s.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // this warp's 24 columns in its lane quarter (row warps only)
  const unsigned tz = s.tmem + ((unsigned)(32 * (warp & 3)) << 16) + 24u * (unsigned)(warp >> 2);

  f2 W0[7], Wp[7];                      // own pair at planes k, k+1 (Wm: k-1)
  f2 B[6], Minv = pk(0.f, 0.f);         // pending update of plane k-1: V_new = B - Minv F
  load_pair(s, slot_of(z0 - 1), q, W0);
  load_pair(s, slot_of(z0), q, Wp);
  if (owned) {
    f2 d[3][6], ev[3], ed[3][3], pl[6], pr[6], ql[6], qr[6];
    differences(s, slot_of(z0 - 1), q, W0, Wm, Wp, d, ev, ed);
    side3<2, OpP>(W0, d, ev, ed, kz, pl, pr, ql, qr);
    const bool zg = !a.per[2] && z0 == 0;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      pl[m] = zg ? pk(0.f, 0.f) : pl[m];
      ql[m] = zg ? pk(0.f, 0.f) : ql[m];
      B[m] = pk(0.f, 0.f);
    }
    tmem_st24(tz, pl, ql);                    // l-side z-vectors of plane z0-1
  } else if (lane < NWO) {
    // x-halo vectors of plane z0 (slots z0-1, z0, z0+1)
    float out[12];
    const int sm = slot_of(z0 - 1), s0 = slot_of(z0), sp = slot_of(z0 + 1);
    halo_x_cell(s, sm, s0, sp, hr, hrm, hrp, ht, htm, htp, kx, h0, hghost, out);
    float *dst = h0 ? s.XL[z0 & 1][lane] : s.XR[z0 & 1][lane];
#pragma unroll
    for (int u = 0; u < 12; ++u) dst[u] = out[u];
  }
#pragma unroll
  for (int m = 0; m < NA; ++m) { Wm[m] = W0[m]; W0[m] = Wp[m]; }
  __syncthreads();

  bool bad = false;
  const bool store_row = owned && y < a.ny;
  // ---------------- march: plane k's x- and y-faces, the z-face below it (completing k-1)
#pragma unroll 1
  for (int k = z0; k <= z1; ++k) {
    const bool last = k == z1;                 // only the z-face below plane z1 remains
    if (issuer && !last && k + 4 <= z1 + 1)
      tma_plane(s, &tmV, &tmE, slot_of(k + 4), X0 - 4, y0 - 2, zidx(k + 4));
    const int s0 = slot_of(k), sp = slot_of(k + 1);
    load_pair(s, sp, q, Wp);
    f2 acc[6];
    if (owned) {
      f2 d[3][6], ev[3], ed[3][3];
      differences(s, s0, q, W0, Wm, Wp, d, ev, ed);
      // z: face k-1/2 = l-side of plane k-1 + r-side of plane k; completes plane k-1
      {
        f2 pl[6], pr[6], ql[6], qr[6];
        side3<2, OpP>(W0, d, ev, ed, kz, pl, pr, ql, qr);
        if (!a.per[2] && k == a.nz) {
#pragma unroll
          for (int m = 0; m < 6; ++m) { pr[m] = pk(0.f, 0.f); qr[m] = pk(0.f, 0.f); }
        }
        const f2 ie = two_over(Wm[6] + W0[6]);
        f2 F[6];
        {
          f2 Lpl[6], Lql[6];                    // l-side z-vectors of plane k-1
          tmem_ld24(tz, Lpl, Lql);
#pragma unroll
          for (int m = 0; m < 6; ++m) F[m] = pfma(ie, Lql[m] + qr[m], Lpl[m] + pr[m]);
        }
        if (!last) tmem_st24(tz, pl, ql);
        if (k > z0 && store_row) {
          const int64_t o = (int64_t)(k - 1) * a.plane + (int64_t)y * a.pitch + x;
          f2 nv[6];
          const f2 nM = pk(-Minv.x, -Minv.y);
#pragma unroll
          for (int m = 0; m < 6; ++m) nv[m] = m < 3 ? pfma(nM, F[m], B[m]) : B[m] - F[m];
          f2 sum = nv[0];
#pragma unroll
          for (int m = 1; m < 6; ++m) sum = sum + nv[m];
          if (st1) {
#pragma unroll
            for (int m = 0; m < 6; ++m) *reinterpret_cast<f2 *>(a.Vout + m * a.cstride + o) = nv[m];
            bad |= !(isfinite(sum.x) && isfinite(sum.y));
          } else if (st0) {
#pragma unroll
            for (int m = 0; m < 6; ++m) a.Vout[m * a.cstride + o] = nv[m].x;
            bad |= !isfinite(sum.x);
          }
        }
        if (last) break;
#pragma unroll
        for (int m = 0; m < 6; ++m) acc[m] = pk(-F[m].x, -F[m].y);
      }
      // x: faces x+1/2 of both cells; the second needs the r-side of the next lane's first cell
      {
        f2 pl[6], pr[6], ql[6], qr[6];
        side3<0, OpP>(W0, d, ev, ed, kx, pl, pr, ql, qr);
        if (xg0 | xg1) {                        // ghost columns past the high x side
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            if (xg0) { pl[m].x = 0.f; pr[m].x = 0.f; ql[m].x = 0.f; qr[m].x = 0.f; }
            if (xg1) { pl[m].y = 0.f; pr[m].y = 0.f; ql[m].y = 0.f; qr[m].y = 0.f; }
          }
        }
        const int par = k & 1;
        float rp[6], rq[6], re;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          rp[m] = __shfl_down_sync(FULL, pr[m].x, 1);
          rq[m] = __shfl_down_sync(FULL, qr[m].x, 1);
        }
        re = __shfl_down_sync(FULL, W0[6].x, 1);
        if (lane == 31) {                       // right neighbour: column X0+64 (halo warp H1)
#pragma unroll
          for (int m = 0; m < 6; ++m) rp[m] = s.XR[par][warp][m];
          rq[0] = 0.f;
#pragma unroll
          for (int m = 1; m < 6; ++m) rq[m] = s.XR[par][warp][5 + m];
          re = s.XR[par][warp][11];
        }
        const f2 ie = two_over(W0[6] + pk(W0[6].y, re));
        f2 F[6];
#pragma unroll
        for (int m = 0; m < 6; ++m)
          F[m] = pfma(ie, ql[m] + pk(qr[m].y, rq[m]), pl[m] + pk(pr[m].y, rp[m]));
        float Fm[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) Fm[m] = __shfl_up_sync(FULL, F[m].y, 1);
        if (lane == 0) {                        // left face of the tile: column X0-1 (H0)
          const float ie0 = __fdividef(2.f, s.XL[par][warp][11] + W0[6].x);
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            const float lq = m == 0 ? 0.f : s.XL[par][warp][5 + m];
            Fm[m] = fmaf(ie0, lq + qr[m].x, s.XL[par][warp][m] + pr[m].x);
          }
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) acc[m] = acc[m] + (F[m] - pk(Fm[m], F[m].x));
      }
      // y: r-side vectors published for the row below; the face above waits for the barrier
      f2 pl[6], pr[6], ql[6], qr[6];
      side3<1, OpP>(W0, d, ev, ed, ky, pl, pr, ql, qr);
      if (yghost) {
#pragma unroll
        for (int m = 0; m < 6; ++m) { pl[m] = pr[m] = ql[m] = qr[m] = pk(0.f, 0.f); }
      }
#pragma unroll
      for (int m = 0; m < 6; ++m) s.Y[warp][m][lane] = pr[m];
      s.Y[warp][6][lane] = qr[0];
#pragma unroll
      for (int m = 2; m < 6; ++m) s.Y[warp][5 + m][lane] = qr[m];
      __syncthreads();                          // B1: r-side vectors of every row
      {
        const f2 eu = q.pair ? *reinterpret_cast<const f2 *>(&s.V[s0].a[6][q.rp][q.t0])
                             : pk(s.V[s0].a[6][q.rp][q.t0], s.V[s0].a[6][q.rp][q.t1]);
        const f2 ie = two_over(W0[6] + eu);
        f2 Rp[6], Rq[6];
#pragma unroll
        for (int m = 0; m < 6; ++m) Rp[m] = s.Y[warp + 1][m][lane];
        Rq[0] = s.Y[warp + 1][6][lane];
        Rq[1] = pk(0.f, 0.f);
#pragma unroll
        for (int m = 2; m < 6; ++m) Rq[m] = s.Y[warp + 1][5 + m][lane];
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          const f2 F = pfma(ie, ql[m] + Rq[m], pl[m] + Rp[m]);
          s.F[warp][m][lane] = F;
          acc[m] = acc[m] + F;
        }
      }
    } else {
      // halo warps: the y-vectors of their row, and the x-halo columns of plane k+1
      if (last) break;
      f2 d[3][6], ev[3], ed[3][3], pl[6], pr[6], ql[6], qr[6];
      differences(s, s0, q, W0, Wm, Wp, d, ev, ed);
      side3<1, OpP>(W0, d, ev, ed, ky, pl, pr, ql, qr);
      if (yghost) {
#pragma unroll
        for (int m = 0; m < 6; ++m) { pl[m] = pr[m] = ql[m] = qr[m] = pk(0.f, 0.f); }
      }
      if (h1) {
#pragma unroll
        for (int m = 0; m < 6; ++m) s.Y[NWO][m][lane] = pr[m];
        s.Y[NWO][6][lane] = qr[0];
#pragma unroll
        for (int m = 2; m < 6; ++m) s.Y[NWO][5 + m][lane] = qr[m];
      }
      if (lane < NWO) {
        float out[12];
        const int sm = s0, sc = sp, sn = slot_of(k + 2);
        halo_x_cell(s, sm, sc, sn, hr, hrm, hrp, ht, htm, htp, kx, h0, hghost, out);
        float *dst = h0 ? s.XL[(k + 1) & 1][lane] : s.XR[(k + 1) & 1][lane];
#pragma unroll
        for (int u = 0; u < 12; ++u) dst[u] = out[u];
      }
      __syncthreads();                          // B1
      if (h0) {                                 // face below row y0
        const f2 eu = q.pair ? *reinterpret_cast<const f2 *>(&s.V[s0].a[6][q.rp][q.t0])
                             : pk(s.V[s0].a[6][q.rp][q.t0], s.V[s0].a[6][q.rp][q.t1]);
        const f2 ie = two_over(W0[6] + eu);
#pragma unroll
        for (int m = 0; m < 6; ++m) {
          f2 Rq = pk(0.f, 0.f);
          if (m == 0) Rq = s.Y[0][6][lane];
          if (m >= 2) Rq = s.Y[0][5 + m][lane];
          s.F[NWO][m][lane] = pfma(ie, ql[m] + Rq, pl[m] + s.Y[0][m][lane]);
        }
      }
    }
    if (k + 3 <= last_plane) {
      if (!mbar_wait(&s.bar[slot_of(k + 3)], parity_of(k + 3))) {
        s.err = 1;                              // plane k+3 never landed
        atomicOr(a.flag, 2);
      } else if (s.nfix) {
        fix_plane(s, a, slot_of(k + 3), zidx(k + 3), tid);   // periodic sides: wrapped cells
      }
    }
    __syncthreads();                            // B2: face fluxes; plane k+3 visible
    if (s.err) {                                // leave together; wait (bounded) for the copy
      if (k + 4 <= last_plane) mbar_wait(&s.bar[slot_of(k + 4)], parity_of(k + 4));
      break;
    }
    if (owned) {
      const int below = warp == 0 ? NWO : warp - 1;
      f2 nv_src = pk(0.f, 0.f);
      if (a.src && y >= a.sy0 && y < a.sy1 && k >= a.sz0 && k < a.sz1) {
        const int64_t o = (int64_t)k * a.plane + (int64_t)y * a.pitch;
        const float s0v = (x >= a.sx0 && x < a.sx1) ? a.src[o + x] : 0.f;
        const float s1v = (x + 1 >= a.sx0 && x + 1 < a.sx1) ? a.src[o + x + 1] : 0.f;
        nv_src = pk(a.src_amp * s0v, a.src_amp * s1v);
      }
      Minv = pk(__fdividef(1.f, W0[6].x), __fdividef(1.f, W0[6].y));
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        f2 am = acc[m] - s.F[below][m][lane];
        if (m == 2) am = am + nv_src;
        B[m] = m < 3 ? pfma(pk(-Minv.x, -Minv.y), am, W0[m]) : W0[m] - am;
      }
    }
#pragma unroll
    for (int m = 0; m < NA; ++m) Wm[m] = W0[m];
    load_pair(s, sp, q, W0);                   // plane k+1 (still staged) is the next W0
  }
  // release the tensor memory once every row warp's accesses are done
  if (owned) asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == NWO + 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s.tmem),
                 "r"(kTmemCols)
                 : "memory");
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(a.flag, 1);
}

}  // namespace

namespace {

// Tensor map of `rank` dims over a [ncomp][nz][ny][pitch] FP32 array: dims (nx, ny, nz[, 6]),
// box (TW, NR, 1[, 6]); entries past the grid read as zero.
bool encode_map(CUtensorMap *m, const float *base, const CartGeom &g, int rank) {
  const cuuint64_t dim[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, 6};
  const cuuint64_t stride[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.plane * 4,
                                (cuuint64_t)g.cstride * 4};
  const cuuint32_t box[4] = {TW, NR, 1, 6};
  return encode_f32_map(m, base, rank, dim, stride, box);
}

}  // namespace

bool cart3d_side_supported(const CartGeom &g, const CartStepArgs &a, bool fp64) {
  if (fp64 || a.mu || a.limiter) return false;
  if (!tensor_map_encoder()) return false;
  for (int k = 0; k < 6; ++k)
    if (g.pec[k]) return false;
  // the wrap list holds in-plane offsets as int
  return g.dim == 3 && g.plane < (int64_t(1) << 31);
}

cudaError_t launch_cart3d_side(const CartGeom &g, const CartStepArgs &a, cudaStream_t st) {
  Side3Args p;
  p.V = static_cast<const float *>(a.V);
  p.Vout = static_cast<float *>(a.Vout);
  p.eps = static_cast<const float *>(a.eps);
  p.src = static_cast<const float *>(a.src);
  p.sx0 = a.src_box[0]; p.sx1 = a.src_box[1];
  p.sy0 = a.src_box[2]; p.sy1 = a.src_box[3];
  p.sz0 = a.src_box[4]; p.sz1 = a.src_box[5];
  p.src_amp = float(a.src_amp);
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz;
  p.pitch = g.pitch; p.plane = g.plane; p.cstride = g.cstride;
  for (int d = 0; d < 3; ++d) p.per[d] = g.periodic[d];
  p.flag = a.flag;
  for (int A = 0; A < 3; ++A) {
    double k[kSide3K];
    side3_coefficients(a.C, g.h, a.c, A, k);
    for (int i = 0; i < kSide3K; ++i) p.k[A][i] = float(k[i]);
  }
  const int gx = (g.nx + TCOLS - 1) / TCOLS, gy = (g.ny + NWO - 1) / NWO;
  const int smem = (int)sizeof(SideSmem);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(cart3d_side_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  // z chunks: one CTA per SM; pick the chunk count that fills whole waves best.  A CTA's fixed
  // cost -- staging its first four planes with nothing to overlap them, the z-vectors of the
  // plane below its chunk and the closing z-face -- counts as 2.7 planes of work: the value that
  // fits measured step times at 256^3 over 1 to 32 chunks (7 chunks, 0.511 ms; 16, 0.529 ms)
  constexpr double kChunkCost = 2.7;
  const int64_t tiles = (int64_t)gx * gy;
  int zchunks = 1;
  double best = -1.0;
  for (int zc = 1; zc <= 64 && zc <= g.nz; ++zc) {
    const int len = (g.nz + zc - 1) / zc;
    const int nzc = (g.nz + len - 1) / len;
    const int64_t ctas = tiles * nzc;
    const double waves = (double)((ctas + sms - 1) / sms);
    const double eff =
        (double)ctas / (waves * sms) * (double)g.nz / ((double)nzc * (len + kChunkCost));
    if (eff > best + 1e-9) { best = eff; zchunks = nzc; }
  }
  p.zchunk = (g.nz + zchunks - 1) / zchunks;
  zchunks = (g.nz + p.zchunk - 1) / p.zchunk;
  CUtensorMap tmV, tmE;
  if (!encode_map(&tmV, p.V, g, 4) || !encode_map(&tmE, p.eps, g, 3)) return cudaErrorInvalidValue;
  dim3 grid(gx, gy, zchunks);
  cart3d_side_kernel<<<grid, NTH, smem, st>>>(tmV, tmE, p);
  return cudaGetLastError();
}

}  // namespace gks
