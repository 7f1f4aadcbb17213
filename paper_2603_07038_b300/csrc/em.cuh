// Fused leapfrog step of the Maxwell system (Sec. II-A, Eqs. 1-3 in E/H form)
// with the Joule heat of the step (P_total = D_sigma e^2), one launch per step.
//
// Each CTA owns a (TX-1) x (TY-1) tile of nodes in x-y and marches through
// every node plane k = 0..nz. Its threads cover the tile plus one halo column
// (i-1) and row (j-1): at plane k every thread forms H^{n+1/2}(i,j,k) from
// E^n (own plane and plane k+1), shares it through shared memory, and forms
// E^{n+1} on its edges from the H of the thread to its -x/-y side and from its
// own H of plane k-1 (kept in registers). Halo threads recompute the H and the
// single E edge their neighbours need (for Joule) but write nothing.
// E, H and the CPML auxiliaries are double-buffered (read *_o, write *_n), so
// CTAs never see each other's half-updated values.
//
// Joule heat: the edge from node n to n+e_a dissipates sigma_e V_e ebar^2 in
// one step, ebar = (E^n + E^{n+1})/2; half of dt times that goes to each end
// node, i.e. (sum_c w_c sigma_c dt/2) * l_e * ebar^2 per end node, where w_c is
// the quarter cross-section of voxel c around the edge. The node sums the six
// halves of its incident edges (x from the thread at i-1, y from j-1 through
// shared memory, z from its own previous plane) into a short-window
// accumulator that is folded into the FP64 total every few steps (FP64 runs at
// a small fraction of the FP32 rate on this GPU, so none is used per step).
//
// Inputs of planes k+2 and k+3 are copied to shared memory by TMA (one thread
// issues a 2-D box per array and plane, completion tracked by one mbarrier per
// stage, four stages) while plane k is computed. Waits on those barriers are
// bounded: a copy that never arrives sets an error word instead of hanging.
//
// Material averaging (per edge: area-weighted eps, sigma over the <=4 voxels;
// per face: series mean of mu over the 2 voxels) is recomputed from the 1-byte
// voxel IDs every step instead of streaming per-edge coefficient arrays.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "common.cuh"

namespace cosim {

template <typename R>
struct EmArgs {
  Geo<R> g;
  const R *Eo[3];
  R *En[3];
  const R *Ho[3];
  R *Hn[3];
  // CPML state for derivative axis d, slot s (field component (d+1+s)%3).
  // The CPML recursion psi^n = b psi^{n-1} + c dF^n with c = b - 1 (kappa = 1,
  // alpha = 0) is carried in the equivalent form
  //   chi^n = dF^n + psi^n = b (chi^{n-1} + dF^n - dF^{n-1}),
  // storing chi and the previous derivative dF^{n-1}. Inside a layer psi tends
  // to -dF for slowly varying fields, so dF + psi cancels and FP32 kept no bits
  // of the residue; chi is that residue itself. Near the inner edge of a layer
  // b is close to 1 and chi sums the derivative changes of thousands of steps,
  // so in FP32 it is carried as an unevaluated pair chi = hi + lo (lEo..lHn,
  // null in FP64 contexts) updated with error-free transformations.
  const R *xEo[3][2], *dEo[3][2], *lEo[3][2];
  R *xEn[3][2], *dEn[3][2], *lEn[3][2];
  const R *xHo[3][2], *dHo[3][2], *lHo[3][2];
  R *xHn[3][2], *dHn[3][2], *lHn[3][2];
  int slo[3], shi[3], sn[3];  // CPML cells at the low / high end, slab extent
  const R *cpml;              // 1 - b per [axis][E,H][kMaxSlab] (computed as -expm1 on the host)
  int fixlo[3], fixhi[3];     // wall holds tangential E at zero (PEC or CPML backing)
  R dt;
  const int *src_row;         // per (k,j) row: first source entry, (nz+1)(ny+1)+1 ints,
                              // readable from index -4 to 15 past the end (zero padding)
  const int4 *src_ent;        // (i, axis, source index, 0)
  const R *src_amp;           // [source][amp_len]
  long long amp_len;
  // source time index of this launch = *step_base + step_off: the base lives
  // in device memory and is advanced once per call, so a captured CUDA graph
  // of several steps replays with the right source samples
  const long long *step_base;
  int step_off;
  // Joule energy: each step adds to the short-window accumulator Qs (context
  // precision); on fold steps the owner moves Qs into the FP64 total Q instead,
  // so FP64 arithmetic runs once per window rather than every step.
  R *Qs;                      // null: not accumulating
  double *Q;
  int fold;
  // tiles [ibx0, ibx1) x [iby0, iby1) lie off the lateral walls and CPML slabs
  int ibx0, ibx1, iby0, iby1;
  // TMA descriptors of E^n, H^{n-1/2} (per component) and Qs: 3-D node
  // arrays (x, y, z) with boxes of kEmBoxX x (TY+1 for E, TY otherwise) x 1
  CUtensorMap tmE[3], tmH[3], tmQ;
  CUtensorMap tmV;  // voxel IDs (x, y, z), box em_vox_box_x x (TY+1) x 1
  // two-way coupling (the CPL specialisation, Sec. II-A): the temperature
  // rise T^n - T_init (node array, staged like E), the step's Joule power per
  // node written to Pout [W], 1 / dt
  CUtensorMap tmT;
  R *Pout;
  R inv_dt;
  const R *zt;      // per node plane: hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
  int *err;         // set to 1 when a bounded wait for a staged plane gave up
};

// index of position p (node or cell) of an axis inside its CPML slabs, or -1
__device__ __forceinline__ int slab_index(int p, int n, int lo, int hi) {
  if (lo > 0 && p <= lo) return p;
  if (hi > 0 && p >= n - hi) return (lo > 0 ? lo + 1 : 0) + (p - (n - hi));
  return -1;
}

template <typename R>
__device__ __forceinline__ long long psi_index(const EmArgs<R> &A, int d, int s, int i, int j, int k) {
  if (d == 0) return ((long long)k * (A.g.ny + 1) + j) * A.sn[0] + s;
  if (d == 1) return ((long long)k * A.sn[1] + s) * A.g.px + i;
  return ((long long)s * (A.g.ny + 1) + j) * A.g.px + i;
}

// chi^n = b (chi^{n-1} + dF^n - dF^{n-1}), evaluated as t - (1-b) t; returns
// chi^n = dF + psi (new values written only by the owner)
template <typename R>
__device__ __forceinline__ R chi_update(const EmArgs<R> &A, const R *s_cp, int d, int type, int slot, int s, int i,
                                        int j, int k, R deriv, bool write) {
  const long long q = psi_index(A, d, s, i, j, k);
  const R omb = s_cp[(d * 2 + type) * kMaxSlab + s];
  const R *xo = type == 0 ? A.xEo[d][slot] : A.xHo[d][slot];
  const R *dd = type == 0 ? A.dEo[d][slot] : A.dHo[d][slot];
  if constexpr (sizeof(R) == 8) {
    const R t = xo[q] + (deriv - dd[q]);
    const R chi = t - omb * t;
    if (write) {
      (type == 0 ? A.xEn[d][slot] : A.xHn[d][slot])[q] = chi;
      (type == 0 ? A.dEn[d][slot] : A.dHn[d][slot])[q] = deriv;
    }
    return chi;
  } else {
    // (hi + lo + D)(1 - omb) with Knuth's TwoSum for the additions, an FMA
    // product error for omb * hi, and a final renormalisation (Fast2Sum).
    const R hi = xo[q];
    const R lo = (type == 0 ? A.lEo[d][slot] : A.lHo[d][slot])[q];
    const R D = deriv - dd[q];
    const R sh = hi + D;
    const R bv = sh - hi;
    const R e1 = (hi - (sh - bv)) + (D - bv);
    const R l1 = lo + e1;
    const R p = __fmul_rn(omb, sh);
    const R pe = __fmaf_rn(omb, sh, -p);
    const R s2 = sh - p;
    const R bv2 = s2 - sh;
    const R e2 = (sh - (s2 - bv2)) + (-p - bv2);
    const R l2 = (l1 + e2) - pe - __fmul_rn(omb, l1);
    const R h3 = s2 + l2;
    const R l3 = l2 - (h3 - s2);
    if (write) {
      (type == 0 ? A.xEn[d][slot] : A.xHn[d][slot])[q] = h3;
      (type == 0 ? A.lEn[d][slot] : A.lHn[d][slot])[q] = l3;
      (type == 0 ? A.dEn[d][slot] : A.dHn[d][slot])[q] = deriv;
    }
    return h3;
  }
}

// (dF1 + psi1) - (dF2 + psi2) for the two derivatives of one curl component;
// the CPML state is touched only inside a slab (s1/s2 >= 0).
template <typename R>
__device__ __forceinline__ R curl_with_psi(const EmArgs<R> &A, const R *s_cp, int type, int comp, int d1, int s1,
                                           int d2, int s2, int i, int j, int k, R v1, R v2, bool write) {
  (void)comp;
  if (s1 < 0 && s2 < 0) return v1 - v2;
  const R a = s1 >= 0 ? chi_update(A, s_cp, d1, type, 1, s1, i, j, k, v1, write) : v1;
  const R b = s2 >= 0 ? chi_update(A, s_cp, d2, type, 0, s2, i, j, k, v2, write) : v2;
  return a - b;
}

static_assert(M_EPS == 0 && M_SDT2 == 1 && M_IMU == 2 && M_COLS % 4 == 0,
              "the EM kernel reads eps, sigma dt/2, 1/mu of a material row with one aligned vector load");
// Four consecutive values from 16-byte aligned shared memory in one vector load.
__device__ __forceinline__ void load4(const float *p, float &a, float &b, float &c, float &d) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  a = v.x, b = v.y, c = v.z, d = v.w;
}
__device__ __forceinline__ void load4(const double *p, double &a, double &b, double &c, double &d) {
  const double2 v = reinterpret_cast<const double2 *>(p)[0], w = reinterpret_cast<const double2 *>(p)[1];
  a = v.x, b = v.y, c = w.x, d = w.y;
}

// Reciprocal of a positive normal number: in FP32 the hardware approximation
// refined by one Newton-Raphson step (r' = r + r (1 - x r)), within about an
// ulp of 1/x; in FP64 the exact division.
__device__ __forceinline__ float em_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}
__device__ __forceinline__ double em_rcp(double x) { return 1.0 / x; }

// E^{n+1} of one edge from the area-weighted sums over its <= 4 voxels, all
// taken without the quarter factor of the voxel cross-sections (it cancels):
//   Se = sum w eps, Ss = sum w sigma dt/2 (w = product of the two transverse
//   cell sizes of the voxel), dtW = dt x (sum of those products) = 4 dt x the
//   dual-face area, lq = edge length / 4.
// The update E' = ca E + cb (curl - J) (ca = (Se - Ss)/(Se + Ss),
// cb = dt W/(Se + Ss)) is evaluated in the equivalent incremental form
// E' = E + r (dtW (curl - J) - 2 Ss E), r = 1/(Se + Ss), which keeps the decay
// 1 - ca of weakly lossy media at full precision. *half_q receives the edge's
// Joule energy per end node, (Ss/4) l ebar^2 with ebar = (E + E')/2.
template <typename R>
__device__ __forceinline__ R e_update(R e_old, R dtW, R drive, R Se, R Ss, R lq, R *half_q) {
  const R r = em_rcp(Se + Ss);
  const R e_new = e_old + r * (dtW * drive - R(2) * Ss * e_old);
  const R eb = R(0.5) * (e_old + e_new);
  *half_q = Ss * lq * eb * eb;
  return e_new;
}

// One plane of the CTA's inputs, staged in shared memory by TMA: E^n of the
// tile plus its +x/+y neighbours, H^{n-1/2} and the Joule accumulator. A TMA
// box must start at an x coordinate that is a multiple of 16 bytes, so the
// box starts at the tile's first node rounded down to a multiple of 4 and is
// kEmBoxX = TX + 4 nodes wide; threads index it from that remainder.
template <int TX>
__host__ __device__ constexpr int em_box_x() { return TX + 4; }
// voxel box: columns i0-1 .. i0+TX-1 from x rounded down to 16 bytes
template <int TX>
__host__ __device__ constexpr int em_vox_box_x() { return (TX + 1 + 15 + 15) / 16 * 16; }
// source-row box: rows j0 .. j0+TY (+1 for the end offset) from a multiple of 4
template <int TY>
__host__ __device__ constexpr int em_src_box() { return (TY + 1 + 3 + 3) / 4 * 4; }
template <typename R, int TX, int TY>
struct EmStage {
  EmBox<R, TY + 1, em_box_x<TX>()> E[3];
  EmBox<R, TY, em_box_x<TX>()> H[3];
  EmBox<R, TY, em_box_x<TX>()> Qs;
  EmBox<uint8_t, TY + 1, em_vox_box_x<TX>()> V;  // voxel IDs of layer k, rows j0-1 .. j0+TY-1
  EmBox<int, 1, em_src_box<TY>()> S;             // source-row offsets of plane k
  EmBox<R, 1, 4> Z;                              // hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
  EmBox<R, TY + 1, em_box_x<TX>()> T;            // temperature rise (coupled steps only)
};

constexpr int kCpmlTable = 6 * kMaxSlab;  // (1 - b) per [axis][E,H][slab position]

// Shared-memory offset of the stages: the CPML table, then nmat + 1 material
// rows (row nmat is all zero and stands for voxels outside the grid).
template <typename R, int TX, int TY>
__host__ __device__ constexpr size_t em_stage_offset(int nmat) {
  return ((kCpmlTable + (size_t)(nmat + 1) * M_COLS) * sizeof(R) + 127) & ~size_t(127);
}

// Shared-memory stages (a power of two) and the prefetch distance: at plane k
// the copy of plane k + kEmAhead is issued and planes k, k+1 must have landed.
#ifndef COSIM_EM_STAGES
#define COSIM_EM_STAGES 4
#endif
#ifndef COSIM_EM_AHEAD
#define COSIM_EM_AHEAD 3
#endif
#ifndef COSIM_EM_MIN_CTAS
#define COSIM_EM_MIN_CTAS 3  // resident CTAs of 8 warps per SM the FP32 kernel is compiled for (scaled for other heights)
#endif
constexpr int kEmStages = COSIM_EM_STAGES;
constexpr int kEmAhead = COSIM_EM_AHEAD;
static_assert((kEmStages & (kEmStages - 1)) == 0, "stage count must be a power of two");
static_assert(kEmAhead >= 2 && kEmAhead <= kEmStages - 1, "prefetch distance must leave the stage of plane k-1 free");

// Body of the fused step for one CTA tile. BORDER = false is the interior
// specialisation: every node of the tile and its +x/+y neighbours lies inside
// the grid, off the lateral walls and outside the x/y CPML slabs, so the
// bounds, wall and lateral-CPML tests fold away at compile time (only the
// z-direction slab and walls remain, decided per plane for the whole CTA).
// I: index type of node offsets (int when the padded node arrays have fewer
// than 2^31 elements, long long otherwise).
template <typename R, typename I, int TX, int TY, bool BORDER, bool CPL>
__device__ __forceinline__ void em_tile(const EmArgs<R> &A, const R *s_cp, const R *s_mt,
                                        EmStage<R, TX, TY> *stg, R (*sHxz)[TY][TX], R (*sQy)[TX], uint64_t *bars,
                                        int *s_abort) {
  const Geo<R> &g = A.g;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int vd = g.nmat * M_COLS;  // row offset of the all-zero material
  const int i0 = blockIdx.x * (TX - 1) - 1, j0 = blockIdx.y * (TY - 1) - 1;  // node of thread (0, 0)
  const int i = i0 + tx, j = j0 + ty;
  const bool act = !BORDER || (i >= 0 && i <= nx && j >= 0 && j <= ny);
  const bool own = act && tx > 0 && ty > 0;
  const bool need_ex = act && ty > 0 && (!BORDER || i < nx);  // own, or the halo column
  const bool need_ey = act && tx > 0 && (!BORDER || j < ny);  // own, or the halo row
  const bool in_x = !BORDER || i < nx, in_y = !BORDER || j < ny;
  const bool accum = A.Qs != nullptr;

  // Plane k of E^n (tile + neighbours), H^{n-1/2} and Qs -> stage k mod
  // kEmStages, by TMA: one thread announces the bytes on the stage's mbarrier
  // and issues the seven box copies; positions outside the grid arrive as zero.
  // Box x starts at the tile's first node rounded down to a multiple of 4
  // (two's complement: i0 = -1 gives x0 = -4); threads read from column tx + xr.
  const int xr = i0 & 3, x0 = i0 - xr;
  const bool leader = tx == 0 && ty == 0;
  // The voxel box starts at column i0 - 1 rounded down to 16 bytes, the
  // source-row box at entry k (ny+1) + j0 rounded down to 4 ints.
  const int xvr = (i0 - 1) & 15, xv0 = (i0 - 1) - xvr;
  const bool has_src = A.src_row != nullptr;
  // transaction bytes of one stage: the boxes themselves, not their padding
  const unsigned fixed_bytes =
      (unsigned)((6 * TY + 3 + (accum ? TY : 0) + (CPL ? TY + 1 : 0)) * em_box_x<TX>() * (int)sizeof(R) +
                 4 * (int)sizeof(R) + (has_src ? em_src_box<TY>() * 4 : 0));
  const unsigned vox_bytes = (unsigned)((TY + 1) * em_vox_box_x<TX>());
  auto issue = [&](int k) {
    if (k > nz) return;
    const int s = k & (kEmStages - 1);
    EmStage<R, TX, TY> &S = stg[s];
    mbar_arrive_expect_tx(&bars[s], fixed_bytes + (k < nz ? vox_bytes : 0u));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      tma_load_3d(&S.E[c].v[0][0], &A.tmE[c], x0, j0, k, &bars[s]);
      tma_load_3d(&S.H[c].v[0][0], &A.tmH[c], x0, j0, k, &bars[s]);
    }
    if (accum) tma_load_3d(&S.Qs.v[0][0], &A.tmQ, x0, j0, k, &bars[s]);
    if (CPL) tma_load_3d(&S.T.v[0][0], &A.tmT, x0, j0, k, &bars[s]);
    if (k < nz) tma_load_3d(&S.V.v[0][0], &A.tmV, xv0, j0 - 1, k, &bars[s]);
    bulk_load(&S.Z.v[0][0], A.zt + 4 * (size_t)k, 4 * sizeof(R), &bars[s]);
    if (has_src) {  // 16-byte aligned: src_row itself is, the start is a multiple of 4 from -4
      const int base = k * (ny + 1) + j0;
      bulk_load(&S.S.v[0][0], A.src_row + (base - (base & 3)), em_src_box<TY>() * 4, &bars[s]);
    }
  };
  const I plane = (I)g.plane;
  const I o_own = act ? (I)g.nid(i, j, 0) : I(0);
  // Material rows (id x M_COLS) of voxels (i-1+dx, j-1+dy, k) from the staged
  // voxel box; the zero row outside the grid.
  const bool cx0 = !BORDER || (i - 1 >= 0 && i - 1 < nx), cx1 = !BORDER || (i >= 0 && i < nx);
  const bool cy0 = !BORDER || (j - 1 >= 0 && j - 1 < ny), cy1 = !BORDER || (j >= 0 && j < ny);
  const int cv = tx + xvr;  // column of voxel i-1 in the box

  const R hxm = (act && (!BORDER || i > 0)) ? g.h[0][i - 1] : R(0), hx0 = (act && in_x) ? g.h[0][i] : R(0);
  const R hym = (act && (!BORDER || j > 0)) ? g.h[1][j - 1] : R(0), hy0 = (act && in_y) ? g.h[1][j] : R(0);
  const R ihx = (act && in_x) ? g.ih[0][i] : R(0), ihy = (act && in_y) ? g.ih[1][j] : R(0);
  const R idx = act ? g.idual[0][i] : R(0), idy = act ? g.idual[1][j] : R(0);
  const bool fix_x = BORDER && ((i == 0 && A.fixlo[0]) || (i == nx && A.fixhi[0]));
  const bool fix_y = BORDER && ((j == 0 && A.fixlo[1]) || (j == ny && A.fixhi[1]));
  // CPML slab positions along x and y (E: nodes, H: cells); none inside
  const int sxE = BORDER ? slab_index(i, nx, A.slo[0], A.shi[0]) : -1;
  const int syE = BORDER ? slab_index(j, ny, A.slo[1], A.shi[1]) : -1;
  const int sxH = in_x ? sxE : -1;
  const int syH = in_y ? syE : -1;
  const R dt = A.dt;
  const R half_dt = R(0.5) * dt;
  // per-thread geometry of the face and edge coefficients
  const R hdx = half_dt * idx, hdy = half_dt * idy;
  const R dtWx_y = dt * (hym + hy0), dtWy_x = dt * (hxm + hx0);
  const R lqx = R(0.25) * hx0, lqy = R(0.25) * hy0;
  const I id0 = o_own;

  if (leader) {
#pragma unroll
    for (int q = 0; q < kEmAhead; ++q) issue(q);
  }
  R hx_km1 = 0, hy_km1 = 0, qz_km1 = 0;
  // layer k-1 partial sums of the x / y edges and 1/mu of voxel (i, j, k-1);
  // zero below the grid
  R pxe_b = 0, pxs_b = 0, pye_b = 0, pys_b = 0, u11_b = 0;
  R q_pend = 0;  // Joule sum of node (i, j, k-1) still missing the y-edge share from j-1
  R e_pend = 0;  // the same without the accumulator's earlier energy (this step's only)
  int b01 = vd, b10 = vd, b11 = vd;  // coupled steps: material rows of layer k-1
  // sigma dt / 2 of a voxel at the edge temperature rise te (coupled steps):
  // sigma0 dt/2 / (1 + alpha (T_init + te - T0)) = M_SDT2 / (M_TC0 + M_TCR te)
  auto sig = [&](int row, R te) -> R {
    return s_mt[row + M_SDT2] * em_rcp(s_mt[row + M_TC0] + s_mt[row + M_TCR] * te);
  };

  for (int k = 0; k <= nz; ++k) {
    if (leader) {  // the stage of plane k-1 is free: every thread passed the last barrier
      fence_proxy_async_smem();
      issue(k + kEmAhead);
    }
    {  // planes k and k+1 have landed (phase parity: use count of the stage)
      bool ok = mbar_wait(&bars[k & (kEmStages - 1)], (unsigned)(k / kEmStages) & 1u);
      if (k + 1 <= nz) ok = mbar_wait(&bars[(k + 1) & (kEmStages - 1)], (unsigned)((k + 1) / kEmStages) & 1u) && ok;
      if (!ok) *s_abort = 1;
    }
    __syncthreads();
    if (*s_abort) {  // a copy did not arrive in time: drain what is in flight (bounded), flag, leave
      if (leader) {
        for (int q = k; q <= k + kEmAhead && q <= nz; ++q)
          mbar_wait(&bars[q & (kEmStages - 1)], (unsigned)(q / kEmStages) & 1u);
        atomicExch(A.err, 1);
      }
      return;
    }
    const I id = id0 + (I)k * plane;
    // Joule energy of node (i, j, k-1): its y-edge share from j-1 is now visible
    if (accum && own && k > 0) {
      const R s = q_pend + sQy[ty - 1][tx];
      if (A.fold) {
        A.Q[id - plane] += (double)s;
        A.Qs[id - plane] = R(0);
      } else {
        A.Qs[id - plane] = s;
      }
    }
    if (CPL && own && k > 0) A.Pout[id - plane] = (e_pend + sQy[ty - 1][tx]) * A.inv_dt;
    const EmStage<R, TX, TY> &S0 = stg[k & (kEmStages - 1)];
    const EmStage<R, TX, TY> &S1 = stg[(k + 1) & (kEmStages - 1)];
    R hz0, ihz, idz, hzm;
    load4(&S0.Z.v[0][0], hz0, ihz, idz, hzm);
    // material rows of voxel layer k (the layer above node plane k)
    const bool kz = k < nz;
    const int a00 = (kz && cx0 && cy0) ? (int)S0.V.v[ty][cv] * M_COLS : vd;
    const int a01 = (kz && cx1 && cy0) ? (int)S0.V.v[ty][cv + 1] * M_COLS : vd;
    const int a10 = (kz && cx0 && cy1) ? (int)S0.V.v[ty + 1][cv] * M_COLS : vd;
    const int a11 = (kz && cx1 && cy1) ? (int)S0.V.v[ty + 1][cv + 1] * M_COLS : vd;
    int r0 = 0, r1 = 0;  // source entries of row (k, j)
    if (has_src && act) {
      const int base = k * (ny + 1) + j0, sr = (base & 3) + ty;
      r0 = S0.S.v[0][sr];
      r1 = S0.S.v[0][sr + 1];
    }
    const R hdz = half_dt * idz;
    const bool fix_z = (k == 0 && A.fixlo[2]) || (k == nz && A.fixhi[2]);
    const int szE = slab_index(k, nz, A.slo[2], A.shi[2]);
    const int szH = (k < nz) ? szE : -1;

    const int cx = tx + xr;  // this node's column in the staged boxes
    const R ex = S0.E[0].v[ty][cx], ey = S0.E[1].v[ty][cx], ez = S0.E[2].v[ty][cx];
    const R ex_up = S1.E[0].v[ty][cx], ey_up = S1.E[1].v[ty][cx];
    const R ez_jp = S0.E[2].v[ty + 1][cx], ex_jp = S0.E[0].v[ty + 1][cx];
    const R ez_ip = S0.E[2].v[ty][cx + 1], ey_ip = S0.E[1].v[ty][cx + 1];
    const R hx_o = S0.H[0].v[ty][cx], hy_o = S0.H[1].v[ty][cx], hz_o = S0.H[2].v[ty][cx];
    const R q_old = accum ? S0.Qs.v[ty][cx] : R(0);
    // coupled steps: temperature rise at this node and its +x, +y, +z neighbours
    R th = 0, th_ip = 0, th_jp = 0, th_kp = 0;
    if (CPL) {
      th = S0.T.v[ty][cx];
      th_ip = S0.T.v[ty][cx + 1];
      th_jp = S0.T.v[ty + 1][cx];
      th_kp = k < nz ? S1.T.v[ty][cx] : R(0);
    }

    // material constants of voxel layer k
    // (columns M_EPS, M_SDT2, M_IMU, M_K are adjacent: one vector load per voxel)
    R e00, s00, u00, k00, e01, s01, u01, k01, e10, s10, u10, k10, e11, s11, u11, k11;
    load4(s_mt + a00, e00, s00, u00, k00);
    load4(s_mt + a01, e01, s01, u01, k01);
    load4(s_mt + a10, e10, s10, u10, k10);
    load4(s_mt + a11, e11, s11, u11, k11);

    // ---- H^{n+1/2} at (i,j,k): H -= dt/mu (curl E + psi terms); dt/mu of a
    // face is the series mean over the two voxels its dual edge crosses
    R Hx = 0, Hy = 0, Hz = 0;
    if (act) {
      if (in_y && k < nz) {  // Hx: (curl E)_x = dEz/dy - dEy/dz, voxels (i-1..i, j, k)
        const R d1 = (ez_jp - ez) * ihy, d2 = (ey_up - ey) * ihz;
        const R curl = curl_with_psi(A, s_cp, 1, 0, 1, syH, 2, szH, i, j, k, d1, d2, own);
        Hx = hx_o - hdx * (hxm * u10 + hx0 * u11) * curl;
      }
      if (in_x && k < nz) {  // Hy: dEx/dz - dEz/dx, voxels (i, j-1..j, k)
        const R d1 = (ex_up - ex) * ihz, d2 = (ez_ip - ez) * ihx;
        const R curl = curl_with_psi(A, s_cp, 1, 1, 2, szH, 0, sxH, i, j, k, d1, d2, own);
        Hy = hy_o - hdy * (hym * u01 + hy0 * u11) * curl;
      }
      if (in_x && in_y) {  // Hz: dEy/dx - dEx/dy, voxels (i, j, k-1..k)
        const R d1 = (ey_ip - ey) * ihx, d2 = (ex_jp - ex) * ihy;
        const R curl = curl_with_psi(A, s_cp, 1, 2, 0, sxH, 1, syH, i, j, k, d1, d2, own);
        Hz = hz_o - hdz * (hzm * u11_b + hz0 * u11) * curl;
      }
    }
    sHxz[0][ty][tx] = Hx;
    sHxz[1][ty][tx] = Hz;
    const R hy_l = __shfl_up_sync(0xffffffffu, Hy, 1);  // H of node i-1 (same warp)
    const R hz_l = __shfl_up_sync(0xffffffffu, Hz, 1);
    __syncthreads();

    // ---- source current on this node's edges (three scalars selected by
    // axis: a dynamically indexed array would live in local memory)
    R Jx = 0, Jy = 0, Jz = 0;
    for (int e = r0; e < r1; ++e) {
      const int4 s = A.src_ent[e];
      const long long step = *A.step_base + A.step_off;
      if (s.x == i && step < A.amp_len) {
        const R a = A.src_amp[(long long)s.z * A.amp_len + step];
        Jx += s.y == 0 ? a : R(0);
        Jy += s.y == 1 ? a : R(0);
        Jz += s.y == 2 ? a : R(0);
      }
    }

    // ---- E^{n+1} on the node's edges and their Joule shares. Layer-k partial
    // sums of the x / y edges (voxel pairs across y / x); the layer k-1 halves
    // were formed one plane earlier.
    const R pxe_a = hym * e01 + hy0 * e11, pxs_a = hym * s01 + hy0 * s11;
    const R pye_a = hxm * e10 + hx0 * e11, pys_a = hxm * s10 + hx0 * s11;
    R exn = ex, eyn = ey, ezn = ez, qx = 0, qy = 0, qz = 0;
    if (need_ex && !(fix_y || fix_z)) {  // Ex: dHz/dy - dHy/dz, voxels (i, j-1..j, k-1..k)
      const R d1 = (Hz - sHxz[1][ty - 1][tx]) * idy;
      const R d2 = (Hy - hy_km1) * idz;
      const R curl = curl_with_psi(A, s_cp, 0, 0, 1, syE, 2, szE, i, j, k, d1, d2, own);
      R Ss = hzm * pxs_b + hz0 * pxs_a;
      if (CPL) {
        const R te = R(0.5) * (th + th_ip);
        Ss = hzm * (hym * sig(b01, te) + hy0 * sig(b11, te)) + hz0 * (hym * sig(a01, te) + hy0 * sig(a11, te));
      }
      exn = e_update(ex, dtWx_y * (hzm + hz0), curl - Jx, hzm * pxe_b + hz0 * pxe_a, Ss, lqx, &qx);
    }
    // (interior tiles also run Ey / Ez on the halo lane tx = 0 and discard
    // them: the warp stays convergent; only the owners store)
    if ((BORDER ? need_ey : true) && !(fix_x || fix_z)) {  // Ey: dHx/dz - dHz/dx, voxels (i-1..i, j, k-1..k)
      const R d1 = (Hx - hx_km1) * idz;
      const R d2 = (Hz - hz_l) * idx;
      const R curl = curl_with_psi(A, s_cp, 0, 1, 2, szE, 0, sxE, i, j, k, d1, d2, own);
      R Ss = hzm * pys_b + hz0 * pys_a;
      if (CPL) {
        const R te = R(0.5) * (th + th_jp);
        Ss = hzm * (hxm * sig(b10, te) + hx0 * sig(b11, te)) + hz0 * (hxm * sig(a10, te) + hx0 * sig(a11, te));
      }
      eyn = e_update(ey, dtWy_x * (hzm + hz0), curl - Jy, hzm * pye_b + hz0 * pye_a, Ss, lqy, &qy);
    }
    if ((BORDER ? own : ty > 0) && k < nz && !(fix_x || fix_y)) {  // Ez: dHy/dx - dHx/dy, voxels (i-1..i, j-1..j, k)
      const R d1 = (Hy - hy_l) * idx;
      const R d2 = (Hx - sHxz[0][ty - 1][tx]) * idy;
      const R curl = curl_with_psi(A, s_cp, 0, 2, 0, sxE, 1, syE, i, j, k, d1, d2, own);
      const R Se = hym * (hxm * e00 + hx0 * e01) + hy0 * (hxm * e10 + hx0 * e11);
      R Ss = hym * (hxm * s00 + hx0 * s01) + hy0 * (hxm * s10 + hx0 * s11);
      if (CPL) {
        const R te = R(0.5) * (th + th_kp);
        Ss = hym * (hxm * sig(a00, te) + hx0 * sig(a01, te)) + hy0 * (hxm * sig(a10, te) + hx0 * sig(a11, te));
      }
      ezn = e_update(ez, dtWx_y * (hxm + hx0), curl - Jz, Se, Ss, R(0.25) * hz0, &qz);
    }
    const R qx_l = __shfl_up_sync(0xffffffffu, qx, 1);  // x-edge share from node i-1
    sQy[ty][tx] = qy;

    if (own) {
      A.Hn[0][id] = Hx;
      A.Hn[1][id] = Hy;
      A.Hn[2][id] = Hz;
      A.En[0][id] = exn;
      A.En[1][id] = eyn;
      if (k < nz) A.En[2][id] = ezn;
    }
    e_pend = (qx + qx_l) + qy + (qz + qz_km1);
    q_pend = q_old + e_pend;
    hx_km1 = Hx;
    hy_km1 = Hy;
    qz_km1 = qz;
    pxe_b = pxe_a;
    pxs_b = pxs_a;
    pye_b = pye_a;
    pys_b = pys_a;
    u11_b = u11;
    if (CPL) {
      b01 = a01;
      b10 = a10;
      b11 = a11;
    }
  }
  __syncthreads();
  if (accum && own) {  // Joule energy of the top plane k = nz
    const I id = id0 + (I)nz * plane;
    const R s = q_pend + sQy[ty - 1][tx];
    if (A.fold) {
      A.Q[id] += (double)s;
      A.Qs[id] = R(0);
    } else {
      A.Qs[id] = s;
    }
  }
  if (CPL && own) A.Pout[id0 + (I)nz * plane] = (e_pend + sQy[ty - 1][tx]) * A.inv_dt;
}

// One launch per step over all tiles; tiles in [ibx0, ibx1) x [iby0, iby1)
// take the interior specialisation.
template <typename R, typename I, int TX, int TY, bool CPL>
__global__ void __launch_bounds__(TX *TY, sizeof(R) == 4 ? COSIM_EM_MIN_CTAS * 8 / TY : 2)
    em_step_kernel(const __grid_constant__ EmArgs<R> A) {
  static_assert(TX == 32, "a tile row is one warp: x neighbours are exchanged by shuffles");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the launch adds 128 bytes so that the tables and stages can start on a
  // 128-byte boundary of the shared window (TMA destinations must)
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  R *s_cp = reinterpret_cast<R *>(smem);
  R *s_mt = s_cp + kCpmlTable;
  EmStage<R, TX, TY> *stg = reinterpret_cast<EmStage<R, TX, TY> *>(smem + em_stage_offset<R, TX, TY>(A.g.nmat));
  __shared__ R sHxz[2][TY][TX];  // Hx, Hz of the plane, read by the +y neighbour
  __shared__ R sQy[TY][TX];      // Joule share of the y-edge, read by the +y neighbour one plane later
  __shared__ uint64_t s_bar[kEmStages];  // one transaction barrier per stage
  __shared__ int s_abort;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    // TMA preconditions checked once per CTA: 128-byte aligned destinations
    // and 64-byte aligned descriptors; otherwise flag the error and leave
    // without issuing a copy
    bool ok = (smem_u32(stg) & 127u) == 0 && (sizeof(EmStage<R, TX, TY>) & 127u) == 0;
    for (int c = 0; c < 3; ++c)
      ok = ok && ((size_t)&A.tmE[c] & 63u) == 0 && ((size_t)&A.tmH[c] & 63u) == 0;
    ok = ok && ((size_t)&A.tmQ & 63u) == 0;
    s_abort = ok ? 0 : 1;
    if (!ok) atomicExch(A.err, 2);
    for (int q = 0; q < kEmStages; ++q) mbar_init(&s_bar[q], 1);
    fence_mbar_init();
  }
  stage_table(s_mt, A.g.mtab, (A.g.nmat + 1) * M_COLS);
  stage_table(s_cp, A.cpml, kCpmlTable);
  __syncthreads();
  if (s_abort) return;
  const bool interior = (int)blockIdx.x >= A.ibx0 && (int)blockIdx.x < A.ibx1 && (int)blockIdx.y >= A.iby0 &&
                        (int)blockIdx.y < A.iby1;
  if (interior)
    em_tile<R, I, TX, TY, false, CPL>(A, s_cp, s_mt, stg, sHxz, sQy, s_bar, &s_abort);
  else
    em_tile<R, I, TX, TY, true, CPL>(A, s_cp, s_mt, stg, sHxz, sQy, s_bar, &s_abort);
}

// advance the device-resident source time index after a group of steps
__global__ void step_advance_kernel(long long *step_base, long long n) { *step_base += n; }

}  // namespace cosim
