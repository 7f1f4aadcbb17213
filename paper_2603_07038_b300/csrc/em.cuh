// Fused leapfrog step of the Maxwell system (Sec. II-A, Eqs. 1-3 in E/H form)
// with the Joule heat of the step (P_total = D_sigma e^2), one launch per step.
//
// The node grid is cut into tiles of 31 x (TY-1) nodes in x-y; each CTA
// marches its tile (or, in the interior, a pair of x-adjacent tiles) through
// every node plane k = 0..nz. Its threads cover the tile plus one halo column
// (i-1) and row (j-1): at plane k a thread forms H^{n+1/2}(i,j,k) from E^n
// (own plane and plane k+1), shares it through shared memory, and forms
// E^{n+1} on its edges from the H of the node to its -x/-y side and from its
// own H of plane k-1 (kept in registers). Halo threads recompute the H and the
// single E edge their neighbours need (for Joule) but write nothing.
// E, H and the CPML auxiliaries are double-buffered (read *_o, write *_n), so
// CTAs never see each other's half-updated values.
//
// Interior tile pairs (every node off the lateral walls and outside the x/y
// CPML slabs) run two nodes per thread: a warp row covers 64 nodes (62 owned
// plus a halo pair), and the arithmetic of both nodes is issued as packed FP32
// instructions. The border tiles run one node per thread with the wall and
// lateral-CPML logic. Every formula is written once against the element-wise
// helpers of common.cuh. Runs of one launch shape are bitwise reproducible; a
// node that falls in a pair tile at one tile height and in a border tile at
// another agrees to FP32 rounding (packed products contracted into FMAs).
//
// Joule heat: the edge from node n to n+e_a dissipates sigma_e V_e ebar^2 in
// one step, ebar = (E^n + E^{n+1})/2; half of dt times that goes to each end
// node, i.e. (sum_c w_c sigma_c dt/2) * l_e * ebar^2 per end node, where w_c is
// the quarter cross-section of voxel c around the edge. The node sums the six
// halves of its incident edges (x from the node at i-1, y from j-1 through
// shared memory, z from its own previous plane) into a short-window
// accumulator that is folded into the FP64 total every few steps (FP64 runs at
// a small fraction of the FP32 rate on this GPU, so none is used per step).
//
// Inputs of planes k+1..k+2 are copied to shared memory by TMA (one thread
// issues a box per array and plane, completion tracked by one mbarrier per
// stage, four stages) while plane k is computed. Waits on those barriers are
// bounded: a copy that never arrives sets an error word instead of hanging.
//
// Material averaging (per edge: area-weighted eps, sigma over the <=4 voxels;
// per face: series mean of mu over the 2 voxels) is recomputed from the 1-byte
// voxel IDs every step instead of streaming per-edge coefficient arrays.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "common.cuh"
#include "thermal.cuh"

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
  // so in FP32 it is carried as an unevaluated pair chi = hi + lo updated
  // with error-free transformations. The x and y slabs (d = 0, 1: the border
  // tiles) keep one 16-byte record per element in xEo..xHn: FP32 {chi hi,
  // chi lo, dF^{n-1}, unused}, FP64 {chi, dF^{n-1}}, so that a state takes one
  // vector load, store or copy; dEo..lHn are null there. The z slab (d = 2,
  // mostly read by the pair tiles as x-adjacent node pairs) keeps separate
  // arrays: chi (hi) in xEo.., dF^{n-1} in dEo.., chi lo in lEo.. (null in
  // FP64 contexts).
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
  // precision); once per window of kJouleWindow steps the owner moves a node's
  // Qs into the FP64 total Q instead, so FP64 arithmetic runs once per window
  // rather than every step. The folds are spread over the window by plane:
  // fold = the step's position p in the window (-1: no fold, the kernel
  // parameter of batch launches instead), and node plane k folds when
  // (p + k) mod kJouleWindow = kJouleWindow - 1, so no step carries all of it.
  R *Qs;                      // null: not accumulating
  double *Q;
  int fold;
  // Tiling of the node grid. Rows of TY-1 owned nodes (row tile by owns
  // j = (TY-1) by .. (TY-1) by + TY - 2). In the rows [iby0, iby1) the nodes
  // xb0 .. xb1-1 (xb0 even, xb1 = xb0 + 62 npx) are owned by npx interior
  // pairs per row (CTAs n_border ..); the rest of those rows by nl border
  // tiles of up to 31 nodes from x = 0 and nr from x = xb1. Rows outside
  // [iby0, iby1) are cut into nbx border tiles of 31 nodes from x = 0.
  int nbx, xb0, xb1, npx, nl, nr, iby0, iby1, n_border;
  // TMA descriptors of E^n, H^{n-1/2} (per component) and Qs: 3-D node
  // arrays (x, y, z) with boxes of em_box_x x (TY+1 for E, TY otherwise) x 1
  // for border tiles and the *2 ones, em2_box_x wide, for interior pairs
  CUtensorMap tmE[3], tmH[3], tmQ;
  CUtensorMap tmE2[3], tmH2[3], tmQ2;
  CUtensorMap tmV, tmV2;  // voxel IDs (x, y, z), boxes em_vox_box_x / em2_vox_box_x x (TY+1) x 1
  // two-way coupling (the CPL specialisation, Sec. II-A): the temperature
  // rise T^n - T_init (node array, staged like E), the step's Joule power per
  // node written to Pout [W], 1 / dt
  CUtensorMap tmT, tmT2;
  R *Pout;
  R inv_dt;
  // the thermal step of the coupled path (Eq. 5 with the EM dt), fused into
  // the same launch: T^{n+1} - T_init written to Tth (the other temperature
  // buffer); T_amb as a rise over T_init; per-face film coefficients; the
  // maximum of the written rises goes to *peak as an order-preserving
  // integer image (null: not tracked)
  R *Tth;
  R T_amb;
  R hconv[6];
  unsigned long long *peak;
  const R *zt;      // per node plane: hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
  int *err;         // set to 1 when a bounded wait for a staged plane gave up
  long long wait;   // the bound of those waits, in SM clock cycles
};

// EM steps per short-window Joule accumulation (a power of two), and whether
// node plane kk folds its window at the step of window position `fold`
constexpr int kJouleWindow = 32;
static_assert((kJouleWindow & (kJouleWindow - 1)) == 0, "the Joule window is a power of two");
__device__ __forceinline__ bool plane_folds(int fold, int kk) {
  return fold >= 0 && ((fold + kk) & (kJouleWindow - 1)) == kJouleWindow - 1;
}

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

// The record layout of the x / y slab states: kPsiRec values of R per
// element (16 bytes), read and written as one vector.
template <typename R>
struct PsiVec;
template <>
struct PsiVec<float> {
  using T = float4;
};
template <>
struct PsiVec<double> {
  using T = double2;
};
template <typename R>
constexpr int kPsiRec = 16 / (int)sizeof(R);
template <typename R>
__device__ __forceinline__ void ld_rec(const R *p, R &hi, R &lo, R &d) {
  const typename PsiVec<R>::T v = *reinterpret_cast<const typename PsiVec<R>::T *>(p);
  if constexpr (sizeof(R) == 4) {
    hi = v.x, lo = v.y, d = v.z;
  } else {
    hi = v.x, lo = R(0), d = v.y;
  }
}
template <typename R>
__device__ __forceinline__ void st_rec(R *p, R hi, R lo, R d) {
  typename PsiVec<R>::T v;
  if constexpr (sizeof(R) == 4) {
    v = make_float4(hi, lo, d, 0.0f);
  } else {
    v = make_double2(hi, d);
  }
  *reinterpret_cast<typename PsiVec<R>::T *>(p) = v;
}

// CPML state of one derivative at element q of the slab arrays of axis d,
// slot `slot` (V: one node, or an x-adjacent node pair at an even q): chi,
// its low part (FP32 contexts) and the previous derivative. The loads of a
// plane's states are issued together, ahead of their use, so that their
// latencies overlap.
template <typename V>
struct ChiIn {
  V hi, lo, d;
};
template <typename V>
struct Psi {
  int s;        // slab position, -1: none (no state is read or written)
  long long q;  // element of the slab arrays
  ChiIn<V> c;
};
template <typename R, typename V>
__device__ __forceinline__ Psi<V> psi_pre(const EmArgs<R> &A, int d, int type, int slot, int s, long long q) {
  Psi<V> p;
  p.s = s;
  p.q = q;
  if (s >= 0) {
    if (d < 2) {  // a record (single nodes only: the pair tiles hold no x / y slab node)
      static_assert(sizeof(V) == sizeof(R) || sizeof(V) == 2 * sizeof(R), "one node or a node pair");
      if constexpr (sizeof(V) == sizeof(R))
        ld_rec<R>((type == 0 ? A.xEo[d][slot] : A.xHo[d][slot]) + q * kPsiRec<R>, p.c.hi, p.c.lo, p.c.d);
    } else {
      p.c.hi = ldv_<V>((type == 0 ? A.xEo[d][slot] : A.xHo[d][slot]) + q);
      p.c.d = ldv_<V>((type == 0 ? A.dEo[d][slot] : A.dHo[d][slot]) + q);
      if constexpr (sizeof(R) == 4) p.c.lo = ldv_<V>((type == 0 ? A.lEo[d][slot] : A.lHo[d][slot]) + q);
    }
  }
  return p;
}

// chi^n = b (chi^{n-1} + dF^n - dF^{n-1}), omb = 1 - b, from the state in p;
// returns chi^n = dF + psi (the derivative itself outside the slabs); the
// owner writes the new state.
template <typename R, typename V>
__device__ __forceinline__ V psi_apply(const EmArgs<R> &A, V omb, int d, int type, int slot, const Psi<V> &p, V deriv,
                                       bool write) {
  static_assert(sizeof(V) == sizeof(R), "one node at a time");
  if (p.s < 0) return deriv;
  const long long q = p.q;
  R *xn = type == 0 ? A.xEn[d][slot] : A.xHn[d][slot];
  R *dn = type == 0 ? A.dEn[d][slot] : A.dHn[d][slot];
  if constexpr (sizeof(R) == 8) {
    const V t = add_(p.c.hi, sub_(deriv, p.c.d));
    const V chi = fma_(neg_(omb), t, t);
    if (write) {
      if (d < 2) {
        st_rec<R>(xn + q * kPsiRec<R>, chi, R(0), deriv);
      } else {
        stv_(xn + q, chi);
        stv_(dn + q, deriv);
      }
    }
    return chi;
  } else {
    // (hi + lo + D)(1 - omb) with Knuth's TwoSum for hi + D, an FMA product
    // error for omb * sh, Dekker's Fast2Sum for sh - omb sh (exact: omb is in
    // [0, 1), so |omb sh| <= |sh|) and a final renormalisation (Fast2Sum).
    const V hi = p.c.hi, lo = p.c.lo;
    const V D = sub_(deriv, p.c.d);
    const V sh = add_(hi, D);
    const V bv = sub_(sh, hi);
    const V e1 = add_(sub_(hi, sub_(sh, bv)), sub_(D, bv));
    const V l1 = add_(lo, e1);
    const V pr = mul_(omb, sh);
    const V pe = fma_(omb, sh, neg_(pr));
    const V s2 = sub_(sh, pr);
    const V e2 = sub_(neg_(pr), sub_(s2, sh));
    const V l2 = sub_(sub_(add_(l1, e2), pe), mul_(omb, l1));
    const V h3 = add_(s2, l2);
    const V l3 = sub_(l2, sub_(h3, s2));
    if (write) {
      if (d < 2) {
        st_rec<R>(xn + q * kPsiRec<R>, h3, l3, deriv);
      } else {
        stv_(xn + q, h3);
        stv_((type == 0 ? A.lEn[d][slot] : A.lHn[d][slot]) + q, l3);
        stv_(dn + q, deriv);
      }
    }
    return h3;
  }
}

// (dF1 + psi1) - (dF2 + psi2) of one curl component of a single node: the
// first derivative's state is in slot 1, the second's in slot 0
template <typename R>
__device__ __forceinline__ R curl_psi(const EmArgs<R> &A, const R *s_cp, int type, int d1, const Psi<R> &p1, int d2,
                                      const Psi<R> &p2, R v1, R v2, bool write) {
  const R a = p1.s >= 0 ? psi_apply<R, R>(A, s_cp[(d1 * 2 + type) * kMaxSlab + p1.s], d1, type, 1, p1, v1, write) : v1;
  const R b = p2.s >= 0 ? psi_apply<R, R>(A, s_cp[(d2 * 2 + type) * kMaxSlab + p2.s], d2, type, 0, p2, v2, write) : v2;
  return sub_(a, b);
}

static_assert(M_EPS == 0 && M_SDT2 == 1 && M_IMU == 2 && M_COLS % 4 == 0,
              "the EM kernel reads eps, sigma dt/2, 1/mu of a material row with one aligned vector load");
static_assert(M_TC0 == M_TCR + 1 && M_TCR % 2 == 0, "alpha and its offset are read as one aligned pair");
// Four consecutive values from 16-byte aligned shared memory in one vector load.
__device__ __forceinline__ void load4(const float *p, float &a, float &b, float &c, float &d) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  a = v.x, b = v.y, c = v.z, d = v.w;
}
__device__ __forceinline__ void load4(const double *p, double &a, double &b, double &c, double &d) {
  const double2 v = reinterpret_cast<const double2 *>(p)[0], w = reinterpret_cast<const double2 *>(p)[1];
  a = v.x, b = v.y, c = w.x, d = w.y;
}

// E^{n+1} of an edge (V: one node or a node pair) from the area-weighted sums
// over its <= 4 voxels, all taken without the quarter factor of the voxel
// cross-sections (it cancels):
//   Se = sum w eps, Ss = sum w sigma dt/2 (w = product of the two transverse
//   cell sizes of the voxel), dtW = dt x (sum of those products) = 4 dt x the
//   dual-face area, lq = edge length / 4.
// The update E' = ca E + cb (curl - J) (ca = (Se - Ss)/(Se + Ss),
// cb = dt W/(Se + Ss)) is evaluated in the equivalent incremental form
// E' = E + r (dtW (curl - J) - 2 Ss E), r = 1/(Se + Ss), which keeps the decay
// 1 - ca of weakly lossy media at full precision. *half_q receives the edge's
// Joule energy per end node, (Ss/4) l ebar^2 with ebar = (E + E')/2.
template <typename V, typename R>
__device__ __forceinline__ V e_update(V e_old, V dtW, V drive, V Se, V Ss, V lq, V *half_q) {
  const V r = rcp_(add_(Se, Ss));
  const V t = fma_(dtW, drive, mul_(mul_(bc_<V>(R(-2)), Ss), e_old));
  const V e_new = fma_(r, t, e_old);
  const V eb = mul_(bc_<V>(R(0.5)), add_(e_old, e_new));
  *half_q = mul_(mul_(mul_(Ss, lq), eb), eb);
  return e_new;
}

// H^{n+1/2} = H^{n-1/2} - (dt/2 / dual length) (series mean of 1/mu) curl:
// hd = dt/2 x the inverse dual length, (ha, ua), (hb, ub) the two voxels'
// lengths along the dual edge and their 1/mu.
template <typename V>
__device__ __forceinline__ V h_update(V h_old, V hd, V ha, V ua, V hb, V ub, V curl) {
  return fma_(neg_(mul_(hd, fma_(ha, ua, mul_(hb, ub)))), curl, h_old);
}

// The sum over an edge's four voxels of w_c sigma_c(T) dt/2, with a_c = w_c
// M_SDT2_c and d_c = M_TC0_c + M_TCR_c te, over a common denominator so that
// one reciprocal serves the edge instead of one per voxel:
//   sum a_c / d_c = ((a1 d2 + a2 d1) d3 d4 + (a3 d4 + a4 d3) d1 d2) / (d1 d2 d3 d4).
// (Every d_c is positive: 1 for temperature-independent materials and for the
// zero row that stands for voxels outside the grid.)
template <typename V>
__device__ __forceinline__ V sig_sum4(V a1, V d1, V a2, V d2, V a3, V d3, V a4, V d4) {
  const V p12 = mul_(d1, d2), p34 = mul_(d3, d4);
  const V n12 = fma_(a1, d2, mul_(a2, d1)), n34 = fma_(a3, d4, mul_(a4, d3));
  return mul_(fma_(n12, p34, mul_(n34, p12)), rcp_(mul_(p12, p34)));
}

// Peak-temperature snapshots of the coupled marching. pk[0]: the maximum
// rise of the current check step (image); pk[1]: the highest recorded; pk[2]:
// 1 if the check step set a new peak; pk[3]: the number of peaks recorded;
// pk[4]: the step count of the recorded peak.
__global__ void peak_check_kernel(unsigned long long *pk, long long step) {
  const bool up = pk[0] > pk[1];
  if (up) {
    pk[1] = pk[0];
    pk[3] += 1;
    pk[4] = (unsigned long long)step;
  }
  pk[2] = up ? 1ull : 0ull;
  pk[0] = 0;  // the smallest image: the next check step starts afresh
}
// copy the temperature field into the snapshot when the check set a new peak
template <typename R>
__global__ void __launch_bounds__(256) peak_snapshot_kernel(long long n, const unsigned long long *pk, const R *T,
                                                            R *Tpk) {
  if (pk[2] == 0) return;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  for (long long q = first; q < n; q += stride) Tpk[q] = T[q];
}

// derivative (b - a) / h
template <typename V>
__device__ __forceinline__ V dif_(V b, V a, V ih) {
  return mul_(sub_(b, a), ih);
}

// One plane of the CTA's inputs, staged in shared memory by TMA: E^n of the
// tile plus its +x/+y neighbours, H^{n-1/2} and the Joule accumulator. A TMA
// box must start at an x coordinate that is a multiple of 16 bytes, so the
// box starts at the tile's first node rounded down to a multiple of 4 and is
// TX + 4 nodes wide; threads index it from that remainder.
template <int TX>
__host__ __device__ constexpr int em_box_x() { return TX + 4; }
// voxel box: columns i0-1 .. i0+TX-1 from x rounded down to 16 bytes
template <int TX>
__host__ __device__ constexpr int em_vox_box_x() { return (TX + 1 + 15 + 15) / 16 * 16; }
// source-row box: rows j0 .. j0+TY (+1 for the end offset) from a multiple of 4
template <int TY>
__host__ __device__ constexpr int em_src_box() { return (TY + 1 + 3 + 3) / 4 * 4; }
// interior pairs: 64 nodes per warp row (+ the +x neighbour, + the rounding)
constexpr int kEm2Nodes = 64;
__host__ __device__ constexpr int em2_box_x() { return em_box_x<kEm2Nodes>(); }
__host__ __device__ constexpr int em2_vox_box_x() { return em_vox_box_x<kEm2Nodes>(); }
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
template <typename R>
__host__ __device__ constexpr size_t em_stage_offset(int nmat) {
  return ((kCpmlTable + (size_t)(nmat + 1) * M_COLS) * sizeof(R) + 127) & ~size_t(127);
}
// bytes of one stage slot: large enough for either tile kind
template <typename R, int TY>
__host__ __device__ constexpr size_t em_stage_bytes() {
  return sizeof(EmStage<R, kEm2Nodes, TY>) > sizeof(EmStage<R, 32, TY>) ? sizeof(EmStage<R, kEm2Nodes, TY>)
                                                                        : sizeof(EmStage<R, 32, TY>);
}

// Shared-memory stages (a power of two) and the prefetch distance: at plane k
// the copy of plane k + kEmAhead is issued and planes k, k+1 must have landed.
#ifndef COSIM_EM_STAGES
#define COSIM_EM_STAGES 4
#endif
#ifndef COSIM_EM_AHEAD
#define COSIM_EM_AHEAD 2
#endif
#ifndef COSIM_EM_MIN_CTAS
#define COSIM_EM_MIN_CTAS 2  // resident CTAs of 8 warps per SM the FP32 kernel is compiled for (scaled for other heights)
#endif
constexpr int kEmStages = COSIM_EM_STAGES;
constexpr int kEmAhead = COSIM_EM_AHEAD;
static_assert((kEmStages & (kEmStages - 1)) == 0, "stage count must be a power of two");
static_assert(kEmAhead >= 2 && kEmAhead <= kEmStages - 1, "prefetch distance must leave the stage of plane k-1 free");
// Border tiles (FP32) keep the H side's CPML states of the next plane in a
// per-thread shared-memory ring filled by cp.async: 2 planes x 6 states x
// one 16-byte slot (chi high, chi low, previous derivative, unused).
constexpr int kPsiH = 6;
template <typename R, int TY>
__host__ __device__ constexpr size_t em_psi_ring_bytes() {
  return sizeof(R) == 4 ? (size_t)32 * TY * 2 * kPsiH * 4 * sizeof(R) : 0;
}
template <typename R, int TY>
__host__ __device__ constexpr size_t em_smem_bytes(int nmat) {
  return em_stage_offset<R>(nmat) +
         (kEmStages * em_stage_bytes<R, TY>() > kEmStages * sizeof(EmStage<R, 32, TY>) + em_psi_ring_bytes<R, TY>()
              ? kEmStages * em_stage_bytes<R, TY>()
              : kEmStages * sizeof(EmStage<R, 32, TY>) + em_psi_ring_bytes<R, TY>()) +
         128;  // + alignment slack
}

// Bounded waits for the planes a CTA reads at plane k: plane k+1 (plane k was
// waited for one plane earlier, plane 0 before the loop). Sets *s_abort when
// a copy did not arrive in time.
__device__ __forceinline__ void em_wait_next(uint64_t *bars, int k, int nz, int *s_abort, long long lim) {
  if (k + 1 <= nz && !mbar_wait(&bars[(k + 1) & (kEmStages - 1)], (unsigned)((k + 1) / kEmStages) & 1u, lim))
    *s_abort = 1;
}
// after a failed wait at plane k: let the copies issued so far (planes up to
// k + kEmAhead) land (bounded), flag the error and let the CTA leave
__device__ __forceinline__ void em_abort(uint64_t *bars, int k, int nz, int *err, long long lim) {
  for (int q = k; q <= k + kEmAhead && q <= nz; ++q)
    mbar_wait(&bars[q & (kEmStages - 1)], (unsigned)(q / kEmStages) & 1u, lim);
  atomicExch(err, 1);
}

// ---- border tiles: one node per thread. The tile starting at node xs of row
// tile by owns the nodes i = xs .. min(xs + 30, xe - 1), j = (TY-1) by ..
// (TY-1) by + TY - 2; thread (tx, ty) holds node (xs - 1 + tx, (TY-1) by - 1
// + ty). Nodes outside the grid, on the walls and inside the CPML slabs are
// all handled here. XS / YS: the tile may hold nodes of an x / y slab (when
// false, that axis's CPML code is left out of the instantiation).
template <typename R, typename I, int TY, bool CPL, bool TH, bool XS, bool YS>
__device__ __forceinline__ void em_tile_border(const EmArgs<R> &A, const R *s_cp, const R *s_mt,
                                               EmStage<R, 32, TY> *stg, R (*sHxz)[2][TY][32], R (*sQy)[TY][32],
                                               uint64_t *bars, int *s_abort, int xs, int xe, int by, int step_off,
                                               int fold) {
  constexpr int TX = 32;
  const Geo<R> &g = A.g;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int vd = g.nmat * M_COLS;  // row offset of the all-zero material
  const int i0 = xs - 1, j0 = by * (TY - 1) - 1;  // node of thread (0, 0)
  const int i = i0 + tx, j = j0 + ty;
  const bool act = i >= 0 && i <= nx && j >= 0 && j <= ny;
  const bool own = act && tx > 0 && ty > 0 && i < xe;
  const bool need_ex = act && ty > 0 && i < nx;  // own, or the halo column
  const bool need_ey = act && tx > 0 && j < ny;  // own, or the halo row
  const bool in_x = i < nx, in_y = j < ny;
  const bool accum = A.Qs != nullptr;

  // Plane k of E^n (tile + neighbours), H^{n-1/2}, Qs, voxels, z record and
  // source rows -> stage k mod kEmStages, by TMA: one thread announces the
  // bytes on the stage's mbarrier and issues the copies; positions outside the
  // grid arrive as zero. Box x starts at the tile's first node rounded down to
  // a multiple of 4 (two's complement: i0 = -1 gives x0 = -4); threads read
  // from column tx + xr.
  const int xr = i0 & 3, x0 = i0 - xr;
  const bool leader = tx == 0 && ty == 0;
  // The voxel box starts at column i0 - 1 rounded down to 16 bytes, the
  // source-row box at entry k (ny+1) + j0 rounded down to 4 ints.
  const int xvr = (i0 - 1) & 15, xv0 = (i0 - 1) - xvr;
  const bool has_src = A.src_row != nullptr;
  // transaction bytes of one stage: the boxes themselves, not their padding
  const unsigned stage_bytes =
      (unsigned)((6 * TY + 3 + (accum ? TY : 0) + (CPL ? TY + 1 : 0)) * em_box_x<TX>() * (int)sizeof(R) +
                 4 * (int)sizeof(R) + (has_src ? em_src_box<TY>() * 4 : 0) + (TY + 1) * em_vox_box_x<TX>());
  auto issue = [&](int k) {
    if (k > nz) return;
    const int s = k & (kEmStages - 1);
    EmStage<R, TX, TY> &S = stg[s];
    mbar_arrive_expect_tx(&bars[s], stage_bytes);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      tma_load_3d(&S.E[c].v[0][0], &A.tmE[c], x0, j0, k, &bars[s]);
      tma_load_3d(&S.H[c].v[0][0], &A.tmH[c], x0, j0, k, &bars[s]);
    }
    if (accum) tma_load_3d(&S.Qs.v[0][0], &A.tmQ, x0, j0, k, &bars[s]);
    if (CPL) tma_load_3d(&S.T.v[0][0], &A.tmT, x0, j0, k, &bars[s]);
    // the voxel layer above plane k; at k = nz the box lies above the grid
    // and arrives as zeros (the thread masks select the zero material row)
    tma_load_3d(&S.V.v[0][0], &A.tmV, xv0, j0 - 1, k, &bars[s]);
    bulk_load(&S.Z.v[0][0], A.zt + 4 * (size_t)k, 4 * sizeof(R), &bars[s]);
    if (has_src) {  // 16-byte aligned: src_row itself is, the start is a multiple of 4 from -4
      const int base = k * (ny + 1) + j0;
      bulk_load(&S.S.v[0][0], A.src_row + (base - (base & 3)), em_src_box<TY>() * 4, &bars[s]);
    }
  };
  const I plane = (I)g.plane;
  const I id0 = act ? (I)g.nid(i, j, 0) : I(0);
  // Material rows (id x M_COLS) of voxels (i-1+dx, j-1+dy, k) from the staged
  // voxel box; the zero row outside the grid.
  const bool cx0 = i - 1 >= 0 && i - 1 < nx, cx1 = i >= 0 && i < nx;
  const bool cy0 = j - 1 >= 0 && j - 1 < ny, cy1 = j >= 0 && j < ny;
  const int cv = tx + xvr;  // column of voxel i-1 in the box

  const R hxm = (act && i > 0) ? g.h[0][i - 1] : R(0), hx0 = (act && in_x) ? g.h[0][i] : R(0);
  const R hym = (act && j > 0) ? g.h[1][j - 1] : R(0), hy0 = (act && in_y) ? g.h[1][j] : R(0);
  const R ihx = (act && in_x) ? g.ih[0][i] : R(0), ihy = (act && in_y) ? g.ih[1][j] : R(0);
  const R idx = act ? g.idual[0][i] : R(0), idy = act ? g.idual[1][j] : R(0);
  const bool fix_x = (i == 0 && A.fixlo[0]) || (i == nx && A.fixhi[0]);
  const bool fix_y = (j == 0 && A.fixlo[1]) || (j == ny && A.fixhi[1]);
  // CPML slab positions along x and y (E: nodes, H: cells); none inside
  const int sxE = XS ? slab_index(i, nx, A.slo[0], A.shi[0]) : -1;
  const int syE = YS ? slab_index(j, ny, A.slo[1], A.shi[1]) : -1;
  const int sxH = in_x ? sxE : -1;
  const int syH = in_y ? syE : -1;
  const R dt = A.dt;
  const R half_dt = mul_(R(0.5), dt);
  // per-thread geometry of the face and edge coefficients
  const R hdx = mul_(half_dt, idx), hdy = mul_(half_dt, idy);
  const R dtWx_y = mul_(dt, add_(hym, hy0)), dtWy_x = mul_(dt, add_(hxm, hx0));
  const R lqx = mul_(R(0.25), hx0), lqy = mul_(R(0.25), hy0);
  // this node's element of the slab arrays (the layout of psi_index) in the
  // index type: x and y slabs at plane 0 plus kk planes, z slab at position
  // 0 plus s positions (each slab array is smaller than a padded node array)
  const I qx0 = (I)j * (I)A.sn[0] + (I)sxE, qxs = (I)(ny + 1) * (I)A.sn[0];
  const I qy0 = (I)syE * (I)g.px + (I)i, qys = (I)A.sn[1] * (I)g.px;
  const I qz0 = (I)j * (I)g.px + (I)i, qzs = (I)(ny + 1) * (I)g.px;
  auto qof = [&](int d, int s, int kk) -> long long {
    return d == 0 ? (long long)(qx0 + (I)kk * qxs) : d == 1 ? (long long)(qy0 + (I)kk * qys) : (long long)(qz0 + (I)s * qzs);
  };
  auto psi_at = [&](int d, int type, int slot, int s, int kk) -> Psi<R> {
    return psi_pre<R, R>(A, d, type, slot, s, s >= 0 ? qof(d, s, kk) : 0);
  };

  // The H side's CPML states of plane kk (d, slot; slab position s or -1):
  // Hx (y: slot 1, z: slot 0), Hy (z: slot 1, x: slot 0), Hz (x: slot 1,
  // y: slot 0). FP32 border tiles request them one plane ahead by cp.async
  // into this thread's slots of the ring behind the stages.
  auto h_state = [&](int e, int kk, int &d, int &slot, bool plain = false) -> int {
    const bool kzz = plain || kk < nz;
    const int szz = plain ? -1 : kzz ? slab_index(kk, nz, A.slo[2], A.shi[2]) : -1;
    const bool hx_on = act && in_y && kzz, hy_on = act && in_x && kzz, hz_on = act && in_x && in_y && kk <= nz;
    switch (e) {
      case 0: d = 1, slot = 1; return hx_on ? syH : -1;
      case 1: d = 2, slot = 0; return hx_on ? szz : -1;
      case 2: d = 2, slot = 1; return hy_on ? szz : -1;
      case 3: d = 0, slot = 0; return hy_on ? sxH : -1;
      case 4: d = 0, slot = 1; return hz_on ? sxH : -1;
      default: d = 1, slot = 0; return hz_on ? syH : -1;
    }
  };
  R *ring = reinterpret_cast<R *>(stg + kEmStages) + (ty * 32 + tx) * (2 * kPsiH * 4);
  auto prefetch_h = [&](int kk) {
    if constexpr (sizeof(R) == 4) {
      R *r = ring + (kk & 1) * (kPsiH * 4);
#pragma unroll
      for (int e = 0; e < kPsiH; ++e) {
        int d, slot;
        const int sp = h_state(e, kk, d, slot);
        if (sp >= 0) {
          const long long q = qof(d, sp, kk);
          if (d < 2) {  // the record
            cp_async<16>(r + 4 * e, A.xHo[d][slot] + q * kPsiRec<R>, true);
          } else {
            cp_async<4>(r + 4 * e, A.xHo[d][slot] + q, true);
            cp_async<4>(r + 4 * e + 1, A.lHo[d][slot] + q, true);
            cp_async<4>(r + 4 * e + 2, A.dHo[d][slot] + q, true);
          }
        }
      }
      cp_async_commit();
    }
  };

  if (leader) {
#pragma unroll
    for (int q = 0; q < kEmAhead; ++q) issue(q);
  }
  prefetch_h(0);
  if (!mbar_wait(&bars[0], 0u, A.wait)) *s_abort = 1;
  R hx_km1 = 0, hy_km1 = 0, qz_km1 = 0;
  // layer k-1 partial sums of the x / y edges and 1/mu of voxel (i, j, k-1);
  // zero below the grid
  R pxe_b = 0, pxs_b = 0, pye_b = 0, pys_b = 0, u11_b = 0;
  R q_pend = 0;  // Joule sum of node (i, j, k-1) still missing the y-edge share from j-1
  R e_pend = 0;  // the same without the accumulator's earlier energy (this step's only)
  int b00 = vd, b01 = vd, b10 = vd, b11 = vd;  // coupled steps: material rows of layer k-1
  // coupled steps: sigma dt/2 of voxel `row` (returned) and its denominator
  // M_TC0 + M_TCR te (in d), for sig_sum4
  auto sgd = [&](int row, R te, R &d) -> R {
    d = fma_(s_mt[row + M_TCR], te, s_mt[row + M_TC0]);
    return s_mt[row + M_SDT2];
  };
  // TH (coupled steps with the thermal step in the same launch): node (i, j,
  // k-1) takes its step at the start of plane k, from plane k-1's stage
  // (still resident until plane k's barrier: its temperatures and z record),
  // T at plane k, the layer sums of voxel layer k-2 (carried) and k-1 (rows
  // b), and its Joule energy of the step without the y-edge share of row j-1;
  // that share becomes visible with plane k's barrier and completes T^{n+1}
  // and P^{n+1}. The node column's constants (th_column) come from the tile's
  // own geometry: only the lateral film and the inverse sizes of cells i-1,
  // j-1 are kept.
  static_assert(CPL || !TH, "the fused thermal step belongs to coupled steps");
  R fxy_th = 0, ihxm_th = 0, ihym_th = 0;
  if (TH) {
    const ThCol<R> c0 = th_column_h(g, A.hconv, i, j);
    fxy_th = c0.fxy;
    ihxm_th = (act && i > 0) ? g.ih[0][i - 1] : R(0);
    ihym_th = (act && j > 0) ? g.ih[1][j - 1] : R(0);
  }
  auto tcol_of = [&]() -> ThCol<R> {
    ThCol<R> c;
    c.hxm = hxm, c.hx0 = hx0, c.hym = hym, c.hy0 = hy0;
    c.qxm = mul_(R(0.25), ihxm_th), c.qx0 = mul_(R(0.25), ihx);
    c.qym = mul_(R(0.25), ihym_th), c.qy0 = mul_(R(0.25), ihy);
    c.fxy = fxy_th;
    c.az = mul_(R(0.25), mul_(add_(hxm, hx0), add_(hym, hy0)));
    return c;
  };
  ThLayer<R> tl_lo = th_layer_zero<R, R>();  // sums of voxel layer k-2
  R th_m2 = 0, gz_th = 0;                    // T of (i, j, k-2); the conductance of the z edge below node k-1
  R t_max = R(-3.0e38);
  // the thermal step of node (i, j, kk) from plane kk's stage Sm (its
  // temperatures and z record), T at plane kk+1 (tkp), the layer sums of voxel
  // layers kk-1 (tl_lo) and kk (up), and the step's power without the y-edge
  // share of row j-1 (e_pend): returns T + dt/C (flux + P_partial) in tpart and
  // dt/C in dtc; the share is added once the plane's barrier has made it visible
  auto th_partial = [&](const EmStage<R, TX, TY> &Sm, int kk, const ThLayer<R> &up, R tkp, R &tpart, R &dtc) {
    const int cx = tx + xr;
    const ThCoeffs<R> q = th_coeffs<R, R>(tcol_of(), tl_lo, up, Sm.Z.v[0][0], Sm.Z.v[0][1], Sm.Z.v[0][3], kk == 0,
                                          kk == nz, A.hconv, gz_th);
    const R tc = Sm.T.v[ty][cx];
    if (own) {
      dtc = mul_(A.dt, rcp_(q.C));
      const R p = mul_(e_pend, A.inv_dt);
      R f = fma_(q.Gxm, sub_(Sm.T.v[ty][cx - 1], tc), p);  // owners: tx, ty >= 1, so cx - 1, ty - 1 exist
      f = fma_(q.Gxp, sub_(Sm.T.v[ty][cx + 1], tc), f);
      f = fma_(q.Gym, sub_(Sm.T.v[ty - 1][cx], tc), f);
      f = fma_(q.Gyp, sub_(Sm.T.v[ty + 1][cx], tc), f);
      f = fma_(q.Gzm, sub_(th_m2, tc), f);
      f = fma_(q.Gzp, sub_(tkp, tc), f);
      f = fma_(q.film, sub_(A.T_amb, tc), f);
      tpart = fma_(dtc, f, tc);
    }
    th_m2 = tc;
    tl_lo = up;
  };
  // the share of row j-1 (energy) completes node kk's step and power
  auto th_finish = [&](I idn, R share, R tpart, R dtc) {
    const R pw = mul_(add_(e_pend, share), A.inv_dt);
    A.Pout[idn] = pw;
    const R tn = fma_(dtc, mul_(share, A.inv_dt), tpart);
    A.Tth[idn] = tn;
    t_max = fmax(t_max, tn);
  };

  // The plane body, compiled twice as in the pair tiles: PL for the planes
  // 0 < k < nz outside the z slabs, the general copy for the others. Returns
  // false when the CTA must leave.
  auto plane_body = [&](const int k, auto plain_tag) -> bool {
    constexpr bool PL = decltype(plain_tag)::value;
    if (leader) {  // the stage of plane k-1 is free: every thread passed the last barrier
      fence_proxy_async_smem();
      issue(k + kEmAhead);
    }
    em_wait_next(bars, k, nz, s_abort, A.wait);
    prefetch_h(k + 1);
    const int par = k & 1;  // parity of the double-buffered exchange arrays
    const I id = id0 + (I)k * plane;
    const EmStage<R, TX, TY> &S0 = stg[k & (kEmStages - 1)];
    const EmStage<R, TX, TY> &S1 = stg[(k + 1) & (kEmStages - 1)];
    R hz0, ihz, idz, hzm;
    load4(&S0.Z.v[0][0], hz0, ihz, idz, hzm);
    // material rows of voxel layer k (the layer above node plane k)
    const bool kz = PL || k < nz;
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
    const R hdz = mul_(half_dt, idz);
    const bool fix_z = !PL && ((k == 0 && A.fixlo[2]) || (k == nz && A.fixhi[2]));
    const int szE = PL ? -1 : slab_index(k, nz, A.slo[2], A.shi[2]);

    const int cx = tx + xr;  // this node's column in the staged boxes
    const R ex = S0.E[0].v[ty][cx], ey = S0.E[1].v[ty][cx], ez = S0.E[2].v[ty][cx];
    const R ex_up = S1.E[0].v[ty][cx], ey_up = S1.E[1].v[ty][cx];
    const R ez_jp = S0.E[2].v[ty + 1][cx], ex_jp = S0.E[0].v[ty + 1][cx];
    const R ez_ip = S0.E[2].v[ty][cx + 1], ey_ip = S0.E[1].v[ty][cx + 1];
    const R hx_o = S0.H[0].v[ty][cx], hy_o = S0.H[1].v[ty][cx], hz_o = S0.H[2].v[ty][cx];
    const R q_old = accum ? S0.Qs.v[ty][cx] : R(0);
    // coupled steps: temperature rise at this node and its +x, +y, +z neighbours
    R th = 0, th_ip = 0, th_jp = 0, th_kp = 0;
    R t_part = 0, t_dtc = 0;  // node (i, j, k-1)'s thermal step without the y-edge share of row j-1
    if (CPL) {
      th = S0.T.v[ty][cx];
      th_ip = S0.T.v[ty][cx + 1];
      th_jp = S0.T.v[ty + 1][cx];
      th_kp = kz ? S1.T.v[ty][cx] : R(0);
      if (TH && (PL || k > 0)) {  // plane k-1's stage is resident until this plane's barrier
        const ThLayer<R> up = th_layer<R>(s_mt[b00 + M_K], s_mt[b01 + M_K], s_mt[b10 + M_K], s_mt[b11 + M_K],
                                          s_mt[b00 + M_RHOCP], s_mt[b01 + M_RHOCP], s_mt[b10 + M_RHOCP],
                                          s_mt[b11 + M_RHOCP], tcol_of());
        th_partial(stg[(k - 1) & (kEmStages - 1)], k - 1, up, th, t_part, t_dtc);
      }
    }

    // material constants of voxel layer k
    // (columns M_EPS, M_SDT2, M_IMU, M_K are adjacent: one vector load per voxel)
    R e00, s00, u00, k00, e01, s01, u01, k01, e10, s10, u10, k10, e11, s11, u11, k11;
    load4(s_mt + a00, e00, s00, u00, k00);
    load4(s_mt + a01, e01, s01, u01, k01);
    load4(s_mt + a10, e10, s10, u10, k10);
    load4(s_mt + a11, e11, s11, u11, k11);

    // ---- H^{n+1/2} at (i,j,k); dt/mu of a face is the series mean over the
    // two voxels its dual edge crosses
    const bool hx_on = act && in_y && kz, hy_on = act && in_x && kz, hz_on = act && in_x && in_y;
    Psi<R> ph[kPsiH];
    if constexpr (sizeof(R) == 4) {  // this plane's states landed in the ring (the group of plane k+1 may still fly)
      cp_async_wait<1>();
      const R *r = ring + (k & 1) * (kPsiH * 4);
#pragma unroll
      for (int e = 0; e < kPsiH; ++e) {
        int d, slot;
        ph[e].s = h_state(e, k, d, slot, PL);
        ph[e].q = ph[e].s >= 0 ? qof(d, ph[e].s, k) : 0;
        const float4 v = *reinterpret_cast<const float4 *>(r + 4 * e);
        ph[e].c.hi = v.x;
        ph[e].c.lo = v.y;
        ph[e].c.d = v.z;
      }
    } else {
#pragma unroll
      for (int e = 0; e < kPsiH; ++e) {
        int d, slot;
        const int sp = h_state(e, k, d, slot, PL);
        ph[e] = psi_at(d, 1, slot, sp, k);
      }
    }
    const Psi<R> &pHx1 = ph[0], &pHx2 = ph[1], &pHy1 = ph[2], &pHy2 = ph[3], &pHz1 = ph[4], &pHz2 = ph[5];
    R Hx = 0, Hy = 0, Hz = 0;
    if (hx_on)  // Hx: (curl E)_x = dEz/dy - dEy/dz, voxels (i-1..i, j, k)
      Hx = h_update(hx_o, hdx, hxm, u10, hx0, u11,
                    curl_psi(A, s_cp, 1, 1, pHx1, 2, pHx2, dif_(ez_jp, ez, ihy), dif_(ey_up, ey, ihz), own));
    if (hy_on)  // Hy: dEx/dz - dEz/dx, voxels (i, j-1..j, k)
      Hy = h_update(hy_o, hdy, hym, u01, hy0, u11,
                    curl_psi(A, s_cp, 1, 2, pHy1, 0, pHy2, dif_(ex_up, ex, ihz), dif_(ez_ip, ez, ihx), own));
    if (hz_on)  // Hz: dEy/dx - dEx/dy, voxels (i, j, k-1..k)
      Hz = h_update(hz_o, hdz, hzm, u11_b, hz0, u11,
                    curl_psi(A, s_cp, 1, 0, pHz1, 1, pHz2, dif_(ey_ip, ey, ihx), dif_(ex_jp, ex, ihy), own));
    sHxz[par][0][ty][tx] = Hx;
    sHxz[par][1][ty][tx] = Hz;
    const R hy_l = __shfl_up_sync(0xffffffffu, Hy, 1);  // H of node i-1 (same warp)
    const R hz_l = __shfl_up_sync(0xffffffffu, Hz, 1);
    // the E side's CPML states, in flight across the barrier
    const bool ex_on = need_ex && !(fix_y || fix_z), ey_on = need_ey && !(fix_x || fix_z);
    const bool ez_on = own && kz && !(fix_x || fix_y);
    const Psi<R> pEx1 = psi_at(1, 0, 1, ex_on ? syE : -1, k), pEx2 = psi_at(2, 0, 0, ex_on ? szE : -1, k);
    const Psi<R> pEy1 = psi_at(2, 0, 1, ey_on ? szE : -1, k), pEy2 = psi_at(0, 0, 0, ey_on ? sxE : -1, k);
    const Psi<R> pEz1 = psi_at(0, 0, 1, ez_on ? sxE : -1, k), pEz2 = psi_at(1, 0, 0, ez_on ? syE : -1, k);
    // the one barrier of the plane: H of this plane and the y-edge Joule
    // shares of the previous one are visible; every thread is past its reads
    // of plane k-1's stage
    __syncthreads();
    if (*s_abort) {  // a copy did not arrive in time: drain what is in flight (bounded), flag, leave
      if constexpr (sizeof(R) == 4) cp_async_wait<0>();
      if (leader) em_abort(bars, k, nz, A.err, A.wait);
      return false;
    }
    // Joule energy of node (i, j, k-1): its y-edge share from j-1 is now visible
    if (accum && own && (PL || k > 0)) {
      const R s = add_(q_pend, sQy[par ^ 1][ty - 1][tx]);
      if (plane_folds(fold, k - 1)) {
        A.Q[id - plane] += (double)s;
        A.Qs[id - plane] = R(0);
      } else {
        A.Qs[id - plane] = s;
      }
    }
    if (TH && own && (PL || k > 0)) th_finish(id - plane, sQy[par ^ 1][ty - 1][tx], t_part, t_dtc);
    if (CPL && !TH && own && (PL || k > 0)) A.Pout[id - plane] = mul_(add_(e_pend, sQy[par ^ 1][ty - 1][tx]), A.inv_dt);

    // ---- source current on this node's edges (three scalars selected by
    // axis: a dynamically indexed array would live in local memory)
    R Jx = 0, Jy = 0, Jz = 0;
    for (int e = r0; e < r1; ++e) {
      const int4 s = A.src_ent[e];
      const long long step = *A.step_base + step_off;
      if (s.x == i && step < A.amp_len) {
        const R a = A.src_amp[(long long)s.z * A.amp_len + step];
        Jx = add_(Jx, s.y == 0 ? a : R(0));
        Jy = add_(Jy, s.y == 1 ? a : R(0));
        Jz = add_(Jz, s.y == 2 ? a : R(0));
      }
    }

    // ---- E^{n+1} on the node's edges and their Joule shares. Layer-k partial
    // sums of the x / y edges (voxel pairs across y / x); the layer k-1 halves
    // were formed one plane earlier.
    const R pxe_a = fma_(hym, e01, mul_(hy0, e11)), pxs_a = fma_(hym, s01, mul_(hy0, s11));
    const R pye_a = fma_(hxm, e10, mul_(hx0, e11)), pys_a = fma_(hxm, s10, mul_(hx0, s11));
    R exn = ex, eyn = ey, ezn = ez, qx = 0, qy = 0, qz = 0;
    if (ex_on) {  // Ex: dHz/dy - dHy/dz, voxels (i, j-1..j, k-1..k)
      const R curl = curl_psi(A, s_cp, 0, 1, pEx1, 2, pEx2, dif_(Hz, sHxz[par][1][ty - 1][tx], idy), dif_(Hy, hy_km1, idz),
                              own);
      R Ss = fma_(hzm, pxs_b, mul_(hz0, pxs_a));
      if (CPL) {
        const R te = mul_(R(0.5), add_(th, th_ip));
        R d1, d2, d3, d4;
        const R a1 = mul_(mul_(hzm, hym), sgd(b01, te, d1)), a2 = mul_(mul_(hzm, hy0), sgd(b11, te, d2));
        const R a3 = mul_(mul_(hz0, hym), sgd(a01, te, d3)), a4 = mul_(mul_(hz0, hy0), sgd(a11, te, d4));
        Ss = sig_sum4(a1, d1, a2, d2, a3, d3, a4, d4);
      }
      exn = e_update<R, R>(ex, mul_(dtWx_y, add_(hzm, hz0)), sub_(curl, Jx), fma_(hzm, pxe_b, mul_(hz0, pxe_a)), Ss,
                           lqx, &qx);
    }
    if (ey_on) {  // Ey: dHx/dz - dHz/dx, voxels (i-1..i, j, k-1..k)
      const R curl = curl_psi(A, s_cp, 0, 2, pEy1, 0, pEy2, dif_(Hx, hx_km1, idz), dif_(Hz, hz_l, idx), own);
      R Ss = fma_(hzm, pys_b, mul_(hz0, pys_a));
      if (CPL) {
        const R te = mul_(R(0.5), add_(th, th_jp));
        R d1, d2, d3, d4;
        const R a1 = mul_(mul_(hzm, hxm), sgd(b10, te, d1)), a2 = mul_(mul_(hzm, hx0), sgd(b11, te, d2));
        const R a3 = mul_(mul_(hz0, hxm), sgd(a10, te, d3)), a4 = mul_(mul_(hz0, hx0), sgd(a11, te, d4));
        Ss = sig_sum4(a1, d1, a2, d2, a3, d3, a4, d4);
      }
      eyn = e_update<R, R>(ey, mul_(dtWy_x, add_(hzm, hz0)), sub_(curl, Jy), fma_(hzm, pye_b, mul_(hz0, pye_a)), Ss,
                           lqy, &qy);
    }
    if (ez_on) {  // Ez: dHy/dx - dHx/dy, voxels (i-1..i, j-1..j, k)
      const R curl = curl_psi(A, s_cp, 0, 0, pEz1, 1, pEz2, dif_(Hy, hy_l, idx), dif_(Hx, sHxz[par][0][ty - 1][tx], idy),
                              own);
      const R Se = fma_(hym, fma_(hxm, e00, mul_(hx0, e01)), mul_(hy0, fma_(hxm, e10, mul_(hx0, e11))));
      R Ss = fma_(hym, fma_(hxm, s00, mul_(hx0, s01)), mul_(hy0, fma_(hxm, s10, mul_(hx0, s11))));
      if (CPL) {
        const R te = mul_(R(0.5), add_(th, th_kp));
        R d1, d2, d3, d4;
        const R a1 = mul_(mul_(hym, hxm), sgd(a00, te, d1)), a2 = mul_(mul_(hym, hx0), sgd(a01, te, d2));
        const R a3 = mul_(mul_(hy0, hxm), sgd(a10, te, d3)), a4 = mul_(mul_(hy0, hx0), sgd(a11, te, d4));
        Ss = sig_sum4(a1, d1, a2, d2, a3, d3, a4, d4);
      }
      ezn = e_update<R, R>(ez, mul_(dtWx_y, add_(hxm, hx0)), sub_(curl, Jz), Se, Ss, mul_(R(0.25), hz0), &qz);
    }
    const R qx_l = __shfl_up_sync(0xffffffffu, qx, 1);  // x-edge share from node i-1
    sQy[par][ty][tx] = qy;

    if (own) {
      A.Hn[0][id] = Hx;
      A.Hn[1][id] = Hy;
      A.Hn[2][id] = Hz;
      A.En[0][id] = exn;
      A.En[1][id] = eyn;
      if (kz) A.En[2][id] = ezn;
    }
    e_pend = add_(add_(add_(qx, qx_l), qy), add_(qz, qz_km1));
    q_pend = add_(q_old, e_pend);
    hx_km1 = Hx;
    hy_km1 = Hy;
    qz_km1 = qz;
    pxe_b = pxe_a;
    pxs_b = pxs_a;
    pye_b = pye_a;
    pys_b = pys_a;
    u11_b = u11;
    if (CPL) {
      b00 = a00;
      b01 = a01;
      b10 = a10;
      b11 = a11;
    }
    return true;
  };
  for (int k = 0; k <= nz; ++k) {
    const bool plain = k > 0 && k < nz && slab_index(k, nz, A.slo[2], A.shi[2]) < 0;
    if (!(plain ? plane_body(k, BoolTag<true>{}) : plane_body(k, BoolTag<false>{}))) return;
  }
  __syncthreads();
  if (accum && own) {  // Joule energy of the top plane k = nz
    const I id = id0 + (I)nz * plane;
    const R s = add_(q_pend, sQy[nz & 1][ty - 1][tx]);
    if (plane_folds(fold, nz)) {
      A.Q[id] += (double)s;
      A.Qs[id] = R(0);
    } else {
      A.Qs[id] = s;
    }
  }
  if (CPL && !TH && own) A.Pout[id0 + (I)nz * plane] = mul_(add_(e_pend, sQy[nz & 1][ty - 1][tx]), A.inv_dt);
  if (TH) {  // node (i, j, nz): no voxel layer above; plane nz's stage is resident (nothing is issued after it)
    R t_part = 0, t_dtc = 0;
    th_partial(stg[nz & (kEmStages - 1)], nz, th_layer_zero<R, R>(), R(0), t_part, t_dtc);
    if (own) th_finish(id0 + (I)nz * plane, sQy[nz & 1][ty - 1][tx], t_part, t_dtc);
    if (A.peak != nullptr) peak_max(t_max, A.peak);
  }
}

// ---- interior tile pairs: two nodes per thread. The pair tile starting at
// node xs (even) of row tile by owns the nodes i = xs .. xs + 61; thread
// (tx, ty) holds the nodes i0 + 2 tx (.x) and i0 + 2 tx + 1 (.y), i0 = xs - 2
// (lane 0 is the halo pair), of row j0 + ty. Every node, its
// +x/+y neighbours and its voxels lie inside the grid, off the lateral walls
// and outside the x/y CPML slabs; only the z slab and walls remain, decided
// per plane for the whole CTA.
template <typename R, typename I, int TY, bool CPL, bool TH, bool ES>
__device__ __forceinline__ void em_tile_pair(const EmArgs<R> &A, const R *s_cp, const R *s_mt,
                                             EmStage<R, kEm2Nodes, TY> *stg, typename Pair2<R>::T (*sHxz)[2][TY][32],
                                             typename Pair2<R>::T (*sQy)[TY][32], uint64_t *bars, int *s_abort, int xs,
                                             int by, int step_off, int fold) {
  using R2 = typename Pair2<R>::T;
  constexpr int BX = em2_box_x(), BV = em2_vox_box_x();
  const Geo<R> &g = A.g;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ny = g.ny, nz = g.nz;
  const int vd = g.nmat * M_COLS;
  const int i0 = xs - 2, j0 = by * (TY - 1) - 1;
  const int ia = i0 + 2 * tx, j = j0 + ty;
  const bool own = tx > 0 && ty > 0;
  const bool accum = A.Qs != nullptr;
  const bool leader = tx == 0 && ty == 0;
  // node boxes from i0 rounded down to 4 (i0 is even: a pair starts at an
  // even column, 8 / 16-byte aligned), the voxel box from i0 - 1 rounded down
  // to 16, the source-row box as for border tiles
  const int xr = i0 & 3, x0 = i0 - xr;
  const int xvr = (i0 - 1) & 15, xv0 = (i0 - 1) - xvr;
  const bool has_src = A.src_row != nullptr;
  const unsigned stage_bytes =
      (unsigned)((6 * TY + 3 + (accum ? TY : 0) + (CPL ? TY + 1 : 0)) * BX * (int)sizeof(R) + 4 * (int)sizeof(R) +
                 (has_src ? em_src_box<TY>() * 4 : 0) + (TY + 1) * BV);
  auto issue = [&](int k) {
    if (k > nz) return;
    const int s = k & (kEmStages - 1);
    EmStage<R, kEm2Nodes, TY> &S = stg[s];
    mbar_arrive_expect_tx(&bars[s], stage_bytes);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      tma_load_3d(&S.E[c].v[0][0], &A.tmE2[c], x0, j0, k, &bars[s]);
      tma_load_3d(&S.H[c].v[0][0], &A.tmH2[c], x0, j0, k, &bars[s]);
    }
    if (accum) tma_load_3d(&S.Qs.v[0][0], &A.tmQ2, x0, j0, k, &bars[s]);
    if (CPL) tma_load_3d(&S.T.v[0][0], &A.tmT2, x0, j0, k, &bars[s]);
    tma_load_3d(&S.V.v[0][0], &A.tmV2, xv0, j0 - 1, k, &bars[s]);
    bulk_load(&S.Z.v[0][0], A.zt + 4 * (size_t)k, 4 * sizeof(R), &bars[s]);
    if (has_src) {
      const int base = k * (ny + 1) + j0;
      bulk_load(&S.S.v[0][0], A.src_row + (base - (base & 3)), em_src_box<TY>() * 4, &bars[s]);
    }
  };
  const I plane = (I)g.plane;
  const I id0 = (I)g.nid(ia, j, 0);
  const int cv = 2 * tx + xvr;  // column of voxel ia - 1 in the voxel box
  const int cx = 2 * tx + xr;   // column of node ia in the node boxes
  const R2 z2 = bc_<R2>(R(0));

  // geometry: x per node, y per row (the same arithmetic as the border path)
  const R2 hxm = {g.h[0][ia - 1], g.h[0][ia]}, hx0 = {g.h[0][ia], g.h[0][ia + 1]};
  const R2 ihx = {g.ih[0][ia], g.ih[0][ia + 1]}, idx = {g.idual[0][ia], g.idual[0][ia + 1]};
  const R hym_s = g.h[1][j - 1], hy0_s = g.h[1][j];
  const R2 hym = bc_<R2>(hym_s), hy0 = bc_<R2>(hy0_s), ihy = bc_<R2>(g.ih[1][j]), idy = bc_<R2>(g.idual[1][j]);
  const R dt = A.dt;
  const R half_dt = mul_(R(0.5), dt);
  const R2 hdx = mul_(bc_<R2>(half_dt), idx), hdy = bc_<R2>(mul_(half_dt, g.idual[1][j]));
  const R2 dtWx_y = bc_<R2>(mul_(dt, add_(hym_s, hy0_s))), dtWy_x = mul_(bc_<R2>(dt), add_(hxm, hx0));
  const R2 lqx = mul_(bc_<R2>(R(0.25)), hx0), lqy = bc_<R2>(mul_(R(0.25), hy0_s));

  if (leader) {
#pragma unroll
    for (int q = 0; q < kEmAhead; ++q) issue(q);
  }
  if (!mbar_wait(&bars[0], 0u, A.wait)) *s_abort = 1;
  R2 hx_km1 = z2, hy_km1 = z2, qz_km1 = z2;
  R2 pxe_b = z2, pxs_b = z2, pye_b = z2, pys_b = z2, u11_b = z2;
  R2 q_pend = z2, e_pend = z2;
  int p0a = vd, p0b = vd, p0c = vd, p1a = vd, p1b = vd, p1c = vd;  // coupled steps: material rows of layer k-1
  // sigma dt/2 of the voxels ra (node .x) and rb (node .y) (returned) and their
  // denominators at the edge temperatures te (in d), for sig_sum4
  auto sgdp = [&](int ra, int rb, R2 te, R2 &d) -> R2 {
    d = fma_(R2{s_mt[ra + M_TCR], s_mt[rb + M_TCR]}, te, R2{s_mt[ra + M_TC0], s_mt[rb + M_TC0]});
    return R2{s_mt[ra + M_SDT2], s_mt[rb + M_SDT2]};
  };
  // coupled steps, the fused thermal step of the node pair at plane k-1 (see
  // the border tiles)
  // the node columns' constants from the tile's geometry (interior pairs lie
  // off the lateral walls: no lateral film); the inverse sizes of cells ia-1
  // and j-1 are kept
  static_assert(CPL || !TH, "the fused thermal step belongs to coupled steps");
  R2 ihxm_th = z2;
  R ihym_th = 0;
  if (TH) {
    ihxm_th = R2{g.ih[0][ia - 1], g.ih[0][ia]};
    ihym_th = g.ih[1][j - 1];
  }
  auto tcol_of = [&]() -> ThCol<R2> {
    ThCol<R2> c;
    c.hxm = hxm, c.hx0 = hx0, c.hym = hym, c.hy0 = hy0;
    c.qxm = mul_(bc_<R2>(R(0.25)), ihxm_th), c.qx0 = mul_(bc_<R2>(R(0.25)), ihx);
    c.qym = bc_<R2>(mul_(R(0.25), ihym_th)), c.qy0 = mul_(bc_<R2>(R(0.25)), ihy);
    c.fxy = z2;
    c.az = mul_(bc_<R2>(R(0.25)), mul_(add_(hxm, hx0), add_(hym, hy0)));
    return c;
  };
  ThLayer<R2> tl_lo = th_layer_zero<R2, R>();  // sums of voxel layer k-2
  R2 th_m2 = z2, gz_th = z2;                   // T of the pair at plane k-2; the z-edge conductance below
  R t_max = R(-3.0e38);
  // the pair's thermal step at plane kk without the y-edge share of row j-1
  // (see the border tiles)
  auto th_partial = [&](const EmStage<R, kEm2Nodes, TY> &Sm, int kk, const ThLayer<R2> &up, R2 tkp, R2 &tpart,
                        R2 &dtc) {
    const ThCoeffs<R2> q = th_coeffs<R2, R>(tcol_of(), tl_lo, up, Sm.Z.v[0][0], Sm.Z.v[0][1], Sm.Z.v[0][3], kk == 0,
                                            kk == nz, A.hconv, gz_th);
    const R2 tc = ldv_<R2>(&Sm.T.v[ty][cx]);
    if (own) {
      dtc = mul_(bc_<R2>(A.dt), rcp_(q.C));
      const R2 p = mul_(e_pend, bc_<R2>(A.inv_dt));
      R2 f = fma_(q.Gxm, sub_(R2{Sm.T.v[ty][cx - 1], tc.x}, tc), p);  // owners: tx, ty >= 1
      f = fma_(q.Gxp, sub_(R2{tc.y, Sm.T.v[ty][cx + 2]}, tc), f);
      f = fma_(q.Gym, sub_(ldv_<R2>(&Sm.T.v[ty - 1][cx]), tc), f);
      f = fma_(q.Gyp, sub_(ldv_<R2>(&Sm.T.v[ty + 1][cx]), tc), f);
      f = fma_(q.Gzm, sub_(th_m2, tc), f);
      f = fma_(q.Gzp, sub_(tkp, tc), f);
      f = fma_(q.film, sub_(bc_<R2>(A.T_amb), tc), f);
      tpart = fma_(dtc, f, tc);
    }
    th_m2 = tc;
    tl_lo = up;
  };
  auto th_finish = [&](I idn, R2 share, R2 tpart, R2 dtc) {
    const R2 inv = bc_<R2>(A.inv_dt);
    stv_(A.Pout + idn, mul_(add_(e_pend, share), inv));
    const R2 tn = fma_(dtc, mul_(share, inv), tpart);
    stv_(A.Tth + idn, tn);
    t_max = fmax(t_max, fmax(tn.x, tn.y));
  };

  // The plane body, compiled twice: PL (planes 0 < k < nz outside the z
  // slabs, most of them) knows that the plane has a voxel layer above, no
  // wall and no CPML state, so its wall, slab and end-plane branches fold
  // away; the other planes take the general copy. Returns false when the CTA
  // must leave (a copy did not arrive in time).
  auto plane_body = [&](const int k, auto plain_tag) -> bool {
    constexpr bool PL = decltype(plain_tag)::value;
    if (leader) {
      fence_proxy_async_smem();
      issue(k + kEmAhead);
    }
    em_wait_next(bars, k, nz, s_abort, A.wait);
    const int par = k & 1;  // parity of the double-buffered exchange arrays
    const I id = id0 + (I)k * plane;
    const EmStage<R, kEm2Nodes, TY> &S0 = stg[k & (kEmStages - 1)];
    const EmStage<R, kEm2Nodes, TY> &S1 = stg[(k + 1) & (kEmStages - 1)];
    R hz0s, ihzs, idzs, hzms;
    load4(&S0.Z.v[0][0], hz0s, ihzs, idzs, hzms);
    const R2 hz0 = bc_<R2>(hz0s), ihz = bc_<R2>(ihzs), idz = bc_<R2>(idzs), hzm = bc_<R2>(hzms);
    const bool kz = PL || k < nz;
    // voxels ia-1 (a), ia (b), ia+1 (c) of rows j-1 (0) and j (1) in layer k;
    // at k = nz the zero-filled box gives material 0, which the zero layer
    // height then removes
    const int r0a = (int)S0.V.v[ty][cv] * M_COLS, r0b = (int)S0.V.v[ty][cv + 1] * M_COLS,
              r0c = (int)S0.V.v[ty][cv + 2] * M_COLS;
    const int r1a = (int)S0.V.v[ty + 1][cv] * M_COLS, r1b = (int)S0.V.v[ty + 1][cv + 1] * M_COLS,
              r1c = (int)S0.V.v[ty + 1][cv + 2] * M_COLS;
    int r0 = 0, r1 = 0;  // source entries of row (k, j)
    if (has_src) {
      const int base = k * (ny + 1) + j0, sr = (base & 3) + ty;
      r0 = S0.S.v[0][sr];
      r1 = S0.S.v[0][sr + 1];
    }
    // ---- source currents on the pair's edges. ES (plain single-context
    // steps) forms them here, before the H update, so that the E update after
    // the barrier is one block; the coupled and batch kernels (more live
    // state: measured slower) keep them after the barrier.
    R2 Jx = z2, Jy = z2, Jz = z2;
    auto add_sources = [&]() {
      for (int e = r0; e < r1; ++e) {
        const int4 s = A.src_ent[e];
        const long long step = *A.step_base + step_off;
        if ((s.x == ia || s.x == ia + 1) && step < A.amp_len) {
          const R a = A.src_amp[(long long)s.z * A.amp_len + step];
          if (s.x == ia) {
            Jx.x = add_(Jx.x, s.y == 0 ? a : R(0));
            Jy.x = add_(Jy.x, s.y == 1 ? a : R(0));
            Jz.x = add_(Jz.x, s.y == 2 ? a : R(0));
          } else {
            Jx.y = add_(Jx.y, s.y == 0 ? a : R(0));
            Jy.y = add_(Jy.y, s.y == 1 ? a : R(0));
            Jz.y = add_(Jz.y, s.y == 2 ? a : R(0));
          }
        }
      }
    };
    if constexpr (ES) add_sources();

    const R2 hdz = bc_<R2>(mul_(half_dt, idzs));
    const bool fix_z = !PL && ((k == 0 && A.fixlo[2]) || (k == nz && A.fixhi[2]));
    const int szE = PL ? -1 : slab_index(k, nz, A.slo[2], A.shi[2]);
    const int szH = kz ? szE : -1;

    const R2 ex = ldv_<R2>(&S0.E[0].v[ty][cx]), ey = ldv_<R2>(&S0.E[1].v[ty][cx]), ez = ldv_<R2>(&S0.E[2].v[ty][cx]);
    const R2 ex_up = ldv_<R2>(&S1.E[0].v[ty][cx]), ey_up = ldv_<R2>(&S1.E[1].v[ty][cx]);
    const R2 ez_jp = ldv_<R2>(&S0.E[2].v[ty + 1][cx]), ex_jp = ldv_<R2>(&S0.E[0].v[ty + 1][cx]);
    const R2 ez_ip = {ez.y, S0.E[2].v[ty][cx + 2]}, ey_ip = {ey.y, S0.E[1].v[ty][cx + 2]};
    const R2 hx_o = ldv_<R2>(&S0.H[0].v[ty][cx]), hy_o = ldv_<R2>(&S0.H[1].v[ty][cx]),
             hz_o = ldv_<R2>(&S0.H[2].v[ty][cx]);
    const R2 q_old = accum ? ldv_<R2>(&S0.Qs.v[ty][cx]) : z2;
    R2 th = z2, th_ip = z2, th_jp = z2, th_kp = z2;
    R2 t_part = z2, t_dtc = z2;  // the pair's thermal step at plane k-1 without the y-edge share of row j-1
    if (CPL) {
      th = ldv_<R2>(&S0.T.v[ty][cx]);
      th_ip = R2{th.y, S0.T.v[ty][cx + 2]};
      th_jp = ldv_<R2>(&S0.T.v[ty + 1][cx]);
      th_kp = kz ? ldv_<R2>(&S1.T.v[ty][cx]) : z2;
      if (TH && (PL || k > 0)) {  // plane k-1's stage is resident until this plane's barrier
        const ThLayer<R2> up = th_layer<R2>(
            R2{s_mt[p0a + M_K], s_mt[p0b + M_K]}, R2{s_mt[p0b + M_K], s_mt[p0c + M_K]},
            R2{s_mt[p1a + M_K], s_mt[p1b + M_K]}, R2{s_mt[p1b + M_K], s_mt[p1c + M_K]},
            R2{s_mt[p0a + M_RHOCP], s_mt[p0b + M_RHOCP]}, R2{s_mt[p0b + M_RHOCP], s_mt[p0c + M_RHOCP]},
            R2{s_mt[p1a + M_RHOCP], s_mt[p1b + M_RHOCP]}, R2{s_mt[p1b + M_RHOCP], s_mt[p1c + M_RHOCP]}, tcol_of());
        th_partial(stg[(k - 1) & (kEmStages - 1)], k - 1, up, th, t_part, t_dtc);
      }
    }

    R e0a, s0a, u0a, k0a, e0b, s0b, u0b, k0b, e0c, s0c, u0c, k0c;
    R e1a, s1a, u1a, k1a, e1b, s1b, u1b, k1b, e1c, s1c, u1c, k1c;
    load4(s_mt + r0a, e0a, s0a, u0a, k0a);
    load4(s_mt + r0b, e0b, s0b, u0b, k0b);
    load4(s_mt + r0c, e0c, s0c, u0c, k0c);
    load4(s_mt + r1a, e1a, s1a, u1a, k1a);
    load4(s_mt + r1b, e1b, s1b, u1b, k1b);
    load4(s_mt + r1c, e1c, s1c, u1c, k1c);
    // the voxels (i-1+dx, j-1+dy) of each node as pairs <dy><dx>
    const R2 e00 = {e0a, e0b}, e01 = {e0b, e0c}, e10 = {e1a, e1b}, e11 = {e1b, e1c};
    const R2 s00 = {s0a, s0b}, s01 = {s0b, s0c}, s10 = {s1a, s1b}, s11 = {s1b, s1c};
    const R2 u01 = {u0b, u0c}, u10 = {u1a, u1b}, u11 = {u1b, u1c};

    // CPML states of the z slab for the node pair (derivative axis z)
    auto psi_z = [&](int type, int slot, int s) -> Psi<R2> {
      return psi_pre<R, R2>(A, 2, type, slot, s, s >= 0 ? ((long long)s * (ny + 1) + j) * g.px + ia : 0);
    };
    // chi of the z derivative (b - a) ih for each node of the pair, in the
    // scalar forms: the compensated update relies on every step being
    // rounded separately, which packed code does not guarantee (a packed
    // product feeding an addition is contracted into an FMA)
    auto chi_z = [&](int type, int slot, const Psi<R2> &p, R2 b, R2 a, R ih) -> R2 {
      const R omb = s_cp[(2 * 2 + type) * kMaxSlab + p.s];
      Psi<R> px, py;
      px.s = py.s = p.s;
      px.q = p.q;
      py.q = p.q + 1;
      px.c.hi = p.c.hi.x, py.c.hi = p.c.hi.y;
      px.c.d = p.c.d.x, py.c.d = p.c.d.y;
      if constexpr (sizeof(R) == 4) px.c.lo = p.c.lo.x, py.c.lo = p.c.lo.y;
      return R2{psi_apply<R, R>(A, omb, 2, type, slot, px, dif_(b.x, a.x, ih), own),
                psi_apply<R, R>(A, omb, 2, type, slot, py, dif_(b.y, a.y, ih), own)};
    };

    // ---- H^{n+1/2}
    R2 Hx = z2, Hy = z2;
    if (kz) {
      const Psi<R2> pHx = psi_z(1, 0, szH), pHy = psi_z(1, 1, szH);
      const R2 d1 = dif_(ez_jp, ez, ihy), d2 = dif_(ey_up, ey, ihz);
      Hx = h_update(hx_o, hdx, hxm, u10, hx0, u11, szH >= 0 ? sub_(d1, chi_z(1, 0, pHx, ey_up, ey, ihzs)) : sub_(d1, d2));
      const R2 f1 = dif_(ex_up, ex, ihz), f2 = dif_(ez_ip, ez, ihx);
      Hy = h_update(hy_o, hdy, hym, u01, hy0, u11,
                    szH >= 0 ? sub_(chi_z(1, 1, pHy, ex_up, ex, ihzs), f2) : sub_(f1, f2));
    }
    const R2 Hz = h_update(hz_o, hdz, hzm, u11_b, hz0, u11, sub_(dif_(ey_ip, ey, ihx), dif_(ex_jp, ex, ihy)));
    sHxz[par][0][ty][tx] = Hx;
    sHxz[par][1][ty][tx] = Hz;
    const R2 hy_l = {__shfl_up_sync(0xffffffffu, Hy.y, 1), Hy.x};  // H of nodes ia-1, ia
    const R2 hz_l = {__shfl_up_sync(0xffffffffu, Hz.y, 1), Hz.x};
    // the one barrier of the plane (see the border tiles)
    __syncthreads();
    if (*s_abort) {
      if (leader) em_abort(bars, k, nz, A.err, A.wait);
      return false;
    }
    if (accum && own && (PL || k > 0)) {
      const R2 s = add_(q_pend, sQy[par ^ 1][ty - 1][tx]);
      if (plane_folds(fold, k - 1)) {
        double2 *qp = reinterpret_cast<double2 *>(A.Q + (id - plane));
        double2 qv = *qp;
        qv.x += (double)s.x;
        qv.y += (double)s.y;
        *qp = qv;
        stv_(A.Qs + (id - plane), z2);
      } else {
        stv_(A.Qs + (id - plane), s);
      }
    }
    if (TH && own && (PL || k > 0)) th_finish(id - plane, sQy[par ^ 1][ty - 1][tx], t_part, t_dtc);
    if (CPL && !TH && own && (PL || k > 0))
      stv_(A.Pout + (id - plane), mul_(add_(e_pend, sQy[par ^ 1][ty - 1][tx]), bc_<R2>(A.inv_dt)));

    if constexpr (!ES) add_sources();

    // ---- E^{n+1} and the Joule shares
    const R2 pxe_a = fma_(hym, e01, mul_(hy0, e11)), pxs_a = fma_(hym, s01, mul_(hy0, s11));
    const R2 pye_a = fma_(hxm, e10, mul_(hx0, e11)), pys_a = fma_(hxm, s10, mul_(hx0, s11));
    R2 exn = ex, eyn = ey, ezn = ez, qx = z2, qy = z2, qz = z2;
    if (ty > 0 && !fix_z) {  // Ex (owners and the halo lane, whose x-edge share lane 1 needs)
      const R2 d1 = dif_(Hz, sHxz[par][1][ty - 1][tx], idy), d2 = dif_(Hy, hy_km1, idz);
      const R2 curl = szE >= 0 ? sub_(d1, chi_z(0, 0, psi_z(0, 0, szE), Hy, hy_km1, idzs)) : sub_(d1, d2);
      R2 Ss = fma_(hzm, pxs_b, mul_(hz0, pxs_a));
      if (CPL) {
        const R2 te = mul_(bc_<R2>(R(0.5)), add_(th, th_ip));
        R2 d1, d2, d3, d4;
        const R2 a1 = mul_(mul_(hzm, hym), sgdp(p0b, p0c, te, d1)), a2 = mul_(mul_(hzm, hy0), sgdp(p1b, p1c, te, d2));
        const R2 a3 = mul_(mul_(hz0, hym), sgdp(r0b, r0c, te, d3)), a4 = mul_(mul_(hz0, hy0), sgdp(r1b, r1c, te, d4));
        Ss = sig_sum4(a1, d1, a2, d2, a3, d3, a4, d4);
      }
      exn = e_update<R2, R>(ex, mul_(dtWx_y, add_(hzm, hz0)), sub_(curl, Jx), fma_(hzm, pxe_b, mul_(hz0, pxe_a)), Ss,
                            lqx, &qx);
    }
    if (!fix_z) {  // Ey (every row: the halo row's y-edge share goes to row ty+1)
      const R2 d1 = dif_(Hx, hx_km1, idz), d2 = dif_(Hz, hz_l, idx);
      const R2 curl = szE >= 0 ? sub_(chi_z(0, 1, psi_z(0, 1, szE), Hx, hx_km1, idzs), d2) : sub_(d1, d2);
      R2 Ss = fma_(hzm, pys_b, mul_(hz0, pys_a));
      if (CPL) {
        const R2 te = mul_(bc_<R2>(R(0.5)), add_(th, th_jp));
        R2 d1, d2, d3, d4;
        const R2 a1 = mul_(mul_(hzm, hxm), sgdp(p1a, p1b, te, d1)), a2 = mul_(mul_(hzm, hx0), sgdp(p1b, p1c, te, d2));
        const R2 a3 = mul_(mul_(hz0, hxm), sgdp(r1a, r1b, te, d3)), a4 = mul_(mul_(hz0, hx0), sgdp(r1b, r1c, te, d4));
        Ss = sig_sum4(a1, d1, a2, d2, a3, d3, a4, d4);
      }
      eyn = e_update<R2, R>(ey, mul_(dtWy_x, add_(hzm, hz0)), sub_(curl, Jy), fma_(hzm, pye_b, mul_(hz0, pye_a)), Ss,
                            lqy, &qy);
    }
    if (ty > 0 && kz) {  // Ez
      const R2 curl = sub_(dif_(Hy, hy_l, idx), dif_(Hx, sHxz[par][0][ty - 1][tx], idy));
      const R2 Se = fma_(hym, fma_(hxm, e00, mul_(hx0, e01)), mul_(hy0, fma_(hxm, e10, mul_(hx0, e11))));
      R2 Ss = fma_(hym, fma_(hxm, s00, mul_(hx0, s01)), mul_(hy0, fma_(hxm, s10, mul_(hx0, s11))));
      if (CPL) {
        const R2 te = mul_(bc_<R2>(R(0.5)), add_(th, th_kp));
        R2 d1, d2, d3, d4;
        const R2 a1 = mul_(mul_(hym, hxm), sgdp(r0a, r0b, te, d1)), a2 = mul_(mul_(hym, hx0), sgdp(r0b, r0c, te, d2));
        const R2 a3 = mul_(mul_(hy0, hxm), sgdp(r1a, r1b, te, d3)), a4 = mul_(mul_(hy0, hx0), sgdp(r1b, r1c, te, d4));
        Ss = sig_sum4(a1, d1, a2, d2, a3, d3, a4, d4);
      }
      ezn = e_update<R2, R>(ez, mul_(dtWx_y, add_(hxm, hx0)), sub_(curl, Jz), Se, Ss, bc_<R2>(mul_(R(0.25), hz0s)),
                            &qz);
    }
    const R2 qx_l = {__shfl_up_sync(0xffffffffu, qx.y, 1), qx.x};  // x-edge shares from nodes ia-1, ia
    sQy[par][ty][tx] = qy;

    if (own) {
      stv_(A.Hn[0] + id, Hx);
      stv_(A.Hn[1] + id, Hy);
      stv_(A.Hn[2] + id, Hz);
      stv_(A.En[0] + id, exn);
      stv_(A.En[1] + id, eyn);
      if (kz) stv_(A.En[2] + id, ezn);
    }
    e_pend = add_(add_(add_(qx, qx_l), qy), add_(qz, qz_km1));
    q_pend = add_(q_old, e_pend);
    hx_km1 = Hx;
    hy_km1 = Hy;
    qz_km1 = qz;
    pxe_b = pxe_a;
    pxs_b = pxs_a;
    pye_b = pye_a;
    pys_b = pys_a;
    u11_b = u11;
    if (CPL) {
      p0a = r0a, p0b = r0b, p0c = r0c, p1a = r1a, p1b = r1b, p1c = r1c;
    }
    return true;
  };
  for (int k = 0; k <= nz; ++k) {
    const bool plain = k > 0 && k < nz && slab_index(k, nz, A.slo[2], A.shi[2]) < 0;
    if (!(plain ? plane_body(k, BoolTag<true>{}) : plane_body(k, BoolTag<false>{}))) return;
  }
  __syncthreads();
  if (accum && own) {  // Joule energy of the top plane k = nz
    const I id = id0 + (I)nz * plane;
    const R2 s = add_(q_pend, sQy[nz & 1][ty - 1][tx]);
    if (plane_folds(fold, nz)) {
      double2 *qp = reinterpret_cast<double2 *>(A.Q + id);
      double2 qv = *qp;
      qv.x += (double)s.x;
      qv.y += (double)s.y;
      *qp = qv;
      stv_(A.Qs + id, z2);
    } else {
      stv_(A.Qs + id, s);
    }
  }
  if (CPL && !TH && own)
    stv_(A.Pout + (id0 + (I)nz * plane), mul_(add_(e_pend, sQy[nz & 1][ty - 1][tx]), bc_<R2>(A.inv_dt)));
  if (TH) {  // the pair at plane nz: no voxel layer above; plane nz's stage is resident
    R2 t_part = z2, t_dtc = z2;
    th_partial(stg[nz & (kEmStages - 1)], nz, th_layer_zero<R2, R>(), z2, t_part, t_dtc);
    if (own) th_finish(id0 + (I)nz * plane, sQy[nz & 1][ty - 1][tx], t_part, t_dtc);
    if (A.peak != nullptr) peak_max(t_max, A.peak);
  }
}

// Resident CTAs per SM the kernel is compiled for: FP32 8-row tiles at
// COSIM_EM_MIN_CTAS (scaled for other heights), FP64 one.
__host__ __device__ constexpr int em_min_ctas(int rsz, int ty) { return rsz == 4 ? COSIM_EM_MIN_CTAS * 8 / ty : 1; }

// One CTA's share of a step: tile b of the context described by A (tiles
// 0 .. n_border-1 are the border tiles, the frame around the interior
// rectangle row by row; the rest the interior pairs). smem: the dynamic
// shared window, 128-byte aligned; sHxz, sQy, s_bar, s_abort: the CTA's
// static exchange arrays, stage barriers (initialised here) and abort flag.
// CPL: the coupled step (sigma(T), Joule power of the step); TH: with the
// thermal step of Eq. 5 in the same launch (else a thermal launch follows);
// ES: the pair tiles form the source currents before the H update.
template <typename R, typename I, int TX, int TY, bool CPL, bool TH, bool ES = !CPL>
__device__ __forceinline__ void em_cta(const EmArgs<R> &A, int b, int step_off, int fold, unsigned char *smem,
                                       typename Pair2<R>::T (*sHxz)[2][TY][TX], typename Pair2<R>::T (*sQy)[TY][TX],
                                       uint64_t *s_bar, int *s_abort) {
  static_assert(TX == 32, "a tile row is one warp: x neighbours are exchanged by shuffles");
  R *s_cp = reinterpret_cast<R *>(smem);
  R *s_mt = s_cp + kCpmlTable;
  unsigned char *stg = smem + em_stage_offset<R>(A.g.nmat);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    // (a CTA that took an earlier tile read these stages: order those reads
    // before the copies of this tile)
    fence_proxy_async_smem();
    // TMA preconditions checked once per tile: 128-byte aligned destinations
    // and 64-byte aligned descriptors; otherwise flag the error and leave
    // without issuing a copy
    bool ok = (smem_u32(stg) & 127u) == 0 && (sizeof(EmStage<R, TX, TY>) & 127u) == 0 &&
              (sizeof(EmStage<R, kEm2Nodes, TY>) & 127u) == 0;
    for (int c = 0; c < 3; ++c)
      ok = ok && ((size_t)&A.tmE[c] & 63u) == 0 && ((size_t)&A.tmH[c] & 63u) == 0 &&
           ((size_t)&A.tmE2[c] & 63u) == 0 && ((size_t)&A.tmH2[c] & 63u) == 0;
    ok = ok && ((size_t)&A.tmQ & 63u) == 0 && ((size_t)&A.tmQ2 & 63u) == 0 && ((size_t)&A.tmV & 63u) == 0 &&
         ((size_t)&A.tmV2 & 63u) == 0 && ((size_t)&A.tmT & 63u) == 0 && ((size_t)&A.tmT2 & 63u) == 0;
    *s_abort = ok ? 0 : 1;
    if (!ok) atomicExch(A.err, 2);
    for (int q = 0; q < kEmStages; ++q) mbar_init(&s_bar[q], 1);
    fence_mbar_init();
  }
  stage_table(s_mt, A.g.mtab, (A.g.nmat + 1) * M_COLS);
  stage_table(s_cp, A.cpml, kCpmlTable);
  __syncthreads();
  if (*s_abort) return;
  if (b < A.n_border) {
    // border tile b: the rows below the interior rows, then the left and
    // right parts of the interior rows, then the rows above them
    const int nbx = A.nbx, below = A.iby0 * nbx, w = A.nl + A.nr, mid = (A.iby1 - A.iby0) * w;
    int xs, xe = A.g.nx + 1, by;
    auto *sb = reinterpret_cast<EmStage<R, TX, TY> *>(stg);
    auto *sh = reinterpret_cast<R(*)[2][TY][TX]>(&sHxz[0][0][0][0]);
    auto *sq = reinterpret_cast<R(*)[TY][TX]>(&sQy[0][0][0]);
    if (b >= below && b - below < mid) {  // beside the interior pairs: no y slab row
      b -= below;
      by = b / w;
      const int c = b - by * w;
      by += A.iby0;
      if (c < A.nl) {
        xs = (TX - 1) * c;
        xe = A.xb0;
      } else {
        xs = A.xb1 + (TX - 1) * (c - A.nl);
      }
      em_tile_border<R, I, TY, CPL, TH, true, false>(A, s_cp, s_mt, sb, sh, sq, s_bar, s_abort, xs, xe, by, step_off,
                                                     fold);
    } else {
      if (b >= below) {
        b -= below + mid;
        by = b / nbx;
        xs = (TX - 1) * (b - by * nbx);
        by += A.iby1;
      } else {
        by = b / nbx;
        xs = (TX - 1) * (b - by * nbx);
      }
      // nodes i = xs - 1 .. xs + 30: does the tile reach an x slab?
      const bool xsl = (A.slo[0] > 0 && xs - 1 <= A.slo[0]) || (A.shi[0] > 0 && xs + TX - 2 >= A.g.nx - A.shi[0]);
      if (xsl)
        em_tile_border<R, I, TY, CPL, TH, true, true>(A, s_cp, s_mt, sb, sh, sq, s_bar, s_abort, xs, xe, by, step_off,
                                                      fold);
      else
        em_tile_border<R, I, TY, CPL, TH, false, true>(A, s_cp, s_mt, sb, sh, sq, s_bar, s_abort, xs, xe, by,
                                                       step_off, fold);
    }
  } else {
    b -= A.n_border;
    const int py = b / A.npx, px = b - py * A.npx;
    em_tile_pair<R, I, TY, CPL, TH, ES>(A, s_cp, s_mt, reinterpret_cast<EmStage<R, kEm2Nodes, TY> *>(stg), sHxz, sQy, s_bar,
                                    s_abort, A.xb0 + 62 * px, A.iby0 + py, step_off, fold);
  }
}

// One launch per step of one context: CTA b takes tile b.
template <typename R, typename I, int TX, int TY, bool CPL, bool TH>
__global__ void __launch_bounds__(TX *TY, em_min_ctas(sizeof(R), TY))
    em_step_kernel(const __grid_constant__ EmArgs<R> A) {
  using R2 = typename Pair2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the launch adds 128 bytes so that the tables and stages can start on a
  // 128-byte boundary of the shared window (TMA destinations must)
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  // double-buffered by plane parity, so that a plane needs one barrier
  __shared__ R2 sHxz[2][2][TY][TX];  // Hx, Hz of the plane, read by the +y neighbour
  __shared__ R2 sQy[2][TY][TX];      // Joule share of the y-edge, read by the +y neighbour one plane later
  __shared__ uint64_t s_bar[kEmStages];  // one transaction barrier per stage
  __shared__ int s_abort;
  em_cta<R, I, TX, TY, CPL, TH>(A, (int)blockIdx.x, A.step_off, A.fold, smem, sHxz, sQy, s_bar, &s_abort);
}

// A group of up to kBatchMax contexts (independent package designs) for one
// launch of a batch step: their arguments for the step's E/H parity and
// Joule accumulation, by value in the kernel's parameter space (8 designs fill most
// of the 32 KB a launch may pass), and cta_start[d], the first tile of design
// d in the group's tile order (cta_start[n] = all tiles).
constexpr int kBatchMax = 8;
template <typename R>
struct EmBatchArgs {
  EmArgs<R> a[kBatchMax];
  int cta_start[kBatchMax + 1];
  int n;
};

// One launch per step of a group of designs. work == null: CTA b takes tile
// b. Otherwise the launch is persistent: a grid of about the resident CTAs
// takes tiles in order from the counter *work (tiles of the larger designs
// first, so that the small ones fill the tail), and zeroes *next_work, the
// counter of the group's next launch (launches alternate between two
// counters, so that no launch resets a counter in use). The stage barriers
// are invalidated after each tile and initialised again for the next. fold:
// the step's Joule window position (-1: no fold), as EmArgs::fold.
template <typename R, typename I, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, em_min_ctas(sizeof(R), TY))
    em_batch_kernel(const __grid_constant__ EmBatchArgs<R> P, int step_off, int fold, unsigned *work,
                    unsigned *next_work) {
  using R2 = typename Pair2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  __shared__ R2 sHxz[2][2][TY][TX];
  __shared__ R2 sQy[2][TY][TX];
  __shared__ uint64_t s_bar[kEmStages];
  __shared__ int s_abort, s_tile;
  const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
  const int n = P.n, total = P.cta_start[n];
  auto design = [&](int b) -> int {  // the last d with cta_start[d] <= b
    int d = 0;
    while (d + 1 < n && P.cta_start[d + 1] <= b) ++d;
    return d;
  };
  // One call site for both modes: the tile code is then compiled once for the
  // batch kernel. (The slot is a run-time index into the parameter space; a
  // compile-time index per slot, one inlined tile body each, made the
  // compiler outline the bodies with kilobyte stack frames.)
  const bool persistent = work != nullptr;
  if (persistent && blockIdx.x == 0 && t0) *next_work = 0u;
  int b = (int)blockIdx.x;
  while (true) {
    if (persistent) {
      if (t0) s_tile = (int)atomicAdd(work, 1u);
      __syncthreads();
      b = s_tile;
      if (b >= total) return;
    }
    const int d = design(b);
    em_cta<R, I, TX, TY, false, false, false>(P.a[d], b - P.cta_start[d], step_off, fold, smem, sHxz, sQy, s_bar,
                                              &s_abort);
    if (!persistent) return;
    __syncthreads();  // every thread is past the tile's waits and its reads of s_tile
    if (s_abort) return;
    if (t0)
      for (int q = 0; q < kEmStages; ++q) mbar_inval(&s_bar[q]);
  }
}

// advance the device-resident source time index after a group of steps
__global__ void step_advance_kernel(long long *step_base, long long n) { *step_base += n; }

}  // namespace cosim
