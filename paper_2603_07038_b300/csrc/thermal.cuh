// Nodal heat diffusion (Sec. II-A, Eqs. 4-5) and the Joule-source hand-off.
//
// T lives on grid nodes; the stencil is the 7-point form of
// M_kk = V0a^T D_k V0: node i exchanges G_ij (T_j - T_i) with its six
// neighbours, G_ij = (sum over the <=4 voxels around the edge of
// k_c * quarter cross-section) / edge length; the node's heat capacity is
// C_i = sum over its <=8 voxels of rho_cp V / 8; a convective face adds
// h A_i (T_amb - T_i), A_i the node's share of the face.
// Conductances and capacities are recomputed from the voxel IDs on the fly
// (1 byte per cell streamed) instead of being stored per node.
//
// The arithmetic of a node is written once (th_layer, th_coeffs, th_update)
// for a scalar or for a pair of adjacent nodes; both kernels below use it.
// It feeds no product into an addition (products enter FMAs only), so no
// contraction can differ between the forms: every launch shape gives the
// same bits.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "common.cuh"

namespace cosim {

template <typename R>
struct ThArgs {
  Geo<R> g;
  const R *To;
  R *Tn;
  const R *P;       // W per node, may be null
  const R *zt;      // per node plane k: hz(k), 1/hz(k), 1/dual_z(k), hz(k-1) (zero outside the grid)
  R dt;
  R T_amb;
  R hconv[6];
  R *ratio_out;     // dt-limit kernel: C_i / (sum G + film) per node
};

// Per-material {k, rho_cp} pairs (rows 0 .. nmat, row nmat all zero) from the
// device material table into shared memory (call by all threads, then sync).
template <typename R>
__device__ __forceinline__ void stage_kc(typename Pair2<R>::T *dst, const R *mtab, int nmat) {
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  const int t = (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
  for (int m = t; m <= nmat; m += nt) {
    typename Pair2<R>::T v;
    v.x = mtab[m * M_COLS + M_K];
    v.y = mtab[m * M_COLS + M_RHOCP];
    dst[m] = v;
  }
}

// Constants of a node column (i, j); V is R for one node or R2 for a pair.
// Cell sizes and quarter inverse lengths of cells outside the grid are zero,
// which removes every term of a voxel outside the grid whatever its material
// value (any finite value).
template <typename V>
struct ThCol {
  V hxm, hx0, hym, hy0;  // sizes of the cells i-1, i (x) and j-1, j (y)
  V qxm, qx0, qym, qy0;  // a quarter of their inverse sizes
  V fxy;                 // lateral film: sum of (h_conv x half the face's other extent) / 2
  V az;                  // the node's share of a z face
};

template <typename R>
__device__ __forceinline__ ThCol<R> th_column_h(const Geo<R> &g, const R *hconv, int i, int j) {
  const int nx = g.nx, ny = g.ny;
  const bool in = i >= 0 && i <= nx && j >= 0 && j <= ny;
  ThCol<R> c;
  c.hxm = (in && i > 0) ? g.h[0][i - 1] : R(0);
  c.hx0 = (in && i < nx) ? g.h[0][i] : R(0);
  c.hym = (in && j > 0) ? g.h[1][j - 1] : R(0);
  c.hy0 = (in && j < ny) ? g.h[1][j] : R(0);
  c.qxm = (in && i > 0) ? mul_(R(0.25), g.ih[0][i - 1]) : R(0);
  c.qx0 = (in && i < nx) ? mul_(R(0.25), g.ih[0][i]) : R(0);
  c.qym = (in && j > 0) ? mul_(R(0.25), g.ih[1][j - 1]) : R(0);
  c.qy0 = (in && j < ny) ? mul_(R(0.25), g.ih[1][j]) : R(0);
  const R hcx = add_(i == 0 ? hconv[0] : R(0), i == nx ? hconv[1] : R(0));
  const R hcy = add_(j == 0 ? hconv[2] : R(0), j == ny ? hconv[3] : R(0));
  c.fxy = mul_(R(0.25), fma_(hcx, add_(c.hym, c.hy0), mul_(hcy, add_(c.hxm, c.hx0))));
  c.az = mul_(R(0.25), mul_(add_(c.hxm, c.hx0), add_(c.hym, c.hy0)));
  return c;
}
template <typename R>
__device__ __forceinline__ ThCol<R> th_column(const Geo<R> &g, const ThArgs<R> &A, int i, int j) {
  return th_column_h(g, A.hconv, i, j);
}

template <typename R>
__device__ __forceinline__ ThCol<typename Pair2<R>::T> th_pair(const ThCol<R> &a, const ThCol<R> &b) {
  ThCol<typename Pair2<R>::T> c;
  c.hxm = {a.hxm, b.hxm}, c.hx0 = {a.hx0, b.hx0}, c.hym = {a.hym, b.hym}, c.hy0 = {a.hy0, b.hy0};
  c.qxm = {a.qxm, b.qxm}, c.qx0 = {a.qx0, b.qx0}, c.qym = {a.qym, b.qym}, c.qy0 = {a.qy0, b.qy0};
  c.fxy = {a.fxy, b.fxy}, c.az = {a.az, b.az};
  return c;
}

// Sums of one voxel layer seen from a node column: the voxels
// (i-1+dx, j-1+dy) of the layer (k<dy><dx> conductivities, c<dy><dx>
// capacities) give, before the layer height and the quarter factor,
//   kxm / kxp: the x-edges i-1 -> i and i -> i+1 (k_c times the cell's y size),
//   kym / kyp: the y-edges j-1 -> j and j -> j+1 (k_c times the x size),
//   gzs: the z-edge sum of k_c hx hy, cs: the capacity sum of rho_cp hx hy.
// A node at plane k adds the sums of the layers k-1 and k, so each layer is
// formed once and carried to the next plane in registers.
template <typename V>
struct ThLayer {
  V kxm, kxp, kym, kyp, gzs, cs;
};

template <typename V>
__device__ __forceinline__ ThLayer<V> th_layer(V k00, V k01, V k10, V k11, V c00, V c01, V c10, V c11,
                                               const ThCol<V> &c) {
  ThLayer<V> L;
  L.kxm = fma_(k00, c.hym, mul_(k10, c.hy0));
  L.kxp = fma_(k01, c.hym, mul_(k11, c.hy0));
  L.kym = fma_(k00, c.hxm, mul_(k01, c.hx0));
  L.kyp = fma_(k10, c.hxm, mul_(k11, c.hx0));
  L.gzs = fma_(c.hym, L.kym, mul_(c.hy0, L.kyp));
  L.cs = fma_(c.hym, fma_(c00, c.hxm, mul_(c01, c.hx0)), mul_(c.hy0, fma_(c10, c.hxm, mul_(c11, c.hx0))));
  return L;
}

template <typename V, typename R>
__device__ __forceinline__ ThLayer<V> th_layer_zero() {
  const V z = bc_<V>(R(0));
  return {z, z, z, z, z, z};
}

// Conductances of the six edges, the film coefficient and the capacity of a
// node at plane k from the layers below (lo, height hzm) and above (up, hz);
// gz carries the z-edge conductance: in, the edge below (the previous plane's
// upper edge); out, this plane's upper edge.
template <typename V>
struct ThCoeffs {
  V Gxm, Gxp, Gym, Gyp, Gzm, Gzp, film, C;
};

template <typename V, typename R>
__device__ __forceinline__ ThCoeffs<V> th_coeffs(const ThCol<V> &c, const ThLayer<V> &lo, const ThLayer<V> &up,
                                                 R hz, R ihz, R hzm, bool bottom, bool top, const R *hconv, V &gz) {
  ThCoeffs<V> q;
  const V vz = bc_<V>(hz), vzm = bc_<V>(hzm);
  q.Gxm = mul_(fma_(vzm, lo.kxm, mul_(vz, up.kxm)), c.qxm);
  q.Gxp = mul_(fma_(vzm, lo.kxp, mul_(vz, up.kxp)), c.qx0);
  q.Gym = mul_(fma_(vzm, lo.kym, mul_(vz, up.kym)), c.qym);
  q.Gyp = mul_(fma_(vzm, lo.kyp, mul_(vz, up.kyp)), c.qy0);
  q.Gzm = gz;
  q.Gzp = mul_(up.gzs, bc_<V>(mul_(R(0.25), ihz)));
  gz = q.Gzp;
  q.C = mul_(fma_(vzm, lo.cs, mul_(vz, up.cs)), bc_<V>(R(0.125)));
  q.film = mul_(c.fxy, bc_<V>(add_(hzm, hz)));
  if (bottom) q.film = fma_(bc_<V>(hconv[4]), c.az, q.film);
  if (top) q.film = fma_(bc_<V>(hconv[5]), c.az, q.film);
  return q;
}

// Forward-Euler step of the node (Eq. 5): T + dt (sum G (T_nb - T) + film
// (T_amb - T) + P) / C.
template <typename V, typename R>
__device__ __forceinline__ V th_update(const ThCoeffs<V> &q, V Tc, V Tim, V Tip, V Tjm, V Tjp, V Tkm, V Tkp, V p,
                                       R T_amb, R dt) {
  V f = fma_(q.Gxm, sub_(Tim, Tc), p);
  f = fma_(q.Gxp, sub_(Tip, Tc), f);
  f = fma_(q.Gym, sub_(Tjm, Tc), f);
  f = fma_(q.Gyp, sub_(Tjp, Tc), f);
  f = fma_(q.Gzm, sub_(Tkm, Tc), f);
  f = fma_(q.Gzp, sub_(Tkp, Tc), f);
  f = fma_(q.film, sub_(bc_<V>(T_amb), Tc), f);
  return fma_(mul_(bc_<V>(dt), f), rcp_(q.C), Tc);
}

// One forward-Euler step (Eq. 5). Thread per (i, j) node column, marching in z.
// MODE 0: step T; MODE 1: write the per-node stability ratio C / (sum G + film).
template <typename R, int MODE>
__global__ void __launch_bounds__(512) thermal_kernel(const ThArgs<R> A) {  // blocks of 32 x (4, 8 or 16)
  using R2 = typename Pair2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  R2 *s_kc = reinterpret_cast<R2 *>(smem_raw);
  const Geo<R> &g = A.g;
  stage_kc<R>(s_kc, g.mtab, g.nmat);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz, vd = g.nmat;
  if (i > nx || j > ny) return;
  const ThCol<R> c = th_column(g, A, i, j);
  const long long id0 = g.nid(i, j, 0);
  // Software pipeline: the values of plane k+1 (its voxels, the in-plane and
  // upper neighbours of T, the source) are requested one iteration ahead so
  // that their memory latency overlaps the arithmetic of plane k.
  auto load_plane = [&](int k, int m[4], R t[6], R &p) {
    m[0] = g.cell(i - 1, j - 1, k);
    m[1] = g.cell(i, j - 1, k);
    m[2] = g.cell(i - 1, j, k);
    m[3] = g.cell(i, j, k);
#pragma unroll
    for (int q = 0; q < 4; ++q) m[q] = m[q] < 0 ? vd : m[q];
    if (MODE == 0 && k <= nz) {
      const long long id = id0 + (long long)k * g.plane;
      t[0] = k < nz ? A.To[id + g.plane] : R(0);
      t[1] = i > 0 ? A.To[id - 1] : R(0);
      t[2] = i < nx ? A.To[id + 1] : R(0);
      t[3] = j > 0 ? A.To[id - g.px] : R(0);
      t[4] = j < ny ? A.To[id + g.px] : R(0);
      p = A.P != nullptr ? A.P[id] : R(0);
    }
  };
  int m_cur[4], m_nxt[4];
  R t_cur[6] = {0, 0, 0, 0, 0, 0}, t_nxt[6] = {0, 0, 0, 0, 0, 0}, p_cur = 0, p_nxt = 0;
  load_plane(0, m_cur, t_cur, p_cur);
  R T_km1 = 0, T_c = MODE == 0 ? A.To[id0] : R(0), gz = 0;
  ThLayer<R> lo = th_layer_zero<R, R>();
  for (int k = 0; k <= nz; ++k) {
    const long long id = id0 + (long long)k * g.plane;
    if (k < nz) load_plane(k + 1, m_nxt, t_nxt, p_nxt);
    const R hz = A.zt[4 * k], ihz = A.zt[4 * k + 1], hzm = A.zt[4 * k + 3];
    const R2 v0 = s_kc[m_cur[0]], v1 = s_kc[m_cur[1]], v2 = s_kc[m_cur[2]], v3 = s_kc[m_cur[3]];
    const ThLayer<R> up = th_layer<R>(v0.x, v1.x, v2.x, v3.x, v0.y, v1.y, v2.y, v3.y, c);
    const ThCoeffs<R> q = th_coeffs<R, R>(c, lo, up, hz, ihz, hzm, k == 0, k == nz, A.hconv, gz);
    if (MODE == 1) {
      A.ratio_out[id] = q.C / (q.Gxp + q.Gxm + q.Gyp + q.Gym + q.Gzp + q.Gzm + q.film);
    } else {
      const R T_kp1 = t_cur[0];
      A.Tn[id] = th_update<R, R>(q, T_c, t_cur[1], t_cur[2], t_cur[3], t_cur[4], T_km1, T_kp1, p_cur, A.T_amb, A.dt);
      T_km1 = T_c;
      T_c = T_kp1;
    }
    lo = up;
#pragma unroll
    for (int q = 0; q < 4; ++q) m_cur[q] = m_nxt[q];
#pragma unroll
    for (int q = 0; q < 6; ++q) t_cur[q] = t_nxt[q];
    p_cur = p_nxt;
  }
}

// ---- the same step with TMA-staged planes and NP node pairs per thread.
// A CTA of 32 x kThTY threads owns a th_tx(NP) x kThTY tile of node columns
// (thread tx: nodes i0 + 2 NP tx .. i0 + 2 NP tx + 2 NP - 1 of row
// j0 + ty; no halo compute: the update of a node reads only old
// temperatures) and marches in z. Per plane one thread copies into shared
// memory the temperature with a one-node halo (x from i0 - 4, the 16-byte
// rule; y from j0 - 1), the tile's source power and the voxel IDs of the
// layer above (x from i0 - 16), plus the plane's z record; four stages, one
// mbarrier each, bounded waits. Positions outside the grid arrive as zero (a
// valid material ID and a finite temperature that the zero geometry factors
// then remove). More nodes per thread share the per-plane waits, barrier and
// addressing; each pair's arithmetic is the pair form of th_layer /
// th_coeffs / th_update.
// NP node pairs per thread (1 or 2, chosen per grid: two pairs amortise the
// per-plane work better, one pair keeps more CTAs in flight on small grids).
constexpr int kThTY = 8;
constexpr int kThStages = 4, kThAhead = 3;
__host__ __device__ constexpr int th_tx(int np) { return 64 * np; }         // nodes per tile row
__host__ __device__ constexpr int th_box_t(int np) { return 64 * np + 8; }  // T box: columns i0-4 .. i0+TX+3
__host__ __device__ constexpr int th_box_v(int np) { return 64 * np + 32; } // voxel box: columns i0-16 .. i0+TX+15
template <typename R, int NP>
struct ThStage {
  EmBox<R, kThTY + 2, th_box_t(NP)> T;        // rows j0-1 .. j0+kThTY
  EmBox<R, kThTY, th_tx(NP)> P;               // the tile's nodes
  EmBox<uint8_t, kThTY + 1, th_box_v(NP)> V;  // voxel rows j0-1 .. j0+kThTY-1
  EmBox<R, 1, 4> Z;                           // hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
};
template <typename R>
__host__ __device__ constexpr size_t th_stage_offset(int nmat) {
  return ((size_t)(nmat + 1) * sizeof(typename Pair2<R>::T) + 127) & ~size_t(127);
}

template <typename R>
struct ThTmaArgs {
  ThArgs<R> a;                // geometry, T in / out, P, z records, dt, films
  CUtensorMap tmT, tmP, tmV;  // boxes th_box_t x (kThTY+2), th_tx x kThTY, th_box_v x (kThTY+1) (one plane)
  int *err;
  long long wait;             // bound of the waits for staged planes, SM clock cycles
  unsigned long long *peak;   // the maximum of the written T (its ordered_bits image) goes here; null: not tracked
};

// Order-preserving integer image of a value (larger value, larger image): an
// atomic maximum over the images is the maximum of the values in any order.
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}
// warp maximum of v into *peak (every lane of the warp calls it)
template <typename R>
__device__ __forceinline__ void peak_max(R v, unsigned long long *peak) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(peak, ordered_bits((double)v));
}

// resident CTAs per SM the kernel is compiled for (FP32 one / two pairs)
#ifndef COSIM_TH1_MIN_CTAS
#define COSIM_TH1_MIN_CTAS 3
#endif
#ifndef COSIM_TH2_MIN_CTAS
#define COSIM_TH2_MIN_CTAS 2
#endif
#ifndef COSIM_TH_UNROLL
#define COSIM_TH_UNROLL 8
#endif
constexpr int kThUnroll = COSIM_TH_UNROLL;  // plane-loop unroll (twice the stage count by default)
template <typename R, int NP>
__global__ void __launch_bounds__(32 * kThTY, sizeof(R) == 4 ? (NP == 1 ? COSIM_TH1_MIN_CTAS : COSIM_TH2_MIN_CTAS)
                                                             : (NP == 1 ? 2 : 1))
    thermal_tma_kernel(const __grid_constant__ ThTmaArgs<R> TA) {
  using R2 = typename Pair2<R>::T;
  constexpr int kThTX = th_tx(NP), kThBoxT = th_box_t(NP), kThBoxV = th_box_v(NP);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const ThArgs<R> &A = TA.a;
  const Geo<R> &g = A.g;
  R2 *s_kc = reinterpret_cast<R2 *>(smem);
  ThStage<R, NP> *stg = reinterpret_cast<ThStage<R, NP> *>(smem + th_stage_offset<R>(g.nmat));
  __shared__ uint64_t bars[kThStages];
  __shared__ int s_abort;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool leader = tx == 0 && ty == 0;
  if (leader) {
    bool ok = (smem_u32(stg) & 127u) == 0 && (sizeof(ThStage<R, NP>) & 127u) == 0 && ((size_t)&TA.tmT & 63u) == 0 &&
              ((size_t)&TA.tmP & 63u) == 0 && ((size_t)&TA.tmV & 63u) == 0;
    s_abort = ok ? 0 : 1;
    if (!ok) atomicExch(TA.err, 2);
    for (int q = 0; q < kThStages; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  stage_kc<R>(s_kc, g.mtab, g.nmat);
  __syncthreads();
  if (s_abort) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = blockIdx.x * kThTX, j0 = blockIdx.y * kThTY;
  const int ia = i0 + 2 * NP * tx, j = j0 + ty;  // first node of the thread, row j
  const int n_act = j <= ny ? max(0, min(2 * NP, nx + 1 - ia)) : 0;  // nodes of the thread inside the grid
  const bool has_p = A.P != nullptr;
  const unsigned stage_bytes = (unsigned)(((kThTY + 2) * kThBoxT + (has_p ? kThTY * kThTX : 0)) * (int)sizeof(R) +
                                          4 * (int)sizeof(R) + (kThTY + 1) * kThBoxV);
  auto issue = [&](int k) {
    if (k > nz) return;
    const int s = k & (kThStages - 1);
    ThStage<R, NP> &S = stg[s];
    mbar_arrive_expect_tx(&bars[s], stage_bytes);
    tma_load_3d(&S.T.v[0][0], &TA.tmT, i0 - 4, j0 - 1, k, &bars[s]);
    if (has_p) tma_load_3d(&S.P.v[0][0], &TA.tmP, i0, j0, k, &bars[s]);
    // the voxel layer above plane k; at k = nz the box lies wholly above the
    // grid and arrives as zeros
    tma_load_3d(&S.V.v[0][0], &TA.tmV, i0 - 16, j0 - 1, k, &bars[s]);
    bulk_load(&S.Z.v[0][0], A.zt + 4 * (size_t)k, 4 * sizeof(R), &bars[s]);
  };
  ThCol<R2> c[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) c[q] = th_pair<R>(th_column(g, A, ia + 2 * q, j), th_column(g, A, ia + 2 * q + 1, j));
  const int cT = 2 * NP * tx + 4, cV = 2 * NP * tx + 15, r1 = ty + 1;  // columns / row of node ia in the boxes
  R *tp = A.Tn + (n_act > 0 ? g.nid(ia, j, 0) : 0);
  ThLayer<R2> lo[NP];
  R2 T_km1[NP], gz[NP];
  R t_max = R(-3.0e38);  // the largest T written (peak tracking)
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    lo[q] = th_layer_zero<R2, R>();
    T_km1[q] = gz[q] = bc_<R2>(R(0));
  }
  if (leader)
    for (int q = 0; q < kThAhead; ++q) issue(q);
  bool ok0 = mbar_wait(&bars[0], 0u, TA.wait);
  // unrolled by twice the stage count: stage slots and carried sums resolve
  // at compile time (measured: 4 -> 0.473, 8 -> 0.453 ms per full-package step)
#pragma unroll kThUnroll
  for (int k = 0; k <= nz; ++k) {
    {  // plane k landed one iteration earlier (or above, for k = 0); wait for plane k+1
      const bool ok =
          (k + 1 > nz || mbar_wait(&bars[(k + 1) & (kThStages - 1)], (unsigned)((k + 1) / kThStages) & 1u, TA.wait)) &&
          ok0;
      if (!ok) s_abort = 1;
    }
    __syncthreads();  // every thread is done with plane k-1: its stage can be refilled
    if (s_abort) {
      if (leader) {
        for (int q = k; q < k + kThAhead && q <= nz; ++q)  // the planes issued so far
          mbar_wait(&bars[q & (kThStages - 1)], (unsigned)(q / kThStages) & 1u, TA.wait);
        atomicExch(TA.err, 1);
      }
      return;
    }
    if (leader) {
      fence_proxy_async_smem();
      issue(k + kThAhead);
    }
    const ThStage<R, NP> &S0 = stg[k & (kThStages - 1)];
    const ThStage<R, NP> &S1 = stg[(k + 1) & (kThStages - 1)];
    const R hz = S0.Z.v[0][0], ihz = S0.Z.v[0][1], hzm = S0.Z.v[0][3];
    // {k, rho_cp} of the voxels ia-1 .. ia+2NP-1 in rows j-1 (a) and j (b)
    R2 a[2 * NP + 1], b[2 * NP + 1];
#pragma unroll
    for (int q = 0; q <= 2 * NP; ++q) {
      a[q] = s_kc[S0.V.v[ty][cV + q]];
      b[q] = s_kc[S0.V.v[r1][cV + q]];
    }
    R2 Tc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) Tc[q] = ldv_<R2>(&S0.T.v[r1][cT + 2 * q]);
    const R T_left = S0.T.v[r1][cT - 1], T_right = S0.T.v[r1][cT + 2 * NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const int o = cT + 2 * q;
      const ThLayer<R2> up = th_layer<R2>(R2{a[2 * q].x, a[2 * q + 1].x}, R2{a[2 * q + 1].x, a[2 * q + 2].x},
                                          R2{b[2 * q].x, b[2 * q + 1].x}, R2{b[2 * q + 1].x, b[2 * q + 2].x},
                                          R2{a[2 * q].y, a[2 * q + 1].y}, R2{a[2 * q + 1].y, a[2 * q + 2].y},
                                          R2{b[2 * q].y, b[2 * q + 1].y}, R2{b[2 * q + 1].y, b[2 * q + 2].y}, c[q]);
      const ThCoeffs<R2> cf = th_coeffs<R2, R>(c[q], lo[q], up, hz, ihz, hzm, k == 0, k == nz, A.hconv, gz[q]);
      const R2 Tjm = ldv_<R2>(&S0.T.v[ty][o]), Tjp = ldv_<R2>(&S0.T.v[r1 + 1][o]);
      const R2 Tkp = k < nz ? ldv_<R2>(&S1.T.v[r1][o]) : bc_<R2>(R(0));
      const R2 Tim = {q == 0 ? T_left : Tc[q - 1].y, Tc[q].x};
      const R2 Tip = {Tc[q].y, q == NP - 1 ? T_right : Tc[q + 1].x};
      const R2 p = has_p ? ldv_<R2>(&S0.P.v[ty][2 * NP * tx + 2 * q]) : bc_<R2>(R(0));
      const R2 Tn = th_update<R2, R>(cf, Tc[q], Tim, Tip, Tjm, Tjp, T_km1[q], Tkp, p, A.T_amb, A.dt);
      if (n_act >= 2 * q + 2) {
        stv_(tp + 2 * q, Tn);
        t_max = fmax(t_max, fmax(Tn.x, Tn.y));
      } else if (n_act == 2 * q + 1) {
        tp[2 * q] = Tn.x;
        t_max = fmax(t_max, Tn.x);
      }
      T_km1[q] = Tc[q];
      lo[q] = up;
    }
    tp += g.plane;
  }
  if (TA.peak != nullptr) peak_max(t_max, TA.peak);
}

// Joule finalisation: op 1 -> P = Q * inv_t (burst-averaged power per node);
// op 2 -> T += Q / C_i (energy deposited at once). Thread per (i, j) column.
template <typename R>
__global__ void __launch_bounds__(256) joule_finalize_kernel(Geo<R> g, const double *Q, R *P, R *T, double inv_t,
                                                              int op) {
  extern __shared__ unsigned char smem_raw[];
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.nx || j > g.ny) return;
  for (int k = 0; k <= g.nz; ++k) {
    const long long id = g.nid(i, j, k);
    if (op == 1) {
      P[id] = (R)(Q[id] * inv_t);
    } else {
      R C = 0;
      for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            const int m = g.cell(i - 1 + dx, j - 1 + dy, k - 1 + dz);
            if (m < 0) continue;
            C += s_mt[m * M_COLS + M_RHOCP] * g.h[0][i - 1 + dx] * g.h[1][j - 1 + dy] * g.h[2][k - 1 + dz];
          }
      T[id] = (R)((double)T[id] + Q[id] / (double)(R(0.125) * C));
    }
  }
}

}  // namespace cosim
