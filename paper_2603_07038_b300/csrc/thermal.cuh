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
  R dt;
  R T_amb;
  R hconv[6];
  R *ratio_out;     // dt-limit kernel: C_i / (sum G + film) per node
};

// Voxel-layer sums of one node column (thread (i, j)) for the layer of cells
// kk, between node planes kk and kk+1. Each of the four voxels
// (i-1+dx, j-1+dy, kk) contributes k_c times its quarter cross-section to the
// edges it borders and rho_cp V / 8 to the node capacities. A node at plane k
// adds the sums of layers k-1 and k, so each layer is evaluated once and
// carried to the next plane in registers.
template <typename R>
struct LayerSums {
  R ax_p, ax_m;  // x-edges i -> i+1 and i-1 -> i: sum k_c * hy_c * hz / 4
  R ay_p, ay_m;  // y-edges j -> j+1 and j-1 -> j: sum k_c * hx_c * hz / 4
  R gz;          // z-edge kk -> kk+1 conductance: sum k_c hx_c hy_c / 4 / hz
  R cap;         // sum rho_cp V / 8
};

template <typename R>
__device__ __forceinline__ LayerSums<R> layer_sums(const R *s_mt, int m00, int m01, int m10, int m11, R hxm, R hx0,
                                                   R hym, R hy0, R hz, R ihz) {
  // m<dy><dx>: voxel (i-1+dx, j-1+dy, kk); missing voxels contribute zero
  const R k00 = mconst(s_mt, m00, M_K), k01 = mconst(s_mt, m01, M_K);
  const R k10 = mconst(s_mt, m10, M_K), k11 = mconst(s_mt, m11, M_K);
  const R q = R(0.25) * hz;
  LayerSums<R> L;
  L.ax_p = q * (k01 * hym + k11 * hy0);
  L.ax_m = q * (k00 * hym + k10 * hy0);
  L.ay_p = q * (k10 * hxm + k11 * hx0);
  L.ay_m = q * (k00 * hxm + k01 * hx0);
  L.gz = R(0.25) * ihz * (hym * (k00 * hxm + k01 * hx0) + hy0 * (k10 * hxm + k11 * hx0));
  L.cap = R(0.125) * hz *
          (hym * (mconst(s_mt, m00, M_RHOCP) * hxm + mconst(s_mt, m01, M_RHOCP) * hx0) +
           hy0 * (mconst(s_mt, m10, M_RHOCP) * hxm + mconst(s_mt, m11, M_RHOCP) * hx0));
  return L;
}

// One forward-Euler step (Eq. 5). Thread per (i, j) node column, marching in z.
// MODE 0: step T; MODE 1: write the per-node stability ratio C / (sum G + film).
template <typename R, int MODE>
__global__ void __launch_bounds__(512) thermal_kernel(const ThArgs<R> A) {  // blocks of 32 x (4, 8 or 16)
  extern __shared__ unsigned char smem_raw[];
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  const Geo<R> &g = A.g;
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i > nx || j > ny) return;
  const R hxm = i > 0 ? g.h[0][i - 1] : R(0), hx0 = i < nx ? g.h[0][i] : R(0);
  const R hym = j > 0 ? g.h[1][j - 1] : R(0), hy0 = j < ny ? g.h[1][j] : R(0);
  const R ihxm = i > 0 ? g.ih[0][i - 1] : R(0), ihx0 = i < nx ? g.ih[0][i] : R(0);
  const R ihym = j > 0 ? g.ih[1][j - 1] : R(0), ihy0 = j < ny ? g.ih[1][j] : R(0);
  // convective faces touching this column: x/y walls (per plane: times the dual z length)
  const R fxy = ((i == 0 ? A.hconv[0] : R(0)) + (i == nx ? A.hconv[1] : R(0))) * R(0.5) * (hym + hy0) +
                ((j == 0 ? A.hconv[2] : R(0)) + (j == ny ? A.hconv[3] : R(0))) * R(0.5) * (hxm + hx0);
  const R az = R(0.25) * (hxm + hx0) * (hym + hy0);  // z-face share of the node
  LayerSums<R> lo = {0, 0, 0, 0, 0, 0};
  const long long id0 = g.nid(i, j, 0);
  // Software pipeline: the values of plane k+1 (its voxels, the in-plane and
  // upper neighbours of T, the source) are requested one iteration ahead so
  // that their memory latency overlaps the arithmetic of plane k.
  auto load_plane = [&](int k, int m[4], R t[6], R &p) {
    m[0] = g.cell(i - 1, j - 1, k);
    m[1] = g.cell(i, j - 1, k);
    m[2] = g.cell(i - 1, j, k);
    m[3] = g.cell(i, j, k);
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
  R T_km1 = 0, T_c = MODE == 0 ? A.To[id0] : R(0);
  for (int k = 0; k <= nz; ++k) {
    const long long id = id0 + (long long)k * g.plane;
    if (k < nz) load_plane(k + 1, m_nxt, t_nxt, p_nxt);
    const R hz = k < nz ? g.h[2][k] : R(0), ihz = k < nz ? g.ih[2][k] : R(0);
    const R hzm = k > 0 ? g.h[2][k - 1] : R(0);
    const LayerSums<R> up = layer_sums(s_mt, m_cur[0], m_cur[1], m_cur[2], m_cur[3], hxm, hx0, hym, hy0, hz, ihz);
    const R Gxp = (lo.ax_p + up.ax_p) * ihx0, Gxm = (lo.ax_m + up.ax_m) * ihxm;
    const R Gyp = (lo.ay_p + up.ay_p) * ihy0, Gym = (lo.ay_m + up.ay_m) * ihym;
    const R Gzp = up.gz, Gzm = lo.gz;
    const R C = lo.cap + up.cap;
    R film = fxy * R(0.5) * (hzm + hz);
    if (k == 0) film += A.hconv[4] * az;
    if (k == nz) film += A.hconv[5] * az;
    if (MODE == 1) {
      A.ratio_out[id] = C / (Gxp + Gxm + Gyp + Gym + Gzp + Gzm + film);
    } else {
      const R T_kp1 = t_cur[0];
      const R flux = Gxm * (t_cur[1] - T_c) + Gxp * (t_cur[2] - T_c) + Gym * (t_cur[3] - T_c) +
                     Gyp * (t_cur[4] - T_c) + Gzm * (T_km1 - T_c) + Gzp * (T_kp1 - T_c) +
                     film * (A.T_amb - T_c) + p_cur;
      A.Tn[id] = T_c + A.dt * flux / C;
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

// ---- the same step with TMA-staged planes. A CTA of 32 x kThTY threads owns
// a 32 x kThTY tile of node columns (no halo compute: the update of a node
// reads only old temperatures) and marches in z. Per plane one thread copies
// into shared memory the temperature with a one-node halo (x from i0 - 4, the
// 16-byte rule; y from j0 - 1), the source power of the tile and the voxel IDs
// of the layer above (x from i0 - 16), plus the plane's z record; four
// stages, one mbarrier each, bounded waits. The arithmetic per node is that
// of thermal_kernel<R, 0>, term for term, so both give identical results.
constexpr int kThTY = 8;
constexpr int kThStages = 4, kThAhead = 3;
template <typename R>
struct ThStage {
  EmBox<R, kThTY + 2, 40> T;     // rows j0-1 .. j0+kThTY, columns i0-4 .. i0+35
  EmBox<R, kThTY, 32> P;         // the tile's nodes
  EmBox<uint8_t, kThTY + 1, 48> V;  // voxel rows j0-1 .. j0+kThTY-1, columns i0-16 ..
  EmBox<R, 1, 4> Z;              // hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
};
template <typename R>
__host__ __device__ constexpr size_t th_stage_offset(int nmat) {
  return ((size_t)(nmat + 1) * M_COLS * sizeof(R) + 127) & ~size_t(127);
}

template <typename R>
struct ThTmaArgs {
  ThArgs<R> a;               // geometry, T in / out, P, dt, films
  CUtensorMap tmT, tmP, tmV;  // boxes 40 x (kThTY+2), 32 x kThTY, 48 x (kThTY+1) (x, y, 1 plane)
  const R *zt;               // per node plane: hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
  int *err;
};

template <typename R>
__global__ void __launch_bounds__(32 * kThTY, 4) thermal_tma_kernel(const __grid_constant__ ThTmaArgs<R> TA) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const ThArgs<R> &A = TA.a;
  const Geo<R> &g = A.g;
  R *s_mt = reinterpret_cast<R *>(smem);
  ThStage<R> *stg = reinterpret_cast<ThStage<R> *>(smem + th_stage_offset<R>(g.nmat));
  __shared__ uint64_t bars[kThStages];
  __shared__ int s_abort;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const bool leader = tx == 0 && ty == 0;
  if (leader) {
    bool ok = (smem_u32(stg) & 127u) == 0 && (sizeof(ThStage<R>) & 127u) == 0 && ((size_t)&TA.tmT & 63u) == 0 &&
              ((size_t)&TA.tmP & 63u) == 0 && ((size_t)&TA.tmV & 63u) == 0;
    s_abort = ok ? 0 : 1;
    if (!ok) atomicExch(TA.err, 2);
    for (int q = 0; q < kThStages; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  stage_table(s_mt, g.mtab, (g.nmat + 1) * M_COLS);  // row nmat: all zero (outside the grid)
  __syncthreads();
  if (s_abort) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz, vd = g.nmat;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * kThTY;
  const int i = i0 + tx, j = j0 + ty;
  const bool act = i <= nx && j <= ny;
  const bool has_p = A.P != nullptr;
  const unsigned fixed_bytes =
      (unsigned)(((kThTY + 2) * 40 + (has_p ? kThTY * 32 : 0)) * (int)sizeof(R) + 4 * (int)sizeof(R));
  const unsigned vox_bytes = (unsigned)((kThTY + 1) * 48);
  auto issue = [&](int k) {
    if (k > nz) return;
    const int s = k % kThStages;
    ThStage<R> &S = stg[s];
    mbar_arrive_expect_tx(&bars[s], fixed_bytes + (k < nz ? vox_bytes : 0u));
    tma_load_3d(&S.T.v[0][0], &TA.tmT, i0 - 4, j0 - 1, k, &bars[s]);
    if (has_p) tma_load_3d(&S.P.v[0][0], &TA.tmP, i0, j0, k, &bars[s]);
    if (k < nz) tma_load_3d(&S.V.v[0][0], &TA.tmV, i0 - 16, j0 - 1, k, &bars[s]);
    bulk_load(&S.Z.v[0][0], TA.zt + 4 * (size_t)k, 4 * sizeof(R), &bars[s]);
  };
  const R hxm = (act && i > 0) ? g.h[0][i - 1] : R(0), hx0 = (act && i < nx) ? g.h[0][i] : R(0);
  const R hym = (act && j > 0) ? g.h[1][j - 1] : R(0), hy0 = (act && j < ny) ? g.h[1][j] : R(0);
  const R ihxm = (act && i > 0) ? g.ih[0][i - 1] : R(0), ihx0 = (act && i < nx) ? g.ih[0][i] : R(0);
  const R ihym = (act && j > 0) ? g.ih[1][j - 1] : R(0), ihy0 = (act && j < ny) ? g.ih[1][j] : R(0);
  const R fxy = ((i == 0 ? A.hconv[0] : R(0)) + (i == nx ? A.hconv[1] : R(0))) * R(0.5) * (hym + hy0) +
                ((j == 0 ? A.hconv[2] : R(0)) + (j == ny ? A.hconv[3] : R(0))) * R(0.5) * (hxm + hx0);
  const R az = R(0.25) * (hxm + hx0) * (hym + hy0);
  const bool cx0 = i - 1 >= 0 && i - 1 < nx, cx1 = i < nx, cy0 = j - 1 >= 0 && j - 1 < ny, cy1 = j < ny;
  const long long id0 = act ? g.nid(i, j, 0) : 0;
  const int cT = tx + 4, cV = tx + 15, r1 = ty + 1;  // columns / row of this node in the boxes
  LayerSums<R> lo = {0, 0, 0, 0, 0, 0};
  R T_km1 = 0;
  if (leader)
    for (int q = 0; q < kThAhead; ++q) issue(q);
  for (int k = 0; k <= nz; ++k) {
    {
      bool ok = mbar_wait(&bars[k % kThStages], (unsigned)(k / kThStages) & 1u);
      if (k + 1 <= nz) ok = mbar_wait(&bars[(k + 1) % kThStages], (unsigned)((k + 1) / kThStages) & 1u) && ok;
      if (!ok) s_abort = 1;
    }
    __syncthreads();  // every thread is done with plane k-1: its stage can be refilled
    if (s_abort) {
      if (leader) {
        for (int q = k; q <= k + kThAhead && q <= nz; ++q)
          mbar_wait(&bars[q % kThStages], (unsigned)(q / kThStages) & 1u);
        atomicExch(TA.err, 1);
      }
      return;
    }
    if (leader) {
      fence_proxy_async_smem();
      issue(k + kThAhead);
    }
    const ThStage<R> &S0 = stg[k % kThStages];
    const ThStage<R> &S1 = stg[(k + 1) % kThStages];
    R hz, ihz, idz_unused, hzm;
    {
      const R *z = &S0.Z.v[0][0];
      hz = z[0], ihz = z[1], idz_unused = z[2], hzm = z[3];
      (void)idz_unused;
    }
    const bool kz = k < nz;
    const int m00 = (kz && cx0 && cy0) ? (int)S0.V.v[ty][cV] : vd;
    const int m01 = (kz && cx1 && cy0) ? (int)S0.V.v[ty][cV + 1] : vd;
    const int m10 = (kz && cx0 && cy1) ? (int)S0.V.v[r1][cV] : vd;
    const int m11 = (kz && cx1 && cy1) ? (int)S0.V.v[r1][cV + 1] : vd;
    const LayerSums<R> up = layer_sums(s_mt, m00, m01, m10, m11, hxm, hx0, hym, hy0, hz, ihz);
    const R Gxp = (lo.ax_p + up.ax_p) * ihx0, Gxm = (lo.ax_m + up.ax_m) * ihxm;
    const R Gyp = (lo.ay_p + up.ay_p) * ihy0, Gym = (lo.ay_m + up.ay_m) * ihym;
    const R Gzp = up.gz, Gzm = lo.gz;
    const R C = lo.cap + up.cap;
    R film = fxy * R(0.5) * (hzm + hz);
    if (k == 0) film += A.hconv[4] * az;
    if (k == nz) film += A.hconv[5] * az;
    const R T_c = S0.T.v[r1][cT];
    const R T_kp1 = kz ? S1.T.v[r1][cT] : R(0);
    const R p = has_p ? S0.P.v[ty][tx] : R(0);
    const R flux = Gxm * (S0.T.v[r1][cT - 1] - T_c) + Gxp * (S0.T.v[r1][cT + 1] - T_c) +
                   Gym * (S0.T.v[ty][cT] - T_c) + Gyp * (S0.T.v[r1 + 1][cT] - T_c) + Gzm * (T_km1 - T_c) +
                   Gzp * (T_kp1 - T_c) + film * (A.T_amb - T_c) + p;
    if (act) A.Tn[id0 + (long long)k * g.plane] = T_c + A.dt * flux / C;
    T_km1 = T_c;
    lo = up;
  }
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
