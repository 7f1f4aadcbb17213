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

// Terms of node (i,j,k) from its eight voxels c[dz][dy][dx] = (i-1+dx, j-1+dy, k-1+dz).
template <typename R>
struct NodeTerms {
  R C;           // heat capacity
  R G[6];        // conductances to -x, +x, -y, +y, -z, +z
  R film;        // sum of h_f * A_f over convective faces at the node
};

template <typename R>
__device__ __forceinline__ NodeTerms<R> node_terms(const R *s_mt, const int c[2][2][2], const R hx[2],
                                                   const R hy[2], const R hz[2], const R ih[6],
                                                   const bool onface[6], const R hconv[6]) {
  NodeTerms<R> t;
  R k[2][2][2], C = 0;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int m = c[dz][dy][dx];
        k[dz][dy][dx] = mconst(s_mt, m, M_K);
        C += mconst(s_mt, m, M_RHOCP) * hx[dx] * hy[dy] * hz[dz];
      }
  t.C = R(0.125) * C;
  const R q = R(0.25);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    t.G[0 + s] = q * ih[0 + s] *
                 (k[0][0][s] * hy[0] * hz[0] + k[0][1][s] * hy[1] * hz[0] + k[1][0][s] * hy[0] * hz[1] +
                  k[1][1][s] * hy[1] * hz[1]);
    t.G[2 + s] = q * ih[2 + s] *
                 (k[0][s][0] * hx[0] * hz[0] + k[0][s][1] * hx[1] * hz[0] + k[1][s][0] * hx[0] * hz[1] +
                  k[1][s][1] * hx[1] * hz[1]);
    t.G[4 + s] = q * ih[4 + s] *
                 (k[s][0][0] * hx[0] * hy[0] + k[s][0][1] * hx[1] * hy[0] + k[s][1][0] * hx[0] * hy[1] +
                  k[s][1][1] * hx[1] * hy[1]);
  }
  const R ax = R(0.25) * (hy[0] + hy[1]) * (hz[0] + hz[1]);
  const R ay = R(0.25) * (hx[0] + hx[1]) * (hz[0] + hz[1]);
  const R az = R(0.25) * (hx[0] + hx[1]) * (hy[0] + hy[1]);
  R f = 0;
  if (onface[0]) f += hconv[0] * ax;
  if (onface[1]) f += hconv[1] * ax;
  if (onface[2]) f += hconv[2] * ay;
  if (onface[3]) f += hconv[3] * ay;
  if (onface[4]) f += hconv[4] * az;
  if (onface[5]) f += hconv[5] * az;
  t.film = f;
  return t;
}

// One forward-Euler step (Eq. 5). Thread per (i, j) column, marching in z;
// the voxel IDs of the layer below are carried in registers.
// MODE 0: step T; MODE 1: write the per-node stability ratio instead.
template <typename R, int MODE>
__global__ void __launch_bounds__(256) thermal_kernel(const ThArgs<R> A) {
  extern __shared__ unsigned char smem_raw[];
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  const Geo<R> &g = A.g;
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i > nx || j > ny) return;
  R hx[2], hy[2], ih[6];
  hx[0] = i > 0 ? g.h[0][i - 1] : R(0);
  hx[1] = i < nx ? g.h[0][i] : R(0);
  hy[0] = j > 0 ? g.h[1][j - 1] : R(0);
  hy[1] = j < ny ? g.h[1][j] : R(0);
  ih[0] = i > 0 ? g.ih[0][i - 1] : R(0);
  ih[1] = i < nx ? g.ih[0][i] : R(0);
  ih[2] = j > 0 ? g.ih[1][j - 1] : R(0);
  ih[3] = j < ny ? g.ih[1][j] : R(0);
  int c[2][2][2];
  c[0][0][0] = c[0][0][1] = c[0][1][0] = c[0][1][1] = -1;
  const long long id0 = g.nid(i, j, 0);
  R T_km1 = 0, T_c = A.To[id0];
  for (int k = 0; k <= nz; ++k) {
    const long long id = id0 + (long long)k * g.plane;
    c[1][0][0] = g.cell(i - 1, j - 1, k);
    c[1][0][1] = g.cell(i, j - 1, k);
    c[1][1][0] = g.cell(i - 1, j, k);
    c[1][1][1] = g.cell(i, j, k);
    R hz[2];
    hz[0] = k > 0 ? g.h[2][k - 1] : R(0);
    hz[1] = k < nz ? g.h[2][k] : R(0);
    ih[4] = k > 0 ? g.ih[2][k - 1] : R(0);
    ih[5] = k < nz ? g.ih[2][k] : R(0);
    const bool onface[6] = {i == 0, i == nx, j == 0, j == ny, k == 0, k == nz};
    const NodeTerms<R> t = node_terms(s_mt, c, hx, hy, hz, ih, onface, A.hconv);
    if (MODE == 1) {
      R gs = t.film;
#pragma unroll
      for (int s = 0; s < 6; ++s) gs += t.G[s];
      A.ratio_out[id] = t.C / gs;
    } else {
      const R T_kp1 = k < nz ? A.To[id + g.plane] : R(0);
      const R T_xm = i > 0 ? A.To[id - 1] : R(0), T_xp = i < nx ? A.To[id + 1] : R(0);
      const R T_ym = j > 0 ? A.To[id - g.px] : R(0), T_yp = j < ny ? A.To[id + g.px] : R(0);
      R flux = t.G[0] * (T_xm - T_c) + t.G[1] * (T_xp - T_c) + t.G[2] * (T_ym - T_c) + t.G[3] * (T_yp - T_c) +
               t.G[4] * (T_km1 - T_c) + t.G[5] * (T_kp1 - T_c) + t.film * (A.T_amb - T_c);
      if (A.P != nullptr) flux += A.P[id];
      A.Tn[id] = T_c + A.dt * flux / t.C;
      T_km1 = T_c;
      T_c = T_kp1;
    }
    c[0][0][0] = c[1][0][0];
    c[0][0][1] = c[1][0][1];
    c[0][1][0] = c[1][1][0];
    c[0][1][1] = c[1][1][1];
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
