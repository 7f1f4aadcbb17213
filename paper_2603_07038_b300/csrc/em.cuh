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
// shared memory, z from its own previous plane) and adds them to its FP64
// accumulator.
//
// Material averaging (per edge: area-weighted eps, sigma over the <=4 voxels;
// per face: series mean of mu over the 2 voxels) is recomputed from the 1-byte
// voxel IDs every step instead of streaming per-edge coefficient arrays.
#pragma once
#include "common.cuh"

namespace cosim {

template <typename R>
struct EmArgs {
  Geo<R> g;
  const R *Eo[3];
  R *En[3];
  const R *Ho[3];
  R *Hn[3];
  // CPML auxiliaries for derivative axis d, slot s (field component (d+1+s)%3)
  const R *pEo[3][2];
  R *pEn[3][2];
  const R *pHo[3][2];
  R *pHn[3][2];
  int slo[3], shi[3], sn[3];  // CPML cells at the low / high end, slab extent
  const R *cpml;              // [axis][E,H][b,c][kMaxSlab]
  int fixlo[3], fixhi[3];     // wall holds tangential E at zero (PEC or CPML backing)
  R dt;
  const int *src_row;         // per (k,j) row: first source entry, (nz+1)(ny+1)+1 ints
  const int4 *src_ent;        // (i, axis, source index, 0)
  const R *src_amp;           // [source][amp_len]
  long long amp_len;
  long long step;
  double *Q;                  // Joule energy per node (null: not accumulating)
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

// psi <- b psi + c dF, returns the new psi (written only by the owner)
template <typename R>
__device__ __forceinline__ R psi_update(const EmArgs<R> &A, const R *s_cp, int d, int type, int slot, int s,
                                        int i, int j, int k, R deriv, bool write) {
  const long long q = psi_index(A, d, s, i, j, k);
  const R b = s_cp[((d * 2 + type) * 2 + 0) * kMaxSlab + s];
  const R c = s_cp[((d * 2 + type) * 2 + 1) * kMaxSlab + s];
  const R *po = type == 0 ? A.pEo[d][slot] : A.pHo[d][slot];
  const R v = b * po[q] + c * deriv;
  if (write) (type == 0 ? A.pEn[d][slot] : A.pHn[d][slot])[q] = v;
  return v;
}

// E^{n+1} of one edge: ca, cb from the four voxels (m0..m3 with area weights
// w0..w3, quarter factor folded in), W = dual-face area, l = edge length.
// Returns E^{n+1}; *half_q receives the edge's Joule energy share per end node.
template <typename R>
__device__ __forceinline__ R edge_update(const R *s_mt, int m0, R w0, int m1, R w1, int m2, R w2, int m3, R w3,
                                         R W, R l, R dt, R e_old, R curl, R J, R *half_q) {
  const R Se = w0 * mconst(s_mt, m0, M_EPS) + w1 * mconst(s_mt, m1, M_EPS) + w2 * mconst(s_mt, m2, M_EPS) +
               w3 * mconst(s_mt, m3, M_EPS);
  const R Ss = w0 * mconst(s_mt, m0, M_SDT2) + w1 * mconst(s_mt, m1, M_SDT2) + w2 * mconst(s_mt, m2, M_SDT2) +
               w3 * mconst(s_mt, m3, M_SDT2);
  const R r = R(1) / (Se + Ss);
  const R ca = (Se - Ss) * r;
  const R cb = dt * W * r;
  const R e_new = ca * e_old + cb * (curl - J);
  const R eb = R(0.5) * (e_old + e_new);
  *half_q = Ss * l * eb * eb;
  return e_new;
}

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) em_step_kernel(const EmArgs<R> A) {
  extern __shared__ unsigned char smem_raw[];
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  R *s_cp = s_mt + A.g.nmat * M_COLS;
  __shared__ R sH[3][TY][TX];
  __shared__ R sP[2][TY][TX];
  const Geo<R> &g = A.g;
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  stage_table(s_cp, A.cpml, 12 * kMaxSlab);
  __syncthreads();

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i = blockIdx.x * (TX - 1) - 1 + tx;
  const int j = blockIdx.y * (TY - 1) - 1 + ty;
  const bool act = (i >= 0 && i <= nx && j >= 0 && j <= ny);
  const bool own = act && tx > 0 && ty > 0;
  const bool need_ex = act && ty > 0 && i < nx;  // own, or the halo column
  const bool need_ey = act && tx > 0 && j < ny;  // own, or the halo row
  const bool need_ez = own;

  const R hxm = (act && i > 0) ? g.h[0][i - 1] : R(0), hx0 = (act && i < nx) ? g.h[0][i] : R(0);
  const R hym = (act && j > 0) ? g.h[1][j - 1] : R(0), hy0 = (act && j < ny) ? g.h[1][j] : R(0);
  const R ihx = (act && i < nx) ? g.ih[0][i] : R(0), ihy = (act && j < ny) ? g.ih[1][j] : R(0);
  const R idx = act ? g.idual[0][i] : R(0), idy = act ? g.idual[1][j] : R(0);
  const bool fix_x = (i == 0 && A.fixlo[0]) || (i == nx && A.fixhi[0]);
  const bool fix_y = (j == 0 && A.fixlo[1]) || (j == ny && A.fixhi[1]);
  // CPML slab positions along x and y (E: nodes, H: cells)
  const int sxE = slab_index(i, nx, A.slo[0], A.shi[0]);
  const int syE = slab_index(j, ny, A.slo[1], A.shi[1]);
  const int sxH = (i < nx) ? sxE : -1;
  const int syH = (j < ny) ? syE : -1;
  const R dt = A.dt;
  const R half_dt = R(0.5) * dt;
  const long long px = g.px, plane = g.plane;
  const long long id0 = act ? g.nid(i, j, 0) : 0;

  // voxels of the layer below the current node plane: (i-1+dx, j-1+dy, k-1)
  int b00 = -1, b01 = -1, b10 = -1, b11 = -1;  // index order (dy, dx)
  R ex = act ? A.Eo[0][id0] : R(0);
  R ey = act ? A.Eo[1][id0] : R(0);
  R hx_km1 = 0, hy_km1 = 0, qz_km1 = 0;

  for (int k = 0; k <= nz; ++k) {
    const long long id = id0 + (long long)k * plane;
    const int a00 = g.cell(i - 1, j - 1, k), a01 = g.cell(i, j - 1, k);
    const int a10 = g.cell(i - 1, j, k), a11 = g.cell(i, j, k);
    const R hzm = (k > 0) ? g.h[2][k - 1] : R(0), hz0 = (k < nz) ? g.h[2][k] : R(0);
    const R ihz = (k < nz) ? g.ih[2][k] : R(0), idz = g.idual[2][k];
    const bool fix_z = (k == 0 && A.fixlo[2]) || (k == nz && A.fixhi[2]);
    const int szE = slab_index(k, nz, A.slo[2], A.shi[2]);
    const int szH = (k < nz) ? szE : -1;

    // ---- E^n needed at this plane
    R ez = 0, ex_up = 0, ey_up = 0, ez_jp = 0, ex_jp = 0, ez_ip = 0, ey_ip = 0;
    if (act) {
      if (k < nz) {
        ez = A.Eo[2][id];
        ex_up = A.Eo[0][id + plane];
        ey_up = A.Eo[1][id + plane];
      }
      if (j < ny) {
        ex_jp = A.Eo[0][id + px];
        if (k < nz) ez_jp = A.Eo[2][id + px];
      }
      if (i < nx) {
        ey_ip = A.Eo[1][id + 1];
        if (k < nz) ez_ip = A.Eo[2][id + 1];
      }
    }

    // ---- H^{n+1/2} at (i,j,k): H -= dt/mu (curl E + psi terms)
    R Hx = 0, Hy = 0, Hz = 0;
    if (act) {
      if (j < ny && k < nz) {  // Hx: (curl E)_x = dEz/dy - dEy/dz
        const R d1 = (ez_jp - ez) * ihy, d2 = (ey_up - ey) * ihz;
        R curl = d1 - d2;
        if (syH >= 0) curl += psi_update(A, s_cp, 1, 1, 1, syH, i, j, k, d1, own);
        if (szH >= 0) curl -= psi_update(A, s_cp, 2, 1, 0, szH, i, j, k, d2, own);
        const R coef = half_dt * idx * (hxm * mconst(s_mt, a10, M_IMU) + hx0 * mconst(s_mt, a11, M_IMU));
        Hx = A.Ho[0][id] - coef * curl;
      }
      if (i < nx && k < nz) {  // Hy: dEx/dz - dEz/dx
        const R d1 = (ex_up - ex) * ihz, d2 = (ez_ip - ez) * ihx;
        R curl = d1 - d2;
        if (szH >= 0) curl += psi_update(A, s_cp, 2, 1, 1, szH, i, j, k, d1, own);
        if (sxH >= 0) curl -= psi_update(A, s_cp, 0, 1, 0, sxH, i, j, k, d2, own);
        const R coef = half_dt * idy * (hym * mconst(s_mt, a01, M_IMU) + hy0 * mconst(s_mt, a11, M_IMU));
        Hy = A.Ho[1][id] - coef * curl;
      }
      if (i < nx && j < ny) {  // Hz: dEy/dx - dEx/dy
        const R d1 = (ey_ip - ey) * ihx, d2 = (ex_jp - ex) * ihy;
        R curl = d1 - d2;
        if (sxH >= 0) curl += psi_update(A, s_cp, 0, 1, 1, sxH, i, j, k, d1, own);
        if (syH >= 0) curl -= psi_update(A, s_cp, 1, 1, 0, syH, i, j, k, d2, own);
        const R coef = half_dt * idz * (hzm * mconst(s_mt, b11, M_IMU) + hz0 * mconst(s_mt, a11, M_IMU));
        Hz = A.Ho[2][id] - coef * curl;
      }
    }
    sH[0][ty][tx] = Hx;
    sH[1][ty][tx] = Hy;
    sH[2][ty][tx] = Hz;
    __syncthreads();

    // ---- source current on this node's edges
    R J[3] = {0, 0, 0};
    if (A.src_row != nullptr && act) {
      const int row = k * (ny + 1) + j;
      const int r0 = __ldg(A.src_row + row), r1 = __ldg(A.src_row + row + 1);
      for (int e = r0; e < r1; ++e) {
        const int4 s = A.src_ent[e];
        if (s.x == i && A.step < A.amp_len) J[s.y] += A.src_amp[(long long)s.z * A.amp_len + A.step];
      }
    }

    // ---- E^{n+1} on the node's edges and their Joule shares
    R exn = ex, eyn = ey, ezn = ez, qx = 0, qy = 0, qz = 0;
    if (need_ex && !(fix_y || fix_z)) {  // Ex: dHz/dy - dHy/dz, voxels (i, j-1..j, k-1..k)
      const R d1 = (sH[2][ty][tx] - sH[2][ty - 1][tx]) * idy;
      const R d2 = (sH[1][ty][tx] - hy_km1) * idz;
      R curl = d1 - d2;
      if (syE >= 0) curl += psi_update(A, s_cp, 1, 0, 1, syE, i, j, k, d1, own);
      if (szE >= 0) curl -= psi_update(A, s_cp, 2, 0, 0, szE, i, j, k, d2, own);
      const R q = R(0.25);
      exn = edge_update(s_mt, b01, q * hym * hzm, b11, q * hy0 * hzm, a01, q * hym * hz0, a11, q * hy0 * hz0,
                        q * (hym + hy0) * (hzm + hz0), hx0, dt, ex, curl, J[0], &qx);
    }
    if (need_ey && !(fix_x || fix_z)) {  // Ey: dHx/dz - dHz/dx, voxels (i-1..i, j, k-1..k)
      const R d1 = (sH[0][ty][tx] - hx_km1) * idz;
      const R d2 = (sH[2][ty][tx] - sH[2][ty][tx - 1]) * idx;
      R curl = d1 - d2;
      if (szE >= 0) curl += psi_update(A, s_cp, 2, 0, 1, szE, i, j, k, d1, own);
      if (sxE >= 0) curl -= psi_update(A, s_cp, 0, 0, 0, sxE, i, j, k, d2, own);
      const R q = R(0.25);
      eyn = edge_update(s_mt, b10, q * hxm * hzm, b11, q * hx0 * hzm, a10, q * hxm * hz0, a11, q * hx0 * hz0,
                        q * (hxm + hx0) * (hzm + hz0), hy0, dt, ey, curl, J[1], &qy);
    }
    if (need_ez && k < nz && !(fix_x || fix_y)) {  // Ez: dHy/dx - dHx/dy, voxels (i-1..i, j-1..j, k)
      const R d1 = (sH[1][ty][tx] - sH[1][ty][tx - 1]) * idx;
      const R d2 = (sH[0][ty][tx] - sH[0][ty - 1][tx]) * idy;
      R curl = d1 - d2;
      if (sxE >= 0) curl += psi_update(A, s_cp, 0, 0, 1, sxE, i, j, k, d1, own);
      if (syE >= 0) curl -= psi_update(A, s_cp, 1, 0, 0, syE, i, j, k, d2, own);
      const R q = R(0.25);
      ezn = edge_update(s_mt, a00, q * hxm * hym, a01, q * hx0 * hym, a10, q * hxm * hy0, a11, q * hx0 * hy0,
                        q * (hxm + hx0) * (hym + hy0), hz0, dt, ez, curl, J[2], &qz);
    }
    sP[0][ty][tx] = qx;
    sP[1][ty][tx] = qy;
    __syncthreads();

    if (own) {
      A.Hn[0][id] = Hx;
      A.Hn[1][id] = Hy;
      A.Hn[2][id] = Hz;
      A.En[0][id] = exn;
      A.En[1][id] = eyn;
      if (k < nz) A.En[2][id] = ezn;
      if (A.Q != nullptr) {
        const R s = (qx + sP[0][ty][tx - 1]) + (qy + sP[1][ty - 1][tx]) + (qz + qz_km1);
        A.Q[id] += (double)s;
      }
    }
    hx_km1 = Hx;
    hy_km1 = Hy;
    qz_km1 = qz;
    ex = ex_up;
    ey = ey_up;
    b00 = a00;
    b01 = a01;
    b10 = a10;
    b11 = a11;
  }
}

}  // namespace cosim
