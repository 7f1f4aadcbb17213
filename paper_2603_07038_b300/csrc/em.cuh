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
  // CPML auxiliaries for derivative axis d, slot s (field component (d+1+s)%3).
  // Always FP64: inside a layer psi tends to -dF for slowly varying fields, so
  // dF + psi cancels and an FP32 psi would lose the residue.
  const double *pEo[3][2];
  double *pEn[3][2];
  const double *pHo[3][2];
  double *pHn[3][2];
  int slo[3], shi[3], sn[3];  // CPML cells at the low / high end, slab extent
  const double *cpml;         // [axis][E,H][b,c][kMaxSlab]
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

// psi <- b psi + c dF in FP64, returns dF + psi_new (written only by the owner)
template <typename R>
__device__ __forceinline__ double psi_update(const EmArgs<R> &A, const double *s_cp, int d, int type, int slot,
                                             int s, int i, int j, int k, R deriv, bool write) {
  const long long q = psi_index(A, d, s, i, j, k);
  const double b = s_cp[((d * 2 + type) * 2 + 0) * kMaxSlab + s];
  const double c = s_cp[((d * 2 + type) * 2 + 1) * kMaxSlab + s];
  const double *po = type == 0 ? A.pEo[d][slot] : A.pHo[d][slot];
  const double v = b * po[q] + c * (double)deriv;
  if (write) (type == 0 ? A.pEn[d][slot] : A.pHn[d][slot])[q] = v;
  return (double)deriv + v;
}

// (dF1 + psi1) - (dF2 + psi2) for the two derivatives of one curl component;
// FP64 only where a CPML slab is present (s1/s2 >= 0).
template <typename R>
__device__ __forceinline__ R curl_with_psi(const EmArgs<R> &A, const double *s_cp, int type, int comp, int d1,
                                           int s1, int d2, int s2, int i, int j, int k, R v1, R v2, bool write) {
  (void)comp;
  if (s1 < 0 && s2 < 0) return v1 - v2;
  const double a = s1 >= 0 ? psi_update(A, s_cp, d1, type, 1, s1, i, j, k, v1, write) : (double)v1;
  const double b = s2 >= 0 ? psi_update(A, s_cp, d2, type, 0, s2, i, j, k, v2, write) : (double)v2;
  return (R)(a - b);
}

// E^{n+1} of one edge from the four voxels (m0..m3 with area weights w0..w3,
// quarter factor folded in), W = dual-face area, l = edge length:
//   E' = ca E + cb (curl - J),  ca = (Se - Ss)/(Se + Ss),  cb = dt W/(Se + Ss)
// (Se = sum w eps, Ss = sum w sigma dt/2), evaluated in the equivalent
// incremental form E' = E + r (dt W (curl - J) - 2 Ss E), r = 1/(Se + Ss),
// which keeps the decay 1 - ca of weakly lossy media at full precision.
// Returns E^{n+1}; *half_q receives the edge's Joule energy share per end node.
template <typename R>
__device__ __forceinline__ R edge_update(const R *s_mt, int m0, R w0, int m1, R w1, int m2, R w2, int m3, R w3,
                                         R W, R l, R dt, R e_old, R curl, R J, R *half_q) {
  const R Se = w0 * mconst(s_mt, m0, M_EPS) + w1 * mconst(s_mt, m1, M_EPS) + w2 * mconst(s_mt, m2, M_EPS) +
               w3 * mconst(s_mt, m3, M_EPS);
  const R Ss = w0 * mconst(s_mt, m0, M_SDT2) + w1 * mconst(s_mt, m1, M_SDT2) + w2 * mconst(s_mt, m2, M_SDT2) +
               w3 * mconst(s_mt, m3, M_SDT2);
  const R r = R(1) / (Se + Ss);
  const R e_new = e_old + r * (dt * W * (curl - J) - R(2) * Ss * e_old);
  const R eb = R(0.5) * (e_old + e_new);
  *half_q = Ss * l * eb * eb;
  return e_new;
}

// One plane of the CTA's inputs, staged in shared memory: E^n of the tile plus
// its +x/+y neighbours, H^{n-1/2} and the Joule accumulator of the owned nodes.
template <typename R, int TX, int TY>
struct EmStage {
  R E[3][TY + 1][TX + 1];
  R H[3][TY][TX];
  double Q[TY][TX];
};

template <typename R, int TX, int TY>
__host__ __device__ constexpr size_t em_stage_offset(int nmat) {
  return (12 * kMaxSlab * sizeof(double) + (size_t)nmat * M_COLS * sizeof(R) + 15) & ~size_t(15);
}

constexpr int kEmStages = 3;  // planes k (in use), k+1 (ready), k+2 (in flight)

template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) em_step_kernel(const EmArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *s_cp = reinterpret_cast<double *>(smem_raw);
  R *s_mt = reinterpret_cast<R *>(s_cp + 12 * kMaxSlab);
  const Geo<R> &g = A.g;
  EmStage<R, TX, TY> *stg = reinterpret_cast<EmStage<R, TX, TY> *>(smem_raw + em_stage_offset<R, TX, TY>(g.nmat));
  __shared__ R sH[3][TY][TX];
  __shared__ R sP[2][TY][TX];
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  stage_table(s_cp, A.cpml, 12 * kMaxSlab);

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = blockIdx.x * (TX - 1) - 1, j0 = blockIdx.y * (TY - 1) - 1;  // node of thread (0, 0)
  const int i = i0 + tx, j = j0 + ty;
  const bool act = (i >= 0 && i <= nx && j >= 0 && j <= ny);
  const bool own = act && tx > 0 && ty > 0;
  const bool need_ex = act && ty > 0 && i < nx;  // own, or the halo column
  const bool need_ey = act && tx > 0 && j < ny;  // own, or the halo row
  const bool need_ez = own;

  // Plane k of E^n (tile + neighbours), H^{n-1/2} and Q (owned nodes) -> stage s.
  // Positions outside the grid are zero-filled without a read.
  auto load_stage = [&](int k, int s) {
    EmStage<R, TX, TY> &S = stg[s];
    const bool kin = k <= nz;
    constexpr int NE = (TY + 1) * (TX + 1);
    for (int q = tid; q < 3 * NE; q += TX * TY) {
      const int c = q / NE, r = q - c * NE;
      const int yy = r / (TX + 1), xx = r - yy * (TX + 1);
      const int ii = i0 + xx, jj = j0 + yy;
      const bool ok = kin && ii >= 0 && ii <= nx && jj >= 0 && jj <= ny;
      cp_async<sizeof(R)>(&S.E[c][yy][xx], ok ? A.Eo[c] + g.nid(ii, jj, k) : A.Eo[c], ok);
    }
    const bool okh = kin && act;
    const long long idk = okh ? g.nid(i, j, k) : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) cp_async<sizeof(R)>(&S.H[c][ty][tx], A.Ho[c] + idk, okh);
    if (A.Q != nullptr) cp_async<8>(&S.Q[ty][tx], A.Q + (kin && own ? idk : 0), kin && own);
    cp_async_commit();
  };

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
  const long long plane = g.plane;
  const long long id0 = act ? g.nid(i, j, 0) : 0;

  load_stage(0, 0);
  load_stage(1, 1);
  // voxels (i-1+dx, j-1+dy) of the layer below (b..) and above (a..) the node plane
  int b00 = -1, b01 = -1, b10 = -1, b11 = -1;
  int a00 = g.cell(i - 1, j - 1, 0), a01 = g.cell(i, j - 1, 0), a10 = g.cell(i - 1, j, 0), a11 = g.cell(i, j, 0);
  int r0 = 0, r1 = 0;  // source entries of row (k, j)
  if (A.src_row != nullptr && act) {
    r0 = __ldg(A.src_row + j);
    r1 = __ldg(A.src_row + j + 1);
  }
  R hx_km1 = 0, hy_km1 = 0, qz_km1 = 0;

  for (int k = 0; k <= nz; ++k) {
    load_stage(k + 2, (k + 2) % kEmStages);
    // next layer's voxels and source row, consumed in the next iteration
    const int n00 = g.cell(i - 1, j - 1, k + 1), n01 = g.cell(i, j - 1, k + 1);
    const int n10 = g.cell(i - 1, j, k + 1), n11 = g.cell(i, j, k + 1);
    int nr0 = 0, nr1 = 0;
    if (A.src_row != nullptr && act && k < nz) {
      const int row = (k + 1) * (ny + 1) + j;
      nr0 = __ldg(A.src_row + row);
      nr1 = __ldg(A.src_row + row + 1);
    }
    cp_async_wait<1>();  // planes k and k+1 have landed
    __syncthreads();
    const EmStage<R, TX, TY> &S0 = stg[k % kEmStages];
    const EmStage<R, TX, TY> &S1 = stg[(k + 1) % kEmStages];
    const long long id = id0 + (long long)k * plane;
    const R hzm = (k > 0) ? g.h[2][k - 1] : R(0), hz0 = (k < nz) ? g.h[2][k] : R(0);
    const R ihz = (k < nz) ? g.ih[2][k] : R(0), idz = g.idual[2][k];
    const bool fix_z = (k == 0 && A.fixlo[2]) || (k == nz && A.fixhi[2]);
    const int szE = slab_index(k, nz, A.slo[2], A.shi[2]);
    const int szH = (k < nz) ? szE : -1;

    const R ex = S0.E[0][ty][tx], ey = S0.E[1][ty][tx], ez = S0.E[2][ty][tx];
    const R ex_up = S1.E[0][ty][tx], ey_up = S1.E[1][ty][tx];
    const R ez_jp = S0.E[2][ty + 1][tx], ex_jp = S0.E[0][ty + 1][tx];
    const R ez_ip = S0.E[2][ty][tx + 1], ey_ip = S0.E[1][ty][tx + 1];
    const double q_old = (A.Q != nullptr) ? S0.Q[ty][tx] : 0.0;

    // ---- H^{n+1/2} at (i,j,k): H -= dt/mu (curl E + psi terms)
    R Hx = 0, Hy = 0, Hz = 0;
    if (act) {
      if (j < ny && k < nz) {  // Hx: (curl E)_x = dEz/dy - dEy/dz
        const R d1 = (ez_jp - ez) * ihy, d2 = (ey_up - ey) * ihz;
        const R curl = curl_with_psi(A, s_cp, 1, 0, 1, syH, 2, szH, i, j, k, d1, d2, own);
        const R coef = half_dt * idx * (hxm * mconst(s_mt, a10, M_IMU) + hx0 * mconst(s_mt, a11, M_IMU));
        Hx = S0.H[0][ty][tx] - coef * curl;
      }
      if (i < nx && k < nz) {  // Hy: dEx/dz - dEz/dx
        const R d1 = (ex_up - ex) * ihz, d2 = (ez_ip - ez) * ihx;
        const R curl = curl_with_psi(A, s_cp, 1, 1, 2, szH, 0, sxH, i, j, k, d1, d2, own);
        const R coef = half_dt * idy * (hym * mconst(s_mt, a01, M_IMU) + hy0 * mconst(s_mt, a11, M_IMU));
        Hy = S0.H[1][ty][tx] - coef * curl;
      }
      if (i < nx && j < ny) {  // Hz: dEy/dx - dEx/dy
        const R d1 = (ey_ip - ey) * ihx, d2 = (ex_jp - ex) * ihy;
        const R curl = curl_with_psi(A, s_cp, 1, 2, 0, sxH, 1, syH, i, j, k, d1, d2, own);
        const R coef = half_dt * idz * (hzm * mconst(s_mt, b11, M_IMU) + hz0 * mconst(s_mt, a11, M_IMU));
        Hz = S0.H[2][ty][tx] - coef * curl;
      }
    }
    sH[0][ty][tx] = Hx;
    sH[1][ty][tx] = Hy;
    sH[2][ty][tx] = Hz;
    __syncthreads();

    // ---- source current on this node's edges
    R J[3] = {0, 0, 0};
    for (int e = r0; e < r1; ++e) {
      const int4 s = A.src_ent[e];
      if (s.x == i && A.step < A.amp_len) J[s.y] += A.src_amp[(long long)s.z * A.amp_len + A.step];
    }

    // ---- E^{n+1} on the node's edges and their Joule shares
    R exn = ex, eyn = ey, ezn = ez, qx = 0, qy = 0, qz = 0;
    if (need_ex && !(fix_y || fix_z)) {  // Ex: dHz/dy - dHy/dz, voxels (i, j-1..j, k-1..k)
      const R d1 = (sH[2][ty][tx] - sH[2][ty - 1][tx]) * idy;
      const R d2 = (sH[1][ty][tx] - hy_km1) * idz;
      const R curl = curl_with_psi(A, s_cp, 0, 0, 1, syE, 2, szE, i, j, k, d1, d2, own);
      const R q = R(0.25);
      exn = edge_update(s_mt, b01, q * hym * hzm, b11, q * hy0 * hzm, a01, q * hym * hz0, a11, q * hy0 * hz0,
                        q * (hym + hy0) * (hzm + hz0), hx0, dt, ex, curl, J[0], &qx);
    }
    if (need_ey && !(fix_x || fix_z)) {  // Ey: dHx/dz - dHz/dx, voxels (i-1..i, j, k-1..k)
      const R d1 = (sH[0][ty][tx] - hx_km1) * idz;
      const R d2 = (sH[2][ty][tx] - sH[2][ty][tx - 1]) * idx;
      const R curl = curl_with_psi(A, s_cp, 0, 1, 2, szE, 0, sxE, i, j, k, d1, d2, own);
      const R q = R(0.25);
      eyn = edge_update(s_mt, b10, q * hxm * hzm, b11, q * hx0 * hzm, a10, q * hxm * hz0, a11, q * hx0 * hz0,
                        q * (hxm + hx0) * (hzm + hz0), hy0, dt, ey, curl, J[1], &qy);
    }
    if (need_ez && k < nz && !(fix_x || fix_y)) {  // Ez: dHy/dx - dHx/dy, voxels (i-1..i, j-1..j, k)
      const R d1 = (sH[1][ty][tx] - sH[1][ty][tx - 1]) * idx;
      const R d2 = (sH[0][ty][tx] - sH[0][ty - 1][tx]) * idy;
      const R curl = curl_with_psi(A, s_cp, 0, 2, 0, sxE, 1, syE, i, j, k, d1, d2, own);
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
        A.Q[id] = q_old + (double)s;
      }
    }
    hx_km1 = Hx;
    hy_km1 = Hy;
    qz_km1 = qz;
    b00 = a00;
    b01 = a01;
    b10 = a10;
    b11 = a11;
    a00 = n00;
    a01 = n01;
    a10 = n10;
    a11 = n11;
    r0 = nr0;
    r1 = nr1;
  }
  cp_async_wait<0>();
}

}  // namespace cosim
