// Linear thermoelasticity on the voxel grid (Sec. II-B, Eqs. 7-9).
//
// Elements are the voxels (bricks hx*hy*hz), nodes carry (ux, uy, uz).
// K_e = int B^T E_c B dV with 2x2x2 Gauss points, which integrates a brick's
// stiffness exactly. The kernels evaluate K_e u_e without forming K_e, in
// the basis of the eight trilinear monomials {1, xi, eta, zeta, xi eta,
// eta zeta, zeta xi, xi eta zeta}: a 2x2x2 butterfly (Walsh-Hadamard) maps the
// nodal values to monomial coefficients, the displacement gradient of each
// monomial group is a 3x3 matrix with a few nonzeros, the monomials are
// orthogonal on the reference cube (mean 1, 1/3, 1/9 of their squares), so
// the element energy is a weighted sum of isotropic energies
// W(G) = lambda tr(G)^2 + mu G:(G + G^T) over the groups, and its gradient
// maps back through the transposed butterfly. About 300 flops per element.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "common.cuh"

namespace cosim {

// The element arithmetic is written once for one element (V = R) or two
// x-adjacent elements (V = the pair type), with the element-wise helpers of
// common.cuh: every operation rounds once and the pair forms act element by
// element (the packed path may contract a product into the following
// addition, one FP32 rounding apart from the one-element path).

// q[m] = sum_a P_m(s_a) v[a]; a = ax + 2 ay + 4 az, m bit d set <=> factor s_d
template <typename V>
__device__ __forceinline__ void modal_fwd(V v[8]) {
#pragma unroll
  for (int b = 1; b < 8; b <<= 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!(a & b)) {
        const V lo = v[a], hi = v[a | b];
        v[a] = add_(hi, lo);
        v[a | b] = sub_(hi, lo);
      }
}

// r[a] = sum_m P_m(s_a) F[m] (transpose of modal_fwd)
template <typename V>
__device__ __forceinline__ void modal_bwd(V v[8]) {
#pragma unroll
  for (int b = 1; b < 8; b <<= 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!(a & b)) {
        const V s = v[a], d = v[a | b];
        v[a] = sub_(s, d);
        v[a | b] = add_(s, d);
      }
}

// One monomial group: the nonzero gradient columns of the group (G[c][d],
// d with slot[d] >= 0; the others are zero), slot[d] = monomial receiving
// column d of the energy gradient (-1: none), wg[d] = w g_d s with the
// group's weight w = <phi^2> and the element's volume factor s.
// S_cd = delta_cd lambda tr(G) + mu (G_cd + G_dc); F[c][slot d] += S_cd wg_d.
template <typename V, typename R>
__device__ __forceinline__ void group_term(const V G[3][3], V lam, V mu, const V wg[3], const int slot[3],
                                           V F[3][8]) {
  V tr = bc_<V>(R(0));
  bool first = true;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    if (slot[d] >= 0) {
      tr = first ? G[d][d] : add_(tr, G[d][d]);
      first = false;
    }
  const V lt = mul_(lam, tr);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (slot[d] >= 0) {
        const V sym = slot[c] >= 0 ? add_(G[c][d], G[d][c]) : G[c][d];
        const V S = c == d ? fma_(mu, sym, lt) : mul_(mu, sym);
        F[c][slot[d]] = fma_(S, wg[d], F[c][slot[d]]);
      }
}

// u[c][a] (nodal displacement of one element, or of an element pair) ->
// K_e u_e in place; ih* are the inverse sizes (2 ih = 2/h exactly: scaling by
// two is exact).
template <typename V, typename R>
__device__ __forceinline__ void hex8_apply(V u[3][8], V lam, V mu, V hx, V hy, V hz, V ihx, V ihy, V ihz) {
  const V g[3] = {mul_(bc_<V>(R(2)), ihx), mul_(bc_<V>(R(2)), ihy), mul_(bc_<V>(R(2)), ihz)};
  const V g8[3] = {mul_(g[0], bc_<V>(R(0.125))), mul_(g[1], bc_<V>(R(0.125))), mul_(g[2], bc_<V>(R(0.125)))};
#pragma unroll
  for (int c = 0; c < 3; ++c) modal_fwd(u[c]);
  V F[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int m = 0; m < 8; ++m) F[c][m] = bc_<V>(R(0));
  const R third = R(1) / R(3), ninth = R(1) / R(9);
  // the volume factor s = hx hy hz / 8 and the group weights folded into the
  // gradient factors once: w1 (w = 1), w3 (1/3), w9 (1/9)
  const V s = mul_(mul_(mul_(bc_<V>(R(0.125)), hx), hy), hz);
  const V w1[3] = {mul_(g[0], s), mul_(g[1], s), mul_(g[2], s)};
  const V w3[3] = {mul_(w1[0], bc_<V>(third)), mul_(w1[1], bc_<V>(third)), mul_(w1[2], bc_<V>(third))};
  const V w9[3] = {mul_(w1[0], bc_<V>(ninth)), mul_(w1[1], bc_<V>(ninth)), mul_(w1[2], bc_<V>(ninth))};
  V G[3][3];
  {  // constant gradient: columns from the linear monomials xi, eta, zeta
    const int slot[3] = {1, 2, 4};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      G[c][0] = mul_(g8[0], u[c][1]);
      G[c][1] = mul_(g8[1], u[c][2]);
      G[c][2] = mul_(g8[2], u[c][4]);
    }
    group_term<V, R>(G, lam, mu, w1, slot, F);
  }
  {  // terms linear in xi: d/deta of (xi eta), d/dzeta of (zeta xi)
    const int slot[3] = {-1, 3, 5};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      G[c][1] = mul_(g8[1], u[c][3]);
      G[c][2] = mul_(g8[2], u[c][5]);
    }
    group_term<V, R>(G, lam, mu, w3, slot, F);
  }
  {  // linear in eta: d/dxi of (xi eta), d/dzeta of (eta zeta)
    const int slot[3] = {3, -1, 6};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      G[c][0] = mul_(g8[0], u[c][3]);
      G[c][2] = mul_(g8[2], u[c][6]);
    }
    group_term<V, R>(G, lam, mu, w3, slot, F);
  }
  {  // linear in zeta: d/dxi of (zeta xi), d/deta of (eta zeta)
    const int slot[3] = {5, 6, -1};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      G[c][0] = mul_(g8[0], u[c][5]);
      G[c][1] = mul_(g8[1], u[c][6]);
    }
    group_term<V, R>(G, lam, mu, w3, slot, F);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {  // bilinear monomials from (xi eta zeta)
    int slot[3] = {-1, -1, -1};
    slot[d] = 7;
#pragma unroll
    for (int c = 0; c < 3; ++c) G[c][d] = mul_(g8[d], u[c][7]);
    group_term<V, R>(G, lam, mu, w9, slot, F);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    modal_bwd(F[c]);
#pragma unroll
    for (int a = 0; a < 8; ++a) u[c][a] = F[c][a];
  }
}

template <typename R>
struct MvArgs {
  Geo<R> g;
  const R *u[3];
  R *y[3];
  const uint8_t *mask;  // per node: bit c set = component c constrained
  double *partial;      // per-CTA sum of u.y (null: not needed)
};

// y = K u with constrained DOFs eliminated (their columns are dropped by
// zeroing u there, their rows give y_c = u_c). CTAs own (TX-1) x (TY-1) node
// columns and march through the element layers; each thread computes one
// element of the tile plus a one-element halo at -x/-y, writes its 24 nodal
// forces to shared memory, and the owner of each node sums its four in-plane
// elements; the forces of the layer's top face are carried to the next
// layer in registers. No atomics: deterministic.
template <typename R, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) hex8_matvec_kernel(const MvArgs<R> A) {
  extern __shared__ unsigned char smem_raw[];
  const Geo<R> &g = A.g;
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  R *su = s_mt + g.nmat * M_COLS;          // [2 planes][3][TY+1][TX+1]
  R *sr = su + 2 * 3 * (TY + 1) * (TX + 1); // [24][TY][TX]
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int X0 = blockIdx.x * (TX - 1) - 1, Y0 = blockIdx.y * (TY - 1) - 1;
  const int ex = X0 + tx, ey = Y0 + ty;
  const bool elem_xy = ex >= 0 && ex < nx && ey >= 0 && ey < ny;
  const int X = ex + 1, Y = ey + 1;
  const bool own = tx < TX - 1 && ty < TY - 1 && X <= nx && Y <= ny;
  const R hx = elem_xy ? g.h[0][ex] : R(1), hy = elem_xy ? g.h[1][ey] : R(1);
  const R ihx = elem_xy ? g.ih[0][ex] : R(1), ihy = elem_xy ? g.ih[1][ey] : R(1);

  auto su_at = [&](int buf, int c, int qy, int qx) -> R & {
    return su[((buf * 3 + c) * (TY + 1) + qy) * (TX + 1) + qx];
  };
  auto stage = [&](int kp, int buf) {
    for (int q = tid; q < (TX + 1) * (TY + 1); q += TX * TY) {
      const int qx = q % (TX + 1), qy = q / (TX + 1);
      const int Xn = X0 + qx, Yn = Y0 + qy;
      R v0 = 0, v1 = 0, v2 = 0;
      if (Xn >= 0 && Xn <= nx && Yn >= 0 && Yn <= ny) {
        const long long id = g.nid(Xn, Yn, kp);
        const uint8_t mk = A.mask[id];
        v0 = (mk & 1) ? R(0) : A.u[0][id];
        v1 = (mk & 2) ? R(0) : A.u[1][id];
        v2 = (mk & 4) ? R(0) : A.u[2][id];
      }
      su_at(buf, 0, qy, qx) = v0;
      su_at(buf, 1, qy, qx) = v1;
      su_at(buf, 2, qy, qx) = v2;
    }
  };
  auto sr_at = [&](int slot, int qy, int qx) -> R & { return sr[(slot * TY + qy) * TX + qx]; };

  stage(0, 0);
  R acc[3] = {0, 0, 0};
  double dot = 0.0;
  for (int k = 0; k < nz; ++k) {
    stage(k + 1, (k + 1) & 1);
    __syncthreads();
    R r[3][8];
    if (elem_xy) {
      const int m = g.cell(ex, ey, k);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 8; ++a)
          r[c][a] = su_at((k + (a >> 2)) & 1, c, ty + ((a >> 1) & 1), tx + (a & 1));
      hex8_apply<R, R>(r, s_mt[m * M_COLS + M_LAM], s_mt[m * M_COLS + M_MU], hx, hy, g.h[2][k], ihx, ihy, g.ih[2][k]);
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 8; ++a) r[c][a] = 0;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int a = 0; a < 8; ++a) sr_at(c * 8 + a, ty, tx) = r[c][a];
    __syncthreads();
    if (own) {
      const long long id = g.nid(X, Y, k);
      const uint8_t mk = A.mask[id];
      R part = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R bottom = (sr_at(c * 8 + 3, ty, tx) + sr_at(c * 8 + 2, ty, tx + 1)) +
                         (sr_at(c * 8 + 1, ty + 1, tx) + sr_at(c * 8 + 0, ty + 1, tx + 1));
        const R top = (sr_at(c * 8 + 7, ty, tx) + sr_at(c * 8 + 6, ty, tx + 1)) +
                      (sr_at(c * 8 + 5, ty + 1, tx) + sr_at(c * 8 + 4, ty + 1, tx + 1));
        const R uc = A.u[c][id];
        const R yv = ((mk >> c) & 1) ? uc : acc[c] + bottom;
        A.y[c][id] = yv;
        part += yv * uc;
        acc[c] = top;
      }
      dot += (double)part;
    }
  }
  if (own) {
    const long long id = g.nid(X, Y, nz);
    const uint8_t mk = A.mask[id];
    R part = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R uc = A.u[c][id];
      const R yv = ((mk >> c) & 1) ? uc : acc[c];
      A.y[c][id] = yv;
      part += yv * uc;
    }
    dot += (double)part;
  }
  if (A.partial != nullptr) {
    const double s = block_sum(dot);
    if (tid == 0) A.partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// ---- the same matvec with TMA-staged planes and two elements per thread.
// A CTA of 32 x TY threads covers 64 x TY elements (thread tx: elements
// X0 + 2 tx and X0 + 2 tx + 1 of row Y0 + ty, X0 = 63 bx - 1, Y0 = (TY-1) by
// - 1) and owns the 63 x (TY-1) node columns inside them. Per node plane one
// thread copies the three components of u (68 x (TY+1) node boxes from x
// rounded down to a multiple of 4), the constraint bits of those nodes and
// the voxel IDs of the element layer (80-byte rows from x rounded down to 16)
// and the plane's z record into four mbarrier-tracked shared-memory stages
// while the threads work on earlier planes. The element arithmetic is the
// pair form of hex8_apply (packed FP32). The nodal forces are gathered
// without a full shared-memory copy of the element forces: a node's two
// elements along x are summed in the thread (node ea+1) or with the next
// lane's element through a shuffle (node ea+2); the corners facing the row
// below (y) go through a small shared array to the thread row that owns
// that node row; the top corners of a layer stay in registers for the next
// plane. The sums are grouped as in hex8_matvec_kernel, term for term (equal
// to FP32 rounding).
//
// DIR: the Jacobi-PCG direction update p = D^-1 r + beta p_old (beta =
// r.z / r.z of the previous iteration) is fused into the staging: the
// residual, the inverse diagonal and the previous direction of each plane
// are copied instead of p, the new direction of the whole staged box is
// formed in shared memory two planes ahead of its first use (so that the
// plane's first barrier also publishes it), the product uses it, and the
// owners write it to the other direction buffer (p is double-buffered:
// neighbouring CTAs still read the old one).
constexpr int kMvStages = 4, kMvAhead = 3;
constexpr int kMvElems = 64;  // elements per warp row
template <typename R, int TY, bool DIR>
struct MvStage;
template <typename R, int TY>
struct MvStage<R, TY, false> {
  EmBox<R, TY + 1, kMvElems + 4> U[3];         // nodes X0 .. X0+64, Y0 .. Y0+TY (from x rounded to 4)
  EmBox<uint8_t, TY + 1, kMvElems + 16> M;     // constraint bits of the same nodes (from x rounded to 16)
  EmBox<uint8_t, TY, kMvElems + 16> V;         // voxel IDs of elements X0 .. X0+63, Y0 .. Y0+TY-1
  EmBox<R, 1, 4> Z;                            // hz(k), 1/hz(k), 1/dual_z(k), hz(k-1)
};
template <typename R, int TY>
struct MvStage<R, TY, true> : MvStage<R, TY, false> {  // U: p_old as copied, then the new p
  EmBox<R, TY + 1, kMvElems + 4> Rr[3];        // residual of the same nodes
  EmBox<R, TY + 1, kMvElems + 4> Dd[3];        // inverse Jacobi diagonal of the same nodes
};
// shared memory: the material table, then the exchange array of the row
// sums (6 pairs per thread), then the stages (128-byte aligned)
template <typename R, int TY>
__host__ __device__ constexpr size_t mv_stage_offset(int nmat) {
  return (((size_t)(nmat + 1) * M_COLS + 12 * TY * 32) * sizeof(R) + 127) & ~size_t(127);
}
template <typename R, int TY, bool DIR>
__host__ __device__ constexpr size_t mv_smem_bytes(int nmat) {
  return mv_stage_offset<R, TY>(nmat) + kMvStages * sizeof(MvStage<R, TY, DIR>) + 128;
}

struct CgScalars {  // device-resident scalars of the Jacobi-PCG, FP64
  double rz[2];     // r.z of the current / next iteration (ping-pong by parity)
  double pq;        // p.Kp
  double rr;        // r.r
  double bb;        // f.f
};

template <typename R>
struct MvTmaArgs {
  MvArgs<R> a;                 // u: the staged input (DIR: the new direction), y, mask, partial sums of u.y
  CUtensorMap tmU[3], tmM, tmV;
  CUtensorMap tmR[3], tmD[3];  // DIR: residual, inverse diagonal
  R *pn[3];                    // DIR: the new direction, written at the owned nodes
  R *x[3];                     // DIR: the iterate, x += alpha p_old at the owned nodes (alpha of the previous
                               // iteration, sc->rz[parity] / sc->pq); null: left to the update pass
  const R *po[3];              // DIR with x: p_old in global memory (the buffer the stages copy)
  const CgScalars *sc;         // DIR: beta = sc->rz[parity ^ 1] / sc->rz[parity]
  int parity;
  const R *zt;
  int *err;
  long long wait;              // bound of the waits for staged planes, SM clock cycles
};

template <typename R, int TY, bool DIR>
__global__ void __launch_bounds__(32 * TY, sizeof(R) == 4 ? 2 : 1)
    hex8_matvec_tma_kernel(const __grid_constant__ MvTmaArgs<R> TA) {
  using R2 = typename Pair2<R>::T;
  using Stage = MvStage<R, TY, DIR>;
  constexpr int EX = kMvElems, BX = kMvElems + 4;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char *smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  const MvArgs<R> &A = TA.a;
  const Geo<R> &g = A.g;
  R *s_mt = reinterpret_cast<R *>(smem);
  // ay = 0 corner sums of each thread's node pair, [c * 2 + az][ty][tx], read by thread row ty - 1
  R2 *s_lo = reinterpret_cast<R2 *>(s_mt + (g.nmat + 1) * M_COLS);
  Stage *stg = reinterpret_cast<Stage *>(smem + mv_stage_offset<R, TY>(g.nmat));
  __shared__ uint64_t bars[kMvStages];
  __shared__ int s_abort;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const bool leader = tid == 0;
  if (leader) {
    bool ok = (smem_u32(stg) & 127u) == 0 && (sizeof(Stage) & 127u) == 0 && ((size_t)&TA.tmU[0] & 63u) == 0 &&
              ((size_t)&TA.tmM & 63u) == 0 && ((size_t)&TA.tmV & 63u) == 0 && ((size_t)&TA.tmR[0] & 63u) == 0 &&
              ((size_t)&TA.tmD[0] & 63u) == 0;
    s_abort = ok ? 0 : 1;
    if (!ok) atomicExch(TA.err, 2);
    for (int q = 0; q < kMvStages; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
  }
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  __syncthreads();
  if (s_abort) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int X0 = blockIdx.x * (EX - 1) - 1, Y0 = blockIdx.y * (TY - 1) - 1;
  const int xr = X0 & 3, xu0 = X0 - xr;      // u boxes
  const int xmr = X0 & 15, xm0 = X0 - xmr;   // mask and voxel boxes
  const int ea = X0 + 2 * tx, ey = Y0 + ty;  // elements ea (.x) and ea + 1 (.y)
  const bool ey_ok = ey >= 0 && ey < ny;
  const bool va = ey_ok && ea >= 0 && ea < nx, vb = ey_ok && ea + 1 >= 0 && ea + 1 < nx;
  // owned nodes (ea + 1, ey + 1) and (ea + 2, ey + 1); the last lane's second
  // node belongs to the next tile
  const int XA = ea + 1, Y = ey + 1;
  const bool rowown = ty < TY - 1 && Y <= ny;
  const bool oa = rowown && XA <= nx, ob = rowown && tx < 31 && XA + 1 <= nx;
  const R2 hx = {va ? g.h[0][ea] : R(1), vb ? g.h[0][ea + 1] : R(1)};
  const R2 ihx = {va ? g.ih[0][ea] : R(1), vb ? g.ih[0][ea + 1] : R(1)};
  const R2 hy = bc_<R2>(ey_ok ? g.h[1][ey] : R(1)), ihy = bc_<R2>(ey_ok ? g.ih[1][ey] : R(1));
  const unsigned fixed_bytes = (unsigned)((DIR ? 9 : 3) * (TY + 1) * BX * (int)sizeof(R) + (TY + 1) * (EX + 16) +
                                          4 * (int)sizeof(R));
  const unsigned vox_bytes = (unsigned)(TY * (EX + 16));
  auto issue = [&](int k) {
    if (k > nz) return;
    const int s = k % kMvStages;
    Stage &S = stg[s];
    mbar_arrive_expect_tx(&bars[s], fixed_bytes + (k < nz ? vox_bytes : 0u));
#pragma unroll
    for (int c = 0; c < 3; ++c) tma_load_3d(&S.U[c].v[0][0], &TA.tmU[c], xu0, Y0, k, &bars[s]);
    if constexpr (DIR) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        tma_load_3d(&S.Rr[c].v[0][0], &TA.tmR[c], xu0, Y0, k, &bars[s]);
        tma_load_3d(&S.Dd[c].v[0][0], &TA.tmD[c], xu0, Y0, k, &bars[s]);
      }
    }
    tma_load_3d(&S.M.v[0][0], &TA.tmM, xm0, Y0, k, &bars[s]);
    if (k < nz) tma_load_3d(&S.V.v[0][0], &TA.tmV, xm0, Y0, k, &bars[s]);
    bulk_load(&S.Z.v[0][0], TA.zt + 4 * (size_t)k, 4 * sizeof(R), &bars[s]);
  };
  // DIR: the new direction of every staged node of plane kk, in place of the
  // old one (positions outside the grid arrived as zeros and stay zero); the
  // proxy fence orders these writes before the stage's next TMA fill
  R beta = R(0), alpha = R(0);
  if constexpr (DIR) {
    beta = (R)(TA.sc->rz[TA.parity ^ 1] / TA.sc->rz[TA.parity]);
    alpha = (R)(TA.sc->rz[TA.parity] / TA.sc->pq);  // (the previous iteration's step length)
  }
  const bool with_x = DIR && TA.x[0] != nullptr;
  auto convert = [&](int kk) {
    if constexpr (DIR) {
      Stage &S = stg[kk % kMvStages];
      for (int q = tid; q < (TY + 1) * BX; q += 32 * TY) {
        const int qy = q / BX, qx = q - qy * BX;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          S.U[c].v[qy][qx] = fma_(S.Dd[c].v[qy][qx], S.Rr[c].v[qy][qx], mul_(beta, S.U[c].v[qy][qx]));
      }
      fence_proxy_async_smem();
    }
  };
  if (leader)
    for (int q = 0; q < kMvAhead; ++q) issue(q);
  if constexpr (DIR) {  // planes 0 and 1 are converted before the loop (nz >= 1)
    bool ok = mbar_wait(&bars[0], 0u, TA.wait);
    ok = mbar_wait(&bars[1], 0u, TA.wait) && ok;
    if (!ok) s_abort = 1;
    __syncthreads();
    if (s_abort) {
      if (leader) {
        for (int q = 0; q < kMvAhead && q <= nz; ++q)
          mbar_wait(&bars[q % kMvStages], (unsigned)(q / kMvStages) & 1u, TA.wait);
        atomicExch(TA.err, 1);
      }
      return;
    }
    convert(0);
    convert(1);
  }
  R2 acc[3] = {bc_<R2>(R(0)), bc_<R2>(R(0)), bc_<R2>(R(0))};
  double dot = 0.0;
  R part4 = 0;  // the thread's u.y terms of up to four planes, one FP64 addition per four
  const int cu = 2 * tx + xr;  // element corner (ea, ey) column in the u boxes
  for (int k = 0; k < nz; ++k) {
    {
      bool ok = mbar_wait(&bars[k % kMvStages], (unsigned)(k / kMvStages) & 1u, TA.wait);
      ok = mbar_wait(&bars[(k + 1) % kMvStages], (unsigned)((k + 1) / kMvStages) & 1u, TA.wait) && ok;
      // DIR: plane k+2 is converted in this iteration, for use from the next
      if (DIR && k + 2 <= nz)
        ok = mbar_wait(&bars[(k + 2) % kMvStages], (unsigned)((k + 2) / kMvStages) & 1u, TA.wait) && ok;
      if (!ok) s_abort = 1;
    }
    // planes k, k+1 (and k+2) landed, k and k+1 converted; every thread is
    // done with plane k-1 and with s_lo
    __syncthreads();
    if (s_abort) {
      if (leader) {
        for (int q = k; q <= k + kMvAhead && q <= nz; ++q)
          mbar_wait(&bars[q % kMvStages], (unsigned)(q / kMvStages) & 1u, TA.wait);
        atomicExch(TA.err, 1);
      }
      return;
    }
    if (leader) {
      fence_proxy_async_smem();
      issue(k + kMvAhead);
    }
    // DIR: the new direction of plane k+2 (its stage is read from the next
    // iteration on, after that iteration's barrier)
    if constexpr (DIR)
      if (k + 2 <= nz) convert(k + 2);
    const Stage &S0 = stg[k % kMvStages];
    const Stage &S1 = stg[(k + 1) % kMvStages];
    // DIR with x: the owned nodes' x and p_old of this plane, requested now and
    // used in the owner phase (the element arithmetic hides their latency)
    R xo[3][2], pv[3][2];
    if (with_x && (oa || ob)) {
      const long long id = g.nid(XA, Y, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        xo[c][0] = oa ? TA.x[c][id] : R(0);
        pv[c][0] = oa ? TA.po[c][id] : R(0);
        xo[c][1] = ob ? TA.x[c][id + 1] : R(0);
        pv[c][1] = ob ? TA.po[c][id + 1] : R(0);
      }
    }
    R2 r[3][8];
    if (va || vb) {
      const int ma = va ? (int)S0.V.v[ty][2 * tx + xmr] : 0, mb = vb ? (int)S0.V.v[ty][2 * tx + 1 + xmr] : 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {  // corner rows (ay, az) = (q & 1, q >> 1): nodes cu .. cu + 2 of one staged row
        const Stage &S = (q >> 1) ? S1 : S0;
        const int qy = ty + (q & 1), mx = cu - xr + xmr;
        const unsigned m0 = S.M.v[qy][mx], m1 = S.M.v[qy][mx + 1], m2 = S.M.v[qy][mx + 2];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const R v0 = ((m0 >> c) & 1) ? R(0) : S.U[c].v[qy][cu];
          const R v1 = ((m1 >> c) & 1) ? R(0) : S.U[c].v[qy][cu + 1];
          const R v2 = ((m2 >> c) & 1) ? R(0) : S.U[c].v[qy][cu + 2];
          r[c][2 * q] = R2{v0, v1};
          r[c][2 * q + 1] = R2{v1, v2};
        }
      }
      hex8_apply<R2, R>(r, R2{s_mt[ma * M_COLS + M_LAM], s_mt[mb * M_COLS + M_LAM]},
                        R2{s_mt[ma * M_COLS + M_MU], s_mt[mb * M_COLS + M_MU]}, hx, hy, bc_<R2>(S0.Z.v[0][0]), ihx,
                        ihy, bc_<R2>(S0.Z.v[0][1]));
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 8; ++a) r[c][a] = R2{va ? r[c][a].x : R(0), vb ? r[c][a].y : R(0)};
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int a = 0; a < 8; ++a) r[c][a] = bc_<R2>(R(0));
    }
    // corner a = ax + 2 ay + 4 az. Node A (ea+1) takes corner ax=1 of element
    // ea and ax=0 of ea+1; node B (ea+2) ax=1 of ea+1 and ax=0 of the next
    // lane's element ea+2. The ay=1 sums stay here (this row's nodes), the
    // ay=0 sums go to the thread row below's nodes through s_lo.
    R2 hi[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int az = 0; az < 2; ++az) {
        const int b = 4 * az;
        const R n2 = __shfl_down_sync(0xffffffffu, r[c][b + 2].x, 1);
        const R n0 = __shfl_down_sync(0xffffffffu, r[c][b + 0].x, 1);
        hi[c][az] = add_(R2{r[c][b + 3].x, r[c][b + 3].y}, R2{r[c][b + 2].y, n2});
        s_lo[((c * 2 + az) * TY + ty) * 32 + tx] = add_(R2{r[c][b + 1].x, r[c][b + 1].y}, R2{r[c][b + 0].y, n0});
      }
    __syncthreads();
    if (oa || ob) {
      const long long id = g.nid(XA, Y, k);
      R part = 0;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R2 bottom = add_(hi[c][0], s_lo[((c * 2) * TY + ty + 1) * 32 + tx]);
        const R2 top = add_(hi[c][1], s_lo[((c * 2 + 1) * TY + ty + 1) * 32 + tx]);
        const uint8_t mka = S0.M.v[ty + 1][cu + 1 - xr + xmr], mkb = S0.M.v[ty + 1][cu + 2 - xr + xmr];
        const R ua = S0.U[c].v[ty + 1][cu + 1], ub = S0.U[c].v[ty + 1][cu + 2];
        const R2 sum = add_(acc[c], bottom);
        const R ya = ((mka >> c) & 1) ? ua : sum.x, yb = ((mkb >> c) & 1) ? ub : sum.y;
        if (oa) {
          A.y[c][id] = ya;
          part += ya * ua;
          if constexpr (DIR) {
            TA.pn[c][id] = ua;
            if (with_x) TA.x[c][id] = fma_(alpha, pv[c][0], xo[c][0]);
          }
        }
        if (ob) {
          A.y[c][id + 1] = yb;
          part += yb * ub;
          if constexpr (DIR) {
            TA.pn[c][id + 1] = ub;
            if (with_x) TA.x[c][id + 1] = fma_(alpha, pv[c][1], xo[c][1]);
          }
        }
        acc[c] = top;
      }
      part4 += part;
      if ((k & 3) == 3) {
        dot += (double)part4;
        part4 = 0;
      }
    }
  }
  if (oa || ob) {  // the top node plane: plane nz is still staged (nothing was issued after it)
    const Stage &S = stg[nz % kMvStages];
    const long long id = g.nid(XA, Y, nz);
    R part = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint8_t mka = S.M.v[ty + 1][cu + 1 - xr + xmr], mkb = S.M.v[ty + 1][cu + 2 - xr + xmr];
      const R ua = S.U[c].v[ty + 1][cu + 1], ub = S.U[c].v[ty + 1][cu + 2];
      const R ya = ((mka >> c) & 1) ? ua : acc[c].x, yb = ((mkb >> c) & 1) ? ub : acc[c].y;
      if (oa) {
        A.y[c][id] = ya;
        part += ya * ua;
        if constexpr (DIR) {
          TA.pn[c][id] = ua;
          if (with_x) TA.x[c][id] = fma_(alpha, TA.po[c][id], TA.x[c][id]);
        }
      }
      if (ob) {
        A.y[c][id + 1] = yb;
        part += yb * ub;
        if constexpr (DIR) {
          TA.pn[c][id + 1] = ub;
          if (with_x) TA.x[c][id + 1] = fma_(alpha, TA.po[c][id + 1], TA.x[c][id + 1]);
        }
      }
    }
    part4 += part;
  }
  dot += (double)part4;
  if (A.partial != nullptr) {
    const double s = block_sum(dot);
    if (tid == 0) A.partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// Node-gather kernels over the <=8 elements around node (i,j,k):
// element e = (i-1+dx, j-1+dy, k-1+dz), the node is its corner (1-dx, 1-dy, 1-dz).
//
// MODE 0 (Jacobi diagonal, stores 1/diag): K_e(a c, a c) =
//   (lambda + mu) V/(9 h_c^2) + mu V/9 (1/hx^2 + 1/hy^2 + 1/hz^2) for every corner a.
// MODE 1 (thermal load, Eq. 8 right-hand side): f_{a,c} = beta_e int dN_a/dx_c dT dV,
//   beta = (3 lambda + 2 mu) alpha_L, dT trilinear from nodal T - T_ref; with the
//   monomial coefficients t of dT, int dN_a/dx_c dT dV = V (2/h_c)(s_c/8)
//   [t_0 + s_d1 t_d1/3 + s_d2 t_d2/3 + s_d1 s_d2 t_d1d2/9], (d1, d2) the other axes.
//
// A thread owns the node column (i, j) and marches k = 0..nz: the four
// elements of layer k are formed once and give the node of plane k its terms
// as their bottom corner (dz = 1) and the node of plane k+1 its terms as
// their top corner (dz = 0, carried in registers), and the nodal dT of a
// plane's 3 x 3 neighbourhood is read once and kept for the next layer. Each
// node adds the same terms in the same order as an 8-element gather
// (layer k-1 first, then layer k; dy, dx inner).
template <typename R, int MODE>
__global__ void __launch_bounds__(256) hex8_node_kernel(Geo<R> g, const uint8_t *mask, const R *T, R T_ref,
                                                         R *o0, R *o1, R *o2) {
  extern __shared__ unsigned char smem_raw[];
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i > nx || j > ny) return;
  // dT of node plane k (tp) and k+1 (tq) at (i-1+qx, j-1+qy), q = qx + 3 qy
  R tp[9], tq[9];
  auto load_plane = [&](int kk, R t9[9]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const int ni = i - 1 + q % 3, nj = j - 1 + q / 3;
      t9[q] = (ni >= 0 && ni <= nx && nj >= 0 && nj <= ny) ? T[g.nid(ni, nj, kk)] - T_ref : R(0);
    }
  };
  if (MODE == 1) load_plane(0, tp);
  R carry[3] = {0, 0, 0};  // top-corner terms of layer k-1 for the node of plane k
  R *out[3] = {o0, o1, o2};
  // the column's lateral cell sizes, read once (the stores below could alias
  // the geometry arrays for the compiler, which would then reload them)
  R hxc[2], ihxc[2], hyc[2], ihyc[2];
#pragma unroll
  for (int d = 0; d < 2; ++d) {
    const int ei = i - 1 + d, ej = j - 1 + d;
    hxc[d] = (ei >= 0 && ei < nx) ? g.h[0][ei] : R(0);
    ihxc[d] = (ei >= 0 && ei < nx) ? g.ih[0][ei] : R(0);
    hyc[d] = (ej >= 0 && ej < ny) ? g.h[1][ej] : R(0);
    ihyc[d] = (ej >= 0 && ej < ny) ? g.ih[1][ej] : R(0);
  }
  for (int k = 0; k <= nz; ++k) {
    R acc[3] = {carry[0], carry[1], carry[2]};
    carry[0] = carry[1] = carry[2] = R(0);
    if (k < nz) {
      if (MODE == 1) load_plane(k + 1, tq);
      const R hzk = g.h[2][k], ihzk = g.ih[2][k];
#pragma unroll
      for (int dy = 0; dy < 2; ++dy)
#pragma unroll
        for (int dx = 0; dx < 2; ++dx) {
          const int ei = i - 1 + dx, ej = j - 1 + dy;
          const int m = g.cell(ei, ej, k);
          if (m < 0) continue;
          const R h[3] = {hxc[dx], hyc[dy], hzk};
          const R ih[3] = {ihxc[dx], ihyc[dy], ihzk};  // inverse sizes (no divisions)
          const R V = h[0] * h[1] * h[2];
          const R lam = s_mt[m * M_COLS + M_LAM], mu = s_mt[m * M_COLS + M_MU];
          if (MODE == 0) {
            const R lap = ih[0] * ih[0] + ih[1] * ih[1] + ih[2] * ih[2];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              acc[c] += (lam + mu) * V * (ih[c] * ih[c]) * (R(1) / R(9)) + mu * V * lap * (R(1) / R(9));
              carry[c] += (lam + mu) * V * (ih[c] * ih[c]) * (R(1) / R(9)) + mu * V * lap * (R(1) / R(9));
            }
          } else {
            R t[8];  // corner a = (ax, ay, az): node (ei + ax, ej + ay, k + az)
#pragma unroll
            for (int a = 0; a < 8; ++a) {
              const int q = (dx + (a & 1)) + 3 * (dy + ((a >> 1) & 1));
              t[a] = (a >> 2) ? tq[q] : tp[q];
            }
            modal_fwd(t);
            const int lin[3] = {1, 2, 4};
            const R beta = s_mt[m * M_COLS + M_BETA];
#pragma unroll
            for (int dz = 0; dz < 2; ++dz) {  // dz = 1: the node of plane k; dz = 0: the node of plane k+1
              const R s[3] = {R(1 - 2 * dx), R(1 - 2 * dy), R(1 - 2 * dz)};  // node's corner signs
              R *dst = dz ? acc : carry;
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                const int d1 = (c + 1) % 3, d2 = (c + 2) % 3;
                const R br = t[0] + s[d1] * t[lin[d1]] * (R(1) / R(3)) + s[d2] * t[lin[d2]] * (R(1) / R(3)) +
                             s[d1] * s[d2] * t[lin[d1] | lin[d2]] * (R(1) / R(9));
                // t holds 8x the monomial coefficients: fold 1/8 here
                dst[c] += beta * V * (R(2) * ih[c]) * s[c] * R(0.125) * R(0.125) * br;
              }
            }
          }
        }
    }
    const long long id = g.nid(i, j, k);
    const uint8_t mk = mask[id];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const bool fixed = (mk >> c) & 1;
      if (MODE == 0)
        out[c][id] = fixed ? R(1) : R(1) / acc[c];
      else
        out[c][id] = fixed ? R(0) : acc[c];
    }
    if (MODE == 1 && k < nz) {
#pragma unroll
      for (int q = 0; q < 9; ++q) tp[q] = tq[q];
    }
  }
}

// Eq. 9 at the centroid of every element: strain from the constant part of
// the gradient (linear monomials), dT_c = mean of the 8 nodal dT,
// sigma = lambda tr(eps) I + 2 mu eps - beta dT_c I. Cell-sized output.
template <typename R>
__global__ void __launch_bounds__(256) von_mises_kernel(Geo<R> g, const R *u0, const R *u1, const R *u2, const R *T,
                                                         R T_ref, R *vm) {
  extern __shared__ unsigned char smem_raw[];
  R *s_mt = reinterpret_cast<R *>(smem_raw);
  stage_table(s_mt, g.mtab, g.nmat * M_COLS);
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const R *u[3] = {u0, u1, u2};
  const R qh[3] = {R(0.25) * g.ih[0][i], R(0.25) * g.ih[1][j], R(0.25) * g.ih[2][k]};  // (2/h) / 8
  R G[3][3];
  R tm = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R v[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = u[c][g.nid(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))];
    modal_fwd(v);
    G[c][0] = v[1] * qh[0];  // (2/h) * (sum / 8)
    G[c][1] = v[2] * qh[1];
    G[c][2] = v[4] * qh[2];
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) tm += T[g.nid(i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))] - T_ref;
  const int m = g.cell(i, j, k);
  const R lam = s_mt[m * M_COLS + M_LAM], mu = s_mt[m * M_COLS + M_MU], beta = s_mt[m * M_COLS + M_BETA];
  const R tr = G[0][0] + G[1][1] + G[2][2];
  const R th = lam * tr - beta * R(0.125) * tm;
  const R sx = th + 2 * mu * G[0][0], sy = th + 2 * mu * G[1][1], sz = th + 2 * mu * G[2][2];
  const R txy = mu * (G[0][1] + G[1][0]), tyz = mu * (G[1][2] + G[2][1]), tzx = mu * (G[2][0] + G[0][2]);
  const R v2 = R(0.5) * ((sx - sy) * (sx - sy) + (sy - sz) * (sy - sz) + (sz - sx) * (sz - sx)) +
               R(3) * (txy * txy + tyz * tyz + tzx * tzx);
  vm[((long long)k * g.ny + j) * g.nx + i] = sqrt(v2);
}

// ---- Jacobi-PCG vector kernels over the padded SoA node arrays (padding is 0).
// Grid-stride with a fixed grid: the per-CTA partial sums, and therefore the
// reductions, are deterministic. Dot products accumulate in FP64 (FP32
// contexts: over partial sums of four nodes formed in FP32).


template <typename R>
__global__ void __launch_bounds__(256) cg_init_kernel(long long n, const R *f0, const R *f1, const R *f2,
                                                       const R *d0, const R *d1, const R *d2, R *x0, R *x1,
                                                       R *x2, R *r0, R *r1, R *r2, R *p0, R *p1, R *p2,
                                                       double *part_rz, double *part_bb, R scale) {
  // scale: a power of two that brings the right-hand side to order one
  // (exact: the iteration is then the unscaled one times that factor)
  double rz = 0, bb = 0;
  const long long stride = (long long)gridDim.x * blockDim.x, first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {  // four nodes per access (n is a multiple of 4), one FP64 addition per group
    const R *F[3] = {f0, f1, f2}, *Dg[3] = {d0, d1, d2};
    R *Xv[3] = {x0, x1, x2}, *Rv[3] = {r0, r1, r2}, *Pv[3] = {p0, p1, p2};
    for (long long v = first; v < (n >> 2); v += stride) {
      float4 a[3], z[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 f = reinterpret_cast<const float4 *>(F[c])[v], d = reinterpret_cast<const float4 *>(Dg[c])[v];
        a[c] = make_float4(scale * f.x, scale * f.y, scale * f.z, scale * f.w);
        z[c] = make_float4(d.x * a[c].x, d.y * a[c].y, d.z * a[c].z, d.w * a[c].w);
        reinterpret_cast<float4 *>(Xv[c])[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<float4 *>(Rv[c])[v] = a[c];
        reinterpret_cast<float4 *>(Pv[c])[v] = z[c];
      }
      const float zx = a[0].x * z[0].x + a[1].x * z[1].x + a[2].x * z[2].x;
      const float zy = a[0].y * z[0].y + a[1].y * z[1].y + a[2].y * z[2].y;
      const float zz = a[0].z * z[0].z + a[1].z * z[1].z + a[2].z * z[2].z;
      const float zw = a[0].w * z[0].w + a[1].w * z[1].w + a[2].w * z[2].w;
      const float sx = a[0].x * a[0].x + a[1].x * a[1].x + a[2].x * a[2].x;
      const float sy = a[0].y * a[0].y + a[1].y * a[1].y + a[2].y * a[2].y;
      const float sz = a[0].z * a[0].z + a[1].z * a[1].z + a[2].z * a[2].z;
      const float sw = a[0].w * a[0].w + a[1].w * a[1].w + a[2].w * a[2].w;
      rz += (double)((zx + zy) + (zz + zw));
      bb += (double)((sx + sy) + (sz + sw));
    }
  } else {
    for (long long q = first; q < n; q += stride) {
      const R a0 = scale * f0[q], a1 = scale * f1[q], a2 = scale * f2[q];
      const R z0 = d0[q] * a0, z1 = d1[q] * a1, z2 = d2[q] * a2;
      x0[q] = 0; x1[q] = 0; x2[q] = 0;
      r0[q] = a0; r1[q] = a1; r2[q] = a2;
      p0[q] = z0; p1[q] = z1; p2[q] = z2;
      rz += (double)(a0 * z0 + a1 * z1 + a2 * z2);
      bb += (double)(a0 * a0 + a1 * a1 + a2 * a2);
    }
  }
  rz = block_sum(rz);
  bb = block_sum(bb);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = rz;
    part_bb[blockIdx.x] = bb;
  }
}

// partial sums of f.f (each node's three-component term in the context
// precision; FP32 contexts sum four nodes in FP32 per FP64 addition)
template <typename R>
__global__ void __launch_bounds__(256) sumsq3_kernel(long long n, const R *f0, const R *f1, const R *f2,
                                                      double *part) {
  double ss = 0;
  const long long stride = (long long)gridDim.x * blockDim.x, first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {  // four nodes per access (n is a multiple of 4)
    for (long long v = first; v < (n >> 2); v += stride) {
      const float4 a = reinterpret_cast<const float4 *>(f0)[v], b = reinterpret_cast<const float4 *>(f1)[v],
                   c = reinterpret_cast<const float4 *>(f2)[v];
      const float sx = a.x * a.x + b.x * b.x + c.x * c.x, sy = a.y * a.y + b.y * b.y + c.y * c.y;
      const float sz = a.z * a.z + b.z * b.z + c.z * c.z, sw = a.w * a.w + b.w * b.w + c.w * c.w;
      ss += (double)((sx + sy) + (sz + sw));  // one FP64 addition per four nodes
    }
  } else {
    for (long long q = first; q < n; q += stride) {
      const R a0 = f0[q], a1 = f1[q], a2 = f2[q];
      ss += (double)(a0 * a0 + a1 * a1 + a2 * a2);
    }
  }
  ss = block_sum(ss);
  if (threadIdx.x == 0) part[blockIdx.x] = ss;
}

// x += alpha p (X; otherwise the next product applies it), r -= alpha q,
// alpha = rz/pq; partial sums of r.(D^-1 r) and r.r (each node's
// three-component terms in the context precision; FP32 contexts sum the
// terms of each group of four nodes in FP32, and the groups are accumulated
// in FP64). FP32 vectors are streamed four nodes per load (n is a multiple of
// 4: the padded node arrays have rows of a multiple of 32).
template <typename R, bool X>
__global__ void __launch_bounds__(256) cg_update_kernel(long long n, const CgScalars *sc, int parity, R *x0, R *x1,
                                                         R *x2, R *r0, R *r1, R *r2, const R *p0, const R *p1,
                                                         const R *p2, const R *q0, const R *q1, const R *q2,
                                                         const R *d0, const R *d1, const R *d2, double *part_rz,
                                                         double *part_rr) {
  const R alpha = (R)(sc->rz[parity] / sc->pq);
  double rz = 0, rr = 0;
  const long long stride = (long long)gridDim.x * blockDim.x, first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    R *Xv[3] = {x0, x1, x2}, *Rr[3] = {r0, r1, r2};
    const R *P[3] = {p0, p1, p2}, *Q[3] = {q0, q1, q2}, *D[3] = {d0, d1, d2};
    for (long long v = first; v < (n >> 2); v += stride) {
      float4 a[3], dd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float4 qv = reinterpret_cast<const float4 *>(Q[c])[v];
        float4 rv = reinterpret_cast<const float4 *>(Rr[c])[v];
        dd[c] = reinterpret_cast<const float4 *>(D[c])[v];
        if constexpr (X) {
          const float4 pv = reinterpret_cast<const float4 *>(P[c])[v];
          float4 xv = reinterpret_cast<const float4 *>(Xv[c])[v];
          xv.x += alpha * pv.x, xv.y += alpha * pv.y, xv.z += alpha * pv.z, xv.w += alpha * pv.w;
          reinterpret_cast<float4 *>(Xv[c])[v] = xv;
        }
        rv.x -= alpha * qv.x, rv.y -= alpha * qv.y, rv.z -= alpha * qv.z, rv.w -= alpha * qv.w;
        reinterpret_cast<float4 *>(Rr[c])[v] = rv;
        a[c] = rv;
      }
      // the four nodes' terms summed in FP32, one FP64 addition per group
      // (FP64 arithmetic is slow on this part: per-node FP64 additions made
      // the pass bound by them rather than by DRAM)
      const float zx = a[0].x * dd[0].x * a[0].x + a[1].x * dd[1].x * a[1].x + a[2].x * dd[2].x * a[2].x;
      const float zy = a[0].y * dd[0].y * a[0].y + a[1].y * dd[1].y * a[1].y + a[2].y * dd[2].y * a[2].y;
      const float zz = a[0].z * dd[0].z * a[0].z + a[1].z * dd[1].z * a[1].z + a[2].z * dd[2].z * a[2].z;
      const float zw = a[0].w * dd[0].w * a[0].w + a[1].w * dd[1].w * a[1].w + a[2].w * dd[2].w * a[2].w;
      const float sx = a[0].x * a[0].x + a[1].x * a[1].x + a[2].x * a[2].x;
      const float sy = a[0].y * a[0].y + a[1].y * a[1].y + a[2].y * a[2].y;
      const float sz = a[0].z * a[0].z + a[1].z * a[1].z + a[2].z * a[2].z;
      const float sw = a[0].w * a[0].w + a[1].w * a[1].w + a[2].w * a[2].w;
      rz += (double)((zx + zy) + (zz + zw));
      rr += (double)((sx + sy) + (sz + sw));
    }
  } else {
    for (long long q = first; q < n; q += stride) {
      if constexpr (X) {
        x0[q] += alpha * p0[q];
        x1[q] += alpha * p1[q];
        x2[q] += alpha * p2[q];
      }
      const R a0 = r0[q] - alpha * q0[q], a1 = r1[q] - alpha * q1[q], a2 = r2[q] - alpha * q2[q];
      r0[q] = a0; r1[q] = a1; r2[q] = a2;
      rz += (double)(a0 * d0[q] * a0 + a1 * d1[q] * a1 + a2 * d2[q] * a2);
      rr += (double)(a0 * a0 + a1 * a1 + a2 * a2);
    }
  }
  rz = block_sum(rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = rz;
    part_rr[blockIdx.x] = rr;
  }
}

// x += alpha p, alpha = rz[parity] / pq: the last direction's step when the
// products applied the earlier ones (FP32: four nodes per access)
template <typename R>
__global__ void __launch_bounds__(256) cg_axpy_kernel(long long n, const CgScalars *sc, int parity, R *x0, R *x1,
                                                       R *x2, const R *p0, const R *p1, const R *p2, R s) {
  // s: the solution's final scale (1: none), applied in the same pass
  const R alpha = (R)(sc->rz[parity] / sc->pq);
  const bool scaled = s != R(1);
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(R) == 4) {
    float4 *X[3] = {reinterpret_cast<float4 *>(x0), reinterpret_cast<float4 *>(x1), reinterpret_cast<float4 *>(x2)};
    const float4 *P[3] = {reinterpret_cast<const float4 *>(p0), reinterpret_cast<const float4 *>(p1),
                          reinterpret_cast<const float4 *>(p2)};
    for (long long v = first; v < (n >> 2); v += stride)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float4 x = X[c][v];
        const float4 p = P[c][v];
        x.x += alpha * p.x, x.y += alpha * p.y, x.z += alpha * p.z, x.w += alpha * p.w;
        if (scaled) x.x *= s, x.y *= s, x.z *= s, x.w *= s;
        X[c][v] = x;
      }
  } else {
    for (long long q = first; q < n; q += stride) {
      R a = x0[q] + alpha * p0[q], b = x1[q] + alpha * p1[q], c = x2[q] + alpha * p2[q];
      if (scaled) a *= s, b *= s, c *= s;
      x0[q] = a;
      x1[q] = b;
      x2[q] = c;
    }
  }
}

// x *= s for the three components (undoes the right-hand-side scaling)
template <typename R>
__global__ void __launch_bounds__(256) scale3_kernel(long long n, R *x0, R *x1, R *x2, R s) {
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(R) == 4) {  // four nodes per access (n is a multiple of 4)
    float4 *X[3] = {reinterpret_cast<float4 *>(x0), reinterpret_cast<float4 *>(x1), reinterpret_cast<float4 *>(x2)};
    for (long long v = first; v < (n >> 2); v += stride)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float4 x = X[c][v];
        x.x *= s, x.y *= s, x.z *= s, x.w *= s;
        X[c][v] = x;
      }
  } else {
    for (long long q = first; q < n; q += stride) {
      x0[q] *= s;
      x1[q] *= s;
      x2[q] *= s;
    }
  }
}

// p = D^-1 r + beta p, beta = rz_new / rz_old (FP32: four nodes per load)
template <typename R>
__global__ void __launch_bounds__(256) cg_direction_kernel(long long n, const CgScalars *sc, int parity, R *p0,
                                                            R *p1, R *p2, const R *r0, const R *r1, const R *r2,
                                                            const R *d0, const R *d1, const R *d2) {
  const R beta = (R)(sc->rz[parity ^ 1] / sc->rz[parity]);
  const long long stride = (long long)gridDim.x * blockDim.x, first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    R *P[3] = {p0, p1, p2};
    const R *Rr[3] = {r0, r1, r2}, *D[3] = {d0, d1, d2};
    for (long long v = first; v < (n >> 2); v += stride) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float4 pv = reinterpret_cast<const float4 *>(P[c])[v];
        const float4 rv = reinterpret_cast<const float4 *>(Rr[c])[v], dv = reinterpret_cast<const float4 *>(D[c])[v];
        pv.x = dv.x * rv.x + beta * pv.x, pv.y = dv.y * rv.y + beta * pv.y;
        pv.z = dv.z * rv.z + beta * pv.z, pv.w = dv.w * rv.w + beta * pv.w;
        reinterpret_cast<float4 *>(P[c])[v] = pv;
      }
    }
  } else {
    for (long long q = first; q < n; q += stride) {
      p0[q] = d0[q] * r0[q] + beta * p0[q];
      p1[q] = d1[q] * r1[q] + beta * p1[q];
      p2[q] = d2[q] * r2[q] + beta * p2[q];
    }
  }
}

__global__ void __launch_bounds__(1024) reduce_final_kernel(const double *part, int n, double *out) {
  double s = 0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += part[q];
  s = block_sum(s);
  if (threadIdx.x == 0) *out = s;
}

// sum of a padded FP64 array (first stage)
__global__ void __launch_bounds__(256) sum_partial_kernel(long long n, const double *a, double *part) {
  double s = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    s += a[q];
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// min of a node-sized ratio array restricted to real nodes (first stage)
template <typename R>
__global__ void __launch_bounds__(256) min_partial_kernel(Geo<R> g, const R *a, double *part) {
  __shared__ double s_min[256];
  double m = 1e300;
  const long long n = g.plane * (g.nz + 1);
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % g.px);
    const int j = (int)((q / g.px) % (g.ny + 1));
    if (i <= g.nx && j <= g.ny) m = fmin(m, (double)a[q]);
  }
  s_min[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s_min[0];
}

__global__ void __launch_bounds__(256) min_final_kernel(const double *part, int n, double *out) {
  __shared__ double s_min[256];
  double m = 1e300;
  for (int q = threadIdx.x; q < n; q += blockDim.x) m = fmin(m, part[q]);
  s_min[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s_min[0];
}

// ---- mixed-precision iterative refinement (FP64 outer residual, context-precision CG)

// d_c = (D) s_c for three SoA arrays
template <typename S, typename D>
__global__ void __launch_bounds__(256) cast3_kernel(long long n, const S *s0, const S *s1, const S *s2, D *d0, D *d1,
                                                     D *d2) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    d0[q] = (D)s0[q];
    d1[q] = (D)s1[q];
    d2[q] = (D)s2[q];
  }
}

// r = f - Ku in FP64 (Ku given in r, overwritten); per-CTA partial sums of r.r
__global__ void __launch_bounds__(256) residual64_kernel(long long n, const double *f0, const double *f1,
                                                          const double *f2, double *r0, double *r1, double *r2,
                                                          double *part_rr) {
  double rr = 0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double a0 = f0[q] - r0[q], a1 = f1[q] - r1[q], a2 = f2[q] - r2[q];
    r0[q] = a0;
    r1[q] = a1;
    r2[q] = a2;
    rr += a0 * a0 + a1 * a1 + a2 * a2;
  }
  rr = block_sum(rr);
  if (threadIdx.x == 0) part_rr[blockIdx.x] = rr;
}

// u += d (FP64 solution, correction in the context precision)
template <typename R>
__global__ void __launch_bounds__(256) add_correction_kernel(long long n, double *u0, double *u1, double *u2,
                                                              const R *d0, const R *d1, const R *d2) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    u0[q] += (double)d0[q];
    u1[q] += (double)d1[q];
    u2[q] += (double)d2[q];
  }
}

// |u| per node
template <typename R>
__global__ void __launch_bounds__(256) umag_kernel(long long n, const R *u0, const R *u1, const R *u2, R *out) {
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(R) == 4) {  // four nodes per access (n is a multiple of 4)
    for (long long v = first; v < (n >> 2); v += stride) {
      const float4 a = reinterpret_cast<const float4 *>(u0)[v], b = reinterpret_cast<const float4 *>(u1)[v],
                   c = reinterpret_cast<const float4 *>(u2)[v];
      reinterpret_cast<float4 *>(out)[v] = make_float4(sqrt(a.x * a.x + b.x * b.x + c.x * c.x),
                                                       sqrt(a.y * a.y + b.y * b.y + c.y * c.y),
                                                       sqrt(a.z * a.z + b.z * b.z + c.z * c.z),
                                                       sqrt(a.w * a.w + b.w * b.w + c.w * c.w));
    }
  } else {
    for (long long q = first; q < n; q += stride) out[q] = sqrt(u0[q] * u0[q] + u1[q] * u1[q] + u2[q] * u2[q]);
  }
}

// Fixed-component bits of the built-in supports (bit c: component c held at
// zero), written into a zeroed padded mask: clamped bottom (bc 0, every z = 0
// node) or the three-node kinematic mount (bc 1: the bottom centre fixed in
// x, y, z, the +x edge node in y, z and the +y edge node in z, six DOFs).
__global__ void __launch_bounds__(256) support_mask_kernel(uint8_t *mask, int nx, int ny, int px, int bc) {
  if (bc == 0) {
    const long long n = (long long)(nx + 1) * (ny + 1);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
      mask[(q / (nx + 1)) * px + q % (nx + 1)] = 7;
  } else if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int ic = nx / 2, jc = ny / 2;
    mask[(long long)jc * px + ic] |= 7;
    mask[(long long)jc * px + nx] |= 6;
    mask[(long long)ny * px + ic] |= 4;
  }
}

}  // namespace cosim
