/*
 * Plain FP64 CPU oracle of the transient EM-thermal-mechanical package solver.
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA path and is used by
 * tests/, by the smoke check and by the CPU-baseline leg of the benchmark; the
 * product path never loads it. It shares no code, header or table with the
 * CUDA sources. Every function is a direct, unblocked loop over the discrete
 * unknowns in double precision, written for a reader checking it against the
 * paper by eye, not for speed.
 *
 * Discretisation (one voxel grid for all three physics, Sec. II):
 *   cells (i,j,k) with sizes dx[i], dy[j], dz[k]; nodes (i,j,k), 0<=i<=nx ...;
 *   every node-sized array has (nx+1)(ny+1)(nz+1) entries, x fastest.
 *   E of axis a lives on the primal edge from node n to n+e_a (n[a] < n_a);
 *   H of axis a lives on the primal face normal to a whose lowest corner is n
 *   (n[b] < n_b for the two other axes b); T and displacement live on nodes;
 *   materials live on voxels.
 *
 * EM (Sec. II-A, Eqs. 1-3): the second-order system of Eq. 1 is advanced with
 * the equivalent staggered E/H leapfrog. Eliminating H from
 *   mu dH/dt = -curl E,   eps dE/dt + sigma E = curl H - J
 * discretised centrally in time gives M e^{n+1} = N e^n - K e^{n-1} - dt^2 (dJ/dt)^n
 * with M = D_eps + dt/2 D_sigma, N = 2 D_eps - dt^2 S, K = D_eps - dt/2 D_sigma
 * and S = C^T D_{1/mu} C (Eq. 2-3), (dJ/dt)^n ~ (J^{n+1/2} - J^{n-1/2})/dt.
 * Joule power (Sec. II-A, P_total = D_sigma e^2) uses the time-centred edge field.
 * Two-way coupling (Sec. II-A): sigma(T) = sigma0 / (1 + alpha (T - T0)) per
 * voxel at the edge temperature (mean of the end nodes); the synchronized
 * step (og_coupled_step) advances EM with D_sigma(T^n) and then T with the
 * same dt and that step's Joule power.
 * Thermal (Eqs. 4-5): nodal forward Euler with M_kk = V0a^T D_k V0 (7-point).
 * Mechanics (Sec. II-B, Eqs. 7-9): HEX8, 2x2x2 Gauss, isotropic E_c(lambda,mu),
 * thermal strain alpha*dT*[1,1,1,0,0,0], von Mises at the element centroid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_EPS0 8.8541878128e-12
#define OG_MU0 1.25663706212e-6

enum { OG_PEC = 0, OG_PMC = 1, OG_CPML = 2 };
/* material table columns */
enum { T_EPSR, T_MUR, T_SIGMA, T_TCR, T_T0, T_K, T_RHOCP, T_E, T_NU, T_ALPHA, T_NCOL };

typedef struct {
  int nx, ny, nz;
  const double *h[3];     /* cell sizes along x, y, z */
  const uint8_t *mat;     /* voxel material id, nz*ny*nx, x fastest */
  int nmat;
  const double *tab;      /* nmat rows of T_NCOL columns */
  int em_bc[6];           /* faces x-, x+, y-, y+, z-, z+ */
  int cpml_cells;
  double cpml_order;
  double cpml_eps_r;
  double h_conv[6];       /* convective film coefficient per face */
  double T_amb;
} og_grid;

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */

static int n_of(const og_grid *g, int a) { return a == 0 ? g->nx : (a == 1 ? g->ny : g->nz); }

static size_t nid(const og_grid *g, const int n[3]) {
  return ((size_t)n[2] * (g->ny + 1) + n[1]) * (g->nx + 1) + n[0];
}

static size_t n_nodes(const og_grid *g) {
  return (size_t)(g->nx + 1) * (g->ny + 1) * (g->nz + 1);
}

static int voxel(const og_grid *g, const int c[3]) {
  return g->mat[((size_t)c[2] * g->ny + c[1]) * g->nx + c[0]];
}

static double prop(const og_grid *g, int m, int col) { return g->tab[m * T_NCOL + col]; }

/* length of the dual edge through node p along axis a (half cells at walls) */
static double dual_len(const og_grid *g, int a, int p) {
  double s = 0.0;
  if (p > 0) s += 0.5 * g->h[a][p - 1];
  if (p < n_of(g, a)) s += 0.5 * g->h[a][p];
  return s;
}

static int e_valid(const og_grid *g, int a, const int n[3]) { return n[a] < n_of(g, a); }

static int h_valid(const og_grid *g, int a, const int n[3]) {
  int b = (a + 1) % 3, c = (a + 2) % 3;
  return n[b] < n_of(g, b) && n[c] < n_of(g, c);
}

/* An E edge tangential to a PEC wall (PEC faces and the PEC backing of CPML
 * faces) is held at zero; PMC walls leave it free (ghost tangential H = 0). */
static int e_fixed(const og_grid *g, int a, const int n[3]) {
  for (int b = 0; b < 3; b++) {
    if (b == a) continue;
    if (n[b] == 0 && g->em_bc[2 * b] != OG_PMC) return 1;
    if (n[b] == n_of(g, b) && g->em_bc[2 * b + 1] != OG_PMC) return 1;
  }
  return 0;
}

/* Sums over the (up to four) voxels that share the edge of axis a at node n.
 * Each voxel c contributes its quarter cross-section w_c normal to the edge:
 *   W  = sum w_c           (dual-face area of the edge)
 *   Se = sum w_c eps_c,  Ss = sum w_c sigma_c,  Sk = sum w_c k_c
 * so the edge's eps, sigma and k are the area-weighted voxel means. */
static void edge_sums(const og_grid *g, int a, const int n[3],
                      double *W, double *Se, double *Ss, double *Sk) {
  int b = (a + 1) % 3, c = (a + 2) % 3;
  *W = *Se = *Ss = *Sk = 0.0;
  for (int db = -1; db <= 0; db++)
    for (int dc = -1; dc <= 0; dc++) {
      int cell[3];
      cell[a] = n[a];
      cell[b] = n[b] + db;
      cell[c] = n[c] + dc;
      if (cell[b] < 0 || cell[b] >= n_of(g, b) || cell[c] < 0 || cell[c] >= n_of(g, c)) continue;
      int m = voxel(g, cell);
      double w = 0.25 * g->h[b][cell[b]] * g->h[c][cell[c]];
      *W += w;
      *Se += w * OG_EPS0 * prop(g, m, T_EPSR);
      *Ss += w * prop(g, m, T_SIGMA);
      *Sk += w * prop(g, m, T_K);
    }
}

/* dt / mu of the H unknown of axis a at node n: the dual edge crosses the two
 * voxels n[a]-1 and n[a] (half of each); mu_face = sum(l) / sum(l / mu)
 * (reluctances in series). */
static double face_dt_over_mu(const og_grid *g, int a, const int n[3], double dt) {
  double sl = 0.0, L = 0.0;
  for (int d = -1; d <= 0; d++) {
    int cell[3] = {n[0], n[1], n[2]};
    cell[a] = n[a] + d;
    if (cell[a] < 0 || cell[a] >= n_of(g, a)) continue;
    double l = 0.5 * g->h[a][cell[a]];
    sl += l / (OG_MU0 * prop(g, voxel(g, cell), T_MUR));
    L += l;
  }
  return dt * sl / L;
}

/* ------------------------------------------------------------------------ */
/* EM                                                                        */

/* Time step: cfl times the Courant limit of the finest cells at the largest
 * wave speed present (Sec. II-A). */
double og_cfl_dt(const og_grid *g, double cfl) {
  double vmax = 0.0;
  for (int m = 0; m < g->nmat; m++) {
    double v = 1.0 / sqrt(OG_EPS0 * prop(g, m, T_EPSR) * OG_MU0 * prop(g, m, T_MUR));
    if (v > vmax) vmax = v;
  }
  double s = 0.0;
  for (int a = 0; a < 3; a++) {
    double hmin = g->h[a][0];
    for (int p = 1; p < n_of(g, a); p++)
      if (g->h[a][p] < hmin) hmin = g->h[a][p];
    s += 1.0 / (hmin * hmin);
  }
  return cfl / (vmax * sqrt(s));
}

/* CPML stretching coefficients (kappa = 1, alpha = 0):
 *   sigma(x) = sigma_max (rho/d)^m inside a layer of thickness d (rho = depth),
 *   sigma_max = 0.8 (m+1) / (eta0 * (d/L) * sqrt(eps_r_bg)),
 *   b = exp(-sigma dt / eps0), c = b - 1, psi <- b psi + c dF/dx.
 * at = 0: values at nodes p = 0..n (derivatives taken for E unknowns);
 * at = 1: values at the centres of cells p = 0..n-1 (for H unknowns).
 * Outside the layers b = 1, c = 0. Fills b[], c[] for every p of axis a. */
static void cpml_table(const og_grid *g, int a, int at, double dt, double *b, double *c) {
  int L = g->cpml_cells, n = n_of(g, a), np = at ? n : n + 1;
  double *x = (double *)malloc(sizeof(double) * (n + 1));
  x[0] = 0.0;
  for (int q = 0; q < n; q++) x[q + 1] = x[q] + g->h[a][q];
  double m = g->cpml_order, eta0 = sqrt(OG_MU0 / OG_EPS0);
  for (int p = 0; p < np; p++) {
    double pos = at ? 0.5 * (x[p] + x[p + 1]) : x[p], sig = 0.0;
    if (L > 0 && g->em_bc[2 * a] == OG_CPML) {
      double xi = x[L], d = x[L] - x[0];
      if (pos < xi) sig = 0.8 * (m + 1) / (eta0 * (d / L) * sqrt(g->cpml_eps_r)) * pow((xi - pos) / d, m);
    }
    if (L > 0 && g->em_bc[2 * a + 1] == OG_CPML) {
      double xi = x[n - L], d = x[n] - x[n - L];
      if (pos > xi) sig = 0.8 * (m + 1) / (eta0 * (d / L) * sqrt(g->cpml_eps_r)) * pow((pos - xi) / d, m);
    }
    b[p] = 1.0;
    c[p] = 0.0;
    if (sig > 0.0) {
      b[p] = exp(-sig * dt / OG_EPS0);
      c[p] = b[p] - 1.0;
    }
  }
  free(x);
}

/* per-axis CPML tables for one update */
typedef struct { double *b[3], *c[3]; } cpml_tabs;

static void cpml_build(const og_grid *g, int at, double dt, cpml_tabs *t) {
  for (int a = 0; a < 3; a++) {
    t->b[a] = (double *)malloc(sizeof(double) * (n_of(g, a) + 1));
    t->c[a] = (double *)malloc(sizeof(double) * (n_of(g, a) + 1));
    cpml_table(g, a, at, dt, t->b[a], t->c[a]);
  }
}

static void cpml_free(cpml_tabs *t) {
  for (int a = 0; a < 3; a++) { free(t->b[a]); free(t->c[a]); }
}

/* CPML coefficients exported for inspection by tests */
void og_cpml_table(const og_grid *g, int a, int at, double dt, double *b, double *c) {
  cpml_table(g, a, at, dt, b, c);
}

/* psi storage: 6 node-sized arrays for H then 6 for E. Slot 2*a + s holds the
 * auxiliary of component a for the derivative along axis (a+1+s)%3. */
static double *psi_slot(double *psi, const og_grid *g, int is_e, int a, int s) {
  return psi + ((size_t)(is_e ? 6 : 0) + 2 * a + s) * n_nodes(g);
}

/* Faraday half-step (Sec. II-A): H^{n+1/2} = H^{n-1/2} - (dt/mu) curl E^n.
 * (curl E)_a = dE_c/db - dE_b/dc with (a,b,c) cyclic; primal edge lengths.
 * Inside CPML layers the derivative along axis d gets + psi_d. */
void og_h_update(const og_grid *g, double dt, double *const E[3], double *const H[3], double *psi) {
  cpml_tabs t;
  if (psi) cpml_build(g, 1, dt, &t);
  for (int a = 0; a < 3; a++) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double *pb = psi ? psi_slot(psi, g, 0, a, 0) : NULL;
    double *pc = psi ? psi_slot(psi, g, 0, a, 1) : NULL;
    int n[3];
    for (n[2] = 0; n[2] <= g->nz; n[2]++)
      for (n[1] = 0; n[1] <= g->ny; n[1]++)
        for (n[0] = 0; n[0] <= g->nx; n[0]++) {
          if (!h_valid(g, a, n)) continue;
          size_t id = nid(g, n);
          int nb[3] = {n[0], n[1], n[2]}, nc[3] = {n[0], n[1], n[2]};
          nb[b] += 1;
          nc[c] += 1;
          double dEc_db = (E[c][nid(g, nb)] - E[c][id]) / g->h[b][n[b]];
          double dEb_dc = (E[b][nid(g, nc)] - E[b][id]) / g->h[c][n[c]];
          double curl = dEc_db - dEb_dc;
          if (psi) {
            pb[id] = t.b[b][n[b]] * pb[id] + t.c[b][n[b]] * dEc_db;
            pc[id] = t.b[c][n[c]] * pc[id] + t.c[c][n[c]] * dEb_dc;
            curl += pb[id] - pc[id];
          }
          H[a][id] -= face_dt_over_mu(g, a, n, dt) * curl;
        }
  }
  if (psi) cpml_free(&t);
}

/* Ampere step (Sec. II-A, Eq. 2-3 in leapfrog form):
 *   eps_e (E^{n+1} - E^n)/dt + sigma_e (E^{n+1} + E^n)/2 = (curl H^{n+1/2})_e - J_e^{n+1/2}
 * i.e. E^{n+1} = ca E^n + cb (curl H - J) with
 *   ca = (Se - Ss dt/2) / (Se + Ss dt/2),  cb = dt W / (Se + Ss dt/2).
 * (curl H)_a = dH_c/db - dH_b/dc over dual lengths; an H unknown outside the
 * domain (beyond a wall) counts as zero. J may be NULL. */
static double edge_sigma_T(const og_grid *g, int a, const int n[3], const double *theta, double T_off);

/* theta == NULL: the voxels' own conductivities; otherwise the conductivities
 * at temperature T = theta + T_off (edge_sigma_T, Sec. II-A coupling). */
static void e_update(const og_grid *g, double dt, double *const H[3], double *const E[3], double *psi,
                     double *const J[3], const double *theta, double T_off) {
  cpml_tabs t;
  if (psi) cpml_build(g, 0, dt, &t);
  for (int a = 0; a < 3; a++) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double *pb = psi ? psi_slot(psi, g, 1, a, 0) : NULL;
    double *pc = psi ? psi_slot(psi, g, 1, a, 1) : NULL;
    int n[3];
    for (n[2] = 0; n[2] <= g->nz; n[2]++)
      for (n[1] = 0; n[1] <= g->ny; n[1]++)
        for (n[0] = 0; n[0] <= g->nx; n[0]++) {
          if (!e_valid(g, a, n) || e_fixed(g, a, n)) continue;
          size_t id = nid(g, n);
          int mb[3] = {n[0], n[1], n[2]}, mc[3] = {n[0], n[1], n[2]};
          mb[b] -= 1;
          mc[c] -= 1;
          double Hc_hi = h_valid(g, c, n) ? H[c][id] : 0.0;
          double Hc_lo = (mb[b] >= 0 && h_valid(g, c, mb)) ? H[c][nid(g, mb)] : 0.0;
          double Hb_hi = h_valid(g, b, n) ? H[b][id] : 0.0;
          double Hb_lo = (mc[c] >= 0 && h_valid(g, b, mc)) ? H[b][nid(g, mc)] : 0.0;
          double dHc_db = (Hc_hi - Hc_lo) / dual_len(g, b, n[b]);
          double dHb_dc = (Hb_hi - Hb_lo) / dual_len(g, c, n[c]);
          double curl = dHc_db - dHb_dc;
          if (psi) {
            pb[id] = t.b[b][n[b]] * pb[id] + t.c[b][n[b]] * dHc_db;
            pc[id] = t.b[c][n[c]] * pc[id] + t.c[c][n[c]] * dHb_dc;
            curl += pb[id] - pc[id];
          }
          double W, Se, Ss, Sk;
          edge_sums(g, a, n, &W, &Se, &Ss, &Sk);
          if (theta) Ss = edge_sigma_T(g, a, n, theta, T_off);
          double den = Se + 0.5 * dt * Ss;
          double ca = (Se - 0.5 * dt * Ss) / den;
          double cb_ = dt * W / den;
          double j = J ? J[a][id] : 0.0;
          E[a][id] = ca * E[a][id] + cb_ * (curl - j);
        }
  }
  if (psi) cpml_free(&t);
}

void og_e_update(const og_grid *g, double dt, double *const H[3], double *const E[3], double *psi,
                 double *const J[3]) {
  e_update(g, dt, H, E, psi, J, NULL, 0.0);
}

/* Joule heat of one step (Sec. II-A, P_total = D_sigma e^2): every edge
 * dissipates p_e = sigma_e V_e ebar^2 with ebar = (E^n + E^{n+1})/2 and
 * sigma_e V_e = Ss * edge length; dt * p_e / 2 goes to each end node. */
void og_joule_accumulate(const og_grid *g, double dt, double *const Eold[3], double *const Enew[3],
                         double *Q) {
  for (int a = 0; a < 3; a++) {
    int n[3];
    for (n[2] = 0; n[2] <= g->nz; n[2]++)
      for (n[1] = 0; n[1] <= g->ny; n[1]++)
        for (n[0] = 0; n[0] <= g->nx; n[0]++) {
          if (!e_valid(g, a, n)) continue;
          double W, Se, Ss, Sk;
          edge_sums(g, a, n, &W, &Se, &Ss, &Sk);
          size_t id = nid(g, n);
          double eb = 0.5 * (Eold[a][id] + Enew[a][id]);
          double p = Ss * g->h[a][n[a]] * eb * eb;
          int m[3] = {n[0], n[1], n[2]};
          m[a] += 1;
          Q[id] += 0.5 * dt * p;
          Q[nid(g, m)] += 0.5 * dt * p;
        }
  }
}

/* Counts of unknowns: EM = primal edges that are updated, thermal = nodes,
 * mechanical = 3 x nodes (before kinematic constraints). */
void og_count_dofs(const og_grid *g, int64_t *n_em, int64_t *n_th, int64_t *n_mech) {
  int64_t ne = 0;
  for (int a = 0; a < 3; a++) {
    int n[3];
    for (n[2] = 0; n[2] <= g->nz; n[2]++)
      for (n[1] = 0; n[1] <= g->ny; n[1]++)
        for (n[0] = 0; n[0] <= g->nx; n[0]++)
          if (e_valid(g, a, n) && !e_fixed(g, a, n)) ne++;
  }
  *n_em = ne;
  *n_th = (int64_t)n_nodes(g);
  *n_mech = 3 * (int64_t)n_nodes(g);
}

/* ------------------------------------------------------------------------ */
/* thermal (Sec. II-A, Eqs. 4-5)                                             */

/* rho*c_p of the node's dual volume: sum over adjacent voxels of rho_cp V/8 */
static double node_capacity(const og_grid *g, const int n[3]) {
  double C = 0.0;
  for (int dz = -1; dz <= 0; dz++)
    for (int dy = -1; dy <= 0; dy++)
      for (int dx = -1; dx <= 0; dx++) {
        int c[3] = {n[0] + dx, n[1] + dy, n[2] + dz};
        if (c[0] < 0 || c[1] < 0 || c[2] < 0 || c[0] >= g->nx || c[1] >= g->ny || c[2] >= g->nz) continue;
        double V = g->h[0][c[0]] * g->h[1][c[1]] * g->h[2][c[2]];
        C += prop(g, voxel(g, c), T_RHOCP) * V / 8.0;
      }
  return C;
}

/* conductance of the edge of axis a at node n: k_e A*_e / l_e = Sk / l_e */
static double edge_conductance(const og_grid *g, int a, const int n[3]) {
  double W, Se, Ss, Sk;
  edge_sums(g, a, n, &W, &Se, &Ss, &Sk);
  return Sk / g->h[a][n[a]];
}

/* sum over convective faces touching node n of h_f times the node's share of
 * the face area (product of its two transverse dual lengths) */
static double node_film(const og_grid *g, const int n[3]) {
  double s = 0.0;
  for (int a = 0; a < 3; a++) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    double A = dual_len(g, b, n[b]) * dual_len(g, c, n[c]);
    if (n[a] == 0) s += g->h_conv[2 * a] * A;
    if (n[a] == n_of(g, a)) s += g->h_conv[2 * a + 1] * A;
  }
  return s;
}

/* sum of the conductances of the (up to six) edges at node n */
static double node_gsum(const og_grid *g, const int n[3]) {
  double s = 0.0;
  for (int a = 0; a < 3; a++) {
    if (n[a] < n_of(g, a)) s += edge_conductance(g, a, n);
    if (n[a] > 0) {
      int m[3] = {n[0], n[1], n[2]};
      m[a] -= 1;
      s += edge_conductance(g, a, m);
    }
  }
  return s;
}

/* Forward-Euler stability (monotonicity) limit: min_i C_i / (sum_j G_ij + h A_i) */
double og_thermal_dt_limit(const og_grid *g) {
  double lim = INFINITY;
  int n[3];
  for (n[2] = 0; n[2] <= g->nz; n[2]++)
    for (n[1] = 0; n[1] <= g->ny; n[1]++)
      for (n[0] = 0; n[0] <= g->nx; n[0]++) {
        double r = node_capacity(g, n) / (node_gsum(g, n) + node_film(g, n));
        if (r < lim) lim = r;
      }
  return lim;
}

/* Eq. 5: T^{n+1}_i = T^n_i + dt/C_i [ sum_j G_ij (T_j - T_i) + h A_i (T_amb - T_i) + P_i ]
 * (-M_kk T expanded edge by edge). P [W per node] may be NULL. */
void og_thermal_step(const og_grid *g, double dt, const double *T, const double *P, double *Tout) {
  int n[3];
  for (n[2] = 0; n[2] <= g->nz; n[2]++)
    for (n[1] = 0; n[1] <= g->ny; n[1]++)
      for (n[0] = 0; n[0] <= g->nx; n[0]++) {
        size_t id = nid(g, n);
        double flux = 0.0;
        for (int a = 0; a < 3; a++) {
          if (n[a] < n_of(g, a)) {
            int m[3] = {n[0], n[1], n[2]};
            m[a] += 1;
            flux += edge_conductance(g, a, n) * (T[nid(g, m)] - T[id]);
          }
          if (n[a] > 0) {
            int m[3] = {n[0], n[1], n[2]};
            m[a] -= 1;
            flux += edge_conductance(g, a, m) * (T[nid(g, m)] - T[id]);
          }
        }
        flux += node_film(g, n) * (g->T_amb - T[id]);
        if (P) flux += P[id];
        Tout[id] = T[id] + dt / node_capacity(g, n) * flux;
      }
}

/* Node heat capacities (rho c_p V summed over the node's dual volume). */
void og_node_capacity(const og_grid *g, double *C) {
  int n[3];
  for (n[2] = 0; n[2] <= g->nz; n[2]++)
    for (n[1] = 0; n[1] <= g->ny; n[1]++)
      for (n[0] = 0; n[0] <= g->nx; n[0]++) C[nid(g, n)] = node_capacity(g, n);
}

/* ------------------------------------------------------------------------ */
/* mechanics (Sec. II-B, Eqs. 7-9)                                           */

/* local node a = ax + 2 ay + 4 az; reference coordinates s = 2*bit - 1 */
static double sgn(int a, int d) { return ((a >> d) & 1) ? 1.0 : -1.0; }

/* shape function N_a and its physical derivatives at reference point xi[3] */
static void shape(int a, const double xi[3], const double hh[3], double *N, double dN[3]) {
  double f[3], df[3];
  for (int d = 0; d < 3; d++) {
    f[d] = 0.5 * (1.0 + sgn(a, d) * xi[d]);
    df[d] = 0.5 * sgn(a, d) * 2.0 / hh[d];   /* d/dx = (2/h) d/dxi */
  }
  *N = f[0] * f[1] * f[2];
  dN[0] = df[0] * f[1] * f[2];
  dN[1] = f[0] * df[1] * f[2];
  dN[2] = f[0] * f[1] * df[2];
}

/* strain-displacement matrix B (6 x 24), Voigt order xx yy zz xy yz zx,
 * engineering shear strains */
static void bmatrix(const double xi[3], const double hh[3], double B[6][24], double N[8]) {
  memset(B, 0, sizeof(double) * 6 * 24);
  for (int a = 0; a < 8; a++) {
    double dN[3];
    shape(a, xi, hh, &N[a], dN);
    B[0][3 * a + 0] = dN[0];
    B[1][3 * a + 1] = dN[1];
    B[2][3 * a + 2] = dN[2];
    B[3][3 * a + 0] = dN[1];
    B[3][3 * a + 1] = dN[0];
    B[4][3 * a + 1] = dN[2];
    B[4][3 * a + 2] = dN[1];
    B[5][3 * a + 0] = dN[2];
    B[5][3 * a + 2] = dN[0];
  }
}

/* isotropic E_c (Voigt, engineering shear) */
static void elasticity(double lam, double mu, double D[6][6]) {
  memset(D, 0, sizeof(double) * 36);
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) D[i][j] = lam;
    D[i][i] = lam + 2.0 * mu;
    D[3 + i][3 + i] = mu;
  }
}

static void lame(const og_grid *g, int m, double *lam, double *mu) {
  double E = prop(g, m, T_E), nu = prop(g, m, T_NU);
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  *mu = E / (2.0 * (1.0 + nu));
}

/* Element stiffness of an hx*hy*hz brick (Eq. 8 left-hand side), split as
 * K_e = lambda * Kl + mu * Km, integrated with 2x2x2 Gauss points at +-1/sqrt(3). */
void og_hex8_element(const double hh[3], double *Kl, double *Km) {
  const double gp = 1.0 / sqrt(3.0);
  double detJ = hh[0] * hh[1] * hh[2] / 8.0;
  double Dl[6][6], Dm[6][6];
  elasticity(1.0, 0.0, Dl);
  elasticity(0.0, 1.0, Dm);
  memset(Kl, 0, sizeof(double) * 576);
  memset(Km, 0, sizeof(double) * 576);
  for (int q = 0; q < 8; q++) {
    double xi[3] = {sgn(q, 0) * gp, sgn(q, 1) * gp, sgn(q, 2) * gp};
    double B[6][24], N[8];
    bmatrix(xi, hh, B, N);
    for (int r = 0; r < 24; r++)
      for (int s = 0; s < 24; s++) {
        double al = 0.0, am = 0.0;
        for (int p = 0; p < 6; p++)
          for (int t = 0; t < 6; t++) {
            al += B[p][r] * Dl[p][t] * B[t][s];
            am += B[p][r] * Dm[p][t] * B[t][s];
          }
        Kl[r * 24 + s] += detJ * al;
        Km[r * 24 + s] += detJ * am;
      }
  }
}

/* global node of local node a of element (i,j,k) */
static size_t elem_node(const og_grid *g, int i, int j, int k, int a) {
  int n[3] = {i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1)};
  return nid(g, n);
}

typedef struct { double hh[3]; double Kl[576], Km[576]; int valid; } elem_cache;

static const double *cached_element(elem_cache *ec, const double hh[3], int which) {
  if (!ec->valid || ec->hh[0] != hh[0] || ec->hh[1] != hh[1] || ec->hh[2] != hh[2]) {
    og_hex8_element(hh, ec->Kl, ec->Km);
    memcpy(ec->hh, hh, sizeof(double) * 3);
    ec->valid = 1;
  }
  return which ? ec->Km : ec->Kl;
}

/* y = K u with the constrained DOFs (fixed[dof] != 0) eliminated: their rows
 * and columns are zeroed and the diagonal set to one, so y_c = u_c.
 * DOF index = 3*node + component. */
void og_hex8_matvec(const og_grid *g, const uint8_t *fixed, const double *u, double *y) {
  size_t ndof = 3 * n_nodes(g);
  memset(y, 0, sizeof(double) * ndof);
  elem_cache *ec = (elem_cache *)calloc(1, sizeof(elem_cache));
  for (int k = 0; k < g->nz; k++)
    for (int j = 0; j < g->ny; j++)
      for (int i = 0; i < g->nx; i++) {
        double hh[3] = {g->h[0][i], g->h[1][j], g->h[2][k]};
        int c[3] = {i, j, k};
        double lam, mu;
        lame(g, voxel(g, c), &lam, &mu);
        const double *Kl = cached_element(ec, hh, 0);
        const double *Km = cached_element(ec, hh, 1);
        size_t dof[24];
        double ue[24];
        for (int a = 0; a < 8; a++)
          for (int d = 0; d < 3; d++) {
            dof[3 * a + d] = 3 * elem_node(g, i, j, k, a) + d;
            ue[3 * a + d] = fixed[dof[3 * a + d]] ? 0.0 : u[dof[3 * a + d]];
          }
        for (int r = 0; r < 24; r++) {
          if (fixed[dof[r]]) continue;
          double s = 0.0;
          for (int t = 0; t < 24; t++) s += (lam * Kl[r * 24 + t] + mu * Km[r * 24 + t]) * ue[t];
          y[dof[r]] += s;
        }
      }
  for (size_t d = 0; d < ndof; d++)
    if (fixed[d]) y[d] = u[d];
  free(ec);
}

/* diagonal of the constrained stiffness (Jacobi preconditioner) */
void og_hex8_diag(const og_grid *g, const uint8_t *fixed, double *dg) {
  size_t ndof = 3 * n_nodes(g);
  memset(dg, 0, sizeof(double) * ndof);
  elem_cache *ec = (elem_cache *)calloc(1, sizeof(elem_cache));
  for (int k = 0; k < g->nz; k++)
    for (int j = 0; j < g->ny; j++)
      for (int i = 0; i < g->nx; i++) {
        double hh[3] = {g->h[0][i], g->h[1][j], g->h[2][k]};
        int c[3] = {i, j, k};
        double lam, mu;
        lame(g, voxel(g, c), &lam, &mu);
        const double *Kl = cached_element(ec, hh, 0);
        const double *Km = cached_element(ec, hh, 1);
        for (int a = 0; a < 8; a++)
          for (int d = 0; d < 3; d++) {
            int r = 3 * a + d;
            dg[3 * elem_node(g, i, j, k, a) + d] += lam * Kl[r * 24 + r] + mu * Km[r * 24 + r];
          }
      }
  for (size_t d = 0; d < ndof; d++)
    if (fixed[d]) dg[d] = 1.0;
  free(ec);
}

/* Thermal load (Eq. 8 right-hand side): f_e = sum_q detJ B^T E_c eps_T(q),
 * eps_T = alpha_L dT(q) [1,1,1,0,0,0], dT(q) trilinear from nodal T - Tref. */
void og_thermal_load(const og_grid *g, const uint8_t *fixed, const double *T, double Tref, double *f) {
  size_t ndof = 3 * n_nodes(g);
  memset(f, 0, sizeof(double) * ndof);
  const double gp = 1.0 / sqrt(3.0);
  for (int k = 0; k < g->nz; k++)
    for (int j = 0; j < g->ny; j++)
      for (int i = 0; i < g->nx; i++) {
        double hh[3] = {g->h[0][i], g->h[1][j], g->h[2][k]};
        int c[3] = {i, j, k};
        int m = voxel(g, c);
        double lam, mu, D[6][6];
        lame(g, m, &lam, &mu);
        elasticity(lam, mu, D);
        double alpha = prop(g, m, T_ALPHA), detJ = hh[0] * hh[1] * hh[2] / 8.0;
        for (int q = 0; q < 8; q++) {
          double xi[3] = {sgn(q, 0) * gp, sgn(q, 1) * gp, sgn(q, 2) * gp};
          double B[6][24], N[8];
          bmatrix(xi, hh, B, N);
          double dT = 0.0;
          for (int a = 0; a < 8; a++) dT += N[a] * (T[elem_node(g, i, j, k, a)] - Tref);
          double epsT[6] = {alpha * dT, alpha * dT, alpha * dT, 0, 0, 0};
          double sig[6];
          for (int p = 0; p < 6; p++) {
            sig[p] = 0.0;
            for (int t = 0; t < 6; t++) sig[p] += D[p][t] * epsT[t];
          }
          for (int a = 0; a < 8; a++)
            for (int d = 0; d < 3; d++) {
              double s = 0.0;
              for (int p = 0; p < 6; p++) s += B[p][3 * a + d] * sig[p];
              f[3 * elem_node(g, i, j, k, a) + d] += detJ * s;
            }
        }
      }
  for (size_t d = 0; d < ndof; d++)
    if (fixed[d]) f[d] = 0.0;
}

/* Jacobi-preconditioned conjugate gradients on K u = f (u starts at zero).
 * Stops when ||r|| <= rtol ||f|| or after maxit iterations. */
void og_pcg(const og_grid *g, const uint8_t *fixed, const double *f, double *u, double rtol,
            int64_t maxit, int64_t *iters, double *relres) {
  size_t nd = 3 * n_nodes(g);
  double *r = (double *)malloc(sizeof(double) * nd), *z = (double *)malloc(sizeof(double) * nd);
  double *p = (double *)malloc(sizeof(double) * nd), *q = (double *)malloc(sizeof(double) * nd);
  double *dg = (double *)malloc(sizeof(double) * nd);
  og_hex8_diag(g, fixed, dg);
  double bb = 0.0, rz = 0.0, rr;
  for (size_t d = 0; d < nd; d++) {
    u[d] = 0.0;
    r[d] = f[d];
    z[d] = r[d] / dg[d];
    p[d] = z[d];
    bb += f[d] * f[d];
    rz += r[d] * z[d];
  }
  double bnorm = sqrt(bb);
  int64_t it = 0;
  *relres = bnorm > 0 ? 1.0 : 0.0;
  while (bnorm > 0 && it < maxit) {
    og_hex8_matvec(g, fixed, p, q);
    double pq = 0.0;
    for (size_t d = 0; d < nd; d++) pq += p[d] * q[d];
    double alpha = rz / pq;
    rr = 0.0;
    for (size_t d = 0; d < nd; d++) {
      u[d] += alpha * p[d];
      r[d] -= alpha * q[d];
      rr += r[d] * r[d];
    }
    it++;
    *relres = sqrt(rr) / bnorm;
    if (*relres <= rtol) break;
    double rz_new = 0.0;
    for (size_t d = 0; d < nd; d++) {
      z[d] = r[d] / dg[d];
      rz_new += r[d] * z[d];
    }
    double beta = rz_new / rz;
    rz = rz_new;
    for (size_t d = 0; d < nd; d++) p[d] = z[d] + beta * p[d];
  }
  *iters = it;
  free(r); free(z); free(p); free(q); free(dg);
}

/* Eq. 9 at each element centroid (xi = 0): sigma = E_c (B(0) q_e - alpha dT_c [1,1,1,0,0,0]),
 * dT_c = mean of the eight nodal T - Tref. Also |u| at every node. */
void og_von_mises(const og_grid *g, const double *u, const double *T, double Tref, double *vm,
                  double *umag) {
  const double xi[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g->nz; k++)
    for (int j = 0; j < g->ny; j++)
      for (int i = 0; i < g->nx; i++) {
        double hh[3] = {g->h[0][i], g->h[1][j], g->h[2][k]};
        int c[3] = {i, j, k};
        int m = voxel(g, c);
        double lam, mu, D[6][6], B[6][24], N[8];
        lame(g, m, &lam, &mu);
        elasticity(lam, mu, D);
        bmatrix(xi, hh, B, N);
        double dTc = 0.0;
        for (int a = 0; a < 8; a++) dTc += (T[elem_node(g, i, j, k, a)] - Tref) / 8.0;
        double alpha = prop(g, m, T_ALPHA), eps[6];
        for (int p = 0; p < 6; p++) {
          eps[p] = 0.0;
          for (int a = 0; a < 8; a++)
            for (int d = 0; d < 3; d++) eps[p] += B[p][3 * a + d] * u[3 * elem_node(g, i, j, k, a) + d];
          if (p < 3) eps[p] -= alpha * dTc;
        }
        double s[6];
        for (int p = 0; p < 6; p++) {
          s[p] = 0.0;
          for (int t = 0; t < 6; t++) s[p] += D[p][t] * eps[t];
        }
        vm[((size_t)k * g->ny + j) * g->nx + i] =
            sqrt(0.5 * ((s[0] - s[1]) * (s[0] - s[1]) + (s[1] - s[2]) * (s[1] - s[2]) +
                        (s[2] - s[0]) * (s[2] - s[0]) +
                        6.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5])));
      }
  size_t nn = n_nodes(g);
  for (size_t d = 0; d < nn; d++)
    umag[d] = sqrt(u[3 * d] * u[3 * d] + u[3 * d + 1] * u[3 * d + 1] + u[3 * d + 2] * u[3 * d + 2]);
}

/* ------------------------------------------------------------------------ */
/* Two-way electro-thermal coupling (Sec. II-A)                              */

/* Electrical conductivity of material m at absolute temperature T_abs, the
 * coupling law of Sec. II-A: sigma(T) = sigma0 / (1 + alpha (T - T0)), alpha
 * the temperature coefficient of resistance. */
static double sigma_at(const og_grid *g, int m, double T_abs) {
  return prop(g, m, T_SIGMA) / (1.0 + prop(g, m, T_TCR) * (T_abs - prop(g, m, T_T0)));
}

/* Ss = sum_c w_c sigma_c(T_e) over the voxels of the edge of axis a at node n
 * (the voxels and weights of edge_sums, in the same order), every voxel's
 * conductivity taken at the edge temperature T_e = mean of the edge's two end
 * nodes, T = theta + T_off. With alpha = 0 this is edge_sums' Ss exactly. */
static double edge_sigma_T(const og_grid *g, int a, const int n[3], const double *theta, double T_off) {
  int m1[3] = {n[0], n[1], n[2]};
  m1[a] += 1;
  const double Te = 0.5 * (theta[nid(g, n)] + theta[nid(g, m1)]) + T_off;
  int b = (a + 1) % 3, c = (a + 2) % 3;
  double Ss = 0.0;
  for (int db = -1; db <= 0; db++)
    for (int dc = -1; dc <= 0; dc++) {
      int cell[3];
      cell[a] = n[a];
      cell[b] = n[b] + db;
      cell[c] = n[c] + dc;
      if (cell[b] < 0 || cell[b] >= n_of(g, b) || cell[c] < 0 || cell[c] >= n_of(g, c)) continue;
      double w = 0.25 * g->h[b][cell[b]] * g->h[c][cell[c]];
      Ss += w * sigma_at(g, voxel(g, cell), Te);
    }
  return Ss;
}

/* Joule power of one step with the conductivities at temperature theta
 * (P_total = D_sigma(T) e^2 of Sec. II-A with the time-centred field): each
 * edge's p_e = sigma_e(T) V_e ebar^2 [W], half to each end node; P is zeroed
 * first. */
void og_joule_power_T(const og_grid *g, double *const Eold[3], double *const Enew[3], const double *theta,
                      double T_off, double *P) {
  memset(P, 0, sizeof(double) * n_nodes(g));
  for (int a = 0; a < 3; a++) {
    int n[3];
    for (n[2] = 0; n[2] <= g->nz; n[2]++)
      for (n[1] = 0; n[1] <= g->ny; n[1]++)
        for (n[0] = 0; n[0] <= g->nx; n[0]++) {
          if (!e_valid(g, a, n)) continue;
          size_t id = nid(g, n);
          double eb = 0.5 * (Eold[a][id] + Enew[a][id]);
          double p = edge_sigma_T(g, a, n, theta, T_off) * g->h[a][n[a]] * eb * eb;
          int m[3] = {n[0], n[1], n[2]};
          m[a] += 1;
          P[id] += 0.5 * p;
          P[nid(g, m)] += 0.5 * p;
        }
  }
}

/* One step of the synchronized electro-thermal marching of Sec. II-A, in the
 * paper's order: the conductivities are taken at T^n (D_sigma(T^n) in M and
 * K of Eq. 3), H and E advance one leapfrog step (Eqs. 2-3 in E/H form), the
 * step's Joule power P^{n+1} = D_sigma(T^n) ebar^2 is formed, and the
 * temperature takes one forward-Euler step of Eq. 5 with the same dt and
 * that power: theta_out = theta + dt/C (sum G (theta_j - theta) + film + P).
 * theta = T - T_off (kelvin); P receives P^{n+1} [W per node]; Q, if not
 * NULL, accumulates the step's Joule energy dt P. */
void og_coupled_step(const og_grid *g, double dt, double *const E[3], double *const H[3], double *psi,
                     double *const J[3], const double *theta, double T_off, double *P, double *theta_out,
                     double *Q) {
  size_t nn = n_nodes(g);
  og_h_update(g, dt, E, H, psi);
  double *Eold[3];
  for (int a = 0; a < 3; a++) {
    Eold[a] = (double *)malloc(sizeof(double) * nn);
    memcpy(Eold[a], E[a], sizeof(double) * nn);
  }
  e_update(g, dt, H, E, psi, J, theta, T_off);
  og_joule_power_T(g, Eold, E, theta, T_off, P);
  og_thermal_step(g, dt, theta, P, theta_out);
  if (Q)
    for (size_t i = 0; i < nn; i++) Q[i] += dt * P[i];
  for (int a = 0; a < 3; a++) free(Eold[a]);
}
