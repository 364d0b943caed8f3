/*
 * Plain, slow FP64 CPU oracle of the probabilistic VLBM for the Mach 2000 jet.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may build, load or call it.  It shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * Built with `gcc -O2 -ffp-contract=off` (no fast-math, no FMA contraction).
 * Every loop runs over realizations / rows / columns in plain order; nothing is
 * blocked or fused.  Sources followed (paper: "Computing statistical solutions
 * of a Mach 2000 astrophysical jet"):
 *   - Euler fluxes f, g and the ideal-gas EOS: Sec. 2.1, Eqs. (euler),
 *     (fluxF), (fluxG), (eos).
 *   - D2Q5 vector Maxwellians M_1..M_5 and the kinetic speed a: Sec. 2.1,
 *     Eqs. (maxwellians12), (maxwellians34), (maxwellians5); a is re-evaluated
 *     every step to bound the flux-Jacobian spectral radius (Bouchut), with
 *     dt = dx / a_n (Sec. 2.3, CFL statement).
 *   - Blended stream-collide update: Sec. 2.1, Eqs. (vlbm1)-(vlbm5); the u_5
 *     rule is skipped as the paper states.
 *   - Inlet Dirichlet condition, initial condition, outflow and transverse
 *     zero-gradient conditions: Sec. 2.2, Eqs. (inletBC), (rho_inlet_def),
 *     (u0_def), (outletBC), (transverseBC).
 *   - Truncated Karhunen-Loeve inlet perturbation: Sec. 2.3, Eq. (karhunenExp).
 *
 * Readings of points the paper leaves open (the blending parameter and RLMP
 * limiter are only defined in the cited VLBM paper, which is not available):
 *   - theta: convex-split limiter "R-theta".  For face f of cell c with sign
 *     s (+1 when c is the right/upper cell), V(theta) = U_LF + 4 s theta d_f
 *     must keep rho >= eps_rho, p >= eps_p and rho inside the relaxed local
 *     bounds [lo - delta, hi + delta] of c; theta_f = min over both cells.
 *     limiter = 0 gives theta = 0 (first order), limiter = 1 gives theta = 1.
 *     On a face between an interior node and a boundary node only the
 *     interior cell's bounds apply (the boundary node is overwritten by its
 *     boundary condition and is not updated by the scheme).
 *   - Every boundary node carries the equilibria of its nodal state: the
 *     inlet's M_k(u_inlet) (Eq. inletBC) and, for the zero-gradient sides,
 *     M_k of the copied interior nodal state.  They are re-evaluated with the
 *     current a_n whenever a step reads them.
 *   - a_n = kappa * 2 * lambda / (1 - alpha), lambda = max over all nodes of
 *     max(|v1|, |v2|) + sqrt(gamma p / rho).
 *   - Landing on an output time t*: a_n <- max(a_n, dx / (t* - t_n)).
 *   - Nodes x_i = i dx (the inlet column sits at x = 0), y_j = y_min + (j+1/2) dx.
 *   - KL perturbation in the normalised coordinate ybar = y / r_jet with
 *     window W = cos^2(pi ybar / 2); coefficients from Philox4x32-10
 *     (key = seed, counter = (m, block, 0, 0)), U(-1,1) = ((w>>8)+1/2) 2^-23 - 1.
 *   - Initial populations are the equilibria M_k(u_0; a_0).
 *   - Boundary order on the new level: interior update, inlet column
 *     (Dirichlet, all rows), outlet column copy (rows 1..ny-2), then the first
 *     and last rows copy from their inner neighbours (columns 1..nx-1), so the
 *     outlet corners receive the diagonal interior node.
 *
 * Layouts (row-major, x fastest):
 *   u    [4][ny][nx]      conserved (rho, rho v1, rho v2, E)
 *   pops [4][4][ny][nx]   populations u_1..u_4, each a 4-vector
 *   inlet[4][ny]          conserved inlet state per row
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENONPOSITIVE 4
#define ORC_ENONFINITE 5

#define BC_JET 0
#define BC_PERIODIC 1
#define BC_NEUMANN 2
#define BC_TUBE 3 /* zero-gradient columns in x, periodic in y (1-D tests) */

typedef struct {
  int nx, ny;
  double dx;     /* square cells: dx = x_max / nx */
  double y_min;  /* y_j = y_min + (j + 1/2) dx */
} orc_grid;

typedef struct {
  double gamma;
  double alpha;     /* weight of M_5 = alpha u */
  double kappa;     /* safety factor on the kinetic speed */
  int limiter;      /* 0: theta = 0, 1: theta = 1, 2: R-theta */
  double rlmp_rel;  /* relative widening of the local density bounds */
  double rlmp_abs;  /* absolute widening of the local density bounds */
  double eps_pos;   /* positivity floor for rho and p */
  int bc;           /* BC_JET, BC_PERIODIC, BC_NEUMANN or BC_TUBE */
} orc_params;

typedef struct {
  double rho, v1, v2, p;
} orc_prim;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its definition.   */
/* ------------------------------------------------------------------------- */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* 24-bit uniform on the open interval (-1, 1). */
static double orc_uniform_pm1(uint32_t w) {
  return ((double)(w >> 8) + 0.5) * (1.0 / 8388608.0) - 1.0;
}

/* KL coefficients of realization m: Y_k = word k-1, Z_k = word K+k-1 of the
 * Philox stream with counter (m, block, 0, 0), 4 words per block. */
void orc_kl_coefficients(uint64_t seed, int m, int K, double* Y, double* Z) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  int nwords = 2 * K;
  for (int w = 0; w < nwords; ++w) {
    uint32_t ctr[4] = {(uint32_t)m, (uint32_t)(w / 4), 0u, 0u};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    double u = orc_uniform_pm1(out[w % 4]);
    if (w < K)
      Y[w] = u;
    else
      Z[w - K] = u;
  }
}

/* Eq. (karhunenExp): rho' = rho_bar [1 + sum_k amp_k (Y_k cos(k pi yb) +
 * Z_k sin(k pi yb)) W(yb)], amp_k = A k^-p unless overridden, W = cos^2(pi yb/2). */
double orc_kl_density(double ybar, double rho_bar, int K, const double* amp, const double* Y,
                      const double* Z) {
  const double pi = 3.14159265358979323846;
  double s = 0.0;
  for (int k = 1; k <= K; ++k) {
    double arg = (double)k * pi * ybar;
    s = s + amp[k - 1] * (Y[k - 1] * cos(arg) + Z[k - 1] * sin(arg));
  }
  double cw = cos(0.5 * pi * ybar);
  double W = cw * cw;
  return rho_bar * (1.0 + s * W);
}

static void orc_prim_to_cons(const orc_prim* w, double gamma, double q[4]) {
  q[0] = w->rho;
  q[1] = w->rho * w->v1;
  q[2] = w->rho * w->v2;
  q[3] = w->p / (gamma - 1.0) + 0.5 * w->rho * (w->v1 * w->v1 + w->v2 * w->v2);
}

/* Eqs. (inletBC), (rho_inlet_def): inlet state per row j of realization m.
 * amp[k-1] is the amplitude of mode k (A k^-p by default). */
int orc_inlet(const orc_grid* g, double gamma, const orc_prim* jet, const orc_prim* amb, double r_jet,
              int K, const double* amp, uint64_t seed, int m, double* inlet) {
  if (K < 0 || K > 64) return ORC_EINVAL;
  double Y[64], Z[64];
  orc_kl_coefficients(seed, m, K, Y, Z);
  for (int j = 0; j < g->ny; ++j) {
    double y = g->y_min + ((double)j + 0.5) * g->dx;
    orc_prim w;
    if (fabs(y) <= r_jet) {
      w.rho = orc_kl_density(y / r_jet, jet->rho, K, amp, Y, Z);
      w.v1 = jet->v1;
      w.v2 = 0.0;
      w.p = jet->p;
    } else {
      w = *amb;
      w.v1 = 0.0;
      w.v2 = 0.0;
    }
    double q[4];
    orc_prim_to_cons(&w, gamma, q);
    for (int c = 0; c < 4; ++c) inlet[c * g->ny + j] = q[c];
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Primitive recovery (Eq. eos), fluxes (Eqs. fluxF, fluxG), Maxwellians.    */
/* ------------------------------------------------------------------------- */

static void orc_primitive(const double q[4], double gamma, double* v1, double* v2, double* p) {
  *v1 = q[1] / q[0];
  *v2 = q[2] / q[0];
  *p = (gamma - 1.0) * (q[3] - 0.5 * q[0] * ((*v1) * (*v1) + (*v2) * (*v2)));
}

static void orc_fluxes(const double q[4], double gamma, double f[4], double gf[4]) {
  double v1, v2, p;
  orc_primitive(q, gamma, &v1, &v2, &p);
  f[0] = q[1];
  f[1] = q[1] * v1 + p;
  f[2] = q[1] * v2;
  f[3] = (q[3] + p) * v1;
  gf[0] = q[2];
  gf[1] = q[1] * v2;
  gf[2] = q[2] * v2 + p;
  gf[3] = (q[3] + p) * v2;
}

/* M_k(q; a), k = 1..4, Eqs. (maxwellians12), (maxwellians34). */
static void orc_maxwellian(const double q[4], double gamma, double alpha, double inv2a, int k,
                           double M[4]) {
  double f[4], gf[4];
  orc_fluxes(q, gamma, f, gf);
  double c1 = (1.0 - alpha) / 4.0;
  for (int c = 0; c < 4; ++c) {
    double F = (k < 2) ? f[c] : gf[c];
    double sgn = (k % 2 == 0) ? 1.0 : -1.0;
    M[c] = c1 * q[c] + sgn * (F * inv2a);
  }
}

/* ------------------------------------------------------------------------- */
/* Kinetic speed a_n (Sec. 2.1 Bouchut criterion, Sec. 2.3 CFL).             */
/* ------------------------------------------------------------------------- */

int orc_kinetic_speed(const orc_grid* g, const orc_params* P, const double* u, double* a_out) {
  size_t n = (size_t)g->nx * g->ny;
  double lam = 0.0;
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      size_t id = (size_t)j * g->nx + i;
      double q[4] = {u[id], u[n + id], u[2 * n + id], u[3 * n + id]};
      double v1, v2, p;
      orc_primitive(q, P->gamma, &v1, &v2, &p);
      if (!(q[0] > 0.0) || !(p > 0.0)) return ORC_ENONPOSITIVE;
      double c = sqrt(P->gamma * p / q[0]);
      double vmax = fabs(v1) > fabs(v2) ? fabs(v1) : fabs(v2);
      double l = vmax + c;
      if (!isfinite(l)) return ORC_ENONFINITE;
      if (l > lam) lam = l;
    }
  *a_out = P->kappa * 2.0 * lam / (1.0 - P->alpha);
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Initial condition, Eq. (u0_def), with equilibrium populations.            */
/* ------------------------------------------------------------------------- */

int orc_init_state(const orc_grid* g, const orc_params* P, const double* inlet, const orc_prim* amb,
                   double* u, double* pops, double* a0) {
  size_t n = (size_t)g->nx * g->ny;
  double qa[4];
  orc_prim wa = *amb;
  wa.v1 = 0.0;
  wa.v2 = 0.0;
  orc_prim_to_cons(&wa, P->gamma, qa);
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      size_t id = (size_t)j * g->nx + i;
      for (int c = 0; c < 4; ++c) u[c * n + id] = (i == 0) ? inlet[c * g->ny + j] : qa[c];
    }
  int st = orc_kinetic_speed(g, P, u, a0);
  if (st) return st;
  double inv2a = 0.5 / *a0;
  for (size_t id = 0; id < n; ++id) {
    double q[4] = {u[id], u[n + id], u[2 * n + id], u[3 * n + id]};
    for (int k = 0; k < 4; ++k) {
      double M[4];
      orc_maxwellian(q, P->gamma, P->alpha, inv2a, k, M);
      for (int c = 0; c < 4; ++c) pops[(size_t)(k * 4 + c) * n + id] = M[c];
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Limiter R-theta for one face seen from one cell.                          */
/* ------------------------------------------------------------------------- */

/* Largest theta in [0,1] such that V(theta) = U0 + theta D keeps
 * rho >= max(eps_r, lo_b), rho <= hi_b and p >= eps_p.  The admissible set is
 * convex, so the feasible thetas form an interval starting at 0. */
static double orc_theta_star(const double U0[4], const double D[4], double lo_b, double hi_b,
                             double eps_r, double eps_p, double gamma) {
  double th = 1.0;
  double lower = eps_r > lo_b ? eps_r : lo_b;
  if (D[0] < 0.0) {
    double lim = (U0[0] - lower) / (-D[0]);
    if (lim < th) th = lim;
  } else if (D[0] > 0.0) {
    double lim = (hi_b - U0[0]) / D[0];
    if (lim < th) th = lim;
  }
  if (th < 0.0) th = 0.0;
  /* q(t) = rho(t) E(t) - |m(t)|^2 / 2 - eps_p rho(t) / (gamma - 1) */
  double kk = eps_p / (gamma - 1.0);
  double C = U0[0] * U0[3] - 0.5 * (U0[1] * U0[1] + U0[2] * U0[2]) - kk * U0[0];
  double B = U0[0] * D[3] + D[0] * U0[3] - (U0[1] * D[1] + U0[2] * D[2]) - kk * D[0];
  double A = D[0] * D[3] - 0.5 * (D[1] * D[1] + D[2] * D[2]);
  double qth = C + th * (B + th * A);
  if (qth >= 0.0) return th;
  if (C <= 0.0) return 0.0;
  double r;
  if (A == 0.0) {
    r = -C / B;
  } else {
    double disc = B * B - 4.0 * A * C;
    if (disc < 0.0) disc = 0.0;
    double sq = sqrt(disc);
    double Q = -0.5 * (B + (B >= 0.0 ? sq : -sq));
    if (Q == 0.0) return 0.0;
    double r1 = Q / A;
    double r2 = C / Q;
    r = -1.0;
    if (r1 > 0.0) r = r1;
    if (r2 > 0.0 && (r < 0.0 || r2 < r)) r = r2;
    if (r < 0.0) return 0.0;
  }
  if (r > th) r = th;
  if (r < 0.0) r = 0.0;
  return r;
}

/* Exported for the limiter's own pins. */
double orc_theta_star_export(const double U0[4], const double D[4], double lo_b, double hi_b,
                             double eps_r, double eps_p, double gamma) {
  return orc_theta_star(U0, D, lo_b, hi_b, eps_r, eps_p, gamma);
}

/* ------------------------------------------------------------------------- */
/* One blended stream-collide step, Eqs. (vlbm1)-(vlbm5), plus boundaries.   */
/* ------------------------------------------------------------------------- */

static int orc_is_boundary(const orc_grid* g, const orc_params* P, int i, int j) {
  if (P->bc == BC_PERIODIC) return 0;
  if (P->bc == BC_TUBE) return i == 0 || i == g->nx - 1;
  return i == 0 || i == g->nx - 1 || j == 0 || j == g->ny - 1;
}

static size_t orc_idx(const orc_grid* g, const orc_params* P, int i, int j) {
  if (P->bc == BC_PERIODIC) i = (i + g->nx) % g->nx;
  if (P->bc == BC_PERIODIC || P->bc == BC_TUBE) j = (j + g->ny) % g->ny;
  return (size_t)j * g->nx + i;
}

static void orc_load(const double* u, size_t n, size_t id, double q[4]) {
  for (int c = 0; c < 4; ++c) q[c] = u[c * n + id];
}

static void orc_load_pop(const double* pops, size_t n, size_t id, int k, double q[4]) {
  for (int c = 0; c < 4; ++c) q[c] = pops[(size_t)(k * 4 + c) * n + id];
}

/* Zero-gradient copy of the nodal state (Eqs. outletBC, transverseBC); the
 * boundary populations are set to the equilibria of the copied state. */
static void orc_copy_node(double* u, double* pops, size_t n, size_t dst, size_t src, double gamma,
                          double alpha, double inv2a) {
  double q[4];
  for (int c = 0; c < 4; ++c) {
    u[c * n + dst] = u[c * n + src];
    q[c] = u[c * n + src];
  }
  for (int k = 0; k < 4; ++k) {
    double M[4];
    orc_maxwellian(q, gamma, alpha, inv2a, k, M);
    for (int c = 0; c < 4; ++c) pops[(size_t)(k * 4 + c) * n + dst] = M[c];
  }
}

/* Advances one realization by one step with kinetic speed a.
 * inlet may be NULL unless bc == BC_JET.  Work arrays are allocated here. */
int orc_step(const orc_grid* g, const orc_params* P, double a, const double* inlet, const double* u,
             const double* pops, double* u_new, double* pops_new) {
  const int nx = g->nx, ny = g->ny;
  const size_t n = (size_t)nx * ny;
  if (nx < 3 || ny < 3 || !(a > 0.0)) return ORC_EINVAL;
  const double inv2a = 0.5 / a;
  const double gamma = P->gamma, alpha = P->alpha;

  double* ulf = (double*)calloc(4 * n, sizeof(double));     /* U_LF per node */
  double* bnd = (double*)calloc(4 * n, sizeof(double));     /* lo_b, hi_b, eps_r, eps_p */
  double* thx = (double*)calloc(n, sizeof(double));         /* theta at face (i+1/2, j) */
  double* thy = (double*)calloc(n, sizeof(double));         /* theta at face (i, j+1/2) */
  double* dx_ = (double*)calloc(4 * n, sizeof(double));     /* d at face (i+1/2, j) */
  double* dy_ = (double*)calloc(4 * n, sizeof(double));     /* d at face (i, j+1/2) */
  if (!ulf || !bnd || !thx || !thy || !dx_ || !dy_) {
    free(ulf); free(bnd); free(thx); free(thy); free(dx_); free(dy_);
    return ORC_ENOMEM;
  }

  /* Step 3: Lax-Friedrichs part U_LF = alpha u_c + M1(u_W) + M2(u_E) + M3(u_S) + M4(u_N),
   * and the relaxed local bounds of every non-boundary node. */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (orc_is_boundary(g, P, i, j)) continue;
      size_t c = orc_idx(g, P, i, j);
      size_t W = orc_idx(g, P, i - 1, j), E = orc_idx(g, P, i + 1, j);
      size_t S = orc_idx(g, P, i, j - 1), N = orc_idx(g, P, i, j + 1);
      double qc[4], qW[4], qE[4], qS[4], qN[4];
      orc_load(u, n, c, qc);
      orc_load(u, n, W, qW);
      orc_load(u, n, E, qE);
      orc_load(u, n, S, qS);
      orc_load(u, n, N, qN);
      double M1W[4], M2E[4], M3S[4], M4N[4];
      orc_maxwellian(qW, gamma, alpha, inv2a, 0, M1W);
      orc_maxwellian(qE, gamma, alpha, inv2a, 1, M2E);
      orc_maxwellian(qS, gamma, alpha, inv2a, 2, M3S);
      orc_maxwellian(qN, gamma, alpha, inv2a, 3, M4N);
      double U[4];
      for (int q = 0; q < 4; ++q) {
        U[q] = alpha * qc[q] + M1W[q] + M2E[q] + M3S[q] + M4N[q];
        ulf[q * n + c] = U[q];
      }
      double lo = qc[0], hi = qc[0];
      double rs[5] = {qW[0], qE[0], qS[0], qN[0], U[0]};
      for (int r = 0; r < 5; ++r) {
        if (rs[r] < lo) lo = rs[r];
        if (rs[r] > hi) hi = rs[r];
      }
      double delta = P->rlmp_rel * (hi - lo) + P->rlmp_abs;
      double v1, v2, pLF;
      orc_primitive(U, gamma, &v1, &v2, &pLF);
      bnd[0 * n + c] = lo - delta;
      bnd[1 * n + c] = hi + delta;
      bnd[2 * n + c] = P->eps_pos < U[0] ? P->eps_pos : U[0];
      bnd[3 * n + c] = P->eps_pos < pLF ? P->eps_pos : pLF;
    }

  /* Step 4: face corrections d_f and blending parameters theta_f. */
  for (int dir = 0; dir < 2; ++dir)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int iR = dir == 0 ? i + 1 : i, jR = dir == 0 ? j : j + 1;
        if (iR >= nx && P->bc != BC_PERIODIC) continue;
        if (jR >= ny && P->bc != BC_PERIODIC && P->bc != BC_TUBE) continue;
        size_t L = orc_idx(g, P, i, j), R = orc_idx(g, P, iR, jR);
        double qL[4], qR[4], pL[4], pR[4], Mo[4], Mi[4], d[4];
        orc_load(u, n, L, qL);
        orc_load(u, n, R, qR);
        int kout = dir == 0 ? 0 : 2, kin = dir == 0 ? 1 : 3;
        orc_load_pop(pops, n, L, kout, pL);
        orc_load_pop(pops, n, R, kin, pR);
        orc_maxwellian(qL, gamma, alpha, inv2a, kout, Mo);
        orc_maxwellian(qR, gamma, alpha, inv2a, kin, Mi);
        int bL = orc_is_boundary(g, P, i, j), bR = orc_is_boundary(g, P, iR, jR);
        /* Boundary nodes carry the equilibria of their imposed (inlet) or
         * copied (zero-gradient) nodal state at the current a_n. */
        if (bL)
          for (int q = 0; q < 4; ++q) pL[q] = Mo[q];
        if (bR)
          for (int q = 0; q < 4; ++q) pR[q] = Mi[q];
        for (int q = 0; q < 4; ++q) d[q] = (Mo[q] - pL[q]) - (Mi[q] - pR[q]);
        double th;
        if (bL && bR) {
          th = 0.0; /* no interior node uses this face */
        } else if (P->limiter == 0) {
          th = 0.0;
        } else if (P->limiter == 1) {
          th = 1.0;
        } else {
          /* theta_f = min of theta*_c(f) over the interior cells of the face;
           * a boundary node is not updated by the scheme and sets no bound. */
          double UL[4], UR[4], DL[4], DR[4];
          for (int q = 0; q < 4; ++q) {
            UL[q] = ulf[q * n + L];
            UR[q] = ulf[q * n + R];
            DL[q] = -4.0 * d[q];
            DR[q] = 4.0 * d[q];
          }
          double tL = bL ? 1.0 : orc_theta_star(UL, DL, bnd[L], bnd[n + L], bnd[2 * n + L], bnd[3 * n + L], gamma);
          double tR = bR ? 1.0 : orc_theta_star(UR, DR, bnd[R], bnd[n + R], bnd[2 * n + R], bnd[3 * n + R], gamma);
          th = tL < tR ? tL : tR;
        }
        double* dd = dir == 0 ? dx_ : dy_;
        double* tt = dir == 0 ? thx : thy;
        tt[L] = th;
        for (int q = 0; q < 4; ++q) dd[q * n + L] = d[q];
      }

  /* Step 5: populations by Eqs. (vlbm1)-(vlbm4) and the macroscopic state by
   * Eq. (vlbm5), written literally (sum of the new populations, alpha u, and
   * the four theta-weighted non-equilibrium terms of the cell itself). */
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (orc_is_boundary(g, P, i, j)) continue;
      size_t c = orc_idx(g, P, i, j);
      size_t W = orc_idx(g, P, i - 1, j), E = orc_idx(g, P, i + 1, j);
      size_t S = orc_idx(g, P, i, j - 1), N = orc_idx(g, P, i, j + 1);
      double th_w = thx[W], th_e = thx[c], th_s = thy[S], th_n = thy[c];
      double qc[4], qW[4], qE[4], qS[4], qN[4];
      orc_load(u, n, c, qc);
      orc_load(u, n, W, qW);
      orc_load(u, n, E, qE);
      orc_load(u, n, S, qS);
      orc_load(u, n, N, qN);
      double M1W[4], M2E[4], M3S[4], M4N[4];
      orc_maxwellian(qW, gamma, alpha, inv2a, 0, M1W);
      orc_maxwellian(qE, gamma, alpha, inv2a, 1, M2E);
      orc_maxwellian(qS, gamma, alpha, inv2a, 2, M3S);
      orc_maxwellian(qN, gamma, alpha, inv2a, 3, M4N);
      double p1W[4], p2E[4], p3S[4], p4N[4];
      orc_load_pop(pops, n, W, 0, p1W);
      orc_load_pop(pops, n, E, 1, p2E);
      orc_load_pop(pops, n, S, 2, p3S);
      orc_load_pop(pops, n, N, 3, p4N);
      for (int q = 0; q < 4; ++q) {
        if (orc_is_boundary(g, P, i - 1, j)) p1W[q] = M1W[q];
        if (orc_is_boundary(g, P, i + 1, j)) p2E[q] = M2E[q];
        if (orc_is_boundary(g, P, i, j - 1)) p3S[q] = M3S[q];
        if (orc_is_boundary(g, P, i, j + 1)) p4N[q] = M4N[q];
      }
      double M1c[4], M2c[4], M3c[4], M4c[4], p1c[4], p2c[4], p3c[4], p4c[4];
      orc_maxwellian(qc, gamma, alpha, inv2a, 0, M1c);
      orc_maxwellian(qc, gamma, alpha, inv2a, 1, M2c);
      orc_maxwellian(qc, gamma, alpha, inv2a, 2, M3c);
      orc_maxwellian(qc, gamma, alpha, inv2a, 3, M4c);
      orc_load_pop(pops, n, c, 0, p1c);
      orc_load_pop(pops, n, c, 1, p2c);
      orc_load_pop(pops, n, c, 2, p3c);
      orc_load_pop(pops, n, c, 3, p4c);
      for (int q = 0; q < 4; ++q) {
        double n1 = M1W[q] + th_w * (M1W[q] - p1W[q]);
        double n2 = M2E[q] + th_e * (M2E[q] - p2E[q]);
        double n3 = M3S[q] + th_s * (M3S[q] - p3S[q]);
        double n4 = M4N[q] + th_n * (M4N[q] - p4N[q]);
        pops_new[(size_t)(0 * 4 + q) * n + c] = n1;
        pops_new[(size_t)(1 * 4 + q) * n + c] = n2;
        pops_new[(size_t)(2 * 4 + q) * n + c] = n3;
        pops_new[(size_t)(3 * 4 + q) * n + c] = n4;
        u_new[q * n + c] = n1 + n2 + n3 + n4 + alpha * qc[q] - th_w * (M2c[q] - p2c[q]) -
                           th_e * (M1c[q] - p1c[q]) - th_s * (M4c[q] - p4c[q]) - th_n * (M3c[q] - p3c[q]);
      }
    }

  /* Step 6: boundaries on the new level. */
  if (P->bc == BC_JET || P->bc == BC_NEUMANN) {
    for (int j = 0; j < ny; ++j) {
      size_t id = (size_t)j * nx;
      if (P->bc == BC_JET) {
        double q[4];
        for (int c = 0; c < 4; ++c) q[c] = inlet[c * ny + j];
        for (int c = 0; c < 4; ++c) u_new[c * n + id] = q[c];
        for (int k = 0; k < 4; ++k) {
          double M[4];
          orc_maxwellian(q, gamma, alpha, inv2a, k, M);
          for (int c = 0; c < 4; ++c) pops_new[(size_t)(k * 4 + c) * n + id] = M[c];
        }
      } else if (j >= 1 && j <= ny - 2) {
        orc_copy_node(u_new, pops_new, n, id, id + 1, gamma, alpha, inv2a);
      }
    }
    for (int j = 1; j <= ny - 2; ++j) {
      size_t id = (size_t)j * nx + (nx - 1);
      orc_copy_node(u_new, pops_new, n, id, id - 1, gamma, alpha, inv2a);
    }
    int i0 = (P->bc == BC_JET) ? 1 : 0;
    for (int i = i0; i < nx; ++i) {
      orc_copy_node(u_new, pops_new, n, (size_t)i, (size_t)nx + i, gamma, alpha, inv2a);
      orc_copy_node(u_new, pops_new, n, (size_t)(ny - 1) * nx + i, (size_t)(ny - 2) * nx + i, gamma,
                    alpha, inv2a);
    }
  }

  if (P->bc == BC_TUBE) {
    for (int j = 0; j < ny; ++j) {
      size_t id = (size_t)j * nx;
      orc_copy_node(u_new, pops_new, n, id, id + 1, gamma, alpha, inv2a);
      orc_copy_node(u_new, pops_new, n, id + nx - 1, id + nx - 2, gamma, alpha, inv2a);
    }
  }

  free(ulf); free(bnd); free(thx); free(thy); free(dx_); free(dy_);

  /* Positivity and finiteness of the new level. */
  for (size_t id = 0; id < n; ++id) {
    double q[4] = {u_new[id], u_new[n + id], u_new[2 * n + id], u_new[3 * n + id]};
    double v1, v2, p;
    orc_primitive(q, gamma, &v1, &v2, &p);
    if (!isfinite(q[0]) || !isfinite(q[1]) || !isfinite(q[2]) || !isfinite(q[3])) return ORC_ENONFINITE;
    if (!(q[0] > 0.0) || !(p > 0.0)) return ORC_ENONPOSITIVE;
  }
  return ORC_OK;
}

/* Moments (rho, v1, v2, p) of a conserved field, Eq. (eos). */
void orc_moments(const orc_grid* g, double gamma, const double* u, double* rho, double* v1,
                 double* v2, double* p) {
  size_t n = (size_t)g->nx * g->ny;
  for (size_t id = 0; id < n; ++id) {
    double q[4] = {u[id], u[n + id], u[2 * n + id], u[3 * n + id]};
    rho[id] = q[0];
    orc_primitive(q, gamma, &v1[id], &v2[id], &p[id]);
  }
}

/* Runs realizations m0 .. m0+count-1 of the jet from t = 0: either nsteps
 * steps (t_end < 0) or until t_end with the landing rule (nsteps is then a
 * cap).  Outputs per realization r = m - m0:
 *   u_out [r][4][ny][nx], pops_out [r][16][ny][nx] (may be NULL),
 *   t_out[r], steps_out[r]. */
int orc_run_jet(const orc_grid* g, const orc_params* P, const orc_prim* jet, const orc_prim* amb,
                double r_jet, int K, const double* amp, uint64_t seed, int m0, int count, int nsteps,
                double t_end, double* u_out, double* pops_out, double* t_out, long long* steps_out) {
  size_t n = (size_t)g->nx * g->ny;
  double* inlet = (double*)malloc(4 * (size_t)g->ny * sizeof(double));
  double* u0 = (double*)malloc(4 * n * sizeof(double));
  double* u1 = (double*)malloc(4 * n * sizeof(double));
  double* f0 = (double*)malloc(16 * n * sizeof(double));
  double* f1 = (double*)malloc(16 * n * sizeof(double));
  int st = ORC_OK;
  if (!inlet || !u0 || !u1 || !f0 || !f1) st = ORC_ENOMEM;
  for (int r = 0; r < count && st == ORC_OK; ++r) {
    st = orc_inlet(g, P->gamma, jet, amb, r_jet, K, amp, seed, m0 + r, inlet);
    if (st) break;
    double a;
    st = orc_init_state(g, P, inlet, amb, u0, f0, &a);
    if (st) break;
    double t = 0.0;
    long long s = 0;
    while (s < nsteps) {
      if (t_end >= 0.0 && t >= t_end) break;
      st = orc_kinetic_speed(g, P, u0, &a);
      if (st) break;
      int landing = 0;
      if (t_end >= 0.0) {
        double a_land = g->dx / (t_end - t);
        if (a_land >= a) {
          a = a_land;
          landing = 1;
        }
      }
      st = orc_step(g, P, a, inlet, u0, f0, u1, f1);
      if (st) break;
      t = landing ? t_end : t + g->dx / a;
      ++s;
      double* tmp = u0; u0 = u1; u1 = tmp;
      tmp = f0; f0 = f1; f1 = tmp;
    }
    if (st) break;
    memcpy(u_out + (size_t)r * 4 * n, u0, 4 * n * sizeof(double));
    if (pops_out) memcpy(pops_out + (size_t)r * 16 * n, f0, 16 * n * sizeof(double));
    t_out[r] = t;
    steps_out[r] = s;
  }
  free(inlet); free(u0); free(u1); free(f0); free(f1);
  return st;
}
