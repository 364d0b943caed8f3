// Discrete adjoint of the FP64 VLBM step (Sec. 2.1-2.3): gradients of an
// ensemble observable J = (1/M) sum_m sum_x w(x) rho_m(x, t_N) with respect
// to the per-mode amplitudes a_k of the KL inlet perturbation
// (Eq. (karhunenExp)).
//
// The reverse of one step s (u^s, pops^s, a_s -> u^{s+1}, pops^{s+1}) takes
// the adjoints of the new state and returns those of the old one, in the
// order the forward step computes (reversed):
//   F1 (nodes)  Maxwellians M_k(u_x; a_s), U_LF, the relaxed bounds and the
//               sources of their minimum and maximum (recomputed);
//   F2 (faces)  d_f, theta_L, theta_R, theta_f (recomputed; the same branches
//               as the forward step: same arithmetic, no FMA contraction);
//   R0 (inlet)  the inlet column of u^{s+1} is the Dirichlet datum: its
//               adjoint is accumulated for the amplitude gradient;
//   R1 (cells)  adjoint of u^{s+1} gathered over its zero-gradient copies, and
//               of the four new populations n_k (Eqs. (vlbm1)-(vlbm5));
//   R2 (faces)  theta_f-bar from the two cells using the face, through the
//               limiter's taken branch (min of theta_L, theta_R; the linear
//               density bounds or the root of the pressure quadratic) to
//               U_LF-bar, d-bar and the bounds' adjoint of the selected side;
//   R3 (cells)  bounds -> lo, hi and the floors; U_LF-bar of each cell;
//   R4 (nodes)  every use of M_k(u_x) and of the populations read at x,
//               gathered; through the Maxwellian to u_x, and the share of
//               d J / d(1/2a_s);
//   R5 (realization)  a_s = kappa 2 lambda / (1 - alpha), lambda at the first
//               maximum of max(|v1|, |v2|) + c in row-major order.
// Every reduction runs in a fixed order; every adjoint is gathered by the
// thread that owns it (no atomics), so a gradient is reproducible bit for
// bit.  Piecewise-smooth operations (argmax, min, max, the limiter's
// branches) are differentiated on the branch the forward step took, with the
// forward step's tie rules.
#include "vlbm_f64_math.cuh"
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

using namespace f64;

constexpr int kT = 256;

// per-realization scratch planes (FP64)
enum : int {
  kM = 0,    // 16: M_k(u_x; a_s), plane kM + 4 k + c
  kU = 16,   // 4: U_LF (interior nodes)
  kB = 20,   // 4: lo - delta, hi + delta, eps_rho, eps_p
  kDX = 24,  // 4: d of the face (x, x + 1)
  kTX = 28,  // 3: theta_L, theta_R, theta_f of that face
  kDY = 31,  // 4: d of the face (x, x + row)
  kTY = 35,  // 3
  kNB = 38,  // 16: adjoint of the new population n_k of cell x
  kUE = 54,  // 4: adjoint of u^{s+1}_x with its copies gathered
  kFX = 58,  // 4: d-bar of the face (x, x + 1)
  kUX = 62,  // 4: U_LF-bar sent by that face to its selected side
  kGX = 66,  // 4: bounds-bar sent to the selected side
  kFY = 70,  // 4
  kUY = 74,  // 4
  kGY = 78,  // 4
  kUB = 82,  // 4: U_LF-bar of interior cell x
  kLH = 86,  // 2: lo-bar, hi-bar
  kHB = 88,  // 1: node share of d J / d(1/2a)
  kPlanes = 89
};
// int planes: 0 lo source | hi source << 4; 1 selected side of the x face | of the y face << 2
constexpr int kIntPlanes = 2;

struct Geo {
  int nx, ny, nxp;
  size_t plane;
  int M;
};

__device__ __forceinline__ bool node_of(const Geo& g, int& i, int& j) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (long long)g.nx * g.ny) return false;
  j = (int)(n / g.nx);
  i = (int)(n % g.nx);
  return true;
}

__device__ __forceinline__ bool interior(const Geo& g, int i, int j) {
  return i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2;
}

__device__ __forceinline__ void ld4(const double* p, size_t plane, size_t id, double q[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) q[c] = p[c * plane + id];
}

// M_k(q; a) as the FP64 step evaluates it: c1 q + f h (k = 0), c1 q - f h (1),
// c1 q + g h (2), c1 q - g h (3).
__device__ __forceinline__ void maxwellians(const double q[4], double gamma, double c1, double h, double M[4][4]) {
  double f[4], g[4];
  fluxes(q, gamma, f, g);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    M[0][c] = c1 * q[c] + f[c] * h;
    M[1][c] = c1 * q[c] - f[c] * h;
    M[2][c] = c1 * q[c] + g[c] * h;
    M[3][c] = c1 * q[c] - g[c] * h;
  }
}

// Adjoint of p = (gamma - 1)(q3 - q0 (v1^2 + v2^2) / 2), v = m / q0, added to qb.
__device__ __forceinline__ void pressure_bwd(const double q[4], double gamma, double pb, double qb[4]) {
  const double v1 = q[1] / q[0], v2 = q[2] / q[0];
  qb[3] += (gamma - 1.0) * pb;
  const double tb = -(gamma - 1.0) * pb;  // adjoint of q0 (v1^2 + v2^2) / 2
  qb[0] += tb * 0.5 * (v1 * v1 + v2 * v2);
  const double v1b = tb * q[0] * v1, v2b = tb * q[0] * v2;
  qb[1] += v1b / q[0];
  qb[2] += v2b / q[0];
  qb[0] -= (v1b * v1 + v2b * v2) / q[0];
}

// Adjoint of the Maxwellians M_k(q; h) of one node for given M-bar: adds to qb
// and returns the node's share of d/dh.
__device__ __forceinline__ double maxwellians_bwd(const double q[4], double gamma, double c1, double h,
                                                  const double Mb[4][4], double qb[4]) {
  double f[4], g[4];
  fluxes(q, gamma, f, g);
  double Fb[4], Gb[4], hb = 0.0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    qb[c] += c1 * (Mb[0][c] + Mb[1][c] + Mb[2][c] + Mb[3][c]);
    const double fx = Mb[0][c] - Mb[1][c], gy = Mb[2][c] - Mb[3][c];
    Fb[c] = fx * h;
    Gb[c] = gy * h;
    hb += f[c] * fx + g[c] * gy;
  }
  const double v1 = q[1] / q[0], v2 = q[2] / q[0];
  double pv;
  {
    double a1, a2;
    primitive(q, gamma, a1, a2, pv);
  }
  double v1b = 0.0, v2b = 0.0, pb = 0.0;
  // f = (q1, q1 v1 + p, q1 v2, (q3 + p) v1)
  qb[1] += Fb[0];
  qb[1] += Fb[1] * v1;
  v1b += Fb[1] * q[1];
  pb += Fb[1];
  qb[1] += Fb[2] * v2;
  v2b += Fb[2] * q[1];
  qb[3] += Fb[3] * v1;
  pb += Fb[3] * v1;
  v1b += Fb[3] * (q[3] + pv);
  // g = (q2, q1 v2, q2 v2 + p, (q3 + p) v2)
  qb[2] += Gb[0];
  qb[1] += Gb[1] * v2;
  v2b += Gb[1] * q[1];
  qb[2] += Gb[2] * v2;
  v2b += Gb[2] * q[2];
  pb += Gb[2];
  qb[3] += Gb[3] * v2;
  pb += Gb[3] * v2;
  v2b += Gb[3] * (q[3] + pv);
  qb[1] += v1b / q[0];
  qb[2] += v2b / q[0];
  qb[0] -= (v1b * v1 + v2b * v2) / q[0];
  pressure_bwd(q, gamma, pb, qb);
  return hb;
}

// Adjoint of theta_star (the branch the forward evaluation takes) for the
// output adjoint tb: adds to U0b, Db and the adjoints of lo_b, hi_b, eps_r, eps_p.
__device__ void theta_star_bwd(const double U0[4], const double D[4], double lo_b, double hi_b, double eps_r,
                               double eps_p, double gamma, double tb, double U0b[4], double Db[4], double Bb[4]) {
  // forward replay
  double th = 1.0;
  int th_src = 0;  // 0 constant, 1 density floor, 2 density ceiling
  const bool lower_eps = eps_r > lo_b;
  const double lower = lower_eps ? eps_r : lo_b;
  if (D[0] < 0.0) {
    const double lim = (U0[0] - lower) / (-D[0]);
    if (lim < th) {
      th = lim;
      th_src = 1;
    }
  } else if (D[0] > 0.0) {
    const double lim = (hi_b - U0[0]) / D[0];
    if (lim < th) {
      th = lim;
      th_src = 2;
    }
  }
  if (th < 0.0) {
    th = 0.0;
    th_src = 0;
  }
  const double kk = eps_p / (gamma - 1.0);
  const double C = U0[0] * U0[3] - 0.5 * (U0[1] * U0[1] + U0[2] * U0[2]) - kk * U0[0];
  const double B = U0[0] * D[3] + D[0] * U0[3] - (U0[1] * D[1] + U0[2] * D[2]) - kk * D[0];
  const double A = D[0] * D[3] - 0.5 * (D[1] * D[1] + D[2] * D[2]);
  const double qth = C + th * (B + th * A);
  double thb = 0.0;  // adjoint of th (the bound branch)
  double Cb = 0.0, Bqb = 0.0, Ab = 0.0;
  if (qth >= 0.0) {
    thb = tb;
  } else if (C <= 0.0) {
    // theta = 0: constant
  } else {
    int r_src = 0;  // 1 linear root, 2 Q / A, 3 C / Q
    double r = 0.0, sq = 0.0, Q = 0.0;
    bool zero = false, disc_pos = false;
    if (A == 0.0) {
      r = -C / B;
      r_src = 1;
    } else {
      double disc = B * B - 4.0 * A * C;
      if (disc < 0.0) disc = 0.0;
      disc_pos = disc > 0.0;
      sq = sqrt(disc);
      Q = -0.5 * (B + (B >= 0.0 ? sq : -sq));
      if (Q == 0.0) {
        zero = true;
      } else {
        const double r1 = Q / A, r2 = C / Q;
        r = -1.0;
        if (r1 > 0.0) {
          r = r1;
          r_src = 2;
        }
        if (r2 > 0.0 && (r < 0.0 || r2 < r)) {
          r = r2;
          r_src = 3;
        }
        if (r < 0.0) zero = true;
      }
    }
    if (!zero) {
      if (r > th) {
        thb = tb;  // clamped to the bound branch
      } else if (r < 0.0) {
        // clamped to 0
      } else {
        double Qb = 0.0;
        if (r_src == 1) {
          Cb += -tb / B;
          Bqb += tb * C / (B * B);
        } else if (r_src == 2) {
          Qb += tb / A;
          Ab += -tb * Q / (A * A);
        } else if (r_src == 3) {
          Cb += tb / Q;
          Qb += -tb * C / (Q * Q);
        }
        if (Qb != 0.0) {
          // Q = -(B + sign(B) sq) / 2, sq = sqrt(disc), disc = B^2 - 4 A C (clamped at 0)
          Bqb += -0.5 * Qb;
          const double sqb = -0.5 * Qb * (B >= 0.0 ? 1.0 : -1.0);
          if (disc_pos) {
            const double db = sqb * 0.5 / sq;
            Bqb += db * 2.0 * B;
            Ab += -db * 4.0 * C;
            Cb += -db * 4.0 * A;
          }
        }
      }
    }
  }
  // th: the bound branch
  if (thb != 0.0) {
    if (th_src == 1) {
      // th = (U0 - lower) / (-D0)
      U0b[0] += thb / (-D[0]);
      const double lb = -thb / (-D[0]);
      if (lower_eps)
        Bb[2] += lb;
      else
        Bb[0] += lb;
      Db[0] += thb * (U0[0] - lower) / (D[0] * D[0]);
    } else if (th_src == 2) {
      // th = (hi_b - U0) / D0
      Bb[1] += thb / D[0];
      U0b[0] += -thb / D[0];
      Db[0] += -thb * (hi_b - U0[0]) / (D[0] * D[0]);
    }
  }
  // C, B, A -> U0, D, kk
  double kkb = 0.0;
  if (Cb != 0.0) {
    U0b[0] += Cb * (U0[3] - kk);
    U0b[3] += Cb * U0[0];
    U0b[1] += -Cb * U0[1];
    U0b[2] += -Cb * U0[2];
    kkb += -Cb * U0[0];
  }
  if (Bqb != 0.0) {
    U0b[0] += Bqb * D[3];
    Db[3] += Bqb * U0[0];
    Db[0] += Bqb * (U0[3] - kk);
    U0b[3] += Bqb * D[0];
    U0b[1] += -Bqb * D[1];
    Db[1] += -Bqb * U0[1];
    U0b[2] += -Bqb * D[2];
    Db[2] += -Bqb * U0[2];
    kkb += -Bqb * D[0];
  }
  if (Ab != 0.0) {
    Db[0] += Ab * D[3];
    Db[3] += Ab * D[0];
    Db[1] += -Ab * D[1];
    Db[2] += -Ab * D[2];
  }
  Bb[3] += kkb / (gamma - 1.0);
}

struct AdjArgs {
  Geo g;
  double gamma, alpha, c1, kappa, rel, absb, eps;
  int limiter;
  const double* state;     // [M][20][plane]: u (4), populations (16) at step s
  const RealState* rs;     // [M] at step s (a_s, 1/2a_s)
  const double* ain;       // [M][20][plane]: adjoint of u^{s+1}, populations^{s+1}
  double* aout;            // [M][20][plane]: adjoint of u^s, populations^s
  double* scr;             // [M][kPlanes][plane]
  int* iscr;               // [M][kIntPlanes][plane]
  double* inlet_acc;       // [M][ny]: adjoint of the inlet density, summed over steps
  double jet_u, y_min, dx, r_jet;
};

__device__ __forceinline__ const double* st_of(const AdjArgs& A, int m) {
  return A.state + (size_t)m * 20 * A.g.plane;
}
__device__ __forceinline__ double* scr_of(const AdjArgs& A, int m) { return A.scr + (size_t)m * kPlanes * A.g.plane; }
__device__ __forceinline__ int* iscr_of(const AdjArgs& A, int m) {
  return A.iscr + (size_t)m * kIntPlanes * A.g.plane;
}

// ---- F1: per node ------------------------------------------------------------
__global__ void adj_f1(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp + i;
  const double* st = st_of(A, m);
  double* S = scr_of(A, m);
  const double h = A.rs[m].inv2a;
  double q[4], M[4][4];
  ld4(st, P, id, q);
  maxwellians(q, A.gamma, A.c1, h, M);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) S[(kM + 4 * k + c) * P + id] = M[k][c];
  if (!interior(A.g, i, j)) return;
  const size_t W = id - 1, E = id + 1, Sd = id - A.g.nxp, N = id + A.g.nxp;
  double qW[4], qE[4], qS[4], qN[4], fW[4], gW[4], fE[4], gE[4], fS[4], gS[4], fN[4], gN[4];
  ld4(st, P, W, qW);
  ld4(st, P, E, qE);
  ld4(st, P, Sd, qS);
  ld4(st, P, N, qN);
  fluxes(qW, A.gamma, fW, gW);
  fluxes(qE, A.gamma, fE, gE);
  fluxes(qS, A.gamma, fS, gS);
  fluxes(qN, A.gamma, fN, gN);
  double U[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double M1W = A.c1 * qW[c] + fW[c] * h;
    const double M2E = A.c1 * qE[c] - fE[c] * h;
    const double M3S = A.c1 * qS[c] + gS[c] * h;
    const double M4N = A.c1 * qN[c] - gN[c] * h;
    U[c] = A.alpha * q[c] + M1W + M2E + M3S + M4N;
    S[(kU + c) * P + id] = U[c];
  }
  double lo = q[0], hi = lo;
  int lc = 0, hc = 0;
  const double r5[5] = {qW[0], qE[0], qS[0], qN[0], U[0]};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    if (r5[r] < lo) {
      lo = r5[r];
      lc = r + 1;
    }
    if (r5[r] > hi) {
      hi = r5[r];
      hc = r + 1;
    }
  }
  const double delta = A.rel * (hi - lo) + A.absb;
  double v1, v2, pLF;
  primitive(U, A.gamma, v1, v2, pLF);
  S[(kB + 0) * P + id] = lo - delta;
  S[(kB + 1) * P + id] = hi + delta;
  S[(kB + 2) * P + id] = A.eps < U[0] ? A.eps : U[0];
  S[(kB + 3) * P + id] = A.eps < pLF ? A.eps : pLF;
  iscr_of(A, m)[id] = lc | (hc << 4);
}

// the populations read at a node: their equilibria at boundary nodes
__device__ __forceinline__ void pops_read(const AdjArgs& A, int m, int i, int j, size_t id, int k, double p[4]) {
  const size_t P = A.g.plane;
  if (interior(A.g, i, j)) {
    const double* st = st_of(A, m);
#pragma unroll
    for (int c = 0; c < 4; ++c) p[c] = st[(4 + 4 * k + c) * P + id];
  } else {
    const double* S = scr_of(A, m);
#pragma unroll
    for (int c = 0; c < 4; ++c) p[c] = S[(kM + 4 * k + c) * P + id];
  }
}

// ---- F2: faces owned by node x: (x, x + 1) and (x, x + row) -------------------
__global__ void adj_f2(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp + i;
  double* S = scr_of(A, m);
  for (int dir = 0; dir < 2; ++dir) {
    const int iR = dir == 0 ? i + 1 : i, jR = dir == 0 ? j : j + 1;
    if (iR >= A.g.nx || jR >= A.g.ny) continue;
    const size_t idR = (size_t)jR * A.g.nxp + iR;
    const int kout = dir == 0 ? 0 : 2, kin = dir == 0 ? 1 : 3;
    double Mo[4], Mi[4], pL[4], pR[4], d[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      Mo[c] = S[(kM + 4 * kout + c) * P + id];
      Mi[c] = S[(kM + 4 * kin + c) * P + idR];
    }
    pops_read(A, m, i, j, id, kout, pL);
    pops_read(A, m, iR, jR, idR, kin, pR);
#pragma unroll
    for (int c = 0; c < 4; ++c) d[c] = (Mo[c] - pL[c]) - (Mi[c] - pR[c]);
    const bool bL = !interior(A.g, i, j), bR = !interior(A.g, iR, jR);
    double tL = 1.0, tR = 1.0, th;
    if (bL && bR) {
      th = 0.0;
    } else if (A.limiter == 0) {
      th = 0.0;
    } else if (A.limiter == 1) {
      th = 1.0;
    } else {
      if (!bL) {
        double U0[4], DD[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          U0[c] = S[(kU + c) * P + id];
          DD[c] = -4.0 * d[c];
        }
        tL = theta_star(U0, DD, S[(kB + 0) * P + id], S[(kB + 1) * P + id], S[(kB + 2) * P + id],
                        S[(kB + 3) * P + id], A.gamma);
      }
      if (!bR) {
        double U0[4], DD[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          U0[c] = S[(kU + c) * P + idR];
          DD[c] = 4.0 * d[c];
        }
        tR = theta_star(U0, DD, S[(kB + 0) * P + idR], S[(kB + 1) * P + idR], S[(kB + 2) * P + idR],
                        S[(kB + 3) * P + idR], A.gamma);
      }
      th = tL < tR ? tL : tR;
    }
    const int kd = dir == 0 ? kDX : kDY, kt = dir == 0 ? kTX : kTY;
#pragma unroll
    for (int c = 0; c < 4; ++c) S[(kd + c) * P + id] = d[c];
    S[(kt + 0) * P + id] = tL;
    S[(kt + 1) * P + id] = tR;
    S[(kt + 2) * P + id] = th;
  }
}

// ---- R0: the inlet column of u^{s+1} is the Dirichlet datum -----------------
// inlet q = (rho, rho v1, 0, p / (gamma - 1) + rho v1^2 / 2): d q / d rho = (1, v1, 0, v1^2 / 2)
__global__ void adj_r0(const AdjArgs A) {
  const int m = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.g.ny) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp;
  const double* ab = A.ain + (size_t)m * 20 * P;
  const double y = A.y_min + ((double)j + 0.5) * A.dx;
  const double v1 = fabs(y) <= A.r_jet ? A.jet_u : 0.0;
  A.inlet_acc[(size_t)m * A.g.ny + j] += ab[0 * P + id] + v1 * ab[1 * P + id] + 0.5 * (v1 * v1) * ab[3 * P + id];
}

// ---- R1: per interior cell -----------------------------------------------------
__global__ void adj_r1(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp + i;
  double* S = scr_of(A, m);
  if (!interior(A.g, i, j)) {
#pragma unroll
    for (int c = 0; c < 4; ++c) S[(kUE + c) * P + id] = 0.0;
#pragma unroll
    for (int c = 0; c < 16; ++c) S[(kNB + c) * P + id] = 0.0;
    return;
  }
  const double* ab = A.ain + (size_t)m * 20 * P;
  const int nx = A.g.nx, ny = A.g.ny, nxp = A.g.nxp;
  auto at = [&](int c, int ii, int jj) { return ab[c * P + (size_t)jj * nxp + ii]; };
  double ue[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    double v = at(c, i, j);
    if (j == 1) v += at(c, i, 0);
    if (j == ny - 2) v += at(c, i, ny - 1);
    if (i == nx - 2) {
      double w = at(c, nx - 1, j);
      if (j == 1) w += at(c, nx - 1, 0);
      if (j == ny - 2) w += at(c, nx - 1, ny - 1);
      v += w;
    }
    ue[c] = v;
    S[(kUE + c) * P + id] = v;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) S[(kNB + 4 * k + c) * P + id] = ab[(4 + 4 * k + c) * P + id] + ue[c];
}

// ---- R2: faces -------------------------------------------------------------------
__global__ void adj_r2(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp + i;
  double* S = scr_of(A, m);
  int sides = 0;
  for (int dir = 0; dir < 2; ++dir) {
    const int kd = dir == 0 ? kDX : kDY, kt = dir == 0 ? kTX : kTY;
    const int kf = dir == 0 ? kFX : kFY, ku = dir == 0 ? kUX : kUY, kg = dir == 0 ? kGX : kGY;
    double db[4] = {0, 0, 0, 0}, Ub[4] = {0, 0, 0, 0}, Bb[4] = {0, 0, 0, 0};
    int side = 0;
    const int iR = dir == 0 ? i + 1 : i, jR = dir == 0 ? j : j + 1;
    if (iR < A.g.nx && jR < A.g.ny) {
      const size_t idR = (size_t)jR * A.g.nxp + iR;
      const int kout = dir == 0 ? 0 : 2, kin = dir == 0 ? 1 : 3;
      const bool inL = interior(A.g, i, j), inR = interior(A.g, iR, jR);
      double eo[4], ei[4], pL[4], pR[4];
      pops_read(A, m, i, j, id, kout, pL);
      pops_read(A, m, iR, jR, idR, kin, pR);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        eo[c] = S[(kM + 4 * kout + c) * P + id] - pL[c];
        ei[c] = S[(kM + 4 * kin + c) * P + idR] - pR[c];
      }
      // R uses the face in its population k_out (n1 or n3) and in its own
      // u-term -theta (M_kin(R) - P_kin(R)); L in n_kin and -theta (M_kout(L) - P_kout(L))
      double thb = 0.0;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (inR) thb += S[(kNB + 4 * kout + c) * P + idR] * eo[c] - S[(kUE + c) * P + idR] * ei[c];
        if (inL) thb += S[(kNB + 4 * kin + c) * P + id] * ei[c] - S[(kUE + c) * P + id] * eo[c];
      }
      const double tL = S[(kt + 0) * P + id], tR = S[(kt + 1) * P + id];
      const bool bL = !inL, bR = !inR;
      if (A.limiter == 2 && !(bL && bR) && thb != 0.0) {
        const bool selL = tL < tR;  // the forward rule: tL < tR ? tL : tR
        if ((selL && !bL) || (!selL && !bR)) {
          const size_t ids = selL ? id : idR;
          double U0[4], DD[4], Dbar[4] = {0, 0, 0, 0};
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            U0[c] = S[(kU + c) * P + ids];
            DD[c] = (selL ? -4.0 : 4.0) * S[(kd + c) * P + id];
          }
          theta_star_bwd(U0, DD, S[(kB + 0) * P + ids], S[(kB + 1) * P + ids], S[(kB + 2) * P + ids],
                         S[(kB + 3) * P + ids], A.gamma, thb, Ub, Dbar, Bb);
#pragma unroll
          for (int c = 0; c < 4; ++c) db[c] = (selL ? -4.0 : 4.0) * Dbar[c];
          side = selL ? 1 : 2;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      S[(kf + c) * P + id] = db[c];
      S[(ku + c) * P + id] = Ub[c];
      S[(kg + c) * P + id] = Bb[c];
    }
    sides |= side << (2 * dir);
  }
  iscr_of(A, m)[P + id] = sides;
}

// ---- R3: per interior cell: bounds and U_LF adjoints --------------------------
__global__ void adj_r3(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp + i;
  double* S = scr_of(A, m);
  const int* I = iscr_of(A, m);
  if (!interior(A.g, i, j)) {
#pragma unroll
    for (int c = 0; c < 4; ++c) S[(kUB + c) * P + id] = 0.0;
    S[(kLH + 0) * P + id] = 0.0;
    S[(kLH + 1) * P + id] = 0.0;
    return;
  }
  const size_t W = id - 1, Sd = id - A.g.nxp;
  double Ub[4] = {0, 0, 0, 0}, Bb[4] = {0, 0, 0, 0};
  // faces where this cell is the selected side: R of (W, c), L of (c, E), R of (S, c), L of (c, N)
  const int sW = I[P + W] & 3, sC = I[P + id], sS = (I[P + Sd] >> 2) & 3;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (sW == 2) {
      Ub[c] += S[(kUX + c) * P + W];
      Bb[c] += S[(kGX + c) * P + W];
    }
    if ((sC & 3) == 1) {
      Ub[c] += S[(kUX + c) * P + id];
      Bb[c] += S[(kGX + c) * P + id];
    }
    if (sS == 2) {
      Ub[c] += S[(kUY + c) * P + Sd];
      Bb[c] += S[(kGY + c) * P + Sd];
    }
    if (((sC >> 2) & 3) == 1) {
      Ub[c] += S[(kUY + c) * P + id];
      Bb[c] += S[(kGY + c) * P + id];
    }
  }
  // bounds: lo - delta, hi + delta with delta = rel (hi - lo) + abs
  const double deltab = -Bb[0] + Bb[1];
  double lob = Bb[0] - A.rel * deltab, hib = Bb[1] + A.rel * deltab;
  double U[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) U[c] = S[(kU + c) * P + id];
  if (!(A.eps < U[0])) Ub[0] += Bb[2];
  {
    double v1, v2, pLF;
    primitive(U, A.gamma, v1, v2, pLF);
    if (!(A.eps < pLF)) pressure_bwd(U, A.gamma, Bb[3], Ub);
  }
  const int codes = I[id];
  if ((codes & 15) == 5) {
    Ub[0] += lob;
    lob = 0.0;
  }
  if (((codes >> 4) & 15) == 5) {
    Ub[0] += hib;
    hib = 0.0;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) S[(kUB + c) * P + id] = Ub[c];
  S[(kLH + 0) * P + id] = lob;
  S[(kLH + 1) * P + id] = hib;
}

// ---- R4: per node ------------------------------------------------------------------
__global__ void adj_r4(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const int nx = A.g.nx, ny = A.g.ny, nxp = A.g.nxp;
  const size_t P = A.g.plane, id = (size_t)j * nxp + i;
  const double* S = scr_of(A, m);
  const int* I = iscr_of(A, m);
  const double* st = st_of(A, m);
  double* out = A.aout + (size_t)m * 20 * P;
  const bool in = interior(A.g, i, j);
  double Mb[4][4], Pb[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) Mb[k][c] = Pb[k][c] = 0.0;
  // (k, neighbour offset, the face's owner, the face's direction, sign of d in it)
  // k = 0: E neighbour, face (x, E) owned by x, x-dir, +; k = 1: W, face (W, x) owned by W, -
  // k = 2: N neighbour, face (x, N) owned by x, y-dir, +; k = 3: S, face (S, x) owned by S, -
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int di = k == 0 ? 1 : (k == 1 ? -1 : 0), dj = k == 2 ? 1 : (k == 3 ? -1 : 0);
    const int in_ = i + di, jn = j + dj;
    if (in_ < 0 || in_ >= nx || jn < 0 || jn >= ny) continue;  // no such face
    const size_t idn = (size_t)jn * nxp + in_;
    const size_t owner = (k == 0 || k == 2) ? id : idn;
    const int kt = (k < 2) ? kTX : kTY, kf = (k < 2) ? kFX : kFY;
    const double th = S[(kt + 2) * P + owner];
    const double sg = (k == 0 || k == 2) ? 1.0 : -1.0;
    const bool inn = interior(A.g, in_, jn);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double dbar = S[(kf + c) * P + owner];
      double mb = sg * dbar, pb = -sg * dbar;
      if (inn) {
        const double nb = S[(kNB + 4 * k + c) * P + idn];
        mb += (1.0 + th) * nb + S[(kUB + c) * P + idn];
        pb += -th * nb;
      }
      if (in) {
        const double ue = S[(kUE + c) * P + id];
        mb += -th * ue;
        pb += th * ue;
      }
      Mb[k][c] += mb;
      Pb[k][c] += pb;
    }
  }
  // populations read at x: its stored ones (interior) or its equilibria
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      if (in)
        out[(4 + 4 * k + c) * P + id] = Pb[k][c];
      else {
        Mb[k][c] += Pb[k][c];
        out[(4 + 4 * k + c) * P + id] = 0.0;
      }
    }
  double q[4], qb[4] = {0, 0, 0, 0};
  ld4(st, P, id, q);
  const double h = A.rs[m].inv2a;
  const double hb = maxwellians_bwd(q, A.gamma, A.c1, h, Mb, qb);
  if (in) {
#pragma unroll
    for (int c = 0; c < 4; ++c) qb[c] += A.alpha * (S[(kUE + c) * P + id] + S[(kUB + c) * P + id]);
  }
  // density bounds of the cells whose minimum / maximum is this node
  // (cell y, code): (x, 0), (E, 1: x is W of E), (W, 2), (N, 3), (S, 4)
  const int cells[5][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}};
#pragma unroll
  for (int t = 0; t < 5; ++t) {
    const int ci = i + cells[t][0], cj = j + cells[t][1];
    if (!interior(A.g, ci, cj)) continue;
    const size_t idc = (size_t)cj * nxp + ci;
    const int codes = I[idc];
    if ((codes & 15) == t) qb[0] += S[(kLH + 0) * P + idc];
    if (((codes >> 4) & 15) == t) qb[0] += S[(kLH + 1) * P + idc];
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c * P + id] = qb[c];
  A.scr[(size_t)m * kPlanes * P + kHB * P + id] = hb;
}

// ---- R5: per realization: d J / d a_s through lambda's argmax ------------------
// One CTA per realization; fixed-order sums and a first-maximum argmax.
constexpr int kR = 1024;

__global__ void __launch_bounds__(kR) adj_r5(const AdjArgs A) {
  __shared__ double sh[kR];
  __shared__ double sl[kR];
  __shared__ int si[kR];
  const int m = blockIdx.x;
  const int nx = A.g.nx, ny = A.g.ny, nxp = A.g.nxp;
  const size_t P = A.g.plane;
  const long long n = (long long)nx * ny;
  const double* S = scr_of(A, m);
  const double* st = st_of(A, m);
  double hsum = 0.0, best = -1.0;
  int bi = -1;
  for (long long t = threadIdx.x; t < n; t += kR) {
    const int jj = (int)(t / nx), ii = (int)(t % nx);
    const size_t id = (size_t)jj * nxp + ii;
    hsum += S[kHB * P + id];
    double q[4], v1, v2, p;
    ld4(st, P, id, q);
    primitive(q, A.gamma, v1, v2, p);
    const double c = sqrt(A.gamma * p / q[0]);
    const double a1 = fabs(v1), a2 = fabs(v2);
    const double l = (a1 > a2 ? a1 : a2) + c;
    if (l > best) {
      best = l;
      bi = (int)t;
    }
  }
  sh[threadIdx.x] = hsum;
  sl[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = kR / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh[threadIdx.x] += sh[threadIdx.x + o];
      const double lb = sl[threadIdx.x + o];
      const int ib = si[threadIdx.x + o];
      if (lb > sl[threadIdx.x] || (lb == sl[threadIdx.x] && ib >= 0 && ib < si[threadIdx.x])) {
        sl[threadIdx.x] = lb;
        si[threadIdx.x] = ib;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x != 0 || si[0] < 0) return;
  const double a = A.rs[m].a;
  const double ab = sh[0] * (-0.5 / (a * a));           // h = 1 / (2 a)
  const double lamb = ab * (A.kappa * 2.0 / (1.0 - A.alpha));  // a = kappa 2 lambda / (1 - alpha)
  const int jj = si[0] / nx, ii = si[0] % nx;
  const size_t id = (size_t)jj * nxp + ii;
  double q[4], v1, v2, p;
  ld4(st, P, id, q);
  primitive(q, A.gamma, v1, v2, p);
  const double c = sqrt(A.gamma * p / q[0]);
  double qb[4] = {0, 0, 0, 0};
  // l = max(|v1|, |v2|) + c
  double v1b = 0.0, v2b = 0.0;
  if (fabs(v1) > fabs(v2))
    v1b = lamb * (v1 > 0.0 ? 1.0 : (v1 < 0.0 ? -1.0 : 0.0));
  else
    v2b = lamb * (v2 > 0.0 ? 1.0 : (v2 < 0.0 ? -1.0 : 0.0));
  // c = sqrt(gamma p / rho)
  const double xb = lamb * 0.5 / c;
  const double pb = xb * A.gamma / q[0];
  qb[0] += -xb * A.gamma * p / (q[0] * q[0]);
  pressure_bwd(q, A.gamma, pb, qb);
  qb[1] += v1b / q[0];
  qb[2] += v2b / q[0];
  qb[0] -= (v1b * v1 + v2b * v2) / q[0];
  double* out = A.aout + (size_t)m * 20 * P;
#pragma unroll
  for (int c2 = 0; c2 < 4; ++c2) out[c2 * P + id] += qb[c2];
}

// ---- the initial state: populations = M_k(u^0; a_0) at every node -------------
__global__ void adj_init_nodes(const AdjArgs A) {
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(A.g, i, j)) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp + i;
  const double* ab = A.ain + (size_t)m * 20 * P;  // adjoint of u^0, populations^0
  double* out = A.aout + (size_t)m * 20 * P;
  double Mb[4][4];
  const bool in = interior(A.g, i, j);
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int c = 0; c < 4; ++c) Mb[k][c] = in ? ab[(4 + 4 * k + c) * P + id] : 0.0;
  double q[4], qb[4];
  ld4(st_of(A, m), P, id, q);
#pragma unroll
  for (int c = 0; c < 4; ++c) qb[c] = ab[c * P + id];
  const double hb = maxwellians_bwd(q, A.gamma, A.c1, A.rs[m].inv2a, Mb, qb);
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c * P + id] = qb[c];
#pragma unroll
  for (int c = 0; c < 16; ++c) out[(4 + c) * P + id] = 0.0;
  A.scr[(size_t)m * kPlanes * P + kHB * P + id] = hb;
}

// ---- J and the seed of the reverse sweep ---------------------------------------
// J_m = sum_x w(x) rho_m(x) (fixed order, one CTA per realization); seed
// u-bar = (w / M, 0, 0, 0), populations-bar = 0.
__global__ void __launch_bounds__(kR) adj_objective(const AdjArgs A, const double* w, double* Jm) {
  __shared__ double sh[kR];
  const int m = blockIdx.x;
  const int nx = A.g.nx, ny = A.g.ny, nxp = A.g.nxp;
  const size_t P = A.g.plane;
  const long long n = (long long)nx * ny;
  const double* st = st_of(A, m);
  double* out = A.aout + (size_t)m * 20 * P;
  double s = 0.0;
  for (long long t = threadIdx.x; t < n; t += kR) {
    const int jj = (int)(t / nx), ii = (int)(t % nx);
    const size_t id = (size_t)jj * nxp + ii;
    const double wx = w[t];
    s += wx * st[id];
    out[id] = wx / (double)A.g.M;
#pragma unroll
    for (int c = 1; c < 20; ++c) out[c * P + id] = 0.0;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kR / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) Jm[m] = sh[0];
}

// inlet column of the initial state (Eq. (u0_def)): its adjoint joins the inlet's
__global__ void adj_init_inlet(const AdjArgs A) {
  const int m = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.g.ny) return;
  const size_t P = A.g.plane, id = (size_t)j * A.g.nxp;
  const double* ab = A.aout + (size_t)m * 20 * P;
  const double y = A.y_min + ((double)j + 0.5) * A.dx;
  const double v1 = fabs(y) <= A.r_jet ? A.jet_u : 0.0;
  A.inlet_acc[(size_t)m * A.g.ny + j] += ab[0 * P + id] + v1 * ab[1 * P + id] + 0.5 * (v1 * v1) * ab[3 * P + id];
}

// d J / d a_k = sum_m sum_j rho-bar_{m,j} rho_jet (Y_k cos(k pi yb) + Z_k sin(k pi yb)) W(yb)
// over the jet rows; one CTA per mode, fixed order.
__global__ void __launch_bounds__(kR) adj_amplitudes(const AdjArgs A, const double* xi, int K, double rho_jet,
                                                     double* grad) {
  __shared__ double sh[kR];
  const int k = blockIdx.x + 1;
  const int ny = A.g.ny, M = A.g.M;
  const double pi = 3.14159265358979323846;
  double s = 0.0;
  for (long long t = threadIdx.x; t < (long long)M * ny; t += kR) {
    const int m = (int)(t / ny), j = (int)(t % ny);
    const double y = A.y_min + ((double)j + 0.5) * A.dx;
    if (!(fabs(y) <= A.r_jet)) continue;
    const double yb = y / A.r_jet;
    const double arg = (double)k * pi * yb;
    const double cw = cos(0.5 * pi * yb);
    const double dr = rho_jet * (xi[(size_t)m * 2 * K + k - 1] * cos(arg) + xi[(size_t)m * 2 * K + K + k - 1] * sin(arg)) *
                      (cw * cw);
    s += A.inlet_acc[t] * dr;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = kR / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) grad[k - 1] = sh[0];
}

AdjArgs make_args(const Launch& L, int level, const double* state, const RealState* rs, const double* ain,
                  double* aout, double* scr, int* iscr, double* inlet_acc) {
  const LevelDesc& D = L.lv[level];
  AdjArgs A{};
  A.g = Geo{D.nx, D.ny, D.nx_pad, D.plane, L.M};
  A.gamma = L.ph.gamma;
  A.alpha = L.ph.alpha;
  A.c1 = (1.0 - L.ph.alpha) / 4.0;
  A.kappa = L.ph.kappa;
  A.rel = L.ph.rlmp_rel;
  A.absb = L.ph.rlmp_abs;
  A.eps = L.ph.eps_pos;
  A.limiter = L.ph.limiter;
  A.state = state;
  A.rs = rs;
  A.ain = ain;
  A.aout = aout;
  A.scr = scr;
  A.iscr = iscr;
  A.inlet_acc = inlet_acc;
  A.jet_u = L.ph.jet_u;
  A.y_min = D.y_min;
  A.dx = D.dx;
  return A;
}

dim3 node_grid(const LevelDesc& D, int M) {
  const long long n = (long long)D.nx * D.ny;
  return dim3((unsigned)((n + kT - 1) / kT), (unsigned)M);
}

}  // namespace

size_t adjoint_scratch_doubles(const LevelDesc& D, int M) { return (size_t)M * kPlanes * D.plane; }
size_t adjoint_scratch_ints(const LevelDesc& D, int M) { return (size_t)M * kIntPlanes * D.plane; }

cudaError_t adjoint_objective(const Launch& L, int level, const double* state, const double* w, double* Jm,
                              double* aseed, cudaStream_t s) {
  AdjArgs A = make_args(L, level, state, nullptr, nullptr, aseed, nullptr, nullptr, nullptr);
  adj_objective<<<L.M, kR, 0, s>>>(A, w, Jm);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t adjoint_step(const Launch& L, int level, double r_jet, const double* state, const RealState* rs,
                         const double* ain, double* aout, double* scr, int* iscr, double* inlet_acc,
                         cudaStream_t s) {
  AdjArgs A = make_args(L, level, state, rs, ain, aout, scr, iscr, inlet_acc);
  A.r_jet = r_jet;
  const LevelDesc& D = L.lv[level];
  const dim3 g = node_grid(D, L.M);
  adj_f1<<<g, kT, 0, s>>>(A);
  adj_f2<<<g, kT, 0, s>>>(A);
  adj_r0<<<dim3((D.ny + kT - 1) / kT, L.M), kT, 0, s>>>(A);
  adj_r1<<<g, kT, 0, s>>>(A);
  adj_r2<<<g, kT, 0, s>>>(A);
  adj_r3<<<g, kT, 0, s>>>(A);
  adj_r4<<<g, kT, 0, s>>>(A);
  adj_r5<<<L.M, kR, 0, s>>>(A);
  add_launches(8);
  return cudaGetLastError();
}

cudaError_t adjoint_initial(const Launch& L, int level, double r_jet, const double* state0, const RealState* rs0,
                            const double* ain, double* aout, double* scr, double* inlet_acc, cudaStream_t s) {
  AdjArgs A = make_args(L, level, state0, rs0, ain, aout, scr, nullptr, inlet_acc);
  A.r_jet = r_jet;
  const LevelDesc& D = L.lv[level];
  adj_init_nodes<<<node_grid(D, L.M), kT, 0, s>>>(A);
  adj_r5<<<L.M, kR, 0, s>>>(A);
  adj_init_inlet<<<dim3((D.ny + kT - 1) / kT, L.M), kT, 0, s>>>(A);
  add_launches(3);
  return cudaGetLastError();
}

cudaError_t adjoint_amplitudes(const Launch& L, int level, double r_jet, const double* inlet_acc, const double* xi,
                               int K, double* grad, cudaStream_t s) {
  AdjArgs A = make_args(L, level, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                        const_cast<double*>(inlet_acc));
  A.r_jet = r_jet;
  adj_amplitudes<<<K, kR, 0, s>>>(A, xi, K, L.ph.jet_rho, grad);
  add_launches(1);
  return cudaGetLastError();
}

}  // namespace vlbm
