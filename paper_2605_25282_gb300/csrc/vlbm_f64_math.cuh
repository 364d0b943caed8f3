// FP64 arithmetic of the paper's update shared by the FP64 step kernel and
// its adjoint: primitive recovery (Eq. (eos)), the Euler fluxes
// (Eqs. (fluxF), (fluxG)) and the R-theta limiter.  Both translation units are
// compiled without FMA contraction and evaluate these in the oracle's order,
// so the adjoint re-evaluates exactly the branches the forward step took.
#pragma once

namespace vlbm {
namespace f64 {

__device__ __forceinline__ void primitive(const double q[4], double gamma, double& v1, double& v2,
                                          double& p) {
  v1 = q[1] / q[0];
  v2 = q[2] / q[0];
  p = (gamma - 1.0) * (q[3] - 0.5 * q[0] * (v1 * v1 + v2 * v2));
}

__device__ __forceinline__ void fluxes(const double q[4], double gamma, double f[4], double g[4]) {
  double v1, v2, p;
  primitive(q, gamma, v1, v2, p);
  f[0] = q[1];
  f[1] = q[1] * v1 + p;
  f[2] = q[1] * v2;
  f[3] = (q[3] + p) * v1;
  g[0] = q[2];
  g[1] = q[1] * v2;
  g[2] = q[2] * v2 + p;
  g[3] = (q[3] + p) * v2;
}

// Largest theta in [0, 1] keeping U0 + theta D inside the admissible,
// relaxed-bounded set (convex: the feasible thetas form [0, theta*]); the
// pressure floor enters as kk = eps_p / (gamma - 1).  theta_star_kk composes
// the parts below in this order: the density limit (theta_pre, a division
// where it binds, theta_density), the pressure test q(th) >= 0 with
// q(theta) = A theta^2 + B theta + C (C = q(0) = theta_c of the node), and
// where it fails the root (theta_root).  A kernel that evaluates many sides
// at once may take their divisions and roots together; every part is the
// same arithmetic, so the result is the same.

// q(0) of a node: U0's pressure function rho E - |m|^2 / 2 - kk rho.
__device__ __forceinline__ double theta_c(const double U0[4], double kk) {
  return U0[0] * U0[3] - 0.5 * (U0[1] * U0[1] + U0[2] * U0[2]) - kk * U0[0];
}

// The density limit num / den of one side (a division only where it binds:
// num < den; a correctly rounded quotient of num >= den > 0 is >= 1, so the
// result is the same as dividing always) and the coefficients A, B of q.
struct ThetaPre {
  double num, den, A, B;
  bool divide;
};
__device__ __forceinline__ void theta_pre(const double U0[4], const double D[4], double lo_b, double hi_b,
                                          double eps_r, double kk, ThetaPre& t) {
  const double lower = eps_r > lo_b ? eps_r : lo_b;
  t.divide = false;
  t.num = 0.0;
  t.den = 1.0;
  if (D[0] < 0.0) {
    t.num = U0[0] - lower;
    t.den = -D[0];
    t.divide = t.num < t.den;
  } else if (D[0] > 0.0) {
    t.num = hi_b - U0[0];
    t.den = D[0];
    t.divide = t.num < t.den;
  }
  t.B = U0[0] * D[3] + D[0] * U0[3] - (U0[1] * D[1] + U0[2] * D[2]) - kk * D[0];
  t.A = D[0] * D[3] - 0.5 * (D[1] * D[1] + D[2] * D[2]);
}

// theta after the density limit: 1, or the quotient lim where it is smaller;
// never below 0.
__device__ __forceinline__ double theta_density(bool divided, double lim) {
  double th = 1.0;
  if (divided && lim < th) th = lim;
  if (th < 0.0) th = 0.0;
  return th;
}

// The pressure test at th: true with the final theta in *out when q(th) >= 0
// (th) or C <= 0 (0); false when the root of q below th is needed.
__device__ __forceinline__ bool theta_final(double th, double A, double B, double C, double* out) {
  const double qth = C + th * (B + th * A);
  if (qth >= 0.0) {
    *out = th;
    return true;
  }
  if (C <= 0.0) {
    *out = 0.0;
    return true;
  }
  return false;
}

// The smallest positive root of q (C > 0 > q(th)), clamped to [0, th].
__device__ __forceinline__ double theta_root(double A, double B, double C, double th) {
  double r;
  if (A == 0.0) {
    r = -C / B;
  } else {
    double disc = B * B - 4.0 * A * C;
    if (disc < 0.0) disc = 0.0;
    const double sq = sqrt(disc);
    const double Q = -0.5 * (B + (B >= 0.0 ? sq : -sq));
    if (Q == 0.0) return 0.0;
    const double r1 = Q / A;
    const double r2 = C / Q;
    r = -1.0;
    if (r1 > 0.0) r = r1;
    if (r2 > 0.0 && (r < 0.0 || r2 < r)) r = r2;
    if (r < 0.0) return 0.0;
  }
  if (r > th) r = th;
  if (r < 0.0) r = 0.0;
  return r;
}

static __device__ double theta_star_kk(const double U0[4], const double D[4], double lo_b, double hi_b,
                                       double eps_r, double kk) {
  ThetaPre t;
  theta_pre(U0, D, lo_b, hi_b, eps_r, kk, t);
  const double th = theta_density(t.divide, t.divide ? t.num / t.den : 0.0);
  const double C = theta_c(U0, kk);
  double out;
  if (theta_final(th, t.A, t.B, C, &out)) return out;
  return theta_root(t.A, t.B, C, th);
}

static __device__ double theta_star(const double U0[4], const double D[4], double lo_b, double hi_b,
                                    double eps_r, double eps_p, double gamma) {
  return theta_star_kk(U0, D, lo_b, hi_b, eps_r, eps_p / (gamma - 1.0));
}

__device__ __forceinline__ bool is_boundary(int i, int j, int nx, int ny) {
  return i == 0 || i == nx - 1 || j == 0 || j == ny - 1;
}

}  // namespace f64
}  // namespace vlbm
