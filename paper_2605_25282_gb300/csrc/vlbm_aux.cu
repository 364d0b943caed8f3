// Ensemble set-up, per-realization time stepping bookkeeping and state I/O.
//
//  - inlet_kernel     Sec. 2.3, Eq. (karhunenExp) and Sec. 2.2, Eq. (rho_inlet_def):
//                     Philox4x32-10 (Salmon et al., SC'11) -> 2K uniforms on (-1, 1)
//                     -> inlet density per row -> conserved inlet state.
//  - init_state       Eq. (u0_def): inlet column + quiescent ambient state.
//  - lambda_kernel    lambda = max over nodes of max(|v1|, |v2|) + sqrt(gamma p / rho).
//  - tick_kernel      a_n = kappa 2 lambda / (1 - alpha) (Bouchut bound, Sec. 2.1),
//                     dt = dx / a_n (Sec. 2.3), landing on t*, and the advance of
//                     t, step count and lambda after a step.
//  - moments / density / get_state / set_state: layout conversions.
//  - bounded_wait_probe: one mbarrier wait that nothing completes, bounded
//    like the step kernels' waits (the failure-detection check).
#include <cmath>

#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

struct PerturbDev {
  double r_jet;
  int K;
  int m_begin;
  double amp[kMaxModes];
  uint32_t key0, key1;
  const double* xi;  // [M][2K] given uniforms (Y then Z), or NULL: Philox draws
  double* xi_out;    // [M][2K]: where the drawn uniforms are recorded (may be NULL)
};

// One thread per (level, realization, row).
__global__ void inlet_kernel(const Launch L, const PerturbDev P) {
  const int lvl = blockIdx.z;
  const int m = blockIdx.y;
  const LevelDesc& D = L.lv[lvl];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= D.ny) return;
  // coefficients of realization m (the same for every row; recomputed per thread)
  double Y[kMaxModes], Z[kMaxModes];
  if (P.xi) {
    for (int k = 0; k < P.K; ++k) {
      Y[k] = P.xi[(size_t)m * 2 * P.K + k];
      Z[k] = P.xi[(size_t)m * 2 * P.K + P.K + k];
    }
  }
  for (int w = 0; !P.xi && w < 2 * P.K; w += 4) {
    uint32_t o[4];
    philox4x32_10((uint32_t)(P.m_begin + m), (uint32_t)(w / 4), 0u, 0u, P.key0, P.key1, o);
    for (int l = 0; l < 4 && w + l < 2 * P.K; ++l) {
      const double u = __dadd_rn(__dmul_rn((double)(o[l] >> 8) + 0.5, 1.0 / 8388608.0), -1.0);
      const int idx = w + l;
      if (idx < P.K)
        Y[idx] = u;
      else
        Z[idx - P.K] = u;
    }
  }
  if (P.xi_out && j == 0) {
    for (int k = 0; k < P.K; ++k) {
      P.xi_out[(size_t)m * 2 * P.K + k] = Y[k];
      P.xi_out[(size_t)m * 2 * P.K + P.K + k] = Z[k];
    }
  }
  const double y = __dadd_rn(D.y_min, __dmul_rn((double)j + 0.5, D.dx));
  const double gamma = L.ph.gamma;
  double rho, v1;
  if (fabs(y) <= P.r_jet) {
    const double pi = 3.14159265358979323846;
    const double yb = y / P.r_jet;
    double s = 0.0;
    for (int k = 1; k <= P.K; ++k) {
      const double arg = __dmul_rn(__dmul_rn((double)k, pi), yb);
      s = __dadd_rn(s, __dmul_rn(P.amp[k - 1], __dadd_rn(__dmul_rn(Y[k - 1], cos(arg)), __dmul_rn(Z[k - 1], sin(arg)))));
    }
    const double cw = cos(__dmul_rn(__dmul_rn(0.5, pi), yb));
    const double W = __dmul_rn(cw, cw);
    rho = __dmul_rn(L.ph.jet_rho, __dadd_rn(1.0, __dmul_rn(s, W)));
    v1 = L.ph.jet_u;
  } else {
    rho = L.ph.amb_rho;
    v1 = 0.0;
  }
  const double p = fabs(y) <= P.r_jet ? L.ph.jet_p : L.ph.amb_p;
  double* inl = D.inlet + (size_t)m * 4 * D.ny;
  D.inlet_f[(size_t)m * D.ny + j] = make_float4((float)rho, (float)v1, 0.0f, (float)p);
  inl[0 * D.ny + j] = rho;
  inl[1 * D.ny + j] = __dmul_rn(rho, v1);
  inl[2 * D.ny + j] = 0.0;
  inl[3 * D.ny + j] = __dadd_rn(p / (gamma - 1.0), __dmul_rn(__dmul_rn(0.5, rho), __dmul_rn(v1, v1)));
}

__device__ __forceinline__ void cons_to_prim(const double q[4], double gamma, double& v1, double& v2, double& p) {
  v1 = q[1] / q[0];
  v2 = q[2] / q[0];
  p = (gamma - 1.0) * (q[3] - 0.5 * q[0] * (v1 * v1 + v2 * v2));
}

// Grid: x over nodes of a row range, y = m, z = level.  Each thread one node.
__device__ __forceinline__ bool node_of(const LevelDesc& D, int& i, int& j) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= (long long)D.nx * D.ny) return false;
  j = (int)(n / D.nx);
  i = (int)(n % D.nx);
  return true;
}

// amb: the ambient state at rest as FP32 primitives, formed once on the host
// (the FP32 path writes it without FP64 arithmetic per node).
__global__ void init_state_kernel(const Launch L, int precision, float4 amb) {
  const LevelDesc& D = L.lv[blockIdx.z];
  const int m = blockIdx.y;
  int i, j;
  if (!node_of(D, i, j)) return;
  if (precision != VLBM_FP64 && i != 0) {
    float4* s = reinterpret_cast<float4*>(D.lat) + (size_t)m * D.real_stride;
    const size_t off = (size_t)j * D.nx_pad + i;
    s[off] = amb;
    for (int k = 0; k < 4; ++k) s[(1 + k) * D.plane + off] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const double gamma = L.ph.gamma;
  double q[4];
  if (i == 0) {
    const double* inl = D.inlet + (size_t)m * 4 * D.ny;
    for (int c = 0; c < 4; ++c) q[c] = inl[c * D.ny + j];
  } else {
    q[0] = L.ph.amb_rho;
    q[1] = 0.0;
    q[2] = 0.0;
    q[3] = __dadd_rn(L.ph.amb_p / (gamma - 1.0), 0.0);
  }
  const size_t off = (size_t)j * D.nx_pad + i;
  if (precision == VLBM_FP64) {
    double* s = reinterpret_cast<double*>(D.lat) + (size_t)m * D.real_stride;
    for (int c = 0; c < 4; ++c) s[c * D.plane + off] = q[c];
  } else {
    float4* s = reinterpret_cast<float4*>(D.lat) + (size_t)m * D.real_stride;
    double v1, v2, p;
    cons_to_prim(q, gamma, v1, v2, p);
    s[off] = make_float4((float)q[0], (float)v1, (float)v2, (float)p);
    for (int k = 0; k < 4; ++k) s[(1 + k) * D.plane + off] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void reset_rs_kernel(const Launch L, int level, int m0, int count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  RealState* s = L.lv[level].rs + m0 + r;
  s->t = 0.0;
  s->t_target = __longlong_as_double(0x7ff0000000000000LL);
  s->a = 0.0;
  s->inv2a = 0.0;
  s->dt = 0.0;
  s->inv2a_prev = 0.0;
  s->inv2a_f = 0.f;
  s->dinv2a_f = 0.f;
  s->steps = 0;
  s->lam_bits = 0;
  s->lam_next_bits = 0;
  s->active = 0;
  s->landing = 0;
  s->flags = 0;
  s->gref_set = 0;
}

// lambda of the current lattice of realizations m0..m0+count-1 -> rs.lam_bits
__global__ void lambda_kernel(const Launch L, int precision, int level, int m0) {
  const LevelDesc& D = L.lv[level];
  const int m = m0 + blockIdx.y;
  int i, j;
  double lam = 0.0;
  int flags = 0;
  RealState* rs = D.rs + m;
  if (node_of(D, i, j)) {
    const int par = (int)(rs->steps & 1);
    const size_t off = (size_t)j * D.nx_pad + i;
    if (precision == VLBM_FP64) {
      const double* s = reinterpret_cast<const double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
      double q[4], v1, v2, p;
      for (int c = 0; c < 4; ++c) q[c] = s[c * D.plane + off];
      const double rho = q[0];
      cons_to_prim(q, L.ph.gamma, v1, v2, p);
      if (!(rho > 0.0) || !(p > 0.0)) flags |= 1;
      if (!isfinite(rho) || !isfinite(v1) || !isfinite(v2) || !isfinite(p)) flags |= 2;
      if (!flags) lam = fmax(fabs(v1), fabs(v2)) + sqrt(L.ph.gamma * p / rho);
    } else {
      // FP32 throughout (the stored state is FP32); the value is exact in FP64
      const float4* s = reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
      const float4 w = s[off];
      if (!(w.x > 0.0f) || !(w.w > 0.0f)) flags |= 1;
      if (!isfinite(w.x) || !isfinite(w.y) || !isfinite(w.z) || !isfinite(w.w)) flags |= 2;
      if (!flags) lam = (double)(fmaxf(fabsf(w.y), fabsf(w.z)) + sqrtf(L.pf.gamma * w.w / w.x));
    }
  }
  unsigned long long b = lam_to_bits(lam);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
    b = ob > b ? ob : b;
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&rs->lam_bits, b);
    if (flags) atomicOr(&rs->flags, flags);
  }
}

// Equilibrium populations M_k(u; a0) of the current FP64 state, with a0 the
// kinetic speed of that state (no landing): the oracle's initial populations.
__global__ void fill_equilibrium_f64_kernel(const Launch L, int level, int m0) {
  const LevelDesc& D = L.lv[level];
  const int m = m0 + blockIdx.y;
  int i, j;
  if (!node_of(D, i, j)) return;
  const RealState* rs = D.rs + m;
  const double lam = bits_to_lam(rs->lam_bits);
  const double a = L.ph.kappa * 2.0 * lam / (1.0 - L.ph.alpha);
  const double inv2a = 0.5 / a;
  const double c1 = (1.0 - L.ph.alpha) / 4.0;
  const int par = (int)(rs->steps & 1);
  double* s = reinterpret_cast<double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
  const size_t off = (size_t)j * D.nx_pad + i;
  double q[4], v1, v2, p;
  for (int c = 0; c < 4; ++c) q[c] = s[c * D.plane + off];
  cons_to_prim(q, L.ph.gamma, v1, v2, p);
  const double f[4] = {q[1], q[1] * v1 + p, q[1] * v2, (q[3] + p) * v1};
  const double g[4] = {q[2], q[1] * v2, q[2] * v2 + p, (q[3] + p) * v2};
  for (int c = 0; c < 4; ++c) {
    s[(4 + 0 + c) * D.plane + off] = c1 * q[c] + f[c] * inv2a;
    s[(4 + 4 + c) * D.plane + off] = c1 * q[c] - f[c] * inv2a;
    s[(4 + 8 + c) * D.plane + off] = c1 * q[c] + g[c] * inv2a;
    s[(4 + 12 + c) * D.plane + off] = c1 * q[c] - g[c] * inv2a;
  }
}

// One thread per (level, realization).
__global__ void tick_kernel(const Launch L, int precision, int advance) {
  const int lvl = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L.M) return;
  const LevelDesc& D = L.lv[lvl];
  RealState* s = D.rs + m;
  if (advance && s->active) {
    s->t = s->landing ? s->t_target : s->t + s->dt;
    s->steps += 1;
    s->lam_bits = s->lam_next_bits;
    s->lam_next_bits = 0;
    if (precision == VLBM_MIXED) s->inv2a_prev = (double)s->inv2a_f;
  }
  // prepare the next step
  const double lam = bits_to_lam(s->lam_bits);
  double a = L.ph.kappa * 2.0 * lam / (1.0 - L.ph.alpha);
  int landing = 0;
  int active = 1;
  if (s->flags || !(a > 0.0)) active = 0;
  if (isfinite(s->t_target)) {
    if (s->t >= s->t_target) {
      active = 0;
    } else {
      const double a_land = D.dx / (s->t_target - s->t);
      if (a_land >= a) {
        a = a_land;
        landing = 1;
      }
    }
  }
  s->a = a;
  s->inv2a = 0.5 / a;
  s->landing = landing;
  s->active = active;
  if (precision == VLBM_MIXED) {
    // The FP32 kernel uses 1/(2a) rounded down, i.e. a slightly larger kinetic
    // speed a_eff >= a_n; time advances with that same a_eff.
    const float f = __double2float_rd(0.5 / a);
    s->inv2a_f = f;
    const double a_eff = 0.5 / (double)f;
    s->dt = D.dx / a_eff;
    if (!s->gref_set) {
      s->inv2a_prev = (double)f;
      s->gref_set = 1;
    }
    s->dinv2a_f = (float)(s->inv2a_prev - (double)f);
  } else {
    s->dt = D.dx / a;
  }
}

__global__ void set_target_kernel(const Launch L, double t_target) {
  const int lvl = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L.M) return;
  L.lv[lvl].rs[m].t_target = t_target;
}

__global__ void count_active_kernel(const Launch L, int* out) {
  const int lvl = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L.M) return;
  if (L.lv[lvl].rs[m].active) atomicAdd(out, 1);
}

__device__ __forceinline__ void load_cons(const Launch& L, const LevelDesc& D, int precision, int m, size_t off,
                                          double q[4], float4* prim_out) {
  const RealState* rs = D.rs + m;
  const int par = (int)(rs->steps & 1);
  if (precision == VLBM_FP64) {
    const double* s = reinterpret_cast<const double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
    for (int c = 0; c < 4; ++c) q[c] = s[c * D.plane + off];
  } else {
    const float4* s = reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
    const float4 w = s[off];
    if (prim_out) *prim_out = w;
    const double rho = w.x, v1 = w.y, v2 = w.z, p = w.w;
    q[0] = rho;
    q[1] = rho * v1;
    q[2] = rho * v2;
    q[3] = p / (L.ph.gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2);
  }
}

__global__ void moments_kernel(const Launch L, int precision, int level, int m0, double* rho, double* u,
                               double* v, double* p) {
  const LevelDesc& D = L.lv[level];
  const int r = blockIdx.y;
  const int m = m0 + r;
  int i, j;
  if (!node_of(D, i, j)) return;
  const size_t off = (size_t)j * D.nx_pad + i;
  const size_t o = ((size_t)r * D.ny + j) * D.nx + i;
  double R, V1, V2, P;
  if (precision == VLBM_FP64) {
    double q[4];
    load_cons(L, D, precision, m, off, q, nullptr);
    R = q[0];
    cons_to_prim(q, L.ph.gamma, V1, V2, P);
  } else {
    const RealState* rs = D.rs + m;
    const int par = (int)(rs->steps & 1);
    const float4* s = reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
    const float4 w = s[off];
    R = w.x;
    V1 = w.y;
    V2 = w.z;
    P = w.w;
  }
  if (rho) rho[o] = R;
  if (u) u[o] = V1;
  if (v) v[o] = V2;
  if (p) p[o] = P;
}

__global__ void density_kernel(const Launch L, int precision, int level, int m0, void* out, int as_f32) {
  const LevelDesc& D = L.lv[level];
  const int r = blockIdx.y;
  const int m = m0 + r;
  int i, j;
  if (!node_of(D, i, j)) return;
  const size_t off = (size_t)j * D.nx_pad + i;
  const size_t o = ((size_t)r * D.ny + j) * D.nx + i;
  const RealState* rs = D.rs + m;
  const int par = (int)(rs->steps & 1);
  double R;
  if (precision == VLBM_FP64)
    R = (reinterpret_cast<const double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride)[off];
  else
    R = (reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride)[off].x;
  if (as_f32)
    reinterpret_cast<float*>(out)[o] = (float)R;
  else
    reinterpret_cast<double*>(out)[o] = R;
}

__device__ __forceinline__ bool node_is_boundary(const LevelDesc& D, int i, int j) {
  return i == 0 || i == D.nx - 1 || j == 0 || j == D.ny - 1;
}

// MIXED populations from the stored rest-frame non-equilibrium parts:
// u_k = M_k(u; a_prev) + B_v^{-1} g'_k, with the Galilean boost
// B_w (rho, m, E) = (rho, m - rho w, E - m.w + rho |w|^2 / 2).
__global__ void get_state_kernel(const Launch L, int precision, int level, int m0, double* u, double* pops) {
  const LevelDesc& D = L.lv[level];
  const int r = blockIdx.y;
  const int m = m0 + r;
  int i, j;
  if (!node_of(D, i, j)) return;
  const size_t off = (size_t)j * D.nx_pad + i;
  const size_t nn = (size_t)D.nx * D.ny;
  const size_t o = (size_t)j * D.nx + i;
  const RealState* rs = D.rs + m;
  const int par = (int)(rs->steps & 1);
  if (precision == VLBM_FP64) {
    const double* s = reinterpret_cast<const double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
    for (int c = 0; c < 4; ++c) u[((size_t)r * 4 + c) * nn + o] = s[c * D.plane + off];
    if (pops)
      for (int k = 0; k < 16; ++k) pops[((size_t)r * 16 + k) * nn + o] = s[(4 + k) * D.plane + off];
    return;
  }
  double q[4];
  float4 w;
  load_cons(L, D, precision, m, off, q, &w);
  for (int c = 0; c < 4; ++c) u[((size_t)r * 4 + c) * nn + o] = q[c];
  if (!pops) return;
  const float4* s = reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
  const double gamma = L.ph.gamma, c1 = (1.0 - L.ph.alpha) / 4.0;
  const double v1 = w.y, v2 = w.z, p = w.w;
  const double f[4] = {q[1], q[1] * v1 + p, q[1] * v2, (q[3] + p) * v1};
  const double g[4] = {q[2], q[1] * v2, q[2] * v2 + p, (q[3] + p) * v2};
  const double inv2a = rs->gref_set ? rs->inv2a_prev : 0.5 / (L.ph.kappa * 2.0 * bits_to_lam(rs->lam_bits) / (1.0 - L.ph.alpha));
  const bool bnd = node_is_boundary(D, i, j);
  (void)gamma;
  for (int k = 0; k < 4; ++k) {
    const float4 gp = bnd ? make_float4(0.f, 0.f, 0.f, 0.f) : s[(1 + k) * D.plane + off];
    // lab-frame non-equilibrium part: B_v^{-1} g'
    const double gr = gp.x, gm1 = gp.y + v1 * gp.x, gm2 = gp.z + v2 * gp.x;
    const double gE = gp.w + v1 * gp.y + v2 * gp.z + 0.5 * (v1 * v1 + v2 * v2) * gp.x;
    const double gl[4] = {gr, gm1, gm2, gE};
    for (int c = 0; c < 4; ++c) {
      const double F = (k < 2) ? f[c] : g[c];
      const double M = (k % 2 == 0) ? c1 * q[c] + F * inv2a : c1 * q[c] - F * inv2a;
      pops[((size_t)r * 16 + 4 * k + c) * nn + o] = M + gl[c];
    }
  }
}

// Writes u (and, FP64, the raw populations) of the current lattice (steps = 0
// after the reset, so lattice 0).  MIXED populations are converted by
// set_pops_mixed_kernel once the kinetic speed of the new state is known.
__global__ void set_state_kernel(const Launch L, int precision, int level, int m0, const double* u,
                                 const double* pops) {
  const LevelDesc& D = L.lv[level];
  const int r = blockIdx.y;
  const int m = m0 + r;
  int i, j;
  if (!node_of(D, i, j)) return;
  const size_t off = (size_t)j * D.nx_pad + i;
  const size_t nn = (size_t)D.nx * D.ny;
  const size_t o = (size_t)j * D.nx + i;
  if (precision == VLBM_FP64) {
    double* s = reinterpret_cast<double*>(D.lat) + (size_t)m * D.real_stride;
    for (int c = 0; c < 4; ++c) s[c * D.plane + off] = u[((size_t)r * 4 + c) * nn + o];
    for (int k = 0; k < 16; ++k) s[(4 + k) * D.plane + off] = pops[((size_t)r * 16 + k) * nn + o];
  } else {
    float4* s = reinterpret_cast<float4*>(D.lat) + (size_t)m * D.real_stride;
    double q[4];
    for (int c = 0; c < 4; ++c) q[c] = u[((size_t)r * 4 + c) * nn + o];
    double v1, v2, p;
    cons_to_prim(q, L.ph.gamma, v1, v2, p);
    s[off] = make_float4((float)q[0], (float)v1, (float)v2, (float)p);
  }
}

__global__ void set_pops_mixed_kernel(const Launch L, int level, int m0, const double* u, const double* pops) {
  const LevelDesc& D = L.lv[level];
  const int r = blockIdx.y;
  const int m = m0 + r;
  int i, j;
  if (!node_of(D, i, j)) return;
  const size_t off = (size_t)j * D.nx_pad + i;
  const size_t nn = (size_t)D.nx * D.ny;
  const size_t o = (size_t)j * D.nx + i;
  RealState* rs = D.rs + m;
  const double lam = bits_to_lam(rs->lam_bits);
  const double a = L.ph.kappa * 2.0 * lam / (1.0 - L.ph.alpha);
  const float inv2a_f = __double2float_rd(0.5 / a);
  const double inv2a = (double)inv2a_f;
  if (i == 0 && j == 0) {
    rs->inv2a_prev = inv2a;
    rs->gref_set = 1;
  }
  float4* s = reinterpret_cast<float4*>(D.lat) + (size_t)m * D.real_stride;
  const float4 w = s[off];
  const double v1 = w.y, v2 = w.z;
  double q[4];
  for (int c = 0; c < 4; ++c) q[c] = u[((size_t)r * 4 + c) * nn + o];
  double u1, u2, p;
  cons_to_prim(q, L.ph.gamma, u1, u2, p);
  const double f[4] = {q[1], q[1] * u1 + p, q[1] * u2, (q[3] + p) * u1};
  const double g[4] = {q[2], q[1] * u2, q[2] * u2 + p, (q[3] + p) * u2};
  const double c1 = (1.0 - L.ph.alpha) / 4.0;
  const bool bnd = node_is_boundary(D, i, j);
  for (int k = 0; k < 4; ++k) {
    double gl[4];
    for (int c = 0; c < 4; ++c) {
      const double F = (k < 2) ? f[c] : g[c];
      const double M = (k % 2 == 0) ? c1 * q[c] + F * inv2a : c1 * q[c] - F * inv2a;
      gl[c] = pops[((size_t)r * 16 + 4 * k + c) * nn + o] - M;
    }
    // boost into the node's rest frame (stored velocity)
    const double gm1 = gl[1] - v1 * gl[0], gm2 = gl[2] - v2 * gl[0];
    const double gE = gl[3] - v1 * gl[1] - v2 * gl[2] + 0.5 * (v1 * v1 + v2 * v2) * gl[0];
    s[(1 + k) * D.plane + off] =
        bnd ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4((float)gl[0], (float)gm1, (float)gm2, (float)gE);
  }
}

inline dim3 node_grid(const LevelDesc& D, int count) {
  const long long n = (long long)D.nx * D.ny;
  return dim3((unsigned)((n + kThreads - 1) / kThreads), (unsigned)count, 1);
}

// A device wait that nothing completes, bounded like every wait of the step
// kernels: one mbarrier expecting 16 bytes that no copy delivers.  The wait
// gives up after limit_ns of %globaltimer, records 4 in *status (the bit the
// step kernels raise) and the kernel returns; no copy is in flight.
__global__ void bounded_wait_probe_kernel(int* status, unsigned long long limit_ns) {
  __shared__ alignas(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(16) : "memory");
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(b), "r"(0)
        : "memory");
    if (ok) {
      *status = 0;
      return;
    }
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) {
      *status = 4;
      return;
    }
  }
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int* status, unsigned long long limit_ns, cudaStream_t s) {
  bounded_wait_probe_kernel<<<1, 32, 0, s>>>(status, limit_ns);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_inlet(const Launch& L, uint64_t seed, int m_begin, const vlbm_perturb& P, const double* xi,
                         double* xi_out, cudaStream_t s) {
  PerturbDev pd{};
  pd.xi = xi;
  pd.r_jet = P.r_jet;
  pd.K = P.K;
  pd.m_begin = m_begin;
  for (int k = 1; k <= P.K; ++k) pd.amp[k - 1] = P.use_amp ? P.amp[k - 1] : P.A * std::pow((double)k, -P.p_decay);
  pd.key0 = (uint32_t)(seed & 0xffffffffu);
  pd.key1 = (uint32_t)(seed >> 32);
  for (int l = 0; l < L.nlevels; ++l) {
    dim3 grid((L.lv[l].ny + kThreads - 1) / kThreads, L.M, 1);
    Launch one = L;
    one.lv[0] = L.lv[l];
    pd.xi_out = (l == 0 && !xi) ? xi_out : nullptr;
    inlet_kernel<<<grid, kThreads, 0, s>>>(one, pd);
    add_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_init_state(const Launch& L, int precision, cudaStream_t s) {
  for (int l = 0; l < L.nlevels; ++l) {
    reset_rs_kernel<<<(L.M + kThreads - 1) / kThreads, kThreads, 0, s>>>(L, l, 0, L.M);
    add_launches(2);
    Launch one = L;
    one.lv[0] = L.lv[l];
    dim3 g = node_grid(L.lv[l], L.M);
    // cons_to_prim of the ambient state at rest reduces exactly to
    // (rho, 0, 0, (gamma - 1) E) with E = p / (gamma - 1) + 0
    const double E = L.ph.amb_p / (L.ph.gamma - 1.0) + 0.0;
    const float4 amb = make_float4((float)L.ph.amb_rho, 0.0f, 0.0f, (float)((L.ph.gamma - 1.0) * E));
    init_state_kernel<<<g, kThreads, 0, s>>>(one, precision, amb);
  }
  return cudaGetLastError();
}

cudaError_t launch_lambda(const Launch& L, int precision, int level, int m0, int count, cudaStream_t s) {
  lambda_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, precision, level, m0);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fill_equilibrium_f64(const Launch& L, int level, int m0, int count, cudaStream_t s) {
  fill_equilibrium_f64_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, level, m0);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_tick(const Launch& L, int precision, int advance, cudaStream_t s) {
  dim3 grid((L.M + 127) / 128, L.nlevels);
  tick_kernel<<<grid, 128, 0, s>>>(L, precision, advance);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_set_target(const Launch& L, double t_target, cudaStream_t s) {
  dim3 grid((L.M + 127) / 128, L.nlevels);
  set_target_kernel<<<grid, 128, 0, s>>>(L, t_target);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_count_active(const Launch& L, int* d_count, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  dim3 grid((L.M + 127) / 128, L.nlevels);
  count_active_kernel<<<grid, 128, 0, s>>>(L, d_count);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_moments(const Launch& L, int precision, int level, int m0, int count, double* rho, double* u,
                           double* v, double* p, cudaStream_t s) {
  moments_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, precision, level, m0, rho, u, v, p);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_density(const Launch& L, int precision, int level, int m0, int count, void* rho, int as_f32,
                           cudaStream_t s) {
  density_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, precision, level, m0, rho, as_f32);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_get_state(const Launch& L, int precision, int level, int m0, int count, double* u, double* pops,
                             cudaStream_t s) {
  get_state_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, precision, level, m0, u, pops);
  add_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_set_state(const Launch& L, int precision, int level, int m0, int count, const double* u,
                             const double* pops, cudaStream_t s) {
  reset_rs_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, s>>>(L, level, m0, count);
  set_state_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, precision, level, m0, u, pops);
  lambda_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, precision, level, m0);
  add_launches(precision == VLBM_MIXED ? 4 : 3);
  if (precision == VLBM_MIXED)
    set_pops_mixed_kernel<<<node_grid(L.lv[level], count), kThreads, 0, s>>>(L, level, m0, u, pops);
  return cudaGetLastError();
}

}  // namespace vlbm
