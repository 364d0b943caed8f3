// FP64 VLBM step: the paper's arithmetic in the lab frame (Sec. 2.1, Eqs.
// (maxwellians12)-(maxwellians34), (vlbm1)-(vlbm5); Sec. 2.2 boundaries).
//
// One CTA advances a TX x TY tile of interior nodes of one realization on one
// level.  Phases (shared memory, radius-2 halo for u, radius-1 for U_LF):
//   P1  u, fluxes f, g of every node of the tile + 2 halo            (Eq. eos)
//   P2  first-order state U_LF = alpha u + M1(W) + M2(E) + M3(S) + M4(N) and
//       the relaxed local density bounds of every node of tile + 1 halo
//   P3  every face touching the tile: d_f, blending parameter theta_f
//       (R-theta limiter), and the two streamed populations it owns
//   P4  every tile node: u^{n+1} by Eq. (vlbm5) in the order it is written,
//       zero-gradient copies, inlet column, lambda for the next kinetic speed
//       (block max + one atomicMax per CTA).
// The translation unit is compiled without FMA contraction and evaluates every
// expression in the oracle's order, so the two agree to round-off.
// FP64 is the slow path on GB300 (1/58 of the FP32 rate): this kernel is
// bound by the FP64 pipe, not by HBM.
#include <cfloat>

#include "vlbm_f64_math.cuh"
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

using namespace f64;

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HX = TX + 4, HY = TY + 4;  // tile + radius-2 halo
constexpr int GX = TX + 2, GY = TY + 2;  // tile + radius-1 halo

struct Smem {
  double u[4][HY][HX];
  double f[4][HY][HX];
  double g[4][HY][HX];
  double ulf[4][GY][GX];
  double bnd[4][GY][GX];  // lo_b, hi_b, eps_rho, eps_p / (gamma - 1)
  // per face: theta, the two non-equilibrium terms M_out(u_L) - u_out,L and
  // M_in(u_R) - u_in,R, and the two streamed populations of Eqs. (vlbm1)-(vlbm4)
  double thx[TY][TX + 1];
  double thy[TY + 1][TX];
  double eox[4][TY][TX + 1], eix[4][TY][TX + 1], nox[4][TY][TX + 1], nix[4][TY][TX + 1];
  double eoy[4][TY + 1][TX], eiy[4][TY + 1][TX], noy[4][TY + 1][TX], niy[4][TY + 1][TX];
  unsigned long long lam[NT / 32];
  int flags[NT / 32];
};

// Writes the conserved state q and its equilibrium populations M_k(q; a).
__device__ __forceinline__ void write_equilibrium_node(double* dst, size_t plane, size_t off,
                                                       const double q[4], double gamma, double c1,
                                                       double inv2a) {
  double f[4], g[4];
  fluxes(q, gamma, f, g);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    dst[c * plane + off] = q[c];
    dst[(4 + 0 * 4 + c) * plane + off] = c1 * q[c] + f[c] * inv2a;
    dst[(4 + 1 * 4 + c) * plane + off] = c1 * q[c] - f[c] * inv2a;
    dst[(4 + 2 * 4 + c) * plane + off] = c1 * q[c] + g[c] * inv2a;
    dst[(4 + 3 * 4 + c) * plane + off] = c1 * q[c] - g[c] * inv2a;
  }
}

__global__ void __launch_bounds__(NT, 1) step_f64_kernel(const Launch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x;

  int tile = blockIdx.x;
  int lvl = 0;
  while (lvl + 1 < L.nlevels && tile >= L.lv[lvl + 1].tile_begin) ++lvl;
  const LevelDesc& D = L.lv[lvl];
  tile -= D.tile_begin;
  const int m = blockIdx.y;
  RealState* rs = D.rs + m;
  if (!rs->active) return;

  const int nx = D.nx, ny = D.ny;
  const size_t plane = D.plane;
  const int nxp = D.nx_pad;
  const int par = (int)(rs->steps & 1);
  const double* __restrict__ src =
      reinterpret_cast<const double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
  double* __restrict__ dst = reinterpret_cast<double*>(D.lat) + ((size_t)(par ^ 1) * L.M + m) * D.real_stride;
  const double inv2a = rs->inv2a;
  const double gamma = L.ph.gamma, alpha = L.ph.alpha;
  const double c1 = (1.0 - alpha) / 4.0;
  const int limiter = L.ph.limiter;

  const int i0 = 1 + (tile % D.tiles_x) * TX;
  const int j0 = 1 + (tile / D.tiles_x) * TY;

  // ---- P1: u, f, g on tile + 2 halo ----------------------------------------
  for (int idx = tid; idx < HX * HY; idx += NT) {
    const int li = idx % HX, lj = idx / HX;
    int gi = i0 - 2 + li, gj = j0 - 2 + lj;
    gi = gi < 0 ? 0 : (gi > nx - 1 ? nx - 1 : gi);
    gj = gj < 0 ? 0 : (gj > ny - 1 ? ny - 1 : gj);
    const size_t off = (size_t)gj * nxp + gi;
    double q[4], f[4], g[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) q[c] = src[c * plane + off];
    fluxes(q, gamma, f, g);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      S.u[c][lj][li] = q[c];
      S.f[c][lj][li] = f[c];
      S.g[c][lj][li] = g[c];
    }
  }
  __syncthreads();

  // ---- P2: U_LF and bounds on tile + 1 halo ---------------------------------
  for (int idx = tid; idx < GX * GY; idx += NT) {
    const int li = idx % GX, lj = idx / GX;
    const int gi = i0 - 1 + li, gj = j0 - 1 + lj;
    if (gi < 1 || gi > nx - 2 || gj < 1 || gj > ny - 2) continue;
    const int hx = li + 1, hy = lj + 1;
    double U[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double M1W = c1 * S.u[c][hy][hx - 1] + S.f[c][hy][hx - 1] * inv2a;
      const double M2E = c1 * S.u[c][hy][hx + 1] - S.f[c][hy][hx + 1] * inv2a;
      const double M3S = c1 * S.u[c][hy - 1][hx] + S.g[c][hy - 1][hx] * inv2a;
      const double M4N = c1 * S.u[c][hy + 1][hx] - S.g[c][hy + 1][hx] * inv2a;
      U[c] = alpha * S.u[c][hy][hx] + M1W + M2E + M3S + M4N;
      S.ulf[c][lj][li] = U[c];
    }
    double lo = S.u[0][hy][hx], hi = lo;
    const double rs5[5] = {S.u[0][hy][hx - 1], S.u[0][hy][hx + 1], S.u[0][hy - 1][hx], S.u[0][hy + 1][hx], U[0]};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
      lo = rs5[r] < lo ? rs5[r] : lo;
      hi = rs5[r] > hi ? rs5[r] : hi;
    }
    const double delta = L.ph.rlmp_rel * (hi - lo) + L.ph.rlmp_abs;
    double v1, v2, pLF;
    primitive(U, gamma, v1, v2, pLF);
    S.bnd[0][lj][li] = lo - delta;
    S.bnd[1][lj][li] = hi + delta;
    S.bnd[2][lj][li] = L.ph.eps_pos < U[0] ? L.ph.eps_pos : U[0];
    S.bnd[3][lj][li] = (L.ph.eps_pos < pLF ? L.ph.eps_pos : pLF) / (gamma - 1.0);
  }
  __syncthreads();

  // ---- P3: faces ------------------------------------------------------------
  constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);
  for (int idx = tid; idx < NXF + NYF; idx += NT) {
    const bool xdir = idx < NXF;
    int fa, fb;  // x-face: fa = face column (0..TX), fb = row; y-face: fa = column, fb = face row
    int iL, jL, iR, jR;
    bool L_in, R_in;
    if (xdir) {
      fa = idx % (TX + 1);
      fb = idx / (TX + 1);
      iL = i0 + fa - 1;
      jL = j0 + fb;
      iR = iL + 1;
      jR = jL;
      if (jL > ny - 2) continue;
      L_in = fa >= 1 && iL <= nx - 2;
      R_in = fa < TX && iR <= nx - 2;
    } else {
      const int k = idx - NXF;
      fa = k % TX;
      fb = k / TX;
      iL = i0 + fa;
      jL = j0 + fb - 1;
      iR = iL;
      jR = jL + 1;
      if (iL > nx - 2) continue;
      L_in = fb >= 1 && jL <= ny - 2;
      R_in = fb < TY && jR <= ny - 2;
    }
    if (!L_in && !R_in) continue;
    const int hxL = iL - i0 + 2, hyL = jL - j0 + 2, hxR = iR - i0 + 2, hyR = jR - j0 + 2;
    const int kout = xdir ? 0 : 2, kin = xdir ? 1 : 3;
    const bool bL = is_boundary(iL, jL, nx, ny), bR = is_boundary(iR, jR, nx, ny);
    const size_t offL = (size_t)jL * nxp + iL, offR = (size_t)jR * nxp + iR;
    double Mo[4], Mi[4], pL[4], pR[4], d[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double FL = xdir ? S.f[c][hyL][hxL] : S.g[c][hyL][hxL];
      const double FR = xdir ? S.f[c][hyR][hxR] : S.g[c][hyR][hxR];
      Mo[c] = c1 * S.u[c][hyL][hxL] + FL * inv2a;
      Mi[c] = c1 * S.u[c][hyR][hxR] - FR * inv2a;
      pL[c] = bL ? Mo[c] : src[(4 + kout * 4 + c) * plane + offL];
      pR[c] = bR ? Mi[c] : src[(4 + kin * 4 + c) * plane + offR];
      d[c] = (Mo[c] - pL[c]) - (Mi[c] - pR[c]);
    }
    double th;
    if (bL && bR) {
      th = 0.0;
    } else if (limiter == 0) {
      th = 0.0;
    } else if (limiter == 1) {
      th = 1.0;
    } else {
      double tL = 1.0, tR = 1.0;
      if (!bL) {
        const int gx = iL - i0 + 1, gy = jL - j0 + 1;
        double U0[4], DD[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          U0[c] = S.ulf[c][gy][gx];
          DD[c] = -4.0 * d[c];
        }
        tL = theta_star_kk(U0, DD, S.bnd[0][gy][gx], S.bnd[1][gy][gx], S.bnd[2][gy][gx], S.bnd[3][gy][gx]);
      }
      if (!bR) {
        const int gx = iR - i0 + 1, gy = jR - j0 + 1;
        double U0[4], DD[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          U0[c] = S.ulf[c][gy][gx];
          DD[c] = 4.0 * d[c];
        }
        tR = theta_star_kk(U0, DD, S.bnd[0][gy][gx], S.bnd[1][gy][gx], S.bnd[2][gy][gx], S.bnd[3][gy][gx]);
      }
      th = tL < tR ? tL : tR;
    }
    // streamed populations owned by this face (Eqs. (vlbm1)-(vlbm4))
    double no[4], ni[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      no[c] = Mo[c] + th * (Mo[c] - pL[c]);
      ni[c] = Mi[c] + th * (Mi[c] - pR[c]);
    }
    if (xdir) {
      S.thx[fb][fa] = th;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        S.eox[c][fb][fa] = Mo[c] - pL[c];
        S.eix[c][fb][fa] = Mi[c] - pR[c];
        S.nox[c][fb][fa] = no[c];
        S.nix[c][fb][fa] = ni[c];
      }
    } else {
      S.thy[fb][fa] = th;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        S.eoy[c][fb][fa] = Mo[c] - pL[c];
        S.eiy[c][fb][fa] = Mi[c] - pR[c];
        S.noy[c][fb][fa] = no[c];
        S.niy[c][fb][fa] = ni[c];
      }
    }
    if (R_in) {
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[(4 + kout * 4 + c) * plane + offR] = no[c];
    }
    if (L_in) {
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[(4 + kin * 4 + c) * plane + offL] = ni[c];
    }
  }
  __syncthreads();

  // ---- P4: macroscopic update, boundaries, lambda ---------------------------
  double lam = 0.0;
  int flags = 0;
  {
    const int lx = tid % TX, ly = tid / TX;
    const int gi = i0 + lx, gj = j0 + ly;
    if (gi <= nx - 2 && gj <= ny - 2) {
      // Eq. (vlbm5) as written: the new populations, alpha u, and the four
      // theta-weighted non-equilibrium terms of the cell itself
      const double thw = S.thx[ly][lx], the = S.thx[ly][lx + 1], ths = S.thy[ly][lx], thn = S.thy[ly + 1][lx];
      double q[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const double n1 = S.nox[c][ly][lx], n2 = S.nix[c][ly][lx + 1];
        const double n3 = S.noy[c][ly][lx], n4 = S.niy[c][ly + 1][lx];
        double v = n1 + n2;
        v = v + n3;
        v = v + n4;
        v = v + alpha * S.u[c][ly + 2][lx + 2];
        v = v - thw * S.eix[c][ly][lx];
        v = v - the * S.eox[c][ly][lx + 1];
        v = v - ths * S.eiy[c][ly][lx];
        v = v - thn * S.eoy[c][ly + 1][lx];
        q[c] = v;
      }
      const size_t off = (size_t)gj * nxp + gi;
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[c * plane + off] = q[c];
      double v1, v2, p;
      primitive(q, gamma, v1, v2, p);
      const bool fin = isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]) && isfinite(q[3]);
      if (!fin) flags |= 2;
      if (!(q[0] > 0.0) || !(p > 0.0)) flags |= 1;
      if (!flags) {
        const double l = fmax(fabs(v1), fabs(v2)) + sqrt(gamma * p / q[0]);
        lam = fmax(lam, l);
      }
      // zero-gradient copies (outlet column, then the first / last rows)
      const bool cx = gi == nx - 2, cyl = gj == 1, cyh = gj == ny - 2;
      if (cx || cyl || cyh) {
        if (cx) write_equilibrium_node(dst, plane, off + 1, q, gamma, c1, inv2a);
        if (cyl) {
          write_equilibrium_node(dst, plane, off - nxp, q, gamma, c1, inv2a);
          if (cx) write_equilibrium_node(dst, plane, off - nxp + 1, q, gamma, c1, inv2a);
        }
        if (cyh) {
          write_equilibrium_node(dst, plane, off + nxp, q, gamma, c1, inv2a);
          if (cx) write_equilibrium_node(dst, plane, off + nxp + 1, q, gamma, c1, inv2a);
        }
      }
      // inlet column (Dirichlet, every row): written by the first interior column
      if (gi == 1) {
        const double* inl = D.inlet + (size_t)m * 4 * ny;
        int rows[3] = {gj, -1, -1};
        if (gj == 1) rows[1] = 0;
        if (gj == ny - 2) rows[2] = ny - 1;
        for (int r = 0; r < 3; ++r) {
          const int jj = rows[r];
          if (jj < 0) continue;
          double qi[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) qi[c] = inl[c * ny + jj];
          write_equilibrium_node(dst, plane, (size_t)jj * nxp, qi, gamma, c1, inv2a);
          double w1, w2, pi;
          primitive(qi, gamma, w1, w2, pi);
          lam = fmax(lam, fmax(fabs(w1), fabs(w2)) + sqrt(gamma * pi / qi[0]));
        }
      }
    }
  }
  // block reduction of lambda and flags
  unsigned long long lb = lam_to_bits(lam);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, lb, o);
    lb = ob > lb ? ob : lb;
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if ((tid & 31) == 0) {
    S.lam[tid >> 5] = lb;
    S.flags[tid >> 5] = flags;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long best = 0;
    int fl = 0;
    for (int w = 0; w < NT / 32; ++w) {
      best = S.lam[w] > best ? S.lam[w] : best;
      fl |= S.flags[w];
    }
    atomicMax(&rs->lam_next_bits, best);
    if (fl) atomicOr(&rs->flags, fl);
  }
}

// ---- warp-marching design ----------------------------------------------------
// A warp owns 28 interior columns (lanes 2..29; lanes 0, 1 and 30, 31 hold the
// halo columns) and marches up D.wrows rows.  Each lane evaluates its own
// node once per row (the state, its fluxes and its four Maxwellians
// M_k(u; a_n)), x-neighbours' values come by warp shuffle, and a sliding
// window of rows stays in registers: the tile design evaluates a node's fluxes
// 1.69 times and U_LF 1.33 times per cell (its halos), this one 1.14 times
// each.  The FP64 pipe executes every lane of a warp instruction, so no lane
// takes extra halo work: with two halo lanes on each side every U_LF and face
// the updated cells need is in the warp.  Every expression is the tile
// design's (and the oracle's), in the same order: the results are identical.
constexpr int kFW = 28;     // columns updated per warp
constexpr int kFNW = 4;     // warps per CTA
constexpr int kFRows = 16;  // target rows per warp

// The state u of a node and its Maxwellians, Eqs. (maxwellians12), (maxwellians34):
// M1 = c1 u + f / 2a, M2 = c1 u - f / 2a, M3 = c1 u + g / 2a, M4 = c1 u - g / 2a.
struct NodeF64 {
  double u[4], M1[4], M2[4], M3[4], M4[4];
};

__device__ __forceinline__ void eval_node(const double* __restrict__ src, size_t plane, size_t off, double gamma,
                                          double c1, double inv2a, NodeF64& n) {
#pragma unroll
  for (int c = 0; c < 4; ++c) n.u[c] = __ldg(src + c * plane + off);
  double f[4], g[4];
  fluxes(n.u, gamma, f, g);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    n.M1[c] = c1 * n.u[c] + f[c] * inv2a;
    n.M2[c] = c1 * n.u[c] - f[c] * inv2a;
    n.M3[c] = c1 * n.u[c] + g[c] * inv2a;
    n.M4[c] = c1 * n.u[c] - g[c] * inv2a;
  }
}

// U_LF of an interior node (Eq. (vlbm5)'s first-order part) and its limits:
// relaxed density bounds, eps_rho, eps_p / (gamma - 1).
__device__ __forceinline__ void node_lf(const double u[4], const double M1W[4], const double M2E[4],
                                        const double M3S[4], const double M4N[4], double rW, double rE, double rS,
                                        double rN, const Physics& ph, double alpha, double gamma, double U[4],
                                        double bnd[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) U[c] = alpha * u[c] + M1W[c] + M2E[c] + M3S[c] + M4N[c];
  double lo = u[0], hi = lo;
  const double rs5[5] = {rW, rE, rS, rN, U[0]};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    lo = rs5[r] < lo ? rs5[r] : lo;
    hi = rs5[r] > hi ? rs5[r] : hi;
  }
  const double delta = ph.rlmp_rel * (hi - lo) + ph.rlmp_abs;
  double v1, v2, pLF;
  primitive(U, gamma, v1, v2, pLF);
  bnd[0] = lo - delta;
  bnd[1] = hi + delta;
  bnd[2] = ph.eps_pos < U[0] ? ph.eps_pos : U[0];
  bnd[3] = (ph.eps_pos < pLF ? ph.eps_pos : pLF) / (gamma - 1.0);
}

// Face (L, R): theta_f, the non-equilibrium terms eo = Mo - pL, ei = Mi - pR
// and the streamed populations no, ni (Eqs. (vlbm1)-(vlbm4)).  Mo = M_out(u_L),
// Mi = M_in(u_R); pLraw, pRraw the stored populations (a boundary node's
// stand in by its equilibrium).
__device__ __forceinline__ void face_f64(const double Mo[4], const double Mi[4], const double pLraw[4],
                                         const double pRraw[4], bool bL, bool bR, const double UL[4],
                                         const double BL[4], const double UR[4], const double BR[4], int limiter,
                                         double& th, double eo[4], double ei[4], double no[4], double ni[4]) {
  double pL[4], pR[4], d[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    pL[c] = bL ? Mo[c] : pLraw[c];
    pR[c] = bR ? Mi[c] : pRraw[c];
    d[c] = (Mo[c] - pL[c]) - (Mi[c] - pR[c]);
  }
  if (bL && bR) {
    th = 0.0;
  } else if (limiter == 0) {
    th = 0.0;
  } else if (limiter == 1) {
    th = 1.0;
  } else {
    double tL = 1.0, tR = 1.0;
    if (!bL) {
      double DD[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) DD[c] = -4.0 * d[c];
      tL = theta_star_kk(UL, DD, BL[0], BL[1], BL[2], BL[3]);
    }
    if (!bR) {
      double DD[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) DD[c] = 4.0 * d[c];
      tR = theta_star_kk(UR, DD, BR[0], BR[1], BR[2], BR[3]);
    }
    th = tL < tR ? tL : tR;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    eo[c] = Mo[c] - pL[c];
    ei[c] = Mi[c] - pR[c];
    no[c] = Mo[c] + th * (Mo[c] - pL[c]);
    ni[c] = Mi[c] + th * (Mi[c] - pR[c]);
  }
}

__device__ __forceinline__ double shup(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shdn(double v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// The limiter's sides of one warp and row (north face L, R; east face L, R):
// their density-limit quotients num / den, the coefficients A, B, C of the
// pressure function, theta before the root, and the results; `items` lists
// the pending sides (side * 32 + lane) of one stage.
struct SideSlots {
  double num[4][32], den[4][32], A[4][32], B[4][32], C[4][32], th[4][32], res[4][32];
  int items[128];
};

// The FP64 pipe executes every lane of a warp instruction, so a division or a
// root that one lane of a warp needs costs the whole warp; evaluated side by
// side, a row pays for up to four of each.  Here the lanes queue the sides
// that need one (pend[s]) and the warp evaluates the queue, one side per lane:
// one pass for up to 32 sides.  root = false: res = num / den; root = true:
// res = theta_root(A, B, C, th).
__device__ __forceinline__ void warp_queue_eval(SideSlots& S, const bool pend[4], int lane, bool root) {
  const unsigned lt = (1u << lane) - 1u;
  int n = 0;
#pragma unroll
  for (int sd = 0; sd < 4; ++sd) {
    const unsigned mk = __ballot_sync(0xffffffffu, pend[sd]);
    if (pend[sd]) S.items[n + __popc(mk & lt)] = sd * 32 + lane;
    n += __popc(mk);
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    const int it = S.items[i], sd = it >> 5, l = it & 31;
    S.res[sd][l] = root ? theta_root(S.A[sd][l], S.B[sd][l], S.C[sd][l], S.th[sd][l]) : S.num[sd][l] / S.den[sd][l];
  }
  __syncwarp();
}

// blockIdx.x = (strip, row chunk) over all levels, blockIdx.y = realization.
__global__ void __launch_bounds__(kFNW * 32, 1) step_f64_march_kernel(const Launch L) {
  __shared__ SideSlots slots[kFNW];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int unit = blockIdx.x, lvl = 0;
  while (lvl + 1 < L.nlevels && unit >= L.lv[lvl + 1].tile_begin) ++lvl;
  const LevelDesc& D = L.lv[lvl];
  unit -= D.tile_begin;
  const int m = blockIdx.y;
  RealState* rs = D.rs + m;
  if (!rs->active) return;
  const int nx = D.nx, ny = D.ny, nxp = D.nx_pad;
  const int ra = 1 + ((unit / D.tiles_x) * kFNW + wid) * D.wrows;
  const int rb = min(ra + D.wrows - 1, ny - 2);
  if (ra > rb) return;
  // lane l holds column 28 strip + l - 1 (lanes 2..29: the strip's columns)
  const int c = (unit % D.tiles_x) * kFW + lane - 1;
  const int cl = c < 0 ? 0 : (c > nx - 1 ? nx - 1 : c);
  const bool upd = lane >= 2 && lane <= kFW + 1 && c <= nx - 2;
  const bool colin = c >= 1 && c <= nx - 2;
  const size_t plane = D.plane;
  const int par = (int)(rs->steps & 1);
  const double* __restrict__ src =
      reinterpret_cast<const double*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
  double* __restrict__ dst = reinterpret_cast<double*>(D.lat) + ((size_t)(par ^ 1) * L.M + m) * D.real_stride;
  const double inv2a = rs->inv2a;
  const double gamma = L.ph.gamma, alpha = L.ph.alpha;
  const double c1 = (1.0 - alpha) / 4.0;
  const int limiter = L.ph.limiter;
  auto off_of = [&](int row) {
    const int r = row < 0 ? 0 : (row > ny - 1 ? ny - 1 : row);
    return (size_t)r * nxp + cl;
  };
  auto pop = [&](int k, int row, double p[4]) {
    const size_t o = off_of(row);
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) p[cc] = __ldg(src + (size_t)(4 + k * 4 + cc) * plane + o);
  };
  // U_LF of row `row` of this lane from the nodes of rows row - 1 (S), row
  // (this one, W/E by shuffle) and row + 1 (N); all lanes take part in the
  // shuffles, only interior nodes' results are used
  auto lf = [&](int row, const NodeF64& S, const NodeF64& C, const NodeF64& N, double U[4], double B[4]) {
    double M1W[4], M2E[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      M1W[cc] = shup(C.M1[cc]);
      M2E[cc] = shdn(C.M2[cc]);
    }
    const double rW = shup(C.u[0]), rE = shdn(C.u[0]);
    if (colin && row >= 1 && row <= ny - 2) node_lf(C.u, M1W, M2E, S.M3, N.M4, rW, rE, S.u[0], N.u[0], L.ph, alpha, gamma, U, B);
  };

  // ---- warm-up: rows ra - 2 .. ra + 1, U_LF of ra - 1 and ra, face (ra - 1, ra)
  NodeF64 nm2, nm1, n0, n1;
  eval_node(src, plane, off_of(ra - 2), gamma, c1, inv2a, nm2);
  eval_node(src, plane, off_of(ra - 1), gamma, c1, inv2a, nm1);
  eval_node(src, plane, off_of(ra), gamma, c1, inv2a, n0);
  eval_node(src, plane, off_of(ra + 1), gamma, c1, inv2a, n1);
  double Um[4] = {0, 0, 0, 0}, Bm[4] = {0, 0, 0, 0}, U0[4] = {0, 0, 0, 0}, B0[4] = {0, 0, 0, 0};
  lf(ra - 1, nm2, nm1, n0, Um, Bm);
  lf(ra, nm1, n0, n1, U0, B0);
  double ths, n3[4], eis[4];
  {
    double pLr[4], pRr[4], eo[4], no_unused[4];
    pop(2, ra - 1, pLr);
    pop(3, ra, pRr);
    face_f64(nm1.M3, n0.M4, pLr, pRr, is_boundary(c, ra - 1, nx, ny), is_boundary(c, ra, nx, ny), Um, Bm, U0, B0,
             limiter, ths, eo, eis, n3, no_unused);
  }

  double lam = 0.0;
  int flags = 0;
  for (int q = ra; q <= rb; ++q) {
    // row q + 2 and U_LF of row q + 1
    NodeF64 n2;
    eval_node(src, plane, off_of(q + 2), gamma, c1, inv2a, n2);
    double U1[4] = {0, 0, 0, 0}, B1[4] = {0, 0, 0, 0};
    lf(q + 1, n0, n1, n2, U1, B1);
    const bool bq = is_boundary(c, q, nx, ny);
    const bool bn = is_boundary(c, q + 1, nx, ny), be = is_boundary(c + 1, q, nx, ny);
    // north face (q, q + 1) and east face (c, c + 1) of row q (its data for
    // the west face of lane + 1): the non-equilibrium terms eo = Mo - pL,
    // ei = Mi - pR (a boundary node's populations stand in by its
    // equilibria), theta_f, and the streamed populations no, ni
    double thn, eon[4], ein[4], non[4], nin[4];
    double the, eoe[4], eie[4], noe[4], nie[4];
    double MiE[4];
    {
      double pN[4], pNr[4], pE[4], p2[4], pEr[4];
      pop(2, q, pN);
      pop(3, q + 1, pNr);
      pop(0, q, pE);
      pop(1, q, p2);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        MiE[cc] = shdn(n0.M2[cc]);
        pEr[cc] = shdn(p2[cc]);
        const double pl = bq ? n0.M3[cc] : pN[cc], pr = bn ? n1.M4[cc] : pNr[cc];
        const double ple = bq ? n0.M1[cc] : pE[cc], pre = be ? MiE[cc] : pEr[cc];
        eon[cc] = n0.M3[cc] - pl;
        ein[cc] = n1.M4[cc] - pr;
        eoe[cc] = n0.M1[cc] - ple;
        eie[cc] = MiE[cc] - pre;
      }
    }
    {
      double UR[4], BR[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        UR[cc] = shdn(U0[cc]);
        BR[cc] = shdn(B0[cc]);
      }
      const bool upd_e = __shfl_down_sync(0xffffffffu, upd, 1) && lane < 31;
      thn = (bq && bn) || limiter == 0 ? 0.0 : 1.0;
      the = (bq && be) || limiter == 0 ? 0.0 : 1.0;
      if (limiter == 2) {
        // sides: 0 north L (this node), 1 north R (row q + 1), 2 east L (this
        // node), 3 east R (lane + 1); a face no updated cell uses is skipped
        SideSlots& S = slots[wid];
        const bool needN = upd && !(bq && bn), needE = (upd || upd_e) && !(bq && be);
        const bool act[4] = {needN && !bq, needN && !bn, needE && !bq, needE && !be};
        bool pend[4];
        {
          const double C0 = theta_c(U0, B0[3]);
          const double Cs[4] = {C0, theta_c(U1, B1[3]), C0, shdn(C0)};
#pragma unroll
          for (int sd = 0; sd < 4; ++sd) {
            const double* U = sd == 0 || sd == 2 ? U0 : (sd == 1 ? U1 : UR);
            const double* B = sd == 0 || sd == 2 ? B0 : (sd == 1 ? B1 : BR);
            const double sg = sd == 0 || sd == 2 ? -4.0 : 4.0;
            double DD[4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) DD[cc] = sg * (sd < 2 ? eon[cc] - ein[cc] : eoe[cc] - eie[cc]);
            ThetaPre t;
            theta_pre(U, DD, B[0], B[1], B[2], B[3], t);
            S.num[sd][lane] = t.num;
            S.den[sd][lane] = t.den;
            S.A[sd][lane] = t.A;
            S.B[sd][lane] = t.B;
            S.C[sd][lane] = Cs[sd];
            pend[sd] = act[sd] && t.divide;
          }
        }
        warp_queue_eval(S, pend, lane, false);
        double t[4];
#pragma unroll
        for (int sd = 0; sd < 4; ++sd) {
          const double th = theta_density(pend[sd], pend[sd] ? S.res[sd][lane] : 0.0);
          t[sd] = 1.0;
          const bool fin = !act[sd] || theta_final(th, S.A[sd][lane], S.B[sd][lane], S.C[sd][lane], &t[sd]);
          S.th[sd][lane] = th;
          pend[sd] = !fin;
        }
        __syncwarp();
        warp_queue_eval(S, pend, lane, true);
#pragma unroll
        for (int sd = 0; sd < 4; ++sd)
          if (pend[sd]) t[sd] = S.res[sd][lane];
        if (needN) thn = t[0] < t[1] ? t[0] : t[1];
        if (needE) the = t[2] < t[3] ? t[2] : t[3];
      }
    }
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      non[cc] = n0.M3[cc] + thn * eon[cc];
      nin[cc] = n1.M4[cc] + thn * ein[cc];
      noe[cc] = n0.M1[cc] + the * eoe[cc];
      nie[cc] = MiE[cc] + the * eie[cc];
    }
    const double thw = shup(the);
    double n1w[4], eiw[4];
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      n1w[cc] = shup(noe[cc]);
      eiw[cc] = shup(eie[cc]);
    }
    if (upd) {
      // Eq. (vlbm5) as written: the new populations, alpha u, and the four
      // theta-weighted non-equilibrium terms of the cell itself
      double qn[4];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        double v = n1w[cc] + nie[cc];
        v = v + n3[cc];
        v = v + nin[cc];
        v = v + alpha * n0.u[cc];
        v = v - thw * eiw[cc];
        v = v - the * eoe[cc];
        v = v - ths * eis[cc];
        v = v - thn * eon[cc];
        qn[cc] = v;
      }
      const size_t off = (size_t)q * nxp + c;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        dst[cc * plane + off] = qn[cc];
        dst[(size_t)(4 + 0 * 4 + cc) * plane + off] = n1w[cc];
        dst[(size_t)(4 + 1 * 4 + cc) * plane + off] = nie[cc];
        dst[(size_t)(4 + 2 * 4 + cc) * plane + off] = n3[cc];
        dst[(size_t)(4 + 3 * 4 + cc) * plane + off] = nin[cc];
      }
      double v1, v2, p;
      primitive(qn, gamma, v1, v2, p);
      const bool fin = isfinite(qn[0]) && isfinite(qn[1]) && isfinite(qn[2]) && isfinite(qn[3]);
      int fl = 0;
      if (!fin) fl |= 2;
      if (!(qn[0] > 0.0) || !(p > 0.0)) fl |= 1;
      if (!fl) {
        const double l = fmax(fabs(v1), fabs(v2)) + sqrt(gamma * p / qn[0]);
        lam = fmax(lam, l);
      }
      flags |= fl;
      // zero-gradient copies (outlet column, then the first / last rows)
      const bool cx = c == nx - 2, cyl = q == 1, cyh = q == ny - 2;
      if (cx || cyl || cyh) {
        if (cx) write_equilibrium_node(dst, plane, off + 1, qn, gamma, c1, inv2a);
        if (cyl) {
          write_equilibrium_node(dst, plane, off - nxp, qn, gamma, c1, inv2a);
          if (cx) write_equilibrium_node(dst, plane, off - nxp + 1, qn, gamma, c1, inv2a);
        }
        if (cyh) {
          write_equilibrium_node(dst, plane, off + nxp, qn, gamma, c1, inv2a);
          if (cx) write_equilibrium_node(dst, plane, off + nxp + 1, qn, gamma, c1, inv2a);
        }
      }
      // inlet column (Dirichlet, every row): written by the first interior column
      if (c == 1) {
        const double* inl = D.inlet + (size_t)m * 4 * ny;
        int rows[3] = {q, -1, -1};
        if (q == 1) rows[1] = 0;
        if (q == ny - 2) rows[2] = ny - 1;
        for (int r = 0; r < 3; ++r) {
          const int jj = rows[r];
          if (jj < 0) continue;
          double qi[4];
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) qi[cc] = inl[cc * ny + jj];
          write_equilibrium_node(dst, plane, (size_t)jj * nxp, qi, gamma, c1, inv2a);
          double w1, w2, pi;
          primitive(qi, gamma, w1, w2, pi);
          lam = fmax(lam, fmax(fabs(w1), fabs(w2)) + sqrt(gamma * pi / qi[0]));
        }
      }
    }
    // slide the window
    n0 = n1;
    n1 = n2;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      U0[cc] = U1[cc];
      B0[cc] = B1[cc];
      n3[cc] = non[cc];
      eis[cc] = ein[cc];
    }
    ths = thn;
  }
  // lambda >= 0: its FP64 bit pattern orders like an unsigned integer
  unsigned long long lb = lam_to_bits(lam);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, lb, o);
    lb = ob > lb ? ob : lb;
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if (lane == 0) {
    atomicMax(&rs->lam_next_bits, lb);
    if (flags) atomicOr(&rs->flags, flags);
  }
}

// Strips of kFW columns, rows in chunks of kFNW warps with about kFRows rows
// per warp (fewer, down to 4, when the launch would not give every SM two
// CTAs); the split changes no result.
cudaError_t launch_march_f64(const Launch& Lin, cudaStream_t s) {
  static thread_local Launch L;
  L = Lin;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int target = kFRows;
  for (;;) {
    long long ctas = 0;
    for (int l = 0; l < L.nlevels; ++l) {
      const LevelDesc& D = L.lv[l];
      const int rows = D.ny - 2;
      ctas += (long long)((D.nx - 2 + kFW - 1) / kFW) * ((rows + kFNW * target - 1) / (kFNW * target));
    }
    if (ctas * L.M >= 2LL * sms || target <= 4) break;
    target = target / 2 < 4 ? 4 : target / 2;
  }
  int units = 0;
  for (int l = 0; l < L.nlevels; ++l) {
    LevelDesc& D = L.lv[l];
    const int rows = D.ny - 2;
    const int chunks = (rows + kFNW * target - 1) / (kFNW * target);
    D.tiles_x = (D.nx - 2 + kFW - 1) / kFW;
    D.tiles_y = chunks;
    D.wrows = (rows + chunks * kFNW - 1) / (chunks * kFNW);
    D.tile_begin = units;
    units += D.tiles_x * D.tiles_y;
  }
  L.total_tiles = units;
  step_f64_march_kernel<<<dim3(units, L.M), kFNW * 32, 0, s>>>(L);
  add_launches(1);
  return cudaGetLastError();
}

}  // namespace

size_t step_f64_smem_bytes() { return sizeof(Smem); }

int f64_variants() { return 2; }

const char* f64_variant_name(int v) { return v == 0 ? "tile32x8" : v == 1 ? "march28x4w" : "?"; }

cudaError_t launch_step_f64(const Launch& L, int variant, cudaStream_t s) {
  if (variant != 0) return launch_march_f64(L, s);
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = once_per_device(configured, [] {
    return cudaFuncSetAttribute(step_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  });
  if (e != cudaSuccess) return e;
  dim3 grid(L.total_tiles, L.M);
  step_f64_kernel<<<grid, NT, sizeof(Smem), s>>>(L);
  add_launches(1);
  return cudaGetLastError();
}

void tiles_f64(int nx, int ny, int* tx, int* ty) {
  *tx = (nx - 2 + TX - 1) / TX;
  *ty = (ny - 2 + TY - 1) / TY;
}

}  // namespace vlbm
