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

}  // namespace

size_t step_f64_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_step_f64(const Launch& L, cudaStream_t s) {
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
