// FP32 VLBM step evaluated in each node's rest frame (VLBM_MIXED).
//
// The paper's update (Sec. 2.1, Eqs. (vlbm1)-(vlbm5)) acts on the lab-frame
// conserved state.  At Mach 2000 the kinetic energy exceeds the internal energy
// by ~2.6e6, so recovering p from E - |m|^2/(2 rho) (Eq. (eos)) in FP32 loses
// the pressure entirely.  This kernel instead stores the nodal state as
// (rho, v1, v2, p) and the non-equilibrium parts g_k = u_k - M_k(u) boosted
// into the node's own rest frame, and evaluates every update in the frame
// moving with the node being updated.  It relies on two exact identities of
// the Galilean boost B_w u = (rho, m - rho w, E - m.w + rho |w|^2 / 2):
//   B_w f(u) = f(B_w u) + w1 B_w u,   B_w g(u) = g(B_w u) + w2 B_w u,
// so B_w M_1(u) = c1 B_w u + (f(B_w u) + w1 B_w u) / (2a) (likewise M_2..M_4),
// and the internal energy is frame invariant.  In the cell's frame every term
// is of the size of the local velocity differences and the internal energy,
// so FP32 keeps p to FP32 relative accuracy: no FP64 in the loop (GB300's
// FP64 rate is 1/58 of FP32).
//
// Tile phases as in the FP64 kernel: P1 nodal states (radius-2 halo), P2
// first-order state U_LF and bounds in each node's frame (radius-1 halo), P3
// faces (theta_f with the R-theta limiter in both cells' frames), P4 update,
// new rest-frame non-equilibrium parts, boundaries and lambda.
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int HX = TX + 4, HY = TY + 4;
constexpr int GX = TX + 2, GY = TY + 2;

struct Smem {
  float4 P[HY][HX];      // (rho, v1, v2, p) of tile + 2 halo
  float4 U[GY][GX];      // U_LF in the node's own frame, tile + 1 halo
  float4 B[GY][GX];      // lo_b, hi_b, eps_rho, eps_p
  float4 gLx[TY][TX + 1];  // x faces: g'_1(L) (a_n), L frame
  float4 gRx[TY][TX + 1];  //          g'_2(R) (a_n), R frame
  float4 gLy[TY + 1][TX];  // y faces: g'_3(L), L frame
  float4 gRy[TY + 1][TX];  //          g'_4(R), R frame
  float thx[TY][TX + 1];
  float thy[TY + 1][TX];
  unsigned lam[NT / 32];
  int flags[NT / 32];
};

struct Ctx {
  float gamma, gm1, rg;  // gamma, gamma - 1, 1 / (gamma - 1)
  float alpha, c1;
  float h;               // 1 / (2 a_n), FP32 (rounded down)
  float rel, absb, eps;
};

// B_w u of a node with primitive state P; d = velocity relative to w.
__device__ __forceinline__ float4 boosted(const float4 P, float w1, float w2, const Ctx& k, float& d1, float& d2) {
  d1 = P.y - w1;
  d2 = P.z - w2;
  const float r = P.x;
  return make_float4(r, r * d1, r * d2, P.w * k.rg + 0.5f * r * (d1 * d1 + d2 * d2));
}

// Boosted lab fluxes B_w f(u) = f(u') + w1 u' and B_w g(u) = g(u') + w2 u'.
__device__ __forceinline__ float4 xflux(const float4 u, float d1, float d2, float p, float w1) {
  return make_float4(u.y + w1 * u.x, u.y * d1 + p + w1 * u.y, u.y * d2 + w1 * u.z, (u.w + p) * d1 + w1 * u.w);
}
__device__ __forceinline__ float4 yflux(const float4 u, float d1, float d2, float p, float w2) {
  return make_float4(u.z + w2 * u.x, u.y * d2 + w2 * u.y, u.z * d2 + p + w2 * u.z, (u.w + p) * d2 + w2 * u.w);
}

// Boost of a rest-frame vector x by dw = w_new - w_old.
__device__ __forceinline__ float4 boost(const float4 x, float dw1, float dw2) {
  const float m1 = x.y - dw1 * x.x, m2 = x.z - dw2 * x.x;
  const float E = x.w - (dw1 * x.y + dw2 * x.z) + 0.5f * (dw1 * dw1 + dw2 * dw2) * x.x;
  return make_float4(x.x, m1, m2, E);
}

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ float4 add(float4 a, float4 b) { return f4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 sub(float4 a, float4 b) { return f4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 axpy(float s, float4 x, float4 y) {
  return f4(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y), fmaf(s, x.z, y.z), fmaf(s, x.w, y.w));
}

// d_f = [M_out(u_L) - u_out,L] - [M_in(u_R) - u_in,R] = g_in(R) - g_out(L)
// (g = u_k - M_k), seen in L's frame and in R's frame.
__device__ __forceinline__ float4 d_in_L(const float4 gL, const float4 gR, float4 PL, float4 PR) {
  return sub(boost(gR, PL.y - PR.y, PL.z - PR.z), gL);
}
__device__ __forceinline__ float4 d_in_R(const float4 gL, const float4 gR, float4 PL, float4 PR) {
  return sub(gR, boost(gL, PR.y - PL.y, PR.z - PL.z));
}

// Largest theta in [0, 1] keeping U0 + theta D admissible and inside the
// relaxed density bounds; the same convex-set argument as the FP64 rule, in
// the cell's rest frame (no cancellation in the pressure quadratic).
__device__ float theta_star(const float4 U0, const float4 D, const float4 Bd, const Ctx& k) {
  float th = 1.0f;
  const float lower = fmaxf(Bd.z, Bd.x);
  if (D.x < 0.0f) {
    th = fminf(th, (U0.x - lower) / (-D.x));
  } else if (D.x > 0.0f) {
    th = fminf(th, (Bd.y - U0.x) / D.x);
  }
  th = fmaxf(th, 0.0f);
  const float kk = Bd.w * k.rg;
  const float C = U0.x * U0.w - 0.5f * (U0.y * U0.y + U0.z * U0.z) - kk * U0.x;
  const float Bq = U0.x * D.w + D.x * U0.w - (U0.y * D.y + U0.z * D.z) - kk * D.x;
  const float A = D.x * D.w - 0.5f * (D.y * D.y + D.z * D.z);
  const float qth = C + th * (Bq + th * A);
  if (qth >= 0.0f) return th;
  if (C <= 0.0f) return 0.0f;
  float r;
  if (A == 0.0f) {
    r = -C / Bq;
  } else {
    const float disc = fmaxf(Bq * Bq - 4.0f * A * C, 0.0f);
    const float sq = sqrtf(disc);
    const float Q = -0.5f * (Bq + copysignf(sq, Bq));
    if (Q == 0.0f) return 0.0f;
    const float r1 = Q / A, r2 = C / Q;
    r = -1.0f;
    if (r1 > 0.0f) r = r1;
    if (r2 > 0.0f && (r < 0.0f || r2 < r)) r = r2;
    if (r < 0.0f) return 0.0f;
  }
  return fminf(fmaxf(r, 0.0f), th);
}

__device__ __forceinline__ bool is_boundary(int i, int j, int nx, int ny) {
  return i == 0 || i == nx - 1 || j == 0 || j == ny - 1;
}

// non-equilibrium part g'_k(a_n) of an interior node: stored part plus the
// exact change of its equilibrium from a_prev to a_n, B_v F(u) (1/2a_prev - 1/2a_n)
// with B_v f(u) = (rho v1, p, 0, v1 rho e) and B_v g(u) = (rho v2, 0, p, v2 rho e).
__device__ __forceinline__ float4 corrected(float4 g, const float4 P, int k, float dinv, const Ctx& c) {
  const float re = P.w * c.rg;
  float4 F = (k < 2) ? f4(P.x * P.y, P.w, 0.0f, P.y * re) : f4(P.x * P.z, 0.0f, P.w, P.z * re);
  const float s = (k % 2 == 0) ? dinv : -dinv;
  return axpy(s, F, g);
}

__global__ void __launch_bounds__(NT, 4) step_mixed_kernel(const Launch L) {
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

  const int nx = D.nx, ny = D.ny, nxp = D.nx_pad;
  const size_t plane = D.plane;
  const int par = (int)(rs->steps & 1);
  const float4* __restrict__ src =
      reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
  float4* __restrict__ dst = reinterpret_cast<float4*>(D.lat) + ((size_t)(par ^ 1) * L.M + m) * D.real_stride;

  Ctx k;
  k.gamma = L.pf.gamma;
  k.gm1 = L.pf.gm1;
  k.rg = L.pf.rg;
  k.alpha = L.pf.alpha;
  k.c1 = L.pf.c1;
  k.h = rs->inv2a_f;
  k.rel = L.pf.rel;
  k.absb = L.pf.absb;
  k.eps = L.pf.eps;
  const float dinv = rs->dinv2a_f;
  const int limiter = L.ph.limiter;

  const int i0 = 1 + (tile % D.tiles_x) * TX;
  const int j0 = 1 + (tile / D.tiles_x) * TY;

  // ---- P1 -------------------------------------------------------------------
  for (int idx = tid; idx < HX * HY; idx += NT) {
    const int li = idx % HX, lj = idx / HX;
    int gi = i0 - 2 + li, gj = j0 - 2 + lj;
    gi = gi < 0 ? 0 : (gi > nx - 1 ? nx - 1 : gi);
    gj = gj < 0 ? 0 : (gj > ny - 1 ? ny - 1 : gj);
    S.P[lj][li] = src[(size_t)gj * nxp + gi];
  }
  __syncthreads();

  // ---- P2: U_LF in each node's own frame, bounds ----------------------------
  for (int idx = tid; idx < GX * GY; idx += NT) {
    const int li = idx % GX, lj = idx / GX;
    const int gi = i0 - 1 + li, gj = j0 - 1 + lj;
    if (gi < 1 || gi > nx - 2 || gj < 1 || gj > ny - 2) continue;
    const int hx = li + 1, hy = lj + 1;
    const float4 Pc = S.P[hy][hx];
    const float w1 = Pc.y, w2 = Pc.z;
    float d1, d2;
    const float4 PW = S.P[hy][hx - 1], PE = S.P[hy][hx + 1], PS = S.P[hy - 1][hx], PN = S.P[hy + 1][hx];
    const float4 uW = boosted(PW, w1, w2, k, d1, d2);
    const float4 FW = xflux(uW, d1, d2, PW.w, w1);
    const float4 uE = boosted(PE, w1, w2, k, d1, d2);
    const float4 FE = xflux(uE, d1, d2, PE.w, w1);
    const float4 uS = boosted(PS, w1, w2, k, d1, d2);
    const float4 GS = yflux(uS, d1, d2, PS.w, w2);
    const float4 uN = boosted(PN, w1, w2, k, d1, d2);
    const float4 GN = yflux(uN, d1, d2, PN.w, w2);
    const float4 sumu = add(add(uW, uE), add(uS, uN));
    const float4 sumF = add(sub(FW, FE), sub(GS, GN));
    float4 U = axpy(k.h, sumF, f4(k.c1 * sumu.x, k.c1 * sumu.y, k.c1 * sumu.z, k.c1 * sumu.w));
    if (k.alpha != 0.0f) U = add(U, f4(k.alpha * Pc.x, 0.0f, 0.0f, k.alpha * Pc.w * k.rg));
    S.U[lj][li] = U;
    float lo = fminf(fminf(Pc.x, fminf(PW.x, PE.x)), fminf(fminf(PS.x, PN.x), U.x));
    float hi = fmaxf(fmaxf(Pc.x, fmaxf(PW.x, PE.x)), fmaxf(fmaxf(PS.x, PN.x), U.x));
    const float delta = k.rel * (hi - lo) + k.absb;
    const float pLF = k.gm1 * (U.w - 0.5f * (U.y * U.y + U.z * U.z) / U.x);
    // FP32 floors: a relative margin of 1e-5 keeps the final average
    // admissible despite FP32 rounding (the FP64 rule uses eps_pos alone).
    const float er = fminf(U.x, fmaxf(k.eps, 1e-5f * U.x));
    const float ep = fminf(pLF, fmaxf(k.eps, 1e-5f * pLF));
    S.B[lj][li] = f4(lo - delta, hi + delta, er, ep);
  }
  __syncthreads();

  // ---- P3: faces -------------------------------------------------------------
  constexpr int NXF = (TX + 1) * TY, NYF = TX * (TY + 1);
  for (int idx = tid; idx < NXF + NYF; idx += NT) {
    const bool xdir = idx < NXF;
    int fa, fb, iL, jL, iR, jR;
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
      const int q = idx - NXF;
      fa = q % TX;
      fb = q / TX;
      iL = i0 + fa;
      jL = j0 + fb - 1;
      iR = iL;
      jR = jL + 1;
      if (iL > nx - 2) continue;
      L_in = fb >= 1 && jL <= ny - 2;
      R_in = fb < TY && jR <= ny - 2;
    }
    if (!L_in && !R_in) continue;
    const int kout = xdir ? 0 : 2, kin = xdir ? 1 : 3;
    const bool bL = is_boundary(iL, jL, nx, ny), bR = is_boundary(iR, jR, nx, ny);
    const float4 PL = S.P[jL - j0 + 2][iL - i0 + 2], PR = S.P[jR - j0 + 2][iR - i0 + 2];
    const float4 zero = f4(0.f, 0.f, 0.f, 0.f);
    const float4 gL = bL ? zero : corrected(src[(1 + kout) * plane + (size_t)jL * nxp + iL], PL, kout, dinv, k);
    const float4 gR = bR ? zero : corrected(src[(1 + kin) * plane + (size_t)jR * nxp + iR], PR, kin, dinv, k);
    float th;
    if (bL && bR) {
      th = 0.0f;
    } else if (limiter == 0) {
      th = 0.0f;
    } else if (limiter == 1) {
      th = 1.0f;
    } else {
      float tL = 1.0f, tR = 1.0f;
      if (!bL) {
        const float4 dL = d_in_L(gL, gR, PL, PR);
        const int gx = iL - i0 + 1, gy = jL - j0 + 1;
        tL = theta_star(S.U[gy][gx], f4(-4.f * dL.x, -4.f * dL.y, -4.f * dL.z, -4.f * dL.w), S.B[gy][gx], k);
      }
      if (!bR) {
        const float4 dR = d_in_R(gL, gR, PL, PR);
        const int gx = iR - i0 + 1, gy = jR - j0 + 1;
        tR = theta_star(S.U[gy][gx], f4(4.f * dR.x, 4.f * dR.y, 4.f * dR.z, 4.f * dR.w), S.B[gy][gx], k);
      }
      th = fminf(tL, tR);
    }
    if (xdir) {
      S.thx[fb][fa] = th;
      S.gLx[fb][fa] = gL;
      S.gRx[fb][fa] = gR;
    } else {
      S.thy[fb][fa] = th;
      S.gLy[fb][fa] = gL;
      S.gRy[fb][fa] = gR;
    }
  }
  __syncthreads();

  // ---- P4: update, new non-equilibrium parts, boundaries, lambda ------------
  float lam = 0.0f;
  int flags = 0;
  {
    const int lx = tid % TX, ly = tid / TX;
    const int gi = i0 + lx, gj = j0 + ly;
    if (gi <= nx - 2 && gj <= ny - 2) {
      const int hx = lx + 2, hy = ly + 2;
      const float4 Pc = S.P[hy][hx];
      const float4 PW = S.P[hy][hx - 1], PE = S.P[hy][hx + 1], PS = S.P[hy - 1][hx], PN = S.P[hy + 1][hx];
      const float thW = S.thx[ly][lx], thE = S.thx[ly][lx + 1], thS = S.thy[ly][lx], thN = S.thy[ly + 1][lx];
      const float4 g1W = S.gLx[ly][lx], g2c = S.gRx[ly][lx];
      const float4 g1c = S.gLx[ly][lx + 1], g2E = S.gRx[ly][lx + 1];
      const float4 g3S = S.gLy[ly][lx], g4c = S.gRy[ly][lx];
      const float4 g3c = S.gLy[ly + 1][lx], g4N = S.gRy[ly + 1][lx];
      float4 U = S.U[ly + 1][lx + 1];
      U = axpy(thW, d_in_R(g1W, g2c, PW, Pc), U);
      U = axpy(-thE, d_in_L(g1c, g2E, Pc, PE), U);
      U = axpy(thS, d_in_R(g3S, g4c, PS, Pc), U);
      U = axpy(-thN, d_in_L(g3c, g4N, Pc, PN), U);
      // new nodal state (rest frame of the old velocity -> primitive)
      const float rn = U.x;
      const float inv = 1.0f / rn;
      const float dv1 = U.y * inv, dv2 = U.z * inv;
      const float ren = U.w - 0.5f * (U.y * dv1 + U.z * dv2);
      const float pn = k.gm1 * ren;
      const float wn1 = Pc.y + dv1, wn2 = Pc.z + dv2;
      const float4 Pn = f4(rn, wn1, wn2, pn);
      const size_t off = (size_t)gj * nxp + gi;
      dst[off] = Pn;
      if (!(isfinite(rn) && isfinite(wn1) && isfinite(wn2) && isfinite(pn))) flags |= 2;
      if (!(rn > 0.0f) || !(pn > 0.0f)) flags |= 1;
      if (!flags) lam = fmaxf(lam, fmaxf(fabsf(wn1), fabsf(wn2)) + sqrtf(k.gamma * pn / rn));
      // new non-equilibrium parts in the new rest frame (velocity wn):
      // g_k^{n+1} = M_k(u_X) - M_k(u^{n+1}) - theta_f g_k(X), Eqs. (vlbm1)-(vlbm4)
      {
        const float4 un = f4(rn, 0.0f, 0.0f, ren);
        float d1, d2;
        // k = 1, upwind W
        {
          const float4 uX = boosted(PW, wn1, wn2, k, d1, d2);
          const float4 dF = sub(xflux(uX, d1, d2, PW.w, wn1), f4(wn1 * rn, pn, 0.0f, wn1 * ren));
          const float4 du = sub(uX, un);
          float4 g = axpy(k.h, dF, f4(k.c1 * du.x, k.c1 * du.y, k.c1 * du.z, k.c1 * du.w));
          g = axpy(-thW, boost(g1W, wn1 - PW.y, wn2 - PW.z), g);
          dst[1 * plane + off] = g;
        }
        // k = 2, upwind E
        {
          const float4 uX = boosted(PE, wn1, wn2, k, d1, d2);
          const float4 dF = sub(xflux(uX, d1, d2, PE.w, wn1), f4(wn1 * rn, pn, 0.0f, wn1 * ren));
          const float4 du = sub(uX, un);
          float4 g = axpy(-k.h, dF, f4(k.c1 * du.x, k.c1 * du.y, k.c1 * du.z, k.c1 * du.w));
          g = axpy(-thE, boost(g2E, wn1 - PE.y, wn2 - PE.z), g);
          dst[2 * plane + off] = g;
        }
        // k = 3, upwind S
        {
          const float4 uX = boosted(PS, wn1, wn2, k, d1, d2);
          const float4 dG = sub(yflux(uX, d1, d2, PS.w, wn2), f4(wn2 * rn, 0.0f, pn, wn2 * ren));
          const float4 du = sub(uX, un);
          float4 g = axpy(k.h, dG, f4(k.c1 * du.x, k.c1 * du.y, k.c1 * du.z, k.c1 * du.w));
          g = axpy(-thS, boost(g3S, wn1 - PS.y, wn2 - PS.z), g);
          dst[3 * plane + off] = g;
        }
        // k = 4, upwind N
        {
          const float4 uX = boosted(PN, wn1, wn2, k, d1, d2);
          const float4 dG = sub(yflux(uX, d1, d2, PN.w, wn2), f4(wn2 * rn, 0.0f, pn, wn2 * ren));
          const float4 du = sub(uX, un);
          float4 g = axpy(-k.h, dG, f4(k.c1 * du.x, k.c1 * du.y, k.c1 * du.z, k.c1 * du.w));
          g = axpy(-thN, boost(g4N, wn1 - PN.y, wn2 - PN.z), g);
          dst[4 * plane + off] = g;
        }
      }
      // zero-gradient copies: nodal state, equilibrium populations (g' = 0)
      const bool cx = gi == nx - 2, cyl = gj == 1, cyh = gj == ny - 2;
      if (cx || cyl || cyh) {
        const float4 z = f4(0.f, 0.f, 0.f, 0.f);
        size_t outs[5];
        int no = 0;
        if (cx) outs[no++] = off + 1;
        if (cyl) {
          outs[no++] = off - nxp;
          if (cx) outs[no++] = off - nxp + 1;
        }
        if (cyh) {
          outs[no++] = off + nxp;
          if (cx) outs[no++] = off + nxp + 1;
        }
        for (int o = 0; o < no; ++o) {
          dst[outs[o]] = Pn;
          for (int q = 1; q <= 4; ++q) dst[q * plane + outs[o]] = z;
        }
      }
      // inlet column (Dirichlet datum, equilibrium populations)
      if (gi == 1) {
        const double* inl = D.inlet + (size_t)m * 4 * ny;
        int rows[3] = {gj, -1, -1};
        if (gj == 1) rows[1] = 0;
        if (gj == ny - 2) rows[2] = ny - 1;
        for (int r = 0; r < 3; ++r) {
          const int jj = rows[r];
          if (jj < 0) continue;
          const double q0 = inl[jj], q1 = inl[ny + jj], q2 = inl[2 * ny + jj], q3 = inl[3 * ny + jj];
          const double u1 = q1 / q0, u2 = q2 / q0;
          const double pi = (L.ph.gamma - 1.0) * (q3 - 0.5 * q0 * (u1 * u1 + u2 * u2));
          const float4 Pi = f4((float)q0, (float)u1, (float)u2, (float)pi);
          const size_t oi = (size_t)jj * nxp;
          dst[oi] = Pi;
          for (int q = 1; q <= 4; ++q) dst[q * plane + oi] = f4(0.f, 0.f, 0.f, 0.f);
          lam = fmaxf(lam, fmaxf(fabsf(Pi.y), fabsf(Pi.z)) + sqrtf(k.gamma * Pi.w / Pi.x));
        }
      }
    }
  }
  // lambda >= 0: its FP32 bit pattern orders like an unsigned integer
  unsigned lb = __float_as_uint(lam);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lb = max(lb, __shfl_xor_sync(0xffffffffu, lb, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if ((tid & 31) == 0) {
    S.lam[tid >> 5] = lb;
    S.flags[tid >> 5] = flags;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned best = 0;
    int fl = 0;
    for (int w = 0; w < NT / 32; ++w) {
      best = max(best, S.lam[w]);
      fl |= S.flags[w];
    }
    // one FP32 -> FP64 conversion per CTA
    atomicMax(&rs->lam_next_bits, lam_to_bits((double)__uint_as_float(best)));
    if (fl) atomicOr(&rs->flags, fl);
  }
}

}  // namespace

size_t step_mixed_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_step_mixed(const Launch& L, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid(L.total_tiles, L.M);
  step_mixed_kernel<<<grid, NT, sizeof(Smem), s>>>(L);
  add_launches(1);
  return cudaGetLastError();
}

void tiles_mixed(int nx, int ny, int* tx, int* ty) {
  *tx = (nx - 2 + TX - 1) / TX;
  *ty = (ny - 2 + TY - 1) / TY;
}

}  // namespace vlbm
