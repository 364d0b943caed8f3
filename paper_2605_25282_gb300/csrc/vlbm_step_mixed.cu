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
// One CTA advances a 32 x TY tile of one realization on one level:
//   load  one elected thread issues two TMA tensor loads on an mbarrier: the
//         nodal states of the tile + radius-2 halo, and the four
//         non-equilibrium planes of the tile + radius-1 halo
//   P2    first-order state U_LF and relaxed density bounds of every node of
//         the tile + radius-1 halo, each in its own rest frame; the four
//         boosted upwind Maxwellians of every tile cell are kept
//   P3    every face touching the tile: the exact a_{n-1} -> a_n change of its
//         two non-equilibrium parts, theta_f (R-theta limiter, evaluated in
//         both cells' frames; a division-free test covers the common case)
//         and theta_f d_f in both frames
//   P4    update (Eq. (vlbm5) regrouped per face, in the cell's frame), new
//         nodal state, new rest-frame non-equilibrium parts (Eqs. (vlbm1)-(vlbm4))
//         from the kept Maxwellians and theta_f d_f, zero-gradient copies,
//         inlet column, lambda for a_{n+1}.
// Every wait on the mbarrier is bounded; a CTA that gives up raises flag 4 on
// its realization and returns.
#include <cudaTypedefs.h>

#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int TX = 32;

// Limits of theta_star at a node with first-order state U: room below and
// above its density bounds (rho_LF - lower bound, upper bound - rho_LF, both
// >= 0), its energy less the pressure floor Ek = E_LF - eps_p / (gamma - 1),
// and the pressure function q(0) = rho Ek - |m|^2 / 2 of U itself.
struct Bnd {
  float gap_lo, gap_hi, Ek, C;
};

template <int TY>
struct Boxes {
  static constexpr int HX = TX + 4, HY = TY + 4, GX = TX + 2, GY = TY + 2;
  alignas(128) float4 P[HY][HX];     // TMA box: (rho, v1, v2, p), tile + 2 halo
  alignas(128) float4 G[4][GY][GX];  // TMA box: g'_k, tile + 1 halo
};

template <int TY>
struct Work {
  static constexpr int GX = TX + 2, GY = TY + 2;
  float4 U[GY][GX];                  // U_LF in the node's own frame
  Bnd B[GY][GX];                     // theta limits of the node (see node_p2)
  float4 Mk[4][TY][TX];              // B_vc M_k(u_upwind) of every tile cell (frame of the cell)
  float4 tdLx[TY][TX + 1], tdRx[TY][TX + 1];  // theta_f d_f in L's / R's frame, x faces
  float4 tdLy[TY + 1][TX], tdRy[TY + 1][TX];  // same, y faces
  float thx[TY][TX + 1];
  float thy[TY + 1][TX];
  unsigned lam[TX * TY / 32];
  int flags[TX * TY / 32];
};

// one tile per CTA
template <int TY>
struct SmemTile {
  Boxes<TY> box;
  Work<TY> w;
  alignas(8) unsigned long long bar;
};

// persistent CTA: tile k and the prefetch of tile k + 1
template <int TY>
struct SmemPersist {
  Boxes<TY> buf[2];
  Work<TY> w;
  int issued[2];  // a TMA load is in flight for buf[b]
  alignas(8) unsigned long long bar[2];
};

struct Ctx {
  float gamma, gm1, rg;
  float alpha, c1;
  float h;
  float rel, absb, eps;
};

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
// Component-wise float4 arithmetic on packed FP32 pairs (sm_100 and later):
// each packed operation is, per component, the same IEEE operation as its
// scalar form (a - b = a + (-b) exactly), so results are unchanged and each
// float4 operation issues two instructions instead of four.
__device__ __forceinline__ float2 lo2(const float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(const float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 cat4(const float2 l, const float2 h) { return f4(l.x, l.y, h.x, h.y); }
__device__ __forceinline__ float4 add(float4 a, float4 b) {
  return cat4(__fadd2_rn(lo2(a), lo2(b)), __fadd2_rn(hi2(a), hi2(b)));
}
__device__ __forceinline__ float4 sub(float4 a, float4 b) {
  return cat4(__fadd2_rn(lo2(a), make_float2(-b.x, -b.y)), __fadd2_rn(hi2(a), make_float2(-b.z, -b.w)));
}
__device__ __forceinline__ float4 scale(float s, float4 x) {
  const float2 ss = make_float2(s, s);
  return cat4(__fmul2_rn(ss, lo2(x)), __fmul2_rn(ss, hi2(x)));
}
__device__ __forceinline__ float4 axpy(float s, float4 x, float4 y) {
  const float2 ss = make_float2(s, s);
  return cat4(__ffma2_rn(ss, lo2(x), lo2(y)), __ffma2_rn(ss, hi2(x), hi2(y)));
}

// Boost of a rest-frame vector x by dw = w_new - w_old.
__device__ __forceinline__ float4 boost(const float4 x, float dw1, float dw2) {
  const float m1 = fmaf(-dw1, x.x, x.y), m2 = fmaf(-dw2, x.x, x.z);
  const float E = fmaf(0.5f * fmaf(dw1, dw1, dw2 * dw2), x.x, x.w - fmaf(dw1, x.y, dw2 * x.z));
  return f4(x.x, m1, m2, E);
}

// d_f = [M_out(u_L) - u_out,L] - [M_in(u_R) - u_in,R] = g_in(R) - g_out(L)
// (g = u_k - M_k), seen in L's frame (gR boosted by w = v_L - v_R) and in R's
// frame (gL boosted by -w); the two boosts share w and |w|^2 / 2 (the values
// are those of boost() with each side's own velocity difference, exactly:
// a - b = -(b - a) in IEEE arithmetic).
__device__ __forceinline__ void d_in_both(const float4 gL, const float4 gR, const float4 PL, const float4 PR,
                                          float4& dL, float4& dR) {
  const float w1 = PL.y - PR.y, w2 = PL.z - PR.z;
  const float hw = 0.5f * fmaf(w1, w1, w2 * w2);
  dL = sub(f4(gR.x, fmaf(-w1, gR.x, gR.y), fmaf(-w2, gR.x, gR.z), fmaf(hw, gR.x, gR.w - fmaf(w1, gR.y, w2 * gR.z))),
           gL);
  dR = sub(gR, f4(gL.x, fmaf(w1, gL.x, gL.y), fmaf(w2, gL.x, gL.z), fmaf(hw, gL.x, gL.w - fmaf(-w1, gL.y, -w2 * gL.z))));
}

// The R-theta limit of one side of a face: the largest theta in [0, 1]
// keeping V(theta) = U + theta D admissible and inside the relaxed density
// bounds, D = -+4 d_f seen in the side's own (rest) frame, so the pressure
// quadratic has no cancellation.  The floors eps_rho, eps_p are
// min(value, max(eps_pos, 1e-5 value)) of U: the relative margin keeps the
// final average admissible despite FP32 rounding.
//
// side_bound: the density limit th_rho (linear in theta), the coefficients of
// q(theta) = rho E - |m|^2 / 2 - eps_p rho / (gamma - 1) = A theta^2 + Bq theta
// + C, and whether q(th_rho) < 0 (the pressure then binds first).  Branch free.
__device__ __forceinline__ float side_bound(const float4 U, const Bnd b, const float4 D, float& A, float& Bq,
                                            bool& binds) {
  const float ax = fabsf(D.x);
  const float gap = D.x < 0.0f ? b.gap_lo : b.gap_hi;
  const float th = ax <= gap ? 1.0f : __fdividef(gap, ax);
  A = fmaf(D.x, D.w, -0.5f * fmaf(D.y, D.y, D.z * D.z));
  Bq = fmaf(U.x, D.w, fmaf(D.x, b.Ek, -fmaf(U.y, D.y, U.z * D.z)));
  binds = !(fmaf(th, fmaf(th, A, Bq), b.C) >= 0.0f);
  return th;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The pressure root where it binds: C = q(0) > 0 > q(th) leaves exactly one
// root in (0, th), the smallest positive one.  The stable form
// Q = -(Bq + sign(Bq) sqrt(Bq^2 - 4 A C)) / 2 gives the roots Q / A and C / Q,
// and the one sought is C / Q when Q > 0, else Q / A: for A > 0 both roots
// are positive, Bq < 0, Q > 0 and C / Q is the smaller; for A < 0 the roots
// have opposite signs, and C / Q is the positive one exactly when Q > 0; for
// A = 0, Q = -Bq > 0 and C / Q = -C / Bq.  C <= 0 (U itself on the floor)
// gives 0.  The square root is the hardware approximation (relative error of
// a few ulp): the 1e-5 margin of the floors absorbs it.
__device__ __forceinline__ float side_root(float th, float A, float Bq, float C) {
  const float sq = sqrt_approx(fmaxf(fmaf(Bq, Bq, -4.0f * (A * C)), 0.0f));
  const float Q = -0.5f * (Bq + copysignf(sq, Bq));
  const bool qp = Q > 0.0f;
  const float r = __fdividef(qp ? C : Q, qp ? Q : A);
  return C > 0.0f ? fminf(fmaxf(r, 0.0f), th) : 0.0f;
}

__device__ __forceinline__ bool is_boundary(int i, int j, int nx, int ny) {
  return i == 0 || i == nx - 1 || j == 0 || j == ny - 1;
}

// ---- TMA / mbarrier (inline PTX) ------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for phase `phase` of the barrier for at most one second.
__device__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t phase) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, phase))
    if (globaltimer() - t0 > 1000000000ull) return false;
  return true;
}

// ---- per-node and per-face arithmetic shared by every launch design --------
// Each design calls these with the same operands, so all of them produce
// bit-identical results (the translation unit is compiled without FMA
// contraction; every fused multiply-add is an explicit fmaf).

// Maxwellian of a neighbour node X (primitive state P) boosted into the frame
// moving with w (Eqs. (maxwellians12), (maxwellians34) and the boost
// identities): B_w M(u_X) = s u' + hs f(u') (x) or s u' + hs g(u') (y), with
// u' = B_w u_X = (rho, rho d1, rho d2, E'), d = v_X - w the relative velocity,
// E' = rho |d|^2 / 2 + p / (gamma - 1), s = c1 + hs w_dir and hs = +1/(2a)
// for M_1, M_3, -1/(2a) for M_2, M_4.  With sig = s + hs d_dir (>= 0 under
// the kinetic-speed bound) it reads
//   x: (rho sig, rho sig d1 + hs p, rho sig d2, E' sig + hs p d1)
//   y: (rho sig, rho sig d1, rho sig d2 + hs p, E' sig + hs p d2).
template <int DIR>
__device__ __forceinline__ float4 maxwellian_in_frame(const float4 P, float w1, float w2, float s, float hs,
                                                      float rg) {
  const float d1 = P.y - w1, d2 = P.z - w2;
  const float sig = fmaf(hs, DIR == 1 ? d1 : d2, s);
  const float rs = P.x * sig;
  const float hp = hs * P.w;
  const float Ep = fmaf(0.5f * P.x, fmaf(d1, d1, d2 * d2), P.w * rg);
  if (DIR == 1) return f4(rs, fmaf(rs, d1, hp), rs * d2, fmaf(Ep, sig, hp * d1));
  return f4(rs, rs * d1, fmaf(rs, d2, hp), fmaf(Ep, sig, hp * d2));
}

// P2 of an interior node c: U_LF (Eq. (vlbm5)'s first-order part) and the
// relaxed density bounds, in c's own frame, and the four boosted upwind
// Maxwellians B_vc M_k(u_upwind) (Eqs. (maxwellians12), (maxwellians34)).
__device__ __forceinline__ void node_p2(const float4 Pc, const float4 PW, const float4 PE, const float4 PS,
                                        const float4 PN, const Ctx& k, float4& U, Bnd& B, float4& M1, float4& M2,
                                        float4& M3, float4& M4) {
  const float w1 = Pc.y, w2 = Pc.z;
  M1 = maxwellian_in_frame<1>(PW, w1, w2, fmaf(k.h, w1, k.c1), k.h, k.rg);
  M2 = maxwellian_in_frame<1>(PE, w1, w2, fmaf(-k.h, w1, k.c1), -k.h, k.rg);
  M3 = maxwellian_in_frame<2>(PS, w1, w2, fmaf(k.h, w2, k.c1), k.h, k.rg);
  M4 = maxwellian_in_frame<2>(PN, w1, w2, fmaf(-k.h, w2, k.c1), -k.h, k.rg);
  U = add(add(M1, M2), add(M3, M4));
  if (k.alpha != 0.0f) U = add(U, f4(k.alpha * Pc.x, 0.0f, 0.0f, (k.alpha * Pc.w) * k.rg));
  const float lo = fminf(fminf(Pc.x, fminf(PW.x, PE.x)), fminf(fminf(PS.x, PN.x), U.x));
  const float hi = fmaxf(fmaxf(Pc.x, fmaxf(PW.x, PE.x)), fmaxf(fmaxf(PS.x, PN.x), U.x));
  const float delta = fmaf(k.rel, hi - lo, k.absb);
  // limits of theta_star at this node: density floor max(eps_rho, lo - delta)
  // with eps_rho = min(rho_LF, max(eps_pos, 1e-5 rho_LF)), ceiling hi + delta,
  // and kk = eps_p / (gamma - 1) with eps_p = min(p_LF, max(eps_pos, 1e-5 p_LF))
  const float er = fminf(U.x, fmaxf(k.eps, 1e-5f * U.x));
  const float pLF = k.gm1 * fmaf(-0.5f, __fdividef(fmaf(U.y, U.y, U.z * U.z), U.x), U.w);
  const float ep = fminf(pLF, fmaxf(k.eps, 1e-5f * pLF));
  B.gap_lo = U.x - fmaxf(er, lo - delta);
  B.gap_hi = (hi + delta) - U.x;
  B.Ek = U.w - ep * k.rg;
  B.C = fmaf(U.x, B.Ek, -0.5f * fmaf(U.y, U.y, U.z * U.z));
}

// The exact a_{n-1} -> a_n change of a rest-frame non-equilibrium part:
// g += s (1/2a_{n-1} - 1/2a_n) B_v f(u) with B_v f(u) = (rho v1, p, 0, v1 rho e)
// (x populations) or B_v g(u) = (rho v2, 0, p, v2 rho e) (y populations);
// s = +1 for the outgoing populations 1, 3 and -1 for the incoming 2, 4.
__device__ __forceinline__ float4 a_change_x(const float4 g, const float4 P, float sdinv, float rg) {
  const float re = P.w * rg;
  return axpy(sdinv, f4(P.x * P.y, P.w, 0.0f, P.y * re), g);
}
__device__ __forceinline__ float4 a_change_y(const float4 g, const float4 P, float sdinv, float rg) {
  const float re = P.w * rg;
  return axpy(sdinv, f4(P.x * P.z, 0.0f, P.w, P.z * re), g);
}

// theta_f of face (L, R) and theta_f d_f in L's and R's frames; gL, gR are the
// face's outgoing part of L and incoming part of R, already at a_n.  Both
// sides' density limits and pressure tests are evaluated unconditionally
// (no lane of a warp waits for another); a pressure root is taken, one side
// per pass, only where the pressure binds.  A boundary node sets no limit.
__device__ __forceinline__ float face_theta(const float4 PL, const float4 PR, const float4 gL, const float4 gR,
                                            const float4 UL, const Bnd BL, const float4 UR, const Bnd BR,
                                            bool bL, bool bR, int limiter, const Ctx& k, float4& tdL, float4& tdR) {
  float4 dL, dR;
  d_in_both(gL, gR, PL, PR, dL, dR);
  float th;
  if (limiter == 0) {
    th = 0.0f;
  } else if (limiter == 1) {
    th = 1.0f;
  } else {
    float AL, BqL, AR, BqR;
    bool nL, nR;
    float tL = side_bound(UL, BL, scale(-4.f, dL), AL, BqL, nL);
    float tR = side_bound(UR, BR, scale(4.f, dR), AR, BqR, nR);
    tL = bL ? 1.0f : tL;
    tR = bR ? 1.0f : tR;
    int pend = (nL && !bL ? 1 : 0) | (nR && !bR ? 2 : 0);
    while (pend) {
      const bool sl = (pend & 1) != 0;
      const float t = side_root(sl ? tL : tR, sl ? AL : AR, sl ? BqL : BqR, sl ? BL.C : BR.C);
      if (sl) {
        tL = t;
        pend &= 2;
      } else {
        tR = t;
        pend = 0;
      }
    }
    th = fminf(tL, tR);
  }
  th = (bL && bR) ? 0.0f : th;
  tdL = scale(th, dL);
  tdR = scale(th, dR);
  return th;
}

// P4 of an interior cell: Eq. (vlbm5) regrouped per face in the cell's frame,
// the new nodal state (returned) and its four new rest-frame non-equilibrium
// parts (Eqs. (vlbm1)-(vlbm4)), written at dst + off.  src.g(k) are the
// cell's own parts at a_n, src.mk(k) its kept Maxwellians; tdRW, tdLE, tdRS,
// tdLN the faces' theta_f d_f in this cell's frame.  Sets bit 1 / 2 of flags on a non-positive / non-finite
// result; otherwise raises lam to the node's max(|v1|, |v2|) + c.
// The kept Maxwellians and the cell's parts are fetched through src.mk(k) and
// src.g(k) where they are used (k = 0..3), which keeps them out of registers
// until then.
template <class Src, class I>
__device__ __forceinline__ float4 update_cell(float4* __restrict__ dst, I plane, I off, const float4 Pc,
                                              const float4 ULF, float thW, const float4 tdRW, float thE,
                                              const float4 tdLE, float thS, const float4 tdRS, float thN,
                                              const float4 tdLN, const Src& src, const Ctx& k, float& lam,
                                              int& flags) {
  const float4 U = add(sub(add(ULF, tdRW), tdLE), sub(tdRS, tdLN));
  // new nodal state (rest frame of the old velocity -> primitive)
  const float rn = U.x;
  const float inv = __fdividef(1.0f, rn);
  const float dv1 = U.y * inv, dv2 = U.z * inv;
  const float ren = fmaf(-0.5f, fmaf(U.y, dv1, U.z * dv2), U.w);
  const float pn = k.gm1 * ren;
  const float wn1 = Pc.y + dv1, wn2 = Pc.z + dv2;
  const float4 Pn = f4(rn, wn1, wn2, pn);
  dst[off] = Pn;
  int fl = 0;
  if (!(rn > 0.0f) || !(pn > 0.0f)) fl |= 1;
  if (!(fabsf(wn1) + fabsf(wn2) + rn + pn < __int_as_float(0x7f800000))) fl |= 2;
  // lambda, rounded up by 2^-20 so that a_{n+1} >= 2 lambda despite the
  // approximate reciprocal
  if (!fl) lam = fmaxf(lam, (fmaxf(fabsf(wn1), fabsf(wn2)) + sqrtf(k.gamma * pn * inv)) * (1.0f + 0x1p-20f));
  flags |= fl;
  // g_k^{n+1} = M_k(u_X) - theta_f g_k(X) - M_k(u^{n+1}), X the upwind node,
  // formed in the cell's old frame and boosted once to the new one.  In that
  // frame B g_1(W) = g_2(c) - d_W (the face's d seen by c), and likewise for
  // the other three faces.  The new state's Maxwellians in the old frame take
  // the factored form of the neighbours' (maxwellian_in_frame) with the new
  // state's relative velocity dv and lab velocity wn:
  //   M_1,2 = (rho s, rho s dv1 +- hp, rho s dv2, E' s +- hp dv1),
  //   s = c1 +- h wn1 (M_3,4 likewise with the y components), E' = U.w.
  const float dw1 = wn1 - Pc.y, dw2 = wn2 - Pc.z;
  const float hp = k.h * pn, hpx = hp * dv1, hpy = hp * dv2;
  const float s1 = fmaf(k.h, wn1, k.c1), s2 = fmaf(-k.h, wn1, k.c1);
  const float s3 = fmaf(k.h, wn2, k.c1), s4 = fmaf(-k.h, wn2, k.c1);
  const float r1 = rn * s1, r2 = rn * s2, r3 = rn * s3, r4 = rn * s4;
  float4 X;
  X = add(axpy(-thW, src.g(1), sub(src.mk(0), f4(r1, fmaf(r1, dv1, hp), r1 * dv2, fmaf(U.w, s1, hpx)))), tdRW);
  dst[1 * plane + off] = boost(X, dw1, dw2);
  X = sub(axpy(-thE, src.g(0), sub(src.mk(1), f4(r2, fmaf(r2, dv1, -hp), r2 * dv2, fmaf(U.w, s2, -hpx)))), tdLE);
  dst[2 * plane + off] = boost(X, dw1, dw2);
  X = add(axpy(-thS, src.g(3), sub(src.mk(2), f4(r3, r3 * dv1, fmaf(r3, dv2, hp), fmaf(U.w, s3, hpy)))), tdRS);
  dst[3 * plane + off] = boost(X, dw1, dw2);
  X = sub(axpy(-thN, src.g(2), sub(src.mk(3), f4(r4, r4 * dv1, fmaf(r4, dv2, -hp), fmaf(U.w, s4, -hpy)))), tdLN);
  dst[4 * plane + off] = boost(X, dw1, dw2);
  return Pn;
}

// Boundary writes owned by interior cell (gi, gj) (Eqs. (inletBC),
// (outletBC), (transverseBC)): zero-gradient copies of its new state with
// equilibrium populations (g' = 0) into the outlet column and the first / last
// rows next to it, and, in the first interior column, the inlet datum of its
// row (and of the corner rows) as FP32 primitives with equilibrium populations.
template <class I>
__device__ __forceinline__ void boundary_writes(float4* __restrict__ dst, I plane, I off, int gi, int gj,
                                                int nx, int ny, int nxp, const float4 Pn,
                                                const float4* __restrict__ inl, const Ctx& k, float& lam) {
  const bool cxl = gi == nx - 2, cyl = gj == 1, cyh = gj == ny - 2;
  if (cxl || cyl || cyh) {
    // targets: east (cxl), south / north (cyl / cyh), their east corners
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const bool on = t == 0 ? cxl : t == 1 ? cyl : t == 2 ? (cyl && cxl) : t == 3 ? cyh : (cyh && cxl);
      if (!on) continue;
      // the row below (t = 1, 2) wraps around in unsigned index arithmetic
      const I dj = t == 0 ? I(0) : (t <= 2 ? I(0) - I(nxp) : I(nxp));
      const I o = off + dj + I(t == 0 || t == 2 || t == 4 ? 1 : 0);
      dst[o] = Pn;
#pragma unroll
      for (int q = 1; q <= 4; ++q) dst[q * plane + o] = f4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (gi == 1) {
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      // rows: this one, and the corner rows 0 / ny - 1 next to the sides
      const int jj = r == 0 ? gj : r == 1 ? (gj == 1 ? 0 : -1) : (gj == ny - 2 ? ny - 1 : -1);
      if (jj < 0) continue;
      const float4 Pi = inl[jj];
      const I oi = I(jj) * I(nxp);
      dst[oi] = Pi;
#pragma unroll
      for (int q = 1; q <= 4; ++q) dst[q * plane + oi] = f4(0.f, 0.f, 0.f, 0.f);
      lam = fmaxf(lam, (fmaxf(fabsf(Pi.y), fabsf(Pi.z)) + sqrtf(k.gamma * Pi.w / Pi.x)) * (1.0f + 0x1p-20f));
    }
  }
}

__device__ __forceinline__ Ctx make_ctx(const Launch& L, const RealState* rs) {
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
  return k;
}

// Work unit u -> (level, realization, tile within the level); units run over
// the tiles of realization 0 first, so CTAs in flight share halos through L2.
__device__ __forceinline__ void decode_unit(const Launch& L, long long u, int& lvl, int& m, int& tile) {
  m = (int)(u / L.total_tiles);
  tile = (int)(u - (long long)m * L.total_tiles);
  lvl = 0;
  while (lvl + 1 < L.nlevels && tile >= L.lv[lvl + 1].tile_begin) ++lvl;
  tile -= L.lv[lvl].tile_begin;
}

// Computes one tile whose boxes are in Bx (P2, P3, P4 and the lambda
// reduction); ends with every thread past a barrier after its last use of W.
template <int TY>
__device__ __forceinline__ void compute_tile(const Launch& L, Boxes<TY>& Bx, Work<TY>& W, int lvl, int m, int tile) {
  constexpr int NT = TX * TY, GX = Boxes<TY>::GX, GY = Boxes<TY>::GY;
  const int tid = threadIdx.x;
  const LevelDesc& D = L.lv[lvl];
  RealState* rs = D.rs + m;
  const int nx = D.nx, ny = D.ny, nxp = D.nx_pad;
  const size_t plane = D.plane;
  const int par = (int)(rs->steps & 1);
  float4* __restrict__ dst = reinterpret_cast<float4*>(D.lat) + ((size_t)(par ^ 1) * L.M + m) * D.real_stride;
  const Ctx k = make_ctx(L, rs);
  const float dinv = rs->dinv2a_f;
  const int limiter = L.ph.limiter;
  const int i0 = 1 + (tile % D.tiles_x) * TX;
  const int j0 = 1 + (tile / D.tiles_x) * TY;

  // ---- P2: U_LF in each node's own frame, bounds ----------------------------
  for (int idx = tid; idx < GX * GY; idx += NT) {
    const int li = idx % GX, lj = idx / GX;
    const int gi = i0 - 1 + li, gj = j0 - 1 + lj;
    if (gi < 1 || gi > nx - 2 || gj < 1 || gj > ny - 2) continue;
    const int hx = li + 1, hy = lj + 1;
    float4 U, M1, M2, M3, M4;
    Bnd B;
    node_p2(Bx.P[hy][hx], Bx.P[hy][hx - 1], Bx.P[hy][hx + 1], Bx.P[hy - 1][hx], Bx.P[hy + 1][hx], k, U, B, M1, M2,
            M3, M4);
    W.U[lj][li] = U;
    W.B[lj][li] = B;
    if (li >= 1 && li <= TX && lj >= 1 && lj <= TY) {
      W.Mk[0][lj - 1][li - 1] = M1;
      W.Mk[1][lj - 1][li - 1] = M2;
      W.Mk[2][lj - 1][li - 1] = M3;
      W.Mk[3][lj - 1][li - 1] = M4;
    }
  }
  __syncthreads();

  // ---- P3: faces -------------------------------------------------------------
  // Thread (lx, ly) owns the west and south faces of its cell; the east faces
  // of the last column and the north faces of the top row go to the first
  // warps.  A face brings its two non-equilibrium parts to a_n, writes them
  // back (each is used by this face alone), and stores theta_f and
  // theta_f d_f in both cells' frames.
  {
    const int lx = tid % TX, ly = tid / TX;
    constexpr int NEXTRA = TY + TX;
    for (int pass = 0; pass < 3; ++pass) {
      bool xdir;
      int fa, fb;
      if (pass < 2) {
        xdir = pass == 0;
        fa = lx;
        fb = ly;
      } else {
        if (tid >= NEXTRA) break;
        xdir = tid < TY;
        fa = xdir ? TX : tid - TY;
        fb = xdir ? tid : TY;
      }
      int iL, jL, iR, jR;
      bool L_in, R_in;
      if (xdir) {
        iL = i0 + fa - 1;
        jL = j0 + fb;
        iR = iL + 1;
        jR = jL;
        if (jL > ny - 2) continue;
        L_in = fa >= 1 && iL <= nx - 2;
        R_in = fa < TX && iR <= nx - 2;
      } else {
        iL = i0 + fa;
        jL = j0 + fb - 1;
        iR = iL;
        jR = jL + 1;
        if (iL > nx - 2) continue;
        L_in = fb >= 1 && jL <= ny - 2;
        R_in = fb < TY && jR <= ny - 2;
      }
      if (!L_in && !R_in) continue;
      const bool bL = is_boundary(iL, jL, nx, ny), bR = is_boundary(iR, jR, nx, ny);
      const int kout = xdir ? 0 : 2, kin = xdir ? 1 : 3;
      const int gxL = iL - i0 + 1, gyL = jL - j0 + 1, gxR = iR - i0 + 1, gyR = jR - j0 + 1;
      const float4 PL = Bx.P[gyL + 1][gxL + 1], PR = Bx.P[gyR + 1][gxR + 1];
      float4 gL = Bx.G[kout][gyL][gxL], gR = Bx.G[kin][gyR][gxR];
      if (dinv != 0.0f) {
        if (!bL) {
          gL = xdir ? a_change_x(gL, PL, dinv, k.rg) : a_change_y(gL, PL, dinv, k.rg);
          Bx.G[kout][gyL][gxL] = gL;
        }
        if (!bR) {
          gR = xdir ? a_change_x(gR, PR, -dinv, k.rg) : a_change_y(gR, PR, -dinv, k.rg);
          Bx.G[kin][gyR][gxR] = gR;
        }
      }
      float4 tdL, tdR;
      const float th = face_theta(PL, PR, gL, gR, W.U[gyL][gxL], W.B[gyL][gxL], W.U[gyR][gxR], W.B[gyR][gxR], bL,
                                  bR, limiter, k, tdL, tdR);
      if (xdir) {
        W.thx[fb][fa] = th;
        W.tdLx[fb][fa] = tdL;
        W.tdRx[fb][fa] = tdR;
      } else {
        W.thy[fb][fa] = th;
        W.tdLy[fb][fa] = tdL;
        W.tdRy[fb][fa] = tdR;
      }
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
      const int cx = lx + 1, cy = ly + 1;
      const size_t off = (size_t)gj * nxp + gi;
      struct {
        const Boxes<TY>& bx;
        const Work<TY>& w;
        int lx, ly;
        __device__ float4 mk(int q) const { return w.Mk[q][ly][lx]; }
        __device__ float4 g(int q) const { return bx.G[q][ly + 1][lx + 1]; }
      } src{Bx, W, lx, ly};
      const float4 Pn = update_cell(dst, plane, off, Bx.P[ly + 2][lx + 2], W.U[cy][cx], W.thx[ly][lx],
                                    W.tdRx[ly][lx], W.thx[ly][lx + 1], W.tdLx[ly][lx + 1], W.thy[ly][lx],
                                    W.tdRy[ly][lx], W.thy[ly + 1][lx], W.tdLy[ly + 1][lx], src, k, lam, flags);
      boundary_writes(dst, plane, off, gi, gj, nx, ny, nxp, Pn, D.inlet_f + (size_t)m * ny, k, lam);
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
    W.lam[tid >> 5] = lb;
    W.flags[tid >> 5] = flags;
  }
  __syncthreads();
  if (tid == 0) {
    unsigned best = 0;
    int fl = 0;
    for (int w = 0; w < NT / 32; ++w) {
      best = max(best, W.lam[w]);
      fl |= W.flags[w];
    }
    atomicMax(&rs->lam_next_bits, lam_to_bits((double)__uint_as_float(best)));
    if (fl) atomicOr(&rs->flags, fl);
  }
}

// Thread 0: starts the two TMA loads of tile (lvl, m, tile) into Bx on bar.
// The proxy fence orders earlier generic-proxy accesses of Bx before the
// async-proxy overwrite.
template <int TY>
__device__ __forceinline__ void issue_tile(Boxes<TY>& Bx, unsigned long long* bar, const Launch& L, int lvl, int m,
                                           int tile) {
  const LevelDesc& D = L.lv[lvl];
  const int par = (int)(D.rs[m].steps & 1);
  const int i0 = 1 + (tile % D.tiles_x) * TX, j0 = 1 + (tile / D.tiles_x) * TY;
  constexpr uint32_t bytes = sizeof(float4) * (Boxes<TY>::HX * Boxes<TY>::HY + 4 * Boxes<TY>::GX * Boxes<TY>::GY);
  fence_proxy_async();
  mbar_arrive_expect_tx(bar, bytes);
  const int zP = (par * L.M + m) * 5;
  tma_load_4d(&Bx.P[0][0], &L.tmP[lvl], 0, i0 - 2, j0 - 2, zP, bar);
  tma_load_4d(&Bx.G[0][0][0], &L.tmG[lvl], 0, i0 - 1, j0 - 1, zP + 1, bar);
}

// One tile per CTA: blockIdx.x = tile over all levels, blockIdx.y = realization.
template <int TY>
__global__ void __launch_bounds__(TX* TY, 1024 / (TX * TY)) step_mixed_tile_kernel(const __grid_constant__ Launch L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemTile<TY>& S = *reinterpret_cast<SmemTile<TY>*>(smem_raw);
  const int tid = threadIdx.x;
  int tile = blockIdx.x, lvl = 0;
  while (lvl + 1 < L.nlevels && tile >= L.lv[lvl + 1].tile_begin) ++lvl;
  tile -= L.lv[lvl].tile_begin;
  const int m = blockIdx.y;
  RealState* rs = L.lv[lvl].rs + m;
  if (!rs->active) return;
  if (tid == 0) {
    mbar_init(&S.bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) issue_tile<TY>(S.box, &S.bar, L, lvl, m, tile);
  const bool ok = mbar_wait_bounded(&S.bar, 0);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) {
      mbar_wait_bounded(&S.bar, 0);
      atomicOr(&rs->flags, 4);
    }
    return;
  }
  compute_tile<TY>(L, S.box, S.w, lvl, m, tile);
}

// Persistent: CTA b takes units b, b + gridDim.x, ...; while it computes one
// tile the TMA engine fills the other buffer with the next one.
template <int TY>
__global__ void __launch_bounds__(TX* TY, 1) step_mixed_persistent_kernel(const __grid_constant__ Launch L) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemPersist<TY>& S = *reinterpret_cast<SmemPersist<TY>*>(smem_raw);
  const int tid = threadIdx.x;
  const long long total = (long long)L.M * L.total_tiles;
  long long u = blockIdx.x;
  auto issue = [&](int b, long long unit) {
    int lvl, m, tile;
    decode_unit(L, unit, lvl, m, tile);
    if (!L.lv[lvl].rs[m].active) {
      S.issued[b] = 0;
      return;
    }
    issue_tile<TY>(S.buf[b], &S.bar[b], L, lvl, m, tile);
    S.issued[b] = 1;
  };
  if (tid == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    mbar_fence_init();
    S.issued[0] = S.issued[1] = 0;
  }
  __syncthreads();
  if (tid == 0 && u < total) issue(0, u);
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};
  for (int it = 0; u < total; ++it, u += gridDim.x) {
    const int b = it & 1;
    if (tid == 0 && u + gridDim.x < total) issue(b ^ 1, u + gridDim.x);
    if (!S.issued[b]) {
      __syncthreads();
      continue;
    }
    int lvl, m, tile;
    decode_unit(L, u, lvl, m, tile);
    const bool ok = mbar_wait_bounded(&S.bar[b], phase[b]);
    phase[b] ^= 1u;
    if (__syncthreads_or(!ok)) {
      // leave only once the copies in flight have landed (bounded again)
      if (tid == 0) {
        mbar_wait_bounded(&S.bar[b], phase[b] ^ 1u);
        if (S.issued[b ^ 1]) mbar_wait_bounded(&S.bar[b ^ 1], phase[b ^ 1]);
        atomicOr(&L.lv[lvl].rs[m].flags, 4);
      }
      return;
    }
    compute_tile<TY>(L, S.buf[b], S.w, lvl, m, tile);
    __syncthreads();
  }
}

// ---- warp-marching design ----------------------------------------------------
// A warp owns a strip of kMW interior columns (lanes 1..kMW; lanes 0 and 31
// hold the halo columns) and marches up D.wrows rows of it.  Nodal states and
// non-equilibrium parts go straight from global memory into registers, each
// lane loading its own column (512 contiguous bytes per row and plane for the
// warp); x-neighbours come by warp shuffle.  The window in registers holds
// three rows of nodal states, U_LF and bounds of the current and the next row,
// and the face between them; the Maxwellians kept for the next row wait in
// the lane's own shared-memory slot.  A warp never waits for another warp.
constexpr int kMW = 30;      // columns updated per warp
constexpr int kMNW = 4;      // warps per CTA
constexpr int kMarchRows = 25;  // target rows per warp

__device__ __forceinline__ float4 shfl_up4(const float4 v) {
  return f4(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1),
            __shfl_up_sync(0xffffffffu, v.z, 1), __shfl_up_sync(0xffffffffu, v.w, 1));
}
__device__ __forceinline__ float4 shfl_down4(const float4 v) {
  return f4(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1),
            __shfl_down_sync(0xffffffffu, v.z, 1), __shfl_down_sync(0xffffffffu, v.w, 1));
}
__device__ __forceinline__ Bnd shfl_down_b(const Bnd v) {
  return Bnd{__shfl_down_sync(0xffffffffu, v.gap_lo, 1), __shfl_down_sync(0xffffffffu, v.gap_hi, 1),
             __shfl_down_sync(0xffffffffu, v.Ek, 1), __shfl_down_sync(0xffffffffu, v.C, 1)};
}

// blockIdx.x = (strip, row chunk) over all levels, blockIdx.y = realization;
// MINB CTAs per SM bound the registers.
// Asynchronous 16-byte copy global -> shared (cp.async, L2 only); with
// valid false it writes zeros and reads nothing.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// PF: the rows a march step reads are copied into the lane's own shared-memory
// ring by cp.async one step ahead (no registers held while they travel);
// otherwise they are loaded into registers at the top of the step.
template <int MINB, bool PF>
__global__ void __launch_bounds__(kMNW * 32, MINB) step_mixed_march_kernel(const __grid_constant__ Launch L) {
  __shared__ float4 smk[2][4][kMNW][32];
  __shared__ float4 ring[PF ? 2 : 1][6][kMNW][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int unit = blockIdx.x, lvl = 0;
  while (lvl + 1 < L.nlevels && unit >= L.lv[lvl + 1].tile_begin) ++lvl;
  unit -= L.lv[lvl].tile_begin;
  const int m = blockIdx.y;
  const LevelDesc& D = L.lv[lvl];
  RealState* rs = D.rs + m;
  if (!rs->active) return;
  const int nx = D.nx, ny = D.ny, nxp = D.nx_pad;
  const int ra = 1 + ((unit / D.tiles_x) * kMNW + wid) * D.wrows;
  const int rb = min(ra + D.wrows - 1, ny - 2);
  if (ra > rb) return;
  // lane l holds column x0 - 1 + l of the strip starting at x0 = 1 + kMW * strip
  const int c = (unit % D.tiles_x) * kMW + lane;
  // element offsets within one realization's lattice fit in 32 bits (the
  // launcher checks 5 planes < 2^31), which keeps the per-row address
  // arithmetic in 32-bit integers
  const int plane = (int)D.plane;
  const int par = (int)(rs->steps & 1);
  const float4* __restrict__ src =
      reinterpret_cast<const float4*>(D.lat) + ((size_t)par * L.M + m) * D.real_stride;
  float4* __restrict__ dst = reinterpret_cast<float4*>(D.lat) + ((size_t)(par ^ 1) * L.M + m) * D.real_stride;
  const float4* __restrict__ inl = D.inlet_f + (size_t)m * ny;
  const Ctx k = make_ctx(L, rs);
  const float dinv = rs->dinv2a_f;
  const int limiter = L.ph.limiter;
  const bool colin = c >= 1 && c <= nx - 2;          // interior column
  const bool colin_e = c + 1 <= nx - 2;              // east neighbour's column interior
  const bool upd = lane >= 1 && lane <= kMW && colin;  // this lane updates cells
  const int cl = min(c, nx - 1);
  const int cf = lane == 0 ? c - 1 : c + 1;  // the halo lanes' far column
  const bool far = (lane == 0 || lane == 31) && cf >= 0 && cf <= nx - 1;
  const float4 z4 = f4(0.f, 0.f, 0.f, 0.f);
  auto ldP = [&](int q) { return q >= 0 && q <= ny - 1 ? __ldg(src + (q * nxp + cl)) : z4; };
  auto ldF = [&](int q) { return far && q >= 0 && q <= ny - 1 ? __ldg(src + (q * nxp + cf)) : z4; };
  auto ldG = [&](int kk, int q) {
    return q >= 0 && q <= ny - 1 ? __ldg(src + ((kk + 1) * plane + q * nxp + cl)) : z4;
  };
  auto inner = [&](int q) { return colin && q >= 1 && q <= ny - 2; };
  auto west = [&](const float4 P, const float4 F) {
    const float4 w = shfl_up4(P);
    return lane == 0 ? F : w;
  };
  auto east = [&](const float4 P, const float4 F) {
    const float4 e = shfl_down4(P);
    return lane == 31 ? F : e;
  };
  auto keep = [&](int q, const float4 M1, const float4 M2, const float4 M3, const float4 M4) {
    smk[q & 1][0][wid][lane] = M1;
    smk[q & 1][1][wid][lane] = M2;
    smk[q & 1][2][wid][lane] = M3;
    smk[q & 1][3][wid][lane] = M4;
  };

  // ---- warm-up: rows ra - 1 and ra, and the face between them ----------------
  float4 M1, M2, M3, M4;
  float4 Pq = ldP(ra), Pq1 = ldP(ra + 1), Fq1 = ldF(ra + 1);
  float4 Uq = z4, PEq;
  Bnd Bq{0.f, 0.f, 0.f, 0.f};
  float thS;
  float4 tdRS, g4q;
  {
    const float4 Pm2 = ldP(ra - 2), Pm = ldP(ra - 1), Fm = ldF(ra - 1), Fq = ldF(ra);
    float4 Um = z4;
    Bnd Bm{0.f, 0.f, 0.f, 0.f};
    const float4 PWm = west(Pm, Fm), PEm = east(Pm, Fm);
    if (inner(ra - 1)) node_p2(Pm, PWm, PEm, Pm2, Pq, k, Um, Bm, M1, M2, M3, M4);
    const float4 PWq = west(Pq, Fq);
    PEq = east(Pq, Fq);
    if (inner(ra)) {
      node_p2(Pq, PWq, PEq, Pm, Pq1, k, Uq, Bq, M1, M2, M3, M4);
      keep(ra, M1, M2, M3, M4);
    }
    const bool bm = !inner(ra - 1), bq = !inner(ra);
    float4 g3m = ldG(2, ra - 1);
    g4q = ldG(3, ra);
    if (dinv != 0.0f) {
      if (!bm) g3m = a_change_y(g3m, Pm, dinv, k.rg);
      if (!bq) g4q = a_change_y(g4q, Pq, -dinv, k.rg);
    }
    float4 unused;
    thS = face_theta(Pm, Pq, g3m, g4q, Um, Bm, Uq, Bq, bm, bq, limiter, k, unused, tdRS);
  }

  // ---- march -----------------------------------------------------------------
  // the rows step q reads: nodal state and far column of row q + 2, parts
  // 1..3 of row q, part 4 of row q + 1
  auto prefetch = [&](int q) {
    float4(&r)[6][kMNW][32] = ring[q & 1];
    const bool v2 = q + 2 <= ny - 1;
    const int row2 = (v2 ? q + 2 : 0) * nxp, row0 = q * nxp + cl;
    cp_async16(&r[0][wid][lane], src + (row2 + cl), v2);
    cp_async16(&r[1][wid][lane], src + (row2 + (far ? cf : cl)), v2 && far);
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) cp_async16(&r[2 + kk][wid][lane], src + ((kk + 1) * plane + row0), true);
    cp_async16(&r[5][wid][lane], src + (4 * plane + nxp + row0), true);
  };
  if (PF) {
    prefetch(ra);
    cp_async_commit();
  }
  float lam = 0.0f;
  int flags = 0;
  for (int q = ra; q <= rb; ++q) {
    float4 Pq2, Fq2, G1, G2, G3, g4n;
    if (PF) {
      if (q < rb) prefetch(q + 1);
      cp_async_commit();
      cp_async_wait_prev();
      const float4(&r)[6][kMNW][32] = ring[q & 1];
      Pq2 = r[0][wid][lane];
      Fq2 = r[1][wid][lane];
      G1 = r[2][wid][lane];
      G2 = r[3][wid][lane];
      G3 = r[4][wid][lane];
      g4n = r[5][wid][lane];
    } else {
      Pq2 = ldP(q + 2);
      Fq2 = ldF(q + 2);
      G1 = ldG(0, q);
      G2 = ldG(1, q);
      G3 = ldG(2, q);
      g4n = ldG(3, q + 1);
    }
    // P2 of row q + 1
    float4 U1 = z4;
    Bnd B1{0.f, 0.f, 0.f, 0.f};
    const float4 PW1 = west(Pq1, Fq1), PE1 = east(Pq1, Fq1);
    const bool bq = !colin, b1 = !inner(q + 1);
    if (!b1) {
      node_p2(Pq1, PW1, PE1, Pq, Pq2, k, U1, B1, M1, M2, M3, M4);
      keep(q + 1, M1, M2, M3, M4);
    }
    // this row's parts 1..3 and the next row's part 4 at a_n
    if (dinv != 0.0f) {
      if (!bq) {
        G1 = a_change_x(G1, Pq, dinv, k.rg);
        G2 = a_change_x(G2, Pq, -dinv, k.rg);
        G3 = a_change_y(G3, Pq, dinv, k.rg);
      }
      if (!b1) g4n = a_change_y(g4n, Pq1, -dinv, k.rg);
    }
    // north face of row q (= south face of row q + 1)
    float4 tdLN, tdRN;
    const float thN = face_theta(Pq, Pq1, G3, g4n, Uq, Bq, U1, B1, bq, b1, limiter, k, tdLN, tdRN);
    // east face (R = lane + 1); the west face comes from lane - 1
    const float4 gR = shfl_down4(G2), UR = shfl_down4(Uq);
    const Bnd BR = shfl_down_b(Bq);
    float4 tdLE, tdRE;
    const float thE = face_theta(Pq, PEq, G1, gR, Uq, Bq, UR, BR, bq, !colin_e, limiter, k, tdLE, tdRE);
    const float thW = __shfl_up_sync(0xffffffffu, thE, 1);
    const float4 tdRW = shfl_up4(tdRE);
    if (upd) {
      struct {
        const float4 (*mk_)[kMNW][32];
        int wid, lane;
        float4 g0, g1, g2, g3;
        __device__ float4 mk(int i) const { return mk_[i][wid][lane]; }
        __device__ float4 g(int i) const { return i == 0 ? g0 : i == 1 ? g1 : i == 2 ? g2 : g3; }
      } cell{smk[q & 1], wid, lane, G1, G2, G3, g4q};
      const int off = q * nxp + c;
      const float4 Pn =
          update_cell(dst, plane, off, Pq, Uq, thW, tdRW, thE, tdLE, thS, tdRS, thN, tdLN, cell, k, lam, flags);
      boundary_writes(dst, plane, off, c, q, nx, ny, nxp, Pn, inl, k, lam);
    }
    Pq = Pq1;
    PEq = PE1;
    Pq1 = Pq2;
    Fq1 = Fq2;
    Uq = U1;
    Bq = B1;
    g4q = g4n;
    thS = thN;
    tdRS = tdRN;
  }
  // lambda >= 0: its FP32 bit pattern orders like an unsigned integer
  unsigned lb = __float_as_uint(lam);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lb = max(lb, __shfl_xor_sync(0xffffffffu, lb, o));
    flags |= __shfl_xor_sync(0xffffffffu, flags, o);
  }
  if (lane == 0) {
    atomicMax(&rs->lam_next_bits, lam_to_bits((double)__uint_as_float(lb)));
    if (flags) atomicOr(&rs->flags, flags);
  }
}

// Variants: 32 x 4 tiles, 32 x 8 tiles, persistent 32 x 8 tiles, warp march
// with 4 or 5 CTAs of 4 warps per SM, loading into registers or prefetching
// into shared memory.
constexpr const char* kVariantNames[] = {"tile32x4",   "tile32x8",     "persistent32x8",
                                         "march30x4w", "march30x5w",   "march30pf4w",
                                         "march30pf5w"};
constexpr int kNumVariants = 7;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 4-D view of one level's storage as FP32: (4 components, x, y, 10 M planes);
// plane index (lattice * M + m) * 5 + q.  Out-of-range boxes fill with zeros.
cudaError_t encode_level(CUtensorMap* map, const LevelDesc& D, int M, int box_x, int box_y, int box_planes) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[4] = {4, (cuuint64_t)D.nx, (cuuint64_t)D.ny, (cuuint64_t)10 * M};
  cuuint64_t strides[3] = {16, (cuuint64_t)D.nx_pad * 16, (cuuint64_t)D.plane * 16};
  cuuint32_t box[4] = {4, (cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_planes};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, D.lat, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tile decomposition and TMA descriptors of a 32 x TY tile shape.
template <int TY>
cudaError_t layout(Launch& L) {
  int tiles = 0;
  for (int l = 0; l < L.nlevels; ++l) {
    LevelDesc& D = L.lv[l];
    D.tiles_x = (D.nx - 2 + TX - 1) / TX;
    D.tiles_y = (D.ny - 2 + TY - 1) / TY;
    D.tile_begin = tiles;
    tiles += D.tiles_x * D.tiles_y;
    cudaError_t e = encode_level(&L.tmP[l], D, L.M, Boxes<TY>::HX, Boxes<TY>::HY, 1);
    if (e == cudaSuccess) e = encode_level(&L.tmG[l], D, L.M, Boxes<TY>::GX, Boxes<TY>::GY, 4);
    if (e != cudaSuccess) return e;
  }
  L.total_tiles = tiles;
  return cudaSuccess;
}

template <int TY>
cudaError_t launch_tile(Launch& L, cudaStream_t s) {
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = once_per_device(configured, [] {
    return cudaFuncSetAttribute(step_mixed_tile_kernel<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(SmemTile<TY>));
  });
  if (e == cudaSuccess) e = layout<TY>(L);
  if (e != cudaSuccess) return e;
  step_mixed_tile_kernel<TY><<<dim3(L.total_tiles, L.M), TX * TY, sizeof(SmemTile<TY>), s>>>(L);
  add_launches(1);
  return cudaGetLastError();
}

template <int TY>
cudaError_t launch_persistent(Launch& L, cudaStream_t s) {
  // one persistent CTA per SM slot: the occupancy and the SM count are those
  // of the current device
  static std::atomic<unsigned long long> configured{0};
  const int smem = (int)sizeof(SmemPersist<TY>);
  cudaError_t e = once_per_device(configured, [smem] {
    return cudaFuncSetAttribute(step_mixed_persistent_kernel<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_mixed_persistent_kernel<TY>, TX * TY, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int grid_ctas = (per_sm > 0 ? per_sm : 1) * sms;
  e = layout<TY>(L);
  if (e != cudaSuccess) return e;
  const long long units = (long long)L.M * L.total_tiles;
  const int grid = (int)(units < grid_ctas ? units : grid_ctas);
  step_mixed_persistent_kernel<TY><<<grid, TX * TY, sizeof(SmemPersist<TY>), s>>>(L);
  add_launches(1);
  return cudaGetLastError();
}

int sm_count() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// CTAs of one realization's launch (all levels) with `rows` rows per warp.
long long march_ctas(const Launch& L, int rows) {
  long long ctas = 0;
  for (int l = 0; l < L.nlevels; ++l) {
    const LevelDesc& D = L.lv[l];
    const int r = D.ny - 2;
    ctas += (long long)((D.nx - 2 + kMW - 1) / kMW) * ((r + kMNW * rows - 1) / (kMNW * rows));
  }
  return ctas;
}

// Rows per warp: L.march_rows when set; else kMarchRows, fewer (down to 4)
// when the launch would not give every SM two rounds of MINB CTAs (a single
// small grid): each warp then re-evaluates one more halo row per fewer rows,
// but the GPU fills.  The split does not change any result; the context's
// tuning times other counts on small launches.
int march_rows_for(const Launch& L, int minb) {
  if (L.march_rows > 0) return L.march_rows;
  const long long slots = (long long)sm_count() * minb;
  int target = kMarchRows;
  while (march_ctas(L, target) * L.M < 2 * slots && target > 4) target = target / 2 < 4 ? 4 : target / 2;
  return target;
}

// Strips of kMW columns; rows split into chunks of kMNW warps with about
// march_rows_for rows per warp.
template <int MINB, bool PF>
cudaError_t launch_march(Launch& L, cudaStream_t s) {
  // the march indexes a realization's five planes with 32-bit offsets; a
  // level beyond that (over 429 M nodes) runs on the tile design instead
  for (int l = 0; l < L.nlevels; ++l)
    if (5 * L.lv[l].plane >= ((size_t)1 << 31)) return launch_tile<8>(L, s);
  const int target = march_rows_for(L, MINB);
  int units = 0;
  for (int l = 0; l < L.nlevels; ++l) {
    LevelDesc& D = L.lv[l];
    const int rows = D.ny - 2;
    const int chunks = (rows + kMNW * target - 1) / (kMNW * target);
    D.tiles_x = (D.nx - 2 + kMW - 1) / kMW;
    D.tiles_y = chunks;
    D.wrows = (rows + chunks * kMNW - 1) / (chunks * kMNW);
    D.tile_begin = units;
    units += D.tiles_x * D.tiles_y;
  }
  L.total_tiles = units;
  step_mixed_march_kernel<MINB, PF><<<dim3(units, L.M), kMNW * 32, 0, s>>>(L);
  add_launches(1);
  return cudaGetLastError();
}

// CTAs per SM of the march designs 3..6 (register bound MINB)
int march_minb(int v) { return v == 4 || v == 6 ? 5 : 4; }

}  // namespace

int mixed_variants() { return kNumVariants; }
int mixed_march_rows(const Launch& L, int v) { return v >= 3 && v < kNumVariants ? march_rows_for(L, march_minb(v)) : 0; }
double mixed_march_waves(const Launch& L, int v, int rows) {
  if (v < 3 || v >= kNumVariants) return 0.0;
  Launch c = L;
  c.march_rows = rows;
  const int r = march_rows_for(c, march_minb(v));
  return (double)march_ctas(c, r) * L.M / ((double)sm_count() * march_minb(v));
}
const char* mixed_variant_name(int v) { return v >= 0 && v < kNumVariants ? kVariantNames[v] : "?"; }

cudaError_t launch_step_mixed(const Launch& Lin, int variant, cudaStream_t s) {
  static thread_local Launch L;  // large (TMA descriptors): kept off the stack
  L = Lin;
  switch (variant) {
    case 0:
      return launch_tile<4>(L, s);
    case 1:
      return launch_tile<8>(L, s);
    case 2:
      return launch_persistent<8>(L, s);
    case 3:
      return launch_march<4, false>(L, s);
    case 4:
      return launch_march<5, false>(L, s);
    case 5:
      return launch_march<4, true>(L, s);
    default:
      return launch_march<5, true>(L, s);
  }
}

}  // namespace vlbm
