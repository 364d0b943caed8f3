// Internal declarations of libvlbm (not part of the public C ABI).
//
// Device layout of one level (per realization m, lattice L in {0, 1}):
//   VLBM_FP64 : 20 planes of double [ny][nx_pad]:
//               planes 0..3   conserved u = (rho, rho v1, rho v2, E)
//               planes 4..19  raw populations u_k, plane 4 + 4(k-1) + c
//   VLBM_MIXED: 5 planes of float4 [ny][nx_pad]:
//               plane 0       nodal state (rho, v1, v2, p)
//               planes 1..4   non-equilibrium part of population k = 1..4,
//                             (rho, m1, m2, E)-components, boosted into the
//                             node's rest frame (velocity = stored v)
// Lattice L of realization m starts at  base + (L * M + m) * real_stride.
// The two lattices ping-pong per realization with the parity of its own step
// count, so realizations that stop early (landing) keep a consistent state.
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/vlbm.h"

namespace vlbm {

constexpr int kMaxLevels = 8;
constexpr int kMaxModes = 16;

// Per (level, realization) bookkeeping, device resident.
struct RealState {
  double t;            // time t_n of the current state
  double t_target;     // landing target (+inf for fixed step counts)
  double a;            // kinetic speed a_n of the pending step
  double inv2a;        // 0.5 / a_n
  double dt;           // dx / a_n (or t_target - t_n when landing)
  double inv2a_prev;   // MIXED: the 1/(2a) the stored non-equilibrium parts refer to
  float inv2a_f;       // MIXED: 1/(2a_n) rounded down to FP32 (a_eff >= a_n)
  float dinv2a_f;      // MIXED: inv2a_prev - inv2a_f, the correction of the stored parts
  long long steps;     // steps taken; lattice parity = steps & 1
  unsigned long long lam_bits;       // lambda(u^n) as ordered bits of a non-negative double
  unsigned long long lam_next_bits;  // lambda(u^{n+1}) accumulated by the running step
  int active;          // the pending step runs for this realization
  int landing;         // the pending step lands on t_target
  int flags;           // sticky: 1 non-positive, 2 non-finite, 4 bounded wait gave up
  int gref_set;        // MIXED: inv2a_prev is valid
};

struct LevelDesc {
  int nx, ny, nx_pad;
  int tiles_x, tiles_y;
  int tile_begin;        // first flattened tile index of this level in a step launch
  int wrows;             // rows per warp (warp-marching step kernel)
  double dx, y_min;
  size_t plane;          // elements per plane (ny * nx_pad)
  size_t real_stride;    // elements (double or float4) per realization and lattice
  void* lat;             // lattice storage base
  double* inlet;         // [M][4][ny] conserved inlet state (FP64)
  float4* inlet_f;       // [M][ny] inlet primitives (rho, v1, v2, p) in FP32 (mixed kernel)
  RealState* rs;         // [M]
};

struct Physics {
  double gamma, alpha, kappa;
  int limiter;
  double rlmp_rel, rlmp_abs, eps_pos;
  double jet_rho, jet_u, jet_v, jet_p;
  double amb_rho, amb_u, amb_v, amb_p;
};

// FP32 constants of the mixed kernel, rounded once on the host so the kernel
// issues no FP64 instruction (GB300's FP64 pipe runs at 1/58 of FP32).
struct PhysicsF32 {
  float gamma, gm1, rg;  // gamma, gamma - 1, 1 / (gamma - 1)
  float alpha, c1;       // alpha, (1 - alpha) / 4
  float rel, absb, eps;  // rlmp_rel, rlmp_abs, eps_pos
};

struct Launch {
  Physics ph;
  PhysicsF32 pf;
  int nlevels;
  int M;
  int total_tiles;
  int march_rows;  // rows per warp of the mixed warp-march designs (0: the launcher's rule)
  LevelDesc lv[kMaxLevels];
  // TMA descriptors of the mixed kernel, filled per launch for the tile shape
  // in use: nodal-state boxes (radius-2 halo) and non-equilibrium boxes
  // (radius-1 halo, all four populations) of each level's lattice storage.
  CUtensorMap tmP[kMaxLevels];
  CUtensorMap tmG[kMaxLevels];
};

// Ordered bits of a non-negative double (monotone as unsigned integers).
__host__ __device__ inline unsigned long long lam_to_bits(double x) {
  union {
    double d;
    unsigned long long u;
  } c;
  c.d = x;
  return c.u;
}
__host__ __device__ inline double bits_to_lam(unsigned long long b) {
  union {
    double d;
    unsigned long long u;
  } c;
  c.u = b;
  return c.d;
}

// Counts kernel launches enqueued by the library (see vlbm_kernel_launches).
void add_launches(unsigned n);

// Runs set() once per device (the current one) for the flag word `done`.
// Kernel attributes such as the dynamic shared-memory limit are per device,
// so a process that uses several GPUs configures each of them.  Two threads
// may both run set() for a device the first time; it is idempotent.
template <class F>
cudaError_t once_per_device(std::atomic<unsigned long long>& done, F set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return set();
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Launch helpers implemented in the kernel translation units.
// FP64 step kernel designs 0..f64_variants()-1: 32 x 8 tiles, warps marching
// up 28-column strips.  Both compute identical results.
cudaError_t launch_step_f64(const Launch& L, int variant, cudaStream_t s);
int f64_variants();
const char* f64_variant_name(int variant);
size_t step_f64_smem_bytes();
void tiles_f64(int nx, int ny, int* tx, int* ty);

// Mixed kernel launch designs 0..mixed_variants()-1: 32 x TY tiles (one tile
// per CTA, or persistent CTAs with double-buffered TMA prefetch) and warps
// marching up column strips.  All compute bit-identical results.
int mixed_variants();
const char* mixed_variant_name(int variant);
// For the warp-march designs: the rows per warp a launch of L uses
// (L.march_rows, or the launcher's rule when 0), and the CTAs of that launch
// over the CTAs the GPU holds at once; 0 for the other designs.
int mixed_march_rows(const Launch& L, int variant);
double mixed_march_waves(const Launch& L, int variant, int rows);
// Fills the tile decomposition and TMA descriptors of `variant` into a copy of
// L and launches; returns cudaErrorNotSupported if the driver lacks TMA encode.
cudaError_t launch_step_mixed(const Launch& L, int variant, cudaStream_t s);

// xi: NULL (Philox draws from seed, m_begin) or device [M][2K] given uniforms.
// Block average of M fields [ny][nx] onto [ny / r][nx / r] (r divides both).
cudaError_t restrict_launch(const void* ens, int is_f32, int nx, int ny, int M, int r, void* out, int out_f32,
                            cudaStream_t s);

// Statistics launchers (vlbm_stats.cu, vlbm_diag.cu); the int-returning ones
// report a status code and, on failure, a reason in *why.
size_t functional_scratch_doubles(int M);
int noalloc_max_m();
cudaError_t noalloc_scratch(double** out, bool lookup);
int functional_check(int nxa, int nya, int nxb, int nyb, int M, const char** why);
cudaError_t functional_launch(const void* a, int a_f32, int nxa, int nya, const void* b, int b_f32, int nxb, int M,
                              double* scratch, double* out, cudaStream_t s);
int quantile_launch(const void* ens, int f32, int nx, int ny, int M, const double* probs, int nprob, double* out,
                    cudaStream_t s, const char** why);
int histogram_launch(const void* ens, int f32, int nx, int ny, int M, const double* edges, int nbins, double* out,
                     cudaStream_t s, const char** why);
int stats_launch(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32, int nxb,
                 int nyb, int M, double* mean_a, double* std_a, double* mean_b, double* std_b, double* w1,
                 cudaStream_t s, const char** why);

// Two-point Wasserstein distance (vlbm_w12.cu): per-pair values into pair_w
// [npd^4] and their mean into *out (device).  Dynamic shared memory per CTA:
size_t w12_smem_bytes(int M);
cudaError_t w12_launch(const void* a, int a_f32, int nxa, int nya, const void* b, int b_f32, int nxb, int r, int M,
                       int npd, double* pair_w, double* out, cudaStream_t s);

// One mbarrier wait that nothing completes, bounded by limit_ns; *status = 4
// (device int) when the bound ended it.
cudaError_t launch_bounded_wait_probe(int* status, unsigned long long limit_ns, cudaStream_t s);

// xi: NULL (Philox draws from seed, m_begin) or device [M][2K] given uniforms;
// with Philox draws, xi_out (device [M][2K], may be NULL) receives them.
cudaError_t launch_inlet(const Launch& L, uint64_t seed, int m_begin, const vlbm_perturb& P, const double* xi,
                         double* xi_out, cudaStream_t s);

// Discrete adjoint of the FP64 step on one level (vlbm_adjoint.cu).  States
// are [M][20][plane] FP64 (u, populations) in the lattice layout.
size_t adjoint_scratch_doubles(const LevelDesc& D, int M);
size_t adjoint_scratch_ints(const LevelDesc& D, int M);
cudaError_t adjoint_objective(const Launch& L, int level, const double* state, const double* w, double* Jm,
                              double* aseed, cudaStream_t s);
cudaError_t adjoint_step(const Launch& L, int level, double r_jet, const double* state, const RealState* rs,
                         const double* ain, double* aout, double* scr, int* iscr, double* inlet_acc,
                         cudaStream_t s);
cudaError_t adjoint_initial(const Launch& L, int level, double r_jet, const double* state0, const RealState* rs0,
                            const double* ain, double* aout, double* scr, double* inlet_acc, cudaStream_t s);
cudaError_t adjoint_amplitudes(const Launch& L, int level, double r_jet, const double* inlet_acc, const double* xi,
                               int K, double* grad, cudaStream_t s);
cudaError_t launch_init_state(const Launch& L, int precision, cudaStream_t s);
cudaError_t launch_lambda(const Launch& L, int precision, int level, int m0, int count, cudaStream_t s);
cudaError_t launch_fill_equilibrium_f64(const Launch& L, int level, int m0, int count, cudaStream_t s);
cudaError_t launch_tick(const Launch& L, int precision, int advance, cudaStream_t s);
cudaError_t launch_set_target(const Launch& L, double t_target, cudaStream_t s);
cudaError_t launch_moments(const Launch& L, int precision, int level, int m0, int count, double* rho,
                           double* u, double* v, double* p, cudaStream_t s);
cudaError_t launch_density(const Launch& L, int precision, int level, int m0, int count, void* rho,
                           int as_f32, cudaStream_t s);
cudaError_t launch_get_state(const Launch& L, int precision, int level, int m0, int count, double* u,
                             double* pops, cudaStream_t s);
cudaError_t launch_set_state(const Launch& L, int precision, int level, int m0, int count, const double* u,
                             const double* pops, cudaStream_t s);
cudaError_t launch_count_active(const Launch& L, int* d_count, cudaStream_t s);

}  // namespace vlbm
