// Host side of the C ABI declared in include/vlbm.h: validation, device
// memory, the per-step launch sequence and its CUDA-graph capture, I/O, the
// statistics entry points, and the checkpointed gradient driver
// (vlbm_grad_amplitudes: forward with checkpoints, then the reverse sweep of
// the adjoint kernels window by window).
//
// One step of the ensemble is two launches on the context stream:
//   step kernel  (every level, realization and tile in one grid)
//   tick kernel  (per realization: t, step count, lambda -> a_{n+1}, landing)
// vlbm_step / vlbm_advance_to replay a captured graph of kGraphSteps such
// pairs, so a long run costs one graph launch per kGraphSteps steps.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <vector>

#include "vlbm_internal.cuh"


using namespace vlbm;

namespace {

constexpr int kGraphSteps = 32;
constexpr uint32_t kSaveMagic = 0x564c424du;  // "VLBM"
constexpr uint32_t kSaveVersion = 1;

thread_local std::string g_thread_error = "no error";
std::atomic<unsigned long long> g_launches{0};
thread_local bool g_capturing = false;

struct LevelMem {
  void* lat = nullptr;
  double* inlet = nullptr;
  float4* inlet_f = nullptr;
  RealState* rs = nullptr;
  size_t lat_bytes = 0, inlet_bytes = 0, inlet_f_bytes = 0, rs_bytes = 0;
};

}  // namespace

namespace vlbm {
void add_launches(unsigned n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
}  // namespace vlbm

struct vlbm_ctx {
  std::vector<vlbm_grid> grids;
  Physics ph{};
  int precision = VLBM_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  vlbm_alloc_fn alloc = nullptr;
  vlbm_free_fn free_fn = nullptr;
  void* user = nullptr;
  int M = 0;
  bool initialized = false;
  bool prepared = false;
  double target = std::numeric_limits<double>::infinity();
  std::vector<LevelMem> mem;
  Launch launch{};
  int* d_count = nullptr;
  double* d_xi = nullptr;  // KL uniforms of every realization, given or drawn: [M][2K]
  size_t xi_bytes = 0;
  std::vector<double> amp;  // per-mode amplitudes of the last initialisation
  double r_jet = 0.05;
  cudaGraphExec_t graph = nullptr;
  bool warmed = false;
  int variant = -1;  // step kernel launch design (index), -1: not tuned yet
  std::vector<float> tune_ms;  // time per step of every variant when tuned
  std::string err = "no error";
};

namespace {

int fail(vlbm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  g_thread_error = msg;
  return code;
}

int cuda_fail(vlbm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, VLBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dev_alloc(vlbm_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 256;
  if (c->alloc) return c->alloc(bytes, c->user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(vlbm_ctx* c, void* p) {
  if (!p) return;
  if (c->free_fn)
    c->free_fn(p, c->user);
  else if (!c->alloc)
    cudaFree(p);
}

void release_levels(vlbm_ctx* c) {
  for (auto& m : c->mem) {
    dev_free(c, m.lat);
    dev_free(c, m.inlet);
    dev_free(c, m.inlet_f);
    dev_free(c, m.rs);
  }
  c->mem.clear();
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->warmed = false;
  c->variant = -1;  // a new ensemble size is tuned again
}

// Launch designs of the context's step kernel: count, and one step launch of
// design v (no tick).
int step_designs(const vlbm_ctx* c) { return c->precision == VLBM_FP64 ? f64_variants() : mixed_variants(); }
cudaError_t launch_design(vlbm_ctx* c, int v) {
  if (v < 0) v = step_designs(c) - 1;  // not tuned yet: the last design
  return c->precision == VLBM_FP64 ? launch_step_f64(c->launch, v, c->stream)
                                   : launch_step_mixed(c->launch, v, c->stream);
}

// Picks the step kernel's launch design (mixed: tile shapes, persistent CTAs,
// warp marches; FP64: tiles or the warp march) by timing every design on the
// live state.  A step launch without the tick that follows it is idempotent:
// it rewrites the same next lattice and max-reduces the same lambda.  On a
// mixed launch that does not fill the GPU once (a single small grid) each
// design is timed over more launches and every warp march also at several
// rows per warp: fewer rows give more CTAs and a shorter march each but
// re-evaluate more halo rows.  The environment variable
// VLBM_MIXED_VARIANT / VLBM_F64_VARIANT (an index) forces a design (no
// timing), VLBM_MARCH_ROWS the rows per warp of a mixed march.
int tune_design(vlbm_ctx* c) {
  if (c->variant >= 0) return VLBM_OK;
  const int n = step_designs(c);
  const bool mixed = c->precision == VLBM_MIXED;
  c->launch.march_rows = 0;
  const char* env_rows = mixed ? std::getenv("VLBM_MARCH_ROWS") : nullptr;
  if (env_rows && std::atoi(env_rows) > 0) c->launch.march_rows = std::atoi(env_rows);
  if (const char* env = std::getenv(mixed ? "VLBM_MIXED_VARIANT" : "VLBM_F64_VARIANT")) {
    const int v = std::atoi(env);
    if (v >= 0 && v < n) {
      c->variant = v;
      return VLBM_OK;
    }
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(c, VLBM_ECUDA, "cudaEventCreate");
  // time per launch of design v over `reps` launches after an untimed one
  auto time_design = [&](int v, int reps, float& ms) {
    cudaError_t e = launch_design(c, v);
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_design(c, v);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    return e;
  };
  // a launch that does not fill the GPU once with the march rule's rows (a
  // single small grid) is timed over more launches, and a march there over
  // several row counts; larger launches keep the rule, whose rows suit the
  // developed flow as well as the first step that the tuning sees
  const bool tune_rows = mixed && c->launch.march_rows == 0;
  bool small = false;
  for (int v = 0; v < n && mixed; ++v) {
    const double w = mixed_march_waves(c->launch, v, 0);
    small = small || (w > 0.0 && w < 1.0);
  }
  const int reps = small ? 16 : 2;
  static const int kRows[] = {0, 1, 2, 3, 4, 6, 8, 12, 16};  // 0: the launcher's rule
  float best = 1e30f;
  int best_v = n - 1, best_rows = c->launch.march_rows;
  c->tune_ms.assign(n, 0.0f);
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < n && e == cudaSuccess; ++v) {
    const bool rows_too = tune_rows && small && mixed_march_rows(c->launch, v) > 0;
    for (int r : kRows) {
      if (r != 0 && !rows_too) break;
      if (tune_rows) c->launch.march_rows = r;
      float ms = 0;
      e = time_design(v, reps, ms);
      if (e != cudaSuccess) break;
      if (r == 0) c->tune_ms[v] = ms;
      if (ms < best) {
        best = ms;
        best_v = v;
        best_rows = c->launch.march_rows;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->launch.march_rows = e == cudaSuccess ? best_rows : 0;
  if (e != cudaSuccess) return cuda_fail(c, e, "tuning the step kernel");
  c->variant = best_v;
  return VLBM_OK;
}

int launch_one_step(vlbm_ctx* c) {
  cudaError_t e = launch_design(c, c->variant);
  if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
  e = launch_tick(c->launch, c->precision, 1, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "tick kernel launch");
  return VLBM_OK;
}

int build_graph(vlbm_ctx* c) {
  if (c->graph) return VLBM_OK;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
  int st = VLBM_OK;
  g_capturing = true;
  for (int s = 0; s < kGraphSteps && st == VLBM_OK; ++s) st = launch_one_step(c);
  g_capturing = false;
  e = cudaStreamEndCapture(c->stream, &g);
  if (st != VLBM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    return cuda_fail(c, e, "cudaGraphInstantiate");
  }
  return VLBM_OK;
}

int run_steps(vlbm_ctx* c, long long n) {
  // the first steps run as plain launches (this also configures the kernels'
  // shared-memory limits before any capture)
  if (n > 0) {
    int st = tune_design(c);
    if (st) return st;
  }
  while (n > 0 && !c->warmed) {
    int st = launch_one_step(c);
    if (st) return st;
    --n;
    c->warmed = true;
  }
  while (n >= kGraphSteps) {
    int st = build_graph(c);
    if (st) return st;
    cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
    add_launches(2 * kGraphSteps);
    n -= kGraphSteps;
  }
  while (n-- > 0) {
    int st = launch_one_step(c);
    if (st) return st;
  }
  return VLBM_OK;
}

int prepare(vlbm_ctx* c, double target) {
  if (c->prepared && (c->target == target || (std::isinf(c->target) && std::isinf(target)))) return VLBM_OK;
  cudaError_t e = launch_set_target(c->launch, target, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_target");
  e = launch_tick(c->launch, c->precision, 0, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "tick");
  c->target = target;
  c->prepared = true;
  return VLBM_OK;
}

int read_flags(vlbm_ctx* c, int level_only, std::vector<RealState>* out_level) {
  int worst = VLBM_OK;
  for (int l = 0; l < (int)c->mem.size(); ++l) {
    if (level_only >= 0 && l != level_only) continue;
    std::vector<RealState> h(c->M);
    cudaError_t e = cudaMemcpy(h.data(), c->mem[l].rs, sizeof(RealState) * c->M, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading realization state");
    for (int m = 0; m < c->M; ++m) {
      if (h[m].flags & 4) {
        worst = VLBM_ETIMEOUT;
        fail(c, worst, "level " + std::to_string(l) + " realization " + std::to_string(m) +
                           ": a bounded device wait gave up");
      } else if ((h[m].flags & 2) && worst != VLBM_ETIMEOUT) {
        worst = VLBM_ENONFINITE;
        fail(c, worst, "level " + std::to_string(l) + " realization " + std::to_string(m) + ": non-finite state");
      } else if ((h[m].flags & 1) && worst == VLBM_OK) {
        worst = VLBM_ENONPOSITIVE;
        fail(c, worst,
             "level " + std::to_string(l) + " realization " + std::to_string(m) + ": rho or p not positive");
      }
    }
    if (out_level) *out_level = h;
  }
  return worst;
}

int check_level(vlbm_ctx* c, int level, int m0, int count) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  if (!c->initialized) return fail(c, VLBM_ESTATE, "vlbm_init_ensemble has not been called");
  if (level < 0 || level >= (int)c->grids.size()) return fail(c, VLBM_EINVAL, "level out of range");
  if (m0 < 0 || count < 0 || m0 + count > c->M) return fail(c, VLBM_EINVAL, "realization range out of [0, M)");
  return VLBM_OK;
}

}  // namespace

namespace {

// Returns true when p is device (or managed) memory; host memory otherwise,
// including when no device is present.
bool is_device_pointer(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}


int init_impl(vlbm_ctx* c, uint64_t seed, int m_begin, int M, const vlbm_perturb* perturb, const double* xi) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  if (c->own_stream && !c->stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      c->stream = nullptr;
      return cuda_fail(c, e, "cudaStreamCreate");
    }
  }
  if (M < 1 || M > 65535) return fail(c, VLBM_EINVAL, "M must be in [1, 65535]");
  if (m_begin < 0 || (long long)m_begin + M > 0xffffffffLL)
    return fail(c, VLBM_EINVAL, "realization block must lie in [0, 2^32)");
  vlbm_perturb P;
  vlbm_default_perturb(&P);
  if (perturb) P = *perturb;
  if (P.K < 0 || P.K > kMaxModes) return fail(c, VLBM_EINVAL, "K must be in [0, 16]");
  if (!(P.r_jet > 0.0) || !std::isfinite(P.r_jet)) return fail(c, VLBM_EINVAL, "r_jet must be finite and > 0");
  if (!std::isfinite(P.A) || !std::isfinite(P.p_decay))
    return fail(c, VLBM_EINVAL, "the perturbation amplitude A and decay p must be finite");
  if (P.use_amp)
    for (int k = 0; k < P.K; ++k)
      if (!std::isfinite(P.amp[k])) return fail(c, VLBM_EINVAL, "amp[" + std::to_string(k) + "] is not finite");
  // from here on the context's state changes: until this call completes it
  // holds no ensemble (a failure below leaves VLBM_ESTATE for the next call)
  c->initialized = false;
  c->prepared = false;
  if (c->M != M || c->mem.empty()) {
    release_levels(c);
    c->mem.resize(c->grids.size());
    for (size_t l = 0; l < c->grids.size(); ++l) {
      const vlbm_grid& g = c->grids[l];
      const int nx_pad = (g.nx + 31) / 32 * 32;
      const size_t plane = (size_t)g.ny * nx_pad;
      const size_t real = c->precision == VLBM_FP64 ? 20 * plane * sizeof(double) : 5 * plane * sizeof(float4);
      LevelMem& mm = c->mem[l];
      mm.lat_bytes = 2 * (size_t)M * real;
      mm.inlet_bytes = (size_t)M * 4 * g.ny * sizeof(double);
      mm.inlet_f_bytes = (size_t)M * g.ny * sizeof(float4);
      mm.rs_bytes = (size_t)M * sizeof(RealState);
      mm.lat = dev_alloc(c, mm.lat_bytes);
      mm.inlet = static_cast<double*>(dev_alloc(c, mm.inlet_bytes));
      mm.inlet_f = static_cast<float4*>(dev_alloc(c, mm.inlet_f_bytes));
      mm.rs = static_cast<RealState*>(dev_alloc(c, mm.rs_bytes));
      if (!mm.lat || !mm.inlet || !mm.inlet_f || !mm.rs) {
        release_levels(c);
        c->M = 0;
        return fail(c, VLBM_ENOMEM,
                    "device allocation of " + std::to_string(mm.lat_bytes) + " bytes for level " +
                        std::to_string(l) + " failed");
      }
    }
    if (!c->d_count) {
      c->d_count = static_cast<int*>(dev_alloc(c, sizeof(int)));
      if (!c->d_count) {
        release_levels(c);
        c->M = 0;
        return fail(c, VLBM_ENOMEM, "device allocation of the active-realization counter failed");
      }
    }
    c->M = M;
  }
  // launch descriptor
  Launch& L = c->launch;
  const int rows = L.march_rows;  // tuned for this ensemble size (0 after release_levels)
  L = Launch{};
  L.march_rows = c->variant >= 0 ? rows : 0;
  L.ph = c->ph;
  L.pf.gamma = (float)c->ph.gamma;
  L.pf.gm1 = (float)(c->ph.gamma - 1.0);
  L.pf.rg = (float)(1.0 / (c->ph.gamma - 1.0));
  L.pf.alpha = (float)c->ph.alpha;
  L.pf.c1 = (float)((1.0 - c->ph.alpha) / 4.0);
  L.pf.rel = (float)c->ph.rlmp_rel;
  L.pf.absb = (float)c->ph.rlmp_abs;
  L.pf.eps = (float)c->ph.eps_pos;
  L.nlevels = (int)c->grids.size();
  L.M = M;
  int tiles = 0;
  for (int l = 0; l < L.nlevels; ++l) {
    const vlbm_grid& g = c->grids[l];
    LevelDesc& D = L.lv[l];
    D.nx = g.nx;
    D.ny = g.ny;
    D.nx_pad = (g.nx + 31) / 32 * 32;
    D.dx = g.x_max / g.nx;
    D.y_min = g.y_min;
    D.plane = (size_t)g.ny * D.nx_pad;
    D.real_stride = c->precision == VLBM_FP64 ? 20 * D.plane : 5 * D.plane;
    // FP64 tiles here; the mixed kernel lays out its own tiles per shape
    tiles_f64(g.nx, g.ny, &D.tiles_x, &D.tiles_y);
    D.tile_begin = tiles;
    tiles += D.tiles_x * D.tiles_y;
    D.lat = c->mem[l].lat;
    D.inlet = c->mem[l].inlet;
    D.inlet_f = c->mem[l].inlet_f;
    D.rs = c->mem[l].rs;
  }
  L.total_tiles = tiles;
  if (c->graph) {
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  cudaError_t e;
  for (int l = 0; l < L.nlevels; ++l) {
    e = cudaMemsetAsync(c->mem[l].lat, 0, c->mem[l].lat_bytes, c->stream);
    add_launches(1);
    if (e != cudaSuccess) return cuda_fail(c, e, "clearing the lattice");
  }
  // the KL uniforms are kept (given, or recorded when drawn) for gradients
  const size_t xi_bytes = (size_t)M * 2 * P.K * sizeof(double);
  if (xi_bytes > c->xi_bytes) {
    dev_free(c, c->d_xi);
    c->d_xi = static_cast<double*>(dev_alloc(c, xi_bytes));
    c->xi_bytes = c->d_xi ? xi_bytes : 0;
    if (!c->d_xi) return fail(c, VLBM_ENOMEM, "device allocation of the KL uniforms failed");
  }
  const double* d_xi = nullptr;
  if (xi) {
    if (xi_bytes) {
      e = cudaMemcpyAsync(c->d_xi, xi, xi_bytes, cudaMemcpyDefault, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "copying the KL uniforms");
    }
    d_xi = c->d_xi;
  }
  c->amp.assign(P.K, 0.0);
  for (int k = 1; k <= P.K; ++k) c->amp[k - 1] = P.use_amp ? P.amp[k - 1] : P.A * std::pow((double)k, -P.p_decay);
  c->r_jet = P.r_jet;
  e = launch_inlet(L, seed, m_begin, P, d_xi, c->d_xi, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "inlet kernel");
  e = launch_init_state(L, c->precision, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "initial state kernel");
  for (int l = 0; l < L.nlevels; ++l) {
    e = launch_lambda(L, c->precision, l, 0, M, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "kinetic speed kernel");
    if (c->precision == VLBM_FP64) {
      e = launch_fill_equilibrium_f64(L, l, 0, M, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "equilibrium kernel");
    }
  }
  c->initialized = true;
  c->prepared = false;
  return VLBM_OK;
}

}  // namespace

extern "C" {

void vlbm_default_relax(vlbm_relax* r) {
  if (!r) return;
  r->alpha = 0.0;
  r->kappa = 1.0;
  r->limiter = VLBM_LIMITER_RTHETA;
  r->rlmp_rel = 0.1;
  r->rlmp_abs = 0.0;
  r->eps_pos = 1e-13;
}

void vlbm_default_perturb(vlbm_perturb* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->r_jet = 0.05;
  p->A = 0.1;
  p->p_decay = 2.0;
  p->K = 10;
  p->use_amp = 0;
}

int vlbm_create(const vlbm_grid* levels, int nlevels, double gamma, const vlbm_prim* jet,
                const vlbm_prim* ambient, const vlbm_relax* relax, int precision, void* cuda_stream,
                vlbm_alloc_fn alloc, vlbm_free_fn free_fn, void* alloc_user, vlbm_ctx** out) {
  if (!out) return fail(nullptr, VLBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!levels || nlevels < 1 || nlevels > kMaxLevels)
    return fail(nullptr, VLBM_EINVAL, "need 1..8 grid levels");
  if (!jet || !ambient) return fail(nullptr, VLBM_EINVAL, "jet and ambient states are required");
  if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(nullptr, VLBM_EINVAL, "gamma must be > 1");
  if (!(jet->rho > 0) || !(jet->p > 0) || !(ambient->rho > 0) || !(ambient->p > 0))
    return fail(nullptr, VLBM_EINVAL, "jet and ambient states need rho > 0 and p > 0");
  for (const vlbm_prim* s : {jet, ambient})
    if (!std::isfinite(s->rho) || !std::isfinite(s->u) || !std::isfinite(s->v) || !std::isfinite(s->p))
      return fail(nullptr, VLBM_EINVAL, "jet and ambient states must be finite");
  if (precision != VLBM_FP64 && precision != VLBM_MIXED) return fail(nullptr, VLBM_EINVAL, "unknown precision");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, VLBM_EINVAL, "alloc and free callbacks must be given together");
  vlbm_relax R;
  vlbm_default_relax(&R);
  if (relax) R = *relax;
  for (double v : {R.alpha, R.kappa, R.rlmp_rel, R.rlmp_abs, R.eps_pos})
    if (!std::isfinite(v)) return fail(nullptr, VLBM_EINVAL, "relaxation parameters must be finite");
  if (!(R.alpha >= 0.0 && R.alpha < 1.0)) return fail(nullptr, VLBM_EINVAL, "alpha must be in [0, 1)");
  if (!(R.kappa >= 1.0)) return fail(nullptr, VLBM_EINVAL, "kappa must be >= 1 (Bouchut bound)");
  if (R.limiter < 0 || R.limiter > 2) return fail(nullptr, VLBM_EINVAL, "unknown limiter");
  if (!(R.rlmp_rel >= 0.0) || !(R.rlmp_abs >= 0.0) || !(R.eps_pos >= 0.0))
    return fail(nullptr, VLBM_EINVAL, "rlmp_rel, rlmp_abs and eps_pos must be >= 0");
  for (int l = 0; l < nlevels; ++l) {
    const vlbm_grid& g = levels[l];
    if (g.nx < 3 || g.ny < 3) return fail(nullptr, VLBM_EINVAL, "every level needs nx, ny >= 3");
    if ((long long)g.nx * g.ny > (1LL << 31)) return fail(nullptr, VLBM_EINVAL, "level too large");
    if (!std::isfinite(g.x_max) || !std::isfinite(g.y_min) || !std::isfinite(g.y_max))
      return fail(nullptr, VLBM_EINVAL, "grid extents must be finite");
    if (!(g.x_max > 0) || !(g.y_max > g.y_min)) return fail(nullptr, VLBM_EINVAL, "empty domain");
    const double dx = g.x_max / g.nx, dy = (g.y_max - g.y_min) / g.ny;
    if (std::fabs(dx - dy) > 1e-12 * dx) return fail(nullptr, VLBM_EINVAL, "cells must be square");
  }
  vlbm_ctx* c = new (std::nothrow) vlbm_ctx();
  if (!c) return fail(nullptr, VLBM_ENOMEM, "host allocation failed");
  c->grids.assign(levels, levels + nlevels);
  c->ph.gamma = gamma;
  c->ph.alpha = R.alpha;
  c->ph.kappa = R.kappa;
  c->ph.limiter = R.limiter;
  c->ph.rlmp_rel = R.rlmp_rel;
  c->ph.rlmp_abs = R.rlmp_abs;
  c->ph.eps_pos = R.eps_pos;
  c->ph.jet_rho = jet->rho;
  c->ph.jet_u = jet->u;
  c->ph.jet_v = jet->v;
  c->ph.jet_p = jet->p;
  c->ph.amb_rho = ambient->rho;
  c->ph.amb_u = ambient->u;
  c->ph.amb_v = ambient->v;
  c->ph.amb_p = ambient->p;
  c->precision = precision;
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = alloc_user;
  // a private stream (cuda_stream NULL) is created by the first call that
  // enqueues work, so that creating a context touches no device
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->own_stream = cuda_stream == nullptr;
  *out = c;
  return VLBM_OK;
}

int vlbm_init_ensemble(vlbm_ctx* c, uint64_t seed, int M, const vlbm_perturb* perturb) {
  return vlbm_init_ensemble_block(c, seed, 0, M, perturb);
}


int vlbm_init_ensemble_samples(vlbm_ctx* c, const double* xi, int M, const vlbm_perturb* perturb) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  if (!xi) return fail(c, VLBM_EINVAL, "xi is NULL");
  if (M < 1 || M > 65535) return fail(c, VLBM_EINVAL, "M must be in [1, 65535]");
  vlbm_perturb P;
  vlbm_default_perturb(&P);
  if (perturb) P = *perturb;
  if (P.K < 0 || P.K > kMaxModes) return fail(c, VLBM_EINVAL, "K must be in [0, 16]");
  if (!is_device_pointer(xi)) {
    const size_t n = (size_t)M * 2 * P.K;
    for (size_t i = 0; i < n; ++i)
      if (!(xi[i] >= -1.0 && xi[i] <= 1.0))
        return fail(c, VLBM_EINVAL, "xi[" + std::to_string(i) + "] is not in [-1, 1]");
  }
  return init_impl(c, 0, 0, M, &P, xi);
}

int vlbm_init_ensemble_block(vlbm_ctx* c, uint64_t seed, int m_begin, int M, const vlbm_perturb* perturb) {
  return init_impl(c, seed, m_begin, M, perturb, nullptr);
}


int vlbm_step(vlbm_ctx* c, int n) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  if (!c->initialized) return fail(c, VLBM_ESTATE, "vlbm_init_ensemble has not been called");
  if (n < 0) return fail(c, VLBM_EINVAL, "n must be >= 0");
  int st = prepare(c, std::numeric_limits<double>::infinity());
  if (st) return st;
  return run_steps(c, n);
}

int vlbm_advance_to(vlbm_ctx* c, double t) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  if (!c->initialized) return fail(c, VLBM_ESTATE, "vlbm_init_ensemble has not been called");
  if (!(t >= 0.0) || !std::isfinite(t)) return fail(c, VLBM_EINVAL, "t must be finite and >= 0");
  int st = prepare(c, t);
  if (st) return st;
  for (long long guard = 0; guard < (1LL << 40); guard += kGraphSteps) {
    cudaError_t e = launch_count_active(c->launch, c->d_count, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "count kernel");
    int h = 0;
    e = cudaMemcpyAsync(&h, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the active count");
    if (h == 0) break;
    st = run_steps(c, kGraphSteps);
    if (st) return st;
  }
  return read_flags(c, -1, nullptr);
}

int vlbm_moments(vlbm_ctx* c, int level, int m0, int count, double* rho, double* u, double* v, double* p) {
  int st = check_level(c, level, m0, count);
  if (st) return st;
  if (count == 0) return VLBM_OK;
  cudaError_t e = launch_moments(c->launch, c->precision, level, m0, count, rho, u, v, p, c->stream);
  return e == cudaSuccess ? VLBM_OK : cuda_fail(c, e, "moments kernel");
}

int vlbm_density(vlbm_ctx* c, int level, int m0, int count, void* rho, int as_f32) {
  int st = check_level(c, level, m0, count);
  if (st) return st;
  if (!rho) return fail(c, VLBM_EINVAL, "rho is NULL");
  if (count == 0) return VLBM_OK;
  cudaError_t e = launch_density(c->launch, c->precision, level, m0, count, rho, as_f32, c->stream);
  return e == cudaSuccess ? VLBM_OK : cuda_fail(c, e, "density kernel");
}

int vlbm_time(vlbm_ctx* c, int level, double* t_host, long long* steps_host) {
  int st = check_level(c, level, 0, 0);
  if (st) return st;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  std::vector<RealState> h;
  st = read_flags(c, level, &h);
  if (h.size() != (size_t)c->M) return st;  // the device read itself failed
  for (int m = 0; m < c->M; ++m) {
    if (t_host) t_host[m] = h[m].t;
    if (steps_host) steps_host[m] = h[m].steps;
  }
  return st;
}

int vlbm_sync(vlbm_ctx* c) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  if (!c->initialized) return VLBM_OK;
  return read_flags(c, -1, nullptr);
}

int vlbm_get_state(vlbm_ctx* c, int level, int m0, int count, double* u, double* pops) {
  int st = check_level(c, level, m0, count);
  if (st) return st;
  if (!u) return fail(c, VLBM_EINVAL, "u is NULL");
  if (count == 0) return VLBM_OK;
  cudaError_t e = launch_get_state(c->launch, c->precision, level, m0, count, u, pops, c->stream);
  return e == cudaSuccess ? VLBM_OK : cuda_fail(c, e, "get_state kernel");
}

int vlbm_set_state(vlbm_ctx* c, int level, int m0, int count, const double* u, const double* pops) {
  int st = check_level(c, level, m0, count);
  if (st) return st;
  if (!u || !pops) return fail(c, VLBM_EINVAL, "u and pops are required");
  if (count == 0) return VLBM_OK;
  cudaError_t e = launch_set_state(c->launch, c->precision, level, m0, count, u, pops, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "set_state kernels");
  c->prepared = false;
  return VLBM_OK;
}

int stats_w1_mean_std(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32,
                      int nxb, int nyb, int M, double* mean_a, double* std_a, double* mean_b, double* std_b,
                      double* w1, void* cuda_stream) {
  const char* why = "";
  int st = stats_launch(ens_a, a_is_f32, nxa, nya, ens_b, b_is_f32, nxb, nyb, M, mean_a, std_a, mean_b, std_b, w1,
                        static_cast<cudaStream_t>(cuda_stream), &why);
  if (st) return fail(nullptr, st, why);
  return VLBM_OK;
}

int stats_w1_two_point(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32, int nxb,
                       int nyb, int M, int npd, double* w12, double* pairs, void* cuda_stream) {
  if (!ens_a || !ens_b || !w12) return fail(nullptr, VLBM_EINVAL, "ensemble and output pointers must be non-NULL");
  if (nxa < 1 || nya < 1 || nxb < nxa || nxb % nxa || nyb != nya * (nxb / nxa))
    return fail(nullptr, VLBM_EINVAL, "ensemble b must be an integer refinement of ensemble a");
  if (M < 1 || M > 2048) return fail(nullptr, VLBM_EINVAL, "M must be in [1, 2048]");
  if (npd < 1 || npd > nxa || npd > nya || npd > 215)
    return fail(nullptr, VLBM_EINVAL, "npd must be in [1, min(nx, ny, 215)]");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t P = (size_t)npd * npd * npd * npd;
  double* scratch = nullptr;
  cudaError_t e = cudaSuccess;
  if (!pairs) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), P * sizeof(double), s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMallocAsync for the pair values");
  }
  e = w12_launch(ens_a, a_is_f32 != 0, nxa, nya, ens_b, b_is_f32 != 0, nxb, nxb / nxa, M, npd, pairs ? pairs : scratch,
                 w12, s);
  cudaError_t e2 = scratch ? cudaFreeAsync(scratch, s) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "two-point Wasserstein kernels");
  if (e2 != cudaSuccess) return cuda_fail(nullptr, e2, "cudaFreeAsync");
  return VLBM_OK;
}

int stats_restrict(const void* ens, int is_f32, int nx, int ny, int M, int r, void* out, int out_is_f32,
                   void* cuda_stream) {
  if (!ens || !out) return fail(nullptr, VLBM_EINVAL, "ensemble and output pointers must be non-NULL");
  if (nx < 1 || ny < 1 || M < 1 || r < 1) return fail(nullptr, VLBM_EINVAL, "nx, ny, M and r must be >= 1");
  if (nx % r || ny % r) return fail(nullptr, VLBM_EINVAL, "r must divide nx and ny");
  if (M > 65535) return fail(nullptr, VLBM_EINVAL, "M must be <= 65535");
  cudaError_t e = restrict_launch(ens, is_f32 != 0, nx, ny, M, r, out, out_is_f32 != 0,
                                  static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "restriction kernel");
  return VLBM_OK;
}

int stats_error_functionals(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32,
                            int nxb, int nyb, int M, double* out, void* cuda_stream) {
  const char* why = "";
  if (!ens_a || !ens_b || !out) return fail(nullptr, VLBM_EINVAL, "ensemble and output pointers must be non-NULL");
  int st = functional_check(nxa, nya, nxb, nyb, M, &why);
  if (st) return fail(nullptr, st, why);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), functional_scratch_doubles(M) * sizeof(double), s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMallocAsync for the functional scratch");
  e = functional_launch(ens_a, a_is_f32, nxa, nya, ens_b, b_is_f32, nxb, M, scratch, out, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "error functional kernels");
  if (e2 != cudaSuccess) return cuda_fail(nullptr, e2, "cudaFreeAsync");
  return VLBM_OK;
}

int stats_error_functionals_noalloc(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b,
                                    int b_is_f32, int nxb, int nyb, int M, double* out, void* cuda_stream) {
  const char* why = "";
  if (!ens_a || !ens_b || !out) return fail(nullptr, VLBM_EINVAL, "ensemble and output pointers must be non-NULL");
  if (M > noalloc_max_m())
    return fail(nullptr, VLBM_EINVAL,
                "M = " + std::to_string(M) + " exceeds the " + std::to_string(noalloc_max_m()) +
                    " realizations the allocation-free scratch holds; use stats_error_functionals");
  int st = functional_check(nxa, nya, nxb, nyb, M, &why);
  if (st) return fail(nullptr, st, why);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cs);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaStreamIsCapturing");
  double* scratch = nullptr;
  e = noalloc_scratch(&scratch, cs == cudaStreamCaptureStatusNone);
  if (e == cudaErrorStreamCaptureUnsupported)
    return fail(nullptr, VLBM_ESTATE,
                "the first stats_error_functionals_noalloc call on a device must come before any stream capture "
                "(it looks up the scratch array's device address)");
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress of the functional scratch");
  e = functional_launch(ens_a, a_is_f32, nxa, nya, ens_b, b_is_f32, nxb, M, scratch, out,
                        static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? VLBM_OK : cuda_fail(nullptr, e, "error functional kernels");
}

int stats_quantiles(const void* ens, int is_f32, int nx, int ny, int M, const double* probs, int nprob, double* out,
                    void* cuda_stream) {
  const char* why = "";
  int st = quantile_launch(ens, is_f32, nx, ny, M, probs, nprob, out, static_cast<cudaStream_t>(cuda_stream), &why);
  return st ? fail(nullptr, st, why) : VLBM_OK;
}

int stats_histogram(const void* ens, int is_f32, int nx, int ny, int M, const double* edges, int nbins, double* out,
                    void* cuda_stream) {
  const char* why = "";
  int st = histogram_launch(ens, is_f32, nx, ny, M, edges, nbins, out, static_cast<cudaStream_t>(cuda_stream), &why);
  return st ? fail(nullptr, st, why) : VLBM_OK;
}

int vlbm_save(vlbm_ctx* c, void* host_buf, size_t* bytes) {
  if (!c || !bytes) return fail(c, VLBM_EINVAL, "ctx and bytes are required");
  if (!c->initialized) return fail(c, VLBM_ESTATE, "nothing to save before vlbm_init_ensemble");
  size_t need = 5 * sizeof(uint32_t) + sizeof(uint8_t) * 8;
  for (auto& m : c->mem) need += m.rs_bytes + m.inlet_bytes + m.inlet_f_bytes + m.lat_bytes;
  if (!host_buf) {
    *bytes = need;
    return VLBM_OK;
  }
  if (*bytes < need) return fail(c, VLBM_EINVAL, "host buffer too small");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  unsigned char* p = static_cast<unsigned char*>(host_buf);
  const uint32_t hdr[5] = {kSaveMagic, kSaveVersion, (uint32_t)c->precision, (uint32_t)c->grids.size(),
                           (uint32_t)c->M};
  std::memcpy(p, hdr, sizeof(hdr));
  p += sizeof(hdr);
  std::memset(p, 0, 8);
  p += 8;
  for (auto& m : c->mem) {
    for (auto [src, n] : {std::pair<const void*, size_t>{m.rs, m.rs_bytes}, {m.inlet, m.inlet_bytes},
                          {m.inlet_f, m.inlet_f_bytes}, {m.lat, m.lat_bytes}}) {
      e = cudaMemcpy(p, src, n, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
      p += n;
    }
  }
  *bytes = need;
  return read_flags(c, -1, nullptr);
}

int vlbm_load(vlbm_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf) return fail(c, VLBM_EINVAL, "ctx and host_buf are required");
  if (!c->initialized) return fail(c, VLBM_ESTATE, "call vlbm_init_ensemble with the same M before vlbm_load");
  size_t need = 5 * sizeof(uint32_t) + 8;
  for (auto& m : c->mem) need += m.rs_bytes + m.inlet_bytes + m.inlet_f_bytes + m.lat_bytes;
  if (bytes != need) return fail(c, VLBM_EINVAL, "checkpoint size does not match this context");
  const unsigned char* p = static_cast<const unsigned char*>(host_buf);
  uint32_t hdr[5];
  std::memcpy(hdr, p, sizeof(hdr));
  if (hdr[0] != kSaveMagic || hdr[1] != kSaveVersion || hdr[2] != (uint32_t)c->precision ||
      hdr[3] != (uint32_t)c->grids.size() || hdr[4] != (uint32_t)c->M)
    return fail(c, VLBM_EINVAL, "checkpoint header does not match this context");
  p += sizeof(hdr) + 8;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
  for (auto& m : c->mem) {
    for (auto [dst, n] : {std::pair<void*, size_t>{m.rs, m.rs_bytes}, {m.inlet, m.inlet_bytes},
                          {m.inlet_f, m.inlet_f_bytes}, {m.lat, m.lat_bytes}}) {
      e = cudaMemcpy(dst, p, n, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint restore");
      p += n;
    }
  }
  c->prepared = false;
  return VLBM_OK;
}

int vlbm_grad_amplitudes(vlbm_ctx* c, int nsteps, int checkpoint_every, const double* w, double* J_out,
                         double* grad_out) {
  if (!c) return fail(nullptr, VLBM_EINVAL, "ctx is NULL");
  if (!c->initialized) return fail(c, VLBM_ESTATE, "vlbm_init_ensemble has not been called");
  if (c->precision != VLBM_FP64) return fail(c, VLBM_EINVAL, "gradients need an FP64 context");
  if (c->grids.size() != 1) return fail(c, VLBM_EINVAL, "gradients need a single-level context");
  if (nsteps < 0 || checkpoint_every < 1) return fail(c, VLBM_EINVAL, "need nsteps >= 0 and checkpoint_every >= 1");
  if (!w || !grad_out) return fail(c, VLBM_EINVAL, "w and grad_out are required");
  const int K = (int)c->amp.size();
  const int M = c->M;
  const Launch& L = c->launch;
  const LevelDesc& D = L.lv[0];
  cudaStream_t st = c->stream;
  const size_t sdoubles = (size_t)M * D.real_stride;  // one lattice of every realization
  const size_t sbytes = sdoubles * sizeof(double), rbytes = (size_t)M * sizeof(RealState);
  const int ncp = nsteps == 0 ? 0 : (nsteps + checkpoint_every - 1) / checkpoint_every;
  const int wlen = nsteps < checkpoint_every ? (nsteps > 0 ? nsteps : 1) : checkpoint_every;
  // device buffers (the context's allocator), released on every exit
  std::vector<void*> owned;
  bool alloc_failed = false;
  auto get = [&](size_t bytes) -> void* {
    void* p = dev_alloc(c, bytes ? bytes : 16);
    if (p)
      owned.push_back(p);
    else
      alloc_failed = true;
    return p;
  };
  auto release = [&]() {
    for (void* p : owned) dev_free(c, p);
    owned.clear();
  };
  double* ck = static_cast<double*>(get(sbytes * (size_t)(ncp > 0 ? ncp : 1)));
  RealState* ckr = static_cast<RealState*>(get(rbytes * (size_t)(ncp > 0 ? ncp : 1)));
  double* tr = static_cast<double*>(get(sbytes * (size_t)wlen));
  RealState* trr = static_cast<RealState*>(get(rbytes * (size_t)wlen));
  double* fin = static_cast<double*>(get(sbytes));
  RealState* finr = static_cast<RealState*>(get(rbytes));
  double* adj = static_cast<double*>(get(2 * sbytes));
  double* scr = static_cast<double*>(get(adjoint_scratch_doubles(D, M) * sizeof(double)));
  int* iscr = static_cast<int*>(get(adjoint_scratch_ints(D, M) * sizeof(int)));
  double* inl = static_cast<double*>(get((size_t)M * D.ny * sizeof(double)));
  double* Jm = static_cast<double*>(get((size_t)M * sizeof(double)));
  double* gd = static_cast<double*>(get((size_t)(K > 0 ? K : 1) * sizeof(double)));
  if (alloc_failed) {
    release();
    return fail(c, VLBM_ENOMEM, "device allocation for the adjoint failed");
  }
  double* lat = static_cast<double*>(D.lat);
  auto parity_ptr = [&](long long s) { return lat + (size_t)(s & 1) * sdoubles; };
  cudaError_t e = cudaSuccess;
  auto save = [&](long long s, double* dst, RealState* dr) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, parity_ptr(s), sbytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dr, D.rs, rbytes, cudaMemcpyDeviceToDevice, st);
  };
  auto restore = [&](long long s, const double* src, const RealState* sr) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(parity_ptr(s), src, sbytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(D.rs, sr, rbytes, cudaMemcpyDeviceToDevice, st);
  };
  // 1. back to the initial state (the inlet data persist) and forward with checkpoints
  e = launch_init_state(L, c->precision, st);
  if (e == cudaSuccess) e = launch_lambda(L, c->precision, 0, 0, M, st);
  if (e == cudaSuccess) e = launch_fill_equilibrium_f64(L, 0, 0, M, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(inl, 0, (size_t)M * D.ny * sizeof(double), st);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(c, e, "resetting the initial state");
  }
  c->prepared = false;
  int stt = prepare(c, std::numeric_limits<double>::infinity());
  if (stt == VLBM_OK && nsteps > 0) stt = tune_design(c);
  for (long long s = 0; s < nsteps && stt == VLBM_OK && e == cudaSuccess; ++s) {
    if (s % checkpoint_every == 0) save(s, ck + (size_t)(s / checkpoint_every) * sdoubles, ckr + (s / checkpoint_every) * M);
    stt = launch_one_step(c);
  }
  save(nsteps, fin, finr);
  if (stt == VLBM_OK && e == cudaSuccess) stt = read_flags(c, -1, nullptr);
  if (stt != VLBM_OK || e != cudaSuccess) {
    release();
    return stt != VLBM_OK ? stt : cuda_fail(c, e, "forward sweep");
  }
  // 2. J and the seed; 3. reverse sweep window by window
  int cur = 0;
  double* A[2] = {adj, adj + sdoubles};
  e = adjoint_objective(L, 0, fin, w, Jm, A[cur], st);
  for (int wi = ncp - 1; wi >= 0 && e == cudaSuccess && stt == VLBM_OK; --wi) {
    const long long s0 = (long long)wi * checkpoint_every;
    const long long s1 = std::min<long long>(s0 + checkpoint_every, nsteps);
    restore(s0, ck + (size_t)wi * sdoubles, ckr + (size_t)wi * M);
    for (long long s = s0; s < s1 && e == cudaSuccess && stt == VLBM_OK; ++s) {
      save(s, tr + (size_t)(s - s0) * sdoubles, trr + (size_t)(s - s0) * M);
      if (s + 1 < s1) stt = launch_one_step(c);
    }
    for (long long s = s1 - 1; s >= s0 && e == cudaSuccess; --s) {
      e = adjoint_step(L, 0, c->r_jet, tr + (size_t)(s - s0) * sdoubles, trr + (size_t)(s - s0) * M, A[cur],
                       A[cur ^ 1], scr, iscr, inl, st);
      cur ^= 1;
    }
  }
  // 4. the initial state and the amplitudes
  if (e == cudaSuccess && stt == VLBM_OK) {
    const double* s0 = nsteps > 0 ? tr : fin;
    const RealState* r0 = nsteps > 0 ? trr : finr;
    e = adjoint_initial(L, 0, c->r_jet, s0, r0, A[cur], A[cur ^ 1], scr, inl, st);
  }
  if (e == cudaSuccess && stt == VLBM_OK && K > 0) e = adjoint_amplitudes(L, 0, c->r_jet, inl, c->d_xi, K, gd, st);
  // 5. the context is left at step nsteps of the forward run
  restore(nsteps, fin, finr);
  std::vector<double> hJ(M);
  if (e == cudaSuccess && stt == VLBM_OK && K > 0)
    e = cudaMemcpyAsync(grad_out, gd, (size_t)K * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && stt == VLBM_OK)
    e = cudaMemcpyAsync(hJ.data(), Jm, (size_t)M * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  release();
  if (stt != VLBM_OK) return stt;
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint sweep");
  if (J_out) {
    double J = 0.0;
    for (int m = 0; m < M; ++m) J += hJ[m];
    *J_out = J / M;
  }
  return VLBM_OK;
}

int vlbm_amplitudes(const vlbm_ctx* c, double* amp, int* K) {
  if (!c) return VLBM_EINVAL;
  if (K) *K = (int)c->amp.size();
  if (amp)
    for (size_t k = 0; k < c->amp.size(); ++k) amp[k] = c->amp[k];
  return VLBM_OK;
}

int vlbm_check_bounded_wait(double limit_s) {
  if (!(limit_s > 0.0) || limit_s > 10.0) return fail(nullptr, VLBM_EINVAL, "limit_s must be in (0, 10]");
  int* d = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&d), sizeof(int));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMalloc");
  int h = -1;
  e = cudaMemset(d, 0xff, sizeof(int));
  if (e == cudaSuccess) e = launch_bounded_wait_probe(d, (unsigned long long)(limit_s * 1e9), nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "bounded wait probe");
  if (h == 4) return fail(nullptr, VLBM_ETIMEOUT, "the bounded device wait gave up as designed");
  return fail(nullptr, VLBM_ECUDA, "the bounded device wait returned status " + std::to_string(h));
}

unsigned long long vlbm_kernel_launches(void) { return g_launches.load(); }

int vlbm_step_rows(const vlbm_ctx* c, int* rows) {
  if (!c || !rows) return VLBM_EINVAL;
  const int v = c->variant;
  *rows = v < 0 || c->precision == VLBM_FP64 ? 0 : mixed_march_rows(c->launch, v);
  return VLBM_OK;
}

int vlbm_step_design(const vlbm_ctx* c, int* index, const char** name, int* count) {
  if (!c) return VLBM_EINVAL;
  const int v = c->variant;
  const bool f64 = c->precision == VLBM_FP64;
  if (index) *index = v;
  if (name) *name = v < 0 ? "none" : (f64 ? f64_variant_name(v) : mixed_variant_name(v));
  if (count) *count = f64 ? f64_variants() : mixed_variants();
  return VLBM_OK;
}

const char* vlbm_last_error(const vlbm_ctx* c) { return c ? c->err.c_str() : g_thread_error.c_str(); }

void vlbm_destroy(vlbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  release_levels(c);
  dev_free(c, c->d_count);
  dev_free(c, c->d_xi);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
