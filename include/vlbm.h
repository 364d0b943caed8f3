/*
 * libvlbm: GB300 (sm_103a) implementation of the probabilistic vectorial lattice
 * Boltzmann method (VLBM) for Monte-Carlo ensembles of the Mach 2000 jet, from
 * "Computing statistical solutions of a Mach 2000 astrophysical jet".
 *
 * Conventions shared by every call:
 *   - Plain C ABI: plain pointers and sizes, no exceptions cross the boundary;
 *     every call returns a vlbm_status (VLBM_OK = 0) and, on failure, records a
 *     message readable with vlbm_last_error().
 *   - Work is enqueued on the CUDA stream given to vlbm_create and is
 *     asynchronous unless a call says otherwise.  Calls that read results back
 *     to the host (vlbm_time, vlbm_sync, vlbm_save) synchronise that stream.
 *   - "device pointer" arguments must be CUDA device (or managed) memory owned
 *     by the caller; the library never frees them.
 *   - Field layouts are realization-major and row-major with x fastest:
 *     field[r][j][i] for r = 0..count-1, j = 0..ny-1, i = 0..nx-1.
 *   - Node placement: x_i = i dx (the inlet column sits at x = 0),
 *     y_j = y_min + (j + 1/2) dx, dx = x_max / nx; cells are square.
 */
#ifndef VLBM_H
#define VLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vlbm_ctx vlbm_ctx;

/* Status codes. */
typedef enum {
  VLBM_OK = 0,
  VLBM_EINVAL = 1,        /* invalid argument (message says which) */
  VLBM_ENOMEM = 2,        /* device allocation failed */
  VLBM_ECUDA = 3,         /* a CUDA runtime call failed */
  VLBM_ENONPOSITIVE = 4,  /* a realization produced rho <= 0 or p <= 0 (sticky) */
  VLBM_ENONFINITE = 5,    /* a realization produced a non-finite value (sticky) */
  VLBM_ETIMEOUT = 6,      /* a bounded device wait gave up */
  VLBM_ESTATE = 7         /* call out of order (e.g. step before init_ensemble) */
} vlbm_status;

/* Arithmetic of the solver (fixed at creation). */
enum {
  /* Conserved variables and raw populations in FP64, the paper's arithmetic
   * in the lab frame (320 B per cell update). */
  VLBM_FP64 = 0,
  /* FP32 storage of the nodal state (rho, v1, v2, p) and of the populations'
   * non-equilibrium parts, expressed in each node's rest frame; the update is
   * evaluated in the frame moving with the node so that pressure never comes
   * from E - |m|^2 / (2 rho) (160 B per cell update). */
  VLBM_MIXED = 1
};

/* Blending-parameter rule (Sec. 2.1: theta in [0, 1] per face). */
enum {
  VLBM_LIMITER_NONE = 0,       /* theta = 0: first-order scheme */
  VLBM_LIMITER_UNLIMITED = 1,  /* theta = 1: unlimited second-order scheme (tests) */
  VLBM_LIMITER_RTHETA = 2      /* convex-split positivity + relaxed local bounds */
};

/* One grid level on [0, x_max] x [y_min, y_max]; requires
 * x_max / nx == (y_max - y_min) / ny (square cells), nx, ny >= 3. */
typedef struct {
  int nx, ny;
  double x_max, y_min, y_max;
} vlbm_grid;

/* Primitive state (rho, velocity (u, v), pressure).  Sec. 2.2: the jet is
 * {5, 800, 0, 0.4127}, the ambient medium {0.5, 0, 0, 0.4127}. */
typedef struct {
  double rho, u, v, p;
} vlbm_prim;

/* Relaxation / limiting parameters.
 *   alpha    weight of the rest population M_5 = alpha u (Eq. maxwellians5), [0, 1)
 *   kappa    safety factor on the kinetic speed, a_n = kappa 2 lambda / (1 - alpha), >= 1
 *   limiter  VLBM_LIMITER_*
 *   rlmp_rel, rlmp_abs  widening of the local density bounds:
 *            [lo - d, hi + d], d = rlmp_rel (hi - lo) + rlmp_abs
 *   eps_pos  positivity floor for rho and p (the floor is min(eps_pos, value of
 *            the first-order state)) */
typedef struct {
  double alpha, kappa;
  int limiter;
  double rlmp_rel, rlmp_abs, eps_pos;
} vlbm_relax;

/* Inlet perturbation, Eq. (karhunenExp):
 *   rho' = rho_jet [1 + sum_{k<=K} amp_k (Y_k cos(k pi yb) + Z_k sin(k pi yb)) W(yb)],
 *   yb = y / r_jet, W = cos^2(pi yb / 2), amp_k = A k^-p_decay, or amp[k-1]
 *   when use_amp != 0.  Y_k, Z_k ~ U(-1, 1) from Philox4x32-10 with
 *   key = seed and counter = (m, block, 0, 0) (K <= 16).  r_jet is also the
 *   half-width of the inlet velocity step (Sec. 2.2). */
typedef struct {
  double r_jet, A, p_decay;
  int K;
  double amp[16];
  int use_amp;
} vlbm_perturb;

/* Device memory callbacks (e.g. a framework's caching allocator).  alloc
 * returns a 256-byte aligned device pointer or NULL. */
typedef void* (*vlbm_alloc_fn)(size_t bytes, void* user);
typedef void (*vlbm_free_fn)(void* ptr, void* user);

/* Paper defaults: alpha 0, kappa 1, R-theta limiter with rlmp_rel 0.1,
 * rlmp_abs 0, eps_pos 1e-13; r_jet 0.05, A 0.1, p_decay 2, K 10. */
void vlbm_default_relax(vlbm_relax* relax);
void vlbm_default_perturb(vlbm_perturb* perturb);

/* Sec. 2.1-2.2: validates the problem (grids with finite extents and square
 * cells, gamma > 1, finite states with rho, p > 0, finite relaxation
 * parameters in range; VLBM_EINVAL otherwise) and creates a context.  Several levels (e.g. the refinement
 * ladder of Sec. 3.3) advance together in every call.  cuda_stream may be
 * NULL: the context then creates and owns a non-blocking stream (at the
 * first initialising call).  alloc/free may be NULL (cudaMalloc/cudaFree).
 * No device work is done here.  On success *out owns the context. */
int vlbm_create(const vlbm_grid* levels, int nlevels, double gamma, const vlbm_prim* jet,
                const vlbm_prim* ambient, const vlbm_relax* relax, int precision, void* cuda_stream,
                vlbm_alloc_fn alloc, vlbm_free_fn free_fn, void* alloc_user, vlbm_ctx** out);

/* Sec. 2.3, Eqs. (karhunenExp), (rho_inlet_def), (u0_def): allocates the state
 * of M realizations on every level (re-allocates if M changes), draws the inlet
 * density of realization m = 0..M-1, sets the initial condition with
 * equilibrium populations and resets t = 0, steps = 0.  perturb may be NULL
 * (defaults).  Realization m is identical for every M > m (nested prefixes).
 * Invalid arguments (M outside [1, 65535], K > 16, r_jet <= 0, non-finite A,
 * p_decay or amp[k]) return VLBM_EINVAL and leave an existing ensemble as it
 * was; a failure after that (allocation: VLBM_ENOMEM, a launch: VLBM_ECUDA)
 * leaves the context without an ensemble, so that stepping calls return
 * VLBM_ESTATE until an initialisation succeeds. */
int vlbm_init_ensemble(vlbm_ctx* ctx, uint64_t seed, int M, const vlbm_perturb* perturb);

/* As vlbm_init_ensemble, for the block of realizations m_begin..m_begin+M-1
 * of the same nested sequence (Sec. 3.1: realization m is fixed by the seed and
 * m alone), so that independent processes can each own a block of one ensemble.
 * Local index r of the context holds global realization m_begin + r. */
int vlbm_init_ensemble_block(vlbm_ctx* ctx, uint64_t seed, int m_begin, int M, const vlbm_perturb* perturb);

/* As vlbm_init_ensemble, with the random coefficients of Eq. (karhunenExp)
 * given instead of drawn: realization r = 0..M-1 uses Y_k = xi[r*2K + k - 1]
 * and Z_k = xi[r*2K + K + k - 1], k = 1..K (K = perturb->K), each the paper's
 * U(-1, 1) draw (any values in [-1, 1]: quasi-random points, stratified
 * samples, another code's draws).  Layout: M x 2K doubles, row-major.  xi may
 * be host or device memory.  Host values are checked to lie in [-1, 1]
 * (VLBM_EINVAL otherwise); device values are not checked.  The M*2K doubles
 * are copied on the context's stream: pageable host memory before the call
 * returns, pinned or device memory asynchronously (keep it valid until the
 * stream has passed the call).  The coefficients equal to a seed's Philox
 * draws reproduce vlbm_init_ensemble with that seed bit for bit. */
int vlbm_init_ensemble_samples(vlbm_ctx* ctx, const double* xi, int M, const vlbm_perturb* perturb);

/* Sec. 2.1, Eqs. (vlbm1)-(vlbm5), with a_n re-evaluated every step
 * (Sec. 2.3): advances every realization on every level by n steps. */
int vlbm_step(vlbm_ctx* ctx, int n);

/* Advances every realization until its own time reaches t exactly; the last
 * step of each lands on t (a_n <- max(a_n, dx / (t - t_n))).  Realizations
 * that finish early stop stepping.  Synchronises the stream. */
int vlbm_advance_to(vlbm_ctx* ctx, double t);

/* Eq. (eos): writes rho, velocity (u, v) and p of realizations m0..m0+count-1
 * of one level into caller device buffers laid out [count][ny][nx] (FP64).
 * Any output pointer may be NULL. */
int vlbm_moments(vlbm_ctx* ctx, int level, int m0, int count, double* rho, double* u, double* v,
                 double* p);

/* Density only, [count][ny][nx], FP32 (as_f32 != 0) or FP64; the input layout
 * of stats_w1_mean_std. */
int vlbm_density(vlbm_ctx* ctx, int level, int m0, int count, void* rho, int as_f32);

/* Host copies of the per-realization time and step count of one level
 * (arrays of length M; either may be NULL).  Synchronises the stream and
 * returns the first sticky error flag of the level, if any. */
int vlbm_time(vlbm_ctx* ctx, int level, double* t_host, long long* steps_host);

/* Waits for the stream and reports sticky per-realization flags:
 * VLBM_ENONPOSITIVE / VLBM_ENONFINITE if any realization raised one. */
int vlbm_sync(vlbm_ctx* ctx);

/* Full state of realizations m0..m0+count-1 as FP64 device arrays:
 * u [count][4][ny][nx] conserved (rho, rho v1, rho v2, E) and pops
 * [count][16][ny][nx] (population k = 1..4 at rows 4(k-1)..4(k-1)+3).
 * In VLBM_MIXED the populations are rebuilt from the stored non-equilibrium
 * parts.  pops may be NULL. */
int vlbm_get_state(vlbm_ctx* ctx, int level, int m0, int count, double* u, double* pops);

/* Overwrites the state of realizations m0..m0+count-1 (same layouts as
 * vlbm_get_state, device pointers), resets their t and step count to 0 and
 * re-evaluates their kinetic speed.  The inlet column keeps its Dirichlet
 * datum from vlbm_init_ensemble at the next step. */
int vlbm_set_state(vlbm_ctx* ctx, int level, int m0, int count, const double* u, const double* pops);

/* Sec. 3.2 and 3.4, Eqs. (mean), (std), (w1disc): per-cell statistics between
 * ensemble a [M][nya][nxa] and ensemble b [M][nyb][nxb] (device pointers; FP32
 * when *_is_f32 != 0, else FP64).  When nxb = r nxa and nyb = r nya (r >= 1)
 * each realization of b is first block-averaged onto a's grid.  Outputs
 * (device, FP64, [nya][nxa], any may be NULL): mean and population std of a and
 * of the restricted b, and the one-point W1 = (1/M) sum_m |a_(m) - b_(m)| over
 * the ascending order statistics.  1 <= M <= 4096, nxa nya < 2^31; a b that
 * is not an integer refinement of a (same factor in x and y) is VLBM_EINVAL.
 * Asynchronous on cuda_stream (may be NULL). */
int stats_w1_mean_std(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b,
                      int b_is_f32, int nxb, int nyb, int M, double* mean_a, double* std_a,
                      double* mean_b, double* std_b, double* w1, void* cuda_stream);

/* Sec. 3.4, Eq. (w2): the two-point Wasserstein distance W_{1,2} between
 * ensemble a [M][nya][nxa] and ensemble b [M][nyb][nxb] (device pointers;
 * FP32 when *_is_f32 != 0, else FP64), b block-restricted onto a's grid
 * (nxb = r nxa, nyb = r nya).  The grid is subsampled to npd x npd points,
 * x_k = the centre cell (((2 kx + 1) nxa) / (2 npd), ((2 ky + 1) nya) / (2 npd))
 * of each of npd equal strips per direction, k = ky npd + kx; for every
 * ordered pair (k, k'), the first Wasserstein distance on R^2 (Euclidean
 * cost) between the empirical joint laws of (rho(x_k), rho(x_k')) of the two
 * ensembles is computed exactly (optimal assignment of the M points, FP64).
 * *w12 (device) receives the mean over the P = npd^4 pairs; pairs (device
 * [P], pair k npd^2 + k', may be NULL: scratch then comes from the
 * stream-ordered allocator) the per-pair values.  1 <= M <= 2048,
 * 1 <= npd <= min(nxa, nya, 215).  Asynchronous on cuda_stream (may be NULL);
 * results are reproducible bit for bit. */
int stats_w1_two_point(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32, int nxb,
                       int nyb, int M, int npd, double* w12, double* pairs, void* cuda_stream);

/* Sec. 3.3: the conservative restriction operator R, block averaging of each
 * of the M fields ens [M][ny][nx] (device; FP32 when is_f32 != 0, else FP64)
 * onto the coarse grid [M][ny/r][nx/r]: coarse cell (I, J) is the mean of
 * fine cells (r I .. r I + r - 1, r J .. r J + r - 1), summed in FP64 (fine
 * rows outer, columns inner, as in stats_w1_mean_std).  out (device) is FP32
 * when out_is_f32 != 0, else FP64, and must not overlap ens.  r must divide
 * nx and ny; 1 <= M <= 65535.  Asynchronous on cuda_stream (may be NULL).
 * Comparing several levels on one common grid (the paper's protocol) is
 * restricting each level onto it, then calling the statistics with r = 1. */
int stats_restrict(const void* ens, int is_f32, int nx, int ny, int M, int r, void* out, int out_is_f32,
                   void* cuda_stream);

/* Sec. 3.3-3.4, Eqs. (mean), (std), (w1disc), (strongError): the error
 * functionals between ensemble a [M][nya][nxa] and ensemble b [M][nyb][nxb]
 * (b block-restricted onto a's grid as in stats_w1_mean_std), written to the
 * device array out[4] = {E_mean, E_std, W_11, E_strong}: cell averages of
 * |mean_a - mean_b|, |std_a - std_b| and of the one-point W1, and the
 * realization average of ||a_m - R b_m||_1 / ||R b_m||_1.  Every sum runs in a
 * fixed order (the result is reproducible bit for bit).  Scratch memory
 * (3 * 512 + 128 M doubles) comes from the stream-ordered allocator
 * (cudaMallocAsync) and is released on the stream.  1 <= M <= 4096.  Asynchronous. */
int stats_error_functionals(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32,
                            int nxb, int nyb, int M, double* out, void* cuda_stream);

/* stats_error_functionals without any device allocation.  Some callers
 * cannot allocate device memory once they are running: a host that hands the
 * whole GPU to its own pool allocator and forbids other allocations, or a
 * real-time loop where an allocation's latency or failure is not acceptable.
 * This call takes its scratch from a fixed device array compiled into the
 * library (4.2 MB on every GPU that loads it, held until the process exits)
 * and never calls cudaMalloc, cudaFree or any allocating routine; the caller
 * still passes the ensembles and the output array.  M must be <= 4096
 * (VLBM_EINVAL beyond).  The first call on a device looks up the array's
 * device address: make it before any stream capture on that device (a first
 * call on a capturing stream returns VLBM_ESTATE and enqueues nothing).  All
 * calls share the array: calls that overlap on the GPU race; consecutive
 * calls do not interfere (each overwrites every partial sum it reads).
 * Results are identical to stats_error_functionals.  The paper has no
 * counterpart: it is an interface for such callers.  Asynchronous. */
int stats_error_functionals_noalloc(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b,
                                    int b_is_f32, int nxb, int nyb, int M, double* out, void* cuda_stream);

/* Sec. 4.3, Eq. (empcdf): per-cell empirical quantiles
 * p_alpha = inf{xi : F(xi) >= alpha} (the ceil(alpha M)-th smallest sample) of
 * ensemble [M][ny][nx] (device; FP32 when is_f32 != 0) for the probabilities
 * probs[0..nprob-1] (host array, each in (0, 1], nprob <= 16); out is a device
 * array [nprob][ny][nx] (FP64).  1 <= M <= 4096.  Asynchronous. */
int stats_quantiles(const void* ens, int is_f32, int nx, int ny, int M, const double* probs, int nprob, double* out,
                    void* cuda_stream);

/* Sec. 4.4, Eq. (hist): per-cell histogram density of ensemble [M][ny][nx]
 * on the bins [edges[j], edges[j+1]), j = 0..nbins-1 (edges: device array of
 * nbins + 1 increasing values), out[j][y][x] = count / (M (edges[j+1] -
 * edges[j])); samples outside [edges[0], edges[nbins]) are not counted.
 * nbins <= 8192.  Asynchronous. */
int stats_histogram(const void* ens, int is_f32, int nx, int ny, int M, const double* edges, int nbins, double* out,
                    void* cuda_stream);

/* Checkpoint of the whole context state (every level and realization, times,
 * step counts, kinetic-speed bookkeeping) to host memory.  With host_buf NULL,
 * *bytes receives the size needed.  Synchronises the stream.  Restoring with
 * vlbm_load into a context created with the same levels, precision and M
 * resumes bit-identically.  vlbm_load needs an initialised context (its
 * device memory is reused) and returns VLBM_EINVAL when the header (format,
 * precision, level count, M) or the size does not match.  The KL uniforms and
 * amplitudes that vlbm_grad_amplitudes differentiates with respect to are not
 * part of the checkpoint: they stay those of the context's last
 * vlbm_init_ensemble* call.  vlbm_save returns the sticky realization flags
 * (VLBM_ENONPOSITIVE ...) after a complete save. */
int vlbm_save(vlbm_ctx* ctx, void* host_buf, size_t* bytes);
int vlbm_load(vlbm_ctx* ctx, const void* host_buf, size_t bytes);

/* Message of the last failing call on ctx (or of the last failing call in this
 * thread when ctx is NULL).  Never NULL. */
const char* vlbm_last_error(const vlbm_ctx* ctx);

/* Number of kernel launches this library has enqueued in this process so far
 * (graph replays count every kernel node).  Instrumentation for benchmarks. */
unsigned long long vlbm_kernel_launches(void);

/* Gradient of an ensemble observable with respect to the per-mode amplitudes
 * a_1..a_K of the KL inlet perturbation (Sec. 2.3, Eq. (karhunenExp)): the
 * hand-written discrete adjoint of the FP64 step (Eqs. (vlbm1)-(vlbm5), the
 * R-theta limiter, the boundaries of Sec. 2.2 and the kinetic speed of
 * Sec. 2.1).  From the initial state of the context's last initialisation
 * (re-created here), the context advances nsteps fixed FP64 steps, keeping a
 * checkpoint every checkpoint_every steps; then the reverse sweep restores
 * each checkpoint, recomputes the states of its window and runs the adjoint
 * step backwards through them.  The observable is
 *   J = (1/M) sum_m sum_{i,j} w[j][i] rho_m(i, j, t_nsteps),
 * w a device array [ny][nx] (the axial ensemble-mean density is w = 1/2 on
 * the two rows next to y = 0, times the weight of each column).  On return
 * grad_out[k - 1] = dJ/da_k (host, K doubles, K of the last initialisation)
 * and, if J_out is not NULL, *J_out = J; the context is left at step nsteps.
 * The discrete map is piecewise smooth: the argmax of lambda, the limiter's
 * minima and branches are differentiated on the branch the forward step
 * takes.  Realizations of the jet diverge pathwise (Sec. 4: the strong error
 * does not converge), so such a gradient describes the ensemble only over
 * windows shorter than the divergence time.  Needs an FP64 single-level
 * context; device memory for ceil(nsteps / checkpoint_every) + checkpoint_every
 * + 4 states plus ~90 FP64 planes per realization comes from the context's
 * allocator and is released before return.  Synchronises the stream.
 * Returns VLBM_EINVAL (wrong context or arguments), VLBM_ENOMEM, VLBM_ECUDA,
 * or the positivity / finiteness status of the forward run.  No counterpart
 * in the paper, which computes no gradients. */
int vlbm_grad_amplitudes(vlbm_ctx* ctx, int nsteps, int checkpoint_every, const double* w, double* J_out,
                         double* grad_out);

/* The per-mode amplitudes of the context's last initialisation: *K (may be
 * NULL) receives their number, amp (host, may be NULL) the values
 * (A k^-p unless overridden).  VLBM_EINVAL for a NULL ctx. */
int vlbm_amplitudes(const vlbm_ctx* ctx, double* amp, int* K);

/* The launch design the mixed-precision step kernel runs with in ctx: its
 * index, its name (static storage) and the number of designs.  The designs
 * (tile shapes, persistent CTAs, warps marching up column strips) compute
 * bit-identical results; the context picks the fastest by timing each on its
 * first step, unless the environment variable VLBM_MIXED_VARIANT holds a valid
 * index; *index is -1 (and *name "none") before the first step.  An FP64
 * context likewise picks among two designs (0: 32 x 8 tiles, 1: warps
 * marching up 28-column strips; VLBM_F64_VARIANT forces one), which compute
 * identical results.  Any output pointer may be NULL.  No counterpart in the
 * paper, whose update has a single implementation.  Returns VLBM_EINVAL for a
 * NULL ctx. */
int vlbm_step_design(const vlbm_ctx* ctx, int* index, const char** name, int* count);

/* Rows per warp of the mixed warp-march design in use (*rows = 0 for the
 * other designs, for FP64 contexts and before the first step).  A march splits each level into strips
 * of columns, one warp per strip and chunk of rows; the split changes no
 * result.  On a small launch (a single small grid) the context times several
 * row counts on its first step and keeps the fastest; the environment
 * variable VLBM_MARCH_ROWS (> 0) forces the count of a mixed march.  No
 * counterpart in the paper.  Returns VLBM_EINVAL for a NULL ctx or rows. */
int vlbm_step_rows(const vlbm_ctx* ctx, int* rows);

/* Failure-detection check of the device waits: runs on the current device
 * one mbarrier wait that nothing completes, bounded by limit_s seconds
 * (0 < limit_s <= 10) as every wait of the step kernels is bounded, and
 * reports how it ended.  Returns VLBM_ETIMEOUT when the bound ended the wait
 * (the designed outcome: the kernel returned, nothing is in flight, the
 * context stays usable), VLBM_ECUDA otherwise, VLBM_EINVAL for a bad limit.
 * Synchronous.  No counterpart in the paper. */
int vlbm_check_bounded_wait(double limit_s);

/* Frees the context and everything it allocated.  Accepts NULL. */
void vlbm_destroy(vlbm_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VLBM_H */
