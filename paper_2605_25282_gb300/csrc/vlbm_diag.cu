// Diagnostics of the ensemble statistics (Sec. 3.3-3.4 error functionals,
// Sec. 4.3 quantiles, Sec. 4.4 histograms).
//
//  - functional_cells_kernel: a fixed grid of kFuncCtas CTAs walks the coarse
//    cells (cell = blockIdx.x + k kFuncCtas); per cell it gathers the M samples
//    of a and the M restricted samples of b, forms mean and population std of
//    both and the one-point W1 from a bitonic sort, and accumulates
//    |mean_a - mean_b|, |std_a - std_b| and W1 in cell order.  Each CTA writes
//    one partial triple.
//  - functional_strong_kernel: CTA (chunk, m) sums |a_m - R b_m| and |R b_m|
//    over its chunk of cells.
//  - functional_final_kernel: one CTA adds the partials in a fixed order:
//    E_mean, E_std, W_11 = sums / cells (Eqs. mean, std, w1disc);
//    E_strong = (1/M) sum_m ||a_m - R b_m||_1 / ||R b_m||_1 (Eq. strongError).
// Every sum runs in a fixed order, so the result does not depend on scheduling.
#include <cmath>
#include <mutex>

#include "vlbm_internal.cuh"

namespace vlbm {

constexpr int kFuncCtas = 512;   // CTAs of the cell pass (one partial triple each)
constexpr int kStrongChunks = 64;  // cell chunks per realization in the strong pass
constexpr int kDiagThreads = 256;

namespace {

__device__ __forceinline__ double load_sample(const void* p, int is_f32, size_t idx) {
  return is_f32 ? (double)reinterpret_cast<const float*>(p)[idx] : reinterpret_cast<const double*>(p)[idx];
}

__device__ __forceinline__ double restricted(const void* b, int b_f32, size_t nb, int nxb, int r, int m, int I, int J) {
  double s = 0.0;
  for (int aa = 0; aa < r; ++aa)
    for (int bb = 0; bb < r; ++bb)
      s += load_sample(b, b_f32, (size_t)m * nb + (size_t)(r * J + aa) * nxb + (size_t)(r * I + bb));
  return s / (double)(r * r);
}

__device__ void bitonic(double* x, int P) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
        const int lo = 2 * j * (t / j) + (t % j), hi = lo + j;
        const bool up = (lo & k) == 0;
        const double a = x[lo], b = x[hi];
        if ((a > b) == up) {
          x[lo] = b;
          x[hi] = a;
        }
      }
      __syncthreads();
    }
}

// Sum over the block in a fixed order (warp shuffle tree, then warps in order).
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kDiagThreads) functional_cells_kernel(const void* __restrict__ a, int a_f32, int nxa,
                                                                        int nya, const void* __restrict__ b, int b_f32,
                                                                        int nxb, int r, int M, int P,
                                                                        double* __restrict__ partial) {
  extern __shared__ double sm[];
  double* xa = sm;
  double* xb = sm + P;
  __shared__ double red[kDiagThreads / 32];
  const size_t na = (size_t)nxa * nya, nb = na * (size_t)r * r;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double acc_m = 0.0, acc_s = 0.0, acc_w = 0.0;
  for (size_t cell = blockIdx.x; cell < na; cell += gridDim.x) {
    const int I = (int)(cell % nxa), J = (int)(cell / nxa);
    for (int m = threadIdx.x; m < P; m += blockDim.x) {
      if (m < M) {
        xa[m] = load_sample(a, a_f32, (size_t)m * na + cell);
        xb[m] = restricted(b, b_f32, nb, nxb, r, m, I, J);
      } else {
        xa[m] = inf;
        xb[m] = inf;
      }
    }
    __syncthreads();
    double sa = 0.0, sb = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      sa += xa[m];
      sb += xb[m];
    }
    const double ma = block_sum(sa, red) / M, mb = block_sum(sb, red) / M;
    double va = 0.0, vb = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      const double da = xa[m] - ma, db = xb[m] - mb;
      va += da * da;
      vb += db * db;
    }
    const double sda = sqrt(block_sum(va, red) / M), sdb = sqrt(block_sum(vb, red) / M);
    __syncthreads();
    bitonic(xa, P);
    bitonic(xb, P);
    double w = 0.0;
    for (int m = threadIdx.x; m < M; m += blockDim.x) w += fabs(xa[m] - xb[m]);
    const double W = block_sum(w, red) / M;
    acc_m += fabs(ma - mb);
    acc_s += fabs(sda - sdb);
    acc_w += W;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x + 0] = acc_m;
    partial[3 * blockIdx.x + 1] = acc_s;
    partial[3 * blockIdx.x + 2] = acc_w;
  }
}

__global__ void __launch_bounds__(kDiagThreads) functional_strong_kernel(const void* __restrict__ a, int a_f32,
                                                                         int nxa, int nya, const void* __restrict__ b,
                                                                         int b_f32, int nxb, int r,
                                                                         double* __restrict__ partial2) {
  __shared__ double red[kDiagThreads / 32];
  const int chunk = blockIdx.x, m = blockIdx.y;
  const size_t na = (size_t)nxa * nya, nb = na * (size_t)r * r;
  const size_t c0 = na * chunk / gridDim.x, c1 = na * (chunk + 1) / gridDim.x;
  double d = 0.0, n = 0.0;
  for (size_t cell = c0 + threadIdx.x; cell < c1; cell += blockDim.x) {
    const int I = (int)(cell % nxa), J = (int)(cell / nxa);
    const double rb = restricted(b, b_f32, nb, nxb, r, m, I, J);
    d += fabs(load_sample(a, a_f32, (size_t)m * na + cell) - rb);
    n += fabs(rb);
  }
  const double D = block_sum(d, red), N = block_sum(n, red);
  if (threadIdx.x == 0) {
    partial2[((size_t)m * gridDim.x + chunk) * 2 + 0] = D;
    partial2[((size_t)m * gridDim.x + chunk) * 2 + 1] = N;
  }
}

__global__ void __launch_bounds__(kDiagThreads) functional_final_kernel(const double* __restrict__ partial,
                                                                        const double* __restrict__ partial2,
                                                                        size_t cells, int M, double* out) {
  __shared__ double red[kDiagThreads / 32];
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < kFuncCtas; i += blockDim.x)
    for (int q = 0; q < 3; ++q) s[q] += partial[3 * i + q];
  double tot[3];
  for (int q = 0; q < 3; ++q) tot[q] = block_sum(s[q], red);
  double rat = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    double D = 0.0, N = 0.0;
    for (int c = 0; c < kStrongChunks; ++c) {
      D += partial2[((size_t)m * kStrongChunks + c) * 2 + 0];
      N += partial2[((size_t)m * kStrongChunks + c) * 2 + 1];
    }
    rat += D / N;
  }
  const double R = block_sum(rat, red);
  if (threadIdx.x == 0) {
    out[0] = tot[0] / (double)cells;
    out[1] = tot[1] / (double)cells;
    out[2] = tot[2] / (double)cells;
    out[3] = R / M;
  }
}

// Per-cell empirical quantiles: sort the M samples, pick the k-th smallest.
struct QuantileIdx {
  int n;
  int k[16];
};

__global__ void __launch_bounds__(kDiagThreads) quantile_kernel(const void* __restrict__ s, int f32, size_t cells, int M,
                                                                int P, QuantileIdx q, double* __restrict__ out) {
  extern __shared__ double sm[];
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  for (size_t cell = blockIdx.x; cell < cells; cell += gridDim.x) {
    for (int m = threadIdx.x; m < P; m += blockDim.x) sm[m] = m < M ? load_sample(s, f32, (size_t)m * cells + cell) : inf;
    __syncthreads();
    bitonic(sm, P);
    for (int i = threadIdx.x; i < q.n; i += blockDim.x) out[(size_t)i * cells + cell] = sm[q.k[i]];
    __syncthreads();
  }
}

// Per-cell histogram density on the bins [edges[j], edges[j+1]).
__global__ void __launch_bounds__(kDiagThreads) histogram_kernel(const void* __restrict__ s, int f32, size_t cells, int M,
                                                                 const double* __restrict__ edges, int nbins,
                                                                 double* __restrict__ out) {
  extern __shared__ unsigned int cnt[];
  for (size_t cell = blockIdx.x; cell < cells; cell += gridDim.x) {
    for (int j = threadIdx.x; j < nbins; j += blockDim.x) cnt[j] = 0u;
    __syncthreads();
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
      const double x = load_sample(s, f32, (size_t)m * cells + cell);
      if (!(x >= edges[0]) || !(x < edges[nbins])) continue;
      int lo = 0, hi = nbins;  // edges[lo] <= x < edges[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (x >= edges[mid])
          lo = mid;
        else
          hi = mid;
      }
      atomicAdd(&cnt[lo], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nbins; j += blockDim.x)
      out[(size_t)j * cells + cell] = (double)cnt[j] / ((double)M * (edges[j + 1] - edges[j]));
    __syncthreads();
  }
}

int pow2_at_least(int M) {
  int P = 1;
  while (P < M) P <<= 1;
  return P;
}

}  // namespace

size_t functional_scratch_doubles(int M) { return (size_t)3 * kFuncCtas + (size_t)2 * kStrongChunks * M; }

// ---- allocation-free variant -------------------------------------------------
// Scratch of stats_error_functionals_noalloc: a file-scope device array that
// every GPU loading the library holds until the process exits (4.2 MB, enough
// for M <= kNoAllocMaxM).  Every call overwrites all the partial sums it later
// reads, so nothing carries over from the previous call; calls that overlap on
// the GPU share the array and race.
constexpr int kNoAllocMaxM = 4096;
constexpr size_t kNoAllocDoubles = (size_t)3 * kFuncCtas + (size_t)2 * kStrongChunks * kNoAllocMaxM;
static __device__ __align__(256) double g_functional_scratch[kNoAllocDoubles];

int noalloc_max_m() { return kNoAllocMaxM; }

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.  With lookup false
// an address not cached yet is not looked up (cudaErrorStreamCaptureUnsupported):
// the lookup may load the module, which a stream capture does not allow.
cudaError_t noalloc_scratch(double** out, bool lookup) {
  static std::mutex mu;
  static double* cached[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!cached[dev]) {
    if (!lookup) return cudaErrorStreamCaptureUnsupported;
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_functional_scratch);
    if (e != cudaSuccess) return e;
    cached[dev] = static_cast<double*>(p);
  }
  *out = cached[dev];
  return cudaSuccess;
}

int functional_check(int nxa, int nya, int nxb, int nyb, int M, const char** why) {
  if (nxa < 1 || nya < 1 || M < 1 || M > 4096) {
    *why = "need nxa, nya >= 1 and 1 <= M <= 4096";
    return VLBM_EINVAL;
  }
  if (nxb < nxa || nyb < nya || nxb % nxa != 0 || nyb % nya != 0 || nxb / nxa != nyb / nya) {
    *why = "ensemble b must be an integer refinement (same factor in x and y) of ensemble a";
    return VLBM_EINVAL;
  }
  return VLBM_OK;
}

cudaError_t functional_launch(const void* a, int a_f32, int nxa, int nya, const void* b, int b_f32, int nxb, int M,
                              double* scratch, double* out, cudaStream_t s) {
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = once_per_device(configured, [] {
    return cudaFuncSetAttribute(functional_cells_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                2 * 4096 * (int)sizeof(double));
  });
  if (e != cudaSuccess) return e;
  const int r = nxb / nxa, P = pow2_at_least(M);
  double* partial = scratch;
  double* partial2 = scratch + 3 * kFuncCtas;
  functional_cells_kernel<<<kFuncCtas, kDiagThreads, 2 * P * sizeof(double), s>>>(a, a_f32, nxa, nya, b, b_f32, nxb, r,
                                                                                M, P, partial);
  functional_strong_kernel<<<dim3(kStrongChunks, M), kDiagThreads, 0, s>>>(a, a_f32, nxa, nya, b, b_f32, nxb, r,
                                                                           partial2);
  functional_final_kernel<<<1, kDiagThreads, 0, s>>>(partial, partial2, (size_t)nxa * nya, M, out);
  add_launches(3);
  return cudaGetLastError();
}

int quantile_launch(const void* ens, int f32, int nx, int ny, int M, const double* probs, int nprob, double* out,
                    cudaStream_t s, const char** why) {
  if (!ens || !out || !probs || nx < 1 || ny < 1 || M < 1 || M > 4096 || nprob < 1 || nprob > 16) {
    *why = "need non-NULL pointers, 1 <= M <= 4096 and 1 <= nprob <= 16";
    return VLBM_EINVAL;
  }
  QuantileIdx q{};
  q.n = nprob;
  for (int i = 0; i < nprob; ++i) {
    if (!(probs[i] > 0.0 && probs[i] <= 1.0)) {
      *why = "quantile probabilities must lie in (0, 1]";
      return VLBM_EINVAL;
    }
    int k = (int)std::ceil(probs[i] * (double)M);  // p_alpha = the ceil(alpha M)-th smallest
    k = k < 1 ? 1 : (k > M ? M : k);
    q.k[i] = k - 1;
  }
  static std::atomic<unsigned long long> configured{0};
  if (once_per_device(configured, [] {
        return cudaFuncSetAttribute(quantile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * 8);
      }) != cudaSuccess) {
    *why = "cudaFuncSetAttribute failed";
    return VLBM_ECUDA;
  }
  const int P = pow2_at_least(M);
  const size_t cells = (size_t)nx * ny;
  const int grid = (int)(cells < 4096 ? cells : 4096);
  quantile_kernel<<<grid, kDiagThreads, P * sizeof(double), s>>>(ens, f32, cells, M, P, q, out);
  add_launches(1);
  if (cudaGetLastError() != cudaSuccess) {
    *why = "quantile kernel launch failed";
    return VLBM_ECUDA;
  }
  return VLBM_OK;
}

int histogram_launch(const void* ens, int f32, int nx, int ny, int M, const double* edges, int nbins, double* out,
                     cudaStream_t s, const char** why) {
  if (!ens || !out || !edges || nx < 1 || ny < 1 || M < 1 || nbins < 1 || nbins > 8192) {
    *why = "need non-NULL pointers, M >= 1 and 1 <= nbins <= 8192";
    return VLBM_EINVAL;
  }
  const size_t cells = (size_t)nx * ny;
  const int grid = (int)(cells < 4096 ? cells : 4096);
  histogram_kernel<<<grid, kDiagThreads, nbins * sizeof(unsigned), s>>>(ens, f32, cells, M, edges, nbins, out);
  add_launches(1);
  if (cudaGetLastError() != cudaSuccess) {
    *why = "histogram kernel launch failed";
    return VLBM_ECUDA;
  }
  return VLBM_OK;
}

}  // namespace vlbm
