// Per-cell ensemble statistics between two grid levels (Sec. 3.2 restriction,
// Sec. 3.4 Eqs. (mean), (std), (w1disc)).
//
// One CTA per coarse cell.  The M samples of ensemble a and the M restricted
// samples of ensemble b (each realization of b block-averaged over its r x r
// fine cells onto the coarse cell) are gathered into shared memory, padded to
// a power of two with +inf, bitonic-sorted (as order-preserving integer keys),
// and reduced in FP64:
//   mean = sum / M, std = sqrt(sum (x - mean)^2 / M)  (population variance),
//   W1   = sum_m |a_(m) - b_(m)| / M  over the ascending order statistics.
// The gather is strided by the field size; consecutive CTAs are neighbouring
// cells, so the rest of each 32-byte sector is reused from L2.
// restrict_kernel applies the restriction alone (one thread per coarse cell
// and realization, the same summation order), for comparisons of several
// levels on one common grid.
#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kStatThreads = 256;

__device__ __forceinline__ double load_sample(const void* p, int is_f32, size_t idx) {
  return is_f32 ? (double)reinterpret_cast<const float*>(p)[idx] : reinterpret_cast<const double*>(p)[idx];
}

// Order-preserving 64-bit keys of doubles: key(a) < key(b) as unsigned
// integers exactly when a < b (a non-negative double's bits with the sign bit
// set; a negative one's bits inverted).  Sorting the keys on the integer ALU
// sorts the values: GB300 runs FP64 compares on its FP64 pipe (2 operations
// per SM and clock), integer compares at 64 lanes per SM and clock.
__device__ __forceinline__ unsigned long long order_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// Sorts x[0..P) and y[0..P) ascending together (bitonic network, P a power
// of two; each stage's P/2 compare-exchanges shared by the threads, thread t
// taking t, t + blockDim.x, ...).  In a stage of distance j <= 32 the
// exchanges of a warp stay inside the 64-element blocks of its own indices,
// so two such stages in a row need only the warp's own ordering; a CTA
// barrier separates a stage from the next one only when the next reaches
// further (j > 32), and the sort ends with one.
__device__ void bitonic_sort2(unsigned long long* x, unsigned long long* y, int P) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
        const int lo = 2 * j * (t / j) + (t % j);
        const int hi = lo + j;
        const bool up = (lo & k) == 0;
        const unsigned long long a = x[lo], b = x[hi];
        if ((a > b) == up) {
          x[lo] = b;
          x[hi] = a;
        }
        const unsigned long long c = y[lo], d = y[hi];
        if ((c > d) == up) {
          y[lo] = d;
          y[hi] = c;
        }
      }
      const int next = j > 1 ? j >> 1 : k;  // the next stage's distance
      if (next > 32)
        __syncthreads();
      else
        __syncwarp();
    }
  }
  __syncthreads();
}

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

__global__ void __launch_bounds__(kStatThreads) stats_kernel(const void* __restrict__ ens_a, int a_f32, int nxa,
                                                             int nya, const void* __restrict__ ens_b, int b_f32,
                                                             int nxb, int r, int M, int P, double* mean_a,
                                                             double* std_a, double* mean_b, double* std_b,
                                                             double* w1) {
  extern __shared__ double sm[];
  double* xa = sm;
  double* xb = sm + P;
  __shared__ double red[kStatThreads / 32];
  const int cell = blockIdx.x;
  const int I = cell % nxa, J = cell / nxa;
  const size_t na = (size_t)nxa * nya;
  const size_t nb = na * (size_t)r * r;
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  // the block mean: a power-of-two block size divides exactly by multiplying
  const int rr = r * r;
  const bool rr_pow2 = (rr & (rr - 1)) == 0;
  const double inv_rr = 1.0 / (double)rr;
  for (int m = threadIdx.x; m < P; m += blockDim.x) {
    if (m < M) {
      xa[m] = load_sample(ens_a, a_f32, (size_t)m * na + cell);
      double s = 0.0;
      for (int aa = 0; aa < r; ++aa)
        for (int bb = 0; bb < r; ++bb)
          s += load_sample(ens_b, b_f32, (size_t)m * nb + (size_t)(r * J + aa) * nxb + (size_t)(r * I + bb));
      xb[m] = rr_pow2 ? s * inv_rr : s / (double)rr;
    } else {
      xa[m] = inf;
      xb[m] = inf;
    }
  }
  __syncthreads();
  // moments (before sorting; order-independent up to round-off)
  double sa = 0.0, sb = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    sa += xa[m];
    sb += xb[m];
  }
  const double ma = block_sum(sa, red) / (double)M;
  const double mb = block_sum(sb, red) / (double)M;
  double va = 0.0, vb = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const double da = xa[m] - ma, db = xb[m] - mb;
    va += da * da;
    vb += db * db;
  }
  const double vA = block_sum(va, red) / (double)M;
  const double vB = block_sum(vb, red) / (double)M;
  // sort the samples' order keys in place (each thread converts its own)
  unsigned long long* ka = reinterpret_cast<unsigned long long*>(xa);
  unsigned long long* kb = reinterpret_cast<unsigned long long*>(xb);
  for (int m = threadIdx.x; m < P; m += blockDim.x) {
    ka[m] = order_key(xa[m]);
    kb[m] = order_key(xb[m]);
  }
  __syncthreads();
  bitonic_sort2(ka, kb, P);
  double w = 0.0;
  for (int m = threadIdx.x; m < M; m += blockDim.x) w += fabs(key_value(ka[m]) - key_value(kb[m]));
  const double W = block_sum(w, red) / (double)M;
  if (threadIdx.x == 0) {
    if (mean_a) mean_a[cell] = ma;
    if (std_a) std_a[cell] = sqrt(vA);
    if (mean_b) mean_b[cell] = mb;
    if (std_b) std_b[cell] = sqrt(vB);
    if (w1) w1[cell] = W;
  }
}

}  // namespace

int stats_launch(const void* ens_a, int a_is_f32, int nxa, int nya, const void* ens_b, int b_is_f32, int nxb,
                 int nyb, int M, double* mean_a, double* std_a, double* mean_b, double* std_b, double* w1,
                 cudaStream_t s, const char** why) {
  if (!ens_a || !ens_b) {
    *why = "ensemble pointers must be non-NULL";
    return VLBM_EINVAL;
  }
  if (nxa < 1 || nya < 1 || M < 1 || M > 4096) {
    *why = "need nxa, nya >= 1 and 1 <= M <= 4096";
    return VLBM_EINVAL;
  }
  if ((long long)nxa * nya > 0x7fffffffLL) {
    *why = "the coarse grid has more than 2^31 - 1 cells";
    return VLBM_EINVAL;
  }
  if (nxb < nxa || nyb < nya || nxb % nxa != 0 || nyb % nya != 0 || nxb / nxa != nyb / nya) {
    *why = "ensemble b must be an integer refinement (same factor in x and y) of ensemble a";
    return VLBM_EINVAL;
  }
  const int r = nxb / nxa;
  int P = 1;
  while (P < M) P <<= 1;
  const size_t smem = 2 * (size_t)P * sizeof(double);
  static std::atomic<unsigned long long> configured{0};
  if (once_per_device(configured, [] {
        return cudaFuncSetAttribute(stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 4096 * 8);
      }) != cudaSuccess) {
    *why = "cudaFuncSetAttribute failed for the statistics kernel";
    return VLBM_ECUDA;
  }
  stats_kernel<<<nxa * nya, kStatThreads, smem, s>>>(ens_a, a_is_f32, nxa, nya, ens_b, b_is_f32, nxb, r, M, P,
                                                     mean_a, std_a, mean_b, std_b, w1);
  add_launches(1);
  if (cudaGetLastError() != cudaSuccess) {
    *why = "statistics kernel launch failed";
    return VLBM_ECUDA;
  }
  return VLBM_OK;
}

namespace {

// One thread per (coarse cell, realization): the block average in the
// summation order of stats_kernel (fine rows outer, fine columns inner).
__global__ void restrict_kernel(const void* __restrict__ ens, int is_f32, int nx, int r, int nxc, int nyc,
                                void* __restrict__ out, int out_f32) {
  const int m = blockIdx.y;
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)nxc * nyc;
  if (cell >= nc) return;
  const int I = (int)(cell % nxc), J = (int)(cell / nxc);
  const size_t nf = (size_t)nc * r * r;
  double s = 0.0;
  for (int aa = 0; aa < r; ++aa)
    for (int bb = 0; bb < r; ++bb)
      s += load_sample(ens, is_f32, (size_t)m * nf + (size_t)(r * J + aa) * nx + (size_t)(r * I + bb));
  const double v = s / (double)(r * r);
  const size_t o = (size_t)m * nc + cell;
  if (out_f32)
    reinterpret_cast<float*>(out)[o] = (float)v;
  else
    reinterpret_cast<double*>(out)[o] = v;
}

}  // namespace

cudaError_t restrict_launch(const void* ens, int is_f32, int nx, int ny, int M, int r, void* out, int out_f32,
                            cudaStream_t s) {
  const int nxc = nx / r, nyc = ny / r;
  const long long nc = (long long)nxc * nyc;
  if (nc == 0 || M == 0) return cudaSuccess;
  restrict_kernel<<<dim3((unsigned)((nc + 255) / 256), (unsigned)M), 256, 0, s>>>(ens, is_f32, nx, r, nxc, nyc, out,
                                                                                   out_f32);
  add_launches(1);
  return cudaGetLastError();
}

}  // namespace vlbm
