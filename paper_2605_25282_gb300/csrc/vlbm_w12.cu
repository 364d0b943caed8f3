// Two-point Wasserstein distance W_{1,2} (Sec. 3.4, Eq. (w2)).
//
// The grid is subsampled to npd x npd points (the centre cell of each of npd
// equal strips per direction).  For every ordered pair (x_k, x_k') of them,
// the empirical joint laws of (rho(x_k), rho(x_k')) over the M realizations of
// the two ensembles are M points each on R^2; their first Wasserstein distance
// with Euclidean ground cost is an assignment problem,
//   W = (1/M) min over permutations sigma of sum_i |a_i - b_sigma(i)|,
// solved exactly by the shortest-augmenting-path (Hungarian) method with dual
// potentials: one CTA per pair, the columns spread over the threads, one
// deterministic block argmin per Dijkstra step.  The fine ensemble is block-
// averaged onto the coarse grid at the sampled cells first (Sec. 3.3).
// W_{1,2} is the mean over the P = npd^4 pairs, summed in a fixed order.
#include <cfloat>

#include "vlbm_internal.cuh"

namespace vlbm {
namespace {

constexpr int kWT = 256;

__device__ __forceinline__ double sample(const void* p, int f32, size_t idx) {
  return f32 ? (double)reinterpret_cast<const float*>(p)[idx] : reinterpret_cast<const double*>(p)[idx];
}

__device__ __forceinline__ int strip_centre(int k, int n, int npd) { return ((2 * k + 1) * n) / (2 * npd); }

struct W12Args {
  const void* a;
  int a_f32, nxa, nya;
  const void* b;
  int b_f32, nxb, r;
  int M, npd;
  double* pair_w;
};

// shared layout: ax, ay, bx, by [M]; u, v, minv [M + 1]; p, way [M + 1]; used [M + 1]
__global__ void __launch_bounds__(kWT) w12_pair_kernel(const W12Args A) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int M = A.M;
  double* ax = reinterpret_cast<double*>(sm_raw);
  double* ay = ax + M;
  double* bx = ay + M;
  double* by = bx + M;
  double* u = by + M;
  double* v = u + (M + 1);
  double* minv = v + (M + 1);
  int* pa = reinterpret_cast<int*>(minv + (M + 1));
  int* way = pa + (M + 1);
  unsigned char* used = reinterpret_cast<unsigned char*>(way + (M + 1));
  __shared__ double red_v[kWT / 32];
  __shared__ int red_j[kWT / 32];
  __shared__ double s_delta;
  __shared__ int s_j1, s_done;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int npp = A.npd * A.npd;
  const int k1 = blockIdx.x / npp, k2 = blockIdx.x % npp;
  const int i1 = strip_centre(k1 % A.npd, A.nxa, A.npd), j1c = strip_centre(k1 / A.npd, A.nya, A.npd);
  const int i2 = strip_centre(k2 % A.npd, A.nxa, A.npd), j2c = strip_centre(k2 / A.npd, A.nya, A.npd);
  const size_t na = (size_t)A.nxa * A.nya, nb = na * (size_t)A.r * A.r;
  for (int m = tid; m < M; m += kWT) {
    ax[m] = sample(A.a, A.a_f32, (size_t)m * na + (size_t)j1c * A.nxa + i1);
    ay[m] = sample(A.a, A.a_f32, (size_t)m * na + (size_t)j2c * A.nxa + i2);
    double s1 = 0.0, s2 = 0.0;
    for (int aa = 0; aa < A.r; ++aa)
      for (int bb = 0; bb < A.r; ++bb) {
        s1 += sample(A.b, A.b_f32, (size_t)m * nb + (size_t)(A.r * j1c + aa) * A.nxb + (size_t)(A.r * i1 + bb));
        s2 += sample(A.b, A.b_f32, (size_t)m * nb + (size_t)(A.r * j2c + aa) * A.nxb + (size_t)(A.r * i2 + bb));
      }
    bx[m] = s1 / (double)(A.r * A.r);
    by[m] = s2 / (double)(A.r * A.r);
  }
  for (int j = tid; j <= M; j += kWT) {
    u[j] = 0.0;
    v[j] = 0.0;
    pa[j] = 0;
    way[j] = 0;
  }
  __syncthreads();
  auto cost = [&](int i, int j) {  // 1-based row (a) and column (b)
    const double dx = ax[i - 1] - bx[j - 1], dy = ay[i - 1] - by[j - 1];
    return sqrt(dx * dx + dy * dy);
  };
  for (int i = 1; i <= M; ++i) {
    for (int j = tid; j <= M; j += kWT) {
      minv[j] = DBL_MAX;
      used[j] = 0;
    }
    if (tid == 0) {
      pa[0] = i;
      s_j1 = 0;  // j0 of the first Dijkstra step
    }
    __syncthreads();
    for (int guard = 0; guard <= M + 1; ++guard) {
      const int j0 = s_j1;
      if (tid == 0) used[j0] = 1;
      __syncthreads();
      const int i0 = pa[j0];
      // relax the columns not yet in the tree; argmin of minv (smallest j on ties)
      double best = DBL_MAX;
      int bj = 0x7fffffff;
      for (int j = tid + 1; j <= M; j += kWT) {
        if (used[j]) continue;
        const double cur = cost(i0, j) - u[i0] - v[j];
        if (cur < minv[j]) {
          minv[j] = cur;
          way[j] = j0;
        }
        if (minv[j] < best || (minv[j] == best && j < bj)) {
          best = minv[j];
          bj = j;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob < best || (ob == best && oj < bj)) {
          best = ob;
          bj = oj;
        }
      }
      if (lane == 0) {
        red_v[wid] = best;
        red_j[wid] = bj;
      }
      __syncthreads();
      if (tid == 0) {
        double bv = red_v[0];
        int bjj = red_j[0];
        for (int w = 1; w < kWT / 32; ++w)
          if (red_v[w] < bv || (red_v[w] == bv && red_j[w] < bjj)) {
            bv = red_v[w];
            bjj = red_j[w];
          }
        s_delta = bv;
        s_j1 = bjj;
      }
      __syncthreads();
      const double delta = s_delta;
      // update the potentials of the tree and the keys of the other columns
      for (int j = tid; j <= M; j += kWT) {
        if (used[j]) {
          u[pa[j]] += delta;
          v[j] -= delta;
        } else {
          minv[j] -= delta;
        }
      }
      __syncthreads();
      if (tid == 0) s_done = pa[s_j1] == 0;
      __syncthreads();
      if (s_done) break;
    }
    // augment along the path (sequential)
    if (tid == 0) {
      int j0 = s_j1;
      for (int guard = 0; guard <= M + 1 && j0 != 0; ++guard) {
        const int jp = way[j0];
        pa[j0] = pa[jp];
        j0 = jp;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    double s = 0.0;
    for (int j = 1; j <= M; ++j) s += cost(pa[j], j);
    A.pair_w[blockIdx.x] = s / (double)M;
  }
}

// mean of the P pair values in a fixed order (one CTA)
__global__ void __launch_bounds__(1024) w12_mean_kernel(const double* pair_w, long long P, double* out) {
  __shared__ double sh[1024];
  double s = 0.0;
  for (long long t = threadIdx.x; t < P; t += 1024) s += pair_w[t];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] / (double)P;
}

}  // namespace

size_t w12_smem_bytes(int M) {
  return (size_t)4 * M * sizeof(double) + (size_t)3 * (M + 1) * sizeof(double) + (size_t)2 * (M + 1) * sizeof(int) +
         (size_t)(M + 1);
}

cudaError_t w12_launch(const void* a, int a_f32, int nxa, int nya, const void* b, int b_f32, int nxb, int r, int M,
                       int npd, double* pair_w, double* out, cudaStream_t s) {
  const size_t smem = w12_smem_bytes(M);
  cudaError_t e = cudaFuncSetAttribute(w12_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  W12Args A{a, a_f32, nxa, nya, b, b_f32, nxb, r, M, npd, pair_w};
  const long long P = (long long)npd * npd * npd * npd;
  w12_pair_kernel<<<(unsigned)P, kWT, smem, s>>>(A);
  w12_mean_kernel<<<1, 1024, 0, s>>>(pair_w, P, out);
  add_launches(2);
  return cudaGetLastError();
}

}  // namespace vlbm
