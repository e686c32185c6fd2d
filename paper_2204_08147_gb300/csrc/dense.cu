// The small dense step of the estimator on the device (Sec. 3.1-3.2, eq. fT):
//
//   c_{r,beta} = exp(-beta (T_r - t_r I) / 2) E1,   t_r = lambda_min(T_r),
//
// for every recurrence r (a bath vector's block-tridiagonal T_r of order n = k d_s with
// blocks A_j on the diagonal, B_j below and B_j^T above) and every beta of the grid,
// in float64. The host computes the same quantity from an eigendecomposition; here it
// is computed without one:
//
//   k_dense_bounds   t_r by 32-way multisection: each lane counts the eigenvalues of
//                    T_r below its shift sigma from the inertia of the block LDL^T
//                    factorisation of T_r - sigma I (Sylvester's law of inertia; the
//                    blocks D_j are d_s x d_s). Gershgorin bounds start the search and
//                    give the top of the spectrum; the first rounds count in float32
//                    (GB300's float64 pipe is narrow) down to a bracket of 1e-4 of the
//                    spectrum's scale, widened by its own width, the rest in float64.
//   k_cheb_vectors   the Chebyshev vectors v_i = C_i(T~) E1, i = 0..m, of T~ = the
//                    spectrum interval [t_r, top] mapped to [-1, 1], by the three-term
//                    recurrence C_{i+1} = 2 T~ C_i - C_{i-1} (block-tridiagonal
//                    products in shared memory).
//   k_cheb_combine   c = sum_i alpha_i(omega) v_i with omega = beta (top - t_r) / 4 and
//                    exp(-omega (1 + x)) = sum_i alpha_i C_i(x),
//                    alpha_0 = e^-omega I_0(omega), alpha_i = 2 (-1)^i e^-omega I_i(omega)
//                    (the generating function of the modified Bessel functions I_i);
//                    e^-omega I_i(omega) come from Miller's backward recurrence
//                    I_{i-1} = (2i / omega) I_i + I_{i+1}, normalised by
//                    I_0 + 2 sum_{i>=1} I_i = e^omega.
//
// The degree m is where e^-omega I_i(omega) ~ exp(-i^2 / (2 omega)) / sqrt(2 pi omega)
// falls below 1e-17 for the largest beta: m = sqrt(78 omega + 1) + 8.
//
// One launch of each kernel covers every recurrence of every job (estimate) of a batch
// with the same d_s: block g of a launch is recurrence g - pre[j] of job j.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "rdm_internal.h"

namespace rdm {
namespace {

constexpr int kChebThreads = 256;
constexpr int kDenseSmemMax = 200 * 1024;  // dynamic shared memory of the largest launch
constexpr int kCombineBetas = 16;

__device__ __forceinline__ double blk(const double* m, int ds, int a, int b) { return m[a * ds + b]; }

// Block g of a launch -> its job (largest j with pre[j] <= g among n jobs).
__device__ __forceinline__ int job_of(const int* pre, int n, int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Eigenvalues of T - sigma I below zero, in arithmetic R (block LDL^T with no pivoting
// inside the d_s x d_s blocks; a pivot smaller than pivmin counts as negative and is
// replaced by -pivmin).
template <int DS, typename R>
__device__ int count_below(int k, int ng, int g, const double* ta, const double* tb, R sigma, R pivmin) {
  constexpr int NV = DS * DS;
  R D[DS][DS];
#pragma unroll
  for (int a = 0; a < DS; ++a)
#pragma unroll
    for (int b = 0; b < DS; ++b) D[a][b] = (R)ta[(size_t)g * NV + a * DS + b] - (a == b ? sigma : (R)0);
  int cnt = 0;
  for (int j = 0;; ++j) {
    R L[DS][DS], d[DS], id[DS];
#pragma unroll
    for (int i = 0; i < DS; ++i) {
      R di = D[i][i];
#pragma unroll
      for (int m = 0; m < DS; ++m)
        if (m < i) di -= L[i][m] * L[i][m] * d[m];
      if (!(fabs(di) >= pivmin)) di = -pivmin;  // also catches NaN
      if (di < (R)0) ++cnt;
      d[i] = di;
      id[i] = (R)1 / di;
#pragma unroll
      for (int r = 0; r < DS; ++r) {
        if (r <= i) continue;
        R x = D[r][i];
#pragma unroll
        for (int m = 0; m < DS; ++m)
          if (m < i) x -= L[r][m] * L[i][m] * d[m];
        L[r][i] = x * id[i];
      }
    }
    if (j + 1 >= k) break;
    // D_{j+1} = A_{j+1} - sigma I - B_j D_j^{-1} B_j^T; with X = L^{-1} B_j^T,
    // B_j D_j^{-1} B_j^T = X^T diag(1/d) X.
    const double* B = tb + ((size_t)j * ng + g) * NV;
    R X[DS][DS];
#pragma unroll
    for (int c = 0; c < DS; ++c)      // column c of B_j^T = row c of B_j
#pragma unroll
      for (int i = 0; i < DS; ++i) {  // forward substitution with unit lower L
        R x = (R)blk(B, DS, c, i);
#pragma unroll
        for (int m = 0; m < DS; ++m)
          if (m < i) x -= L[i][m] * X[m][c];
        X[i][c] = x;
      }
    const double* A = ta + ((size_t)(j + 1) * ng + g) * NV;
#pragma unroll
    for (int a = 0; a < DS; ++a)
#pragma unroll
      for (int b = 0; b < DS; ++b) {
        R s = (R)0;
#pragma unroll
        for (int i = 0; i < DS; ++i) s += X[i][a] * X[i][b] * id[i];
        D[a][b] = (R)blk(A, DS, a, b) - (a == b ? sigma : (R)0) - s;
      }
  }
  return cnt;
}

// One multisection round in arithmetic R: every lane counts at its own shift of the 32
// that split [lo, hi] into 33; the bracket becomes the pair of shifts around the first
// nonzero count.
template <int DS, typename R>
__device__ void multisect(int k, int ng, int g, const double* ta, const double* tb, double pivmin, double& lo,
                          double& hi) {
  const int lane = threadIdx.x & 31;
  const double sigma = lo + (hi - lo) * (double)(lane + 1) / 33.0;
  const int c = count_below<DS, R>(k, ng, g, ta, tb, (R)sigma, (R)pivmin);
  const unsigned m = __ballot_sync(0xffffffffu, c >= 1);
  if (m == 0u) {
    lo = lo + (hi - lo) * 32.0 / 33.0;
  } else {
    const int i = __ffs(m) - 1;
    const double si = lo + (hi - lo) * (double)(i + 1) / 33.0;
    const double sp = i > 0 ? lo + (hi - lo) * (double)i / 33.0 : lo;
    hi = si;
    lo = sp;
  }
}

// One warp per recurrence: Gershgorin bounds, then the smallest eigenvalue by
// multisection. lohi[2r] = a lower bound of lambda_min within 4e-16 of the spectrum's
// scale (count 0 there), lohi[2r+1] = the top of the Chebyshev interval.
template <int DS>
__global__ void __launch_bounds__(32) k_dense_bounds(const DenseJob* jobs, const int* pre, int n_jobs) {
  constexpr int NV = DS * DS;
  const int jb = job_of(pre, n_jobs, blockIdx.x);
  const DenseJob J = jobs[jb];
  const int g = blockIdx.x - pre[jb];
  const int lane = threadIdx.x, k = J.k, ng = J.ng;
  const double* ta = J.ta;
  const double* tb = J.tb;
  double lo = INFINITY, hi = -INFINITY, scale = 0.0;
  for (int j = lane; j < k; j += 32) {
    const double* A = ta + ((size_t)j * ng + g) * NV;
    const double* Bp = j > 0 ? tb + ((size_t)(j - 1) * ng + g) * NV : nullptr;
    const double* Bn = j + 1 < k ? tb + ((size_t)j * ng + g) * NV : nullptr;
    for (int a = 0; a < DS; ++a) {
      double rad = 0.0;
      for (int b = 0; b < DS; ++b) {
        if (b != a) rad += fabs(blk(A, DS, a, b));
        if (Bp) rad += fabs(blk(Bp, DS, a, b));  // T_{j,j-1} = B_{j-1}: row a
        if (Bn) rad += fabs(blk(Bn, DS, b, a));  // T_{j,j+1} = B_j^T: row a
      }
      const double c = blk(A, DS, a, a);
      lo = fmin(lo, c - rad);
      hi = fmax(hi, c + rad);
      scale = fmax(scale, fabs(c) + rad);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    scale = fmax(scale, __shfl_xor_sync(0xffffffffu, scale, o));
  }
  double* lohi = J.lohi;
  if (!(scale > 0.0)) {  // T = 0
    if (lane == 0) {
      lohi[2 * g] = 0.0;
      lohi[2 * g + 1] = 0.0;
    }
    return;
  }
  // the spectrum of T lies within [-||H||, ||H||] <= hnorm (the norm bound of the
  // terms), which caps the Gershgorin top and so the Chebyshev degree
  const double top = fmin(hi, J.hnorm * (1.0 + 1e-3));
  const double glo = lo, ghi = hi;
  // float32 rounds down to 1e-4 of the scale; the bracket is then widened by its width
  // on both sides (float32 counts near lambda_min may be off) and clipped to Gershgorin
  for (int round = 0; round < 8 && hi - lo > 1e-4 * scale; ++round)
    multisect<DS, float>(k, ng, g, ta, tb, 1e-6 * scale, lo, hi);
  const double w = hi - lo;
  lo = fmax(glo, lo - w);
  hi = fmin(ghi, hi + w);
  for (int round = 0; round < 16 && hi - lo > 4e-16 * scale; ++round)
    multisect<DS, double>(k, ng, g, ta, tb, 1e-13 * scale, lo, hi);
  if (lane == 0) {
    lohi[2 * g] = lo;
    lohi[2 * g + 1] = fmax(top, lo);
  }
}

__device__ __forceinline__ int cheb_degree(double omega, int vstride) {
  const int m = (int)ceil(sqrt(78.0 * fmax(omega, 0.0) + 1.0)) + 8;
  return m < vstride - 1 ? m : vstride - 1;
}

// One block per recurrence: v_0 = E1, v_1 = T~ v_0, v_{i+1} = 2 T~ v_i - v_{i-1}, written to
// V[g][i][row * DS + col] for i <= m_g (m_g from omega_max = beta_max (top - t) / 4).
template <int DS>
__global__ void __launch_bounds__(kChebThreads) k_cheb_vectors(const DenseJob* jobs, const int* pre, int n_jobs) {
  constexpr int NV = DS * DS;
  extern __shared__ __align__(16) double sm[];
  const int jb = job_of(pre, n_jobs, blockIdx.x);
  const DenseJob J = jobs[jb];
  const int g = blockIdx.x - pre[jb];
  const int k = J.k, ng = J.ng, vstride = J.vstride;
  const int n = k * DS, ne = n * DS;
  double* sA = sm;                  // [k][NV]
  double* sB = sA + (size_t)k * NV;  // [k][NV]
  double* v0 = sB + (size_t)k * NV;
  double* v1 = v0 + ne;
  double* v2 = v1 + ne;
  for (int i = threadIdx.x; i < k * NV; i += blockDim.x) {
    const int j = i / NV, e = i % NV;
    sA[i] = J.ta[((size_t)j * ng + g) * NV + e];
    sB[i] = J.tb[((size_t)j * ng + g) * NV + e];
  }
  const double lo = J.lohi[2 * g], top = J.lohi[2 * g + 1];
  const double width = top - lo > 0.0 ? top - lo : 1.0;
  const double s = 2.0 / width, c = (lo + top) / width;  // T~ = s T - c I
  const int m = cheb_degree(J.beta_max * width / 4.0, vstride);
  double* Vg = J.V + (size_t)g * vstride * ne;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    const int row = e / DS, col = e % DS;
    const double x = row == col ? 1.0 : 0.0;
    v0[e] = x;
    Vg[e] = x;
  }
  __syncthreads();
  double* prev = nullptr;
  double* cur = v0;
  double* nxt = v1;
  for (int i = 1; i <= m; ++i) {
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int row = e / DS, col = e % DS, j = row / DS, a = row % DS;
      const double* A = sA + (size_t)j * NV;
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < DS; ++b) t += A[a * DS + b] * cur[(j * DS + b) * DS + col];
      if (j > 0) {
        const double* Bp = sB + (size_t)(j - 1) * NV;
#pragma unroll
        for (int b = 0; b < DS; ++b) t += Bp[a * DS + b] * cur[((j - 1) * DS + b) * DS + col];
      }
      if (j + 1 < k) {
        const double* Bn = sB + (size_t)j * NV;
#pragma unroll
        for (int b = 0; b < DS; ++b) t += Bn[b * DS + a] * cur[((j + 1) * DS + b) * DS + col];
      }
      const double tv = s * t - c * cur[e];
      const double r = prev ? 2.0 * tv - prev[e] : tv;
      nxt[e] = r;
      Vg[(size_t)i * ne + e] = r;
    }
    __syncthreads();
    double* np = prev ? prev : v2;
    prev = cur;
    cur = nxt;
    nxt = np;
  }
}

// e^-omega I_i(omega), i = 0..m, into out (Miller's backward recurrence from M > m).
__device__ void scaled_bessel_i(double omega, int m, double* out) {
  if (!(omega > 1e-20)) {  // exp(-omega (1 + x)) = 1 to working precision
    out[0] = 1.0;
    for (int i = 1; i <= m; ++i) out[i] = 0.0;
    return;
  }
  const int M = m + 24 + m / 4;
  double ip1 = 0.0, ii = 1e-280, sum = 0.0;
  for (int i = 0; i <= m; ++i) out[i] = 0.0;
  for (int i = M; i >= 1; --i) {
    const double im1 = (2.0 * i / omega) * ii + ip1;  // I_{i-1}
    if (i <= m) out[i] = ii;
    sum += 2.0 * ii;
    ip1 = ii;
    ii = im1;
    if (fabs(ii) > 1e250) {  // rescale everything kept so far
      const double f = 1e-250;
      ii *= f;
      ip1 *= f;
      sum *= f;
      for (int q = i; q <= m; ++q) out[q] *= f;
    }
  }
  out[0] = ii;
  sum += ii;
  const double inv = 1.0 / sum;
  for (int i = 0; i <= m; ++i) out[i] *= inv;
}

// c[g][beta][row][col] = sum_i alpha_i(omega_beta) V[g][i][row][col] for the betas
// b0 .. b0 + kCombineBetas - 1 of block row blockIdx.y (blocks past a job's grid exit).
template <int DS>
__global__ void __launch_bounds__(kChebThreads) k_cheb_combine(const DenseJob* jobs, const int* pre, int n_jobs) {
  extern __shared__ __align__(16) double sa[];  // [kCombineBetas][vstride]
  const int jb = job_of(pre, n_jobs, blockIdx.x);
  const DenseJob J = jobs[jb];
  const int g = blockIdx.x - pre[jb];
  const int b0 = blockIdx.y * kCombineBetas;
  if (b0 >= J.n_beta) return;
  const int nb = min(kCombineBetas, J.n_beta - b0), vstride = J.vstride;
  const int n = J.k * DS, ne = n * DS;
  const double lo = J.lohi[2 * g], top = J.lohi[2 * g + 1];
  const double width = top - lo > 0.0 ? top - lo : 1.0;
  const int m = cheb_degree(J.beta_max * width / 4.0, vstride);
  if ((int)threadIdx.x < nb) {
    double* al = sa + (size_t)threadIdx.x * vstride;
    scaled_bessel_i(J.betas[b0 + threadIdx.x] * width / 4.0, m, al);
    for (int i = 1; i <= m; ++i) al[i] *= (i & 1) ? -2.0 : 2.0;
  }
  __syncthreads();
  const double* Vg = J.V + (size_t)g * vstride * ne;
  for (int e = threadIdx.x; e < ne; e += blockDim.x) {
    double acc[kCombineBetas];
#pragma unroll
    for (int b = 0; b < kCombineBetas; ++b) acc[b] = 0.0;
    for (int i = 0; i <= m; ++i) {
      const double v = Vg[(size_t)i * ne + e];
#pragma unroll
      for (int b = 0; b < kCombineBetas; ++b)
        if (b < nb) acc[b] = fma(sa[(size_t)b * vstride + i], v, acc[b]);
    }
#pragma unroll
    for (int b = 0; b < kCombineBetas; ++b)
      if (b < nb) J.cout[((size_t)g * J.n_beta + b0 + b) * ne + e] = acc[b];
  }
}

template <int DS>
cudaError_t launch_dense(const DenseJob* jobs, const int* pre, int n_jobs, int n_blocks, int max_k,
                         int max_beta_chunks, int max_vstride, cudaStream_t st) {
  // Both Chebyshev kernels' dynamic shared-memory limits are raised once, to the largest
  // size any launch uses (kDenseSmemMax), so concurrent host threads cannot lower one
  // under another's launch.
  static std::once_flag once;
  static cudaError_t set_err = cudaSuccess;
  std::call_once(once, [] {
    set_err = cudaFuncSetAttribute(k_cheb_vectors<DS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmemMax);
    if (set_err == cudaSuccess)
      set_err = cudaFuncSetAttribute(k_cheb_combine<DS>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDenseSmemMax);
  });
  if (set_err != cudaSuccess) return set_err;
  k_dense_bounds<DS><<<n_blocks, 32, 0, st>>>(jobs, pre, n_jobs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smv = (size_t)5 * max_k * DS * DS * sizeof(double);
  k_cheb_vectors<DS><<<n_blocks, kChebThreads, smv, st>>>(jobs, pre, n_jobs);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smc = (size_t)kCombineBetas * max_vstride * sizeof(double);
  k_cheb_combine<DS><<<dim3((unsigned)n_blocks, (unsigned)max_beta_chunks), kChebThreads, smc, st>>>(jobs, pre,
                                                                                                     n_jobs);
  return cudaGetLastError();
}

}  // namespace

bool dense_device_fits(int k, int ds) {
  const size_t smv = (size_t)5 * k * ds * ds * sizeof(double);
  return ds >= 1 && ds <= 4 && smv <= (size_t)kDenseSmemMax &&
         (size_t)kCombineBetas * (kChebMaxDegree + 1) * sizeof(double) <= (size_t)kDenseSmemMax;
}

int dense_device_max_degree(double beta_max, double hnorm) {
  // the Chebyshev interval lies in [-hnorm, 1.001 hnorm] (k_dense_bounds)
  const double omega = beta_max * 2.002 * hnorm / 4.0;
  int m = (int)ceil(sqrt(78.0 * (omega > 0 ? omega : 0.0) + 1.0)) + 8;
  return m < kChebMaxDegree ? m : kChebMaxDegree;
}

size_t dense_jobs_bytes(int n_jobs) {
  return (sizeof(DenseJob) * (size_t)n_jobs + sizeof(int) * ((size_t)n_jobs + 1) + 255) / 256 * 256;
}

cudaError_t launch_dense_jobs(int ds, const DenseJob* host_jobs, int n_jobs, void* scratch, cudaStream_t st) {
  if (n_jobs < 1 || !scratch) return cudaErrorInvalidValue;
  int n_blocks = 0, max_k = 1, max_chunks = 1, max_vs = 2;
  for (int i = 0; i < n_jobs; ++i) {
    const DenseJob& J = host_jobs[i];
    if (J.n_rec < 1 || J.k < 1 || J.n_beta < 1 || J.vstride < 2 || J.vstride > kChebMaxDegree + 1 ||
        !dense_device_fits(J.k, ds))
      return cudaErrorInvalidValue;
    n_blocks += J.n_rec;
    max_k = std::max(max_k, J.k);
    max_chunks = std::max(max_chunks, (J.n_beta + kCombineBetas - 1) / kCombineBetas);
    max_vs = std::max(max_vs, J.vstride);
  }
  // descriptors + prefix sums, one copy into the caller's scratch (dense_jobs_bytes)
  std::vector<unsigned char> img(dense_jobs_bytes(n_jobs));
  DenseJob* dj = reinterpret_cast<DenseJob*>(img.data());
  int* pre = reinterpret_cast<int*>(img.data() + sizeof(DenseJob) * (size_t)n_jobs);
  int acc = 0;
  for (int i = 0; i < n_jobs; ++i) {
    dj[i] = host_jobs[i];
    pre[i] = acc;
    acc += host_jobs[i].n_rec;
  }
  pre[n_jobs] = acc;
  cudaError_t e = cudaMemcpyAsync(scratch, img.data(), img.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);  // the pageable image must outlive its copy
  if (e != cudaSuccess) return e;
  const DenseJob* d_jobs = reinterpret_cast<const DenseJob*>(scratch);
  const int* d_pre = reinterpret_cast<const int*>(static_cast<unsigned char*>(scratch) +
                                                  sizeof(DenseJob) * (size_t)n_jobs);
  switch (ds) {
    case 1: return launch_dense<1>(d_jobs, d_pre, n_jobs, n_blocks, max_k, max_chunks, max_vs, st);
    case 2: return launch_dense<2>(d_jobs, d_pre, n_jobs, n_blocks, max_k, max_chunks, max_vs, st);
    case 4: return launch_dense<4>(d_jobs, d_pre, n_jobs, n_blocks, max_k, max_chunks, max_vs, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace rdm
