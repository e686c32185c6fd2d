// CUDA kernels of the estimator's hot path (sm_103a).
//
//   k_init_block   the starting block V = [I_s (x) |v_l>]_l (Sec. 3.1, eq. trace_est)
//                  from the counter-based generator (SplitMix64 on a counter)
//   k_spmm         Z = (H W_j) M_j + W_{j-1} Cp_j: the matrix-free spin-Hamiltonian
//                  block SpMM (eq. Ht) fused with the first line of Algorithm 1's
//                  loop, and the partial sums of W_j^T Z for A_j
//   k_orth         W_{j+1} = Z + W_j Cw_j (Algorithm 1, Z - Q_j A_j) with the
//                  partial sums of W_{j+1}^T W_{j+1} for the QR (pass 1), or the
//                  accumulation psi_beta += W_{j+1} E_{j+1,beta} (pass 2)
//   k_small_a/b    per bath vector, float64: A_j, Cholesky QR with breakdown
//                  deflation, the next step's mixing coefficients
//   k_final_gram   the bath-traced Gram psi_l^T psi_l per bath vector
//
// The Krylov block of every bath vector l is never normalised in memory: the
// stored W_j relates to the orthonormal Q_j of Algorithm 1 by Q_j = W_j M_j with
// a d_s x d_s matrix M_j (the inverse Cholesky factor), applied on the fly.
// Reductions are deterministic: per-thread partial sums, a fixed-order block
// reduction into per-block partials, and a fixed-order sum over blocks.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <set>

#include "rdm_internal.h"

namespace rdm {
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

__device__ __forceinline__ double gauss_raw(uint64_t seed, uint64_t l, uint64_t b) {
  const uint64_t base = l << 40;
  const uint64_t z1 = splitmix64(seed, (base | (2 * b)) + 1);
  const uint64_t z2 = splitmix64(seed, (base | (2 * b + 1)) + 1);
  const double u1 = ((double)(z1 >> 11) + 0.5) * 0x1.0p-53;
  const double u2 = ((double)(z2 >> 11) + 0.5) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// ---- VW-wide vector access (VW * sizeof(T) is 8, 16 or 32 bytes).
template <typename T, int VW>
struct VecIO;
template <>
struct VecIO<float, 4> {
  __device__ static void st_cs(float* p, const float* r) {  // streaming (evict-first) store
    __stcs(reinterpret_cast<float4*>(p), make_float4(r[0], r[1], r[2], r[3]));
  }
  __device__ static void ld(float* r, const float* p) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
  __device__ static void ld_rw(float* r, const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
  __device__ static void st(float* p, const float* r) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
  }
};
template <>
struct VecIO<double, 2> {
  __device__ static void st_cs(double* p, const double* r) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(r[0], r[1]));
  }
  __device__ static void ld(double* r, const double* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    r[0] = v.x; r[1] = v.y;
  }
  __device__ static void ld_rw(double* r, const double* p) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    r[0] = v.x; r[1] = v.y;
  }
  __device__ static void st(double* p, const double* r) {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
  }
};
template <>
struct VecIO<double, 4> {
  __device__ static void st_cs(double* p, const double* r) {
    VecIO<double, 2>::st_cs(p, r);
    VecIO<double, 2>::st_cs(p + 2, r + 2);
  }
  __device__ static void ld(double* r, const double* p) {
    VecIO<double, 2>::ld(r, p);
    VecIO<double, 2>::ld(r + 2, p + 2);
  }
  __device__ static void ld_rw(double* r, const double* p) {
    VecIO<double, 2>::ld_rw(r, p);
    VecIO<double, 2>::ld_rw(r + 2, p + 2);
  }
  __device__ static void st(double* p, const double* r) {
    VecIO<double, 2>::st(p, r);
    VecIO<double, 2>::st(p + 2, r + 2);
  }
};

// Mask of the lanes of this thread's row group inside its warp.
__device__ __forceinline__ unsigned group_mask(int tpr) {
  if (tpr >= 32) return 0xffffffffu;
  const unsigned lane = threadIdx.x & 31u;
  return ((1u << tpr) - 1u) << (lane & ~(unsigned)(tpr - 1));
}

// Fixed-order block reduction of NV values per thread into per-block float64
// partials: partials[((slice*gridx + bx)*G_s + lane*NG + g)*NVG + v] where
// vals[g*NVG + v] belongs to group g of the thread and lane = threadIdx.x % tpr
// (tpr <= 8, a power of two), slot = slice*gridx + bx the block's place in the grid
// (blockIdx.y * gridDim.x + blockIdx.x for a plain launch). A butterfly over the lanes of a warp with the same
// lane in the type R of vals, then the warps' sums added in float64 in warp order:
// the same order on every run. The float32 path runs the butterfly in float32 (its
// per-thread sums are float32 already): GB300's float64 pipe is narrow, and a float64
// butterfly in every block made launches of many short blocks float64-bound.
template <int NG, int NVG, typename R = double>
__device__ void block_reduce_store(const R* vals, int tpr, double* partials, int gs, size_t slot) {
  constexpr int NV = NG * NVG;
  constexpr int kWarps = kThreads / 32;
  __shared__ double red[kWarps * 8 * NV];
  const int warp = threadIdx.x >> 5, wl = threadIdx.x & 31;
  R v[NV];
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    R x = vals[e];
    for (int o = tpr; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[e] = x;
  }
  if (wl < tpr) {
#pragma unroll
    for (int e = 0; e < NV; ++e) red[(warp * tpr + wl) * NV + e] = (double)v[e];
  }
  __syncthreads();
  if ((int)threadIdx.x < tpr * NV) {
    const int lane = threadIdx.x / NV, e = threadIdx.x % NV;
    double sum = 0.0;
    for (int w = 0; w < kWarps; ++w) sum += red[(w * tpr + lane) * NV + e];
    const size_t base = (slot * gs + (size_t)lane * NG) * NVG;
    partials[base + e] = sum;
  }
}

// ---------------------------------------------------------------- init

__global__ void k_gauss_sumsq(int64_t d_b, uint64_t seed, int64_t l0, double* part, double* graw) {
  __shared__ double sh[kThreads];
  const int l = blockIdx.y;
  const int64_t chunk = (d_b + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  const int64_t hi = lo + chunk < d_b ? lo + chunk : d_b;
  double acc = 0.0;
  for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x) {
    const double g = gauss_raw(seed, (uint64_t)(l0 + l), (uint64_t)b);
    if (graw) graw[(size_t)l * d_b + b] = g;
    acc += g * g;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)l * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void k_gauss_finish(int n_v, int gx, const double* part, double* inv_norm) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_v) return;
  double s = 0.0;
  for (int i = 0; i < gx; ++i) s += part[(size_t)l * gx + i];
  inv_norm[l] = 1.0 / sqrt(s);
}

template <typename T, int DS, int VW>
__global__ void __launch_bounds__(kThreads) k_init_block(Layout L, int dist, uint64_t seed,
                                                         int64_t l0, int nvr, const double* inv_norm,
                                                         const T* vbuf, T* W, int sub, BathPerm bp) {
  constexpr int NG = VW / DS;
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = blockIdx.y;
  T* base = W + (size_t)slice * L.D * L.Bs + lane * VW;
  const int g0 = (slice * L.Bs + lane * VW) / DS;
  const uint64_t bmask = (1ull << L.n_bath_bits) - 1ull;
  const double rad = 1.0 / sqrt((double)(1ull << L.n_bath_bits));
  for (int64_t s = (int64_t)blockIdx.x * rpb + rs; s < L.D; s += (int64_t)gridDim.x * rpb) {
    const int i = (int)(s >> L.n_bath_bits);
    uint64_t b = (uint64_t)s & bmask;
    if (bp.n) {  // the caller's bath index of internal bath index b
      uint64_t bc = 0;
      for (int q = 0; q < bp.n; ++q) bc |= ((b >> q) & 1ull) << bp.src[q];
      b = bc;
    }
    T v[VW];
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      // group g0 + g: bath vector l, system index ic of its column when the groups are
      // single columns of sub-column bath vectors (per-column recurrences), else 0
      const int l = (g0 + g) / sub, ic = (g0 + g) % sub;
      double val = 0.0;
      if (l < nvr) {
        const uint64_t lg = (uint64_t)(l0 + l);  // index in the seeded sequence
        if (dist == RDM_RADEMACHER) {
          const uint64_t z = splitmix64(seed, ((lg << 40) | b) + 1);
          val = (z >> 63) ? -rad : rad;
        } else if (dist == RDM_GAUSS) {
          val = inv_norm ? gauss_raw(seed, lg, b) * inv_norm[l]
                         : (double)vbuf[((size_t)l << L.n_bath_bits) + b];
        } else {
          val = (b == lg) ? 1.0 : 0.0;
        }
      }
#pragma unroll
      for (int a = 0; a < DS; ++a) v[g * DS + a] = (a + ic == i) ? (T)val : (T)0;
    }
    VecIO<T, VW>::st(base + (size_t)s * L.Bs, v);
  }
}

__global__ void k_gauss_fill(int64_t d_b, uint64_t seed, int64_t l0, const double* inv_norm,
                             const double* graw, int precision, void* vbuf) {
  const int l = blockIdx.y;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < d_b;
       b += (int64_t)gridDim.x * blockDim.x) {
    const double g = graw ? graw[(size_t)l * d_b + b] : gauss_raw(seed, (uint64_t)(l0 + l), (uint64_t)b);
    const double v = g * inv_norm[l];
    if (precision == RDM_FP32)
      reinterpret_cast<float*>(vbuf)[(size_t)l * d_b + b] = (float)v;
    else
      reinterpret_cast<double*>(vbuf)[(size_t)l * d_b + b] = v;
  }
}

// A table of the tiled diagonal (TileDiag): one block per tile (grid stride). The block
// first sums K_0 .. K_G of the tile (float64, shared memory), then thread rg writes
// A_q(tile, rg) of every row-group-dependent character q and thread 0 the others.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_tile_diag(int64_t tiles, TileDiag dg, int stride, T* out) {
  extern __shared__ __align__(16) unsigned char smem_k[];
  double* sK = reinterpret_cast<double*>(smem_k);  // [G + 1]
  constexpr int kRG = 1 << kTileRegShift;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t ut = (uint32_t)t;
    for (int g = threadIdx.x; g <= dg.n_groups; g += blockDim.x) {
      double k = 0.0;
      for (int i = dg.slot_start[g]; i < dg.slot_start[g + 1]; ++i)
        k += (__popc(ut & dg.thi[i]) & 1) ? -dg.tc[i] : dg.tc[i];
      sK[g] = k;
    }
    __syncthreads();
    T* o = out + t * stride;
    for (int rg = threadIdx.x; rg < kRG; rg += blockDim.x) {
      for (int q = 0; q < 8; ++q) {
        const bool dep = (dg.dep >> q) & 1u;
        if (!dep && rg != 0) continue;
        double a = q == 0 ? sK[0] : 0.0;
        for (int g = dg.hstart[q]; g < dg.hstart[q + 1]; ++g)
          a += (__popc((uint32_t)rg & dg.mlo[g]) & 1) ? -sK[1 + g] : sK[1 + g];
        o[dg.off[q] + (dep ? rg : 0)] = (T)a;
      }
    }
    for (int e = dg.n_entries + threadIdx.x; e < stride; e += blockDim.x) o[e] = (T)0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- SpMM step

template <typename T>
struct TermsSmem {
  uint32_t* fmask;
  T* fodd;
  T* feven;
  uint32_t* dmask;
  T* dc;
};

template <typename T>
__device__ TermsSmem<T> load_terms(const FlipTerm* flips, int nf, const DiagTerm* diags, int nd) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TermsSmem<T> t;
  T* tp = reinterpret_cast<T*>(smem_raw);
  t.fodd = tp;
  t.feven = tp + nf;
  t.dc = tp + 2 * nf;
  uint32_t* up = reinterpret_cast<uint32_t*>(tp + 2 * nf + nd);
  t.fmask = up;
  t.dmask = up + nf;
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    t.fmask[i] = flips[i].mask;
    t.fodd[i] = (T)flips[i].c_odd;
    t.feven[i] = (T)flips[i].c_even;
  }
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    t.dmask[i] = diags[i].mask;
    t.dc[i] = (T)diags[i].c;
  }
  __syncthreads();
  return t;
}

// The rows of block (bx, by) of a grid of gx x n_slices blocks of the untiled SpMM:
// rows bx*rpb + rs + i*gx*rpb of slice by (the grid-stride walk of a plain launch), and,
// in pass 1, its partial sums of W_j^T Z at slot by*gx + bx. `terms` are the term tables
// in shared memory (load_terms).
template <typename T, int VW, bool COH>
__device__ __forceinline__ void ld_vec(T* r, const T* p) {
  if constexpr (COH)
    VecIO<T, VW>::ld_rw(r, p);
  else
    VecIO<T, VW>::ld(r, p);
}

// COH: coherent loads only (no read-only cache path), for blocks written earlier in the
// same launch (the packed kernel).
template <typename T, int DS, int VW, int MODE, bool COH = false>
__device__ __forceinline__ void spmm_block(const Layout& L, const SpmmArgs& a, const TermsSmem<T>& terms,
                                           int bx, int by, int gx) {
  constexpr int NG = VW / DS;
  constexpr int NVG = DS * DS;
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = by;
  const size_t soff = (size_t)slice * L.D * L.Bs + (size_t)lane * VW;
  const T* __restrict__ W = reinterpret_cast<const T*>(a.w) + soff;
  const T* __restrict__ Wp = a.w_prev ? reinterpret_cast<const T*>(a.w_prev) + soff : nullptr;
  T* __restrict__ Z = reinterpret_cast<T*>(a.z) + soff;
  const int g0 = (slice * L.Bs + lane * VW) / DS;
  const unsigned gmask = group_mask(tpr);

  T mz[NG][DS][DS], cp[NG][DS][DS];
  if (MODE != kModeApply) {
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < DS; ++i)
#pragma unroll
        for (int j = 0; j < DS; ++j) {
          mz[g][i][j] = (T)a.mz[(size_t)(g0 + g) * NVG + i * DS + j];
          cp[g][i][j] = Wp ? (T)a.cp[(size_t)(g0 + g) * NVG + i * DS + j] : (T)0;
        }
  }
  T acc[NG][DS][DS];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < DS; ++i)
#pragma unroll
      for (int j = 0; j < DS; ++j) acc[g][i][j] = (T)0;

  const int nf = a.n_flip, nd = a.n_diag;
  for (int64_t s = (int64_t)bx * rpb + rs; s < L.D; s += (int64_t)gx * rpb) {
    const uint32_t su = (uint32_t)s;
    T x[VW];
    ld_vec<T, VW, COH>(x, W + (size_t)s * L.Bs);
    // Diagonal: sum_t c_t (1 - 2 parity(s & m_t)), split over the row group.
    T dg = (T)0;
    for (int t = lane; t < nd; t += tpr) {
      const T c = terms.dc[t];
      dg += (__popc(su & terms.dmask[t]) & 1) ? -c : c;
    }
    for (int off = tpr >> 1; off > 0; off >>= 1) dg += __shfl_xor_sync(gmask, dg, off, tpr);
    T y[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) y[v] = dg * x[v];
    // Off-diagonal: y += c(parity(s & m)) x[s ^ m].
    for (int t = 0; t < nf; ++t) {
      const uint32_t m = terms.fmask[t];
      const T c = (__popc(su & m) & 1) ? terms.fodd[t] : terms.feven[t];
      if (c != (T)0) {
        T xp[VW];
        ld_vec<T, VW, COH>(xp, W + (size_t)(su ^ m) * L.Bs);
#pragma unroll
        for (int v = 0; v < VW; ++v) y[v] = fma(c, xp[v], y[v]);
      }
    }
    if (MODE == kModeApply) {
      VecIO<T, VW>::st(Z + (size_t)s * L.Bs, y);
      continue;
    }
    T z[VW];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int j = 0; j < DS; ++j) {
        T t = (T)0;
#pragma unroll
        for (int i = 0; i < DS; ++i) t = fma(y[g * DS + i], mz[g][i][j], t);
        z[g * DS + j] = t;
      }
    if (Wp) {
      T xp[VW];
      ld_vec<T, VW, COH>(xp, Wp + (size_t)s * L.Bs);
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int j = 0; j < DS; ++j) {
          T t = z[g * DS + j];
#pragma unroll
          for (int i = 0; i < DS; ++i) t = fma(xp[g * DS + i], cp[g][i][j], t);
          z[g * DS + j] = t;
        }
    }
    VecIO<T, VW>::st(Z + (size_t)s * L.Bs, z);
    if (MODE == kModePass1) {
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int i = 0; i < DS; ++i)
#pragma unroll
          for (int j = 0; j < DS; ++j) acc[g][i][j] = fma(x[g * DS + i], z[g * DS + j], acc[g][i][j]);
    }
  }
  if (MODE == kModePass1) {
    T vals[NG * NVG];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < DS; ++i)
#pragma unroll
        for (int j = 0; j < DS; ++j) vals[g * NVG + i * DS + j] = acc[g][i][j];
    block_reduce_store<NG, NVG, T>(vals, tpr, a.partials, L.groups_per_slice(), (size_t)by * gx + bx);
  }
}

template <typename T, int DS, int VW, int MODE>
__global__ void __launch_bounds__(kThreads) k_spmm(Layout L, SpmmArgs a) {
  const TermsSmem<T> terms = load_terms<T>(a.flips, a.n_flip, a.diags, a.n_diag);
  spmm_block<T, DS, VW, MODE>(L, a, terms, blockIdx.x, blockIdx.y, gridDim.x);
}

// ---------------------------------------------------------------- tiled SpMM
//
// Same result as k_spmm, organised around tiles of 2^kTileBits consecutive states of
// one slice (32 KB) held in shared memory. The own tile and, one after another, every
// partner tile tile ^ m_high that an active term needs are fetched with TMA bulk
// copies (cp.async.bulk, completion on an mbarrier) through a ring of slots, so later
// tiles stream in while the current one is consumed. Every flip term is then a
// shared-memory (or register) read; the diagonal is rebuilt per tile from a small
// table (TileDiag). The blocks walk the (slice, tile) pairs with one grid stride,
// slice by slice, so all SMs work on neighbouring tiles of one slice and partner
// tiles are mostly served from L2.

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bulk copy with an L2 eviction-priority policy (createpolicy value).
__device__ __forceinline__ void bulk_load_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                               uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, "
      "[%3], %4;\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Producer/consumer layout of the tiled SpMM: warps 8 and 9 issue TMA bulk copies
// into a ring of shared-memory slots; the consumer warps read them. A slot holds one
// 32 KB tile (kTileRows rows of a slice) plus, for the own tile, its row of the K
// table of the diagonal. Per tile the stage sequence is: own tile, each needed partner
// tile, then the W_{j-1} tile (if any). Full barriers (count 1, transaction bytes)
// and empty barriers (one arrival per consumer warp) order the ring.
constexpr int kConsumerWarps = (kTileRows >> kTileRegBits) * kTiledLanes / 32;
constexpr int kProducerWarps = 2;  // each issues the copies of every other ring slot
constexpr int kTiledThreads = (kConsumerWarps + kProducerWarps) * 32;
constexpr uint32_t kTileBytes = (uint32_t)kTileRows * kTiledLanes * 16;  // 32 KB
constexpr int kMaxStages = 8;
// Slot = tile + the A-table row of the diagonal (rounded to 128 bytes).
__host__ __device__ inline uint32_t tiled_slot_bytes(int n_entries, int elem) {
  return kTileBytes + ((uint32_t)(tile_diag_stride(n_entries, elem) * elem) + 127u) / 128u * 128u;
}

// Shared-memory records of the tiled SpMM's term tables. A pattern record carries its
// first term inline; `single` marks a pattern of one term with c_odd = c_even (one
// coefficient for the whole tile), the common case of a transverse field.
template <typename T>
struct alignas(16) PatS {
  uint32_t high;   // m_high: the partner tile is tile ^ high
  uint32_t flags;  // bit0 uniform activity, bit1/bit2 some c_odd/c_even nonzero
  int start, end;  // its terms
  uint32_t low0;   // m_low of its first term
  uint32_t single; // bit0: one term, c_odd = c_even; bit1: one term with m_low = 0
  T c0;            // c_odd of its first term
  T c1;            // c_even of its first term
};
template <typename T>
struct alignas(16) TermS {
  T co, ce;        // c_odd, c_even
  uint32_t low;    // m_low
};

template <typename T>
__host__ __device__ inline size_t tiled_smem_bytes(int n_pat, int n_terms, int n_entries, int stages) {
  size_t off = (size_t)stages * tiled_slot_bytes(n_entries, (int)sizeof(T));
  off += 2 * kMaxStages * 8 + 64;                  // full/empty barriers, control
  off += 2 * 8 * 16 * sizeof(T);                   // mixing coefficients of the lanes
  off += (size_t)kConsumerWarps * kTiledLanes * 16 * 8;  // reduction scratch
  off = (off + 15) / 16 * 16;
  off += (size_t)n_pat * sizeof(PatS<T>);          // pattern records
  off += (size_t)kTileRows * sizeof(T);            // low table of the diagonal
  off += (size_t)n_terms * sizeof(TermS<T>);       // term records
  return off + 64;
}

// First pattern >= p that tile tix needs (uniform patterns may be inactive).
template <typename T>
__device__ __forceinline__ int tiled_next(int p, int npat, uint32_t tix, const PatS<T>* pat) {
  for (; p < npat; ++p) {
    const uint32_t f = pat[p].flags;
    if (!(f & 1u)) return p;
    const bool odd = (__popc(tix & pat[p].high) & 1) != 0;
    if (odd ? (f & 2u) : (f & 4u)) return p;
  }
  return p;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
// Named barrier over the consumer warps with an OR of `pred` (bar.red.or).
__device__ __forceinline__ bool consumers_sync_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(kConsumerWarps * 32)
      : "memory");
  return r != 0;
}
// Bounded wait that also gives up when another thread has raised the abort flag.
__device__ __forceinline__ bool ring_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < (1u << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

// In-tile flip whose partner rows belong to the same thread: the thread's rows
// rg + RG m (m = 0..7) form a subcube over the top three tile bits, so a mask with
// no bit below log2(RG) maps row m to row m ^ K of the same thread.
template <int K, int RG, bool UNI, typename T, int VW, int RPT>
__device__ __forceinline__ void reg_flip(T (&y)[RPT][VW], const T (&xo)[RPT][VW], int rg, uint32_t ml,
                                         T co, T ce) {
  if constexpr (K >= RPT) return;
  if (UNI || co == ce) {
#pragma unroll
    for (int m = 0; m < RPT; ++m)
#pragma unroll
      for (int v = 0; v < VW; ++v) y[m][v] = fma(co, xo[(m ^ K) & (RPT - 1)][v], y[m][v]);
    return;
  }
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    const uint32_t r = (uint32_t)(rg + RG * m);
    const T c = (__popc(r & ml) & 1) ? co : ce;
#pragma unroll
    for (int v = 0; v < VW; ++v) y[m][v] = fma(c, xo[(m ^ K) & (RPT - 1)][v], y[m][v]);
  }
}

// Rows of a consumer thread and their partners: row rg + RG m (m = 0..7) of a tile sits
// at element offset rgoff + m * kStep (rgoff = rg * BS + lane * VW, kStep = RG * BS,
// both powers of two apart), so under an in-tile mask ml = (mh << log2 RG) | mlow its
// partner row rg ^ mlow + RG (m ^ mh) sits at (rgoff ^ mlow * BS | mh * kStep) ^ m * kStep.
// With mh = 0 that is a base plus a constant per row.
template <int RG, int BS>
__device__ __forceinline__ int partner_base(int rgoff, uint32_t ml) {
  return (rgoff ^ (int)((ml & (uint32_t)(RG - 1)) * BS)) | (int)((ml / RG) * (uint32_t)(RG * BS));
}

// Rows m and m ^ K (K a register-row bit of mh) of this thread for a parity-only term:
// the pair's active row a (parity p0 ^ parity(a & mh) selects the nonzero coefficient)
// loads its partner row once; y[a] += c * partner, y[other] += 0 * partner.
template <int K, typename T, int VW, int RPT>
__device__ __forceinline__ void pair_rows(T (&y)[RPT][VW], const T* P, int x, int kStep, uint32_t mh, uint32_t p0,
                                          T co, T ce) {
  if constexpr (K >= RPT) return;
  const T c = co != (T)0 ? co : ce;
  const uint32_t want = co != (T)0 ? 1u : 0u;  // the parity with the nonzero coefficient
  if (mh == (uint32_t)K) {
    // one register-row bit in the mask: every pair (m, m ^ K) with m & K = 0 has its
    // active row on the same side, so the side, its coefficients and the partner
    // offset are chosen once
    const bool lo = p0 == want;
    const T cl = lo ? c : (T)0, ch = lo ? (T)0 : c;
    const int xs = lo ? x : (x ^ (K * kStep));
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      if (m & K) continue;
      T xp[VW];
      VecIO<T, VW>::ld_rw(xp, P + (xs ^ (m * kStep)));
#pragma unroll
      for (int v = 0; v < VW; ++v) {
        y[m][v] = fma(cl, xp[v], y[m][v]);
        y[m ^ K][v] = fma(ch, xp[v], y[m ^ K][v]);
      }
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    if (m & K) continue;
    const bool lo = ((p0 ^ (uint32_t)__popc((uint32_t)m & mh)) & 1u) == want;
    const int a = lo ? m : (m ^ K);
    T xp[VW];
    VecIO<T, VW>::ld_rw(xp, P + (x ^ (a * kStep)));
    const T cl = lo ? c : (T)0, ch = lo ? (T)0 : c;
#pragma unroll
    for (int v = 0; v < VW; ++v) {
      y[m][v] = fma(cl, xp[v], y[m][v]);
      y[m ^ K][v] = fma(ch, xp[v], y[m ^ K][v]);
    }
  }
}

// y[m] += c * P[row m ^ ml] for one term whose coefficient depends on the parity of
// (row0 + row) & mparity (c_odd / c_even), rows of this thread.
// UNI: every term of the Hamiltonian has c_odd = c_even (a separate instantiation,
// so the parity-dependent code below is not compiled into it).
template <typename T, int VW, int RPT, int RG, int BS, bool UNI>
__device__ __forceinline__ void apply_term(T (&y)[RPT][VW], int rgoff, int rg, const T* P, uint32_t ml,
                                           uint32_t mparity, T co, T ce, uint32_t row0) {
  constexpr int kStep = RG * BS;
  const int x = partner_base<RG, BS>(rgoff, ml);
  const bool flat = ml < (uint32_t)RG;  // mh = 0: partner offsets x + m * kStep
  if (UNI || co == ce) {
    if (flat) {
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        T xp[VW];
        VecIO<T, VW>::ld_rw(xp, P + x + m * kStep);
#pragma unroll
        for (int v = 0; v < VW; ++v) y[m][v] = fma(co, xp[v], y[m][v]);
      }
    } else {
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        T xp[VW];
        VecIO<T, VW>::ld_rw(xp, P + (x ^ (m * kStep)));
#pragma unroll
        for (int v = 0; v < VW; ++v) y[m][v] = fma(co, xp[v], y[m][v]);
      }
    }
  } else if constexpr (!UNI) {
    // Row row0 + rg + RG m is row0 | rg | m << log2(RG) (disjoint bits), so its parity
    // under mparity is p0 (that of row0 | rg) xor the parity of m & mh. With mh = 0 the
    // coefficient is the same for all of this thread's rows: one test per term.
    const uint32_t mh = (mparity / (uint32_t)RG) & (uint32_t)(RPT - 1);
    const uint32_t p0 = (uint32_t)__popc((row0 + (uint32_t)rg) & mparity) & 1u;
    if (mh == 0u) {
      // the same coefficient for all of this thread's rows; where it differs across the
      // warp's lanes they all run the term (a zero coefficient on the others) rather
      // than diverge, and a warp none of whose lanes has it skips the term
      const T c = p0 ? co : ce;
      if (__any_sync(0xffffffffu, c != (T)0)) {
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          T xp[VW];
          VecIO<T, VW>::ld_rw(xp, P + (x ^ (m * kStep)));
#pragma unroll
          for (int v = 0; v < VW; ++v) y[m][v] = fma(c, xp[v], y[m][v]);
        }
      }
    } else if (co == (T)0 || ce == (T)0) {
      // Parity-only coefficient (one of c_odd, c_even zero, e.g. XX + YY with J^x = J^y):
      // rows m and m ^ hb (hb the lowest bit of mh) have opposite parities, so exactly one
      // of each such pair is active. One load serves the pair: the active row's partner,
      // added to the active row (the other row's product is with zero).
      switch (mh & (0u - mh)) {
        case 1u: pair_rows<1, T, VW, RPT>(y, P, x, kStep, mh, p0, co, ce); break;
        case 2u: pair_rows<2, T, VW, RPT>(y, P, x, kStep, mh, p0, co, ce); break;
        default: pair_rows<4, T, VW, RPT>(y, P, x, kStep, mh, p0, co, ce); break;
      }
    } else {
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        const T c = ((p0 ^ (uint32_t)__popc((uint32_t)m & mh)) & 1u) ? co : ce;
        if (c != (T)0) {
          T xp[VW];
          VecIO<T, VW>::ld_rw(xp, P + (x ^ (m * kStep)));
#pragma unroll
          for (int v = 0; v < VW; ++v) y[m][v] = fma(c, xp[v], y[m][v]);
        }
      }
    }
  }
}

// Two uniform-coefficient terms at once (loads of both issued before their FMAs).
template <typename T, int VW, int RPT, int RG, int BS>
__device__ __forceinline__ void apply2_uniform(T (&y)[RPT][VW], int rgoff, const T* PA, uint32_t mlA, T cA,
                                               const T* PB, uint32_t mlB, T cB) {
  constexpr int kStep = RG * BS;
  const int xa = partner_base<RG, BS>(rgoff, mlA), xb = partner_base<RG, BS>(rgoff, mlB);
  if (mlA < (uint32_t)RG && mlB < (uint32_t)RG) {
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      T a[VW], b[VW];
      VecIO<T, VW>::ld_rw(a, PA + xa + m * kStep);
      VecIO<T, VW>::ld_rw(b, PB + xb + m * kStep);
#pragma unroll
      for (int v = 0; v < VW; ++v) y[m][v] = fma(cB, b[v], fma(cA, a[v], y[m][v]));
    }
  } else {
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      T a[VW], b[VW];
      VecIO<T, VW>::ld_rw(a, PA + (xa ^ (m * kStep)));
      VecIO<T, VW>::ld_rw(b, PB + (xb ^ (m * kStep)));
#pragma unroll
      for (int v = 0; v < VW; ++v) y[m][v] = fma(cB, b[v], fma(cA, a[v], y[m][v]));
    }
  }
}

// Pairable partner tiles (TiledTerms::n_pair): for a tile, the groups of one high spin h
// whose h is down (zm, bit q = pattern q + 1) and up (om). The i-th stage of the block:
// down and up groups alternate (z_0, o_0, z_1, o_1, ..), then the rest of the longer list.
__device__ __forceinline__ int pair_pattern(int i, uint32_t zm, uint32_t om) {
  const int nz = __popc(zm), no = __popc(om), mn = nz < no ? nz : no;
  uint32_t m;
  int k;
  if (i < 2 * mn) {
    m = (i & 1) ? om : zm;
    k = i >> 1;
  } else {
    m = nz > no ? zm : om;
    k = i - mn;
  }
  for (; k > 0; --k) m &= m - 1u;
  return __ffs((int)m);
}

// Term i of both groups hops the same in-tile spin l with h (parity-only coefficient,
// active where l and h differ): with h down in PZ and up in PO, a row whose spin l is up
// takes PZ's term and a row whose spin l is down PO's, so every row loads once per l.
template <int K, typename T, int VW, int RPT>
__device__ __forceinline__ void paired_reg(T (&y)[RPT][VW], const T* PZ, const T* PO, int x, int kStep, T cz,
                                           T co) {
  if constexpr (K >= RPT) return;
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    T xp[VW];
    VecIO<T, VW>::ld_rw(xp, ((m & K) ? PZ : PO) + (x ^ (m * kStep)));
    const T c = (m & K) ? cz : co;
#pragma unroll
    for (int v = 0; v < VW; ++v) y[m][v] = fma(c, xp[v], y[m][v]);
  }
}
template <typename T, int VW, int RPT, int RG, int BS>
__device__ __forceinline__ void apply_paired(T (&y)[RPT][VW], int rgoff, int rg, const T* PZ, const T* PO,
                                             const TermS<T>* tz, const TermS<T>* to, int nt) {
  constexpr int kStep = RG * BS;
  for (int i = 0; i < nt; ++i) {
    const uint32_t ml = tz[i].low;
    const T cz = tz[i].co, co = to[i].co;
    const int x = partner_base<RG, BS>(rgoff, ml);
    if (ml < (uint32_t)RG) {  // spin l is a bit of rg: the same for all of this thread's rows
      const bool up = ((uint32_t)rg & ml) != 0u;
      const T* P = up ? PZ : PO;
      const T c = up ? cz : co;
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        T xp[VW];
        VecIO<T, VW>::ld_rw(xp, P + x + m * kStep);
#pragma unroll
        for (int v = 0; v < VW; ++v) y[m][v] = fma(c, xp[v], y[m][v]);
      }
    } else {
      switch (ml / (uint32_t)RG) {
        case 1u: paired_reg<1, T, VW, RPT>(y, PZ, PO, x, kStep, cz, co); break;
        case 2u: paired_reg<2, T, VW, RPT>(y, PZ, PO, x, kStep, cz, co); break;
        default: paired_reg<4, T, VW, RPT>(y, PZ, PO, x, kStep, cz, co); break;
      }
    }
  }
}

// Diagonal of H on this thread's RPT rows rg + RG m of a tile, from the tile's A-table
// row hk (TileDiag): low[r] + sum_q A_q (-1)^popc(q & m), one RPT-point Walsh-Hadamard
// transform of the A_q.
template <typename T, int RPT, int RG>
__device__ __forceinline__ void tile_diagonal(T (&dg)[RPT], const T* low, const T* hk, int rg,
                                              const TileDiag& td) {
  static_assert(RPT == (1 << kTileRegBits) && RG == (1 << kTileRegShift), "register rows per thread");
  T A[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) A[q] = hk[td.off[q] + (((td.dep >> q) & 1u) ? rg : 0)];
#pragma unroll
  for (int len = 1; len < RPT; len <<= 1)
#pragma unroll
    for (int i = 0; i < RPT; ++i)
      if (!(i & len)) {
        const T u = A[i], w = A[i | len];
        A[i] = u + w;
        A[i | len] = u - w;
      }
#pragma unroll
  for (int m = 0; m < RPT; ++m) dg[m] = low[rg + RG * m] + A[m];
}

template <typename T, int DS, int MODE, bool UNI = false>
__global__ void __launch_bounds__(kTiledThreads, 1) k_spmm_tiled(Layout L, SpmmArgs a) {
  constexpr int VW = 16 / (int)sizeof(T);
  constexpr int LPR = kTiledLanes;          // 16-byte vectors per row
  constexpr int BS = VW * LPR;              // elements per row of a slice
  // HG: a bath-vector group is wider than one lane's 16-byte vector (float64 with
  // d_s = 4: the group is the whole 32-byte row, half in each of the row's two lanes).
  // Its mixing and partial sums then take the other lane's half by a shuffle.
  constexpr bool HG = DS > VW;
  static_assert(!HG || DS == VW * LPR, "a wide group spans exactly the lanes of a row");
  constexpr int NG = HG ? 1 : VW / DS;
  constexpr int NVG = DS * DS;
  constexpr int NV = HG ? DS * VW : NG * NVG;  // partial sums per thread
  constexpr int NVC = HG ? NVG : NV;           // mixing coefficients per lane
  constexpr int RG = kConsumerWarps * 32 / LPR;  // row groups
  constexpr int RGL = (RG >= 256) ? 8 : (RG >= 128) ? 7 : (RG >= 64) ? 6 : 5;  // log2(RG)
  constexpr int RPT = kTileRows / RG;            // rows per consumer thread
  const int kStages = a.stages;
  static_assert(RPT == (1 << kTileRegBits), "rows per consumer thread");
  static_assert((1 << RGL) == RG && RGL == kTileRegShift, "row groups are the low tile bits");
  extern __shared__ __align__(128) unsigned char smem[];
  const TiledTerms& tt = a.tiled;
  const int npat = tt.n_pat, nterm = tt.n_terms, npair = tt.n_pair;
  const int hstride = tile_diag_stride(tt.dg.n_entries, (int)sizeof(T));
  const uint32_t kSlotBytes = tiled_slot_bytes(tt.dg.n_entries, (int)sizeof(T));
  unsigned char* const ring = smem;
  uint64_t* const full = reinterpret_cast<uint64_t*>(smem + (size_t)kStages * kSlotBytes);
  uint64_t* const empty = full + kMaxStages;
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(empty + kMaxStages);
  T* const s_mz = reinterpret_cast<T*>(smem + (size_t)kStages * kSlotBytes + 2 * kMaxStages * 8 + 64);
  T* const s_cp = s_mz + 8 * 16;
  double* const red = reinterpret_cast<double*>(s_cp + 8 * 16);
  size_t off = (size_t)(reinterpret_cast<unsigned char*>(red + kConsumerWarps * kTiledLanes * 16) - smem);
  off = (off + 15) / 16 * 16;
  PatS<T>* const pat = reinterpret_cast<PatS<T>*>(smem + off);
  T* const s_low = reinterpret_cast<T*>(pat + npat);
  TermS<T>* const term = reinterpret_cast<TermS<T>*>(s_low + kTileRows);

  for (int i = threadIdx.x; i < npat; i += blockDim.x) {
    PatS<T> r;
    r.high = tt.pat_high[i];
    r.flags = tt.pat_flags[i];
    r.start = tt.pat_start[i];
    r.end = tt.pat_start[i + 1];
    const bool any = r.start < r.end;
    r.low0 = any ? tt.term_low[r.start] : 0u;
    r.c0 = any ? (T)tt.term_odd[r.start] : (T)0;
    r.c1 = any ? (T)tt.term_even[r.start] : (T)0;
    const bool one = r.end - r.start == 1;
    r.single = ((one && tt.term_odd[r.start] == tt.term_even[r.start]) ? 1u : 0u) |
               ((one && tt.term_low[r.start] == 0u) ? 2u : 0u);
    pat[i] = r;
  }
  for (int i = threadIdx.x; i < nterm; i += blockDim.x) {
    TermS<T> r;
    r.co = (T)tt.term_odd[i];
    r.ce = (T)tt.term_even[i];
    r.low = tt.term_low[i];
    term[i] = r;
  }
  for (int i = threadIdx.x; i < kTileRows; i += blockDim.x) s_low[i] = (T)tt.dg.low[i];
  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kConsumerWarps);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5;
  const int tile_log = L.n_bits - kTileBits;  // tiles per slice = 2^tile_log
  const int64_t n_tiles = (int64_t)L.n_slices << tile_log;
  const uint32_t tile_mask = (uint32_t)(((int64_t)1 << tile_log) - 1);
  const bool has_prev = a.w_prev != nullptr;
  // every partner pattern is needed by every tile: the stage sequence is fixed
  const bool all_active = tt.all_active != 0;
  const bool partners_flat = tt.partners_flat != 0;
  const int n_reg0 = tt.n_reg0;

  if (warp >= kConsumerWarps) {
    // ------------------------------------------------ producers (lane 0 of each)
    // Both walk the whole stage sequence; producer q issues the stages with
    // seq % kProducerWarps == q (the ring depth is a multiple of kProducerWarps, so
    // each owns fixed slots).
    if ((threadIdx.x & 31) != 0) return;
    const uint32_t q = (uint32_t)(warp - kConsumerWarps);
    // W_j tiles are reused as partners of neighbouring tiles: keep them in L2;
    // W_{j-1} tiles are read once: let them leave first.
    const uint64_t keep = policy_evict_last();
    const uint64_t stream = policy_evict_first();
    const uint32_t hk_bytes = (uint32_t)hstride * (uint32_t)sizeof(T);
    const T* const hk_table = reinterpret_cast<const T*>(a.tile_k);
    // stage counter kept as (slot, round) so no division by the runtime ring depth
    uint32_t seq = 0, round = 0;
    int slot = 0;
    bool stop = false;
    for (int64_t gt = blockIdx.x; gt < n_tiles && !stop; gt += gridDim.x) {
      const int slice = (int)(gt >> tile_log);
      const uint32_t ut = tt.tile_order[(uint32_t)gt & tile_mask];
      const size_t soff = (size_t)slice * L.D * BS;
      const T* W = reinterpret_cast<const T*>(a.w) + soff;
      const T* Wp = has_prev ? reinterpret_cast<const T*>(a.w_prev) + soff : nullptr;
      uint32_t zm = 0u, om = 0u;  // pairable groups with their high spin down / up here
      for (int i = 0; i < npair; ++i) {
        if (ut & pat[1 + i].high) om |= 1u << i;
        else zm |= 1u << i;
      }
      // stage kinds: -1 = own, -2 = W_{j-1}, p >= 1 = partner pattern p
      int kind = -1;
      int pi = 0;  // pairable stages issued
      while (true) {
        if (seq % kProducerWarps == q) {
          if (round > 0 && !ring_wait(&empty[slot], (round - 1u) & 1u, abort_flag)) {
            stop = true;
            break;
          }
          unsigned char* dst = ring + (size_t)slot * kSlotBytes;
          fence_proxy_async();
          if (kind == -1) {
            mbar_expect_tx(&full[slot], kTileBytes + hk_bytes);
            bulk_load_hint(dst, W + ((size_t)ut << kTileBits) * BS, kTileBytes, &full[slot], keep);
            bulk_load_hint(dst + kTileBytes, hk_table + (size_t)ut * hstride, hk_bytes, &full[slot], keep);
          } else if (kind == -2) {
            mbar_expect_tx(&full[slot], kTileBytes);
            bulk_load_hint(dst, Wp + ((size_t)ut << kTileBits) * BS, kTileBytes, &full[slot], stream);
          } else {
            mbar_expect_tx(&full[slot], kTileBytes);
            bulk_load_hint(dst, W + ((size_t)(ut ^ pat[kind].high) << kTileBits) * BS, kTileBytes,
                           &full[slot], keep);
          }
        }
        ++seq;
        if (++slot == kStages) {
          slot = 0;
          ++round;
        }
        // next stage of this tile
        if (kind == -2) break;
        int p;
        if (pi < npair) {
          p = pair_pattern(pi++, zm, om);
        } else {
          const int from = kind <= npair ? npair + 1 : kind + 1;
          p = all_active ? from : tiled_next(from, npat, ut, pat);
        }
        if (p < npat) {
          kind = p;
        } else if (has_prev) {
          kind = -2;
        } else {
          break;
        }
      }
    }
    if (stop) atomicOr(a.err, 1u);
    return;
  }

  // -------------------------------------------------- consumers
  const int lane = threadIdx.x % LPR;  // 16-byte column chunk of a row
  const int rg = threadIdx.x / LPR;    // row group: rows rg + RG*m
  constexpr int kStep = RG * BS;        // elements between a thread's rows
  const int rgoff = rg * BS + lane * VW;  // element offset of its first row in a tile
  const bool leader = (threadIdx.x & 31) == 0;
  // next unreleased ring stage as (slot, phase parity): no division by the runtime depth
  int rslot = 0;
  uint32_t rphase = 0;
  bool aborted = false;
  // Waits for the ring slot `ahead` (0 or 1) stages past the next unreleased one.
  auto acquire = [&](const unsigned char*& slot_ptr, int ahead) -> bool {
    int slot = rslot + ahead;
    uint32_t ph = rphase;
    if (slot >= kStages) {
      slot -= kStages;
      ph ^= 1u;
    }
    if (!ring_wait(&full[slot], ph, abort_flag)) return false;
    slot_ptr = ring + (size_t)slot * kSlotBytes;
    return true;
  };
  auto release = [&]() {
    __syncwarp();
    if (leader) mbar_arrive(&empty[rslot]);
    if (++rslot == kStages) {
      rslot = 0;
      rphase ^= 1u;
    }
  };
  auto release2 = [&]() {  // the next two stages
    __syncwarp();
    const int s2 = rslot + 1 == kStages ? 0 : rslot + 1;
    if (leader) {
      mbar_arrive(&empty[rslot]);
      mbar_arrive(&empty[s2]);
    }
    if (s2 < rslot) rphase ^= 1u;
    rslot = s2 + 1;
    if (rslot == kStages) {
      rslot = 0;
      rphase ^= 1u;
    }
  };
  // Partials of W_j^T Z of this block for one slice (zero for a slice it has no tile
  // of); every (slice, block) entry is written once.
  const int gs = BS / DS;
  auto partial_base = [&](int slice) -> size_t {
    return ((size_t)(slice * gridDim.x + blockIdx.x) * gs + (HG ? 0 : (size_t)threadIdx.x * NG)) * NVG;
  };
  // Entry e of a lane's partial sums in its group's DS x DS block: (i, j) = (e / VW,
  // lane * VW + e % VW) for wide groups (lane = threadIdx.x here, < LPR).
  auto partial_entry = [&](int e) -> int {
    return HG ? (e / VW) * DS + (int)threadIdx.x * VW + e % VW : e;
  };

  T acc[NV];  // W_j^T Z sums of this lane's bath-vector groups
#pragma unroll
  for (int e = 0; e < NV; ++e) acc[e] = (T)0;
  T* __restrict__ Z = nullptr;
  int cur = -1;       // slice of the tiles in progress
  int unwritten = 0;  // slices [unwritten, n_slices) have no partials yet

  // The consumers walk the same (slice, tile) sequence as the producers. At every
  // change of slice (and at the end) they close the finished slice; every consumer
  // thread passes the same barriers, also after an abort.
  for (int64_t gt = blockIdx.x;; gt += gridDim.x) {
    const int slice = gt < n_tiles ? (int)(gt >> tile_log) : L.n_slices;
    if (slice != cur) {
      if (consumers_sync_or(aborted)) aborted = true;
      if (MODE == kModePass1 && !aborted) {
        if (cur >= 0) {
          // fixed-order reduction: shuffles within a warp (in T, like the per-thread
          // sums), then the warps in order in float64
          T v[NV];
#pragma unroll
          for (int e = 0; e < NV; ++e) {
            T x = acc[e];
#pragma unroll
            for (int o = LPR; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            v[e] = x;
          }
          if ((threadIdx.x & 31) < LPR) {
#pragma unroll
            for (int e = 0; e < NV; ++e) red[(warp * LPR + lane) * 16 + e] = (double)v[e];
          }
          consumers_sync_or(false);
          if (threadIdx.x < LPR) {
            const size_t base = partial_base(cur);
            for (int e = 0; e < NV; ++e) {
              double sum = 0.0;
              for (int w = 0; w < kConsumerWarps; ++w) sum += red[(w * LPR + threadIdx.x) * 16 + e];
              a.partials[base + partial_entry(e)] = sum;
            }
          }
          unwritten = cur + 1;
        }
        if (threadIdx.x < LPR)
          for (int c = unwritten; c < slice; ++c)
            for (int e = 0; e < NV; ++e) a.partials[partial_base(c) + partial_entry(e)] = 0.0;
        unwritten = slice;
      }
      if (slice >= L.n_slices) break;
      cur = slice;
      Z = reinterpret_cast<T*>(a.z) + (size_t)slice * L.D * BS;
      consumers_sync_or(false);  // the previous slice's coefficients have been read
      if (MODE != kModeApply && threadIdx.x < LPR * NVC) {
        const int ln = threadIdx.x / NVC, e = threadIdx.x % NVC;
        const size_t gidx = (size_t)((slice * BS + ln * VW) / DS) * NVG + e;
        s_mz[ln * 16 + e] = (T)a.mz[gidx];
        s_cp[ln * 16 + e] = has_prev ? (T)a.cp[gidx] : (T)0;
      }
      consumers_sync_or(false);
#pragma unroll
      for (int e = 0; e < NV; ++e) acc[e] = (T)0;
    }
    if (aborted) continue;

    const uint32_t ut = tt.tile_order[(uint32_t)gt & tile_mask];
    const uint32_t row0 = ut << kTileBits;
    const unsigned char* sp;
    // own tile: diagonal and in-tile terms
    if (!acquire(sp, 0)) {
      aborted = true;
      continue;
    }
    const T* own = reinterpret_cast<const T*>(sp);
    T xo[RPT][VW], y[RPT][VW];
    {
      T dg[RPT];
      tile_diagonal<T, RPT, RG>(dg, s_low, reinterpret_cast<const T*>(sp + kTileBytes), rg, tt.dg);
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        VecIO<T, VW>::ld_rw(xo[m], own + rgoff + m * kStep);
#pragma unroll
        for (int v = 0; v < VW; ++v) y[m][v] = dg[m] * xo[m][v];
      }
    }
    const int t1 = pat[0].end, tr = pat[0].start + n_reg0;
    for (int t = pat[0].start; t < tr; ++t) {  // masks on the register rows only
      const TermS<T> d = term[t];
      switch (d.low >> RGL) {
        case 1: reg_flip<1, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
        case 2: reg_flip<2, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
        case 3: reg_flip<3, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
        case 4: reg_flip<4, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
        case 5: reg_flip<5, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
        case 6: reg_flip<6, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
        default: reg_flip<7, RG, UNI>(y, xo, rg, d.low, d.co, d.ce); break;
      }
    }
    for (int t = tr; t < t1;) {
      const TermS<T> d = term[t];
      if (d.co == d.ce && t + 1 < t1) {
        const TermS<T> d2 = term[t + 1];
        if (d2.co == d2.ce) {
          apply2_uniform<T, VW, RPT, RG, BS>(y, rgoff, own, d.low, d.co, own, d2.low, d2.co);
          t += 2;
          continue;
        }
      }
      apply_term<T, VW, RPT, RG, BS, UNI>(y, rgoff, rg, own, d.low, d.low, d.co, d.ce, 0u);
      ++t;
    }
    release();
    // the terms of one partner pattern A, copied to P (any coefficients)
    auto pattern_terms = [&](const PatS<T>& A, const T* P) {
      const uint32_t hi_bits = A.high << kTileBits;
      for (int t = A.start; t < A.end;) {
        const TermS<T> d = term[t];
        if (d.co == d.ce && t + 1 < A.end) {
          const TermS<T> d2 = term[t + 1];
          if (d2.co == d2.ce) {
            apply2_uniform<T, VW, RPT, RG, BS>(y, rgoff, P, d.low, d.co, P, d2.low, d2.co);
            t += 2;
            continue;
          }
        }
        apply_term<T, VW, RPT, RG, BS, UNI>(y, rgoff, rg, P, d.low, d.low | hi_bits, d.co, d.ce, row0);
        ++t;
      }
    };
    if constexpr (!UNI) {
      // pairable partner tiles: a group with its high spin down and one with it up
      // together, then the rest of the longer list one by one
      if (npair > 0) {
        uint32_t zm = 0u, om = 0u;
        for (int q = 0; q < npair; ++q) {
          if (ut & pat[1 + q].high) om |= 1u << q;
          else zm |= 1u << q;
        }
        const int nz = __popc(zm), no = __popc(om);
        const int n2 = 2 * (nz < no ? nz : no);
        for (int i = 0; i < npair;) {
          const PatS<T> A = pat[pair_pattern(i, zm, om)];
          if (i < n2) {
            const PatS<T> B = pat[pair_pattern(i + 1, zm, om)];
            const unsigned char* sp2;
            if (!acquire(sp, 0) || !acquire(sp2, 1)) {
              aborted = true;
              break;
            }
            apply_paired<T, VW, RPT, RG, BS>(y, rgoff, rg, reinterpret_cast<const T*>(sp),
                                             reinterpret_cast<const T*>(sp2), term + A.start, term + B.start,
                                             A.end - A.start);
            release2();
            i += 2;
          } else {
            if (!acquire(sp, 0)) {
              aborted = true;
              break;
            }
            pattern_terms(A, reinterpret_cast<const T*>(sp));
            release();
            ++i;
          }
        }
        if (aborted) continue;
      }
    }
    // partner tiles; two single-term patterns are consumed together so their
    // shared-memory loads overlap
    if (partners_flat) {
      // one uniform term per partner tile, partner row = same row: no term records
      int p = 1;
      for (; p + 1 < npat; p += 2) {
        const T cA = pat[p].c0, cB = pat[p + 1].c0;
        const unsigned char* sb;
        if (!acquire(sp, 0) || !acquire(sb, 1)) {
          aborted = true;
          break;
        }
        const T* PA = reinterpret_cast<const T*>(sp) + rgoff;
        const T* PB = reinterpret_cast<const T*>(sb) + rgoff;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          T u[VW], w[VW];
          VecIO<T, VW>::ld_rw(u, PA + m * kStep);
          VecIO<T, VW>::ld_rw(w, PB + m * kStep);
#pragma unroll
          for (int v = 0; v < VW; ++v) y[m][v] = fma(cB, w[v], fma(cA, u[v], y[m][v]));
        }
        release2();
      }
      if (!aborted && p < npat) {
        const T cA = pat[p].c0;
        if (!acquire(sp, 0)) {
          aborted = true;
        } else {
          const T* PA = reinterpret_cast<const T*>(sp) + rgoff;
#pragma unroll
          for (int m = 0; m < RPT; ++m) {
            T u[VW];
            VecIO<T, VW>::ld_rw(u, PA + m * kStep);
#pragma unroll
            for (int v = 0; v < VW; ++v) y[m][v] = fma(cA, u[v], y[m][v]);
          }
          release();
        }
      }
    } else
    for (int p = all_active ? npair + 1 : tiled_next(npair + 1, npat, ut, pat); p < npat;) {
      const int pn = all_active ? p + 1 : tiled_next(p + 1, npat, ut, pat);
      const PatS<T> A = pat[p];
      if (A.single & 2u) {
        // One term whose partner row is the same row (m_low = 0): its coefficient is
        // the same for every row of this tile (the parity of its mask is that of the
        // tile bits). Two such partner tiles are consumed together when they follow
        // each other.
        const T cA = (__popc(ut & A.high) & 1) ? A.c0 : A.c1;
        if (pn < npat && (pat[pn].single & 2u)) {
          const PatS<T> Bq = pat[pn];
          const T cB = (__popc(ut & Bq.high) & 1) ? Bq.c0 : Bq.c1;
          const unsigned char* sp2;
          if (!acquire(sp, 0) || !acquire(sp2, 1)) {
            aborted = true;
            break;
          }
          apply2_uniform<T, VW, RPT, RG, BS>(y, rgoff, reinterpret_cast<const T*>(sp), 0u, cA,
                                             reinterpret_cast<const T*>(sp2), 0u, cB);
          release2();
          p = all_active ? pn + 1 : tiled_next(pn + 1, npat, ut, pat);
          continue;
        }
        if (!acquire(sp, 0)) {
          aborted = true;
          break;
        }
        const T* PA = reinterpret_cast<const T*>(sp) + rgoff;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          T u[VW];
          VecIO<T, VW>::ld_rw(u, PA + m * kStep);
#pragma unroll
          for (int v = 0; v < VW; ++v) y[m][v] = fma(cA, u[v], y[m][v]);
        }
        release();
        p = pn;
        continue;
      }
      if (pn < npat && A.single) {
        const PatS<T> Bq = pat[pn];
        if (Bq.single) {
          const unsigned char* sp2;
          if (!acquire(sp, 0) || !acquire(sp2, 1)) {
            aborted = true;
            break;
          }
          apply2_uniform<T, VW, RPT, RG, BS>(y, rgoff, reinterpret_cast<const T*>(sp), A.low0, A.c0,
                                             reinterpret_cast<const T*>(sp2), Bq.low0, Bq.c0);
          release();
          release();
          p = all_active ? pn + 1 : tiled_next(pn + 1, npat, ut, pat);
          continue;
        }
      }
      if (!acquire(sp, 0)) {
        aborted = true;
        break;
      }
      pattern_terms(A, reinterpret_cast<const T*>(sp));
      release();
      p = pn;
    }
    if (aborted) continue;
    // Z = (H W) M + W_prev Cp, row by row, with the W_j^T Z partial sums
    const T* Pp = nullptr;
    if (has_prev) {
      if (!acquire(sp, 0)) {
        aborted = true;
        continue;
      }
      Pp = reinterpret_cast<const T*>(sp);
    }
    T* const zrow = Z + (size_t)row0 * BS + rgoff;  // this thread's first row of the tile
    if constexpr (MODE == kModeApply) {  // Z = H W
#pragma unroll
      for (int m = 0; m < RPT; ++m) VecIO<T, VW>::st_cs(zrow + m * kStep, y[m]);
    } else {
      // this lane's mixing coefficients, read per tile (broadcast shared-memory reads)
      // so they hold no registers while the partner tiles are consumed. M_j is upper
      // triangular (the inverse Cholesky factor, exact zeros below the diagonal), so
      // z = y M_j skips the zero products: the same fma chain, ended early.
      T mz[NVC], cp[NVC];
#pragma unroll
      for (int e = 0; e < NVC; ++e) {
        mz[e] = s_mz[lane * 16 + e];
        cp[e] = s_cp[lane * 16 + e];
      }
      if constexpr (HG) {
        // the row's DS columns: this lane holds columns lane*VW .. lane*VW+VW-1; the whole
        // row of Z is formed (static register indices) and the lane keeps its half
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          T yf[DS], xf[DS], zf[DS];
#pragma unroll
          for (int v = 0; v < VW; ++v) {
            const T yo = __shfl_xor_sync(0xffffffffu, y[m][v], 1);
            const T xx = __shfl_xor_sync(0xffffffffu, xo[m][v], 1);
            yf[v] = lane == 0 ? y[m][v] : yo;
            yf[VW + v] = lane == 0 ? yo : y[m][v];
            xf[v] = lane == 0 ? xo[m][v] : xx;
            xf[VW + v] = lane == 0 ? xx : xo[m][v];
          }
#pragma unroll
          for (int j = 0; j < DS; ++j) {
            T t = (T)0;
#pragma unroll
            for (int i = 0; i <= j; ++i) t = fma(yf[i], mz[i * DS + j], t);
            zf[j] = t;
          }
          if (has_prev) {
            T xp[VW], pf[DS];
            VecIO<T, VW>::ld_rw(xp, Pp + rgoff + m * kStep);
#pragma unroll
            for (int v = 0; v < VW; ++v) {
              const T po = __shfl_xor_sync(0xffffffffu, xp[v], 1);
              pf[v] = lane == 0 ? xp[v] : po;
              pf[VW + v] = lane == 0 ? po : xp[v];
            }
#pragma unroll
            for (int j = 0; j < DS; ++j) {
              T t = zf[j];
#pragma unroll
              for (int i = 0; i < DS; ++i) t = fma(pf[i], cp[i * DS + j], t);
              zf[j] = t;
            }
          }
          T z[VW];
#pragma unroll
          for (int v = 0; v < VW; ++v) z[v] = lane == 0 ? zf[v] : zf[VW + v];
          VecIO<T, VW>::st_cs(zrow + m * kStep, z);
          if (MODE == kModePass1) {
#pragma unroll
            for (int i = 0; i < DS; ++i)
#pragma unroll
              for (int jj = 0; jj < VW; ++jj) acc[i * VW + jj] = fma(xf[i], z[jj], acc[i * VW + jj]);
          }
        }
      } else
#pragma unroll
      for (int m = 0; m < RPT; ++m) {
        T z[VW];
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int j = 0; j < DS; ++j) {
            T t = (T)0;
#pragma unroll
            for (int i = 0; i <= j; ++i) t = fma(y[m][g * DS + i], mz[g * NVG + i * DS + j], t);
            z[g * DS + j] = t;
          }
        if (has_prev) {
          T xp[VW];
          VecIO<T, VW>::ld_rw(xp, Pp + rgoff + m * kStep);
#pragma unroll
          for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int j = 0; j < DS; ++j) {
              T t = z[g * DS + j];
#pragma unroll
              for (int i = 0; i < DS; ++i) t = fma(xp[g * DS + i], cp[g * NVG + i * DS + j], t);
              z[g * DS + j] = t;
            }
        }
        VecIO<T, VW>::st_cs(zrow + m * kStep, z);
        if (MODE == kModePass1) {
#pragma unroll
          for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int i = 0; i < DS; ++i)
#pragma unroll
              for (int j = 0; j < DS; ++j)
                acc[g * NVG + i * DS + j] = fma(xo[m][g * DS + i], z[g * DS + j], acc[g * NVG + i * DS + j]);
        }
      }
      if (has_prev) release();
    }
  }
  if (aborted && threadIdx.x == 0) atomicOr(a.err, 1u);
}

// ---------------------------------------------------------------- orthogonalisation

// Block (bx, by) of a gx x n_slices grid of the orthogonalisation (grid-stride rows as
// in spmm_block).
template <typename T, int DS, int VW, bool PASS1, bool COH = false>
__device__ __forceinline__ void orth_block(const Layout& L, const T* __restrict__ Wg, T* __restrict__ Zg,
                                           const double* cw, double* partials, T* psi, const double* e,
                                           int nb, int bx, int by, int gx) {
  constexpr int NG = VW / DS;
  constexpr int NVG = DS * DS;
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = by;
  const size_t soff = (size_t)slice * L.D * L.Bs + (size_t)lane * VW;
  const T* W = Wg + soff;
  T* Z = Zg + soff;
  const int g0 = (slice * L.Bs + lane * VW) / DS;
  const size_t bstride = (size_t)L.D * L.B;  // elements per psi block
  T c[NG][DS][DS];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < DS; ++i)
#pragma unroll
      for (int j = 0; j < DS; ++j) c[g][i][j] = (T)cw[(size_t)(g0 + g) * NVG + i * DS + j];
  T acc[NG][DS][DS];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < DS; ++i)
#pragma unroll
      for (int j = 0; j < DS; ++j) acc[g][i][j] = (T)0;
  // pass 2: this slice's E coefficients for all nb betas, as T, in shared memory
  extern __shared__ __align__(16) unsigned char smem_e[];
  T* sE = reinterpret_cast<T*>(smem_e);
  const int gs = L.groups_per_slice();
  if (!PASS1) {
    const int ngs = L.n_groups();
    for (int i = threadIdx.x; i < nb * gs * NVG; i += blockDim.x) {
      const int bi = i / (gs * NVG), rem = i % (gs * NVG);
      sE[i] = (T)e[(size_t)bi * ngs * NVG + (size_t)slice * gs * NVG + rem];
    }
    __syncthreads();
  }
  for (int64_t s = (int64_t)bx * rpb + rs; s < L.D; s += (int64_t)gx * rpb) {
    T x[VW], z[VW];
    ld_vec<T, VW, COH>(x, W + (size_t)s * L.Bs);
    VecIO<T, VW>::ld_rw(z, Z + (size_t)s * L.Bs);
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int j = 0; j < DS; ++j) {
        T t = z[g * DS + j];
#pragma unroll
        for (int i = 0; i < DS; ++i) t = fma(x[g * DS + i], c[g][i][j], t);
        z[g * DS + j] = t;
      }
    VecIO<T, VW>::st(Z + (size_t)s * L.Bs, z);
    if (PASS1) {
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int i = 0; i < DS; ++i)
#pragma unroll
          for (int j = 0; j < DS; ++j) acc[g][i][j] = fma(z[g * DS + i], z[g * DS + j], acc[g][i][j]);
    } else {
      for (int bi = 0; bi < nb; ++bi) {
        T* P = psi + bi * bstride + soff + (size_t)s * L.Bs;
        T p[VW];
        VecIO<T, VW>::ld_rw(p, P);
        const T* eb = sE + ((size_t)bi * gs + (size_t)lane * NG) * NVG;
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int j = 0; j < DS; ++j) {
            T t = p[g * DS + j];
#pragma unroll
            for (int i = 0; i < DS; ++i) t = fma(z[g * DS + i], eb[g * NVG + i * DS + j], t);
            p[g * DS + j] = t;
          }
        VecIO<T, VW>::st(P, p);
      }
    }
  }
  if (PASS1) {
    T vals[NG * NVG];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < DS; ++i)
#pragma unroll
        for (int j = 0; j < DS; ++j) vals[g * NVG + i * DS + j] = acc[g][i][j];
    block_reduce_store<NG, NVG, T>(vals, tpr, partials, L.groups_per_slice(), (size_t)by * gx + bx);
  }
}

template <typename T, int DS, int VW, bool PASS1>
__global__ void __launch_bounds__(kThreads) k_orth(Layout L, const T* __restrict__ Wg,
                                                   T* __restrict__ Zg, const double* cw,
                                                   double* partials, T* psi, const double* e,
                                                   int nb) {
  orth_block<T, DS, VW, PASS1>(L, Wg, Zg, cw, partials, psi, e, nb, blockIdx.x, blockIdx.y, gridDim.x);
}

// psi_beta = W_1 E_{1,beta} (start of pass 2).
template <typename T, int DS, int VW>
__global__ void __launch_bounds__(kThreads) k_psi_init(Layout L, const T* __restrict__ Wg,
                                                       T* psi, const double* e, int nb) {
  constexpr int NG = VW / DS;
  constexpr int NVG = DS * DS;
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = blockIdx.y;
  const size_t soff = (size_t)slice * L.D * L.Bs + (size_t)lane * VW;
  const int g0 = (slice * L.Bs + lane * VW) / DS;
  const size_t bstride = (size_t)L.D * L.B;
  const int ngs = L.n_groups();
  for (int64_t s = (int64_t)blockIdx.x * rpb + rs; s < L.D; s += (int64_t)gridDim.x * rpb) {
    T x[VW];
    VecIO<T, VW>::ld(x, Wg + soff + (size_t)s * L.Bs);
    for (int bi = 0; bi < nb; ++bi) {
      const double* eb = e + (size_t)bi * ngs * NVG;
      T p[VW];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int j = 0; j < DS; ++j) {
          T t = (T)0;
#pragma unroll
          for (int i = 0; i < DS; ++i) t = fma(x[g * DS + i], (T)eb[(size_t)(g0 + g) * NVG + i * DS + j], t);
          p[g * DS + j] = t;
        }
      VecIO<T, VW>::st(psi + bi * bstride + soff + (size_t)s * L.Bs, p);
    }
  }
}

// psi_beta += sum_{a < m} W_a E_{j0+a,beta} (pass 2, m kept basis blocks): each psi
// element is read and written once for m steps instead of once per step.
template <typename T, int DS, int VW>
__global__ void __launch_bounds__(kThreads) k_psi_batch(Layout L, PsiBatch wb, int m, T* psi,
                                                        const double* e, size_t estride, int nb) {
  constexpr int NG = VW / DS;
  constexpr int NVG = DS * DS;
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = blockIdx.y;
  const size_t soff = (size_t)slice * L.D * L.Bs + (size_t)lane * VW;
  const size_t bstride = (size_t)L.D * L.B;
  const int gs = L.groups_per_slice(), ngs = L.n_groups();
  // this slice's E coefficients, [a][beta][group][DS*DS], as T
  extern __shared__ __align__(16) unsigned char smem_e[];
  T* sE = reinterpret_cast<T*>(smem_e);
  const int per = nb * gs * NVG;
  for (int i = threadIdx.x; i < m * per; i += blockDim.x) {
    const int a = i / per, rem = i % per, bi = rem / (gs * NVG), r2 = rem % (gs * NVG);
    sE[i] = (T)e[(size_t)a * estride + (size_t)bi * ngs * NVG + (size_t)slice * gs * NVG + r2];
  }
  __syncthreads();
  for (int64_t s = (int64_t)blockIdx.x * rpb + rs; s < L.D; s += (int64_t)gridDim.x * rpb) {
    T x[kPsiBatchMax][VW];
#pragma unroll
    for (int a = 0; a < kPsiBatchMax; ++a)
      if (a < m) VecIO<T, VW>::ld(x[a], reinterpret_cast<const T*>(wb.w[a]) + soff + (size_t)s * L.Bs);
    for (int bi = 0; bi < nb; ++bi) {
      T* P = psi + bi * bstride + soff + (size_t)s * L.Bs;
      T p[VW];
      VecIO<T, VW>::ld_rw(p, P);
#pragma unroll
      for (int a = 0; a < kPsiBatchMax; ++a) {
        if (a >= m) break;
        const T* eb = sE + ((size_t)(a * nb + bi) * gs + (size_t)lane * NG) * NVG;
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int j = 0; j < DS; ++j) {
            T t = p[g * DS + j];
#pragma unroll
            for (int i = 0; i < DS; ++i) t = fma(x[a][g * DS + i], eb[g * NVG + i * DS + j], t);
            p[g * DS + j] = t;
          }
      }
      VecIO<T, VW>::st(P, p);
    }
  }
}

// Gram partials of one psi block. The Gram is accumulated in float64 whatever the
// vectors' precision (eq. rho_est): a product of two float32 values is exact in float64,
// so each fma rounds only the sum. Only the upper triangle is summed; the lower one is
// its mirror (the same products, so the same bits).
template <typename T, int DS, int VW>
__global__ void __launch_bounds__(kThreads) k_final_gram(Layout L, const T* __restrict__ P,
                                                         double* partials) {
  constexpr int NG = VW / DS;
  constexpr int NVG = DS * DS;
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = blockIdx.y;
  const size_t soff = (size_t)slice * L.D * L.Bs + (size_t)lane * VW;
  double acc[NG][DS][DS];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < DS; ++i)
#pragma unroll
      for (int j = 0; j < DS; ++j) acc[g][i][j] = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * rpb + rs; s < L.D; s += (int64_t)gridDim.x * rpb) {
    T p[VW];
    VecIO<T, VW>::ld(p, P + soff + (size_t)s * L.Bs);
    double pd[VW];
#pragma unroll
    for (int v = 0; v < VW; ++v) pd[v] = (double)p[v];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < DS; ++i)
#pragma unroll
        for (int j = i; j < DS; ++j) acc[g][i][j] = fma(pd[g * DS + i], pd[g * DS + j], acc[g][i][j]);
  }
  double vals[NG * NVG];
#pragma unroll
  for (int g = 0; g < NG; ++g)
#pragma unroll
    for (int i = 0; i < DS; ++i)
#pragma unroll
      for (int j = 0; j < DS; ++j) vals[g * NVG + i * DS + j] = j >= i ? acc[g][i][j] : acc[g][j][i];
  block_reduce_store<NG, NVG, double>(vals, tpr, partials, L.groups_per_slice(),
                                       (size_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// Stored-basis Gram: psi_beta = sum_{j=1..k} W_j E_{j,beta} row by row (the same
// fma sequence as the two-pass accumulation, so the result is bit-identical) and
// the partial sums of psi_beta^T psi_beta, for up to kGramBetas betas per launch.
// W_j = W1 + (j-1) * D * B elements; e: [j][beta (stride nbs)][group][DS*DS].
constexpr int kGramBetas = 4;
// With d_s <= 2 a beta's psi and Gram partials take few registers: twice the betas per
// launch, half the passes over the stored basis.
constexpr int kGramBetasWide = 8;

template <typename T, int DS>
struct RowVec;  // DS consecutive coefficients as one shared-memory load
template <>
struct RowVec<float, 4> {
  __device__ static void ld(float* r, const float* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
};
template <>
struct RowVec<float, 2> {
  __device__ static void ld(float* r, const float* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    r[0] = v.x; r[1] = v.y;
  }
};
template <>
struct RowVec<float, 1> {
  __device__ static void ld(float* r, const float* p) { r[0] = *p; }
};
template <>
struct RowVec<double, 4> {
  __device__ static void ld(double* r, const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  }
};
template <>
struct RowVec<double, 2> {
  __device__ static void ld(double* r, const double* p) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    r[0] = v.x; r[1] = v.y;
  }
};
template <>
struct RowVec<double, 1> {
  __device__ static void ld(double* r, const double* p) { r[0] = *p; }
};

// Each thread takes two rows at a time so every coefficient row read from shared
// memory serves both.
template <typename T, int DS, int VW, int NBT>
__global__ void __launch_bounds__(kThreads) k_gram_stored(Layout L, const T* __restrict__ W1, int k,
                                                          const double* e, int nbs, int b0, int nb,
                                                          double* partials, size_t pstride) {
  constexpr int NG = VW / DS;
  constexpr int NVG = DS * DS;
  extern __shared__ __align__(16) unsigned char smem_g[];
  T* sE = reinterpret_cast<T*>(smem_g);  // [j][bi][gs][NVG]
  const int tpr = L.TPR, rpb = kThreads / tpr;
  const int lane = threadIdx.x % tpr, rs = threadIdx.x / tpr;
  const int slice = blockIdx.y;
  const int gs = L.groups_per_slice(), ng = L.n_groups();
  const size_t soff = (size_t)slice * L.D * L.Bs + (size_t)lane * VW;
  const size_t bstride = (size_t)L.D * L.B;
  for (int i = threadIdx.x; i < k * nb * gs * NVG; i += blockDim.x) {
    const int j = i / (nb * gs * NVG);
    const int rem = i % (nb * gs * NVG);
    const int bi = rem / (gs * NVG), r2 = rem % (gs * NVG);
    sE[i] = (T)e[(((size_t)j * nbs + b0 + bi) * ng) * NVG + (size_t)slice * gs * NVG + r2];
  }
  __syncthreads();
  // the Gram in float64 (upper triangle; see k_final_gram)
  double acc[NBT][NG][DS][DS];
#pragma unroll
  for (int bi = 0; bi < NBT; ++bi)
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int i = 0; i < DS; ++i)
#pragma unroll
        for (int j = 0; j < DS; ++j) acc[bi][g][i][j] = 0.0;
  // Rows s and s + stride form a pair; the accumulation order per row is the same
  // as for single rows (rows are visited in the same sequence per thread).
  const int64_t stride = (int64_t)gridDim.x * rpb;
  for (int64_t s0 = (int64_t)blockIdx.x * rpb + rs; s0 < L.D; s0 += 2 * stride) {
    const int64_t s1 = s0 + stride;
    const bool two = s1 < L.D;
    T psi[2][NBT][VW];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int bi = 0; bi < NBT; ++bi)
#pragma unroll
        for (int v = 0; v < VW; ++v) psi[h][bi][v] = (T)0;
    auto step = [&](int j, const T (&x)[2][VW]) {
#pragma unroll
      for (int bi = 0; bi < NBT; ++bi) {
        if (bi >= nb) break;
        const T* eb = sE + (((size_t)j * nb + bi) * gs + (size_t)lane * NG) * NVG;
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int i = 0; i < DS; ++i) {
            T er[DS];
            RowVec<T, DS>::ld(er, eb + g * NVG + i * DS);
#pragma unroll
            for (int jj = 0; jj < DS; ++jj) {
              psi[0][bi][g * DS + jj] = fma(x[0][g * DS + i], er[jj], psi[0][bi][g * DS + jj]);
              psi[1][bi][g * DS + jj] = fma(x[1][g * DS + i], er[jj], psi[1][bi][g * DS + jj]);
            }
          }
      }
    };
    int j = 0;
    for (; j + 4 <= k; j += 4) {  // four blocks' loads in flight before their use
      T x[4][2][VW];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T* wj = W1 + (size_t)(j + u) * bstride + soff;
        VecIO<T, VW>::ld(x[u][0], wj + (size_t)s0 * L.Bs);
        if (two) VecIO<T, VW>::ld(x[u][1], wj + (size_t)s1 * L.Bs);
        else
#pragma unroll
          for (int v = 0; v < VW; ++v) x[u][1][v] = (T)0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) step(j + u, x[u]);
    }
    for (; j < k; ++j) {
      T x[2][VW];
      const T* wj = W1 + (size_t)j * bstride + soff;
      VecIO<T, VW>::ld(x[0], wj + (size_t)s0 * L.Bs);
      if (two) VecIO<T, VW>::ld(x[1], wj + (size_t)s1 * L.Bs);
      else
#pragma unroll
        for (int v = 0; v < VW; ++v) x[1][v] = (T)0;
      step(j, x);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
#pragma unroll
      for (int bi = 0; bi < NBT; ++bi) {
        double pd[VW];
#pragma unroll
        for (int v = 0; v < VW; ++v) pd[v] = (double)psi[h][bi][v];
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int i = 0; i < DS; ++i)
#pragma unroll
            for (int j = i; j < DS; ++j)
              acc[bi][g][i][j] = fma(pd[g * DS + i], pd[g * DS + j], acc[bi][g][i][j]);
      }
    }
  }
#pragma unroll
  for (int bi = 0; bi < NBT; ++bi) {  // static indices keep acc in registers
    if (bi < nb) {
      double vals[NG * NVG];
#pragma unroll
      for (int g = 0; g < NG; ++g)
#pragma unroll
        for (int i = 0; i < DS; ++i)
#pragma unroll
          for (int j = 0; j < DS; ++j)
            vals[g * NVG + i * DS + j] = j >= i ? acc[bi][g][i][j] : acc[bi][g][j][i];
      block_reduce_store<NG, NVG, double>(vals, tpr, partials + (size_t)bi * pstride, gs,
                                           (size_t)blockIdx.y * gridDim.x + blockIdx.x);
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- per-group small steps

constexpr int kSmallThreads = 128;

// Sums the NV partials of group l over the gridx blocks (fixed order: thread t < 128
// takes bx = t, t + 128, ..., then a tree over the 128 sums). Every thread of the block
// must call it; threads beyond the first kSmallThreads only pass the barriers.
template <int NV>
__device__ void reduce_group(const Layout& L, const double* partials, double* out, int l) {
  __shared__ double sh[kSmallThreads];
  const int gs = L.groups_per_slice();
  const int slice = l / gs, gis = l % gs;
  const bool part = threadIdx.x < kSmallThreads;
  for (int v = 0; v < NV; ++v) {
    if (part) {
      double s = 0.0;
      for (int bx = threadIdx.x; bx < L.gridx; bx += kSmallThreads)
        s += partials[((size_t)(slice * L.gridx + bx) * gs + gis) * NV + v];
      sh[threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = kSmallThreads / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = sh[0];
    __syncthreads();
  }
}

template <int DS>
__global__ void k_coef_init(int n_groups, double* mz, double* cp) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_groups) return;
  for (int i = 0; i < DS; ++i)
    for (int j = 0; j < DS; ++j) {
      mz[(size_t)l * DS * DS + i * DS + j] = i == j ? 1.0 : 0.0;
      cp[(size_t)l * DS * DS + i * DS + j] = 0.0;
    }
}

// After the SpMM, for group l (every thread of the block calls it): A_j and Cw_j.
template <int DS>
__device__ void small_a_group(const Layout& L, const double* partials, const double* mz, double* a_out,
                              double* cw_out, uint32_t* flags, int l) {
  constexpr int NV = DS * DS;
  __shared__ double tot[NV];
  reduce_group<NV>(L, partials, tot, l);
  if (threadIdx.x != 0) return;
  const double* M = mz + (size_t)l * NV;
  double p1[DS][DS], A[DS][DS];
  // P1 = M^T (W^T Z) = Q_j^T Z
  for (int i = 0; i < DS; ++i)
    for (int j = 0; j < DS; ++j) {
      double s = 0.0;
      for (int c = 0; c < DS; ++c) s += M[c * DS + i] * tot[c * DS + j];
      p1[i][j] = s;
    }
  bool finite = true;
  for (int i = 0; i < DS; ++i)
    for (int j = 0; j < DS; ++j) {
      A[i][j] = 0.5 * (p1[i][j] + p1[j][i]);
      finite = finite && isfinite(A[i][j]);
    }
  for (int i = 0; i < DS; ++i)
    for (int j = 0; j < DS; ++j) {
      a_out[(size_t)l * NV + i * DS + j] = A[i][j];
      double s = 0.0;
      for (int c = 0; c < DS; ++c) s += M[i * DS + c] * A[c][j];
      cw_out[(size_t)l * NV + i * DS + j] = -s;
    }
  if (!finite) atomicOr(flags, kFlagNonFinite);
}

template <int DS>
__global__ void k_small_a(Layout L, const double* partials, const double* mz, double* a_out,
                          double* cw_out, uint32_t* flags) {
  small_a_group<DS>(L, partials, mz, a_out, cw_out, flags, blockIdx.x);
}

// After the orthogonalisation, for group l (every thread of the block calls it): the
// Cholesky QR with deflation -> B_j, M_{j+1}, Cp_{j+1}.
template <int DS>
__device__ void small_b_group(const Layout& L, const double* partials, const double* mz_j, double* b_out,
                              double* mz_next, double* cp_next, double thr_abs_sq, double thr_rel_sq,
                              int n_real, uint32_t* flags, int l) {
  constexpr int NV = DS * DS;
  __shared__ double tot[NV];
  reduce_group<NV>(L, partials, tot, l);
  if (threadIdx.x != 0) return;
  double G[DS][DS], R[DS][DS], Ri[DS][DS];
  bool kept[DS];
  for (int i = 0; i < DS; ++i)
    for (int j = 0; j < DS; ++j) {
      G[i][j] = 0.5 * (tot[i * DS + j] + tot[j * DS + i]);
      R[i][j] = 0.0;
      Ri[i][j] = 0.0;
    }
  // Cholesky G = R^T R column by column, dropping numerically dependent columns
  // (Gram-Schmidt in the G inner product; same rule as a column-wise QR).
  bool dropped = false, finite = true;
  for (int c = 0; c < DS; ++c) {
    for (int k = 0; k < c; ++k) {
      if (!kept[k]) continue;
      double s = G[k][c];
      for (int i = 0; i < k; ++i)
        if (kept[i]) s -= R[i][k] * R[i][c];
      R[k][c] = s / R[k][k];
    }
    double piv = G[c][c];
    for (int k = 0; k < c; ++k)
      if (kept[k]) piv -= R[k][c] * R[k][c];
    finite = finite && isfinite(piv);
    if (!(piv > thr_abs_sq) || !(piv > thr_rel_sq * G[c][c])) {
      kept[c] = false;
      R[c][c] = 0.0;
      dropped = true;
    } else {
      kept[c] = true;
      R[c][c] = sqrt(piv);
    }
  }
  // Inverse of R restricted to the kept columns (back substitution), zero elsewhere.
  for (int c = 0; c < DS; ++c) {
    if (!kept[c]) continue;
    Ri[c][c] = 1.0 / R[c][c];
    for (int r = c - 1; r >= 0; --r) {
      if (!kept[r]) continue;
      double s = 0.0;
      for (int m = r + 1; m <= c; ++m)
        if (kept[m]) s += R[r][m] * Ri[m][c];
      Ri[r][c] = -s / R[r][r];
    }
  }
  const double* Mj = mz_j + (size_t)l * NV;
  for (int i = 0; i < DS; ++i)
    for (int j = 0; j < DS; ++j) {
      b_out[(size_t)l * NV + i * DS + j] = R[i][j];
      mz_next[(size_t)l * NV + i * DS + j] = Ri[i][j];
      double s = 0.0;
      for (int c = 0; c < DS; ++c) s += Mj[i * DS + c] * R[j][c];
      cp_next[(size_t)l * NV + i * DS + j] = -s;
    }
  if (dropped && l < n_real) atomicOr(flags, (uint32_t)RDM_FLAG_DEFLATED);
  if (!finite) atomicOr(flags, kFlagNonFinite);
}

template <int DS>
__global__ void k_small_b(Layout L, const double* partials, const double* mz_j, double* b_out,
                          double* mz_next, double* cp_next, double thr_abs_sq, double thr_rel_sq,
                          int n_real, uint32_t* flags) {
  small_b_group<DS>(L, partials, mz_j, b_out, mz_next, cp_next, thr_abs_sq, thr_rel_sq, n_real, flags,
                    blockIdx.x);
}

template <int DS>
__global__ void k_reduce_gram(Layout L, const double* partials, double* gram) {
  constexpr int NV = DS * DS;
  __shared__ double tot[NV];
  reduce_group<NV>(L, partials, tot, blockIdx.x);
  if (threadIdx.x != 0) return;
  for (int v = 0; v < NV; ++v) gram[(size_t)blockIdx.x * NV + v] = tot[v];
}

// ---------------------------------------------------------------- packed first pass
//
// The first pass (Algorithm 1's k steps) of several estimates in ONE cooperative
// launch: every block of a persistent grid walks the work units of a phase, and a grid
// barrier separates the phases of a step: SpMM (+ W_j^T Z partials), A_j per bath
// vector, orthogonalisation (+ Gram partials), Cholesky QR per bath vector. A unit is
// exactly one block of the corresponding plain launch of that estimate (block (bx, by)
// of its gridx x n_slices grid, or group l), so each estimate's arithmetic and
// reduction order depend on its own layout only: results are the same whichever
// estimates share the launch and however the units are spread over the grid. Items are
// sorted by k, largest first, so the items still running at step j are a prefix.

// Grid barrier: arrival counter, generation word, error word (zero before the launch).
// The last block to arrive resets the counter and advances the generation; the others
// wait for that with a bounded spin. A wait that gives up sets the error word, and a
// block that sees the error word set leaves at its next barrier.
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ bool grid_barrier(uint32_t* bar, uint32_t& gen) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    if (ld_acquire_gpu(bar + 2) != 0u) {
      ok = 0;
    } else if (atomicAdd(bar, 1u) == gridDim.x - 1u) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicExch(bar + 1, gen + 1u);
    } else {
      uint32_t it = 0;
      while (ld_acquire_gpu(bar + 1) == gen) {
        if (++it > (1u << 24) || ld_acquire_gpu(bar + 2) != 0u) {
          atomicOr(bar + 2, 1u);
          ok = 0;
          break;
        }
        if (it > 64) __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  ++gen;
  return ok_s != 0;
}

// Unit u of a phase -> its item (largest i with pre[i] <= u among the first n).
__device__ __forceinline__ int packed_item_of(const int* pre, int n, int u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <typename T, int DS, int VW>
__global__ void __launch_bounds__(kThreads) k_pass1_packed(PackedPlan pp) {
  constexpr int NVG = DS * DS;
  uint32_t gen = 0;
  for (int j = 1; j <= pp.k_max; ++j) {
    const int na = pp.active[j];
    // phase A: Z = (H W_j) M_j + W_{j-1} Cp_j and the partial sums of W_j^T Z
    for (int u = blockIdx.x; u < pp.pre_rows[na]; u += gridDim.x) {
      const int i = packed_item_of(pp.pre_rows, na, u);
      const PackedItem& it = pp.items[i];
      const int r = u - pp.pre_rows[i];
      const size_t bb = it.L.block_bytes(), cs = (size_t)it.L.n_groups() * NVG;
      SpmmArgs a = it.sa;
      a.w = it.blk + (size_t)(j - 1) * bb;
      a.w_prev = j > 1 ? it.blk + (size_t)(j - 2) * bb : nullptr;
      a.z = it.blk + (size_t)j * bb;
      a.mz = it.coef + (size_t)j * cs;
      a.cp = it.coef + (size_t)(it.k + 2) * cs + (size_t)j * cs;
      const TermsSmem<T> terms = load_terms<T>(a.flips, a.n_flip, a.diags, a.n_diag);
      spmm_block<T, DS, VW, kModePass1, true>(it.L, a, terms, r % it.L.gridx, r / it.L.gridx, it.L.gridx);
      __syncthreads();  // the next unit rewrites the term tables
    }
    if (!grid_barrier(pp.bar, gen)) return;
    // phase B: A_j and Cw_j per bath vector
    for (int u = blockIdx.x; u < pp.pre_groups[na]; u += gridDim.x) {
      const int i = packed_item_of(pp.pre_groups, na, u);
      const PackedItem& it = pp.items[i];
      const size_t cs = (size_t)it.L.n_groups() * NVG;
      small_a_group<DS>(it.L, it.sa.partials, it.coef + (size_t)j * cs, it.ta + (size_t)(j - 1) * cs,
                        it.coef + (size_t)2 * (it.k + 2) * cs + (size_t)j * cs, it.flags, u - pp.pre_groups[i]);
      __syncthreads();
    }
    if (!grid_barrier(pp.bar, gen)) return;
    // phase C: W_{j+1} = Z + W_j Cw_j in place, partial sums of W_{j+1}^T W_{j+1}
    for (int u = blockIdx.x; u < pp.pre_rows[na]; u += gridDim.x) {
      const int i = packed_item_of(pp.pre_rows, na, u);
      const PackedItem& it = pp.items[i];
      const int r = u - pp.pre_rows[i];
      const size_t bb = it.L.block_bytes(), cs = (size_t)it.L.n_groups() * NVG;
      orth_block<T, DS, VW, true, true>(it.L, reinterpret_cast<const T*>(it.blk + (size_t)(j - 1) * bb),
                                        reinterpret_cast<T*>(it.blk + (size_t)j * bb),
                                        it.coef + (size_t)2 * (it.k + 2) * cs + (size_t)j * cs, it.sa.partials,
                                        nullptr, nullptr, 0, r % it.L.gridx, r / it.L.gridx, it.L.gridx);
      __syncthreads();
    }
    if (!grid_barrier(pp.bar, gen)) return;
    // phase D: Cholesky QR with deflation -> B_j, M_{j+1}, Cp_{j+1}
    for (int u = blockIdx.x; u < pp.pre_groups[na]; u += gridDim.x) {
      const int i = packed_item_of(pp.pre_groups, na, u);
      const PackedItem& it = pp.items[i];
      const size_t cs = (size_t)it.L.n_groups() * NVG;
      small_b_group<DS>(it.L, it.sa.partials, it.coef + (size_t)j * cs, it.tb + (size_t)(j - 1) * cs,
                        it.coef + (size_t)(j + 1) * cs, it.coef + (size_t)(it.k + 2) * cs + (size_t)(j + 1) * cs,
                        it.thr_abs_sq, it.thr_rel_sq, it.n_rec, it.flags, u - pp.pre_groups[i]);
      __syncthreads();
    }
    if (!grid_barrier(pp.bar, gen)) return;
  }
}

// The first pass of k_pass1_packed for one slice of one item per block: the recurrences
// of a slice's bath vectors read and write nothing of other slices, so the block runs
// every phase of every step for its slice alone -- the same row-block units and group
// units as the packed launch, in order, with block barriers between phases.
template <typename T, int DS, int VW>
__global__ void __launch_bounds__(kThreads) k_pass1_local(PackedPlan pp) {
  constexpr int NVG = DS * DS;
  const int u = blockIdx.x;
  const int i = packed_item_of(pp.pre_slices, pp.n_items, u);
  const PackedItem& it = pp.items[i];
  const int sl = u - pp.pre_slices[i];
  const size_t bb = it.L.block_bytes(), cs = (size_t)it.L.n_groups() * NVG;
  const int gx = it.L.gridx, gs = it.L.groups_per_slice();
  const TermsSmem<T> terms = load_terms<T>(it.sa.flips, it.sa.n_flip, it.sa.diags, it.sa.n_diag);
  for (int j = 1; j <= it.k; ++j) {
    SpmmArgs a = it.sa;
    a.w = it.blk + (size_t)(j - 1) * bb;
    a.w_prev = j > 1 ? it.blk + (size_t)(j - 2) * bb : nullptr;
    a.z = it.blk + (size_t)j * bb;
    a.mz = it.coef + (size_t)j * cs;
    a.cp = it.coef + (size_t)(it.k + 2) * cs + (size_t)j * cs;
    for (int bx = 0; bx < gx; ++bx) {
      spmm_block<T, DS, VW, kModePass1, true>(it.L, a, terms, bx, sl, gx);
      __syncthreads();
    }
    for (int g = 0; g < gs; ++g) {
      small_a_group<DS>(it.L, it.sa.partials, it.coef + (size_t)j * cs, it.ta + (size_t)(j - 1) * cs,
                        it.coef + (size_t)2 * (it.k + 2) * cs + (size_t)j * cs, it.flags, sl * gs + g);
      __syncthreads();
    }
    for (int bx = 0; bx < gx; ++bx) {
      orth_block<T, DS, VW, true, true>(it.L, reinterpret_cast<const T*>(it.blk + (size_t)(j - 1) * bb),
                                        reinterpret_cast<T*>(it.blk + (size_t)j * bb),
                                        it.coef + (size_t)2 * (it.k + 2) * cs + (size_t)j * cs, it.sa.partials,
                                        nullptr, nullptr, 0, bx, sl, gx);
      __syncthreads();
    }
    for (int g = 0; g < gs; ++g) {
      small_b_group<DS>(it.L, it.sa.partials, it.coef + (size_t)j * cs, it.tb + (size_t)(j - 1) * cs,
                        it.coef + (size_t)(j + 1) * cs, it.coef + (size_t)(it.k + 2) * cs + (size_t)(j + 1) * cs,
                        it.thr_abs_sq, it.thr_rel_sq, it.n_rec, it.flags, sl * gs + g);
      __syncthreads();
    }
  }
}

inline dim3 grid_of(const Layout& L) { return dim3((unsigned)L.gridx, (unsigned)L.n_slices); }

template <typename T>
size_t terms_smem(int nf, int nd) {
  return (size_t)(2 * nf + nd) * sizeof(T) + (size_t)(nf + nd) * sizeof(uint32_t) + 16;
}

}  // namespace

// Raises a kernel's dynamic shared-memory limit to the device maximum (minus its
// static shared memory), once per kernel. Setting it to the largest value once,
// instead of to each launch's size, keeps concurrent host threads from lowering it
// under one another's launches.
static cudaError_t opt_in_smem(const void* func) {
  static std::mutex mu;
  static std::set<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(func)) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert(func);
  return e;
}

// ---------------------------------------------------------------- dispatch

#define RDM_DISPATCH(L, ...)                                         \
  do {                                                                \
    if ((L).precision == RDM_FP32) {                                  \
      using T = float;                                                \
      constexpr int VW = 4;                                           \
      if ((L).DS == 1) { constexpr int DS = 1; __VA_ARGS__; }                \
      else if ((L).DS == 2) { constexpr int DS = 2; __VA_ARGS__; }           \
      else { constexpr int DS = 4; __VA_ARGS__; }                            \
    } else {                                                          \
      using T = double;                                               \
      if ((L).DS == 1) { constexpr int DS = 1; constexpr int VW = 2; __VA_ARGS__; } \
      else if ((L).DS == 2) { constexpr int DS = 2; constexpr int VW = 2; __VA_ARGS__; } \
      else { constexpr int DS = 4; constexpr int VW = 4; __VA_ARGS__; }      \
    }                                                                 \
  } while (0)

#define RDM_DISPATCH_DS(DSV, ...)                      \
  do {                                                  \
    if ((DSV) == 1) { constexpr int DS = 1; __VA_ARGS__; }     \
    else if ((DSV) == 2) { constexpr int DS = 2; __VA_ARGS__; } \
    else { constexpr int DS = 4; __VA_ARGS__; }                \
  } while (0)

cudaError_t launch_gauss_norms(int64_t d_b, int n_v, uint64_t seed, int64_t l0, double* partials,
                               double* inv_norm, cudaStream_t st, double* graw) {
  int gx = (int)((d_b + 4095) / 4096);
  if (gx > 64) gx = 64;
  if (gx < 1) gx = 1;
  k_gauss_sumsq<<<dim3(gx, n_v), kThreads, 0, st>>>(d_b, seed, l0, partials, graw);
  k_gauss_finish<<<(n_v + 127) / 128, 128, 0, st>>>(n_v, gx, partials, inv_norm);
  return cudaGetLastError();
}

cudaError_t launch_init_block(const Layout& L, int dist, uint64_t seed, int64_t l0, int n_v_real,
                              const double* inv_norm, const void* vbuf, void* W, cudaStream_t st,
                              int sub, const BathPerm* bp) {
  BathPerm id{};
  const BathPerm perm = bp ? *bp : id;
  if (perm.n < 0 || perm.n > L.n_bath_bits) return cudaErrorInvalidValue;
  for (int q = 0; q < perm.n; ++q)
    if (perm.src[q] >= perm.n) return cudaErrorInvalidValue;
  RDM_DISPATCH(L, (k_init_block<T, DS, VW><<<grid_of(L), kThreads, 0, st>>>(
                      L, dist, seed, l0, n_v_real, inv_norm, reinterpret_cast<const T*>(vbuf),
                      reinterpret_cast<T*>(W), sub, perm)));
  return cudaGetLastError();
}

cudaError_t launch_gauss_fill(const Layout& L, int n_v, uint64_t seed, int64_t l0,
                              const double* inv_norm, void* vbuf, cudaStream_t st, const double* graw) {
  const int64_t d_b = int64_t(1) << L.n_bath_bits;
  int gx = (int)std::min<int64_t>((d_b + 255) / 256, 1024);
  k_gauss_fill<<<dim3(gx, n_v), 256, 0, st>>>(d_b, seed, l0, inv_norm, graw, L.precision, vbuf);
  return cudaGetLastError();
}

cudaError_t launch_tile_diag(const Layout& L, const TileDiag& dg, void* out, cudaStream_t st) {
  const int64_t tiles = L.D >> kTileBits;
  const int stride = tile_diag_stride(dg.n_entries, L.elem);
  const int gx = (int)std::min<int64_t>(tiles, 4096);
  const size_t sm = (size_t)(dg.n_groups + 1) * sizeof(double);
  if (sm > 48 * 1024) return cudaErrorInvalidValue;
  if (L.precision == RDM_FP32)
    k_tile_diag<float><<<gx, kThreads, sm, st>>>(tiles, dg, stride, reinterpret_cast<float*>(out));
  else
    k_tile_diag<double><<<gx, kThreads, sm, st>>>(tiles, dg, stride, reinterpret_cast<double*>(out));
  return cudaGetLastError();
}

template <typename T, int DS, int MODE, bool UNI = false>
static cudaError_t launch_tiled(const Layout& L, const SpmmArgs& a0, cudaStream_t st) {
  cudaError_t e = opt_in_smem(reinterpret_cast<const void*>(k_spmm_tiled<T, DS, MODE, UNI>));
  if (e != cudaSuccess) return e;
  static int optin = 0;
  if (!optin) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
  }
  // Deepest ring (up to 6 slots) that fits beside this Hamiltonian's term tables.
  SpmmArgs a = a0;
  const TiledTerms& tt = a.tiled;
  a.stages = 6;  // a multiple of kProducerWarps
  while (a.stages > kProducerWarps &&
         tiled_smem_bytes<T>(tt.n_pat, tt.n_terms, tt.dg.n_entries, a.stages) > (size_t)optin)
    a.stages -= kProducerWarps;
  const size_t sm = tiled_smem_bytes<T>(tt.n_pat, tt.n_terms, tt.dg.n_entries, a.stages);
  if (sm > (size_t)optin) return cudaErrorInvalidValue;
  k_spmm_tiled<T, DS, MODE, UNI><<<dim3((unsigned)spmm_tiled_grid(L), 1), kTiledThreads, sm, st>>>(L, a);
  return cudaGetLastError();
}

cudaError_t launch_spmm(const Layout& L, int mode, const SpmmArgs& a, cudaStream_t st) {
  if (layout_tiled(L) && a.tiled.n_pat > 0 && a.tile_k) {
    const bool f32 = L.precision == RDM_FP32;
    if (mode == kModeApply) {
      if (L.DS != 1) return cudaErrorInvalidValue;
      return f32 ? launch_tiled<float, 1, kModeApply>(L, a, st) : launch_tiled<double, 1, kModeApply>(L, a, st);
    }
    const bool p1 = mode == kModePass1;
    if (f32 && a.tiled.all_uniform) {  // no parity-dependent coefficient anywhere
      if (L.DS == 1)
        return p1 ? launch_tiled<float, 1, kModePass1, true>(L, a, st) : launch_tiled<float, 1, kModePass2, true>(L, a, st);
      if (L.DS == 2)
        return p1 ? launch_tiled<float, 2, kModePass1, true>(L, a, st) : launch_tiled<float, 2, kModePass2, true>(L, a, st);
      return p1 ? launch_tiled<float, 4, kModePass1, true>(L, a, st) : launch_tiled<float, 4, kModePass2, true>(L, a, st);
    }
    if (f32) {
      if (L.DS == 1) return p1 ? launch_tiled<float, 1, kModePass1>(L, a, st) : launch_tiled<float, 1, kModePass2>(L, a, st);
      if (L.DS == 2) return p1 ? launch_tiled<float, 2, kModePass1>(L, a, st) : launch_tiled<float, 2, kModePass2>(L, a, st);
      return p1 ? launch_tiled<float, 4, kModePass1>(L, a, st) : launch_tiled<float, 4, kModePass2>(L, a, st);
    }
    if (L.DS == 1) return p1 ? launch_tiled<double, 1, kModePass1>(L, a, st) : launch_tiled<double, 1, kModePass2>(L, a, st);
    if (L.DS == 2) return p1 ? launch_tiled<double, 2, kModePass1>(L, a, st) : launch_tiled<double, 2, kModePass2>(L, a, st);
    return p1 ? launch_tiled<double, 4, kModePass1>(L, a, st) : launch_tiled<double, 4, kModePass2>(L, a, st);
  }
  RDM_DISPATCH(L, {
    const size_t sm = terms_smem<T>(a.n_flip, a.n_diag);
    if (mode == kModeApply)
      k_spmm<T, DS, VW, kModeApply><<<grid_of(L), kThreads, sm, st>>>(L, a);
    else if (mode == kModePass1)
      k_spmm<T, DS, VW, kModePass1><<<grid_of(L), kThreads, sm, st>>>(L, a);
    else
      k_spmm<T, DS, VW, kModePass2><<<grid_of(L), kThreads, sm, st>>>(L, a);
  });
  return cudaGetLastError();
}

cudaError_t launch_orth(const Layout& L, const void* w, void* z, const double* cw,
                        double* partials, cudaStream_t st) {
  RDM_DISPATCH(L, (k_orth<T, DS, VW, true><<<grid_of(L), kThreads, 0, st>>>(
                      L, reinterpret_cast<const T*>(w), reinterpret_cast<T*>(z), cw, partials,
                      nullptr, nullptr, 0)));
  return cudaGetLastError();
}

cudaError_t launch_orth_psi(const Layout& L, const void* w, void* z, const double* cw, void* psi,
                            const double* e, int nb, cudaStream_t st) {
  RDM_DISPATCH(L, {
    const size_t sm = (size_t)nb * L.groups_per_slice() * DS * DS * sizeof(T) + 16;
    cudaError_t ce = opt_in_smem(reinterpret_cast<const void*>(k_orth<T, DS, VW, false>));
    if (ce != cudaSuccess) return ce;
    k_orth<T, DS, VW, false><<<grid_of(L), kThreads, sm, st>>>(
        L, reinterpret_cast<const T*>(w), reinterpret_cast<T*>(z), cw, nullptr,
        reinterpret_cast<T*>(psi), e, nb);
  });
  return cudaGetLastError();
}

cudaError_t launch_psi_batch(const Layout& L, const PsiBatch& wb, int m, void* psi, const double* e,
                             size_t estride, int nb, cudaStream_t st) {
  if (m < 1 || m > kPsiBatchMax) return cudaErrorInvalidValue;
  RDM_DISPATCH(L, {
    const size_t sm = (size_t)m * nb * L.groups_per_slice() * DS * DS * sizeof(T) + 16;
    cudaError_t ce = opt_in_smem(reinterpret_cast<const void*>(k_psi_batch<T, DS, VW>));
    if (ce != cudaSuccess) return ce;
    k_psi_batch<T, DS, VW><<<grid_of(L), kThreads, sm, st>>>(L, wb, m, reinterpret_cast<T*>(psi), e, estride,
                                                             nb);
  });
  return cudaGetLastError();
}

cudaError_t launch_psi_init(const Layout& L, const void* w, void* psi, const double* e, int nb,
                            cudaStream_t st) {
  RDM_DISPATCH(L, (k_psi_init<T, DS, VW><<<grid_of(L), kThreads, 0, st>>>(
                      L, reinterpret_cast<const T*>(w), reinterpret_cast<T*>(psi), e, nb)));
  return cudaGetLastError();
}

cudaError_t launch_coef_init(const Layout& L, StepCoefs c1, cudaStream_t st) {
  const int ng = L.n_groups();
  RDM_DISPATCH_DS(L.DS, (k_coef_init<DS><<<(ng + 127) / 128, 128, 0, st>>>(ng, c1.mz, c1.cp)));
  return cudaGetLastError();
}

cudaError_t launch_small_a(const Layout& L, const double* partials, const double* mz,
                           double* a_out, double* cw_out, uint32_t* flags, cudaStream_t st) {
  RDM_DISPATCH_DS(L.DS, (k_small_a<DS><<<L.n_groups(), kSmallThreads, 0, st>>>(
                           L, partials, mz, a_out, cw_out, flags)));
  return cudaGetLastError();
}

cudaError_t launch_small_b(const Layout& L, const double* partials, const double* mz_j,
                           double* b_out, double* mz_next, double* cp_next, double thr_abs_sq,
                           double thr_rel_sq, int n_groups_real, uint32_t* flags,
                           cudaStream_t st) {
  RDM_DISPATCH_DS(L.DS, (k_small_b<DS><<<L.n_groups(), kSmallThreads, 0, st>>>(
                           L, partials, mz_j, b_out, mz_next, cp_next, thr_abs_sq, thr_rel_sq,
                           n_groups_real, flags)));
  return cudaGetLastError();
}

template <typename T, int DS, int VW>
static cudaError_t packed_kernel_info(const void** fn) {
  *fn = reinterpret_cast<const void*>(k_pass1_packed<T, DS, VW>);
  return opt_in_smem(*fn);
}

static cudaError_t packed_fn(int precision, int ds, const void** fn) {
  Layout L{};
  L.precision = precision;
  L.DS = ds;
  cudaError_t e = cudaErrorInvalidValue;
  RDM_DISPATCH(L, e = (packed_kernel_info<T, DS, VW>(fn)));
  return e;
}

size_t spmm_terms_smem(int precision, int n_flip, int n_diag) {
  return precision == RDM_FP32 ? terms_smem<float>(n_flip, n_diag) : terms_smem<double>(n_flip, n_diag);
}

int packed_max_blocks_per_sm(int precision, int ds, size_t smem) {
  const void* fn = nullptr;
  if (packed_fn(precision, ds, &fn) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kThreads, smem) != cudaSuccess) return 0;
  return n;
}

template <typename T, int DS, int VW>
static cudaError_t local_kernel_info(const void** fn) {
  *fn = reinterpret_cast<const void*>(k_pass1_local<T, DS, VW>);
  return opt_in_smem(*fn);
}

cudaError_t launch_pass1_local(int precision, int ds, const PackedPlan& pp, int grid, size_t smem,
                               cudaStream_t st) {
  Layout L{};
  L.precision = precision;
  L.DS = ds;
  const void* fn = nullptr;
  cudaError_t e = cudaErrorInvalidValue;
  RDM_DISPATCH(L, e = (local_kernel_info<T, DS, VW>(&fn)));
  if (e != cudaSuccess) return e;
  PackedPlan arg = pp;
  void* args[] = {&arg};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kThreads), args, smem, st);
}

cudaError_t launch_pass1_packed(int precision, int ds, const PackedPlan& pp, int grid, size_t smem,
                                cudaStream_t st) {
  const void* fn = nullptr;
  cudaError_t e = packed_fn(precision, ds, &fn);
  if (e != cudaSuccess) return e;
  PackedPlan arg = pp;
  void* args[] = {&arg};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)grid), dim3(kThreads), args, smem, st);
}

cudaError_t launch_final_gram(const Layout& L, const void* psi, double* partials,
                              cudaStream_t st) {
  RDM_DISPATCH(L, (k_final_gram<T, DS, VW><<<grid_of(L), kThreads, 0, st>>>(
                      L, reinterpret_cast<const T*>(psi), partials)));
  return cudaGetLastError();
}

cudaError_t launch_gram_stored(const Layout& L, const void* w1, int k, const double* e, int nbs,
                               int b0, int nb, double* partials, size_t pstride, cudaStream_t st) {
  RDM_DISPATCH(L, {
    // static reduction scratch (block_reduce_store) + dynamic coefficients: opt in
    const size_t sm = (size_t)k * nb * L.groups_per_slice() * DS * DS * sizeof(T) + 16;
    cudaError_t ce = opt_in_smem(reinterpret_cast<const void*>(k_gram_stored<T, DS, VW, 1>));
    if (ce == cudaSuccess) ce = opt_in_smem(reinterpret_cast<const void*>(k_gram_stored<T, DS, VW, 2>));
    if (ce == cudaSuccess)
      ce = opt_in_smem(reinterpret_cast<const void*>(k_gram_stored<T, DS, VW, kGramBetas>));
    if (ce != cudaSuccess) return ce;
    if constexpr (DS <= 2) {
      if (nb > kGramBetas) {
        ce = opt_in_smem(reinterpret_cast<const void*>(k_gram_stored<T, DS, VW, kGramBetasWide>));
        if (ce != cudaSuccess) return ce;
        k_gram_stored<T, DS, VW, kGramBetasWide><<<grid_of(L), kThreads, sm, st>>>(
            L, reinterpret_cast<const T*>(w1), k, e, nbs, b0, nb, partials, pstride);
        return cudaGetLastError();
      }
    }
    if (nb == 1)
      k_gram_stored<T, DS, VW, 1><<<grid_of(L), kThreads, sm, st>>>(
          L, reinterpret_cast<const T*>(w1), k, e, nbs, b0, nb, partials, pstride);
    else if (nb == 2)
      k_gram_stored<T, DS, VW, 2><<<grid_of(L), kThreads, sm, st>>>(
          L, reinterpret_cast<const T*>(w1), k, e, nbs, b0, nb, partials, pstride);
    else
      k_gram_stored<T, DS, VW, kGramBetas><<<grid_of(L), kThreads, sm, st>>>(
          L, reinterpret_cast<const T*>(w1), k, e, nbs, b0, nb, partials, pstride);
  });
  return cudaGetLastError();
}

int gram_stored_max_betas(const Layout& L, int k) {
  const size_t per = (size_t)k * L.groups_per_slice() * L.DS * L.DS * L.elem;
  int nb = (int)((160 * 1024) / (per ? per : 1));
  return std::max(0, std::min(nb, L.DS <= 2 ? kGramBetasWide : kGramBetas));
}

cudaError_t launch_reduce_gram(const Layout& L, const double* partials, double* gram,
                               cudaStream_t st) {
  RDM_DISPATCH_DS(L.DS, (k_reduce_gram<DS><<<L.n_groups(), kSmallThreads, 0, st>>>(
                           L, partials, gram)));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- copy-rate probe
//
// The rate at which TMA bulk copies (the tiled SpMM's only way of filling shared
// memory) move 32 KB chunks from device memory into shared memory: one block per SM,
// one issuing thread, `stages` copies in flight in a ring of shared-memory slots (the
// SpMM's ring depth); the copied data is not read. At step i block b takes chunk
// (i * gridDim.x + b) mod n_chunks: the blocks sweep the buffer together, front to
// back, so a buffer smaller than L2 measures L2 -> shared memory after its first pass
// and a larger one DRAM -> shared memory (no chunk is read twice within a sweep).
// Every wait is
// bounded; a wait that gives up sets *err and the block still waits (bounded) for its
// other copies before it exits.
__global__ void __launch_bounds__(32, 1) k_probe_copy(const unsigned char* src, int64_t n_chunks, int iters,
                                                      int stages, int keep_in_l2, uint32_t* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* const full = reinterpret_cast<uint64_t*>(smem + (size_t)stages * kTileBytes);
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(full + kMaxStages);
  if (threadIdx.x != 0) return;
  for (int i = 0; i < stages; ++i) mbar_init(&full[i], 1);
  *abort_flag = 0;
  fence_mbar_init();
  // normal priority for the L2-resident buffer (it fits anyway; no evict-last lines are
  // left behind for later kernels), evict-first for the streamed one
  uint64_t policy;
  if (keep_in_l2)
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;\n" : "=l"(policy));
  else
    policy = policy_evict_first();
  bool ok = true;
  int issued = 0;
  for (int it = 0; it < iters && ok; ++it) {
    const int slot = it % stages;
    if (it >= stages && !ring_wait(&full[slot], (uint32_t)((it / stages - 1) & 1), abort_flag)) {
      ok = false;
      break;
    }
    const int64_t g = ((int64_t)it * gridDim.x + blockIdx.x) % n_chunks;
    mbar_expect_tx(&full[slot], kTileBytes);
    bulk_load_hint(smem + (size_t)slot * kTileBytes, src + (size_t)g * kTileBytes, kTileBytes, &full[slot],
                   policy);
    issued = it + 1;
  }
  // drain: the last min(stages, issued) copies (their slots' most recent phases)
  for (int it = issued > stages ? issued - stages : 0; it < issued; ++it) {
    const int slot = it % stages;
    *abort_flag = 0;
    if (!ring_wait(&full[slot], (uint32_t)((it / stages) & 1), abort_flag)) ok = false;
  }
  if (!ok) atomicOr(err, 1u);
}

cudaError_t launch_probe_copy(const void* src, int64_t n_chunks, int iters, int stages, bool keep_in_l2,
                              uint32_t* err, cudaStream_t st) {
  if (n_chunks <= 0 || iters <= 0 || stages < 1 || stages > kMaxStages) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = opt_in_smem(reinterpret_cast<const void*>(k_probe_copy));
  if (e != cudaSuccess) return e;
  const size_t sm = (size_t)stages * kTileBytes + kMaxStages * 8 + 16;
  k_probe_copy<<<sms, 32, sm, st>>>(static_cast<const unsigned char*>(src), n_chunks, iters, stages,
                                    keep_in_l2 ? 1 : 0, err);
  return cudaGetLastError();
}

}  // namespace rdm
