// rdm_starting_block_noalloc: the starting block without any device allocation.
//
// rdm_starting_block draws its Gaussian bath vectors in two steps, and the first
// step (the norm of every vector) needs device scratch, which it allocates per call.
// This variant keeps that scratch in a fixed array of this file instead, so a call
// never allocates or frees device memory.
//
// The array is a static __device__ symbol, so every GPU that loads this library
// holds it (kNoAllocScratchBytes) until the process exits. In host code the name
// g_noalloc_scratch is only a host-side stand-in for the symbol, not a device
// address: its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached for the life of the
// process. A cudaDeviceReset (or any teardown of the device's primary context)
// reloads the module, possibly at another address, so the cache is only valid
// while the context that looked it up lives.
#include <mutex>

#include "rdm_api_internal.h"

namespace rdm {
namespace {

// Largest n_v the variant accepts, and the scratch it needs: n_v * 64 per-block
// partial sums plus n_v inverse norms, float64. The column rule of the starting block
// (d_s * n_v columns, at most 32 float32 or 16 float64) already caps n_v at 32 (float32
// with d_s = 1), so the array is sized for exactly that.
constexpr int kNoAllocMaxVectors = 32;
constexpr size_t kNoAllocScratchDoubles = (size_t)kNoAllocMaxVectors * 65;
constexpr size_t kNoAllocScratchBytes = kNoAllocScratchDoubles * sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double* g_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), looked up on first use.
rdm_status scratch_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) {
    set_error("rdm_starting_block_noalloc: device %d out of range", device);
    return RDM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("rdm_starting_block_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return RDM_ECUDA;
    }
    g_addr[device] = static_cast<double*>(p);
  }
  *out = g_addr[device];
  return RDM_OK;
}

}  // namespace
}  // namespace rdm

using namespace rdm;

extern "C" rdm_status rdm_starting_block_noalloc(rdm_ham* ham, int precision, int n_v, uint64_t seed,
                                                 int dist, void* x) {
  if (!ham || !x || n_v < 1) {
    set_error("rdm_starting_block_noalloc: NULL argument or n_v < 1");
    return RDM_EINVAL;
  }
  if (n_v > kNoAllocMaxVectors) {
    set_error("rdm_starting_block_noalloc: n_v = %d exceeds the maximum of %d bath vectors "
              "(fixed scratch of %zu bytes)", n_v, kNoAllocMaxVectors, kNoAllocScratchBytes);
    return RDM_EINVAL;
  }
  if (dist != RDM_RADEMACHER && dist != RDM_GAUSS && dist != RDM_BASIS) {
    set_error("rdm_starting_block_noalloc: bad distribution %d", dist);
    return RDM_EINVAL;
  }
  if (precision != RDM_FP32 && precision != RDM_FP64) {
    set_error("rdm_starting_block_noalloc: bad precision %d", precision);
    return RDM_EINVAL;
  }
  ham = ham->caller_view();  // x is in the caller's state order
  const HostModel& h = ham->model;
  const int ds = 1 << h.ns;
  if (dist == RDM_BASIS && (int64_t)n_v > (int64_t(1) << (h.n - h.ns))) {
    set_error("rdm_starting_block_noalloc: RDM_BASIS needs n_v <= d_b");
    return RDM_EINVAL;
  }
  // Same column layout rules as rdm_starting_block (one slice of d_s*n_v columns).
  Layout L{};
  L.n_bits = h.n;
  L.n_bath_bits = h.n - h.ns;
  L.D = int64_t(1) << h.n;
  L.DS = ds;
  L.precision = precision;
  L.elem = precision == RDM_FP32 ? 4 : 8;
  L.VW = precision == RDM_FP32 ? 4 : (ds == 4 ? 4 : 2);
  const int n_cols = ds * n_v;
  const int maxc = 128 / L.elem;
  int pow2 = L.VW;
  while (pow2 < n_cols) pow2 *= 2;
  if (n_cols < L.VW || n_cols > maxc || pow2 != n_cols) {
    set_error("rdm_starting_block_noalloc: %d columns unsupported: need %d * 2^m, at most %d",
              n_cols, L.VW, maxc);
    return RDM_EINVAL;
  }
  L.B = L.Bs = n_cols;
  L.n_slices = 1;
  L.TPR = n_cols / L.VW;
  const int rpb = kThreads / L.TPR;
  L.gridx = (int)std::min<int64_t>((L.D + rpb - 1) / rpb, 1216);

  if (cudaSetDevice(ham->ctx->device) != cudaSuccess) {
    set_error("rdm_starting_block_noalloc: cudaSetDevice failed");
    return RDM_ECUDA;
  }
  cudaStream_t s = ham->ctx->stream;
  double* norms = nullptr;
  if (dist == RDM_GAUSS) {
    double* scratch = nullptr;
    rdm_status st = scratch_address(ham->ctx->device, &scratch);
    if (st != RDM_OK) return st;
    // Layout of the scratch: inv_norm[0..n_v), then n_v * 64 partial sums. Every
    // entry the kernels read is written earlier in the same call, so nothing needs
    // clearing.
    norms = scratch;
    cudaError_t e = launch_gauss_norms(int64_t(1) << L.n_bath_bits, n_v, seed, 0, scratch + n_v, norms, s);
    if (e != cudaSuccess) {
      set_error("rdm_starting_block_noalloc: norm kernels failed: %s", cudaGetErrorString(e));
      return RDM_ECUDA;
    }
  }
  const cudaError_t e = launch_init_block(L, dist, seed, 0, n_v, norms, nullptr, x, s);
  if (e != cudaSuccess) {
    set_error("rdm_starting_block_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
    return RDM_ECUDA;
  }
  return RDM_OK;
}
