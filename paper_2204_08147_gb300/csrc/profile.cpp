// Launch counting and CUDA-event timing of the hot-path kernels (rdm_profile*), the
// first-pass launch mode and the bulk-copy rate probe.
#include <algorithm>
#include <cstring>

#include "rdm_api_internal.h"

namespace rdm {

const char* Profiler::name(int k) {
  static const char* names[kKNumKinds] = {"init_block", "spmm_pass1", "spmm_pass2",
                                          "orth_pass1", "orth_pass2", "psi_init",
                                          "final_gram", "small",      "apply",
                                          "packed_pass1", "dense_fT", "psi_batch",
                                          "host_small_dense"};
  return (k >= 0 && k < kKNumKinds) ? names[k] : "?";
}

void Profiler::reset() {
  for (int k = 0; k < kKNumKinds; ++k) {
    launches[k] = 0;
    ms[k] = 0.0;
    bytes[k] = 0.0;
  }
  pending.clear();
  next = 0;
}

int Profiler::begin(int kind, cudaStream_t s, bool timed) {
  if (!on) return -1;
  launches[kind]++;
  if (!timed) return -1;
  if (next + 2 > (int)events.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      events.push_back(e);
    }
  }
  const int idx = next;
  next += 2;
  cudaEventRecord(events[idx], s);
  pending.emplace_back(kind, idx);
  return idx;
}

void Profiler::end(int kind, int ev, cudaStream_t s, double b) {
  if (!on) return;
  bytes[kind] += b;
  if (ev >= 0) cudaEventRecord(events[ev + 1], s);
}

void Profiler::collect() {
  for (auto& p : pending) {
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, events[p.second], events[p.second + 1]) == cudaSuccess)
      ms[p.first] += t;
  }
  pending.clear();
  next = 0;
}

Profiler::~Profiler() {
  for (auto e : events) cudaEventDestroy(e);
}

}  // namespace rdm

using namespace rdm;

extern "C" rdm_status rdm_profile(rdm_ctx* ctx, int enable) {
  if (!ctx) {
    set_error("rdm_profile: ctx is NULL");
    return RDM_EINVAL;
  }
  if (enable) ctx->prof.reset();
  ctx->prof.on = enable != 0;
  return RDM_OK;
}

extern "C" rdm_status rdm_probe_copy_rate(rdm_ctx* ctx, size_t buffer_bytes, int stages, double* gbs) {
  constexpr size_t kChunk = 32768;
  if (!ctx || !gbs || stages < 1 || stages > 8) {
    set_error("rdm_probe_copy_rate: ctx and gbs must be non-NULL and 1 <= stages <= 8");
    return RDM_EINVAL;
  }
  *gbs = 0.0;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    set_error("rdm_probe_copy_rate: cudaSetDevice failed");
    return RDM_ECUDA;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int64_t n_chunks = (int64_t)(buffer_bytes / kChunk);
  if (sms <= 0 || n_chunks < sms) {
    set_error("rdm_probe_copy_rate: buffer must hold at least one 32 KB chunk per SM");
    return RDM_EINVAL;
  }
  // each block copies >= its share of the buffer once and >= 16 GB in total overall
  const int64_t by_total = ((int64_t)16 << 30) / ((int64_t)sms * (int64_t)kChunk);
  const int iters = (int)std::max<int64_t>((n_chunks + sms - 1) / sms, by_total);
  const bool keep = buffer_bytes <= ((size_t)64 << 20);
  char* buf = nullptr;
  uint32_t* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rdm_status st = RDM_OK;
  float ms = 0.f;
  uint32_t herr = 0;
  cudaStream_t s = ctx->stream;
  auto fail = [&](const char* what) {
    set_error("rdm_probe_copy_rate: %s: %s", what, cudaGetErrorString(cudaGetLastError()));
    st = RDM_ECUDA;
  };
  if (cudaMalloc(&buf, (size_t)n_chunks * kChunk) != cudaSuccess || cudaMalloc(&err, sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    set_error("rdm_probe_copy_rate: device allocation failed");
    st = RDM_ENOMEM;
  }
  if (st == RDM_OK && (cudaMemsetAsync(buf, 0, (size_t)n_chunks * kChunk, s) != cudaSuccess ||
                       cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess))
    fail("memset");
  if (st == RDM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    fail("event");
  // one untimed launch (fills L2 for a small buffer), then the timed one
  if (st == RDM_OK && launch_probe_copy(buf, n_chunks, iters, stages, keep, err, s) != cudaSuccess)
    fail("launch");
  if (st == RDM_OK && (cudaEventRecord(e0, s) != cudaSuccess ||
                       launch_probe_copy(buf, n_chunks, iters, stages, keep, err, s) != cudaSuccess ||
                       cudaEventRecord(e1, s) != cudaSuccess))
    fail("timed launch");
  if (st == RDM_OK && (cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
    fail("readback");
  if (st == RDM_OK && herr) {
    set_error("rdm_probe_copy_rate: a bulk-copy wait gave up");
    st = RDM_ECUDA;
  }
  if (st == RDM_OK) *gbs = (double)sms * iters * (double)kChunk / (ms * 1e-3) / 1e9;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  if (buf) cudaFree(buf);
  if (err) cudaFree(err);
  return st;
}

extern "C" rdm_status rdm_set_graphs(rdm_ctx* ctx, int enable) {
  if (!ctx) {
    set_error("rdm_set_graphs: ctx is NULL");
    return RDM_EINVAL;
  }
  ctx->graphs = enable != 0;
  return RDM_OK;
}

extern "C" rdm_status rdm_profile_stats(rdm_ctx* ctx, rdm_kernel_stat* out, int max, int* n) {
  if (!ctx || (!out && max > 0) || !n) {
    set_error("rdm_profile_stats: NULL argument");
    return RDM_EINVAL;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    set_error("rdm_profile_stats: stream synchronisation failed");
    return RDM_ECUDA;
  }
  ctx->prof.collect();
  *n = kKNumKinds;
  for (int k = 0; k < kKNumKinds && k < max; ++k) {
    std::memset(out[k].name, 0, sizeof out[k].name);
    std::strncpy(out[k].name, Profiler::name(k), sizeof out[k].name - 1);
    out[k].launches = ctx->prof.launches[k];
    out[k].ms = ctx->prof.ms[k];
    out[k].bytes = ctx->prof.bytes[k];
  }
  return RDM_OK;
}
