// Launch counting and CUDA-event timing of the hot-path kernels (rdm_profile*).
#include <cstring>

#include "rdm_api_internal.h"

namespace rdm {

const char* Profiler::name(int k) {
  static const char* names[kKNumKinds] = {"init_block", "spmm_pass1", "spmm_pass2",
                                          "orth_pass1", "orth_pass2", "psi_init",
                                          "final_gram", "small",      "apply",
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
