// Host-side structures behind the opaque ABI handles.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "rdm_internal.h"

namespace rdm {

// A model compiled to term descriptors (host copy).
struct HostModel {
  int n = 0, ns = 0;
  double lambda = 1.0;
  double hnorm = 0.0;  // sum of |coefficients|, an upper bound on ||H||_2
  std::vector<FlipTerm> flips;
  std::vector<DiagTerm> diags;
  // internal bath bit i carries the caller's bath bit bath_src[i] (empty: caller's order)
  std::vector<uint8_t> bath_src;
  BathPerm perm() const {
    BathPerm p{};
    p.n = (int)bath_src.size();
    for (int i = 0; i < p.n; ++i) p.src[i] = bath_src[i];
    return p;
  }
};

struct ServeState;

// Launch shape of the packed first pass chosen by measurement (the autotuner of
// rdm_estimate_batch): per key (precision, d_s, size class of the batch), the blocks per
// SM of the cooperative grid that ran fastest. The shape does not change any result
// (every work unit is one block of a plain launch whatever block runs it).
struct PackedTuning {
  std::mutex mu;
  std::map<uint64_t, int> blocks_per_sm;
  uint64_t tuning_runs = 0;  // candidate launches timed so far
};

// Launch statistics with CUDA-event timing on the launching stream.
enum KernelKind {
  kKInit = 0, kKSpmm1, kKSpmm2, kKOrth1, kKOrth2, kKPsiInit, kKGram, kKSmall, kKApply,
  kKPacked,     // the packed first pass of a batch (one cooperative launch)
  kKDense,      // the small dense step on the device (bounds, Chebyshev vectors, combination)
  kKPsiBatch,   // pass 2: psi updated from several kept basis blocks at once
  kKHostDense,  // not a kernel: host wall time of the small dense step (eigen + coefficients)
  kKNumKinds
};
struct Profiler {
  bool on = false;
  uint64_t launches[kKNumKinds] = {};
  double ms[kKNumKinds] = {};
  double bytes[kKNumKinds] = {};
  std::vector<cudaEvent_t> events;  // pool, reused
  std::vector<std::pair<int, int>> pending;  // (kind, index of the start event)
  int next = 0;
  static const char* name(int k);
  void reset();
  // Counts a launch; with `timed`, records events around it (call before/after).
  int begin(int kind, cudaStream_t s, bool timed);
  void end(int kind, int ev, cudaStream_t s, double bytes);
  // After the stream has been synchronised: folds pending event pairs into ms.
  void collect();
  ~Profiler();
};

}  // namespace rdm

struct rdm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  char* ws = nullptr;  // caller-attached workspace
  size_t ws_bytes = 0;
  char* own_ws = nullptr;  // context-owned workspace, grown on demand, kept between calls
  size_t own_bytes = 0;
  std::unique_ptr<rdm::ServeState> serve;
  rdm::Profiler prof;
  bool graphs = true;  // replay repeated pass-1 configurations from CUDA graphs
  bool bath_order = true;  // rdm_build_hamiltonian reorders bath bits for the tiled SpMM
  int device_dense = 1;  // small dense step: 0 host, 1 device for grids of >= 8 betas, 2 device
  int packed_form = 0;   // packed first pass: 0 autotuned, 1 cooperative grid only, 2 per-slice only
  int spmm_form = 0;     // estimator SpMM: 0 tiled from 32 tiles on, 1 tiled, 2 untiled
  rdm::PackedTuning tuning;
  rdm_ctx();
  ~rdm_ctx();  // defined where ServeState is complete
};

namespace rdm {
// TMA bulk-copy rate probe (kernels.cu): `stages` 32 KB copies in flight per SM into
// shared memory from n_chunks chunks of src, iters copies per block (one block per SM).
cudaError_t launch_probe_copy(const void* src, int64_t n_chunks, int iters, int stages, bool keep_in_l2,
                              uint32_t* err, cudaStream_t st);

// The pass-1 launch sequence of one estimator configuration (Algorithm 1's k steps:
// SpMM, A_j, orthogonalisation, B_j) captured as a CUDA graph. Its kernels take only
// device pointers and sizes fixed by the configuration, so a graph recorded for one
// call replays any later call whose key (workspace pointers, layout, k, thresholds)
// is the same. A configuration is captured on its second use, so one-off calls pay
// no capture cost.
struct Pass1Graph {
  std::mutex mu;
  std::vector<uint64_t> seen, key;  // last configuration run; the captured one
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;  // capture needs a stream other than the legacy default
  void reset();
  ~Pass1Graph() { reset(); }
};
}  // namespace rdm

struct rdm_ham {
  rdm_ctx* ctx = nullptr;
  int device = 0;
  rdm::HostModel model;
  void* d_terms = nullptr;  // owns flips, diags and the tiled tables
  rdm::FlipTerm* d_flips = nullptr;
  rdm::DiagTerm* d_diags = nullptr;
  rdm::TiledTerms tiled{};
  void* d_apply_aux[2] = {};  // tiled apply: error word + K table (float64, float32)
  rdm::Pass1Graph graph;
  // With reordered bath bits: the same model in the caller's order, for the entry points
  // whose device blocks are in the caller's state order (apply, starting block).
  rdm_ham* caller = nullptr;
  rdm_ham* caller_view() { return caller ? caller : this; }
};

namespace rdm {

void set_error(const char* fmt, ...);
rdm_status compile_model(const rdm_model* m, HostModel* out);
// Partner tiles a 2^kTileBits-state tile of the tiled SpMM copies, on average, for this
// term list: one per distinct high part of the flip masks, half for a group that only
// hops a pair of high spins with a parity-only coefficient (the tiles where that pair is
// antiparallel).
double partner_tiles(const HostModel& h);
// Reorders the bath bits of h (deterministic local search) when that lowers
// partner_tiles; records the order in h->bath_src.
void order_bath_bits(HostModel* h);
// rec_ds: block size of one recurrence (-1: d_s; 1: one recurrence per column)
rdm_status plan_layout(const HostModel& h, int n_v, int precision, Layout* L, int* n_v_pad,
                       int rec_ds = -1);
rdm_status check_estimate_args(const rdm_ham* ham, const double* betas, int n_beta,
                               const rdm_opts* opts, const rdm_result* out);
// Runs the whole estimator on stream s, carving its scratch from ws/ws_bytes.
rdm_status estimate_impl(rdm_ham* ham, cudaStream_t s, char* ws, size_t ws_bytes,
                         const double* betas, int n_beta, int n_v, int k, uint64_t seed,
                         const rdm_opts* o, rdm_result* out, Profiler* prof);
// Host image of every device-side term table of a model (flips, diagonal terms and
// the tiled SpMM's pattern tables), uploaded with one copy.
struct TermImage {
  std::vector<unsigned char> bytes;
  size_t off_flips = 0, off_diags = 0, off_pat_high = 0, off_pat_start = 0, off_pat_flags = 0,
         off_term_low = 0, off_term_odd = 0, off_term_even = 0, off_dg_low = 0, off_dg_mlo = 0,
         off_dg_hstart = 0, off_dg_thi = 0, off_dg_tc = 0, off_dg_slot = 0, off_tile_order = 0;
  int n_pat = 0, n_pair = 0, n_terms = 0, all_active = 1, partners_flat = 0, all_uniform = 1, n_reg0 = 0, n_dg_groups = 0,
      n_dg_terms = 0, dg_entries = 0;
  uint32_t dg_dep = 0;
  int dg_off[8] = {};
};
// Order of the tiled SpMM's walk over the 2^b tiles of a slice (a permutation).
std::vector<uint32_t> tile_walk_order(int b);
void make_term_image(const HostModel& h, TermImage* img);
// Points ham's device term pointers into `dev`, a device copy of img.bytes.
void bind_terms(const TermImage& img, char* dev, rdm_ham* ham);

// Runs the items of a batch on stream s with workspace ws (need[i] bytes per item after
// the packed launches' descriptors); see rdm_estimate_batch.
rdm_status estimate_batch_impl(rdm_ctx* ctx, cudaStream_t s, char* ws, size_t ws_bytes,
                               rdm_batch_item* items, int n, const size_t* need, Profiler* prof);
// Workspace of a batch (0 if an item's sizes are invalid); need[i] per item, planned
// with at most avail[i] bytes.
size_t batch_workspace_bytes(const rdm_batch_item* items, int n, const size_t* avail, size_t* need);
// Bytes of a request's workspace with its Krylov basis stored when the packed first
// pass can take it (block recurrences, block of at most 64 MB), else 0.
size_t packed_store_footprint(const HostModel& h, int n_beta, int n_v, int k, const rdm_opts* o,
                              double beta_max = -1.0);

// Device bytes estimate_impl needs with a pass-2 chunk of nbc betas.
// Bytes the estimator would use given `avail` bytes (0 if the sizes are invalid).
// beta_max: the largest beta of the grid (< 0: unknown; plans the device small dense
// step for its largest Chebyshev degree).
size_t estimate_bytes(const HostModel& h, int n_beta, int n_v, int k, const rdm_opts* o, size_t avail,
                      rdm_status* status = nullptr, double beta_max = -1.0);
size_t estimate_footprint(const HostModel& h, int n_beta, int n_v, int k, int precision, int dist,
                          int passes, int nbc, int recurrence = 0, double beta_max = -1.0);

}  // namespace rdm
