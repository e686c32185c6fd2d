/*
 * rdm.h -- C ABI of the GB300 library for the equilibrium-reduced density matrix
 * rho*_s = tr_b(exp(-beta H_t)) / Z_t and the mean-force Hamiltonian
 * H* = -ln(rho*_s)/beta of strongly coupled spin systems, computed with the
 * typicality + block-Lanczos estimator of Chen & Cheng, "Numerical computation of
 * the equilibrium-reduced density matrix for strongly coupled open quantum
 * systems" (arXiv:2204.08147).
 *
 * Conventions (Sec. 2.2, eq. Ht):
 *   - spins 1/2, sigma = Pauli matrices; sites 0..N-1, site 0 is the leftmost
 *     Kronecker factor, i.e. site q is bit (N-1-q) of a basis-state index s, and a
 *     0 bit is spin up (Z = +1);
 *   - the system is sites 0..N_s-1 (the top N_s bits of s), the bath the rest:
 *     s = i*d_b + b with system index i < d_s = 2^N_s and bath index b < d_b;
 *   - couplings are given once per unordered pair a < b.
 *
 * Every function returns an rdm_status; no C++ exception crosses this boundary.
 * On failure, rdm_last_error() returns a thread-local message describing it.
 * All host arrays are owned by the caller. Handles and the device memory the
 * library allocates for them are owned by the library.
 */
#ifndef RDM_H
#define RDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rdm_ctx rdm_ctx;
typedef struct rdm_ham rdm_ham;

typedef enum {
  RDM_OK = 0,
  RDM_EINVAL = -1,   /* invalid argument or unsupported size */
  RDM_ENOMEM = -2,   /* device or host memory exhausted, or workspace too small */
  RDM_ECUDA = -3,    /* a CUDA runtime call failed */
  RDM_ENUMERIC = -4, /* a non-finite Lanczos coefficient or Gram entry */
  RDM_ETIMEOUT = -5, /* rdm_wait gave up before the request finished */
  RDM_EBUSY = -6,    /* request still pending (rdm_poll) */
  RDM_ENOTPD = -7,   /* rho is not positive definite: ln(rho) undefined */
  RDM_ENOTFOUND = -8 /* unknown request ticket */
} rdm_status;

/* Arithmetic of the Lanczos vectors and the matrix-free SpMM. Recurrence
 * scalars, the eigendecomposition of T, exp(-beta T/2), the Gram and ln Z are
 * float64 in both modes. With RDM_FP32 the vectors, the SpMM and psi = Q c are
 * float32 with float32 accumulation; the Gram psi^T psi (eq. rho_est) is accumulated
 * in float64 from the first product on (a product of two float32 values is exact in
 * float64); the inner products behind the recurrence scalars (A_j = Q_j^T Z and the
 * QR Gram Z^T Z) are summed in float32 within a thread and a warp and in float64
 * across warps and blocks, and everything after that is float64. */
enum { RDM_FP64 = 0, RDM_FP32 = 1 };

/* Distribution of the bath vectors |v_l> (Sec. 3.1, eq. trace_est), drawn from a
 * counter-based generator: the n-th output of SplitMix64 (Steele, Lea & Flood
 * 2014) seeded with `seed`, mix(seed + n*0x9E3779B97F4A7C15), at counter
 * n = ((l << 40) | b) + 1 for element b of vector l (Gaussian: counters for 2b
 * and 2b+1).
 *   RDM_RADEMACHER: +-1/sqrt(d_b), sign = top bit of the draw;
 *   RDM_GAUSS:      Box-Muller cos(2 pi u2) sqrt(-2 ln u1), u = ((draw>>11)+0.5)/2^53,
 *                   then normalised to unit Euclidean norm;
 *   RDM_BASIS:      v_l = e_l; with n_v = d_b the average is the exact partial
 *                   trace (Sec. 2.1), used for exactness tests. */
enum { RDM_RADEMACHER = 0, RDM_GAUSS = 1, RDM_BASIS = 2 };

/* Which estimator form fills rdm_result.rho (the other fills rho_other).
 *   RDM_GRAM:       psi_l = Q_l exp(-beta (T_l - E0)/2) E1, G_l = psi_l^T psi_l
 *                   (the function-application form of the sqrt(rho) construction
 *                   of Sec. 2.1);
 *   RDM_QUADRATURE: G_l = E1^T exp(-beta (T_l - E0)) E1 (eq. fT, trB_est).
 * Both are normalised as eq. rho_est. They agree while Q_l^T Q_l = I. */
enum { RDM_GRAM = 0, RDM_QUADRATURE = 1 };

/* rdm_result.flags bits */
#define RDM_FLAG_DEFLATED 1u   /* a Lanczos column was dropped (Krylov breakdown) */
#define RDM_FLAG_PADDED 2u     /* n_v was padded with zero vectors for alignment */

/* A real spin-1/2 Hamiltonian (eq. Ht):
 *   H = sum_{a<b} s_ab (jx[a,b] X_a X_b + jy[a,b] Y_a Y_b + jz[a,b] Z_a Z_b)
 *     + sum_q (hz[q] Z_q + gx[q] X_q),
 * s_ab = lambda_sb if exactly one of a, b is a system site, else 1 (the
 * epsilon-scaled coupling of Sec. 5.5). jx, jy, jz are n_sites*n_sites row-major
 * arrays of which entries [a*n_sites + b] with a < b are read; hz, gx have
 * n_sites entries (hz is the paper's h/2). Any pointer may be NULL (all zero).
 * Limits: 1 <= n_sites <= 30, 0 <= n_sys <= 2, n_sys < n_sites. */
typedef struct {
  int n_sites;
  int n_sys;
  const double* jx;
  const double* jy;
  const double* jz;
  const double* hz;
  const double* gx;
  double lambda_sb;
} rdm_model;

/* How the Gram form obtains Q_1..Q_k (Algorithm 1 returns them all):
 *   RDM_PASSES_AUTO:      store them if k+1 Krylov blocks fit the device memory the
 *                         call may use; else, if those of a group of slices (bath
 *                         vectors) fit, rdm_estimate runs the bath vectors in consecutive
 *                         shards that each store their basis (one pass of the recurrence)
 *                         and folds them on the host with each shard's shift E0_r, as a
 *                         run split over GPUs is folded (results agree with one run to
 *                         rounding); else recompute;
 *   RDM_PASSES_STORE:     keep every block of pass 1 (k+1 blocks of D x B);
 *   RDM_PASSES_RECOMPUTE: keep 3 blocks and run the recurrence a second time with
 *                         the stored coefficients (bit-identical blocks).
 * STORE and RECOMPUTE give bit-identical results. */
enum { RDM_PASSES_AUTO = 0, RDM_PASSES_STORE = 1, RDM_PASSES_RECOMPUTE = 2 };

/* The Lanczos recurrences per bath vector:
 *   RDM_BLOCK:  one block Lanczos recurrence of block size d_s on I_s (x) |v_l>
 *               (Algorithm 1);
 *   RDM_SINGLE: one regular Lanczos recurrence (block size 1) per column e_i (x) |v_l>,
 *               the alternative named in Sec. 4.2 (exact for polynomials of lower degree
 *               at equal k). The Gram form takes G_l[i][j] = psi_{l,i}^T psi_{l,j}
 *               with psi_{l,i} = Q_{l,i} exp(-beta (T_{l,i} - E0)/2) e1; the quadrature
 *               form has only the diagonal e1^T exp(-beta (T_{l,i} - E0)) e1 (its
 *               off-diagonal entries are left zero). E0 is the smallest eigenvalue of all
 *               T_{l,i}; t_a/t_b hold each column's scalar coefficients on the diagonal.
 *               Needs float32, or float64 with d_s <= 2 (RDM_EINVAL otherwise). */
enum { RDM_BLOCK = 0, RDM_SINGLE = 1 };

typedef struct {
  int precision; /* RDM_FP64 | RDM_FP32 */
  int vec_dist;  /* RDM_RADEMACHER | RDM_GAUSS | RDM_BASIS */
  int form;      /* RDM_GRAM | RDM_QUADRATURE */
  int passes;    /* RDM_PASSES_* */
  int64_t first_vector; /* bath vectors l = first_vector .. first_vector+n_v-1 of the
                           seeded sequence (0 for a whole run; a shard of a run split
                           over GPUs starts further in, eq. trace_est is a sum over l) */
  int recurrence; /* RDM_BLOCK | RDM_SINGLE */
} rdm_opts;

/* Outputs of rdm_estimate; every pointer is a caller-owned host array. rho is
 * required, the rest may be NULL. Per-vector arrays are indexed [beta][l][i][j]
 * or [l][step][i][j], row-major, with d_s = 2^n_sys. */
typedef struct {
  double* rho;       /* n_beta*d_s*d_s: rho*_s(beta) in the chosen form (eq. rho_est) */
  double* ln_z;      /* n_beta: ln Z_t estimate, ln(d_b tr(sum_l G_l)/n_v) - beta E0 */
  double* rho_other; /* n_beta*d_s*d_s: rho* in the other form (diagnostic) */
  double* gram_l;    /* n_beta*n_v*d_s*d_s: un-normalised Gram-form G_l */
  double* quad_l;    /* n_beta*n_v*d_s*d_s: un-normalised quadrature-form G_l */
  double* t_a;       /* n_v*k*d_s*d_s: A_j of Algorithm 1 */
  double* t_b;       /* n_v*k*d_s*d_s: B_j of Algorithm 1 (upper triangular) */
  double e0;         /* out: the shift E0 = min_l lambda_min(T_l) (Sec. 3.2) */
  uint32_t flags;    /* out: RDM_FLAG_* */
  uint64_t h2d_bytes; /* out: host->device bytes this call copied (coefficients) */
  uint64_t d2h_bytes; /* out: device->host bytes this call copied (T, Gram, flags) */
} rdm_result;

/* ---------------------------------------------------------------- context */

/* Creates a context on CUDA device `device`. `stream` is a cudaStream_t owned by
 * the caller (NULL = the context creates and owns its own stream). Device work of
 * every call on this context is ordered on that stream. */
rdm_status rdm_create(rdm_ctx** out, int device, void* stream);
void rdm_destroy(rdm_ctx* ctx);

/* Attaches caller-owned device memory (e.g. a framework tensor) that rdm_estimate
 * carves its scratch from; NULL/0 detaches. The memory must stay valid and unused
 * by others while calls on this context run. Without an attached workspace the
 * context allocates its own (sized for the call, grown when a later call needs
 * more, kept between calls, freed by rdm_destroy). */
rdm_status rdm_set_workspace(rdm_ctx* ctx, void* device_ptr, size_t bytes);

/* Bytes of device scratch rdm_estimate needs for these sizes: with opts->passes
 * RDM_PASSES_STORE all k+1 Krylov blocks; otherwise the smallest recompute plan (3
 * Krylov blocks, the psi accumulators of one beta, reduction partials, coefficients).
 * A larger workspace lets rdm_estimate take more betas per pass-2 sweep, sweep slice
 * groups with every beta, keep the basis of one-pass shards or the whole basis. */
rdm_status rdm_workspace_size(const rdm_ham* ham, int n_beta, int n_v, int k,
                              const rdm_opts* opts, size_t* bytes);

/* Waits for all device work issued on the context's stream. */
rdm_status rdm_synchronize(rdm_ctx* ctx);

/* Measures the rate (GB/s into *gbs) at which TMA bulk copies fill shared memory: one
 * block per SM keeps `stages` (1..8) 32 KB copies in flight from a device buffer of
 * buffer_bytes (at least one 32 KB chunk per SM), >= 16 GB in total, timed with CUDA
 * events on the context's stream after one untimed launch. A buffer of up to 64 MB
 * stays in L2 (the L2 -> shared-memory rate, the level that feeds the tiled SpMM's
 * partner tiles); a buffer larger than L2 gives the DRAM -> shared-memory rate.
 * Allocates and frees its buffer; synchronous. RDM_ENOMEM if the buffer does not fit,
 * RDM_ECUDA if a copy wait gave up (a copy may then still be in flight into shared
 * memory: destroy the context rather than time anything further on it). The paper
 * has no counterpart: this is the
 * denominator of the SpMM's on-chip roofline. */
rdm_status rdm_probe_copy_rate(rdm_ctx* ctx, size_t buffer_bytes, int stages, double* gbs);

/* Launch mode of rdm_estimate's first pass (Algorithm 1's k steps, four kernels per
 * step). With enable != 0 (the default) a Hamiltonian handle records that launch
 * sequence as a CUDA graph the second time it runs one configuration (same
 * workspace, layout, k, precision and options) and replays the graph on later calls;
 * 0 launches every kernel directly. The kernels, their arguments and their order are
 * the same either way, so results are bit-identical. Graphs are not used while
 * rdm_profile is recording (each launch is timed on its own) nor by the serving
 * loop. The paper has no counterpart: this is launch overhead only. */
rdm_status rdm_set_graphs(rdm_ctx* ctx, int enable);

/* Where rdm_estimate's small dense step runs (Sec. 3.1-3.2, eq. fT:
 * exp(-beta (T_l - t_l)/2) E1 for every bath vector l and beta, t_l = lambda_min(T_l)).
 * On the device: t_l by multisection on the inertia of the block LDL^T factors of
 * T_l - sigma I (float32 rounds, then float64), then a Chebyshev expansion of the
 * exponential on [t_l, top of the spectrum] whose coefficients are scaled Bessel values
 * e^-w I_i(w) from Miller's backward recurrence; float64, within ~1e-13 of the host path
 * on the Gram. On the host: tridiagonal reduction, implicit QR, rotations applied back
 * for every beta, on the host worker pool. mode 0: always the host; 1 (the default):
 * the device for beta grids of at least 8 points (where the host's per-beta
 * back-transformation dominates) when T_l fits (k d_s^2 <= 5120); 2: the device
 * whenever T_l fits. rdm_estimate_batch launches the device steps of all its items at
 * once. RDM_EINVAL for another mode. The paper has no counterpart. */
rdm_status rdm_set_device_dense(rdm_ctx* ctx, int mode);

/* Thread-local description of the last failure on this thread ("" if none). */
const char* rdm_last_error(void);

/* Per-kernel statistics of the work issued through a context: launches, device
 * time (CUDA events recorded on the launching stream around each launch of the
 * timed kernels) and algorithmic bytes (the compulsory device-memory traffic of
 * each launch: blocks read and written once). */
typedef struct {
  char name[32];
  uint64_t launches;
  double ms;     /* summed event time; 0 for kernels that are only counted */
  double bytes;  /* summed algorithmic bytes */
} rdm_kernel_stat;

/* enable != 0 starts recording (and clears earlier statistics); 0 stops. */
rdm_status rdm_profile(rdm_ctx* ctx, int enable);
/* Copies up to `max` entries into out; *n = number of kinds recorded. The entry
 * "host_small_dense" is not a kernel: its ms is the host wall time of the small dense
 * step of rdm_estimate (eigen-solves of T_l and the Gram coefficients), launches the
 * number of estimates. */
rdm_status rdm_profile_stats(rdm_ctx* ctx, rdm_kernel_stat* out, int max, int* n);

/* ---------------------------------------------------------------- model */

/* Compiles a model into compact term descriptors (flip masks with their
 * aligned/anti-aligned coefficients, Z-parity masks, fields) and uploads them to
 * the context's device. The handle keeps a pointer to ctx; destroy it first. */
rdm_status rdm_build_hamiltonian(rdm_ctx* ctx, const rdm_model* model, rdm_ham** out);
void rdm_destroy_hamiltonian(rdm_ham* ham);

/* The bare bath Hamiltonian H_b of a model (Sec. 3.2): the terms of `model` acting on
 * bath sites only (sites n_sys .. n_sites-1, renumbered from 0; the spin at bath site q
 * keeps its bit, so bath basis states index alike), as a Hamiltonian with no system
 * sites (d_s = 1). rdm_estimate on it with the same seed, n_v, vector distribution and
 * first_vector as on the total model draws the same bath vectors v_l and returns in
 * ln_z the Lanczos quadrature estimate of ln Z_b = ln tr exp(-beta H_b), the
 * denominator of eq. H_est. Free with rdm_destroy_hamiltonian. Errors as
 * rdm_build_hamiltonian. */
rdm_status rdm_build_bath_hamiltonian(rdm_ctx* ctx, const rdm_model* model, rdm_ham** out);

/* The bare system Hamiltonian H_s of a model (its terms on system sites only) as a
 * dense d_s x d_s row-major real matrix, host, d_s = 2^n_sys (eq. Ht restricted to
 * the system; the basis order of rho). RDM_EINVAL as rdm_build_hamiltonian. */
rdm_status rdm_system_hamiltonian(const rdm_model* model, double* hs_out);

/* Bath-bit order. rdm_build_hamiltonian may store a Hamiltonian with its bath sites in
 * another order than the caller's: the order that minimises the partner tiles the
 * tiled SpMM copies per tile (flip masks are grouped by their bits above the tile's
 * 10 in-tile bits; sites coupled to many others belong in the tile), found by a
 * deterministic local search over transpositions of bath sites from the coupling graph
 * (the ladder of Sec. 5.2 numbered leg by leg goes from 13.5 to 8.5 partner tiles),
 * skipped when no order can differ (the set of flip masks maps onto itself under every
 * swap of neighbouring bath sites: a field on every site, all-to-all couplings) and
 * kept per structure for models that repeat one with other couplings. Only the device layout
 * changes: rdm_estimate draws the bath vectors in the caller's bath order, so results
 * equal those of the caller's order up to rounding, and rdm_apply_hamiltonian /
 * rdm_starting_block keep the caller's state order. The paper has no counterpart.
 * rdm_set_bath_order(ctx, 0) keeps the caller's order for Hamiltonians built afterwards
 * on ctx (default 1). rdm_bath_order (host only, no device) reports the order chosen for
 * a model: order_out[q] = caller site at internal site q (n_sites entries; system sites
 * unchanged), and the average partner tiles per tile in the caller's order and in the
 * chosen one. Any output pointer may be NULL; RDM_EINVAL as rdm_build_hamiltonian. */
rdm_status rdm_set_bath_order(rdm_ctx* ctx, int enable);
rdm_status rdm_bath_order(const rdm_model* model, int* order_out, double* tiles_caller,
                          double* tiles_chosen);

/* Sizes and the bound ||H||_2 <= sum of |term coefficients| used to scale the
 * Lanczos breakdown tolerance. Any output pointer may be NULL. */
rdm_status rdm_hamiltonian_info(const rdm_ham* ham, int* n_sites, int* n_sys,
                                int* n_flip_terms, int* n_diag_terms, double* norm_bound);

/* ---------------------------------------------------------------- hot path */

/* The estimator (eq. trB_est with eq. rho_est and the E0 shift of Sec. 3.2):
 * n_v bath vectors, each running k steps of block Lanczos (Algorithm 1) with
 * block size d_s from V_l = I_s (x) |v_l>, all n_v recurrences batched into one
 * matrix-free block SpMM; then exp(-beta (T_l - E0)/2) for every beta of the grid
 * and the bath-traced d_s x d_s Gram, averaged over l and trace-normalised.
 * betas: n_beta >= 1 values >= 0 (host). 1 <= n_v <= 4096, 1 <= k <= 512.
 * Blocking: returns when the results are in `out` (host). */
rdm_status rdm_estimate(rdm_ham* ham, const double* betas, int n_beta, int n_v, int k,
                        uint64_t seed, const rdm_opts* opts, rdm_result* out);

/* One estimate of a batch (rdm_estimate_batch): the arguments of rdm_estimate, and the
 * item's own status on return. */
typedef struct {
  rdm_ham* ham;          /* a Hamiltonian of the batch's context */
  const double* betas;   /* n_beta values (host, caller-owned) */
  int n_beta;
  int n_v;
  int k;
  uint64_t seed;
  rdm_opts opts;
  rdm_result* out;       /* caller-owned results, as for rdm_estimate */
  rdm_status status;     /* out: this item's status */
} rdm_batch_item;

/* Many estimates at once, of Hamiltonians of any sizes (the paper's independent
 * recurrences of Sec. 3.1, over several models): every item that keeps its Krylov basis
 * (k+1 blocks fit) and whose block is at most 64 MB runs its first pass (Algorithm 1's k
 * steps) in ONE persistent cooperative launch with the other such items of its
 * precision and d_s -- the SpMM, A_j, orthogonalisation and QR phases of every item,
 * separated by grid barriers; larger items run as rdm_estimate does. Each work unit of
 * that launch is one block of the plain kernels of its item, so an item's result does
 * not depend on which other items share the batch (bit-identical alone or in any mix).
 * Its launch form is chosen by an autotuner: the cooperative grid with 1, 2, 4 or 8
 * blocks per SM (as many as fit; grid barriers between the phases of a step), or one
 * block per slice of each item running all its steps with block barriers only (the
 * recurrences of a slice read nothing of other slices; no co-residency needed). The
 * first batch of each size class times the candidates and the fastest is kept on the
 * context; every form runs the same units with the same arithmetic, so the choice
 * changes no result (rdm_set_packed_form restricts it).
 * Items whose workspaces do not fit the device together run in consecutive
 * sub-batches. Blocking. Returns RDM_OK when every item succeeded, else the first
 * failure (each item's own status is in items[i].status); RDM_EINVAL for a NULL
 * argument or an item of another context, RDM_ECUDA if a grid-barrier wait gave up. */
rdm_status rdm_estimate_batch(rdm_ctx* ctx, rdm_batch_item* items, int n_items);

/* The autotuner's state on a context: size classes tuned (*n_keys) and candidate
 * launches timed so far (*tuning_runs). Either pointer may be NULL. */
rdm_status rdm_packed_tuning(rdm_ctx* ctx, int* n_keys, uint64_t* tuning_runs);

/* Which SpMM rdm_estimate's recurrences use: 0 (the default) the tiled kernel (bulk
 * copies of 1024-state tiles into a shared-memory ring, 152 persistent blocks) when the
 * layout allows it and the block has at least 32 tiles in all, else the plain kernel
 * (a block per row range and slice; tiny problems leave most persistent blocks idle);
 * 1 the tiled kernel whenever the layout allows it; 2 always the plain kernel. Results
 * agree within rounding (float64: ~1e-15 relative). rdm_apply_hamiltonian always takes
 * the tiled kernel where it can. RDM_EINVAL for another value. */
rdm_status rdm_set_spmm_form(rdm_ctx* ctx, int form);

/* Launch forms rdm_estimate_batch's first pass may take: 0 (the default) any, chosen
 * by the autotuner; 1 only the cooperative grid; 2 only one block per slice. The
 * tuned choices of the context are cleared. RDM_EINVAL for another value. */
rdm_status rdm_set_packed_form(rdm_ctx* ctx, int form);

/* Y = H X for a caller-owned device block of n_cols columns stored state-major,
 * vector-minor (element (s, c) at s*n_cols + c), float64 (RDM_FP64) or float32
 * (RDM_FP32). n_cols must be 2^m times 4 (FP32) or 2 (FP64), at most 32 (FP32) or
 * 16 (FP64). X and Y must not overlap. Asynchronous on the context's stream,
 * except when the block takes the tiled SpMM (32-byte rows: n_cols = 8 FP32 or
 * 4 FP64, N >= 10): then the call waits for the kernel to read back its copy-ring
 * status (RDM_ECUDA if a copy wait gave up). This is the SpMM of the hot path (the
 * matrix-vector products of Sec. 2.4), exposed for verification. */
rdm_status rdm_apply_hamiltonian(rdm_ham* ham, int precision, const void* x, void* y,
                                 int n_cols);

/* Fills a caller-owned device block (state-major, d_s*n_v columns, same column
 * rules as rdm_apply_hamiltonian) with the starting block V = [I_s (x) |v_l>]_l:
 * element (s, l*d_s + i) = [s >> N_b == i] * v_l[s & (d_b - 1)] (Sec. 3.1).
 * Asynchronous on the context's stream. */
rdm_status rdm_starting_block(rdm_ham* ham, int precision, int n_v, uint64_t seed,
                              int vec_dist, void* x);

/* The starting block of rdm_starting_block, computed without allocating device
 * memory. The paper has no counterpart: this is a service for callers that may not
 * allocate device memory themselves, e.g. code running inside a framework whose
 * caching allocator owns the device memory budget (a side cudaMalloc can fail or
 * fragment it), or latency-critical loops where cudaMalloc/cudaFree would
 * synchronise the device. Same arguments, layout and result as
 * rdm_starting_block; x is still caller-owned device memory.
 * Scratch: the Gaussian vectors' norms use a fixed device array of this library
 * (32 * 65 float64 = 16,640 bytes), which every GPU that loads the library holds
 * until the process exits. n_v may be at most 32 (the most the column rule allows:
 * d_s * n_v <= 32 float32 columns with d_s = 1); larger n_v returns RDM_EINVAL, as
 * does any n_v whose d_s * n_v columns break the column rule. The first call on a
 * device looks up the array's device address (once per device, with that device
 * current) and caches it for the life of the process; make that first call before
 * any stream capture, and do not use this entry point after a cudaDeviceReset of
 * that device (the array may move). All calls share the one array: calls whose device work overlaps
 * (different streams, or different contexts on the same device) race on it and
 * must be ordered by the caller. Each call writes every scratch entry it reads,
 * so no clearing is needed between calls. */
rdm_status rdm_starting_block_noalloc(rdm_ham* ham, int precision, int n_v, uint64_t seed,
                                      int vec_dist, void* x);

/* ---------------------------------------------------------------- post-processing
 * Host float64, no device work. rho is d_s x d_s row-major, symmetric. */

/* H_out = -(1/beta) ln(rho) through the eigendecomposition of rho (Sec. 3.2 end:
 * transform eigenvalues, no matrix logarithm): H* up to the additive constant
 * -(1/beta) ln Z*. RDM_ENOTPD if an eigenvalue of rho is <= 0. 1 <= d_s <= 64,
 * beta > 0. */
rdm_status rdm_mean_force(const double* rho, int d_s, double beta, double* h_out);

/* H*(beta) with its constant, eq. H_est (Sec. 3.2):
 *   H* = -(1/beta) ln(Z_t rho* / Z_b) = -(1/beta) ln(rho*) - (1/beta)(ln Z_t - ln Z_b) I,
 * from rho* and ln Z_t of rdm_estimate on the total model and ln Z_b of rdm_estimate on
 * rdm_build_bath_hamiltonian of the same model (same bath vectors). Errors as
 * rdm_mean_force; RDM_EINVAL for non-finite ln_z_t or ln_z_b. */
rdm_status rdm_mean_force_abs(const double* rho, int d_s, double beta, double ln_z_t,
                              double ln_z_b, double* h_out);

/* Deviation of the system's internal energy by the coupling (Sec. 5.3.2, eq.
 * deviation_of_Hamiltonian): tr(H* rho*) - tr(H_s rho_s) with
 * rho_s = exp(-beta H_s) / tr exp(-beta H_s). h_star from rdm_mean_force_abs, h_s
 * from rdm_system_hamiltonian, all d_s x d_s row-major host arrays. */
rdm_status rdm_energy_deviation(const double* rho, const double* h_star, const double* h_s,
                                int d_s, double beta, double* out);

/* S = -tr(rho ln rho) = -sum_i p_i ln p_i with 0 ln 0 = 0 (Sec. 5.3.1). */
rdm_status rdm_entropy(const double* rho, int d_s, double* s_out);

/* The small dense step of rdm_estimate for one recurrence (eq. fT, Sec. 3.1-3.2):
 * c_beta = exp(-beta (T - t_min I) / 2) E1 for every beta of the grid, where T is the
 * symmetric n x n matrix t (row-major; the block tridiagonal T_l of Algorithm 1 with
 * blocks of p = d_s, n = k p), E1 its first p columns of the identity and t_min its
 * smallest eigenvalue (returned in *t_min; rdm_estimate rescales by
 * exp(-beta (t_min - E0) / 2) once the common E0 is known). c: n_beta * n * p, row-major
 * per beta. Computed without eigenvectors: band or Householder reduction to
 * tridiagonal form, implicit QR, rotations applied to E1 and back. Host float64;
 * RDM_EINVAL for bad sizes, a negative or non-finite beta or a non-finite T,
 * RDM_ENUMERIC if the QR iteration does not converge. */
rdm_status rdm_function_of_t(int n, int p, const double* t, int n_beta, const double* betas,
                             double* t_min, double* c);

/* rdm_function_of_t for n_mat matrices at once (t: n_mat*n*n, t_min: n_mat,
 * c: n_mat*n_beta*n*p), spread over the host worker pool that rdm_estimate's small
 * dense step uses; several callers may run at once. Same per-matrix results as
 * rdm_function_of_t; RDM_ENUMERIC names the first matrix that did not converge. */
rdm_status rdm_function_of_t_batch(int n_mat, int n, int p, const double* t, int n_beta,
                                   const double* betas, double* t_min, double* c);

/* Eigendecomposition of a dense symmetric n x n matrix (row-major a), used by
 * the small dense step of the estimator: w ascending (n), v (n*n, row-major,
 * column j = eigenvector j; NULL for values only). Host float64. */
rdm_status rdm_symmetric_eig(int n, const double* a, double* w, double* v);

/* ---------------------------------------------------------------- serving
 * A request loop on the context (continuous batching): requests are queued, admitted
 * while their device footprint fits the context's budget, and run concurrently by up
 * to max_inflight workers, each on its own stream, so requests that arrive while
 * others run overlap with them. A request small enough for the packed first pass
 * (its basis stored, at most a quarter of the budget) joins the other queued such
 * requests a worker takes along, and they run as one rdm_estimate_batch (first passes
 * in one launch); others run as rdm_estimate. Each request's result is the same served
 * alone or in any mix (bit for bit for the packed requests). The result arrays of a
 * request must stay valid until rdm_poll/rdm_wait reports completion. */

/* hbm_budget_bytes: device bytes the loop may hold for requests at once;
 * max_inflight: how many requests may run concurrently (>= 1). */
rdm_status rdm_serve_start(rdm_ctx* ctx, size_t hbm_budget_bytes, int max_inflight);
rdm_status rdm_serve_stop(rdm_ctx* ctx);

/* Queues a copy of the request (the model is copied; betas are copied) and
 * returns a ticket. `out` is written when the request completes. */
rdm_status rdm_submit(rdm_ctx* ctx, const rdm_model* model, const double* betas, int n_beta,
                      int n_v, int k, uint64_t seed, const rdm_opts* opts, rdm_result* out,
                      uint64_t* ticket);

/* RDM_OK with *status_out the request's own status when it has finished,
 * RDM_EBUSY while pending, RDM_ENOTFOUND for an unknown ticket. Finished tickets
 * stay queryable until rdm_serve_stop. */
rdm_status rdm_poll(rdm_ctx* ctx, uint64_t ticket, rdm_status* status_out);

/* As rdm_poll but waits up to timeout_ms (< 0: forever); RDM_ETIMEOUT on expiry. */
rdm_status rdm_wait(rdm_ctx* ctx, uint64_t ticket, int timeout_ms, rdm_status* status_out);

/* Wall-clock seconds from submission to completion of a finished ticket and the
 * part of it spent queued before admission. RDM_EBUSY while pending. */
rdm_status rdm_request_times(rdm_ctx* ctx, uint64_t ticket, double* latency_s, double* queued_s);

#ifdef __cplusplus
}
#endif

#endif /* RDM_H */
