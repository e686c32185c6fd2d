// Internal declarations shared by the host translation units and the CUDA kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rdm.h"

#ifdef __CUDACC__
#define RDM_HD __host__ __device__
#else
#define RDM_HD
#endif

namespace rdm {

// One off-diagonal term family with flip mask m: H[s ^ m, s] = c_odd if
// popcount(s & m) is odd, c_even otherwise (eq. Ht). A pair (a, b) gives
// m = bit(a)|bit(b), c_odd = s_ab (jx + jy) (anti-aligned spins), c_even =
// s_ab (jx - jy) (aligned); a transverse field gives m = bit(q), c_odd = c_even = gx.
struct FlipTerm {
  uint32_t mask;
  uint32_t pad;
  double c_odd;
  double c_even;
};

// One diagonal term: contributes c * (1 - 2*parity(s & mask)), i.e. c * Z_a Z_b
// for a pair mask or c * Z_q for a single-site mask.
struct DiagTerm {
  uint32_t mask;
  uint32_t pad;
  double c;
};

// Geometry of a Krylov block in device memory. The B = d_s * n_v_pad columns are
// split into n_slices slices of Bs columns; slice k is a contiguous D x Bs
// state-major, vector-minor array starting at k * D * Bs. A thread owns VW
// consecutive columns (VW / DS whole bath-vector groups) of one row; TPR = Bs/VW
// threads cover a row of a slice.
struct Layout {
  int n_bits;      // N
  int n_bath_bits; // N_b
  int64_t D;       // 2^N
  int DS;          // d_s
  int B;           // columns (padded)
  int Bs;          // columns per slice
  int n_slices;
  int VW;          // columns per thread
  int TPR;         // threads per row of a slice
  int gridx;       // blocks per slice in the row dimension
  int precision;   // RDM_FP64 | RDM_FP32
  int elem;        // bytes per element
  RDM_HD int groups_per_slice() const { return Bs / DS; }
  RDM_HD int n_groups() const { return B / DS; }
  RDM_HD size_t block_bytes() const { return (size_t)D * (size_t)B * (size_t)elem; }
};

constexpr int kThreads = 256;

// Number of float64 reduction values per bath-vector group for each kernel kind.
inline int nv_full(int ds) { return ds * ds; }

// Per-step coefficient arrays (device, float64), each [step][group][DS*DS]:
//   mz   = M_j            (true Q_j = W_j M_j)
//   cp   = -M_{j-1} B_{j-1}^T
//   cw   = -M_j A_j
struct StepCoefs {
  double* mz;
  double* cp;
  double* cw;
};

// Bath-bit order of a Hamiltonian's internal state index: internal bath bit i carries
// the caller's bath bit src[i] (n = 0: the caller's order). The starting block maps an
// internal bath index back to the caller's before drawing v_l[b], so the same bath
// vectors enter whatever order the library chose.
struct BathPerm {
  int n;
  uint8_t src[32];
};

// ---- launchers (kernels.cu) ------------------------------------------------

// Zero vector blocks etc. are plain cudaMemsetAsync on the host side.

// Gaussian bath-vector norms: inv_norm[l] = 1/||g_l|| for l < n_v (float64),
// partials scratch of n_v * gx doubles. If graw is not NULL the raw values are kept
// there (graw[l][b], float64) for launch_gauss_fill.
cudaError_t launch_gauss_norms(int64_t d_b, int n_v, uint64_t seed, int64_t l0, double* partials,
                               double* inv_norm, cudaStream_t st, double* graw = nullptr);

// W = [I_s (x) v_l] for l < n_v_real, zero columns beyond; vector l of the block is
// vector l0 + l of the seeded sequence. Gaussian values come from inv_norm
// (computed on the fly) or, if inv_norm is NULL, from vbuf[l][b] (T). With sub > 1 the
// layout's groups are single columns (L.DS = 1) and column c = l sub + i holds
// e_i (x) v_l (the per-column recurrences).
cudaError_t launch_init_block(const Layout& L, int dist, uint64_t seed, int64_t l0, int n_v_real,
                              const double* inv_norm, const void* vbuf, void* W, cudaStream_t st,
                              int sub = 1, const BathPerm* bp = nullptr);
// vbuf[l][b] = normalised Gaussian bath vector l0 + l (T = the layout's precision),
// from graw (the norm pass's raw values) when given, else regenerated.
cudaError_t launch_gauss_fill(const Layout& L, int n_v, uint64_t seed, int64_t l0,
                              const double* inv_norm, void* vbuf, cudaStream_t st,
                              const double* graw = nullptr);

// Flip terms grouped for the tiled SpMM. In the tiled layout a row of a slice is
// kTiledLanes 16-byte vectors (32 bytes: 8 float32 / 4 float64 columns) and a tile
// is 2^kTileBits consecutive states of one slice, 32 KB. Narrow rows put many
// states into each byte of L2, so the partner tiles of a tile stay cached. A flip
// mask m splits into m_high = m >> kTileBits (which tile the partner row lies in,
// relative to this one: tile ^ m_high) and m_low (the row permutation inside that
// tile). Pattern p collects the terms with one m_high; pattern 0 has m_high = 0
// (in-tile terms). Flags: bit0 = every term has m_low = 0 (its activity is uniform
// over a tile), bit1/bit2 = some c_odd/c_even is nonzero.
constexpr int kTiledLanesLog = 1;
constexpr int kTiledLanes = 1 << kTiledLanesLog;
constexpr int kTileBits = 11 - kTiledLanesLog;
constexpr int kTileRows = 1 << kTileBits;
// A consumer thread of the tiled SpMM owns the rows r0 + m * 2^kTileRegShift of a
// tile (m = 0 .. 2^kTileRegBits - 1): the top kTileRegBits tile bits index its
// registers.
constexpr int kTileRegBits = 3;
constexpr int kTileRegShift = kTileBits - kTileRegBits;

// The diagonal of H inside the tiled SpMM, rebuilt per tile from a short table instead
// of read per state. For state s = (tile << kTileBits) | r and a diagonal term
// c (1 - 2 parity(s & m)) with m = (m_hi << kTileBits) | m_lo, the sign factorises as
// sigma(tile & m_hi) * sigma(r & m_lo), sigma(x) = 1 - 2 parity(x). So
//   diag(s) = low[r] + K_0(tile) + sum_g K_g(tile) sigma(r & mlo_g),
// where low[] sums the terms with m_hi = 0 (the same for every tile), K_0 the terms
// with m_lo = 0, and K_g the terms whose m_lo is the g-th distinct value mlo_g among
// the terms with both parts nonzero. A consumer thread of the SpMM owns the rows
// r = rg + 2^kTileRegShift m (m < 2^kTileRegBits), so with q_g = mlo_g >> kTileRegShift,
//   diag = low[r] + sum_q A_q(tile, rg) (-1)^popc(q & m),
//   A_q = [q = 0] K_0 + sum_{g: q_g = q} sigma(rg & mlo_g) K_g,
// a 2^kTileRegBits-point Walsh-Hadamard transform per thread. The A table holds, per tile, A_q for
// every rg (2^kTileRegShift entries at off[q]) when bit q of dep is set (some group of
// character q has a mask bit below kTileRegShift), else one entry (then the same for
// every rg). It is filled once per estimate (launch_tile_diag); groups are sorted by
// q_g, with hstart[q]..hstart[q+1] the groups of character q.
struct TileDiag {
  int n_groups;          // G: distinct mixed m_lo values
  int n_terms;           // terms with m_hi != 0
  uint32_t dep;          // bit q: A_q depends on the row group
  int off[8];            // element offset of A_q in a table row (q < 2^kTileRegBits)
  int n_entries;         // table entries per tile (before padding)
  const double* low;     // [kTileRows]
  const uint32_t* mlo;   // [G]
  const int* hstart;     // [9]
  const uint32_t* thi;   // [n_terms] m_hi, sorted by slot (0 = K_0, 1 + g = K_g)
  const double* tc;      // [n_terms] coefficients
  const int* slot_start; // [G + 2]
};
// Elements per tile row of the A table (n_entries rounded up to 16 bytes).
RDM_HD inline int tile_diag_stride(int n_entries, int elem) {
  const int per16 = 16 / elem;
  return (n_entries + per16 - 1) / per16 * per16;
}

struct TiledTerms {
  int n_pat;
  int n_pair;                 // patterns 1..n_pair: one high spin, the same in-tile hop
                              // partners, parity-only (consumed in opposite-spin pairs)
  int n_terms;
  int all_active;             // 1: every tile needs every partner pattern
  int partners_flat;          // 1: and each is one uniform term with m_low = 0
  int all_uniform;            // 1: every term has c_odd = c_even
  int n_reg0;                 // leading in-tile terms that act on register rows only
  const uint32_t* pat_high;   // [n_pat]
  const int* pat_start;       // [n_pat + 1]
  const uint32_t* pat_flags;  // [n_pat]
  const uint32_t* term_low;   // [n_terms]
  const double* term_odd;     // [n_terms]
  const double* term_even;    // [n_terms]
  const uint32_t* tile_order;  // [tiles per slice]: the walk's k-th tile of a slice
  TileDiag dg;
};

struct SpmmArgs {
  const FlipTerm* flips;
  int n_flip;
  const DiagTerm* diags;
  int n_diag;
  const void* w;       // W_j
  const void* w_prev;  // W_{j-1} (nullable)
  void* z;             // output
  const double* mz;    // [group][DS*DS] (nullable: identity, no mixing)
  const double* cp;    // [group][DS*DS]
  double* partials;    // PASS1 reduction partials (nullable)
  // pass 2: psi accumulation
  void* psi;           // [nb][block] (nullable)
  const double* e;     // [nb][group][DS*DS]
  int nb;
  int psi_first;       // 1: psi = w E (no read)
  TiledTerms tiled;    // n_pat = 0: not available
  const void* tile_k;  // [tiles][stride] A table of the tiled diagonal (launch_tile_diag)
  uint32_t* err;       // bit 0 set if a bulk-copy wait gave up
  int stages;          // tiled SpMM: copy-ring depth (set by the launcher)
};

// True if the tiled SpMM applies to this layout: rows of kTiledLanes 16-byte vectors
// (32 bytes: 8 float32 or 4 float64 columns) holding whole bath-vector groups, at least
// one full tile per slice. (The tiled kernel reads a row as kTiledLanes 16-byte lanes
// whatever L.VW the plain kernels use on the same memory.)
inline bool layout_tiled(const Layout& L) {
  return L.Bs * L.elem == 16 * kTiledLanes && L.Bs % L.DS == 0 && L.n_bits >= kTileBits;
}
// Blocks of the tiled SpMM (one persistent block per SM; the blocks walk the
// (slice, tile) pairs of the whole block with one stride).
inline int spmm_tiled_grid(const Layout& L) {
  const int64_t tiles = (L.D >> kTileBits) * L.n_slices;
  return (int)(tiles < 152 ? tiles : 152);
}

// A table of the tiled diagonal (TileDiag), out[tile][0 .. stride): summed in float64,
// stored in the layout's precision, padding zero.
cudaError_t launch_tile_diag(const Layout& L, const TileDiag& dg, void* out, cudaStream_t st);

enum SpmmMode { kModeApply = 0, kModePass1 = 1, kModePass2 = 2 };
cudaError_t launch_spmm(const Layout& L, int mode, const SpmmArgs& a, cudaStream_t st);

// W_{j+1} = Z + W_j Cw in place over Z; partials of W_{j+1}^T W_{j+1} if non-null.
cudaError_t launch_orth(const Layout& L, const void* w, void* z, const double* cw,
                        double* partials, cudaStream_t st);

// Per-group small steps.
cudaError_t launch_coef_init(const Layout& L, StepCoefs c1, cudaStream_t st);
// After the SpMM: A_j and Cw_j from the P1 partials.
cudaError_t launch_small_a(const Layout& L, const double* partials, const double* mz,
                           double* a_out, double* cw_out, uint32_t* flags, cudaStream_t st);
// After the orthogonalisation: B_j, M_{j+1}, Cp_{j+1} from the Gram partials.
cudaError_t launch_small_b(const Layout& L, const double* partials, const double* mz_j,
                           double* b_out, double* mz_next, double* cp_next, double thr_abs_sq,
                           double thr_rel_sq, int n_groups_real, uint32_t* flags,
                           cudaStream_t st);

// Pass 2: W_{j+1} = Z + W_j Cw in place over Z, then psi_beta += W_{j+1} E_beta for
// the nb betas of the chunk (psi blocks are consecutive, D*B elements apart).
cudaError_t launch_orth_psi(const Layout& L, const void* w, void* z, const double* cw, void* psi,
                            const double* e, int nb, cudaStream_t st);
// Pass 2 with the last m <= kPsiBatchMax blocks of the basis kept: psi_beta +=
// sum_{a < m} W_a E_{j0+a,beta} for the first nb betas, E of step j0 + a at e + a *
// estride; per element the same fma sequence as m single steps of launch_orth_psi.
constexpr int kPsiBatchMax = 8;
struct PsiBatch {
  const void* w[kPsiBatchMax];
};
cudaError_t launch_psi_batch(const Layout& L, const PsiBatch& wb, int m, void* psi, const double* e,
                             size_t estride, int nb, cudaStream_t st);
// Pass 2 start: psi_beta = W_1 E_{1,beta}.
cudaError_t launch_psi_init(const Layout& L, const void* w, void* psi, const double* e, int nb,
                            cudaStream_t st);
// Partials of psi^T psi per group for one psi block.
cudaError_t launch_final_gram(const Layout& L, const void* psi, double* partials, cudaStream_t st);
// Stored-basis Gram for betas b0..b0+nb-1 of the E array (beta stride nbs):
// partials for beta b0+i at partials + i*pstride.
cudaError_t launch_gram_stored(const Layout& L, const void* w1, int k, const double* e, int nbs,
                               int b0, int nb, double* partials, size_t pstride, cudaStream_t st);
// Betas one stored-basis Gram launch can take (0: the coefficients do not fit).
int gram_stored_max_betas(const Layout& L, int k);
// Sum gram partials -> gram[group][DS*DS].
cudaError_t launch_reduce_gram(const Layout& L, const double* partials, double* gram,
                               cudaStream_t st);

// One estimate's first pass inside the packed launch (k_pass1_packed). The layout is
// the untiled one (blocks of kThreads threads, gridx x n_slices per block-sized
// phase); blocks blk + j * block_bytes hold W_{j+1} (stored basis); coef holds
// M_j | Cp_j | Cw_j, each (k + 2) * n_groups * d_s^2 float64.
struct PackedItem {
  Layout L;
  SpmmArgs sa;  // term tables and the partials buffer; the block pointers are set per step
  char* blk;
  double* coef;
  double* ta;
  double* tb;
  uint32_t* flags;
  double thr_abs_sq, thr_rel_sq;
  int k, n_rec;
};
// A packed launch: items sorted by k (largest first); active[j] = items with k >= j;
// pre_rows / pre_groups: prefix sums over the items of their block-sized units
// (gridx * n_slices) and of their groups; bar: three zeroed words for the grid barrier
// (arrivals, generation, error).
struct PackedPlan {
  const PackedItem* items;
  int n_items;
  int k_max;
  const int* active;
  const int* pre_rows;
  const int* pre_groups;
  const int* pre_slices;  // prefix sums of the items' slices (the slice-local launch)
  uint32_t* bar;
};
// Blocks of the packed kernel that fit one SM with `smem` dynamic bytes (0: unsupported).
int packed_max_blocks_per_sm(int precision, int ds, size_t smem);
// Cooperative launch of the packed first pass on `grid` blocks (all co-resident).
cudaError_t launch_pass1_packed(int precision, int ds, const PackedPlan& pp, int grid, size_t smem,
                                cudaStream_t st);
// The same first pass with one block per (item, slice), pre_slices[n_items] blocks: each
// runs all k steps of its slice's recurrences with block barriers (no grid barrier, no
// co-residency needed); the units and their arithmetic are those of the packed launch.
cudaError_t launch_pass1_local(int precision, int ds, const PackedPlan& pp, int grid, size_t smem,
                               cudaStream_t st);
// Dynamic shared memory of the untiled SpMM's term tables.
size_t spmm_terms_smem(int precision, int n_flip, int n_diag);

// The small dense step on the device (dense.cu), for the n_rec recurrences of one
// estimate (a job): c[r][beta] = exp(-beta (T_r - t_r)/2) E1 (n x d_s, row-major per
// beta) and lohi[2r] = t_r = lambda_min(T_r), lohi[2r+1] = the top of the Chebyshev
// interval, from the step arrays ta, tb ([k][ng][d_s^2]); betas on the device; V
// scratch of n_rec * vstride * k d_s * d_s float64 (vstride = the Chebyshev degree
// bound + 1, dense_device_max_degree + 1).
struct DenseJob {
  int k, ng, n_rec, n_beta, vstride;
  double hnorm, beta_max;
  const double* ta;
  const double* tb;
  const double* betas;
  double* lohi;
  double* V;
  double* cout;
};
constexpr int kChebMaxDegree = 400;
bool dense_device_fits(int k, int ds);
int dense_device_max_degree(double beta_max, double hnorm);
// Device bytes of the descriptors of n_jobs jobs (scratch of launch_dense_jobs).
size_t dense_jobs_bytes(int n_jobs);
// One launch of each dense kernel over all recurrences of all jobs (same d_s).
cudaError_t launch_dense_jobs(int ds, const DenseJob* host_jobs, int n_jobs, void* scratch, cudaStream_t st);

constexpr uint32_t kFlagNonFinite = 0x100u;

}  // namespace rdm
