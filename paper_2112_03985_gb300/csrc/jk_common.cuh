// Internal declarations shared by the translation units of libjkcals.so.
//
// Device data layout (one handle):
//   Tn64[n]   FP64 mode-n unfolding T_(n), I_n x J_n row-major, columns in the
//             order of Eq. kolda_mapping (lowest other mode fastest)       [FP64 form]
//   U[n]      FP64 multi-matrix Ubar^(n), I_n x C row-major
//   gram[n]   FP64 Grams G^(n)_g = Ubar^(n)_{|g}^T Ubar^(n)_{|g}, block g at gram_off[g]
//             (R_g x R_g row-major, packed one block after another)
//   part      split-K partial MTTKRPs, S x I_n x C (FP64 or FP32 by form)
//   gpart     per (block, row chunk) partial Grams, K x RC x 32 x 32 FP64
//   fpart     per (block, row chunk) partial sum(U_N * M_N), K x RC FP64
//   normT2    ||T_{-g}||^2 per block, FP64
//   status    per-block status bits (JKCALS_BLOCK_*)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/jkcals.h"

namespace jk {

constexpr int kMaxModes = 8;
constexpr int kMaxRank = 32;

// Metadata of the blocks, device side.
struct BlockMeta {
  const int* R;          // K
  const int* off;        // K: first column of block g
  const int* gram_off;   // K: offset of block g's R_g x R_g Gram
  const int64_t* lo_ptr; // K+1
  const int64_t* lo_idx; // left-out sample indices (sorted within a block)
};

// Factor operands of the on-the-fly Khatri-Rao product of one mode.
struct KrpOperands {
  const double* U[kMaxModes - 1];  // other modes in increasing mode order
  int dims[kMaxModes - 1];         // their sizes
  int nother;                      // N - 1
};

// Row-chunk plan of the update kernels for one mode.
struct UpdatePlan {
  int rows_per_chunk;
  int RC;
  int fused;          // 1: one CTA per block over the reduced Mbar_n (jk_update_fused.cu)
  size_t fused_smem;  // its dynamic shared memory
};

struct ModePlan {
  int splits;          // split-K factor of the MTTKRP
  int64_t kchunk;      // columns of T_(n) per split
  UpdatePlan upd;
};

namespace tc {
// MMAs of one 32-byte K slice of a stage: entry m multiplies A part a[m] by
// n[m] consecutive B parts starting at b[m] (descriptor offsets in 16-byte
// units from the stage bases) into TMEM columns d[m] onward; bit m of first:
// the MMA overwrites those columns on the first K slice of the chain.
struct MmaList {
  int n;
  uint32_t a[10], b[10], d[10], idesc[10];
  uint32_t first;
};

// Tensor-core form of one mode (see jk_tc.cuh).
struct TcPlan {
  int BN;          // N tile (rows of T_(n)), multiple of 16, <= 256
  int tiles_c;     // ceil(C / 128)
  int tiles_n;     // ceil(I_n / BN)
  int splits;      // split-K factor
  int stages;      // pipeline depth (stages of A and B tiles)
  int tmem_cols;   // power of two >= nlev * lstride
  int nlev;        // accumulators (product levels) in TMEM
  int lstride;     // TMEM columns between accumulators (multiple of 32)
  int merged;      // exact form with BN > 128: levels 2 and 3 share an accumulator
  int stack;       // B parts stacked per MMA along N (1, 2 or 4; 1 when merged)
  int nsplit;      // operand parts of the form
  int row_bytes;   // bytes of K per operand row and stage (128 or 64)
  int a_mode;      // fastest other mode
  int Ia_pad;      // its padded size
  int64_t Jp;      // padded columns of the unfolding
  int64_t kchunk;  // padded columns per split (multiple of the k-step)
  int64_t nkt;     // k-steps per N tile: ceil(Jp / BK)
  int ua_smem;     // 1: the CTA keeps its 128 factor rows of mode a (hi, lo) in shared memory
  int ua_stride;   // floats per staged FP32 row (Ia_pad plus a bank skew)
  int ua_parts;    // staged copies: 1 (FP32 hi) or 2 (plus BF16 lo)
  // two-step exact form (narrow modes): Y_o = U_a^T T_(n)(:, o)^T per index o of
  // the remaining modes on the tensor cores, scaled by Q(c, o) and summed in the drain
  int tts;         // 1: this mode runs the two-step form
  int nkt_a;       // k-steps per o (Ia_pad / BK)
  int n_o;         // values of o
  int o_per_cta;   // o values per CTA (one split)
  int nbuf;        // TMEM accumulator sets (2: the next o accumulates while one drains)
  int nis;         // MMA-issuing threads (1 or 2; each owns stages / nis ring stages)
  MmaList mma;     // MMAs per K slice
};
}  // namespace tc

}  // namespace jk

struct jkcals_ctx {
  int N = 0;
  int64_t dims[jk::kMaxModes] = {0};
  int64_t J[jk::kMaxModes] = {0};
  int n_hat = 0;
  int K = 0;
  int C = 0;
  int Rmax = 0;
  bool uniform_rank = true;  // every block has R_g == Rmax
  jkcals_options opt{};
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  int device = 0;
  int num_sms = 0;
  bool broken = false;
  int64_t bytes_allocated = 0;
  std::vector<void*> allocations;
  cudaMemPool_t pool = nullptr;   // the library's stream-ordered pool of this device (null: cudaMalloc)

  std::vector<int> R, off, gram_off;
  std::vector<int64_t> lo_ptr, lo_idx;
  int gram_total = 0;  // sum R_g^2

  // device metadata
  int* d_R = nullptr;
  int* d_off = nullptr;
  int* d_gram_off = nullptr;
  int64_t* d_lo_ptr = nullptr;
  int64_t* d_lo_idx = nullptr;
  int32_t* d_status = nullptr;
  double* d_normT2 = nullptr;
  double* d_loss_prev = nullptr;
  double* d_loss_last = nullptr;
  double* d_tol = nullptr;
  int* d_sweep_idx = nullptr;

  // tensor copies and factors
  double* Tn64[jk::kMaxModes] = {nullptr};
  double* U[jk::kMaxModes] = {nullptr};
  double* gram[jk::kMaxModes] = {nullptr};

  // workspace
  void* part = nullptr;
  size_t part_bytes = 0;
  double* gpart = nullptr;
  double* fpart = nullptr;
  size_t upd_chunks = 0;  // capacity K * RC_max
  double* mbuf = nullptr; // I_max x C FP64 scratch for jkcals_mttkrp / grad
  double* loss_hist = nullptr;
  int loss_cap = 0;

  jk::ModePlan plan[jk::kMaxModes];

  // gradient state (allocated on the first jkcals_grad)
  bool grad_ready = false;
  double* gU[jk::kMaxModes] = {nullptr};
  double* ggram[jk::kMaxModes] = {nullptr};
  double* gG[jk::kMaxModes] = {nullptr};
  double* geg = nullptr;  // K per-block losses + their sum

  double tol_host = 0.0;

  // tensor-core forms (precision != JKCALS_FP64)
  bool tc = false;
  void* Tt[jk::kMaxModes] = {nullptr};  // split, padded, pre-tiled unfoldings
  void* At = nullptr;                    // two-step modes: sliced, pre-tiled U_a^T (rewritten per launch)
  float* UT[jk::kMaxModes] = {nullptr};      // C x Ipad FP32 transposed factors
  float* gUT[jk::kMaxModes] = {nullptr};     // same, for the gradient's factor set
  float* UTlo[jk::kMaxModes] = {nullptr};    // exact-chain form: low parts, U = UT + UTlo
  float* gUTlo[jk::kMaxModes] = {nullptr};
  int64_t Ipad[jk::kMaxModes] = {0};
  jk::tc::TcPlan tcplan[jk::kMaxModes];
  float* cmax[jk::kMaxModes] = {nullptr};    // column maxima of UT (exact-chain grid)
  float* gcmax[jk::kMaxModes] = {nullptr};
  int* rowexp[jk::kMaxModes] = {nullptr};    // row exponents of T_(n) (exact-chain grid)
  int* d_err = nullptr;                      // bounded-wait expiry code of the TC kernel
  std::vector<int32_t> run_block_sweeps;     // sweeps each block ran in the latest jkcals_run

  // compaction of converged blocks inside jkcals_run: while compacted, the
  // handle's block arrays hold only the active blocks (block p is the original
  // block cur_to_orig[p]); the full layout is kept here and restored at the end
  struct Compaction {
    bool on = false;
    std::vector<int> cur_to_orig;
    int K = 0, C = 0, Rmax = 0, gram_total = 0;
    bool uniform_rank = true;
    std::vector<int> R, off, gram_off;
    std::vector<int64_t> lo_ptr, lo_idx;
    std::vector<int32_t> status;
    std::vector<double> normT2, loss_prev, loss_last;
    std::vector<double> gram[jk::kMaxModes];   // host copies of the packed Grams
    double* U[jk::kMaxModes] = {nullptr};      // device, full I_n x C layout
    int* d_cols = nullptr;                     // device column map (C ints)
    jk::ModePlan plan[jk::kMaxModes];          // the full layout's plans, restored as they were
    jk::tc::TcPlan tcplan[jk::kMaxModes];
  } cmp;

  cudaGraphExec_t sweep_exec = nullptr;
  bool graph_valid = false;

  // kernel timing (opt.kernel_timing): events around each mode's MTTKRP
  cudaEvent_t ev_start[jk::kMaxModes] = {nullptr};
  cudaEvent_t ev_stop[jk::kMaxModes] = {nullptr};
  int kernels_per_sweep = 0;
};

namespace jk {

// ---- split-K partial sums --------------------------------------------------------
// Double-float accumulation (unevaluated FP32 pair hi + lo, Knuth TwoSum): about
// 2^-44 relative, on the FP32 pipe; one conversion to FP64 per output.  GB300
// issues FP64 (and FP64 conversions) at a small fraction of the FP32 rate, so
// summing S partials in FP64 would make the reduction FP64-bound.  The
// reduction kernels and the fused update (which sums a block's partials itself)
// add the S partials of an element in split order with exactly these steps.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  lo = __fadd_rn(lo, e);
  hi = s;
}

// The double equal to a float (exact), built from its bit pattern with integer
// operations for zeros and normal numbers (a conversion instruction would run
// on the narrow FP64 pipe); subnormals, Inf and NaN take the conversion.
__device__ __forceinline__ double f32_to_f64_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7fffffffu) == 0) return __longlong_as_double((long long)sign);
  if (e == 0 || e == 255) return (double)f;
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

__device__ __forceinline__ double df_to_double(float hi, float lo) {
  const float s = __fadd_rn(hi, lo);
  const float r = __fsub_rn(lo, __fsub_rn(s, hi));
  return f32_to_f64_exact(s) + f32_to_f64_exact(r);
}

// ---- error plumbing (jk_capi.cu) --------------------------------------------
void set_error(const std::string& msg);

// ---- jackknife adjustment and standard errors (jk_se.cu) ---------------------
struct SeArgs {
  int N, n_hat, R, G;              // modes, sampled mode, common rank, submodels
  int64_t dims[kMaxModes];
  int64_t C;                       // columns of the multi-matrices
  const double* U[kMaxModes];      // multi-matrices, I_k x C row-major
  const int64_t* col_off;          // G: first column of submodel g
  const double* ref[kMaxModes];    // reference factors, I_k x R, row stride ref_ld
  int64_t ref_ld;
  double* aligned[kMaxModes];      // G x I_k x R: adjusted submodels
  int32_t* perm;                   // G x R: reference column s <- submodel column perm[s]
  double* S[kMaxModes];            // I_k x R standard errors (k != n_hat)
};
cudaError_t launch_jackknife_se(const SeArgs& a, cudaStream_t s);

// ---- create-time preparation (jk_prep.cu) -----------------------------------
// T_(n) in Kolda column order from a dense C-order FP64 tensor on the device.
cudaError_t launch_unfold_f64(const double* Tc, const int64_t* dims, int N, int n, double* out,
                              cudaStream_t s);
// Convert an FP32 device buffer to FP64.
cudaError_t launch_f32_to_f64(const float* in, double* out, int64_t count, cudaStream_t s);
// slice[i] = sum_j T_(n)(i, j)^2 for the I rows of an unfolding.
cudaError_t launch_row_sumsq(const double* Tn, int64_t I, int64_t J, double* out, cudaStream_t s);
// normT2[g] = sum over i not in D_g of slice[i].
cudaError_t launch_block_norms(const double* slice, int64_t I, int K, BlockMeta bm, double* normT2,
                               cudaStream_t s);
// Zero rows D_g of block g of the sampled mode's multi-matrix.
cudaError_t launch_zero_left_out(double* U, int C, int K, BlockMeta bm, cudaStream_t s);
// column moves between row-major matrices (compaction of converged blocks, jk_capi.cu)
cudaError_t launch_gather_columns(const double* src, int64_t ld_src, double* dst, int64_t ld_dst, const int* src_col,
                                  int ncols, int64_t rows, cudaStream_t s);
cudaError_t launch_scatter_columns(const double* src, int64_t ld_src, double* dst, int64_t ld_dst, const int* dst_col,
                                   int ncols, int64_t rows, cudaStream_t s);
// G^(n)_g for every block of one mode.
cudaError_t launch_grams(const double* U, int64_t I, int C, int K, BlockMeta bm, double* gram,
                         cudaStream_t s);

// ---- concurrent MTTKRP, FP64 CUDA-core form (jk_mttkrp_f64.cu) --------------
cudaError_t launch_mttkrp_f64(const double* Tn, int64_t I, int64_t J, int C, const KrpOperands& kr,
                              int splits, int64_t kchunk, double* part, cudaStream_t s);
// out = sum_{s < S} part[s] (fixed order), count elements.
cudaError_t launch_reduce_partials_f64(const double* part, int S, int64_t count, double* out,
                                       cudaStream_t s);
// same for FP32 partials, summed in FP64
cudaError_t launch_reduce_partials_f32(const float* part, int S, int64_t count, double* out,
                                       cudaStream_t s);

// Storage of split-K partials: FP64, FP32, or an unevaluated FP32 pair (hi, lo).
constexpr int kPartF64 = 0, kPartF32 = 1, kPartF32x2 = 2;
cudaError_t launch_reduce_partials_f32x2(const float2* part, int S, int64_t count, double* out,
                                         cudaStream_t s);

// ---- per-block update (jk_update.cu) ----------------------------------------
struct UpdateArgs {
  int N, n, n_hat, K, C;
  int64_t I;
  BlockMeta bm;
  double* U;                        // Ubar^(n), written
  const double* gram[kMaxModes];    // Grams of every mode (gram[n] written in phase B)
  double* gram_n;
  const void* part;                 // S x I x C partial MTTKRPs
  int part_kind;                    // kPartF64 / kPartF32 / kPartF32x2
  int S;
  int rows_per_chunk, RC;
  double* gpart;
  double* fpart;
  int32_t* status;
  int normalise;
  const double* normT2;
  double* loss_prev;
  double* loss_last;
  const double* tol;                // device scalar
  double* loss_hist;                // NULL or cap x K
  int loss_cap;
  const int* sweep_idx;             // device scalar
  float* UT;                        // NULL or C x I_pad FP32 transposed copy of Ubar^(n), refreshed
  int64_t I_pad;
  float* cmax;                      // NULL or C column maxima of UT, refreshed
  float* UT_lo;                     // NULL or the low parts fl32(U - UT), refreshed
};
cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s);
// fused one-CTA-per-block update (jk_update_fused.cu); part = reduced Mbar_n (FP64)
size_t update_fused_smem(int64_t I, int Rmax);
cudaError_t prepare_update_fused(size_t smem, int Rmax, bool uniform_rank);
cudaError_t launch_update_fused(const UpdateArgs& a, size_t smem, int Rmax, bool uniform_rank, cudaStream_t s);
// The fused updates of several problems of one rank class (Rmax, uniform) in one
// launch: args[b] (device) is problem b's UpdateArgs, first[b] its first block
// (nprob + 1 entries); threads: the largest update_fused_threads of the
// problems (a CTA's surplus threads take no rows); smem: the largest
// update_fused_smem.  Each block's arithmetic is that of launch_update_fused
// for its problem.
int update_fused_threads(int64_t I, int Rmax, bool uniform);
// Whether the wide update of a tensor-core form (the update writes FP32 factor
// copies) runs its row work in double-float: on modes of more than 128 rows,
// where a row thread solves two rows and FP64 throughput bounds the block; with
// one row per thread the chain's latency bounds it and FP64's shorter chain wins.
inline bool wide_update_double_float(bool tc, int64_t I) { return tc && I > 128; }
std::string grouped_update_attrs();   // diagnostics of the last grouped update launch
// df: the classes' wide_update_double_float (one value per grouped launch)
cudaError_t prepare_update_grouped(int threads, int Rmax, bool uniform, bool df, size_t smem);
cudaError_t launch_update_grouped(const UpdateArgs* args, const int* first, int nprob, int total, int threads,
                                  int Rmax, bool uniform, bool df, size_t smem, cudaStream_t s);

cudaError_t launch_advance_sweep(int* sweep_idx, cudaStream_t s);
cudaError_t launch_advance_sweeps(int* const* sweep_idx, int n, cudaStream_t s);   // n device counters

// ---- gradient epilogue (jk_update.cu) ----------------------------------------
// G_n(i, c) = 2 (U_n H_n - M_n)(i, c) per block, rows D_g of the sampled mode set to 0.
cudaError_t launch_grad_epilogue(int N, int n, int n_hat, int64_t I, int C, int K, BlockMeta bm,
                                 const double* U, const double* const* gram, const double* M,
                                 double* G, cudaStream_t s);
// eg[g] = ||T_{-g}||^2 + sum(*_k G^(k)_g) - 2 sum(U_{N-1|g} * M_{N-1|g}) for every block,
// eg[K] = sum_g eg[g] (fixed order).  M is the last mode's concurrent MTTKRP.
cudaError_t launch_grad_loss(int N, int64_t I, int C, int K, BlockMeta bm, const double* U,
                             const double* const* gram, const double* M, const double* normT2,
                             double* eg, cudaStream_t s);

}  // namespace jk
