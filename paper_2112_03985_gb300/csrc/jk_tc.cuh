// Declarations of the tensor-core (tcgen05) forms of the concurrent MTTKRP.
//
// Operand layouts in HBM (one handle, forms TF32 / 3xTF32 / BF16 / BF16x3 / exact BF16):
//   Tt[n]     the split mode-n unfolding, pre-tiled into the exact shared-memory
//             image of the MMA's B operand: for N tile t (BN rows of I_n, zero
//             padded) and k-step s (BK columns of the padded unfolding), the
//             nsplit parts follow each other, each BN rows x ROW bytes, K-major,
//             in the ROW-byte swizzle (128 or 64).  One stage of the pipeline is
//             then one contiguous bulk copy.  Columns jp = ia + Ia_pad * o: ia
//             indexes the fastest other mode a, padded with zeros to Ia_pad (a
//             multiple of the 16-byte chunk) so that a chunk never straddles two
//             rows of the remaining modes; o runs mixed-radix over the others.
//   UT[n]     FP32 transposed copy of Ubar^(n): C x I_pad_n (zero padded), written
//             by the update kernel after every mode update.
//   cmax[n]   C floats, max_i |UT[n][c][i]| (exact-chain form: per-row grid of KRP^T).
//   rowexp[n] I_n ints, F_i with max_j |T_(n)(i, j)| < 2^F_i (exact-chain form).
#pragma once

#include "jk_common.cuh"

namespace jk {
namespace tc {

// Exact-chain sliced-BF16 form: 4 slices of 7-bit integers per operand on a
// per-row power-of-two grid; the TMEM accumulators are drained after at most
// this many columns of T_(n) (one segment of a CTA's chain), so that the two
// leading product levels sum exactly in FP32.
constexpr int kExactChainMax = 1024;
constexpr int kSliceBits = 7;


struct TcArgs {
  int64_t I, Jp, kchunk;
  int C, BN, tmem_cols;
  int stages;                      // pipeline depth
  int nlev, lstride, merged;       // accumulators in TMEM (see TcPlan)
  int stack;                       // B parts stacked per MMA along N
  int Ia_pad;
  int64_t nkt;                     // k-steps per N tile in Tt
  const unsigned char* Tt;         // pre-tiled unfolding (layout above)
  int nq;                          // remaining other modes (N - 2)
  int qdims[kMaxModes - 2];
  int qpad[kMaxModes - 2];
  const float* UTa;                // C x Ia_pad
  const float* UTq[kMaxModes - 2];  // C x qpad[t]
  float* part;                     // splits x I x C
  int* err;                        // device error word (bounded-wait expiry)
  // exact-chain form only:
  const float* UTa_lo;             // low parts: U = UT + UT_lo to ~2^-48
  const float* UTq_lo[kMaxModes - 2];
  const float* cmax_a;             // C: max_i |UT_a[c][i]|
  const float* cmax_q[kMaxModes - 2];
  const int* rowexp;               // I_n: F_i of this mode's unfolding
  int ua_smem;                     // stage the 128 rows of UTa (and UTa_lo) in shared memory
  int ua_stride;                   // floats per staged FP32 row (BF16 low rows: Ia_pad elements)
  // two-step exact form only (TcPlan::tts):
  const unsigned char* At;         // sliced, pre-tiled U_a^T: per 128-row tile and k-step one A stage image
  int nkt_a, n_o, o_per_cta, nbuf;
  int nis;                         // MMA-issuing threads (1 or 2), each with S / nis ring stages
  int tiles_c, tiles_n;            // grid of this problem (C tiles x N tiles x splits): grouped launches
  int Ia;                          // size of mode a
  int64_t ut_stride_a;             // row stride of UTa / UTa_lo (floats)
  int skip_slice;                  // At already holds the current slices of U_a
};

int form_nsplit(int precision);
int form_row_bytes(int precision);
int form_bk(int precision);
int form_elem_bytes(int precision);
int form_chunk(int precision);
int form_passes(int precision);
size_t tc_smem_bytes(const TcPlan& p);
// Accumulator layout and MMA list of a plan whose BN, nsplit and row_bytes are
// set: levels s + t of the part products, B parts stacked along N where the
// TMEM columns allow; JKCALS_ERR_UNSUPPORTED if the accumulators exceed TMEM.
int build_mma_list(int precision, TcPlan& p);
// Raise the kernel's dynamic shared-memory limit (call once, outside stream capture).
cudaError_t prepare_mttkrp_tc(int precision, size_t max_smem);
cudaError_t launch_mttkrp_tc(int precision, const TcPlan& p, const TcArgs& a, cudaStream_t s);
// The one-step MTTKRPs of several problems in one launch (the two-step form is
// not grouped): args[b] (device) is problem b's TcArgs, first[b] its first CTA
// (nprob + 1 entries, first[nprob] = total); qm_small: every problem has at most
// two remaining modes (nq <= 2); smem: the largest problem's tc_smem_bytes.
cudaError_t prepare_mttkrp_tc_grouped(int precision, bool qm_small, size_t smem);
cudaError_t launch_mttkrp_tc_grouped(int precision, const TcArgs* args, const int* first, int nprob, int total,
                                     bool qm_small, size_t smem, cudaStream_t s);
// Bytes of the A images of a two-step plan (tiles_c x nkt_a stage images).
size_t tts_a_bytes(const TcPlan& p);

// create-time conversions (jk_tc_prep.cu)
// rowexp[i] = smallest F with max_j |Tn64(i, j)| < 2^F (0 for an all-zero row)
cudaError_t launch_row_exponent(const double* Tn64, int64_t I, int64_t J, int* rowexp, cudaStream_t s);
// Column map of a padded unfolding: Kolda stride sa of the fastest mode a, and
// sizes qd / Kolda strides qs of the remaining modes in increasing order.
struct UnfoldMap {
  int64_t sa;
  int nq;
  int64_t qd[kMaxModes - 2];
  int64_t qs[kMaxModes - 2];
};
// Split (and for the exact form slice, using rowexp) the padded unfolding into
// its parts and write them pre-tiled (layout above) into Tt, whose size is
// tiles_n * nkt * nsplit * BN * row_bytes bytes.
cudaError_t launch_tile_unfold(int precision, const double* Tn64, int64_t I, int64_t J, int64_t Ia, int64_t Ia_pad,
                               int64_t Jp, const UnfoldMap& mp, const int* rowexp, int BN, int tiles_n, int64_t nkt,
                               void* Tt, cudaStream_t s);
// UT[c][i] = fl32(U[i][c]); if UT_lo != NULL also UT_lo[c][i] = fl32(U[i][c] - UT[c][i])
cudaError_t launch_factor_to_ut(const double* U, int64_t I, int C, float* UT, float* UT_lo, int64_t I_pad,
                                cudaStream_t s);
// cmax[c] = max_{i < I} |UT[c][i]| for all C columns
cudaError_t launch_colmax(const float* UT, int64_t I, int64_t I_pad, int C, float* cmax, cudaStream_t s);

}  // namespace tc
}  // namespace jk
