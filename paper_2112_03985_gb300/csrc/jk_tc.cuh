// Declarations of the tensor-core (tcgen05) form of the concurrent MTTKRP.
//
// Operand layouts in HBM (one handle, precision forms TF32 / 3xTF32 / BF16 / BF16x3):
//   Tp[n][p]  part p of the split mode-n unfolding, I_n x Jp_n row-major (FP32
//             holding TF32 values, or BF16), Jp_n = Ia_pad * prod(remaining dims):
//             the fastest other mode a is padded with zeros to Ia_pad (a multiple
//             of the 16-byte chunk) so that a chunk never straddles two rows of
//             the remaining modes.
//   UT[n]     FP32 transposed copy of Ubar^(n): C x I_pad_n (zero padded), written
//             by the update kernel after every mode update.
#pragma once

#include <cuda.h>

#include "jk_common.cuh"

namespace jk {
namespace tc {

constexpr int kKindTF32 = 0;
constexpr int kKindBF16 = 1;

struct TcPlan {
  int BN;          // N tile (rows of T_(n)), multiple of 16, <= 256
  int tiles_c;     // ceil(C / 128)
  int tiles_n;     // ceil(I_n / BN)
  int splits;      // split-K factor
  int stages;      // pipeline depth
  int tmem_cols;   // power of two >= BN
  int nsplit;      // operand parts of the form
  int a_mode;      // fastest other mode
  int Ia_pad;      // its padded size
  int64_t Jp;      // padded columns of the unfolding
  int64_t kchunk;  // padded columns per split (multiple of the k-step)
};

struct TcArgs {
  int64_t I, Jp, kchunk;
  int C, BN, tmem_cols, stages;
  int Ia_pad;
  int nq;                          // remaining other modes (N - 2)
  int qdims[kMaxModes - 2];
  int qpad[kMaxModes - 2];
  const float* UTa;                // C x Ia_pad
  const float* UTq[kMaxModes - 2];  // C x qpad[t]
  float* part;                     // splits x I x C
  int* err;                        // device error word (bounded-wait expiry)
};

int form_nsplit(int precision);
int form_bk(int precision);
int form_elem_bytes(int precision);
int form_chunk(int precision);
int form_passes(int precision);
size_t tc_smem_bytes(const TcPlan& p);
// Raise the kernel's dynamic shared-memory limit (call once, outside stream capture).
cudaError_t prepare_mttkrp_tc(int precision, size_t max_smem);
cudaError_t launch_mttkrp_tc(int precision, const TcPlan& p, const CUtensorMap* maps, const TcArgs& a,
                             cudaStream_t s);

// create-time conversions (jk_tc_prep.cu)
cudaError_t launch_split_unfold(int precision, const double* Tn64, int64_t I, int64_t J, int64_t Ia,
                                int64_t Ia_pad, int64_t Jp, void* const* parts, cudaStream_t s);
cudaError_t launch_factor_to_ut(const double* U, int64_t I, int C, float* UT, int64_t I_pad, cudaStream_t s);

}  // namespace tc
}  // namespace jk
