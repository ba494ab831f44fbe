// Create-time operand preparation for the tensor-core MTTKRP: the padded,
// precision-split unfoldings and the transposed FP32 factor copies.
#include <cuda_bf16.h>

#include "jk_tc.cuh"

namespace jk {
namespace tc {
namespace {

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// parts[p][i * Jp + jp] = part p of T_(n)(i, ia + Ia * o), jp = ia + Ia_pad * o,
// zero where ia >= Ia.  Splits are taken from the FP64 value.
template <int PREC>
__global__ void split_unfold_kernel(const double* __restrict__ Tn, int64_t I, int64_t J, int64_t Ia,
                                    int64_t Ia_pad, int64_t Jp, void* p0, void* p1, void* p2) {
  const int64_t total = I * Jp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Jp;
    const int64_t jp = e - i * Jp;
    const int64_t o = jp / Ia_pad;
    const int64_t ia = jp - o * Ia_pad;
    const double x = (ia < Ia) ? Tn[i * J + ia + Ia * o] : 0.0;
    if constexpr (PREC == JKCALS_TF32 || PREC == JKCALS_3XTF32) {
      const float h = tf32_rna((float)x);
      static_cast<float*>(p0)[e] = h;
      if constexpr (PREC == JKCALS_3XTF32) static_cast<float*>(p1)[e] = tf32_rna((float)(x - (double)h));
    } else {
      const __nv_bfloat16 h = __double2bfloat16(x);
      static_cast<__nv_bfloat16*>(p0)[e] = h;
      if constexpr (PREC == JKCALS_SPLIT_BF16) {
        const double r1 = x - (double)__bfloat162float(h);
        const __nv_bfloat16 m = __double2bfloat16(r1);
        static_cast<__nv_bfloat16*>(p1)[e] = m;
        static_cast<__nv_bfloat16*>(p2)[e] = __double2bfloat16(r1 - (double)__bfloat162float(m));
      }
    }
  }
}

__global__ void factor_to_ut_kernel(const double* __restrict__ U, int64_t I, int C, float* __restrict__ UT,
                                    int64_t I_pad) {
  const int64_t total = I * (int64_t)C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / I;
    const int64_t i = e - c * I;
    UT[c * I_pad + i] = (float)U[i * C + c];
  }
}

inline unsigned grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 65535 * 8) b = 65535 * 8;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_split_unfold(int precision, const double* Tn64, int64_t I, int64_t J, int64_t Ia,
                                int64_t Ia_pad, int64_t Jp, void* const* parts, cudaStream_t s) {
  const unsigned g = grid_for(I * Jp);
  switch (precision) {
    case JKCALS_TF32:
      split_unfold_kernel<JKCALS_TF32><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, parts[0], nullptr, nullptr);
      break;
    case JKCALS_3XTF32:
      split_unfold_kernel<JKCALS_3XTF32><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, parts[0], parts[1], nullptr);
      break;
    case JKCALS_BF16:
      split_unfold_kernel<JKCALS_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, parts[0], nullptr, nullptr);
      break;
    case JKCALS_SPLIT_BF16:
      split_unfold_kernel<JKCALS_SPLIT_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, parts[0], parts[1],
                                                              parts[2]);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_factor_to_ut(const double* U, int64_t I, int C, float* UT, int64_t I_pad, cudaStream_t s) {
  factor_to_ut_kernel<<<grid_for(I * (int64_t)C), 256, 0, s>>>(U, I, C, UT, I_pad);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace jk
