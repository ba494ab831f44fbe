// Create-time operand preparation for the tensor-core MTTKRP: the padded,
// precision-split unfoldings, the transposed FP32 factor copies, and the
// per-row grids (row exponents, column maxima) of the exact-chain form.
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

// One CTA per row: max |T| -> smallest F with max < 2^F.
__global__ void row_exponent_kernel(const double* __restrict__ Tn, int64_t J, int* __restrict__ rowexp) {
  __shared__ double red[256];
  const int64_t i = blockIdx.x;
  double m = 0.0;
  for (int64_t j = threadIdx.x; j < J; j += blockDim.x) m = fmax(m, fabs(Tn[i * J + j]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int e = 0;
    if (red[0] > 0.0) frexp(red[0], &e);   // max = f 2^e, f in [0.5, 1) -> max < 2^e
    rowexp[i] = e;
  }
}

// parts[p][i * Jp + jp] = part p of T_(n)(i, j) with jp = ia + Ia_pad * o: ia is
// the index of the fastest mode a, o runs mixed-radix over the remaining modes
// in increasing order, and j is the Eq. kolda_mapping column of those indices;
// zero where ia >= Ia.  Splits are taken from the FP64 value.
template <int PREC>
__global__ void split_unfold_kernel(const double* __restrict__ Tn, int64_t I, int64_t J, int64_t Ia,
                                    int64_t Ia_pad, int64_t Jp, UnfoldMap mp, const int* __restrict__ rowexp,
                                    void* p0, void* p1, void* p2, void* p3) {
  const int64_t total = I * Jp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Jp;
    const int64_t jp = e - i * Jp;
    const int64_t o = jp / Ia_pad;
    const int64_t ia = jp - o * Ia_pad;
    double x = 0.0;
    if (ia < Ia) {
      int64_t j = ia * mp.sa, rem = o;
      for (int t = 0; t < mp.nq; ++t) {
        const int64_t qq = rem / mp.qd[t];
        j += (rem - qq * mp.qd[t]) * mp.qs[t];
        rem = qq;
      }
      x = Tn[i * J + j];
    }
    if constexpr (PREC == JKCALS_TF32 || PREC == JKCALS_3XTF32) {
      const float h = tf32_rna((float)x);
      static_cast<float*>(p0)[e] = h;
      if constexpr (PREC == JKCALS_3XTF32) static_cast<float*>(p1)[e] = tf32_rna((float)(x - (double)h));
    } else if constexpr (PREC == JKCALS_EXACT_BF16) {
      // x = 2^(F-7) (s0 + s1 2^-7 + s2 2^-14 + s3 2^-21), |s_k| <= 128, stored as s_k 2^(-7k)
      double y = ldexp(x, kSliceBits - rowexp[i]);
      const double s0 = rint(y);
      y = (y - s0) * 128.0;
      const double s1 = rint(y);
      y = (y - s1) * 128.0;
      const double s2 = rint(y);
      y = (y - s2) * 128.0;
      const double s3 = rint(y);
      static_cast<__nv_bfloat16*>(p0)[e] = __double2bfloat16(s0);
      static_cast<__nv_bfloat16*>(p1)[e] = __double2bfloat16(s1 / 128.0);
      static_cast<__nv_bfloat16*>(p2)[e] = __double2bfloat16(s2 / 16384.0);
      static_cast<__nv_bfloat16*>(p3)[e] = __double2bfloat16(s3 / 2097152.0);
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
                                    float* __restrict__ UT_lo, int64_t I_pad) {
  const int64_t total = I * (int64_t)C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / I;
    const int64_t i = e - c * I;
    const double u = U[i * C + c];
    const float hi = (float)u;
    UT[c * I_pad + i] = hi;
    if (UT_lo != nullptr) UT_lo[c * I_pad + i] = (float)(u - (double)hi);
  }
}

// One warp per column.
__global__ void colmax_kernel(const float* __restrict__ UT, int64_t I, int64_t I_pad, int C,
                              float* __restrict__ cmax) {
  const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= C) return;
  float m = 0.f;
  for (int64_t i = lane; i < I; i += 32) m = fmaxf(m, fabsf(UT[(int64_t)c * I_pad + i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) cmax[c] = m;
}

inline unsigned grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  if (b > 65535 * 8) b = 65535 * 8;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_row_exponent(const double* Tn64, int64_t I, int64_t J, int* rowexp, cudaStream_t s) {
  row_exponent_kernel<<<(unsigned)I, 256, 0, s>>>(Tn64, J, rowexp);
  return cudaGetLastError();
}

cudaError_t launch_split_unfold(int precision, const double* Tn64, int64_t I, int64_t J, int64_t Ia,
                                int64_t Ia_pad, int64_t Jp, const UnfoldMap& mp, const int* rowexp,
                                void* const* parts, cudaStream_t s) {
  const unsigned g = grid_for(I * Jp);
  switch (precision) {
    case JKCALS_TF32:
      split_unfold_kernel<JKCALS_TF32><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, parts[0], nullptr,
                                                         nullptr, nullptr);
      break;
    case JKCALS_3XTF32:
      split_unfold_kernel<JKCALS_3XTF32><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, parts[0],
                                                           parts[1], nullptr, nullptr);
      break;
    case JKCALS_BF16:
      split_unfold_kernel<JKCALS_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, parts[0], nullptr,
                                                         nullptr, nullptr);
      break;
    case JKCALS_SPLIT_BF16:
      split_unfold_kernel<JKCALS_SPLIT_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, parts[0],
                                                               parts[1], parts[2], nullptr);
      break;
    case JKCALS_EXACT_BF16:
      split_unfold_kernel<JKCALS_EXACT_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, parts[0],
                                                               parts[1], parts[2], parts[3]);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_factor_to_ut(const double* U, int64_t I, int C, float* UT, float* UT_lo, int64_t I_pad,
                                cudaStream_t s) {
  factor_to_ut_kernel<<<grid_for(I * (int64_t)C), 256, 0, s>>>(U, I, C, UT, UT_lo, I_pad);
  return cudaGetLastError();
}

cudaError_t launch_colmax(const float* UT, int64_t I, int64_t I_pad, int C, float* cmax, cudaStream_t s) {
  colmax_kernel<<<(unsigned)((C + 7) / 8), 256, 0, s>>>(UT, I, I_pad, C, cmax);
  return cudaGetLastError();
}

}  // namespace tc
}  // namespace jk
