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

// Byte offset of element (r, col) of one part tile (BN rows x ROW bytes,
// K-major) in the ROW-byte swizzle of the MMA's shared-memory operands: rows
// in groups of 8 (8 * ROW bytes apart), the 16-byte chunk index XORed with
// the row (ROW = 128) or with row / 2 (ROW = 64).
__device__ __forceinline__ int64_t swizzled_offset(int r, int cb, int row_bytes) {
  const int sw = row_bytes == 128 ? (r & 7) : ((r >> 1) & 3);
  return (int64_t)(r >> 3) * (8 * row_bytes) + (int64_t)(r & 7) * row_bytes + (((cb >> 4) ^ sw) << 4) + (cb & 15);
}

// Tt holds, for N tile t and k-step s, the parts of rows t*BN .. t*BN+BN-1 and
// padded columns s*BK .. s*BK+BK-1 (see jk_tc.cuh).  Logical element (i, jp):
// jp = ia + Ia_pad * o with ia the index of the fastest mode a and o running
// mixed-radix over the remaining modes in increasing order; j is the Eq.
// kolda_mapping column of those indices; zero where i >= I, jp >= Jp or
// ia >= Ia.  Splits are taken from the FP64 value.
template <int PREC>
__global__ void tile_unfold_kernel(const double* __restrict__ Tn, int64_t I, int64_t J, int64_t Ia, int64_t Ia_pad,
                                   int64_t Jp, UnfoldMap mp, const int* __restrict__ rowexp, int BN, int tiles_n,
                                   int64_t nkt, unsigned char* __restrict__ Tt) {
  constexpr int EB = (PREC == JKCALS_TF32 || PREC == JKCALS_3XTF32) ? 4 : 2;
  constexpr int ROW = PREC == JKCALS_EXACT_BF16 ? 64 : 128;
  constexpr int BK = ROW / EB;
  constexpr int NS = PREC == JKCALS_EXACT_BF16 ? 4 : (PREC == JKCALS_SPLIT_BF16 ? 3 : (PREC == JKCALS_3XTF32 ? 2 : 1));
  const int64_t cols = nkt * BK;
  const int64_t total = (int64_t)tiles_n * BN * cols;
  const int64_t part_bytes = (int64_t)BN * ROW;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols;
    const int64_t jp = e - i * cols;
    double x = 0.0;
    if (i < I && jp < Jp) {
      const int64_t o = jp / Ia_pad;
      const int64_t ia = jp - o * Ia_pad;
      if (ia < Ia) {
        int64_t j = ia * mp.sa, rem = o;
        for (int t = 0; t < mp.nq; ++t) {
          const int64_t qq = rem / mp.qd[t];
          j += (rem - qq * mp.qd[t]) * mp.qs[t];
          rem = qq;
        }
        x = Tn[i * J + j];
      }
    }
    float v[NS];
    if constexpr (PREC == JKCALS_TF32 || PREC == JKCALS_3XTF32) {
      const float h = tf32_rna((float)x);
      v[0] = h;
      if constexpr (NS > 1) v[1] = tf32_rna((float)(x - (double)h));
    } else if constexpr (PREC == JKCALS_EXACT_BF16) {
      // x = 2^(F-7) (s0 + s1 2^-7 + s2 2^-14 + s3 2^-21), |s_k| <= 128, stored as s_k 2^(-7k)
      double y = i < I ? ldexp(x, kSliceBits - rowexp[i]) : 0.0;
      const double s0 = rint(y);
      y = (y - s0) * 128.0;
      const double s1 = rint(y);
      y = (y - s1) * 128.0;
      const double s2 = rint(y);
      y = (y - s2) * 128.0;
      const double s3 = rint(y);
      v[0] = (float)s0;
      v[1] = (float)(s1 / 128.0);
      v[2] = (float)(s2 / 16384.0);
      v[3] = (float)(s3 / 2097152.0);
    } else {
      const float h = __bfloat162float(__double2bfloat16(x));
      v[0] = h;
      if constexpr (NS > 1) {
        const double r1 = x - (double)h;
        const float m = __bfloat162float(__double2bfloat16(r1));
        v[1] = m;
        v[2] = __bfloat162float(__double2bfloat16(r1 - (double)m));
      }
    }
    const int64_t tn = i / BN, ks = jp / BK;
    const int r = (int)(i - tn * BN), col = (int)(jp - ks * BK);
    const int64_t tile = (tn * nkt + ks) * NS * part_bytes;
    const int64_t off = swizzled_offset(r, col * EB, ROW);
#pragma unroll
    for (int p = 0; p < NS; ++p) {
      unsigned char* dst = Tt + tile + p * part_bytes + off;
      if constexpr (EB == 4)
        *reinterpret_cast<float*>(dst) = v[p];
      else
        *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v[p]);   // exact: v[p] is a BF16 value
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

cudaError_t launch_tile_unfold(int precision, const double* Tn64, int64_t I, int64_t J, int64_t Ia, int64_t Ia_pad,
                               int64_t Jp, const UnfoldMap& mp, const int* rowexp, int BN, int tiles_n, int64_t nkt,
                               void* Tt, cudaStream_t s) {
  const unsigned g = grid_for((int64_t)tiles_n * BN * nkt * form_bk(precision));
  unsigned char* out = static_cast<unsigned char*>(Tt);
  switch (precision) {
    case JKCALS_TF32:
      tile_unfold_kernel<JKCALS_TF32><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, BN, tiles_n, nkt, out);
      break;
    case JKCALS_3XTF32:
      tile_unfold_kernel<JKCALS_3XTF32><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, BN, tiles_n, nkt, out);
      break;
    case JKCALS_BF16:
      tile_unfold_kernel<JKCALS_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, BN, tiles_n, nkt, out);
      break;
    case JKCALS_SPLIT_BF16:
      tile_unfold_kernel<JKCALS_SPLIT_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, BN, tiles_n, nkt,
                                                              out);
      break;
    case JKCALS_EXACT_BF16:
      tile_unfold_kernel<JKCALS_EXACT_BF16><<<g, 256, 0, s>>>(Tn64, I, J, Ia, Ia_pad, Jp, mp, rowexp, BN, tiles_n, nkt,
                                                              out);
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
