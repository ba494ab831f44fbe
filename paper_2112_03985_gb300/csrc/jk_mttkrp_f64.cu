// Concurrent MTTKRP, FP64 form (CUDA cores, DFMA).
//
//   Mbar_n = T_(n) * KRP_n,  KRP_n(j, c) = prod_{k != n} Ubar^(k)(i_k(j), c)
//
// (Alg. 3 MTTKRP line; the Khatri-Rao order of Eq. MTTKRP with the column
// index j of Eq. kolda_mapping.)  The Khatri-Rao product is never stored: each
// CTA builds its BK x BN tile of it in shared memory from factor rows (which
// stay in L1/L2: the multi-matrices are small), multiplies it with a BM x BK
// tile of T_(n), and accumulates a BM x BN tile of Mbar_n in registers.
//
// The contraction over j is split across gridDim.z CTAs (split-K): each split
// writes its partial tile to part[split]; the consumer (the update kernel or
// the reduce kernel) sums the splits in a fixed order, so results are
// bit-reproducible run to run.
//
// Bound: FP64 FMA throughput (GB300 issues FP64 at a small fraction of its
// FP32 rate), so a plain register-tiled SIMT GEMM with 16 FMAs per operand
// pair is enough; the tile loads and the Khatri-Rao generation are a few
// percent of the issue slots.
#include "jk_common.cuh"

namespace jk {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__global__ void __launch_bounds__(NT) mttkrp_f64_kernel(const double* __restrict__ Tn, int64_t I,
                                                        int64_t J, int C, KrpOperands kr,
                                                        int64_t kchunk, double* __restrict__ part) {
  __shared__ double As[BK][BM];                 // As[k][m] = T_(n)(m0 + m, j0 + k)
  __shared__ __align__(16) double Bs[BK][BN];   // Bs[k][c] = KRP(j0 + k, c0 + c)
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;   // grid.x: row tiles (< 2^31)
  const int c0 = blockIdx.y * BN;                 // grid.y: column tiles (< 65536)
  const int64_t jb = (int64_t)blockIdx.z * kchunk;
  const int64_t je = (jb + kchunk < J) ? jb + kchunk : J;

  const int a_row = tid >> 2, a_k = (tid & 3) * 4;   // T tile: 4 consecutive j of one row
  const int b_k = tid >> 4, b_c = (tid & 15) * 4;    // KRP tile: 4 consecutive c of one j

  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.0;

  for (int64_t j0 = jb; j0 < je; j0 += BK) {
    {
      const int64_t row = m0 + a_row;
      const double* src = Tn + row * J;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t j = j0 + a_k + e;
        As[a_k + e][a_row] = (row < I && j < je) ? __ldg(src + j) : 0.0;
      }
    }
    {
      const int64_t j = j0 + b_k;
      double v[4] = {0.0, 0.0, 0.0, 0.0};
      if (j < je) {
        v[0] = v[1] = v[2] = v[3] = 1.0;
        int64_t rem = j;
        for (int o = 0; o < kr.nother; ++o) {
          const int64_t d = kr.dims[o];
          const int64_t q = rem / d;
          const int64_t io = rem - q * d;
          rem = q;
          const double* urow = kr.U[o] + io * C;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int c = c0 + b_c + e;
            v[e] = (c < C) ? v[e] * __ldg(urow + c) : 0.0;
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) Bs[b_k][b_c + e] = v[e];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
      const double2 b01 = *reinterpret_cast<const double2*>(&Bs[k][tx * 4]);
      const double2 b23 = *reinterpret_cast<const double2*>(&Bs[k][tx * 4 + 2]);
      b[0] = b01.x; b[1] = b01.y; b[2] = b23.x; b[3] = b23.y;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fma(a[i], b[c], acc[i][c]);
    }
    __syncthreads();
  }

  double* out = part + (int64_t)blockIdx.z * I * C;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = m0 + ty * 4 + i;
    if (row >= I) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = c0 + tx * 4 + c;
      if (col < C) out[row * C + col] = acc[i][c];
    }
  }
}

// The split-K reductions below add the S partials of an element in split order.
// A thread first loads a batch of kRedBatch partials (independent loads, all in
// flight together), then adds them in order: one L2 round trip per batch
// instead of one per split.
constexpr int kRedBatch = 8;

__global__ void reduce_partials_f64_kernel(const double* __restrict__ part, int S, int64_t count,
                                           double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s0 = 0; s0 < S; s0 += kRedBatch) {
      double v[kRedBatch];
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u) v[u] = s0 + u < S ? __ldg(part + (int64_t)(s0 + u) * count + e) : 0.0;
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u) {
        if (s0 + u < S) acc = (s0 + u == 0) ? v[u] : acc + v[u];
      }
    }
    out[e] = acc;
  }
}

__global__ void reduce_partials_f32_kernel(const float* __restrict__ part, int S, int64_t count,
                                           double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    float hi = 0.f, lo = 0.f;
    for (int s0 = 0; s0 < S; s0 += kRedBatch) {
      float v[kRedBatch];
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u) v[u] = s0 + u < S ? __ldg(part + (int64_t)(s0 + u) * count + e) : 0.f;
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u)
        if (s0 + u < S) df_add(hi, lo, v[u]);
    }
    out[e] = df_to_double(hi, lo);
  }
}

__global__ void reduce_partials_f32x2_kernel(const float2* __restrict__ part, int S, int64_t count,
                                             double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    float hi = 0.f, lo = 0.f;
    for (int s0 = 0; s0 < S; s0 += kRedBatch) {
      float2 v[kRedBatch];
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u)
        v[u] = s0 + u < S ? __ldg(part + (int64_t)(s0 + u) * count + e) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kRedBatch; ++u) {
        if (s0 + u < S) {
          df_add(hi, lo, v[u].x);
          lo = __fadd_rn(lo, v[u].y);
        }
      }
    }
    out[e] = df_to_double(hi, lo);
  }
}

}  // namespace

cudaError_t launch_reduce_partials_f32x2(const float2* part, int S, int64_t count, double* out,
                                         cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  reduce_partials_f32x2_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, S, count, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials_f32(const float* part, int S, int64_t count, double* out,
                                       cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  reduce_partials_f32_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, S, count, out);
  return cudaGetLastError();
}

cudaError_t launch_mttkrp_f64(const double* Tn, int64_t I, int64_t J, int C, const KrpOperands& kr,
                              int splits, int64_t kchunk, double* part, cudaStream_t s) {
  dim3 grid((unsigned)((I + BM - 1) / BM), (unsigned)((C + BN - 1) / BN), (unsigned)splits);
  mttkrp_f64_kernel<<<grid, NT, 0, s>>>(Tn, I, J, C, kr, kchunk, part);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials_f64(const double* part, int S, int64_t count, double* out,
                                       cudaStream_t s) {
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  reduce_partials_f64_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, S, count, out);
  return cudaGetLastError();
}

}  // namespace jk
