// Create-time preparation: per-mode unfoldings, slice norms, zero rows, Grams.
//
// These run once per jkcals_create / jkcals_set_factors and are not on the
// per-sweep path; they are written for clarity and full coalescing of the
// large output (the unfoldings), not for peak bandwidth of the gathers.
#include "jk_common.cuh"

namespace jk {
namespace {

struct Dims8 {
  int64_t d[kMaxModes];
};

// out[i_n * J + j] = T(i_0, ..., i_{N-1}) with j from Eq. kolda_mapping
// (0-based: j = sum_{k != n} i_k prod_{m < k, m != n} I_m).  T is C-order.
__global__ void unfold_f64_kernel(const double* __restrict__ Tc, Dims8 dims, int N, int n, int64_t J,
                                  int64_t total, double* __restrict__ out) {
  int64_t cstride[kMaxModes];
  int64_t s = 1;
  for (int k = N - 1; k >= 0; --k) {
    cstride[k] = s;
    s *= dims.d[k];
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i_n = e / J;
    int64_t rem = e - i_n * J;
    int64_t src = i_n * cstride[n];
    for (int k = 0; k < N; ++k) {
      if (k == n) continue;
      const int64_t q = rem / dims.d[k];
      src += (rem - q * dims.d[k]) * cstride[k];
      rem = q;
    }
    out[e] = Tc[src];
  }
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (double)in[e];
}

// One CTA per row; fixed-order tree reduction (deterministic).
__global__ void row_sumsq_kernel(const double* __restrict__ Tn, int64_t J, double* __restrict__ out) {
  __shared__ double red[256];
  const int64_t i = blockIdx.x;
  double acc = 0.0;
  for (int64_t j = threadIdx.x; j < J; j += blockDim.x) {
    const double v = Tn[i * J + j];
    acc = fma(v, v, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[i] = red[0];
}

// ||T_{-g}||^2 = sum_{i not in D_g} ||slice i||^2 (error line of Alg. 3).
__global__ void block_norms_kernel(const double* __restrict__ slice, int64_t I, int K, BlockMeta bm,
                                   double* __restrict__ normT2) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= K) return;
  const int64_t b = bm.lo_ptr[g], e = bm.lo_ptr[g + 1];
  int64_t p = b;
  double acc = 0.0;
  for (int64_t i = 0; i < I; ++i) {
    while (p < e && bm.lo_idx[p] < i) ++p;
    if (p < e && bm.lo_idx[p] == i) continue;
    acc += slice[i];
  }
  normT2[g] = acc;
}

__global__ void zero_left_out_kernel(double* __restrict__ U, int C, BlockMeta bm) {
  const int g = blockIdx.x;
  const int R = bm.R[g], off = bm.off[g];
  const int64_t b = bm.lo_ptr[g], e = bm.lo_ptr[g + 1];
  for (int64_t t = threadIdx.x; t < (e - b) * R; t += blockDim.x) {
    const int64_t i = bm.lo_idx[b + t / R];
    U[i * C + off + (int)(t % R)] = 0.0;
  }
}

__global__ void grams_kernel(const double* __restrict__ U, int64_t I, int C, BlockMeta bm,
                             double* __restrict__ gram) {
  const int g = blockIdx.x;
  const int R = bm.R[g], off = bm.off[g];
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) {
    const int r = p / R, c = p % R;
    double acc = 0.0;
    for (int64_t i = 0; i < I; ++i) acc = fma(U[i * C + off + r], U[i * C + off + c], acc);
    gram[bm.gram_off[g] + p] = acc;
  }
}

inline int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 65535 * 8) b = 65535 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_unfold_f64(const double* Tc, const int64_t* dims, int N, int n, double* out,
                              cudaStream_t s) {
  Dims8 d{};
  int64_t total = 1;
  for (int k = 0; k < N; ++k) {
    d.d[k] = dims[k];
    total *= dims[k];
  }
  const int64_t J = total / dims[n];
  unfold_f64_kernel<<<grid_for(total, 256), 256, 0, s>>>(Tc, d, N, n, J, total, out);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* in, double* out, int64_t count, cudaStream_t s) {
  f32_to_f64_kernel<<<grid_for(count, 256), 256, 0, s>>>(in, out, count);
  return cudaGetLastError();
}

cudaError_t launch_row_sumsq(const double* Tn, int64_t I, int64_t J, double* out, cudaStream_t s) {
  row_sumsq_kernel<<<(unsigned)I, 256, 0, s>>>(Tn, J, out);
  return cudaGetLastError();
}

cudaError_t launch_block_norms(const double* slice, int64_t I, int K, BlockMeta bm, double* normT2,
                               cudaStream_t s) {
  block_norms_kernel<<<(K + 127) / 128, 128, 0, s>>>(slice, I, K, bm, normT2);
  return cudaGetLastError();
}

cudaError_t launch_zero_left_out(double* U, int C, int K, BlockMeta bm, cudaStream_t s) {
  zero_left_out_kernel<<<K, 128, 0, s>>>(U, C, bm);
  return cudaGetLastError();
}

cudaError_t launch_grams(const double* U, int64_t I, int C, int K, BlockMeta bm, double* gram,
                         cudaStream_t s) {
  grams_kernel<<<K, 256, 0, s>>>(U, I, C, bm, gram);
  return cudaGetLastError();
}

namespace {
// Column moves between two row-major matrices of `rows` rows: gather takes
// column src_col[j] of src into column j of dst; scatter puts column j of src
// into column dst_col[j] of dst.
__global__ void gather_columns_kernel(const double* __restrict__ src, int64_t ld_src, double* __restrict__ dst,
                                      int64_t ld_dst, const int* __restrict__ src_col, int ncols, int64_t rows) {
  const int64_t total = rows * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols;
    const int j = (int)(e - i * ncols);
    dst[i * ld_dst + j] = src[i * ld_src + src_col[j]];
  }
}

__global__ void scatter_columns_kernel(const double* __restrict__ src, int64_t ld_src, double* __restrict__ dst,
                                       int64_t ld_dst, const int* __restrict__ dst_col, int ncols, int64_t rows) {
  const int64_t total = rows * ncols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ncols;
    const int j = (int)(e - i * ncols);
    dst[i * ld_dst + dst_col[j]] = src[i * ld_src + j];
  }
}

unsigned col_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}
}  // namespace

cudaError_t launch_gather_columns(const double* src, int64_t ld_src, double* dst, int64_t ld_dst, const int* src_col,
                                  int ncols, int64_t rows, cudaStream_t s) {
  if (ncols <= 0 || rows <= 0) return cudaSuccess;
  gather_columns_kernel<<<col_blocks(rows * ncols), 256, 0, s>>>(src, ld_src, dst, ld_dst, src_col, ncols, rows);
  return cudaGetLastError();
}

cudaError_t launch_scatter_columns(const double* src, int64_t ld_src, double* dst, int64_t ld_dst, const int* dst_col,
                                   int ncols, int64_t rows, cudaStream_t s) {
  if (ncols <= 0 || rows <= 0) return cudaSuccess;
  scatter_columns_kernel<<<col_blocks(rows * ncols), 256, 0, s>>>(src, ld_src, dst, ld_dst, dst_col, ncols, rows);
  return cudaGetLastError();
}

}  // namespace jk
