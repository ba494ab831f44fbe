// Per-submodel update after the concurrent MTTKRP of one mode (Alg. 3, the
// loop over p inside the mode loop), all in FP64:
//
//   H^(n)_g  = *_{k != n} G^(k)_g                       (Hadamard line)
//   L L^T    = H^(n)_g                                  (Cholesky; non-positive pivot -> NOT_SPD)
//   Ubar^(n)_{|g} = Mbar_{n|g} (H^(n)_g)^{-1}           (update line, two triangular solves per row)
//   rows D_g := 0                      if n == n_hat    (zeroing line)
//   columns scaled to unit norm        if n < N-1       (normalisation, a reading; see oracle)
//   G^(n)_g  = Ubar^(n)_{|g}^T Ubar^(n)_{|g}            (Gram refresh for the next Hadamard)
//   e_g = ||T_{-g}||^2 + sum(H*G) - 2 sum(U*M)  if n == N-1   (error line)
//
// Phase A (grid: row chunks x blocks) sums the split-K partials of its rows in
// a fixed order, solves, zeroes, writes the unscaled rows and a partial Gram
// (upper triangle) and partial sum(U*M) per chunk.  Phase B (one CTA per
// block) reduces the chunk partials in a fixed order, normalises, stores the
// Gram and evaluates the error.  Both are deterministic.
//
// Bound: latency and FP64 issue rate (the work is O(I_n C R) flops per mode,
// R <= 32, against O(prod I * C) for the MTTKRP); the memory traffic is one read
// of the S partials and one write + one read-modify-write of Ubar^(n).
#include <math.h>

#include "jk_common.cuh"

namespace jk {
namespace {

constexpr int NTA = 128;  // threads of phase A = max rows per chunk
constexpr int NTB = 128;
constexpr int GP = kMaxRank * kMaxRank;  // stride of one partial Gram

__device__ __forceinline__ bool is_left_out(const BlockMeta& bm, int g, int64_t i) {
  const int64_t b = bm.lo_ptr[g], e = bm.lo_ptr[g + 1];
  for (int64_t p = b; p < e; ++p)
    if (bm.lo_idx[p] == i) return true;
  return false;
}

template <typename PT>
__device__ __forceinline__ double load_part(const PT* p) {
  return (double)__ldg(p);
}

// unevaluated FP32 pair (hi, lo) of the exact-chain tensor-core form
template <>
__device__ __forceinline__ double load_part<float2>(const float2* p) {
  const float2 v = __ldg(p);
  return (double)v.x + (double)v.y;
}

constexpr int kPartBatch = 8;   // split-K partials loaded together per element

template <typename PT>
__global__ void __launch_bounds__(NTA) update_phase_a(UpdateArgs a) {
  const int g = blockIdx.x, rc = blockIdx.y;
  const int tid = threadIdx.x;
  if (a.status[g] != 0) return;
  const int R = a.bm.R[g], off = a.bm.off[g];
  const int go = a.bm.gram_off[g];

  __shared__ double Hs[kMaxRank][kMaxRank + 1];
  __shared__ double invd[kMaxRank];   // 1 / L_jj
  __shared__ double X[NTA * kMaxRank];
  __shared__ double red[NTA];
  __shared__ int spd_ok;

  for (int p = tid; p < R * R; p += NTA) {
    const int r = p / R, c = p % R;
    double h = 1.0;
    for (int k = 0; k < a.N; ++k)
      if (k != a.n) h *= a.gram[k][go + p];
    Hs[r][c] = h;
  }
  if (tid == 0) spd_ok = 1;
  __syncthreads();

  // Cholesky H = L L^T in place (lower triangle), column by column, one warp.
  if (tid < 32) {
    const int lane = tid;
    bool ok = true;
    for (int j = 0; j < R; ++j) {
      if (lane == 0) {
        double d = Hs[j][j];
        for (int k = 0; k < j; ++k) d -= Hs[j][k] * Hs[j][k];
        if (!(d > 0.0) || !isfinite(d)) {
          spd_ok = 0;
          d = 1.0;
        }
        // 1 / L_jj from the reciprocal square root: the column below and both
        // substitutions multiply by it (no FP64 division on the serial paths)
        const double rs = rsqrt(d);
        Hs[j][j] = d * rs;
        invd[j] = rs;
      }
      __syncwarp();
      const int i = j + 1 + lane;
      if (i < R) {
        double v = Hs[i][j];
        for (int k = 0; k < j; ++k) v -= Hs[i][k] * Hs[j][k];
        Hs[i][j] = v * invd[j];
      }
      __syncwarp();
    }
    (void)ok;
  }
  __syncthreads();
  if (!spd_ok) {
    if (rc == 0 && tid == 0) atomicOr(&a.status[g], (int)JKCALS_BLOCK_NOT_SPD);
    return;
  }

  const int64_t r0 = (int64_t)rc * a.rows_per_chunk;
  int64_t r1 = r0 + a.rows_per_chunk;
  if (r1 > a.I) r1 = a.I;
  const int64_t row = r0 + tid;
  const bool active = row < r1;
  const PT* part = reinterpret_cast<const PT*>(a.part);
  const int64_t IC = a.I * (int64_t)a.C;
  double fit = 0.0;
  if (active) {
    double m[kMaxRank], x[kMaxRank];
#pragma unroll
    for (int r = 0; r < kMaxRank; ++r) {
      double v = 0.0;
      if (r < R) {
        // the S partials in split order, loaded kPartBatch at a time (all in flight)
        const PT* p = part + row * a.C + off + r;
        for (int s0 = 0; s0 < a.S; s0 += kPartBatch) {
          double t[kPartBatch];
#pragma unroll
          for (int u = 0; u < kPartBatch; ++u) t[u] = s0 + u < a.S ? load_part(p + (int64_t)(s0 + u) * IC) : 0.0;
#pragma unroll
          for (int u = 0; u < kPartBatch; ++u)
            if (s0 + u < a.S) v += t[u];
        }
      }
      m[r] = v;
    }
    const bool zero = (a.n == a.n_hat) && is_left_out(a.bm, g, row);
    if (zero) {
#pragma unroll
      for (int r = 0; r < kMaxRank; ++r) x[r] = 0.0;
    } else {
      // forward: L y = m
#pragma unroll
      for (int r = 0; r < kMaxRank; ++r) {
        if (r < R) {
          double v = m[r];
#pragma unroll
          for (int k = 0; k < r; ++k) v -= Hs[r][k] * x[k];
          x[r] = v * invd[r];
        } else {
          x[r] = 0.0;
        }
      }
      // backward: L^T u = y
#pragma unroll
      for (int r = kMaxRank - 1; r >= 0; --r) {
        if (r < R) {
          double v = x[r];
#pragma unroll
          for (int k = r + 1; k < kMaxRank; ++k)
            if (k < R) v -= Hs[k][r] * x[k];
          x[r] = v * invd[r];
        }
      }
    }
    double* urow = a.U + row * a.C + off;
#pragma unroll
    for (int r = 0; r < kMaxRank; ++r) {
      if (r < R) {
        urow[r] = x[r];
        X[tid * R + r] = x[r];
        fit = fma(x[r], m[r], fit);
      }
    }
  }
  __syncthreads();

  // Partial Gram (upper triangle) over this chunk's rows.
  const int nrows = (int)(r1 > r0 ? r1 - r0 : 0);
  double* gp = a.gpart + ((int64_t)g * a.RC + rc) * GP;
  for (int p = tid; p < R * R; p += NTA) {
    const int r = p / R, c = p % R;
    if (c < r) continue;
    double acc = 0.0;
    for (int t = 0; t < nrows; ++t) acc = fma(X[t * R + r], X[t * R + c], acc);
    gp[r * kMaxRank + c] = acc;
  }
  if (a.n == a.N - 1) {
    red[tid] = fit;
    __syncthreads();
    for (int w = NTA / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) a.fpart[(int64_t)g * a.RC + rc] = red[0];
  }
}

__global__ void __launch_bounds__(NTB) update_phase_b(UpdateArgs a) {
  const int g = blockIdx.x;
  const int tid = threadIdx.x;
  const bool last = (a.n == a.N - 1);
  const int sweep = last ? *a.sweep_idx : 0;
  if (a.status[g] != 0) {
    if (last && tid == 0 && a.loss_hist != nullptr && sweep < a.loss_cap)
      a.loss_hist[(int64_t)sweep * a.K + g] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  const int R = a.bm.R[g], off = a.bm.off[g];
  const int go = a.bm.gram_off[g];
  __shared__ double G[kMaxRank][kMaxRank + 1];
  __shared__ double nrm[kMaxRank];
  __shared__ double red[NTB];

  for (int p = tid; p < R * R; p += NTB) {
    const int r = p / R, c = p % R;
    if (c < r) continue;
    double acc = 0.0;
    for (int rc = 0; rc < a.RC; ++rc) acc += a.gpart[((int64_t)g * a.RC + rc) * GP + r * kMaxRank + c];
    G[r][c] = acc;
    G[c][r] = acc;
  }
  __syncthreads();
  if (a.normalise && a.n < a.N - 1) {
    if (tid < R) {
      const double v = sqrt(G[tid][tid]);
      nrm[tid] = (v > 0.0) ? v : 1.0;
    }
    __syncthreads();
    for (int p = tid; p < R * R; p += NTB) {
      const int r = p / R, c = p % R;
      G[r][c] = G[r][c] / (nrm[r] * nrm[c]);
    }
    for (int64_t t = tid; t < a.I * R; t += NTB) {
      const int64_t i = t / R;
      const int r = (int)(t - i * R);
      double* u = a.U + i * a.C + off + r;
      *u = *u / nrm[r];
    }
    __syncthreads();
  }
  for (int p = tid; p < R * R; p += NTB) a.gram_n[go + p] = G[p / R][p % R];
  if (a.UT != nullptr) {
    // FP32 transposed copy for the tensor-core MTTKRP: UT[c][i], i fastest
    for (int64_t t = tid; t < a.I * R; t += NTB) {
      const int r = (int)(t / a.I);
      const int64_t i = t - (int64_t)r * a.I;
      const double u = a.U[i * a.C + off + r];
      const float hi = (float)u;
      a.UT[(int64_t)(off + r) * a.I_pad + i] = hi;
      if (a.UT_lo != nullptr) a.UT_lo[(int64_t)(off + r) * a.I_pad + i] = (float)(u - (double)hi);
    }
    if (a.cmax != nullptr) {
      __syncthreads();
      const int warp = tid >> 5, lane = tid & 31;
      for (int r = warp; r < R; r += NTB / 32) {
        float mx = 0.f;
        const float* col = a.UT + (int64_t)(off + r) * a.I_pad;
        for (int64_t i = lane; i < a.I; i += 32) mx = fmaxf(mx, fabsf(col[i]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) a.cmax[off + r] = mx;
      }
    }
  }
  if (!last) return;

  // e_g = ||T_{-g}||^2 + sum(H * G) - 2 sum(U * M)
  double hg = 0.0;
  for (int p = tid; p < R * R; p += NTB) {
    double h = 1.0;
    for (int k = 0; k < a.N; ++k)
      if (k != a.n) h *= a.gram[k][go + p];
    hg = fma(h, G[p / R][p % R], hg);
  }
  red[tid] = hg;
  __syncthreads();
  for (int w = NTB / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) {
    double fit = 0.0;
    for (int rc = 0; rc < a.RC; ++rc) fit += a.fpart[(int64_t)g * a.RC + rc];
    const double nt = a.normT2[g];
    const double e = nt + red[0] - 2.0 * fit;
    a.loss_last[g] = e;
    if (a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = e;
    const double tol = *a.tol;
    const double prev = a.loss_prev[g];
    if (tol > 0.0 && isfinite(prev) && fabs(prev - e) / nt < tol)
      a.status[g] |= JKCALS_BLOCK_CONVERGED;
    a.loss_prev[g] = e;
  }
}

__global__ void advance_sweep_kernel(int* sweep_idx) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *sweep_idx += 1;
}

// the sweep counters of several problems (a grouped batch sweep)
__global__ void advance_sweeps_kernel(int* const* sweep_idx, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) *sweep_idx[i] += 1;
}

// ---- gradient ---------------------------------------------------------------

struct GradArgs {
  int N, n, n_hat, C;
  int64_t I;
  BlockMeta bm;
  const double* U;
  const double* gram[kMaxModes];
  const double* M;
  double* G;
};

__global__ void __launch_bounds__(128) grad_epilogue_kernel(GradArgs a, int rows_per_chunk) {
  const int g = blockIdx.x;
  const int R = a.bm.R[g], off = a.bm.off[g], go = a.bm.gram_off[g];
  __shared__ double Hs[kMaxRank][kMaxRank + 1];
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) {
    double h = 1.0;
    for (int k = 0; k < a.N; ++k)
      if (k != a.n) h *= a.gram[k][go + p];
    Hs[p / R][p % R] = h;
  }
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  int64_t r1 = r0 + rows_per_chunk;
  if (r1 > a.I) r1 = a.I;
  for (int64_t row = r0 + threadIdx.x; row < r1; row += blockDim.x) {
    const bool zero = (a.n == a.n_hat) && is_left_out(a.bm, g, row);
    const double* u = a.U + row * a.C + off;
    const double* m = a.M + row * a.C + off;
    double* out = a.G + row * a.C + off;
    for (int r = 0; r < R; ++r) {
      double v = 0.0;
      if (!zero) {
        for (int s = 0; s < R; ++s) v = fma(u[s], Hs[s][r], v);
        v = 2.0 * (v - m[r]);
      }
      out[r] = v;
    }
  }
}

__global__ void __launch_bounds__(128) grad_block_loss_kernel(GradArgs a, const double* normT2,
                                                              double* eg) {
  const int g = blockIdx.x;
  const int R = a.bm.R[g], off = a.bm.off[g], go = a.bm.gram_off[g];
  __shared__ double red[128];
  double acc = 0.0;
  // -2 sum(U * M) over the block (rows D_g of the sampled mode are zero in U)
  for (int64_t t = threadIdx.x; t < a.I * R; t += blockDim.x) {
    const int64_t i = t / R;
    const int r = (int)(t - i * R);
    acc = fma(-2.0 * a.U[i * a.C + off + r], a.M[i * a.C + off + r], acc);
  }
  // + sum(H * G_{N-1})
  for (int p = threadIdx.x; p < R * R; p += blockDim.x) {
    double h = 1.0;
    for (int k = 0; k < a.N; ++k) h *= a.gram[k][go + p];
    acc += h;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) eg[g] = normT2[g] + red[0];
}

__global__ void sum_blocks_kernel(const double* eg, int K, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc = 0.0;
    for (int g = 0; g < K; ++g) acc += eg[g];
    out[0] = acc;
  }
}

}  // namespace

cudaError_t launch_update(const UpdateArgs& a, cudaStream_t s) {
  dim3 ga((unsigned)a.K, (unsigned)a.RC);
  if (a.part_kind == kPartF32)
    update_phase_a<float><<<ga, NTA, 0, s>>>(a);
  else if (a.part_kind == kPartF32x2)
    update_phase_a<float2><<<ga, NTA, 0, s>>>(a);
  else
    update_phase_a<double><<<ga, NTA, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  update_phase_b<<<a.K, NTB, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_advance_sweep(int* sweep_idx, cudaStream_t s) {
  advance_sweep_kernel<<<1, 32, 0, s>>>(sweep_idx);
  return cudaGetLastError();
}

cudaError_t launch_advance_sweeps(int* const* sweep_idx, int n, cudaStream_t s) {
  advance_sweeps_kernel<<<(n + 127) / 128, 128, 0, s>>>(sweep_idx, n);
  return cudaGetLastError();
}

cudaError_t launch_grad_epilogue(int N, int n, int n_hat, int64_t I, int C, int K, BlockMeta bm,
                                 const double* U, const double* const* gram, const double* M,
                                 double* G, cudaStream_t s) {
  GradArgs a{};
  a.N = N; a.n = n; a.n_hat = n_hat; a.C = C; a.I = I; a.bm = bm; a.U = U; a.M = M; a.G = G;
  for (int k = 0; k < N; ++k) a.gram[k] = gram[k];
  const int rpc = 128;
  dim3 grid((unsigned)K, (unsigned)((I + rpc - 1) / rpc));
  grad_epilogue_kernel<<<grid, 128, 0, s>>>(a, rpc);
  return cudaGetLastError();
}

cudaError_t launch_grad_loss(int N, int64_t I, int C, int K, BlockMeta bm, const double* U,
                             const double* const* gram, const double* M, const double* normT2,
                             double* eg_and_out, cudaStream_t s) {
  // eg_and_out: K per-block values followed by the sum
  GradArgs a{};
  a.N = N; a.n = N - 1; a.C = C; a.I = I; a.bm = bm; a.U = U; a.M = M;
  for (int k = 0; k < N; ++k) a.gram[k] = gram[k];
  grad_block_loss_kernel<<<K, 128, 0, s>>>(a, normT2, eg_and_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sum_blocks_kernel<<<1, 32, 0, s>>>(eg_and_out, K, eg_and_out + K);
  return cudaGetLastError();
}

}  // namespace jk
