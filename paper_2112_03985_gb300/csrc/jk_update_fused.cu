// Fused per-submodel update, one CTA per block (Alg. 3, the loop over p inside
// the mode loop), in FP64 (for the tensor-core forms the wide kernel's row work
// runs in double-float on the FP32 pipe, see update_wide_body).  Input: the S split-K partials of the
// concurrent MTTKRP Mbar_n (S x I_n x C: FP64, FP32 or FP32 pairs by form); the
// block sums the partials of its own rows in split order, with the steps of the
// reduction kernels, so Mbar_n is the same FP64 value they would give.
//
//   H = *_{k != n} G^(k)_g ; L L^T = H            (Hadamard line; Cholesky)
//   x_i = L^-T L^-1 m_i for every row i            (update line)
//   x_i = 0 for i in D_g when n == n_hat           (zeroing line)
//   G = sum_i x_i x_i^T                            (Gram refresh)
//   columns scaled to unit norm if n < N-1         (normalisation reading)
//   e_g = ||T_{-g}||^2 + sum(H*G) - 2 sum(x*m)     (error line, last mode)
//
// The block's rows stay in shared memory between the solve, the Gram and the
// scaling, so Ubar^(n)_{|g} is written once (FP64 row-major for the update,
// plus the transposed FP32 hi/lo copies and column maxima that the
// tensor-core MTTKRP reads).  The Gram is reduced over row groups in a fixed
// order: deterministic.  Used when every block's rows fit in shared memory and
// there are enough blocks to fill the GPU; otherwise the two-phase update runs.
#include <math.h>

#include <string>

#include "jk_common.cuh"

namespace jk {
namespace {

constexpr int NT = 128;

__device__ __forceinline__ bool left_out(const BlockMeta& bm, int g, int64_t i) {
  const int64_t b = bm.lo_ptr[g], e = bm.lo_ptr[g + 1];
  for (int64_t p = b; p < e; ++p)
    if (bm.lo_idx[p] == i) return true;
  return false;
}

// FP32 pair of a double u: hi = fl32(u), lo = fl32(u - hi), both rounded to
// nearest even, as the conversions give them, but formed from u's bit pattern
// with integer operations: the FP64 pipe (which also runs FP64 conversions) is
// narrow on this part and the update is bound by it.  hi keeps the top 24
// significant bits of u's 53 (round half to even on the low 29); u - hi is
// that remainder, at most 29 bits, converted exactly to FP32 and scaled by the
// power of two of its unit.  Magnitudes outside [2^-70, 2^120) (and 0, Inf,
// NaN) take the conversions.
__device__ __forceinline__ void split_f32_pair(double u, float& hi, float& lo) {
  const long long bits = __double_as_longlong(u);
  const uint32_t hw = (uint32_t)((unsigned long long)bits >> 32), lw = (uint32_t)bits;
  const int e = (int)((hw >> 20) & 0x7ffu) - 1023;   // unbiased exponent
  if (e < -70 || e >= 120) {
    hi = __double2float_rn(u);
    lo = __double2float_rn(u - (double)hi);
    return;
  }
  const uint32_t sign = hw & 0x80000000u;
  uint32_t keep = ((hw & 0xfffffu) << 3) | (lw >> 29);   // the 23 stored bits of hi
  const uint32_t rem = lw & 0x1fffffffu;                  // the 29 bits below them
  const bool up = rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u));
  uint32_t fexp = (uint32_t)(e + 127);
  uint32_t r;   // |u - hi| in units of 2^(e - 52)
  if (up) {
    r = 0x20000000u - rem;
    if (++keep == 0x800000u) {
      keep = 0;
      ++fexp;
    }
  } else {
    r = rem;
  }
  hi = __uint_as_float(sign | (fexp << 23) | keep);
  if (r == 0) {
    lo = 0.f;
    return;
  }
  const float mag = __uint2float_rn(r) * __uint_as_float((uint32_t)(e - 52 + 127) << 23);   // exact
  lo = (up != (sign != 0u)) ? -mag : mag;   // u - hi has u's sign when hi was rounded down
}

// ---- double-float arithmetic for the tensor-core forms' row work ----------------
// A value is an unevaluated pair h + l of FP32 numbers with |l| <= ulp(h)/2 (about
// 48 significant bits).  Sums use Knuth's TwoSum on the leading parts, products
// the FMA-exact product of the leading parts plus the cross terms; each result is
// renormalised with a fast two-sum.  Relative error of one operation about
// 2^-44, far below the tensor-core forms' MTTKRP error (>= 2e-9).  All steps
// are explicit round-to-nearest intrinsics, so no contraction or reassociation
// changes them.
struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl dfl_of(double x) {
  dfl r;
  split_f32_pair(x, r.h, r.l);
  return r;
}

__device__ __forceinline__ double dfl_to_double(dfl a) { return df_to_double(a.h, a.l); }

__device__ __forceinline__ dfl dfl_renorm(float s, float t) {
  const float h = __fadd_rn(s, t);
  return dfl{h, __fsub_rn(t, __fsub_rn(h, s))};
}

__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return dfl_renorm(s, __fadd_rn(__fadd_rn(e, a.l), b.l));
}

__device__ __forceinline__ dfl dfl_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dfl_renorm(p, e);
}

// c - a * b
__device__ __forceinline__ dfl dfl_sub_mul(dfl c, dfl a, dfl b) {
  const dfl p = dfl_mul(a, b);
  return dfl_add(c, dfl{-p.h, -p.l});
}

// c + a * b
__device__ __forceinline__ dfl dfl_add_mul(dfl c, dfl a, dfl b) { return dfl_add(c, dfl_mul(a, b)); }

__device__ __forceinline__ dfl dfl_shfl_xor(dfl a, int o) {
  return dfl{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}

// RMAX bounds the rank of every block; FIXED means every block has exactly RMAX
// components, so the per-rank guards fold away at compile time.
template <int RMAX, bool FIXED>
__device__ __forceinline__ void update_fused_body(const UpdateArgs& a, int g, double* X) {
  const int tid = threadIdx.x;
  const bool last = (a.n == a.N - 1);
  const int sweep = last ? *a.sweep_idx : 0;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  if (a.status[g] != 0) {
    if (last && tid == 0 && a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = qnan;
    return;
  }
  const int R = FIXED ? RMAX : a.bm.R[g];
  const int off = a.bm.off[g], go = a.bm.gram_off[g];
  const int64_t I = a.I;
  const int64_t count = I * (int64_t)a.C;   // elements of one partial

  // X: I x R rows of this block, dynamic shared memory
  __shared__ double L[RMAX][RMAX + 1];      // H, then its Cholesky factor
  __shared__ double Hc[RMAX * RMAX];        // H kept for the error
  __shared__ double G[RMAX][RMAX + 1];
  __shared__ double invd[RMAX];
  __shared__ double scale[RMAX];
  __shared__ double red[NT];
  __shared__ int spd_ok;
  __shared__ int colmax[RMAX];   // FP32 bit patterns of max |hi| per column (non-negative: int order)

  if (tid < RMAX) colmax[tid] = 0;
  const int warp = tid >> 5;
  if (warp == 0) {
    // warp 0: H (its R^2 entries over the lanes), then its Cholesky factor,
    // while the other warps load the block's rows of Mbar_n
    const int lane = tid;
    if (lane == 0) spd_ok = 1;
    for (int p = lane; p < R * R; p += 32) {
      double h = 1.0;
      for (int k = 0; k < a.N; ++k)
        if (k != a.n) h *= a.gram[k][go + p];
      L[p / R][p % R] = h;
      Hc[p] = h;
    }
    __syncwarp();
    for (int j = 0; j < R; ++j) {
      if (lane == 0) {
        double d = L[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0) || !isfinite(d)) {
          spd_ok = 0;
          d = 1.0;
        }
        // 1 / L_jj straight from the reciprocal square root (the solves use
        // only the reciprocals; one FP64 sequence instead of a root and a
        // division on the serial path)
        const double rs = rsqrt(d);
        L[j][j] = d * rs;
        invd[j] = rs;
      }
      __syncwarp();
      const int i = j + 1 + lane;
      if (i < R) {
        double v = L[i][j];
        for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
        L[i][j] = v * invd[j];
      }
      __syncwarp();
    }
  } else {
    // warps 1.. : this block's rows of Mbar_n into X, each element the sum of its
    // S partials in split order (a few rows per thread, each split's loads
    // issued before its adds)
    constexpr int kLd = RMAX <= 4 ? 4 : (RMAX < 8 ? 2 : 1);
    constexpr int NL = NT - 32;
    for (int64_t i0 = tid - 32; i0 < I; i0 += (int64_t)kLd * NL) {
      double v[kLd][RMAX];
      // partials loaded PB splits at a time, then added in split order
      constexpr int PB = RMAX <= 8 ? 2 : 1;
      if (a.part_kind == kPartF64) {
        const double* P = reinterpret_cast<const double*>(a.part);
        for (int s0 = 0; s0 < a.S; s0 += PB) {
          double t[PB][kLd][RMAX];
#pragma unroll
          for (int q = 0; q < PB; ++q)
#pragma unroll
            for (int u = 0; u < kLd; ++u) {
              const int64_t i = i0 + (int64_t)u * NL;
#pragma unroll
              for (int r = 0; r < RMAX; ++r)
                t[q][u][r] = (s0 + q < a.S && i < I && r < R) ? __ldg(P + (s0 + q) * count + i * a.C + off + r) : 0.0;
            }
#pragma unroll
          for (int q = 0; q < PB; ++q)
            if (s0 + q < a.S) {
#pragma unroll
              for (int u = 0; u < kLd; ++u)
#pragma unroll
                for (int r = 0; r < RMAX; ++r) v[u][r] = s0 + q == 0 ? t[q][u][r] : v[u][r] + t[q][u][r];
            }
        }
      } else {
        float hi[kLd][RMAX], lo[kLd][RMAX];
#pragma unroll
        for (int u = 0; u < kLd; ++u)
#pragma unroll
          for (int r = 0; r < RMAX; ++r) hi[u][r] = lo[u][r] = 0.f;
        const bool pairs = a.part_kind == kPartF32x2;
        for (int s0 = 0; s0 < a.S; s0 += PB) {
          float2 t[PB][kLd][RMAX];
#pragma unroll
          for (int q = 0; q < PB; ++q)
#pragma unroll
            for (int u = 0; u < kLd; ++u) {
              const int64_t i = i0 + (int64_t)u * NL;
#pragma unroll
              for (int r = 0; r < RMAX; ++r) {
                t[q][u][r] = make_float2(0.f, 0.f);
                if (s0 + q < a.S && i < I && r < R) {
                  const int64_t e = (s0 + q) * count + i * a.C + off + r;
                  if (pairs)
                    t[q][u][r] = __ldg(reinterpret_cast<const float2*>(a.part) + e);
                  else
                    t[q][u][r].x = __ldg(reinterpret_cast<const float*>(a.part) + e);
                }
              }
            }
#pragma unroll
          for (int q = 0; q < PB; ++q)
            if (s0 + q < a.S) {
#pragma unroll
              for (int u = 0; u < kLd; ++u)
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                  df_add(hi[u][r], lo[u][r], t[q][u][r].x);
                  if (pairs) lo[u][r] = __fadd_rn(lo[u][r], t[q][u][r].y);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kLd; ++u)
#pragma unroll
          for (int r = 0; r < RMAX; ++r) v[u][r] = df_to_double(hi[u][r], lo[u][r]);
      }
#pragma unroll
      for (int u = 0; u < kLd; ++u) {
        const int64_t i = i0 + (int64_t)u * NL;
        if (i < I) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < R) X[i * R + r] = v[u][r];
        }
      }
    }
  }
  __syncthreads();
  if (!spd_ok) {
    if (tid == 0) {
      atomicOr(&a.status[g], (int)JKCALS_BLOCK_NOT_SPD);
      if (last && a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = qnan;
    }
    return;
  }

  // solve every row in place in X
  double fit = 0.0;
  for (int64_t i = tid; i < I; i += NT) {
    double x[RMAX], m[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) m[r] = (r < R) ? X[i * R + r] : 0.0;
    if (a.n == a.n_hat && left_out(a.bm, g, i)) {
#pragma unroll
      for (int r = 0; r < RMAX; ++r) x[r] = 0.0;
    } else {
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        if (r < R) {
          double v = m[r];
#pragma unroll
          for (int k = 0; k < r; ++k) v -= L[r][k] * x[k];
          x[r] = v * invd[r];
        } else {
          x[r] = 0.0;
        }
      }
#pragma unroll
      for (int r = RMAX - 1; r >= 0; --r) {
        if (r < R) {
          double v = x[r];
#pragma unroll
          for (int k = r + 1; k < RMAX; ++k)
            if (k < R) v -= L[k][r] * x[k];
          x[r] = v * invd[r];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      if (r < R) {
        X[i * R + r] = x[r];
        if (last) fit = fma(x[r], m[r], fit);   // sum(x * m) enters the error only
      }
    }
  }
  __syncthreads();

  // Gram (upper triangle), row groups reduced in a fixed order
  const int npairs = R * (R + 1) / 2;
  const int groups = NT / npairs;
  if (groups == 0) {
    // R > 22: one thread per pair, all rows
    for (int p = tid; p < npairs; p += NT) {
      int q = p, r0 = 0;
      while (q >= R - r0) {
        q -= R - r0;
        ++r0;
      }
      double acc = 0.0;
      for (int64_t i = 0; i < I; ++i) acc = fma(X[i * R + r0], X[i * R + r0 + q], acc);
      G[r0][r0 + q] = acc;
      G[r0 + q][r0] = acc;
    }
    __syncthreads();
  } else {
    double acc = 0.0;
    int pr = 0, pc = 0;
    const int p = tid % npairs, grp = tid / npairs;
    if (grp < groups) {
      int q = p;
      while (q >= R - pr) {
        q -= R - pr;
        ++pr;
      }
      pc = pr + q;
      for (int64_t i = grp; i < I; i += groups) acc = fma(X[i * R + pr], X[i * R + pc], acc);
    }
    red[tid] = acc;
    __syncthreads();
    if (tid < npairs) {
      double s = 0.0;
      for (int gg = 0; gg < groups; ++gg) s += red[gg * npairs + tid];
      int q = tid, r0 = 0;
      while (q >= R - r0) {
        q -= R - r0;
        ++r0;
      }
      G[r0][r0 + q] = s;
      G[r0 + q][r0] = s;
    }
    __syncthreads();
  }

  // normalisation (modes n < N-1): unit columns, norm dropped
  const bool norm = a.normalise && a.n < a.N - 1;
  if (tid < R) {
    double sc = 1.0;
    if (norm) {
      const double v = sqrt(G[tid][tid]);
      sc = (v > 0.0) ? 1.0 / v : 1.0;
    }
    scale[tid] = sc;
  }
  __syncthreads();
  if (norm) {
    for (int p = tid; p < R * R; p += NT) G[p / R][p % R] *= scale[p / R] * scale[p % R];
    for (int64_t t = tid; t < I * R; t += NT) X[t] *= scale[t % R];
    __syncthreads();
  }

  // write the factor block: FP64 row-major, and the transposed FP32 hi/lo copies
  for (int64_t t = tid; t < I * R; t += NT) {
    const int64_t i = t / R;
    const int r = (int)(t - i * R);
    a.U[i * a.C + off + r] = X[t];
  }
  if (a.UT != nullptr) {
    // transposed FP32 copies, and the column maxima of the high parts (the
    // bound of |U| that the tensor-core form scales by)
    for (int64_t t = tid; t < I * R; t += NT) {
      const int r = (int)(t / I);
      const int64_t i = t - (int64_t)r * I;
      float hi, lo;
      split_f32_pair(X[i * R + r], hi, lo);
      a.UT[(int64_t)(off + r) * a.I_pad + i] = hi;
      if (a.UT_lo != nullptr) a.UT_lo[(int64_t)(off + r) * a.I_pad + i] = lo;
      if (a.cmax != nullptr) atomicMax(&colmax[r], __float_as_int(fabsf(hi)));
    }
    if (a.cmax != nullptr) {
      __syncthreads();
      if (tid < R) a.cmax[off + tid] = __int_as_float(colmax[tid]);
    }
  }
  for (int p = tid; p < R * R; p += NT) a.gram_n[go + p] = G[p / R][p % R];
  if (!last) return;

  // e_g = ||T_{-g}||^2 + sum(H * G) - 2 sum(x * m): warp sums, then the warps'
  // partials in order (fixed order: deterministic)
  double hg = 0.0;
  for (int p = tid; p < R * R; p += NT) hg = fma(Hc[p], G[p / R][p % R], hg);
  double v = hg - 2.0 * fit;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((tid & 31) == 0) red[warp] = v;
  __syncthreads();
  if (tid == 0) {
    double acc = 0.0;
    for (int w = 0; w < NT / 32; ++w) acc += red[w];
    const double nt = a.normT2[g];
    const double e = nt + acc;
    a.loss_last[g] = e;
    if (a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = e;
    const double tol = *a.tol;
    const double prev = a.loss_prev[g];
    if (tol > 0.0 && isfinite(prev) && fabs(prev - e) / nt < tol) a.status[g] |= JKCALS_BLOCK_CONVERGED;
    a.loss_prev[g] = e;
  }
}

template <int RMAX, bool FIXED>
__global__ void __launch_bounds__(NT, FIXED ? 4 : 2) update_fused_kernel(UpdateArgs a) {
  extern __shared__ double X[];
  update_fused_body<RMAX, FIXED>(a, blockIdx.x, X);
}

// Wide form of the same update for ranks <= 7: one CTA per block, warp 0 forms
// H and its Cholesky factor while up to 224 row threads (one or two rows each, or more)
// sum their rows' split-K partials; then every row thread solves its rows and
// keeps its contributions to the Gram entries G_ab (a <= b) and to sum(x * m)
// in registers.  A reduce-scatter across the lanes of each warp (halving the
// number of values per lane at each of five shuffle steps: about NPAD adds per
// lane instead of 5 NPAD for a plain butterfly) and a fixed-order sum over the
// warps give the Gram and the fit term; all arithmetic stays in FP64 and the
// order of every sum is fixed (deterministic).  One row per thread shortens
// each block's chain of dependent FP64 operations, which bounds the
// narrow-row-count updates.
constexpr int kWideRows = 224;   // row threads per CTA at most (two CTAs of rank 5 fit an SM)

__host__ __device__ constexpr int wide_npad(int rmax) {
  return rmax * (rmax + 1) / 2 + 1 <= 16 ? 16 : 32;
}

// Row threads of the wide update of a mode with I rows: one row each for I <= 128
// (those updates are bound by one block's chain of dependent operations), two
// for wider ones (fewer warps, so fewer FP64 adds in the cross-lane reduction).
__host__ __device__ inline int wide_row_threads(int64_t I) {
  int64_t rt = I <= 128 ? (I + 31) / 32 * 32 : ((I + 1) / 2 + 31) / 32 * 32;
  return (int)(rt > kWideRows ? kWideRows : rt);
}

// Block g of one problem; the CTA has at least 32 + wide_row_threads(a.I)
// threads; the ones beyond take no rows but meet every barrier.
// DF (tensor-core forms): the split-K sums stay FP32 pairs, and the row solves,
// the Gram and fit sums and their reduction run in double-float arithmetic on the
// FP32 pipe; the R x R Hadamard, its Cholesky factor, the normalisation and the
// error stay FP64.  Without DF (the FP64 form) every step is FP64.
template <int RMAX, bool FIXED, bool DF>
__device__ __forceinline__ void update_wide_body(const UpdateArgs& a, int g, double* X) {
  constexpr int NP = RMAX * (RMAX + 1) / 2;   // Gram entries (upper triangle), then the fit term
  constexpr int NPAD = wide_npad(RMAX);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int RT = wide_row_threads(a.I);       // row threads
  const bool rows = warp > 0 && tid < 32 + RT;   // this thread takes rows
  const bool last = (a.n == a.N - 1);
  const int sweep = last ? *a.sweep_idx : 0;
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  if (a.status[g] != 0) {
    if (last && tid == 0 && a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = qnan;
    return;
  }
  const int R = FIXED ? RMAX : a.bm.R[g];
  const int off = a.bm.off[g], go = a.bm.gram_off[g];
  const int64_t I = a.I;
  const int64_t count = I * (int64_t)a.C;   // elements of one partial

  // X: I x R rows of this block (Mbar rows, then the solutions), dynamic shared memory
  __shared__ double L[RMAX][RMAX + 1];
  __shared__ double Hc[RMAX * RMAX];
  __shared__ double invd[RMAX];
  __shared__ dfl Lp[DF ? RMAX : 1][RMAX + 1];   // DF: L and 1 / diag(L) as pairs
  __shared__ dfl invdp[DF ? RMAX : 1];
  __shared__ double scale[RMAX];
  __shared__ double wsum[(kWideRows + 32) / 32][NPAD];
  __shared__ double tot[NPAD];
  __shared__ int spd_ok;
  __shared__ int colmax[RMAX];

  if (tid < RMAX) colmax[tid] = 0;
  if (warp == 0) {
    if (lane == 0) spd_ok = 1;
    for (int p = lane; p < R * R; p += 32) {
      double h = 1.0;
      for (int k = 0; k < a.N; ++k)
        if (k != a.n) h *= a.gram[k][go + p];
      L[p / R][p % R] = h;
      Hc[p] = h;
    }
    __syncwarp();
    for (int j = 0; j < R; ++j) {
      if (lane == 0) {
        double d = L[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0) || !isfinite(d)) {
          spd_ok = 0;
          d = 1.0;
        }
        const double rs = rsqrt(d);
        L[j][j] = d * rs;
        invd[j] = rs;
      }
      __syncwarp();
      const int i = j + 1 + lane;
      if (i < R) {
        double v = L[i][j];
        for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
        L[i][j] = v * invd[j];
      }
      __syncwarp();
    }
    if constexpr (DF) {
      for (int p = lane; p < R * R; p += 32) {
        const int r = p / R, k = p % R;
        if (k < r) Lp[r][k] = dfl_of(L[r][k]);
        if (k == r) invdp[r] = dfl_of(invd[r]);
      }
    }
  } else {
    // the block's rows of Mbar_n: each element the sum of its S partials in split
    // order; the partials are loaded PB splits at a time (all in flight together)
    // and then added in order, one memory round trip per batch
    constexpr int PB = RMAX <= 4 ? 8 : 4;
    for (int64_t i = tid - 32; rows && i < I; i += RT) {
      double v[RMAX];
      if (a.part_kind == kPartF64) {
        const double* P = reinterpret_cast<const double*>(a.part);
#pragma unroll
        for (int r = 0; r < RMAX; ++r) v[r] = 0.0;
        for (int s0 = 0; s0 < a.S; s0 += PB) {
          double t[PB][RMAX];
#pragma unroll
          for (int u = 0; u < PB; ++u)
#pragma unroll
            for (int r = 0; r < RMAX; ++r)
              t[u][r] = (s0 + u < a.S && r < R) ? __ldg(P + (s0 + u) * count + i * a.C + off + r) : 0.0;
#pragma unroll
          for (int u = 0; u < PB; ++u)
            if (s0 + u < a.S) {
#pragma unroll
              for (int r = 0; r < RMAX; ++r) v[r] = s0 + u == 0 ? t[u][r] : v[r] + t[u][r];
            }
        }
      } else {
        float hi[RMAX], lo[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) hi[r] = lo[r] = 0.f;
        const bool pairs = a.part_kind == kPartF32x2;
        for (int s0 = 0; s0 < a.S; s0 += PB) {
          float2 t[PB][RMAX];
#pragma unroll
          for (int u = 0; u < PB; ++u)
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
              t[u][r] = make_float2(0.f, 0.f);
              if (s0 + u < a.S && r < R) {
                const int64_t e = (s0 + u) * count + i * a.C + off + r;
                if (pairs)
                  t[u][r] = __ldg(reinterpret_cast<const float2*>(a.part) + e);
                else
                  t[u][r].x = __ldg(reinterpret_cast<const float*>(a.part) + e);
              }
            }
#pragma unroll
          for (int u = 0; u < PB; ++u)
            if (s0 + u < a.S) {
#pragma unroll
              for (int r = 0; r < RMAX; ++r) {
                df_add(hi[r], lo[r], t[u][r].x);
                if (pairs) lo[r] = __fadd_rn(lo[r], t[u][r].y);
              }
            }
        }
        if constexpr (DF) {
          // the pair itself (renormalised), no FP64 conversion
          float2* X2 = reinterpret_cast<float2*>(X);
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < R) {
              const dfl m = dfl_renorm(hi[r], lo[r]);
              X2[i * R + r] = make_float2(m.h, m.l);
            }
          continue;
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r) v[r] = df_to_double(hi[r], lo[r]);
      }
      if constexpr (DF) {
        float2* X2 = reinterpret_cast<float2*>(X);
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) {
            const dfl m = dfl_of(v[r]);
            X2[i * R + r] = make_float2(m.h, m.l);
          }
      } else {
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) X[i * R + r] = v[r];
      }
    }
  }
  __syncthreads();
  if (!spd_ok) {
    if (tid == 0) {
      atomicOr(&a.status[g], (int)JKCALS_BLOCK_NOT_SPD);
      if (last && a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = qnan;
    }
    return;
  }

  // solve this thread's rows; Gram and fit contributions in registers
  double acc[NPAD];
#pragma unroll
  for (int p = 0; p < NPAD; ++p) acc[p] = 0.0;
  if constexpr (DF) {
    dfl accp[NPAD];
#pragma unroll
    for (int p = 0; p < NPAD; ++p) accp[p] = dfl{0.f, 0.f};
    float2* X2 = reinterpret_cast<float2*>(X);
    if (rows) {
      for (int64_t i = tid - 32; i < I; i += RT) {
        dfl x[RMAX], m[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
          const float2 t = (r < R) ? X2[i * R + r] : make_float2(0.f, 0.f);
          m[r] = dfl{t.x, t.y};
          x[r] = dfl{0.f, 0.f};
        }
        if (!(a.n == a.n_hat && left_out(a.bm, g, i))) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r) {
            if (r < R) {
              dfl v = m[r];
#pragma unroll
              for (int k = 0; k < r; ++k) v = dfl_sub_mul(v, Lp[r][k], x[k]);
              x[r] = dfl_mul(v, invdp[r]);
            }
          }
#pragma unroll
          for (int r = RMAX - 1; r >= 0; --r) {
            if (r < R) {
              dfl v = x[r];
#pragma unroll
              for (int k = r + 1; k < RMAX; ++k)
                if (k < R) v = dfl_sub_mul(v, Lp[k][r], x[k]);
              x[r] = dfl_mul(v, invdp[r]);
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) X2[i * R + r] = make_float2(x[r].h, x[r].l);
        int p = 0;
#pragma unroll
        for (int r0 = 0; r0 < RMAX; ++r0)
#pragma unroll
          for (int r1 = r0; r1 < RMAX; ++r1) accp[p] = dfl_add_mul(accp[p], x[r0], x[r1]), ++p;   // zero beyond R
        if (last) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r) accp[NP] = dfl_add_mul(accp[NP], x[r], m[r]);
        }
      }
    }
    // reduce-scatter as below, on the pairs
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int o = 16 >> st;
      const bool up = (lane & o) != 0;
      const int half = NPAD >> (st + 1);
      if (half >= 1) {
#pragma unroll
        for (int jj = 0; jj < NPAD / 2; ++jj) {
          if (jj < half) {
            const dfl send = up ? accp[jj] : accp[half + jj];
            const dfl keep = up ? accp[half + jj] : accp[jj];
            accp[jj] = dfl_add(keep, dfl_shfl_xor(send, o));
          }
        }
      } else {
        accp[0] = dfl_add(accp[0], dfl_shfl_xor(accp[0], o));
      }
    }
    constexpr int KEEPP = NPAD >= 32 ? NPAD / 32 : 1;
#pragma unroll
    for (int jj = 0; jj < KEEPP; ++jj) acc[jj] = dfl_to_double(accp[jj]);
  } else {
    if (rows) {
      for (int64_t i = tid - 32; i < I; i += RT) {
        double x[RMAX], m[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) m[r] = (r < R) ? X[i * R + r] : 0.0;
        if (a.n == a.n_hat && left_out(a.bm, g, i)) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r) x[r] = 0.0;
        } else {
#pragma unroll
          for (int r = 0; r < RMAX; ++r) {
            if (r < R) {
              double v = m[r];
#pragma unroll
              for (int k = 0; k < r; ++k) v -= L[r][k] * x[k];
              x[r] = v * invd[r];
            } else {
              x[r] = 0.0;
            }
          }
#pragma unroll
          for (int r = RMAX - 1; r >= 0; --r) {
            if (r < R) {
              double v = x[r];
#pragma unroll
              for (int k = r + 1; k < RMAX; ++k)
                if (k < R) v -= L[k][r] * x[k];
              x[r] = v * invd[r];
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
          if (r < R) X[i * R + r] = x[r];
        int p = 0;
#pragma unroll
        for (int r0 = 0; r0 < RMAX; ++r0)
#pragma unroll
          for (int r1 = r0; r1 < RMAX; ++r1) acc[p] = fma(x[r0], x[r1], acc[p]), ++p;   // zero beyond R
        if (last) {
#pragma unroll
          for (int r = 0; r < RMAX; ++r) acc[NP] = fma(x[r], m[r], acc[NP]);
        }
      }
    }
    // reduce-scatter across the warp: at the step with lane offset o a lane keeps
    // the half of its values that its bit o selects and adds its partner's copy
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int o = 16 >> st;
      const bool up = (lane & o) != 0;
      const int half = NPAD >> (st + 1);
      if (half >= 1) {
#pragma unroll
        for (int j = 0; j < NPAD / 2; ++j) {
          if (j < half) {
            const double send = up ? acc[j] : acc[half + j];
            const double keep = up ? acc[half + j] : acc[j];
            acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
      } else {
        acc[0] = acc[0] + __shfl_xor_sync(0xffffffffu, acc[0], o);
      }
    }
  }
  {
    // the entries this lane now holds: base index from its lane bits, then j
    constexpr int KEEP = NPAD >= 32 ? NPAD / 32 : 1;
    int base = 0;
#pragma unroll
    for (int st = 0; st < 5; ++st) {
      const int half = NPAD >> (st + 1);
      if (half >= 1 && (lane & (16 >> st))) base += half;
    }
    if (NPAD >= 32 || (lane & 1) == 0) {
#pragma unroll
      for (int j = 0; j < KEEP; ++j) wsum[warp][base + j] = acc[j];
    }
  }
  __syncthreads();
  const int nw = (int)blockDim.x >> 5;   // warps beyond 32 + RT threads hold zeros
  if (tid <= NP) {
    double sacc = wsum[0][tid];
    for (int w = 1; w < nw; ++w) sacc += wsum[w][tid];
    tot[tid] = sacc;
  }
  __syncthreads();

  // normalisation (modes n < N-1): unit columns, norm dropped
  const bool norm = a.normalise && a.n < a.N - 1;
  auto gidx = [&](int r0, int r1) {   // position of G(r0, r1), r0 <= r1, in the packed upper triangle
    return r0 * RMAX - r0 * (r0 - 1) / 2 + (r1 - r0);
  };
  if (tid < R) {
    double sc = 1.0;
    if (norm) {
      const double v = sqrt(tot[gidx(tid, tid)]);
      sc = (v > 0.0) ? 1.0 / v : 1.0;
    }
    scale[tid] = sc;
  }
  __syncthreads();

  // the factor block: FP64 row-major, the transposed FP32 hi/lo copies and the
  // column maxima of the high parts
  float cm[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) cm[r] = 0.f;
  if (rows) {
    for (int64_t i = tid - 32; i < I; i += RT) {
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        if (r < R) {
          double x;
          if constexpr (DF) {
            const float2 t = reinterpret_cast<const float2*>(X)[i * R + r];
            const dfl xp = norm ? dfl_mul(dfl{t.x, t.y}, dfl_of(scale[r])) : dfl{t.x, t.y};
            x = dfl_to_double(xp);
          } else {
            x = norm ? X[i * R + r] * scale[r] : X[i * R + r];
          }
          a.U[i * a.C + off + r] = x;
          if (a.UT != nullptr) {
            float hi, lo;
            split_f32_pair(x, hi, lo);
            a.UT[(int64_t)(off + r) * a.I_pad + i] = hi;
            if (a.UT_lo != nullptr) a.UT_lo[(int64_t)(off + r) * a.I_pad + i] = lo;
            cm[r] = fmaxf(cm[r], fabsf(hi));
          }
        }
      }
    }
  }
  if (a.UT != nullptr && a.cmax != nullptr) {
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
      float v = cm[r];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0 && r < R) atomicMax(&colmax[r], __float_as_int(v));
    }
    __syncthreads();
    if (tid < R) a.cmax[off + tid] = __int_as_float(colmax[tid]);
  }
  // the refreshed Gram, scaled like the columns
  for (int p = tid; p < R * R; p += blockDim.x) {
    const int r0 = p / R, r1 = p % R;
    const double v = tot[r0 <= r1 ? gidx(r0, r1) : gidx(r1, r0)];
    a.gram_n[go + p] = norm ? v * scale[r0] * scale[r1] : v;
  }
  if (!last || tid != 0) return;

  // e_g = ||T_{-g}||^2 + sum(H * G) - 2 sum(x * m)
  double hg = 0.0;
  for (int p = 0; p < R * R; ++p) {
    const int r0 = p / R, r1 = p % R;
    hg = fma(Hc[p], tot[r0 <= r1 ? gidx(r0, r1) : gidx(r1, r0)], hg);
  }
  const double nt = a.normT2[g];
  const double e = nt + (hg - 2.0 * tot[NP]);
  a.loss_last[g] = e;
  if (a.loss_hist != nullptr && sweep < a.loss_cap) a.loss_hist[(int64_t)sweep * a.K + g] = e;
  const double tol = *a.tol;
  const double prev = a.loss_prev[g];
  if (tol > 0.0 && isfinite(prev) && fabs(prev - e) / nt < tol) a.status[g] |= JKCALS_BLOCK_CONVERGED;
  a.loss_prev[g] = e;
}

template <int RMAX, bool FIXED, bool DF>
__global__ void __launch_bounds__(kWideRows + 32, 1) update_wide_kernel(UpdateArgs a) {
  extern __shared__ double X[];
  update_wide_body<RMAX, FIXED, DF>(a, blockIdx.x, X);
}

// Block x of a grouped launch belongs to problem b with first[b] <= x < first[b + 1].
__device__ __forceinline__ int group_problem_u(const int* first, int nprob, int x) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(first + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void load_args(UpdateArgs& sa, const UpdateArgs* args, int b) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(args + b);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
  for (int i = threadIdx.x; i < (int)(sizeof(UpdateArgs) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
}

template <int RMAX, bool FIXED, bool DF>
__global__ void __launch_bounds__(kWideRows + 32, 1) update_wide_grouped_kernel(const UpdateArgs* __restrict__ args,
                                                                               const int* __restrict__ first,
                                                                               int nprob) {
  extern __shared__ double X[];
  __shared__ __align__(16) UpdateArgs sa;
  const int b = group_problem_u(first, nprob, (int)blockIdx.x);
  load_args(sa, args, b);
  __syncthreads();
  update_wide_body<RMAX, FIXED, DF>(sa, (int)blockIdx.x - __ldg(first + b), X);
}

template <int RMAX, bool FIXED>
__global__ void __launch_bounds__(NT, 2) update_fused_grouped_kernel(const UpdateArgs* __restrict__ args,
                                                                                const int* __restrict__ first,
                                                                                int nprob) {
  extern __shared__ double X[];
  __shared__ __align__(16) UpdateArgs sa;
  const int b = group_problem_u(first, nprob, (int)blockIdx.x);
  load_args(sa, args, b);
  __syncthreads();
  update_fused_body<RMAX, FIXED>(sa, (int)blockIdx.x - __ldg(first + b), X);
}

template <int RM, bool F, bool DF>
cudaError_t raise_wide_smem(size_t smem) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, update_wide_kernel<RM, F, DF>);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(update_wide_kernel<RM, F, DF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Tensor-core forms take the double-float row work where wide_update_double_float says so.
template <int RM, bool F>
cudaError_t run_wide(const UpdateArgs* a, size_t smem, cudaStream_t s, bool prepare) {
  if (prepare) {
    const cudaError_t e = raise_wide_smem<RM, F, false>(smem);
    return e != cudaSuccess ? e : raise_wide_smem<RM, F, true>(smem);
  }
  const unsigned threads = (unsigned)(wide_row_threads(a->I) + 32);
  if (wide_update_double_float(a->UT != nullptr, a->I))
    update_wide_kernel<RM, F, true><<<a->K, threads, smem, s>>>(*a);
  else
    update_wide_kernel<RM, F, false><<<a->K, threads, smem, s>>>(*a);
  return cudaGetLastError();
}

// Instances: exact ranks 1..8 when all blocks share one rank, otherwise the
// rank classes 8, 16, 32 with per-rank guards.
template <int RM, bool F>
cudaError_t run_fused(const UpdateArgs* a, size_t smem, cudaStream_t s, bool prepare) {
  if (prepare) {
    // the limit is per kernel and process-wide: only ever raise it, so that a
    // handle needing less never lowers it under another handle
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, update_fused_kernel<RM, F>);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(update_fused_kernel<RM, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  update_fused_kernel<RM, F><<<a->K, NT, smem, s>>>(*a);
  return cudaGetLastError();
}

static cudaError_t dispatch_fused(const UpdateArgs* a, size_t smem, int Rmax, bool uniform, cudaStream_t s,
                                  bool prepare) {
  if (uniform) {
    switch (Rmax) {
      case 1: return run_wide<1, true>(a, smem, s, prepare);
      case 2: return run_wide<2, true>(a, smem, s, prepare);
      case 3: return run_wide<3, true>(a, smem, s, prepare);
      case 4: return run_wide<4, true>(a, smem, s, prepare);
      case 5: return run_wide<5, true>(a, smem, s, prepare);
      case 6: return run_wide<6, true>(a, smem, s, prepare);
      case 7: return run_wide<7, true>(a, smem, s, prepare);
      case 8: return run_fused<8, true>(a, smem, s, prepare);
      default: break;
    }
  }
  if (Rmax <= 8) return run_fused<8, false>(a, smem, s, prepare);
  if (Rmax <= 16) return run_fused<16, false>(a, smem, s, prepare);
  return run_fused<32, false>(a, smem, s, prepare);
}

std::string g_grouped_attrs;   // attributes of the last grouped update kernel launched (diagnostics)

template <class KF>
cudaError_t run_grouped(KF kernel, bool prepare, unsigned threads, const UpdateArgs* args, const int* first,
                        int nprob, int total, size_t smem, cudaStream_t s) {
  if (prepare) {
    // the limit is per kernel and process-wide: only ever raise it
    cudaFuncAttributes fa{};
    const cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess)
    g_grouped_attrs = "max threads " + std::to_string(fa.maxThreadsPerBlock) + ", registers " +
                      std::to_string(fa.numRegs) + ", static smem " + std::to_string(fa.sharedSizeBytes) +
                      ", max dynamic smem " + std::to_string(fa.maxDynamicSharedSizeBytes);
  kernel<<<(unsigned)total, threads, smem, s>>>(args, first, nprob);
  return cudaGetLastError();
}

// The same instance that dispatch_fused picks for (Rmax, uniform), grouped; df:
// the double-float row work of the wide kernel (every problem of the launch
// agrees on it); threads: the largest CTA that a problem of the group takes on
// its own.
template <bool DF>
cudaError_t dispatch_wide_grouped(bool prepare, const UpdateArgs* args, const int* first, int nprob, int total,
                                  unsigned tw, int Rmax, size_t smem, cudaStream_t s) {
  switch (Rmax) {
    case 1: return run_grouped(update_wide_grouped_kernel<1, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
    case 2: return run_grouped(update_wide_grouped_kernel<2, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
    case 3: return run_grouped(update_wide_grouped_kernel<3, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
    case 4: return run_grouped(update_wide_grouped_kernel<4, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
    case 5: return run_grouped(update_wide_grouped_kernel<5, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
    case 6: return run_grouped(update_wide_grouped_kernel<6, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
    default: return run_grouped(update_wide_grouped_kernel<7, true, DF>, prepare, tw, args, first, nprob, total, smem, s);
  }
}

cudaError_t dispatch_grouped(bool prepare, const UpdateArgs* args, const int* first, int nprob, int total,
                             int threads, int Rmax, bool uniform, bool df, size_t smem, cudaStream_t s) {
  const unsigned tw = (unsigned)threads;
  if (uniform && Rmax >= 1 && Rmax <= 7)
    return df ? dispatch_wide_grouped<true>(prepare, args, first, nprob, total, tw, Rmax, smem, s)
              : dispatch_wide_grouped<false>(prepare, args, first, nprob, total, tw, Rmax, smem, s);
  if (uniform) {
    switch (Rmax) {
      case 8:
        return run_grouped(update_fused_grouped_kernel<8, true>, prepare, NT, args, first, nprob, total, smem, s);
      default: break;
    }
  }
  if (Rmax <= 8) return run_grouped(update_fused_grouped_kernel<8, false>, prepare, NT, args, first, nprob, total, smem, s);
  if (Rmax <= 16)
    return run_grouped(update_fused_grouped_kernel<16, false>, prepare, NT, args, first, nprob, total, smem, s);
  return run_grouped(update_fused_grouped_kernel<32, false>, prepare, NT, args, first, nprob, total, smem, s);
}

}  // namespace

std::string grouped_update_attrs() { return g_grouped_attrs; }

int update_fused_threads(int64_t I, int Rmax, bool uniform) {
  return (uniform && Rmax <= 7) ? wide_row_threads(I) + 32 : NT;
}

cudaError_t prepare_update_grouped(int threads, int Rmax, bool uniform, bool df, size_t smem) {
  return dispatch_grouped(true, nullptr, nullptr, 0, 0, threads, Rmax, uniform, df, smem, nullptr);
}

cudaError_t launch_update_grouped(const UpdateArgs* args, const int* first, int nprob, int total, int threads,
                                  int Rmax, bool uniform, bool df, size_t smem, cudaStream_t s) {
  return dispatch_grouped(false, args, first, nprob, total, threads, Rmax, uniform, df, smem, s);
}

size_t update_fused_smem(int64_t I, int Rmax) { return (size_t)I * Rmax * sizeof(double); }


cudaError_t prepare_update_fused(size_t smem, int Rmax, bool uniform) {
  return dispatch_fused(nullptr, smem, Rmax, uniform, nullptr, true);
}

cudaError_t launch_update_fused(const UpdateArgs& a, size_t smem, int Rmax, bool uniform, cudaStream_t s) {
  return dispatch_fused(&a, smem, Rmax, uniform, s, false);
}

}  // namespace jk
