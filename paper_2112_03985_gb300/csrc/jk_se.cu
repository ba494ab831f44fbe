// Alg. 2 post-processing on the device: each jackknife submodel is adjusted to a
// reference model (Alg. 2 adjustment line: column signs by the largest-magnitude
// rule, then the column permutation that best matches the reference), and the
// jackknife standard error of every factor entry is formed over the adjusted
// submodels (Alg. 2 std line), modes other than the sampled mode.
//
// align_kernel: one CTA per submodel.  Signs: in every mode but the last, the
// entry of largest magnitude of each column (the first such row on ties) is made
// positive and the flip is carried into the last mode, so the model is unchanged.
// Match score of submodel column r against reference column s: the product over
// the modes other than the sampled one of |cos| of the two columns.  The
// permutation maximises the summed score: for R <= 8 by walking all R!
// permutations in lexicographic order (a later one replaces the best only when it
// is larger by more than 1e-15, so ties go to the lexicographically first); for
// larger R by the Hungarian method (Kuhn-Munkres, shortest augmenting paths with
// row and column potentials, O(R^3)) on one thread.
//
// se_kernel: one thread per factor entry; S = sqrt((G-1)/G * sum_g (x_g - mean)^2)
// with the sums taken in submodel order and every operation rounded on its own
// (no fused multiply-add).
#include "jk_common.cuh"

namespace jk {

namespace {

constexpr int kSeThreads = 128;
constexpr int kSeWarps = kSeThreads / 32;
constexpr int kMaxBruteR = 8;
constexpr int kMaxSeR = kMaxRank;

__device__ __forceinline__ double warp_sum(double v) {
  for (int s = 16; s; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  return v;
}

__global__ void __launch_bounds__(kSeThreads) align_kernel(SeArgs a) {
  __shared__ double score[kMaxSeR][kMaxSeR + 1];
  __shared__ double nA[kMaxModes][kMaxSeR], nB[kMaxModes][kMaxSeR];
  __shared__ signed char sgn[kMaxModes][kMaxSeR];
  __shared__ int perm[kMaxSeR];
  // Hungarian method state (thread 0)
  __shared__ double hu[kMaxSeR + 1], hv[kMaxSeR + 1], minv[kMaxSeR + 1];
  __shared__ int hp[kMaxSeR + 1], way[kMaxSeR + 1];
  __shared__ bool used[kMaxSeR + 1];

  const int g = blockIdx.x;
  const int R = a.R, N = a.N, last = N - 1;
  const int64_t C = a.C;
  const int64_t o = a.col_off[g];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // signs: largest-|.| entry of each column positive, modes 0 .. N-2
  for (int t = warp; t < last * R; t += kSeWarps) {
    const int k = t / R, r = t % R;
    const double* u = a.U[k] + o + r;
    double best = -1.0;
    long long bi = -1;
    for (int64_t i = lane; i < a.dims[k]; i += 32) {
      const double v = fabs(u[i * C]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
    for (int s = 16; s; s >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, s);
      const long long oi = __shfl_xor_sync(0xffffffffu, bi, s);
      if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) sgn[k][r] = (bi >= 0 && u[bi * C] < 0.0) ? -1 : 1;
  }

  // column norms (floored at 1e-300) of submodel and reference, modes != sampled
  for (int t = warp; t < N * R; t += kSeWarps) {
    const int k = t / R, r = t % R;
    if (k == a.n_hat) continue;
    double sa = 0.0, sb = 0.0;
    for (int64_t i = lane; i < a.dims[k]; i += 32) {
      const double x = a.U[k][i * C + o + r];
      const double y = a.ref[k][i * a.ref_ld + r];
      sa += x * x;
      sb += y * y;
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (lane == 0) {
      nA[k][r] = fmax(sqrt(sa), 1e-300);
      nB[k][r] = fmax(sqrt(sb), 1e-300);
    }
  }
  __syncthreads();

  // score[r][s] = prod_{k != sampled} |cos(submodel column r, reference column s)|
  for (int t = warp; t < R * R; t += kSeWarps) {
    const int r = t / R, s = t % R;
    double prod = 1.0;
    for (int k = 0; k < N; ++k) {
      if (k == a.n_hat) continue;
      double d = 0.0;
      for (int64_t i = lane; i < a.dims[k]; i += 32) d += a.U[k][i * C + o + r] * a.ref[k][i * a.ref_ld + s];
      d = warp_sum(d);
      prod *= fabs(d / (nA[k][r] * nB[k][s]));
    }
    // |cos| <= 1 up to rounding; a NaN (non-finite factors) scores 0 so that the
    // assignment below always finds a column
    if (lane == 0) score[r][s] = (prod >= 0.0 && prod <= 2.0) ? prod : 0.0;
  }
  __syncthreads();

  if (threadIdx.x == 0) {
    for (int r = 0; r < R; ++r) {
      int f = 1;
      for (int k = 0; k < last; ++k) f *= sgn[k][r];
      sgn[last][r] = (signed char)f;
    }
    if (R <= kMaxBruteR) {
      int p[kMaxBruteR], bp[kMaxBruteR];
      for (int i = 0; i < R; ++i) p[i] = bp[i] = i;
      double best = -1.0;
      for (;;) {
        double s = 0.0;
        for (int j = 0; j < R; ++j) s = __dadd_rn(s, score[p[j]][j]);
        if (s > __dadd_rn(best, 1e-15)) {
          best = s;
          for (int j = 0; j < R; ++j) bp[j] = p[j];
        }
        // next permutation in lexicographic order
        int i = R - 2;
        while (i >= 0 && p[i] > p[i + 1]) --i;
        if (i < 0) break;
        int j = R - 1;
        while (p[j] < p[i]) --j;
        int tmp = p[i];
        p[i] = p[j];
        p[j] = tmp;
        for (int lo = i + 1, hi = R - 1; lo < hi; ++lo, --hi) {
          tmp = p[lo];
          p[lo] = p[hi];
          p[hi] = tmp;
        }
      }
      for (int j = 0; j < R; ++j) perm[j] = bp[j];
    } else {
      // minimise cost(r, s) = -score[r][s]; rows r and columns s are 1-based here,
      // hp[s] = row matched to column s (0: none)
      const double inf = 1e300;
      for (int j = 0; j <= R; ++j) {
        hu[j] = 0.0;
        hv[j] = 0.0;
        hp[j] = 0;
        way[j] = 0;
      }
      bool failed = false;
      for (int i = 1; i <= R && !failed; ++i) {
        hp[0] = i;
        int j0 = 0;
        for (int j = 0; j <= R; ++j) {
          minv[j] = inf;
          used[j] = false;
        }
        do {
          used[j0] = true;
          const int i0 = hp[j0];
          double delta = inf;
          int j1 = 0;
          for (int j = 1; j <= R; ++j) {
            if (used[j]) continue;
            const double cur = -score[i0 - 1][j - 1] - hu[i0] - hv[j];
            if (cur < minv[j]) {
              minv[j] = cur;
              way[j] = j0;
            }
            if (minv[j] < delta) {
              delta = minv[j];
              j1 = j;
            }
          }
          for (int j = 0; j <= R; ++j) {
            if (used[j]) {
              hu[hp[j]] += delta;
              hv[j] -= delta;
            } else {
              minv[j] -= delta;
            }
          }
          if (j1 == 0) {  // unreachable with finite scores; never loop on it
            failed = true;
            break;
          }
          j0 = j1;
        } while (hp[j0] != 0);
        if (failed) break;
        do {
          const int j1 = way[j0];
          hp[j0] = hp[j1];
          j0 = j1;
        } while (j0 != 0);
      }
      for (int s = 0; s < R; ++s) perm[s] = failed ? s : hp[s + 1] - 1;
    }
  }
  __syncthreads();

  if (threadIdx.x < R) a.perm[(int64_t)g * R + threadIdx.x] = perm[threadIdx.x];
  // adjusted submodel: column s of the output is column perm[s], sign-fixed
  for (int k = 0; k < N; ++k) {
    const int64_t E = a.dims[k] * R;
    double* out = a.aligned[k] + (int64_t)g * E;
    for (int64_t e = threadIdx.x; e < E; e += kSeThreads) {
      const int64_t i = e / R;
      const int s = (int)(e % R);
      const int r = perm[s];
      const double x = a.U[k][i * C + o + r];
      out[e] = sgn[k][r] < 0 ? -x : x;
    }
  }
}

__global__ void se_kernel(SeArgs a) {
  const int k = blockIdx.y;
  if (k == a.n_hat) return;
  const int64_t E = a.dims[k] * a.R;
  const double* x = a.aligned[k];
  const double f = __ddiv_rn((double)(a.G - 1), (double)a.G);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    double sum = x[e];
    for (int g = 1; g < a.G; ++g) sum = __dadd_rn(sum, x[(int64_t)g * E + e]);
    const double mean = __ddiv_rn(sum, (double)a.G);
    double ss = 0.0;
    for (int g = 0; g < a.G; ++g) {
      const double d = __dsub_rn(x[(int64_t)g * E + e], mean);
      ss = __dadd_rn(ss, __dmul_rn(d, d));
    }
    a.S[k][e] = __dsqrt_rn(__dmul_rn(f, ss));
  }
}

}  // namespace

cudaError_t launch_jackknife_se(const SeArgs& a, cudaStream_t s) {
  if (a.R < 1 || a.R > kMaxSeR || a.G < 1 || a.N < 2 || a.N > kMaxModes) return cudaErrorInvalidValue;
  align_kernel<<<(unsigned)a.G, kSeThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t Emax = 0;
  for (int k = 0; k < a.N; ++k) Emax = a.dims[k] * a.R > Emax ? a.dims[k] * a.R : Emax;
  const unsigned bx = (unsigned)((Emax + 255) / 256 < 4096 ? (Emax + 255) / 256 : 4096);
  se_kernel<<<dim3(bx, (unsigned)a.N), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace jk
