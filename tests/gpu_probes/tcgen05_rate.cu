// Microbenchmark of the tcgen05 MMA issue rate on one SM (cta_group::1, M = 128,
// kind::f16 with BF16 operands and kind::tf32, K-major operands in shared memory),
// used to size the MMA lists of the tensor-core MTTKRP.  One CTA per SM; one thread
// issues a stream of MMAs and times it with clock64 until their commit completes.
//
//   part 1: cycles per MMA against N (32 ... 256), operand row width (64- or
//           128-byte swizzle) and the number of accumulators written in turn;
//   part 2: one pipeline stage of the exact-chain two-step kernel in isolation
//           (2 K slices x 4 stacked MMAs of N = 256, 192, 128, 64) with and without
//           the per-stage commit and the wait on an already complete barrier.
//
// All operands are finite BF16 values in shared memory; every descriptor stays
// inside the CTA's buffers and every accumulator inside its TMEM allocation; the
// one wait is bounded.  Prints one JSON line.
#include <cstdio>
#include <vector>

#include <cuda_runtime.h>

#include "../../paper_2112_03985_gb300/csrc/jk_ptx.cuh"

using namespace jk::ptx;

namespace {

template <int ROW>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  constexpr uint64_t layout = ROW == 128 ? 2 : 4;   // 128-byte swizzle 2, 64-byte 4
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * ROW) >> 4) << 32) |
         ((uint64_t)1 << 46) | (layout << 61);
}

__device__ __forceinline__ uint32_t idesc_for(int kind, int N) {
  const uint32_t fmt = kind == kKindTF32 ? 2u : 1u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (((uint32_t)N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

constexpr int kIters = 4096;     // MMAs per measurement (part 1)
constexpr int kStages = 512;     // stages per measurement (part 2)
constexpr int kBufBytes = 96 * 1024;

// fills the CTA's operand buffers with finite BF16 values in [0.5, 2)
__device__ void fill_operands(unsigned char* sm) {
  for (int i = threadIdx.x * 4; i < kBufBytes; i += blockDim.x * 4) {
    uint32_t x = (uint32_t)i * 2654435761u + 12345u;
    x ^= x >> 13;
    x *= 0x5bd1e995u;
    x ^= x >> 15;
    *(uint32_t*)(sm + i) = (0x3F00u | (x & 0xFFu)) | ((0x3F00u | ((x >> 16) & 0xFFu)) << 16);
  }
}

// part 1: A = 128 rows x ROW bytes at sm, B = 256 rows x ROW bytes at sm + 32 KB
template <int ROW, int KIND>
__global__ void __launch_bounds__(128, 1) rate_kernel(int N, int nacc, long long* cyc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  fill_operands(sm);
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  fence_async_shared();
  __syncthreads();
  if (threadIdx.x < 32) tmem_alloc(&tslot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    const uint32_t id = idesc_for(KIND, N);
    const uint64_t ad = sdesc<ROW>(smem_u32(sm));
    const uint64_t bd = sdesc<ROW>(smem_u32(sm + 32 * 1024));
    constexpr int KS = ROW / 32;   // 32-byte K slices per operand row
    const long long t0 = clock64();
    int acc = 0;
    for (int it = 0; it < kIters / KS; ++it) {
#pragma unroll
      for (int kk = 0; kk < KS; ++kk) {
        tc_mma<KIND>(tmem + (uint32_t)(acc * N), ad + 2 * kk, bd + 2 * kk, id, it > 0 ? 1u : 0u);
        if (++acc == nacc) acc = 0;
      }
    }
    tc_commit(&bar);
    wait_bounded(&bar, 0, &abort_flag, err, 1);
    cyc[blockIdx.x] = clock64() - t0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(tmem, 512);
}

// part 2: A = 4 parts x 128 rows x 64 B at sm, B = 256 rows x 64 B at sm + 32 KB
__global__ void __launch_bounds__(128, 1) stage_kernel(int variant, long long* cyc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[4], empty[4], fin;
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  fill_operands(sm);
  if (threadIdx.x == 0) {
    for (int s = 0; s < 4; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&fin, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  fence_async_shared();
  __syncthreads();
  if (threadIdx.x == 0)
    for (int s = 0; s < 4; ++s) mbar_arrive(&full[s]);   // phase 0 of every full barrier completes
  if (threadIdx.x < 32) tmem_alloc(&tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  if (threadIdx.x == 0) {
    uint32_t id[5];
    for (int c = 0; c < 5; ++c) id[c] = idesc_for(kKindBF16, 64 * c);
    const uint64_t ad = sdesc<64>(smem_u32(sm));
    const uint64_t bd = sdesc<64>(smem_u32(sm + 32 * 1024));
    constexpr uint32_t a16 = (128 * 64) >> 4;
    const long long t0 = clock64();
    int s = 0;
    for (int st = 0; st < kStages; ++st) {
      if (variant >= 2) {
        wait_bounded(&full[s], 0, &abort_flag, err, 1);
        tc_fence_after();
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          tc_mma<kKindBF16>(tmem + (uint32_t)p * 64, ad + (uint64_t)(p * a16 + 2 * kk), bd + (uint64_t)(2 * kk),
                            id[4 - p], (st > 0 || kk > 0) ? 1u : 0u);
      if (variant >= 1) tc_commit(&empty[s]);
      if (++s == 4) s = 0;
    }
    tc_commit(&fin);
    wait_bounded(&fin, 0, &abort_flag, err, 2);
    cyc[blockIdx.x] = clock64() - t0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(tmem, 256);
}

constexpr int kGrid = 148;
constexpr int kSmem = 120 * 1024;   // with the 1024-byte alignment slack; one CTA per SM

double mean_cycles(const long long* d) {
  std::vector<long long> h(kGrid);
  cudaMemcpy(h.data(), d, kGrid * sizeof(long long), cudaMemcpyDeviceToHost);
  double m = 0;
  for (long long v : h) m += (double)v;
  return m / kGrid;
}

template <int ROW, int KIND>
double rate(int N, int nacc, long long* d, int* e) {
  cudaFuncSetAttribute(rate_kernel<ROW, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  for (int rep = 0; rep < 2; ++rep) rate_kernel<ROW, KIND><<<kGrid, 128, kSmem>>>(N, nacc, d, e);
  cudaDeviceSynchronize();
  return mean_cycles(d) / kIters;
}

double stage(int variant, long long* d, int* e) {
  cudaFuncSetAttribute(stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  for (int rep = 0; rep < 2; ++rep) stage_kernel<<<kGrid, 128, kSmem>>>(variant, d, e);
  cudaDeviceSynchronize();
  return mean_cycles(d) / kStages;
}

}  // namespace

int main() {
  long long* d = nullptr;
  int* e = nullptr;
  if (cudaMalloc(&d, kGrid * sizeof(long long)) != cudaSuccess || cudaMalloc(&e, sizeof(int)) != cudaSuccess) {
    printf("{\"error\": \"cudaMalloc\"}\n");
    return 1;
  }
  cudaMemset(e, 0, sizeof(int));
  printf("{\"cycles_per_mma\": [");
  const int Ns[] = {32, 64, 128, 256};
  bool first = true;
  for (int N : Ns) {
    const double b64 = rate<64, kKindBF16>(N, 1, d, e);
    const double b128 = rate<128, kKindBF16>(N, 1, d, e);
    const double b64r = rate<64, kKindBF16>(N, N <= 128 ? 4 : 2, d, e);
    const double t128 = rate<128, kKindTF32>(N, 1, d, e);
    printf("%s{\"N\": %d, \"bf16_row64\": %.1f, \"bf16_row128\": %.1f, \"bf16_row64_rotating_acc\": %.1f, "
           "\"tf32_row128\": %.1f}",
           first ? "" : ", ", N, b64, b128, b64r, t128);
    first = false;
  }
  const double s0 = stage(0, d, e), s1 = stage(1, d, e), s2 = stage(2, d, e);
  int he = 0;
  cudaMemcpy(&he, e, sizeof(int), cudaMemcpyDeviceToHost);
  const cudaError_t st = cudaGetLastError();
  printf("], \"stage_cycles\": {\"mmas_only\": %.1f, \"with_commit\": %.1f, \"with_commit_wait_fence\": %.1f, "
         "\"ideal\": 704}, \"wait_errors\": %d, \"cuda\": \"%s\"}\n",
         s0, s1, s2, he, cudaGetErrorString(st));
  cudaFree(d);
  cudaFree(e);
  return (st == cudaSuccess && he == 0) ? 0 : 1;
}
