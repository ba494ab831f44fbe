// Self-test of the bounded waits that every pipelined kernel of the library
// relies on (jk_ptx.cuh: wait_bounded): a wait on a barrier phase that nothing
// completes must give up after its limit, raise the CTA's abort flag and record
// its code in the error word, and another role blocked in a wait of its own
// must then leave through the abort flag, long before its own limit.  No trap,
// no fault: the kernel returns and the context stays usable.
#include <string>

#include "jk_common.cuh"
#include "jk_ptx.cuh"

namespace jk {
namespace {

using namespace ptx;

constexpr int kSelftestCodeA = 3;   // code the timing-out role records
constexpr int kSelftestCodeB = 4;   // code of the role that must leave through the abort flag

// out[0]: role A's wait returned true (must not); out[1]: role B's likewise;
// out[2]: microseconds from the start until role B left its wait.
__global__ void bounded_wait_selftest_kernel(int* err, int* out, uint64_t limit_ns) {
  __shared__ uint64_t never[2];
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&never[0], 1);
    mbar_init(&never[1], 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  __syncthreads();
  const uint64_t t0 = global_ns();
  if (threadIdx.x == 0) {
    // role A: phase 0 of a fresh barrier with one expected arrival and none coming
    out[0] = wait_bounded_ns(&never[0], 0, &abort_flag, err, kSelftestCodeA, limit_ns) ? 1 : 0;
  } else if (threadIdx.x == 32) {
    // role B (another warp): a limit 64 times longer; the abort flag ends it
    out[1] = wait_bounded_ns(&never[1], 0, &abort_flag, err, kSelftestCodeB, 64 * limit_ns) ? 1 : 0;
    out[2] = (int)((global_ns() - t0) / 1000);
  }
  __syncthreads();
}

jkcals_status fail(jkcals_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

}  // namespace
}  // namespace jk

extern "C" jkcals_status jkcals_selftest_bounded_wait(double limit_ms, int* code, double* left_after_ms) {
  using namespace jk;
  if (!(limit_ms > 0.0) || limit_ms > 100.0 || code == nullptr || left_after_ms == nullptr)
    return fail(JKCALS_ERR_ARG, "jkcals_selftest_bounded_wait: 0 < limit_ms <= 100 and both outputs are required");
  int* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 4 * sizeof(int));
  if (e != cudaSuccess) return fail(JKCALS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  int h[4] = {0, 0, 0, 0};
  e = cudaMemset(d, 0, 4 * sizeof(int));
  if (e == cudaSuccess) {
    bounded_wait_selftest_kernel<<<1, 64>>>(d, d + 1, (uint64_t)(limit_ms * 1e6));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, d, 4 * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
  *code = h[0];
  *left_after_ms = h[3] / 1000.0;
  if (h[1] != 0 || h[2] != 0)
    return fail(JKCALS_ERR_STATE, "bounded-wait self-test: a wait on a phase that never completes returned true");
  set_error("");
  return JKCALS_OK;
}
