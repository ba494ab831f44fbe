// jkcals_mttkrp_f64_noalloc: the FP64 concurrent MTTKRP without any device
// allocation, for callers that cannot call cudaMalloc (see include/jkcals.h).
//
// The split-K partial products live in one file-scope device array of fixed
// size instead of a handle's workspace.  In host code the array's name is a
// host-side stand-in, not a device address, so its device address is looked
// up once per device with cudaGetSymbolAddress (with that device current) and
// that pointer is what the kernels receive.
#include <algorithm>
#include <mutex>
#include <string>

#include "jk_common.cuh"

namespace jk {
namespace {

// 2^21 doubles = 16 MiB of split-K partials, held by every GPU that loads the
// library until the process exits.
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up on first use).
cudaError_t scratch_for_current_device(double** out, int* device) {
  cudaError_t e = cudaGetDevice(device);
  if (e != cudaSuccess) return e;
  if (*device < 0 || *device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[*device] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[*device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[*device];
  return cudaSuccess;
}

// True for device memory of `device` (or managed memory).  A pointer into
// another GPU's memory is refused: the kernels would read it through peer
// access, which need not be enabled.
bool is_device_pointer(const void* p, int device) {
  cudaPointerAttributes attr{};
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeManaged) return true;
  return attr.type == cudaMemoryTypeDevice && attr.device == device;
}

jkcals_status fail_na(jkcals_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

}  // namespace
}  // namespace jk

using namespace jk;

extern "C" jkcals_status jkcals_mttkrp_f64_noalloc(int N, const int64_t* dims, int mode, const double* Tn,
                                                   const double* const* U, int C, double* M_out,
                                                   void* stream) {
  set_error("");
  if (N < 2 || N > kMaxModes) return fail_na(JKCALS_ERR_ARG, "N must be in [2, 8]");
  if (dims == nullptr || U == nullptr || Tn == nullptr || M_out == nullptr)
    return fail_na(JKCALS_ERR_ARG, "NULL argument");
  if (mode < 0 || mode >= N) return fail_na(JKCALS_ERR_ARG, "mode out of range");
  if (C < 1) return fail_na(JKCALS_ERR_ARG, "C must be >= 1");
  if ((int64_t)C > 65535LL * 64) return fail_na(JKCALS_ERR_UNSUPPORTED, "C must be <= 4194240");
  int64_t total = 1;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1) return fail_na(JKCALS_ERR_ARG, "dims must be >= 1");
    if (dims[k] > 2147483647LL) return fail_na(JKCALS_ERR_UNSUPPORTED, "dims must be < 2^31");
    total *= dims[k];
    if (total >= (int64_t(1) << 40)) return fail_na(JKCALS_ERR_UNSUPPORTED, "prod(dims) must be < 2^40");
  }
  const int64_t I = dims[mode];
  const int64_t J = total / I;
  if (I * (int64_t)C > kNoAllocScratchDoubles)
    return fail_na(JKCALS_ERR_UNSUPPORTED,
                   "dims[mode] * C exceeds the static scratch of 2^21 doubles (16 MiB)");
  double* scratch = nullptr;
  int device = 0;
  cudaError_t e = scratch_for_current_device(&scratch, &device);
  if (e != cudaSuccess) return fail_na(JKCALS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  if (!is_device_pointer(Tn, device) || !is_device_pointer(M_out, device))
    return fail_na(JKCALS_ERR_ARG, "Tn and M_out must be device memory of the current device");
  KrpOperands kr{};
  int o = 0;
  for (int k = 0; k < N; ++k) {
    if (k == mode) continue;
    if (U[k] == nullptr || !is_device_pointer(U[k], device))
      return fail_na(JKCALS_ERR_ARG, "U[k] must be device memory of the current device");
    kr.U[o] = U[k];
    kr.dims[o] = (int)dims[k];
    ++o;
  }
  kr.nother = o;

  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return fail_na(JKCALS_ERR_CUDA, cudaGetErrorString(e));

  // split-K factor: about 4 CTAs per SM, at least 4 k-steps of 16 per split,
  // and no more partials than the scratch holds
  const int64_t BK = 16, BM = 64, BN = 64;
  const int64_t tiles = ((I + BM - 1) / BM) * ((C + BN - 1) / BN);
  const int64_t ksteps = (J + BK - 1) / BK;
  int64_t S = (4 * (int64_t)sms + tiles - 1) / tiles;
  S = std::min<int64_t>(S, std::max<int64_t>(1, ksteps / 4));
  S = std::min<int64_t>(S, kNoAllocScratchDoubles / (I * (int64_t)C));
  S = std::max<int64_t>(1, std::min<int64_t>(S, ksteps));
  const int64_t kchunk = ((ksteps + S - 1) / S) * BK;
  S = (J + kchunk - 1) / kchunk;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = launch_mttkrp_f64(Tn, I, J, C, kr, (int)S, kchunk, scratch, st);
  if (e == cudaSuccess) e = launch_reduce_partials_f64(scratch, (int)S, I * (int64_t)C, M_out, st);
  if (e != cudaSuccess) return fail_na(JKCALS_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return JKCALS_OK;
}
