// C ABI of libjkcals.so: handle lifecycle, planning, and the host-side
// orchestration of Alg. 3 (one concurrent MTTKRP + one fused per-block update
// per mode, the error after the last mode), replayed from a CUDA graph.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "jk_common.cuh"
#include "jk_tc.cuh"

namespace jk {
thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace jk

using namespace jk;

namespace {

constexpr int kMttkrpBK = 16;   // k-step of the FP64 MTTKRP kernel
constexpr int kMttkrpBM = 64;
constexpr int kMttkrpBN = 64;

jkcals_status fail(jkcals_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

jkcals_status fail_cuda(jkcals_ctx* h, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(JKCALS_ERR_OOM, m);
  }
  if (h != nullptr) {
    // Sticky errors poison the context; a later call returns STATE.
    cudaError_t sticky = cudaDeviceSynchronize();
    if (sticky != cudaSuccess) h->broken = true;
  }
  return fail(JKCALS_ERR_CUDA, m);
}

#define JK_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return fail_cuda((h), e_, #call); \
  } while (0)

#define JK_TRY(call)                         \
  do {                                       \
    jkcals_status s_ = (call);               \
    if (s_ != JKCALS_OK) return s_;          \
  } while (0)

// The library's stream-ordered memory pool of a device, created on first use.
// Handles allocate from it on their stream and free into it in stream order, so
// creating and destroying handles neither calls cudaMalloc nor waits for the
// device in cudaFree; up to kPoolKeepBytes of freed memory stays in the pool for
// the next handle (more is returned to the device at synchronisation points).
constexpr uint64_t kPoolKeepBytes = 2ull << 30;

cudaMemPool_t library_pool(int device) {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(device);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    pool = nullptr;   // the handles of this device then use cudaMalloc / cudaFree
  } else {
    uint64_t keep = kPoolKeepBytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  pools[device] = pool;
  return pool;
}

jkcals_status dalloc(jkcals_ctx* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->opt.max_device_bytes > 0 && h->bytes_allocated + (int64_t)bytes > h->opt.max_device_bytes)
    return fail(JKCALS_ERR_OOM, "device memory cap (max_device_bytes) reached");
  cudaError_t e = h->pool ? cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream) : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail_cuda(nullptr, e, h->pool ? "cudaMallocFromPoolAsync" : "cudaMalloc");
  }
  h->allocations.push_back(*p);
  h->bytes_allocated += (int64_t)bytes;
  return JKCALS_OK;
}

template <typename T>
jkcals_status dalloc_t(jkcals_ctx* h, T** p, size_t count) {
  void* v = nullptr;
  jkcals_status s = dalloc(h, &v, count * sizeof(T));
  *p = static_cast<T*>(v);
  return s;
}

// Frees p.  Unless only the handle's own stream used p (stream_only), first
// waits for the device as cudaFree does: a batch on another stream may still be
// reading it.
void dfree(jkcals_ctx* h, void* p, bool stream_only = false) {
  if (p == nullptr) return;
  auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
  if (it != h->allocations.end()) h->allocations.erase(it);
  if (!h->pool) {
    cudaFree(p);
    return;
  }
  if (!stream_only) cudaDeviceSynchronize();
  cudaFreeAsync(p, h->stream);
}

bool is_host_pointer(const void* p) {
  cudaPointerAttributes attr{};
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return attr.type == cudaMemoryTypeHost || attr.type == cudaMemoryTypeUnregistered;
}

BlockMeta block_meta(const jkcals_ctx* h) {
  BlockMeta bm;
  bm.R = h->d_R;
  bm.off = h->d_off;
  bm.gram_off = h->d_gram_off;
  bm.lo_ptr = h->d_lo_ptr;
  bm.lo_idx = h->d_lo_idx;
  return bm;
}

KrpOperands krp_operands(const jkcals_ctx* h, int n, double* const* U) {
  KrpOperands kr{};
  int o = 0;
  for (int k = 0; k < h->N; ++k) {
    if (k == n) continue;
    kr.U[o] = U[k];
    kr.dims[o] = (int)h->dims[k];
    ++o;
  }
  kr.nother = o;
  return kr;
}

void make_plan(jkcals_ctx* h) {
  const int target = 4 * h->num_sms;
  for (int n = 0; n < h->N; ++n) {
    ModePlan& p = h->plan[n];
    const int64_t I = h->dims[n], J = h->J[n];
    const int64_t tiles = ((I + kMttkrpBM - 1) / kMttkrpBM) * ((h->C + kMttkrpBN - 1) / kMttkrpBN);
    const int64_t ksteps = (J + kMttkrpBK - 1) / kMttkrpBK;
    int64_t S = h->opt.splits > 0 ? h->opt.splits : (target + tiles - 1) / tiles;
    // at least 4 k-steps per split, unless the output is small enough that its
    // partials cost little (at most 64 Ki elements per split): a short
    // contraction then still spreads over the SMs (GB300 runs about two FP64
    // FMAs per clock and SM, so a few busy SMs bound a small mode)
    const int64_t min_ksteps = I * h->C <= 65536 ? 1 : 4;
    if (h->opt.splits <= 0) S = std::min<int64_t>(S, std::max<int64_t>(1, ksteps / min_ksteps));
    S = std::max<int64_t>(1, std::min<int64_t>(S, ksteps));
    int64_t kchunk = ((ksteps + S - 1) / S) * kMttkrpBK;
    S = (J + kchunk - 1) / kchunk;
    p.splits = (int)S;
    p.kchunk = kchunk;
    // update: about two CTAs per SM, at most 128 rows per chunk
    int64_t RC = std::max<int64_t>(1, (2 * h->num_sms + h->K - 1) / h->K);
    RC = std::min<int64_t>(RC, std::max<int64_t>(1, (I + 31) / 32));
    int64_t rpc = (I + RC - 1) / RC;
    if (rpc > 128) {
      RC = (I + 127) / 128;
      rpc = (I + RC - 1) / RC;
    }
    RC = (I + rpc - 1) / rpc;
    p.upd.rows_per_chunk = (int)rpc;
    p.upd.RC = (int)RC;
    // fused update: every block's rows fit in shared memory and the blocks fill the GPU
    p.upd.fused_smem = update_fused_smem(I, h->Rmax);
    const bool fits = p.upd.fused_smem <= 160 * 1024;
    if (h->opt.update_mode == 1)
      p.upd.fused = fits ? 1 : 0;
    else if (h->opt.update_mode == 2)
      p.upd.fused = 0;
    else   // one CTA per block unless few blocks each carry much FP64 work (large I R^2)
      p.upd.fused = (fits && (h->K >= h->num_sms / 2 || I * h->Rmax * h->Rmax <= 16384)) ? 1 : 0;
  }
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Tensor-core plan of every mode: N tile, split-K factor, pipeline depths.
// dynamic shared memory per CTA (opt-in limit 227 KB, less 512 bytes for the
// arguments that a grouped launch keeps in static shared memory)
constexpr size_t kSmemOptin = 227 * 1024 - 512;

jkcals_status make_tc_plan(jkcals_ctx* h) {
  const int prec = h->opt.precision;
  const bool exact = prec == JKCALS_EXACT_BF16;
  const int nsplit = tc::form_nsplit(prec), bk = tc::form_bk(prec), chunk = tc::form_chunk(prec);
  const int row = tc::form_row_bytes(prec);
  const int bn_max = (nsplit >= 3) ? 160 : 256;
  for (int n = 0; n < h->N; ++n) {
    tc::TcPlan& p = h->tcplan[n];
    const int64_t I = h->dims[n];
    p.nsplit = nsplit;
    p.row_bytes = row;
    // fastest column mode: the smallest other mode, so that its factor rows for
    // one 128-column tile can sit in shared memory
    p.a_mode = -1;
    for (int k = 0; k < h->N; ++k)
      if (k != n && (p.a_mode < 0 || h->dims[k] < h->dims[p.a_mode])) p.a_mode = k;
    p.Ia_pad = (int)round_up(h->dims[p.a_mode], chunk);
    p.Jp = (int64_t)p.Ia_pad * (h->J[n] / h->dims[p.a_mode]);
    if (p.Jp > 2147483647LL - 4096)   // the kernel indexes columns in 32 bits
      return fail(JKCALS_ERR_UNSUPPORTED, "tensor-core forms need prod of the other dims < 2^31");
    // N tile: one tile of a multiple of 32 rows when I_n <= 128 for the split
    // forms (their part products then stack along N into few, wide MMAs),
    // otherwise balanced tiles of at most bn_max rows
    if (nsplit > 1 && I <= 128) {
      p.BN = (int)round_up(I, 32);
    } else {
      const int64_t nt = (I + bn_max - 1) / bn_max;
      p.BN = (int)round_up((I + nt - 1) / nt, 16);
    }
    p.tiles_c = (h->C + 127) / 128;
    p.tiles_n = (int)((I + p.BN - 1) / p.BN);
    if (tc::build_mma_list(prec, p) != JKCALS_OK) return fail(JKCALS_ERR_UNSUPPORTED, "accumulators exceed TMEM");
    p.tts = 0;
    p.nkt_a = p.n_o = p.o_per_cta = 0;
    p.nbuf = 1;
    p.nis = 1;
    if (exact && I <= 128) {
      // Two-step form: a narrow mode would reuse each Khatri-Rao entry only BN
      // times; with the largest other mode as a (long exact chains per o) the
      // tensor cores take U_a^T directly and the drain applies Q(c, o).  N
      // tiles of at most 64 rows (two accumulator sets fit TMEM).
      int amax = -1;
      for (int k = 0; k < h->N; ++k)
        if (k != n && (amax < 0 || h->dims[k] > h->dims[amax])) amax = k;
      const int64_t iap = round_up(h->dims[amax], bk);
      if (h->dims[amax] >= 128 && iap <= tc::kExactChainMax) {
        if (p.BN > 64) {
          p.BN = 64;
          p.tiles_n = (int)((I + p.BN - 1) / p.BN);
          if (tc::build_mma_list(prec, p) != JKCALS_OK) return fail(JKCALS_ERR_UNSUPPORTED, "accumulators exceed TMEM");
        }
        p.tts = 1;
        p.a_mode = amax;
        p.Ia_pad = (int)iap;
        p.n_o = (int)(h->J[n] / h->dims[amax]);
        p.nkt_a = (int)(iap / bk);
        p.Jp = iap * p.n_o;
        p.nbuf = 2 * p.tmem_cols <= 512 ? 2 : 1;
        p.tmem_cols *= p.nbuf;
        p.ua_smem = 0;
        p.ua_parts = 0;
        p.ua_stride = 0;
        p.stages = 2;
        if (tc::tc_smem_bytes(p) > kSmemOptin) return fail(JKCALS_ERR_UNSUPPORTED, "two-step tile does not fit");
        while (p.stages < 4) {
          ++p.stages;
          if (tc::tc_smem_bytes(p) > kSmemOptin) {
            --p.stages;
            break;
          }
        }
        // MMA issuers: one (the ring of 48 KB stages is too shallow to split)
        p.nis = 1;
        p.nkt = (int64_t)p.n_o * p.nkt_a;
        const int64_t base = (int64_t)p.tiles_c * p.tiles_n;
        const int64_t want = h->opt.splits > 0 ? h->opt.splits : std::max<int64_t>(1, h->num_sms / base);
        p.o_per_cta = (int)((p.n_o + want - 1) / want);
        p.splits = (p.n_o + p.o_per_cta - 1) / p.o_per_cta;
        p.kchunk = (int64_t)p.o_per_cta * iap;
        if (p.splits > 65535) return fail(JKCALS_ERR_UNSUPPORTED, "grid too large");
        continue;
      }
    }
    // Shared memory: the mode-a factor rows of the CTA's 128 columns (FP32 hi,
    // BF16 lo) staged once when they fit beside two pipeline stages; then as
    // many stages as fit, up to 4.
    p.ua_parts = exact ? 2 : 1;
    p.ua_stride = p.Ia_pad + 4;   // 16-byte skew between FP32 rows: fewer bank conflicts
    p.stages = 2;
    p.ua_smem = 1;
    if (tc::tc_smem_bytes(p) > kSmemOptin) p.ua_smem = 0;
    if (tc::tc_smem_bytes(p) > kSmemOptin)
      return fail(JKCALS_ERR_UNSUPPORTED, "tensor-core tile does not fit shared memory");
    while (p.stages < 4) {
      ++p.stages;
      if (tc::tc_smem_bytes(p) > kSmemOptin) {
        --p.stages;
        break;
      }
    }
    const int64_t base = (int64_t)p.tiles_c * p.tiles_n;
    const int64_t ksteps = (p.Jp + bk - 1) / bk;
    int64_t S = h->opt.splits > 0 ? h->opt.splits : std::max<int64_t>(1, h->num_sms / base);
    if (h->opt.splits <= 0) S = std::min<int64_t>(S, std::max<int64_t>(1, ksteps / 4));
    S = std::max<int64_t>(1, std::min<int64_t>(S, ksteps));
    int64_t kchunk = ((ksteps + S - 1) / S) * bk;
    if (exact && h->opt.splits <= 0) {
      // Exact chains stop every kExactChainMax columns.  Either each CTA runs
      // one chain (many CTAs, several waves) or its chain in segments drained
      // from TMEM in between (one wave, a drain per segment).  Estimated cost in
      // k-steps per SM: waves x (k-steps + 3 per drain + 6 per CTA), the loop
      // about 10% slower with segments.
      const int64_t segk = tc::kExactChainMax / bk;
      auto cost = [&](int64_t kc) {
        const int64_t ks = kc / bk, nspl = (ksteps + ks - 1) / ks;
        const int64_t waves = (base * nspl + h->num_sms - 1) / h->num_sms;
        const int64_t nseg = (ks + segk - 1) / segk;
        return (double)waves * (ks * (nseg > 1 ? 1.1 : 1.0) + 3.0 * (nseg - 1) + 6.0);
      };
      const int64_t capped = std::min<int64_t>(kchunk, tc::kExactChainMax);
      if (cost(capped) <= cost(kchunk)) kchunk = capped;
    }
    p.kchunk = kchunk;
    p.splits = (int)((p.Jp + p.kchunk - 1) / p.kchunk);
    p.nkt = ksteps;
    if (p.tiles_n > 65535 || p.splits > 65535) return fail(JKCALS_ERR_UNSUPPORTED, "grid too large");
  }
  return JKCALS_OK;
}

jkcals_status ensure_loss_cap(jkcals_ctx* h, int need) {
  if (need <= h->loss_cap) return JKCALS_OK;
  if (h->loss_hist) dfree(h, h->loss_hist);
  h->loss_hist = nullptr;
  h->loss_cap = 0;
  int cap = std::max(need, 64);
  JK_TRY(dalloc_t(h, &h->loss_hist, (size_t)cap * h->K));
  h->loss_cap = cap;
  if (h->sweep_exec) {
    cudaGraphExecDestroy(h->sweep_exec);
    h->sweep_exec = nullptr;
  }
  h->graph_valid = false;
  return JKCALS_OK;
}

UpdateArgs update_args(jkcals_ctx* h, int n, const void* part, int part_kind, int S) {
  UpdateArgs a{};
  a.N = h->N;
  a.n = n;
  a.n_hat = h->n_hat;
  a.K = h->K;
  a.C = h->C;
  a.I = h->dims[n];
  a.bm = block_meta(h);
  a.U = h->U[n];
  for (int k = 0; k < h->N; ++k) a.gram[k] = h->gram[k];
  a.gram_n = h->gram[n];
  a.part = part;
  a.part_kind = part_kind;
  a.S = S;
  a.rows_per_chunk = h->plan[n].upd.rows_per_chunk;
  a.RC = h->plan[n].upd.RC;
  a.gpart = h->gpart;
  a.fpart = h->fpart;
  a.status = h->d_status;
  a.normalise = h->opt.normalise;
  a.normT2 = h->d_normT2;
  a.loss_prev = h->d_loss_prev;
  a.loss_last = h->d_loss_last;
  a.tol = h->d_tol;
  a.loss_hist = h->loss_hist;
  a.loss_cap = h->loss_cap;
  a.sweep_idx = h->d_sweep_idx;
  a.UT = h->tc ? h->UT[n] : nullptr;
  a.I_pad = h->Ipad[n];
  a.cmax = h->tc ? h->cmax[n] : nullptr;
  a.UT_lo = h->tc ? h->UTlo[n] : nullptr;
  return a;
}

tc::TcArgs make_tc_args(jkcals_ctx* h, int n, float* const* UT, float* const* UTlo, float* const* cmax,
                        bool reuse_slices);

// Enqueue the concurrent MTTKRP of mode n for factor set (U, UT, cmax) into h->part.
// reuse_slices: a two-step mode may reuse the U_a slices left in At by the
// previous two-step launch of the same sweep when mode a was not updated since.
jkcals_status enqueue_mttkrp(jkcals_ctx* h, int n, double* const* U, float* const* UT, float* const* UTlo,
                             float* const* cmax, bool reuse_slices = false) {
  if (!h->tc) {
    const ModePlan& p = h->plan[n];
    KrpOperands kr = krp_operands(h, n, U);
    JK_CUDA(h, launch_mttkrp_f64(h->Tn64[n], h->dims[n], h->J[n], h->C, kr, p.splits, p.kchunk,
                                 static_cast<double*>(h->part), h->stream));
    return JKCALS_OK;
  }
  const tc::TcArgs a = make_tc_args(h, n, UT, UTlo, cmax, reuse_slices);
  JK_CUDA(h, tc::launch_mttkrp_tc(h->opt.precision, h->tcplan[n], a, h->stream));
  return JKCALS_OK;
}

// Arguments of mode n's tensor-core MTTKRP for factor copies (UT, UTlo, cmax).
tc::TcArgs make_tc_args(jkcals_ctx* h, int n, float* const* UT, float* const* UTlo, float* const* cmax,
                        bool reuse_slices) {
  const tc::TcPlan& p = h->tcplan[n];
  tc::TcArgs a{};
  a.I = h->dims[n];
  a.Jp = p.Jp;
  a.kchunk = p.kchunk;
  a.C = h->C;
  a.BN = p.BN;
  a.tmem_cols = p.tmem_cols;
  a.nlev = p.nlev;
  a.lstride = p.lstride;
  a.merged = p.merged;
  a.stack = p.stack;
  a.nkt = p.nkt;
  a.Tt = static_cast<const unsigned char*>(h->Tt[n]);
  a.stages = p.stages;
  a.Ia_pad = p.Ia_pad;
  a.UTa = UT[p.a_mode];
  a.UTa_lo = UTlo[p.a_mode];
  a.cmax_a = cmax[p.a_mode];
  int t = 0;
  for (int k = 0; k < h->N; ++k) {
    if (k == n || k == p.a_mode) continue;
    a.qdims[t] = (int)h->dims[k];
    a.qpad[t] = (int)h->Ipad[k];
    a.UTq[t] = UT[k];
    a.UTq_lo[t] = UTlo[k];
    a.cmax_q[t] = cmax[k];
    ++t;
  }
  a.nq = t;
  a.part = static_cast<float*>(h->part);
  a.err = h->d_err;
  a.rowexp = h->rowexp[n];
  a.ua_smem = p.ua_smem;
  a.ua_stride = p.ua_stride;
  a.At = static_cast<const unsigned char*>(h->At);
  a.nkt_a = p.nkt_a;
  a.n_o = p.n_o;
  a.o_per_cta = p.o_per_cta;
  a.nbuf = p.nbuf;
  a.nis = p.nis > 0 ? p.nis : 1;
  a.Ia = (int)h->dims[p.a_mode];
  a.ut_stride_a = h->Ipad[p.a_mode];
  a.skip_slice = (p.tts && reuse_slices) ? 1 : 0;
  a.tiles_c = p.tiles_c;
  a.tiles_n = p.tiles_n;
  return a;
}

int mode_splits(const jkcals_ctx* h, int n) { return h->tc ? h->tcplan[n].splits : h->plan[n].splits; }

int part_kind(const jkcals_ctx* h) {
  if (!h->tc) return kPartF64;
  return h->opt.precision == JKCALS_EXACT_BF16 ? kPartF32x2 : kPartF32;
}

jkcals_status reduce_into(jkcals_ctx* h, int n, double* out) {
  const int64_t cnt = h->dims[n] * (int64_t)h->C;
  if (part_kind(h) == kPartF32x2)
    JK_CUDA(h, launch_reduce_partials_f32x2(static_cast<float2*>(h->part), mode_splits(h, n), cnt, out, h->stream));
  else if (part_kind(h) == kPartF32)
    JK_CUDA(h, launch_reduce_partials_f32(static_cast<float*>(h->part), mode_splits(h, n), cnt, out, h->stream));
  else
    JK_CUDA(h, launch_reduce_partials_f64(static_cast<double*>(h->part), mode_splits(h, n), cnt, out, h->stream));
  return JKCALS_OK;
}

// Kernels one sweep launches (enqueue_sweep's launches, counted without
// launching): per mode the MTTKRP, the slicing of a two-step mode whose slices
// are stale, and the fused update (or the reduction and the two-phase update's
// three kernels); then the sweep counter.
int count_sweep_kernels(const jkcals_ctx* h) {
  int kernels = 0;
  int sliced = -1;
  for (int n = 0; n < h->N; ++n) {
    const bool tts = h->tc && h->tcplan[n].tts;
    if (tts) {
      kernels += sliced == h->tcplan[n].a_mode ? 0 : 1;
      sliced = h->tcplan[n].a_mode;
    }
    kernels += h->plan[n].upd.fused ? 2 : 4;
    if (n == sliced) sliced = -1;
  }
  return kernels + 1;
}

jkcals_status enqueue_sweep(jkcals_ctx* h) {
  int kernels = 0;
  int sliced = -1;   // mode whose current slices At holds (two-step modes)
  for (int n = 0; n < h->N; ++n) {
    const bool tts = h->tc && h->tcplan[n].tts;
    const bool reuse = tts && sliced == h->tcplan[n].a_mode;
    if (h->opt.kernel_timing) JK_CUDA(h, cudaEventRecordWithFlags(h->ev_start[n], h->stream, cudaEventRecordExternal));
    JK_TRY(enqueue_mttkrp(h, n, h->U, h->UT, h->UTlo, h->cmax, reuse));
    if (tts) {
      sliced = h->tcplan[n].a_mode;
      kernels += reuse ? 0 : 1;
    }
    if (h->opt.kernel_timing) JK_CUDA(h, cudaEventRecordWithFlags(h->ev_stop[n], h->stream, cudaEventRecordExternal));
    if (h->plan[n].upd.fused) {
      // the fused update sums each block's split-K partials itself (fixed order)
      UpdateArgs a = update_args(h, n, h->part, part_kind(h), mode_splits(h, n));
      JK_CUDA(h, launch_update_fused(a, h->plan[n].upd.fused_smem, h->Rmax, h->uniform_rank, h->stream));
      kernels += 2;
    } else {
      // fixed-order split-K reduction into FP64 Mbar_n, then the two-phase update
      JK_TRY(reduce_into(h, n, h->mbuf));
      UpdateArgs a = update_args(h, n, h->mbuf, kPartF64, 1);
      JK_CUDA(h, launch_update(a, h->stream));
      kernels += 4;
    }
    if (n == sliced) sliced = -1;   // U_a changed: the slices in At are stale
  }
  JK_CUDA(h, launch_advance_sweep(h->d_sweep_idx, h->stream));
  h->kernels_per_sweep = kernels + 1;   // = count_sweep_kernels(h)
  return JKCALS_OK;
}

jkcals_status build_graph(jkcals_ctx* h) {
  if (h->graph_valid) return JKCALS_OK;
  if (h->sweep_exec) {
    cudaGraphExecDestroy(h->sweep_exec);
    h->sweep_exec = nullptr;
  }
  JK_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  jkcals_status s = enqueue_sweep(h);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
  if (s != JKCALS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return fail_cuda(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->sweep_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail_cuda(h, e, "cudaGraphInstantiate");
  h->graph_valid = true;
  return JKCALS_OK;
}

jkcals_status run_sweeps(jkcals_ctx* h, int nsweeps) {
  if (h->opt.use_graph) {
    JK_TRY(build_graph(h));
    for (int s = 0; s < nsweeps; ++s) JK_CUDA(h, cudaGraphLaunch(h->sweep_exec, h->stream));
  } else {
    for (int s = 0; s < nsweeps; ++s) JK_TRY(enqueue_sweep(h));
  }
  return JKCALS_OK;
}

jkcals_status refresh_factor_state(jkcals_ctx* h) {
  BlockMeta bm = block_meta(h);
  JK_CUDA(h, launch_zero_left_out(h->U[h->n_hat], h->C, h->K, bm, h->stream));
  for (int n = 0; n < h->N; ++n)
    JK_CUDA(h, launch_grams(h->U[n], h->dims[n], h->C, h->K, bm, h->gram[n], h->stream));
  if (h->tc)
    for (int n = 0; n < h->N; ++n) {
      JK_CUDA(h, tc::launch_factor_to_ut(h->U[n], h->dims[n], h->C, h->UT[n], h->UTlo[n], h->Ipad[n], h->stream));
      JK_CUDA(h, tc::launch_colmax(h->UT[n], h->dims[n], h->Ipad[n], h->C, h->cmax[n], h->stream));
    }
  JK_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(int32_t) * h->K, h->stream));
  JK_CUDA(h, cudaMemsetAsync(h->d_loss_prev, 0xff, sizeof(double) * h->K, h->stream));
  JK_CUDA(h, cudaMemsetAsync(h->d_loss_last, 0xff, sizeof(double) * h->K, h->stream));
  return JKCALS_OK;
}

jkcals_status copy_out(jkcals_ctx* h, void* dst, const void* src, size_t bytes) {
  JK_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
  if (is_host_pointer(dst)) JK_CUDA(h, cudaStreamSynchronize(h->stream));
  return JKCALS_OK;
}

// Reads the tensor-core kernel's error word (set when a bounded wait expired).
jkcals_status check_device_error(jkcals_ctx* h) {
  if (!h->tc || h->d_err == nullptr) return JKCALS_OK;
  int err = 0;
  JK_CUDA(h, cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (err != 0) {
    JK_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
    return fail(JKCALS_ERR_TIMEOUT, "a bounded wait in the tensor-core MTTKRP expired (code " +
                                        std::to_string(err) + "); results of that call are invalid");
  }
  return JKCALS_OK;
}

// Set the split-K factor of mode n's MTTKRP to about S (clamped to the
// column count).
void set_mode_splits(jkcals_ctx* h, int n, int64_t S) {
  if (h->tc && h->tcplan[n].tts) {
    // two-step form: whole o values per split
    tc::TcPlan& p = h->tcplan[n];
    S = std::max<int64_t>(1, std::min<int64_t>(S, p.n_o));
    p.o_per_cta = (int)((p.n_o + S - 1) / S);
    p.splits = (p.n_o + p.o_per_cta - 1) / p.o_per_cta;
    p.kchunk = (int64_t)p.o_per_cta * p.Ia_pad;
  } else if (h->tc) {
    tc::TcPlan& p = h->tcplan[n];
    const int64_t bk = tc::form_bk(h->opt.precision);
    S = std::max<int64_t>(1, std::min<int64_t>(S, p.nkt));
    int64_t kchunk = ((p.nkt + S - 1) / S) * bk;
    p.kchunk = kchunk;
    p.splits = (int)((p.Jp + kchunk - 1) / kchunk);
  } else {
    ModePlan& p = h->plan[n];
    const int64_t ksteps = (h->J[n] + kMttkrpBK - 1) / kMttkrpBK;
    S = std::max<int64_t>(1, std::min<int64_t>(S, ksteps));
    const int64_t kchunk = ((ksteps + S - 1) / S) * kMttkrpBK;
    p.kchunk = kchunk;
    p.splits = (int)((h->J[n] + kchunk - 1) / kchunk);
  }
  h->graph_valid = false;
}

int64_t mode_kchunk(const jkcals_ctx* h, int n) { return h->tc ? h->tcplan[n].kchunk : h->plan[n].kchunk; }

// Autotuner: per mode, time the MTTKRP + split-K reduction on the handle's
// current factors for split factors {S, S/2, 2S, 4S} around the planned S
// (three timed runs after one warm-up each, CUDA events on the handle's
// stream) and keep the fastest.  The partial-sum workspace grows as needed.
jkcals_status autotune_splits(jkcals_ctx* h) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  JK_CUDA(h, cudaEventCreate(&e0));
  JK_CUDA(h, cudaEventCreate(&e1));
  const size_t eb = part_kind(h) == kPartF32 ? sizeof(float) : sizeof(double);
  jkcals_status st = JKCALS_OK;
  for (int n = 0; n < h->N && st == JKCALS_OK; ++n) {
    const int64_t S0 = mode_splits(h, n);
    const int64_t cands[4] = {S0, std::max<int64_t>(1, S0 / 2), 2 * S0, 4 * S0};
    int64_t best_S = S0, tried[4] = {0, 0, 0, 0};
    float best_ms = 1e30f;
    for (int c = 0; c < 4 && st == JKCALS_OK; ++c) {
      set_mode_splits(h, n, cands[c]);
      const int64_t kc = mode_kchunk(h, n);
      bool seen = false;
      for (int d = 0; d < c; ++d) seen = seen || tried[d] == kc;
      tried[c] = kc;
      if (seen) continue;
      const size_t need = (size_t)mode_splits(h, n) * h->dims[n] * h->C * eb;
      if (need > h->part_bytes) {
        JK_CUDA(h, cudaStreamSynchronize(h->stream));
        dfree(h, h->part);
        h->part = nullptr;
        h->part_bytes = 0;
        if ((st = dalloc(h, &h->part, need)) != JKCALS_OK) break;
        h->part_bytes = need;
      }
      for (int rep = 0; rep < 4 && st == JKCALS_OK; ++rep) {
        if (rep == 1) JK_CUDA(h, cudaEventRecord(e0, h->stream));
        if ((st = enqueue_mttkrp(h, n, h->U, h->UT, h->UTlo, h->cmax)) != JKCALS_OK) break;
        st = reduce_into(h, n, h->mbuf);
      }
      if (st != JKCALS_OK) break;
      JK_CUDA(h, cudaEventRecord(e1, h->stream));
      JK_CUDA(h, cudaEventSynchronize(e1));
      float ms = 0.f;
      JK_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best_S = cands[c];
      }
    }
    set_mode_splits(h, n, best_S);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != JKCALS_OK) return st;
  return check_device_error(h);
}

jkcals_status check_handle(jkcals_t h) {
  if (h == nullptr) return fail(JKCALS_ERR_ARG, "NULL handle");
  if (h->broken) return fail(JKCALS_ERR_STATE, "handle unusable after an earlier CUDA error");
  JK_CUDA(h, cudaSetDevice(h->device));
  return JKCALS_OK;
}

void destroy_impl(jkcals_ctx* h) {
  if (h == nullptr) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->sweep_exec) cudaGraphExecDestroy(h->sweep_exec);
  for (int n = 0; n < kMaxModes; ++n) {
    if (h->ev_start[n]) cudaEventDestroy(h->ev_start[n]);
    if (h->ev_stop[n]) cudaEventDestroy(h->ev_stop[n]);
  }
  // the handle's stream is idle (synchronised above) and no batch uses the handle any more
  for (void* p : h->allocations) {
    if (h->pool)
      cudaFreeAsync(p, h->stream);
    else
      cudaFree(p);
  }
  h->allocations.clear();
  if (h->pool && h->stream) cudaStreamSynchronize(h->stream);
  if (h->stream && h->owns_stream) cudaStreamDestroy(h->stream);
  cudaSetDevice(cur);
  delete h;
}

}  // namespace

namespace {

jkcals_status create_impl(jkcals_ctx* h, const void* T, int T_dtype, const int32_t* ranks,
                          const int64_t* left_out_ptr, const int64_t* left_out_idx,
                          const double* const* init) {
  const int N = h->N, K = h->K;
  int64_t total = 1;
  for (int k = 0; k < N; ++k) total *= h->dims[k];
  for (int k = 0; k < N; ++k) h->J[k] = total / h->dims[k];

  // block metadata
  h->R.assign(ranks, ranks + K);
  h->off.resize(K);
  h->gram_off.resize(K);
  int c = 0, go = 0;
  for (int g = 0; g < K; ++g) {
    h->off[g] = c;
    h->gram_off[g] = go;
    c += h->R[g];
    go += h->R[g] * h->R[g];
    h->Rmax = std::max(h->Rmax, h->R[g]);
  }
  h->C = c;
  h->gram_total = go;
  for (int g = 0; g < K; ++g) h->uniform_rank = h->uniform_rank && (h->R[g] == h->Rmax);
  h->lo_ptr.assign(left_out_ptr, left_out_ptr + K + 1);
  h->lo_idx.assign(left_out_idx, left_out_idx + left_out_ptr[K]);
  for (int g = 0; g < K; ++g) std::sort(h->lo_idx.begin() + h->lo_ptr[g], h->lo_idx.begin() + h->lo_ptr[g + 1]);

  JK_TRY(dalloc_t(h, &h->d_R, K));
  JK_TRY(dalloc_t(h, &h->d_off, K));
  JK_TRY(dalloc_t(h, &h->d_gram_off, K));
  JK_TRY(dalloc_t(h, &h->d_lo_ptr, K + 1));
  JK_TRY(dalloc_t(h, &h->d_lo_idx, std::max<size_t>(1, h->lo_idx.size())));
  JK_TRY(dalloc_t(h, &h->d_status, K));
  JK_TRY(dalloc_t(h, &h->d_normT2, K));
  JK_TRY(dalloc_t(h, &h->d_loss_prev, K));
  JK_TRY(dalloc_t(h, &h->d_loss_last, K));
  JK_TRY(dalloc_t(h, &h->d_tol, 1));
  JK_TRY(dalloc_t(h, &h->d_sweep_idx, 1));
  cudaStream_t st = h->stream;
  JK_CUDA(h, cudaMemcpyAsync(h->d_R, h->R.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_off, h->off.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_gram_off, h->gram_off.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_lo_ptr, h->lo_ptr.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st));
  if (!h->lo_idx.empty())
    JK_CUDA(h, cudaMemcpyAsync(h->d_lo_idx, h->lo_idx.data(), sizeof(int64_t) * h->lo_idx.size(),
                               cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemsetAsync(h->d_tol, 0, sizeof(double), st));
  JK_CUDA(h, cudaMemsetAsync(h->d_sweep_idx, 0, sizeof(int), st));
  // host-side vectors above are pageable: make sure the copies finished
  JK_CUDA(h, cudaStreamSynchronize(st));

  // tensor -> per-mode unfoldings (FP64)
  double* Tc = nullptr;
  JK_TRY(dalloc_t(h, &Tc, total));
  if (T_dtype == JKCALS_DTYPE_F64) {
    JK_CUDA(h, cudaMemcpyAsync(Tc, T, sizeof(double) * total, cudaMemcpyDefault, st));
  } else {
    float* T32 = nullptr;
    JK_TRY(dalloc_t(h, &T32, total));
    JK_CUDA(h, cudaMemcpyAsync(T32, T, sizeof(float) * total, cudaMemcpyDefault, st));
    JK_CUDA(h, launch_f32_to_f64(T32, Tc, total, st));
    JK_CUDA(h, cudaStreamSynchronize(st));
    dfree(h, T32, true);
  }
  for (int n = 0; n < N; ++n) {
    JK_TRY(dalloc_t(h, &h->Tn64[n], total));
    JK_CUDA(h, launch_unfold_f64(Tc, h->dims, N, n, h->Tn64[n], st));
  }
  double* slice = nullptr;
  JK_TRY(dalloc_t(h, &slice, h->dims[h->n_hat]));
  JK_CUDA(h, launch_row_sumsq(h->Tn64[h->n_hat], h->dims[h->n_hat], h->J[h->n_hat], slice, st));
  JK_CUDA(h, launch_block_norms(slice, h->dims[h->n_hat], K, block_meta(h), h->d_normT2, st));
  JK_CUDA(h, cudaStreamSynchronize(st));
  dfree(h, slice, true);
  dfree(h, Tc, true);

  // tensor-core forms: padded, precision-split, pre-tiled unfoldings replace the FP64 ones
  if (h->tc) {
    JK_TRY(make_tc_plan(h));
    const int chunk = tc::form_chunk(h->opt.precision);
    size_t at_bytes = 0;
    for (int n = 0; n < N; ++n) at_bytes = std::max(at_bytes, tc::tts_a_bytes(h->tcplan[n]));
    if (at_bytes > 0) JK_TRY(dalloc(h, &h->At, at_bytes));
    for (int n = 0; n < N; ++n) {
      const tc::TcPlan& p = h->tcplan[n];
      JK_TRY(dalloc(h, &h->Tt[n], (size_t)p.tiles_n * p.nkt * p.nsplit * p.BN * p.row_bytes));
      JK_TRY(dalloc_t(h, &h->rowexp[n], (size_t)h->dims[n]));
      JK_CUDA(h, tc::launch_row_exponent(h->Tn64[n], h->dims[n], h->J[n], h->rowexp[n], st));
      tc::UnfoldMap mp{};
      {
        int64_t stride = 1;
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          if (k == p.a_mode) {
            mp.sa = stride;
          } else {
            mp.qd[mp.nq] = h->dims[k];
            mp.qs[mp.nq] = stride;
            ++mp.nq;
          }
          stride *= h->dims[k];
        }
      }
      JK_CUDA(h, tc::launch_tile_unfold(h->opt.precision, h->Tn64[n], h->dims[n], h->J[n], h->dims[p.a_mode],
                                        p.Ia_pad, p.Jp, mp, h->rowexp[n], p.BN, p.tiles_n, p.nkt, h->Tt[n], st));
      h->Ipad[n] = round_up(h->dims[n], chunk);
    }
    JK_CUDA(h, cudaStreamSynchronize(st));
    for (int n = 0; n < N; ++n) {
      dfree(h, h->Tn64[n], true);
      h->Tn64[n] = nullptr;
      JK_TRY(dalloc_t(h, &h->UT[n], (size_t)h->C * h->Ipad[n]));
      JK_CUDA(h, cudaMemsetAsync(h->UT[n], 0, sizeof(float) * h->C * h->Ipad[n], st));
      JK_TRY(dalloc_t(h, &h->cmax[n], (size_t)h->C));
      if (h->opt.precision == JKCALS_EXACT_BF16) {
        JK_TRY(dalloc_t(h, &h->UTlo[n], (size_t)h->C * h->Ipad[n]));
        JK_CUDA(h, cudaMemsetAsync(h->UTlo[n], 0, sizeof(float) * h->C * h->Ipad[n], st));
      }
    }
    size_t smem = 0;
    for (int n = 0; n < N; ++n) smem = std::max(smem, tc::tc_smem_bytes(h->tcplan[n]));
    JK_CUDA(h, tc::prepare_mttkrp_tc(h->opt.precision, smem));
    JK_TRY(dalloc_t(h, &h->d_err, 1));
    JK_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), st));
  }

  // factors and Grams
  int64_t Imax = 0;
  for (int n = 0; n < N; ++n) {
    JK_TRY(dalloc_t(h, &h->U[n], (size_t)h->dims[n] * h->C));
    JK_TRY(dalloc_t(h, &h->gram[n], (size_t)h->gram_total));
    JK_CUDA(h, cudaMemcpyAsync(h->U[n], init[n], sizeof(double) * h->dims[n] * h->C, cudaMemcpyDefault, st));
    Imax = std::max(Imax, h->dims[n]);
  }

  // plan + workspace
  make_plan(h);
  size_t part_bytes = 0, chunks = 0;
  for (int n = 0; n < N; ++n) {
    const size_t eb = part_kind(h) == kPartF32 ? sizeof(float) : sizeof(double);
    const size_t pb = (size_t)mode_splits(h, n) * h->dims[n] * h->C * eb;
    part_bytes = std::max(part_bytes, pb);
    chunks = std::max(chunks, (size_t)h->plan[n].upd.RC * K);
  }
  // room for the two-phase update of any subset of the blocks (compaction):
  // RC is at most ceil(2 SMs / K') for K' blocks, so RC K' < 2 SMs + K'
  chunks = std::max(chunks, (size_t)(2 * h->num_sms + K));
  size_t part_elems = part_bytes / sizeof(double) + 1;
  h->part_bytes = part_elems * sizeof(double);
  JK_TRY(dalloc(h, &h->part, h->part_bytes));
  JK_TRY(dalloc_t(h, &h->gpart, chunks * kMaxRank * kMaxRank));
  JK_TRY(dalloc_t(h, &h->fpart, chunks));
  h->upd_chunks = chunks;
  JK_TRY(dalloc_t(h, &h->mbuf, (size_t)Imax * h->C));
  JK_TRY(ensure_loss_cap(h, 64));
  if (h->opt.kernel_timing) {
    for (int n = 0; n < N; ++n) {
      JK_CUDA(h, cudaEventCreate(&h->ev_start[n]));
      JK_CUDA(h, cudaEventCreate(&h->ev_stop[n]));
    }
  }
  size_t fsmem = 0;
  for (int n = 0; n < N; ++n)
    if (h->plan[n].upd.fused) fsmem = std::max(fsmem, h->plan[n].upd.fused_smem);
  if (fsmem > 0) JK_CUDA(h, prepare_update_fused(fsmem, h->Rmax, h->uniform_rank));
  h->kernels_per_sweep = count_sweep_kernels(h);
  JK_TRY(refresh_factor_state(h));
  if (h->opt.autotune && h->opt.splits <= 0) JK_TRY(autotune_splits(h));
  JK_CUDA(h, cudaStreamSynchronize(st));
  return JKCALS_OK;
}

jkcals_status grad_impl(jkcals_ctx* h, const double* const* U, double* const* G, double* loss) {
  const int N = h->N;
  cudaStream_t st = h->stream;
  if (!h->grad_ready) {
    for (int n = 0; n < N; ++n) {
      JK_TRY(dalloc_t(h, &h->gU[n], (size_t)h->dims[n] * h->C));
      JK_TRY(dalloc_t(h, &h->ggram[n], (size_t)h->gram_total));
      JK_TRY(dalloc_t(h, &h->gG[n], (size_t)h->dims[n] * h->C));
    }
    JK_TRY(dalloc_t(h, &h->geg, (size_t)h->K + 1));
    if (h->tc) {
      for (int n = 0; n < N; ++n) {
        JK_TRY(dalloc_t(h, &h->gUT[n], (size_t)h->C * h->Ipad[n]));
        JK_CUDA(h, cudaMemsetAsync(h->gUT[n], 0, sizeof(float) * h->C * h->Ipad[n], st));
        JK_TRY(dalloc_t(h, &h->gcmax[n], (size_t)h->C));
        if (h->opt.precision == JKCALS_EXACT_BF16) {
          JK_TRY(dalloc_t(h, &h->gUTlo[n], (size_t)h->C * h->Ipad[n]));
          JK_CUDA(h, cudaMemsetAsync(h->gUTlo[n], 0, sizeof(float) * h->C * h->Ipad[n], st));
        }
      }
    }
    h->grad_ready = true;
  }
  BlockMeta bm = block_meta(h);
  for (int n = 0; n < N; ++n) {
    const double* src = U ? U[n] : h->U[n];
    JK_CUDA(h, cudaMemcpyAsync(h->gU[n], src, sizeof(double) * h->dims[n] * h->C, cudaMemcpyDefault, st));
  }
  JK_CUDA(h, launch_zero_left_out(h->gU[h->n_hat], h->C, h->K, bm, st));
  for (int n = 0; n < N; ++n) {
    JK_CUDA(h, launch_grams(h->gU[n], h->dims[n], h->C, h->K, bm, h->ggram[n], st));
    if (h->tc) {
      JK_CUDA(h, tc::launch_factor_to_ut(h->gU[n], h->dims[n], h->C, h->gUT[n], h->gUTlo[n], h->Ipad[n], st));
      JK_CUDA(h, tc::launch_colmax(h->gUT[n], h->dims[n], h->Ipad[n], h->C, h->gcmax[n], st));
    }
  }
  const bool want_g = G != nullptr;
  for (int n = 0; n < N; ++n) {
    // the loss needs only the last mode's MTTKRP (its inner product term)
    if (!want_g && n != N - 1) continue;
    JK_TRY(enqueue_mttkrp(h, n, h->gU, h->gUT, h->gUTlo, h->gcmax));
    const int64_t cnt = h->dims[n] * (int64_t)h->C;
    JK_TRY(reduce_into(h, n, h->mbuf));
    if (G != nullptr && G[n] != nullptr) {
      JK_CUDA(h, launch_grad_epilogue(N, n, h->n_hat, h->dims[n], h->C, h->K, bm, h->gU[n], h->ggram,
                                      h->mbuf, h->gG[n], st));
      JK_CUDA(h, cudaMemcpyAsync(G[n], h->gG[n], sizeof(double) * cnt, cudaMemcpyDefault, st));
    }
    if (n == N - 1)
      JK_CUDA(h, launch_grad_loss(N, h->dims[n], h->C, h->K, bm, h->gU[n], h->ggram, h->mbuf,
                                  h->d_normT2, h->geg, st));
  }
  if (loss != nullptr) {
    JK_CUDA(h, cudaMemcpyAsync(loss, h->geg + h->K, sizeof(double), cudaMemcpyDefault, st));
  }
  JK_CUDA(h, cudaStreamSynchronize(st));
  return check_device_error(h);
}

}  // namespace

extern "C" {

void jkcals_default_options(jkcals_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = JKCALS_FP64;
  opt->normalise = 1;
  opt->use_graph = 1;
  opt->splits = 0;
  opt->max_device_bytes = 0;
  opt->compact = 1;
}

const char* jkcals_last_error(void) { return jk::g_last_error.c_str(); }

const char* jkcals_version(void) { return "jkcals 0.1 (sm_103a)"; }

jkcals_status jkcals_create(jkcals_t* out, int N, const int64_t* dims, const void* T, int T_dtype,
                            int sampled_mode, int K, const int32_t* ranks,
                            const int64_t* left_out_ptr, const int64_t* left_out_idx,
                            const double* const* init, const jkcals_options* opt, void* stream) {
  set_error("");
  if (out == nullptr) return fail(JKCALS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (N < 2 || N > kMaxModes) return fail(N < 2 ? JKCALS_ERR_ARG : JKCALS_ERR_UNSUPPORTED, "N must be in [2, 8]");
  if (dims == nullptr || T == nullptr || ranks == nullptr || left_out_ptr == nullptr || init == nullptr)
    return fail(JKCALS_ERR_ARG, "NULL argument");
  if (T_dtype != JKCALS_DTYPE_F32 && T_dtype != JKCALS_DTYPE_F64) return fail(JKCALS_ERR_ARG, "bad T_dtype");
  double vol = 1.0;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1) return fail(JKCALS_ERR_ARG, "dims must be >= 1");
    vol *= (double)dims[k];
  }
  if (vol >= 1099511627776.0) return fail(JKCALS_ERR_UNSUPPORTED, "prod(dims) must be < 2^40");
  // grid limits: row chunks of 128 on grid.y of the update kernels
  for (int k = 0; k < N; ++k)
    if (dims[k] > 65535LL * 128) return fail(JKCALS_ERR_UNSUPPORTED, "dims must be <= 8388480");
  if (sampled_mode < 0 || sampled_mode >= N) return fail(JKCALS_ERR_ARG, "sampled_mode out of range");
  if (K < 1) return fail(JKCALS_ERR_ARG, "K must be >= 1");
  int64_t Csum = 0;
  for (int g = 0; g < K; ++g) {
    if (ranks[g] < 1) return fail(JKCALS_ERR_ARG, "ranks must be >= 1");
    if (ranks[g] > kMaxRank) return fail(JKCALS_ERR_UNSUPPORTED, "ranks must be <= 32");
    Csum += ranks[g];
  }
  // column tiles of 64 on grid.y of the MTTKRP kernel
  if (Csum > 65535LL * 64) return fail(JKCALS_ERR_UNSUPPORTED, "sum of ranks must be <= 4194240");
  if (left_out_ptr[0] != 0) return fail(JKCALS_ERR_ARG, "left_out_ptr[0] must be 0");
  for (int g = 0; g < K; ++g)
    if (left_out_ptr[g + 1] < left_out_ptr[g]) return fail(JKCALS_ERR_ARG, "left_out_ptr must be non-decreasing");
  if (left_out_ptr[K] > 0 && left_out_idx == nullptr) return fail(JKCALS_ERR_ARG, "left_out_idx is NULL");
  const int64_t Ihat = dims[sampled_mode];
  for (int g = 0; g < K; ++g) {
    std::vector<int64_t> d(left_out_idx + left_out_ptr[g], left_out_idx + left_out_ptr[g + 1]);
    std::sort(d.begin(), d.end());
    for (size_t q = 0; q < d.size(); ++q) {
      if (d[q] < 0 || d[q] >= Ihat) return fail(JKCALS_ERR_ARG, "left-out index out of range");
      if (q > 0 && d[q] == d[q - 1]) return fail(JKCALS_ERR_ARG, "duplicate left-out index");
    }
    if ((int64_t)d.size() >= Ihat) return fail(JKCALS_ERR_ARG, "a block leaves out every sample");
  }
  for (int k = 0; k < N; ++k)
    if (init[k] == nullptr) return fail(JKCALS_ERR_ARG, "init[n] is NULL");
  jkcals_options o;
  jkcals_default_options(&o);
  if (opt) o = *opt;
  if (o.precision < JKCALS_FP64 || o.precision > JKCALS_EXACT_BF16) return fail(JKCALS_ERR_ARG, "bad precision");
  if (o.splits < 0) return fail(JKCALS_ERR_ARG, "splits must be >= 0");
  if (o.update_mode < 0 || o.update_mode > 2) return fail(JKCALS_ERR_ARG, "update_mode must be 0, 1 or 2");

  jkcals_ctx* h = new jkcals_ctx();
  h->N = N;
  for (int k = 0; k < N; ++k) h->dims[k] = dims[k];
  h->n_hat = sampled_mode;
  h->K = K;
  h->opt = o;
  h->tc = (o.precision != JKCALS_FP64);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail_cuda(nullptr, e, "cudaGetDevice");
  }
  if (stream != nullptr) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    // The legacy default stream cannot be captured into a graph; use a
    // blocking stream, which synchronises with it implicitly.
    e = cudaStreamCreate(&h->stream);
    if (e != cudaSuccess) {
      delete h;
      return fail_cuda(nullptr, e, "cudaStreamCreate");
    }
    h->owns_stream = true;
  }
  h->pool = library_pool(h->device);
  jkcals_status s = create_impl(h, T, T_dtype, ranks, left_out_ptr, left_out_idx, init);
  if (s != JKCALS_OK) {
    std::string msg = g_last_error;
    destroy_impl(h);
    set_error(msg);
    return s;
  }
  *out = h;
  return JKCALS_OK;
}

void jkcals_destroy(jkcals_t h) { destroy_impl(h); }

jkcals_status jkcals_mttkrp(jkcals_t h, int mode, double* M_out) {
  JK_TRY(check_handle(h));
  if (mode < 0 || mode >= h->N) return fail(JKCALS_ERR_ARG, "mode out of range");
  if (M_out == nullptr) return fail(JKCALS_ERR_ARG, "M_out is NULL");
  JK_TRY(enqueue_mttkrp(h, mode, h->U, h->UT, h->UTlo, h->cmax));
  const int64_t cnt = h->dims[mode] * (int64_t)h->C;
  JK_TRY(reduce_into(h, mode, h->mbuf));
  JK_TRY(copy_out(h, M_out, h->mbuf, sizeof(double) * cnt));
  return check_device_error(h);
}

static jkcals_status any_not_spd(jkcals_ctx* h) {
  JK_TRY(check_device_error(h));
  std::vector<int32_t> st(h->K);
  JK_CUDA(h, cudaMemcpyAsync(st.data(), h->d_status, sizeof(int32_t) * h->K, cudaMemcpyDeviceToHost, h->stream));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int32_t v : st)
    if (v & JKCALS_BLOCK_NOT_SPD) return fail(JKCALS_ERR_NOT_SPD, "a submodel met a non-SPD Hadamard-of-Grams matrix");
  return JKCALS_OK;
}

jkcals_status jkcals_als_sweep(jkcals_t h, int nsweeps, double* losses) {
  JK_TRY(check_handle(h));
  if (nsweeps < 0) return fail(JKCALS_ERR_ARG, "nsweeps must be >= 0");
  if (nsweeps == 0) return JKCALS_OK;
  JK_TRY(ensure_loss_cap(h, nsweeps));
  h->tol_host = 0.0;
  JK_CUDA(h, cudaMemsetAsync(h->d_tol, 0, sizeof(double), h->stream));
  JK_CUDA(h, cudaMemsetAsync(h->d_sweep_idx, 0, sizeof(int), h->stream));
  JK_TRY(run_sweeps(h, nsweeps));
  if (losses != nullptr) JK_TRY(copy_out(h, losses, h->loss_hist, sizeof(double) * nsweeps * h->K));
  return any_not_spd(h);
}

jkcals_status jkcals_als_sweep_async(jkcals_t h, int nsweeps, double* losses_dev) {
  JK_TRY(check_handle(h));
  if (nsweeps < 0) return fail(JKCALS_ERR_ARG, "nsweeps must be >= 0");
  if (nsweeps == 0) return JKCALS_OK;
  if (losses_dev != nullptr && is_host_pointer(losses_dev))
    return fail(JKCALS_ERR_ARG, "losses_dev must be device memory");
  JK_TRY(ensure_loss_cap(h, nsweeps));
  JK_CUDA(h, cudaMemsetAsync(h->d_tol, 0, sizeof(double), h->stream));
  JK_CUDA(h, cudaMemsetAsync(h->d_sweep_idx, 0, sizeof(int), h->stream));
  JK_TRY(run_sweeps(h, nsweeps));
  if (losses_dev != nullptr)
    JK_CUDA(h, cudaMemcpyAsync(losses_dev, h->loss_hist, sizeof(double) * nsweeps * h->K,
                               cudaMemcpyDeviceToDevice, h->stream));
  return JKCALS_OK;
}

jkcals_status jkcals_kernel_times(jkcals_t h, double* ms) {
  JK_TRY(check_handle(h));
  if (ms == nullptr) return fail(JKCALS_ERR_ARG, "ms is NULL");
  if (!h->opt.kernel_timing) return fail(JKCALS_ERR_STATE, "kernel_timing was not enabled at create");
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int n = 0; n < h->N; ++n) {
    float t = 0.f;
    cudaError_t e = cudaEventElapsedTime(&t, h->ev_start[n], h->ev_stop[n]);
    if (e == cudaErrorInvalidResourceHandle || e == cudaErrorNotReady) {
      cudaGetLastError();
      return fail(JKCALS_ERR_STATE, "no completed sweep to time yet");
    }
    JK_CUDA(h, e);
    ms[n] = (double)t;
  }
  return JKCALS_OK;
}

jkcals_status jkcals_sweep_info(jkcals_t h, int* kernels_per_sweep, int* splits) {
  JK_TRY(check_handle(h));
  if (kernels_per_sweep == nullptr) return fail(JKCALS_ERR_ARG, "kernels_per_sweep is NULL");
  *kernels_per_sweep = h->kernels_per_sweep;
  if (splits)
    for (int n = 0; n < h->N; ++n) splits[n] = mode_splits(h, n);
  return JKCALS_OK;
}

// Mode n's plan as reported by jkcals_mode_plan / jkcals_plan_query.
static void report_plan(const jkcals_ctx* h, int n, int* kernel, int* tile_rows, int* stages, int* fastest_mode,
                        int* splits) {
  if (!h->tc) {
    *kernel = 0;
    if (tile_rows) *tile_rows = kMttkrpBM;
    if (stages) *stages = 0;
    if (fastest_mode) *fastest_mode = -1;
    if (splits) *splits = h->plan[n].splits;
    return;
  }
  const tc::TcPlan& p = h->tcplan[n];
  *kernel = p.tts ? 2 : 1;
  if (tile_rows) *tile_rows = p.BN;
  if (stages) *stages = p.stages;
  if (fastest_mode) *fastest_mode = p.a_mode;
  if (splits) *splits = p.splits;
}

jkcals_status jkcals_mode_plan(jkcals_t h, int mode, int* kernel, int* tile_rows, int* stages, int* fastest_mode) {
  JK_TRY(check_handle(h));
  if (mode < 0 || mode >= h->N) return fail(JKCALS_ERR_ARG, "mode out of range");
  if (kernel == nullptr) return fail(JKCALS_ERR_ARG, "kernel is NULL");
  report_plan(h, mode, kernel, tile_rows, stages, fastest_mode, nullptr);
  return JKCALS_OK;
}

jkcals_status jkcals_plan_query(int N, const int64_t* dims, int K, const int32_t* ranks, const jkcals_options* opt,
                                int num_sms, int* kernel, int* tile_rows, int* stages, int* splits) {
  if (dims == nullptr || ranks == nullptr || kernel == nullptr) return fail(JKCALS_ERR_ARG, "NULL argument");
  if (N < 2 || N > kMaxModes) return fail(JKCALS_ERR_ARG, "N must be in [2, 8]");
  if (K < 1) return fail(JKCALS_ERR_ARG, "K must be >= 1");
  if (num_sms < 1) return fail(JKCALS_ERR_ARG, "num_sms must be >= 1");
  jkcals_options o;
  jkcals_default_options(&o);
  if (opt) o = *opt;
  if (o.precision < JKCALS_FP64 || o.precision > JKCALS_EXACT_BF16) return fail(JKCALS_ERR_ARG, "bad precision");
  if (o.splits < 0) return fail(JKCALS_ERR_ARG, "splits must be >= 0");
  jkcals_ctx c;
  c.N = N;
  c.K = K;
  c.opt = o;
  c.tc = (o.precision != JKCALS_FP64);
  c.num_sms = num_sms;
  int64_t total = 1;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1) return fail(JKCALS_ERR_ARG, "dims must be >= 1");
    c.dims[k] = dims[k];
    total *= dims[k];
  }
  for (int k = 0; k < N; ++k) c.J[k] = total / dims[k];
  int64_t C = 0;
  for (int g = 0; g < K; ++g) {
    if (ranks[g] < 1) return fail(JKCALS_ERR_ARG, "ranks must be >= 1");
    if (ranks[g] > kMaxRank) return fail(JKCALS_ERR_UNSUPPORTED, "ranks must be <= 32");
    c.Rmax = std::max(c.Rmax, (int)ranks[g]);
    C += ranks[g];
  }
  if (C > 2147483647LL) return fail(JKCALS_ERR_UNSUPPORTED, "too many columns");
  c.C = (int)C;
  make_plan(&c);
  if (c.tc) JK_TRY(make_tc_plan(&c));
  for (int n = 0; n < N; ++n)
    report_plan(&c, n, &kernel[n], tile_rows ? &tile_rows[n] : nullptr, stages ? &stages[n] : nullptr, nullptr,
                splits ? &splits[n] : nullptr);
  return JKCALS_OK;
}

jkcals_status jkcals_jackknife_se(jkcals_t h, int ref_block, const double* const* ref, double* const* S,
                                  int32_t* perm, double* const* aligned, int* n_submodels) {
  JK_TRY(check_handle(h));
  const int N = h->N;
  if (S == nullptr) return fail(JKCALS_ERR_ARG, "S is NULL");
  for (int n = 0; n < N; ++n)
    if (n != h->n_hat && S[n] == nullptr) return fail(JKCALS_ERR_ARG, "S[n] is NULL for a mode other than sampled_mode");
  std::vector<int64_t> col_off;
  for (int g = 0; g < h->K; ++g)
    if (h->lo_ptr[g + 1] > h->lo_ptr[g]) col_off.push_back(h->off[g]);
  const int G = (int)col_off.size();
  if (G < 2) return fail(JKCALS_ERR_ARG, "the jackknife needs at least two submodels (blocks with left-out rows)");
  int R = -1;
  for (int g = 0; g < h->K; ++g) {
    if (h->lo_ptr[g + 1] == h->lo_ptr[g]) continue;
    if (R < 0) R = h->R[g];
    if (h->R[g] != R) return fail(JKCALS_ERR_ARG, "the submodels differ in rank");
  }
  if (ref_block >= h->K) return fail(JKCALS_ERR_ARG, "ref_block out of range");
  if (ref_block >= 0 && h->R[ref_block] != R) return fail(JKCALS_ERR_ARG, "ref_block's rank differs from the submodels'");
  if (ref_block < 0) {
    if (ref == nullptr) return fail(JKCALS_ERR_ARG, "ref is NULL and no ref_block given");
    for (int n = 0; n < N; ++n)
      if (ref[n] == nullptr) return fail(JKCALS_ERR_ARG, "ref[n] is NULL");
  }
  if (aligned != nullptr)
    for (int n = 0; n < N; ++n)
      if (aligned[n] == nullptr) return fail(JKCALS_ERR_ARG, "aligned[n] is NULL");

  // workspace: submodel offsets, permutations, adjusted factors, S, external reference
  size_t elems = 0;
  for (int n = 0; n < N; ++n) elems += (size_t)h->dims[n] * R * ((size_t)G + 2);
  const size_t perm_bytes = (sizeof(int32_t) * (size_t)G * R + 7) / 8 * 8;  // keeps the doubles 8-byte aligned
  void* ws = nullptr;
  JK_TRY(dalloc(h, &ws, sizeof(int64_t) * G + perm_bytes + sizeof(double) * elems));
  struct Free {
    jkcals_ctx* h;
    void* p;
    ~Free() { dfree(h, p); }
  } free_ws{h, ws};
  char* cur = static_cast<char*>(ws);
  SeArgs a{};
  a.N = N;
  a.n_hat = h->n_hat;
  a.R = R;
  a.G = G;
  a.C = h->C;
  a.col_off = reinterpret_cast<const int64_t*>(cur);
  JK_CUDA(h, cudaMemcpyAsync(cur, col_off.data(), sizeof(int64_t) * G, cudaMemcpyHostToDevice, h->stream));
  cur += sizeof(int64_t) * G;
  a.perm = reinterpret_cast<int32_t*>(cur);
  cur += perm_bytes;
  double* dcur = reinterpret_cast<double*>(cur);
  for (int n = 0; n < N; ++n) {
    a.dims[n] = h->dims[n];
    a.U[n] = h->U[n];
    const size_t E = (size_t)h->dims[n] * R;
    a.aligned[n] = dcur;
    dcur += E * G;
    a.S[n] = dcur;
    dcur += E;
    if (ref_block >= 0) {
      a.ref[n] = h->U[n] + h->off[ref_block];
    } else {
      JK_CUDA(h, cudaMemcpyAsync(dcur, ref[n], sizeof(double) * E, cudaMemcpyDefault, h->stream));
      a.ref[n] = dcur;
    }
    dcur += E;
  }
  a.ref_ld = ref_block >= 0 ? h->C : R;
  JK_CUDA(h, launch_jackknife_se(a, h->stream));
  for (int n = 0; n < N; ++n) {
    const size_t E = (size_t)h->dims[n] * R;
    if (n != h->n_hat) JK_CUDA(h, cudaMemcpyAsync(S[n], a.S[n], sizeof(double) * E, cudaMemcpyDefault, h->stream));
    if (aligned != nullptr)
      JK_CUDA(h, cudaMemcpyAsync(aligned[n], a.aligned[n], sizeof(double) * E * G, cudaMemcpyDefault, h->stream));
  }
  if (perm != nullptr)
    JK_CUDA(h, cudaMemcpyAsync(perm, a.perm, sizeof(int32_t) * G * R, cudaMemcpyDefault, h->stream));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (n_submodels != nullptr) *n_submodels = G;
  return JKCALS_OK;
}

// ---- compaction of converged blocks (jkcals_run) ---------------------------------
// While compacted, the handle's block arrays (U, Grams, tensor-core factor
// copies, block metadata, status and losses) hold only the active blocks, side
// by side; h->cmp keeps the full layout.  Each block's arithmetic does not
// depend on its position among the columns, so a compacted sweep computes the
// same per-block update as a full one (the split-K grouping of the sums follows
// the new plan).

// Fits the current plan into the workspace allocated at create (never
// reallocated here, so captured graphs, a batch's included, keep valid
// pointers): a mode whose split-K partials would not fit gets fewer splits, a
// two-phase update more rows per chunk.
void fit_plan_to_workspace(jkcals_ctx* h) {
  const size_t eb = part_kind(h) == kPartF32 ? sizeof(float) : sizeof(double);
  for (int n = 0; n < h->N; ++n) {
    while (mode_splits(h, n) > 1 && (size_t)mode_splits(h, n) * h->dims[n] * h->C * eb > h->part_bytes)
      set_mode_splits(h, n, mode_splits(h, n) / 2);
    UpdatePlan& u = h->plan[n].upd;
    if ((size_t)u.RC * h->K > h->upd_chunks) {
      int64_t RC = std::max<int64_t>(1, (int64_t)(h->upd_chunks / std::max(1, h->K)));
      const int64_t rpc = (h->dims[n] + RC - 1) / RC;
      u.rows_per_chunk = (int)rpc;
      u.RC = (int)((h->dims[n] + rpc - 1) / rpc);
    }
  }
}

// Writes the current (compacted) blocks' state into the full layout of h->cmp.
jkcals_status compaction_save(jkcals_ctx* h) {
  jkcals_ctx::Compaction& c = h->cmp;
  cudaStream_t st = h->stream;
  std::vector<int> cols(h->C);
  for (int p = 0; p < h->K; ++p)
    for (int r = 0; r < h->R[p]; ++r) cols[h->off[p] + r] = c.off[c.cur_to_orig[p]] + r;
  JK_CUDA(h, cudaMemcpyAsync(c.d_cols, cols.data(), sizeof(int) * h->C, cudaMemcpyHostToDevice, st));
  for (int n = 0; n < h->N; ++n)
    JK_CUDA(h, launch_scatter_columns(h->U[n], h->C, c.U[n], c.C, c.d_cols, h->C, h->dims[n], st));
  std::vector<double> gram(h->gram_total);
  std::vector<int32_t> status(h->K);
  std::vector<double> lp(h->K), ll(h->K);
  for (int n = 0; n < h->N; ++n) {
    JK_CUDA(h, cudaMemcpyAsync(gram.data(), h->gram[n], sizeof(double) * h->gram_total, cudaMemcpyDeviceToHost, st));
    JK_CUDA(h, cudaStreamSynchronize(st));
    for (int p = 0; p < h->K; ++p) {
      const int a = c.cur_to_orig[p];
      std::copy(gram.begin() + h->gram_off[p], gram.begin() + h->gram_off[p] + h->R[p] * h->R[p],
                c.gram[n].begin() + c.gram_off[a]);
    }
  }
  JK_CUDA(h, cudaMemcpyAsync(status.data(), h->d_status, sizeof(int32_t) * h->K, cudaMemcpyDeviceToHost, st));
  JK_CUDA(h, cudaMemcpyAsync(lp.data(), h->d_loss_prev, sizeof(double) * h->K, cudaMemcpyDeviceToHost, st));
  JK_CUDA(h, cudaMemcpyAsync(ll.data(), h->d_loss_last, sizeof(double) * h->K, cudaMemcpyDeviceToHost, st));
  JK_CUDA(h, cudaStreamSynchronize(st));
  for (int p = 0; p < h->K; ++p) {
    const int a = c.cur_to_orig[p];
    c.status[a] = status[p];
    c.loss_prev[a] = lp[p];
    c.loss_last[a] = ll[p];
  }
  return JKCALS_OK;
}

// Loads the original blocks `sel` (in this order) from the full layout of
// h->cmp into the handle's arrays and plans for them.  full: sel is every block
// and the full layout's plans come back unchanged.
jkcals_status compaction_load(jkcals_ctx* h, const std::vector<int>& sel, bool full) {
  jkcals_ctx::Compaction& c = h->cmp;
  cudaStream_t st = h->stream;
  const int K = (int)sel.size();
  h->R.resize(K);
  h->off.resize(K);
  h->gram_off.resize(K);
  h->lo_ptr.assign(1, 0);
  h->lo_idx.clear();
  int col = 0, go = 0;
  h->Rmax = 0;
  for (int p = 0; p < K; ++p) {
    const int a = sel[p];
    h->R[p] = c.R[a];
    h->off[p] = col;
    h->gram_off[p] = go;
    col += c.R[a];
    go += c.R[a] * c.R[a];
    h->Rmax = std::max(h->Rmax, c.R[a]);
    h->lo_idx.insert(h->lo_idx.end(), c.lo_idx.begin() + c.lo_ptr[a], c.lo_idx.begin() + c.lo_ptr[a + 1]);
    h->lo_ptr.push_back((int64_t)h->lo_idx.size());
  }
  h->K = K;
  h->C = col;
  h->gram_total = go;
  h->uniform_rank = true;
  for (int p = 0; p < K; ++p) h->uniform_rank = h->uniform_rank && h->R[p] == h->Rmax;
  if (full) {
    h->Rmax = c.Rmax;
    h->uniform_rank = c.uniform_rank;
  }
  std::vector<int> cols(h->C);
  for (int p = 0; p < K; ++p)
    for (int r = 0; r < h->R[p]; ++r) cols[h->off[p] + r] = c.off[sel[p]] + r;
  std::vector<double> gram(std::max(1, go));
  std::vector<int32_t> status(K);
  std::vector<double> nt(K), lp(K), ll(K);
  for (int p = 0; p < K; ++p) {
    status[p] = c.status[sel[p]];
    nt[p] = c.normT2[sel[p]];
    lp[p] = c.loss_prev[sel[p]];
    ll[p] = c.loss_last[sel[p]];
  }
  JK_CUDA(h, cudaMemcpyAsync(c.d_cols, cols.data(), sizeof(int) * h->C, cudaMemcpyHostToDevice, st));
  for (int n = 0; n < h->N; ++n)
    JK_CUDA(h, launch_gather_columns(c.U[n], c.C, h->U[n], h->C, c.d_cols, h->C, h->dims[n], st));
  for (int n = 0; n < h->N; ++n) {
    for (int p = 0; p < K; ++p)
      std::copy(c.gram[n].begin() + c.gram_off[sel[p]], c.gram[n].begin() + c.gram_off[sel[p]] + h->R[p] * h->R[p],
                gram.begin() + h->gram_off[p]);
    JK_CUDA(h, cudaMemcpyAsync(h->gram[n], gram.data(), sizeof(double) * go, cudaMemcpyHostToDevice, st));
    JK_CUDA(h, cudaStreamSynchronize(st));   // gram is reused for the next mode
  }
  JK_CUDA(h, cudaMemcpyAsync(h->d_R, h->R.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_off, h->off.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_gram_off, h->gram_off.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_lo_ptr, h->lo_ptr.data(), sizeof(int64_t) * (K + 1), cudaMemcpyHostToDevice, st));
  if (!h->lo_idx.empty())
    JK_CUDA(h, cudaMemcpyAsync(h->d_lo_idx, h->lo_idx.data(), sizeof(int64_t) * h->lo_idx.size(),
                               cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_status, status.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_normT2, nt.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_loss_prev, lp.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaMemcpyAsync(h->d_loss_last, ll.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st));
  JK_CUDA(h, cudaStreamSynchronize(st));   // the host vectors above are pageable
  c.cur_to_orig = sel;

  // plans for the new column count; the full layout's plans come back as they were
  if (full) {
    for (int n = 0; n < h->N; ++n) {
      h->plan[n] = c.plan[n];
      h->tcplan[n] = c.tcplan[n];
    }
  } else {
    if (h->tc) JK_TRY(make_tc_plan(h));
    make_plan(h);
    fit_plan_to_workspace(h);
    size_t fsmem = 0;
    for (int n = 0; n < h->N; ++n)
      if (h->plan[n].upd.fused) fsmem = std::max(fsmem, h->plan[n].upd.fused_smem);
    if (fsmem > 0) JK_CUDA(h, prepare_update_fused(fsmem, h->Rmax, h->uniform_rank));
  }
  // the tensor-core forms' transposed FP32 factor copies and column maxima
  if (h->tc)
    for (int n = 0; n < h->N; ++n) {
      JK_CUDA(h, tc::launch_factor_to_ut(h->U[n], h->dims[n], h->C, h->UT[n], h->UTlo[n], h->Ipad[n], st));
      JK_CUDA(h, tc::launch_colmax(h->UT[n], h->dims[n], h->Ipad[n], h->C, h->cmax[n], st));
    }
  h->graph_valid = false;
  return JKCALS_OK;
}

// Compacts the handle to the blocks whose status (current positions) is 0.
jkcals_status compaction_shrink(jkcals_ctx* h, const std::vector<int32_t>& status) {
  jkcals_ctx::Compaction& c = h->cmp;
  if (!c.on) {
    c.K = h->K;
    c.C = h->C;
    c.Rmax = h->Rmax;
    c.gram_total = h->gram_total;
    c.uniform_rank = h->uniform_rank;
    c.R = h->R;
    c.off = h->off;
    c.gram_off = h->gram_off;
    c.lo_ptr = h->lo_ptr;
    c.lo_idx = h->lo_idx;
    for (int n = 0; n < h->N; ++n) {
      c.plan[n] = h->plan[n];
      c.tcplan[n] = h->tcplan[n];
    }
    c.status.assign(h->K, 0);
    c.normT2.assign(h->K, 0.0);
    c.loss_prev.assign(h->K, 0.0);
    c.loss_last.assign(h->K, 0.0);
    JK_CUDA(h, cudaMemcpyAsync(c.normT2.data(), h->d_normT2, sizeof(double) * h->K, cudaMemcpyDeviceToHost,
                               h->stream));
    for (int n = 0; n < h->N; ++n) {
      c.gram[n].assign(std::max(1, h->gram_total), 0.0);
      if (c.U[n] == nullptr) JK_TRY(dalloc_t(h, &c.U[n], (size_t)h->dims[n] * h->C));
    }
    if (c.d_cols == nullptr) JK_TRY(dalloc_t(h, &c.d_cols, (size_t)h->C));
    c.cur_to_orig.resize(h->K);
    std::iota(c.cur_to_orig.begin(), c.cur_to_orig.end(), 0);
    c.on = true;
  }
  JK_TRY(compaction_save(h));
  std::vector<int> sel;
  for (int p = 0; p < h->K; ++p)
    if (status[p] == 0) sel.push_back(c.cur_to_orig[p]);
  return compaction_load(h, sel, false);
}

// Restores the full layout (every block in its original place).
jkcals_status compaction_restore(jkcals_ctx* h) {
  jkcals_ctx::Compaction& c = h->cmp;
  if (!c.on) return JKCALS_OK;
  JK_TRY(compaction_save(h));
  std::vector<int> all(c.K);
  std::iota(all.begin(), all.end(), 0);
  JK_TRY(compaction_load(h, all, true));
  c.on = false;
  return JKCALS_OK;
}

jkcals_status jkcals_run(jkcals_t h, int max_sweeps, double tol, int* sweeps_done, double* final_loss) {
  JK_TRY(check_handle(h));
  if (max_sweeps < 0 || !(tol >= 0.0)) return fail(JKCALS_ERR_ARG, "bad max_sweeps or tol");
  const int chunk = 16;
  JK_TRY(ensure_loss_cap(h, chunk));
  h->tol_host = tol;
  JK_CUDA(h, cudaMemcpyAsync(h->d_tol, &h->tol_host, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  int done = 0;
  std::vector<int32_t> st;
  std::vector<double> lh;
  h->run_block_sweeps.assign(h->K, 0);
  // one chunk of sweeps, the per-block bookkeeping, and the compaction once at
  // most half of the blocks being swept are still active
  auto chunk_step = [&](bool& stop) -> jkcals_status {
    const int n = std::min(chunk, max_sweeps - done);
    JK_CUDA(h, cudaMemsetAsync(h->d_sweep_idx, 0, sizeof(int), h->stream));
    JK_TRY(run_sweeps(h, n));
    done += n;
    st.resize(h->K);
    lh.resize((size_t)n * h->K);
    JK_CUDA(h, cudaMemcpyAsync(st.data(), h->d_status, sizeof(int32_t) * h->K, cudaMemcpyDeviceToHost, h->stream));
    // a block's loss is NaN in the sweeps after it froze: its sweeps are the finite ones
    JK_CUDA(h, cudaMemcpyAsync(lh.data(), h->loss_hist, sizeof(double) * n * h->K, cudaMemcpyDeviceToHost,
                               h->stream));
    JK_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int t = 0; t < n; ++t)
      for (int p = 0; p < h->K; ++p)
        if (std::isfinite(lh[(size_t)t * h->K + p])) ++h->run_block_sweeps[h->cmp.on ? h->cmp.cur_to_orig[p] : p];
    int active = 0;
    for (int32_t v : st) active += v == 0 ? 1 : 0;
    if (active == 0 || done >= max_sweeps) {
      stop = true;
      return JKCALS_OK;
    }
    if (h->opt.compact && 2 * active <= h->K) JK_TRY(compaction_shrink(h, st));
    return JKCALS_OK;
  };
  jkcals_status rs = JKCALS_OK;
  bool stop = max_sweeps == 0;
  while (!stop && rs == JKCALS_OK) rs = chunk_step(stop);
  // every block back in its original place, also after a failure
  const jkcals_status rr = compaction_restore(h);
  if (rs != JKCALS_OK) return rs;
  JK_TRY(rr);
  h->tol_host = 0.0;
  JK_CUDA(h, cudaMemsetAsync(h->d_tol, 0, sizeof(double), h->stream));
  if (sweeps_done) *sweeps_done = done;
  if (final_loss) JK_TRY(copy_out(h, final_loss, h->d_loss_last, sizeof(double) * h->K));
  return any_not_spd(h);
}

jkcals_status jkcals_run_block_sweeps(jkcals_t h, int32_t* sweeps) {
  JK_TRY(check_handle(h));
  if (sweeps == nullptr) return fail(JKCALS_ERR_ARG, "sweeps is NULL");
  if ((int)h->run_block_sweeps.size() != h->K) return fail(JKCALS_ERR_STATE, "no jkcals_run on this handle yet");
  std::copy(h->run_block_sweeps.begin(), h->run_block_sweeps.end(), sweeps);
  return JKCALS_OK;
}

jkcals_status jkcals_get_factors(jkcals_t h, double* const* U) {
  JK_TRY(check_handle(h));
  if (U == nullptr) return fail(JKCALS_ERR_ARG, "U is NULL");
  for (int n = 0; n < h->N; ++n)
    if (U[n] == nullptr) return fail(JKCALS_ERR_ARG, "U[n] is NULL");
  for (int n = 0; n < h->N; ++n)
    JK_CUDA(h, cudaMemcpyAsync(U[n], h->U[n], sizeof(double) * h->dims[n] * h->C, cudaMemcpyDefault, h->stream));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  return JKCALS_OK;
}

jkcals_status jkcals_set_factors(jkcals_t h, const double* const* U) {
  JK_TRY(check_handle(h));
  if (U == nullptr) return fail(JKCALS_ERR_ARG, "U is NULL");
  for (int n = 0; n < h->N; ++n)
    if (U[n] == nullptr) return fail(JKCALS_ERR_ARG, "U[n] is NULL");
  for (int n = 0; n < h->N; ++n)
    JK_CUDA(h, cudaMemcpyAsync(h->U[n], U[n], sizeof(double) * h->dims[n] * h->C, cudaMemcpyDefault, h->stream));
  JK_TRY(refresh_factor_state(h));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  return JKCALS_OK;
}

jkcals_status jkcals_get_block_status(jkcals_t h, int32_t* status) {
  JK_TRY(check_handle(h));
  if (status == nullptr) return fail(JKCALS_ERR_ARG, "status is NULL");
  JK_CUDA(h, cudaMemcpyAsync(status, h->d_status, sizeof(int32_t) * h->K, cudaMemcpyDefault, h->stream));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  return JKCALS_OK;
}

jkcals_status jkcals_grad(jkcals_t h, const double* const* U, double* const* G, double* loss) {
  JK_TRY(check_handle(h));
  if (U != nullptr)
    for (int n = 0; n < h->N; ++n)
      if (U[n] == nullptr) return fail(JKCALS_ERR_ARG, "U[n] is NULL");
  return grad_impl(h, U, G, loss);
}

jkcals_status jkcals_loss_history(jkcals_t h, int nsweeps, double* losses) {
  JK_TRY(check_handle(h));
  if (nsweeps < 0 || nsweeps > h->loss_cap || losses == nullptr)
    return fail(JKCALS_ERR_ARG, "nsweeps outside the loss history, or losses is NULL");
  return copy_out(h, losses, h->loss_hist, sizeof(double) * nsweeps * h->K);
}

jkcals_status jkcals_sync(jkcals_t h) {
  JK_TRY(check_handle(h));
  JK_CUDA(h, cudaStreamSynchronize(h->stream));
  return JKCALS_OK;
}


}  // extern "C"

struct jkcals_batch_ctx {
  std::vector<jkcals_ctx*> hs;
  std::vector<double*> loss_ptrs;   // each handle's loss history when the graph was captured
  std::vector<cudaEvent_t> ready;   // per handle: its stream's work before a batch sweep
  cudaEvent_t done = nullptr;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  cudaGraphExec_t exec = nullptr;
  int max_sweeps = 0;
  bool grouped = false;             // one launch per kernel step for all problems
  std::vector<void*> dev;           // device tables of the grouped launches
};

namespace {

// A batch sweep runs as grouped launches when every problem uses the same
// tensor-core form and order, no mode takes the two-step form and no handle
// asked for per-problem branches.
bool batch_groupable(const std::vector<jkcals_ctx*>& hs) {
  for (jkcals_ctx* h : hs) {
    if (h->opt.batch_branches || !h->tc || h->opt.precision != hs[0]->opt.precision || h->N != hs[0]->N)
      return false;
    for (int n = 0; n < h->N; ++n)
      if (h->tcplan[n].tts) return false;
  }
  return true;
}

jkcals_status batch_upload(jkcals_batch_ctx* b, void** dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return fail(JKCALS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  b->dev.push_back(*dst);
  e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
  return JKCALS_OK;
}

// One grouped MTTKRP of mode n over all problems, from their current plans.
struct GroupedMttkrp {
  const tc::TcArgs* args = nullptr;
  const int* first = nullptr;
  int total = 0;
  bool qm_small = true;
  size_t smem = 0;
};

jkcals_status build_grouped_mttkrp(jkcals_batch_ctx* b, int n, GroupedMttkrp& g) {
  const int P = (int)b->hs.size();
  std::vector<tc::TcArgs> args(P);
  std::vector<int> first(P + 1, 0);
  g = GroupedMttkrp{};
  for (int i = 0; i < P; ++i) {
    jkcals_ctx* h = b->hs[i];
    const tc::TcPlan& p = h->tcplan[n];
    args[i] = make_tc_args(h, n, h->UT, h->UTlo, h->cmax, false);
    first[i + 1] = first[i] + p.tiles_c * p.tiles_n * p.splits;
    g.qm_small = g.qm_small && args[i].nq <= 2;
    g.smem = std::max(g.smem, tc::tc_smem_bytes(p));
  }
  g.total = first[P];
  void* da = nullptr;
  void* df = nullptr;
  JK_TRY(batch_upload(b, &da, args.data(), sizeof(tc::TcArgs) * P));
  JK_TRY(batch_upload(b, &df, first.data(), sizeof(int) * (P + 1)));
  g.args = static_cast<const tc::TcArgs*>(da);
  g.first = static_cast<const int*>(df);
  const cudaError_t e = tc::prepare_mttkrp_tc_grouped(b->hs[0]->opt.precision, g.qm_small, g.smem);
  if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("grouped MTTKRP attributes: ") + cudaGetErrorString(e));
  return JKCALS_OK;
}

jkcals_status launch_grouped_mttkrp(jkcals_batch_ctx* b, const GroupedMttkrp& g) {
  const cudaError_t e = tc::launch_mttkrp_tc_grouped(b->hs[0]->opt.precision, g.args, g.first, (int)b->hs.size(),
                                                     g.total, g.qm_small, g.smem, b->stream);
  if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("grouped MTTKRP: ") + cudaGetErrorString(e));
  return JKCALS_OK;
}

// Batch autotuner (any handle created with opt.autotune): per mode, the split
// factor of every problem scaled by 1, 1/2, 1/4 or 1/8 (a CTA's share of the
// contraction grows as the problems share the GPU), the fastest grouped MTTKRP
// kept (one warm-up and three timed launches each, CUDA events on the batch's
// stream; the launches write only the split-K partials).
jkcals_status autotune_grouped(jkcals_batch_ctx* b) {
  const int P = (int)b->hs.size();
  const int N = b->hs[0]->N;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(JKCALS_ERR_CUDA, "cudaEventCreate");
  jkcals_status st = JKCALS_OK;
  for (int n = 0; n < N && st == JKCALS_OK; ++n) {
    std::vector<int> base(P);
    for (int i = 0; i < P; ++i) base[i] = mode_splits(b->hs[i], n);
    int best_scale = 1;
    float best_ms = 1e30f;
    for (int scale = 1; scale <= 8 && st == JKCALS_OK; scale *= 2) {
      for (int i = 0; i < P; ++i) set_mode_splits(b->hs[i], n, std::max(1, base[i] / scale));
      GroupedMttkrp g;
      st = build_grouped_mttkrp(b, n, g);
      float tot = 0.f;
      for (int r = 0; r < 4 && st == JKCALS_OK; ++r) {
        cudaEventRecord(e0, b->stream);
        st = launch_grouped_mttkrp(b, g);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(JKCALS_ERR_CUDA, "grouped MTTKRP timing");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) tot += ms;
      }
      if (st == JKCALS_OK && tot < best_ms) {
        best_ms = tot;
        best_scale = scale;
      }
    }
    for (int i = 0; i < P; ++i) set_mode_splits(b->hs[i], n, std::max(1, base[i] / best_scale));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// Captures one grouped sweep of every problem on the batch's stream: per mode,
// one MTTKRP launch for all problems, then side by side one fused-update launch
// per rank class (each problem's block arithmetic is that of its own sweep) and
// the other problems' split-K reduction and two-phase update; after the last
// mode, every sweep counter.
jkcals_status capture_grouped(jkcals_batch_ctx* b, cudaGraph_t* graph) {
  const int P = (int)b->hs.size();
  const int N = b->hs[0]->N;
  std::vector<GroupedMttkrp> mt(N);
  struct UpdClass {
    int Rmax;
    bool uniform;
    bool df;   // wide_update_double_float of the class's problems (this mode)
    int threads = 0;
    size_t smem = 0;
    std::vector<UpdateArgs> args;
    std::vector<int> first{0};
    const UpdateArgs* dargs = nullptr;
    const int* dfirst = nullptr;
  };
  std::vector<std::vector<UpdClass>> upd(N);
  for (int n = 0; n < N; ++n) {
    JK_TRY(build_grouped_mttkrp(b, n, mt[n]));
    for (jkcals_ctx* h : b->hs) {
      if (!h->plan[n].upd.fused) continue;
      UpdClass* c = nullptr;
      const bool df = wide_update_double_float(h->tc, h->dims[n]);
      for (UpdClass& u : upd[n])
        if (u.Rmax == h->Rmax && u.uniform == h->uniform_rank && u.df == df) c = &u;
      if (c == nullptr) {
        upd[n].push_back(UpdClass{h->Rmax, h->uniform_rank, df});
        c = &upd[n].back();
      }
      c->args.push_back(update_args(h, n, h->part, part_kind(h), mode_splits(h, n)));
      c->first.push_back(c->first.back() + h->K);
      c->threads = std::max(c->threads, update_fused_threads(h->dims[n], h->Rmax, h->uniform_rank));
      c->smem = std::max(c->smem, h->plan[n].upd.fused_smem);
    }
    for (UpdClass& c : upd[n]) {
      void* da = nullptr;
      void* df = nullptr;
      JK_TRY(batch_upload(b, &da, c.args.data(), sizeof(UpdateArgs) * c.args.size()));
      JK_TRY(batch_upload(b, &df, c.first.data(), sizeof(int) * c.first.size()));
      c.dargs = static_cast<const UpdateArgs*>(da);
      c.dfirst = static_cast<const int*>(df);
      const cudaError_t e = prepare_update_grouped(c.threads, c.Rmax, c.uniform, c.df, c.smem);
      if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("grouped update attributes: ") + cudaGetErrorString(e));
    }
  }
  std::vector<int*> counters(P);
  for (int i = 0; i < P; ++i) counters[i] = b->hs[i]->d_sweep_idx;
  void* dc = nullptr;
  JK_TRY(batch_upload(b, &dc, counters.data(), sizeof(int*) * P));

  // The update launches of one mode touch disjoint problems: each runs on a
  // side stream forked from the batch's stream after the grouped MTTKRP and
  // joined before the next mode, so the graph holds them as parallel nodes.
  size_t nside = 1;
  for (int n = 0; n < N; ++n) nside = std::max(nside, upd[n].size() + 1);
  std::vector<cudaStream_t> side(nside, nullptr);
  std::vector<cudaEvent_t> evs;
  auto cleanup = [&]() {
    for (cudaStream_t x : side)
      if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : evs) cudaEventDestroy(x);
  };
  cudaError_t e = cudaSuccess;
  for (cudaStream_t& x : side)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
  // one fork event per mode and one join event per (mode, side stream)
  for (size_t k = 0; e == cudaSuccess && k < (size_t)N * (nside + 1); ++k) {
    cudaEvent_t x = nullptr;
    e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) evs.push_back(x);
  }
  if (e != cudaSuccess) {
    cleanup();
    return fail(JKCALS_ERR_CUDA, std::string("batch side streams: ") + cudaGetErrorString(e));
  }
  e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cleanup();
    return fail(JKCALS_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
  }
  jkcals_status st = JKCALS_OK;
  for (int n = 0; n < N && st == JKCALS_OK; ++n) {
    st = launch_grouped_mttkrp(b, mt[n]);
    cudaEvent_t fork = evs[(size_t)n * (nside + 1)];
    if (st == JKCALS_OK && (e = cudaEventRecord(fork, b->stream)) != cudaSuccess)
      st = fail(JKCALS_ERR_CUDA, std::string("batch fork: ") + cudaGetErrorString(e));
    for (size_t k = 0; k < nside && st == JKCALS_OK; ++k)
      if ((e = cudaStreamWaitEvent(side[k], fork, 0)) != cudaSuccess)
        st = fail(JKCALS_ERR_CUDA, std::string("batch fork: ") + cudaGetErrorString(e));
    for (size_t ci = 0; ci < upd[n].size(); ++ci) {
      const UpdClass& c = upd[n][ci];
      if (st != JKCALS_OK) break;
      e = launch_update_grouped(c.dargs, c.dfirst, (int)c.args.size(), c.first.back(), c.threads, c.Rmax, c.uniform,
                                c.df, c.smem, side[ci]);
      if (e != cudaSuccess)
        st = fail(JKCALS_ERR_CUDA, std::string("grouped update (mode ") + std::to_string(n) + ", rank class " +
                                       std::to_string(c.Rmax) + (c.uniform ? " uniform" : " mixed") + ", " +
                                       std::to_string(c.threads) + " threads, " + std::to_string(c.smem) +
                                       " B dynamic shared memory, " + std::to_string(c.first.back()) +
                                       " blocks; " + grouped_update_attrs() + "): " + cudaGetErrorString(e));
    }
    cudaStream_t s2 = side[nside - 1];   // the other problems' reduction and two-phase update
    for (jkcals_ctx* h : b->hs) {
      if (st != JKCALS_OK || h->plan[n].upd.fused) continue;
      const int64_t cnt = h->dims[n] * (int64_t)h->C;
      e = part_kind(h) == kPartF32x2
              ? launch_reduce_partials_f32x2(static_cast<float2*>(h->part), mode_splits(h, n), cnt, h->mbuf, s2)
              : launch_reduce_partials_f32(static_cast<float*>(h->part), mode_splits(h, n), cnt, h->mbuf, s2);
      if (e == cudaSuccess) e = launch_update(update_args(h, n, h->mbuf, kPartF64, 1), s2);
      if (e != cudaSuccess) st = fail(JKCALS_ERR_CUDA, std::string("batched two-phase update: ") + cudaGetErrorString(e));
    }
    for (size_t k = 0; k < nside && st == JKCALS_OK; ++k) {
      cudaEvent_t join = evs[(size_t)n * (nside + 1) + 1 + k];
      if ((e = cudaEventRecord(join, side[k])) != cudaSuccess || (e = cudaStreamWaitEvent(b->stream, join, 0)) != cudaSuccess)
        st = fail(JKCALS_ERR_CUDA, std::string("batch join: ") + cudaGetErrorString(e));
    }
  }
  if (st == JKCALS_OK) {
    e = launch_advance_sweeps(static_cast<int* const*>(dc), P, b->stream);
    if (e != cudaSuccess) st = fail(JKCALS_ERR_CUDA, std::string("sweep counters: ") + cudaGetErrorString(e));
  }
  e = cudaStreamEndCapture(b->stream, graph);
  cleanup();
  if (st != JKCALS_OK) {
    if (*graph) cudaGraphDestroy(*graph);
    *graph = nullptr;
    return st;
  }
  if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  return JKCALS_OK;
}

}  // namespace

extern "C" {

void jkcals_batch_destroy(jkcals_batch_t b) {
  if (b == nullptr) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (void* p : b->dev) cudaFree(p);
  for (cudaEvent_t e : b->ready)
    if (e) cudaEventDestroy(e);
  if (b->done) cudaEventDestroy(b->done);
  if (b->owns_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

jkcals_status jkcals_batch_create(jkcals_batch_t* out, int n, const jkcals_t* handles, int max_sweeps,
                                  void* stream) {
  if (out == nullptr || handles == nullptr || n <= 0 || max_sweeps <= 0)
    return fail(JKCALS_ERR_ARG, "jkcals_batch_create: out, handles, n > 0 and max_sweeps > 0 are required");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    JK_TRY(check_handle(handles[i]));
    if (handles[i]->opt.kernel_timing) return fail(JKCALS_ERR_ARG, "batched handles cannot use kernel_timing");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(JKCALS_ERR_ARG, "a handle appears twice in the batch");
  }
  jkcals_batch_ctx* b = new jkcals_batch_ctx();
  b->max_sweeps = max_sweeps;
  auto bail = [&](jkcals_status s) {
    jkcals_batch_destroy(b);
    return s;
  };
  cudaError_t e = cudaSuccess;
  if (stream != nullptr) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(JKCALS_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    b->owns_stream = true;
  }
  if ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess)
    return bail(fail(JKCALS_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e)));
  std::vector<jkcals_ctx*> hv(handles, handles + n);
  if (batch_groupable(hv)) {
    // one launch per kernel step for all problems (see capture_grouped)
    b->grouped = true;
    for (int i = 0; i < n; ++i) {
      jkcals_ctx* h = handles[i];
      jkcals_status s = ensure_loss_cap(h, max_sweeps);
      if (s != JKCALS_OK) return bail(s);
      cudaEvent_t ev = nullptr;
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return bail(fail(JKCALS_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e)));
      b->ready.push_back(ev);
      if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess)
        return bail(fail(JKCALS_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e)));
      b->hs.push_back(h);
      b->loss_ptrs.push_back(h->loss_hist);
    }
    bool tune = false;
    for (jkcals_ctx* h : b->hs) tune = tune || (h->opt.autotune && h->opt.splits <= 0);
    if (tune) {
      const jkcals_status s = autotune_grouped(b);
      if (s != JKCALS_OK) return bail(s);
    }
    cudaGraph_t gg = nullptr;
    const jkcals_status s = capture_grouped(b, &gg);
    if (s != JKCALS_OK) return bail(s);
    e = cudaGraphInstantiate(&b->exec, gg, 0);
    cudaGraphDestroy(gg);
    if (e != cudaSuccess)
      return bail(fail(JKCALS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)));
    *out = b;
    return JKCALS_OK;
  }
  cudaGraph_t g = nullptr;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess)
    return bail(fail(JKCALS_ERR_CUDA, std::string("cudaGraphCreate: ") + cudaGetErrorString(e)));
  for (int i = 0; i < n; ++i) {
    jkcals_ctx* h = handles[i];
    jkcals_status s = ensure_loss_cap(h, max_sweeps);
    cudaEvent_t ev = nullptr;
    if (s == JKCALS_OK && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      s = fail(JKCALS_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    if (ev) b->ready.push_back(ev);
    cudaGraph_t hg = nullptr;
    if (s == JKCALS_OK) {
      // one sweep of this problem, captured from its own stream
      if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        s = fail(JKCALS_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
      } else {
        s = enqueue_sweep(h);
        e = cudaStreamEndCapture(h->stream, &hg);
        if (s == JKCALS_OK && e != cudaSuccess)
          s = fail(JKCALS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
      }
    }
    if (s == JKCALS_OK) {
      cudaGraphNode_t node;
      if ((e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, hg)) != cudaSuccess)
        s = fail(JKCALS_ERR_CUDA, std::string("cudaGraphAddChildGraphNode: ") + cudaGetErrorString(e));
    }
    if (hg) cudaGraphDestroy(hg);
    if (s != JKCALS_OK) {
      cudaGraphDestroy(g);
      return bail(s);
    }
    b->hs.push_back(h);
    b->loss_ptrs.push_back(h->loss_hist);
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bail(fail(JKCALS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)));
  *out = b;
  return JKCALS_OK;
}

jkcals_status jkcals_batch_sweep(jkcals_batch_t b, int nsweeps) {
  if (b == nullptr) return fail(JKCALS_ERR_ARG, "null batch");
  if (nsweeps < 0 || nsweeps > b->max_sweeps) return fail(JKCALS_ERR_ARG, "nsweeps outside [0, max_sweeps]");
  if (nsweeps == 0) return JKCALS_OK;
  cudaError_t e = cudaSuccess;
  auto cu = [&](cudaError_t r, const char* what) {
    if (r != cudaSuccess) e = r;
    return r == cudaSuccess ? JKCALS_OK : fail(JKCALS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(r));
  };
  for (size_t i = 0; i < b->hs.size(); ++i) {
    jkcals_ctx* h = b->hs[i];
    if (h->loss_hist != b->loss_ptrs[i])
      return fail(JKCALS_ERR_STATE, "a batched handle's loss history was reallocated; recreate the batch");
    JK_TRY(cu(cudaEventRecord(b->ready[i], h->stream), "cudaEventRecord"));
    JK_TRY(cu(cudaStreamWaitEvent(b->stream, b->ready[i], 0), "cudaStreamWaitEvent"));
    h->tol_host = 0.0;
    JK_TRY(cu(cudaMemsetAsync(h->d_tol, 0, sizeof(double), b->stream), "cudaMemsetAsync"));
    JK_TRY(cu(cudaMemsetAsync(h->d_sweep_idx, 0, sizeof(int), b->stream), "cudaMemsetAsync"));
  }
  for (int s = 0; s < nsweeps; ++s) JK_TRY(cu(cudaGraphLaunch(b->exec, b->stream), "cudaGraphLaunch"));
  JK_TRY(cu(cudaEventRecord(b->done, b->stream), "cudaEventRecord"));
  for (jkcals_ctx* h : b->hs) JK_TRY(cu(cudaStreamWaitEvent(h->stream, b->done, 0), "cudaStreamWaitEvent"));
  (void)e;
  return JKCALS_OK;
}

jkcals_status jkcals_batch_sync(jkcals_batch_t b) {
  if (b == nullptr) return fail(JKCALS_ERR_ARG, "null batch");
  const cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return fail(JKCALS_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
  for (jkcals_ctx* h : b->hs) JK_TRY(check_device_error(h));
  return JKCALS_OK;
}

}  // extern "C"
