// Concurrent MTTKRP on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
//   Mbar_n^T (C x I_n) = KRP_n^T (C x J) * T_(n)^T (J x I_n)
//
// (Alg. 3 MTTKRP line; the Khatri-Rao order of Eq. MTTKRP; columns of T_(n)
// by Eq. kolda_mapping.)  The product is taken transposed so that the MMA's M
// dimension (128 accumulator lanes) runs over the C = sum_g R_g columns of all
// submodels and its N dimension over the I_n rows of the mode (<= 256 per
// tile), while the long contraction over J is split across CTAs (split-K).
//
// Roles inside one CTA (6 warps, one CTA per SM):
//   warp 0     TMA producer: streams BN x 128-byte tiles of the (pre-split)
//              unfolding T_(n) into shared memory (128B swizzle, K-major).
//   warp 1     owns TMEM; one lane issues tcgen05.mma (kind::tf32 or
//              kind::f16 with BF16 operands) for every (A-part, B-part) pair
//              of the precision form, accumulating in FP32 in TMEM.
//   warps 2-5  build the 128 x BK tile of KRP_n^T in shared memory straight
//              into the UMMA K-major 128B-swizzled layout: element (c, j) =
//              U_a^T(c, i_a(j)) * prod_{other k} U_k^T(c, i_k(j)), computed in
//              FP32 from transposed FP32 copies of the factor multi-matrices,
//              then split into TF32 hi/lo or BF16 hi/mid/lo parts.  After the
//              main loop they drain TMEM (tcgen05.ld 32x32b) and write the
//              FP32 partial tile of Mbar_n for this split.
// The Khatri-Rao product never exists in global memory.
//
// Synchronisation: mbarriers per stage (T tile landed / KRP tile written /
// stage consumed) plus one for the accumulator.  Every wait is bounded by a
// wall-clock limit; on expiry the CTA records an error code, stops, waits
// (bounded) for its own TMA copies, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "jk_common.cuh"
#include "jk_tc.cuh"

namespace jk {
namespace tc {
namespace {

constexpr int kThreads = 192;
constexpr int kProducerWarp0 = 2;
constexpr int kRowsM = 128;                       // MMA M
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per wait

// ---- small PTX wrappers ------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase with the given parity.  Returns false if this
// CTA aborted (another role timed out) or the limit expired (then it aborts).
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                             int* err, int code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (global_ns() - t0 > kWaitLimitNs) {
      *abort_flag = 1;
      atomicExch(err, code);
      return false;
    }
  }
}

// Bounded wait that ignores the abort flag (used to drain own TMA copies).
__device__ __forceinline__ void wait_drain(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) return;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (KIND == kKindTF32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// 32 lanes x 32 consecutive 32-bit TMEM columns -> 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
        "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
        "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// UMMA shared-memory descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), version 1 (tcgen05).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: FP32 accumulator, A/B format fmt (TF32 = 2 under
// kind::tf32, BF16 = 1 under kind::f16), both K-major, N and M.
__device__ __forceinline__ uint32_t make_idesc(uint32_t fmt, uint32_t M, uint32_t N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split one FP32 value into NS parts (Cfg::kind) and return their bit patterns.
template <class Cfg>
__device__ __forceinline__ void split_value(float v, float (&p)[3]) {
  if constexpr (Cfg::kind == kKindTF32) {
    const float h = tf32_rna(v);
    p[0] = h;
    if constexpr (Cfg::nsplit > 1) p[1] = tf32_rna(v - h);
  } else {
    const float h = __bfloat162float(__float2bfloat16_rn(v));
    p[0] = h;
    if constexpr (Cfg::nsplit > 1) {
      const float r1 = v - h;
      const float m = __bfloat162float(__float2bfloat16_rn(r1));
      p[1] = m;
      if constexpr (Cfg::nsplit > 2) p[2] = __bfloat162float(__float2bfloat16_rn(r1 - m));
    }
  }
}

// Shared-memory plan (host and device agree through TcArgs).
struct SmemPlan {
  uint32_t a_bytes;      // one A part: 128 rows x 128 B
  uint32_t b_bytes;      // one B part: BN rows x 128 B
  uint32_t stage_bytes;  // nsplit * (a + b)
};

template <class Cfg>
__global__ void __launch_bounds__(kThreads, 1)
    mttkrp_tc_kernel(const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
                     const __grid_constant__ CUtensorMap tm2, const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int NS = Cfg::nsplit;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t a_bytes = kRowsM * 128;
  const uint32_t b_bytes = (uint32_t)a.BN * 128;
  const uint32_t stage_bytes = NS * (a_bytes + b_bytes);
  const int STAGES = a.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)STAGES * stage_bytes);
  uint64_t* full_a = bars;
  uint64_t* full_b = bars + STAGES;
  uint64_t* empty = bars + 2 * STAGES;
  uint64_t* accum = bars + 3 * STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int c0 = blockIdx.x * kRowsM;
  const int n0 = blockIdx.y * a.BN;
  const int64_t jb = (int64_t)blockIdx.z * a.kchunk;
  int64_t je = jb + a.kchunk;
  if (je > a.Jp) je = a.Jp;
  const int nk = (je > jb) ? (int)((je - jb + Cfg::bk - 1) / Cfg::bk) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_a[s], 32 * 4);
      mbar_init(&full_b[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    fence_barrier_init();
    tma_prefetch_desc(&tm0);
    if (NS > 1) tma_prefetch_desc(&tm1);
    if (NS > 2) tma_prefetch_desc(&tm2);
  }
  if (warp == 1) tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto a_tile = [&](int s, int p) -> unsigned char* { return smem + (size_t)s * stage_bytes + p * a_bytes; };
  auto b_tile = [&](int s, int p) -> unsigned char* {
    return smem + (size_t)s * stage_bytes + NS * a_bytes + p * b_bytes;
  };

  if (warp == 0) {
    // ---------------- TMA producer: tiles of T_(n) ------------------------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nk; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        if (!wait_bounded(&empty[s], ph ^ 1u, abort_flag, a.err, 1)) break;
        mbar_arrive_expect_tx(&full_b[s], NS * b_bytes);
        const int x = (int)(jb + (int64_t)it * Cfg::bk);
        tma_load_2d(b_tile(s, 0), &tm0, &full_b[s], x, n0);
        if (NS > 1) tma_load_2d(b_tile(s, 1), &tm1, &full_b[s], x, n0);
        if (NS > 2) tma_load_2d(b_tile(s, 2), &tm2, &full_b[s], x, n0);
        issued = it + 1;
      }
      if (*abort_flag) {
        // let every copy this thread started land before the CTA exits
        for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
          wait_drain(&full_b[it % STAGES], (uint32_t)(it / STAGES) & 1u);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer --------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = make_idesc(Cfg::fmt, kRowsM, (uint32_t)a.BN);
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
        ok = wait_bounded(&full_b[s], ph, abort_flag, a.err, 2) &&
             wait_bounded(&full_a[s], ph, abort_flag, a.err, 3);
        if (!ok) break;
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
          for (int q = 0; q < Cfg::npass; ++q) {
            const uint64_t ad = sw128_desc(smem_u32(a_tile(s, Cfg::pass_a(q))) + kk * 32);
            const uint64_t bd = sw128_desc(smem_u32(b_tile(s, Cfg::pass_b(q))) + kk * 32);
            tc_mma<Cfg::kind>(tmem, ad, bd, idesc, (it > 0 || kk > 0 || q > 0) ? 1u : 0u);
          }
        }
        tc_commit(&empty[s]);
      }
      // Always signal the accumulator: its phase completes once every MMA issued
      // above has finished, so on an abort this lane drains them before TMEM is freed.
      tc_commit(accum);
      if (!ok) wait_drain(accum, 0);
    }
  } else {
    // ---------------- Khatri-Rao producers (warps 2..5) ------------------------------
    const int pw = warp - kProducerWarp0;   // 0..3
    const int r4 = lane >> 3;               // row within a group of 4
    const int q = lane & 7;                 // 16-byte chunk within the 128-byte row
    bool ok = true;
    for (int it = 0; it < nk && ok; ++it) {
      const int s = it % STAGES;
      const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
      if (!wait_bounded(&empty[s], ph ^ 1u, abort_flag, a.err, 4)) {
        ok = false;
        break;
      }
      const int64_t j = jb + (int64_t)it * Cfg::bk + q * Cfg::chunk;
      const bool jvalid = j < je;
      int ia = 0;
      int iq[kMaxModes - 2];
      if (jvalid) {
        const int64_t o = j / a.Ia_pad;
        ia = (int)(j - o * a.Ia_pad);
        int64_t rem = o;
#pragma unroll
        for (int t = 0; t < kMaxModes - 2; ++t) {
          if (t < a.nq) {
            const int64_t qq = rem / a.qdims[t];
            iq[t] = (int)(rem - qq * a.qdims[t]);
            rem = qq;
          }
        }
      }
#pragma unroll 2
      for (int rr = 0; rr < 8; ++rr) {
        const int m = pw * 32 + rr * 4 + r4;   // row of the A tile = column c0 + m
        const int c = c0 + m;
        float v[Cfg::chunk];
#pragma unroll
        for (int e = 0; e < Cfg::chunk; ++e) v[e] = 0.f;
        if (jvalid && c < a.C) {
          float qv = 1.f;
#pragma unroll
          for (int t = 0; t < kMaxModes - 2; ++t)
            if (t < a.nq) qv *= __ldg(a.UTq[t] + (int64_t)c * a.qpad[t] + iq[t]);
          const float4* src = reinterpret_cast<const float4*>(a.UTa + (int64_t)c * a.Ia_pad + ia);
#pragma unroll
          for (int e4 = 0; e4 < Cfg::chunk / 4; ++e4) {
            const float4 u = __ldg(src + e4);
            v[4 * e4 + 0] = u.x * qv;
            v[4 * e4 + 1] = u.y * qv;
            v[4 * e4 + 2] = u.z * qv;
            v[4 * e4 + 3] = u.w * qv;
          }
        }
        // split and store the 16-byte chunk of every part (128B swizzle)
        const uint32_t off = (uint32_t)(m >> 3) * 1024u + (uint32_t)(m & 7) * 128u + (uint32_t)((q ^ (m & 7)) << 4);
        float parts[NS][Cfg::chunk];
#pragma unroll
        for (int e = 0; e < Cfg::chunk; ++e) {
          float p3[3];
          split_value<Cfg>(v[e], p3);
#pragma unroll
          for (int p = 0; p < NS; ++p) parts[p][e] = p3[p];
        }
#pragma unroll
        for (int p = 0; p < NS; ++p) {
          uint4 w;
          if constexpr (Cfg::kind == kKindTF32) {
            w.x = __float_as_uint(parts[p][0]);
            w.y = __float_as_uint(parts[p][1]);
            w.z = __float_as_uint(parts[p][2]);
            w.w = __float_as_uint(parts[p][3]);
          } else {
            __nv_bfloat162 b0 = __floats2bfloat162_rn(parts[p][0], parts[p][1]);
            __nv_bfloat162 b1 = __floats2bfloat162_rn(parts[p][2], parts[p][3]);
            __nv_bfloat162 b2 = __floats2bfloat162_rn(parts[p][4], parts[p][5]);
            __nv_bfloat162 b3 = __floats2bfloat162_rn(parts[p][6], parts[p][7]);
            w.x = *reinterpret_cast<uint32_t*>(&b0);
            w.y = *reinterpret_cast<uint32_t*>(&b1);
            w.z = *reinterpret_cast<uint32_t*>(&b2);
            w.w = *reinterpret_cast<uint32_t*>(&b3);
          }
          *reinterpret_cast<uint4*>(a_tile(s, p) + off) = w;
        }
      }
      fence_async_shared();
      mbar_arrive(&full_a[s]);
    }

    // ---------------- epilogue: TMEM -> FP32 partial of Mbar_n --------------------
    bool have = ok && nk > 0 && wait_bounded(accum, 0, abort_flag, a.err, 5);
    have = __all_sync(0xffffffffu, have);   // tcgen05.ld is warp-collective
    tc_fence_after();
    const int quarter = warp & 3;             // TMEM lanes 32*quarter .. +31
    const int m = quarter * 32 + lane;
    const int c = c0 + m;
    float* out = a.part + (int64_t)blockIdx.z * a.I * a.C;
    for (int cc = 0; cc < a.BN; cc += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)cc;
      const int width = (a.BN - cc >= 32) ? 32 : 16;
      if (have) {
        if (width == 32)
          tmem_ld32(taddr, v);
        else
          tmem_ld16(taddr, v);
        tmem_ld_wait();
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int64_t i = (int64_t)n0 + cc + r;
        if (r < width && i < a.I && c < a.C) out[i * a.C + c] = have ? __uint_as_float(v[r]) : 0.f;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
  }
}

// ---- precision forms -----------------------------------------------------------

struct CfgTF32 {
  static constexpr int kind = kKindTF32, fmt = 2, nsplit = 1, npass = 1, bk = 32, chunk = 4;
  __device__ static constexpr int pass_a(int) { return 0; }
  __device__ static constexpr int pass_b(int) { return 0; }
};
struct Cfg3xTF32 {
  // hi*hi + hi*lo + lo*hi
  static constexpr int kind = kKindTF32, fmt = 2, nsplit = 2, npass = 3, bk = 32, chunk = 4;
  __device__ static constexpr int pass_a(int q) { return q == 2 ? 1 : 0; }
  __device__ static constexpr int pass_b(int q) { return q == 1 ? 1 : 0; }
};
struct CfgBF16 {
  static constexpr int kind = kKindBF16, fmt = 1, nsplit = 1, npass = 1, bk = 64, chunk = 8;
  __device__ static constexpr int pass_a(int) { return 0; }
  __device__ static constexpr int pass_b(int) { return 0; }
};
struct CfgBF16x3 {
  // (a, b) part pairs with a + b <= 2: hh, hm, mh, hl, lh, mm
  static constexpr int kind = kKindBF16, fmt = 1, nsplit = 3, npass = 6, bk = 64, chunk = 8;
  __device__ static constexpr int pass_a(int q) { return q == 2 ? 1 : q == 4 ? 2 : q == 5 ? 1 : 0; }
  __device__ static constexpr int pass_b(int q) { return q == 1 ? 1 : q == 3 ? 2 : q == 5 ? 1 : 0; }
};

template <class Cfg>
cudaError_t set_smem_cfg(size_t smem) {
  return cudaFuncSetAttribute(mttkrp_tc_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class Cfg>
cudaError_t launch_cfg(const TcPlan& p, const CUtensorMap* maps, const TcArgs& a, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(p);
  dim3 grid((unsigned)p.tiles_c, (unsigned)p.tiles_n, (unsigned)p.splits);
  mttkrp_tc_kernel<Cfg><<<grid, kThreads, smem, s>>>(maps[0], maps[1], maps[2], a);
  return cudaGetLastError();
}

}  // namespace

int form_nsplit(int precision) {
  switch (precision) {
    case JKCALS_TF32: return CfgTF32::nsplit;
    case JKCALS_3XTF32: return Cfg3xTF32::nsplit;
    case JKCALS_BF16: return CfgBF16::nsplit;
    case JKCALS_SPLIT_BF16: return CfgBF16x3::nsplit;
    default: return 0;
  }
}

int form_bk(int precision) { return (precision == JKCALS_BF16 || precision == JKCALS_SPLIT_BF16) ? 64 : 32; }
int form_elem_bytes(int precision) { return (precision == JKCALS_BF16 || precision == JKCALS_SPLIT_BF16) ? 2 : 4; }
int form_chunk(int precision) { return form_bk(precision) / 8; }
int form_passes(int precision) {
  switch (precision) {
    case JKCALS_TF32: return CfgTF32::npass;
    case JKCALS_3XTF32: return Cfg3xTF32::npass;
    case JKCALS_BF16: return CfgBF16::npass;
    case JKCALS_SPLIT_BF16: return CfgBF16x3::npass;
    default: return 0;
  }
}

size_t tc_smem_bytes(const TcPlan& p) {
  const size_t stage = (size_t)p.nsplit * (kRowsM * 128 + (size_t)p.BN * 128);
  return 1024 /*alignment slack*/ + (size_t)p.stages * stage + (3 * p.stages + 1) * 8 + 16;
}

cudaError_t prepare_mttkrp_tc(int precision, size_t max_smem) {
  switch (precision) {
    case JKCALS_TF32: return set_smem_cfg<CfgTF32>(max_smem);
    case JKCALS_3XTF32: return set_smem_cfg<Cfg3xTF32>(max_smem);
    case JKCALS_BF16: return set_smem_cfg<CfgBF16>(max_smem);
    case JKCALS_SPLIT_BF16: return set_smem_cfg<CfgBF16x3>(max_smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mttkrp_tc(int precision, const TcPlan& p, const CUtensorMap* maps, const TcArgs& a,
                             cudaStream_t s) {
  switch (precision) {
    case JKCALS_TF32: return launch_cfg<CfgTF32>(p, maps, a, s);
    case JKCALS_3XTF32: return launch_cfg<Cfg3xTF32>(p, maps, a, s);
    case JKCALS_BF16: return launch_cfg<CfgBF16>(p, maps, a, s);
    case JKCALS_SPLIT_BF16: return launch_cfg<CfgBF16x3>(p, maps, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tc
}  // namespace jk
