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
// Roles inside one CTA (10 warps, one CTA per SM):
//   warp 0     TMA producer: streams BN-row tiles of the (pre-split) unfolding
//              T_(n) into a ring of B stages.  The unfolding is stored pre-tiled
//              in the exact shared-memory image of a stage (K-major, 128- or
//              64-byte swizzle), so each stage is one contiguous bulk copy per
//              part instead of BN short rows strided across T_(n).
//   warp 1     owns TMEM; one lane issues tcgen05.mma (kind::tf32, or
//              kind::f16 with BF16 operands) for every (A-part, B-part) pair
//              of the precision form, accumulating in FP32 in TMEM.
//   warps 2-9  build the 128 x BK tile of KRP_n^T into a ring of A stages,
//              straight in the UMMA K-major swizzled layout: element (c, j) =
//              U_a^T(c, i_a(j)) * prod_{other k} U_k^T(c, i_k(j)), in FP32 from
//              transposed FP32 copies of the factor multi-matrices (the rows of
//              the fastest mode a are staged in shared memory once per CTA),
//              then split into the form's parts.  After the main loop they drain
//              TMEM (tcgen05.ld 32x32b) and write this split's partial of Mbar_n.
// The A and B rings are separate: the small TMA-fed B ring gets as many stages
// as fit, so T-tile latency is hidden even when the A ring is double-buffered.
// The Khatri-Rao product never exists in global memory.
//
// Exact-chain form (JKCALS_EXACT_BF16): every operand value x of a row whose
// magnitudes stay below 2^E is written as x = 2^(E-7) (s0 + s1/2^7 + s2/2^14 +
// s3/2^21) with integers |s_k| <= 128 (round-to-nearest extraction, exact in
// FP32) and stored as BF16 s_k * 2^(-7k).  Products of level 0 (s0 t0) and of
// level 1 (s0 t1 + s1 t0) are integer multiples of 1 and 2^-7 whose chain sums
// stay below 2^24 units for chains of <= 1024 columns, so they accumulate
// exactly in FP32 TMEM; levels 2-3 share a third accumulator whose truncation
// is scaled by 2^-14.  The Khatri-Rao entries themselves are formed as
// unevaluated FP32 pairs (error-free FMA products of hi/lo factor copies).  The
// epilogue adds the three accumulators with TwoSum into an FP32 pair and
// applies 2^(E_c - 7) 2^(F_i - 7).
//
// Synchronisation: mbarriers per A stage (tile written / consumed), per B stage
// (tile landed / consumed) and one for the accumulator.  Every wait is bounded
// by a wall-clock limit; on expiry the CTA records an error code, stops, waits
// (bounded) for its own TMA copies and MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "jk_common.cuh"
#include "jk_ptx.cuh"
#include "jk_tc.cuh"

namespace jk {
namespace tc {
namespace {

using namespace ptx;

constexpr int kProducerWarps = 8;                    // two per scheduler: hides load latency
constexpr int kThreads = 32 * (2 + kProducerWarps);  // + the TMA warp and the MMA warp
constexpr int kProducerWarp0 = 2;
constexpr int kRowsPerWarp = 128 / kProducerWarps;   // rows of the A tile per producer warp
constexpr int kRowsM = 128;                          // MMA M

// UMMA shared-memory descriptor: K-major operand, ROW-byte swizzle (128 -> 2,
// 64 -> 4), 8-row groups 8*ROW bytes apart (SBO), version 1 (tcgen05).
template <int ROW>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  constexpr uint64_t layout = ROW == 128 ? 2 : 4;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * ROW) >> 4) << 32) |
         ((uint64_t)1 << 46) | (layout << 61);
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

// 2^k as FP32 for k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// Smallest E (clamped to [-110, 110]) with |values| < 2^E given a bound b >= 0.
__device__ __forceinline__ int bound_exponent(double b) {
  if (!(b > 0.0)) return 0;
  int e;
  frexp(b, &e);   // b = m 2^e, m in [0.5, 1)
  return e < -110 ? -110 : (e > 110 ? 110 : e);
}

// BF16 bit patterns of values that BF16 represents exactly (the slices and
// splits): the upper 16 bits of the FP32 pattern; two per 32-bit word.
__device__ __forceinline__ uint32_t pack_bf16_exact(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Split one FP32 value (plus a low part for the exact-chain form) into the
// form's parts, returned as FP32 values that the part's storage represents exactly.
template <class Cfg>
__device__ __forceinline__ void split_value(float v, float vl, float scale, float (&p)[4]) {
  if constexpr (Cfg::exact) {
    // y = (v + vl) * scale lies in [-128, 128].  (r + M_k) - M_k with M_k =
    // 1.5 * 2^(23 - 7k) rounds r to the nearest multiple of 2^(-7k) (FP32
    // round-to-nearest), so each slice comes out already scaled by 2^(-7k);
    // every step is exact except adding the low part after the first slice
    // (error below 2^-25 of the grid unit).
    float y = __fmul_rn(v, scale);
    const float s0 = __fsub_rn(__fadd_rn(y, 12582912.f), 12582912.f);          // M = 1.5 * 2^23
    y = __fadd_rn(__fsub_rn(y, s0), __fmul_rn(vl, scale));
    const float s1 = __fsub_rn(__fadd_rn(y, 98304.f), 98304.f);                 // M = 1.5 * 2^16
    y = __fsub_rn(y, s1);
    const float s2 = __fsub_rn(__fadd_rn(y, 768.f), 768.f);                     // M = 1.5 * 2^9
    y = __fsub_rn(y, s2);
    const float s3 = __fsub_rn(__fadd_rn(y, 6.f), 6.f);                         // M = 1.5 * 2^2
    p[0] = s0;
    p[1] = s1;
    p[2] = s2;
    p[3] = s3;
  } else if constexpr (Cfg::kind == kKindTF32) {
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

template <class Cfg>
__global__ void __launch_bounds__(kThreads, 1)
    mttkrp_tc_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int NS = Cfg::nsplit;
  constexpr int ROW = Cfg::row_bytes;            // bytes of K per operand row in one stage
  constexpr int BK = ROW / Cfg::elem;            // columns of T_(n) per stage
  constexpr int CHUNK = 16 / Cfg::elem;          // elements per 16-byte chunk
  constexpr int CPR = ROW / 16;                  // chunks per row
  constexpr int RPI = 32 / CPR;                  // rows covered by one warp instruction
  constexpr int ROWS_PER_THREAD = kRowsPerWarp / RPI;  // rows per producer thread per stage
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t a_bytes = kRowsM * ROW;
  const uint32_t b_bytes = (uint32_t)a.BN * ROW;
  const uint32_t a_stage = NS * a_bytes, b_stage = NS * b_bytes;
  const int SA = a.stages_a, SB = a.stages_b;
  // layout: A ring | B ring | staged mode-a rows (FP32 hi, BF16 lo) | barriers
  unsigned char* a_ring = smem;
  unsigned char* b_ring = smem + (size_t)SA * a_stage;
  float* ua_hi = reinterpret_cast<float*>(b_ring + (size_t)SB * b_stage);
  // staged rows: FP32 with a 16-byte skew (ua_stride floats), BF16 low parts
  // densely (Ia_pad elements: a multiple of 8, so rows stay 16-byte aligned)
  const size_t ua_n = a.ua_smem ? (size_t)kRowsM * a.ua_stride : 0;
  const size_t ua_ln = (a.ua_smem && Cfg::exact) ? (size_t)kRowsM * a.Ia_pad : 0;
  __nv_bfloat16* ua_lo = reinterpret_cast<__nv_bfloat16*>(ua_hi + ua_n);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ua_lo + ua_ln);
  uint64_t* full_a = bars;
  uint64_t* empty_a = bars + SA;
  uint64_t* full_b = bars + 2 * SA;
  uint64_t* empty_b = bars + 2 * SA + SB;
  uint64_t* accum = bars + 2 * SA + 2 * SB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int c0 = blockIdx.x * kRowsM;
  const int n0 = blockIdx.y * a.BN;
  const int64_t jb = (int64_t)blockIdx.z * a.kchunk;
  int64_t je = jb + a.kchunk;
  if (je > a.Jp) je = a.Jp;
  const int nk = (je > jb) ? (int)((je - jb + BK - 1) / BK) : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SA; ++s) {
      mbar_init(&full_a[s], kProducerWarps);   // one arrival per producer warp
      mbar_init(&empty_a[s], 1);
    }
    for (int s = 0; s < SB; ++s) {
      mbar_init(&full_b[s], 1);
      mbar_init(&empty_b[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer: tiles of T_(n) ------------------------------
    if (lane == 0) {
      int issued = 0;
      // this CTA's first stage image: N tile blockIdx.y, k-step jb / BK
      const unsigned char* src = a.Tt + ((int64_t)blockIdx.y * a.nkt + jb / BK) * (int64_t)b_stage;
      for (int it = 0; it < nk; ++it) {
        const int s = it % SB;
        const uint32_t ph = (uint32_t)(it / SB) & 1u;
        if (!wait_bounded(&empty_b[s], ph ^ 1u, abort_flag, a.err, 1)) break;
        mbar_arrive_expect_tx(&full_b[s], b_stage);
        unsigned char* dst = b_ring + (size_t)s * b_stage;
#pragma unroll
        for (int p = 0; p < NS; ++p) bulk_load(dst + p * b_bytes, src + p * b_bytes, b_bytes, &full_b[s]);
        src += b_stage;
        issued = it + 1;
      }
      if (*abort_flag) {
        // let every copy this thread started land before the CTA exits
        for (int it = (issued > SB ? issued - SB : 0); it < issued; ++it)
          wait_drain(&full_b[it % SB], (uint32_t)(it / SB) & 1u);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer --------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = make_idesc(Cfg::fmt, kRowsM, (uint32_t)a.BN);
      // The descriptor's start-address field is (address >> 4) in its low 14
      // bits, so every operand descriptor is the region's base descriptor plus
      // (byte offset >> 4): one add per MMA instead of rebuilding it.
      const uint64_t adesc0 = smem_desc<ROW>(smem_u32(a_ring));
      const uint64_t bdesc0 = smem_desc<ROW>(smem_u32(b_ring));
      const uint32_t tmem_acc1 = tmem + (uint32_t)a.acc_cols, tmem_acc2 = tmem + 2u * (uint32_t)a.acc_cols;
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int sa = it % SA, sb = it % SB;
        ok = wait_bounded(&full_b[sb], (uint32_t)(it / SB) & 1u, abort_flag, a.err, 2) &&
             wait_bounded(&full_a[sa], (uint32_t)(it / SA) & 1u, abort_flag, a.err, 3);
        if (!ok) break;
        tc_fence_after();
        const uint64_t ad0 = adesc0 + (uint64_t)(((uint32_t)sa * a_stage) >> 4);
        const uint64_t bd0 = bdesc0 + (uint64_t)(((uint32_t)sb * b_stage) >> 4);
#pragma unroll
        for (int kk = 0; kk < ROW / 32; ++kk) {
#pragma unroll
          for (int q = 0; q < Cfg::npass; ++q) {
            const uint64_t ad = ad0 + (uint64_t)((Cfg::pass_a(q) * a_bytes + kk * 32) >> 4);
            const uint64_t bd = bd0 + (uint64_t)((Cfg::pass_b(q) * b_bytes + kk * 32) >> 4);
            const uint32_t d = Cfg::pass_acc(q) == 0 ? tmem : (Cfg::pass_acc(q) == 1 ? tmem_acc1 : tmem_acc2);
            const bool first = (it == 0 && kk == 0 && Cfg::first_of_acc(q));
            tc_mma<Cfg::kind>(d, ad, bd, idesc, first ? 0u : 1u);
          }
        }
        tc_commit(&empty_a[sa]);
        tc_commit(&empty_b[sb]);
      }
      // Always signal the accumulator: its phase completes once every MMA issued
      // above has finished, so on an abort this lane drains them before TMEM is freed.
      tc_commit(accum);
      if (!ok) wait_drain(accum, 0);
    }
  } else {
    // ---------------- Khatri-Rao producers (warps 2..9) ------------------------------
    const int pw = warp - kProducerWarp0;   // 0..kProducerWarps-1
    const int rg = lane / CPR;              // row within a group of RPI rows
    const int q = lane % CPR;               // 16-byte chunk within the row
    // per-row constants, hoisted out of the k loop
    bool cval[ROWS_PER_THREAD];
    float rscale[ROWS_PER_THREAD];
    uint32_t soff[ROWS_PER_THREAD];                      // swizzled offset in an A tile
    const float* ra[ROWS_PER_THREAD];                    // global rows of UTa (unstaged path)
    const float* ral[ROWS_PER_THREAD];
    const float* rq0[ROWS_PER_THREAD];
    const float* rq0l[ROWS_PER_THREAD];
    const float* rq1[ROWS_PER_THREAD];
    const float* rq1l[ROWS_PER_THREAD];
    uint32_t ua_row[ROWS_PER_THREAD], ua_rowl[ROWS_PER_THREAD];   // staged rows (shared addresses)
#pragma unroll
    for (int rr = 0; rr < ROWS_PER_THREAD; ++rr) {
      const int m = pw * kRowsPerWarp + rr * RPI + rg;   // row of the A tile = column c0 + m
      const int c = c0 + m;
      cval[rr] = c < a.C;
      const int cc = cval[rr] ? c : 0;
      const int sw = (ROW == 128) ? (m & 7) : ((m >> 1) & 3);
      soff[rr] = (uint32_t)(m >> 3) * (8u * ROW) + (uint32_t)(m & 7) * ROW + (uint32_t)((q ^ sw) << 4);
      ra[rr] = a.UTa + (int64_t)cc * a.Ia_pad;
      ral[rr] = Cfg::exact ? a.UTa_lo + (int64_t)cc * a.Ia_pad : nullptr;
      rq0[rr] = a.nq > 0 ? a.UTq[0] + (int64_t)cc * a.qpad[0] : nullptr;
      rq0l[rr] = (Cfg::exact && a.nq > 0) ? a.UTq_lo[0] + (int64_t)cc * a.qpad[0] : nullptr;
      rq1[rr] = a.nq > 1 ? a.UTq[1] + (int64_t)cc * a.qpad[1] : nullptr;
      rq1l[rr] = (Cfg::exact && a.nq > 1) ? a.UTq_lo[1] + (int64_t)cc * a.qpad[1] : nullptr;
      ua_row[rr] = smem_u32(ua_hi + (size_t)m * a.ua_stride);
      ua_rowl[rr] = smem_u32(ua_lo + (size_t)m * a.Ia_pad);
      rscale[rr] = 1.f;
      if constexpr (Cfg::exact) {
        if (cval[rr]) {
          double b = (double)__ldg(a.cmax_a + c);
#pragma unroll
          for (int t = 0; t < kMaxModes - 2; ++t)
            if (t < a.nq) b *= (double)__ldg(a.cmax_q[t] + c);
          rscale[rr] = pow2f(7 - bound_exponent(b));
        }
      }
    }
    if (a.ua_smem) {
      // stage the CTA's 128 factor rows of mode a once (FP32 hi; BF16 lo for
      // the exact-chain form, which keeps the pair to ~2^-32): the k loop then
      // reads them from shared memory instead of L2
      const int ptid = threadIdx.x - 32 * kProducerWarp0;
      const int n4 = a.Ia_pad / 4;
      const int total = kRowsM * n4;
      constexpr int kU = 4;   // loads in flight per thread
      for (int idx0 = ptid; idx0 < total; idx0 += kU * 32 * kProducerWarps) {
        float4 hv[kU], lv[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = idx0 + u * 32 * kProducerWarps;
          const int row = idx / n4, col = (idx - row * n4) * 4;
          const int c = c0 + row;
          hv[u] = lv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (idx < total && c < a.C) {
            hv[u] = __ldg(reinterpret_cast<const float4*>(a.UTa + (int64_t)c * a.Ia_pad + col));
            if constexpr (Cfg::exact)
              lv[u] = __ldg(reinterpret_cast<const float4*>(a.UTa_lo + (int64_t)c * a.Ia_pad + col));
          }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = idx0 + u * 32 * kProducerWarps;
          if (idx < total) {
            const int row = idx / n4, col = (idx - row * n4) * 4;
            sts128(smem_u32(ua_hi + (size_t)row * a.ua_stride + col),
                   make_uint4(__float_as_uint(hv[u].x), __float_as_uint(hv[u].y), __float_as_uint(hv[u].z),
                              __float_as_uint(hv[u].w)));
            if constexpr (Cfg::exact) {
              const __nv_bfloat162 l01 = __floats2bfloat162_rn(lv[u].x, lv[u].y);
              const __nv_bfloat162 l23 = __floats2bfloat162_rn(lv[u].z, lv[u].w);
              uint2 pk;
              pk.x = *reinterpret_cast<const uint32_t*>(&l01);
              pk.y = *reinterpret_cast<const uint32_t*>(&l23);
              *reinterpret_cast<uint2*>(ua_lo + (size_t)row * a.Ia_pad + col) = pk;
            }
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(32 * kProducerWarps) : "memory");   // producer warps only
    }
    float qhc[ROWS_PER_THREAD], qlc[ROWS_PER_THREAD];   // cached remaining-mode products
    bool qstale = true;
    // this thread's column j of the unfolding: j = ia + Ia_pad * o, o mixed-radix
    // over the remaining modes; advanced incrementally by BK per k-step
    const int je32 = (int)je;
    int jcur = (int)jb + q * CHUNK;
    int ia = 0;
    int iq[kMaxModes - 2];
    {
      const int o = jcur / a.Ia_pad;
      ia = jcur - o * a.Ia_pad;
      int rem = o;
#pragma unroll
      for (int t = 0; t < kMaxModes - 2; ++t) {
        iq[t] = 0;
        if (t < a.nq) {
          const int qq = rem / a.qdims[t];
          iq[t] = rem - qq * a.qdims[t];
          rem = qq;
        }
      }
    }
    const uint32_t a_ring_s = smem_u32(a_ring);
    bool ok = true;
    for (int it = 0; it < nk && ok; ++it) {
      const int s = it % SA;
      // one lane per warp polls the barrier; __syncwarp orders the others after it
      bool got = true;
      if (lane == 0) got = wait_bounded(&empty_a[s], ((uint32_t)(it / SA) & 1u) ^ 1u, abort_flag, a.err, 4);
      got = __shfl_sync(0xffffffffu, got, 0);
      __syncwarp();
      if (!got) {
        ok = false;
        break;
      }
      const bool jvalid = jcur < je32;
      if (qstale && jvalid) {
        // product of the remaining modes' factor entries for each row: it only
        // changes when the column index carries out of mode a
#pragma unroll
        for (int rr = 0; rr < ROWS_PER_THREAD; ++rr) {
          float qh = 1.f, ql = 0.f;
          if (cval[rr]) {
#pragma unroll
            for (int t = 0; t < kMaxModes - 2; ++t) {
              if (t < a.nq) {
                float bh, bl = 0.f;
                if (t == 0) {
                  bh = __ldg(rq0[rr] + iq[0]);
                  if constexpr (Cfg::exact) bl = __ldg(rq0l[rr] + iq[0]);
                } else if (t == 1) {
                  bh = __ldg(rq1[rr] + iq[1]);
                  if constexpr (Cfg::exact) bl = __ldg(rq1l[rr] + iq[1]);
                } else {
                  const int64_t idx = (int64_t)(c0 + pw * kRowsPerWarp + rr * RPI + rg) * a.qpad[t] + iq[t];
                  bh = __ldg(a.UTq[t] + idx);
                  if constexpr (Cfg::exact) bl = __ldg(a.UTq_lo[t] + idx);
                }
                if constexpr (Cfg::exact) {
                  // error-free product of the pairs (qh + ql)(bh + bl)
                  const float pq = __fmul_rn(qh, bh);
                  const float eq = __fadd_rn(__fmaf_rn(qh, bh, -pq), __fmaf_rn(qh, bl, __fmul_rn(ql, bh)));
                  qh = pq;
                  ql = eq;
                } else {
                  qh *= bh;
                }
              }
            }
          }
          qhc[rr] = qh;
          qlc[rr] = ql;
        }
        qstale = false;
      }
      const uint32_t a_tile_s = a_ring_s + (uint32_t)s * a_stage;
#pragma unroll
      for (int rr = 0; rr < ROWS_PER_THREAD; ++rr) {
        float v[CHUNK], vl[CHUNK];
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) v[e] = vl[e] = 0.f;
        if (jvalid && cval[rr]) {
          const float qh = qhc[rr];
          if constexpr (!Cfg::exact) {
            const float4* src = reinterpret_cast<const float4*>(ra[rr] + ia);
#pragma unroll
            for (int e4 = 0; e4 < CHUNK / 4; ++e4) {
              const float4 u = a.ua_smem ? lds128(ua_row[rr] + (uint32_t)(ia + 4 * e4) * 4u) : __ldg(src + e4);
              v[4 * e4 + 0] = u.x * qh;
              v[4 * e4 + 1] = u.y * qh;
              v[4 * e4 + 2] = u.z * qh;
              v[4 * e4 + 3] = u.w * qh;
            }
          } else {
            // Khatri-Rao entry as an unevaluated pair (v + vl) from hi/lo factor
            // copies: error-free products (FMA) keep it far below FP32 rounding
            const float ql = qlc[rr];
            float uh[CHUNK], ul[CHUNK];
            if (a.ua_smem) {
#pragma unroll
              for (int e4 = 0; e4 < CHUNK / 4; ++e4) {
                const float4 u = lds128(ua_row[rr] + (uint32_t)(ia + 4 * e4) * 4u);
                uh[4 * e4 + 0] = u.x;
                uh[4 * e4 + 1] = u.y;
                uh[4 * e4 + 2] = u.z;
                uh[4 * e4 + 3] = u.w;
              }
              // CHUNK (8) BF16 low parts in one 16-byte load
              const float4 lraw = lds128(ua_rowl[rr] + (uint32_t)ia * 2u);
              const uint32_t w4[4] = {__float_as_uint(lraw.x), __float_as_uint(lraw.y), __float_as_uint(lraw.z),
                                      __float_as_uint(lraw.w)};
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                ul[2 * k] = __uint_as_float(w4[k] << 16);
                ul[2 * k + 1] = __uint_as_float(w4[k] & 0xffff0000u);
              }
            } else {
              const float4* src = reinterpret_cast<const float4*>(ra[rr] + ia);
              const float4* srcl = reinterpret_cast<const float4*>(ral[rr] + ia);
#pragma unroll
              for (int e4 = 0; e4 < CHUNK / 4; ++e4) {
                const float4 u = __ldg(src + e4), l = __ldg(srcl + e4);
                uh[4 * e4 + 0] = u.x;
                uh[4 * e4 + 1] = u.y;
                uh[4 * e4 + 2] = u.z;
                uh[4 * e4 + 3] = u.w;
                ul[4 * e4 + 0] = l.x;
                ul[4 * e4 + 1] = l.y;
                ul[4 * e4 + 2] = l.z;
                ul[4 * e4 + 3] = l.w;
              }
            }
#pragma unroll
            for (int k = 0; k < CHUNK; ++k) {
              const float p = __fmul_rn(uh[k], qh);
              v[k] = p;
              vl[k] = __fadd_rn(__fmaf_rn(uh[k], qh, -p), __fmaf_rn(uh[k], ql, __fmul_rn(ul[k], qh)));
            }
          }
        }
        float parts[NS][CHUNK];
#pragma unroll
        for (int e = 0; e < CHUNK; ++e) {
          float p4[4];
          split_value<Cfg>(v[e], vl[e], rscale[rr], p4);
#pragma unroll
          for (int p = 0; p < NS; ++p) parts[p][e] = p4[p];
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
            w.x = pack_bf16_exact(parts[p][0], parts[p][1]);
            w.y = pack_bf16_exact(parts[p][2], parts[p][3]);
            w.z = pack_bf16_exact(parts[p][4], parts[p][5]);
            w.w = pack_bf16_exact(parts[p][6], parts[p][7]);
          }
          sts128(a_tile_s + (uint32_t)p * a_bytes + soff[rr], w);
        }
      }
      fence_async_shared();   // each writer: generic-proxy stores -> visible to the MMA
      __syncwarp();
      if (lane == 0) mbar_arrive(&full_a[s]);
      // advance this thread's column by BK: carry i_a into the remaining modes
      jcur += BK;
      ia += BK;
      while (ia >= a.Ia_pad) {
        ia -= a.Ia_pad;
        qstale = true;
#pragma unroll
        for (int t = 0; t < kMaxModes - 2; ++t) {
          if (t < a.nq) {
            if (++iq[t] < a.qdims[t]) break;
            iq[t] = 0;
          }
        }
      }
    }

    // ---------------- epilogue: TMEM -> partial of Mbar_n ----------------------------
    bool have = ok && nk > 0 && wait_bounded(accum, 0, abort_flag, a.err, 5);
    have = __all_sync(0xffffffffu, have);   // tcgen05.ld is warp-collective
    tc_fence_after();
    const int quarter = warp & 3;                    // TMEM lanes 32*quarter .. +31
    const int half = (warp - kProducerWarp0) >> 2;   // two warps per lane quarter split the columns
    const int m = quarter * 32 + lane;
    const int c = c0 + m;
    int Ec = 0;
    if constexpr (Cfg::exact) {
      if (c < a.C) {
        double b = (double)__ldg(a.cmax_a + c);
#pragma unroll
        for (int t = 0; t < kMaxModes - 2; ++t)
          if (t < a.nq) b *= (double)__ldg(a.cmax_q[t] + c);
        Ec = bound_exponent(b);
      }
    }
    float* out = a.part + (int64_t)blockIdx.z * a.I * a.C;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int cc = 32 * half; cc < a.BN; cc += 64) {
      const int width = (a.BN - cc >= 32) ? 32 : 16;
      uint32_t v[32];
      if constexpr (!Cfg::exact) {
        if (have) {
          if (width == 32)
            tmem_ld32(lane_base + (uint32_t)cc, v);
          else
            tmem_ld16(lane_base + (uint32_t)cc, v);
          tmem_ld_wait();
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int64_t i = (int64_t)n0 + cc + r;
          if (r < width && i < a.I && c < a.C) out[i * a.C + c] = have ? __uint_as_float(v[r]) : 0.f;
        }
      } else {
        uint32_t v1[32], v2[32];
        if (have) {
          if (width == 32) {
            tmem_ld32(lane_base + (uint32_t)cc, v);
            tmem_ld32(lane_base + (uint32_t)(a.acc_cols + cc), v1);
            tmem_ld32(lane_base + (uint32_t)(2 * a.acc_cols + cc), v2);
          } else {
            tmem_ld16(lane_base + (uint32_t)cc, v);
            tmem_ld16(lane_base + (uint32_t)(a.acc_cols + cc), v1);
            tmem_ld16(lane_base + (uint32_t)(2 * a.acc_cols + cc), v2);
          }
          tmem_ld_wait();
        }
        // level 0 and level 1 are exact; add the three as an unevaluated FP32 pair
        // (hi, lo) with error-free TwoSum steps, scale by 2^(E_c + F_i - 14) and
        // store the pair; the consumer adds hi + lo
        float2* out2 = reinterpret_cast<float2*>(a.part) + (int64_t)blockIdx.z * a.I * a.C;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int64_t i = (int64_t)n0 + cc + r;
          if (r < width && i < a.I && c < a.C) {
            float2 val = make_float2(0.f, 0.f);
            if (have) {
              const float l0 = __uint_as_float(v[r]), l1 = __uint_as_float(v1[r]), l2 = __uint_as_float(v2[r]);
              const float s = __fadd_rn(l0, l1);
              const float bb = __fsub_rn(s, l0);
              const float e1 = __fadd_rn(__fsub_rn(l0, __fsub_rn(s, bb)), __fsub_rn(l1, bb));
              const float t = __fadd_rn(s, l2);
              const float b2 = __fsub_rn(t, s);
              const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(t, b2)), __fsub_rn(l2, b2));
              float lo = __fadd_rn(e1, e2);
              const float hi = __fadd_rn(t, lo);
              lo = __fsub_rn(lo, __fsub_rn(hi, t));
              const int k = Ec + __ldg(a.rowexp + i) - 2 * kSliceBits;
              val = make_float2(ldexpf(hi, k), ldexpf(lo, k));
            }
            out2[i * a.C + c] = val;
          }
        }
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
  static constexpr int kind = kKindTF32, fmt = 2, nsplit = 1, npass = 1, row_bytes = 128, elem = 4;
  static constexpr bool exact = false;
  __device__ static constexpr int pass_a(int) { return 0; }
  __device__ static constexpr int pass_b(int) { return 0; }
  __device__ static constexpr int pass_acc(int) { return 0; }
  __device__ static constexpr bool first_of_acc(int q) { return q == 0; }
};
struct Cfg3xTF32 {
  // hi*hi + hi*lo + lo*hi
  static constexpr int kind = kKindTF32, fmt = 2, nsplit = 2, npass = 3, row_bytes = 128, elem = 4;
  static constexpr bool exact = false;
  __device__ static constexpr int pass_a(int q) { return q == 2 ? 1 : 0; }
  __device__ static constexpr int pass_b(int q) { return q == 1 ? 1 : 0; }
  __device__ static constexpr int pass_acc(int) { return 0; }
  __device__ static constexpr bool first_of_acc(int q) { return q == 0; }
};
struct CfgBF16 {
  static constexpr int kind = kKindBF16, fmt = 1, nsplit = 1, npass = 1, row_bytes = 128, elem = 2;
  static constexpr bool exact = false;
  __device__ static constexpr int pass_a(int) { return 0; }
  __device__ static constexpr int pass_b(int) { return 0; }
  __device__ static constexpr int pass_acc(int) { return 0; }
  __device__ static constexpr bool first_of_acc(int q) { return q == 0; }
};
struct CfgBF16x3 {
  // (a, b) part pairs with a + b <= 2: hh, hm, mh, hl, lh, mm
  static constexpr int kind = kKindBF16, fmt = 1, nsplit = 3, npass = 6, row_bytes = 128, elem = 2;
  static constexpr bool exact = false;
  __device__ static constexpr int pass_a(int q) { return q == 2 ? 1 : q == 4 ? 2 : q == 5 ? 1 : 0; }
  __device__ static constexpr int pass_b(int q) { return q == 1 ? 1 : q == 3 ? 2 : q == 5 ? 1 : 0; }
  __device__ static constexpr int pass_acc(int) { return 0; }
  __device__ static constexpr bool first_of_acc(int q) { return q == 0; }
};
struct CfgExact {
  // slice pairs (s, t) with s + t <= 3; accumulators: level 0 | level 1 | levels 2-3
  static constexpr int kind = kKindBF16, fmt = 1, nsplit = 4, npass = 10, row_bytes = 64, elem = 2;
  static constexpr bool exact = true;
  __device__ static constexpr int pass_a(int q) {
    return q == 2 ? 1 : q == 4 ? 1 : q == 5 ? 2 : q == 7 ? 1 : q == 8 ? 2 : q == 9 ? 3 : 0;
  }
  __device__ static constexpr int pass_b(int q) {
    return q == 1 ? 1 : q == 3 ? 2 : q == 4 ? 1 : q == 6 ? 3 : q == 7 ? 2 : q == 8 ? 1 : 0;
  }
  __device__ static constexpr int pass_acc(int q) { return q == 0 ? 0 : (q <= 2 ? 1 : 2); }
  __device__ static constexpr bool first_of_acc(int q) { return q == 0 || q == 1 || q == 3; }
};

template <class Cfg>
cudaError_t set_smem_cfg(size_t smem) {
  return cudaFuncSetAttribute(mttkrp_tc_kernel<Cfg>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class Cfg>
cudaError_t launch_cfg(const TcPlan& p, const TcArgs& a, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(p);
  dim3 grid((unsigned)p.tiles_c, (unsigned)p.tiles_n, (unsigned)p.splits);
  mttkrp_tc_kernel<Cfg><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int form_nsplit(int precision) {
  switch (precision) {
    case JKCALS_TF32: return CfgTF32::nsplit;
    case JKCALS_3XTF32: return Cfg3xTF32::nsplit;
    case JKCALS_BF16: return CfgBF16::nsplit;
    case JKCALS_SPLIT_BF16: return CfgBF16x3::nsplit;
    case JKCALS_EXACT_BF16: return CfgExact::nsplit;
    default: return 0;
  }
}

int form_row_bytes(int precision) { return precision == JKCALS_EXACT_BF16 ? 64 : 128; }
int form_elem_bytes(int precision) { return (precision == JKCALS_TF32 || precision == JKCALS_3XTF32) ? 4 : 2; }
int form_bk(int precision) { return form_row_bytes(precision) / form_elem_bytes(precision); }
int form_chunk(int precision) { return 16 / form_elem_bytes(precision); }
int form_passes(int precision) {
  switch (precision) {
    case JKCALS_TF32: return CfgTF32::npass;
    case JKCALS_3XTF32: return Cfg3xTF32::npass;
    case JKCALS_BF16: return CfgBF16::npass;
    case JKCALS_SPLIT_BF16: return CfgBF16x3::npass;
    case JKCALS_EXACT_BF16: return CfgExact::npass;
    default: return 0;
  }
}

size_t tc_ua_bytes(const TcPlan& p) {
  if (!p.ua_smem) return 0;
  return (size_t)kRowsM * p.ua_stride * sizeof(float) +
         (p.ua_parts > 1 ? (size_t)kRowsM * p.Ia_pad * sizeof(__nv_bfloat16) : 0);
}

size_t tc_smem_bytes(const TcPlan& p) {
  const size_t row = (size_t)p.row_bytes;
  const size_t a_stage = (size_t)p.nsplit * kRowsM * row;
  const size_t b_stage = (size_t)p.nsplit * p.BN * row;
  return 1024 /*alignment slack*/ + (size_t)p.stages_a * a_stage + (size_t)p.stages_b * b_stage + tc_ua_bytes(p) +
         (2 * p.stages_a + 2 * p.stages_b + 1) * 8 + 16;
}

cudaError_t prepare_mttkrp_tc(int precision, size_t max_smem) {
  switch (precision) {
    case JKCALS_TF32: return set_smem_cfg<CfgTF32>(max_smem);
    case JKCALS_3XTF32: return set_smem_cfg<Cfg3xTF32>(max_smem);
    case JKCALS_BF16: return set_smem_cfg<CfgBF16>(max_smem);
    case JKCALS_SPLIT_BF16: return set_smem_cfg<CfgBF16x3>(max_smem);
    case JKCALS_EXACT_BF16: return set_smem_cfg<CfgExact>(max_smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mttkrp_tc(int precision, const TcPlan& p, const TcArgs& a, cudaStream_t s) {
  switch (precision) {
    case JKCALS_TF32: return launch_cfg<CfgTF32>(p, a, s);
    case JKCALS_3XTF32: return launch_cfg<Cfg3xTF32>(p, a, s);
    case JKCALS_BF16: return launch_cfg<CfgBF16>(p, a, s);
    case JKCALS_SPLIT_BF16: return launch_cfg<CfgBF16x3>(p, a, s);
    case JKCALS_EXACT_BF16: return launch_cfg<CfgExact>(p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tc
}  // namespace jk
