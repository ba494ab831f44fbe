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
// Roles inside one CTA (12 warps, one CTA per SM):
//   warp 0      TMA producer: streams BN-row tiles of the (pre-split) unfolding
//               T_(n) into the B half of each pipeline stage.  The unfolding is
//               stored pre-tiled in the exact shared-memory image of a stage
//               (K-major, 128- or 64-byte swizzle, parts adjacent), so each stage
//               is one contiguous bulk copy instead of BN short rows strided
//               across T_(n); lane s issues the copies of ring stage s.
//   warp 1      owns TMEM; one lane issues the stage's tcgen05.mma list
//               (kind::tf32, or kind::f16 with BF16 operands), FP32 accumulators
//               in TMEM.  It is alone on its scheduler (warps 5 and 9, which share
//               it, only sleep until the epilogue): busy warps there would cut its
//               issue rate several-fold and starve the tensor pipe.
//   warps 2, 3, 4, 6, 7, 8, 10, 11
//               build the 128 x BK tile of KRP_n^T into the A half of each stage,
//               straight in the UMMA K-major swizzled layout: element (c, j) =
//               U_a^T(c, i_a(j)) * prod_{other k} U_k^T(c, i_k(j)), in FP32 from
//               transposed FP32 copies of the factor multi-matrices (the rows of
//               the fastest mode a are staged in shared memory once per CTA; the
//               remaining modes' entries are fetched one k-step ahead), then
//               split into the form's parts.
//   warps 4-11  after the main loop drain TMEM (tcgen05.ld 32x32b, two warps per
//               lane quarter) and write this split's partial of Mbar_n.
// The Khatri-Rao product never exists in global memory.
//
// Split forms: with operand parts A_s, B_t (s, t < P), the products A_s B_t with
// s + t < P are accumulated per level l = s + t in TMEM columns [l L, l L + BN)
// (L = lstride).  The B parts of a stage are contiguous BN-row blocks, so one
// MMA of A_s against the parts t0..t1 (N = (t1 - t0 + 1) BN <= 256) lands part
// t in level s + t directly when L = BN: the exact form needs 4 MMAs per K slice
// instead of 10 for BN = 64.
//
// Exact-chain form (JKCALS_EXACT_BF16): every operand value x of a row whose
// magnitudes stay below 2^E is written as x = 2^(E-7) (s0 + s1/2^7 + s2/2^14 +
// r3) with integers |s_0| <= 128, |s_1|, |s_2| <= 64 (round-to-nearest
// extraction, exact in FP32), stored as BF16 s_k * 2^(-7k), and a BF16 last
// slice r3 of the remainder (the T side keeps it on the grid 2^-21 too; the
// Khatri-Rao side rounds it to 8 significant bits).  Products of
// level 0 (s0 t0) and of level 1 (s0 t1 + s1 t0) are integer multiples of 1 and
// 2^-7 whose chain sums stay below 2^24 units for chains of <= 1024 columns, so
// they accumulate exactly in FP32 TMEM; levels 2 and 3 carry truncation scaled
// by 2^-14.  The Khatri-Rao entries themselves are formed as unevaluated FP32
// pairs (error-free FMA products of hi/lo factor copies), with packed f32x2
// arithmetic.  The epilogue adds the levels with TwoSum into an FP32 pair and
// applies 2^(E_c - 7) 2^(F_i - 7).
//
// Synchronisation: per stage one "full" mbarrier (the producer warps' arrivals
// plus the TMA arrival and its bytes) and one "empty" mbarrier (the MMAs'
// commit), so the MMA lane waits once per stage; one more for the accumulator.  Every wait is bounded
// by a wall-clock limit; on expiry the CTA records an error code, stops, waits
// (bounded) for its own TMA copies and MMAs, frees its TMEM and returns.
//
// The exact-chain form has a second kernel for narrow modes (mttkrp_tts_kernel,
// further down): no Khatri-Rao producers, one GEMM per index of the remaining
// modes, the scaling by their factor entries done in the epilogue.
#include <cuda_bf16.h>

#include "jk_common.cuh"
#include "jk_ptx.cuh"
#include "jk_tc.cuh"

namespace jk {
namespace tc {
namespace {

using namespace ptx;

// Warp roles.  A warp runs on scheduler (warp id mod 4); the MMA warp must not
// share its scheduler with busy warps (four arithmetic warps there cut its
// issue rate about fourfold), so warps 5 and 9 only drain TMEM.
//   0: TMA  1: MMA  2, 3, 4, 6, 7, 8, 10, 11: Khatri-Rao producers
//   4..11: epilogue (two warps per TMEM lane quarter)
constexpr int kWarps = 12;
constexpr int kThreads = 32 * kWarps;
constexpr int kProducerWarps = 8;
constexpr int kRowsPerWarp = 128 / kProducerWarps;   // rows of the A tile per producer warp
constexpr int kEpilogueWarp0 = 4;
constexpr int kEpilogueWarps = kWarps - kEpilogueWarp0;
__device__ __forceinline__ bool is_producer_warp(int w) { return w >= 2 && (w & 3) != 1; }
__device__ __forceinline__ int producer_index(int w) { return w - 2 - (w > 5) - (w > 9); }
constexpr int kRowsM = 128;                          // MMA M
constexpr int kMaxMma = 10;                          // entries of an MmaList

// UMMA shared-memory descriptor: K-major operand, ROW-byte swizzle (128 -> 2,
// 64 -> 4), 8-row groups 8*ROW bytes apart (SBO), version 1 (tcgen05).
template <int ROW>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  constexpr uint64_t layout = ROW == 128 ? 2 : 4;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((8 * ROW) >> 4) << 32) |
         ((uint64_t)1 << 46) | (layout << 61);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// 2^k as FP32 for k in [-126, 127]
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// Smallest E (clamped to [-110, 110]) with prod_k x_k < 2^E for the maxima
// x_k >= 0 of the factors of one Khatri-Rao column (0 when a factor is zero).
// Exponents add exactly; the mantissas (in [0.5, 1)) multiply in FP32, whose
// rounding is monotonic, so the bound can only come out one binade looser,
// never tighter.  No FP64: its pipe is narrow on this part.
__device__ __forceinline__ int bound_exponent_prod(float x0, const float* const* more, int nmore, int c) {
  if (!(x0 > 0.f)) return 0;
  int e, esum;
  float m = frexpf(x0, &esum);
#pragma unroll
  for (int t = 0; t < kMaxModes - 2; ++t) {
    if (t < nmore) {
      const float x = __ldg(more[t] + c);
      if (!(x > 0.f)) return 0;
      m *= frexpf(x, &e);
      esum += e;
    }
  }
  frexpf(m, &e);
  esum += e;
  return esum < -110 ? -110 : (esum > 110 ? 110 : esum);
}

// BF16 bit patterns of values that BF16 represents exactly (the slices and
// splits): the upper 16 bits of the FP32 pattern; two per 32-bit word.
__device__ __forceinline__ uint32_t pack_bf16_exact(float lo, float hi) {
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// ---- packed FP32 pairs (two lanes of f32x2 arithmetic, round to nearest) ----
struct f2 {
  uint64_t r;
};
__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
  f2 v;
  asm("mov.b64 %0, {%1, %2};" : "=l"(v.r) : "f"(lo), "f"(hi));
  return v;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v.r));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
  return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
  return d;
}

// Split one FP32 value into the parts of a non-exact form, returned as FP32
// values that the part's storage represents exactly.
template <class Cfg>
__device__ __forceinline__ void split_value(float v, float (&p)[4]) {
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

// Exact-chain form, two Khatri-Rao entries at once: the pairs (u_e + ul_e) *
// (qh + ql), with the row's power of two already folded into (qh, ql) so that
// the product lies in [-128, 128], as unevaluated FP32 pairs (error-free FMA
// products), cut into four BF16 slices.  Slices 0-2 are rounded onto the grids
// 1, 2^-7 and 2^-14: (r + M_k) - M_k with M_k = 1.5 * 2^(23 - 7k) rounds r to
// the nearest multiple of 2^(-7k).  On these grids the products of levels 0
// and 1, and in practice level 2 (its terms are multiples of 2^-14 and its
// chain sums stay near 2^24 units), accumulate exactly.  Slice 3 only meets
// the truncating level-3 accumulator, so plain round-to-nearest BF16
// conversion suffices (the remainder is below 2^-24 of the grid 2^-14).
// Every step is exact except adding the low part after the first slice.
// Returns the BF16 patterns of the two entries' slices, one word per slice.
__device__ __forceinline__ uint32_t cvt_bf16x2(f2 v) {   // {bf16(lo) | bf16(hi) << 16}
  float lo, hi;
  f2_unpack(v, lo, hi);
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
__device__ __forceinline__ void exact_slices2(f2 u, f2 ul, f2 qh2, f2 nqh2, f2 ql2, uint32_t (&w)[4]) {
  const f2 p = f2_mul(u, qh2);
  const f2 e1n = f2_fma(u, nqh2, p);                           // p - u qh, exact
  const f2 e2 = f2_fma(u, ql2, f2_mul(ul, qh2));               // u ql + ul qh
  const f2 vl = f2_sub(e2, e1n);
  const f2 m0 = f2_pack(12582912.f, 12582912.f);               // 1.5 * 2^23
  const f2 m1 = f2_pack(98304.f, 98304.f);                     // 1.5 * 2^16
  const f2 s0 = f2_sub(f2_add(p, m0), m0);
  const f2 y1 = f2_add(f2_sub(p, s0), vl);
  const f2 s1 = f2_sub(f2_add(y1, m1), m1);
  const f2 m2 = f2_pack(768.f, 768.f);                         // 1.5 * 2^9
  const f2 y2 = f2_sub(y1, s1);
  const f2 s2 = f2_sub(f2_add(y2, m2), m2);
  w[3] = cvt_bf16x2(f2_sub(y2, s2));
  float a, b;
  f2_unpack(s0, a, b);
  w[0] = pack_bf16_exact(a, b);
  f2_unpack(s1, a, b);
  w[1] = pack_bf16_exact(a, b);
  f2_unpack(s2, a, b);
  w[2] = pack_bf16_exact(a, b);
}

// Error-free product of the pairs (qh + ql)(bh + bl), renormalised.
__device__ __forceinline__ void pair_mul(float& qh, float& ql, float bh, float bl) {
  const float pq = __fmul_rn(qh, bh);
  const float eq = __fadd_rn(__fmaf_rn(qh, bh, -pq), __fmaf_rn(qh, bl, __fmul_rn(ql, bh)));
  qh = pq;
  ql = eq;
}

// The MMAs of one 32-byte K slice kk of a stage, unrolled at compile time for
// P operand parts, B parts stacked G at a time along N and, for MERGED, levels
// 2 and 3 sharing one accumulator: A part s times B parts t0..t1 into TMEM
// columns (level of s + t0) * L.  (A list read from kernel parameters at run
// time costs the issuing lane about half the stage time.)  Only BN enters at
// run time: the B part stride b_bytes and the N field, idesc[c] for c parts.
template <class Cfg, int G, bool MERGED>
__device__ __forceinline__ void issue_slice(uint32_t tmem, uint64_t ad0, uint64_t bd0, uint32_t L, uint32_t b16,
                                            const uint32_t (&idesc)[5], int kk, bool first_slice) {
  constexpr int P = Cfg::nsplit;
  constexpr uint32_t a16 = (uint32_t)(128 * Cfg::row_bytes) >> 4;   // A part stride in 16-byte units
#pragma unroll
  for (int s = 0; s < P; ++s) {
#pragma unroll
    for (int t0 = 0; t0 < P - s; t0 += G) {
      const int cnt = (t0 + G <= P - s) ? G : P - s - t0;
      const int lev = MERGED ? (s + t0 < 2 ? s + t0 : 2) : s + t0;
      // an MMA overwrites its columns on the chain's first slice iff none of
      // its levels was written before it: the s = 0 MMAs (merged: the first
      // one per level)
      const bool fresh = s == 0 && (!MERGED || t0 <= 2);
      tc_mma<Cfg::kind>(tmem + (uint32_t)lev * L, ad0 + (uint64_t)(s * a16 + 2 * kk),
                        bd0 + (uint64_t)((uint32_t)t0 * b16 + 2 * kk), idesc[cnt], (first_slice && fresh) ? 0u : 1u);
    }
  }
}

// All MMAs of one stage (K slices kk = 0 .. KS-1), ordered so that the MMAs
// into one accumulator follow each other: for each (s, t0) of issue_slice the
// K slices back to back.  On the chain's first stage the s = 0 MMAs of slice 0
// overwrite their columns; they still come before every other MMA into them.
template <class Cfg, int G, bool MERGED, int KS>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint64_t ad0, uint64_t bd0, uint32_t L, uint32_t b16,
                                            const uint32_t (&idesc)[5], bool first_stage) {
  constexpr int P = Cfg::nsplit;
  constexpr uint32_t a16 = (uint32_t)(128 * Cfg::row_bytes) >> 4;
#pragma unroll
  for (int s = 0; s < P; ++s) {
#pragma unroll
    for (int t0 = 0; t0 < P - s; t0 += G) {
      const int cnt = (t0 + G <= P - s) ? G : P - s - t0;
      const int lev = MERGED ? (s + t0 < 2 ? s + t0 : 2) : s + t0;
      const bool fresh = s == 0 && (!MERGED || t0 <= 2);
#pragma unroll
      for (int kk = 0; kk < KS; ++kk)
        tc_mma<Cfg::kind>(tmem + (uint32_t)lev * L, ad0 + (uint64_t)(s * a16 + 2 * kk),
                          bd0 + (uint64_t)((uint32_t)t0 * b16 + 2 * kk), idesc[cnt],
                          (first_stage && fresh && kk == 0) ? 0u : 1u);
    }
  }
}

// QM: slots for the remaining modes beyond a that the producers track (the
// column index carry, the factor entries of Q) — 2 covers tensors of up to 4
// modes with short per-k-step index code, kMaxModes - 2 the rest.
// The CTA (bx, by, bz) of one problem's launch: C tile bx, N tile by, split bz.
// smem: the 1024-byte aligned dynamic shared memory.
template <class Cfg, int QM>
__device__ __forceinline__ void mttkrp_tc_body(const TcArgs& a, int bx, int by, int bz, unsigned char* smem) {
  constexpr int NS = Cfg::nsplit;
  constexpr int ROW = Cfg::row_bytes;            // bytes of K per operand row in one stage
  constexpr int BK = ROW / Cfg::elem;            // columns of T_(n) per stage
  constexpr int CHUNK = 16 / Cfg::elem;          // elements per 16-byte chunk
  constexpr int CPR = ROW / 16;                  // chunks per row
  constexpr int RPI = 32 / CPR;                  // rows covered by one warp instruction
  constexpr int RPT = kRowsPerWarp / RPI;        // rows per producer thread per stage
  static_assert(RPT >= 1 && RPT * RPI == kRowsPerWarp, "producer mapping");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t a_bytes = kRowsM * ROW;
  const uint32_t b_bytes = (uint32_t)a.BN * ROW;
  const uint32_t a_stage = NS * a_bytes, b_stage = NS * b_bytes;
  const uint32_t stage_bytes = a_stage + b_stage;   // a multiple of 1024
  const int S = a.stages;
  // layout: S stages of (A parts | B parts) | staged mode-a rows (FP32 hi, BF16 lo) | barriers
  unsigned char* ring = smem;
  float* ua_hi = reinterpret_cast<float*>(ring + (size_t)S * stage_bytes);
  // staged rows: FP32 with a 16-byte skew (ua_stride floats), BF16 low parts
  // densely (Ia_pad elements: a multiple of 8, so rows stay 16-byte aligned)
  const size_t ua_n = a.ua_smem ? (size_t)kRowsM * a.ua_stride : 0;
  const size_t ua_ln = (a.ua_smem && Cfg::exact) ? (size_t)kRowsM * a.Ia_pad : 0;
  __nv_bfloat16* ua_lo = reinterpret_cast<__nv_bfloat16*>(ua_hi + ua_n);
  uint64_t* bars = reinterpret_cast<uint64_t*>(ua_lo + ua_ln);
  uint64_t* full = bars;          // stage written: producer warps + the TMA arrival and its bytes
  uint64_t* empty = bars + S;     // stage consumed: the MMAs' commit
  uint64_t* accum = bars + 2 * S;        // a segment's MMAs are complete
  uint64_t* tmem_empty = accum + 1;       // the epilogue warps drained a segment
  uint64_t* drain = accum + 2;            // abort path: the MMAs issued so far are complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* srowexp = const_cast<int*>(abort_flag + 1);   // BN row exponents of this N tile (exact form)

  const int c0 = bx * kRowsM;
  const int n0 = by * a.BN;
  const int64_t jb = (int64_t)bz * a.kchunk;
  int64_t je = jb + a.kchunk;
  if (je > a.Jp) je = a.Jp;
  const int nk = (je > jb) ? (int)((je - jb + BK - 1) / BK) : 0;
  // Exact-chain form: the exactly accumulated levels hold at most
  // kExactChainMax columns, so a CTA's chain runs in segments of that length;
  // after each the epilogue warps drain TMEM into the CTA's partial.  Other
  // forms: one segment.
  const int seg = Cfg::exact ? kExactChainMax / BK : (nk > 0 ? nk : 1);
  const int nseg = Cfg::exact ? (nk + seg - 1) / seg : (nk > 0 ? 1 : 0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], kProducerWarps + 1);   // one arrival per producer warp + the TMA thread
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    mbar_init(tmem_empty, kEpilogueWarps);
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
  if constexpr (Cfg::exact) {
    // the drains scale every row by its exponent: read them once
    if ((int)threadIdx.x < a.BN) {
      const int64_t i = (int64_t)n0 + threadIdx.x;
      srowexp[threadIdx.x] = i < a.I ? __ldg(a.rowexp + i) : 0;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer: tiles of T_(n) ------------------------------
    // Lane s serves ring stage s: one bulk copy of the stage's B parts (contiguous
    // in the pre-tiled image and in the ring) per k-step it = s, s + S, ...  One
    // thread's bulk copies complete one after another (~0.3-0.4 us each for
    // 4-40 KB from L2), copies from different threads overlap, so the loads of
    // the S stages are issued by S lanes.
    if (lane < S) {
      int issued = 0;
      // this CTA's first stage image: N tile by, k-step jb / BK
      const unsigned char* src = a.Tt + ((int64_t)by * a.nkt + jb / BK) * (int64_t)b_stage;
      unsigned char* dst = ring + (size_t)lane * stage_bytes + a_stage;
      uint32_t ph = 0;   // parity of this stage's pass
      for (int it = lane; it < nk; it += S, ph ^= 1u) {
        if (!wait_bounded(&empty[lane], ph ^ 1u, abort_flag, a.err, 1)) break;
        mbar_arrive_expect_tx(&full[lane], b_stage);
        bulk_load(dst, src + (int64_t)it * b_stage, b_stage, &full[lane]);
        issued = it + 1;
      }
      if (*abort_flag && issued > 0) {
        // let the copies this thread started land before the CTA exits (a
        // stage's phase may never complete once producers stopped, so wait a
        // fixed, ample time instead of on the barrier)
        const uint64_t t0 = global_ns();
        while (global_ns() - t0 < 200000ull) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer --------------------------------------------------
    if (lane == 0) {
      // The descriptor's start-address field is (address >> 4) in its low 14
      // bits, so every operand descriptor is the region's base descriptor plus
      // (byte offset >> 4): the list holds those offsets per MMA.
      const uint64_t desc0 = smem_desc<ROW>(smem_u32(ring));
      const uint32_t L = (uint32_t)a.lstride, b16 = b_bytes >> 4;
      uint32_t idesc[5];   // FP32 accumulator, A/B formats, both K-major, N = c BN, M = 128
#pragma unroll
      for (int c = 0; c < 5; ++c)
        idesc[c] = (1u << 4) | ((uint32_t)Cfg::fmt << 7) | ((uint32_t)Cfg::fmt << 10) |
                   (((uint32_t)(c * a.BN) >> 3) << 17) | ((uint32_t)(kRowsM >> 4) << 24);
      const int variant = a.merged ? 0 : (a.stack >= 4 ? 4 : a.stack);   // uniform over the kernel
      bool ok = true;
      int j = 0, kin = 0;   // segment and k-step within it, tracked without divisions
      int s = 0;            // ring stage and the parity of its pass, likewise
      uint32_t ph = 0;
      for (int it = 0; it < nk && ok; ++it) {
        if (Cfg::exact && kin == 0 && j > 0) {
          // the next segment overwrites the accumulators once they are drained
          ok = wait_bounded(tmem_empty, (uint32_t)(j - 1) & 1u, abort_flag, a.err, 7);
          if (!ok) break;
        }
        ok = wait_bounded(&full[s], ph, abort_flag, a.err, 2);
        if (!ok) break;
        tc_fence_after();
        const uint64_t ad0 = desc0 + (uint64_t)(((uint32_t)s * stage_bytes) >> 4);
        const uint64_t bd0 = ad0 + (uint64_t)(a_stage >> 4);
        {
          constexpr int KS = ROW / 32;
          const bool first = kin == 0;
          switch (variant) {
            case 4: issue_stage<Cfg, 4, false, KS>(tmem, ad0, bd0, L, b16, idesc, first); break;
            case 2: issue_stage<Cfg, 2, false, KS>(tmem, ad0, bd0, L, b16, idesc, first); break;
            case 1: issue_stage<Cfg, 1, false, KS>(tmem, ad0, bd0, L, b16, idesc, first); break;
            default: issue_stage<Cfg, 1, true, KS>(tmem, ad0, bd0, L, b16, idesc, first); break;
          }
        }
        tc_commit(&empty[s]);
        if (kin == seg - 1 || it == nk - 1) tc_commit(accum);   // segment j complete
        if (++kin == seg) {
          kin = 0;
          ++j;
        }
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
      // On an abort, wait (bounded) until every MMA issued so far has finished,
      // so that TMEM is not freed under them.
      if (!ok) {
        tc_commit(drain);
        wait_drain(drain, 0);
      }
    }
  } else {
    bool ok = true;
    int drained = 0;   // segments drained so far (epilogue warps)
    // ---------------- epilogue: TMEM -> partial of Mbar_n, once per segment -------------
    // Segment j's accumulators are added into this split's partial (stored for
    // j = 0) and the MMA warp is released to overwrite them.  Warps 5 and 9
    // share the MMA warp's scheduler: they sleep in the wait.
    const int quarter = warp & 3;                      // TMEM lanes 32*quarter .. +31
    const int grp = (warp - kEpilogueWarp0) >> 2;      // two warps per lane quarter split the columns
    const int m_e = quarter * 32 + lane;
    const int c_e = c0 + m_e;
    int Ec = 0;
    if constexpr (Cfg::exact) {
      if (warp >= kEpilogueWarp0 && c_e < a.C)
        Ec = bound_exponent_prod(__ldg(a.cmax_a + c_e), a.cmax_q, a.nq, c_e);
    }
    auto drain_segment = [&](int j) {
      const int c = c_e;
      bool have = ok && nk > 0 && wait_sleepy(accum, (uint32_t)j & 1u, abort_flag, a.err, 5);
      have = __all_sync(0xffffffffu, have);   // tcgen05.ld is warp-collective
      tc_fence_after();
      const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
      const uint32_t L = (uint32_t)a.lstride;
      // 16-column slices (BN is a multiple of 16), dealt round-robin to the two
      // warps of each lane quarter
      for (int cc = 16 * grp; cc < a.BN && have; cc += 32) {
        const uint32_t col = lane_base + (uint32_t)cc;
        if constexpr (!Cfg::exact) {
          uint32_t v0[32], v1[32], v2[32];
          tmem_ld16(col, v0);
          if (a.nlev > 1) tmem_ld16(col + L, v1);
          if (a.nlev > 2) tmem_ld16(col + 2 * L, v2);
          tmem_ld_wait();
          float* out = a.part + (int64_t)bz * a.I * a.C;
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int64_t i = (int64_t)n0 + cc + r;
            if (i < a.I && c < a.C) {
              float lo = 0.f;   // the smaller levels first
              if (a.nlev > 2) lo = __uint_as_float(v2[r]);
              if (a.nlev > 1) lo += __uint_as_float(v1[r]);
              out[i * a.C + c] = __uint_as_float(v0[r]) + lo;
            }
          }
        } else {
          uint32_t v0[32], v1[32], v2[32], v3[32];
          tmem_ld16(col, v0);
          tmem_ld16(col + L, v1);
          tmem_ld16(col + 2 * L, v2);
          if (!a.merged) tmem_ld16(col + 3 * L, v3);
          tmem_ld_wait();
          // levels 0 and 1 are exact; add the levels as an unevaluated FP32 pair
          // (hi, lo) with error-free TwoSum steps, scale by 2^(E_c + F_i - 14)
          // and add the pair into the partial; the consumer adds hi + lo
          float2* out2 = reinterpret_cast<float2*>(a.part) + (int64_t)bz * a.I * a.C;
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const int64_t i = (int64_t)n0 + cc + r;
            if (i < a.I && c < a.C) {
              const float l0 = __uint_as_float(v0[r]), l1 = __uint_as_float(v1[r]);
              const float l2 = a.merged ? __uint_as_float(v2[r]) : __uint_as_float(v2[r]) + __uint_as_float(v3[r]);
              const float s = __fadd_rn(l0, l1);
              const float bb = __fsub_rn(s, l0);
              const float e1 = __fadd_rn(__fsub_rn(l0, __fsub_rn(s, bb)), __fsub_rn(l1, bb));
              const float t = __fadd_rn(s, l2);
              const float b2 = __fsub_rn(t, s);
              const float e2 = __fadd_rn(__fsub_rn(s, __fsub_rn(t, b2)), __fsub_rn(l2, b2));
              float lo = __fadd_rn(e1, e2);
              float hi = __fadd_rn(t, lo);
              lo = __fsub_rn(lo, __fsub_rn(hi, t));
              int k = Ec + srowexp[cc + r] - 2 * kSliceBits;
              // 2^k as two exact power-of-two factors; beyond +-250 every FP32
              // result has over- or underflowed already
              k = k < -250 ? -250 : (k > 250 ? 250 : k);
              const float s1 = pow2f(k >> 1), s2 = pow2f(k - (k >> 1));
              hi = hi * s1 * s2;
              lo = lo * s1 * s2;
              if (j > 0) {
                // double-float sum with the earlier segments' pair
                const float2 o = out2[i * a.C + c];
                const float sh = __fadd_rn(o.x, hi);
                const float bv = __fsub_rn(sh, o.x);
                const float eh = __fadd_rn(__fsub_rn(o.x, __fsub_rn(sh, bv)), __fsub_rn(hi, bv));
                const float el = __fadd_rn(eh, __fadd_rn(o.y, lo));
                hi = __fadd_rn(sh, el);
                lo = __fsub_rn(el, __fsub_rn(hi, sh));
              }
              out2[i * a.C + c] = make_float2(hi, lo);
            }
          }
        }
      }
      // this warp's TMEM reads are complete: release the accumulators
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_empty);
      drained = j + 1;
    };

    if (is_producer_warp(warp)) {
    // ---------------- Khatri-Rao producers ------------------------------------------
    const int pw = producer_index(warp);    // 0..kProducerWarps-1
    const int rg = lane / CPR;              // row within a group of RPI rows
    const int q = lane % CPR;               // 16-byte chunk within the row
    // per-row constants, hoisted out of the k loop
    bool cval[RPT];
    float rscale[RPT];
    uint32_t soff[RPT];                                  // swizzled offset in an A tile
    const float* ra[RPT];                                // global rows of UTa (unstaged path)
    const float* ral[RPT];
    const float* rq0[RPT];
    const float* rq0l[RPT];
    const float* rq1[RPT];
    const float* rq1l[RPT];
    int crow[RPT];
    uint32_t ua_row[RPT], ua_rowl[RPT];   // staged rows (shared addresses)
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int m = pw * kRowsPerWarp + rr * RPI + rg;   // row of the A tile = column c0 + m
      const int c = c0 + m;
      cval[rr] = c < a.C;
      const int cc = cval[rr] ? c : 0;
      crow[rr] = cc;
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
    }
    // this thread's column j of the unfolding: j = ia + Ia_pad * o, o mixed-radix
    // over the remaining modes; advanced incrementally by BK per k-step
    const int je32 = (int)je;
    int jcur = (int)jb + q * CHUNK;
    int ia = 0;
    int iq[QM];
    {
      const int o = jcur / a.Ia_pad;
      ia = jcur - o * a.Ia_pad;
      int rem = o;
#pragma unroll
      for (int t = 0; t < QM; ++t) {
        iq[t] = 0;
        if (t < a.nq) {
          const int qq = rem / a.qdims[t];
          iq[t] = rem - qq * a.qdims[t];
          rem = qq;
        }
      }
    }
    // Q(c, o) = prod of the remaining modes' factor entries of row c at the
    // column's indices, as an FP32 pair; it changes only when the column index
    // carries out of mode a.  Raw entries of modes t < 2 are loaded one k-step
    // ahead (pf*), further modes when the product is formed.
    float qhc[RPT], qlc[RPT];
    float pf0[RPT], pf0l[RPT], pf1[RPT], pf1l[RPT];
    auto load_raw = [&](const int (&ix)[QM]) {
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        pf0[rr] = pf1[rr] = 1.f;
        pf0l[rr] = pf1l[rr] = 0.f;
        if (a.nq > 0) {
          pf0[rr] = __ldg(rq0[rr] + ix[0]);
          if constexpr (Cfg::exact) pf0l[rr] = __ldg(rq0l[rr] + ix[0]);
        }
        if (a.nq > 1) {
          pf1[rr] = __ldg(rq1[rr] + ix[1]);
          if constexpr (Cfg::exact) pf1l[rr] = __ldg(rq1l[rr] + ix[1]);
        }
      }
    };
    auto form_q = [&](const int (&ix)[QM]) {
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        float qh = 1.f, ql = 0.f;
        if (a.nq > 0) {
          if constexpr (Cfg::exact) {
            qh = pf0[rr];
            ql = pf0l[rr];
            if (a.nq > 1) pair_mul(qh, ql, pf1[rr], pf1l[rr]);
          } else {
            qh = pf0[rr] * pf1[rr];
          }
#pragma unroll
          for (int t = 2; t < QM; ++t) {
            if (t < a.nq) {
              const int64_t idx = (int64_t)crow[rr] * a.qpad[t] + ix[t];
              const float bh = __ldg(a.UTq[t] + idx);
              if constexpr (Cfg::exact) {
                pair_mul(qh, ql, bh, __ldg(a.UTq_lo[t] + idx));
              } else {
                qh *= bh;
              }
            }
          }
        }
        qhc[rr] = qh;
        qlc[rr] = ql;
      }
    };
    // prologue: the first remaining-mode entries are in flight while the factor
    // rows are staged; the row scales are formed after it
    load_raw(iq);
    if (a.ua_smem) {
      // stage the CTA's 128 factor rows of mode a once (FP32 hi; BF16 lo for
      // the exact form; zero past C): the k loop then reads them from shared
      // memory instead of L2
      constexpr int kStagers = 32 * kProducerWarps;
      constexpr int kU = 4;   // loads in flight per thread
      const int tid = pw * 32 + lane;
      const int n4 = a.Ia_pad / 4;
      for (int idx0 = tid; idx0 < kRowsM * n4; idx0 += kU * kStagers) {
        float4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = idx0 + u * kStagers;
          const int row = idx / n4, col = (idx - row * n4) * 4;
          v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (idx < kRowsM * n4 && c0 + row < a.C)
            v[u] = __ldg(reinterpret_cast<const float4*>(a.UTa + (int64_t)(c0 + row) * a.Ia_pad + col));
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int idx = idx0 + u * kStagers;
          if (idx < kRowsM * n4) {
            const int row = idx / n4, col = (idx - row * n4) * 4;
            sts128(smem_u32(ua_hi + (size_t)row * a.ua_stride + col),
                   make_uint4(__float_as_uint(v[u].x), __float_as_uint(v[u].y), __float_as_uint(v[u].z),
                              __float_as_uint(v[u].w)));
          }
        }
      }
      if constexpr (Cfg::exact) {
        // FP32 low parts rounded to BF16 (the pair then holds U to ~2^-32)
        for (int idx0 = tid; idx0 < kRowsM * n4; idx0 += kU * kStagers) {
          float4 v[kU];
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int idx = idx0 + u * kStagers;
            const int row = idx / n4, col = (idx - row * n4) * 4;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < kRowsM * n4 && c0 + row < a.C)
              v[u] = __ldg(reinterpret_cast<const float4*>(a.UTa_lo + (int64_t)(c0 + row) * a.Ia_pad + col));
          }
#pragma unroll
          for (int u = 0; u < kU; ++u) {
            const int idx = idx0 + u * kStagers;
            if (idx < kRowsM * n4) {
              const int row = idx / n4, col = (idx - row * n4) * 4;
              const __nv_bfloat162 l01 = __floats2bfloat162_rn(v[u].x, v[u].y);
              const __nv_bfloat162 l23 = __floats2bfloat162_rn(v[u].z, v[u].w);
              uint2 pk;
              pk.x = *reinterpret_cast<const uint32_t*>(&l01);
              pk.y = *reinterpret_cast<const uint32_t*>(&l23);
              *reinterpret_cast<uint2*>(ua_lo + (size_t)row * a.Ia_pad + col) = pk;
            }
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"r"(kStagers) : "memory");   // producer warps only
    }
    if constexpr (Cfg::exact) {
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr)
        if (cval[rr]) rscale[rr] = pow2f(7 - bound_exponent_prod(__ldg(a.cmax_a + crow[rr]), a.cmax_q, a.nq, crow[rr]));
    }
    form_q(iq);
    const uint32_t ring_s = smem_u32(ring);
    // The k loop runs in stretches between this warp's drains (a drain of
    // segment j comes after the warp has also filled the first stages of
    // segment j + 1, so the MMA warp resumes without a gap); the drain code
    // stays out of the hot loop.
    const bool drains_here = warp >= kEpilogueWarp0;
    int it = 0;
    int s = 0;          // ring stage of k-step it and the parity of its pass
    uint32_t ph = 0;
    bool pre = false;   // this stage seen released by a probe during the previous k-step
    while (it < nk && ok) {
      int stop = nk;
      if (Cfg::exact && drains_here && drained < nseg - 1) {
        const int end_j = (drained + 1) * seg - 1;
        stop = end_j + S < nk ? end_j + S : nk;   // produce through end_j + S - 1
      }
    for (; it < stop && ok; ++it) {
      // next k-step's indices; on a carry fetch its factor entries now
      int ia_n = ia + BK;
      int iq_n[QM];
#pragma unroll
      for (int t = 0; t < QM; ++t) iq_n[t] = iq[t];
      bool wrap = false;
      while (ia_n >= a.Ia_pad) {
        ia_n -= a.Ia_pad;
        wrap = true;
#pragma unroll
        for (int t = 0; t < QM; ++t) {
          if (t < a.nq) {
            if (++iq_n[t] < a.qdims[t]) break;
            iq_n[t] = 0;
          }
        }
      }
      if (wrap) load_raw(iq_n);
      // The stage is nearly always released already: a probe issued during the
      // previous k-step's work usually answers that, off the critical path;
      // otherwise every lane polls the barrier (no divergent branch, no
      // broadcast); the votes keep the warp's outcome uniform.
      if (!__all_sync(0xffffffffu, pre)) {
        if (!__all_sync(0xffffffffu, wait_bounded(&empty[s], ph ^ 1u, abort_flag, a.err, 4))) {
          ok = false;
          break;
        }
      }
      {
        const bool wrap_s = s + 1 == S;
        pre = mbar_test_wait(&empty[wrap_s ? 0 : s + 1], (wrap_s ? ph ^ 1u : ph) ^ 1u);   // k-step it + 1
      }
      const bool jvalid = jcur < je32;
      const uint32_t a_tile_s = ring_s + (uint32_t)s * stage_bytes;
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr) {
        const bool live = jvalid && cval[rr];
        if constexpr (Cfg::exact) {
          // CHUNK (8) entries: FP32 hi and BF16 lo of the staged (or global) row
          float uh[8], ul[8];
          if (a.ua_smem) {
            const float4 u0 = lds128(ua_row[rr] + (uint32_t)ia * 4u);
            const float4 u1 = lds128(ua_row[rr] + (uint32_t)ia * 4u + 16u);
            const float4 lraw = lds128(ua_rowl[rr] + (uint32_t)ia * 2u);
            uh[0] = u0.x; uh[1] = u0.y; uh[2] = u0.z; uh[3] = u0.w;
            uh[4] = u1.x; uh[5] = u1.y; uh[6] = u1.z; uh[7] = u1.w;
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
            const float4 u0 = __ldg(src), u1 = __ldg(src + 1), l0 = __ldg(srcl), l1 = __ldg(srcl + 1);
            uh[0] = u0.x; uh[1] = u0.y; uh[2] = u0.z; uh[3] = u0.w;
            uh[4] = u1.x; uh[5] = u1.y; uh[6] = u1.z; uh[7] = u1.w;
            ul[0] = l0.x; ul[1] = l0.y; ul[2] = l0.z; ul[3] = l0.w;
            ul[4] = l1.x; ul[5] = l1.y; ul[6] = l1.z; ul[7] = l1.w;
          }
          // the row's power of two folded into Q (exact)
          const float qh = live ? qhc[rr] * rscale[rr] : 0.f, ql = live ? qlc[rr] * rscale[rr] : 0.f;
          const f2 qh2 = f2_pack(qh, qh), nqh2 = f2_pack(-qh, -qh), ql2 = f2_pack(ql, ql);
          uint32_t w[4][4];   // [slice][pair]
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uint32_t ws[4];
            exact_slices2(f2_pack(uh[2 * e], uh[2 * e + 1]), f2_pack(ul[2 * e], ul[2 * e + 1]), qh2, nqh2, ql2, ws);
#pragma unroll
            for (int p = 0; p < 4; ++p) w[p][e] = ws[p];
          }
#pragma unroll
          for (int p = 0; p < 4; ++p)
            sts128(a_tile_s + (uint32_t)p * a_bytes + soff[rr], make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]));
        } else {
          float v[CHUNK];
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) v[e] = 0.f;
          if (live) {
            const float qh = qhc[rr];
            const float4* src = reinterpret_cast<const float4*>(ra[rr] + ia);
#pragma unroll
            for (int e4 = 0; e4 < CHUNK / 4; ++e4) {
              const float4 u = a.ua_smem ? lds128(ua_row[rr] + (uint32_t)(ia + 4 * e4) * 4u) : __ldg(src + e4);
              v[4 * e4 + 0] = u.x * qh;
              v[4 * e4 + 1] = u.y * qh;
              v[4 * e4 + 2] = u.z * qh;
              v[4 * e4 + 3] = u.w * qh;
            }
          }
          float parts[NS][CHUNK];
#pragma unroll
          for (int e = 0; e < CHUNK; ++e) {
            float p4[4];
            split_value<Cfg>(v[e], p4);
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
      }
      fence_async_shared();   // each writer: generic-proxy stores -> visible to the MMA
      __syncwarp();
      mbar_arrive_lane0(&full[s], lane);
      if (wrap) form_q(iq_n);
      jcur += BK;
      ia = ia_n;
#pragma unroll
      for (int t = 0; t < QM; ++t) iq[t] = iq_n[t];
      if (++s == S) {
        s = 0;
        ph ^= 1u;
      }
    }
      if (Cfg::exact && drains_here && drained < nseg - 1 && it == stop && ok) drain_segment(drained);
    }

    }   // producers

    if (warp >= kEpilogueWarp0) {
      // segments not drained inside the producer loop
      for (int j = drained; j < nseg; ++j) drain_segment(j);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
  }
}

template <class Cfg, int QM>
__global__ void __launch_bounds__(kThreads, 1) mttkrp_tc_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  mttkrp_tc_body<Cfg, QM>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

// Several problems' MTTKRPs of one mode in one launch: CTA x belongs to the
// problem b with first[b] <= x < first[b + 1] and is CTA (x - first[b]) of that
// problem's own grid (C tiles fastest, then N tiles, then splits).  The
// problem's arguments are copied into shared memory once per CTA.
__device__ __forceinline__ int group_problem(const int* first, int nprob, int x) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(first + mid) <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class Cfg, int QM>
__global__ void __launch_bounds__(kThreads, 1) mttkrp_tc_grouped_kernel(const TcArgs* __restrict__ args,
                                                                        const int* __restrict__ first, int nprob) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(16) TcArgs sa;
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int b = group_problem(first, nprob, (int)blockIdx.x);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(args + b);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sa);
    for (int i = threadIdx.x; i < (int)(sizeof(TcArgs) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const int local = (int)blockIdx.x - __ldg(first + b);
  const int gx = sa.tiles_c, gy = sa.tiles_n;
  mttkrp_tc_body<Cfg, QM>(sa, local % gx, (local / gx) % gy, local / (gx * gy), smem);
}

// ---- precision forms -----------------------------------------------------------
// nsplit parts per operand; the products of parts s, t with s + t < nsplit are
// taken (TF32 / BF16: one; 3xTF32: hh, hl, lh; BF16x3: six; exact: ten).

struct CfgTF32 {
  static constexpr int fmt = 2;   // A/B format: TF32 2, BF16 1
  static constexpr int kind = kKindTF32, nsplit = 1, row_bytes = 128, elem = 4;
  static constexpr bool exact = false;
};
struct Cfg3xTF32 {
  static constexpr int fmt = 2;   // A/B format: TF32 2, BF16 1
  static constexpr int kind = kKindTF32, nsplit = 2, row_bytes = 128, elem = 4;
  static constexpr bool exact = false;
};
struct CfgBF16 {
  static constexpr int fmt = 1;   // A/B format: TF32 2, BF16 1
  static constexpr int kind = kKindBF16, nsplit = 1, row_bytes = 128, elem = 2;
  static constexpr bool exact = false;
};
struct CfgBF16x3 {
  static constexpr int fmt = 1;   // A/B format: TF32 2, BF16 1
  static constexpr int kind = kKindBF16, nsplit = 3, row_bytes = 128, elem = 2;
  static constexpr bool exact = false;
};
struct CfgExact {
  static constexpr int fmt = 1;   // A/B format: TF32 2, BF16 1
  static constexpr int kind = kKindBF16, nsplit = 4, row_bytes = 64, elem = 2;
  static constexpr bool exact = true;
};

// ---- two-step exact form ----------------------------------------------------------
// For a mode whose rows fit one narrow N tile (BN <= 64) each Khatri-Rao entry would
// be reused only BN times, so building the KRP bounds the kernel.  Instead, with a
// the largest other mode and o the index of the remaining ones,
//   Mbar_n^T(c, i) = sum_o Q(c, o) Y_o(c, i),   Y_o = U_a^T (C x I_a) . T_(n)(:, o)^T,
// Q(c, o) the product of the remaining modes' factor entries of column c (the
// Khatri-Rao factorisation of Eq. MTTKRP taken one mode at a time).  Each Y_o is
// one exact-chain GEMM over I_a <= 1024 columns: A = U_a^T sliced like T (4 BF16
// slices on the row's power-of-two grid, sliced once per launch into stage
// images read by TMA), B = the pre-tiled unfolding as for the other forms.  The
// epilogue warps drain each o's accumulators (double-buffered in TMEM, so the
// next o accumulates meanwhile), combine the levels into an FP32 pair, multiply
// by Q(c, o) as an FP32 pair (error-free products) and add into per-thread
// double-float sums; the column powers of two are applied once at the end.

// exponent E with max |U_a(:, c)| < 2^E (0 for an all-zero column)
__device__ __forceinline__ int col_exponent(float cmax) {
  if (!(cmax > 0.f)) return 0;
  int e;
  frexpf(cmax, &e);
  return e < -110 ? -110 : (e > 110 ? 110 : e);
}

// A stage images of U_a^T: for 128-row tile tc and k-step ks (columns ia in
// [32 ks, 32 ks + 32) of the padded mode a), 4 parts of 128 rows x 64 bytes in
// the 64-byte swizzle, the layout the producers of the one-step form write.
__global__ void slice_a_kernel(const float* __restrict__ UT, const float* __restrict__ UT_lo, int64_t ut_stride,
                               int Ia, int Ia_pad, const float* __restrict__ cmax, int C, int tiles_c,
                               unsigned char* __restrict__ At) {
  constexpr int ROW = CfgExact::row_bytes, BK = ROW / 2;
  const int chunks = Ia_pad / 8;
  const int nkt_a = Ia_pad / BK;
  const int64_t total = (int64_t)tiles_c * kRowsM * chunks;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / chunks);
    const int ch = (int)(e - (int64_t)c * chunks);
    const int ia0 = ch * 8;
    float uh[8], ul[8];
    float sc = 0.f;
    if (c < C) sc = pow2f(kSliceBits - col_exponent(__ldg(cmax + c)));
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const bool in = c < C && ia0 + k < Ia;
      uh[k] = in ? __ldg(UT + (int64_t)c * ut_stride + ia0 + k) : 0.f;
      ul[k] = in ? __ldg(UT_lo + (int64_t)c * ut_stride + ia0 + k) : 0.f;
    }
    const f2 s2 = f2_pack(sc, sc), ns2 = f2_pack(-sc, -sc), z2 = f2_pack(0.f, 0.f);
    uint32_t w[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      uint32_t ws[4];
      exact_slices2(f2_pack(uh[2 * p], uh[2 * p + 1]), f2_pack(ul[2 * p], ul[2 * p + 1]), s2, ns2, z2, ws);
#pragma unroll
      for (int t = 0; t < 4; ++t) w[t][p] = ws[t];
    }
    const int tc = c / kRowsM, m = c - tc * kRowsM, ks = ia0 / BK, q = (ia0 - ks * BK) / 8;
    unsigned char* img = At + ((int64_t)tc * nkt_a + ks) * 4 * (kRowsM * ROW);
    const uint32_t off = (uint32_t)(m >> 3) * (8u * ROW) + (uint32_t)(m & 7) * ROW + (uint32_t)((q ^ ((m >> 1) & 3)) << 4);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      *reinterpret_cast<uint4*>(img + t * (kRowsM * ROW) + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
  }
}

// k-steps issued per trip through the two-step kernel's issue loop at most
constexpr int kTtsUnroll = 4;

// VAR: the B parts stacked per MMA (4, 2 or 1; from the plan's stack), fixed at
// compile time: a runtime switch over the variants costs the issuing lane about
// 50 cycles per stage, where a stage has ~700 cycles of tensor work.
template <int QM, int VAR>
__global__ void __launch_bounds__(kThreads, 1) mttkrp_tts_kernel(const TcArgs a) {
  using Cfg = CfgExact;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int NS = Cfg::nsplit;
  constexpr int ROW = Cfg::row_bytes;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t a_bytes = kRowsM * ROW;
  const uint32_t b_bytes = (uint32_t)a.BN * ROW;
  const uint32_t a_stage = NS * a_bytes, b_stage = NS * b_bytes;
  const uint32_t stage_bytes = a_stage + b_stage;   // a multiple of 1024
  const int S = a.stages;
  unsigned char* ring = smem;
  uint64_t* bars = reinterpret_cast<uint64_t*>(ring + (size_t)S * stage_bytes);
  uint64_t* full = bars;                  // stage loaded (the TMA arrival and its bytes)
  uint64_t* empty = bars + S;             // stage consumed (the MMAs' commit)
  uint64_t* accum = bars + 2 * S;         // [2] one o's MMAs complete in accumulator set b
  uint64_t* tmem_empty = accum + 2;       // [2] the epilogue warps drained set b
  uint64_t* drain = accum + 4;            // [2] abort path: issuer e's MMAs so far are complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* srowexp = const_cast<int*>(abort_flag + 1);   // BN row exponents of this N tile

  const int c0 = blockIdx.x * kRowsM;
  const int n0 = blockIdx.y * a.BN;
  const int o0 = blockIdx.z * a.o_per_cta;
  const int o1 = o0 + a.o_per_cta < a.n_o ? o0 + a.o_per_cta : a.n_o;
  const int nseg = o1 > o0 ? o1 - o0 : 0;
  const int nkt_a = a.nkt_a;
  const int nbuf = a.nbuf;
  // nis MMA issuers (1 or 2): issuer e (warp 1 + e) takes the CTA's o's
  // j = e, e + nis, ... through its own S / nis ring stages; o j accumulates in
  // set j % nbuf.  With two issuers the tensor pipe runs one issuer's MMAs while
  // the other commits, waits for its next stage or starts its next o.
  const int nis = a.nis;
  const int Sh = S / nis;
  const uint32_t set_cols = (uint32_t)(a.nlev * a.lstride);   // columns of one accumulator set

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&accum[0], 1);
    mbar_init(&accum[1], 1);
    mbar_init(&tmem_empty[0], kEpilogueWarps);
    mbar_init(&tmem_empty[1], kEpilogueWarps);
    mbar_init(&drain[0], 1);
    mbar_init(&drain[1], 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, (uint32_t)a.tmem_cols);
  if ((int)threadIdx.x < a.BN) {
    const int64_t i = (int64_t)n0 + threadIdx.x;
    srowexp[threadIdx.x] = i < a.I ? __ldg(a.rowexp + i) : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && nis == 1) {
    // ---------------- TMA: one lane refills the ring in order --------------------
    // k-step it of the CTA (o = it / nkt_a, k-step kk within it) goes to stage
    // it mod S.  One lane in order, rather than lane s for stage s: diverged
    // lanes of one warp blocked in their own barrier waits delay each other's
    // refills.
    if (lane == 0) {
      const int nke = nseg * nkt_a;
      int issued = 0;
      const unsigned char* srcb = a.Tt + ((int64_t)blockIdx.y * a.nkt + (int64_t)o0 * nkt_a) * (int64_t)b_stage;
      const unsigned char* srca = a.At + (int64_t)blockIdx.x * nkt_a * (int64_t)a_stage;
      int s = 0, kk = 0;
      uint32_t ph = 0;
      for (int it = 0; it < nke; ++it) {
        if (!wait_bounded(&empty[s], ph ^ 1u, abort_flag, a.err, 1)) break;
        unsigned char* dst = ring + (size_t)s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], a_stage + b_stage);
        bulk_load(dst, srca + (int64_t)kk * a_stage, a_stage, &full[s]);
        bulk_load(dst + a_stage, srcb + (int64_t)it * b_stage, b_stage, &full[s]);
        issued = it + 1;
        if (++kk == nkt_a) kk = 0;
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (*abort_flag && issued > 0) {
        const uint64_t t0 = global_ns();
        while (global_ns() - t0 < 200000ull) {
        }
      }
    }
  } else if (warp == 0) {
    // ---------------- TMA (two issuers): lane s loads ring stage s -----------------
    // Stage s belongs to issuer e = s / Sh; it carries that issuer's k-steps
    // it = s - e Sh, + Sh, ... (k-step kk of its o number it / nkt_a).
    if (lane < S) {
      const int e = lane / Sh;
      const int ne = nseg > e ? (nseg - e + nis - 1) / nis : 0;   // o's of issuer e
      const int nke = ne * nkt_a;
      int issued = 0;
      const unsigned char* srcb = a.Tt + ((int64_t)blockIdx.y * a.nkt + (int64_t)o0 * nkt_a) * (int64_t)b_stage;
      const unsigned char* srca = a.At + (int64_t)blockIdx.x * nkt_a * (int64_t)a_stage;
      unsigned char* dst = ring + (size_t)lane * stage_bytes;
      uint32_t ph = 0;
      for (int it = lane - e * Sh; it < nke; it += Sh, ph ^= 1u) {
        const int jj = it / nkt_a;
        const int kk = it - jj * nkt_a;
        const int j = e + jj * nis;   // o of the CTA
        if (!wait_bounded(&empty[lane], ph ^ 1u, abort_flag, a.err, 1)) break;
        mbar_arrive_expect_tx(&full[lane], a_stage + b_stage);
        bulk_load(dst, srca + (int64_t)kk * a_stage, a_stage, &full[lane]);
        bulk_load(dst + a_stage, srcb + ((int64_t)j * nkt_a + kk) * b_stage, b_stage, &full[lane]);
        issued = it + 1;
      }
      if (*abort_flag && issued > 0) {
        const uint64_t t0 = global_ns();
        while (global_ns() - t0 < 200000ull) {
        }
      }
    }
  } else if (warp == 1 || (warp == 2 && nis == 2)) {
    // ---------------- MMA issuers ---------------------------------------------------
    if (lane == 0) {
      const int e = warp - 1;
      const int ne = nseg > e ? (nseg - e + nis - 1) / nis : 0;
      const int nke = ne * nkt_a;
      const uint64_t desc0 = smem_desc<ROW>(smem_u32(ring));
      const uint32_t L = (uint32_t)a.lstride, b16 = b_bytes >> 4;
      uint32_t idesc[5];
#pragma unroll
      for (int c = 0; c < 5; ++c)
        idesc[c] = (1u << 4) | ((uint32_t)Cfg::fmt << 7) | ((uint32_t)Cfg::fmt << 10) |
                   (((uint32_t)(c * a.BN) >> 3) << 17) | ((uint32_t)(kRowsM >> 4) << 24);
      bool ok = true;
      int jj = 0, kin = 0;   // this issuer's o and the k-step within it
      int j = e, b = e % nbuf;   // o of the CTA and its accumulator set
      int sp = 0;            // stage within this issuer's ring, and the parity of its pass
      uint32_t ph = 0;
      for (int it = 0; it < nke && ok; ++it) {
        if (kin == 0 && j >= nbuf) {
          // set b is refilled once the epilogue drained its previous o (o j - nbuf,
          // the set's (j / nbuf)-th use)
          ok = wait_bounded(&tmem_empty[b], (uint32_t)(j / nbuf - 1) & 1u, abort_flag, a.err, 7);
          if (!ok) break;
        }
        const uint32_t td = tmem + (uint32_t)b * set_cols;
        const int st = e * Sh + sp;
        ok = wait_bounded(&full[st], ph, abort_flag, a.err, 2);
        if (!ok) break;
        tc_fence_after();
        const uint64_t ad0 = desc0 + (uint64_t)(((uint32_t)st * stage_bytes) >> 4);
        const uint64_t bd0 = ad0 + (uint64_t)(a_stage >> 4);
        issue_stage<Cfg, VAR, false, ROW / 32>(td, ad0, bd0, L, b16, idesc, kin == 0);
        tc_commit(&empty[st]);
        // the following k-steps of the same o in the following stages of the same
        // pass, up to the whole ring, in the same trip through the loop (each stage
        // still released by its own commit right after its MMAs)
#pragma unroll
        for (int u = 1; u < kTtsUnroll; ++u) {
          if (!(kin + 1 < nkt_a && sp + 1 < Sh && it + 1 < nke)) break;
          ++it;
          ++kin;
          ++sp;
          ok = wait_bounded(&full[st + u], ph, abort_flag, a.err, 2);
          if (!ok) break;
          tc_fence_after();
          const uint64_t stu = (uint64_t)(((uint32_t)u * stage_bytes) >> 4);
          issue_stage<Cfg, VAR, false, ROW / 32>(td, ad0 + stu, bd0 + stu, L, b16, idesc, false);
          tc_commit(&empty[st + u]);
        }
        if (++kin == nkt_a) {
          tc_commit(&accum[b]);   // o j complete in set b
          kin = 0;
          ++jj;
          j += nis;
          b = j % nbuf;
        }
        if (++sp == Sh) {
          sp = 0;
          ph ^= 1u;
        }
      }
      if (!ok) {
        tc_commit(&drain[e]);
        wait_drain(&drain[e], 0);
      }
    }
  } else if (warp >= kEpilogueWarp0) {
    // ---------------- epilogue: per o, scale by Q(c, o) and accumulate ---------------
    const int quarter = warp & 3;                   // TMEM lanes 32 quarter .. + 31
    const int grp = (warp - kEpilogueWarp0) >> 2;   // two warps per quarter split the columns
    const int m_e = quarter * 32 + lane;
    const int c = c0 + m_e;
    const bool cv = c < a.C;
    const int cc_ = cv ? c : 0;
    const int Ec = cv ? col_exponent(__ldg(a.cmax_a + c)) : 0;
    const float rsc = pow2f(Ec - 2 * kSliceBits);   // 2^(E_c - 14): the row part of the level scale
    // Q(c, o) as an FP32 pair, times rsc (exact)
    auto load_q = [&](int o, float& qh, float& ql) {
      qh = rsc;
      ql = 0.f;
      int rem = o;
#pragma unroll
      for (int t = 0; t < QM; ++t) {
        if (t < a.nq) {
          const int qq = rem / a.qdims[t];
          const int idx = rem - qq * a.qdims[t];
          rem = qq;
          const int64_t off = (int64_t)cc_ * a.qpad[t] + idx;
          pair_mul(qh, ql, __ldg(a.UTq[t] + off), __ldg(a.UTq_lo[t] + off));
        }
      }
    };
    // this warp's columns: 16-column slices cc = 16 grp + 32 k (BN <= 64: at most 2),
    // as 16 pairs of adjacent rows in packed FP32x2 registers: every step below is
    // the same round-to-nearest operation per lane as the scalar formulas
    f2 acc_h[16], acc_l[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) acc_h[r] = acc_l[r] = f2_pack(0.f, 0.f);
    const f2 m1 = f2_pack(-1.f, -1.f);
    bool ok = true;
    float qh = 0.f, ql = 0.f;
    if (nseg > 0) load_q(o0, qh, ql);
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t L = (uint32_t)a.lstride;
    int b = 0;
    uint32_t uses0 = 0, uses1 = 0;   // drains of each accumulator set so far
    for (int j = 0; j < nseg; ++j) {
      bool have = ok && wait_sleepy(&accum[b], (b ? uses1 : uses0) & 1u, abort_flag, a.err, 5);
      have = __all_sync(0xffffffffu, have);
      if (!have) {
        ok = false;
        break;
      }
      tc_fence_after();
      float qhn = 0.f, qln = 0.f;
      if (j + 1 < nseg) load_q(o0 + j + 1, qhn, qln);   // in flight during this drain
      const f2 qh2 = f2_pack(qh, qh), ql2 = f2_pack(ql, ql);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int cc = 16 * grp + 32 * k;
        if (cc < a.BN) {
          uint32_t v0[32], v1[32], v2[32], v3[32];
          const uint32_t col = lane_base + (uint32_t)b * set_cols + (uint32_t)cc;
          tmem_ld16(col, v0);
          tmem_ld16(col + L, v1);
          tmem_ld16(col + 2 * L, v2);
          tmem_ld16(col + 3 * L, v3);
          tmem_ld_wait();
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            // levels as an FP32 pair (TwoSum; levels 0 and 1 exact, 2 and 3 small)
            const f2 l0 = f2_pack(__uint_as_float(v0[2 * r]), __uint_as_float(v0[2 * r + 1]));
            const f2 l1 = f2_pack(__uint_as_float(v1[2 * r]), __uint_as_float(v1[2 * r + 1]));
            const f2 l2 = f2_add(f2_pack(__uint_as_float(v2[2 * r]), __uint_as_float(v2[2 * r + 1])),
                                 f2_pack(__uint_as_float(v3[2 * r]), __uint_as_float(v3[2 * r + 1])));
            const f2 s_ = f2_add(l0, l1);
            const f2 bb = f2_sub(s_, l0);
            const f2 e1 = f2_add(f2_sub(l0, f2_sub(s_, bb)), f2_sub(l1, bb));
            const f2 t = f2_add(s_, l2);
            const f2 b2 = f2_sub(t, s_);
            const f2 e2 = f2_add(f2_sub(s_, f2_sub(t, b2)), f2_sub(l2, b2));
            const f2 lo0 = f2_add(e1, e2);
            const f2 hi = f2_add(t, lo0);
            const f2 lo = f2_sub(lo0, f2_sub(hi, t));
            // times Q (pair): error-free leading product, cross terms
            const f2 p = f2_mul(hi, qh2);
            const f2 pe = f2_fma(lo, qh2, f2_fma(hi, ql2, f2_fma(hi, qh2, f2_mul(p, m1))));
            // accumulate (double-float)
            const int idx = 8 * k + r;
            const f2 sh = f2_add(acc_h[idx], p);
            const f2 bv = f2_sub(sh, acc_h[idx]);
            const f2 eh = f2_add(f2_sub(acc_h[idx], f2_sub(sh, bv)), f2_sub(p, bv));
            const f2 el = f2_add(eh, f2_add(acc_l[idx], pe));
            acc_h[idx] = f2_add(sh, el);
            acc_l[idx] = f2_sub(el, f2_sub(acc_h[idx], sh));
          }
        }
      }
      // this warp's TMEM reads are complete: release set b
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tmem_empty[b]);
      if (b) ++uses1; else ++uses0;
      b = (nbuf == 2) ? b ^ 1 : 0;
      qh = qhn;
      ql = qln;
    }
    // the column powers of two, then this split's partial (the consumer adds hi + lo)
    float2* out2 = reinterpret_cast<float2*>(a.part) + (int64_t)blockIdx.z * a.I * a.C;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int cc = 16 * grp + 32 * k;
      if (cc < a.BN) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int64_t i = (int64_t)n0 + cc + r;
          if (i < a.I && cv) {
            int kx = srowexp[cc + r];
            kx = kx < -120 ? -120 : (kx > 120 ? 120 : kx);
            const float sx = pow2f(kx);
            float ah0, ah1, al0, al1;
            f2_unpack(acc_h[8 * k + (r >> 1)], ah0, ah1);
            f2_unpack(acc_l[8 * k + (r >> 1)], al0, al1);
            const float ah = (r & 1) ? ah1 : ah0, al = (r & 1) ? al1 : al0;
            out2[i * a.C + c] = ok ? make_float2(ah * sx, al * sx) : make_float2(0.f, 0.f);
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

// The limit is per kernel and process-wide: only ever raise it, so that a
// handle needing less never lowers it under another handle.
template <class Cfg, int QM>
cudaError_t set_smem_cfg1(size_t smem) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, mttkrp_tc_kernel<Cfg, QM>);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(mttkrp_tc_kernel<Cfg, QM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <class Cfg>
cudaError_t set_smem_cfg(size_t smem) {
  const cudaError_t e = set_smem_cfg1<Cfg, 2>(smem);
  if (e != cudaSuccess) return e;
  return set_smem_cfg1<Cfg, kMaxModes - 2>(smem);
}

template <int QM, int VAR>
cudaError_t set_smem_tts2(size_t smem) {
  cudaFuncAttributes fa;
  const cudaError_t e = cudaFuncGetAttributes(&fa, mttkrp_tts_kernel<QM, VAR>);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  return cudaFuncSetAttribute(mttkrp_tts_kernel<QM, VAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int QM>
cudaError_t set_smem_tts1(size_t smem) {
  cudaError_t e = set_smem_tts2<QM, 4>(smem);
  if (e == cudaSuccess) e = set_smem_tts2<QM, 2>(smem);
  if (e == cudaSuccess) e = set_smem_tts2<QM, 1>(smem);
  return e;
}

// stacking variant of the two-step kernel for a plan's stack (issue_stage's G)
inline int tts_variant(int stack) { return stack >= 4 ? 4 : (stack == 2 ? 2 : 1); }

template <int QM>
void launch_tts_qm(dim3 grid, size_t smem, cudaStream_t s, const TcArgs& a) {
  switch (tts_variant(a.stack)) {
    case 4: mttkrp_tts_kernel<QM, 4><<<grid, kThreads, smem, s>>>(a); break;
    case 2: mttkrp_tts_kernel<QM, 2><<<grid, kThreads, smem, s>>>(a); break;
    default: mttkrp_tts_kernel<QM, 1><<<grid, kThreads, smem, s>>>(a); break;
  }
}

cudaError_t launch_tts(const TcPlan& p, const TcArgs& a, cudaStream_t s) {
  // slice U_a^T into the A stage images (unless they are current), then the
  // two-step GEMMs
  if (!a.skip_slice) {
    const int64_t work = (int64_t)p.tiles_c * kRowsM * (p.Ia_pad / 8);
    int64_t blocks = (work + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    slice_a_kernel<<<(unsigned)blocks, 256, 0, s>>>(a.UTa, a.UTa_lo, a.ut_stride_a, a.Ia, p.Ia_pad, a.cmax_a, a.C,
                                                    p.tiles_c, const_cast<unsigned char*>(a.At));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = tc_smem_bytes(p);
  dim3 grid((unsigned)p.tiles_c, (unsigned)p.tiles_n, (unsigned)p.splits);
  if (a.nq <= 2)
    launch_tts_qm<2>(grid, smem, s, a);
  else
    launch_tts_qm<kMaxModes - 2>(grid, smem, s, a);
  return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_cfg(const TcPlan& p, const TcArgs& a, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(p);
  dim3 grid((unsigned)p.tiles_c, (unsigned)p.tiles_n, (unsigned)p.splits);
  if (a.nq <= 2)
    mttkrp_tc_kernel<Cfg, 2><<<grid, kThreads, smem, s>>>(a);
  else
    mttkrp_tc_kernel<Cfg, kMaxModes - 2><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Cfg>
cudaError_t grouped_cfg(bool prepare, const TcArgs* args, const int* first, int nprob, int total, bool qm_small,
                        size_t smem, cudaStream_t s) {
  if (prepare) {
    // the limit is per kernel and process-wide: only ever raise it
    auto kern = qm_small ? mttkrp_tc_grouped_kernel<Cfg, 2> : mttkrp_tc_grouped_kernel<Cfg, kMaxModes - 2>;
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (qm_small)
    mttkrp_tc_grouped_kernel<Cfg, 2><<<(unsigned)total, kThreads, smem, s>>>(args, first, nprob);
  else
    mttkrp_tc_grouped_kernel<Cfg, kMaxModes - 2><<<(unsigned)total, kThreads, smem, s>>>(args, first, nprob);
  return cudaGetLastError();
}

cudaError_t grouped_dispatch(int precision, bool prepare, const TcArgs* args, const int* first, int nprob, int total,
                             bool qm_small, size_t smem, cudaStream_t s) {
  switch (precision) {
    case JKCALS_TF32: return grouped_cfg<CfgTF32>(prepare, args, first, nprob, total, qm_small, smem, s);
    case JKCALS_3XTF32: return grouped_cfg<Cfg3xTF32>(prepare, args, first, nprob, total, qm_small, smem, s);
    case JKCALS_BF16: return grouped_cfg<CfgBF16>(prepare, args, first, nprob, total, qm_small, smem, s);
    case JKCALS_SPLIT_BF16: return grouped_cfg<CfgBF16x3>(prepare, args, first, nprob, total, qm_small, smem, s);
    case JKCALS_EXACT_BF16: return grouped_cfg<CfgExact>(prepare, args, first, nprob, total, qm_small, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t prepare_mttkrp_tc_grouped(int precision, bool qm_small, size_t smem) {
  return grouped_dispatch(precision, true, nullptr, nullptr, 0, 0, qm_small, smem, nullptr);
}

cudaError_t launch_mttkrp_tc_grouped(int precision, const TcArgs* args, const int* first, int nprob, int total,
                                     bool qm_small, size_t smem, cudaStream_t s) {
  return grouped_dispatch(precision, false, args, first, nprob, total, qm_small, smem, s);
}

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
  const int p = form_nsplit(precision);
  return p * (p + 1) / 2;
}

int build_mma_list(int precision, TcPlan& p) {
  const int P = p.nsplit;
  const uint32_t fmt = (precision == JKCALS_TF32 || precision == JKCALS_3XTF32) ? 2u : 1u;   // TF32 : BF16
  p.lstride = (p.BN + 31) / 32 * 32;
  p.nlev = P;
  p.merged = 0;
  if (P * p.lstride > 512) {
    // exact form with BN > 128: levels 2 and 3 share one accumulator
    if (precision != JKCALS_EXACT_BF16 || 3 * p.lstride > 512) return JKCALS_ERR_UNSUPPORTED;
    p.merged = 1;
  }
  const int nacc = p.merged ? 3 : P;
  p.tmem_cols = 32;
  while (p.tmem_cols < nacc * p.lstride) p.tmem_cols *= 2;
  // parts stack along N when each level starts right where the previous ends
  const int G = (!p.merged && p.lstride == p.BN) ? 256 / p.BN : 1;
  p.stack = G >= 4 ? 4 : G;
  const uint32_t a_bytes = (uint32_t)kRowsM * p.row_bytes, b_bytes = (uint32_t)p.BN * p.row_bytes;
  auto level = [&](int l) { return l > nacc - 1 ? nacc - 1 : l; };
  MmaList& L = p.mma;
  L.n = 0;
  L.first = 0;
  uint32_t started = 0;   // accumulators written by an earlier MMA of the list
  for (int s = 0; s < P; ++s) {
    for (int t0 = 0; t0 < P - s; t0 += G) {
      const int t1 = (t0 + G - 1 < P - 1 - s) ? t0 + G - 1 : P - 1 - s;
      const uint32_t N = (uint32_t)(t1 - t0 + 1) * (uint32_t)p.BN;
      const int m = L.n++;
      L.a[m] = ((uint32_t)s * a_bytes) >> 4;
      L.b[m] = ((uint32_t)t0 * b_bytes) >> 4;
      L.d[m] = (uint32_t)level(s + t0) * (uint32_t)p.lstride;
      // FP32 accumulator, A/B formats, both K-major, N >> 3, M >> 4
      L.idesc[m] = (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((uint32_t)(kRowsM >> 4) << 24);
      // on the first K slice an MMA overwrites its columns iff none is started
      bool fresh = true;
      for (int t = t0; t <= t1; ++t)
        if (started & (1u << level(s + t))) fresh = false;
      if (fresh) L.first |= 1u << m;
      for (int t = t0; t <= t1; ++t) started |= 1u << level(s + t);
    }
  }
  return JKCALS_OK;
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
  if (p.tts)   // ring | barriers (2 S + 6) | TMEM slot, abort word | row exponents
    return 1024 + (size_t)p.stages * (a_stage + b_stage) + (2 * p.stages + 6) * 8 + 16 + 4 * (size_t)p.BN;
  return 1024 /*alignment slack*/ + (size_t)p.stages * (a_stage + b_stage) + tc_ua_bytes(p) + (2 * p.stages + 3) * 8 +
         16 + 4 * (size_t)p.BN;
}

size_t tts_a_bytes(const TcPlan& p) {
  if (!p.tts) return 0;
  return (size_t)p.tiles_c * p.nkt_a * p.nsplit * kRowsM * p.row_bytes;
}

cudaError_t prepare_mttkrp_tc(int precision, size_t max_smem) {
  switch (precision) {
    case JKCALS_TF32: return set_smem_cfg<CfgTF32>(max_smem);
    case JKCALS_3XTF32: return set_smem_cfg<Cfg3xTF32>(max_smem);
    case JKCALS_BF16: return set_smem_cfg<CfgBF16>(max_smem);
    case JKCALS_SPLIT_BF16: return set_smem_cfg<CfgBF16x3>(max_smem);
    case JKCALS_EXACT_BF16: {
      const cudaError_t e = set_smem_cfg<CfgExact>(max_smem);
      if (e != cudaSuccess) return e;
      const cudaError_t e2 = set_smem_tts1<2>(max_smem);
      if (e2 != cudaSuccess) return e2;
      return set_smem_tts1<kMaxModes - 2>(max_smem);
    }
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_mttkrp_tc(int precision, const TcPlan& p, const TcArgs& a, cudaStream_t s) {
  switch (precision) {
    case JKCALS_TF32: return launch_cfg<CfgTF32>(p, a, s);
    case JKCALS_3XTF32: return launch_cfg<Cfg3xTF32>(p, a, s);
    case JKCALS_BF16: return launch_cfg<CfgBF16>(p, a, s);
    case JKCALS_SPLIT_BF16: return launch_cfg<CfgBF16x3>(p, a, s);
    case JKCALS_EXACT_BF16: return p.tts ? launch_tts(p, a, s) : launch_cfg<CfgExact>(p, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tc
}  // namespace jk
