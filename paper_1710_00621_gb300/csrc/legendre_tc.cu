// Legendre synthesis on the fifth-generation tensor cores (tcgen05, TF32 inputs,
// FP32 accumulation in tensor memory).
//
// Per m and ring pair the synthesis F_m(theta) = sum_l lambda_lm(theta) a_lm (Sec. 2.1)
// is, for a tile of 128 ring pairs, the product D[pair][col] = sum_l Lambda[pair][l] B[l][col]
// with B[l][parity(l - m) * 8 + part] = a_lm part (real / imaginary of each map), so that
// columns 0..7 accumulate the even sums E and 8..15 the odd sums O of every map, and
// F_north = E + O, F_south = E - O.
//
// * Lambda is generated on the fly by the recurrence of legendre.cu (one thread per ring
//   pair, start values injected at the pair's first significant l), rounded to TF32 and
//   written by each thread into its own lane of tensor memory (tcgen05.st), so the A operand
//   of the MMA never passes through shared memory;
// * B (the block's coefficients, 16 x 32 TF32) is written to shared memory in the
//   K-major core-matrix layout and described by a shared-memory descriptor;
// * blocks of 32 values of l alternate between two shared-memory stages of B; one thread
//   issues the MMAs (M = 128, N = 16, K = 8) and commits them to the block's mbarrier; the A
//   operand (TF32) has one tensor-memory buffer, which the threads overwrite after a bounded
//   wait for the previous block's MMAs, placed after the block's recurrence so that those
//   MMAs run during it (64 tensor-memory columns per CTA: 8 CTAs per SM; BF16 packs two values
//   of l per column and keeps two buffers in the same 64);
// * SPLIT = 1 keeps FP32-level accuracy with the split-TF32 product
//   A_hi B_hi + A_hi B_lo + A_lo B_hi (x = hi + lo, hi = tf32(x), lo = tf32(x - hi));
// * BF = 1 takes BF16 operands instead (kind::f16, K = 16 per MMA, two values of l packed per
//   tensor-memory column, 8 significant bits per factor); the split BF16 mode runs the
//   checkpointed kernel k_leg_synth_tc2 below.
#include <climits>

#include "common.h"

namespace cmbws {

namespace {

constexpr int kTcNT = 128;  // threads = ring pairs per CTA = MMA M
constexpr int kTcKB = 32;   // values of l per stage (4 MMAs of K = 8)

// Round to TF32 (10 explicit significand bits), nearest with ties away from zero: adding
// half a unit of the 11th bit to the bit pattern carries into the kept bits exactly when the
// dropped 13 bits are at least half a unit (sign-magnitude format, finite inputs).  The MMA
// reads only the upper 19 bits of a TF32 operand, so tf32_bits() leaves the low bits for it
// to drop; tf32_rna() clears them (needed where the rounded value is reused).
__device__ __forceinline__ uint32_t tf32_bits(float x) { return __float_as_uint(x) + 0x1000u; }
__device__ __forceinline__ uint32_t tf32_rna(float x) { return tf32_bits(x) & 0xFFFFE000u; }

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// K-major, no-swizzle shared-memory matrix descriptor: core matrices of 8 rows x 16 bytes,
// LBO = byte step between core matrices along K, SBO = along N; descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N = 16, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(kIdesc), "r"(acc));
}

// Instruction descriptor of kind::f16 with both operands BF16: D FP32, A and B BF16 (both the
// same 16-bit type), both K-major, N = 16, M = 128.
constexpr uint32_t kIdescBf16 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d, uint32_t a, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
      "r"(a), "l"(bdesc), "r"(kIdescBf16), "r"(acc));
}

// Two FP32 values rounded to BF16 (nearest even) and packed: lo in bits 0-15, hi in 16-31.
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
// the FP32 values of the two BF16 halves of a packed word
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Device-side status of this file's kernels (one word per device): bit 0 is set when a
// bounded mbarrier wait ran out; cmbws_device_status reads and clears it.
__device__ unsigned int g_tc_status = 0;
// Test support (cmbws_testing_stall_waits): when > 0, every CTA first waits at most this many
// SM clocks on an mbarrier phase that nothing completes, so the wait runs out.
__device__ long long g_tc_stall_cycles = 0;

constexpr long long kWaitCycles = 1ll << 32;  // about two seconds at 2 GHz

// Wait for the completion of phase `parity` of an mbarrier; false after `limit` SM clocks (or
// 2^26 polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitCycles) {
  const uint32_t a = smem_addr(bar);
  const long long t0 = clock64();
  for (int it = 0; it < (1 << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) break;
  }
  return false;
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
      "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
      "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16};\n" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}

template <int SPLIT, int BF>
struct TcLayout {
  static constexpr int kBStage = 4 * 512;                         // one 16 x 32 TF32 tile
  static constexpr int kStage = (SPLIT ? 2 : 1) * kBStage;        // hi (+ lo) per stage
  static constexpr int kOffA = 2 * kStage;                        // float sAc[2][4][32]: A, B, R, S
  static constexpr int kOffBar = kOffA + 2 * 4 * kTcKB * 4;       // uint64_t mbar[3]
  static constexpr int kOffT = kOffBar + 24;                      // uint32_t tmem base, bad flag
  static constexpr int kUsed = kOffT + 16;
  // Tensor memory: one A buffer of 32 columns of TF32 values of l (split TF32 adds the lo
  // part) or two of 16 columns of packed BF16 pairs, then 16 accumulator columns.  Shared
  // memory requested per CTA: caps residency so that the CTAs of an SM never ask for more
  // than its 512 columns (4 x 128 split TF32, 8 x 64 TF32 or BF16).
  static constexpr int kSmem = SPLIT ? 48 * 1024 : 26 * 1024;
  static constexpr uint32_t kCols = SPLIT ? 128 : 64;
  static constexpr uint32_t kColA = 0, kColAlo = 32, kColD = SPLIT ? 64 : 32;
};

// Byte offset of B[n][k] (n < 16 output column, k < 32 within the block) in a stage tile:
// core matrices of 8 rows x 16 bytes (4 TF32 or 8 BF16 values of k), two along K per MMA
// (LBO 128 bytes), two along N (SBO 256 bytes), one 512-byte slice per MMA (K = 8 for TF32,
// K = 16 for BF16).
__device__ __forceinline__ int b_off(int n, int k) {
  return (k >> 3) * 512 + (n >> 3) * 256 + ((k >> 2) & 1) * 128 + (n & 7) * 16 + (k & 3) * 4;
}
__device__ __forceinline__ int b_off16(int n, int k) {
  return (k >> 4) * 512 + (n >> 3) * 256 + ((k >> 3) & 1) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

// BF = 1: BF16 operands (kind::f16, K = 16 per MMA, two values of l per tensor-memory column)
// instead of TF32 (kind::tf32, K = 8).
template <int NM, int SPLIT, int BF>
__device__ __forceinline__ void
synth_tc_body(const float2* __restrict__ alm, int64_t alm_stride, const float* __restrict__ Acoef,
              const float* __restrict__ brs, const int* __restrict__ ls_tab,
              const float2* __restrict__ st,
              const float* __restrict__ yr, const int2* __restrict__ pring, float2* __restrict__ F,
              int64_t F_stride, int L, int npair) {
  using LY = TcLayout<SPLIT, BF>;
  static_assert(NM >= 1 && NM <= 4, "at most 4 maps (16 output columns)");
  static_assert(!(SPLIT && BF), "split BF16 runs k_leg_synth_tc2");
  extern __shared__ __align__(1024) unsigned char sm[];
  float* sAc = reinterpret_cast<float*>(sm + LY::kOffA);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + LY::kOffBar);
  uint32_t* s_tb = reinterpret_cast<uint32_t*>(sm + LY::kOffT);
  int* s_lo = reinterpret_cast<int*>(sm + LY::kOffT + 4);
  int* s_bad = reinterpret_cast<int*>(sm + LY::kOffT + 8);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = blockIdx.y;
  const int64_t lmo = lm_off(L, m) - m;
  const int p = blockIdx.x * kTcNT + tid;
  const bool valid = p < npair;
  const int ls = valid ? ls_tab[(int64_t)m * npair + p] : INT_MAX;
  const float y = valid ? yr[p] : 0.f;
  const float2 inj = valid ? st[(int64_t)m * npair + p] : make_float2(0.f, 0.f);

  if (tid == 0) {
    *s_lo = INT_MAX;
    *s_bad = 0;
  }
  __syncthreads();
  atomicMin(s_lo, ls);
  __syncthreads();
  const int lo = *s_lo;
  if (lo > L) {  // no pair of the tile has a significant value at this m
    if (valid) {
      const int2 rr = pring[p];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        F[k * F_stride + (int64_t)rr.x * (L + 1) + m] = make_float2(0.f, 0.f);
        if (rr.y >= 0) F[k * F_stride + (int64_t)rr.y * (L + 1) + m] = make_float2(0.f, 0.f);
      }
    }
    return;
  }
  const int nb = (L - lo + kTcKB) / kTcKB;

  // zero the B tiles (positions of the other parity and of absent maps stay zero)
  for (int i = tid; i < 2 * LY::kStage / 16; i += kTcNT)
    reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(s_tb)),
                 "r"(LY::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[2])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    // test support: a wait on mbar[2], which no thread or copy ever arrives at, runs out;
    // the CTA then issues no MMA and writes NaN, as after a failed wait on a stage
    const long long stall = g_tc_stall_cycles;
    if (stall > 0 && !mbar_wait(&mbar[2], 0, stall)) *s_bad = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tb = *s_tb;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

  // B element of this thread: block position k, map j (real and imaginary columns)
  const int kk = tid & 31, jj = tid >> 5;
  const int n_re = (kk & 1) * 8 + 2 * jj;
  auto load_coef = [&](int b) {
    const int l = lo + b * kTcKB + kk;
    float2 v = make_float2(0.f, 0.f);
    if (jj < NM && l <= L) v = alm[jj * alm_stride + lmo + l];
    return v;
  };
  // recurrence coefficients of a block: thread tid loads A (tid < 32) or B, R, S (the
  // difference form near the poles) of l = lo + 32 b + tid % 32
  auto load_A = [&](int b) {
    const int l = lo + b * kTcKB + (tid & 31);
    if (l > L) return 0.f;
    return tid < kTcKB ? Acoef[lmo + l] : brs[3 * (lmo + l) + (tid / kTcKB - 1)];
  };
  float2 cnext = load_coef(0);
  float anext = load_A(0);
  // warps holding a polar ring pair run the difference form (warp-uniform)
  const bool polar = __any_sync(0xffffffffu, valid && y < kPolarY);

  float mu1 = 0.f, mu2 = 0.f;
  bool bad = false;
  for (int b = 0; b < nb; ++b) {
    const int s = b & 1;
    // once a wait has failed no more MMAs are issued, so later waits are skipped
    // BF16 keeps two A buffers (16 columns each): wait here for the MMAs of block b - 2, which
    // read this stage.  TF32 kinds have one A buffer and wait after the recurrence (below);
    // their B stage was last read by the MMAs of block b - 2, waited for in block b - 1.
    if constexpr (BF)
      if (b >= 2 && !*s_bad && !mbar_wait(&mbar[s], ((b - 2) >> 1) & 1)) bad = true;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    // stage the block's coefficients (B) and recurrence coefficients A_l
    {
      unsigned char* bs = sm + s * LY::kStage;
      if (jj < NM) {
        if constexpr (BF) {
          const uint32_t w = bf16x2_rn(cnext.x, cnext.y);
          *reinterpret_cast<uint16_t*>(bs + b_off16(n_re, kk)) = (uint16_t)(w & 0xFFFFu);
          *reinterpret_cast<uint16_t*>(bs + b_off16(n_re + 1, kk)) = (uint16_t)(w >> 16);
        } else {
          const uint32_t hr = tf32_rna(cnext.x), hi = tf32_rna(cnext.y);
          *reinterpret_cast<uint32_t*>(bs + b_off(n_re, kk)) = hr;
          *reinterpret_cast<uint32_t*>(bs + b_off(n_re + 1, kk)) = hi;
          if constexpr (SPLIT) {
            *reinterpret_cast<uint32_t*>(bs + LY::kBStage + b_off(n_re, kk)) =
                tf32_bits(cnext.x - __uint_as_float(hr));
            *reinterpret_cast<uint32_t*>(bs + LY::kBStage + b_off(n_re + 1, kk)) =
                tf32_bits(cnext.y - __uint_as_float(hi));
          }
        }
      }
      sAc[s * 4 * kTcKB + tid] = anext;
    }
    if (b + 1 < nb) {  // prefetch the next block (consumed next iteration)
      cnext = load_coef(b + 1);
      anext = load_A(b + 1);
    }
    __syncthreads();
    // recurrence over the block: lambda values (rescaled) of this thread's pair
    uint32_t vh[kTcKB];
    uint32_t vl[kTcKB];
    const int jinj = ls - (lo + b * kTcKB);  // start of this thread's pair within the block
    // one step pair (l, l + 1) of the recurrence, TF32 parts written to vh / vl (BF16: the
    // pair packed into word j / 2, l in the low half)
    auto step = [&](int j, float2 a2) {
      const float ma = fmaf(fmaf(-a2.x, y, a2.x), mu1, -mu2);
      const float mb = fmaf(fmaf(-a2.y, y, a2.y), ma, -mu1);
      mu2 = ma;
      mu1 = mb;
    };
    auto emit2 = [&](int j, float ma, float mb) {
      if constexpr (BF) {
        vh[j >> 1] = bf16x2_rn(ma, mb);
      } else if constexpr (SPLIT) {
        vh[j] = tf32_rna(ma);
        vh[j + 1] = tf32_rna(mb);
        vl[j] = tf32_bits(ma - __uint_as_float(vh[j]));
        vl[j + 1] = tf32_bits(mb - __uint_as_float(vh[j + 1]));
      } else {
        vh[j] = tf32_bits(ma);
        vh[j + 1] = tf32_bits(mb);
      }
    };
    auto emit = [&](int j) { emit2(j, mu2, mu1); };
    const float* sa = &sAc[s * 4 * kTcKB];
    if (polar) {
      // difference form: mu2 holds e_{l-1} = mu_{l-1} - R_{l-1} mu_{l-2}
#pragma unroll
      for (int j = 0; j < kTcKB; j += 2) {
        const float2 a2 = *reinterpret_cast<const float2*>(sa + j);
        const float2 b2 = *reinterpret_cast<const float2*>(sa + kTcKB + j);
        const float2 r2 = *reinterpret_cast<const float2*>(sa + 2 * kTcKB + j);
        const float2 s2 = *reinterpret_cast<const float2*>(sa + 3 * kTcKB + j);
        float e = fmaf(fmaf(-a2.x, y, b2.x), mu1, s2.x * mu2);
        float ma = fmaf(r2.x, mu1, e);
        e = fmaf(fmaf(-a2.y, y, b2.y), ma, s2.y * e);
        float mb = fmaf(r2.y, ma, e);
        if (j == jinj) {
          ma = inj.x;
          mb = inj.y;
          e = fmaf(-r2.y, inj.x, inj.y);
        }
        mu2 = e;
        mu1 = mb;
        emit2(j, ma, mb);
      }
    } else if (__any_sync(0xffffffffu, jinj >= 0 && jinj < kTcKB)) {
      // a pair of this warp starts in the block: inject its start values at jinj
#pragma unroll
      for (int j = 0; j < kTcKB; j += 2) {
        step(j, *reinterpret_cast<const float2*>(sa + j));
        if (j == jinj) {
          mu2 = inj.x;
          mu1 = inj.y;
        }
        emit(j);
      }
    } else {
#pragma unroll
      for (int j = 0; j < kTcKB; j += 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(sa + j);
        step(j, make_float2(a4.x, a4.y));
        emit(j);
        step(j + 2, make_float2(a4.z, a4.w));
        emit(j + 2);
      }
    }
    // TF32 kinds: one A buffer in tensor memory, which the MMAs of block b - 1 (issued after
    // the last barrier) have read by now (bounded wait; once a wait has failed no more MMAs
    // are issued and later waits are skipped)
    if constexpr (!BF) {
      if (b >= 1 && !*s_bad && !mbar_wait(&mbar[(b - 1) & 1], ((b - 1) >> 1) & 1)) bad = true;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    }
    if constexpr (BF) {
      tmem_st16(tb + lane_base + LY::kColA + 16 * s, *reinterpret_cast<const uint32_t(*)[16]>(vh));
    } else {
      tmem_st32(tb + lane_base + LY::kColA, vh);
      if constexpr (SPLIT) tmem_st32(tb + lane_base + LY::kColAlo, vl);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::);
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    if (bad) atomicOr(s_bad, 1);
    __syncthreads();
    if (tid == 0 && !*s_bad) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t bh = smem_addr(sm + s * LY::kStage);
      if constexpr (BF) {
#pragma unroll
        for (int i = 0; i < kTcKB / 16; ++i) {  // K = 16: 8 columns of packed pairs per MMA
          const uint32_t a_hi = tb + LY::kColA + 16 * s + 8 * i;
          const uint64_t dh = smem_desc(bh + 512 * i, 128, 256);
          mma_bf16(tb + LY::kColD, a_hi, dh, (b > 0 || i > 0) ? 1u : 0u);
        }
      } else {
#pragma unroll
        for (int i = 0; i < kTcKB / 8; ++i) {
          const uint32_t a_hi = tb + LY::kColA + 8 * i;
          const uint64_t dh = smem_desc(bh + 512 * i, 128, 256);
          mma_tf32(tb + LY::kColD, a_hi, dh, (b > 0 || i > 0) ? 1u : 0u);
          if constexpr (SPLIT) {
            const uint64_t dl = smem_desc(bh + LY::kBStage + 512 * i, 128, 256);
            mma_tf32(tb + LY::kColD, a_hi, dl, 1u);
            mma_tf32(tb + LY::kColD, tb + LY::kColAlo + 8 * i, dh, 1u);
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(&mbar[s])));
    }
  }
  // accumulators of the last block
  if (!*s_bad && !mbar_wait(&mbar[(nb - 1) & 1], ((nb - 1) >> 1) & 1)) bad = true;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  uint32_t d[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
        "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
      : "r"(tb + lane_base + LY::kColD));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
  if (bad) atomicOr(s_bad, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  const bool failed = *s_bad != 0;
  if (failed && tid == 0) atomicOr(&g_tc_status, 1u);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tb), "r"(LY::kCols));
  if (!valid) return;
  const int2 rr = pring[p];
  const float nan = __int_as_float(0x7fc00000);
#pragma unroll
  for (int k = 0; k < NM; ++k) {
    const float er = __uint_as_float(d[2 * k]), ei = __uint_as_float(d[2 * k + 1]);
    const float orr = __uint_as_float(d[8 + 2 * k]), oi = __uint_as_float(d[8 + 2 * k + 1]);
    // a timed-out wait leaves NaN in the output, which the solver reports as a breakdown
    const float2 fn = failed ? make_float2(nan, nan) : make_float2(er + orr, ei + oi);
    const float2 fs = failed ? make_float2(nan, nan) : make_float2(er - orr, ei - oi);
    F[k * F_stride + (int64_t)rr.x * (L + 1) + m] = fn;
    if (rr.y >= 0) F[k * F_stride + (int64_t)rr.y * (L + 1) + m] = fs;
  }
}

// The kernels: the BF16 instance keeps the compiler's own register choice (64, no spill:
// 8 CTAs per SM, measured 1.84 ms at Nside 1024 against 2.05 ms when bounded to 8 CTAs,
// which made it spill); the TF32 kinds are bounded to 8 (4 split) CTAs per SM.
#define CMBWS_SYNTH_TC_ARGS                                                                    \
  const float2 *__restrict__ alm, int64_t alm_stride, const float *__restrict__ Acoef,        \
      const float *__restrict__ brs, const int *__restrict__ ls_tab,                          \
      const float2 *__restrict__ st, const float *__restrict__ yr,                            \
      const int2 *__restrict__ pring, float2 *__restrict__ F, int64_t F_stride, int L, int npair
template <int NM>
__global__ void __launch_bounds__(kTcNT) k_leg_synth_tc_bf16(CMBWS_SYNTH_TC_ARGS) {
  synth_tc_body<NM, 0, 1>(alm, alm_stride, Acoef, brs, ls_tab, st, yr, pring, F, F_stride, L, npair);
}
template <int NM, int SPLIT>
__global__ void __launch_bounds__(kTcNT, SPLIT ? 4 : 8) k_leg_synth_tc(CMBWS_SYNTH_TC_ARGS) {
  synth_tc_body<NM, SPLIT, 0>(alm, alm_stride, Acoef, brs, ls_tab, st, yr, pring, F, F_stride, L,
                              npair);
}
#undef CMBWS_SYNTH_TC_ARGS

template <int NM, int SPLIT, int BF>
int launch_synth_tc(const Grid& g, const void* alm, int64_t as, void* F, int64_t fs, cudaStream_t s) {
  using LY = TcLayout<SPLIT, BF>;
  const int L = g.lmax;
  dim3 grd((g.npair + kTcNT - 1) / kTcNT, L + 1);
  static_assert(!(SPLIT && BF), "split BF16 runs k_leg_synth_tc2");
  auto kern = BF ? k_leg_synth_tc_bf16<NM> : k_leg_synth_tc<NM, SPLIT>;
  CMBWS_TRY(ensure_dyn_smem((const void*)kern, LY::kSmem));
  // profiling arithmetic kinds: 3 TF32, 4 split TF32, 5 BF16, 6 split BF16
  ProfScope ps(PROF_LEG_SYNTH, s, 3 + SPLIT + 2 * BF, leg_work(g, NM));
  kern<<<grd, kTcNT, LY::kSmem, s>>>((const float2*)alm, as, g.A32.as<float>(), g.BRS32.as<float>(),
                                     g.ls.as<int>(),
                                     g.st32.as<float2>(), g.y32.as<float>(), g.pair_ring.as<int2>(),
                                     (float2*)F, fs, L, g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

template <int SPLIT, int BF>
int launch_synth_tc_nm(int nm, const Grid& g, const void* a, int64_t as, void* f, int64_t fs,
                       cudaStream_t s) {
  switch (nm) {
    case 1: return launch_synth_tc<1, SPLIT, BF>(g, a, as, f, fs, s);
    case 2: return launch_synth_tc<2, SPLIT, BF>(g, a, as, f, fs, s);
    case 3: return launch_synth_tc<3, SPLIT, BF>(g, a, as, f, fs, s);
    default: return launch_synth_tc<4, SPLIT, BF>(g, a, as, f, fs, s);
  }
}

// ---- adjoint synthesis (analysis) on the tensor cores ----
//
// Per m the adjoint a_lm = sum over ring pairs of lambda_lm(theta) times the pair's even or
// odd part (Sec. 2.1) is, for a tile of 128 values of l, the product
// D[l][col] = sum_p Lambda[l][p] B[p][col] with B[p][h * 8 + part] the pair's even (h = 0,
// north + south) and odd (h = 1, north - south) parts, so that row l reads its sum from the
// columns of the parity of l - m.  The contraction runs over ring pairs (K), 64 per stage.
// * Lambda^T (A operand, M = l, K = pairs) is generated by the recurrence: thread (chunk c,
//   octet o) restarts each of 8 pairs at the FP64-computed checkpoint of its chunk of
//   kChunk = 8 values of l (as the FP32 adjoint does) and writes the 8 x 8 BF16 values as one
//   core matrix (8 rows of l x 16 bytes of pairs) of the K-major shared-memory layout; core
//   matrices of consecutive chunks are 144 bytes apart, so that the 16-byte row stores of a
//   warp fall on distinct banks;
// * B (the pairs' parts, FP32 from the ring FFT) is rounded to BF16 into the K-major layout
//   of the synthesis;
// * SA = 2 splits both operands into hi + lo BF16 slices: A_hi [B_hi | B_lo] (N = 32) and
//   A_lo B_hi accumulate into the same 32 columns, whose halves are summed at the end;
// * two stages alternate; one thread issues the MMAs (M = 128, K = 16) after the stage's
//   barrier and commits them to the stage's mbarrier, on which the producers wait (bounded)
//   before overwriting it.
constexpr int kAtM = 128;     // values of l per CTA (MMA M, threads) = 16 chunks of kChunk
constexpr int kAtKS = 64;     // ring pairs per stage: 8 octets, 4 MMAs of K = 16
constexpr int kAtCore = 144;  // bytes between the core matrices of consecutive chunks
constexpr int kAtOct = (kAtM / 8) * kAtCore;  // bytes between the core matrices of consecutive octets
constexpr int kAtASlice = (kAtKS / 8) * kAtOct;
constexpr int kAtMaxStage = 128;  // stages of a launch (ring pairs <= 8192)

template <int SA>
struct AtLayout {
  static constexpr int kBStep = 512 * SA;  // one K step of B: 16 SA rows x 16 pairs, BF16
  static constexpr int kBTile = (kAtKS / 16) * kBStep;
  static constexpr int kStage = SA * kAtASlice + kBTile;  // one stage, single-buffered
  // inputs of one stage, copied (cp.async) one stage ahead: the stage's starts, y, start
  // values and even / odd parts (up to 4 maps)
  static constexpr int kPLs = 0;
  static constexpr int kPY = kPLs + kAtKS * 4;
  static constexpr int kPSt = kPY + kAtKS * 4;
  static constexpr int kPEo = kPSt + kAtKS * 8;
  static constexpr int kPre = kPEo + kAtKS * 16 * 4;
  static constexpr int kOffPre = kStage;
  static constexpr int kOffBar = kOffPre + 2 * kPre;  // uint64_t mbar[2]
  static constexpr int kOffT = kOffBar + 16;          // uint32_t tensor-memory base, bad flag
  static constexpr int kOffMask = kOffT + 16;         // uint32_t stage mask[kAtMaxStage / 32]
  static constexpr int kSmem = kOffMask + kAtMaxStage / 8;
  static constexpr uint32_t kCols = 32;
};

// kind::f16 instruction descriptor, BF16 A and B (K-major), FP32 D, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
}

// D (+)= A B with both operands in shared memory (descriptors)
__device__ __forceinline__ void mma_bf16_ss(uint32_t d, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// byte offset of B[n][p] (output column n, pair p < 64 of the stage) in a stage's B tile
template <int SA>
__device__ __forceinline__ int at_boff(int n, int p) {
  return (p >> 4) * AtLayout<SA>::kBStep + (n >> 3) * 256 + ((p >> 3) & 1) * 128 + (n & 7) * 16 +
         (p & 7) * 2;
}

template <int NM, int SA>
__global__ void __launch_bounds__(kAtM, SA == 1 ? 5 : 4)
k_leg_adj_tc(const float* __restrict__ eo, const float* __restrict__ Acoef,
             const int* __restrict__ ls_tab, const float2* __restrict__ st,
             const float* __restrict__ yr, const float2* __restrict__ ck,
             const int64_t* __restrict__ ck_base, const int* __restrict__ tmin,
             const double* __restrict__ c64, double2* __restrict__ out, int64_t nlm, int L,
             int npair) {
  using LY = AtLayout<SA>;
  static_assert(kChunk == 8, "one core matrix holds one chunk of 8 values of l");
  static_assert(NM >= 1 && NM <= 4, "at most 4 maps (8 columns per parity)");
  static_assert(kAtKS % kTileMinPT == 0, "a stage covers whole entries of the tile-start table");
  constexpr int P = 2 * NM;
  constexpr int NTM = kAtKS / kTileMinPT;
  const int m = blockIdx.y;
  const int lb0 = m + kAtM * (int)blockIdx.x;  // first l of the tile
  if (lb0 > L) return;                         // CTA-uniform, before any barrier
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ci = tid & 15, oc = tid >> 4;  // chunk of the tile, octet of the stage
  const int nck = (L - m + kChunk) / kChunk;
  const int c = (int)blockIdx.x * (kAtM / kChunk) + ci;
  const int l0 = m + kChunk * c;
  const bool cval = c < nck;
  const int64_t lmo = lm_off(L, m) - m;
  const int llast = min(L, lb0 + kAtM - 1);
  const int ntm = (npair + kTileMinPT - 1) / kTileMinPT;
  const int nst = (npair + kAtKS - 1) / kAtKS;  // <= kAtMaxStage (checked by the host)

  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + LY::kOffBar);
  uint32_t* s_tb = reinterpret_cast<uint32_t*>(sm + LY::kOffT);
  int* s_bad = reinterpret_cast<int*>(sm + LY::kOffT + 8);
  uint32_t* s_mask = reinterpret_cast<uint32_t*>(sm + LY::kOffMask);
  // stages with a pair that starts by the tile's last l (the others add nothing): lane s of
  // a warp tests stage s against the smallest start of each of its tiles of pairs
  {
    const int* tm = tmin + (int64_t)m * ntm;
    for (int s0 = warp * 32; s0 < kAtMaxStage; s0 += kAtM) {
      const int s = s0 + lane;
      bool any = false;
      if (s < nst)
#pragma unroll
        for (int e = 0; e < NTM; ++e) {
          const int t = s * NTM + e;
          any |= t < ntm && tm[t] <= llast;
        }
      const uint32_t bal = __ballot_sync(0xffffffffu, any);
      if (lane == 0) s_mask[s0 >> 5] = bal;
    }
  }
  __syncthreads();
  // first stage at or after s whose bit is set (nst if none)
  auto next_stage = [&](int s) {
    for (; s < nst; s = (s | 31) + 1) {
      const uint32_t w = s_mask[s >> 5] >> (s & 31);
      if (w) return min(nst, s + __ffs(w) - 1);
    }
    return nst;
  };
  int s = next_stage(0);
  if (s >= nst) {  // no pair has a significant value in the tile: the sums are zero
    const int l = lb0 + tid;
    if (l <= L)
#pragma unroll
      for (int k = 0; k < NM; ++k) out[k * nlm + lmo + l] = make_double2(0.0, 0.0);
    return;
  }

  if (tid == 0) *s_bad = 0;
  // zero the stage (B columns of absent maps stay zero)
  for (int i = tid; i < LY::kStage / 16; i += kAtM)
    reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(s_tb)),
                 "r"(LY::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    // test support, as in the synthesis: a wait that nothing completes runs out
    const long long stall = g_tc_stall_cycles;
    if (stall > 0 && !mbar_wait(&mbar[1], 0, stall)) *s_bad = 1;
  }

  float Al[kChunk];
#pragma unroll
  for (int j = 0; j < kChunk; ++j) Al[j] = (cval && l0 + j <= L) ? Acoef[lmo + l0 + j] : 0.f;
  const float2* ckc = ck + (cval ? ck_base[m] + c : 0);  // + p * nck
  const int* lsm = ls_tab + (int64_t)m * npair;
  const float2* stm = st + (int64_t)m * npair;
  const float* eom = eo + (int64_t)m * npair * 2 * P;

  // copy the starts, y and even / odd parts of stage s into prefetch buffer pb (one commit
  // group); pairs past the last get start INT_MAX (never started) and y = 0
  auto prefetch = [&](int s, int pb) {
    unsigned char* pre = sm + LY::kOffPre + pb * LY::kPre;
    const int p0 = s * kAtKS;
    const int np = min(kAtKS, npair - p0);
    if (tid < kAtKS) {
      if (tid < np) {
        cp_async4(pre + LY::kPLs + 4 * tid, lsm + p0 + tid);
        cp_async4(pre + LY::kPY + 4 * tid, yr + p0 + tid);
        cp_async8(pre + LY::kPSt + 8 * tid, stm + p0 + tid);
      } else {
        reinterpret_cast<int*>(pre + LY::kPLs)[tid] = INT_MAX;
        reinterpret_cast<float*>(pre + LY::kPY)[tid] = 0.f;
      }
    }
    // the even / odd parts of the stage's pairs are contiguous (2P floats per pair)
    for (int i = tid; i < np * P / 2; i += kAtM)
      cp_async16(pre + LY::kPEo + 16 * i, eom + (int64_t)p0 * 2 * P + 4 * i);
    cp_async_commit();
  };
  // this thread's 8 checkpoints of stage s
  auto load_ck = [&](int s, float2 (&cv)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = s * kAtKS + 8 * oc + i;
      cv[i] = (cval && p < npair) ? ckc[(int64_t)p * nck] : make_float2(0.f, 0.f);
    }
  };

  float2 ckA[8], ckB[8];
  load_ck(s, ckA);
  prefetch(s, 0);
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tb = *s_tb;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  unsigned char* As = sm;
  unsigned char* Bs = As + SA * kAtASlice;

  bool bad = false;
  int k = 0;
  // one stage: inputs of stage s in prefetch buffer k & 1 and in cv; the next stage's
  // checkpoints are loaded into cvn
  auto run_stage = [&](const float2 (&cv)[8], float2 (&cvn)[8]) {
    const int sn = next_stage(s + 1);
    if (sn < nst) {
      load_ck(sn, cvn);
      prefetch(sn, (k + 1) & 1);
    }
    const unsigned char* pre = sm + LY::kOffPre + (k & 1) * LY::kPre;
    const int p0 = s * kAtKS;
    const int np = min(kAtKS, npair - p0);
    // B values and A start values into registers before waiting for the previous MMAs
    const int n = tid & 15, q = n & 7, ob = tid >> 4;
    float v[8];
    {
      const float* e = reinterpret_cast<const float*>(pre + LY::kPEo) + (n >> 3) * P + q;
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = (q < P && 8 * ob + i < np) ? e[(8 * ob + i) * 2 * P] : 0.f;
    }
    const int4* lsb = reinterpret_cast<const int4*>(pre + LY::kPLs) + 2 * oc;
    const float4* yb = reinterpret_cast<const float4*>(pre + LY::kPY) + 2 * oc;
    const float2* stb = reinterpret_cast<const float2*>(pre + LY::kPSt) + 8 * oc;
    const int4 la = lsb[0], lb = lsb[1];
    const float4 ya = yb[0], yb2 = yb[1];
    const int jinj[8] = {la.x - l0, la.y - l0, la.z - l0, la.w - l0,
                         lb.x - l0, lb.y - l0, lb.z - l0, lb.w - l0};
    const float y[8] = {ya.x, ya.y, ya.z, ya.w, yb2.x, yb2.y, yb2.z, yb2.w};
    float ma[8], mb[8];
    bool mid = false, first = false;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      ma[i] = jinj[i] > 0 ? 0.f : cv[i].x;  // before its start a pair's values are zero
      mb[i] = jinj[i] > 0 ? 0.f : cv[i].y;
      first |= jinj[i] == 0;
      mid |= (unsigned)(jinj[i] - 1) < (unsigned)(kChunk - 1);  // starts after the chunk's first l
    }
    if (first)
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (jinj[i] == 0) {
          const float2 w = stb[i];
          ma[i] = w.x;
          mb[i] = w.y;
        }
    // the previous stage's MMAs have read the tile
    if (k >= 1 && !*s_bad && !mbar_wait(&mbar[0], (k - 1) & 1)) bad = true;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (q < P) {  // B: column n (parity n / 8, part q) of pair octet ob, one core-matrix row
      uint4 w;
      w.x = bf16x2_rn(v[0], v[1]);
      w.y = bf16x2_rn(v[2], v[3]);
      w.z = bf16x2_rn(v[4], v[5]);
      w.w = bf16x2_rn(v[6], v[7]);
      const int off = (ob >> 1) * LY::kBStep + (n >> 3) * 256 + (ob & 1) * 128 + q * 16;
      *reinterpret_cast<uint4*>(Bs + off) = w;
      if constexpr (SA == 2) {
        uint4 u;
        u.x = bf16x2_rn(v[0] - bf16_lo(w.x), v[1] - bf16_hi(w.x));
        u.y = bf16x2_rn(v[2] - bf16_lo(w.y), v[3] - bf16_hi(w.y));
        u.z = bf16x2_rn(v[4] - bf16_lo(w.z), v[5] - bf16_hi(w.z));
        u.w = bf16x2_rn(v[6] - bf16_lo(w.w), v[7] - bf16_hi(w.w));
        *reinterpret_cast<uint4*>(Bs + off + 512) = u;  // rows 16..31
      }
    }
    // A: the chunk's 8 values of l for the octet's 8 pairs, one core matrix per slice
    unsigned char* arow = As + oc * kAtOct + ci * kAtCore;
    auto put = [&](int j, const float (&x)[8]) {
      uint4 w;
      w.x = bf16x2_rn(x[0], x[1]);
      w.y = bf16x2_rn(x[2], x[3]);
      w.z = bf16x2_rn(x[4], x[5]);
      w.w = bf16x2_rn(x[6], x[7]);
      *reinterpret_cast<uint4*>(arow + 16 * j) = w;
      if constexpr (SA == 2) {
        uint4 u;
        u.x = bf16x2_rn(x[0] - bf16_lo(w.x), x[1] - bf16_hi(w.x));
        u.y = bf16x2_rn(x[2] - bf16_lo(w.y), x[3] - bf16_hi(w.y));
        u.z = bf16x2_rn(x[4] - bf16_lo(w.z), x[5] - bf16_hi(w.z));
        u.w = bf16x2_rn(x[6] - bf16_lo(w.w), x[7] - bf16_hi(w.w));
        *reinterpret_cast<uint4*>(arow + kAtASlice + 16 * j) = u;
      }
    };
    put(0, ma);
    put(1, mb);
    if (__any_sync(0xffffffffu, mid)) {  // warp-uniform: some start is injected mid-chunk
#pragma unroll
      for (int j = 2; j < kChunk; j += 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float na = fmaf(fmaf(-Al[j], y[i], Al[j]), mb[i], -ma[i]);
          float nb = fmaf(fmaf(-Al[j + 1], y[i], Al[j + 1]), na, -mb[i]);
          if (jinj[i] == j) {
            const float2 w = stb[i];
            na = w.x;
            nb = w.y;
          }
          ma[i] = na;
          mb[i] = nb;
        }
        put(j, ma);
        put(j + 1, mb);
      }
    } else {
#pragma unroll
      for (int j = 2; j < kChunk; j += 2) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float na = fmaf(fmaf(-Al[j], y[i], Al[j]), mb[i], -ma[i]);
          mb[i] = fmaf(fmaf(-Al[j + 1], y[i], Al[j + 1]), na, -mb[i]);
          ma[i] = na;
        }
        put(j, ma);
        put(j + 1, mb);
      }
    }
    cp_async_wait<0>();  // the next stage's inputs, visible to all after the barrier
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    if (bad) atomicOr(s_bad, 1);
    __syncthreads();
    if (tid == 0 && !*s_bad) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t ab = smem_addr(As), bb = smem_addr(Bs);
#pragma unroll
      for (int ks = 0; ks < kAtKS / 16; ++ks) {
        const uint64_t bd = smem_desc(bb + ks * LY::kBStep, 128, 256);
#pragma unroll
        for (int i = 0; i < SA; ++i) {
          const uint64_t ad = smem_desc(ab + i * kAtASlice + ks * 2 * kAtOct, kAtOct, kAtCore);
          mma_bf16_ss(tb + 16 * i, ad, bd, idesc_bf16(16 * (SA - i)),
                      (k > 0 || ks > 0 || i > 0) ? 1u : 0u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(&mbar[0])));
    }
    s = sn;
    ++k;
  };
  // two stages per trip, so that the checkpoint registers alternate without copies
  while (true) {
    run_stage(ckA, ckB);
    if (s >= nst) break;
    run_stage(ckB, ckA);
    if (s >= nst) break;
  }
  // accumulators after the last stage
  if (!*s_bad && !mbar_wait(&mbar[0], (k - 1) & 1)) bad = true;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  uint32_t d[16 * SA];
  if constexpr (SA == 1) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
        : "r"(tb + lane_base));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15]),
          "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]), "=r"(d[22]),
          "=r"(d[23]), "=r"(d[24]), "=r"(d[25]), "=r"(d[26]), "=r"(d[27]), "=r"(d[28]), "=r"(d[29]),
          "=r"(d[30]), "=r"(d[31])
        : "r"(tb + lane_base));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
  if (bad) atomicOr(s_bad, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  const bool failed = *s_bad != 0;
  if (failed && tid == 0) atomicOr(&g_tc_status, 1u);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tb), "r"(LY::kCols));
  const int l = lb0 + tid;  // row tid of D
  if (l > L) return;
  const int h = (l - m) & 1;
  const double cc = c64[lmo + l];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    // static register indices: the parity selects between the two column groups
    double re = (double)__uint_as_float(h ? d[8 + 2 * q] : d[2 * q]);
    double im = (double)__uint_as_float(h ? d[8 + 2 * q + 1] : d[2 * q + 1]);
    if constexpr (SA == 2) {
      re += (double)__uint_as_float(h ? d[24 + 2 * q] : d[16 + 2 * q]);
      im += (double)__uint_as_float(h ? d[24 + 2 * q + 1] : d[16 + 2 * q + 1]);
    }
    // a timed-out wait leaves NaN in the output, which the solver reports as a breakdown
    out[q * nlm + lmo + l] = failed ? make_double2(nan, nan) : make_double2(cc * re, cc * im);
  }
}

template <int NM, int SA>
int launch_adj_tc(const Grid& g, const float* eo, double* out, cudaStream_t s) {
  using LY = AtLayout<SA>;
  const int L = g.lmax;
  if (g.npair > kAtMaxStage * kAtKS) {
    set_error("tensor-core adjoint: more than 8192 ring pairs");
    return CMBWS_ERR_ARG;
  }
  dim3 grd((L + kAtM) / kAtM, L + 1);
  auto kern = k_leg_adj_tc<NM, SA>;
  CMBWS_TRY(ensure_dyn_smem((const void*)kern, LY::kSmem));
  // profiling arithmetic kinds: 5 BF16, 6 split BF16
  ProfScope ps(PROF_LEG_ADJ, s, 4 + SA, leg_work(g, NM));
  kern<<<grd, kAtM, LY::kSmem, s>>>(eo, g.A32.as<float>(), g.ls.as<int>(), g.st32.as<float2>(),
                                    g.y32.as<float>(), g.ck32.as<float2>(), g.ck_base.as<int64_t>(),
                                    g.ls_tmin.as<int>(), g.c64.as<double>(), (double2*)out,
                                    nlm_of(L), L, g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

template <int SA>
int launch_adj_tc_nm(int nm, const Grid& g, const float* e, double* o, cudaStream_t s) {
  switch (nm) {
    case 1: return launch_adj_tc<1, SA>(g, e, o, s);
    case 2: return launch_adj_tc<2, SA>(g, e, o, s);
    case 3: return launch_adj_tc<3, SA>(g, e, o, s);
    default: return launch_adj_tc<4, SA>(g, e, o, s);
  }
}

// ---- synthesis on the tensor cores from checkpoints (BF16 / split BF16) ----
//
// The same product as k_leg_synth_tc, D[pair][col] = sum_l Lambda[pair][l] B[l][col], with the
// A operand built the way the tensor-core adjoint builds it: thread (octet of 8 ring pairs,
// chunk of kChunk = 8 values of l) restarts each pair's recurrence at the chunk's
// FP64-computed checkpoint and writes the 8 x 8 BF16 values as one core matrix (8 rows of
// ring pairs x 16 bytes of l) of the K-major shared-memory tile.  Eight independent chains
// per thread replace the single chain of k_leg_synth_tc, the recurrence never runs more than
// 8 steps in FP32 (no difference form near the poles), and consecutive threads take
// consecutive chunks of a pair, so the checkpoint loads are contiguous.  Core matrices of
// consecutive chunks sit 144 bytes apart (LBO 144, SBO 1152), so that a warp's 16-byte row
// stores fall on distinct banks.  Stages of 64 values of l: the coefficients and A_l of the
// next stage arrive by cp.async, the checkpoints in two alternating register sets; the tile
// is single-buffered (5 CTAs per SM).
constexpr int kSt2M = 128;                        // ring pairs per CTA (MMA M, threads)
constexpr int kSt2KS = 64;                        // values of l per stage: 8 chunks
constexpr int kSt2Core = 144;                     // bytes between core matrices of consecutive chunks
constexpr int kSt2Oct = (kSt2KS / 8) * kSt2Core;  // bytes between consecutive octets of pairs
constexpr int kSt2ASlice = (kSt2M / 8) * kSt2Oct;

template <int SA>
struct St2Layout {
  static constexpr int kBStep = 512 * SA;  // one K step of B: 16 SA rows x 16 values of l
  static constexpr int kBTile = (kSt2KS / 16) * kBStep;
  static constexpr int kStage = SA * kSt2ASlice + kBTile;
  // per-stage inputs (two buffers): the coefficients of up to 4 maps and A_l
  static constexpr int kPAlm = 0;
  static constexpr int kPA = kPAlm + 4 * kSt2KS * 8;
  static constexpr int kPre = kPA + kSt2KS * 4;
  static constexpr int kOffPre = kStage;
  // per-pair data of the CTA: start values, starts, y
  static constexpr int kOffSt = kOffPre + 2 * kPre;
  static constexpr int kOffLs = kOffSt + kSt2M * 8;
  static constexpr int kOffY = kOffLs + kSt2M * 4;
  static constexpr int kOffBar = kOffY + kSt2M * 4;  // uint64_t mbar[2]
  static constexpr int kOffT = kOffBar + 16;          // tensor-memory base, bad flag, min start
  static constexpr int kSmem = kOffT + 16;
  static constexpr uint32_t kCols = 32;
};

template <int NM, int SA>
__global__ void __launch_bounds__(kSt2M, SA == 1 ? 5 : 4)
k_leg_synth_tc2(const float2* __restrict__ alm, int64_t alm_stride, const float* __restrict__ Acoef,
                const int* __restrict__ ls_tab, const float2* __restrict__ st,
                const float* __restrict__ yr, const float2* __restrict__ ck,
                const int64_t* __restrict__ ck_base, const int2* __restrict__ pring,
                float2* __restrict__ F, int64_t F_stride, int L, int npair) {
  using LY = St2Layout<SA>;
  static_assert(kChunk == 8, "one core matrix holds one chunk of 8 values of l");
  static_assert(NM >= 1 && NM <= 4, "at most 4 maps (8 columns per parity)");
  constexpr int P = 2 * NM;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + LY::kOffBar);
  uint32_t* s_tb = reinterpret_cast<uint32_t*>(sm + LY::kOffT);
  int* s_bad = reinterpret_cast<int*>(sm + LY::kOffT + 4);
  int* s_lo = reinterpret_cast<int*>(sm + LY::kOffT + 8);
  float2* s_st = reinterpret_cast<float2*>(sm + LY::kOffSt);
  int* s_ls = reinterpret_cast<int*>(sm + LY::kOffLs);
  float* s_y = reinterpret_cast<float*>(sm + LY::kOffY);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = blockIdx.y;
  const int p0 = blockIdx.x * kSt2M;
  const int64_t lmo = lm_off(L, m) - m;
  const int nck = (L - m + kChunk) / kChunk;
  // this CTA's pairs: start values, starts (INT_MAX past the last pair), y
  {
    const int p = p0 + tid;
    const bool ok = p < npair;
    const int ls = ok ? ls_tab[(int64_t)m * npair + p] : INT_MAX;
    s_ls[tid] = ls;
    s_y[tid] = ok ? yr[p] : 0.f;
    s_st[tid] = ok ? st[(int64_t)m * npair + p] : make_float2(0.f, 0.f);
    if (tid == 0) {
      *s_lo = INT_MAX;
      *s_bad = 0;
    }
    __syncthreads();
    atomicMin(s_lo, ls);
    __syncthreads();
  }
  const int lo = *s_lo;
  if (lo > L) {  // no pair of the tile has a significant value at this m
    const int p = p0 + tid;
    if (p < npair) {
      const int2 rr = pring[p];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        F[k * F_stride + (int64_t)rr.x * (L + 1) + m] = make_float2(0.f, 0.f);
        if (rr.y >= 0) F[k * F_stride + (int64_t)rr.y * (L + 1) + m] = make_float2(0.f, 0.f);
      }
    }
    return;
  }
  const int nst = (L - m + kSt2KS) / kSt2KS;
  int s = (lo - m) / kSt2KS;  // stages before the first start add nothing

  // zero the tile (B columns of absent maps and of the other parity stay zero)
  for (int i = tid; i < LY::kStage / 16; i += kSt2M)
    reinterpret_cast<float4*>(sm)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(s_tb)),
                 "r"(LY::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    // test support, as in the other tensor-core kernels: a wait that nothing completes runs out
    const long long stall = g_tc_stall_cycles;
    if (stall > 0 && !mbar_wait(&mbar[1], 0, stall)) *s_bad = 1;
  }

  const int ch = tid & 7, oc = tid >> 3;  // chunk of the stage, octet of pairs
  // the octet's starts and y, kept in registers
  int lsr[8];
  float y[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    lsr[i] = s_ls[8 * oc + i];
    y[i] = s_y[8 * oc + i];
  }
  const int64_t ckb = ck_base[m];

  // copy the coefficients and A_l of stage s into prefetch buffer pb (one commit group);
  // values past L are zero
  auto prefetch = [&](int s, int pb) {
    unsigned char* pre = sm + LY::kOffPre + pb * LY::kPre;
    const int ls0 = m + s * kSt2KS;
    for (int i = tid; i < (NM + 1) * kSt2KS; i += kSt2M) {
      const int q = i / kSt2KS, j = i % kSt2KS;
      const int l = ls0 + j;
      if (q < NM) {
        float2* dst = reinterpret_cast<float2*>(pre + LY::kPAlm) + q * kSt2KS + j;
        if (l <= L) cp_async8(dst, alm + q * alm_stride + lmo + l);
        else *dst = make_float2(0.f, 0.f);
      } else {
        float* dst = reinterpret_cast<float*>(pre + LY::kPA) + j;
        if (l <= L) cp_async4(dst, Acoef + lmo + l);
        else *dst = 0.f;
      }
    }
    cp_async_commit();
  };
  // this thread's 8 checkpoints of stage s (chunk 8 s + ch of its 8 pairs)
  auto load_ck = [&](int s, float2 (&cv)[8]) {
    const int c = s * (kSt2KS / kChunk) + ch;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = p0 + 8 * oc + i;
      cv[i] = (c < nck && p < npair) ? ck[ckb + (int64_t)p * nck + c] : make_float2(0.f, 0.f);
    }
  };

  float2 ckA[8], ckB[8];
  load_ck(s, ckA);
  prefetch(s, 0);
  cp_async_wait<0>();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  const uint32_t tb = *s_tb;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  unsigned char* As = sm;
  unsigned char* Bs = As + SA * kSt2ASlice;

  bool bad = false;
  int k = 0;
  auto run_stage = [&](const float2 (&cv)[8], float2 (&cvn)[8]) {
    const int sn = s + 1;
    if (sn < nst) {
      load_ck(sn, cvn);
      prefetch(sn, (k + 1) & 1);
    }
    const unsigned char* pre = sm + LY::kOffPre + (k & 1) * LY::kPre;
    const int ls0 = m + s * kSt2KS;
    const int l0 = ls0 + kChunk * ch;
    // B values (column n = tid % 16: parity n / 8, part n % 8, of the l-octet tid / 16)
    const int n = tid & 15, q = n & 7, ob = tid >> 4;
    float v[8];
    {
      const float* a = reinterpret_cast<const float*>(pre + LY::kPAlm) + (q >> 1) * 2 * kSt2KS + (q & 1);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = 8 * ob + i;
        v[i] = (q < P && ((ls0 + j - m) & 1) == (n >> 3)) ? a[2 * j] : 0.f;
      }
    }
    float Al[kChunk];
    {
      const float4* ap = reinterpret_cast<const float4*>(pre + LY::kPA) + 2 * ch;
      const float4 a0 = ap[0], a1 = ap[1];
      Al[0] = a0.x; Al[1] = a0.y; Al[2] = a0.z; Al[3] = a0.w;
      Al[4] = a1.x; Al[5] = a1.y; Al[6] = a1.z; Al[7] = a1.w;
    }
    // the previous stage's MMAs have read the tile
    if (k >= 1 && !*s_bad && !mbar_wait(&mbar[0], (k - 1) & 1)) bad = true;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (q < P) {  // B: one 16-byte row of a core matrix per slice
      uint4 w;
      w.x = bf16x2_rn(v[0], v[1]);
      w.y = bf16x2_rn(v[2], v[3]);
      w.z = bf16x2_rn(v[4], v[5]);
      w.w = bf16x2_rn(v[6], v[7]);
      const int off = (ob >> 1) * LY::kBStep + (n >> 3) * 256 + (ob & 1) * 128 + q * 16;
      *reinterpret_cast<uint4*>(Bs + off) = w;
      if constexpr (SA == 2) {
        uint4 u;
        u.x = bf16x2_rn(v[0] - bf16_lo(w.x), v[1] - bf16_hi(w.x));
        u.y = bf16x2_rn(v[2] - bf16_lo(w.y), v[3] - bf16_hi(w.y));
        u.z = bf16x2_rn(v[4] - bf16_lo(w.z), v[5] - bf16_hi(w.z));
        u.w = bf16x2_rn(v[6] - bf16_lo(w.w), v[7] - bf16_hi(w.w));
        *reinterpret_cast<uint4*>(Bs + off + 512) = u;  // rows 16..31
      }
    }
    // A: for each pair of the octet its 8 values of the chunk, one 16-byte row per slice;
    // two passes of four interleaved chains
    unsigned char* arow = As + oc * kSt2Oct + ch * kSt2Core;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float x[4][kChunk];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = 4 * h + u;
        const int jinj = lsr[i] - l0;  // where the pair starts, relative to the chunk
        float ma = jinj > 0 ? 0.f : cv[i].x;  // before its start a pair's values are zero
        float mb = jinj > 0 ? 0.f : cv[i].y;
        if (jinj == 0) {
          ma = s_st[8 * oc + i].x;
          mb = s_st[8 * oc + i].y;
        }
        x[u][0] = ma;
        x[u][1] = mb;
#pragma unroll
        for (int j = 2; j < kChunk; j += 2) {
          float na = fmaf(fmaf(-Al[j], y[i], Al[j]), mb, -ma);
          float nb = fmaf(fmaf(-Al[j + 1], y[i], Al[j + 1]), na, -mb);
          if (jinj == j) {
            na = s_st[8 * oc + i].x;
            nb = s_st[8 * oc + i].y;
          }
          ma = na;
          mb = nb;
          x[u][j] = ma;
          x[u][j + 1] = mb;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        uint4 w;
        w.x = bf16x2_rn(x[u][0], x[u][1]);
        w.y = bf16x2_rn(x[u][2], x[u][3]);
        w.z = bf16x2_rn(x[u][4], x[u][5]);
        w.w = bf16x2_rn(x[u][6], x[u][7]);
        *reinterpret_cast<uint4*>(arow + 16 * (4 * h + u)) = w;
        if constexpr (SA == 2) {
          uint4 z;
          z.x = bf16x2_rn(x[u][0] - bf16_lo(w.x), x[u][1] - bf16_hi(w.x));
          z.y = bf16x2_rn(x[u][2] - bf16_lo(w.y), x[u][3] - bf16_hi(w.y));
          z.z = bf16x2_rn(x[u][4] - bf16_lo(w.z), x[u][5] - bf16_hi(w.z));
          z.w = bf16x2_rn(x[u][6] - bf16_lo(w.w), x[u][7] - bf16_hi(w.w));
          *reinterpret_cast<uint4*>(arow + kSt2ASlice + 16 * (4 * h + u)) = z;
        }
      }
    }
    cp_async_wait<0>();  // the next stage's inputs, visible to all after the barrier
    asm volatile("fence.proxy.async.shared::cta;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    if (bad) atomicOr(s_bad, 1);
    __syncthreads();
    if (tid == 0 && !*s_bad) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
      const uint32_t ab = smem_addr(As), bb = smem_addr(Bs);
#pragma unroll
      for (int ks = 0; ks < kSt2KS / 16; ++ks) {
        const uint64_t bd = smem_desc(bb + ks * LY::kBStep, 128, 256);
#pragma unroll
        for (int i = 0; i < SA; ++i) {
          const uint64_t ad = smem_desc(ab + i * kSt2ASlice + ks * 2 * kSt2Core, kSt2Core, kSt2Oct);
          mma_bf16_ss(tb + 16 * i, ad, bd, idesc_bf16(16 * (SA - i)),
                      (k > 0 || ks > 0 || i > 0) ? 1u : 0u);
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_addr(&mbar[0])));
    }
    s = sn;
    ++k;
  };
  // two stages per trip, so that the checkpoint registers alternate without copies
  while (true) {
    run_stage(ckA, ckB);
    if (s >= nst) break;
    run_stage(ckB, ckA);
    if (s >= nst) break;
  }
  // accumulators after the last stage
  if (!*s_bad && !mbar_wait(&mbar[0], (k - 1) & 1)) bad = true;
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
  uint32_t d[16 * SA];
  if constexpr (SA == 1) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15])
        : "r"(tb + lane_base));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15]),
          "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]), "=r"(d[22]),
          "=r"(d[23]), "=r"(d[24]), "=r"(d[25]), "=r"(d[26]), "=r"(d[27]), "=r"(d[28]), "=r"(d[29]),
          "=r"(d[30]), "=r"(d[31])
        : "r"(tb + lane_base));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
  if (bad) atomicOr(s_bad, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
  __syncthreads();
  const bool failed = *s_bad != 0;
  if (failed && tid == 0) atomicOr(&g_tc_status, 1u);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tb), "r"(LY::kCols));
  const int p = p0 + tid;  // row tid of D
  if (p >= npair) return;
  const int2 rr = pring[p];
  const float nan = __int_as_float(0x7fc00000);
#pragma unroll
  for (int q = 0; q < NM; ++q) {
    float er = __uint_as_float(d[2 * q]), ei = __uint_as_float(d[2 * q + 1]);
    float orr = __uint_as_float(d[8 + 2 * q]), oi = __uint_as_float(d[8 + 2 * q + 1]);
    if constexpr (SA == 2) {
      er += __uint_as_float(d[16 + 2 * q]);
      ei += __uint_as_float(d[16 + 2 * q + 1]);
      orr += __uint_as_float(d[24 + 2 * q]);
      oi += __uint_as_float(d[24 + 2 * q + 1]);
    }
    // a timed-out wait leaves NaN in the output, which the solver reports as a breakdown
    const float2 fn = failed ? make_float2(nan, nan) : make_float2(er + orr, ei + oi);
    const float2 fsv = failed ? make_float2(nan, nan) : make_float2(er - orr, ei - oi);
    F[q * F_stride + (int64_t)rr.x * (L + 1) + m] = fn;
    if (rr.y >= 0) F[q * F_stride + (int64_t)rr.y * (L + 1) + m] = fsv;
  }
}

template <int NM, int SA>
int launch_synth_tc2(const Grid& g, const void* alm, int64_t as, void* F, int64_t fs, cudaStream_t s) {
  using LY = St2Layout<SA>;
  const int L = g.lmax;
  dim3 grd((g.npair + kSt2M - 1) / kSt2M, L + 1);
  auto kern = k_leg_synth_tc2<NM, SA>;
  CMBWS_TRY(ensure_dyn_smem((const void*)kern, LY::kSmem));
  // profiling arithmetic kinds: 5 BF16, 6 split BF16
  ProfScope ps(PROF_LEG_SYNTH, s, 4 + SA, leg_work(g, NM));
  kern<<<grd, kSt2M, LY::kSmem, s>>>((const float2*)alm, as, g.A32.as<float>(), g.ls.as<int>(),
                                     g.st32.as<float2>(), g.y32.as<float>(), g.ck32.as<float2>(),
                                     g.ck_base.as<int64_t>(), g.pair_ring.as<int2>(), (float2*)F, fs, L,
                                     g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

template <int SA>
int launch_synth_tc2_nm(int nm, const Grid& g, const void* a, int64_t as, void* f, int64_t fs,
                        cudaStream_t s) {
  switch (nm) {
    case 1: return launch_synth_tc2<1, SA>(g, a, as, f, fs, s);
    case 2: return launch_synth_tc2<2, SA>(g, a, as, f, fs, s);
    case 3: return launch_synth_tc2<3, SA>(g, a, as, f, fs, s);
    default: return launch_synth_tc2<4, SA>(g, a, as, f, fs, s);
  }
}

static_assert(TcLayout<0, 0>::kUsed <= TcLayout<0, 0>::kSmem &&
                  TcLayout<1, 0>::kUsed <= TcLayout<1, 0>::kSmem &&
                  TcLayout<0, 1>::kUsed <= TcLayout<0, 1>::kSmem,
              "shared-memory layout exceeds the request");
static_assert(TcLayout<0, 0>::kColD >= 32 && TcLayout<0, 0>::kColD + 16 <= TcLayout<0, 0>::kCols &&
                  TcLayout<1, 0>::kColD >= 64 && TcLayout<1, 0>::kColD + 16 <= TcLayout<1, 0>::kCols,
              "an A buffer of 32 (hi + lo: 64) columns, then 16 accumulator columns");

}  // namespace

int legendre_adjoint_tc(const Grid& g, int prec, int nmaps, const float* eo, double* out,
                        cudaStream_t s) {
  const int64_t nlm = nlm_of(g.lmax), cs = (int64_t)(g.lmax + 1) * g.npair * 4;
  for (int k0 = 0; k0 < nmaps; k0 += 4) {
    const int nm = nmaps - k0 < 4 ? nmaps - k0 : 4;
    const float* e = eo + k0 * cs;
    double* o = out + 2 * k0 * nlm;
    const int st = prec == CMBWS_BF16 ? launch_adj_tc_nm<1>(nm, g, e, o, s)
                                      : launch_adj_tc_nm<2>(nm, g, e, o, s);
    if (st != CMBWS_OK) return st;
  }
  return CMBWS_OK;
}

int legendre_synth_tc(const Grid& g, int prec, int nmaps, const void* alm, void* F, cudaStream_t s) {
  const int64_t as = nlm_of(g.lmax), fs = (int64_t)g.nring * (g.lmax + 1);
  for (int k0 = 0; k0 < nmaps; k0 += 4) {
    const int nm = nmaps - k0 < 4 ? nmaps - k0 : 4;
    const void* a = (const float2*)alm + k0 * as;
    void* f = (float2*)F + k0 * fs;
    int st;
    switch (prec) {
      case CMBWS_TF32: st = launch_synth_tc_nm<0, 0>(nm, g, a, as, f, fs, s); break;
      case CMBWS_3XTF32: st = launch_synth_tc_nm<1, 0>(nm, g, a, as, f, fs, s); break;
      // BF16: the single-chain kernel (2.57 against 3.09 ms for the checkpointed one at
      // Nside 1024, L = 3071, 3 maps); split BF16: the checkpointed kernel (3.88 against 5.45 ms)
      case CMBWS_BF16: st = launch_synth_tc_nm<0, 1>(nm, g, a, as, f, fs, s); break;
      default: st = launch_synth_tc2_nm<2>(nm, g, a, as, f, fs, s); break;
    }
    if (st != CMBWS_OK) return st;
  }
  return CMBWS_OK;
}

int tc_status_take(bool* timed_out) {
  unsigned int v = 0;
  CMBWS_CUDA(cudaMemcpyFromSymbol(&v, g_tc_status, sizeof(v)));
  *timed_out = (v & 1u) != 0;
  if (v) {
    const unsigned int zero = 0;
    CMBWS_CUDA(cudaMemcpyToSymbol(g_tc_status, &zero, sizeof(zero)));
  }
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_device_status(void* stream) {
  clear_error();
  CMBWS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  bool to = false;
  CMBWS_TRY(tc_status_take(&to));
  if (to) {
    set_error("a bounded device-side wait ran out in a tensor-core Legendre kernel; its outputs "
              "hold NaN");
    return CMBWS_ERR_TIMEOUT;
  }
  return CMBWS_OK;
}

extern "C" int cmbws_testing_stall_waits(long long wait_cycles) {
  clear_error();
  if (wait_cycles < 0 || wait_cycles > kWaitCycles) {
    set_error("cmbws_testing_stall_waits: wait_cycles must be in [0, 2^32]");
    return CMBWS_ERR_ARG;
  }
  CMBWS_CUDA(cudaMemcpyToSymbol(g_tc_stall_cycles, &wait_cycles, sizeof(wait_cycles)));
  return CMBWS_OK;
}
