// Tensor-core contractions of the mixed tent kernel (tcgen05, sm_103a).
//
// The data moments and the outflow of a tent with many right-hand sides are
// dense contractions (rows: right-hand side x component; columns: basis
// functions or points; contracted over points or basis functions).  Their
// float-float operands are split into S = kSlices = 5 signed 9-bit digits each,
//   x = 2^(e - 8) sum_{i=1..S} d_i 512^(1-i) + r,  |r| <= 2^(e - 45),  d_i in [-256, 256],
// with a power-of-two scale 2^e per row of A and per column of B (the
// exponents of their largest entries), so every digit is an integer that
// bf16 holds exactly and every digit product an integer below 2^16.  The
// products of digit planes i and j with i + j = L (L = 2 .. S + 1; the
// omitted planes i + j > S + 1 lie below ~2^-43 of the scales) are summed by
// tcgen05.mma (bf16 x bf16 -> binary32 in tensor memory) into one
// accumulator per level L.  While every partial sum stays below 2^24 in
// magnitude those binary32 sums are exact integers (the contraction length
// K, the number of pairs per level and the digit bound are chosen for that),
// so the only roundings are the digit split of the operands and the final
// combination of the levels: each product is exact to about 2^-42 of the
// product of the scales, as close as the compensated float-float sums it
// replaces (an Ozaki-style scheme with exact integer accumulation; four
// digits, ~2^-33, moved a 1D sweep by 5e-10 from the float-float one).
//
// Operands are staged in shared memory in the canonical K-major layout
// without swizzle: core matrices of 8 rows x 16 bytes (8 bf16 along K);
// A (M = 128 rows) as [k / 8][row group][8][8], B (N rows) as
// [k / 8][row group][8][8].  Rows of A beyond the stored row groups are read
// from whatever follows (their accumulator rows are never read).
#pragma once

#include <cstdint>

namespace tp {
namespace tc {

constexpr int kSlices = kTcSlices;   // digits per operand
constexpr int kMaxM = 128;    // rows of A per contraction (one M = 128 tile)
constexpr long long kMaxPolls = 1ll << 22;   // bounded wait for the MMAs of one contraction

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (tcgen05): start address, byte offsets
// between core matrices adjacent along K (lbo) and along M/N (sbo), the
// fixed version bits 0b001 at 46..48, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
         ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D binary32 (bits 4..5 = 1), A and B
// bf16 (7..9 = 1, 10..12 = 1), both K-major, N >> 3 at 17..22, M >> 4 at 24..28
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// tensor memory: allocated and freed by one whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy writes of shared memory made visible to the tensor core
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// bounded wait for the completion of the given phase parity; false when it
// did not complete within max_polls polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_polls) {
  const uint32_t a = smem_addr(bar);
  for (long long it = 0; it < max_polls; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// D[tmem] (+)= A B, issued by one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread is complete
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 8 consecutive binary32 columns of the warp's 32 tensor-memory lanes (lane
// quarter warp % 4); one register per column
__device__ __forceinline__ void ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// binary exponent e of a row or column whose largest |hi| is mx: mx < 2^e
// (e = 0 for an all-zero row, -125 for a subnormal maximum)
__device__ __forceinline__ int scale_exp(float mx) {
  const int ef = (int)((__float_as_uint(mx) >> 23) & 0xFF);
  return ef == 0 ? (mx == 0.f ? 0 : -125) : ef - 126;
}
// 2^k as binary32, |k| <= 126
__device__ __forceinline__ float pow2f(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }

// round to the nearest integer (ties to even), |x| <= 2^22
__device__ __forceinline__ float rne(float x) {
  const float M = 12582912.f;   // 1.5 * 2^23
  return __fsub_rn(__fadd_rn(x, M), M);
}

// the kSlices digits of the float-float value (hi, lo) of a row with
// exponent e: with u = (hi + lo) 2^(8 - e) in (-256, 256) (scaled by two
// exact power-of-two factors, so that rows down to the subnormal range keep
// their digits), u = sum_i d_i 512^(1-i) + r, |r| <= 512^(1-S) / 2.  Digit
// i takes the remainder of digits 1..i-1 (kept exactly as u_i + ul_i, the
// low part ul_i never rounded) to the nearest integer; |d_i| <= 256 because
// each remainder is within half a unit.
__device__ __forceinline__ void digits(float hi, float lo, int e, float (&d)[kSlices]) {
  const int k = 8 - e;   // in [-121, 133]
  const float s1 = pow2f(min(k, 126)), s2 = pow2f(max(k - 126, 0));
  float u = __fmul_rn(__fmul_rn(hi, s1), s2), ul = __fmul_rn(__fmul_rn(lo, s1), s2);
  d[0] = rne(u);
#pragma unroll
  for (int s = 1; s < kSlices; ++s) {
    u = __fmul_rn(__fsub_rn(u, d[s - 1]), 512.f);
    ul = __fmul_rn(ul, 512.f);
    d[s] = rne(__fadd_rn(u, ul));
  }
}
// bf16 bit pattern of an integer-valued binary32 with at most 8 significant bits (exact)
__device__ __forceinline__ uint32_t bf16_bits(float x) { return __float_as_uint(x) >> 16; }

// the kSlices planes of 8 consecutive K entries of one row: 16 bytes per plane
__device__ __forceinline__ void store_row8(uint16_t* base, int plane_stride, const float (&d)[8][kSlices]) {
#pragma unroll
  for (int s = 0; s < kSlices; ++s) {
    uint4 w;
    w.x = bf16_bits(d[0][s]) | (bf16_bits(d[1][s]) << 16);
    w.y = bf16_bits(d[2][s]) | (bf16_bits(d[3][s]) << 16);
    w.z = bf16_bits(d[4][s]) | (bf16_bits(d[5][s]) << 16);
    w.w = bf16_bits(d[6][s]) | (bf16_bits(d[7][s]) << 16);
    *reinterpret_cast<uint4*>(base + (size_t)s * plane_stride) = w;
  }
}

// The level sums of one output (acc_l = sum of the digit products of planes
// i + j = l + 2, integers below 2^24, exact in binary32) as the float-float
// value (s, e) of sum_l acc_l 512^-l: the two leading levels by TwoSum, the
// others into the low part, then renormalised.  Rounding enters only in the
// low part, below 2^-42 of the leading level's scale.
__device__ __forceinline__ void combine_ff(const float (&acc)[kSlices], float& s, float& e) {
  const float a = acc[0], b = __fmul_rn(acc[1], 1.f / 512.f);
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  float w = 1.f / 262144.f;
#pragma unroll
  for (int l = 2; l < kSlices; ++l) {
    e = fmaf(acc[l], w, e);
    w *= 1.f / 512.f;
  }
  const float t = __fadd_rn(s, e);
  e = __fsub_rn(e, __fsub_rn(t, s));
  s = t;
}
// (s + e) 2^P as binary64 for a pair from combine_ff (|e| <= ulp(s) / 2, so
// s + e has at most 49 significant bits), built with integer operations:
// the binary32 mantissa of s widened, e added in units of the result's last
// place; flushed to zero below the normal range
__device__ __forceinline__ double ff_to_double(float s, float e, int P) {
  if (s == 0.f) return 0.0;
  const uint32_t bs = __float_as_uint(s);
  const int Es = (int)((bs >> 23) & 0xFF) - 127;   // s is an integer combination, >= 2^-36: normal
  const long long ms = (long long)((bs & 0x7FFFFFu) | 0x800000u) << 29;
  const int me = __float2int_rn(__fmul_rn(e, pow2f(52 - Es)));   // |.| <= 2^28
  long long m = ms + ((bs >> 31) ? -(long long)me : (long long)me);
  int ex = Es + 1023 + P;
  if (m >= (1ll << 53)) {
    m = (m + 1) >> 1;
    ++ex;
  } else if (m < (1ll << 52)) {
    m <<= 1;
    --ex;
  }
  if (ex <= 0) return 0.0;
  return __longlong_as_double((long long)(((unsigned long long)(bs >> 31) << 63) |
                                          ((unsigned long long)ex << 52) |
                                          ((unsigned long long)m & ((1ull << 52) - 1))));
}
// (s, e) 2^P as a float-float pair (two exact power-of-two factors; zero
// below binary32's range, which sums of this path never reach)
__device__ __forceinline__ void ff_scale(float& s, float& e, int P) {
  const int p1 = P / 2, p2 = P - p1;
  if (p1 < -126 || p2 < -126) {
    s = e = 0.f;
    return;
  }
  const float f1 = pow2f(min(p1, 126)), f2 = pow2f(min(p2, 126));
  s = __fmul_rn(__fmul_rn(s, f1), f2);
  e = __fmul_rn(__fmul_rn(e, f1), f2);
}

}  // namespace tc
}  // namespace tp
