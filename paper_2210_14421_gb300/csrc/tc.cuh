// Fifth-generation tensor-core (tcgen05) building blocks for sm_103a: tensor-memory
// allocation, shared-memory matrix descriptors, the bf16 x bf16 -> f32 MMA issued by
// one thread, completion through an mbarrier with a bounded wait, and accumulator
// loads back to registers.  Operands are kept in the no-swizzle K-major layout:
// an R x K bf16 tile is a grid of 8-row x 16-byte core matrices, element (r, k) at
//   (r % 8) * 16 + (r / 8) * SBO + (k % 8) * 2 + (k / 8) * LBO      (bytes)
// with LBO = 128 (core matrices adjacent along K) and SBO = (K / 8) * 128.
#pragma once
#include <cstdint>

namespace efe {
namespace tc {

constexpr uint32_t kLBO = 128;

__host__ __device__ constexpr uint32_t kmajor_offset(int r, int k, uint32_t sbo) {
  return (uint32_t)(r & 7) * 16u + (uint32_t)(r >> 3) * sbo + (uint32_t)(k & 7) * 2u + (uint32_t)(k >> 3) * kLBO;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte
// offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both K-major,
// N >> 3 in bits 17..22, M >> 4 in bits 24..28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// --- tensor memory (one warp) ---
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core's (async) proxy
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, one thread
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}
// the same, executed by a converged warp and issued by its lane 0 (the predicate is formed inside the
// instruction block, so the operands stay warp-uniform; lane 0 also commits, see mma_commit_lane0)
__device__ __forceinline__ void mma_bf16_lane0(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred e, p;\n\t.reg .u32 l;\n\t"
      "mov.u32 l, %%laneid;\n\t"
      "setp.eq.u32 e, l, 0;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit_lane0(uint64_t* mbar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\t.reg .u32 l;\n\t"
      "mov.u32 l, %%laneid;\n\t"
      "setp.eq.u32 e, l, 0;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}\n" ::"r"(
          smem_u32(mbar))
      : "memory");
}
// arrive on the mbarrier once every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
               : "memory");
}

// --- mbarrier ---
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
// Wait for completion of phase `parity`; gives up after `limit` polls (returns false).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(mbar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// --- accumulator loads: warp w reads lanes 32 (w % 4) .. + 31, 8 consecutive columns ---
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// three 8-column loads, one wait
__device__ __forceinline__ void tmem_ld8x3(uint32_t t0, uint32_t t1, uint32_t t2, float* a, float* b, float* c) {
  uint32_t r[24];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(t0)
               : "memory");
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(t1)
               : "memory");
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
               : "r"(t2)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[8 + i]);
    c[i] = __uint_as_float(r[16 + i]);
  }
}

// two 8-column stores (lanes of this warp's quarter), then the wait for them
__device__ __forceinline__ void tmem_st8x2(uint32_t t0, uint32_t t1, const float* a, const float* b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(t0),
               "r"(__float_as_uint(a[0])), "r"(__float_as_uint(a[1])), "r"(__float_as_uint(a[2])),
               "r"(__float_as_uint(a[3])), "r"(__float_as_uint(a[4])), "r"(__float_as_uint(a[5])),
               "r"(__float_as_uint(a[6])), "r"(__float_as_uint(a[7]))
               : "memory");
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(t1),
               "r"(__float_as_uint(b[0])), "r"(__float_as_uint(b[1])), "r"(__float_as_uint(b[2])),
               "r"(__float_as_uint(b[3])), "r"(__float_as_uint(b[4])), "r"(__float_as_uint(b[5])),
               "r"(__float_as_uint(b[6])), "r"(__float_as_uint(b[7]))
               : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// two 8-column loads and one wait
__device__ __forceinline__ void tmem_ld8x2(uint32_t t0, uint32_t t1, float* a, float* b) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(t0)
               : "memory");
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(t1)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a[i] = __uint_as_float(r[i]);
    b[i] = __uint_as_float(r[8 + i]);
  }
}

// --- mbarrier arrivals, bulk (non-tensor) copies global -> shared, L2 prefetch ---
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
// arrive and add `bytes` to the transaction count the current phase waits for
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
               : "memory");
}
// `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to this CTA's shared memory,
// completing as transactions on `mbar`
__device__ __forceinline__ void bulk_g2s(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ void bulk_prefetch_l2(const void* g, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(bytes) : "memory");
}
// barrier `id` (1..15) among n threads of whole warps (the warps that execute it)
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// --- splitting on the FP32 pipe ---
// alpha = a + b (|a| < 1, |b| <= ulp(a)) cut into four values r_k on the grids 2^-7, 2^-15,
// 2^-23 and 2^-31 by round-to-nearest digit extraction: each step adds and removes
// 1.5 * 2^(23 - q), which rounds to the grid 2^-q, and the remainder is exact; |r_0| <= 1,
// |r_k| <= 2^(-8k) for k >= 1, so every r_k has at most 8 significant bits and its bf16
// pattern is the upper half of its binary32 pattern.  |alpha - sum r_k| <= 2^-32 + 2^-33.
__device__ __forceinline__ void digits4(float a, float b, uint32_t bits[4]) {
  const float r0 = __fsub_rn(__fadd_rn(a, 98304.0f), 98304.0f);
  float t = __fadd_rn(__fsub_rn(a, r0), b);
  const float r1 = __fsub_rn(__fadd_rn(t, 384.0f), 384.0f);
  t = __fsub_rn(t, r1);
  const float r2 = __fsub_rn(__fadd_rn(t, 1.5f), 1.5f);
  t = __fsub_rn(t, r2);
  const float r3 = __fsub_rn(__fadd_rn(t, 0.005859375f), 0.005859375f);
  bits[0] = __float_as_uint(r0);
  bits[1] = __float_as_uint(r1);
  bits[2] = __float_as_uint(r2);
  bits[3] = __float_as_uint(r3);
}
// two bf16 patterns (the upper halves of two binary32 patterns) in one 32-bit word, lo first
__device__ __forceinline__ uint32_t pack_hi16(uint32_t lo, uint32_t hi) { return __byte_perm(lo, hi, 0x7632); }
// 2^-e as a binary32 for -126 <= e <= 126
__device__ __forceinline__ float exp2_neg(int e) { return __uint_as_float((uint32_t)(127 - e) << 23); }

// --- Ampere-style asynchronous 16-byte copies global -> shared ---
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// --- splitting a float64 into four bf16 slices ---
// x = 2^e * alpha with |alpha| <= 1 is rounded to alpha ~ Q 2^-31 (|Q| <= 2^31) and
// |Q| cut into 7 + 8 + 8 + 8 bits c0..c3, slice k carrying sign(x) c_k 2^-(7 + 8k).
// Each slice has at most 8 significant bits, so it is exact in bf16; returns the
// bf16 bit patterns.
__device__ __forceinline__ uint16_t bf16_of_chunk(uint32_t c, int k, uint32_t sign) {
  if (c == 0u) return 0;
  const int msb = 31 - __clz((int)c);                       // 0..7 (c0 may be 128: msb 7)
  const uint32_t mant = (c << (7 - msb)) & 0x7Fu;
  const uint32_t ex = (uint32_t)(msb - 7 - 8 * k + 127);
  return (uint16_t)(sign | (ex << 7) | mant);
}
// alpha already scaled: q31 = |alpha| 2^31 rounded, sign in bit 15
__device__ __forceinline__ void split4(long long Q, uint16_t s[4]) {
  const uint32_t sign = Q < 0 ? 0x8000u : 0u;
  const unsigned long long q = (unsigned long long)(Q < 0 ? -Q : Q);
  s[0] = bf16_of_chunk((uint32_t)(q >> 24), 0, sign);
  s[1] = bf16_of_chunk((uint32_t)((q >> 16) & 255u), 1, sign);
  s[2] = bf16_of_chunk((uint32_t)((q >> 8) & 255u), 2, sign);
  s[3] = bf16_of_chunk((uint32_t)(q & 255u), 3, sign);
}
// --- float64 <-> fixed point on the integer pipes (GB300's float64 pipe is ~1/64 of float32) ---
// round(x 2^(31 - e)) for |x| < 2^e, from the bit pattern of x (ties away from zero)
__device__ __forceinline__ long long q31_bits(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)(b >> 52) & 0x7FF;
  if (be == 0) return 0;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = e + 1044 - be;   // right shift of the 53-bit significand, >= 22 since |x| < 2^e
  if (sh >= 64) return 0;
  const long long q = (long long)((m + (1ull << (sh - 1))) >> sh);
  return (b >> 63) ? -q : q;
}
// A float64 as a 64-bit significand and exponent: |x| = m 2^e with m in [2^63, 2^64)
// (m = 0 for zero and subnormals).
struct Wide {
  unsigned long long m;
  int e;
  bool neg;
};
__device__ __forceinline__ Wide wide_of(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)(b >> 52) & 0x7FF;
  if (be == 0) return Wide{0ull, 0, false};
  return Wide{((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 11, be - 1086, (b >> 63) != 0};
}
// x d for d > 0 given as its 64-bit significand dm and exponent de (the product's low
// 64 bits are dropped: relative error below 2^-62)
__device__ __forceinline__ Wide wide_mul(Wide x, unsigned long long dm, int de) {
  if (x.m == 0ull) return x;
  unsigned long long h = __umul64hi(x.m, dm);   // in [2^62, 2^64)
  int e = x.e + de + 64;
  if (!(h >> 63)) {
    h <<= 1;
    e -= 1;
  }
  return Wide{h, e, x.neg};
}
// floor(log2 |x|) + 2048 (0 for zero): an order-preserving key for the largest |x|
__device__ __forceinline__ int wide_key(Wide x) { return x.m ? x.e + 63 + 2048 : 0; }
// round(|x| 2^(31 - e)) with sign, for |x| < 2^e
__device__ __forceinline__ long long q31_wide(Wide x, int e) {
  if (x.m == 0ull) return 0;
  const int sh = e - 31 - x.e;   // >= 33 since x.m >= 2^63 and |x| < 2^e
  if (sh >= 65) return 0;
  const long long q = (long long)(((x.m >> (sh - 1)) + 1ull) >> 1);
  return x.neg ? -q : q;
}

// x 2^q as an integer (bits below 2^-q dropped), from the bit pattern of a float
__device__ __forceinline__ long long fixed_of_float(float x, int q) {
  const uint32_t b = __float_as_uint(x);
  const int be = (int)(b >> 23) & 0xFF;
  if (be == 0) return 0;
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = be - 150 + q;    // m 2^(be - 150) = |x|
  long long v;
  if (sh >= 0) v = m << sh;
  else v = sh > -32 ? (m >> -sh) : 0;
  return (b >> 31) ? -v : v;
}
// I 2^e as a double (the bits below the 53 kept are dropped), from integer operations
__device__ __forceinline__ double double_of_fixed(long long I, int e) {
  if (I == 0) return 0.0;
  const unsigned long long sign = I < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = (unsigned long long)(I < 0 ? -I : I);
  const int p = 63 - __clzll((long long)u);   // leading bit
  const int ex = p + e + 1023;
  if (ex <= 0 || ex >= 2047) return 0.0;
  u = p > 52 ? (u >> (p - 52)) : (u << (52 - p));
  return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) | (u & 0xFFFFFFFFFFFFFull)));
}

// I1 2^e1 + I2 2^e2 as a double: the addend with the smaller exponent is shifted onto the other's
// grid (an error below one unit of that grid); |I1|, |I2| < 2^55
__device__ __forceinline__ double double_of_fixed2(long long I1, int e1, long long I2, int e2) {
  if (I2 == 0) return double_of_fixed(I1, e1);
  if (I1 == 0) return double_of_fixed(I2, e2);
  if (e1 < e2) {
    const long long ti = I1;
    I1 = I2;
    I2 = ti;
    const int te = e1;
    e1 = e2;
    e2 = te;
  }
  const int d = e1 - e2;
  return double_of_fixed(I1 + (d < 63 ? (I2 >> d) : (I2 < 0 ? -1LL : 0LL)), e1);
}

// --- float-pair epilogue arithmetic ---
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// a0 + a1 + a2 (+ c0 + c1) as a normalised pair (s, t), |t| <= ulp(s) / 2; the rounding of the
// small terms' sum is far below the last bit of s
__device__ __forceinline__ void sum3_pair(float a0, float a1, float a2, float& s, float& t) {
  float s1, e1, s2, e2;
  two_sum_f(a0, a1, s1, e1);
  two_sum_f(s1, a2, s2, e2);
  two_sum_f(s2, __fadd_rn(e1, e2), s, t);
}
__device__ __forceinline__ void sum5_pair(float a0, float a1, float a2, float c0, float c1, float& s, float& t) {
  float s1, e1, s2, e2, s3, e3;
  two_sum_f(a0, c0, s1, e1);
  two_sum_f(s1, a1, s2, e2);
  two_sum_f(s2, a2, s3, e3);
  two_sum_f(s3, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, c1)), s, t);
}
// (s + t) 2^E as a double from integer operations only, for a normalised pair (|t| <= ulp(s) / 2):
// the pattern of s 2^E, plus t counted in units of the double's last place (for t against the
// sign of s across a power of two the result is within a few units of the last place)
__device__ __forceinline__ double double_of_pair(float s, float t, int E) {
  const uint32_t us = __float_as_uint(s);
  const int bs = (int)((us >> 23) & 0xFFu);
  if (bs == 0) return 0.0;
  const int ed = bs + 896 + E;
  if (ed <= 0 || ed >= 2047) return 0.0;
  unsigned long long mag = ((unsigned long long)ed << 52) | ((unsigned long long)(us & 0x7FFFFFu) << 29);
  const uint32_t ut = __float_as_uint(t);
  const int bt = (int)((ut >> 23) & 0xFFu);
  if (bt != 0) {
    const unsigned long long mt = (ut & 0x7FFFFFu) | 0x800000u;
    const int sh = bt - bs + 29;   // t / ulp = mt 2^(bt - bs + 29), bt <= bs - 24
    const unsigned long long q = sh >= 0 ? (mt << sh) : (sh > -25 ? (mt >> -sh) : 0ull);
    mag = ((ut ^ us) >> 31) ? mag - q : mag + q;
  }
  return __longlong_as_double((long long)((((unsigned long long)us >> 31) << 63) | mag));
}
// 2^k as a binary32 for -126 <= k <= 127
__device__ __forceinline__ float exp2_pos(int k) { return __uint_as_float((uint32_t)(127 + k) << 23); }

// exponent e with |x| < 2^e for the largest |x| whose biased exponent is be (be > 0)
__device__ __forceinline__ int scale_exp(int be) { return be - 1022; }
__device__ __forceinline__ int biased_exp(double x) {
  return (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
}

}  // namespace tc
}  // namespace efe
