// Device helpers of the digit-split (Ozaki) FP64 products, shared by the GEMM (qtt_ozaki.cu)
// and the tensor-core ALS local solve (qtt_cg_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace qtt {
namespace {

constexpr int OZ_S = 7;            // digits per operand

// The fixed-point integer F = round(x 2^(8S - e)) of an FP64 value, from its bit pattern with
// integer operations only (|x| 2^-e < 1/2 gives |F| < 2^(8S-1)); zeros, subnormals, infinities
// and NaNs give 0 (callers flag non-finite operands through the exponent field 0x7ff).
__device__ __forceinline__ long long oz_fixed(double x, int e) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
  const int bexp = int((bits >> 52) & 0x7ff);
  if (bexp == 0 || bexp == 0x7ff) return 0;
  const long long mant = static_cast<long long>((bits & 0xfffffffffffffull) | 0x10000000000000ull);
  const int sh = bexp - 1075 + 8 * OZ_S - e;
  long long v;
  if (sh >= 0) v = mant << sh;
  else if (sh > -63) v = (mant + (1ll << (-sh - 1))) >> (-sh);
  else v = 0;
  return (bits >> 63) ? -v : v;
}

// Exponent field of x (0 for zero and subnormals, 0x7ff for infinities and NaNs).
__device__ __forceinline__ int oz_field(double x) {
  return int((static_cast<unsigned long long>(__double_as_longlong(x)) >> 52) & 0x7ff);
}

// Scale exponent of a row or column from the largest exponent field mx of its entries:
// max |x| < 2^(mx - 1022), so e = mx - 1021 gives |x| 2^-e < 1/2 (0 for a zero row).
__device__ __forceinline__ int oz_scale(int mx) { return mx > 0 ? mx - 1021 : 0; }

// value G 2^shift added exactly to the 128-bit fixed-point accumulator (hi 2^64 + lo);
// |G| < 2^24, 0 <= shift <= 48.
__device__ __forceinline__ void oz_acc(long long& hi, unsigned long long& lo, long long G, int shift) {
  unsigned long long add_lo;
  long long add_hi;
  if (shift >= 32) {
    const long long v = G << (shift - 32);
    add_lo = static_cast<unsigned long long>(v) << 32;
    add_hi = v >> 32;
  } else {
    const long long v = G << shift;
    add_lo = static_cast<unsigned long long>(v);
    add_hi = v >> 63;
  }
  const unsigned long long nl = lo + add_lo;
  hi += add_hi + (nl < add_lo ? 1 : 0);
  lo = nl;
}

// (hi, lo) += (h2, l2), exact.
__device__ __forceinline__ void oz_add128(long long& hi, unsigned long long& lo, long long h2, unsigned long long l2) {
  const unsigned long long nl = lo + l2;
  hi += h2 + (nl < l2 ? 1 : 0);
  lo = nl;
}

// (hi 2^64 + lo) 2^E as a double, rounded to nearest even, by integer operations on the bit
// pattern (the FP64 unit of this part is ~64x slower than its integer units).  |value| < 2^127.
__device__ __forceinline__ double fixed_to_double(long long hi, unsigned long long lo, int E) {
  const bool neg = hi < 0;
  unsigned long long h = static_cast<unsigned long long>(hi), l = lo;
  if (neg) {
    l = ~l + 1ull;
    h = ~h + (l == 0ull ? 1ull : 0ull);
  }
  if (h == 0ull && l == 0ull) return 0.0;
  // normalise so that bit 127 is set
  const int lz = h ? __clzll(static_cast<long long>(h)) : 64 + __clzll(static_cast<long long>(l));
  if (lz >= 64) {
    h = l << (lz - 64);
    l = 0ull;
  } else if (lz > 0) {
    h = (h << lz) | (l >> (64 - lz));
    l <<= lz;
  }
  unsigned long long m = h >> 11;                                  // 53 bits
  const bool guard = (h >> 10) & 1ull;
  const bool sticky = ((h & 0x3ffull) != 0ull) || (l != 0ull);
  int X = 127 - lz + E;                                           // exponent of the leading bit
  if (guard && (sticky || (m & 1ull))) {
    ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++X;
    }
  }
  if (X < -1022 || X > 1023) {                                    // outside the normal range
    const double r = scalbn(static_cast<double>(m), X - 52);
    return neg ? -r : r;
  }
  const unsigned long long bits = (neg ? (1ull << 63) : 0ull) | (static_cast<unsigned long long>(X + 1023) << 52) |
                                  (m & 0xfffffffffffffull);
  return __longlong_as_double(static_cast<long long>(bits));
}

// 16-byte global -> shared copy that does not stall the thread; full = false writes zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool full) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  const int n = full ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(a), "l"(gmem), "r"(n) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}


__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}

}  // namespace
}  // namespace qtt
