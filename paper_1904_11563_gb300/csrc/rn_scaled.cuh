// RN_fp32(q 2^e) for an exact integer q (the exact-slice peel's final
// rounding), in integer arithmetic: keep the top 24 bits of |q| (fewer where
// the result is subnormal: its last bit is worth 2^-149), round the dropped
// bits to nearest even, and assemble the float's bits; a carry out of the
// significand moves into the exponent field, and a result past the largest
// float becomes infinity.  One rounding of the exact value, so the same bits
// as rounding the exact FP64 product q 2^e (|q| < 2^53) to FP32, without the
// FP64 pipe.  Host and device: the CPU tests compile it with the host
// compiler and compare it with the C library's rounding.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define BPX_RN_HD __host__ __device__ __forceinline__
#else
#define BPX_RN_HD inline
#endif

namespace bpx {

BPX_RN_HD int rn_clz64(uint64_t x) {  // x != 0
#if defined(__CUDA_ARCH__)
  return __clzll(static_cast<long long>(x));
#else
  return __builtin_clzll(x);
#endif
}

BPX_RN_HD float rn_bits_to_float(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
#endif
}

BPX_RN_HD float rn_float_scaled(long long q, int e) {
  if (q == 0) return 0.f;
  const uint32_t sign = q < 0 ? 0x80000000u : 0u;
  const uint64_t m = q < 0 ? 0ull - static_cast<uint64_t>(q) : static_cast<uint64_t>(q);
  const int top = 63 - rn_clz64(m);              // m in [2^top, 2^(top + 1))
  const int E = top + e;                         // result in [2^E, 2^(E + 1))
  const int keep = E >= -126 ? 24 : E + 150;     // significand bits the float holds
  if (keep < 0) return rn_bits_to_float(sign);   // below half the smallest subnormal
  const int drop = top + 1 - keep;
  uint64_t mant;
  if (drop <= 0) {
    mant = m << -drop;
  } else {
    mant = drop >= 64 ? 0ull : m >> drop;
    const uint64_t rem = drop >= 64 ? m : m & ((1ull << drop) - 1ull);
    const uint64_t half = 1ull << (drop - 1);
    mant += (rem > half || (rem == half && (mant & 1ull))) ? 1ull : 0ull;
  }
  // normal: ((E + 126) << 23) + mant, mant in [2^23, 2^24]; subnormal: mant
  const long long bits =
      E >= -126 ? (static_cast<long long>(E + 126) << 23) + static_cast<long long>(mant) : static_cast<long long>(mant);
  return rn_bits_to_float(sign | static_cast<uint32_t>(bits >= 0x7F800000LL ? 0x7F800000LL : bits));
}

}  // namespace bpx
