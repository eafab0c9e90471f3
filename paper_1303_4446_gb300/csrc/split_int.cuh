// Integer arithmetic of the split-precision path (host and device): exponents and fixed
// point from IEEE-754 bits, balanced base-256 digits, and int64 x 2^E back to double.  No
// floating-point arithmetic is used, so the results are exact and identical on any host.
#pragma once

#include <cstdint>
#include <cstring>

namespace x2c {

constexpr int kNoExp = -4000;

__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<unsigned long long>(__double_as_longlong(x));
#else
  unsigned long long b;
  std::memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double bits_to_double(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(b));
#else
  double x;
  std::memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ int clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(v));
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// e with |x| < 2^e (x normal); kNoExp for zero and subnormals.
__host__ __device__ __forceinline__ int frexp_exp(double x) {
  const int be = static_cast<int>((dbits(x) >> 52) & 0x7FF);
  return be == 0 ? kNoExp : be - 1022;
}

// round(x 2^shift) for |x 2^shift| < 2^62 (round half away from zero; subnormals -> 0).
__host__ __device__ __forceinline__ long long fixed_point(double x, int shift) {
  const unsigned long long b = dbits(x);
  const int be = static_cast<int>((b >> 52) & 0x7FF);
  if (be == 0) return 0;
  const long long m = static_cast<long long>((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int e = be - 1075 + shift;
  long long v;
  if (e >= 0) v = m << e;
  else if (e <= -62) v = 0;
  else v = (m + (1ll << (-e - 1))) >> (-e);
  return (b >> 63) ? -v : v;
}

// round(I 2^shift) for integers (round half up), |I 2^shift| < 2^62.
__host__ __device__ __forceinline__ long long shift_round(long long I, int shift) {
  if (shift >= 0) return I << shift;
  if (shift <= -62) return 0;
  return (I + (1ll << (-shift - 1))) >> (-shift);
}

// Balanced base-256 digits of F (|F| <= 2^(8S), S <= 6): F = sum_s d_s 2^8(S-1-s),
// d_s in [-128, 127] for s >= 1 and |d_0| <= 256.  For S >= 4 the low 24 bits and the high
// part are cut with 32-bit arithmetic (one carry between them).
template <int S>
__host__ __device__ __forceinline__ void digits(long long F, int (&d)[S]) {
  if constexpr (S <= 3) {
    for (int s = S - 1; s >= 1; --s) {
      const long long q = (F + 128) >> 8;
      d[s] = static_cast<int>(F - (q << 8));
      F = q;
    }
    d[0] = static_cast<int>(F);
  } else {
    int lo = static_cast<int>(F & 0xFFFFFF);
    int hi = static_cast<int>(F >> 24);
    for (int s = 0; s < 3; ++s) {
      const int dd = ((lo + 128) & 0xFF) - 128;
      d[S - 1 - s] = dd;
      lo = (lo - dd) >> 8;
    }
    hi += lo;  // carry (0 or 1) out of the low 24 bits
    for (int s = 3; s < S - 1; ++s) {
      const int dd = ((hi + 128) & 0xFF) - 128;
      d[S - 1 - s] = dd;
      hi = (hi - dd) >> 8;
    }
    d[0] = hi;
  }
}

// The IEEE-754 bits of I 2^E as a double, by integer operations only (round half up on the
// magnitude; underflow to a signed zero, overflow to a signed infinity).
__host__ __device__ __forceinline__ unsigned long long scaled_to_bits(long long I, int E) {
  if (I == 0) return 0ull;
  const unsigned long long neg = I < 0;
  const unsigned long long v = neg ? static_cast<unsigned long long>(-I) : static_cast<unsigned long long>(I);
  const int lz = clz64(v);
  const unsigned long long m = v << lz;
  unsigned long long mant = (m >> 11) + ((m >> 10) & 1ull);
  int ex = 63 - lz + E;
  if (mant >> 53) {
    mant >>= 1;
    ex += 1;
  }
  const int be = ex + 1023;
  if (be <= 0) return neg << 63;
  if (be >= 2047) return (neg << 63) | (0x7FFull << 52);
  return (neg << 63) | (static_cast<unsigned long long>(be) << 52) | (mant & 0xFFFFFFFFFFFFFull);
}

// I 2^E as a double (the value of scaled_to_bits).
__host__ __device__ __forceinline__ double scaled_to_double(long long I, int E) {
  return bits_to_double(scaled_to_bits(I, E));
}

}  // namespace x2c
