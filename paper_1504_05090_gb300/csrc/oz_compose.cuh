// Rounding of the digit-product sums to FP64 with integer instructions only.
//
// The epilogues of the tensor-core FP64 products (Sec. 2: the stabilised
// matrix products behind Eq. (3)) hold, per output element, the exact value
//   v = 2^E (hi + 2^-28 lo)
// with 64-bit integers hi and lo below 2^47 in magnitude.  Converting hi and
// lo to FP64 and combining them with one FMA rounds v once, but each of those
// three instructions runs on the FP64 pipe, which issues two lanes per clock
// and SM on GB300 (against 64 for integer instructions).  oz_compose forms
// the same correctly rounded value (round to nearest, ties to even) from the
// integers: with W = hi 2^28 + lo = H 2^28 + R (H = floor(W / 2^28),
// 0 <= R < 2^28), the leading bit P of |W| fixes the 53-bit significand, the
// bits of R below it give the guard and sticky bits, and P + E the exponent
// field.  ok = false (value unusable) when the result would be subnormal,
// infinite or zero-exponent; the caller then takes the FP64 path.  A zero W
// gives +0 with ok = true.
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace dqmc {

__host__ __device__ __forceinline__ int oz_clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(x));
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ int oz_clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz(static_cast<int>(x));
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// v = (-1)^neg 2^E (hi + 2^-28 lo), |hi|, |lo| < 2^47.
__host__ __device__ __forceinline__ double oz_compose(long long hi, long long lo, int E, bool neg,
                                                     bool& ok) {
  long long H = hi + (lo >> 28);  // arithmetic shift: floor(lo / 2^28)
  uint32_t R = static_cast<uint32_t>(lo) & 0x0FFFFFFFu;
  if (H < 0) {  // |W| = (-H - 1) 2^28 + (2^28 - R), or -H 2^28 when R = 0
    neg = !neg;
    if (R != 0u) {
      H = ~H;
      R = 0x10000000u - R;
    } else {
      H = -H;
    }
  }
  const uint64_t Hu = static_cast<uint64_t>(H);
  if (Hu == 0 && R == 0u) {
    ok = true;
    return 0.0;
  }
  // leading bit of |W| = Hu 2^28 + R
  const int P = (Hu != 0) ? (63 - oz_clz64(Hu) + 28) : (31 - oz_clz32(R));
  uint64_t m;
  int Pr = P;
  if (P <= 52) {  // |W| < 2^53: exact
    m = ((Hu << 28) | R) << (52 - P);
  } else {  // drop s = P - 52 (1 .. 22) bits, all of them in R
    const int s = P - 52;
    m = (Hu << (28 - s)) | (R >> s);
    const uint32_t guard = (R >> (s - 1)) & 1u;
    const uint32_t sticky = R & ((1u << (s - 1)) - 1u);
    if (guard && (sticky != 0u || (m & 1u))) {
      ++m;
      if (m >> 53) {
        m >>= 1;
        ++Pr;
      }
    }
  }
  const int ef = Pr + E + 995;  // value = m 2^(Pr - 52 - 28 + E), m in [2^52, 2^53)
  ok = ef > 0 && ef < 2047;
  const uint64_t bits = (static_cast<uint64_t>(neg) << 63) | (static_cast<uint64_t>(ef & 0x7FF) << 52) |
                        (m & ((1ULL << 52) - 1));
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(bits));
#else
  double d;
  __builtin_memcpy(&d, &bits, sizeof d);
  return d;
#endif
}

}  // namespace dqmc
