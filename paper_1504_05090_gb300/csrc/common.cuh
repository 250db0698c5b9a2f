// Shared device helpers of libdqmc: Philox4x32-10, lattice geometry, the
// argument blocks passed by value to the kernels, and launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

namespace dqmc {

constexpr int kMaxSide = 16;
constexpr int kMaxN = kMaxSide * kMaxSide;  // 256 sites
constexpr int kMaxDelay = 32;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor bijection with a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Uniform double in [0, 1) from the top 53 of the 64 bits (x0:x1).
__device__ __forceinline__ double uniform53(uint32_t x0, uint32_t x1) {
  const uint64_t b = ((static_cast<uint64_t>(x0) << 32) | x1) >> 11;
  return static_cast<double>(b) * 0x1.0p-53;
}

// |x| by clearing the sign bit (exact for every double, NaN stays NaN).  Used
// instead of the fabs overload set, which under this build's host-constexpr
// relaxation returned its argument unchanged in device code.
__device__ __forceinline__ double absd(double x) {
  return __longlong_as_double(__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL);
}

// ---------------------------------------------------------------------------
// df32: an unevaluated sum hi + lo of two floats (about 48 significant bits),
// with the error-free transformations TwoSum (Knuth) and FMA-based TwoProd
// (Dekker's double-length arithmetic).  It runs on the FP32 pipe, which on
// GB300 issues 59x more FMAs per second than the FP64 pipe.  Exponent range
// is that of FP32; the sweep's G, U, V and exp(-dtau K) entries are O(1).
// ---------------------------------------------------------------------------
struct __align__(8) df32 {
  float hi, lo;
  df32() = default;
  __host__ __device__ __forceinline__ constexpr df32(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ df32(int x) : hi(static_cast<float>(x)), lo(0.0f) {}
  __host__ __device__ __forceinline__ df32(float x) : hi(x), lo(0.0f) {}
  __host__ __device__ __forceinline__ df32(double x)
      : hi(static_cast<float>(x)), lo(static_cast<float>(x - static_cast<double>(static_cast<float>(x)))) {}
  __host__ __device__ __forceinline__ explicit operator double() const {
    return static_cast<double>(hi) + static_cast<double>(lo);
  }
};

__device__ __forceinline__ df32 df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df32(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ df32 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df32(s, b - (s - a));
}
__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
  const df32 s = df_two_sum(x.hi, y.hi);
  const df32 t = df_two_sum(x.lo, y.lo);
  const df32 u = df_fast_two_sum(s.hi, s.lo + t.hi);
  return df_fast_two_sum(u.hi, u.lo + t.lo);
}
__device__ __forceinline__ df32 operator-(df32 x) { return df32(-x.hi, -x.lo); }
__device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }
__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df32& operator+=(df32& x, df32 y) { return x = x + y; }
__device__ __forceinline__ df32& operator-=(df32& x, df32 y) { return x = x - y; }
__device__ __forceinline__ df32& operator*=(df32& x, df32 y) { return x = x * y; }
// a * b + c in the working precision (one overload set, so that no type converts).
__device__ __forceinline__ float madd(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double madd(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ df32 madd(df32 a, df32 b, df32 c) { return a * b + c; }

// Sum of products s = sum_m u_m v_m.  For df32 the products are accumulated
// with one TwoSum per term into (hi, lo) and rounded once at the end (about
// 12 FP32 instructions per term instead of 27 for an exact df32 multiply-add;
// relative error ~ m 2^-48).
template <typename T>
struct ProdSum {
  T s;
  __device__ __forceinline__ ProdSum() : s(T(0)) {}
  __device__ __forceinline__ void add(T u, T v) { s = madd(u, v, s); }
  __device__ __forceinline__ T get() const { return s; }
};
template <>
struct ProdSum<df32> {
  float hi, lo;
  __device__ __forceinline__ ProdSum() : hi(0.0f), lo(0.0f) {}
  __device__ __forceinline__ void add(df32 u, df32 v) {
    const float p = u.hi * v.hi;
    float e = fmaf(u.hi, v.hi, -p);
    e = fmaf(u.hi, v.lo, e);
    e = fmaf(u.lo, v.hi, e);
    const float t = hi + p;
    const float bb = t - hi;
    lo += ((hi - (t - bb)) + (p - bb)) + e;
    hi = t;
  }
  __device__ __forceinline__ df32 get() const { return df_fast_two_sum(hi, lo); }
};

// Counter tags of the two random streams.
constexpr uint32_t kTagProposal = 0u;
constexpr uint32_t kTagInitField = 1u;

// ---------------------------------------------------------------------------
// Geometry: site i = x + Lx*y on a periodic Lx x Ly cluster.
// ---------------------------------------------------------------------------
struct Geom {
  int Lx, Ly, N;
};

// Site index of (i shifted by -r) used by the separation bins r = r_i - r_j.
__device__ __forceinline__ int sep_index(int i, int j, const Geom& g) {
  const int xi = i % g.Lx, yi = i / g.Lx, xj = j % g.Lx, yj = j / g.Lx;
  const int rx = (xi - xj + g.Lx) % g.Lx, ry = (yi - yj + g.Ly) % g.Ly;
  return rx + g.Lx * ry;
}

// ---------------------------------------------------------------------------
// Kronecker application of exp(-+dtau K) = Ey (x) Ex to vectors of length N,
// optionally combined with the diagonal exp(+-sigma lambda s_l).  Ex and Ey
// are circulant: Ex[x][x'] = ex[(x - x') mod Lx].  Kinds:
//   kB   : v <- E  (e^{+c s_l} o v)     = B_l v          (c = sigma lambda)
//   kBT  : v <- e^{+c s_l} o (E v)      = B_l^T v
//   kBIT : v <- E^{-1} (e^{-c s_l} o v) = B_l^{-T} v
// ---------------------------------------------------------------------------
enum KronKind : int { kB = 0, kBT = 1, kBIT = 2 };

struct KronTaps {
  double ex[kMaxSide], ey[kMaxSide];    // circulant taps of exp(-dtau K_x), exp(-dtau K_y)
  double exi[kMaxSide], eyi[kMaxSide];  // taps of the inverses
};

// Error/status word written by device code (never trapped).
enum DevStatus : int { kDevOk = 0, kDevBadArg = 1, kDevNonFinite = 2, kDevSingular = 3, kDevTimeout = 4 };

}  // namespace dqmc
