// Kronecker products with exp(-+dtau K) = E_y (x) E_x of Eq. (2) on the
// tcgen05 tensor cores, for the FP64 UDV stack products X = B_l ... B_1 (U D)
// (Sec. 2: the O(Lambda N^3) stabilised matrix work behind Eq. (3)).
//
// A vector v of length N = Lx Ly is the Ly x Lx grid V[y][x] = v[x + Lx y],
// and E v = E_y V E_x^T with the circulant E_x[x][x'] = ex[(x - x') mod Lx].
// Eight (in general 128 / max(Lx, Ly)) vectors of one matrix stay in shared
// memory for all the slices of a call.  Per slice:
//   x step: rows (vector, y) of length Lx times E_x^T      (M = 128, N = K = 16)
//   y step: rows (vector, x) of length Ly times E_y^T      (M = 128, N = K = 16)
// each one digit-sliced product as in k_ozaki.cu: every row of the left
// operand and every column of the taps is aligned to its largest exponent
// and cut into eight signed 7-bit digits (exact in BF16), the 36 digit
// products with p + q <= 7 accumulate in eight FP32 TMEM accumulators, and
// the epilogue recombines them exactly in 64-bit integers.  Rows and
// columns past Lx, Ly are zero padding.  The diagonal factor e^{+-c s_l} is
// an FP64 product per element, before (B, B^{-T}) or after (B^T) the taps.
//
// FP64 work per element and slice: the diagonal product and two
// recombinations (conversions and one FMA each), against Lx + Ly FMAs for the
// FP64 Kronecker kernel.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace dqmc {
namespace {

constexpr int kS = 8;       // digit slices
constexpr int kR = 128;     // rows of one product (TMEM lanes)
constexpr int kK = 16;      // inner dimension (padded side)
constexpr int kTC = 128;    // threads
constexpr long long kWaitLimit = 1LL << 26;
constexpr int kASlice = kR * kK * 2;   // bytes of one digit slice of the rows (4 KB)
constexpr int kBSlice = kK * kK * 2;   // of the taps (512 B)

__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// No-swizzle K-major descriptor: core matrices of 8 rows x 16 bytes, the next
// one along K 128 bytes on, the next 8 rows 256 bytes on (K = 16).
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  constexpr uint32_t lbo = 128, sbo = 256;
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}

// Element offset of (row r, k) in one digit slice.
__device__ __forceinline__ int tc_off(int r, int k) {
  return (r >> 3) * (kK / 8 * 64) + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, int parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kWaitLimit && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(tc_smem(bar)), "r"(parity));
  return done != 0;
}

// The 8 digits of x aligned to emax (as k_ozaki.cu), BF16 bit patterns.
__device__ __forceinline__ void tc_digits(double x, int emax, uint16_t (&dg)[kS]) {
  const long long bits = __double_as_longlong(x);
  const int E = static_cast<int>((bits >> 52) & 0x7FF);
  unsigned long long al = 0ULL;
  if (E != 0) {
    const unsigned long long mant =
        (static_cast<unsigned long long>(bits) & ((1ULL << 52) - 1)) | (1ULL << 52);
    const int sh = emax - (E - 1023);
    al = (sh < 64) ? (mant >> sh) : 0ULL;
  }
  const float sg = (bits < 0) ? -1.0f : 1.0f;
#pragma unroll
  for (int p = 0; p < kS; ++p) {
    const int d = (p < 7) ? static_cast<int>((al >> (46 - 7 * p)) & 127ULL)
                          : static_cast<int>((al & 15ULL) << 3);
    const __nv_bfloat16 hb = __float2bfloat16_rn(sg * static_cast<float>(d));
    dg[p] = *reinterpret_cast<const uint16_t*>(&hb);
  }
}

// Digits of the taps as the right operand: column j, inner index k,
// t[(j - k) mod n] for j, k < n (zero padding beyond); column exponents out.
__device__ void tc_tap_digits(const double* t, int n, unsigned char* bs, int* ex) {
  for (int j = threadIdx.x; j < kK; j += blockDim.x) {
    int emax = -100000;
    for (int k = 0; k < n && j < n; ++k) {
      const double v = t[((j - k) % n + n) % n];
      const int E = static_cast<int>((__double_as_longlong(v) >> 52) & 0x7FF);
      if (E != 0) emax = max(emax, E - 1023);
    }
    ex[j] = emax - 6;
    for (int k = 0; k < kK; ++k) {
      const double v = (j < n && k < n) ? t[((j - k) % n + n) % n] : 0.0;
      uint16_t dg[kS];
      tc_digits(v, emax, dg);
      for (int p = 0; p < kS; ++p)
        reinterpret_cast<uint16_t*>(bs + p * kBSlice)[tc_off(j, k)] = dg[p];
    }
  }
}

// Shared-memory state of one CTA of the tensor-core Kronecker kernels.
struct TcState {
  unsigned char* as;  // digit slices of the rows (8 x 4 KB)
  unsigned char* bx;  // digit slices of the taps along x (8 x 512 B)
  unsigned char* by;  // along y
  double* V;          // the CTA's vectors [nvpc][N]
  uint64_t* mbar;     // MMA completion
  int* exx;           // column exponents of the taps
  int* exy;
  int* fail;          // a bounded wait gave up
  uint32_t tbase;     // TMEM accumulators (8 x 16 columns)
};

// TMEM, barrier and the digits of the taps of E_x, E_y (kind: E or E^{-1}).
__device__ void tc_setup(TcState& s, uint32_t* tmem_sh, const KronTaps& taps, bool inv, double* tx,
                         double* ty, int Lx, int Ly) {
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
        tc_smem(tmem_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(s.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    *s.fail = 0;
  }
  if (threadIdx.x < kMaxSide) {
    tx[threadIdx.x] = inv ? taps.exi[threadIdx.x] : taps.ex[threadIdx.x];
    ty[threadIdx.x] = inv ? taps.eyi[threadIdx.x] : taps.ey[threadIdx.x];
  }
  __syncthreads();
  tc_tap_digits(tx, Lx, s.bx, s.exx);
  tc_tap_digits(ty, Ly, s.by, s.exy);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  s.tbase = *tmem_sh;
}

__device__ void tc_teardown(const TcState& s) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(s.tbase));
}

// One factor B on the nv vectors in s.V: the diagonal sc before the taps
// (post = false: B, B^{-T}) or after them (post = true: B^T), then the x and
// y steps as digit-sliced products.  All threads; false if a wait gave up.
__device__ bool tc_slice(TcState& s, const double* sc, bool post, int nv, int N, int Lx, int Ly,
                         int& phase) {
  const int warp = threadIdx.x >> 5;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kK >> 3) << 17) | ((kR >> 4) << 24);
  double* V = s.V;
  if (!post)
    for (int e = threadIdx.x; e < nv * N; e += blockDim.x) V[e] *= sc[e % N];
  __syncthreads();
  const int r = threadIdx.x;  // the row of both products this thread owns
  for (int dir = 0; dir < 2; ++dir) {
    // row r: (vector, y) with elements x' (x step) or (vector, x) with y' (y step)
    const int side = dir == 0 ? Ly : Lx, klen = dir == 0 ? Lx : Ly;
    const int vi = r / side, o = r - vi * side;
    const bool live = vi < nv;
    double row[kK];
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      double v = 0.0;
      if (live && k < klen) v = (dir == 0) ? V[vi * N + k + Lx * o] : V[vi * N + o + Lx * k];
      row[k] = v;
    }
    int emax = -100000;
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      const int E = static_cast<int>((__double_as_longlong(row[k]) >> 52) & 0x7FF);
      if (E != 0) emax = max(emax, E - 1023);
    }
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      uint16_t dg[kS];
      tc_digits(row[k], emax, dg);
#pragma unroll
      for (int p = 0; p < kS; ++p) reinterpret_cast<uint16_t*>(s.as + p * kASlice)[tc_off(r, k)] = dg[p];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned char* bs = dir == 0 ? s.bx : s.by;
    if (threadIdx.x == 0) {
      for (int d = 0; d < kS; ++d)
        for (int p = 0; p <= d; ++p) {
          const int q = d - p;
          const uint64_t ad = tc_desc(tc_smem(s.as + p * kASlice));
          const uint64_t bd = tc_desc(tc_smem(bs + q * kBSlice));
          const uint32_t acc = p > 0 ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred pa;\n setp.ne.u32 pa, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(s.tbase + d * kK),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          tc_smem(s.mbar)));
    }
    if (!tc_wait(s.mbar, phase)) *s.fail = 1;
    phase ^= 1;
    const bool ok = __syncthreads_and(*s.fail == 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) return false;
    // recombination: (hi + 2^-28 lo) 2^{e_r + f_j - 21}, the power of two in
    // the exponent field (FP64 products where it would leave the normal
    // range); the accumulators are read eight columns at a time
    const int* exj = dir == 0 ? s.exx : s.exy;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      uint32_t acc[kS][8];
#pragma unroll
      for (int d = 0; d < kS; ++d) {
        const uint32_t ta = s.tbase + (static_cast<uint32_t>(warp * 32) << 16) + d * kK + half * 8;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(acc[d][0]), "=r"(acc[d][1]), "=r"(acc[d][2]), "=r"(acc[d][3]), "=r"(acc[d][4]),
              "=r"(acc[d][5]), "=r"(acc[d][6]), "=r"(acc[d][7])
            : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (live) {
#pragma unroll
        for (int jq = 0; jq < 8; ++jq) {
          const int j = half * 8 + jq;
          if (j >= klen) continue;
          long long hi = 0, lo = 0;
#pragma unroll
          for (int d = 0; d < 4; ++d)
            hi += static_cast<long long>(__float2int_rn(__uint_as_float(acc[d][jq]))) << (7 * (3 - d));
#pragma unroll
          for (int d = 4; d < kS; ++d)
            lo += static_cast<long long>(__float2int_rn(__uint_as_float(acc[d][jq]))) << (7 * (7 - d));
          const double sum = fma(static_cast<double>(lo), 0x1p-28, static_cast<double>(hi));
          const int e2 = (emax - 6) + exj[j] - 21;
          const long long bits = __double_as_longlong(sum);
          const int E = static_cast<int>((bits >> 52) & 0x7FF), E2 = E + e2;
          double val;
          if (E != 0 && E != 0x7FF && E2 > 0 && E2 < 2047)
            val = __longlong_as_double((bits & ~(0x7FFLL << 52)) | (static_cast<long long>(E2) << 52));
          else
            val = sum * ldexp(1.0, emax - 6) * ldexp(1.0, exj[j] - 21);
          // rows are read above and written only here, each by its owner
          if (dir == 0)
            V[vi * N + j + Lx * o] = val;
          else
            V[vi * N + o + Lx * j] = val;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  if (post)
    for (int e = threadIdx.x; e < nv * N; e += blockDim.x) V[e] *= sc[e % N];
  __syncthreads();
  return true;
}

}  // namespace

// One CTA per (group of nvpc vectors, batch entry); the arguments and slice
// ranges are those of k_kron_rows<double>.
__global__ void __launch_bounds__(kTC) k_kron_tc(const double* in, double* out, KronArgs a,
                                                int nvpc, int* status) {
  const int b = blockIdx.y;
  int chain, first, count;
  chain = b / a.per_chain;
  if (a.cp) {
    const int blk = b - chain * a.per_chain;
    const int lo = a.cp[blk] + a.step, hi = a.cp[blk + 1];
    first = lo;
    count = (lo < hi) ? 1 : 0;
  } else {
    first = a.l0_first;
    count = a.n_slices;
  }
  const int N = a.N;
  const int v0 = blockIdx.x * nvpc;
  const int nv = min(nvpc, N - v0);
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  __shared__ int exx[kK], exy[kK], fail_sh;
  __shared__ double tx[kMaxSide], ty[kMaxSide], sc[kMaxN];
  TcState s;
  s.as = tc_sm;
  s.bx = s.as + kS * kASlice;
  s.by = s.bx + kS * kBSlice;
  s.V = reinterpret_cast<double*>(s.by + kS * kBSlice);
  s.mbar = &mbar;
  s.exx = exx;
  s.exy = exy;
  s.fail = &fail_sh;
  const double* src = in + static_cast<size_t>(b) * a.mat_stride;
  for (int e = threadIdx.x; e < nvpc * N; e += blockDim.x) {
    const int vi = e / N, i = e - vi * N;
    double val = 0.0;
    if (vi < nv) {
      val = src[static_cast<size_t>(v0 + vi) * N + i];
      if (a.vscale) val *= a.vscale[static_cast<size_t>(b) * a.vscale_stride + v0 + vi];
    }
    s.V[e] = val;
  }
  tc_setup(s, &tmem_sh, a.taps, a.kind == kBIT, tx, ty, a.Lx, a.Ly);
  const double up = (a.kind == kBIT) ? a.emc : a.ec, dn = (a.kind == kBIT) ? a.ec : a.emc;
  const int8_t* f = a.field + static_cast<size_t>(chain) * a.L * N;
  int phase = 0;
  bool ok = true;
  for (int stp = 0; stp < count && ok; ++stp) {
    const int l0 = first + stp * a.dir;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sc[i] = f[static_cast<size_t>(l0) * N + i] > 0 ? up : dn;
    __syncthreads();
    ok = tc_slice(s, sc, a.kind == kBT, nv, N, a.Lx, a.Ly, phase);
  }
  if (!ok && threadIdx.x == 0) atomicExch(status, kDevTimeout);
  double* dst = out + static_cast<size_t>(b) * a.out_stride;
  for (int e = threadIdx.x; e < nv * N; e += blockDim.x) {
    const int vi = e / N, i = e - vi * N;
    dst[static_cast<size_t>(v0 + vi) * N + i] = s.V[e];
  }
  tc_teardown(s);
}

// Unequal-time propagation of k_gtau_propagate on the tensor cores: the rows
// of one stabilisation point's G(c,0)^T (kind B) or Y (kind B^{-T}) are
// propagated over the slices of its block, and after each slice every
// element is added to the bin of its separation (spin-up G(l,0) bins or Y
// bins of slice l), first in shared memory, then into bins[chain][l][slot].
__global__ void __launch_bounds__(kTC) k_gtau_tc(const double* Xall, GtauArgs a, int nvpc,
                                                int* status) {
  const int b = blockIdx.y;
  const int chain = b / a.per_chain, blk = b - chain * a.per_chain;
  const int N = a.N;
  const int v0 = blockIdx.x * nvpc;
  const int nv = min(nvpc, N - v0);
  const int lo = a.cp[blk], hi = a.cp[blk + 1];
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  __shared__ int exx[kK], exy[kK], fail_sh;
  __shared__ double tx[kMaxSide], ty[kMaxSide], sc[kMaxN], sbin[kMaxN];
  TcState s;
  s.as = tc_sm;
  s.bx = s.as + kS * kASlice;
  s.by = s.bx + kS * kBSlice;
  s.V = reinterpret_cast<double*>(s.by + kS * kBSlice);
  s.mbar = &mbar;
  s.exx = exx;
  s.exy = exy;
  s.fail = &fail_sh;
  const double* X = Xall + static_cast<size_t>(b) * a.mat_stride;
  for (int e = threadIdx.x; e < nvpc * N; e += blockDim.x) {
    const int vi = e / N, i = e - vi * N;
    s.V[e] = (vi < nv) ? X[static_cast<size_t>(v0 + vi) * N + i] : 0.0;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) sbin[i] = 0.0;
  tc_setup(s, &tmem_sh, a.taps, a.kind == kBIT, tx, ty, a.Lx, a.Ly);
  const Geom g{a.Lx, a.Ly, N};
  const int8_t* f = a.field + static_cast<size_t>(chain) * a.L * N;
  const double up = (a.kind == kBIT) ? a.emc : a.ec, dn = (a.kind == kBIT) ? a.ec : a.emc;
  int phase = 0;
  bool ok = true;
  for (int l = lo; l < hi && ok; ++l) {
    if (l > lo) {
      for (int i = threadIdx.x; i < N; i += blockDim.x)
        sc[i] = f[static_cast<size_t>(l - 1) * N + i] > 0 ? up : dn;
      __syncthreads();
      ok = tc_slice(s, sc, false, nv, N, a.Lx, a.Ly, phase);
      if (!ok) break;
    }
    for (int e = threadIdx.x; e < nv * N; e += blockDim.x) {
      const int vi = e / N, el = e - vi * N;
      const int q = v0 + vi;
      const int sep = a.vec_is_col ? sep_index(el, q, g) : sep_index(q, el, g);
      atomicAdd(&sbin[sep], s.V[e]);
    }
    __syncthreads();
    double* out = a.bins + ((static_cast<size_t>(chain) * (a.L + 1) + l) * 2 + a.bin_slot) * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      atomicAdd(&out[i], sbin[i]);
      sbin[i] = 0.0;
    }
    __syncthreads();
  }
  if (!ok && threadIdx.x == 0) atomicExch(status, kDevTimeout);
  tc_teardown(s);
}

int kron_tc_vectors(int Lx, int Ly) { return kR / max(Lx, Ly); }

static size_t tc_bytes(int nvpc, int N) {
  return static_cast<size_t>(kS) * kASlice + 2ull * kS * kBSlice +
         static_cast<size_t>(nvpc) * N * sizeof(double);
}

cudaError_t launch_kron_tc(const double* in, double* out, int batch, const KronArgs& a, int* status,
                           cudaStream_t st) {
  if (a.Lx > kK || a.Ly > kK) return cudaErrorInvalidValue;
  const int nvpc = kron_tc_vectors(a.Lx, a.Ly);
  const size_t smem = tc_bytes(nvpc, a.N);
  cudaError_t e = cudaFuncSetAttribute(k_kron_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + nvpc - 1) / nvpc, batch);
  k_kron_tc<<<grid, kTC, smem, st>>>(in, out, a, nvpc, status);
  return cudaGetLastError();
}

cudaError_t launch_gtau_tc(const double* X, int batch, const GtauArgs& a, int* status,
                           cudaStream_t st) {
  if (a.Lx > kK || a.Ly > kK) return cudaErrorInvalidValue;
  const int nvpc = kron_tc_vectors(a.Lx, a.Ly);
  const size_t smem = tc_bytes(nvpc, a.N);
  cudaError_t e = cudaFuncSetAttribute(k_gtau_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + nvpc - 1) / nvpc, batch);
  k_gtau_tc<<<grid, kTC, smem, st>>>(X, a, nvpc, status);
  return cudaGetLastError();
}

}  // namespace dqmc
