// FP64 matrix products on the tcgen05 tensor cores (BF16 x BF16 -> FP32),
// exact to FP64 rounding level, for the stabilisation GEMMs of the UDV chain
// (Sec. 2: the O(Lambda N^3) matrix work behind Eq. (3) and G_ij(tau_l)).
//
// On GB300 the FP64 pipe issues 1.2 TFLOP/s, the BF16 tensor cores 2.25
// PFLOP/s.  Each FP64 row of op(A) diag(ks) (and column of op(B)) is written
// as x = 2^e sum_{p<8} a_p 2^{-7p} with signed 7-bit integers a_p, where e is
// fixed per row (column) by its largest element: the 53-bit significand of
// every element is aligned to that exponent with integer shifts and cut into
// eight 7-bit digits.  Digits are exact in BF16, products of two digits need
// 14 bits, and a sum of 256 of them fits the 24-bit FP32 significand, so every
// digit product A_p B_q is exact in the FP32 accumulator.  The products with
// p + q = d (d = 0..7) share one TMEM accumulator; the eight accumulators are
// combined in FP64 in the epilogue:
//   C_ij = alpha rs_i cs_j 2^{e_i + f_j} sum_d 2^{-7d} P_d,ij + beta C_ij.
// Digits beyond p + q = 7 are below 2^-56 relative and dropped.
//
// Tile: one CTA computes 128 x 64 of C for one matrix, K streamed in chunks of
// 64; all 8 digit slices of the chunk sit in shared memory (128 + 64 KB) in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix).
// One thread issues the 36 x 4 MMAs of a chunk (M = 128, N = 64, K = 16) and
// commits them to an mbarrier; the CTA owns all 512 TMEM columns (8 x 64).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace dqmc {
namespace {

constexpr int kS = 8;
constexpr int kTM = 128, kTN = 64, kTK = 64;
constexpr int kATile = kTM * kTK * 2;
constexpr int kBTile = kTN * kTK * 2;
constexpr int kOzSmem = kS * (kATile + kBTile);
constexpr long long kWaitLimit = 1LL << 26;

__device__ __forceinline__ double oz_scale(const double* p, int mode, int i) {
  if (mode == 0 || p == nullptr) return 1.0;
  const double d = p[i];
  switch (mode) {
    case 1: return d;
    case 2: return 1.0 / fmax(d, 1.0);
    case 3: return fmin(d, 1.0);
    default: return 1.0 / d;
  }
}

// One warp per vector v of the batch entry: element k of vector v is
// M[v sv + k sk] (times the inner scale of k).  Writes the 8 digit slices
// out[p][v][k] (row length np, zero tail) and the scale exponent ex[v].
__global__ void __launch_bounds__(256) k_oz_split(const double* Mall, long long sM, int n, int np,
                                                 long long sv, long long sk, const double* ksall,
                                                 long long sks, int ks_mode, __nv_bfloat16* outall,
                                                 long long sOut, int* exall, long long sEx) {
  const int b = blockIdx.y;
  const double* M = Mall + b * sM;
  __shared__ double ksv[kMaxN];
  const double* ks = ksall ? ksall + b * sks : nullptr;
  for (int k = threadIdx.x; k < n; k += blockDim.x) ksv[k] = oz_scale(ks, ks_mode, k);
  __syncthreads();
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (v >= n) return;
  __nv_bfloat16* out = outall + b * sOut;
  int emax = -2000;
  for (int k = lane; k < n; k += 32) {
    const double x = (ks_mode != 0) ? M[v * sv + k * sk] * ksv[k] : M[v * sv + k * sk];
    const int E = static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF);
    if (E != 0) emax = max(emax, E - 1023);
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, o));
  if (lane == 0) exall[b * sEx + v] = emax - 6;
  for (int k = lane; k < np; k += 32) {
    unsigned long long al = 0;
    float sg = 1.0f;
    if (k < n) {
      const double x = (ks_mode != 0) ? M[v * sv + k * sk] * ksv[k] : M[v * sv + k * sk];
      const long long bits = __double_as_longlong(x);
      const int E = static_cast<int>((bits >> 52) & 0x7FF);
      if (E != 0) {  // zero and subnormal inputs contribute zero digits
        const unsigned long long mant =
            (static_cast<unsigned long long>(bits) & ((1ULL << 52) - 1)) | (1ULL << 52);
        const int sh = emax - (E - 1023);
        al = (sh < 64) ? (mant >> sh) : 0ULL;
      }
      sg = (bits < 0) ? -1.0f : 1.0f;
    }
#pragma unroll
    for (int p = 0; p < kS; ++p) {
      const int a = (p < 7) ? static_cast<int>((al >> (46 - 7 * p)) & 127ULL)
                            : static_cast<int>((al & 15ULL) << 3);
      out[(static_cast<size_t>(p) * n + v) * np + k] = __float2bfloat16_rn(sg * static_cast<float>(a));
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: no swizzle, K-major; LBO = distance of the
// next core matrix along K, SBO = along M/N (bytes, encoded >> 4), version 1.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  constexpr uint32_t lbo = 128, sbo = (kTK / 8) * 128;
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}

// Digit slices [kS][n][np] of rows r0 .. r0+R-1 and k0 .. k0+kTK-1 into shared
// memory, core-matrix layout; rows >= n and k >= np are zero.
__device__ __forceinline__ void oz_load(unsigned char* sm, const __nv_bfloat16* src, int n, int np,
                                        int r0, int R, int k0) {
  const int chunks = kS * R * (kTK / 8);
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int kg = c % (kTK / 8);
    const int r = (c / (kTK / 8)) % R;
    const int p = c / ((kTK / 8) * R);
    const int gr = r0 + r, gk = k0 + kg * 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (gr < n && gk < np)
      v = *reinterpret_cast<const uint4*>(src + (static_cast<size_t>(p) * n + gr) * np + gk);
    const int off = p * (R * kTK * 2) + (r >> 3) * ((kTK / 8) * 128) + kg * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(sm + off) = v;
  }
}

struct OzMmaArgs {
  const __nv_bfloat16* As;
  long long sAs;
  const int* exA;
  long long sExA;
  const __nv_bfloat16* Bs;
  long long sBs;
  const int* exB;
  long long sExB;
  double* C;
  long long sC;
  int n, np;
  const double* rs;
  long long srs;
  int rs_mode;
  const double* cs;
  long long scs;
  int cs_mode;
  double alpha, beta;
  int* status;
};

__global__ void __launch_bounds__(128) k_oz_mma(OzMmaArgs a) {
  extern __shared__ __align__(1024) unsigned char oz_sm[];
  unsigned char* smA = oz_sm;
  unsigned char* smB = oz_sm + kS * kATile;
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_sh;
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * kTM, j0 = blockIdx.x * kTN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, np = a.np;
  const __nv_bfloat16* As = a.As + b * a.sAs;
  const __nv_bfloat16* Bs = a.Bs + b * a.sBs;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_sh;
  // kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N, M.
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kTN >> 3) << 17) | ((kTM >> 4) << 24);
  int phase = 0;
  bool ok = true;
  for (int k0 = 0; k0 < np; k0 += kTK) {
    oz_load(smA, As, n, np, i0, kTM, k0);
    oz_load(smB, Bs, n, np, j0, kTN, k0);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int d = 0; d < kS; ++d)
        for (int p = 0; p <= d; ++p) {
          const int q = d - p;
          for (int ks = 0; ks < kTK / 16; ++ks) {
            const uint64_t ad = oz_desc(smem_u32(smA + p * kATile + ks * 256));
            const uint64_t bd = oz_desc(smem_u32(smB + q * kBTile + ks * 256));
            const uint32_t acc = (k0 > 0 || p > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred pa;\n setp.ne.u32 pa, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tbase + d * kTN),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&bar)));
    }
    uint32_t done = 0;
    for (long long it = 0; it < kWaitLimit && !done; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(smem_u32(&bar)), "r"(phase));
    }
    if (!done) {  // bounded wait gave up: record it, leave C untouched, free TMEM
      ok = false;
      if (threadIdx.x == 0) atomicExch(a.status, kDevTimeout);
      break;
    }
    phase ^= 1;
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int i = i0 + warp * 32 + lane;
    const bool row_ok = i < n;
    const double rsi = row_ok ? a.alpha * oz_scale(a.rs ? a.rs + b * a.srs : nullptr, a.rs_mode, i) : 0.0;
    const int ei = row_ok ? a.exA[b * a.sExA + i] : 0;
    double* C = a.C + b * a.sC;
    const double* cs = a.cs ? a.cs + b * a.scs : nullptr;
    for (int c = 0; c < kTN / 16; ++c) {
      double acc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc[q] = 0.0;
      for (int d = 0; d < kS; ++d) {
        uint32_t v[16];
        const uint32_t ta = tbase + (static_cast<uint32_t>(warp * 32) << 16) + d * kTN + c * 16;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const double w = ldexp(1.0, -7 * d);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = fma(static_cast<double>(__uint_as_float(v[q])), w, acc[q]);
      }
      if (row_ok) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = j0 + c * 16 + q;
          if (j < n) {
            const double sc = rsi * oz_scale(cs, a.cs_mode, j);
            double val = sc * ldexp(acc[q], ei + a.exB[b * a.sExB + j]);
            const size_t o = static_cast<size_t>(i) * n + j;
            if (a.beta != 0.0) val += a.beta * C[o];
            C[o] = val;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase));
}

}  // namespace

size_t ozaki_scratch_bytes(int n, int max_batch) {
  const size_t np = (n + 7) / 8 * 8;
  return static_cast<size_t>(max_batch) * (2ull * kS * n * np * 2 + 2ull * n * sizeof(int)) + 256;
}

cudaError_t launch_gemm_ozaki(const GemmArgs& g, int batch, void* scratch, int max_batch,
                              int* status, cudaStream_t st) {
  const int n = g.n;
  const int np = (n + 7) / 8 * 8;
  const long long sl = static_cast<long long>(kS) * n * np;  // bf16 elements per operand
  __nv_bfloat16* As = static_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* Bs = As + sl * max_batch;
  int* exA = reinterpret_cast<int*>(Bs + sl * max_batch);
  int* exB = exA + static_cast<long long>(n) * max_batch;
  cudaError_t e = cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, kOzSmem);
  if (e != cudaSuccess) return e;
  for (int b0 = 0; b0 < batch; b0 += max_batch) {
    const int nb = std::min(max_batch, batch - b0);
    // rows of op(A) diag(ks): tA = 0 -> A[i][k]; tA = 1 -> A[k][i]
    k_oz_split<<<dim3((n + 7) / 8, nb), 256, 0, st>>>(
        g.A + b0 * g.sA, g.sA, n, np, g.tA ? 1 : n, g.tA ? n : 1, g.ks ? g.ks + b0 * g.sks : nullptr,
        g.sks, g.ks ? g.ks_mode : 0, As, sl, exA, n);
    // columns of op(B): tB = 0 -> B[k][j]; tB = 1 -> B[j][k]
    k_oz_split<<<dim3((n + 7) / 8, nb), 256, 0, st>>>(g.B + b0 * g.sB, g.sB, n, np, g.tB ? n : 1,
                                                       g.tB ? 1 : n, nullptr, 0, 0, Bs, sl, exB, n);
    OzMmaArgs m;
    m.As = As; m.sAs = sl; m.exA = exA; m.sExA = n;
    m.Bs = Bs; m.sBs = sl; m.exB = exB; m.sExB = n;
    m.C = g.C + b0 * g.sC; m.sC = g.sC;
    m.n = n; m.np = np;
    m.rs = g.rs ? g.rs + b0 * g.srs : nullptr; m.srs = g.srs; m.rs_mode = g.rs ? g.rs_mode : 0;
    m.cs = g.cs ? g.cs + b0 * g.scs : nullptr; m.scs = g.scs; m.cs_mode = g.cs ? g.cs_mode : 0;
    m.alpha = g.alpha; m.beta = g.beta;
    m.status = status;
    k_oz_mma<<<dim3((n + kTN - 1) / kTN, (n + kTM - 1) / kTM, nb), 128, kOzSmem, st>>>(m);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dqmc
