// FP64 matrix products on the tcgen05 tensor cores (BF16 x BF16 -> FP32)
// for the stabilisation GEMMs of the UDV chain (Sec. 2: the O(Lambda N^3)
// matrix work behind Eq. (3) and G_ij(tau_l)).
//
// On GB300 the FP64 pipe issues 1.2 TFLOP/s, the BF16 tensor cores 2.25
// PFLOP/s.  Each FP64 row of op(A) (and column of op(B)), with the optional
// inner scale folded into one of the two, is written as
// x = 2^e sum_{p<8} a_p 2^{-7p} with signed 7-bit integers a_p, where e is
// fixed per row (column) by its largest element: the 53-bit significand of
// every element is aligned to that exponent with integer shifts and cut into
// eight 7-bit digits.  Digits are exact in BF16 and products of two digits
// need 14 bits.  The products with p + q = d (d = 0..7) share one TMEM
// accumulator P_d; a sum of up to 2^24 / 127^2 = 1040 digit products is exact
// in FP32, which covers every accumulator with d <= 3 for K <= 256; the
// higher ones (weights 2^-28 and below) stay exact unless their digits are
// systematically near 127.  The epilogue combines the accumulators exactly in
// 64-bit integers:
//   C_ij = alpha rs_i cs_j 2^{e_i + f_j} sum_d 2^{-7d} P_d,ij + beta C_ij.
// Digits beyond p + q = 7 are below 2^-56 of the row-times-column scale and
// dropped.  Accuracy is therefore relative to max_k |a_ik| max_k |b_kj|, not
// to sum_k |a_ik b_kj| as in an FP64 GEMM: a product in which op(A)'s row is
// small where op(B)'s column is large (opposite grading along k) loses the
// small entries; callers place the inner scale so that this does not occur.
//
// Tile: one CTA computes 128 x 64 of C for one matrix, K streamed in chunks of
// 32.  The split kernel writes the digit slices tile-blocked, each (slice, row
// tile, K chunk) block contiguous in the no-swizzle K-major core-matrix order
// (8 rows x 16 bytes per core matrix), so one thread moves a chunk -- all 8
// slices of A and B, 96 KB -- with 16 bulk async copies (cp.async.bulk)
// completing on an mbarrier.  Two stages: the copy of chunk c + 1 runs while
// the tensor pipe works on the 36 x 2 MMAs (M = 128, N = 64, K = 16) of chunk
// c; MMA completion is committed to a second mbarrier per stage.  The CTA owns
// all 512 TMEM columns (8 accumulators x 64).
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "oz_compose.cuh"

namespace dqmc {
namespace {

constexpr int kS = 8;
constexpr int kTM = 128, kTN = 64, kTK = 32;
constexpr int kATile = kTM * kTK * 2;  // bytes of one digit slice of an A chunk (8 KB)
constexpr int kStages = 2;
constexpr long long kWaitLimit = 1LL << 26;
// Tile width BN (columns of C per CTA) is 64, or 32 for products with at most
// 32 columns (the panel products of the blocked QR).
template <int BN>
struct OzTile {
  static constexpr int kBTile = BN * kTK * 2;               // one B digit slice of a chunk
  static constexpr int kStage = kS * (kATile + kBTile);     // all digits of one K chunk
  static constexpr int kTmemCols = kS * BN;                  // 8 accumulators of BN columns
};

// Element offset of (slice p, vector v, k) in the tile-blocked digit layout:
// blocks [p][row tile][K chunk] of R x kTK elements, each block in the
// no-swizzle K-major core-matrix order (8 rows x 8 elements per core matrix,
// core matrices along K first), so that one K chunk of one slice of one row
// tile is a single contiguous run for a bulk copy.
__host__ __device__ __forceinline__ size_t oz_offset(int p, int v, int k, int R, int nrt, int nkc) {
  const int rt = v / R, r = v - rt * R, kc = k / kTK, kk = k - kc * kTK;
  const size_t block = (static_cast<size_t>(p) * nrt + rt) * nkc + kc;
  return block * (static_cast<size_t>(R) * kTK) + (r >> 3) * (kTK / 8 * 64) + (kk >> 3) * 64 +
         (r & 7) * 8 + (kk & 7);
}

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

// Inner-index balance: kexp[k] = unbiased exponent of max_j |op(B)_kj s_k|
// (s the inner scale when it goes with op(B)), 0 for a zero row.  Integer
// work only.  One warp per k.
__global__ void __launch_bounds__(256) k_oz_kexp(const double* Mall, long long sM, int nvec, int K,
                                                long long sv, long long sk, const double* ksall,
                                                long long sks, int ks_mode, int* kexpall) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= K) return;
  const double* M = Mall + b * sM;
  int emax = -1;
  for (int j = lane; j < nvec; j += 32)
    emax = max(emax, static_cast<int>((__double_as_longlong(M[j * sv + k * sk]) >> 52) & 0x7FF));
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, o));
  if (lane == 0) {
    int e = 0;
    if (emax > 0) {
      e = emax - 1023;
      if (ks_mode != 0 && ksall) {
        const double sc = oz_scale(ksall + b * sks, ks_mode, k);
        const int Es = static_cast<int>((__double_as_longlong(sc) >> 52) & 0x7FF);
        if (Es > 0) e += Es - 1023;
      }
    }
    kexpall[b * static_cast<long long>(K) + k] = e;
  }
}

// One operand of a product for the split kernel: vector v (a row of op(A) or
// a column of op(B)) has element k at M[v sv + k sk] of batch entry b
// (M + b sM), times the inner scale of k if it goes with this operand.
struct OzSplitOp {
  const double* M;
  long long sM;
  int nvec, R;  // vectors, and the row tile they are padded to
  long long sv, sk;
  const double* ks;
  long long sks;
  int ks_mode;
  int ksign;  // +1 for op(A), -1 for op(B): sign of the balance exponent
  __nv_bfloat16* out;
  long long sOut;
  int* ex;
  long long sEx;
  int blocks;  // blocks of the grid's x dimension that work on this operand
};

// Both operands of a product in one launch: blocks [0, opA.blocks) split the
// rows of op(A), the others the columns of op(B).  A block takes kSV vectors:
// it stages them (times the inner scale) in shared memory with coalesced
// loads whichever way the vectors lie in memory, finds each vector's largest
// exponent (plus 2^{ksign kexp[k]} when balancing; the power of two only
// moves the digit alignment, as an integer exponent offset), and cuts every
// element into 8 digit slices written in the tile-blocked layout (rows padded
// to a multiple of R, K to a multiple of the chunk, zero padding), with the
// scale exponent ex[v].
constexpr int kSV = 32;  // vectors per split block
__host__ __device__ constexpr int oz_split_ld(int n) { return ((n + 7) & ~7) + 1; }
__host__ __device__ constexpr size_t oz_split_smem(int n) {
  return static_cast<size_t>(kSV) * oz_split_ld(n) * sizeof(double);
}
// Position of element k within a staged vector: each group of 8 is rotated by
// (k / 16) mod 8, so that the 16 lanes of a half warp reading element e of
// their groups 8L + e hit 16 different bank pairs.
__device__ __forceinline__ int oz_swz(int k) { return (k & ~7) | ((k + (k >> 4)) & 7); }

__global__ void __launch_bounds__(256) k_oz_split(OzSplitOp opA, OzSplitOp opB, int n,
                                                 const int* kexpall) {
  const bool isA = static_cast<int>(blockIdx.x) < opA.blocks;
  const OzSplitOp o = isA ? opA : opB;
  const int bx = isA ? static_cast<int>(blockIdx.x) : static_cast<int>(blockIdx.x) - opA.blocks;
  // nvec vectors of length n (the inner dimension K)
  const int nvec = o.nvec, R = o.R;
  const long long sv = o.sv, sk = o.sk;
  const int ks_mode = o.ks_mode;
  const int nrt = (nvec + R - 1) / R, nkc = (n + kTK - 1) / kTK;
  const int b = blockIdx.y;
  const double* M = o.M + b * o.sM;
  extern __shared__ __align__(16) double xs[];  // [kSV][oz_split_ld(n)], swizzled along k
  __shared__ double ksv[kMaxN];
  __shared__ int kev[kMaxN];
  const double* ks = o.ks ? o.ks + b * o.sks : nullptr;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    ksv[k] = oz_scale(ks, ks_mode, k);
    kev[k] = kexpall ? o.ksign * kexpall[b * static_cast<long long>(n) + k] : 0;
  }
  __syncthreads();
  const int v0 = bx * kSV, ld = oz_split_ld(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (v0 >= nrt * R) return;
  // 1. stage the block's vectors; lanes run along the contiguous index, and
  // every thread has 8 loads in flight before it stores
  constexpr int kU = 8;
  if (sv == 1) {
    const int v = v0 + lane;
    for (int k0 = warp; k0 < n; k0 += nw * kU) {
      double x[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int k = k0 + u * nw;
        x[u] = (v < nvec && k < n) ? M[v + k * sk] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int k = k0 + u * nw;
        if (k < n) xs[lane * ld + oz_swz(k)] = (ks_mode != 0) ? x[u] * ksv[k] : x[u];
      }
    }
  } else {
    for (int r = warp; r < kSV; r += nw) {
      const int v = v0 + r;
      for (int k0 = lane; k0 < n; k0 += 32 * kU) {
        double x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int k = k0 + 32 * u;
          x[u] = (v < nvec && k < n) ? M[v * sv + k * sk] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int k = k0 + 32 * u;
          if (k < n) xs[r * ld + oz_swz(k)] = (ks_mode != 0) ? x[u] * ksv[k] : x[u];
        }
      }
    }
  }
  __syncthreads();
  __nv_bfloat16* out = o.out + b * o.sOut;
  // 2. exponent of every vector, one warp per vector
  __shared__ int exs[kSV];
  for (int r = warp; r < kSV; r += nw) {
    const double* xr = xs + r * ld;
    int emax = -100000;
    for (int k = lane; k < n; k += 32) {
      const int E = static_cast<int>((__double_as_longlong(xr[oz_swz(k)]) >> 52) & 0x7FF);
      if (E != 0) emax = max(emax, E - 1023 + kev[k]);
    }
    for (int q = 16; q > 0; q >>= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, q));
    if (lane == 0) {
      exs[r] = emax;
      if (v0 + r < nvec) o.ex[b * o.sEx + v0 + r] = emax - 6;
    }
  }
  __syncthreads();
  // 3. digits: a warp task is 8 vectors x one K chunk of 32, lane = (vector
  // r & 7, 8-element group of the chunk), so that the 32 16-byte stores of a
  // slice fill one contiguous 512-byte run of the core-matrix layout
  const int ntask = (kSV / 8) * nkc;
  for (int task = warp; task < ntask; task += nw) {
    const int rg = task / nkc, kc = task - rg * nkc;
    const int r = rg * 8 + (lane & 7), v = v0 + r, k0 = kc * kTK + (lane >> 3) * 8;
    const double* xr = xs + r * ld;
    const int emax = exs[r];
    unsigned long long al[8];
    float sg[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      al[e] = 0;
      sg[e] = 1.0f;
      if (k < n && v < nvec) {  // padding rows and columns give zero digits
        const long long bits = __double_as_longlong(xr[oz_swz(k)]);
        const int E = static_cast<int>((bits >> 52) & 0x7FF);
        if (E != 0) {  // zero and subnormal inputs contribute zero digits
          const unsigned long long mant =
              (static_cast<unsigned long long>(bits) & ((1ULL << 52) - 1)) | (1ULL << 52);
          const int sh = emax - (E - 1023 + kev[k]);
          al[e] = (sh < 64) ? (mant >> sh) : 0ULL;
        }
        sg[e] = (bits < 0) ? -1.0f : 1.0f;
      }
    }
#pragma unroll
    for (int p = 0; p < kS; ++p) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float f[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const unsigned long long a = al[e + q];
          const int d = (p < 7) ? static_cast<int>((a >> (46 - 7 * p)) & 127ULL)
                                : static_cast<int>((a & 15ULL) << 3);
          f[q] = sg[e + q] * static_cast<float>(d);
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[0], f[1]);  // .x = f[0], low half
        w[e >> 1] = *reinterpret_cast<const uint32_t*>(&h);
      }
      *reinterpret_cast<uint4*>(out + oz_offset(p, v, k0, R, nrt, nkc)) =
          make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: no swizzle, K-major; LBO = distance of the
// next core matrix along K, SBO = along M/N (bytes, encoded >> 4), version 1.
__device__ __forceinline__ uint64_t oz_desc(uint32_t addr) {
  constexpr uint32_t lbo = 128, sbo = (kTK / 8) * 128;  // 128 B, 512 B
  return static_cast<uint64_t>((addr >> 4) & 0x3FFF) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (1ULL << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait on an mbarrier phase; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, int parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kWaitLimit && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
  return done != 0;
}

// One thread: bulk-copy all digit slices of K chunk kc (A rows of tile ra, B
// rows of tile rb) into stage smem; completion is counted on `bar`.
template <int BN>
__device__ __forceinline__ void oz_issue_chunk(unsigned char* stage, const __nv_bfloat16* As,
                                               const __nv_bfloat16* Bs, int ra, int rb, int kc,
                                               int nrtA, int nrtB, int nkc, uint64_t* bar) {
  using Tl = OzTile<BN>;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(static_cast<uint32_t>(Tl::kStage)));
  for (int p = 0; p < kS; ++p) {
    const __nv_bfloat16* ga = As + ((static_cast<size_t>(p) * nrtA + ra) * nkc + kc) * (kTM * kTK);
    const __nv_bfloat16* gb = Bs + ((static_cast<size_t>(p) * nrtB + rb) * nkc + kc) * (BN * kTK);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(stage + p * kATile)),
        "l"(ga), "r"(static_cast<uint32_t>(kATile)), "r"(smem_u32(bar))
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(stage + kS * kATile + p * Tl::kBTile)),
        "l"(gb), "r"(static_cast<uint32_t>(Tl::kBTile)), "r"(smem_u32(bar))
        : "memory");
  }
}

// C (M x Nc, leading dimension ldc) = alpha diag(rs) [digit product] diag(cs)
// + beta C for each batch entry; K is the inner dimension.
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
  int M, Nc, K, ldc;
  const double* rs;
  long long srs;
  int rs_mode;
  const double* cs;
  long long scs;
  int cs_mode;
  double alpha, beta;
  int* status;
};

// 256 threads.  Thread 0 issues the MMAs of each K chunk once its copies
// have landed; thread 32 (warp 1) is the producer: it loads chunk c into stage
// c & 1 as soon as the MMAs of chunk c - 2 that read that stage are done, so
// the copy of chunk c + 1 runs while the tensor pipe works on chunk c (the
// issuing thread blocks while the MMA queue is full and cannot do both).  All
// eight warps then drain TMEM: warp w reads the lanes (rows) 32 (w & 3) ..
// and half w >> 2 of the columns.
template <int BN>
__global__ void __launch_bounds__(256) k_oz_mma(OzMmaArgs a) {
  using Tl = OzTile<BN>;
  extern __shared__ __align__(1024) unsigned char oz_sm[];
  __shared__ uint64_t full[kStages], mmad[kStages];
  __shared__ uint32_t tmem_sh;
  __shared__ int fail_sh;
  __shared__ int loaded[kStages], consumed[kStages];  // last chunk loaded into / read from a stage
  __shared__ int committed_sh;
  __shared__ double colf[BN];  // cs_j 2^{f_j - 21} of this CTA's columns
  __shared__ int colx[BN];     // f_j of this CTA's columns
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * kTM, j0 = blockIdx.x * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = a.M, Nc = a.Nc;
  const int nrtA = (M + kTM - 1) / kTM, nrtB = (Nc + BN - 1) / BN, nkc = (a.K + kTK - 1) / kTK;
  const __nv_bfloat16* As = a.As + b * a.sAs;
  const __nv_bfloat16* Bs = a.Bs + b * a.sBs;
  if (threadIdx.x >= 256 - BN) {
    const int q = threadIdx.x - (256 - BN), j = j0 + q;
    colf[q] = (j < Nc) ? oz_scale(a.cs ? a.cs + b * a.scs : nullptr, a.cs_mode, j) *
                             ldexp(1.0, a.exB[b * a.sExB + j] - 21)
                       : 0.0;
    colx[q] = (j < Nc) ? a.exB[b * a.sExB + j] : 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_sh)),
                 "n"(Tl::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < kStages; ++s2) {
      mbar_init(&full[s2], 1);
      mbar_init(&mmad[s2], 1);
      loaded[s2] = consumed[s2] = -1;
    }
    fail_sh = 0;
    committed_sh = -1;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_sh;
  // kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N, M.
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((BN >> 3) << 17) | ((kTM >> 4) << 24);
  volatile int* fail_v = &fail_sh;
  if (threadIdx.x == 32) {  // producer
    for (int c = 0; c < nkc && !*fail_v; ++c) {
      const int st = c & 1;
      // stage st was last read by the MMAs of chunk c - 2
      if (c >= kStages && !mbar_wait(&mmad[st], ((c - kStages) >> 1) & 1)) {
        *fail_v = 1;
        break;
      }
      oz_issue_chunk<BN>(oz_sm + st * Tl::kStage, As, Bs, blockIdx.y, blockIdx.x, c, nrtA, nrtB,
                         nkc, &full[st]);
      loaded[st] = c;
    }
  } else if (threadIdx.x == 0) {  // MMA issuer
    for (int c = 0; c < nkc; ++c) {
      const int st = c & 1;
      if (!mbar_wait(&full[st], (c >> 1) & 1)) {
        *fail_v = 1;
        break;
      }
      consumed[st] = c;
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned char* smA = oz_sm + st * Tl::kStage;
      unsigned char* smB = smA + kS * kATile;
      for (int d = 0; d < kS; ++d)
        for (int p = 0; p <= d; ++p) {
          const int q = d - p;
          for (int ks = 0; ks < kTK / 16; ++ks) {
            const uint64_t ad = oz_desc(smem_u32(smA + p * kATile + ks * 256));
            const uint64_t bd = oz_desc(smem_u32(smB + q * Tl::kBTile + ks * 256));
            const uint32_t acc = (c > 0 || p > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred pa;\n setp.ne.u32 pa, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tbase + d * BN),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mmad[st])));
      committed_sh = c;
      if (*fail_v) break;
    }
  }
  __syncthreads();
  if (fail_sh && threadIdx.x == 0) {
    // drain what is still in flight before TMEM and smem go away: loads that
    // no MMA waited for, and the last committed MMAs (which cover all earlier)
    for (int s2 = 0; s2 < kStages; ++s2)
      if (loaded[s2] > consumed[s2]) mbar_wait(&full[s2], (loaded[s2] >> 1) & 1);
    const int cm = committed_sh;
    if (cm >= 0) mbar_wait(&mmad[cm & 1], (cm >> 1) & 1);
  }
  // Everyone waits for the MMAs of the last chunk (tcgen05.commit tracks all
  // earlier MMAs of the issuing thread, so this covers every chunk).
  bool ok = fail_sh == 0;
  if (ok) {
    const int last = nkc - 1;
    ok = mbar_wait(&mmad[last & 1], (last >> 1) & 1);
  }
  ok = __syncthreads_and(ok) != 0;  // one decision for the block (the epilogue has a barrier)
  if (!ok && threadIdx.x == 0) atomicExch(a.status, kDevTimeout);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // Recombination.  Every accumulator holds an integer P_d (a sum of digit
    // products); sum_d P_d 2^{-7d} = 2^{-21} (hi + 2^{-28} lo) with the exact
    // 64-bit integers hi = sum_{d<4} P_d 2^{7(3-d)} and lo = sum_{d>=4} P_d
    // 2^{7(7-d)} (both below 2^47), rounded once to FP64 by oz_compose with
    // integer instructions.  Without row and column scales (alpha = +-1) the
    // power of two 2^{e_i + f_j - 21} and the sign go into the exponent and
    // sign fields there; otherwise the scales are two FP64 products.
    const int quarter = warp & 3, half = warp >> 2;
    const int i = i0 + quarter * 32 + lane;
    const bool row_ok = i < M;
    const double rowf =
        row_ok ? a.alpha * oz_scale(a.rs ? a.rs + b * a.srs : nullptr, a.rs_mode, i) *
                     ldexp(1.0, a.exA[b * a.sExA + i])
               : 0.0;
    const bool pow2 = (a.rs == nullptr || a.rs_mode == 0) && (a.cs == nullptr || a.cs_mode == 0) &&
                      (a.alpha == 1.0 || a.alpha == -1.0);
    const int rowx = row_ok ? a.exA[b * a.sExA + i] : 0;
    double* C = a.C + b * a.sC;
    for (int c = half * (BN / 32); c < (half + 1) * (BN / 32); ++c) {
      uint32_t v[kS][16];
#pragma unroll
      for (int d = 0; d < kS; ++d) {
        const uint32_t ta = tbase + (static_cast<uint32_t>(quarter * 32) << 16) + d * BN + c * 16;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]), "=r"(v[d][5]),
              "=r"(v[d][6]), "=r"(v[d][7]), "=r"(v[d][8]), "=r"(v[d][9]), "=r"(v[d][10]), "=r"(v[d][11]),
              "=r"(v[d][12]), "=r"(v[d][13]), "=r"(v[d][14]), "=r"(v[d][15])
            : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row_ok) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int jj = c * 16 + q, j = j0 + jj;
          if (j < Nc) {
            long long hi = 0, lo = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d)
              hi += static_cast<long long>(__float2int_rn(__uint_as_float(v[d][q]))) << (7 * (3 - d));
#pragma unroll
            for (int d = 4; d < kS; ++d)
              lo += static_cast<long long>(__float2int_rn(__uint_as_float(v[d][q]))) << (7 * (7 - d));
            double val;
            bool ok2 = false;
            if (pow2) val = oz_compose(hi, lo, rowx + colx[jj] - 21, a.alpha < 0.0, ok2);
            if (!ok2) val = (oz_compose(hi, lo, 0, false, ok2) * rowf) * colf[jj];
            const size_t o = static_cast<size_t>(i) * a.ldc + j;
            if (a.beta != 0.0) val = fma(a.beta, C[o], val);
            C[o] = val;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "n"(Tl::kTmemCols));
}

// ---------------------------------------------------------------------------
// Fused product: the digit slices are cut by the CTA itself, straight into
// the shared-memory stage the tensor cores read, so no slice makes a round
// trip through global memory and no split kernel runs.  544 threads: the
// kFT = 512 threads of warps 0-15 split (the 128 rows of op(A) and BN columns
// of op(B) of the tile, one K chunk of 32 at a time, two stages) and arrive
// on the stage's `full` barrier, each after a proxy fence that makes its
// shared-memory writes visible to the tensor cores; one thread of warp 16
// issues the MMAs of the chunk, so splitting chunk c + 1 overlaps the MMAs of
// chunk c.  Before the K loop the split threads find the exponent of every
// row of op(A) and column of op(B) of the tile over the whole K range (the
// digit alignment).  Memory access follows the operand's layout: a vector
// contiguous along k is read by lanes along k, otherwise lanes run along the
// vectors.
// ---------------------------------------------------------------------------
struct OzFusedArgs {
  const double* A; long long sA, a_sv, a_sk;
  const double* B; long long sB, b_sv, b_sk;
  int M, Nc, K;
  const double* ks; long long sks; int ks_mode, ks_on_b;
  const int* kexp;  // balance exponents [batch][K] or null
  double* C; long long sC; int ldc;
  const double* rs; long long srs; int rs_mode;
  const double* cs; long long scs; int cs_mode;
  double alpha, beta;
  int* status;
};

constexpr int kFT = 512;  // split (and epilogue) threads of the fused kernel

// ex_s[r] = (exponent, unbiased, plus the balance offset ksign kev[k], of the
// largest element of vector v0 + r of an operand over k < K) - 6, for the R
// vectors of a tile; -100006 for a zero or missing vector.  The kFT split
// threads take part; every thread has several loads in flight before it
// reduces (the pass is latency-bound otherwise).  A vector contiguous along k
// is read by a warp along k, four vectors at a time; otherwise lanes run
// along the vectors and the threads split the k range, combined with shared
// atomics.  Ends with a barrier of the split threads.
// Barrier of the kFT split threads only (named barrier 1).
__device__ __forceinline__ void oz_split_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kFT) : "memory"); }

__device__ __forceinline__ int oz_elem_exp(double x, int kv) {
  const int E = static_cast<int>((__double_as_longlong(x) >> 52) & 0x7FF);
  return (E != 0) ? E - 1023 + kv : -100000;
}

__device__ void oz_tile_emax(const double* Mp, long long sv, long long sk, int v0, int nvec, int R,
                             int K, const double* kss, const int* kev, int ksign, bool scaled,
                             int* ex_s) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  constexpr int nw = kFT / 32;
  if (sk == 1) {
    for (int r0 = warp * 4; r0 < R; r0 += 4 * nw) {
      int em[4] = {-100000, -100000, -100000, -100000};
      for (int k = lane; k < K; k += 32) {
        double x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int v = v0 + r0 + u;
          x[u] = (r0 + u < R && v < nvec) ? Mp[v * sv + k] : 0.0;
        }
        const double kf = scaled ? kss[k] : 1.0;
        const int kv = ksign * kev[k];
#pragma unroll
        for (int u = 0; u < 4; ++u) em[u] = max(em[u], oz_elem_exp(scaled ? x[u] * kf : x[u], kv));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        for (int q = 16; q > 0; q >>= 1) em[u] = max(em[u], __shfl_xor_sync(0xFFFFFFFFu, em[u], q));
        if (lane == 0 && r0 + u < R) ex_s[r0 + u] = em[u] - 6;
      }
    }
    oz_split_sync();
  } else {
    for (int r = t; r < R; r += kFT) ex_s[r] = -100000;
    oz_split_sync();
    const int tpv = kFT / R;  // threads per vector (R divides kFT)
    const int r = t % R, ks0 = t / R, v = v0 + r;
    int em = -100000;
    if (v < nvec) {
      constexpr int kU = 8;
      for (int k0 = ks0; k0 < K; k0 += tpv * kU) {
        double x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int k = k0 + u * tpv;
          x[u] = (k < K) ? Mp[v * sv + k * sk] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int k = k0 + u * tpv;
          if (k < K) em = max(em, oz_elem_exp(scaled ? x[u] * kss[k] : x[u], ksign * kev[k]));
        }
      }
    }
    atomicMax(&ex_s[r], em);
    oz_split_sync();
    for (int q = t; q < R; q += kFT) ex_s[q] -= 6;
    oz_split_sync();
  }
}

// The 8 digit slices of elements k0 .. k0 + 7 of vector v (already scaled;
// kv = balance exponent offsets; aligned to the vector's exponent emax), one
// 16-byte unit per slice in the core-matrix layout of a stage operand with R
// rows.  The aligned 53-bit magnitude is cut with 32-bit bit-field extracts
// (digit p = bits 46 - 7p .. 52 - 7p; the last digit is bits 0 .. 3 moved up
// by 3); a digit d becomes the float +-d through the exponent of 2^23
// (bits 0x4B000000 | d are 2^23 + d) and one FMA with the sign, and two floats
// are packed to a BF16 pair (exact: d < 128).
__device__ __forceinline__ uint32_t oz_bfe(uint32_t x, int pos) {
  uint32_t d;
  asm("bfe.u32 %0, %1, %2, 7;" : "=r"(d) : "r"(x), "r"(pos));
  return d;
}

__device__ __forceinline__ void oz_split_unit(const double (&x)[8], const int (&kv)[8], int emax,
                                              unsigned char* op, int R, int v, int kg) {
  uint32_t h[8], l[8];
  float sg[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const long long bits = __double_as_longlong(x[e]);
    const int E = static_cast<int>((bits >> 52) & 0x7FF);
    unsigned long long al = 0ULL;
    if (E != 0) {  // zero and subnormal inputs contribute zero digits
      const unsigned long long mant =
          (static_cast<unsigned long long>(bits) & ((1ULL << 52) - 1)) | (1ULL << 52);
      const int sh = emax - (E - 1023 + kv[e]);
      al = (sh < 64) ? (mant >> sh) : 0ULL;
    }
    h[e] = static_cast<uint32_t>(al >> 32);
    l[e] = static_cast<uint32_t>(al);
    sg[e] = (bits < 0) ? -1.0f : 1.0f;
  }
  // element offset of (v, 8 kg) within one slice: core matrices of 8 rows x 8 k
  const int off = (v >> 3) * (kTK / 8 * 64) + kg * 64 + (v & 7) * 8;
  constexpr float kTwo23 = 8388608.0f;
#pragma unroll
  for (int p = 0; p < kS; ++p) {
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float f[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        uint32_t d;
        if (p < 3)
          d = oz_bfe(h[e + q], 14 - 7 * p);
        else if (p == 3)
          d = l[e + q] >> 25;
        else if (p < 7)
          d = oz_bfe(l[e + q], 46 - 7 * p);
        else
          d = (l[e + q] & 15u) << 3;
        f[q] = fmaf(__uint_as_float(0x4B000000u | d), sg[e + q], -kTwo23 * sg[e + q]);
      }
      const __nv_bfloat162 hb = __floats2bfloat162_rn(f[0], f[1]);
      w[e >> 1] = *reinterpret_cast<const uint32_t*>(&hb);
    }
    *reinterpret_cast<uint4*>(op + (static_cast<size_t>(p) * R * kTK + off) * 2) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// One operand of the fused product as the split of a K chunk sees it.
struct OzOperand {
  const double* M;
  long long sv, sk;
  int v0, nvec, R, ksign;
  bool scaled;
  const int* ex;
  unsigned char* op;  // the operand's slices in the stage
};

// Unit u of a K chunk of one operand: vector v and k group kg.  A vector
// contiguous along k gives 8 consecutive vectors x 4 k groups per 32 units
// (conflict-free 16-byte stores), otherwise lanes run along the vectors.
__device__ __forceinline__ void oz_unit_coords(const OzOperand& o, int u, int& v, int& kg) {
  if (o.sk == 1) {
    v = (u & 7) + 8 * (u >> 5);
    kg = (u >> 3) & 3;
  } else {
    kg = u / o.R;
    v = u - kg * o.R;
  }
}

// Split K chunk kc of both operands into the stage: every split thread takes
// up to kUnitsPerThread units (the (128 + BN) x 4 units of a chunk need at
// most two per thread), loads all their elements first (independent loads in
// flight), then cuts them.
constexpr int kUnitsPerThread = 2;
static_assert((kTM + 64) * (kTK / 8) <= kUnitsPerThread * kFT, "units of a chunk per thread");
__device__ __forceinline__ void oz_split_chunk2(const OzOperand& oa, const OzOperand& ob, int K,
                                                int kc, const double* kss, const int* kev) {
  const int ua = oa.R * (kTK / 8), ub = ob.R * (kTK / 8), total = ua + ub;
  double x[kUnitsPerThread][8];
  int vv[kUnitsPerThread], kgs[kUnitsPerThread];
  bool isA[kUnitsPerThread], live[kUnitsPerThread];
#pragma unroll
  for (int t = 0; t < kUnitsPerThread; ++t) {
    const int u = t * kFT + static_cast<int>(threadIdx.x);
    live[t] = u < total;
    isA[t] = u < ua;
    const OzOperand& o = isA[t] ? oa : ob;
    int v = 0, kg = 0;
    if (live[t]) oz_unit_coords(o, isA[t] ? u : u - ua, v, kg);
    vv[t] = v;
    kgs[t] = kg;
    const int vg = o.v0 + v, k0 = kc * kTK + kg * 8;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      x[t][e] = (live[t] && vg < o.nvec && k < K) ? o.M[vg * o.sv + k * o.sk] : 0.0;
    }
  }
#pragma unroll
  for (int t = 0; t < kUnitsPerThread; ++t) {
    if (!live[t]) continue;
    const OzOperand& o = isA[t] ? oa : ob;
    const int k0 = kc * kTK + kgs[t] * 8;
    int kv[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = k0 + e;
      kv[e] = (k < K) ? o.ksign * kev[k] : 0;
      if (o.scaled && k < K) x[t][e] *= kss[k];
    }
    oz_split_unit(x[t], kv, o.ex[vv[t]] + 6, o.op, o.R, vv[t], kgs[t]);  // ex holds emax - 6
  }
}

template <int BN>
__global__ void __launch_bounds__(kFT + 32, 1) k_oz_fused(OzFusedArgs a) {
  using Tl = OzTile<BN>;
  extern __shared__ __align__(1024) unsigned char oz_sm[];
  __shared__ uint64_t full[kStages], mmad[kStages];
  __shared__ uint32_t tmem_sh;
  __shared__ int fail_sh;
  __shared__ int exA_s[kTM], exB_s[BN];
  __shared__ double ks_s[kMaxN];
  __shared__ int kev_s[kMaxN];
  __shared__ double colf[BN];
  __shared__ int colx[BN];
  const int b = blockIdx.z;
  const int i0 = blockIdx.y * kTM, j0 = blockIdx.x * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int M = a.M, Nc = a.Nc, K = a.K;
  const int nkc = (K + kTK - 1) / kTK;
  const double* A = a.A + b * a.sA;
  const double* B = a.B + b * a.sB;
  const bool scA = a.ks_mode != 0 && a.ks != nullptr && !a.ks_on_b;
  const bool scB = a.ks_mode != 0 && a.ks != nullptr && a.ks_on_b;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_sh)),
                 "n"(Tl::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s2 = 0; s2 < kStages; ++s2) {
      mbar_init(&full[s2], kFT);
      mbar_init(&mmad[s2], 1);
    }
    fail_sh = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const double* ksb = a.ks ? a.ks + b * a.sks : nullptr;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    ks_s[k] = oz_scale(ksb, a.ks_mode, k);
    kev_s[k] = a.kexp ? a.kexp[b * static_cast<long long>(K) + k] : 0;
  }
  __syncthreads();
  // exponents of the tile's rows of op(A) and columns of op(B) (split
  // threads; the MMA warp waits at the barrier below)
  if (threadIdx.x < kFT) {
    oz_tile_emax(A, a.a_sv, a.a_sk, i0, M, kTM, K, ks_s, kev_s, 1, scA, exA_s);
    oz_tile_emax(B, a.b_sv, a.b_sk, j0, Nc, BN, K, ks_s, kev_s, -1, scB, exB_s);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_sh;
  if (threadIdx.x < BN) {
    const int q = threadIdx.x, j = j0 + q;
    colf[q] = (j < Nc) ? oz_scale(a.cs ? a.cs + b * a.scs : nullptr, a.cs_mode, j) *
                             ldexp(1.0, exB_s[q] - 21)
                       : 0.0;
    colx[q] = exB_s[q];
  }
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((BN >> 3) << 17) | ((kTM >> 4) << 24);
  volatile int* fail_v = &fail_sh;
  if (threadIdx.x < kFT) {
    // split threads: chunk c goes to stage c & 1 once the MMAs of chunk c - 2,
    // which read that stage, are done
    for (int c = 0; c < nkc; ++c) {
      const int st = c & 1;
      unsigned char* smA = oz_sm + st * Tl::kStage;
      unsigned char* smB = smA + kS * kATile;
      if (c >= kStages && !mbar_wait(&mmad[st], ((c - kStages) >> 1) & 1)) *fail_v = 1;
      if (*fail_v) break;
      const OzOperand oa{A, a.a_sv, a.a_sk, i0, M, kTM, 1, scA, exA_s, smA};
      const OzOperand ob{B, a.b_sv, a.b_sk, j0, Nc, BN, -1, scB, exB_s, smB};
      oz_split_chunk2(oa, ob, K, c, ks_s, kev_s);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[st])) : "memory");
    }
  } else if (threadIdx.x == kFT) {
    // MMA issuer (warp 16): the split warps go on with the next chunk while
    // this thread blocks on the MMA queue
    int committed = -1;
    for (int c = 0; c < nkc; ++c) {
      const int st = c & 1;
      if (*fail_v || !mbar_wait(&full[st], (c >> 1) & 1)) {
        *fail_v = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned char* smA = oz_sm + st * Tl::kStage;
      unsigned char* smB = smA + kS * kATile;
      for (int d = 0; d < kS; ++d)
        for (int p = 0; p <= d; ++p) {
          const int q = d - p;
          for (int ks = 0; ks < kTK / 16; ++ks) {
            const uint64_t ad = oz_desc(smem_u32(smA + p * kATile + ks * 256));
            const uint64_t bd = oz_desc(smem_u32(smB + q * Tl::kBTile + ks * 256));
            const uint32_t acc = (c > 0 || p > 0 || ks > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred pa;\n setp.ne.u32 pa, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pa;\n}" ::"r"(tbase + d * BN),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mmad[st])));
      committed = c;
    }
    // the MMAs of the last committed chunk (commit tracks all earlier MMAs too)
    if (committed >= 0 && !mbar_wait(&mmad[committed & 1], (committed >> 1) & 1)) *fail_v = 1;
    if (committed != nkc - 1) *fail_v = 1;
  }
  __syncthreads();
  const bool ok = *reinterpret_cast<volatile int*>(&fail_sh) == 0;
  if (!ok && threadIdx.x == 0) atomicExch(a.status, kDevTimeout);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    // Recombination as in k_oz_mma: the kFT / 128 warps w = q, q + 4, ...
    // share the TMEM lanes of quarter q, each taking an equal part of the
    // columns; staged through shared memory for row-wise access to C.
    constexpr int kGroups = kFT / 128;  // warps sharing the TMEM lanes of one quarter
    const int quarter = warp & 3, half = warp >> 2;
    const int rl = quarter * 32 + lane;
    const int i = i0 + rl;
    const bool row_ok = i < M;
    const double rowf =
        row_ok ? a.alpha * oz_scale(a.rs ? a.rs + b * a.srs : nullptr, a.rs_mode, i) *
                     ldexp(1.0, exA_s[rl])
               : 0.0;
    const bool pow2 = (a.rs == nullptr || a.rs_mode == 0) && (a.cs == nullptr || a.cs_mode == 0) &&
                      (a.alpha == 1.0 || a.alpha == -1.0);
    const int rowx = exA_s[rl];
    constexpr int kLd = BN + 1;
    double* stg = reinterpret_cast<double*>(oz_sm);
    // eight columns at a time (64 accumulator registers), so that several
    // elements' integer chains are in flight per thread
    constexpr int kCg = BN / 8 / kGroups;  // 8-column groups per warp
    const int c_end = (warp < kFT / 32) ? (half + 1) * kCg : 0;  // the MMA warp: none
    for (int c = half * kCg; c < c_end; ++c) {
      uint32_t v[kS][8];
#pragma unroll
      for (int d = 0; d < kS; ++d) {
        const uint32_t ta = tbase + (static_cast<uint32_t>(quarter * 32) << 16) + d * BN + c * 8;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]),
                       "=r"(v[d][5]), "=r"(v[d][6]), "=r"(v[d][7])
                     : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row_ok) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int jj = c * 8 + q;
          long long hi = 0, lo = 0;
#pragma unroll
          for (int d = 0; d < 4; ++d)
            hi += static_cast<long long>(__float2int_rn(__uint_as_float(v[d][q]))) << (7 * (3 - d));
#pragma unroll
          for (int d = 4; d < kS; ++d)
            lo += static_cast<long long>(__float2int_rn(__uint_as_float(v[d][q]))) << (7 * (7 - d));
          double val;
          bool ok2 = false;
          if (pow2) val = oz_compose(hi, lo, rowx + colx[jj] - 21, a.alpha < 0.0, ok2);
          if (!ok2) val = (oz_compose(hi, lo, 0, false, ok2) * rowf) * colf[jj];
          stg[rl * kLd + jj] = val;
        }
      }
    }
    __syncthreads();
    // C = staged + beta C, row-wise (coalesced), eight loads of C in flight
    // per thread before the first store
    double* C = a.C + b * a.sC;
    const int rows = min(kTM, M - i0), tot = rows * BN;
    constexpr int kU = 8;
    for (int e0 = threadIdx.x; e0 < tot; e0 += kU * blockDim.x) {
      double cv[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x, r = e / BN, jj = e - r * BN, j = j0 + jj;
        cv[u] = (a.beta != 0.0 && e < tot && j < Nc) ? C[static_cast<size_t>(i0 + r) * a.ldc + j] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x, r = e / BN, jj = e - r * BN, j = j0 + jj;
        if (e < tot && j < Nc) {
          double val = stg[r * kLd + jj];
          if (a.beta != 0.0) val = fma(a.beta, cv[u], val);
          C[static_cast<size_t>(i0 + r) * a.ldc + j] = val;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "n"(Tl::kTmemCols));
}

template <int BN>
cudaError_t oz_run_fused(const OzProduct& g, int batch, void* scratch, int max_batch, int* status,
                         cudaStream_t st) {
  using Tl = OzTile<BN>;
  const int M = g.M, Nc = g.Nc, K = g.K;
  int* kexp = static_cast<int*>(scratch);  // [max_batch][K] balance exponents
  const int nkc = (K + kTK - 1) / kTK;
  const int smem = (nkc > 1 ? kStages : 1) * Tl::kStage;
  cudaError_t e = cudaFuncSetAttribute(k_oz_fused<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStages * Tl::kStage);
  if (e != cudaSuccess) return e;
  for (int b0 = 0; b0 < batch; b0 += max_batch) {
    const int nb = std::min(max_batch, batch - b0);
    const double* ks = g.ks ? g.ks + b0 * g.sks : nullptr;
    const int ks_mode = g.ks ? g.ks_mode : 0;
    if (g.balance)
      k_oz_kexp<<<dim3((K + 7) / 8, nb), 256, 0, st>>>(g.B + b0 * g.sB, g.sB, Nc, K, g.b_sv,
                                                       g.b_sk, g.ks_on_b ? ks : nullptr, g.sks,
                                                       g.ks_on_b ? ks_mode : 0, kexp);
    OzFusedArgs f;
    f.A = g.A + b0 * g.sA; f.sA = g.sA; f.a_sv = g.a_sv; f.a_sk = g.a_sk;
    f.B = g.B + b0 * g.sB; f.sB = g.sB; f.b_sv = g.b_sv; f.b_sk = g.b_sk;
    f.M = M; f.Nc = Nc; f.K = K;
    f.ks = ks; f.sks = g.sks; f.ks_mode = ks_mode; f.ks_on_b = g.ks_on_b;
    f.kexp = g.balance ? kexp : nullptr;
    f.C = g.C + b0 * g.sC; f.sC = g.sC; f.ldc = g.ldc;
    f.rs = g.rs ? g.rs + b0 * g.srs : nullptr; f.srs = g.srs; f.rs_mode = g.rs ? g.rs_mode : 0;
    f.cs = g.cs ? g.cs + b0 * g.scs : nullptr; f.scs = g.scs; f.cs_mode = g.cs ? g.cs_mode : 0;
    f.alpha = g.alpha; f.beta = g.beta;
    f.status = status;
    k_oz_fused<BN><<<dim3((Nc + BN - 1) / BN, (M + kTM - 1) / kTM, nb), kFT + 32, smem, st>>>(f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t oz_slice_elems(int nvec, int K, int R) {
  const size_t nrt = (nvec + R - 1) / R, nkc = (K + kTK - 1) / kTK;
  return static_cast<size_t>(kS) * nrt * R * nkc * kTK;
}

template <int BN>
cudaError_t oz_run(const OzProduct& g, int batch, void* scratch, int max_batch, int* status,
                   cudaStream_t st) {
  using Tl = OzTile<BN>;
  const int M = g.M, Nc = g.Nc, K = g.K;
  const long long slA = static_cast<long long>(oz_slice_elems(M, K, kTM));
  const long long slB = static_cast<long long>(oz_slice_elems(Nc, K, BN));
  __nv_bfloat16* As = static_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* Bs = As + slA * max_batch;
  int* exA = reinterpret_cast<int*>(Bs + slB * max_batch);
  int* exB = exA + static_cast<long long>(M) * max_batch;
  int* kexp = exB + static_cast<long long>(Nc) * max_batch;
  const int nkc = (K + kTK - 1) / kTK;
  const int stages = nkc > 1 ? kStages : 1;  // a single K chunk needs one stage
  const int smem = stages * Tl::kStage;
  cudaError_t e = cudaFuncSetAttribute(k_oz_mma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kStages * Tl::kStage);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_oz_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(oz_split_smem(kMaxN)));
  if (e != cudaSuccess) return e;
  const int rowsA = (M + kTM - 1) / kTM * kTM, rowsB = (Nc + BN - 1) / BN * BN;
  for (int b0 = 0; b0 < batch; b0 += max_batch) {
    const int nb = std::min(max_batch, batch - b0);
    // The inner scale goes with op(A) (ks_on_b = 0) or with op(B).
    const double* ks = g.ks ? g.ks + b0 * g.sks : nullptr;
    const int ks_mode = g.ks ? g.ks_mode : 0;
    const bool on_b = g.ks_on_b != 0;
    if (g.balance)
      k_oz_kexp<<<dim3((K + 7) / 8, nb), 256, 0, st>>>(g.B + b0 * g.sB, g.sB, Nc, K, g.b_sv,
                                                       g.b_sk, on_b ? ks : nullptr, g.sks,
                                                       on_b ? ks_mode : 0, kexp);
    const int* kx = g.balance ? kexp : nullptr;
    // rows of op(A) [diag(ks)] and columns of [diag(ks)] op(B), one launch
    OzSplitOp oa{g.A + b0 * g.sA, g.sA, M, kTM, g.a_sv, g.a_sk, on_b ? nullptr : ks, g.sks,
                 on_b ? 0 : ks_mode, 1, As, slA, exA, M, (rowsA + kSV - 1) / kSV};
    OzSplitOp ob{g.B + b0 * g.sB, g.sB, Nc, BN, g.b_sv, g.b_sk, on_b ? ks : nullptr, g.sks,
                 on_b ? ks_mode : 0, -1, Bs, slB, exB, Nc, (rowsB + kSV - 1) / kSV};
    k_oz_split<<<dim3(oa.blocks + ob.blocks, nb), 256, oz_split_smem(K), st>>>(oa, ob, K, kx);
    OzMmaArgs m;
    m.As = As; m.sAs = slA; m.exA = exA; m.sExA = M;
    m.Bs = Bs; m.sBs = slB; m.exB = exB; m.sExB = Nc;
    m.C = g.C + b0 * g.sC; m.sC = g.sC;
    m.M = M; m.Nc = Nc; m.K = K; m.ldc = g.ldc;
    m.rs = g.rs ? g.rs + b0 * g.srs : nullptr; m.srs = g.srs; m.rs_mode = g.rs ? g.rs_mode : 0;
    m.cs = g.cs ? g.cs + b0 * g.scs : nullptr; m.scs = g.scs; m.cs_mode = g.cs ? g.cs_mode : 0;
    m.alpha = g.alpha; m.beta = g.beta;
    m.status = status;
    k_oz_mma<BN><<<dim3((Nc + BN - 1) / BN, (M + kTM - 1) / kTM, nb), 256, smem, st>>>(m);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

size_t ozaki_scratch_bytes(int n, int max_batch) {
  return static_cast<size_t>(max_batch) *
             ((oz_slice_elems(n, n, kTM) + oz_slice_elems(n, n, kTN)) * 2 + 3ull * n * sizeof(int)) +
         1024;
}

cudaError_t launch_ozaki_product(const OzProduct& g, int batch, void* scratch, int max_batch,
                                 int* status, cudaStream_t st) {
  if (g.M <= 0 || g.Nc <= 0 || g.K <= 0 || batch <= 0) return cudaSuccess;
  if (g.K > kMaxN) return cudaErrorInvalidValue;  // the split kernel stages K scales in smem
  // Products with a short inner dimension or few columns (the panel updates
  // of the blocked QR) are cut into digits by the product kernel itself; the
  // square products split both operands once in a separate kernel, which on
  // this part measured faster than re-cutting op(A) for every column tile.
  if (g.K <= 64 || g.Nc <= 32) {
    if (g.Nc <= 32) return oz_run_fused<32>(g, batch, scratch, max_batch, status, st);
    return oz_run_fused<64>(g, batch, scratch, max_batch, status, st);
  }
  return oz_run<64>(g, batch, scratch, max_batch, status, st);
}

cudaError_t launch_gemm_ozaki(const GemmArgs& g, int batch, void* scratch, int max_batch,
                              int* status, cudaStream_t st) {
  const int n = g.n;
  OzProduct p{};
  p.M = p.Nc = p.K = n;
  p.A = g.A; p.sA = g.sA;
  // rows of op(A): tA = 0 -> A[i][k]; tA = 1 -> A[k][i]
  p.a_sv = g.tA ? 1 : n; p.a_sk = g.tA ? n : 1;
  p.B = g.B; p.sB = g.sB;
  // op(B) element (k, j): tB = 0 -> B[k][j]; tB = 1 -> B[j][k]
  p.b_sv = g.tB ? n : 1; p.b_sk = g.tB ? 1 : n;
  p.C = g.C; p.sC = g.sC; p.ldc = n;
  p.rs = g.rs; p.srs = g.srs; p.rs_mode = g.rs_mode;
  p.ks = g.ks; p.sks = g.sks; p.ks_mode = g.ks_mode; p.ks_on_b = g.ks_on_b;
  p.balance = g.balance;
  p.cs = g.cs; p.scs = g.scs; p.cs_mode = g.cs_mode;
  p.alpha = g.alpha; p.beta = g.beta;
  return launch_ozaki_product(p, batch, scratch, max_batch, status, st);
}

}  // namespace dqmc
