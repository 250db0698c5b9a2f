// FP64 stabilisation kernels that spread one matrix over a thread-block
// cluster of CS CTAs (one SM each), so that a batch of 64 matrices of order
// 256 keeps 128 SMs busy instead of 64.  The matrices stay in global memory
// (L2-resident: 512 KB each); each CTA updates the columns (QR) or rows
// (Gauss-Jordan) it owns, and the CTAs meet at cluster barriers.  Within a
// CTA every warp works on four columns at a time so that the FP64 pipe sees
// independent dot products instead of one shuffle-reduction chain.
//
// Same mathematics as k_qrp / k_gj_inverse in k_linalg.cu (paper: the UDV
// stabilisation behind Eq. (3) and G_ij(tau_l), Sec. 2).
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace dqmc {
namespace {

// Pivot search keys are compared in FP32: the choice of pivot only steers the
// numerics (any pivot order gives an exact factorisation), and FP64 compares
// cost a full pass of the 1/64-rate FP64 pipe on this part.
struct AM {
  float v;
  int i;
};

__device__ __forceinline__ AM am_combine(AM a, AM b) {
  return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
}

__device__ __forceinline__ AM warp_am(AM x) {
  for (int o = 16; o > 0; o >>= 1) {
    AM y;
    y.v = __shfl_xor_sync(0xFFFFFFFFu, x.v, o);
    y.i = __shfl_xor_sync(0xFFFFFFFFu, x.i, o);
    x = am_combine(x, y);
  }
  return x;
}

// log2 |x| of a double in integer and FP32 arithmetic (exponent field plus
// the FP32 log2 of the leading 23 mantissa bits): -2000 for zero and
// subnormals, NaN for Inf/NaN.  Used for the pivoting norms, which only steer
// the column order.
__device__ __forceinline__ float log2_abs(double x) {
  const long long bits = __double_as_longlong(x);
  const int e = static_cast<int>((bits >> 52) & 0x7FF);
  if (e == 0) return -2000.0f;
  if (e == 0x7FF) return __int_as_float(0x7FC00000);
  const float m = __int_as_float(0x3F800000 | static_cast<int>((bits >> 29) & 0x7FFFFF));
  return static_cast<float>(e - 1023) + __log2f(m);
}

__device__ __forceinline__ double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Warp sums of four values per lane with 6 FP64 additions instead of 20: the
// first two butterfly stages exchange the halves each lane gives away, so a
// lane carries 2, then 1 partial sum; afterwards lanes 8q .. 8q+7 hold the
// sum of value q, which is scaled by `scale` and broadcast.
__device__ __forceinline__ void wsum4(double (&a)[4], double scale) {
  const int lane = threadIdx.x & 31;
  const bool lo16 = lane < 16;
  const double s0 = lo16 ? a[2] : a[0], s1 = lo16 ? a[3] : a[1];
  const double k0 = lo16 ? a[0] : a[2], k1 = lo16 ? a[1] : a[3];
  const double b0 = k0 + __shfl_xor_sync(0xFFFFFFFFu, s0, 16);
  const double b1 = k1 + __shfl_xor_sync(0xFFFFFFFFu, s1, 16);
  const bool hi8 = (lane & 8) != 0;
  double c = (hi8 ? b1 : b0) + __shfl_xor_sync(0xFFFFFFFFu, hi8 ? b0 : b1, 8);
  c += __shfl_xor_sync(0xFFFFFFFFu, c, 4);
  c += __shfl_xor_sync(0xFFFFFFFFu, c, 2);
  c += __shfl_xor_sync(0xFFFFFFFFu, c, 1);
  c *= scale;
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = __shfl_sync(0xFFFFFFFFu, c, 8 * q);
}

// Apply I - tau v v^T (v = vsh[j..n), v_j = 1) to the rows M[c][j..n) of
// columns owned by this CTA, four columns per warp at a time.
// The columns are cols[0 .. m) or, without a list, c0 + CS i (i < m).  If
// ln1 != nullptr the partial column norms are downdated.  The norms
// are kept as FP32 log2 values (ln1: current, ln2: at the last exact
// recomputation); the downdate of LAPACK's xLAQP2,
//   n1 <- n1 sqrt(1 - (|r|/n1)^2), recomputed when (1 - (|r|/n1)^2)(n1/n2)^2
//   falls below sqrt(eps),
// runs in that form on one lane.
template <int CS>
__device__ __forceinline__ void reflect_owned(double* M, int n, int j, const int* cols, int m,
                                              int c0, double tau, const double* vsh, float* ln1,
                                              float* ln2, float tol3z) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int g = w; 4 * g < m; g += nw) {
    int c[4];
    bool ok[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = 4 * g + q;
      ok[q] = idx < m;
      const int ci = cols ? cols[ok[q] ? idx : 0] : c0 + CS * (ok[q] ? idx : 0);
      c[q] = ci;
    }
    // All rows of the four columns are loaded before any arithmetic, so each
    // lane has up to 4 x kRPL independent loads in flight.
    constexpr int kRPL = kMaxN / 32;
    const int tmax = (n - j + 31) >> 5;  // warp-uniform: row slots that still hold live rows
    double x[4][kRPL];
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      if (t < tmax) {
        const int r = j + lane + 32 * t;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          x[q][t] = (ok[q] && r < n) ? M[static_cast<size_t>(c[q]) * n + r] : 0.0;
      }
    }
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      if (t < tmax) {
        const int r = j + lane + 32 * t;
        const double vr = (r < n) ? vsh[r] : 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(vr, x[q][t], acc[q]);
      }
    }
    wsum4(acc, tau);
    double top[4];
#pragma unroll
    for (int t = 0; t < kRPL; ++t) {
      if (t < tmax) {
        const int r = j + lane + 32 * t;
        const double vr = (r < n) ? vsh[r] : 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          x[q][t] -= acc[q] * vr;
          if (ok[q] && r < n) M[static_cast<size_t>(c[q]) * n + r] = x[q][t];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) top[q] = x[q][0];  // row j lives in lane 0, t = 0
    if (ln1 == nullptr) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (!ok[q]) continue;
      int rec = 0;
      float nl1 = 0.0f, nl2 = 0.0f;
      if (lane == 0) {
        const float l1 = ln1[c[q]], l2 = ln2[c[q]];
        nl1 = l1;
        nl2 = l2;
        if (l1 > -1000.0f) {
          const float rt = log2_abs(top[q]) - l1;  // log2(|r| / n1)
          const float t = fmaxf(0.0f, 1.0f - exp2f(2.0f * rt));
          if (!(t * exp2f(2.0f * (l1 - l2)) > tol3z))
            rec = 1;
          else
            nl1 = l1 + 0.5f * __log2f(t);
        }
      }
      if (__shfl_sync(0xFFFFFFFFu, rec, 0) != 0) {
        double s2 = 0.0;
        for (int r = j + 1 + lane; r < n; r += 32) {
          const double x = M[static_cast<size_t>(c[q]) * n + r];
          s2 = fma(x, x, s2);
        }
        s2 = wsum(s2);
        nl1 = nl2 = 0.5f * log2_abs(s2);
      }
      __syncwarp();
      if (lane == 0) {
        ln1[c[q]] = nl1;
        ln2[c[q]] = nl2;
      }
    }
  }
}

// Element helpers of the Gauss-Jordan kernel for FP64 and float pairs.
__device__ __forceinline__ float gj_mag(double x) { return static_cast<float>(absd(x)); }
__device__ __forceinline__ float gj_mag(df32 x) { return fabsf(x.hi); }
__device__ __forceinline__ double gj_d(double x) { return x; }
__device__ __forceinline__ double gj_d(df32 x) { return static_cast<double>(x); }
__device__ __forceinline__ double gj_shfl(double x, int l) { return __shfl_sync(0xFFFFFFFFu, x, l); }
__device__ __forceinline__ df32 gj_shfl(df32 x, int l) {
  return df32(__shfl_sync(0xFFFFFFFFu, x.hi, l), __shfl_sync(0xFFFFFFFFu, x.lo, l));
}
// a b + c: for float pairs the product's error terms and one TwoSum with
// c.hi, rounded once (about 15 FP32 instructions, relative error ~2^-48)
__device__ __forceinline__ double gj_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ df32 gj_fma(df32 a, df32 b, df32 c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df32 s = df_two_sum(c.hi, p);
  return df_fast_two_sum(s.hi, s.lo + (c.lo + e));
}

// In-place FP64 -> float pair of a batch of matrices (same 8 bytes per entry).
__global__ void __launch_bounds__(256) k_to_pair(double* A, long long count) {
  for (long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const double x = A[e];
    reinterpret_cast<df32*>(A)[e] = df32(x);
  }
}

// First column >= lo owned by cluster rank `rank` (ownership: c % CS == rank).
template <int CS>
__device__ __forceinline__ int first_owned(int lo, int rank) {
  return lo + ((rank - lo % CS) % CS + CS) % CS;
}

}  // namespace

// ---------------------------------------------------------------------------
// Householder QR with column pivoting of X^T (row c = column c of X), one
// cluster of CS CTAs per matrix.  Outputs as k_qrp: Q^T, D = |diag R| and
// Rtil = D^{-1} R P^T.  The Householder vectors are parked in the Rtil buffer
// until Q is formed.
//
// Pivoting is logical: a chosen column stays where it is and records its
// step, each CTA keeps the columns it owns (c % CS == rank) that are still
// live in a compact list and their partial norms (log2, FP32) in shared
// memory.  After updating its columns a CTA publishes the best of them to
// every CTA of the cluster (distributed shared memory, buffered by step
// parity), so one cluster barrier per step orders both the column data in
// global memory and the pivot candidates.  The head of a step (combining the
// candidates, the reflector of the pivot column) runs in warp 0 of every CTA.
// ---------------------------------------------------------------------------
template <int CS>
__global__ void __launch_bounds__(512) k_qrp_cluster(double* Xall, long long sX, double* Qall,
                                                    long long sQ, double* Dall, long long sD,
                                                    double* Rall, long long sR, double* Vn, int n,
                                                    int* status) {
  (void)Vn;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int b = blockIdx.x / CS;
  double* X = Xall + b * sX;
  double* Qt = Qall + b * sQ;
  double* D = Dall + b * sD;
  double* Rt = Rall + b * sR;
  __shared__ double vsh[kMaxN], taus[kMaxN], betas[kMaxN];
  __shared__ float ln1[kMaxN], ln2[kMaxN];  // log2 partial norms of the owned columns
  __shared__ int stepof[kMaxN];             // step at which column c was chosen (n: not yet)
  __shared__ int live[kMaxN], pos[kMaxN];   // owned live columns and their list positions
  __shared__ int nlive;
  __shared__ AM cand[2][CS];                // best live column of every CTA, by step parity
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const float tol3z = 1.4901161193847656e-08f;  // sqrt(DBL_EPSILON)

  for (int c = rank + CS * w; c < n; c += CS * nw) {
    double s = 0.0;
    for (int r = lane; r < n; r += 32) {
      const double x = X[static_cast<size_t>(c) * n + r];
      s = fma(x, x, s);
    }
    s = wsum(s);
    if (lane == 0) ln1[c] = ln2[c] = 0.5f * log2_abs(s);
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) stepof[c] = n;
  if (threadIdx.x == 0) {
    int m = 0;
    for (int c = rank; c < n; c += CS) {
      pos[c] = m;
      live[m++] = c;
    }
    nlive = m;
  }
  __syncthreads();
  // publish the best owned column for step 0 (warp 0)
  auto publish = [&](int slot) {
    AM m{-3.0e38f, n};
    for (int i = lane; i < nlive; i += 32) m = am_combine(m, AM{ln1[live[i]], live[i]});
    m = warp_am(m);
    if (lane < CS) *cl.map_shared_rank(&cand[slot][rank], lane) = m;
  };
  if (w == 0) publish(0);
  cl.sync();

  for (int j = 0; j < n; ++j) {
    if (w == 0) {
      // pivot: best candidate over the cluster (same order everywhere)
      AM m{-3.0e38f, n};
#pragma unroll
      for (int r = 0; r < CS; ++r) m = am_combine(m, cand[j & 1][r]);
      int p = m.i;
      if (p < 0 || p >= n || stepof[p] != n) {  // no finite candidate: flag, take a free column
        if (lane == 0) atomicExch(status, kDevNonFinite);
        p = 0;
        while (p < n - 1 && stepof[p] != n) ++p;
      }
      // reflector of column p (rows j .. n-1)
      const double* xp = X + static_cast<size_t>(p) * n;
      double sig = 0.0;
      for (int r = j + 1 + lane; r < n; r += 32) sig = fma(xp[r], xp[r], sig);
      sig = wsum(sig);
      const double alpha = xp[j];
      double tau = 0.0, beta = alpha, scal = 1.0;
      if (lane == 0 && sig != 0.0) {  // scalars on one lane, then broadcast
        const double nr = sqrt(alpha * alpha + sig);
        beta = (alpha <= 0.0) ? nr : -nr;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      tau = __shfl_sync(0xFFFFFFFFu, tau, 0);
      beta = __shfl_sync(0xFFFFFFFFu, beta, 0);
      scal = __shfl_sync(0xFFFFFFFFu, scal, 0);
      for (int r = j + lane; r < n; r += 32) {
        const double v = (r == j) ? 1.0 : xp[r] * scal;
        vsh[r] = v;
        if (rank == 0 && r > j) Rt[static_cast<size_t>(j) * n + r] = v;
      }
      if (lane == 0) {
        taus[j] = tau;
        betas[j] = beta;
        stepof[p] = j;
        if (p % CS == rank) {  // drop p from the owned live list
          const int at = pos[p], last = live[nlive - 1];
          live[at] = last;
          pos[last] = at;
          --nlive;
        }
      }
    }
    __syncthreads();
    reflect_owned<CS>(X, n, j, live, nlive, 0, taus[j], vsh, ln1, ln2, tol3z);
    __syncthreads();
    if (w == 0) publish((j + 1) & 1);
    cl.sync();
  }

  // Q = H_0 ... H_{n-1} accumulated backwards, owned columns (rows of Q^T).
  for (int c = rank; c < n; c += CS)
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      Qt[static_cast<size_t>(c) * n + r] = (c == r) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    for (int r = j + threadIdx.x; r < n; r += blockDim.x)
      vsh[r] = (r == j) ? 1.0 : Rt[static_cast<size_t>(j) * n + r];
    __syncthreads();
    const double tau = taus[j];
    const int c0 = first_owned<CS>(j, rank);
    if (tau != 0.0)
      reflect_owned<CS>(Qt, n, j, nullptr, (c0 < n) ? (n - c0 + CS - 1) / CS : 0, c0, tau, vsh,
                        nullptr, nullptr, tol3z);
    __syncthreads();
  }
  cl.sync();  // every CTA is done with the Householder vectors in Rt

  // D = |beta|; Rtil[i][c] = R[i][s] / D[i] with s = stepof[c] the pivot
  // position of column c: R[i][s] = X[c][i] for s > i, beta_i for s = i.
  for (int i = rank; i < n; i += CS) {
    double d = absd(betas[i]);
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicExch(status, kDevSingular);
      d = DBL_MIN;
    }
    if (threadIdx.x == 0) D[i] = d;
    const double rd = 1.0 / d;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int sc = stepof[c];
      double v = 0.0;
      if (sc > i)
        v = X[static_cast<size_t>(c) * n + i] * rd;
      else if (sc == i)
        v = betas[i] * rd;
      Rt[static_cast<size_t>(i) * n + c] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inverse, one cluster of CS CTAs per matrix, rows owned by
// CTA (row % CS).  Pivot rows are chosen (partial pivoting over the rows not
// yet used) but never moved; with pr[k] the pivot row of step k and ip its
// inverse permutation, the in-place result Z gives A^{-1}[k][j] = Z[pr[k]][ip[j]],
// written to Ainv at the end.  A is overwritten.
//
// One cluster barrier per step.  Within a step a CTA reads only its own rows
// and the pivot row, which no CTA writes during the step (its scaled values
// are written by the owner one step late, when no CTA reads that row any
// more).  The pivot search therefore cannot look at a peer's rows: after its
// elimination every CTA takes the largest |A[i][k+1]| over its own unused
// rows and publishes it to every CTA of the cluster (distributed shared
// memory, buffered by step parity), before the barrier.
// ---------------------------------------------------------------------------
template <int CS, typename T>
__global__ void __launch_bounds__(512) k_gj_cluster(T* Aall, long long sA, double* Iall,
                                                   long long sI, int n, double* logabs,
                                                   int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int b = blockIdx.x / CS;
  T* A = Aall + b * sA;
  double* Ainv = Iall + b * sI;
  __shared__ T prow[kMaxN], pend[kMaxN];
  __shared__ int pr[kMaxN], ip[kMaxN];
  __shared__ unsigned char used[kMaxN];
  __shared__ AM cand[2][CS];  // best unused owned row of every CTA for the next column
  __shared__ T sinv;
  __shared__ double pivs[kMaxN];  // |pivot| of every step (log|det A| after the loop)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) used[i] = 0;
  int pend_row = -1;  // owned pivot row whose scaled values wait in pend[]
  __syncthreads();
  // warp 0: best |A[i][col]| over the owned unused rows, sent to every CTA
  auto publish = [&](int col, int slot) {
    AM m{-1.0f, n};
    for (int i = rank + CS * lane; i < n; i += CS * 32)
      if (!used[i]) m = am_combine(m, AM{gj_mag(A[static_cast<size_t>(i) * n + col]), i});
    m = warp_am(m);
    if (lane < CS) *cl.map_shared_rank(&cand[slot][rank], lane) = m;
  };
  if (w == 0) publish(0, 0);
  cl.sync();
  for (int k = 0; k < n; ++k) {
    if (pend_row >= 0) {
      for (int jj = threadIdx.x; jj < n; jj += blockDim.x)
        A[static_cast<size_t>(pend_row) * n + jj] = pend[jj];
      pend_row = -1;
    }
    AM m{-1.0f, n};
#pragma unroll
    for (int r = 0; r < CS; ++r) m = am_combine(m, cand[k & 1][r]);
    int p = m.i;
    if (p < 0 || p >= n || used[p]) {  // no finite pivot left: flag, take the first free row
      if (threadIdx.x == 0) atomicExch(status, kDevNonFinite);
      p = 0;
      while (p < n - 1 && used[p]) ++p;
    }
    if (threadIdx.x == 0) {  // pivot scalars: one thread, then broadcast
      double piv = gj_d(A[static_cast<size_t>(p) * n + k]);
      if (!(absd(piv) > 0.0)) {
        atomicExch(status, kDevSingular);
        piv = DBL_MIN;
      }
      pivs[k] = absd(piv);
      sinv = T(1.0 / piv);  // a float pair takes the FP64 reciprocal, split
    }
    __syncthreads();
    const T ipiv = sinv;
    for (int jj = threadIdx.x; jj < n; jj += blockDim.x)
      prow[jj] = (jj == k) ? ipiv : A[static_cast<size_t>(p) * n + jj] * ipiv;
    __syncthreads();
    if (threadIdx.x == 0) {
      used[p] = 1;
      pr[k] = p;
    }
    // eliminate column k from the owned rows (the owned pivot row is only scaled)
    constexpr int kRPL = kMaxN / 32;
    const int tk = k >> 5, lk = k & 31;
    for (int i0 = rank + CS * w; i0 < n; i0 += 2 * CS * nw) {
      // two owned rows per warp and iteration, all their loads issued together
      const int ii[2] = {i0, i0 + CS * nw};
      T xv[2][kRPL];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int t = 0; t < kRPL; ++t) {
          const int jj = lane + 32 * t;
          xv[h][t] = (ii[h] < n && jj < n) ? A[static_cast<size_t>(ii[h]) * n + jj] : T(0.0f);
        }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = ii[h];
        if (i >= n) continue;
        T* Ai = A + static_cast<size_t>(i) * n;
        if (i == p) {
          for (int jj = lane; jj < n; jj += 32) pend[jj] = prow[jj];
          continue;
        }
        T fk = T(0.0f);
#pragma unroll
        for (int t = 0; t < kRPL; ++t)
          if (t == tk) fk = xv[h][t];
        const T nf = -gj_shfl(fk, lk);
        const T vk = nf * prow[k];  // new entry of the pivot column (one product per row)
#pragma unroll
        for (int t = 0; t < kRPL; ++t) {
          const int jj = lane + 32 * t;
          if (jj < n) {
            const T v = gj_fma(nf, prow[jj], xv[h][t]);
            Ai[jj] = (jj == k) ? vk : v;
          }
        }
      }
    }
    if (p % CS == rank) pend_row = p;
    __syncthreads();  // this CTA's eliminated rows and used[] are complete
    if (w == 0 && k + 1 < n) publish(k + 1, (k + 1) & 1);
    cl.sync();
  }
  if (pend_row >= 0)
    for (int jj = threadIdx.x; jj < n; jj += blockDim.x)
      A[static_cast<size_t>(pend_row) * n + jj] = pend[jj];
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) ip[pr[k]] = k;
  cl.sync();
  for (int k = rank; k < n; k += CS) {
    const T* Zr = A + static_cast<size_t>(pr[k]) * n;
    for (int jj = threadIdx.x; jj < n; jj += blockDim.x)
      Ainv[static_cast<size_t>(k) * n + jj] = gj_d(Zr[ip[jj]]);
  }
  if (logabs && rank == 0) {  // log|det| = sum_k log|pivot_k|, off the step loop
    double la = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) la += log(pivs[k]);
    la = wsum(la);
    __shared__ double lsum[32];
    if (lane == 0) lsum[w] = la;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < nw; ++q) t += lsum[q];
      logabs[b] = t;
    }
  }
}

template <typename K, typename... Args>
static cudaError_t launch_cluster(K kern, int cs, int batch, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs * batch, 1, 1);
  cfg.blockDim = dim3(512, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_qrp_cluster(double* Xt, long long sX, double* Qt, long long sQ, double* D,
                               long long sD, double* Rtil, long long sR, double* vnorm, int n,
                               int batch, int* status, cudaStream_t st) {
  return launch_cluster(k_qrp_cluster<2>, 2, batch, st, Xt, sX, Qt, sQ, D, sD, Rtil, sR, vnorm, n,
                        status);
}

cudaError_t launch_gj_cluster(double* A, long long sA, double* Ainv, long long sI, int n, int batch,
                              double* logabs, int* status, cudaStream_t st, bool pair) {
  // Small batches (the per-point recompute: one matrix per chain) spread each
  // matrix over 4 CTAs, two of which fit on an SM (512 threads x 64
  // registers), so that twice as many warps hide the step latency; large
  // batches keep 2 CTAs per matrix.
  // SM count of the current device, cached per device (a process may drive
  // several GPUs)
  constexpr int kMaxDev = 64;
  static int nsm_of[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  int nsm = (dev >= 0 && dev < kMaxDev) ? nsm_of[dev] : 0;
  if (nsm == 0) {
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 1;
    if (dev >= 0 && dev < kMaxDev) nsm_of[dev] = nsm;
  }
  if (pair) {  // float-pair elimination: A becomes an array of pairs in place
    const long long count = static_cast<long long>(batch - 1) * sA + static_cast<long long>(n) * n;
    k_to_pair<<<static_cast<int>(std::min<long long>((count + 255) / 256, 4096)), 256, 0, st>>>(A, count);
    df32* Ap = reinterpret_cast<df32*>(A);
    if (4LL * batch <= 2LL * nsm)
      return launch_cluster(k_gj_cluster<4, df32>, 4, batch, st, Ap, sA, Ainv, sI, n, logabs, status);
    return launch_cluster(k_gj_cluster<2, df32>, 2, batch, st, Ap, sA, Ainv, sI, n, logabs, status);
  }
  if (4LL * batch <= 2LL * nsm)
    return launch_cluster(k_gj_cluster<4, double>, 4, batch, st, A, sA, Ainv, sI, n, logabs, status);
  return launch_cluster(k_gj_cluster<2, double>, 2, batch, st, A, sA, Ainv, sI, n, logabs, status);
}

}  // namespace dqmc
