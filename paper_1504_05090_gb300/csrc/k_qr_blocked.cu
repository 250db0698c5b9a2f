// Blocked Householder QR with panel-wise pivoting for the UDV stack of
// Eq. (3) (Sec. 2: the O(Lambda N^3) stabilised matrix work behind
// G_ij(tau_l)).
//
// Input and output as the column-pivoted QR of k_cluster.cu: X^T stored
// row-major (row c = column c of X) in; Q^T, D = |diag R| and
// Rtil = D^{-1} R P^T with X = Q diag(D) Rtil out.  Pivoting works on blocks
// of kNB columns: at the start of each panel the columns not yet factorised
// are sorted by the norm of their remaining part (rows c0 .. n - 1, after all
// earlier reflectors), the kNB largest form the panel, and within the panel
// each step takes the column of largest remaining norm (downdated as in
// LAPACK's xGEQP3).  For the graded products B_l ... B_1 U D of the stack
// this keeps |R_ij| close to |R_ii| as column pivoting does, so that
// T = D^{-1} R P^T stays well conditioned, while the trailing updates run as
// matrix products:
//
//   for each panel of w <= kNB columns (rows c0 .. n - 1):
//     k_qrb_panel  sort the remaining columns, FP64 Householder QR of the
//                  panel in shared memory with local pivoting, the compact-WY
//                  factor T of its reflectors (H_0 ... H_{w-1} = I - V T V^T)
//                  and Y = T^T V^T;
//     trailing columns A <- (I - V T^T V^T) A = A - V (Y A), written in the
//     transposed storage (rows of A_rows = columns of A) as two tensor-core
//     products:
//       W^T = A_rows Y^T          (M = trailing columns, N = w, K = m)
//       A_rows -= W^T V^T         (M = trailing columns, N = m, K = w)
//   Q^T accumulated backwards from I, Q^T <- Q^T (I - V T^T V^T):
//       W^T = Qt_rows V           (M = m, N = w, K = m)
//       Qt_rows -= W^T Y          (M = m, N = m, K = w)
//
// The products run on the digit-sliced tcgen05 path (k_ozaki.cu), which keeps
// FP64-level accuracy relative to the size of each row and column; only the
// panels use the FP64 pipe.
//
// Storage per matrix: two buffers that the panels alternate between (the
// rows of panel p, R on and above the diagonal, stay in the buffer that
// panel wrote), the Householder vectors V^T in the Rtil buffer and
// Y = T^T V^T in the X buffer (each consumed before it is overwritten).
#include <cooperative_groups.h>

#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace dqmc {
namespace {

namespace cg = cooperative_groups;

constexpr int kNB = 32;  // panel width

__device__ __forceinline__ double qb_wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// log2 of the squared norm of x[0 .. len) as an FP32 sort key, from the
// exponent fields and the FP32 mantissas (the order only steers the
// numerics; any order gives an exact factorisation).  One warp, len <= kMaxN;
// every element is loaded once, all loads of a lane in flight together.  The
// key is returned on every lane: +3e38 for Inf/NaN entries, -3e38 for a zero
// vector.
__device__ __forceinline__ float qb_norm_key(const double* x, int len, int lane) {
  constexpr int kR = kMaxN / 32;
  long long bits[kR];
#pragma unroll
  for (int t = 0; t < kR; ++t) {
    const int r = lane + 32 * t;
    bits[t] = (r < len) ? __double_as_longlong(x[r]) : 0LL;
  }
  int emax = 0;
  bool bad = false;
#pragma unroll
  for (int t = 0; t < kR; ++t) {
    const int E = static_cast<int>((bits[t] >> 52) & 0x7FF);
    bad |= (E == 0x7FF);
    emax = max(emax, E);
  }
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, o));
  bad = __any_sync(0xFFFFFFFFu, bad);
  float s = 0.0f;
#pragma unroll
  for (int t = 0; t < kR; ++t) {
    const int E = static_cast<int>((bits[t] >> 52) & 0x7FF);
    if (E != 0) {
      const float mt = __int_as_float(0x3F800000 | static_cast<int>((bits[t] >> 29) & 0x7FFFFF));
      const float y = ldexpf(mt, E - emax);
      s = fmaf(y, y, s);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (bad) return 3.0e38f;
  if (emax == 0) return -3.0e38f;
  return 2.0f * static_cast<float>(emax - 1023) + __log2f(s);
}

// Warp sums of four values per lane: lanes 8q .. 8q + 7 end with the sum of
// value q, which is broadcast back to every lane (6 FP64 additions instead
// of 20: the first two butterfly stages exchange the halves each lane gives
// away).
__device__ __forceinline__ void qb_wsum4(double (&a)[4]) {
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
#pragma unroll
  for (int q = 0; q < 4; ++q) a[q] = __shfl_sync(0xFFFFFFFFu, c, 8 * q);
}

constexpr int kPT = 512;  // threads of each CTA of the panel kernel

// Rows of a panel per CTA: the pair of CTAs of a matrix splits the m rows,
// CTA 0 taking rows [0, h) with h >= w, so that the diagonal block (rows
// q < w, where the reflectors start and R ends) is entirely its own.
__host__ __device__ __forceinline__ int qb_split(int m, int w) {
  const int half = (m + 1) / 2;
  const int h = half > w ? half : w;
  return h < m ? h : m;
}

// One exchange between the two CTAs of a matrix (distributed shared memory):
// a[r][s] is CTA r's partial sum for panel column s, b[s] a value that only
// CTA 0 holds (an entry of the diagonal block).
struct QbXch {
  double a[2][kNB];
  double b[kNB];
};

// One panel, one cluster of two CTAs per matrix, the panel's rows split
// between them (qb_split); rows of the transposed storage are columns of X;
// `src` holds the matrix after the previous panel (the input X^T for the
// first), `dst` receives the rows c0 .. n - 1.
//  1. Sort: the rows c >= c0 of src by the norm of their entries c0 .. n - 1
//     (each CTA finds the keys of half of them and writes them to both);
//     rank w .. m - 1 go to dst rows c0 + w .. n - 1 (whole rows), perm
//     follows.
//  2. The w largest are the panel: P[q][rl] = entry c0 + r0 + rl of panel
//     column q for the CTA's rows r0 + rl.  Step q (as LAPACK's xGEQP3 within
//     the panel): take the panel column of largest remaining norm (rows q ..)
//     into position q, the reflector H_q = I - tau_q v_q v_q^T with v_q[q] = 1
//     that maps P[q][q..m) to beta_q e_q, applied to the panel columns
//     q + 1 .. w - 1.  The norms are not downdated: the same pass that
//     applies H_q sums the squares of every column's rows q + 2 .. (the
//     reflector's sigma at the next step) and CTA 0 reads off row q + 1, so
//     that both CTAs hold the exact alpha^2 + sigma of every candidate.
//     Two exchanges per step, each closed by a cluster barrier (the same
//     number in both CTAs, independent of the data): the partial dot
//     products v_q . x_s, then the partial sums of squares with row q + 1.
//     Every value both CTAs use is summed in the same order on both, so
//     their pivots and reflector scalars are identical.
//  3. Gram matrix V^T V from the partial sums of both CTAs; T column by
//     column, T[0:q, q] = -tau_q T[0:q, 0:q] (V^T v_q)[0:q], T[q][q] = tau_q
//     (on both CTAs); then Y = T^T V^T for the CTA's rows.
//  4. Panel rows to dst rows c0 .. c0 + w - 1 (entries below c0 moved with
//     their column, R on and above the diagonal, beta_q on it, v_q below),
//     v_q to row c0 + q of Vt, Y to rows c0 .. of Yt (entries c0 ..),
//     D[c0 + q] = |beta_q|, perm.
__global__ void __launch_bounds__(kPT) k_qrb_panel(const double* Wsall, long long sWs, double* Wdall,
                                                  long long sWd, int* permall, double* Vall,
                                                  long long sV, double* Yall, long long sY,
                                                  double* Dall, long long sD, int n, int c0, int w,
                                                  int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank()), peer = rank ^ 1;
  const int b = blockIdx.x >> 1;
  const int m = n - c0;
  const int h = qb_split(m, w);
  const int r0 = rank ? h : 0, ml = (rank ? m : h) - r0;  // this CTA's rows r0 .. r0 + ml - 1
  const double* Ws = Wsall + b * sWs;
  double* Wd = Wdall + b * sWd;
  int* perm = permall + static_cast<long long>(b) * n;
  double* Vt = Vall + b * sV;
  double* Yt = Yall + b * sY;
  double* D = Dall + b * sD;
  extern __shared__ __align__(16) double qb_sm[];
  double* P = qb_sm;  // [w][ml]
  __shared__ float key[kMaxN];
  __shared__ int src_of[kMaxN];  // rank -> source row - c0
  __shared__ int pold[kMaxN];    // perm[c0 ..] on entry
  __shared__ double T[kNB][kNB + 1];
  __shared__ double Gp[2][kNB][kNB + 1];  // Gram partials of the two CTAs, [s][q] for s < q
  __shared__ QbXch xch[2];
  __shared__ double taus[kNB], betas[kNB], sig[kNB], alp[kNB];
  __shared__ double scal_sh;
  __shared__ int lp[kNB];  // panel position -> rank of its column
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  // 1. sort the remaining columns
  {
    float* key_peer = cl.map_shared_rank(key, peer);
    const int kh = (m + 1) / 2, k0 = rank ? kh : 0, k1 = rank ? m : kh;
    for (int c = k0 + wp; c < k1; c += nw) {
      const float k = qb_norm_key(Ws + static_cast<size_t>(c0 + c) * n + c0, m, lane);
      if (lane == 0) {
        key[c] = k;
        key_peer[c] = k;
      }
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) pold[i] = (c0 == 0) ? i : perm[c0 + i];
  cl.sync();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const float ki = key[i];
    int rk = 0;
    for (int i2 = 0; i2 < m; ++i2) {
      const float k2 = key[i2];
      rk += (k2 > ki || (k2 == ki && i2 < i)) ? 1 : 0;
    }
    src_of[rk] = i;
  }
  __syncthreads();
  {  // whole rows, a warp per row (rows interleaved between the CTAs), all
     // loads of a lane in flight before its stores
    constexpr int kR = kMaxN / 32;
    for (int pos = w + rank * nw + wp; pos < m; pos += 2 * nw) {
      const double* srow = Ws + static_cast<size_t>(c0 + src_of[pos]) * n;
      double* drow = Wd + static_cast<size_t>(c0 + pos) * n;
      double t[kR];
#pragma unroll
      for (int u = 0; u < kR; ++u) t[u] = (lane + 32 * u < n) ? srow[lane + 32 * u] : 0.0;
#pragma unroll
      for (int u = 0; u < kR; ++u)
        if (lane + 32 * u < n) drow[lane + 32 * u] = t[u];
    }
  }
  if (rank == 0)
    for (int pos = w + threadIdx.x; pos < m; pos += blockDim.x) perm[c0 + pos] = pold[src_of[pos]];
  // 2. the panel: this CTA's rows of the w columns
  {
    constexpr int kU = kNB * kMaxN / 2 / kPT;
    double t[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = threadIdx.x + u * kPT, q = e / max(ml, 1), rl = e - q * max(ml, 1);
      t[u] = (e < w * ml) ? Ws[static_cast<size_t>(c0 + src_of[q]) * n + c0 + r0 + rl] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = threadIdx.x + u * kPT;
      if (e < w * ml) P[e] = t[u];
    }
  }
  if (threadIdx.x < w) lp[threadIdx.x] = threadIdx.x;
  __syncthreads();
  int xk = 0;  // exchanges so far; exchange k uses slot k & 1
  {  // sigma (rows 1 ..) and alpha (row 0) of every column before step 0
    QbXch* mine = &xch[0];
    QbXch* theirs = cl.map_shared_rank(mine, peer);
    for (int q = wp; q < w; q += nw) {
      double a = 0.0;
      for (int rl = lane; rl < ml; rl += 32)
        if (r0 + rl > 0) a = fma(P[q * ml + rl], P[q * ml + rl], a);
      a = qb_wsum(a);
      if (lane == 0) {
        mine->a[rank][q] = a;
        theirs->a[rank][q] = a;
        if (rank == 0) {
          mine->b[q] = P[q * ml];
          theirs->b[q] = P[q * ml];
        }
      }
    }
    cl.sync();
    if (threadIdx.x < w) {
      sig[threadIdx.x] = mine->a[0][threadIdx.x] + mine->a[1][threadIdx.x];
      alp[threadIdx.x] = mine->b[threadIdx.x];
    }
    xk = 1;
    __syncthreads();
  }
  constexpr int kRPL = kMaxN / 2 / 32;  // local rows per lane (ml <= 128)
  for (int q = 0; q < w; ++q) {
    double* x = P + static_cast<size_t>(q) * ml;
    if (wp == 0) {
      // pivot: largest alpha^2 + sigma among positions q .. w - 1 (compared
      // in FP32: the keys only choose the order)
      const int s = q + lane;
      float kv = (s < w) ? static_cast<float>(fma(alp[s], alp[s], sig[s])) : -1.0f;
      int ks = (s < w) ? s : w;
      for (int o = 16; o > 0; o >>= 1) {
        const float kv2 = __shfl_xor_sync(0xFFFFFFFFu, kv, o);
        const int ks2 = __shfl_xor_sync(0xFFFFFFFFu, ks, o);
        if (kv2 > kv || (kv2 == kv && ks2 < ks)) {
          kv = kv2;
          ks = ks2;
        }
      }
      const int piv = (ks < w) ? ks : q;
      if (piv != q) {
        double* y = P + static_cast<size_t>(piv) * ml;
        for (int rl = lane; rl < ml; rl += 32) {
          const double t = x[rl];
          x[rl] = y[rl];
          y[rl] = t;
        }
        if (lane == 0) {
          double t = sig[q];
          sig[q] = sig[piv];
          sig[piv] = t;
          t = alp[q];
          alp[q] = alp[piv];
          alp[piv] = t;
          const int ti = lp[q];
          lp[q] = lp[piv];
          lp[piv] = ti;
        }
      }
      __syncwarp();
      if (lane == 0) {  // reflector scalars, the same on both CTAs
        const double alpha = alp[q], sg = sig[q];
        double tau = 0.0, beta = alpha, scal = 1.0;
        if (sg != 0.0) {
          const double nr = sqrt(fma(alpha, alpha, sg));
          beta = (alpha <= 0.0) ? nr : -nr;
          // tau = (beta - alpha) / beta and scal = 1 / (alpha - beta) from
          // one reciprocal
          const double am = alpha - beta, rb = 1.0 / (beta * am);
          tau = -(am * am) * rb;
          scal = beta * rb;
        }
        taus[q] = tau;
        betas[q] = beta;
        scal_sh = scal;
      }
    }
    __syncthreads();
    const double tau = taus[q], scal = scal_sh;
    for (int rl = threadIdx.x; rl < ml; rl += blockDim.x)
      if (r0 + rl > q) x[rl] *= scal;
    __syncthreads();
    // columns s0 .. s0 + 3 per warp (one group: 4 x 16 warps > kNB)
    const int s0 = q + 1 + 4 * wp;
    const bool has = s0 < w;
    double xv[4][kRPL], vr[kRPL];
    {
      QbXch* mine = &xch[xk & 1];
      QbXch* theirs = cl.map_shared_rank(mine, peer);
      if (has) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int t = 0; t < kRPL; ++t) {
          const int rl = lane + 32 * t, r = r0 + rl;
          vr[t] = (rl < ml && r >= q) ? ((r == q) ? 1.0 : x[rl]) : 0.0;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            xv[u][t] = (s0 + u < w && rl < ml) ? P[static_cast<size_t>(s0 + u) * ml + rl] : 0.0;
            acc[u] = fma(vr[t], xv[u][t], acc[u]);
          }
        }
        qb_wsum4(acc);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (s0 + u < w) {
              mine->a[rank][s0 + u] = acc[u];
              theirs->a[rank][s0 + u] = acc[u];
            }
      }
      cl.sync();
      ++xk;
      QbXch* mine2 = &xch[xk & 1];
      QbXch* theirs2 = cl.map_shared_rank(mine2, peer);
      if (has) {
        // apply H_q; sums of squares of rows q + 2 .., row q + 1 read off
        double sq[4] = {0.0, 0.0, 0.0, 0.0}, nx[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int su = (s0 + u < w) ? s0 + u : s0;
          const double dt = tau * (mine->a[0][su] + mine->a[1][su]);
#pragma unroll
          for (int t = 0; t < kRPL; ++t) {
            const int rl = lane + 32 * t, r = r0 + rl;
            if (s0 + u < w && rl < ml) {
              if (r >= q) {
                xv[u][t] = fma(-dt, vr[t], xv[u][t]);
                P[static_cast<size_t>(s0 + u) * ml + rl] = xv[u][t];
              }
              if (r > q + 1) sq[u] = fma(xv[u][t], xv[u][t], sq[u]);
              if (r == q + 1) nx[u] = xv[u][t];
            }
          }
        }
        qb_wsum4(sq);
        // row q + 1 < w is on CTA 0, lane q + 1 (t = 0): broadcast it
#pragma unroll
        for (int u = 0; u < 4; ++u) nx[u] = __shfl_sync(0xFFFFFFFFu, nx[u], (q + 1) & 31);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (s0 + u < w) {
              mine2->a[rank][s0 + u] = sq[u];
              theirs2->a[rank][s0 + u] = sq[u];
              if (rank == 0) {
                mine2->b[s0 + u] = nx[u];
                theirs2->b[s0 + u] = nx[u];
              }
            }
      }
      cl.sync();
      ++xk;
      if (threadIdx.x > q && threadIdx.x < w) {
        sig[threadIdx.x] = mine2->a[0][threadIdx.x] + mine2->a[1][threadIdx.x];
        alp[threadIdx.x] = mine2->b[threadIdx.x];
      }
      __syncthreads();
    }
  }
  // 3. Gram matrix of the reflectors (partials of both CTAs) and T
  auto vv = [&](int s2, int rl) -> double {  // v_s2 at this CTA's row r0 + rl
    const int r = r0 + rl;
    return (r < s2) ? 0.0 : (r == s2 ? 1.0 : P[static_cast<size_t>(s2) * ml + rl]);
  };
  {
    double(*gpeer)[kNB + 1] = cl.map_shared_rank(Gp[rank], peer);
    // four pairs (s0 .. s0 + 3, q) per warp task, one butterfly for the four
    // sums; only the tasks with s0 < q are enumerated (q = 1 .. w - 1 has
    // ceil(q / 4) of them), so that the warps share them evenly
    int ntask = 0;
    for (int q = 1; q < w; ++q) ntask += (q + 3) / 4;
    for (int task = wp; task < ntask; task += nw) {
      int q = 1, rest = task;
      while (rest >= (q + 3) / 4) {
        rest -= (q + 3) / 4;
        ++q;
      }
      const int s0 = 4 * rest;
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (int rl = lane; rl < ml; rl += 32) {
        const double vq = vv(q, rl);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (s0 + u < q) acc[u] = fma(vv(s0 + u, rl), vq, acc[u]);
      }
      qb_wsum4(acc);
      if (lane == 0)
        for (int u = 0; u < 4 && s0 + u < q; ++u) {
          Gp[rank][s0 + u][q] = acc[u];
          gpeer[s0 + u][q] = acc[u];
        }
    }
  }
  cl.sync();  // no shared memory of the peer is touched after this point
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {  // Gp[0] <- V^T V (s < q)
    const int s2 = e / w, q2 = e - s2 * w;
    if (s2 < q2) Gp[0][s2][q2] += Gp[1][s2][q2];
  }
  __syncthreads();
  if (wp == 0) {  // lanes over the rows i < q; four partial sums shorten the chain
    auto gm = [&](int s2, int q2) -> double { return Gp[0][s2][q2]; };
    for (int q = 0; q < w; ++q) {
      const double tq = taus[q];
      double ti = 0.0;
      if (lane < q) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        for (int j = lane; j < q; j += 4) {
          a0 = fma(T[lane][j], gm(j, q), a0);
          if (j + 1 < q) a1 = fma(T[lane][j + 1], gm(j + 1, q), a1);
          if (j + 2 < q) a2 = fma(T[lane][j + 2], gm(j + 2, q), a2);
          if (j + 3 < q) a3 = fma(T[lane][j + 3], gm(j + 3, q), a3);
        }
        ti = -tq * ((a0 + a1) + (a2 + a3));
      }
      __syncwarp();
      if (lane < q) T[lane][q] = ti;
      if (lane == 0) T[q][q] = tq;
      for (int i = q + 1 + lane; i < w; i += 32) T[i][q] = 0.0;
      __syncwarp();
    }
  }
  __syncthreads();
  // 4. outputs (this CTA's rows)
  for (int e = threadIdx.x; e < w * ml; e += blockDim.x) {
    const int q = e / ml, rl = e - q * ml, r = r0 + rl;
    double y = 0.0;
    for (int s2 = 0; s2 <= q; ++s2) y = fma(T[s2][q], vv(s2, rl), y);
    Yt[static_cast<size_t>(c0 + q) * n + c0 + r] = y;
    Vt[static_cast<size_t>(c0 + q) * n + c0 + r] = vv(q, rl);
    Wd[static_cast<size_t>(c0 + q) * n + c0 + r] = (r == q) ? betas[q] : P[e];
  }
  for (int e = threadIdx.x + rank * blockDim.x; e < w * c0; e += 2 * blockDim.x) {
    const int q = e / c0, r = e - q * c0;  // entries above the panel
    Wd[static_cast<size_t>(c0 + q) * n + r] = Ws[static_cast<size_t>(c0 + src_of[lp[q]]) * n + r];
  }
  if (rank == 0 && threadIdx.x < w) {
    const int q = threadIdx.x;
    perm[c0 + q] = pold[src_of[lp[q]]];
    double d = absd(betas[q]);
    if (!(d > 0.0) || !isfinite(d)) {
      atomicExch(status, d > 0.0 ? kDevNonFinite : kDevSingular);
      if (!(d > 0.0)) d = DBL_MIN;
    }
    D[c0 + q] = d;
  }
}

// Rtil[i][perm[c']] = R[i][c'] / D[i]: R[i][c'] = W[c'][i] for c' >= i (the
// diagonal holding beta_i), 0 below the diagonal, with W the buffer the panel
// of c' wrote (WA for even panels, WB for odd ones).
__global__ void __launch_bounds__(256) k_qrb_finalize(const double* WAall, const double* WBall,
                                                     long long sW, const int* permall,
                                                     const double* Dall, long long sD,
                                                     double* Rall, long long sR, int n) {
  const int b = blockIdx.y;
  const double* WA = WAall + b * sW;
  const double* WB = WBall + b * sW;
  const int* perm = permall + static_cast<long long>(b) * n;
  const double* D = Dall + b * sD;
  double* Rt = Rall + b * sR;
  __shared__ double tile[32][33];
  const int tiles = (n + 31) / 32;
  const int ti = blockIdx.x / tiles, tc = blockIdx.x - ti * tiles;  // rows i, columns c'
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;           // 32 x 8
  for (int k = ty; k < 32; k += 8) {  // read W[c'][i], i fastest
    const int cp = tc * 32 + k, i = ti * 32 + tx;
    const double* W = ((cp / kNB) & 1) ? WB : WA;
    tile[k][tx] = (cp < n && i < n) ? W[static_cast<size_t>(cp) * n + i] : 0.0;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int i = ti * 32 + k, cp = tc * 32 + tx;
    if (i < n && cp < n) {
      const double v = (cp >= i) ? tile[tx][k] / D[i] : 0.0;
      Rt[static_cast<size_t>(i) * n + perm[cp]] = v;
    }
  }
}

// One tensor-core product of the blocked QR (no scales).
OzProduct qb_prod(int M, int Nc, int K, const double* A, long long sA, long long a_sv,
                  long long a_sk, const double* B, long long sB, long long b_sv, long long b_sk,
                  double* C, long long sC, int ldc, double alpha, double beta) {
  OzProduct p{};
  p.M = M; p.Nc = Nc; p.K = K;
  p.A = A; p.sA = sA; p.a_sv = a_sv; p.a_sk = a_sk;
  p.B = B; p.sB = sB; p.b_sv = b_sv; p.b_sk = b_sk;
  p.C = C; p.sC = sC; p.ldc = ldc;
  p.alpha = alpha; p.beta = beta;
  return p;
}

}  // namespace

int qr_blocked_launches(int n, int batch, int oz_batch) {
  const int panels = (n + kNB - 1) / kNB;
  const int chunks = (batch + oz_batch - 1) / oz_batch;
  // identity and finalize; one panel kernel per panel; two products (one
  // kernel per chunk of the batch) per panel except the last, which has no
  // trailing columns, and two per panel of the Q accumulation
  return 2 + panels + (4 * panels - 2) * chunks;
}

size_t qr_blocked_smem(int n) { return static_cast<size_t>(kNB) * qb_split(n, kNB) * sizeof(double); }

cudaError_t launch_qr_blocked(double* Xt, long long sX, double* Qt, long long sQ, double* D,
                              long long sD, double* Rtil, long long sR, const QrbWork& wk, int n,
                              int batch, void* oz, int oz_batch, int* status, cudaStream_t st) {
  if (n <= 0 || batch <= 0 || n > kMaxN) return n > kMaxN ? cudaErrorInvalidValue : cudaSuccess;
  double* WA = wk.W0;
  double* WB = wk.W1;
  const long long sW = wk.sW;
  double* Vt = Rtil;  // Householder vectors, row c0 + q = v_q
  double* Yt = Xt;    // Y = T^T V^T of every panel
  double* Wt = wk.Wt;
  const long long sWt = wk.sWt;
  const int smem = static_cast<int>(qr_blocked_smem(n));
  cudaError_t e = cudaFuncSetAttribute(k_qrb_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  for (int c0 = 0, p = 0; c0 < n; c0 += kNB, ++p) {
    const int w = std::min(kNB, n - c0), m = n - c0, nt = n - c0 - w;
    const double* src = (p == 0) ? Xt : ((p & 1) ? WA : WB);
    const long long sSrc = (p == 0) ? sX : sW;
    double* dst = (p & 1) ? WB : WA;
    {  // one cluster of two CTAs per matrix
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(2 * batch, 1, 1);
      cfg.blockDim = dim3(kPT, 1, 1);
      cfg.dynamicSmemBytes = static_cast<size_t>(w) * qb_split(m, w) * sizeof(double);
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k_qrb_panel, src, sSrc, dst, sW, wk.perm, Vt, sR, Yt, sX, D, sD,
                             n, c0, w, status);
    }
    if (e != cudaSuccess) return e;
    if (nt == 0) continue;
    const long long off_trail = static_cast<long long>(c0 + w) * n + c0;
    const long long off_p = static_cast<long long>(c0) * n + c0;
    // W^T = A_rows Y^T: A_rows = trailing rows of dst from column c0
    OzProduct p1 = qb_prod(nt, w, m, dst + off_trail, sW, n, 1, Yt + off_p, sX, n, 1, Wt, sWt, w,
                           1.0, 0.0);
    e = launch_ozaki_product(p1, batch, oz, oz_batch, status, st);
    if (e != cudaSuccess) return e;
    // A_rows -= W^T V^T
    OzProduct p2 = qb_prod(nt, m, w, Wt, sWt, w, 1, Vt + off_p, sR, 1, n, dst + off_trail, sW, n,
                           -1.0, 1.0);
    e = launch_ozaki_product(p2, batch, oz, oz_batch, status, st);
    if (e != cudaSuccess) return e;
  }
  e = launch_set_identity(Qt, sQ, nullptr, 0, n, batch, st);
  if (e != cudaSuccess) return e;
  const int last = ((n - 1) / kNB) * kNB;
  for (int c0 = last; c0 >= 0; c0 -= kNB) {
    const int w = std::min(kNB, n - c0), m = n - c0;
    const long long off_p = static_cast<long long>(c0) * n + c0;
    // W^T = Qt_rows V (rows c0.. of Q^T, columns c0..)
    OzProduct p3 = qb_prod(m, w, m, Qt + off_p, sQ, n, 1, Vt + off_p, sR, n, 1, Wt, sWt, w, 1.0,
                           0.0);
    e = launch_ozaki_product(p3, batch, oz, oz_batch, status, st);
    if (e != cudaSuccess) return e;
    // Qt_rows -= W^T Y
    OzProduct p4 = qb_prod(m, m, w, Wt, sWt, w, 1, Yt + off_p, sX, 1, n, Qt + off_p, sQ, n, -1.0,
                           1.0);
    e = launch_ozaki_product(p4, batch, oz, oz_batch, status, st);
    if (e != cudaSuccess) return e;
  }
  const int tiles = (n + 31) / 32;
  k_qrb_finalize<<<dim3(tiles * tiles, batch), 256, 0, st>>>(WA, WB, sW, wk.perm, D, sD, Rtil, sR,
                                                             n);
  return cudaGetLastError();
}

}  // namespace dqmc
