// Sweep kernels of libdqmc: HS-field initialisation, the Metropolis pass of
// one time slice with delayed rank-k Sherman-Morrison updates, Kronecker
// multiplication by B_l = exp(-dtau K) exp(V_l) (slice wrap and UDV stack
// products), drift check and equal-time observables.
//
// Paper: Rost & Bluemer, arXiv:1504.05090, Sec. 2, Eqs. (1)-(3).  The
// Metropolis ratio and the Sherman-Morrison update follow from Eq. (3) for a
// single flip s -> -s of the Ising field (e^{V'} = e^{V}(I + Delta e_i e_i^T)):
//   R_sigma = 1 + Delta_sigma (1 - G_ii),  Delta_sigma = e^{-2 sigma lambda s} - 1,
//   G' = G - (Delta/R) (I - G) e_i e_i^T G.
// Only spin up is evolved: on the bipartite half-filled lattice
// G_dn = I - P G_up^T P (P = diag((-1)^{x+y})), so G_dn,ii = 1 - G_up,ii.
#include <cooperative_groups.h>

#include <math_constants.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace dqmc {
namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
// Initial Ising field: s = +1 iff word 0 of Philox(i + N*l, ~0, chain, 1) is odd.
// ---------------------------------------------------------------------------
__global__ void k_init_field(int8_t* field, int C, int L, int N, int chain0, uint32_t k0,
                             uint32_t k1) {
  const long long total = static_cast<long long>(C) * L * N;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e / (static_cast<long long>(L) * N));
    const int rem = static_cast<int>(e - static_cast<long long>(c) * L * N);  // l*N + i
    const uint4 r = philox4x32_10(make_uint4(static_cast<uint32_t>(rem), 0xFFFFFFFFu,
                                             static_cast<uint32_t>(chain0 + c), kTagInitField),
                                  k0, k1);
    field[e] = (r.x & 1u) ? int8_t(1) : int8_t(-1);
  }
}

// ---------------------------------------------------------------------------
// Metropolis pass over the N sites of one slice, one CTA per chain, one
// thread per row/column index j.  G (row-major, working precision) stays in
// global memory (L2-resident); accepted flips are buffered as column vectors
// U[m] and row vectors V[m] in shared memory, G_cur = G + sum_m U[m] V[m]^T,
// and folded into G every k accepts (delayed rank-k update).  The diagonal of
// G_cur is tracked in shared memory so that a rejected proposal costs O(1).
// The accept/reject decision is taken in FP64 by lane 0 of every warp and
// broadcast with a shuffle, so all threads agree without a barrier.
// ---------------------------------------------------------------------------
// Working-precision helpers.
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(double x) { return static_cast<float>(x); }
__device__ __forceinline__ float to_f32(df32 x) { return x.hi + x.lo; }
__device__ __forceinline__ float shfl0(float x) { return __shfl_sync(0xFFFFFFFFu, x, 0); }
__device__ __forceinline__ double shfl0(double x) { return __shfl_sync(0xFFFFFFFFu, x, 0); }
__device__ __forceinline__ df32 shfl0(df32 x) { return df32(shfl0(x.hi), shfl0(x.lo)); }

// Sherman-Morrison coefficient -Delta_up / R_up in the working precision:
// FP32 for float, FP64 for double, and a float reciprocal refined by one
// Newton step in df32 arithmetic for df32 (no FP64 instruction).
__device__ __forceinline__ float sm_coef(const MetroArgs& a, int s, float g) {
  const float du = s > 0 ? a.em2h : a.ep2h;
  return -du / fmaf(du, 1.0f - g, 1.0f);
}
__device__ __forceinline__ double sm_coef(const MetroArgs& a, int s, double g) {
  const double du = s > 0 ? a.em2 : a.ep2;
  return -du / fma(du, 1.0 - g, 1.0);
}
__device__ __forceinline__ df32 sm_coef(const MetroArgs& a, int s, df32 g) {
  const df32 du = s > 0 ? df32(a.em2h, a.em2l) : df32(a.ep2h, a.ep2l);
  const df32 one(1.0f, 0.0f);
  const df32 ru = one + du * (one - g);
  const df32 y0(1.0f / ru.hi, 0.0f);
  const df32 y = y0 + y0 * (one - ru * y0);
  return -(du * y);
}

// Column j of G, rows ra .. rb-1: G += U V^T over the cnt pending updates.
// MC = kMaxDelay keeps all of column j of V in registers for the whole flush;
// a smaller MC reloads it in chunks of MC per row batch (fewer registers, the
// same additions in the same order).
template <typename T, int RB = 8, int MC = kMaxDelay>
__device__ __forceinline__ void delayed_flush(T* G, const T* U, const T* V, int cnt, int N, int NP,
                                              int j, int ra, int rb) {
  if (j >= N) return;
  T v[MC];
  if constexpr (MC == kMaxDelay) {
#pragma unroll
    for (int m = 0; m < kMaxDelay; ++m) v[m] = (m < cnt) ? V[m * NP + j] : T(0);
  }
  // Rows in batches of RB, the next batch loaded while the current one is
  // computed, so two batches of L2 loads are in flight per thread.
  T cur[RB], nxt[RB];
#pragma unroll
  for (int q = 0; q < RB; ++q) cur[q] = (ra + q < rb) ? G[static_cast<size_t>(ra + q) * N + j] : T(0);
  for (int r0 = ra; r0 < rb; r0 += RB) {
    const int r1 = r0 + RB;
#pragma unroll
    for (int q = 0; q < RB; ++q)
      nxt[q] = (r1 + q < rb) ? G[static_cast<size_t>(r1 + q) * N + j] : T(0);
    ProdSum<T> acc[RB];
    for (int m0 = 0; m0 < cnt; m0 += MC) {
      if constexpr (MC != kMaxDelay) {
#pragma unroll
        for (int mm = 0; mm < MC; ++mm) v[mm] = (m0 + mm < cnt) ? V[(m0 + mm) * NP + j] : T(0);
      }
      if constexpr (std::is_same<T, df32>::value && RB % 2 == 0) {
        // two rows of U per 16-byte load when the row pair is 16-byte aligned
        // (r0 even: U rows of NP entries start 16-byte aligned); the sums of
        // each row see the same additions in the same order either way
        if ((r0 & 1) == 0) {
#pragma unroll
          for (int q = 0; q < RB; q += 2) {
#pragma unroll
            for (int mm = 0; mm < MC; ++mm)
              if (m0 + mm < cnt) {
                const float4 u2 = *reinterpret_cast<const float4*>(U + (m0 + mm) * NP + r0 + q);
                acc[q].add(df32(u2.x, u2.y), v[mm]);
                acc[q + 1].add(df32(u2.z, u2.w), v[mm]);
              }
          }
          continue;
        }
      }
#pragma unroll
      for (int q = 0; q < RB; ++q) {
#pragma unroll
        for (int mm = 0; mm < MC; ++mm)
          if (m0 + mm < cnt) acc[q].add(U[(m0 + mm) * NP + r0 + q], v[mm]);
      }
    }
#pragma unroll
    for (int q = 0; q < RB; ++q)
      if (r0 + q < rb) G[static_cast<size_t>(r0 + q) * N + j] = cur[q] + acc[q].get();
#pragma unroll
    for (int q = 0; q < RB; ++q) cur[q] = nxt[q];
  }
}

// Barrier between the cs CTAs of one chain's cluster around the flushes of G
// (global memory).  Thread 0 arrives on every peer's mbarrier (release at
// cluster scope) and waits for its own for at most 0.2 s; a wait that gives up
// sets kDevTimeout and lets the CTA go on, so the kernel always ends.  The __threadfence pair makes the CTA's global writes visible before
// the arrival and the peers' writes after the wait.  Barrier phases alternate
// between two mbarriers: a peer can be at most one phase ahead (it cannot pass
// phase f + 1 before this CTA arrived for it), so an arrival for phase f + 1
// never lands on the mbarrier that still collects phase f.
constexpr unsigned long long kPeerWaitNs = 200000000ull;  // 0.2 s of %globaltimer
constexpr long long kPeerWaitPolls = 1LL << 24;             // and at most this many polls

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// `broken` (shared) is set once a wait gave up; later barriers of the launch
// then only synchronise the CTA.
__device__ __forceinline__ void peer_barrier(uint64_t* bars, int cs, int rank, int& phase,
                                             int* status, int* broken) {
  __syncthreads();
  if (threadIdx.x == 0 && !*broken) {
    __threadfence();
    const uint32_t local = static_cast<uint32_t>(__cvta_generic_to_shared(bars + (phase & 1)));
    for (int r = 0; r < cs; ++r) {
      if (r == rank) continue;
      uint32_t remote;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(r));
      asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote)
                   : "memory");
    }
    uint32_t done = 0;
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < kPeerWaitPolls && !done; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(done)
          : "r"(local), "r"((phase >> 1) & 1)
          : "memory");
      if (!done && (it & 255) == 255 && global_ns() - t0 > kPeerWaitNs) break;
    }
    if (!done) {
      atomicExch(status, kDevTimeout);
      *broken = 1;
    }
    __threadfence();
  }
  ++phase;
  __syncthreads();
}

// Threads per column of G: two for float pairs (one computes the column and
// one the row correction of an accepted flip, and they split the rows of the
// flush), one otherwise.
// Columns of G staged in shared memory per window of sites (k_metropolis).
constexpr int kWin = 32;

// Pending updates per register chunk of the flush: all of them for one
// thread per column; eight for float pairs, whose two threads per column
// each fold eight rows at a time (more independent sums in flight at the
// 128-register limit of 512 threads).
template <typename T>
constexpr int kFlushMC() {
  return std::is_same<T, df32>::value ? 8 : kMaxDelay;
}

template <typename T>
constexpr int metro_halves() {
  return std::is_same<T, df32>::value ? 2 : 1;
}

// Thread-block cluster of cs CTAs per chain (cs = 1: one CTA).  Every CTA
// takes the same site decisions and builds the same U, V from the same data
// (identical instruction streams, so identical results); in a flush each CTA
// adds U V^T to its own block of N / cs rows of G.  Two peer barriers bracket
// every flush: no CTA overwrites rows that a peer may still read for the
// sites before the flush, and every CTA reads the new rows after it.
template <typename T>
__global__ void __launch_bounds__(256 * metro_halves<T>()) k_metropolis(T* Gall, int8_t* fieldall,
                                                                      MetroArgs a) {
  constexpr int kH = metro_halves<T>();
  const int cs = a.cs;
  const int c = blockIdx.x / cs;
  const int rank = blockIdx.x - c * cs;  // cluster rank (the cluster spans blockIdx.x)
  const int N = a.N;
  const int NP = blockDim.x / kH;                // columns (N rounded up to a warp)
  const int h = (kH == 2 && static_cast<int>(threadIdx.x) >= NP) ? 1 : 0;
  // rows of G this thread folds the delayed updates into: the CTA's block of
  // N / cs rows, split between the two halves when kH = 2
  const int ra0 = (rank * N) / cs, rb0 = ((rank + 1) * N) / cs, rmid = ra0 + (rb0 - ra0 + 1) / 2;
  const int ra = (kH == 2 && h) ? rmid : ra0, rb = (kH == 2 && !h) ? rmid : rb0;
  __shared__ uint64_t xbar[2];
  __shared__ int xbroken;
  int xphase = 0;
  if (cs > 1) {
    if (threadIdx.x == 0) {
      // a peer wait of an earlier launch gave up: results are void already,
      // so this launch does not wait again
      xbroken = (*reinterpret_cast<volatile int*>(a.status) == kDevTimeout);
      for (int b = 0; b < 2; ++b)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                         static_cast<uint32_t>(__cvta_generic_to_shared(xbar + b))),
                     "r"(cs - 1));
      asm volatile("fence.mbarrier_init.release.cluster;");
    }
    cooperative_groups::this_cluster().sync();
  }
  const int j = threadIdx.x - h * NP;  // column of this thread
  const int lane = threadIdx.x & 31;
  const bool act = j < N;
  T* G = Gall + static_cast<size_t>(c) * N * N;
  int8_t* s_l = fieldall + (static_cast<size_t>(c) * a.L + a.l0) * N;

  extern __shared__ __align__(16) unsigned char sm_raw[];
  double* uu = reinterpret_cast<double*>(sm_raw);  // [NP] proposal uniforms
  float* uuf = reinterpret_cast<float*>(uu + NP);   // [NP] the same, rounded to float
  T* U = reinterpret_cast<T*>(uuf + NP);            // [k][NP]
  T* V = U + a.k * NP;                              // [k][NP]
  T* d = V + a.k * NP;                              // [NP] diag of G_cur
  float* df = reinterpret_cast<float*>(d + NP);     // [NP] diag of G_cur, rounded to float
  int* ss = reinterpret_cast<int*>(df + NP);        // [NP] field of the slice
  T* cw = reinterpret_cast<T*>(ss + NP);            // [kWin][NP + 1] window of columns of G

  const uint32_t sweep = *a.sweep_ctr;
  if (act && h == 0) {
    const T gjj = G[static_cast<size_t>(j) * N + j];
    d[j] = gjj;
    df[j] = to_f32(gjj);
    ss[j] = s_l[j];
    const uint4 r = philox4x32_10(make_uint4(static_cast<uint32_t>(j + N * a.l0), sweep,
                                             static_cast<uint32_t>(a.chain0 + c), kTagProposal),
                                  a.key0, a.key1);
    const double u = uniform53(r.x, r.y);
    uu[j] = u;
    uuf[j] = static_cast<float>(u);
  }
  __syncthreads();

  // Columns wb .. wb + kWin - 1 of G in shared memory, cw[c][j] = G[j][wb + c]:
  // loaded with whole-row segments (a column of the row-major G would take one
  // memory transaction per row), reloaded every kWin sites and after a flush.
  const int ldw = NP + 1;  // odd stride in 8-byte words: conflict-free transposed stores
  auto load_window = [&](int wb) {
    constexpr int kU = 8;
    const int tot = N * kWin;
    for (int e0 = threadIdx.x; e0 < tot; e0 += kU * blockDim.x) {
      T t[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x, r = e / kWin, c = e - r * kWin;
        t[u] = (e < tot && wb + c < N) ? G[static_cast<size_t>(r) * N + wb + c] : T(0);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int e = e0 + u * blockDim.x, r = e / kWin, c = e - r * kWin;
        if (e < tot) cw[c * ldw + r] = t[u];
      }
    }
  };
  int wb = 0;
  load_window(0);
  __syncthreads();
  // Row i of G for the next kPre sites, loaded ahead into registers (rows
  // are contiguous; a flush rewrites G, after which the window is reloaded).
  // With two threads per column only the row half uses it.
  constexpr int kPre = 4;
  T pr[kPre];
  auto ld_r = [&](int q) -> T {
    return (act && q < N && (kH == 1 || h == 1)) ? G[static_cast<size_t>(q) * N + j] : T(0);
  };
#pragma unroll
  for (int q = 0; q < kPre; ++q) pr[q] = ld_r(q);
  int cnt = 0;
  unsigned naccept = 0;
  // The field is written back after the slice: a peer CTA of the cluster may
  // still be reading the slice's initial field when this one accepts a flip.
  bool flip = false;
  for (int i = 0; i < N; ++i) {
    if (i == wb + kWin) {  // every warp is past site i - 1
      __syncthreads();
      wb = i;
      load_window(wb);
      __syncthreads();
    }
    // kH == 2: colv is G[j][i] for h = 0 and rowv G[i][j] for h = 1
    const T colv = act ? cw[(i - wb) * ldw + j] : T(0);
    const T rowv = pr[0];
#pragma unroll
    for (int q = 0; q + 1 < kPre; ++q) pr[q] = pr[q + 1];
    pr[kPre - 1] = ld_r(i + kPre);
    // Decision u < R_up R_dn with R_up = 1 + D_up (1 - G_ii), R_dn = 1 + D_dn G_ii
    // (G_dn,ii = 1 - G_up,ii).  Lane 0 of every warp takes it in FP32 unless u
    // lies within 1e-4 of R, where it is retaken in FP64; all warps agree
    // without a barrier.
    int acc_i = 0;
    T coef = T(0);
    if (lane == 0) {
      const int s = ss[i];
      const float gf = df[i];
      const float duf = s > 0 ? a.em2h : a.ep2h, ddf = s > 0 ? a.ep2h : a.em2h;
      const float Rf = fmaf(duf, 1.0f - gf, 1.0f) * fmaf(ddf, gf, 1.0f);
      const float uf = uuf[i];
      if (uf < Rf * 0.9999f) {
        acc_i = 1;
      } else if (!(uf > Rf * 1.0001f)) {
        const double g = static_cast<double>(d[i]);
        const double du = s > 0 ? a.em2 : a.ep2, dd = s > 0 ? a.ep2 : a.em2;
        acc_i = uu[i] < fma(du, 1.0 - g, 1.0) * fma(dd, g, 1.0);
      }
      if (acc_i) coef = sm_coef(a, s, d[i]);
    }
    acc_i = __shfl_sync(0xFFFFFFFFu, acc_i, 0);
    if (acc_i) {
      coef = shfl0(coef);
      ++naccept;
      if constexpr (kH == 1) {
        if (act) {
          ProdSum<T> sc, sr;
          for (int m = 0; m < cnt; ++m) {
            sc.add(U[m * NP + j], V[m * NP + i]);
            sr.add(U[m * NP + i], V[m * NP + j]);
          }
          const T gc = colv + sc.get(), gr = rowv + sr.get();
          const T uj = coef * ((j == i ? T(1) : T(0)) - gc);
          U[cnt * NP + j] = uj;
          V[cnt * NP + j] = gr;
          // Only the diagonal of sites still to come (j > i) is updated.  Warps
          // pass rejected sites without a barrier, so a slower warp may still be
          // deciding an earlier site j <= i: its d[j], df[j] (dead for the rest
          // of the slice) must keep the value every other warp decided with.
          if (j > i) {
            const T dj = d[j] + uj * gr;
            d[j] = dj;
            df[j] = to_f32(dj);
          } else if (j == i) {
            flip = true;
          }
        }
      } else {
        // column correction (h = 0) and row correction (h = 1) of the flip
        if (act) {
          ProdSum<T> sa;
          if (h == 0) {
            for (int m = 0; m < cnt; ++m) sa.add(U[m * NP + j], V[m * NP + i]);
            const T gc = colv + sa.get();
            U[cnt * NP + j] = coef * ((j == i ? T(1) : T(0)) - gc);
          } else {
            for (int m = 0; m < cnt; ++m) sa.add(U[m * NP + i], V[m * NP + j]);
            V[cnt * NP + j] = rowv + sa.get();
          }
        }
        __syncthreads();
        // every warp is at site i here, so the diagonal of the sites to come
        // is updated before anyone decides the next site (barrier below)
        if (act && h == 0) {
          if (j > i) {
            const T dj = d[j] + U[cnt * NP + j] * V[cnt * NP + j];
            d[j] = dj;
            df[j] = to_f32(dj);
          } else if (j == i) {
            flip = true;
          }
        }
      }
      __syncthreads();
      ++cnt;
      if (cnt == a.k) {
        if (cs > 1) peer_barrier(xbar, cs, rank, xphase, a.status, &xbroken);
        delayed_flush<T, 8, kFlushMC<T>()>(G, U, V, cnt, N, NP, j, ra, rb);
        cnt = 0;
        if (cs > 1)
          peer_barrier(xbar, cs, rank, xphase, a.status, &xbroken);
        else
          __syncthreads();
        wb = i + 1;
        load_window(wb);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kPre; ++q) pr[q] = ld_r(i + 1 + q);
      }
    }
  }
  if (cnt > 0) {
    if (cs > 1) peer_barrier(xbar, cs, rank, xphase, a.status, &xbroken);
    delayed_flush<T, 8, kFlushMC<T>()>(G, U, V, cnt, N, NP, j, ra, rb);
  }
  // No CTA leaves while a peer may still arrive on its barrier or read the
  // slice's field.
  if (cs > 1) cooperative_groups::this_cluster().sync();
  if (rank == 0) {
    if (flip) s_l[j] = static_cast<int8_t>(-ss[j]);
    if (threadIdx.x == 0) a.accepted[c] += naccept;
  }
}

// ---------------------------------------------------------------------------
// Kronecker transform of nv vectors held in shared memory (row stride ld):
// v <- Ey (x) Ex applied to (pre o v), then multiplied by post.
// ---------------------------------------------------------------------------
// Two taps read with one load (16 bytes for 8-byte types).
template <typename T>
struct alignas(2 * sizeof(T)) KronPair {
  T a, b;
};

template <typename T>
__device__ __forceinline__ void kron_transform(T* v, T* tmp, int nv, int ld, int Lx, int Ly, int N,
                                               const T* tx, const T* ty, const T* txs,
                                               const T* tys, const T* pre, const T* post) {
  const int tot = nv * N;
  if (pre) {  // diagonal factor applied once per element, not once per tap
    for (int e = threadIdx.x; e < tot; e += blockDim.x) {
      const int vi = e / N, i = e - vi * N;
      v[vi * ld + i] *= pre[i];
    }
    __syncthreads();
  }
  if ((Lx & 1) == 0 && (Ly & 1) == 0) {
    // Even sides: a thread takes two neighbouring outputs (x, x + 1) of one
    // row (then (y, y + 1) of one column).  Both sums read the same input
    // entry (one load), and their taps E[x - x'], E[x + 1 - x'] are adjacent:
    // one 16-byte load from tx (tap index even) or from txs, the same taps
    // shifted by one (odd).  Same additions in the same order per output.
    const int hx = Lx >> 1, hy = Ly >> 1;
    const int ptx = nv * Ly * hx;
    for (int e = threadIdx.x; e < ptx; e += blockDim.x) {
      const int vi = e / (Ly * hx), rr = e - vi * (Ly * hx), y = rr / hx, x = 2 * (rr - y * hx);
      const T* row = v + vi * ld + Lx * y;
      ProdSum<T> a0, a1;
      for (int xp = 0; xp < Lx; ++xp) {
        const int b = x + Lx - xp;  // tap index of output x; b + 1 that of x + 1
        const KronPair<T> t2 = (b & 1) ? *reinterpret_cast<const KronPair<T>*>(txs + b - 1)
                                       : *reinterpret_cast<const KronPair<T>*>(tx + b);
        const T r = row[xp];
        a0.add(t2.a, r);
        a1.add(t2.b, r);
      }
      tmp[vi * ld + Lx * y + x] = a0.get();
      tmp[vi * ld + Lx * y + x + 1] = a1.get();
    }
    __syncthreads();
    const int pty = nv * hy * Lx;
    for (int e = threadIdx.x; e < pty; e += blockDim.x) {
      const int vi = e / (hy * Lx), rr = e - vi * (hy * Lx), yp2 = rr / Lx, x = rr - yp2 * Lx;
      const int y = 2 * yp2;
      const T* col = tmp + vi * ld + x;
      ProdSum<T> a0, a1;
      for (int yp = 0; yp < Ly; ++yp) {
        const int b = y + Ly - yp;
        const KronPair<T> t2 = (b & 1) ? *reinterpret_cast<const KronPair<T>*>(tys + b - 1)
                                       : *reinterpret_cast<const KronPair<T>*>(ty + b);
        const T c = col[Lx * yp];
        a0.add(t2.a, c);
        a1.add(t2.b, c);
      }
      const int i0 = x + Lx * y, i1 = i0 + Lx;
      v[vi * ld + i0] = post ? a0.get() * post[i0] : a0.get();
      v[vi * ld + i1] = post ? a1.get() * post[i1] : a1.get();
    }
    __syncthreads();
    return;
  }
  // A thread takes the same element of two vectors (2 vp, 2 vp + 1): the two
  // sums are independent and share every tap load.  The taps are stored twice
  // over (tx[k] = Ex[k mod Lx] for k < 2 Lx), so that tap x - x' mod Lx is
  // tx[x + Lx - x'] without a wrap test.
  const int npair = (nv + 1) >> 1, ptot = npair * N;
  for (int e = threadIdx.x; e < ptot; e += blockDim.x) {
    const int vp = e / N, i = e - vp * N;
    const int x = i % Lx, y = i / Lx;
    const bool two = 2 * vp + 1 < nv;
    const T* row0 = v + (2 * vp) * ld + Lx * y;
    const T* row1 = two ? row0 + ld : row0;
    const T* tp = tx + x + Lx;
    ProdSum<T> a0, a1;
    for (int xp = 0; xp < Lx; ++xp) {
      const T t = tp[-xp];
      a0.add(t, row0[xp]);
      a1.add(t, row1[xp]);
    }
    tmp[(2 * vp) * ld + i] = a0.get();
    if (two) tmp[(2 * vp + 1) * ld + i] = a1.get();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ptot; e += blockDim.x) {
    const int vp = e / N, i = e - vp * N;
    const int x = i % Lx, y = i / Lx;
    const bool two = 2 * vp + 1 < nv;
    const T* col0 = tmp + (2 * vp) * ld + x;
    const T* col1 = two ? col0 + ld : col0;
    const T* tp = ty + y + Ly;
    ProdSum<T> a0, a1;
    for (int yp = 0; yp < Ly; ++yp) {
      const T t = tp[-yp];
      a0.add(t, col0[Lx * yp]);
      a1.add(t, col1[Lx * yp]);
    }
    const T sc = post ? post[i] : T(1);
    v[(2 * vp) * ld + i] = post ? a0.get() * sc : a0.get();
    if (two) v[(2 * vp + 1) * ld + i] = post ? a1.get() * sc : a1.get();
  }
  __syncthreads();
}

// Shared-memory staging common to both Kronecker kernels.
template <typename T>
struct KronStage {
  T* v;
  T* tmp;
  T* tx;   // active taps x
  T* ty;   // active taps y
  T* txs;  // the same taps shifted by one, txs[k] = tx[k + 1] (paired loads)
  T* tys;
  T* sc;   // diag scale of the current slice
};

template <typename T>
__device__ __forceinline__ KronStage<T> kron_stage(unsigned char* raw, int nv, int ld) {
  KronStage<T> s;
  s.v = reinterpret_cast<T*>(raw);
  s.tmp = s.v + nv * ld;
  s.tx = s.tmp + nv * ld;
  s.ty = s.tx + 2 * kMaxSide;
  s.txs = s.ty + 2 * kMaxSide;
  s.tys = s.txs + 2 * kMaxSide;
  s.sc = s.tys + 2 * kMaxSide;
  return s;
}

// Resolve the slice range of batch entry b (one chain, or one chain x block).
__device__ __forceinline__ bool kron_entry_range(const KronArgs& a, int b, int* chain, int* first,
                                                 int* count) {
  *chain = b / a.per_chain;
  if (a.cp) {
    const int blk = b - *chain * a.per_chain;
    const int lo = a.cp[blk] + a.step, hi = a.cp[blk + 1];
    *first = lo;
    *count = (lo < hi) ? 1 : 0;
    return lo < hi;
  }
  *first = a.l0_first;
  *count = a.n_slices;
  return a.n_slices > 0;
}

template <typename T>
__device__ __forceinline__ void kron_load_taps(const KronArgs& a, KronStage<T> s) {
  if (threadIdx.x < 2 * kMaxSide) {  // each circulant row twice over (kron_transform)
    const int t = threadIdx.x, tx = t % a.Lx, ty = t % a.Ly;
    const bool inv = (a.kind == kBIT);
    s.tx[t] = static_cast<T>(inv ? a.taps.exi[tx] : a.taps.ex[tx]);
    s.ty[t] = static_cast<T>(inv ? a.taps.eyi[ty] : a.taps.ey[ty]);
    const int tx1 = (t + 1) % a.Lx, ty1 = (t + 1) % a.Ly;
    s.txs[t] = static_cast<T>(inv ? a.taps.exi[tx1] : a.taps.ex[tx1]);
    s.tys[t] = static_cast<T>(inv ? a.taps.eyi[ty1] : a.taps.ey[ty1]);
  }
}

template <typename T>
__device__ __forceinline__ void kron_load_scale(const KronArgs& a, KronStage<T> s,
                                                const int8_t* f_l, int N) {
  // e^{+-c}, precomputed on the host: FP64 exp is dozens of FP64-pipe passes.
  const T up = static_cast<T>((a.kind == kBIT) ? a.emc : a.ec);
  const T dn = static_cast<T>((a.kind == kBIT) ? a.ec : a.emc);
  for (int i = threadIdx.x; i < N; i += blockDim.x) s.sc[i] = f_l[i] > 0 ? up : dn;
}

// Vectors are contiguous rows of each N x N matrix.  Each CTA owns nv rows of
// one batch entry and applies `count` successive slice factors to them.
template <typename T>
__global__ void __launch_bounds__(256) k_kron_rows(const T* in, T* out, KronArgs a) {
  const int b = blockIdx.y;
  int chain, first, count;
  if (!kron_entry_range(a, b, &chain, &first, &count)) return;
  const int N = a.N, nv = a.nv, ld = N + 1;
  const int r0 = blockIdx.x * nv;
  const int nrows = min(nv, N - r0);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  KronStage<T> s = kron_stage<T>(sm_raw, nv, ld);
  kron_load_taps(a, s);
  const T* src = in + static_cast<size_t>(b) * a.mat_stride;
  T* dst = out + static_cast<size_t>(b) * a.out_stride;
  for (int e = threadIdx.x; e < nrows * N; e += blockDim.x) {
    const int vi = e / N, i = e - vi * N;
    T val = src[static_cast<size_t>(r0 + vi) * N + i];
    if (a.vscale) val *= static_cast<T>(a.vscale[static_cast<size_t>(b) * a.vscale_stride + r0 + vi]);
    s.v[vi * ld + i] = val;
  }
  const int8_t* f = a.field + static_cast<size_t>(chain) * a.L * N;
  for (int st = 0; st < count; ++st) {
    const int l0 = first + st * a.dir;
    __syncthreads();
    kron_load_scale(a, s, f + static_cast<size_t>(l0) * N, N);
    __syncthreads();
    if (a.kind == kBT)
      kron_transform(s.v, s.tmp, nrows, ld, a.Lx, a.Ly, N, s.tx, s.ty, s.txs, s.tys, (const T*)nullptr,
                     (const T*)s.sc);
    else
      kron_transform(s.v, s.tmp, nrows, ld, a.Lx, a.Ly, N, s.tx, s.ty, s.txs, s.tys, (const T*)s.sc,
                     (const T*)nullptr);
  }
  for (int e = threadIdx.x; e < nrows * N; e += blockDim.x) {
    const int vi = e / N, i = e - vi * N;
    dst[static_cast<size_t>(r0 + vi) * N + i] = s.v[vi * ld + i];
  }
}

// Vectors are the columns of each row-major N x N matrix (in place).
template <typename T>
__global__ void __launch_bounds__(256) k_kron_cols(T* X, KronArgs a) {
  const int b = blockIdx.y;
  int chain, first, count;
  if (!kron_entry_range(a, b, &chain, &first, &count)) return;
  const int N = a.N, nv = a.nv, ld = N + 1;
  const int c0 = blockIdx.x * nv;
  const int ncols = min(nv, N - c0);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  KronStage<T> s = kron_stage<T>(sm_raw, nv, ld);
  kron_load_taps(a, s);
  T* M = X + static_cast<size_t>(b) * a.mat_stride;
  for (int e = threadIdx.x; e < ncols * N; e += blockDim.x) {
    const int i = e / ncols, jj = e - i * ncols;
    s.v[jj * ld + i] = M[static_cast<size_t>(i) * N + c0 + jj];
  }
  const int8_t* f = a.field + static_cast<size_t>(chain) * a.L * N;
  for (int st = 0; st < count; ++st) {
    const int l0 = first + st * a.dir;
    __syncthreads();
    kron_load_scale(a, s, f + static_cast<size_t>(l0) * N, N);
    __syncthreads();
    if (a.kind == kBT)
      kron_transform(s.v, s.tmp, ncols, ld, a.Lx, a.Ly, N, s.tx, s.ty, s.txs, s.tys, (const T*)nullptr,
                     (const T*)s.sc);
    else
      kron_transform(s.v, s.tmp, ncols, ld, a.Lx, a.Ly, N, s.tx, s.ty, s.txs, s.tys, (const T*)s.sc,
                     (const T*)nullptr);
  }
  for (int e = threadIdx.x; e < ncols * N; e += blockDim.x) {
    const int i = e / ncols, jj = e - i * ncols;
    M[static_cast<size_t>(i) * N + c0 + jj] = s.v[jj * ld + i];
  }
}

// ---------------------------------------------------------------------------
// Drift check: drift[c] = max(drift[c], max|Gw - G64| / max|G64|), then the
// working G is replaced by the stabilised one.  One CTA per chain.
// ---------------------------------------------------------------------------
// One cluster of kDriftCS CTAs per chain, each over an interleaved share of
// the elements: max |Gw - G64| and max |G64| are taken on the bit patterns of
// the absolute values (non-negative doubles order as integers), so the only
// FP64 work per element is the conversion and the difference; non-finite
// entries of G64 are left out of the maxima and flagged, an infinite
// difference counts, a NaN difference does not (as fmax would have it).  CTA 0 combines the
// partial maxima of the cluster through distributed shared memory.
constexpr int kDriftCS = 2;
template <typename T>
__global__ void __launch_bounds__(256) k_drift_reset(const double* G64, T* Gw, int N, double* drift,
                                                    int* status) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  const int c = blockIdx.x / kDriftCS;
  const size_t nn = static_cast<size_t>(N) * N;
  const double* g = G64 + c * nn;
  T* w = Gw + c * nn;
  unsigned long long md = 0ull, mg = 0ull;
  bool bad = false;
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull;
  for (size_t e = rank * blockDim.x + threadIdx.x; e < nn; e += kDriftCS * blockDim.x) {
    const double ge = g[e];
    const unsigned long long ga = static_cast<unsigned long long>(__double_as_longlong(ge)) & kAbs;
    if (ga >= 0x7FF0000000000000ull) {  // Inf or NaN
      bad = true;
    } else {
      const unsigned long long da =
          static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(w[e]) - ge)) & kAbs;
      md = (da <= 0x7FF0000000000000ull && da > md) ? da : md;  // Inf counts, NaN not
      mg = ga > mg ? ga : mg;
    }
    w[e] = static_cast<T>(ge);
  }
  __shared__ unsigned long long s1[32], s2[32];
  __shared__ int sb;
  if (threadIdx.x == 0) sb = 0;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long m1 = __shfl_xor_sync(0xFFFFFFFFu, md, o);
    const unsigned long long m2 = __shfl_xor_sync(0xFFFFFFFFu, mg, o);
    md = m1 > md ? m1 : md;
    mg = m2 > mg ? m2 : mg;
  }
  __syncthreads();
  if (bad) atomicOr(&sb, 1);
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = md;
    s2[threadIdx.x >> 5] = mg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w2 = 1; w2 < static_cast<int>(blockDim.x >> 5); ++w2) {
      md = s1[w2] > md ? s1[w2] : md;
      mg = s2[w2] > mg ? s2[w2] : mg;
    }
    s1[0] = md;
    s2[0] = mg;
    if (sb) atomicExch(status, kDevNonFinite);
  }
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) {
    for (int r = 1; r < kDriftCS; ++r) {
      const unsigned long long m1 = *cl.map_shared_rank(&s1[0], r);
      const unsigned long long m2 = *cl.map_shared_rank(&s2[0], r);
      md = m1 > md ? m1 : md;
      mg = m2 > mg ? m2 : mg;
    }
    const double mdd = __longlong_as_double(static_cast<long long>(md));
    const double mgd = __longlong_as_double(static_cast<long long>(mg));
    const double dr = mgd > 0.0 ? mdd / mgd : mdd;
    if (!(dr <= drift[c])) drift[c] = dr;
  }
  cl.sync();  // the peers' shared memory stays until CTA 0 has read it
}

// ---------------------------------------------------------------------------
// Equal-time observables of one configuration from the stabilised G_up
// (G_dn = I - P G_up^T P):  n = (1/N) sum_i [(1 - G_ii) + G_ii],
// docc = (1/N) sum_i (1 - G_ii) G_ii,
// ekin = (1/N) sum_sigma sum_ij K_ij <c^dag_i c_j> = (2t/N) sum_j sum_delta G_{j, j+delta},
// and the translation-averaged spin correlation of Sec. 4 (Fig. 5),
// C(r) = (1/N) sum_i <S^z_i S^z_{i+r}>, S^z = (n_up - n_dn)/2, accumulated into
// spin[c][r], r = dx + Lx dy.  Wick's theorem per spin with G_dn = I - P G_up^T P
// gives, for a = G_ij, b = G_ji, d = delta_ij, p = p_i p_j = (-1)^(dx+dy) (even
// sides) and m_i = n_i,up - n_i,dn = 1 - 2 G_ii:
//   4 <S^z_i S^z_j> = m_i m_j + (d - b) a + p a (d - p b)
// (spin-up exchange, then spin-down exchange).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_observables(const double* G64, int Lx, int Ly, double t,
                                                    double* obs, double* spin) {
  const int c = blockIdx.x;
  const int N = Lx * Ly;
  const double* G = G64 + static_cast<size_t>(c) * N * N;
  __shared__ double m[kMaxN];
  for (int i = threadIdx.x; i < N; i += blockDim.x) m[i] = 1.0 - 2.0 * G[static_cast<size_t>(i) * N + i];
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int dx = r % Lx, dy = r / Lx;
    const double p = ((dx + dy) & 1) ? -1.0 : 1.0;
    double acc = 0.0;
    int y = 0, yj = dy;
    for (; y < Ly; ++y) {
      const int row0 = Lx * y, rowj = Lx * yj;
#pragma unroll 4
      for (int x = 0; x < Lx; ++x) {
        const int xj = (x + dx < Lx) ? x + dx : x + dx - Lx;
        const int i = row0 + x, j = rowj + xj;
        const double a = G[static_cast<size_t>(i) * N + j];
        const double b = G[static_cast<size_t>(j) * N + i];
        const double d = (i == j) ? 1.0 : 0.0;
        acc += m[i] * m[j] + (d - b) * a + p * a * (d - p * b);
      }
      yj = (yj + 1 == Ly) ? 0 : yj + 1;
    }
    spin[static_cast<size_t>(c) * N + r] += acc / (4.0 * N);
  }
  double n = 0.0, dc = 0.0, ek = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double g = G[static_cast<size_t>(j) * N + j];
    n += (1.0 - g) + g;
    dc += (1.0 - g) * g;
    const int x = j % Lx, y = j / Lx;
    const int nb[4] = {(x + 1) % Lx + Lx * y, (x + Lx - 1) % Lx + Lx * y, x + Lx * ((y + 1) % Ly),
                       x + Lx * ((y + Ly - 1) % Ly)};
    for (int q = 0; q < 4; ++q) ek += G[static_cast<size_t>(j) * N + nb[q]];
  }
  __shared__ double sm[3][32];
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    dc += __shfl_xor_sync(0xFFFFFFFFu, dc, o);
    ek += __shfl_xor_sync(0xFFFFFFFFu, ek, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sm[0][threadIdx.x >> 5] = n;
    sm[1][threadIdx.x >> 5] = dc;
    sm[2][threadIdx.x >> 5] = ek;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) {
      n += sm[0][w];
      dc += sm[1][w];
      ek += sm[2][w];
    }
    double* o = obs + static_cast<size_t>(c) * 4;
    o[0] += n / N;
    o[1] += dc / N;
    o[2] += 2.0 * t * ek / N;
    o[3] += 1.0;
  }
}

// ---------------------------------------------------------------------------
// Correlation length of Sec. 4 (Fig. 5): least-squares line through
// (|r|, ln c(r)), c(r) = (-1)^(dx+dy) C(r) the staggered correlation,
// |r| = sqrt(min(dx, Lx-dx)^2 + min(dy, Ly-dy)^2), over 0 < |r| <= dmax and
// c(r) > 0; xi = -1/slope (+inf for a slope >= 0, nan below two distinct
// distances).  C(r) = spin[c][r] / obs[c][3] for block c < C; block C takes
// the chain average sum_c spin[c][r] / sum_c obs[c][3].  One thread per r.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_corr_length(const double* spin, const double* obs, int C,
                                                    int Lx, int Ly, double dmax, double* out) {
  const int b = blockIdx.x, N = Lx * Ly;
  __shared__ double cnt_sh;
  if (threadIdx.x == 0) {
    double cnt = 0.0;
    if (b < C) {
      cnt = obs[static_cast<size_t>(b) * 4 + 3];
    } else {
      for (int c = 0; c < C; ++c) cnt += obs[static_cast<size_t>(c) * 4 + 3];
    }
    cnt_sh = cnt;
  }
  __syncthreads();
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // n, S_d, S_y, S_dd, S_dy
  double dmin = CUDART_INF, dmaxp = -1.0;     // smallest / largest distance used
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    double v = 0.0;
    if (b < C) {
      v = spin[static_cast<size_t>(b) * N + r];
    } else {
      for (int c = 0; c < C; ++c) v += spin[static_cast<size_t>(c) * N + r];
    }
    const int dx = r % Lx, dy = r / Lx;
    const double cr = (((dx + dy) & 1) ? -v : v) / cnt_sh;
    const int ax = min(dx, Lx - dx), ay = min(dy, Ly - dy);
    const double d = sqrt(static_cast<double>(ax * ax + ay * ay));
    if (d > 0.0 && d <= dmax && cr > 0.0) {
      const double y = log(cr);
      s[0] += 1.0;
      s[1] += d;
      s[2] += y;
      s[3] += d * d;
      s[4] += d * y;
      dmin = fmin(dmin, d);
      dmaxp = fmax(dmaxp, d);
    }
  }
  __shared__ double red[8][7];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 5; ++q) s[q] += __shfl_xor_sync(0xFFFFFFFFu, s[q], o);
    dmin = fmin(dmin, __shfl_xor_sync(0xFFFFFFFFu, dmin, o));
    dmaxp = fmax(dmaxp, __shfl_xor_sync(0xFFFFFFFFu, dmaxp, o));
  }
  if (lane == 0) {
    for (int q = 0; q < 5; ++q) red[w][q] = s[q];
    red[w][5] = dmin;
    red[w][6] = dmaxp;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double lo = CUDART_INF, hi = -1.0;
    for (int q = 0; q < nw; ++q) {
      for (int k = 0; k < 5; ++k) t[k] += red[q][k];
      lo = fmin(lo, red[q][5]);
      hi = fmax(hi, red[q][6]);
    }
    double xi = CUDART_NAN;
    const double den = t[0] * t[3] - t[1] * t[1];
    if (t[0] >= 2.0 && hi > lo && den > 0.0) {
      const double slope = (t[0] * t[4] - t[1] * t[2]) / den;
      xi = (slope < 0.0) ? -1.0 / slope : CUDART_INF;
    }
    out[b] = xi;
  }
}

// ---------------------------------------------------------------------------
// Host launch wrappers.
// ---------------------------------------------------------------------------
cudaError_t launch_init_field(int8_t* field, int C, int L, int N, int chain0, uint64_t seed,
                              cudaStream_t st) {
  const long long total = static_cast<long long>(C) * L * N;
  const int blocks = static_cast<int>(std::min<long long>((total + 255) / 256, 152 * 16));
  k_init_field<<<blocks, 256, 0, st>>>(field, C, L, N, chain0, static_cast<uint32_t>(seed),
                                       static_cast<uint32_t>(seed >> 32));
  return cudaGetLastError();
}

template <typename T>
size_t metropolis_smem(int N, int k) {
  const int NP = ((N + 31) / 32) * 32;
  return static_cast<size_t>(NP) * (sizeof(double) + sizeof(float)) + 2ull * k * NP * sizeof(T) +
         static_cast<size_t>(NP) * (sizeof(T) + sizeof(float) + sizeof(int)) +
         static_cast<size_t>(kWin) * (NP + 1) * sizeof(T);
}

template <typename T>
cudaError_t launch_metropolis(T* G, int8_t* field, int C, const MetroArgs& a, cudaStream_t st) {
  const int NP = ((a.N + 31) / 32) * 32;
  const int threads = NP * metro_halves<T>();
  const size_t sm = metropolis_smem<T>(a.N, a.k);
  cudaError_t e = cudaFuncSetAttribute(k_metropolis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  if (a.cs <= 1) {
    k_metropolis<T><<<C, threads, sm, st>>>(G, field, a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * a.cs, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_metropolis<T>, G, field, a);
}

template <typename T>
size_t kron_smem(int N, int nv) {
  return (2ull * nv * (N + 1) + 8 * kMaxSide + N) * sizeof(T);
}

template <typename T>
cudaError_t launch_kron_rows(const T* in, T* out, int batch, const KronArgs& a, cudaStream_t st) {
  const size_t sm = kron_smem<T>(a.N, a.nv);
  cudaError_t e = cudaFuncSetAttribute(k_kron_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + a.nv - 1) / a.nv, batch);
  k_kron_rows<T><<<grid, 256, sm, st>>>(in, out, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kron_cols(T* X, int batch, const KronArgs& a, cudaStream_t st) {
  const size_t sm = kron_smem<T>(a.N, a.nv);
  cudaError_t e = cudaFuncSetAttribute(k_kron_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + a.nv - 1) / a.nv, batch);
  k_kron_cols<T><<<grid, 256, sm, st>>>(X, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_drift_reset(const double* G64, T* Gw, int C, int N, double* drift, int* status,
                               cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * kDriftCS, 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kDriftCS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_drift_reset<T>, G64, Gw, N, drift, status);
}

cudaError_t launch_observables(const double* G64, int C, int Lx, int Ly, double t, double* obs,
                               double* spin, cudaStream_t st) {
  k_observables<<<C, 256, 0, st>>>(G64, Lx, Ly, t, obs, spin);
  return cudaGetLastError();
}

cudaError_t launch_corr_length(const double* spin, const double* obs, int C, int Lx, int Ly,
                               double dmax, double* out, cudaStream_t st) {
  k_corr_length<<<C + 1, 256, 0, st>>>(spin, obs, C, Lx, Ly, dmax, out);
  return cudaGetLastError();
}

#define DQMC_INST(T)                                                                              \
  template cudaError_t launch_metropolis<T>(T*, int8_t*, int, const MetroArgs&, cudaStream_t);   \
  template cudaError_t launch_kron_rows<T>(const T*, T*, int, const KronArgs&, cudaStream_t);    \
  template cudaError_t launch_kron_cols<T>(T*, int, const KronArgs&, cudaStream_t);              \
  template cudaError_t launch_drift_reset<T>(const double*, T*, int, int, double*, int*,         \
                                             cudaStream_t);                                      \
  template size_t metropolis_smem<T>(int, int);
DQMC_INST(double)
DQMC_INST(float)
DQMC_INST(df32)
#undef DQMC_INST

}  // namespace dqmc
