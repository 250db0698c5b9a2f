// dtau -> 0 extrapolation of the momentum-resolved Green function G_k(tau)
// (Sec. 3, Fig. 2): runs at several Trotter steps live on different grids
// tau_l = l dtau_r; each is averaged over its chains, put on one common fine
// grid by a cubic spline, and extrapolated pointwise in dtau^2.
//
// Three FP64 kernels, all data-parallel with the momentum index k fastest in
// every array, so that every access is coalesced:
//   k_tx_mean    (32 elements x 8 chain groups) per CTA: average over the run's
//                chains of the [C][L+1][N] layout dqmc_measure_Gtau writes,
//                partial sums combined in shared memory in a fixed order;
//   k_tx_spline  one thread per (l, k): second derivative M_l of the
//                not-a-knot spline through the run's L+1 points, from the
//                closed-form inverse of its tridiagonal system (below);
//   k_tx_fit     one thread per (m, k): every run's spline at tau_m = m beta/M,
//                then the least-squares line in dtau^2, whose intercept is kept.
// The chain average reads every input byte once and dominates; the other two
// touch only the averaged arrays (L2-resident).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/dqmc.h"

namespace dqmc {
namespace {

constexpr int kTxMaxRuns = DQMC_TX_MAX_RUNS;

struct TxRun {
  const double* g;  // [C][L+1][N] chain data of the run (device)
  long long off;    // offset of the run's rows in y and m2 ([L+1][N] each)
  double h;         // dtau of the run
  double inv_h, inv_6h;
  int L, C;
};

struct TxArgs {
  TxRun run[kTxMaxRuns];
  int R, N, M;
  double beta;
};

__global__ void __launch_bounds__(256) k_tx_mean(TxArgs a, double* y) {
  const TxRun& r = a.run[blockIdx.y];
  const long long n = static_cast<long long>(r.L + 1) * a.N;
  const long long e = static_cast<long long>(blockIdx.x) * 32 + threadIdx.x;
  double sv[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (e < n) {
    int c = threadIdx.y;  // chains threadIdx.y, +8, +16, ...: 8 loads in flight per thread
    for (; c + 56 < r.C; c += 64) {
#pragma unroll
      for (int u = 0; u < 8; ++u) sv[u] += r.g[(c + 8 * u) * n + e];
    }
    for (; c < r.C; c += 8) sv[0] += r.g[c * n + e];
  }
  __shared__ double part[8][33];
  part[threadIdx.y][threadIdx.x] = ((sv[0] + sv[1]) + (sv[2] + sv[3])) + ((sv[4] + sv[5]) + (sv[6] + sv[7]));
  __syncthreads();
  if (threadIdx.y == 0 && e < n) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += part[q][threadIdx.x];
    y[r.off * a.N + e] = t / r.C;
  }
}

// Not-a-knot cubic spline on the uniform grid x_i = i h, i = 0..n (n = L >= 3),
// second derivatives M_i.  Continuity of the spline's second derivative gives
//   M_{i-1} + 4 M_i + M_{i+1} = d_i = 6 (y_{i+1} - 2 y_i + y_{i-1}) / h^2,  i = 1..n-1,
// and not-a-knot (continuous third derivative at x_1 and x_{n-1}) gives
// M_0 = 2 M_1 - M_2 and M_n = 2 M_{n-1} - M_{n-2}.  Substituted into the
// equations for i = 1 and i = n-1 these leave M_1 = d_1 / 6 and
// M_{n-1} = d_{n-1} / 6.  The rows i = 2..n-2 form T x = b with
// T = tridiag(1, 4, 1) of order n' = n - 3, x_p = M_{p+1} and
// b_p = d_{p+1} - [p = 1] M_1 - [p = n'] M_{n-1}.  With rho = 2 + sqrt 3 the
// inverse is (Chebyshev polynomials U_m(2) = (rho^{m+1} - rho^{-m-1}) / (2 sqrt 3))
//   (T^-1)_pq = (-1)^{p+q} U_{lo-1}(2) U_{n'-hi}(2) / U_{n'}(2),   lo = min, hi = max,
// which in powers of r = 2 - sqrt 3 = 1/rho < 1 (no overflow at any n') reads
//   (T^-1)_pq = (-1)^{p+q} r^{hi-lo} (1 - r^{2 lo}) (1 - r^{2(n'-hi+1)})
//               / ((1 - r^{2(n'+1)}) 2 sqrt 3).
// Entries decay like r^{|p-q|}; terms with |p - q| > kTxW = 32 are below
// r^33 < 2e-19 of the largest and are dropped, so every M_l is an independent
// 65-tap sum.  M_0 and M_n are formed where they are used (k_tx_fit).
constexpr int kTxW = 32;
constexpr int kTxE = 24;  // 1 - r^{2m} == 1 in FP64 for m >= kTxE (r^48 < 1e-27)

__global__ void __launch_bounds__(256) k_tx_spline(TxArgs a, const double* y, double* m2) {
  // sr[m] = (-1)^m r^m, m = 0..kTxW;  e1[m] = 1 - r^{2m}, m < kTxE
  __shared__ double sr[kTxW + 1], e1[kTxE];
  const double rr = 2.0 - sqrt(3.0);
  for (int m = threadIdx.x; m <= kTxW; m += blockDim.x)
    sr[m] = ((m & 1) ? -1.0 : 1.0) * pow(rr, static_cast<double>(m));
  for (int m = threadIdx.x; m < kTxE; m += blockDim.x) e1[m] = 1.0 - pow(rr, 2.0 * m);
  __syncthreads();
  const TxRun& r = a.run[blockIdx.y];
  const int n = r.L, N = a.N;
  const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= static_cast<long long>(n - 1) * N) return;
  const int i = 1 + static_cast<int>(e / N), k = static_cast<int>(e % N);
  const double* yy = y + r.off * N + k;
  const double s = 6.0 / (r.h * r.h);
  // second difference D_j = y_{j+1} - 2 y_j + y_{j-1}, so d_j = s D_j
  auto D = [&](int j) { return yy[(j + 1) * N] - 2.0 * yy[j * N] + yy[(j - 1) * N]; };
  const double m1 = s * D(1) / 6.0, mn1 = s * D(n - 1) / 6.0;
  double mi;
  if (i == 1) {
    mi = m1;
  } else if (i == n - 1) {
    mi = mn1;
  } else {
    const int np = n - 3, p = i - 1;
    const int q0 = max(1, p - kTxW), q1 = min(np, p + kTxW);
    auto E = [&](int m) { return m < kTxE ? e1[m] : 1.0; };
    // (T^-1)_pq = sr[|p-q|] E(lo) E(np - hi + 1) / (E(np + 1) 2 sqrt 3); the E factors
    // differ from 1 only within kTxE rows of either end of the system
    const bool edge = (p - kTxW < kTxE) || (np - (p + kTxW) + 1 < kTxE);
    double acc = 0.0;
    double ya = yy[q0 * N], yb = yy[(q0 + 1) * N];  // window y_q, y_{q+1}, y_{q+2} for D_{q+1}
    if (edge) {
      for (int q = q0; q <= q1; ++q) {
        const double yc = yy[(q + 2) * N];
        const int lo = min(p, q), hi = max(p, q);
        acc += sr[hi - lo] * E(lo) * E(np - hi + 1) * ((yc - 2.0 * yb) + ya);
        ya = yb;
        yb = yc;
      }
    } else {
      for (int q = q0; q <= q1; ++q) {
        const double yc = yy[(q + 2) * N];
        acc += sr[q > p ? q - p : p - q] * ((yc - 2.0 * yb) + ya);
        ya = yb;
        yb = yc;
      }
    }
    acc *= s;
    // the known neighbours M_1 and M_{n-1} moved to the right-hand side of rows 1 and np
    if (q0 == 1) acc -= sr[p - 1] * E(1) * E(np - p + 1) * m1;
    if (q1 == np) acc -= sr[np - p] * E(p) * E(1) * mn1;
    mi = acc / (E(np + 1) * 2.0 * sqrt(3.0));
  }
  m2[r.off * N + static_cast<long long>(i) * N + k] = mi;
}

__global__ void __launch_bounds__(256) k_tx_fit(TxArgs a, const double* y, const double* m2,
                                                double* out) {
  const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int N = a.N;
  if (e >= static_cast<long long>(a.M + 1) * N) return;
  const int m = static_cast<int>(e / N), k = static_cast<int>(e - static_cast<long long>(m) * N);
  const double tau = m * (a.beta / a.M);
  double sx = 0.0, sxx = 0.0, sy = 0.0, sxy = 0.0, last = 0.0;
  for (int q = 0; q < a.R; ++q) {
    const TxRun& r = a.run[q];
    const int n = r.L;
    const double h = r.h, ih = r.inv_h, i6h = r.inv_6h, h6 = h / 6.0;
    int l = static_cast<int>(floor(tau * ih));
    l = l < 0 ? 0 : (l > n - 1 ? n - 1 : l);
    const double t = tau - l * h, u = h - t;
    const double* yy = y + r.off * N + k;
    const double* mm = m2 + r.off * N + k;
    // M_0 = 2 M_1 - M_2 and M_n = 2 M_{n-1} - M_{n-2} (not-a-knot ends)
    auto M = [&](int j) {
      if (j == 0) return 2.0 * mm[N] - mm[2 * N];
      if (j == n) return 2.0 * mm[(n - 1) * N] - mm[(n - 2) * N];
      return mm[j * N];
    };
    const double y0 = yy[l * N], y1 = yy[(l + 1) * N], M0 = M(l), M1 = M(l + 1);
    const double v = (M0 * u * u * u + M1 * t * t * t) * i6h + (y0 * ih - M0 * h6) * u +
                     (y1 * ih - M1 * h6) * t;
    const double x = h * h;
    sx += x;
    sxx += x * x;
    sy += v;
    sxy += x * v;
    last = v;
  }
  if (a.R == 1) {
    out[e] = last;
    return;
  }
  // intercept of the least-squares line v = a + b x over the runs
  out[e] = (sxx * sy - sx * sxy) / (a.R * sxx - sx * sx);
}

// Scratch kept between calls, one buffer per device, grown on demand and
// never shrunk (freed with the process).  The mutex serialises calls, which
// would otherwise share the buffer.
constexpr int kTxMaxDevices = 64;
struct TxScratch {
  void* p = nullptr;
  size_t bytes = 0;
  cudaEvent_t ev[4] = {};
  float last_ms[3] = {0.0f, 0.0f, 0.0f};  // device time of the three kernels, last call
};
TxScratch g_tx_scratch[kTxMaxDevices];
std::mutex g_tx_mu;

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

}  // namespace
}  // namespace dqmc

using namespace dqmc;

extern "C" int dqmc_trotter_extrapolate(int R, const double* dtau, const int* L, const int* C,
                                        const double* const* gk, int N, double beta, int M,
                                        double* out, int on_device) {
  if (R < 1 || R > kTxMaxRuns || !dtau || !L || !C || !gk || !out || N < 1 || M < 1 ||
      !(beta > 0.0))
    return DQMC_ERR_ARG;
  TxArgs a{};
  a.R = R;
  a.N = N;
  a.M = M;
  a.beta = beta;
  long long rows = 0, chain_elems = 0;
  int maxrow = 0;
  double sx = 0.0, sxx = 0.0;
  for (int r = 0; r < R; ++r) {
    if (!gk[r] || L[r] < 3 || C[r] < 1 || !(dtau[r] > 0.0)) return DQMC_ERR_ARG;
    if (std::fabs(L[r] * dtau[r] - beta) > 1e-9 * beta) return DQMC_ERR_ARG;
    a.run[r].off = rows;
    a.run[r].h = dtau[r];
    a.run[r].inv_h = 1.0 / dtau[r];
    a.run[r].inv_6h = 1.0 / (6.0 * dtau[r]);
    a.run[r].L = L[r];
    a.run[r].C = C[r];
    rows += L[r] + 1;
    chain_elems += static_cast<long long>(C[r]) * (L[r] + 1) * N;
    maxrow = std::max(maxrow, L[r] + 1);
    sx += dtau[r] * dtau[r];
    sxx += dtau[r] * dtau[r] * dtau[r] * dtau[r];
  }
  if (R >= 2 && !(R * sxx - sx * sx > 1e-12 * sxx * R)) return DQMC_ERR_ARG;  // all dtau equal
  const size_t ybytes = align256(static_cast<size_t>(rows) * N * sizeof(double));
  const size_t ibytes = on_device ? 0 : align256(static_cast<size_t>(chain_elems) * sizeof(double));
  const size_t obytes = static_cast<size_t>(M + 1) * N * sizeof(double);
  const size_t need = 2 * ybytes + ibytes + (on_device ? 0 : align256(obytes));
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTxMaxDevices) return DQMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_tx_mu);
  TxScratch& sc = g_tx_scratch[dev];
  if (sc.bytes < need) {
    if (sc.p) cudaFree(sc.p);
    sc.p = nullptr;
    sc.bytes = 0;
    if (cudaMalloc(&sc.p, need) != cudaSuccess) {
      cudaGetLastError();
      sc.p = nullptr;
      return DQMC_ERR_OOM;
    }
    sc.bytes = need;
  }
  char* base = static_cast<char*>(sc.p);
  double* y = reinterpret_cast<double*>(base);
  double* m2 = reinterpret_cast<double*>(base + ybytes);
  double* stage_in = reinterpret_cast<double*>(base + 2 * ybytes);
  double* stage_out = reinterpret_cast<double*>(base + 2 * ybytes + ibytes);
  if (!sc.ev[0]) {
    for (cudaEvent_t& ev : sc.ev)
      if (cudaEventCreate(&ev) != cudaSuccess) return DQMC_ERR_CUDA;
  }
  cudaStream_t st = 0;
  long long coff = 0;
  for (int r = 0; r < R; ++r) {
    const long long n = static_cast<long long>(C[r]) * (L[r] + 1) * N;
    if (on_device) {
      a.run[r].g = gk[r];
    } else {
      double* dst = stage_in + coff;
      if (cudaMemcpyAsync(dst, gk[r], n * sizeof(double), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
        return DQMC_ERR_CUDA;
      a.run[r].g = dst;
    }
    coff += n;
  }
  double* o = on_device ? out : stage_out;
  const long long mean_elems = static_cast<long long>(maxrow) * N;
  const long long spline_elems = static_cast<long long>(maxrow - 2) * N;
  const long long fit_elems = static_cast<long long>(M + 1) * N;
  cudaEventRecord(sc.ev[0], st);
  k_tx_mean<<<dim3(static_cast<unsigned>((mean_elems + 31) / 32), R), dim3(32, 8), 0, st>>>(a, y);
  cudaEventRecord(sc.ev[1], st);
  k_tx_spline<<<dim3(static_cast<unsigned>((spline_elems + 255) / 256), R), 256, 0, st>>>(a, y, m2);
  cudaEventRecord(sc.ev[2], st);
  k_tx_fit<<<static_cast<unsigned>((fit_elems + 255) / 256), 256, 0, st>>>(a, y, m2, o);
  cudaEventRecord(sc.ev[3], st);
  if (cudaGetLastError() != cudaSuccess) return DQMC_ERR_CUDA;
  if (!on_device &&
      cudaMemcpyAsync(out, o, obytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return DQMC_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return DQMC_ERR_CUDA;
  for (int q = 0; q < 3; ++q)
    if (cudaEventElapsedTime(&sc.last_ms[q], sc.ev[q], sc.ev[q + 1]) != cudaSuccess)
      return DQMC_ERR_CUDA;
  return DQMC_OK;
}

extern "C" int dqmc_trotter_timing(float* ms_out) {
  if (!ms_out) return DQMC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTxMaxDevices) return DQMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_tx_mu);
  for (int q = 0; q < 3; ++q) ms_out[q] = g_tx_scratch[dev].last_ms[q];
  return DQMC_OK;
}
