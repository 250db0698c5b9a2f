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
//
// The Matsubara transform of a G_k(tau) grid with the Dyson self-energy
// (dqmc_matsubara_sigma) reuses k_tx_spline and adds k_mats_setup (root and
// weight tables) and k_mats (one CTA per frequency and 32 momenta).
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

// Matsubara transform of the spline (Eq. 5) and Dyson equation (Eq. 6).  On
// interval j (tau_j = j h, t = tau - tau_j in [0, h]) the spline is
//   p_j(t) = y_j + c1_j t + (M_j / 2) t^2 + (M_{j+1} - M_j) / (6h) t^3,
//   c1_j = (y_{j+1} - y_j) / h - h (2 M_j + M_{j+1}) / 6,
// and each interval is integrated exactly with the moments
//   K_m = int_0^h t^m e^{i w t} dt = h^{m+1} J_m(theta),  theta = w h,
//   J_m(theta) = int_0^1 u^m e^{i theta u} du
// (series in theta below 1.5; above, J_0 = (e^{i theta} - 1)/(i theta) and
// J_m = (e^{i theta} - m J_{m-1})/(i theta), amplifying rounding by at most
// m / theta <= 2 per step).  Collecting terms,
//   int p_j e^{i w tau} = z_j (y_j P + y_{j+1} Q + M_j R + M_{j+1} S),  z_j = e^{i w tau_j},
//   P = K_0 - K_1/h,  Q = K_1/h,  R = K_2/2 - (h/3) K_1 - K_3/(6h),  S = K_3/(6h) - (h/6) K_1,
// and since z_{j-1} = z_j e^{-i theta} the sum over intervals is one sum over
// the knots with weights (P + e^{-i theta} Q, R + e^{-i theta} S), only the
// first halves at j = 0 and only the second halves at j = M.  Nothing
// cancels at low frequencies.  z_j = e^{i pi (2n+1) j / M} comes from a table
// of the 2M roots e^{i pi r / M}, r = (2n+1) j mod 2M kept exact in integers.
// The samples are the non-negative G of the sweeps: the standard-sign
// G(i w_n) is minus the integral, and Sigma = i w_n - eps_k - 1/G (mu = 0).
struct Cx {
  double re, im;
};
__device__ __forceinline__ Cx cmul(Cx a, Cx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ Cx cadd(Cx a, Cx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Cx cscale(Cx a, double s) { return {a.re * s, a.im * s}; }

// J_m(theta), m = 0..3
__device__ void moments01(double theta, double ct, double st, Cx J[4]) {
  if (theta < 1.5) {
    // J_m = sum_k (i theta)^k / (k! (m + k + 1))
    for (int m = 0; m < 4; ++m) J[m] = {0.0, 0.0};
    Cx term = {1.0, 0.0};  // (i theta)^k / k!
    for (int k = 0; k < 32; ++k) {
      for (int m = 0; m < 4; ++m) J[m] = cadd(J[m], cscale(term, 1.0 / (m + k + 1)));
      term = cscale(cmul(term, Cx{0.0, theta}), 1.0 / (k + 1));
    }
  } else {
    // 1 / (i theta) = -i / theta
    const Cx e = {ct, st}, inv = {0.0, -1.0 / theta};
    J[0] = cmul(Cx{e.re - 1.0, e.im}, inv);
    for (int m = 1; m < 4; ++m) J[m] = cmul(Cx{e.re - m * J[m - 1].re, e.im - m * J[m - 1].im}, inv);
  }
}

// Tables shared by all momenta: ph[r] = e^{i pi r / M} (r < 2M) and, per
// frequency n, the knot weights wt[n] = {P, R, Wy, Wm, e^{-i theta} Q, e^{-i theta} S}.
constexpr int kMatsW = 6;
__global__ void __launch_bounds__(256) k_mats_setup(int M, double beta, int n_freq, Cx* ph, Cx* wt) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < 2 * M) {
    double sn, cs;
    sincospi(static_cast<double>(x) / M, &sn, &cs);
    ph[x] = {cs, sn};
  }
  if (x < n_freq) {
    const int f = 2 * x + 1;
    const double h = beta / M;
    double st, ct;  // e^{i theta}, theta = w h = pi (2n+1) / M
    sincospi(static_cast<double>(f % (2 * M)) / M, &st, &ct);
    Cx J[4];
    moments01(f * (3.141592653589793238 / M), ct, st, J);
    const Cx K0 = cscale(J[0], h), K1 = cscale(J[1], h * h), K2 = cscale(J[2], h * h * h),
             K3 = cscale(J[3], h * h * h * h);
    const double ih = 1.0 / h;
    const Cx P = cadd(K0, cscale(K1, -ih)), Q = cscale(K1, ih);
    const Cx R = cadd(cadd(cscale(K2, 0.5), cscale(K1, -h / 3.0)), cscale(K3, -ih / 6.0));
    const Cx S = cadd(cscale(K3, ih / 6.0), cscale(K1, -h / 6.0));
    const Cx em = {ct, -st};
    const Cx Qm = cmul(em, Q), Sm = cmul(em, S);
    Cx* o = wt + static_cast<size_t>(x) * kMatsW;
    o[0] = P;
    o[1] = R;
    o[2] = cadd(P, Qm);
    o[3] = cadd(R, Sm);
    o[4] = Qm;
    o[5] = Sm;
  }
}

// One CTA per (frequency, 32 momenta); its 8 warps split the interior knots
// 1..M-1 into 8 contiguous segments and their partial sums are combined in
// shared memory in a fixed order.
__global__ void __launch_bounds__(256) k_mats(const double* y, const double* m2, const Cx* ph,
                                              const Cx* wt, int M, int Lx, int Ly, double t,
                                              double beta, int n_freq, double* g_iw,
                                              double* sigma) {
  const int N = Lx * Ly, nkc = (N + 31) / 32;
  const int n = blockIdx.x / nkc, k = (blockIdx.x - n * nkc) * 32 + threadIdx.x;
  const int f = 2 * n + 1, twoM = 2 * M, step = f % twoM;
  const Cx* W = wt + static_cast<size_t>(n) * kMatsW;
  const bool live = k < N;
  const double* yy = y + (live ? k : 0);
  const double* mm = m2 + (live ? k : 0);
  // second derivatives M_0..M_M (rows 1..M-1 are stored; not-a-knot ends)
  auto Md = [&](int j) {
    if (j == 0) return 2.0 * mm[N] - mm[2 * N];
    if (j == M) return 2.0 * mm[static_cast<long long>(M - 1) * N] -
                       mm[static_cast<long long>(M - 2) * N];
    return mm[static_cast<long long>(j) * N];
  };
  // interior knots: the weights are the same for every knot, so only the
  // sums A = sum_j z_j y_j and B = sum_j z_j M_j are accumulated (4 FMAs a knot)
  const int len = (M - 1 + 7) / 8;
  const int j0 = 1 + threadIdx.y * len, j1 = min(M, j0 + len);
  Cx A = {0.0, 0.0}, B = {0.0, 0.0};
  if (live && j0 < j1) {
    int r = static_cast<int>((static_cast<long long>(step) * j0) % twoM);
    for (int j = j0; j < j1; ++j) {
      const double yj = yy[static_cast<long long>(j) * N], mj = mm[static_cast<long long>(j) * N];
      const Cx z = ph[r];
      A.re += z.re * yj;
      A.im += z.im * yj;
      B.re += z.re * mj;
      B.im += z.im * mj;
      r += step;
      if (r >= twoM) r -= twoM;
    }
  }
  __shared__ Cx part[2][8][32];
  part[0][threadIdx.y][threadIdx.x] = A;
  part[1][threadIdx.y][threadIdx.x] = B;
  __syncthreads();
  if (threadIdx.y != 0 || !live) return;
  A = part[0][0][threadIdx.x];
  B = part[1][0][threadIdx.x];
  for (int q = 1; q < 8; ++q) {
    A = cadd(A, part[0][q][threadIdx.x]);
    B = cadd(B, part[1][q][threadIdx.x]);
  }
  // knot 0 (z_0 = 1): first halves only; knot M (z_M = e^{i w beta} = -1): second halves only
  Cx tot = cadd(cscale(W[0], yy[0]), cscale(W[1], Md(0)));
  tot = cadd(tot, cadd(cmul(W[2], A), cmul(W[3], B)));
  const Cx cM = cadd(cscale(W[4], yy[static_cast<long long>(M) * N]), cscale(W[5], Md(M)));
  tot = {tot.re - cM.re, tot.im - cM.im};
  const long long e = static_cast<long long>(n) * N + k;
  if (g_iw) {  // standard sign: G = -I
    g_iw[2 * e] = -tot.re;
    g_iw[2 * e + 1] = -tot.im;
  }
  const int kx = k % Lx, ky = k / Lx;
  const double eps = -2.0 * t * (cospi(2.0 * kx / Lx) + cospi(2.0 * ky / Ly));
  const double w = f * (3.141592653589793238 / beta);
  // Sigma = i w - eps - 1/G = i w - eps + 1/I
  const double den = tot.re * tot.re + tot.im * tot.im;
  sigma[2 * e] = -eps + tot.re / den;
  sigma[2 * e + 1] = w - tot.im / den;
}

// Scratch kept between calls, one buffer per device, grown on demand and
// never shrunk (freed with the process).  The mutex serialises calls, which
// would otherwise share the buffer.
constexpr int kTxMaxDevices = 64;
struct TxScratch {
  void* p = nullptr;
  size_t bytes = 0;
  cudaEvent_t ev[4] = {};
  float last_ms[3] = {0.0f, 0.0f, 0.0f};  // extrapolation: its three kernels, last call
  float mats_ms[2] = {0.0f, 0.0f};        // Matsubara: spline, transform, last call
};
TxScratch g_tx_scratch[kTxMaxDevices];
std::mutex g_tx_mu;

size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

// Make sc hold at least `need` bytes and its timing events (caller holds g_tx_mu).
int grow(TxScratch& sc, size_t need) {
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
  if (!sc.ev[0]) {
    for (cudaEvent_t& ev : sc.ev)
      if (cudaEventCreate(&ev) != cudaSuccess) return DQMC_ERR_CUDA;
  }
  return DQMC_OK;
}

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
  const int rc = grow(sc, need);
  if (rc != DQMC_OK) return rc;
  char* base = static_cast<char*>(sc.p);
  double* y = reinterpret_cast<double*>(base);
  double* m2 = reinterpret_cast<double*>(base + ybytes);
  double* stage_in = reinterpret_cast<double*>(base + 2 * ybytes);
  double* stage_out = reinterpret_cast<double*>(base + 2 * ybytes + ibytes);
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

extern "C" int dqmc_matsubara_sigma(const double* gk, int M, int Lx, int Ly, double t, double beta,
                                    int n_freq, double* g_iw, double* sigma, int on_device) {
  if (!gk || !sigma || M < 3 || Lx < 1 || Ly < 1 || !(beta > 0.0) || n_freq < 1 ||
      !std::isfinite(t))
    return DQMC_ERR_ARG;
  const int N = Lx * Ly;
  TxArgs a{};
  a.R = 1;
  a.N = N;
  a.M = M;
  a.beta = beta;
  a.run[0].off = 0;
  a.run[0].h = beta / M;
  a.run[0].inv_h = M / beta;
  a.run[0].inv_6h = 1.0 / (6.0 * a.run[0].h);
  a.run[0].L = M;
  a.run[0].C = 1;
  const size_t ybytes = align256(static_cast<size_t>(M + 1) * N * sizeof(double));
  const size_t pbytes = align256(static_cast<size_t>(2 * M) * sizeof(Cx)) +
                        align256(static_cast<size_t>(n_freq) * kMatsW * sizeof(Cx));
  const size_t obytes = static_cast<size_t>(n_freq) * N * 2 * sizeof(double);
  const size_t need = ybytes + pbytes + (on_device ? 0 : ybytes + 2 * align256(obytes));
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTxMaxDevices) return DQMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_tx_mu);
  TxScratch& sc = g_tx_scratch[dev];
  const int rc = grow(sc, need);
  if (rc != DQMC_OK) return rc;
  char* base = static_cast<char*>(sc.p);
  double* m2 = reinterpret_cast<double*>(base);
  Cx* ph = reinterpret_cast<Cx*>(base + ybytes);
  Cx* wt = reinterpret_cast<Cx*>(base + ybytes + align256(static_cast<size_t>(2 * M) * sizeof(Cx)));
  const double* y = gk;
  double* s_out = sigma;
  double* g_out = g_iw;
  cudaStream_t st = 0;
  if (!on_device) {
    double* ys = reinterpret_cast<double*>(base + ybytes + pbytes);
    s_out = reinterpret_cast<double*>(base + 2 * ybytes + pbytes);
    g_out = g_iw ? reinterpret_cast<double*>(base + 2 * ybytes + pbytes + align256(obytes)) : nullptr;
    if (cudaMemcpyAsync(ys, gk, static_cast<size_t>(M + 1) * N * sizeof(double),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
      return DQMC_ERR_CUDA;
    y = ys;
  }
  const long long spline_elems = static_cast<long long>(M - 1) * N;
  cudaEventRecord(sc.ev[0], st);
  k_tx_spline<<<dim3(static_cast<unsigned>((spline_elems + 255) / 256), 1), 256, 0, st>>>(a, y, m2);
  cudaEventRecord(sc.ev[1], st);
  k_mats_setup<<<(std::max(2 * M, n_freq) + 255) / 256, 256, 0, st>>>(M, beta, n_freq, ph, wt);
  k_mats<<<static_cast<unsigned>(n_freq) * ((N + 31) / 32), dim3(32, 8), 0, st>>>(
      y, m2, ph, wt, M, Lx, Ly, t, beta, n_freq, g_out, s_out);
  cudaEventRecord(sc.ev[2], st);
  if (cudaGetLastError() != cudaSuccess) return DQMC_ERR_CUDA;
  if (!on_device) {
    if (cudaMemcpyAsync(sigma, s_out, obytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        (g_iw && cudaMemcpyAsync(g_iw, g_out, obytes, cudaMemcpyDeviceToHost, st) != cudaSuccess))
      return DQMC_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return DQMC_ERR_CUDA;
  for (int q = 0; q < 2; ++q)
    if (cudaEventElapsedTime(&sc.mats_ms[q], sc.ev[q], sc.ev[q + 1]) != cudaSuccess)
      return DQMC_ERR_CUDA;
  return DQMC_OK;
}

extern "C" int dqmc_matsubara_timing(float* ms_out) {
  if (!ms_out) return DQMC_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTxMaxDevices) return DQMC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_tx_mu);
  for (int q = 0; q < 2; ++q) ms_out[q] = g_tx_scratch[dev].mats_ms[q];
  return DQMC_OK;
}
