// Host runtime and C ABI of libdqmc (see include/dqmc.h).
//
// One context holds groups of independent Markov chains.  Device state per
// group (FP64 unless noted, chains batch-major):
//   field  int8 [C][L][N]           Ising HS field (Sec. 2)
//   Gw     T    [C][N][N]           working G(l) of spin up (T = double/float)
//   G64         [C][N][N]           last stabilised G
//   RU,RT       [C][nc+1][N][N]     right stack R_c = B_c..B_1 = U D T (U stored transposed)
//   RD          [C][nc+1][N]
//   LU,LT,LD                        left stack, UDT factors of L_c^T = (B_L..B_{c+1})^T
//   X,Rtil      [C][N][N]           QR workspace
//   Mid,W1,W2,A1,A2 [C][nc+1][N][N] stabilised-G workspaces (all stabilisation points at once)
// Stabilisation points cp[j] = min(j n_s, L), j = 0..nc.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/dqmc.h"
#include "common.cuh"
#include "kernels.h"

namespace dqmc {

__global__ void k_increment(uint32_t* ctr) { *ctr += 1u; }

__global__ void k_zero(double* p, long long n) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    p[e] = 0.0;
}

// acc += a x
__global__ void k_axpy(double* acc, const double* x, double a, long long n) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    acc[e] += a * x[e];
}

// Field rotated by s slices: out[c][l][i] = in[c][(l + s) mod L][i].
__global__ void k_rotate_field(const int8_t* in, int8_t* out, int C, int L, int N, int s) {
  const long long n = static_cast<long long>(C) * L * N;
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const long long c = e / (static_cast<long long>(L) * N);
    const long long r = e - c * L * N;
    const int l = static_cast<int>(r / N), i = static_cast<int>(r - static_cast<long long>(l) * N);
    const int ls = (l + s) % L;
    out[e] = in[(c * L + ls) * N + i];
  }
}

// log W = 2 (sum log Db_L(0) + log|det Mid(0)|) - lambda sum_il s_il   (det M_dn = e^{-lambda sum s} det M_up)
__global__ void k_logw(const double* LD0, long long sLD, const double* logabs_mid, long long sMid,
                       const int8_t* field, int L, int N, double lam, double* out) {
  const int c = blockIdx.x;
  double a = 0.0, s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a += log(fmax(LD0[c * sLD + i], 1.0));
  for (long long e = threadIdx.x; e < static_cast<long long>(L) * N; e += blockDim.x)
    s += field[static_cast<size_t>(c) * L * N + e];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  }
  __shared__ double sa[32], ss[32];
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    ss[threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) {
      a += sa[w];
      s += ss[w];
    }
    out[c] = 2.0 * (a + logabs_mid[c * sMid]) - lam * s;
  }
}

__global__ void k_pick3(const double* acc, double* dt, double* dl, int C) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
    if (dt) dt[c] = acc[c * 3 + 0];
    if (dl) dl[c] = acc[c * 3 + 1];
  }
}

struct Group {
  dqmc_group p;
  int N = 0, L = 0, nc = 0, C = 0, chain0 = 0;
  double lam = 0.0;
  std::vector<int> cp;
  KronTaps taps{};
  int8_t* field = nullptr;
  void* Gw = nullptr;
  double *G64 = nullptr, *RU = nullptr, *RD = nullptr, *RT = nullptr;
  double *LU = nullptr, *LD = nullptr, *LT = nullptr;
  double *X = nullptr, *Rtil = nullptr;
  double *Mid = nullptr, *W1 = nullptr, *W2 = nullptr, *A1 = nullptr, *A2 = nullptr;
  double *logabs = nullptr, *obs = nullptr, *drift = nullptr, *bins = nullptr, *gacc = nullptr;
  double* spin = nullptr;  // [C][N] accumulated spin correlation C(r)
  double* gout = nullptr;  // [C][L+1][N] staging of G(tau) for host output
  double* qrs = nullptr;   // [C][2N] column norms of the QR
  void* oz = nullptr;      // digit slices of the tensor-core FP64 GEMM
  int oz_batch = 0;
  QrbWork qrb{};           // blocked-QR workspace (tensor-core path)
  // tile shapes (dqmc_set_tiles; 0 = the built-in choice)
  int tile_kron = 0, tile_wrap = 0, tile_metro = 0;
  cudaStream_t st = nullptr;   // stream this group's work is enqueued on
  cudaStream_t cap = nullptr;  // the group's own stream (graph capture branches)
  cudaEvent_t join = nullptr;
  unsigned long long* acc = nullptr;
  int *d_cp_gtau = nullptr, *d_cp_grad = nullptr;
  long long nn() const { return static_cast<long long>(N) * N; }
  long long sstride() const { return static_cast<long long>(nc + 1) * N * N; }
};

thread_local cudaError_t g_last_cuda = cudaSuccess;  // last failing CUDA call (this thread)
thread_local int g_last_line = 0;

void record_cuda_error(cudaError_t e, int line) {
  g_last_cuda = e;
  g_last_line = line;
}

}  // namespace dqmc

using namespace dqmc;

// Kernel classes for the optional per-launch timing (dqmc_timing_*).
enum TimingClass : int {
  kTMetropolis = 0, kTWrap, kTStackKron, kTQR, kTGemm, kTInverse, kTGtauProp, kTGtauFinal,
  kTGrad, kTInversePair, kTMisc, kTNumClasses
};
static const char* kTimingNames[kTNumClasses] = {
    "metropolis", "wrap", "stack_kron", "qr_pivot", "gemm_f64", "gj_inverse", "gtau_propagate",
    "gtau_finalize", "grad_terms", "gj_inverse_pair", "misc"};

struct dqmc_ctx {
  std::vector<Group> g;
  cudaStream_t st = nullptr;
  int gemm_mode = DQMC_GEMM_TENSOR;
  int qr_mode = DQMC_QR_BLOCKED;
  // CUDA graph of one sweep of all groups (index: measure flag), captured on
  // cap_main with one forked branch per group, replayed on st.
  bool use_graph = true;
  cudaStream_t cap_main = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  long long graph_launches[2] = {0, 0};
  // timing: event pairs recorded around launches while enabled
  bool timing = false;
  int tclass = kTMisc;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_class;
  size_t ev_used = 0;
  double tms[kTNumClasses] = {};
  long long tcount[kTNumClasses] = {};
  uint64_t seed = 0;
  int64_t chain_offset = 0;  // global id of this context's first chain (Philox counter word)
  uint32_t* d_sweep = nullptr;
  int* d_status = nullptr;
  int total = 0;
  int nsm = 0;       // SMs of the device
  int metro_cs = 0;  // CTAs per chain in the Metropolis pass (0 = automatic)
  long long launches = 0;
  std::vector<void*> allocs;
};

namespace {

constexpr int kOzakiMinN = 64;  // smaller matrices stay on the FP64 pipe
constexpr double kTuneMargin = 0.05;  // probe drift must stay below 5% of the target


#define DQ_CK(call)                                 \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      g_last_cuda = e_;                             \
      g_last_line = __LINE__;                       \
      return DQMC_ERR_CUDA;                         \
    }                                               \
  } while (0)
#define DQ_RET(call)                 \
  do {                               \
    int r_ = (call);                 \
    if (r_ != DQMC_OK) return r_;    \
  } while (0)
#define DQ_LAUNCH(ctx, call)                        \
  do {                                              \
    ++(ctx)->launches;                              \
    const int slot_ = timing_begin(ctx);            \
    DQ_CK(call);                                    \
    if (slot_ >= 0) DQ_CK(timing_end(ctx, slot_));  \
  } while (0)
int timing_begin(dqmc_ctx* ctx);
cudaError_t timing_end(dqmc_ctx* ctx, int slot);
#define DQ_CLASS(ctx, c) ((ctx)->tclass = (c))
#define DQ_LAUNCH_C(ctx, c, call) \
  do {                            \
    DQ_CLASS(ctx, c);             \
    DQ_LAUNCH(ctx, call);         \
  } while (0)

// Fold the elapsed times of all recorded pairs into the per-class sums.
int timing_fold(dqmc_ctx* ctx) {
  if (ctx->ev_used == 0) return DQMC_OK;
  DQ_CK(cudaEventSynchronize(ctx->ev[2 * (ctx->ev_used - 1) + 1]));
  for (size_t i = 0; i < ctx->ev_used; ++i) {
    float ms = 0.f;
    DQ_CK(cudaEventElapsedTime(&ms, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    ctx->tms[ctx->ev_class[i]] += ms;
    ctx->tcount[ctx->ev_class[i]] += 1;
  }
  ctx->ev_used = 0;
  return DQMC_OK;
}

int timing_begin(dqmc_ctx* ctx) {
  if (!ctx->timing) return -1;
  if (ctx->ev_used * 2 >= ctx->ev.size()) {
    if (timing_fold(ctx) != DQMC_OK) return -1;
  }
  const size_t slot = ctx->ev_used++;
  ctx->ev_class[slot] = ctx->tclass;
  if (cudaEventRecord(ctx->ev[2 * slot], ctx->st) != cudaSuccess) return -1;
  return static_cast<int>(slot);
}

cudaError_t timing_end(dqmc_ctx* ctx, int slot) {
  return cudaEventRecord(ctx->ev[2 * slot + 1], ctx->st);
}

template <typename P>
int dev_alloc(dqmc_ctx* ctx, P** p, size_t bytes) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    return DQMC_ERR_OOM;
  }
  ctx->allocs.push_back(q);
  *p = static_cast<P*>(q);
  return DQMC_OK;
}

// Circulant taps of exp(-+dtau K_1D) on a periodic ring of length n with
// one-dimensional band -2t cos k: e[d] = (1/n) sum_m cos(2 pi m d / n) exp(+-2 t dtau cos(2 pi m / n)).
void ring_taps(int n, double t, double dtau, double* e, double* ei) {
  for (int d = 0; d < kMaxSide; ++d) {
    e[d] = 0.0;
    ei[d] = 0.0;
  }
  for (int d = 0; d < n; ++d) {
    double a = 0.0, b = 0.0;
    for (int m = 0; m < n; ++m) {
      const double k = 2.0 * M_PI * m / n;
      const double c = std::cos(k * d);
      a += c * std::exp(2.0 * t * dtau * std::cos(k));
      b += c * std::exp(-2.0 * t * dtau * std::cos(k));
    }
    e[d] = a / n;
    ei[d] = b / n;
  }
}

KronArgs kron_base(const Group& g, int kind, int nv) {
  KronArgs a{};
  a.N = g.N;
  a.Lx = g.p.Lx;
  a.Ly = g.p.Ly;
  a.L = g.L;
  a.nv = nv;
  a.kind = kind;
  a.c = g.lam;  // sigma = +1 (spin up)
  a.ec = std::exp(g.lam);
  a.emc = std::exp(-g.lam);
  a.taps = g.taps;
  a.field = g.field;
  a.mat_stride = g.nn();
  a.out_stride = g.nn();
  a.per_chain = 1;
  a.dir = 1;
  return a;
}

int kron_nv(const Group& g, bool fp64) {
  if (g.tile_kron > 0) return std::min(g.tile_kron, g.N);
  // Vectors per CTA of the FP64 Kronecker transforms (stack products, G(tau)
  // of FP64 groups, gradient): small tiles, so that several CTAs share an SM
  // and their independent FMA chains keep the FP64 pipe busy (measured on the
  // 16x16 sweep: 4 vectors 73 ms, 8 vectors 75 ms, 29 vectors 87 ms for the
  // stack products).
  const int budget = fp64 ? 120 * 1024 : 110 * 1024;
  const int per = (g.N + 1) * 2 * (fp64 ? 8 : 4);
  int nv = std::max(1, std::min(4, budget / per));
  return std::min(nv, g.N);
}

// Vectors per CTA of the slice wrap in the working precision.  The
// float-pair and FP32 transforms run serial chains of compensated sums per
// element and need many resident warps to hide their latency: small tiles
// (4 vectors, about 17 KB of shared memory at N = 256).
template <typename T>
int wrap_nv(const Group& g) {
  if (g.tile_wrap > 0) return std::min(g.tile_wrap, g.N);
  if (sizeof(T) == 8 && !std::is_same<T, df32>::value) return kron_nv(g, true);
  return std::min(4, g.N);
}

GemmArgs gemm0(int n) {
  GemmArgs a{};
  a.n = n;
  a.alpha = 1.0;
  return a;
}

// FP64 products: on the tensor cores (digit-sliced, FP64-level accuracy) for
// N >= kOzakiMinN unless the context asks for the FP64 pipe.
cudaError_t gemm(dqmc_ctx* ctx, Group& g, const GemmArgs& m, int batch) {
  if (ctx->gemm_mode == DQMC_GEMM_TENSOR && g.oz) {
    // the split and the MMA kernel (plus the balance pass) per chunk of the
    // batch (the square products take the split path)
    const int chunks = (batch + g.oz_batch - 1) / g.oz_batch;
    ctx->launches += static_cast<long long>(chunks) * (m.balance ? 3 : 2) - 1;
    return launch_gemm_ozaki(m, batch, g.oz, g.oz_batch, ctx->d_status, g.st);
  }
  return launch_gemm(m, batch, g.st);
}

// QR of the stack step X = B..B (U D) (rows of g.X = columns of X) into the
// stack entry (Q^T at Qt, D at Dv) and g.Rtil: the blocked, pre-pivoted QR
// with tensor-core updates where the tensor-core products are in use, the
// column-pivoted cluster QR on the FP64 pipe otherwise.
cudaError_t stack_qr(dqmc_ctx* ctx, Group& g, double* Qt, double* Dv) {
  const long long sD = static_cast<long long>(g.nc + 1) * g.N;
  if (ctx->gemm_mode == DQMC_GEMM_TENSOR && ctx->qr_mode == DQMC_QR_BLOCKED && g.oz) {
    ctx->launches += qr_blocked_launches(g.N, g.C, g.oz_batch) - 1;
    return launch_qr_blocked(g.X, g.nn(), Qt, g.sstride(), Dv, sD, g.Rtil, g.nn(), g.qrb, g.N, g.C,
                             g.oz, g.oz_batch, ctx->d_status, g.st);
  }
  return launch_qrp_cluster(g.X, g.nn(), Qt, g.sstride(), Dv, sD, g.Rtil, g.nn(), g.qrs, g.N, g.C,
                            ctx->d_status, g.st);
}

// ---- UDV stack steps ------------------------------------------------------

// X = B ... B (U D) for a stack step: on the tensor cores where the
// tensor-core products are in use (N >= 64), else on the FP64 pipe.
cudaError_t stack_kron(dqmc_ctx* ctx, Group& g, const double* in, const KronArgs& a) {
  if (ctx->gemm_mode == DQMC_GEMM_TENSOR && g.oz)
    return launch_kron_tc(in, g.X, g.C, a, ctx->d_status, g.st);
  return launch_kron_rows<double>(in, g.X, g.C, a, g.st);
}

// Right stack entry j from entry j-1 and slices cp[j-1]+1 .. cp[j].
int stack_right(dqmc_ctx* ctx, Group& g, int j) {
  KronArgs a = kron_base(g, kB, kron_nv(g, true));
  a.mat_stride = g.sstride();
  a.out_stride = g.nn();
  a.vscale = g.RD + static_cast<long long>(j - 1) * g.N;
  a.vscale_stride = static_cast<long long>(g.nc + 1) * g.N;
  a.l0_first = g.cp[j - 1];
  a.dir = 1;
  a.n_slices = g.cp[j] - g.cp[j - 1];
  DQ_CLASS(ctx, kTStackKron);
  DQ_LAUNCH(ctx, stack_kron(ctx, g, g.RU + (j - 1) * g.nn(), a));
  DQ_CLASS(ctx, kTQR);
  DQ_LAUNCH(ctx, stack_qr(ctx, g, g.RU + j * g.nn(), g.RD + j * g.N));
  GemmArgs m = gemm0(g.N);
  m.A = g.Rtil; m.sA = g.nn();
  m.balance = 1;  // the rows of T differ in magnitude; Rtil is triangular
  m.B = g.RT + (j - 1) * g.nn(); m.sB = g.sstride();
  m.C = g.RT + j * g.nn(); m.sC = g.sstride();
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, g.C));
  return DQMC_OK;
}

// Left stack entry j from entry j+1 and slices cp[j+1] .. cp[j]+1 (descending).
int stack_left(dqmc_ctx* ctx, Group& g, int j) {
  KronArgs a = kron_base(g, kBT, kron_nv(g, true));
  a.mat_stride = g.sstride();
  a.out_stride = g.nn();
  a.vscale = g.LD + static_cast<long long>(j + 1) * g.N;
  a.vscale_stride = static_cast<long long>(g.nc + 1) * g.N;
  a.l0_first = g.cp[j + 1] - 1;
  a.dir = -1;
  a.n_slices = g.cp[j + 1] - g.cp[j];
  DQ_CLASS(ctx, kTStackKron);
  DQ_LAUNCH(ctx, stack_kron(ctx, g, g.LU + (j + 1) * g.nn(), a));
  DQ_CLASS(ctx, kTQR);
  DQ_LAUNCH(ctx, stack_qr(ctx, g, g.LU + j * g.nn(), g.LD + j * g.N));
  GemmArgs m = gemm0(g.N);
  m.A = g.Rtil; m.sA = g.nn();
  m.balance = 1;  // the rows of T differ in magnitude; Rtil is triangular
  m.B = g.LT + (j + 1) * g.nn(); m.sB = g.sstride();
  m.C = g.LT + j * g.nn(); m.sC = g.sstride();
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, g.C));
  return DQMC_OK;
}

// Mid = Db_R^{-1} (U_R^T U_L) Db_L^{-1} + Ds_R (T_R T_L^T) Ds_L for `batch`
// stack entries starting at entry j0 of every chain (stride `es` between the
// entries of one batch), written to out (stride N^2).
int form_mid(dqmc_ctx* ctx, Group& g, int j0, long long es, int batch, double* out) {
  const long long dstride = es / g.N;  // D vectors have stride es/N
  GemmArgs m = gemm0(g.N);
  m.A = g.RU + j0 * g.nn(); m.sA = es; m.tA = 0;
  m.B = g.LU + j0 * g.nn(); m.sB = es; m.tB = 1;
  m.C = out; m.sC = g.nn();
  m.rs = g.RD + j0 * g.N; m.srs = dstride; m.rs_mode = 2;
  m.cs = g.LD + j0 * g.N; m.scs = dstride; m.cs_mode = 2;
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
  m.A = g.RT + j0 * g.nn();
  m.B = g.LT + j0 * g.nn();
  m.balance = 1;
  m.rs_mode = 3;
  m.cs_mode = 3;
  m.beta = 1.0;
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
  return DQMC_OK;
}

// G64 = U_L Db_L^{-1} Mid^{-1} Db_R^{-1} U_R^T at stack entry j of every chain.
int recompute(dqmc_ctx* ctx, Group& g, int j) {
  DQ_RET(form_mid(ctx, g, j, g.sstride(), g.C, g.X));
  DQ_CLASS(ctx, kTInverse);
  DQ_LAUNCH(ctx, launch_gj_cluster(g.X, g.nn(), g.G64, g.nn(), g.N, g.C, nullptr, ctx->d_status,
                                   g.st));
  // U_L (Db_L^{-1} Mid^{-1}): Mid^{-1} grows like Db_L along its rows, so the
  // scale is folded into them (Db_L^{-1} Mid^{-1} Db_R^{-1} is O(|G|)).
  GemmArgs m = gemm0(g.N);
  m.A = g.LU + j * g.nn(); m.sA = g.sstride(); m.tA = 1;
  m.ks = g.LD + j * g.N; m.sks = static_cast<long long>(g.nc + 1) * g.N; m.ks_mode = 2;
  m.ks_on_b = 1;
  m.balance = 1;
  m.B = g.G64; m.sB = g.nn();
  m.C = g.Rtil; m.sC = g.nn();
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, g.C));
  m = gemm0(g.N);
  m.A = g.Rtil; m.sA = g.nn();
  m.ks = g.RD + j * g.N; m.sks = static_cast<long long>(g.nc + 1) * g.N; m.ks_mode = 2;
  m.B = g.RU + j * g.nn(); m.sB = g.sstride();
  m.C = g.G64; m.sC = g.nn();
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, g.C));
  return DQMC_OK;
}

template <typename T>
int drift_reset(dqmc_ctx* ctx, Group& g) {
  DQ_CLASS(ctx, kTMisc);
  DQ_LAUNCH(ctx, launch_drift_reset<T>(g.G64, static_cast<T*>(g.Gw), g.C, g.N, g.drift,
                                        ctx->d_status, g.st));
  return DQMC_OK;
}

int drift_reset_any(dqmc_ctx* ctx, Group& g) {
  if (g.p.precision == DQMC_FP32) return drift_reset<float>(ctx, g);
  if (g.p.precision == DQMC_DF32) return drift_reset<df32>(ctx, g);
  return drift_reset<double>(ctx, g);
}

// Working G <- stabilised G64 (no drift recorded).
int load_working(dqmc_ctx* ctx, Group& g) {
  ++ctx->launches;
  cudaError_t e;
  if (g.p.precision == DQMC_FP32)
    e = launch_convert<float>(g.G64, static_cast<float*>(g.Gw), g.C * g.nn(), g.st);
  else if (g.p.precision == DQMC_DF32)
    e = launch_convert<df32>(g.G64, static_cast<df32*>(g.Gw), g.C * g.nn(), g.st);
  else
    e = launch_convert<double>(g.G64, static_cast<double*>(g.Gw), g.C * g.nn(), g.st);
  if (e != cudaSuccess) {
    g_last_cuda = e;
    g_last_line = __LINE__;
    return DQMC_ERR_CUDA;
  }
  return DQMC_OK;
}

int left_pass(dqmc_ctx* ctx, Group& g) {
  for (int j = g.nc - 1; j >= 0; --j) DQ_RET(stack_left(ctx, g, j));
  return DQMC_OK;
}

int right_pass(dqmc_ctx* ctx, Group& g) {
  for (int j = 1; j <= g.nc; ++j) DQ_RET(stack_right(ctx, g, j));
  return DQMC_OK;
}

// Both stacks from the current field and the stabilised G(0); the working G
// is overwritten (its drift against G(0) is recorded when record != 0).
int rebuild(dqmc_ctx* ctx, Group& g) {
  DQ_CLASS(ctx, kTMisc);
  DQ_LAUNCH(ctx, launch_set_identity(g.RU, g.sstride(), g.RD, static_cast<long long>(g.nc + 1) * g.N,
                                     g.N, g.C, g.st));
  DQ_CLASS(ctx, kTMisc);
  DQ_LAUNCH(ctx, launch_set_identity(g.RT, g.sstride(), nullptr, 0, g.N, g.C, g.st));
  DQ_CLASS(ctx, kTMisc);
  DQ_LAUNCH(ctx, launch_set_identity(g.LU + g.nc * g.nn(), g.sstride(), g.LD + g.nc * g.N,
                                     static_cast<long long>(g.nc + 1) * g.N, g.N, g.C, g.st));
  DQ_CLASS(ctx, kTMisc);
  DQ_LAUNCH(ctx, launch_set_identity(g.LT + g.nc * g.nn(), g.sstride(), nullptr, 0, g.N, g.C,
                                     g.st));
  DQ_RET(right_pass(ctx, g));
  DQ_RET(left_pass(ctx, g));
  DQ_RET(recompute(ctx, g, 0));
  return DQMC_OK;
}

template <typename T>
int up_pass(dqmc_ctx* ctx, Group& g, int measure) {
  const double em2 = std::expm1(-2.0 * g.lam), ep2 = std::expm1(2.0 * g.lam);
  MetroArgs ma{};
  ma.N = g.N;
  ma.L = g.L;
  ma.k = g.p.delay_k;
  ma.chain0 = static_cast<int>(g.chain0 + ctx->chain_offset);  // Philox chain word
  ma.key0 = static_cast<uint32_t>(ctx->seed);
  ma.key1 = static_cast<uint32_t>(ctx->seed >> 32);
  ma.sweep_ctr = ctx->d_sweep;
  ma.em2 = em2;
  ma.ep2 = ep2;
  ma.em2h = static_cast<float>(em2);
  ma.em2l = static_cast<float>(em2 - static_cast<double>(ma.em2h));
  ma.ep2h = static_cast<float>(ep2);
  ma.ep2l = static_cast<float>(ep2 - static_cast<double>(ma.ep2h));
  ma.accepted = g.acc;
  ma.status = ctx->d_status;
  ma.cs = g.tile_metro > 0 ? g.tile_metro : ctx->metro_cs;
  if (ma.cs == 0) {  // all chains of all groups run their Metropolis passes side by side
    ma.cs = 1;
    for (int cs : {4, 2})
      if (static_cast<long long>(cs) * ctx->total <= ctx->nsm && g.N >= 4 * cs) {
        ma.cs = cs;
        break;
      }
  }
  KronArgs wl = kron_base(g, kB, wrap_nv<T>(g));
  KronArgs wr = kron_base(g, kBIT, wrap_nv<T>(g));
  wl.n_slices = wr.n_slices = 1;
  T* Gw = static_cast<T*>(g.Gw);
  int j = 1;
  for (int l = 1; l <= g.L; ++l) {
    ma.l0 = l - 1;
    DQ_CLASS(ctx, kTMetropolis);
    DQ_LAUNCH(ctx, launch_metropolis<T>(Gw, g.field, g.C, ma, g.st));
    wl.l0_first = wr.l0_first = l - 1;
    DQ_CLASS(ctx, kTWrap);
    DQ_LAUNCH(ctx, launch_kron_cols<T>(Gw, g.C, wl, g.st));
    DQ_CLASS(ctx, kTWrap);
    DQ_LAUNCH(ctx, launch_kron_rows<T>(Gw, Gw, g.C, wr, g.st));
    if (l == g.cp[j]) {
      DQ_RET(stack_right(ctx, g, j));
      DQ_RET(recompute(ctx, g, j));
      DQ_RET(drift_reset<T>(ctx, g));
      if (measure)
        DQ_LAUNCH_C(ctx, kTMisc, launch_observables(g.G64, g.C, g.p.Lx, g.p.Ly, g.p.t, g.obs, g.spin,
                                                       g.st));
      ++j;
    }
  }
  return DQMC_OK;
}

int sweep_group(dqmc_ctx* ctx, Group& g, int measure) {
  if (g.p.precision == DQMC_FP32)
    DQ_RET(up_pass<float>(ctx, g, measure));
  else if (g.p.precision == DQMC_DF32)
    DQ_RET(up_pass<df32>(ctx, g, measure));
  else
    DQ_RET(up_pass<double>(ctx, g, measure));
  return left_pass(ctx, g);
}

int check_status(dqmc_ctx* ctx) {
  DQ_CK(cudaStreamSynchronize(ctx->st));
  int s = 0;
  DQ_CK(cudaMemcpy(&s, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (s == kDevTimeout) return DQMC_ERR_TIMEOUT;
  if (s != 0) return DQMC_ERR_NAN;
  return DQMC_OK;
}

// Stabilised matrices at all stabilisation points of every chain:
// Mid^{-1} in g.A2 and W1 = U_L Db_L^{-1} Mid^{-1} in g.W1 (g.Mid is overwritten).
// pair: invert the middle matrices in float pairs (G(tau) of float-pair
// groups, where log|det| is not needed); FP64 otherwise.
int all_points_w1(dqmc_ctx* ctx, Group& g, bool pair) {
  const int batch = g.C * (g.nc + 1);
  DQ_RET(form_mid(ctx, g, 0, g.nn(), batch, g.Mid));
  DQ_CLASS(ctx, pair ? kTInversePair : kTInverse);
  DQ_LAUNCH(ctx, launch_gj_cluster(g.Mid, g.nn(), g.A2, g.nn(), g.N, batch, pair ? nullptr : g.logabs,
                                   ctx->d_status, g.st, pair));
  GemmArgs m = gemm0(g.N);
  m.A = g.LU; m.sA = g.nn(); m.tA = 1;
  m.ks = g.LD; m.sks = g.N; m.ks_mode = 2;
  m.ks_on_b = 1;  // as in recompute: the scale goes with the rows of Mid^{-1}
  m.balance = 1;
  m.B = g.A2; m.sB = g.nn();
  m.C = g.W1; m.sC = g.nn();
  DQ_CLASS(ctx, kTGemm);
  DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
  return DQMC_OK;
}

void drop_graphs(dqmc_ctx* ctx) {
  for (int m = 0; m < 2; ++m) {
    if (ctx->gexec[m]) cudaGraphExecDestroy(ctx->gexec[m]);
    ctx->gexec[m] = nullptr;
  }
}

// Capture one sweep of every group (each on its own branch, forked from and
// joined into cap_main) followed by the sweep-counter increment.
int build_sweep_graph(dqmc_ctx* ctx, int m) {
  DQ_CK(cudaStreamBeginCapture(ctx->cap_main, cudaStreamCaptureModeRelaxed));
  const long long l0 = ctx->launches;
  int rc = DQMC_OK;
  if (cudaEventRecord(ctx->fork, ctx->cap_main) != cudaSuccess) rc = DQMC_ERR_CUDA;
  for (Group& g : ctx->g) {
    if (rc != DQMC_OK) break;
    if (cudaStreamWaitEvent(g.cap, ctx->fork, 0) != cudaSuccess) {
      rc = DQMC_ERR_CUDA;
      break;
    }
    g.st = g.cap;
    rc = sweep_group(ctx, g, m);
    g.st = ctx->st;
    if (rc == DQMC_OK && (cudaEventRecord(g.join, g.cap) != cudaSuccess ||
                          cudaStreamWaitEvent(ctx->cap_main, g.join, 0) != cudaSuccess))
      rc = DQMC_ERR_CUDA;
  }
  if (rc == DQMC_OK) {
    ++ctx->launches;
    k_increment<<<1, 1, 0, ctx->cap_main>>>(ctx->d_sweep);
    if (cudaGetLastError() != cudaSuccess) rc = DQMC_ERR_CUDA;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(ctx->cap_main, &graph);
  for (Group& g : ctx->g) g.st = ctx->st;
  if (rc == DQMC_OK && ec != cudaSuccess) {
    g_last_cuda = ec;
    g_last_line = __LINE__;
    rc = DQMC_ERR_CUDA;
  }
  if (rc == DQMC_OK) {
    const cudaError_t ei = cudaGraphInstantiate(&ctx->gexec[m], graph, 0);
    if (ei != cudaSuccess) {
      g_last_cuda = ei;
      g_last_line = __LINE__;
      ctx->gexec[m] = nullptr;
      rc = DQMC_ERR_CUDA;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  ctx->graph_launches[m] = ctx->launches - l0;
  ctx->launches = l0;
  return rc;
}

int validate(const dqmc_group& p) {
  if (p.Lx < 2 || p.Ly < 2 || p.Lx > DQMC_MAX_SIDE || p.Ly > DQMC_MAX_SIDE) return DQMC_ERR_ARG;
  if ((p.Lx & 1) || (p.Ly & 1)) return DQMC_ERR_ARG;
  if (!(p.dtau > 0.0) || !(p.beta > 0.0) || !(p.U >= 0.0) || !std::isfinite(p.t)) return DQMC_ERR_ARG;
  const double r = p.beta / p.dtau;
  const long long L = std::llround(r);
  if (L < 1 || std::fabs(r - static_cast<double>(L)) > 1e-9 || L > 100000) return DQMC_ERR_ARG;
  if (p.n_chains < 1 || p.stab_interval < 1 || p.delay_k < 1 || p.delay_k > DQMC_MAX_DELAY)
    return DQMC_ERR_ARG;
  if (p.precision != DQMC_FP64 && p.precision != DQMC_FP32 && p.precision != DQMC_DF32)
    return DQMC_ERR_ARG;
  return DQMC_OK;
}

int setup_group(dqmc_ctx* ctx, Group& g) {
  const dqmc_group& p = g.p;
  g.N = p.Lx * p.Ly;
  g.L = static_cast<int>(std::llround(p.beta / p.dtau));
  g.C = p.n_chains;
  g.lam = std::acosh(std::exp(0.5 * p.dtau * p.U));
  g.cp.clear();
  for (int j = 0;; ++j) {
    const int c = std::min(j * p.stab_interval, g.L);
    g.cp.push_back(c);
    if (c == g.L) break;
  }
  g.nc = static_cast<int>(g.cp.size()) - 1;
  ring_taps(p.Lx, p.t, p.dtau, g.taps.ex, g.taps.exi);
  ring_taps(p.Ly, p.t, p.dtau, g.taps.ey, g.taps.eyi);
  const size_t C = g.C, N = g.N, NN = N * N, S = static_cast<size_t>(g.nc + 1);
  const size_t tsz = p.precision == DQMC_FP32 ? 4 : 8;  // df32 and double: 8 bytes
  DQ_RET(dev_alloc(ctx, &g.field, C * g.L * N));
  DQ_RET(dev_alloc(ctx, &g.Gw, C * NN * tsz));
  DQ_RET(dev_alloc(ctx, &g.G64, C * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.RU, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.RT, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.RD, C * S * N * 8));
  DQ_RET(dev_alloc(ctx, &g.LU, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.LT, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.LD, C * S * N * 8));
  DQ_RET(dev_alloc(ctx, &g.X, C * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.Rtil, C * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.Mid, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.W1, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.W2, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.A1, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.A2, C * S * NN * 8));
  DQ_RET(dev_alloc(ctx, &g.logabs, C * S * 8));
  DQ_RET(dev_alloc(ctx, &g.obs, C * 4 * 8));
  DQ_RET(dev_alloc(ctx, &g.spin, C * N * 8));
  DQ_RET(dev_alloc(ctx, &g.drift, C * 8));
  DQ_RET(dev_alloc(ctx, &g.acc, C * 8));
  DQ_RET(dev_alloc(ctx, &g.bins, C * (g.L + 1) * 2 * N * 8));
  DQ_RET(dev_alloc(ctx, &g.gacc, C * 3 * 8));
  DQ_RET(dev_alloc(ctx, &g.gout, C * (g.L + 1) * N * 8));
  DQ_RET(dev_alloc(ctx, &g.qrs, C * 2 * N * 8));
  if (static_cast<int>(N) >= kOzakiMinN) {
    g.oz_batch = static_cast<int>(std::min<size_t>(C * S, 256));
    DQ_RET(dev_alloc(ctx, &g.oz, ozaki_scratch_bytes(static_cast<int>(N), g.oz_batch)));
    DQ_RET(dev_alloc(ctx, &g.qrb.W0, C * NN * 8));
    DQ_RET(dev_alloc(ctx, &g.qrb.W1, C * NN * 8));
    DQ_RET(dev_alloc(ctx, &g.qrb.Wt, C * N * 32 * 8));
    DQ_RET(dev_alloc(ctx, &g.qrb.perm, C * N * sizeof(int)));
    g.qrb.sW = static_cast<long long>(NN);
    g.qrb.sWt = static_cast<long long>(N) * 32;
  }
  std::vector<int> cpg = g.cp, cpd = g.cp;
  cpg.push_back(g.L + 1);
  cpd.push_back(g.L);
  DQ_RET(dev_alloc(ctx, &g.d_cp_gtau, cpg.size() * sizeof(int)));
  DQ_RET(dev_alloc(ctx, &g.d_cp_grad, cpd.size() * sizeof(int)));
  DQ_CK(cudaMemcpyAsync(g.d_cp_gtau, cpg.data(), cpg.size() * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->st));
  DQ_CK(cudaMemcpyAsync(g.d_cp_grad, cpd.data(), cpd.size() * sizeof(int), cudaMemcpyHostToDevice,
                        ctx->st));
  DQ_CK(cudaMemsetAsync(g.obs, 0, C * 4 * 8, ctx->st));
  DQ_CK(cudaMemsetAsync(g.spin, 0, C * N * 8, ctx->st));
  DQ_CK(cudaMemsetAsync(g.drift, 0, C * 8, ctx->st));
  DQ_CK(cudaMemsetAsync(g.acc, 0, C * 8, ctx->st));
  return DQMC_OK;
}

}  // namespace

extern "C" {

const char* dqmc_last_cuda_error(int* line) {
  if (line) *line = g_last_line;
  return cudaGetErrorString(g_last_cuda);
}

const char* dqmc_strerror(int code) {
  switch (code) {
    case DQMC_OK: return "ok";
    case DQMC_ERR_ARG: return "invalid argument";
    case DQMC_ERR_CUDA: return "CUDA error";
    case DQMC_ERR_OOM: return "device out of memory";
    case DQMC_ERR_DRIFT: return "Green-function drift above limit";
    case DQMC_ERR_TIMEOUT: return "device-side wait timed out";
    case DQMC_ERR_NAN: return "non-finite or singular value in a stabilised matrix";
    case DQMC_ERR_STATE: return "call not valid in the current state";
    default: return "unknown error";
  }
}

void dqmc_destroy(dqmc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  cudaDeviceSynchronize();
  drop_graphs(ctx);
  for (Group& g : ctx->g) {
    if (g.cap) cudaStreamDestroy(g.cap);
    if (g.join) cudaEventDestroy(g.join);
  }
  if (ctx->cap_main) cudaStreamDestroy(ctx->cap_main);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  for (void* p : ctx->allocs) cudaFree(p);
  delete ctx;
}

int dqmc_init(const dqmc_group* groups, int n_groups, uint64_t seed, void* stream, dqmc_ctx** out) {
  return dqmc_init_at(groups, n_groups, seed, 0, stream, out);
}

int dqmc_init_at(const dqmc_group* groups, int n_groups, uint64_t seed, int64_t chain_offset,
                 void* stream, dqmc_ctx** out) {
  if (!groups || n_groups < 1 || !out || chain_offset < 0) return DQMC_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n_groups; ++i) DQ_RET(validate(groups[i]));
  {  // every chain id must fit the (signed) chain index of the kernels
    int64_t total = chain_offset;
    for (int i = 0; i < n_groups; ++i) total += groups[i].n_chains;
    if (total > 0x7FFFFFFFLL) return DQMC_ERR_ARG;
  }
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
      prop.major * 10 + prop.minor < 100)
    return DQMC_ERR_CUDA;
  dqmc_ctx* ctx = new (std::nothrow) dqmc_ctx();
  if (!ctx) return DQMC_ERR_OOM;
  ctx->st = static_cast<cudaStream_t>(stream);
  ctx->seed = seed;
  ctx->chain_offset = chain_offset;
  ctx->nsm = prop.multiProcessorCount;
  ctx->g.resize(n_groups);
  int rc = dev_alloc(ctx, &ctx->d_sweep, sizeof(uint32_t));
  if (rc == DQMC_OK) rc = dev_alloc(ctx, &ctx->d_status, sizeof(int));
  if (rc == DQMC_OK) {
    if (cudaMemsetAsync(ctx->d_sweep, 0, sizeof(uint32_t), ctx->st) != cudaSuccess ||
        cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->st) != cudaSuccess)
      rc = DQMC_ERR_CUDA;
  }
  int chain0 = 0;
  for (int i = 0; i < n_groups && rc == DQMC_OK; ++i) {
    Group& g = ctx->g[i];
    g.p = groups[i];
    g.chain0 = chain0;
    g.st = ctx->st;
    rc = setup_group(ctx, g);
    chain0 += g.C;
    if (rc == DQMC_OK) {
      ++ctx->launches;
      const cudaError_t e = launch_init_field(g.field, g.C, g.L, g.N,
                                              static_cast<int>(g.chain0 + chain_offset), seed, ctx->st);
      if (e != cudaSuccess) {
        g_last_cuda = e;
        g_last_line = __LINE__;
        rc = DQMC_ERR_CUDA;
      }
    }
    if (rc == DQMC_OK) rc = rebuild(ctx, g);
    if (rc == DQMC_OK) rc = load_working(ctx, g);
  }
  ctx->total = chain0;
  if (rc == DQMC_OK) {
    if (cudaStreamCreateWithFlags(&ctx->cap_main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming) != cudaSuccess)
      rc = DQMC_ERR_CUDA;
    for (Group& g : ctx->g) {
      g.st = ctx->st;
      if (rc == DQMC_OK && (cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking) != cudaSuccess ||
                            cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess))
        rc = DQMC_ERR_CUDA;
    }
  }
  if (rc == DQMC_OK) rc = check_status(ctx);
  if (rc != DQMC_OK) {
    dqmc_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return DQMC_OK;
}

int dqmc_sweep(dqmc_ctx* ctx, int n_sweeps, int measure) {
  if (!ctx || n_sweeps < 0) return DQMC_ERR_ARG;
  const int m = measure ? 1 : 0;
  if (ctx->timing || !ctx->use_graph) {
    for (int s = 0; s < n_sweeps; ++s) {
      for (Group& g : ctx->g) DQ_RET(sweep_group(ctx, g, m));
      DQ_CLASS(ctx, kTMisc);
      DQ_LAUNCH(ctx, (k_increment<<<1, 1, 0, ctx->st>>>(ctx->d_sweep), cudaGetLastError()));
    }
    return DQMC_OK;
  }
  if (n_sweeps > 0 && !ctx->gexec[m]) DQ_RET(build_sweep_graph(ctx, m));
  for (int s = 0; s < n_sweeps; ++s) {
    DQ_CK(cudaGraphLaunch(ctx->gexec[m], ctx->st));
    ctx->launches += ctx->graph_launches[m];
  }
  return DQMC_OK;
}

int dqmc_autotune(const dqmc_group* groups, int n_groups, double drift_target, uint64_t seed,
                  void* stream, dqmc_group* out) {
  if (!groups || n_groups < 1 || !out || !(drift_target > 0.0)) return DQMC_ERR_ARG;
  for (int i = 0; i < n_groups; ++i) DQ_RET(validate(groups[i]));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int gi = 0; gi < n_groups; ++gi) {
    const dqmc_group& g = groups[gi];
    const int L = static_cast<int>(std::llround(g.beta / g.dtau));
    // Candidate stabilisation intervals, largest first (at most 64 slices,
    // beyond which the unstabilised B products lose all small scales); all
    // probed at once, each as its own group.
    std::vector<int> cands;
    for (int ns : {L, 64, 48, 40, 32, 25, 20, 16, 12, 10, 8, 6, 5, 4, 3, 2})
      if (ns <= L && ns <= 64 && ns >= 2 && (cands.empty() || ns < cands.back()))
        cands.push_back(ns);
    if (cands.empty()) cands.push_back(1);
    std::vector<dqmc_group> probe;
    std::vector<double> drift;
    int rc = DQMC_OK;
    // A candidate so large that its G overflows sets the context's non-finite
    // status for every probe; it is too large by definition, so the largest
    // candidate is dropped and the rest probed again.
    while (true) {
      probe.clear();
      for (int ns : cands) {
        dqmc_group p = g;
        p.n_chains = std::min(g.n_chains, 4);
        p.stab_interval = ns;
        probe.push_back(p);
      }
      dqmc_ctx* pc = nullptr;
      rc = dqmc_init(probe.data(), static_cast<int>(probe.size()), seed, stream, &pc);
      if (rc == DQMC_OK) {
        rc = dqmc_sweep(pc, 2, 0);
        if (rc == DQMC_OK) rc = dqmc_reset_stats(pc);
        if (rc == DQMC_OK) rc = dqmc_sweep(pc, 3, 0);
        drift.assign(pc->total, 0.0);
        if (rc == DQMC_OK) rc = dqmc_get_stats(pc, drift.data(), nullptr);
        dqmc_destroy(pc);
      }
      if (rc != DQMC_ERR_NAN || cands.size() <= 1) break;
      cands.erase(cands.begin());
    }
    DQ_RET(rc);
    int chosen = 1;
    for (size_t c = 0; c < cands.size(); ++c) {
      const int per = probe[c].n_chains;
      double dmax = 0.0;
      for (int q = 0; q < per; ++q) dmax = std::max(dmax, drift[c * per + q]);
      // The drift over chains and sweeps is heavy-tailed: a probe of a few
      // chains must sit well below the target to keep a long run under it.
      if (dmax <= kTuneMargin * drift_target) {
        chosen = cands[c];
        break;
      }
    }
    // Delay depth: fastest of 8, 16, 32 at the chosen interval.
    dqmc_group best = g;
    best.stab_interval = chosen;
    float best_ms = 0.0f;
    for (int k : {8, 16, 32}) {
      dqmc_group p = best;
      p.delay_k = k;
      p.n_chains = std::min(g.n_chains, 8);
      dqmc_ctx* kc = nullptr;
      DQ_RET(dqmc_init(&p, 1, seed, stream, &kc));
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      float ms = 0.0f;
      int r = dqmc_sweep(kc, 1, 0);
      if (r == DQMC_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        r = DQMC_ERR_CUDA;
      if (r == DQMC_OK) {
        cudaEventRecord(e0, st);
        r = dqmc_sweep(kc, 2, 0);
        cudaEventRecord(e1, st);
        if (r == DQMC_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          r = DQMC_ERR_CUDA;
      }
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      dqmc_destroy(kc);
      DQ_RET(r);
      if (best_ms == 0.0f || ms < best_ms) {
        best_ms = ms;
        best.delay_k = k;
      }
    }
    out[gi] = best;
  }
  return DQMC_OK;
}

namespace {
bool tile_ok(int v, int N) {
  return v == 0 || ((v == 1 || v == 2 || v == 4 || v == 8 || v == 16) && v <= N);
}
}  // namespace

int dqmc_set_tiles(dqmc_ctx* ctx, int group, const dqmc_tiles* t) {
  if (!ctx || !t || group < 0 || group >= static_cast<int>(ctx->g.size())) return DQMC_ERR_ARG;
  Group& g = ctx->g[group];
  if (!tile_ok(t->kron_nv, g.N) || !tile_ok(t->wrap_nv, g.N)) return DQMC_ERR_ARG;
  if (t->metro_ctas != 0 && t->metro_ctas != 1 && t->metro_ctas != 2 && t->metro_ctas != 4)
    return DQMC_ERR_ARG;
  if (t->metro_ctas > 1 && g.N < 4 * t->metro_ctas) return DQMC_ERR_ARG;
  if (g.tile_kron != t->kron_nv || g.tile_wrap != t->wrap_nv || g.tile_metro != t->metro_ctas)
    drop_graphs(ctx);
  g.tile_kron = t->kron_nv;
  g.tile_wrap = t->wrap_nv;
  g.tile_metro = t->metro_ctas;
  return DQMC_OK;
}

int dqmc_get_tiles(const dqmc_ctx* ctx, int group, dqmc_tiles* out) {
  if (!ctx || !out || group < 0 || group >= static_cast<int>(ctx->g.size())) return DQMC_ERR_ARG;
  const Group& g = ctx->g[group];
  out->kron_nv = kron_nv(g, true);
  if (g.p.precision == DQMC_FP32)
    out->wrap_nv = wrap_nv<float>(g);
  else if (g.p.precision == DQMC_DF32)
    out->wrap_nv = wrap_nv<df32>(g);
  else
    out->wrap_nv = wrap_nv<double>(g);
  int cs = g.tile_metro > 0 ? g.tile_metro : ctx->metro_cs;
  if (cs == 0) {
    cs = 1;
    for (int c : {4, 2})
      if (static_cast<long long>(c) * ctx->total <= ctx->nsm && g.N >= 4 * c) {
        cs = c;
        break;
      }
  }
  out->metro_ctas = cs;
  return DQMC_OK;
}

int dqmc_autotune_tiles(const dqmc_group* groups, int n_groups, uint64_t seed, void* stream,
                        dqmc_tiles* out) {
  if (!groups || n_groups < 1 || !out) return DQMC_ERR_ARG;
  for (int i = 0; i < n_groups; ++i) DQ_RET(validate(groups[i]));
  // Each class of kernels depends on one tile parameter only (metropolis on
  // the CTAs per chain, wrap on wrap_nv, the FP64 Kronecker classes on
  // kron_nv), so one timed sweep per candidate index tunes all three.
  const int kron_c[3] = {2, 4, 8}, wrap_c[3] = {2, 4, 8}, metro_c[3] = {1, 2, 4};
  for (int gi = 0; gi < n_groups; ++gi) {
    dqmc_ctx* pc = nullptr;
    DQ_RET(dqmc_init(&groups[gi], 1, seed, stream, &pc));
    const int N = pc->g[0].N;
    double best[3] = {1e300, 1e300, 1e300};
    dqmc_tiles pick{0, 0, 0};
    int rc = dqmc_sweep(pc, 1, 0);  // warm-up (and graph-free first launches)
    for (int c = 0; c < 3 && rc == DQMC_OK; ++c) {
      dqmc_tiles t{std::min(kron_c[c], N), std::min(wrap_c[c], N),
                   N >= 4 * metro_c[c] ? metro_c[c] : 1};
      rc = dqmc_set_tiles(pc, 0, &t);
      if (rc == DQMC_OK) rc = dqmc_timing_enable(pc, 1);
      if (rc == DQMC_OK) rc = dqmc_timing_reset(pc);
      if (rc == DQMC_OK) rc = dqmc_sweep(pc, 1, 0);
      double ms[kTNumClasses] = {};
      if (rc == DQMC_OK && dqmc_timing_read(pc, ms, nullptr, kTNumClasses) < 0) rc = DQMC_ERR_CUDA;
      if (rc == DQMC_OK) rc = dqmc_timing_enable(pc, 0);
      if (rc != DQMC_OK) break;
      const double tm = ms[kTMetropolis], tw = ms[kTWrap], tk = ms[kTStackKron];
      if (tk < best[0]) { best[0] = tk; pick.kron_nv = t.kron_nv; }
      if (tw < best[1]) { best[1] = tw; pick.wrap_nv = t.wrap_nv; }
      if (tm < best[2]) { best[2] = tm; pick.metro_ctas = t.metro_ctas; }
    }
    if (rc == DQMC_OK) rc = check_status(pc);
    dqmc_destroy(pc);
    DQ_RET(rc);
    out[gi] = pick;
  }
  return DQMC_OK;
}

int dqmc_use_graphs(dqmc_ctx* ctx, int on) {
  if (!ctx) return DQMC_ERR_ARG;
  ctx->use_graph = on != 0;
  return DQMC_OK;
}

int dqmc_recompute_G(dqmc_ctx* ctx, double* max_drift_out) {
  if (!ctx) return DQMC_ERR_ARG;
  std::vector<double> saved;
  int off = 0;
  for (Group& g : ctx->g) {
    DQ_CK(cudaMemsetAsync(g.drift, 0, g.C * sizeof(double), ctx->st));
    DQ_RET(rebuild(ctx, g));
    DQ_RET(drift_reset_any(ctx, g));
    if (max_drift_out)
      DQ_CK(cudaMemcpyAsync(max_drift_out + off, g.drift, g.C * sizeof(double),
                            cudaMemcpyDeviceToHost, ctx->st));
    off += g.C;
  }
  return check_status(ctx);
}

int64_t dqmc_gtau_size(const dqmc_ctx* ctx) {
  if (!ctx) return DQMC_ERR_ARG;
  int64_t s = 0;
  for (const Group& g : ctx->g) s += static_cast<int64_t>(g.C) * (g.L + 1) * g.N;
  return s;
}

// G_k(tau_l) of every chain of group g, from its current stacks, into the
// device array dst [C][L+1][N].
int measure_gtau_group(dqmc_ctx* ctx, Group& g, double* dst) {
  {
    const int batch = g.C * (g.nc + 1);
    DQ_RET(all_points_w1(ctx, g, g.p.precision == DQMC_DF32));
    // G(c,0)^T = T_R^T Ds_R W1^T  and  W2 = T_L^T Ds_L Mid^{-1}, Y = W2 Db_R^{-1} U_R^T
    GemmArgs m = gemm0(g.N);
    m.A = g.RT; m.sA = g.nn(); m.tA = 1;
    m.ks = g.RD; m.sks = g.N; m.ks_mode = 3;
    m.B = g.W1; m.sB = g.nn(); m.tB = 1;
    m.C = g.A1; m.sC = g.nn();
    DQ_CLASS(ctx, kTGemm);
    DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
    m = gemm0(g.N);
    m.A = g.LT; m.sA = g.nn(); m.tA = 1;
    m.ks = g.LD; m.sks = g.N; m.ks_mode = 3;
    m.B = g.A2; m.sB = g.nn();
    m.C = g.W2; m.sC = g.nn();
    DQ_CLASS(ctx, kTGemm);
    DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
    m = gemm0(g.N);
    m.A = g.W2; m.sA = g.nn();
    m.ks = g.RD; m.sks = g.N; m.ks_mode = 2;
    m.B = g.RU; m.sB = g.nn();
    m.C = g.A2; m.sC = g.nn();
    DQ_CLASS(ctx, kTGemm);
    DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
    const long long nb = static_cast<long long>(g.C) * (g.L + 1) * 2 * g.N;
    DQ_CLASS(ctx, kTMisc);
    DQ_LAUNCH(ctx, (k_zero<<<static_cast<int>(std::min<long long>((nb + 255) / 256, 1024)), 256, 0,
                             g.st>>>(g.bins, nb),
                    cudaGetLastError()));
    GtauArgs ga{};
    ga.N = g.N; ga.Lx = g.p.Lx; ga.Ly = g.p.Ly; ga.L = g.L;
    // float-pair groups propagate in their working precision (small tiles,
    // latency-bound like the wrap); FP64 and FP32 groups in FP64
    const bool pair = g.p.precision == DQMC_DF32;
    ga.nv = pair ? (g.tile_wrap > 0 ? std::min(2 * g.tile_wrap, g.N) : std::min(8, g.N))
                 : kron_nv(g, true);
    ga.per_chain = g.nc + 1;
    ga.c = g.lam;
    ga.ec = std::exp(g.lam);
    ga.emc = std::exp(-g.lam);
    ga.taps = g.taps;
    ga.field = g.field;
    ga.cp = g.d_cp_gtau;
    ga.mat_stride = g.nn();
    ga.bins = g.bins;
    // FP64 groups on the tensor cores where the tensor-core products are in
    // use (measured faster than the FP64 pipe); float-pair groups keep their
    // float-pair propagation, which measured faster than the tensor path
    const bool tc = ctx->gemm_mode == DQMC_GEMM_TENSOR && g.oz && !pair;
    ga.kind = kB; ga.vec_is_col = 1; ga.bin_slot = 0;
    DQ_CLASS(ctx, kTGtauProp);
    DQ_LAUNCH(ctx, tc ? launch_gtau_tc(g.A1, batch, ga, ctx->d_status, g.st)
                      : launch_gtau_propagate(g.A1, batch, ga, pair, g.st));
    ga.kind = kBIT; ga.vec_is_col = 0; ga.bin_slot = 1;
    DQ_CLASS(ctx, kTGtauProp);
    DQ_LAUNCH(ctx, tc ? launch_gtau_tc(g.A2, batch, ga, ctx->d_status, g.st)
                      : launch_gtau_propagate(g.A2, batch, ga, pair, g.st));
    DQ_CLASS(ctx, kTGtauFinal);
    DQ_LAUNCH(ctx, launch_gtau_finalize(g.bins, dst, g.C, g.L, g.p.Lx, g.p.Ly, g.st));
  }
  return DQMC_OK;
}

int dqmc_measure_Gtau(dqmc_ctx* ctx, double* out, int out_on_device) {
  if (!ctx || !out) return DQMC_ERR_ARG;
  size_t off = 0;
  for (Group& g : ctx->g) {
    const size_t cnt = static_cast<size_t>(g.C) * (g.L + 1) * g.N;
    if (out_on_device) {
      DQ_RET(measure_gtau_group(ctx, g, out + off));
    } else {
      DQ_RET(measure_gtau_group(ctx, g, g.gout));
      DQ_CK(cudaMemcpyAsync(out + off, g.gout, cnt * sizeof(double), cudaMemcpyDeviceToHost, g.st));
    }
    off += cnt;
  }
  if (!out_on_device) return check_status(ctx);
  return DQMC_OK;
}

int dqmc_measure_Gtau_origins(dqmc_ctx* ctx, int n_origins, double* out, int out_on_device) {
  if (!ctx || !out || n_origins < 1) return DQMC_ERR_ARG;
  for (const Group& g : ctx->g)
    if (n_origins > g.L) return DQMC_ERR_ARG;
  size_t off = 0;
  for (Group& g : ctx->g) {
    const size_t cnt = static_cast<size_t>(g.C) * (g.L + 1) * g.N;
    const long long nf = static_cast<long long>(g.C) * g.L * g.N;
    int8_t* saved = nullptr;
    double* acc = nullptr;
    if (cudaMalloc(&saved, nf) != cudaSuccess ||
        (!out_on_device && cudaMalloc(&acc, cnt * sizeof(double)) != cudaSuccess)) {
      cudaGetLastError();
      if (saved) cudaFree(saved);
      return DQMC_ERR_OOM;
    }
    if (out_on_device) acc = out + off;
    const int blocks = static_cast<int>(std::min<long long>((static_cast<long long>(cnt) + 255) / 256, 1024));
    int rc = DQMC_OK;
    auto run = [&]() -> int {
      DQ_CK(cudaMemcpyAsync(saved, g.field, nf, cudaMemcpyDeviceToDevice, g.st));
      DQ_CLASS(ctx, kTMisc);
      DQ_LAUNCH(ctx, (k_zero<<<blocks, 256, 0, g.st>>>(acc, static_cast<long long>(cnt)),
                      cudaGetLastError()));
      bool rotated = false;
      for (int o = 0; o < n_origins; ++o) {
        const int s = static_cast<int>((static_cast<long long>(o) * g.L) / n_origins);
        if (s != 0) {  // the field rotated by s slices, and its stacks
          DQ_CLASS(ctx, kTMisc);
          DQ_LAUNCH(ctx, (k_rotate_field<<<static_cast<int>(std::min<long long>((nf + 255) / 256, 1024)),
                                           256, 0, g.st>>>(saved, g.field, g.C, g.L, g.N, s),
                          cudaGetLastError()));
          DQ_RET(rebuild(ctx, g));
          rotated = true;
        }
        DQ_RET(measure_gtau_group(ctx, g, g.gout));
        DQ_CLASS(ctx, kTMisc);
        DQ_LAUNCH(ctx, (k_axpy<<<blocks, 256, 0, g.st>>>(acc, g.gout, 1.0 / n_origins,
                                                           static_cast<long long>(cnt)),
                        cudaGetLastError()));
      }
      if (rotated) {  // the chain's own field and freshly stabilised stacks and G
        DQ_CK(cudaMemcpyAsync(g.field, saved, nf, cudaMemcpyDeviceToDevice, g.st));
        DQ_RET(rebuild(ctx, g));
        DQ_RET(load_working(ctx, g));
      }
      if (!out_on_device)
        DQ_CK(cudaMemcpyAsync(out + off, acc, cnt * sizeof(double), cudaMemcpyDeviceToHost, g.st));
      DQ_CK(cudaStreamSynchronize(g.st));
      return DQMC_OK;
    };
    rc = run();
    if (rc != DQMC_OK) {
      // Best effort: give the chains their own field back, ordered after any
      // rotation still queued on the group's stream, and rebuild the stacks
      // and G from it.  If this fails too, the context needs
      // dqmc_recompute_G (or dqmc_set_field) before further sweeps.
      cudaStreamSynchronize(g.st);
      cudaGetLastError();
      if (cudaMemcpyAsync(g.field, saved, nf, cudaMemcpyDeviceToDevice, g.st) == cudaSuccess &&
          rebuild(ctx, g) == DQMC_OK && load_working(ctx, g) == DQMC_OK)
        cudaStreamSynchronize(g.st);
    }
    cudaFree(saved);
    if (!out_on_device) cudaFree(acc);
    if (rc != DQMC_OK) return rc;
    off += cnt;
  }
  return check_status(ctx);
}

int dqmc_grad(dqmc_ctx* ctx, double* dlogW_dt, double* dlogW_dlambda, double* logW,
              int out_on_device) {
  if (!ctx) return DQMC_ERR_ARG;
  int off = 0;
  for (Group& g : ctx->g) {
    const int batch = g.C * (g.nc + 1);
    DQ_RET(all_points_w1(ctx, g, false));
    // G at every stabilisation point: W1 Db_R^{-1} U_R^T
    GemmArgs m = gemm0(g.N);
    m.A = g.W1; m.sA = g.nn();
    m.ks = g.RD; m.sks = g.N; m.ks_mode = 2;
    m.B = g.RU; m.sB = g.nn();
    m.C = g.A1; m.sC = g.nn();
    DQ_CLASS(ctx, kTGemm);
    DQ_LAUNCH(ctx, gemm(ctx, g, m, batch));
    DQ_CK(cudaMemsetAsync(g.gacc, 0, g.C * 3 * sizeof(double), g.st));
    int maxlen = 0;
    for (int j = 0; j < g.nc; ++j) maxlen = std::max(maxlen, g.cp[j + 1] - g.cp[j]);
    KronArgs wl = kron_base(g, kB, kron_nv(g, true));
    KronArgs wr = kron_base(g, kBIT, kron_nv(g, true));
    wl.per_chain = wr.per_chain = g.nc + 1;
    wl.cp = wr.cp = g.d_cp_grad;
    for (int step = 0; step < maxlen; ++step) {
      DQ_CLASS(ctx, kTGrad);
      DQ_LAUNCH(ctx, launch_grad_terms(g.A1, g.nn(), g.nc + 1, g.d_cp_grad, step, g.p.Lx, g.p.Ly,
                                       g.L, g.field, g.p.dtau, g.gacc, batch, g.st));
      if (step + 1 < maxlen) {
        wl.step = wr.step = step;
        DQ_CLASS(ctx, kTGrad);
        DQ_LAUNCH(ctx, launch_kron_cols<double>(g.A1, batch, wl, g.st));
        DQ_CLASS(ctx, kTGrad);
        DQ_LAUNCH(ctx, launch_kron_rows<double>(g.A1, g.A1, batch, wr, g.st));
      }
    }
    // results into W2 scratch: [0, C) dt, [C, 2C) dlambda, [2C, 3C) logW
    double* tmp = g.W2;
    DQ_CLASS(ctx, kTMisc);
    DQ_LAUNCH(ctx, (k_pick3<<<1, 256, 0, g.st>>>(g.gacc, tmp, tmp + g.C, g.C), cudaGetLastError()));
    DQ_CLASS(ctx, kTMisc);
    DQ_LAUNCH(ctx, (k_logw<<<g.C, 256, 0, g.st>>>(g.LD, static_cast<long long>(g.nc + 1) * g.N,
                                                      g.logabs, g.nc + 1, g.field, g.L, g.N, g.lam,
                                                      tmp + 2 * g.C),
                    cudaGetLastError()));
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (dlogW_dt) DQ_CK(cudaMemcpyAsync(dlogW_dt + off, tmp, g.C * 8, kind, g.st));
    if (dlogW_dlambda) DQ_CK(cudaMemcpyAsync(dlogW_dlambda + off, tmp + g.C, g.C * 8, kind, g.st));
    if (logW) DQ_CK(cudaMemcpyAsync(logW + off, tmp + 2 * g.C, g.C * 8, kind, g.st));
    off += g.C;
  }
  if (!out_on_device) return check_status(ctx);
  return DQMC_OK;
}

int64_t dqmc_field_size(const dqmc_ctx* ctx) {
  if (!ctx) return DQMC_ERR_ARG;
  int64_t s = 0;
  for (const Group& g : ctx->g) s += static_cast<int64_t>(g.C) * g.L * g.N;
  return s;
}

int dqmc_get_field(const dqmc_ctx* ctx, int8_t* out) {
  if (!ctx || !out) return DQMC_ERR_ARG;
  size_t off = 0;
  for (const Group& g : ctx->g) {
    const size_t n = static_cast<size_t>(g.C) * g.L * g.N;
    DQ_CK(cudaMemcpyAsync(out + off, g.field, n, cudaMemcpyDeviceToHost, ctx->st));
    off += n;
  }
  DQ_CK(cudaStreamSynchronize(ctx->st));
  return DQMC_OK;
}

int dqmc_set_field(dqmc_ctx* ctx, const int8_t* in) {
  if (!ctx || !in) return DQMC_ERR_ARG;
  const int64_t total = dqmc_field_size(ctx);
  for (int64_t e = 0; e < total; ++e)
    if (in[e] != 1 && in[e] != -1) return DQMC_ERR_ARG;
  size_t off = 0;
  for (Group& g : ctx->g) {
    const size_t n = static_cast<size_t>(g.C) * g.L * g.N;
    DQ_CK(cudaMemcpyAsync(g.field, in + off, n, cudaMemcpyHostToDevice, ctx->st));
    off += n;
    DQ_RET(rebuild(ctx, g));
    DQ_RET(load_working(ctx, g));
  }
  return check_status(ctx);
}

int dqmc_get_G(const dqmc_ctx* ctx, int chain, int spin, double* out) {
  if (!ctx || !out || chain < 0 || chain >= ctx->total || (spin != 0 && spin != 1))
    return DQMC_ERR_ARG;
  for (const Group& g : ctx->g) {
    if (chain >= g.chain0 + g.C) continue;
    const int c = chain - g.chain0;
    DQ_CK(cudaMemcpyAsync(out, g.G64 + c * g.nn(), g.nn() * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->st));
    DQ_CK(cudaStreamSynchronize(ctx->st));
    if (spin == 1) {
      const int N = g.N, Lx = g.p.Lx;
      std::vector<double> up(out, out + g.nn());
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
          const int pij = ((i % Lx + i / Lx + j % Lx + j / Lx) & 1) ? -1 : 1;
          out[static_cast<size_t>(i) * N + j] =
              (i == j ? 1.0 : 0.0) - pij * up[static_cast<size_t>(j) * N + i];
        }
    }
    return DQMC_OK;
  }
  return DQMC_ERR_ARG;
}

int dqmc_get_observables(const dqmc_ctx* ctx, double* out) {
  if (!ctx || !out) return DQMC_ERR_ARG;
  size_t off = 0;
  for (const Group& g : ctx->g) {
    DQ_CK(cudaMemcpyAsync(out + off, g.obs, g.C * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                          ctx->st));
    off += static_cast<size_t>(g.C) * 4;
  }
  DQ_CK(cudaStreamSynchronize(ctx->st));
  return DQMC_OK;
}

int dqmc_reset_observables(dqmc_ctx* ctx) {
  if (!ctx) return DQMC_ERR_ARG;
  for (Group& g : ctx->g) {
    DQ_CK(cudaMemsetAsync(g.obs, 0, g.C * 4 * sizeof(double), ctx->st));
    DQ_CK(cudaMemsetAsync(g.spin, 0, static_cast<size_t>(g.C) * g.N * sizeof(double), ctx->st));
  }
  return DQMC_OK;
}

int64_t dqmc_spin_correlation_size(const dqmc_ctx* ctx) {
  if (!ctx) return -1;
  int64_t n = 0;
  for (const Group& g : ctx->g) n += static_cast<int64_t>(g.C) * g.N;
  return n;
}

int dqmc_get_spin_correlation(const dqmc_ctx* ctx, double* out) {
  if (!ctx || !out) return DQMC_ERR_ARG;
  size_t off = 0;
  for (const Group& g : ctx->g) {
    const size_t n = static_cast<size_t>(g.C) * g.N;
    DQ_CK(cudaMemcpyAsync(out + off, g.spin, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    off += n;
  }
  DQ_CK(cudaStreamSynchronize(ctx->st));
  return DQMC_OK;
}

int dqmc_correlation_length(dqmc_ctx* ctx, double dmax, double* xi, int out_on_device) {
  if (!ctx || !xi || !(dmax > 0.0)) return DQMC_ERR_ARG;
  const int ng = static_cast<int>(ctx->g.size());
  // per group: C + 1 results (chains, then the chain average), staged in the
  // group's G(tau) buffer and copied to the caller's layout
  size_t chain_off = 0;
  for (int gi = 0; gi < ng; ++gi) {
    Group& g = ctx->g[gi];
    DQ_LAUNCH_C(ctx, kTMisc, launch_corr_length(g.spin, g.obs, g.C, g.p.Lx, g.p.Ly, dmax, g.gout,
                                                  ctx->st));
    const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    DQ_CK(cudaMemcpyAsync(xi + chain_off, g.gout, g.C * sizeof(double), kind, ctx->st));
    DQ_CK(cudaMemcpyAsync(xi + ctx->total + gi, g.gout + g.C, sizeof(double), kind, ctx->st));
    chain_off += g.C;
  }
  if (!out_on_device) DQ_CK(cudaStreamSynchronize(ctx->st));
  return DQMC_OK;
}

int dqmc_get_stats(const dqmc_ctx* ctx, double* max_drift, uint64_t* accepted) {
  if (!ctx) return DQMC_ERR_ARG;
  size_t off = 0;
  for (const Group& g : ctx->g) {
    if (max_drift)
      DQ_CK(cudaMemcpyAsync(max_drift + off, g.drift, g.C * sizeof(double), cudaMemcpyDeviceToHost,
                            ctx->st));
    if (accepted)
      DQ_CK(cudaMemcpyAsync(accepted + off, g.acc, g.C * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            ctx->st));
    off += g.C;
  }
  return check_status(const_cast<dqmc_ctx*>(ctx));
}

int dqmc_reset_stats(dqmc_ctx* ctx) {
  if (!ctx) return DQMC_ERR_ARG;
  for (Group& g : ctx->g) {
    DQ_CK(cudaMemsetAsync(g.drift, 0, g.C * sizeof(double), ctx->st));
    DQ_CK(cudaMemsetAsync(g.acc, 0, g.C * sizeof(uint64_t), ctx->st));
  }
  return DQMC_OK;
}

int dqmc_num_chains(const dqmc_ctx* ctx) { return ctx ? ctx->total : DQMC_ERR_ARG; }

int64_t dqmc_launch_count(const dqmc_ctx* ctx) { return ctx ? ctx->launches : DQMC_ERR_ARG; }

int dqmc_set_gemm_mode(dqmc_ctx* ctx, int mode) {
  if (!ctx || (mode != DQMC_GEMM_TENSOR && mode != DQMC_GEMM_FP64)) return DQMC_ERR_ARG;
  if (ctx->gemm_mode != mode) drop_graphs(ctx);
  ctx->gemm_mode = mode;
  return DQMC_OK;
}

int dqmc_set_qr_mode(dqmc_ctx* ctx, int mode) {
  if (!ctx || (mode != DQMC_QR_BLOCKED && mode != DQMC_QR_PIVOTED)) return DQMC_ERR_ARG;
  if (ctx->qr_mode != mode) drop_graphs(ctx);
  ctx->qr_mode = mode;
  return DQMC_OK;
}

int dqmc_set_metropolis_split(dqmc_ctx* ctx, int ctas_per_chain) {
  if (!ctx || (ctas_per_chain != 0 && ctas_per_chain != 1 && ctas_per_chain != 2 &&
               ctas_per_chain != 4))
    return DQMC_ERR_ARG;
  if (ctx->metro_cs != ctas_per_chain) drop_graphs(ctx);
  ctx->metro_cs = ctas_per_chain;
  return DQMC_OK;
}

int dqmc_timing_enable(dqmc_ctx* ctx, int on) {
  if (!ctx) return DQMC_ERR_ARG;
  if (on && ctx->ev.empty()) {
    const size_t pairs = 4096;
    ctx->ev.resize(2 * pairs);
    ctx->ev_class.resize(pairs);
    for (cudaEvent_t& e : ctx->ev) DQ_CK(cudaEventCreate(&e));
  }
  if (!on) DQ_RET(timing_fold(ctx));
  ctx->timing = on != 0;
  return DQMC_OK;
}

int dqmc_timing_read(dqmc_ctx* ctx, double* ms, int64_t* launches, int n_classes) {
  if (!ctx || n_classes < 0) return DQMC_ERR_ARG;
  DQ_RET(timing_fold(ctx));
  for (int c = 0; c < n_classes && c < kTNumClasses; ++c) {
    if (ms) ms[c] = ctx->tms[c];
    if (launches) launches[c] = ctx->tcount[c];
  }
  return kTNumClasses;
}

int dqmc_timing_reset(dqmc_ctx* ctx) {
  if (!ctx) return DQMC_ERR_ARG;
  DQ_RET(timing_fold(ctx));
  for (int c = 0; c < kTNumClasses; ++c) {
    ctx->tms[c] = 0.0;
    ctx->tcount[c] = 0;
  }
  return DQMC_OK;
}

const char* dqmc_timing_class_name(int c) {
  return (c >= 0 && c < kTNumClasses) ? kTimingNames[c] : "";
}

}  // extern "C"
