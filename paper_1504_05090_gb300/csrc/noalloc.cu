// dqmc_green_noalloc: the stabilised equal-time Green function of one field
// configuration, computed without allocating device memory.
//
// Who needs this: callers that cannot call cudaMalloc -- code that runs while
// another framework owns the device memory budget (a host process that hands
// the GPU to its own caching allocator and forbids raw allocations), clients
// of a shared GPU with a hard memory quota, and latency-sensitive loops in
// which the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable.  Such a caller passes its own device buffers for the field and
// for G; the intermediate matrices live in the fixed array below.
//
// The scratch array is a file-scope __device__ array: every GPU that loads
// libdqmc holds it (kScratchDoubles = 459,296 doubles, 3.67 MB) until the
// process exits.  In host code its name
// is only a host-side stand-in, so its device address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and passed
// to the kernels.  All calls share the one array, which keeps the contents
// of the last call: the status word is cleared at the start of every call,
// everything else is fully overwritten before it is read.  Calls whose work
// overlaps on the GPU (on different streams, or from different host threads)
// race on the array and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "../../include/dqmc.h"
#include "common.cuh"
#include "kernels.h"

namespace dqmc {
namespace {

constexpr int kNoAllocMaxN = DQMC_NOALLOC_MAX_N;
constexpr size_t kNN = static_cast<size_t>(kNoAllocMaxN) * kNoAllocMaxN;
// Layout: U0, U1, T0, T1, X, Rtil, Mid (7 N x N), D0, D1 (2 N), status word.
constexpr size_t kScratchDoubles = 7 * kNN + 2 * kNoAllocMaxN + 32;
static_assert(DQMC_MAX_SIDE * DQMC_MAX_SIDE <= DQMC_NOALLOC_MAX_N,
              "every cluster that dqmc_init accepts fits the scratch array");

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once).
int scratch_address(double** out) {
  int dev = 0;
  const cudaError_t eg = cudaGetDevice(&dev);
  if (eg != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    record_cuda_error(eg != cudaSuccess ? eg : cudaErrorInvalidDevice, __LINE__);
    return DQMC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      record_cuda_error(e != cudaSuccess ? e : cudaErrorInvalidSymbol, __LINE__);
      return DQMC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DQMC_OK;
}

// Circulant taps of exp(-+dtau K) on a ring of n sites with band -2t cos k.
void taps_1d(int n, double t, double dtau, double* e, double* ei) {
  for (int d = 0; d < kMaxSide; ++d) e[d] = ei[d] = 0.0;
  for (int d = 0; d < n; ++d) {
    double a = 0.0, b = 0.0;
    for (int m = 0; m < n; ++m) {
      const double k = 2.0 * M_PI * m / n;
      a += std::cos(k * d) * std::exp(2.0 * t * dtau * std::cos(k));
      b += std::cos(k * d) * std::exp(-2.0 * t * dtau * std::cos(k));
    }
    e[d] = a / n;
    ei[d] = b / n;
  }
}

// Mid = Db^{-1} U^T + Ds T for (I + U D T) = U Db Mid (U^T stored as Ut).
__global__ void k_noalloc_mid(const double* Ut, const double* T, const double* D, double* Mid,
                              int n) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
       e < static_cast<size_t>(n) * n; e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / n);
    const double d = D[i];
    Mid[e] = Ut[e] / fmax(d, 1.0) + fmin(d, 1.0) * T[e];
  }
}

}  // namespace
}  // namespace dqmc

using namespace dqmc;

extern "C" int dqmc_green_noalloc(const dqmc_group* p, const int8_t* field, double* G_out,
                                  void* stream) {
  if (!p || !field || !G_out) return DQMC_ERR_ARG;
  if (p->Lx < 2 || p->Ly < 2 || (p->Lx & 1) || (p->Ly & 1) || p->Lx > DQMC_MAX_SIDE ||
      p->Ly > DQMC_MAX_SIDE)
    return DQMC_ERR_ARG;
  const int N = p->Lx * p->Ly;
  if (N > kNoAllocMaxN) return DQMC_ERR_ARG;  // scratch holds N <= DQMC_NOALLOC_MAX_N
  if (!(p->dtau > 0.0) || !(p->beta > 0.0) || !(p->U >= 0.0) || !std::isfinite(p->t) ||
      p->stab_interval < 1)
    return DQMC_ERR_ARG;
  const double r = p->beta / p->dtau;
  const long long Lll = std::llround(r);
  if (Lll < 1 || Lll > 100000 || std::fabs(r - static_cast<double>(Lll)) > 1e-9) return DQMC_ERR_ARG;
  const int L = static_cast<int>(Lll);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  double* s = nullptr;
  int rc = scratch_address(&s);
  if (rc != DQMC_OK) return rc;
  const long long nn = static_cast<long long>(N) * N;
  double* U[2] = {s, s + nn};
  double* T[2] = {s + 2 * nn, s + 3 * nn};
  double* X = s + 4 * nn;
  double* Rt = s + 5 * nn;
  double* Mid = s + 6 * nn;
  double* D[2] = {s + 7 * nn, s + 7 * nn + N};
  int* status = reinterpret_cast<int*>(s + 7 * nn + 2 * N);

#define NA_CK(call)                   \
  do {                                \
    const cudaError_t e_ = (call);    \
    if (e_ != cudaSuccess) {          \
      record_cuda_error(e_, __LINE__); \
      return DQMC_ERR_CUDA;           \
    }                                 \
  } while (0)
  NA_CK(cudaMemsetAsync(status, 0, sizeof(int), st));

  KronArgs a{};
  a.N = N;
  a.Lx = p->Lx;
  a.Ly = p->Ly;
  a.L = L;
  a.kind = kB;
  a.c = std::acosh(std::exp(0.5 * p->dtau * p->U));
  a.ec = std::exp(a.c);
  a.emc = std::exp(-a.c);
  taps_1d(p->Lx, p->t, p->dtau, a.taps.ex, a.taps.exi);
  taps_1d(p->Ly, p->t, p->dtau, a.taps.ey, a.taps.eyi);
  a.field = field;
  a.mat_stride = nn;
  a.out_stride = nn;
  a.vscale_stride = N;
  a.per_chain = 1;
  a.dir = 1;
  a.nv = std::max(1, std::min({32, N, (120 * 1024) / ((N + 1) * 16)}));

  // B_L ... B_1 = U D T, re-orthogonalised every stab_interval slices.
  NA_CK(launch_set_identity(U[0], nn, D[0], N, N, 1, st));
  NA_CK(launch_set_identity(T[0], nn, nullptr, 0, N, 1, st));
  int cur = 0;
  for (int l0 = 0; l0 < L; l0 += p->stab_interval) {
    a.l0_first = l0;
    a.n_slices = std::min(p->stab_interval, L - l0);
    a.vscale = D[cur];
    NA_CK(launch_kron_rows<double>(U[cur], X, 1, a, st));
    NA_CK(launch_qrp(X, nn, U[1 - cur], nn, D[1 - cur], N, Rt, nn, N, 1, status, st));
    GemmArgs m{};
    m.n = N;
    m.alpha = 1.0;
    m.A = Rt;
    m.B = T[cur];
    m.C = T[1 - cur];
    NA_CK(launch_gemm(m, 1, st));
    cur = 1 - cur;
  }
  // G = (I + U D T)^{-1} = Mid^{-1} Db^{-1} U^T.
  const int blocks = static_cast<int>(std::min<long long>((nn + 255) / 256, 256));
  k_noalloc_mid<<<blocks, 256, 0, st>>>(U[cur], T[cur], D[cur], Mid, N);
  NA_CK(cudaGetLastError());
  NA_CK(launch_gj_inverse(Mid, nn, N, 1, nullptr, nullptr, status, st));
  GemmArgs m{};
  m.n = N;
  m.alpha = 1.0;
  m.A = Mid;
  m.B = U[cur];
  m.ks = D[cur];
  m.ks_mode = 2;
  m.C = G_out;
  NA_CK(launch_gemm(m, 1, st));
  int hs = 0;
  NA_CK(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
  return hs == 0 ? DQMC_OK : DQMC_ERR_NAN;
}
