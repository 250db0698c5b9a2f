// FP64 linear algebra of libdqmc: the UDV stabilisation of the B-matrix
// chain and the stabilised Green functions built from it.
//
// Paper: Rost & Bluemer, arXiv:1504.05090, Sec. 2 -- the determinants of
// Eq. (3) and the Green functions G_ij(tau_l) need the products
// B_l ... B_1 (cost O(Lambda N^3)), which are numerically unstable at low
// temperature.  They are kept as U diag(D) T (U orthogonal, D graded, T well
// conditioned) by Householder QR with column pivoting, and G is formed with
// D split into Db = max(D,1) and Ds = min(D,1):
//   I + R L = U_R Db_R Mid Db_L U_L^T,
//   Mid = Db_R^{-1} (U_R^T U_L) Db_L^{-1} + Ds_R (T_R T_L^T) Ds_L,
// for R = U_R D_R T_R and L^T = U_L D_L T_L.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace dqmc {

__device__ __forceinline__ double scale_of(const double* p, int mode, int i) {
  if (mode == 0 || p == nullptr) return 1.0;
  const double d = p[i];
  switch (mode) {
    case 1: return d;
    case 2: return 1.0 / fmax(d, 1.0);
    case 3: return fmin(d, 1.0);
    default: return 1.0 / d;
  }
}

// ---------------------------------------------------------------------------
// Batched FP64 GEMM, 64x64 output tile per CTA, 16x16 threads with 4x4 each.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gemm_f64(GemmArgs a) {
  const int b = blockIdx.z;
  const int n = a.n;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const double* A = a.A + b * a.sA;
  const double* B = a.B + b * a.sB;
  double* C = a.C + b * a.sC;
  const double* rs = a.rs ? a.rs + b * a.srs : nullptr;
  const double* ks = a.ks ? a.ks + b * a.sks : nullptr;
  const double* cs = a.cs ? a.cs + b * a.scs : nullptr;
  __shared__ double As[16][64 + 2];
  __shared__ double Bs[16][64 + 2];
  // Diagonal scale factors of this tile, formed once per tile (a division per
  // loaded element would cost more FP64 issue than the tile's FMAs).
  __shared__ double rsv[64], csv[64], ksv[16];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (threadIdx.x < 64) {
    const int i = i0 + threadIdx.x, jx = j0 + threadIdx.x;
    rsv[threadIdx.x] = (i < n) ? a.alpha * scale_of(rs, a.rs_mode, i) : 0.0;
    csv[threadIdx.x] = (jx < n) ? scale_of(cs, a.cs_mode, jx) : 0.0;
  }
  double acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 16) {
    if (threadIdx.x < 16) ksv[threadIdx.x] = (k0 + threadIdx.x < n) ? scale_of(ks, a.ks_mode, k0 + threadIdx.x) : 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int ii, kk;
      double v = 0.0;
      if (a.tA == 0) {
        ii = e >> 4;
        kk = e & 15;
        if (i0 + ii < n && k0 + kk < n) v = A[static_cast<size_t>(i0 + ii) * n + k0 + kk];
      } else {
        kk = e >> 6;
        ii = e & 63;
        if (i0 + ii < n && k0 + kk < n) v = A[static_cast<size_t>(k0 + kk) * n + i0 + ii];
      }
      As[kk][ii] = (a.ks_mode != 0) ? v * ksv[kk] : v;
      int jj;
      double w = 0.0;
      if (a.tB == 0) {
        kk = e >> 6;
        jj = e & 63;
        if (k0 + kk < n && j0 + jj < n) w = B[static_cast<size_t>(k0 + kk) * n + j0 + jj];
      } else {
        jj = e >> 4;
        kk = e & 15;
        if (k0 + kk < n && j0 + jj < n) w = B[static_cast<size_t>(j0 + jj) * n + k0 + kk];
      }
      Bs[kk][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty * 4 + r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx * 4 + q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fma(av[r], bv[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= n) continue;
    const double rv = rsv[ty * 4 + r];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tx * 4 + q;
      if (j >= n) continue;
      double v = rv * acc[r][q] * csv[tx * 4 + q];
      const size_t o = static_cast<size_t>(i) * n + j;
      if (a.beta != 0.0) v += a.beta * C[o];
      C[o] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Block reductions.
// ---------------------------------------------------------------------------
struct ArgMax {
  double v;
  int i;
};

__device__ __forceinline__ ArgMax argmax_combine(ArgMax a, ArgMax b) {
  if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
  return a;
}

__device__ ArgMax block_argmax(ArgMax x, ArgMax* sbuf) {
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax y;
    y.v = __shfl_xor_sync(0xFFFFFFFFu, x.v, o);
    y.i = __shfl_xor_sync(0xFFFFFFFFu, x.i, o);
    x = argmax_combine(x, y);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sbuf[w] = x;
  __syncthreads();
  ArgMax r = sbuf[0];
  for (int q = 1; q < nw; ++q) r = argmax_combine(r, sbuf[q]);
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Householder QR with column pivoting (partial column norms downdated, with
// recomputation when cancellation is detected, as in LAPACK's xLAQP2), one
// CTA per matrix.  Storage is X^T row-major so that a column of X is a
// contiguous row; one warp updates one column at a time.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_qrp(double* Xall, long long sX, double* Qall, long long sQ,
                                            double* Dall, long long sD, double* Rall, long long sR,
                                            int n, int* status) {
  const int b = blockIdx.x;
  double* X = Xall + b * sX;
  double* Qt = Qall + b * sQ;
  double* D = Dall + b * sD;
  double* Rt = Rall + b * sR;
  __shared__ double vn1[kMaxN], vn2[kMaxN], vsh[kMaxN], taus[kMaxN];
  __shared__ int perm[kMaxN];
  __shared__ ArgMax sred[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double tol3z = sqrt(DBL_EPSILON);

  for (int c = w; c < n; c += nw) {
    double s = 0.0;
    for (int r = lane; r < n; r += 32) {
      const double x = X[static_cast<size_t>(c) * n + r];
      s += x * x;
    }
    s = warp_sum(s);
    if (lane == 0) {
      vn1[c] = sqrt(s);
      vn2[c] = vn1[c];
      perm[c] = c;
    }
  }
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    ArgMax m{-1.0, n};
    for (int c = j + threadIdx.x; c < n; c += blockDim.x) m = argmax_combine(m, ArgMax{vn1[c], c});
    int p = block_argmax(m, sred).i;
    if (p < j || p >= n) {  // only non-finite norms left: keep the column, flag it
      if (threadIdx.x == 0) atomicExch(status, kDevNonFinite);
      p = j;
    }
    if (p != j) {
      for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const double t = X[static_cast<size_t>(j) * n + r];
        X[static_cast<size_t>(j) * n + r] = X[static_cast<size_t>(p) * n + r];
        X[static_cast<size_t>(p) * n + r] = t;
      }
      if (threadIdx.x == 0) {
        int ti = perm[j]; perm[j] = perm[p]; perm[p] = ti;
        double tv = vn1[j]; vn1[j] = vn1[p]; vn1[p] = tv;
        tv = vn2[j]; vn2[j] = vn2[p]; vn2[p] = tv;
      }
    }
    __syncthreads();
    double* xj = X + static_cast<size_t>(j) * n;
    if (w == 0) {
      double sig = 0.0;
      for (int r = j + 1 + lane; r < n; r += 32) sig += xj[r] * xj[r];
      sig = warp_sum(sig);
      const double alpha = xj[j];
      double tau = 0.0, beta = alpha, scal = 1.0;
      if (sig != 0.0) {
        const double nr = sqrt(alpha * alpha + sig);
        beta = (alpha <= 0.0) ? nr : -nr;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      for (int r = j + 1 + lane; r < n; r += 32) xj[r] *= scal;
      __syncwarp();
      if (lane == 0) {
        xj[j] = beta;
        taus[j] = tau;
      }
    }
    __syncthreads();
    for (int r = j + threadIdx.x; r < n; r += blockDim.x) vsh[r] = (r == j) ? 1.0 : xj[r];
    __syncthreads();
    const double tau = taus[j];
    for (int c = j + 1 + w; c < n; c += nw) {
      double* xc = X + static_cast<size_t>(c) * n;
      double s = 0.0;
      for (int r = j + lane; r < n; r += 32) s += vsh[r] * xc[r];
      s = warp_sum(s) * tau;
      for (int r = j + lane; r < n; r += 32) xc[r] -= s * vsh[r];
      __syncwarp();
      if (lane == 0 && vn1[c] != 0.0) {
        double t = absd(xc[j]) / vn1[c];
        t = fmax(0.0, 1.0 - t * t);
        const double q = vn1[c] / vn2[c];
        if (t * q * q <= tol3z) vn1[c] = -1.0;  // flag: recompute below
        else vn1[c] *= sqrt(t);
      }
      __syncwarp();
      if (vn1[c] < 0.0) {
        double s2 = 0.0;
        for (int r = j + 1 + lane; r < n; r += 32) s2 += xc[r] * xc[r];
        s2 = warp_sum(s2);
        __syncwarp();
        if (lane == 0) {
          vn1[c] = sqrt(s2);
          vn2[c] = vn1[c];
        }
      }
    }
    __syncthreads();
  }

  // D = |diag R|, Rtil[i][perm[c]] = R[i][c] / D[i]  (R[i][c] = X[c][i], c >= i).
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d = absd(X[static_cast<size_t>(i) * n + i]);
    if (!(d > 0.0)) {
      atomicExch(status, kDevSingular);
      d = DBL_MIN;
    }
    D[i] = d;
  }
  __syncthreads();
  for (size_t e = threadIdx.x; e < static_cast<size_t>(n) * n; e += blockDim.x) {
    const int i = static_cast<int>(e / n), c = static_cast<int>(e - static_cast<size_t>(i) * n);
    const double v = (c >= i) ? X[static_cast<size_t>(c) * n + i] / D[i] : 0.0;
    Rt[static_cast<size_t>(i) * n + perm[c]] = v;
  }
  // Q = H_0 H_1 ... H_{n-1}, accumulated backwards into Q^T (row c = column c).
  for (size_t e = threadIdx.x; e < static_cast<size_t>(n) * n; e += blockDim.x) {
    const int c = static_cast<int>(e / n), r = static_cast<int>(e - static_cast<size_t>(c) * n);
    Qt[e] = (c == r) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const double* xj = X + static_cast<size_t>(j) * n;
    for (int r = j + threadIdx.x; r < n; r += blockDim.x) vsh[r] = (r == j) ? 1.0 : xj[r];
    __syncthreads();
    const double tau = taus[j];
    if (tau != 0.0) {
      for (int c = j + w; c < n; c += nw) {
        double* qc = Qt + static_cast<size_t>(c) * n;
        double s = 0.0;
        for (int r = j + lane; r < n; r += 32) s += vsh[r] * qc[r];
        s = warp_sum(s) * tau;
        for (int r = j + lane; r < n; r += 32) qc[r] -= s * vsh[r];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// In-place Gauss-Jordan inverse with row pivoting, one CTA per matrix;
// also log|det| and sign(det).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_gj_inverse(double* Aall, long long sA, int n,
                                                   double* logabs, double* sgn, int* status) {
  const int b = blockIdx.x;
  double* A = Aall + b * sA;
  __shared__ double prow[kMaxN], fcol[kMaxN];
  __shared__ int perm[kMaxN];
  __shared__ ArgMax sred[32];
  double la = 0.0, sg = 1.0;
  for (int k = 0; k < n; ++k) {
    ArgMax m{-1.0, n};
    for (int i = k + threadIdx.x; i < n; i += blockDim.x)
      m = argmax_combine(m, ArgMax{absd(A[static_cast<size_t>(i) * n + k]), i});
    int p = block_argmax(m, sred).i;
    if (p < k || p >= n) {  // non-finite column: no valid pivot, flag it
      if (threadIdx.x == 0) atomicExch(status, kDevNonFinite);
      p = k;
    }
    if (p != k) {
      for (int jj = threadIdx.x; jj < n; jj += blockDim.x) {
        const double t = A[static_cast<size_t>(k) * n + jj];
        A[static_cast<size_t>(k) * n + jj] = A[static_cast<size_t>(p) * n + jj];
        A[static_cast<size_t>(p) * n + jj] = t;
      }
      sg = -sg;
    }
    if (threadIdx.x == 0) perm[k] = p;
    __syncthreads();
    double piv = A[static_cast<size_t>(k) * n + k];
    if (!(absd(piv) > 0.0)) {
      if (threadIdx.x == 0) atomicExch(status, kDevSingular);
      piv = DBL_MIN;
    }
    la += log(absd(piv));
    if (piv < 0.0) sg = -sg;
    const double ipiv = 1.0 / piv;
    for (int jj = threadIdx.x; jj < n; jj += blockDim.x) {
      const double v = (jj == k) ? ipiv : A[static_cast<size_t>(k) * n + jj] * ipiv;
      prow[jj] = v;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      fcol[i] = (i == k) ? 0.0 : A[static_cast<size_t>(i) * n + k];
    __syncthreads();
    for (size_t e = threadIdx.x; e < static_cast<size_t>(n) * n; e += blockDim.x) {
      const int i = static_cast<int>(e / n), jj = static_cast<int>(e - static_cast<size_t>(i) * n);
      if (i == k) {
        A[e] = prow[jj];
      } else {
        const double f = fcol[i];
        A[e] = (jj == k) ? -f * prow[k] : A[e] - f * prow[jj];
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double t = A[static_cast<size_t>(i) * n + k];
        A[static_cast<size_t>(i) * n + k] = A[static_cast<size_t>(i) * n + p];
        A[static_cast<size_t>(i) * n + p] = t;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (logabs) logabs[b] = la;
    if (sgn) sgn[b] = sg;
  }
}

__global__ void k_set_identity(double* M, long long sM, double* D, long long sD, int n) {
  const int b = blockIdx.y;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
       e < static_cast<size_t>(n) * n; e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(e / n), j = static_cast<int>(e - static_cast<size_t>(i) * n);
    M[b * sM + e] = (i == j) ? 1.0 : 0.0;
    if (D && j == 0) D[b * sD + i] = 1.0;
  }
}

template <typename T>
__global__ void k_convert(const double* src, T* dst, long long n) {
  for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<long long>(gridDim.x) * blockDim.x)
    dst[e] = static_cast<T>(src[e]);
}

// ---------------------------------------------------------------------------
// Unequal-time G: starting from the matrix of a stabilisation point, apply
// the slice factors of the block and, after each slice, add every element
// into the bin of its separation r = r_i - r_j.  Vectors are contiguous rows
// (G(l,0)^T or Y = (I - G(0)) R_l^{-1}).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void kron_transform_d(T* v, T* tmp, int nv, int ld, int Lx, int Ly, int N, const T* tx,
                                 const T* ty, const T* txs, const T* tys, const T* pre,
                                 const T* post);

// Two taps read with one load (16 bytes for 8-byte types).
template <typename T>
struct alignas(2 * sizeof(T)) GtPair {
  T a, b;
};

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(df32 x) { return static_cast<double>(x); }

// T = double, or df32 (float pairs) for groups whose working precision is
// df32: the propagation between stabilisation points then runs on the FP32
// pipe; the loaded G(c,0) / Y and the bins stay FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_gtau_propagate(double* Xall, GtauArgs a) {
  const int b = blockIdx.y;
  const int chain = b / a.per_chain, blk = b - chain * a.per_chain;
  const int N = a.N, nv = a.nv, ld = N + 1;
  const int r0 = blockIdx.x * nv;
  const int nrows = min(nv, N - r0);
  const int lo = a.cp[blk], hi = a.cp[blk + 1];
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* v = reinterpret_cast<T*>(sm_raw);
  T* tmp = v + nv * ld;
  T* tx = tmp + nv * ld;
  T* ty = tx + 2 * kMaxSide;
  T* txs = ty + 2 * kMaxSide;  // the taps shifted by one, txs[k] = tx[k + 1]
  T* tys = txs + 2 * kMaxSide;
  T* sc = tys + 2 * kMaxSide;
  const bool inv = (a.kind == kBIT);
  if (threadIdx.x < 2 * kMaxSide) {  // each circulant row twice over (kron_transform_d)
    const int t = threadIdx.x, tx_ = t % a.Lx, ty_ = t % a.Ly;
    tx[t] = static_cast<T>(inv ? a.taps.exi[tx_] : a.taps.ex[tx_]);
    ty[t] = static_cast<T>(inv ? a.taps.eyi[ty_] : a.taps.ey[ty_]);
    const int tx1 = (t + 1) % a.Lx, ty1 = (t + 1) % a.Ly;
    txs[t] = static_cast<T>(inv ? a.taps.exi[tx1] : a.taps.ex[tx1]);
    tys[t] = static_cast<T>(inv ? a.taps.eyi[ty1] : a.taps.ey[ty1]);
  }
  double* X = Xall + static_cast<size_t>(b) * a.mat_stride;
  for (int e = threadIdx.x; e < nrows * N; e += blockDim.x) {
    const int vi = e / N, i = e - vi * N;
    v[vi * ld + i] = static_cast<T>(X[static_cast<size_t>(r0 + vi) * N + i]);
  }
  const Geom g{a.Lx, a.Ly, N};
  const int8_t* f = a.field + static_cast<size_t>(chain) * a.L * N;
  const T up = static_cast<T>(inv ? a.emc : a.ec), dn = static_cast<T>(inv ? a.ec : a.emc);
  for (int l = lo; l < hi; ++l) {
    __syncthreads();
    if (l > lo) {
      for (int i = threadIdx.x; i < N; i += blockDim.x)
        sc[i] = f[static_cast<size_t>(l - 1) * N + i] > 0 ? up : dn;
      __syncthreads();
      kron_transform_d<T>(v, tmp, nrows, ld, a.Lx, a.Ly, N, tx, ty, txs, tys, sc, nullptr);
    }
    // every vector has exactly one element per separation r: the thread of
    // bin r sums them over the block's vectors in the working precision and
    // adds the block's sum to the global bin
    double* out = a.bins + ((static_cast<size_t>(chain) * (a.L + 1) + l) * 2 + a.bin_slot) * N;
    for (int r = threadIdx.x; r < N; r += blockDim.x) {
      const int rx = r % a.Lx, ry = r / a.Lx;
      T acc = T(0);
      for (int vi = 0; vi < nrows; ++vi) {
        const int q = r0 + vi, qx = q % a.Lx, qy = q / a.Lx;
        // vec_is_col: r = r_el - r_q, else r = r_q - r_el
        const int ex = a.vec_is_col ? qx + rx : qx - rx + a.Lx;
        const int ey = a.vec_is_col ? qy + ry : qy - ry + a.Ly;
        const int el = (ex % a.Lx) + a.Lx * (ey % a.Ly);
        acc = acc + v[vi * ld + el];
      }
      atomicAdd(&out[r], to_d(acc));
    }
  }
}

template <typename T>
__device__ void kron_transform_d(T* v, T* tmp, int nv, int ld, int Lx, int Ly, int N, const T* tx,
                                 const T* ty, const T* txs, const T* tys, const T* pre,
                                 const T* post) {
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
        const GtPair<T> t2 = (b & 1) ? *reinterpret_cast<const GtPair<T>*>(txs + b - 1)
                                       : *reinterpret_cast<const GtPair<T>*>(tx + b);
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
        const GtPair<T> t2 = (b & 1) ? *reinterpret_cast<const GtPair<T>*>(tys + b - 1)
                                       : *reinterpret_cast<const GtPair<T>*>(ty + b);
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
  // Two vectors per thread sharing each tap load; taps stored twice over
  // (tx[k] = Ex[k mod Lx] for k < 2 Lx), tap x - x' mod Lx = tx[x + Lx - x'].
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
    v[(2 * vp) * ld + i] = post ? a0.get() * post[i] : a0.get();
    if (two) v[(2 * vp + 1) * ld + i] = post ? a1.get() * post[i] : a1.get();
  }
  __syncthreads();
}

// out[c][l][k] = 1/(2N) sum_r cos(k.r) (binG[r] + (-1)^{rx+ry} binY[r]); the
// second term is the spin-down G at k from Y at k + (pi, pi).
__global__ void __launch_bounds__(256) k_gtau_finalize(const double* bins, double* out, int L,
                                                      int Lx, int Ly) {
  const int cl = blockIdx.x;  // chain * (L+1) + l
  const int N = Lx * Ly;
  const double* bg = bins + static_cast<size_t>(cl) * 2 * N;
  const double* by = bg + N;
  __shared__ double fr[kMaxN], hc[kMaxN], hs[kMaxN];
  // cos and sin of the Lx (Ly) distinct phases 2 pi m / Lx, once per block
  __shared__ double cxs[kMaxSide], sxs[kMaxSide], cys[kMaxSide], sys[kMaxSide];
  if (threadIdx.x < Lx) {
    const double ph = 2.0 * threadIdx.x / Lx;
    cxs[threadIdx.x] = cospi(ph);
    sxs[threadIdx.x] = sinpi(ph);
  }
  if (threadIdx.x < Ly) {
    const double ph = 2.0 * threadIdx.x / Ly;
    cys[threadIdx.x] = cospi(ph);
    sys[threadIdx.x] = sinpi(ph);
  }
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    const int rx = r % Lx, ry = r / Lx;
    fr[r] = bg[r] + (((rx + ry) & 1) ? -by[r] : by[r]);
  }
  __syncthreads();
  // hc/hs[kx + Lx ry] = sum_rx cos/sin(2 pi kx rx / Lx) f(rx, ry)
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int kx = e % Lx, ry = e / Lx;
    double c = 0.0, s = 0.0;
    for (int rx = 0; rx < Lx; ++rx) {
      const int m = (kx * rx) % Lx;
      c += cxs[m] * fr[rx + Lx * ry];
      s += sxs[m] * fr[rx + Lx * ry];
    }
    hc[e] = c;
    hs[e] = s;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N; e += blockDim.x) {
    const int kx = e % Lx, ky = e / Lx;
    double acc = 0.0;
    for (int ry = 0; ry < Ly; ++ry) {
      const int m = (ky * ry) % Ly;
      acc += cys[m] * hc[kx + Lx * ry] - sys[m] * hs[kx + Lx * ry];
    }
    out[static_cast<size_t>(cl) * N + e] = acc / (2.0 * N);
  }
}

__global__ void __launch_bounds__(256) k_grad_terms(const double* Gall, long long sG, int per_chain,
                                                   const int* cp, int step, int Lx, int Ly, int L,
                                                   const int8_t* field, double dtau, double* acc) {
  const int b = blockIdx.x;
  const int chain = b / per_chain, blk = b - chain * per_chain;
  const int m = cp[blk] + step;
  if (m >= cp[blk + 1]) return;
  const int N = Lx * Ly;
  const double* G = Gall + b * sG;
  const int8_t* s = field + (static_cast<size_t>(chain) * L + m) * N;
  double tt = 0.0, tl = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int x = j % Lx, y = j / Lx;
    const int nb[4] = {(x + 1) % Lx + Lx * y, (x + Lx - 1) % Lx + Lx * y, x + Lx * ((y + 1) % Ly),
                       x + Lx * ((y + Ly - 1) % Ly)};
    for (int q = 0; q < 4; ++q) tt += G[static_cast<size_t>(j) * N + nb[q]];
    tl += static_cast<double>(s[j]) * (1.0 - 2.0 * G[static_cast<size_t>(j) * N + j]);
  }
  tt = warp_sum(tt);
  tl = warp_sum(tl);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[chain * 3 + 0], -2.0 * dtau * tt);
    atomicAdd(&acc[chain * 3 + 1], tl);
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_gemm(const GemmArgs& a, int batch, cudaStream_t st) {
  dim3 grid((a.n + 63) / 64, (a.n + 63) / 64, batch);
  k_gemm_f64<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_qrp(double* Xt, long long sX, double* Qt, long long sQ, double* D, long long sD,
                       double* Rtil, long long sR, int n, int batch, int* status, cudaStream_t st) {
  k_qrp<<<batch, 512, 0, st>>>(Xt, sX, Qt, sQ, D, sD, Rtil, sR, n, status);
  return cudaGetLastError();
}

cudaError_t launch_gj_inverse(double* A, long long sA, int n, int batch, double* logabs,
                              double* sign, int* status, cudaStream_t st) {
  k_gj_inverse<<<batch, 512, 0, st>>>(A, sA, n, logabs, sign, status);
  return cudaGetLastError();
}

cudaError_t launch_set_identity(double* M, long long sM, double* D, long long sD, int n, int batch,
                                cudaStream_t st) {
  dim3 grid(std::max(1, std::min((n * n + 255) / 256, 64)), batch);
  k_set_identity<<<grid, 256, 0, st>>>(M, sM, D, sD, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert(const double* src, T* dst, long long n, cudaStream_t st) {
  const int blocks = static_cast<int>(std::min<long long>((n + 255) / 256, 152 * 8));
  k_convert<T><<<std::max(blocks, 1), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double>(const double*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<df32>(const double*, df32*, long long, cudaStream_t);

template <typename T>
static cudaError_t gtau_launch(double* X, int batch, const GtauArgs& a, cudaStream_t st) {
  const size_t sm =
                    (2ull * a.nv * (a.N + 1) + 8 * kMaxSide + static_cast<size_t>(a.N)) * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(k_gtau_propagate<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
  if (e != cudaSuccess) return e;
  dim3 grid((a.N + a.nv - 1) / a.nv, batch);
  k_gtau_propagate<T><<<grid, 256, sm, st>>>(X, a);
  return cudaGetLastError();
}

cudaError_t launch_gtau_propagate(double* X, int batch, const GtauArgs& a, bool pair,
                                  cudaStream_t st) {
  return pair ? gtau_launch<df32>(X, batch, a, st) : gtau_launch<double>(X, batch, a, st);
}

cudaError_t launch_gtau_finalize(const double* bins, double* out, int C, int L, int Lx, int Ly,
                                 cudaStream_t st) {
  k_gtau_finalize<<<C * (L + 1), 256, 0, st>>>(bins, out, L, Lx, Ly);
  return cudaGetLastError();
}

cudaError_t launch_grad_terms(const double* G, long long sG, int per_chain, const int* cp, int step,
                              int Lx, int Ly, int L, const int8_t* field, double dtau, double* acc,
                              int batch, cudaStream_t st) {
  k_grad_terms<<<batch, 256, 0, st>>>(G, sG, per_chain, cp, step, Lx, Ly, L, field, dtau, acc);
  return cudaGetLastError();
}

}  // namespace dqmc
