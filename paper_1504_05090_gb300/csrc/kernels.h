// Host-side declarations of the libdqmc kernel launchers and their argument
// blocks (passed to the kernels by value).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"

namespace dqmc {

struct MetroArgs {
  int N, L, l0, k, chain0;
  uint32_t key0, key1;
  const uint32_t* sweep_ctr;  // device word: index of the running sweep
  double em2, ep2;            // exp(-2 lambda) - 1, exp(+2 lambda) - 1
  float em2h, em2l, ep2h, ep2l;  // the same as float pairs (hi + lo)
  unsigned long long* accepted;
  int cs;       // CTAs per chain (thread-block cluster of cs, 1 = no cluster)
  int* status;  // device status word (kDevTimeout if a peer wait gave up)
};

struct KronArgs {
  int N, Lx, Ly, L;
  int nv;                // vectors per CTA
  int kind;              // KronKind
  double c;              // sigma * lambda
  double ec, emc;        // exp(c), exp(-c), formed on the host
  KronTaps taps;
  const int8_t* field;   // [chain][L][N]
  long long mat_stride;  // elements between batch matrices (input / in place)
  long long out_stride;  // elements between output matrices (k_kron_rows)
  const double* vscale;  // optional per-vector scale (applied on load)
  long long vscale_stride;
  int per_chain;         // batch entries per chain
  // Fixed slice range (cp == nullptr): factors l0_first, l0_first+dir, ... (n_slices of them).
  int l0_first, dir, n_slices;
  // Block mode (cp != nullptr): entry blk of a chain applies factor cp[blk] + step
  // if it is < cp[blk+1] (0-based slice index), else leaves the matrix as is.
  const int* cp;
  int step;
};

// Batched square FP64 GEMM with diagonal scalings:
//   C = alpha * diag(rs) op(A) diag(ks) op(B) diag(cs) + beta * C.
// Scale modes: 0 none, 1 d, 2 1/max(d,1), 3 min(d,1), 4 1/d.
struct GemmArgs {
  int n;
  const double* A; long long sA; int tA;
  const double* B; long long sB; int tB;
  double* C; long long sC;
  const double* rs; long long srs; int rs_mode;
  const double* ks; long long sks; int ks_mode;
  // The digit-sliced tensor-core path aligns the digits of every row of op(A)
  // and every column of op(B) to that vector's largest element, so entries far
  // below it lose bits.  ks_on_b = 1 folds the inner scale into the rows of
  // op(B) instead of the columns of op(A): chosen where op(A) diag(ks) would
  // be graded along k while op(B) grows to compensate.  The FP64 pipe forms
  // a_ik ks_k b_kj either way.
  int ks_on_b;
  // balance = 1 (tensor path): before the split, the inner index k of both
  // operands is rescaled by a power of two -- op(B)'s row k down to a largest
  // entry of about 1, op(A)'s column k up by the same factor -- so that a row
  // of op(A) aligns its digits to the terms that actually occur.  Used where
  // the rows of op(B) differ in magnitude (triangular or UDV factors).
  int balance;
  const double* cs; long long scs; int cs_mode;
  double alpha, beta;
};

// Remember the CUDA error (and library source line) that makes a C-ABI call
// on this host thread return DQMC_ERR_CUDA, for dqmc_last_cuda_error.
void record_cuda_error(cudaError_t e, int line);

cudaError_t launch_init_field(int8_t* field, int C, int L, int N, int chain0, uint64_t seed,
                              cudaStream_t st);
template <typename T>
size_t metropolis_smem(int N, int k);
template <typename T>
cudaError_t launch_metropolis(T* G, int8_t* field, int C, const MetroArgs& a, cudaStream_t st);
template <typename T>
cudaError_t launch_kron_rows(const T* in, T* out, int batch, const KronArgs& a, cudaStream_t st);
template <typename T>
cudaError_t launch_kron_cols(T* X, int batch, const KronArgs& a, cudaStream_t st);
template <typename T>
cudaError_t launch_drift_reset(const double* G64, T* Gw, int C, int N, double* drift, int* status,
                               cudaStream_t st);
// The FP64 Kronecker products of k_kron_rows<double> (same arguments, vectors
// are rows) on the tcgen05 tensor cores, digit-sliced (k_kron_tc.cu); sides
// Lx, Ly <= 16.
cudaError_t launch_kron_tc(const double* in, double* out, int batch, const KronArgs& a, int* status,
                           cudaStream_t st);
cudaError_t launch_observables(const double* G64, int C, int Lx, int Ly, double t, double* obs,
                               double* spin, cudaStream_t st);

// Correlation length of every chain (out[0..C-1]) and of the chain average
// (out[C]) from the accumulated spin correlation [C][N] and observables [C][4].
cudaError_t launch_corr_length(const double* spin, const double* obs, int C, int Lx, int Ly,
                               double dmax, double* out, cudaStream_t st);

cudaError_t launch_gemm(const GemmArgs& a, int batch, cudaStream_t st);
// The same product on the tcgen05 tensor cores with FP64-level accuracy
// (k_ozaki.cu); scratch of ozaki_scratch_bytes(n, max_batch) bytes, batches
// processed max_batch matrices at a time.
size_t ozaki_scratch_bytes(int n, int max_batch);
cudaError_t launch_gemm_ozaki(const GemmArgs& a, int batch, void* scratch, int max_batch,
                              int* status, cudaStream_t st);
// General form of the same tensor-core product: for each batch entry b,
//   C[i*ldc + j] = alpha rs_i sum_k opA(i,k) ks_k opB(k,j) cs_j + beta C[i*ldc + j]
// with opA(i,k) = A[i a_sv + k a_sk] (i < M, k < K) and opB(k,j) = B[j b_sv + k b_sk]
// (j < Nc), batch strides sA, sB, sC; scale modes and balance as in GemmArgs.
// M, Nc, K <= n of the scratch (ozaki_scratch_bytes(n, max_batch)); K <= 256.
struct OzProduct {
  int M, Nc, K;
  const double* A; long long sA, a_sv, a_sk;
  const double* B; long long sB, b_sv, b_sk;
  double* C; long long sC; int ldc;
  const double* rs; long long srs; int rs_mode;
  const double* ks; long long sks; int ks_mode; int ks_on_b;
  int balance;
  const double* cs; long long scs; int cs_mode;
  double alpha, beta;
};
cudaError_t launch_ozaki_product(const OzProduct& p, int batch, void* scratch, int max_batch,
                                 int* status, cudaStream_t st);
// Householder QR with column pivoting of X^T stored row-major (row c = column
// c of X).  Outputs Q^T (row c = column c of Q), D = |diag R| and
// Rtil = D^{-1} R P^T with X = Q diag(D) Rtil.  X is overwritten.
cudaError_t launch_qrp(double* Xt, long long sX, double* Qt, long long sQ, double* D, long long sD,
                       double* Rtil, long long sR, int n, int batch, int* status, cudaStream_t st);
// In-place Gauss-Jordan inverse with row pivoting; logabs/sign of det (may be null).
cudaError_t launch_gj_inverse(double* A, long long sA, int n, int batch, double* logabs,
                              double* sign, int* status, cudaStream_t st);
// Cluster variants (k_cluster.cu): one 2-CTA cluster per matrix.
// QR: vnorm is scratch of 2 n doubles per matrix.
cudaError_t launch_qrp_cluster(double* Xt, long long sX, double* Qt, long long sQ, double* D,
                               long long sD, double* Rtil, long long sR, double* vnorm, int n,
                               int batch, int* status, cudaStream_t st);
// Blocked Householder QR with panel-wise pivoting (k_qr_blocked.cu): the same
// inputs and outputs as launch_qrp_cluster (X^T in, Q^T, D, Rtil out); the
// remaining columns are sorted by norm at every panel of 32 and pivoted within
// it, and the trailing updates and the accumulation of Q run on the
// tensor-core products (oz: scratch of ozaki_scratch_bytes(n, oz_batch)).
// X and Rtil double as workspace; QrbWork adds two n x n buffers W0, W1, Wt
// (n x 32) and perm (n ints) per matrix.
struct QrbWork {
  double* W0; double* W1; long long sW;
  double* Wt; long long sWt;
  int* perm;
};
cudaError_t launch_qr_blocked(double* Xt, long long sX, double* Qt, long long sQ, double* D,
                              long long sD, double* Rtil, long long sR, const QrbWork& wk, int n,
                              int batch, void* oz, int oz_batch, int* status, cudaStream_t st);
// Kernel launches of one launch_qr_blocked call.
int qr_blocked_launches(int n, int batch, int oz_batch);
// Gauss-Jordan: A (overwritten) -> Ainv, out of place; logabs may be null.
// pair: eliminate in float pairs (A is converted in place first; Ainv and
// logabs stay FP64).
cudaError_t launch_gj_cluster(double* A, long long sA, double* Ainv, long long sI, int n, int batch,
                              double* logabs, int* status, cudaStream_t st, bool pair = false);
cudaError_t launch_set_identity(double* M, long long sM, double* D, long long sD, int n, int batch,
                                cudaStream_t st);
template <typename T>
cudaError_t launch_convert(const double* src, T* dst, long long n, cudaStream_t st);

// Unequal-time propagation with separation bins (see k_linalg.cu).
struct GtauArgs {
  int N, Lx, Ly, L, nv, per_chain;
  int kind;              // kB for G(l,0)^T rows, kBIT for Y rows
  int vec_is_col;        // 1: vector q is column q of G(l,0); 0: vector q is row q of Y
  double c;
  double ec, emc;        // exp(c), exp(-c)
  KronTaps taps;
  const int8_t* field;
  const int* cp;         // checkpoint slices, per_chain + 1 entries... (block b: cp[b]..cp[b+1])
  long long mat_stride;
  double* bins;          // [chain][L+1][2][N]
  int bin_slot;          // 0 for G(l,0), 1 for Y
};
// pair: propagate in float pairs (groups whose working precision is df32).
cudaError_t launch_gtau_propagate(double* X, int batch, const GtauArgs& a, bool pair,
                                  cudaStream_t st);
// The same propagation and binning with the Kronecker products on the tcgen05
// tensor cores (k_kron_tc.cu), FP64-accurate; sides Lx, Ly <= 16.
cudaError_t launch_gtau_tc(const double* X, int batch, const GtauArgs& a, int* status,
                           cudaStream_t st);
// out[chain][l][k] from the bins (spin average, momentum transform).
cudaError_t launch_gtau_finalize(const double* bins, double* out, int C, int L, int Lx, int Ly,
                                 cudaStream_t st);
// Gradient terms of the current equal-time G of every (chain, block) entry
// whose factor cp[blk] + step exists: acc[chain][0] += -2 dtau sum_j sum_delta G_{j,j+delta}
// (t derivative, both spins), acc[chain][1] += sum_i s_{l0,i} (1 - 2 G_ii) (lambda).
cudaError_t launch_grad_terms(const double* G, long long sG, int per_chain, const int* cp, int step,
                              int Lx, int Ly, int L, const int8_t* field, double dtau, double* acc,
                              int batch, cudaStream_t st);

}  // namespace dqmc
