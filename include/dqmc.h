/*
 * dqmc.h -- C ABI of the GB300 BSS determinant quantum Monte Carlo library
 * (libdqmc.so) for the half-filled Hubbard model on periodic Lx x Ly square
 * clusters, after Rost & Bluemer, arXiv:1504.05090, Sec. 2 "Model and
 * Methods", Eqs. (1)-(3), with the analysis steps of Sec. 3 (dtau -> 0
 * extrapolation of G_k(tau), Fig. 2; Matsubara transform and self-energy,
 * Eqs. (5)-(6)) and Sec. 4 (real-space spin correlation, Fig. 5).
 *
 * Notation.  N = Lx*Ly sites, site i = x + Lx*y.  L = beta/dtau Trotter slices
 * (the paper's Lambda, Eq. (2)).  K is the hopping matrix of Eq. (1)
 * (K_ij = -t per nearest-neighbour bond and direction, periodic; a side of
 * length 2 counts the +x and -x bond separately, so K_ij = -2t there).
 * The Ising Hubbard-Stratonovich field s[l][i] = +-1 couples through
 * V_l^sigma = sigma*lambda*diag(s_l) with cosh(lambda) = exp(dtau*U/2), and
 * B_l^sigma = exp(-dtau K) exp(V_l^sigma); the weight of a field is
 * det M_up det M_dn with M_sigma = I + B_L ... B_1 (Eq. (3)).
 * G_sigma(l) = (I + B_l..B_1 B_L..B_{l+1})^{-1} is the equal-time Green
 * function G_ij = <c_i c_j^dag>; G(l,0) = B_l .. B_1 G(0) the unequal-time one.
 *
 * Conventions for every entry point.
 *  - Return 0 on success or a negative DQMC_ERR_* code; nothing throws or
 *    aborts across this boundary.  dqmc_strerror() names a code.
 *  - The context and all device state belong to the library and are freed by
 *    dqmc_destroy().  Output buffers belong to the caller.
 *  - Work is enqueued on the CUDA stream given to dqmc_init (NULL = the legacy
 *    default stream).  Calls that write host memory synchronise that stream
 *    before returning; calls with out_on_device != 0 do not.  The stateless
 *    analysis calls (dqmc_trotter_extrapolate, dqmc_matsubara_sigma) run on
 *    the legacy default stream and always synchronise it.
 *  - Chains are numbered globally in group order: group 0's chains first.
 *    Arrays "per chain" are laid out in that order; a group's block of a
 *    per-chain array with a group-dependent row length (field, G(tau)) has the
 *    group's own length.
 *  - The library needs a CUDA device of compute capability 10.3 (GB300) and
 *    fails with DQMC_ERR_CUDA otherwise.  There is no CPU fallback.
 */
#ifndef DQMC_H
#define DQMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define DQMC_OK 0
#define DQMC_ERR_ARG (-1)     /* invalid argument (sizes, ranges, NULL)          */
#define DQMC_ERR_CUDA (-2)    /* a CUDA runtime call or kernel launch failed     */
#define DQMC_ERR_OOM (-3)     /* device allocation failed                        */
#define DQMC_ERR_DRIFT (-4)   /* G drift above the context's drift limit         */
#define DQMC_ERR_TIMEOUT (-5) /* a bounded device-side wait gave up              */
#define DQMC_ERR_NAN (-6)     /* a non-finite value appeared in G                */
#define DQMC_ERR_STATE (-7)   /* call not valid in the context's current state   */

/* Working precision of the Metropolis update, the delayed rank-k update and
 * the slice wrap.  The QR/UDV stabilisation, the stabilised G recompute, the
 * drift check, the unequal-time G at stabilisation points and all reported
 * observables are FP64 in every mode. */
#define DQMC_FP64 0
#define DQMC_FP32 1
#define DQMC_DF32 2 /* pairs of floats (hi + lo, ~48 bits) on the FP32 pipe */

/* Limits of this build. */
#define DQMC_MAX_SIDE 16  /* Lx, Ly <= 16, so N <= 256                          */
#define DQMC_MAX_DELAY 32 /* delay_k <= 32                                       */
#define DQMC_TX_MAX_RUNS 16 /* runs per dqmc_trotter_extrapolate call           */

/* One group of chains with identical parameters (Eqs. (1)-(2)). */
typedef struct {
    int32_t Lx, Ly;        /* cluster sides; even, 2 <= Lx,Ly <= DQMC_MAX_SIDE.
                              Even sides make the lattice bipartite, which the
                              particle-hole evaluation of spin down requires. */
    double t;              /* hopping, Eq. (1); the paper uses t = 0.25        */
    double U;              /* interaction, Eq. (1); U >= 0                     */
    double beta;           /* inverse temperature                              */
    double dtau;           /* Trotter step; beta/dtau must be an integer to 1e-9 */
    int32_t n_chains;      /* >= 1 independent Markov chains                   */
    int32_t stab_interval; /* n_s >= 1: stabilise after every slice l with
                              l % n_s == 0 and after l = L                      */
    int32_t delay_k;       /* 1..DQMC_MAX_DELAY accepted flips per rank-k update */
    int32_t precision;     /* DQMC_FP64, DQMC_FP32 or DQMC_DF32                */
} dqmc_group;

typedef struct dqmc_ctx dqmc_ctx; /* opaque, library-owned */

/* Create a context: build exp(-+dtau K) (Eqs. (1)-(2)), draw each chain's
 * initial field from Philox4x32-10 with key = seed (counter
 * (i + N*l, 0xFFFFFFFF, chain, 1); s = +1 iff the first output word is odd),
 * build the UDV stacks and the stabilised G(0) of every chain.
 * groups: host array of n_groups >= 1 descriptors (copied).  stream: a
 * cudaStream_t or NULL.  *out receives the context.  Errors: DQMC_ERR_ARG,
 * DQMC_ERR_OOM, DQMC_ERR_CUDA.  Synchronises the stream. */
int dqmc_init(const dqmc_group* groups, int n_groups, uint64_t seed,
              void* stream, dqmc_ctx** out);

/* As dqmc_init, with the chains numbered from chain_offset >= 0 in the
 * Philox counter (initial field and proposals): a context holding chains
 * chain_offset .. chain_offset + n - 1 draws exactly what those chains draw
 * in a single context of all chains, so results do not depend on how the
 * chains are split over contexts or GPUs.  Chain indices of the accessors
 * stay local (0 .. n - 1).  chain_offset + n must not exceed 2^31 - 1.
 * Errors as dqmc_init. */
int dqmc_init_at(const dqmc_group* groups, int n_groups, uint64_t seed, int64_t chain_offset,
                 void* stream, dqmc_ctx** out);

/* Run n_sweeps >= 0 Monte Carlo sweeps of every chain (Sec. 2: the sum of
 * Eq. (3) sampled by Metropolis).  A sweep visits slices l = 1..L in order
 * and sites i = 0..N-1 within a slice; the flip of s[l][i] is accepted iff
 * u < R_up*R_dn, R_sigma = 1 + Delta_sigma (1 - G_sigma,ii),
 * Delta_sigma = exp(-2 sigma lambda s) - 1, with u from Philox4x32-10
 * (counter (i + N*(l-1), sweep, chain, 0), u = ((x0<<32|x1)>>11) 2^-53).
 * Accepted flips update G by Sherman-Morrison, applied as delayed rank-k
 * updates; G is wrapped to the next slice by B_l G B_l^{-1} and replaced by
 * a freshly stabilised FP64 G after every stabilisation point, where the
 * drift max|G_wrapped - G_fresh| / max|G_fresh| is recorded.  After the slice
 * loop the left UDV stack is rebuilt for the new field.
 * measure != 0: accumulate the equal-time observables (density, double
 * occupancy, kinetic energy per site) at every stabilisation point.
 * Enqueued asynchronously; errors of device-side checks surface at the next
 * synchronising call.  Errors: DQMC_ERR_ARG, DQMC_ERR_CUDA. */
int dqmc_sweep(dqmc_ctx* ctx, int n_sweeps, int measure);

/* Autotuner: for each group choose the stabilisation interval and the delay
 * depth for this GPU.  n_s: all candidates (L, 64, 48, ..., 3, 2 that are
 * <= L and <= 64) run side by side in one probe context of 4 chains each;
 * after two warm-up sweeps the largest n_s whose G drift over three sweeps
 * stays below drift_target / 20 is taken (1 if none; the drift over many
 * chains and sweeps is heavy-tailed, hence the margin).  If the probe reports
 * non-finite values, the largest candidate is dropped and the rest probed
 * again.  k: the fastest of 8, 16, 32 at that
 * n_s (8 chains, two timed sweeps).  out receives copies of groups with
 * stab_interval and delay_k replaced.  Creates and destroys its own contexts
 * on `stream`.  Errors: as dqmc_init. */
int dqmc_autotune(const dqmc_group* groups, int n_groups, double drift_target, uint64_t seed,
                  void* stream, dqmc_group* out);

/* Tile shapes of one group's kernels (implementation choices only: results
 * are bit-identical for every allowed value).
 *   kron_nv     vectors per CTA of the FP64 Kronecker products with
 *               exp(-+dtau K) = E_y (x) E_x of Eq. (2) (UDV stack, G(tau)
 *               propagation of FP64 groups, gradient): 1, 2, 4, 8 or 16
 *               (<= N); 0 = built-in (4)
 *   wrap_nv     vectors per CTA of the slice wrap B_l G B_l^{-1} in the
 *               working precision (float-pair groups propagate G(tau) with
 *               twice as many): same values; 0 = built-in
 *   metro_ctas  CTAs per chain of the Metropolis pass, one thread-block
 *               cluster (as dqmc_set_metropolis_split, for this group): 1, 2
 *               or 4 (4 * metro_ctas <= N); 0 = the context's setting */
typedef struct {
    int32_t kron_nv, wrap_nv, metro_ctas;
} dqmc_tiles;

/* Set the tile shapes of group `group` (creation order).  Drops captured
 * sweep graphs if anything changes.  Errors: DQMC_ERR_ARG. */
int dqmc_set_tiles(dqmc_ctx* ctx, int group, const dqmc_tiles* tiles);

/* The tile shapes in effect for group `group` (built-in choices resolved). */
int dqmc_get_tiles(const dqmc_ctx* ctx, int group, dqmc_tiles* out);

/* Tile autotuner: for each group (alone, with its full chain count) time one
 * sweep per candidate (kron_nv, wrap_nv, metro_ctas) in {(2,2,1), (4,4,2),
 * (8,8,4)} with the per-kernel-class timing, and take for each parameter the
 * candidate whose kernel class (stack_kron, wrap, metropolis) was fastest.
 * out: host array [n_groups].  Creates and destroys its own contexts on
 * `stream` (seed as dqmc_init).  Errors: as dqmc_init. */
int dqmc_autotune_tiles(const dqmc_group* groups, int n_groups, uint64_t seed, void* stream,
                        dqmc_tiles* out);

/* Sweeps are replayed as one CUDA graph per measure flag (captured at the
 * first dqmc_sweep: one branch per group, the groups run concurrently); with
 * on = 0, or while timing is enabled, kernels are launched one by one on the
 * context's stream in group order.  Default on. */
int dqmc_use_graphs(dqmc_ctx* ctx, int on);

/* Rebuild both UDV stacks of every chain from its current field and replace
 * the working G by the stabilised G(0).  max_drift_out: host array [chains]
 * receiving max|G_working - G_fresh| / max|G_fresh| before the replacement,
 * or NULL.  Synchronises. */
int dqmc_recompute_G(dqmc_ctx* ctx, double* max_drift_out);

/* Unequal-time Green function of the current field of every chain, on the
 * Trotter grid tau_l = l dtau (Sec. 2, the G_ij(tau_l) the method produces):
 * out[chain][l][k] = 1/2 sum_sigma Re G_sigma,k(tau_l), l = 0..L, where
 * G_k = (1/N) sum_ij cos(k.(r_i - r_j)) G_ij(l,0), k = 2 pi (kx/Lx, ky/Ly)
 * with index kx + Lx*ky.  G(l,0) is formed stably (FP64) at every
 * stabilisation point and propagated by B_l in between: in FP64, or in float
 * pairs for groups with DQMC_DF32 working precision (agreeing to about 1e-9
 * of the maximum).  Row length per chain is
 * (L_g + 1) * N_g of its group; dqmc_gtau_size() gives the total.
 * out: caller-owned doubles, on the device if out_on_device else on the host.
 * Requires current UDV stacks (true after dqmc_init, dqmc_sweep,
 * dqmc_set_field and dqmc_recompute_G). */
int dqmc_measure_Gtau(dqmc_ctx* ctx, double* out, int out_on_device);

/* Time-origin averaged G_k(tau): the mean over n_origins origins
 * tau_0 = s dtau, s = (o L_g) / n_origins (integer division, o < n_origins),
 * of G_k(tau_0 + tau_l, tau_0), in the layout of dqmc_measure_Gtau.  Each
 * origin is evaluated as G(tau) of the field rotated cyclically by s slices
 * (slice l of the rotated field is slice l + s mod L of the chain's), whose
 * weight in Eq. (3) is the same; the paper does not state this estimator.
 * n_origins = 1 is dqmc_measure_Gtau.  Each further origin costs a rebuild of
 * both UDV stacks and one G(tau) pass; afterwards every chain has its own
 * field again, with rebuilt stacks and the working G replaced by the freshly
 * stabilised G(0) (as dqmc_recompute_G, no drift recorded).  Requires
 * 1 <= n_origins <= L of every group; allocates and frees a field copy and,
 * for host output, one accumulator per group.  Synchronises.  Errors:
 * DQMC_ERR_ARG, DQMC_ERR_OOM, DQMC_ERR_CUDA.  After an error the call tries
 * to restore every chain's own field and to rebuild its stacks and G; if that
 * fails as well, call dqmc_recompute_G before sweeping again. */
int dqmc_measure_Gtau_origins(dqmc_ctx* ctx, int n_origins, double* out, int out_on_device);

/* dtau -> 0 extrapolation of G_k(tau) (Sec. 3, Fig. 2): runs at different
 * Trotter steps, each on its own grid tau_l = l dtau[r], are averaged over
 * their chains, put on the common fine grid tau_m = m beta / M (m = 0..M) by
 * the not-a-knot cubic spline through each run's L[r] + 1 points (the paper
 * does not name its spline; this is the reading taken), and fitted at every
 * (tau_m, k) by least squares to a + b dtau^2; out[m][k] = a.  With R = 1 the
 * result is the run's interpolation.
 *   R        1..DQMC_TX_MAX_RUNS runs; for R >= 2 the dtau must not all be equal
 *   dtau, L, C  host arrays [R]: time step, slices (L[r] >= 3, L[r] dtau[r] =
 *            beta to 1e-9) and chain count of each run
 *   gk       host array [R] of pointers to [C[r]][L[r] + 1][N] doubles, the
 *            layout dqmc_measure_Gtau writes for one group
 *   N        momenta per row (N of the lattice)
 *   out      [M + 1][N] doubles, caller-owned
 * The gk data and out are device pointers if on_device, else host.  FP64;
 * stateless (no context); runs on the legacy default stream and synchronises
 * it before returning, so device inputs written on other streams must be
 * complete.  Keeps a scratch buffer per device between calls (grown when a
 * call needs more, released at process exit); concurrent calls are
 * serialised.  Errors: DQMC_ERR_ARG, DQMC_ERR_OOM, DQMC_ERR_CUDA. */
int dqmc_trotter_extrapolate(int R, const double* dtau, const int* L, const int* C,
                             const double* const* gk, int N, double beta, int M, double* out,
                             int on_device);

/* Device time in ms of the three kernels of the last dqmc_trotter_extrapolate
 * call on the current device (chain average, spline, interpolation and fit),
 * from CUDA events recorded around them: host array ms_out[3].  Zeros before
 * the first call.  Errors: DQMC_ERR_ARG, DQMC_ERR_CUDA. */
int dqmc_trotter_timing(float* ms_out);

/* Matsubara Green function (Eq. 5) and self-energy from the Dyson equation
 * (Eq. 6) at half filling (mu = 0):
 *   G_k(i w_n) = -int_0^beta S_k(tau) e^{i w_n tau} dtau,  w_n = (2n+1) pi / beta,
 *   Sigma_k(i w_n) = i w_n - eps_k - 1 / G_k(i w_n),  eps_k = -2t (cos kx + cos ky),
 * where S_k is the not-a-knot cubic spline through the samples gk[m][k] =
 * G_k(tau_m) >= 0 (the convention of dqmc_measure_Gtau) on tau_m = m beta / M,
 * integrated exactly (the minus sign gives the standard G = -<T c c^dag>;
 * the exponent is the one under which Eq. 6 gives Sigma = 0 at U = 0).
 *   gk       [M + 1][N] doubles, N = Lx * Ly, k = kx + Lx ky (for instance the
 *            output of dqmc_trotter_extrapolate); M >= 3
 *   n_freq   frequencies n = 0..n_freq-1
 *   g_iw     [n_freq][N] complex (re, im interleaved) or NULL
 *   sigma    [n_freq][N] complex (re, im interleaved)
 * Pointers are device pointers if on_device, else host.  FP64, stateless,
 * on the legacy default stream (synchronised before returning); shares the
 * scratch and serialisation of dqmc_trotter_extrapolate.  Errors:
 * DQMC_ERR_ARG, DQMC_ERR_OOM, DQMC_ERR_CUDA. */
int dqmc_matsubara_sigma(const double* gk, int M, int Lx, int Ly, double t, double beta,
                         int n_freq, double* g_iw, double* sigma, int on_device);

/* Device time in ms of the last dqmc_matsubara_sigma call on the current
 * device: ms_out[0] the spline, ms_out[1] the transform and Dyson step. */
int dqmc_matsubara_timing(float* ms_out);
int64_t dqmc_gtau_size(const dqmc_ctx* ctx);

/* Derivatives of log W = log|det M_up| + log|det M_dn| (Eq. (3)) of the
 * current field of every chain, with respect to the hopping t (lambda and
 * the field fixed) and to the HS coupling lambda (t fixed):
 *   dlogW/dt      = dtau sum_sigma sum_l tr[A (I - G_sigma(l))], K = -t A,
 *   dlogW/dlambda = sum_sigma sigma sum_{l,i} s_li (1 - G_sigma,ii(l-1)),
 * and log W itself.  Each output: per-chain doubles or NULL, on the device if
 * out_on_device else on the host. */
int dqmc_grad(dqmc_ctx* ctx, double* dlogW_dt, double* dlogW_dlambda,
              double* logW, int out_on_device);

/* Copy all fields out (int8 [chain][L_g][N_g], host) / in.  dqmc_set_field
 * rebuilds the stacks and G(0) of every chain; values must be +-1. */
int dqmc_get_field(const dqmc_ctx* ctx, int8_t* out);
int dqmc_set_field(dqmc_ctx* ctx, const int8_t* in);
int64_t dqmc_field_size(const dqmc_ctx* ctx);

/* Stabilised FP64 G(0) of one chain and spin (0 = up, 1 = down) into a host
 * N*N row-major array.  Spin down is I - P G_up^T P, P = diag((-1)^(x+y)). */
int dqmc_get_G(const dqmc_ctx* ctx, int chain, int spin, double* out);

/* Accumulated equal-time observables, host [chain][4]:
 * sum of density, sum of double occupancy, sum of kinetic energy per site,
 * number of measurements.  dqmc_reset_observables zeroes them. */
int dqmc_get_observables(const dqmc_ctx* ctx, double* out);
int dqmc_reset_observables(dqmc_ctx* ctx);

/* Accumulated real-space spin correlation of Sec. 4 (Fig. 5), measured at the
 * same points as the observables above and zeroed with them by
 * dqmc_reset_observables:
 *   C(r) = (1/N) sum_i <S^z_i S^z_{i+r}>,  S^z_i = (n_i,up - n_i,dn) / 2,
 * r = (dx, dy) periodic, from Wick's theorem on the stabilised FP64 G_up and
 * G_dn = I - P G_up^T P of each configuration.  out: host doubles, for each
 * group in creation order [chain][N_g] with element dx + Lx dy, summed over
 * the measurements (divide by the count in the observables' last column);
 * dqmc_spin_correlation_size gives the total count of doubles (-1 for a null
 * context).  DQMC_ERR_ARG for null pointers; DQMC_ERR_CUDA if the copy fails. */
int64_t dqmc_spin_correlation_size(const dqmc_ctx* ctx);
int dqmc_get_spin_correlation(const dqmc_ctx* ctx, double* out);

/* Spin correlation length of Sec. 4 (Fig. 5, "an exponential fit" to the
 * real-space spin correlation), from the C(r) accumulated by the sweeps (see
 * dqmc_get_spin_correlation) divided by the number of measurements.  The
 * paper states neither the fitted form nor the range; the reading taken is
 * the least-squares line through the points (|r|, ln c(r)) with
 *   c(r) = (-1)^(dx+dy) C(r)        (staggered: > 0 for antiferromagnetic order)
 *   |r|  = sqrt(min(dx,Lx-dx)^2 + min(dy,Ly-dy)^2)   (minimum image)
 * over every displacement with 0 < |r| <= dmax and c(r) > 0, and
 * xi = -1/slope; +inf if the slope is >= 0 (no decay within the cluster), NaN
 * if the points span fewer than two distinct distances (or nothing has been
 * measured).  FP64.
 *   dmax  > 0, the largest distance fitted (min(Lx,Ly)/2 is the usual choice)
 *   xi    dqmc_num_chains(ctx) + n_groups doubles, caller-owned: xi of every
 *         chain in global chain order, then one per group of C(r) averaged
 *         over the group's chains (sum of C(r) over sum of measurement counts)
 *         -- device memory if out_on_device, else host (then synchronises).
 * Errors: DQMC_ERR_ARG (null pointers, dmax <= 0), DQMC_ERR_CUDA. */
int dqmc_correlation_length(dqmc_ctx* ctx, double dmax, double* xi, int out_on_device);

/* Per-chain statistics since the last reset: maximum G drift seen at a
 * stabilisation point (host doubles [chain]) and accepted flips (host
 * uint64 [chain]); either pointer may be NULL. */
int dqmc_get_stats(const dqmc_ctx* ctx, double* max_drift, uint64_t* accepted);
int dqmc_reset_stats(dqmc_ctx* ctx);

/* Total number of chains in the context. */
int dqmc_num_chains(const dqmc_ctx* ctx);

/* Number of kernel launches the library enqueued since the context was
 * created (for launch accounting). */
int64_t dqmc_launch_count(const dqmc_ctx* ctx);

/* Implementation of the FP64 matrix products of the stabilisation (UDV stack
 * updates, the split-D Green-function formula, G(tau) at stabilisation
 * points), N >= 64 only:
 *   DQMC_GEMM_TENSOR (default): tcgen05 tensor cores, each FP64 row/column
 *     cut into eight exponent-aligned 7-bit digits (BF16 operands, FP32
 *     accumulation of digit products, exact integer recombination); the
 *     error of an element is below about 2^-53 max_k|a_ik| max_k|b_kj|.
 *     The library arranges the scaled products of the stabilisation so that
 *     this matches the FP64 result to rounding level.
 *   DQMC_GEMM_FP64: the FP64 pipe.
 * Smaller clusters always use the FP64 pipe.  Errors: DQMC_ERR_ARG. */
#define DQMC_GEMM_TENSOR 0
#define DQMC_GEMM_FP64 1
int dqmc_set_gemm_mode(dqmc_ctx* ctx, int mode);

/* QR factorisation of the UDV stack steps (Sec. 2, the stabilisation of
 * Eq. (3)):
 *   DQMC_QR_BLOCKED (default): the columns of each step's product are sorted
 *     by decreasing norm once (pre-pivoting), then factorised without further
 *     pivoting by blocked Householder QR: FP64 panels of 32 columns, the
 *     trailing updates and the accumulation of Q on the tensor-core FP64
 *     products.  Used where those products are (DQMC_GEMM_TENSOR, N >= 64).
 *   DQMC_QR_PIVOTED: Householder QR with column pivoting on the FP64 pipe
 *     (always used for N < 64 and in DQMC_GEMM_FP64 mode).
 * Both give X = U D T with |diag| T = 1; G agrees between them to the
 * conditioning of the problem.  Drops captured sweep graphs.  Errors:
 * DQMC_ERR_ARG. */
#define DQMC_QR_BLOCKED 0
#define DQMC_QR_PIVOTED 1
int dqmc_set_qr_mode(dqmc_ctx* ctx, int mode);

/* CTAs per chain in the Metropolis pass (the site loop of Sec. 2 with the
 * delayed updates of G, Eq. (3)): 1, 2 or 4 CTAs of one thread-block cluster
 * share a chain, each folding the pending rank-k update into its own block of
 * rows of G; 0 (default) picks the largest of 4, 2, 1 for which all chains'
 * CTAs fit on the SMs at once.  The result does not depend on the split: the
 * CTAs take identical decisions and every element of G is formed by the same
 * operations.  Errors: DQMC_ERR_ARG for another value. */
int dqmc_set_metropolis_split(dqmc_ctx* ctx, int ctas_per_chain);

/* Optional per-launch timing (library tracing).  While enabled, every kernel
 * launch is bracketed by a pair of CUDA events on the context's stream and its
 * device time is added to the class of the kernel (metropolis, wrap,
 * stack_kron, qr_pivot, gemm_f64, gj_inverse, gtau_propagate, gtau_finalize,
 * grad_terms, misc).  dqmc_timing_read synchronises, writes up to n_classes
 * summed milliseconds and launch counts (either pointer may be NULL) and
 * returns the number of classes; dqmc_timing_class_name names a class. */
int dqmc_timing_enable(dqmc_ctx* ctx, int on);
int dqmc_timing_read(dqmc_ctx* ctx, double* ms, int64_t* launches, int n_classes);
int dqmc_timing_reset(dqmc_ctx* ctx);
const char* dqmc_timing_class_name(int cls);

/* Allocation-free entry point.  The paper has no counterpart: this exists for
 * callers that may not allocate device memory (a process whose device memory
 * belongs to another framework's allocator, a client under a hard memory
 * quota, or a latency-critical loop that cannot absorb the device-wide
 * synchronisation of cudaMalloc).  It computes the stabilised equal-time
 * Green function of spin up, G = (I + B_L ... B_1)^{-1}, for ONE field
 * configuration, exactly as dqmc_set_field + dqmc_get_G would, without any
 * cudaMalloc/cudaFree: the intermediate matrices live in a fixed device
 * array inside libdqmc of 7 N_max^2 + 2 N_max + 32 doubles (N_max =
 * DQMC_NOALLOC_MAX_N: 459,296 doubles, 3.67 MB) that every GPU loading the
 * library holds until the process exits.
 *   params: Lx, Ly, t, U, beta, dtau and stab_interval are used (validated as
 *           for dqmc_init); n_chains, delay_k and precision are ignored.
 *           Lx*Ly must not exceed DQMC_NOALLOC_MAX_N (else DQMC_ERR_ARG).
 *   field:  device pointer, int8 [L][N] with values +-1 (caller-owned).
 *   G_out:  device pointer, double [N][N] row-major (caller-owned).
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  Every call ends by reading a status
 * word back to the host and synchronising `stream`, so the function must
 * never be called while `stream` is being captured into a CUDA graph.  All
 * calls share the one array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised.
 * Returns DQMC_ERR_NAN if a pivot was singular or non-finite;
 * dqmc_last_cuda_error names the CUDA error behind a DQMC_ERR_CUDA. */
#define DQMC_NOALLOC_MAX_N 256
int dqmc_green_noalloc(const dqmc_group* params, const int8_t* field, double* G_out,
                       void* stream);

void dqmc_destroy(dqmc_ctx* ctx);
const char* dqmc_strerror(int code);
/* Message of the last CUDA runtime error that made a call on this host thread
 * return DQMC_ERR_CUDA ("no error" if none); *line (may be NULL) receives the
 * library source line that saw it. */
const char* dqmc_last_cuda_error(int* line);

#ifdef __cplusplus
}
#endif
#endif /* DQMC_H */
