"""Oracle: plain FP64 CPU BSS-DQMC for the half-filled 2D Hubbard model.

TEST INFRASTRUCTURE ONLY -- imported by `tests/`, `__graft_entry__.smoke()`
and the CPU legs of `bench.py`, never by the CUDA product path.  It is written
to be read against the paper, not to be fast:

  * everything is float64 numpy; QR with column pivoting, eigh and slogdet are
    library primitives (scipy/numpy) used as single steps;
  * both spin species are evolved explicitly (the particle-hole identity
    G_dn = I - P G_up^T P is tested, not assumed);
  * every stabilised Green function is recomputed from scratch from the whole
    chain of B matrices (no stored stacks), so no bookkeeping can go stale.

Paper map (Rost & Bluemer, arXiv:1504.05090, Sec. 2 "Model and Methods"):
  Eq. (1)  Hubbard Hamiltonian, hopping t = 0.25 on periodic clusters
           -> hopping_matrix, exp_hopping
  Eq. (2)  Trotter decomposition Z_dtau = Tr prod_l e^{-dtau H_t} e^{-dtau H_U},
           Lambda = beta/dtau slices -> b_matrix (B_l = e^{-dtau K} e^{V_l})
  Sec. 2   discrete Hubbard-Stratonovich transform to an Ising field h
           -> hs_lambda, hs_prefactor
  Eq. (3)  Z_dtau = sum_h det M_up det M_dn, M = I + B_L ... B_1
           -> weight_log, green_*
  Sec. 2   Monte Carlo over h; main output G_ij(tau_l) on the slice grid;
           cost O(Lambda N^3)  -> Chain.sweep, Chain.gtau
The paper prints no sweep internals; the steps below (Metropolis ratio,
Sherman-Morrison update, slice wrap, UDV stabilisation, unequal-time G) are
the standard consequences of Eq. (3) derived in the docstrings.  Readings of
points the paper leaves open:
  R1  slices l = 1..L, B_l = E e^{V_l}, E = e^{-dtau K} (kinetic factor on the
      left, the order of Eq. (2)); the product index of Eq. (2) is read as
      running over L = beta/dtau factors.
  R2  K_ij = -t per nearest-neighbour bond in each of the four directions
      +-x, +-y; on a side of length 2 both directions reach the same site, so
      K_ij = -2t there (keeps eps_k = -2t (cos kx + cos ky)).  Lx, Ly >= 2.
  R3  spin-channel Ising HS field: cosh(lambda) = exp(dtau U / 2),
      e^{-dtau U (n_up - 1/2)(n_dn - 1/2)} = C sum_s e^{lambda s (n_up - n_dn)},
      C = exp(-dtau U / 4) / 2; V_l^sigma = sigma lambda diag(s_l).
  R4  single-site Metropolis, acceptance iff u < R with R = R_up R_dn
      (min(1, R) is implied), sites i = 0..N-1 within a slice, slices
      ascending; u from Philox4x32-10 (R6).
  R5  stabilisation: the running G is replaced by a freshly stabilised one
      after every slice l with l % n_s == 0 and after l = L; equal-time
      observables are measured at those points.
  R6  random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low
      32 bits, seed high 32 bits); proposal at (site i, 0-based slice l0,
      sweep w, chain c) uses counter (i + N l0, w, c, 0) and
      u = ((x0 << 32 | x1) >> 11) * 2^-53; the initial field uses counter
      (i + N l0, 0xFFFFFFFF, c, 1) and s = +1 iff x0 is odd.
  R7  G_ij(tau) = <c_i(tau) c_j^dag> (non-negative convention); the paper's
      Eq. (4) Green function is its negative.
  R8  G(tau_l) on l = 0..L with origin tau = 0; the momentum-resolved output
      is Re G_k(tau_l) = (1/N) sum_ij cos(k.(r_i - r_j)) G_ij(l, 0),
      averaged over the two spins.
  R14 the real-space spin correlation of Sec. 4 (Fig. 5) is read as the
      longitudinal C(r) = (1/N) sum_i <S^z_i S^z_{i+r}>, S^z = (n_up - n_dn)/2,
      averaged over translations and accumulated at the R5 measurement points;
      the paper names neither the component nor the normalisation.
  R15 dtau -> 0 extrapolation of G_k(tau) (Sec. 3, Fig. 2): the alignment
      spline is not given (its footnote is missing) and is read as the
      not-a-knot cubic spline on each run's uniform grid; the pointwise
      extrapolation is a least-squares fit in dtau^2, the order of the
      Trotter error of the momentum-diagonal G_k(tau) (the K/V split is
      similar to the symmetric one there).
  R16 Matsubara transform (Eq. 5) and Dyson equation (Eq. 6): the transform
      is taken of the standard-sign G(tau) = -<T c(tau) c^dag> (the negative
      of R7's) with kernel e^{+i w_n tau}, which is what makes Eq. 6 give
      Sigma = 0 at U = 0; the printed exponent e^{-i w_n tau} with either
      sign of G would leave Sigma = 2 i w_n or -2 eps_k there.  mu = 0 (half
      filling with the (n - 1/2) form of Eq. 1).  The quasi-continuous G(tau)
      between samples is the not-a-knot cubic spline of R15.
  R17 time-origin averaging of G(tau) (an estimator, not stated in the
      paper): the mean of G(tau_0 + tau, tau_0) over origins tau_0 on the
      slice grid, each evaluated as G(tau) of the cyclically rotated field.
  R18 the correlation length of Sec. 4 (Fig. 5, "an exponential fit" to the
      real-space spin correlation) is read as the least-squares line through
      (|r|, ln((-1)^(dx+dy) C(r))) over 0 < |r| <= dmax, |r| the minimum-image
      distance, points with a non-positive staggered value left out;
      xi = -1/slope.  The paper names neither the form, the distance nor the
      fitted range.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.interpolate
import scipy.linalg

__all__ = [
    "MASK32", "philox4x32_10", "philox4x32_10_np", "uniform53", "initial_field",
    "proposal_uniforms", "site_index", "sublattice_sign", "hopping_matrix",
    "adjacency", "dispersion", "exp_hopping", "hs_lambda", "hs_prefactor",
    "n_slices", "b_matrix", "b_inverse", "udv_chain", "green_from_udv",
    "two_stack_green", "Params", "Chain", "observables_from_g",
    "spin_correlation_from_g", "min_image_distance", "correlation_length",
    "momentum_diag", "weight_log", "trotter_extrapolate", "matsubara_sigma",
]

MASK32 = 0xFFFFFFFF

# ---------------------------------------------------------------------------
# Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
# "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Reading R6.
# ---------------------------------------------------------------------------
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9  # golden ratio
_PHILOX_W1 = 0xBB67AE85  # sqrt(3) - 1


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on Python ints: 4-word counter, 2-word key."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in ctr)
    k0, k1 = (int(v) & MASK32 for v in key)
    for _ in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & MASK32,
                          (p0 >> 32) ^ c3 ^ k1, p0 & MASK32)
        k0 = (k0 + _PHILOX_W0) & MASK32
        k1 = (k1 + _PHILOX_W1) & MASK32
    return c0, c1, c2, c3


def philox4x32_10_np(c0, c1, c2, c3, k0, k1):
    """Same generator, vectorised over numpy arrays of counters (uint64 math)."""
    m = np.uint64(MASK32)
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & m for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    for _ in range(10):
        p0 = np.uint64(_PHILOX_M0) * c0
        p1 = np.uint64(_PHILOX_M1) * c2
        c0, c1, c2, c3 = ((p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & m,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & m)
        k0 = np.uint64((int(k0) + _PHILOX_W0) & MASK32)
        k1 = np.uint64((int(k1) + _PHILOX_W1) & MASK32)
    return c0, c1, c2, c3


def uniform53(x0, x1):
    """Uniform double in [0, 1) from two 32-bit words (53 random bits)."""
    x0 = np.asarray(x0, dtype=np.uint64)
    x1 = np.asarray(x1, dtype=np.uint64)
    bits = ((x0 << np.uint64(32)) | x1) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53)


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32


def initial_field(seed, chain, N, L):
    """Initial Ising field s[l0, i] in {-1, +1} (int8), reading R6."""
    k0, k1 = _key(seed)
    l0, i = np.meshgrid(np.arange(L), np.arange(N), indexing="ij")
    x0, _, _, _ = philox4x32_10_np(i + N * l0, MASK32, chain, 1, k0, k1)
    return np.where((x0 & np.uint64(1)) == 1, 1, -1).astype(np.int8)


def proposal_uniforms(seed, chain, sweep, l0, N):
    """Uniforms u_i for the N proposals of 0-based slice l0 in a sweep (R6)."""
    k0, k1 = _key(seed)
    i = np.arange(N)
    x0, x1, _, _ = philox4x32_10_np(i + N * l0, sweep, chain, 0, k0, k1)
    return uniform53(x0, x1)


# ---------------------------------------------------------------------------
# Lattice and hopping, Eq. (1): H_t = -t sum_<ij>,sigma c^dag_i c_j, periodic.
# ---------------------------------------------------------------------------
def site_index(x, y, Lx):
    """Site i = x + Lx*y (x runs fastest)."""
    return x + Lx * y


def sublattice_sign(Lx, Ly):
    """p_i = (-1)^(x+y), the bipartite sign used by the particle-hole map."""
    y, x = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    return ((-1.0) ** (x + y)).reshape(-1)


def hopping_matrix(Lx, Ly, t):
    """K with H_t = sum_ij K_ij c^dag_i c_j (Eq. (1)), reading R2."""
    if Lx < 2 or Ly < 2:
        raise ValueError("Lx and Ly must be >= 2")
    N = Lx * Ly
    K = np.zeros((N, N))
    for y in range(Ly):
        for x in range(Lx):
            i = site_index(x, y, Lx)
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                j = site_index((x + dx) % Lx, (y + dy) % Ly, Lx)
                K[j, i] -= t
    return K


def adjacency(Lx, Ly):
    """A = -K/t: bond multiplicities (so that dK/dt = -A)."""
    return -hopping_matrix(Lx, Ly, 1.0)


def dispersion(Lx, Ly, t):
    """eps_k = -2t (cos kx + cos ky), k index kx + Lx*ky, k = 2 pi (kx/Lx, ky/Ly)."""
    ky, kx = np.meshgrid(np.arange(Ly), np.arange(Lx), indexing="ij")
    return (-2.0 * t * (np.cos(2 * np.pi * kx / Lx) + np.cos(2 * np.pi * ky / Ly))).reshape(-1)


def exp_hopping(K, dtau):
    """E = e^{-dtau K} and E^{-1} = e^{+dtau K} by symmetric eigendecomposition."""
    w, v = np.linalg.eigh(K)
    E = (v * np.exp(-dtau * w)) @ v.T
    Einv = (v * np.exp(dtau * w)) @ v.T
    return E, Einv


# ---------------------------------------------------------------------------
# Trotter slices (Eq. (2)) and the discrete HS transform (Sec. 2), R1 and R3.
# ---------------------------------------------------------------------------
def n_slices(beta, dtau):
    """L = beta/dtau; it must be an integer (to 1e-9)."""
    L = int(round(beta / dtau))
    if L < 1 or abs(beta / dtau - L) > 1e-9:
        raise ValueError("beta/dtau must be a positive integer")
    return L


def hs_lambda(U, dtau):
    """lambda with cosh(lambda) = exp(dtau U / 2)."""
    return math.acosh(math.exp(0.5 * dtau * U))


def hs_prefactor(U, dtau):
    """C in e^{-dtau U (n_up-1/2)(n_dn-1/2)} = C sum_s e^{lambda s (n_up-n_dn)}."""
    return 0.5 * math.exp(-0.25 * dtau * U)


def b_matrix(E, lam, sigma, s_l):
    """B_l^sigma = E e^{V_l}, V_l = sigma lambda diag(s_l)."""
    return E * np.exp(sigma * lam * np.asarray(s_l, dtype=np.float64))[None, :]


def b_inverse(Einv, lam, sigma, s_l):
    """(B_l^sigma)^{-1} = e^{-V_l} E^{-1}."""
    return np.exp(-sigma * lam * np.asarray(s_l, dtype=np.float64))[:, None] * Einv


# ---------------------------------------------------------------------------
# Stabilised products and Green functions (the O(Lambda N^3) matrix work of
# Sec. 2).  A chain A = X_m ... X_1 is kept as U diag(D) T with U orthogonal,
# D > 0 graded and T well conditioned; every n_s factors the partial product
# is re-orthogonalised by QR with column pivoting.
# ---------------------------------------------------------------------------
def udv_chain(mats, n_s):
    """UDT factors of mats[-1] @ ... @ mats[0] (mats[0] is applied first)."""
    N = mats[0].shape[0] if mats else 0
    U = np.eye(N)
    D = np.ones(N)
    T = np.eye(N)
    for start in range(0, len(mats), n_s):
        X = U * D[None, :]
        for Bm in mats[start:start + n_s]:
            X = Bm @ X
        Q, R, piv = scipy.linalg.qr(X, pivoting=True)
        d = np.abs(np.diag(R))
        Rn = R / d[:, None]
        RPt = np.empty_like(Rn)
        RPt[:, piv] = Rn  # (D^{-1} R) P^T, since X[:, piv] = Q R
        T = RPt @ T
        U, D = Q, d
    return U, D, T


def green_from_udv(U, D, T):
    """(I + U D T)^{-1} = (Db^{-1} U^T + Ds T)^{-1} Db^{-1} U^T, D = Db Ds."""
    Db = np.maximum(D, 1.0)
    Ds = np.minimum(D, 1.0)
    Mid = U.T / Db[:, None] + Ds[:, None] * T
    return np.linalg.solve(Mid, U.T / Db[:, None])


def two_stack_green(right, left):
    """G = (I + R L)^{-1} and G(l,0) = (R^{-1} + L)^{-1} from R = U_R D_R T_R and
    L^T = U_L D_L T_L; also returns Y = (I - G(0)) R^{-1} = L G.

    With D = Db Ds (Db = max(D,1), Ds = min(D,1)) and
      Mid = Db_R^{-1} (U_R^T U_L) Db_L^{-1} + Ds_R (T_R T_L^T) Ds_L,
    I + R L = U_R Db_R Mid Db_L U_L^T, hence
      G      = U_L Db_L^{-1} Mid^{-1} Db_R^{-1} U_R^T,
      G(l,0) = G R = U_L Db_L^{-1} Mid^{-1} Ds_R T_R,
      Y      = L G = T_L^T Ds_L Mid^{-1} Db_R^{-1} U_R^T.
    """
    UR, DR, TR = right
    UL, DL, TL = left
    DbR, DsR = np.maximum(DR, 1.0), np.minimum(DR, 1.0)
    DbL, DsL = np.maximum(DL, 1.0), np.minimum(DL, 1.0)
    Mid = (UR.T @ UL) / DbR[:, None] / DbL[None, :] + DsR[:, None] * (TR @ TL.T) * DsL[None, :]
    Minv = np.linalg.inv(Mid)
    G = (UL / DbL[None, :]) @ Minv @ (UR.T / DbR[:, None])
    Gl0 = (UL / DbL[None, :]) @ Minv @ (DsR[:, None] * TR)
    Y = (TL.T * DsL[None, :]) @ Minv @ (UR.T / DbR[:, None])
    return G, Gl0, Y


def weight_log(U, D, T):
    """log|det(I + U D T)| and its sign, split-D form of green_from_udv."""
    Db = np.maximum(D, 1.0)
    Ds = np.minimum(D, 1.0)
    Mid = U.T / Db[:, None] + Ds[:, None] * T
    sU, lU = np.linalg.slogdet(U)
    sM, lM = np.linalg.slogdet(Mid)
    return lU + np.sum(np.log(Db)) + lM, sU * sM


# ---------------------------------------------------------------------------
# Observables.
# ---------------------------------------------------------------------------
def observables_from_g(G_up, G_dn, K):
    """Per-site density, double occupancy and kinetic energy of one
    configuration from the equal-time G_sigma,ij = <c_i c_j^dag>:
      n    = (1/N) sum_i,sigma (1 - G_ii)
      docc = (1/N) sum_i (1 - G_up,ii)(1 - G_dn,ii)          (Wick)
      ekin = (1/N) sum_sigma sum_ij K_ij (delta_ij - G_ji)    (<c^dag_i c_j>)."""
    N = K.shape[0]
    n = (np.sum(1.0 - np.diag(G_up)) + np.sum(1.0 - np.diag(G_dn))) / N
    docc = np.sum((1.0 - np.diag(G_up)) * (1.0 - np.diag(G_dn))) / N
    ekin = 0.0
    for G in (G_up, G_dn):
        ekin += np.sum(K * (np.eye(N) - G.T))
    return np.array([n, docc, ekin / N])


def spin_correlation_from_g(G_up, G_dn, Lx, Ly):
    """Real-space equal-time spin correlation of one configuration, averaged
    over lattice translations (Sec. 4, Fig. 5; reading R14):
      C(r) = (1/N) sum_i <S^z_i S^z_{i+r}>,   S^z_i = (n_i,up - n_i,dn) / 2,
    r = (dx, dy) periodic, stored at index dx + Lx dy.  For a fixed Ising
    field the two spins are independent one-body problems, so Wick's theorem
    gives, with n_i,s = 1 - G_s,ii and <c^dag_i c_j> = delta_ij - G_s,ji,
      <n_i,s n_j,s'> = n_i,s n_j,s' + delta_ss' (delta_ij - G_s,ji) G_s,ij.
    Both spins are used as given (no particle-hole identity)."""
    N = Lx * Ly
    nu = 1.0 - np.diag(G_up)
    nd = 1.0 - np.diag(G_dn)
    x = np.arange(N) % Lx
    y = np.arange(N) // Lx
    i = np.arange(N)
    C = np.zeros(N)
    for dy in range(Ly):
        for dx in range(Lx):
            j = site_index((x + dx) % Lx, (y + dy) % Ly, Lx)
            d = (i == j).astype(np.float64)
            uu = nu[i] * nu[j] + (d - G_up[j, i]) * G_up[i, j]
            dd = nd[i] * nd[j] + (d - G_dn[j, i]) * G_dn[i, j]
            ud = nu[i] * nd[j]
            du = nd[i] * nu[j]
            C[site_index(dx, dy, Lx)] = np.sum(0.25 * (uu + dd - ud - du)) / N
    return C


def min_image_distance(Lx, Ly):
    """|r| of every displacement r = dx + Lx dy on the periodic cluster, in the
    minimum-image convention: sqrt(min(dx, Lx - dx)^2 + min(dy, Ly - dy)^2)."""
    d = np.empty(Lx * Ly)
    for dy in range(Ly):
        for dx in range(Lx):
            ax, ay = min(dx, Lx - dx), min(dy, Ly - dy)
            d[site_index(dx, dy, Lx)] = math.sqrt(ax * ax + ay * ay)
    return d


def correlation_length(C, Lx, Ly, dmax=None):
    """Spin correlation length xi of Sec. 4 (Fig. 5) from one real-space
    C(r) (index dx + Lx dy, as spin_correlation_from_g), by the exponential fit
    the paper names (reading R18; the paper gives neither the fitted form,
    the distance nor the range):
      * staggered magnitude c(r) = (-1)^(dx + dy) C(r), positive where the
        correlations are antiferromagnetic, as at half filling;
      * distance d(r) = min_image_distance;
      * least squares, unweighted, of ln c(r) = a - d(r) / xi over every r
        with 0 < d(r) <= dmax and c(r) > 0 (dmax = min(Lx, Ly) / 2 if None),
        i.e. the straight line through the points (d, ln c):
          b = (n S_dy - S_d S_y) / (n S_dd - S_d^2);
    xi = -1 / b for b < 0, +inf for b >= 0 (no decay within the cluster), and
    nan when the points have fewer than two distinct distances."""
    C = np.asarray(C, dtype=np.float64)
    if dmax is None:
        dmax = 0.5 * min(Lx, Ly)
    d = min_image_distance(Lx, Ly)
    sgn = np.array([(-1.0) ** (i % Lx + i // Lx) for i in range(Lx * Ly)])
    c = sgn * C
    pts = [(d[r], math.log(c[r])) for r in range(Lx * Ly) if 0.0 < d[r] <= dmax and c[r] > 0.0]
    n = len(pts)
    if len({p[0] for p in pts}) < 2:
        return float("nan")
    sd = sum(p[0] for p in pts)
    sy = sum(p[1] for p in pts)
    sdd = sum(p[0] * p[0] for p in pts)
    sdy = sum(p[0] * p[1] for p in pts)
    den = n * sdd - sd * sd
    if not den > 0.0:
        return float("nan")
    b = (n * sdy - sd * sy) / den
    return -1.0 / b if b < 0.0 else float("inf")


def momentum_diag(X, Lx, Ly):
    """Re X_k = (1/N) sum_ij cos(k.(r_i - r_j)) X_ij for all k (index kx + Lx ky).
    Written as the sum over separations r = r_i - r_j first, then cosines."""
    N = Lx * Ly
    g = np.zeros((Ly, Lx))
    Xg = X.reshape(Ly, Lx, Ly, Lx)  # [yi, xi, yj, xj]
    for yj in range(Ly):
        for xj in range(Lx):
            col = Xg[:, :, yj, xj]  # indexed by (yi, xi)
            g += np.roll(np.roll(col, -yj, axis=0), -xj, axis=1)
    ky, kx, ry, rx = np.meshgrid(np.arange(Ly), np.arange(Lx), np.arange(Ly), np.arange(Lx),
                                 indexing="ij")
    phase = np.cos(2 * np.pi * (kx * rx / Lx + ky * ry / Ly))
    return (phase * g[None, None, :, :]).sum(axis=(2, 3)).reshape(-1) / N


# ---------------------------------------------------------------------------
# Trotter extrapolation of G_k(tau) (Sec. 3, Fig. 2; reading R15).
# ---------------------------------------------------------------------------
def trotter_extrapolate(dtaus, gks, beta, M):
    """dtau -> 0 limit of G_k(tau) from runs at several time steps.
    Run r has time step dtaus[r] and data gks[r] of shape [C_r, L_r + 1, N]
    (G_k(tau_l) on its own grid tau_l = l dtau_r, per chain).  Steps, as the
    paper orders them: average each run over its chains; put every run on
    the common fine grid tau_m = m beta / M (m = 0..M) with a cubic spline
    through its L_r + 1 points (not-a-knot ends); at every (tau_m, k) fit the
    runs by least squares to a + b dtau^2 and keep a.  One run returns its
    interpolation.  Returns [M + 1, N]."""
    taus = np.arange(M + 1) * (beta / M)
    vals = []
    for dt, g in zip(dtaus, gks):
        g = np.asarray(g, dtype=np.float64)
        mean = g.mean(axis=0)
        grid = np.arange(g.shape[1]) * dt
        vals.append(scipy.interpolate.CubicSpline(grid, mean, axis=0, bc_type="not-a-knot")(taus))
    vals = np.array(vals)
    if len(vals) == 1:
        return vals[0]
    A = np.stack([np.ones(len(dtaus)), np.asarray(dtaus, dtype=np.float64) ** 2], axis=1)
    coef = np.linalg.lstsq(A, vals.reshape(len(dtaus), -1), rcond=None)[0]
    return coef[0].reshape(M + 1, -1)


# ---------------------------------------------------------------------------
# Matsubara Green function and self-energy (Sec. 3, Eqs. 5-6; reading R16).
# ---------------------------------------------------------------------------
def matsubara_sigma(gk, beta, Lx, Ly, t, n_freq, nodes=12):
    """G_k(i w_n) and Sigma_k(i w_n), w_n = (2n + 1) pi / beta, n < n_freq,
    from G_k(tau) sampled on tau_m = m beta / M (gk [M + 1, N], the
    non-negative convention <c_k(tau) c_k^dag> of R7, e.g. the output of
    trotter_extrapolate).  Steps, in the order of Eqs. 5-6: the not-a-knot
    cubic spline S_k(tau) through the samples; the standard-sign transform
      G_k(i w_n) = - int_0^beta S_k(tau) e^{i w_n tau} dtau,
    each grid interval integrated by Gauss-Legendre quadrature with `nodes`
    points (exact to rounding while w_n h stays of order a few); the Dyson
    equation at half filling (mu = 0),
      Sigma_k(i w_n) = i w_n - eps_k - 1 / G_k(i w_n).
    Returns (G [n_freq, N], Sigma [n_freq, N]), complex."""
    gk = np.asarray(gk, dtype=np.float64)
    M = gk.shape[0] - 1
    h = beta / M
    spline = scipy.interpolate.CubicSpline(np.arange(M + 1) * h, gk, axis=0, bc_type="not-a-knot")
    x, w = np.polynomial.legendre.leggauss(nodes)
    tau = (np.arange(M)[:, None] * h + 0.5 * h * (x[None, :] + 1.0)).reshape(-1)  # all nodes
    wt = np.tile(0.5 * h * w, M)
    S = spline(tau)  # [M * nodes, N]
    wn = (2 * np.arange(n_freq) + 1) * np.pi / beta
    G = np.empty((n_freq, gk.shape[1]), dtype=np.complex128)
    for n in range(n_freq):
        G[n] = -np.sum((wt * np.exp(1j * wn[n] * tau))[:, None] * S, axis=0)
    eps = dispersion(Lx, Ly, t)
    sigma = 1j * wn[:, None] - eps[None, :] - 1.0 / G
    return G, sigma


# ---------------------------------------------------------------------------
# One Markov chain.
# ---------------------------------------------------------------------------
class Params:
    """Physical and algorithmic parameters of one chain (Eqs. (1)-(3))."""

    def __init__(self, Lx, Ly, t, U, beta, dtau, n_s=10):
        self.Lx, self.Ly = int(Lx), int(Ly)
        self.N = self.Lx * self.Ly
        self.t, self.U, self.beta, self.dtau = float(t), float(U), float(beta), float(dtau)
        self.L = n_slices(beta, dtau)
        self.n_s = int(n_s)
        if self.n_s < 1:
            raise ValueError("n_s must be >= 1")
        self.K = hopping_matrix(self.Lx, self.Ly, self.t)
        self.E, self.Einv = exp_hopping(self.K, self.dtau)
        self.lam = hs_lambda(self.U, self.dtau)


class Chain:
    """A single BSS-DQMC Markov chain, both spins explicit.

    G(l) = (I + B_l ... B_1 B_L ... B_{l+1})^{-1}; slice l (1-based) is
    updated with G(l-1), whose rightmost factor is B_l = E e^{V_l}.
    """

    def __init__(self, params: Params, seed=0, chain=0, field=None):
        self.p = params
        self.seed = int(seed)
        self.chain = int(chain)
        self.sweeps_done = 0
        if field is None:
            self.field = initial_field(self.seed, self.chain, params.N, params.L)
        else:
            self.field = np.array(field, dtype=np.int8).reshape(params.L, params.N).copy()

    # -- B matrices --------------------------------------------------------
    def B(self, l, sigma):
        """B_l for 1-based slice l."""
        return b_matrix(self.p.E, self.p.lam, sigma, self.field[l - 1])

    def Binv(self, l, sigma):
        return b_inverse(self.p.Einv, self.p.lam, sigma, self.field[l - 1])

    # -- stabilised Green functions, from scratch ---------------------------
    def right_udv(self, l, sigma):
        """R_l = B_l ... B_1 (identity for l = 0)."""
        return udv_chain([self.B(m, sigma) for m in range(1, l + 1)], self.p.n_s) if l > 0 \
            else (np.eye(self.p.N), np.ones(self.p.N), np.eye(self.p.N))

    def left_udv(self, l, sigma):
        """UDT factors of L_l^T where L_l = B_L ... B_{l+1} (identity for l = L)."""
        L = self.p.L
        mats = [self.B(m, sigma).T for m in range(L, l, -1)]
        return udv_chain(mats, self.p.n_s) if mats else \
            (np.eye(self.p.N), np.ones(self.p.N), np.eye(self.p.N))

    def green(self, l, sigma):
        """Equal-time G(l) from the cyclic chain B_l..B_1 B_L..B_{l+1}."""
        L = self.p.L
        order = list(range(l + 1, L + 1)) + list(range(1, l + 1))  # applied first -> last
        U, D, T = udv_chain([self.B(m, sigma) for m in order], self.p.n_s)
        return green_from_udv(U, D, T)

    def logdet(self, sigma):
        """log|det M_sigma| and sign, M = I + B_L ... B_1 (Eq. (3))."""
        U, D, T = udv_chain([self.B(m, sigma) for m in range(1, self.p.L + 1)], self.p.n_s)
        return weight_log(U, D, T)

    # -- Monte Carlo --------------------------------------------------------
    def checkpoint(self, l):
        return l % self.p.n_s == 0 or l == self.p.L

    def sweep(self, measure=True):
        """One Metropolis sweep over all (slice, site) pairs (R4, R5).

        Ratio (det M'/det M for s_il -> -s_il, with e^{V'} = e^{V}(I + D e_i e_i^T)):
          Delta_sigma = exp(-2 sigma lambda s_il) - 1,
          R_sigma = 1 + Delta_sigma (1 - G_sigma,ii),   R = R_up R_dn.
        Accepted flip, Sherman-Morrison:
          G <- G - (Delta/R_sigma) (I - G) e_i e_i^T G.
        Wrap to the next slice: G(l) = B_l G(l-1) B_l^{-1}.
        """
        p = self.p
        N, L, lam = p.N, p.L, p.lam
        w = self.sweeps_done
        G = {s: self.green(0, s) for s in (1, -1)}
        accepted = 0
        drift = 0.0
        obs = []
        spin = []
        ratios = []
        for l in range(1, L + 1):
            u = proposal_uniforms(self.seed, self.chain, w, l - 1, N)
            for i in range(N):
                s = float(self.field[l - 1, i])
                delta = {sg: math.exp(-2.0 * sg * lam * s) - 1.0 for sg in (1, -1)}
                r = {sg: 1.0 + delta[sg] * (1.0 - G[sg][i, i]) for sg in (1, -1)}
                R = r[1] * r[-1]
                ratios.append(R)
                if u[i] < R:
                    accepted += 1
                    self.field[l - 1, i] = -self.field[l - 1, i]
                    for sg in (1, -1):
                        col = -G[sg][:, i].copy()
                        col[i] += 1.0
                        G[sg] = G[sg] - (delta[sg] / r[sg]) * np.outer(col, G[sg][i, :])
            for sg in (1, -1):
                G[sg] = self.B(l, sg) @ G[sg] @ self.Binv(l, sg)
            if self.checkpoint(l):
                for sg in (1, -1):
                    Gf = self.green(l, sg)
                    drift = max(drift, np.max(np.abs(G[sg] - Gf)) / np.max(np.abs(Gf)))
                    G[sg] = Gf
                if measure:
                    obs.append(observables_from_g(G[1], G[-1], p.K))
                    spin.append(spin_correlation_from_g(G[1], G[-1], p.Lx, p.Ly))
        self.sweeps_done += 1
        return {"accepted": accepted, "drift": drift, "obs": obs, "spin": spin,
                "ratios": np.array(ratios), "G_up": G[1], "G_dn": G[-1]}

    # -- unequal-time Green function (Sec. 2: G_ij(tau_l) on the slice grid) --
    def gtau_matrices(self, sigma):
        """G(l,0) = B_l ... B_1 G(0) for l = 0..L: fresh at every checkpoint
        c (l % n_s == 0 or l == L) as (R_c^{-1} + L_c)^{-1}, propagated by
        G(l,0) = B_l G(l-1,0) in between."""
        p = self.p
        out = []
        Gl0 = None
        for l in range(0, p.L + 1):
            if l == 0 or self.checkpoint(l):
                _, Gl0, _ = two_stack_green(self.right_udv(l, sigma), self.left_udv(l, sigma))
            else:
                Gl0 = self.B(l, sigma) @ Gl0
            out.append(Gl0)
        return out

    def gtau(self):
        """Spin-averaged Re G_k(tau_l), shape [L+1, N] (R8)."""
        p = self.p
        acc = np.zeros((p.L + 1, p.N))
        for sg in (1, -1):
            for l, X in enumerate(self.gtau_matrices(sg)):
                acc[l] += 0.5 * momentum_diag(X, p.Lx, p.Ly)
        return acc

    def gtau_origins(self, n_origins):
        """Time-origin average of G_k(tau) (reading R17): the mean over the
        origins tau_0 = s dtau, s = (o L) // n_origins (o < n_origins), of
        G_k(tau_0 + tau, tau_0).  By the cyclic invariance of the trace in
        Eq. (3) that is G_k(tau) of the field rotated by s slices, whose slice
        l is slice l + s (mod L) of this one; its weight is the same."""
        p = self.p
        acc = np.zeros((p.L + 1, p.N))
        for o in range(n_origins):
            s = (o * p.L) // n_origins
            acc += Chain(p, field=np.roll(self.field, -s, axis=0)).gtau()
        return acc / n_origins

    # -- derivatives of log W = log|det M_up| + log|det M_dn| ---------------
    def logw(self):
        return sum(self.logdet(s)[0] for s in (1, -1))

    def grad(self):
        """d log W / dt and d log W / d lambda for the current field.

        From d log det M = tr(M^{-1} dM) with M = I + B_L ... B_1:
          dB_l/dt      = dtau A B_l      (E = e^{dtau t A}, K = -t A)
            -> d log det M_sigma / dt = dtau sum_l tr[A (I - G_sigma(l))]
          dB_l/dlambda = B_l sigma diag(s_l)
            -> d log det M_sigma / dlambda = sigma sum_il s_il (1 - G_sigma,ii(l-1)).
        """
        p = self.p
        A = adjacency(p.Lx, p.Ly)
        dt = 0.0
        dlam = 0.0
        for sg in (1, -1):
            for l in range(1, p.L + 1):
                Gl = self.green(l, sg)
                dt += p.dtau * np.sum(A * (np.eye(p.N) - Gl).T)
                Gm = self.green(l - 1, sg)
                dlam += sg * np.sum(self.field[l - 1] * (1.0 - np.diag(Gm)))
        return dt, dlam
