"""Pins of the oracle against facts fixed by the paper and by mathematics.

Each test compares the oracle with something that is not the oracle:
published known-answer vectors, closed forms, the exact Fock-space trace of
Eq. (2), brute-force sums over all fields of Eq. (3), direct determinants,
finite differences, and symmetry identities of the half-filled bipartite
model.  None of these recomputes an oracle formula a second way.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import dqmc as o
from tests import enumerate_fields as en
from tests import fock


# --------------------------------------------------------------------------
# Philox4x32-10: known-answer vectors published with the Random123 library
# (Salmon et al., SC'11), stored in tests/golden/philox4x32_10_kat.txt.
# --------------------------------------------------------------------------
def _kat_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].split()
        if len(line) == 10:
            rows.append([int(v, 16) for v in line])
    assert rows
    return rows


def test_philox_known_answers():
    for r in _kat_rows():
        ctr, key, out = r[0:4], r[4:6], r[6:10]
        assert list(o.philox4x32_10(ctr, key)) == out


def test_philox_vectorised_matches_scalar():
    rng = np.random.default_rng(1)
    c = rng.integers(0, 2**32, size=(4, 50), dtype=np.uint64)
    k = (0x12345678, 0x9ABCDEF0)
    vec = o.philox4x32_10_np(c[0], c[1], c[2], c[3], *k)
    for j in range(50):
        assert tuple(int(v[j]) for v in vec) == o.philox4x32_10(tuple(int(x) for x in c[:, j]), k)


def test_uniform53_edges():
    assert o.uniform53(0, 0) == 0.0
    top = float(o.uniform53(0xFFFFFFFF, 0xFFFFFFFF))
    assert top < 1.0 and top == 1.0 - 2.0 ** -53


def test_initial_field_is_balanced_and_seeded():
    f0 = o.initial_field(0, 0, 64, 100)
    f1 = o.initial_field(0, 1, 64, 100)
    assert set(np.unique(f0)) == {-1, 1}
    assert abs(f0.mean()) < 0.05
    assert (f0 != f1).any()
    assert (o.initial_field(0, 0, 64, 100) == f0).all()


# --------------------------------------------------------------------------
# Eq. (1): lattice and hopping.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("Lx,Ly", [(2, 2), (3, 2), (4, 4), (6, 4), (5, 3)])
def test_hopping_spectrum_is_cosine_band(Lx, Ly):
    K = o.hopping_matrix(Lx, Ly, 0.25)
    ev = np.sort(np.linalg.eigvalsh(K))
    closed = np.sort(-2 * 0.25 * np.add.outer(np.cos(2 * np.pi * np.arange(Ly) / Ly),
                                              np.cos(2 * np.pi * np.arange(Lx) / Lx)).ravel())
    np.testing.assert_allclose(ev, closed, atol=1e-13)
    np.testing.assert_allclose(np.sort(o.dispersion(Lx, Ly, 0.25)), closed, atol=1e-13)


def test_hopping_matches_fock_bond_list():
    K = o.hopping_matrix(4, 2, 0.3)
    K2 = np.zeros_like(K)
    for j, i in fock.bonds(4, 2):
        K2[j, i] -= 0.3
    assert np.array_equal(K, K2)


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (4, 4), (6, 2)])
def test_bipartite_sign_flips_hopping(Lx, Ly):
    K = o.hopping_matrix(Lx, Ly, 0.25)
    P = np.diag(o.sublattice_sign(Lx, Ly))
    np.testing.assert_array_equal(P @ K @ P, -K)


def test_exp_hopping_against_expm():
    K = o.hopping_matrix(4, 4, 0.25)
    E, Einv = o.exp_hopping(K, 0.125)
    np.testing.assert_allclose(E, scipy.linalg.expm(-0.125 * K), atol=1e-14)
    np.testing.assert_allclose(E @ Einv, np.eye(16), atol=1e-14)


# --------------------------------------------------------------------------
# Sec. 2: discrete Hubbard-Stratonovich transform.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("U,dtau", [(1.0, 0.25), (2.0, 0.125), (3.0, 0.1), (8.0, 0.05)])
def test_hs_identity(U, dtau):
    lam = o.hs_lambda(U, dtau)
    C = o.hs_prefactor(U, dtau)
    for nu in (0, 1):
        for nd in (0, 1):
            lhs = math.exp(-dtau * U * (nu - 0.5) * (nd - 0.5))
            rhs = C * sum(math.exp(lam * s * (nu - nd)) for s in (-1, 1))
            assert rhs == pytest.approx(lhs, rel=1e-14)


# --------------------------------------------------------------------------
# Eq. (3) against Eq. (2): brute-force field sum == exact Trotter trace.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("Lx,Ly,t,U,dtau,L", [
    (2, 2, 0.25, 2.0, 0.25, 3),
    (2, 2, 0.25, 1.0, 0.5, 4),
    (2, 2, 0.4, 4.0, 0.2, 2),
    (2, 2, 0.25, 0.0, 0.25, 3),
    (3, 2, 0.25, 2.0, 0.25, 2),
    (2, 2, 0.25, 2.0, 0.1, 5),
])
def test_partition_function_enumeration_vs_fock(Lx, Ly, t, U, dtau, L):
    p = o.Params(Lx, Ly, t, U, L * dtau, dtau, n_s=2)
    _, _, Z, _ = en.enumerate_sum(p)
    Zf = fock.trotter_trace_sectors(Lx, Ly, t, U, dtau, L)
    assert Z == pytest.approx(Zf, rel=1e-12)


def test_fock_full_and_sector_traces_agree():
    F = fock.FockHubbard(2, 2, 0.25, 2.0, 0.25, 3)
    assert F.Z == pytest.approx(fock.trotter_trace_sectors(2, 2, 0.25, 2.0, 0.25, 3), rel=1e-12)


@pytest.fixture(scope="module")
def tiny():
    """2x2 cluster, L = 3: every field (4096) and the exact Fock space."""
    p = o.Params(2, 2, 0.25, 2.0, 0.75, 0.25, n_s=2)
    fields, w, Z, greens = en.enumerate_sum(p, want_g=True)
    F = fock.FockHubbard(2, 2, 0.25, 2.0, 0.25, 3)
    return p, fields, w, greens, F


def test_equal_time_observables_enumeration_vs_fock(tiny):
    p, fields, w, greens, F = tiny
    obs = np.array([o.observables_from_g(greens[1][f], greens[-1][f], p.K) for f in range(len(w))])
    mean = (w[:, None] * obs).sum(0) / w.sum()
    assert mean[0] == pytest.approx(1.0, abs=1e-13)
    assert mean[1] == pytest.approx(F.docc(), rel=1e-11)
    assert mean[2] == pytest.approx(F.ekin(), rel=1e-11)


def _fock_szsz_by_displacement(nu, nd, Lx, Ly):
    """Diagonal of (1/N) sum_i S^z_i S^z_{i+r} in the occupation basis, one
    row per displacement r = dx + Lx dy, from the occupation arrays alone."""
    N = Lx * Ly
    m = 0.5 * (nu - nd)
    out = np.empty((N, nu.shape[0]))
    for dy in range(Ly):
        for dx in range(Lx):
            shift = [((i % Lx + dx) % Lx) + Lx * ((i // Lx + dy) % Ly) for i in range(N)]
            out[dx + Lx * dy] = np.sum(m * m[:, shift], axis=1) / N
    return out


def test_spin_correlation_enumeration_vs_fock(tiny):
    """Weighted field average of the oracle's C(r) == Tr[T^L S^z_i S^z_{i+r}]/Z
    of the interacting model, for every displacement of the 2x2 cluster."""
    p, fields, w, greens, F = tiny
    C = np.array([o.spin_correlation_from_g(greens[1][f], greens[-1][f], p.Lx, p.Ly)
                  for f in range(len(w))])
    mean = (w[:, None] * C).sum(0) / w.sum()
    ops = _fock_szsz_by_displacement(F.nu, F.nd, p.Lx, p.Ly)
    exact = np.array([F.expect(np.diag(op)) for op in ops])
    np.testing.assert_allclose(mean, exact, rtol=1e-11, atol=1e-14)
    assert exact[0] > 0.0 and exact[p.Lx + 0] < 0.0  # local moment; nearest neighbours anti-aligned


def test_spin_correlation_single_field_vs_fock():
    """For ONE Ising field the fermions are free: C(r) from the oracle's Wick
    contraction equals the Fock-space trace Tr[P O_r]/Tr[P] with
    P = prod_l (e^{-dtau h} x e^{-dtau h}) e^{lambda s_l (n_up - n_dn)},
    built from the occupation basis, for random fields of a 3x2 cluster.
    Tr P = det(I + A_up) det(I + A_dn) pins the Fock product itself."""
    Lx, Ly, L = 3, 2, 3
    p = o.Params(Lx, Ly, 0.25, 3.0, L * 0.2, 0.2, n_s=1)
    N = p.N
    occ = fock.occupations(N)
    eh = fock._expm_sym(fock.single_spin_hopping(Lx, Ly, p.t), -p.dtau)
    ops = _fock_szsz_by_displacement(
        np.tile(occ, (1 << N, 1)), np.repeat(occ, 1 << N, axis=0), Lx, Ly)
    rng = np.random.default_rng(7)
    for _ in range(3):
        s = rng.choice([-1, 1], size=(L, N)).astype(np.int8)
        P = np.eye(1 << (2 * N))
        for l in range(L):
            hu = np.exp(p.lam * (occ @ s[l].astype(np.float64)))   # up:  e^{+lambda s.n}
            hd = np.exp(-p.lam * (occ @ s[l].astype(np.float64)))  # down: e^{-lambda s.n}
            T = np.kron(eh * hd[None, :], eh * hu[None, :])          # down slow, up fast
            P = T @ P
        trP = np.trace(P)
        G, det = {}, {}
        for sg in (1, -1):
            A = np.eye(N)
            for l in range(L):
                A = o.b_matrix(p.E, p.lam, sg, s[l]) @ A
            det[sg] = np.linalg.det(np.eye(N) + A)
            G[sg] = np.linalg.inv(np.eye(N) + A)
        assert trP == pytest.approx(det[1] * det[-1], rel=1e-10)
        exact = np.array([np.sum(np.diag(P) * op) for op in ops]) / trP
        got = o.spin_correlation_from_g(G[1], G[-1], Lx, Ly)
        np.testing.assert_allclose(got, exact, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_unequal_time_green_enumeration_vs_fock(tiny, l):
    """Weighted field average of the oracle's G(l,0) == Tr[T^{L-l} c_i T^l c_j^dag]/Z."""
    p, fields, w, _, F = tiny
    acc = np.zeros((p.N, p.N))
    for f in range(len(w)):
        ch = o.Chain(p, field=fields[f])
        acc += w[f] * ch.gtau_matrices(1)[l]
    np.testing.assert_allclose(acc / w.sum(), F.gtau_up(l), atol=1e-12)


# --------------------------------------------------------------------------
# Metropolis ratio and Sherman-Morrison update against direct determinants.
# --------------------------------------------------------------------------
def _direct_M(p, field, sigma):
    A = np.eye(p.N)
    for l in range(p.L):
        A = o.b_matrix(p.E, p.lam, sigma, field[l]) @ A
    return np.eye(p.N) + A


def test_metropolis_ratio_and_update_vs_determinants():
    p = o.Params(4, 2, 0.25, 2.0, 1.0, 0.25, n_s=2)
    ch = o.Chain(p, seed=3)
    rng = np.random.default_rng(0)
    for _ in range(6):
        l = int(rng.integers(1, p.L + 1))
        i = int(rng.integers(0, p.N))
        for sg in (1, -1):
            G = ch.green(l - 1, sg)
            s = float(ch.field[l - 1, i])
            delta = math.exp(-2 * sg * p.lam * s) - 1
            R = 1 + delta * (1 - G[i, i])
            f2 = ch.field.copy()
            f2[l - 1, i] *= -1
            # det M'/det M with slice l rotated to the right end (cyclic invariance)
            rot = np.concatenate([ch.field[l - 1:], ch.field[:l - 1]])
            rot2 = np.concatenate([f2[l - 1:], f2[:l - 1]])
            ratio = np.linalg.det(_direct_M(p, rot2, sg)) / np.linalg.det(_direct_M(p, rot, sg))
            assert R == pytest.approx(ratio, rel=1e-12)
            col = -G[:, i].copy()
            col[i] += 1
            Gn = G - (delta / R) * np.outer(col, G[i, :])
            ch2 = o.Chain(p, field=f2)
            np.testing.assert_allclose(Gn, ch2.green(l - 1, sg), atol=1e-12)


def test_sweep_running_green_matches_fresh():
    """After each slice the wrapped, updated G equals the freshly stabilised G."""
    p = o.Params(4, 4, 0.25, 2.0, 2.0, 0.125, n_s=4)
    ch = o.Chain(p, seed=1)
    out = ch.sweep()
    assert out["accepted"] > 0
    assert out["drift"] < 1e-10
    np.testing.assert_allclose(out["G_up"], ch.green(p.L, 1), atol=1e-12)


def test_wrap_identity():
    p = o.Params(4, 2, 0.25, 2.0, 1.0, 0.25, n_s=2)
    ch = o.Chain(p, seed=5)
    for l in range(1, p.L + 1):
        for sg in (1, -1):
            G = ch.B(l, sg) @ ch.green(l - 1, sg) @ ch.Binv(l, sg)
            np.testing.assert_allclose(G, ch.green(l, sg), atol=1e-12)


# --------------------------------------------------------------------------
# Stabilisation.
# --------------------------------------------------------------------------
def test_stable_green_equals_naive_inverse_at_small_beta():
    p = o.Params(4, 4, 0.25, 2.0, 1.0, 0.125, n_s=3)
    ch = o.Chain(p, seed=2)
    for sg in (1, -1):
        np.testing.assert_allclose(ch.green(0, sg), np.linalg.inv(_direct_M(p, ch.field, sg)),
                                   atol=1e-12)


def test_stable_green_independent_of_grouping_at_large_beta():
    """At beta = 20 the naive product is singular in FP64; two stabilisation
    intervals must still agree."""
    G = []
    for n_s in (2, 8):
        p = o.Params(4, 4, 0.25, 2.0, 20.0, 0.125, n_s=n_s)
        G.append(o.Chain(p, seed=4).green(37, 1))
    np.testing.assert_allclose(G[0], G[1], atol=1e-10)
    assert np.all(np.isfinite(G[0]))


def test_two_stack_green_matches_cyclic_chain():
    p = o.Params(4, 4, 0.25, 2.0, 10.0, 0.125, n_s=8)
    ch = o.Chain(p, seed=7)
    for l in (0, 24, 40, p.L):
        G, _, _ = o.two_stack_green(ch.right_udv(l, 1), ch.left_udv(l, 1))
        np.testing.assert_allclose(G, ch.green(l, 1), atol=1e-11)


def test_two_stack_unequal_time_matches_direct_products():
    """G(l,0) = R_l G(0) and Y = (I - G(0)) R_l^{-1} by direct products (small beta)."""
    p = o.Params(4, 4, 0.25, 2.0, 1.0, 0.125, n_s=3)
    ch = o.Chain(p, seed=8)
    G0 = np.linalg.inv(_direct_M(p, ch.field, 1))
    for l in (0, 3, 5, p.L):
        R = np.eye(p.N)
        for m in range(1, l + 1):
            R = ch.B(m, 1) @ R
        _, Gl0, Y = o.two_stack_green(ch.right_udv(l, 1), ch.left_udv(l, 1))
        np.testing.assert_allclose(Gl0, R @ G0, atol=1e-12)
        np.testing.assert_allclose(Y, (np.eye(p.N) - G0) @ np.linalg.inv(R), atol=1e-12)


# --------------------------------------------------------------------------
# U = 0 closed form: lambda = 0, no Trotter error.
# --------------------------------------------------------------------------
def test_u0_closed_form_gtau_and_ratios():
    p = o.Params(4, 4, 0.25, 0.0, 4.0, 0.25, n_s=4)
    ch = o.Chain(p, seed=0)
    eps = o.dispersion(4, 4, 0.25)
    gt = ch.gtau()
    for l in range(p.L + 1):
        tau = l * p.dtau
        closed = np.exp(-tau * eps) / (1 + np.exp(-p.beta * eps))
        np.testing.assert_allclose(gt[l], closed, atol=1e-13)
    out = ch.sweep()
    np.testing.assert_allclose(out["ratios"], 1.0, atol=1e-14)
    assert out["accepted"] == p.N * p.L
    ekin = out["obs"][-1][2]
    exact = 2 * np.sum(eps / (1 + np.exp(p.beta * eps))) / p.N
    assert ekin == pytest.approx(exact, rel=1e-12)


# --------------------------------------------------------------------------
# Atomic limit t = 0: no Trotter error; per-site closed form.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("U,beta,dtau", [(2.0, 1.0, 0.25), (4.0, 0.5, 0.125)])
def test_atomic_limit_enumeration(U, beta, dtau):
    p = o.Params(2, 2, 0.0, U, beta, dtau, n_s=2)
    if p.N * p.L > 20:
        pytest.skip("too many fields")
    fields, w, Z, greens = en.enumerate_sum(p, want_g=True)
    docc = np.array([o.observables_from_g(greens[1][f], greens[-1][f], p.K)[1] for f in range(len(w))])
    d_exact = math.exp(-beta * U / 4) / (2 * math.exp(-beta * U / 4) + 2 * math.exp(beta * U / 4))
    assert (w * docc).sum() / w.sum() == pytest.approx(d_exact, rel=1e-12)
    z_site = 2 * math.exp(-beta * U / 4) + 2 * math.exp(beta * U / 4)
    assert Z == pytest.approx(z_site ** p.N, rel=1e-12)


# --------------------------------------------------------------------------
# Half filling on a bipartite lattice (the paper's case): particle-hole.
# --------------------------------------------------------------------------
def test_particle_hole_identities():
    p = o.Params(4, 4, 0.25, 2.0, 4.0, 0.125, n_s=5)
    ch = o.Chain(p, seed=9)
    P = np.diag(o.sublattice_sign(4, 4))
    for l in (0, 7, 20, p.L):
        Gu, Gd = ch.green(l, 1), ch.green(l, -1)
        np.testing.assert_allclose(Gd, np.eye(p.N) - P @ Gu.T @ P, atol=1e-12)
        assert o.observables_from_g(Gu, Gd, p.K)[0] == pytest.approx(1.0, abs=1e-12)
    lu, su = ch.logdet(1)
    ld, sd = ch.logdet(-1)
    assert ld - lu == pytest.approx(-p.lam * ch.field.astype(float).sum(), abs=1e-9)
    assert su * sd > 0


def test_gtau_boundary_sum():
    p = o.Params(4, 4, 0.25, 2.0, 2.0, 0.25, n_s=4)
    ch = o.Chain(p, seed=11)
    gt = ch.gtau()
    np.testing.assert_allclose(gt[0] + gt[-1], 1.0, atol=1e-12)


def test_gtau_spin_down_from_spin_up_backward_propagator():
    """Per configuration, G_dn(l,0) = P [(I - G_up(0)) R_l^{-1}]^T P, so the
    spin-down momentum diagonal at k is that of Y_l = (I - G_up(0)) R_l^{-1}
    at k + Q, Q = (pi, pi)."""
    Lx = Ly = 4
    p = o.Params(Lx, Ly, 0.25, 2.0, 4.0, 0.125, n_s=5)
    ch = o.Chain(p, seed=12)
    P = np.diag(o.sublattice_sign(Lx, Ly))
    kq = [((i % Lx + Lx // 2) % Lx) + Lx * (((i // Lx) + Ly // 2) % Ly) for i in range(p.N)]
    gdn = ch.gtau_matrices(-1)
    for l in (0, 5, 13, p.L):
        _, _, Y = o.two_stack_green(ch.right_udv(l, 1), ch.left_udv(l, 1))
        np.testing.assert_allclose(gdn[l], P @ Y.T @ P, atol=1e-11)
        np.testing.assert_allclose(o.momentum_diag(gdn[l], Lx, Ly),
                                   o.momentum_diag(Y, Lx, Ly)[kq], atol=1e-11)


def test_gtau_ensemble_ph_symmetry_by_enumeration():
    """<G_k(tau)> = <G_{k+Q}(beta - tau)> over all fields (2x2, L = 3)."""
    p = o.Params(2, 2, 0.25, 2.0, 0.75, 0.25, n_s=2)
    fields, w, _, _ = en.enumerate_sum(p)
    acc = np.zeros((p.L + 1, p.N))
    for f in range(len(w)):
        acc += w[f] * o.Chain(p, field=fields[f]).gtau()
    acc /= w.sum()
    kq = [((i % 2 + 1) % 2) + 2 * (((i // 2) + 1) % 2) for i in range(4)]
    np.testing.assert_allclose(acc[:, kq], acc[::-1, :], atol=1e-12)


# --------------------------------------------------------------------------
# Derivatives of log W.
# --------------------------------------------------------------------------
def _logw_with(Lx, Ly, t, U, beta, dtau, field, lam=None):
    p = o.Params(Lx, Ly, t, U, beta, dtau, n_s=4)
    if lam is not None:
        p.lam = lam
    return o.Chain(p, field=field).logw()


def test_gradients_vs_central_differences():
    Lx, Ly, t, U, beta, dtau = 4, 2, 0.25, 2.0, 2.0, 0.125
    p = o.Params(Lx, Ly, t, U, beta, dtau, n_s=4)
    ch = o.Chain(p, seed=13)
    dt, dlam = ch.grad()
    h = 1e-5
    fd_t = (_logw_with(Lx, Ly, t + h, U, beta, dtau, ch.field)
            - _logw_with(Lx, Ly, t - h, U, beta, dtau, ch.field)) / (2 * h)
    fd_l = (_logw_with(Lx, Ly, t, U, beta, dtau, ch.field, p.lam + h)
            - _logw_with(Lx, Ly, t, U, beta, dtau, ch.field, p.lam - h)) / (2 * h)
    assert dt == pytest.approx(fd_t, rel=1e-7)
    assert dlam == pytest.approx(fd_l, rel=1e-7)


def test_t_gradient_expectation_is_hellmann_feynman():
    """<d log W/dt> over all fields == d ln Z_dtau/dt of the Fock trace."""
    Lx, Ly, t, U, dtau, L = 2, 2, 0.25, 2.0, 0.25, 3
    p = o.Params(Lx, Ly, t, U, L * dtau, dtau, n_s=2)
    fields, w, Z, _ = en.enumerate_sum(p)
    g = np.array([o.Chain(p, field=fields[f]).grad()[0] for f in range(len(w))])
    h = 1e-5
    zp = fock.trotter_trace_sectors(Lx, Ly, t + h, U, dtau, L)
    zm = fock.trotter_trace_sectors(Lx, Ly, t - h, U, dtau, L)
    assert (w * g).sum() / w.sum() == pytest.approx((math.log(zp) - math.log(zm)) / (2 * h), rel=1e-7)


def _docc_from_lambda_gradient(p, fields, w):
    """Double occupancy from the field average of d log W / d lambda.  With
    Z_dtau = C^{NL} sum_h W(h), d ln C/dU = -dtau/4 and (cosh lambda =
    e^{dtau U/2}) d lambda/dU = (dtau/2) coth lambda, equating
    d ln Z_dtau/dU = -beta sum_i <(n_up - 1/2)(n_dn - 1/2)> gives
      d = <n>/2 - coth(lambda) <d log W/d lambda> / (2 N L)."""
    dl = np.array([o.Chain(p, field=fields[f]).grad()[1] for f in range(len(w))])
    return dl, (w * dl).sum() / w.sum()


def test_lambda_gradient_expectation_is_double_occupancy(tiny):
    """<d log W/d lambda> over all fields of the 2x2 cluster (L = 3) turns into
    the exact Fock-space double occupancy through the relation above; a wrong
    sign of sigma, a wrong slice of G or a dropped spin in the oracle's
    lambda-gradient breaks it."""
    p, fields, w, greens, F = tiny
    _, mean = _docc_from_lambda_gradient(p, fields, w)
    d = 0.5 - mean / math.tanh(p.lam) / (2 * p.N * p.L)
    assert d == pytest.approx(F.docc(), rel=1e-11)


def test_lambda_gradient_double_occupancy_away_from_half_filling():
    """The same relation on the 3x2 cluster (L = 2, t = 1, U = 4, dtau = 0.5),
    whose odd ring makes it non-bipartite, so <n> != 1: the <n>/2 term is
    checked too."""
    Lx, Ly, t, U, dtau, L = 3, 2, 1.0, 4.0, 0.5, 2
    p = o.Params(Lx, Ly, t, U, L * dtau, dtau, n_s=2)
    fields, w, Z, greens = en.enumerate_sum(p, want_g=True)
    F = fock.FockHubbard(Lx, Ly, t, U, dtau, L)
    n = np.array([o.observables_from_g(greens[1][f], greens[-1][f], p.K)[0]
                  for f in range(len(w))])
    n_mean = (w * n).sum() / w.sum()
    n_fock = F.expect(np.diag(np.sum(F.nu + F.nd, axis=1))) / F.N
    assert n_mean == pytest.approx(n_fock, rel=1e-11)
    assert abs(n_mean - 1.0) > 1e-3  # the check below sees the <n> term
    _, mean = _docc_from_lambda_gradient(p, fields, w)
    d = 0.5 * n_mean - mean / math.tanh(p.lam) / (2 * p.N * p.L)
    assert d == pytest.approx(F.docc(), rel=1e-11)


# --------------------------------------------------------------------------
# Monte Carlo statistics: the Markov chain samples Eq. (3).
# --------------------------------------------------------------------------
def test_mc_double_occupancy_and_kinetic_energy_vs_exact():
    Lx, Ly, t, U, dtau, L = 2, 2, 0.25, 2.0, 0.25, 4
    F = fock.FockHubbard(Lx, Ly, t, U, dtau, L)
    p = o.Params(Lx, Ly, t, U, L * dtau, dtau, n_s=2)
    samples = []
    for c in range(4):
        ch = o.Chain(p, seed=100, chain=c)
        for _ in range(30):
            ch.sweep(measure=False)
        for _ in range(250):
            samples.append(np.mean(ch.sweep()["obs"], axis=0))
    s = np.array(samples).reshape(4, -1, 3)
    bins = s.reshape(4, 25, 10, 3).mean(axis=2).reshape(-1, 3)
    mean = bins.mean(0)
    err = bins.std(0, ddof=1) / math.sqrt(len(bins))
    assert abs(mean[1] - F.docc()) < 4 * err[1]
    assert abs(mean[2] - F.ekin()) < 4 * err[2]
    assert np.allclose(s[..., 0], 1.0, atol=1e-12)


# --------------------------------------------------------------------------
# dtau -> 0 extrapolation of G_k(tau) (Sec. 3, Fig. 2).
# --------------------------------------------------------------------------
def test_trotter_extrapolation_exact_for_cubic_data():
    """Runs whose data are cubics in tau with an exactly quadratic dtau
    dependence, y = P(tau) + Q(tau) dtau^2 plus chain noise that averages to
    zero: the not-a-knot spline reproduces cubics and the fit in dtau^2 is
    exact, so the result is P on the fine grid.  A natural spline, a fit in
    dtau, a shifted grid or a skipped chain average would all miss."""
    rng = np.random.default_rng(3)
    beta, N, C, M = 2.0, 5, 4, 37
    P = rng.standard_normal((4, N))
    Q = rng.standard_normal((4, N))
    cubic = lambda c, tau: sum(c[p][None, :] * tau[:, None] ** p for p in range(4))
    dts = [0.4, 0.2, 0.1]
    gks = []
    for dt in dts:
        tau = np.arange(int(round(beta / dt)) + 1) * dt
        y = cubic(P, tau) + cubic(Q, tau) * dt ** 2
        noise = rng.standard_normal((C, len(tau), N))
        gks.append(y[None] + noise - noise.mean(axis=0, keepdims=True))
    taus = np.arange(M + 1) * beta / M
    got = o.trotter_extrapolate(dts, gks, beta, M)
    np.testing.assert_allclose(got, cubic(P, taus), rtol=0, atol=1e-11)
    one = o.trotter_extrapolate(dts[:1], gks[:1], beta, M)
    np.testing.assert_allclose(one, cubic(P, taus) + cubic(Q, taus) * 0.16, rtol=0, atol=1e-11)


def test_trotter_extrapolation_u0_closed_form():
    """U = 0 has no Trotter error: runs sampled from the closed form
    G_k(tau) = e^{-tau eps_k} / (1 + e^{-beta eps_k}) at three time steps
    extrapolate to the closed form on the fine grid (spline error only)."""
    Lx, Ly, beta, M = 4, 4, 4.0, 64
    eps = o.dispersion(Lx, Ly, 0.25)
    closed = lambda tau: np.exp(-tau[:, None] * eps[None, :]) / (1.0 + np.exp(-beta * eps[None, :]))
    dts = [0.1, 0.05, 0.025]
    gks = [closed(np.arange(int(round(beta / dt)) + 1) * dt)[None] for dt in dts]
    got = o.trotter_extrapolate(dts, gks, beta, M)
    # cubic-spline error on a uniform grid: (5/384) h^4 max|d^4 G/d tau^4|, at most
    # (5/384) h^4 max|eps|^4 = 1.3e-6 for the coarsest run (h = 0.1, |eps| <= 4t = 1);
    # the fit weights of the three runs sum to 1 with absolute sum 4/3
    bound = (4.0 / 3.0) * (5.0 / 384.0) * dts[0] ** 4 * np.max(np.abs(eps)) ** 4
    np.testing.assert_allclose(got, closed(np.arange(M + 1) * beta / M), rtol=0, atol=bound)


def _gk_from_gij(G, Lx, Ly):
    N = Lx * Ly
    out = np.zeros(N)
    for ky in range(Ly):
        for kx in range(Lx):
            acc = 0.0
            for i in range(N):
                for j in range(N):
                    dx, dy = i % Lx - j % Lx, i // Lx - j // Lx
                    acc += math.cos(2 * math.pi * (kx * dx / Lx + ky * dy / Ly)) * G[i, j]
            out[kx + Lx * ky] = acc / N
    return out


def test_trotter_extrapolation_removes_fock_trotter_error():
    """2x2 Hubbard cluster at U = 2: Trotterised G_k(tau) from the Fock-space
    transfer matrices at L = 8, 12, 16, extrapolated, against the exact
    continuous-time Tr[e^{-(beta-tau)H} c_k e^{-tau H} c_k^dag] / Z.  The raw
    error falls like dtau^2; the extrapolation removes it to O(dtau^4) where
    all grids have points, and to spline accuracy in between."""
    Lx, Ly, t, U, beta, M = 2, 2, 0.25, 2.0, 2.0, 48
    N = Lx * Ly
    dts, gks = [], []
    for L in (8, 12, 16):
        F = fock.FockHubbard(Lx, Ly, t, U, beta / L, L)
        dts.append(beta / L)
        gks.append(np.array([_gk_from_gij(F.gtau_up(l), Lx, Ly) for l in range(L + 1)])[None])
    H = F.Ht + np.diag(U * np.sum((F.nu - 0.5) * (F.nd - 0.5), axis=1))
    w, v = np.linalg.eigh(H)
    eH = lambda a: (v * np.exp(-a * w)) @ v.T
    Z = np.sum(np.exp(-beta * w))
    cs = [F.c_up(i) for i in range(N)]
    taus = np.arange(M + 1) * beta / M
    exact = []
    for tau in taus:
        A, B = eH(beta - tau), eH(tau)
        G = np.array([[np.trace(A @ cs[i] @ B @ cs[j].T) for j in range(N)] for i in range(N)]) / Z
        exact.append(_gk_from_gij(G, Lx, Ly))
    exact = np.array(exact)
    raw = [np.max(np.abs(o.trotter_extrapolate([d], [g], beta, M) - exact)) for d, g in zip(dts, gks)]
    assert raw[0] / raw[2] == pytest.approx((dts[0] / dts[2]) ** 2, rel=0.1)  # dtau^2 error
    got = o.trotter_extrapolate(dts, gks, beta, M)
    nodes = [0, 12, 24, 36, 48]  # tau = 0, 0.5, 1, 1.5, 2 lie on every grid
    assert np.max(np.abs(got[nodes] - exact[nodes])) < raw[2] / 20
    assert np.max(np.abs(got - exact)) < raw[2] / 4


# --------------------------------------------------------------------------
# Matsubara transform and Dyson self-energy (Sec. 3, Eqs. 5-6).
# --------------------------------------------------------------------------
def test_matsubara_transform_exact_for_cubic_data():
    """Samples of a cubic G(tau): the spline is the cubic itself, so the
    transform equals -int_0^beta p(tau) e^{i w tau} dtau, written here by
    integration by parts, [e^{a tau} (p/a - p'/a^2 + p''/a^3 - p'''/a^4)]_0^beta
    with a = i w_n."""
    rng = np.random.default_rng(5)
    beta, M, N, nf = 3.0, 60, 3, 40
    c = rng.standard_normal((4, N))
    tau = np.arange(M + 1) * beta / M
    g = sum(c[p][None, :] * tau[:, None] ** p for p in range(4))
    G, _ = o.matsubara_sigma(g, beta, N, 1, 0.25, nf)
    for n in range(nf):
        a = 1j * (2 * n + 1) * np.pi / beta
        def prim(x):
            p0 = c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3
            p1 = c[1] + 2 * c[2] * x + 3 * c[3] * x ** 2
            p2 = 2 * c[2] + 6 * c[3] * x
            p3 = 6 * c[3]
            return np.exp(a * x) * (p0 / a - p1 / a ** 2 + p2 / a ** 3 - p3 / a ** 4)
        exact = -(prim(beta) - prim(0.0))
        np.testing.assert_allclose(G[n], exact, rtol=1e-12, atol=1e-13 * np.max(np.abs(exact)))


def test_matsubara_sigma_vanishes_at_u0():
    """U = 0: G_k(tau) = e^{-tau eps_k} / (1 + e^{-beta eps_k}) transforms to
    1 / (i w_n - eps_k) and Eq. 6 gives Sigma = 0, up to the spline error:
    |dG(i w)| <= beta max|dS| with |dS| <= (5/384) h^4 max|eps|^4, and
    |dSigma| = |dG| / |G|^2 <= |dG| (w^2 + eps^2) to first order."""
    Lx, Ly, t, beta, M, nf = 4, 4, 0.25, 10.0, 1000, 24
    eps = o.dispersion(Lx, Ly, t)
    tau = np.arange(M + 1) * beta / M
    g = np.exp(-tau[:, None] * eps[None, :]) / (1.0 + np.exp(-beta * eps[None, :]))
    G, sigma = o.matsubara_sigma(g, beta, Lx, Ly, t, nf)
    wn = (2 * np.arange(nf) + 1) * np.pi / beta
    np.testing.assert_allclose(G, 1.0 / (1j * wn[:, None] - eps[None, :]), rtol=0, atol=1e-7)
    dG = beta * 5.0 / 384.0 * (beta / M) ** 4 * np.max(np.abs(eps)) ** 4
    bound = 2.0 * dG * (wn[:, None] ** 2 + eps[None, :] ** 2) + 1e-12
    assert np.all(np.abs(sigma) <= bound)


def test_matsubara_sigma_2x2_hubbard_vs_lehmann():
    """2x2 cluster at U = 2: the exact continuous-time G_k(tau) of the Fock
    space, sampled on a fine grid and transformed, against the Lehmann sum
    G_k(i w) = (1/Z) sum_ab |<b|c_k^dag|a>|^2 (e^{-beta E_a} + e^{-beta E_b})
    / (i w - (E_b - E_a)).  Sigma is then exact up to the spline error, and
    Re Sigma vanishes at k = (pi, 0), where eps_k = 0 (particle-hole)."""
    Lx, Ly, t, U, beta, M, nf = 2, 2, 0.25, 2.0, 2.0, 400, 12
    N = Lx * Ly
    F = fock.FockHubbard(Lx, Ly, t, U, beta, 1)
    H = F.Ht + np.diag(U * np.sum((F.nu - 0.5) * (F.nd - 0.5), axis=1))
    E, V = np.linalg.eigh(H)
    Z = np.sum(np.exp(-beta * E))
    cs = [F.c_up(i) for i in range(N)]
    tau = np.arange(M + 1) * beta / M
    wn = (2 * np.arange(nf) + 1) * np.pi / beta
    g = np.zeros((M + 1, N))
    Gex = np.zeros((nf, N), dtype=np.complex128)
    for ky in range(Ly):
        for kx in range(Lx):
            k = kx + Lx * ky
            phase = [np.exp(-2j * np.pi * (kx * (j % Lx) / Lx + ky * (j // Lx) / Ly)) for j in range(N)]
            ck = sum(phase[j] * cs[j] for j in range(N)) / np.sqrt(N)
            C = V.T @ ck @ V                   # <a| c_k |b>
            A2 = np.abs(C) ** 2
            # our G_k(tau) = (1/Z) sum_ab e^{-(beta - tau) E_a} |<a|c_k|b>|^2 e^{-tau E_b}
            for m, tt in enumerate(tau):
                g[m, k] = np.sum(np.exp(-(beta - tt) * E)[:, None] * A2 * np.exp(-tt * E)[None, :]) / Z
            # Lehmann with c_k^dag: <b|c_k^dag|a> = conj(<a|c_k|b>)
            boltz = np.exp(-beta * E)[:, None] + np.exp(-beta * E)[None, :]
            for n in range(nf):
                Gex[n, k] = np.sum(A2 * boltz / (1j * wn[n] - (E[None, :] - E[:, None]))) / Z
    G, sigma = o.matsubara_sigma(g, beta, Lx, Ly, t, nf)
    np.testing.assert_allclose(G, Gex, rtol=0, atol=1e-9)
    eps = o.dispersion(Lx, Ly, t)
    sig_ex = 1j * wn[:, None] - eps[None, :] - 1.0 / Gex
    np.testing.assert_allclose(sigma, sig_ex, rtol=0, atol=1e-6)
    assert np.max(np.abs(sig_ex)) > 0.05                 # the interaction is visible
    assert np.max(np.abs(sigma[:, 1].real)) < 1e-9       # k = (pi, 0)


# --------------------------------------------------------------------------
# Time-origin averaged G(tau).
# --------------------------------------------------------------------------
def test_gtau_origin_rotation_is_the_shifted_unequal_time_green():
    """For one field at small beta (no stabilisation needed), G(tau) of the
    field rotated by s slices equals the direct product
    B_{l+s} ... B_{s+1} (I + B_s ... B_1 B_L ... B_{s+1})^{-1}, slices mod L,
    i.e. G(tau_s + tau_l, tau_s) of the original field."""
    p = o.Params(2, 2, 0.25, 2.0, 1.0, 0.25, n_s=2)
    rng = np.random.default_rng(9)
    field = rng.choice([-1, 1], size=(p.L, p.N)).astype(np.int8)
    ch = o.Chain(p, field=field)
    s = 1
    rot = o.Chain(p, field=np.roll(field, -s, axis=0))
    got = rot.gtau()
    B = lambda m, sg: ch.B((m - 1) % p.L + 1, sg)
    ref = np.zeros((p.L + 1, p.N))
    for sg in (1, -1):
        A = np.eye(p.N)
        for m in range(s + 1, s + p.L + 1):
            A = B(m, sg) @ A                       # B_{s+L} ... B_{s+1}
        G0 = np.linalg.inv(np.eye(p.N) + A)
        X = G0
        for l in range(p.L + 1):
            if l > 0:
                X = B(s + l, sg) @ X
            ref[l] += 0.5 * o.momentum_diag(X, p.Lx, p.Ly)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    # and the average with one origin is the plain estimator
    np.testing.assert_array_equal(ch.gtau_origins(1), ch.gtau())


def test_gtau_origin_average_is_unbiased_by_enumeration(tiny):
    """Rotating the field is a weight-preserving bijection of the fields, so
    the weighted mean of the origin-averaged estimator over all fields equals
    the exact Fock-space G_k(tau) of the plain estimator."""
    p, fields, w, _, F = tiny
    avg = np.zeros((p.L + 1, p.N))
    for f in range(len(w)):
        avg += w[f] * o.Chain(p, field=fields[f]).gtau_origins(3)
    avg /= w.sum()
    exact = np.zeros((p.L + 1, p.N))
    for l in range(p.L + 1):
        G = F.gtau_up(l)
        exact[l] = o.momentum_diag(G, p.Lx, p.Ly)   # spin down gives the same G_k at U > 0 half filling
    np.testing.assert_allclose(avg, exact, rtol=0, atol=1e-11)


# --------------------------------------------------------------------------
# Correlation length of Sec. 4 (Fig. 5): the exponential fit (reading R18).
# --------------------------------------------------------------------------
def _staggered_exponential(Lx, Ly, xi, amp):
    """C(r) = amp (-1)^(dx+dy) e^{-|r|/xi}, |r| the minimum-image distance,
    written out here from the coordinates (not from the oracle's helpers)."""
    C = np.empty(Lx * Ly)
    for dy in range(Ly):
        for dx in range(Lx):
            rx, ry = min(dx, Lx - dx), min(dy, Ly - dy)
            C[dx + Lx * dy] = amp * (-1) ** (dx + dy) * math.exp(-math.hypot(rx, ry) / xi)
    return C


@pytest.mark.parametrize("Lx,Ly,xi,amp,dmax", [(8, 8, 1.7, 0.3, None), (16, 16, 3.7, 0.05, None),
                                               (8, 6, 2.2, 1.0, 2.5), (16, 4, 0.9, 0.2, 8.0)])
def test_correlation_length_recovers_an_exact_exponential(Lx, Ly, xi, amp, dmax):
    """A staggered exponential returns its own xi (any amplitude, range, and
    rectangular clusters, where mixing dx and dy or dropping the minimum
    image shifts the distances and the fit)."""
    C = _staggered_exponential(Lx, Ly, xi, amp)
    assert o.correlation_length(C, Lx, Ly, dmax) == pytest.approx(xi, rel=1e-12)


def test_correlation_length_skips_non_positive_staggered_values():
    """Points whose staggered value is <= 0 (noise at long distance) carry no
    logarithm and are left out; the rest still give the exact xi."""
    Lx = Ly = 8
    C = _staggered_exponential(Lx, Ly, 2.0, 0.25)
    flip = [3 + Lx * 3, 4 + Lx * 4, 4 + Lx * 1]  # far points turned ferromagnetic
    C[flip] *= -1.0
    C[2 + Lx * 3] = 0.0
    assert o.correlation_length(C, Lx, Ly) == pytest.approx(2.0, rel=1e-12)


def test_correlation_length_degenerate_cases():
    Lx = Ly = 8
    # no decay: a constant staggered pattern has slope 0 -> infinite xi
    C = _staggered_exponential(Lx, Ly, 1e300, 0.1)
    assert o.correlation_length(C, Lx, Ly) == math.inf
    # growing correlations -> infinite xi as well
    assert o.correlation_length(-_staggered_exponential(Lx, Ly, -3.0, -0.1), Lx, Ly) == math.inf
    # a single distance (only the nearest neighbours in range) -> nan
    assert math.isnan(o.correlation_length(_staggered_exponential(Lx, Ly, 2.0, 1.0), Lx, Ly, 1.0))
    # no positive staggered value at all -> nan
    assert math.isnan(o.correlation_length(-_staggered_exponential(Lx, Ly, 2.0, 1.0), Lx, Ly))


def test_correlation_length_is_the_least_squares_line():
    """On noisy data the fit equals the slope of numpy's degree-1 polynomial
    least squares through the same points, selected here independently."""
    Lx, Ly = 12, 10
    rng = np.random.default_rng(5)
    C = _staggered_exponential(Lx, Ly, 2.5, 0.2) * np.exp(0.2 * rng.standard_normal(Lx * Ly))
    dmax = 4.2
    d, y = [], []
    for dy in range(Ly):
        for dx in range(Lx):
            r = math.hypot(min(dx, Lx - dx), min(dy, Ly - dy))
            c = (-1) ** (dx + dy) * C[dx + Lx * dy]
            if 0 < r <= dmax and c > 0:
                d.append(r)
                y.append(math.log(c))
    slope = np.polyfit(d, y, 1)[0]
    assert o.correlation_length(C, Lx, Ly, dmax) == pytest.approx(-1.0 / slope, rel=1e-11)
