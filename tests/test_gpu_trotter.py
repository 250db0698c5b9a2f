"""dtau -> 0 extrapolation of G_k(tau) (Sec. 3, Fig. 2) and the Matsubara
transform with the Dyson self-energy (Eqs. 5-6) through the C-ABI.

The kernels and the oracle run the same FP64 steps (chain average, not-a-knot
spline, least-squares line in dtau^2) in different orders: the spline solve
and the fit are well conditioned (diagonally dominant tridiagonal system;
the fit weights have absolute sum below 2 for the time steps used here), so
the results agree to 1e-12 of the largest value.  The Matsubara kernel
integrates every spline interval exactly through the moments
int_0^h t^m e^{i w t} dt, the oracle by Gauss-Legendre quadrature: both sum
M well-scaled terms, so G(i w_n) agrees to 1e-11 of its largest value, and
Sigma = i w - eps - 1/G, whose error is |dG| / |G|^2 <= |dG| (w^2 + 4), to
1e-11 (1 + w^2).
"""
import numpy as np
import pytest

from oracle import dqmc as o

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _runs(seed, beta, Ls, C, N):
    """Seeded G_k(tau)-like runs: a smooth decay per k, a dtau^2 shift and
    chain noise, shape [C, L + 1, N] per run."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(-1.0, 1.0, N)
    out = []
    for L in Ls:
        dt = beta / L
        tau = np.arange(L + 1) * dt
        g = np.exp(-tau[:, None] * eps[None, :]) / (1.0 + np.exp(-beta * eps[None, :]))
        g = g * (1.0 + 0.3 * dt * dt)
        out.append(g[None] + 0.05 * rng.standard_normal((C, L + 1, N)))
    return out


@pytest.mark.parametrize("beta,Ls,C,N,M", [
    (20.0, (50, 100, 200), 256, 64, 400),   # 8x8, dtau 0.4 / 0.2 / 0.1, 256 chains per run
    (1.2, (3, 4, 5), 3, 36, 7),             # the smallest grids (L = 3 and 4 take the short paths)
    (0.7, (7,), 1, 5, 13),                  # one run: interpolation only
    (3.6, (4, 9), 2, 100, 1),               # two runs, ragged N, coarse output grid
    (1.0, (4, 5), 3, 5, 9),                 # odd row length (L + 1) N = 25: element-wise loads
])
def test_extrapolation_matches_oracle_host_and_device(beta, Ls, C, N, M):
    import torch
    import paper_1504_05090_gb300 as pkg
    gks = _runs(7, beta, Ls, C, N)
    dts = [beta / L for L in Ls]
    ref = o.trotter_extrapolate(dts, gks, beta, M)
    host = pkg.trotter_extrapolate(dts, gks, beta, M)
    assert host.shape == (M + 1, N)
    np.testing.assert_allclose(host, ref, rtol=0, atol=TOL * np.max(np.abs(ref)))
    assert all(ms > 0.0 for ms in pkg.trotter_timing())
    dev = pkg.trotter_extrapolate(dts, [torch.from_numpy(g).cuda() for g in gks], beta, M)
    assert dev.is_cuda
    np.testing.assert_array_equal(dev.cpu().numpy(), host)  # same kernels on the same data


def test_simulated_u0_runs_extrapolate_to_the_closed_form():
    """U = 0 has no Trotter error: G_k(tau) measured by dqmc_measure_Gtau at
    three time steps equals e^{-tau eps_k} / (1 + e^{-beta eps_k}) on every
    grid, and the extrapolation from the device buffers equals the closed
    form on the fine grid up to the cubic-spline error bound."""
    import torch
    import paper_1504_05090_gb300 as pkg
    Lx = Ly = 4
    beta, M = 2.0, 40
    eps = o.dispersion(Lx, Ly, 0.25)
    closed = lambda tau: np.exp(-tau[:, None] * eps[None, :]) / (1.0 + np.exp(-beta * eps[None, :]))
    dts, bufs = [0.25, 0.125, 0.1], []
    for dt in dts:
        g = pkg.Group(Lx=Lx, Ly=Ly, t=0.25, U=0.0, beta=beta, dtau=dt, n_chains=2,
                      stab_interval=4, delay_k=4, precision="fp64")
        with pkg.DQMC([g], seed=3) as sim:
            sim.sweep(1)
            L = g.L
            buf = torch.empty(2 * (L + 1) * g.N, dtype=torch.float64, device="cuda")
            sim.gtau(out=buf)
            torch.cuda.synchronize()
            runs = buf.view(2, L + 1, g.N)
            np.testing.assert_allclose(runs.cpu().numpy(), np.broadcast_to(
                closed(np.arange(L + 1) * dt), (2, L + 1, g.N)), rtol=0, atol=1e-10)
            bufs.append(runs)
    got = pkg.trotter_extrapolate(dts, bufs, beta, M).cpu().numpy()
    A = np.stack([np.ones(3), np.array(dts) ** 2], axis=1)
    wsum = np.sum(np.abs(np.linalg.pinv(A)[0]))
    # uniform-grid cubic spline error (5/384) h^4 max|d^4 G/d tau^4| <= (5/384) h^4 max|eps|^4
    bound = wsum * 5.0 / 384.0 * max(dts) ** 4 * np.max(np.abs(eps)) ** 4 + 1e-10
    np.testing.assert_allclose(got, closed(np.arange(M + 1) * beta / M), rtol=0, atol=bound)


@pytest.mark.parametrize("Lx,Ly,beta,M,nf", [
    (8, 8, 20.0, 400, 200),   # the extrapolated 8x8 grid, 200 frequencies (w_n h up to 3.1)
    (6, 4, 5.0, 50, 30),      # ragged N
    (2, 2, 2.0, 3, 5),        # the smallest grid
])
def test_matsubara_matches_oracle_host_and_device(Lx, Ly, beta, M, nf):
    import torch
    import paper_1504_05090_gb300 as pkg
    rng = np.random.default_rng(11)
    eps = o.dispersion(Lx, Ly, 0.25)
    tau = np.arange(M + 1) * beta / M
    g = np.exp(-tau[:, None] * eps[None, :]) / (1.0 + np.exp(-beta * eps[None, :]))
    g = g + 1e-3 * rng.standard_normal(g.shape)
    Gref, Sref = o.matsubara_sigma(g, beta, Lx, Ly, 0.25, nf)
    G, S = pkg.matsubara_sigma(g, beta, Lx, Ly, 0.25, nf)
    wn = (2 * np.arange(nf) + 1) * np.pi / beta
    np.testing.assert_allclose(G, Gref, rtol=0, atol=1e-11 * np.max(np.abs(Gref)))
    assert np.all(np.abs(S - Sref) <= 1e-11 * (1.0 + wn[:, None] ** 2))
    assert all(ms > 0.0 for ms in pkg.matsubara_timing())
    Gd, Sd = pkg.matsubara_sigma(torch.from_numpy(g).cuda(), beta, Lx, Ly, 0.25, nf)
    np.testing.assert_array_equal(Gd.cpu().numpy(), G)
    np.testing.assert_array_equal(Sd.cpu().numpy(), S)


def test_u0_sweeps_to_self_energy_on_the_device():
    """The whole chain on device buffers: U = 0 sweeps at three dtau, their
    G(tau) extrapolated, transformed and put through Eq. 6.  There is no
    interaction, so Sigma = 0 up to the two cubic-spline errors: |dS| <=
    wsum (5/384) h_run^4 + (5/384) h_fine^4 (max|eps| = 1), |dG| <= beta |dS|
    and |dSigma| <= |dG| (w^2 + eps^2) to first order (doubled for margin)."""
    import torch
    import paper_1504_05090_gb300 as pkg
    Lx = Ly = 4
    beta, M, nf = 2.0, 40, 8
    dts, bufs = [0.25, 0.125, 0.1], []
    for dt in dts:
        g = pkg.Group(Lx=Lx, Ly=Ly, t=0.25, U=0.0, beta=beta, dtau=dt, n_chains=2,
                      stab_interval=4, delay_k=4, precision="fp64")
        with pkg.DQMC([g], seed=4) as sim:
            sim.sweep(1)
            buf = torch.empty(2 * (g.L + 1) * g.N, dtype=torch.float64, device="cuda")
            sim.gtau(out=buf)
            torch.cuda.synchronize()
            bufs.append(buf.view(2, g.L + 1, g.N))
    fine = pkg.trotter_extrapolate(dts, bufs, beta, M)
    G, S = pkg.matsubara_sigma(fine, beta, Lx, Ly, 0.25, nf)
    assert G.is_cuda and S.is_cuda
    A = np.stack([np.ones(3), np.array(dts) ** 2], axis=1)
    wsum = np.sum(np.abs(np.linalg.pinv(A)[0]))
    dS = 5.0 / 384.0 * (wsum * max(dts) ** 4 + (beta / M) ** 4)
    eps = o.dispersion(Lx, Ly, 0.25)
    wn = (2 * np.arange(nf) + 1) * np.pi / beta
    bound = 2.0 * beta * dS * (wn[:, None] ** 2 + eps[None, :] ** 2) + 1e-10
    assert np.all(np.abs(S.cpu().numpy()) <= bound)
    np.testing.assert_allclose(G.cpu().numpy(), 1.0 / (1j * wn[:, None] - eps[None, :]),
                               rtol=0, atol=2.0 * beta * dS)
