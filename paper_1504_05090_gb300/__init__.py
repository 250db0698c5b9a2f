"""GB300 BSS determinant QMC for the half-filled 2D Hubbard model.

Python binding of libdqmc (include/dqmc.h): argument marshalling around the
CUDA library, plus `LogWeight`, a torch.autograd.Function whose backward is
the library's adjoint of log det(I + B_L ... B_1).  Model and notation follow
Rost & Bluemer, arXiv:1504.05090, Sec. 2, Eqs. (1)-(3).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib

__all__ = ["Group", "DQMC", "LogWeight", "DqmcError", "n_slices", "autotune", "autotune_tiles"]

DqmcError = _lib.DqmcError
_LIB = None


def lib():
    """The loaded libdqmc (raises ImportError if it has not been built)."""
    global _LIB
    if _LIB is None:
        _LIB = _lib.load()
    return _LIB


def n_slices(beta, dtau):
    return int(round(beta / dtau))


@dataclass
class Group:
    """One group of identical chains: cluster Lx x Ly, Eq. (1) parameters t, U,
    inverse temperature beta, Trotter step dtau (Eq. (2)), n_chains chains,
    stabilisation interval n_s, delay depth k and working precision."""
    Lx: int
    Ly: int
    t: float = 0.25
    U: float = 2.0
    beta: float = 2.0
    dtau: float = 0.125
    n_chains: int = 1
    stab_interval: int = 10
    delay_k: int = 16
    precision: str = "fp64"

    @property
    def N(self):
        return self.Lx * self.Ly

    @property
    def L(self):
        return n_slices(self.beta, self.dtau)

    def _c(self):
        prec = {"fp64": _lib.DQMC_FP64, "fp32": _lib.DQMC_FP32, "df32": _lib.DQMC_DF32}[self.precision]
        return _lib.DqmcGroup(self.Lx, self.Ly, self.t, self.U, self.beta, self.dtau,
                              self.n_chains, self.stab_interval, self.delay_k, prec)


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


class DQMC:
    """A context of Markov chains living on the current CUDA device.

    All work is enqueued on the torch stream current at construction."""

    def __init__(self, groups, seed=0, stream=None, chain_offset=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("DQMC needs a CUDA device")
        self.groups = list(groups)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        arr = (_lib.DqmcGroup * len(self.groups))(*[g._c() for g in self.groups])
        h = ctypes.c_void_p()
        _lib.check(lib().dqmc_init_at(arr, len(self.groups), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                      int(chain_offset), ctypes.c_void_p(stream.cuda_stream),
                                      ctypes.byref(h)),
                   "dqmc_init_at", lib())
        self._h = h
        self.n_chains = lib().dqmc_num_chains(h)

    def close(self):
        if getattr(self, "_h", None):
            lib().dqmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- Monte Carlo --------------------------------------------------------
    def sweep(self, n=1, measure=True):
        _lib.check(lib().dqmc_sweep(self._h, int(n), int(bool(measure))), "dqmc_sweep", lib())

    def recompute_G(self):
        out = np.zeros(self.n_chains)
        _lib.check(lib().dqmc_recompute_G(self._h, _ptr(out)), "dqmc_recompute_G", lib())
        return out

    # -- state --------------------------------------------------------------
    def field(self):
        out = np.empty(lib().dqmc_field_size(self._h), dtype=np.int8)
        _lib.check(lib().dqmc_get_field(self._h, _ptr(out)), "dqmc_get_field", lib())
        return self._split(out, lambda g: (g.n_chains, g.L, g.N))

    def set_field(self, fields):
        flat = np.concatenate([np.ascontiguousarray(f, dtype=np.int8).ravel() for f in fields])
        _lib.check(lib().dqmc_set_field(self._h, _ptr(flat)), "dqmc_set_field", lib())

    def G(self, chain, spin=0):
        g = self._group_of(chain)
        out = np.empty((g.N, g.N))
        _lib.check(lib().dqmc_get_G(self._h, int(chain), int(spin), _ptr(out)), "dqmc_get_G", lib())
        return out

    def observables(self):
        out = np.empty((self.n_chains, 4))
        _lib.check(lib().dqmc_get_observables(self._h, _ptr(out)), "dqmc_get_observables", lib())
        return out

    def spin_correlation(self):
        """Accumulated C(r) per group, arrays [chain, N] with r = dx + Lx dy
        (sums over the measurements; reset with reset_observables)."""
        out = np.empty(lib().dqmc_spin_correlation_size(self._h))
        _lib.check(lib().dqmc_get_spin_correlation(self._h, _ptr(out)),
                   "dqmc_get_spin_correlation", lib())
        return self._split(out, lambda g: (g.n_chains, g.N))

    def correlation_length(self, dmax=None, out=None):
        """Spin correlation length of every chain and of each group's chain
        average from the accumulated C(r) (see dqmc_correlation_length):
        (per-chain array [chains], per-group array [groups]).  dmax defaults
        to min(Lx, Ly) / 2 of the first group.  With `out` (a CUDA float64
        tensor of chains + groups elements) the result stays on the device."""
        if dmax is None:
            dmax = 0.5 * min(self.groups[0].Lx, self.groups[0].Ly)
        n = self.n_chains + len(self.groups)
        if out is not None:
            assert out.is_cuda and out.numel() == n
            _lib.check(lib().dqmc_correlation_length(self._h, float(dmax), _ptr(out), 1),
                       "dqmc_correlation_length", lib())
            return out
        host = np.empty(n)
        _lib.check(lib().dqmc_correlation_length(self._h, float(dmax), _ptr(host), 0),
                   "dqmc_correlation_length", lib())
        return host[:self.n_chains], host[self.n_chains:]

    def reset_observables(self):
        _lib.check(lib().dqmc_reset_observables(self._h), "dqmc_reset_observables", lib())

    def stats(self):
        drift = np.empty(self.n_chains)
        acc = np.empty(self.n_chains, dtype=np.uint64)
        _lib.check(lib().dqmc_get_stats(self._h, _ptr(drift), _ptr(acc)), "dqmc_get_stats", lib())
        return drift, acc

    def reset_stats(self):
        _lib.check(lib().dqmc_reset_stats(self._h), "dqmc_reset_stats", lib())

    def launch_count(self):
        return int(lib().dqmc_launch_count(self._h))

    def use_graphs(self, on=True):
        """Replay sweeps as captured CUDA graphs (default) or launch one by one."""
        _lib.check(lib().dqmc_use_graphs(self._h, int(bool(on))), "dqmc_use_graphs", lib())

    def set_gemm_mode(self, mode):
        """'tensor' (default, tcgen05 digit-sliced FP64 products) or 'fp64'."""
        code = {"tensor": _lib.DQMC_GEMM_TENSOR, "fp64": _lib.DQMC_GEMM_FP64}[mode]
        _lib.check(lib().dqmc_set_gemm_mode(self._h, code), "dqmc_set_gemm_mode", lib())

    def set_qr_mode(self, mode):
        """'blocked' (default: pre-pivoted blocked Householder QR on the tensor
        cores) or 'pivoted' (column-pivoted QR on the FP64 pipe)."""
        code = {"blocked": _lib.DQMC_QR_BLOCKED, "pivoted": _lib.DQMC_QR_PIVOTED}[mode]
        _lib.check(lib().dqmc_set_qr_mode(self._h, code), "dqmc_set_qr_mode", lib())

    def set_metropolis_split(self, ctas_per_chain=0):
        """CTAs per chain in the Metropolis pass: 1, 2, 4, or 0 for automatic."""
        _lib.check(lib().dqmc_set_metropolis_split(self._h, int(ctas_per_chain)),
                   "dqmc_set_metropolis_split", lib())

    def set_tiles(self, group, kron_nv=0, wrap_nv=0, metro_ctas=0):
        """Tile shapes of one group's kernels (see dqmc_set_tiles); 0 = built-in."""
        t = _lib.DqmcTiles(int(kron_nv), int(wrap_nv), int(metro_ctas))
        _lib.check(lib().dqmc_set_tiles(self._h, int(group), ctypes.byref(t)), "dqmc_set_tiles",
                   lib())

    def tiles(self, group):
        """Tile shapes in effect for one group: dict(kron_nv, wrap_nv, metro_ctas)."""
        t = _lib.DqmcTiles()
        _lib.check(lib().dqmc_get_tiles(self._h, int(group), ctypes.byref(t)), "dqmc_get_tiles",
                   lib())
        return dict(kron_nv=t.kron_nv, wrap_nv=t.wrap_nv, metro_ctas=t.metro_ctas)

    def timing(self, on=True):
        """Enable/disable per-launch CUDA-event timing by kernel class."""
        _lib.check(lib().dqmc_timing_enable(self._h, int(bool(on))), "dqmc_timing_enable", lib())

    def timing_reset(self):
        _lib.check(lib().dqmc_timing_reset(self._h), "dqmc_timing_reset", lib())

    def timing_read(self):
        """{class name: (total ms, launches)} since the last reset."""
        ms = np.zeros(16)
        n = np.zeros(16, dtype=np.int64)
        k = _lib.check(lib().dqmc_timing_read(self._h, _ptr(ms), _ptr(n), 16), "dqmc_timing_read", lib())
        return {lib().dqmc_timing_class_name(c).decode(): (float(ms[c]), int(n[c]))
                for c in range(k)}

    # -- measurements -------------------------------------------------------
    def gtau(self, out=None):
        """Spin-averaged Re G_k(tau_l) per chain: a list (per group) of arrays
        [chains, L+1, N]; with `out` (a CUDA float64 tensor of
        dqmc_gtau_size elements) the result stays on the device."""
        n = int(lib().dqmc_gtau_size(self._h))
        if out is not None:
            assert out.is_cuda and out.numel() == n
            _lib.check(lib().dqmc_measure_Gtau(self._h, _ptr(out), 1), "dqmc_measure_Gtau", lib())
            return out
        host = np.empty(n)
        _lib.check(lib().dqmc_measure_Gtau(self._h, _ptr(host), 0), "dqmc_measure_Gtau", lib())
        return self._split(host, lambda g: (g.n_chains, g.L + 1, g.N))

    def gtau_origins(self, n_origins, out=None):
        """Time-origin averaged G_k(tau) (see dqmc_measure_Gtau_origins), in
        the layout of gtau(); with `out` (a CUDA float64 tensor of
        dqmc_gtau_size elements) the result stays on the device."""
        n = int(lib().dqmc_gtau_size(self._h))
        if out is not None:
            assert out.is_cuda and out.numel() == n
            _lib.check(lib().dqmc_measure_Gtau_origins(self._h, int(n_origins), _ptr(out), 1),
                       "dqmc_measure_Gtau_origins", lib())
            return out
        host = np.empty(n)
        _lib.check(lib().dqmc_measure_Gtau_origins(self._h, int(n_origins), _ptr(host), 0),
                   "dqmc_measure_Gtau_origins", lib())
        return self._split(host, lambda g: (g.n_chains, g.L + 1, g.N))

    def grad(self):
        """(dlogW/dt, dlogW/dlambda, logW) per chain, host arrays."""
        dt = np.empty(self.n_chains)
        dl = np.empty(self.n_chains)
        lw = np.empty(self.n_chains)
        _lib.check(lib().dqmc_grad(self._h, _ptr(dt), _ptr(dl), _ptr(lw), 0), "dqmc_grad", lib())
        return dt, dl, lw

    def grad_device(self, dt, dl, lw):
        _lib.check(lib().dqmc_grad(self._h, _ptr(dt), _ptr(dl), _ptr(lw), 1), "dqmc_grad", lib())

    # -- helpers ------------------------------------------------------------
    def _group_of(self, chain):
        c = 0
        for g in self.groups:
            if chain < c + g.n_chains:
                return g
            c += g.n_chains
        raise IndexError(chain)

    def _split(self, flat, shape_of):
        out, off = [], 0
        for g in self.groups:
            shp = shape_of(g)
            n = int(np.prod(shp))
            out.append(flat[off:off + n].reshape(shp))
            off += n
        return out


def autotune(groups, drift_target=1e-6, seed=0):
    """Groups with stab_interval and delay_k chosen by the library's autotuner
    for this GPU (see dqmc_autotune)."""
    import torch
    groups = list(groups)
    arr = (_lib.DqmcGroup * len(groups))(*[g._c() for g in groups])
    out = (_lib.DqmcGroup * len(groups))()
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(lib().dqmc_autotune(arr, len(groups), float(drift_target), int(seed),
                                   ctypes.c_void_p(st), out), "dqmc_autotune", lib())
    res = []
    for g, o in zip(groups, out):
        res.append(Group(Lx=g.Lx, Ly=g.Ly, t=g.t, U=g.U, beta=g.beta, dtau=g.dtau,
                         n_chains=g.n_chains, stab_interval=int(o.stab_interval),
                         delay_k=int(o.delay_k), precision=g.precision))
    return res


def autotune_tiles(groups, seed=0):
    """Tile shapes chosen by the library's tile autotuner for each group
    (see dqmc_autotune_tiles): a list of dict(kron_nv, wrap_nv, metro_ctas)."""
    import torch
    groups = list(groups)
    arr = (_lib.DqmcGroup * len(groups))(*[g._c() for g in groups])
    out = (_lib.DqmcTiles * len(groups))()
    st = torch.cuda.current_stream().cuda_stream
    _lib.check(lib().dqmc_autotune_tiles(arr, len(groups), int(seed), ctypes.c_void_p(st), out),
               "dqmc_autotune_tiles", lib())
    return [dict(kron_nv=o.kron_nv, wrap_nv=o.wrap_nv, metro_ctas=o.metro_ctas) for o in out]


def trotter_extrapolate(dtaus, gks, beta, M):
    """dtau -> 0 extrapolation of G_k(tau) (see dqmc_trotter_extrapolate).
    gks[r]: run r's G_k(tau_l) per chain, shape [C, L + 1, N], as returned by
    DQMC.gtau() for one group: all numpy arrays (host) or all CUDA tensors
    (device).  Returns [M + 1, N] on the same side as the inputs."""
    R = len(gks)
    if R != len(dtaus) or R < 1:
        raise ValueError("one dtau per run")
    on_dev = all(hasattr(g, "is_cuda") and g.is_cuda for g in gks)
    if on_dev:
        import torch
        gks = [g.contiguous().to(torch.float64) for g in gks]
    else:
        gks = [np.ascontiguousarray(g, dtype=np.float64) for g in gks]
    shapes = [tuple(g.shape) for g in gks]
    N = shapes[0][2]
    if any(len(s) != 3 or s[2] != N for s in shapes):
        raise ValueError("each run must be [chains, L + 1, N] with the same N")
    dt = np.ascontiguousarray(dtaus, dtype=np.float64)
    L = np.array([s[1] - 1 for s in shapes], dtype=np.int32)
    C = np.array([s[0] for s in shapes], dtype=np.int32)
    ptrs = (ctypes.c_void_p * R)(*[_ptr(g).value for g in gks])
    if on_dev:
        torch.cuda.current_stream().synchronize()
        out = torch.empty((M + 1, N), dtype=torch.float64, device=gks[0].device)
    else:
        out = np.empty((M + 1, N))
    _lib.check(lib().dqmc_trotter_extrapolate(R, _ptr(dt), _ptr(L), _ptr(C), ptrs, int(N),
                                              float(beta), int(M), _ptr(out), int(on_dev)),
               "dqmc_trotter_extrapolate", lib())
    return out


def trotter_timing():
    """Device ms of the three kernels of the last trotter_extrapolate call on
    the current device: (chain average, spline, interpolation and fit)."""
    out = np.zeros(3, dtype=np.float32)
    _lib.check(lib().dqmc_trotter_timing(_ptr(out)), "dqmc_trotter_timing", lib())
    return tuple(float(v) for v in out)


def matsubara_sigma(gk, beta, Lx, Ly, t, n_freq):
    """(G_k(i w_n), Sigma_k(i w_n)) for n < n_freq from G_k(tau_m) on
    tau_m = m beta / M (see dqmc_matsubara_sigma).  gk: [M + 1, Lx*Ly], a numpy
    array (host; complex numpy results) or a CUDA tensor (complex CUDA
    tensors)."""
    on_dev = hasattr(gk, "is_cuda") and gk.is_cuda
    if on_dev:
        import torch
        gk = gk.contiguous().to(torch.float64)
    else:
        gk = np.ascontiguousarray(gk, dtype=np.float64)
    M, N = gk.shape[0] - 1, gk.shape[1]
    if N != Lx * Ly:
        raise ValueError("gk must have Lx * Ly columns")
    if on_dev:
        g = torch.empty((n_freq, N, 2), dtype=torch.float64, device=gk.device)
        s = torch.empty_like(g)
        torch.cuda.current_stream().synchronize()
    else:
        g = np.empty((n_freq, N, 2))
        s = np.empty((n_freq, N, 2))
    _lib.check(lib().dqmc_matsubara_sigma(_ptr(gk), int(M), int(Lx), int(Ly), float(t),
                                          float(beta), int(n_freq), _ptr(g), _ptr(s), int(on_dev)),
               "dqmc_matsubara_sigma", lib())
    if on_dev:
        return torch.view_as_complex(g), torch.view_as_complex(s)
    return g[..., 0] + 1j * g[..., 1], s[..., 0] + 1j * s[..., 1]


def matsubara_timing():
    """Device ms of the last matsubara_sigma call: (spline, transform)."""
    out = np.zeros(2, dtype=np.float32)
    _lib.check(lib().dqmc_matsubara_timing(_ptr(out)), "dqmc_matsubara_timing", lib())
    return tuple(float(v) for v in out)


class LogWeight:
    """torch.autograd.Function: log W = log|det M_up| + log|det M_dn| of the
    current field of every chain as a function of (t, lambda).  The forward
    value and both derivatives come from one dqmc_grad call; backward returns
    sum_c grad_out[c] * dlogW_c/dt and the same for lambda.  The inputs must
    equal the parameters the context was built with, t of every group and
    lambda = arccosh(exp(dtau U / 2)) of every group (the field and the
    B matrices are not re-derived from them); anything else raises
    ValueError instead of returning the derivatives of another function."""

    @staticmethod
    def check_parameters(sim: DQMC, t, lam):
        import math
        for g in sim.groups:
            lam_g = math.acosh(math.exp(0.5 * g.dtau * g.U))
            if not math.isclose(float(t), g.t, rel_tol=1e-12, abs_tol=1e-300):
                raise ValueError("LogWeight: t = %r differs from the context's t = %r" % (float(t), g.t))
            if not math.isclose(float(lam), lam_g, rel_tol=1e-12, abs_tol=1e-300):
                raise ValueError("LogWeight: lambda = %r differs from the context's "
                                 "lambda = %r" % (float(lam), lam_g))

    @staticmethod
    def apply(sim: DQMC, t, lam):
        import torch

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, t_, lam_):
                LogWeight.check_parameters(sim, t_.item(), lam_.item())
                dev = torch.device("cuda")
                dt = torch.empty(sim.n_chains, dtype=torch.float64, device=dev)
                dl = torch.empty_like(dt)
                lw = torch.empty_like(dt)
                sim.grad_device(dt, dl, lw)
                ctx.save_for_backward(dt, dl)
                return lw

            @staticmethod
            def backward(ctx, gout):
                dt, dl = ctx.saved_tensors
                return (gout * dt).sum().to(t.dtype), (gout * dl).sum().to(lam.dtype)

        return _Fn.apply(t, lam)
