"""Brute-force sum over every Ising field of a tiny cluster (test pin).

Uses the oracle's B matrices, then sums det M_up det M_dn and configuration
observables over all 2^(N L) fields, so that Eq. (3) and the oracle's
building blocks can be compared with the exact Fock-space trace.
"""
from __future__ import annotations

import numpy as np

from oracle import dqmc as o


def all_fields(N, L):
    n = N * L
    codes = np.arange(1 << n, dtype=np.int64)
    bits = (codes[:, None] >> np.arange(n)[None, :]) & 1
    return (2 * bits - 1).astype(np.int8).reshape(-1, L, N)


def products(E, lam, sigma, fields):
    """A = B_L ... B_1 for every field, shape [F, N, N]."""
    F, L, N = fields.shape
    A = np.broadcast_to(np.eye(N), (F, N, N)).copy()
    for l in range(L):
        B = E[None, :, :] * np.exp(sigma * lam * fields[:, l, :].astype(np.float64))[:, None, :]
        A = B @ A
    return A


def enumerate_sum(p: "o.Params", want_g=False):
    fields = all_fields(p.N, p.L)
    dets = {}
    greens = {}
    for sg in (1, -1):
        A = products(p.E, p.lam, sg, fields)
        M = np.eye(p.N)[None] + A
        dets[sg] = np.linalg.det(M)
        if want_g:
            greens[sg] = np.linalg.inv(M)
    C = o.hs_prefactor(p.U, p.dtau)
    w = dets[1] * dets[-1]
    Z = C ** (p.N * p.L) * np.sum(w)
    return fields, w, Z, greens
