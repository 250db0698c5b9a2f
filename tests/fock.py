"""Exact Fock-space reference for tiny Hubbard clusters (test pin, not the oracle).

Builds the second-quantised operators of Eq. (1) in the occupation basis of
all 4^N states, with Jordan-Wigner signs, and evaluates the Trotterised trace
of Eq. (2), Z_dtau = Tr (e^{-dtau H_t} e^{-dtau H_U})^L, without any
Hubbard-Stratonovich field or determinant.  It shares no code with
`oracle/`: the hopping matrix is rebuilt here from the bond list.
"""
from __future__ import annotations

import itertools

import numpy as np


def bonds(Lx, Ly):
    """Directed hops (j <- i) of the periodic Lx x Ly cluster, one per
    direction +-x, +-y (a side of length 2 repeats the same neighbour)."""
    out = []
    for y in range(Ly):
        for x in range(Lx):
            i = x + Lx * y
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                out.append((((x + dx) % Lx) + Lx * ((y + dy) % Ly), i))
    return out


def single_spin_hopping(Lx, Ly, t):
    """h = -t sum_bonds c^dag_j c_i on the 2^N single-spin Fock space."""
    N = Lx * Ly
    dim = 1 << N
    h = np.zeros((dim, dim))
    for j, i in bonds(Lx, Ly):
        for state in range(dim):
            if not (state >> i) & 1:
                continue
            s1 = state & ~(1 << i)
            sign = (-1) ** bin(state & ((1 << i) - 1)).count("1")
            if (s1 >> j) & 1:
                continue
            sign *= (-1) ** bin(s1 & ((1 << j) - 1)).count("1")
            h[s1 | (1 << j), state] += -t * sign
    return h


def _expm_sym(h, a):
    w, v = np.linalg.eigh(h)
    return (v * np.exp(a * w)) @ v.T


def occupations(N):
    dim = 1 << N
    return np.array([[(s >> i) & 1 for i in range(N)] for s in range(dim)], dtype=np.float64)


class FockHubbard:
    """Full 4^N Fock space, index = up_state + 2^N * dn_state (all up modes
    precede all down modes in the Jordan-Wigner order)."""

    def __init__(self, Lx, Ly, t, U, dtau, L):
        self.N = N = Lx * Ly
        self.dim1 = 1 << N
        self.L = L
        h = single_spin_hopping(Lx, Ly, t)
        self.h = h
        eh = _expm_sym(h, -dtau)
        occ = occupations(N)
        nu = np.repeat(occ[None, :, :], self.dim1, axis=0).reshape(-1, N)   # up = fast index
        nd = np.repeat(occ[:, None, :], self.dim1, axis=1).reshape(-1, N)   # dn = slow index
        self.nu, self.nd = nu, nd
        hu = U * np.sum((nu - 0.5) * (nd - 0.5), axis=1)
        self.T = np.kron(eh, eh) * np.exp(-dtau * hu)[None, :]
        self.Ht = np.kron(h, np.eye(self.dim1)) + np.kron(np.eye(self.dim1), h)
        self.TL = np.linalg.matrix_power(self.T, L)
        self.Z = np.trace(self.TL)

    def expect(self, O):
        return np.trace(self.TL @ O) / self.Z

    def docc(self):
        return self.expect(np.diag(np.sum(self.nu * self.nd, axis=1))) / self.N

    def ekin(self):
        return self.expect(self.Ht) / self.N

    def c_up(self, i):
        """Annihilator of an up electron on site i in the full space."""
        dim1 = self.dim1
        c1 = np.zeros((dim1, dim1))
        for s in range(dim1):
            if (s >> i) & 1:
                c1[s & ~(1 << i), s] = (-1) ** bin(s & ((1 << i) - 1)).count("1")
        return np.kron(np.eye(dim1), c1)

    def gtau_up(self, l):
        """G_ij(l,0) = Tr[T^{L-l} c_i T^l c^dag_j] / Z for spin up."""
        N = self.N
        Tl = np.linalg.matrix_power(self.T, l)
        TLl = np.linalg.matrix_power(self.T, self.L - l)
        cs = [self.c_up(i) for i in range(N)]
        G = np.empty((N, N))
        for i in range(N):
            A = TLl @ cs[i] @ Tl
            for j in range(N):
                G[i, j] = np.trace(A @ cs[j].T) / self.Z
        return G


def trotter_trace_sectors(Lx, Ly, t, U, dtau, L):
    """Tr (e^{-dtau H_t} e^{-dtau H_U})^L summed over (N_up, N_dn) sectors, for
    clusters up to N = 6 where the full 4^N matrix would be slow."""
    N = Lx * Ly
    h = single_spin_hopping(Lx, Ly, t)
    occ = occupations(N)
    counts = occ.sum(axis=1).astype(int)
    total = 0.0
    blocks = {}
    for n in range(N + 1):
        idx = np.nonzero(counts == n)[0]
        blocks[n] = (idx, _expm_sym(h[np.ix_(idx, idx)], -dtau))
    for nu, nd in itertools.product(range(N + 1), repeat=2):
        iu, eu = blocks[nu]
        idn, ed = blocks[nd]
        ou = occ[iu]
        od = occ[idn]
        hu = U * np.einsum("ak,bk->ba", ou - 0.5, od - 0.5).reshape(-1)  # dn slow, up fast
        T = np.kron(ed, eu) * np.exp(-dtau * hu)[None, :]
        total += np.trace(np.linalg.matrix_power(T, L))
    return total
