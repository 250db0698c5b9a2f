"""Oracle work for the full-size GPU parity tests, run in spawned worker
processes (one chain per process; each takes a minute or two of CPU time).

Test infrastructure: calls only `oracle/`.
"""
from __future__ import annotations

import numpy as np

from oracle import dqmc as o

# The benchmarked workload: 16x16, t = 0.25, U = 2, beta = 20, dtau = 0.125
# (L = 160), n_s = 10, seed 0.
FULL = dict(Lx=16, Ly=16, t=0.25, U=2.0, beta=20.0, dtau=0.125, n_s=10, seed=0)


def full_size_chain(chain):
    """Initial field and G(0), one measured sweep and the G(tau) of the new
    field of one chain of the benchmarked workload."""
    f = FULL
    p = o.Params(f["Lx"], f["Ly"], f["t"], f["U"], f["beta"], f["dtau"], n_s=f["n_s"])
    ch = o.Chain(p, seed=f["seed"], chain=chain)
    field0 = ch.field.copy()
    g0 = ch.green(0, 1)
    out = ch.sweep()
    return {
        "field0": field0, "G0_up": g0,
        "field": ch.field.copy(), "G_up": out["G_up"], "G_dn": out["G_dn"],
        "accepted": int(out["accepted"]),
        "obs": np.sum(out["obs"], axis=0), "n_meas": len(out["obs"]),
        "spin": np.sum(out["spin"], axis=0),
        "gtau": ch.gtau(),
    }
