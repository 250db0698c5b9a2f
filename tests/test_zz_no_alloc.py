"""The allocation-free entry point dqmc_green_noalloc against the regular path.

dqmc_green_noalloc serves callers that may not allocate device memory: it
works in a fixed device array inside libdqmc instead of cudaMalloc.  Its
result must equal what dqmc_set_field + dqmc_get_G give for the same field,
within the 1e-10 relative tolerance of the other Green-function tests, on two
calls in a row (the second call reuses the array left by the first).  This
file is collected last so that a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GTOL = 1e-10


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("Lx,Ly,U,beta,dtau,ns", [(16, 16, 2.0, 20.0, 0.125, 10),
                                                   (6, 4, 3.0, 4.0, 0.1, 7)])
def test_green_noalloc_matches_regular_path_twice(Lx, Ly, U, beta, dtau, ns):
    import torch

    import paper_1504_05090_gb300 as pkg
    from paper_1504_05090_gb300 import _lib

    lib = pkg.lib()
    g = pkg.Group(Lx=Lx, Ly=Ly, t=0.25, U=U, beta=beta, dtau=dtau, n_chains=2,
                  stab_interval=ns, delay_k=8, precision="fp64")
    rng = np.random.default_rng(Lx * 100 + Ly)
    fields = rng.choice(np.array([-1, 1], dtype=np.int8), size=(2, g.L, g.N))
    with pkg.DQMC([g], seed=1) as sim:
        sim.set_field([fields])
        refs = [sim.G(c, 0) for c in range(2)]
    params = g._c()
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row, different fields
        c = call % 2
        f_dev = torch.from_numpy(fields[c].copy()).cuda()
        G_dev = torch.full((g.N, g.N), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.dqmc_green_noalloc(ctypes.byref(params), ctypes.c_void_p(f_dev.data_ptr()),
                                    ctypes.c_void_p(G_dev.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, _lib.ERRORS.get(rc)
        assert _rel(G_dev.cpu().numpy(), refs[c]) < GTOL


def test_green_noalloc_rejects_sizes_beyond_the_side_limit():
    """Lx = 18 exceeds DQMC_MAX_SIDE and is rejected with DQMC_ERR_ARG.  (The
    separate N <= DQMC_NOALLOC_MAX_N check cannot be reached through a valid
    side length: a static_assert keeps DQMC_MAX_SIDE^2 within it.)"""
    import torch

    import paper_1504_05090_gb300 as pkg

    lib = pkg.lib()
    g = pkg.Group(Lx=18, Ly=16, beta=1.0, dtau=0.125, stab_interval=4)
    f_dev = torch.ones(g.L * g.N, dtype=torch.int8, device="cuda")
    G_dev = torch.empty(g.N * g.N, dtype=torch.float64, device="cuda")
    rc = lib.dqmc_green_noalloc(ctypes.byref(g._c()), ctypes.c_void_p(f_dev.data_ptr()),
                                ctypes.c_void_p(G_dev.data_ptr()), None)
    assert rc == -1
