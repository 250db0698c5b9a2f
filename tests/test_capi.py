"""The C-ABI library builds, loads and exports every symbol that
include/dqmc.h declares (CPU-only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dqmc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dqmc_[a-zA-Z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1504_05090_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dqmc_init", "dqmc_sweep", "dqmc_recompute_G", "dqmc_measure_Gtau",
                     "dqmc_grad", "dqmc_destroy", "dqmc_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1504_05090_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_strerror_and_argument_checks_without_gpu(libpath):
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    assert lib.dqmc_strerror(0) == b"ok"
    assert lib.dqmc_strerror(-1) == b"invalid argument"
    h = ctypes.c_void_p()
    # rejected before any CUDA call: no groups / odd side / k out of range
    assert lib.dqmc_init(None, 0, 0, None, ctypes.byref(h)) == -1
    g = _lib.DqmcGroup(5, 4, 0.25, 2.0, 2.0, 0.125, 1, 4, 4, 0)
    assert lib.dqmc_init(ctypes.byref(g), 1, 0, None, ctypes.byref(h)) == -1
    g = _lib.DqmcGroup(4, 4, 0.25, 2.0, 2.0, 0.125, 1, 4, 33, 0)
    assert lib.dqmc_init(ctypes.byref(g), 1, 0, None, ctypes.byref(h)) == -1
    g = _lib.DqmcGroup(4, 4, 0.25, 2.0, 2.0, 0.3, 1, 4, 4, 0)  # beta/dtau not an integer
    assert lib.dqmc_init(ctypes.byref(g), 1, 0, None, ctypes.byref(h)) == -1
    assert lib.dqmc_sweep(None, 1, 0) == -1
    assert lib.dqmc_num_chains(None) == -1
    lib.dqmc_destroy(None)


def test_package_fails_loudly_without_library(tmp_path):
    from paper_1504_05090_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "missing.so"))


def test_trotter_extrapolate_argument_checks_without_gpu(libpath):
    """dqmc_trotter_extrapolate rejects bad runs before any CUDA call."""
    import numpy as np
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    buf = np.zeros(4 * 9 * 2)
    out = np.zeros(5 * 2)
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)

    def call(R, dts, Ls, Cs, N=2, beta=2.0, M=4, null_run=False):
        dt = np.array(dts, dtype=np.float64)
        L = np.array(Ls, dtype=np.int32)
        C = np.array(Cs, dtype=np.int32)
        ptrs = (ctypes.c_void_p * max(R, 1))(*([None if null_run else buf.ctypes.data] * max(R, 1)))
        return lib.dqmc_trotter_extrapolate(R, P(dt), P(L), P(C), ptrs, N, beta, M, P(out), 0)

    assert call(0, [0.25], [8], [1]) == -1                      # no runs
    assert call(17, [0.25] * 17, [8] * 17, [1] * 17) == -1      # more than DQMC_TX_MAX_RUNS
    assert call(1, [1.0], [2], [1]) == -1                       # L < 3
    assert call(1, [0.25], [7], [1]) == -1                      # L dtau != beta
    assert call(2, [0.25, 0.25], [8, 8], [1, 1]) == -1          # all dtau equal
    assert call(1, [0.25], [8], [0]) == -1                      # no chains
    assert call(1, [0.25], [8], [1], null_run=True) == -1       # missing data
    assert call(1, [0.25], [8], [1], N=0) == -1
    assert call(1, [0.25], [8], [1], M=0) == -1
    assert call(1, [0.25], [8], [1], beta=-2.0) == -1


def test_matsubara_sigma_argument_checks_without_gpu(libpath):
    """dqmc_matsubara_sigma rejects bad sizes before any CUDA call."""
    import numpy as np
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    g = np.zeros((9, 4))
    out = np.zeros((3, 4, 2))
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    ok = dict(M=8, Lx=2, Ly=2, t=0.25, beta=2.0, nf=3)

    def call(gk=g, sig=out, **kw):
        a = dict(ok, **kw)
        return lib.dqmc_matsubara_sigma(None if gk is None else P(gk), a["M"], a["Lx"], a["Ly"],
                                        a["t"], a["beta"], a["nf"], None,
                                        None if sig is None else P(sig), 0)

    assert call(gk=None) == -1
    assert call(sig=None) == -1
    assert call(M=2) == -1
    assert call(Lx=0) == -1
    assert call(beta=0.0) == -1
    assert call(nf=0) == -1
    assert call(t=float("nan")) == -1


def test_gtau_origins_argument_checks_without_gpu(libpath):
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    import numpy as np
    buf = np.zeros(4)
    assert lib.dqmc_measure_Gtau_origins(None, 2, buf.ctypes.data_as(ctypes.c_void_p), 0) == -1


def test_init_at_rejects_bad_chain_offsets_without_gpu(libpath):
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    h = ctypes.c_void_p()
    g = _lib.DqmcGroup(4, 4, 0.25, 2.0, 2.0, 0.125, 2, 4, 4, 0)
    assert lib.dqmc_init_at(ctypes.byref(g), 1, 0, -1, None, ctypes.byref(h)) == -1
    assert lib.dqmc_init_at(ctypes.byref(g), 1, 0, 0x7FFFFFFF, None, ctypes.byref(h)) == -1


def test_every_timed_kernel_class_has_a_roofline_formula(libpath):
    """bench.py turns the library's per-class device times into roofline
    fractions; every class that does arithmetic needs a work formula there,
    for every working precision (host logic, no GPU)."""
    import sys
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    sys.path.insert(0, ROOT)
    import bench
    names = []
    for c in range(64):
        name = lib.dqmc_timing_class_name(c)
        if not name:
            break
        names.append(name.decode())
    assert "qr_pivot" in names and "gj_inverse_pair" in names
    bookkeeping = {"gtau_finalize", "grad_terms", "misc"}
    for prec in ("df32", "fp64", "fp32"):
        for name in names:
            bound, work = bench.class_work(name, 0.6, prec)
            if name in bookkeeping:
                assert bound is None
            else:
                assert bound in ("alu", "alu64", "alu32x2", "tensor") and work > 0, (name, prec)


def test_correlation_length_argument_checks_without_gpu(libpath):
    import numpy as np
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    buf = np.zeros(4)
    assert lib.dqmc_correlation_length(None, 4.0, buf.ctypes.data_as(ctypes.c_void_p), 0) == -1


def test_logweight_rejects_parameters_other_than_the_contexts():
    """LogWeight differentiates log W of the context's own B matrices; a t or
    lambda that differs from the context's must raise, not return the
    derivatives of another function (host logic, no GPU)."""
    import math
    import paper_1504_05090_gb300 as pkg

    class FakeSim:
        groups = [pkg.Group(Lx=4, Ly=4, t=0.25, U=2.0, dtau=0.125),
                  pkg.Group(Lx=8, Ly=8, t=0.25, U=2.0, dtau=0.125)]

    lam = math.acosh(math.exp(0.5 * 0.125 * 2.0))
    pkg.LogWeight.check_parameters(FakeSim, 0.25, lam)
    with pytest.raises(ValueError):
        pkg.LogWeight.check_parameters(FakeSim, 0.26, lam)
    with pytest.raises(ValueError):
        pkg.LogWeight.check_parameters(FakeSim, 0.25, lam * (1 + 1e-9))
    FakeSim.groups.append(pkg.Group(Lx=4, Ly=4, t=0.25, U=3.0, dtau=0.125))
    with pytest.raises(ValueError):  # groups with different lambda: no single (t, lambda)
        pkg.LogWeight.check_parameters(FakeSim, 0.25, lam)


def test_set_tiles_argument_checks_without_gpu(libpath):
    from paper_1504_05090_gb300 import _lib
    lib = _lib.load(libpath)
    t = _lib.DqmcTiles(4, 4, 2)
    assert lib.dqmc_set_tiles(None, 0, ctypes.byref(t)) == -1
    out = _lib.DqmcTiles()
    assert lib.dqmc_get_tiles(None, 0, ctypes.byref(out)) == -1
    assert lib.dqmc_autotune_tiles(None, 1, 0, None, ctypes.byref(out)) == -1
