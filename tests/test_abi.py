"""The C-ABI library builds, loads and exports every function include/slab.h declares (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "slab.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(slab_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    from paper_2211_07572_gb300 import _lib
    lib = _lib.load()
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding misses {name}"
    assert set(_lib.SIGNATURES) == set(names)


def test_argument_validation_needs_no_gpu():
    from paper_2211_07572_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    g = _lib.SlabGrid(2, 64)
    co = _lib.SlabCoeffs(_lib.POISSON, None, None, 0.0)
    assert lib.slab_factor(ctypes.byref(g), ctypes.byref(co), 7, None, ctypes.byref(h)) == _lib.SLAB_EINVAL
    assert lib.slab_factor(ctypes.byref(g), ctypes.byref(co), 1, None, ctypes.byref(h)) == _lib.SLAB_EINVAL
    assert lib.slab_factor(ctypes.byref(g), ctypes.byref(co), 64, None, ctypes.byref(h)) == _lib.SLAB_EINVAL
    co2 = _lib.SlabCoeffs(_lib.DIFFUSION, None, None, 0.0)      # diffusion needs kappa
    assert lib.slab_factor(ctypes.byref(g), ctypes.byref(co2), 8, None, ctypes.byref(h)) == _lib.SLAB_EINVAL
    g4 = _lib.SlabGrid(4, 64)
    assert lib.slab_factor(ctypes.byref(g4), ctypes.byref(co), 8, None, ctypes.byref(h)) == _lib.SLAB_EINVAL
    assert lib.slab_solve(None, None, None, 1, None, None) == _lib.SLAB_EINVAL
    assert lib.slab_boundary_lift(None, None, None, None, 1) == _lib.SLAB_EINVAL
    assert lib.slab_strerror(_lib.SLAB_ENOCONV).decode().startswith("iterative refinement")
    o = _lib.SlabOpts()
    lib.slab_default_opts(ctypes.byref(o))
    assert o.factor_prec == _lib.PREC_FP32 and o.rtol == 1e-10 and o.max_refine == 30
    assert o.pivot == 0


def test_convection_argument_validation_needs_no_gpu():
    """The nonsymmetric kind's checks all come before any device call (the pointers below are
    never dereferenced on the host)."""
    from paper_2211_07572_gb300 import _lib
    lib = _lib.load()
    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(256)
    g2, g3 = _lib.SlabGrid(2, 64), _lib.SlabGrid(3, 16)
    args = lambda g, co, b, o=None: (ctypes.byref(g), ctypes.byref(co), b, o, ctypes.byref(h))
    no_beta = _lib.SlabCoeffs(_lib.CONVECTION, dummy, None, 0.0, None)
    no_kappa = _lib.SlabCoeffs(_lib.CONVECTION, None, None, 0.0, dummy)
    full = _lib.SlabCoeffs(_lib.CONVECTION, dummy, None, 0.0, dummy)
    assert lib.slab_factor(*args(g2, no_beta, 8)) == _lib.SLAB_EINVAL
    assert lib.slab_factor(*args(g2, no_kappa, 8)) == _lib.SLAB_EINVAL
    assert lib.slab_factor(*args(g3, full, 4)) == _lib.SLAB_EUNSUPPORTED          # 2-D only
    o = _lib.SlabOpts()
    lib.slab_default_opts(ctypes.byref(o))
    o.stage2 = 2                                                               # odd-even: Cholesky based
    assert lib.slab_factor(*args(g2, full, 8, ctypes.byref(o))) == _lib.SLAB_EUNSUPPORTED
    lib.slab_default_opts(ctypes.byref(o))
    o.pivot = 2
    assert lib.slab_factor(*args(g2, full, 8, ctypes.byref(o))) == _lib.SLAB_EINVAL
    bad_kind = _lib.SlabCoeffs(4, dummy, None, 0.0, dummy)
    assert lib.slab_factor(*args(g2, bad_kind, 8)) == _lib.SLAB_EINVAL
    assert lib.slab_apply_transpose(None, None, None, 1) == _lib.SLAB_EINVAL


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle and never falls back to a CPU solve."""
    pkg = os.path.join(ROOT, "paper_2211_07572_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            txt = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, fn
            assert "numpy.linalg" not in txt and "np.linalg" not in txt, fn
