"""The C ABI library without a GPU: it loads, exports every entry point that
include/s2.h declares, and rejects invalid configurations before touching
the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "s2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(s2_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2304_05494_gb300 import build
    build.build()
    return C.CDLL(build.LIB)


def test_header_declares_the_problem_statement_calls():
    names = header_functions()
    for f in ("s2_create", "s2_set_state", "s2_step", "s2_get_state", "s2_stats", "s2_destroy", "s2_strerror"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for f in header_functions():
        assert hasattr(lib, f), f


def test_strerror_and_invalid_arguments(lib):
    from paper_2304_05494_gb300 import s2
    assert s2.s2_strerror(0) == "ok"
    assert "invalid" in s2.s2_strerror(s2.S2_EINVAL)
    assert s2.s2_strerror(12345) == "unknown error"

    def create(**over):
        g = s2.s2_grid(16, 16, 16, 1.0, 1.0, 1.0)
        gas = s2.s2_gas(1.4, 0.72, 0.5, 100.0, 0.76, 1.0)
        b = s2.s2_bcs(0, 0, 0, 1.0, 0)
        sch = s2.s2_scheme(6, 5, 6, 0.2, 0, 0.8, 0.0, 10)
        for k, v in over.items():
            obj, field = k.split("__")
            setattr({"g": g, "gas": gas, "b": b, "sch": sch}[obj], field, v)
        h = C.c_void_p()
        rc = s2._lib.s2_create(C.byref(g), None, C.byref(gas), C.byref(b), C.byref(sch), None, C.byref(h))
        return rc

    assert create(g__nx=0) == s2.S2_EINVAL
    assert create(g__ly=-1.0) == s2.S2_EINVAL
    assert create(b__x=1) == s2.S2_EINVAL                  # walls only in y
    assert create(b__y=1, g__ny=2) == s2.S2_EINVAL         # walls need ny >= 4
    assert create(sch__weno_order=4) == s2.S2_EINVAL
    assert create(sch__central_order=5) == s2.S2_EINVAL
    assert create(sch__keep=-2) == s2.S2_EINVAL             # KEEP-n: n >= 1, or -1 for exact means
    assert create(sch__visc_order=10) == s2.S2_EINVAL
    assert create(sch__cfl=0.0, sch__dt_fixed=0.0) == s2.S2_EINVAL
    assert create(gas__gamma=1.0) == s2.S2_EINVAL
    # point and interface indices are split in 32-bit arithmetic
    assert create(g__nx=2000, g__ny=1100, g__nz=1000) == s2.S2_EINVAL
    # thermally perfect gas: c_v = c_p - R must be positive (c_p/R = 0.9 at
    # T = 1 is not), coefficients finite
    for bad in ([0.0, 0.0, 0.9, 0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 3.5, float("nan"), 0.0, 0.0, 0.0]):
        a = (C.c_double * 7)(*bad)
        assert create(gas__cp_coeffs=C.cast(a, C.POINTER(C.c_double))) == s2.S2_EINVAL
    # null arguments
    h = C.c_void_p()
    assert s2._lib.s2_create(None, None, None, None, None, None, C.byref(h)) == s2.S2_EINVAL
    assert s2._lib.s2_step(None, 1) == s2.S2_EINVAL
    assert s2._lib.s2_stats(None, None) == s2.S2_EINVAL
    assert s2._lib.s2_stream_states(None, None, 0, None, 0, 1, 1) == s2.S2_EINVAL
    s2._lib.s2_destroy(None)


def test_python_binding_names_match_header():
    from paper_2304_05494_gb300 import s2
    for f in header_functions():
        assert hasattr(s2, f), f


def test_binding_refuses_wrong_state_sizes():
    """The Solver wrapper checks a buffer's shape before the library reads
    or writes 5 nx ny nz doubles through it (no device needed: the check
    runs before any call)."""
    import numpy as np
    import pytest
    from paper_2304_05494_gb300 import s2
    sv = object.__new__(s2.Solver)
    sv.shape, sv.n, sv.h = (5, 4, 3, 2), 24, None
    assert sv._fits(np.zeros((5, 4, 3, 2))) is not None
    assert sv._fits(np.zeros(120)) is not None
    for bad in (np.zeros((5, 4, 3, 3)), np.zeros(119), np.zeros((4, 4, 3, 2))):
        with pytest.raises(ValueError):
            sv._fits(bad)


def test_binding_stream_states_checks_stacks():
    """Solver.stream_states accepts a stack of states or one reused state,
    and refuses other shapes or a stack shorter than count, before any
    library call."""
    import numpy as np
    import pytest
    from paper_2304_05494_gb300 import s2
    sv = object.__new__(s2.Solver)
    sv.shape, sv.n, sv.h = (5, 4, 3, 2), 24, None
    calls = []
    orig = s2.s2_stream_states
    s2.s2_stream_states = lambda h, wi, si, wo, so, count, nsteps: calls.append((si, so, count, nsteps))
    try:
        sv.stream_states(np.zeros((3, 5, 4, 3, 2)), np.zeros((3, 5, 4, 3, 2)), 2)
        sv.stream_states(np.zeros((5, 4, 3, 2)), np.zeros((5, 4, 3, 2)), 1, count=4)
        sv.stream_states(np.zeros((5, 4, 3, 2)), np.zeros((2, 5, 4, 3, 2)), 1, count=2)
        with pytest.raises(ValueError):
            sv.stream_states(np.zeros((5, 4, 3, 2)), np.zeros((5, 4, 3, 2)), 1)  # count needed
        with pytest.raises(ValueError):
            sv.stream_states(np.zeros((2, 5, 4, 3, 2)), np.zeros((2, 5, 4, 3, 2)), 1, count=3)
        with pytest.raises(ValueError):
            sv.stream_states(np.zeros((2, 5, 4, 3, 3)), np.zeros((2, 5, 4, 3, 2)), 1)
    finally:
        s2.s2_stream_states = orig
    assert calls == [(120, 120, 3, 2), (0, 0, 4, 1), (0, 120, 2, 1)]
