"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/nmpc.h (no compute calls; runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header=None):
    names = set()
    for h in ([header] if header else sorted(os.listdir(os.path.join(ROOT, "include")))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(nmpc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2004_02484_gb300 import build as b
    return b.build()


def test_library_exports_every_declared_symbol(lib_path):
    declared = _declared()
    assert len(declared) >= 10
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\b(nmpc_[a-z0-9_]+)\b", out))
    assert set(declared) <= exported


def test_binding_covers_the_headers(lib_path):
    from paper_2004_02484_gb300 import nmpc as G
    from paper_2004_02484_gb300 import mlp as GM
    from paper_2004_02484_gb300 import plate as GP
    from paper_2004_02484_gb300 import wave as GW
    assert sorted(G.EXPORTED) == _declared("nmpc.h")
    assert sorted(GM.EXPORTED) == _declared("nmpc_mlp.h")
    assert sorted(GP.EXPORTED) == _declared("nmpc_plate.h")
    assert sorted(GW.EXPORTED) == _declared("nmpc_wave.h")


def test_strerror_and_defaults(lib_path):
    from paper_2004_02484_gb300 import nmpc as G
    o = G.nmpc_default_opts()
    assert o.n_lo == 2 and o.n_u_it == 2 and o.tol == 1e-6 and o.precision == G.NMPC_FP64
    assert G.LIB.nmpc_strerror(G.NMPC_ERR_DIVERGED).decode().startswith("diverged")


def test_setup_rejects_bad_descriptors_before_touching_the_device(lib_path):
    """Descriptor validation happens on the host before any CUDA call."""
    from paper_2004_02484_gb300 import nmpc as G
    from paper_2004_02484_gb300 import workloads as wl
    bad = []
    i = wl.heat1d_single(); i.horizon = 0; bad.append((i, G.NMPC_ERR_BAD_ARG))
    i = wl.heat1d_single(); i.act = [0, 32]; bad.append((i, G.NMPC_ERR_BAD_ARG))
    i = wl.heat1d_single(); i.my = 2; bad.append((i, G.NMPC_ERR_BAD_ARG))
    i = wl.heat1d_single(); i.act = list(range(65)); bad.append((i, G.NMPC_ERR_UNSUPPORTED))
    i = wl.heat1d_single(); i.r = 0.0; bad.append((i, G.NMPC_ERR_BAD_ARG))
    for inst, code in bad:
        descs, keep = G.make_descs([inst])
        h = ctypes.c_void_p()
        rc = G.LIB.nmpc_setup(descs, 1, None, ctypes.byref(h))
        assert rc == code, (rc, code)
    o = G.nmpc_default_opts()
    o.n_lo = 0
    descs, keep = G.make_descs([wl.heat1d_single()])
    h = ctypes.c_void_p()
    assert G.LIB.nmpc_setup(descs, 1, ctypes.byref(o), ctypes.byref(h)) == G.NMPC_ERR_BAD_ARG


def test_path_options_default_to_auto_and_are_validated_on_the_host(lib_path):
    """strips / strip_rows / lines (the last fields of nmpc_opts: a layout
    mismatch between the binding and the header would show here) default to
    0 = automatic, and out-of-range values are rejected before any CUDA call."""
    from paper_2004_02484_gb300 import nmpc as G
    from paper_2004_02484_gb300 import workloads as wl
    o = G.nmpc_default_opts()
    assert (o.strips, o.strip_rows, o.lines) == (0, 0, 0)
    assert (o.strip_cols, o.tail_rows, o.tail_below) == (0, 0, 0)
    for field, value in (("lines", 3), ("lines", -1), ("strips", 3), ("tail_rows", -2),
                         ("tail_rows", 7), ("tail_below", -1), ("strip_cols", 2)):
        o = G.nmpc_default_opts()
        setattr(o, field, value)
        descs, keep = G.make_descs([wl.heat1d_single()])
        h = ctypes.c_void_p()
        assert G.LIB.nmpc_setup(descs, 1, ctypes.byref(o), ctypes.byref(h)) == G.NMPC_ERR_BAD_ARG


def test_plate_setup_rejects_bad_descriptors_before_touching_the_device(lib_path):
    """Pinned-actuator descriptors are validated on the host before any CUDA
    call: repeated or out-of-grid actuators, empty bounds, oversize grids."""
    import numpy as np
    from paper_2004_02484_gb300 import plate as GP
    from paper_2004_02484_gb300 import workloads as wl
    base = wl.plate_instance(m=7, horizon=3, T=15.0, act_idx=(1, 4))
    bad = []
    b1 = wl.plate_instance(m=7, horizon=3, T=15.0, act_idx=(1, 4))
    b1.act = np.array([8, 8, 11, 29], dtype=np.int32)       # repeated actuator
    bad.append((b1, -1))
    b2 = wl.plate_instance(m=7, horizon=3, T=15.0, act_idx=(1, 4))
    b2.act = np.array([8, 11, 29, 49], dtype=np.int32)      # outside the 7x7 grid
    bad.append((b2, -1))
    b3 = wl.plate_instance(m=7, horizon=3, T=15.0, act_idx=(1, 4))
    b3.u_lo, b3.u_hi = 700.0, 300.0                          # empty bounds
    bad.append((b3, -1))
    b4 = wl.plate_instance(m=33, horizon=3, T=15.0, act_idx=(1, 4))  # 1089 points
    bad.append((b4, -6))
    for inst, code in bad:
        descs, keep = GP.make_descs([inst])
        h = ctypes.c_void_p()
        o = GP.default_opts()
        assert GP.LIB.nmpc_plate_setup(descs, 1, ctypes.byref(o), ctypes.byref(h)) == code
    assert base.ns == 45


def test_wave_setup_rejects_bad_descriptors_before_touching_the_device(lib_path):
    """Second-order descriptors are validated on the host before any CUDA
    call: a <= 0, repeated or out-of-grid actuators, r <= 0, oversize grids."""
    import numpy as np
    from paper_2004_02484_gb300 import wave as GW
    from paper_2004_02484_gb300 import workloads as wl
    mk = lambda **kw: wl.wave_instance(dim=1, m=16, horizon=3, **kw)
    bad = []
    b = mk()
    b.a = 0.0
    bad.append((b, -1))
    b = mk()
    b.act = np.array([3, 3], dtype=np.int32)
    bad.append((b, -1))
    b = mk()
    b.act = np.array([3, 16], dtype=np.int32)
    bad.append((b, -1))
    bad.append((mk(r=0.0), -1))
    bad.append((wl.wave_instance(dim=2, m=33, horizon=2), -6))
    for inst, code in bad:
        descs, keep = GW.make_descs([inst])
        h = ctypes.c_void_p()
        o = GW.default_opts()
        assert GW.LIB.nmpc_wave_setup(descs, 1, ctypes.byref(o), ctypes.byref(h)) == code
    o = GW.default_opts(variant=7)
    descs, keep = GW.make_descs([mk()])
    assert GW.LIB.nmpc_wave_setup(descs, 1, ctypes.byref(o), ctypes.byref(ctypes.c_void_p())) == -1
