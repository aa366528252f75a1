"""The C-ABI library loads and exports every entry point that include/topo.h declares; pure-host
entry points (element stiffness, descriptor validation) behave as documented.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in os.listdir(os.path.join(ROOT, "include"))
           if h.endswith(".h")]


def _lib():
    from paper_1606_06201_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(topo_[A-Za-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = _lib()
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    _lib()
    from paper_1606_06201_gb300 import topo
    assert set(topo.exported_symbols()) == set(_declared())


def test_element_stiffness_entry_point_matches_oracle():
    from oracle import fe
    from paper_1606_06201_gb300 import topo
    for dim in (2, 3):
        np.testing.assert_allclose(topo.element_stiffness(dim, 1.0, 0.3), fe.element_stiffness(dim),
                                   rtol=0, atol=1e-15)
    with pytest.raises(topo.TopoError):
        topo.element_stiffness(4)
    with pytest.raises(topo.TopoError):
        topo.element_stiffness(2, 1.0, 0.5)


def test_descriptor_validation_needs_no_device():
    from paper_1606_06201_gb300 import topo
    fixed = np.zeros(2 * 9 * 5, dtype=np.uint8)
    bad = [dict(levels=5), dict(levels=0), dict(nu1=-1), dict(omega=1.5), dict(nrhs=0),
           dict(precision=7), dict(smoother=2),
           # 2^31 or more DOFs (rejected before the mask is read)
           dict(dim=3, nx=1024, ny=1024, nz=1024, levels=9)]
    for kw in bad:
        args = dict(dim=2, nx=8, ny=4, nz=0, E=1.0, nu=0.3, levels=2, precision=0, nu1=2, nu2=2,
                    omega=0.6, max_iter=10, nrhs=1, flexible=0, generic_kernels=0, smoother=0, omega_auto=0)
        args.update(kw)
        d = topo.SolverDesc(args["dim"], args["nx"], args["ny"], args["nz"], args["E"], args["nu"],
                            fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), args["levels"],
                            args["precision"], args["nu1"], args["nu2"], args["omega"],
                            args["max_iter"], args["nrhs"], args["flexible"],
                            args["generic_kernels"], args["smoother"], args["omega_auto"])
        h = ctypes.c_void_p()
        st = topo._lib.topo_solver_create(ctypes.byref(d), ctypes.byref(h))
        assert st == topo.E_INVALID_ARG, kw
        assert not h.value


def test_null_handles_are_rejected_without_a_device():
    """Entry points given a null handle return TOPO_E_INVALID_ARG before any CUDA call."""
    from paper_1606_06201_gb300 import topo
    L = topo._lib
    buf = (ctypes.c_double * 4)()
    assert L.topo_ip_set_simp(None, ctypes.c_double(3.0), ctypes.c_double(2.0)) == topo.E_INVALID_ARG
    assert L.topo_ip_filtered_density(None, buf) == topo.E_INVALID_ARG
    assert L.topo_ip_set_vcycle_fusion(None, 1) == topo.E_INVALID_ARG
    assert L.topo_set_outer_precision(None, 1) == topo.E_INVALID_ARG
    assert L.topo_oc_get_state(None, buf, buf, buf) == topo.E_INVALID_ARG
    assert L.topo_oc_set_state(None, buf, buf, buf) == topo.E_INVALID_ARG


def test_workspace_query_needs_no_device():
    """topo_solver_workspace_bytes is pure host arithmetic: it answers here, grows with the
    number of right-hand sides and with mixed precision's FP32 copies dropped for FP64 vectors as
    expected, and rejects what topo_solver_create rejects (including an asymmetric K0)."""
    from oracle import fe
    from paper_1606_06201_gb300 import topo
    from paper_1606_06201_gb300 import workloads as W
    f = W.clamp_xmin(64, 32)
    b1 = topo.workspace_bytes(64, 32, fixed=f, levels=3)
    b2 = topo.workspace_bytes(64, 32, fixed=f, levels=3, nrhs=2)
    assert 0 < b1 < b2
    # the FP64 solver's five CG vectors alone
    assert b1 >= 5 * 8 * f.size
    # the caller's analytic K0 costs the same
    assert topo.workspace_bytes(64, 32, fixed=f, levels=3, K0=fe.element_stiffness(2)) == b1
    with pytest.raises(topo.TopoError):
        topo.workspace_bytes(64, 32, fixed=f, levels=7)       # not divisible by 2^(levels-1)
    K0 = fe.element_stiffness(2)
    K0[0, 1] += 1e-3
    with pytest.raises(topo.TopoError):
        topo.workspace_bytes(64, 32, fixed=f, levels=3, K0=K0)
    K0 = fe.element_stiffness(2)
    K0[3, 3] = np.nan
    with pytest.raises(topo.TopoError):
        topo.workspace_bytes(64, 32, fixed=f, levels=3, K0=K0)
    # a mask that coarsening cannot keep (a fixed fine DOF between free coarse ones)
    bad = np.zeros_like(f)
    bad[2 * 1] = 1
    with pytest.raises(topo.TopoError):
        topo.workspace_bytes(64, 32, fixed=bad, levels=3)
