"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
symbol include/*.h declares (no compute calls here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(inc, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(lbm\w*_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2205_00686_gb300 import _build
    return _build.build()


def test_header_declares_the_abi():
    names = declared_functions()
    import paper_2205_00686_gb300 as lbm
    assert set(names) == set(lbm.ABI_FUNCTIONS)
    for core in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_get_rho_u_T",
                 "lbm_diagnostics", "lbm3d_create", "lbm3d_step"):
        assert core in names


def test_library_exports_every_declared_symbol(built_lib):
    L = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_binding_loads_and_reports_sizes(built_lib):
    import paper_2205_00686_gb300 as lbm
    # pure host arithmetic: state bytes of a 4096^2 FP32 domain
    b = lbm.lbm_state_bytes(4096, 4096, "fp32")
    assert b == 2 * 15 * 4096 * 4096 * 4
    assert lbm.lbm_state_bytes(0, 10, "fp32") == 0
    p = lbm.make_params({})
    assert abs(p.sigma - 1.25) < 1e-15 and abs(p.cv - 5.0) < 1e-15


def test_3d_state_bytes(built_lib):
    import paper_2205_00686_gb300 as lbm
    # 69 planes of [nz][ny][pitch] (pitch = nx rounded up to 32) and the two
    # wall ghost layers [2][ny][pitch]
    assert lbm.lbm3d_state_bytes(64, 48, 40, "fp32") == (69 * 40 + 2) * 64 * 48 * 4
    assert lbm.lbm3d_state_bytes(33, 2, 3, "fp64") == (69 * 3 + 2) * 64 * 2 * 8
    assert lbm.lbm3d_state_bytes(8, 8, 8, "fp32_g16") == 0


def test_sizes_beyond_the_plane_limit_are_refused(built_lib):
    """lbm_create refuses, before any device call, a domain whose nine f
    planes would pass 2^31 elements (the kernels' 32-bit plane offsets):
    15424^2 is the largest square accepted, 15488^2 is refused."""
    import paper_2205_00686_gb300 as lbm
    from paper_2205_00686_gb300 import workloads as W
    with pytest.raises(lbm.LbmError) as e:
        lbm.Domain(15488, 15488, W.params(), W.periodic_bc(), prec="fp32")
    assert e.value.code == lbm.LBM_EINVAL
