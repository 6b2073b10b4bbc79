"""The C-ABI library: it builds for sm_103a, loads, exports every entry
point that include/*.h declares, and rejects invalid descriptions on the
host (no CUDA call is made for those)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mmx.h")
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def declared_symbols():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mmx_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2107_06729_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["mmx_create", "mmx_set_m", "mmx_get_m", "mmx_demag", "mmx_run", "mmx_step",
              "mmx_get_stats", "mmx_save_state", "mmx_load_state", "mmx_last_error", "mmx_destroy"]:
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mmx_[a-z_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_covers_every_symbol(libpath):
    import paper_2107_06729_gb300 as pkg
    assert set(declared_symbols()) == set(pkg.SIGNATURES)
    L = pkg.lib()
    for s in declared_symbols():
        assert hasattr(L, s)
        assert hasattr(pkg, s)  # same names in the Python binding


def test_binary_is_sm_103a(libpath):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath],
                         capture_output=True, text=True).stdout
    assert "sm_103a" in out


BAD = [
    ({"n": (3, 4, 1), "d": (1e-9,) * 3}, {}, "powers of two"),
    ({"n": (1, 4, 1), "d": (1e-9,) * 3}, {}, "nx must be at least 2"),
    ({"n": (4, 4, 1), "d": (0.0, 1e-9, 1e-9)}, {}, "cell sizes"),
    ({"n": (4, 4, 1), "d": (1e-9,) * 3}, {"extrap_order": 9}, "extrap_order"),
    ({"n": (4, 4, 1), "d": (1e-9,) * 3}, {"h": -1.0}, "h must be"),
    ({"n": (4, 4, 1), "d": (1e-9,) * 3}, {"adaptive": True, "hmin": 1e-12, "hmax": 1e-13}, "hmin <= hmax"),
]


@pytest.mark.parametrize("mesh,integ,msg", BAD)
def test_invalid_descriptions_are_rejected_on_the_host(libpath, mesh, integ, msg):
    import paper_2107_06729_gb300 as pkg
    mat = {"Ms": 8e5, "A": 1.3e-11, "alpha": 0.02, "gamma": 2.211e5}
    I = dict({"method": "RK4", "h": 1e-13}, **integ)
    with pytest.raises(pkg.MMXError) as ei:
        pkg.mmx_create(*pkg.make_structs(mesh, mat, {}, I), pkg.MMX_FP64)
    assert ei.value.code == pkg.MMX_ERR_ARG
    assert msg in pkg.mmx_last_error(None)


def test_unknown_method_and_precision(libpath):
    import paper_2107_06729_gb300 as pkg
    mat = {"Ms": 8e5, "alpha": 0.02, "gamma": 2.211e5}
    M, A, F, I = pkg.make_structs({"n": (4, 4, 1), "d": (1e-9,) * 3}, mat, {}, {"method": "RK4", "h": 1e-13})
    I.method = 42
    with pytest.raises(pkg.MMXError):
        pkg.mmx_create(M, A, F, I, pkg.MMX_FP64)
    I.method = 0
    with pytest.raises(pkg.MMXError):
        pkg.mmx_create(M, A, F, I, 7)


def test_batch_arguments_are_checked_on_the_host(libpath):
    """mmx_batch_create rejects an empty batch and NULL members before any
    CUDA call; mmx_last_error(NULL) / mmx_batch_last_error(NULL) say why."""
    import ctypes
    import paper_2107_06729_gb300 as pkg
    L = pkg.lib()
    out = ctypes.c_void_p(123)
    assert L.mmx_batch_create(0, None, None, ctypes.byref(out)) == pkg.MMX_ERR_ARG
    assert out.value is None
    assert "n <= 4096" in pkg.mmx_batch_last_error(None)
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.mmx_batch_create(2, arr, None, ctypes.byref(out)) == pkg.MMX_ERR_ARG
    assert "NULL member" in pkg.mmx_last_error(None)
    assert L.mmx_batch_run(None, None, None) == pkg.MMX_ERR_ARG
    L.mmx_batch_destroy(None)


def test_residual_net_rejects_invalid_arguments_on_the_host(libpath):
    """No CUDA call is made for these."""
    import ctypes
    import paper_2107_06729_gb300 as pkg
    L = pkg.lib()
    out = ctypes.c_void_p()
    assert L.mmx_rnet_create(0, None, ctypes.byref(out)) == pkg.MMX_ERR_ARG
    assert L.mmx_rnet_create(1 << 27, None, ctypes.byref(out)) == pkg.MMX_ERR_ARG
    assert L.mmx_rnet_create(16, None, None) == pkg.MMX_ERR_ARG
    assert L.mmx_residual_sample(None, 2, None, None, None, 0.0, None, None) == pkg.MMX_ERR_ARG
    assert L.mmx_rnet_forward(None, 4, 4, 1, None, None) == pkg.MMX_ERR_ARG
    assert pkg.mmx_rnet_last_error(None) == ""
    assert L.mmx_set_residual(None, None) == pkg.MMX_ERR_ARG
