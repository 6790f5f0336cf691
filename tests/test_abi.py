"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol declared in include/*.h, and rejects bad arguments before touching
the device."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1607_08710_gb300 import build

    build.build()
    from paper_1607_08710_gb300 import lagflux

    return lagflux


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_api():
    names = declared_functions()
    for required in ("lf_init", "lf_step", "lf_run", "lf_destroy", "lf_set_state", "lf_get_state"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True, check=True)
    exported = set(re.findall(r"\sT\s+(lf_\w+)", out.stdout))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    cdll = ctypes.CDLL(lib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(cdll, n)


def test_binding_covers_every_declared_symbol(lib):
    assert sorted(lib.SIGNATURES) == [n for n in declared_functions() if n in lib.SIGNATURES]
    missing = [n for n in declared_functions() if n not in lib.SIGNATURES]
    assert not missing, missing


def test_status_strings(lib):
    assert lib.lf_status_string(0) == b"LF_OK"
    assert lib.lf_status_string(4) == b"LF_ERR_NONPHYSICAL"
    assert lib.lf_status_string(99) == b"LF_ERR_UNKNOWN"


@pytest.mark.parametrize(
    "field,value",
    [("dim", 4), ("dim", 0), ("nz", 2), ("tile_rows", -1), ("tile_rows", 4097), ("nx", 0), ("ny", 0), ("limiter", 7), ("bc", 2), ("precision", 5), ("riemann", 2), ("gamma", 1.0),
     ("gamma", 3.5), ("cfl", 0.0), ("cfl", 1.5), ("beta", 2.5), ("xmax", 0.0), ("device", -1), ("nspecies", 3),
     ("nspecies", -1), ("time_order", 4)],
)
def test_init_rejects_bad_config_without_gpu(lib, field, value):
    cfg = lib.Config(nx=16, ny=16, limiter="sweby").to_c()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = lib.lf_init(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == lib.LF_ERR_ARG
    assert h.value is None
    assert b"invalid configuration" in lib.lf_last_error(None)


@pytest.mark.parametrize("dims,precision", [((46340, 46340, 1), "fp32"), ((46340, 46340, 1), "fp64"),
                                            ((46337, 46340, 1), "fp32"), ((2048, 1024, 1025), "fp32"),
                                            ((1, 2**30, 1), "fp32")])
def test_init_rejects_meshes_past_the_32_bit_plane_without_gpu(lib, dims, precision):
    """Element offsets inside a field plane are 32-bit in the kernels and rows
    are padded to 128 bytes: a mesh whose padded plane reaches 2^31 elements
    is refused before anything touches a GPU, even when its cell count is
    below 2^31 (46340^2 cells = 2,147,395,600 < 2^31, but the padded FP32
    plane of 46368 x 46340 elements is not)."""
    nx, ny, nz = dims
    kw = dict(nx=nx, ny=ny, precision=precision)
    if nz > 1:
        kw.update(nz=nz, dim=3)
    cfg = lib.Config(**kw).to_c()
    h = ctypes.c_void_p()
    assert lib.lf_init(ctypes.byref(cfg), None, ctypes.byref(h)) == lib.LF_ERR_ARG
    assert b"2^31" in lib.lf_last_error(None)


@pytest.mark.parametrize("field,value", [("zmax", 0.0), ("nz", 0), ("nspecies", 3)])
def test_init_rejects_bad_3d_config_without_gpu(lib, field, value):
    cfg = lib.Config(nx=8, ny=8, nz=8, dim=3).to_c()
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.lf_init(ctypes.byref(cfg), None, ctypes.byref(h)) == lib.LF_ERR_ARG
    assert b"invalid configuration" in lib.lf_last_error(None)


def test_init_rejects_1d_with_ny(lib):
    cfg = lib.Config(nx=16, ny=4, dim=1).to_c()
    cfg.ny = 4
    h = ctypes.c_void_p()
    assert lib.lf_init(ctypes.byref(cfg), None, ctypes.byref(h)) == lib.LF_ERR_ARG


def test_null_arguments(lib):
    cfg = lib.Config(nx=8, ny=8).to_c()
    assert lib.lf_init(ctypes.byref(cfg), None, None) == lib.LF_ERR_ARG
    assert lib.lf_step(None, None) == lib.LF_ERR_ARG
    assert lib.lf_run(None, 0.0, 1, None, None) == lib.LF_ERR_ARG
    assert lib.lf_set_state(None, None, None, None, None, 0) == lib.LF_ERR_ARG
    assert lib.lf_set_mass_fractions(None, None, 0) == lib.LF_ERR_ARG
    assert lib.lf_get_partial_densities(None, None, 0) == lib.LF_ERR_ARG
    lib.lf_destroy(None)  # no-op


def test_species_limit_matches_header(lib):
    hdr = open(os.path.join(ROOT, "include", "lagflux.h")).read()
    assert f"#define LF_MAX_SPECIES {lib.MAX_SPECIES}" in hdr


def test_simulated_allocation_failure():
    # A fresh process so the environment hook is seen; no GPU is touched.
    code = (
        "import ctypes, sys; sys.path.insert(0, %r)\n"
        "from paper_1607_08710_gb300 import lagflux as L\n"
        "c = L.Config(nx=64, ny=64).to_c(); h = ctypes.c_void_p()\n"
        "st = L.lf_init(ctypes.byref(c), None, ctypes.byref(h))\n"
        "print(st, L.lf_last_error(None).decode())\n" % ROOT
    )
    env = dict(os.environ, LF_TEST_FAIL_ALLOC="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    st, msg = r.stdout.split(" ", 1)
    assert int(st) == 3  # LF_ERR_OOM
    assert "simulated" in msg


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1607_08710_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), f
                assert "lagflux_oracle" not in text and "liblagflux_oracle" not in text, f


def test_batch_init_rejects_problems_past_the_32_bit_plane_without_gpu(lib):
    cfgs = (lib.lf_config * 2)(lib.Config(nx=64, ny=64, precision="fp32").to_c(),
                               lib.Config(nx=1, ny=2**26 + 1, precision="fp32").to_c())
    h = ctypes.c_void_p()
    assert lib.lf_batch_init(cfgs, 2, None, ctypes.byref(h)) == lib.LF_ERR_ARG
    assert h.value is None
