"""CPU checks of the C ABI: the library builds, loads without a GPU and exports every symbol the
header declares; the header is strict C and a C program links against the library; host-side
argument checks that need no device."""
import ctypes
import os
import re

import pytest

from paper_1810_07772_gb300 import build as gbuild
from paper_1810_07772_gb300 import gw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    gbuild.build()
    return gw.lib()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "gw.h")).read()
    return sorted(set(re.findall(r"^GW_API[^;(]*?\b(gw_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_path_calls():
    names = declared_symbols()
    for call in ("gw_load_states", "gw_build_P", "gw_P_to_G", "gw_eps_inv", "gw_create", "gw_destroy"):
        assert call in names
    assert len(names) == 57


def test_every_declared_symbol_is_exported(L):
    for name in declared_symbols():
        assert hasattr(L, name), name
        assert name in gw.SIGNATURES, f"binding has no signature for {name}"
    assert set(gw.SIGNATURES) == set(declared_symbols())


def test_status_strings(L):
    assert L.gw_version() == 1
    assert L.gw_status_str(0) == b"ok"
    assert L.gw_status_str(5) == b"eps not positive definite"
    assert L.gw_status_str(99) == b"unknown status"


def test_null_handles_are_rejected(L):
    assert L.gw_destroy(None) == gw.GW_E_INVALID
    assert L.gw_build_P(None, 0, None) == gw.GW_E_INVALID
    assert L.gw_sync(None) == gw.GW_E_INVALID
    assert L.gw_create(None, 0, None) == gw.GW_E_INVALID


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = L.gw_create(ctypes.byref(h), 0, None)
    assert st in (gw.GW_E_INVALID, gw.GW_E_CUDA)
    assert not h.value


def test_only_sm103a_code():
    """The build targets sm_103a only (no PTX for other archs, no multi-arch fat binary)."""
    assert gbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_rejects_undersized_buffers(L):
    """The binding checks the size of every tensor or array it passes where the call's size is
    known; raw addresses and NULL pass unchecked."""
    import types

    import numpy as np
    import torch

    from oracle import gw_oracle as O
    gw._fits(np.zeros(4, np.complex64), 32, "x")
    gw._fits(None, 1 << 40, "x")
    gw._fits(12345, 1 << 40, "x")
    gw._fits(torch.zeros(4, dtype=torch.complex128), 64, "t")
    for buf, need in ((np.zeros(3, np.complex64), 32), (torch.zeros(4, dtype=torch.complex128), 65)):
        with pytest.raises(gw.GwError) as e:
            gw._fits(buf, need, "x")
        assert e.value.status == gw.GW_E_INVALID
    # the sphere size the P~ check uses: the documented N_g of the three workloads and the oracle's
    # sphere on a non-cubic grid
    for dims, gcut, ng in (((12, 12, 12), 8, 93), ((24, 24, 24), 29, 691), ((36, 36, 36), 61, 2007)):
        assert gw.Context._sphere_size(types.SimpleNamespace(dims=dims), gcut) == ng
    dims = (10, 14, 9)
    assert gw.Context._sphere_size(types.SimpleNamespace(dims=dims), 5) == len(O.sphere(dims, 5))


def test_header_is_c_and_links_from_c(L):
    """include/gw.h compiles as strict C99 (and as C++17), and a C program linked against libgw.so
    reaches the entry points that need no GPU with the documented results."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    src = os.path.join(ROOT, "tests", "abi_check.c")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    for std in ("-std=c99", "-std=c11"):
        subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc, "-fsyntax-only", src],
                       check=True, timeout=120)
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx:
        subprocess.run([cxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I", inc, "-fsyntax-only", "-x", "c++",
                        src], check=True, timeout=120)
    lib_dir = os.path.dirname(gbuild.LIB_PATH)
    exe = os.path.join(out_dir, "abi_check")
    subprocess.run([cc, "-std=c99", "-I", inc, src, "-o", exe, "-L", lib_dir, "-lgw", f"-Wl,-rpath,{lib_dir}"],
                   check=True, timeout=120)
    res = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=60)
    got = dict(line.split(" ", 1) for line in res.stdout.strip().splitlines())
    assert got["version"] == "1" and got["status0"] == "ok" and got["status5"] == "eps not positive definite"
    for k in ("null_destroy", "null_create", "null_eps_inv"):
        assert int(got[k]) == gw.GW_E_INVALID


def _header_decls():
    text = open(os.path.join(ROOT, "include", "gw.h")).read()
    out = {}
    for ret, name, params in re.findall(r"^GW_API\s+([^;(]*?)\b(gw_\w+)\s*\(([^)]*)\)\s*;", text, flags=re.M | re.S):
        ps = [" ".join(p.split()) for p in params.replace("\n", " ").split(",")]
        ps = [] if ps in ([""], ["void"]) else ps
        # drop the parameter name: the type is what precedes it (a pointer keeps its stars)
        types = [" ".join(re.sub(r"\b\w+$", "", p).split()) for p in ps]
        out[name] = (" ".join(ret.split()), types)
    return text, out


def test_binding_signatures_and_constants_match_the_header():
    """Every ctypes signature of the binding has the header's arity and, argument by argument, a
    ctypes type of the same kind and size (a pointer for a pointer, c_int for int and the enums,
    c_double for double, c_size_t for size_t, c_long for long; POINTER(T) only onto the header's
    pointee type), and every enumerator the binding uses has the header's value."""
    text, decls = _header_decls()
    assert set(decls) == set(gw.SIGNATURES)
    scalar = {"int": ctypes.c_int, "double": ctypes.c_double, "size_t": ctypes.c_size_t, "long": ctypes.c_long,
              "gw_status": ctypes.c_int}
    pointee = {"double": ctypes.c_double, "float": ctypes.c_float, "int": ctypes.c_int, "size_t": ctypes.c_size_t,
               "void *": ctypes.c_void_p}
    for name, (ret, types) in decls.items():
        res, args = gw.SIGNATURES[name]
        assert len(args) == len(types), name
        if ret.endswith("*"):
            assert res is ctypes.c_char_p, name
        else:
            assert res is ctypes.c_int, name
        for t, a in zip(types, args):
            if t.endswith("*"):
                base = " ".join(t.replace("const", " ").split())[:-1].strip()   # the pointee
                if base == "char":
                    assert a is ctypes.c_char_p, (name, t)
                elif hasattr(a, "_type_") and a not in (ctypes.c_void_p, ctypes.c_char_p):
                    want = pointee.get(base, ctypes.c_void_p if base.endswith("*") else None)
                    assert want is not None and a._type_ is want, (name, t, a)
                else:
                    assert a is ctypes.c_void_p, (name, t, a)
            else:
                assert ctypes.sizeof(a) == ctypes.sizeof(scalar[t]) and a is scalar[t], (name, t, a)
    enums = {k: int(v) for k, v in re.findall(r"\b(GW_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    for k in ("GW_OK", "GW_E_INVALID", "GW_E_NOMEM", "GW_E_CUDA", "GW_E_NOT_READY", "GW_E_NUMERIC",
              "GW_E_TIMEOUT", "GW_E_UNSUPPORTED", "GW_C64", "GW_C128"):
        assert getattr(gw, k) == enums[k], k
    for table, prefix in ((gw.PRECISION, "GW_PREC_"), (gw.INV_METHOD, "GW_INV_"), (gw.HERK_KERNEL, "GW_HERK_"),
                          (gw.TRANSFORM_KERNEL, "GW_TRANSFORM_"), (gw.BUF, "GW_BUF_")):
        for key, value in table.items():
            assert enums[prefix + key.upper()] == value, (prefix, key)
