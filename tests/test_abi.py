"""The C ABI library builds, loads and exports every declared symbol (CPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpip.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mp_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2509_21694_gb300 import build
    return build.build()


def test_header_declares_the_four_hot_path_calls():
    names = _declared()
    for n in ("mp_build_neighbors", "mp_partition", "mp_energy_forces", "mp_md_step"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mp_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_answers_host_only_calls(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.mp_strerror.restype = ctypes.c_char_p
    assert lib.mp_strerror(-2) == b"box edge shorter than 2 r_c"
    from paper_2509_21694_gb300 import binding as mp
    import synth
    d = synth.model_alloy(n_layers_full=6)
    w = synth.make_weights(d, 1)
    vec = mp.pack_weights(w, d)       # checks the count against mp_weights_count
    assert vec.dtype.name == "float64"
    # null arguments are rejected without touching a GPU
    assert lib.mp_create(None, None, None, ctypes.c_int64(0), None) == -1


def test_binding_raises_without_library(lib_path, tmp_path, monkeypatch):
    import paper_2509_21694_gb300.binding as b
    monkeypatch.setattr(b, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        b._load()


def test_header_is_plain_c():
    """include/mpip.h is a C header (no C++ or torch types in the ABI)."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", "-x", "c",
                        os.path.join(ROOT, "include", "mpip.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_noalloc_sum_rejects_bad_arguments_before_any_gpu_work(lib_path):
    """The energy sum without allocation refuses, on the host, what would make
    its kernels read or write past a buffer: wrong dtypes, n beyond the tensor,
    no room for the result; the C entry point refuses n < 0, null pointers and
    n beyond its fixed scratch."""
    import torch
    from paper_2509_21694_gb300 import binding as mp
    e64 = torch.zeros(8, dtype=torch.float64)
    out = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError):
        mp.mp_energy_sum_noalloc(e64.float(), out)
    with pytest.raises(ValueError):
        mp.mp_energy_sum_noalloc(e64, out.float())
    with pytest.raises(ValueError):
        mp.mp_energy_sum_noalloc(e64, torch.zeros(0, dtype=torch.float64))
    with pytest.raises(ValueError):
        mp.mp_energy_sum_noalloc(e64, out, n=9)
    with pytest.raises(ValueError):
        mp.mp_energy_sum_noalloc(e64, out, n=-1)
    lib = mp._lib
    dummy = ctypes.c_void_p(256)       # never dereferenced: the checks come first
    assert lib.mp_energy_sum_noalloc(dummy, -1, dummy, None) == -1
    assert lib.mp_energy_sum_noalloc(None, 5, dummy, None) == -1
    assert lib.mp_energy_sum_noalloc(dummy, 5, None, None) == -1
    assert lib.mp_energy_sum_noalloc(dummy, mp.MP_NOALLOC_MAX_ATOMS + 1, dummy, None) == -10
