"""CPU checks of the boundary: the CUDA library loads without a GPU and
exports every entry point that ``include/cellfsi.h`` declares; the product
code and the oracle share no code."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cellfsi.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cf_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2003_03130_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for required in ("cf_create", "cf_destroy", "cf_mesh_init", "cf_set_material", "cf_lbm_init", "cf_step",
                     "cf_get_forces", "cf_get_positions", "cf_compute_forces", "cf_get_velocity", "cf_get_energy",
                     "cf_get_csr", "cf_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cf_\w+)", out))
    assert set(declared()) <= exported


def test_binding_wraps_every_entry_point():
    import paper_2003_03130_gb300 as P

    for name in declared():
        assert callable(getattr(P, name)), name


def test_no_code_shared_with_the_oracle():
    pkg = os.path.join(ROOT, "paper_2003_03130_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", src), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2003_03130_gb300" not in src and "cellfsi.h" not in src, f


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2003_03130_gb300 as P

    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        P.lib()


def _gcc(args, tmp_path):
    r = subprocess.run(["gcc", *args], capture_output=True, text=True, cwd=tmp_path)
    assert r.returncode == 0, r.stderr


def test_header_is_plain_c_and_every_symbol_links(libpath, tmp_path):
    """The header compiles as strict C99 (no C++ in it), and a C program
    that takes the address of every declared entry point links against the
    library (run without a GPU: nothing is called)."""
    names = declared()
    src = tmp_path / "all.c"
    src.write_text('#include "cellfsi.h"\ntypedef void (*fn)(void);\nfn table[] = {\n' +
                   ",\n".join(f"    (fn){n}" for n in names) +
                   "\n};\nint main(void) { return table[0] == 0; }\n")
    libdir = os.path.dirname(libpath)
    _gcc(["-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
          str(src), "-L", libdir, "-lcellfsi", "-o", str(tmp_path / "all")], tmp_path)


def test_c_driver_compiles_and_links(libpath, tmp_path):
    """tests/c_abi_shear.c (the C program of the GPU test that drives a
    coupled run through the ABI alone) builds warning-free as C99."""
    _gcc(["-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
          os.path.join(ROOT, "tests", "c_abi_shear.c"), "-L", os.path.dirname(libpath), "-lcellfsi",
          "-o", str(tmp_path / "c_abi_shear")], tmp_path)
